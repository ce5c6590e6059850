// cox_ballot_compact: stable stream compaction from warp ballots.
//
// One CTA per tile of 16384 keys (64 KB), taken from an atomic ticket in the
// order CTAs start; the CTA's 256 threads cover the tile in 4 passes of 16
// keys each (the result does not depend on the caller's block size, so
// every launch takes the shape that keeps three tiles in flight per SM --
// 1024-thread CTAs fit two per SM and ran ~2x slower).  The tile arrives in shared memory by one
// TMA bulk copy (plain loads for a ragged or unaligned tile), so keys never
// occupy registers and three 64 KB tiles fit in flight per SM -- a tile's
// chain of round trips (ticket, copy, look-back) is what bounds this op, and
// only bytes in flight hide it.  In the tile:
//   count   per pass, 16 keys per thread, each warp on its own run of 512
//           keys: lanes count kept keys (key < t), redux.sync sums the
//           warp's count (32 counts per tile whatever B);
//   scan    warp 0 scans the counts in (pass, warp) order and publishes the
//           tile's count for the look-back;
//   compact the same passes again: per chunk of the run, b = __ballot_sync
//           (keep) for each of a lane's four key slots, rank = offset +
//           earlier chunks + popc(b & lanemask_lt) + kept keys before it in
//           the lane; kept keys move in place to their rank (a key's rank
//           never exceeds its own index, and pass j only writes below
//           16B(j+1), where pass j+1 reads, so one barrier per pass between
//           its reads and writes suffices);
//   prefix  warp 0's decoupled look-back (compact_tile.cuh);
//   out     coalesced copy of the compacted keys to out[prefix ..].
// Each CTA's ticket is taken as it starts and its tile finished before it
// exits, so every look-back wait ends; each is bounded all the same.
#include <mutex>

#include "compact_tile.cuh"

namespace cox {

constexpr int kCompactThreads = 256;

template <bool SIGNED>
__global__ void __launch_bounds__(kCompactThreads, 3) k_ballot_compact(const uint32_t* __restrict__ keys, int64_t n,
                                                         int64_t thr, uint32_t* __restrict__ out,
                                                         int64_t* __restrict__ d_count, unsigned* ticket,
                                                         uint64_t* desc, int64_t ntiles, uint32_t limit,
                                                         unsigned* status, int vec) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int B = blockDim.x, nw = B >> 5;
  const int64_t TILE = kBigTile;
  const int passes = (int)(TILE / (16 * B));
  const int m = passes * nw;                              // warp-run counts per tile: TILE / 512
  uint32_t* buf = smem;                                   // TILE keys, compacted in place
  uint32_t* wcnt = smem + TILE;                           // m counts, then offsets
  uint64_t* bar = reinterpret_cast<uint64_t*>(wcnt + m);
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= ntiles) return;
  const int64_t base = tile * TILE;
  const int64_t valid = min(TILE, n - base);
  // ---- the tile into shared memory
  const bool bulk = vec && valid == TILE;  // 16-byte aligned start, whole tile, size a multiple of 16
  if (bulk) {
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, (uint32_t)(TILE * 4));
      tma_load_1d(buf, keys + base, (uint32_t)(TILE * 4), bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0u, limit);
    if (__syncthreads_or(!ok)) {  // the copy did not land in time: record it, wait once more, stop
      if (tid == 0) {
        atomicOr(status, (unsigned)kDevTimeout);
        mbar_wait_bounded(bar, 0u, limit);
        st_relaxed_u64(desc + tile, kFlagP);  // successors end with a zero prefix
      }
      return;
    }
  } else {
    for (int64_t i = tid; i < valid; i += B) buf[i] = keys[base + i];
    __syncthreads();
  }
  compact_big_tile<SIGNED>(buf, (int)valid, thr, out, d_count, desc, tile, ntiles, n, limit, status, wcnt);
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_ballot_compact_workspace(int64_t n, int block_dim) {
  if (n < 0 || !valid_block(block_dim)) return 0;
  const int64_t tile = kBigTile;
  return compact_ws_bytes((n + tile - 1) / tile);
}

extern "C" cox_status cox_ballot_compact(cox_dtype dt, int width, int block_dim, const void* d_keys, int64_t n,
                                         int64_t threshold, void* d_out, int64_t* d_count, void* d_workspace,
                                         size_t workspace_bytes, unsigned flags, void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32) return COX_EINVAL;
  if (flags & ~(unsigned)COX_F_WS_READY) return COX_EINVAL;
  if (!d_count || (n > 0 && (!d_keys || !d_out))) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  if (n == 0) {
    return cudaMemsetAsync(d_count, 0, sizeof(int64_t), st) == cudaSuccess ? COX_OK : COX_ECUDA;
  }
  const size_t need = cox_ballot_compact_workspace(n, block_dim);
  if (!d_workspace || workspace_bytes < need) return COX_ENOMEM;
  if (!aligned16(d_workspace)) return COX_EINVAL;
  if (!(flags & COX_F_WS_READY) && cudaMemsetAsync(d_workspace, 0, need, st) != cudaSuccess) return COX_ECUDA;
  const int64_t tile = kBigTile;
  const int64_t ntiles = (n + tile - 1) / tile;
  if (ntiles > 0xFFFFFFFFll) return COX_EUNSUPPORTED;  // 32-bit ticket
  const size_t smem = ((size_t)tile + (size_t)(tile / 128)) * sizeof(uint32_t) + sizeof(uint64_t);
  unsigned* ticket = static_cast<unsigned*>(d_workspace);
  uint64_t* desc = reinterpret_cast<uint64_t*>(static_cast<char*>(d_workspace) + kCompactWsHeader);
  const int vec = aligned16(d_keys);
  auto launch = [&](auto kern) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return COX_ECUDA;
    kern<<<(unsigned)ntiles, kCompactThreads, smem, st>>>(static_cast<const uint32_t*>(d_keys), n, threshold,
                                                  static_cast<uint32_t*>(d_out), d_count, ticket, desc, ntiles,
                                                  spin_limit(), device_status_word(), vec);
    return launch_status();
  };
  return dt == COX_I32 ? launch(k_ballot_compact<true>) : launch(k_ballot_compact<false>);
}

// ---------------------------------------------------------------------------
// cox_ballot_compact_static: the same compaction for callers that cannot
// allocate device memory.  Its scratch (the ticket and the per-tile
// look-back descriptors) lives in the fixed array below instead of a
// caller-provided workspace.
//
// The array belongs to the library image: every GPU that loads libcox.so
// holds these bytes until the process exits.  In host code the name
// g_compact_scratch is only a host-side stand-in for the symbol, not a
// device address, so it is never passed to a kernel; the device address is
// looked up with cudaGetSymbolAddress once per device (on that device's first
// call of this entry point, with the device current) and cached.
namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;  // COX_COMPACT_STATIC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_compact_scratch[kStaticScratchBytes];

constexpr int kStaticMaxDevices = 64;
void* g_scratch_addr[kStaticMaxDevices];
std::mutex g_scratch_mu;

cox_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return COX_ECUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return COX_EUNSUPPORTED;
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_compact_scratch) != cudaSuccess || !p) return COX_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return COX_OK;
}

}  // namespace

extern "C" cox_status cox_ballot_compact_static(cox_dtype dt, int width, int block_dim, const void* d_keys,
                                                int64_t n, int64_t threshold, void* d_out, int64_t* d_count,
                                                void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32) return COX_EINVAL;
  if (!d_count || (n > 0 && (!d_keys || !d_out))) return COX_EINVAL;
  // Larger inputs need more tile descriptors than the fixed scratch holds.
  if (cox_ballot_compact_workspace(n, block_dim) > kStaticScratchBytes) return COX_ENOMEM;
  void* scratch = nullptr;
  const cox_status s = static_scratch(&scratch);
  if (s != COX_OK) return s;
  // The call zeroes the bytes it uses (ticket and descriptors), because the
  // array still holds whatever the previous call left there.
  return cox_ballot_compact(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, scratch,
                            kStaticScratchBytes, 0u, stream);
}
