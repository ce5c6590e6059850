// cox_ballot_compact: stable stream compaction from warp ballots.
//
// A cooperative launch of 256-thread CTAs (three per SM, whatever the
// caller's block size: the result does not depend on it); CTA c takes tiles
// c, c + G, ... of 8192 keys (32 KB).  Each CTA keeps two tiles in shared
// memory: one is worked on while the next arrives by a TMA bulk copy (plain
// loads for a ragged or unaligned tile), so the copies stay in flight while
// tiles wait on their look-backs.  In a tile (compact_tile.cuh):
//   compact every warp compacts its 1024 keys in place in one pass: per
//           chunk of 128 keys, b = __ballot_sync(keep) for each of a lane's
//           four key slots, rank = kept keys before the chunk +
//           popc(b & lanemask_lt) over the slots + kept keys before it in
//           the lane;
//   scan    warp 0 scans the 8 warp counts and publishes the tile's count
//           for the look-back;
//   prefix  warp 0's decoupled look-back;
//   out     every warp copies its kept keys to out[prefix + offset ..].
#include <mutex>

#include "compact_tile.cuh"

namespace cox {

constexpr int kCompactThreads = 256;
constexpr int kCompactNW = kCompactThreads / 32;
constexpr int kCompactReg = 1024;                            // keys per warp
constexpr int64_t kCompactTile = kCompactNW * kCompactReg;  // 8192 keys
constexpr int kCompactBufs = 2;                              // tiles in shared memory per CTA

// A cooperative launch (all CTAs co-resident) of G CTAs, three per SM; CTA c
// takes tiles c, c + G, c + 2G, ... in turn, with the next tile's TMA bulk
// copy in flight while it works on the current one.  Per tile: every warp
// compacts its 1024 keys in place, warp 0 scans the warp counts, publishes
// the tile's count and looks back for its prefix, every warp copies its kept
// keys to out[prefix + the warps before it ..], and the freed buffer starts
// loading the tile after next.  A CTA works on its tiles in increasing order
// and all CTAs run at once, so the lowest unfinished tile always has every
// predecessor finished: every look-back wait ends (each is bounded all the
// same).
template <bool SIGNED>
__global__ void __launch_bounds__(kCompactThreads, 3) k_ballot_compact(const uint32_t* __restrict__ keys, int64_t n,
                                                         int64_t thr, uint32_t* __restrict__ out,
                                                         int64_t* __restrict__ d_count, uint64_t* desc,
                                                         int64_t ntiles, uint32_t limit, unsigned* status, int vec) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int64_t TILE = kCompactTile;
  uint32_t* wcnt = smem + kCompactBufs * TILE;  // warp counts, then offsets
  uint64_t* bar = reinterpret_cast<uint64_t*>(wcnt + kCompactWsWords);
  __shared__ int64_t s_prefix;
  __shared__ uint32_t s_total;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int region = warp * kCompactReg;
  const unsigned lt = lanemask_lt();
  const LeRule rule = le_rule<SIGNED>(thr);
  const int64_t G = gridDim.x;
  // tile k of this CTA: blockIdx.x + k G, in buffer k % kCompactBufs
  auto bulk = [&](int64_t tile) { return vec && (tile + 1) * TILE <= n; };
  auto issue = [&](int64_t k) {  // thread 0: start loading this CTA's tile k
    const int64_t tile = blockIdx.x + k * G;
    if (tile < ntiles && bulk(tile)) {
      uint64_t* b = bar + (k % kCompactBufs);
      mbar_arrive_expect_tx(b, (uint32_t)(TILE * 4));
      tma_load_1d(smem + (k % kCompactBufs) * TILE, keys + tile * TILE, (uint32_t)(TILE * 4), b);
    }
  };
  if (tid == 0) {
    for (int b = 0; b < kCompactBufs; ++b) mbar_init(bar + b, 1);
    mbar_init_fence();
    for (int k = 0; k < kCompactBufs; ++k) issue(k);
  }
  __syncthreads();
  for (int64_t k = 0;; ++k) {
    const int64_t tile = blockIdx.x + k * G;
    if (tile >= ntiles) break;
    uint32_t* buf = smem + (k % kCompactBufs) * TILE;
    const int64_t base = tile * TILE;
    const int valid = (int)min(TILE, n - base);
    // ---- the tile in shared memory
    if (bulk(tile)) {
      const uint32_t parity = (uint32_t)((k / kCompactBufs) & 1);
      const bool ok = mbar_wait_bounded(bar + (k % kCompactBufs), parity, limit);
      if (__syncthreads_or(!ok)) {  // a copy did not land in time: record it, let the copies in flight land, stop
        if (tid == 0) {
          atomicOr(status, (unsigned)kDevTimeout);
          for (int64_t j = k; j < k + kCompactBufs; ++j)
            if (blockIdx.x + j * G < ntiles && bulk(blockIdx.x + j * G))
              mbar_wait_bounded(bar + (j % kCompactBufs), (uint32_t)((j / kCompactBufs) & 1), limit);
          for (int64_t t = tile; t < ntiles; t += G) desc_raise(desc + t, kFlagP);  // successors end
        }
        break;
      }
    } else {
      for (int i = tid; i < valid; i += kCompactThreads) buf[i] = keys[base + i];
      __syncthreads();
    }
    // ---- every warp compacts its region in place
    const uint32_t kept = compact_region<SIGNED, kCompactReg>(buf, region, lane, lt, valid, valid == (int)TILE, rule);
    if (lane == 0) wcnt[warp] = kept;
    __syncthreads();
    // ---- count, look-back, offsets
    if (warp == 0) {
      const uint32_t wc = lane < kCompactNW ? wcnt[lane] : 0u;
      uint32_t incl = wc;
#pragma unroll
      for (int d = 1; d < kCompactNW; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += u;
      }
      const uint32_t total = __shfl_sync(kFull, incl, kCompactNW - 1);
      if (lane < kCompactNW) wcnt[32 + lane] = incl - wc;  // exclusive offsets
      if (lane == 0) publish_count(desc, tile, ntiles, total);
      bool gave_up;
      const int64_t prefix = look_back(desc, tile, ntiles, total, limit, status, gave_up);
      if (lane == 0) {
        s_prefix = prefix;
        s_total = total;
        s_bad = gave_up;
      }
    }
    __syncthreads();
    // ---- copy-out
    const int64_t prefix = s_prefix;
    if (!s_bad && prefix + (int64_t)s_total <= n) {
      uint32_t* dst = out + prefix + wcnt[32 + warp];
      const uint32_t* src = buf + region;
#pragma unroll 4
      for (int i = lane; i < (int)kept; i += 32) dst[i] = src[i];
      if (tile == ntiles - 1 && tid == 0) *d_count = prefix + s_total;
    }
    fence_proxy_async_smem();  // this thread's accesses to the buffer, before the bulk copy that refills it
    __syncthreads();
    if (tid == 0) issue(k + kCompactBufs);
  }
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_ballot_compact_workspace(int64_t n, int block_dim) {
  if (n < 0 || !valid_block(block_dim)) return 0;
  const int64_t tile = kCompactTile;
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
  const int64_t tile = kCompactTile;
  const int64_t ntiles = (n + tile - 1) / tile;
  const size_t smem = ((size_t)kCompactBufs * tile + kCompactWsWords) * sizeof(uint32_t) + kCompactBufs * sizeof(uint64_t);
  uint64_t* desc = reinterpret_cast<uint64_t*>(static_cast<char*>(d_workspace) + kCompactWsHeader);
  const int vec = aligned16(d_keys);
  auto launch = [&](auto kern, int* grid) {
    int& g = grid[device_index()];
    if (g == 0) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COX_ECUDA;
      g = persistent_grid(kern, kCompactThreads, smem, 1 << 30);
    }
    const int64_t ctas = ntiles < g ? ntiles : g;
    const uint32_t* keys = static_cast<const uint32_t*>(d_keys);
    uint32_t* outp = static_cast<uint32_t*>(d_out);
    uint32_t limit = spin_limit();
    unsigned* status = device_status_word();
    void* args[] = {(void*)&keys, (void*)&n, (void*)&threshold, (void*)&outp, (void*)&d_count, (void*)&desc,
                    (void*)&ntiles, (void*)&limit, (void*)&status, (void*)&vec};
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)ctas), dim3(kCompactThreads), args, smem, st) !=
        cudaSuccess) {
      cudaGetLastError();
      return COX_ECUDA;
    }
    return COX_OK;
  };
  static int grid_s[kMaxDevices], grid_u[kMaxDevices];  // co-resident grids, per device
  return dt == COX_I32 ? launch(k_ballot_compact<true>, grid_s) : launch(k_ballot_compact<false>, grid_u);
}

// ---------------------------------------------------------------------------
// cox_ballot_compact_static: the same compaction for callers that cannot
// allocate device memory.  Its scratch (the per-tile and per-group
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
  // The call zeroes the bytes it uses (the descriptors), because the array
  // still holds whatever the previous call left there.
  return cox_ballot_compact(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, scratch,
                            kStaticScratchBytes, 0u, stream);
}
