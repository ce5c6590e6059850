// cox_ballot_compact: stable stream compaction from warp ballots.
//
// The filter of the SDK kernel filter_arr (Table 1 of the paper) with a
// static, full-warp group instead of the dynamically coalesced one (the paper
// covers non-divergent warp functions only, Section 2.2.3):
//   b = __ballot_sync(full, key < t); rank = popc(b & lanemask_lt);
// a shared-memory scan orders the warps of a tile, and tiles are ordered by
// a single-pass decoupled look-back over per-tile descriptors.  Tiles are
// handed out by an atomic ticket, so a tile only ever waits on tiles whose
// CTAs already run: the waits end.  Each wait is still bounded.
//
// Tile layout: a CTA of B threads owns B*16 consecutive keys, read as four
// 128-bit loads per thread; chunk j (4B keys) has thread t holding keys
// j*4B + 4t .. 4t+3.  The rank of key (j, t, k) in the tile is
//   offset(j, warp) + sum_k' popc(ballot_k'(j) & lanemask_lt) + #{k' < k kept}
// which is its position in input order, so the result is the stable filter.
#include <mutex>

#include "cox_common.cuh"

namespace cox {

constexpr int kCompactEpt = 16;
constexpr size_t kCompactWsHeader = 256;
constexpr uint64_t kFlagA = 1ull << 62;  // descriptor holds the tile's own count
constexpr uint64_t kFlagP = 2ull << 62;  // descriptor holds the inclusive prefix
constexpr uint64_t kValMask = (1ull << 62) - 1;

// Look-back by one warp: publish the tile's count, then walk predecessors 32
// at a time until a published inclusive prefix is found.  Returns the
// exclusive prefix of the tile (valid in every lane).
__device__ __forceinline__ int64_t look_back(uint64_t* desc, int64_t tile, uint32_t total, uint32_t limit,
                                             unsigned* status, bool& gave_up) {
  const int lane = lane_id();
  gave_up = false;
  if (tile == 0) {
    if (lane == 0) st_relaxed_u64(desc, kFlagP | total);
    return 0;
  }
  if (lane == 0) st_relaxed_u64(desc + tile, kFlagA | total);
  int64_t prefix = 0;
  bool timed_out = false;
  for (int64_t i = tile - 1 - lane;; i -= 32) {
    uint64_t d = kFlagP;  // index < 0: the virtual predecessor of tile 0, prefix 0
    if (i >= 0) {
      d = ld_relaxed_u64(desc + i);
      uint32_t polls = 0;
      while ((d >> 62) == 0) {
        if (++polls > limit) {
          timed_out = true;
          d = kFlagP;
          break;
        }
        __nanosleep(200);
        d = ld_relaxed_u64(desc + i);
      }
    }
    const unsigned pmask = __ballot_sync(kFull, (d >> 62) == 2);
    const int first = pmask ? __ffs(pmask) - 1 : 31;
    unsigned long long v = lane <= first ? (d & kValMask) : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    prefix += (int64_t)v;
    if (pmask) break;
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    prefix = 0;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(desc + tile, kFlagP);  // release successors with a zero prefix
    }
    return 0;
  }
  if (lane == 0) st_relaxed_u64(desc + tile, kFlagP | ((uint64_t)(prefix + total) & kValMask));
  return prefix;
}

template <bool SIGNED>
__global__ void __launch_bounds__(1024) k_ballot_compact(const uint32_t* __restrict__ keys, int64_t n,
                                                         int64_t thr, uint32_t* __restrict__ out,
                                                         int64_t* __restrict__ d_count, unsigned* ticket,
                                                         uint64_t* desc, int64_t ntiles, uint32_t limit,
                                                         unsigned* status, int vec) {
  extern __shared__ uint32_t smem[];
  const int B = blockDim.x;
  const int nw = B >> 5;
  const int64_t TILE = (int64_t)B * kCompactEpt;
  uint32_t* stage = smem;               // TILE words: the tile's kept keys, compacted
  uint32_t* wcnt = smem + TILE;         // 4 * nw warp counts, then their offsets
  __shared__ int64_t s_tile, s_prefix;
  __shared__ uint32_t s_total;
  __shared__ int s_gave_up;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= ntiles) return;
  const int64_t base = tile * TILE;

  uint32_t key[4][4];
  bool keep[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t e0 = base + (int64_t)j * 4 * B + 4 * tid;
    if (vec && e0 + 4 <= n) {
      const uint4 q = __ldcs(reinterpret_cast<const uint4*>(keys + e0));
      key[j][0] = q.x; key[j][1] = q.y; key[j][2] = q.z; key[j][3] = q.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) keep[j][k] = true;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        keep[j][k] = e0 + k < n;
        key[j][k] = keep[j][k] ? keys[e0 + k] : 0u;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool p = SIGNED ? (int64_t)(int32_t)key[j][k] < thr : (int64_t)key[j][k] < thr;
      keep[j][k] = keep[j][k] && p;
    }
  }
  uint32_t lane_pre[4];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t cnt = 0, pre = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned b = __ballot_sync(kFull, keep[j][k]);
      cnt += __popc(b);
      pre += __popc(b & lt);
    }
    lane_pre[j] = pre;
    if (lane == 0) wcnt[j * nw + warp] = cnt;
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the 4*nw warp counts in (chunk, warp) order
    const int m = 4 * nw;
    uint32_t c[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = lane * 4 + q;
      c[q] = idx < m ? wcnt[idx] : 0u;
      sum += c[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += u;
    }
    uint32_t ex = incl - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = lane * 4 + q;
      if (idx < m) wcnt[idx] = ex;
      ex += c[q];
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    bool gave_up;
    const int64_t prefix = look_back(desc, tile, total, limit, status, gave_up);
    if (lane == 0) {
      s_total = total;
      s_prefix = prefix;
      s_gave_up = gave_up;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t o = wcnt[j * nw + warp] + lane_pre[j];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (keep[j][k]) stage[o++] = key[j][k];
  }
  __syncthreads();
  const int64_t prefix = s_prefix;
  const uint32_t total = s_total;
  if (s_gave_up || prefix + (int64_t)total > n) return;
  for (int i = tid; i < (int)total; i += B) out[prefix + i] = stage[i];
  if (tile == ntiles - 1 && tid == 0) *d_count = prefix + total;
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_ballot_compact_workspace(int64_t n, int block_dim) {
  if (n < 0 || !valid_block(block_dim)) return 0;
  const int64_t tile = (int64_t)block_dim * kCompactEpt;
  const int64_t ntiles = (n + tile - 1) / tile;
  return kCompactWsHeader + (size_t)ntiles * sizeof(uint64_t);
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
  const int64_t tile = (int64_t)block_dim * kCompactEpt;
  const int64_t ntiles = (n + tile - 1) / tile;
  if (ntiles > 0xFFFFFFFFll) return COX_EUNSUPPORTED;
  const size_t smem = ((size_t)tile + 4 * (block_dim / 32)) * sizeof(uint32_t);
  unsigned* ticket = static_cast<unsigned*>(d_workspace);
  uint64_t* desc = reinterpret_cast<uint64_t*>(static_cast<char*>(d_workspace) + kCompactWsHeader);
  const int vec = aligned16(d_keys);
  auto launch = [&](auto kern) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return COX_ECUDA;
    kern<<<(unsigned)ntiles, block_dim, smem, st>>>(static_cast<const uint32_t*>(d_keys), n, threshold,
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
  // Larger inputs need more descriptors than the fixed scratch holds.
  if (cox_ballot_compact_workspace(n, block_dim) > kStaticScratchBytes) return COX_ENOMEM;
  void* scratch = nullptr;
  const cox_status s = static_scratch(&scratch);
  if (s != COX_OK) return s;
  // The call zeroes the bytes it uses (ticket and descriptors), because the
  // array still holds whatever the previous call left there.
  return cox_ballot_compact(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, scratch,
                            kStaticScratchBytes, 0u, stream);
}
