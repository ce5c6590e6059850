// cox_coalesced and cox_filter_aggregated: warp functions over dynamic
// (coalesced) groups -- the runtime member masks and "all active threads"
// groups that COX leaves unsupported (Sections 2.2.2-2.2.3), and the SDK's
// filter_arr that needs them ("activated thread sync", Table 1).
//
// A warp's group is formed by a full-warp ballot of the activity flags; the
// active lanes then run the warp intrinsics with that member mask
// (shfl.sync / vote.sync / redux.sync with a partial mask), exactly as a
// coalesced_group does.  Group ranks are popc(mask & lanemask_lt); the lane
// of rank k is found by a 5-step binary search over popc prefixes.  The
// integer group scan alone runs over the full warp with inactive lanes
// contributing 0 (the same sums, exactly).
#include "cox_common.cuh"
#include "compact_tile.cuh"

namespace cox {

// Lane of the k-th (0-based) set bit of mask; k < popc(mask).
__device__ __forceinline__ int nth_set_lane(unsigned mask, int k) {
  int pos = 0;
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const int below = __popc(mask & ((1u << (pos + b)) - 1u));  // set bits below pos + b
    if (below <= k) pos += b;
  }
  return pos;
}

template <int DT>
__device__ __forceinline__ bool vote_pred(uint32_t u) {
  if constexpr (DT == COX_F32) return __uint_as_float(u) != 0.0f;
  else return u != 0u;
}

// One group's function for one active lane (the lane's value v, the
// group's mask, rank and size).  SCAN_SUM is handled by the caller.
template <int DT>
__device__ __forceinline__ uint32_t group_fn(int fn, uint32_t v, unsigned mask, int rank, int size, int lane,
                                             int param) {
  switch (fn) {
    case COX_CG_SIZE: return (uint32_t)size;
    case COX_CG_RANK: return (uint32_t)rank;
    case COX_CG_SHFL: return __shfl_sync(mask, v, nth_set_lane(mask, param % size));
    case COX_CG_SHFL_UP: return __shfl_sync(mask, v, rank >= param ? nth_set_lane(mask, rank - param) : lane);
    case COX_CG_SHFL_DOWN:
      return __shfl_sync(mask, v, rank + param < size ? nth_set_lane(mask, rank + param) : lane);
    case COX_CG_BALLOT: {
      const unsigned b = __ballot_sync(mask, vote_pred<DT>(v));
      uint32_t r = 0;
      unsigned m = mask;
      for (int k = 0; m; ++k, m &= m - 1u)  // bit k = the k-th member's vote
        if (b & (m & (0u - m))) r |= 1u << k;
      return r;
    }
    case COX_CG_ANY: return __any_sync(mask, vote_pred<DT>(v)) ? 1u : 0u;
    case COX_CG_ALL: return __all_sync(mask, vote_pred<DT>(v)) ? 1u : 0u;
    default: return __reduce_add_sync(mask, v);  // COX_CG_REDUCE_SUM
  }
}

// Persistent warps take 4 consecutive 32-element groups at a time, their
// loads issued together.  SCAN_SUM (integers, exact) runs as a full-warp
// Hillis-Steele scan in which inactive lanes contribute 0: an active lane's
// inclusive prefix over the lanes up to it is its group's prefix by rank.
constexpr int kCgUnroll = 4;

template <int DT>
__global__ void __launch_bounds__(256) k_coalesced(int fn, const uint32_t* __restrict__ in,
                                                   const int32_t* __restrict__ active, uint32_t* __restrict__ out,
                                                   int64_t n, int param) {
  const int lane = lane_id();
  const unsigned lt = lanemask_lt();
  const int64_t nw = (n + 32 * kCgUnroll - 1) / (32 * kCgUnroll);
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += wstep) {
    bool act[kCgUnroll];
    uint32_t v[kCgUnroll];
#pragma unroll
    for (int u = 0; u < kCgUnroll; ++u) {
      const int64_t i = (w * kCgUnroll + u) * 32 + lane;
      act[u] = i < n && __ldcs(active + i) != 0;
      v[u] = i < n ? __ldcs(in + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kCgUnroll; ++u) {
      const int64_t i = (w * kCgUnroll + u) * 32 + lane;
      const unsigned mask = __ballot_sync(kFull, act[u]);  // coalesced_threads()
      if (fn == COX_CG_SCAN_SUM) {
        uint32_t x = act[u] ? v[u] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, x, d);
          if (lane >= d) x += y;
        }
        if (act[u]) out[i] = x;
        continue;
      }
      if (!act[u]) continue;
      out[i] = group_fn<DT>(fn, v[u], mask, __popc(mask & lt), __popc(mask), lane, param);
    }
  }
}

// filter_arr with warp-aggregated slots.  A warp takes 16 rounds of 32 keys
// (round j: keys base + 32j + lane); round j's group is its keeping lanes.
// One atomic per warp reserves the 16 groups' total; group j's range starts
// after groups 0 .. j-1, and a lane's slot is base + that offset + its rank.
constexpr int kFilterRounds = 16;

template <bool SIGNED>
__global__ void __launch_bounds__(256) k_filter_aggregated(const uint32_t* __restrict__ keys, int64_t n,
                                                           KeepRule rule, uint32_t* __restrict__ out,
                                                           unsigned long long* __restrict__ count) {
  const int lane = lane_id();
  const unsigned lt = lanemask_lt();
  constexpr int64_t CH = 32 * kFilterRounds;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += wstep) {
    const int64_t base = c * CH;
    uint32_t k[kFilterRounds];
    unsigned m[kFilterRounds];
#pragma unroll
    for (int j = 0; j < kFilterRounds; ++j) {
      const int64_t i = base + 32 * j + lane;
      k[j] = i < n ? __ldcs(keys + i) : 0u;
      m[j] = __ballot_sync(kFull, i < n && keep_key<SIGNED>(k[j], rule));
    }
    unsigned total = 0;
#pragma unroll
    for (int j = 0; j < kFilterRounds; ++j) total += __popc(m[j]);
    unsigned long long b = 0;
    if (lane == 0 && total) b = atomicAdd(count, (unsigned long long)total);
    b = __shfl_sync(kFull, b, 0);
    unsigned off = 0;
#pragma unroll
    for (int j = 0; j < kFilterRounds; ++j) {
      if (m[j] & (1u << lane)) out[b + off + __popc(m[j] & lt)] = k[j];
      off += __popc(m[j]);
    }
  }
}

template <int DT>
static cox_status launch_coalesced(int fn, const void* d_in, const int32_t* d_active, void* d_out, int64_t n,
                                   int param, cudaStream_t st) {
  auto k = k_coalesced<DT>;
  static int g = 0;  // persistent grid of this instance
  if (g == 0) g = persistent_grid(k, 256, 0, 1 << 30);
  const int64_t ctas = ((n + 32 * kCgUnroll - 1) / (32 * kCgUnroll) + 7) / 8;
  k<<<(int)(ctas < g ? ctas : g), 256, 0, st>>>(fn, static_cast<const uint32_t*>(d_in), d_active,
                                                static_cast<uint32_t*>(d_out), n, param);
  return launch_status();
}

template <bool SIGNED>
static cox_status launch_filter(const void* d_keys, int64_t n, int64_t threshold, void* d_out, int64_t* d_count,
                                cudaStream_t st) {
  auto k = k_filter_aggregated<SIGNED>;
  static int g = 0;
  if (g == 0) g = persistent_grid(k, 256, 0, 1 << 30);
  const int64_t chunks = (n + 32 * kFilterRounds - 1) / (32 * kFilterRounds);
  const int64_t ctas = (chunks + 7) / 8;
  k<<<(int)(ctas < g ? ctas : g), 256, 0, st>>>(static_cast<const uint32_t*>(d_keys), n, keep_rule<SIGNED>(threshold),
                                                static_cast<uint32_t*>(d_out),
                                                reinterpret_cast<unsigned long long*>(d_count));
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_coalesced(cox_cgfn fn, cox_dtype dt, int block_dim, const void* d_in,
                                    const int32_t* d_active, void* d_out, int64_t n, int param, void* stream) {
  if (!valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (fn < COX_CG_SIZE || fn > COX_CG_SCAN_SUM) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32 && dt != COX_F32) return COX_EINVAL;
  if ((fn == COX_CG_REDUCE_SUM || fn == COX_CG_SCAN_SUM) && dt == COX_F32) return COX_EINVAL;
  if ((fn == COX_CG_SHFL || fn == COX_CG_SHFL_UP || fn == COX_CG_SHFL_DOWN) && (param < 0 || param > 31))
    return COX_EINVAL;
  if (n == 0) return COX_OK;
  if (!d_in || !d_active || !d_out) return COX_EINVAL;
  if (dt == COX_F32) return launch_coalesced<COX_F32>((int)fn, d_in, d_active, d_out, n, param, as_stream(stream));
  return launch_coalesced<COX_I32>((int)fn, d_in, d_active, d_out, n, param, as_stream(stream));
}

extern "C" cox_status cox_filter_aggregated(cox_dtype dt, const void* d_keys, int64_t n, int64_t threshold,
                                            void* d_out, int64_t* d_count, void* stream) {
  if (n < 0 || !d_count || (dt != COX_I32 && dt != COX_U32)) return COX_EINVAL;
  if (n > 0 && (!d_keys || !d_out)) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), st) != cudaSuccess) return COX_ECUDA;
  if (n == 0) return COX_OK;
  if (dt == COX_I32) return launch_filter<true>(d_keys, n, threshold, d_out, d_count, st);
  return launch_filter<false>(d_keys, n, threshold, d_out, d_count, st);
}
