// cox_vote_stats: batched statistics of the SDK vote kernels (VoteAny,
// VoteAll; Table 1 of the paper).  A row of 32 predicates is one warp
// ballot (lane l = element 32r + l); the row's tiles of width W are its
// W-bit fields: a tile's any() is its field != 0, its all() is its field
// == all ones, and the row's true predicates are popc of the ballot.
//
// Persistent warps take chunks of 32 rows (1024 elements), 8 rows' loads in
// flight at a time, and add each chunk's counts to its segment with three
// atomics (per row when a chunk spans segments).  Aligned inputs whose
// segments are whole 4096-element chunks take a 128-bit-load form.
#include "cox_common.cuh"

namespace cox {

constexpr int kVoteRows = 32;  // rows per warp chunk
constexpr int kVoteBatch = 8;  // row loads in flight

// Bit jW of the result is the OR (any) or AND (all) of field j of m.
template <int W, bool ALL>
__device__ __forceinline__ unsigned fold_fields(unsigned m) {
#pragma unroll
  for (int s = 1; s < W; s <<= 1) m = ALL ? (m & (m >> s)) : (m | (m >> s));
  return m;
}
template <int W>
__device__ __forceinline__ unsigned field_lows() {  // bit jW set for every field j
  unsigned r = 0;
#pragma unroll
  for (int j = 0; j < 32; j += W) r |= 1u << j;
  return r;
}

template <int W, int DT>
__global__ void __launch_bounds__(256) k_vote_stats(const uint32_t* __restrict__ pred, int64_t n, int64_t seg_len,
                                                    unsigned long long* __restrict__ stats) {
  const int lane = lane_id();
  constexpr int64_t CH = 32 * kVoteRows;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lows = field_lows<W>();
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += wstep) {
    const int64_t base = c * CH;
    const int64_t last = (base + CH < n ? base + CH : n) - 1;
    const bool one_seg = base / seg_len == last / seg_len;
    unsigned long long a = 0, al = 0, pc = 0;  // per-chunk counts (warp-uniform)
#pragma unroll 1
    for (int r0 = 0; r0 < kVoteRows; r0 += kVoteBatch) {
      uint32_t v[kVoteBatch];
#pragma unroll
      for (int r = 0; r < kVoteBatch; ++r) {
        const int64_t i = base + (int64_t)(r0 + r) * 32 + lane;
        v[r] = i < n ? __ldcs(pred + i) : 0u;
      }
#pragma unroll
      for (int r = 0; r < kVoteBatch; ++r) {
        const bool p = DT == COX_F32 ? __uint_as_float(v[r]) != 0.0f : v[r] != 0u;
        const unsigned m = __ballot_sync(kFull, p);
        const int64_t e0 = base + (int64_t)(r0 + r) * 32;
        if (e0 >= n) break;  // warp-uniform
        const unsigned any_bits = fold_fields<W, false>(m) & lows;
        const unsigned all_bits = fold_fields<W, true>(m) & lows;
        if (one_seg) {
          a += __popc(any_bits);
          al += __popc(all_bits);
          pc += __popc(m);
        } else if (lane == 0) {  // tiles of this row may belong to two segments
#pragma unroll
          for (int j = 0; j < 32; j += W) {
            if (e0 + j >= n) break;
            const int64_t s = (e0 + j) / seg_len;
            const unsigned f = (W == 32 ? m : (m >> j) & ((1u << W) - 1u));
            if ((any_bits >> j) & 1u) atomicAdd(stats + 3 * s, 1ull);
            if ((all_bits >> j) & 1u) atomicAdd(stats + 3 * s + 1, 1ull);
            if (f) atomicAdd(stats + 3 * s + 2, (unsigned long long)__popc(f));
          }
        }
      }
    }
    if (one_seg && lane == 0) {
      const int64_t s = base / seg_len;
      if (a) atomicAdd(stats + 3 * s, a);
      if (al) atomicAdd(stats + 3 * s + 1, al);
      if (pc) atomicAdd(stats + 3 * s + 2, pc);
    }
  }
}

// Vectorised form for 16-byte aligned input and segments that are whole
// 4096-element chunks.  Lane l loads elements 4l .. 4l+3 of each 128-element
// group; ballot k has bit l = element 4l + k.  A tile of W >= 4 elements is
// lanes [tW/4, (t+1)W/4) over all four ballots, so its any() / all() are the
// OR / AND of those lanes' bits in (m0|m1|m2|m3) / (m0&m1&m2&m3); a tile of
// 2 is (m0, m1) or (m2, m3) of one lane.
constexpr int kVoteGroups = 32;  // 128-element groups per chunk (4096 elements)
constexpr int kVoteVecBatch = 8;

template <int W, int DT>
__device__ __forceinline__ bool pred_of(uint32_t u) {
  return DT == COX_F32 ? __uint_as_float(u) != 0.0f : u != 0u;
}

template <int W, int DT>
__global__ void __launch_bounds__(256) k_vote_stats_vec(const uint32_t* __restrict__ pred, int64_t n, int64_t seg_len,
                                                        unsigned long long* __restrict__ stats) {
  const int lane = lane_id();
  constexpr int64_t CH = 128 * kVoteGroups;
  const int64_t nch = (n + CH - 1) / CH;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int F = W >= 4 ? W / 4 : 1;
  const unsigned lows = field_lows<F>();
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += wstep) {
    const int64_t base = c * CH;
    const bool full = base + CH <= n;
    unsigned long long a = 0, al = 0, pc = 0;
#pragma unroll 1
    for (int g0 = 0; g0 < kVoteGroups; g0 += kVoteVecBatch) {
      uint4 q[kVoteVecBatch];
#pragma unroll
      for (int g = 0; g < kVoteVecBatch; ++g) {
        const int64_t e = base + (int64_t)(g0 + g) * 128 + 4 * lane;
        if (full) {
          q[g] = __ldcs(reinterpret_cast<const uint4*>(pred + e));
        } else {
          q[g].x = e < n ? pred[e] : 0u;
          q[g].y = e + 1 < n ? pred[e + 1] : 0u;
          q[g].z = e + 2 < n ? pred[e + 2] : 0u;
          q[g].w = e + 3 < n ? pred[e + 3] : 0u;
        }
      }
#pragma unroll
      for (int g = 0; g < kVoteVecBatch; ++g) {
        const unsigned m0 = __ballot_sync(kFull, pred_of<W, DT>(q[g].x));
        const unsigned m1 = __ballot_sync(kFull, pred_of<W, DT>(q[g].y));
        const unsigned m2 = __ballot_sync(kFull, pred_of<W, DT>(q[g].z));
        const unsigned m3 = __ballot_sync(kFull, pred_of<W, DT>(q[g].w));
        pc += __popc(m0) + __popc(m1) + __popc(m2) + __popc(m3);
        if constexpr (W == 2) {
          a += __popc(m0 | m1) + __popc(m2 | m3);
          al += __popc(m0 & m1) + __popc(m2 & m3);
        } else {
          a += __popc(fold_fields<F, false>(m0 | m1 | m2 | m3) & lows);
          al += __popc(fold_fields<F, true>(m0 & m1 & m2 & m3) & lows);
        }
      }
    }
    if (lane == 0) {
      const int64_t s = base / seg_len;
      if (a) atomicAdd(stats + 3 * s, a);
      if (al) atomicAdd(stats + 3 * s + 1, al);
      if (pc) atomicAdd(stats + 3 * s + 2, pc);
    }
  }
}

template <int W, int DT>
static cox_status launch_vote_vec(const void* d_pred, int64_t n, int64_t seg_len, int64_t* d_stats, cudaStream_t st) {
  auto k = k_vote_stats_vec<W, DT>;
  static int g = 0;
  if (g == 0) g = persistent_grid(k, 256, 0, 1 << 30);
  const int64_t ctas = ((n + 128 * kVoteGroups - 1) / (128 * kVoteGroups) + 7) / 8;
  k<<<(int)(ctas < g ? ctas : g), 256, 0, st>>>(static_cast<const uint32_t*>(d_pred), n, seg_len,
                                                reinterpret_cast<unsigned long long*>(d_stats));
  return launch_status();
}

template <int W, int DT>
static cox_status launch_vote(const void* d_pred, int64_t n, int64_t seg_len, int64_t* d_stats, cudaStream_t st) {
  auto k = k_vote_stats<W, DT>;
  static int g = 0;
  if (g == 0) g = persistent_grid(k, 256, 0, 1 << 30);
  const int64_t ctas = ((n + 32 * kVoteRows - 1) / (32 * kVoteRows) + 7) / 8;
  k<<<(int)(ctas < g ? ctas : g), 256, 0, st>>>(static_cast<const uint32_t*>(d_pred), n, seg_len,
                                                reinterpret_cast<unsigned long long*>(d_stats));
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_vote_stats(cox_dtype dt, int width, const void* d_pred, int64_t n, int64_t seg_len,
                                     int64_t* d_stats, void* stream) {
  if (!valid_width(width) || n < 0 || seg_len < 1 || seg_len % width != 0) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32 && dt != COX_F32) return COX_EINVAL;
  if (n == 0) return COX_OK;
  if (!d_pred || !d_stats) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  const int64_t nseg = (n + seg_len - 1) / seg_len;
  if (cudaMemsetAsync(d_stats, 0, (size_t)nseg * 3 * sizeof(int64_t), st) != cudaSuccess) return COX_ECUDA;
  return with_width(width, [&](auto w) {
    constexpr int W = decltype(w)::value;
    if (aligned16(d_pred) && seg_len % (128 * kVoteGroups) == 0) {
      if (dt == COX_F32) return launch_vote_vec<W, COX_F32>(d_pred, n, seg_len, d_stats, st);
      return launch_vote_vec<W, COX_I32>(d_pred, n, seg_len, d_stats, st);
    }
    if (dt == COX_F32) return launch_vote<W, COX_F32>(d_pred, n, seg_len, d_stats, st);
    return launch_vote<W, COX_I32>(d_pred, n, seg_len, d_stats, st);
  });
}
