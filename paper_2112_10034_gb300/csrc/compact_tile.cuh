// Tile body of the ballot-driven stable compaction, shared by
// cox_ballot_compact and the request server.
//
// The filter of the SDK kernel filter_arr (Table 1 of the paper) with a
// static, full-warp group instead of the dynamically coalesced one (the paper
// covers non-divergent warp functions only, Section 2.2.3):
//   b = __ballot_sync(full, key < t); rank = popc(b & lanemask_lt);
// a shared-memory scan orders the warps of a tile, and tiles are ordered by
// a single-pass decoupled look-back over per-tile descriptors.  A tile only
// waits on tiles with smaller indexes, which callers hand out in order to
// CTAs that already run, so the waits end; each wait is still bounded.
//
// Tile layout: a CTA of B threads owns B*16 consecutive keys, read as four
// 128-bit loads per thread; chunk j (4B keys) has thread t holding keys
// j*4B + 4t .. 4t+3.  The rank of key (j, t, k) in the tile is
//   offset(j, warp) + sum_k' popc(ballot_k'(j) & lanemask_lt) + #{k' < k kept}
// which is its position in input order, so the result is the stable filter.
#pragma once

#include "cox_common.cuh"

namespace cox {

constexpr int kCompactEpt = 16;
constexpr size_t kCompactWsHeader = 256;
constexpr uint64_t kFlagA = 1ull << 62;  // descriptor holds the tile's own count
constexpr uint64_t kFlagP = 2ull << 62;  // descriptor holds the inclusive prefix
constexpr uint64_t kValMask = (1ull << 62) - 1;

// Look-back by one warp, after the tile published its own count (flag A; P
// for tile 0).  The warp reads a window of 32 * kLookV predecessors at a
// time -- lane l holds positions l*kLookV .. l*kLookV + kLookV - 1 counted
// back from the tile -- and stops at the closest published inclusive prefix
// (flag P), adding the counts of the tiles in between.  Only descriptors
// closer than that prefix must be published; the warp re-polls just those,
// tightly at first and then with a short back-off, for at most `limit`
// rounds.  Returns the tile's exclusive prefix (every lane) and publishes the
// tile's inclusive prefix.  On time-out: records kDevTimeout, publishes a zero
// prefix so successors end, and sets gave_up.
constexpr int kLookV = 4;

__device__ __forceinline__ int64_t look_back(uint64_t* desc, int64_t tile, uint32_t total, uint32_t limit,
                                             unsigned* status, bool& gave_up) {
  const int lane = lane_id();
  gave_up = false;
  if (tile == 0) return 0;
  int64_t prefix = 0;
  uint32_t polls = 0;
  bool timed_out = false;
  for (int64_t w0 = tile - 1;; w0 -= 32 * kLookV) {
    uint64_t d[kLookV];
#pragma unroll
    for (int v = 0; v < kLookV; ++v) {
      const int64_t i = w0 - (lane * kLookV + v);
      d[v] = i >= 0 ? ld_relaxed_u64(desc + i) : kFlagP;  // before tile 0: prefix 0
    }
    int lp;
    unsigned pm;
    for (;;) {
      lp = kLookV;
#pragma unroll
      for (int v = kLookV - 1; v >= 0; --v)
        if ((d[v] >> 62) == 2) lp = v;
      pm = __ballot_sync(kFull, lp < kLookV);
      const int fl = pm ? __ffs(pm) - 1 : 32;  // lane holding the closest prefix
      bool missing = false;
#pragma unroll
      for (int v = 0; v < kLookV; ++v)
        if ((lane < fl || (lane == fl && v <= lp)) && (d[v] >> 62) == 0) missing = true;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(100);
#pragma unroll
      for (int v = 0; v < kLookV; ++v) {
        const int64_t i = w0 - (lane * kLookV + v);
        if ((d[v] >> 62) == 0 && i >= 0) d[v] = ld_relaxed_u64(desc + i);
      }
    }
    if (timed_out) break;
    const int fl = pm ? __ffs(pm) - 1 : 32;
    unsigned long long sum = 0;
#pragma unroll
    for (int v = 0; v < kLookV; ++v)
      if (lane < fl || (lane == fl && v <= lp)) sum += d[v] & kValMask;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
    prefix += (int64_t)sum;
    if (pm) break;
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(desc + tile, kFlagP);  // release successors with a zero prefix
    }
    return 0;
  }
  if (lane == 0) st_relaxed_u64(desc + tile, kFlagP | ((uint64_t)(prefix + total) & kValMask));
  return prefix;
}

// One compaction tile with the whole CTA.  `smem` holds B*16 + 4*(B/32)
// words.  `sk`, if not null, holds the tile's B*16 keys already in shared
// memory (a full tile); otherwise the keys are read from global memory.
// Ends with every thread past its last shared-memory access except the
// final copy-out; callers that reuse `smem` must __syncthreads first.
template <bool SIGNED>
__device__ __forceinline__ void compact_tile(const uint32_t* __restrict__ keys, int64_t n, int64_t thr,
                                             uint32_t* __restrict__ out, int64_t* __restrict__ d_count,
                                             uint64_t* desc, int64_t tile, int64_t ntiles, uint32_t limit,
                                             unsigned* status, int vec, uint32_t* smem,
                                             const uint32_t* sk = nullptr) {
  const int B = blockDim.x;
  const int nw = B >> 5;
  const int64_t TILE = (int64_t)B * kCompactEpt;
  uint32_t* stage = smem;               // TILE words: the tile's kept keys, compacted
  uint32_t* wcnt = smem + TILE;         // 4 * nw warp counts, then their offsets
  __shared__ int64_t s_prefix;
  __shared__ uint32_t s_total;
  __shared__ int s_gave_up;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = tile * TILE;

  uint32_t key[4][4];
  bool keep[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t e0 = base + (int64_t)j * 4 * B + 4 * tid;
    if (sk) {
      const uint4 q = *reinterpret_cast<const uint4*>(sk + (int64_t)j * 4 * B + 4 * tid);
      key[j][0] = q.x; key[j][1] = q.y; key[j][2] = q.z; key[j][3] = q.w;
#pragma unroll
      for (int k = 0; k < 4; ++k) keep[j][k] = true;
    } else if (vec && e0 + 4 <= n) {
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
    if (lane == 0) {  // publish the tile's count at once (its prefix if it is tile 0)
      st_relaxed_u64(desc + tile, (tile == 0 ? kFlagP : kFlagA) | total);
      s_total = total;
    }
  }
  __syncthreads();
  // every warp stages its kept keys, compacted, in input order; warp 0 then
  // walks back for the tile's prefix while the others are done
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t o = wcnt[j * nw + warp] + lane_pre[j];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (keep[j][k]) stage[o++] = key[j][k];
  }
  if (warp == 0) {
    bool gave_up;
    const int64_t prefix = look_back(desc, tile, s_total, limit, status, gave_up);
    if (lane == 0) {
      s_prefix = prefix;
      s_gave_up = gave_up;
    }
  }
  __syncthreads();
  const int64_t prefix = s_prefix;
  const uint32_t total = s_total;
  if (s_gave_up || prefix + (int64_t)total > n) return;
  for (int i = tid; i < (int)total; i += B) out[prefix + i] = stage[i];
  if (tile == ntiles - 1 && tid == 0) *d_count = prefix + total;
}


}  // namespace cox
