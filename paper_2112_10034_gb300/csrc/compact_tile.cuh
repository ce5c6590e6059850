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
// Tile layout: a tile of kBigTile = 16384 keys sits in shared memory.  Warp
// w of pass j owns the run of 512 keys at 16Bj + 512w; its lanes read them
// as four 128-bit chunks, lane l holding keys 128q + 4l .. 128q + 4l + 3 of
// chunk q.  The rank of a kept key in the tile is
//   offset(j, w) + kept keys of earlier chunks of the run
//     + sum_k' popc(ballot_k'(q) & lanemask_lt) + kept keys before it in the lane,
// which is its position in input order, so the result is the stable filter.
#pragma once

#include "cox_common.cuh"

namespace cox {

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

// ------------------------------------------------------------ big tiles
// Compaction of one tile of up to kBigTile keys already in shared memory
// (`buf`, valid keys at [0, valid)), with the whole CTA of B threads
// (16 * B divides kBigTile).  `wcnt` holds kBigTile / 512 words.  Counts
// with redux.sync, publishes the tile's count, compacts in place (a key's
// rank never exceeds its index), looks back for the prefix and copies the
// kept keys to out[prefix ..]; the last tile writes *d_count.
constexpr int64_t kBigTile = 16384;  // keys per tile (64 KB); 16 * block_dim divides it for every block_dim

// key < thr as one 32-bit compare: thr is clamped into the key range first
// (every key passes if thr is above the range, none if at or below it).
struct KeepRule {
  uint32_t t;  // keep iff key < t in the key's own signedness...
  int mode;    // ...when mode == 0; mode 1 keeps all, mode 2 keeps none
};

template <bool SIGNED>
__host__ __device__ inline KeepRule keep_rule(int64_t thr) {
  const int64_t lo = SIGNED ? -(int64_t(1) << 31) : 0;
  const int64_t hi = SIGNED ? (int64_t(1) << 31) - 1 : (int64_t(1) << 32) - 1;
  if (thr > hi) return {0u, 1};
  if (thr <= lo) return {0u, 2};
  return {(uint32_t)thr, 0};
}

template <bool SIGNED>
__device__ __forceinline__ bool keep_key(uint32_t k, KeepRule r) {
  const bool lt = SIGNED ? (int32_t)k < (int32_t)r.t : k < r.t;
  return r.mode == 0 ? lt : r.mode == 1;
}

// The count and compact passes over one tile; FULL tiles skip bounds checks.
// Pass j covers keys [16Bj, 16B(j+1)) of the tile; warp w owns the run
// [16Bj + 512w, + 512) of it, lane l holding keys 128q + 4l .. + 3 of the run
// for chunks q = 0..3 (128-bit shared loads, no bank conflicts).  Order of a
// tile: pass, warp, chunk, lane, key -- which is input order.
template <bool FULL>
__device__ __forceinline__ int run_index(int j, int B, int warp, int q, int lane) {
  return 16 * B * j + 512 * warp + 128 * q + 4 * lane;
}

// Count: each lane counts its kept keys, redux.sync gives the warp's count.
template <bool SIGNED, bool FULL>
__device__ __forceinline__ void count_pass(const uint32_t* buf, int j, int B, int nw, int warp, int lane,
                                           int valid, KeepRule r, uint32_t* wcnt) {
  uint32_t c = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i0 = run_index<FULL>(j, B, warp, q, lane);
    const uint4 v = *reinterpret_cast<const uint4*>(buf + i0);
    c += (FULL || i0 + 0 < valid) && keep_key<SIGNED>(v.x, r);
    c += (FULL || i0 + 1 < valid) && keep_key<SIGNED>(v.y, r);
    c += (FULL || i0 + 2 < valid) && keep_key<SIGNED>(v.z, r);
    c += (FULL || i0 + 3 < valid) && keep_key<SIGNED>(v.w, r);
  }
  c = __reduce_add_sync(kFull, c);
  if (lane == 0) wcnt[j * nw + warp] = c;
}

// Compact: rank = warp offset + kept keys of earlier chunks of the run +
// popc(ballot & lanemask_lt) over the chunk's four key slots + kept keys
// before it in the lane; every kept key moves to buf[rank].
template <bool SIGNED, bool FULL>
__device__ __forceinline__ void compact_pass(uint32_t* buf, int j, int B, int nw, int warp, int lane, int valid,
                                             KeepRule r, const uint32_t* wcnt, unsigned lt) {
  uint32_t key[4][4], pos[4][4];
  bool kp[4][4];
  uint32_t base = wcnt[j * nw + warp];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i0 = run_index<FULL>(j, B, warp, q, lane);
    const uint4 v = *reinterpret_cast<const uint4*>(buf + i0);
    key[q][0] = v.x; key[q][1] = v.y; key[q][2] = v.z; key[q][3] = v.w;
    uint32_t o = base, chunk = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      kp[q][k] = (FULL || i0 + k < valid) && keep_key<SIGNED>(key[q][k], r);
      const unsigned b = __ballot_sync(kFull, kp[q][k]);
      o += __popc(b & lt);
      chunk += __popc(b);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // o = rank of this lane's first kept key in chunk q
      pos[q][k] = o;
      o += kp[q][k];
    }
    base += chunk;
  }
  __syncthreads();  // every read of pass j before any write of pass j
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (kp[q][k]) buf[pos[q][k]] = key[q][k];
}

template <bool SIGNED>
__device__ __forceinline__ void compact_big_tile(uint32_t* buf, int valid, int64_t thr, uint32_t* __restrict__ out,
                                                 int64_t* __restrict__ d_count, uint64_t* desc, int64_t tile,
                                                 int64_t ntiles, int64_t n, uint32_t limit, unsigned* status,
                                                 uint32_t* wcnt) {
  const int B = blockDim.x, nw = B >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t TILE = kBigTile;
  const int passes = (int)(TILE / (16 * B));
  const int m = passes * nw;
  __shared__ int64_t s_prefix;
  __shared__ uint32_t s_total;
  __shared__ int s_bad;
  // ---- count: pass j, chunk q holds keys j*16B + q*4B + 4t .. + 3
  const KeepRule rule = keep_rule<SIGNED>(thr);
  const int vlen = valid;
#pragma unroll 1
  for (int j = 0; j < passes; ++j) {
    if (valid == TILE) count_pass<SIGNED, true>(buf, j, B, nw, warp, lane, vlen, rule, wcnt);
    else count_pass<SIGNED, false>(buf, j, B, nw, warp, lane, vlen, rule, wcnt);
  }
  __syncthreads();
  // ---- scan of the m = 32 counts (one per lane) and the tile's count
  if (warp == 0) {
    const int per = (m + 31) / 32;
    uint32_t sum = 0;
    for (int k = 0; k < per; ++k) {
      const int idx = lane * per + k;
      if (idx < m) sum += wcnt[idx];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += u;
    }
    uint32_t ex = incl - sum;
    for (int k = 0; k < per; ++k) {
      const int idx = lane * per + k;
      if (idx < m) {
        const uint32_t c = wcnt[idx];
        wcnt[idx] = ex;
        ex += c;
      }
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (lane == 0) {
      st_relaxed_u64(desc + tile, (tile == 0 ? kFlagP : kFlagA) | total);
      s_total = total;
    }
  }
  __syncthreads();
  // ---- compact in place, pass by pass
  const unsigned lt = lanemask_lt();
#pragma unroll 1
  for (int j = 0; j < passes; ++j) {
    if (valid == TILE) compact_pass<SIGNED, true>(buf, j, B, nw, warp, lane, vlen, rule, wcnt, lt);
    else compact_pass<SIGNED, false>(buf, j, B, nw, warp, lane, vlen, rule, wcnt, lt);
  }
  // ---- prefix and copy-out
  if (warp == 0) {
    bool gave_up;
    const int64_t prefix = look_back(desc, tile, s_total, limit, status, gave_up);
    if (lane == 0) {
      s_prefix = prefix;
      s_bad = gave_up;
    }
  }
  __syncthreads();
  const int64_t prefix = s_prefix;
  const uint32_t total = s_total;
  if (s_bad || prefix + (int64_t)total > n) return;
  for (int i = tid; i < (int)total; i += B) out[prefix + i] = buf[i];
  if (tile == ntiles - 1 && tid == 0) *d_count = prefix + total;
}

}  // namespace cox
