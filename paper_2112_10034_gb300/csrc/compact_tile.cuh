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
// The look-back has two levels: within a group of 32 tiles, then over whole
// groups (their counts summed by atomics as the last tile of each arrives).
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

// Two-level decoupled look-back over tile counts.  Tiles form groups of 32
// (group g = tiles 32g .. 32g+31).  Next to the per-tile descriptors
// desc[0 .. ntiles) the workspace holds, per group, a descriptor gdesc[g]
// and an accumulator gacc[g] = (arrivals << 48) | running count.  A tile
// publishes its count (flag A; tile 0: flag P) and adds (1 << 48) | count to
// its group's accumulator; the add that completes a group publishes the
// group's count (flag A) in gdesc[g].  A tile publishes its inclusive prefix
// (flag P) when its look-back ends, and the group's last tile also puts it
// in gdesc[g] (atomicMax: a P word is larger than any A word, so a late A
// never hides a P).  The look-back first reads the tile's own group
// (positions below it): the closest P there, plus the counts after it, is
// the answer; otherwise the in-group counts are summed and the warp walks
// back over whole groups, 32 groups (1024 tiles) per window, to the closest
// group with P, adding the counts of the groups in between.  A tile that
// runs ahead only ever waits on tiles with smaller indexes.  Every wait is
// bounded by `limit` polls; on time-out the tile records kDevTimeout and
// publishes a zero prefix so its successors end.
constexpr int kGroupShift = 5;  // 32 tiles per group
constexpr uint64_t kGroupArrive = 1ull << 48;
constexpr uint64_t kGroupSumMask = kGroupArrive - 1;

__host__ __device__ inline int64_t compact_groups(int64_t ntiles) {
  return (ntiles + (1 << kGroupShift) - 1) >> kGroupShift;
}
// Workspace bytes of a compaction over ntiles tiles: header (ticket), tile
// descriptors, group descriptors and group accumulators.
__host__ __device__ inline size_t compact_ws_bytes(int64_t ntiles) {
  return kCompactWsHeader + (size_t)ntiles * 8 + (size_t)compact_groups(ntiles) * 16;
}

// Publishes a tile's own count (lane 0 of the looking-back warp).
__device__ __forceinline__ void publish_count(uint64_t* desc, int64_t tile, int64_t ntiles, uint32_t total) {
  st_relaxed_u64(desc + tile, (tile == 0 ? kFlagP : kFlagA) | total);
  uint64_t* gdesc = desc + ntiles;
  uint64_t* gacc = gdesc + compact_groups(ntiles);
  const int64_t g = tile >> kGroupShift;
  const int64_t gsize = min((int64_t)1 << kGroupShift, ntiles - (g << kGroupShift));
  const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(gacc + g), kGroupArrive | total);
  if ((int64_t)(old >> 48) + 1 == gsize)
    atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), kFlagA | ((old + total) & kGroupSumMask));
}

// The tile's exclusive prefix (every lane of the calling warp); lane 0
// publishes the inclusive prefix.
__device__ __forceinline__ int64_t look_back(uint64_t* desc, int64_t tile, int64_t ntiles, uint32_t total,
                                             uint32_t limit, unsigned* status, bool& gave_up) {
  const int lane = lane_id();
  gave_up = false;
  uint64_t* gdesc = desc + ntiles;
  const int64_t g = tile >> kGroupShift;
  const int pos = (int)(tile & ((1 << kGroupShift) - 1));
  int64_t prefix = 0;
  uint32_t polls = 0;
  bool timed_out = false;
  bool done = tile == 0;
  // ---- the tile's own group: lane l holds position l < pos
  if (!done && pos > 0) {
    const int64_t g0 = g << kGroupShift;
    uint64_t d = lane < pos ? ld_relaxed_u64(desc + g0 + lane) : kFlagA;
    unsigned pm;
    int fl;
    for (;;) {
      pm = __ballot_sync(kFull, lane < pos && (d >> 62) == 2);
      fl = pm ? 31 - __clz(pm) : -1;  // closest inclusive prefix: the highest position
      const bool missing = lane < pos && lane > fl && (d >> 62) == 0;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(64);
      if (missing) d = ld_relaxed_u64(desc + g0 + lane);
    }
    if (!__any_sync(kFull, timed_out)) {
      unsigned long long v = (lane < pos && lane >= fl) ? (d & kValMask) : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
      prefix = (int64_t)v;
      done = fl >= 0;
    }
  }
  // ---- whole groups before it: lane l holds group gw - l
  if (!done && !__any_sync(kFull, timed_out)) {
    for (int64_t gw = g - 1;; gw -= 32) {
      const int64_t gi = gw - lane;
      uint64_t d = gi >= 0 ? ld_relaxed_u64(gdesc + gi) : kFlagP;  // before group 0: prefix 0
      unsigned pm;
      for (;;) {
        pm = __ballot_sync(kFull, (d >> 62) == 2);
        const int fl = pm ? __ffs(pm) - 1 : 32;  // closest group with an inclusive prefix
        const bool missing = lane <= fl && (d >> 62) == 0;
        if (!__any_sync(kFull, missing)) break;
        if (++polls > limit) {
          timed_out = true;
          break;
        }
        if (polls > 64) __nanosleep(64);
        if (missing && gi >= 0) d = ld_relaxed_u64(gdesc + gi);
      }
      if (__any_sync(kFull, timed_out)) break;
      const int fl = pm ? __ffs(pm) - 1 : 32;
      unsigned long long v = lane <= fl ? (d & kValMask) : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
      prefix += (int64_t)v;
      if (pm) break;
    }
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(desc + tile, kFlagP);  // release successors with a zero prefix
      if (pos == (1 << kGroupShift) - 1) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), kFlagP);
    }
    return 0;
  }
  if (lane == 0) {
    const uint64_t inc = kFlagP | ((uint64_t)(prefix + total) & kValMask);
    if (tile != 0) st_relaxed_u64(desc + tile, inc);
    if (pos == (1 << kGroupShift) - 1) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), inc);
  }
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
      publish_count(desc, tile, ntiles, total);
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
    const int64_t prefix = look_back(desc, tile, ntiles, s_total, limit, status, gave_up);
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
