// Tile body of the ballot-driven stable compaction, shared by
// cox_ballot_compact and the request server.
//
// The filter of the SDK kernel filter_arr (Table 1 of the paper) with a
// static, full-warp group instead of the dynamically coalesced one (the paper
// covers non-divergent warp functions only, Section 2.2.3):
//   b = __ballot_sync(full, key < t); rank = popc(b & lanemask_lt);
// a shared-memory scan orders the warps of a tile, and tiles are ordered by a
// single-pass decoupled look-back over per-tile descriptors.  A tile only
// waits on tiles with smaller indexes, which callers hand out in order to
// CTAs that already run, so the waits end; each wait is still bounded.
// The look-back has two levels: within a group of 32 tiles, then over whole
// groups (their counts summed by atomics as the last tile of each arrives).
//
// Tile layout: a tile of NW * 2048 keys sits in shared memory; warp w owns
// the region of keys [2048w, 2048w + 2048) and compacts it in place to the
// region's front in one pass, then copies it out after the look-back.
#pragma once

#include "cox_common.cuh"

namespace cox {

constexpr size_t kCompactWsHeader = 256;
constexpr uint64_t kFlagA = 1ull << 62;  // descriptor holds the tile's own count
constexpr uint64_t kFlagP = 2ull << 62;  // descriptor holds the inclusive prefix
constexpr uint64_t kValMask = (1ull << 62) - 1;
// Flags 0 (nothing yet) and 3 (withheld) both read as "not published".
// Descriptors only ever grow (atomicMax: A < P < withheld), so a word a
// caller withheld in a zeroed workspace (COX_F_WS_READY) stays withheld; the
// library never writes one itself -- tests use it to make a look-back wait
// run out.
__device__ __forceinline__ bool desc_missing(uint64_t d) {
  const uint64_t f = d >> 62;
  return f == 0 || f == 3;
}
__device__ __forceinline__ void desc_raise(uint64_t* p, uint64_t v) {
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

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
// Workspace bytes of a compaction over ntiles tiles: a header (reserved), tile
// descriptors, group descriptors and group accumulators.
__host__ __device__ inline size_t compact_ws_bytes(int64_t ntiles) {
  return kCompactWsHeader + (size_t)ntiles * 8 + (size_t)compact_groups(ntiles) * 16;
}

// Publishes a tile's own count (lane 0 of the looking-back warp).
__device__ __forceinline__ void publish_count(uint64_t* desc, int64_t tile, int64_t ntiles, uint32_t total) {
  desc_raise(desc + tile, (tile == 0 ? kFlagP : kFlagA) | total);
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
      const bool missing = lane < pos && lane > fl && desc_missing(d);
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
        const bool missing = lane <= fl && desc_missing(d);
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
      desc_raise(desc + tile, kFlagP);  // release successors with a zero prefix
      if (pos == (1 << kGroupShift) - 1) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), kFlagP);
    }
    return 0;
  }
  if (lane == 0) {
    const uint64_t inc = kFlagP | ((uint64_t)(prefix + total) & kValMask);
    if (tile != 0) desc_raise(desc + tile, inc);
    if (pos == (1 << kGroupShift) - 1) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), inc);
  }
  return prefix;
}

// ------------------------------------------------------------ big tiles
// Compaction of one tile of up to NW * 2048 keys already in shared memory
// (`buf`, valid keys at [0, valid)), by a CTA of NW warps.  `wcnt` holds
// kCompactWsWords words.  Each warp compacts its region in place, the tile's
// count is published, the look-back finds the tile's prefix, and every warp
// copies its kept keys to out[prefix + the warps before it ..]; the last
// tile writes *d_count.
constexpr int64_t kBigTile = 16384;  // elements per tile of the request server (64 KB)

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

// key < thr as one compare, key <= tm, in the key's own signedness: tm =
// thr - 1 clamped into the key range; `none` when thr is at or below the
// range's bottom (no key is kept).
struct LeRule {
  uint32_t tm;
  bool none;
};

template <bool SIGNED>
__host__ __device__ inline LeRule le_rule(int64_t thr) {
  const int64_t lo = SIGNED ? -(int64_t(1) << 31) : 0;
  const int64_t hi = SIGNED ? (int64_t(1) << 31) - 1 : (int64_t(1) << 32) - 1;
  if (thr <= lo) return {0u, true};
  return {(uint32_t)(thr - 1 > hi ? hi : thr - 1), false};
}

template <bool SIGNED>
__device__ __forceinline__ bool keep_le(uint32_t k, uint32_t tm) {
  return SIGNED ? (int32_t)k <= (int32_t)tm : k <= tm;
}

// The tile body runs NW warps per CTA on a tile of NW * 2048 keys: each warp
// owns a region of 2048 keys, which it reads as four sub-runs of 512 (lane l
// holds keys 128q + 4l .. 128q + 4l + 3 of a sub-run, q = 0..3:
// conflict-free 128-bit shared loads).
constexpr int kCompactRegion = 2048;  // keys per warp
constexpr int kCompactWsWords = 2 * 32;  // shared words the tile body needs (counts, offsets), any NW <= 32

// One sub-run of a warp's region, compacted in place to the front of the
// region.  Per chunk q and key slot k every lane votes b = __ballot_sync(keep);
// a kept key's rank in the region is
//   kept keys of earlier sub-runs and chunks + sum_k' popc(b_k' & lanes below)
//     + kept keys before it in its lane,
// i.e. its position in input order.  Ranks never exceed the key's own index,
// so the writes only reach keys every lane has already loaded (the
// __syncwarp after the loads orders them).  Returns the sub-run's count.
template <bool SIGNED, bool FULL>
__device__ __forceinline__ uint32_t compact_subrun(uint32_t* buf, int region, int sub, int lane, unsigned lt,
                                                   int valid, uint32_t tm, uint32_t kept_before) {
  const int sb = region + 512 * sub;
  uint32_t key[4][4];
  bool kp[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i0 = sb + 128 * q + 4 * lane;
    const uint4 v = *reinterpret_cast<const uint4*>(buf + i0);
    key[q][0] = v.x; key[q][1] = v.y; key[q][2] = v.z; key[q][3] = v.w;
#pragma unroll
    for (int k = 0; k < 4; ++k) kp[q][k] = (FULL || i0 + k < valid) && keep_le<SIGNED>(key[q][k], tm);
  }
  uint32_t below[4], total[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    below[q] = 0;
    total[q] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned b = __ballot_sync(kFull, kp[q][k]);
      below[q] += __popc(b & lt);
      total[q] += __popc(b);
    }
  }
  __syncwarp();  // every lane's loads of this sub-run before any write into it
  uint32_t chunk_base = kept_before;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t* o = buf + region + chunk_base + below[q];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (kp[q][k]) *o = key[q][k];
      o += kp[q][k];
    }
    chunk_base += total[q];
  }
  return chunk_base - kept_before;
}

// A warp's region of REG keys (a multiple of 512) compacted in place to its
// front, sub-run by sub-run; returns the region's count.
template <bool SIGNED, int REG>
__device__ __forceinline__ uint32_t compact_region(uint32_t* buf, int region, int lane, unsigned lt, int valid,
                                                   bool full, LeRule rule) {
  uint32_t kept = 0;
  if (rule.none) return 0;
  if (full) {
#pragma unroll 1
    for (int sub = 0; sub < REG / 512; ++sub)
      kept += compact_subrun<SIGNED, true>(buf, region, sub, lane, lt, valid, rule.tm, kept);
  } else {
#pragma unroll 1
    for (int sub = 0; sub < REG / 512 && region + 512 * sub < valid; ++sub)
      kept += compact_subrun<SIGNED, false>(buf, region, sub, lane, lt, valid, rule.tm, kept);
  }
  return kept;
}

template <bool SIGNED, int NW>
__device__ __forceinline__ void compact_big_tile(uint32_t* buf, int valid, int64_t thr, uint32_t* __restrict__ out,
                                                 int64_t* __restrict__ d_count, uint64_t* desc, int64_t tile,
                                                 int64_t ntiles, int64_t n, uint32_t limit, unsigned* status,
                                                 uint32_t* wcnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int region = warp * kCompactRegion;
  __shared__ int64_t s_prefix;
  __shared__ uint32_t s_total;
  __shared__ int s_bad;
  // ---- compact each warp's region in place (one pass over the keys)
  const LeRule rule = le_rule<SIGNED>(thr);
  const uint32_t kept =
      compact_region<SIGNED, kCompactRegion>(buf, region, lane, lanemask_lt(), valid, valid == NW * kCompactRegion, rule);
  if (lane == 0) wcnt[warp] = kept;
  __syncthreads();
  // ---- the tile's count, its prefix by look-back, the warps' offsets
  if (warp == 0) {
    const uint32_t c = lane < NW ? wcnt[lane] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < NW; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += u;
    }
    const uint32_t total = __shfl_sync(kFull, incl, NW - 1);
    if (lane < NW) wcnt[32 + lane] = incl - c;  // exclusive offsets
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
  const int64_t prefix = s_prefix;
  if (s_bad || prefix + (int64_t)s_total > n) return;
  // ---- each warp copies its compacted region to out[prefix + offset ..]
  uint32_t* dst = out + prefix + wcnt[32 + warp];
  const uint32_t* src = buf + region;
#pragma unroll 4
  for (int i = lane; i < (int)kept; i += 32) dst[i] = src[i];
  if (tile == ntiles - 1 && tid == 0) *d_count = prefix + s_total;
}

}  // namespace cox
