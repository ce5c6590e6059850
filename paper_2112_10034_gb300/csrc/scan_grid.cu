// cox_scan: block-scope and grid-scope inclusive / exclusive scans.
//
// BLOCK scope follows the SDK's shfl_scan_test (Table 1 of the paper): each
// warp scans its 32 elements with shfl_up (Hillis-Steele), warp totals go to
// shared memory, warp 0 scans them, and every element takes its warp's
// prefix (the uniform_add step).
//
// GRID scope chains tiles with a decoupled look-back.  16-byte aligned
// arrays take the row-tile kernel (k_scan_grid_rows, below); in any other
// layout a CTA takes a tile (16384 elements; 8192 for compensated sums,
// whose pairs need twice the shared memory) from an atomic ticket, receives
// it by one TMA bulk copy,
// and every warp scans its rows of 32 elements with shfl_up, carrying row
// totals across its rows (eight rows at a time for instruction-level
// parallelism).  Lane 0 of warp 0 scans the eight warp totals, the tile
// publishes its aggregate, walks back for its prefix, and every element
// takes prefix op warp-prefix op its value.  Each tile keeps its aggregate
// and its inclusive prefix in separate slots, each written before its flag
// (release store) and read after it (acquire load), so a reader never sees a
// value from the wrong stage.
#include <type_traits>

#include "cox_common.cuh"

namespace cox {

constexpr size_t kScanWsHeader = 256;
constexpr int kScanLookV = 4;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class R>
__device__ __forceinline__ uint64_t pack(typename R::V v) {
  if constexpr (R::kComp) return (uint64_t)__float_as_uint(v.s) | ((uint64_t)__float_as_uint(v.e) << 32);
  else return (uint64_t)to_bits(v);
}
template <class R>
__device__ __forceinline__ typename R::V unpack(uint64_t u) {
  using T = typename R::T;
  if constexpr (R::kComp) return Pair{__uint_as_float((uint32_t)u), __uint_as_float((uint32_t)(u >> 32))};
  else return from_bits<T>((uint32_t)u);
}
template <class R>
__device__ __forceinline__ typename R::V warp_fold(typename R::V v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = R::op(v, R::shfl_xor(v, off));
  return v;
}

// Look-back for generic scan values.  flags[t]: 0 nothing, 1 aggregate in
// agg[t], 2 inclusive prefix in inc[t].  Returns the tile's exclusive prefix.
template <class R>
__device__ typename R::V look_back_op(uint32_t* flags, uint64_t* agg, uint64_t* inc, int64_t tile,
                                      typename R::V total, uint32_t limit, unsigned* status, bool& gave_up) {
  using V = typename R::V;
  const int lane = lane_id();
  gave_up = false;
  if (tile == 0) {
    if (lane == 0) {
      st_relaxed_u64(inc, pack<R>(total));
      st_release_u32(flags, 2u);
    }
    return R::ident();
  }
  if (lane == 0) {
    st_relaxed_u64(agg + tile, pack<R>(total));
    st_release_u32(flags + tile, 1u);
  }
  V prefix = R::ident();
  uint32_t polls = 0;
  bool timed_out = false;
  for (int64_t w0 = tile - 1;; w0 -= 32 * kScanLookV) {
    uint32_t f[kScanLookV];
    uint64_t val[kScanLookV];
#pragma unroll
    for (int v = 0; v < kScanLookV; ++v) {
      const int64_t i = w0 - (lane * kScanLookV + v);
      f[v] = i >= 0 ? ld_acquire_u32(flags + i) : 2u;  // before tile 0: the identity
      val[v] = 0;
    }
    int lp;
    unsigned pm;
    for (;;) {
      lp = kScanLookV;
#pragma unroll
      for (int v = kScanLookV - 1; v >= 0; --v)
        if (f[v] == 2u) lp = v;
      pm = __ballot_sync(kFull, lp < kScanLookV);
      const int fl = pm ? __ffs(pm) - 1 : 32;
      bool missing = false;
#pragma unroll
      for (int v = 0; v < kScanLookV; ++v)
        if ((lane < fl || (lane == fl && v <= lp)) && f[v] == 0u) missing = true;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(100);
#pragma unroll
      for (int v = 0; v < kScanLookV; ++v) {
        const int64_t i = w0 - (lane * kScanLookV + v);
        if (f[v] == 0u && i >= 0) f[v] = ld_acquire_u32(flags + i);
      }
    }
    if (timed_out) break;
    const int fl = pm ? __ffs(pm) - 1 : 32;
    V part = R::ident();
#pragma unroll
    for (int v = kScanLookV - 1; v >= 0; --v) {  // older tiles first
      const int64_t i = w0 - (lane * kScanLookV + v);
      if (lane < fl || (lane == fl && v <= lp)) {
        const V x = i < 0 ? R::ident() : unpack<R>(ld_relaxed_u64((f[v] == 2u ? inc : agg) + i));
        part = R::op(x, part);
      }
    }
    prefix = R::op(warp_fold<R>(part), prefix);
    if (pm) break;
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(inc + tile, pack<R>(total));  // release successors
      st_release_u32(flags + tile, 2u);
    }
    return R::ident();
  }
  if (lane == 0) {
    st_relaxed_u64(inc + tile, pack<R>(R::op(prefix, total)));
    st_release_u32(flags + tile, 2u);
  }
  return prefix;
}

// Look-back for 32-bit scan values over packed descriptors: desc[t] =
// (state << 32) | value bits, state 0 nothing, 1 aggregate, 2 inclusive
// prefix, so one relaxed 64-bit load returns a consistent (state, value)
// pair (one round trip per window, no second load).  Same walk as
// look_back_op.  Returns the tile's exclusive prefix.
template <class R>
__device__ typename R::V look_back_packed(uint64_t* desc, int64_t tile, typename R::V total, uint32_t limit,
                                          unsigned* status, bool& gave_up) {
  using V = typename R::V;
  using T = typename R::T;
  const int lane = lane_id();
  gave_up = false;
  if (tile == 0) {
    if (lane == 0) st_relaxed_u64(desc, (2ull << 32) | to_bits(total));
    return R::ident();
  }
  if (lane == 0) st_relaxed_u64(desc + tile, (1ull << 32) | to_bits(total));
  V prefix = R::ident();
  uint32_t polls = 0;
  bool timed_out = false;
  for (int64_t w0 = tile - 1;; w0 -= 32 * kScanLookV) {
    uint64_t d[kScanLookV];
#pragma unroll
    for (int v = 0; v < kScanLookV; ++v) {
      const int64_t i = w0 - (lane * kScanLookV + v);
      d[v] = i >= 0 ? ld_relaxed_u64(desc + i) : ((2ull << 32) | to_bits(R::ident()));  // before tile 0
    }
    int lp;
    unsigned pm;
    for (;;) {
      lp = kScanLookV;
#pragma unroll
      for (int v = kScanLookV - 1; v >= 0; --v)
        if ((d[v] >> 32) == 2u) lp = v;
      pm = __ballot_sync(kFull, lp < kScanLookV);
      const int fl = pm ? __ffs(pm) - 1 : 32;
      bool missing = false;
#pragma unroll
      for (int v = 0; v < kScanLookV; ++v)
        if ((lane < fl || (lane == fl && v <= lp)) && (d[v] >> 32) == 0u) missing = true;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(64);
#pragma unroll
      for (int v = 0; v < kScanLookV; ++v) {
        const int64_t i = w0 - (lane * kScanLookV + v);
        if ((d[v] >> 32) == 0u && i >= 0) d[v] = ld_relaxed_u64(desc + i);
      }
    }
    if (timed_out) break;
    const int fl = pm ? __ffs(pm) - 1 : 32;
    V part = R::ident();
#pragma unroll
    for (int v = kScanLookV - 1; v >= 0; --v)  // older tiles first
      if (lane < fl || (lane == fl && v <= lp)) part = R::op(from_bits<T>((uint32_t)d[v]), part);
    prefix = R::op(warp_fold<R>(part), prefix);
    if (pm) break;
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(desc + tile, (2ull << 32) | to_bits(total));  // release successors
    }
    return R::ident();
  }
  if (lane == 0) st_relaxed_u64(desc + tile, (2ull << 32) | to_bits(R::op(prefix, total)));
  return prefix;
}

// Two-level form of look_back_packed for 32-bit sums (wrapping adds): tiles
// form groups of 32; a tile adds (1 << 48) | value to its group's
// accumulator gacc[g] after publishing its aggregate, and the add that
// completes the group publishes the group aggregate in gdesc[g]; the last
// tile of a group also puts its inclusive prefix there (atomicMax: a
// state-2 word is larger than any state-1 word).  The look-back reads the
// tile's own group first, then whole groups, 32 per window (1024 tiles), so
// its length no longer grows with the number of tiles in flight.
__device__ unsigned look_back_sum2(uint64_t* desc, uint64_t* gdesc, uint64_t* gacc, int64_t tile, int64_t ntiles,
                                   unsigned total, uint32_t limit, unsigned* status, bool& gave_up) {
  const int lane = lane_id();
  gave_up = false;
  const int64_t g = tile >> 5;
  const int pos = (int)(tile & 31);
  if (lane == 0) {
    st_relaxed_u64(desc + tile, ((tile == 0 ? 2ull : 1ull) << 32) | total);
    const int64_t gsize = min((int64_t)32, ntiles - (g << 5));
    const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(gacc + g), (1ull << 48) | total);
    if ((int64_t)(old >> 48) + 1 == gsize)
      atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), (1ull << 32) | (uint32_t)(old + total));
  }
  unsigned prefix = 0;
  uint32_t polls = 0;
  bool timed_out = false;
  bool done = tile == 0;
  if (!done && pos > 0) {  // own group: lane l holds position l < pos
    const int64_t g0 = g << 5;
    uint64_t d = lane < pos ? ld_relaxed_u64(desc + g0 + lane) : (1ull << 32);
    unsigned pm;
    int fl;
    for (;;) {
      pm = __ballot_sync(kFull, lane < pos && (d >> 32) == 2u);
      fl = pm ? 31 - __clz(pm) : -1;
      const bool missing = lane < pos && lane > fl && (d >> 32) == 0u;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(64);
      if (missing) d = ld_relaxed_u64(desc + g0 + lane);
    }
    if (!__any_sync(kFull, timed_out)) {
      unsigned v = (lane < pos && lane >= fl) ? (unsigned)d : 0u;
      prefix = __reduce_add_sync(kFull, v);
      done = fl >= 0;
    }
  }
  if (!done && !__any_sync(kFull, timed_out)) {  // whole groups: lane l holds group gw - l
    for (int64_t gw = g - 1;; gw -= 32) {
      const int64_t gi = gw - lane;
      uint64_t d = gi >= 0 ? ld_relaxed_u64(gdesc + gi) : (2ull << 32);  // before group 0: 0
      unsigned pm;
      for (;;) {
        pm = __ballot_sync(kFull, (d >> 32) == 2u);
        const int fl = pm ? __ffs(pm) - 1 : 32;
        const bool missing = lane <= fl && (d >> 32) == 0u;
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
      prefix += __reduce_add_sync(kFull, lane <= fl ? (unsigned)d : 0u);
      if (pm) break;
    }
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(desc + tile, (2ull << 32) | total);
      if (pos == 31) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), (2ull << 32) | total);
    }
    return 0u;
  }
  if (lane == 0) {
    const uint64_t inc = (2ull << 32) | (uint32_t)(prefix + total);
    if (tile != 0) st_relaxed_u64(desc + tile, inc);
    if (pos == 31) atomicMax(reinterpret_cast<unsigned long long*>(gdesc + g), inc);
  }
  return prefix;
}

// Look-back state and value in one 64-bit word, so a predecessor costs one
// load: bits 62-63 the state (1 aggregate, 2 inclusive prefix), below them
// the value -- a 32-bit value as is; a compensated pair as its sum word (bits
// 0-31) and its error word rounded to 21 mantissa bits (bits 32-61).  The
// rounding of an error word is at most 2^-22 of it, about 2^-46 of the sum:
// far below the 1e-5 bar.  Tile aggregates also go, exact, to their own slot
// for the group fold.
template <class R>
__device__ __forceinline__ uint64_t pk_word(uint64_t state, typename R::V v) {
  if constexpr (R::kComp) {
    const uint32_t eb = __float_as_uint(v.e);
    // round to nearest on the 30-bit field; a carry into the exponent is the
    // correct rounding up to the next binade
    const uint64_t e30 = ((uint64_t)eb + 2u) >> 2;
    return (state << 62) | ((e30 & 0x3FFFFFFFull) << 32) | (uint64_t)__float_as_uint(v.s);
  } else {
    return (state << 62) | (uint64_t)to_bits(v);
  }
}
template <class R>
__device__ __forceinline__ typename R::V pk_value(uint64_t w) {
  using T = typename R::T;
  if constexpr (R::kComp) return Pair{__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)((w >> 32) << 2))};
  else return from_bits<T>((uint32_t)w);
}

// Two-level look-back over packed words (any value except 32-bit sums, which
// take look_back_sum2).  word[t]: the tile's state|value; agg[t]: its exact
// aggregate; per group of 32 tiles gword[g] (state|value, only growing:
// atomicMax, and a prefix word is above any aggregate word) and an arrival
// counter gcnt[g].  The tile whose arrival completes its group folds the
// group's 32 aggregates in tile order and publishes the group aggregate; the
// group's last tile publishes its inclusive prefix as the group's.  Called by
// a whole warp; returns the exclusive prefix.
template <class R>
__device__ typename R::V look_back_pk(uint64_t* word, uint64_t* agg, uint64_t* gword, uint32_t* gcnt, int64_t tile,
                                      int64_t ntiles, typename R::V total, uint32_t limit, unsigned* status,
                                      bool& gave_up) {
  using V = typename R::V;
  const int lane = lane_id();
  gave_up = false;
  const int64_t g = tile >> 5;
  const int pos = (int)(tile & 31);
  const int64_t g0 = g << 5;
  int last = 0;
  if (lane == 0) {
    st_relaxed_u64(agg + tile, pack<R>(total));
    st_relaxed_u64(word + tile, pk_word<R>(tile == 0 ? 2u : 1u, total));
    __threadfence();
    const int64_t gsize = min((int64_t)32, ntiles - g0);
    last = (int64_t)atomicAdd(gcnt + g, 1u) + 1 == gsize;
    if (last) __threadfence();
  }
  if (__shfl_sync(kFull, last, 0)) {
    const int64_t gsize = min((int64_t)32, ntiles - g0);
    V v = lane < gsize ? unpack<R>(ld_relaxed_u64(agg + g0 + lane)) : R::ident();
    v = warp_fold<R>(v);
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(gword + g), pk_word<R>(1u, v));
  }
  V prefix = R::ident();
  uint32_t polls = 0;
  bool timed_out = false;
  bool done = tile == 0;
  if (!done && pos > 0) {  // own group: lane l holds position l < pos
    uint64_t w = lane < pos ? ld_relaxed_u64(word + g0 + lane) : (1ull << 62);
    unsigned pm;
    int fl;
    for (;;) {
      pm = __ballot_sync(kFull, lane < pos && (w >> 62) == 2u);
      fl = pm ? 31 - __clz(pm) : -1;
      const bool missing = lane < pos && lane > fl && (w >> 62) == 0u;
      if (!__any_sync(kFull, missing)) break;
      if (++polls > limit) {
        timed_out = true;
        break;
      }
      if (polls > 64) __nanosleep(64);
      if (missing) w = ld_relaxed_u64(word + g0 + lane);
    }
    if (!__any_sync(kFull, timed_out)) {
      V part = R::ident();
      if (lane < pos && lane >= fl) part = pk_value<R>(w);
      prefix = warp_fold<R>(part);
      done = fl >= 0;
    }
  }
  if (!done && !__any_sync(kFull, timed_out)) {  // whole groups: lane l holds group gw0 - l
    V gsum = R::ident();
    for (int64_t gw0 = g - 1;; gw0 -= 32) {
      const int64_t gi = gw0 - lane;
      uint64_t w = gi >= 0 ? ld_relaxed_u64(gword + gi) : (2ull << 62) | pk_word<R>(0u, R::ident());
      unsigned pm;
      for (;;) {
        pm = __ballot_sync(kFull, (w >> 62) == 2u);
        const int fl = pm ? __ffs(pm) - 1 : 32;
        const bool missing = lane <= fl && (w >> 62) == 0u;
        if (!__any_sync(kFull, missing)) break;
        if (++polls > limit) {
          timed_out = true;
          break;
        }
        if (polls > 64) __nanosleep(64);
        if (missing && gi >= 0) w = ld_relaxed_u64(gword + gi);
      }
      if (__any_sync(kFull, timed_out)) break;
      const int fl = pm ? __ffs(pm) - 1 : 32;
      V part = R::ident();
      if (lane <= fl && gi >= 0) part = pk_value<R>(w);
      gsum = R::op(warp_fold<R>(part), gsum);  // older windows on the left
      if (pm) break;
    }
    prefix = R::op(gsum, prefix);
  }
  if (__any_sync(kFull, timed_out)) {
    gave_up = true;
    if (lane == 0) {
      atomicOr(status, (unsigned)kDevTimeout);
      st_relaxed_u64(word + tile, pk_word<R>(2u, total));  // release successors
      if (pos == 31) atomicMax(reinterpret_cast<unsigned long long*>(gword + g), pk_word<R>(2u, total));
    }
    return R::ident();
  }
  if (lane == 0) {
    const V incl = R::op(prefix, total);
    if (tile != 0) st_relaxed_u64(word + tile, pk_word<R>(2u, incl));
    if (pos == 31) atomicMax(reinterpret_cast<unsigned long long*>(gword + g), pk_word<R>(2u, incl));
  }
  return prefix;
}

// Rows per lane of the row-tile grid scan (tiles of RPL x 8192 elements):
// one for 32-bit values (33 KB tiles, six CTAs per SM), two for compensated
// pairs (their registers allow four CTAs per SM, and the larger tile halves
// the look-backs).
template <class R>
__host__ __device__ constexpr int grid_rows_rpl() {
  return R::kComp ? 2 : 1;
}

template <class R>
__host__ __device__ constexpr int grid_scan_tile() {
  return R::kComp ? 8192 : 16384;
}

template <class R>
__global__ void __launch_bounds__(256) k_scan_grid(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                   int64_t n, unsigned* ticket, uint32_t* flags, uint64_t* agg,
                                                   uint64_t* inc, int64_t ntiles, int excl, uint32_t limit,
                                                   unsigned* status, int vec) {
  using T = typename R::T;
  using V = typename R::V;
  constexpr int TILE = grid_scan_tile<R>();
  constexpr int NW = 8;
  constexpr int RPW = TILE / 32 / NW;  // rows per warp
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* bs = smem;                                        // values (or sum words)
  float* be = reinterpret_cast<float*>(smem + TILE);          // error words (compensated)
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + TILE * (R::kComp ? 2 : 1));
  __shared__ V s_wtot[NW], s_cp[NW];
  __shared__ int64_t s_tile;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= ntiles) return;
  const int64_t base = tile * TILE;
  const int valid = (int)min((int64_t)TILE, n - base);
  if (vec && valid == TILE) {
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, (uint32_t)(TILE * 4));
      tma_load_1d(bs, in + base, (uint32_t)(TILE * 4), bar);
    }
    const bool ok = mbar_wait_bounded(bar, 0u, limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(status, (unsigned)kDevTimeout);
        mbar_wait_bounded(bar, 0u, limit);
        st_relaxed_u64(inc + tile, pack<R>(R::ident()));
        st_release_u32(flags + tile, 2u);
      }
      return;
    }
  } else {
    const uint32_t pad = to_bits(R::pad());
    for (int i = tid; i < TILE; i += blockDim.x) bs[i] = i < valid ? in[base + i] : pad;
    __syncthreads();
  }
  // rows of warp w: w*RPW .. w*RPW + RPW - 1, eight at a time
  V carry = R::ident();
#pragma unroll 1
  for (int g = 0; g < RPW / 8; ++g) {
    V v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = R::load(from_bits<T>(bs[(warp * RPW + g * 8 + i) * 32 + lane]));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const V u = R::shfl_up_fresh(v[i], 1, 32);
      if (lane >= 1) v[i] = R::op_fresh(u, v[i]);
    }
#pragma unroll
    for (int d = 2; d < 32; d <<= 1) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const V u = R::shfl_up(v[i], d, 32);
        if (lane >= d) v[i] = R::op(u, v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {  // carry the running total into each row
      const V tot = R::shfl_idx(v[i], 31, 32);
      v[i] = R::op(carry, v[i]);
      carry = R::op(carry, tot);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int idx = (warp * RPW + g * 8 + i) * 32 + lane;
      if constexpr (R::kComp) {
        bs[idx] = __float_as_uint(v[i].s);
        be[idx] = v[i].e;
      } else {
        bs[idx] = to_bits(v[i]);
      }
    }
  }
  if (lane == 0) s_wtot[warp] = carry;
  __syncthreads();
  if (warp == 0) {
    V total = R::ident();
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        s_cp[k] = total;  // warp-exclusive prefix for now
        total = R::op(total, s_wtot[k]);
      }
    }
    total = R::shfl_idx(total, 0, 32);
    bool gave_up;
    const V prefix = look_back_op<R>(flags, agg, inc, tile, total, limit, status, gave_up);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NW; ++k) s_cp[k] = R::op(prefix, s_cp[k]);
      s_bad = gave_up;
    }
  }
  __syncthreads();
  if (s_bad) return;
  const V cp = s_cp[warp];
  auto value = [&](int idx) -> V {
    if constexpr (R::kComp) return Pair{__uint_as_float(bs[idx]), be[idx]};
    else return from_bits<T>(bs[idx]);
  };
  const int first = warp * RPW * 32;
#pragma unroll 4
  for (int rr = 0; rr < RPW; ++rr) {
    const int idx = (warp * RPW + rr) * 32 + lane;
    const int64_t gi = base + idx;
    T y;
    if (!excl) y = R::out(R::op(cp, value(idx)));
    else y = idx == first ? R::out(cp) : R::out(R::op(cp, value(idx - 1)));
    if (gi < n) out[gi] = to_bits(y);
  }
}

// GRID scope over aligned arrays of at least one full row: tiles of RPL x 256
// rows of 32 elements (grid_rows_rpl) arrive by RPL 2D TMA boxes with
// 128-byte swizzle; lane t of warp w owns rows 32 (RPL w + j) + t, j < RPL,
// of the tile.  Pass A folds each row (its total), shuffle scans over the
// warp's rows and a
// scan of the 8 warp totals give every row's exclusive prefix, the tile
// looks back for its own prefix (32-bit values: packed state|value
// descriptors in `agg`), and pass B re-reads the row, carrying
// prefix op value into each element (in place), before one TMA store.
// Sums are folded left to right within a row, so fp32 results differ from
// the shuffle form in their last bits (tolerance-checked).  The partial last
// row (n % 32 elements) is read and written by its lane from global memory.
constexpr int kGridBoxRows = 256;  // rows per TMA box; a tile is RPL boxes (RPL rows per lane)

// a op x for one element x: for a compensated pair the element's error word
// is zero, so the error words need one add (a.e + t), not two.
template <class R>
__device__ __forceinline__ typename R::V op_elem(typename R::V a, typename R::T x) {
  if constexpr (R::kComp) {
    Pair r;
    float t;
    two_sum(a.s, x, r.s, t);
    r.e = __fadd_rn(a.e, t);
    return r;
  } else {
    return R::op(a, R::load(x));
  }
}

template <class R, int RPL>
__global__ void __launch_bounds__(256) k_scan_grid_rows(const __grid_constant__ CUtensorMap tin,
                                                        const __grid_constant__ CUtensorMap tout,
                                                        const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                        int64_t n, unsigned* ticket, uint32_t* flags, uint64_t* agg,
                                                        uint64_t* inc, int64_t ntiles, int excl, uint32_t limit,
                                                        unsigned* status) {
  using T = typename R::T;
  using V = typename R::V;
  extern __shared__ uint8_t gsr_raw[];
  uint4* buf = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(gsr_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t s_bar;
  __shared__ V s_wtot[8], s_cp[8];
  __shared__ int64_t s_tile;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t rows = n / 32;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    s_bad = 0;
    mbar_init(&s_bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= ntiles) return;
  constexpr int kTileRows = RPL * kGridBoxRows;
  const int64_t r0 = tile * kTileRows;
  // boxes holding full rows
  const int nbox = r0 >= rows ? 0 : (int)min((int64_t)RPL, (rows - r0 + kGridBoxRows - 1) / kGridBoxRows);
  if (tid == 0 && nbox > 0) {
    mbar_arrive_expect_tx(&s_bar, (uint32_t)nbox * kGridBoxRows * 128u);
    for (int bx = 0; bx < nbox; ++bx)
      tma_load_2d(buf + bx * kGridBoxRows * 8, &tin, 0, (int)(r0 + bx * kGridBoxRows), &s_bar);
  }
  // lane owns rows 32 * (RPL * w + j) + lane, j < RPL, of the tile
  int rl[RPL];
#pragma unroll
  for (int j = 0; j < RPL; ++j) rl[j] = 32 * (RPL * warp + j) + lane;
  const uint32_t pad = to_bits(R::pad());
  if (nbox > 0) {
    const bool ok = mbar_wait_bounded(&s_bar, 0u, limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(status, (unsigned)kDevTimeout);
        mbar_wait_bounded(&s_bar, 0u, limit);
        if constexpr (!std::is_same<R, Plain<AddU>>::value) {
          // a zero prefix for successors; the group level counts this tile's
          // arrival and, if it completes the group, publishes some aggregate
          // (the device status already says the results are not to be used)
          const int64_t ngroups = (ntiles + 31) / 32, g = tile >> 5;
          const int64_t gsize = min((int64_t)32, ntiles - (g << 5));
          uint64_t* gword = inc + ntiles;
          uint32_t* gcnt = reinterpret_cast<uint32_t*>(gword + ngroups);
          st_relaxed_u64(agg + tile, pack<R>(R::ident()));
          st_relaxed_u64(inc + tile, pk_word<R>(2u, R::ident()));
          __threadfence();
          if ((int64_t)atomicAdd(gcnt + g, 1u) + 1 == gsize)
            atomicMax(reinterpret_cast<unsigned long long*>(gword + g), pk_word<R>(1u, R::ident()));
          if ((tile & 31) == 31)
            atomicMax(reinterpret_cast<unsigned long long*>(gword + g), pk_word<R>(2u, R::ident()));
        } else {
          st_relaxed_u64(agg + tile, (2ull << 32) | to_bits(R::ident()));
          if constexpr (std::is_same<R, Plain<AddU>>::value) {  // keep the group level consistent
            const int64_t ngroups = (ntiles + 31) / 32, g = tile >> 5;
            const int64_t gsize = min((int64_t)32, ntiles - (g << 5));
            uint64_t* gd = inc + ntiles;
            const unsigned long long old =
                atomicAdd(reinterpret_cast<unsigned long long*>(gd + ngroups + g), 1ull << 48);
            if ((int64_t)(old >> 48) + 1 == gsize)
              atomicMax(reinterpret_cast<unsigned long long*>(gd + g), (1ull << 32) | (uint32_t)old);
            if ((tile & 31) == 31) atomicMax(reinterpret_cast<unsigned long long*>(gd + g), 2ull << 32);
          }
        }
      }
      return;
    }
  }
  // The partial last row (n % 32 elements) comes from global memory, after the
  // boxes have landed (they fill rows past the end with zeros).
  auto fill_partial = [&](int rl) {
    const int64_t row = r0 + rl;
    if (!(row == rows && rows * 32 < n)) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t e = row * 32 + 4 * j;
      uint4 q;
      q.x = e < n ? in[e] : pad;
      q.y = e + 1 < n ? in[e + 1] : pad;
      q.z = e + 2 < n ? in[e + 2] : pad;
      q.w = e + 3 < n ? in[e + 3] : pad;
      buf[rl * 8 + (j ^ (rl & 7))] = q;
    }
  };
#pragma unroll
  for (int j = 0; j < RPL; ++j) fill_partial(rl[j]);
  // ---- pass A: row totals (left folds)
  auto row_total = [&](int rl) {
    V tot = R::ident();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 q = buf[rl * 8 + (j ^ (rl & 7))];
      tot = op_elem<R>(tot, from_bits<T>(q.x));
      tot = op_elem<R>(tot, from_bits<T>(q.y));
      tot = op_elem<R>(tot, from_bits<T>(q.z));
      tot = op_elem<R>(tot, from_bits<T>(q.w));
    }
    return tot;
  };
  auto warp_incl = [&](V v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const V u = R::shfl_up(v, d, 32);
      if (lane >= d) v = R::op(u, v);
    }
    return v;
  };
  V pre[RPL], run = R::ident();  // run: the warp's earlier rows in all
#pragma unroll
  for (int j = 0; j < RPL; ++j) {
    const V ij = R::op(run, warp_incl(row_total(rl[j])));
    const V ej = R::shfl_up(ij, 1, 32);
    pre[j] = lane == 0 ? run : ej;
    run = R::shfl_idx(ij, 31, 32);
  }
  if (lane == 31) s_wtot[warp] = run;
  __syncthreads();
  if (warp == 0) {
    V total = R::ident();
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        s_cp[k] = total;
        total = R::op(total, s_wtot[k]);
      }
    }
    total = R::shfl_idx(total, 0, 32);
    bool gave_up;
    V prefix;
    const int64_t ngroups = (ntiles + 31) / 32;
    if constexpr (std::is_same<R, Plain<AddU>>::value) {
      // group descriptors and accumulators after the tile slots
      prefix = look_back_sum2(agg, inc + ntiles, inc + ntiles + ngroups, tile, ntiles, total, limit, status, gave_up);
    } else {
      // packed tile words in `inc`, exact aggregates in `agg`; after the tile
      // slots the group words (64-bit), then the group arrival counters
      uint64_t* gword = inc + ntiles;
      uint32_t* gcnt = reinterpret_cast<uint32_t*>(gword + ngroups);
      prefix = look_back_pk<R>(inc, agg, gword, gcnt, tile, ntiles, total, limit, status, gave_up);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) s_cp[k] = R::op(prefix, s_cp[k]);
      s_bad = gave_up;
    }
  }
  __syncthreads();
  if (s_bad) return;
  // ---- pass B: carry prefix op value through each row, in place
  auto carry_row = [&](int rl, V carry) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint4& slot = buf[rl * 8 + (j ^ (rl & 7))];
      uint4 q = slot;
      uint32_t* w = &q.x;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const V nx = op_elem<R>(carry, from_bits<T>(w[k]));
        w[k] = to_bits(R::out(excl ? carry : nx));
        carry = nx;
      }
      slot = q;
    }
  };
  const V cw = s_cp[warp];
#pragma unroll
  for (int j = 0; j < RPL; ++j) carry_row(rl[j], R::op(cw, pre[j]));
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0)
    for (int bx = 0; bx < nbox; ++bx) tma_store_2d(&tout, 0, (int)(r0 + bx * kGridBoxRows), buf + bx * kGridBoxRows * 8);
  auto store_partial = [&](int rl) {
    const int64_t row = r0 + rl;
    if (!(row == rows && rows * 32 < n)) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 q = buf[rl * 8 + (j ^ (rl & 7))];
      const int64_t e = row * 32 + 4 * j;
      if (e < n) out[e] = q.x;
      if (e + 1 < n) out[e + 1] = q.y;
      if (e + 2 < n) out[e + 2] = q.z;
      if (e + 3 < n) out[e + 3] = q.w;
    }
  };
#pragma unroll
  for (int j = 0; j < RPL; ++j) store_partial(rl[j]);
  if (tid == 0 && nbox > 0) tma_store_wait_read();  // the boxes have left shared memory
}

// BLOCK scope: the CTA is the logical block (persistent over blocks).
template <class R>
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int64_t n, int excl) {
  using T = typename R::T;
  using V = typename R::V;
  __shared__ V s_wt[32], s_wp[32];
  const int B = blockDim.x, nw = B >> 5, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nblk = (n + B - 1) / B;
  for (int64_t lb = blockIdx.x; lb < nblk; lb += gridDim.x) {
    const int64_t i = lb * B + tid;
    V v = R::load(i < n ? from_bits<T>(__ldcs(in + i)) : R::pad());
    {
      const V u = R::shfl_up_fresh(v, 1, 32);
      if (lane >= 1) v = R::op_fresh(u, v);
    }
#pragma unroll
    for (int d = 2; d < 32; d <<= 1) {
      const V u = R::shfl_up(v, d, 32);
      if (lane >= d) v = R::op(u, v);
    }
    if (lane == 31) s_wt[warp] = v;
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the warp totals
      V w = lane < nw ? s_wt[lane] : R::ident();
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const V u = R::shfl_up(w, d, 32);
        if (lane >= d) w = R::op(u, w);
      }
      const V ex = R::shfl_up(w, 1, 32);
      s_wp[lane] = lane == 0 ? R::ident() : ex;
    }
    __syncthreads();
    const V incl = R::op(s_wp[warp], v);
    T y;
    if (!excl) {
      y = R::out(incl);
    } else {
      const V e = R::shfl_up(incl, 1, 32);
      y = R::out(lane == 0 ? s_wp[warp] : e);
    }
    if (i < n) out[i] = to_bits(y);
    __syncthreads();
  }
}

struct ScanWs {
  unsigned* ticket;
  uint32_t* flags;
  uint64_t* agg;
  uint64_t* inc;
};

inline size_t scan_ws_bytes(int64_t ntiles) {
  const size_t f = ((size_t)ntiles * 4 + 255) & ~(size_t)255;
  return kScanWsHeader + f + 2 * (size_t)ntiles * 8;
}

inline ScanWs scan_ws(void* ws, int64_t ntiles) {
  char* p = static_cast<char*>(ws);
  ScanWs w;
  w.ticket = reinterpret_cast<unsigned*>(p);
  w.flags = reinterpret_cast<uint32_t*>(p + kScanWsHeader);
  const size_t f = ((size_t)ntiles * 4 + 255) & ~(size_t)255;
  w.agg = reinterpret_cast<uint64_t*>(p + kScanWsHeader + f);
  w.inc = w.agg + ntiles;
  return w;
}

template <class R>
static cox_status launch_scan_scope(cox_scope scope, int block, const void* d_in, void* d_out, int64_t n, int excl,
                                    void* ws, size_t ws_bytes, cudaStream_t st) {
  const uint32_t* in = static_cast<const uint32_t*>(d_in);
  uint32_t* out = static_cast<uint32_t*>(d_out);
  if (scope == COX_SCOPE_BLOCK) {
    auto k = k_scan_block<R>;
    static int gmax[33];
    int& g = gmax[block / 32];
    if (g == 0) g = persistent_grid(k, block, 0, 1 << 30);
    const int64_t nblk = (n + block - 1) / block;
    k<<<(int)(nblk < g ? nblk : g), block, 0, st>>>(in, out, n, excl);
    return launch_status();
  }
  if (n >= 32 && n / 32 < (int64_t(1) << 31) && aligned16(d_in) && aligned16(d_out)) {
    constexpr int RPL = grid_rows_rpl<R>();
    constexpr int64_t kTileElems = (int64_t)RPL * kGridBoxRows * 32;
    const int64_t ntiles = (n + kTileElems - 1) / kTileElems;
    const size_t need = scan_ws_bytes(ntiles) + 24 * (size_t)((ntiles + 31) / 32);  // + group words
    if (!ws || ws_bytes < need) return COX_ENOMEM;
    if (!aligned16(ws)) return COX_EINVAL;
    CUtensorMap tin, tout;
    if (!encode_rows32_map(&tin, d_in, n / 32, kGridBoxRows) || !encode_rows32_map(&tout, d_out, n / 32, kGridBoxRows))
      return COX_ECUDA;
    if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) return COX_ECUDA;
    const ScanWs w = scan_ws(ws, ntiles);
    auto k = k_scan_grid_rows<R, RPL>;
    const size_t smem = (size_t)RPL * kGridBoxRows * 128 + 1024;
    static bool attr[kMaxDevices];  // per device
    if (!attr[device_index()]) {
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COX_ECUDA;
      attr[device_index()] = true;
    }
    k<<<(unsigned)ntiles, 256, smem, st>>>(tin, tout, in, out, n, w.ticket, w.flags, w.agg, w.inc, ntiles, excl,
                                           spin_limit(), device_status_word());
    return launch_status();
  }
  constexpr int TILE = grid_scan_tile<R>();
  const int64_t ntiles = (n + TILE - 1) / TILE;
  if (ntiles > 0xFFFFFFFFll) return COX_EUNSUPPORTED;
  const size_t need = scan_ws_bytes(ntiles);
  if (!ws || ws_bytes < need) return COX_ENOMEM;
  if (!aligned16(ws)) return COX_EINVAL;
  if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) return COX_ECUDA;
  const ScanWs w = scan_ws(ws, ntiles);
  auto k = k_scan_grid<R>;
  const size_t smem = (size_t)TILE * 4 * (R::kComp ? 2 : 1) + 16;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return COX_ECUDA;
  k<<<(unsigned)ntiles, 256, smem, st>>>(in, out, n, w.ticket, w.flags, w.agg, w.inc, ntiles, excl, spin_limit(),
                                         device_status_word(), aligned16(d_in));
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_scan_workspace(cox_scope scope, int64_t n) {
  if (scope != COX_SCOPE_GRID || n <= 0) return 0;
  const int64_t t = (n + 8191) / 8192;  // enough for either tile size, plus group words
  return scan_ws_bytes(t) + 24 * (size_t)((t + 31) / 32);
}

extern "C" cox_status cox_scan(cox_op op, cox_dtype dt, cox_scope scope, int block_dim, const void* d_in, void* d_out,
                               int64_t n, unsigned flags, int exclusive, void* d_workspace, size_t workspace_bytes,
                               void* stream) {
  if (scope != COX_SCOPE_BLOCK && scope != COX_SCOPE_GRID) return COX_EINVAL;
  if (!valid_block(block_dim) || n < 0 || (exclusive != 0 && exclusive != 1)) return COX_EINVAL;
  if (flags & ~(unsigned)COX_F_COMPENSATED) return COX_EINVAL;
  if (n > 0 && (!d_in || !d_out)) return COX_EINVAL;
  const bool comp = flags & COX_F_COMPENSATED;
  return with_reducer(op, dt, comp, [&](auto r) {
    using R = decltype(r);
    if (n == 0) return COX_OK;
    return launch_scan_scope<R>(scope, block_dim, d_in, d_out, n, exclusive, d_workspace, workspace_bytes,
                                as_stream(stream));
  });
}
