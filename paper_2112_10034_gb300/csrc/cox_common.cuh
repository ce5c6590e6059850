// Internal helpers shared by the libcox kernels: reducer types, the staging
// layer that moves warp chunks between HBM and registers, and host dispatch.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "cox.h"

namespace cox {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------ device basics
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t to_bits(uint32_t v) { return v; }
__device__ __forceinline__ uint32_t to_bits(int32_t v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t to_bits(float v) { return __float_as_uint(v); }

template <class T>
__device__ __forceinline__ T from_bits(uint32_t u);
template <>
__device__ __forceinline__ uint32_t from_bits<uint32_t>(uint32_t u) { return u; }
template <>
__device__ __forceinline__ int32_t from_bits<int32_t>(uint32_t u) { return (int32_t)u; }
template <>
__device__ __forceinline__ float from_bits<float>(uint32_t u) { return __uint_as_float(u); }

// Knuth's TwoSum: s = fl(a + b), t = (a + b) - s exactly, for any |a|, |b|
// (Ogita, Rump & Oishi 2005, Alg. 3.1).  The _rn intrinsics are never fused.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// ----------------------------------------------------------------- reducers
// A reducer R names the element type T in memory, the register value V, the
// identity, the combine `op(a, b)`, and how V moves through a shuffle.  For
// integer ops `redux32` gives the full-warp reduction by redux.sync.

struct AddU {
  using T = uint32_t;
  __device__ static T ident() { return 0u; }
  __device__ static T op(T a, T b) { return a + b; }
  __device__ static T redux(T v) { return __reduce_add_sync(kFull, v); }
};
struct AndU {
  using T = uint32_t;
  __device__ static T ident() { return 0xFFFFFFFFu; }
  __device__ static T op(T a, T b) { return a & b; }
  __device__ static T redux(T v) { return __reduce_and_sync(kFull, v); }
};
struct OrU {
  using T = uint32_t;
  __device__ static T ident() { return 0u; }
  __device__ static T op(T a, T b) { return a | b; }
  __device__ static T redux(T v) { return __reduce_or_sync(kFull, v); }
};
struct XorU {
  using T = uint32_t;
  __device__ static T ident() { return 0u; }
  __device__ static T op(T a, T b) { return a ^ b; }
  __device__ static T redux(T v) { return __reduce_xor_sync(kFull, v); }
};
struct MinI {
  using T = int32_t;
  __device__ static T ident() { return 0x7FFFFFFF; }
  __device__ static T op(T a, T b) { return min(a, b); }
  __device__ static T redux(T v) { return __reduce_min_sync(kFull, v); }
};
struct MaxI {
  using T = int32_t;
  __device__ static T ident() { return (int32_t)0x80000000; }
  __device__ static T op(T a, T b) { return max(a, b); }
  __device__ static T redux(T v) { return __reduce_max_sync(kFull, v); }
};
struct MinU {
  using T = uint32_t;
  __device__ static T ident() { return 0xFFFFFFFFu; }
  __device__ static T op(T a, T b) { return min(a, b); }
  __device__ static T redux(T v) { return __reduce_min_sync(kFull, v); }
};
struct MaxU {
  using T = uint32_t;
  __device__ static T ident() { return 0u; }
  __device__ static T op(T a, T b) { return max(a, b); }
  __device__ static T redux(T v) { return __reduce_max_sync(kFull, v); }
};
struct AddF {
  using T = float;
  __device__ static T ident() { return 0.0f; }
  __device__ static T op(T a, T b) { return __fadd_rn(a, b); }
};
struct MinF {
  using T = float;
  __device__ static T ident() { return __int_as_float(0x7F800000); }
  __device__ static T op(T a, T b) { return fminf(a, b); }
};
struct MaxF {
  using T = float;
  __device__ static T ident() { return __int_as_float(0xFF800000); }
  __device__ static T op(T a, T b) { return fmaxf(a, b); }
};

template <class Op>
struct has_redux {
  template <class U>
  static auto test(int) -> decltype(U::redux(typename U::T{}), std::true_type{});
  template <class>
  static std::false_type test(...);
  static constexpr bool value = decltype(test<Op>(0))::value;
};

// Plain reducer: V == T.
template <class Op>
struct Plain {
  using T = typename Op::T;
  using V = T;
  static constexpr bool kComp = false;
  static constexpr bool kRedux = has_redux<Op>::value;
  __device__ static V ident() { return Op::ident(); }
  __device__ static T pad() { return Op::ident(); }  // padding lanes' element
  __device__ static V load(T x) { return x; }
  __device__ static V op(V a, V b) { return Op::op(a, b); }
  __device__ static V shfl_down(V v, int d, int w) { return __shfl_down_sync(kFull, v, d, w); }
  __device__ static V shfl_up(V v, int d, int w) { return __shfl_up_sync(kFull, v, d, w); }
  __device__ static V shfl_idx(V v, int s, int w) { return __shfl_sync(kFull, v, s, w); }
  __device__ static V shfl_xor(V v, int m) { return __shfl_xor_sync(kFull, v, m); }
  // First step on freshly loaded values (nothing to carry): same as op/shfl_up.
  __device__ static V shfl_up_fresh(V v, int d, int w) { return shfl_up(v, d, w); }
  __device__ static V op_fresh(V a, V b) { return op(a, b); }
  __device__ static V redux32(V v) {
    if constexpr (kRedux) return Op::redux(v);
    else return v;
  }
  __device__ static T out(V v) { return v; }
  __device__ static float lo(V) { return 0.0f; }
};

// Compensated fp32 sum: a pair (s, e), (s1,e1) (+) (s2,e2) =
// (s, (e1 + e2) + t) with (s, t) = TwoSum(s1, s2).  Output fl(s + e); the low
// word `lo` makes out + lo == s + e exactly.
struct Pair {
  float s, e;
};
struct Comp {
  using T = float;
  using V = Pair;
  static constexpr bool kComp = true;
  static constexpr bool kRedux = false;
  __device__ static V ident() { return {0.0f, 0.0f}; }
  __device__ static T pad() { return 0.0f; }
  __device__ static V load(T x) { return {x, 0.0f}; }
  __device__ static V op(V a, V b) {
    V r;
    float t;
    two_sum(a.s, b.s, r.s, t);
    r.e = __fadd_rn(__fadd_rn(a.e, b.e), t);
    return r;
  }
  __device__ static V shfl_down(V v, int d, int w) {
    return {__shfl_down_sync(kFull, v.s, d, w), __shfl_down_sync(kFull, v.e, d, w)};
  }
  __device__ static V shfl_up(V v, int d, int w) {
    return {__shfl_up_sync(kFull, v.s, d, w), __shfl_up_sync(kFull, v.e, d, w)};
  }
  __device__ static V shfl_idx(V v, int s, int w) {
    return {__shfl_sync(kFull, v.s, s, w), __shfl_sync(kFull, v.e, s, w)};
  }
  __device__ static V shfl_xor(V v, int m) { return {__shfl_xor_sync(kFull, v.s, m), __shfl_xor_sync(kFull, v.e, m)}; }
  // First step on freshly loaded pairs, whose error words are all zero:
  // only s moves, and (u, 0) (+) (s, 0) = (fl(u + s), (0 + 0) + t) = (., t)
  // exactly, so the result equals op() bit for bit.
  __device__ static V shfl_up_fresh(V v, int d, int w) { return {__shfl_up_sync(kFull, v.s, d, w), 0.0f}; }
  __device__ static V op_fresh(V a, V b) {
    V r;
    two_sum(a.s, b.s, r.s, r.e);
    return r;
  }
  __device__ static V redux32(V v) { return v; }
  __device__ static T out(V v) { return __fadd_rn(v.s, v.e); }
  __device__ static float lo(V v) {
    float y, l;
    two_sum(v.s, v.e, y, l);
    return l;
  }
};

// Width-W shfl_down tree (Code 1 generalised): the tile's rank-0 lane ends
// with the tile's value.  Integer reducers at W == 32 use redux.sync, which
// gives every lane the same (exact) value.
template <class R, int W>
__device__ __forceinline__ typename R::V tile_tree(typename R::V v) {
  if constexpr (W == 32 && R::kRedux) {
    return R::redux32(v);
  } else {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v = R::op(v, R::shfl_down(v, off, W));
    return v;
  }
}

// Block reduction in the order of the BLOCK scope: width-32 tree per warp,
// warp partials to shared memory, warp 0 lane l folds partials l, l+32, ...
// then a width-32 tree.  The result is valid in thread 0; `wpart` holds 32
// values.  Contains two __syncthreads (all threads must call it).
template <class R>
__device__ __forceinline__ typename R::V block_reduce32(typename R::V v, typename R::V* wpart) {
  using V = typename R::V;
  v = tile_tree<R, 32>(v);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (lane == 0) wpart[warp] = v;
  __syncthreads();
  V acc = R::ident();
  if (warp == 0) {
    for (int k = lane; k < (int)(blockDim.x >> 5); k += 32) acc = R::op(acc, wpart[k]);
    acc = tile_tree<R, 32>(acc);
  }
  __syncthreads();
  return acc;
}

// Peer mask of __match_any_sync(full, key) among the lanes with `in` set,
// for keys that fit in BITS bits, built from BITS + 1 warp ballots: two lanes
// hold the same key exactly when they agree on every bit.  On sm_103a the
// match.sync instruction costs roughly 40 SM cycles per warp instruction and
// grows with the number of distinct keys, while a ballot is a plain vote, so
// this form is the fast one for histogram-sized keys.  Lanes without `in`
// get an arbitrary mask and must not use it.
template <int BITS>
__device__ __forceinline__ unsigned match_any_bits(uint32_t key, bool in) {
  unsigned peers = __ballot_sync(kFull, in);
#pragma unroll
  for (int i = 0; i < BITS; ++i) {
    const bool b = (key >> i) & 1u;
    const unsigned m = __ballot_sync(kFull, b);
    peers &= b ? m : ~m;
  }
  return peers;
}

// Match-histogram step for NK keys per lane with peer groups from a table
// in shared memory (S tables per round, all zero at the kernel's start).  In
// a round every in-range lane ORs its lane bit into its key's word of its
// tile; after a __syncwarp the words hold exactly the masks __match_any_sync
// returns within each tile.  A lane whose OR found its word empty takes the
// mask with an atomic exchange that also clears it, and adds the mask's
// popcount to the key's bin.  Two layouts:
//   SPLIT   (hist_table_words(W, bins, true) words per table, S tables):
//           at width 32 a key's mask is split over two adjacent words --
//           lanes 0-15 OR into the first, lanes 16-31 into the second --
//           which halves the lanes that hit one address on a hot key (shared
//           atomics on one address are serialised); the first lane of each
//           half swaps the pair out as one 64-bit word, so the first swap
//           takes the whole mask and a later one finds zero and adds
//           nothing.  A second __syncwarp orders a round's exchanges before
//           the next round's ORs.
//   !SPLIT  (2 x SET tables of hist_table_words(W, bins, false) words): one
//           word per key and tile, and the rounds alternate between two sets
//           of SET tables (a round uses the first S of its set), so one
//           __syncwarp per round suffices: a round's ORs follow the previous
//           round's __syncwarp, which every lane reaches only after its
//           exchanges of the round before.
// Below width 32 every tile of the warp has its own words (word tile * bins
// + key), so one lane per peer group finds its word empty.
__host__ __device__ constexpr uint32_t hist_table_words(int W, uint32_t bins, bool split) {
  return W == 32 ? (split ? 2 : 1) * bins : (uint32_t)(32 / W) * bins;
}

template <int W, int S, int NK, bool SPLIT, int SET = S>
__device__ __forceinline__ void hist_peer_table(const uint32_t (&key)[NK], const bool (&in)[NK], uint32_t bins,
                                                uint32_t* my, uint32_t* tab, int& parity) {
  static_assert(NK % S == 0 && S <= SET, "S tables serve S keys per round; a set holds SET tables");
  constexpr bool kSplit = SPLIT && W == 32;
  const int lane = lane_id();
  const uint32_t words = hist_table_words(W, bins, SPLIT);
#pragma unroll
  for (int q0 = 0; q0 < NK; q0 += S) {
    uint32_t* t = tab;
    if constexpr (!SPLIT) {
      t += (uint32_t)parity * SET * words;
      parity ^= 1;
    }
    uint32_t old[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const uint32_t w = kSplit ? 2 * key[q0 + s] + (uint32_t)(lane >> 4) : (uint32_t)(lane / W) * bins + key[q0 + s];
      old[s] = in[q0 + s] ? atomicOr(t + s * words + w, 1u << lane) : 1u;
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (old[s] == 0u) {
        uint32_t c;
        if constexpr (kSplit) {
          unsigned long long* pair = reinterpret_cast<unsigned long long*>(t + s * words + 2 * key[q0 + s]);
          c = (uint32_t)__popcll(atomicExch(pair, 0ull));
        } else {
          c = (uint32_t)__popc(atomicExch(t + s * words + (uint32_t)(lane / W) * bins + key[q0 + s], 0u));
        }
        if (c) atomicAdd(my + key[q0 + s], c);
      }
    }
    if constexpr (SPLIT) __syncwarp();
  }
}

// ------------------------------------------------------------ staging layer
// A warp chunk is ROWS rows of 32 consecutive 32-bit elements; after loading,
// lane l holds row[r] = element base + 32 r + l (the paper's lane numbering:
// element i is the operand of global thread i).  Full chunks move as 128-bit
// (ROWS >= 4), 64-bit (ROWS == 2) or 32-bit (ROWS == 1) coalesced accesses
// and are transposed through a warp-private shared-memory buffer of ROWS*32
// words; partial chunks use 32-bit accesses with padding.

template <int ROWS>
__device__ __forceinline__ void load_rows_full(const uint32_t* __restrict__ g, uint32_t* sm,
                                               uint32_t (&row)[ROWS]) {
  const int lane = lane_id();
  if constexpr (ROWS >= 4) {
    constexpr int NV = ROWS / 4;
    uint4 v[NV];
    const uint4* src = reinterpret_cast<const uint4*>(g);
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = __ldcs(src + j * 32 + lane);
#pragma unroll
    for (int j = 0; j < NV; ++j) reinterpret_cast<uint4*>(sm)[j * 32 + lane] = v[j];
  } else if constexpr (ROWS == 2) {
    const uint2 v = __ldcs(reinterpret_cast<const uint2*>(g) + lane);
    reinterpret_cast<uint2*>(sm)[lane] = v;
  } else {
    row[0] = __ldcs(g + lane);
    return;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < ROWS; ++r) row[r] = sm[r * 32 + lane];
  __syncwarp();
}

template <int ROWS>
__device__ __forceinline__ void load_rows_tail(const uint32_t* __restrict__ g, int64_t avail,
                                               uint32_t pad, uint32_t (&row)[ROWS]) {
  const int lane = lane_id();
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = (int64_t)r * 32 + lane;
    row[r] = i < avail ? g[i] : pad;
  }
}

template <int ROWS>
__device__ __forceinline__ void store_rows_full(uint32_t* __restrict__ g, uint32_t* sm,
                                                const uint32_t (&row)[ROWS]) {
  const int lane = lane_id();
  if constexpr (ROWS == 1) {
    __stcs(g + lane, row[0]);
    return;
  } else {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) sm[r * 32 + lane] = row[r];
    __syncwarp();
    if constexpr (ROWS >= 4) {
#pragma unroll
      for (int j = 0; j < ROWS / 4; ++j)
        __stcs(reinterpret_cast<uint4*>(g) + j * 32 + lane, reinterpret_cast<const uint4*>(sm)[j * 32 + lane]);
    } else {
      __stcs(reinterpret_cast<uint2*>(g) + lane, reinterpret_cast<const uint2*>(sm)[lane]);
    }
    __syncwarp();
  }
}

template <int ROWS>
__device__ __forceinline__ void store_rows_tail(uint32_t* __restrict__ g, int64_t avail,
                                                const uint32_t (&row)[ROWS]) {
  const int lane = lane_id();
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = (int64_t)r * 32 + lane;
    if (i < avail) g[i] = row[r];
  }
}

// ------------------------------------------------------------ tile scan body
// One warp chunk (ROWS x 32 elements starting at element c * ROWS * 32) of
// the tile inclusive scan: Hillis-Steele steps d = 1, 2, .., W/2 of
// u = shfl_up(x, d, W); if (rank >= d) x = u op x, ROWS independent rows.
// `sm` is the warp's ROWS*32-word staging buffer; `vec` says whether full
// chunks may use vector accesses (16-byte aligned in and out).
template <class R, int W, int ROWS>
__device__ __forceinline__ void scan_chunk(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                                           int64_t c, uint32_t* sm, bool vec) {
  using T = typename R::T;
  using V = typename R::V;
  constexpr int64_t CH = ROWS * 32;
  const int rank = lane_id() & (W - 1);
  const int64_t base = c * CH;
  const bool full = vec && base + CH <= n;
  uint32_t row[ROWS];
  if (full) load_rows_full<ROWS>(in + base, sm, row);
  else load_rows_tail<ROWS>(in + base, n - base, to_bits(R::pad()), row);
  V v[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) v[r] = R::load(from_bits<T>(row[r]));
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {  // d = 1 on fresh values
    const V u = R::shfl_up_fresh(v[r], 1, W);
    if (rank >= 1) v[r] = R::op_fresh(u, v[r]);
  }
#pragma unroll
  for (int d = 2; d < W; d <<= 1) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const V u = R::shfl_up(v[r], d, W);
      if (rank >= d) v[r] = R::op(u, v[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) row[r] = to_bits(R::out(v[r]));
  if (full) store_rows_full<ROWS>(out + base, sm, row);
  else store_rows_tail<ROWS>(out + base, n - base, row);
}

// ------------------------------------------------- device status + waits
// Bit flags of the device-side status word read by cox_device_status().
enum : unsigned { kDevTimeout = 1u };

// Defined in api.cu (relocatable device code is not used: each kernel file
// reaches the word through this accessor, which api.cu implements).
__host__ unsigned* device_status_word();
__host__ uint32_t spin_limit();

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------- TMA bulk copies and mbarriers
// One-dimensional bulk copies (cp.async.bulk) from global into shared memory,
// completing on an mbarrier in shared memory.  Callers guarantee 16-byte
// aligned source and destination and a byte count that is a multiple of 16.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes initialised mbarriers visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival (release semantics at CTA scope: the arriving thread's earlier
// writes, and those it has observed, are visible to a thread whose wait sees
// the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bulk copy from shared memory to global memory (TMA store), tracked by the
// issuing thread's bulk async-group.  Threads that wrote the source with
// ordinary stores must each run fence_proxy_async_smem() and then meet at a
// barrier before one thread issues the copy.
__device__ __forceinline__ void tma_store_1d(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the issuing thread's bulk stores have read their shared-memory
// source (the buffer may be reused), or have completed entirely.
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Two-dimensional tiled TMA through a tensor map (a __grid_constant__ kernel
// parameter).  The innermost coordinate x is always 0 here (16-byte aligned);
// rows past the tensor's end read as 0 and are not written.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until at most one of the issuing thread's bulk stores still reads
// shared memory.
__device__ __forceinline__ void tma_store_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// True once the phase with the given parity has completed; a thread whose
// phase is still open is suspended for up to 1 us before the answer.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}
// Bounded wait: at most `limit` polls (try_wait itself suspends briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i <= limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// --------------------------------------------------- per-warp row ring
// Streams chunks of 32 rows x 32 elements (4 KB) of a tensor map built by
// encode_rows32_map (box 32 x 32) through a ring of kRingStages buffers per
// warp, two chunks in flight while one is processed.  Warp `gw` of `nw` takes
// chunks gw, gw + nw, ...; for each, lane 0 has armed the slot's mbarrier and
// issued the 2D TMA load, every lane waits (bounded), then
//   body(c, buf)  reads the chunk (row r at uint4 r*8, its unit j at unit
//                 j ^ (r & 7)) and, when STORE, leaves its results there;
// with STORE the ring writes the buffer back through `tout` by TMA store and
// refills a slot only after the previous store has read it.  Chunks past the
// tensor's last row read as 0 and are not stored.  A load that does not land
// within `limit` polls records kDevTimeout, gives the copies in flight a
// bounded wait and ends the warp's loop.  CTAs are kRingWarps warps.
constexpr int kRingStages = 3;
constexpr int kRingWarps = 8;
constexpr uint32_t kRingChunkBytes = 32 * 32 * 4;
constexpr size_t kRingSmem = (size_t)kRingWarps * kRingStages * kRingChunkBytes + 1024 + kRingWarps * kRingStages * 8;

template <bool STORE, class Body>
__device__ __forceinline__ void row_ring(const CUtensorMap* tin, const CUtensorMap* tout, int64_t nch, uint32_t limit,
                                         unsigned* status, Body&& body) {
  extern __shared__ uint8_t ring_smem_raw[];
  uint8_t* base =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ring_smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* ring = base + (size_t)warp * kRingStages * kRingChunkBytes;
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(base + (size_t)kRingWarps * kRingStages * kRingChunkBytes) + warp * kRingStages;
  const int64_t gw = (int64_t)blockIdx.x * kRingWarps + warp, nw = (int64_t)gridDim.x * kRingWarps;
  if (lane == 0) {
    for (int k = 0; k < kRingStages; ++k) mbar_init(bars + k, 1);
    mbar_init_fence();
    for (int k = 0; k < kRingStages - 1; ++k) {
      const int64_t c = gw + k * nw;
      if (c < nch) {
        mbar_arrive_expect_tx(bars + k, kRingChunkBytes);
        tma_load_2d(ring + k * kRingChunkBytes, tin, 0, (int)(c * 32), bars + k);
      }
    }
  }
  __syncwarp();
  bool ok = true;
  int64_t k = 0;
  for (int64_t c = gw; c < nch; c += nw, ++k) {
    const int slot = (int)(k % kRingStages);
    uint4* buf = reinterpret_cast<uint4*>(ring + slot * kRingChunkBytes);
    ok = mbar_wait_bounded(bars + slot, (uint32_t)((k / kRingStages) & 1), limit);
    if (!__all_sync(kFull, ok)) {
      ok = false;
      break;
    }
    body(c, buf);
    fence_proxy_async_smem();  // this lane's accesses to the buffer, before the async proxy's
    __syncwarp();
    if (lane == 0) {
      if constexpr (STORE) tma_store_2d(tout, 0, (int)(c * 32), buf);
      const int64_t cn = c + (kRingStages - 1) * nw;  // refill the previous chunk's slot
      if (cn < nch) {
        const int ns = (int)((k + kRingStages - 1) % kRingStages);
        if constexpr (STORE) tma_store_wait_read1();  // the previous chunk's store has read it
        mbar_arrive_expect_tx(bars + ns, kRingChunkBytes);
        tma_load_2d(ring + ns * kRingChunkBytes, tin, 0, (int)(cn * 32), bars + ns);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (!ok) {
      atomicOr(status, 1u);  // kDevTimeout
      for (int j = 0; j < kRingStages - 1; ++j) {
        const int64_t kk = k + j;
        if (gw + kk * nw < nch)
          mbar_wait_bounded(bars + (int)(kk % kRingStages), (uint32_t)((kk / kRingStages) & 1), limit);
      }
    }
    if constexpr (STORE) tma_store_wait_all();
  }
  __syncwarp();
}

// ------------------------------------------------ one tile row per lane
// The same Hillis-Steele combines with each width-W tile collapsed into one
// thread -- the paper's intra-warp loop (Section 2.3, Code 3), applied on
// the GPU: lane t of a warp holds row t (32 consecutive elements, 32/W
// tiles) of the warp's 1024-element chunk, and step d sets
// x[i] = x[i-d] op x[i] for rank i from W-1 down to d, so x[i-d] still holds
// the previous step's value, exactly as the shuffle's source lane does.
// Same operands in the same order, hence the same bits, with no shuffles,
// selects or idle lanes.
template <class R, int W>
__device__ __forceinline__ void scan_row_regs(typename R::V (&v)[32]) {
#pragma unroll
  for (int t0 = 0; t0 < 32; t0 += W) {
#pragma unroll
    for (int i = W - 1; i >= 1; --i) v[t0 + i] = R::op_fresh(v[t0 + i - 1], v[t0 + i]);
#pragma unroll
    for (int d = 2; d < W; d <<= 1)
#pragma unroll
      for (int i = W - 1; i >= d; --i) v[t0 + i] = R::op(v[t0 + i - d], v[t0 + i]);
  }
}

// ------------------------------------------------------------ host helpers
// The driver's tensor-map encoder (looked up once; null if unavailable).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  return encode;
}

// Tensor map of a 32-bit array viewed as `rows` rows of 32 elements (128 B),
// boxes of 32 x `box_rows`, 128-byte swizzle: in shared memory the 16-byte
// unit j of row r sits at unit j ^ (r & 7) of the row (conflict-free
// per-lane row reads).  `base` must be 16-byte aligned; 1 <= rows < 2^31.
inline bool encode_rows32_map(CUtensorMap* map, const void* base, int64_t rows, int box_rows) {
  const auto encode = tensor_map_encoder();
  if (!encode) return false;
  const cuuint64_t dims[2] = {32, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline bool valid_width(int w) { return w == 2 || w == 4 || w == 8 || w == 16 || w == 32; }
inline bool valid_block(int b) { return b >= 32 && b <= 1024 && b % 32 == 0; }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int sm_count();  // of the current device (cached per device)
constexpr int kMaxDevices = 64;  // per-device caches hold this many ordinals
int device_index();  // the current device's ordinal, clamped into [0, kMaxDevices)

inline cox_status launch_status() {
  return cudaGetLastError() == cudaSuccess ? COX_OK : COX_ECUDA;
}

// Calls f(Reducer{}) for the reducer of (op, dt, compensated).
template <class F>
cox_status with_reducer(cox_op op, cox_dtype dt, bool comp, F&& f) {
  if (comp) {
    if (dt != COX_F32 || op != COX_SUM) return COX_EINVAL;
    return f(Comp{});
  }
  if (dt == COX_F32) {
    switch (op) {
      case COX_SUM: return f(Plain<AddF>{});
      case COX_MIN: return f(Plain<MinF>{});
      case COX_MAX: return f(Plain<MaxF>{});
      default: return COX_EINVAL;
    }
  }
  if (dt != COX_I32 && dt != COX_U32) return COX_EINVAL;
  switch (op) {
    case COX_SUM: return f(Plain<AddU>{});
    case COX_AND: return f(Plain<AndU>{});
    case COX_OR: return f(Plain<OrU>{});
    case COX_XOR: return f(Plain<XorU>{});
    case COX_MIN: return dt == COX_I32 ? f(Plain<MinI>{}) : f(Plain<MinU>{});
    case COX_MAX: return dt == COX_I32 ? f(Plain<MaxI>{}) : f(Plain<MaxU>{});
    default: return COX_EINVAL;
  }
}

template <class F>
cox_status with_width(int w, F&& f) {
  switch (w) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    default: return COX_EINVAL;
  }
}

// Persistent-grid size for a kernel: resident CTAs per SM (occupancy query,
// cached by the caller) x SMs, capped by the work available.
template <class K>
int persistent_grid(K kernel, int block, size_t dyn_smem, int64_t work_ctas) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, dyn_smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int64_t g = (int64_t)per_sm * sm_count();
  if (work_ctas < g) g = work_ctas;
  return g < 1 ? 1 : (int)g;
}

}  // namespace cox
