// Batched uneven arrays: per array a compensated fp32 sum and a 256-bin
// histogram built from match_any peer groups, all arrays in one persistent
// launch.
//
// Work split.  The arrays are laid end to end in a virtual index space of E
// elements (prefix sums of the lengths, written once by cox_batch_prepare).
// Persistent CTA i of G owns the element range [i*E/G, (i+1)*E/G): every CTA
// streams the same number of bytes whatever the length mix (32 .. 2^20 here),
// so there is no tail of idle CTAs and no work queue to contend on.  A CTA
// walks its range array by array; each (array, CTA) piece is a segment.
//
// Per segment: every thread folds its elements into a TwoSum-compensated
// pair in a fixed order, the block reduces the pairs (shfl_down trees, then
// warp 0) and stores one pair at slot a + i -- slots are unique and, for one
// array, consecutive in CTA order -- and the per-warp match_any histograms
// are flushed into the array's 256 bins with global atomics (exact integers).
// A second small kernel folds each array's pairs in CTA order, in FP64 when
// the array spans at least `fp64_segments` CTAs.  Every result depends only on
// the data, E and G: never on timing or on the order CTAs run in.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cox_common.cuh"

namespace cox {

constexpr int kBatchBins = 256;
constexpr int kBatchMaxCtas = 4096;
constexpr size_t kBatchHeader = 256;
constexpr cox_batch_tune kDefaultTune = {512, 2, 32, 8, 3, 8};
constexpr size_t kBatchSmemPerSm = 220 * 1024;  // dynamic shared memory the CTAs of one SM may take

__host__ __device__ __forceinline__ int64_t cta_begin(int64_t i, int64_t E, int64_t G) {
  return (int64_t)(((uint64_t)i * (uint64_t)E) / (uint64_t)G);
}

// CTA whose range holds virtual index pos (0 <= pos < E): the largest i with
// cta_begin(i) <= pos.
__device__ __forceinline__ int64_t cta_of(int64_t pos, int64_t E, int64_t G) {
  return (int64_t)((((uint64_t)pos + 1) * (uint64_t)G + (uint64_t)E - 1) / (uint64_t)E) - 1;
}

// Histogram step of one warp: peers among the lane's width-W tile with the
// same in-range key; one lane of each peer group adds the group's size to
// the warp's bins.  PEER: 0 the match_any mask from 9 ballots over the key
// bits, 1 the match.any.sync instruction, 3 per-warp tables of masks in
// shared memory (hist_peer_table: lanes OR their bit into their key's word;
// the lane that found it empty takes the mask and clears the word) -- the
// same mask every way; 2 no peer groups (one shared atomic per key; same
// counts).
template <int W, int PEER, int S>
__device__ __forceinline__ void batch_hist_step(uint32_t key, bool valid, uint32_t* my, uint32_t* tab, int& parity) {
  const int lane = lane_id();
  const bool in = valid && key < (uint32_t)kBatchBins;
  if constexpr (PEER == 2) {
    if (in) atomicAdd(my + key, 1u);
  } else if constexpr (PEER == 3 || PEER == 4) {
    const uint32_t k1[1] = {key};
    const bool in1[1] = {in};
    hist_peer_table<W, 1, 1, PEER == 4, S>(k1, in1, kBatchBins, my, tab, parity);  // the first table (of a set)
  } else {
    const unsigned tmask = W == 32 ? kFull : (((1u << W) - 1u) << (lane & ~(W - 1)));
    const unsigned lt = lanemask_lt();
    unsigned peers;
    if constexpr (PEER == 1) {
      peers = __match_any_sync(kFull, key) & __ballot_sync(kFull, in);
    } else {
      peers = match_any_bits<8>(key, in);
    }
    peers &= tmask;
    if (in && (peers & lt) == 0u) atomicAdd(my + key, (uint32_t)__popc(peers));
  }
}

// Four keys of one lane; S peer tables serve S keys per round (PEER 3).
template <int W, int PEER, int S>
__device__ __forceinline__ void batch_hist_quad(const uint32_t* key, const bool* ok, uint32_t* my, uint32_t* tab,
                                                int& parity) {
  if constexpr (PEER == 3 || PEER == 4) {
    uint32_t k4[4];
    bool in4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      k4[j] = key[j];
      in4[j] = ok[j] && key[j] < (uint32_t)kBatchBins;
    }
    hist_peer_table<W, S, 4, PEER == 4>(k4, in4, kBatchBins, my, tab, parity);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) batch_hist_step<W, PEER, S>(key[j], ok[j], my, tab, parity);
  }
}

__device__ __forceinline__ void fold(Pair& acc, float x) { acc = Comp::op(acc, Comp::load(x)); }

// One segment [s0, s1) of one array, all warps of the CTA.  Warp-uniform
// loops: every lane of a warp runs every match_any step (invalid lanes take
// part with valid = false).
template <int W, int PEER, int S, int H>
__device__ void batch_segment(const float* __restrict__ v, const int32_t* __restrict__ k, int64_t s0, int64_t s1,
                              Pair& acc, uint32_t* my, uint32_t* tab, int& parity) {
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uintptr_t pv = reinterpret_cast<uintptr_t>(v), pk = reinterpret_cast<uintptr_t>(k);
  // 128-bit loads need values and keys at the same phase modulo 16 bytes
  const bool al = ((pv ^ pk) & 15u) == 0 && (pv & 3u) == 0;
  if (!al) {  // scalar path: one element per lane per warp step
    for (int64_t q = s0 + (int64_t)warp * 32; q < s1; q += (int64_t)nw * 32) {
      const int64_t e = q + lane;
      const bool ok = e < s1;
      const float x = ok ? __ldcs(v + e) : 0.0f;
      const uint32_t key = ok ? (uint32_t)__ldcs(k + e) : 0u;
      if (ok) fold(acc, x);
      batch_hist_step<W, PEER, S>(key, ok, my, tab, parity);
    }
    return;
  }
  // 16-byte aligned body [vb, ve): element e is aligned when (e + phase) % 4 == 0
  const int64_t phase = (int64_t)((pv >> 2) & 3u);
  const int64_t vb = min(s1, s0 + ((4 - ((s0 + phase) & 3)) & 3));
  const int64_t ve = vb + ((s1 - vb) & ~(int64_t)3);
  if (warp == 0) {  // head [s0, vb) and tail [ve, s1): at most 3 + 3 elements
    const int h = (int)(vb - s0), t = (int)(s1 - ve);
    const int64_t e = lane < h ? s0 + lane : ve + (lane - h);
    const bool ok = lane < h + t;
    const float x = ok ? __ldcs(v + e) : 0.0f;
    const uint32_t key = ok ? (uint32_t)__ldcs(k + e) : 0u;
    if (ok) fold(acc, x);
    batch_hist_step<W, PEER, S>(key, ok, my, tab, parity);
  }
  // body: warp steps of 128 elements (one 128-bit load of values and of keys
  // per lane), H steps in flight (4H elements per thread per round: the tuned
  // "elements per thread"); a thread folds its elements in the same order for
  // every H
  const int64_t stride = (int64_t)nw * 128;
  for (int64_t q = vb + (int64_t)warp * 128; q < ve; q += H * stride) {
    float x[4 * H];
    uint32_t key[4 * H];
    bool ok[4 * H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int64_t e = q + h * stride + 4 * lane;
      if (e + 4 <= ve) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(v + e));
        const int4 b = __ldcs(reinterpret_cast<const int4*>(k + e));
        x[4 * h + 0] = a.x; x[4 * h + 1] = a.y; x[4 * h + 2] = a.z; x[4 * h + 3] = a.w;
        key[4 * h + 0] = b.x; key[4 * h + 1] = b.y; key[4 * h + 2] = b.z; key[4 * h + 3] = b.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[4 * h + j] = true;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ok[4 * h + j] = e + j < ve;
          x[4 * h + j] = ok[4 * h + j] ? __ldcs(v + e + j) : 0.0f;
          key[4 * h + j] = ok[4 * h + j] ? (uint32_t)__ldcs(k + e + j) : 0u;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4 * H; ++j)
      if (ok[j]) fold(acc, x[j]);
#pragma unroll
    for (int h = 0; h < H; ++h) batch_hist_quad<W, PEER, S>(key + 4 * h, ok + 4 * h, my, tab, parity);
  }
}

template <int W, int PEER, int S, int H>
__global__ void __launch_bounds__(1024) k_batch_sum_hist(const float* const* __restrict__ vals,
                                                         const int32_t* const* __restrict__ keys,
                                                         const int64_t* __restrict__ off, int64_t A,
                                                         float2* __restrict__ part, int32_t* __restrict__ hists) {
  extern __shared__ __align__(16) uint32_t sh[];  // (blockDim / 32) x 256 per-warp bins, then the peer tables
  __shared__ Pair wpart[32];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int ntab = PEER == 3   ? 2 * S * (int)hist_table_words(W, kBatchBins, false)  // two sets of S
                   : PEER == 4 ? S * (int)hist_table_words(W, kBatchBins, true)        // S split tables
                               : 0;  // peer tables per warp
  for (int i = threadIdx.x; i < nw * (kBatchBins + ntab); i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  uint32_t* tab = sh + nw * kBatchBins + warp * ntab;
  int parity = 0;
  const int64_t E = off[A];
  const int64_t G = gridDim.x;
  const int64_t lo = cta_begin(blockIdx.x, E, G), hi = cta_begin(blockIdx.x + 1, E, G);
  if (lo >= hi) return;
  // first array holding `lo`: the last a with off[a] <= lo
  int64_t a0 = 0, a1 = A;  // invariant: off[a0] <= lo < off[a1]
  while (a1 - a0 > 1) {
    const int64_t m = (a0 + a1) >> 1;
    if (off[m] <= lo) a0 = m;
    else a1 = m;
  }
  int64_t a = a0;
  uint32_t* my = sh + warp * kBatchBins;
  for (int64_t pos = lo; pos < hi; ++a) {
    while (off[a + 1] <= pos) ++a;  // skip empty arrays
    const int64_t base = off[a];
    const int64_t end = min(hi, off[a + 1]);
    Pair acc = Comp::ident();
    batch_segment<W, PEER, S, H>(vals[a], keys[a], pos - base, end - base, acc, my, tab, parity);
    const Pair s = block_reduce32<Comp>(acc, wpart);  // ends with __syncthreads
    if (threadIdx.x == 0) part[a + blockIdx.x] = make_float2(s.s, s.e);
    for (int b = threadIdx.x; b < kBatchBins; b += blockDim.x) {
      uint32_t c = 0;
      for (int w = 0; w < nw; ++w) {
        c += sh[w * kBatchBins + b];
        sh[w * kBatchBins + b] = 0u;
      }
      if (c) atomicAdd(hists + a * kBatchBins + b, (int32_t)c);
    }
    __syncthreads();
    pos = end;
  }
}

// Per array: fold its CTA pairs (slots a + first .. a + last) in CTA order.
__global__ void k_batch_combine(const int64_t* __restrict__ off, int64_t A, int G, const float2* __restrict__ part,
                                int fp64_segments, float* __restrict__ sums, double* __restrict__ sums64) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  const int64_t E = off[A];
  const int64_t b0 = off[a], b1 = off[a + 1];
  if (b1 <= b0) {
    sums[a] = 0.0f;
    if (sums64) sums64[a] = 0.0;
    return;
  }
  const int64_t first = cta_of(b0, E, G), last = cta_of(b1 - 1, E, G);
  if (last - first + 1 >= fp64_segments) {
    double d = 0.0;
    for (int64_t i = first; i <= last; ++i) {
      if (cta_begin(i, E, G) == cta_begin(i + 1, E, G)) continue;  // empty range, never written
      const float2 p = part[a + i];
      d += (double)p.x + (double)p.y;
    }
    sums[a] = (float)d;
    if (sums64) sums64[a] = d;
    return;
  }
  Pair acc = Comp::ident();
  for (int64_t i = first; i <= last; ++i) {
    if (cta_begin(i, E, G) == cta_begin(i + 1, E, G)) continue;
    const float2 p = part[a + i];
    acc = Comp::op(acc, Pair{p.x, p.y});
  }
  sums[a] = Comp::out(acc);
  if (sums64) sums64[a] = (double)acc.s + (double)acc.e;
}

bool tune_ok(const cox_batch_tune& t) {
  return t.block_dim >= 64 && t.block_dim <= 1024 && t.block_dim % 32 == 0 && t.ctas_per_sm >= 1 &&
         t.ctas_per_sm <= 8 && valid_width(t.width) && t.fp64_segments >= 1 &&
         (t.native_match >= 0 && t.native_match <= 4) && (t.ept == 4 || t.ept == 8 || t.ept == 16);
}

struct BatchWs {
  int64_t* off;
  float2* part;
};

BatchWs batch_layout(void* ws, int64_t A) {
  char* p = static_cast<char*>(ws) + kBatchHeader;
  BatchWs w;
  w.off = reinterpret_cast<int64_t*>(p);
  const size_t off_bytes = ((size_t)(A + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
  w.part = reinterpret_cast<float2*>(p + off_bytes);
  return w;
}

template <int W, int PEER, int S, int H>
cox_status launch_batch1(int G, int block_dim, size_t smem, cudaStream_t st, const float* const* d_vals,
                         const int32_t* const* d_keys, const BatchWs& w, int64_t num_arrays, int32_t* d_hists) {
  auto k = k_batch_sum_hist<W, PEER, S, H>;
  static size_t attr[kMaxDevices];  // per device: the dynamic shared size this kernel may take so far
  size_t& a = attr[device_index()];
  if (smem > a) {  // (static shared memory counts against the 48 KB default too)
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return COX_ECUDA;
    a = smem;
  }
  k<<<G, block_dim, smem, st>>>(d_vals, d_keys, w.off, num_arrays, w.part, d_hists);
  return launch_status();
}

// Elements per thread per round (4 per 128-bit step in flight): 4, 8 or 16.
template <int W, int PEER, int S>
cox_status launch_batch(int ept, int G, int block_dim, size_t smem, cudaStream_t st, const float* const* d_vals,
                        const int32_t* const* d_keys, const BatchWs& w, int64_t num_arrays, int32_t* d_hists) {
  if (ept == 4) return launch_batch1<W, PEER, S, 1>(G, block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
  if (ept == 16) return launch_batch1<W, PEER, S, 4>(G, block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
  return launch_batch1<W, PEER, S, 2>(G, block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_batch_workspace(int64_t num_arrays) {
  if (num_arrays < 0) return 0;
  const size_t off_bytes = ((size_t)(num_arrays + 1) * sizeof(int64_t) + 255) & ~(size_t)255;
  return kBatchHeader + off_bytes + (size_t)(num_arrays + kBatchMaxCtas) * sizeof(float2);
}

extern "C" cox_status cox_batch_prepare(int64_t num_arrays, const int64_t* h_lens, void* d_workspace,
                                        size_t workspace_bytes, void* stream) {
  if (num_arrays < 1 || !h_lens || !d_workspace) return COX_EINVAL;
  if (workspace_bytes < cox_batch_workspace(num_arrays)) return COX_ENOMEM;
  if (!aligned16(d_workspace)) return COX_EINVAL;
  std::vector<int64_t> off((size_t)num_arrays + 1);
  off[0] = 0;
  for (int64_t a = 0; a < num_arrays; ++a) {
    if (h_lens[a] < 0) return COX_EINVAL;
    off[a + 1] = off[a] + h_lens[a];
  }
  if (off[num_arrays] >= (int64_t(1) << 50)) return COX_EUNSUPPORTED;
  const BatchWs w = batch_layout(d_workspace, num_arrays);
  cudaStream_t st = as_stream(stream);
  if (cudaMemcpyAsync(w.off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return COX_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? COX_OK : COX_ECUDA;
}

extern "C" cox_status cox_batch_sum_hist(int64_t num_arrays, const float* const* d_vals, const int32_t* const* d_keys,
                                         const cox_batch_tune* tune, void* d_workspace, size_t workspace_bytes,
                                         float* d_sums, double* d_sums64, int32_t* d_hists, void* stream) {
  if (num_arrays < 1 || !d_vals || !d_keys || !d_workspace || !d_sums || !d_hists) return COX_EINVAL;
  if (workspace_bytes < cox_batch_workspace(num_arrays)) return COX_ENOMEM;
  const cox_batch_tune t = tune ? *tune : kDefaultTune;
  if (!tune_ok(t)) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  const BatchWs w = batch_layout(d_workspace, num_arrays);
  int G = sm_count() * t.ctas_per_sm;
  if (G > kBatchMaxCtas) G = kBatchMaxCtas;
  if (cudaMemsetAsync(d_hists, 0, (size_t)num_arrays * kBatchBins * sizeof(int32_t), st) != cudaSuccess)
    return COX_ECUDA;
  // per-warp bins, then the peer tables (two sets of S tables of
  // hist_table_words words per warp): four per set where that leaves room for
  // ctas_per_sm CTAs on an SM, else two, else one
  const size_t bins_bytes = (size_t)(t.block_dim / 32) * kBatchBins * sizeof(uint32_t);
  const size_t tab_bytes =  // per table round: one table of each of the two sets, or one split table
      (size_t)(t.block_dim / 32) *
      (t.native_match == 4 ? hist_table_words(t.width, kBatchBins, true)
                           : 2 * hist_table_words(t.width, kBatchBins, false)) *
      sizeof(uint32_t);
  // (tables that do not fit one SM at all: the same masks from ballots)
  const bool table = t.native_match == 3 || t.native_match == 4;
  const int peer = table && bins_bytes + tab_bytes > kBatchSmemPerSm ? 0 : t.native_match;
  int tables = 0;
  if (peer == 3 || peer == 4)
    for (tables = 4; tables > 1 && (bins_bytes + tables * tab_bytes) * (size_t)t.ctas_per_sm > kBatchSmemPerSm;)
      tables >>= 1;
  if (peer == 4 && tables > 2) tables = 2;  // (split tables: one or two per round)
  const size_t smem = bins_bytes + (size_t)tables * tab_bytes;
  const cox_status s = with_width(t.width, [&](auto wc) {
    constexpr int W = decltype(wc)::value;
    if (peer == 3 && tables == 4)
      return launch_batch<W, 3, 4>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 3 && tables == 2)
      return launch_batch<W, 3, 2>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 3) return launch_batch<W, 3, 1>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 4 && tables >= 2)
      return launch_batch<W, 4, 2>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 4) return launch_batch<W, 4, 1>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 1) return launch_batch<W, 1, 1>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    if (peer == 2) return launch_batch<W, 2, 1>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
    return launch_batch<W, 0, 1>(t.ept, G, t.block_dim, smem, st, d_vals, d_keys, w, num_arrays, d_hists);
  });
  if (s != COX_OK) return s;
  const int cb = 256;
  k_batch_combine<<<(unsigned)((num_arrays + cb - 1) / cb), cb, 0, st>>>(w.off, num_arrays, G, w.part,
                                                                        t.fp64_segments, d_sums, d_sums64);
  return launch_status();
}

// ------------------------------------------------------- one launch per array
// The baseline the batched launch is measured against: the same results from
// one compensated grid-scope reduction and one match histogram per array,
// launched back to back from this loop on one stream.
extern "C" size_t cox_batch_percall_scratch(int64_t max_len) {
  if (max_len < 1) return 0;
  return (cox_tile_reduce_workspace(COX_SCOPE_GRID, max_len, 256) + 255) & ~(size_t)255;
}

extern "C" cox_status cox_batch_percall(int64_t num_arrays, const float* const* h_vals, const int32_t* const* h_keys,
                                        const int64_t* h_lens, float* d_sums, int32_t* d_hists, void* d_scratch,
                                        size_t scratch_bytes, void* const* events, void* stream) {
  if (num_arrays < 1 || !h_vals || !h_keys || !h_lens || !d_sums || !d_hists || !d_scratch) return COX_EINVAL;
  int64_t max_len = 1;
  for (int64_t a = 0; a < num_arrays; ++a) {
    if (h_lens[a] < 0) return COX_EINVAL;
    max_len = std::max<int64_t>(max_len, h_lens[a]);
  }
  if (scratch_bytes < cox_batch_percall_scratch(max_len)) return COX_ENOMEM;
  cudaStream_t st = as_stream(stream);
  for (int64_t a = 0; a < num_arrays; ++a) {
    cox_status s = COX_OK;
    if (h_lens[a] == 0) {
      if (cudaMemsetAsync(d_sums + a, 0, sizeof(float), st) != cudaSuccess ||
          cudaMemsetAsync(d_hists + a * kBatchBins, 0, kBatchBins * sizeof(int32_t), st) != cudaSuccess)
        return COX_ECUDA;
    } else {
      s = cox_tile_reduce(COX_SUM, COX_F32, 32, 256, COX_SCOPE_GRID, h_vals[a], d_sums + a, h_lens[a],
                          COX_F_COMPENSATED, nullptr, d_scratch, scratch_bytes, stream);
      if (s == COX_OK)
        s = cox_match_histogram(COX_I32, 32, 256, h_keys[a], h_lens[a], kBatchBins, d_hists + a * kBatchBins,
                                nullptr, 0u, stream);
    }
    if (s != COX_OK) return s;
    if (events && events[a] && cudaEventRecord(static_cast<cudaEvent_t>(events[a]), st) != cudaSuccess)
      return COX_ECUDA;
  }
  return COX_OK;
}

// ------------------------------------------------------------------ graphs
struct cox_graph {
  cudaGraphExec_t exec = nullptr;
};

extern "C" cox_status cox_batch_graph_create(int64_t num_arrays, const float* const* d_vals,
                                             const int32_t* const* d_keys, const cox_batch_tune* tune,
                                             void* d_workspace, size_t workspace_bytes, float* d_sums,
                                             double* d_sums64, int32_t* d_hists, cox_graph** out) {
  if (!out) return COX_EINVAL;
  *out = nullptr;
  sm_count();  // device queries before capture
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return COX_ECUDA;
  cox_status st = COX_OK;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(s);
    return COX_ECUDA;
  }
  st = cox_batch_sum_hist(num_arrays, d_vals, d_keys, tune, d_workspace, workspace_bytes, d_sums, d_sums64, d_hists,
                          s);
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  cudaStreamDestroy(s);
  if (st != COX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess || !graph) return COX_ECUDA;
  cox_graph* g = new (std::nothrow) cox_graph;
  if (!g) {
    cudaGraphDestroy(graph);
    return COX_ENOMEM;
  }
  const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    delete g;
    return COX_ECUDA;
  }
  *out = g;
  return COX_OK;
}

extern "C" cox_status cox_graph_launch(cox_graph* g, void* stream) {
  if (!g || !g->exec) return COX_EINVAL;
  return cudaGraphLaunch(g->exec, as_stream(stream)) == cudaSuccess ? COX_OK : COX_ECUDA;
}

extern "C" void cox_graph_destroy(cox_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

// --------------------------------------------------------------- autotuner
namespace {

int log2_bucket(int64_t v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

std::string gpu_name() {
  int d = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&d) != cudaSuccess || cudaGetDeviceProperties(&p, d) != cudaSuccess) return "unknown";
  std::string n = p.name;
  for (char& c : n)
    if (c == '|' || c == '\n') c = '_';
  return n;
}

}  // namespace

extern "C" cox_status cox_batch_autotune(int64_t num_arrays, const float* const* d_vals,
                                         const int32_t* const* d_keys, void* d_workspace, size_t workspace_bytes,
                                         float* d_sums, int32_t* d_hists, int reps, const char* cache_path,
                                         cox_batch_tune* best, float* best_ms, void* stream) {
  if (!best || reps < 1) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return COX_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return COX_ECUDA;
  }
  float best_t = 1e30f;
  cox_batch_tune win = kDefaultTune;
  cox_status rc = COX_OK;
  const int blocks[] = {256, 512, 1024};
  const int cpsm[] = {1, 2, 4};
  const int widths[] = {8, 32};
  const int epts[] = {4, 8, 16};
  const int peers[] = {3, 4};
  for (int b : blocks)
    for (int c : cpsm)
      for (int wdt : widths)
        for (int e : epts)
          for (int pm : peers) {
        if (b * c > 2048) continue;  // more threads than an SM holds
        const cox_batch_tune t = {b, c, wdt, kDefaultTune.fp64_segments, pm, e};
        rc = cox_batch_sum_hist(num_arrays, d_vals, d_keys, &t, d_workspace, workspace_bytes, d_sums, nullptr,
                                d_hists, stream);  // warm-up
        if (rc != COX_OK) goto done;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r)
          cox_batch_sum_hist(num_arrays, d_vals, d_keys, &t, d_workspace, workspace_bytes, d_sums, nullptr, d_hists,
                             stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = COX_ECUDA;
          goto done;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_t) {
          best_t = ms;
          win = t;
        }
      }
  *best = win;
  if (best_ms) *best_ms = best_t;
  if (cache_path) {
    int64_t E = 0;
    const BatchWs w = batch_layout(d_workspace, num_arrays);
    if (cudaMemcpy(&E, w.off + num_arrays, sizeof E, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = COX_ECUDA;
      goto done;
    }
    FILE* f = std::fopen(cache_path, "a");
    if (!f) {
      rc = COX_EINVAL;
      goto done;
    }
    std::fprintf(f, "%s|batch_sum_hist|%d|%d|%d,%d,%d,%d,%d,%d|%.4f\n", gpu_name().c_str(), log2_bucket(num_arrays),
                 log2_bucket(E), win.block_dim, win.ctas_per_sm, win.width, win.fp64_segments, win.native_match,
                 win.ept, best_t);
    std::fclose(f);
  }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

extern "C" cox_status cox_batch_tune_lookup(const char* cache_path, int64_t num_arrays, int64_t total_elems,
                                            cox_batch_tune* tune) {
  if (!cache_path || !tune) return COX_EINVAL;
  FILE* f = std::fopen(cache_path, "r");
  if (!f) return COX_EINVAL;
  const std::string want = gpu_name() + "|batch_sum_hist|" + std::to_string(log2_bucket(num_arrays)) + "|" +
                           std::to_string(log2_bucket(total_elems)) + "|";
  char line[512];
  bool found = false;
  cox_batch_tune t{};
  while (std::fgets(line, sizeof line, f)) {
    if (std::strncmp(line, want.c_str(), want.size()) != 0) continue;
    cox_batch_tune c{};
    if (std::sscanf(line + want.size(), "%d,%d,%d,%d,%d,%d", &c.block_dim, &c.ctas_per_sm, &c.width, &c.fp64_segments,
                    &c.native_match, &c.ept) == 6 &&
        tune_ok(c)) {
      t = c;
      found = true;  // the last matching line wins
    }
  }
  std::fclose(f);
  if (!found) return COX_EINVAL;
  *tune = t;
  return COX_OK;
}
