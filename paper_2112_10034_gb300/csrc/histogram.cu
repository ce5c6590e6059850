// cox_match_histogram: histogram from match_any peer groups.
//
// Per warp step every lane holds four keys (one 128-bit load); for each key,
// peers = match_any(key) restricted to the lane's width-W tile and to lanes
// whose key is in [0, bins); one lane of each peer group adds popc(peers) to
// a shared-memory bin, so equal keys in a tile cost one shared atomic
// instead of one each.  Keys outside [0, bins) are counted as ignored.  The
// peer mask comes, by default, from a per-warp table in shared memory
// (hist_peer_table in cox_common.cuh: lanes OR their bit into their key's
// word; a lane that found its word empty takes the mask and clears it),
// else from ballots over the key bits (match_any_bits), or with
// COX_F_NATIVE_MATCH from the match.any.sync instruction; all give the same
// mask.  Shared histograms are per warp when they fit (no cross-warp
// contention on hot bins, e.g. Zipf keys), else per CTA; each CTA merges its
// non-zero bins into the output with global atomics.  Integer counts: exact
// whatever the grouping.
#include "cox_common.cuh"

namespace cox {

// One warp step: every lane holds one key.  Keys in [0, bins) form peer
// groups (match_any restricted to the lane's width-W tile and to in-range
// lanes); the lowest lane of each group adds the group's size to its bin.
// PEER selects how equal keys are grouped: kPeerBallot (ballots over the key
// bits), kPeerNative (match.any.sync), kPeerNone (no grouping: every lane
// adds one to its own bin -- the same counts, without the warp function);
// kPeerTable (a per-warp table of masks) runs four keys at a time in
// hist_peer_table.  Keys outside the range are counted per lane.
enum { kPeerBallot = 0, kPeerNative = 1, kPeerNone = 2, kPeerTable = 3 };

template <int W, int BITS, int PEER>
__device__ __forceinline__ void hist_step(uint32_t key, bool valid, uint32_t bins, uint32_t* my, uint32_t& ign) {
  const int lane = lane_id();
  const bool in = valid && key < bins;
  if constexpr (PEER == kPeerNone) {
    if (in) atomicAdd(my + key, 1u);
  } else {
    const unsigned tmask = W == 32 ? kFull : (((1u << W) - 1u) << (lane & ~(W - 1)));
    const unsigned lt = lanemask_lt();
    unsigned peers;
    if constexpr (PEER == kPeerNative) {
      peers = __match_any_sync(kFull, key) & __ballot_sync(kFull, in);
    } else {
      peers = match_any_bits<BITS>(key, in);
    }
    peers &= tmask;
    if (in && (peers & lt) == 0u) atomicAdd(my + key, (uint32_t)__popc(peers));
  }
  ign += valid && !in;
}

// Four keys of one lane (one 128-bit load); S peer tables for kPeerTable.
template <int W, int BITS, int PEER, int S>
__device__ __forceinline__ void hist_quad(const uint32_t (&k)[4], const bool (&v)[4], uint32_t bins, uint32_t* my,
                                          uint32_t& ign, uint32_t* tab) {
  if constexpr (PEER == kPeerTable) {
    bool in[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      in[q] = v[q] && k[q] < bins;
      ign += v[q] && !in[q];
    }
    int parity = 0;  // (unused by the split layout)
    hist_peer_table<W, S, 4, true>(k, in, bins, my, tab, parity);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) hist_step<W, BITS, PEER>(k[q], v[q], bins, my, ign);
  }
}

template <int W, int BITS, int PEER, int S>
__global__ void __launch_bounds__(1024) k_match_hist(const uint32_t* __restrict__ keys, int64_t n, uint32_t bins,
                                                     int per_warp, int32_t* __restrict__ hist,
                                                     unsigned long long* ignored, int vec) {
  extern __shared__ __align__(16) uint32_t sh[];
  __shared__ uint32_t s_ign;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int nsh = ((per_warp ? nw * (int)bins : (int)bins) + 1) & ~1;  // even: the tables hold 64-bit pairs
  const int ntab = PEER == kPeerTable ? S * (int)hist_table_words(W, bins, true) : 0;  // per warp
  // histograms, then the peer tables; all start at zero
  for (int i = threadIdx.x; i < nsh + nw * ntab; i += blockDim.x) sh[i] = 0u;
  if (threadIdx.x == 0) s_ign = 0u;
  __syncthreads();
  uint32_t* my = per_warp ? sh + warp * bins : sh;
  uint32_t* tab = sh + nsh + warp * ntab;  // 8-byte aligned: nsh and ntab are even
  uint32_t ign = 0;  // this lane's keys outside [0, bins)
  // Each warp step covers 128 consecutive keys (one 128-bit load per lane).
  const int64_t nsteps = (n + 127) / 128;
  const int64_t gw = (int64_t)blockIdx.x * nw + warp, gws = (int64_t)gridDim.x * nw;
  int64_t s = gw;
  const bool vall[4] = {true, true, true, true};
  // pairs of steps (s, s + gws) whose keys are all in range, the next pair's
  // two 128-bit loads in flight while this pair is counted
  auto full_pair = [&](int64_t t) { return t + gws < nsteps && (t + gws + 1) * 128 <= n; };
  if (vec && full_pair(s)) {
    uint4 a = __ldcs(reinterpret_cast<const uint4*>(keys + s * 128) + lane);
    uint4 b = __ldcs(reinterpret_cast<const uint4*>(keys + (s + gws) * 128) + lane);
    for (;;) {
      const int64_t sn = s + 2 * gws;
      const bool more = full_pair(sn);
      uint4 a2 = a, b2 = b;
      if (more) {
        a2 = __ldcs(reinterpret_cast<const uint4*>(keys + sn * 128) + lane);
        b2 = __ldcs(reinterpret_cast<const uint4*>(keys + (sn + gws) * 128) + lane);
      }
      const uint32_t ka[4] = {a.x, a.y, a.z, a.w}, kb[4] = {b.x, b.y, b.z, b.w};
      hist_quad<W, BITS, PEER, S>(ka, vall, bins, my, ign, tab);
      hist_quad<W, BITS, PEER, S>(kb, vall, bins, my, ign, tab);
      s = sn;
      if (!more) break;
      a = a2;
      b = b2;
    }
  }
  for (; s < nsteps; s += gws) {
    const int64_t e0 = s * 128 + 4 * lane;
    uint32_t k[4];
    bool v[4];
    if (vec && s * 128 + 128 <= n) {
      const uint4 a = __ldcs(reinterpret_cast<const uint4*>(keys + s * 128) + lane);
      k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
      v[0] = v[1] = v[2] = v[3] = true;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = e0 + q < n;
        k[q] = v[q] ? keys[e0 + q] : 0u;
      }
    }
    hist_quad<W, BITS, PEER, S>(k, v, bins, my, ign, tab);
  }
  ign = __reduce_add_sync(kFull, ign);
  if (lane == 0 && ign) atomicAdd(&s_ign, ign);
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < bins; b += blockDim.x) {
    uint32_t c = 0;
    if (per_warp) {
      for (int w = 0; w < nw; ++w) c += sh[w * bins + b];
    } else {
      c = sh[b];
    }
    if (c) atomicAdd(hist + b, (int32_t)c);
  }
  if (threadIdx.x == 0 && s_ign && ignored) atomicAdd(ignored, (unsigned long long)s_ign);
}

template <int W, int BITS, int PEER, int S>
static cox_status launch_hist(const void* d_keys, int64_t n, int bins, int block_dim, int per_warp, size_t smem,
                              int32_t* d_hist, int64_t* d_ignored, cudaStream_t st) {
  auto k = k_match_hist<W, BITS, PEER, S>;
  const int nw = block_dim / 32;
  struct Shape {
    size_t smem;
    int grid;
  };
  static Shape cache[kMaxDevices][33];  // per device and warps per CTA: the last shared size and its grid
  Shape& c = cache[device_index()][nw];
  if (c.grid == 0 || c.smem != smem) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return COX_ECUDA;
    c.grid = persistent_grid(k, block_dim, smem, 1 << 30);
    c.smem = smem;
  }
  const int g = c.grid;
  const int64_t steps = (n + 127) / 128;
  const int64_t ctas = (steps + nw - 1) / nw;
  k<<<(int)(ctas < g ? ctas : g), block_dim, smem, st>>>(static_cast<const uint32_t*>(d_keys), n, (uint32_t)bins,
                                                         per_warp, d_hist,
                                                         reinterpret_cast<unsigned long long*>(d_ignored),
                                                         aligned16(d_keys));
  return launch_status();
}

template <int PEER, int S = 1>
static cox_status dispatch_hist(int width, const void* d_keys, int64_t n, int bins, int block_dim, int per_warp,
                                size_t smem, int32_t* d_hist, int64_t* d_ignored, cudaStream_t st) {
  return with_width(width, [&](auto w) {
    constexpr int W = decltype(w)::value;
    if (PEER != kPeerBallot || bins <= 256)
      return launch_hist<W, 8, PEER, S>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
    if (bins <= 1024)
      return launch_hist<W, 10, PEER, S>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
    return launch_hist<W, 13, PEER, S>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
  });
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_match_histogram(cox_dtype dt, int width, int block_dim, const void* d_keys, int64_t n,
                                          int bins, int32_t* d_hist, int64_t* d_ignored, unsigned flags,
                                          void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32) return COX_EINVAL;
  if (bins < 1 || bins > 8192 || !d_hist || (n > 0 && !d_keys)) return COX_EINVAL;
  const unsigned modes = flags & (COX_F_NATIVE_MATCH | COX_F_DIRECT_ATOMICS | COX_F_BALLOT_MATCH);
  if (flags != modes || (modes & (modes - 1u))) return COX_EINVAL;  // at most one mode
  cudaStream_t st = as_stream(stream);
  if (cudaMemsetAsync(d_hist, 0, (size_t)bins * sizeof(int32_t), st) != cudaSuccess) return COX_ECUDA;
  if (d_ignored && cudaMemsetAsync(d_ignored, 0, sizeof(int64_t), st) != cudaSuccess) return COX_ECUDA;
  if (n == 0) return COX_OK;
  const int nw = block_dim / 32;
  const int per_warp = (size_t)nw * bins * 4 <= 48 * 1024;
  const size_t smem = (((size_t)(per_warp ? nw * bins : bins) + 1) & ~(size_t)1) * 4;  // even word count
  // peer tables: S tables of hist_table_words(width, bins) words per warp;
  // four where a CTA stays within 40 KB (five CTAs per SM), else two, else one
  const size_t tab1 = (size_t)nw * (width == 32 ? 2 * (size_t)bins : (size_t)(32 / width) * bins) * 4;
  if (modes == 0) {
    if (smem + 4 * tab1 <= 40 * 1024)
      return dispatch_hist<kPeerTable, 4>(width, d_keys, n, bins, block_dim, per_warp, smem + 4 * tab1, d_hist,
                                          d_ignored, st);
    if (smem + 2 * tab1 <= 40 * 1024)
      return dispatch_hist<kPeerTable, 2>(width, d_keys, n, bins, block_dim, per_warp, smem + 2 * tab1, d_hist,
                                          d_ignored, st);
    if (smem + tab1 <= 100 * 1024)
      return dispatch_hist<kPeerTable, 1>(width, d_keys, n, bins, block_dim, per_warp, smem + tab1, d_hist,
                                          d_ignored, st);
  }
  if (flags & COX_F_NATIVE_MATCH)
    return dispatch_hist<kPeerNative>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
  if (flags & COX_F_DIRECT_ATOMICS)
    return dispatch_hist<kPeerNone>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
  return dispatch_hist<kPeerBallot>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
}
