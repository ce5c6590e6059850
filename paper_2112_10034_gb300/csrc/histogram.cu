// cox_match_histogram: histogram from match_any peer groups.
//
// Per warp step every lane holds one key; peers = match_any(key) restricted to
// the lane's width-W tile and to lanes whose key is in [0, bins); the lowest
// peer (the group's leader) adds popc(peers) to a shared-memory bin, so equal
// keys in a tile cost one shared atomic instead of one each.  Keys outside
// [0, bins) are counted as ignored.  The peer mask comes from ballots over
// the key bits (match_any_bits), from a per-warp table in shared memory
// (each lane ORs its bit into its key's word and reads it back; the default
// when the tables fit) or, with COX_F_NATIVE_MATCH, from the match.any.sync
// instruction; all give the same mask.  Shared histograms are
// per warp when they fit (no cross-warp contention on hot bins, e.g. Zipf
// keys), else per CTA; each CTA merges its non-zero bins into the output with
// global atomics.  Integer counts: exact whatever the grouping.
#include "cox_common.cuh"

namespace cox {

// One warp step: every lane holds one key.  Keys in [0, bins) form peer
// groups (match_any restricted to the lane's width-W tile and to in-range
// lanes); the lowest lane of each group adds the group's size to its bin.
// Valid keys outside the range are counted by lane 0 through one ballot --
// the same total as summing their peer groups.
// PEER selects how equal keys are grouped: kPeerBallot (ballots over the key
// bits), kPeerNative (match.any.sync), kPeerTable (a per-warp table in shared
// memory: each in-range lane ORs its lane bit into its key's word, then reads
// the word back -- the lanes holding that key, i.e. the same mask), kPeerNone
// (no grouping: every lane adds one to its own bin -- the same counts,
// without the warp function).  Keys outside the range are counted per lane.
enum { kPeerBallot = 0, kPeerNative = 1, kPeerNone = 2, kPeerTable = 3 };

template <int W, int BITS, int PEER>
__device__ __forceinline__ void hist_step(uint32_t key, bool valid, uint32_t bins, uint32_t* my, uint32_t& ign,
                                          uint32_t* tab, int& tsel) {
  const int lane = lane_id();
  const bool in = valid && key < bins;
  if constexpr (PEER == kPeerNone) {
    if (in) atomicAdd(my + key, 1u);
  } else {
    const unsigned tmask = W == 32 ? kFull : (((1u << W) - 1u) << (lane & ~(W - 1)));
    const unsigned lt = lanemask_lt();
    unsigned peers;
    if constexpr (PEER == kPeerTable) {
      // two tables used in turn: a table's words are cleared (by each key's
      // lowest lane, after every lane has read) before its next use
      uint32_t* t = tab + tsel * bins;
      tsel ^= 1;
      if (in) atomicOr(t + key, 1u << lane);
      __syncwarp();
      const unsigned all = in ? t[key] : 0u;  // the warp's lanes holding this key
      __syncwarp();
      if (in && (all & lt) == 0u) t[key] = 0u;
      peers = all;
    } else if constexpr (PEER == kPeerNative) {
      peers = __match_any_sync(kFull, key) & __ballot_sync(kFull, in);
    } else {
      peers = match_any_bits<BITS>(key, in);
    }
    peers &= tmask;
    if (in && (peers & lt) == 0u) atomicAdd(my + key, (uint32_t)__popc(peers));
  }
  ign += valid && !in;
}

template <int W, int BITS, int PEER>
__global__ void __launch_bounds__(1024) k_match_hist(const uint32_t* __restrict__ keys, int64_t n, uint32_t bins,
                                                     int per_warp, int32_t* __restrict__ hist,
                                                     unsigned long long* ignored, int vec) {
  extern __shared__ uint32_t sh[];
  __shared__ uint32_t s_ign;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int nsh = per_warp ? nw * (int)bins : (int)bins;
  const int ntab = PEER == kPeerTable ? nw * 2 * (int)bins : 0;  // peer tables after the histograms
  for (int i = threadIdx.x; i < nsh + ntab; i += blockDim.x) sh[i] = 0u;
  if (threadIdx.x == 0) s_ign = 0u;
  __syncthreads();
  uint32_t* my = per_warp ? sh + warp * bins : sh;
  uint32_t* tab = sh + nsh + warp * 2 * bins;
  int tsel = 0;
  uint32_t ign = 0;  // this lane's keys outside [0, bins)
  // Each warp step covers 128 consecutive keys (one 128-bit load per lane).
  const int64_t nsteps = (n + 127) / 128;
  const int64_t gw = (int64_t)blockIdx.x * nw + warp, gws = (int64_t)gridDim.x * nw;
  int64_t s = gw;
  if (vec) {
    for (; s + gws < nsteps && (s + gws + 1) * 128 <= n; s += 2 * gws) {  // two loads in flight
      const uint4 a = __ldcs(reinterpret_cast<const uint4*>(keys + s * 128) + lane);
      const uint4 b = __ldcs(reinterpret_cast<const uint4*>(keys + (s + gws) * 128) + lane);
      hist_step<W, BITS, PEER>(a.x, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(a.y, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(a.z, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(a.w, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(b.x, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(b.y, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(b.z, true, bins, my, ign, tab, tsel);
      hist_step<W, BITS, PEER>(b.w, true, bins, my, ign, tab, tsel);
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
#pragma unroll
    for (int q = 0; q < 4; ++q) hist_step<W, BITS, PEER>(k[q], v[q], bins, my, ign, tab, tsel);
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

template <int W, int BITS, int PEER>
static cox_status launch_hist(const void* d_keys, int64_t n, int bins, int block_dim, int per_warp, size_t smem,
                              int32_t* d_hist, int64_t* d_ignored, cudaStream_t st) {
  auto k = k_match_hist<W, BITS, PEER>;
  const int nw = block_dim / 32;
  static int gmax[33][113];  // by warps per CTA and shared KiB
  int& g = gmax[nw][(smem + 1023) / 1024];
  if (g == 0) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return COX_ECUDA;
    g = persistent_grid(k, block_dim, smem, 1 << 30);
  }
  const int64_t steps = (n + 127) / 128;
  const int64_t ctas = (steps + nw - 1) / nw;
  k<<<(int)(ctas < g ? ctas : g), block_dim, smem, st>>>(static_cast<const uint32_t*>(d_keys), n, (uint32_t)bins,
                                                         per_warp, d_hist,
                                                         reinterpret_cast<unsigned long long*>(d_ignored),
                                                         aligned16(d_keys));
  return launch_status();
}

template <int PEER>
static cox_status dispatch_hist(int width, const void* d_keys, int64_t n, int bins, int block_dim, int per_warp,
                                size_t smem, int32_t* d_hist, int64_t* d_ignored, cudaStream_t st) {
  return with_width(width, [&](auto w) {
    constexpr int W = decltype(w)::value;
    if (PEER != kPeerBallot || bins <= 256)
      return launch_hist<W, 8, PEER>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
    if (bins <= 1024)
      return launch_hist<W, 10, PEER>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
    return launch_hist<W, 13, PEER>(d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
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
  const size_t smem = (size_t)(per_warp ? nw * bins : bins) * 4;
  const size_t tab = (size_t)nw * 2 * bins * 4;  // two peer tables per warp
  if (modes == 0 && smem + tab <= 100 * 1024)
    return dispatch_hist<kPeerTable>(width, d_keys, n, bins, block_dim, per_warp, smem + tab, d_hist, d_ignored, st);
  if (flags & COX_F_NATIVE_MATCH)
    return dispatch_hist<kPeerNative>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
  if (flags & COX_F_DIRECT_ATOMICS)
    return dispatch_hist<kPeerNone>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
  return dispatch_hist<kPeerBallot>(width, d_keys, n, bins, block_dim, per_warp, smem, d_hist, d_ignored, st);
}
