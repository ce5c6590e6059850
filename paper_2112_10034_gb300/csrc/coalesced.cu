// cox_coalesced and cox_filter_aggregated: warp functions over dynamic
// (coalesced) groups -- the runtime member masks and "all active threads"
// groups that COX leaves unsupported (Sections 2.2.2-2.2.3), and the SDK's
// filter_arr that needs them ("activated thread sync", Table 1).
//
// A warp's group is formed by a full-warp ballot of the activity flags; the
// active lanes then run the warp intrinsics with that member mask
// (shfl.sync / vote.sync / redux.sync with a partial mask), exactly as a
// coalesced_group does.  Group ranks are popc(mask & lanemask_lt); for the
// shuffles, members write their lane into a per-warp rank -> lane table
// and read the source rank's lane from it; the group ballot is an
// OR-reduction of each member's vote shifted to its rank.  The
// integer group scan alone runs over the full warp with inactive lanes
// contributing 0 (the same sums, exactly).
#include "cox_common.cuh"
#include "compact_tile.cuh"

namespace cox {

template <int DT>
__device__ __forceinline__ bool vote_pred(uint32_t u) {
  if constexpr (DT == COX_F32) return __uint_as_float(u) != 0.0f;
  else return u != 0u;
}

// One group's function for one active lane (the lane's value v, the
// group's mask, rank and size).  SCAN_SUM and the shuffles are handled by
// the caller.
template <int DT>
__device__ __forceinline__ uint32_t group_fn(int fn, uint32_t v, unsigned mask, int rank, int size) {
  switch (fn) {
    case COX_CG_SIZE: return (uint32_t)size;
    case COX_CG_RANK: return (uint32_t)rank;
    case COX_CG_BALLOT:  // bit k = the vote of rank k: each member ORs its vote in at its rank
      return __reduce_or_sync(mask, (vote_pred<DT>(v) ? 1u : 0u) << rank);
    case COX_CG_ANY: return __any_sync(mask, vote_pred<DT>(v)) ? 1u : 0u;
    case COX_CG_ALL: return __all_sync(mask, vote_pred<DT>(v)) ? 1u : 0u;
    default: return __reduce_add_sync(mask, v);  // COX_CG_REDUCE_SUM
  }
}

// Persistent warps take 8 consecutive 32-element groups at a time, their
// loads issued together.  SCAN_SUM (integers, exact) runs as a full-warp
// Hillis-Steele scan in which inactive lanes contribute 0: an active lane's
// inclusive prefix over the lanes up to it is its group's prefix by rank.
constexpr int kCgUnroll = 8;

template <int DT>
__global__ void __launch_bounds__(256) k_coalesced(int fn, const uint32_t* __restrict__ in,
                                                   const int32_t* __restrict__ active, uint32_t* __restrict__ out,
                                                   int64_t n, int param) {
  __shared__ uint8_t s_lane[8][32];  // per warp: lane of each group rank (shuffle functions)
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int64_t nw = (n + 32 * kCgUnroll - 1) / (32 * kCgUnroll);
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += wstep) {
    bool act[kCgUnroll];
    uint32_t v[kCgUnroll];
#pragma unroll
    for (int u = 0; u < kCgUnroll; ++u) {
      const int64_t i = (w * kCgUnroll + u) * 32 + lane;
      act[u] = i < n && __ldcs(active + i) != 0;
      v[u] = i < n ? __ldcs(in + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kCgUnroll; ++u) {
      const int64_t i = (w * kCgUnroll + u) * 32 + lane;
      const unsigned mask = __ballot_sync(kFull, act[u]);  // coalesced_threads()
      if (fn == COX_CG_SCAN_SUM) {
        uint32_t x = act[u] ? v[u] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, x, d);
          if (lane >= d) x += y;
        }
        if (act[u]) out[i] = x;
        continue;
      }
      if (fn == COX_CG_SHFL || fn == COX_CG_SHFL_UP || fn == COX_CG_SHFL_DOWN) {
        // rank -> lane table of this round's group: members write their lane
        // at their rank, then read the source rank's lane
        const int rank = __popc(mask & lt), size = __popc(mask);
        if (act[u]) s_lane[wib][rank] = (uint8_t)lane;
        __syncwarp();
        if (act[u]) {
          int want;
          bool own = false;
          if (fn == COX_CG_SHFL) {
            want = param < size ? param : param % size;
          } else if (fn == COX_CG_SHFL_UP) {
            own = rank < param;
            want = rank - param;
          } else {
            own = rank + param >= size;
            want = rank + param;
          }
          out[i] = __shfl_sync(mask, v[u], own ? lane : (int)s_lane[wib][want]);
        }
        __syncwarp();  // the table's readers are done before the next round writes it
        continue;
      }
      if (!act[u]) continue;
      out[i] = group_fn<DT>(fn, v[u], mask, __popc(mask & lt), __popc(mask));
    }
  }
}

// filter_arr with warp-aggregated slots.  A warp owns 512 keys of a chunk;
// each group of keeping lanes (a ballot per key slot) takes the next
// popc(ballot) slots of the warp's range, a lane's key landing at the
// warp's offset + the keeping lanes before it -- the same order as 16
// rounds of 32 keys each taking its group's slots, computed by the
// compaction's one-pass body (compact_region), which packs the kept keys
// in place at the front of the warp's 512 in shared memory.  The warps of
// a CTA aggregate once more: one atomic per CTA per chunk of 8 x 512 keys
// reserves the warps' totals, warp w's base follows warps 0 .. w-1, and
// each warp copies its packed keys out with coalesced stores.  Chunks
// (16 KB) reach shared memory by TMA bulk copies, one ahead of the one
// being processed: two slots keep the kernel at 40 registers and 32 KB of
// shared memory, so six CTAs fit per SM.
constexpr int kFilterRounds = 16;
constexpr int kFilterWarps = 8;
constexpr int kFilterStages = 2;
constexpr int kFilterChunk = 32 * kFilterRounds * kFilterWarps;  // keys per CTA iteration
constexpr size_t kFilterSmem = (size_t)kFilterStages * kFilterChunk * sizeof(uint32_t);

template <bool SIGNED>
__global__ void __launch_bounds__(32 * kFilterWarps, 6)
    k_filter_aggregated(const uint32_t* __restrict__ keys, int64_t n, LeRule rule, uint32_t* __restrict__ out,
                        unsigned long long* __restrict__ count, uint32_t limit, unsigned* status, int vec) {
  extern __shared__ __align__(16) uint32_t fbuf[];
  __shared__ __align__(8) uint64_t bar[kFilterStages];
  __shared__ unsigned s_tot[2][kFilterWarps];  // by iteration parity: a warp runs at most one iteration ahead
  __shared__ unsigned long long s_base[2];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const unsigned lt = lanemask_lt();
  const int64_t nch = (n + kFilterChunk - 1) / kFilterChunk;
  const int64_t nfull = vec ? n / kFilterChunk : 0;  // chunks that arrive by bulk copy
  const int64_t G = gridDim.x;
  auto issue = [&](int64_t j) {  // thread 0: this CTA's iteration j into slot j % stages
    const int64_t c = blockIdx.x + j * G;
    if (c < nfull) {
      uint64_t* b = bar + (int)(j % kFilterStages);
      mbar_arrive_expect_tx(b, kFilterChunk * 4);
      tma_load_1d(fbuf + (j % kFilterStages) * kFilterChunk, keys + c * kFilterChunk, kFilterChunk * 4, b);
    }
  };
  if (tid == 0) {
    for (int s = 0; s < kFilterStages; ++s) mbar_init(bar + s, 1);
    mbar_init_fence();
    for (int j = 0; j < kFilterStages - 1; ++j) issue(j);
  }
  __syncthreads();
  bool ok = true;
  int64_t it = 0;
  const int region = wib * (32 * kFilterRounds);  // this warp's keys in a slot
  for (int64_t c = blockIdx.x; c < nch; c += G, ++it) {
    // slot (it - 1) % stages was last read (copied out) before the barrier
    // that ended the previous iteration
    if (tid == 0) issue(it + kFilterStages - 1);
    const int par = (int)(it & 1);
    const int slot = (int)(it % kFilterStages);
    uint32_t* buf = fbuf + slot * kFilterChunk;
    const int valid = (int)min((int64_t)kFilterChunk, n - c * kFilterChunk);  // keys of this chunk
    if (c < nfull) {
      ok = mbar_wait_bounded(bar + slot, (uint32_t)((it / kFilterStages) & 1), limit);
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
    } else {  // a ragged or unaligned chunk: plain loads into the slot
      for (int i = tid; i < valid; i += 32 * kFilterWarps) buf[i] = __ldcs(keys + c * kFilterChunk + i);
      __syncthreads();
    }
    // every warp compacts its 512 keys in place (input order), then one
    // atomic per CTA claims the chunk's output slots
    const uint32_t kept = compact_region<SIGNED, 32 * kFilterRounds>(buf, region, lane, lt, valid,
                                                                     valid == kFilterChunk, rule);
    if (lane == 0) s_tot[par][wib] = kept;
    __syncthreads();
    if (tid == 0) {  // the CTA's slots, and each warp's offset in them (in place of its count)
      unsigned sum = 0;
#pragma unroll
      for (int w = 0; w < kFilterWarps; ++w) {
        const unsigned t = s_tot[par][w];
        s_tot[par][w] = sum;
        sum += t;
      }
      s_base[par] = sum ? atomicAdd(count, (unsigned long long)sum) : 0ull;
    }
    __syncthreads();
    uint32_t* o = out + (s_base[par] + s_tot[par][wib]);
    const uint32_t* src = buf + region;
#pragma unroll 4
    for (int i = lane; i < (int)kept; i += 32) o[i] = src[i];
    fence_proxy_async_smem();  // this thread's accesses to the slot, before the bulk copy that refills it
    __syncthreads();
  }
  if (!ok && tid == 0) {  // a copy did not land in time: record it, give the copies in flight a bounded wait
    atomicOr(status, (unsigned)kDevTimeout);
    for (int64_t j = it; j < it + kFilterStages; ++j)  // iterations it .. it + stages - 1 were issued
      if (blockIdx.x + j * G < nfull)
        mbar_wait_bounded(bar + (int)(j % kFilterStages), (uint32_t)((j / kFilterStages) & 1), limit);
  }
}

template <int DT>
static cox_status launch_coalesced(int fn, const void* d_in, const int32_t* d_active, void* d_out, int64_t n,
                                   int param, cudaStream_t st) {
  auto k = k_coalesced<DT>;
  static int grid[kMaxDevices];  // persistent grid of this instance, per device
  int& g = grid[device_index()];
  if (g == 0) g = persistent_grid(k, 256, 0, 1 << 30);
  const int64_t ctas = ((n + 32 * kCgUnroll - 1) / (32 * kCgUnroll) + 7) / 8;
  k<<<(int)(ctas < g ? ctas : g), 256, 0, st>>>(fn, static_cast<const uint32_t*>(d_in), d_active,
                                                static_cast<uint32_t*>(d_out), n, param);
  return launch_status();
}

template <bool SIGNED>
static cox_status launch_filter(const void* d_keys, int64_t n, int64_t threshold, void* d_out, int64_t* d_count,
                                cudaStream_t st) {
  auto k = k_filter_aggregated<SIGNED>;
  static int grid[kMaxDevices];  // per device: the attribute and the occupancy are per-device state
  int& g = grid[device_index()];
  if (g == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFilterSmem) != cudaSuccess)
      return COX_ECUDA;
    g = persistent_grid(k, 32 * kFilterWarps, kFilterSmem, 1 << 30);
  }
  const int64_t ctas = (n + kFilterChunk - 1) / kFilterChunk;
  k<<<(int)(ctas < g ? ctas : g), 32 * kFilterWarps, kFilterSmem, st>>>(
      static_cast<const uint32_t*>(d_keys), n, le_rule<SIGNED>(threshold), static_cast<uint32_t*>(d_out),
      reinterpret_cast<unsigned long long*>(d_count), spin_limit(), device_status_word(), aligned16(d_keys) ? 1 : 0);
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_coalesced(cox_cgfn fn, cox_dtype dt, int block_dim, const void* d_in,
                                    const int32_t* d_active, void* d_out, int64_t n, int param, void* stream) {
  if (!valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (fn < COX_CG_SIZE || fn > COX_CG_SCAN_SUM) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32 && dt != COX_F32) return COX_EINVAL;
  if ((fn == COX_CG_REDUCE_SUM || fn == COX_CG_SCAN_SUM) && dt == COX_F32) return COX_EINVAL;
  if ((fn == COX_CG_SHFL || fn == COX_CG_SHFL_UP || fn == COX_CG_SHFL_DOWN) && (param < 0 || param > 31))
    return COX_EINVAL;
  if (n == 0) return COX_OK;
  if (!d_in || !d_active || !d_out) return COX_EINVAL;
  if (dt == COX_F32) return launch_coalesced<COX_F32>((int)fn, d_in, d_active, d_out, n, param, as_stream(stream));
  return launch_coalesced<COX_I32>((int)fn, d_in, d_active, d_out, n, param, as_stream(stream));
}

extern "C" cox_status cox_filter_aggregated(cox_dtype dt, const void* d_keys, int64_t n, int64_t threshold,
                                            void* d_out, int64_t* d_count, void* stream) {
  if (n < 0 || !d_count || (dt != COX_I32 && dt != COX_U32)) return COX_EINVAL;
  if (n > 0 && (!d_keys || !d_out)) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), st) != cudaSuccess) return COX_ECUDA;
  if (n == 0) return COX_OK;
  if (dt == COX_I32) return launch_filter<true>(d_keys, n, threshold, d_out, d_count, st);
  return launch_filter<false>(d_keys, n, threshold, d_out, d_count, st);
}
