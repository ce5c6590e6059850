// cox_grid_broadcast: reduce over the whole array, grid-wide barrier, then a
// per-element step that uses the result -- one cooperative kernel.
//
// This is the grid synchronisation of cooperative groups that the SDK's
// gpuConjugateGradient relies on and COX cannot support (Table 1 of the
// paper, Section 5.1).  The CTAs of a cooperative launch are co-resident, so
// a CTA may wait for the others; the barrier here is a counter plus a
// release flag in a zeroed workspace, and its waits are bounded.
//
// Arrays that fit on chip (one slice per CTA, one CTA per SM, up to 196 KB
// of shared memory each) are read once: each CTA's slice arrives by TMA bulk
// copies, is reduced from shared memory, kept there across the barrier,
// transformed in place and written back by TMA bulk stores.  Larger arrays
// are streamed twice (grid-stride loops before and after the barrier, the
// second one backwards so that it starts on the lines still in L2).
#include "cox_common.cuh"

namespace cox {

constexpr int kGbThreads = 512;
constexpr size_t kGbWsHeader = 256;
constexpr size_t kGbResidentBytes = 196 * 1024;
constexpr uint32_t kGbPiece = 32 * 1024;  // bytes per TMA bulk copy

// Order-preserving 32-bit keys: the minimum key is the minimum element.
// F32 keys follow totalOrder (-0 below +0); every NaN maps to the largest
// key, so NaNs are ignored unless all elements are NaN.
template <int DT>
__device__ __forceinline__ uint32_t min_key(uint32_t u) {
  if constexpr (DT == COX_I32) return u ^ 0x80000000u;
  else if constexpr (DT == COX_U32) return u;
  else {
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return 0xFFFFFFFFu;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  }
}
template <int DT>
__device__ __forceinline__ uint32_t min_unkey(uint32_t k) {
  if constexpr (DT == COX_I32) return k ^ 0x80000000u;
  else if constexpr (DT == COX_U32) return k;
  else {
    if (k == 0xFFFFFFFFu) return 0x7FFFFFFFu;
    return (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  }
}

// Per-op state: SUB_MIN folds keys with min; NORMALIZE folds fl(x*x) into
// TwoSum pairs.
template <int OP, int DT>
struct GbAcc {
  uint32_t k = 0xFFFFFFFFu;
  __device__ void add(uint32_t u) { k = min(k, min_key<DT>(u)); }
};
template <>
struct GbAcc<COX_GRID_NORMALIZE, COX_F32> {
  Pair p{0.0f, 0.0f};
  __device__ void add(uint32_t u) {
    const float x = __uint_as_float(u);
    p = Comp::op(p, Comp::load(__fmul_rn(x, x)));
  }
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One-use grid barrier over a zeroed (count, open) pair.  Returns false in
// every thread of a CTA whose wait ran out (status recorded).
__device__ bool grid_barrier(unsigned* count, unsigned* open, uint32_t limit, unsigned* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      __threadfence();
      st_release_u32(open, 1u);
    } else {
      ok = 0;
      for (uint32_t i = 0; i <= limit; ++i) {
        if (ld_acquire_u32(open) != 0u) {
          ok = 1;
          break;
        }
        if (i > 64) __nanosleep(128);
      }
      if (!ok) atomicOr(status, (unsigned)kDevTimeout);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int OP, int DT>
__device__ __forceinline__ uint32_t apply(uint32_t u, uint32_t mbits, float norm) {
  if constexpr (OP == COX_GRID_NORMALIZE) return __float_as_uint(__fdiv_rn(__uint_as_float(u), norm));
  else if constexpr (DT == COX_F32) return __float_as_uint(__fsub_rn(__uint_as_float(u), __uint_as_float(mbits)));
  else return u - mbits;
}

// resident != 0: CTA c owns elements [c*S, min(n, (c+1)*S)), S a multiple of
// 4, held in dynamic shared memory across the barrier (in and out 16-byte
// aligned).  resident == 0: grid-stride streaming (`vec` = in and out
// 16-byte aligned).
template <int OP, int DT>
__global__ void __launch_bounds__(kGbThreads) k_grid_bcast(const uint32_t* in, uint32_t* out, int64_t n,
                                                           int64_t S, int resident, int vec, uint8_t* ws,
                                                           uint32_t limit, unsigned* status) {
  extern __shared__ __align__(16) uint32_t gb_smem[];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_min[32];
  __shared__ Pair s_pair[32];
  __shared__ uint32_t s_mbits;
  __shared__ float s_norm;
  __shared__ int s_loaded;
  unsigned* count = reinterpret_cast<unsigned*>(ws);
  unsigned* open = count + 1;
  const int tid = threadIdx.x;
  const int64_t c0 = resident ? (int64_t)blockIdx.x * S : 0;
  const int64_t len = resident ? (c0 < n ? (n - c0 < S ? n - c0 : S) : 0) : 0;
  const int64_t nv = len / 4;  // whole 16-byte units of the slice
  GbAcc<OP, DT> acc;
  // ---------------------------------------------------------- phase 1
  if (resident) {
    if (tid == 0) {
      s_loaded = 1;
      if (nv > 0) {
        mbar_init(&s_bar, 1);
        mbar_init_fence();
        mbar_arrive_expect_tx(&s_bar, (uint32_t)(nv * 16));
        for (int64_t off = 0; off < nv * 16; off += kGbPiece) {
          const uint32_t b = (uint32_t)(nv * 16 - off < kGbPiece ? nv * 16 - off : kGbPiece);
          tma_load_1d(reinterpret_cast<uint8_t*>(gb_smem) + off, reinterpret_cast<const uint8_t*>(in + c0) + off, b,
                      &s_bar);
        }
      }
    }
    for (int64_t i = nv * 4 + tid; i < len; i += kGbThreads) gb_smem[i] = in[c0 + i];  // the last < 4 elements
    __syncthreads();
    if (nv > 0 && !mbar_wait_bounded(&s_bar, 0, limit)) s_loaded = 0;  // benign race: all writers store 0
    __syncthreads();
    if (!s_loaded) {
      if (tid == 0) {
        atomicOr(status, (unsigned)kDevTimeout);
        mbar_wait_bounded(&s_bar, 0, limit);  // the copies in flight, before the CTA ends
      }
    } else {
      for (int64_t i = tid; i < len; i += kGbThreads) acc.add(gb_smem[i]);
    }
  } else if (vec) {
    const int64_t gt = (int64_t)blockIdx.x * kGbThreads + tid, gs = (int64_t)gridDim.x * kGbThreads;
    const uint4* p = reinterpret_cast<const uint4*>(in);
    for (int64_t i = gt; i < n / 4; i += gs) {
      const uint4 q = __ldcg(p + i);  // kept in L2: phase 2 re-reads the last of it from there
      acc.add(q.x);
      acc.add(q.y);
      acc.add(q.z);
      acc.add(q.w);
    }
    for (int64_t i = n / 4 * 4 + gt; i < n; i += gs) acc.add(in[i]);
  } else {
    const int64_t gt = (int64_t)blockIdx.x * kGbThreads + tid, gs = (int64_t)gridDim.x * kGbThreads;
    for (int64_t i = gt; i < n; i += gs) acc.add(in[i]);
  }
  // CTA partial: key min through redux.sync, or a TwoSum block tree.
  if constexpr (OP == COX_GRID_NORMALIZE) {
    const Pair b = block_reduce32<Comp>(acc.p, s_pair);
    if (tid == 0) reinterpret_cast<float2*>(ws + kGbWsHeader)[blockIdx.x] = make_float2(b.s, b.e);
  } else {
    const uint32_t w = __reduce_min_sync(kFull, acc.k);
    if ((tid & 31) == 0) s_min[tid >> 5] = w;
    __syncthreads();
    if (tid < 32) {
      uint32_t v = tid < kGbThreads / 32 ? s_min[tid] : 0xFFFFFFFFu;
      v = __reduce_min_sync(kFull, v);
      if (tid == 0) reinterpret_cast<uint32_t*>(ws + kGbWsHeader)[blockIdx.x] = v;
    }
  }
  // ---------------------------------------------------------- barrier
  const bool ok = grid_barrier(count, open, limit, status);
  if (!ok || (resident && !s_loaded)) return;
  // Every CTA folds the partials in CTA order: the same result everywhere.
  if (tid < 32) {
    __threadfence();
    const int G = gridDim.x;
    if constexpr (OP == COX_GRID_NORMALIZE) {
      double d = 0.0;
      for (int k = tid; k < G; k += 32) {
        const float2 f = __ldcg(reinterpret_cast<const float2*>(ws + kGbWsHeader) + k);
        d += (double)f.x + (double)f.y;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(kFull, d, off);
      if (tid == 0) s_norm = (float)sqrt(d);
    } else {
      uint32_t v = 0xFFFFFFFFu;
      for (int k = tid; k < G; k += 32) v = min(v, __ldcg(reinterpret_cast<const uint32_t*>(ws + kGbWsHeader) + k));
      v = __reduce_min_sync(kFull, v);
      if (tid == 0) s_mbits = min_unkey<DT>(v);
    }
  }
  __syncthreads();
  const uint32_t mbits = s_mbits;
  const float norm = s_norm;
  // ---------------------------------------------------------- phase 2
  if (resident) {
    for (int64_t i = tid; i < len; i += kGbThreads) gb_smem[i] = apply<OP, DT>(gb_smem[i], mbits, norm);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && nv > 0) {
      for (int64_t off = 0; off < nv * 16; off += kGbPiece) {
        const uint32_t b = (uint32_t)(nv * 16 - off < kGbPiece ? nv * 16 - off : kGbPiece);
        tma_store_1d(reinterpret_cast<uint8_t*>(out + c0) + off, reinterpret_cast<const uint8_t*>(gb_smem) + off, b);
      }
    }
    for (int64_t i = nv * 4 + tid; i < len; i += kGbThreads) out[c0 + i] = gb_smem[i];
    if (tid == 0) tma_store_wait_all();
  } else if (vec) {
    const int64_t gt = (int64_t)blockIdx.x * kGbThreads + tid, gs = (int64_t)gridDim.x * kGbThreads;
    const uint4* p = reinterpret_cast<const uint4*>(in);
    uint4* q = reinterpret_cast<uint4*>(out);
    // backwards: phase 1 ended on the array's tail, whose lines are still in
    // L2, so those are read first (output stores stream past L2)
    for (int64_t j = gt; j < n / 4; j += gs) {
      const int64_t i = n / 4 - 1 - j;
      uint4 v = __ldcs(p + i);
      v.x = apply<OP, DT>(v.x, mbits, norm);
      v.y = apply<OP, DT>(v.y, mbits, norm);
      v.z = apply<OP, DT>(v.z, mbits, norm);
      v.w = apply<OP, DT>(v.w, mbits, norm);
      __stcs(q + i, v);
    }
    for (int64_t i = n / 4 * 4 + gt; i < n; i += gs) out[i] = apply<OP, DT>(in[i], mbits, norm);
  } else {
    const int64_t gt = (int64_t)blockIdx.x * kGbThreads + tid, gs = (int64_t)gridDim.x * kGbThreads;
    for (int64_t i = gt; i < n; i += gs) out[i] = apply<OP, DT>(in[i], mbits, norm);
  }
}

template <int OP, int DT>
static cox_status launch_gb(const void* d_in, void* d_out, int64_t n, void* ws, cudaStream_t st) {
  auto k = k_grid_bcast<OP, DT>;
  static int per_sm_stream = 0;
  if (per_sm_stream == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGbResidentBytes) != cudaSuccess)
      return COX_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_stream, k, kGbThreads, 0) != cudaSuccess ||
        per_sm_stream < 1)
      return COX_ECUDA;
  }
  const int sms = sm_count();
  const bool aligned = aligned16(d_in) && aligned16(d_out);
  // Resident: one CTA per SM (at most), slices of S elements, S a multiple of 4.
  int64_t G = (n + 4095) / 4096;
  if (G > sms) G = sms;
  if (G < 1) G = 1;
  int64_t S = ((n + G - 1) / G + 3) / 4 * 4;
  int resident = aligned && S * 4 <= (int64_t)kGbResidentBytes;
  size_t smem = 0;
  if (resident) {
    G = (n + S - 1) / S;  // every CTA owns a non-empty slice
    smem = (size_t)S * 4;
  } else {
    G = (int64_t)per_sm_stream * sms;
    const int64_t need = (n + kGbThreads * 4 - 1) / (kGbThreads * 4);
    if (need < G) G = need < 1 ? 1 : need;
    S = 0;
  }
  if (cudaMemsetAsync(ws, 0, kGbWsHeader, st) != cudaSuccess) return COX_ECUDA;
  const uint32_t* in = static_cast<const uint32_t*>(d_in);
  uint32_t* out = static_cast<uint32_t*>(d_out);
  int vec = aligned ? 1 : 0;
  uint8_t* w = static_cast<uint8_t*>(ws);
  uint32_t limit = spin_limit();
  unsigned* status = device_status_word();
  void* args[] = {(void*)&in, (void*)&out, (void*)&n, (void*)&S, (void*)&resident, (void*)&vec,
                  (void*)&w,  (void*)&limit, (void*)&status};
  if (cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)G), dim3(kGbThreads), args, smem, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return COX_ECUDA;
  }
  return COX_OK;
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_grid_broadcast_workspace(int64_t n) {
  (void)n;
  return kGbWsHeader + (size_t)sm_count() * 8 * 8;  // partials of up to 8 CTAs per SM
}

extern "C" cox_status cox_grid_broadcast(cox_gridop op, cox_dtype dt, const void* d_in, void* d_out, int64_t n,
                                         void* d_workspace, size_t workspace_bytes, void* stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_out))) return COX_EINVAL;
  if (op != COX_GRID_SUB_MIN && op != COX_GRID_NORMALIZE) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32 && dt != COX_F32) return COX_EINVAL;
  if (op == COX_GRID_NORMALIZE && dt != COX_F32) return COX_EINVAL;
  if (n == 0) return COX_OK;
  if (!d_workspace || workspace_bytes < cox_grid_broadcast_workspace(n)) return COX_ENOMEM;
  if (!aligned16(d_workspace)) return COX_EINVAL;
  cudaStream_t st = as_stream(stream);
  if (op == COX_GRID_NORMALIZE) return launch_gb<COX_GRID_NORMALIZE, COX_F32>(d_in, d_out, n, d_workspace, st);
  if (dt == COX_I32) return launch_gb<COX_GRID_SUB_MIN, COX_I32>(d_in, d_out, n, d_workspace, st);
  if (dt == COX_U32) return launch_gb<COX_GRID_SUB_MIN, COX_U32>(d_in, d_out, n, d_workspace, st);
  return launch_gb<COX_GRID_SUB_MIN, COX_F32>(d_in, d_out, n, d_workspace, st);
}
