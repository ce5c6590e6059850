// cox_tile_reduce: tile, block and grid reductions.
//
// Code 1 of the paper is the warp stage: for offset = W/2 .. 1,
// v = v op shfl_down(v, offset) leaves the tile's value in its rank-0 lane
// (Section 2.3).  The block stage follows the SDK reduction kernels named in
// Table 1: tile partials go to shared memory and warp 0 combines them -- lane
// l folds partials l, l+32, ... into an accumulator that starts at the
// identity, then a width-32 shfl_down tree.  Integer width-32 trees use
// redux.sync (exact, so the order does not matter for integers).
//
// TILE and BLOCK results follow that order exactly in every kernel here, so
// fp32 results are the same bits whichever kernel runs.  GRID scope folds
// elements per thread first (tolerance-checked for fp32) and combines the
// per-CTA partials in CTA order in the last CTA to finish.
#include "cox_common.cuh"
#include "reduce_block_rows.cuh"

namespace cox {


constexpr int kRedRows = 8;
constexpr int kGridMaxCtas = 4096;
constexpr size_t kGridWsHeader = 256;

// ---------------------------------------------------------------- TILE scope
template <class R, int W, int ROWS>
__global__ void __launch_bounds__(1024) k_reduce_tile(const uint32_t* __restrict__ in,
                                                      uint32_t* __restrict__ out, float* __restrict__ lo,
                                                      int64_t n, int vec) {
  using T = typename R::T;
  extern __shared__ uint32_t smem[];
  uint32_t* sm = smem + (threadIdx.x >> 5) * (ROWS * 32);
  constexpr int64_t CH = ROWS * 32;
  const int64_t nchunks = (n + CH - 1) / CH;
  const int64_t nfull = vec ? n / CH : 0;
  const int64_t ntiles = (n + W - 1) / W;
  const int lane = lane_id();
  const int64_t wpb = blockDim.x >> 5;
  const uint32_t pad = to_bits(R::pad());
  for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks; c += gridDim.x * wpb) {
    const int64_t base = c * CH;
    uint32_t row[ROWS];
    if (c < nfull) load_rows_full<ROWS>(in + base, sm, row);
    else load_rows_tail<ROWS>(in + base, n - base, pad, row);
    typename R::V v[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) v[r] = tile_tree<R, W>(R::load(from_bits<T>(row[r])));
    if ((lane & (W - 1)) == 0) {
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const int64_t t = (base + r * 32 + lane) / W;
        if (t < ntiles) {
          out[t] = to_bits(R::out(v[r]));
          if (lo) lo[t] = R::lo(v[r]);
        }
      }
    }
  }
}

// ------------------------------------------- TILE scope, one row per lane
// Code 1's tree with each width-W tile collapsed into one thread (the
// paper's intra-warp loop): for offset = W/2 .. 1, x[i] = x[i] op x[i + offset]
// for i < offset -- the operands the rank-i lane combines in the shuffle form
// (lanes at or past the offset only compute values that rank 0 never reads).
// Same combines, same order, same bits.
template <class R, int W>
__device__ __forceinline__ void reduce_row_regs(typename R::V (&v)[32]) {
#pragma unroll
  for (int t0 = 0; t0 < 32; t0 += W)
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < off; ++i) v[t0 + i] = R::op(v[t0 + i], v[t0 + i + off]);
}

// Writes the 32 / W tile results of one row (tiles t0 .. t0 + 32/W - 1);
// used for the partial last row.
template <class R, int W>
__device__ __forceinline__ void reduce_row_out(const typename R::V (&v)[32], int64_t t0, int64_t ntiles,
                                               uint32_t* __restrict__ out, float* __restrict__ lo) {
  constexpr int NT = 32 / W;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (t0 + j < ntiles) {
      out[t0 + j] = to_bits(R::out(v[j * W]));
      if (lo) lo[t0 + j] = R::lo(v[j * W]);
    }
  }
}

// Writes the chunk's results (lane t's NT values at shared word t*P + j, P =
// NT + 1 for NT > 1 so that the 32 lanes' writes hit 32 banks) to dst[0 ..
// cnt) in tile order with coalesced warp stores.
template <int NT>
__device__ __forceinline__ void copy_out_padded(const uint32_t* so, uint32_t* __restrict__ dst, int cnt, int lane) {
  constexpr int P = NT > 1 ? NT + 1 : 1;
  for (int e = lane; e < cnt; e += 32) dst[e] = so[(e / NT) * P + (e % NT)];
}

// Persistent warps stream chunks of 32 rows through row_ring (load only);
// lane t reduces row t's NT = 32 / W tiles in registers.  The chunk's
// 32 x NT results (tiles (32c + t) NT + j, contiguous) are staged in the
// chunk's own buffer -- free once every lane holds its row -- and leave by
// coalesced warp stores; then the low words the same way.  The last n % 32 elements (a
// partial row, padded) go to thread 0 of CTA 0.
template <class R, int W>
__global__ void __launch_bounds__(kRingWarps * 32, 2)
    k_reduce_tile_rows(const __grid_constant__ CUtensorMap tin, const uint32_t* __restrict__ in,
                       uint32_t* __restrict__ out, float* __restrict__ lo, int64_t n, uint32_t limit,
                       unsigned* status) {
  using T = typename R::T;
  using V = typename R::V;
  constexpr int NT = 32 / W;
  const int lane = threadIdx.x & 31;
  const int64_t rows = n / 32;
  const int64_t ntiles = (n + W - 1) / W;
  row_ring<false>(&tin, nullptr, (rows + 31) / 32, limit, status, [&](int64_t c, uint4* buf) {
    V v[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 q = buf[lane * 8 + (j ^ (lane & 7))];
      v[4 * j] = R::load(from_bits<T>(q.x));
      v[4 * j + 1] = R::load(from_bits<T>(q.y));
      v[4 * j + 2] = R::load(from_bits<T>(q.z));
      v[4 * j + 3] = R::load(from_bits<T>(q.w));
    }
    reduce_row_regs<R, W>(v);
    __syncwarp();  // every lane holds its row: the buffer is free for the results
    constexpr int P = NT > 1 ? NT + 1 : 1;
    uint32_t* so = reinterpret_cast<uint32_t*>(buf);
    const int64_t r0 = c * 32;
    const int valid = (int)((rows - r0 < 32 ? rows - r0 : 32) * NT);  // rows past the end are not written
#pragma unroll
    for (int j = 0; j < NT; ++j) so[lane * P + j] = to_bits(R::out(v[j * W]));
    __syncwarp();
    copy_out_padded<NT>(so, out + r0 * NT, valid, lane);
    if (lo) {
      __syncwarp();
#pragma unroll
      for (int j = 0; j < NT; ++j) so[lane * P + j] = __float_as_uint(R::lo(v[j * W]));
      __syncwarp();
      copy_out_padded<NT>(so, reinterpret_cast<uint32_t*>(lo) + r0 * NT, valid, lane);
    }
  });
  if (blockIdx.x == 0 && threadIdx.x == 0 && rows * 32 < n) {
    const int64_t b = rows * 32;
    const int m = (int)(n - b);
    V v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = R::load(i < m ? from_bits<T>(in[b + i]) : R::pad());
    reduce_row_regs<R, W>(v);
    reduce_row_out<R, W>(v, rows * NT, ntiles, out, lo);
  }
}

// -------------------------------------------- BLOCK scope, one CTA per block
// The CUDA-shaped kernel (Code 1 inside an SDK-style block reduction): the
// CTA is the logical block.  Used when the grid is small (e.g. 64 blocks).
template <class R, int W>
__global__ void __launch_bounds__(1024) k_reduce_block_cta(const uint32_t* __restrict__ in,
                                                           uint32_t* __restrict__ out,
                                                           float* __restrict__ lo, int64_t n) {
  using T = typename R::T;
  using V = typename R::V;
  extern __shared__ uint8_t smem_raw[];
  V* part = reinterpret_cast<V*>(smem_raw);
  const int B = blockDim.x;
  const int P = B / W;
  const int tid = threadIdx.x;
  const int64_t nblk = (n + B - 1) / B;
  for (int64_t lb = blockIdx.x; lb < nblk; lb += gridDim.x) {
    const int64_t i = lb * B + tid;
    const T x = i < n ? from_bits<T>(__ldcs(in + i)) : R::pad();
    const V v = tile_tree<R, W>(R::load(x));
    if ((tid & (W - 1)) == 0) part[tid / W] = v;
    __syncthreads();
    if (tid < 32) {
      V acc = R::ident();
      for (int k = tid; k < P; k += 32) acc = R::op(acc, part[k]);
      acc = tile_tree<R, 32>(acc);
      if (tid == 0) {
        out[lb] = to_bits(R::out(acc));
        if (lo) lo[lb] = R::lo(acc);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------- BLOCK scope, persistent warp per group
// Each warp takes K = max(1, 256 / B) whole logical blocks at a time (S = K*B
// elements), streams their rows through the staging layer in groups of
// 8/4/2/1 rows, keeps the tile partials in warp-private shared memory, then
// folds each logical block exactly as the CTA kernel's warp 0 does.
template <class R, int W, int G>
__device__ __forceinline__ void block_rows(const uint32_t* __restrict__ in, int64_t n, int64_t gbase,
                                           int q0, uint32_t* stage, typename R::V* part, int vec) {
  using T = typename R::T;
  const int lane = lane_id();
  uint32_t row[G];
  const int64_t b = gbase + (int64_t)q0 * 32;
  if (vec && b + G * 32 <= n) load_rows_full<G>(in + b, stage, row);
  else load_rows_tail<G>(in + b, n - b, to_bits(R::pad()), row);
#pragma unroll
  for (int r = 0; r < G; ++r) {
    const typename R::V v = tile_tree<R, W>(R::load(from_bits<T>(row[r])));
    if ((lane & (W - 1)) == 0) part[((q0 + r) * 32 + lane) / W] = v;
  }
}

template <class R, int W>
__global__ void __launch_bounds__(256) k_reduce_block_warp(const uint32_t* __restrict__ in,
                                                           uint32_t* __restrict__ out,
                                                           float* __restrict__ lo, int64_t n, int B,
                                                           int vec) {
  using V = typename R::V;
  extern __shared__ uint8_t smem_raw[];
  const int K = B >= 256 ? 1 : 256 / B;
  const int S = K * B;
  const int P = B / W;
  const int warp = threadIdx.x >> 5;
  const int lane = lane_id();
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem_raw) + warp * 256;
  V* part = reinterpret_cast<V*>(reinterpret_cast<uint32_t*>(smem_raw) + (blockDim.x >> 5) * 256) +
            warp * (S / W);
  const int64_t nblk = (n + B - 1) / B;
  const int64_t nsuper = (nblk + K - 1) / K;
  const int64_t wpb = blockDim.x >> 5;
  const int rows = S / 32;
  for (int64_t sc = blockIdx.x * wpb + warp; sc < nsuper; sc += gridDim.x * wpb) {
    const int64_t gbase = sc * S;
    int q = 0;
    for (; q + 8 <= rows; q += 8) block_rows<R, W, 8>(in, n, gbase, q, stage, part, vec);
    if (q + 4 <= rows) { block_rows<R, W, 4>(in, n, gbase, q, stage, part, vec); q += 4; }
    if (q + 2 <= rows) { block_rows<R, W, 2>(in, n, gbase, q, stage, part, vec); q += 2; }
    if (q + 1 <= rows) { block_rows<R, W, 1>(in, n, gbase, q, stage, part, vec); q += 1; }
    __syncwarp();
    for (int j = 0; j < K; ++j) {
      const int64_t lb = sc * K + j;
      if (lb >= nblk) break;
      V acc = R::ident();
      for (int k = lane; k < P; k += 32) acc = R::op(acc, part[j * P + k]);
      acc = tile_tree<R, 32>(acc);
      if (lane == 0) {
        out[lb] = to_bits(R::out(acc));
        if (lo) lo[lb] = R::lo(acc);
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- GRID scope
// Per thread: fold a grid-stride sequence of 128-bit loads (four independent
// loads in flight per thread); then the block stage above (W = 32); CTA
// partial to the workspace; the last CTA to arrive folds all partials in CTA
// order (FP64 for F32 sums with fp64 set) and re-arms the counter.
__device__ __forceinline__ double block_reduce_f64(double v, double* wpart) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (lane == 0) wpart[warp] = v;
  __syncthreads();
  double acc = 0.0;
  if (warp == 0) {
    for (int k = lane; k < (int)(blockDim.x >> 5); k += 32) acc += wpart[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(kFull, acc, off);
  }
  __syncthreads();
  return acc;
}

template <class R>
__global__ void __launch_bounds__(1024) k_reduce_grid(const uint32_t* __restrict__ in, int64_t n,
                                                      typename R::V* ws_part, unsigned* ws_ctr,
                                                      uint32_t* __restrict__ out, float* __restrict__ lo,
                                                      int fp64, int vec) {
  using T = typename R::T;
  using V = typename R::V;
  __shared__ V wpart[32];
  __shared__ double wpart64[32];
  __shared__ int s_last;
  V acc = R::ident();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  int64_t tail0 = 0;
  if (vec) {
    const uint4* p = reinterpret_cast<const uint4*>(in);
    const int64_t nv = n / 4;
    int64_t i = gt;
    for (; i + 3 * gs < nv; i += 4 * gs) {
      uint4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = __ldcs(p + i + u * gs);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc = R::op(acc, R::load(from_bits<T>(q[u].x)));
        acc = R::op(acc, R::load(from_bits<T>(q[u].y)));
        acc = R::op(acc, R::load(from_bits<T>(q[u].z)));
        acc = R::op(acc, R::load(from_bits<T>(q[u].w)));
      }
    }
    for (; i < nv; i += gs) {
      const uint4 q = __ldcs(p + i);
      acc = R::op(acc, R::load(from_bits<T>(q.x)));
      acc = R::op(acc, R::load(from_bits<T>(q.y)));
      acc = R::op(acc, R::load(from_bits<T>(q.z)));
      acc = R::op(acc, R::load(from_bits<T>(q.w)));
    }
    tail0 = nv * 4;
  }
  for (int64_t i = tail0 + gt; i < n; i += gs) acc = R::op(acc, R::load(from_bits<T>(in[i])));
  const V bsum = block_reduce32<R>(acc, wpart);
  if (threadIdx.x == 0) {
    ws_part[blockIdx.x] = bsum;
    __threadfence();
    s_last = atomicAdd(ws_ctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int G = gridDim.x;
  if constexpr (R::kComp) {
    if (fp64) {
      double d = 0.0;
      for (int k = threadIdx.x; k < G; k += blockDim.x) {
        const float2 f = __ldcg(reinterpret_cast<const float2*>(ws_part) + k);
        d += (double)f.x + (double)f.y;
      }
      const double total = block_reduce_f64(d, wpart64);
      if (threadIdx.x == 0) {
        const float y = (float)total;
        out[0] = to_bits(y);
        if (lo) lo[0] = (float)(total - (double)y);
        *ws_ctr = 0u;
      }
      return;
    }
  }
  V fold = R::ident();
  for (int k = threadIdx.x; k < G; k += blockDim.x) {
    V pv;
    if constexpr (R::kComp) {
      const float2 f = __ldcg(reinterpret_cast<const float2*>(ws_part) + k);
      pv = {f.x, f.y};
    } else {
      pv = from_bits<T>(__ldcg(reinterpret_cast<const uint32_t*>(ws_part) + k));
    }
    fold = R::op(fold, pv);
  }
  const V total = block_reduce32<R>(fold, wpart);
  if (threadIdx.x == 0) {
    out[0] = to_bits(R::out(total));
    if (lo) lo[0] = R::lo(total);
    *ws_ctr = 0u;
  }
}

// ------------------------------------------------------------------ launch
template <class R, int W>
static cox_status launch_reduce(cox_scope scope, const void* d_in, void* d_out, float* d_lo, int64_t n, int B,
                                unsigned flags, void* ws, size_t ws_bytes, cudaStream_t st) {
  const uint32_t* in = static_cast<const uint32_t*>(d_in);
  uint32_t* out = static_cast<uint32_t*>(d_out);
  const int vec = aligned16(d_in);
  using V = typename R::V;
  if (scope == COX_SCOPE_TILE && n >= 32 && n / 32 < (int64_t(1) << 31) && aligned16(d_in)) {
    // Aligned arrays of at least one full row: the row-per-lane kernel.
    const int64_t rows = n / 32;
    CUtensorMap tin;
    if (!encode_rows32_map(&tin, d_in, rows, 32)) return COX_ECUDA;
    auto k = k_reduce_tile_rows<R, W>;
    static int gmax_rows;
    if (gmax_rows == 0) {
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmem) != cudaSuccess)
        return COX_ECUDA;
      gmax_rows = persistent_grid(k, kRingWarps * 32, kRingSmem, 1 << 30);
    }
    const int64_t ctas = ((rows + 31) / 32 + kRingWarps - 1) / kRingWarps;
    k<<<(int)(ctas < gmax_rows ? ctas : gmax_rows), kRingWarps * 32, kRingSmem, st>>>(
        tin, in, out, d_lo, n, spin_limit(), device_status_word());
    return launch_status();
  }
  if (scope == COX_SCOPE_TILE) {
    auto k = k_reduce_tile<R, W, kRedRows>;
    const int block = 256;
    const size_t smem = (block / 32) * kRedRows * 32 * 4;
    static int gmax;
    if (gmax == 0) gmax = persistent_grid(k, block, smem, 1 << 30);
    const int64_t chunks = (n + kRedRows * 32 - 1) / (kRedRows * 32);
    const int64_t ctas = (chunks + block / 32 - 1) / (block / 32);
    k<<<(int)(ctas < gmax ? ctas : gmax), block, smem, st>>>(in, out, d_lo, n, vec);
    return launch_status();
  }
  if (scope == COX_SCOPE_BLOCK) {
    const int64_t nblk = (n + B - 1) / B;
    // One wave of CTA-per-block kernels is the low-latency path for small
    // grids; beyond that, persistent warps stream the input.
    if (nblk <= (int64_t)sm_count() * 4) {
      auto k = k_reduce_block_cta<R, W>;
      const size_t smem = (size_t)(B / W) * sizeof(V);
      k<<<(int)nblk, B, smem, st>>>(in, out, d_lo, n);
      return launch_status();
    }
    if ((B & (B - 1)) == 0 && n >= 32 && n / 32 < (int64_t(1) << 31) && aligned16(d_in))
      return block_rows_launch<R>(W, B, d_in, d_out, d_lo, n, st);
    auto k = k_reduce_block_warp<R, W>;
    const int block = 256;
    const int K = B >= 256 ? 1 : 256 / B;
    const size_t smem = (size_t)(block / 32) * (256 * 4 + (size_t)(K * B / W) * sizeof(V));
    static int gmax[33];
    int& g = gmax[B / 32];
    if (g == 0) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      g = persistent_grid(k, block, smem, 1 << 30);
    }
    const int64_t nsuper = (nblk + K - 1) / K;
    const int64_t ctas = (nsuper + block / 32 - 1) / (block / 32);
    k<<<(int)(ctas < g ? ctas : g), block, smem, st>>>(in, out, d_lo, n, B, vec);
    return launch_status();
  }
  // GRID
  if (!ws || ws_bytes < cox_tile_reduce_workspace(COX_SCOPE_GRID, n, B)) return COX_ENOMEM;
  if (!aligned16(ws)) return COX_EINVAL;
  auto k = k_reduce_grid<R>;
  const int block = 512;
  static int gmax;
  if (gmax == 0) gmax = persistent_grid(k, block, 0, kGridMaxCtas);
  const int64_t ctas = (n + (int64_t)block * 16 - 1) / ((int64_t)block * 16);
  int grid = (int)(ctas < gmax ? ctas : gmax);
  if (grid < 1) grid = 1;
  unsigned* ctr = static_cast<unsigned*>(ws);
  V* part = reinterpret_cast<V*>(static_cast<char*>(ws) + kGridWsHeader);
  if (cudaMemsetAsync(ctr, 0, sizeof(unsigned), st) != cudaSuccess) return COX_ECUDA;
  k<<<grid, block, 0, st>>>(in, n, part, ctr, out, d_lo, (flags & COX_F_FP64_COMBINE) ? 1 : 0, vec);
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_tile_reduce_workspace(cox_scope scope, int64_t n, int block_dim) {
  (void)n;
  (void)block_dim;
  return scope == COX_SCOPE_GRID ? kGridWsHeader + (size_t)kGridMaxCtas * 16 : 0;
}

extern "C" cox_status cox_tile_reduce(cox_op op, cox_dtype dt, int width, int block_dim, cox_scope scope,
                                      const void* d_in, void* d_out, int64_t n, unsigned flags, void* d_err,
                                      void* d_workspace, size_t workspace_bytes, void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (scope != COX_SCOPE_TILE && scope != COX_SCOPE_BLOCK && scope != COX_SCOPE_GRID) return COX_EINVAL;
  if (flags & ~(unsigned)(COX_F_COMPENSATED | COX_F_FP64_COMBINE)) return COX_EINVAL;
  const bool comp = flags & COX_F_COMPENSATED;
  if ((flags & COX_F_FP64_COMBINE) && !(comp && scope == COX_SCOPE_GRID)) return COX_EINVAL;
  if (!d_out || (n > 0 && !d_in)) return COX_EINVAL;
  float* lo = comp ? static_cast<float*>(d_err) : nullptr;
  return with_reducer(op, dt, comp, [&](auto r) {
    using R = decltype(r);
    return with_width(width, [&](auto w) {
      if (n == 0 && scope != COX_SCOPE_GRID) return COX_OK;
      return launch_reduce<R, decltype(w)::value>(scope, d_in, d_out, lo, n, block_dim, flags, d_workspace,
                                                  workspace_bytes, as_stream(stream));
    });
  });
}
