// BLOCK-scope reduction with one row per lane, for power-of-two block sizes.
//
// The order is the BLOCK scope's of reduce.cu, step for step: Code 1's
// width-W tree per tile (collapsed into one thread, as the paper's
// intra-warp loop does), tile partials in tile order, then the block stage
// of the SDK reduction kernels (Table 1): accumulator l starts at the
// identity and folds partials l, l + 32, ..., and a width-32 tree over the
// 32 accumulators gives the block's value.  Here the accumulators are
// computed one per lane (through shared memory when a block has more than
// 32 tile partials) and the trees run as shuffles across the lanes; when a
// block has at most 32 partials each accumulator holds one partial and the
// tree runs within the block's own lanes (for 32-element blocks, each lane
// owns a block and runs its tree in registers) -- the same combines in the
// same order, so the same bits as the shuffle kernels.
//
// A chunk of 32 rows (1024 elements) holds LB = 1024 / B whole logical
// blocks of RB = B / 32 rows and P = B / W tile partials each.  Logical
// blocks made of full 32-element rows come from the TMA ring; the last
// logical block, when it reaches into the partial last row, is reduced by
// warp 0 of CTA 0 from global memory with padding.
#pragma once

#include "cox_common.cuh"

namespace cox {

// Launches the BLOCK-scope rows kernel for reducer R (power-of-two B, a
// 16-byte aligned input of at least 32 elements and fewer than 2^36).
// Instantiated in reduce_block_rows_{a,b,c,d}.cu, three reducers per file,
// so that the kernels compile in parallel.
template <class R>
cox_status block_rows_launch(int W, int B, const void* in, void* out, float* lo, int64_t n, cudaStream_t st);

#ifdef COX_BLOCK_ROWS_IMPL

template <class R, int W>
__device__ __forceinline__ void reduce_row_regs_b(typename R::V (&v)[32]) {
#pragma unroll
  for (int t0 = 0; t0 < 32; t0 += W)
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < off; ++i) v[t0 + i] = R::op(v[t0 + i], v[t0 + i + off]);
}

// Width-32 tree over 32 accumulators held by one thread (Code 1's offsets).
template <class R>
__device__ __forceinline__ typename R::V tree32_regs(typename R::V (&a)[32]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < off; ++i) a[i] = R::op(a[i], a[i + off]);
  return a[0];
}

// Shared-memory slot of chunk partial q: the XOR of q's 32-block index into
// its low bits spreads both the writes (lane stride NT) and the reads (lane
// stride 1) over the banks.
__device__ __forceinline__ int part_slot(int q) { return q ^ ((q >> 5) & 31); }

// Block stage for the LB logical blocks of one chunk.  `v` holds this lane's
// row after the tile trees (tile j's value at v[j * W]); logical block
// lb0 + b is written when lb0 + b < nvalid.  `smem` is a free 4 KB buffer.
template <class R, int W>
__device__ __forceinline__ void block_stage(typename R::V (&v)[32], void* smem, int B, int64_t lb0, int64_t nvalid,
                                            uint32_t* __restrict__ out, float* __restrict__ lo, int lane) {
  using V = typename R::V;
  constexpr int NT = 32 / W;
  if (B == 32) {  // the logical block is this lane's row
    V a[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) a[l] = l < NT ? R::op(R::ident(), v[l * W]) : R::ident();
    const V r = tree32_regs<R>(a);
    if (lb0 + lane < nvalid) {
      out[lb0 + lane] = to_bits(R::out(r));
      if (lo) lo[lb0 + lane] = R::lo(r);
    }
    return;
  }
  const int LB = 1024 / B, P = B / W;
  if (P <= 32) {
    // Accumulator l < P is (ident op partial l), the others stay identities,
    // so the width-32 tree combines position i < P with an identity at every
    // offset >= P, and at offsets below P with position i + off.  Position
    // i = r * NT + j sits in slot j of the block's lane r (RB = B / 32 lanes
    // per block): partners at offsets >= NT are lanes further down (a shuffle
    // within the block for every position that is still read), partners at
    // smaller offsets are slots of the same lane.  Same combines, same order.
    const int RB = B / 32;
    V a[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) a[j] = R::op(R::ident(), v[j * W]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      if (off >= P) {
#pragma unroll
        for (int j = 0; j < NT; ++j) a[j] = R::op(a[j], R::ident());
      } else if (off >= NT) {
#pragma unroll
        for (int j = 0; j < NT; ++j) a[j] = R::op(a[j], R::shfl_down(a[j], off / NT, 32));
      } else {
#pragma unroll
        for (int j = 0; j < NT; ++j)
          if (j < off) a[j] = R::op(a[j], a[j + off]);
      }
    }
    const int64_t blk = lb0 + lane / RB;
    if (lane % RB == 0 && blk < nvalid) {
      out[blk] = to_bits(R::out(a[0]));
      if (lo) lo[blk] = R::lo(a[0]);
    }
    return;
  }
  // More than 32 partials per block (P = 64 .. 512, so LB <= 8): the
  // partials go through shared memory, lane l folds accumulator l of each
  // block in order, and the width-32 tree runs across the lanes by shuffles.
  V* sp = reinterpret_cast<V*>(smem);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < NT; ++j) sp[part_slot(lane * NT + j)] = v[j * W];  // partial q = b * P + k
  __syncwarp();
#pragma unroll 1
  for (int b = 0; b < LB; ++b) {
    V acc = R::ident();
    for (int k = lane; k < P; k += 32) acc = R::op(acc, sp[part_slot(b * P + k)]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = R::op(acc, R::shfl_down(acc, off, 32));
    if (lane == 0 && lb0 + b < nvalid) {
      out[lb0 + b] = to_bits(R::out(acc));
      if (lo) lo[lb0 + b] = R::lo(acc);
    }
  }
  __syncwarp();
}

// The last logical block when it is not made of full rows: lane t takes its
// row t (padded past n); the block is presented as a chunk's first logical
// block, and only it is written (nvalid = nfull + 1).  Run once per launch,
// so kept out of line.
template <class R, int W>
__device__ __noinline__ void tail_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                        float* __restrict__ lo, int64_t n, int B, int64_t nfull, void* sm, int lane) {
  using T = typename R::T;
  using V = typename R::V;
  const int64_t b0 = nfull * B;
  const int rb = B / 32;
  V v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int64_t e = b0 + (int64_t)lane * 32 + i;
    v[i] = R::load(lane < rb && e < n ? from_bits<T>(in[e]) : R::pad());
  }
  reduce_row_regs_b<R, W>(v);
  block_stage<R, W>(v, sm, B, nfull, nfull + 1, out, lo, lane);
}

template <class R, int W>
__global__ void __launch_bounds__(kRingWarps * 32, 2)
    k_reduce_block_rows(const __grid_constant__ CUtensorMap tin, const uint32_t* __restrict__ in,
                        uint32_t* __restrict__ out, float* __restrict__ lo, int64_t n, int B, uint32_t limit,
                        unsigned* status) {
  using T = typename R::T;
  using V = typename R::V;
  const int lane = threadIdx.x & 31;
  const int64_t rows = n / 32;
  const int LB = 1024 / B;
  const int64_t nfull = rows * 32 / B;  // logical blocks of full rows only
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
    reduce_row_regs_b<R, W>(v);
    block_stage<R, W>(v, buf, B, c * LB, nfull, out, lo, lane);
  });
  if (blockIdx.x == 0 && threadIdx.x < 32 && nfull < (n + B - 1) / B) {
    extern __shared__ uint8_t tail_smem_raw[];  // warp 0's first ring buffer, idle now
    void* sm = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(tail_smem_raw) + 1023) & ~uintptr_t(1023));
    tail_block<R, W>(in, out, lo, n, B, nfull, sm, lane);
  }
}

template <class R, int W>
static cox_status launch_block_rows(const void* in, void* out, float* lo, int64_t n, int B, cudaStream_t st) {
  const int64_t rows = n / 32;
  CUtensorMap tin;
  if (!encode_rows32_map(&tin, in, rows, 32)) return COX_ECUDA;
  auto k = k_reduce_block_rows<R, W>;
  static int gmax;
  if (gmax == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmem) != cudaSuccess)
      return COX_ECUDA;
    gmax = persistent_grid(k, kRingWarps * 32, kRingSmem, 1 << 30);
  }
  const int64_t ctas = ((rows + 31) / 32 + kRingWarps - 1) / kRingWarps;
  const int grid = (int)(ctas < gmax ? ctas : gmax);
  k<<<grid < 1 ? 1 : grid, kRingWarps * 32, kRingSmem, st>>>(tin, static_cast<const uint32_t*>(in),
                                                              static_cast<uint32_t*>(out), lo, n, B, spin_limit(),
                                                              device_status_word());
  return launch_status();
}

template <class R>
cox_status block_rows_launch(int W, int B, const void* in, void* out, float* lo, int64_t n, cudaStream_t st) {
  return with_width(W, [&](auto w) { return launch_block_rows<R, decltype(w)::value>(in, out, lo, n, B, st); });
}
#endif  // COX_BLOCK_ROWS_IMPL

}  // namespace cox
