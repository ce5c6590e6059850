// cox_tile_scan: inclusive scan inside cooperative-groups tiles of width W.
//
// The shuffle scan of the SDK kernel shfl_scan_test (Table 1 of the paper),
// run on a tile: Hillis-Steele steps d = 1, 2, .., W/2 of
//   u = shfl_up(x, d, W); if (rank >= d) x = u op x
// with the lane numbering of Code 3 (element i is global thread i's operand).
// Persistent warps stream chunks of ROWS x 32 elements: 128-bit loads,
// a warp-private shared-memory transpose to one element per lane per row,
// ROWS independent shuffle chains (instruction-level parallelism), and the
// inverse transpose to 128-bit stores.
#include "cox_common.cuh"

namespace cox {

// Rows per warp chunk: plain scans are memory-bound and take 8 rows (two
// 128-bit loads per lane); compensated scans are issue-bound and take 16
// independent rows for instruction-level parallelism (measured ~10% faster at
// width 32 on GB300 than 8 rows with more warps).
template <class R>
constexpr int scan_rows() {
  return R::kComp ? 16 : 8;
}

template <class R, int W, int ROWS>
__global__ void __launch_bounds__(R::kComp ? 256 : 1024) k_tile_scan(const uint32_t* __restrict__ in,
                                                   uint32_t* __restrict__ out, int64_t n, int vec) {
  extern __shared__ uint32_t smem[];
  uint32_t* sm = smem + (threadIdx.x >> 5) * (ROWS * 32);
  constexpr int64_t CH = ROWS * 32;
  const int64_t nchunks = (n + CH - 1) / CH;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks; c += gridDim.x * wpb)
    scan_chunk<R, W, ROWS>(in, out, n, c, sm, vec != 0);
}

// ------------------------------------------------ one tile row per lane
// The same Hillis-Steele combines with each width-W tile collapsed into one
// thread -- the paper's intra-warp loop (Section 3), applied on the GPU: lane
// t of a warp holds row t (32 consecutive elements, 32/W tiles) of the warp's
// 1024-element chunk, and step d sets x[i] = x[i-d] op x[i] for rank i from
// W-1 down to d, so x[i-d] still holds the previous step's value, exactly as
// the shuffle's source lane does.  Same operands in the same order, hence the
// same bits, with no shuffles, selects or idle lanes.
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

constexpr int kRowStages = 3;                          // per-warp ring of chunk buffers
constexpr int kRowWarps = 8;                           // 256-thread CTAs
constexpr uint32_t kRowChunkBytes = 32 * 32 * 4;       // 32 rows of 128 B
constexpr size_t kRowSmem = (size_t)kRowWarps * kRowStages * kRowChunkBytes + 1024 + kRowWarps * kRowStages * 8;

// Persistent warps over chunks of 32 rows.  Each warp keeps two chunks in
// flight by 2D TMA (128-byte swizzle) in a 3-stage ring; a chunk is read row
// per lane, scanned in registers, written back in place and leaves by TMA
// store, whose read of the buffer is awaited before the buffer is refilled.
// `rows` = full 32-element rows (>= 1); the n - 32 rows tail elements are
// scanned by warp 0 of CTA 0 from global memory.
template <class R, int W>
__global__ void __launch_bounds__(kRowWarps * 32, 2)
    k_tile_scan_rows(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                     const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n, uint32_t limit,
                     unsigned* status) {
  using T = typename R::T;
  using V = typename R::V;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* ring = base + (size_t)warp * kRowStages * kRowChunkBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)kRowWarps * kRowStages * kRowChunkBytes) +
                   warp * kRowStages;
  const int64_t rows = n / 32;
  const int64_t nch = (rows + 31) / 32;
  const int64_t gw = (int64_t)blockIdx.x * kRowWarps + warp, nw = (int64_t)gridDim.x * kRowWarps;
  if (lane == 0) {
    for (int k = 0; k < kRowStages; ++k) mbar_init(bars + k, 1);
    mbar_init_fence();
    for (int k = 0; k < kRowStages - 1; ++k) {  // prologue: the first two chunks
      const int64_t c = gw + k * nw;
      if (c < nch) {
        mbar_arrive_expect_tx(bars + k, kRowChunkBytes);
        tma_load_2d(ring + k * kRowChunkBytes, &tin, 0, (int)(c * 32), bars + k);
      }
    }
  }
  __syncwarp();
  bool ok = true;
  int64_t k = 0;
  for (int64_t c = gw; c < nch; c += nw, ++k) {
    const int slot = (int)(k % kRowStages);
    uint4* buf = reinterpret_cast<uint4*>(ring + slot * kRowChunkBytes);
    ok = mbar_wait_bounded(bars + slot, (uint32_t)((k / kRowStages) & 1), limit);
    if (!__all_sync(kFull, ok)) {
      ok = false;
      break;
    }
    V v[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // unit j of row `lane` sits at unit j ^ (lane & 7)
      const uint4 q = buf[lane * 8 + (j ^ (lane & 7))];
      v[4 * j] = R::load(from_bits<T>(q.x));
      v[4 * j + 1] = R::load(from_bits<T>(q.y));
      v[4 * j + 2] = R::load(from_bits<T>(q.z));
      v[4 * j + 3] = R::load(from_bits<T>(q.w));
    }
    scan_row_regs<R, W>(v);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      buf[lane * 8 + (j ^ (lane & 7))] = make_uint4(to_bits(R::out(v[4 * j])), to_bits(R::out(v[4 * j + 1])),
                                                    to_bits(R::out(v[4 * j + 2])), to_bits(R::out(v[4 * j + 3])));
    fence_proxy_async_smem();  // this lane's row, before the bulk store reads it
    __syncwarp();
    if (lane == 0) {
      tma_store_2d(&tout, 0, (int)(c * 32), buf);
      const int64_t cn = c + (kRowStages - 1) * nw;  // refill the slot of the previous chunk
      if (cn < nch) {
        const int ns = (int)((k + kRowStages - 1) % kRowStages);
        tma_store_wait_read1();  // the previous chunk's store has read that slot
        mbar_arrive_expect_tx(bars + ns, kRowChunkBytes);
        tma_load_2d(ring + ns * kRowChunkBytes, &tin, 0, (int)(cn * 32), bars + ns);
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (!ok) {  // a load that did not land: record it and give the copies in flight a bounded wait
      atomicOr(status, (unsigned)kDevTimeout);
      for (int j = 0; j < kRowStages - 1; ++j) {
        const int64_t kk = k + j;
        if (gw + kk * nw < nch) mbar_wait_bounded(bars + (int)(kk % kRowStages), (uint32_t)((kk / kRowStages) & 1), limit);
      }
    }
    tma_store_wait_all();  // every store has completed before the CTA ends
  }
  // The last n - 32 rows elements (fewer than 32): one lane, padded.
  if (blockIdx.x == 0 && threadIdx.x == 0 && rows * 32 < n) {
    const int64_t b = rows * 32;
    const int m = (int)(n - b);
    V v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = R::load(i < m ? from_bits<T>(in[b + i]) : R::pad());
    scan_row_regs<R, W>(v);
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < m) out[b + i] = to_bits(R::out(v[i]));
  }
}

template <class R, int W>
static cox_status launch_scan_rows(const void* in, void* out, int64_t n, cudaStream_t st) {
  const int64_t rows = n / 32;
  CUtensorMap tin, tout;
  if (!encode_rows32_map(&tin, in, rows, 32) || !encode_rows32_map(&tout, out, rows, 32)) return COX_ECUDA;
  auto k = k_tile_scan_rows<R, W>;
  static int grid_cache = 0;  // persistent grid (occupancy does not change)
  if (grid_cache == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmem) != cudaSuccess)
      return COX_ECUDA;
    grid_cache = persistent_grid(k, kRowWarps * 32, kRowSmem, 1 << 30);
  }
  const int64_t nch = (rows + 31) / 32;
  const int64_t ctas = (nch + kRowWarps - 1) / kRowWarps;
  const int grid = (int)(ctas < grid_cache ? ctas : grid_cache);
  k<<<grid, kRowWarps * 32, kRowSmem, st>>>(tin, tout, static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out),
                                            n, spin_limit(), device_status_word());
  return launch_status();
}

template <class R, int W>
static cox_status launch_scan(const void* in, void* out, int64_t n, int block, cudaStream_t st) {
  // Aligned arrays of at least one full row take the row-per-lane kernel; the
  // result does not depend on the CTA size, so block_dim is not needed there.
  if (n >= 32 && n / 32 < (int64_t(1) << 31) && aligned16(in) && aligned16(out))
    return launch_scan_rows<R, W>(in, out, n, st);
  constexpr int kScanRows = scan_rows<R>();
  // The result does not depend on the CTA size; compensated scans run 256-thread
  // CTAs so that their 16 rows of pairs fit in registers.
  if (R::kComp && block > 256) block = 256;
  auto k = k_tile_scan<R, W, kScanRows>;
  const size_t smem = (size_t)(block / 32) * kScanRows * 32 * 4;
  const int64_t chunks = (n + kScanRows * 32 - 1) / (kScanRows * 32);
  const int64_t ctas = (chunks + block / 32 - 1) / (block / 32);
  static int grid_cache[33];  // persistent grid per block size (occupancy does not change)
  int& g = grid_cache[block / 32];
  if (g == 0) g = persistent_grid(k, block, smem, 1 << 30);
  const int grid = (int)(ctas < g ? ctas : g);
  const int vec = aligned16(in) && aligned16(out);
  k<<<grid, block, smem, st>>>(static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out), n, vec);
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_tile_scan(cox_op op, cox_dtype dt, int width, int block_dim, const void* d_in,
                                    void* d_out, int64_t n, unsigned flags, void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (flags & ~(unsigned)COX_F_COMPENSATED) return COX_EINVAL;
  if (n > 0 && (!d_in || !d_out)) return COX_EINVAL;
  const bool comp = flags & COX_F_COMPENSATED;
  return with_reducer(op, dt, comp, [&](auto r) {
    using R = decltype(r);
    return with_width(width, [&](auto w) {
      if (n == 0) return COX_OK;
      return launch_scan<R, decltype(w)::value>(d_in, d_out, n, block_dim, as_stream(stream));
    });
  });
}
