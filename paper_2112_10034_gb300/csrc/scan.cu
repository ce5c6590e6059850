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
// (scan_row_regs in cox_common.cuh: each width-W tile collapsed into one
// thread's registers.)

// Persistent warps stream chunks of 32 rows through row_ring: a chunk is
// read row per lane, scanned in registers, written back in place and stored
// by TMA.  `n / 32` full rows go through the tensor maps (>= 1 row); the last
// n % 32 elements are scanned by thread 0 of CTA 0 from global memory.
template <class R, int W>
__global__ void __launch_bounds__(kRingWarps * 32, 2)
    k_tile_scan_rows(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                     const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n, uint32_t limit,
                     unsigned* status) {
  using T = typename R::T;
  using V = typename R::V;
  const int lane = threadIdx.x & 31;
  const int64_t rows = n / 32;
  row_ring<true>(&tin, &tout, (rows + 31) / 32, limit, status, [&](int64_t, uint4* buf) {
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
  });
  // The last n % 32 elements: one lane, padded.
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
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmem) != cudaSuccess)
      return COX_ECUDA;
    grid_cache = persistent_grid(k, kRingWarps * 32, kRingSmem, 1 << 30);
  }
  const int64_t nch = (rows + 31) / 32;
  const int64_t ctas = (nch + kRingWarps - 1) / kRingWarps;
  const int grid = (int)(ctas < grid_cache ? ctas : grid_cache);
  k<<<grid, kRingWarps * 32, kRingSmem, st>>>(tin, tout, static_cast<const uint32_t*>(in),
                                              static_cast<uint32_t*>(out), n, spin_limit(), device_status_word());
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
