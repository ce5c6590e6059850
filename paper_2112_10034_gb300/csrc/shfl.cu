// cox_shfl: one warp-level function on every lane of a grid.
//
// Section 2.2.1 of the paper (warp shuffle and warp vote) with the PTX
// shfl.sync / vote.sync / match.sync semantics it defers to; Code 1 uses
// shfl_down, Code 4 uses __all_sync.  Cooperative-groups tiles of width W
// are the shuffle's segment width; votes and match return tile-local masks.
// Persistent warps stream chunks of 8 x 32 elements through the staging
// layer, so lane l of row r is element base + 32 r + l.
#include "cox_common.cuh"

namespace cox {

constexpr int kShflRows = 8;

template <int FN, int W, bool F32>
__global__ void __launch_bounds__(1024) k_shfl(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                               int64_t n, int param, int vec) {
  extern __shared__ uint32_t smem[];
  uint32_t* sm = smem + (threadIdx.x >> 5) * (kShflRows * 32);
  constexpr int64_t CH = kShflRows * 32;
  const int64_t nchunks = (n + CH - 1) / CH;
  const int64_t nfull = vec ? n / CH : 0;
  const int lane = lane_id();
  const int seg = lane & ~(W - 1);
  const unsigned tbits = W == 32 ? kFull : ((1u << W) - 1u);
  const int64_t wpb = blockDim.x >> 5;
  // Shuffles share the MIO pipe with shared memory, so their full chunks move
  // as coalesced 32-bit rows (row r = one 128-byte access per warp) instead
  // of 128-bit accesses transposed through shared memory.
  constexpr bool kDirect = FN == COX_SHFL_IDX || FN == COX_SHFL_UP || FN == COX_SHFL_DOWN || FN == COX_SHFL_XOR;
  for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks; c += gridDim.x * wpb) {
    const int64_t base = c * CH;
    const bool full = c < nfull;
    uint32_t row[kShflRows];
    if (kDirect && full) {
#pragma unroll
      for (int r = 0; r < kShflRows; ++r) row[r] = __ldcs(in + base + r * 32 + lane);
    } else if (full) {
      load_rows_full<kShflRows>(in + base, sm, row);
    } else {
      load_rows_tail<kShflRows>(in + base, n - base, 0u, row);
    }
#pragma unroll
    for (int r = 0; r < kShflRows; ++r) {
      const uint32_t v = row[r];
      const bool valid = base + r * 32 + lane < n;
      uint32_t res;
      if constexpr (FN == COX_SHFL_IDX) {
        res = __shfl_sync(kFull, v, param, W);
      } else if constexpr (FN == COX_SHFL_UP) {
        res = __shfl_up_sync(kFull, v, param, W);
      } else if constexpr (FN == COX_SHFL_DOWN) {
        res = __shfl_down_sync(kFull, v, param, W);
      } else if constexpr (FN == COX_SHFL_XOR) {
        res = __shfl_xor_sync(kFull, v, param, W);
      } else if constexpr (FN == COX_MATCH_ANY) {
        const unsigned vb = __ballot_sync(kFull, valid);
        res = ((__match_any_sync(kFull, v) & vb) >> seg) & tbits;
      } else {
        const bool p = valid && (F32 ? __uint_as_float(v) != 0.0f : v != 0u);
        const unsigned tb = (__ballot_sync(kFull, p) >> seg) & tbits;
        if constexpr (FN == COX_BALLOT) res = tb;
        else if constexpr (FN == COX_ANY) res = tb != 0u;
        else res = tb == tbits;
      }
      row[r] = res;
    }
    if (kDirect && full) {
#pragma unroll
      for (int r = 0; r < kShflRows; ++r) __stcs(out + base + r * 32 + lane, row[r]);
    } else if (full) {
      store_rows_full<kShflRows>(out + base, sm, row);
    } else {
      store_rows_tail<kShflRows>(out + base, n - base, row);
    }
  }
}

template <int FN, int W, bool F32>
static cox_status launch_shfl(const void* in, void* out, int64_t n, int param, int block, cudaStream_t st) {
  auto k = k_shfl<FN, W, F32>;
  const size_t smem = (size_t)(block / 32) * kShflRows * 32 * 4;
  static int gmax[33];
  int& g = gmax[block / 32];
  if (g == 0) g = persistent_grid(k, block, smem, 1 << 30);
  const int64_t chunks = (n + kShflRows * 32 - 1) / (kShflRows * 32);
  const int64_t ctas = (chunks + block / 32 - 1) / (block / 32);
  const int vec = aligned16(in) && aligned16(out);
  k<<<(int)(ctas < g ? ctas : g), block, smem, st>>>(static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out),
                                                     n, param, vec);
  return launch_status();
}

template <int FN, bool F32>
static cox_status dispatch_w(int width, const void* in, void* out, int64_t n, int param, int block,
                             cudaStream_t st) {
  return with_width(width, [&](auto w) { return launch_shfl<FN, decltype(w)::value, F32>(in, out, n, param, block, st); });
}

}  // namespace cox

using namespace cox;

extern "C" cox_status cox_shfl(cox_warpfn fn, cox_dtype dt, int width, int block_dim, const void* d_in, void* d_out,
                               int64_t n, int param, uint32_t mask, void* stream) {
  if (!valid_width(width) || !valid_block(block_dim) || n < 0) return COX_EINVAL;
  if (dt != COX_I32 && dt != COX_U32 && dt != COX_F32) return COX_EINVAL;
  if (fn < COX_SHFL_IDX || fn > COX_MATCH_ANY) return COX_EINVAL;
  if ((fn == COX_SHFL_UP || fn == COX_SHFL_DOWN || fn == COX_SHFL_XOR) && (param < 0 || param > 31))
    return COX_EINVAL;
  if (mask != 0xFFFFFFFFu) return COX_EUNSUPPORTED;
  if (n > 0 && (!d_in || !d_out)) return COX_EINVAL;
  if (n == 0) return COX_OK;
  cudaStream_t st = as_stream(stream);
  const bool f32 = dt == COX_F32;
  switch (fn) {
    case COX_SHFL_IDX: return dispatch_w<COX_SHFL_IDX, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_SHFL_UP: return dispatch_w<COX_SHFL_UP, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_SHFL_DOWN: return dispatch_w<COX_SHFL_DOWN, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_SHFL_XOR: return dispatch_w<COX_SHFL_XOR, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_MATCH_ANY: return dispatch_w<COX_MATCH_ANY, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_BALLOT:
      return f32 ? dispatch_w<COX_BALLOT, true>(width, d_in, d_out, n, param, block_dim, st)
                 : dispatch_w<COX_BALLOT, false>(width, d_in, d_out, n, param, block_dim, st);
    case COX_ANY:
      return f32 ? dispatch_w<COX_ANY, true>(width, d_in, d_out, n, param, block_dim, st)
                 : dispatch_w<COX_ANY, false>(width, d_in, d_out, n, param, block_dim, st);
    default:
      return f32 ? dispatch_w<COX_ALL, true>(width, d_in, d_out, n, param, block_dim, st)
                 : dispatch_w<COX_ALL, false>(width, d_in, d_out, n, param, block_dim, st);
  }
}
