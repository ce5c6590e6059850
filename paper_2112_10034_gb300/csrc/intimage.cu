// cox_integral_image: integral images of a batch of images -- the SDK's
// shfl_intimage_rows (row scans by warp shuffles) and shfl_vertical_shfl
// (column sums), Table 1 of the paper.  All sums are mod 2^32.
//
// Pass 1 (k_strip_prefix): one warp per image row reads it coalesced, 32
// pixels per step; redux.sync gives each 32-pixel strip's sum, and a running
// sum gives, per row, the prefix of every strip: P[row][s] = sum of the row's
// pixels left of strip s.
// Pass 1 (k_strip_prefix_vec; 16-byte loads when rows allow): per image
// row, the prefix of every 32-pixel strip.  Passes 2a and 2b cut the rows
// into bands of 64 and give every (image, band, strip) its own warp: 2a
// sums the band per column, 2b adds up the bands above and walks the band's
// rows -- a shuffle scan of each row's 32 pixels plus the strip prefix is
// the row prefix, and the running column sum of row prefixes is the
// integral image.  Pixels are read three times (1 B
// each for 8-bit images), the integral written once.
#include <type_traits>

#include "cox_common.cuh"

namespace cox {

constexpr int kWalkBatch = 8;

template <int DT>
__device__ __forceinline__ uint32_t pixel(const void* img, int64_t i) {
  if constexpr (DT == COX_U8) return static_cast<const uint8_t*>(img)[i];
  else return static_cast<const uint32_t*>(img)[i];
}

template <int DT>
__global__ void __launch_bounds__(256) k_strip_prefix(const void* __restrict__ img, int64_t rows, int64_t width,
                                                      uint32_t* __restrict__ P) {
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += wstep) {
    const int64_t rb = row * width;
    uint32_t run = 0;
    for (int64_t s0 = 0; s0 < ns; s0 += 32) {  // 32 strips per round: lane l writes strip s0 + l
      uint32_t mine = 0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const int64_t s = s0 + j;
        if (s >= ns) break;  // warp-uniform
        const int64_t x = s * 32 + lane;
        const uint32_t p = x < width ? pixel<DT>(img, rb + x) : 0u;
        const uint32_t sum = __reduce_add_sync(kFull, p);
        if (lane == j) mine = run;
        run += sum;
      }
      if (s0 + lane < ns) P[row * ns + s0 + lane] = mine;
    }
  }
}

// Pass 1, 16-byte form (8-bit rows whose width is a multiple of 16, 32-bit
// rows whose width is a multiple of 4): lane l loads 16 bytes, so a warp
// covers 512 (8-bit) or 128 (32-bit) pixels = 16 or 4 strips per load; the
// lanes of a strip combine their sums, and the strips' exclusive prefixes
// continue the row's running sum.
template <int DT>
__global__ void __launch_bounds__(256) k_strip_prefix_vec(const void* __restrict__ img, int64_t rows, int64_t width,
                                                          uint32_t* __restrict__ P) {
  constexpr int PX = DT == COX_U8 ? 16 : 4;  // pixels per lane per load
  constexpr int LPS = 32 / PX;                // lanes per strip
  constexpr int SPL = 32 / LPS;               // strips per warp load
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += wstep) {
    const uint8_t* rb = static_cast<const uint8_t*>(img) + row * width * (DT == COX_U8 ? 1 : 4);
    uint32_t run = 0;
    for (int64_t x0 = 0; x0 < width; x0 += 32 * PX) {
      const int64_t x = x0 + (int64_t)lane * PX;
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (x < width) q = __ldcs(reinterpret_cast<const uint4*>(rb + x * (DT == COX_U8 ? 1 : 4)));
      uint32_t sum;
      if constexpr (DT == COX_U8) {
        sum = __dp4a(q.x, 0x01010101u, 0u);
        sum = __dp4a(q.y, 0x01010101u, sum);
        sum = __dp4a(q.z, 0x01010101u, sum);
        sum = __dp4a(q.w, 0x01010101u, sum);
      } else {
        sum = q.x + q.y + q.z + q.w;
      }
#pragma unroll
      for (int m = 1; m < LPS; m <<= 1) sum += __shfl_xor_sync(kFull, sum, m);  // strip sum in its lanes
      // inclusive scan over the SPL strips (lane l's strip = l / LPS)
      uint32_t inc = sum;
#pragma unroll
      for (int d = LPS; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += u;
      }
      const int64_t s = x0 / 32 + lane / LPS;
      if (lane % LPS == 0 && s < ns) P[row * ns + s] = run + inc - sum;
      run += __shfl_sync(kFull, inc, 31);
    }
  }
}

// Rows are cut into bands of kBand rows.  Pass 2a: one warp per (image,
// band, strip) sums the band's pixels per column and the band's strip
// prefixes; the band's contribution to the integral of its last row at
// column x is then scan32(column sums)(x) + sum of P.  Pass 2b: one warp
// per (image, band, strip) adds up the contributions of the bands above it
// and walks the band's rows from there: the row prefix at x is the shuffle
// scan of the row's 32 pixels plus P[row][s], and the running column sum of
// row prefixes is the integral image.
constexpr int kBand = 64;

template <int DT>
using pix_t = typename std::conditional<DT == COX_U8, uint8_t, uint32_t>::type;

template <int DT>
__global__ void __launch_bounds__(256) k_band_sums(const void* __restrict__ img, int64_t batch, int64_t height,
                                                   int64_t width, const uint32_t* __restrict__ P,
                                                   uint32_t* __restrict__ CS) {
  using PT = pix_t<DT>;
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand;
  const int64_t units = batch * nb * ns;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += wstep) {
    const int64_t s = u % ns, k = (u / ns) % nb, b = u / (ns * nb);
    const int64_t x = s * 32 + lane;
    const bool in_img = x < width;
    const int64_t y0 = k * kBand;
    const int nrows = (int)min((int64_t)kBand, height - y0);
    const int64_t row0 = b * height + y0;
    const PT* pin = static_cast<const PT*>(img) + row0 * width + (in_img ? x : 0);
    const uint32_t* pp = P + row0 * ns + s;
    uint32_t cs = 0, ps = 0;
#pragma unroll 8
    for (int y = 0; y < nrows; ++y) {
      cs += in_img ? (uint32_t)pin[(int64_t)y * width] : 0u;
      ps += __ldg(pp + (int64_t)y * ns);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(kFull, cs, d);
      if (lane >= d) cs += v;
    }
    if (in_img) CS[(b * nb + k) * width + x] = cs + ps;
  }
}

template <int DT>
__global__ void __launch_bounds__(256, 4) k_band_walk(const void* __restrict__ img, int64_t batch, int64_t height,
                                                      int64_t width, const uint32_t* __restrict__ P,
                                                      const uint32_t* __restrict__ CS, uint32_t* __restrict__ out) {
  using PT = pix_t<DT>;
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand;
  const int64_t units = batch * nb * ns;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += wstep) {
    const int64_t s = u % ns, k = (u / ns) % nb, b = u / (ns * nb);
    const int64_t x = s * 32 + lane;
    const bool in_img = x < width;
    const int64_t y0 = k * kBand;
    const int nrows = (int)min((int64_t)kBand, height - y0);
    uint32_t col = 0;  // the bands above: their column sums (independent loads)
    if (in_img)
      for (int64_t kk = 0; kk < k; ++kk) col += __ldg(CS + (b * nb + kk) * width + x);
    const int64_t row0 = b * height + y0;
    const PT* pin = static_cast<const PT*>(img) + row0 * width + (in_img ? x : 0);
    const uint32_t* pp = P + row0 * ns + s;
    uint32_t* po = out + row0 * width + (in_img ? x : 0);
    for (int ya = 0; ya < nrows; ya += kWalkBatch) {
      uint32_t pv[kWalkBatch], off[kWalkBatch];
#pragma unroll
      for (int r = 0; r < kWalkBatch; ++r) {
        const bool ok = ya + r < nrows;
        pv[r] = (ok && in_img) ? (uint32_t)pin[(int64_t)(ya + r) * width] : 0u;
        off[r] = ok ? __ldg(pp + (int64_t)(ya + r) * ns) : 0u;
      }
#pragma unroll
      for (int r = 0; r < kWalkBatch; ++r) {
        uint32_t v = pv[r];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {  // inclusive scan of the row's 32 pixels
          const uint32_t w = __shfl_up_sync(kFull, v, d);
          if (lane >= d) v += w;
        }
        col += v + off[r];
        if (ya + r < nrows && in_img) __stcs(po + (int64_t)(ya + r) * width, col);
      }
    }
  }
}

// 16-byte forms of passes 2a and 2b (same condition as pass 1's): lane l
// of a warp owns PX = 16 (8-bit) or 4 (32-bit) consecutive pixels of each
// row, so a warp covers a strip of SW = 32 * PX columns and every row
// access is one coalesced 512-byte (8-bit) or 512-byte (32-bit) segment.
// Within a row: a serial scan of the lane's PX pixels, a warp scan of the
// lane totals, and the row prefix at the strip start (P at 32-pixel
// granularity, SW being a multiple of 32).
template <int DT>
__device__ __forceinline__ void unpack_px(const uint4 q, uint32_t (&v)[DT == COX_U8 ? 16 : 4]) {
  if constexpr (DT == COX_U8) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[4 * i + j] = (w[i] >> (8 * j)) & 0xFFu;
  } else {
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
}

template <int DT>
__global__ void __launch_bounds__(256) k_band_sums_vec(const void* __restrict__ img, int64_t batch, int64_t height,
                                                       int64_t width, const uint32_t* __restrict__ P,
                                                       uint32_t* __restrict__ CS) {
  constexpr int PX = DT == COX_U8 ? 16 : 4, SW = 32 * PX, EB = DT == COX_U8 ? 1 : 4;
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand, nsw = (width + SW - 1) / SW;
  const int64_t units = batch * nb * nsw;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += wstep) {
    const int64_t s = u % nsw, k = (u / nsw) % nb, b = u / (nsw * nb);
    const int64_t x = s * SW + (int64_t)lane * PX;
    const bool in_img = x < width;
    const int64_t y0 = k * kBand;
    const int nrows = (int)min((int64_t)kBand, height - y0);
    const int64_t row0 = b * height + y0;
    const uint8_t* pin = static_cast<const uint8_t*>(img) + (row0 * width + (in_img ? x : 0)) * EB;
    const uint32_t* pp = P + row0 * ns + s * (SW / 32);
    uint32_t cs[PX];
#pragma unroll
    for (int j = 0; j < PX; ++j) cs[j] = 0;
    uint32_t ps = 0;
#pragma unroll 4
    for (int y = 0; y < nrows; ++y) {
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (in_img) q = __ldcs(reinterpret_cast<const uint4*>(pin + (int64_t)y * width * EB));
      uint32_t v[PX];
      unpack_px<DT>(q, v);
#pragma unroll
      for (int j = 0; j < PX; ++j) cs[j] += v[j];
      ps += __ldg(pp + (int64_t)y * ns);
    }
#pragma unroll
    for (int j = 1; j < PX; ++j) cs[j] += cs[j - 1];  // scan within the lane
    uint32_t inc = cs[PX - 1];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t w = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += w;
    }
    const uint32_t ex = inc - cs[PX - 1] + ps;
    if (in_img) {
      uint32_t* dst = CS + (b * nb + k) * width + x;
#pragma unroll
      for (int j = 0; j < PX; j += 4)
        *reinterpret_cast<uint4*>(dst + j) = make_uint4(cs[j] + ex, cs[j + 1] + ex, cs[j + 2] + ex, cs[j + 3] + ex);
    }
  }
}

template <int DT>
__global__ void __launch_bounds__(256) k_band_walk_vec(const void* __restrict__ img, int64_t batch, int64_t height,
                                                       int64_t width, const uint32_t* __restrict__ P,
                                                       const uint32_t* __restrict__ CS, uint32_t* __restrict__ out) {
  constexpr int PX = DT == COX_U8 ? 16 : 4, SW = 32 * PX, EB = DT == COX_U8 ? 1 : 4;
  constexpr int RB = 4;  // rows' loads in flight
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand, nsw = (width + SW - 1) / SW;
  const int64_t units = batch * nb * nsw;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += wstep) {
    const int64_t s = u % nsw, k = (u / nsw) % nb, b = u / (nsw * nb);
    const int64_t x = s * SW + (int64_t)lane * PX;
    const bool in_img = x < width;
    const int64_t y0 = k * kBand;
    const int nrows = (int)min((int64_t)kBand, height - y0);
    uint32_t col[PX];
#pragma unroll
    for (int j = 0; j < PX; ++j) col[j] = 0;
    if (in_img)  // the bands above
      for (int64_t kk = 0; kk < k; ++kk) {
        const uint32_t* src = CS + (b * nb + kk) * width + x;
#pragma unroll
        for (int j = 0; j < PX; j += 4) {
          const uint4 c = __ldg(reinterpret_cast<const uint4*>(src + j));
          col[j] += c.x; col[j + 1] += c.y; col[j + 2] += c.z; col[j + 3] += c.w;
        }
      }
    const int64_t row0 = b * height + y0;
    const uint8_t* pin = static_cast<const uint8_t*>(img) + (row0 * width + (in_img ? x : 0)) * EB;
    const uint32_t* pp = P + row0 * ns + s * (SW / 32);
    uint32_t* po = out + row0 * width + (in_img ? x : 0);
    for (int ya = 0; ya < nrows; ya += RB) {
      uint4 q[RB];
      uint32_t off[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        const bool ok = ya + r < nrows;
        q[r] = make_uint4(0u, 0u, 0u, 0u);
        if (ok && in_img) q[r] = __ldcs(reinterpret_cast<const uint4*>(pin + (int64_t)(ya + r) * width * EB));
        off[r] = ok ? __ldg(pp + (int64_t)(ya + r) * ns) : 0u;
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        uint32_t v[PX];
        unpack_px<DT>(q[r], v);
#pragma unroll
        for (int j = 1; j < PX; ++j) v[j] += v[j - 1];
        uint32_t inc = v[PX - 1];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t w = __shfl_up_sync(kFull, inc, d);
          if (lane >= d) inc += w;
        }
        const uint32_t ex = inc - v[PX - 1] + off[r];
#pragma unroll
        for (int j = 0; j < PX; ++j) col[j] += v[j] + ex;
        if (ya + r < nrows && in_img) {
          uint32_t* dst = po + (int64_t)(ya + r) * width;
#pragma unroll
          for (int j = 0; j < PX; j += 4)
            __stcs(reinterpret_cast<uint4*>(dst + j), make_uint4(col[j], col[j + 1], col[j + 2], col[j + 3]));
        }
      }
    }
  }
}

template <int DT>
static cox_status launch_intimage(const void* d_in, int64_t batch, int64_t height, int64_t width, uint32_t* d_out,
                                  uint32_t* P, uint32_t* CS, cudaStream_t st) {
  const int64_t rows = batch * height;
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand;
  const bool vec = aligned16(d_in) && width % (DT == COX_U8 ? 16 : 4) == 0;
  auto grid_of = [](auto k, int64_t warps) {
    const int g = persistent_grid(k, 256, 0, 1 << 30);
    const int64_t ctas = (warps + 7) / 8;
    return (int)(ctas < g ? (ctas < 1 ? 1 : ctas) : g);
  };
  if (vec && aligned16(d_out)) {
    constexpr int SW = 32 * (DT == COX_U8 ? 16 : 4);
    const int64_t vunits = batch * nb * ((width + SW - 1) / SW);
    auto k1 = k_strip_prefix_vec<DT>;
    k1<<<grid_of(k1, rows), 256, 0, st>>>(d_in, rows, width, P);
    auto k2 = k_band_sums_vec<DT>;
    k2<<<grid_of(k2, vunits), 256, 0, st>>>(d_in, batch, height, width, P, CS);
    auto k3 = k_band_walk_vec<DT>;
    k3<<<grid_of(k3, vunits), 256, 0, st>>>(d_in, batch, height, width, P, CS, d_out);
    return launch_status();
  }
  if (vec) {
    auto k1 = k_strip_prefix_vec<DT>;
    k1<<<grid_of(k1, rows), 256, 0, st>>>(d_in, rows, width, P);
  } else {
    auto k1 = k_strip_prefix<DT>;
    k1<<<grid_of(k1, rows), 256, 0, st>>>(d_in, rows, width, P);
  }
  const int64_t units = batch * nb * ns;
  auto k2 = k_band_sums<DT>;
  k2<<<grid_of(k2, units), 256, 0, st>>>(d_in, batch, height, width, P, CS);
  auto k3 = k_band_walk<DT>;
  k3<<<grid_of(k3, units), 256, 0, st>>>(d_in, batch, height, width, P, CS, d_out);
  return launch_status();
}

}  // namespace cox

using namespace cox;

// Workspace: P (one word per image row and 32-pixel strip), then CS (one
// word per image, band and column), each rounded to 16 bytes.
static size_t ws_p_bytes(int64_t batch, int64_t height, int64_t width) {
  return ((size_t)batch * height * ((width + 31) / 32) * sizeof(uint32_t) + 15) & ~(size_t)15;
}
static size_t ws_cs_bytes(int64_t batch, int64_t height, int64_t width) {
  return ((size_t)batch * ((height + kBand - 1) / kBand) * width * sizeof(uint32_t) + 15) & ~(size_t)15;
}

extern "C" size_t cox_integral_image_workspace(int64_t batch, int64_t height, int64_t width) {
  if (batch < 0 || height < 0 || width < 0) return 0;
  return ws_p_bytes(batch, height, width) + ws_cs_bytes(batch, height, width) + 16;
}

extern "C" cox_status cox_integral_image(cox_dtype in_dt, int64_t batch, int64_t height, int64_t width,
                                         const void* d_in, uint32_t* d_out, void* d_workspace, size_t workspace_bytes,
                                         void* stream) {
  if (batch < 0 || height < 0 || width < 0) return COX_EINVAL;
  if (in_dt != COX_U8 && in_dt != COX_U32 && in_dt != COX_I32) return COX_EINVAL;
  if (batch == 0 || height == 0 || width == 0) return COX_OK;
  if (!d_in || !d_out) return COX_EINVAL;
  if (!d_workspace || workspace_bytes < cox_integral_image_workspace(batch, height, width)) return COX_ENOMEM;
  if (!aligned16(d_workspace)) return COX_EINVAL;
  uint32_t* P = static_cast<uint32_t*>(d_workspace);
  uint32_t* CS = reinterpret_cast<uint32_t*>(static_cast<char*>(d_workspace) + ws_p_bytes(batch, height, width));
  cudaStream_t st = as_stream(stream);
  if (in_dt == COX_U8) return launch_intimage<COX_U8>(d_in, batch, height, width, d_out, P, CS, st);
  return launch_intimage<COX_U32>(d_in, batch, height, width, d_out, P, CS, st);
}
