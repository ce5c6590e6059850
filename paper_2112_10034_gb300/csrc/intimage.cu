// cox_integral_image: integral images of a batch of images -- the SDK's
// shfl_intimage_rows (row scans by warp shuffles) and shfl_vertical_shfl
// (column sums), Table 1 of the paper.  All sums are mod 2^32.
//
// Pass 1 (k_strip_prefix): one warp per image row reads it coalesced, 32
// pixels per step; redux.sync gives each 32-pixel strip's sum, and a running
// sum gives, per row, the prefix of every strip: P[row][s] = sum of the row's
// pixels left of strip s.
// Pass 2 (k_strip_walk): one warp per 32-column strip of one image walks the
// rows top to bottom, 8 rows' loads in flight: an inclusive shuffle scan of
// the row's 32 pixels plus P[row][s] is the row prefix at each column, and a
// running column sum of those is the integral image.  Pixels are read twice
// (1 B each for 8-bit images), the integral written once.
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

template <int DT>
__global__ void __launch_bounds__(256) k_strip_walk(const void* __restrict__ img, int64_t batch, int64_t height,
                                                    int64_t width, const uint32_t* __restrict__ P,
                                                    uint32_t* __restrict__ out) {
  const int lane = lane_id();
  const int64_t ns = (width + 31) / 32;
  const int64_t strips = batch * ns;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < strips; t += wstep) {
    const int64_t b = t / ns, s = t % ns;
    const int64_t x = s * 32 + lane;
    const bool in_img = x < width;
    uint32_t col = 0;
    for (int64_t y0 = 0; y0 < height; y0 += kWalkBatch) {
      uint32_t p[kWalkBatch], off[kWalkBatch];
#pragma unroll
      for (int r = 0; r < kWalkBatch; ++r) {
        const int64_t y = y0 + r;
        const int64_t row = b * height + y;
        p[r] = (y < height && in_img) ? pixel<DT>(img, row * width + x) : 0u;
        off[r] = y < height ? __ldg(P + row * ns + s) : 0u;
      }
#pragma unroll
      for (int r = 0; r < kWalkBatch; ++r) {
        uint32_t v = p[r];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {  // inclusive scan of the row's 32 pixels
          const uint32_t u = __shfl_up_sync(kFull, v, d);
          if (lane >= d) v += u;
        }
        col += v + off[r];
        const int64_t y = y0 + r;
        if (y < height && in_img) __stcs(out + (b * height + y) * width + x, col);
      }
    }
  }
}

template <int DT>
static cox_status launch_intimage(const void* d_in, int64_t batch, int64_t height, int64_t width, uint32_t* d_out,
                                  uint32_t* P, cudaStream_t st) {
  auto k1 = k_strip_prefix<DT>;
  auto k2 = k_strip_walk<DT>;
  static int g1 = 0, g2 = 0;
  if (g1 == 0) g1 = persistent_grid(k1, 256, 0, 1 << 30);
  if (g2 == 0) g2 = persistent_grid(k2, 256, 0, 1 << 30);
  const int64_t rows = batch * height;
  const int64_t c1 = (rows + 7) / 8;
  k1<<<(int)(c1 < g1 ? c1 : g1), 256, 0, st>>>(d_in, rows, width, P);
  const int64_t strips = batch * ((width + 31) / 32);
  const int64_t c2 = (strips + 7) / 8;
  k2<<<(int)(c2 < g2 ? c2 : g2), 256, 0, st>>>(d_in, batch, height, width, P, d_out);
  return launch_status();
}

}  // namespace cox

using namespace cox;

extern "C" size_t cox_integral_image_workspace(int64_t batch, int64_t height, int64_t width) {
  if (batch < 0 || height < 0 || width < 0) return 0;
  return (size_t)batch * height * ((width + 31) / 32) * sizeof(uint32_t) + 16;
}

extern "C" cox_status cox_integral_image(cox_dtype in_dt, int64_t batch, int64_t height, int64_t width,
                                         const void* d_in, uint32_t* d_out, void* d_workspace, size_t workspace_bytes,
                                         void* stream) {
  if (batch < 0 || height < 0 || width < 0) return COX_EINVAL;
  if (in_dt != COX_U8 && in_dt != COX_U32 && in_dt != COX_I32) return COX_EINVAL;
  if (batch == 0 || height == 0 || width == 0) return COX_OK;
  if (!d_in || !d_out) return COX_EINVAL;
  if (!d_workspace || workspace_bytes < cox_integral_image_workspace(batch, height, width)) return COX_ENOMEM;
  uint32_t* P = static_cast<uint32_t*>(d_workspace);
  cudaStream_t st = as_stream(stream);
  if (in_dt == COX_U8) return launch_intimage<COX_U8>(d_in, batch, height, width, d_out, P, st);
  return launch_intimage<COX_U32>(d_in, batch, height, width, d_out, P, st);
}
