// cox_integral_image: integral images of a batch of images -- the SDK's
// shfl_intimage_rows (row scans by warp shuffles) and shfl_vertical_shfl
// (column sums), Table 1 of the paper.  All sums are mod 2^32.
//
// General form (any width, any alignment), three passes.  Pass 1
// (k_strip_prefix; k_strip_prefix_vec with 16-byte loads when rows allow):
// per image row, the prefix of every 32-pixel strip, P[row][s] = sum of the
// row's pixels left of strip s.  Passes 2a and 2b cut the rows into bands of
// 64 and give every (image, band, strip) its own warp: 2a sums the band per
// column, 2b adds up the bands above and walks the band's rows -- a shuffle
// scan of each row's 32 pixels plus the strip prefix is the row prefix, and
// the running column sum of row prefixes is the integral image.
//
// 16-byte forms (16-byte aligned input and output, rows a whole number of
// 16-byte units): with enough 128-column strips to fill the GPU, the strip
// walk (one launch, pixels read once, below); otherwise two passes that read
// the pixels twice -- block sums per (image, band, 512- or 128-column
// strip), then the band walkers.
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
      // inclusive scan over this load's strips (lane l's strip = l / LPS)
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

// 16-byte forms (same condition as pass 1's 16-byte form, plus a 16-byte
// aligned output): lane l of a warp owns PX = 16 (8-bit) or 4 (32-bit)
// consecutive pixels of each row, so a warp covers a strip of SW = 32 * PX
// columns with one coalesced 512-byte load per row.  Two kernels:
//
// k_block_sums_vec, one warp per (image, band, strip), reads the block's
// pixels once and writes the strip total of every row, T[row][s], the
// block's in-strip column prefixes at the band's last row, C[b][k][x], and
// the block total, BT[b][k][s].  For 8-bit pixels, two columns share a
// 32-bit accumulator (16-bit halves; a band of 64 rows sums to at most
// 64 * 255).
//
// k_band_walk_vec, one warp per (image, band, strip), starts from the
// integral at the row above the band -- the C of the bands above plus the
// block totals above and to the left -- and walks the band's rows: the row
// prefix at the strip start is the sum of the row's T to the left, the
// lane's pixels are scanned serially, the lane totals by a warp scan, and
// the running column sums of row prefixes are the integral.  8-bit rows
// leave through a per-warp shared-memory transpose (16-byte units swizzled
// by u ^ ((u >> 3) & 3), conflict-free both ways), so each 16-byte store
// instruction writes 512 contiguous bytes.
template <int DT>
__device__ __forceinline__ void unpack_px(const uint4 q, uint32_t (&v)[DT == COX_U8 ? 16 : 4]) {
  if constexpr (DT == COX_U8) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[4 * i + j] = __byte_perm(w[i], 0u, 0x4440u + j);
  } else {
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
}

template <int DT>
__device__ __forceinline__ uint32_t lane_total(const uint4 q) {
  if constexpr (DT == COX_U8) {
    uint32_t t = __dp4a(q.x, 0x01010101u, 0u);
    t = __dp4a(q.y, 0x01010101u, t);
    t = __dp4a(q.z, 0x01010101u, t);
    return __dp4a(q.w, 0x01010101u, t);
  } else {
    return q.x + q.y + q.z + q.w;
  }
}


template <int DT>
__global__ void __launch_bounds__(256, 4) k_block_sums_vec(const void* __restrict__ img, int64_t batch,
                                                           int64_t height, int64_t width, uint32_t* __restrict__ T,
                                                           uint32_t* __restrict__ C, uint32_t* __restrict__ BT) {
  constexpr int PX = DT == COX_U8 ? 16 : 4, SW = 32 * PX, EB = DT == COX_U8 ? 1 : 4;
  constexpr int NA = DT == COX_U8 ? 8 : 4;  // accumulators per lane
  constexpr int kSumsBatch = DT == COX_U8 ? 4 : 8;  // row loads in flight (divides 32)
  const int lane = lane_id();
  const int64_t nb = (height + kBand - 1) / kBand, nsw = (width + SW - 1) / SW;
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
    uint32_t acc[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = 0;
    uint32_t tv = 0;  // lane r keeps T of row (32-row group start) + r
    for (int ya = 0; ya < nrows; ya += kSumsBatch) {
      uint4 q[kSumsBatch];
#pragma unroll
      for (int r = 0; r < kSumsBatch; ++r) {
        q[r] = make_uint4(0u, 0u, 0u, 0u);
        if (ya + r < nrows && in_img) q[r] = __ldcs(reinterpret_cast<const uint4*>(pin + (int64_t)(ya + r) * width * EB));
      }
#pragma unroll
      for (int r = 0; r < kSumsBatch; ++r) {
        if constexpr (DT == COX_U8) {
          const uint32_t w[4] = {q[r].x, q[r].y, q[r].z, q[r].w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {  // acc[2i]: columns 4i, 4i+2; acc[2i+1]: 4i+1, 4i+3
            acc[2 * i] += w[i] & 0x00FF00FFu;
            acc[2 * i + 1] += (w[i] >> 8) & 0x00FF00FFu;
          }
        } else {
          acc[0] += q[r].x; acc[1] += q[r].y; acc[2] += q[r].z; acc[3] += q[r].w;
        }
        const uint32_t rt = __reduce_add_sync(kFull, lane_total<DT>(q[r]));
        if (lane == ((ya + r) & 31)) tv = rt;
      }
      const int done = ya + kSumsBatch;  // rows [0, done) summed
      if ((done & 31) == 0 || done >= nrows) {
        const int g0 = (ya + kSumsBatch - 1) & ~31;  // start of this 32-row group
        if (g0 + lane < nrows && g0 + lane < done) T[(row0 + g0 + lane) * nsw + s] = tv;
      }
    }
    uint32_t cs[PX];
    if constexpr (DT == COX_U8) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cs[4 * i] = acc[2 * i] & 0xFFFFu;
        cs[4 * i + 1] = acc[2 * i + 1] & 0xFFFFu;
        cs[4 * i + 2] = acc[2 * i] >> 16;
        cs[4 * i + 3] = acc[2 * i + 1] >> 16;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) cs[j] = acc[j];
    }
#pragma unroll
    for (int j = 1; j < PX; ++j) cs[j] += cs[j - 1];  // scan within the lane
    uint32_t inc = cs[PX - 1];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t w = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += w;
    }
    const uint32_t ex = inc - cs[PX - 1];
    if (in_img) {
      uint32_t* dst = C + (b * nb + k) * width + x;
#pragma unroll
      for (int j = 0; j < PX; j += 4)
        *reinterpret_cast<uint4*>(dst + j) = make_uint4(cs[j] + ex, cs[j + 1] + ex, cs[j + 2] + ex, cs[j + 3] + ex);
    }
    if (lane == 31) BT[(b * nb + k) * nsw + s] = inc;
  }
}

// Shared-memory slot of 16-byte unit u (0..127) of a 2 KB row segment.
__device__ __forceinline__ int px_slot(int u) { return u ^ ((u >> 3) & 3); }

template <int DT>
__global__ void __launch_bounds__(256, 4) k_band_walk_vec(const void* __restrict__ img, int64_t batch,
                                                          int64_t height, int64_t width,
                                                          const uint32_t* __restrict__ T,
                                                          const uint32_t* __restrict__ C,
                                                          const uint32_t* __restrict__ BT,
                                                          uint32_t* __restrict__ out) {
  constexpr int PX = DT == COX_U8 ? 16 : 4, SW = 32 * PX, EB = DT == COX_U8 ? 1 : 4;
  constexpr int NBUF = DT == COX_U8 ? 2 : 1;
  constexpr int kWalkRows = DT == COX_U8 ? 2 : 4;  // row loads in flight
  __shared__ __align__(16) uint4 xbuf[DT == COX_U8 ? 8 : 1][NBUF][128];  // per warp: 2 rows of 2 KB
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  const int64_t nb = (height + kBand - 1) / kBand, nsw = (width + SW - 1) / SW;
  const int64_t units = batch * nb * nsw;
  const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int buf = 0;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += wstep) {
    const int64_t s = u % nsw, k = (u / nsw) % nb, b = u / (nsw * nb);
    const int64_t x = s * SW + (int64_t)lane * PX;
    const bool in_img = x < width;
    const int64_t y0 = k * kBand;
    const int nrows = (int)min((int64_t)kBand, height - y0);
    // The integral at the row above the band: the blocks above and to the
    // left (their totals), plus the column prefixes of the blocks above.
    uint32_t above = 0;
    for (int64_t i = lane; i < k * s; i += 32) above += __ldg(BT + (b * nb + i / s) * nsw + i % s);
    above = __reduce_add_sync(kFull, above);
    uint32_t col[PX];
#pragma unroll
    for (int j = 0; j < PX; ++j) col[j] = above;
    if (in_img) {
      const uint32_t* src = C + b * nb * width + x;
      int64_t kk = 0;
      for (; kk + 2 <= k; kk += 2) {
#pragma unroll
        for (int j = 0; j < PX; j += 4) {
          const uint4 c0 = __ldg(reinterpret_cast<const uint4*>(src + kk * width + j));
          const uint4 c1 = __ldg(reinterpret_cast<const uint4*>(src + (kk + 1) * width + j));
          col[j] += c0.x + c1.x; col[j + 1] += c0.y + c1.y; col[j + 2] += c0.z + c1.z; col[j + 3] += c0.w + c1.w;
        }
      }
      if (kk < k) {
#pragma unroll
        for (int j = 0; j < PX; j += 4) {
          const uint4 c0 = __ldg(reinterpret_cast<const uint4*>(src + kk * width + j));
          col[j] += c0.x; col[j + 1] += c0.y; col[j + 2] += c0.z; col[j + 3] += c0.w;
        }
      }
    }
    const int64_t row0 = b * height + y0;
    const uint8_t* pin = static_cast<const uint8_t*>(img) + (row0 * width + (in_img ? x : 0)) * EB;
    const uint32_t* pt = T + row0 * nsw;
    uint32_t* po = out + row0 * width + s * SW;
    for (int ya = 0; ya < nrows; ya += kWalkRows) {
      uint4 q[kWalkRows];
      uint32_t tl[kWalkRows];  // this lane's share of the row's strips to the left
#pragma unroll
      for (int r = 0; r < kWalkRows; ++r) {
        const bool ok = ya + r < nrows;
        q[r] = make_uint4(0u, 0u, 0u, 0u);
        if (ok && in_img) q[r] = __ldcs(reinterpret_cast<const uint4*>(pin + (int64_t)(ya + r) * width * EB));
        tl[r] = 0;
        if (ok)
          for (int64_t i = lane; i < s; i += 32) tl[r] += __ldg(pt + (int64_t)(ya + r) * nsw + i);
      }
#pragma unroll
      for (int r = 0; r < kWalkRows; ++r) {
        const uint32_t left = __reduce_add_sync(kFull, tl[r]);  // row prefix at the strip start
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
        const uint32_t ex = inc - v[PX - 1] + left;
#pragma unroll
        for (int j = 0; j < PX; ++j) col[j] += v[j] + ex;
        if (ya + r >= nrows) continue;  // warp-uniform
        uint32_t* dst = po + (int64_t)(ya + r) * width;
        if constexpr (DT == COX_U8) {
          uint4* xb = xbuf[wib][buf];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            xb[px_slot(4 * lane + j)] = make_uint4(col[4 * j], col[4 * j + 1], col[4 * j + 2], col[4 * j + 3]);
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int un = 32 * i + lane;  // 16-byte unit = columns 4 un .. 4 un + 3 of the strip
            const uint4 o = xb[px_slot(un)];
            if (s * SW + 4 * un < width) __stcs(reinterpret_cast<uint4*>(dst + 4 * un), o);
          }
          buf ^= 1;  // the other buffer's readers passed the __syncwarp above
        } else {
          if (in_img) __stcs(reinterpret_cast<uint4*>(dst + lane * 4), make_uint4(col[0], col[1], col[2], col[3]));
        }
      }
    }
  }
}

// Single-read form (strip walk).  A team of three warps per (image, strip
// of 128 columns) walks the strip's rows from the top of the image to the
// bottom, lane l owning columns 4l .. 4l+3.  Write T(y, l) for lane l's
// pixel total in row y, S(y, l) = sum of T(y', l) over rows y' <= y, and
// c_j(y, l) for the same running sum of the lane's in-lane prefixes
// (pixels 0..j).  At x = x0 + 4l + j, with x0 the strip's first column,
//   I(y, x) = I(y, x0 - 1) + sum_{l' < l} S(y, l') + c_j(y, l).
// c_j is lane-local (one dp4a per column and row for 8-bit pixels).  The
// other two terms depend on the row and lane only and are computed ahead of
// the walk, one stage of RB rows at a time:
//  - the totals warp stores every lane's S column into a shared-memory
//    transpose, scans each row of it across the lanes (exclusive sums back
//    in place), and publishes the row's total A(y) = sum over all lanes of
//    S(y, l) -- the strip's own integral at its last column -- as a tagged
//    word (value | tag << 32; the words are zeroed before the launch);
//  - the left-sum warp adds I(y, x0 - 1), the integral just left of the
//    strip, to each row of the transpose: it is the sum of the left
//    strips' A(y), whose words it loads two stages ahead, re-reading any
//    not yet written.  The transpose then holds
//    E(y, l) = I(y, x0 - 1) + sum_{l' < l} S(y, l');
//  - the walk warp adds E to c_j and stores.
// A depends only on the strip's own pixels, so no chain forms between
// strips.
//
// Rows arrive through a per-team ring of NS stages (TMA boxes of 128
// columns x RB rows of one image; columns and rows past the image read as
// 0), so every pixel is read from memory once; the transpose of a stage
// lives beside its ring slot.  Per slot, `full` completes when the box has
// landed, `tot` when the totals warp is done with it and `ready` when E is
// complete; the walk warp refills the slot when it has walked it.  Every
// team takes its units (one per round, StripSched) in increasing order of
// g = b * nsw + s, and all teams are resident (cooperative launch); a unit
// waits only on units with a smaller g, so the smallest unfinished unit can
// always proceed.
template <int DT>
struct StripCfg {
  static constexpr int EB = DT == COX_U8 ? 1 : 4;
  // rows per stage (multiple of 4, divides 32): 8-bit stages are cheap, so
  // they take 16 rows to halve the per-stage hand-offs between the warps
  static constexpr int RB = DT == COX_U8 ? 16 : 8;
  static constexpr int NS = DT == COX_U8 ? 6 : 5;     // ring stages per team (shared memory allows no more)
  static constexpr int NP = 7;                        // warp teams per CTA
  static constexpr int HL = 32 / RB;                  // lanes per row in the scans across lanes
  static constexpr int SBP = RB + 4;                  // transpose row pitch (words)
  // Lane l's column of a transpose starts at word l * SBP + (l / RB) * RB:
  // the skew puts the HL lanes that scan one row (lanes RB apart, each
  // taking RB columns) in different banks; 16-byte accesses stay aligned.
  static constexpr int kSbWords = 32 * SBP + 32;
  static constexpr uint32_t kStage = (uint32_t)RB * 128 * EB;
  static constexpr uint32_t kSb = kSbWords * 4;       // one transpose (bytes)
  static constexpr uint32_t kTeamBytes = NS * (kStage + kSb);
  static constexpr size_t kSmem = (size_t)NP * kTeamBytes + (size_t)NP * 3 * NS * sizeof(uint64_t) + 128;
};
constexpr int kStripCols = 128;
// The strip walk runs when there are enough strips to fill the GPU (at
// least this many per SM) and few enough that summing the left
// neighbours' A stays cheap; otherwise the band kernels below run.
constexpr int kStripUnitsPerSm = 4;
constexpr int64_t kStripMaxStrips = 64;

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
// Barrier for the three warps of a team (named barrier 1 + team, 96 threads).
__device__ __forceinline__ void team_sync(int team) {
  asm volatile("bar.sync %0, 96;" ::"r"(team + 1) : "memory");
}

// Lane total of stage row r, added to s.
template <int DT>
__device__ __forceinline__ uint32_t strip_add_total(const uint8_t* stage, int r, int lane, uint32_t s) {
  if constexpr (DT == COX_U8) {
    return __dp4a(reinterpret_cast<const uint32_t*>(stage)[r * 32 + lane], 0x01010101u, s);
  } else {
    const uint4 q = reinterpret_cast<const uint4*>(stage)[r * 32 + lane];
    return s + q.x + q.y + q.z + q.w;
  }
}
// Adds the in-lane prefixes of stage row r (pixels 0..j) to c[j].
template <int DT>
__device__ __forceinline__ void strip_add_prefixes(const uint8_t* stage, int r, int lane, uint32_t (&c)[4]) {
  if constexpr (DT == COX_U8) {
    const uint32_t w = reinterpret_cast<const uint32_t*>(stage)[r * 32 + lane];
    c[0] = __dp4a(w, 0x00000001u, c[0]);
    c[1] = __dp4a(w, 0x00000101u, c[1]);
    c[2] = __dp4a(w, 0x00010101u, c[2]);
    c[3] = __dp4a(w, 0x01010101u, c[3]);
  } else {
    const uint4 q = reinterpret_cast<const uint4*>(stage)[r * 32 + lane];
    const uint32_t p1 = q.x + q.y, p2 = p1 + q.z;
    c[0] += q.x;
    c[1] += p1;
    c[2] += p2;
    c[3] = c[3] + p2 + q.w;
  }
}

// Tagged A word: value in the low half, kATag in the high half once written
// (the words are zeroed before the launch).
constexpr uint32_t kATag = 1u;
constexpr int kClGroup = 8;  // left-strip words a lane loads per round trip

__device__ __forceinline__ uint64_t ld_relaxed_u64g(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Adds the tagged words p[j * stride] for j in [j0, j1) (j1 - j0 <= kClGroup)
// to *acc, re-reading (bounded) any word not yet written.  `w` holds the
// words already loaded for this range.  False on timeout.
__device__ __forceinline__ bool add_tagged(const unsigned long long* p, int64_t stride, int64_t j0, int64_t j1,
                                           const uint64_t (&w)[kClGroup], uint32_t limit, uint32_t* acc) {
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kClGroup; ++k) {
    if (j0 + k >= j1) break;
    uint64_t v = w[k];
    for (uint32_t n = 0; (uint32_t)(v >> 32) != kATag;) {
      if (++n > limit) return false;
      __nanosleep(32);
      v = ld_relaxed_u64g(p + (j0 + k) * stride);
    }
    sum += (uint32_t)v;
  }
  *acc += sum;
  return true;
}
__device__ __forceinline__ void load_tagged(const unsigned long long* p, int64_t stride, int64_t j0, int64_t j1,
                                            uint64_t (&w)[kClGroup]) {
#pragma unroll
  for (int k = 0; k < kClGroup; ++k) w[k] = j0 + k < j1 ? ld_relaxed_u64g(p + (j0 + k) * stride) : 0ull;
}

// Which unit a team takes in each round.  Round r covers units
// [r * R, r * R + n) with R = CTAs x teams; CTA c gets a contiguous block of
// them (n / CTAs, one more for the first n % CTAs CTAs) and team p the p-th
// unit of its block.  The strips of an image thus sit on two or three
// neighbouring SMs that carry the same number of units, so no image is
// paced by a busier SM than its neighbours'.
struct StripSched {
  int64_t units, R;
  int G, c, p;
  __device__ int64_t unit(int64_t r) const {  // -1: none
    const int64_t s0 = r * R, n = min(R, units - s0);
    if (n <= 0) return -1;
    const int64_t base = n / G, extra = n % G;
    const int64_t nc = base + (c < extra ? 1 : 0), start = c * base + min((int64_t)c, extra);
    return p < nc ? s0 + start + p : -1;
  }
  __device__ int64_t rounds() const {  // rounds in which the team has a unit
    const int64_t full = units / R;
    return full + (unit(full) >= 0 ? 1 : 0);
  }
};

// A team's position in its (unit, stage) job sequence.
struct StripJob {
  int64_t q = 0;    // job index
  int64_t r = 0;    // round
  int64_t g, b, s;  // unit, its image and strip
  int i = 0;        // stage
  __device__ StripJob(const StripSched& sc, int64_t nsw) : g(sc.unit(0)), b(g / nsw), s(g - (g / nsw) * nsw) {}
  __device__ void next(int nst, const StripSched& sc, int64_t nsw) {
    ++q;
    if (++i == nst) {
      i = 0;
      g = sc.unit(++r);
      b = g / nsw;
      s = g - b * nsw;
    }
  }
};

template <int DT>
__global__ void __launch_bounds__(96 * StripCfg<DT>::NP, 1)
    k_strip_walk(const __grid_constant__ CUtensorMap tin, int64_t batch, int64_t height, int64_t width,
                 uint32_t* __restrict__ out, unsigned long long* A, uint32_t limit, unsigned* status) {
  using C = StripCfg<DT>;
  constexpr int RB = C::RB, NS = C::NS, NP = C::NP, SBP = C::SBP, HL = C::HL;
  extern __shared__ uint8_t strip_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(strip_smem_raw) + 127) & ~uintptr_t(127));
  const int lane = lane_id(), warp = threadIdx.x >> 5, team = warp / 3, role = warp - 3 * team;
  uint8_t* ring = base + (size_t)team * C::kTeamBytes;                  // NS stages
  uint32_t* sbuf = reinterpret_cast<uint32_t*>(ring + NS * C::kStage);  // NS transposes
  const int col0 = lane * SBP + (lane / RB) * RB;  // this lane's column in a transpose
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)NP * C::kTeamBytes) + team * 3 * NS;
  uint64_t* tot = full + NS;    // totals warp done with the slot's S and A
  uint64_t* ready = tot + NS;   // left-sum warp has left E in the slot's transpose
  const int64_t nsw = (width + kStripCols - 1) / kStripCols, units = batch * nsw;
  const int nst = (int)((height + RB - 1) / RB);
  const StripSched sc{units, (int64_t)gridDim.x * NP, (int)gridDim.x, (int)blockIdx.x, team};
  const int64_t njobs = sc.rounds() * nst;  // (unit, stage) jobs of this team, in order
  if (njobs == 0) return;  // the whole team; no CTA-wide barrier follows
  // Job q: stage jb.i of the team's (q / nst)-th unit, ring slot q % NS.
  if (role == 0) {
    // ----------------------------------------------------- totals warp
    team_sync(team);  // the walk warp has initialised the barriers
    constexpr int L = 32 / HL;
    const int r = lane % RB, h = lane / RB;  // row and part of the row in the scan across lanes
    uint32_t s1 = 0;
    bool ok = true;
    for (StripJob jc(sc, nsw); jc.q < njobs; jc.next(nst, sc, nsw)) {
      const int k = (int)(jc.q % NS);
      ok = __all_sync(kFull, mbar_wait_bounded(full + k, (uint32_t)((jc.q / NS) & 1), limit));
      if (!ok) break;
      if (jc.i == 0) s1 = 0;
      const uint8_t* stage = ring + k * C::kStage;
      uint32_t* sb = sbuf + k * C::kSbWords;
#pragma unroll
      for (int r0 = 0; r0 < RB; r0 += 4) {
        uint32_t s4[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          s1 = strip_add_total<DT>(stage, r0 + t, lane, s1);
          s4[t] = s1;
        }
        *reinterpret_cast<uint4*>(sb + col0 + r0) = make_uint4(s4[0], s4[1], s4[2], s4[3]);
      }
      __syncwarp();
      // Lane (r, h) scans lanes [h * L, (h + 1) * L) of row r: the
      // exclusive sums across lanes go back into the transpose, and the
      // row's total is A(y).
      uint32_t* sr = sb + h * L * SBP + h * RB + r;  // column h * L (skewed), row r
      uint32_t seg = 0;
#pragma unroll
      for (int t = 0; t < L; ++t) seg += sr[t * SBP];
      uint32_t pre = seg;
#pragma unroll
      for (int d = RB; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, pre, d);
        if (lane >= d) pre += u;
      }
      const uint32_t a = __shfl_sync(kFull, pre, r + 32 - RB);  // the last part's inclusive sum
      uint32_t e = pre - seg;
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const uint32_t v = sr[t * SBP];
        sr[t * SBP] = e;
        e += v;
      }
      const int64_t y = (int64_t)jc.i * RB + lane;
      if (lane < RB && y < height)
        st_relaxed_u64(reinterpret_cast<uint64_t*>(A + jc.g * height + y), ((uint64_t)kATag << 32) | a);
      __syncwarp();
      if (lane == 0) mbar_arrive(tot + k);
    }
    if (!ok && lane == 0) atomicOr(status, kDevTimeout);
    return;
  }
  if (role == 1) {
    // -------------------------------------------------- left-sum warp
    team_sync(team);
    const int r = lane % RB, h = lane / RB;  // row and part of the row
    // A job's row r, part h: its left-strip words (strips h, h + HL, ...
    // below s; cnt of them from p on, stride apart) and the first group of
    // them, loaded two jobs ahead.
    struct Pre {
      const unsigned long long* p;
      int cnt;
      uint64_t w[kClGroup];
    };
    Pre pa, pb;
    const int64_t stride = (int64_t)HL * height;
    auto prefetch = [&](const StripJob& jb, Pre& pr) {
      const int64_t y = (int64_t)jb.i * RB + r;
      pr.cnt = (jb.q < njobs && y < height && jb.s > h) ? (int)((jb.s - h + HL - 1) / HL) : 0;
      pr.p = A + (jb.g - jb.s + h) * height + y;
      load_tagged(pr.p, stride, 0, min(pr.cnt, kClGroup), pr.w);
    };
    int k = 0;         // the current job's slot
    uint32_t par = 0;  // and the parity of its use
    // Left sum of the current job from its prefetched words, then added into
    // the slot's transpose; false on timeout.
    auto step = [&](const Pre& pr) {
      if (!__all_sync(kFull, mbar_wait_bounded(tot + k, par, limit))) return false;
      uint32_t cl = 0;
      bool good = add_tagged(pr.p, stride, 0, min(pr.cnt, kClGroup), pr.w, limit, &cl);
      for (int j0 = kClGroup; good && j0 < pr.cnt; j0 += kClGroup) {
        const int j1 = min(pr.cnt, j0 + kClGroup);
        uint64_t w2[kClGroup];
        load_tagged(pr.p, stride, j0, j1, w2);
        good = add_tagged(pr.p, stride, j0, j1, w2, limit, &cl);
      }
      if (!__all_sync(kFull, good)) return false;
#pragma unroll
      for (int d = RB; d < 32; d <<= 1) cl += __shfl_xor_sync(kFull, cl, d);
      // Lane (r, h) adds the left sum to lanes [h * L, (h + 1) * L) of row r.
      constexpr int L = 32 / HL;
      uint32_t* sr = sbuf + k * C::kSbWords + h * L * SBP + h * RB + r;
#pragma unroll
      for (int t = 0; t < L; ++t) sr[t * SBP] += cl;
      __syncwarp();
      if (lane == 0) mbar_arrive(ready + k);
      if (++k == NS) {
        k = 0;
        par ^= 1u;
      }
      return true;
    };
    StripJob j2(sc, nsw);  // the job two ahead of the current one
    prefetch(j2, pa);
    j2.next(nst, sc, nsw);
    prefetch(j2, pb);
    j2.next(nst, sc, nsw);
    bool ok = true;
    // Jobs alternate between the two prefetch buffers, each refilled with
    // the job two ahead as soon as its own job is done.
    for (int64_t q = 0; q < njobs; q += 2) {
      ok = step(pa);
      if (!ok) break;
      prefetch(j2, pa);
      j2.next(nst, sc, nsw);
      if (q + 1 >= njobs) break;
      ok = step(pb);
      if (!ok) break;
      prefetch(j2, pb);
      j2.next(nst, sc, nsw);
    }
    if (!ok && lane == 0) atomicOr(status, kDevTimeout);
    return;
  }
  // --------------------------------------------------------- walk warp
  StripJob jw(sc, nsw), ji(sc, nsw);  // walked, next to issue
  auto issue = [&]() {
    const int slot = (int)(ji.q % NS);
    mbar_arrive_expect_tx(full + slot, C::kStage);
    tma_load_3d(ring + slot * C::kStage, &tin, (int)(ji.s * kStripCols), ji.i * RB, (int)ji.b, full + slot);
    ji.next(nst, sc, nsw);
  };
  if (lane == 0) {
    for (int k = 0; k < 3 * NS; ++k) mbar_init(full + k, 1);  // full, tot, ready
    mbar_init_fence();
    while (ji.q < NS && ji.q < njobs) issue();
  }
  __syncwarp();
  team_sync(team);
  bool ok = true;
  uint32_t c[4] = {0u, 0u, 0u, 0u};  // c_j(y, lane)
  for (; jw.q < njobs; jw.next(nst, sc, nsw)) {
    const int k = (int)(jw.q % NS);
    const uint32_t par = (uint32_t)((jw.q / NS) & 1);
    ok = __all_sync(kFull, mbar_wait_bounded(ready + k, par, limit) && mbar_wait_bounded(full + k, par, limit));
    if (!ok) break;
    if (jw.i == 0) c[0] = c[1] = c[2] = c[3] = 0u;
    const uint8_t* stage = ring + k * C::kStage;
    const uint32_t* sb = sbuf + k * C::kSbWords + col0;
    const int64_t y0 = (int64_t)jw.i * RB;
    const int64_t x = jw.s * kStripCols + 4 * lane;
    const bool in_img = x < width;
    uint32_t* po = out + (jw.b * height + y0) * width + x;
    const int nrows = (int)min((int64_t)RB, height - y0);
    // Rows past the image (zeros from the TMA fill) are walked but not
    // stored, so the loop has no exit.
#pragma unroll
    for (int r0 = 0; r0 < RB; r0 += 4) {
      const uint4 e4 = *reinterpret_cast<const uint4*>(sb + r0);
      const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = r0 + t;
        strip_add_prefixes<DT>(stage, r, lane, c);
        if (in_img && r < nrows)
          __stcs(reinterpret_cast<uint4*>(po + (int64_t)r * width),
                 make_uint4(c[0] + e[t], c[1] + e[t], c[2] + e[t], c[3] + e[t]));
      }
    }
    // Release the slot: this lane's reads of it come before the refill.
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0 && ji.q < njobs) issue();
    __syncwarp();
  }
  if (!ok && lane == 0) {
    atomicOr(status, kDevTimeout);
    for (int64_t q = jw.q; q < ji.q; ++q)  // copies still in flight land before the warp exits
      mbar_wait_bounded(full + (int)(q % NS), (uint32_t)((q / NS) & 1), limit);
  }
  __syncwarp();
}

// Tensor map of the images as a 3-D array (columns, rows, images) of
// 8- or 32-bit pixels, boxes of 128 columns x RB rows of one image.
template <int DT>
static bool encode_strip_map(CUtensorMap* map, const void* img, int64_t batch, int64_t height, int64_t width) {
  const auto encode = tensor_map_encoder();
  if (!encode) return false;
  constexpr int EB = StripCfg<DT>::EB;
  const cuuint64_t dims[3] = {(cuuint64_t)width, (cuuint64_t)height, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)width * EB, (cuuint64_t)(width * height) * EB};
  const cuuint32_t box[3] = {kStripCols, (cuuint32_t)StripCfg<DT>::RB, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, DT == COX_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                const_cast<void*>(img), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t ws_p_bytes(int64_t batch, int64_t height, int64_t width);
inline size_t strip_a_bytes(int64_t batch, int64_t height, int64_t width) {
  return (size_t)batch * ((width + kStripCols - 1) / kStripCols) * height * sizeof(unsigned long long);
}

template <int DT>
static cox_status launch_intimage(const void* d_in, int64_t batch, int64_t height, int64_t width, uint32_t* d_out,
                                  uint32_t* P, uint32_t* CS, uint32_t* BT, cudaStream_t st) {
  const int64_t rows = batch * height;
  const int64_t ns = (width + 31) / 32, nb = (height + kBand - 1) / kBand;
  const bool vec = aligned16(d_in) && width % (DT == COX_U8 ? 16 : 4) == 0;
  auto grid_of = [](auto k, int64_t warps) {
    const int g = persistent_grid(k, 256, 0, 1 << 30);
    const int64_t ctas = (warps + 7) / 8;
    return (int)(ctas < g ? (ctas < 1 ? 1 : ctas) : g);
  };
  const int64_t nstrip = (width + kStripCols - 1) / kStripCols;
  if (vec && aligned16(d_out) && batch * nstrip >= (int64_t)kStripUnitsPerSm * sm_count() &&
      nstrip <= kStripMaxStrips && height < (int64_t)1 << 31 && batch < (int64_t)1 << 31 &&
      strip_a_bytes(batch, height, width) <= ws_p_bytes(batch, height, width)) {
    // A (one tagged 8-byte word per image row and strip) in P's space.
    using Cf = StripCfg<DT>;
    CUtensorMap map;
    if (!encode_strip_map<DT>(&map, d_in, batch, height, width)) return COX_ECUDA;
    unsigned long long* A = reinterpret_cast<unsigned long long*>(P);
    if (cudaMemsetAsync(A, 0, strip_a_bytes(batch, height, width), st) != cudaSuccess) return COX_ECUDA;
    auto kern = k_strip_walk<DT>;
    static int grid[kMaxDevices];  // co-resident CTAs, per device
    int& g = grid[device_index()];
    if (g == 0) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::kSmem) != cudaSuccess)
        return COX_ECUDA;
      g = persistent_grid(kern, 96 * Cf::NP, Cf::kSmem, 1 << 30);
    }
    // Every resident CTA, so the units spread over all SMs.
    const int64_t units = batch * nstrip;
    const int ctas = (int)(units < g ? units : g);
    uint32_t limit = spin_limit();
    unsigned* status = device_status_word();
    void* args[] = {(void*)&map, (void*)&batch, (void*)&height, (void*)&width, (void*)&d_out, (void*)&A,
                    (void*)&limit, (void*)&status};
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)ctas), dim3(96 * Cf::NP), args, Cf::kSmem, st) !=
        cudaSuccess) {
      cudaGetLastError();
      return COX_ECUDA;
    }
    return COX_OK;
  }
  if (vec && aligned16(d_out)) {  // T in P's space, C in CS's
    constexpr int SW = 32 * (DT == COX_U8 ? 16 : 4);
    const int64_t vunits = batch * nb * ((width + SW - 1) / SW);
    auto k1 = k_block_sums_vec<DT>;
    k1<<<grid_of(k1, vunits), 256, 0, st>>>(d_in, batch, height, width, P, CS, BT);
    auto k2 = k_band_walk_vec<DT>;
    k2<<<grid_of(k2, vunits), 256, 0, st>>>(d_in, batch, height, width, P, CS, BT, d_out);
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
// word per image, band and column), then BT (one word per image, band and
// 128 columns), each rounded to 16 bytes.
size_t cox::ws_p_bytes(int64_t batch, int64_t height, int64_t width) {
  return ((size_t)batch * height * ((width + 31) / 32) * sizeof(uint32_t) + 15) & ~(size_t)15;
}
static size_t ws_cs_bytes(int64_t batch, int64_t height, int64_t width) {
  return ((size_t)batch * ((height + kBand - 1) / kBand) * width * sizeof(uint32_t) + 15) & ~(size_t)15;
}

static size_t ws_bt_bytes(int64_t batch, int64_t height, int64_t width) {
  return ((size_t)batch * ((height + kBand - 1) / kBand) * ((width + 127) / 128) * sizeof(uint32_t) + 15) &
         ~(size_t)15;
}

extern "C" size_t cox_integral_image_workspace(int64_t batch, int64_t height, int64_t width) {
  if (batch < 0 || height < 0 || width < 0) return 0;
  return ws_p_bytes(batch, height, width) + ws_cs_bytes(batch, height, width) + ws_bt_bytes(batch, height, width) +
         16;
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
  uint32_t* BT = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(CS) + ws_cs_bytes(batch, height, width));
  cudaStream_t st = as_stream(stream);
  if (in_dt == COX_U8) return launch_intimage<COX_U8>(d_in, batch, height, width, d_out, P, CS, BT, st);
  return launch_intimage<COX_U32>(d_in, batch, height, width, d_out, P, CS, BT, st);
}
