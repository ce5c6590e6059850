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
// 16-byte form (16-byte aligned input and output, rows a whole number of
// 16-byte units), two passes that read the pixels twice: block sums per
// (image, band, 512- or 128-column strip), then the band walkers (below).
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
static size_t ws_p_bytes(int64_t batch, int64_t height, int64_t width) {
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
