// Request server: continuous batching of reduce, scan and compact requests.
//
// Host side.  A device arena of `budget` bytes holds every admitted
// request's output and workspace; a scheduler thread admits queued requests
// in arrival order while the arena and the slot count allow, packs all
// admitted, not yet launched requests into one persistent launch on its
// slot's stream (so a batch launched while an earlier one runs overlaps it
// on the device; at most kBatchSlots such batches at a time), and marks each
// request done when the kernel raises the request's flag in pinned host
// memory (after the request's last tile), or at the latest when the batch's
// event fires.  At low load (only lone requests in flight, a short queue)
// every request goes out alone as soon as it arrives, with its op's own
// kernel on one stream shared by all slots, in order, and completes with
// its slot's event: one launch per request, as without the server.
//
// Device side.  A batch is a table of request descriptors; each request is
// cut into tiles of kTile = 16384 elements (64 KB), numbered consecutively
// request by request.  Persistent CTAs take tile numbers from an atomic
// counter, so a request's tiles are taken in order: a compaction tile only
// ever waits (in its look-back) on smaller tiles of its own request, already
// taken by CTAs that run.  A tile arrives in shared memory by one TMA bulk
// copy (plain loads for a ragged or unaligned tile), then:
//   REDUCE  every thread folds its 64 elements (TwoSum pairs for fp32), a
//           block tree gives the tile's partial; the request's last tile
//           folds all partials in tile order;
//   SCAN    every warp scans its 64 rows of 32 in place (shfl_up at the
//           request's tile width) and the tile leaves by one TMA bulk store;
//   COMPACT the big-tile compaction shared with cox_ballot_compact.
// A request's arithmetic depends only on the request, never on its batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "compact_tile.cuh"

namespace cox {

constexpr int kServeBlock = 256;
constexpr int64_t kTile = kBigTile;  // 16384 elements per tile
constexpr int kSlots = 8;            // launches in flight (lone requests or batches)
constexpr int kBatchSlots = 3;       // batches of several requests in flight
constexpr int kMaxBatch = 2048;      // requests per launch
constexpr size_t kAlign = 256;

struct ReqDesc {
  int kind, dt, width;
  unsigned flags;
  int64_t n, threshold;
  const uint32_t* in;
  uint32_t* out;
  uint8_t* ws;
  int64_t item0, nitems;
};

struct BatchHdr {
  int64_t nitems;
  int nreq;
  int pad[13];
};  // 64 bytes, followed by nreq ReqDesc
static_assert(sizeof(BatchHdr) == 64, "batch header layout");

inline size_t table_bytes(size_t nreq) { return sizeof(BatchHdr) + nreq * sizeof(ReqDesc); }

// Batches of at most kParamReqs requests travel as a kernel parameter, so
// their launch needs no copy of the table first.
constexpr int kParamReqs = 24;
struct ParamTable {
  BatchHdr hdr;
  ReqDesc reqs[kParamReqs];
};

// A slot's counters in device memory: the tile counter the CTAs take tiles
// from, per request the tiles finished and the reduce tiles folded, and the
// CTAs that have exited.  Zero before a launch; the launch's last CTA to
// exit zeroes what the batch used, so the next launch on the slot (same
// stream) finds them zero again.
struct SlotCtr {
  unsigned long long next;
  unsigned exited;
  unsigned pad;
  unsigned fin[kMaxBatch];
  unsigned red[kMaxBatch];
};

__host__ __device__ inline int64_t serve_items(int64_t n) { return (n + kTile - 1) / kTile; }

// Dynamic shared memory of k_serve: the tile, the compaction's warp counts,
// the mbarrier, and the per-request first-tile table.
constexpr int kServeCounts = kCompactWsWords;  // the compaction tile body's counts and offsets
inline size_t serve_smem(size_t nreq) { return (size_t)(kTile + kServeCounts + 4) * 4 + nreq * 4; }

// ---------------------------------------------------------------- reduce
// Thread t folds elements 1024 j + 4 t + k (j = 0..blocks-1, k = 0..3) of the
// tile, in that order; elements past the request's end count as 0.  The
// tile's block sum goes to part[c] in the request's workspace; the tile that
// completes the request folds the parts (thread t: parts t, t + 256, ...),
// block-reduces them and writes the sum and its low word.  `ctr` counts the
// request's finished tiles; the folding tile returns true.
template <class R>
__device__ bool reduce_tile_finish(const ReqDesc& d, int64_t c, typename R::V acc, typename R::V* wpart,
                                   unsigned* ctr) {
  using T = typename R::T;
  using V = typename R::V;
  const int tid = threadIdx.x;
  const V bsum = block_reduce32<R>(acc, wpart);
  V* part = reinterpret_cast<V*>(d.ws);
  __shared__ int s_last;
  if (tid == 0) {
    part[c] = bsum;
    __threadfence();
    s_last = d.nitems == 1 || atomicAdd(ctr, 1u) == (unsigned)(d.nitems - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  V fold = R::ident();
  for (int64_t k = tid; k < d.nitems; k += kServeBlock) {
    V pv;
    if constexpr (R::kComp) {
      const float2 f = __ldcg(reinterpret_cast<const float2*>(part) + k);
      pv = {f.x, f.y};
    } else {
      pv = from_bits<T>(__ldcg(reinterpret_cast<const uint32_t*>(part) + k));
    }
    fold = R::op(fold, pv);
  }
  const V total = block_reduce32<R>(fold, wpart);
  if (tid == 0) {
    d.out[0] = to_bits(R::out(total));
    d.out[1] = __float_as_uint(R::lo(total));
  }
  return true;
}

// The fold of a tile staged in shared memory (the batch kernel).
template <class R>
__device__ void serve_reduce_tile(const ReqDesc& d, int64_t c, const uint32_t* buf, int blocks, typename R::V* wpart,
                                  unsigned* ctr) {
  using T = typename R::T;
  using V = typename R::V;
  const int tid = threadIdx.x;
  V acc = R::ident();
#pragma unroll 4
  for (int j = 0; j < blocks; ++j) {  // (the rest of a partial tile would only add the identity)
    const uint4 q = *reinterpret_cast<const uint4*>(buf + j * 4 * kServeBlock + 4 * tid);
    acc = R::op(acc, R::load(from_bits<T>(q.x)));
    acc = R::op(acc, R::load(from_bits<T>(q.y)));
    acc = R::op(acc, R::load(from_bits<T>(q.z)));
    acc = R::op(acc, R::load(from_bits<T>(q.w)));
  }
  reduce_tile_finish<R>(d, c, acc, wpart, ctr);
}

// A lone reduce request (a batch of one): one CTA per tile reads its tile
// straight from global memory in the batch kernel's element order, so the
// sum is the batch kernel's bit for bit, without its tile counter, request
// flags or exit count; the slot's event tells the host it is done.  `ctr`
// is the slot's reduce counter for request 0 (zero between launches; the
// folding CTA zeroes it again).
template <class R>
__global__ void __launch_bounds__(kServeBlock) k_serve_reduce_solo(const ReqDesc d, unsigned* ctr) {
  using T = typename R::T;
  using V = typename R::V;
  __shared__ V wpart[32];
  const int tid = threadIdx.x;
  const int64_t c = blockIdx.x, base = c * kTile;
  const int valid = (int)min(kTile, d.n - base);
  const int blocks = (valid + 1023) / 1024;
  const uint32_t* src = d.in + base;
  const bool vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
  V acc = R::ident();
#pragma unroll 4
  for (int j = 0; j < blocks; ++j) {
    const int e = j * 4 * kServeBlock + 4 * tid;
    uint4 q;
    if (vec && e + 4 <= valid) {
      q = __ldcs(reinterpret_cast<const uint4*>(src + e));
    } else {
      q.x = e < valid ? src[e] : 0u;
      q.y = e + 1 < valid ? src[e + 1] : 0u;
      q.z = e + 2 < valid ? src[e + 2] : 0u;
      q.w = e + 3 < valid ? src[e + 3] : 0u;
    }
    acc = R::op(acc, R::load(from_bits<T>(q.x)));
    acc = R::op(acc, R::load(from_bits<T>(q.y)));
    acc = R::op(acc, R::load(from_bits<T>(q.z)));
    acc = R::op(acc, R::load(from_bits<T>(q.w)));
  }
  if (reduce_tile_finish<R>(d, c, acc, wpart, ctr) && tid == 0) *ctr = 0u;
}

// ------------------------------------------------------------------ scan
// Thread t scans rows t and t + 256 of the tile (row r = elements 32 r ..
// 32 r + 31) in registers, each width-W tile collapsed into the thread
// (scan_row_regs), in place.  The tile is linear in shared memory (one 1D
// bulk copy per request tile), so a lane's 16-byte reads of its row meet
// 8-way bank conflicts; the tile's arithmetic, not shared memory, bounds it.
template <class R, int W>
__device__ void serve_scan_rows(uint32_t* buf, int rows) {
  using T = typename R::T;
  using V = typename R::V;
  uint4* b4 = reinterpret_cast<uint4*>(buf);
#pragma unroll 1
  for (int h = 0; h < (int)(kTile / 32 / kServeBlock); ++h) {
    const int r = h * kServeBlock + threadIdx.x;
    if (r >= rows) break;  // rows past a partial tile's end are not needed
    V v[32];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 q = b4[r * 8 + j];
      v[4 * j] = R::load(from_bits<T>(q.x));
      v[4 * j + 1] = R::load(from_bits<T>(q.y));
      v[4 * j + 2] = R::load(from_bits<T>(q.z));
      v[4 * j + 3] = R::load(from_bits<T>(q.w));
    }
    scan_row_regs<R, W>(v);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      b4[r * 8 + j] = make_uint4(to_bits(R::out(v[4 * j])), to_bits(R::out(v[4 * j + 1])),
                                 to_bits(R::out(v[4 * j + 2])), to_bits(R::out(v[4 * j + 3])));
  }
}

template <class R>
__device__ void serve_scan_tile(const ReqDesc& d, uint32_t* buf, int rows) {
  switch (d.width) {
    case 2: serve_scan_rows<R, 2>(buf, rows); break;
    case 4: serve_scan_rows<R, 4>(buf, rows); break;
    case 8: serve_scan_rows<R, 8>(buf, rows); break;
    case 16: serve_scan_rows<R, 16>(buf, rows); break;
    default: serve_scan_rows<R, 32>(buf, rows); break;
  }
}

// Marks a finished tile of request r (thread 0, after a __syncthreads that
// follows the tile's last writes): the tile that completes the request
// raises the request's flag in host memory, so the host sees each request
// as soon as its own results are in memory, not when the whole launch ends.
__device__ __forceinline__ void serve_tile_done(SlotCtr* ctr, unsigned* hflag, const ReqDesc* reqs, int r) {
  __threadfence();
  if (reqs[r].nitems == 1 || atomicAdd(ctr->fin + r, 1u) == (unsigned)(reqs[r].nitems - 1)) {
    __threadfence_system();
    asm volatile("st.release.sys.u32 [%0], %1;" ::"l"(hflag + r), "r"(1u) : "memory");
  }
}

__device__ __forceinline__ void serve_body(const ReqDesc* reqs, int nreq, int64_t nitems, SlotCtr* ctr,
                                           unsigned* hflag, uint32_t limit, unsigned* status) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Pair wpart_c[32];
  __shared__ uint32_t wpart_u[32];
  __shared__ float wpart_f[32];
  __shared__ int64_t s_item;
  __shared__ int s_req;
  __shared__ int s_last;
  uint32_t* buf = smem;                                           // the tile
  uint32_t* wcnt = smem + kTile;                                  // compaction warp counts
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kTile + kServeCounts);
  uint32_t* first = smem + kTile + kServeCounts + 4;              // first tile of every request
  const int tid = threadIdx.x;
  // Tile numbers fit 32 bits: a batch holds at most kMaxBatch requests of
  // fewer than 2^31 elements each.
  for (int r = tid; r < nreq; r += blockDim.x) first[r] = (uint32_t)reqs[r].item0;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  uint32_t loads = 0;  // bulk copies completed on `bar`
  int pending = -1;    // request of the tile this CTA finished last, not yet marked
  for (;;) {
    // Every thread's accesses to the tile, ordered before the async proxy's
    // next write to it; the previous tile's bulk store has completed.
    fence_proxy_async_smem();
    if (tid == 0) {
      tma_store_wait_all();
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
      if (pending >= 0) serve_tile_done(ctr, hflag, reqs, pending);
      // tiles come from the counter only: a tile is only ever handed to a CTA
      // that runs, which a compaction tile's look-back relies on
      const int64_t item = (int64_t)atomicAdd(&ctr->next, 1ull);
      s_item = item;
      if (item < nitems) {
        int lo = 0, hi = nreq;  // last request whose first tile <= item
        while (hi - lo > 1) {
          const int m = (lo + hi) >> 1;
          if ((int64_t)first[m] <= item) lo = m;
          else hi = m;
        }
        s_req = lo;
      }
    }
    pending = -1;
    __syncthreads();
    const int64_t item = s_item;
    if (item >= nitems) break;
    const ReqDesc d = reqs[s_req];
    const int64_t c = item - d.item0;
    const int64_t base = c * kTile;
    const int valid = (int)min(kTile, d.n - base);
    // ---- the tile into shared memory (0 past the request's end: the sums' identity)
    if (valid == kTile && (reinterpret_cast<uintptr_t>(d.in) & 15u) == 0) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(kTile * 4));
        tma_load_1d(buf, d.in + base, (uint32_t)(kTile * 4), bar);
      }
      const bool ok = mbar_wait_bounded(bar, loads & 1u, limit);
      ++loads;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(status, (unsigned)kDevTimeout);
          mbar_wait_bounded(bar, (loads - 1) & 1u, limit);  // the copy in flight, before the CTA ends
        }
        break;
      }
    } else {
      // a partial tile: its keys, then zeros up to the block (reduce: 1024
      // elements) or row (scan: 32) that holds its end
      const int span = d.kind == COX_REQ_REDUCE ? 1024 : d.kind == COX_REQ_SCAN ? 32 : 1;
      const int end = (valid + span - 1) / span * span;
      for (int i = tid; i < end; i += blockDim.x) buf[i] = i < valid ? d.in[base + i] : 0u;
      __syncthreads();
    }
    if (d.kind == COX_REQ_REDUCE) {
      const int blocks = (valid + 1023) / 1024;
      if (d.dt == COX_F32) {
        if (d.flags & COX_F_COMPENSATED) serve_reduce_tile<Comp>(d, c, buf, blocks, wpart_c, ctr->red + s_req);
        else serve_reduce_tile<Plain<AddF>>(d, c, buf, blocks, wpart_f, ctr->red + s_req);
      } else {
        serve_reduce_tile<Plain<AddU>>(d, c, buf, blocks, wpart_u, ctr->red + s_req);
      }
    } else if (d.kind == COX_REQ_SCAN) {
      const int rows = (valid + 31) / 32;
      if (d.dt == COX_F32) {
        if (d.flags & COX_F_COMPENSATED) serve_scan_tile<Comp>(d, buf, rows);
        else serve_scan_tile<Plain<AddF>>(d, buf, rows);
      } else {
        serve_scan_tile<Plain<AddU>>(d, buf, rows);
      }
      uint32_t* dst = d.out + base;
      if (valid == kTile && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        fence_proxy_async_smem();  // this thread's stores to the tile, before the bulk copy reads it
        __syncthreads();
        if (tid == 0) tma_store_1d(dst, buf, (uint32_t)(kTile * 4));
      } else {
        __syncthreads();
        for (int i = tid; i < valid; i += blockDim.x) dst[i] = buf[i];
      }
    } else {
      int64_t* count = reinterpret_cast<int64_t*>(d.ws);
      uint64_t* desc = reinterpret_cast<uint64_t*>(d.ws + kAlign);
      if (d.dt == COX_I32)
        compact_big_tile<true, kServeBlock / 32>(buf, valid, d.threshold, d.out, count, desc, c, d.nitems, d.n, limit,
                                                 status, wcnt);
      else
        compact_big_tile<false, kServeBlock / 32>(buf, valid, d.threshold, d.out, count, desc, c, d.nitems, d.n, limit,
                                                  status, wcnt);
    }
    pending = s_req;  // marked at the top of the next round, once its writes (and bulk store) are done
  }
  // ---- the last tile's mark; the last CTA out zeroes the slot's counters
  fence_proxy_async_smem();
  if (tid == 0) {
    tma_store_wait_all();  // no bulk store outlives the CTA
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    if (pending >= 0) serve_tile_done(ctr, hflag, reqs, pending);
    __threadfence();
    s_last = atomicAdd(&ctr->exited, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int r = tid; r < nreq; r += blockDim.x) {
      ctr->fin[r] = 0u;
      ctr->red[r] = 0u;
    }
    if (tid == 0) {
      ctr->next = 0ull;
      ctr->exited = 0u;
    }
    __syncthreads();
    if (tid == 0) {  // the whole batch is done: the host may reuse the slot
      __threadfence_system();
      asm volatile("st.release.sys.u32 [%0], %1;" ::"l"(hflag + kMaxBatch), "r"(1u) : "memory");
    }
  }
}


__global__ void __launch_bounds__(kServeBlock, 3) k_serve_tab(const uint8_t* __restrict__ table, SlotCtr* ctr,
                                                              unsigned* hflag, uint32_t limit, unsigned* status) {
  const BatchHdr* hdr = reinterpret_cast<const BatchHdr*>(table);
  serve_body(reinterpret_cast<const ReqDesc*>(table + sizeof(BatchHdr)), hdr->nreq, hdr->nitems, ctr, hflag, limit,
             status);
}

__global__ void __launch_bounds__(kServeBlock, 3) k_serve_par(const __grid_constant__ ParamTable pt, SlotCtr* ctr,
                                                              unsigned* hflag, uint32_t limit, unsigned* status) {
  serve_body(pt.reqs, pt.hdr.nreq, pt.hdr.nitems, ctr, hflag, limit, status);
}

// Zeroes the look-back descriptors of every compaction request of a batch
// (launched only for batches that hold one).
__device__ __forceinline__ void serve_prep(const ReqDesc& d) {
  if (d.kind != COX_REQ_COMPACT) return;
  const size_t words = compact_ws_bytes(d.nitems) / 4;  // count, tile and group descriptors
  uint32_t* w = reinterpret_cast<uint32_t*>(d.ws);
  for (size_t i = threadIdx.x; i < words; i += blockDim.x) w[i] = 0u;
}
__global__ void k_serve_prep_tab(const uint8_t* __restrict__ table) {
  const BatchHdr* hdr = reinterpret_cast<const BatchHdr*>(table);
  if ((int)blockIdx.x < hdr->nreq) serve_prep(reinterpret_cast<const ReqDesc*>(table + sizeof(BatchHdr))[blockIdx.x]);
}
__global__ void k_serve_prep_par(const __grid_constant__ ParamTable pt) {
  if ((int)blockIdx.x < pt.hdr.nreq) serve_prep(pt.reqs[blockIdx.x]);
}

// --------------------------------------------------------------- host side
double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t round_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Bytes a request holds in the arena: [output | workspace].
void request_bytes(const cox_request& r, size_t* out_b, size_t* ws_b) {
  const int64_t items = serve_items(r.n);
  switch (r.kind) {
    case COX_REQ_REDUCE: *out_b = kAlign; *ws_b = round_up((size_t)items * 8); break;
    case COX_REQ_SCAN: *out_b = round_up((size_t)r.n * 4); *ws_b = 0; break;
    default:  // [count | descriptors]: the batch kernel's, or a solo cox_ballot_compact's workspace
      *out_b = round_up((size_t)r.n * 4);
      *ws_b = kAlign + round_up(std::max(compact_ws_bytes(items), cox_ballot_compact_workspace(r.n, 256)));
      break;
  }
}

cox_status check_request(const cox_request& r) {
  if (!r.d_in || r.n < 1) return COX_EINVAL;
  if (r.n >= (int64_t(1) << 31)) return COX_EUNSUPPORTED;  // keeps a batch's tile numbers below 2^31
  switch (r.kind) {
    case COX_REQ_REDUCE:
    case COX_REQ_SCAN:
      if (r.dt != COX_F32 && r.dt != COX_I32) return COX_EINVAL;
      if ((r.flags & COX_F_COMPENSATED) && r.dt != COX_F32) return COX_EINVAL;
      if (r.flags & ~(unsigned)COX_F_COMPENSATED) return COX_EINVAL;
      if (r.kind == COX_REQ_SCAN && !valid_width(r.width)) return COX_EINVAL;
      return COX_OK;
    case COX_REQ_COMPACT:
      return (r.dt == COX_I32 || r.dt == COX_U32) ? COX_OK : COX_EINVAL;
    default:
      return COX_EINVAL;
  }
}

// First-fit allocator over [0, cap) with coalescing; sizes are multiples of kAlign.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }

 private:
  size_t cap_;
  std::map<size_t, size_t> free_;
};

enum ReqState { kQueued, kReady, kRunning, kDone, kFailed };

struct SReq {
  cox_request r;
  ReqState state = kQueued;
  size_t off = 0, bytes = 0, out_b = 0, held = 0;
  double t_submit = 0.0, t_ready = 0.0, t_launch = 0.0, t_done = 0.0;
};

// While two or more batches run, admitted requests wait for the next launch
// until they fill the persistent grid with tiles or the oldest has waited
// this long: fewer, larger batches under load, no added wait at low load.
constexpr double kBatchDelay = 20e-6;
constexpr size_t kSoloQueue = 2;  // ready requests at most, at low load, that each run alone
constexpr double kEventPoll = 100e-6;  // how often a running batch's event is queried

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint8_t* host_tab = nullptr;
  uint8_t* dev_tab = nullptr;
  SlotCtr* ctr = nullptr;     // device counters, zero between launches
  unsigned* hflag = nullptr;  // per request of the batch: 1 once its results are in memory; word kMaxBatch:
                              // 1 once the whole batch is done (pinned, mapped)
  unsigned* dflag = nullptr;  // the same flags' device address
  bool busy = false;
  // Set once the batch's work and event are enqueued: until then the event
  // still describes the slot's previous batch (the launch may run on another
  // thread than the completion checks).
  std::atomic<bool> issued{false};
  bool solo = false;         // the batch ran as one op's own kernel (no flags: its event tells)
  cudaStream_t launched = nullptr;  // the stream the slot's work last went to
  double t_checked = 0.0;    // when the slot's event was last queried
  std::vector<uint64_t> tickets;
  std::vector<char> marked;  // requests of the batch already marked done
};

}  // namespace cox

using namespace cox;

struct cox_server {
  int dev = 0;
  uint8_t* arena_mem = nullptr;
  size_t budget = 0;
  Arena* arena = nullptr;
  size_t used = 0, peak = 0;
  int max_req = 0;
  int admitted = 0;
  int grid = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> ready;
  int64_t ready_items = 0;  // tiles of the admitted, not yet launched requests
  std::unordered_map<uint64_t, SReq> reqs;
  std::vector<std::pair<uint64_t, double>> finished;  // (ticket, t_done) for trace runners
  std::atomic<int64_t> nfinished{0};                   // entries added to `finished`, ever
  // Lone requests of every slot go to one stream, in launch order, as one
  // launch per request would; batches of several run on their slot's stream.
  cudaStream_t solo_st = nullptr;
  bool collect_finished = false;
  Slot slots[kSlots];
  std::thread thr;
  std::atomic<bool> stop{false};
  uint64_t next_ticket = 1;
  cox_server_stats stats{};

  // Writes the batch table of `ts` into the slot's pinned host buffer and
  // marks the requests running (caller holds `mu`).  Returns the table size
  // and sets *items and *has_compact.
  size_t fill_batch(Slot& sl, const std::vector<uint64_t>& ts, int64_t* items_out, bool* has_compact) {
    BatchHdr* h = reinterpret_cast<BatchHdr*>(sl.host_tab);
    ReqDesc* d = reinterpret_cast<ReqDesc*>(sl.host_tab + sizeof(BatchHdr));
    int64_t items = 0;
    bool compact = false;
    const double t_launch = now_s();
    for (size_t i = 0; i < ts.size(); ++i) {
      SReq& q = reqs[ts[i]];
      q.t_launch = t_launch;
      ReqDesc& e = d[i];
      e.kind = q.r.kind;
      e.dt = q.r.dt;
      e.width = q.r.width;
      e.flags = q.r.flags;
      e.n = q.r.n;
      e.threshold = q.r.threshold;
      e.in = static_cast<const uint32_t*>(q.r.d_in);
      e.out = reinterpret_cast<uint32_t*>(arena_mem + q.off);
      e.ws = arena_mem + q.off + q.out_b;
      e.item0 = items;
      e.nitems = serve_items(q.r.n);
      items += e.nitems;
      compact = compact || q.r.kind == COX_REQ_COMPACT;
      q.state = kRunning;
    }
    // (requests are < 2^31 elements each, so 2048 of them stay < 2^31 tiles)
    h->nitems = items;
    h->nreq = (int)ts.size();
    for (size_t i = 0; i < ts.size(); ++i) __atomic_store_n(sl.hflag + i, 0u, __ATOMIC_RELAXED);
    __atomic_store_n(sl.hflag + kMaxBatch, 0u, __ATOMIC_RELAXED);
    sl.t_checked = 0.0;
    sl.tickets = ts;
    sl.marked.assign(ts.size(), 0);
    sl.issued.store(false, std::memory_order_relaxed);
    sl.busy = true;
    stats.batches += 1;
    stats.max_batch = std::max<int64_t>(stats.max_batch, (int64_t)ts.size());
    *items_out = items;
    *has_compact = compact;
    return table_bytes(ts.size());
  }

  // Enqueues a filled batch on the slot's stream (without `mu`: submitters
  // are not held up by the launch calls).
  // A batch of one scan or compaction runs the op's own kernel (cox_tile_scan,
  // cox_ballot_compact), and a lone reduce k_serve_reduce_solo: the same
  // results bit for bit, at the latency of one launch per request.  Other small batches pass their table as a kernel
  // parameter; larger ones copy it to the slot's device table first.
  bool issue_batch(Slot& sl, size_t tab_bytes, int64_t items, bool has_compact) {
    const int nreq = reinterpret_cast<BatchHdr*>(sl.host_tab)->nreq;
    if (nreq == 1) {
      const ReqDesc& d = *reinterpret_cast<const ReqDesc*>(sl.host_tab + sizeof(BatchHdr));
      cox_status c = COX_EINVAL;
      if (d.kind == COX_REQ_SCAN) {
        c = cox_tile_scan(COX_SUM, (cox_dtype)d.dt, d.width, 256, d.in, d.out, d.n, d.flags, solo_st);
      } else if (d.kind == COX_REQ_COMPACT) {
        const size_t wsb = cox_ballot_compact_workspace(d.n, 256);
        c = cox_ballot_compact((cox_dtype)d.dt, 32, 256, d.in, d.n, d.threshold, d.out,
                               reinterpret_cast<int64_t*>(d.ws), d.ws + kAlign, wsb, 0u, solo_st);
      }
      if (d.kind == COX_REQ_REDUCE) {
        const unsigned nblk = (unsigned)d.nitems;
        unsigned* rc = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(sl.ctr) + offsetof(SlotCtr, red));
        if (d.dt == COX_F32 && (d.flags & COX_F_COMPENSATED))
          k_serve_reduce_solo<Comp><<<nblk, kServeBlock, 0, solo_st>>>(d, rc);
        else if (d.dt == COX_F32)
          k_serve_reduce_solo<Plain<AddF>><<<nblk, kServeBlock, 0, solo_st>>>(d, rc);
        else
          k_serve_reduce_solo<Plain<AddU>><<<nblk, kServeBlock, 0, solo_st>>>(d, rc);
        c = cudaGetLastError() == cudaSuccess ? COX_OK : COX_ECUDA;
      }
      sl.solo = true;
      sl.launched = solo_st;
      return c == COX_OK && cudaEventRecord(sl.ev, solo_st) == cudaSuccess;
    }
    sl.solo = false;
    sl.launched = sl.st;
    has_compact = has_compact && items > 1;  // (a lone tile's look-back reads no descriptor)
    const int g = (int)std::min<int64_t>(grid, items);
    const size_t smem = serve_smem((size_t)nreq);
    if (nreq <= kParamReqs) {
      ParamTable pt;
      std::memcpy(&pt.hdr, sl.host_tab, sizeof(BatchHdr));
      std::memcpy(pt.reqs, sl.host_tab + sizeof(BatchHdr), (size_t)nreq * sizeof(ReqDesc));
      if (has_compact) k_serve_prep_par<<<(unsigned)nreq, 256, 0, sl.st>>>(pt);
      k_serve_par<<<g, kServeBlock, smem, sl.st>>>(pt, sl.ctr, sl.dflag, spin_limit(), device_status_word());
    } else {
      if (cudaMemcpyAsync(sl.dev_tab, sl.host_tab, tab_bytes, cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
        return false;
      if (has_compact) k_serve_prep_tab<<<(unsigned)nreq, 256, 0, sl.st>>>(sl.dev_tab);
      k_serve_tab<<<g, kServeBlock, smem, sl.st>>>(sl.dev_tab, sl.ctr, sl.dflag, spin_limit(), device_status_word());
    }
    return cudaGetLastError() == cudaSuccess && cudaEventRecord(sl.ev, sl.st) == cudaSuccess;
  }

  // Marks request i of a running batch done (caller holds `mu`).
  void mark_done(Slot& sl, size_t i, ReqState state, double t) {
    if (sl.marked[i]) return;
    sl.marked[i] = 1;
    auto it = reqs.find(sl.tickets[i]);
    if (it == reqs.end()) return;
    it->second.state = state;
    it->second.t_done = t;
    if (collect_finished) {
      finished.emplace_back(sl.tickets[i], t);
      nfinished.fetch_add(1, std::memory_order_release);
    }
    if (state == kDone) {
      stats.completed += 1;
      stats.wait_s += it->second.t_launch - it->second.t_submit;
      stats.run_s += t - it->second.t_launch;
    } else {
      stats.failed += 1;
    }
  }

  // Admits queued requests in arrival order while the budget and the slot
  // count allow, then picks a free slot for the admitted ones when the rule
  // below says go (caller holds `mu`).  Returns the slot to launch, or null.
  Slot* plan_launch(size_t* tab_bytes, int64_t* items, bool* has_compact) {
    const double now = now_s();
    while (!queue.empty() && admitted < max_req) {
      SReq& q = reqs[queue.front()];
      size_t off;
      if (used + q.held > budget || !arena->alloc(q.bytes, &off)) break;
      q.off = off;
      q.state = kReady;
      q.t_ready = now;
      used += q.held;
      peak = std::max(peak, used);
      ++admitted;
      ready_items += serve_items(q.r.n);
      ready.push_back(queue.front());
      queue.pop_front();
    }
    int inflight = 0, batches = 0;  // busy slots; those running several requests
    for (const Slot& sl : slots) {
      inflight += sl.busy;
      batches += sl.busy && sl.tickets.size() > 1;
    }
    // Low load (only lone requests in flight, at most kSoloQueue ready): the
    // oldest ready request goes out alone at once.  Otherwise all ready
    // requests go out as one batch while at most one slot is busy, or once
    // they fill the grid or the oldest has waited kBatchDelay: fewer, larger
    // batches under load.
    if (ready.empty() || inflight >= kSlots) return nullptr;
    const bool solo_now = batches == 0 && ready.size() <= kSoloQueue;
    const bool batch_go = batches < kBatchSlots && (inflight <= 1 || ready_items >= grid ||
                                                    now - reqs[ready.front()].t_ready >= kBatchDelay);
    if (!solo_now && !batch_go) return nullptr;
    for (Slot& sl : slots) {
      if (sl.busy) continue;
      const size_t k = solo_now ? 1 : std::min<size_t>(ready.size(), kMaxBatch);
      std::vector<uint64_t> ts(ready.begin(), ready.begin() + k);
      ready.erase(ready.begin(), ready.begin() + k);
      *tab_bytes = fill_batch(sl, ts, items, has_compact);
      ready_items -= *items;
      return &sl;
    }
    return nullptr;
  }

  // Enqueues a planned batch (without `mu`); on failure its requests fail.
  void launch_planned(Slot* sl, size_t tab_bytes, int64_t items, bool has_compact) {
    if (issue_batch(*sl, tab_bytes, items, has_compact)) {
      sl->issued.store(true, std::memory_order_release);
      return;
    }
    // What did get enqueued ends before the slot's table is written again.
    cudaStreamSynchronize(sl->launched ? sl->launched : sl->st);
    std::lock_guard<std::mutex> g(mu);
    for (size_t i = 0; i < sl->tickets.size(); ++i) mark_done(*sl, i, kFailed, now_s());
    sl->tickets.clear();
    sl->busy = false;
    cv.notify_all();
  }

  void loop() {
    cudaSetDevice(dev);
    while (!stop.load(std::memory_order_relaxed)) {
      bool progress = false;
      Slot* launch = nullptr;
      size_t tab_bytes = 0;
      int64_t items = 0;
      bool has_compact = false;
      {
        std::lock_guard<std::mutex> g(mu);
        // Completions, from the flags the batch kernel raises in host memory:
        // each request's, then the batch's; its event is queried only now and
        // then (every kEventPoll seconds), for a batch whose kernel failed.  A
        // lone request run as its op's own kernel completes with its event.
        for (Slot& sl : slots) {
          if (!sl.busy || !sl.issued.load(std::memory_order_acquire)) continue;
          const double t = now_s();
          bool any = false;
          for (size_t i = 0; i < sl.tickets.size(); ++i)
            if (!sl.marked[i] && __atomic_load_n(sl.hflag + i, __ATOMIC_ACQUIRE)) {
              mark_done(sl, i, kDone, t);
              any = true;
            }
          bool free_slot = false;
          ReqState rest = kDone;
          if (__atomic_load_n(sl.hflag + kMaxBatch, __ATOMIC_ACQUIRE)) {
            free_slot = true;
          } else if (sl.solo || t - sl.t_checked >= kEventPoll) {
            sl.t_checked = t;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e != cudaErrorNotReady) {
              free_slot = true;
              rest = e == cudaSuccess ? kDone : kFailed;
            }
          }
          if (free_slot) {
            for (size_t i = 0; i < sl.tickets.size(); ++i) mark_done(sl, i, rest, t);
            sl.busy = false;
            sl.tickets.clear();
          }
          if (any || free_slot) {
            progress = true;
            cv.notify_all();
          }
        }
        const size_t queued = queue.size();
        launch = plan_launch(&tab_bytes, &items, &has_compact);
        progress = progress || launch || queue.size() != queued;
      }
      if (launch) launch_planned(launch, tab_bytes, items, has_compact);
      if (!progress) std::this_thread::yield();
    }
  }
};

extern "C" cox_status cox_server_create(size_t budget_bytes, int max_requests, cox_server** out) {
  if (!out || budget_bytes < kAlign || max_requests < 1) return COX_EINVAL;
  *out = nullptr;
  cox_server* s = new (std::nothrow) cox_server;
  if (!s) return COX_ENOMEM;
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return COX_ECUDA;
  }
  s->budget = budget_bytes & ~(kAlign - 1);
  s->max_req = max_requests;
  if (cudaMalloc(&s->arena_mem, s->budget) != cudaSuccess) {
    delete s;
    return COX_ENOMEM;
  }
  s->arena = new Arena(s->budget);
  if (cudaStreamCreateWithFlags(&s->solo_st, cudaStreamNonBlocking) != cudaSuccess) {
    cox_server_destroy(s);
    return COX_ECUDA;
  }
  const size_t tab = table_bytes(kMaxBatch);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&sl.host_tab, tab) != cudaSuccess || cudaMalloc(&sl.dev_tab, tab) != cudaSuccess ||
        cudaMalloc(&sl.ctr, sizeof(SlotCtr)) != cudaSuccess || cudaMemset(sl.ctr, 0, sizeof(SlotCtr)) != cudaSuccess ||
        cudaHostAlloc(&sl.hflag, (kMaxBatch + 1) * sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&sl.dflag, sl.hflag, 0) != cudaSuccess) {
      cox_server_destroy(s);
      return COX_ECUDA;
    }
  }
  const size_t smem = serve_smem(kMaxBatch);
  if (cudaFuncSetAttribute(k_serve_tab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_serve_par, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {  // (the counters' zeroing has landed)
    cox_server_destroy(s);
    return COX_ECUDA;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve_tab, kServeBlock, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  s->grid = per_sm * sm_count();
  device_status_word();
  s->stats.budget_bytes = s->budget;
  s->thr = std::thread([s] { s->loop(); });
  *out = s;
  return COX_OK;
}

namespace {

// A request's host record: validated, its arena bytes computed.
cox_status make_sreq(const cox_server* s, const cox_request& req, SReq* q) {
  const cox_status c = check_request(req);
  if (c != COX_OK) return c;
  q->r = req;
  q->t_submit = now_s();
  size_t ob, wb;
  request_bytes(req, &ob, &wb);
  q->out_b = ob;
  q->bytes = ob + wb;
  q->held = q->bytes + round_up((size_t)req.n * 4);  // input counted as held while in flight
  if (q->bytes > s->budget || q->held > s->budget) return COX_ENOMEM;
  return COX_OK;
}

// Queues count validated requests under one lock.  An idle server (nothing
// queued, ready or running) plans and launches them from the submitting
// thread when the server's device is current there, without waiting for the
// scheduler thread to notice them.
void enqueue(cox_server* s, SReq* qs, int64_t count, uint64_t* tickets) {
  Slot* launch = nullptr;
  size_t tab_bytes = 0;
  int64_t items = 0;
  bool has_compact = false;
  {
    std::lock_guard<std::mutex> g(s->mu);
    bool idle = s->queue.empty() && s->ready.empty();
    for (const Slot& sl : s->slots) idle = idle && !sl.busy;
    for (int64_t i = 0; i < count; ++i) {
      const uint64_t t = s->next_ticket++;
      s->reqs.emplace(t, qs[i]);
      s->queue.push_back(t);
      s->stats.submitted += 1;
      tickets[i] = t;
    }
    int cur = -1;
    if (idle && cudaGetDevice(&cur) == cudaSuccess && cur == s->dev)
      launch = s->plan_launch(&tab_bytes, &items, &has_compact);
  }
  if (launch) s->launch_planned(launch, tab_bytes, items, has_compact);
}

}  // namespace

extern "C" cox_status cox_server_submit(cox_server* s, const cox_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return COX_EINVAL;
  SReq q;
  const cox_status c = make_sreq(s, *req, &q);
  if (c != COX_OK) return c;
  enqueue(s, &q, 1, ticket);
  return COX_OK;
}

extern "C" cox_status cox_server_submit_many(cox_server* s, const cox_request* reqs, int64_t count,
                                             uint64_t* tickets) {
  if (!s || count < 0 || (count > 0 && (!reqs || !tickets))) return COX_EINVAL;
  std::vector<SReq> qs((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    const cox_status c = make_sreq(s, reqs[i], &qs[(size_t)i]);
    if (c != COX_OK) return c;
  }
  if (count > 0) enqueue(s, qs.data(), count, tickets);
  return COX_OK;
}

extern "C" cox_status cox_server_poll(cox_server* s, uint64_t ticket, int* done) {
  if (!s || !done) return COX_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return COX_EINVAL;
  if (it->second.state == kFailed) return COX_ECUDA;
  *done = it->second.state == kDone;
  return COX_OK;
}

extern "C" cox_status cox_server_wait(cox_server* s, uint64_t ticket, double timeout_s) {
  if (!s) return COX_EINVAL;
  std::unique_lock<std::mutex> g(s->mu);
  auto pred = [&] {
    auto it = s->reqs.find(ticket);
    return it == s->reqs.end() || it->second.state == kDone || it->second.state == kFailed;
  };
  if (!s->cv.wait_for(g, std::chrono::duration<double>(timeout_s), pred)) return COX_ETIMEOUT;
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return COX_EINVAL;
  return it->second.state == kDone ? COX_OK : COX_ECUDA;
}

extern "C" cox_status cox_server_result(cox_server* s, uint64_t ticket, void** d_out, int64_t* count) {
  if (!s || !d_out || !count) return COX_EINVAL;
  cox_request r;
  uint8_t* out;
  size_t out_b;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state != kDone) return COX_EINVAL;
    r = it->second.r;
    out = s->arena_mem + it->second.off;
    out_b = it->second.out_b;
  }
  *d_out = out;
  if (r.kind == COX_REQ_REDUCE) *count = 1;
  else if (r.kind == COX_REQ_SCAN) *count = r.n;
  else if (cudaMemcpy(count, out + out_b, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) return COX_ECUDA;
  return COX_OK;
}

static void release_locked(cox_server* s, std::unordered_map<uint64_t, SReq>::iterator it) {
  s->arena->release(it->second.off, it->second.bytes);
  s->used -= it->second.held;
  s->admitted -= 1;
  s->reqs.erase(it);
}

extern "C" cox_status cox_server_release(cox_server* s, uint64_t ticket) {
  if (!s) return COX_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return COX_EINVAL;
  if (it->second.state != kDone && it->second.state != kFailed) return COX_EBUSY;
  release_locked(s, it);
  return COX_OK;
}

extern "C" cox_status cox_server_get_stats(cox_server* s, cox_server_stats* st) {
  if (!s || !st) return COX_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  *st = s->stats;
  st->used_bytes = s->used;
  st->peak_bytes = s->peak;
  st->queued = (int64_t)s->queue.size();
  return COX_OK;
}

extern "C" void cox_server_destroy(cox_server* s) {
  if (!s) return;
  if (s->thr.joinable()) {
    for (;;) {  // let launched batches finish
      bool busy = false;
      {
        std::lock_guard<std::mutex> g(s->mu);
        for (Slot& sl : s->slots) busy = busy || sl.busy;
      }
      if (!busy) break;
      std::this_thread::yield();
    }
    s->stop.store(true);
    s->thr.join();
  }
  if (s->solo_st) {
    cudaStreamSynchronize(s->solo_st);
    cudaStreamDestroy(s->solo_st);
  }
  for (Slot& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.host_tab) cudaFreeHost(sl.host_tab);
    if (sl.dev_tab) cudaFree(sl.dev_tab);
    if (sl.ctr) cudaFree(sl.ctr);
    if (sl.hflag) cudaFreeHost(sl.hflag);
  }
  if (s->arena_mem) cudaFree(s->arena_mem);
  delete s->arena;
  delete s;
}

// ------------------------------------------------------------ trace runners
extern "C" cox_status cox_server_run_trace(cox_server* s, const cox_trace_item* items, int64_t count,
                                           double* latency_s, double* wall_s) {
  if (!s || (count > 0 && (!items || !latency_s)) || !wall_s) return COX_EINVAL;
  std::unordered_map<uint64_t, int64_t> index;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->finished.clear();
    s->collect_finished = true;
  }
  const double t0 = now_s();
  int64_t next = 0, done = 0;
  cox_status rc = COX_OK;
  std::vector<std::pair<uint64_t, double>> fin;
  int64_t seen = s->nfinished.load();
  double last = t0;
  while (done < count) {
    const double t = now_s() - t0;
    while (next < count && items[next].arrival_s <= t) {
      uint64_t tk;
      const cox_status c = cox_server_submit(s, &items[next].req, &tk);
      if (c != COX_OK) {
        rc = c;
        latency_s[next] = -1.0;
        ++done;
      } else {
        index[tk] = next;
      }
      ++next;
    }
    // (the lock only when the scheduler has added entries since the last look)
    const int64_t nf = s->nfinished.load(std::memory_order_acquire);
    if (nf != seen) {
      std::lock_guard<std::mutex> g(s->mu);
      fin.swap(s->finished);
      seen = nf;
    }
    for (auto& f : fin) {
      auto it = index.find(f.first);
      if (it == index.end()) continue;
      latency_s[it->second] = f.second - (t0 + items[it->second].arrival_s);
      last = std::max(last, f.second);
      cox_server_release(s, f.first);
      index.erase(it);
      ++done;
    }
    const bool idle = fin.empty();
    fin.clear();
    if (idle) std::this_thread::yield();
  }
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->collect_finished = false;
    s->finished.clear();
  }
  *wall_s = last - t0;
  return rc;
}

extern "C" size_t cox_percall_scratch(int64_t max_n) {
  if (max_n < 1) return 0;
  return round_up(cox_tile_reduce_workspace(COX_SCOPE_GRID, max_n, 256)) +
         round_up(cox_ballot_compact_workspace(max_n, 256)) + kAlign + round_up((size_t)max_n * 4);
}

extern "C" cox_status cox_percall_run_trace(const cox_trace_item* items, int64_t count, void* d_scratch,
                                            size_t scratch_bytes, double* latency_s, double* wall_s) {
  if ((count > 0 && (!items || !latency_s)) || !wall_s || !d_scratch) return COX_EINVAL;
  int64_t max_n = 1;
  for (int64_t i = 0; i < count; ++i) max_n = std::max(max_n, items[i].req.n);
  if (scratch_bytes < cox_percall_scratch(max_n)) return COX_ENOMEM;
  uint8_t* p = static_cast<uint8_t*>(d_scratch);
  const size_t red_b = round_up(cox_tile_reduce_workspace(COX_SCOPE_GRID, max_n, 256));
  const size_t cmp_b = round_up(cox_ballot_compact_workspace(max_n, 256));
  uint8_t* red_ws = p;
  uint8_t* cmp_ws = p + red_b;
  int64_t* d_count = reinterpret_cast<int64_t*>(p + red_b + cmp_b);
  uint8_t* out = p + red_b + cmp_b + kAlign;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return COX_ECUDA;
  std::vector<cudaEvent_t> ev((size_t)count, nullptr);
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return COX_ECUDA;
  std::vector<std::atomic<int>> launched((size_t)count);
  for (auto& l : launched) l.store(0);
  std::vector<double> t_done((size_t)count, 0.0);
  std::atomic<bool> failed{false};
  std::thread poller([&] {
    for (int64_t i = 0; i < count; ++i) {
      while (!launched[i].load(std::memory_order_acquire)) std::this_thread::yield();
      if (launched[i].load() < 0) continue;
      cudaError_t e;
      while ((e = cudaEventQuery(ev[i])) == cudaErrorNotReady) std::this_thread::yield();
      if (e != cudaSuccess) failed.store(true);
      t_done[i] = now_s();
    }
  });
  const double t0 = now_s();
  cox_status rc = COX_OK;
  for (int64_t i = 0; i < count; ++i) {
    while (now_s() - t0 < items[i].arrival_s) {
    }
    const cox_request& r = items[i].req;
    cox_status c = check_request(r);
    if (c == COX_OK) {
      if (r.kind == COX_REQ_REDUCE)
        c = cox_tile_reduce(COX_SUM, r.dt, 32, 256, COX_SCOPE_GRID, r.d_in, out, r.n, r.flags, out + 4, red_ws,
                            red_b, st);
      else if (r.kind == COX_REQ_SCAN)
        c = cox_tile_scan(COX_SUM, r.dt, r.width, 256, r.d_in, out, r.n, r.flags, st);
      else
        c = cox_ballot_compact(r.dt, 32, 256, r.d_in, r.n, r.threshold, out, d_count, cmp_ws, cmp_b, 0, st);
    }
    if (c == COX_OK && cudaEventRecord(ev[i], st) != cudaSuccess) c = COX_ECUDA;
    if (c != COX_OK) rc = c;
    launched[i].store(c == COX_OK ? 1 : -1, std::memory_order_release);
  }
  poller.join();
  double last = t0;
  for (int64_t i = 0; i < count; ++i) {
    latency_s[i] = launched[i].load() > 0 ? t_done[i] - (t0 + items[i].arrival_s) : -1.0;
    last = std::max(last, t_done[i]);
  }
  *wall_s = last - t0;
  for (auto& e : ev) cudaEventDestroy(e);
  cudaStreamDestroy(st);
  if (failed.load()) return COX_ECUDA;
  return rc;
}
