/*
 * CPU oracle of the warp-collective library -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package's smoke check and the bench's CPU-baseline
 * leg may load this library.  The product path never calls into it, and it
 * shares no code, header or constant with the CUDA library: the numeric codes
 * below are this file's own.
 *
 * What it is.  A plain, slow executor of CUDA warp-level function semantics on
 * CPU threads, built the way the paper collapses a CUDA block for a CPU
 * (Section 2.3, "hierarchical collapsing", Code 3; Section 3.6):
 *   - an inter-warp loop over warp ids (`wid`) wraps intra-warp loops over the
 *     32 lanes (`tx`);
 *   - per-lane registers are arrays replicated over the block (Section 3.6);
 *   - every warp function is a write phase, in which each lane stores its
 *     operand into an exchange array held by the CPU thread running the block
 *     (Section 3.2), followed by a read phase in which each lane computes its
 *     result from that array; the two loops are the implicit warp barriers for
 *     the RAW and WAR hazards of Section 3.2 (Code 5);
 *   - a block barrier ends an inter-warp loop; work done by one warp only is
 *     guarded by the warp-uniform flag of its lane 0 (loop peeling, Section 2.3);
 *   - blocks run one per task on a pool of CPU threads (Section 4).
 *
 * Warp-function semantics are those of the public PTX `shfl.sync`, `vote.sync`
 * and `match.sync` definitions, which the paper defers to (Section 2.2.1).
 * Ragged tails: lanes whose global index is >= n exist, hold the op's padding
 * value (identity of the op, predicate false, no histogram contribution), and
 * write nothing.
 *
 * Float results come in two kinds:
 *   - "emulate" functions run the GPU's shuffle trees in fp32 (plain, or with
 *     TwoSum-compensated pairs) in exactly the order the kernels use, so the
 *     one-element-per-lane kernels must match them value for value;
 *   - "ref" functions give the FP64 value of the plain definition (Neumaier
 *     summation of the fp32 inputs) and the sum of |x| over the contributing
 *     inputs, which the tests use for the relative-error bar.
 *
 * Parity pins (what fixes each function independently of itself) live in the
 * tests: brute-force per-lane formulas, Code 1 and Code 4 of the paper, numpy
 * reductions and filters, math.fsum, and the invariants of each op.
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread.
 * `-ffp-contract=off` keeps every fp32 add a single rounded add (no fused
 * forms), which the TwoSum emulation relies on.
 */

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <mutex>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- codes
enum Status { ST_OK = 0, ST_EINVAL = 1, ST_EUNSUPPORTED = 2 };
enum DType { DT_I32 = 0, DT_U32 = 1, DT_F32 = 2 };
enum Op { OP_SUM = 0, OP_MIN = 1, OP_MAX = 2, OP_AND = 3, OP_OR = 4, OP_XOR = 5 };
enum WarpFn {
  FN_SHFL_IDX = 0, FN_SHFL_UP = 1, FN_SHFL_DOWN = 2, FN_SHFL_XOR = 3,
  FN_BALLOT = 4, FN_ANY = 5, FN_ALL = 6, FN_MATCH_ANY = 7
};
enum Scope { SC_TILE = 0, SC_BLOCK = 1, SC_GRID = 2 };

int g_threads = 0;  // 0: one per hardware thread

int pool_threads() {
  if (g_threads > 0) return g_threads;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

// Section 4: the runtime maps one CUDA block to one CPU thread; a thread pool
// (named there as the natural optimisation of fork/join) runs the grid.
template <class Fn>
void launch_grid(int64_t grid, Fn&& fn) {
  int nt = pool_threads();
  if ((int64_t)nt > grid) nt = (int)grid;
  if (nt <= 1) {
    for (int64_t b = 0; b < grid; ++b) fn(b);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> workers;
  workers.reserve(nt);
  for (int t = 0; t < nt; ++t)
    workers.emplace_back([&] {
      for (;;) {
        int64_t b = next.fetch_add(1, std::memory_order_relaxed);
        if (b >= grid) break;
        fn(b);
      }
    });
  for (auto& w : workers) w.join();
}

bool pow2_width(int w) { return w >= 2 && w <= 32 && (w & (w - 1)) == 0; }
bool valid_block(int b) { return b >= 32 && b <= 1024 && b % 32 == 0; }

inline float as_f(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
inline uint32_t as_u(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

// ------------------------------------------------- Section 3.2: exchange array
// The array every warp function goes through.  It lives in the memory of the
// CPU thread that runs the block, so blocks running on different CPU threads
// never race on it (Section 3.2).
thread_local uint32_t warp_xchg[32];

// Debug switch for the planted-mistake test: when set, warp functions fuse the
// write and read phases into one lane loop, i.e. drop the RAW barrier of
// Section 3.2.  Off in every normal call.
bool g_fuse_phases = false;

// Source lane of shfl.sync for mode `fn` at width W (segment mask 32-W, clamp
// W-1): idx reads lane seg|(b & (W-1)); up reads lane-b if it stays at or
// above the segment start; down/xor read lane+b / lane^b if it stays at or
// below the segment end; otherwise the lane keeps its own value.
inline int shfl_src_lane(int fn, int lane, int b, int W) {
  const int seg = lane & ~(W - 1);
  const int last = seg + W - 1;
  int j;
  bool in;
  switch (fn) {
    case FN_SHFL_IDX: j = seg | (b & (W - 1)); in = true; break;
    case FN_SHFL_UP: j = lane - b; in = j >= seg; break;
    case FN_SHFL_DOWN: j = lane + b; in = j <= last; break;
    default: j = lane ^ b; in = j <= last; break;  // xor (butterfly)
  }
  return in ? j : lane;
}

// One warp shuffle over the 32 registers `reg` of one warp into `res`.
void warp_shfl(int fn, const uint32_t* reg, uint32_t* res, int b, int W) {
  if (g_fuse_phases) {  // planted mistake: read while other lanes still write
    for (int tx = 0; tx < 32; ++tx) {
      warp_xchg[tx] = reg[tx];
      res[tx] = warp_xchg[shfl_src_lane(fn, tx, b, W)];
    }
    return;
  }
  for (int tx = 0; tx < 32; ++tx) warp_xchg[tx] = reg[tx];  // write phase
  // -- implicit warp barrier (RAW) --
  for (int tx = 0; tx < 32; ++tx) res[tx] = warp_xchg[shfl_src_lane(fn, tx, b, W)];
  // -- implicit warp barrier (WAR) --
}

// Vote over tiles of width W: each lane gets its tile's ballot as a tile-local
// mask (bit r <-> lane seg+r), the cooperative-groups form of __ballot_sync.
void warp_ballot(const bool* pred, uint32_t* res, int W) {
  auto read = [&](int tx) {
    const int seg = tx & ~(W - 1);
    uint32_t m = 0;
    for (int r = 0; r < W; ++r)
      if (warp_xchg[seg + r]) m |= 1u << r;
    return m;
  };
  if (g_fuse_phases) {  // planted mistake: no barrier between write and read
    for (int tx = 0; tx < 32; ++tx) {
      warp_xchg[tx] = pred[tx] ? 1u : 0u;
      res[tx] = read(tx);
    }
    return;
  }
  for (int tx = 0; tx < 32; ++tx) warp_xchg[tx] = pred[tx] ? 1u : 0u;  // write phase
  // -- warp barrier (RAW) --
  for (int tx = 0; tx < 32; ++tx) res[tx] = read(tx);  // read phase
  // -- warp barrier (WAR) --
}

// match_any over tiles of width W: the tile-local mask of valid lanes whose
// 32-bit value equals the caller's.  Invalid lanes take part in no mask.
thread_local bool warp_xchg_valid[32];
void warp_match_any(const uint32_t* val, const bool* valid, uint32_t* res, int W) {
  for (int tx = 0; tx < 32; ++tx) {  // write phase
    warp_xchg[tx] = val[tx];
    warp_xchg_valid[tx] = valid[tx];
  }
  // -- warp barrier (RAW) --
  for (int tx = 0; tx < 32; ++tx) {  // read phase
    const int seg = tx & ~(W - 1);
    uint32_t m = 0;
    if (warp_xchg_valid[tx])
      for (int r = 0; r < W; ++r)
        if (warp_xchg_valid[seg + r] && warp_xchg[seg + r] == warp_xchg[tx]) m |= 1u << r;
    res[tx] = m;
  }
  // -- warp barrier (WAR) --
}

// ----------------------------------------------------------- arithmetic
uint32_t identity_bits(int op, int dt) {
  switch (op) {
    case OP_SUM: case OP_OR: case OP_XOR: return 0u;  // 0.0f has bits 0
    case OP_AND: return 0xFFFFFFFFu;
    case OP_MIN:
      return dt == DT_I32 ? 0x7FFFFFFFu : dt == DT_U32 ? 0xFFFFFFFFu : as_u(INFINITY);
    default:  // OP_MAX
      return dt == DT_I32 ? 0x80000000u : dt == DT_U32 ? 0u : as_u(-INFINITY);
  }
}

// a op b in the element type; int sums wrap mod 2^32 (two's complement).
uint32_t combine(int op, int dt, uint32_t a, uint32_t b) {
  if (dt == DT_F32) {
    const float x = as_f(a), y = as_f(b);
    switch (op) {
      case OP_SUM: return as_u(x + y);
      case OP_MIN: return as_u(std::fmin(x, y));
      default: return as_u(std::fmax(x, y));
    }
  }
  switch (op) {
    case OP_SUM: return a + b;
    case OP_AND: return a & b;
    case OP_OR: return a | b;
    case OP_XOR: return a ^ b;
    case OP_MIN:
      return dt == DT_I32 ? (uint32_t)std::min((int32_t)a, (int32_t)b) : std::min(a, b);
    default:
      return dt == DT_I32 ? (uint32_t)std::max((int32_t)a, (int32_t)b) : std::max(a, b);
  }
}

bool op_valid(int op, int dt) {
  if (dt != DT_I32 && dt != DT_U32 && dt != DT_F32) return false;
  if (op < OP_SUM || op > OP_XOR) return false;
  return dt != DT_F32 || op <= OP_MAX;
}

// Knuth's TwoSum (TAOCP vol. 2, 4.2.2; Ogita, Rump & Oishi 2005, Alg. 3.1):
// s = fl(a + b) and t with a + b = s + t exactly, for any order of |a|, |b|.
inline void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bp = s - a;
  const float ap = s - bp;
  t = (a - ap) + (b - bp);
}

// Compensated pair (s, e): a value s with a running error term e.
// (s1,e1) (+) (s2,e2) = (s, (e1 + e2) + t) with (s, t) = TwoSum(s1, s2).
struct Pair { float s, e; };
inline Pair pair_add(Pair a, Pair b) {
  Pair r;
  float t;
  two_sum(a.s, b.s, r.s, t);
  r.e = (a.e + b.e) + t;
  return r;
}

// Neumaier's improved Kahan summation (1974) in FP64 over fp32 inputs.
struct Neumaier {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// ================================================================ kernels
// Each kernel below is written in collapsed form: per block, an inter-warp
// loop (wid) around intra-warp loops (tx), registers as per-lane arrays.

// cox_shfl: element i is the operand of global thread i.
void shfl_block(int64_t blk, int fn, int dt, int W, int B, const uint32_t* in,
                uint32_t* out, int64_t n, int param) {
  std::vector<uint32_t> v(B), r(B);  // replicated registers (Section 3.6)
  bool pred[32], valid[32];
  for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop
    uint32_t* vw = &v[wid * 32];
    uint32_t* rw = &r[wid * 32];
    const int64_t base = blk * B + wid * 32;
    for (int tx = 0; tx < 32; ++tx) {  // intra-warp loop: load
      const int64_t i = base + tx;
      valid[tx] = i < n;
      vw[tx] = valid[tx] ? in[i] : 0u;
      pred[tx] = valid[tx] && (dt == DT_F32 ? as_f(vw[tx]) != 0.0f : vw[tx] != 0u);
    }
    switch (fn) {
      case FN_SHFL_IDX: case FN_SHFL_UP: case FN_SHFL_DOWN: case FN_SHFL_XOR:
        warp_shfl(fn, vw, rw, param, W);
        break;
      case FN_BALLOT: warp_ballot(pred, rw, W); break;
      case FN_ANY: case FN_ALL: {
        warp_ballot(pred, rw, W);
        const uint32_t full = W == 32 ? 0xFFFFFFFFu : ((1u << W) - 1u);
        for (int tx = 0; tx < 32; ++tx)
          rw[tx] = fn == FN_ANY ? (rw[tx] != 0u) : (rw[tx] == full);
        break;
      }
      default: warp_match_any(vw, valid, rw, W); break;
    }
    for (int tx = 0; tx < 32; ++tx)  // intra-warp loop: store
      if (base + tx < n) out[base + tx] = rw[tx];
  }
}

// Tile tree of the reduction kernels (Code 1 generalised to width W):
// for offset = W/2 .. 1: v += shfl_down(v, offset); the tile's lane 0 ends with
// the tile's value.  Plain form on bit patterns.
void tile_tree_plain(int op, int dt, uint32_t* vw, int W) {
  uint32_t sh[32];
  for (int off = W / 2; off > 0; off /= 2) {
    warp_shfl(FN_SHFL_DOWN, vw, sh, off, W);
    for (int tx = 0; tx < 32; ++tx) vw[tx] = combine(op, dt, vw[tx], sh[tx]);
  }
}

// Same tree on compensated pairs: both words of the pair are shuffled.
void tile_tree_pair(float* s, float* e, int W) {
  uint32_t bs[32], be[32], rs[32], re[32];
  for (int off = W / 2; off > 0; off /= 2) {
    for (int tx = 0; tx < 32; ++tx) { bs[tx] = as_u(s[tx]); be[tx] = as_u(e[tx]); }
    warp_shfl(FN_SHFL_DOWN, bs, rs, off, W);
    warp_shfl(FN_SHFL_DOWN, be, re, off, W);
    for (int tx = 0; tx < 32; ++tx) {
      const Pair p = pair_add({s[tx], e[tx]}, {as_f(rs[tx]), as_f(re[tx])});
      s[tx] = p.s;
      e[tx] = p.e;
    }
  }
}

// Optional instrumentation for the Appendix A invariant (each lane runs each
// non-peeled statement once per dynamic instance).  Counters are indexed
// [statement][global thread].
struct Counters {
  std::vector<int32_t>* c = nullptr;
  int64_t threads = 0;
  void hit(int stmt, int64_t thread) {
    if (c) (*c)[stmt * threads + thread] += 1;
  }
};

// Reduction of one block (TILE and BLOCK scope), in the order the kernels use:
//  1. every thread loads its element (identity for padding lanes);
//  2. tile tree at width W (tile leader = tile lane 0);
//  3. block barrier; tile leaders' values are the partials p[0..B/W);
//  4. warp 0 only (peeled on lane 0's flag): lane l folds p[l], p[l+32], ...
//     into an accumulator that starts at the identity, then a width-32 tree;
//     lane 0 holds the block's value.
// `out_tile` gets every tile's value (TILE scope), `out_block` the block's
// value (BLOCK scope); either may be null.
void reduce_block(int64_t blk, int op, int dt, int W, int B, bool comp,
                  const uint32_t* in, int64_t n, uint32_t* out_tile,
                  float* lo_tile, uint32_t* out_block, float* lo_block,
                  Counters cnt) {
  const int P = B / W;
  std::vector<uint32_t> v(B);            // plain registers
  std::vector<float> s(B), e(B);         // compensated registers
  std::vector<uint32_t> part(P);         // shared memory: tile partials
  std::vector<float> part_s(P), part_e(P);
  const uint32_t ident = identity_bits(op, dt);
  const int64_t ntiles = (n + W - 1) / W;

  for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop (first block PR)
    const int64_t base = blk * B + wid * 32;
    for (int tx = 0; tx < 32; ++tx) {  // S0: load
      const int64_t i = base + tx;
      const uint32_t x = i < n ? in[i] : ident;
      v[wid * 32 + tx] = x;
      s[wid * 32 + tx] = as_f(x);
      e[wid * 32 + tx] = 0.0f;
      cnt.hit(0, base + tx);
    }
    for (int off = W / 2; off > 0; off /= 2)  // S1: tree steps (instrumentation only)
      for (int tx = 0; tx < 32; ++tx) cnt.hit(1, base + tx);
    if (comp) tile_tree_pair(&s[wid * 32], &e[wid * 32], W);
    else tile_tree_plain(op, dt, &v[wid * 32], W);
    for (int tx = 0; tx < 32; tx += W) {  // tile leaders publish their partial
      const int k = (wid * 32 + tx) / W;
      part[k] = v[wid * 32 + tx];
      part_s[k] = s[wid * 32 + tx];
      part_e[k] = e[wid * 32 + tx];
      const int64_t t = (blk * B + wid * 32 + tx) / W;
      if (out_tile && t < ntiles) {
        if (comp) {
          float y, lo;
          two_sum(part_s[k], part_e[k], y, lo);
          out_tile[t] = as_u(y);
          if (lo_tile) lo_tile[t] = lo;
        } else {
          out_tile[t] = part[k];
        }
      }
    }
  }
  // -- block barrier --
  if (!out_block) return;
  for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop (second block PR)
    bool flag[32];
    for (int tx = 0; tx < 32; ++tx) flag[tx] = wid == 0;
    if (!flag[0]) continue;  // loop peeling: lane 0 decides for the warp
    uint32_t a[32];
    float as[32], ae[32];
    for (int tx = 0; tx < 32; ++tx) {
      cnt.hit(2, blk * B + wid * 32 + tx);
      a[tx] = ident;
      as[tx] = 0.0f;
      ae[tx] = 0.0f;
      for (int k = tx; k < P; k += 32) {
        a[tx] = combine(op, dt, a[tx], part[k]);
        const Pair p = pair_add({as[tx], ae[tx]}, {part_s[k], part_e[k]});
        as[tx] = p.s;
        ae[tx] = p.e;
      }
    }
    if (comp) tile_tree_pair(as, ae, 32);
    else tile_tree_plain(op, dt, a, 32);
    if (comp) {
      float y, lo;
      two_sum(as[0], ae[0], y, lo);
      out_block[blk] = as_u(y);
      if (lo_block) lo_block[blk] = lo;
    } else {
      out_block[blk] = a[0];
    }
  }
}

// Tile inclusive scan of one block, Hillis-Steele on shfl_up at width W:
// for d = 1, 2, .., W/2: u = shfl_up(x, d); if (rank >= d) x = u op x.
void scan_block(int64_t blk, int op, int dt, int W, int B, bool comp,
                const uint32_t* in, int64_t n, uint32_t* out) {
  const uint32_t ident = identity_bits(op, dt);
  uint32_t x[32], u[32], bs[32], be[32], us[32], ue[32];
  float s[32], e[32];
  for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop
    const int64_t base = blk * B + wid * 32;
    for (int tx = 0; tx < 32; ++tx) {
      const int64_t i = base + tx;
      x[tx] = i < n ? in[i] : ident;
      s[tx] = as_f(x[tx]);
      e[tx] = 0.0f;
    }
    for (int d = 1; d < W; d *= 2) {
      if (comp) {
        for (int tx = 0; tx < 32; ++tx) { bs[tx] = as_u(s[tx]); be[tx] = as_u(e[tx]); }
        warp_shfl(FN_SHFL_UP, bs, us, d, W);
        warp_shfl(FN_SHFL_UP, be, ue, d, W);
        for (int tx = 0; tx < 32; ++tx)
          if ((tx & (W - 1)) >= d) {
            const Pair p = pair_add({as_f(us[tx]), as_f(ue[tx])}, {s[tx], e[tx]});
            s[tx] = p.s;
            e[tx] = p.e;
          }
      } else {
        warp_shfl(FN_SHFL_UP, x, u, d, W);
        for (int tx = 0; tx < 32; ++tx)
          if ((tx & (W - 1)) >= d) x[tx] = combine(op, dt, u[tx], x[tx]);
      }
    }
    for (int tx = 0; tx < 32; ++tx)
      if (base + tx < n) out[base + tx] = comp ? as_u(s[tx] + e[tx]) : x[tx];
  }
}

// ------------------------------------------ coalesced groups (dynamic masks)
// The dynamic group of Section 2.2.2 (coalesced_threads(): every active
// thread of the warp at the call) and the runtime member masks of Section
// 2.2.3, which COX leaves unsupported.  A lane is active when its element
// exists (gi < n) and active[gi] != 0; the group is the warp's active lanes
// in lane order, rank = number of active lanes below, size = their count.
// Write phase: every active lane puts its operand into the exchange array;
// read phase: every active lane takes its result from it by group rank.
// Inactive lanes take no part and get no result.
enum CgFn {
  CG_SIZE = 0, CG_RANK = 1, CG_SHFL = 2, CG_SHFL_UP = 3, CG_SHFL_DOWN = 4,
  CG_BALLOT = 5, CG_ANY = 6, CG_ALL = 7, CG_REDUCE_SUM = 8, CG_SCAN_SUM = 9
};

// Vote predicate of a 32-bit operand: nonzero (fp32: != 0.0f, reading R17).
bool pred_of(int dt, uint32_t u) { return dt == DT_F32 ? as_f(u) != 0.0f : u != 0u; }

void coalesced_block(int64_t blk, int fn, int dt, int B, const uint32_t* in, const int32_t* active,
                     uint32_t* out, int64_t n, int param) {
  for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop
    const int64_t base = blk * B + (int64_t)wid * 32;
    bool act[32];
    int member[32];  // member[k] = lane of group rank k
    int rank[32];
    int size = 0;
    for (int tx = 0; tx < 32; ++tx) {  // intra-warp loop: who is active
      act[tx] = base + tx < n && active[base + tx] != 0;
      rank[tx] = size;
      if (act[tx]) member[size++] = tx;
    }
    if (size == 0) continue;
    for (int tx = 0; tx < 32; ++tx)  // write phase
      if (act[tx]) warp_xchg[tx] = in[base + tx];
    for (int tx = 0; tx < 32; ++tx) {  // read phase
      if (!act[tx]) continue;
      const int r = rank[tx];
      uint32_t res = 0;
      switch (fn) {
        case CG_SIZE: res = (uint32_t)size; break;
        case CG_RANK: res = (uint32_t)r; break;
        case CG_SHFL: res = warp_xchg[member[param % size]]; break;
        case CG_SHFL_UP: res = r >= param ? warp_xchg[member[r - param]] : warp_xchg[tx]; break;
        case CG_SHFL_DOWN: res = r + param < size ? warp_xchg[member[r + param]] : warp_xchg[tx]; break;
        case CG_BALLOT:
          for (int k = 0; k < size; ++k)
            if (pred_of(dt, warp_xchg[member[k]])) res |= 1u << k;
          break;
        case CG_ANY:
          for (int k = 0; k < size; ++k) res |= pred_of(dt, warp_xchg[member[k]]) ? 1u : 0u;
          break;
        case CG_ALL:
          res = 1u;
          for (int k = 0; k < size; ++k) res &= pred_of(dt, warp_xchg[member[k]]) ? 1u : 0u;
          break;
        case CG_REDUCE_SUM:
          for (int k = 0; k < size; ++k) res += warp_xchg[member[k]];
          break;
        default:  // CG_SCAN_SUM: inclusive prefix over ranks 0..r
          for (int k = 0; k <= r; ++k) res += warp_xchg[member[k]];
          break;
      }
      out[base + tx] = res;
    }
  }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

// Coalesced-group warp functions (see coalesced_block).  SHFL takes the
// source rank param mod size; SHFL_UP/DOWN keep the caller's value when the
// source rank is outside the group; BALLOT is group-local (bit k = rank k's
// predicate); REDUCE/SCAN_SUM are integer sums mod 2^32 (I32/U32 only).
int oracle_coalesced(int fn, int dt, int B, const uint32_t* in, const int32_t* active, uint32_t* out, int64_t n,
                     int param) {
  if (!valid_block(B) || n < 0 || fn < CG_SIZE || fn > CG_SCAN_SUM) return ST_EINVAL;
  if (dt < DT_I32 || dt > DT_F32) return ST_EINVAL;
  if ((fn == CG_REDUCE_SUM || fn == CG_SCAN_SUM) && dt == DT_F32) return ST_EINVAL;
  if ((fn == CG_SHFL || fn == CG_SHFL_UP || fn == CG_SHFL_DOWN) && (param < 0 || param > 31)) return ST_EINVAL;
  if (n == 0) return ST_OK;
  launch_grid((n + B - 1) / B, [&](int64_t b) { coalesced_block(b, fn, dt, B, in, active, out, n, param); });
  return ST_OK;
}

void oracle_set_threads(int k) { g_threads = k; }
int oracle_threads(void) { return pool_threads(); }
void oracle_debug_fuse_phases(int on) { g_fuse_phases = on != 0; }

// cox_shfl semantics (Section 2.2.1; Code 1, Code 4): out[i] is global thread
// i's result.  Shuffles return the source lane's 32-bit pattern (0 when the
// source lane is a padding lane); BALLOT and MATCH_ANY return tile-local masks;
// ANY/ALL return 0/1.
int oracle_shfl(int fn, int dt, int W, int B, const uint32_t* in, uint32_t* out,
                int64_t n, int param) {
  if (!pow2_width(W) || !valid_block(B) || n < 0) return ST_EINVAL;
  if (fn < FN_SHFL_IDX || fn > FN_MATCH_ANY) return ST_EINVAL;
  if (dt < DT_I32 || dt > DT_F32) return ST_EINVAL;
  if ((fn == FN_SHFL_UP || fn == FN_SHFL_DOWN || fn == FN_SHFL_XOR) && (param < 0 || param > 31))
    return ST_EINVAL;
  if (n == 0) return ST_OK;
  launch_grid((n + B - 1) / B, [&](int64_t b) { shfl_block(b, fn, dt, W, B, in, out, n, param); });
  return ST_OK;
}

// Code 1 of the paper on one block of B threads: val = 1; if (tid < 32) for
// offset = 16..1: val += shfl_down(val, offset).  mode 0 uses the CUDA/PTX
// rule (an out-of-range source returns the caller's value); mode 1 follows the
// CPU translation of Code 3, which skips the add when tx + offset >= 32.
int oracle_code1(int B, int mode, int32_t* out) {
  if (!valid_block(B)) return ST_EINVAL;
  std::vector<uint32_t> val(B);
  for (int wid = 0; wid < B / 32; ++wid) {
    for (int tx = 0; tx < 32; ++tx) val[wid * 32 + tx] = 1;
    bool flag[32];
    for (int tx = 0; tx < 32; ++tx) flag[tx] = (wid * 32 + tx) < 32;
    if (flag[0]) {  // loop peeling
      for (int offset = 16; offset > 0; offset /= 2) {
        uint32_t sh[32];
        uint32_t* vw = &val[wid * 32];
        if (mode == 0) {
          warp_shfl(FN_SHFL_DOWN, vw, sh, offset, 32);
          for (int tx = 0; tx < 32; ++tx) vw[tx] += sh[tx];
        } else {
          for (int tx = 0; tx < 32; ++tx) warp_xchg[tx] = vw[tx];
          for (int tx = 0; tx < 32; ++tx)
            if (tx + offset < 32) vw[tx] += warp_xchg[tx + offset];
        }
      }
    }
  }
  for (int t = 0; t < B; ++t) out[t] = (int32_t)val[t];
  return ST_OK;
}

// Code 4 of the paper: result[tx] = __all_sync(-1, tx % 2) for one block.
int oracle_code4(int B, int32_t* out) {
  if (!valid_block(B)) return ST_EINVAL;
  for (int wid = 0; wid < B / 32; ++wid) {
    bool pred[32];
    uint32_t r[32];
    for (int tx = 0; tx < 32; ++tx) pred[tx] = ((wid * 32 + tx) % 2) != 0;
    warp_ballot(pred, r, 32);
    for (int tx = 0; tx < 32; ++tx) out[wid * 32 + tx] = r[tx] == 0xFFFFFFFFu;
  }
  return ST_OK;
}

// Two consecutive votes through the one exchange array (Section 3.2, Code 5):
// first all(tx % 2), then all(1).  out[2*t] and out[2*t+1] are thread t's two
// results.
int oracle_vote_pair(int B, int32_t* out) {
  if (!valid_block(B)) return ST_EINVAL;
  for (int wid = 0; wid < B / 32; ++wid) {
    bool p1[32], p2[32];
    uint32_t r1[32], r2[32];
    for (int tx = 0; tx < 32; ++tx) { p1[tx] = tx % 2; p2[tx] = true; }
    warp_ballot(p1, r1, 32);
    warp_ballot(p2, r2, 32);
    for (int tx = 0; tx < 32; ++tx) {
      out[2 * (wid * 32 + tx)] = r1[tx] == 0xFFFFFFFFu;
      out[2 * (wid * 32 + tx) + 1] = r2[tx] == 0xFFFFFFFFu;
    }
  }
  return ST_OK;
}

// Reduction emulation, TILE or BLOCK scope, in the kernels' association order
// (see reduce_block).  out: ceil(n/W) (TILE) or ceil(n/B) (BLOCK) elements.
// lo (optional, compensated fp32 only): the low word, so out + lo equals the
// final compensated pair's s + e exactly.
int oracle_reduce_emulate(int op, int dt, int W, int B, int scope, int comp,
                          const uint32_t* in, uint32_t* out, float* lo, int64_t n) {
  if (!pow2_width(W) || !valid_block(B) || n < 0 || !op_valid(op, dt)) return ST_EINVAL;
  if (scope != SC_TILE && scope != SC_BLOCK) return ST_EINVAL;
  if (comp && (dt != DT_F32 || op != OP_SUM)) return ST_EINVAL;
  if (n == 0) return ST_OK;
  launch_grid((n + B - 1) / B, [&](int64_t b) {
    reduce_block(b, op, dt, W, B, comp != 0, in, n, scope == SC_TILE ? out : nullptr,
                 scope == SC_TILE ? lo : nullptr, scope == SC_BLOCK ? out : nullptr,
                 scope == SC_BLOCK ? lo : nullptr, Counters{});
  });
  return ST_OK;
}

// Appendix A instrumentation: runs the BLOCK-scope int32 sum reduction and
// counts, per global thread, how often each statement ran: [0] the load,
// [1] the tree-step add (log2 W per lane), [2] the warp-0 combine (peeled:
// warp 0's lanes only).  counts has 3 * grid * B entries.
int oracle_reduce_counts(int W, int B, int64_t n, int32_t* counts) {
  if (!pow2_width(W) || !valid_block(B) || n <= 0) return ST_EINVAL;
  const int64_t grid = (n + B - 1) / B;
  std::vector<int32_t> c(3 * grid * B, 0);
  std::vector<uint32_t> in(n, 1u), out(grid);
  Counters cnt{&c, grid * B};
  for (int64_t b = 0; b < grid; ++b)
    reduce_block(b, OP_SUM, DT_I32, W, B, false, in.data(), n, nullptr, nullptr,
                 out.data(), nullptr, cnt);
  std::memcpy(counts, c.data(), c.size() * sizeof(int32_t));
  return ST_OK;
}

// Definition of the reduction (what the emulation must equal up to rounding):
// segments of L consecutive elements (L = W for TILE, B for BLOCK, n for
// GRID).  Integer ops: exact, wrapping.  fp32 sum: FP64 Neumaier value in
// ref64, and sum |x| in abs64 (fp32 min/max: exact value in ref64).  out_bits
// receives integer results (and fp32 min/max bits); may be null for fp32 sum.
int oracle_reduce_ref(int op, int dt, int64_t L, const uint32_t* in, int64_t n,
                      uint32_t* out_bits, double* ref64, double* abs64) {
  if (L <= 0 || n < 0 || !op_valid(op, dt)) return ST_EINVAL;
  if (n == 0) return ST_OK;
  const int64_t nseg = (n + L - 1) / L;
  const int64_t chunk = std::max<int64_t>(1, (1 << 16) / L);
  launch_grid((nseg + chunk - 1) / chunk, [&](int64_t c) {
    for (int64_t g = c * chunk; g < std::min(nseg, (c + 1) * chunk); ++g) {
      const int64_t lo = g * L, hi = std::min(n, lo + L);
      if (dt == DT_F32 && op == OP_SUM) {
        Neumaier acc;
        double a = 0.0;
        for (int64_t i = lo; i < hi; ++i) {
          acc.add((double)as_f(in[i]));
          a += std::fabs((double)as_f(in[i]));
        }
        if (ref64) ref64[g] = acc.value();
        if (abs64) abs64[g] = a;
        if (out_bits) out_bits[g] = as_u((float)acc.value());
      } else {
        uint32_t r = identity_bits(op, dt);
        for (int64_t i = lo; i < hi; ++i) r = combine(op, dt, r, in[i]);
        if (out_bits) out_bits[g] = r;
        if (ref64) ref64[g] = dt == DT_F32 ? (double)as_f(r) : dt == DT_I32 ? (double)(int32_t)r : (double)r;
        if (abs64) abs64[g] = 0.0;
      }
    }
  });
  return ST_OK;
}

// Tile inclusive scan emulation (Hillis-Steele on shfl_up at width W, plain or
// compensated, output fl(s + e) for compensated).
int oracle_scan_emulate(int op, int dt, int W, int B, int comp, const uint32_t* in,
                        uint32_t* out, int64_t n) {
  if (!pow2_width(W) || !valid_block(B) || n < 0 || !op_valid(op, dt)) return ST_EINVAL;
  if (comp && (dt != DT_F32 || op != OP_SUM)) return ST_EINVAL;
  if (n == 0) return ST_OK;
  launch_grid((n + B - 1) / B, [&](int64_t b) { scan_block(b, op, dt, W, B, comp != 0, in, n, out); });
  return ST_OK;
}

// Definition of the tile inclusive scan: within each segment of W consecutive
// elements, out[i] = x[seg] op ... op x[i].  Integer: exact bits.  fp32 sum:
// FP64 Neumaier prefix in ref64 and prefix of |x| in abs64.
int oracle_scan_ref(int op, int dt, int W, const uint32_t* in, int64_t n,
                    uint32_t* out_bits, double* ref64, double* abs64) {
  if (W <= 0 || n < 0 || !op_valid(op, dt)) return ST_EINVAL;
  if (n == 0) return ST_OK;
  const int64_t nseg = (n + W - 1) / W;
  const int64_t chunk = std::max<int64_t>(1, (1 << 16) / W);
  launch_grid((nseg + chunk - 1) / chunk, [&](int64_t c) {
    for (int64_t g = c * chunk; g < std::min(nseg, (c + 1) * chunk); ++g) {
      const int64_t lo = g * W, hi = std::min(n, lo + W);
      Neumaier acc;
      double a = 0.0;
      uint32_t r = identity_bits(op, dt);
      for (int64_t i = lo; i < hi; ++i) {
        if (dt == DT_F32 && op == OP_SUM) {
          acc.add((double)as_f(in[i]));
          a += std::fabs((double)as_f(in[i]));
          if (ref64) ref64[i] = acc.value();
          if (abs64) abs64[i] = a;
          if (out_bits) out_bits[i] = as_u((float)acc.value());
        } else {
          r = combine(op, dt, r, in[i]);
          if (out_bits) out_bits[i] = r;
          if (ref64) ref64[i] = dt == DT_F32 ? (double)as_f(r) : dt == DT_I32 ? (double)(int32_t)r : (double)r;
          if (abs64) abs64[i] = 0.0;
        }
      }
    }
  });
  return ST_OK;
}

// Ballot-driven stream compaction (filter_arr of Table 1 with a static,
// full-tile group; ballot of Section 2.2.1): keep keys with key < t, in input
// order.  Per block, per warp, per tile of width W:
//   b = ballot(pred); rank = popc(b & lanes-below); cnt = popc(b);
// the block scans its tile counts in tile order; blocks then take offsets from
// an exclusive scan of block counts in block order (the value the GPU's
// single-pass look-back computes); every kept key goes to
// out[block offset + tile offset + rank].  dt: 0 = int32 keys (signed
// compare), 1 = uint32 keys (unsigned compare).
int oracle_ballot_compact(int dt, int W, int B, const uint32_t* keys, int64_t n,
                          int64_t t, uint32_t* out, int64_t* count) {
  if (!pow2_width(W) || !valid_block(B) || n < 0 || (dt != DT_I32 && dt != DT_U32)) return ST_EINVAL;
  const int64_t grid = (n + B - 1) / B;
  const int P = B / W;
  auto keep = [&](uint32_t k) {
    return dt == DT_I32 ? (int64_t)(int32_t)k < t : (int64_t)k < t;
  };
  std::vector<int64_t> block_cnt(grid);
  // pass 1: every block's count (per-tile ballots)
  auto block_pass = [&](int64_t blk, int64_t offset, bool scatter) {
    bool pred[32];
    uint32_t bal[32];
    std::vector<int32_t> tile_cnt(P), tile_off(P);
    std::vector<int32_t> rank(B);
    for (int wid = 0; wid < B / 32; ++wid) {  // inter-warp loop
      const int64_t base = blk * B + wid * 32;
      for (int tx = 0; tx < 32; ++tx) pred[tx] = base + tx < n && keep(keys[base + tx]);
      warp_ballot(pred, bal, W);
      for (int tx = 0; tx < 32; ++tx) {
        const int r = tx & (W - 1);
        const uint32_t below = r == 0 ? 0u : (bal[tx] & ((1u << r) - 1u));
        rank[wid * 32 + tx] = __builtin_popcount(below);
        if (r == 0) tile_cnt[(wid * 32 + tx) / W] = __builtin_popcount(bal[tx]);
      }
    }
    // -- block barrier -- exclusive scan of tile counts in tile order
    int32_t acc = 0;
    for (int k = 0; k < P; ++k) { tile_off[k] = acc; acc += tile_cnt[k]; }
    if (!scatter) { block_cnt[blk] = acc; return; }
    for (int wid = 0; wid < B / 32; ++wid) {
      const int64_t base = blk * B + wid * 32;
      for (int tx = 0; tx < 32; ++tx) {
        const int64_t i = base + tx;
        if (i < n && keep(keys[i]))
          out[offset + tile_off[(wid * 32 + tx) / W] + rank[wid * 32 + tx]] = keys[i];
      }
    }
  };
  launch_grid(grid, [&](int64_t b) { block_pass(b, 0, false); });
  std::vector<int64_t> block_off(grid);
  int64_t total = 0;
  for (int64_t b = 0; b < grid; ++b) { block_off[b] = total; total += block_cnt[b]; }
  launch_grid(grid, [&](int64_t b) { block_pass(b, block_off[b], true); });
  *count = total;
  return ST_OK;
}

// Match-based histogram: per tile of width W, peers = match_any(key) among
// valid lanes; the lowest lane of each peer group (its leader) adds
// popc(peers) to the block's shared histogram bin `key`, or to the ignored
// count when key is outside [0, bins); after a block barrier the block merges
// its histogram into hist.  hist has `bins` int32 entries (overwritten).
int oracle_match_histogram(int W, int B, const int32_t* keys, int64_t n, int bins,
                           int32_t* hist, int64_t* ignored) {
  if (!pow2_width(W) || !valid_block(B) || n < 0 || bins <= 0) return ST_EINVAL;
  const int64_t grid = (n + B - 1) / B;
  std::mutex mu;
  std::vector<int64_t> total(bins, 0);
  int64_t ign_total = 0;
  const int64_t per_task = 64;  // blocks per pool task
  launch_grid((grid + per_task - 1) / per_task, [&](int64_t task) {
    std::vector<int64_t> local(bins, 0);
    int64_t ign = 0;
    for (int64_t blk = task * per_task; blk < std::min(grid, (task + 1) * per_task); ++blk) {
      std::vector<int32_t> smem(bins, 0);  // block's shared histogram
      int32_t smem_ign = 0;
      for (int wid = 0; wid < B / 32; ++wid) {
        const int64_t base = blk * B + wid * 32;
        uint32_t v[32], peers[32];
        bool valid[32];
        for (int tx = 0; tx < 32; ++tx) {
          valid[tx] = base + tx < n;
          v[tx] = valid[tx] ? (uint32_t)keys[base + tx] : 0u;
        }
        warp_match_any(v, valid, peers, W);
        for (int tx = 0; tx < 32; ++tx) {
          if (!valid[tx]) continue;
          const int r = tx & (W - 1);
          const bool leader = (peers[tx] & ((1u << r) - 1u)) == 0u;  // lowest peer
          if (!leader) continue;
          const int32_t k = (int32_t)v[tx];
          if (k >= 0 && k < bins) smem[k] += __builtin_popcount(peers[tx]);
          else smem_ign += __builtin_popcount(peers[tx]);
        }
      }
      // -- block barrier -- merge
      for (int k = 0; k < bins; ++k) local[k] += smem[k];
      ign += smem_ign;
    }
    std::lock_guard<std::mutex> g(mu);
    for (int k = 0; k < bins; ++k) total[k] += local[k];
    ign_total += ign;
  });
  for (int k = 0; k < bins; ++k) hist[k] = (int32_t)total[k];
  if (ignored) *ignored = ign_total;
  return ST_OK;
}

// Batched reference: for each array a (offsets[a] .. offsets[a+1] into the
// concatenated vals / keys), the FP64 Neumaier sum of its fp32 values, the sum
// of |x|, and its `bins`-bin key histogram (keys outside [0,bins) ignored).
int oracle_batch_ref(int64_t num_arrays, const int64_t* offsets, const float* vals,
                     const int32_t* keys, int bins, double* sums64, double* abs64,
                     int32_t* hists) {
  if (num_arrays < 0 || bins <= 0) return ST_EINVAL;
  launch_grid(num_arrays, [&](int64_t a) {
    Neumaier acc;
    double ab = 0.0;
    int32_t* h = hists ? hists + a * bins : nullptr;
    if (h) std::fill(h, h + bins, 0);
    for (int64_t i = offsets[a]; i < offsets[a + 1]; ++i) {
      acc.add((double)vals[i]);
      ab += std::fabs((double)vals[i]);
      if (h && keys[i] >= 0 && keys[i] < bins) h[keys[i]] += 1;
    }
    if (sums64) sums64[a] = acc.value();
    if (abs64) abs64[a] = ab;
  });
  return ST_OK;
}

}  // extern "C"
