/*
 * cox.h -- C ABI of the GB300 warp-collective library (libcox.so).
 *
 * The library runs CUDA warp-level functions -- shuffles, votes, match_any and
 * cooperative-groups tiles of width 2..32 -- across whole grids, and the
 * compositions built from them: tile and block reductions, tile inclusive
 * scans, ballot-driven stable compaction and match-based histograms.  The
 * paper (arXiv 2112.10034, COX) defines these functions' semantics by running
 * CUDA kernels that use them on CPUs (Section 2.2.1 "Warp-level collectives",
 * Section 3.2 "Support warp-level functions"); this library runs them on the
 * GPU as hand-written sm_103a kernels.
 *
 * Conventions for every call below:
 *   - d_* pointers are DEVICE pointers owned by the caller; the library keeps
 *     no reference to them after the call returns.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL means
 *     the legacy default stream).  Errors found on the host (bad arguments, a
 *     failed launch) are returned at once and nothing is enqueued.  Errors
 *     found on the device (a bounded wait that ran out) are recorded in a
 *     device-side status word that cox_device_status() reads.
 *   - The element of index i is the operand of global thread i: lane i % 32
 *     of its warp and rank i % width of its width-`width` tile (Code 3's lane
 *     numbering, Section 2.3).  `width` must be 2, 4, 8, 16 or 32.
 *     `block_dim` (threads per block) must be a multiple of 32 in [32, 1024];
 *     it defines the BLOCK scope and is otherwise a launch choice.
 *   - Only full-tile masks are supported: the paper's translator covers
 *     warp functions without divergence only (Section 2.2.3); a call whose
 *     `mask` is not the full mask returns COX_EUNSUPPORTED.
 *   - Ragged tails: lanes whose index is >= n take part as padding -- the
 *     identity of the op, a false predicate, no histogram contribution -- and
 *     nothing is written at an output index that has no input.
 *   - Integer arithmetic wraps modulo 2^32.  fp32 sums round to nearest; the
 *     COMPENSATED flag carries a TwoSum error term next to every partial sum.
 *   - No call allocates device or host memory, and no call synchronises the
 *     stream, except cox_device_status().
 */
#ifndef COX_H_
#define COX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  COX_OK = 0,
  COX_EINVAL = 1,        /* bad argument: null pointer, bad width/block_dim/op/dtype, n < 0 */
  COX_EUNSUPPORTED = 2,  /* valid request outside the supported scope (partial masks, ...) */
  COX_ECUDA = 3,         /* a CUDA runtime call or launch failed */
  COX_ENOMEM = 4,        /* workspace or budget too small */
  COX_ETIMEOUT = 5,      /* a bounded device-side wait ran out (cox_device_status) */
  COX_EBUSY = 6          /* resource in use (server: no free slot) */
} cox_status;

typedef enum { COX_I32 = 0, COX_U32 = 1, COX_F32 = 2, COX_U8 = 3 /* cox_integral_image input only */ } cox_dtype;

typedef enum { COX_SUM = 0, COX_MIN = 1, COX_MAX = 2, COX_AND = 3, COX_OR = 4, COX_XOR = 5 } cox_op;

typedef enum {
  COX_SHFL_IDX = 0,  /* __shfl_sync(mask, v, srcLane, width) */
  COX_SHFL_UP = 1,   /* __shfl_up_sync(mask, v, delta, width) */
  COX_SHFL_DOWN = 2, /* __shfl_down_sync(mask, v, delta, width) */
  COX_SHFL_XOR = 3,  /* __shfl_xor_sync(mask, v, laneMask, width) */
  COX_BALLOT = 4,    /* tile.ballot(v != 0): tile-local mask */
  COX_ANY = 5,       /* tile.any(v != 0) */
  COX_ALL = 6,       /* tile.all(v != 0) */
  COX_MATCH_ANY = 7  /* tile.match_any(v): tile-local mask of equal lanes */
} cox_warpfn;

typedef enum { COX_SCOPE_TILE = 0, COX_SCOPE_BLOCK = 1, COX_SCOPE_GRID = 2 } cox_scope;

enum {
  COX_F_COMPENSATED = 1u,  /* fp32 sums: TwoSum-compensated pairs through every stage */
  COX_F_FP64_COMBINE = 2u, /* GRID scope fp32 sum: final cross-block combine in FP64 */
  COX_F_WS_READY = 4u,     /* compaction: caller zeroed the workspace; skip the memset */
  COX_F_NATIVE_MATCH = 8u, /* histograms: peer groups from the match.any.sync instruction */
  COX_F_DIRECT_ATOMICS = 16u, /* histograms: no peer groups, one shared atomic per key */
  COX_F_BALLOT_MATCH = 32u    /* histograms: peer groups from ballots over the key bits */
};

/* Human-readable name of a status code (static string, never NULL). */
const char* cox_status_string(cox_status s);

/* Library version: major * 10000 + minor * 100 + patch. */
int cox_version(void);

/*
 * cox_shfl -- one warp function on every lane of a 1-D grid.
 *
 * Section 2.2.1 (warp shuffle, warp vote), Code 1 (shfl_down), Code 4
 * (__all_sync); semantics are PTX shfl.sync / vote.sync / match.sync at
 * segment width `width`.
 *   d_in   n elements of dt (32-bit each).  Votes use the predicate v != 0
 *          (for F32: the value compared with 0.0f); MATCH_ANY compares bits.
 *   d_out  n elements.  Shuffles: dt, the source lane's bits (0 when the
 *          source lane is padding); BALLOT/MATCH_ANY: uint32 tile-local masks
 *          (bit r <-> tile rank r); ANY/ALL: int32 0 or 1.
 *   param  srcLane (IDX; taken modulo width), delta (UP/DOWN, 0..31) or
 *          laneMask (XOR, 0..31; may name lanes of earlier tiles of the same
 *          warp, per PTX); ignored by votes and match.
 *   mask   must be 0xFFFFFFFF (COX_EUNSUPPORTED otherwise).
 */
cox_status cox_shfl(cox_warpfn fn, cox_dtype dt, int width, int block_dim, const void* d_in,
                    void* d_out, int64_t n, int param, uint32_t mask, void* stream);

/*
 * cox_tile_reduce -- reductions over tiles, blocks or the whole grid.
 *
 * Code 1 of the paper (a shfl_down tree into lane 0, Section 2.3) and the SDK
 * reduction kernels of Table 1 (reduce0..reduce6, reduce, reduceFinal).
 *   scope TILE:  d_out[t] = x[t*width] op ... op x[t*width + width - 1],
 *                ceil(n / width) outputs.
 *   scope BLOCK: d_out[b] = reduction of x[b*block_dim .. +block_dim),
 *                ceil(n / block_dim) outputs.  Order: width-`width` shfl_down
 *                tree per tile; tile partials to shared memory; warp 0 lane l
 *                folds partials l, l+32, ... then a width-32 shfl_down tree.
 *   scope GRID:  d_out[0] = reduction of all n elements (0 elements: identity).
 *                Needs d_workspace of cox_tile_reduce_workspace() bytes.
 *   op/dt: SUM/MIN/MAX/AND/OR/XOR for I32 and U32; SUM/MIN/MAX for F32.
 *   flags: COX_F_COMPENSATED (F32 SUM only): TwoSum pairs through the tree
 *          and the combine; the output is fl(s + e).  COX_F_FP64_COMBINE
 *          (GRID, F32 SUM): the final combine of block partials in FP64.
 *   d_err: optional (may be NULL); with COX_F_COMPENSATED, receives for each
 *          output the low word lo such that out + lo == s + e exactly.
 *   d_workspace / workspace_bytes: scratch for GRID scope (ignored otherwise;
 *          may be NULL).  Contents need no initialisation; not shared across
 *          concurrent calls.
 * TILE and BLOCK results are reproducible bit for bit: fp32 values follow the
 * stated order exactly, with no fused operations.
 */
cox_status cox_tile_reduce(cox_op op, cox_dtype dt, int width, int block_dim, cox_scope scope,
                           const void* d_in, void* d_out, int64_t n, unsigned flags, void* d_err,
                           void* d_workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes cox_tile_reduce needs for `scope` (0 for TILE and BLOCK). */
size_t cox_tile_reduce_workspace(cox_scope scope, int64_t n, int block_dim);

/*
 * cox_tile_scan -- inclusive scan within each tile of `width` elements.
 *
 * The shuffle scan of the SDK's shfl_scan_test (Table 1) on a
 * cooperative-groups tile: for d = 1, 2, .., width/2: u = shfl_up(x, d);
 * if (rank >= d) x = u op x (Hillis-Steele).
 *   d_out[i] = x[t0] op x[t0+1] op ... op x[i], t0 = i - i % width.
 *   op/dt: as cox_tile_reduce.  flags: COX_F_COMPENSATED for F32 SUM (pairs
 *   (s, e) shuffled together; output fl(s + e)).
 * Results are reproducible bit for bit (the order above, no fused operations).
 */
cox_status cox_tile_scan(cox_op op, cox_dtype dt, int width, int block_dim, const void* d_in,
                         void* d_out, int64_t n, unsigned flags, void* stream);

/*
 * cox_scan -- inclusive or exclusive scan over each block (BLOCK) or over the
 * whole array (GRID).
 *
 * The step after the tile scan: the SDK's shfl_scan_test scans each block
 * with warp shuffle scans and a scan of the warp totals, and uniform_add adds
 * each block's prefix (Table 1).  BLOCK scope does the first part on blocks
 * of block_dim elements; GRID scope chains tiles (16-byte aligned arrays:
 * 8192 elements by TMA, 16384 for compensated sums; other layouts: 16384,
 * 8192 compensated) with the decoupled look-back of cox_ballot_compact: in a
 * tile every warp scans its rows of 32 elements by shfl_up, carries row
 * totals across its rows, the warp totals are scanned, the tile publishes
 * its aggregate, looks back for its prefix and adds it.
 *   d_out[i] = x[s] op ... op x[i] (inclusive) or x[s] op ... op x[i-1] with
 *   the identity at i = s (exclusive), s = the first index of i's block
 *   (BLOCK) or 0 (GRID).
 *   op/dt: as cox_tile_reduce; flags: COX_F_COMPENSATED for F32 SUM.
 *   exclusive: 0 or 1.
 *   d_workspace: GRID only, cox_scan_workspace() bytes, 16-byte aligned,
 *   zeroed by the call (cudaMemsetAsync).  Not shared across concurrent calls.
 * Integer results are exact.  GRID fp32 results take each tile's prefix in
 * the order its look-back found the predecessors' values, so their last bits
 * may differ from run to run (within the stated tolerance); a compensated
 * prefix passes between tiles with its error word rounded to 21 mantissa
 * bits (about 2^-46 of the sum).  BLOCK results are reproducible.
 * Look-back waits are bounded as in cox_ballot_compact.
 */
cox_status cox_scan(cox_op op, cox_dtype dt, cox_scope scope, int block_dim, const void* d_in, void* d_out,
                    int64_t n, unsigned flags, int exclusive, void* d_workspace, size_t workspace_bytes,
                    void* stream);

/* Workspace bytes cox_scan needs (0 for BLOCK scope). */
size_t cox_scan_workspace(cox_scope scope, int64_t n);

/*
 * cox_grid_broadcast -- a reduction over the whole array, a grid-wide
 * barrier, then every element uses the result, in ONE cooperative kernel:
 * the grid sync of cooperative groups that gpuConjugateGradient needs and
 * COX cannot support (Table 1; Section 5.1).
 *   COX_GRID_SUB_MIN   y_i = x_i - min_j x_j.  I32/U32 wrap mod 2^32; F32
 *                      subtracts (IEEE, round to nearest) the minimum in
 *                      totalOrder (-0 below +0, NaNs ignored; all NaN
 *                      gives NaN).  Exact: the same bits for any grid.
 *   COX_GRID_NORMALIZE y_i = x_i / ||x||_2 (F32 only): the squares are
 *                      summed with TwoSum pairs, the CTA partials in FP64
 *                      in CTA order (the same total in every CTA), the
 *                      norm rounded once to fp32, one IEEE division.  A
 *                      zero vector gives 0/0 = NaN.
 * d_in, d_out: n 32-bit elements, device memory (they may be the same
 *   array).  Arrays up to ~29 MB stay in shared memory across the barrier
 *   (read once, by TMA bulk copies, when d_in and d_out are 16-byte
 *   aligned); larger ones are read again after it.
 * d_workspace: cox_grid_broadcast_workspace(n) bytes, 16-byte aligned,
 *   zeroed by the call; not shared across concurrent calls.
 * The barrier waits are bounded (cox_set_spin_limit); one that runs out
 * sets COX_ETIMEOUT in the device status word and the CTA writes nothing.
 * Returns COX_EINVAL for a bad op/dtype pair, COX_ENOMEM for a short
 * workspace, COX_ECUDA if the cooperative launch is refused.
 */
typedef enum { COX_GRID_SUB_MIN = 0, COX_GRID_NORMALIZE = 1 } cox_gridop;
cox_status cox_grid_broadcast(cox_gridop op, cox_dtype dt, const void* d_in, void* d_out, int64_t n,
                              void* d_workspace, size_t workspace_bytes, void* stream);
size_t cox_grid_broadcast_workspace(int64_t n);

/*
 * cox_coalesced -- warp functions over coalesced_threads() groups: the
 * dynamic groups and runtime member masks that COX leaves unsupported
 * (Sections 2.2.2-2.2.3; filter_arr's "activated thread sync", Table 1).
 * Element i is global thread i (block_dim a multiple of 32, so a warp is
 * elements 32w .. 32w+31).  A lane is active when i < n and d_active[i] != 0;
 * a warp's group is its active lanes in lane order, rank = active lanes
 * below, size = their count.  For every active lane:
 *   COX_CG_SIZE / COX_CG_RANK      size / rank
 *   COX_CG_SHFL (param)            the value of group rank param mod size
 *   COX_CG_SHFL_UP / _DOWN (param) the value of rank -/+ param, or the
 *                                  caller's own when that rank is outside
 *   COX_CG_BALLOT                  group-local mask: bit k = rank k's
 *                                  predicate (value != 0; fp32 != 0.0f)
 *   COX_CG_ANY / COX_CG_ALL        0 or 1 over the group's predicates
 *   COX_CG_REDUCE_SUM / _SCAN_SUM  group sum / inclusive prefix by rank,
 *                                  mod 2^32 (I32/U32 only)
 * computed by the warp intrinsics with the group's member mask.  Inactive
 * lanes' outputs are not written.  param in [0, 31] for the shuffles.
 */
typedef enum {
  COX_CG_SIZE = 0, COX_CG_RANK = 1, COX_CG_SHFL = 2, COX_CG_SHFL_UP = 3, COX_CG_SHFL_DOWN = 4,
  COX_CG_BALLOT = 5, COX_CG_ANY = 6, COX_CG_ALL = 7, COX_CG_REDUCE_SUM = 8, COX_CG_SCAN_SUM = 9
} cox_cgfn;
cox_status cox_coalesced(cox_cgfn fn, cox_dtype dt, int block_dim, const void* d_in, const int32_t* d_active,
                         void* d_out, int64_t n, int param, void* stream);

/*
 * cox_filter_aggregated -- the SDK's filter_arr: keys with key < threshold
 * (in the keys' signedness; threshold clamped to the key range) are written
 * through a warp-aggregated atomic: each coalesced group of keeping lanes
 * gets one contiguous range of d_out from an atomic add on *d_count, and a
 * lane's slot is its group rank in it.  A warp aggregates its 16 rounds of
 * 32 keys, and a CTA its 8 warps, into one atomic; a warp packs its kept
 * keys in shared memory (the compaction's one-pass body) and copies them
 * out.  The ORDER of the ranges is the order in which the atomics landed
 * (not deterministic); the kept keys, their count, and the lane order
 * inside each group are.  d_out: room for n keys; d_count:
 * one int64, zeroed by the call, holds the count when the stream reaches
 * the end of the call.  dt: COX_I32 or COX_U32.  Keys arrive in 16 KB
 * chunks by TMA bulk copies (16-byte aligned d_keys); a copy that does not
 * land within the spin limit records COX_ETIMEOUT for cox_device_status().
 */
cox_status cox_filter_aggregated(cox_dtype dt, const void* d_keys, int64_t n, int64_t threshold, void* d_out,
                                 int64_t* d_count, void* stream);

/*
 * cox_vote_stats -- batched statistics of the SDK's vote kernels (VoteAny /
 * VoteAll, Table 1): d_pred (n 32-bit values, predicate = value != 0; fp32
 * 0.0f and -0.0f are false) is cut into segments of seg_len elements (a
 * multiple of width; the last segment may be shorter) and each segment into
 * tiles of `width` lanes, whose tile-local ballot gives any/all/popcount.
 * d_stats (3 int64 per segment, zeroed by the call): [tiles with any() true,
 * tiles with all() true, true predicates].  A ragged last tile's missing
 * lanes are padding with a false predicate, so its all() is false.
 */
cox_status cox_vote_stats(cox_dtype dt, int width, const void* d_pred, int64_t n, int64_t seg_len, int64_t* d_stats,
                          void* stream);

/*
 * cox_integral_image -- integral images of a batch of `batch` images of
 * height x width pixels, stored contiguously (image b, row y, column x at
 * (b*height + y)*width + x): out = sum over y' <= y, x' <= x, mod 2^32 --
 * the SDK's shfl_intimage_rows + shfl_vertical_shfl pair (Table 1).
 * in_dt: COX_U8 (uint8 pixels) or COX_U32 / COX_I32 (32-bit, summed mod
 * 2^32).  d_out: batch*height*width uint32.  d_workspace:
 * cox_integral_image_workspace() bytes (per image row a word per 32-pixel
 * strip; per image, band of 64 rows and column a word; per image, band and
 * 128 columns a word), 16-byte aligned; its contents need no preparation
 * and are scratch after the call.
 * Three forms, chosen on the host from the layout and size:
 *  - strip walk (16-byte aligned input and output, rows of whole 16-byte
 *    units, at least 4 x SMs strips of 128 columns in all and at most 64 per
 *    row): one cooperative launch, every pixel read once.  Three warps per
 *    (image, strip) walk the strip top to bottom through a TMA ring; the
 *    integral just left of the strip comes from the left strips' per-row
 *    totals, published as tagged words (the call zeroes them first with a
 *    cudaMemsetAsync on `stream`).  A wait for a neighbour's words or a ring
 *    stage that runs out records COX_ETIMEOUT for cox_device_status() and
 *    leaves the output incomplete.  COX_ECUDA if the launch is refused.
 *  - band form (same layout, fewer strips): rows cut into bands of 64; per
 *    (image, band, strip) one warp sums its block, then one warp walks the
 *    band's rows from the integral above it; pixels read twice.
 *  - three-pass form (any other layout): pixels read three times.
 */
cox_status cox_integral_image(cox_dtype in_dt, int64_t batch, int64_t height, int64_t width, const void* d_in,
                              uint32_t* d_out, void* d_workspace, size_t workspace_bytes, void* stream);
size_t cox_integral_image_workspace(int64_t batch, int64_t height, int64_t width);

/*
 * cox_ballot_compact -- stable stream compaction driven by warp ballots.
 *
 * The filter of the SDK's filter_arr (Table 1) with a static, full-warp group:
 * b = ballot(key < threshold); rank = popc(b & lanes below); per-block scan of
 * warp counts; blocks ordered by a single-pass look-back over tile
 * descriptors.
 *   dt: COX_I32 (signed compare) or COX_U32 (unsigned compare).
 *   d_out: room for n elements; receives the kept keys in input order.
 *   d_count: one int64 on the device, receives the number kept.
 *   d_workspace: at least cox_ballot_compact_workspace(n, block_dim) bytes,
 *   16-byte aligned; the call zeroes it first (a cudaMemsetAsync on `stream`)
 *   unless flags has COX_F_WS_READY, in which case the caller guarantees those
 *   bytes are zero.  Not shared across concurrent calls.
 *   flags: 0 or COX_F_WS_READY.
 * Tiles of 8192 keys go round-robin to the CTAs of one cooperative launch
 * (256 threads each, whatever block_dim: the result does not depend on the
 * block size, which is only validated); each tile's look-back polls its
 * predecessors' descriptors.  A poll that exceeds the spin limit
 * (cox_set_spin_limit) gives up: the tile publishes a zero prefix, writes
 * nothing, and COX_ETIMEOUT is recorded for cox_device_status().  With
 * COX_F_WS_READY, a descriptor word whose two top bits are both set is
 * "withheld": it reads as not yet published, and no publish overwrites it
 * (a way to test that the waits end).  Every write stays inside d_out[0, n)
 * and d_count.  COX_ECUDA if the cooperative launch is refused.
 */
cox_status cox_ballot_compact(cox_dtype dt, int width, int block_dim, const void* d_keys, int64_t n,
                              int64_t threshold, void* d_out, int64_t* d_count, void* d_workspace,
                              size_t workspace_bytes, unsigned flags, void* stream);

size_t cox_ballot_compact_workspace(int64_t n, int block_dim);

/*
 * cox_ballot_compact_static -- cox_ballot_compact without a workspace, for
 * callers that cannot allocate device memory: code running under a host
 * framework whose allocator owns the whole device budget and forbids side
 * allocations, or a latency-critical loop that must not take the implicit
 * device synchronisation of cudaMalloc/cudaFree, or a plugin that is handed
 * only its input and output buffers.  The paper has no counterpart; this is
 * a library convenience.
 *
 * Same arguments and results as cox_ballot_compact minus the workspace and
 * flags.  The scratch is a fixed array of COX_COMPACT_STATIC_SCRATCH_BYTES
 * (1 MiB) inside libcox.so, held on every GPU that loads the library until
 * the process exits.  It fits 256 bytes of header, 8 bytes per tile of
 * 8192 keys and 16 bytes per group of 32 tiles: n <= 123330 * 8192
 * (1,010,319,360 keys).  Larger n returns COX_ENOMEM before anything is
 * enqueued.
 * The call allocates nothing (no cudaMalloc/cudaFree) and clears the scratch
 * bytes it uses with a cudaMemsetAsync on `stream` before its kernel.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture on the device.  Under CUDA's lazy module loading that lookup may be
 * what loads the library's device code on that device, which takes device
 * memory and synchronises; if that load fails the call returns COX_ECUDA.
 * The cached address belongs to the device's primary context: after
 * cudaDeviceReset on that device, do not call this entry point again in the
 * same process.  All calls share the one array: calls whose work overlaps on
 * the GPU (other streams, other threads) race on it and must be serialised
 * by the caller.
 */
#define COX_COMPACT_STATIC_SCRATCH_BYTES (1u << 20)
cox_status cox_ballot_compact_static(cox_dtype dt, int width, int block_dim, const void* d_keys, int64_t n,
                                     int64_t threshold, void* d_out, int64_t* d_count, void* stream);

/*
 * cox_match_histogram -- histogram built from match_any peer groups.
 *
 * Per tile: peers = match_any(key) among the lanes whose key is in [0, bins);
 * one lane of each peer group adds popc(peers) to a shared-memory bin;
 * blocks merge into d_hist.  Same family of warp functions as Section 2.2.1.
 * By default the peer mask comes from a per-warp table in shared memory
 * (each in-range lane ORs its lane bit into its key's word -- one word per
 * key and tile of the warp -- and the lane whose OR found the word empty
 * takes the mask and clears it) when two tables of (32 / width) * bins words
 * per warp fit next to the histograms, else from ceil(log2(bins)) + 1
 * ballots (lanes agree on a key iff they agree on every key bit); both are
 * exactly the mask __match_any_sync returns, and one lane of each peer
 * group adds its popcount.  COX_F_BALLOT_MATCH forces the
 * ballots; COX_F_NATIVE_MATCH takes the mask from the match.any.sync
 * instruction instead (same result, slower on sm_103a).
 * COX_F_DIRECT_ATOMICS skips the peer groups: every key adds one to its
 * shared bin (same counts; on sm_103a shared atomics absorb Zipf-skewed keys
 * at memory speed, so this is the fastest histogram, but it is not built
 * from match_any).
 *   dt: COX_I32 or COX_U32 keys.  bins: 1..8192.
 *   d_hist: `bins` int32 counters, overwritten (zeroed by the call).
 *   d_ignored: optional int64 (may be NULL): number of keys outside [0, bins),
 *   overwritten.
 *   flags: 0 or one of COX_F_NATIVE_MATCH, COX_F_BALLOT_MATCH,
 *   COX_F_DIRECT_ATOMICS.
 */
cox_status cox_match_histogram(cox_dtype dt, int width, int block_dim, const void* d_keys, int64_t n,
                               int bins, int32_t* d_hist, int64_t* d_ignored, unsigned flags, void* stream);

/* ====================================================================== */
/* Batched uneven arrays: per array, a compensated fp32 sum and a 256-bin   */
/* histogram built with match_any, all arrays in one persistent launch.     */
/* ====================================================================== */

/* Launch shape of the batched kernel.  Every field must be set (or pass a
 * NULL tune to take the library default, {512, 2, 32, 8, 3, 8}). */
typedef struct {
  int block_dim;     /* threads per CTA, multiple of 32 in [64, 1024] */
  int ctas_per_sm;   /* persistent CTAs per SM, 1..8 */
  int width;         /* tile width of the match_any histogram step: 2..32 */
  int fp64_segments; /* arrays split over >= this many CTAs combine in FP64 (>= 1) */
  int native_match;  /* peer groups of the histogram step: 0 the match_any masks from 9 ballots,
                        1 the match.any.sync instruction, 2 none (one shared atomic per key;
                        same counts, not built from match_any), 3 the match_any masks from a
                        per-warp table in shared memory (lanes OR their bit into their key's
                        word in their tile's copy of the table; the lane that found the word
                        empty takes the mask and clears it), or from the ballots of 0 where
                        that table (2 x 32 / width x 1 KB per warp) does not fit an SM;
                        4 the same as 3 with the width-32 masks split over two words by lane
                        half (fewer lanes on a hot key's word) and one set of tables */
  int ept;           /* elements per thread per round: 4, 8 or 16 (128-bit loads in flight per
                        thread: ept / 4); the fold order, and so every result, is the same for all */
} cox_batch_tune;

/* Bytes of device workspace for a batch of num_arrays arrays (any tune). */
size_t cox_batch_workspace(int64_t num_arrays);

/*
 * cox_batch_prepare -- writes the batch's offset table (prefix sums of the
 * host array h_lens[num_arrays], lengths >= 0) into d_workspace.  Copies on
 * `stream` and synchronises it before returning, so h_lens may be freed
 * afterwards.  Must precede cox_batch_sum_hist for this batch and workspace.
 */
cox_status cox_batch_prepare(int64_t num_arrays, const int64_t* h_lens, void* d_workspace,
                             size_t workspace_bytes, void* stream);

/*
 * cox_batch_sum_hist -- for every array a (length h_lens[a] as prepared):
 *   d_sums[a]      compensated fp32 sum of d_vals[a][0 .. len)  (fl(s + e));
 *   d_sums64[a]    optional (may be NULL): the same sum as a double
 *                  (s + e of the final pair, or the FP64 combine);
 *   d_hists[a*256 + k] = #{i : d_keys[a][i] == k}, k in [0, 256) (keys
 *                  outside are ignored); zeroed by the call.
 * d_vals / d_keys are DEVICE arrays of num_arrays device pointers.  The grid
 * splits the concatenation of all arrays into equal element ranges, one per
 * persistent CTA; each CTA folds its part of each array (TwoSum pairs per
 * thread, then a shuffle tree) and flushes per-warp match_any histograms;
 * a second small kernel folds each array's per-CTA pairs in CTA order, in
 * FP64 when the array spans >= tune->fp64_segments CTAs (Section 2.2.1
 * warp functions; the paper has no batching of its own).  Results depend
 * only on the data and the tune, never on timing.  Enqueue only: capturable
 * in a CUDA graph.
 */
cox_status cox_batch_sum_hist(int64_t num_arrays, const float* const* d_vals, const int32_t* const* d_keys,
                              const cox_batch_tune* tune, void* d_workspace, size_t workspace_bytes,
                              float* d_sums, double* d_sums64, int32_t* d_hists, void* stream);

/*
 * cox_batch_percall -- the batch's results the slow way, for comparison: one
 * compensated GRID-scope cox_tile_reduce and one cox_match_histogram (width
 * 32) per array, launched back to back from a C loop on `stream`.  h_vals /
 * h_keys: HOST arrays of the arrays' device pointers; h_lens: host lengths.
 * d_sums / d_hists as cox_batch_sum_hist (d_sums from a different order of
 * additions: within the same tolerance, not the same bits).  d_scratch:
 * cox_batch_percall_scratch(longest length) bytes, 16-byte aligned.
 * events: optional host array of num_arrays cudaEvent_t (entries may be
 * NULL), each recorded after its array's launches.
 */
size_t cox_batch_percall_scratch(int64_t max_len);
cox_status cox_batch_percall(int64_t num_arrays, const float* const* h_vals, const int32_t* const* h_keys,
                             const int64_t* h_lens, float* d_sums, int32_t* d_hists, void* d_scratch,
                             size_t scratch_bytes, void* const* events, void* stream);

/* An instantiated CUDA graph of one cox_batch_sum_hist call. */
typedef struct cox_graph cox_graph;

/* Captures cox_batch_sum_hist with these arguments into a graph (on a private
 * stream) and instantiates it.  Replays read the buffers named here. */
cox_status cox_batch_graph_create(int64_t num_arrays, const float* const* d_vals, const int32_t* const* d_keys,
                                  const cox_batch_tune* tune, void* d_workspace, size_t workspace_bytes,
                                  float* d_sums, double* d_sums64, int32_t* d_hists, cox_graph** out);
cox_status cox_graph_launch(cox_graph* g, void* stream);
void cox_graph_destroy(cox_graph* g);

/*
 * cox_batch_autotune -- times every candidate tune (block_dim 256/512/1024 x
 * ctas_per_sm 1/2/4 x width 8/32 x elements per thread 4/8/16 x table-built
 * peer masks 3/4; fp64_segments 8 in every candidate) on
 * this batch (prepared in d_workspace) with CUDA events, `reps` timed runs
 * each, and returns the fastest in *best (and its mean milliseconds in
 * *best_ms if non-NULL).  If cache_path is not NULL the winner is appended to
 * that file as one line
 * "<gpu name>|batch_sum_hist|<arrays bucket>|<elements bucket>|b,c,w,f,m,e|ms".
 * Synchronises `stream`.  Overwrites the output buffers.
 */
cox_status cox_batch_autotune(int64_t num_arrays, const float* const* d_vals, const int32_t* const* d_keys,
                              void* d_workspace, size_t workspace_bytes, float* d_sums, int32_t* d_hists,
                              int reps, const char* cache_path, cox_batch_tune* best, float* best_ms,
                              void* stream);

/* Looks up a tune for (num_arrays, total elements) in a cache file written by
 * cox_batch_autotune on the current GPU.  COX_EINVAL if none matches. */
cox_status cox_batch_tune_lookup(const char* cache_path, int64_t num_arrays, int64_t total_elems,
                                 cox_batch_tune* tune);

/* ====================================================================== */
/* Request server: continuous batching of reduce / scan / compact requests */
/* ====================================================================== */

typedef enum { COX_REQ_REDUCE = 0, COX_REQ_SCAN = 1, COX_REQ_COMPACT = 2 } cox_req_kind;

/* One request.  REDUCE: the sum of all n elements (COX_F32, compensated with
 * COX_F_COMPENSATED, or COX_I32 wrapping); output one element followed by the
 * fp32 low word.  SCAN: tile inclusive sum scan of width `width` (COX_F32 or
 * COX_I32), n elements out.  COMPACT: keys < threshold in input order
 * (COX_I32 signed or COX_U32 unsigned compare), up to n elements out. */
typedef struct {
  cox_req_kind kind;
  cox_dtype dt;
  int width;
  unsigned flags;
  int64_t n;            /* >= 1 */
  int64_t threshold;    /* COMPACT only */
  const void* d_in;     /* device input, caller-owned, valid until the request completes */
} cox_request;

typedef struct cox_server cox_server;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t batches;      /* persistent launches so far */
  int64_t max_batch;    /* most requests in one launch */
  size_t budget_bytes;  /* admission budget */
  size_t used_bytes;    /* held by admitted, unreleased requests */
  size_t peak_bytes;    /* most ever held */
  int64_t queued;       /* submitted, waiting for admission */
  double wait_s;        /* summed over completed requests: submit to launch (queueing and batching) */
  double run_s;         /* summed over completed requests: launch to done (on the device) */
} cox_server_stats;

/*
 * cox_server_create -- a server on the current device with an arena of
 * budget_bytes of device memory (allocated here, once) and at most
 * max_requests admitted requests at a time.  A scheduler thread admits
 * queued requests in arrival order while the arena has room for their
 * output and workspace (plus their input, counted as held) and a slot is
 * free; it packs every admitted request not yet launched into one
 * persistent kernel -- each request cut into tiles of 16384 elements that
 * CTAs take from an atomic counter in request order -- on one of three
 * streams, so a batch launched while another runs overlaps with it on the
 * device (batches of up to 24 requests pass their table as a kernel
 * parameter, larger ones copy it first); and it marks each request done as
 * soon as the kernel raises that request's flag in pinned host memory --
 * after its last tile's results are in device memory, without waiting for
 * the rest of the batch -- or at the latest when the batch's event fires.
 * A batch of one request runs that op's own kernel instead (a scan or
 * compaction: cox_tile_scan or cox_ballot_compact; a reduce: one CTA per
 * tile in the batch kernel's order) and completes with its event, so an
 * idle server costs one launch per request.
 * Each request's arithmetic depends only on the request (its tiles, its
 * fixed-order combine), never on what else shares its launch.
 */
cox_status cox_server_create(size_t budget_bytes, int max_requests, cox_server** out);

/* Queues a request; COX_ENOMEM if it could never fit the budget. */
cox_status cox_server_submit(cox_server* s, const cox_request* req, uint64_t* ticket);

/* Queues count requests at once (tickets[i] for reqs[i]), so that the
 * scheduler sees them together and, load permitting, packs them into one
 * launch.  All are checked first: on an error (COX_EINVAL, COX_ENOMEM as for
 * cox_server_submit) none is queued. */
cox_status cox_server_submit_many(cox_server* s, const cox_request* reqs, int64_t count, uint64_t* tickets);

/* *done = 1 once the request's results are on the device. */
cox_status cox_server_poll(cox_server* s, uint64_t ticket, int* done);

/* Blocks until the request is done or timeout_s passes (COX_ETIMEOUT). */
cox_status cox_server_wait(cox_server* s, uint64_t ticket, double timeout_s);

/* Device pointer of a done request's output (valid until release) and its
 * element count (REDUCE 1, SCAN n, COMPACT the kept count, read from the
 * device with a synchronous copy). */
cox_status cox_server_result(cox_server* s, uint64_t ticket, void** d_out, int64_t* count);

/* Frees a done request's arena memory and slot. */
cox_status cox_server_release(cox_server* s, uint64_t ticket);

cox_status cox_server_get_stats(cox_server* s, cox_server_stats* st);

/* Stops the scheduler after the work in flight and frees the arena. */
void cox_server_destroy(cox_server* s);

/* A request of a replayed trace: submitted arrival_s seconds after the start. */
typedef struct {
  double arrival_s;
  cox_request req;
} cox_trace_item;

/*
 * cox_server_run_trace -- replays a trace (arrival times non-decreasing)
 * through the server from the calling thread (busy-waiting to each arrival),
 * releases every request as it completes, and writes latency_s[i] =
 * completion - arrival for each item and *wall_s = time to the last
 * completion.
 */
cox_status cox_server_run_trace(cox_server* s, const cox_trace_item* items, int64_t count, double* latency_s,
                                double* wall_s);

/*
 * cox_percall_run_trace -- the same trace with one launch per request: each
 * request goes to cox_tile_reduce (GRID), cox_tile_scan or
 * cox_ballot_compact on one stream as it arrives, outputs and workspaces
 * carved from d_scratch (scratch_bytes >= cox_percall_scratch(max n));
 * latency as above.
 */
size_t cox_percall_scratch(int64_t max_n);
cox_status cox_percall_run_trace(const cox_trace_item* items, int64_t count, void* d_scratch, size_t scratch_bytes,
                                 double* latency_s, double* wall_s);

/*
 * cox_device_status -- synchronises `stream`, then reads and clears the
 * device-side status word of the current device.  Returns COX_ETIMEOUT if
 * any kernel since the last call gave up a bounded wait, COX_ECUDA if the
 * synchronisation failed, COX_OK otherwise.
 */
cox_status cox_device_status(void* stream);

/*
 * cox_set_spin_limit -- iteration cap of every bounded device-side wait
 * (look-back, work queues), taken by kernels launched after the call.
 * 0 restores the default (2^22 polls with back-off, about a second).
 */
void cox_set_spin_limit(uint32_t polls);

#ifdef __cplusplus
}
#endif

#endif /* COX_H_ */
