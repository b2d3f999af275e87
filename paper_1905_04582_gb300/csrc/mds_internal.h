// Internal declarations shared by the host runtime (api.cpp) and the CUDA
// kernels.  Not part of the public ABI (include/mds.h).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace mds {

// ---------------------------------------------------------------------------
// Tile geometry of the pair pass.
//
// The M = N(N-1)/2 pairs i < j are covered by 64 x 64 tiles (I, J), I <= J,
// over row blocks I and column blocks J of 64 items (nt = ceil(N/64) blocks).
// Diagonal tiles (I == J) hold the full square; pairs with j <= i, and items
// past N in the last block, are masked.  Tiles are stored back to back in
// row-block order, t(I, J) = I*nt - I*(I-1)/2 + (J - I), so the tiles of one
// row block are contiguous.
//
// Work split inside a tile (one CTA of 4 warps): warp w takes columns
// [16w, 16w+16).  In the strip pass (and the chunked pass for D > 2) lane
// l = 8b + a takes the 4 columns 16w + 4b + {0..3} and the 8 rows
// 2(a + 8q) + {0, 1}, q = 0..3 (4 row pairs); in the chunked pass for D <= 2
// lane l = 4b + a takes the 2 columns 16w + 2b + {0, 1} and the 16 rows
// 2(a + 4q) + {0, 1}, q = 0..7 (8 row pairs).  Y inside a tile is stored as
// float4 {y(r,c), y(r+1,c), y(r,c+1), y(r+1,c+1)} (two row-packed operands of
// the f32x2 instructions) in the order the first mapping reads them:
//   element (r, c) at  ((w * 8 + t) * 32 + slot) * 4 + e,
//   w = c / 16, b = (c / 4) % 4, half = (c % 4) / 2, rp = r / 2, a = rp % 8,
//   q = rp / 8, slot = 8b + (a XOR 4 half), t = 2q + half, e = 2 (c % 2) + (r % 2),
// so that warp w's quarter of a tile is 4 KB contiguous (one bulk TMA copy).
// A 128-bit shared-memory load of the first mapping reads 512 contiguous
// bytes (lane l at slot l XOR 4 half); the XOR keeps the second mapping's
// loads free of bank conflicts too (each group of 8 lanes covers all banks).
// ---------------------------------------------------------------------------
constexpr int kTile = 64;
constexpr int kTileElems = kTile * kTile;   // 4096 FP32 values = 16 KB
constexpr int kPairWarps = 4;               // warps per CTA in the pair kernel
constexpr int kPairThreads = 32 * kPairWarps;
constexpr int kWarpCols = kTile / kPairWarps;  // 16 columns per warp
constexpr int kWarpTileElems = kTileElems / kPairWarps;  // 1024 floats = 4 KB per warp

__host__ __device__ inline int64_t tile_index(int64_t I, int64_t J, int64_t nt) {
    return I * nt - I * (I - 1) / 2 + (J - I);
}

__host__ __device__ inline int64_t tile_count(int64_t nt) { return nt * (nt + 1) / 2; }

// Slot of tile (I, J), I <= J, in the column partials: column-block-major,
// so that the partials one column block gathers (one per row block I <= J)
// are contiguous for the reduction.
__host__ __device__ inline int64_t col_slot(int64_t I, int64_t J) { return J * (J + 1) / 2 + I; }

// Offset of (r, c) inside a tile (see above).
__host__ __device__ inline int tile_offset(int r, int c) {
    const int w = c >> 4, b = (c >> 2) & 3, half = (c >> 1) & 1, ec = c & 1;
    const int rp = r >> 1, a = rp & 7, q = rp >> 3;
    const int slot = 8 * b + (a ^ (half << 2)), t = 2 * q + half, e = 2 * ec + (r & 1);
    return ((w * 8 + t) * 32 + slot) * 4 + e;
}

// Offset of row i in the packed strict upper triangle (row-major (0,1),(0,2),...).
__host__ __device__ inline int64_t packed_row_start(int64_t i, int64_t n) { return i * n - i * (i + 1) / 2; }

// One unit of work of the pair kernel: row block I against column blocks
// [j0, j1) (j0 >= I).  row_slot indexes this strip's row partial sums; the
// strips of a row block occupy consecutive row slots.
struct Strip {
    int32_t I, j0, j1, row_slot;
};

// One unit of work of the chunked FP32C pair pass (chunk_kernel.cu): the
// tiles [t0, t1) of the row-block-ordered tile sequence, (I0, J0) the blocks
// of tile t0 and I1 the row block of tile t1 - 1.  A segment is a run of at
// most max_seg_tiles(D) of a chunk's tiles in one row block: the chunk's run
// in a row block of L tiles is ceil(L / max_seg_tiles(D)) segments.  seg0 is
// the chunk's first segment in the global order of segments (chunk by
// chunk), which sets its row-partial slots: warp w of segment g writes slot
// 4 g + w.  The segments of one row block are consecutive in that order.
// max_seg_tiles bounds the FP32 row sums a lane keeps in registers at 64
// terms, as the strip pass's longest strip: 2 columns x 32 tiles in the
// 16 x 2 lane mapping of D <= 2, 4 columns x 16 tiles in the 8 x 4 one.  The
// rounding of an FP32 partial sum grows faster than its length: at 256 terms
// a lane, well-conditioned gradient coordinates of N = 20000, D = 2 reached
// 1.25e-5 against the 1e-5 tolerance.
__host__ __device__ constexpr int max_seg_tiles(int d) { return d <= 2 ? 32 : 16; }
struct Chunk {
    int64_t t0, t1;
    int32_t I0, J0, I1;
    int32_t seg0;
};

// Scalar partial sums per strip, in this order.
enum ScalarPart : int {
    kSumE2 = 0,     // sum (y - delta)^2
    kSumMDelta,     // FP32C: sum m' delta, m' = sqrt(2 pi) phi(z)/Phi(z);  FP64: sum (phi/Phi) delta
    kSumLogPhi,     // FP32C: sum log2(1/Phi(z));                           FP64: sum log Phi(z)
    kSumSpare,
    kScalarParts
};

// ---------------------------------------------------------------------------
// Location layouts of the FP32C path.
//
// Exact differences: every coordinate is split x = xh + xl, xh the nearest
// multiple of a power-of-two quantum q (chosen from max |x| so that
// |xh_i - xh_j| / q < 2^B, B = 11 for D <= 4 and 10 for D <= 8).  Then
// Dh = xh_i - xh_j and Dh^2 are exact in FP32, sum_k Dh_k^2 is exact, and
// the squared distance is sum_k Dh^2 + Dl (2 Dh + Dl) with Dl = xl_i - xl_j,
// a small correction computed in FP32 -- which keeps y - delta accurate where
// y and delta nearly cancel.
//   xrow[(I * D + k) * 32 + r] (float4) = { xh_{i,k}, xh_{i+1,k}, xl_{i,k}, xl_{i+1,k} },
//        i = 64 I + 2 r (row block I, row pair r: D x 32 float4, contiguous)
//   xcol[(j  * D + k)] (float4) = { -xh_{j,k}, -xh_{j,k}, -xl_{j,k}, -xl_{j,k} }
// A row block is 32 D float4 in the [k][row pair] order the pair kernel
// reads (one bulk TMA copy per strip); a tile's column block J is 64 D
// float4, contiguous (bulk-copied per warp).
// ---------------------------------------------------------------------------
struct Split {
    float q;       // quantum
    float magic;   // 1.5 * 2^23 * q: (x + magic) - magic rounds x to a multiple of q
    float bound;   // largest |x| this quantum splits exactly: (2^(B-1) - 1) q
    int resplit;   // set by the end-of-trajectory reduction when it chose a new
                   // quantum; the trajectory-end kernel then rewrites the layouts
};

// Arguments of the fused pair pass.
struct PairArgs {
    const float *y;          // tile-packed Y (FP32): tile t at y + (t - y_t0) * kTileElems
    int64_t y_t0;            // first tile held (a shard holds only its range; 0 otherwise)
    const float4 *xrow;      // FP32C: row-pair split layout;  FP64: unused
    const float4 *xcol;      // FP32C: column split layout;   FP64: unused
    const double *x64;       // FP64: plain locations [n_pad][D]
    const Strip *strips;     // work list, one strip per CTA, largest first
    int32_t n_strips;
    int32_t nt;              // blocks per side
    int64_t n;               // N
    void *row_part;          // [row slots][64][D] (float / double)
    void *col_part;          // [tiles][64][D]     (float / double)
    void *scal_part;         // [n_strips][kScalarParts] (float / double)
    const unsigned char *tile_ho;  // [tiles] 1 where a tile holds a held-out pair (y < 0), or null
    const int32_t *perm;     // FP64: item at slot s (locality order, mds_reorder), or null (identity)
    int32_t *far_part;       // FP32C: per strip and warp, the warp blocks (64 x 8 pairs) of the last
                             // pass that skipped the Phi terms (diagnostics), or null
    unsigned *err;           // device error word (see ErrBits)
    const Chunk *chunks;     // chunked FP32C pass: one chunk per CTA (n_strips chunks), else null
    const float2 *xcol2;     // chunked FP32C pass: column layout {-xh_j, -xl_j} [(j * D + k)]
    unsigned char *far_tile; // chunked FP32C pass: per tile and warp, the column pairs (0..2) that took
                             // the far body, for the cost model of the chunking (or null)
    unsigned long long *stamps;  // if not null: [0] earliest start and [1] latest end (%globaltimer ns)
                                 // of the pass's warps after the dependency wait (min / max atomics)
    float far_d2;            // FP32C: (z_c sigma)^2; warp blocks at least this far apart skip the Phi
                             // terms (+inf: never)
    int32_t long_runs;       // chunked FP32C pass: some chunk runs more than max_seg_tiles(D) tiles in
                             // one row block, so its segments are cut every max_seg_tiles(D) tiles (in the
                             // padding before the float2 constants: the layout after it is unchanged)
    // FP32C constants (sigma folded in on the host), each duplicated {c, c}
    // so that it is a ready operand of the packed f32x2 instructions
    float2 mp[4];            // -P(delta/sigma)/sqrt(2 pi) coefficients in powers of delta
    float2 md[4];            // D(delta/sigma) coefficients in powers of delta (md[0] = 1)
    float2 c_phi;            // -log2(e) / (2 sigma^2): 2^(c_phi delta^2) = exp(-z^2/2)
    float2 neg_inv_s2;       // -1/sigma^2
    float2 m_coef;           // 1/(sigma sqrt(2 pi))
    float2 c_m2;             // chunked pass: -sigma / sqrt(2 pi), the Phi term of the gradient weight in
                             // units of -1/sigma^2 (its partial sums carry the factor -sigma^2)
    // FP64 constants
    double sigma;
    double inv_sigma;
    double inv_s2;
};

enum ErrBits : unsigned {
    kErrTimeout = 1u,     // a bounded mbarrier wait gave up
    kErrNonfinite = 2u,   // a partial sum was NaN / Inf
    kErrBadArgs = 4u,     // kernel launched with inconsistent arguments
    kErrBadInput = 8u,    // an input value was negative / NaN / Inf
    kErrRange = 16u,      // locations beyond the range the FP32C split serves
    kErrOverflow = 32u,   // more HMC iterations queued than the result buffers hold
};

// ---------------------------------------------------------------------------
// Batched pair pass (batch_kernel.cu): several datasets (each its own Y, N,
// sigma), each with several HMC chains, in one persistent launch.  A CTA
// takes a strip of one dataset, loads its Y tiles into shared memory once and
// runs the whole strip for every chain of that dataset in turn.
// ---------------------------------------------------------------------------
struct BatchDataset {
    const float *y;            // tile-packed Y
    int64_t n;
    int32_t nt;
    int32_t chain0, n_chains;  // its chains in the chain table
    int32_t pad;
    // FP32C constants (sigma folded in), as in PairArgs
    float2 mp[4];
    float2 md[4];
    float2 c_phi;
    float2 neg_inv_s2;
    float2 m_coef;
};

struct BatchChain {
    const float4 *xrow;
    const float4 *xcol;
    float *row_part;           // [slots][64][D]
    float *col_part;           // [tiles][64][D]
    float *scal_part;          // [strips of its dataset][kScalarParts]
};

struct BatchStrip {
    int32_t dataset, I, j0, j1, row_slot, local;  // local: position in the dataset's strip list
};

struct BatchPairArgs {
    const BatchDataset *ds;
    const BatchChain *ch;
    const BatchStrip *strips;
    int32_t n_strips;
    int32_t strip_cap;         // tiles per strip at most (sizes the shared memory)
    unsigned *err;
};

cudaError_t launch_pair_batch(const BatchPairArgs &a, int d, int grid, cudaStream_t s);
size_t pair_batch_smem(int d, int strip_cap);
int pair_batch_blocks_per_sm(int d, int strip_cap);

// Fault injection for tests: a kernel whose bounded wait on an mbarrier that
// nothing completes runs out and sets kErrTimeout (pair_kernel.cu).
cudaError_t launch_wait_probe(unsigned *err, cudaStream_t s);

// Kernel launchers (pair_kernel.cu).
// pdl: launch with programmatic dependent launch (the kernel may become
// resident while the previous one drains); off when a concurrent kernel on
// another stream should get SMs first.
// smem_min: dynamic shared memory of each CTA at least this (the layout's
// size otherwise): more only to cap the pass's CTAs per SM.
cudaError_t launch_pair_pass_f32(const PairArgs &a, int d, cudaStream_t s, bool pdl = true, int smem_min = 0);
// The chunked FP32C pass (chunk_kernel.cu): a.chunks / a.n_strips chunks,
// one CTA each.
// grouped: one CTA per SM whose groups of four warps each run a chunk
// (pair_chunk_groups(d) groups); otherwise one chunk per CTA.
cudaError_t launch_pair_chunks_f32(const PairArgs &a, int d, cudaStream_t s, bool pdl = true, int smem_min = 0,
                                   bool grouped = false);
int pair_chunk_smem_bytes(int d);
int pair_chunk_blocks_per_sm(int d, bool grouped = false);  // chunk slots resident per SM
int pair_chunk_groups(int d);
int pair_f32_smem_bytes(int d);
cudaError_t launch_pair_pass_f64(const PairArgs &a, int d, cudaStream_t s, bool pdl = true);

// ---------------------------------------------------------------------------
// Reduction, leapfrog updates and HMC bookkeeping (reduce_kernel.cu).
// ---------------------------------------------------------------------------

// Per-context scalars kept on the device (FP64).
enum Scalar : int {
    kLogLik = 0,    // L at the current x (what the API reports)
    kSumR,          // sum r at the current x
    kDSigma,        // dL/dsigma at the current x
    kLogLik0,       // L at the trajectory start (saved by the start kernel)
    kSumR0,
    kDSigma0,
    kLogLikEnd,     // L at the end of the pass just reduced (read by the end kernel)
    kLastDH,        // H(end) - H(start) of the last trajectory
    kPriorLogp,     // log p(X) of the tree prior at the current x (0 without one)
    kPriorLogp0,    // the same at the trajectory start
    kScalars
};

// Per-context counters kept on the device.  The start kernel snapshots the
// running counters into the *Cur slots, which the end kernel only reads, so
// that no CTA of the end kernel can observe CTA 0's increment.
enum Counter : int {
    kIter = 0,      // HMC iterations run (drives the Philox counter)
    kIterLocal,     // iterations run in the current mds_hmc call
    kAccepted,      // accepted proposals (total)
    kIterCur,       // snapshot of kIter for the trajectory in flight
    kIterLocalCur,  // snapshot of kIterLocal
    kCounters
};

// Reduction / update modes of the reduce kernel.
enum ReduceMode : int {
    kModeEval = 0,      // gradient + scalars only
    kModeKickDrift,     // + p += eps g(x); x += eps p            (inner leapfrog steps)
    kModeHalfKick,      // + p += eps/2 g(x); kinetic / ||x||^2 partials (last step)
};

// Location state shared by the update kernels.
struct XState {
    void *x;                  // [n_pad][D] (float / double): the state, in the caller's item order
    const int32_t *inv;       // slot of item k in the tile layouts (locality order), or null (identity)
    float4 *xrow;             // FP32C split layouts (null on the FP64 path)
    float4 *xcol;
    float2 *xcol2;            // FP32C column layout of the chunked pass {-xh, -xl} (or null)
    Split *split;             // FP32C quantum (device; grown by the end-of-trajectory reduction)
    unsigned *xmax_bits;      // FP32C: running max |x| (float bits, atomicMax)
};

struct ReduceArgs {
    const void *row_part;
    const void *col_part;
    const void *scal_part;
    double part_scale;        // the gradient is part_scale (sum of column partials - sum of row partials):
                              // 1 for the strip passes, -1/sigma^2 for the chunked FP32C pass
    float2 part_scale_df;     // part_scale as a double-float (hi, lo) for the FP32C reduction
    bool use_grad;            // sharded update: take the gradient from `grad` (all ranks' partials,
                              // combined) instead of summing partials; the scalar CTA keeps L, sum r
                              // and dL/dsigma as the combine left them
    unsigned long long *stamps;   // the pass's start / end stamps (PairArgs::stamps), or null: the
    double *pass_ns;              // scalar CTA adds end - start to pass_ns[0], counts pass_ns[1], resets
    const int32_t *row_first_slot;  // [nt + 1]
    const int32_t *perm;      // item at slot s of the tile layouts, or null (identity)
    int32_t n_strips;
    int32_t nt;
    int64_t n;
    int32_t d;
    int32_t mode;
    bool fp64;                // context precision (x, p, partial types)
    double m_pairs;           // pairs in the likelihood (M less the held-out ones)
    double sigma;
    double log_sigma, inv_sigma;  // log(sigma), 1 / sigma (host)
    double lambda;            // prior precision
    double eps;               // leapfrog step
    double *grad;             // [N][D] dL/dx (FP64 copy for the API)
    double *scal;             // [kScalars]
    XState xs;
    void *p;                  // [N][D]
    double *energy_part;      // [nt * kReduceQuarters][2] (kModeHalfKick): kinetic, ||x||^2
    const double *prior_grad; // [N][D] d log p / dX of the tree prior at x (added to the kicks), or null
    const double *tree_part;  // the tree prior's per-CTA sums (or null); with tree_const, summed into
    int32_t n_tree_parts;     //   scal[kPriorLogp] by the scalar CTA (evaluations, a trajectory's end)
    double tree_const;
    unsigned *err;
};

// The reduction runs kReduceQuarters CTAs per column block (16 items each)
// plus one CTA for the scalars.
constexpr int kReduceQuarters = 4;
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t s);

// Trajectory start: (optionally) draw / load p, save x0 and the cached
// gradient / scalars, kinetic-energy partials, then p += eps/2 g, x += eps p.
struct TrajArgs {
    int64_t n;
    int32_t d;
    bool fp64;
    double eps;
    double lambda;
    int32_t momentum_src;     // 0: keep p, 1: Philox draw, 2: injected FP64 array
    const double *p_inj;      // [n_iter][N][D] when momentum_src == 2 (indexed by kIterLocal)
    uint64_t seed;
    uint32_t chain;
    XState xs;
    void *p;
    void *x0;
    double *grad;
    double *grad0;
    double *scal;
    int64_t *counters;
    double *energy_part;      // [gridDim][2]: kinetic energy, ||x||^2 at the start
    int32_t drift;            // 1: take the first half kick + drift (n_steps > 0)
    const double *prior_grad; // tree prior gradient at x (or null); saved into prior_grad0
    double *prior_grad0;
};
cudaError_t launch_traj_start(const TrajArgs &a, int *grid_out, cudaStream_t s);

// Trajectory end: sum the energy partials in a fixed order, H0 and H1, the
// Metropolis decision (log u < H0 - H1; u from Philox or injected), restore on
// reject, bookkeeping.  Every CTA takes the same decision.
struct AcceptArgs {
    int64_t n;
    int32_t d;
    bool fp64;
    int32_t metropolis;       // 0: always keep the end point (plain leapfrog)
    int32_t n_start_parts;    // energy partials of the start kernel
    int32_t n_end_parts;      // energy partials of the last reduce
    const double *start_part;
    const double *end_part;
    double lambda;
    int32_t u_src;            // 1: Philox, 2: injected
    const double *u_inj;      // [n_iter]
    uint64_t seed;
    uint32_t chain;
    XState xs;
    const void *x0;
    double *grad;
    const double *grad0;
    double *scal;
    int64_t *counters;
    double *prior_grad;       // tree prior gradient (restored from prior_grad0 on reject), or null
    const double *prior_grad0;
    int32_t *acc_out;         // [out_cap] per-iteration decision (optional)
    double *dh_out;           // [out_cap] per-iteration H1 - H0 (optional)
    int64_t out_cap;          // entries of acc_out / dh_out
    unsigned *err;
};
cudaError_t launch_traj_end(const AcceptArgs &a, cudaStream_t s);
// z (standard normal) and u (uniform) of sigma updates iter0 .. iter0 + n - 1.
cudaError_t launch_sigma_draws(uint64_t seed, uint32_t chain, int64_t iter0, int n, double *z, double *u,
                               cudaStream_t s);

// Batched launches (one per step for all problems): per-problem argument
// tables in device memory.  jobs[k] = (problem, column block J or -1).
cudaError_t launch_reduce_batch(const ReduceArgs *cfg, const int2 *jobs, int n_jobs, int d, int mode, cudaStream_t s);
int traj_start_grid(int64_t n, int d);
cudaError_t launch_traj_start_batch(const TrajArgs *cfg, int n_chains, int max_grid, int d, cudaStream_t s);
cudaError_t launch_traj_end_batch(const AcceptArgs *cfg, int n_chains, int64_t max_nd, int d, cudaStream_t s);

// ---------------------------------------------------------------------------
// Phylogenetic Brownian-diffusion prior (tree_prior.cu).  Internal node
// records, per tree in post-order level order (leaves' parents first, the
// root last); the weights come from the message variances, which depend on
// the tree alone and are computed on the host.
// ---------------------------------------------------------------------------
struct TreeNode {
    int32_t c0, c1;          // children: >= 0 a node of the same part (its local index),
                             // < 0 the part's tip -(c + 1) (index into the part's tip list)
    double alpha;            // upward mean: m_k = m_c1 + alpha (m_c0 - m_c1)
    double cinv;             // 1 / (variance of the contrast m_c0 - m_c1)
    double beta0, beta1;     // downward mean of child i: m_s + beta_i (m_k - m_s), s its sibling
    double g0, g1;           // 1 / (downward variance) of a tip child (gradient scale)
};

// A tree is cut into blocks (whole subtrees of at most S internal nodes)
// and a top (the internal nodes whose subtrees are larger); one cluster of
// `cluster` CTAs evaluates it, CTA c holding part c: the blocks assigned to
// it and, for c = 0, the top.  Local node indices of a part: its blocks'
// internal nodes [0, m_blk) by height; for part 0 then one proxy per block
// root of the tree [m_blk, m_blk + n_prox) (in slot order: they hold the
// block roots' messages, exchanged through `xch`), and the top nodes
// [m_blk + n_prox, m) by height.
struct TreePart {
    int32_t m_blk, n_prox, m_top;
    int32_t lv0;             // the part's first level bound in lv_start: block levels, then top levels
    int32_t nlv_blk, small_blk;  // block levels; levels from small_blk on hold <= 32 nodes each
    int32_t nlv_top, small_top;  // the same for the top levels (part 0)
    int32_t exp0, exp1;      // the part's block roots: exp_loc / exp_slot [exp0, exp1)
    int32_t root_loc;        // part 0: local index of the tree's root (a top node or a proxy); else -1
    int32_t n_slots;         // block roots of the tree
    int64_t xch_off;         // the tree's exchange arrays: up means at xch_off, down means after them
    int64_t scr_off;         // messages in global scratch (smem_bytes == 0): this part's offset
};

struct TreeArgs {
    int64_t n;               // tips (items)
    const void *x;           // locations [N][D] (float or double, item order)
    bool x_f64;
    int32_t n_trees;
    int32_t cluster;         // CTAs (one cluster) per tree; part p = tree p / cluster, rank p % cluster
    const TreePart *parts;   // [n_trees * cluster]
    const TreeNode *nodes;   // part p's local nodes at [node_off[p], node_off[p+1]) (proxies: unused)
    const int32_t *node_off; // [n_parts + 1]
    const int32_t *tip_items;// part p's tips (their items) at [tip_off[p], tip_off[p+1])
    const int32_t *tip_off;  // [n_parts + 1]
    const int32_t *lv_start; // first local index of each level (a level ends where the next starts,
                             // the last block level at m_blk, the last top level at the part's end)
    const int32_t *exp_loc;  // block roots: local index in their part
    const int32_t *exp_slot; //   and slot in the tree's exchange arrays
    double *xch;             // exchange arrays (scratch)
    const double *root_cinv; // per tree: 1 / (v_root + tau0)
    int32_t n_lone;
    const int32_t *lone;     // unsequenced items (tips that are roots)
    double tau_u;
    const double *sigma_inv; // D x D
    const double *mu;        // D
    double const_term;       // sum of the log-determinant and 2 pi terms
    int32_t smem_bytes;      // > 0: each CTA keeps its part's records, messages and tips in shared memory
    double *scratch;         // otherwise: per part (2 m + 2 k) x D + k doubles at scr_off
    double *grad;            // [N][D] d log p / dX (out)
    double *part;            // [grid] per-CTA sums (scratch)
    double *out;             // log p (device scalar): the sum of part and const_term, written by a
                             // one-warp kernel after the traversal when not null
};

// log p of the tree prior from its per-CTA sums: const_term plus the parts
// in a fixed order (lane-strided sums, then a butterfly).  Called by all 32
// lanes of one warp; every lane returns the total.
__device__ inline double tree_parts_sum(const double *part, int n, double const_term) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return const_term + s;
}
// Measured ceiling of the pass's per-pair arithmetic (ceiling.cu): grid
// CTAs of kPairThreads threads, each thread `iters` rounds of 16 pairs (four
// row pairs against two columns, two pairs per call) with every operand in
// registers; sink [grid * kPairThreads] keeps the results live.
int pair_ceiling_blocks_per_sm(int d);
cudaError_t launch_pair_ceiling(const PairArgs &a, int d, bool far, int grid, int iters, float *sink, cudaStream_t s);

constexpr int kTreeMaxCluster = 8;  // CTAs per tree (portable cluster size)
cudaError_t launch_tree_prior(const TreeArgs &a, int d, cudaStream_t s);

// ---------------------------------------------------------------------------
// Single-item random-walk Metropolis (rwmh.cu): one CTA runs the proposals
// in order.
// ---------------------------------------------------------------------------
struct RwmhArgs {
    int64_t n;
    const float *y;           // tile-packed Y
    int32_t nt;
    const int32_t *inv;       // slot of each item (locality order), or null
    const int32_t *perm;      // item at each slot, or null
    void *x;                  // [N][D] state (float or double), updated in place
    bool fp64;
    double sigma, lambda, step;
    int32_t n_prop;
    const int64_t *items;     // the draws (device; injected, or from rwmh_draws_kernel)
    const double *z;          // [n_prop][D]
    const double *logu;       // [n_prop] log of the uniforms
    bool x_in_smem;           // keep X in shared memory (N D values fit)
    int32_t cluster;          // CTAs (one cluster) that share each proposal's row; > 1 only with x_in_smem
    uint64_t seed;
    uint32_t chain;
    int64_t iter0;            // Philox counter of the first proposal
    int32_t *acc_out;         // [n_prop] decisions (optional)
    double *dl_out;           // [n_prop] log-target differences (optional)
    unsigned *xmax_bits;      // FP32C running max |x| (atomicMax), or null
    unsigned *err;
    // FP32 Phi constants (sigma folded in), as in PairArgs: -P(delta/sigma)/sqrt(2 pi)
    // and D(delta/sigma) in powers of delta, and -log2(e) / (2 sigma^2)
    float mp[4], md[4];
    float c_phi;
};
cudaError_t launch_rwmh(const RwmhArgs &a, int d, cudaStream_t s);
// Philox draws of the proposals of `a` (counters as in the chain) into
// device arrays: items [n_prop], z [n_prop][D], log u [n_prop].
cudaError_t launch_rwmh_draws(const RwmhArgs &a, int d, int64_t *items, double *z, double *logu, cudaStream_t s);

// Y ingest: rows [r0, r1) of the caller's Y (full or packed layout; the
// pointer addresses row r0) into the tile-packed FP32 layout.  Entries read
// must be finite and >= 0; the first bad (i, j) is recorded in *bad (i*N+j,
// atomicMin) and kErrBadInput is set.
struct IngestArgs {
    const void *src;
    int64_t t_lo, t_hi;       // tiles held by the destination (a shard's range; 0, tiles otherwise):
                              // tile t is written at y + (t - t_lo) * kTileElems, others skipped
    bool src_f64;
    bool packed;
    int64_t ld;               // full layout: row stride (elements)
    int64_t n;
    int32_t nt;
    int64_t r0, r1;           // rows present at src
    float *y;                 // tile-packed destination
    unsigned long long *bad;
    unsigned *err;
};
cudaError_t launch_ingest(const IngestArgs &a, cudaStream_t s);

// Locations in: src (N x D, f32/f64) -> the state x (zero padded to n_pad)
// and, on the FP32C path, the split layouts (quantum from *split).
cudaError_t launch_set_x(const void *src, bool src_f64, int64_t n, int64_t n_pad, int d, bool fp64, const XState &xs,
                         unsigned *err, cudaStream_t s);
// Recompute the split layouts of the FP32C path from x (after a quantum change).
cudaError_t launch_resplit(const XState &xs, int64_t n_pad, int d, cudaStream_t s);
// Re-pack the tile-packed Y for a new slot order: the pair at new slots
// (s, t) comes from old slots (map[s], map[t]) of old_y (only s < t < n is
// stored; every other element is written 0).
cudaError_t launch_repack(const float *old_y, float *new_y, const int32_t *map, int64_t n, int32_t nt, cudaStream_t s);
// Host: locality order of N points in D dimensions (recursive bisection of
// the widest coordinate, halves cut at multiples of 64 items): perm[s] is the
// item placed at slot s.
void locality_order(int64_t n, int d, const double *x, int32_t *perm);
// max |x| over the state (float bits into *out via atomicMax; *out must be 0).
cudaError_t launch_xmax(const void *x, bool fp64, int64_t count, unsigned *out, cudaStream_t s);
// Copy / convert an array between element types (device to device).
cudaError_t launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t count, cudaStream_t s);

// Cross-validation folds (section 2.4 of the paper).  Held-out pairs are
// marked in the tile-packed Y with a negative value (the pass masks them) and
// their y kept aside; tile_ho[t] = 1 for the tiles that hold one.
cudaError_t launch_ho_mark(float *y, const int64_t *off, int64_t count, float *ho_y, unsigned char *tile_ho,
                           cudaStream_t s);
cudaError_t launch_ho_restore(float *y, const int64_t *off, int64_t count, const float *ho_y, cudaStream_t s);
// Fold the predictive density of every held-out pair at the current state
// into per-pair running log-sum-exp accumulators (lse_m, lse_s); first = no
// earlier draw.
cudaError_t launch_lpd_accumulate(const void *x, bool fp64, int d, const int2 *pairs, const float *ho_y,
                                  int64_t count, double sigma, bool first, double *lse_m, double *lse_s,
                                  unsigned *err, cudaStream_t s);
// lpd-hat = sum over pairs of lse_m + log(lse_s) - log(draws) into *out
// (fixed-order reduction; part holds kLpdParts doubles).
constexpr int kLpdParts = 1024;
cudaError_t launch_lpd_sum(const double *lse_m, const double *lse_s, int64_t count, double draws, double *part,
                           double *out, cudaStream_t s);

// Sharded evaluation (section 2.5: the pairwise sum split over workers, the
// partial sums reduced).  pack: this shard's partials {L, dL/dsigma, sum r,
// gradient [N][D] (item order)} into send (FP64); combine: the n_ranks
// partial vectors of recv (rank-major, `count` doubles each) summed in rank
// order into the context's scalars and gradient (FP32C: (hi, lo) pairs).
cudaError_t launch_shard_pack(const double *scal, const void *grad, bool fp64, int64_t nd, double *send,
                              cudaStream_t s);
cudaError_t launch_shard_combine(const double *recv, int n_ranks, int64_t count, double *scal, void *grad, bool fp64,
                                 cudaStream_t s);

// Set the message mds_last_error(NULL) returns in the calling thread.
void set_thread_error(const char *fmt, ...);

// Bits B of the exact-difference split for D dimensions (see above).
__host__ __device__ inline int split_bits(int d) { return d <= 1 ? 12 : d <= 4 ? 11 : 10; }

// The split quantum for max |x| = m: q = 2^e, the smallest power of two with
// (2^(B-1) - 1) q >= 4 m (4x headroom for the moves of a trajectory).  The
// same function runs on the host (locations set by the caller) and on the
// device (growth during a trajectory), so both pick the same quantum for the
// same m.  False when q would leave [2^-100, 2^103] (x beyond FP32C range).
__host__ __device__ inline bool choose_split(float m, int d, Split &sp) {
    const double lim = static_cast<double>((1 << (split_bits(d) - 1)) - 1);
    const double v = (static_cast<double>(m) > 1e-30 ? static_cast<double>(m) : 1e-30) * 4.0 / lim;
    int e = 0;
    const double f = frexp(v, &e);          // v = f 2^e, f in [0.5, 1)
    const int ex = f == 0.5 ? e - 1 : e;    // ceil(log2 v)
    if (ex < -100 || ex > 103) return false;
    sp.q = ldexpf(1.0f, ex);
    sp.magic = ldexpf(1.5f, ex + 23);
    sp.bound = static_cast<float>(lim * ldexp(1.0, ex));
    sp.resplit = 0;
    return true;
}

// Raise the dynamic shared memory limit of `func` to at least `bytes` on the
// current device.  The attribute belongs to the device's context, so the
// largest value set so far is cached per (kernel, device ordinal) under a
// mutex: a second device gets its own call, and concurrent host threads do
// not race on the cache (defined in pair_kernel.cu).
cudaError_t raise_dyn_smem(const void *func, int bytes);

// Programmatic dependent launch.  The pair pass and the reduction alternate
// 2 L times per trajectory; launched with launch_pdl, a kernel may become
// resident while the previous kernel of the stream is still draining, runs
// its prologue (barrier set-up, prefetch of the constant Y tiles), and must
// call pdl_wait() before it reads anything the previous kernel writes or
// writes anything the previous kernel reads.  pdl_wait() returns at once in
// a kernel launched without the attribute.  pdl_trigger() lets the next
// kernel be scheduled once every CTA of this one has called it (or exited);
// each kernel that calls it is itself only launched after all CTAs of its
// predecessor are resident, so early-resident waiting CTAs never hold back
// a CTA that still has to start.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" : : : "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" : : : "memory"); }
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t launch_maybe_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t s, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    return launch_maybe_pdl(true, kernel, grid, block, smem, s, args...);
}

}  // namespace mds
