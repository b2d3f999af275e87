// Host runtime of the C ABI declared in include/mds.h: argument checks,
// device state, the tile/strip work list, the strip-length autotuner, kernel
// launches, CUDA-graph capture of HMC iterations, and error reporting.
#include "mds.h"

#include <cuda_runtime.h>
#include <dlfcn.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mds_internal.h"
#include "mills_ratio_coeffs.h"
#include "tree_plan.h"

using namespace mds;

namespace {

thread_local std::string g_create_error = "no error";

// Shapes of the FP32C pair pass (mds_ctx::pass_kind).
constexpr int kPassStrips = 0;
constexpr int kPassChunks = 1;
// Shape kind of the tuner and of mds_set_pass_shape for the chunked pass in
// its grouped form (pass_kind kPassChunks with chunk_grouped set).
constexpr int kPassChunksSM = MDS_PASS_SM_CHUNKS;

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct mds_ctx {
    int64_t n = 0;
    int32_t d = 0;
    bool fp64 = false;
    int device = 0;
    int sm_count = 0;
    std::string device_name;
    int64_t nt = 0;
    int64_t n_pad = 0;
    int64_t tiles = 0;
    int32_t strip = 0;        // in use (strip pass)
    int32_t strip_req = 0;    // 0 = autotune
    int32_t n_strips = 0;     // CTAs of the pair pass (strips, or chunks of the chunked pass)
    int32_t n_scal_parts = 0; // scalar partial records the pass writes
    int32_t n_row_slots = 0;
    // the FP32C pass's shape: kPassStrips (one CTA per strip of `strip` tiles)
    // or kPassChunks (chunk_mult chunks per resident chunk slot, one group of
    // four warps each: one CTA per chunk, or with chunk_grouped one CTA per
    // SM holding pair_chunk_groups(d) of them)
    int32_t pass_kind = 0;
    int32_t chunk_mult = 0;       // in use (chunked pass)
    bool chunk_grouped = false;   // in use (chunked pass)
    bool chunk_long_runs = false; // some chunk runs more than max_seg_tiles(d) tiles in one row block
    int32_t chunk_req = 0;        // > 0: chunked pass forced with this multiple
    bool chunk_grouped_req = false;
    Chunk *chunks = nullptr;
    size_t chunks_bytes = 0;
    std::vector<Chunk> chunks_host;
    unsigned char *far_tile = nullptr;       // [tiles][4] far column pairs of the last chunked pass
    std::vector<float> tile_cost;            // cost model of the chunking (empty: uniform)
    float2 *xcol2 = nullptr;                 // FP32C column layout of the chunked pass
    // shard (mds_set_shard): this context's pass covers the tiles [shard_t0,
    // shard_t1) of a pass split over shard_n ranks; Y holds only those tiles
    int32_t shard_n = 1, shard_rank = 0;
    int64_t shard_t0 = 0, shard_t1 = 0;      // set to [0, tiles) in create_ctx
    int64_t shard_pairs = 0;                 // pairs in the range
    mds_allgather_fn shard_fn = nullptr;
    void *shard_user = nullptr;
    int32_t shard_where = MDS_DEVICE;        // memory of the buffers the exchange gets
    double *shard_send = nullptr, *shard_recv = nullptr;    // device
    double *shard_hsend = nullptr, *shard_hrecv = nullptr;  // pinned host (exchange on the host)
    bool stamping = false;                   // pass spans measured with %globaltimer
    unsigned long long *stamps = nullptr;    // [2]
    double *pass_ns = nullptr;               // [2]: total ns, passes
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double sigma = 0.0;
    double lambda = 0.0;
    bool have_data = false, have_x = false, have_sigma = false, grad_valid = false;
    bool eval_unchecked = false;  // a start-point evaluation was queued without a wait (its error
                                  // bits come back with the next HMC read-back)
    uint64_t gen = 1;         // bumps whenever captured kernel arguments would change
    int start_grid = 0;

    // device buffers
    float *y = nullptr;
    void *x = nullptr, *p = nullptr, *x0 = nullptr;   // state (float on FP32C, double on FP64)
    float4 *xrow = nullptr, *xcol = nullptr;          // FP32C split layouts
    Split *split = nullptr;                           // FP32C split quantum (device)
    unsigned *xmax_bits = nullptr;                    // FP32C running max |x|
    void *grad = nullptr, *grad0 = nullptr;           // float2 (hi, lo) on FP32C, double on FP64
    void *col_part = nullptr;
    void *row_part = nullptr;
    size_t row_part_bytes = 0;
    void *scal_part = nullptr;
    size_t scal_part_bytes = 0;
    Strip *strips = nullptr;
    size_t strips_bytes = 0;
    int32_t *row_first = nullptr;
    double *scal = nullptr;
    int64_t *counters = nullptr;
    unsigned *err = nullptr;
    unsigned long long *bad = nullptr;
    double *e_start = nullptr, *e_end = nullptr;
    void *stage = nullptr;    // conversion staging (n_pad * D doubles)
    double *p_inj = nullptr;
    size_t p_inj_bytes = 0;
    double *u_inj = nullptr;
    size_t u_inj_bytes = 0;
    int32_t *acc_out = nullptr;
    double *dh_out = nullptr;
    size_t out_cap = 0;
    int64_t hmc_pending = 0;          // iterations queued since the last collect (results on the device)
    std::vector<int32_t> acc_spill;   // results moved to the host to make room (oldest first)
    std::vector<double> dh_spill;
    void *host_stage = nullptr;       // pinned host memory for the one read-back of a collect
    size_t host_stage_bytes = 0;

    // cross-validation fold (section 2.4): held-out pairs and the lpd-hat accumulators
    int64_t ho_count = 0;
    int64_t *ho_off = nullptr;         // their offsets in the tile-packed Y (marked y = -1 there)
    int2 *ho_pairs = nullptr;          // (i, j), i < j
    float *ho_y = nullptr;             // their y, set aside
    unsigned char *tile_ho = nullptr;  // [tiles] 1 where a tile holds a held-out pair
    double *lse_m = nullptr, *lse_s = nullptr;  // per pair running log-sum-exp of the densities
    double *lpd_part = nullptr;        // kLpdParts partials + the result
    int64_t lpd_draws = 0;

    // sigma updates (random walk on log sigma)
    int64_t sigma_iter = 0;            // updates drawn so far (Philox counter)
    double *sigma_draws = nullptr;     // device z, u of one call
    int64_t sigma_draws_cap = 0;

    // pair-pass timing (mds_set_profiling)
    bool profiling = false;
    std::vector<cudaEvent_t> prof_a, prof_b;
    int prof_used = 0;        // event pairs recorded since the last harvest
    int64_t prof_launches = 0;
    double prof_ms = 0.0;

    // graph cache (one HMC iteration)
    cudaGraphExec_t graph = nullptr;
    std::tuple<uint64_t, int, double, int, int, uint64_t, int> graph_key{};
    int graph_prof = 0;       // event pairs inside the captured graph

    bool y_owned = true;              // false for the chain contexts of a batch that share Y
    std::vector<Strip> strips_host;   // the strip list as uploaded (batched launches reuse it)

    // locality order (mds_reorder): slot s of the tile layouts (Y, split
    // locations, partial sums) holds item perm[s]; the state and every API
    // array stay in the caller's item order
    bool reordered = false;
    std::vector<int32_t> perm_h, inv_h;   // [n_pad], pads map to themselves
    int32_t *perm_d = nullptr, *inv_d = nullptr;
    double tail_z = 8.0;                  // Phi-term cut-off z_c (0: off)
    int32_t *far_part = nullptr;          // [strips][4 warps] far warp blocks of the last pass
    size_t far_part_bytes = 0;

    // phylogenetic Brownian-diffusion prior (mds_set_tree_prior)
    bool tree_on = false;
    TreeArgs tree{};                      // device pointers and constants (x set per launch)
    double *tree_grad0 = nullptr;         // its gradient at the trajectory start (restored on reject)
    cudaStream_t tree_stream = nullptr;   // the traversal runs here, beside the pair pass
    cudaEvent_t tree_fork = nullptr, tree_join = nullptr;
    int tree_pass_smem = 0;               // > 0: the pass's padded shared memory beside the traversal
    int64_t rw_iter = 0;                  // random-walk proposals drawn so far (Philox counter)
    std::vector<void *> tree_bufs;        // its device allocations


    std::string last_error = "no error";
};

namespace {

int fail(mds_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->last_error = buf;
    else
        g_create_error = buf;
    return code;
}

#define CU(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(c, MDS_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                      \
    } while (0)

#define CHECK(st)                        \
    do {                                 \
        int s_ = (st);                   \
        if (s_ != MDS_OK) return s_;     \
    } while (0)

// Fault injection for tests, from the environment: MDS_FAULT=alloc makes
// device allocations fail as out of memory, MDS_FAULT=nan plants a NaN in the
// scalar partials of an evaluation pass, MDS_FAULT=timeout runs a probe kernel
// before an evaluation pass whose bounded device-side wait runs out.  Each
// is active while the variable is set; nothing is injected into captured
// graphs.
bool fault_is(const char *kind) {
    const char *v = std::getenv("MDS_FAULT");
    return v && std::strcmp(v, kind) == 0;
}

int dev_alloc(mds_ctx *c, void **p, size_t bytes) {
    if (fault_is("alloc")) return fail(c, MDS_ERR_OOM, "cudaMalloc of %zu bytes failed (injected: MDS_FAULT=alloc)", bytes);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, MDS_ERR_OOM, "cudaMalloc of %zu bytes failed: out of device memory", bytes);
    }
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    return MDS_OK;
}

template <typename P>
int dev_alloc_t(mds_ctx *c, P **p, size_t bytes) {
    void *v = nullptr;
    int st = dev_alloc(c, &v, bytes);
    *p = static_cast<P *>(v);
    return st;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

size_t elem(const mds_ctx *c) { return c->fp64 ? sizeof(double) : sizeof(float); }
size_t grad_elem(const mds_ctx *c) { return c->fp64 ? sizeof(double) : sizeof(float2); }

XState xstate(const mds_ctx *c) {
    XState xs{};
    xs.x = c->x;
    xs.xrow = c->xrow;
    xs.xcol = c->xcol;
    xs.xcol2 = c->xcol2;
    xs.split = c->split;
    xs.xmax_bits = c->xmax_bits;
    xs.inv = c->reordered ? c->inv_d : nullptr;
    return xs;
}

int check_ctx(mds_ctx *c) {
    if (!c) return MDS_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return MDS_OK;
}

// Map device error bits to a status and message.
int err_status(mds_ctx *c, unsigned h, const char *what) {
    if (h & kErrTimeout) return fail(c, MDS_ERR_TIMEOUT, "%s: a device-side wait timed out", what);
    if (h & kErrBadArgs) return fail(c, MDS_ERR_CUDA, "%s: kernel argument check failed", what);
    if (h & kErrNonfinite) return fail(c, MDS_ERR_NONFINITE, "%s: non-finite result (NaN/Inf)", what);
    if (h & kErrRange) return fail(c, MDS_ERR_INVALID_ARG, "%s: locations moved beyond the FP32C range", what);
    if (h & kErrOverflow) return fail(c, MDS_ERR_STATE, "%s: HMC result buffer overflow", what);
    return fail(c, MDS_ERR_INVALID_ARG, "%s: invalid input value", what);
}

// Read and clear the device error word; map it to a status.
int check_device_err(mds_ctx *c, const char *what) {
    unsigned h = 0;
    CU(cudaMemcpyAsync(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h == 0) return MDS_OK;
    CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return err_status(c, h, what);
}

// ---------------------------------------------------------------- strips

int ensure_part_buffers(mds_ctx *c, size_t row_slots, size_t scal_parts, size_t far_parts);

int build_strips(mds_ctx *c, int strip) {
    const int64_t nt = c->nt;
    std::vector<Strip> v;
    std::vector<int32_t> first(nt + 1, 0);
    int32_t slot = 0;
    for (int64_t I = 0; I < nt; ++I) {
        first[I] = slot;
        // the row block's tiles within this context's range (all of them
        // unless the context is a shard)
        const int64_t td = tile_index(I, I, nt);
        const int64_t jlo = I + std::max<int64_t>(0, c->shard_t0 - td);
        const int64_t jhi = I + std::min<int64_t>(nt - I, c->shard_t1 - td);
        for (int64_t j0 = jlo; j0 < jhi; j0 += strip) {
            Strip s;
            s.I = static_cast<int32_t>(I);
            s.j0 = static_cast<int32_t>(j0);
            s.j1 = static_cast<int32_t>(std::min<int64_t>(jhi, j0 + strip));
            s.row_slot = slot++;
            v.push_back(s);
        }
    }
    first[nt] = slot;
    // largest strips first: blocks are dispatched roughly in index order, so
    // this approximates longest-processing-time-first scheduling; among
    // strips of one length, those that hold a diagonal tile (masked tiles and
    // the nearest pairs, which evaluate Phi) go first
    std::stable_sort(v.begin(), v.end(), [](const Strip &a, const Strip &b) {
        if (a.j1 - a.j0 != b.j1 - b.j0) return (a.j1 - a.j0) > (b.j1 - b.j0);
        return (a.j0 == a.I) && (b.j0 != b.I);
    });
    const size_t sb = v.size() * sizeof(Strip);
    if (sb > c->strips_bytes) {
        dev_free(c->strips);
        c->strips = nullptr;
        CHECK(dev_alloc_t(c, &c->strips, sb));
        c->strips_bytes = sb;
    }
    CHECK(ensure_part_buffers(c, static_cast<size_t>(slot), v.size(), v.size() * kPairWarps));
    c->strips_host = v;
    CU(cudaMemcpyAsync(c->strips, v.data(), sb, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->row_first, first.data(), (nt + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->n_strips = static_cast<int32_t>(v.size());
    c->n_scal_parts = c->n_strips;
    c->n_row_slots = slot;
    c->strip = strip;
    c->pass_kind = kPassStrips;
    c->chunk_mult = 0;
    c->gen++;
    return MDS_OK;
}

int ensure_part_buffers(mds_ctx *c, size_t row_slots, size_t scal_parts, size_t far_parts) {
    const size_t rb = row_slots * kTile * c->d * elem(c);
    if (rb > c->row_part_bytes) {
        dev_free(c->row_part);
        c->row_part = nullptr;
        c->row_part_bytes = 0;
        CHECK(dev_alloc(c, &c->row_part, rb));
        c->row_part_bytes = rb;
    }
    const size_t spb = scal_parts * kScalarParts * elem(c);
    if (spb > c->scal_part_bytes) {
        dev_free(c->scal_part);
        c->scal_part = nullptr;
        c->scal_part_bytes = 0;
        CHECK(dev_alloc(c, &c->scal_part, spb));
        c->scal_part_bytes = spb;
    }
    const size_t fpb = far_parts * sizeof(int32_t);
    if (fpb > c->far_part_bytes) {
        dev_free(c->far_part);
        c->far_part = nullptr;
        c->far_part_bytes = 0;
        CHECK(dev_alloc_t(c, &c->far_part, fpb));
        c->far_part_bytes = fpb;
    }
    return MDS_OK;
}

// Cost model of the chunking, in FP32 lane-operations per warp: a tile is 8
// warp blocks (64 rows x 8 columns; a warp takes two), 16 pairs per lane
// each, at 23 operations per pair for a far block (Phi terms skipped) and 36
// for the others (chunk_kernel.cu), plus about 70 per tile (column
// transposes, block tests, sums, the ring refill) and 150 where a row block
// starts (row sums out, row buffer, row box).
constexpr double kCostFar = 23.0, kCostNear = 36.0, kCostTile = 70.0, kCostSeg = 150.0;

// The chunked pass's work list: the tiles, in row-block order, cut into
// G = (SMs x resident CTAs of the pass) x mult chunks of equal estimated
// cost (c->tile_cost from the far counts of an earlier chunked pass, else
// every block counted near), one CTA each.
int build_chunks(mds_ctx *c, int mult, bool grouped) {
    // the tiles [T0, T0 + T) of this context (a shard's range, or all)
    const int64_t nt = c->nt, T0 = c->shard_t0, T = c->shard_t1 - c->shard_t0;
    int per_sm = pair_chunk_blocks_per_sm(c->d, grouped);
    if (per_sm < 1) per_sm = 1;
    // mult > 0: chunks per resident CTA slot; mult < 0: exactly -mult chunks
    const int64_t want = mult > 0 ? static_cast<int64_t>(c->sm_count) * per_sm * mult : -static_cast<int64_t>(mult);
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(T, want));
    if (T <= 0) {
        // a shard without tiles: no CTA, no partial slot
        std::vector<int32_t> zero(nt + 1, 0);
        CU(cudaMemcpyAsync(c->row_first, zero.data(), (nt + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        c->chunks_host.clear();
        c->n_strips = 0;
        c->n_scal_parts = 0;
        c->n_row_slots = 0;
        c->pass_kind = kPassChunks;
        c->chunk_mult = mult;
        c->chunk_grouped = grouped;
        c->strip = 0;
        c->gen++;
        return MDS_OK;
    }
    const bool have_cost = static_cast<int64_t>(c->tile_cost.size()) == c->tiles;
    // blocks of the first tile of the range
    int64_t Ib = 0;
    while (Ib + 1 < nt && tile_index(Ib + 1, Ib + 1, nt) <= T0) ++Ib;
    const int64_t Jb = Ib + (T0 - tile_index(Ib, Ib, nt));
    std::vector<double> pre(static_cast<size_t>(T) + 1, 0.0);
    {
        int64_t I = Ib, J = Jb;
        for (int64_t t = 0; t < T; ++t) {
            double cst = have_cost ? c->tile_cost[T0 + t] : kCostTile + 4.0 * 8.0 * kCostNear;
            if (J == I || t == 0) cst += kCostSeg;
            pre[t + 1] = pre[t] + cst;
            if (++J == nt) J = ++I;
        }
    }
    // out[0 .. parts]: the boundaries of `parts` pieces of [lo, hi) of equal
    // estimated cost, each of at least min_tiles tiles
    auto cut_range = [&](int64_t lo, int64_t hi, int64_t parts, int64_t min_tiles, int64_t *out) {
        out[0] = lo;
        out[parts] = hi;
        const double c0 = pre[lo], span = pre[hi] - pre[lo];
        for (int64_t g = 1; g < parts; ++g) {
            const double target = c0 + span * static_cast<double>(g) / static_cast<double>(parts);
            // first tile boundary whose prefix reaches the target
            int64_t b = std::lower_bound(pre.begin() + lo, pre.begin() + hi + 1, target) - pre.begin();
            if (b > lo && target - pre[b - 1] < pre[b] - target) --b;
            b = std::max(b, out[g - 1] + min_tiles);
            b = std::min(b, hi - min_tiles * (parts - g));
            out[g] = b;
        }
    };
    std::vector<int64_t> cut(static_cast<size_t>(G) + 1, 0);
    const int64_t groups = grouped ? pair_chunk_groups(c->d) : 1;
    if (groups > 1 && G % groups == 0 && T >= G) {
        // the grouped form: each SM's total decides the end of the pass (its
        // groups share it), so equal-cost pieces per CTA first, where a tile
        // is a smaller part of the share than of one chunk, then each piece
        // into its groups' chunks
        const int64_t P = G / groups;
        std::vector<int64_t> piece(static_cast<size_t>(P) + 1, 0);
        cut_range(0, T, P, groups, piece.data());
        for (int64_t p = 0; p < P; ++p) cut_range(piece[p], piece[p + 1], groups, 1, cut.data() + p * groups);
    } else {
        cut_range(0, T, G, 1, cut.data());
    }
    // blocks of every tile boundary, segments, the first segment of each row block
    std::vector<Chunk> v(static_cast<size_t>(G));
    std::vector<int32_t> first(nt + 1, -1);
    int64_t t = 0, I = Ib, J = Jb;
    int32_t seg = 0;
    bool long_runs = false;
    for (int64_t g = 0; g < G; ++g) {
        while (t < cut[g]) {  // advance (I, J) to tile cut[g] of the range
            if (++J == nt) J = ++I;
            ++t;
        }
        Chunk ch{};
        ch.t0 = T0 + cut[g];
        ch.t1 = T0 + cut[g + 1];
        ch.I0 = static_cast<int32_t>(I);
        ch.J0 = static_cast<int32_t>(J);
        // row block of the last tile: the largest I with tile_index(I, I) <= t1 - 1
        int64_t Il = I;
        while (Il + 1 < nt && tile_index(Il + 1, Il + 1, nt) <= ch.t1 - 1) ++Il;
        ch.I1 = static_cast<int32_t>(Il);
        // segments: the chunk's run in each row block, cut every max_seg_tiles
        ch.seg0 = seg;
        const int64_t cap = max_seg_tiles(c->d);
        for (int64_t r = I; r <= Il; ++r) {
            const int64_t r0 = tile_index(r, r, nt);
            const int64_t len = std::min<int64_t>(ch.t1, r0 + nt - r) - std::max<int64_t>(ch.t0, r0);
            if (first[r] < 0) first[r] = 4 * seg;
            seg += static_cast<int32_t>((len + cap - 1) / cap);
            long_runs = long_runs || len > cap;
        }
        v[g] = ch;
    }
    first[nt] = 4 * seg;
    // row blocks outside the range (a shard) have no slots
    for (int64_t r = nt - 1; r >= 0; --r)
        if (first[r] < 0) first[r] = first[r + 1];
    CHECK(ensure_part_buffers(c, static_cast<size_t>(4) * seg, static_cast<size_t>(4 * G), static_cast<size_t>(4 * G)));
    const size_t cb = v.size() * sizeof(Chunk);
    if (cb > c->chunks_bytes) {
        dev_free(c->chunks);
        c->chunks = nullptr;
        c->chunks_bytes = 0;
        CHECK(dev_alloc_t(c, &c->chunks, cb));
        c->chunks_bytes = cb;
    }
    c->chunks_host = v;
    CU(cudaMemcpyAsync(c->chunks, v.data(), cb, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->row_first, first.data(), (nt + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->n_strips = static_cast<int32_t>(G);
    c->n_scal_parts = static_cast<int32_t>(4 * G);
    c->n_row_slots = 4 * seg;
    c->pass_kind = kPassChunks;
    c->chunk_mult = mult;
    c->chunk_grouped = grouped;
    c->chunk_long_runs = long_runs;
    c->strip = 0;
    c->gen++;
    return MDS_OK;
}

// Pairs i < j < n of the tiles [t0, t1) (row-block order).
int64_t range_pairs(int64_t n, int64_t nt, int64_t t0, int64_t t1) {
    int64_t m = 0;
    for (int64_t I = 0; I < nt; ++I) {
        const int64_t td = tile_index(I, I, nt);
        const int64_t jlo = I + std::max<int64_t>(0, t0 - td);
        const int64_t jhi = I + std::min<int64_t>(nt - I, t1 - td);
        const int64_t r = std::min<int64_t>(kTile, n - I * kTile);
        for (int64_t J = jlo; J < jhi; ++J) {
            const int64_t cc = std::min<int64_t>(kTile, n - J * kTile);
            m += J == I ? r * (r - 1) / 2 : r * cc;
        }
    }
    return m;
}

// The shard ranges: tile boundaries b[0..g] with b[r] the first tile whose
// prefix of pairs reaches r M / g (so every range holds M / g pairs to within
// one tile).
std::vector<int64_t> shard_bounds(int64_t n, int32_t g) {
    const int64_t nt = (n + kTile - 1) / kTile, T = tile_count(nt);
    const int64_t M = n * (n - 1) / 2;
    std::vector<int64_t> b(static_cast<size_t>(g) + 1, T);
    b[0] = 0;
    int64_t t = 0, pre = 0;
    int32_t r = 1;
    for (int64_t I = 0; I < nt && r < g; ++I) {
        const int64_t ri = std::min<int64_t>(kTile, n - I * kTile);
        for (int64_t J = I; J < nt && r < g; ++J) {
            // before tile t: pre pairs; assign every rank whose target is reached
            while (r < g && static_cast<long double>(pre) >= static_cast<long double>(M) * r / g) b[r++] = t;
            const int64_t cc = std::min<int64_t>(kTile, n - J * kTile);
            pre += J == I ? ri * (ri - 1) / 2 : ri * cc;
            ++t;
        }
    }
    while (r < g) b[r++] = T;
    return b;
}

// One exchange of a sharded evaluation: this rank's partials (the scalars
// and gradient its reduction just wrote) out, every rank's in, summed in rank
// order into the scalars and the gradient.
int shard_exchange(mds_ctx *c, cudaStream_t s) {
    const int64_t nd = c->n * c->d, count = 3 + nd;
    cudaError_t e = launch_shard_pack(c->scal, c->grad, c->fp64, nd, c->shard_send, s);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "shard pack: %s", cudaGetErrorString(e));
    int rc = 0;
    if (c->shard_where == MDS_DEVICE) {
        CU(cudaStreamSynchronize(s));
        rc = c->shard_fn(c->shard_user, c->shard_send, c->shard_recv, count, MDS_DEVICE);
    } else {
        CU(cudaMemcpyAsync(c->shard_hsend, c->shard_send, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        rc = c->shard_fn(c->shard_user, c->shard_hsend, c->shard_hrecv, count, MDS_HOST);
        if (rc == 0)
            CU(cudaMemcpyAsync(c->shard_recv, c->shard_hrecv, static_cast<size_t>(c->shard_n) * count * sizeof(double),
                               cudaMemcpyHostToDevice, s));
    }
    if (rc != 0) return fail(c, MDS_ERR_EXCHANGE, "the all-gather of the shard partials returned %d", rc);
    e = launch_shard_combine(c->shard_recv, c->shard_n, count, c->scal, c->grad, c->fp64, s);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "shard combine: %s", cudaGetErrorString(e));
    return MDS_OK;
}

bool sharded(const mds_ctx *c) { return c->shard_n > 1; }

// Per-tile costs from the far counts of the last chunked pass.
int read_tile_costs(mds_ctx *c) {
    std::vector<unsigned char> f(static_cast<size_t>(c->tiles) * kPairWarps);
    CU(cudaMemcpyAsync(f.data(), c->far_tile, f.size(), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->tile_cost.assign(static_cast<size_t>(c->tiles), 0.f);
    for (int64_t t = 0; t < c->tiles; ++t) {
        int far = 0;
        for (int w = 0; w < kPairWarps; ++w) far += f[static_cast<size_t>(t) * kPairWarps + w];
        far = std::min(far, 8);
        c->tile_cost[t] = static_cast<float>(kCostTile + 4.0 * (far * kCostFar + (8 - far) * kCostNear));
    }
    return MDS_OK;
}

// Longest-processing-time-first order of the strips from the far-block
// counts of the last FP32C pass: a strip costs about its tiles' warp blocks,
// a far block (Phi terms skipped) 25/38 of one that evaluates Phi.  Only the
// assignment of strips to CTAs changes (results stay within tolerance; the
// scalar partials are summed in the new order).
int order_strips_by_cost(mds_ctx *c) {
    if (c->fp64 || c->n_strips <= 0) return MDS_OK;
    if (c->pass_kind == kPassChunks) {
        // the chunked pass: cut the tiles again by the measured far counts
        CHECK(read_tile_costs(c));
        CHECK(build_chunks(c, c->chunk_mult, c->chunk_grouped));
        c->grad_valid = false;
        return MDS_OK;
    }
    std::vector<int32_t> parts(static_cast<size_t>(c->n_strips) * kPairWarps);
    CU(cudaMemcpyAsync(parts.data(), c->far_part, parts.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    const int n = c->n_strips;
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) {
        const Strip &st = c->strips_host[k];
        int32_t far = 0;
        for (int w = 0; w < kPairWarps; ++w) far += parts[static_cast<size_t>(k) * kPairWarps + w];
        const double blocks = static_cast<double>(st.j1 - st.j0) * kPairWarps * 2;
        cost[k] = (blocks - far) * 38.0 + far * 25.0;
    }
    std::vector<int> idx(n);
    for (int k = 0; k < n; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<Strip> v(n);
    for (int k = 0; k < n; ++k) v[k] = c->strips_host[idx[k]];
    c->strips_host = v;
    CU(cudaMemcpyAsync(c->strips, v.data(), v.size() * sizeof(Strip), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->grad_valid = false;
    c->gen++;
    return MDS_OK;
}

constexpr int kMaxStrip = 16;  // bounds the FP32 row sums of a lane (<= 64 terms, 4 columns a tile)

// Choose the split quantum from max |x| of locations the caller sets and
// rewrite the split layouts.  During trajectories the end-of-trajectory
// reduction grows the quantum on the device by the same rule (choose_split),
// so no call that runs passes has to read max |x| back.
int set_split_from_xmax(mds_ctx *c) {
    if (c->fp64) return MDS_OK;
    unsigned bits = 0;
    CU(cudaMemcpyAsync(&bits, c->xmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    float m;
    std::memcpy(&m, &bits, sizeof(m));
    Split sp;
    if (!choose_split(m, c->d, sp))
        return fail(c, MDS_ERR_INVALID_ARG, "locations out of the FP32C range (max |x| = %g)", m);
    CU(cudaMemcpyAsync(c->split, &sp, sizeof(sp), cudaMemcpyHostToDevice, c->stream));
    cudaError_t e = launch_resplit(xstate(c), c->n_pad, c->d, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "resplit: %s", cudaGetErrorString(e));
    CU(cudaStreamSynchronize(c->stream));
    return MDS_OK;
}

// --------------------------------------------------------------- passes

PairArgs pair_args(const mds_ctx *c) {
    PairArgs a{};
    a.y = c->y;
    a.y_t0 = c->shard_t0;
    a.xrow = c->xrow;
    a.xcol = c->xcol;
    a.x64 = c->fp64 ? static_cast<const double *>(c->x) : nullptr;
    a.strips = c->strips;
    a.n_strips = c->n_strips;
    a.nt = static_cast<int32_t>(c->nt);
    a.n = c->n;
    a.row_part = c->row_part;
    a.col_part = c->col_part;
    a.scal_part = c->scal_part;
    a.tile_ho = c->ho_count > 0 ? c->tile_ho : nullptr;
    a.perm = c->reordered ? c->perm_d : nullptr;
    a.far_part = c->far_part;
    a.err = c->err;
    a.stamps = c->stamping ? c->stamps : nullptr;
    if (!c->fp64 && c->pass_kind == kPassChunks) {
        a.chunks = c->chunks;
        a.xcol2 = c->xcol2;
        a.far_tile = c->far_tile;
        a.long_runs = c->chunk_long_runs ? 1 : 0;
    }
    const double s = c->sigma;
    // far warp blocks: every pair at z >= z_c (the squared-distance bound in
    // FP32; an overflow to +inf only turns the shortcut off)
    a.far_d2 = c->tail_z > 0.0 ? static_cast<float>((c->tail_z * s) * (c->tail_z * s)) : INFINITY;
    const double inv_sqrt_2pi = 0.39894228040143267794;
    double sk = 1.0;
    for (int k = 0; k < 4; ++k) {
        const float pv = static_cast<float>(-kMillsP[k] * inv_sqrt_2pi / sk);
        const float dv = static_cast<float>(kMillsD[k] / sk);
        a.mp[k] = make_float2(pv, pv);
        a.md[k] = make_float2(dv, dv);
        sk *= s;
    }
    const float cphi = static_cast<float>(-1.4426950408889634074 / (2.0 * s * s));
    const float nis2 = static_cast<float>(-1.0 / (s * s));
    const float mc = static_cast<float>(inv_sqrt_2pi / s);
    a.c_phi = make_float2(cphi, cphi);
    a.neg_inv_s2 = make_float2(nis2, nis2);
    a.m_coef = make_float2(mc, mc);
    const float cm2 = static_cast<float>(-s * inv_sqrt_2pi);
    a.c_m2 = make_float2(cm2, cm2);
    a.sigma = s;
    a.inv_sigma = 1.0 / s;
    a.inv_s2 = 1.0 / (s * s);
    return a;
}

ReduceArgs reduce_args(const mds_ctx *c, int mode, double eps) {
    ReduceArgs r{};
    r.row_part = c->row_part;
    r.col_part = c->col_part;
    r.scal_part = c->scal_part;
    r.row_first_slot = c->row_first;
    r.perm = c->reordered ? c->perm_d : nullptr;
    r.n_strips = c->n_scal_parts;
    r.part_scale = (!c->fp64 && c->pass_kind == kPassChunks) ? -1.0 / (c->sigma * c->sigma) : 1.0;
    {
        const float h = static_cast<float>(r.part_scale);
        r.part_scale_df = make_float2(h, static_cast<float>(r.part_scale - static_cast<double>(h)));
    }
    r.stamps = c->stamping ? c->stamps : nullptr;
    r.pass_ns = c->pass_ns;
    r.nt = static_cast<int32_t>(c->nt);
    r.n = c->n;
    r.d = c->d;
    r.mode = mode;
    r.fp64 = c->fp64;
    r.sigma = c->sigma;
    r.log_sigma = std::log(c->sigma);
    r.inv_sigma = 1.0 / c->sigma;
    r.m_pairs = static_cast<double>(c->shard_pairs) - static_cast<double>(c->ho_count);
    r.lambda = c->lambda;
    r.eps = eps;
    r.grad = static_cast<double *>(c->grad);
    r.scal = c->scal;
    r.xs = xstate(c);
    r.p = c->p;
    r.energy_part = c->e_end;
    r.prior_grad = c->tree_on ? c->tree.grad : nullptr;
    if (c->tree_on) {
        r.tree_part = c->tree.part;
        r.n_tree_parts = (c->tree.n_trees + (c->tree.n_lone > 0 ? 1 : 0)) * c->tree.cluster;
        r.tree_const = c->tree.const_term;
    }
    r.err = c->err;
    return r;
}

int record_prof(mds_ctx *c, cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        CU(cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
    else
        CU(cudaEventRecord(ev, s));
    return MDS_OK;
}

// Add the elapsed times of the event pairs recorded since the last harvest
// (their work must have completed).
int harvest_prof(mds_ctx *c) {
    for (int k = 0; k < c->prof_used; ++k) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, c->prof_a[k], c->prof_b[k]));
        c->prof_ms += ms;
        c->prof_launches++;
    }
    c->prof_used = 0;
    return MDS_OK;
}

int enqueue_pass(mds_ctx *c, int mode, double eps, cudaStream_t s, bool plant_nan = false) {
    PairArgs a = pair_args(c);
    const int pk = c->prof_used;
    if (c->profiling) {
        while (static_cast<int>(c->prof_a.size()) <= pk) {
            cudaEvent_t ea, eb;
            CU(cudaEventCreate(&ea));
            CU(cudaEventCreate(&eb));
            c->prof_a.push_back(ea);
            c->prof_b.push_back(eb);
        }
        CHECK(record_prof(c, c->prof_a[pk], s));
    }
    cudaError_t e = cudaSuccess;
    if (c->tree_on) {
        // the tree prior at the same x (for the kicks and the energies of
        // HMC) on its own stream, concurrent with the pair pass; the reduction
        // waits for both (a fork and a join, also inside captured graphs)
        TreeArgs ta = c->tree;
        ta.x = c->x;
        ta.x_f64 = c->fp64;
        ta.out = nullptr;  // the reduction's scalar CTA adds the parts when it needs log p
        e = cudaEventRecord(c->tree_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->tree_stream, c->tree_fork, 0);
        if (e == cudaSuccess) e = launch_tree_prior(ta, c->d, c->tree_stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->tree_join, c->tree_stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "tree prior launch: %s", cudaGetErrorString(e));
    }
    // With a tree prior, launched early by PDL the pass's CTAs would hold
    // every SM before the traversal's clusters could be placed.  So either
    // the FP32C pass keeps PDL with its shared memory padded to leave room
    // for one traversal CTA beside three pass CTAs on every SM (tree_pass_smem,
    // chosen when the tree prior is set), or it is launched without PDL and
    // becomes eligible when the traversal does.
    const bool capped = c->tree_on && !c->fp64 && c->tree_pass_smem > 0;
    const bool pdl = !c->tree_on || capped;
    if (c->fp64)
        e = launch_pair_pass_f64(a, c->d, s, pdl);
    else if (c->pass_kind == kPassChunks)
        // the grouped form leaves no room for a traversal CTA: with a tree
        // prior the same chunks run one per CTA
        e = launch_pair_chunks_f32(a, c->d, s, pdl, capped ? c->tree_pass_smem : 0, c->chunk_grouped && !c->tree_on);
    else
        e = launch_pair_pass_f32(a, c->d, s, pdl, capped ? c->tree_pass_smem : 0);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "pair pass launch: %s", cudaGetErrorString(e));
    if (c->tree_on) {
        e = cudaStreamWaitEvent(s, c->tree_join, 0);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "tree prior join: %s", cudaGetErrorString(e));
    }
    if (plant_nan) {
        // fault injection: the first strip's sum of squared residuals is NaN
        static const double nan64 = std::nan("");
        static const float nan32 = std::nanf("");
        e = cudaMemcpyAsync(c->scal_part, c->fp64 ? static_cast<const void *>(&nan64) : static_cast<const void *>(&nan32),
                            elem(c), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "fault injection: %s", cudaGetErrorString(e));
    }
    if (c->profiling) {
        CHECK(record_prof(c, c->prof_b[pk], s));
        c->prof_used = pk + 1;
    }
    if (sharded(c)) {
        // this rank's partials (an evaluation-mode reduction), the exchange,
        // then the leapfrog update with the combined gradient
        ReduceArgs r = reduce_args(c, kModeEval, 0.0);
        e = launch_reduce(r, s);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "reduce launch: %s", cudaGetErrorString(e));
        CHECK(shard_exchange(c, s));
        if (mode != kModeEval) {
            ReduceArgs u = reduce_args(c, mode, eps);
            u.use_grad = true;
            u.stamps = nullptr;
            e = launch_reduce(u, s);
            if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "update launch: %s", cudaGetErrorString(e));
        }
        return MDS_OK;
    }
    ReduceArgs r = reduce_args(c, mode, eps);
    e = launch_reduce(r, s);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "reduce launch: %s", cudaGetErrorString(e));
    return MDS_OK;
}

int ready(mds_ctx *c) {
    if (!c->have_data) return fail(c, MDS_ERR_STATE, "no data: call mds_set_data first");
    if (!c->have_x) return fail(c, MDS_ERR_STATE, "no locations: call mds_set_locations first");
    if (!c->have_sigma) return fail(c, MDS_ERR_STATE, "no sigma: call mds_set_sigma first");
    return MDS_OK;
}

// ------------------------------------------------------------ autotuner
//
// The pass's shape (strip pass with S tiles per strip, or chunked pass with
// m chunks per resident CTA slot) is chosen by timing candidates, once per
// (GPU name, N, D, precision, item order).  The choice is kept in memory and
// in a text file, so that later processes on the same machine reuse it: the
// file named by MDS_TUNE_CACHE, else tune_cache.txt beside this library (one
// line per key, tab-separated: GPU name, N, D, precision, order, kind, param,
// milliseconds per pass).  MDS_STRIP or MDS_CHUNKS in the environment, or
// mds_set_strip / mds_set_pass_shape, force a shape.

struct TuneKey {
    std::string gpu;
    int64_t n;
    int d;
    bool fp64;
    bool reordered;
    bool operator<(const TuneKey &o) const {
        return std::tie(gpu, n, d, fp64, reordered) < std::tie(o.gpu, o.n, o.d, o.fp64, o.reordered);
    }
};
struct TuneVal {
    int kind;
    int param;
    double ms;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_file() {
    if (const char *env = getenv("MDS_TUNE_CACHE")) return env;
    Dl_info info{};
    if (dladdr(reinterpret_cast<const void *>(&mds_create), &info) && info.dli_fname) {
        std::string f = info.dli_fname;
        const size_t k = f.find_last_of('/');
        return (k == std::string::npos ? std::string(".") : f.substr(0, k)) + "/tune_cache.txt";
    }
    return "";
}

// Read the file into the cache (caller holds g_tune_mu).
void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_file();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        std::vector<std::string> fld;
        std::string cur;
        for (const char *p = line; *p && *p != '\n'; ++p) {
            if (*p == '\t') {
                fld.push_back(cur);
                cur.clear();
            } else {
                cur.push_back(*p);
            }
        }
        fld.push_back(cur);
        if (fld.size() != 8) continue;
        TuneKey k{fld[0], atoll(fld[1].c_str()), atoi(fld[2].c_str()), fld[3] == "fp64", fld[4] == "locality"};
        TuneVal v{atoi(fld[5].c_str()), atoi(fld[6].c_str()), atof(fld[7].c_str())};
        // chunked: param chunks per slot (1..8), or for kPassChunks minus an
        // exact chunk count
        if ((v.kind == kPassStrips && v.param >= 1 && v.param <= kMaxStrip) ||
            ((v.kind == kPassChunks || v.kind == kPassChunksSM) && v.param >= 1 && v.param <= 8) ||
            (v.kind == kPassChunks && v.param < 0 && v.param >= -(1 << 26)))
            g_tune_cache[k] = v;
    }
    fclose(f);
}

// Write the cache back (caller holds g_tune_mu): a temporary file, then a rename.
void tune_save() {
    const std::string path = tune_file();
    if (path.empty()) return;
    const std::string tmp = path + "." + std::to_string(static_cast<long long>(getpid())) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto &kv : g_tune_cache)
        fprintf(f, "%s\t%lld\t%d\t%s\t%s\t%d\t%d\t%.6f\n", kv.first.gpu.c_str(), static_cast<long long>(kv.first.n),
                kv.first.d, kv.first.fp64 ? "fp64" : "fp32c", kv.first.reordered ? "locality" : "caller",
                kv.second.kind, kv.second.param, kv.second.ms);
    const bool ok = fclose(f) == 0;
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

int apply_shape(mds_ctx *c, int kind, int param) {
    if (kind == kPassChunks || kind == kPassChunksSM) {
        const bool grouped = kind == kPassChunksSM;
        if (c->pass_kind != kPassChunks || c->chunk_mult != param || c->chunk_grouped != grouped)
            CHECK(build_chunks(c, param, grouped));
    } else if (c->pass_kind != kPassStrips || c->strip != param) {
        CHECK(build_strips(c, param));
    }
    return MDS_OK;
}

// Mean milliseconds of `reps` passes (with their reductions) after one warm-up.
int time_shape(mds_ctx *c, int reps, float *ms) {
    CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
    CU(cudaEventRecord(c->ev0, c->stream));
    for (int w = 0; w < reps; ++w) CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
    CU(cudaEventRecord(c->ev1, c->stream));
    CU(cudaEventSynchronize(c->ev1));
    CU(cudaEventElapsedTime(ms, c->ev0, c->ev1));
    *ms /= static_cast<float>(reps);
    return MDS_OK;
}

int autotune(mds_ctx *c) {
    if (sharded(c)) {
        // every rank must make the same passes (each is a collective): a
        // fixed shape, no timing and no counted pass
        if (c->fp64 || c->strip_req > 0) return apply_shape(c, kPassStrips, c->strip_req > 0 ? c->strip_req : 2);
        return apply_shape(c, kPassChunks, c->chunk_req != 0 ? c->chunk_req : 1);
    }
    if (c->strip_req > 0) return apply_shape(c, kPassStrips, c->strip_req);
    if (c->chunk_req != 0 && !c->fp64) {
        CHECK(apply_shape(c, c->chunk_grouped_req ? kPassChunksSM : kPassChunks, c->chunk_req));
        if (c->tile_cost.empty()) {
            // cut by measured costs: one counted pass, then the chunks again
            CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
            CHECK(check_device_err(c, "chunk costs"));
            CHECK(read_tile_costs(c));
            CHECK(build_chunks(c, c->chunk_req, c->chunk_grouped_req));
        }
        return MDS_OK;
    }
    if (const char *env = getenv("MDS_STRIP")) {
        const int s = atoi(env);
        if (s > 0) return apply_shape(c, kPassStrips, std::min(s, kMaxStrip));
    }
    if (const char *env = getenv("MDS_CHUNKS")) {
        const int m = atoi(env);
        if (m > 0 && !c->fp64) return apply_shape(c, kPassChunks, std::min(m, 8));
    }
    const TuneKey key{c->device_name, c->n, static_cast<int>(c->d), c->fp64, c->reordered};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            CHECK(apply_shape(c, it->second.kind, it->second.param));
            if (it->second.kind != kPassStrips && c->tile_cost.empty()) {
                // cut by measured costs: one counted pass, then the chunks again
                CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
                CHECK(check_device_err(c, "autotune"));
                CHECK(read_tile_costs(c));
                CHECK(build_chunks(c, it->second.param, it->second.kind == kPassChunksSM));
            }
            return MDS_OK;
        }
    }
    std::vector<std::pair<int, int>> cands;
    for (int s : {1, 2, 3, 4, 6, 8, 12, 16}) {
        if (s > kMaxStrip || s > c->nt) continue;
        const int64_t strips_est = (c->tiles + s - 1) / s;
        // keep enough CTAs for every SM, unless the problem is tiny anyway
        if (!cands.empty() && strips_est < 2 * c->sm_count) continue;
        cands.emplace_back(kPassStrips, s);
    }
    if (cands.empty()) cands.emplace_back(kPassStrips, 1);
    if (!c->fp64 && c->tiles >= 2) {
        const int per_sm = std::max(1, pair_chunk_blocks_per_sm(c->d));
        // more chunks per slot also keep every chunk's row-block runs within
        // max_seg_tiles at large N, where the uncut loop is the faster build
        for (int m : {1, 2, 3, 4, 6})
            if (static_cast<int64_t>(c->sm_count) * per_sm * m <= c->tiles || m == 1) cands.emplace_back(kPassChunks, m);
        // where even 6 chunks per slot run longer than the segment cut in a row
        // block: enough chunks (0.8 of the cut on average) for the uncut loop
        const int64_t cut = max_seg_tiles(c->d);
        const int64_t uncut = (c->tiles * 5 + 4 * cut - 1) / (4 * cut);
        if (uncut > static_cast<int64_t>(c->sm_count) * per_sm * 6 && uncut <= (1 << 26))
            cands.emplace_back(kPassChunks, -static_cast<int>(uncut));
        // the grouped form (not beside a tree prior's traversal, which it
        // leaves no room for)
        const int per_sm_g = pair_chunk_blocks_per_sm(c->d, true);
        if (!c->tree_on && per_sm_g >= 1)
            for (int m : {1, 2, 3})
                if (static_cast<int64_t>(c->sm_count) * per_sm_g * m <= c->tiles || m == 1)
                    cands.emplace_back(kPassChunksSM, m);
    }
    std::pair<int, int> best = cands[0];
    float best_ms = 1e30f;
    const bool prof = c->profiling;
    c->profiling = false;
    if (cands.size() > 1) {
        for (const auto &cd : cands) {
            CHECK(apply_shape(c, cd.first, cd.second));
            if (cd.first != kPassStrips) {
                // one counted pass, then cut by its far counts
                CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
                CHECK(read_tile_costs(c));
                CHECK(build_chunks(c, cd.second, cd.first == kPassChunksSM));
            }
            float ms = 0.f;
            CHECK(time_shape(c, 5, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = cd;
            }
        }
        CHECK(check_device_err(c, "autotune"));
    }
    c->profiling = prof;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = TuneVal{best.first, best.second, static_cast<double>(best_ms)};
        if (cands.size() > 1) tune_save();
    }
    CHECK(apply_shape(c, best.first, best.second));
    return MDS_OK;
}

// Evaluate at the current x (gradient + scalars) and wait.
int evaluate(mds_ctx *c) {
    CHECK(ready(c));
    CHECK(autotune(c));
    if (fault_is("timeout")) {
        cudaError_t e = launch_wait_probe(c->err, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "wait probe: %s", cudaGetErrorString(e));
    }
    CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream, fault_is("nan")));
    CU(cudaGetLastError());
    CHECK(check_device_err(c, "evaluation"));
    if (c->profiling) CHECK(harvest_prof(c));
    c->grad_valid = true;
    return MDS_OK;
}

// The gradient and L at a new start point of HMC, queued ahead of the
// trajectories without a wait: the evaluation's error bits reach the host
// with the read-back of the HMC results.  With pass profiling or an injected
// fault the evaluation waits and checks as a plain evaluation does.
int queue_start_eval(mds_ctx *c) {
    CHECK(autotune(c));
    if (c->grad_valid) return MDS_OK;
    if (c->profiling || std::getenv("MDS_FAULT")) return evaluate(c);
    CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
    CU(cudaGetLastError());
    c->grad_valid = true;
    c->eval_unchecked = true;
    return MDS_OK;
}

// A queued start-point evaluation followed by no iteration: check it now.
int finish_start_eval(mds_ctx *c, const char *what) {
    if (!c->eval_unchecked) return MDS_OK;
    c->eval_unchecked = false;
    const int st = check_device_err(c, what);
    if (st != MDS_OK) c->grad_valid = false;
    return st;
}

// src_kind: 0 f32, 1 f64, 2 float2 (hi, lo) pairs
int copy_out(mds_ctx *c, const void *dev_src, int src_kind, void *dst, int dtype, int where, int64_t count) {
    const bool dst_f64 = dtype == MDS_F64;
    const size_t eb = dst_f64 ? 8 : 4;
    const int64_t cnt = src_kind == 2 ? -count : count;
    if (where == MDS_DEVICE) {
        cudaError_t e = launch_convert(dev_src, src_kind == 1, dst, dst_f64, cnt, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "convert: %s", cudaGetErrorString(e));
        return MDS_OK;
    }
    if ((src_kind == 0 && !dst_f64) || (src_kind == 1 && dst_f64)) {
        // same element type: straight to the host
        CU(cudaMemcpyAsync(dst, dev_src, count * eb, cudaMemcpyDeviceToHost, c->stream));
    } else {
        cudaError_t e = launch_convert(dev_src, src_kind == 1, c->stage, dst_f64, cnt, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "convert: %s", cudaGetErrorString(e));
        CU(cudaMemcpyAsync(dst, c->stage, count * eb, cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaStreamSynchronize(c->stream));
    return MDS_OK;
}

// Bring a caller N x D array (host or device, f32/f64) onto the device;
// returns a device pointer (the caller's or the staging buffer).
int stage_in(mds_ctx *c, const void *src, int dtype, int where, int64_t count, const void **dev) {
    const size_t eb = dtype == MDS_F64 ? 8 : 4;
    if (where == MDS_DEVICE) {
        *dev = src;
        return MDS_OK;
    }
    CU(cudaMemcpyAsync(c->stage, src, count * eb, cudaMemcpyHostToDevice, c->stream));
    *dev = c->stage;
    return MDS_OK;
}

int valid_enums(mds_ctx *c, int dtype, int where) {
    if (dtype != MDS_F32 && dtype != MDS_F64) return fail(c, MDS_ERR_INVALID_ARG, "dtype must be MDS_F32 or MDS_F64");
    if (where != MDS_HOST && where != MDS_DEVICE)
        return fail(c, MDS_ERR_INVALID_ARG, "where must be MDS_HOST or MDS_DEVICE");
    return MDS_OK;
}

TrajArgs make_traj_args(const mds_ctx *c, int n_steps, double eps, int momentum_src, uint64_t seed, uint32_t chain) {
    TrajArgs t{};
    t.n = c->n;
    t.d = c->d;
    t.fp64 = c->fp64;
    t.eps = eps;
    t.lambda = c->lambda;
    t.momentum_src = momentum_src;
    t.p_inj = c->p_inj;
    t.seed = seed;
    t.chain = chain;
    t.xs = xstate(c);
    t.p = c->p;
    t.x0 = c->x0;
    t.grad = static_cast<double *>(c->grad);
    t.grad0 = static_cast<double *>(c->grad0);
    t.scal = c->scal;
    t.counters = c->counters;
    t.energy_part = c->e_start;
    t.drift = n_steps > 0 ? 1 : 0;
    t.prior_grad = c->tree_on ? c->tree.grad : nullptr;
    t.prior_grad0 = c->tree_on ? c->tree_grad0 : nullptr;
    return t;
}

AcceptArgs make_accept_args(const mds_ctx *c, int n_steps, int metropolis, int u_src, uint64_t seed, uint32_t chain,
                            int start_grid, int32_t *acc_out, double *dh_out, int64_t out_cap) {
    AcceptArgs a{};
    a.n = c->n;
    a.d = c->d;
    a.fp64 = c->fp64;
    a.metropolis = metropolis;
    a.n_start_parts = start_grid;
    a.start_part = c->e_start;
    if (n_steps > 0) {
        a.n_end_parts = static_cast<int32_t>(c->nt * kReduceQuarters);
        a.end_part = c->e_end;
    } else {
        a.n_end_parts = start_grid;
        a.end_part = c->e_start;
    }
    a.lambda = c->lambda;
    a.u_src = u_src;
    a.u_inj = c->u_inj;
    a.seed = seed;
    a.chain = chain;
    a.xs = xstate(c);
    a.x0 = c->x0;
    a.grad = static_cast<double *>(c->grad);
    a.grad0 = static_cast<double *>(c->grad0);
    a.scal = c->scal;
    a.counters = c->counters;
    a.prior_grad = c->tree_on ? c->tree.grad : nullptr;
    a.prior_grad0 = c->tree_on ? c->tree_grad0 : nullptr;
    // per-iteration outputs only for Metropolis runs (their index is the
    // iteration within the current HMC call, below the output capacity)
    a.acc_out = metropolis ? acc_out : nullptr;
    a.dh_out = metropolis ? dh_out : nullptr;
    a.out_cap = out_cap;
    a.err = c->err;
    return a;
}

// Enqueue one trajectory: start kernel, n_steps fused pair passes with their
// leapfrog updates, end kernel (Metropolis when metropolis != 0).
int enqueue_trajectory(mds_ctx *c, int n_steps, double eps, int momentum_src, int u_src, int metropolis,
                       uint64_t seed, cudaStream_t s) {
    TrajArgs t = make_traj_args(c, n_steps, eps, momentum_src, seed, 0);
    int grid = 0;
    cudaError_t e = launch_traj_start(t, &grid, s);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "trajectory start: %s", cudaGetErrorString(e));
    c->start_grid = grid;
    for (int k = 0; k < n_steps; ++k)
        CHECK(enqueue_pass(c, k + 1 < n_steps ? kModeKickDrift : kModeHalfKick, eps, s));
    AcceptArgs a = make_accept_args(c, n_steps, metropolis, u_src, seed, 0, grid, c->acc_out, c->dh_out,
                                    static_cast<int64_t>(c->out_cap));
    e = launch_traj_end(a, s);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "trajectory end: %s", cudaGetErrorString(e));
    return MDS_OK;
}

int ensure_out_cap(mds_ctx *c, size_t n_iter) {
    if (n_iter <= c->out_cap) return MDS_OK;
    dev_free(c->acc_out);
    dev_free(c->dh_out);
    c->acc_out = nullptr;
    c->dh_out = nullptr;
    CHECK(dev_alloc_t(c, &c->acc_out, n_iter * sizeof(int32_t)));
    CHECK(dev_alloc_t(c, &c->dh_out, n_iter * sizeof(double)));
    c->out_cap = n_iter;
    c->gen++;
    return MDS_OK;
}

// Pinned host memory for read-backs (grown on demand, kept).
int ensure_host_stage(mds_ctx *c, size_t bytes) {
    if (bytes <= c->host_stage_bytes) return MDS_OK;
    if (c->host_stage) {
        CU(cudaStreamSynchronize(c->stream));
        cudaFreeHost(c->host_stage);
        c->host_stage = nullptr;
        c->host_stage_bytes = 0;
    }
    const size_t nb = std::max<size_t>(bytes, 4096);
    CU(cudaMallocHost(&c->host_stage, nb));
    c->host_stage_bytes = nb;
    return MDS_OK;
}

// Move the results of the queued iterations to the host (waits) and restart
// the device-side iteration index, making room in the result buffers.
int hmc_spill(mds_ctx *c) {
    const int64_t k = c->hmc_pending;
    if (k <= 0) return MDS_OK;
    CHECK(ensure_host_stage(c, static_cast<size_t>(k) * (sizeof(int32_t) + sizeof(double))));
    double *hd = static_cast<double *>(c->host_stage);
    int32_t *ha = reinterpret_cast<int32_t *>(hd + k);
    CU(cudaMemcpyAsync(hd, c->dh_out, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(ha, c->acc_out, k * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemsetAsync(c->counters + kIterLocal, 0, sizeof(int64_t), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->acc_spill.insert(c->acc_spill.end(), ha, ha + k);
    c->dh_spill.insert(c->dh_spill.end(), hd, hd + k);
    c->hmc_pending = 0;
    return MDS_OK;
}

// Queue n_iter HMC iterations (one CUDA graph launch each) without waiting.
// inj: momenta / uniforms from p_inj / u_inj (indexed by the iteration
// within the queue, which must then start empty).
int hmc_enqueue(mds_ctx *c, int n_iter, int n_steps, double eps, uint64_t seed, int inj) {
    if (inj && c->hmc_pending != 0) return fail(c, MDS_ERR_STATE, "injected momenta need an empty queue");
    if (c->hmc_pending + n_iter > static_cast<int64_t>(c->out_cap)) {
        CHECK(hmc_spill(c));
        CHECK(ensure_out_cap(c, static_cast<size_t>(n_iter)));
    }
    if (sharded(c)) {
        // the exchange is a host call between kernels: iterations run eagerly
        for (int t = 0; t < n_iter; ++t) {
            CHECK(enqueue_trajectory(c, n_steps, eps, inj ? 2 : 1, inj ? 2 : 1, 1, seed, c->stream));
            c->hmc_pending++;
        }
        return MDS_OK;
    }
    // one HMC iteration as a CUDA graph, captured once per configuration
    const auto key = std::make_tuple(c->gen, n_steps, eps, inj ? 2 : 1, c->profiling ? 1 : 0, seed, c->strip);
    if (!c->graph || key != c->graph_key) {
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        c->prof_used = 0;
        int st = enqueue_trajectory(c, n_steps, eps, inj ? 2 : 1, inj ? 2 : 1, 1, seed, c->cap_stream);
        c->graph_prof = c->prof_used;
        c->prof_used = 0;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (st != MDS_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        if (c->graph) {
            // same launches with new arguments (sigma, eps, buffers): update the
            // instantiated graph in place; otherwise instantiate afresh
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(c->graph, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(c->graph);
                c->graph = nullptr;
            }
        }
        if (!c->graph) e = cudaGraphInstantiate(&c->graph, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            return fail(c, MDS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        c->graph_key = key;
    }
    for (int t = 0; t < n_iter; ++t) {
        CU(cudaGraphLaunch(c->graph, c->stream));
        c->hmc_pending++;
        if (c->profiling) {
            CU(cudaStreamSynchronize(c->stream));
            c->prof_used = c->graph_prof;
            CHECK(harvest_prof(c));
        }
    }
    return MDS_OK;
}

// Wait for the queued iterations and hand back their results (spilled ones
// first), with one read-back: error word, scalars, counters, per-iteration
// decisions and H1 - H0.  Entries beyond cap are dropped; *count gets the
// number of iterations collected.
int hmc_collect(mds_ctx *c, int64_t cap, int32_t *accepted, double *dh, int64_t *count, mds_hmc_stats *stats,
                const char *what) {
    const int64_t k = c->hmc_pending;
    const size_t bytes = 8 + kScalars * 8 + kCounters * 8 + static_cast<size_t>(k) * (8 + 4);
    CHECK(ensure_host_stage(c, bytes));
    double *hs = static_cast<double *>(c->host_stage);  // [scalars][counters][dh][acc][err]
    int64_t *hc = reinterpret_cast<int64_t *>(hs + kScalars);
    double *hd = reinterpret_cast<double *>(hc + kCounters);
    int32_t *ha = reinterpret_cast<int32_t *>(hd + k);
    unsigned *he = reinterpret_cast<unsigned *>(ha + k + (k & 1));
    CU(cudaMemcpyAsync(hs, c->scal, kScalars * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hc, c->counters, kCounters * 8, cudaMemcpyDeviceToHost, c->stream));
    if (k > 0) {
        CU(cudaMemcpyAsync(hd, c->dh_out, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(ha, c->acc_out, k * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaMemcpyAsync(he, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemsetAsync(c->counters + kIterLocal, 0, sizeof(int64_t), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> acc = std::move(c->acc_spill);
    std::vector<double> dhv = std::move(c->dh_spill);
    c->acc_spill.clear();
    c->dh_spill.clear();
    acc.insert(acc.end(), ha, ha + k);
    dhv.insert(dhv.end(), hd, hd + k);
    c->hmc_pending = 0;
    const int64_t total = static_cast<int64_t>(acc.size());
    for (int64_t t = 0; t < total && t < cap; ++t) {
        if (accepted) accepted[t] = acc[t];
        if (dh) dh[t] = dhv[t];
    }
    *count = total;
    if (stats) {
        int64_t na = 0;
        for (int32_t v : acc) na += v;
        stats->iterations = total;
        stats->accepted = na;
        stats->last_dh = hs[kLastDH];
        stats->last_loglik = hs[kLogLik];
    }
    c->eval_unchecked = false;
    const unsigned h = *he;
    if (h == 0) return MDS_OK;
    // the start-point evaluation may be the failed step: evaluate afresh next time
    c->grad_valid = false;
    CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return err_status(c, h, what);
}

// Forget the held-out fold: restore the held-out y into the tile-packed Y
// (unless Y is about to be replaced) and free the fold's buffers.
int drop_fold(mds_ctx *c, bool restore) {
    if (c->ho_count > 0) {
        if (restore) {
            cudaError_t e = launch_ho_restore(c->y, c->ho_off, c->ho_count, c->ho_y, c->stream);
            if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "fold restore: %s", cudaGetErrorString(e));
        }
        CU(cudaMemsetAsync(c->tile_ho, 0, static_cast<size_t>(c->tiles), c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    void *bufs[] = {c->ho_off, c->ho_pairs, c->ho_y, c->lse_m, c->lse_s};
    for (void *b : bufs) dev_free(b);
    c->ho_off = nullptr;
    c->ho_pairs = nullptr;
    c->ho_y = nullptr;
    c->lse_m = nullptr;
    c->lse_s = nullptr;
    if (c->ho_count > 0) {
        c->gen++;
        c->grad_valid = false;
    }
    c->ho_count = 0;
    c->lpd_draws = 0;
    return MDS_OK;
}

// Re-pack Y from the current slot order into `order` (new slot -> item, over
// n_pad slots, pads fixed) and make it the context's slot order.  `from_identity`:
// Y is in the caller's item order (just ingested) rather than the current order.
int repack_to(mds_ctx *c, const std::vector<int32_t> &order, bool from_identity) {
    const int64_t np = c->n_pad;
    std::vector<int32_t> map(np), inv(np);
    for (int64_t s = 0; s < np; ++s) {
        map[s] = (c->reordered && !from_identity) ? c->inv_h[order[s]] : order[s];
        inv[order[s]] = static_cast<int32_t>(s);
    }
    int32_t *map_d = nullptr;
    float *ny = nullptr;
    CHECK(dev_alloc_t(c, &map_d, np * sizeof(int32_t)));
    int st = dev_alloc_t(c, &ny, static_cast<size_t>(c->tiles) * kTileElems * sizeof(float));
    if (st != MDS_OK) {
        dev_free(map_d);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(map_d, map.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_repack(c->y, ny, map_d, c->n, static_cast<int32_t>(c->nt), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(map_d);
    if (e != cudaSuccess) {
        dev_free(ny);
        return fail(c, MDS_ERR_CUDA, "reorder: %s", cudaGetErrorString(e));
    }
    dev_free(c->y);
    c->y = ny;
    if (!c->perm_d) {
        CHECK(dev_alloc_t(c, &c->perm_d, np * sizeof(int32_t)));
        CHECK(dev_alloc_t(c, &c->inv_d, np * sizeof(int32_t)));
    }
    CU(cudaMemcpyAsync(c->perm_d, order.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->inv_d, inv.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->perm_h = order;
    c->inv_h = inv;
    c->reordered = true;
    c->tile_cost.clear();  // far counts of the old order
    c->gen++;  // the captured graph holds the old Y pointer
    c->grad_valid = false;
    return MDS_OK;
}

// Y was just ingested in the caller's order: bring it to the context's slot order.
int apply_order(mds_ctx *c, const std::vector<int32_t> &order) { return repack_to(c, order, true); }

// A chain of a batch takes the slot order its dataset's first chain chose
// (their shared Y, already repacked, at y): the order tables, then the split
// locations rewritten at their new slots.  The state stays in item order.
int adopt_order(mds_ctx *c, const std::vector<int32_t> &order, const std::vector<int32_t> &inv, float *y) {
    const int64_t np = c->n_pad;
    c->y = y;
    if (!c->perm_d) {
        CHECK(dev_alloc_t(c, &c->perm_d, np * sizeof(int32_t)));
        CHECK(dev_alloc_t(c, &c->inv_d, np * sizeof(int32_t)));
    }
    CU(cudaMemcpyAsync(c->perm_d, order.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->inv_d, inv.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    c->perm_h = order;
    c->inv_h = inv;
    c->reordered = true;
    c->tile_cost.clear();
    c->gen++;
    c->grad_valid = false;
    cudaError_t e = launch_resplit(xstate(c), np, c->d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "batch order: %s", cudaGetErrorString(e));
    return MDS_OK;
}

}  // namespace

// Recursive bisection: split the range along its widest coordinate (ties
// broken by item index, so the order is the same on every host), at a
// multiple of 64 items while the range is longer than one tile block, so
// that every block of 64 slots is one spatially compact cell.
namespace {
void bisect(const double *x, int d, int32_t *idx, int64_t len) {
    while (len > 2) {
        int best = 0;
        double width = -1.0;
        for (int k = 0; k < d; ++k) {
            double lo = x[static_cast<int64_t>(idx[0]) * d + k], hi = lo;
            for (int64_t t = 1; t < len; ++t) {
                const double v = x[static_cast<int64_t>(idx[t]) * d + k];
                lo = std::min(lo, v);
                hi = std::max(hi, v);
            }
            if (hi - lo > width) {
                width = hi - lo;
                best = k;
            }
        }
        const int64_t h = len > kTile ? std::min<int64_t>(len - 1, (len / 2 + kTile - 1) / kTile * kTile) : len / 2;
        std::nth_element(idx, idx + h, idx + len, [x, d, best](int32_t a, int32_t b) {
            const double va = x[static_cast<int64_t>(a) * d + best], vb = x[static_cast<int64_t>(b) * d + best];
            return va < vb || (va == vb && a < b);
        });
        bisect(x, d, idx, h);
        idx += h;
        len -= h;
    }
}
}  // namespace

void mds::locality_order(int64_t n, int d, const double *x, int32_t *perm) {
    for (int64_t s = 0; s < n; ++s) perm[s] = static_cast<int32_t>(s);
    bisect(x, d, perm, n);
}

void mds::set_thread_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_create_error = buf;
}

// ====================================================================== ABI

extern "C" {

}  // extern "C"

namespace {

int create_ctx(int64_t n, int32_t d, uint32_t flags, bool alloc_y, mds_ctx **out) {
    mds_ctx *c = nullptr;
    if (!out) return fail(c, MDS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 2 || n > 2147483647LL) return fail(c, MDS_ERR_INVALID_ARG, "N must be in [2, 2^31-1], got %lld", (long long)n);
    if (d < 1 || d > MDS_MAX_D) return fail(c, MDS_ERR_INVALID_ARG, "D must be in [1, %d], got %d", MDS_MAX_D, d);
    if (flags != MDS_PREC_FP32C && flags != MDS_PREC_FP64)
        return fail(c, MDS_ERR_INVALID_ARG, "flags must be MDS_PREC_FP32C or MDS_PREC_FP64");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(c, MDS_ERR_UNSUPPORTED, "no CUDA device: %s", cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (prop.major != 10)
        return fail(c, MDS_ERR_UNSUPPORTED, "device %s is compute capability %d.%d; the library is compiled for sm_103a",
                    prop.name, prop.major, prop.minor);
    c = new (std::nothrow) mds_ctx();
    if (!c) return fail(nullptr, MDS_ERR_OOM, "host allocation failed");
    c->n = n;
    c->d = d;
    c->fp64 = flags == MDS_PREC_FP64;
    c->device = dev;
    c->sm_count = prop.multiProcessorCount;
    c->device_name = prop.name;
    c->nt = (n + kTile - 1) / kTile;
    c->n_pad = c->nt * kTile;
    c->tiles = tile_count(c->nt);
    c->shard_t0 = 0;
    c->shard_t1 = c->tiles;
    c->shard_pairs = n * (n - 1) / 2;
    auto cleanup = [&](int st) {
        g_create_error = c->last_error;
        mds_destroy(c);
        return st;
    };
    const size_t eb = elem(c);
    const int64_t nd_pad = c->n_pad * d;
    int st = MDS_OK;
    c->y_owned = alloc_y;
    if (alloc_y && (st = dev_alloc_t(c, &c->y, static_cast<size_t>(c->tiles) * kTileElems * sizeof(float))))
        return cleanup(st);
    if ((st = dev_alloc(c, &c->x, nd_pad * eb))) return cleanup(st);
    if ((st = dev_alloc(c, &c->p, nd_pad * eb))) return cleanup(st);
    if ((st = dev_alloc(c, &c->x0, nd_pad * eb))) return cleanup(st);
    if (!c->fp64) {
        if ((st = dev_alloc_t(c, &c->xrow, nd_pad / 2 * sizeof(float4)))) return cleanup(st);
        if ((st = dev_alloc_t(c, &c->xcol, nd_pad * sizeof(float4)))) return cleanup(st);
        if ((st = dev_alloc_t(c, &c->xcol2, nd_pad * sizeof(float2)))) return cleanup(st);
        if ((st = dev_alloc_t(c, &c->far_tile, static_cast<size_t>(c->tiles) * kPairWarps))) return cleanup(st);
        if ((st = dev_alloc_t(c, &c->split, sizeof(Split)))) return cleanup(st);
        if ((st = dev_alloc_t(c, &c->xmax_bits, sizeof(unsigned)))) return cleanup(st);
    }
    if ((st = dev_alloc(c, &c->grad, nd_pad * grad_elem(c)))) return cleanup(st);
    if ((st = dev_alloc(c, &c->grad0, nd_pad * grad_elem(c)))) return cleanup(st);
    if ((st = dev_alloc(c, &c->col_part, static_cast<size_t>(c->tiles) * kTile * d * eb))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->row_first, (c->nt + 1) * sizeof(int32_t)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->scal, kScalars * sizeof(double)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->counters, kCounters * sizeof(int64_t)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->err, sizeof(unsigned)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->bad, sizeof(unsigned long long)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->stamps, 2 * sizeof(unsigned long long)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->pass_ns, 2 * sizeof(double)))) return cleanup(st);
    const int64_t start_grid_max = (nd_pad + 4 * 256 - 1) / (4 * 256) + 1;
    if ((st = dev_alloc_t(c, &c->e_start, start_grid_max * 2 * sizeof(double)))) return cleanup(st);
    if ((st = dev_alloc_t(c, &c->e_end, (c->nt * kReduceQuarters + 1) * 2 * sizeof(double)))) return cleanup(st);
    if ((st = dev_alloc(c, &c->stage, nd_pad * sizeof(double)))) return cleanup(st);
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        c->last_error = "stream/event creation failed";
        return cleanup(MDS_ERR_CUDA);
    }
    bool ok = cudaMemset(c->x, 0, nd_pad * eb) == cudaSuccess && cudaMemset(c->p, 0, nd_pad * eb) == cudaSuccess &&
              cudaMemset(c->grad, 0, nd_pad * grad_elem(c)) == cudaSuccess &&
              cudaMemset(c->scal, 0, kScalars * 8) == cudaSuccess &&
              cudaMemset(c->counters, 0, kCounters * 8) == cudaSuccess &&
              cudaMemset(c->err, 0, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(c->stamps, 0, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMemset(c->pass_ns, 0, 2 * sizeof(double)) == cudaSuccess;
    if (ok && !c->fp64) {
        ok = cudaMemset(c->xrow, 0, nd_pad / 2 * sizeof(float4)) == cudaSuccess &&
             cudaMemset(c->xcol, 0, nd_pad * sizeof(float4)) == cudaSuccess &&
             cudaMemset(c->xcol2, 0, nd_pad * sizeof(float2)) == cudaSuccess &&
             cudaMemset(c->far_tile, 0, static_cast<size_t>(c->tiles) * kPairWarps) == cudaSuccess &&
             cudaMemset(c->xmax_bits, 0, sizeof(unsigned)) == cudaSuccess;
        Split sp{1.0f, 12582912.0f, 0.0f, 0};  // q = 1 until locations are set
        ok = ok && cudaMemcpy(c->split, &sp, sizeof(sp), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        c->last_error = "initial memset failed";
        return cleanup(MDS_ERR_CUDA);
    }
    if ((st = build_strips(c, 1))) return cleanup(st);
    *out = c;
    return MDS_OK;
}

}  // namespace

extern "C" {

int mds_create(int64_t n, int32_t d, uint32_t flags, mds_ctx **out) { return create_ctx(n, d, flags, true, out); }

int mds_destroy(mds_ctx *c) {
    if (!c) return MDS_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (!c->y_owned) c->y = nullptr;
    void *bufs[] = {c->y,        c->x,        c->p,         c->x0,       c->xrow,      c->xcol,
                    c->split,    c->xmax_bits, c->grad,     c->grad0,    c->col_part,  c->row_part,
                    c->scal_part, c->strips,  c->row_first, c->scal,     c->counters,  c->err,
                    c->bad,      c->e_start,  c->e_end,     c->stage,    c->p_inj,     c->u_inj,
                    c->acc_out,  c->dh_out,    c->perm_d,    c->inv_d,     c->far_part,  c->chunks,
                    c->far_tile, c->xcol2,     c->stamps,    c->pass_ns,   c->shard_send, c->shard_recv};
    for (void *b : bufs) dev_free(b);
    void *ho_bufs[] = {c->ho_off, c->ho_pairs, c->ho_y, c->tile_ho, c->lse_m, c->lse_s, c->lpd_part, c->sigma_draws};
    for (void *b : ho_bufs) dev_free(b);
    for (void *b : c->tree_bufs) dev_free(b);
    if (c->host_stage) cudaFreeHost(c->host_stage);
    if (c->shard_hsend) cudaFreeHost(c->shard_hsend);
    if (c->shard_hrecv) cudaFreeHost(c->shard_hrecv);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->tree_stream) {
        cudaStreamSynchronize(c->tree_stream);
        cudaStreamDestroy(c->tree_stream);
    }
    if (c->tree_fork) cudaEventDestroy(c->tree_fork);
    if (c->tree_join) cudaEventDestroy(c->tree_join);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (cudaEvent_t e : c->prof_a) cudaEventDestroy(e);
    for (cudaEvent_t e : c->prof_b) cudaEventDestroy(e);
    delete c;
    return MDS_OK;
}

int mds_set_stream(mds_ctx *c, void *stream) {
    CHECK(check_ctx(c));
    c->stream = static_cast<cudaStream_t>(stream);
    return MDS_OK;
}

int mds_set_data(mds_ctx *c, const void *y, int dtype, int layout, int64_t ld, int where) {
    CHECK(check_ctx(c));
    if (!y) return fail(c, MDS_ERR_INVALID_ARG, "Y is NULL");
    CHECK(valid_enums(c, dtype, where));
    if (layout != MDS_Y_FULL && layout != MDS_Y_PACKED_UPPER)
        return fail(c, MDS_ERR_INVALID_ARG, "layout must be MDS_Y_FULL or MDS_Y_PACKED_UPPER");
    if (layout == MDS_Y_FULL && ld < c->n) return fail(c, MDS_ERR_INVALID_ARG, "ld (%lld) < N", (long long)ld);
    c->have_data = false;
    c->grad_valid = false;
    CHECK(drop_fold(c, false));  // the new Y replaces the marked values
    const bool f64 = dtype == MDS_F64;
    const size_t eb = f64 ? 8 : 4;
    const unsigned long long none = ~0ull;
    CU(cudaMemcpyAsync(c->bad, &none, sizeof(none), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    IngestArgs a{};
    a.t_lo = c->shard_t0;
    a.t_hi = c->shard_t1;
    a.src_f64 = f64;
    a.packed = layout == MDS_Y_PACKED_UPPER;
    a.ld = ld;
    a.n = c->n;
    a.nt = static_cast<int32_t>(c->nt);
    a.y = c->y;
    a.bad = c->bad;
    a.err = c->err;
    const int64_t n = c->n;
    if (where == MDS_DEVICE) {
        a.src = y;
        a.r0 = 0;
        a.r1 = n;
        cudaError_t e = launch_ingest(a, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "ingest: %s", cudaGetErrorString(e));
    } else {
        // host source: stage groups of row blocks through a device buffer
        // (a shard uploads only the rows of its tiles' row blocks)
        const int64_t rows_per = kTile * std::max<int64_t>(1, (int64_t(64) << 20) / (kTile * n * eb));
        const size_t stage_bytes = static_cast<size_t>(std::min<int64_t>(rows_per, n)) * n * eb;
        int64_t row_lo = 0, row_hi = n;
        if (c->shard_n > 1) {
            if (c->shard_t1 <= c->shard_t0) {
                row_hi = 0;
            } else {
                int64_t I0 = 0, I1 = 0;
                while (I0 + 1 < c->nt && tile_index(I0 + 1, I0 + 1, c->nt) <= c->shard_t0) ++I0;
                I1 = I0;
                while (I1 + 1 < c->nt && tile_index(I1 + 1, I1 + 1, c->nt) <= c->shard_t1 - 1) ++I1;
                row_lo = I0 * kTile;
                row_hi = std::min(n, (I1 + 1) * kTile);
            }
        }
        void *stg = nullptr;
        CHECK(dev_alloc(c, &stg, stage_bytes));
        int st = MDS_OK;
        for (int64_t r0 = row_lo; r0 < row_hi && st == MDS_OK; r0 += rows_per) {
            const int64_t r1 = std::min(row_hi, r0 + rows_per);
            const char *src;
            size_t bytes;
            if (a.packed) {
                const int64_t o0 = packed_row_start(r0, n), o1 = packed_row_start(r1, n);
                src = static_cast<const char *>(y) + o0 * eb;
                bytes = (o1 - o0) * eb;
            } else {
                src = static_cast<const char *>(y) + r0 * ld * eb;
                bytes = ((r1 - r0 - 1) * ld + n) * eb;
            }
            if (bytes > 0) {
                cudaError_t e = cudaMemcpyAsync(stg, src, bytes, cudaMemcpyHostToDevice, c->stream);
                if (e != cudaSuccess) st = fail(c, MDS_ERR_CUDA, "Y upload: %s", cudaGetErrorString(e));
            }
            a.src = stg;
            a.r0 = r0;
            a.r1 = r1;
            if (st == MDS_OK) {
                cudaError_t e = launch_ingest(a, c->stream);
                if (e != cudaSuccess) st = fail(c, MDS_ERR_CUDA, "ingest: %s", cudaGetErrorString(e));
            }
            if (st == MDS_OK) {
                cudaError_t e = cudaStreamSynchronize(c->stream);  // staging buffer reuse
                if (e != cudaSuccess) st = fail(c, MDS_ERR_CUDA, "ingest: %s", cudaGetErrorString(e));
            }
        }
        cudaFree(stg);
        if (st != MDS_OK) return st;
    }
    unsigned h = 0;
    unsigned long long bad = 0;
    CU(cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(&bad, c->bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h & kErrBadInput) {
        CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
        CU(cudaStreamSynchronize(c->stream));
        return fail(c, MDS_ERR_INVALID_ARG,
                    "Y(%llu, %llu) is negative, NaN or Inf; dissimilarities must be finite and >= 0 (no data set)",
                    bad / static_cast<unsigned long long>(n), bad % static_cast<unsigned long long>(n));
    }
    if (h) return check_device_err(c, "set_data");
    if (c->reordered) CHECK(apply_order(c, c->perm_h));  // ingest wrote the caller's order
    c->have_data = true;
    return MDS_OK;
}

int mds_set_locations(mds_ctx *c, const void *x, int dtype, int where) {
    CHECK(check_ctx(c));
    if (!x) return fail(c, MDS_ERR_INVALID_ARG, "X is NULL");
    CHECK(valid_enums(c, dtype, where));
    const void *dev = nullptr;
    CHECK(stage_in(c, x, dtype, where, c->n * c->d, &dev));
    CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    if (!c->fp64) {
        // max |x| of the incoming values; the set_x kernel derives the
        // quantum of the exact-difference split from it on the device
        CU(cudaMemsetAsync(c->xmax_bits, 0, sizeof(unsigned), c->stream));
        cudaError_t e = launch_xmax(dev, dtype == MDS_F64, c->n * c->d, c->xmax_bits, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "set_locations: %s", cudaGetErrorString(e));
    }
    cudaError_t e = launch_set_x(dev, dtype == MDS_F64, c->n, c->n_pad, c->d, c->fp64, xstate(c), c->err, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "set_locations: %s", cudaGetErrorString(e));
    // the one wait of the call: the error word (non-finite entry, range)
    unsigned h = 0;
    CU(cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h) {
        unsigned bits = 0;
        if (!c->fp64) CU(cudaMemcpyAsync(&bits, c->xmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if (h & kErrRange) {
            // nothing was written: the previous locations stay in place
            float m;
            std::memcpy(&m, &bits, sizeof(m));
            return fail(c, MDS_ERR_INVALID_ARG, "locations out of the FP32C range (max |x| = %g)", m);
        }
        c->have_x = false;
        return fail(c, MDS_ERR_INVALID_ARG, "X has a NaN or Inf entry");
    }
    c->have_x = true;
    c->grad_valid = false;
    return MDS_OK;
}

int mds_get_locations(mds_ctx *c, void *x, int dtype, int where) {
    CHECK(check_ctx(c));
    if (!x) return fail(c, MDS_ERR_INVALID_ARG, "X is NULL");
    CHECK(valid_enums(c, dtype, where));
    if (!c->have_x) return fail(c, MDS_ERR_STATE, "no locations set");
    return copy_out(c, c->x, c->fp64 ? 1 : 0, x, dtype, where, c->n * c->d);
}

int mds_set_sigma(mds_ctx *c, double sigma) {
    CHECK(check_ctx(c));
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(c, MDS_ERR_INVALID_ARG, "sigma must be finite and > 0");
    if (!c->fp64 && (sigma < 1e-6 || sigma > 1e6))
        return fail(c, MDS_ERR_INVALID_ARG, "the FP32C path needs 1e-6 <= sigma <= 1e6, got %g", sigma);
    if (sigma != c->sigma) {
        c->sigma = sigma;
        c->grad_valid = false;
        c->gen++;
    }
    c->have_sigma = true;
    return MDS_OK;
}

int mds_set_prior(mds_ctx *c, double lambda) {
    CHECK(check_ctx(c));
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(c, MDS_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    if (lambda != c->lambda) {
        c->lambda = lambda;
        c->gen++;
    }
    return MDS_OK;
}

int mds_log_likelihood(mds_ctx *c, double *loglik, double *sum_r) {
    CHECK(check_ctx(c));
    if (!loglik && !sum_r) return fail(c, MDS_ERR_INVALID_ARG, "no output requested");
    if (!c->grad_valid) CHECK(evaluate(c));
    double s[kScalars];
    CU(cudaMemcpyAsync(s, c->scal, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (loglik) *loglik = s[kLogLik];
    if (sum_r) *sum_r = s[kSumR];
    if (!std::isfinite(s[kLogLik])) return fail(c, MDS_ERR_NONFINITE, "log-likelihood is not finite");
    return MDS_OK;
}

int mds_gradient(mds_ctx *c, double *loglik, void *grad, int dtype, int where, double *dsigma) {
    CHECK(check_ctx(c));
    if (grad) CHECK(valid_enums(c, dtype, where));
    CHECK(evaluate(c));
    if (grad) CHECK(copy_out(c, c->grad, c->fp64 ? 1 : 2, grad, dtype, where, c->n * c->d));
    if (loglik || dsigma) {
        double s[kScalars];
        CU(cudaMemcpyAsync(s, c->scal, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if (loglik) *loglik = s[kLogLik];
        if (dsigma) *dsigma = s[kDSigma];
    }
    return MDS_OK;
}

int mds_set_momentum(mds_ctx *c, const void *p, int dtype, int where) {
    CHECK(check_ctx(c));
    if (!p) return fail(c, MDS_ERR_INVALID_ARG, "p is NULL");
    CHECK(valid_enums(c, dtype, where));
    const void *dev = nullptr;
    CHECK(stage_in(c, p, dtype, where, c->n * c->d, &dev));
    cudaError_t e = launch_convert(dev, dtype == MDS_F64, c->p, c->fp64, c->n * c->d, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "set_momentum: %s", cudaGetErrorString(e));
    CU(cudaStreamSynchronize(c->stream));
    return MDS_OK;
}

int mds_get_momentum(mds_ctx *c, void *p, int dtype, int where) {
    CHECK(check_ctx(c));
    if (!p) return fail(c, MDS_ERR_INVALID_ARG, "p is NULL");
    CHECK(valid_enums(c, dtype, where));
    return copy_out(c, c->p, c->fp64 ? 1 : 0, p, dtype, where, c->n * c->d);
}

int mds_leapfrog(mds_ctx *c, int n_steps, double eps, const void *p0, int p0_dtype, int p0_where, double *dh) {
    CHECK(check_ctx(c));
    if (n_steps < 0) return fail(c, MDS_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (!std::isfinite(eps)) return fail(c, MDS_ERR_INVALID_ARG, "eps must be finite");
    CHECK(ready(c));
    if (p0) CHECK(mds_set_momentum(c, p0, p0_dtype, p0_where));
    if (!c->grad_valid) CHECK(evaluate(c));
    CHECK(autotune(c));
    CHECK(enqueue_trajectory(c, n_steps, eps, 0, 1, 0, 0, c->stream));
    CHECK(check_device_err(c, "leapfrog"));
    if (c->profiling) CHECK(harvest_prof(c));
    if (dh) {
        double s[kScalars];
        CU(cudaMemcpyAsync(s, c->scal, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        *dh = s[kLastDH];
    }
    return MDS_OK;
}

int mds_hmc(mds_ctx *c, int n_iter, int n_steps, double eps, uint64_t seed, const double *p_all, const double *u_all,
            int *accepted, double *dh, mds_hmc_stats *stats) {
    CHECK(check_ctx(c));
    if (n_iter < 0 || n_steps < 0) return fail(c, MDS_ERR_INVALID_ARG, "n_iter and n_steps must be >= 0");
    if (!std::isfinite(eps)) return fail(c, MDS_ERR_INVALID_ARG, "eps must be finite");
    if ((p_all == nullptr) != (u_all == nullptr))
        return fail(c, MDS_ERR_INVALID_ARG, "p_all and u_all must be given together");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    CHECK(ready(c));
    CHECK(queue_start_eval(c));
    if (n_iter == 0) return finish_start_eval(c, "hmc");
    const int inj = p_all != nullptr;
    if (inj) {
        const int64_t nd = c->n * c->d;
        for (int t = 0; t < n_iter; ++t)
            if (!(u_all[t] > 0.0 && u_all[t] < 1.0)) return fail(c, MDS_ERR_INVALID_ARG, "u_all[%d] not in (0,1)", t);
        const size_t pb = static_cast<size_t>(n_iter) * nd * sizeof(double);
        if (pb > c->p_inj_bytes) {
            dev_free(c->p_inj);
            c->p_inj = nullptr;
            CHECK(dev_alloc_t(c, &c->p_inj, pb));
            c->p_inj_bytes = pb;
            c->gen++;
        }
        const size_t ub = static_cast<size_t>(n_iter) * sizeof(double);
        if (ub > c->u_inj_bytes) {
            dev_free(c->u_inj);
            c->u_inj = nullptr;
            CHECK(dev_alloc_t(c, &c->u_inj, ub));
            c->u_inj_bytes = ub;
            c->gen++;
        }
        CU(cudaMemcpyAsync(c->p_inj, p_all, pb, cudaMemcpyHostToDevice, c->stream));
        CU(cudaMemcpyAsync(c->u_inj, u_all, ub, cudaMemcpyHostToDevice, c->stream));
    }
    CHECK(hmc_enqueue(c, n_iter, n_steps, eps, seed, inj));
    int64_t count = 0;
    return hmc_collect(c, n_iter, accepted, dh, &count, stats, "hmc");
}

int mds_hmc_enqueue(mds_ctx *c, int n_iter, int n_steps, double eps, uint64_t seed) {
    CHECK(check_ctx(c));
    if (n_iter < 0 || n_steps < 0) return fail(c, MDS_ERR_INVALID_ARG, "n_iter and n_steps must be >= 0");
    if (!std::isfinite(eps)) return fail(c, MDS_ERR_INVALID_ARG, "eps must be finite");
    CHECK(ready(c));
    CHECK(queue_start_eval(c));
    if (n_iter == 0) return finish_start_eval(c, "hmc");
    return hmc_enqueue(c, n_iter, n_steps, eps, seed, 0);
}

int mds_hmc_collect(mds_ctx *c, int64_t cap, int32_t *accepted, double *dh, int64_t *count, mds_hmc_stats *stats) {
    CHECK(check_ctx(c));
    if (cap < 0) return fail(c, MDS_ERR_INVALID_ARG, "cap must be >= 0");
    int64_t n = 0;
    int st = hmc_collect(c, cap, accepted, dh, &n, stats, "hmc");
    if (count) *count = n;
    return st;
}

int mds_set_heldout(mds_ctx *c, const int64_t *pairs, int64_t n_pairs) {
    CHECK(check_ctx(c));
    if (sharded(c)) return fail(c, MDS_ERR_STATE, "cross-validation folds are not available on a sharded context");
    if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return fail(c, MDS_ERR_INVALID_ARG, "need n_pairs >= 0 and pairs");
    if (n_pairs > 0 && !c->have_data) return fail(c, MDS_ERR_STATE, "no data: call mds_set_data first");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    const int64_t n = c->n;
    std::vector<int64_t> key(static_cast<size_t>(n_pairs));
    for (int64_t k = 0; k < n_pairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j)
            return fail(c, MDS_ERR_INVALID_ARG, "held-out pair %lld = (%lld, %lld) is not a pair of distinct items",
                        (long long)k, (long long)i, (long long)j);
        if (i > j) std::swap(i, j);
        key[k] = packed_row_start(i, n) + (j - i - 1);
    }
    std::sort(key.begin(), key.end());
    key.erase(std::unique(key.begin(), key.end()), key.end());
    CHECK(drop_fold(c, true));
    const int64_t count = static_cast<int64_t>(key.size());
    if (count == 0) return MDS_OK;
    std::vector<int64_t> off(count);
    std::vector<int2> pr(count);
    for (int64_t k = 0; k < count; ++k) {
        // invert the packed index row by row (rows are long; a binary search would do for huge N)
        int64_t lo = 0, hi = n - 2;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (packed_row_start(mid, n) <= key[k]) lo = mid; else hi = mid - 1;
        }
        const int64_t i = lo, j = key[k] - packed_row_start(i, n) + i + 1;
        // the pair's place in the tile layout: by slot (upper triangle in slot order)
        int64_t si = c->reordered ? c->inv_h[i] : i, sj = c->reordered ? c->inv_h[j] : j;
        if (si > sj) std::swap(si, sj);
        const int64_t I = si / kTile, J = sj / kTile;
        off[k] = tile_index(I, J, c->nt) * kTileElems + tile_offset(static_cast<int>(si - I * kTile),
                                                                    static_cast<int>(sj - J * kTile));
        pr[k] = make_int2(static_cast<int>(i), static_cast<int>(j));
    }
    if (!c->tile_ho) {
        CHECK(dev_alloc_t(c, &c->tile_ho, static_cast<size_t>(c->tiles)));
        CU(cudaMemsetAsync(c->tile_ho, 0, static_cast<size_t>(c->tiles), c->stream));
    }
    if (!c->lpd_part) CHECK(dev_alloc_t(c, &c->lpd_part, (kLpdParts + 1) * sizeof(double)));
    CHECK(dev_alloc_t(c, &c->ho_off, count * sizeof(int64_t)));
    CHECK(dev_alloc_t(c, &c->ho_pairs, count * sizeof(int2)));
    CHECK(dev_alloc_t(c, &c->ho_y, count * sizeof(float)));
    CHECK(dev_alloc_t(c, &c->lse_m, count * sizeof(double)));
    CHECK(dev_alloc_t(c, &c->lse_s, count * sizeof(double)));
    CU(cudaMemcpyAsync(c->ho_off, off.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->ho_pairs, pr.data(), count * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    cudaError_t e = launch_ho_mark(c->y, c->ho_off, count, c->ho_y, c->tile_ho, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "fold mark: %s", cudaGetErrorString(e));
    CU(cudaStreamSynchronize(c->stream));  // the host vectors above go out of scope
    c->ho_count = count;
    c->lpd_draws = 0;
    c->gen++;
    c->grad_valid = false;
    return MDS_OK;
}

int mds_heldout_count(const mds_ctx *c, int64_t *count) {
    if (!c || !count) return MDS_ERR_INVALID_ARG;
    *count = c->ho_count;
    return MDS_OK;
}

int mds_lpd_accumulate(mds_ctx *c) {
    CHECK(check_ctx(c));
    if (c->ho_count == 0) return fail(c, MDS_ERR_STATE, "no held-out pairs: call mds_set_heldout first");
    if (!c->have_x) return fail(c, MDS_ERR_STATE, "no locations: call mds_set_locations first");
    if (!c->have_sigma) return fail(c, MDS_ERR_STATE, "no sigma: call mds_set_sigma first");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    cudaError_t e = launch_lpd_accumulate(c->x, c->fp64, c->d, c->ho_pairs, c->ho_y, c->ho_count, c->sigma,
                                          c->lpd_draws == 0, c->lse_m, c->lse_s, c->err, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "lpd: %s", cudaGetErrorString(e));
    CHECK(check_device_err(c, "lpd"));
    c->lpd_draws++;
    return MDS_OK;
}

int mds_lpd(mds_ctx *c, double *lpd, int64_t *draws) {
    CHECK(check_ctx(c));
    if (!lpd) return fail(c, MDS_ERR_INVALID_ARG, "lpd is NULL");
    if (c->lpd_draws == 0) return fail(c, MDS_ERR_STATE, "no draws accumulated (mds_lpd_accumulate)");
    cudaError_t e = launch_lpd_sum(c->lse_m, c->lse_s, c->ho_count, static_cast<double>(c->lpd_draws),
                                   c->lpd_part, c->lpd_part + kLpdParts, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "lpd: %s", cudaGetErrorString(e));
    CU(cudaMemcpyAsync(lpd, c->lpd_part + kLpdParts, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (draws) *draws = c->lpd_draws;
    return MDS_OK;
}

int mds_lpd_reset(mds_ctx *c) {
    CHECK(check_ctx(c));
    c->lpd_draws = 0;
    return MDS_OK;
}

int mds_get_sigma(const mds_ctx *c, double *sigma) {
    if (!c || !sigma) return MDS_ERR_INVALID_ARG;
    *sigma = c->sigma;
    return MDS_OK;
}

int mds_sigma_mh(mds_ctx *c, int n_iter, double step, double shape, double rate, uint64_t seed, const double *z_all,
                 const double *u_all, int32_t *accepted) {
    CHECK(check_ctx(c));
    if (sharded(c)) return fail(c, MDS_ERR_STATE, "sigma updates are not available on a sharded context");
    if (n_iter < 0) return fail(c, MDS_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (!(step >= 0.0) || !std::isfinite(step) || !(shape > 0.0) || !(rate > 0.0) || !std::isfinite(shape) ||
        !std::isfinite(rate))
        return fail(c, MDS_ERR_INVALID_ARG, "need step >= 0 and a Gamma prior with shape > 0 and rate > 0");
    if ((z_all == nullptr) != (u_all == nullptr))
        return fail(c, MDS_ERR_INVALID_ARG, "z_all and u_all must be given together");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    CHECK(ready(c));
    if (n_iter == 0) return MDS_OK;
    std::vector<double> z(n_iter), u(n_iter);
    if (z_all) {
        for (int t = 0; t < n_iter; ++t) {
            if (!(u_all[t] > 0.0 && u_all[t] < 1.0) || !std::isfinite(z_all[t]))
                return fail(c, MDS_ERR_INVALID_ARG, "draw %d: need a finite z and u in (0,1)", t);
            z[t] = z_all[t];
            u[t] = u_all[t];
        }
    } else {
        if (n_iter > c->sigma_draws_cap) {
            dev_free(c->sigma_draws);
            c->sigma_draws = nullptr;
            CHECK(dev_alloc_t(c, &c->sigma_draws, 2 * static_cast<size_t>(n_iter) * sizeof(double)));
            c->sigma_draws_cap = n_iter;
        }
        cudaError_t e = launch_sigma_draws(seed, 0u, c->sigma_iter, n_iter, c->sigma_draws,
                                           c->sigma_draws + n_iter, c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "sigma draws: %s", cudaGetErrorString(e));
        CU(cudaMemcpyAsync(z.data(), c->sigma_draws, n_iter * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(u.data(), c->sigma_draws + n_iter, n_iter * sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CU(cudaStreamSynchronize(c->stream));
        c->sigma_iter += n_iter;
    }
    // log posterior of tau = log sigma: L(X, sigma) + s0 log(sigma^-2) - r0 sigma^-2
    auto log_post = [&](double ll, double sg) {
        const double lam = 1.0 / (sg * sg);
        return ll + shape * std::log(lam) - rate * lam;
    };
    auto eval_ll = [&](double *ll) -> int {
        CHECK(evaluate(c));
        double s[kScalars];
        CU(cudaMemcpyAsync(s, c->scal, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        *ll = s[kLogLik];
        return MDS_OK;
    };
    double ll = 0.0;
    CHECK(eval_ll(&ll));
    double cur = log_post(ll, c->sigma);
    for (int t = 0; t < n_iter; ++t) {
        const double s0 = c->sigma;
        const double s1 = std::exp(std::log(s0) + step * z[t]);
        if (!(s1 > 0.0) || !std::isfinite(s1) || (!c->fp64 && (s1 < 1e-6 || s1 > 1e6))) {
            if (accepted) accepted[t] = 0;  // outside the supported range: rejected
            continue;
        }
        c->sigma = s1;
        c->gen++;
        c->grad_valid = false;
        double ll1 = 0.0;
        CHECK(eval_ll(&ll1));
        const double prop = log_post(ll1, s1);
        const int acc = std::log(u[t]) < prop - cur;
        if (acc) {
            cur = prop;
        } else {
            c->sigma = s0;
            c->gen++;
            c->grad_valid = false;  // the cached pass is at the rejected sigma
        }
        if (accepted) accepted[t] = acc;
    }
    return MDS_OK;
}

int mds_locality_order(int64_t n, int32_t d, const double *x, int32_t *perm) {
    if (n < 1 || n > INT32_MAX || d < 1 || d > 8 || !x || !perm) {
        mds::set_thread_error("mds_locality_order: need 1 <= n < 2^31, 1 <= d <= 8, x and perm");
        return MDS_ERR_INVALID_ARG;
    }
    for (int64_t e = 0; e < n * d; ++e)
        if (!std::isfinite(x[e])) {
            mds::set_thread_error("mds_locality_order: x[%lld] is not finite", (long long)e);
            return MDS_ERR_INVALID_ARG;
        }
    mds::locality_order(n, d, x, perm);
    return MDS_OK;
}

int mds_tree_plan_check(int64_t n, int64_t n_nodes, const int64_t *parent, const double *length, int32_t d,
                        int64_t *stats) {
    if (n < 1 || n > INT32_MAX || d < 1 || d > MDS_MAX_D || !parent || !length) {
        mds::set_thread_error("mds_tree_plan_check: need 1 <= n < 2^31, 1 <= d <= %d, parent and length", MDS_MAX_D);
        return MDS_ERR_INVALID_ARG;
    }
    ForestShape f;
    std::string err = parse_forest(n, n_nodes, parent, length, f);
    if (!err.empty()) {
        mds::set_thread_error("mds_tree_plan_check: %s", err.c_str());
        return MDS_ERR_INVALID_ARG;
    }
    std::vector<TreeWeights> wt;
    std::vector<double> root_cinv;
    double cst = 0.0;
    tree_weights(f, length, 1.0, 1.0, d, wt, root_cinv, cst);
    TreePlan plan;
    plan_forest(f, wt, d, plan);
    err = check_plan(f, plan, d);
    if (!err.empty()) {
        mds::set_thread_error("mds_tree_plan_check: plan violates %s", err.c_str());
        return MDS_ERR_STATE;
    }
    if (stats) {
        int64_t chain = 0, top = 0, blk = 0, slots = 0;
        for (size_t t = 0; t < f.roots.size(); ++t) {
            int64_t lb = 0;
            for (int cr = 0; cr < plan.cluster; ++cr) {
                const TreePart &pt = plan.parts[t * plan.cluster + cr];
                lb = std::max<int64_t>(lb, pt.nlv_blk);
                blk = std::max<int64_t>(blk, pt.m_blk);
            }
            const TreePart &p0 = plan.parts[t * plan.cluster];
            chain = std::max<int64_t>(chain, 2 * (lb + p0.nlv_top));
            top = std::max<int64_t>(top, p0.m_top);
            slots += p0.n_slots;
        }
        stats[0] = plan.cluster;
        stats[1] = static_cast<int64_t>(plan.parts.size());
        stats[2] = chain;
        stats[3] = plan.max_fp;
        stats[4] = slots;
        stats[5] = top;
        stats[6] = blk;
        stats[7] = static_cast<int64_t>(f.roots.size());
    }
    return MDS_OK;
}

namespace {
int reorder_ctx(mds_ctx *c, bool order_strips);
}

int mds_reorder(mds_ctx *c) { return reorder_ctx(c, true); }

}  // extern "C"

namespace {

// The locality order of the current locations; `order_strips`: then one
// counted pass and the strips in order of their cost (single contexts; a
// batch builds its own strip list).
int reorder_ctx(mds_ctx *c, bool order_strips) {
    CHECK(check_ctx(c));
    if (sharded(c))
        return fail(c, MDS_ERR_STATE, "a sharded context holds part of Y and cannot be reordered (permute X and Y "
                                      "before mds_set_data instead)");
    if (!c->y_owned) return fail(c, MDS_ERR_STATE, "the chains of a batch share Y and cannot be reordered");
    if (!c->have_data || !c->have_x) return fail(c, MDS_ERR_STATE, "mds_reorder needs data and locations");
    if (c->ho_count > 0)
        return fail(c, MDS_ERR_STATE, "a cross-validation fold is set: call mds_reorder before mds_set_heldout");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    const int64_t n = c->n, np = c->n_pad;
    std::vector<double> xh(static_cast<size_t>(n * c->d));
    CHECK(copy_out(c, c->x, c->fp64 ? 1 : 0, xh.data(), MDS_F64, MDS_HOST, n * c->d));
    std::vector<int32_t> order(static_cast<size_t>(np));
    locality_order(n, c->d, xh.data(), order.data());
    for (int64_t s = n; s < np; ++s) order[s] = static_cast<int32_t>(s);
    CHECK(repack_to(c, order, false));
    if (!c->fp64) {
        // split locations at their new slots
        cudaError_t e = launch_resplit(xstate(c), np, c->d, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "reorder: %s", cudaGetErrorString(e));
        // one counted pass at the autotuned strip length, then the strips in
        // order of their cost
        if (order_strips && c->have_sigma) {
            CHECK(evaluate(c));
            CHECK(order_strips_by_cost(c));
        }
    }
    return MDS_OK;
}

}  // namespace

extern "C" {

int mds_far_blocks(mds_ctx *c, int64_t *far, int64_t *total) {
    CHECK(check_ctx(c));
    if (!far || !total) return fail(c, MDS_ERR_INVALID_ARG, "far and total must not be NULL");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    CHECK(ready(c));
    CHECK(autotune(c));  // so that the counted pass is the only one
    CHECK(evaluate(c));
    int64_t v = 0;
    if (!c->fp64) {
        std::vector<int32_t> parts(static_cast<size_t>(c->n_strips) * kPairWarps);
        CU(cudaMemcpyAsync(parts.data(), c->far_part, parts.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           c->stream));
        CU(cudaStreamSynchronize(c->stream));
        for (int32_t p : parts) v += p;
    }
    *far = v;
    *total = c->tiles * kPairWarps * 2;  // column pairs of the 4 warps per tile
    return MDS_OK;
}

int mds_pair_body_ceiling(mds_ctx *c, int32_t far, double *pairs_per_s) {
    CHECK(check_ctx(c));
    if (!pairs_per_s) return fail(c, MDS_ERR_INVALID_ARG, "pairs_per_s must not be NULL");
    if (c->fp64) return fail(c, MDS_ERR_STATE, "the per-pair ceiling is measured for the FP32C pass");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    if (!(c->sigma > 0.0)) return fail(c, MDS_ERR_STATE, "sigma is not set (mds_set_sigma)");
    const PairArgs a = pair_args(c);
    const int grid = c->sm_count * pair_ceiling_blocks_per_sm(c->d);
    float *sink = nullptr;
    CHECK(dev_alloc_t(c, &sink, static_cast<size_t>(grid) * kPairThreads * sizeof(float)));
    // a short launch to warm up, then a timed one of 2e10 pair evaluations
    const int iters = std::max(64, static_cast<int>(2.0e10 / (16.0 * grid * kPairThreads)));
    cudaError_t e = launch_pair_ceiling(a, c->d, far != 0, grid, 64, sink, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev0, c->stream);
    if (e == cudaSuccess) e = launch_pair_ceiling(a, c->d, far != 0, grid, iters, sink, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(c->ev1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    dev_free(sink);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "pair ceiling: %s", cudaGetErrorString(e));
    *pairs_per_s = 16.0 * grid * kPairThreads * static_cast<double>(iters) / (ms * 1e-3);
    return MDS_OK;
}

int mds_get_order(const mds_ctx *c, int32_t *perm) {
    if (!c || !perm) return MDS_ERR_INVALID_ARG;
    for (int64_t s = 0; s < c->n; ++s) perm[s] = c->reordered ? c->perm_h[s] : static_cast<int32_t>(s);
    return MDS_OK;
}

int mds_set_tail_cutoff(mds_ctx *c, double z) {
    CHECK(check_ctx(c));
    if (!(z == 0.0 || z >= 8.0) || !std::isfinite(z))
        return fail(c, MDS_ERR_INVALID_ARG, "the Phi cut-off must be 0 (off) or a finite z >= 8, got %g", z);
    if (z != c->tail_z) {
        c->tail_z = z;
        c->gen++;
    }
    return MDS_OK;
}

int mds_set_tree_prior(mds_ctx *c, int64_t n_nodes, const int64_t *parent, const double *length,
                       const double *sigma_mat, const double *mu, double tau0, double tau_u) {
    CHECK(check_ctx(c));
    if (sharded(c)) return fail(c, MDS_ERR_STATE, "the tree prior is not available on a sharded context");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    const int64_t n = c->n;
    const int d = c->d;
    auto drop = [c]() {
        for (void *b : c->tree_bufs) dev_free(b);
        c->tree_bufs.clear();
        c->tree = TreeArgs{};
        c->tree_grad0 = nullptr;
        const double zero[2] = {0.0, 0.0};
        cudaMemcpyAsync(c->scal + kPriorLogp, zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        if (c->tree_on) c->gen++;
        c->tree_on = false;
        c->grad_valid = false;
    };
    if (n_nodes == 0 || !parent) {
        drop();
        return MDS_OK;
    }
    if (!length || !sigma_mat || !mu) return fail(c, MDS_ERR_INVALID_ARG, "length, Sigma and mu are required");
    if (n_nodes < n || n_nodes > 2 * n - 1)
        return fail(c, MDS_ERR_INVALID_ARG, "a binary forest over N = %lld tips has N to 2N-1 nodes, got %lld",
                    (long long)n, (long long)n_nodes);
    if (!(tau0 > 0.0) || !std::isfinite(tau0) || !(tau_u > 0.0) || !std::isfinite(tau_u))
        return fail(c, MDS_ERR_INVALID_ARG, "tau0 and tau_u must be finite and > 0");
    // ---- the forest
    ForestShape f;
    {
        const std::string err = parse_forest(n, n_nodes, parent, length, f);
        if (!err.empty()) return fail(c, MDS_ERR_INVALID_ARG, "%s", err.c_str());
    }
    // ---- Sigma: symmetric positive definite; its inverse and log-determinant
    std::vector<double> L(d * d, 0.0), sinv(d * d, 0.0);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            const double a = sigma_mat[i * d + j], b = sigma_mat[j * d + i];
            if (!std::isfinite(a) || std::fabs(a - b) > 1e-12 * (std::fabs(a) + std::fabs(b)))
                return fail(c, MDS_ERR_INVALID_ARG, "Sigma must be finite and symmetric");
        }
    double logdet = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = sigma_mat[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * d + k] * L[j * d + k];
        if (!(s > 0.0)) return fail(c, MDS_ERR_INVALID_ARG, "Sigma is not positive definite");
        L[j * d + j] = std::sqrt(s);
        logdet += std::log(s);
        for (int i = j + 1; i < d; ++i) {
            double t = sigma_mat[i * d + j];
            for (int k = 0; k < j; ++k) t -= L[i * d + k] * L[j * d + k];
            L[i * d + j] = t / L[j * d + j];
        }
    }
    for (int col = 0; col < d; ++col) {  // Sigma^-1 = L^-T L^-1, column by column
        std::vector<double> y(d, 0.0), z(d, 0.0);
        for (int i = 0; i < d; ++i) {
            double t = i == col ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= L[i * d + k] * y[k];
            y[i] = t / L[i * d + i];
        }
        for (int i = d - 1; i >= 0; --i) {
            double t = y[i];
            for (int k = i + 1; k < d; ++k) t -= L[k * d + i] * z[k];
            z[i] = t / L[i * d + i];
        }
        for (int i = 0; i < d; ++i) sinv[i * d + col] = z[i];
    }
    for (int k = 0; k < d; ++k)
        if (!std::isfinite(mu[k])) return fail(c, MDS_ERR_INVALID_ARG, "mu must be finite");
    // ---- message variances and weights; the cut into per-CTA parts
    std::vector<TreeWeights> wt;
    std::vector<double> root_cinv;
    double cst = 0.0;
    tree_weights(f, length, tau0, tau_u, d, wt, root_cinv, cst);
    cst -= 0.5 * static_cast<double>(n) * logdet;
    TreePlan plan;
    plan_forest(f, wt, d, plan);
    const std::vector<int32_t> &roots = f.roots, &lone = f.lone;
    const int ncl = plan.cluster;
    // ---- device copies
    drop();
    if (!c->tree_stream) {
        int lo = 0, hi = 0;
        CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CU(cudaStreamCreateWithPriority(&c->tree_stream, cudaStreamNonBlocking, hi));
        CU(cudaEventCreateWithFlags(&c->tree_fork, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&c->tree_join, cudaEventDisableTiming));
    }
    TreeArgs ta{};
    auto up = [&](void **dst, const void *src, size_t bytes) -> int {
        void *p = nullptr;
        int st = dev_alloc(c, &p, std::max<size_t>(bytes, 16));
        if (st != MDS_OK) return st;
        c->tree_bufs.push_back(p);
        if (src && bytes) {
            cudaError_t e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "tree prior upload: %s", cudaGetErrorString(e));
        }
        *dst = p;
        return MDS_OK;
    };
    void *p = nullptr;
    CHECK(up(&p, plan.nodes.data(), plan.nodes.size() * sizeof(TreeNode)));
    ta.nodes = static_cast<const TreeNode *>(p);
    CHECK(up(&p, plan.lv_start.data(), plan.lv_start.size() * sizeof(int32_t)));
    ta.lv_start = static_cast<const int32_t *>(p);
    CHECK(up(&p, plan.parts.data(), plan.parts.size() * sizeof(TreePart)));
    ta.parts = static_cast<const TreePart *>(p);
    CHECK(up(&p, plan.exp_loc.data(), plan.exp_loc.size() * sizeof(int32_t)));
    ta.exp_loc = static_cast<const int32_t *>(p);
    CHECK(up(&p, plan.exp_slot.data(), plan.exp_slot.size() * sizeof(int32_t)));
    ta.exp_slot = static_cast<const int32_t *>(p);
    CHECK(up(&p, nullptr, static_cast<size_t>(std::max<int64_t>(plan.xch_total, 1)) * sizeof(double)));
    ta.xch = static_cast<double *>(p);
    CHECK(up(&p, root_cinv.data(), root_cinv.size() * sizeof(double)));
    ta.root_cinv = static_cast<const double *>(p);
    CHECK(up(&p, lone.data(), lone.size() * sizeof(int32_t)));
    ta.lone = static_cast<const int32_t *>(p);
    CHECK(up(&p, sinv.data(), sinv.size() * sizeof(double)));
    ta.sigma_inv = static_cast<const double *>(p);
    CHECK(up(&p, mu, d * sizeof(double)));
    ta.mu = static_cast<const double *>(p);
    CHECK(up(&p, plan.node_off.data(), plan.node_off.size() * sizeof(int32_t)));
    ta.node_off = static_cast<const int32_t *>(p);
    CHECK(up(&p, plan.tip_items.data(), plan.tip_items.size() * sizeof(int32_t)));
    ta.tip_items = static_cast<const int32_t *>(p);
    CHECK(up(&p, plan.tip_off.data(), plan.tip_off.size() * sizeof(int32_t)));
    ta.tip_off = static_cast<const int32_t *>(p);
    // messages and tip locations: in shared memory when the largest part fits
    // (kTreeSmemMax bytes per CTA), else in global scratch
    constexpr int64_t kTreeSmemMax = 200 * 1024;
    if (plan.max_fp > 0 && plan.max_fp <= kTreeSmemMax) {
        ta.smem_bytes = static_cast<int32_t>((plan.max_fp + 15) / 16 * 16);
    } else {
        ta.smem_bytes = 0;
        CHECK(up(&p, nullptr, static_cast<size_t>(std::max<int64_t>(plan.scr_total, 1)) * sizeof(double)));
        ta.scratch = static_cast<double *>(p);
    }
    CHECK(up(&p, nullptr, static_cast<size_t>(c->n_pad) * d * sizeof(double)));
    ta.grad = static_cast<double *>(p);
    CHECK(up(&p, nullptr, static_cast<size_t>(c->n_pad) * d * sizeof(double)));
    c->tree_grad0 = static_cast<double *>(p);
    const size_t grid = (roots.size() + (lone.empty() ? 0 : 1)) * static_cast<size_t>(ncl);
    CHECK(up(&p, nullptr, (grid + 1) * sizeof(double)));
    ta.part = static_cast<double *>(p);
    ta.out = ta.part + grid;
    CU(cudaMemsetAsync(ta.grad, 0, static_cast<size_t>(c->n_pad) * d * sizeof(double), c->stream));
    CU(cudaStreamSynchronize(c->stream));
    // room for one traversal CTA beside three pass CTAs on every SM: the
    // pass's shared memory padded so that a fourth does not fit
    c->tree_pass_smem = 0;
    {
        int smem_sm = 0, reserved = 0;
        CU(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
        CU(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device));
        const int tree_cta = ta.smem_bytes + 1024 + reserved;  // dynamic + static (< 1 KB) + reserved
        const int pad = (smem_sm - tree_cta) / 3 - reserved;
        const int base = pair_f32_smem_bytes(d);
        // measured at D = 2, where the pass's registers allow 4 CTAs per SM and
        // 3 of them leave room for a traversal CTA's registers too; for
        // larger D the pass's register use leaves none, so it runs without PDL
        if (!c->fp64 && d <= 2 && base > 0 && pad >= base && 4 * (pad + reserved) > smem_sm) c->tree_pass_smem = pad;
    }
    ta.n = n;
    ta.n_trees = static_cast<int32_t>(roots.size());
    ta.cluster = ncl;
    ta.n_lone = static_cast<int32_t>(lone.size());
    ta.tau_u = tau_u;
    ta.const_term = cst;
    c->tree = ta;
    c->tree_on = true;
    c->gen++;
    c->grad_valid = false;
    return MDS_OK;
}

int mds_tree_prior(mds_ctx *c, double *logp, void *grad, int dtype, int where) {
    CHECK(check_ctx(c));
    if (!c->tree_on) return fail(c, MDS_ERR_STATE, "no tree prior: call mds_set_tree_prior first");
    if (!c->have_x) return fail(c, MDS_ERR_STATE, "no locations set");
    if (grad) CHECK(valid_enums(c, dtype, where));
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    TreeArgs ta = c->tree;
    ta.x = c->x;
    ta.x_f64 = c->fp64;
    cudaError_t e = launch_tree_prior(ta, c->d, c->stream);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "tree prior: %s", cudaGetErrorString(e));
    if (grad) CHECK(copy_out(c, ta.grad, 1, grad, dtype, where, c->n * c->d));
    if (logp) {
        CU(cudaMemcpyAsync(logp, ta.out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return MDS_OK;
}

int mds_rwmh(mds_ctx *c, int n_prop, double step, uint64_t seed, const int64_t *items, const double *z_all,
             const double *u_all, int32_t *accepted, double *dlogpi) {
    CHECK(check_ctx(c));
    if (sharded(c)) return fail(c, MDS_ERR_STATE, "the random-walk sampler is not available on a sharded context");
    if (n_prop < 0) return fail(c, MDS_ERR_INVALID_ARG, "n_prop must be >= 0");
    if (!(step > 0.0) || !std::isfinite(step)) return fail(c, MDS_ERR_INVALID_ARG, "step must be finite and > 0");
    const bool inj = items || z_all || u_all;
    if (inj && !(items && z_all && u_all))
        return fail(c, MDS_ERR_INVALID_ARG, "inject all of items, z and u, or none");
    CHECK(ready(c));
    if (c->tree_on)
        return fail(c, MDS_ERR_STATE, "the random-walk sampler supports the isotropic prior only (no tree prior)");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    if (n_prop == 0) return MDS_OK;
    const int d = c->d;
    if (inj)
        for (int t = 0; t < n_prop; ++t)
            if (items[t] < 0 || items[t] >= c->n)
                return fail(c, MDS_ERR_INVALID_ARG, "items[%d] = %lld is not an item", t, (long long)items[t]);
    // device copies of the draws and the outputs (freed below)
    std::vector<void *> tmp;
    auto alloc = [&](void **p, size_t bytes) -> int {
        int st = dev_alloc(c, p, std::max<size_t>(bytes, 16));
        if (st == MDS_OK) tmp.push_back(*p);
        return st;
    };
    auto cleanup = [&](int st) {
        for (void *p : tmp) dev_free(p);
        return st;
    };
    RwmhArgs a{};
    void *p = nullptr;
    {
        int st;
        if ((st = alloc(&p, n_prop * sizeof(int64_t)))) return cleanup(st);
        a.items = static_cast<const int64_t *>(p);
        if ((st = alloc(&p, static_cast<size_t>(n_prop) * d * sizeof(double)))) return cleanup(st);
        a.z = static_cast<const double *>(p);
        if ((st = alloc(&p, n_prop * sizeof(double)))) return cleanup(st);
        a.logu = static_cast<const double *>(p);
    }
    if (inj) {
        std::vector<double> lu(n_prop);
        for (int t = 0; t < n_prop; ++t) lu[t] = std::log(u_all[t]);
        cudaError_t e = cudaMemcpyAsync(const_cast<int64_t *>(a.items), items, n_prop * sizeof(int64_t),
                                        cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(const_cast<double *>(a.z), z_all, static_cast<size_t>(n_prop) * d * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(const_cast<double *>(a.logu), lu.data(), n_prop * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // lu goes out of scope
        if (e != cudaSuccess) return cleanup(fail(c, MDS_ERR_CUDA, "rwmh: %s", cudaGetErrorString(e)));
    }
    int st;
    if ((st = alloc(&p, n_prop * sizeof(int32_t)))) return cleanup(st);
    a.acc_out = static_cast<int32_t *>(p);
    if ((st = alloc(&p, n_prop * sizeof(double)))) return cleanup(st);
    a.dl_out = static_cast<double *>(p);
    a.n = c->n;
    a.y = c->y;
    a.nt = static_cast<int32_t>(c->nt);
    a.inv = c->reordered ? c->inv_d : nullptr;
    a.perm = c->reordered ? c->perm_d : nullptr;
    a.x = c->x;
    a.fp64 = c->fp64;
    a.sigma = c->sigma;
    a.lambda = c->lambda;
    a.step = step;
    a.n_prop = n_prop;
    a.seed = seed;
    a.chain = 0;
    a.iter0 = c->rw_iter;
    a.xmax_bits = c->fp64 ? nullptr : c->xmax_bits;
    a.err = c->err;
    {
        const PairArgs pa = pair_args(c);  // the FP32 Phi constants of the pass
        for (int k = 0; k < 4; ++k) {
            a.mp[k] = pa.mp[k].x;
            a.md[k] = pa.md[k].x;
        }
        a.c_phi = pa.c_phi.x;
    }
    // X in shared memory when it fits (160 KB)
    a.x_in_smem = static_cast<int64_t>(c->n) * d * static_cast<int64_t>(elem(c)) <= 160 * 1024;
    // one 1024-thread CTA per 1024 slots of the row, up to a cluster of 8,
    // each CTA with its own copy of X (so only when X fits in shared memory)
    a.cluster = a.x_in_smem ? static_cast<int32_t>(std::min<int64_t>(8, std::max<int64_t>(1, (c->n + 1023) / 1024))) : 1;
    cudaError_t e = cudaSuccess;
    if (!inj)
        e = launch_rwmh_draws(a, d, const_cast<int64_t *>(a.items), const_cast<double *>(a.z),
                              const_cast<double *>(a.logu), c->stream);
    if (e == cudaSuccess) e = launch_rwmh(a, d, c->stream);
    if (e != cudaSuccess) return cleanup(fail(c, MDS_ERR_CUDA, "rwmh: %s", cudaGetErrorString(e)));
    std::vector<int32_t> acc(n_prop);
    std::vector<double> dl(n_prop);
    e = cudaMemcpyAsync(acc.data(), a.acc_out, n_prop * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dl.data(), a.dl_out, n_prop * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup(MDS_OK);
    if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "rwmh: %s", cudaGetErrorString(e));
    if (!inj) c->rw_iter += n_prop;
    c->grad_valid = false;
    CHECK(check_device_err(c, "rwmh"));
    if (!c->fp64) CHECK(set_split_from_xmax(c));  // the split layouts follow the moved items
    if (accepted) std::memcpy(accepted, acc.data(), n_prop * sizeof(int32_t));
    if (dlogpi) std::memcpy(dlogpi, dl.data(), n_prop * sizeof(double));
    return MDS_OK;
}

namespace {
// Layout of a state snapshot (host bytes): this header, then X and p
// (N x D FP64 each, the caller's item order), then the order (N int32) when
// the context is reordered.
struct StateHeader {
    uint64_t magic;
    int64_t n;
    int32_t d, fp64;
    double sigma, lambda, tail_z;
    int64_t counters[kCounters];
    int64_t sigma_iter, rw_iter;
    int32_t reordered, have_sigma;
};
constexpr uint64_t kStateMagic = 0x3154415453534D44ull;  // "DMSSTAT1"

int64_t state_bytes(const mds_ctx *c) {
    return static_cast<int64_t>(sizeof(StateHeader)) + 2 * c->n * c->d * 8 + (c->reordered ? c->n * 4 : 0);
}
}  // namespace

int mds_get_state(mds_ctx *c, void *buf, int64_t *bytes) {
    CHECK(check_ctx(c));
    if (!bytes) return fail(c, MDS_ERR_INVALID_ARG, "bytes is NULL");
    const int64_t need = state_bytes(c);
    if (!buf) {
        *bytes = need;
        return MDS_OK;
    }
    if (*bytes < need) return fail(c, MDS_ERR_INVALID_ARG, "state buffer holds %lld bytes, %lld needed",
                                   (long long)*bytes, (long long)need);
    if (!c->have_x) return fail(c, MDS_ERR_STATE, "no locations set");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    StateHeader h{};
    h.magic = kStateMagic;
    h.n = c->n;
    h.d = c->d;
    h.fp64 = c->fp64 ? 1 : 0;
    h.sigma = c->sigma;
    h.lambda = c->lambda;
    h.tail_z = c->tail_z;
    CU(cudaMemcpyAsync(h.counters, c->counters, sizeof(h.counters), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    h.sigma_iter = c->sigma_iter;
    h.rw_iter = c->rw_iter;
    h.reordered = c->reordered ? 1 : 0;
    h.have_sigma = c->have_sigma ? 1 : 0;
    unsigned char *out = static_cast<unsigned char *>(buf);
    std::memcpy(out, &h, sizeof(h));
    double *xd = reinterpret_cast<double *>(out + sizeof(h));
    const int64_t nd = c->n * c->d;
    CHECK(copy_out(c, c->x, c->fp64 ? 1 : 0, xd, MDS_F64, MDS_HOST, nd));
    CHECK(copy_out(c, c->p, c->fp64 ? 1 : 0, xd + nd, MDS_F64, MDS_HOST, nd));
    if (c->reordered) std::memcpy(xd + 2 * nd, c->perm_h.data(), c->n * 4);
    *bytes = need;
    return MDS_OK;
}

int mds_set_state(mds_ctx *c, const void *buf, int64_t bytes) {
    CHECK(check_ctx(c));
    if (!buf || bytes < static_cast<int64_t>(sizeof(StateHeader)))
        return fail(c, MDS_ERR_INVALID_ARG, "not a state snapshot (too short)");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic) return fail(c, MDS_ERR_INVALID_ARG, "not a state snapshot (bad magic)");
    if (h.n != c->n || h.d != c->d || (h.fp64 != 0) != c->fp64)
        return fail(c, MDS_ERR_INVALID_ARG, "snapshot of N = %lld, D = %d (%s) does not fit this context",
                    (long long)h.n, h.d, h.fp64 ? "FP64" : "FP32C");
    const int64_t nd = c->n * c->d;
    const int64_t need = static_cast<int64_t>(sizeof(StateHeader)) + 2 * nd * 8 + (h.reordered ? c->n * 4 : 0);
    if (bytes < need) return fail(c, MDS_ERR_INVALID_ARG, "snapshot truncated (%lld of %lld bytes)",
                                  (long long)bytes, (long long)need);
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    if (c->ho_count > 0 && h.reordered)
        return fail(c, MDS_ERR_STATE, "a cross-validation fold is set: restore the state before mds_set_heldout");
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    const double *xd = reinterpret_cast<const double *>(in + sizeof(h));
    if (h.have_sigma) CHECK(mds_set_sigma(c, h.sigma));
    CHECK(mds_set_prior(c, h.lambda));
    CHECK(mds_set_tail_cutoff(c, h.tail_z));
    CHECK(mds_set_locations(c, xd, MDS_F64, MDS_HOST));
    CHECK(mds_set_momentum(c, xd + nd, MDS_F64, MDS_HOST));
    if (h.reordered && c->have_data) {
        std::vector<int32_t> order(static_cast<size_t>(c->n_pad));
        std::memcpy(order.data(), xd + 2 * nd, c->n * 4);
        for (int64_t s = c->n; s < c->n_pad; ++s) order[s] = static_cast<int32_t>(s);
        if (!c->reordered || order != c->perm_h) {
            CHECK(repack_to(c, order, false));
            if (!c->fp64) {
                cudaError_t e = launch_resplit(xstate(c), c->n_pad, c->d, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) return fail(c, MDS_ERR_CUDA, "set_state: %s", cudaGetErrorString(e));
            }
        }
    }
    int64_t cnt[kCounters];
    std::memcpy(cnt, h.counters, sizeof(cnt));
    cnt[kIterLocal] = 0;
    CU(cudaMemcpyAsync(c->counters, cnt, sizeof(cnt), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->sigma_iter = h.sigma_iter;
    c->rw_iter = h.rw_iter;
    c->grad_valid = false;
    c->gen++;
    return MDS_OK;
}

int mds_problem_size(const mds_ctx *c, int64_t *pairs, int64_t *y_bytes) {
    if (!c) return MDS_ERR_INVALID_ARG;
    if (pairs) *pairs = c->n * (c->n - 1) / 2;
    if (y_bytes) *y_bytes = (c->shard_t1 - c->shard_t0) * kTileElems * static_cast<int64_t>(sizeof(float));
    return MDS_OK;
}

int mds_set_strip(mds_ctx *c, int32_t strip) {
    CHECK(check_ctx(c));
    if (strip < 0) return fail(c, MDS_ERR_INVALID_ARG, "strip must be >= 0");
    if (strip > kMaxStrip) return fail(c, MDS_ERR_INVALID_ARG, "strip %d exceeds the limit %d", strip, kMaxStrip);
    c->strip_req = strip;
    c->chunk_req = 0;
    c->chunk_grouped_req = false;
    if (strip > 0) CHECK(apply_shape(c, kPassStrips, strip));
    return MDS_OK;
}

int mds_get_strip(const mds_ctx *c, int32_t *strip) {
    if (!c || !strip) return MDS_ERR_INVALID_ARG;
    *strip = c->strip;
    return MDS_OK;
}

int mds_set_pass_shape(mds_ctx *c, int32_t kind, int32_t param) {
    CHECK(check_ctx(c));
    if (kind != MDS_PASS_STRIPS && kind != MDS_PASS_CHUNKS && kind != MDS_PASS_CHUNK_COUNT &&
        kind != MDS_PASS_SM_CHUNKS)
        return fail(c, MDS_ERR_INVALID_ARG,
                    "kind must be MDS_PASS_STRIPS, MDS_PASS_CHUNKS, MDS_PASS_CHUNK_COUNT or MDS_PASS_SM_CHUNKS");
    if (param < 0) return fail(c, MDS_ERR_INVALID_ARG, "param must be >= 0");
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    if (kind == MDS_PASS_STRIPS) {
        if (param > kMaxStrip) return fail(c, MDS_ERR_INVALID_ARG, "strip %d exceeds the limit %d", param, kMaxStrip);
        c->chunk_req = 0;
        c->chunk_grouped_req = false;
        c->strip_req = param;
        if (param > 0) CHECK(apply_shape(c, kPassStrips, param));
    } else {
        if (c->fp64) return fail(c, MDS_ERR_INVALID_ARG, "the FP64 context has the strip pass only");
        if ((kind == MDS_PASS_CHUNKS || kind == MDS_PASS_SM_CHUNKS) && param > 8)
            return fail(c, MDS_ERR_INVALID_ARG, "chunks per slot must be <= 8, got %d", param);
        if (kind == MDS_PASS_CHUNK_COUNT && param == 0)
            return fail(c, MDS_ERR_INVALID_ARG, "MDS_PASS_CHUNK_COUNT needs a chunk count >= 1");
        c->strip_req = 0;
        c->chunk_req = kind == MDS_PASS_CHUNK_COUNT ? -param : param;
        c->chunk_grouped_req = kind == MDS_PASS_SM_CHUNKS && param > 0;
        if (param > 0) CHECK(apply_shape(c, c->chunk_grouped_req ? kPassChunksSM : kPassChunks, c->chunk_req));
    }
    c->grad_valid = false;
    return MDS_OK;
}

int mds_get_pass_shape(const mds_ctx *c, int32_t *kind, int32_t *param, int32_t *ctas) {
    if (!c) return MDS_ERR_INVALID_ARG;
    const bool counted = c->pass_kind == kPassChunks && c->chunk_mult < 0;
    const bool grouped = c->pass_kind == kPassChunks && c->chunk_grouped;
    if (kind) *kind = counted ? MDS_PASS_CHUNK_COUNT : grouped ? MDS_PASS_SM_CHUNKS : c->pass_kind;
    if (param) *param = c->pass_kind == kPassChunks ? (counted ? -c->chunk_mult : c->chunk_mult) : c->strip;
    if (ctas) {
        // the grouped form launches one CTA per pair_chunk_groups(d) chunks
        // (one group alone beside a tree prior)
        const int g = grouped && !c->tree_on ? pair_chunk_groups(c->d) : 1;
        *ctas = (c->n_strips + g - 1) / g;
    }
    return MDS_OK;
}

int mds_set_pass_stamps(mds_ctx *c, int on) {
    CHECK(check_ctx(c));
    if (c->hmc_pending > 0 || !c->acc_spill.empty())
        return fail(c, MDS_ERR_STATE, "queued HMC iterations: collect them first (mds_hmc_collect)");
    const unsigned long long init[2] = {~0ull, 0ull};
    const double zero[2] = {0.0, 0.0};
    CU(cudaMemcpyAsync(c->stamps, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->pass_ns, zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (c->stamping != (on != 0)) c->gen++;  // captured launches carry the stamp pointers
    c->stamping = on != 0;
    return MDS_OK;
}

int mds_shard_range(int64_t n, int32_t n_ranks, int32_t rank, int64_t *t0, int64_t *t1) {
    if (n < 2 || n_ranks < 1 || rank < 0 || rank >= n_ranks || !t0 || !t1) {
        set_thread_error("mds_shard_range: need N >= 2, n_ranks >= 1, 0 <= rank < n_ranks, non-NULL t0, t1");
        return MDS_ERR_INVALID_ARG;
    }
    const std::vector<int64_t> b = shard_bounds(n, n_ranks);
    *t0 = b[rank];
    *t1 = b[rank + 1];
    return MDS_OK;
}

int mds_shard_sum(int32_t n_ranks, int64_t count, const double *gathered, double *out) {
    if (n_ranks < 1 || count < 0 || (count > 0 && (!gathered || !out))) {
        set_thread_error("mds_shard_sum: need n_ranks >= 1, count >= 0, non-NULL buffers");
        return MDS_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < count; ++i) {
        double v = gathered[i];
        for (int32_t r = 1; r < n_ranks; ++r) v += gathered[static_cast<int64_t>(r) * count + i];
        out[i] = v;
    }
    return MDS_OK;
}

int mds_set_shard(mds_ctx *c, int32_t n_ranks, int32_t rank, mds_allgather_fn allgather, void *user,
                  int32_t where_buffers) {
    CHECK(check_ctx(c));
    if (n_ranks < 1 || rank < 0 || rank >= n_ranks)
        return fail(c, MDS_ERR_INVALID_ARG, "need n_ranks >= 1 and 0 <= rank < n_ranks (got %d, %d)", n_ranks, rank);
    if (n_ranks > 1 && !allgather) return fail(c, MDS_ERR_INVALID_ARG, "allgather must not be NULL for n_ranks > 1");
    if (where_buffers != MDS_HOST && where_buffers != MDS_DEVICE)
        return fail(c, MDS_ERR_INVALID_ARG, "where_buffers must be MDS_HOST or MDS_DEVICE");
    if (c->have_data) return fail(c, MDS_ERR_STATE, "mds_set_shard must precede mds_set_data");
    if (!c->y_owned) return fail(c, MDS_ERR_STATE, "the chains of a batch cannot be sharded");
    if (c->reordered || c->ho_count > 0 || c->tree_on)
        return fail(c, MDS_ERR_STATE, "a reordered context, a fold or a tree prior cannot be sharded");
    const std::vector<int64_t> b = shard_bounds(c->n, n_ranks);
    const int64_t t0 = b[rank], t1 = b[rank + 1];
    // Y for the range only
    dev_free(c->y);
    c->y = nullptr;
    if (t1 > t0) CHECK(dev_alloc_t(c, &c->y, static_cast<size_t>(t1 - t0) * kTileElems * sizeof(float)));
    // column partials outside the range are never written: zero once
    CU(cudaMemsetAsync(c->col_part, 0, static_cast<size_t>(c->tiles) * kTile * c->d * elem(c), c->stream));
    const int64_t count = 3 + c->n * c->d;
    dev_free(c->shard_send);
    dev_free(c->shard_recv);
    c->shard_send = c->shard_recv = nullptr;
    if (c->shard_hsend) cudaFreeHost(c->shard_hsend);
    if (c->shard_hrecv) cudaFreeHost(c->shard_hrecv);
    c->shard_hsend = c->shard_hrecv = nullptr;
    if (n_ranks > 1) {
        CHECK(dev_alloc_t(c, &c->shard_send, count * sizeof(double)));
        CHECK(dev_alloc_t(c, &c->shard_recv, static_cast<size_t>(n_ranks) * count * sizeof(double)));
        if (where_buffers == MDS_HOST) {
            if (cudaMallocHost(&c->shard_hsend, count * sizeof(double)) != cudaSuccess ||
                cudaMallocHost(&c->shard_hrecv, static_cast<size_t>(n_ranks) * count * sizeof(double)) != cudaSuccess)
                return fail(c, MDS_ERR_OOM, "pinned host buffers of the exchange");
        }
    }
    c->shard_n = n_ranks;
    c->shard_rank = rank;
    c->shard_t0 = t0;
    c->shard_t1 = t1;
    c->shard_pairs = range_pairs(c->n, c->nt, t0, t1);
    c->shard_fn = allgather;
    c->shard_user = user;
    c->shard_where = where_buffers;
    c->tile_cost.clear();
    c->grad_valid = false;
    // the pass shape over the new range (fixed for shards: see autotune)
    if (c->fp64 || c->strip_req > 0)
        CHECK(build_strips(c, c->strip_req > 0 ? c->strip_req : (c->strip > 0 ? c->strip : 2)));
    else
        CHECK(build_chunks(c, c->chunk_req != 0 ? c->chunk_req : 1, false));
    CU(cudaStreamSynchronize(c->stream));
    return MDS_OK;
}

int mds_get_pass_span(mds_ctx *c, int64_t *passes, double *total_ms) {
    CHECK(check_ctx(c));
    double v[2] = {0.0, 0.0};
    CU(cudaMemcpyAsync(v, c->pass_ns, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (passes) *passes = static_cast<int64_t>(v[1]);
    if (total_ms) *total_ms = v[0] * 1e-6;
    return MDS_OK;
}

int mds_time_pass(mds_ctx *c, int reps, double *ms_per_pass) {
    CHECK(check_ctx(c));
    if (reps < 1 || !ms_per_pass) return fail(c, MDS_ERR_INVALID_ARG, "reps must be >= 1 and ms_per_pass non-NULL");
    CHECK(ready(c));
    CHECK(autotune(c));
    const bool prof = c->profiling;
    c->profiling = false;
    CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
    CU(cudaEventRecord(c->ev0, c->stream));
    for (int r = 0; r < reps; ++r) CHECK(enqueue_pass(c, kModeEval, 0.0, c->stream));
    CU(cudaEventRecord(c->ev1, c->stream));
    CU(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    *ms_per_pass = ms / reps;
    c->profiling = prof;
    c->grad_valid = true;
    return check_device_err(c, "time_pass");
}

int mds_set_profiling(mds_ctx *c, int on) {
    CHECK(check_ctx(c));
    c->profiling = on != 0;
    c->prof_used = 0;
    c->prof_launches = 0;
    c->prof_ms = 0.0;
    return MDS_OK;
}

int mds_get_pass_time(const mds_ctx *c, int64_t *launches, double *total_ms) {
    if (!c) return MDS_ERR_INVALID_ARG;
    if (launches) *launches = c->prof_launches;
    if (total_ms) *total_ms = c->prof_ms;
    return MDS_OK;
}

const char *mds_last_error(const mds_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->last_error.c_str();
}

}  // extern "C"

// ====================================================================== batch
//
// A batch is a set of datasets, each with its own chains.  Every chain is a
// full context (locations, momenta, gradient, partial sums, counters); the
// chains of a dataset share that dataset's tile-packed Y (owned by its first
// chain).  Batched launches read per-chain argument tables in device memory,
// so one launch per step serves all chains.

struct mds_batch {
    int32_t n_data = 0, d = 0;
    std::vector<int64_t> n;
    std::vector<int32_t> chains, chain0;
    std::vector<mds_ctx *> ctx;  // dataset-major
    int device = 0, sm_count = 0;
    std::string device_name;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int32_t strip = 0, strip_req = 0;  // > 0: the batched strip kernel; < 0: per-chain chunked passes
                                       // of about -strip tiles per chunk
    cudaEvent_t fork = nullptr;        // per-chain passes: fork from the batch stream ...
    std::vector<cudaEvent_t> joins;    // ... and join back, one event per chain
    BatchDataset *ds_dev = nullptr;
    BatchChain *ch_dev = nullptr;
    BatchStrip *strips_dev = nullptr;
    size_t strips_cap = 0;
    int32_t n_strips = 0;
    ReduceArgs *rcfg = nullptr;
    int2 *jobs = nullptr;
    size_t jobs_cap = 0;
    int32_t n_jobs = 0;
    TrajArgs *tcfg = nullptr;
    AcceptArgs *acfg = nullptr;
    int32_t *acc_out = nullptr;
    double *dh_out = nullptr;
    size_t out_cap = 0;
    int grid = 0;              // persistent grid of the batched pair pass
    int max_start_grid = 0;
    int64_t max_nd = 0;
    uint64_t gen = 1;
    cudaGraphExec_t graph = nullptr;
    std::tuple<uint64_t, int> graph_key{};
    std::string last_error = "no error";
};

namespace {

int bfail(mds_batch *b, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b)
        b->last_error = buf;
    else
        g_create_error = buf;
    return code;
}

#define BCU(call)                                                                                                 \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess)                                                                                    \
            return bfail(b, MDS_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Run a context-level call and carry its message up to the batch.
int bpass(mds_batch *b, mds_ctx *c, int st) {
    if (st != MDS_OK) b->last_error = c->last_error;
    return st;
}
#define BCHECK(c, call)                      \
    do {                                     \
        int s_ = bpass(b, (c), (call));      \
        if (s_ != MDS_OK) return s_;         \
    } while (0)

int batch_chain(mds_batch *b, int32_t dataset, int32_t chain, mds_ctx **c) {
    if (!b) return MDS_ERR_INVALID_ARG;
    if (dataset < 0 || dataset >= b->n_data) return bfail(b, MDS_ERR_INVALID_ARG, "dataset %d out of range", dataset);
    if (chain < 0 || chain >= b->chains[dataset]) return bfail(b, MDS_ERR_INVALID_ARG, "chain %d out of range", chain);
    *c = b->ctx[b->chain0[dataset] + chain];
    BCU(cudaSetDevice(b->device));
    return MDS_OK;
}

template <typename P>
int bdev_alloc(mds_batch *b, P **p, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, e == cudaErrorMemoryAllocation ? MDS_ERR_OOM : MDS_ERR_CUDA, "cudaMalloc of %zu bytes: %s",
                     bytes, cudaGetErrorString(e));
    }
    *p = static_cast<P *>(v);
    return MDS_OK;
}

// Bring every chain to the batch strip length, refresh the location splits,
// and (re)build the device tables of the batched pair pass and reduction.
int batch_tables(mds_batch *b, int strip) {
    const int total = static_cast<int>(b->ctx.size());
    for (mds_ctx *c : b->ctx) {
        CHECK(bpass(b, c, ready(c)));
        if (strip < 0) {
            // each chain's own chunked pass: about -strip tiles per chunk
            const int32_t G = static_cast<int32_t>(std::max<int64_t>(1, c->tiles / (-strip)));
            if (c->pass_kind != kPassChunks || c->chunk_mult != -G || c->chunk_grouped)
                CHECK(bpass(b, c, build_chunks(c, -G, false)));
            continue;
        }
        c->strip_req = strip;
        if (c->pass_kind != kPassStrips || c->strip != strip) CHECK(bpass(b, c, build_strips(c, strip)));
    }
    std::vector<BatchDataset> ds(b->n_data);
    std::vector<BatchChain> ch(total);
    std::vector<BatchStrip> st;
    std::vector<int2> jobs;
    std::vector<ReduceArgs> rc(total);
    for (int dd = 0; dd < b->n_data; ++dd) {
        const mds_ctx *c0 = b->ctx[b->chain0[dd]];
        const PairArgs pa = pair_args(c0);
        BatchDataset &x = ds[dd];
        x.y = c0->y;
        x.n = c0->n;
        x.nt = static_cast<int32_t>(c0->nt);
        x.chain0 = b->chain0[dd];
        x.n_chains = b->chains[dd];
        for (int k = 0; k < 4; ++k) {
            x.mp[k] = pa.mp[k];
            x.md[k] = pa.md[k];
        }
        x.c_phi = pa.c_phi;
        x.neg_inv_s2 = pa.neg_inv_s2;
        x.m_coef = pa.m_coef;
        for (size_t i = 0; strip > 0 && i < c0->strips_host.size(); ++i) {
            const Strip &s = c0->strips_host[i];
            st.push_back(BatchStrip{dd, s.I, s.j0, s.j1, s.row_slot, static_cast<int32_t>(i)});
        }
    }
    std::stable_sort(st.begin(), st.end(),
                     [](const BatchStrip &p, const BatchStrip &q) { return (p.j1 - p.j0) > (q.j1 - q.j0); });
    for (int g = 0; g < total; ++g) {
        const mds_ctx *c = b->ctx[g];
        ch[g] = BatchChain{c->xrow, c->xcol, static_cast<float *>(c->row_part), static_cast<float *>(c->col_part),
                           static_cast<float *>(c->scal_part)};
        rc[g] = reduce_args(c, kModeEval, 0.0);
        for (int J = 0; J < c->nt * kReduceQuarters; ++J) jobs.push_back(make_int2(g, J));
        jobs.push_back(make_int2(g, -1));
    }
    if (st.size() > b->strips_cap) {
        if (b->strips_dev) cudaFree(b->strips_dev);
        b->strips_dev = nullptr;
        CHECK(bdev_alloc(b, &b->strips_dev, st.size() * sizeof(BatchStrip)));
        b->strips_cap = st.size();
        b->gen++;
    }
    if (jobs.size() > b->jobs_cap) {
        if (b->jobs) cudaFree(b->jobs);
        b->jobs = nullptr;
        CHECK(bdev_alloc(b, &b->jobs, jobs.size() * sizeof(int2)));
        b->jobs_cap = jobs.size();
        b->gen++;
    }
    BCU(cudaMemcpyAsync(b->ds_dev, ds.data(), ds.size() * sizeof(BatchDataset), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->ch_dev, ch.data(), ch.size() * sizeof(BatchChain), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->strips_dev, st.data(), st.size() * sizeof(BatchStrip), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->jobs, jobs.data(), jobs.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->rcfg, rc.data(), rc.size() * sizeof(ReduceArgs), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    if (static_cast<int32_t>(st.size()) != b->n_strips || static_cast<int32_t>(jobs.size()) != b->n_jobs ||
        strip != b->strip)
        b->gen++;
    b->n_strips = static_cast<int32_t>(st.size());
    b->n_jobs = static_cast<int32_t>(jobs.size());
    b->strip = strip;
    if (strip < 0) return MDS_OK;
    const int per_sm = pair_batch_blocks_per_sm(b->d, strip);
    if (per_sm <= 0) return bfail(b, MDS_ERR_CUDA, "batched pass does not fit on an SM (strip %d)", strip);
    b->grid = std::min(b->n_strips, per_sm * b->sm_count);
    return MDS_OK;
}

BatchPairArgs batch_pair_args(const mds_batch *b) {
    BatchPairArgs a{};
    a.ds = b->ds_dev;
    a.ch = b->ch_dev;
    a.strips = b->strips_dev;
    a.n_strips = b->n_strips;
    a.strip_cap = b->strip;
    a.err = b->ctx[0]->err;
    return a;
}

int batch_enqueue_pass(mds_batch *b, int mode, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (b->strip < 0) {
        // every chain's chunked pass on its own stream (graph branches when
        // captured), all after the work before on s, all before the reduction
        e = cudaEventRecord(b->fork, s);
        for (size_t g = 0; e == cudaSuccess && g < b->ctx.size(); ++g) {
            mds_ctx *c = b->ctx[g];
            e = cudaStreamWaitEvent(c->cap_stream, b->fork, 0);
            if (e == cudaSuccess) e = launch_pair_chunks_f32(pair_args(c), static_cast<int>(b->d), c->cap_stream, false, 0);
            if (e == cudaSuccess) e = cudaEventRecord(b->joins[g], c->cap_stream);
        }
        for (size_t g = 0; e == cudaSuccess && g < b->ctx.size(); ++g) e = cudaStreamWaitEvent(s, b->joins[g], 0);
    } else {
        e = launch_pair_batch(batch_pair_args(b), b->d, b->grid, s);
    }
    if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batched pair pass: %s", cudaGetErrorString(e));
    e = launch_reduce_batch(b->rcfg, b->jobs, b->n_jobs, b->d, mode, s);
    if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batched reduction: %s", cudaGetErrorString(e));
    return MDS_OK;
}

int batch_check_errors(mds_batch *b, const char *what) {
    BCU(cudaStreamSynchronize(b->stream));
    for (mds_ctx *c : b->ctx) CHECK(bpass(b, c, check_device_err(c, what)));
    return MDS_OK;
}

std::mutex g_btune_mu;
std::map<std::tuple<std::string, std::vector<int64_t>, int>, int> g_btune_cache;

// Batch strip length: forced, cached, or timed over a few candidates.
int batch_autotune(mds_batch *b) {
    int s = b->strip_req;
    if (s == 0) {
        const auto key = std::make_tuple(b->device_name, b->n, static_cast<int>(b->d));
        {
            std::lock_guard<std::mutex> lk(g_btune_mu);
            auto it = g_btune_cache.find(key);
            if (it != g_btune_cache.end()) s = it->second;
        }
        if (s == 0) {
            float best_ms = 1e30f;
            // each candidate timed as the HMC runs it: a captured graph of
            // five passes with their reductions (the per-chain shapes launch
            // one kernel per chain, which eager launches would slow)
            for (int cand : {1, 2, 3, 4, -2, -4, -6, -8, -16}) {
                if (cand > 0 && pair_batch_blocks_per_sm(b->d, cand) <= 0) continue;
                CHECK(batch_tables(b, cand));
                CHECK(batch_enqueue_pass(b, kModeEval, b->stream));
                cudaGraph_t g = nullptr;
                BCU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
                int st = MDS_OK;
                for (int w = 0; w < 5 && st == MDS_OK; ++w) st = batch_enqueue_pass(b, kModeEval, b->cap_stream);
                cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
                if (st != MDS_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch autotune capture: %s", cudaGetErrorString(e));
                cudaGraphExec_t ge = nullptr;
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch autotune graph: %s", cudaGetErrorString(e));
                float ms = 0.f;
                e = cudaGraphLaunch(ge, b->stream);
                if (e == cudaSuccess) e = cudaEventRecord(b->ev0, b->stream);
                if (e == cudaSuccess) e = cudaGraphLaunch(ge, b->stream);
                if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
                cudaGraphExecDestroy(ge);
                if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch autotune timing: %s", cudaGetErrorString(e));
                if (ms < best_ms) {
                    best_ms = ms;
                    s = cand;
                }
            }
            CHECK(batch_check_errors(b, "batch autotune"));
            std::lock_guard<std::mutex> lk(g_btune_mu);
            g_btune_cache[key] = s;
        }
    }
    return batch_tables(b, s);
}

int batch_evaluate(mds_batch *b) {
    CHECK(batch_autotune(b));
    CHECK(batch_enqueue_pass(b, kModeEval, b->stream));
    CHECK(batch_check_errors(b, "batch evaluation"));
    for (mds_ctx *c : b->ctx) c->grad_valid = true;
    return MDS_OK;
}

}  // namespace

extern "C" {

int mds_batch_create(int32_t n_data, const int64_t *n, int32_t d, const int32_t *chains, uint32_t flags,
                     mds_batch **out) {
    mds_batch *b = nullptr;
    if (!out) return bfail(b, MDS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_data < 1 || !n || !chains) return bfail(b, MDS_ERR_INVALID_ARG, "need n_data >= 1 and the N and chain arrays");
    if (flags != MDS_PREC_FP32C) return bfail(b, MDS_ERR_UNSUPPORTED, "batches run the FP32C path only");
    if (d < 1 || d > MDS_MAX_D) return bfail(b, MDS_ERR_INVALID_ARG, "D must be in [1, %d]", MDS_MAX_D);
    for (int i = 0; i < n_data; ++i)
        if (chains[i] < 1 || chains[i] > 1024 || n[i] < 2)
            return bfail(b, MDS_ERR_INVALID_ARG, "dataset %d: need N >= 2 and 1 <= chains <= 1024", i);
    b = new (std::nothrow) mds_batch();
    if (!b) return bfail(nullptr, MDS_ERR_OOM, "host allocation failed");
    b->n_data = n_data;
    b->d = d;
    int total = 0;
    for (int i = 0; i < n_data; ++i) {
        b->n.push_back(n[i]);
        b->chains.push_back(chains[i]);
        b->chain0.push_back(total);
        total += chains[i];
    }
    auto cleanup = [&](int st) {
        g_create_error = b->last_error;
        mds_batch_destroy(b);
        return st;
    };
    for (int i = 0; i < n_data; ++i) {
        for (int c = 0; c < chains[i]; ++c) {
            mds_ctx *x = nullptr;
            const int st = create_ctx(n[i], d, MDS_PREC_FP32C, c == 0, &x);
            if (st != MDS_OK) {
                b->last_error = g_create_error;
                return cleanup(st);
            }
            if (c > 0) x->y = b->ctx[b->chain0[i]]->y;  // shared, owned by the dataset's first chain
            b->ctx.push_back(x);
        }
    }
    b->device = b->ctx[0]->device;
    b->sm_count = b->ctx[0]->sm_count;
    b->device_name = b->ctx[0]->device_name;
    int st = MDS_OK;
    if ((st = bdev_alloc(b, &b->ds_dev, n_data * sizeof(BatchDataset)))) return cleanup(st);
    if ((st = bdev_alloc(b, &b->ch_dev, total * sizeof(BatchChain)))) return cleanup(st);
    if ((st = bdev_alloc(b, &b->rcfg, total * sizeof(ReduceArgs)))) return cleanup(st);
    if ((st = bdev_alloc(b, &b->tcfg, total * sizeof(TrajArgs)))) return cleanup(st);
    if ((st = bdev_alloc(b, &b->acfg, total * sizeof(AcceptArgs)))) return cleanup(st);
    bool ev_ok = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreate(&b->ev0) == cudaSuccess && cudaEventCreate(&b->ev1) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    b->joins.assign(b->ctx.size(), nullptr);
    for (size_t g = 0; ev_ok && g < b->ctx.size(); ++g)
        ev_ok = cudaEventCreateWithFlags(&b->joins[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ev_ok) {
        b->last_error = "stream/event creation failed";
        return cleanup(MDS_ERR_CUDA);
    }
    *out = b;
    return MDS_OK;
}

int mds_batch_destroy(mds_batch *b) {
    if (!b) return MDS_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void *bufs[] = {b->ds_dev, b->ch_dev, b->strips_dev, b->rcfg, b->jobs, b->tcfg, b->acfg, b->acc_out, b->dh_out};
    for (void *p : bufs)
        if (p) cudaFree(p);
    // chains other than a dataset's first do not own Y
    for (size_t g = 0; g < b->ctx.size(); ++g) mds_destroy(b->ctx[g]);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    delete b;
    return MDS_OK;
}

int mds_batch_set_stream(mds_batch *b, void *stream) {
    if (!b) return MDS_ERR_INVALID_ARG;
    b->stream = static_cast<cudaStream_t>(stream);
    for (mds_ctx *c : b->ctx) c->stream = b->stream;
    return MDS_OK;
}

int mds_batch_set_data(mds_batch *b, int32_t dataset, const void *y, int dtype, int layout, int64_t ld, int where) {
    mds_ctx *c0 = nullptr;
    CHECK(batch_chain(b, dataset, 0, &c0));
    const int st = mds_set_data(c0, y, dtype, layout, ld, where);
    for (int c = 0; c < b->chains[dataset]; ++c) {
        mds_ctx *x = b->ctx[b->chain0[dataset] + c];
        x->have_data = c0->have_data;
        x->y = c0->y;  // the first chain may have repacked Y into a new buffer (its slot order)
        x->grad_valid = false;
    }
    return bpass(b, c0, st);
}

int mds_batch_set_sigma(mds_batch *b, int32_t dataset, double sigma) {
    mds_ctx *c0 = nullptr;
    CHECK(batch_chain(b, dataset, 0, &c0));
    for (int c = 0; c < b->chains[dataset]; ++c) {
        mds_ctx *x = b->ctx[b->chain0[dataset] + c];
        BCHECK(x, mds_set_sigma(x, sigma));
    }
    return MDS_OK;
}

int mds_batch_set_locations(mds_batch *b, int32_t dataset, int32_t chain, const void *x, int dtype, int where) {
    mds_ctx *c = nullptr;
    CHECK(batch_chain(b, dataset, chain, &c));
    return bpass(b, c, mds_set_locations(c, x, dtype, where));
}

int mds_batch_get_locations(mds_batch *b, int32_t dataset, int32_t chain, void *x, int dtype, int where) {
    mds_ctx *c = nullptr;
    CHECK(batch_chain(b, dataset, chain, &c));
    return bpass(b, c, mds_get_locations(c, x, dtype, where));
}

int mds_batch_get_gradient(mds_batch *b, int32_t dataset, int32_t chain, void *g, int dtype, int where) {
    mds_ctx *c = nullptr;
    CHECK(batch_chain(b, dataset, chain, &c));
    if (!g) return bfail(b, MDS_ERR_INVALID_ARG, "g is NULL");
    CHECK(bpass(b, c, valid_enums(c, dtype, where)));
    if (!c->grad_valid) CHECK(batch_evaluate(b));
    return bpass(b, c, copy_out(c, c->grad, 2, g, dtype, where, c->n * c->d));
}

int mds_batch_evaluate(mds_batch *b, double *loglik, double *dlogl_dsigma) {
    if (!b) return MDS_ERR_INVALID_ARG;
    BCU(cudaSetDevice(b->device));
    CHECK(batch_evaluate(b));
    for (size_t g = 0; g < b->ctx.size(); ++g) {
        double s[kScalars];
        BCU(cudaMemcpyAsync(s, b->ctx[g]->scal, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
        BCU(cudaStreamSynchronize(b->stream));
        if (loglik) loglik[g] = s[kLogLik];
        if (dlogl_dsigma) dlogl_dsigma[g] = s[kDSigma];
    }
    return MDS_OK;
}

int mds_batch_hmc(mds_batch *b, int n_iter, int n_steps, const double *eps, uint64_t seed, int32_t *accepted,
                  double *dh) {
    if (!b) return MDS_ERR_INVALID_ARG;
    BCU(cudaSetDevice(b->device));
    if (n_iter < 0 || n_steps < 0 || !eps) return bfail(b, MDS_ERR_INVALID_ARG, "need n_iter, n_steps >= 0 and eps");
    for (int i = 0; i < b->n_data; ++i)
        if (!std::isfinite(eps[i])) return bfail(b, MDS_ERR_INVALID_ARG, "eps[%d] is not finite", i);
    bool valid = true;
    for (mds_ctx *c : b->ctx) valid = valid && c->grad_valid;
    if (!valid)
        CHECK(batch_evaluate(b));
    else
        CHECK(batch_autotune(b));
    if (n_iter == 0) return MDS_OK;
    const int total = static_cast<int>(b->ctx.size());
    if (static_cast<size_t>(n_iter) > b->out_cap) {
        if (b->acc_out) cudaFree(b->acc_out);
        if (b->dh_out) cudaFree(b->dh_out);
        b->acc_out = nullptr;
        b->dh_out = nullptr;
        CHECK(bdev_alloc(b, &b->acc_out, static_cast<size_t>(n_iter) * total * sizeof(int32_t)));
        CHECK(bdev_alloc(b, &b->dh_out, static_cast<size_t>(n_iter) * total * sizeof(double)));
        b->out_cap = n_iter;
    }
    // per-chain trajectory tables (contents may change between calls; the
    // captured graph reads them from device memory)
    std::vector<TrajArgs> tc(total);
    std::vector<AcceptArgs> ac(total);
    int max_grid = 0;
    int64_t max_nd = 0;
    for (int dd = 0; dd < b->n_data; ++dd) {
        for (int k = 0; k < b->chains[dd]; ++k) {
            const int g = b->chain0[dd] + k;
            mds_ctx *c = b->ctx[g];
            const int sg = traj_start_grid(c->n, c->d);
            max_grid = std::max(max_grid, sg);
            max_nd = std::max<int64_t>(max_nd, c->n * c->d);
            tc[g] = make_traj_args(c, n_steps, eps[dd], 1, seed, static_cast<uint32_t>(g));
            ac[g] = make_accept_args(c, n_steps, 1, 1, seed, static_cast<uint32_t>(g), sg,
                                     b->acc_out + static_cast<size_t>(g) * n_iter,
                                     b->dh_out + static_cast<size_t>(g) * n_iter, n_iter);
            BCU(cudaMemsetAsync(c->counters + kIterLocal, 0, sizeof(int64_t), b->stream));
        }
    }
    std::vector<ReduceArgs> rc(total);
    for (int dd = 0; dd < b->n_data; ++dd)
        for (int k = 0; k < b->chains[dd]; ++k) {
            const int g = b->chain0[dd] + k;
            rc[g] = reduce_args(b->ctx[g], kModeEval, eps[dd]);
        }
    BCU(cudaMemcpyAsync(b->tcfg, tc.data(), total * sizeof(TrajArgs), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->acfg, ac.data(), total * sizeof(AcceptArgs), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->rcfg, rc.data(), total * sizeof(ReduceArgs), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    const auto key = std::make_tuple(b->gen, n_steps);
    if (!b->graph || key != b->graph_key || max_grid != b->max_start_grid || max_nd != b->max_nd) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = launch_traj_start_batch(b->tcfg, total, max_grid, b->d, b->cap_stream);
        int st = e == cudaSuccess ? MDS_OK : bfail(b, MDS_ERR_CUDA, "batched start: %s", cudaGetErrorString(e));
        for (int k = 0; k < n_steps && st == MDS_OK; ++k)
            st = batch_enqueue_pass(b, k + 1 < n_steps ? kModeKickDrift : kModeHalfKick, b->cap_stream);
        if (st == MDS_OK) {
            e = launch_traj_end_batch(b->acfg, total, max_nd, b->d, b->cap_stream);
            if (e != cudaSuccess) st = bfail(b, MDS_ERR_CUDA, "batched end: %s", cudaGetErrorString(e));
        }
        e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != MDS_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        b->graph_key = key;
        b->max_start_grid = max_grid;
        b->max_nd = max_nd;
    }
    for (int t = 0; t < n_iter; ++t) BCU(cudaGraphLaunch(b->graph, b->stream));
    int st = batch_check_errors(b, "batch hmc");
    if (accepted || dh) {
        std::vector<int32_t> a(static_cast<size_t>(total) * n_iter);
        std::vector<double> h(static_cast<size_t>(total) * n_iter);
        BCU(cudaMemcpyAsync(a.data(), b->acc_out, a.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
        BCU(cudaMemcpyAsync(h.data(), b->dh_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BCU(cudaStreamSynchronize(b->stream));
        for (int t = 0; t < n_iter; ++t)
            for (int g = 0; g < total; ++g) {
                if (accepted) accepted[static_cast<size_t>(t) * total + g] = a[static_cast<size_t>(g) * n_iter + t];
                if (dh) dh[static_cast<size_t>(t) * total + g] = h[static_cast<size_t>(g) * n_iter + t];
            }
    }
    return st;
}

int mds_batch_set_strip(mds_batch *b, int32_t strip) {
    if (!b) return MDS_ERR_INVALID_ARG;
    if (strip < -256 || strip > 8)
        return bfail(b, MDS_ERR_INVALID_ARG, "batch strip must be in [1, 8] (strip kernel), [-256, -1] (per-chain "
                                             "chunked passes of about -strip tiles per chunk) or 0 (autotune)");
    b->strip_req = strip;
    return MDS_OK;
}

int mds_batch_reorder(mds_batch *b) {
    if (!b) return MDS_ERR_INVALID_ARG;
    BCU(cudaSetDevice(b->device));
    for (int dd = 0; dd < b->n_data; ++dd) {
        mds_ctx *c0 = b->ctx[b->chain0[dd]];
        BCHECK(c0, reorder_ctx(c0, false));
        for (int j = 1; j < b->chains[dd]; ++j) {
            mds_ctx *c = b->ctx[b->chain0[dd] + j];
            if (!c->have_x) return bfail(b, MDS_ERR_STATE, "dataset %d chain %d has no locations", dd, j);
            BCHECK(c, adopt_order(c, c0->perm_h, c0->inv_h, c0->y));
        }
    }
    b->gen++;
    return MDS_OK;
}

int mds_batch_get_strip(const mds_batch *b, int32_t *strip) {
    if (!b || !strip) return MDS_ERR_INVALID_ARG;
    *strip = b->strip;
    return MDS_OK;
}

int mds_batch_time_pass(mds_batch *b, int reps, double *ms_per_pass) {
    if (!b || reps < 1 || !ms_per_pass) return MDS_ERR_INVALID_ARG;
    BCU(cudaSetDevice(b->device));
    CHECK(batch_autotune(b));
    CHECK(batch_enqueue_pass(b, kModeEval, b->stream));
    // timed as the HMC runs the passes: `reps` of them in one captured graph
    cudaGraph_t g = nullptr;
    BCU(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    int st = MDS_OK;
    for (int r = 0; r < reps && st == MDS_OK; ++r) st = batch_enqueue_pass(b, kModeEval, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != MDS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch time_pass capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch time_pass graph: %s", cudaGetErrorString(e));
    float ms = 0.f;
    e = cudaGraphLaunch(ge, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev0, b->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return bfail(b, MDS_ERR_CUDA, "batch time_pass: %s", cudaGetErrorString(e));
    *ms_per_pass = ms / reps;
    for (mds_ctx *c : b->ctx) c->grad_valid = true;
    return batch_check_errors(b, "batch time_pass");
}

const char *mds_batch_last_error(const mds_batch *b) {
    if (!b) return g_create_error.c_str();
    return b->last_error.c_str();
}

}  // extern "C"
