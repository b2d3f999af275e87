// Fused pair pass of the truncated-normal MDS likelihood (arXiv:1905.04582,
// section 2.5 and Algorithms 1-2, re-designed for sm_103a).
//
// One CTA (4 warps) takes one strip: row block I (64 items) against column
// blocks [j0, j1).  For every pair (i, j) of the strip it computes in
// registers, storing nothing per pair,
//   delta = ||x_i - x_j||,  e = y_ij - delta,  z = delta / sigma,
//   r_ij  = e^2 / (2 sigma^2) + log Phi(z)                       (Eq. (2))
//   w_ij  = (delta - y_ij) / sigma^2 + phi(z) / (sigma Phi(z))   (Eq. (9))
// and accumulates
//   row i    : sum_j w_ij (x_i - x_j) / delta   (registers, whole strip)
//   column j : sum_i w_ij (x_i - x_j) / delta   (registers over the lane's 8
//              rows, then a 3-level lane transpose-reduce, once per tile)
//   scalars  : sum e^2, sum phi/Phi * delta, sum log Phi.
// Each pair is visited once (Algorithm 2 of the paper visits it twice); the
// gradient is -row_i + column_i, completed by reduce_kernel.cu.
//
// FP32C path (pair_f32_kernel):
//  - memory: each warp owns a 3-stage ring in shared memory; lane 0 refills
//    it with two bulk TMA copies per tile (its 4 KB quarter of the tile's Y and
//    its 16 columns of split locations), completion on a per-stage mbarrier,
//    so Y streams from HBM/L2 exactly once per pass with no cross-warp waits;
//  - arithmetic: packed f32x2 FMA/ADD/MUL on row pairs, MUFU rsqrt / ex2 /
//    rcp / lg2.  The distance uses the exact split (see mds_internal.h) and
//    a residual correction, e = (y - d0) - (d^2 - d0^2) / (2 d0), so the
//    cancellation in y - delta does not amplify FP32 rounding.  Phi(z) =
//    1 - phi(z) R(z) with the Mills ratio R approximated by the rational P/D
//    of mills_ratio_coeffs.h: one reciprocal gives 1/Phi = D / (D - phi P);
//    log Phi is summed as -log2 of per-tile products of 1/Phi (1/Phi <= 2, so
//    the 16 factors of a lane half cannot overflow).  Sums: FP32 within a
//    tile, Kahan-compensated FP32 across tiles, FP32 trees across lanes and
//    warps; the reduce kernel combines the strips with FP32 two-sums.  No
//    FP64 instruction runs in this kernel (FP64 is 1/64 rate on this GPU).
//
// FP64 path (pair_f64_kernel): same work split, CUDA's double sqrt / erfc /
// log1p / exp per pair and FP64 sums (the plain FP64 GPU path).
#include <cfloat>
#include <cstdint>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "mds_internal.h"
#include "pair_math.cuh"

namespace mds {
namespace {

// --------------------------------------------------------------- FP32C

constexpr int kStages = 3;  // per-warp ring depth

template <int D>
struct F32Layout {
    static constexpr int kXiBytes = 32 * D * 16;                       // 32 row pairs x D float4
    static constexpr int kXjBytes = kWarpCols * D * 16;                // 16 columns x D float4
    static constexpr int kStageBytes = (kWarpTileElems * 4 + kXjBytes + 127) / 128 * 128;
    static constexpr int kRingOffset = (kXiBytes + 127) / 128 * 128;
    static constexpr int kBarOffset = kRingOffset + kPairWarps * kStages * kStageBytes;
    // each warp's copy of the row box (2 D floats) after the barriers
    static constexpr int kBoxOffset = kBarOffset + kPairWarps * kStages * 8;
    // the strip epilogue reuses the (then idle) rings for its reduction scratch
    static constexpr int kRedOffset = kRingOffset;
    static constexpr int kRedBytes = kPairWarps * kTile * D * 4 + kPairWarps * 4 * 4;
    static_assert(kRedBytes <= kPairWarps * kStages * kStageBytes, "scratch must fit in the rings");
    static constexpr int kBytes = kBoxOffset + kPairWarps * 2 * D * 4;
};

// Refill one stage of a warp's ring: its 4 KB quarter of a Y tile and the
// 16 columns of split locations of the tile's column block.
template <int D>
__device__ __forceinline__ void issue_stage(unsigned char *dst, uint64_t *bar, const float *ysrc, const float4 *xsrc) {
    constexpr int kXj = kWarpCols * D * 16;
    mbar_expect_tx(bar, kWarpTileElems * 4 + kXj);
    tma_load_1d(dst, ysrc, kWarpTileElems * 4, bar);
    tma_load_1d(dst + kWarpTileElems * 4, xsrc, kXj, bar);
}

// HELDOUT: the context has a cross-validation fold (tiles flagged in
// a.tile_ho take the masked path, which then also skips y < 0); a separate
// instantiation so that the plain pass carries no extra register pressure.
template <int D, bool HELDOUT>
__global__ void __launch_bounds__(kPairThreads, (D <= 2 ? 4 : D <= 4 ? 3 : 2)) pair_f32_kernel(const __grid_constant__ PairArgs a) {
    using L = F32Layout<D>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    pdl_trigger();
    if (blockIdx.x >= static_cast<unsigned>(a.n_strips)) return;
    const Strip st = a.strips[blockIdx.x];  // the strip table is fixed between passes
    const int nst = st.j1 - st.j0;
    if (nst < 1 || st.j1 > a.nt || st.I > st.j0) {
        if (tid == 0) atomicOr(a.err, kErrBadArgs);
        return;
    }
    float4 *xis = reinterpret_cast<float4 *>(smem);
    unsigned char *ring = smem + L::kRingOffset + warp * kStages * L::kStageBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBarOffset) + warp * kStages;
    const int64_t nt = a.nt;
    const int64_t t0 = tile_index(st.I, st.j0, nt);

    // this warp's quarter of the tile and its 16 columns of split locations
    const float *ysrc0 = a.y + (t0 - a.y_t0) * kTileElems + warp * kWarpTileElems;
    const float4 *xsrc0 = a.xcol + (static_cast<int64_t>(st.j0) * kTile + warp * kWarpCols) * D;

    // prologue: the first stages' Y quarters (Y is constant) may stream in
    // while the previous kernel drains; the locations and every partial
    // buffer belong to it until pdl_wait() returns
    constexpr uint32_t kXjBytes = kWarpCols * D * 16;
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        for (int s = 0; s < kStages && s < nst; ++s) {
            mbar_expect_tx(&bars[s], kWarpTileElems * 4 + kXjBytes);
            tma_load_1d(ring + s * L::kStageBytes, ysrc0 + s * kTileElems, kWarpTileElems * 4, &bars[s]);
        }
    }
    pdl_wait();
    if (a.stamps && lane == 0) atomicMin(&a.stamps[0], global_ns());
    if (lane == 0) {
        for (int s = 0; s < kStages && s < nst; ++s)
            tma_load_1d(ring + s * L::kStageBytes + kWarpTileElems * 4, xsrc0 + s * kTile * D, kXjBytes, &bars[s]);
    }
    // x_i of the row block: 32 row pairs x D, [k][rp] as stored
    const float4 *xsrc_row = a.xrow + static_cast<int64_t>(st.I) * 32 * D;
    for (int idx = tid; idx < 32 * D; idx += kPairThreads) xis[idx] = xsrc_row[idx];
    __syncthreads();
    // the row box of the block (each warp its own copy: no further CTA barrier)
    float *box = reinterpret_cast<float *>(smem + L::kBoxOffset) + warp * 2 * D;
    {
        float b[2 * D];
        row_box<D>(xis, lane, b);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 2 * D; ++i) box[i] = b[i];
        __syncwarp();
    }

    float2 racc[4][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) racc[q][k] = f2(0.f, 0.f);
    float es = 0.f, ec = 0.f, ms = 0.f, mc = 0.f, gs = 0.f, gc = 0.f;

    const int64_t n = a.n;
    const bool ragged = (n % kTile) != 0;
    const int rowbase = st.I * kTile;
    float *colp_base = reinterpret_cast<float *>(a.col_part);
    bool ok = true;
    int n_far = 0;  // warp blocks of this warp that took the far path
    int jt = 0;
    for (; jt < nst; ++jt) {
        const int stage = jt % kStages;
        // every lane observes the phase (visibility of the TMA data); the
        // decision to go on is made warp-uniform
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[stage], (jt / kStages) & 1, a.err))) {
            ok = false;
            break;
        }
        const unsigned char *sbuf = ring + stage * L::kStageBytes;
        const float4 *ys = reinterpret_cast<const float4 *>(sbuf);
        const float4 *xjs = reinterpret_cast<const float4 *>(sbuf + kWarpTileElems * 4);
        const int J = st.j0 + jt;
        const bool masked = (J == st.I) || (ragged && J == nt - 1) || (HELDOUT && a.tile_ho[t0 + jt]);
        float2 e2 = f2(0.f, 0.f), mdv = f2(0.f, 0.f), prod = f2(1.f, 1.f);
        float *colp = colp_base + (col_slot(st.I, J) * kTile + warp * kWarpCols) * D;
        {
            const int row_rel = rowbase - J * kTile;
            const int64_t ncv = n - static_cast<int64_t>(J) * kTile;
            if (masked)
                tile_f32<D, true, PairArgs, HELDOUT>(a, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv, racc, colp,
                                                     e2, mdv, prod);
            else
                n_far += tile_f32<D, false, PairArgs, false, true>(a, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv,
                                                                   racc, colp, e2, mdv, prod, box, a.far_d2);
        }
        // all lanes are done reading this stage: refill it (async proxy after
        // the generic reads)
        __syncwarp();
        if (lane == 0 && jt + kStages < nst) {
            fence_proxy_async();
            const int nx = jt + kStages;
            issue_stage<D>(ring + stage * L::kStageBytes, &bars[stage], ysrc0 + static_cast<int64_t>(nx) * kTileElems,
                           xsrc0 + static_cast<int64_t>(nx) * kTile * D);
        }
        kahan_add(es, ec, e2.x + e2.y);
        kahan_add(ms, mc, mdv.x + mdv.y);
        kahan_add(gs, gc, lg2_approx(prod.x) + lg2_approx(prod.y));
    }
    if (!ok) {
        // let copies still in flight land before the CTA exits (bounded)
        if (lane == 0)
            for (int j = jt; j < nst && j < jt + kStages; ++j) mbar_wait_bounded(&bars[j % kStages], (j / kStages) & 1, a.err);
    }

    if (lane == 0 && a.far_part) a.far_part[blockIdx.x * kPairWarps + warp] = n_far;

    // ---- strip epilogue
    float *red = reinterpret_cast<float *>(smem + L::kRedOffset);
    __syncthreads();  // shared memory of the rings is no longer needed by anyone
    strip_epilogue_f32<D>(racc, es, ec, ms, mc, gs, gc, red,
                          reinterpret_cast<float *>(a.row_part) + static_cast<int64_t>(st.row_slot) * kTile * D,
                          reinterpret_cast<float *>(a.scal_part) + static_cast<int64_t>(blockIdx.x) * kScalarParts,
                          a.err);
    if (a.stamps && lane == 0) atomicMax(&a.stamps[1], global_ns());
}

// ---------------------------------------------------------------- FP64

// The plain FP64 path: same tile work split; Y read straight from global
// memory in the tile layout, locations from the FP64 state.
template <int D>
__global__ void __launch_bounds__(kPairThreads) pair_f64_kernel(const __grid_constant__ PairArgs a) {
    constexpr int V = 4 * D;
    constexpr int P = Pow2<V>::value;
    constexpr double kInvSqrt2Pi = 0.39894228040143267794;
    constexpr double kInvSqrt2 = 0.70710678118654752440;
    __shared__ double red[kPairWarps * kTile * D + kPairWarps * 4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int la = lane & 7, lb = lane >> 3;
    if (blockIdx.x >= static_cast<unsigned>(a.n_strips)) return;
    const Strip st = a.strips[blockIdx.x];
    const int nst = st.j1 - st.j0;
    if (nst < 1 || st.j1 > a.nt || st.I > st.j0) {
        if (tid == 0) atomicOr(a.err, kErrBadArgs);
        return;
    }
    pdl_wait();
    if (a.stamps && lane == 0) atomicMin(&a.stamps[0], global_ns());
    const int64_t nt = a.nt, n = a.n;
    const bool ragged = (n % kTile) != 0;
    const int64_t t0 = tile_index(st.I, st.j0, nt);
    const int rowbase = st.I * kTile;
    double xi[8][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int slot = rowbase + 2 * (la + 8 * q) + h;
                const int64_t item = a.perm ? a.perm[slot] : slot;
                xi[2 * q + h][k] = a.x64[item * D + k];
            }
    double racc[8][D];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int k = 0; k < D; ++k) racc[r][k] = 0.0;
    double e2 = 0.0, md = 0.0, lp = 0.0;
    double *colp_base = reinterpret_cast<double *>(a.col_part);
    for (int jt = 0; jt < nst; ++jt) {
        const int J = st.j0 + jt;
        const bool masked = (J == st.I) || (ragged && J == nt - 1) || (a.tile_ho && a.tile_ho[t0 + jt]);
        const int row_rel = rowbase - J * kTile;
        const int64_t ncv = n - static_cast<int64_t>(J) * kTile;
        const float4 *ys =
            reinterpret_cast<const float4 *>(a.y + (t0 + jt - a.y_t0) * kTileElems + warp * kWarpTileElems);
        double colv[P];
#pragma unroll
        for (int i = 0; i < P; ++i) colv[i] = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = warp * kWarpCols + 4 * lb + c;
            double xj[D];
            const int64_t cslot = static_cast<int64_t>(J) * kTile + col;
            const int64_t citem = a.perm ? a.perm[cslot] : cslot;
#pragma unroll
            for (int k = 0; k < D; ++k) xj[k] = a.x64[citem * D + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 yv = ys[(2 * q + (c >> 1)) * 32 + (lane ^ ((c >> 1) << 2))];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float yf = (c & 1) ? (h ? yv.w : yv.z) : (h ? yv.y : yv.x);
                    const int r = row_rel + 2 * (la + 8 * q) + h;
                    const bool valid = !masked || (col > r && col < ncv && yf >= 0.f);  // y < 0: held out
                    double dl[D];
                    double d2 = 0.0;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        dl[k] = xi[2 * q + h][k] - xj[k];
                        d2 = fma(dl[k], dl[k], d2);
                    }
                    const double del = sqrt(d2);
                    const double inv = del > 0.0 ? 1.0 / del : 0.0;
                    const double e = valid ? static_cast<double>(yf) - del : 0.0;
                    const double z = del * a.inv_sigma;
                    const double qz = 0.5 * erfc(z * kInvSqrt2);
                    const double m = valid ? exp(-0.5 * z * z) * kInvSqrt2Pi / (1.0 - qz) : 0.0;
                    e2 = fma(e, e, e2);
                    md = fma(m, del, md);
                    if (valid) lp += log1p(-qz);
                    const double wi = (m * a.inv_sigma - e * a.inv_s2) * inv;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const double t = wi * dl[k];
                        racc[2 * q + h][k] += t;
                        colv[c * D + k] += t;
                    }
                }
            }
        }
        lane_reduce<P, 3>(colv, lane, 0);
        bool writer;
        const int base = reduced_base<P, 3>(lane, 0, writer);
        constexpr int kHeld = P >= 8 ? P / 8 : 1;
        double *cp = colp_base + (col_slot(st.I, J) * kTile + warp * kWarpCols + 4 * lb) * D;
        if (writer) {
#pragma unroll
            for (int i = 0; i < kHeld; ++i)
                if (base + i < V) cp[base + i] = colv[i];
        }
    }
    constexpr int VR = 8 * D;
    double rv[VR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            rv[(q * D + k) * 2 + 0] = racc[2 * q][k];
            rv[(q * D + k) * 2 + 1] = racc[2 * q + 1][k];
        }
    lane_reduce<VR, 2>(rv, lane, 3);
    {
        bool writer;
        const int base = reduced_base<VR, 2>(lane, 3, writer);
#pragma unroll
        for (int i = 0; i < VR / 4; ++i) {
            const int v = base + i;
            const int h = v & 1, k = (v >> 1) % D, q = (v >> 1) / D;
            red[(warp * kTile + 2 * (la + 8 * q) + h) * D + k] = rv[i];
        }
    }
    double sv[3] = {e2, md, lp};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double v = sv[i];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[kPairWarps * kTile * D + warp * 4 + i] = v;
    }
    __syncthreads();
    double *rp = reinterpret_cast<double *>(a.row_part) + static_cast<int64_t>(st.row_slot) * kTile * D;
    for (int idx = tid; idx < kTile * D; idx += kPairThreads) {
        double v = red[idx];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += red[w * kTile * D + idx];
        rp[idx] = v;
    }
    if (tid < 3) {
        const double *sr = red + kPairWarps * kTile * D;
        double v = sr[tid];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += sr[w * 4 + tid];
        reinterpret_cast<double *>(a.scal_part)[static_cast<int64_t>(blockIdx.x) * kScalarParts + tid] = v;
        if (!isfinite(v)) atomicOr(a.err, kErrNonfinite);
    }
    if (a.stamps && lane == 0) atomicMax(&a.stamps[1], global_ns());
}

template <int D>
cudaError_t launch_f32_d(const PairArgs &a, cudaStream_t s, bool pdl, int smem_min) {
    using L = F32Layout<D>;
    const int smem = smem_min > L::kBytes ? smem_min : L::kBytes;  // more only to cap the CTAs per SM
    {
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(pair_f32_kernel<D, false>), smem);
        if (e == cudaSuccess) e = raise_dyn_smem(reinterpret_cast<const void *>(pair_f32_kernel<D, true>), smem);
        if (e != cudaSuccess) return e;
    }
    if (a.n_strips <= 0) return cudaSuccess;
    const cudaError_t e =
        a.tile_ho ? launch_maybe_pdl(pdl, pair_f32_kernel<D, true>, dim3(a.n_strips), dim3(kPairThreads), smem, s, a)
                  : launch_maybe_pdl(pdl, pair_f32_kernel<D, false>, dim3(a.n_strips), dim3(kPairThreads), smem, s, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int D>
cudaError_t launch_f64_d(const PairArgs &a, cudaStream_t s, bool pdl) {
    if (a.n_strips <= 0) return cudaSuccess;
    const cudaError_t e = launch_maybe_pdl(pdl, pair_f64_kernel<D>, dim3(a.n_strips), dim3(kPairThreads), 0, s, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// A bounded wait on an mbarrier that nothing completes (fault injection for
// tests of the timeout path): it gives up after the wait limit and sets the
// timeout bit of the error word, as a stalled copy in the pair pass would.
__global__ void wait_probe_kernel(unsigned *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait_bounded(&bar, 0, err);
    }
}

}  // namespace

cudaError_t raise_dyn_smem(const void *func, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> set;  // (kernel, device) -> bytes set so far
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    int &cur = set[std::make_pair(func, dev)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t launch_wait_probe(unsigned *err, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

int pair_f32_smem_bytes(int d) {
    switch (d) {
        case 1: return F32Layout<1>::kBytes;
        case 2: return F32Layout<2>::kBytes;
        case 3: return F32Layout<3>::kBytes;
        case 4: return F32Layout<4>::kBytes;
        case 5: return F32Layout<5>::kBytes;
        case 6: return F32Layout<6>::kBytes;
        case 7: return F32Layout<7>::kBytes;
        case 8: return F32Layout<8>::kBytes;
        default: return 0;
    }
}

cudaError_t launch_pair_pass_f32(const PairArgs &a, int d, cudaStream_t s, bool pdl, int smem_min) {
    switch (d) {
        case 1: return launch_f32_d<1>(a, s, pdl, smem_min);
        case 2: return launch_f32_d<2>(a, s, pdl, smem_min);
        case 3: return launch_f32_d<3>(a, s, pdl, smem_min);
        case 4: return launch_f32_d<4>(a, s, pdl, smem_min);
        case 5: return launch_f32_d<5>(a, s, pdl, smem_min);
        case 6: return launch_f32_d<6>(a, s, pdl, smem_min);
        case 7: return launch_f32_d<7>(a, s, pdl, smem_min);
        case 8: return launch_f32_d<8>(a, s, pdl, smem_min);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pair_pass_f64(const PairArgs &a, int d, cudaStream_t s, bool pdl) {
    switch (d) {
        case 1: return launch_f64_d<1>(a, s, pdl);
        case 2: return launch_f64_d<2>(a, s, pdl);
        case 3: return launch_f64_d<3>(a, s, pdl);
        case 4: return launch_f64_d<4>(a, s, pdl);
        case 5: return launch_f64_d<5>(a, s, pdl);
        case 6: return launch_f64_d<6>(a, s, pdl);
        case 7: return launch_f64_d<7>(a, s, pdl);
        case 8: return launch_f64_d<8>(a, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mds
