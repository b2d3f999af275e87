// Batched pair pass: several datasets of uneven N, each with several HMC
// chains, advanced by one persistent launch (arXiv:1905.04582 fits one
// joint Y over four virus subtypes, section 3; batching independent
// datasets and chains is this library's systems choice).
//
// The grid is sized to the GPU and each CTA walks the strip list with a
// fixed stride (deterministic assignment).  For a strip (dataset d, row
// block I, column blocks [j0, j1)) the CTA loads the strip's Y tiles into
// shared memory once (one bulk TMA copy) and then runs the strip for every
// chain of d in turn, double-buffering the chains' split locations (TMA for
// the column blocks, plain loads for the row block), so each Y byte serves
// all chains of its dataset.  The per-pair arithmetic and the per-strip
// epilogue are those of the single-problem FP32C pass (pair_math.cuh); each
// chain writes its own row / column / scalar partials, reduced afterwards by
// reduce_batch_kernel.
#include <cstdint>

#include "mds_internal.h"
#include "pair_math.cuh"

namespace mds {
namespace {

template <int D>
struct BatchLayout {
    int cap;  // tiles per strip at most
    static constexpr int kXiBytes = 32 * D * 16;
    static constexpr int kRedBytes = kPairWarps * kTile * D * 4 + kPairWarps * 4 * 4;
    __host__ __device__ int y_bytes() const { return cap * kTileElems * 4; }
    __host__ __device__ int xj_bytes() const { return cap * kTile * D * 16; }
    __host__ __device__ int off_xj(int b) const { return y_bytes() + b * xj_bytes(); }
    __host__ __device__ int off_xi(int b) const { return y_bytes() + 2 * xj_bytes() + b * kXiBytes; }
    __host__ __device__ int off_red() const { return y_bytes() + 2 * xj_bytes() + 2 * kXiBytes; }
    __host__ __device__ int off_bar() const { return off_red() + kRedBytes; }
    __host__ __device__ int bytes() const { return off_bar() + 3 * 8; }
};

// Row block of one chain into shared memory ([k][row pair], as stored).
template <int D>
__device__ __forceinline__ void copy_xi(const BatchChain &ch, int I, float4 *dst) {
    const float4 *src = ch.xrow + static_cast<int64_t>(I) * 32 * D;
    for (int idx = threadIdx.x; idx < 32 * D; idx += kPairThreads) dst[idx] = src[idx];
}

template <int D>
__global__ void __launch_bounds__(kPairThreads, 3) pair_batch_kernel(const __grid_constant__ BatchPairArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const BatchLayout<D> L{a.strip_cap};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t *bar_y = reinterpret_cast<uint64_t *>(smem + L.off_bar());
    uint64_t *bar_x = bar_y + 1;  // two buffers
    float *ybuf = reinterpret_cast<float *>(smem);
    float *red = reinterpret_cast<float *>(smem + L.off_red());
    if (tid == 0) {
        mbar_init(bar_y, 1);
        mbar_init(&bar_x[0], 1);
        mbar_init(&bar_x[1], 1);
        fence_mbar_init();
    }
    // under PDL the next kernel may become resident now; this one reads the
    // chains' locations and writes their partials only after pdl_wait()
    pdl_trigger();
    __syncthreads();
    uint32_t ph_y = 0, ph_x0 = 0, ph_x1 = 0;
    // copies issued by thread 0 and not yet waited for (for the drain on errors)
    bool pend_y = false, pend_x0 = false, pend_x1 = false;
    bool ok = true;
    for (int w = blockIdx.x; w < a.n_strips && ok; w += gridDim.x) {
        const BatchStrip st = a.strips[w];
        const BatchDataset ds = a.ds[st.dataset];
        const int nst = st.j1 - st.j0;
        if (nst < 1 || nst > a.strip_cap || st.j1 > ds.nt || st.I > st.j0) {
            if (tid == 0) atomicOr(a.err, kErrBadArgs);
            break;  // uniform: every thread read the same strip
        }
        const int64_t t0 = tile_index(st.I, st.j0, ds.nt);
        const int nchains = ds.n_chains;
        const uint32_t xbytes = static_cast<uint32_t>(nst) * kTile * D * 16;
        if (tid == 0) {
            fence_proxy_async();  // earlier generic reads of these buffers before the new copies
            mbar_expect_tx(bar_y, nst * kTileElems * 4);
            tma_load_1d(ybuf, ds.y + t0 * kTileElems, nst * kTileElems * 4, bar_y);  // Y is constant
            pend_y = true;
        }
        pdl_wait();  // returns at once after the first strip
        if (tid == 0) {
            const BatchChain c0 = a.ch[ds.chain0];
            mbar_expect_tx(&bar_x[0], xbytes);
            tma_load_1d(smem + L.off_xj(0), c0.xcol + static_cast<int64_t>(st.j0) * kTile * D, xbytes, &bar_x[0]);
            pend_x0 = true;
        }
        copy_xi<D>(a.ch[ds.chain0], st.I, reinterpret_cast<float4 *>(smem + L.off_xi(0)));
        __syncthreads();
        const bool ragged = (ds.n % kTile) != 0;
        for (int c = 0; c < nchains; ++c) {
            const int b = c & 1;
            const BatchChain ch = a.ch[ds.chain0 + c];
            if (c + 1 < nchains) {
                // next chain's locations into the other buffer (free since the
                // end-of-chain barrier of chain c - 1)
                const BatchChain cn = a.ch[ds.chain0 + c + 1];
                if (tid == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar_x[b ^ 1], xbytes);
                    tma_load_1d(smem + L.off_xj(b ^ 1), cn.xcol + static_cast<int64_t>(st.j0) * kTile * D, xbytes,
                                &bar_x[b ^ 1]);
                    if (b) pend_x0 = true; else pend_x1 = true;
                }
                copy_xi<D>(cn, st.I, reinterpret_cast<float4 *>(smem + L.off_xi(b ^ 1)));
            }
            bool got = true;
            if (c == 0) {
                got = __all_sync(0xffffffffu, mbar_wait_bounded(bar_y, ph_y, a.err));
                ph_y ^= 1;
                if (tid == 0) pend_y = false;
            }
            got = got && __all_sync(0xffffffffu, mbar_wait_bounded(&bar_x[b], b ? ph_x1 : ph_x0, a.err));
            if (b) ph_x1 ^= 1; else ph_x0 ^= 1;
            if (tid == 0) {
                if (b) pend_x1 = false; else pend_x0 = false;
            }
            ok = __syncthreads_and(got) != 0;
            if (!ok) break;

            const float4 *xis = reinterpret_cast<const float4 *>(smem + L.off_xi(b));
            float2 racc[4][D];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < D; ++k) racc[q][k] = make_float2(0.f, 0.f);
            float es = 0.f, ec = 0.f, ms = 0.f, mc = 0.f, gs = 0.f, gc = 0.f;
            for (int jt = 0; jt < nst; ++jt) {
                const int J = st.j0 + jt;
                const bool masked = (J == st.I) || (ragged && J == ds.nt - 1);
                const float4 *ys = reinterpret_cast<const float4 *>(ybuf + jt * kTileElems + warp * kWarpTileElems);
                const float4 *xjs =
                    reinterpret_cast<const float4 *>(smem + L.off_xj(b)) + (jt * kTile + warp * kWarpCols) * D;
                float *colp = ch.col_part + (col_slot(st.I, J) * kTile + warp * kWarpCols) * D;
                const int row_rel = (st.I - J) * kTile;
                const int64_t ncv = ds.n - static_cast<int64_t>(J) * kTile;
                float2 e2 = make_float2(0.f, 0.f), mdv = make_float2(0.f, 0.f), prod = make_float2(1.f, 1.f);
                if (masked)
                    tile_f32<D, true, BatchDataset>(ds, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv, racc, colp,
                                                     e2, mdv, prod);
                else
                    tile_f32<D, false, BatchDataset>(ds, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv, racc,
                                                      colp, e2, mdv, prod);
                kahan_add(es, ec, e2.x + e2.y);
                kahan_add(ms, mc, mdv.x + mdv.y);
                kahan_add(gs, gc, lg2_approx(prod.x) + lg2_approx(prod.y));
            }
            strip_epilogue_f32<D>(racc, es, ec, ms, mc, gs, gc, red,
                                  ch.row_part + static_cast<int64_t>(st.row_slot) * kTile * D,
                                  ch.scal_part + static_cast<int64_t>(st.local) * kScalarParts, a.err);
            __syncthreads();  // this chain's buffers and the scratch are free
        }
        __syncthreads();  // the strip's Y buffer is free
    }
    if (!ok && tid == 0) {
        // let copies still in flight land before the CTA exits (bounded)
        if (pend_y) mbar_wait_bounded(bar_y, ph_y, a.err);
        if (pend_x0) mbar_wait_bounded(&bar_x[0], ph_x0, a.err);
        if (pend_x1) mbar_wait_bounded(&bar_x[1], ph_x1, a.err);
    }
}

}  // namespace

size_t pair_batch_smem(int d, int strip_cap) {
    switch (d) {
        case 1: return BatchLayout<1>{strip_cap}.bytes();
        case 2: return BatchLayout<2>{strip_cap}.bytes();
        case 3: return BatchLayout<3>{strip_cap}.bytes();
        case 4: return BatchLayout<4>{strip_cap}.bytes();
        case 5: return BatchLayout<5>{strip_cap}.bytes();
        case 6: return BatchLayout<6>{strip_cap}.bytes();
        case 7: return BatchLayout<7>{strip_cap}.bytes();
        case 8: return BatchLayout<8>{strip_cap}.bytes();
        default: return 0;
    }
}

template <int D>
int blocks_per_sm_d(int strip_cap) {
    const int bytes = static_cast<int>(BatchLayout<D>{strip_cap}.bytes());
    if (cudaFuncSetAttribute(pair_batch_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_batch_kernel<D>, kPairThreads, bytes) != cudaSuccess)
        return 0;
    return nb;
}

int pair_batch_blocks_per_sm(int d, int strip_cap) {
    switch (d) {
        case 1: return blocks_per_sm_d<1>(strip_cap);
        case 2: return blocks_per_sm_d<2>(strip_cap);
        case 3: return blocks_per_sm_d<3>(strip_cap);
        case 4: return blocks_per_sm_d<4>(strip_cap);
        case 5: return blocks_per_sm_d<5>(strip_cap);
        case 6: return blocks_per_sm_d<6>(strip_cap);
        case 7: return blocks_per_sm_d<7>(strip_cap);
        case 8: return blocks_per_sm_d<8>(strip_cap);
        default: return 0;
    }
}

cudaError_t launch_pair_batch(const BatchPairArgs &a, int d, int grid, cudaStream_t s) {
    if (a.n_strips <= 0 || grid <= 0) return cudaSuccess;
    const size_t bytes = pair_batch_smem(d, a.strip_cap);
    cudaError_t e = cudaSuccess;
    switch (d) {
#define MDS_PB_CASE(DD) \
    case DD: e = launch_pdl(pair_batch_kernel<DD>, dim3(grid), dim3(kPairThreads), bytes, s, a); break;
        MDS_PB_CASE(1) MDS_PB_CASE(2) MDS_PB_CASE(3) MDS_PB_CASE(4)
        MDS_PB_CASE(5) MDS_PB_CASE(6) MDS_PB_CASE(7) MDS_PB_CASE(8)
#undef MDS_PB_CASE
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace mds
