// The measured ceiling of the FP32C pair pass's per-pair arithmetic: the same
// per-pair bodies (pair2_f32 with the Phi terms, pair2_far without them, as
// the pass's tiles call them: four row pairs against two columns per round)
// with every operand in registers, at the pass's occupancy (128 threads, the
// same launch bounds).  No loads, no tile epilogue, no reductions: the rate at
// which the arithmetic of Eq. (2) and its gradient (Eq. (9)) alone can run on
// this GPU, against which the pass's pairs/s are compared (a measured
// per-pair-instruction ceiling rather than a unit count).
#include <cstdint>

#include "mds_internal.h"
#include "pair_math.cuh"

namespace mds {
namespace {

template <int D, bool FAR>
__global__ void __launch_bounds__(kPairThreads, (D <= 2 ? 4 : D <= 4 ? 3 : 2))
    pair_ceiling_kernel(const __grid_constant__ PairArgs a, int iters, float *sink) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const float h = 0.37f + 0.0013f * static_cast<float>(t & 127);
    // split layouts as the pass holds them: rows {xh_i, xh_i+1, xl_i, xl_i+1},
    // columns {-xh_j, -xh_j, -xl_j, -xl_j}
    float4 xi[4][D], xj[2][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) xi[q][k] = make_float4(h * (q + 1) + 0.11f * k, h * (q + 1.5f) - 0.07f * k, 0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = -(0.9f * h + 0.23f * e + 0.05f * k);
            xj[e][k] = make_float4(v, v, 0.f, 0.f);
        }
    const float4 yv = make_float4(0.8f, 1.1f, 0.95f, 1.3f);
    float2 racc[4][D], cacc[2][D];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) racc[q][k] = f2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) cacc[e][k] = f2(0.f, 0.f);
    float2 e2 = f2(0.f, 0.f), md = f2(0.f, 0.f);
    float gs = 0.f;
    for (int it = 0; it < iters; ++it) {
        float2 prod = f2(1.f, 1.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (FAR) {
                pair2_far<D, PairArgs>(a, xi[q], xj[0], f2(yv.x, yv.y), racc[q], cacc[0], e2);
                pair2_far<D, PairArgs>(a, xi[q], xj[1], f2(yv.z, yv.w), racc[q], cacc[1], e2);
            } else {
                pair2_f32<D, false, PairArgs>(a, xi[q], xj[0], f2(yv.x, yv.y), f2(1.f, 1.f), racc[q], cacc[0], e2, md,
                                              prod);
                pair2_f32<D, false, PairArgs>(a, xi[q], xj[1], f2(yv.z, yv.w), f2(1.f, 1.f), racc[q], cacc[1], e2, md,
                                              prod);
            }
        }
        if constexpr (!FAR) gs += lg2_approx(prod.x) + lg2_approx(prod.y);
        // move the columns a little, so that nothing is loop-invariant
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                xj[e][k].x -= 1e-7f;
                xj[e][k].y -= 1e-7f;
            }
    }
    float s = e2.x + e2.y + md.x + md.y + gs;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) s += racc[q][k].x + racc[q][k].y;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) s += cacc[e][k].x + cacc[e][k].y;
    sink[t] = s;
}

template <int D>
cudaError_t launch_d(const PairArgs &a, bool far, int grid, int iters, float *sink, cudaStream_t s) {
    if (far)
        pair_ceiling_kernel<D, true><<<grid, kPairThreads, 0, s>>>(a, iters, sink);
    else
        pair_ceiling_kernel<D, false><<<grid, kPairThreads, 0, s>>>(a, iters, sink);
    return cudaGetLastError();
}

}  // namespace

int pair_ceiling_blocks_per_sm(int d) { return d <= 2 ? 4 : d <= 4 ? 3 : 2; }

cudaError_t launch_pair_ceiling(const PairArgs &a, int d, bool far, int grid, int iters, float *sink, cudaStream_t s) {
    switch (d) {
        case 1: return launch_d<1>(a, far, grid, iters, sink, s);
        case 2: return launch_d<2>(a, far, grid, iters, sink, s);
        case 3: return launch_d<3>(a, far, grid, iters, sink, s);
        case 4: return launch_d<4>(a, far, grid, iters, sink, s);
        case 5: return launch_d<5>(a, far, grid, iters, sink, s);
        case 6: return launch_d<6>(a, far, grid, iters, sink, s);
        case 7: return launch_d<7>(a, far, grid, iters, sink, s);
        case 8: return launch_d<8>(a, far, grid, iters, sink, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mds
