// Single-item random-walk Metropolis: the prior-art sampler that section
// 2.3 of arXiv:1905.04582 contrasts HMC with (a low-dimensional random-walk
// kernel applied to one x_i at a time).  Moving x_i changes only the N - 1
// terms r_ij, j != i, so a proposal costs O(N D): its log-target difference
// is
//   L(X') - L(X) = sum_{j != i} [r_ij(x_i) - r_ij(x_i')] - (lambda/2)(|x_i'|^2 - |x_i|^2)
// (the -M log sigma of Eq. (2) cancels).  Proposals are sequential (each
// depends on the decisions before it), so one CTA runs them in a loop: its
// threads split the row, reading y_ij from the tile-packed Y, and thread 0
// takes the decision.  Per-pair arithmetic is in the precision of the
// context's state (FP32 with CUDA's erfcf / log1pf, or FP64), sums in FP64.
// Held-out pairs of a cross-validation fold (y < 0 in the tile layout) are
// left out, as in the training likelihood.
#include <cmath>
#include <cstdint>

#include "mds_internal.h"
#include "philox.cuh"

namespace mds {
namespace {

constexpr int kRwThreads = 512;

template <typename T>
__device__ __forceinline__ double r_term(T y, T delta, T half_inv_s2, T inv_s_sqrt2) {
    const T e = y - delta;
    T lphi;
    if constexpr (sizeof(T) == 4)
        lphi = log1pf(-0.5f * erfcf(delta * inv_s_sqrt2));
    else
        lphi = log1p(-0.5 * erfc(delta * inv_s_sqrt2));
    return static_cast<double>(e * e * half_inv_s2 + lphi);
}

template <typename T, int D>
__global__ void __launch_bounds__(kRwThreads) rwmh_kernel(const __grid_constant__ RwmhArgs a) {
    __shared__ T xo[D], xn[D];
    __shared__ int64_t s_item;
    __shared__ double s_u;
    __shared__ double sm[kRwThreads / 32];
    T *x = static_cast<T *>(a.x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T half_inv_s2 = static_cast<T>(0.5 / (a.sigma * a.sigma));
    const T inv_s_sqrt2 = static_cast<T>(0.70710678118654752440 / a.sigma);
    for (int t = 0; t < a.n_prop; ++t) {
        if (tid == 0) {
            int64_t i;
            double z[D], u;
            if (a.items) {
                i = a.items[t];
#pragma unroll
                for (int k = 0; k < D; ++k) z[k] = a.z[static_cast<int64_t>(t) * D + k];
                u = a.u[t];
            } else {
                // proposal `it`: counter (it, 0, chain, 3) -> item, u;
                // (it, 1 + q, chain, 3) -> z components 4q .. 4q + 3
                const uint32_t it = static_cast<uint32_t>(a.iter0 + t);
                uint32_t c[4] = {it, 0u, a.chain, 3u};
                philox10(c, a.seed);
                i = static_cast<int64_t>((static_cast<uint64_t>(c[0]) * static_cast<uint64_t>(a.n)) >> 32);
                u = open_unit(c[1]);
#pragma unroll
                for (int q = 0; 4 * q < D; ++q) {
                    uint32_t c2[4] = {it, 1u + static_cast<uint32_t>(q), a.chain, 3u};
                    philox10(c2, a.seed);
                    double zz[4];
                    box_muller(c2[0], c2[1], zz[0], zz[1]);
                    box_muller(c2[2], c2[3], zz[2], zz[3]);
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        if (4 * q + h < D) z[4 * q + h] = zz[h];
                }
            }
            if (i < 0 || i >= a.n) {
                atomicOr(a.err, kErrBadArgs);
                i = 0;
                u = 0.0;  // log u = -inf: never accepted
            }
            s_item = i;
            s_u = u;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T v = x[i * D + k];
                xo[k] = v;
                xn[k] = v + static_cast<T>(a.step * z[k]);
            }
        }
        __syncthreads();
        const int64_t i = s_item;
        const int64_t si = a.inv ? a.inv[i] : i;
        double acc = 0.0;
        for (int64_t j = tid; j < a.n; j += kRwThreads) {
            if (j == i) continue;
            const int64_t sj = a.inv ? a.inv[j] : j;
            const int64_t lo = si < sj ? si : sj, hi = si < sj ? sj : si;
            const int64_t I = lo / kTile, J = hi / kTile;
            const float yf = a.y[tile_index(I, J, a.nt) * kTileElems +
                                 tile_offset(static_cast<int>(lo - I * kTile), static_cast<int>(hi - J * kTile))];
            if (yf < 0.f) continue;  // held out
            T d0 = T(0), d1 = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T xj = x[j * D + k];
                const T a0 = xo[k] - xj, a1 = xn[k] - xj;
                d0 += a0 * a0;
                d1 += a1 * a1;
            }
            const T y = static_cast<T>(yf);
            acc += r_term<T>(y, sqrt(d0), half_inv_s2, inv_s_sqrt2) - r_term<T>(y, sqrt(d1), half_inv_s2, inv_s_sqrt2);
        }
        // fixed-order block sum
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sm[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            double dl = 0.0;
            for (int w = 0; w < kRwThreads / 32; ++w) dl += sm[w];
            double sq0 = 0.0, sq1 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                sq0 += static_cast<double>(xo[k]) * static_cast<double>(xo[k]);
                sq1 += static_cast<double>(xn[k]) * static_cast<double>(xn[k]);
            }
            const double lp = dl - 0.5 * a.lambda * (sq1 - sq0);
            const bool keep = isfinite(lp) && log(s_u) < lp;
            if (keep) {
                float m = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    x[i * D + k] = xn[k];
                    m = fmaxf(m, fabsf(static_cast<float>(xn[k])));
                }
                if (a.xmax_bits && m > 0.f) atomicMax(a.xmax_bits, __float_as_uint(m));
            }
            if (!isfinite(lp)) atomicOr(a.err, kErrNonfinite);
            if (a.acc_out) a.acc_out[t] = keep ? 1 : 0;
            if (a.dl_out) a.dl_out[t] = lp;
        }
        __syncthreads();  // x[i] and the shared proposal are settled before the next one
    }
}

template <int D>
cudaError_t launch_d(const RwmhArgs &a, cudaStream_t s) {
    if (a.fp64)
        rwmh_kernel<double, D><<<1, kRwThreads, 0, s>>>(a);
    else
        rwmh_kernel<float, D><<<1, kRwThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rwmh(const RwmhArgs &a, int d, cudaStream_t s) {
    if (a.n_prop <= 0) return cudaSuccess;
    switch (d) {
        case 1: return launch_d<1>(a, s);
        case 2: return launch_d<2>(a, s);
        case 3: return launch_d<3>(a, s);
        case 4: return launch_d<4>(a, s);
        case 5: return launch_d<5>(a, s);
        case 6: return launch_d<6>(a, s);
        case 7: return launch_d<7>(a, s);
        case 8: return launch_d<8>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mds
