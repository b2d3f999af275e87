// Single-item random-walk Metropolis: the prior-art sampler that section
// 2.3 of arXiv:1905.04582 contrasts HMC with (a low-dimensional random-walk
// kernel applied to one x_i at a time).  Moving x_i changes only the N - 1
// terms r_ij, j != i, so a proposal costs O(N D): its log-target difference
// is
//   L(X') - L(X) = sum_{j != i} [r_ij(x_i) - r_ij(x_i')] - (lambda/2)(|x_i'|^2 - |x_i|^2)
// (the -M log sigma of Eq. (2) cancels).  Proposals are sequential (each
// depends on the decisions before it), so one CTA runs them in a loop: its
// threads split the row by slot of the tile layout (in the locality order of
// mds_reorder neighbouring slots hold nearby items), four slots per thread
// per round with their loads issued together, and thread 0 takes the
// decision.  Per-pair arithmetic is in the precision of the context's state
// (FP32 with CUDA's erfcf / log1pf, or FP64), sums in FP64.  The FP32 path
// skips log Phi where both z = delta / sigma are >= 8 (each term is then
// below 6.3e-16), as the pair pass does.  Held-out pairs of a
// cross-validation fold (y < 0 in the tile layout) are left out, as in the
// training likelihood.
#include <cmath>
#include <cstdint>

#include "mds_internal.h"
#include "philox.cuh"

namespace mds {
namespace {

constexpr int kRwThreads = 1024;
constexpr int kRwUnroll = 4;  // slots per thread per round

// r_ij(delta_old) - r_ij(delta_new) of Eq. (2) for one pair.  FP64: CUDA's
// erfc and log1p.  FP32: Phi(z) = D(z) - phi(z) P(z) over D(z), the Mills-ratio
// rational of the pair pass (coefficients folded with sigma on the host), so
// the difference of the log Phi terms is one log2 of a ratio; where both
// z >= 8 it is below 6.3e-16 and dropped.
__device__ __forceinline__ float poly3(const float *c, float d) { return fmaf(fmaf(fmaf(c[3], d, c[2]), d, c[1]), d, c[0]); }

__device__ __forceinline__ float phi_term_ratio(const RwmhArgs &a, float d0, float d1) {
    // D Phi = D + exp(-z^2/2) (-P / sqrt(2 pi)) at each distance
    const float e0 = exp2f(a.c_phi * d0 * d0), e1 = exp2f(a.c_phi * d1 * d1);
    const float dd0 = poly3(a.md, d0), dd1 = poly3(a.md, d1);
    const float den0 = fmaf(e0, poly3(a.mp, d0), dd0), den1 = fmaf(e1, poly3(a.mp, d1), dd1);
    // log Phi(z0) - log Phi(z1) = ln((den0 dd1) / (dd0 den1))
    return 0.69314718055994531f * __log2f((den0 * dd1) / (dd0 * den1));
}

template <typename T>
__device__ __forceinline__ T r_diff(const RwmhArgs &a, T y, T d0, T d1, T half_inv_s2, T inv_s_sqrt2, T far_delta) {
    const T e0 = y - d0, e1 = y - d1;
    T q = (e0 * e0 - e1 * e1) * half_inv_s2;
    if constexpr (sizeof(T) == 4) {
        if (d0 < far_delta || d1 < far_delta) q += phi_term_ratio(a, d0, d1);
    } else {
        q += log1p(-0.5 * erfc(d0 * inv_s_sqrt2)) - log1p(-0.5 * erfc(d1 * inv_s_sqrt2));
    }
    return q;
}

// Draws of proposals [0, n_prop) from Philox4x32-10, in parallel: proposal
// `it` = iter0 + t uses counter (it, 0, chain, 3) for the item
// floor(word0 N / 2^32) and u (word 1), and (it, 1 + q, chain, 3) for the z
// components 4q .. 4q + 3 (Box-Muller); log u is stored.
template <int D>
__global__ void rwmh_draws_kernel(RwmhArgs a, int64_t *items, double *z, double *logu) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_prop) return;
    const uint32_t it = static_cast<uint32_t>(a.iter0 + t);
    uint32_t c[4] = {it, 0u, a.chain, 3u};
    philox10(c, a.seed);
    items[t] = static_cast<int64_t>((static_cast<uint64_t>(c[0]) * static_cast<uint64_t>(a.n)) >> 32);
    logu[t] = log(open_unit(c[1]));
#pragma unroll
    for (int q = 0; 4 * q < D; ++q) {
        uint32_t c2[4] = {it, 1u + static_cast<uint32_t>(q), a.chain, 3u};
        philox10(c2, a.seed);
        double zz[4];
        box_muller(c2[0], c2[1], zz[0], zz[1]);
        box_muller(c2[2], c2[3], zz[2], zz[3]);
#pragma unroll
        for (int h = 0; h < 4; ++h)
            if (4 * q + h < D) z[static_cast<int64_t>(t) * D + 4 * q + h] = zz[h];
    }
}

constexpr int kRwSlotRegs = 8;  // slots per thread whose items stay in registers (N <= 8192)

// The chain.  X is kept in shared memory when a.x_in_smem (N D values), the
// items of this thread's slots in registers when N <= kRwSlotRegs * threads;
// thread 0 prefetches the next proposal's draws while the block works.
template <typename T, int D>
__global__ void __launch_bounds__(kRwThreads) rwmh_kernel(const __grid_constant__ RwmhArgs a) {
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ T xo[D], xn[D];
    __shared__ int64_t s_item, s_slot;
    __shared__ double sm[kRwThreads / 32];
    T *xg = static_cast<T *>(a.x);
    T *xs = a.x_in_smem ? reinterpret_cast<T *>(rsm) : xg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T half_inv_s2 = static_cast<T>(0.5 / (a.sigma * a.sigma));
    const T inv_s_sqrt2 = static_cast<T>(0.70710678118654752440 / a.sigma);
    const T far_delta = static_cast<T>(8.0 * a.sigma);
    const int64_t n = a.n;
    if (a.x_in_smem)
        for (int64_t e = tid; e < n * D; e += kRwThreads) xs[e] = xg[e];
    // items of this thread's slots (fixed for the whole chain)
    const bool slots_in_regs = n <= static_cast<int64_t>(kRwSlotRegs) * kRwThreads;
    int32_t my_item[kRwSlotRegs];
#pragma unroll
    for (int r = 0; r < kRwSlotRegs; ++r) {
        const int64_t sj = tid + static_cast<int64_t>(r) * kRwThreads;
        my_item[r] = (slots_in_regs && sj < n) ? static_cast<int32_t>(a.perm ? a.perm[sj] : sj) : -1;
    }
    // thread 0: the draws of the current proposal (and the next one, prefetched)
    int64_t i_cur = 0, si_cur = 0;
    double z_cur[D], lu_cur = 0.0;
    if (tid == 0 && a.n_prop > 0) {
        i_cur = a.items[0];
        si_cur = (a.inv && i_cur >= 0 && i_cur < n) ? a.inv[i_cur] : i_cur;
#pragma unroll
        for (int k = 0; k < D; ++k) z_cur[k] = a.z[k];
        lu_cur = a.logu[0];
    }
    __syncthreads();
    for (int t = 0; t < a.n_prop; ++t) {
        int64_t i_nxt = 0, si_nxt = 0;
        double z_nxt[D], lu_nxt = 0.0;
        if (tid == 0) {
            if (t + 1 < a.n_prop) {
                i_nxt = a.items[t + 1];
                si_nxt = (a.inv && i_nxt >= 0 && i_nxt < n) ? a.inv[i_nxt] : i_nxt;
#pragma unroll
                for (int k = 0; k < D; ++k) z_nxt[k] = a.z[static_cast<int64_t>(t + 1) * D + k];
                lu_nxt = a.logu[t + 1];
            }
            if (i_cur < 0 || i_cur >= n) {
                atomicOr(a.err, kErrBadArgs);
                i_cur = 0;
                si_cur = a.inv ? a.inv[0] : 0;
                lu_cur = INFINITY;  // never accepted
#pragma unroll
                for (int k = 0; k < D; ++k) z_cur[k] = 0.0;
            }
            s_item = i_cur;
            s_slot = si_cur;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T v = xs[i_cur * D + k];
                xo[k] = v;
                xn[k] = v + static_cast<T>(a.step * z_cur[k]);
            }
        }
        __syncthreads();
        const int64_t i = s_item;
        const int64_t si = s_slot;
        // this thread's share of the row: a compensated sum in the pair
        // arithmetic's precision (FP64 conversions run at 1/64 rate on this
        // GPU), widened to FP64 once before the block sum
        T acc_s = T(0), acc_c = T(0);
        const int rounds = static_cast<int>((n + kRwThreads - 1) / kRwThreads);
        for (int r0 = 0; r0 < rounds; r0 += kRwUnroll) {
            int64_t item[kRwUnroll];
            float yv[kRwUnroll];
#pragma unroll
            for (int u = 0; u < kRwUnroll; ++u) {
                const int r = r0 + u;
                const int64_t sj = tid + static_cast<int64_t>(r) * kRwThreads;
                int64_t it = -1;
                if (sj < n && sj != si) {
                    if (slots_in_regs) {
#pragma unroll
                        for (int q = 0; q < kRwSlotRegs; ++q)
                            if (q == r) it = my_item[q];
                    } else {
                        it = a.perm ? a.perm[sj] : sj;
                    }
                }
                item[u] = it;
                yv[u] = -1.f;
                if (it >= 0) {
                    const int64_t lo = si < sj ? si : sj, hi = si < sj ? sj : si;
                    const int64_t I = lo / kTile, J = hi / kTile;
                    yv[u] = a.y[tile_index(I, J, a.nt) * kTileElems +
                                tile_offset(static_cast<int>(lo - I * kTile), static_cast<int>(hi - J * kTile))];
                }
            }
#pragma unroll
            for (int u = 0; u < kRwUnroll; ++u) {
                if (item[u] < 0 || yv[u] < 0.f) continue;  // past N, the item itself, or held out
                T d0 = T(0), d1 = T(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T xj = xs[item[u] * D + k];
                    const T a0 = xo[k] - xj, a1 = xn[k] - xj;
                    d0 += a0 * a0;
                    d1 += a1 * a1;
                }
                const T y = static_cast<T>(yv[u]);
                const T v = r_diff<T>(a, y, sqrt(d0), sqrt(d1), half_inv_s2, inv_s_sqrt2, far_delta);
                const T yk = v - acc_c;  // Kahan
                const T tk = acc_s + yk;
                acc_c = (tk - acc_s) - yk;
                acc_s = tk;
            }
        }
        // fixed-order block sum: (sum, compensation) pairs through the warp,
        // FP64 only for the 32 warp totals
        T hs = acc_s, hc = acc_c;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const T os = __shfl_xor_sync(0xffffffffu, hs, o), oc = __shfl_xor_sync(0xffffffffu, hc, o);
            const T s2 = hs + os;
            const T bb = s2 - hs;
            const T err = (hs - (s2 - bb)) + (os - bb);  // exact rounding error of hs + os
            hs = s2;
            hc = hc + oc - err;
        }
        if (lane == 0) sm[warp] = static_cast<double>(hs) - static_cast<double>(hc);
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
            const bool keep = isfinite(lp) && lu_cur < lp;
            if (keep) {
                float mx = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    xs[i * D + k] = xn[k];
                    xg[i * D + k] = xn[k];
                    mx = fmaxf(mx, fabsf(static_cast<float>(xn[k])));
                }
                if (a.xmax_bits && mx > 0.f) atomicMax(a.xmax_bits, __float_as_uint(mx));
            }
            if (!isfinite(lp)) atomicOr(a.err, kErrNonfinite);
            if (a.acc_out) a.acc_out[t] = keep ? 1 : 0;
            if (a.dl_out) a.dl_out[t] = lp;
            i_cur = i_nxt;
            si_cur = si_nxt;
#pragma unroll
            for (int k = 0; k < D; ++k) z_cur[k] = z_nxt[k];
            lu_cur = lu_nxt;
        }
        __syncthreads();  // x and the shared proposal are settled before the next one
    }
}

template <int D>
cudaError_t launch_d(const RwmhArgs &a, cudaStream_t s) {
    const size_t xbytes = static_cast<size_t>(a.n) * D * (a.fp64 ? 8 : 4);
    const int smem = a.x_in_smem ? static_cast<int>(xbytes) : 0;
    cudaError_t e = cudaSuccess;
    if (a.fp64) {
        if (smem) e = cudaFuncSetAttribute(rwmh_kernel<double, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) rwmh_kernel<double, D><<<1, kRwThreads, smem, s>>>(a);
    } else {
        if (smem) e = cudaFuncSetAttribute(rwmh_kernel<float, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) rwmh_kernel<float, D><<<1, kRwThreads, smem, s>>>(a);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int D>
cudaError_t launch_draws_d(const RwmhArgs &a, int64_t *items, double *z, double *logu, cudaStream_t s) {
    rwmh_draws_kernel<D><<<(a.n_prop + 255) / 256, 256, 0, s>>>(a, items, z, logu);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rwmh_draws(const RwmhArgs &a, int d, int64_t *items, double *z, double *logu, cudaStream_t s) {
    if (a.n_prop <= 0) return cudaSuccess;
    switch (d) {
        case 1: return launch_draws_d<1>(a, items, z, logu, s);
        case 2: return launch_draws_d<2>(a, items, z, logu, s);
        case 3: return launch_draws_d<3>(a, items, z, logu, s);
        case 4: return launch_draws_d<4>(a, items, z, logu, s);
        case 5: return launch_draws_d<5>(a, items, z, logu, s);
        case 6: return launch_draws_d<6>(a, items, z, logu, s);
        case 7: return launch_draws_d<7>(a, items, z, logu, s);
        case 8: return launch_draws_d<8>(a, items, z, logu, s);
        default: return cudaErrorInvalidValue;
    }
}

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
