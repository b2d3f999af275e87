// Single-item random-walk Metropolis: the prior-art sampler that section
// 2.3 of arXiv:1905.04582 contrasts HMC with (a low-dimensional random-walk
// kernel applied to one x_i at a time).  Moving x_i changes only the N - 1
// terms r_ij, j != i, so a proposal costs O(N D): its log-target difference
// is
//   L(X') - L(X) = sum_{j != i} [r_ij(x_i) - r_ij(x_i')] - (lambda/2)(|x_i'|^2 - |x_i|^2)
// (the -M log sigma of Eq. (2) cancels).  Proposals are sequential (each
// depends on the decisions before it), so one cluster of CTAs runs them in a
// loop: its threads split the row by slot of the tile layout (in the locality
// order of mds_reorder neighbouring slots hold nearby items), four slots per
// thread per round with their loads issued together, the CTAs' partial sums
// meet through distributed shared memory, and thread 0 of every CTA takes
// the same decision.  Per-pair arithmetic is in the precision of the context's state
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

// (s, c): a sum and the compensation to subtract from it; the 32 lanes'
// pairs added in a fixed butterfly, each addition's rounding error carried
// (two-sum), so every lane ends with the same pair.
template <typename T>
__device__ __forceinline__ void pair_tree(T &hs, T &hc) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const T os = __shfl_xor_sync(0xffffffffu, hs, o), oc = __shfl_xor_sync(0xffffffffu, hc, o);
        const T s2 = hs + os;
        const T bb = s2 - hs;
        const T err = (hs - (s2 - bb)) + (os - bb);  // exact rounding error of hs + os
        hs = s2;
        hc = hc + oc - err;
    }
}

constexpr int kRwSlotRegs = 8;  // slots per thread whose items stay in registers
constexpr int kRwMaxCluster = 8;

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

// v into the shared-memory word `local` of CTA `rank` of this cluster.
__device__ __forceinline__ void st_cluster(double *local, unsigned rank, double v) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(local));
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

// The chain, on one cluster of a.cluster CTAs (gridDim.x).  Every CTA keeps
// its own copy of X (shared memory when a.x_in_smem, which a cluster of more
// than one CTA requires), takes the rounds r = rank, rank + C, ... of the
// row's 1024-slot rounds, and sends its partial sum of the row to every
// CTA; after one cluster barrier per proposal each CTA adds the C partials
// in rank order and takes the same decision.  CTA 0 writes the state and the
// outputs.  Thread 0 of each CTA prefetches the next proposal's draws while
// the block works.
template <typename T, int D>
__global__ void __launch_bounds__(kRwThreads) rwmh_kernel(const __grid_constant__ RwmhArgs a) {
    extern __shared__ __align__(16) unsigned char rsm[];
    __shared__ T xo[D], xn[D];
    __shared__ int64_t s_item, s_slot;
    __shared__ T sm_s[kRwThreads / 32], sm_c[kRwThreads / 32];
    __shared__ double s_dsq;  // |x_i'|^2 - |x_i|^2 of the current proposal
    __shared__ double cl_part[2][kRwMaxCluster];  // per proposal parity: the CTAs' partial sums
    T *xg = static_cast<T *>(a.x);
    T *xs = a.x_in_smem ? reinterpret_cast<T *>(rsm) : xg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncl = static_cast<int>(gridDim.x), rank = static_cast<int>(blockIdx.x);
    const T half_inv_s2 = static_cast<T>(0.5 / (a.sigma * a.sigma));
    const T inv_s_sqrt2 = static_cast<T>(0.70710678118654752440 / a.sigma);
    const T far_delta = static_cast<T>(8.0 * a.sigma);
    const int64_t n = a.n;
    if (a.x_in_smem)
        for (int64_t e = tid; e < n * D; e += kRwThreads) xs[e] = xg[e];
    // this CTA's rounds of the row: r = rank + lr * ncl, lr < nr
    const int rounds = static_cast<int>((n + kRwThreads - 1) / kRwThreads);
    const int nr = rounds > rank ? (rounds - rank + ncl - 1) / ncl : 0;
    // items of this thread's slots (fixed for the whole chain)
    const bool slots_in_regs = nr <= kRwSlotRegs;
    int32_t my_item[kRwSlotRegs];
#pragma unroll
    for (int q = 0; q < kRwSlotRegs; ++q) {
        const int64_t sj = tid + static_cast<int64_t>(rank + q * ncl) * kRwThreads;
        my_item[q] = (slots_in_regs && q < nr && sj < n) ? static_cast<int32_t>(a.perm ? a.perm[sj] : sj) : -1;
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
            double sq0 = 0.0, sq1 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T v = xs[i_cur * D + k];
                const T w = v + static_cast<T>(a.step * z_cur[k]);
                xo[k] = v;
                xn[k] = w;
                sq0 += static_cast<double>(v) * static_cast<double>(v);
                sq1 += static_cast<double>(w) * static_cast<double>(w);
            }
            s_dsq = sq1 - sq0;
        }
        __syncthreads();
        const int64_t i = s_item;
        const int64_t si = s_slot;
        // this thread's share of the row: a compensated sum in the pair
        // arithmetic's precision (FP64 conversions run at 1/64 rate on this
        // GPU), widened to FP64 once before the block sum
        T acc_s = T(0), acc_c = T(0);
        for (int lr0 = 0; lr0 < nr; lr0 += kRwUnroll) {
            int64_t item[kRwUnroll];
            float yv[kRwUnroll];
#pragma unroll
            for (int u = 0; u < kRwUnroll; ++u) {
                const int lr = lr0 + u;
                const int64_t sj = tid + static_cast<int64_t>(rank + lr * ncl) * kRwThreads;
                int64_t it = -1;
                if (lr < nr && sj < n && sj != si) {
                    if (slots_in_regs) {
#pragma unroll
                        for (int q = 0; q < kRwSlotRegs; ++q)
                            if (q == lr) it = my_item[q];
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
        // fixed-order block sum of (sum, compensation) pairs: a shuffle tree
        // in each warp, then one over the 32 warp totals in warp 0 (trees,
        // not serial sums: a dependent FP64 addition costs ~64 cycles here);
        // then the CTA's partial to every CTA of the cluster
        T hs = acc_s, hc = acc_c;
        pair_tree(hs, hc);
        if (lane == 0) {
            sm_s[warp] = hs;
            sm_c[warp] = hc;
        }
        __syncthreads();
        if (warp == 0) {
            hs = sm_s[lane];
            hc = sm_c[lane];
            pair_tree(hs, hc);
            if (lane == 0) {
                const double dc = static_cast<double>(hs) - static_cast<double>(hc);
                for (int r = 0; r < ncl; ++r) st_cluster(&cl_part[t & 1][rank], static_cast<unsigned>(r), dc);
            }
        }
        // the partials of proposal t are in every CTA; a partial of proposal
        // t + 2 (same buffer) is written only after every CTA has passed the
        // next barrier, that is after it has read these
        cluster_sync_all();
        if (tid == 0) {
            double dl = 0.0;
            for (int r = 0; r < ncl; ++r) dl += cl_part[t & 1][r];
            const double lp = dl - 0.5 * a.lambda * s_dsq;
            const bool keep = isfinite(lp) && lu_cur < lp;
            if (keep) {
                float mx = 0.f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    xs[i * D + k] = xn[k];
                    if (rank == 0) xg[i * D + k] = xn[k];
                    mx = fmaxf(mx, fabsf(static_cast<float>(xn[k])));
                }
                if (rank == 0 && a.xmax_bits && mx > 0.f) atomicMax(a.xmax_bits, __float_as_uint(mx));
            }
            if (rank == 0) {
                if (!isfinite(lp)) atomicOr(a.err, kErrNonfinite);
                if (a.acc_out) a.acc_out[t] = keep ? 1 : 0;
                if (a.dl_out) a.dl_out[t] = lp;
            }
            i_cur = i_nxt;
            si_cur = si_nxt;
#pragma unroll
            for (int k = 0; k < D; ++k) z_cur[k] = z_nxt[k];
            lu_cur = lu_nxt;
        }
        __syncthreads();  // x and the shared proposal are settled before the next one
    }
}

template <typename T, int D>
cudaError_t launch_td(const RwmhArgs &a, int smem, cudaStream_t s) {
    if (smem) {
        const cudaError_t e =
            cudaFuncSetAttribute(rwmh_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(a.cluster));
    cfg.blockDim = dim3(kRwThreads);
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(a.cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, rwmh_kernel<T, D>, a);
}

template <int D>
cudaError_t launch_d(const RwmhArgs &a, cudaStream_t s) {
    // a cluster of several CTAs needs each CTA's own copy of X
    if (a.cluster < 1 || a.cluster > kRwMaxCluster || (a.cluster > 1 && !a.x_in_smem)) return cudaErrorInvalidValue;
    const size_t xbytes = static_cast<size_t>(a.n) * D * (a.fp64 ? 8 : 4);
    const int smem = a.x_in_smem ? static_cast<int>(xbytes) : 0;
    const cudaError_t e = a.fp64 ? launch_td<double, D>(a, smem, s) : launch_td<float, D>(a, smem, s);
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
