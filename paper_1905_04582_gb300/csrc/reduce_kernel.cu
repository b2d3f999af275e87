// Second level of the pair pass and the device-side HMC bookkeeping
// (arXiv:1905.04582, section 2.3 "Hamiltonian Monte Carlo", Eq. (6)-(9);
// the final, serial reduction of Algorithm 1 moved onto the device).
//
// reduce:     per column block J of 64 items, gradient of x_k =
//               sum over tiles (I, J), I <= J, of the column partials
//             - sum over the strips of row block J of the row partials,
//             summed in FP64 in a fixed order (4 interleaved splits, then the
//             splits in order), so results are bitwise reproducible.  The
//             last CTA sums the strips' scalar partials into L, sum r and
//             dL/dsigma.  Leapfrog modes also update p and x of the block.
// traj_start: momentum draw (Philox4x32-10 + Box-Muller) or injection,
//             saves the start state, first half kick + drift.
// traj_end:   energies H = -log pi + p^T p / 2 (FP64), Metropolis decision,
//             restore on reject.
// ingest:     Y (full or packed, f32/f64) -> tile-packed FP32 with checks.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "mds_internal.h"

namespace mds {
namespace {

constexpr int kRedThreads = 256;  // 64 items x 4 splits
constexpr int kSplits = kRedThreads / kTile;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kSqrt2Pi = 2.50662827463100050242;
constexpr double kTwoPi = 6.28318530717958647693;

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// Write one coordinate of item k into the negated, column-pair interleaved copy.
template <typename T>
__device__ __forceinline__ void store_xneg(void *xneg, int64_t k, int d, int kk, T v) {
    T *base = reinterpret_cast<T *>(xneg);
    base[((k >> 1) * d + kk) * 2 + (k & 1)] = -v;
}

// Fixed-order block sum of two doubles per thread (power-of-two blockDim).
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *sm) {
    const int tid = threadIdx.x;
    sm[tid] = a;
    sm[NT + tid] = b;
    __syncthreads();
#pragma unroll
    for (int o = NT / 2; o >= 1; o >>= 1) {
        if (tid < o) {
            sm[tid] += sm[tid + o];
            sm[NT + tid] += sm[NT + tid + o];
        }
        __syncthreads();
    }
    a = sm[0];
    b = sm[NT];
}

// --------------------------------------------------------------- reduce

template <typename T, int D>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const __grid_constant__ ReduceArgs a) {
    __shared__ double sm[kSplits * kTile * D > 2 * kRedThreads ? kSplits * kTile * D : 2 * kRedThreads];
    const int tid = threadIdx.x;
    const int nt = a.nt;

    if (blockIdx.x == static_cast<unsigned>(nt)) {
        // scalar partials of all strips -> L, sum r, dL/dsigma (FP64, fixed order)
        double e2 = 0.0, md = 0.0, lp = 0.0;
        for (int s = tid; s < a.n_strips; s += kRedThreads) {
            const double *sp = a.scal_part + static_cast<int64_t>(s) * kScalarParts;
            e2 += sp[kSumE2];
            md += sp[kSumMDelta];
            lp += sp[kSumLogPhi];
        }
        double dummy = 0.0;
        block_sum2<kRedThreads>(e2, md, sm);
        __syncthreads();
        block_sum2<kRedThreads>(lp, dummy, sm);
        if (tid == 0) {
            const double sg = a.sigma;
            const double m = 0.5 * static_cast<double>(a.n) * static_cast<double>(a.n - 1);
            double sum_logphi, sum_mdelta;
            if (a.fp64) {
                sum_logphi = lp;
                sum_mdelta = md;
            } else {
                sum_logphi = -kLn2 * lp;         // lp = sum log2(1/Phi)
                sum_mdelta = md / kSqrt2Pi;      // md = sum sqrt(2 pi) (phi/Phi) delta
            }
            const double sum_r = e2 / (2.0 * sg * sg) + sum_logphi;
            const double ll = -m * log(sg) - sum_r;
            const double ds = -m / sg + e2 / (sg * sg * sg) + sum_mdelta / (sg * sg);
            a.scal[kLogLik] = ll;
            a.scal[kSumR] = sum_r;
            a.scal[kDSigma] = ds;
            a.scal[kLogLikEnd] = ll;
            if (!isfinite(ll) || !isfinite(ds)) atomicOr(a.err, kErrNonfinite);
        }
        return;
    }

    const int J = blockIdx.x;
    const int r = tid & (kTile - 1);
    const int s = tid / kTile;
    const int64_t k = static_cast<int64_t>(J) * kTile + r;
    double acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.0;
    const T *cp = reinterpret_cast<const T *>(a.col_part);
    for (int I = s; I <= J; I += kSplits) {
        const T *c = cp + (tile_index(I, J, nt) * kTile + r) * D;
#pragma unroll
        for (int d = 0; d < D; ++d) acc[d] += static_cast<double>(c[d]);
    }
    const int s0 = a.row_first_slot[J], s1 = a.row_first_slot[J + 1];
    for (int slot = s0 + s; slot < s1; slot += kSplits) {
        const double *rp = a.row_part + (static_cast<int64_t>(slot) * kTile + r) * D;
#pragma unroll
        for (int d = 0; d < D; ++d) acc[d] -= rp[d];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) sm[(s * kTile + r) * D + d] = acc[d];
    __syncthreads();

    double ke = 0.0, xx = 0.0;
    if (s == 0 && k < a.n) {
        T *x = reinterpret_cast<T *>(a.x);
        T *p = reinterpret_cast<T *>(a.p);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            double g = sm[r * D + d];
#pragma unroll
            for (int q = 1; q < kSplits; ++q) g += sm[(q * kTile + r) * D + d];
            a.grad[k * D + d] = g;
            bad |= !isfinite(g);
            if (a.mode != kModeEval) {
                const double xv = static_cast<double>(x[k * D + d]);
                const double tg = g - a.lambda * xv;  // gradient of log pi
                if (a.mode == kModeKickDrift) {
                    const T pn = static_cast<T>(static_cast<double>(p[k * D + d]) + a.eps * tg);
                    const T xn = static_cast<T>(xv + a.eps * static_cast<double>(pn));
                    p[k * D + d] = pn;
                    x[k * D + d] = xn;
                    store_xneg<T>(a.xneg, k, D, d, xn);
                } else {  // kModeHalfKick
                    const T pn = static_cast<T>(static_cast<double>(p[k * D + d]) + 0.5 * a.eps * tg);
                    p[k * D + d] = pn;
                    ke += 0.5 * static_cast<double>(pn) * static_cast<double>(pn);
                    xx += xv * xv;
                }
            }
        }
        if (bad) atomicOr(a.err, kErrNonfinite);
    }
    if (a.mode == kModeHalfKick) {
        __syncthreads();
        block_sum2<kRedThreads>(ke, xx, sm);
        if (tid == 0) {
            a.energy_part[2 * J] = ke;
            a.energy_part[2 * J + 1] = xx;
        }
    }
}

// ------------------------------------------------------------ Philox / RNG

__device__ __forceinline__ void philox_round(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key schedule.
__device__ __forceinline__ void philox10(uint32_t (&c)[4], uint64_t key) {
    uint32_t k0 = static_cast<uint32_t>(key), k1 = static_cast<uint32_t>(key >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
}

__device__ __forceinline__ double open_unit(uint32_t b) { return (static_cast<double>(b) + 0.5) * (1.0 / 4294967296.0); }

// ----------------------------------------------------------- traj start

constexpr int kTrajThreads = 256;

template <typename T, int D>
__global__ void __launch_bounds__(kTrajThreads) traj_start_kernel(const __grid_constant__ TrajArgs a) {
    __shared__ double sm[2 * kTrajThreads];
    const int64_t nd = a.n * D;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * kTrajThreads + threadIdx.x;  // 4 elements each
    T *x = reinterpret_cast<T *>(a.x);
    T *p = reinterpret_cast<T *>(a.p);
    T *x0 = reinterpret_cast<T *>(a.x0);
    const int64_t iter = a.counters[kIter];
    const int64_t iter_local = a.counters[kIterLocal];
    double ke = 0.0, xx = 0.0;
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    if (a.momentum_src == 1 && 4 * q < nd) {
        uint32_t c[4] = {static_cast<uint32_t>(q), static_cast<uint32_t>(iter), a.chain, 0u};
        philox10(c, a.seed);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double u1 = open_unit(c[2 * h]);
            const double u2 = open_unit(c[2 * h + 1]);
            const double rad = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincos(kTwoPi * u2, &sn, &cs);
            z[2 * h] = rad * cs;
            z[2 * h + 1] = rad * sn;
        }
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int64_t e = 4 * q + h;
        if (e >= nd) break;
        T pv;
        if (a.momentum_src == 1)
            pv = static_cast<T>(z[h]);
        else if (a.momentum_src == 2)
            pv = static_cast<T>(a.p_inj[iter_local * nd + e]);
        else
            pv = p[e];
        const T xv = x[e];
        x0[e] = xv;
        a.grad0[e] = a.grad[e];
        ke += 0.5 * static_cast<double>(pv) * static_cast<double>(pv);
        xx += static_cast<double>(xv) * static_cast<double>(xv);
        if (a.drift) {
            const double tg = a.grad[e] - a.lambda * static_cast<double>(xv);
            pv = static_cast<T>(static_cast<double>(pv) + 0.5 * a.eps * tg);
            const T xn = static_cast<T>(static_cast<double>(xv) + a.eps * static_cast<double>(pv));
            x[e] = xn;
            store_xneg<T>(a.xneg, e / D, D, static_cast<int>(e % D), xn);
        }
        p[e] = pv;
    }
    block_sum2<kTrajThreads>(ke, xx, sm);
    if (threadIdx.x == 0) {
        a.energy_part[2 * blockIdx.x] = ke;
        a.energy_part[2 * blockIdx.x + 1] = xx;
        if (blockIdx.x == 0) {
            a.scal[kLogLik0] = a.scal[kLogLik];
            a.scal[kSumR0] = a.scal[kSumR];
            a.scal[kDSigma0] = a.scal[kDSigma];
            a.counters[kIterCur] = iter;
            a.counters[kIterLocalCur] = iter_local;
        }
    }
}

// ------------------------------------------------------------- traj end

template <typename T, int D>
__global__ void __launch_bounds__(kTrajThreads) traj_end_kernel(const __grid_constant__ AcceptArgs a) {
    // every CTA sums the same partials in the same order -> same decision
    __shared__ int keep_s;
    __shared__ double dh_s;
    if (threadIdx.x == 0) {
        double ke0 = 0.0, xx0 = 0.0, ke1 = 0.0, xx1 = 0.0;
        for (int i = 0; i < a.n_start_parts; ++i) {
            ke0 += a.start_part[2 * i];
            xx0 += a.start_part[2 * i + 1];
        }
        for (int i = 0; i < a.n_end_parts; ++i) {
            ke1 += a.end_part[2 * i];
            xx1 += a.end_part[2 * i + 1];
        }
        const double h0 = -(a.scal[kLogLik0] - 0.5 * a.lambda * xx0) + ke0;
        const double h1 = -(a.scal[kLogLikEnd] - 0.5 * a.lambda * xx1) + ke1;
        const double dh = h1 - h0;
        int keep = 1;
        if (a.metropolis) {
            const int64_t iter = a.counters[kIterCur];
            double u;
            if (a.u_src == 2) {
                u = a.u_inj[a.counters[kIterLocalCur]];
            } else {
                uint32_t c[4] = {0u, static_cast<uint32_t>(iter), a.chain, 1u};
                philox10(c, a.seed);
                u = open_unit(c[0]);
            }
            keep = (isfinite(dh) && log(u) < -dh) ? 1 : 0;
        }
        keep_s = keep;
        dh_s = dh;
    }
    __syncthreads();
    const int keep = keep_s;
    const int64_t nd = a.n * D;
    if (!keep) {
        T *x = reinterpret_cast<T *>(a.x);
        const T *x0 = reinterpret_cast<const T *>(a.x0);
        for (int64_t e = static_cast<int64_t>(blockIdx.x) * kTrajThreads + threadIdx.x; e < nd;
             e += static_cast<int64_t>(gridDim.x) * kTrajThreads) {
            const T xv = x0[e];
            x[e] = xv;
            a.grad[e] = a.grad0[e];
            store_xneg<T>(a.xneg, e / D, D, static_cast<int>(e % D), xv);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double dh = dh_s;
        if (!isfinite(dh)) atomicOr(a.err, kErrNonfinite);
        a.scal[kLastDH] = dh;
        if (!keep) {
            a.scal[kLogLik] = a.scal[kLogLik0];
            a.scal[kSumR] = a.scal[kSumR0];
            a.scal[kDSigma] = a.scal[kDSigma0];
        }
        const int64_t il = a.counters[kIterLocalCur];
        if (a.acc_out) a.acc_out[il] = keep;
        if (a.dh_out) a.dh_out[il] = dh;
        if (a.metropolis) {
            a.counters[kIter] = a.counters[kIterCur] + 1;
            a.counters[kIterLocal] = il + 1;
            a.counters[kAccepted] += keep;
        }
    }
}

#define MDS_SWITCH_D(KERNEL, T, GRID, BLOCK, STREAM, ARGS)                        \
    switch ((ARGS).d) {                                                          \
        case 1: KERNEL<T, 1><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 2: KERNEL<T, 2><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 3: KERNEL<T, 3><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 4: KERNEL<T, 4><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 5: KERNEL<T, 5><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 6: KERNEL<T, 6><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 7: KERNEL<T, 7><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        case 8: KERNEL<T, 8><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;           \
        default: return cudaErrorInvalidValue;                                   \
    }

// ----------------------------------------------------------------- ingest

// One thread per destination element of the tiles of row blocks covering
// rows [r0, r1).
__global__ void ingest_kernel(const __grid_constant__ IngestArgs a) {
    const int64_t nt = a.nt;
    const int64_t b0 = a.r0 / kTile;
    const int64_t b1 = (a.r1 + kTile - 1) / kTile;
    const int64_t t_begin = tile_index(b0, b0, nt);
    const int64_t t_end = tile_index(b1 - 1, nt - 1, nt) + 1;
    const int64_t total = (t_end - t_begin) * kTileElems;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t t = t_begin + g / kTileElems;
        const int off = static_cast<int>(g % kTileElems);
        // locate tile (I, J): row block I is the largest with tile_index(I, I) <= t
        int64_t lo = b0, hi = b1 - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (tile_index(mid, mid, nt) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t I = lo;
        const int64_t J = I + (t - tile_index(I, I, nt));
        const int chunk = off / (kTile * kChunkCols);
        const int rem = off % (kTile * kChunkCols);
        const int rr = rem / kChunkCols;
        const int cc = chunk * kChunkCols + rem % kChunkCols;
        const int64_t i = I * kTile + rr;
        const int64_t j = J * kTile + cc;
        float v = 0.0f;
        if (i < j && j < a.n && i >= a.r0 && i < a.r1) {
            double y;
            int64_t idx;
            if (a.packed)
                idx = packed_row_start(i, a.n) - packed_row_start(a.r0, a.n) + (j - i - 1);
            else
                idx = (i - a.r0) * a.ld + j;
            if (a.src_f64)
                y = reinterpret_cast<const double *>(a.src)[idx];
            else
                y = static_cast<double>(reinterpret_cast<const float *>(a.src)[idx]);
            if (!(y >= 0.0) || !isfinite(y)) {
                atomicOr(a.err, kErrBadInput);
                atomicMin(a.bad, static_cast<unsigned long long>(i * a.n + j));
            }
            v = static_cast<float>(y);
        }
        if (i >= a.r0 && i < a.r1) a.y[t * kTileElems + off] = v;
        else if (i >= a.n) a.y[t * kTileElems + off] = 0.0f;  // padding rows of the last block
    }
}

// --------------------------------------------------------------- set x

template <typename T, typename S>
__global__ void set_x_kernel(const S *src, int64_t n, int64_t n_pad, int d, T *x, T *xneg, unsigned *err) {
    const int64_t total = n_pad * d;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = e / d;
        T v = T(0);
        if (k < n) {
            const double sv = static_cast<double>(src[e]);
            if (!isfinite(sv)) atomicOr(err, kErrBadInput);
            v = static_cast<T>(sv);
        }
        x[e] = v;
        store_xneg<T>(xneg, k, d, static_cast<int>(e % d), v);
    }
}

template <typename S, typename T>
__global__ void convert_kernel(const S *src, T *dst, int64_t count) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[e] = static_cast<T>(src[e]);
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t s) {
    const dim3 grid(a.nt + 1);  // one CTA per column block + one for the scalars
    if (a.fp64) {
        MDS_SWITCH_D(reduce_kernel, double, grid, kRedThreads, s, a)
    } else {
        MDS_SWITCH_D(reduce_kernel, float, grid, kRedThreads, s, a)
    }
    return cudaGetLastError();
}

cudaError_t launch_traj_start(const TrajArgs &a, int *grid_out, cudaStream_t s) {
    const int64_t quads = (a.n * a.d + 3) / 4;
    const int grid = static_cast<int>((quads + kTrajThreads - 1) / kTrajThreads);
    if (grid_out) *grid_out = grid;
    if (a.fp64) {
        MDS_SWITCH_D(traj_start_kernel, double, grid, kTrajThreads, s, a)
    } else {
        MDS_SWITCH_D(traj_start_kernel, float, grid, kTrajThreads, s, a)
    }
    return cudaGetLastError();
}

cudaError_t launch_traj_end(const AcceptArgs &a, cudaStream_t s) {
    const int grid = grid_for(a.n * a.d, kTrajThreads);
    if (a.fp64) {
        MDS_SWITCH_D(traj_end_kernel, double, grid, kTrajThreads, s, a)
    } else {
        MDS_SWITCH_D(traj_end_kernel, float, grid, kTrajThreads, s, a)
    }
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs &a, cudaStream_t s) {
    const int64_t b0 = a.r0 / kTile, b1 = (a.r1 + kTile - 1) / kTile;
    const int64_t tiles = tile_index(b1 - 1, a.nt - 1, a.nt) + 1 - tile_index(b0, b0, a.nt);
    ingest_kernel<<<grid_for(tiles * kTileElems, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_x(const void *src, bool src_f64, int64_t n, int64_t n_pad, int d, bool fp64, void *x,
                         void *xneg, unsigned *err, cudaStream_t s) {
    const int g = grid_for(n_pad * d, 256);
    if (fp64) {
        if (src_f64)
            set_x_kernel<double, double><<<g, 256, 0, s>>>(static_cast<const double *>(src), n, n_pad, d,
                                                            static_cast<double *>(x), static_cast<double *>(xneg), err);
        else
            set_x_kernel<double, float><<<g, 256, 0, s>>>(static_cast<const float *>(src), n, n_pad, d,
                                                           static_cast<double *>(x), static_cast<double *>(xneg), err);
    } else {
        if (src_f64)
            set_x_kernel<float, double><<<g, 256, 0, s>>>(static_cast<const double *>(src), n, n_pad, d,
                                                           static_cast<float *>(x), static_cast<float *>(xneg), err);
        else
            set_x_kernel<float, float><<<g, 256, 0, s>>>(static_cast<const float *>(src), n, n_pad, d,
                                                          static_cast<float *>(x), static_cast<float *>(xneg), err);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t count, cudaStream_t s) {
    const int g = grid_for(count, 256);
    if (src_f64 && dst_f64)
        convert_kernel<double, double><<<g, 256, 0, s>>>(static_cast<const double *>(src), static_cast<double *>(dst), count);
    else if (src_f64)
        convert_kernel<double, float><<<g, 256, 0, s>>>(static_cast<const double *>(src), static_cast<float *>(dst), count);
    else if (dst_f64)
        convert_kernel<float, double><<<g, 256, 0, s>>>(static_cast<const float *>(src), static_cast<double *>(dst), count);
    else
        convert_kernel<float, float><<<g, 256, 0, s>>>(static_cast<const float *>(src), static_cast<float *>(dst), count);
    return cudaGetLastError();
}

}  // namespace mds
