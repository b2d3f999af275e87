// Second level of the pair pass and the device-side HMC bookkeeping
// (arXiv:1905.04582, section 2.3 "Hamiltonian Monte Carlo", Eq. (6)-(9);
// the final, serial reduction of Algorithm 1 moved onto the device).
//
// reduce:     per column block J of 64 items, the gradient of x_k is
//               sum over tiles (I, J), I <= J, of the column partials
//             - sum over the strips of row block J of the row partials,
//             summed in a fixed order (8 interleaved splits, then the splits
//             in order) so results are bitwise reproducible.  FP32C: the
//             partials are FP32 and the sums FP32 two-sums (a double-float
//             accumulator); FP64: plain FP64.  The last CTA sums the strips'
//             scalar partials into L, sum r and dL/dsigma (FP64 only in its
//             final few operations).  Leapfrog modes also update p and x of
//             the block and rewrite the split location layouts.
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
#include "philox.cuh"

namespace mds {
namespace {

// One CTA reduces a quarter of a column block (16 items) with 16 splits per
// item: small CTAs become resident beside the pair pass's last CTAs (the
// reduction is launched as a programmatic dependent), and one round of loads
// covers the partials of a block at N = 5392.
constexpr int kRedThreads = 256;
constexpr int kRedRows = 16;                       // items per CTA
constexpr int kRedQuarters = kReduceQuarters;      // CTAs per column block
static_assert(kRedQuarters * kRedRows == kTile, "quarters must cover a block");
constexpr int kSplits = kRedThreads / kRedRows;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kSqrt2Pi = 2.50662827463100050242;

// ------------------------------------------------- double-float accumulator

// hi + lo with |lo| <= ulp(hi)/2, updated with Knuth's two-sum.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DF &a, float v) {
    const float s = __fadd_rn(a.hi, v);
    const float bp = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}

__device__ __forceinline__ void df_add(DF &a, const DF &b) {
    df_add(a, b.hi);
    a.lo = __fadd_rn(a.lo, b.lo);
}

__device__ __forceinline__ float df_float(const DF &a) { return __fadd_rn(a.hi, a.lo); }

// Double-float product a * (b.x + b.y): the exact product of the leading
// parts by an FMA (Dekker's two-product), the cross terms added to its
// error, then a fast two-sum (|p| >= |t|) into (hi, lo); relative error
// about 2^-44, the precision of the double-float sums themselves.
__device__ __forceinline__ DF df_mul(const DF &a, float2 b) {
    const float p = __fmul_rn(a.hi, b.x);
    const float e = __fmaf_rn(a.hi, b.x, -p);
    const float t = __fmaf_rn(a.hi, b.y, __fmaf_rn(a.lo, b.x, e));
    const float hi = __fadd_rn(p, t);
    return DF{hi, __fsub_rn(t, __fsub_rn(hi, p))};
}
__device__ __forceinline__ double df_double(const DF &a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

__device__ __forceinline__ DF df_shfl_xor(const DF &a, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Fixed-order block sums (blockDim a multiple of 32, at most 1024 threads).
template <int NT>
__device__ __forceinline__ DF block_sum_df(DF v, DF *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) df_add(v, df_shfl_xor(v, o));
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    DF t = sm[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) df_add(t, sm[w]);
    __syncthreads();
    return t;
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double t = sm[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) t += sm[w];
    __syncthreads();
    return t;
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    float t = sm[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) t = fmaxf(t, sm[w]);
    __syncthreads();
    return t;
}

// ------------------------------------------------------------ locations

// Rewrite slot k, coordinate kk of the FP32C split layouts from value v.
__device__ __forceinline__ void write_split_slot(const XState &xs, const Split &sp, int64_t k, int d, int kk,
                                                 float v) {
    const float h = __fsub_rn(__fadd_rn(v, sp.magic), sp.magic);  // nearest multiple of q
    const float l = __fsub_rn(v, h);                               // exact
    float *xr = reinterpret_cast<float *>(xs.xrow + (((k >> 6) * d + kk) * 32 + ((k >> 1) & 31)));
    xr[k & 1] = h;
    xr[2 + (k & 1)] = l;
    xs.xcol[k * d + kk] = make_float4(-h, -h, -l, -l);
    if (xs.xcol2) xs.xcol2[k * d + kk] = make_float2(-h, -l);
}

__device__ __forceinline__ void write_split_slot(const XState &xs, int64_t k, int d, int kk, float v) {
    write_split_slot(xs, *xs.split, k, d, kk, v);
}

// The same for item `item` (at its slot of the tile layouts).
__device__ __forceinline__ void write_split(const XState &xs, int64_t item, int d, int kk, float v) {
    write_split_slot(xs, xs.inv ? xs.inv[item] : item, d, kk, v);
}

// Store a coordinate of the state (and the split layouts on the FP32C path).
template <typename T>
__device__ __forceinline__ void store_x(const XState &xs, int64_t k, int d, int kk, T v) {
    reinterpret_cast<T *>(xs.x)[k * d + kk] = v;
    if constexpr (std::is_same<T, float>::value) write_split(xs, k, d, kk, v);
}

// The same, for item k whose slot is known, with the split quantum in hand.
template <typename T>
__device__ __forceinline__ void store_x_at(const XState &xs, const Split &sp, int64_t k, int64_t slot, int d, int kk,
                                           T v) {
    reinterpret_cast<T *>(xs.x)[k * d + kk] = v;
    if constexpr (std::is_same<T, float>::value) write_split_slot(xs, sp, slot, d, kk, v);
}

// Gradient storage: FP32C keeps (hi, lo) float pairs, FP64 doubles.
template <typename T>
struct GradT;
template <>
struct GradT<float> {
    using type = float2;
    __device__ static float value(const float2 &g) { return __fadd_rn(g.x, g.y); }
};
template <>
struct GradT<double> {
    using type = double;
    __device__ static double value(const double &g) { return g; }
};

// --------------------------------------------------------------- reduce

// One CTA of the reduction: column block J of one problem, or its scalar
// sums when J < 0.  `a` may live in global memory (batched launches).
// The D coordinates of one partial (zeros when !ok): FP32 pairs as one 8-byte
// load (a partial's row starts at a multiple of D floats).
template <typename T, int D>
__device__ __forceinline__ void load_coords(const T *p, bool ok, T (&v)[D]) {
    if constexpr (std::is_same<T, float>::value && D % 2 == 0) {
#pragma unroll
        for (int d = 0; d < D; d += 2) {
            const float2 w = ok ? *reinterpret_cast<const float2 *>(p + d) : make_float2(0.f, 0.f);
            v[d] = w.x;
            v[d + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) v[d] = ok ? p[d] : T(0);
    }
}

template <typename T, int D>
__device__ __forceinline__ void reduce_body(const ReduceArgs &a, int mode, int Jq) {
    constexpr bool kF32 = std::is_same<T, float>::value;
    using Acc = typename std::conditional<kF32, DF, double>::type;
    using G = typename GradT<T>::type;
    __shared__ Acc sm[kSplits * kRedRows > 64 ? kSplits * kRedRows : 64];
    const int tid = threadIdx.x;
    const int nt = a.nt;
    // the item at this thread's slot (the order is constant between passes,
    // so it is read before the wait)
    int64_t item_of_slot = -1;
    int s0 = 0, s1 = 0;  // the column block's row-partial slots (fixed between passes too)
    if (Jq >= 0) {
        const int64_t ks = static_cast<int64_t>(Jq / kRedQuarters) * kTile + (Jq % kRedQuarters) * kRedRows +
                           (tid % kRedRows);
        item_of_slot = (a.perm && ks < a.n) ? a.perm[ks] : ks;
        s0 = a.row_first_slot[Jq / kRedQuarters];
        s1 = a.row_first_slot[Jq / kRedQuarters + 1];
    }
    // the split quantum changes only at a trajectory's end (never in a
    // kick-drift launch): read before the wait, so that writing the split
    // layouts after it costs no dependent L2 load
    Split sp_kd{};
    if constexpr (kF32)
        if (mode == kModeKickDrift) sp_kd = *a.xs.split;
    const float xbound = sp_kd.bound;
    // every input (partials, x, p) comes from the pass just before
    pdl_trigger();
    pdl_wait();
    if (a.stamps && blockIdx.x == 0 && tid == 0) {
        // the pass just before is complete: its span (first warp past the
        // dependency wait to the last warp's end) into the running total, and
        // the stamps reset for the next pass (which waits for this kernel)
        const unsigned long long t0 = a.stamps[0], t1 = a.stamps[1];
        if (t1 > t0) {
            a.pass_ns[0] += static_cast<double>(t1 - t0);
            a.pass_ns[1] += 1.0;
        }
        a.stamps[0] = ~0ull;
        a.stamps[1] = 0ull;
    }

    if (Jq < 0 && a.use_grad) {
        // sharded update: L, sum r and dL/dsigma come from the combine; only
        // the end of a trajectory's quantum growth is left for this CTA
        if constexpr (kF32) {
            if (tid == 0 && mode == kModeHalfKick) {
                Split sp = *a.xs.split;
                const float m = __uint_as_float(*a.xs.xmax_bits);
                int rs = 0;
                if (m > sp.bound) {
                    Split ns;
                    if (choose_split(m, D, ns)) {
                        sp = ns;
                        rs = 1;
                    } else {
                        atomicOr(a.err, kErrRange);
                    }
                }
                sp.resplit = rs;
                *a.xs.split = sp;
            }
        }
        return;
    }
    if (Jq < 0) {
        // scalar partials of all strips -> L, sum r, dL/dsigma (fixed order)
        const T *sp = reinterpret_cast<const T *>(a.scal_part);
        Acc e2{}, md{}, lp{};
        for (int s0 = tid; s0 < a.n_strips; s0 += 4 * kRedThreads) {
            T v[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int s = s0 + u * kRedThreads;
                const T *q = sp + static_cast<int64_t>(s) * kScalarParts;
#pragma unroll
                for (int i = 0; i < 3; ++i) v[u][i] = s < a.n_strips ? q[i] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if constexpr (kF32) {
                    df_add(e2, v[u][kSumE2]);
                    df_add(md, v[u][kSumMDelta]);
                    df_add(lp, v[u][kSumLogPhi]);
                } else {
                    e2 += v[u][kSumE2];
                    md += v[u][kSumMDelta];
                    lp += v[u][kSumLogPhi];
                }
            }
        }
        double de2, dmd, dlp;
        if constexpr (kF32) {
            de2 = df_double(block_sum_df<kRedThreads>(e2, sm));
            dmd = df_double(block_sum_df<kRedThreads>(md, sm));
            dlp = df_double(block_sum_df<kRedThreads>(lp, sm));
        } else {
            de2 = block_sum_d<kRedThreads>(e2, sm);
            dmd = block_sum_d<kRedThreads>(md, sm);
            dlp = block_sum_d<kRedThreads>(lp, sm);
        }
        if (a.tree_part && tid < 32) {
            // the tree prior's log density at this x (its traversal ran
            // beside the pass and completed before this kernel)
            const double lp = tree_parts_sum(a.tree_part, a.n_tree_parts, a.tree_const);
            if (tid == 0) {
                a.scal[kPriorLogp] = lp;
                if (!isfinite(lp)) atomicOr(a.err, kErrNonfinite);
            }
        }
        if (tid == 0) {
            // log sigma and 1 / sigma come from the host: FP64 log and
            // division are long dependency chains on this GPU
            const double isg = a.inv_sigma, isg2 = isg * isg;
            const double m = a.m_pairs;
            const double sum_logphi = kF32 ? -kLn2 * dlp : dlp;      // FP32C: sum log2(1/Phi)
            const double sum_mdelta = kF32 ? dmd / kSqrt2Pi : dmd;   // FP32C: sqrt(2 pi) (phi/Phi) delta
            const double sum_r = 0.5 * de2 * isg2 + sum_logphi;
            const double ll = -m * a.log_sigma - sum_r;
            const double ds = -m * isg + de2 * isg2 * isg + sum_mdelta * isg2;
            a.scal[kLogLik] = ll;
            a.scal[kSumR] = sum_r;
            a.scal[kDSigma] = ds;
            a.scal[kLogLikEnd] = ll;
            if (!isfinite(ll) || !isfinite(ds)) atomicOr(a.err, kErrNonfinite);
            if constexpr (kF32) {
                if (mode == kModeHalfKick) {
                    // end of a trajectory (no CTA of this launch reads the split):
                    // grow the quantum if the running max |x| outgrew it; the
                    // trajectory-end kernel rewrites the layouts
                    Split sp = *a.xs.split;
                    const float m = __uint_as_float(*a.xs.xmax_bits);
                    int rs = 0;
                    if (m > sp.bound) {
                        Split ns;
                        if (choose_split(m, D, ns)) {
                            sp = ns;
                            rs = 1;
                        } else {
                            atomicOr(a.err, kErrRange);
                        }
                    }
                    sp.resplit = rs;
                    *a.xs.split = sp;
                }
            }
        }
        return;
    }

    const int J = Jq / kRedQuarters;
    const int r = (Jq % kRedQuarters) * kRedRows + (tid % kRedRows);  // row within the block
    const int s = tid / kRedRows;
    const int64_t k = static_cast<int64_t>(J) * kTile + r;
    Acc acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = Acc{};
    // the state this CTA's writers update: read now, beside the partials
    // (it does not depend on them), so that it costs no L2 latency of its own
    const bool writer = s == 0 && k < a.n && mode != kModeEval;
    T xv0[D], pv0[D];
    double pg0[D];
    if (writer) {
        const T *xs = reinterpret_cast<const T *>(a.xs.x);
        const T *ps = reinterpret_cast<const T *>(a.p);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            xv0[d] = xs[item_of_slot * D + d];
            pv0[d] = ps[item_of_slot * D + d];
            pg0[d] = a.prior_grad ? a.prior_grad[item_of_slot * D + d] : 0.0;
        }
    }
    // column partials (I <= J) added, row partials (slots [s0, s1))
    // subtracted; the loads of a round, of both kinds, are issued together
    // (independent of the running sums), so one round costs one L2 latency;
    // at N = 5392 one round covers every partial of the block
    constexpr int kU = D <= 2 ? 8 : D <= 4 ? 4 : 2;
    const T *cp = reinterpret_cast<const T *>(a.col_part);
    const T *rpart = reinterpret_cast<const T *>(a.row_part);
    for (int q = 0; !a.use_grad && (s + q <= J || s0 + s + q < s1); q += kSplits * kU) {
        T vc[kU][D], vr[kU][D];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int I = s + q + u * kSplits;
            const int slot = s0 + s + q + u * kSplits;
            const T *c = cp + (col_slot(I, J) * kTile + r) * D;
            const T *rp = rpart + (static_cast<int64_t>(slot) * kTile + r) * D;
            load_coords<T, D>(c, I <= J, vc[u]);
            load_coords<T, D>(rp, slot < s1, vr[u]);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
            for (int d = 0; d < D; ++d) {
                if constexpr (kF32) {
                    df_add(acc[d], vc[u][d]);
                    df_add(acc[d], -vr[u][d]);
                } else {
                    acc[d] += vc[u][d];
                    acc[d] -= vr[u][d];
                }
            }
    }
    // the kSplits partial sums of every (row, coordinate), in a fixed order:
    // the two splits of a warp (lanes r and r + 16) by a shuffle, then the
    // warps' sums through shared memory, all coordinates at once
    constexpr int kRedWarps = kRedThreads / 32;
    __shared__ Acc smw[kRedWarps * kRedRows * D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        if constexpr (kF32)
            df_add(acc[d], df_shfl_xor(acc[d], 16));
        else
            acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], 16);
    }
    if ((tid & 31) < kRedRows) {
#pragma unroll
        for (int d = 0; d < D; ++d) smw[((tid >> 5) * kRedRows + (tid & 31)) * D + d] = acc[d];
    }
    __syncthreads();
    Acc gsum[D];
    if (s == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            Acc g = smw[tid * D + d];
#pragma unroll
            for (int w = 1; w < kRedWarps; ++w) {
                if constexpr (kF32)
                    df_add(g, smw[(w * kRedRows + tid) * D + d]);
                else
                    g += smw[(w * kRedRows + tid) * D + d];
            }
            gsum[d] = g;
        }
    }

    Acc ke{}, xx{};
    if (s == 0 && k < a.n) {
        // slot k of the tile layouts holds item `it` of the state
        const int64_t it = item_of_slot;
        T *p = reinterpret_cast<T *>(a.p);
        G *grad = reinterpret_cast<G *>(a.grad);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const Acc g = gsum[d];
            T gv;
            if (a.use_grad) {
                // the combined gradient of all shards, as the combine stored it
                if constexpr (kF32)
                    gv = GradT<T>::value(grad[it * D + d]);
                else
                    gv = grad[it * D + d];
            } else if constexpr (kF32) {
                if (a.part_scale == 1.0) {
                    grad[it * D + d] = make_float2(g.hi, g.lo);
                    gv = df_float(g);
                } else {
                    // partial sums in other units (the chunked pass sums the
                    // gradient weight times -sigma^2): scaled as a
                    // double-float product (FP64 latency is long here)
                    const DF v = df_mul(g, a.part_scale_df);
                    grad[it * D + d] = make_float2(v.hi, v.lo);
                    gv = v.hi;
                }
            } else {
                grad[it * D + d] = g;
                gv = g;
            }
            bad |= !isfinite(gv);
            if (mode != kModeEval) {
                const T xv = xv0[d];
                T tg = gv - static_cast<T>(a.lambda) * xv;  // gradient of log pi
                if (a.prior_grad) tg += static_cast<T>(pg0[d]);
                if (mode == kModeKickDrift) {
                    const T pn = pv0[d] + static_cast<T>(a.eps) * tg;
                    const T xn = xv + static_cast<T>(a.eps) * pn;
                    p[it * D + d] = pn;
                    store_x_at<T>(a.xs, sp_kd, it, k, D, d, xn);
                    // the running max |x| only matters once it passes the
                    // split's bound (the end-of-trajectory reduction then
                    // grows the quantum), so only such values are recorded
                    if constexpr (kF32)
                        if (fabsf(xn) > xbound) atomicMax(a.xs.xmax_bits, __float_as_uint(fabsf(xn)));
                } else {  // kModeHalfKick
                    const T pn = pv0[d] + static_cast<T>(0.5 * a.eps) * tg;
                    p[it * D + d] = pn;
                    if constexpr (kF32) {
                        df_add(ke, 0.5f * pn * pn);
                        df_add(xx, xv * xv);
                    } else {
                        ke += 0.5 * pn * pn;
                        xx += xv * xv;
                    }
                }
            }
        }
        if (bad) atomicOr(a.err, kErrNonfinite);
    }
    if (mode == kModeHalfKick) {
        __syncthreads();
        if constexpr (kF32) {
            const DF tk = block_sum_df<kRedThreads>(ke, sm);
            const DF tx = block_sum_df<kRedThreads>(xx, sm);
            if (tid == 0) {
                a.energy_part[2 * Jq] = df_double(tk);
                a.energy_part[2 * Jq + 1] = df_double(tx);
            }
        } else {
            const double tk = block_sum_d<kRedThreads>(ke, sm);
            const double tx = block_sum_d<kRedThreads>(xx, sm);
            if (tid == 0) {
                a.energy_part[2 * Jq] = tk;
                a.energy_part[2 * Jq + 1] = tx;
            }
        }
    }
}

// CTA b reduces quarter-block last - 1 - b: the blocks with the most
// partials (the last column blocks gather one per row block) start first,
// which measured faster than the natural order (0.524 against 0.528 ms per
// HMC iteration at N = 5392).  The scalar CTA is the last one.
template <typename T, int D>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const __grid_constant__ ReduceArgs a) {
    const int last = a.nt * kRedQuarters;
    const int b = static_cast<int>(blockIdx.x);
    reduce_body<T, D>(a, a.mode, b == last ? -1 : last - 1 - b);
}

// Batched: job (problem index, quarter-block index J * kReduceQuarters + q,
// or -1 for the scalars) per CTA.
template <int D>
__global__ void __launch_bounds__(kRedThreads) reduce_batch_kernel(const ReduceArgs *cfg, const int2 *jobs, int mode) {
    const int2 job = jobs[blockIdx.x];
    reduce_body<float, D>(cfg[job.x], mode, job.y);
}

// ----------------------------------------------------------- traj start

constexpr int kTrajThreads = 128;

template <typename T, int D>
__device__ __forceinline__ void traj_start_body(const TrajArgs &a, int bx) {
    constexpr bool kF32 = std::is_same<T, float>::value;
    using Acc = typename std::conditional<kF32, DF, double>::type;
    using G = typename GradT<T>::type;
    __shared__ Acc sm[kTrajThreads / 32];
    // the first pass of the trajectory may become resident and stage its
    // first Y tiles meanwhile (it waits for this kernel before reading x)
    pdl_trigger();
    const int64_t nd = a.n * D;
    const int64_t q = static_cast<int64_t>(bx) * kTrajThreads + threadIdx.x;  // 4 elements each
    T *x = reinterpret_cast<T *>(a.xs.x);
    T *p = reinterpret_cast<T *>(a.p);
    T *x0 = reinterpret_cast<T *>(a.x0);
    G *grad = reinterpret_cast<G *>(a.grad);
    G *grad0 = reinterpret_cast<G *>(a.grad0);
    const int64_t iter = a.counters[kIter];
    const int64_t iter_local = a.counters[kIterLocal];
    Acc ke{}, xx{};
    T z[4] = {T(0), T(0), T(0), T(0)};
    if (a.momentum_src == 1 && 4 * q < nd) {
        uint32_t c[4] = {static_cast<uint32_t>(q), static_cast<uint32_t>(iter), a.chain, 0u};
        philox10(c, a.seed);
        box_muller(c[0], c[1], z[0], z[1]);
        box_muller(c[2], c[3], z[2], z[3]);
    }
    float xmax = 0.f;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int64_t e = 4 * q + h;
        if (e >= nd) break;
        T pv;
        if (a.momentum_src == 1)
            pv = z[h];
        else if (a.momentum_src == 2)
            pv = static_cast<T>(a.p_inj[iter_local * nd + e]);
        else
            pv = p[e];
        const T xv = x[e];
        x0[e] = xv;
        grad0[e] = grad[e];
        double pg = 0.0;
        if (a.prior_grad) {
            pg = a.prior_grad[e];
            a.prior_grad0[e] = pg;
        }
        if constexpr (kF32) {
            df_add(ke, 0.5f * pv * pv);
            df_add(xx, xv * xv);
        } else {
            ke += 0.5 * pv * pv;
            xx += xv * xv;
        }
        if (a.drift) {
            const T tg = GradT<T>::value(grad[e]) - static_cast<T>(a.lambda) * xv + static_cast<T>(pg);
            pv = pv + static_cast<T>(0.5 * a.eps) * tg;
            const T xn = xv + static_cast<T>(a.eps) * pv;
            store_x<T>(a.xs, e / D, D, static_cast<int>(e % D), xn);
            xmax = fmaxf(xmax, fabsf(static_cast<float>(xn)));
        }
        p[e] = pv;
    }
    double tk, tx;
    if constexpr (kF32) {
        tk = df_double(block_sum_df<kTrajThreads>(ke, sm));
        tx = df_double(block_sum_df<kTrajThreads>(xx, sm));
        if (a.drift) {
            const float m = block_max<kTrajThreads>(xmax, reinterpret_cast<float *>(sm));
            if (threadIdx.x == 0 && m > 0.f) atomicMax(a.xs.xmax_bits, __float_as_uint(m));
        }
    } else {
        tk = block_sum_d<kTrajThreads>(ke, sm);
        tx = block_sum_d<kTrajThreads>(xx, sm);
    }
    if (threadIdx.x == 0) {
        a.energy_part[2 * bx] = tk;
        a.energy_part[2 * bx + 1] = tx;
        if (bx == 0) {
            a.scal[kLogLik0] = a.scal[kLogLik];
            a.scal[kSumR0] = a.scal[kSumR];
            a.scal[kDSigma0] = a.scal[kDSigma];
            a.scal[kPriorLogp0] = a.scal[kPriorLogp];
            a.counters[kIterCur] = iter;
            a.counters[kIterLocalCur] = iter_local;
        }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kTrajThreads) traj_start_kernel(const __grid_constant__ TrajArgs a) {
    traj_start_body<T, D>(a, blockIdx.x);
}

// Batched: chain blockIdx.y; CTAs past that chain's own grid leave at once.
template <int D>
__global__ void __launch_bounds__(kTrajThreads) traj_start_batch_kernel(const TrajArgs *cfg) {
    const TrajArgs &a = cfg[blockIdx.y];
    const int64_t quads = (a.n * D + 3) / 4;
    if (static_cast<int64_t>(blockIdx.x) * kTrajThreads >= quads) return;
    traj_start_body<float, D>(a, blockIdx.x);
}

// ------------------------------------------------------------- traj end

template <typename T, int D>
__device__ __forceinline__ void traj_end_body(const AcceptArgs &a, int bx, int nbx) {
    using G = typename GradT<T>::type;
    // every CTA sums the same partials in the same order -> same decision
    __shared__ int keep_s;
    __shared__ double dh_s;
    // launched with PDL after the trajectory's last reduction: every input
    // comes from it or from kernels before it
    pdl_wait();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double ke0 = 0.0, xx0 = 0.0, ke1 = 0.0, xx1 = 0.0;
        for (int i = lane; i < a.n_start_parts; i += 32) {
            ke0 += a.start_part[2 * i];
            xx0 += a.start_part[2 * i + 1];
        }
        for (int i = lane; i < a.n_end_parts; i += 32) {
            ke1 += a.end_part[2 * i];
            xx1 += a.end_part[2 * i + 1];
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ke0 += __shfl_xor_sync(0xffffffffu, ke0, o);
            xx0 += __shfl_xor_sync(0xffffffffu, xx0, o);
            ke1 += __shfl_xor_sync(0xffffffffu, ke1, o);
            xx1 += __shfl_xor_sync(0xffffffffu, xx1, o);
        }
        if (lane == 0) {
            const double h0 = -(a.scal[kLogLik0] - 0.5 * a.lambda * xx0 + a.scal[kPriorLogp0]) + ke0;
            const double h1 = -(a.scal[kLogLikEnd] - 0.5 * a.lambda * xx1 + a.scal[kPriorLogp]) + ke1;
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
    }
    __syncthreads();
    const int keep = keep_s;
    const int64_t nd = a.n * D;
    bool resplit = false;  // FP32C: the last reduction chose a new quantum
    if constexpr (std::is_same<T, float>::value) resplit = a.xs.split->resplit != 0;
    if (!keep) {
        const T *x0 = reinterpret_cast<const T *>(a.x0);
        G *grad = reinterpret_cast<G *>(a.grad);
        const G *grad0 = reinterpret_cast<const G *>(a.grad0);
        for (int64_t e = static_cast<int64_t>(bx) * kTrajThreads + threadIdx.x; e < nd;
             e += static_cast<int64_t>(nbx) * kTrajThreads) {
            store_x<T>(a.xs, e / D, D, static_cast<int>(e % D), x0[e]);
            grad[e] = grad0[e];
            if (a.prior_grad) a.prior_grad[e] = a.prior_grad0[e];
        }
    } else if (resplit) {
        const T *x = reinterpret_cast<const T *>(a.xs.x);
        for (int64_t e = static_cast<int64_t>(bx) * kTrajThreads + threadIdx.x; e < nd;
             e += static_cast<int64_t>(nbx) * kTrajThreads)
            store_x<T>(a.xs, e / D, D, static_cast<int>(e % D), x[e]);
    }
    if (bx == 0 && threadIdx.x == 0) {
        const double dh = dh_s;
        if (!isfinite(dh)) atomicOr(a.err, kErrNonfinite);
        a.scal[kLastDH] = dh;
        if (!keep) {
            a.scal[kLogLik] = a.scal[kLogLik0];
            a.scal[kSumR] = a.scal[kSumR0];
            a.scal[kDSigma] = a.scal[kDSigma0];
            a.scal[kPriorLogp] = a.scal[kPriorLogp0];
        }
        const int64_t il = a.counters[kIterLocalCur];
        if (il >= 0 && il < a.out_cap) {
            if (a.acc_out) a.acc_out[il] = keep;
            if (a.dh_out) a.dh_out[il] = dh;
        } else if (a.acc_out || a.dh_out) {
            atomicOr(a.err, kErrOverflow);
        }
        if (a.metropolis) {
            a.counters[kIter] = a.counters[kIterCur] + 1;
            a.counters[kIterLocal] = il + 1;
            a.counters[kAccepted] += keep;
        }
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kTrajThreads) traj_end_kernel(const __grid_constant__ AcceptArgs a) {
    traj_end_body<T, D>(a, blockIdx.x, gridDim.x);
}

template <int D>
__global__ void __launch_bounds__(kTrajThreads) traj_end_batch_kernel(const AcceptArgs *cfg) {
    traj_end_body<float, D>(cfg[blockIdx.y], blockIdx.x, gridDim.x);
}

// Draws of the sigma update (section 3's sigma^2 step, a random walk on
// log sigma): update t uses the Philox4x32-10 block at counter
// (0, t, chain, 2): z from words 0 and 1 (Box-Muller), the uniform from word 2.
__global__ void sigma_draws_kernel(uint64_t seed, uint32_t chain, int64_t iter0, int n, double *z, double *u) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t c[4] = {0u, static_cast<uint32_t>(iter0 + t), chain, 2u};
    philox10(c, seed);
    double z0, z1;
    box_muller(c[0], c[1], z0, z1);
    z[t] = z0;
    u[t] = open_unit(c[2]);
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

#define MDS_SWITCH_D_PDL(KERNEL, T, GRID, BLOCK, STREAM, ARGS)                               \
    switch ((ARGS).d) {                                                                     \
        case 1: e = launch_pdl(KERNEL<T, 1>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 2: e = launch_pdl(KERNEL<T, 2>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 3: e = launch_pdl(KERNEL<T, 3>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 4: e = launch_pdl(KERNEL<T, 4>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 5: e = launch_pdl(KERNEL<T, 5>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 6: e = launch_pdl(KERNEL<T, 6>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 7: e = launch_pdl(KERNEL<T, 7>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        case 8: e = launch_pdl(KERNEL<T, 8>, dim3(GRID), dim3(BLOCK), 0, STREAM, ARGS); break; \
        default: return cudaErrorInvalidValue;                                              \
    }

// ------------------------------------------------------------- shards

// This shard's partials: {L, dL/dsigma, sum r, gradient} (FP64).
__global__ void shard_pack_kernel(const double *scal, const void *grad, bool fp64, int64_t nd, double *send) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        send[0] = scal[kLogLik];
        send[1] = scal[kDSigma];
        send[2] = scal[kSumR];
    }
    for (int64_t i = i0; i < nd; i += stride) {
        double v;
        if (fp64) {
            v = reinterpret_cast<const double *>(grad)[i];
        } else {
            const float2 g = reinterpret_cast<const float2 *>(grad)[i];
            v = static_cast<double>(g.x) + static_cast<double>(g.y);
        }
        send[3 + i] = v;
    }
}

// Sum of all ranks' partials in rank order (rank 0 first), FP64, into the
// scalars and the gradient; the same order on every rank, so every rank
// holds bitwise the same combined values.
__global__ void shard_combine_kernel(const double *recv, int n_ranks, int64_t count, double *scal, void *grad,
                                     bool fp64) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        double v = recv[i];
        for (int r = 1; r < n_ranks; ++r) v += recv[static_cast<int64_t>(r) * count + i];
        if (i == 0) {
            scal[kLogLik] = v;
            scal[kLogLikEnd] = v;
        } else if (i == 1) {
            scal[kDSigma] = v;
        } else if (i == 2) {
            scal[kSumR] = v;
        } else if (fp64) {
            reinterpret_cast<double *>(grad)[i - 3] = v;
        } else {
            const float hi = static_cast<float>(v);
            reinterpret_cast<float2 *>(grad)[i - 3] = make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
        }
    }
}

// ----------------------------------------------------------------- ingest

// Inverse of tile_offset(): (row, column) inside a tile of element `off`.
__device__ __forceinline__ void tile_rc(int off, int &r, int &c) {
    const int e = off & 3, slot = (off >> 2) & 31, wt = off >> 7;
    const int t = wt & 7, w = wt >> 3;
    const int q = t >> 1, half = t & 1, a = (slot & 7) ^ (half << 2), b = slot >> 3;
    r = 2 * (a + 8 * q) + (e & 1);
    c = 16 * w + 4 * b + 2 * half + (e >> 1);
}

// One thread per destination element of the tiles of row blocks covering
// rows [r0, r1).
__global__ void ingest_kernel(const __grid_constant__ IngestArgs a) {
    const int64_t nt = a.nt;
    const int64_t b0 = a.r0 / kTile;
    const int64_t b1 = (a.r1 + kTile - 1) / kTile;
    const int64_t t_begin = max(tile_index(b0, b0, nt), a.t_lo);
    const int64_t t_end = min(tile_index(b1 - 1, nt - 1, nt) + 1, a.t_hi);
    if (t_end <= t_begin) return;
    const int64_t total = (t_end - t_begin) * kTileElems;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t t = t_begin + g / kTileElems;
        const int off = static_cast<int>(g % kTileElems);
        // row block I is the largest with tile_index(I, I) <= t
        int64_t lo = b0, hi = b1 - 1;
        if (t < tile_index(b0, b0, nt)) continue;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (tile_index(mid, mid, nt) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t I = lo;
        const int64_t J = I + (t - tile_index(I, I, nt));
        int rr, cc;
        tile_rc(off, rr, cc);
        const int64_t i = I * kTile + rr;
        const int64_t j = J * kTile + cc;
        const bool in_rows = i >= a.r0 && i < a.r1;
        float v = 0.0f;
        if (i < j && j < a.n && in_rows) {
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
        if (in_rows || i >= a.n) a.y[(t - a.t_lo) * kTileElems + off] = v;  // rows past N: padding
    }
}

// One thread per element of the new layout; the old element is found by
// the old slots of the two items (upper triangle: the smaller slot is the row).
__global__ void repack_kernel(const float *old_y, float *new_y, const int32_t *map, int64_t n, int32_t nt_) {
    const int64_t nt = nt_;
    const int64_t total = tile_count(nt) * kTileElems;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t t = g / kTileElems;
        const int off = static_cast<int>(g % kTileElems);
        int64_t lo = 0, hi = nt - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (tile_index(mid, mid, nt) <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int64_t I = lo;
        const int64_t J = I + (t - tile_index(I, I, nt));
        int rr, cc;
        tile_rc(off, rr, cc);
        const int64_t sr = I * kTile + rr, sc = J * kTile + cc;
        float v = 0.0f;
        if (sr < sc && sc < n) {
            int64_t a = map[sr], b = map[sc];
            if (a > b) {
                const int64_t tmp = a;
                a = b;
                b = tmp;
            }
            const int64_t I2 = a / kTile, J2 = b / kTile;
            v = old_y[tile_index(I2, J2, nt) * kTileElems +
                      tile_offset(static_cast<int>(a - I2 * kTile), static_cast<int>(b - J2 * kTile))];
        }
        new_y[g] = v;
    }
}

// --------------------------------------------------------------- set x

// Locations from the caller.  FP32C: the split quantum follows from max |x|
// of the incoming values (xmax_kernel ran just before on the same stream);
// every thread derives the same quantum by the host/device rule
// (choose_split) and CTA 0 stores it.  Outside the FP32C range nothing is
// written and the range bit is raised, so the previous state stays intact.
template <typename T, typename S>
__global__ void set_x_kernel(const S *src, int64_t n, int64_t n_pad, int d, XState xs, unsigned *err) {
    Split sp{};
    if constexpr (std::is_same<T, float>::value) {
        if (!choose_split(__uint_as_float(*xs.xmax_bits), d, sp)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrRange);
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *xs.split = sp;
    }
    const int64_t total = n_pad * d;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t k = e / d;
        const int kk = static_cast<int>(e % d);
        T v = T(0);
        if (k < n) {
            const double sv = static_cast<double>(src[e]);
            if (!isfinite(sv)) atomicOr(err, kErrBadInput);
            v = static_cast<T>(sv);
        }
        if constexpr (std::is_same<T, float>::value)
            store_x_at<T>(xs, sp, k, xs.inv ? xs.inv[k] : k, d, kk, v);
        else
            store_x<T>(xs, k, d, kk, v);
    }
}

__global__ void resplit_kernel(XState xs, int64_t total, int d) {
    const float *x = reinterpret_cast<const float *>(xs.x);
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        write_split(xs, e / d, d, static_cast<int>(e % d), x[e]);
}

template <typename T>
__global__ void xmax_kernel(const T *x, int64_t count, unsigned *out) {
    __shared__ float sm[8];
    float m = 0.f;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = fmaxf(m, fabsf(static_cast<float>(x[e])));
    m = block_max<256>(m, sm);
    if (threadIdx.x == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// src kind: 0 f32, 1 f64, 2 float2 (hi, lo) pairs
template <typename T>
__global__ void convert_kernel(const void *src, int kind, T *dst, int64_t count) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (kind == 0)
            dst[e] = static_cast<T>(reinterpret_cast<const float *>(src)[e]);
        else if (kind == 1)
            dst[e] = static_cast<T>(reinterpret_cast<const double *>(src)[e]);
        else {
            const float2 g = reinterpret_cast<const float2 *>(src)[e];
            dst[e] = static_cast<T>(static_cast<double>(g.x) + static_cast<double>(g.y));
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t s) {
    // kRedQuarters CTAs per column block + one for the scalars (L, sum r,
    // dL/dsigma), which a kick-drift step inside a trajectory does not use:
    // there it is left out
    const dim3 grid(a.nt * kRedQuarters + (a.mode == kModeKickDrift ? 0 : 1));
    cudaError_t e = cudaSuccess;
    if (a.fp64) {
        MDS_SWITCH_D_PDL(reduce_kernel, double, grid, kRedThreads, s, a)
    } else {
        MDS_SWITCH_D_PDL(reduce_kernel, float, grid, kRedThreads, s, a)
    }
    return e != cudaSuccess ? e : cudaGetLastError();
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
    cudaError_t e = cudaSuccess;
    if (a.fp64) {
        MDS_SWITCH_D_PDL(traj_end_kernel, double, grid, kTrajThreads, s, a)
    } else {
        MDS_SWITCH_D_PDL(traj_end_kernel, float, grid, kTrajThreads, s, a)
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

#define MDS_SWITCH_DB(KERNEL, GRID, BLOCK, STREAM, D, ...)                       \
    switch (D) {                                                                 \
        case 1: KERNEL<1><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 2: KERNEL<2><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 3: KERNEL<3><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 4: KERNEL<4><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 5: KERNEL<5><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 6: KERNEL<6><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 7: KERNEL<7><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        case 8: KERNEL<8><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;       \
        default: return cudaErrorInvalidValue;                                   \
    }

cudaError_t launch_reduce_batch(const ReduceArgs *cfg, const int2 *jobs, int n_jobs, int d, int mode, cudaStream_t s) {
    if (n_jobs <= 0) return cudaSuccess;
    // under PDL after the batched pass (reduce_body waits for it)
    cudaError_t e = cudaSuccess;
    switch (d) {
#define MDS_RB_CASE(DD) \
    case DD: e = launch_pdl(reduce_batch_kernel<DD>, dim3(n_jobs), dim3(kRedThreads), 0, s, cfg, jobs, mode); break;
        MDS_RB_CASE(1) MDS_RB_CASE(2) MDS_RB_CASE(3) MDS_RB_CASE(4)
        MDS_RB_CASE(5) MDS_RB_CASE(6) MDS_RB_CASE(7) MDS_RB_CASE(8)
#undef MDS_RB_CASE
        default: return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

int traj_start_grid(int64_t n, int d) { return static_cast<int>(((n * d + 3) / 4 + kTrajThreads - 1) / kTrajThreads); }

cudaError_t launch_traj_start_batch(const TrajArgs *cfg, int n_chains, int max_grid, int d, cudaStream_t s) {
    const dim3 grid(max_grid, n_chains);
    MDS_SWITCH_DB(traj_start_batch_kernel, grid, kTrajThreads, s, d, cfg)
    return cudaGetLastError();
}

cudaError_t launch_sigma_draws(uint64_t seed, uint32_t chain, int64_t iter0, int n, double *z, double *u,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    sigma_draws_kernel<<<(n + 127) / 128, 128, 0, s>>>(seed, chain, iter0, n, z, u);
    return cudaGetLastError();
}

cudaError_t launch_traj_end_batch(const AcceptArgs *cfg, int n_chains, int64_t max_nd, int d, cudaStream_t s) {
    const dim3 grid(grid_for(max_nd, kTrajThreads), n_chains);
    MDS_SWITCH_DB(traj_end_batch_kernel, grid, kTrajThreads, s, d, cfg)
    return cudaGetLastError();
}

cudaError_t launch_shard_pack(const double *scal, const void *grad, bool fp64, int64_t nd, double *send,
                              cudaStream_t s) {
    shard_pack_kernel<<<grid_for(nd, 256), 256, 0, s>>>(scal, grad, fp64, nd, send);
    return cudaGetLastError();
}

cudaError_t launch_shard_combine(const double *recv, int n_ranks, int64_t count, double *scal, void *grad, bool fp64,
                                 cudaStream_t s) {
    shard_combine_kernel<<<grid_for(count, 256), 256, 0, s>>>(recv, n_ranks, count, scal, grad, fp64);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestArgs &a, cudaStream_t s) {
    const int64_t b0 = a.r0 / kTile, b1 = (a.r1 + kTile - 1) / kTile;
    const int64_t tiles = tile_index(b1 - 1, a.nt - 1, a.nt) + 1 - tile_index(b0, b0, a.nt);
    ingest_kernel<<<grid_for(tiles * kTileElems, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_x(const void *src, bool src_f64, int64_t n, int64_t n_pad, int d, bool fp64, const XState &xs,
                         unsigned *err, cudaStream_t s) {
    const int g = grid_for(n_pad * d, 256);
    if (fp64) {
        if (src_f64)
            set_x_kernel<double, double><<<g, 256, 0, s>>>(static_cast<const double *>(src), n, n_pad, d, xs, err);
        else
            set_x_kernel<double, float><<<g, 256, 0, s>>>(static_cast<const float *>(src), n, n_pad, d, xs, err);
    } else {
        if (src_f64)
            set_x_kernel<float, double><<<g, 256, 0, s>>>(static_cast<const double *>(src), n, n_pad, d, xs, err);
        else
            set_x_kernel<float, float><<<g, 256, 0, s>>>(static_cast<const float *>(src), n, n_pad, d, xs, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_repack(const float *old_y, float *new_y, const int32_t *map, int64_t n, int32_t nt, cudaStream_t s) {
    repack_kernel<<<grid_for(tile_count(nt) * kTileElems, 256), 256, 0, s>>>(old_y, new_y, map, n, nt);
    return cudaGetLastError();
}

cudaError_t launch_resplit(const XState &xs, int64_t n_pad, int d, cudaStream_t s) {
    resplit_kernel<<<grid_for(n_pad * d, 256), 256, 0, s>>>(xs, n_pad * d, d);
    return cudaGetLastError();
}

cudaError_t launch_xmax(const void *x, bool fp64, int64_t count, unsigned *out, cudaStream_t s) {
    const int g = grid_for(count, 256);
    if (fp64)
        xmax_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(x), count, out);
    else
        xmax_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(x), count, out);
    return cudaGetLastError();
}

// src_f64: false -> f32, true -> f64; a float2 (hi, lo) source is passed
// with src_f64 = false and count < 0 (|count| elements).
cudaError_t launch_convert(const void *src, bool src_f64, void *dst, bool dst_f64, int64_t count, cudaStream_t s) {
    int kind = src_f64 ? 1 : 0;
    if (count < 0) {
        kind = 2;
        count = -count;
    }
    const int g = grid_for(count, 256);
    if (dst_f64)
        convert_kernel<double><<<g, 256, 0, s>>>(src, kind, static_cast<double *>(dst), count);
    else
        convert_kernel<float><<<g, 256, 0, s>>>(src, kind, static_cast<float *>(dst), count);
    return cudaGetLastError();
}

}  // namespace mds
