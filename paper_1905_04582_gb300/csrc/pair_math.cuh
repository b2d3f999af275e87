// Per-pair arithmetic and warp-level reductions of the FP32C pair pass,
// shared by the single-problem kernel (pair_kernel.cu) and the batched
// multi-dataset / multi-chain kernel (batch_kernel.cu).  See pair_kernel.cu
// for the method (Eq. (2) and (9) of arXiv:1905.04582).
#pragma once

#include <cfloat>
#include <cstdint>

#include "mds_internal.h"

namespace mds {
namespace {

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bulk (1-D TMA) copy global -> shared, completion counted on an mbarrier.
// Addresses 16-byte aligned and sizes multiples of 16 (guaranteed by the
// layouts: 4096 B quarters of 16 KB tiles, 256 D B column blocks).
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :
        : "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" : : "r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory"); }

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" : : : "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// Wait for an mbarrier phase, giving up after the time limit (sets the error
// word).  Every lane of the warp calls it; the result is warp-uniform.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, unsigned *err) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (global_ns() - t0 > kWaitLimitNs) {
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
    return true;
}

// ------------------------------------------------------ packed FP32 helpers

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Kahan-compensated accumulation of v into (s, c): the sum is s - c.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <int V>
struct Pow2 {
    static constexpr int value = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : V <= 16 ? 16 : V <= 32 ? 32 : 64;
};

// Sum the values v[0..P) over the lanes that differ in the bits of `mask`
// (processed from the highest bit down) by recursive halving: at each level
// a lane keeps one half of its values and receives the partner's copy of
// that half.  After all levels a lane holds in v[0..P >> L) the totals of
// the value indices starting at reduced_base<P>(lane bits), L = number of
// halving levels (levels beyond log2 P degrade to plain butterflies).
template <int CNT, int LV, int P, typename T>
__device__ __forceinline__ void lane_reduce_rec(T (&v)[P], int lane, int first_bit) {
    if constexpr (LV >= 0) {
        const int o = 1 << (first_bit + LV);
        if constexpr (CNT > 1) {
            constexpr int half = CNT / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const T send = upper ? v[i] : v[i + half];
                const T keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            lane_reduce_rec<half, LV - 1>(v, lane, first_bit);
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
            lane_reduce_rec<1, LV - 1>(v, lane, first_bit);
        }
    }
}

template <int P, int NBITS, typename T>
__device__ __forceinline__ void lane_reduce(T (&v)[P], int lane, int first_bit) {
    lane_reduce_rec<P, NBITS - 1>(v, lane, first_bit);
}

// First value index held after lane_reduce<P, NBITS> over bits
// [first_bit, first_bit + NBITS), and whether this lane is the one that
// writes it (lanes that only hold duplicates do not).
template <int P, int NBITS>
__device__ __forceinline__ int reduced_base(int lane, int first_bit, bool &writer) {
    int base = 0, cnt = P;
    writer = true;
#pragma unroll
    for (int lv = NBITS - 1; lv >= 0; --lv) {
        const int o = 1 << (first_bit + lv);
        if (cnt > 1) {
            cnt /= 2;
            if (lane & o) base += cnt;
        } else if (lane & o) {
            writer = false;
        }
    }
    return base;
}

// One row pair (rows r, r+1 packed) against one column: the whole per-pair
// body of Eq. (2) and Eq. (9) for two pairs at once.
template <int D, bool MASKED, typename K>
__device__ __forceinline__ void pair2_f32(const K &a, const float4 (&xi)[D], const float4 (&xj)[D], float2 y2,
                                          float2 vmask, float2 (&racc)[D], float2 (&cacc)[D], float2 &e2,
                                          float2 &md, float2 &prod) {
    float2 s[D];
    float2 d2h, cr;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float2 dh = add2(f2(xi[k].x, xi[k].y), f2(xj[k].x, xj[k].y));  // exact
        const float2 dl = add2(f2(xi[k].z, xi[k].w), f2(xj[k].z, xj[k].w));
        s[k] = add2(dh, dl);  // x_i - x_j, rounded once
        if (k == 0) {
            d2h = mul2(dh, dh);
            cr = fma2(dl, add2(s[k], dh), f2(FLT_MIN, FLT_MIN));
        } else {
            d2h = fma2(dh, dh, d2h);                  // exact: sum of Dh^2 needs <= 24 bits
            cr = fma2(dl, add2(s[k], dh), cr);         // Dl (2 Dh + Dl)
        }
    }
    // d^2 = d2h + cr (+FLT_MIN keeps rsqrt finite for coincident points, whose
    // delta is then ~1e-19 and whose gradient term is exactly 0)
    const float2 d2 = add2(d2h, cr);
    const float2 inv = f2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
    const float2 del = f2(sqrt_approx(d2.x), sqrt_approx(d2.y));  // MUFU, frees an FMA-pipe slot
    // residual of the square root: true d^2 - del^2 = (d2h - del^2) + cr;
    // delta_true = del + res / (2 del) to first order
    const float2 res = add2(fma2(neg2(del), del, d2h), cr);
    const float2 hinv = mul2(inv, f2(0.5f, 0.5f));
    float2 e = fma2(neg2(res), hinv, add2(y2, neg2(del)));        // y - delta, corrected
    // Phi via the Mills ratio: phi' = exp(-z^2/2), -P/sqrt(2 pi) and D in delta
    const float2 ea = mul2(d2, a.c_phi);
    const float2 ph = f2(ex2_approx(ea.x), ex2_approx(ea.y));
    float2 pn = fma2(a.mp[3], del, a.mp[2]);
    pn = fma2(pn, del, a.mp[1]);
    pn = fma2(pn, del, a.mp[0]);
    float2 dd = fma2(a.md[3], del, a.md[2]);
    dd = fma2(dd, del, a.md[1]);
    dd = fma2(dd, del, a.md[0]);
    const float2 den = fma2(ph, pn, dd);  // D Phi
    const float2 rden = f2(rcp_approx(den.x), rcp_approx(den.y));
    float2 ip = mul2(dd, rden);  // 1 / Phi
    float2 mm = mul2(ph, ip);    // sqrt(2 pi) phi / Phi
    if (MASKED) {
        e = mul2(e, vmask);
        mm = mul2(mm, vmask);
        ip = f2(vmask.x != 0.f ? ip.x : 1.f, vmask.y != 0.f ? ip.y : 1.f);
    }
    prod = mul2(prod, ip);
    e2 = fma2(e, e, e2);
    md = fma2(mm, del, md);
    // w = (delta - y)/sigma^2 + phi/(sigma Phi); wi = w / delta
    const float2 wi = mul2(fma2(e, a.neg_inv_s2, mul2(mm, a.m_coef)), inv);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        racc[k] = fma2(wi, s[k], racc[k]);
        cacc[k] = fma2(wi, s[k], cacc[k]);
    }
}

// The same two pairs where every pair of the warp's block lies at
// z = delta / sigma >= z_c (z_c = 8 by default): the Phi terms are dropped.
// For z >= 8, log(1/Phi(z)) <= 1.0000001 Q(z) < 6.3e-16 and
// phi(z)/Phi(z) < 5.1e-15, far below the FP32 rounding (2^-24 = 6e-8,
// relative) of the kept terms e^2/(2 sigma^2) and (delta - y)/sigma^2, so
// the result is the same to FP32 precision.  Geometry, residual-corrected e
// and the gradient accumulation are those of pair2_f32.
template <int D, typename K>
__device__ __forceinline__ void pair2_far(const K &a, const float4 (&xi)[D], const float4 (&xj)[D], float2 y2,
                                          float2 (&racc)[D], float2 (&cacc)[D], float2 &e2) {
    float2 s[D];
    float2 d2h, cr;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float2 dh = add2(f2(xi[k].x, xi[k].y), f2(xj[k].x, xj[k].y));
        const float2 dl = add2(f2(xi[k].z, xi[k].w), f2(xj[k].z, xj[k].w));
        s[k] = add2(dh, dl);
        if (k == 0) {
            d2h = mul2(dh, dh);
            cr = fma2(dl, add2(s[k], dh), f2(FLT_MIN, FLT_MIN));
        } else {
            d2h = fma2(dh, dh, d2h);
            cr = fma2(dl, add2(s[k], dh), cr);
        }
    }
    const float2 d2 = add2(d2h, cr);
    const float2 inv = f2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
    const float2 del = f2(sqrt_approx(d2.x), sqrt_approx(d2.y));
    const float2 res = add2(fma2(neg2(del), del, d2h), cr);
    const float2 hinv = mul2(inv, f2(0.5f, 0.5f));
    const float2 e = fma2(neg2(res), hinv, add2(y2, neg2(del)));
    e2 = fma2(e, e, e2);
    // w / delta = -(y - delta) / (sigma^2 delta)
    const float2 wi = mul2(mul2(e, a.neg_inv_s2), inv);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        racc[k] = fma2(wi, s[k], racc[k]);
        cacc[k] = fma2(wi, s[k], cacc[k]);
    }
}

// Row box of a row block: per coordinate the smallest and largest x_i of its
// 64 rows, from the row-pair split layout in shared memory ([k][row pair]
// float4 {xh_i, xh_i+1, xl_i, xl_i+1}; xh + xl is x exactly).  Every lane of
// the calling warp gets box[0..D) = minima, box[D..2D) = maxima.
template <int D>
__device__ __forceinline__ void row_box(const float4 *xis, int lane, float (&box)[2 * D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float4 v = xis[k * 32 + lane];
        const float a0 = v.x + v.z, a1 = v.y + v.w;
        float lo = fminf(a0, a1), hi = fmaxf(a0, a1);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        box[k] = lo;
        box[D + k] = hi;
    }
}

// Whether every pair of the warp's 64 rows x 8 columns lies at squared
// distance >= far_d2: each lane bounds the distance of its two columns
// (split layout {-xh, -xh, -xl, -xl}) from the row box from below; the
// decision is warp-uniform.
template <int D>
__device__ __forceinline__ bool block_far(const float *box, const float4 (&xj)[2][D], float far_d2) {
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float lo = box[k], hi = box[D + k];
        const float c0 = -(xj[0][k].x + xj[0][k].z), c1 = -(xj[1][k].x + xj[1][k].z);
        const float d0 = fmaxf(fmaxf(lo - c0, c0 - hi), 0.f);
        const float d1 = fmaxf(fmaxf(lo - c1, c1 - hi), 0.f);
        g0 = fmaf(d0, d0, g0);
        g1 = fmaf(d1, d1, g1);
    }
    return __all_sync(0xffffffffu, fminf(g0, g1) >= far_d2);
}

// One tile for this lane: 8 rows x 4 columns, column pairs one at a time;
// the column sums of each pair are reduced over the 8 row lanes and written.
// FAR (unmasked tiles only): a column pair whose whole 64 x 8 block of the
// warp lies beyond the cut-off (block_far against the row box `box`) takes
// pair2_far; far_d2 = +inf turns that off.  Returns the number of column
// pairs that took pair2_far (0..2).
template <int D, bool MASKED, typename K, bool HELDOUT = false, bool FAR = false>
__device__ __forceinline__ int tile_f32(const K &a, const float4 *ys, const float4 *xjs, const float4 *xis,
                                         int lane, int row_rel, int col_lo, int64_t ncol_valid,
                                         float2 (&racc)[4][D], float *colp, float2 &e2, float2 &md, float2 &prod,
                                         const float *box = nullptr, float far_d2 = 0.f) {
    constexpr int V = 2 * D;  // column values of one column pair
    constexpr int P = Pow2<V>::value;
    const int la = lane & 7, lb = lane >> 3;
    int n_far = 0;
#pragma unroll 1
    for (int cp = 0; cp < 2; ++cp) {
        float4 xj[2][D];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) xj[e][k] = xjs[(4 * lb + 2 * cp + e) * D + k];
        float2 cacc[2][D];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) cacc[e][k] = f2(0.f, 0.f);
        bool far = false;
        if constexpr (FAR && !MASKED) far = block_far<D>(box, xj, far_d2);
        if (far) {
            ++n_far;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 yv = ys[(2 * q + cp) * 32 + (lane ^ (cp << 2))];
                float4 xi[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xi[k] = xis[k * 32 + la + 8 * q];
                pair2_far<D, K>(a, xi, xj[0], f2(yv.x, yv.y), racc[q], cacc[0], e2);
                pair2_far<D, K>(a, xi, xj[1], f2(yv.z, yv.w), racc[q], cacc[1], e2);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 yv = ys[(2 * q + cp) * 32 + (lane ^ (cp << 2))];
                float4 xi[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xi[k] = xis[k * 32 + la + 8 * q];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float2 y2 = e == 0 ? f2(yv.x, yv.y) : f2(yv.z, yv.w);
                    float2 vm = f2(1.f, 1.f);
                    if (MASKED) {
                        // rows r, r+1 of the row pair, column c (tile-relative,
                        // rows shifted so that the diagonal test is c > r); with
                        // a cross-validation fold, a held-out pair carries y < 0
                        const int r = row_rel + 2 * (la + 8 * q);
                        const int c = col_lo + 4 * lb + 2 * cp + e;
                        const bool cv = c < ncol_valid;
                        if (HELDOUT)
                            vm = f2((cv && c > r && y2.x >= 0.f) ? 1.f : 0.f,
                                    (cv && c > r + 1 && y2.y >= 0.f) ? 1.f : 0.f);
                        else
                            vm = f2((cv && c > r) ? 1.f : 0.f, (cv && c > r + 1) ? 1.f : 0.f);
                    }
                    pair2_f32<D, MASKED, K>(a, xi, xj[e], y2, vm, racc[q], cacc[e], e2, md, prod);
                }
            }
        }
        // column sums over the tile's 64 rows: 3-level transpose over the row lanes
        float colv[P];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) colv[e * D + k] = cacc[e][k].x + cacc[e][k].y;
#pragma unroll
        for (int i = V; i < P; ++i) colv[i] = 0.f;
        lane_reduce<P, 3>(colv, lane, 0);
        bool writer;
        const int base = reduced_base<P, 3>(lane, 0, writer);
        constexpr int kHeld = P >= 8 ? P / 8 : 1;
        if (writer) {
#pragma unroll
            for (int i = 0; i < kHeld; ++i)
                if (base + i < V) colp[(4 * lb + 2 * cp) * D + base + i] = colv[i];
        }
    }
    return n_far;
}

// End of a strip for one problem: the row sums over the lane's 4 column
// lanes (lane transpose) and the 4 warps (shared memory, fixed order) into
// rp[64 * D], and the three scalar sums (Kahan pairs) into sp[0..2].  All
// threads of the CTA call it; `red` is shared scratch of
// 4 * 64 * D + 16 floats that nobody else uses meanwhile.
template <int D>
__device__ __forceinline__ void strip_epilogue_f32(const float2 (&racc)[4][D], float es, float ec, float ms, float mc,
                                                   float gs, float gc, float *red, float *rp, float *sp,
                                                   unsigned *err) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int VR = 8 * D;  // (q, k, half) values per lane
    float rv[VR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            rv[(q * D + k) * 2 + 0] = racc[q][k].x;
            rv[(q * D + k) * 2 + 1] = racc[q][k].y;
        }
    lane_reduce<VR, 2>(rv, lane, 3);
    {
        bool writer;
        const int base = reduced_base<VR, 2>(lane, 3, writer);
        const int la = lane & 7;
#pragma unroll
        for (int i = 0; i < VR / 4; ++i) {
            const int v = base + i;
            const int h = v & 1, k = (v >> 1) % D, q = (v >> 1) / D;
            const int row = 2 * (la + 8 * q) + h;
            red[(warp * kTile + row) * D + k] = rv[i];
        }
    }
    float sv[3] = {es - ec, ms - mc, gs - gc};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float v = sv[i];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[kPairWarps * kTile * D + warp * 4 + i] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < kTile * D; idx += kPairThreads) {
        float v = red[idx];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += red[w * kTile * D + idx];
        rp[idx] = v;
    }
    if (tid < 3) {
        const float *sr = red + kPairWarps * kTile * D;
        float v = sr[tid];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += sr[w * 4 + tid];
        sp[tid] = v;
        if (!isfinite(v)) atomicOr(err, kErrNonfinite);
    }
}

}  // namespace
}  // namespace mds
