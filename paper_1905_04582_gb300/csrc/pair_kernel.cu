// Fused pair pass of the truncated-normal MDS likelihood (arXiv:1905.04582,
// section 2.5 and Algorithms 1-2, re-designed for sm_103a).
//
// One CTA (4 warps) takes one strip: a row block I of 64 items against the
// column blocks [j0, j1).  For every pair (i, j) of the strip it computes, in
// registers and without storing anything per pair,
//   delta = ||x_i - x_j||,  e = y_ij - delta,  z = delta / sigma,
//   r_ij  = e^2 / (2 sigma^2) + log Phi(z)                       (Eq. (2))
//   w_ij  = (delta - y_ij) / sigma^2 + phi(z) / (sigma Phi(z))   (Eq. (9))
// and accumulates
//   row i    : sum_j w_ij (x_i - x_j) / delta     (registers, whole strip)
//   column j : sum_i w_ij (x_i - x_j) / delta     (warp shuffles, per tile)
//   scalars  : sum e^2, sum phi/Phi * delta, sum log Phi.
// Each pair is visited once (Algorithm 2 of the paper visits it twice); the
// gradient of x_i is -row_i - ... and of x_j is +column_j, combined with the
// other strips' partials by reduce_kernel.cu in a fixed order.
//
// Memory: Y streams from HBM/L2 once per pass with coalesced 128-bit loads
// that bypass L1; the strip's x_j (negated, column-pair interleaved) arrive in
// shared memory by one bulk TMA copy (cp.async.bulk + mbarrier); x_i stay in
// registers.
//
// Arithmetic (FP32C): packed f32x2 FMA/ADD/MUL (two column pairs per
// instruction) and MUFU rsqrt / ex2 / rcp / lg2.  Phi(z) = 1 - phi(z) R(z)
// with the Mills ratio R approximated by the rational P/D of
// mills_ratio_coeffs.h, so that one reciprocal gives 1/Phi = D / (D - phi P);
// log Phi is summed as -log2 of running products of 1/Phi (one lg2 per 16
// pairs; 1/Phi <= 2 so 16 factors cannot overflow).  Sums are plain FP32 over
// one tile, Kahan-compensated FP32 across the strip's tiles, and FP64 across
// lanes, warps and strips.
//
// Arithmetic (FP64): CUDA's double sqrt / erfc / log1p / exp per pair, FP64
// sums throughout (the plain FP64 GPU path).
#include <cfloat>
#include <cstdint>
#include <type_traits>

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

// Streaming 128-bit load: read-only path, no L1 allocation (Y is used once
// per pass by exactly one lane).
__device__ __forceinline__ float4 ld_stream(const float *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bulk (1-D TMA) copy global -> shared, completion signalled on an mbarrier.
// Requirements (checked by the host): 16-byte aligned addresses, size a
// multiple of 16 bytes and below the mbarrier transaction limit.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%2], [%3], %1, [%0];"
        :
        : "r"(smem_addr(bar)), "r"(bytes), "r"(smem_addr(dst)), "l"(src)
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
}

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

// Wait for the mbarrier phase with a time limit.  Returns false (and sets the
// error word) when the limit passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, unsigned *err,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (global_ns() - t0 > limit_ns) {
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
    return true;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// ------------------------------------------------------ packed FP32 helpers

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
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

// Sum over the 32 lanes of the values v[0..P), P a power of two <= 32, by
// recursive halving: afterwards lane l holds the full sum of value
// index (l >> (5 - log2 P)) in v[0].
template <int P, typename T>
__device__ __forceinline__ void transpose_reduce(T (&v)[P], int lane) {
    static_assert((P & (P - 1)) == 0 && P <= 32, "P must be a power of two <= 32");
    int cnt = P;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (cnt > 1) {
            const int half = cnt / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                T send = upper ? v[i] : v[i + half];
                T keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

template <int V>
struct Pow2 {
    static constexpr int value = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : V <= 16 ? 16 : 32;
};
template <int P>
struct Log2 {
    static constexpr int value = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
};

// Deterministic FP64 warp sum (fixed butterfly order).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory layout of one CTA: [x_j strip | reduction scratch] + mbarrier.
template <typename T2, int D>
__host__ __device__ constexpr size_t xj_bytes(int strip) {
    return static_cast<size_t>(strip) * (kTile / 2) * D * sizeof(T2);
}
template <int D>
__host__ __device__ constexpr size_t red_bytes() {
    return static_cast<size_t>(kPairWarps) * kTile * D * sizeof(double) + kPairWarps * 4 * sizeof(double);
}

// --------------------------------------------------------------- the pass

template <typename T, int D>
struct Types;
template <int D>
struct Types<float, D> {
    using T2 = float2;
};
template <int D>
struct Types<double, D> {
    using T2 = double2;
};

template <int D, bool MASKED>
__device__ __forceinline__ void chunk_f32(const PairArgs &a, const float4 (&yv)[2], const float2 *xj,
                                          const float2 (&xi)[2][D], int row0, int col0, int64_t n,
                                          float2 (&racc)[2][D], float (&colv)[4 * D], float2 &e2,
                                          float2 &md, float2 &prod) {
    // x_j of the chunk's two column pairs (negated, {j, j+1} interleaved)
    float2 xn[2][D];
#pragma unroll
    for (int cp = 0; cp < 2; ++cp)
#pragma unroll
        for (int k = 0; k < D; ++k) xn[cp][k] = xj[cp * D + k];

    float2 cacc[2][D];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
            const float2 y2 = cp == 0 ? f2(yv[h].x, yv[h].y) : f2(yv[h].z, yv[h].w);
            float2 dl[D];
#pragma unroll
            for (int k = 0; k < D; ++k) dl[k] = add2(xi[h][k], xn[cp][k]);
            float2 d2 = mul2(dl[0], dl[0]);
#pragma unroll
            for (int k = 1; k < D; ++k) d2 = fma2(dl[k], dl[k], d2);
            // +FLT_MIN keeps rsqrt finite for coincident points; their
            // delta = d2 * inv is then 0 and so is their gradient term.
            d2 = add2(d2, f2(FLT_MIN, FLT_MIN));
            const float2 inv = f2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
            const float2 del = mul2(d2, inv);
            float2 e = fma2(del, f2(-1.f, -1.f), y2);  // y - delta
            const float2 ea = mul2(d2, a.c_phi);
            const float2 ph = f2(ex2_approx(ea.x), ex2_approx(ea.y));  // exp(-z^2/2)
            // -P(z)/sqrt(2 pi) and D(z) by Horner in delta (sigma folded in)
            float2 pn = fma2(a.mp[3], del, a.mp[2]);
            pn = fma2(pn, del, a.mp[1]);
            pn = fma2(pn, del, a.mp[0]);
            float2 dd = fma2(a.md[3], del, a.md[2]);
            dd = fma2(dd, del, a.md[1]);
            dd = fma2(dd, del, a.md[0]);
            const float2 den = fma2(ph, pn, dd);  // D - phi' P / sqrt(2 pi) = D Phi
            const float2 rden = f2(rcp_approx(den.x), rcp_approx(den.y));
            float2 ip = mul2(dd, rden);  // 1 / Phi
            float2 mm = mul2(ph, ip);    // sqrt(2 pi) phi / Phi
            if (MASKED) {
                const int r = row0 + h * 32;
                const int c = col0 + cp * 2;
                const bool v0 = (c > r) && (c < n);
                const bool v1 = (c + 1 > r) && (c + 1 < n);
                const float2 vm = f2(v0 ? 1.f : 0.f, v1 ? 1.f : 0.f);
                e = mul2(e, vm);
                mm = mul2(mm, vm);
                ip = f2(v0 ? ip.x : 1.f, v1 ? ip.y : 1.f);
            }
            prod = mul2(prod, ip);
            e2 = fma2(e, e, e2);
            md = fma2(mm, del, md);
            // w = (delta - y)/sigma^2 + phi/(sigma Phi); wi = w / delta
            const float2 w = fma2(e, a.neg_inv_s2, mul2(mm, a.m_coef));
            const float2 wi = mul2(w, inv);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float2 c = mul2(wi, dl[k]);
                racc[h][k] = add2(racc[h][k], c);
                cacc[cp][k] = (h == 0) ? c : add2(cacc[cp][k], c);
            }
        }
    }
#pragma unroll
    for (int cp = 0; cp < 2; ++cp)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            colv[(2 * cp) * D + k] = cacc[cp][k].x;
            colv[(2 * cp + 1) * D + k] = cacc[cp][k].y;
        }
}

template <int D, bool MASKED>
__device__ __forceinline__ void chunk_f64(const PairArgs &a, const float4 (&yv)[2], const double2 *xj,
                                          const double (&xi)[2][D], int row0, int col0, int64_t n,
                                          double (&racc)[2][D], double (&colv)[4 * D], double &e2,
                                          double &md, double &lphi) {
    constexpr double kInvSqrt2Pi = 0.39894228040143267794;
    constexpr double kInvSqrt2 = 0.70710678118654752440;
    double cacc[4][D];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float yq = q == 0 ? yv[h].x : q == 1 ? yv[h].y : q == 2 ? yv[h].z : yv[h].w;
            const int cp = q >> 1;
            double dl[D];
            double d2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double2 xn = xj[cp * D + k];
                dl[k] = xi[h][k] + ((q & 1) ? xn.y : xn.x);
                d2 = fma(dl[k], dl[k], d2);
            }
            const double del = sqrt(d2);
            const double inv = del > 0.0 ? 1.0 / del : 0.0;
            double e = static_cast<double>(yq) - del;
            const double z = del * a.inv_sigma;
            const double qz = 0.5 * erfc(z * kInvSqrt2);
            const double phi = exp(-0.5 * z * z) * kInvSqrt2Pi;
            double m = phi / (1.0 - qz);  // phi / Phi
            double lp = log1p(-qz);       // log Phi
            if (MASKED) {
                const int r = row0 + h * 32;
                const int c = col0 + q;
                const bool v = (c > r) && (c < n);
                e = v ? e : 0.0;
                m = v ? m : 0.0;
                lp = v ? lp : 0.0;
            }
            e2 = fma(e, e, e2);
            md = fma(m, del, md);
            lphi += lp;
            const double wi = (m * a.inv_sigma - e * a.inv_s2) * inv;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double c = wi * dl[k];
                racc[h][k] += c;
                cacc[q][k] = (h == 0) ? c : cacc[q][k] + c;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) colv[q * D + k] = cacc[q][k];
}

template <typename T, int D>
__global__ void __launch_bounds__(kPairThreads) pair_pass_kernel(const __grid_constant__ PairArgs a, int strip_cap) {
    using T2 = typename Types<T, D>::T2;
    constexpr int V = 4 * D;              // column values per chunk per lane
    constexpr int P = Pow2<V>::value;     // padded to a power of two for the lane transpose
    constexpr int kLog2P = Log2<P>::value;

    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    if (blockIdx.x >= static_cast<unsigned>(a.n_strips)) return;
    const Strip st = a.strips[blockIdx.x];
    const int nst = st.j1 - st.j0;
    if (nst < 1 || nst > strip_cap) {
        if (tid == 0) atomicOr(a.err, kErrBadArgs);
        return;
    }

    T2 *xj_s = reinterpret_cast<T2 *>(smem);
    const size_t xjb = xj_bytes<T2, D>(strip_cap);
    const size_t rb = red_bytes<D>();
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + ((xjb > rb ? xjb : rb) + 15) / 16 * 16);

    if (tid == 0) {
        mbar_init(bar, 1);
        const T2 *src = reinterpret_cast<const T2 *>(a.xneg) + static_cast<int64_t>(st.j0) * (kTile / 2) * D;
        tma_load_1d(xj_s, src, static_cast<uint32_t>(xj_bytes<T2, D>(nst)), bar);
    }

    // x_i of this lane's two rows, broadcast {x, x} for the packed f32 math
    const int64_t rowbase = static_cast<int64_t>(st.I) * kTile;
    const T *xr = reinterpret_cast<const T *>(a.xrow);
    using XI = typename std::conditional<std::is_same<T, float>::value, float2, double>::type;
    XI xi[2][D];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const T v = xr[(rowbase + h * 32 + lane) * D + k];
            if constexpr (std::is_same<T, float>::value)
                xi[h][k] = f2(v, v);
            else
                xi[h][k] = v;
        }

    // accumulators
    XI racc[2][D];
    float rs[2][D], rc[2][D];  // FP32C: Kahan state across tiles
    double rsd[2][D];          // FP64: plain across tiles
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if constexpr (std::is_same<T, float>::value)
                racc[h][k] = f2(0.f, 0.f);
            else
                racc[h][k] = 0.0;
            rs[h][k] = rc[h][k] = 0.f;
            rsd[h][k] = 0.0;
        }
    float es = 0.f, ec = 0.f, ms = 0.f, mc = 0.f, gs = 0.f, gc = 0.f;  // FP32C scalars
    double e2d = 0.0, mdd = 0.0, lpd = 0.0;                             // FP64 scalars

    // One thread waits (bounded) for the x_j copy and tells the others; a
    // block-wide barrier then orders the copied data before every reader.
    __shared__ int xj_ok;
    if (tid == 0) {
        bool ok = mbar_wait_bounded(bar, 0, a.err, kWaitLimitNs);
        if (!ok) ok = mbar_wait_bounded(bar, 0, a.err, kWaitLimitNs);  // copy still in flight
        xj_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!xj_ok) return;

    const int64_t n = a.n;
    const int nt = a.nt;
    const bool ragged = (n % kTile) != 0;
    const int total = nst * kChunksPerWarp;  // chunks this warp processes in the strip
    const int64_t t0 = tile_index(st.I, st.j0, nt);

    // software pipeline: chunk u+1 is in flight while chunk u is computed.
    // Chunk u of this warp: tile t0 + u/4, chunk warp*4 + u%4 of that tile.
    const float *yp = a.y + t0 * kTileElems + (warp * kChunksPerWarp) * (kTile * kChunkCols) + lane * 4;
    float4 ycur[2], ynext[2];
    ycur[0] = ld_stream(yp);
    ycur[1] = ld_stream(yp + 32 * 4);

    float2 e2 = f2(0.f, 0.f), mdv = f2(0.f, 0.f), prod = f2(1.f, 1.f);
    double e2t = 0.0, mdt = 0.0, lpt = 0.0;
    T *colp = reinterpret_cast<T *>(a.col_part) + (t0 * kTile + warp * kChunksPerWarp * kChunkCols) * D;

    for (int jt = 0; jt < nst; ++jt) {
        const int J = st.j0 + jt;
        const bool masked = (J == st.I) || (ragged && J == nt - 1);
        // this lane's first row relative to column block J (diagonal test),
        // and the number of valid columns left in block J
        const int row0 = static_cast<int>(rowbase - static_cast<int64_t>(J) * kTile) + lane;
        const int64_t nrel = n - static_cast<int64_t>(J) * kTile;
#pragma unroll 1
        for (int cc = 0; cc < kChunksPerWarp; ++cc) {
            const int u = jt * kChunksPerWarp + cc;
            if (u + 1 < total) {
                const float *pn = yp + (cc + 1 < kChunksPerWarp ? (kTile * kChunkCols)
                                                                : (kTileElems - (kChunksPerWarp - 1) * kTile * kChunkCols));
                ynext[0] = ld_stream(pn);
                ynext[1] = ld_stream(pn + 32 * 4);
                yp = pn;
            }
            const int c = warp * kChunksPerWarp + cc;  // chunk within the tile
            const int col0 = c * kChunkCols;
            const T2 *xjc = xj_s + (jt * (kTile / 2) + c * 2) * D;

            T colv[P];
            if constexpr (std::is_same<T, float>::value) {
                float cv[V];
                if (masked)
                    chunk_f32<D, true>(a, ycur, xjc, xi, row0, col0, nrel, racc, cv, e2, mdv, prod);
                else
                    chunk_f32<D, false>(a, ycur, xjc, xi, row0, col0, nrel, racc, cv, e2, mdv, prod);
#pragma unroll
                for (int i = 0; i < P; ++i) colv[i] = i < V ? cv[i] : 0.f;
            } else {
                double cv[V];
                if (masked)
                    chunk_f64<D, true>(a, ycur, xjc, xi, row0, col0, nrel, racc, cv, e2t, mdt, lpt);
                else
                    chunk_f64<D, false>(a, ycur, xjc, xi, row0, col0, nrel, racc, cv, e2t, mdt, lpt);
#pragma unroll
                for (int i = 0; i < P; ++i) colv[i] = i < V ? cv[i] : 0.0;
            }

            // column sums over the tile's 64 rows: lane transpose + butterfly
            transpose_reduce<P>(colv, lane);
            {
                const int idx = lane >> (5 - kLog2P);
                if ((lane & ((32 >> kLog2P) - 1)) == 0 && idx < V) colp[cc * kChunkCols * D + idx] = colv[0];
            }
            if (u + 1 < total) {
                ycur[0] = ynext[0];
                ycur[1] = ynext[1];
            }
        }
        colp += kTile * D;

        // end of this warp's share of tile J: fold the tile sums
        if constexpr (std::is_same<T, float>::value) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    kahan_add(rs[h][k], rc[h][k], racc[h][k].x + racc[h][k].y);
                    racc[h][k] = f2(0.f, 0.f);
                }
            kahan_add(es, ec, e2.x + e2.y);
            kahan_add(ms, mc, mdv.x + mdv.y);
            kahan_add(gs, gc, lg2_approx(prod.x) + lg2_approx(prod.y));
            e2 = f2(0.f, 0.f);
            mdv = f2(0.f, 0.f);
            prod = f2(1.f, 1.f);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    rsd[h][k] += racc[h][k];
                    racc[h][k] = 0.0;
                }
            e2d += e2t;
            mdd += mdt;
            lpd += lpt;
            e2t = mdt = lpt = 0.0;
        }
    }

    // ---- strip epilogue: combine the 4 warps in a fixed order (FP64)
    __syncthreads();  // everyone done with the x_j strip; reuse smem
    double *red = reinterpret_cast<double *>(smem);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double v;
            if constexpr (std::is_same<T, float>::value)
                v = static_cast<double>(rs[h][k]) - static_cast<double>(rc[h][k]);
            else
                v = rsd[h][k];
            red[(warp * kTile + h * 32 + lane) * D + k] = v;
        }
    double sv[3];
    if constexpr (std::is_same<T, float>::value) {
        sv[0] = static_cast<double>(es) - static_cast<double>(ec);
        sv[1] = static_cast<double>(ms) - static_cast<double>(mc);
        sv[2] = static_cast<double>(gs) - static_cast<double>(gc);
    } else {
        sv[0] = e2d;
        sv[1] = mdd;
        sv[2] = lpd;
    }
    double *sred = red + kPairWarps * kTile * D;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double w = warp_sum(sv[i]);
        if (lane == 0) sred[warp * 4 + i] = w;
    }
    __syncthreads();
    double *rp = a.row_part + static_cast<int64_t>(st.row_slot) * kTile * D;
    for (int idx = tid; idx < kTile * D; idx += kPairThreads) {
        double v = red[idx];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += red[w * kTile * D + idx];
        rp[idx] = v;
    }
    if (tid < 3) {
        double v = sred[tid];
#pragma unroll
        for (int w = 1; w < kPairWarps; ++w) v += sred[w * 4 + tid];
        a.scal_part[static_cast<int64_t>(blockIdx.x) * kScalarParts + tid] = v;
        if (!isfinite(v)) atomicOr(a.err, kErrNonfinite);
    }
}

template <typename T, int D>
cudaError_t launch_d(const PairArgs &a, int strip_len, cudaStream_t s) {
    using T2 = typename Types<T, D>::T2;
    const size_t xjb = xj_bytes<T2, D>(strip_len);
    const size_t rb = red_bytes<D>();
    const size_t smem = ((xjb > rb ? xjb : rb) + 15) / 16 * 16 + 16;
    auto kern = pair_pass_kernel<T, D>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    if (a.n_strips <= 0) return cudaSuccess;
    kern<<<a.n_strips, kPairThreads, smem, s>>>(a, strip_len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_any(const PairArgs &a, int d, int strip_len, cudaStream_t s) {
    switch (d) {
        case 1: return launch_d<T, 1>(a, strip_len, s);
        case 2: return launch_d<T, 2>(a, strip_len, s);
        case 3: return launch_d<T, 3>(a, strip_len, s);
        case 4: return launch_d<T, 4>(a, strip_len, s);
        case 5: return launch_d<T, 5>(a, strip_len, s);
        case 6: return launch_d<T, 6>(a, strip_len, s);
        case 7: return launch_d<T, 7>(a, strip_len, s);
        case 8: return launch_d<T, 8>(a, strip_len, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T2, int D>
size_t smem_d(int strip_len) {
    const size_t xjb = xj_bytes<T2, D>(strip_len);
    const size_t rb = red_bytes<D>();
    return ((xjb > rb ? xjb : rb) + 15) / 16 * 16 + 16;
}

template <typename T2>
size_t smem_any(int d, int strip_len) {
    switch (d) {
        case 1: return smem_d<T2, 1>(strip_len);
        case 2: return smem_d<T2, 2>(strip_len);
        case 3: return smem_d<T2, 3>(strip_len);
        case 4: return smem_d<T2, 4>(strip_len);
        case 5: return smem_d<T2, 5>(strip_len);
        case 6: return smem_d<T2, 6>(strip_len);
        case 7: return smem_d<T2, 7>(strip_len);
        case 8: return smem_d<T2, 8>(strip_len);
        default: return 0;
    }
}

}  // namespace

cudaError_t launch_pair_pass_f32(const PairArgs &a, int d, int strip_len, cudaStream_t s) {
    return launch_any<float>(a, d, strip_len, s);
}
cudaError_t launch_pair_pass_f64(const PairArgs &a, int d, int strip_len, cudaStream_t s) {
    return launch_any<double>(a, d, strip_len, s);
}
size_t pair_smem_bytes(int d, int strip_len, bool fp64) {
    return fp64 ? smem_any<double2>(d, strip_len) : smem_any<float2>(d, strip_len);
}

}  // namespace mds
