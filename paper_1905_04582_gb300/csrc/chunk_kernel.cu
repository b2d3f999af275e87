// Chunked fused pair pass of the truncated-normal MDS likelihood, FP32C
// (arXiv:1905.04582, section 2.5 and Algorithms 1-2: the transformation of
// every pair and the reduction of the per-pair terms, re-designed for sm_103a).
//
// The per-pair terms are those of pair_kernel.cu: for every pair i < j
//   delta = ||x_i - x_j||,  e = y_ij - delta,  z = delta / sigma,
//   r_ij  = e^2 / (2 sigma^2) + log Phi(z)                       (Eq. (2))
//   w_ij  = (delta - y_ij) / sigma^2 + phi(z) / (sigma Phi(z))   (Eq. (9))
// with the row sum  sum_j w_ij (x_i - x_j) / delta  and the column sum
// sum_i w_ij (x_i - x_j) / delta  of the gradient, each pair visited once.
//
// What differs from the strip pass:
//  - work split: the tiles, in row-block order, are cut into one contiguous
//    chunk per group of four warps, of equal estimated cost (far and near
//    tiles weighted by the per-tile far counts of an earlier pass), so that
//    the pass is one wave of chunks that end together.  Each warp keeps its
//    3-stage TMA ring (its 4 KB quarter of every Y tile and its 16 columns of
//    locations) running across row-block boundaries; at a boundary, and
//    after every max_seg_tiles(D) tiles of one row block, it writes its row sums
//    to its own partial slot and goes on.  No barrier of the group runs
//    inside the loop.
//  - the row block's split locations sit in three shared-memory buffers
//    shared by the group's warps: the last warp to finish a row block (a
//    count in shared memory) issues the bulk copy of the row block three
//    ahead into the buffer it frees, so even a run of one-tile row blocks
//    (the last ones of the triangle) finds its locations landed.
//  - the gradient weight is summed without its factor -1/sigma^2:
//    w' = -sigma^2 w = (e - sigma phi'/sqrt(2 pi)) ... (one FMA fewer per
//    pair); the reduction multiplies the partial sums by -1/sigma^2 in FP64.
//  - the column locations are {-xh_j, -xl_j} (8 bytes per coordinate, half
//    the shared memory of the duplicated form, which is built in registers).
#include <cfloat>
#include <cstdint>

#include "mds_internal.h"
#include "pair_math.cuh"

namespace mds {
namespace {

constexpr int kChunkStages = 3;  // per-warp ring depth
constexpr int kXisBufs = 3;      // row-block location buffers of a group (two row blocks of lead)

__host__ __device__ constexpr int align128(int b) { return (b + 127) / 128 * 128; }

template <int D>
struct ChunkLayout {
    static constexpr int kXjBytes = kWarpCols * D * 8;  // 16 columns x D float2
    static constexpr int kYBytes = kWarpTileElems * 4;  // a warp's quarter of a Y tile
    static constexpr int kStageBytes = align128(kYBytes + kXjBytes);
    static constexpr int kXiBytes = 32 * D * 16;         // a row block: 32 row pairs x D float4
    static constexpr int kXiOffset = kPairWarps * kChunkStages * kStageBytes;
    static constexpr int kBarOffset = kXiOffset + kXisBufs * align128(kXiBytes);
    // mbarriers: [warp][stage], then the row-block buffers
    static constexpr int kCntOffset = kBarOffset + (kPairWarps * kChunkStages + kXisBufs) * 8;
    // done[kXisBufs] (warps that finished a row block on each buffer), issued[kXisBufs] (copies into it)
    static constexpr int kBoxOffset = kCntOffset + 2 * kXisBufs * 4;
    static constexpr int kBytes = kBoxOffset + kPairWarps * 2 * D * 4;
};

// x / 2 for a normal, positive FP32 x: one less in the exponent field (an
// integer subtraction on the ALU pipe instead of an FP32 multiply).
__device__ __forceinline__ float half_of(float x) { return __int_as_float(__float_as_int(x) - 0x00800000); }

// Geometry of two pairs (rows r, r+1 packed) against one column: the exact
// split differences per coordinate, delta, 1 / delta and the
// residual-corrected e = y - delta (see mds_internal.h, Split).
template <int D>
__device__ __forceinline__ void geom2(const float4 (&xi)[D], const float4 (&xj)[D], float2 y2, float2 (&s)[D],
                                      float2 &d2, float2 &inv, float2 &del, float2 &e) {
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
            d2h = fma2(dh, dh, d2h);           // exact
            cr = fma2(dl, add2(s[k], dh), cr);  // Dl (2 Dh + Dl)
        }
    }
    d2 = add2(d2h, cr);
    inv = f2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
    del = f2(sqrt_approx(d2.x), sqrt_approx(d2.y));
    // delta_true = del + res / (2 del), res = (d2h - del^2) + cr
    const float2 res = add2(fma2(neg2(del), del, d2h), cr);
    const float2 hinv = f2(half_of(inv.x), half_of(inv.y));
    e = fma2(neg2(res), hinv, add2(y2, neg2(del)));
}

// Both-sided accumulation of the scaled gradient weight wi' = -sigma^2 w / delta
// (INIT: the column sums start here, a multiply instead of zeroing them).
template <int D, bool INIT = false>
__device__ __forceinline__ void accum2(float2 wi, const float2 (&s)[D], float2 (&racc)[D], float2 (&cacc)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        racc[k] = fma2(wi, s[k], racc[k]);
        cacc[k] = INIT ? mul2(wi, s[k]) : fma2(wi, s[k], cacc[k]);
    }
}

// The full body: Phi via the Mills ratio (pair_kernel.cu), e^2, phi'/Phi
// delta and the product of 1/Phi accumulated; MASKED zeroes the pairs with
// vmask = 0.
template <int D, bool MASKED, bool INIT = false>
__device__ __forceinline__ void body_full(const PairArgs &a, const float4 (&xi)[D], const float4 (&xj)[D], float2 y2,
                                          float2 vmask, float2 (&racc)[D], float2 (&cacc)[D], float2 &e2, float2 &md,
                                          float2 &prod) {
    float2 s[D], d2, inv, del, e;
    geom2<D>(xi, xj, y2, s, d2, inv, del, e);
    const float2 ea = mul2(d2, a.c_phi);
    const float2 ph = f2(ex2_approx(ea.x), ex2_approx(ea.y));  // exp(-z^2 / 2)
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
    // wi' = (e - sigma phi'/sqrt(2 pi)) / delta
    accum2<D, INIT>(mul2(fma2(mm, a.c_m2, e), inv), s, racc, cacc);
}

// The far body (every pair of the warp's block at z >= z_c): the Phi terms
// are below FP32 resolution and dropped (pair_math.cuh, pair2_far).
template <int D, bool INIT = false>
__device__ __forceinline__ void body_far(const float4 (&xi)[D], const float4 (&xj)[D], float2 y2, float2 (&racc)[D],
                                         float2 (&cacc)[D], float2 &e2) {
    float2 s[D], d2, inv, del, e;
    geom2<D>(xi, xj, y2, s, d2, inv, del, e);
    e2 = fma2(e, e, e2);
    accum2<D, INIT>(mul2(e, inv), s, racc, cacc);
}

// Whether every pair of the warp's 64 rows x 8 columns lies at squared
// distance >= far_d2 (the columns in the {-xh, -xl} form).
template <int D>
__device__ __forceinline__ bool block_far2(const float *box, const float2 (&c)[2][D], float far_d2) {
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float lo = box[k], hi = box[D + k];
        const float c0 = -(c[0][k].x + c[0][k].y), c1 = -(c[1][k].x + c[1][k].y);
        const float d0 = fmaxf(fmaxf(lo - c0, c0 - hi), 0.f);
        const float d1 = fmaxf(fmaxf(lo - c1, c1 - hi), 0.f);
        g0 = fmaf(d0, d0, g0);
        g1 = fmaf(d1, d1, g1);
    }
    return __all_sync(0xffffffffu, fminf(g0, g1) >= far_d2);
}

// One tile for this lane (8 rows x 4 columns, column pairs in turn; see
// pair_math.cuh tile_f32).  Returns the column pairs that took the far body.
template <int D, bool MASKED, bool HELDOUT>
__device__ __forceinline__ int tile_chunk(const PairArgs &a, const float4 *ys, const float2 *xjs, const float4 *xis,
                                          int lane, int row_rel, int col_lo, int64_t ncol_valid, float2 (&racc)[4][D],
                                          float *colp, float2 &e2, float2 &md, float2 &prod, const float *box) {
    constexpr int V = 2 * D;
    constexpr int P = Pow2<V>::value;
    const int la = lane & 7, lb = lane >> 3;
    int n_far = 0;
#pragma unroll 1
    for (int cp = 0; cp < 2; ++cp) {
        float2 cj[2][D];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) cj[e][k] = xjs[(4 * lb + 2 * cp + e) * D + k];
        float4 xj[2][D];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) xj[e][k] = make_float4(cj[e][k].x, cj[e][k].x, cj[e][k].y, cj[e][k].y);
        float2 cacc[2][D];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int k = 0; k < D; ++k) cacc[e][k] = f2(0.f, 0.f);
        bool far = false;
        if constexpr (!MASKED) far = block_far2<D>(box, cj, a.far_d2);
        if (far) {
            ++n_far;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 yv = ys[(2 * q + cp) * 32 + (lane ^ (cp << 2))];
                float4 xi[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xi[k] = xis[k * 32 + la + 8 * q];
                body_far<D>(xi, xj[0], f2(yv.x, yv.y), racc[q], cacc[0], e2);
                body_far<D>(xi, xj[1], f2(yv.z, yv.w), racc[q], cacc[1], e2);
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
                            vm = f2((cv && c > r && y2.x >= 0.f) ? 1.f : 0.f, (cv && c > r + 1 && y2.y >= 0.f) ? 1.f : 0.f);
                        else
                            vm = f2((cv && c > r) ? 1.f : 0.f, (cv && c > r + 1) ? 1.f : 0.f);
                    }
                    body_full<D, MASKED>(a, xi, xj[e], y2, vm, racc[q], cacc[e], e2, md, prod);
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

// One tile for this lane in the tall mapping (D <= 2): lane 4b + a takes the
// 16 rows 2(a + 4q) + {0, 1}, q = 0..7, against the 2 columns 2b, 2b + 1 of
// the warp's 16: one block test, one load of the column locations and one
// 2-level column transpose per tile.  ybe / ybo: the lane's float4 index in
// the warp's Y quarter for even / odd q (tile layout, mds_internal.h), plus
// (q / 2) * 64.  Returns the 64 x 8 blocks of the warp that took the far body
// (0 or 2).
template <int D, bool MASKED, bool HELDOUT>
__device__ __forceinline__ int tile_tall(const PairArgs &a, const float4 *ys, const float2 *xjs, const float4 *xis,
                                         int lane, int ybe, int ybo, int row_rel, int col_lo, int64_t ncol_valid,
                                         float2 (&racc)[8][D], float *colp, float2 &e2, float2 &md, float2 &prod,
                                         const float *box) {
    constexpr int V = 2 * D;
    constexpr int P = Pow2<V>::value;
    const int la = lane & 3, lb = lane >> 2;
    float2 cj[2][D];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) cj[e][k] = xjs[(2 * lb + e) * D + k];
    float4 xj[2][D];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) xj[e][k] = make_float4(cj[e][k].x, cj[e][k].x, cj[e][k].y, cj[e][k].y);
    float2 cacc[2][D];
    bool far = false;
    if constexpr (!MASKED) far = block_far2<D>(box, cj, a.far_d2);
    if (far) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 yv = ys[(q >> 1) * 64 + ((q & 1) ? ybo : ybe)];
            float4 xi[D];
#pragma unroll
            for (int k = 0; k < D; ++k) xi[k] = xis[k * 32 + la + 4 * q];
            if (q == 0) {
                body_far<D, true>(xi, xj[0], f2(yv.x, yv.y), racc[q], cacc[0], e2);
                body_far<D, true>(xi, xj[1], f2(yv.z, yv.w), racc[q], cacc[1], e2);
            } else {
                body_far<D>(xi, xj[0], f2(yv.x, yv.y), racc[q], cacc[0], e2);
                body_far<D>(xi, xj[1], f2(yv.z, yv.w), racc[q], cacc[1], e2);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 yv = ys[(q >> 1) * 64 + ((q & 1) ? ybo : ybe)];
            float4 xi[D];
#pragma unroll
            for (int k = 0; k < D; ++k) xi[k] = xis[k * 32 + la + 4 * q];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float2 y2 = e == 0 ? f2(yv.x, yv.y) : f2(yv.z, yv.w);
                float2 vm = f2(1.f, 1.f);
                if (MASKED) {
                    const int r = row_rel + 2 * (la + 4 * q);
                    const int c = col_lo + 2 * lb + e;
                    const bool cv = c < ncol_valid;
                    if (HELDOUT)
                        vm = f2((cv && c > r && y2.x >= 0.f) ? 1.f : 0.f, (cv && c > r + 1 && y2.y >= 0.f) ? 1.f : 0.f);
                    else
                        vm = f2((cv && c > r) ? 1.f : 0.f, (cv && c > r + 1) ? 1.f : 0.f);
                }
                if (q == 0)
                    body_full<D, MASKED, true>(a, xi, xj[e], y2, vm, racc[q], cacc[e], e2, md, prod);
                else
                    body_full<D, MASKED>(a, xi, xj[e], y2, vm, racc[q], cacc[e], e2, md, prod);
            }
        }
    }
    // column sums over the tile's 64 rows: 2-level transpose over the row lanes
    float colv[P];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int k = 0; k < D; ++k) colv[e * D + k] = cacc[e][k].x + cacc[e][k].y;
#pragma unroll
    for (int i = V; i < P; ++i) colv[i] = 0.f;
    lane_reduce<P, 2>(colv, lane, 0);
    bool writer;
    const int base = reduced_base<P, 2>(lane, 0, writer);
    constexpr int kHeld = P >= 4 ? P / 4 : 1;
    if (writer) {
#pragma unroll
        for (int i = 0; i < kHeld; ++i)
            if (base + i < V) colp[2 * lb * D + base + i] = colv[i];
    }
    return far ? 2 : 0;
}

// Row sums of one segment in the tall mapping into the warp's partial slot:
// sums over the 8 column lanes of each row (3-level lane transpose).
template <int D>
__device__ __forceinline__ void flush_rows_tall(float2 (&racc)[8][D], int lane, float *rp) {
    constexpr int VR = 16 * D;
    float rv[VR];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            rv[(q * D + k) * 2 + 0] = racc[q][k].x;
            rv[(q * D + k) * 2 + 1] = racc[q][k].y;
            racc[q][k] = f2(0.f, 0.f);
        }
    lane_reduce<VR, 3>(rv, lane, 2);
    bool writer;
    const int base = reduced_base<VR, 3>(lane, 2, writer);
    const int la = lane & 3;
#pragma unroll
    for (int i = 0; i < VR / 8; ++i) {
        const int v = base + i;
        const int h = v & 1, k = (v >> 1) % D, q = (v >> 1) / D;
        rp[(2 * (la + 4 * q) + h) * D + k] = rv[i];
    }
}

// A warp's row sums of one segment (its 16 columns of every tile) into its
// partial slot rp[64 * D]: sums over the 4 column lanes of each row
// (lane transpose), then one store per value.
template <int D>
__device__ __forceinline__ void flush_rows(float2 (&racc)[4][D], int lane, float *rp) {
    constexpr int VR = 8 * D;
    float rv[VR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            rv[(q * D + k) * 2 + 0] = racc[q][k].x;
            rv[(q * D + k) * 2 + 1] = racc[q][k].y;
            racc[q][k] = f2(0.f, 0.f);
        }
    lane_reduce<VR, 2>(rv, lane, 3);
    bool writer;
    const int base = reduced_base<VR, 2>(lane, 3, writer);
    const int la = lane & 7;
#pragma unroll
    for (int i = 0; i < VR / 4; ++i) {
        const int v = base + i;
        const int h = v & 1, k = (v >> 1) % D, q = (v >> 1) / D;
        rp[(2 * (la + 8 * q) + h) * D + k] = rv[i];
    }
}

__device__ __forceinline__ void next_tile(int &I, int &J, int nt) {
    if (++J == nt) J = ++I;
}

// Bulk copy of row block I's split locations into a row buffer, completion
// on its mbarrier (the issuing thread arms it).
template <int D>
__device__ __forceinline__ void issue_rows(const PairArgs &a, int I, void *dst, uint64_t *bar) {
    constexpr uint32_t kB = ChunkLayout<D>::kXiBytes;
    mbar_expect_tx(bar, kB);
    tma_load_1d(dst, a.xrow + static_cast<int64_t>(I) * 32 * D, kB, bar);
}

// CTAs of the pass that fit one SM: three for D <= 4 (the register budget of
// up to 168 per thread lets the compiler interleave more of a tile's 16
// bodies per warp, which measured faster than four CTAs at 128 registers),
// two beyond.
template <int D>
constexpr int chunk_slots_per_sm() {
    return D <= 4 ? 3 : 2;
}

// One chunk per group of four warps.  G = 1: one group per CTA, several
// CTAs per SM.  G = chunk_slots_per_sm<D>(): one CTA per SM whose G groups
// each run a chunk in their own slice of shared memory.  CTAs that share an
// SM do not progress alike (the first resident one runs ahead: the three
// chunks of an SM ended at 12, 15 and 18 us at N = 5392), while the groups of
// one CTA do (17.6, 17.5, 17.2 us), so the grouped form ends with the SM's
// work instead of its slowest CTA.  Its groups cannot be replaced one by
// one, which favours the one-group form when there are several chunks per
// slot.  CAP: some chunk runs more than max_seg_tiles(D) tiles in one row
// block, so segments are cut every max_seg_tiles(D) tiles (without it the
// loop keeps only the row-block boundaries, which is the same cut for shorter
// runs, and compiles to faster code).
template <int D, bool HELDOUT, int G, bool CAP>
__global__ void __launch_bounds__(kPairThreads * G, (G > 1 ? 1 : chunk_slots_per_sm<D>()))
    pair_chunk_kernel(const __grid_constant__ PairArgs a) {
    using L = ChunkLayout<D>;
    // tall mapping (16 rows x 2 columns per lane) for D <= 2; 8 x 4 beyond,
    // where 16 rows of row sums would not fit the registers
    constexpr bool kTall = D <= 2;
    constexpr int kRP = kTall ? 8 : 4;  // row pairs per lane
    extern __shared__ __align__(128) unsigned char smem_cta[];
    // group, warp within it, thread within it, and the group's chunk
    const int lane = static_cast<int>(threadIdx.x) & 31;
    const int grp = static_cast<int>(threadIdx.x >> 5) / kPairWarps;
    const int warp = static_cast<int>(threadIdx.x >> 5) % kPairWarps;
    const int tid = static_cast<int>(threadIdx.x) % kPairThreads;
    const unsigned vb = blockIdx.x * G + static_cast<unsigned>(grp);
    unsigned char *const smem = smem_cta + grp * align128(L::kBytes);
    pdl_trigger();
    const bool active = vb < static_cast<unsigned>(a.n_strips);
    Chunk ch{};
    if (active) ch = a.chunks[vb];  // the chunk table is fixed between passes
    const int nt = a.nt;
    const int ntile = static_cast<int>(ch.t1 - ch.t0);
    const bool bad = active && (ntile < 1 || ch.t1 - ch.t0 > 0x7fffffff || ch.I0 < 0 || ch.I0 > ch.J0 ||
                                ch.J0 >= nt || ch.I1 < ch.I0 || ch.I1 >= nt || tile_index(ch.I0, ch.J0, nt) != ch.t0);
    if (bad && tid == 0) atomicOr(a.err, kErrBadArgs);
    unsigned char *ring = smem + warp * kChunkStages * L::kStageBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBarOffset) + warp * kChunkStages;
    uint64_t *xbar = reinterpret_cast<uint64_t *>(smem + L::kBarOffset) + kPairWarps * kChunkStages;
    unsigned *done = reinterpret_cast<unsigned *>(smem + L::kCntOffset);
    unsigned *issued = done + kXisBufs;
    float *box = reinterpret_cast<float *>(smem + L::kBoxOffset) + warp * 2 * D;
    auto xbuf = [&](int b) { return smem + L::kXiOffset + b * align128(L::kXiBytes); };

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < kChunkStages; ++s) mbar_init(&bars[s], 1);
        if (warp == 0) {
#pragma unroll
            for (int b = 0; b < kXisBufs; ++b) {
                mbar_init(&xbar[b], 1);
                done[b] = 0u;
                issued[b] = 0u;
            }
        }
        fence_mbar_init();
    }
    __syncthreads();  // the only CTA-wide barrier: every group passes it before any leaves
    if (!active || bad) return;

    // prologue: the first stages' Y quarters (Y is constant) may stream in
    // while the previous kernel drains; locations and partial buffers belong
    // to it until pdl_wait() returns
    const float *ynext = a.y + (ch.t0 - a.y_t0) * kTileElems + warp * kWarpTileElems;  // Y of the next tile to load
    if (lane == 0) {
        for (int s = 0; s < kChunkStages && s < ntile; ++s) {
            mbar_expect_tx(&bars[s], L::kYBytes + L::kXjBytes);
            tma_load_1d(ring + s * L::kStageBytes, ynext + s * kTileElems, L::kYBytes, &bars[s]);
        }
    }
    ynext += kChunkStages * kTileElems;
    pdl_wait();
    if (a.stamps && lane == 0) atomicMin(&a.stamps[0], global_ns());
    // the prefetch cursor: column block of the tile the next refill loads
    int Ip = ch.I0, Jp = ch.J0;
    const float2 *xcol_w = a.xcol2 + warp * kWarpCols * D;
    if (lane == 0) {
        for (int s = 0; s < kChunkStages && s < ntile; ++s) {
            tma_load_1d(ring + s * L::kStageBytes + L::kYBytes, xcol_w + static_cast<int64_t>(Jp) * kTile * D,
                        L::kXjBytes, &bars[s]);
            next_tile(Ip, Jp, nt);
        }
        if (warp == 0) {
            for (int b = 0; b < kXisBufs && ch.I0 + b <= ch.I1; ++b) {
                issued[b] = 1u;
                issue_rows<D>(a, ch.I0 + b, xbuf(b), &xbar[b]);
            }
        }
    } else {
        for (int s = 0; s < kChunkStages && s < ntile; ++s) next_tile(Ip, Jp, nt);
    }

    float2 racc[kRP][D];
#pragma unroll
    for (int q = 0; q < kRP; ++q)
#pragma unroll
        for (int k = 0; k < D; ++k) racc[q][k] = f2(0.f, 0.f);
    float2 es = f2(0.f, 0.f), ec = f2(0.f, 0.f);  // Kahan pairs: {sum e^2, sum m' delta}
    float gs = 0.f, gc = 0.f;                    // Kahan pair: sum log2(1/Phi)

    // the tall mapping's float4 indices into a Y quarter (tile layout,
    // mds_internal.h): lane 4b + a reads row pair a + 4q against column pair b
    const int tla = lane & 3, tlb = lane >> 2;
    const int ybe = (tlb & 1) * 32 + 8 * (tlb >> 1) + (tla | ((tlb & 1) << 2));
    const int ybo = (tlb & 1) * 32 + 8 * (tlb >> 1) + (tla | ((~tlb & 1) << 2));

    const int64_t n = a.n;
    const bool ragged = (n % kTile) != 0;
    float *const colp_base = reinterpret_cast<float *>(a.col_part) + warp * kWarpCols * D;
    float *rowp_base = reinterpret_cast<float *>(a.row_part);
    unsigned char *far_tile = a.far_tile ? a.far_tile + ch.t0 * kPairWarps + warp : nullptr;
    bool ok = true;
    int n_far = 0;
    int I = ch.I0, J = ch.J0;
    int cslot = static_cast<int>(col_slot(I, J));  // column-partial slot of tile (I, J), kept in step
    int seg = -1;  // segment of the chunk (row-partial slot 4 (seg0 + seg) + warp)
    int rb = -1;   // CAP: row block of the chunk, I - I0 (location buffer rb % kXisBufs)
    int run = 0;   // CAP: tiles of the current segment
    const float4 *xis = nullptr;
    int stage = 0;
    uint32_t phase = 0;
    int k = 0;
    for (; k < ntile; ++k) {
        if constexpr (!CAP) {
            if (k == 0 || J == I) {
                if (seg >= 0) {
                    // the previous segment (a row block) is done: its row sums
                    // out, its row buffer released (the last warp to release
                    // it refills it with the row block kXisBufs ahead)
                    float *rp = rowp_base + static_cast<int64_t>(4 * (ch.seg0 + seg) + warp) * kTile * D;
                    if constexpr (kTall)
                        flush_rows_tall<D>(racc, lane, rp);
                    else
                        flush_rows<D>(racc, lane, rp);
                    __syncwarp();
                    if (lane == 0) {
                        const int b = seg % kXisBufs;
                        __threadfence_block();
                        const unsigned old = atomicAdd(&done[b], 1u);
                        if ((old + 1u) % kPairWarps == 0u && ch.I0 + seg + kXisBufs <= ch.I1) {
                            fence_proxy_async();
                            issued[b] += 1u;
                            issue_rows<D>(a, ch.I0 + seg + kXisBufs, xbuf(b), &xbar[b]);
                        }
                    }
                }
                ++seg;
                if (!__all_sync(0xffffffffu,
                                mbar_wait_bounded(&xbar[seg % kXisBufs], static_cast<uint32_t>(seg / kXisBufs) & 1u,
                                                  a.err))) {
                    ok = false;
                    break;
                }
                xis = reinterpret_cast<const float4 *>(xbuf(seg % kXisBufs));
                float b[2 * D];
                row_box<D>(xis, lane, b);
                if (lane == 0)
#pragma unroll
                    for (int i = 0; i < 2 * D; ++i) box[i] = b[i];
                __syncwarp();
            }
        } else {
            const bool new_rb = k == 0 || J == I;
            if (new_rb || run == max_seg_tiles(D)) {
                if (seg >= 0) {
                    // the previous segment is done: its row sums out
                    float *rp = rowp_base + static_cast<int64_t>(4 * (ch.seg0 + seg) + warp) * kTile * D;
                    if constexpr (kTall)
                        flush_rows_tall<D>(racc, lane, rp);
                    else
                        flush_rows<D>(racc, lane, rp);
                    __syncwarp();
                }
                ++seg;
                run = 0;
            }
            if (new_rb) {
                if (rb >= 0 && lane == 0) {
                    // the previous row block is done: its buffer released (the
                    // last warp to release it refills it with the row block
                    // kXisBufs ahead)
                    const int b = rb % kXisBufs;
                    __threadfence_block();
                    const unsigned old = atomicAdd(&done[b], 1u);
                    if ((old + 1u) % kPairWarps == 0u && ch.I0 + rb + kXisBufs <= ch.I1) {
                        fence_proxy_async();
                        issued[b] += 1u;
                        issue_rows<D>(a, ch.I0 + rb + kXisBufs, xbuf(b), &xbar[b]);
                    }
                }
                ++rb;
                if (!__all_sync(0xffffffffu,
                                mbar_wait_bounded(&xbar[rb % kXisBufs], static_cast<uint32_t>(rb / kXisBufs) & 1u,
                                                  a.err))) {
                    ok = false;
                    break;
                }
                xis = reinterpret_cast<const float4 *>(xbuf(rb % kXisBufs));
                float b[2 * D];
                row_box<D>(xis, lane, b);
                if (lane == 0)
#pragma unroll
                    for (int i = 0; i < 2 * D; ++i) box[i] = b[i];
                __syncwarp();
            }
            ++run;
        }
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[stage], phase, a.err))) {
            ok = false;
            break;
        }
        const unsigned char *sbuf = ring + stage * L::kStageBytes;
        const float4 *ys = reinterpret_cast<const float4 *>(sbuf);
        const float2 *xjs = reinterpret_cast<const float2 *>(sbuf + L::kYBytes);
        const bool masked = (J == I) || (ragged && J == nt - 1) || (HELDOUT && a.tile_ho[ch.t0 + k]);
        float *const colp = colp_base + static_cast<int64_t>(cslot) * (kTile * D);
        float2 e2 = f2(0.f, 0.f), mdv = f2(0.f, 0.f), prod = f2(1.f, 1.f);
        const int row_rel = (I - J) * kTile;
        const int64_t ncv = n - static_cast<int64_t>(J) * kTile;
        int tf = 0;
        if constexpr (kTall) {
            if (masked)
                tf = tile_tall<D, true, HELDOUT>(a, ys, xjs, xis, lane, ybe, ybo, row_rel, warp * kWarpCols, ncv,
                                                 racc, colp, e2, mdv, prod, box);
            else
                tf = tile_tall<D, false, false>(a, ys, xjs, xis, lane, ybe, ybo, row_rel, warp * kWarpCols, ncv,
                                                racc, colp, e2, mdv, prod, box);
        } else {
            if (masked)
                tf = tile_chunk<D, true, HELDOUT>(a, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv, racc, colp,
                                                 e2, mdv, prod, box);
            else
                tf = tile_chunk<D, false, false>(a, ys, xjs, xis, lane, row_rel, warp * kWarpCols, ncv, racc, colp,
                                                e2, mdv, prod, box);
        }
        n_far += tf;
        if (far_tile && lane == 0) far_tile[static_cast<int64_t>(k) * kPairWarps] = static_cast<unsigned char>(tf);
        // all lanes are done reading this stage: refill it (async proxy after
        // the generic reads)
        __syncwarp();
        if (lane == 0 && k + kChunkStages < ntile) {
            fence_proxy_async();
            unsigned char *dst = ring + stage * L::kStageBytes;
            mbar_expect_tx(&bars[stage], L::kYBytes + L::kXjBytes);
            tma_load_1d(dst, ynext, L::kYBytes, &bars[stage]);
            tma_load_1d(dst + L::kYBytes, xcol_w + static_cast<int64_t>(Jp) * kTile * D, L::kXjBytes, &bars[stage]);
        }
        ynext += kTileElems;
        next_tile(Ip, Jp, nt);
        if (++stage == kChunkStages) {
            stage = 0;
            phase ^= 1u;
        }
        // per-tile sums into the Kahan pairs (packed: e^2 and m' delta together)
        {
            const float2 v = f2(e2.x + e2.y, mdv.x + mdv.y);
            const float2 yk = add2(v, neg2(ec));
            const float2 tk = add2(es, yk);
            ec = add2(add2(tk, neg2(es)), neg2(yk));
            es = tk;
        }
        kahan_add(gs, gc, lg2_approx(prod.x) + lg2_approx(prod.y));
        // col_slot(I, J + 1) = col_slot(I, J) + J + 1; a new row block
        // starts at its diagonal tile
        if (J + 1 < nt) {
            cslot += J + 1;
        } else {
            cslot = (I + 1) * (I + 2) / 2 + I + 1;
        }
        next_tile(I, J, nt);
    }
    if (!ok) {
        // let copies still in flight land before the CTA exits (bounded)
        if (lane == 0) {
            int st = stage;
            uint32_t ph = phase;
            for (int j = k; j < ntile && j < k + kChunkStages; ++j) {
                mbar_wait_bounded(&bars[st], ph, a.err);
                if (++st == kChunkStages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            for (int b = 0; b < kXisBufs; ++b) {
                const unsigned c = *reinterpret_cast<volatile unsigned *>(&issued[b]);
                if (c > 0u) mbar_wait_bounded(&xbar[b], (c - 1u) & 1u, a.err);
            }
        }
        return;
    }
    {
        float *rp = rowp_base + static_cast<int64_t>(4 * (ch.seg0 + seg) + warp) * kTile * D;
        if constexpr (kTall)
            flush_rows_tall<D>(racc, lane, rp);
        else
            flush_rows<D>(racc, lane, rp);
    }
    if (a.far_part && lane == 0) a.far_part[vb * kPairWarps + warp] = n_far;
    // this warp's scalar sums (lane order fixed)
    float sv[3] = {es.x - ec.x, es.y - ec.y, gs - gc};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) sv[i] += __shfl_xor_sync(0xffffffffu, sv[i], o);
    if (lane == 0) {
        float *sp = reinterpret_cast<float *>(a.scal_part) +
                    static_cast<int64_t>(vb * kPairWarps + warp) * kScalarParts;
        sp[kSumE2] = sv[0];
        sp[kSumMDelta] = sv[1];
        sp[kSumLogPhi] = sv[2];
        sp[kSumSpare] = 0.f;
        if (!isfinite(sv[0]) || !isfinite(sv[1]) || !isfinite(sv[2])) atomicOr(a.err, kErrNonfinite);
        if (a.stamps) atomicMax(&a.stamps[1], global_ns());
    }
}

// Shared memory of a CTA with G groups.
template <int D, int G>
constexpr int chunk_cta_smem() {
    return G > 1 ? G * align128(ChunkLayout<D>::kBytes) : ChunkLayout<D>::kBytes;
}

template <int D, bool HO, int G, bool CAP>
cudaError_t launch_one(const PairArgs &a, cudaStream_t s, bool pdl, int smem) {
    cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(pair_chunk_kernel<D, HO, G, CAP>), smem);
    if (e != cudaSuccess) return e;
    if (a.n_strips <= 0) return cudaSuccess;
    e = launch_maybe_pdl(pdl, pair_chunk_kernel<D, HO, G, CAP>, dim3((a.n_strips + G - 1) / G),
                         dim3(kPairThreads * G), smem, s, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int D, bool HO, int G>
cudaError_t launch_cap(const PairArgs &a, cudaStream_t s, bool pdl, int smem) {
    return a.long_runs ? launch_one<D, HO, G, true>(a, s, pdl, smem) : launch_one<D, HO, G, false>(a, s, pdl, smem);
}

template <int D>
cudaError_t launch_d(const PairArgs &a, cudaStream_t s, bool pdl, int smem_min, bool grouped) {
    constexpr int G = chunk_slots_per_sm<D>();
    if (grouped && !a.tile_ho) {
        // held-out passes keep the one-group form (the chunk table serves both:
        // the same chunk slots per SM)
        const int smem = smem_min > chunk_cta_smem<D, G>() ? smem_min : chunk_cta_smem<D, G>();
        return launch_cap<D, false, G>(a, s, pdl, smem);
    }
    const int smem = smem_min > chunk_cta_smem<D, 1>() ? smem_min : chunk_cta_smem<D, 1>();
    return a.tile_ho ? launch_cap<D, true, 1>(a, s, pdl, smem) : launch_cap<D, false, 1>(a, s, pdl, smem);
}

// Chunk slots per SM (groups of four warps that are resident at once): the
// CTAs per SM of the one-group form, or G per CTA of the grouped form.
template <int D>
int blocks_per_sm_d(bool grouped) {
    constexpr int G = chunk_slots_per_sm<D>();
    int nb = 0;
    if (grouped) {
        constexpr int smem = chunk_cta_smem<D, G>();
        const void *fn = reinterpret_cast<const void *>(pair_chunk_kernel<D, false, G, false>);
        if (raise_dyn_smem(fn, smem) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_chunk_kernel<D, false, G, false>,
                                                          kPairThreads * G, smem) != cudaSuccess)
            return 0;
        return nb * G;
    }
    constexpr int smem = chunk_cta_smem<D, 1>();
    const void *fn = reinterpret_cast<const void *>(pair_chunk_kernel<D, false, 1, false>);
    if (raise_dyn_smem(fn, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_chunk_kernel<D, false, 1, false>, kPairThreads,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace

int pair_chunk_smem_bytes(int d) {
    switch (d) {
        case 1: return ChunkLayout<1>::kBytes;
        case 2: return ChunkLayout<2>::kBytes;
        case 3: return ChunkLayout<3>::kBytes;
        case 4: return ChunkLayout<4>::kBytes;
        case 5: return ChunkLayout<5>::kBytes;
        case 6: return ChunkLayout<6>::kBytes;
        case 7: return ChunkLayout<7>::kBytes;
        case 8: return ChunkLayout<8>::kBytes;
        default: return 0;
    }
}

int pair_chunk_blocks_per_sm(int d, bool grouped) {
    switch (d) {
        case 1: return blocks_per_sm_d<1>(grouped);
        case 2: return blocks_per_sm_d<2>(grouped);
        case 3: return blocks_per_sm_d<3>(grouped);
        case 4: return blocks_per_sm_d<4>(grouped);
        case 5: return blocks_per_sm_d<5>(grouped);
        case 6: return blocks_per_sm_d<6>(grouped);
        case 7: return blocks_per_sm_d<7>(grouped);
        case 8: return blocks_per_sm_d<8>(grouped);
        default: return 0;
    }
}

int pair_chunk_groups(int d) { return d <= 4 ? chunk_slots_per_sm<1>() : chunk_slots_per_sm<8>(); }

cudaError_t launch_pair_chunks_f32(const PairArgs &a, int d, cudaStream_t s, bool pdl, int smem_min, bool grouped) {
    switch (d) {
        case 1: return launch_d<1>(a, s, pdl, smem_min, grouped);
        case 2: return launch_d<2>(a, s, pdl, smem_min, grouped);
        case 3: return launch_d<3>(a, s, pdl, smem_min, grouped);
        case 4: return launch_d<4>(a, s, pdl, smem_min, grouped);
        case 5: return launch_d<5>(a, s, pdl, smem_min, grouped);
        case 6: return launch_d<6>(a, s, pdl, smem_min, grouped);
        case 7: return launch_d<7>(a, s, pdl, smem_min, grouped);
        case 8: return launch_d<8>(a, s, pdl, smem_min, grouped);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mds
