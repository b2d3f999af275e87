// Phylogenetic Brownian-diffusion prior on the latent locations
// (arXiv:1905.04582, section 2.2: the matrix-normal density of X with the
// tree covariance V and the diffusion covariance Sigma), its log density and
// its gradient in X, by message passing on the forest: O(N D^2) work.
//
// Section 2.3 notes that the density is computable in time linear in N by
// post-order traversals of the trees instead of factorising V (O(N^3)).
// Gaussian messages on a tree carry a mean and a variance scalar; the
// variances depend on the tree alone (branch lengths, tau0), not on X, so
// the host computes them once per tree (mds_set_tree_prior) and folds them
// into per-node weights.  Per evaluation the device moves only means:
//  - post-order, level by level (height = 1 + the children's largest): node
//    k with children a, b sends up m_k = alpha_k m_a + (1 - alpha_k) m_b and
//    adds the contrast term -1/2 (m_a - m_b)^T Sigma^-1 (m_a - m_b) c_k,
//    c_k = 1 / (v_a + t_a + v_b + t_b); a tip sends its location.  The root
//    adds -1/2 (m_root - mu)^T Sigma^-1 (m_root - mu) / (v_root + tau0).
//    With the constant log-determinant terms (host) these N contrasts sum to
//    the log density (each contrast carries -1/2 log|Sigma|, and their
//    variances multiply to |V|).
//  - pre-order, level by level from the roots (downward mean of a root: mu):
//    child c of node k with sibling s receives
//    m_c = beta_c m_k + (1 - beta_c) m_s (precision weights of k's downward
//    message and s's upward message through its branch).  At a tip the
//    downward message is the law of x_c given every other item,
//    N(m_c, v_c Sigma), so d log p / d x_c = -Sigma^-1 (x_c - m_c) / v_c.
// One CTA per tree keeps the tree's node records, messages and tip
// locations in shared memory (global scratch when a tree is too large);
// unsequenced items (tips that are roots, variance tau_u) get one more CTA.
// FP64 throughout; every sum has a fixed order, so results are
// deterministic.
#include <cstdint>

#include "mds_internal.h"

namespace mds {
namespace {

constexpr int kTreeThreads = 512;

template <int D>
__device__ __forceinline__ double quad_form(const double *sinv, const double (&v)[D]) {
    double q = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < D; ++c) t = fma(sinv[r * D + c], v[c], t);
        q = fma(v[r], t, q);
    }
    return q;
}

// Upward mean of child reference c: an internal node's message (c >= 0) or
// a tip's location (c < 0).
template <int D>
__device__ __forceinline__ void mean_of(const double *up, const double *tx, int c, double (&m)[D]) {
    const double *src = c >= 0 ? up + static_cast<int64_t>(c) * D : tx + static_cast<int64_t>(-c - 1) * D;
#pragma unroll
    for (int k = 0; k < D; ++k) m[k] = src[k];
}

__device__ __forceinline__ double block_sum(double v, double *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kTreeThreads / 32; ++w) t += sm[w];
    return t;  // valid in thread 0
}

// The level-synchronous traversals move only means (a few dependent FP64
// operations per node, so each level costs little more than a barrier); the
// quadratic forms of the contrasts and the tips' gradients depend on the
// finished messages alone and are computed afterwards by every thread in
// parallel.
template <int D, typename T>
__global__ void __launch_bounds__(kTreeThreads) tree_prior_kernel(const __grid_constant__ TreeArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ double sm[kTreeThreads / 32];
    __shared__ double s_sinv[D * D], s_mu[D];
    const T *x = static_cast<const T *>(a.x);
    const int tid = threadIdx.x;
    double acc = 0.0;  // this thread's quadratic terms (fixed assignment)
    const int t = blockIdx.x;
    if (tid < D * D) s_sinv[tid] = a.sigma_inv[tid];
    if (tid < D) s_mu[tid] = a.mu[tid];
    if (t < a.n_trees) {
        const int m = a.node_off[t + 1] - a.node_off[t];
        const int k = a.tip_off[t + 1] - a.tip_off[t];
        const int32_t *tips = a.tip_items + a.tip_off[t];
        const TreeNode *rec;
        double *up;
        if (a.smem_bytes > 0) {
            // stage the tree's records in shared memory, in batches of
            // independent loads (the copy is latency-bound)
            TreeNode *srec = reinterpret_cast<TreeNode *>(tsm);
            const uint64_t *src = reinterpret_cast<const uint64_t *>(a.nodes + a.node_off[t]);
            uint64_t *dst = reinterpret_cast<uint64_t *>(srec);
            constexpr int kWords = sizeof(TreeNode) / 8;
            constexpr int kB = 8;
            const int words = m * kWords;
            for (int i0 = tid; i0 < words; i0 += kTreeThreads * kB) {
                uint64_t w[kB];
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (i < words) w[b] = src[i];
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (i < words) dst[i] = w[b];
                }
            }
            rec = srec;
            up = reinterpret_cast<double *>(srec + m);
        } else {
            rec = a.nodes + a.node_off[t];
            up = a.scratch + a.scr_off[t];
        }
        double *dn = up + static_cast<int64_t>(m) * D;   // downward means of internal nodes
        double *tx = dn + static_cast<int64_t>(m) * D;   // tip locations
        double *tdn = tx + static_cast<int64_t>(k) * D;  // downward means of tips
        double *tg = tdn + static_cast<int64_t>(k) * D;  // 1 / downward variance of tips
        {
            constexpr int kB = 8;
            for (int i0 = tid; i0 < k * D; i0 += kTreeThreads * kB) {
                int32_t item[kB];
                T v[kB];
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    item[b] = i < k * D ? tips[i / D] : -1;
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (item[b] >= 0) v[b] = x[static_cast<int64_t>(item[b]) * D + i % D];
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (item[b] >= 0) tx[i] = static_cast<double>(v[b]);
                }
            }
        }
        // the tree's level bounds, read at every level: in shared memory too
        const int lv0 = a.tree_lv[t], lv1 = a.tree_lv[t + 1];
        const int32_t *lvs = a.lv_start + lv0;
        if (a.smem_bytes > 0) {
            int32_t *slv = reinterpret_cast<int32_t *>(tg + k);
            for (int i = tid; i < lv1 - lv0; i += kTreeThreads) slv[i] = lvs[i];
            lvs = slv;
        }
        __syncthreads();
        // ---- post-order: upward means, level by level (lvs relative to lv0).
        // Levels from `small` up hold at most 32 nodes each (the top of the
        // tree): warp 0 alone runs them, with warp-level barriers.
        const int nlv = lv1 - lv0;
        const int small = a.tree_small[t];
        auto up_node = [&](int idx) {
            const int c0 = rec[idx].c0, c1 = rec[idx].c1;
            const double al = rec[idx].alpha;
            double ma[D], mb[D];
            mean_of<D>(up, tx, c0, ma);
            mean_of<D>(up, tx, c1, mb);
#pragma unroll
            for (int c = 0; c < D; ++c) up[static_cast<int64_t>(idx) * D + c] = fma(al, ma[c] - mb[c], mb[c]);
        };
        for (int lv = 0; lv < small; ++lv) {
            const int end = lv + 1 < nlv ? lvs[lv + 1] : m;
            for (int idx = lvs[lv] + tid; idx < end; idx += kTreeThreads) up_node(idx);
            __syncthreads();
        }
        if (tid < 32) {
            for (int lv = small; lv < nlv; ++lv) {
                const int end = lv + 1 < nlv ? lvs[lv + 1] : m;
                const int idx = lvs[lv] + tid;
                if (idx < end) up_node(idx);
                __syncwarp();
            }
            // the root's downward mean is mu
            if (tid < D) dn[static_cast<int64_t>(m - 1) * D + tid] = s_mu[tid];
            __syncwarp();
        }
        // ---- pre-order: downward means, from the root down (the small
        // levels by warp 0 again, then the rest by the block)
        auto down_node = [&](int idx) {
                const TreeNode nd = rec[idx];
                double mk[D], m0[D], m1[D];
#pragma unroll
                for (int c = 0; c < D; ++c) mk[c] = dn[static_cast<int64_t>(idx) * D + c];
                mean_of<D>(up, tx, nd.c0, m0);
                mean_of<D>(up, tx, nd.c1, m1);
                // child 0 (its sibling is child 1) and child 1
                double *o0 = nd.c0 < 0 ? tdn + static_cast<int64_t>(-nd.c0 - 1) * D : dn + static_cast<int64_t>(nd.c0) * D;
                double *o1 = nd.c1 < 0 ? tdn + static_cast<int64_t>(-nd.c1 - 1) * D : dn + static_cast<int64_t>(nd.c1) * D;
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    o0[c] = fma(nd.beta0, mk[c] - m1[c], m1[c]);
                    o1[c] = fma(nd.beta1, mk[c] - m0[c], m0[c]);
                }
                if (nd.c0 < 0) tg[-nd.c0 - 1] = nd.g0;
                if (nd.c1 < 0) tg[-nd.c1 - 1] = nd.g1;
        };
        if (tid < 32) {
            for (int lv = nlv - 1; lv >= small; --lv) {
                const int end = lv + 1 < nlv ? lvs[lv + 1] : m;
                const int idx = lvs[lv] + tid;
                if (idx < end) down_node(idx);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int lv = small - 1; lv >= 0; --lv) {
            const int end = lv + 1 < nlv ? lvs[lv + 1] : m;
            for (int idx = lvs[lv] + tid; idx < end; idx += kTreeThreads) down_node(idx);
            __syncthreads();
        }
        // ---- in parallel: the contrast terms of every node and the root term
        for (int idx = tid; idx < m; idx += kTreeThreads) {
            double ma[D], mb[D], dv[D];
            mean_of<D>(up, tx, rec[idx].c0, ma);
            mean_of<D>(up, tx, rec[idx].c1, mb);
#pragma unroll
            for (int c = 0; c < D; ++c) dv[c] = ma[c] - mb[c];
            acc = fma(-0.5 * rec[idx].cinv, quad_form<D>(s_sinv, dv), acc);
        }
        if (tid == 0) {
            double dv[D];
#pragma unroll
            for (int c = 0; c < D; ++c) dv[c] = up[static_cast<int64_t>(m - 1) * D + c] - s_mu[c];
            acc = fma(-0.5 * a.root_cinv[t], quad_form<D>(s_sinv, dv), acc);
        }
        // ---- in parallel: the tips' gradients -Sigma^-1 (x - m) / v
        for (int tp = tid; tp < k; tp += kTreeThreads) {
            double e[D];
#pragma unroll
            for (int q = 0; q < D; ++q) e[q] = tx[static_cast<int64_t>(tp) * D + q] - tdn[static_cast<int64_t>(tp) * D + q];
            const int64_t item = tips[tp];
            const double g = tg[tp];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                double sg = 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) sg = fma(s_sinv[r * D + q], e[q], sg);
                a.grad[item * D + r] = -sg * g;
            }
        }
    } else {
        __syncthreads();  // Sigma^-1 and mu staged
        // unsequenced items: x_i ~ N(mu, tau_u Sigma) on their own
        const double g = 1.0 / a.tau_u;
        for (int idx = tid; idx < a.n_lone; idx += kTreeThreads) {
            const int64_t i = a.lone[idx];
            double e[D];
#pragma unroll
            for (int q = 0; q < D; ++q) e[q] = static_cast<double>(x[i * D + q]) - s_mu[q];
            double qf = 0.0;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                double sg = 0.0;
#pragma unroll
                for (int q = 0; q < D; ++q) sg = fma(s_sinv[r * D + q], e[q], sg);
                qf = fma(e[r], sg, qf);
                a.grad[i * D + r] = -sg * g;
            }
            acc = fma(-0.5 * g, qf, acc);
        }
    }
    const double tot = block_sum(acc, sm);
    if (tid == 0) a.part[t] = tot;
}

// Fixed-order sum of the per-CTA parts plus the constant (log-determinant)
// terms.
__global__ void tree_prior_final_kernel(const double *part, int n_parts, double const_term, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = const_term;
        for (int i = 0; i < n_parts; ++i) s += part[i];
        *out = s;
    }
}

template <int D, typename T>
cudaError_t launch_t(const TreeArgs &a, int grid, cudaStream_t s) {
    static int attr_bytes = 0;  // per instantiation, raised once as needed
    if (a.smem_bytes > attr_bytes) {
        const cudaError_t e =
            cudaFuncSetAttribute(tree_prior_kernel<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes);
        if (e != cudaSuccess) return e;
        attr_bytes = a.smem_bytes;
    }
    // the highest stream priority, so that its few CTAs get SMs ahead of a
    // concurrent pair pass's pending CTAs
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTreeThreads);
    cfg.dynamicSmemBytes = static_cast<size_t>(a.smem_bytes);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tree_prior_kernel<D, T>, a);
}

template <int D>
cudaError_t launch_d(const TreeArgs &a, cudaStream_t s) {
    const int grid = a.n_trees + (a.n_lone > 0 ? 1 : 0);
    if (grid > 0) {
        const cudaError_t e = a.x_f64 ? launch_t<D, double>(a, grid, s) : launch_t<D, float>(a, grid, s);
        if (e != cudaSuccess) return e;
    }
    tree_prior_final_kernel<<<1, 32, 0, s>>>(a.part, grid, a.const_term, a.out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tree_prior(const TreeArgs &a, int d, cudaStream_t s) {
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
