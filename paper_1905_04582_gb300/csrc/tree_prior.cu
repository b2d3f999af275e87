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
//
// Work split: one cluster of CTAs per tree.  The host cuts the tree into
// blocks (whole subtrees of at most S internal nodes, spread over the
// cluster's CTAs) and a top (the nodes above them, CTA 0).  Each CTA runs the
// upward pass of its blocks; the block roots' means go to CTA 0 through a
// small exchange array; CTA 0 runs the top up and down; the block roots'
// downward means come back; each CTA runs the downward pass of its blocks.
// Two cluster barriers order the exchanges.  A level costs an FP64
// dependency chain (GB300 runs FP64 at 1/64 of the FP32 rate, with ~64
// cycles of latency per operation) and a barrier, so the levels of one tree
// are as many as its height however it is cut; the cut spreads the wide
// levels and the contrast and gradient sweeps (FP64-throughput bound) over
// the cluster.  Unsequenced items (tips that are roots, variance tau_u) go to
// one more cluster.  Each CTA leaves its sum of the contrast terms; the
// consumer adds them (tree_parts_sum).  FP64 throughout; every sum has a
// fixed order, so results are deterministic.
#include <cstdint>

#include "mds_internal.h"

namespace mds {
namespace {

constexpr int kTreeThreads = 128;  // small enough to share an SM with three pair-pass CTAs
constexpr int kTreeWarps = kTreeThreads / 32;

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Every thread of every CTA of the cluster: writes before, reads after
// (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

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

// Upward mean of child reference c: a node of the part (c >= 0: its message
// or, for a proxy, the exchanged one) or a tip's location (c < 0).
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

// One part's records and messages, wherever they live (shared memory or
// scratch), and its level-synchronous passes.
template <int D>
struct PartView {
    const TreeNode *rec;
    const int32_t *lvs;  // the part's level bounds
    double *up, *dn, *tx, *tdn, *tg;

    __device__ void up_node(int idx) const {
        const int c0 = rec[idx].c0, c1 = rec[idx].c1;
        const double al = rec[idx].alpha;
        double ma[D], mb[D];
        mean_of<D>(up, tx, c0, ma);
        mean_of<D>(up, tx, c1, mb);
#pragma unroll
        for (int c = 0; c < D; ++c) up[static_cast<int64_t>(idx) * D + c] = fma(al, ma[c] - mb[c], mb[c]);
    }

    __device__ void down_node(int idx) const { down_rec(idx, rec[idx]); }

    __device__ void down_rec(int idx, const TreeNode &nd) const {
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
    }

    // levels [0, nlv) with bounds lv (a level ends where the next starts, the
    // last at `end`), upward.  The wide ones (before `small`): a node per
    // thread.  The narrow ones (at most 32 nodes each): a node per lane and a
    // coordinate per warp, so that a level's FP64 operations are spread over
    // the SM's four sub-partitions (an FP64 warp instruction holds its
    // sub-partition's FP64 unit for ~64 cycles however few lanes are active).
    __device__ void run_up(const int32_t *lv, int nlv, int small, int end) const {
        const int tid = threadIdx.x;
        for (int l = 0; l < small; ++l) {
            const int e = l + 1 < nlv ? lv[l + 1] : end;
            for (int idx = lv[l] + tid; idx < e; idx += kTreeThreads) up_node(idx);
            __syncthreads();
        }
        const int lane = tid & 31, warp = tid >> 5;
        for (int l = small; l < nlv; ++l) {
            const int e = l + 1 < nlv ? lv[l + 1] : end;
            const int idx = lv[l] + lane;
            if (idx < e && warp < D) {
                const int c0 = rec[idx].c0, c1 = rec[idx].c1;
                const double al = rec[idx].alpha;
                for (int c = warp; c < D; c += kTreeWarps) {
                    const double ma = c0 >= 0 ? up[static_cast<int64_t>(c0) * D + c] : tx[static_cast<int64_t>(-c0 - 1) * D + c];
                    const double mb = c1 >= 0 ? up[static_cast<int64_t>(c1) * D + c] : tx[static_cast<int64_t>(-c1 - 1) * D + c];
                    up[static_cast<int64_t>(idx) * D + c] = fma(al, ma - mb, mb);
                }
            }
            __syncthreads();
        }
    }

    // the same levels downward (narrow ones first): in the narrow ones a warp
    // takes (child side, coordinate) pairs j = warp, warp + 4, ... of the 2 D
    __device__ void run_down(const int32_t *lv, int nlv, int small, int end) const {
        const int tid = threadIdx.x;
        const int lane = tid & 31, warp = tid >> 5;
        for (int l = nlv - 1; l >= small; --l) {
            const int e = l + 1 < nlv ? lv[l + 1] : end;
            const int idx = lv[l] + lane;
            if (idx < e && warp < 2 * D) {
                const TreeNode &nd = rec[idx];
                for (int j = warp; j < 2 * D; j += kTreeWarps) {
                    const int side = j & 1, c = j >> 1;
                    const int ch = side ? nd.c1 : nd.c0, sib = side ? nd.c0 : nd.c1;
                    const double beta = side ? nd.beta1 : nd.beta0;
                    const double mk = dn[static_cast<int64_t>(idx) * D + c];
                    const double ms = sib >= 0 ? up[static_cast<int64_t>(sib) * D + c] : tx[static_cast<int64_t>(-sib - 1) * D + c];
                    const double o = fma(beta, mk - ms, ms);
                    if (ch < 0) {
                        tdn[static_cast<int64_t>(-ch - 1) * D + c] = o;
                        if (c == 0) tg[-ch - 1] = side ? nd.g1 : nd.g0;
                    } else {
                        dn[static_cast<int64_t>(ch) * D + c] = o;
                    }
                }
            }
            __syncthreads();
        }
        for (int l = small - 1; l >= 0; --l) {
            const int e = l + 1 < nlv ? lv[l + 1] : end;
            for (int idx = lv[l] + tid; idx < e; idx += kTreeThreads) down_node(idx);
            __syncthreads();
        }
    }
};

// grid = (trees + 1 if there are unsequenced items) x cluster CTAs, one
// cluster per tree.  Every thread reaches both cluster barriers of a tree
// cluster; the last cluster (unsequenced items) has none.
template <int D, typename T>
__global__ void __launch_bounds__(kTreeThreads, 1) tree_prior_kernel(const __grid_constant__ TreeArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ double sm[kTreeThreads / 32];
    __shared__ double s_sinv[D * D], s_mu[D];
    const T *x = static_cast<const T *>(a.x);
    const int tid = threadIdx.x;
    double acc = 0.0;  // this thread's quadratic terms (fixed assignment)
    const int cl = a.cluster;
    const int t = blockIdx.x / cl, rank = blockIdx.x % cl;
    if (tid < D * D) s_sinv[tid] = a.sigma_inv[tid];
    if (tid < D) s_mu[tid] = a.mu[tid];
    if (t < a.n_trees) {
        const int p = blockIdx.x;
        const TreePart info = a.parts[p];
        const int m = a.node_off[p + 1] - a.node_off[p];
        const int k = a.tip_off[p + 1] - a.tip_off[p];
        const int nlv = info.nlv_blk + info.nlv_top;
        const int32_t *tips = a.tip_items + a.tip_off[p];
        PartView<D> v;
        double *msg;
        if (a.smem_bytes > 0) {
            // stage the part's records in shared memory with asynchronous
            // copies (8-byte words), in flight while the tips' locations are
            // gathered below
            TreeNode *srec = reinterpret_cast<TreeNode *>(tsm);
            const uint64_t *src = reinterpret_cast<const uint64_t *>(a.nodes + a.node_off[p]);
            uint64_t *dst = reinterpret_cast<uint64_t *>(srec);
            constexpr int kWords = sizeof(TreeNode) / 8;
            const int words = m * kWords;
            for (int i = tid; i < words; i += kTreeThreads) cp_async8(dst + i, src + i);
            v.rec = srec;
            msg = reinterpret_cast<double *>(srec + m);
        } else {
            v.rec = a.nodes + a.node_off[p];
            msg = a.scratch + info.scr_off;
        }
        v.up = msg;                                    // upward means of the part's nodes
        v.dn = v.up + static_cast<int64_t>(m) * D;     // downward means of the part's nodes
        v.tx = v.dn + static_cast<int64_t>(m) * D;     // tip locations
        v.tdn = v.tx + static_cast<int64_t>(k) * D;    // downward means of tips
        v.tg = v.tdn + static_cast<int64_t>(k) * D;    // 1 / downward variance of tips
        {
            constexpr int kB = 8;
            for (int i0 = tid; i0 < k * D; i0 += kTreeThreads * kB) {
                int32_t item[kB];
                T xv[kB];
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    item[b] = i < k * D ? tips[i / D] : -1;
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (item[b] >= 0) xv[b] = x[static_cast<int64_t>(item[b]) * D + i % D];
                }
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    const int i = i0 + b * kTreeThreads;
                    if (item[b] >= 0) v.tx[i] = static_cast<double>(xv[b]);
                }
            }
        }
        // the part's level bounds, read at every level: in shared memory too
        v.lvs = a.lv_start + info.lv0;
        if (a.smem_bytes > 0) {
            int32_t *slv = reinterpret_cast<int32_t *>(v.tg + k);
            for (int i = tid; i < nlv; i += kTreeThreads) cp_async4(slv + i, v.lvs + i);
            v.lvs = slv;
            cp_async_wait_all();
        }
        __syncthreads();
        double *xup = a.xch + info.xch_off;                          // the tree's block roots: upward means
        double *xdn = xup + static_cast<int64_t>(info.n_slots) * D;  // and downward means

        // ---- blocks, upward; the block roots' means to the exchange
        v.run_up(v.lvs, info.nlv_blk, info.small_blk, info.m_blk);
        for (int i = info.exp0 + tid; i < info.exp1; i += kTreeThreads) {
            const int64_t loc = a.exp_loc[i], slot = a.exp_slot[i];
#pragma unroll
            for (int c = 0; c < D; ++c) __stcg(xup + slot * D + c, v.up[loc * D + c]);
        }
        cluster_sync_all();

        // ---- the top (CTA 0): the block roots in as proxies, up, the root,
        // down, the proxies' downward means out
        if (rank == 0) {
            const int64_t prox0 = info.m_blk;
            for (int i = tid; i < info.n_prox * D; i += kTreeThreads) v.up[prox0 * D + i] = __ldcg(xup + i);
            __syncthreads();
            const int32_t *tlv = v.lvs + info.nlv_blk;
            v.run_up(tlv, info.nlv_top, info.small_top, m);
            if (tid == 0) {
                const int64_t r = info.root_loc;
                double dv[D];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    dv[c] = v.up[r * D + c] - s_mu[c];
                    v.dn[r * D + c] = s_mu[c];  // the root's downward mean
                }
                acc = fma(-0.5 * a.root_cinv[t], quad_form<D>(s_sinv, dv), acc);
            }
            __syncthreads();
            v.run_down(tlv, info.nlv_top, info.small_top, m);
            for (int i = tid; i < info.n_prox * D; i += kTreeThreads) __stcg(xdn + i, v.dn[prox0 * D + i]);
        }
        cluster_sync_all();

        // ---- blocks, downward from their roots' exchanged means
        for (int i = info.exp0 + tid; i < info.exp1; i += kTreeThreads) {
            const int64_t loc = a.exp_loc[i], slot = a.exp_slot[i];
#pragma unroll
            for (int c = 0; c < D; ++c) v.dn[loc * D + c] = __ldcg(xdn + slot * D + c);
        }
        __syncthreads();
        v.run_down(v.lvs, info.nlv_blk, info.small_blk, info.m_blk);

        // ---- in parallel: the contrast terms of the part's nodes (not of the
        // proxies: their own parts count them)
        const int top0 = info.m_blk + info.n_prox;
        for (int idx = tid; idx < m; idx += kTreeThreads) {
            if (idx >= info.m_blk && idx < top0) continue;
            double ma[D], mb[D], dv[D];
            mean_of<D>(v.up, v.tx, v.rec[idx].c0, ma);
            mean_of<D>(v.up, v.tx, v.rec[idx].c1, mb);
#pragma unroll
            for (int c = 0; c < D; ++c) dv[c] = ma[c] - mb[c];
            acc = fma(-0.5 * v.rec[idx].cinv, quad_form<D>(s_sinv, dv), acc);
        }
        // ---- in parallel: the tips' gradients -Sigma^-1 (x - m) / v
        for (int tp = tid; tp < k; tp += kTreeThreads) {
            double e[D];
#pragma unroll
            for (int q = 0; q < D; ++q)
                e[q] = v.tx[static_cast<int64_t>(tp) * D + q] - v.tdn[static_cast<int64_t>(tp) * D + q];
            const int64_t item = tips[tp];
            const double g = v.tg[tp];
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
        // unsequenced items: x_i ~ N(mu, tau_u Sigma) on their own, spread
        // over the last cluster's CTAs
        const double g = 1.0 / a.tau_u;
        for (int idx = rank * kTreeThreads + tid; idx < a.n_lone; idx += cl * kTreeThreads) {
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
    // the CTA's sum (the consumers add the parts: tree_parts_sum)
    const double tot = block_sum(acc, sm);
    if (tid == 0) a.part[blockIdx.x] = tot;
}

__global__ void tree_prior_sum_kernel(const double *part, int n, double const_term, double *out) {
    const double v = tree_parts_sum(part, n, const_term);
    if (threadIdx.x == 0) *out = v;
}

template <int D, typename T>
cudaError_t launch_t(const TreeArgs &a, int grid, cudaStream_t s) {
    {
        const cudaError_t e = raise_dyn_smem(reinterpret_cast<const void *>(tree_prior_kernel<D, T>), a.smem_bytes);
        if (e != cudaSuccess) return e;
    }
    // one cluster per tree, at the highest stream priority, so that its CTAs
    // get SMs ahead of a concurrent pair pass's pending CTAs
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTreeThreads);
    cfg.dynamicSmemBytes = static_cast<size_t>(a.smem_bytes);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = static_cast<unsigned>(a.cluster);
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, tree_prior_kernel<D, T>, a);
}

template <int D>
cudaError_t launch_d(const TreeArgs &a, cudaStream_t s) {
    const int grid = (a.n_trees + (a.n_lone > 0 ? 1 : 0)) * a.cluster;
    if (grid <= 0) return cudaErrorInvalidValue;
    const cudaError_t e = a.x_f64 ? launch_t<D, double>(a, grid, s) : launch_t<D, float>(a, grid, s);
    if (e != cudaSuccess || !a.out) return e;
    tree_prior_sum_kernel<<<1, 32, 0, s>>>(a.part, grid, a.const_term, a.out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tree_prior(const TreeArgs &a, int d, cudaStream_t s) {
    if (a.cluster < 1 || a.cluster > kTreeMaxCluster) return cudaErrorInvalidValue;
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
