/*
 * mds.h -- C ABI of the GB300 (sm_103a) library for the hot path of Bayesian
 * multidimensional scaling fitted by Hamiltonian Monte Carlo
 * (Holbrook et al., "Massive parallelization boosts big Bayesian
 * multidimensional scaling", arXiv:1905.04582).
 *
 * Model (section 2.1, Eq. (1)-(2)).  N items with latent locations
 * x_i in R^D, observed dissimilarities y_ij >= 0 (i != j, symmetric),
 * y_ij ~ N(delta_ij, sigma^2) truncated to y_ij > 0, delta_ij = ||x_i - x_j||.
 * The library evaluates, over the M = N(N-1)/2 pairs i < j,
 *
 *   L(X, sigma) = -M log sigma - sum_{i<j} r_ij,
 *   r_ij        = (y_ij - delta_ij)^2 / (2 sigma^2) + log Phi(delta_ij / sigma),
 *   dL/dx_i     = -sum_{j != i} [ (delta_ij - y_ij)/sigma^2
 *                                 + phi(delta_ij/sigma) / (sigma Phi(delta_ij/sigma)) ]
 *                              (x_i - x_j) / delta_ij                  (Eq. (9)),
 *   dL/dsigma   = -M/sigma + sum_{i<j} [ (y_ij - delta_ij)^2 / sigma^3
 *                                 + phi(z_ij) delta_ij / (sigma^2 Phi(z_ij)) ]
 *                 (Eq. (2) differentiated in sigma; not printed in the paper),
 *
 * in ONE fused pass over the pairs (section 2.5: the per-pair terms are a
 * transformation, their sums a reduction, and nothing per pair is stored).
 * L keeps the sigma^(-M) factor of Eq. (2) and drops the (2 pi)^(-M/2)
 * constant.  Coincident points (delta_ij = 0) contribute r_ij at delta = 0
 * and nothing to the gradient.
 *
 * HMC (section 2.3, Eq. (6)-(8)) uses the identity mass matrix: the target is
 * log pi(X) = L(X, sigma) - (lambda/2) ||X||_F^2 (lambda >= 0, default 0),
 * H = -log pi(X) + p^T p / 2, leapfrog steps
 *   p += eps/2 grad;  x += eps p;  p += eps/2 grad,
 * and a proposal is accepted when log u < H(start) - H(end).
 *
 * Conventions for every call:
 *   - Return value: MDS_OK (0) or an MDS_ERR_* code; mds_last_error() then
 *     gives a one-line message.  No call aborts the process or throws across
 *     the ABI.  After MDS_ERR_CUDA the context must be destroyed.
 *   - Sizes and offsets are 64-bit.  All matrices are row-major, contiguous.
 *   - `where` says whether a caller pointer is host (MDS_HOST) or device
 *     (MDS_DEVICE) memory.  Caller buffers are never retained: inputs are
 *     copied in, outputs copied out; the caller keeps ownership.
 *   - Work is enqueued on the context's stream (mds_set_stream; default: the
 *     legacy default stream).  Calls that return host values synchronise that
 *     stream before returning; calls whose outputs are device buffers are
 *     asynchronous.
 *   - One context per host thread; contexts are independent.
 *   - Results are bitwise reproducible for a fixed context configuration
 *     (precision, tile strip length): every reduction has a fixed order and
 *     no floating-point atomics are used.
 */
#ifndef MDS_H_
#define MDS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define MDS_OK 0
#define MDS_ERR_INVALID_ARG 1 /* bad pointer, size, enum, or non-finite / negative input */
#define MDS_ERR_STATE 2       /* call order: e.g. evaluation before mds_set_data */
#define MDS_ERR_CUDA 3        /* a CUDA runtime call failed; destroy the context */
#define MDS_ERR_OOM 4         /* device or host allocation failed */
#define MDS_ERR_TIMEOUT 5     /* a bounded device-side wait gave up */
#define MDS_ERR_NONFINITE 6   /* a result was NaN/Inf (reported, not hidden) */
#define MDS_ERR_UNSUPPORTED 7 /* no sm_100-family GPU, or a size beyond the limits */
#define MDS_ERR_EXCHANGE 8    /* the all-gather of a sharded evaluation failed */

/* mds_create flags: arithmetic of the pair pass. */
#define MDS_PREC_FP32C 0u /* FP32 per-pair math, compensated FP32 partials reduced in FP64 */
#define MDS_PREC_FP64 1u  /* FP64 per-pair math and sums (the plain FP64 GPU path) */

/* Element types of caller buffers. */
#define MDS_F32 0
#define MDS_F64 1

/* Where a caller buffer lives. */
#define MDS_HOST 0
#define MDS_DEVICE 1

/* Layouts of Y for mds_set_data. */
#define MDS_Y_FULL 0         /* N x N row-major, leading dimension ld >= N */
#define MDS_Y_PACKED_UPPER 1 /* M entries (0,1),(0,2),...,(0,N-1),(1,2),...,(N-2,N-1) */

/* Limits. */
#define MDS_MAX_D 8

typedef struct mds_ctx mds_ctx;

/* Create a context for N items in D latent dimensions (2 <= N <= 2^31 - 1,
 * 1 <= D <= MDS_MAX_D) on the current CUDA device.  flags: MDS_PREC_FP32C
 * (default) or MDS_PREC_FP64.  Allocates the device state (tile-packed Y:
 * about 4 M bytes; locations, momenta, gradients and partial sums: O(N D)
 * plus about D/16 of the Y bytes).  *out receives the context, owned by the
 * library until mds_destroy.  Errors: INVALID_ARG, UNSUPPORTED (device is not
 * compute capability 10.x), OOM, CUDA. */
int mds_create(int64_t n, int32_t d, uint32_t flags, mds_ctx **out);

/* Free the context and all its device memory.  NULL is allowed. */
int mds_destroy(mds_ctx *ctx);

/* Enqueue all later work of `ctx` on `stream` (a cudaStream_t, e.g. torch's
 * current stream); NULL selects the legacy default stream. */
int mds_set_stream(mds_ctx *ctx, void *stream);

/* Set the observed dissimilarities Y (section 2.1; symmetric, section 2.2).
 * dtype MDS_F32 or MDS_F64; layout MDS_Y_FULL (ld = row stride in elements,
 * ld >= N; only the strict upper triangle i < j is read, the diagonal and the
 * lower triangle are ignored) or MDS_Y_PACKED_UPPER (ld ignored).  Values are
 * rounded once to FP32 and re-packed into the library's tile layout.
 * Errors: INVALID_ARG if any read entry is negative, NaN or Inf (the message
 * names the first offending (i, j)); the previous Y stays in place then. */
int mds_set_data(mds_ctx *ctx, const void *y, int dtype, int layout, int64_t ld, int where);

/* Set the latent locations X (N x D row-major, dtype MDS_F32 or MDS_F64).
 * The FP32C path keeps X in FP32, the FP64 path in FP64.  Errors:
 * INVALID_ARG for a non-finite entry. */
int mds_set_locations(mds_ctx *ctx, const void *x, int dtype, int where);

/* Copy the current locations out (N x D row-major). */
int mds_get_locations(mds_ctx *ctx, void *x, int dtype, int where);

/* Set sigma (> 0, finite; the FP32C path accepts 1e-6 <= sigma <= 1e6). */
int mds_set_sigma(mds_ctx *ctx, double sigma);

/* Set the isotropic Gaussian prior precision lambda >= 0 of the HMC target
 * (default 0: the target is the likelihood alone). */
int mds_set_prior(mds_ctx *ctx, double lambda);

/* Log-likelihood L(X, sigma) of Eq. (2) (incl. -M log sigma).  sum_r
 * (optional) receives sum_{i<j} r_ij.  Synchronises.  Errors: STATE before
 * set_data / set_locations / set_sigma; NONFINITE. */
int mds_log_likelihood(mds_ctx *ctx, double *loglik, double *sum_r);

/* One fused pass: L (optional), the gradient dL/dX of Eq. (9) into `grad`
 * (N x D row-major, dtype MDS_F32/MDS_F64, host or device; optional) and
 * dL/dsigma (optional).  Synchronises when any output is on the host. */
int mds_gradient(mds_ctx *ctx, double *loglik, void *grad, int dtype, int where,
                 double *dlogl_dsigma);

/* Set / get the HMC momentum p (N x D). */
int mds_set_momentum(mds_ctx *ctx, const void *p, int dtype, int where);
int mds_get_momentum(mds_ctx *ctx, void *p, int dtype, int where);

/* Advance (x, p) in place by n_steps >= 0 leapfrog steps of size eps
 * (section 2.3, Eq. (7) with M = I), entirely on the device.  p0 (optional,
 * N x D) replaces the momentum first.  dh (optional) receives
 * H(end) - H(start) in FP64.  No Metropolis step.  Synchronises when dh is
 * requested. */
int mds_leapfrog(mds_ctx *ctx, int n_steps, double eps, const void *p0, int p0_dtype,
                 int p0_where, double *dh);

/* Statistics of an mds_hmc run. */
typedef struct mds_hmc_stats {
    int64_t iterations; /* iterations run */
    int64_t accepted;   /* proposals accepted */
    double last_dh;     /* H(end) - H(start) of the last iteration */
    double last_loglik; /* L at the state after the last iteration */
} mds_hmc_stats;

/* n_iter HMC iterations of n_steps leapfrog steps each (step size eps), on
 * the device, captured once into a CUDA graph and replayed.  Momenta and
 * uniforms come from the Philox4x32-10 stream keyed by `seed` (counter
 * layout: element e of iteration t uses counter (e/4, t0+t, chain, 0), the
 * uniform counter (0, t0+t, chain, 1), chain = 0, t0 = iterations run so far
 * by this context), unless p_all (n_iter x N x D, FP64, host) and u_all
 * (n_iter uniforms in (0,1), FP64, host) are given, which makes runs
 * comparable with an external implementation.  accepted (optional, n_iter
 * ints, host) and dh (optional, n_iter doubles, host) receive per-iteration
 * results.  Synchronises.  Errors: NONFINITE if an energy was not finite (the
 * proposal is then rejected and the run continues). */
int mds_hmc(mds_ctx *ctx, int n_iter, int n_steps, double eps, uint64_t seed, const double *p_all,
            const double *u_all, int *accepted, double *dh, mds_hmc_stats *stats);

/* Asynchronous HMC (section 2.3 of arXiv:1905.04582, Eq. (6)-(8), as mds_hmc, Philox
 * momenta only): queue n_iter iterations on the context's stream and return
 * without waiting for the device.  The chain state stays on the device; the
 * per-iteration decisions and H1 - H0 accumulate there (moved to the host
 * automatically when the queue outgrows its buffer, which then waits once).
 * Any number of enqueue calls may precede one mds_hmc_collect.  mds_hmc
 * refuses to run (STATE) while queued results are uncollected.  Errors found
 * by the device during queued iterations are reported by the collect. */
int mds_hmc_enqueue(mds_ctx *ctx, int n_iter, int n_steps, double eps, uint64_t seed);

/* Wait for the queued iterations and return their results in queue order:
 * accepted (optional, int32, host) and dh (optional, FP64, host) receive up
 * to `cap` entries (the rest are dropped), *count (optional) the number of
 * iterations collected, stats (optional) their totals and the state after
 * the last one.  One device-to-host read-back.  Errors: NONFINITE (an energy
 * was not finite; that proposal was rejected), INVALID_ARG (the locations
 * left the FP32C range), TIMEOUT, CUDA. */
int mds_hmc_collect(mds_ctx *ctx, int64_t cap, int32_t *accepted, double *dh, int64_t *count,
                    mds_hmc_stats *stats);

/* The current sigma (set by mds_set_sigma or moved by mds_sigma_mh). */
int mds_get_sigma(const mds_ctx *ctx, double *sigma);

/* Update sigma given X: the sigma^2 step of the paper's Gibbs scheme
 * (section 3) with the prior sigma^-2 ~ Gamma(shape, rate) (section 2.2).
 * The Phi term of Eq. (2) makes that full conditional non-standard, so each
 * of the n_iter updates is a random-walk Metropolis step on tau = log sigma:
 *   tau' = tau + step z,  accepted iff  log u < P(tau') - P(tau),
 *   P(tau) = L(X, sigma) + shape log(sigma^-2) - rate sigma^-2
 * (L of Eq. (2) over the training pairs; the Jacobian of the log scale is
 * included).  Each proposal costs one fused pass.  z_all / u_all (host,
 * n_iter each, u in (0,1)) inject the draws; otherwise update t of the
 * context uses the Philox4x32-10 block at counter (0, t, 0, 2) keyed by
 * `seed` (z by Box-Muller from words 0 and 1, u from word 2), t counting
 * every update drawn so far.  accepted (optional, n_iter int32, host).
 * Proposals outside the FP32C range of sigma are rejected.  Synchronises.
 * Errors: INVALID_ARG, STATE (no data/locations/sigma; queued HMC
 * iterations), NONFINITE, CUDA. */
int mds_sigma_mh(mds_ctx *ctx, int n_iter, double step, double shape, double rate, uint64_t seed,
                 const double *z_all, const double *u_all, int32_t *accepted);

/* ------------------------------------------------------------------------
 * Cross-validation (section 2.4 "Model selection" of arXiv:1905.04582).  A
 * fold holds out a set of observations y_ij; the model is trained on the rest
 * and scored on the held-out pairs by the log pointwise predictive density,
 * estimated from S posterior draws (X_s, sigma_s) as
 *   lpd-hat = sum_{held-out i<j} log( (1/S) sum_s p(y_ij | X_s, sigma_s) ),
 * p the truncated-normal density of Eq. (1):
 *   p(y | delta, sigma) = phi((y - delta) / sigma) / (sigma Phi(delta / sigma)), y > 0.
 * (The paper's formula also multiplies each density by the posterior density
 * of its draw; with draws taken from that posterior the plain average is the
 * standard estimate, which is the one computed.)
 * ------------------------------------------------------------------------ */

/* Hold out the pairs pairs[2k], pairs[2k+1] (k < n_pairs; int64, host; each
 * pair of distinct items in [0, N), in either order; duplicates count once):
 * from now on L, dL/dX, dL/dsigma, leapfrog and HMC use the other pairs only,
 * with M = the number of those (the training likelihood of the fold).  The
 * held-out y are kept aside for the predictive density; the lpd-hat
 * accumulators restart.  n_pairs = 0 (pairs may be NULL) restores every
 * pair.  mds_set_data drops the fold.  Errors: INVALID_ARG (a bad pair),
 * STATE (no data; queued HMC iterations), OOM, CUDA. */
int mds_set_heldout(mds_ctx *ctx, const int64_t *pairs, int64_t n_pairs);

/* Number of distinct held-out pairs of the current fold. */
int mds_heldout_count(const mds_ctx *ctx, int64_t *count);

/* Add the current state (X, sigma) as one posterior draw: the density p of
 * every held-out pair enters its running average (FP64, per pair a running
 * log-sum-exp, so no density underflows).  Synchronises.  Errors: STATE (no
 * fold, locations or sigma; queued HMC iterations), NONFINITE, CUDA. */
int mds_lpd_accumulate(mds_ctx *ctx);

/* lpd-hat over the draws accumulated so far (fixed-order FP64 sum over the
 * held-out pairs) into *lpd, and the number of draws S into *draws
 * (optional).  Errors: STATE (no draw yet), CUDA. */
int mds_lpd(mds_ctx *ctx, double *lpd, int64_t *draws);

/* Forget the accumulated draws (the fold stays). */
int mds_lpd_reset(mds_ctx *ctx);

/* ------------------------------------------------------------------------
 * Locality order and the Phi-term cut-off.  The paper's pass (section 2.5)
 * evaluates Phi for every pair, and calls it the rate-limiting cost of the
 * likelihood and gradient (sections 2.3 and 4, where dropping the truncation
 * term speeds the evaluation up several-fold).  For z = delta/sigma >= 8,
 * log(1/Phi(z)) < 6.3e-16 and phi(z)/Phi(z) < 5.1e-15: far below the FP32
 * rounding of the other terms.  The FP32C pass therefore skips the Phi terms
 * for a warp's block of 64 x 8 pairs when a bounding-box test shows every
 * pair of the block at z >= z_c.  Such blocks exist only when items that lie
 * close in the latent space also sit close in the item order; mds_reorder
 * arranges that inside the library.  Results stay within the FP32C tolerances
 * either way; only the speed changes.
 * ------------------------------------------------------------------------ */

/* Measured ceiling of the FP32C pass's per-pair arithmetic on this GPU:
 * pairs/s of the pass's own per-pair bodies (far != 0: the body without the
 * Phi terms that far warp blocks take; 0: the full body of Eq. (2) and its
 * gradient) run on operands held in registers (four row pairs against two
 * columns per round, as the tiles call them), at the pass's occupancy, over
 * every SM, with no memory traffic, no tile epilogue and no reductions.  The
 * context's sigma and D set the constants and the body; nothing of its state
 * is read or changed.  Synchronises (about 10^10 pair evaluations, tens of
 * ms).  Errors: INVALID_ARG (NULL output), STATE (FP64 context, no sigma,
 * HMC iterations queued), OOM, CUDA. */
int mds_pair_body_ceiling(mds_ctx *ctx, int32_t far, double *pairs_per_s);

/* Host-only (no GPU needed): a locality-preserving order of N points x
 * (N x D row-major, FP64, finite): recursive bisection of the widest
 * coordinate, cut at multiples of 64 items, so that each run of 64
 * consecutive items of the order is one compact cell.  perm[s] receives the
 * item placed at position s (a permutation of 0..N-1).  Deterministic.
 * Errors: INVALID_ARG (sizes, NULL pointers, non-finite x). */
int mds_locality_order(int64_t n, int32_t d, const double *x, int32_t *perm);

/* Re-arrange the context's tile layouts (Y, split locations, partial sums)
 * in the locality order of the current locations (mds_locality_order).  Every
 * API array keeps the caller's item order: locations, gradients, momenta,
 * injected draws, held-out pairs and the Philox draws of item k are those of
 * the unordered context; sums are taken in another order, so results agree
 * within rounding, not bitwise.  It can be called again later (e.g. after a
 * burn-in moved the points).  Needs data and locations; call it before
 * mds_set_heldout (STATE otherwise) and with no HMC iterations queued.
 * Re-packs Y on the device (a second copy of Y exists briefly).  Errors:
 * STATE, OOM, CUDA. */
int mds_reorder(mds_ctx *ctx);

/* Diagnostics: run one evaluation pass and report how many warp blocks
 * (64 x 8 pairs; total = 8 per 64 x 64 tile) skipped the Phi terms.
 * Synchronises.  Errors: STATE (as mds_gradient). */
int mds_far_blocks(mds_ctx *ctx, int64_t *far, int64_t *total);

/* The current order: perm[s] = item at slot s (N entries; identity before
 * mds_reorder). */
int mds_get_order(const mds_ctx *ctx, int32_t *perm);

/* Cut-off z_c of the Phi-term skip of the FP32C pass: 0 turns it off, else
 * z_c >= 8 (default 8).  The FP64 path evaluates Phi for every pair.
 * Errors: INVALID_ARG for 0 < z < 8 or a non-finite z. */
int mds_set_tail_cutoff(mds_ctx *ctx, double z);

/* ------------------------------------------------------------------------
 * Phylogenetic Brownian-diffusion prior (section 2.2).  The items are the
 * tips of a forest: nodes 0..N-1 are the tips (item i is node i), nodes
 * N..n_nodes-1 internal, each with exactly two children; parent[k] = -1
 * marks a root, and a tip that is a root is an unsequenced item.  A tree's
 * root value is N(mu, tau0 Sigma), each child N(parent value,
 * length[k] Sigma); an unsequenced item is N(mu, tau_u Sigma).  Then X is
 * matrix normal with row covariance V (V_ij = tau0 + root-to-MRCA time within
 * a tree, V_ii = tau0 + root-to-tip time, tau_u for an unsequenced item, 0
 * across trees) and column covariance Sigma (D x D):
 *   log p(X) = -1/2 tr[Sigma^-1 (X - 1 mu^T)^T V^-1 (X - 1 mu^T)]
 *              - (N D/2) log 2 pi - (N/2) log|Sigma| - (D/2) log|V|.
 * ------------------------------------------------------------------------ */

/* Set the forest and its parameters (all host arrays, copied): parent and
 * length [n_nodes] (length > 0 off the roots), sigma_mat D x D symmetric
 * positive definite, mu [D], tau0 > 0, tau_u > 0.  N <= n_nodes <= 2N - 1.
 * The message variances of the traversals depend on the forest alone and are
 * computed here, once.  n_nodes = 0 (or parent NULL) removes the prior.
 * Errors: INVALID_ARG (not a binary forest over the N tips, a length <= 0,
 * Sigma not SPD, ...), STATE (HMC iterations queued), OOM, CUDA. */
int mds_set_tree_prior(mds_ctx *ctx, int64_t n_nodes, const int64_t *parent, const double *length,
                       const double *sigma_mat, const double *mu, double tau0, double tau_u);

/* Host-only (no GPU needed): checks the work split that mds_set_tree_prior
 * would use for this forest (parent / length as there, over n tips, for D
 * coordinates).  Each tree is cut into blocks (the largest subtrees of at
 * most S = ceil(m / 4C) internal nodes, m the tree's internal nodes, C the
 * CTAs of its cluster) and a top (the nodes above them); the device
 * evaluates a tree with one cluster: each CTA its blocks upward, CTA 0 the
 * top up and down, each CTA its blocks downward.  The check verifies that
 * every node and tip of every tree lies in exactly one part, that child
 * references, levels, block-root exchanges and buffer offsets are
 * consistent.  stats (optional, 8 entries): cluster size C, parts, the
 * longest chain of levels (2 x (block + top levels)), the largest part's
 * shared-memory bytes, block roots in all, the largest top, the largest
 * part's block nodes, trees.  Errors: INVALID_ARG (not a binary forest, as
 * mds_set_tree_prior), STATE (the split is inconsistent: a library defect);
 * the message from mds_last_error(NULL). */
int mds_tree_plan_check(int64_t n, int64_t n_nodes, const int64_t *parent, const double *length, int32_t d,
                        int64_t *stats);

/* log p(X) of the prior at the current locations (optional) and its
 * gradient d log p / dX = -V^-1 (X - 1 mu^T) Sigma^-1 into `grad` (N x D,
 * optional, dtype and where as in mds_gradient), by two level-synchronous
 * traversals of each tree on the device, one cluster of CTAs per tree (the
 * split of mds_tree_plan_check; O(N D^2), FP64; section 2.3 cites the
 * linear-time post-order evaluation).  Synchronises when an output is
 * on the host.  Errors: STATE (no prior or no locations). */
int mds_tree_prior(mds_ctx *ctx, double *logp, void *grad, int dtype, int where);

/* Single-item random-walk Metropolis, the prior-art sampler of section 2.3
 * (a random-walk kernel applied to one x_i at a time; moving x_i changes only
 * its N - 1 terms r_ij).  Proposal t moves item i_t to x_i + step z_t and is
 * accepted iff log u_t < log pi(X') - log pi(X), log pi = L(X, sigma) -
 * (lambda/2) ||X||^2 (mds_set_prior; no tree prior), with
 * L(X') - L(X) = sum_{j != i} [r_ij(x_i) - r_ij(x_i')].  Proposals run in
 * order (each depends on the decisions before it), each row split over one
 * cluster of up to 8 CTAs: O(N D) work
 * each.  Draws: items [n_prop] (0..N-1), z_all [n_prop x D] and u_all
 * [n_prop] in (0,1), host arrays, all three given or all NULL; NULL draws
 * from Philox4x32-10 keyed by seed: proposal t (a per-context counter)
 * uses counter (t, 0, 0, 3) for the item floor(word0 N / 2^32) and u from
 * word 1, and (t, 1 + q, 0, 3) for z components 4q..4q+3 (Box-Muller).
 * accepted [n_prop] and dlogpi [n_prop] (host, optional) receive the
 * decisions and the log-target differences.  Synchronises.  Errors:
 * INVALID_ARG, STATE (no data / locations / sigma, a tree prior, HMC
 * iterations queued). */
int mds_rwmh(mds_ctx *ctx, int n_prop, double step, uint64_t seed, const int64_t *items, const double *z_all,
             const double *u_all, int32_t *accepted, double *dlogpi);

/* Checkpoint and resume of a chain: a snapshot holds the locations and
 * momenta (FP64, the caller's order), sigma, lambda, the Phi cut-off, the
 * counters that drive the Philox draws (HMC iterations, sigma updates,
 * random-walk proposals) and the accept count, and the locality order if
 * one is set; not Y, the fold or the tree prior (set those as before).
 * mds_get_state with buf = NULL stores the size in *bytes; else buf (host,
 * *bytes long) receives the snapshot.  mds_set_state restores one into a
 * context of the same N, D and precision (with the same data set): the next
 * draws are those the saved chain would have drawn, and with the same strip
 * length and order the continuation is bitwise identical.  Errors:
 * INVALID_ARG (size, magic, N / D / precision mismatch), STATE (queued HMC
 * iterations; restoring an order while a fold is set). */
int mds_get_state(mds_ctx *ctx, void *buf, int64_t *bytes);
int mds_set_state(mds_ctx *ctx, const void *buf, int64_t bytes);

/* Number of pairs M = N(N-1)/2 and the bytes of tile-packed Y resident on
 * the device. */
int mds_problem_size(const mds_ctx *ctx, int64_t *pairs, int64_t *y_bytes);

/* Tile strip length S (tiles of 64 x 64 pairs processed by one CTA).  0 picks
 * the autotuned value for this (GPU, N, D, precision).  Changing it changes
 * the summation order (results stay within tolerance but not bit-identical). */
int mds_set_strip(mds_ctx *ctx, int32_t strip);
int mds_get_strip(const mds_ctx *ctx, int32_t *strip);

/* ------------------------------------------------------------------------
 * Sharded evaluation over several ranks (section 2.5 of arXiv:1905.04582:
 * the pairwise sum is split over workers and their partial sums are reduced).
 *
 * mds_shard_range: the tiles of the pass (64 x 64 pairs, in row-block
 * order) cut into n_ranks contiguous ranges of equal pair count to within one
 * tile; rank `rank` gets tiles [*t0, *t1) (possibly empty for tiny N).  Host
 * only; needs no device.
 *
 * mds_set_shard: make ctx rank `rank` of `n_ranks` (n_ranks 1: no sharding).
 * Call before mds_set_data: the context then holds only its range's tiles of
 * Y (about 4 M / n_ranks bytes) and its pair pass covers only them.  Every
 * evaluation (mds_log_likelihood, mds_gradient, each leapfrog step of
 * mds_leapfrog / mds_hmc) computes this rank's partials {L_r, dL/dsigma_r,
 * sum r_r, dL/dX_r} (L_r = -M_r log sigma - sum r over the range's M_r pairs,
 * so that all four add up over the ranks), hands them to `allgather`, sums
 * the n_ranks vectors it gets back in rank order (FP64; every rank gets
 * bitwise the same totals) and takes its leapfrog updates with the total
 * gradient, so the chains of all ranks stay identical (replicated updates).
 * allgather(user, send, recv, count, where) must place every rank's `count`
 * doubles of send into recv (rank-major, n_ranks * count doubles) and return
 * 0 (nonzero: the evaluation fails with MDS_ERR_EXCHANGE); send and recv are
 * device memory when where_buffers is MDS_DEVICE (for NCCL), pinned host
 * memory when MDS_HOST (for host transports); the call is made with the
 * context's stream synchronised, and recv must be complete when it returns.
 * count = 3 + N D.  All ranks must make the same sequence of calls (each
 * evaluation is a collective).  A sharded context uses a fixed pass shape
 * (no timing autotuner), runs HMC without CUDA graphs, and refuses
 * mds_reorder, cross-validation folds, the tree prior, sigma updates and the
 * random-walk sampler (STATE).  Errors: INVALID_ARG (rank, n_ranks, NULL
 * allgather with n_ranks > 1), STATE (data already set), OOM.
 *
 * mds_shard_sum: the fixed-order sum of the exchange on the host:
 * out[i] = gathered[i] + gathered[count + i] + ... (rank 0 first), the order
 * the device combine uses. */
typedef int (*mds_allgather_fn)(void *user, const double *send, double *recv, int64_t count, int32_t where);
int mds_shard_range(int64_t n, int32_t n_ranks, int32_t rank, int64_t *t0, int64_t *t1);
int mds_set_shard(mds_ctx *ctx, int32_t n_ranks, int32_t rank, mds_allgather_fn allgather, void *user,
                  int32_t where_buffers);
int mds_shard_sum(int32_t n_ranks, int64_t count, const double *gathered, double *out);

/* Shape of the FP32C pair pass (section 2.5 of arXiv:1905.04582: the
 * pairwise transformation split into work units and the partial sums reduced;
 * the paper fixes its work-group shapes, this library picks one by timing).
 * kind MDS_PASS_STRIPS: one CTA per strip of `param` tiles of a row block;
 * kind MDS_PASS_CHUNKS: the tiles cut into `param` x (resident CTA slots)
 * chunks of equal estimated cost, one CTA each (the estimate uses the
 * per-tile counts of pairs whose Phi terms were skipped in an earlier pass);
 * kind MDS_PASS_CHUNK_COUNT: the same with exactly `param` chunks (at most
 * one per tile; param >= 1);
 * kind MDS_PASS_SM_CHUNKS: the chunks of MDS_PASS_CHUNKS (`param` per
 * resident slot), with one CTA per SM that runs the SM's slots as groups of
 * four warps (the CTAs sharing an SM progress unequally, the groups of one
 * CTA alike).  While a tree prior is set the same chunks run one per CTA.
 * param 0 returns to the autotuner, which times the candidates once per
 * (GPU name, N, D, precision, item order) and keeps the result in memory and
 * in the file named by MDS_TUNE_CACHE (default: tune_cache.txt beside the
 * library).  The FP64 context has the strip pass only (INVALID_ARG for
 * chunks).  mds_get_pass_shape returns the kind, its param and the number of
 * CTAs of the pass in use (any pointer may be NULL).  Changing the shape
 * changes the summation order (results stay within tolerance). */
#define MDS_PASS_STRIPS 0
#define MDS_PASS_CHUNKS 1
#define MDS_PASS_CHUNK_COUNT 2
#define MDS_PASS_SM_CHUNKS 3
int mds_set_pass_shape(mds_ctx *ctx, int32_t kind, int32_t param);
int mds_get_pass_shape(const mds_ctx *ctx, int32_t *kind, int32_t *param, int32_t *ctas);

/* Span of the pair pass inside real work, without events between launches
 * (benchmarks): while on, every pair-pass warp records %globaltimer after
 * its dependency wait (earliest, atomic min) and at its end (latest, atomic
 * max), and the reduction that follows adds end - start to a device total;
 * this keeps programmatic dependent launch intact, so the span is the pass's
 * time inside an HMC step.  mds_set_pass_stamps resets the total;
 * mds_get_pass_span synchronises the stream and returns the number of
 * passes and their total milliseconds since then. */
int mds_set_pass_stamps(mds_ctx *ctx, int on);
int mds_get_pass_span(mds_ctx *ctx, int64_t *passes, double *total_ms);

/* Time the fused pass: run `reps` evaluations back to back on the context's
 * stream and return the mean milliseconds per pass (CUDA events). */
int mds_time_pass(mds_ctx *ctx, int reps, double *ms_per_pass);

/* Kernel timing of the pair pass inside real work (benchmarks): while
 * profiling is on, every pair-pass launch -- also inside the CUDA graphs of
 * mds_hmc -- is bracketed by two CUDA events on the context's stream, and
 * mds_hmc synchronises after each iteration to read them.
 * mds_get_pass_time returns the number of timed launches and their total
 * milliseconds since profiling was switched on. */
int mds_set_profiling(mds_ctx *ctx, int on);
int mds_get_pass_time(const mds_ctx *ctx, int64_t *launches, double *total_ms);

/* ------------------------------------------------------------------------
 * Batches: several independent datasets (own Y, N, sigma; the same D), each
 * with several HMC chains, advanced together (the paper fits four virus
 * subtypes, section 3; batching independent problems is this library's
 * service).  Each leapfrog step of all chains is ONE persistent launch of the
 * batched pair pass (every Y tile is read once per step and serves all chains
 * of its dataset) plus one batched reduction; an HMC iteration of all chains
 * is one CUDA graph.  FP32C arithmetic only.  Datasets are numbered
 * 0..n_data-1, chains 0..chains[d]-1; "global chain" g counts chains dataset
 * by dataset and keys each chain's Philox stream (counter word 2 = g).
 * ------------------------------------------------------------------------ */
typedef struct mds_batch mds_batch;

/* n[n_data] item counts, chains[n_data] chains per dataset (1..1024), D for
 * all, flags MDS_PREC_FP32C.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
int mds_batch_create(int32_t n_data, const int64_t *n, int32_t d, const int32_t *chains, uint32_t flags,
                     mds_batch **out);
int mds_batch_destroy(mds_batch *b);
int mds_batch_set_stream(mds_batch *b, void *stream);
/* As mds_set_data / mds_set_sigma, for one dataset (all its chains). */
int mds_batch_set_data(mds_batch *b, int32_t dataset, const void *y, int dtype, int layout, int64_t ld, int where);
int mds_batch_set_sigma(mds_batch *b, int32_t dataset, double sigma);
/* As mds_set_locations / mds_get_locations, for one chain. */
int mds_batch_set_locations(mds_batch *b, int32_t dataset, int32_t chain, const void *x, int dtype, int where);
int mds_batch_get_locations(mds_batch *b, int32_t dataset, int32_t chain, void *x, int dtype, int where);
/* dL/dX of one chain at its current locations (evaluates the batch if needed). */
int mds_batch_get_gradient(mds_batch *b, int32_t dataset, int32_t chain, void *g, int dtype, int where);
/* One batched pass for all chains: loglik[g] and dlogl_dsigma[g] (host, per
 * global chain, optional).  Synchronises. */
int mds_batch_evaluate(mds_batch *b, double *loglik, double *dlogl_dsigma);
/* n_iter HMC iterations of n_steps leapfrog steps for every chain, eps[d] the
 * step size of dataset d; momenta and uniforms from Philox keyed by `seed`
 * (counters as in mds_hmc with chain = global chain).  accepted and dh
 * (optional, host) receive n_iter x (total chains) values, iteration-major.
 * Synchronises. */
int mds_batch_hmc(mds_batch *b, int n_iter, int n_steps, const double *eps, uint64_t seed, int32_t *accepted,
                  double *dh);
/* Shape of the batched pass.  strip in [1, 8]: the batched strip kernel,
 * strip tiles of one row block per CTA, each Y tile loaded into shared memory
 * once for all chains of its dataset.  strip in [-256, -1]: every chain's own
 * chunked pass (chunks of about -strip tiles), all chains' passes as
 * concurrent branches between the same reduction steps; Y is read once per
 * chain, from L2 where the datasets' Y fit.  0: autotune over both by timing
 * (strips of 1-4 tiles, chunks of 2-16 tiles).
 * mds_batch_get_strip returns the shape in use in the same encoding. */
int mds_batch_set_strip(mds_batch *b, int32_t strip);
/* Locality order for every dataset of a batch (as mds_reorder, section 2.5's
 * blocks of pairs made far enough apart that the Phi terms drop out): the
 * order is computed from each dataset's first chain, its Y repacked once,
 * and every chain of the dataset adopts the same slot order.  Every array of
 * the batch API stays in the caller's item order.  Call after the data and
 * all chains' locations are set (MDS_ERR_STATE otherwise). */
int mds_batch_reorder(mds_batch *b);
int mds_batch_get_strip(const mds_batch *b, int32_t *strip);
/* Mean milliseconds of one batched evaluation (pair pass + reduction) over
 * reps, timed as the HMC runs them: reps evaluations captured in one CUDA
 * graph, launched once to warm up and once timed.  The autotuner (strip 0)
 * times its candidates the same way. */
int mds_batch_time_pass(mds_batch *b, int reps, double *ms_per_pass);
/* Message of the last failed batch call (NULL: last failed mds_batch_create). */
const char *mds_batch_last_error(const mds_batch *b);

/* Allocation-free evaluation, for callers that must not let a library
 * allocate device memory: a host program that budgets every byte of the GPU
 * itself, code running inside a memory allocator's callback (where a nested
 * allocation could deadlock or recurse), or a real-time loop that must not
 * allocate after start-up.  The paper has no counterpart to this call; it is
 * a service of this library.
 *
 * Inputs (device memory, caller-owned): y, the full symmetric N x N matrix
 * (FP32, row stride ld >= N elements, diagonal ignored, values not checked);
 * x, the N x D locations (FP64).  Outputs: grad, N x D dL/dX (FP64, device);
 * loglik and dlogl_dsigma (host, optional; when either is given the call
 * synchronises `stream`).  Work goes on `stream` (NULL: legacy default).
 * Limits: 2 <= N <= 65536, 1 <= D <= MDS_MAX_D; larger N is rejected with
 * MDS_ERR_INVALID_ARG and a message from mds_last_error(NULL).
 *
 * It calls no cudaMalloc / cudaFree.  Its scratch is one fixed 256 KB array
 * in the library's device memory (held by every GPU that loads the library
 * until the process exits), shared by all calls: calls that overlap on the
 * GPU (different streams, or threads) race on it and must be serialised by
 * the caller.  Nothing in it needs clearing: every slot a call reads is
 * written earlier in the same call.  The first call on each device looks up
 * the scratch's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and do not use this entry point on a device
 * after cudaDeviceReset there (the kept address would belong to the
 * destroyed context).  Each pair is
 * evaluated twice in FP64 (once per row), so this call is slower than the
 * context path. */
int mds_loglik_grad_noalloc(int64_t n, int32_t d, const float *y, int64_t ld, const double *x, double sigma,
                            double *grad, double *loglik, double *dlogl_dsigma, void *stream);

/* Message of the last failed call on ctx (or of the last failed mds_create
 * in this thread when ctx is NULL).  Never NULL. */
const char *mds_last_error(const mds_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MDS_H_ */
