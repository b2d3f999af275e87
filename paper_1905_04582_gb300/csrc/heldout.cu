// Cross-validation folds (arXiv:1905.04582, section 2.4 "Model selection").
//
// A fold holds out a set of observations y_ij; the model is trained on the
// rest (the pair pass skips pairs whose tile-packed y is negative) and the
// held-out pairs are scored by the log pointwise predictive density,
// estimated from S posterior draws as
//   lpd-hat = sum_ij log( (1/S) sum_s p(y_ij | X_s, sigma_s) ),
// p the truncated-normal density of Eq. (1):
//   log p(y | delta, sigma) = -log(sqrt(2 pi) sigma) - (y - delta)^2 / (2 sigma^2)
//                             - log Phi(delta / sigma).
// The estimate is accumulated one draw at a time as a running log-sum-exp per
// pair (max m and scaled sum s, so no exp underflows), in FP64: the held-out
// set is small next to the M pairs of the pass and is scored once per draw.
#include <cstdint>

#include "mds_internal.h"

namespace mds {
namespace {

constexpr int kHoThreads = 256;

__global__ void ho_mark_kernel(float *y, const int64_t *off, int64_t count, float *ho_y, unsigned char *tile_ho) {
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < count;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t o = off[k];
        ho_y[k] = y[o];
        y[o] = -1.0f;
        tile_ho[o / kTileElems] = 1;
    }
}

__global__ void ho_restore_kernel(float *y, const int64_t *off, int64_t count, const float *ho_y) {
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < count;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[off[k]] = ho_y[k];
}

template <typename T>
__global__ void lpd_accumulate_kernel(const T *x, int d, const int2 *pairs, const float *ho_y, int64_t count,
                                      double sigma, bool first, double *lse_m, double *lse_s, unsigned *err) {
    constexpr double kLogSqrt2Pi = 0.91893853320467274178;
    constexpr double kInvSqrt2 = 0.70710678118654752440;
    const double log_sigma = log(sigma);
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < count;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int2 p = pairs[k];
        double d2 = 0.0;
        for (int c = 0; c < d; ++c) {
            const double t = static_cast<double>(x[static_cast<int64_t>(p.x) * d + c]) -
                             static_cast<double>(x[static_cast<int64_t>(p.y) * d + c]);
            d2 += t * t;
        }
        const double delta = sqrt(d2);
        const double e = static_cast<double>(ho_y[k]) - delta;
        const double log_phi_cdf = log1p(-0.5 * erfc(delta / sigma * kInvSqrt2));
        const double lp = -kLogSqrt2Pi - log_sigma - e * e / (2.0 * sigma * sigma) - log_phi_cdf;
        if (!isfinite(lp)) atomicOr(err, kErrNonfinite);
        if (first) {
            lse_m[k] = lp;
            lse_s[k] = 1.0;
        } else {
            const double m = lse_m[k];
            if (lp > m) {
                lse_s[k] = lse_s[k] * exp(m - lp) + 1.0;
                lse_m[k] = lp;
            } else {
                lse_s[k] += exp(lp - m);
            }
        }
    }
}

// Block b sums the terms k = b, b + kLpdParts, ... in a fixed order (each
// thread a strided subset, then a tree); the second launch (one block) sums
// the kLpdParts partials the same way.
__device__ __forceinline__ double block_sum(double v, double *sm) {
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = kHoThreads / 2; o > 0; o >>= 1) {
        if (static_cast<int>(threadIdx.x) < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    return sm[0];
}

__global__ void lpd_partial_kernel(const double *lse_m, const double *lse_s, int64_t count, double log_draws,
                                   double *part) {
    __shared__ double sm[kHoThreads];
    double v = 0.0;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * kHoThreads + threadIdx.x; k < count;
         k += static_cast<int64_t>(kLpdParts) * kHoThreads)
        v += lse_m[k] + log(lse_s[k]) - log_draws;
    const double t = block_sum(v, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void lpd_final_kernel(const double *part, double *out) {
    __shared__ double sm[kHoThreads];
    double v = 0.0;
    for (int k = threadIdx.x; k < kLpdParts; k += kHoThreads) v += part[k];
    const double t = block_sum(v, sm);
    if (threadIdx.x == 0) *out = t;
}

int grid_of(int64_t count) {
    const int64_t g = (count + kHoThreads - 1) / kHoThreads;
    return static_cast<int>(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

cudaError_t launch_ho_mark(float *y, const int64_t *off, int64_t count, float *ho_y, unsigned char *tile_ho,
                           cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    ho_mark_kernel<<<grid_of(count), kHoThreads, 0, s>>>(y, off, count, ho_y, tile_ho);
    return cudaGetLastError();
}

cudaError_t launch_ho_restore(float *y, const int64_t *off, int64_t count, const float *ho_y, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    ho_restore_kernel<<<grid_of(count), kHoThreads, 0, s>>>(y, off, count, ho_y);
    return cudaGetLastError();
}

cudaError_t launch_lpd_accumulate(const void *x, bool fp64, int d, const int2 *pairs, const float *ho_y,
                                  int64_t count, double sigma, bool first, double *lse_m, double *lse_s,
                                  unsigned *err, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (fp64)
        lpd_accumulate_kernel<double><<<grid_of(count), kHoThreads, 0, s>>>(
            static_cast<const double *>(x), d, pairs, ho_y, count, sigma, first, lse_m, lse_s, err);
    else
        lpd_accumulate_kernel<float><<<grid_of(count), kHoThreads, 0, s>>>(
            static_cast<const float *>(x), d, pairs, ho_y, count, sigma, first, lse_m, lse_s, err);
    return cudaGetLastError();
}

cudaError_t launch_lpd_sum(const double *lse_m, const double *lse_s, int64_t count, double draws, double *part,
                           double *out, cudaStream_t s) {
    lpd_partial_kernel<<<kLpdParts, kHoThreads, 0, s>>>(lse_m, lse_s, count, log(draws), part);
    lpd_final_kernel<<<1, kHoThreads, 0, s>>>(part, out);
    return cudaGetLastError();
}

}  // namespace mds
