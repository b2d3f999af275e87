// Allocation-free evaluation of the likelihood and its gradients.
//
// Some callers cannot let a library allocate device memory: a host program
// that budgets every byte of the GPU itself, code that runs inside a memory
// allocator's own callback (where a nested cudaMalloc could deadlock or
// recurse), or a real-time loop that must not allocate after start-up.  For
// them, mds_loglik_grad_noalloc() evaluates L, dL/dX and dL/dsigma from
// caller-owned device buffers and allocates nothing: its only scratch is the
// fixed file-scope array below, which every GPU that loads this library
// holds until the process exits.
//
// Work split: one warp per row i of the full N x N matrix Y; the lanes stride
// over j != i, so every pair is visited twice (once per end, as the per-row
// gradient sums of the paper's Algorithm 2) and no column partials are
// needed.  Arithmetic is FP64 (CUDA's sqrt / erfc / log1p / exp), the same
// per-pair formulas as the FP64 path.  Each block writes its partial sums of
// the scalar terms into the scratch array; a second, single-block kernel sums
// them in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "mds.h"
#include "mds_internal.h"

namespace {

constexpr int kNaWarps = 8;                       // rows per block
constexpr int kNaThreads = 32 * kNaWarps;
constexpr int kNaMaxBlocks = 8192;                // => N <= 65536
constexpr int kNaParts = 4;                       // e^2, m*delta, log Phi, spare

// The scratch: per-block partial sums, then the three final sums.
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks * kNaParts + kNaParts];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double *g_na_ptr[kMaxDevices] = {};

template <int D>
__global__ void __launch_bounds__(kNaThreads) noalloc_rows_kernel(int64_t n, const float *y, int64_t ld,
                                                                  const double *x, double sigma, double *grad,
                                                                  double *part) {
    constexpr double kInvSqrt2Pi = 0.39894228040143267794;
    constexpr double kInvSqrt2 = 0.70710678118654752440;
    __shared__ double red[kNaWarps][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kNaWarps + warp;
    const double inv_s = 1.0 / sigma, inv_s2 = inv_s * inv_s;
    double g[D];
#pragma unroll
    for (int k = 0; k < D; ++k) g[k] = 0.0;
    double e2 = 0.0, md = 0.0, lp = 0.0;
    if (i < n) {
        double xi[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = x[i * D + k];
        const float *yrow = y + i * ld;
        for (int64_t j = lane; j < n; j += 32) {
            if (j == i) continue;
            double dl[D];
            double d2 = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                dl[k] = xi[k] - x[j * D + k];
                d2 = fma(dl[k], dl[k], d2);
            }
            const double del = sqrt(d2);
            const double inv = del > 0.0 ? 1.0 / del : 0.0;
            const double e = static_cast<double>(yrow[j]) - del;
            const double z = del * inv_s;
            const double qz = 0.5 * erfc(z * kInvSqrt2);
            const double m = exp(-0.5 * z * z) * kInvSqrt2Pi / (1.0 - qz);
            const double wi = (m * inv_s - e * inv_s2) * inv;
#pragma unroll
            for (int k = 0; k < D; ++k) g[k] -= wi * dl[k];
            if (j > i) {  // scalar terms once per pair
                e2 = fma(e, e, e2);
                md = fma(m, del, md);
                lp += log1p(-qz);
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
        for (int k = 0; k < D; ++k) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        md += __shfl_xor_sync(0xffffffffu, md, o);
        lp += __shfl_xor_sync(0xffffffffu, lp, o);
    }
    if (lane == 0) {
        if (i < n) {
#pragma unroll
            for (int k = 0; k < D; ++k) grad[i * D + k] = g[k];
        }
        red[warp][0] = e2;
        red[warp][1] = md;
        red[warp][2] = lp;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = red[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < kNaWarps; ++w) v += red[w][threadIdx.x];
        part[blockIdx.x * kNaParts + threadIdx.x] = v;
    }
}

// Sums the per-block partials in a fixed order into the three final slots.
__global__ void noalloc_sum_kernel(int nblocks, double *part) {
    __shared__ double sm[3][256];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += 256)
        for (int q = 0; q < 3; ++q) acc[q] += part[b * kNaParts + q];
    for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[kNaMaxBlocks * kNaParts + threadIdx.x] = sm[threadIdx.x][0];
}

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol itself as a device pointer).
int scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        mds::set_thread_error("mds_loglik_grad_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return MDS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        mds::set_thread_error("mds_loglik_grad_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
        return MDS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            mds::set_thread_error("mds_loglik_grad_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return MDS_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_na_ptr[dev];
    return MDS_OK;
}

}  // namespace

extern "C" int mds_loglik_grad_noalloc(int64_t n, int32_t d, const float *y, int64_t ld, const double *x,
                                       double sigma, double *grad, double *loglik, double *dlogl_dsigma,
                                       void *stream) {
    if (n < 2 || d < 1 || d > MDS_MAX_D || !y || !x || !grad || ld < n || !(sigma > 0.0) || !std::isfinite(sigma)) {
        mds::set_thread_error("mds_loglik_grad_noalloc: invalid argument (need 2 <= N, 1 <= D <= %d, ld >= N, "
                              "sigma > 0, non-NULL y, x, grad)", MDS_MAX_D);
        return MDS_ERR_INVALID_ARG;
    }
    const int64_t nblocks = (n + kNaWarps - 1) / kNaWarps;
    if (nblocks > kNaMaxBlocks) {
        mds::set_thread_error("mds_loglik_grad_noalloc: N = %lld exceeds the maximum %d of the fixed scratch",
                              static_cast<long long>(n), kNaMaxBlocks * kNaWarps);
        return MDS_ERR_INVALID_ARG;
    }
    double *part = nullptr;
    int st = scratch_address(&part);
    if (st != MDS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (d) {
#define MDS_NA_CASE(DD) \
    case DD: noalloc_rows_kernel<DD><<<static_cast<int>(nblocks), kNaThreads, 0, s>>>(n, y, ld, x, sigma, grad, part); break;
        MDS_NA_CASE(1) MDS_NA_CASE(2) MDS_NA_CASE(3) MDS_NA_CASE(4)
        MDS_NA_CASE(5) MDS_NA_CASE(6) MDS_NA_CASE(7) MDS_NA_CASE(8)
#undef MDS_NA_CASE
        default: break;
    }
    noalloc_sum_kernel<<<1, 256, 0, s>>>(static_cast<int>(nblocks), part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mds::set_thread_error("mds_loglik_grad_noalloc: launch: %s", cudaGetErrorString(e));
        return MDS_ERR_CUDA;
    }
    if (loglik || dlogl_dsigma) {
        double sums[3];
        e = cudaMemcpyAsync(sums, part + kNaMaxBlocks * kNaParts, sizeof(sums), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            mds::set_thread_error("mds_loglik_grad_noalloc: %s", cudaGetErrorString(e));
            return MDS_ERR_CUDA;
        }
        const double m = 0.5 * static_cast<double>(n) * static_cast<double>(n - 1);
        const double sum_r = sums[0] / (2.0 * sigma * sigma) + sums[2];
        const double ll = -m * std::log(sigma) - sum_r;
        const double ds = -m / sigma + sums[0] / (sigma * sigma * sigma) + sums[1] / (sigma * sigma);
        if (loglik) *loglik = ll;
        if (dlogl_dsigma) *dlogl_dsigma = ds;
        if (!std::isfinite(ll) || !std::isfinite(ds)) {
            mds::set_thread_error("mds_loglik_grad_noalloc: non-finite result");
            return MDS_ERR_NONFINITE;
        }
    }
    return MDS_OK;
}
