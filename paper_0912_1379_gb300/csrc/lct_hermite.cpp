// Hermite-zero discrete fractional Fourier transform (Sec. 2, eq. (tmat)):
// the entry points frft_hermite_execute and frft_hermite_basis
// (include/lct.h) and the per-device cache of the basis (nodes x_k and the
// orthogonal matrix U) that k_hermite.cu builds on the GPU.
#include "lct_plan.h"

#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

cudaError_t lct_launch_hermite_basis(int n, double* x, double* U, float* Uf, cudaStream_t stream);
cudaError_t lct_launch_hermite_apply(int dtype, int n, const void* in, void* out, void* work,
                                     const void* alpha, const void* U, int64_t batch,
                                     cudaStream_t stream);

namespace {

constexpr int64_t kHermMaxN = 4096;

struct herm_basis {
    double* x = nullptr;   // n nodes, ascending
    double* U = nullptr;   // n x n, row-major U[m][k] (component m of u_k)
    float* Uf = nullptr;   // the same in FP32 (complex64 transforms)
};

std::mutex g_herm_mu;
std::map<std::pair<int, int64_t>, herm_basis> g_herm;   // (device, N) -> basis

// The basis of N on the current device, built (synchronously, on a private
// stream) at its first use and kept for the process.
lct_status herm_get(int64_t n, herm_basis* out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LCT_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_herm_mu);
    auto it = g_herm.find({dev, n});
    if (it != g_herm.end()) {
        *out = it->second;
        return LCT_OK;
    }
    herm_basis b;
    const size_t nn = (size_t)n * (size_t)n;
    if (cudaMalloc(&b.x, sizeof(double) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&b.U, sizeof(double) * nn) != cudaSuccess ||
        cudaMalloc(&b.Uf, sizeof(float) * nn) != cudaSuccess) {
        cudaFree(b.x);
        cudaFree(b.U);
        cudaFree(b.Uf);
        return LCT_ERR_OOM;
    }
    cudaStream_t s = nullptr;
    lct_status st = LCT_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = LCT_ERR_CUDA;
    if (st == LCT_OK && lct_launch_hermite_basis((int)n, b.x, b.U, b.Uf, s) != cudaSuccess)
        st = LCT_ERR_CUDA;
    if (st == LCT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = LCT_ERR_CUDA;
    if (s) cudaStreamDestroy(s);
    if (st != LCT_OK) {
        cudaFree(b.x);
        cudaFree(b.U);
        cudaFree(b.Uf);
        return st;
    }
    g_herm[{dev, n}] = b;
    *out = b;
    return LCT_OK;
}

// alpha_m = sqrt(2 pi) z^m, m < n, with |z|^m and m arg z in long double.
template <class T>
std::vector<T> herm_alpha(int64_t n, double z_re, double z_im) {
    const long double r = hypotl((long double)z_re, (long double)z_im);
    const long double th = atan2l((long double)z_im, (long double)z_re);
    const long double s2pi = sqrtl(2.0L * 3.141592653589793238462643383279502884L);
    std::vector<T> a(2 * (size_t)n);
    for (int64_t m = 0; m < n; ++m) {
        const long double mag = s2pi * (m == 0 ? 1.0L : powl(r, (long double)m));
        const long double ang = th * (long double)m;
        a[2 * m] = (T)(mag * cosl(ang));
        a[2 * m + 1] = (T)(mag * sinl(ang));
    }
    return a;
}

}  // namespace

extern "C" {

lct_status frft_hermite_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                                int64_t batch, lct_dtype dtype, lct_stream_t stream_) {
    lcth::trace_range trace("frft_hermite_execute");
    if (N < 2 || N > kHermMaxN) return LCT_ERR_N;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    const double az = std::hypot(z_re, z_im);
    if (!std::isfinite(z_re) || !std::isfinite(z_im) || az > 1.0 + 1e-15) return LCT_ERR_ARG;
    if (batch < 0 || batch > (int64_t)65535 * 32) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    lct_status st = lcth::check_ptr(in, dtype);
    if (st == LCT_OK) st = lcth::check_ptr(out, dtype);
    if (st != LCT_OK) return st;
    herm_basis b;
    if ((st = herm_get(N, &b)) != LCT_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t es = lcth::sample_bytes(dtype);
    const size_t work_bytes = (size_t)batch * (size_t)N * es;
    const size_t alpha_bytes = (size_t)N * es;
    void* work = nullptr;
    if (cudaMallocAsync(&work, work_bytes + alpha_bytes, stream) != cudaSuccess) return LCT_ERR_OOM;
    void* alpha = (char*)work + work_bytes;
    cudaError_t e;
    if (dtype == LCT_C64) {
        const std::vector<float> a = herm_alpha<float>(N, z_re, z_im);
        e = cudaMemcpyAsync(alpha, a.data(), alpha_bytes, cudaMemcpyHostToDevice, stream);
    } else {
        const std::vector<double> a = herm_alpha<double>(N, z_re, z_im);
        e = cudaMemcpyAsync(alpha, a.data(), alpha_bytes, cudaMemcpyHostToDevice, stream);
    }
    if (e == cudaSuccess)
        e = lct_launch_hermite_apply((int)dtype, (int)N, in, out, work, alpha,
                                     dtype == LCT_C64 ? (const void*)b.Uf : (const void*)b.U, batch,
                                     stream);
    const cudaError_t ef = cudaFreeAsync(work, stream);
    if (e != cudaSuccess) return lcth::from_cuda(e);
    return lcth::from_cuda(ef);
}

lct_status frft_hermite_basis(int64_t N, double* x, double* U) {
    if (N < 2 || N > kHermMaxN) return LCT_ERR_N;
    if (!x) return LCT_ERR_ARG;
    herm_basis b;
    lct_status st = herm_get(N, &b);
    if (st != LCT_OK) return st;
    if (cudaMemcpy(x, b.x, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LCT_ERR_CUDA;
    if (U && cudaMemcpy(U, b.U, sizeof(double) * (size_t)N * (size_t)N, cudaMemcpyDeviceToHost) !=
                 cudaSuccess)
        return LCT_ERR_CUDA;
    return LCT_OK;
}

}  // extern "C"
