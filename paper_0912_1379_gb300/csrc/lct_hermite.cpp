// Hermite-zero discrete fractional Fourier transform (Sec. 2, eq. (tmat)):
// the entry points frft_hermite_execute and frft_hermite_basis
// (include/lct.h) and the per-device cache of the basis (nodes x_k and the
// orthogonal matrix U) that k_hermite.cu builds on the GPU.
#include "lct_plan.h"

#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

cudaError_t lct_launch_hermite_basis(int n, double* x, double* U, float* Uf, cudaStream_t stream);
cudaError_t lct_launch_hermite_apply(int dtype, int n, const void* in, void* out, void* work,
                                     const void* alpha, const void* U, int64_t batch,
                                     cudaStream_t stream);
size_t lct_hermite_umma_bytes(int n);
cudaError_t lct_launch_hermite_umma_pack(int n, const double* U, float* B1, float* B2,
                                         cudaStream_t stream);
cudaError_t lct_launch_hermite_apply_umma(int n, const void* in, void* out, void* work,
                                          const void* alpha, const float* B1, const float* B2,
                                          int64_t batch, cudaStream_t stream);
cudaError_t lct_hermite_read_status(int32_t* v);
cudaError_t lct_launch_hermite_alpha(int dtype, int n, double t_hi, double t_lo, double log_r,
                                     int zero, void* alpha, cudaStream_t stream);

namespace {

constexpr int64_t kHermMaxN = 4096;

struct herm_basis {
    double* x = nullptr;   // n nodes, ascending
    double* U = nullptr;   // n x n, row-major U[m][k] (component m of u_k)
    float* Uf = nullptr;   // the same in FP32 (complex64 transforms)
    float* B1 = nullptr;   // tensor-core operands of the two products (complex64,
    float* B2 = nullptr;   // N >= kUmmaMinN): TF32 hi/lo parts, tiled
};

// complex64 transforms take the tensor cores from this N up (below, the
// 256-column tiles would be mostly padding); LCT_HERMITE_FP32=simt selects
// the CUDA-core product for every N (a diagnostic).
constexpr int64_t kUmmaMinN = 128;

bool umma_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("LCT_HERMITE_FP32");
        return !(e && std::strcmp(e, "simt") == 0);
    }();
    return on;
}

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

// The tensor-core operands of N's basis (built at their first use).
lct_status herm_get_umma(int64_t n, herm_basis* out) {
    lct_status st = herm_get(n, out);
    if (st != LCT_OK) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LCT_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_herm_mu);
    herm_basis& b = g_herm[{dev, n}];
    if (!b.B1) {
        const size_t bytes = lct_hermite_umma_bytes((int)n);
        float *b1 = nullptr, *b2 = nullptr;
        if (cudaMalloc(&b1, bytes) != cudaSuccess || cudaMalloc(&b2, bytes) != cudaSuccess) {
            cudaFree(b1);
            return LCT_ERR_OOM;
        }
        cudaStream_t s = nullptr;
        lct_status r = LCT_OK;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) r = LCT_ERR_CUDA;
        if (r == LCT_OK && lct_launch_hermite_umma_pack((int)n, b.U, b1, b2, s) != cudaSuccess)
            r = LCT_ERR_CUDA;
        if (r == LCT_OK && cudaStreamSynchronize(s) != cudaSuccess) r = LCT_ERR_CUDA;
        if (s) cudaStreamDestroy(s);
        if (r != LCT_OK) {
            cudaFree(b1);
            cudaFree(b2);
            return r;
        }
        b.B1 = b1;
        b.B2 = b2;
    }
    *out = b;
    return LCT_OK;
}

// arg(z) / (2 pi) as a double-double (t_hi + t_lo), and log|z|, for the
// device table of z^m (one long-double evaluation per call).
void herm_z_params(double z_re, double z_im, double* t_hi, double* t_lo, double* log_r) {
    const long double two_pi = 6.283185307179586476925286766559005768L;
    const long double t = atan2l((long double)z_im, (long double)z_re) / two_pi;
    *t_hi = (double)t;
    *t_lo = (double)(t - (long double)*t_hi);
    *log_r = (double)logl(hypotl((long double)z_re, (long double)z_im));
}

}  // namespace

extern "C" {

lct_status frft_hermite_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                                int64_t batch, lct_dtype dtype, lct_stream_t stream_) {
    lcth::trace_range trace("frft_hermite_execute");
    lcth::launch_lock launch;
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
    const bool tensor = dtype == LCT_C64 && N >= kUmmaMinN && umma_enabled();
    if ((st = tensor ? herm_get_umma(N, &b) : herm_get(N, &b)) != LCT_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t es = lcth::sample_bytes(dtype);
    const size_t work_bytes = (size_t)batch * (size_t)N * es;
    const size_t alpha_bytes = (size_t)N * es;
    void* work = nullptr;
    if (cudaMallocAsync(&work, work_bytes + alpha_bytes, stream) != cudaSuccess) return LCT_ERR_OOM;
    void* alpha = (char*)work + work_bytes;
    double t_hi = 0.0, t_lo = 0.0, log_r = 0.0;
    const int zero = (z_re == 0.0 && z_im == 0.0) ? 1 : 0;
    if (!zero) herm_z_params(z_re, z_im, &t_hi, &t_lo, &log_r);
    cudaError_t e = lct_launch_hermite_alpha((int)dtype, (int)N, t_hi, t_lo, log_r, zero, alpha, stream);
    if (e == cudaSuccess) {
        if (tensor)
            e = lct_launch_hermite_apply_umma((int)N, in, out, work, alpha, b.B1, b.B2, batch,
                                              stream);
        else
            e = lct_launch_hermite_apply((int)dtype, (int)N, in, out, work, alpha,
                                         dtype == LCT_C64 ? (const void*)b.Uf : (const void*)b.U,
                                         batch, stream);
    }
    const cudaError_t ef = cudaFreeAsync(work, stream);
    if (e != cudaSuccess) return lcth::from_cuda(e);
    return lcth::from_cuda(ef);
}

lct_status frft_hermite_status(lct_stream_t stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCT_ERR_CUDA;
    int32_t v = 0;
    if (lct_hermite_read_status(&v) != cudaSuccess) return LCT_ERR_CUDA;
    return v == LCT_DEV_OK ? LCT_OK : (v == LCT_DEV_TIMEOUT ? LCT_ERR_TIMEOUT : LCT_ERR_DEVICE);
}

lct_status frft_hermite_basis(int64_t N, double* x, double* U) {
    if (N < 2 || N > kHermMaxN) return LCT_ERR_N;
    if (!x) return LCT_ERR_ARG;
    lcth::launch_lock launch;
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
