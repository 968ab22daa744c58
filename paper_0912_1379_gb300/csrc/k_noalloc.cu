// lct_execute_noalloc: the unfused FP64 path (chirp kernel -> DFT ->
// chirp + scale kernel) without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- a process whose device
// memory is fully reserved up front by its own pool allocator, or a
// latency-critical caller that must not hit cudaMalloc's implicit device
// synchronisation.  The regular entry points allocate plan descriptors and,
// on the FP64 path, an FP64 workspace plus a cuFFT plan; this one does not.
//
// Where the memory comes from: the FP64 intermediate lives in the file-scope
// array g_noalloc_work below (32 MiB, LCT_NOALLOC_MAX_POINTS complex128
// samples), which every GPU that loads the library holds until the process
// exits.  The per-signal constants travel as a kernel argument.  The DFT is
// this file's own FP64 shared-memory Stockham kernel, because a cuFFT plan
// allocates.  Calls share the array: two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it.  Nothing
// in it has to start at zero: every sample a call reads was written earlier
// in the same call.
//
// When the memory is committed: with CUDA's lazy module loading this file's
// module, and with it the array, is loaded on the first call on a device
// (the symbol lookup in setup_device).  That first call -- a call with
// batch 0 is enough -- should therefore come before the caller reserves its
// device memory, and before any stream capture.
#include "lct_internal.h"
#include "xft_common.cuh"
#include "../../include/lct.h"

#include <mutex>

static __device__ __align__(256) cpx<double> g_noalloc_work[LCT_NOALLOC_MAX_POINTS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_work_ptr[kMaxDevices] = {};   // device address of g_noalloc_work, per device
int g_sm_count[kMaxDevices] = {};     // multiprocessors of each device (grid sizing)

__global__ void k_na_pre(const void* __restrict__ in_, int dtype, cpx<double>* __restrict__ work,
                         lct_desc D, int64_t total, int log2n) {
    const int64_t N = 1ll << log2n;
    const uint64_t cen = (uint64_t)(N - 1) << (63 - log2n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(t & (N - 1));
        cpx<double> f;
        if (dtype == LCT_C64) {
            cpx<float> v = ((const cpx<float>*)in_)[t];
            f = {(double)v.x, (double)v.y};
        } else {
            f = ((const cpx<double>*)in_)[t];
        }
        const uint32_t m2 = m_squared(n, (int)N);
        if (D.kind == LCT_KIND_DIAG) {
            // b = 0: the whole transform is this diagonal; the DFT is skipped.
            cpx<double> w = expi_turn64(phase64(D.out_hi, D.out_lo, m2) + D.out_c);
            work[t] = cscale(cmul(f, w), D.scale);
        } else {
            cpx<double> w = expi_turn64(phase64(D.in_hi, D.in_lo, m2) + (uint64_t)n * cen);
            if (D.flags & LCT_FLAG_DECAY) w = cscale(w, exp(-D.decay * (double)m2));
            work[t] = cmul(f, w);
        }
    }
}

// In-place forward DFT of each N-sample row of work, one CTA per row,
// radix-2 Stockham passes between two shared-memory buffers.
__global__ void k_na_dft(cpx<double>* work, int log2n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = 1 << log2n, half = N >> 1;
    cpx<double>* a = reinterpret_cast<cpx<double>*>(smem_raw);
    cpx<double>* b = a + N;
    cpx<double>* x = work + (int64_t)blockIdx.x * N;
    for (int t = threadIdx.x; t < N; t += blockDim.x) a[t] = x[t];
    __syncthreads();
    for (int ns = 1; ns < N; ns <<= 1) {
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (ns - 1);
            double s, c;
            sincospi(-(double)k / (double)ns, &s, &c);      // e^{-2 pi i k / (2 ns)}
            const cpx<double> u = a[j], v = cmul(a[j + half], cpx<double>{c, s});
            const int o = ((j - k) << 1) + k;
            b[o] = u + v;
            b[o + ns] = u - v;
        }
        __syncthreads();
        cpx<double>* t = a;
        a = b;
        b = t;
    }
    for (int t = threadIdx.x; t < N; t += blockDim.x) x[t] = a[t];
}

__global__ void k_na_post(const cpx<double>* __restrict__ work, void* __restrict__ out_, int dtype,
                          lct_desc D, int64_t total, int log2n) {
    const int64_t N = 1ll << log2n;
    const uint64_t cen = (uint64_t)(N - 1) << (63 - log2n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        cpx<double> g = work[t];
        if (D.kind != LCT_KIND_DIAG) {
            const int n = (int)(t & (N - 1));
            const uint32_t m2 = m_squared(n, (int)N);
            cpx<double> w =
                expi_turn64(phase64(D.out_hi, D.out_lo, m2) + (uint64_t)n * cen + D.out_c);
            g = cscale(cmul(g, w), D.scale);
        }
        if (dtype == LCT_C64) ((cpx<float>*)out_)[t] = {(float)g.x, (float)g.y};
        else ((cpx<double>*)out_)[t] = g;
    }
}

// First call on a device: look up the array's device address (the host-side
// name g_noalloc_work is only a stand-in and must never reach a kernel),
// allow the DFT kernel its shared memory and read the multiprocessor count.
// The cache is keyed by device ordinal, so it does not survive
// cudaDeviceReset (documented in include/lct.h).
lct_status setup_device(cpx<double>** work, int* sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LCT_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_work_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_work) != cudaSuccess || !p) return LCT_ERR_CUDA;
        if (cudaFuncSetAttribute(k_na_dft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * LCT_NOALLOC_MAX_N * sizeof(cpx<double>))) != cudaSuccess)
            return LCT_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return LCT_ERR_CUDA;
        g_sm_count[dev] = n;
        g_work_ptr[dev] = p;
    }
    *work = (cpx<double>*)g_work_ptr[dev];
    *sms = g_sm_count[dev];
    return LCT_OK;
}

// Grid of the grid-stride kernels: one 256-thread block per 256 samples, at
// most 16 resident blocks per multiprocessor.
unsigned grid_for(int64_t total, int sms) {
    const int64_t cap = (int64_t)sms * 16;
    int64_t b = (total + 255) / 256;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

extern "C" lct_status lct_execute_noalloc(int64_t N, double a, double b, double c, double d,
                                          lct_dtype dtype, const void* in, void* out,
                                          int64_t batch, lct_stream_t stream_) {
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    if (N < 2 || N > LCT_NOALLOC_MAX_N || (N & (N - 1)) != 0) return LCT_ERR_N;
    if (batch < 0) return LCT_ERR_ARG;
    if (batch > LCT_NOALLOC_MAX_POINTS / N) return LCT_ERR_ARG;   // beyond the static array
    const double p[8] = {a, 0.0, b, 0.0, c, 0.0, d, 0.0};
    lct_desc D;
    lct_status st = (lct_status)lct_make_desc_host(N, p, 0, &D);
    if (st != LCT_OK) return st;
    // Set-up first, also for batch 0: that call commits the array (module
    // load) without running anything.
    cpx<double>* work = nullptr;
    int sms = 0;
    st = setup_device(&work, &sms);
    if (st != LCT_OK) return st;
    if (batch == 0) return LCT_OK;
    const uintptr_t align = dtype == LCT_C64 ? 8 : 16;
    if (!in || !out) return LCT_ERR_ARG;
    if (((uintptr_t)in) % align || ((uintptr_t)out) % align) return LCT_ERR_ALIGN;
    // An error left pending by earlier work on this thread is reported as
    // LCT_ERR_CUDA without launching and is not cleared, so the caller can
    // still read it; after that, an error is this call's own launch failure.
    if (cudaPeekAtLastError() != cudaSuccess) return LCT_ERR_CUDA;
    cudaStream_t stream = (cudaStream_t)stream_;
    int log2n = 0;
    while ((int64_t(1) << log2n) < N) ++log2n;
    const int64_t total = batch * N;
    k_na_pre<<<grid_for(total, sms), 256, 0, stream>>>(in, dtype, work, D, total, log2n);
    if (cudaGetLastError() != cudaSuccess) return LCT_ERR_CUDA;
    if (D.kind != LCT_KIND_DIAG) {
        const int threads = N >= 512 ? 256 : (int)(N / 2 > 32 ? N / 2 : 32);
        k_na_dft<<<(unsigned)batch, threads, 2 * N * sizeof(cpx<double>), stream>>>(work, log2n);
        if (cudaGetLastError() != cudaSuccess) return LCT_ERR_CUDA;
    }
    k_na_post<<<grid_for(total, sms), 256, 0, stream>>>(work, out, dtype, D, total, log2n);
    return cudaGetLastError() == cudaSuccess ? LCT_OK : LCT_ERR_CUDA;
}
