// Large-N XFT in two passes over the samples (four-step factorisation of
// the N-point DFT of Sec. 3, N = N1 N2, log2 N1 = floor(log2 N / 2)):
//   n = n2 + N2 n1, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_N^{n2 k1} sum_{n1} W_{N1}^{n1 k1} u[n2 + N2 n1]
// with u the pre-chirped input and W_M = e^{-2 pi i / M} (forward sign).
//
// Pass A (a tile of GA consecutive columns n2 of one signal): loads u with
// the pre-chirp (each row n1 of the tile is GA consecutive samples), runs the
// N1-point DFT down every column with the Stockham engine, multiplies by
// W_N^{n2 k1} and stores Y[k1][n2] row-major in a workspace slot.
// Pass B (a tile of GB consecutive rows k1): the N2-point DFT along every
// row (contiguous loads), a transpose through shared memory, then
// X[k1 + N1 k2] with the post-chirp and scale (GB consecutive k1 per k2).
#include "xft_twopass.cuh"

namespace {

using namespace xft;
using namespace xtp;

template <int L1, int L2, class R>
__global__ void __launch_bounds__(PT_THREADS, (sizeof(R) == 4 ? 4 : 2))
k_xft_twopass(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, cpx<R>* __restrict__ work,
              int32_t* __restrict__ sync, const lct_desc* __restrict__ desc, int desc_step,
              int64_t count, int64_t lag, int64_t slots, const int32_t* __restrict__ idx,
              int32_t* __restrict__ status, const cpx<R>* __restrict__ tw1,
              const cpx<R>* __restrict__ tw2) {
    using P = pt_shape<L1, L2, R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    __shared__ long long s_item;
    unsigned long long* queue = reinterpret_cast<unsigned long long*>(sync);
    const int64_t total = count * (P::CB + P::RB);
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t p = s_item;
        if (p >= total) break;
        tp_item<L1, L2, R>(p, in, out, work, sync, desc, desc_step, count, lag, slots, idx, status,
                           tw1, tw2, smem);
    }
}

// Grid of the persistent kernel on the current device (resident CTAs).
template <int L1, int L2, class R>
cudaError_t pt_grid(int64_t* grid) {
    using P = pt_shape<L1, L2, R>;
    auto kern = k_xft_twopass<L1, L2, R>;
    static int per_sm[64] = {}, sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!per_sm[dev]) {
        if (P::SMEM > 48 * 1024 &&
            (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM)) != cudaSuccess)
            return e;
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, PT_THREADS, P::SMEM)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        per_sm[dev] = nb > 0 ? nb : 1;
    }
    *grid = (int64_t)per_sm[dev] * sms[dev];
    return cudaSuccess;
}

// Lag D (signals) and ring slots W = D + 2 for `count` signals: the B tiles
// trail by about twice the number of tiles in flight (measured on GB300 at
// N = 65536: 1x, 2x, 4x, 8x gave 0.40, 0.37, 0.38, 0.41 ms per 64M points).
template <int L1, int L2, class R>
cudaError_t pt_ring(int64_t count, int64_t* lag, int64_t* slots) {
    using P = pt_shape<L1, L2, R>;
    int64_t grid = 0;
    cudaError_t e = pt_grid<L1, L2, R>(&grid);
    if (e != cudaSuccess) return e;
    int64_t d = (2 * grid + (P::CB + P::RB) - 1) / (P::CB + P::RB);
    if (d < 2) d = 2;
    if (d > count) d = count;
    *lag = d;
    *slots = d + 2;
    return cudaSuccess;
}

template <int L1, int L2, class R>
cudaError_t launch_pt(const void* in, void* out, void* work, int32_t* sync, const lct_desc* desc,
                      int desc_step, int64_t count, const int32_t* idx, int32_t* status,
                      const void* tw1, const void* tw2, cudaStream_t stream) {
    using P = pt_shape<L1, L2, R>;
    int64_t grid = 0, lag = 0, slots = 0;
    cudaError_t e = pt_grid<L1, L2, R>(&grid);
    if (e != cudaSuccess) return e;
    if ((e = pt_ring<L1, L2, R>(count, &lag, &slots)) != cudaSuccess) return e;
    const int64_t total = count * (P::CB + P::RB);
    if (grid > total) grid = total;
    if ((e = cudaMemsetAsync(sync, 0, (size_t)(4 + 2 * slots) * sizeof(int32_t), stream)) != cudaSuccess)
        return e;
    k_xft_twopass<L1, L2, R><<<(unsigned)grid, PT_THREADS, P::SMEM, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)out, (cpx<R>*)work, sync, desc, desc_step, count, lag, slots,
        idx, status, (const cpx<R>*)tw1, (const cpx<R>*)tw2);
    return cudaGetLastError();
}

#define LCT_TP_SIZES(X, R) \
    case 13: X(6, 7, R)    \
    case 14: X(7, 7, R)    \
    case 15: X(7, 8, R)    \
    case 16: X(8, 8, R)

}  // namespace

bool lct_twopass_supported(int dtype, int log2n) {
    (void)dtype;
    return log2n >= 13 && log2n <= 16;
}

void lct_twopass_split(int log2n, int* l1, int* l2) {
    *l1 = log2n / 2;
    *l2 = log2n - log2n / 2;
}

// Ring workspace of the persistent form: `slots` signals of N samples, plus
// (4 + 2 slots) int32 of queue, abort flag and counters.
cudaError_t lct_twopass_ring(int dtype, int log2n, int64_t count, int64_t* slots) {
    int64_t lag = 0;
    *slots = 0;
    if (count <= 0) return cudaSuccess;
#define LCT_TP_RING(A, B, R) return pt_ring<A, B, R>(count, &lag, slots);
    if (dtype == 0) {
        switch (log2n) { LCT_TP_SIZES(LCT_TP_RING, float) default: return cudaErrorInvalidValue; }
    }
    switch (log2n) { LCT_TP_SIZES(LCT_TP_RING, double) default: return cudaErrorInvalidValue; }
#undef LCT_TP_RING
}

cudaError_t lct_launch_twopass(int dtype, int log2n, const void* in, void* out, void* work,
                               int32_t* sync, const lct_desc* desc, int desc_step, int64_t count,
                               const int32_t* idx, int32_t* status, const void* tw1,
                               const void* tw2, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
#define LCT_TP_LAUNCH(A, B, R) \
    return launch_pt<A, B, R>(in, out, work, sync, desc, desc_step, count, idx, status, tw1, tw2, stream);
    if (dtype == 0) {
        switch (log2n) { LCT_TP_SIZES(LCT_TP_LAUNCH, float) default: return cudaErrorInvalidValue; }
    }
    switch (log2n) { LCT_TP_SIZES(LCT_TP_LAUNCH, double) default: return cudaErrorInvalidValue; }
#undef LCT_TP_LAUNCH
}
