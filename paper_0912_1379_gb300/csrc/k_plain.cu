// Element-wise kernels: the b = 0 branch (a diagonal transform, definition
// below eq. (lctuno)) and the two chirp kernels of the plain FP64 baseline
// (chirp -> library FFT -> chirp + scale, unfused, FP64 workspace).
// All phases are the exact fixed-point turn fractions of the descriptor.
#include "xft_common.cuh"

namespace {

template <class R>
__device__ __forceinline__ cpx<double> load_c128(const cpx<R>* p, int64_t i) {
    cpx<R> v = p[i];
    return {(double)v.x, (double)v.y};
}

// b = 0: G_j = scale e^{2 pi i [phi_out m_j^2 + c_out]} f_j
// idx (may be null): signal s of this launch is descriptor idx[s] (ragged
// groups of equal N); mismatching descriptors are skipped and flagged.
template <class R>
__global__ void k_diag(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                       const lct_desc* __restrict__ desc, int desc_step, int64_t count, int log2n,
                       const int32_t* __restrict__ idx, int32_t* __restrict__ status) {
    const int64_t N = 1ll << log2n;
    const int64_t total = count * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sig = t >> log2n;
        const int n = (int)(t & (N - 1));
        const lct_desc& D = desc[desc_step ? (idx ? idx[sig] : sig) : 0];
        if (idx && (D.kind != LCT_KIND_DIAG || D.log2n != log2n || D.offset < 0)) {
            if (n == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
            continue;
        }
        const int64_t base = desc_step ? D.offset : sig * N;
        const uint32_t m2 = m_squared(n, (int)N);
        if constexpr (sizeof(R) == 4) {
            const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
            cpx<float> w = expi_turn32<true>(phase32(D.out_hi, m2) + off);
            out[base + n] = cscale(cmul(in[base + n], w), (float)D.scale);
        } else {
            cpx<double> w = expi_turn64(phase64(D.out_hi, D.out_lo, m2) + D.out_c);
            cpx<double> g = cscale(cmul(load_c128(in, base + n), w), D.scale);
            out[base + n] = {(R)g.x, (R)g.y};
        }
    }
}

// b = 0 over the ragged list of every diagonal signal of a batch, one launch:
// chunk c = {pos, start, log2n, nsig} covers elements start .. start + 2047
// of signal idx[pos] (nsig == 1, N >= 2048) or the nsig whole signals
// idx[pos .. pos + nsig - 1] of equal N (nsig N <= 2048).  Mismatching
// descriptors are skipped and flagged.
template <class R>
__global__ void k_diag_chunks(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                              const lct_desc* __restrict__ desc, const int32_t* __restrict__ idx,
                              const int4* __restrict__ chunks, int64_t nchunks,
                              int32_t* __restrict__ status) {
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int4 ch = chunks[c];
        const int L = ch.z, N = 1 << L;
        const int len = ch.w > 1 ? (ch.w << L) : min(N - ch.y, kDiagChunk);
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int j = ch.w > 1 ? (e >> L) : 0;
            const int n = ch.w > 1 ? (e & (N - 1)) : ch.y + e;
            const lct_desc& D = desc[idx[ch.x + j]];
            if (D.kind != LCT_KIND_DIAG || D.log2n != L || D.offset < 0) {
                if (n == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
                continue;
            }
            const uint32_t m2 = m_squared(n, N);
            if constexpr (sizeof(R) == 4) {
                const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
                cpx<float> w = expi_turn32<true>(phase32(D.out_hi, m2) + off);
                out[D.offset + n] = cscale(cmul(in[D.offset + n], w), (float)D.scale);
            } else {
                cpx<double> w = expi_turn64(phase64(D.out_hi, D.out_lo, m2) + D.out_c);
                cpx<double> g = cscale(cmul(load_c128(in, D.offset + n), w), D.scale);
                out[D.offset + n] = {(R)g.x, (R)g.y};
            }
        }
    }
}

// Debug scan for NaN / infinite samples, one CTA per signal (grid-stride).
template <class R>
__global__ void k_scan(const cpx<R>* __restrict__ out, const lct_desc* __restrict__ desc,
                       int desc_step, int64_t count, int64_t len, int32_t* __restrict__ status) {
    for (int64_t s = blockIdx.x; s < count; s += gridDim.x) {
        const int64_t nn = desc_step ? desc[s].n : len;
        const int64_t base = desc_step ? desc[s].offset : s * len;
        bool bad = false;
        for (int64_t n = threadIdx.x; n < nn; n += blockDim.x) {
            const cpx<R> v = out[base + n];
            bad |= !isfinite(v.x) || !isfinite(v.y);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_NONFINITE);
    }
}

// plain path, step 1: u_k = e^{2 pi i [phi_in m^2 + (N-1)k/(2N)]} e^{-decay m^2} f_k (FP64)
template <class R>
__global__ void k_plain_pre(const cpx<R>* __restrict__ in, cpx<double>* __restrict__ work,
                            const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                            int log2n) {
    const int64_t N = 1ll << log2n;
    const int64_t total = count * N;
    const uint64_t cen = (uint64_t)(N - 1) << (63 - log2n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sig = t >> log2n;
        const int n = (int)(t & (N - 1));
        const lct_desc& D = desc[desc_step ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * N;
        const uint32_t m2 = m_squared(n, (int)N);
        cpx<double> w = expi_turn64(phase64(D.in_hi, D.in_lo, m2) + (uint64_t)n * cen);
        if (D.flags & LCT_FLAG_DECAY) w = cscale(w, exp(-D.decay * (double)m2));
        work[t] = cmul(load_c128(in, base + n), w);
    }
}

// plain path, step 3: G_j = scale e^{2 pi i [phi_out m^2 + (N-1)j/(2N) + c_out]} U_j
template <class R>
__global__ void k_plain_post(const cpx<double>* __restrict__ work, cpx<R>* __restrict__ out,
                             const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                             int log2n) {
    const int64_t N = 1ll << log2n;
    const int64_t total = count * N;
    const uint64_t cen = (uint64_t)(N - 1) << (63 - log2n);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sig = t >> log2n;
        const int n = (int)(t & (N - 1));
        const lct_desc& D = desc[desc_step ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * N;
        const uint32_t m2 = m_squared(n, (int)N);
        cpx<double> w =
            expi_turn64(phase64(D.out_hi, D.out_lo, m2) + (uint64_t)n * cen + D.out_c);
        cpx<double> g = cscale(cmul(work[t], w), D.scale);
        out[base + n] = {(R)g.x, (R)g.y};
    }
}

// Plain FP32 path (complex64 plans): the same two chirp kernels in FP32 with
// the 64-bit phase words, around a single-precision library FFT (C2C), so
// that the fused kernel can be compared with an unfused path of the same
// arithmetic precision.
__global__ void k_plain_pre32(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ work,
                              const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                              int log2n) {
    const int64_t N = 1ll << log2n;
    const int64_t total = count * N;
    const uint32_t cen = (uint32_t)((N - 1) << (31 - log2n));      // (N-1)/(2N) turns
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sig = t >> log2n;
        const int n = (int)(t & (N - 1));
        const lct_desc& D = desc[desc_step ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * N;
        const uint32_t m2 = m_squared(n, (int)N);
        cpx<float> w = expi_turn32<true>(phase32(D.in_hi, m2) + (uint32_t)n * cen);
        if (D.flags & LCT_FLAG_DECAY) w = cscale(w, expf(-(float)D.decay * (float)m2));
        work[t] = cmul(in[base + n], w);
    }
}

__global__ void k_plain_post32(const cpx<float>* __restrict__ work, cpx<float>* __restrict__ out,
                               const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                               int log2n) {
    const int64_t N = 1ll << log2n;
    const int64_t total = count * N;
    const uint32_t cen = (uint32_t)((N - 1) << (31 - log2n));
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sig = t >> log2n;
        const int n = (int)(t & (N - 1));
        const lct_desc& D = desc[desc_step ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * N;
        const uint32_t m2 = m_squared(n, (int)N);
        const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
        cpx<float> w = expi_turn32<true>(phase32(D.out_hi, m2) + (uint32_t)n * cen + off);
        out[base + n] = cscale(cmul(work[t], w), (float)D.scale);
    }
}

unsigned grid_for(int64_t total, int threads) {
    int64_t b = (total + threads - 1) / threads;
    const int64_t cap = 152 * 32;  // grid-stride beyond this
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

cudaError_t lct_launch_diag(int dtype, int log2n, const void* in, void* out,
                            const lct_desc* desc, int desc_step, int64_t count,
                            const int32_t* idx, int32_t* status, cudaStream_t stream) {
    const int64_t total = count << log2n;
    const int th = 256;
    if (dtype == 0)
        k_diag<float><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<float>*)in, (cpx<float>*)out, desc, desc_step, count, log2n, idx, status);
    else
        k_diag<double><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<double>*)in, (cpx<double>*)out, desc, desc_step, count, log2n, idx, status);
    return cudaGetLastError();
}

cudaError_t lct_launch_diag_chunks(int dtype, const void* in, void* out, const lct_desc* desc,
                                   const int32_t* idx, const int32_t* chunks, int64_t nchunks,
                                   int32_t* status, cudaStream_t stream) {
    if (nchunks <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t cap = (int64_t)sms * 8;
    const unsigned grid = (unsigned)(nchunks < cap ? nchunks : cap);
    if (dtype == 0)
        k_diag_chunks<float><<<grid, 256, 0, stream>>>((const cpx<float>*)in, (cpx<float>*)out,
                                                       desc, idx, (const int4*)chunks, nchunks, status);
    else
        k_diag_chunks<double><<<grid, 256, 0, stream>>>((const cpx<double>*)in, (cpx<double>*)out,
                                                        desc, idx, (const int4*)chunks, nchunks, status);
    return cudaGetLastError();
}

cudaError_t lct_launch_scan(int dtype, const void* out, const lct_desc* desc, int desc_step,
                            int64_t count, int64_t len, int32_t* status, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(count < 4096 ? count : 4096);
    if (dtype == 0)
        k_scan<float><<<grid, 256, 0, stream>>>((const cpx<float>*)out, desc, desc_step, count,
                                                len, status);
    else
        k_scan<double><<<grid, 256, 0, stream>>>((const cpx<double>*)out, desc, desc_step, count,
                                                 len, status);
    return cudaGetLastError();
}

cudaError_t lct_launch_plain_pre(int dtype, int log2n, const void* in, void* work,
                                 const lct_desc* desc, int desc_step, int64_t count,
                                 cudaStream_t stream) {
    const int64_t total = count << log2n;
    const int th = 256;
    if (dtype == 0)
        k_plain_pre<float><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<float>*)in, (cpx<double>*)work, desc, desc_step, count, log2n);
    else
        k_plain_pre<double><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<double>*)in, (cpx<double>*)work, desc, desc_step, count, log2n);
    return cudaGetLastError();
}

cudaError_t lct_launch_plain_post(int dtype, int log2n, const void* work, void* out,
                                  const lct_desc* desc, int desc_step, int64_t count,
                                  cudaStream_t stream) {
    const int64_t total = count << log2n;
    const int th = 256;
    if (dtype == 0)
        k_plain_post<float><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<double>*)work, (cpx<float>*)out, desc, desc_step, count, log2n);
    else
        k_plain_post<double><<<grid_for(total, th), th, 0, stream>>>(
            (const cpx<double>*)work, (cpx<double>*)out, desc, desc_step, count, log2n);
    return cudaGetLastError();
}

cudaError_t lct_launch_plain32_pre(const void* in, void* work, const lct_desc* desc, int log2n,
                                   int desc_step, int64_t count, cudaStream_t stream) {
    const int64_t total = count << log2n;
    k_plain_pre32<<<grid_for(total, 256), 256, 0, stream>>>(
        (const cpx<float>*)in, (cpx<float>*)work, desc, desc_step, count, log2n);
    return cudaGetLastError();
}

cudaError_t lct_launch_plain32_post(const void* work, void* out, const lct_desc* desc, int log2n,
                                    int desc_step, int64_t count, cudaStream_t stream) {
    const int64_t total = count << log2n;
    k_plain_post32<<<grid_for(total, 256), 256, 0, stream>>>(
        (const cpx<float>*)work, (cpx<float>*)out, desc, desc_step, count, log2n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise complex conjugate (in == out allowed): the conjugations around
// the forward kernels in the adjoint of plans the backward kernel does not take.
// ---------------------------------------------------------------------------
namespace {
template <class R>
__global__ void k_conj(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const cpx<R> v = in[e];
        out[e] = {v.x, -v.y};
    }
}
}  // namespace

cudaError_t lct_launch_conj(int dtype, const void* in, void* out, int64_t n, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int th = 256;
    if (dtype == 0)
        k_conj<float><<<grid_for(n, th), th, 0, stream>>>((const cpx<float>*)in, (cpx<float>*)out, n);
    else
        k_conj<double><<<grid_for(n, th), th, 0, stream>>>((const cpx<double>*)in, (cpx<double>*)out, n);
    return cudaGetLastError();
}
