// XFT for N that is not a power of two (Sec. 3: the Algorithm's DFT is "any
// FFT").  The kernel e^{-i pi m_j m_k / (2N)} of the factorisation splits
// exactly into two chirps and a convolution with h_n = e^{i pi n^2 / N}
// (lct_internal.h), so one CTA per signal computes, on a shared-memory tile
// of M = 2^L >= 2N - 1 samples:
//   pre-chirp (samples k < N, zeros above) -> forward DFT_M -> times the
//   kernel spectrum H/M -> inverse DFT_M -> post-chirp + scale (j < N),
// a circular convolution of length M that equals the linear one for j < N
// (Bluestein's algorithm).  Each sample is read from HBM once and written
// once; the spectrum table (M complex values per N) is shared by every
// signal of that N and stays in L2.  Both DFTs are the Stockham engine of
// xft_engine.cuh.  Sizes: N <= 8192 (complex64, M <= 16384), N <= 4096
// (complex128, M <= 8192).
#include "xft_engine.cuh"
#include "xft_chirp.cuh"

namespace {

using namespace xft;

template <int L>
struct blue_shape {
    static constexpr int T = shape<L>::T;
    static constexpr int SPC = T >= 256 ? 1 : 256 / T;     // signals per CTA
    static constexpr int THREADS = T * SPC;
};

// Resident threads per SM the register budget is sized for: 1024 (64
// registers a thread).  The two DFTs then spill a few hundred bytes to L1,
// but twice the warps hide more latency: measured 10-11% faster at M = 8192
// than 512 threads at 128 registers without spills.
template <int L, class R>
constexpr int blue_min_blocks() {
    constexpr int per_sm = 1024;
    constexpr int b = per_sm / blue_shape<L>::THREADS;
    return b > 0 ? b : 1;
}

// e^{2 pi i [phi m^2 + off]} with m = 2k - n + 1 (|m| < 2^16), phi the
// descriptor's turn fraction (64 bits for FP32, 128 for FP64).
template <class R>
__device__ __forceinline__ cpx<R> chirp_any(uint64_t phi_hi, uint64_t phi_lo, uint64_t off, int k,
                                            int n) {
    const uint32_t m2 = m_squared(k, n);
    if constexpr (sizeof(R) == 4)
        return expi_turn32<true>(phase32(phi_hi, m2) + (uint32_t)((off + 0x80000000ull) >> 32));
    else
        return expi_turn64(phase64(phi_hi, phi_lo, m2) + off);
}

template <class R>
__device__ __forceinline__ cpx<R> ld_spec(const cpx<R>* p) {
    return ld_tw<R>(p);
}

// MEH: kind LCT_KIND_MEHLER (output weight with its magnitude, optional
// reversal); a separate instantiation, so the LCT path keeps its registers.
template <int L, class R, bool MEH>
__global__ void __launch_bounds__(blue_shape<L>::THREADS, (blue_min_blocks<L, R>()))
k_xft_blue(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
           const lct_desc* __restrict__ desc, int desc_step, int64_t count, int n,
           const cpx<R>* __restrict__ tw, const cpx<R>* __restrict__ spec,
           const int32_t* __restrict__ idx, int32_t* __restrict__ status) {
    using S = shape<L>;
    using F = blue_shape<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int sl = tid / S::T;
    const int i = tid - sl * S::T;
    const int64_t sig = (int64_t)blockIdx.x * F::SPC + sl;
    bool active = sig < count;
    const int64_t gsig = idx ? (active ? idx[sig] : 0) : sig;
    const lct_desc* Dp = desc + (desc_step && active ? gsig : 0);
    if (active && (Dp->kind != (MEH ? LCT_KIND_MEHLER : LCT_KIND_BLUE) || Dp->n != n ||
                   Dp->log2n != L || Dp->offset < 0)) {
        if (i == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        active = false;
    }
    const int64_t base = desc_step ? Dp->offset : sig * (int64_t)n;
    buf += sl * S::NP;

    cpx<R> v[S::E];
    // load samples k < N with the pre-chirp; the rest of the tile is zero.
    // (The descriptor is read where it is used, not held in registers across
    // the two DFTs, which would spill at this register budget.)
    {
        const uint64_t in_hi = Dp->in_hi, in_lo = Dp->in_lo;
        const bool decay = (Dp->flags & LCT_FLAG_DECAY) != 0;
        const double dec = Dp->decay;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int k = i + e * S::T;
            cpx<R> f = {R(0), R(0)};
            if (active && k < n) {
                f = ld_stream(in + base + k);
                cpx<R> w = chirp_any<R>(in_hi, in_lo, 0, k, n);
                if (decay) {
                    const uint32_t m2 = m_squared(k, n);
                    if constexpr (sizeof(R) == 4) w = cscale(w, expf(-(float)dec * (float)m2));
                    else w = cscale(w, exp(-dec * (double)m2));
                }
                f = cmul(f, w);
            }
            v[e] = f;
        }
    }
    // Circular convolution with h: DFT_M, times the spectrum of h (already
    // divided by M), inverse DFT_M.  The inverse is taken as
    // conj(DFT_M(conj(.))), so both transforms are the same forward DFT run
    // by a two-trip loop the compiler keeps rolled: one copy of the engine's
    // code, and the register footprint of a single DFT.  Twiddles are
    // computed in registers (one sincospi per butterfly group and a product
    // tree), not read from the table: 8-10% faster here, where the table
    // loads stalled the few resident warps.
#pragma unroll 1
    for (int round = 0; round < 2; ++round) {
        dft_signal<L, -1, true>(v, buf, i, tw);
        if (round == 0) {
#pragma unroll
            for (int e = 0; e < S::E; ++e) {
                const cpx<R> y = cmul(v[e], ld_spec<R>(spec + i + e * S::T));
                v[e] = {y.x, -y.y};
            }
            __syncthreads();          // the first DFT's last exchange is fully read
        }
    }
    if (MEH && active) {
        const uint64_t out_hi = Dp->out_hi, out_lo = Dp->out_lo, out_c = Dp->out_c;
        const R sc = (R)Dp->scale;
        const int fl = Dp->flags;
        const bool odecay = (fl & LCT_FLAG_OUT_DECAY) != 0;   // kind LCT_KIND_MEHLER
        const int rev = (fl & LCT_FLAG_REVERSE) ? n - 1 : 0;
        const double dec = Dp->decay;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int j = i + e * S::T;
            const cpx<R> y = {v[e].x, -v[e].y};         // the conj of the inverse's form
            if (j < n) {
                cpx<R> w = chirp_any<R>(out_hi, out_lo, out_c, j, n);
                if (odecay) {
                    const uint32_t m2 = m_squared(j, n);
                    if constexpr (sizeof(R) == 4) w = cscale(w, expf(-(float)dec * (float)m2));
                    else w = cscale(w, exp(-dec * (double)m2));
                }
                out[base + (rev ? rev - j : j)] = cscale(cmul(y, w), sc);
            }
        }
    } else if (active) {
        const uint64_t out_hi = Dp->out_hi, out_lo = Dp->out_lo, out_c = Dp->out_c;
        const R sc = (R)Dp->scale;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int j = i + e * S::T;
            const cpx<R> y = {v[e].x, -v[e].y};         // the conj of the inverse's form
            if (j < n) out[base + j] = cscale(cmul(y, chirp_any<R>(out_hi, out_lo, out_c, j, n)), sc);
        }
    }
}

template <int L, class R, bool MEH>
cudaError_t launch_blue_l(int n, const void* in, void* out, const lct_desc* desc, int desc_step,
                          int64_t count, const void* tw, const void* spec, const int32_t* idx,
                          int32_t* status, cudaStream_t stream) {
    using S = shape<L>;
    using F = blue_shape<L>;
    const size_t smem = S::P > 1 ? (size_t)F::SPC * S::NP * sizeof(cpx<R>) : 0;
    auto kern = k_xft_blue<L, R, MEH>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (count + F::SPC - 1) / F::SPC;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, F::THREADS, smem, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)out, desc, desc_step, count, n, (const cpx<R>*)tw,
        (const cpx<R>*)spec, idx, status);
    return cudaGetLastError();
}

template <class R, bool MEH>
cudaError_t blue_dispatch(int n, const void* in, void* out, const lct_desc* desc, int desc_step,
                          int64_t count, const void* tw, const void* spec, const int32_t* idx,
                          int32_t* status, cudaStream_t stream) {
    switch (lct_blue_log2m(n)) {
#define LCT_CASE(L) \
    case L: return launch_blue_l<L, R, MEH>(n, in, out, desc, desc_step, count, tw, spec, idx, status, stream);
        LCT_CASE(2) LCT_CASE(3) LCT_CASE(4) LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8)
        LCT_CASE(9) LCT_CASE(10) LCT_CASE(11) LCT_CASE(12) LCT_CASE(13)
#undef LCT_CASE
        case 14:
            if constexpr (sizeof(R) == 4)
                return launch_blue_l<14, R, MEH>(n, in, out, desc, desc_step, count, tw, spec, idx,
                                                 status, stream);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

// Kernel spectrum of the complex-z fractional transform on the nodes (kind
// LCT_KIND_MEHLER, lct_internal.h): one CTA forms h_l = e^{-a_h l^2}
// e^{2 pi i phi_h l^2} at the circular positions of the lags |l| < n (the
// phase from the exact turn fraction, the magnitude in FP64), takes DFT_M
// with the same engine, and stores c/M times it.  Thread 0 also stores the
// signal descriptor and clears the status word, so the host needs no copy.
template <int L, class R>
__global__ void __launch_bounds__(shape<L>::T)
k_mehler_spectrum(int n, double a_h, uint64_t phi_hi, uint64_t phi_lo, double c_re, double c_im,
                  const lct_desc D, lct_desc* __restrict__ d_desc, cpx<R>* __restrict__ spec,
                  int32_t* __restrict__ status, const cpx<R>* __restrict__ tw) {
    using S = shape<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
    const int i = threadIdx.x;
    if (i == 0) {
        *d_desc = D;
        *status = LCT_DEV_OK;
    }
    cpx<R> v[S::E];
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int t = i + e * S::T;
        const int l = t < n ? t : (t > S::N - n ? t - S::N : 0x40000000);
        cpx<R> h = {R(0), R(0)};
        if (l != 0x40000000) {
            const uint32_t l2 = (uint32_t)(l * l);
            const cpx<double> w = expi_turn64(phase64(phi_hi, phi_lo, l2));
            const double mag = exp(-a_h * (double)l2);
            h = {(R)(w.x * mag), (R)(w.y * mag)};
        }
        v[e] = h;
    }
    dft_signal<L, -1, true>(v, buf, i, tw);
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const double x = (double)v[e].x, y = (double)v[e].y;
        spec[i + e * S::T] = {(R)(x * c_re - y * c_im), (R)(x * c_im + y * c_re)};
    }
}

template <int L, class R>
cudaError_t launch_mehler_spec_l(int n, double a_h, uint64_t phi_hi, uint64_t phi_lo, double c_re,
                                 double c_im, const lct_desc& D, lct_desc* d_desc, void* spec,
                                 int32_t* status, const void* tw, cudaStream_t stream) {
    using S = shape<L>;
    const size_t smem = S::P > 1 ? (size_t)S::NP * sizeof(cpx<R>) : 0;
    auto kern = k_mehler_spectrum<L, R>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const double inv_m = 1.0 / (double)S::N;
    kern<<<1, S::T, smem, stream>>>(n, a_h, phi_hi, phi_lo, c_re * inv_m, c_im * inv_m, D, d_desc,
                                    (cpx<R>*)spec, status, (const cpx<R>*)tw);
    return cudaGetLastError();
}

template <class R>
cudaError_t mehler_spec_dispatch(int n, double a_h, uint64_t phi_hi, uint64_t phi_lo, double c_re,
                                 double c_im, const lct_desc& D, lct_desc* d_desc, void* spec,
                                 int32_t* status, const void* tw, cudaStream_t stream) {
    switch (lct_blue_log2m(n)) {
#define LCT_CASE(L)                                                                                \
    case L:                                                                                        \
        return launch_mehler_spec_l<L, R>(n, a_h, phi_hi, phi_lo, c_re, c_im, D, d_desc, spec, status, \
                                          tw, stream);
        LCT_CASE(2) LCT_CASE(3) LCT_CASE(4) LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8)
        LCT_CASE(9) LCT_CASE(10) LCT_CASE(11) LCT_CASE(12) LCT_CASE(13)
#undef LCT_CASE
        case 14:
            if constexpr (sizeof(R) == 4)
                return launch_mehler_spec_l<14, R>(n, a_h, phi_hi, phi_lo, c_re, c_im, D, d_desc, spec,
                                                   status, tw, stream);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

// b == 0 for N that is not a power of two: G_j = scale e^{2 pi i [phi_out m_j^2 + c_out]} f_j,
// one CTA per signal (grid-stride over signals), threads over samples.
template <class R>
__global__ void k_diag_any(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                           const lct_desc* __restrict__ desc, int desc_step, int64_t count, int n,
                           const int32_t* __restrict__ idx, int32_t* __restrict__ status) {
    for (int64_t s = blockIdx.x; s < count; s += gridDim.x) {
        const lct_desc& D = desc[desc_step ? (idx ? idx[s] : s) : 0];
        if (D.kind != LCT_KIND_DIAGN || D.n != n || D.offset < 0) {
            if (threadIdx.x == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
            continue;
        }
        const int64_t base = desc_step ? D.offset : s * (int64_t)n;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const cpx<R> w = chirp_any<R>(D.out_hi, D.out_lo, D.out_c, j, n);
            out[base + j] = cscale(cmul(in[base + j], w), (R)D.scale);
        }
    }
}

}  // namespace

cudaError_t lct_launch_blue(int dtype, int64_t n, const void* in, void* out, const lct_desc* desc,
                            int desc_step, int64_t count, const void* tw, const void* spec,
                            const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (!lct_blue_supported(dtype, n) || !spec) return cudaErrorInvalidValue;
    if (dtype == 0)
        return blue_dispatch<float, false>((int)n, in, out, desc, desc_step, count, tw, spec, idx,
                                           status, stream);
    return blue_dispatch<double, false>((int)n, in, out, desc, desc_step, count, tw, spec, idx,
                                        status, stream);
}

static bool mehler_size_ok(int dtype, int64_t n) {
    return n >= 2 && n <= (dtype == 0 ? kBlueMaxN64 : kBlueMaxN128);
}

cudaError_t lct_launch_mehler(int dtype, int64_t n, const void* in, void* out, const lct_desc* desc,
                              int64_t count, const void* tw, const void* spec, int32_t* status,
                              cudaStream_t stream) {
    if (!mehler_size_ok(dtype, n) || !spec) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    if (dtype == 0)
        return blue_dispatch<float, true>((int)n, in, out, desc, 0, count, tw, spec, nullptr, status,
                                          stream);
    return blue_dispatch<double, true>((int)n, in, out, desc, 0, count, tw, spec, nullptr, status,
                                       stream);
}

cudaError_t lct_launch_mehler_spectrum(int dtype, int64_t n, double a_h, uint64_t phi_hi,
                                       uint64_t phi_lo, double c_re, double c_im,
                                       const lct_desc& D, lct_desc* d_desc, void* spec,
                                       int32_t* status, const void* tw, cudaStream_t stream) {
    if (!mehler_size_ok(dtype, n) || !spec || !d_desc || !status) return cudaErrorInvalidValue;
    if (dtype == 0)
        return mehler_spec_dispatch<float>((int)n, a_h, phi_hi, phi_lo, c_re, c_im, D, d_desc, spec,
                                           status, tw, stream);
    return mehler_spec_dispatch<double>((int)n, a_h, phi_hi, phi_lo, c_re, c_im, D, d_desc, spec,
                                        status, tw, stream);
}

cudaError_t lct_launch_diag_any(int dtype, int64_t n, const void* in, void* out,
                                const lct_desc* desc, int desc_step, int64_t count,
                                const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(count < 152 * 16 ? count : 152 * 16);
    const int th = n >= 256 ? 256 : 64;
    if (dtype == 0)
        k_diag_any<float><<<grid, th, 0, stream>>>((const cpx<float>*)in, (cpx<float>*)out, desc,
                                                   desc_step, count, (int)n, idx, status);
    else
        k_diag_any<double><<<grid, th, 0, stream>>>((const cpx<double>*)in, (cpx<double>*)out, desc,
                                                    desc_step, count, (int)n, idx, status);
    return cudaGetLastError();
}
