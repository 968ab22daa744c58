// Fused XFT kernel: pre-chirp -> N-point DFT -> post-chirp + scale, with the
// whole signal resident in registers and shared memory, so each sample is
// read from HBM once and written once (Sec. 3, Algorithm, steps 1-3; the DFT
// with the forward sign, see include/lct.h).
//
// DFT: self-sorting Stockham formulation.  Every thread owns E = 16 samples
// (E = N for N < 16), T = N/E threads per signal.  Pass p has radix R_p
// (first pass 2^(log2N mod 4) or 16, then 16) and sub-length Ns_p (product
// of the previous radices).  In every pass thread i holds the samples
// i + e T (e = 0..15) -- the coalesced pattern, so the first pass reads
// global memory directly and the last pass writes it directly -- applies
// twiddles e^{-2 pi i j k / (Ns R)} (k = i' mod Ns) and a radix-R DFT in
// registers, and writes sample j of virtual thread i' to position
// (i' - k) R + k + j Ns.  Shared memory is padded by one slot per 16 so
// that every exchange is free of bank conflicts.
#include "xft_common.cuh"

namespace {

constexpr int pass_count(int L) { return L >= 4 ? (L + 3) / 4 : 1; }
constexpr int first_radix(int L) { return 1 << (L - 4 * (pass_count(L) - 1)); }
__host__ __device__ constexpr int pad_idx(int i) { return i + (i >> 4); }

template <int L>
struct xft_shape {
    static constexpr int N = 1 << L;
    static constexpr int E = L >= 4 ? 16 : N;
    static constexpr int T = N / E;
    static constexpr int SPC = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = T * SPC;
    static constexpr int NP = N + (N >> 4);
    static constexpr int P = pass_count(L);
};

template <int L, int p>
struct pass_info {
    static constexpr int RADIX = p == 0 ? first_radix(L) : 16;
    static constexpr int NS = p == 0 ? 1 : first_radix(L) << (4 * (p - 1));
    static constexpr int ns() { return NS; }
};

// e^{SGN 2 pi i k / M} (M a power of two, so 2k/M is exact).
template <class R, int SGN>
__device__ __forceinline__ cpx<R> twiddle_base(int k, int M) {
    R s, c;
    if constexpr (sizeof(R) == 4) sincospif((float)(2 * k) / (float)M, &s, &c);
    else sincospi((double)(2 * k) / (double)M, &s, &c);
    return {c, SGN < 0 ? -s : s};
}

// Twiddles + radix-R DFTs of one pass on the registers of thread i.
template <int RADIX, int NS, int E, int T, int SGN, class R>
__device__ __forceinline__ void butterflies(cpx<R>* v, int i) {
    constexpr int V = E / RADIX;
#pragma unroll
    for (int vv = 0; vv < V; ++vv) {
        cpx<R> u[RADIX];
#pragma unroll
        for (int j = 0; j < RADIX; ++j) u[j] = v[vv + j * V];
        if (NS > 1) {
            const int ip = i + vv * T;
            const int k = ip & (NS - 1);
            cpx<R> w[RADIX];
            twiddle_powers<RADIX>(twiddle_base<R, SGN>(k, NS * RADIX), w);
#pragma unroll
            for (int j = 1; j < RADIX; ++j) u[j] = cmul(u[j], w[j]);
        }
        dft<RADIX, SGN>(u);
#pragma unroll
        for (int j = 0; j < RADIX; ++j) v[vv + j * V] = u[j];
    }
}

template <int RADIX, int NS, int E, int T, class R>
__device__ __forceinline__ void stockham_store(const cpx<R>* v, cpx<R>* buf, int i) {
    constexpr int V = E / RADIX;
#pragma unroll
    for (int vv = 0; vv < V; ++vv) {
        const int ip = i + vv * T;
        const int k = ip & (NS - 1);
        const int base = (ip - k) * RADIX + k;
#pragma unroll
        for (int j = 0; j < RADIX; ++j) buf[pad_idx(base + j * NS)] = v[vv + j * V];
    }
}

template <int E, int T, class R>
__device__ __forceinline__ void stockham_load(cpx<R>* v, const cpx<R>* buf, int i) {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = buf[pad_idx(i + e * T)];
}

// Passes 1..P-1 (pass 0 is done by the caller right after the global load).
template <int L, int p, int SGN, class R>
struct run_passes {
    __device__ __forceinline__ static void go(cpx<R>* v, cpx<R>* buf, int i) {
        using S = xft_shape<L>;
        using PP = pass_info<L, p - 1>;
        using PI = pass_info<L, p>;
        // results of pass p-1 -> shared memory
        __syncthreads();
        stockham_store<PP::RADIX, PP::NS, S::E, S::T>(v, buf, i);
        __syncthreads();
        stockham_load<S::E, S::T>(v, buf, i);
        butterflies<PI::RADIX, PI::NS, S::E, S::T, SGN>(v, i);
        run_passes<L, p + 1, SGN, R>::go(v, buf, i);
    }
};
template <int L, int SGN, class R>
struct run_passes<L, xft_shape<L>::P, SGN, R> {
    __device__ __forceinline__ static void go(cpx<R>*, cpx<R>*, int) {}
};

// Pre-chirp e^{2 pi i [phi_in m^2 + (N-1) n/(2N)]} e^{-decay m^2} of sample n.
template <int L, bool FAST>
__device__ __forceinline__ cpx<float> pre_chirp(const lct_desc& D, int n, bool decay) {
    constexpr uint32_t CEN = (uint32_t)(((1u << L) - 1u) << (31 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    cpx<float> w = expi_turn32<FAST>(phase32(D.in_hi, m2) + (uint32_t)n * CEN);
    if (decay) w = cscale(w, expf(-(float)D.decay * (float)m2));
    return w;
}
template <int L, bool FAST>
__device__ __forceinline__ cpx<double> pre_chirp64(const lct_desc& D, int n, bool decay) {
    constexpr uint64_t CEN = (uint64_t)(((1ull << L) - 1ull) << (63 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    cpx<double> w = expi_turn64(phase64(D.in_hi, D.in_lo, m2) + (uint64_t)n * CEN);
    if (decay) w = cscale(w, exp(-D.decay * (double)m2));
    return w;
}
template <int L, bool FAST>
__device__ __forceinline__ cpx<float> post_chirp(const lct_desc& D, int n) {
    constexpr uint32_t CEN = (uint32_t)(((1u << L) - 1u) << (31 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
    return expi_turn32<FAST>(phase32(D.out_hi, m2) + (uint32_t)n * CEN + off);
}
template <int L, bool FAST>
__device__ __forceinline__ cpx<double> post_chirp64(const lct_desc& D, int n) {
    constexpr uint64_t CEN = (uint64_t)(((1ull << L) - 1ull) << (63 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    return expi_turn64(phase64(D.out_hi, D.out_lo, m2) + (uint64_t)n * CEN + D.out_c);
}

template <int L, class R, bool FAST>
__device__ __forceinline__ cpx<R> pre_w(const lct_desc& D, int n, bool decay) {
    if constexpr (sizeof(R) == 4) return pre_chirp<L, FAST>(D, n, decay);
    else return pre_chirp64<L, FAST>(D, n, decay);
}
template <int L, class R, bool FAST>
__device__ __forceinline__ cpx<R> post_w(const lct_desc& D, int n) {
    if constexpr (sizeof(R) == 4) return post_chirp<L, FAST>(D, n);
    else return post_chirp64<L, FAST>(D, n);
}

template <int L, class R, bool FAST>
__global__ void __launch_bounds__(xft_shape<L>::THREADS)
k_xft_fused(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
            const lct_desc* __restrict__ desc, int desc_step, int64_t count) {
    using S = xft_shape<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int sl = tid / S::T;
    const int i = tid - sl * S::T;
    const int64_t sig = (int64_t)blockIdx.x * S::SPC + sl;
    const bool active = sig < count;
    const lct_desc D = desc[desc_step && active ? sig : 0];
    const int64_t base = desc_step ? D.offset : sig * (int64_t)S::N;
    cpx<R>* buf = smem + sl * S::NP;
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;

    cpx<R> v[S::E];
    // global load (coalesced: sample i + e T) with the pre-chirp
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int n = i + e * S::T;
        cpx<R> f = {R(0), R(0)};
        if (active) f = in[base + n];
        v[e] = cmul(f, pre_w<L, R, FAST>(D, n, decay));
    }
    butterflies<pass_info<L, 0>::RADIX, pass_info<L, 0>::ns(), S::E, S::T, -1>(v, i);
    run_passes<L, 1, -1, R>::go(v, buf, i);
    // global store (sample i + e T) with the post-chirp and scale
    if (active) {
        const R sc = (R)D.scale;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            out[base + n] = cscale(cmul(v[e], post_w<L, R, FAST>(D, n)), sc);
        }
    }
}

template <int L, class R>
cudaError_t launch_one(const void* in, void* out, const lct_desc* desc, int desc_step,
                       int64_t count, cudaStream_t stream) {
    using S = xft_shape<L>;
    const size_t smem = S::P > 1 ? (size_t)S::SPC * S::NP * sizeof(cpx<R>) : 0;
    auto kern = k_xft_fused<L, R, true>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (count + S::SPC - 1) / S::SPC;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, S::THREADS, smem, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)out, desc, desc_step, count);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_dispatch(int log2n, const void* in, void* out, const lct_desc* desc,
                            int desc_step, int64_t count, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_one<L, R>(in, out, desc, desc_step, count, stream);
        LCT_CASE(1) LCT_CASE(2) LCT_CASE(3) LCT_CASE(4) LCT_CASE(5) LCT_CASE(6)
        LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10) LCT_CASE(11) LCT_CASE(12)
#undef LCT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool lct_fused_supported(int dtype, int log2n) {
    (void)dtype;
    return log2n >= 1 && log2n <= 12;
}

cudaError_t lct_launch_fused(int dtype, int log2n, const void* in, void* out,
                             const lct_desc* desc, int desc_step, int64_t count,
                             cudaStream_t stream) {
    if (dtype == 0) return launch_dispatch<float>(log2n, in, out, desc, desc_step, count, stream);
    return launch_dispatch<double>(log2n, in, out, desc, desc_step, count, stream);
}
