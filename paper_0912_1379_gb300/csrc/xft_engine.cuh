// Stockham DFT engine shared by the XFT kernels.
//
// Self-sorting Stockham formulation of the N-point DFT (N = 2^L).  Every
// thread owns E = 2^LE samples (LE = 4 by default, 3 for the low-register
// kernels; E = N for smaller N), T = N/E threads per signal.  Pass p has
// radix R_p (first pass 2^(L mod LE) or E, then E) and sub-length
// Ns_p = product of the previous radices.  In every pass thread i
// holds the samples i + e T (e = 0..E-1) -- the coalesced pattern, so the
// first pass can read global memory directly and the last pass can write it
// directly -- multiplies sample j of its group by the twiddle
// e^{S 2 pi i j k / (Ns R)} (k = i' mod Ns), applies a radix-R DFT in
// registers, and writes sample j of virtual thread i' to position
// (i' - k) R + k + j Ns of the next pass's buffer.  Shared memory is padded
// by one slot per 16 samples, which makes every exchange free of bank
// conflicts (for T >= 16).
//
// Twiddles come from a per-(N, E) table laid out [pass][j-1][k] (see
// lct_twiddle_table), so that the 32 lanes of a warp read 32 consecutive
// entries.  Entry (p, j, k) = e^{-2 pi i j k / (E Ns_p)}; the inverse
// transform (S = +1) uses the conjugate.  Offset of pass p:
// sum_{q<p} (E-1) Ns_q = Ns_p - R_0.
#pragma once
#include "xft_common.cuh"

namespace xft {

constexpr int pass_count(int L, int LE = 4) { return L >= LE ? (L + LE - 1) / LE : 1; }
constexpr int first_radix(int L, int LE = 4) { return 1 << (L - LE * (pass_count(L, LE) - 1)); }
// Shared-memory padding: one slot every 2^PS samples (PS = 4 makes the
// exchanges of 8-byte samples with E = 16 conflict-free; PS = 3 those of
// 16-byte samples with E = 8).
template <int PS = 4>
__host__ __device__ constexpr int pad_idx(int i) { return i + (i >> PS); }
template <int L, int PS = 4>
constexpr int padded_len() { return (1 << L) + ((1 << L) >> PS); }

template <int L, int LE = 4>
struct shape {
    static constexpr int N = 1 << L;
    static constexpr int E = L >= LE ? (1 << LE) : N;
    static constexpr int T = N / E;
    static constexpr int P = pass_count(L, LE);
    static constexpr int NP = N + (N >> 4);
};

template <int L, int p, int LE = 4>
struct pass {
    static constexpr int RADIX = p == 0 ? first_radix(L, LE) : (1 << LE);
    static constexpr int NS = p == 0 ? 1 : first_radix(L, LE) << (LE * (p - 1));
    static constexpr int TW_OFF = NS - first_radix(L, LE);   // sum of (E-1) Ns_q over q < p
};

template <class R>
__device__ __forceinline__ cpx<R> ld_tw(const cpx<R>* p);
template <>
__device__ __forceinline__ cpx<float> ld_tw<float>(const cpx<float>* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
template <>
__device__ __forceinline__ cpx<double> ld_tw<double>(const cpx<double>* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
// broadcast-form entry {(wx, wx), (wy, wy)} for packed pairs
template <>
__device__ __forceinline__ cpx<pf> ld_tw<pf>(const cpx<pf>* p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {pf{make_float2(v.x, v.y)}, pf{make_float2(v.z, v.w)}};
}

// e^{SGN 2 pi i k / M} (M a power of two, so 2k/M is exact), correctly
// rounded library sincospi.
template <class R, int SGN>
__device__ __forceinline__ cpx<R> twiddle_exact(int k, int M) {
    R s, c;
    if constexpr (sizeof(R) == 4) sincospif((float)(2 * k) / (float)M, &s, &c);
    else sincospi((double)(2 * k) / (double)M, &s, &c);
    return {c, SGN < 0 ? -s : s};
}

// Twiddles + radix-R DFTs of pass p on the registers of thread i.
// TWC = false: twiddles read from the table; TWC = true: computed (one
// sincospi for w = e^{S 2 pi i k/(Ns R)}, then powers by a product tree).
template <int L, int p, int SGN, bool TWC, int LE = 4, class R>
__device__ __forceinline__ void butterflies(cpx<R>* v, int i, const cpx<R>* __restrict__ tw) {
    using S = shape<L, LE>;
    using PI = pass<L, p, LE>;
    constexpr int RADIX = PI::RADIX, NS = PI::NS, V = S::E / RADIX;
#pragma unroll
    for (int vv = 0; vv < V; ++vv) {
        cpx<R> u[RADIX];
#pragma unroll
        for (int j = 0; j < RADIX; ++j) u[j] = v[vv + j * V];
        if (NS > 1) {
            const int k = (i + vv * S::T) & (NS - 1);
            if constexpr (TWC) {
                cpx<R> w[RADIX];
                twiddle_powers<RADIX>(twiddle_exact<R, SGN>(k, NS * RADIX), w);
#pragma unroll
                for (int j = 1; j < RADIX; ++j) u[j] = cmul(u[j], w[j]);
            } else {
                const cpx<R>* t = tw + PI::TW_OFF + k;
#pragma unroll
                for (int j = 1; j < RADIX; ++j) {
                    cpx<R> w = ld_tw<R>(t + (j - 1) * NS);
                    if (SGN > 0) w.y = -w.y;
                    u[j] = cmul(u[j], w);
                }
            }
        }
        dft<RADIX, SGN>(u);
#pragma unroll
        for (int j = 0; j < RADIX; ++j) v[vv + j * V] = u[j];
    }
}

template <int L, int p, int LE = 4, int PS = 4, class R>
__device__ __forceinline__ void smem_store(const cpx<R>* v, cpx<R>* buf, int i) {
    using S = shape<L, LE>;
    using PI = pass<L, p, LE>;
    constexpr int RADIX = PI::RADIX, NS = PI::NS, V = S::E / RADIX;
#pragma unroll
    for (int vv = 0; vv < V; ++vv) {
        const int ip = i + vv * S::T;
        const int k = ip & (NS - 1);
        const int base = (ip - k) * RADIX + k;
#pragma unroll
        for (int j = 0; j < RADIX; ++j) buf[pad_idx<PS>(base + j * NS)] = v[vv + j * V];
    }
}

template <int L, int LE = 4, int PS = 4, class R>
__device__ __forceinline__ void smem_load(cpx<R>* v, const cpx<R>* buf, int i) {
    using S = shape<L, LE>;
#pragma unroll
    for (int e = 0; e < S::E; ++e) v[e] = buf[pad_idx<PS>(i + e * S::T)];
}

// Exchange barrier: the whole CTA, or only the warp when every signal's
// threads lie within one warp (WS: T <= 32 consecutive threads per signal).
template <bool WS>
__device__ __forceinline__ void exchange_sync() {
    if constexpr (WS) __syncwarp();
    else __syncthreads();
}

// Passes p..P-1, the first of which reads the shared-memory output of pass p-1.
template <int L, int p, int SGN, bool TWC, class R, int LE, int PS, bool WS = false,
          bool DONE = (p >= shape<L, LE>::P)>
struct passes_from {
    __device__ __forceinline__ static void run(cpx<R>* v, cpx<R>* buf, int i,
                                               const cpx<R>* __restrict__ tw) {
        if (p > 1) exchange_sync<WS>();      // previous exchange fully read
        smem_store<L, p - 1, LE, PS>(v, buf, i);
        exchange_sync<WS>();
        smem_load<L, LE, PS>(v, buf, i);
        butterflies<L, p, SGN, TWC, LE>(v, i, tw);
        passes_from<L, p + 1, SGN, TWC, R, LE, PS, WS>::run(v, buf, i, tw);
    }
};
template <int L, int p, int SGN, bool TWC, class R, int LE, int PS, bool WS>
struct passes_from<L, p, SGN, TWC, R, LE, PS, WS, true> {
    __device__ __forceinline__ static void run(cpx<R>*, cpx<R>*, int, const cpx<R>* __restrict__) {}
};

// Whole DFT on the registers v (thread i holds samples i + e T on entry and
// output samples i + e T on exit).  buf: this signal's padded shared buffer.
template <int L, int SGN, bool TWC = false, int LE = 4, int PS = 4, class R>
__device__ __forceinline__ void dft_signal(cpx<R>* v, cpx<R>* buf, int i,
                                           const cpx<R>* __restrict__ tw) {
    butterflies<L, 0, SGN, TWC, LE>(v, i, tw);
    passes_from<L, 1, SGN, TWC, R, LE, PS>::run(v, buf, i, tw);
}

// The same for a signal whose T <= 32 threads are consecutive (lie within one
// warp): the exchanges synchronise that warp only, so the other signals of
// the CTA are not held at its barriers.
template <int L, int SGN, bool TWC = false, int LE = 4, int PS = 4, class R>
__device__ __forceinline__ void dft_signal_warp(cpx<R>* v, cpx<R>* buf, int i,
                                                const cpx<R>* __restrict__ tw) {
    static_assert(shape<L, LE>::T <= 32, "signal wider than a warp");
    butterflies<L, 0, SGN, TWC, LE>(v, i, tw);
    passes_from<L, 1, SGN, TWC, R, LE, PS, true>::run(v, buf, i, tw);
}

// Streaming global load that does not allocate in L1 (keeps the twiddle
// table resident): ld.global.nc.L1::no_allocate.
__device__ __forceinline__ cpx<float> ld_stream(const cpx<float>* p) {
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ld_stream(const cpx<double>* p) {
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];"
                 : "=d"(v.x), "=d"(v.y)
                 : "l"(p));
    return {v.x, v.y};
}

}  // namespace xft
