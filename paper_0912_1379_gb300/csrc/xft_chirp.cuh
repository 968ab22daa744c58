// Exact chirp phasors of the XFT (Sec. 3, Algorithm, steps 1-2), from the
// fixed-point turn fractions of the descriptor (see lct_internal.h).
#pragma once
#include "xft_common.cuh"

namespace xft {

// Pre-chirp e^{2 pi i [phi_in m^2 + (N-1) n/(2N)]} e^{-decay m^2} of sample n.
template <int L>
__device__ __forceinline__ cpx<float> pre_chirp(const lct_desc& D, int n, bool decay) {
    constexpr uint32_t CEN = (uint32_t)(((1u << L) - 1u) << (31 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    cpx<float> w = expi_turn32<true>(phase32(D.in_hi, m2) + (uint32_t)n * CEN);
    if (decay) w = cscale(w, expf(-(float)D.decay * (float)m2));
    return w;
}
template <int L>
__device__ __forceinline__ cpx<double> pre_chirp64(const lct_desc& D, int n, bool decay) {
    constexpr uint64_t CEN = (uint64_t)(((1ull << L) - 1ull) << (63 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    cpx<double> w = expi_turn64(phase64(D.in_hi, D.in_lo, m2) + (uint64_t)n * CEN);
    if (decay) w = cscale(w, exp(-D.decay * (double)m2));
    return w;
}
// Post-chirp e^{2 pi i [phi_out m^2 + (N-1) n/(2N) + c_out]} of sample n.
template <int L>
__device__ __forceinline__ cpx<float> post_chirp(const lct_desc& D, int n) {
    constexpr uint32_t CEN = (uint32_t)(((1u << L) - 1u) << (31 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
    return expi_turn32<true>(phase32(D.out_hi, m2) + (uint32_t)n * CEN + off);
}
template <int L>
__device__ __forceinline__ cpx<double> post_chirp64(const lct_desc& D, int n) {
    constexpr uint64_t CEN = (uint64_t)(((1ull << L) - 1ull) << (63 - L));
    const uint32_t m2 = m_squared(n, 1 << L);
    return expi_turn64(phase64(D.out_hi, D.out_lo, m2) + (uint64_t)n * CEN + D.out_c);
}

template <int L, class R>
__device__ __forceinline__ cpx<R> pre_w(const lct_desc& D, int n, bool decay) {
    if constexpr (sizeof(R) == 4) return pre_chirp<L>(D, n, decay);
    else return pre_chirp64<L>(D, n, decay);
}
template <int L, class R>
__device__ __forceinline__ cpx<R> post_w(const lct_desc& D, int n) {
    if constexpr (sizeof(R) == 4) return post_chirp<L>(D, n);
    else return post_chirp64<L>(D, n);
}

}  // namespace xft
