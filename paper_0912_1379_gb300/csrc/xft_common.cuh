// Device building blocks shared by the XFT kernels: complex arithmetic,
// in-register radix-2/4/8/16 DFTs, and the exact fixed-point chirp phases.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "lct_internal.h"

template <class R>
struct __align__(2 * sizeof(R)) cpx {
    R x, y;
};

template <class R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R>
__device__ __forceinline__ cpx<R> cscale(cpx<R> a, R s) { return {a.x * s, a.y * s}; }
template <class R>
__device__ __forceinline__ cpx<R> cconj(cpx<R> a) { return {a.x, -a.y}; }

// Multiply by S*i (S = -1: by -i; S = +1: by +i).
template <int S, class R>
__device__ __forceinline__ cpx<R> mul_si(cpx<R> a) {
    if (S < 0) return {a.y, -a.x};
    return {-a.y, a.x};
}

// ---------------------------------------------------------------------------
// In-register DFTs, X[k] = sum_n a[n] e^{S 2 pi i n k / R}; S = -1 forward.
// Input a[0..R-1] in natural order, output in natural order (in place).
// ---------------------------------------------------------------------------
template <int S, class R>
__device__ __forceinline__ void dft2(cpx<R>* a) {
    cpx<R> t = a[0];
    a[0] = t + a[1];
    a[1] = t - a[1];
}

template <int S, class R>
__device__ __forceinline__ void dft4_idx(cpx<R>& a0, cpx<R>& a1, cpx<R>& a2, cpx<R>& a3) {
    cpx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = mul_si<S>(a1 - a3);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}

template <int S, class R>
__device__ __forceinline__ void dft4(cpx<R>* a) { dft4_idx<S>(a[0], a[1], a[2], a[3]); }

template <class R>
struct dft_consts;
template <>
struct dft_consts<float> {
    static constexpr float RS2 = 0.70710678118654752440f;   // sqrt(1/2)
    static constexpr float C8 = 0.92387953251128675613f;    // cos(pi/8)
    static constexpr float S8 = 0.38268343236508977173f;    // sin(pi/8)
};
template <>
struct dft_consts<double> {
    static constexpr double RS2 = 0.70710678118654752440;
    static constexpr double C8 = 0.92387953251128675613;
    static constexpr double S8 = 0.38268343236508977173;
};

// Multiply by W8^e = e^{S 2 pi i e / 8}, e in 0..3.
template <int S, int E, class R>
__device__ __forceinline__ cpx<R> mul_w8(cpx<R> a) {
    const R h = dft_consts<R>::RS2;
    if (E == 0) return a;
    if (E == 2) return mul_si<S>(a);
    if (E == 1) {  // h (1 + S i)
        cpx<R> t = a + mul_si<S>(a);
        return cscale(t, h);
    }
    // E == 3: h (-1 + S i)
    cpx<R> t = mul_si<S>(a) - a;
    return cscale(t, h);
}

template <int S, class R>
__device__ __forceinline__ void dft8(cpx<R>* a) {
    cpx<R> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    cpx<R> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4_idx<S>(e0, e1, e2, e3);
    dft4_idx<S>(o0, o1, o2, o3);
    o1 = mul_w8<S, 1>(o1);
    o2 = mul_w8<S, 2>(o2);
    o3 = mul_w8<S, 3>(o3);
    a[0] = e0 + o0; a[4] = e0 - o0;
    a[1] = e1 + o1; a[5] = e1 - o1;
    a[2] = e2 + o2; a[6] = e2 - o2;
    a[3] = e3 + o3; a[7] = e3 - o3;
}

// Multiply by W16^e = e^{S 2 pi i e / 16} for the exponents 0..9 of the
// 4 x 4 radix-16 split.
template <int S, int E, class R>
__device__ __forceinline__ cpx<R> mul_w16(cpx<R> a) {
    const R c = dft_consts<R>::C8, s = dft_consts<R>::S8;
    if (E == 0) return a;
    if (E % 2 == 0) return mul_w8<S, (E / 2) % 4>(E >= 8 ? cpx<R>{-a.x, -a.y} : a);
    // odd exponents: cos/sin of multiples of pi/8
    R cr, ci;  // W16^E = cr + S i ci
    if (E == 1) { cr = c; ci = s; }
    else if (E == 3) { cr = s; ci = c; }
    else if (E == 5) { cr = -s; ci = c; }
    else if (E == 7) { cr = -c; ci = s; }
    else { cr = -c; ci = -s; }  // E == 9
    const R si = S < 0 ? -ci : ci;
    return {a.x * cr - a.y * si, a.x * si + a.y * cr};
}

// Radix-16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <int S, class R>
__device__ __forceinline__ void dft16(cpx<R>* a) {
    // step 1: DFT4 over n1 for each n2 -> A[n2][k1] at a[n2 + 4 k1]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4_idx<S>(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    // step 2: twiddles W16^{n2 k1}
    a[5] = mul_w16<S, 1>(a[5]);
    a[6] = mul_w16<S, 2>(a[6]);
    a[7] = mul_w16<S, 3>(a[7]);
    a[9] = mul_w16<S, 2>(a[9]);
    a[10] = mul_w16<S, 4>(a[10]);
    a[11] = mul_w16<S, 6>(a[11]);
    a[13] = mul_w16<S, 3>(a[13]);
    a[14] = mul_w16<S, 6>(a[14]);
    a[15] = mul_w16<S, 9>(a[15]);
    // step 3: DFT4 over n2 for each k1 -> X[k1 + 4 k2] at a[4 k1 + k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4_idx<S>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    // digit reversal to natural order
    cpx<R> t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = a[4 * (k & 3) + (k >> 2)];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = t[k];
}

template <int RADIX, int S, class R>
__device__ __forceinline__ void dft(cpx<R>* a) {
    if (RADIX == 2) dft2<S>(a);
    else if (RADIX == 4) dft4<S>(a);
    else if (RADIX == 8) dft8<S>(a);
    else if (RADIX == 16) dft16<S>(a);
}

// Powers w^0..w^(R-1) of a unit twiddle by a shallow product tree.
template <int RADIX, class R>
__device__ __forceinline__ void twiddle_powers(cpx<R> w1, cpx<R>* w) {
    w[0] = {R(1), R(0)};
    if (RADIX > 1) w[1] = w1;
    if (RADIX > 2) { w[2] = cmul(w1, w1); w[3] = cmul(w[2], w1); }
    if (RADIX > 4) {
        w[4] = cmul(w[2], w[2]);
        w[5] = cmul(w[4], w1);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
    }
    if (RADIX > 8) {
        w[8] = cmul(w[4], w[4]);
#pragma unroll
        for (int j = 9; j < 16; ++j) w[j] = cmul(w[8], w[j - 8]);
    }
}

// ---------------------------------------------------------------------------
// Exact chirp phases.  m = 2k - N + 1; the turn fraction of the phase
//   phi * m^2 + c * k + off   (mod 1)
// with phi a 128-bit (FP64) or 64-bit (FP32) fraction, c the centring step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t m_squared(int k, int n) {
    int m = 2 * k - n + 1;
    uint32_t um = (uint32_t)m;
    return um * um;  // m^2 < 2^32 for |m| < 65536
}

// FP32 path: top 32 bits of the wrapped 64-bit product phi * m^2.
__device__ __forceinline__ uint32_t phase32(uint64_t phi, uint32_t m2) {
    uint32_t lo = (uint32_t)phi, hi = (uint32_t)(phi >> 32);
    return __umulhi(lo, m2) + hi * m2;
}

// FP64 path: top 64 bits of the wrapped 128-bit product phi * m^2.
__device__ __forceinline__ uint64_t phase64(uint64_t phi_hi, uint64_t phi_lo, uint32_t m2) {
    return phi_hi * (uint64_t)m2 + __umul64hi(phi_lo, (uint64_t)m2);
}

// e^{2 pi i t}, t = turn fraction in 32-bit (FP32) or 64-bit (FP64) fixed point.
template <bool FAST>
__device__ __forceinline__ cpx<float> expi_turn32(uint32_t t) {
    float f = (float)(int32_t)t;  // in [-2^31, 2^31): turns * 2^32
    float s, c;
    if (FAST) {
        __sincosf(f * 1.46291807926715968e-9f, &s, &c);   // 2 pi / 2^32
    } else {
        sincospif(f * 4.65661287307739257812e-10f, &s, &c);  // 2 / 2^32
    }
    return {c, s};
}

__device__ __forceinline__ cpx<double> expi_turn64(uint64_t t) {
    double f = (double)(int64_t)t * 1.08420217248550443401e-19;  // 2 / 2^64
    double s, c;
    sincospi(f, &s, &c);
    return {c, s};
}
