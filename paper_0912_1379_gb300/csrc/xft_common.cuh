// Device building blocks shared by the XFT kernels: complex arithmetic,
// in-register radix-2/4/8/16 DFTs, and the exact fixed-point chirp phases.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "lct_internal.h"

// ---------------------------------------------------------------------------
// Packed FP32 pair (sm_100+ f32x2 arithmetic): one register pair holding the
// same component of two independent samples, one instruction per operation.
// A subtraction is written as b * (-1) + a so that it stays one instruction.
// ---------------------------------------------------------------------------
struct __align__(8) pf {
    float2 v;
};
__device__ __forceinline__ pf pf_make(float lo, float hi) { return {make_float2(lo, hi)}; }
__device__ __forceinline__ pf pf_bcast(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ pf operator+(pf a, pf b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ pf operator*(pf a, pf b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ pf operator-(pf a, pf b) {
    return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};
}
__device__ __forceinline__ pf operator-(pf a) { return {__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))}; }

// a * b + c
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ pf madd(pf a, pf b, pf c) { return {__ffma2_rn(a.v, b.v, c.v)}; }

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
    return {madd(a.y, -b.y, a.x * b.x), madd(a.y, b.x, a.x * b.y)};
}
// a * b where nby = -b.y is supplied by the caller (saves the negation).
template <class R>
__device__ __forceinline__ cpx<R> cmul_nb(cpx<R> a, R bx, R by, R nby) {
    return {madd(a.y, nby, a.x * bx), madd(a.y, bx, a.x * by)};
}
template <class R>
__device__ __forceinline__ cpx<R> cscale(cpx<R> a, R s) { return {a.x * s, a.y * s}; }

// ---------------------------------------------------------------------------
// In-register DFTs, X[k] = sum_n a[n] e^{S 2 pi i n k / R}; S = -1 forward.
// Input a[0..R-1] in natural order, output in natural order (in place).
// Written with component additions only (multiplications by +-i folded
// into the additions) so that no negation instruction is needed.
// ---------------------------------------------------------------------------
template <int S, class R>
__device__ __forceinline__ void dft2(cpx<R>* a) {
    cpx<R> t = a[0];
    a[0] = t + a[1];
    a[1] = t - a[1];
}

// t + S i d  and  t - S i d
template <int S, class R>
__device__ __forceinline__ cpx<R> add_si(cpx<R> t, cpx<R> d) {
    if (S < 0) return {t.x + d.y, t.y - d.x};
    return {t.x - d.y, t.y + d.x};
}
template <int S, class R>
__device__ __forceinline__ cpx<R> sub_si(cpx<R> t, cpx<R> d) {
    if (S < 0) return {t.x - d.y, t.y + d.x};
    return {t.x + d.y, t.y - d.x};
}

template <int S, class R>
__device__ __forceinline__ void dft4_idx(cpx<R>& a0, cpx<R>& a1, cpx<R>& a2, cpx<R>& a3) {
    const cpx<R> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, d = a1 - a3;
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = add_si<S>(t1, d);
    a3 = sub_si<S>(t1, d);
}

template <int S, class R>
__device__ __forceinline__ void dft4(cpx<R>* a) { dft4_idx<S>(a[0], a[1], a[2], a[3]); }

template <class R>
struct dft_consts;
template <>
struct dft_consts<float> {
    __device__ static float c(float v) { return v; }
};
template <>
struct dft_consts<double> {
    __device__ static double c(double v) { return v; }
};
template <>
struct dft_consts<pf> {
    __device__ static pf c(float v) { return pf_bcast(v); }
};
#define LCT_RS2 0.70710678118654752440   // sqrt(1/2)
#define LCT_C8 0.92387953251128675613    // cos(pi/8)
#define LCT_S8 0.38268343236508977173    // sin(pi/8)

template <class R>
__device__ __forceinline__ R kconst(double v) {
    if constexpr (sizeof(R) == 8 && !__is_same(R, pf)) return dft_consts<R>::c(v);
    else return dft_consts<R>::c((float)v);
}

// Multiply by W8^E = e^{S 2 pi i E / 8} for E = 1 (h (1 + S i)) and E = 3
// (h (-1 + S i) = -h (1 - S i)).
template <int S, int E, class R>
__device__ __forceinline__ cpx<R> mul_w8_odd(cpx<R> a) {
    if (E == 1) {  // h (1 + S i) a = h (a.x - S a.y, a.y + S a.x)
        const R h = kconst<R>(LCT_RS2);
        cpx<R> t = add_si<S>(a, a);
        return cscale(t, h);
    }
    // E == 3: -h (a.x + S a.y, a.y - S a.x)
    const R mh = kconst<R>(-LCT_RS2);
    cpx<R> t = sub_si<S>(a, a);
    return cscale(t, mh);
}

template <int S, class R>
__device__ __forceinline__ void dft8(cpx<R>* a) {
    cpx<R> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    cpx<R> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4_idx<S>(e0, e1, e2, e3);
    dft4_idx<S>(o0, o1, o2, o3);
    o1 = mul_w8_odd<S, 1>(o1);
    o3 = mul_w8_odd<S, 3>(o3);
    a[0] = e0 + o0; a[4] = e0 - o0;
    a[1] = e1 + o1; a[5] = e1 - o1;
    a[2] = add_si<S>(e2, o2); a[6] = sub_si<S>(e2, o2);     // W8^2 = S i
    a[3] = e3 + o3; a[7] = e3 - o3;
}

// Multiply by the odd power W16^E = e^{S 2 pi i E / 16} = cr + S i ci.
template <int S, int E, class R>
__device__ __forceinline__ cpx<R> mul_w16_odd(cpx<R> a) {
    double cr, ci;
    if (E == 1) { cr = LCT_C8; ci = LCT_S8; }
    else if (E == 3) { cr = LCT_S8; ci = LCT_C8; }
    else if (E == 5) { cr = -LCT_S8; ci = LCT_C8; }
    else if (E == 7) { cr = -LCT_C8; ci = LCT_S8; }
    else { cr = -LCT_C8; ci = -LCT_S8; }  // E == 9
    const double si = S < 0 ? -ci : ci;
    return cmul_nb(a, kconst<R>(cr), kconst<R>(si), kconst<R>(-si));
}

// Radix-16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <int S, class R>
__device__ __forceinline__ void dft16(cpx<R>* a) {
    // step 1: DFT4 over n1 for each n2 -> A[n2][k1] at a[n2 + 4 k1]
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4_idx<S>(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    // step 2: twiddles W16^{n2 k1}
    a[5] = mul_w16_odd<S, 1>(a[5]);
    a[6] = mul_w8_odd<S, 1>(a[6]);                 // W16^2 = W8^1
    a[7] = mul_w16_odd<S, 3>(a[7]);
    a[9] = mul_w8_odd<S, 1>(a[9]);
    {                                              // W16^4 = S i
        cpx<R> t = a[10];
        a[10] = S < 0 ? cpx<R>{t.y, -t.x} : cpx<R>{-t.y, t.x};
    }
    a[11] = mul_w8_odd<S, 3>(a[11]);               // W16^6 = W8^3
    a[13] = mul_w16_odd<S, 3>(a[13]);
    a[14] = mul_w8_odd<S, 3>(a[14]);
    a[15] = mul_w16_odd<S, 9>(a[15]);
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
