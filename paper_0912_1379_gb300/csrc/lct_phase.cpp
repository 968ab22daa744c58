// Exact phase constants, per-signal descriptors and the Stockham twiddle
// tables (host side of the chirp phases of Sec. 3, Algorithm, steps 1-2).
//
// Phase constants.  The chirp coefficients
//   Re(beta_in)/(2 pi)  = Re(a/b) pi / (32 N)
//   Re(beta_out)/(2 pi) = Re(b d) / (2 pi N)
// are evaluated in double-double arithmetic (about 106 significant bits)
// from the exact FP64 parameters and reduced modulo one turn into 128-bit
// fixed-point fractions.  The output constant e^{-i pi (N-1)^2/(2N)} is an
// exact dyadic turn fraction; the argument of dx/sqrt(2 pi i b) is added to
// it in double precision.
#include "lct_plan.h"

#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace lcth {
namespace {

// ---------------------------------------------------------------------------
// double-double arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------
struct dd { double hi, lo; };

dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(b, {q1, 0.0}));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(b, {q2, 0.0}));
    double q3 = r.hi / b.hi;
    return dd_add(quick_two_sum(q1, q2), {q3, 0.0});
}
dd dd_ldexp(dd a, int e) { return {std::ldexp(a.hi, e), std::ldexp(a.lo, e)}; }

// pi to about 107 bits
const dd DD_PI = {3.141592653589793116e+00, 1.224646799147353207e-16};

typedef unsigned __int128 u128;

// round(v * 2^128) mod 2^128 for |v| < 1.
u128 frac_to_q128(double v) {
    if (v == 0.0) return 0;
    int e;
    double m = std::frexp(std::fabs(v), &e);          // |v| = m 2^e, m in [1/2, 1)
    uint64_t M = (uint64_t)std::ldexp(m, 53);         // exact 53-bit integer
    int sh = e - 53 + 128;                            // |v| 2^128 = M 2^sh, sh <= 75
    u128 r;
    if (sh >= 0) r = (u128)M << sh;
    else if (sh > -64) r = (u128)((M + ((uint64_t)1 << (-sh - 1))) >> (-sh));
    else r = 0;
    return v < 0 ? (u128)0 - r : r;
}

// Fractional part of a double-double as a 128-bit turn fraction.
void dd_to_turns128(dd t, uint64_t* hi, uint64_t* lo) {
    // x - trunc(x) is exact for every double (x - floor(x) is not for small
    // negative x); the signed fractions wrap modulo one turn below.
    double fh = t.hi - std::trunc(t.hi);
    double fl = t.lo - std::trunc(t.lo);
    u128 q = frac_to_q128(fh) + frac_to_q128(fl);
    *hi = (uint64_t)(q >> 64);
    *lo = (uint64_t)q;
}

}  // namespace

// Fractional part of a double (|v| moderate) as a 64-bit turn fraction.
uint64_t double_to_turns64(double v) {
    uint64_t hi, lo;
    dd_to_turns128({v, 0.0}, &hi, &lo);
    return hi + (lo >> 63);
}

int ilog2_exact(int64_t N) {
    if (N < 2 || N > 65536) return -1;
    if ((N & (N - 1)) != 0) return -1;
    int p = 0;
    while ((int64_t(1) << p) < N) ++p;
    return p;
}

namespace {
// Re(x/y) of complex FP64 numbers, in double-double.
dd dd_re_div(cplx x, cplx y) {
    dd num = dd_add(two_prod(x.real(), y.real()), two_prod(x.imag(), y.imag()));
    dd den = dd_add(two_prod(y.real(), y.real()), two_prod(y.imag(), y.imag()));
    return dd_div(num, den);
}
// Re(x*y) in double-double.
dd dd_re_mul(cplx x, cplx y) {
    return dd_sub(two_prod(x.real(), y.real()), two_prod(x.imag(), y.imag()));
}

bool symplectic(cplx a, cplx b, cplx c, cplx d) {
    cplx ad = a * d, bc = b * c;
    double tol = 1e-9 * std::fmax(1.0, std::fmax(std::abs(ad), std::abs(bc)));
    return std::abs(ad - bc - 1.0) <= tol;
}

}  // namespace

// Build the descriptor of one signal.  Returns LCT_OK or a validation error.
// N = 2 .. 65536; N that is not a power of two gets the chirp-convolution
// form (kinds LCT_KIND_BLUE / LCT_KIND_DIAGN, see lct_internal.h); which
// such N a dtype supports is checked by the plan.
lct_status make_desc(int64_t N, const double* p, int64_t offset, lct_desc* D) {
    if (N < 2 || N > 65536) return LCT_ERR_N;
    const int log2n = ilog2_exact(N);
    const bool pow2 = log2n >= 0;
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(p[i])) return LCT_ERR_ARG;
    cplx a(p[0], p[1]), b(p[2], p[3]), c(p[4], p[5]), d(p[6], p[7]);
    if (!symplectic(a, b, c, d)) return LCT_ERR_NOT_SYMPLECTIC;
    std::memset(D, 0, sizeof(*D));
    D->offset = offset;
    D->log2n = pow2 ? log2n : 0;
    D->n = (int32_t)N;
    const dd DN = {(double)N, 0.0};
    uint64_t hi, lo;
    if (b == cplx(0.0, 0.0)) {
        // b = 0: G_j = sqrt(d) e^{i c x_j^2 / (2d)} f_j on y_j = x_j / d;
        // c x^2/(2d) = Re(c/d) pi^2 m^2/(16N) -> turns Re(c/d) pi / (32N).
        D->kind = pow2 ? LCT_KIND_DIAG : LCT_KIND_DIAGN;
        dd t = pow2 ? dd_ldexp(dd_mul(dd_re_div(c, d), DD_PI), -(5 + log2n))
                    : dd_div(dd_ldexp(dd_mul(dd_re_div(c, d), DD_PI), -5), DN);
        dd_to_turns128(t, &hi, &lo);
        D->out_hi = hi;
        D->out_lo = lo;
        cplx sd = std::sqrt(d);                       // principal root
        D->scale = std::abs(sd);
        D->out_c = double_to_turns64(std::arg(sd) / (2.0 * M_PI));
        return LCT_OK;
    }
    cplx ab = a / b;
    double decay = ab.imag() * M_PI * M_PI / (16.0 * (double)N);
    D->decay = decay;
    if (decay != 0.0) D->flags |= LCT_FLAG_DECAY;
    double dx = M_PI / std::sqrt(2.0 * (double)N);
    cplx pre = dx / std::sqrt(cplx(0.0, 2.0 * M_PI) * b);
    D->scale = std::abs(pre);
    if (!pow2 && lct_mixed_ok(N)) {
        // direct form with a mixed-radix DFT: the XFT phases with N in place
        // of 2^log2n; the centring phases are formed in the kernel
        D->kind = LCT_KIND_MIXED;
        D->log2n = lct_blue_log2m(N) - 1;          // ceil(log2 N): orders the plan's groups
        dd tin = dd_div(dd_ldexp(dd_mul(dd_re_div(a, b), DD_PI), -5), DN);   // Re(a/b) pi/(32N)
        dd_to_turns128(tin, &hi, &lo);
        D->in_hi = hi;
        D->in_lo = lo;
        dd tout = dd_div(dd_div(dd_re_mul(b, d), dd_ldexp(DD_PI, 1)), DN);  // Re(bd)/(2 pi N)
        dd_to_turns128(tout, &hi, &lo);
        D->out_hi = hi;
        D->out_lo = lo;
        // constant -(N-1)^2/(4N) turns: -r/(4N), r = (N-1)^2 mod 4N, in Q0.64
        const uint64_t r = (uint64_t)(((N - 1) * (N - 1)) % (4 * N));
        const uint64_t centre = (uint64_t)0 - (uint64_t)((((unsigned __int128)r) << 64) / (uint64_t)(4 * N));
        D->out_c = centre + double_to_turns64(std::arg(pre) / (2.0 * M_PI));
        return LCT_OK;
    }
    if (!pow2) {
        // chirp-convolution form: phi_in - 1/(8N), phi_out - 1/(8N), constant
        // arg(dx / sqrt(2 pi i b)) only
        D->kind = LCT_KIND_BLUE;
        D->log2n = lct_blue_log2m(N);
        const dd one = {1.0, 0.0};
        dd tin = dd_div(dd_sub(dd_ldexp(dd_mul(dd_re_div(a, b), DD_PI), -2), one),
                        dd_ldexp(DN, 3));                     // (Re(a/b) pi/4 - 1) / (8N)
        dd_to_turns128(tin, &hi, &lo);
        D->in_hi = hi;
        D->in_lo = lo;
        dd tout = dd_div(dd_sub(dd_div(dd_re_mul(b, d), dd_ldexp(DD_PI, 1)), {0.125, 0.0}),
                         DN);                                 // (Re(bd)/(2 pi) - 1/8) / N
        dd_to_turns128(tout, &hi, &lo);
        D->out_hi = hi;
        D->out_lo = lo;
        D->out_c = double_to_turns64(std::arg(pre) / (2.0 * M_PI));
        return LCT_OK;
    }
    D->kind = LCT_KIND_XFT;
    // pre-chirp a x_k^2/(2b) = (a/b) pi^2 m^2 / (16 N): turns (a/b) pi / (32 N)
    dd tin = dd_ldexp(dd_mul(dd_re_div(a, b), DD_PI), -(5 + log2n));
    dd_to_turns128(tin, &hi, &lo);
    D->in_hi = hi;
    D->in_lo = lo;
    // post-chirp d y_j^2/(2b) = b d m^2 / N: turns Re(b d) / (2 pi N)
    dd tout = dd_ldexp(dd_div(dd_re_mul(b, d), DD_PI), -(1 + log2n));
    dd_to_turns128(tout, &hi, &lo);
    D->out_hi = hi;
    D->out_lo = lo;
    // constant: -(N-1)^2/(4N) turns (exact) + arg(dx / sqrt(2 pi i b)) / (2 pi)
    uint64_t r = (uint64_t)(((N - 1) * (N - 1)) % (4 * N));
    uint64_t centre = (uint64_t)0 - (r << (62 - log2n));       // -r / (4N) as Q0.64
    D->out_c = centre + double_to_turns64(std::arg(pre) / (2.0 * M_PI));
    return LCT_OK;
}

// Complex-z fractional transform on the nodes (Sec. 2, eqs. (fasy),
// (primcuad)); the convolution form is derived in lct_internal.h.  With
// z = x + i y (after the parity step x >= 0):
//   B = (1 - z)/(2(1 + z)):  Re B = (1 - |z|^2)/(2|1 + z|^2),  Im B = -y/|1 + z|^2
//   A = z/(1 - z^2):         Re A = x (1 - |z|^2)/|1 - z^2|^2,
//                            Im A = y (1 + |z|^2)/|1 - z^2|^2
// The phase coefficients are formed in double-double from the FP64 z and
// reduced to 128-bit turn fractions; the magnitudes in FP64.
lct_status mehler_setup(int64_t N, double z_re, double z_im, lct_desc* D, mehler_consts* K) {
    if (!std::isfinite(z_re) || !std::isfinite(z_im)) return LCT_ERR_ARG;
    if (std::hypot(z_re, z_im) > 1.0 + 1e-15) return LCT_ERR_ARG;
    if (z_im == 0.0 && std::fabs(z_re) == 1.0) return LCT_ERR_ARG;       // 1 - z^2 = 0
    const bool rev = z_re < 0.0;
    const double x = rev ? -z_re : z_re, y = rev ? -z_im : z_im;
    const dd one = {1.0, 0.0}, X = {x, 0.0}, Y = {y, 0.0}, DN = {(double)N, 0.0};
    const dd x2 = two_prod(x, x), y2 = two_prod(y, y);
    const dd r2 = dd_add(x2, y2);                                // |z|^2
    dd omr2 = dd_sub(one, r2);                                   // 1 - |z|^2
    if (omr2.hi < 0.0) omr2 = {0.0, 0.0};                        // |z| = 1 up to rounding
    const dd opx = two_sum(1.0, x);
    const dd q = dd_add(dd_mul(opx, opx), y2);                   // |1 + z|^2
    const dd u = dd_add(dd_sub(one, x2), y2);                    // Re(1 - z^2)
    const dd v = dd_ldexp(two_prod(x, y), 1);                    // -Im(1 - z^2)
    const dd den = dd_add(dd_mul(u, u), dd_mul(v, v));           // |1 - z^2|^2
    const double re_b = dd_div(omr2, dd_ldexp(q, 1)).hi;
    const dd im_b = dd_neg(dd_div(Y, q));
    const double re_a = dd_div(dd_mul(X, omr2), den).hi;
    const dd im_a = dd_div(dd_mul(Y, dd_add(one, r2)), den);
    std::memset(D, 0, sizeof(*D));
    D->kind = LCT_KIND_MEHLER;
    D->n = (int32_t)N;
    D->log2n = lct_blue_log2m(N);
    D->scale = 1.0;
    // weight e^{-B x^2}, x^2 = pi^2 m^2/(8N): phase -Im(B) pi/(16N) turns per m^2
    uint64_t hi, lo;
    dd_to_turns128(dd_div(dd_mul(dd_neg(im_b), DD_PI), dd_ldexp(DN, 4)), &hi, &lo);
    D->in_hi = D->out_hi = hi;
    D->in_lo = D->out_lo = lo;
    D->decay = re_b * M_PI * M_PI / (8.0 * (double)N);
    if (D->decay != 0.0) D->flags |= LCT_FLAG_DECAY | LCT_FLAG_OUT_DECAY;
    if (rev) D->flags |= LCT_FLAG_REVERSE;
    // lag kernel e^{-A (x_j - x_k)^2}, (x_j - x_k)^2 = pi^2 l^2/(2N)
    K->a_h = re_a * M_PI * M_PI / (2.0 * (double)N);
    dd_to_turns128(dd_div(dd_mul(dd_neg(im_a), DD_PI), dd_ldexp(DN, 2)), &K->phi_hi, &K->phi_lo);
    // sqrt(2/(1 - z^2)) dx, principal root (1 - z^2 is even in z)
    const cplx c = std::sqrt(2.0 / cplx(u.hi, -v.hi)) * (M_PI / std::sqrt(2.0 * (double)N));
    K->c_re = c.real();
    K->c_im = c.imag();
    return LCT_OK;
}

}  // namespace lcth

using namespace lcth;

// ---------------------------------------------------------------------------
// twiddle tables of the Stockham engine (xft_engine.cuh)
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tw_mu;
std::map<std::tuple<int, int, int>, void*> g_tw;   // (device, dtype, log2n) -> table

// Table of the Stockham engine with radix E = 2^le passes (see xft_engine.cuh).
template <class T>
std::vector<T> build_twiddles(int log2n, int le = 4) {
    const int E = 1 << le;
    const int P = log2n >= le ? (log2n + le - 1) / le : 1;
    const int R0 = 1 << (log2n - le * (P - 1));
    std::vector<T> t;
    for (int p = 1; p < P; ++p) {
        const int64_t ns = (int64_t)R0 << (le * (p - 1));
        const int64_t M = E * ns;
        for (int j = 1; j < E; ++j)
            for (int64_t k = 0; k < ns; ++k) {
                const double ang = 2.0 * M_PI * (double)((j * k) % M) / (double)M;
                t.push_back((T)std::cos(ang));
                t.push_back((T)-std::sin(ang));
            }
    }
    return t;
}

// The cached device copy of the table `key`, built by make() on first use.
// Caller holds g_tw_mu.
template <class F>
const void* cached_table(const std::tuple<int, int, int>& key, F make) {
    auto it = g_tw.find(key);
    if (it != g_tw.end()) return it->second;
    const auto t = make();
    const size_t bytes = t.size() * sizeof(t[0]);
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, t.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    g_tw[key] = d;
    return d;
}
}  // namespace

const void* lct_twiddle_table(int dtype, int log2n) {
    if (log2n < 5) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    const auto key = std::make_tuple(dev, dtype, log2n);
    if (dtype == LCT_C64) return cached_table(key, [&] { return build_twiddles<float>(log2n); });
    return cached_table(key, [&] { return build_twiddles<double>(log2n); });
}

const void* lct_twiddle_table_le(int dtype, int log2n, int le) {
    if (le < 2 || le > 4 || log2n <= le) return nullptr;
    if (le == 4) return lct_twiddle_table(dtype, log2n);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    const auto key = std::make_tuple(dev, 40 + 2 * le + dtype, log2n);
    if (dtype == LCT_C64) return cached_table(key, [&] { return build_twiddles<float>(log2n, le); });
    return cached_table(key, [&] { return build_twiddles<double>(log2n, le); });
}

const void* lct_twiddle_table_r8(int log2n) {
    if (log2n < 4) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    return cached_table(std::make_tuple(dev, 30, log2n), [&] { return build_twiddles<float>(log2n, 3); });
}

const void* lct_twiddle_table_pair(int log2n, int le) {
    if (log2n <= le) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    return cached_table(std::make_tuple(dev, 10 + le, log2n), [&] {
        std::vector<float> t = build_twiddles<float>(log2n, le);
        std::vector<float> b(2 * t.size());
        for (size_t k = 0; k < t.size() / 2; ++k) {
            b[4 * k + 0] = t[2 * k];
            b[4 * k + 1] = t[2 * k];
            b[4 * k + 2] = t[2 * k + 1];
            b[4 * k + 3] = t[2 * k + 1];
        }
        return b;
    });
}

// ---------------------------------------------------------------------------
// chirp-convolution (Bluestein) spectra for N that is not a power of two
// ---------------------------------------------------------------------------
int lct_blue_log2m(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < 2 * n - 1) ++l;
    return l;
}

bool lct_blue_supported(int dtype, int64_t n) {
    return n >= 3 && n <= (dtype == LCT_C64 ? kBlueMaxN64 : kBlueMaxN128) && ilog2_exact(n) < 0;
}

namespace {
// In-place forward DFT (sign -1) of a power-of-two length: iterative radix-2
// with the twiddles e^{-2 pi i k / M} taken in long double.
void host_fft(std::vector<std::complex<double>>& a) {
    const size_t M = a.size();
    for (size_t i = 1, j = 0; i < M; ++i) {
        size_t bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    std::vector<std::complex<double>> w(M / 2);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (size_t k = 0; k < M / 2; ++k) {
        const long double ang = -two_pi * (long double)k / (long double)M;
        w[k] = {(double)cosl(ang), (double)sinl(ang)};
    }
    for (size_t len = 2; len <= M; len <<= 1) {
        const size_t step = M / len;
        for (size_t i = 0; i < M; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w[k * step];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// H_j / M for the chirp h_n = e^{i pi n^2 / N}, |n| < N, placed circularly
// (h[n] for n >= 0, h[M - n] for n < 0) in length M; the phase n^2/(2N)
// turns is reduced exactly in integers.
template <class T>
std::vector<T> build_blue_spectrum(int64_t n) {
    const int64_t M = (int64_t)1 << lct_blue_log2m(n);
    std::vector<std::complex<double>> h((size_t)M, {0.0, 0.0});
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int64_t t = 0; t < n; ++t) {
        const int64_t r = (t * t) % (2 * n);
        const long double ang = two_pi * (long double)r / (long double)(2 * n);
        const std::complex<double> v = {(double)cosl(ang), (double)sinl(ang)};
        h[(size_t)t] = v;
        if (t > 0) h[(size_t)(M - t)] = v;
    }
    host_fft(h);
    std::vector<T> out(2 * (size_t)M);
    for (int64_t j = 0; j < M; ++j) {
        out[2 * j] = (T)(h[(size_t)j].real() / (double)M);
        out[2 * j + 1] = (T)(h[(size_t)j].imag() / (double)M);
    }
    return out;
}
}  // namespace

const void* lct_blue_spectrum(int dtype, int64_t n) {
    if (!lct_blue_supported(dtype, n)) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    const auto key = std::make_tuple(dev, 100 + dtype, (int)n);
    if (dtype == LCT_C64) return cached_table(key, [&] { return build_blue_spectrum<float>(n); });
    return cached_table(key, [&] { return build_blue_spectrum<double>(n); });
}

// ---------------------------------------------------------------------------
// mixed-radix plans and twiddles for 7-smooth N that is not a power of two
// ---------------------------------------------------------------------------
bool lct_mixed_ok(int64_t n) {
    if (n < 3 || n > 8192 || ilog2_exact(n) >= 0) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

bool lct_mixed_make_plan(int64_t n, int dtype, lct_mixed_plan* pl) {
    if (!lct_mixed_ok(n)) return false;
    std::memset(pl, 0, sizeof(*pl));
    pl->n = (int)n;
    // radices: the power of two as 16s, then one 8, 4 or 2; then 7s, 5s, 3s
    int64_t m = n;
    int twos = 0;
    while (m % 2 == 0) { m /= 2; ++twos; }
    int np = 0;
    while (twos >= 4) { pl->radix[np++] = 16; twos -= 4; }
    if (twos > 0) pl->radix[np++] = 1 << twos;
    for (int p : {7, 5, 3})
        while (m % p == 0) { pl->radix[np++] = p; m /= p; }
    if (np > kMixedMaxPasses) return false;
    pl->npass = np;
    int64_t ns = 1, off = 0, threads = 32;
    for (int p = 0; p < np; ++p) {
        const int r = pl->radix[p];
        pl->ns[p] = (int)ns;
        pl->magic[p] = ns > 1 ? (uint32_t)((((uint64_t)1) << 32) / (uint64_t)ns + 1) : 0;
        pl->twoff[p] = (int)off;
        if (p > 0) off += ns * (r - 1);
        const int64_t per = (int64_t)r * (16 / r);          // samples a thread holds in a pass
        const int64_t t = (n + per - 1) / per;
        if (t > threads) threads = t;
        ns *= r;
    }
    threads = (threads + 31) / 32 * 32;
    if (threads > (dtype == LCT_C64 ? 1024 : 512)) return false;
    pl->threads = (int)threads;
    const unsigned __int128 inv = (~(unsigned __int128)0) / (unsigned __int128)(2 * n);   // 2^128/(2N)
    pl->inv_hi = (uint64_t)(inv >> 64);
    pl->inv_lo = (uint64_t)inv;
    return true;
}

namespace {
// e^{-2 pi i j r / (Ns R)} for every pass p >= 1 (j < Ns, 1 <= r < R), the
// angle reduced exactly in integers, sine and cosine in long double.
template <class T>
std::vector<T> build_mixed_twiddles(const lct_mixed_plan& pl) {
    size_t total = 0;
    for (int p = 1; p < pl.npass; ++p) total += (size_t)pl.ns[p] * (pl.radix[p] - 1);
    const size_t head = kMixedPlanBytes / sizeof(T);        // the plan, then the table
    std::vector<T> out(head + 2 * (total ? total : 1), (T)0);
    std::memcpy(out.data(), &pl, sizeof(pl));
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int p = 1; p < pl.npass; ++p) {
        const int64_t ns = pl.ns[p], R = pl.radix[p], L = ns * R;
        for (int64_t r = 1; r < R; ++r)
            for (int64_t j = 0; j < ns; ++j) {
                const int64_t q = (j * r) % L;
                const long double ang = -two_pi * (long double)q / (long double)L;
                const size_t e = (size_t)pl.twoff[p] + (size_t)((r - 1) * ns + j);
                out[head + 2 * e] = (T)cosl(ang);
                out[head + 2 * e + 1] = (T)sinl(ang);
            }
    }
    return out;
}
}  // namespace

const void* lct_mixed_twiddles(int dtype, int64_t n) {
    lct_mixed_plan pl;
    if (!lct_mixed_make_plan(n, dtype, &pl)) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    const auto key = std::make_tuple(dev, 200 + dtype, (int)n);
    if (dtype == LCT_C64) return cached_table(key, [&] { return build_mixed_twiddles<float>(pl); });
    return cached_table(key, [&] { return build_mixed_twiddles<double>(pl); });
}

int lct_make_desc_host(int64_t N, const double* p, int64_t offset, lct_desc* D) {
    return (int)make_desc(N, p, offset, D);
}
