/*
 * CPU oracle for the discrete linear canonical transform (XFT) of
 * Campos & Figueroa, "A fast algorithm for the linear canonical transform".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test suite, the package smoke
 * check and the CPU-baseline leg of the benchmark may load or call it.  It
 * shares no code, header, table or constant with the CUDA library, and the
 * library never calls it.
 *
 * What it computes (all in FP64, phases in extended precision):
 *
 *   Sampling nodes, eq. (asymcer):   x_k = (2k - N - 1) pi / (2 sqrt(2N)),  k = 1..N
 *   Node spacing,   eq. (deltk):     dx  = pi / sqrt(2N)
 *   Output points,  Algorithm:       y_j = 4 b x_j / pi
 *
 *   For b != 0, the Riemann sum of the chirp-FT-chirp form of the LCT,
 *   eq. (lctdos), on those nodes (this is the matrix L = S1 F S2 of Sec. 3):
 *
 *     G_j = e^{i d y_j^2 / (2b)} / sqrt(2 pi i b)
 *           * sum_k e^{-i x_k y_j / b} e^{i a x_k^2 / (2b)} f_k dx
 *
 *   For b == 0, the definition below eq. (lctuno):  G(y) = sqrt(d) e^{i c d y^2/2} f(d y),
 *   evaluated on the output grid y_j = x_j / d so that f(d y_j) = f_k=j exactly.
 *
 *   Complex parameters (the fractional transform for complex z, Sec. 1):
 *   the same sums with complex a, b, c, d.  The output chirp may then carry
 *   a real exponential e^{-rho_j}, rho_j = -Im(d y_j^2/(2b)) (b != 0) or
 *   -Im(c d y_j^2 / 2) (b == 0); the oracle returns Ghat_j = G_j e^{-rho_j}
 *   and rho_j separately, so that no value overflows.  For real parameters
 *   rho is identically zero and Ghat = G.
 *
 * Exactness of the phases.  The parameters are taken as exact FP64 values.
 * Every phase is reduced modulo one turn in long double (64-bit significand
 * on x86-64, binary128 on aarch64) before its sine and cosine are taken:
 *   a x_k^2 / (2b)   = (a/b) pi^2 m_k^2 / (16 N),     m_k = 2k - N - 1 (odd)
 *   d y_j^2 / (2b)   = b d m_j^2 / N
 *   x_k y_j / b      = pi m_j m_k / (2N)   (b cancels exactly)
 * The last one is an exact rational multiple of pi; its exponential is read
 * from a table of the 4N-th roots of unity indexed by (m_j m_k) mod 4N.
 * Sums use Neumaier compensated summation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

static const ld PI_L = 3.141592653589793238462643383279502884L;

/* Complex helpers (explicit re/im keeps every step visible). */
typedef struct { double re, im; } cplx;

static cplx c_mul(cplx a, cplx b) {
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}
static cplx c_conj(cplx a) { cplx r = {a.re, -a.im}; return r; }
static cplx c_scale(cplx a, double s) { cplx r = {a.re * s, a.im * s}; return r; }
static cplx c_div(cplx a, cplx b) {
    /* Plain complex division, scaled to avoid overflow. */
    double s = fabs(b.re) > fabs(b.im) ? fabs(b.re) : fabs(b.im);
    double br = b.re / s, bi = b.im / s;
    double den = br * br + bi * bi;
    cplx r = {(a.re * br + a.im * bi) / (s * den), (a.im * br - a.re * bi) / (s * den)};
    return r;
}
/* Principal square root (branch cut on the negative real axis). */
static cplx c_sqrt(cplx a) {
    double r = hypot(a.re, a.im);
    double t = sqrt(0.5 * (r + fabs(a.re)));
    cplx out;
    if (t == 0.0) { out.re = 0.0; out.im = 0.0; return out; }
    if (a.re >= 0.0) { out.re = t; out.im = a.im / (2.0 * t); }
    else { out.re = fabs(a.im) / (2.0 * t); out.im = (a.im >= 0.0 ? t : -t); }
    return out;
}

/* Parameter products and quotients in long double, so that the phases
 * below keep the precision of their exact-FP64 inputs. */
typedef struct { ld re, im; } lcplx;
static lcplx l_mul(cplx a, cplx b) {
    lcplx r = {(ld)a.re * b.re - (ld)a.im * b.im, (ld)a.re * b.im + (ld)a.im * b.re};
    return r;
}
static lcplx l_div(cplx a, cplx b) {
    ld den = (ld)b.re * b.re + (ld)b.im * b.im;
    lcplx r = {((ld)a.re * b.re + (ld)a.im * b.im) / den, ((ld)a.im * b.re - (ld)a.re * b.im) / den};
    return r;
}

/* e^{i * 2 pi * turns}, with the turn count reduced to [-1/2, 1/2] first. */
static cplx expi_turns(ld turns) {
    ld t = turns - floorl(turns + 0.5L);
    ld ang = 2.0L * PI_L * t;
    cplx r = {(double)cosl(ang), (double)sinl(ang)};
    return r;
}

/* Neumaier compensated accumulator for one real component. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum* a) { return a->s + a->c; }

/* Odd integer index of node k (0-based): m_k = 2(k+1) - N - 1. */
static int64_t node_m(int64_t N, int64_t k) { return 2 * k - N + 1; }

/* Nodes x_k of eq. (asymcer), 0-based. */
void oracle_nodes(int64_t N, double* x) {
    for (int64_t k = 0; k < N; ++k)
        x[k] = (double)(PI_L * (ld)node_m(N, k) / (2.0L * sqrtl(2.0L * (ld)N)));
}

/* Per-signal description shared by the transform, adjoint and gradient. */
typedef struct {
    int64_t N;
    int b_zero;          /* 1: b == 0 branch */
    cplx pre;            /* dx / sqrt(2 pi i b)                         (b != 0) */
    cplx sqrt_d;         /* sqrt(d)                                     (b == 0) */
    cplx* chirp_in;      /* e^{i a x_k^2/(2b)}                          (b != 0) */
    cplx* chirp_out;     /* e^{i d y_j^2/(2b)} e^{-rho_j}  or  e^{i c d y_j^2/2} e^{-rho_j} */
    double* rho;         /* rho_j */
    cplx* root;          /* root[r] = e^{-i pi r / (2N)}, r = 0 .. 4N-1   (b != 0) */
} signal_ops;

static int ops_build(signal_ops* op, int64_t N, const double* abcd) {
    cplx a = {abcd[0], abcd[1]}, b = {abcd[2], abcd[3]};
    cplx c = {abcd[4], abcd[5]}, d = {abcd[6], abcd[7]};
    memset(op, 0, sizeof(*op));
    op->N = N;
    op->b_zero = (b.re == 0.0 && b.im == 0.0);
    op->chirp_out = (cplx*)malloc(sizeof(cplx) * N);
    op->rho = (double*)malloc(sizeof(double) * N);
    if (!op->chirp_out || !op->rho) return -1;
    if (op->b_zero) {
        /* G_j = sqrt(d) e^{i c d y_j^2 / 2} f_j with y_j = x_j / d, so the
         * phase is (c/(2d)) x_j^2 = (c/d) pi^2 m_j^2 / (16 N). */
        op->sqrt_d = c_sqrt(d);
        lcplx cd = l_div(c, d);
        for (int64_t j = 0; j < N; ++j) {
            ld m2 = (ld)node_m(N, j) * (ld)node_m(N, j);
            ld re_turns = cd.re * PI_L * m2 / (32.0L * (ld)N);   /* Re(phase)/(2 pi) */
            double im = (double)(cd.im * PI_L * PI_L * m2 / (16.0L * (ld)N));
            op->rho[j] = -im;
            /* e^{i phase} e^{-rho_j} = e^{i Re(phase)}: the real exponential cancels. */
            op->chirp_out[j] = expi_turns(re_turns);
        }
        return 0;
    }
    op->chirp_in = (cplx*)malloc(sizeof(cplx) * N);
    op->root = (cplx*)malloc(sizeof(cplx) * 4 * N);
    if (!op->chirp_in || !op->root) return -1;

    /* dx / sqrt(2 pi i b), eq. (deltk) and eq. (lctuno) with principal root. */
    double dx = (double)(PI_L / sqrtl(2.0L * (ld)N));
    cplx two_pi_i_b = {-2.0 * (double)PI_L * b.im, 2.0 * (double)PI_L * b.re};
    cplx one = {1.0, 0.0};
    op->pre = c_scale(c_div(one, c_sqrt(two_pi_i_b)), dx);

    /* a x_k^2/(2b) with x_k^2 = pi^2 m_k^2 / (8N). */
    lcplx ab = l_div(a, b);
    for (int64_t k = 0; k < N; ++k) {
        ld m2 = (ld)node_m(N, k) * (ld)node_m(N, k);
        ld re_turns = ab.re * PI_L * m2 / (32.0L * (ld)N);
        double im = (double)(ab.im * PI_L * PI_L * m2 / (16.0L * (ld)N));
        /* e^{i phase} = e^{i Re(phase)} e^{-Im(phase)} */
        op->chirp_in[k] = c_scale(expi_turns(re_turns), exp(-im));
    }
    /* d y_j^2/(2b) with y_j = 4 b x_j / pi:  = b d m_j^2 / N. */
    lcplx bd = l_mul(b, d);
    for (int64_t j = 0; j < N; ++j) {
        ld m2 = (ld)node_m(N, j) * (ld)node_m(N, j);
        ld re_turns = bd.re * m2 / (2.0L * PI_L * (ld)N);
        double im = (double)(bd.im * m2 / (ld)N);
        op->rho[j] = -im;
        op->chirp_out[j] = expi_turns(re_turns);   /* e^{i phase} e^{-rho_j} */
    }
    /* e^{-i x_k y_j / b} = e^{-i pi (m_j m_k) / (2N)}: the 4N-th roots of unity. */
    for (int64_t r = 0; r < 4 * N; ++r)
        op->root[r] = expi_turns(-(ld)r / (4.0L * (ld)N));
    return 0;
}

static void ops_free(signal_ops* op) {
    free(op->chirp_in); free(op->chirp_out); free(op->rho); free(op->root);
    memset(op, 0, sizeof(*op));
}

static int64_t root_index(int64_t N, int64_t mj, int64_t mk) {
    int64_t q = 4 * N;
    int64_t r = (mj * mk) % q;
    return r < 0 ? r + q : r;
}

/* Dense matrix element Lhat_jk = e^{-rho_j} L_jk (b != 0 branch). */
static cplx ops_element(const signal_ops* op, int64_t j, int64_t k) {
    cplx kern = op->root[root_index(op->N, node_m(op->N, j), node_m(op->N, k))];
    cplx v = c_mul(op->chirp_out[j], c_mul(kern, op->chirp_in[k]));
    return c_mul(op->pre, v);
}

/*
 * Forward transform of `count` signals of length N (complex, interleaved
 * re/im, row-major [count][N]).  abcd: count x 8 doubles
 * (a_re, a_im, b_re, b_im, c_re, c_im, d_re, d_im).  If abcd_stride is 0 the
 * same parameters serve every signal.  Writes Ghat (count x N complex) and,
 * if rho != NULL, rho (count x N).  Returns 0 on success.
 */
int oracle_lct(int64_t N, int64_t count, const double* abcd, int64_t abcd_stride,
               const double* f, double* G, double* rho) {
    for (int64_t s = 0; s < count; ++s) {
        signal_ops op;
        if (ops_build(&op, N, abcd + s * abcd_stride) != 0) { ops_free(&op); return -1; }
        const cplx* fs = (const cplx*)(f + 2 * s * N);
        cplx* Gs = (cplx*)(G + 2 * s * N);
        if (rho) memcpy(rho + s * N, op.rho, sizeof(double) * N);
        if (op.b_zero) {
            for (int64_t j = 0; j < N; ++j)
                Gs[j] = c_mul(op.sqrt_d, c_mul(op.chirp_out[j], fs[j]));
            ops_free(&op);
            continue;
        }
        /* g_k = e^{i a x_k^2/(2b)} f_k, then the sum over k for every j. */
        cplx* g = (cplx*)malloc(sizeof(cplx) * N);
        if (!g) { ops_free(&op); return -1; }
        for (int64_t k = 0; k < N; ++k) g[k] = c_mul(op.chirp_in[k], fs[k]);
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < N; ++j) {
            nsum sr = {0, 0}, si = {0, 0};
            int64_t mj = node_m(N, j);
            for (int64_t k = 0; k < N; ++k) {
                cplx t = c_mul(op.root[root_index(N, mj, node_m(N, k))], g[k]);
                nsum_add(&sr, t.re);
                nsum_add(&si, t.im);
            }
            cplx acc = {nsum_get(&sr), nsum_get(&si)};
            Gs[j] = c_mul(op.pre, c_mul(op.chirp_out[j], acc));
        }
        free(g);
        ops_free(&op);
    }
    return 0;
}

/*
 * Adjoint: h = Lhat^H g for each signal (h_k = sum_j conj(Lhat_jk) g_j).
 * Same argument conventions as oracle_lct.
 */
int oracle_lct_adjoint(int64_t N, int64_t count, const double* abcd, int64_t abcd_stride,
                       const double* g, double* h) {
    for (int64_t s = 0; s < count; ++s) {
        signal_ops op;
        if (ops_build(&op, N, abcd + s * abcd_stride) != 0) { ops_free(&op); return -1; }
        const cplx* gs = (const cplx*)(g + 2 * s * N);
        cplx* hs = (cplx*)(h + 2 * s * N);
        if (op.b_zero) {
            for (int64_t k = 0; k < N; ++k)
                hs[k] = c_mul(c_conj(c_mul(op.sqrt_d, op.chirp_out[k])), gs[k]);
            ops_free(&op);
            continue;
        }
        #pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < N; ++k) {
            nsum sr = {0, 0}, si = {0, 0};
            for (int64_t j = 0; j < N; ++j) {
                cplx t = c_mul(c_conj(ops_element(&op, j, k)), gs[j]);
                nsum_add(&sr, t.re);
                nsum_add(&si, t.im);
            }
            hs[k].re = nsum_get(&sr);
            hs[k].im = nsum_get(&si);
        }
        ops_free(&op);
    }
    return 0;
}

/*
 * Dense-matrix gradient of a real loss with respect to the real parameters
 * (a, b, d) of each signal, b != 0, real parameters only.  With the output
 * points y_j = 4 b x_j / pi moving with b, each matrix element is
 *   L_jk = dx (2 pi i b)^{-1/2} e^{i 8 b d x_j^2 / pi^2} e^{-i 4 x_j x_k / pi} e^{i a x_k^2/(2b)}
 * and its partial derivatives are L_jk times
 *   d/da : i x_k^2 / (2b)
 *   d/db : -1/(2b) + i 8 d x_j^2 / pi^2 - i a x_k^2 / (2 b^2)
 *   d/dd : i 8 b x_j^2 / pi^2.
 * With the cotangent g_j = dl/dRe(G_j) + i dl/dIm(G_j), dl/dp = Re sum_j conj(g_j) sum_k (dL_jk/dp) f_k.
 * grad: count x 3 doubles (dl/da, dl/db, dl/dd).
 */
int oracle_lct_grad_params(int64_t N, int64_t count, const double* abcd, int64_t abcd_stride,
                           const double* f, const double* g, double* grad) {
    double* x = (double*)malloc(sizeof(double) * N);
    if (!x) return -1;
    oracle_nodes(N, x);
    const double pi = (double)PI_L;
    for (int64_t s = 0; s < count; ++s) {
        const double* p = abcd + s * abcd_stride;
        double a = p[0], b = p[2], d = p[6];
        if (b == 0.0 || p[1] != 0.0 || p[3] != 0.0 || p[5] != 0.0 || p[7] != 0.0) { free(x); return -2; }
        signal_ops op;
        if (ops_build(&op, N, p) != 0) { ops_free(&op); free(x); return -1; }
        const cplx* fs = (const cplx*)(f + 2 * s * N);
        const cplx* gs = (const cplx*)(g + 2 * s * N);
        double ga = 0.0, gb = 0.0, gd = 0.0;
        #pragma omp parallel for schedule(static) reduction(+:ga, gb, gd)
        for (int64_t j = 0; j < N; ++j) {
            nsum sa_r = {0, 0}, sa_i = {0, 0}, sb_r = {0, 0}, sb_i = {0, 0}, sd_r = {0, 0}, sd_i = {0, 0};
            double xj2 = x[j] * x[j];
            for (int64_t k = 0; k < N; ++k) {
                cplx Lf = c_mul(ops_element(&op, j, k), fs[k]);
                double xk2 = x[k] * x[k];
                cplx da = {0.0, xk2 / (2.0 * b)};
                cplx db = {-1.0 / (2.0 * b), 8.0 * d * xj2 / (pi * pi) - a * xk2 / (2.0 * b * b)};
                cplx dd = {0.0, 8.0 * b * xj2 / (pi * pi)};
                cplx ta = c_mul(da, Lf), tb = c_mul(db, Lf), td = c_mul(dd, Lf);
                nsum_add(&sa_r, ta.re); nsum_add(&sa_i, ta.im);
                nsum_add(&sb_r, tb.re); nsum_add(&sb_i, tb.im);
                nsum_add(&sd_r, td.re); nsum_add(&sd_i, td.im);
            }
            cplx gj = c_conj(gs[j]);
            cplx va = {nsum_get(&sa_r), nsum_get(&sa_i)};
            cplx vb = {nsum_get(&sb_r), nsum_get(&sb_i)};
            cplx vd = {nsum_get(&sd_r), nsum_get(&sd_i)};
            ga += c_mul(gj, va).re;
            gb += c_mul(gj, vb).re;
            gd += c_mul(gj, vd).re;
        }
        grad[3 * s + 0] = ga;
        grad[3 * s + 1] = gb;
        grad[3 * s + 2] = gd;
        ops_free(&op);
    }
    free(x);
    return 0;
}

/* The full dense matrix Lhat (N x N complex, row-major [j][k]) of one signal. */
int oracle_lct_matrix(int64_t N, const double* abcd, double* L) {
    signal_ops op;
    if (ops_build(&op, N, abcd) != 0) { ops_free(&op); return -1; }
    cplx* Lc = (cplx*)L;
    for (int64_t j = 0; j < N; ++j)
        for (int64_t k = 0; k < N; ++k) {
            if (op.b_zero) {
                cplx z = {0.0, 0.0};
                Lc[j * N + k] = (j == k) ? c_mul(op.sqrt_d, op.chirp_out[j]) : z;
            } else {
                Lc[j * N + k] = ops_element(&op, j, k);
            }
        }
    ops_free(&op);
    return 0;
}

/* Number of OpenMP threads a parallel region of this library would use. */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Fractional transform for complex z on the real nodes, Sec. 2: the matrix
 * of eq. (fasy) (the large-N form of eq. (tmat) by Mehler's formula) applied
 * to the samples f_k = f(x_k), eq. (primcuad), i.e. the Riemann sum of
 * eq. (eqifft) at y_j = x_j (eq. (cuadtrfor)):
 *
 *   g_j = sqrt(2/(1 - z^2)) dx sum_k e^{E_jk} f_k,
 *   E_jk = -[(1 + z^2)(x_j^2 + x_k^2) - 4 x_j x_k z] / (2 (1 - z^2)),
 *
 * for |z| <= 1, z != +-1 (the paper states |z| < 1; on the unit circle the
 * same sum is the real-angle kernel).  With x_k = pi m_k / (2 sqrt(2N)),
 *   x_j^2 + x_k^2 = pi^2 (m_j^2 + m_k^2) / (8N),  x_j x_k = pi^2 m_j m_k / (8N),
 * integers formed exactly.  P = (1 + z^2) / (2 (1 - z^2)) and
 * Q = 2 z / (1 - z^2) are formed in long double from the FP64 z, so that
 *   E_jk = -P pi^2 (m_j^2 + m_k^2)/(8N) + Q pi^2 m_j m_k/(8N),
 * and Im E is reduced modulo one turn in long double before its sine and
 * cosine are taken.  f, g: count signals of N interleaved complex doubles.
 * Returns -1 for |z| > 1 or z = +-1.
 */
int oracle_frft_mehler(int64_t N, int64_t count, double z_re, double z_im, const double* f,
                       double* g) {
    const ld zr = z_re, zi = z_im;
    if (zr * zr + zi * zi > 1.0L + 1e-15L || (zi == 0.0L && fabsl(zr) == 1.0L)) return -1;
    /* z^2, 1 + z^2, 1 - z^2 */
    const ld z2r = zr * zr - zi * zi, z2i = 2.0L * zr * zi;
    const ld pr = 1.0L + z2r, pi_ = z2i;          /* 1 + z^2 */
    const ld mr = 1.0L - z2r, mi = -z2i;          /* 1 - z^2 */
    const ld den = mr * mr + mi * mi;
    /* P = (1 + z^2) / (2 (1 - z^2)),  Q = 2 z / (1 - z^2) */
    const ld Pr = (pr * mr + pi_ * mi) / (2.0L * den), Pi = (pi_ * mr - pr * mi) / (2.0L * den);
    const ld Qr = 2.0L * (zr * mr + zi * mi) / den, Qi = 2.0L * (zi * mr - zr * mi) / den;
    const ld unit = PI_L * PI_L / (8.0L * (ld)N);
    /* prefactor sqrt(2/(1 - z^2)) dx, principal root */
    cplx two = {2.0, 0.0};
    cplx omz2 = {(double)mr, (double)mi};
    cplx pre = c_scale(c_sqrt(c_div(two, omz2)), (double)(PI_L / sqrtl(2.0L * (ld)N)));
    const cplx* fc = (const cplx*)f;
    cplx* gc = (cplx*)g;
    int fail = 0;
    #pragma omp parallel
    {
        cplx* row = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!row) {
            #pragma omp atomic write
            fail = 1;
        }
        #pragma omp for schedule(dynamic, 4)
        for (int64_t j = 0; j < N; ++j) {
            if (!row) continue;
            const int64_t mj = node_m(N, j);
            for (int64_t k = 0; k < N; ++k) {
                const int64_t mk = node_m(N, k);
                const ld S = (ld)(mj * mj + mk * mk) * unit;
                const ld T = (ld)(mj * mk) * unit;
                const ld er = -Pr * S + Qr * T;
                const ld ei = -Pi * S + Qi * T;
                cplx w = expi_turns(ei / (2.0L * PI_L));
                row[k] = c_scale(w, (double)expl(er));
            }
            for (int64_t s = 0; s < count; ++s) {
                nsum sr = {0, 0}, si = {0, 0};
                const cplx* fs = fc + s * N;
                for (int64_t k = 0; k < N; ++k) {
                    cplx t = c_mul(row[k], fs[k]);
                    nsum_add(&sr, t.re);
                    nsum_add(&si, t.im);
                }
                cplx acc = {nsum_get(&sr), nsum_get(&si)};
                gc[s * N + j] = c_mul(pre, acc);
            }
        }
        free(row);
    }
    return fail ? -1 : 0;
}
