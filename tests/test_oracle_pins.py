"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a library routine, an exact invariant, or the paper's own formula
restated independently.  A plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand, an imprecise phase) fails at
least one of them.
"""
import json
import os
from math import factorial

import numpy as np
import pytest
from scipy import integrate
from scipy.special import eval_hermite, roots_hermite

import oracle as O
from oracle import closed_forms as C
from oracle import hermite as H
from conftest import rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


def rot(t):
    return [np.cos(t), np.sin(t), -np.sin(t), np.cos(t)]


# --------------------------------------------------------------------------
# nodes and grid (eq. asymcer, eq. deltk)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [64, 256])
def test_asymptotic_nodes_approach_hermite_zeros(N):
    """eq. (asymcer) approximates the zeros of H_N near the origin (library zeros)."""
    xa = O.nodes(N)
    xr, _ = roots_hermite(N)
    centre = np.abs(xa) < 1.0
    assert np.abs(xa - xr)[centre].max() < 4.0 / N
    # uniform spacing pi/sqrt(2N) of eq. (deltk), symmetric about 0
    assert np.allclose(np.diff(xa), np.pi / np.sqrt(2 * N), rtol=0, atol=1e-13)
    assert np.allclose(xa, -xa[::-1], rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# Sec. 4 worked example: Gaussian closed form
# --------------------------------------------------------------------------
def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.mark.parametrize("case", ["fig1", "fig2"])
def test_gaussian_closed_form_paper_examples(case):
    """XFT of the Gaussian of Sec. 4 against its closed form, at the paper's
    parameters (Fig. 1: N=512; Fig. 2, Fresnel b=100: N=1024)."""
    g = _golden()[case]
    N = g["N"]
    abcd = [g["a"], g["b"], g["c"], g["d"]]
    x = O.nodes(N)
    f = C.gaussian(x, g["alpha"], g["beta"], g["gamma"])
    y = O.output_grid(N, abcd).real
    G = O.lct(f, abcd)
    ref = C.gaussian_lct(y, g["alpha"], g["beta"], g["gamma"], g["a"], g["b"], g["d"])
    assert rel_l2(G, ref) < 1e-12


@pytest.mark.parametrize("case", ["fig1", "fig2"])
def test_paper_formula_matches_gaussian_integral(case):
    """eq. (exa1) as printed equals the Gaussian-integral derivation."""
    g = _golden()[case]
    y = np.linspace(-60, 60, 241)
    p = C.paper_gaussian_lct(y, g["alpha"], g["beta"], g["gamma"], g["a"], g["b"], g["c"], g["d"])
    q = C.gaussian_lct(y, g["alpha"], g["beta"], g["gamma"], g["a"], g["b"], g["d"])
    assert rel_l2(p, q) < 1e-12


def test_gaussian_closed_form_against_quadrature():
    """The closed form equals adaptive quadrature of eq. (lctuno) itself."""
    al, be, ga, a, b, d = 1.0, 2.0, 3.0, 1.0, 2.0, 2.0
    for y in [-3.0, -0.5, 0.0, 1.7]:
        def integrand(x, part):
            v = np.exp(-(al * x * x + 2 * be * x + ga)) * np.exp(1j * (a * x * x - 2 * x * y + d * y * y) / (2 * b))
            return v.real if part == 0 else v.imag
        re = integrate.quad(integrand, -30, 30, args=(0,), limit=400, epsabs=1e-14, epsrel=1e-13)[0]
        im = integrate.quad(integrand, -30, 30, args=(1,), limit=400, epsabs=1e-14, epsrel=1e-13)[0]
        direct = (re + 1j * im) / np.sqrt(2j * np.pi * b)
        closed = C.gaussian_lct(np.array([y]), al, be, ga, a, b, d)[0]
        assert abs(direct - closed) < 1e-11 * max(1.0, abs(closed))


# --------------------------------------------------------------------------
# Hermite functions: eigenfunctions of the rotation LCT / F_z
# --------------------------------------------------------------------------
def test_hermite_functions_match_library():
    x = np.linspace(-6, 6, 101)
    psi = H.hermite_functions(10, x)
    for n in range(11):
        ref = eval_hermite(n, x) * np.exp(-x * x / 2) / np.sqrt(2.0 ** n * factorial(n) * np.sqrt(np.pi))
        assert np.abs(psi[n] - ref).max() < 1e-12


def test_config0_polynomial_is_hermite_combination():
    x = np.linspace(-5, 5, 51)
    expansion = sum(cn * eval_hermite(n, x) for n, cn in C.CONFIG0_HERMITE.items()) * np.exp(-x * x / 2)
    assert np.abs(C.config0_poly(x) - expansion).max() < 1e-13


@pytest.mark.parametrize("N", [128, 256])
def test_config0_polynomial_rotation(N):
    """Rotation LCT (angle 0.7) of exp(-x^2/2)(1+0.3x+0.1x^3) = sum of eigenfunctions."""
    t = 0.7
    x = O.nodes(N)
    y = O.output_grid(N, rot(t)).real
    G = O.lct(C.config0_poly(x), rot(t))
    assert rel_l2(G, C.config0_poly_lct(t, y)) < 1e-13


def test_hermite_eigenfunctions_n0_to_10():
    N, t = 256, 0.7
    x = O.nodes(N)
    y = O.output_grid(N, rot(t)).real
    psi = H.hermite_functions(10, x)
    G = O.lct(psi, rot(t))
    for n in range(11):
        assert rel_l2(G[n], C.hermite_lct(n, t, y)) < 1e-13


@pytest.mark.parametrize("t", [0.8, np.pi / 2, 2.3])
def test_rotation_angles_including_fourier(t):
    """t = pi/2 is the ordinary Fourier transform (a = d = 0, b = 1).  Angles keep
    |cot t| < 4/pi so that the input chirp is not aliased on the grid."""
    N = 128
    x = O.nodes(N)
    y = O.output_grid(N, rot(t)).real
    psi = H.hermite_functions(6, x)
    G = O.lct(psi, rot(t))
    for n in range(7):
        assert rel_l2(G[n], C.hermite_lct(n, t, y)) < 1e-12


def test_spectral_convergence_of_xft():
    """The XFT of a smooth decaying function converges at least like 1/N (faster in fact)."""
    t = 0.7
    errs = []
    for N in [16, 32, 64]:
        x = O.nodes(N)
        y = O.output_grid(N, rot(t)).real
        errs.append(rel_l2(O.lct(C.config0_poly(x), rot(t)), C.config0_poly_lct(t, y)))
    assert errs[1] < errs[0] / 2 and errs[2] < errs[1] / 2
    assert errs[2] < 1e-9


# --------------------------------------------------------------------------
# fractional transform, real and complex z (eq. fasy/eqifft)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("z", [np.exp(-0.7j), 0.5, 0.3 + 0.4j, 0.9 * np.exp(2.0j)])
def test_frft_hermite_eigenvalues(z):
    """F_z psi_n = sqrt(2 pi) z^n psi_n (Mehler), at the XFT output points
    y_j = 4 b(z) x_j / pi (complex for |z| < 1); returned as G e^{-rho}."""
    N = 256
    x = O.nodes(N)
    y = O.output_grid(N, O.abcd_of_z(z))
    psi = H.hermite_functions(10, x)
    G, rho = O.frft(psi, z, return_rho=True)
    for n in range(11):
        ref = C.hermite_frft(n, z, y) * np.exp(-rho[n])
        assert rel_l2(G[n], ref) < 1e-12


def test_frft_matches_riemann_sum_of_mehler_kernel():
    """The z -> (a,b,c,d) mapping and the normalisation, against the Riemann
    sum of the kernel of eq. (eqifft) written out directly."""
    N = 64
    x = O.nodes(N)
    dx = np.pi / np.sqrt(2 * N)
    rng = np.random.default_rng(5)
    f = np.exp(-x * x / 3) * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    for z in [0.5 + 0.3j, 0.8 * np.exp(-1.1j), np.exp(-0.4j)]:
        y = O.output_grid(N, O.abcd_of_z(z))
        X, Y = np.meshgrid(x, y)          # [j, k]
        K = np.sqrt(2 / (1 - z * z)) * np.exp(-((1 + z * z) * (X * X + Y * Y) - 4 * X * Y * z) / (2 * (1 - z * z)))
        direct = (K * dx) @ f
        G, rho = O.frft(f, z, return_rho=True)
        assert rel_l2(G, direct * np.exp(-rho)) < 1e-12


def test_frft_unit_circle_equals_scaled_rotation():
    N, t = 128, 0.9
    z = np.exp(-1j * t)
    x = O.nodes(N)
    f = C.config0_poly(x)
    lhs = O.frft(f, z)
    rhs = O.lct(f, rot(t)) * np.sqrt(2 / (1 - z * z)) * np.sqrt(2j * np.pi * np.sin(t))
    assert rel_l2(lhs, rhs) < 1e-13


# --------------------------------------------------------------------------
# the Algorithm of Sec. 3: chirp - DFT - chirp factorisation
# --------------------------------------------------------------------------
def _algorithm_literal(f, N, a, b, d, dft_sign):
    """Steps 1-3 of the Algorithm with numpy's FFT as the DFT.  dft_sign=-1
    is the reading used by the library (forward DFT, centring phases
    conjugated); dft_sign=+1 is the sign as printed."""
    k = np.arange(N)                       # 0-based (k-1 in the paper)
    x = (2 * (k + 1) - N - 1) / np.sqrt(2 * N) * np.pi / 2
    y = 4 * b * x / np.pi
    s = -dft_sign
    u = np.exp(s * 1j * np.pi * k * (N - 1) / N) * np.exp(1j * a * x * x / (2 * b)) * f
    if dft_sign < 0:
        U = np.fft.fft(u)
    else:
        U = np.fft.ifft(u) * N
    S = (np.pi * np.exp(-s * 1j * np.pi / 2 * (N - 1) ** 2 / N) / np.sqrt(2 * N)
         * np.exp(1j * d * y * y / (2 * b)) * np.exp(s * 1j * np.pi * (N - 1) / N * k)
         / np.sqrt(2j * np.pi * b))
    return S * U


@pytest.mark.parametrize("N,abcd", [(64, (0.3, -1.2, (0.3 * 1.7 - 1) / -1.2, 1.7)),
                                    (512, (1.0, 2.0, 0.5, 2.0))])
def test_factorisation_equals_direct_sum(N, abcd):
    a, b, c, d = abcd
    rng = np.random.default_rng(N)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    G = O.lct(f, abcd)
    assert rel_l2(_algorithm_literal(f, N, a, b, d, -1), G) < 1e-12
    # With the DFT sign as printed, the same steps give the mirror image G(-y_j).
    assert rel_l2(_algorithm_literal(f, N, a, b, d, +1), G[::-1]) < 1e-12


# --------------------------------------------------------------------------
# invariants: scaled unitarity, adjoint, b = 0 branch
# --------------------------------------------------------------------------
@pytest.mark.parametrize("abcd", [(1.0, 2.0, 0.5, 2.0), (0.3, -1.5, (0.3 * 0.7 - 1) / -1.5, 0.7),
                                  (0.0, 1.0, -1.0, 0.0)])
def test_scaled_unitarity(abcd):
    """(4|b|/pi) L^H L = I: the XFT is unitary up to a scale (Sec. 5)."""
    N = 64
    L = O.lct_matrix(N, abcd)
    assert np.abs(4 * abs(abcd[1]) / np.pi * L.conj().T @ L - np.eye(N)).max() < 1e-13


def test_matrix_matches_transform_and_adjoint():
    N = 32
    abcd = (0.7, 0.9, (0.7 * 1.3 - 1) / 0.9, 1.3)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    L = O.lct_matrix(N, abcd)
    assert rel_l2(O.lct(f, abcd), L @ f) < 1e-13
    assert rel_l2(O.lct_adjoint(g, abcd), L.conj().T @ g) < 1e-13
    lhs = np.vdot(g, O.lct(f, abcd))
    rhs = np.vdot(O.lct_adjoint(g, abcd), f)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("d", [0.5, 1.7, -1.3])
def test_b_zero_branch(d):
    """b = 0: G(y) = sqrt(d) e^{i c d y^2/2} f(d y) on y_j = x_j / d."""
    N = 128
    c = 0.8
    abcd = (1.0 / d, 0.0, c, d)
    x = O.nodes(N)
    f = C.gaussian(x, 0.5, 0.3, 0.1)
    y = O.output_grid(N, abcd).real
    ref = np.sqrt(complex(d)) * np.exp(0.5j * c * d * y * y) * C.gaussian(d * y, 0.5, 0.3, 0.1)
    assert rel_l2(O.lct(f, abcd), ref) < 1e-14


# --------------------------------------------------------------------------
# dense-matrix parameter gradient vs finite differences
# --------------------------------------------------------------------------
def test_param_gradient_vs_finite_differences():
    N = 64
    a, b, d = 0.6, 1.1, -0.8
    rng = np.random.default_rng(2)
    x = O.nodes(N)
    f = np.exp(-x * x / 4) * (1 + 0.1 * rng.standard_normal(N))
    T = rng.standard_normal(N) + 1j * rng.standard_normal(N)

    def loss(a_, b_, d_):
        G = O.lct(f, (a_, b_, (a_ * d_ - 1) / b_, d_))
        return float(np.sum(np.abs(G - T) ** 2))

    G = O.lct(f, (a, b, (a * d - 1) / b, d))
    g = 2.0 * (G - T)                      # dl/dRe G + i dl/dIm G
    grad = O.lct_grad_params(f, g, (a, b, (a * d - 1) / b, d))[0]
    h = 1e-4
    fd = []
    for i in range(3):
        def at(s):
            p = [a, b, d]
            p[i] += s
            return loss(*p)
        # Richardson-extrapolated central difference
        d1 = (at(h) - at(-h)) / (2 * h)
        d2 = (at(h / 2) - at(-h / 2)) / h
        fd.append((4 * d2 - d1) / 3)
    assert np.allclose(grad, fd, rtol=1e-7, atol=1e-9)


# --------------------------------------------------------------------------
# oracle B: the Hermite-zero discrete FrFT of Sec. 2
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [8, 16, 64])
def test_hermite_zero_nodes_are_zeros_of_HN(N):
    x, _ = H.hermite_zero_basis(N)
    xr, _ = roots_hermite(N)
    assert np.abs(x - xr).max() < 1e-12


def test_eigenvectors_match_ortvec():
    """Columns of U equal eq. (ortvec), evaluated literally at small N."""
    N = 12
    x, U = H.hermite_zero_basis(N)
    Hp = H.hermite_polynomials(N, x)
    Ul = np.empty((N, N))
    for k in range(1, N + 1):
        for n in range(1, N + 1):
            Ul[n - 1, k - 1] = ((-1) ** (N + k) * np.sqrt(2.0 ** (N - n) * factorial(N - 1) / (N * factorial(n - 1)))
                                * Hp[n - 1, k - 1] / Hp[N - 1, k - 1])
    assert np.abs(Ul - U).max() < 1e-12


def test_hermite_zero_frft_identities():
    N = 64
    z = np.exp(-0.8j)
    x, F = H.hermite_zero_frft(N, z)
    assert np.abs(F.conj().T @ F - 2 * np.pi * np.eye(N)).max() < 1e-12     # unitary up to sqrt(2 pi)
    _, U = H.hermite_zero_basis(N)
    for n in [0, 1, 5, 20]:
        v = U[n, :]                                                      # row n of U
        assert np.abs(F @ v - np.sqrt(2 * np.pi) * z ** n * v).max() < 1e-12
    z1, z2 = 0.7 * np.exp(0.3j), 0.9 * np.exp(-1.2j)
    _, F1 = H.hermite_zero_frft(N, z1)
    _, F2 = H.hermite_zero_frft(N, z2)
    _, F12 = H.hermite_zero_frft(N, z1 * z2)
    assert np.abs(F1 @ F2 - np.sqrt(2 * np.pi) * F12).max() < 1e-12      # group law


@pytest.mark.parametrize("z", [np.exp(-0.7j), 0.5, 0.6 + 0.3j])
def test_hermite_zero_frft_converges_like_one_over_N(z):
    """Sec. 1: the quadrature converges O(1/N) to the continuous transform."""
    scaled = []
    for N in [32, 64, 128, 256]:
        x, F = H.hermite_zero_frft(N, z)
        err = rel_l2(F @ C.config0_poly(x), C.config0_poly_frft(z, x))
        scaled.append(err * N)
    scaled = np.array(scaled)
    assert scaled.max() / scaled.min() < 1.1


# --------------------------------------------------------------------------
# group law of the LCT (Sec. 1: LCT(M2) LCT(M1) = LCT(M2 M1), up to the
# metaplectic sign) on the discrete transform
# --------------------------------------------------------------------------
def _mat(p):
    a, b, c, d = p
    return np.array([[a, b], [c, d]], dtype=np.float64)


# (a1, d1, b2, d2); b1 = s pi/4 makes the first output grid y_j = 4 b1 x_j / pi
# equal to +-x_j, so the first output is a sample vector on the second input
# grid.  a2 = b2 (1 - d1) / b1 then makes the composed b equal b2, so both
# sides land on the same output points.
GROUP_CASES = [(0.6, 1.3, -1.3, 0.8), (-1.1, 0.4, 0.7, -1.5),
               (0.2, -0.9, 1.9, 0.3), (0.9, 0.5, -0.6, 1.7)]


@pytest.mark.parametrize("s", [+1, -1])
@pytest.mark.parametrize("case", GROUP_CASES)
def test_group_law_on_gaussians(case, s):
    """O.lct(O.lct(f, M1), M2) = +-O.lct(f, M2 M1) for chirped, shifted
    Gaussians (well resolved, so the discretisation error is spectrally small).
    s = -1: b1 = -pi/4, the first output grid is the reversed input grid
    (y_j = -x_j = x_{N-1-j}), so the intermediate is reversed before the second
    transform; with case 2 the first factor then has b < 0 and the product
    b > 0, so a wrong branch of sqrt(2 pi i b) at b < 0 does not cancel."""
    N = 512
    a1, d1, b2, d2 = case
    b1 = s * np.pi / 4
    M1 = (a1, b1, (a1 * d1 - 1) / b1, d1)
    a2 = b2 * (1 - d1) / b1
    M2 = (a2, b2, (a2 * d2 - 1) / b2, d2)
    M = _mat(M2) @ _mat(M1)
    assert abs(np.linalg.det(M) - 1) < 1e-12 and abs(M[0, 1] - b2) < 1e-12
    x = O.nodes(N)
    f = C.gaussian(x, 0.5, 0.4, 0.2) * np.exp(0.3j * x * x)
    G1 = O.lct(f, M1)
    if s < 0:
        G1 = G1[::-1]
    lhs = O.lct(G1, M2)
    rhs = O.lct(f, tuple(M.ravel()))
    assert min(rel_l2(lhs, rhs), rel_l2(-lhs, rhs)) < 1e-12


def test_group_law_fails_for_a_swapped_composition():
    """The same check rejects the product taken in the wrong order (M1 M2), so
    it does test how the two parameter sets compose."""
    N = 512
    a1, d1, b2, d2 = GROUP_CASES[0]
    b1 = np.pi / 4
    M1 = (a1, b1, (a1 * d1 - 1) / b1, d1)
    a2 = b2 * (1 - d1) / b1
    M2 = (a2, b2, (a2 * d2 - 1) / b2, d2)
    x = O.nodes(N)
    f = C.gaussian(x, 0.5, 0.4, 0.2) * np.exp(0.3j * x * x)
    lhs = O.lct(O.lct(f, M1), M2)
    wrong = tuple((_mat(M1) @ _mat(M2)).ravel())
    rhs = O.lct(f, wrong)
    assert min(rel_l2(lhs, rhs), rel_l2(-lhs, rhs)) > 1e-2


def _gaussian_lct_branches_written_out(y, al, be, ga, a, b, d):
    """The Gaussian integral of eq. (lctuno) for real parameters, alpha > 0,
    with every square root written as modulus and argument:
      1/sqrt(2 pi i b) = e^{-i sgn(b) pi/4} / sqrt(2 pi |b|)   (principal root),
      sqrt(pi/A) = sqrt(pi/|A|) e^{-i arg(A)/2},  A = alpha - i a/(2b),
      arg(A) = -arctan(a / (2 b alpha))  (Re A = alpha > 0).
    The same phase term appears in eq. (exa1) as e^{(i/2) arctan(a/(2 alpha b))}."""
    y = np.asarray(y, dtype=np.float64)
    inv_root = np.exp(-1j * np.sign(b) * np.pi / 4) / np.sqrt(2 * np.pi * abs(b))
    A = al - 1j * a / (2 * b)
    sqrt_pi_over_A = np.sqrt(np.pi / abs(A)) * np.exp(0.5j * np.arctan(a / (2 * b * al)))
    B = -2 * be - 1j * y / b
    return inv_root * sqrt_pi_over_A * np.exp(B * B / (4 * A) - ga + 1j * d * y * y / (2 * b))


@pytest.mark.parametrize("N,abcd,gauss", [
    (512, (1.0, -2.0, -0.5, 2.0), (1.0, 2.0, 3.0)),        # Fig. 1 case with b -> -b
    (1024, (1.0, -100.0, 0.0, 1.0), (2.0, 1.0, 3.0)),      # Fig. 2 (Fresnel) with b -> -b
    (512, (-0.7, -1.4, (-0.7 * 0.9 - 1) / -1.4, 0.9), (0.6, -0.3, 0.2)),
])
def test_gaussian_at_negative_b_with_branches_written_out(N, abcd, gauss):
    """b < 0: modulus and phase of the oracle's output against the closed form
    whose roots are written as modulus and argument (independent of the complex
    square root used by the oracle and by gaussian_lct)."""
    a, b, c, d = abcd
    al, be, ga = gauss
    x = O.nodes(N)
    G = O.lct(C.gaussian(x, al, be, ga), abcd)
    y = O.output_grid(N, abcd).real
    ref = _gaussian_lct_branches_written_out(y, al, be, ga, a, b, d)
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert np.abs(np.abs(G) - np.abs(ref)).max() < 1e-12 * np.abs(ref).max()
    dphi = np.angle(G[big] / ref[big])
    assert np.abs(dphi).max() < 1e-10
    assert rel_l2(G, ref) < 1e-12


@pytest.mark.parametrize("N", [64, 256])
def test_eigenvectors_match_recurrence_in_high_precision(N):
    """Every column of U (signs included) equals the normalised vector
    (p_0(x_k), ..., p_{N-1}(x_k)), p_n = H_n / sqrt(2^n n!), evaluated at the
    oracle's nodes in 50-digit arithmetic: eq. (ortvec) up to its positive
    normalisation (the sign factor (-1)^{N+k} / H_{N-1}(x_k) is positive).
    Edge columns, whose first components are far below 1e-16, pin the sign
    rule where a first-component test cannot."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    x, U = H.hermite_zero_basis(N)
    ks = sorted(set([0, 1, 2, N // 4, N // 2, N - 3, N - 2, N - 1]))
    for k in ks:
        xx = mpmath.mpf(x[k])
        p = [mpmath.mpf(1), mpmath.sqrt(2) * xx]
        for n in range(1, N - 1):
            p.append((mpmath.sqrt(2) * xx * p[-1] - mpmath.sqrt(n) * p[-2]) / mpmath.sqrt(n + 1))
        norm = mpmath.sqrt(mpmath.fsum(v * v for v in p[:N]))
        ref = np.array([float(v / norm) for v in p[:N]])
        assert np.abs(U[:, k] - ref).max() < 1e-12, k


# ---- fractional transform for complex z on the real nodes ------------------
# Sec. 2: the matrix of eq. (fasy) times the samples, eq. (primcuad), the
# Riemann sum of eq. (eqifft) at y_j = x_j (eq. (cuadtrfor)).
MEHLER_Z = [0.5, 0.5j, -0.7 + 0.3j, 0.9 * np.exp(0.3j), 0.95 * np.exp(2.5j), 0.3 * np.exp(-1.2j),
            0.0, np.exp(1.2j), -0.2 - 0.85j]


@pytest.mark.parametrize("z", MEHLER_Z)
def test_mehler_sum_hermite_eigenfunctions(z):
    """Mehler's formula makes the Hermite functions eigenfunctions of the
    integral eq. (eqifft): F_z psi_n = sqrt(2 pi) z^n psi_n.  Its Riemann sum
    on the N = 256 nodes, whose integrand is a resolved Gaussian for these z,
    reaches that to rounding.  A wrong sign of the cross term (z -> -z)
    fails every odd n, a dropped (1 + z^2) or a wrong dx or prefactor every n."""
    N = 256
    x = O.nodes(N)
    psi = H.hermite_functions(12, x)
    g = O.frft_mehler(psi, z)
    for n in range(13):
        ref = np.sqrt(2 * np.pi) * complex(z) ** n * psi[n]
        assert np.linalg.norm(g[n] - ref) < 1e-12 * np.linalg.norm(psi[n]), n


@pytest.mark.parametrize("N", [64, 100, 257])
def test_mehler_sum_parity(N):
    """The nodes are symmetric (x_{N-1-k} = -x_k) and the exponent of
    eq. (fasy) is unchanged by (x_j, z) -> (-x_j, -z): F_{-z} is F_z with
    the output reversed."""
    x = O.nodes(N)
    rng = np.random.default_rng(N)
    f = (rng.standard_normal((3, N)) + 1j * rng.standard_normal((3, N))) * np.exp(-x * x / 4)
    for z in [0.6 + 0.2j, 0.3 - 0.8j, -0.5]:
        a = O.frft_mehler(f, -z)
        b = O.frft_mehler(f, z)[:, ::-1]
        assert rel_l2(a, b).max() < 1e-15


def test_mehler_sum_converges_with_n():
    """Away from the resolved regime (|z| close to 1 at a small angle) the
    Riemann sum approaches the eigen-relation as N grows, as eq. (cuadtrfor)
    states for N -> infinity."""
    z = 0.99 * np.exp(0.1j)
    errs = []
    for N in [128, 256, 512, 1024]:
        x = O.nodes(N)
        psi = H.hermite_functions(4, x)
        g = O.frft_mehler(psi, z)
        errs.append(max(np.linalg.norm(g[n] - np.sqrt(2 * np.pi) * z ** n * psi[n]) /
                        np.linalg.norm(psi[n]) for n in range(5)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-12, errs


def test_mehler_sum_rejects_bad_z():
    x = O.nodes(8)
    for z in [1.0, -1.0, 1.1, 0.9 + 0.5j]:
        with pytest.raises(ValueError):
            O.frft_mehler(x, z)
