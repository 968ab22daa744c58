"""Closed forms the oracle is pinned to.  TEST INFRASTRUCTURE ONLY.

* ``gaussian_lct``: the LCT of f(x) = exp(-(alpha x^2 + 2 beta x + gamma)),
  from the Gaussian integral  int exp(-A x^2 + B x) dx = sqrt(pi/A) exp(B^2/(4A))
  (Re A > 0) applied to eq. (lctuno):
      A = alpha - i a/(2b),   B = -2 beta - i y / b,
      G(y) = (2 pi i b)^{-1/2} sqrt(pi/A) exp(B^2/(4A) - gamma + i d y^2/(2b)).
* ``paper_gaussian_lct``: the same transform as printed in Sec. 4, eq. (exa1),
  restated term by term (the paper writes f in the variable y; it means x).
* ``hermite_lct``: LCT of a Hermite function under the rotation
  (a, b, c, d) = (cos t, sin t, -sin t, cos t), 0 < t < pi:
  e^{-i (n + 1/2) t} psi_n(y)  (Hermite functions are the eigenfunctions of
  the fractional Fourier transform; the extra e^{-i t/2} comes from the
  principal root sqrt(2 pi i sin t)).
* ``hermite_frft``: F_z psi_n = sqrt(2 pi) z^n psi_n, the Mehler expansion of
  the kernel of eq. (eqifft), valid for |z| < 1 and, as a limit, |z| = 1.
* ``config0_poly``: exp(-x^2/2) (1 + 0.3 x + 0.1 x^3)
  = exp(-x^2/2) (H_0 + 0.225 H_1 + 0.0125 H_3), so its rotation LCT is a sum
  of three Hermite eigenfunctions.
"""
from __future__ import annotations

import numpy as np

from .hermite import hermite_functions


def gaussian_lct(y, alpha, beta, gamma, a, b, d):
    y = np.asarray(y, dtype=np.complex128)
    A = alpha - 1j * a / (2.0 * b)
    B = -2.0 * beta - 1j * y / b
    pref = 1.0 / np.sqrt(2j * np.pi * b) * np.sqrt(np.pi / A)
    return pref * np.exp(B * B / (4.0 * A) - gamma + 1j * d * y * y / (2.0 * b))


def paper_gaussian_lct(y, alpha, beta, gamma, a, b, c, d):
    """Sec. 4, eq. (exa1), for real parameters with alpha > 0."""
    y = np.asarray(y, dtype=np.float64)
    q = alpha * alpha + a * a / (4.0 * b * b)
    den = 4.0 * b * b * alpha * alpha + a * a
    t1 = np.sqrt(np.pi) / (np.sqrt(2j * np.pi * b) * q ** 0.25)
    t2 = np.exp(alpha * (beta * beta - alpha * gamma) / q)
    t3 = np.exp(0.5j * np.arctan(a / (2.0 * alpha * b)))
    t4 = np.exp(-(alpha * y * y + 2.0 * beta * a * y + a * a * gamma) / den)
    t5 = np.exp(1j * a * c * y * y / (2.0 * den))
    t6 = np.exp(1j * 2.0 * b * (alpha * alpha * d * y * y + 2.0 * beta * alpha * y + beta * beta * a) / den)
    return t1 * t2 * t3 * t4 * t5 * t6


def gaussian(x, alpha, beta, gamma):
    x = np.asarray(x)
    return np.exp(-(alpha * x * x + 2.0 * beta * x + gamma))


def hermite_lct(n, t, y):
    psi = hermite_functions(n, np.asarray(y))[n]
    return np.exp(-1j * (n + 0.5) * t) * psi


def hermite_frft(n, z, y):
    psi = hermite_functions(n, np.asarray(y))[n]
    return np.sqrt(2.0 * np.pi) * complex(z) ** n * psi


CONFIG0_HERMITE = {0: 1.0, 1: 0.225, 3: 0.0125}


def config0_poly(x):
    x = np.asarray(x)
    return np.exp(-x * x / 2.0) * (1.0 + 0.3 * x + 0.1 * x ** 3)


def config0_poly_lct(t, y):
    """Rotation LCT (angle t) of config0_poly, via its Hermite expansion.
    psi_n = H_n e^{-x^2/2} / sqrt(2^n n! sqrt(pi)) so H_n e^{-x^2/2} = norm_n psi_n."""
    out = np.zeros(np.shape(y), dtype=np.complex128)
    for n, cn in CONFIG0_HERMITE.items():
        norm = np.sqrt(2.0 ** n * np.prod(np.arange(1, n + 1, dtype=np.float64)) * np.sqrt(np.pi))
        out += cn * norm * hermite_lct(n, t, y)
    return out


def config0_poly_frft(z, y):
    """F_z of config0_poly (same expansion, eigenvalues sqrt(2 pi) z^n)."""
    out = np.zeros(np.shape(y), dtype=np.complex128)
    for n, cn in CONFIG0_HERMITE.items():
        norm = np.sqrt(2.0 ** n * np.prod(np.arange(1, n + 1, dtype=np.float64)) * np.sqrt(np.pi))
        out += cn * norm * hermite_frft(n, z, y)
    return out
