"""Hermite-zero discrete fractional Fourier transform (Sec. 2) and Hermite
functions.  TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``jacobi_matrix(N)``: the symmetric tridiagonal matrix H = S Hcal S^{-1} of
  Sec. 2: zero diagonal, off-diagonal entries sqrt(n/2), n = 1..N-1.
* ``hermite_zero_frft(N, z)``: nodes x_k (eigenvalues of H, the zeros of
  H_N) and the N x N matrix F_z = sqrt(2 pi) U^T D(z) U of eq. (tmat), with
  U's k-th column the normalised eigenvector u_k.  The eigenvectors come from
  a library tridiagonal eigensolver; their signs are fixed to those of
  eq. (ortvec): component n (0-based) of u_k is
  (-1)^{N+k} / H_{N-1}(x_k) times a positive factor times H_n(x_k), and
  sign((-1)^{N+k} / H_{N-1}(x_k)) = +1 because the signs of H_{N-1} at the
  ordered zeros of H_N alternate and are positive at the largest one; so
  component n has the sign of H_n(x_k).  The sign is read at the component
  of largest magnitude (the first component of an edge eigenvector is far
  below the solver's absolute accuracy: about 1e-24 at N = 64), and the sign
  of H_n(x_k) is taken from the three-term recurrence in ratio form (no
  overflow).  eq. (ortvec) itself is not evaluated literally (its factor
  2^{N-1} (N-1)! overflows FP64 near N = 170).
* ``hermite_functions(nmax, x)``: psi_n(x) = H_n(x) e^{-x^2/2} / sqrt(2^n n! sqrt(pi))
  for n = 0..nmax, real or complex x, from the three-term recurrence of
  eq. (receqg) written for the normalised functions.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal


def jacobi_matrix(N: int):
    """(diagonal, off-diagonal) of the symmetric Jacobi matrix H of Sec. 2."""
    n = np.arange(1, N, dtype=np.float64)
    return np.zeros(N), np.sqrt(n / 2.0)


def hermite_sign(n, x):
    """sign(H_n(x)) for integer arrays n >= 0 and real arrays x (same shape),
    from eq. (receqg) written for the ratios r_m = p_m / p_{m-1} of the
    normalised polynomials p_m = H_m / sqrt(2^m m!):
    p_0 = 1, r_1 = sqrt(2) x, r_{m+1} = (sqrt(2) x - sqrt(m) / r_m) / sqrt(m+1);
    sign(p_n) = product of the signs of r_1 .. r_n."""
    n = np.asarray(n)
    x = np.asarray(x, dtype=np.float64)
    sign = np.ones(x.shape)
    r = np.sqrt(2.0) * x
    with np.errstate(divide="ignore", invalid="ignore"):
        for m in range(1, int(n.max()) + 1):
            if m > 1:
                r = (np.sqrt(2.0) * x - np.sqrt(m - 1.0) / r) / np.sqrt(float(m))
            sign = np.where(m <= n, sign * np.sign(r), sign)
    return sign


def hermite_zero_basis(N: int):
    """Nodes x_k (ascending) and the orthogonal matrix U (U[n, k] = (u_k)_{n+1})
    with the signs of eq. (ortvec)."""
    d, e = jacobi_matrix(N)
    x, U = eigh_tridiagonal(d, e)
    k = np.arange(N)
    nstar = np.argmax(np.abs(U), axis=0)            # largest component of each column
    want = hermite_sign(nstar, x)
    flip = np.sign(U[nstar, k]) != want
    U[:, flip] *= -1.0
    return x, U


def hermite_zero_frft(N: int, z: complex):
    """Nodes and the matrix F_z = sqrt(2 pi) U^{-1} D(z) U of eq. (tmat)."""
    x, U = hermite_zero_basis(N)
    zn = np.power(complex(z), np.arange(N))
    F = np.sqrt(2.0 * np.pi) * (U.T * zn[None, :]) @ U
    return x, F


def hermite_functions(nmax: int, x):
    """psi_0..psi_nmax at x (array, real or complex); shape [nmax+1, len(x)].

    Recurrence: psi_{n+1} = sqrt(2/(n+1)) x psi_n - sqrt(n/(n+1)) psi_{n-1},
    which is eq. (receqg) divided through by the normalisation."""
    x = np.asarray(x)
    dt = np.complex128 if np.iscomplexobj(x) else np.float64
    out = np.empty((nmax + 1,) + x.shape, dtype=dt)
    out[0] = np.pi ** -0.25 * np.exp(-x * x / 2.0)
    if nmax >= 1:
        out[1] = np.sqrt(2.0) * x * out[0]
    for n in range(1, nmax):
        out[n + 1] = np.sqrt(2.0 / (n + 1)) * x * out[n] - np.sqrt(n / (n + 1.0)) * out[n - 1]
    return out


def hermite_polynomials(nmax: int, x):
    """Physicists' H_0..H_nmax at x by eq. (receqg): H_{n+1} = 2x H_n - 2n H_{n-1}."""
    x = np.asarray(x)
    dt = np.complex128 if np.iscomplexobj(x) else np.float64
    out = np.empty((nmax + 1,) + x.shape, dtype=dt)
    out[0] = 1.0
    if nmax >= 1:
        out[1] = 2.0 * x
    for n in range(1, nmax):
        out[n + 1] = 2.0 * x * out[n] - 2.0 * n * out[n - 1]
    return out
