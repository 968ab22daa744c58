"""Hermite-zero discrete fractional Fourier transform (Sec. 2) and Hermite
functions.  TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``jacobi_matrix(N)``: the symmetric tridiagonal matrix H = S Hcal S^{-1} of
  Sec. 2: zero diagonal, off-diagonal entries sqrt(n/2), n = 1..N-1.
* ``hermite_zero_frft(N, z)``: nodes x_k (eigenvalues of H, the zeros of
  H_N) and the N x N matrix F_z = sqrt(2 pi) U^T D(z) U of eq. (tmat), with
  U's k-th column the normalised eigenvector u_k.  The eigenvectors come from
  a library tridiagonal eigensolver; their signs are fixed so that the first
  component is positive, which is the sign of eq. (ortvec):
  (u_k)_1 = c_k with sign((-1)^{N+k} / H_{N-1}(x_k)) = +1 because the signs
  of H_{N-1} at the ordered zeros of H_N alternate and are positive at the
  largest one.  eq. (ortvec) itself is not evaluated literally (its factor
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


def hermite_zero_basis(N: int):
    """Nodes x_k (ascending) and the orthogonal matrix U (U[n, k] = (u_k)_{n+1})."""
    d, e = jacobi_matrix(N)
    x, U = eigh_tridiagonal(d, e)
    sign = np.sign(U[0, :])
    sign[sign == 0] = 1.0
    return x, U * sign[None, :]


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
