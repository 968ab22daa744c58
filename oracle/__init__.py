"""CPU oracle for the discrete linear canonical transform (XFT).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never imports it and shares no code with it.

Contents
--------
* ``xft_oracle.c`` (built here into ``liboracle.so``): the XFT of Sec. 3 --
  the Riemann sum of eq. (lctdos) on the asymptotic Hermite nodes of
  eq. (asymcer), output points y_j = 4 b x_j / pi -- by direct O(N^2)
  summation in FP64 with phases reduced in extended precision.  Also the
  b = 0 branch of eq. (lctuno), the adjoint, and the dense-matrix parameter
  gradient.
* ``hermite.py``: the Hermite-zero discrete fractional Fourier transform of
  Sec. 2, eq. (tmat), and Hermite functions.
* ``closed_forms.py``: closed forms the oracle is pinned to (the Gaussian of
  Sec. 4, Hermite eigenfunctions, the continuous transforms).

Every function takes and returns complex128 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/liboracle.so."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-Wall", "-Wextra", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
            lib.oracle_nodes.argtypes = [i64, dp]
            lib.oracle_nodes.restype = None
            lib.oracle_lct.argtypes = [i64, i64, dp, i64, dp, dp, dp]
            lib.oracle_lct.restype = ctypes.c_int
            lib.oracle_lct_adjoint.argtypes = [i64, i64, dp, i64, dp, dp]
            lib.oracle_lct_adjoint.restype = ctypes.c_int
            lib.oracle_lct_grad_params.argtypes = [i64, i64, dp, i64, dp, dp, dp]
            lib.oracle_lct_grad_params.restype = ctypes.c_int
            lib.oracle_lct_matrix.argtypes = [i64, dp, dp]
            lib.oracle_lct_matrix.restype = ctypes.c_int
            lib.oracle_frft_mehler.argtypes = [i64, i64, ctypes.c_double, ctypes.c_double, dp, dp]
            lib.oracle_frft_mehler.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(abcd, count: int):
    """abcd: 4 numbers (shared) or an array [count, 4] (per signal), real or
    complex.  Returns (array [k, 8] float64, stride in doubles)."""
    p = np.asarray(abcd, dtype=np.complex128)
    if p.ndim == 1:
        if p.shape[0] != 4:
            raise ValueError("abcd must hold 4 values (a, b, c, d)")
        return np.ascontiguousarray(p.view(np.float64).reshape(1, 8)), 0
    if p.shape != (count, 4):
        raise ValueError("per-signal abcd must have shape (count, 4)")
    return np.ascontiguousarray(p.view(np.float64).reshape(count, 8)), 8


def _signals(f, N=None):
    f = np.ascontiguousarray(np.asarray(f, dtype=np.complex128))
    if f.ndim == 1:
        f = f.reshape(1, -1)
    if N is not None and f.shape[-1] != N:
        raise ValueError("signal length mismatch")
    return f


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


def nodes(N: int) -> np.ndarray:
    """Asymptotic Hermite zeros x_k, eq. (asymcer), 0-based (k = 0..N-1)."""
    x = np.empty(N, dtype=np.float64)
    _load().oracle_nodes(N, _dp(x))
    return x


def output_grid(N: int, abcd) -> np.ndarray:
    """Output points of the transform: y_j = 4 b x_j / pi (Algorithm, b != 0),
    y_j = x_j / d for b == 0 (the reading that makes f(d y_j) a sample)."""
    a, b, c, d = np.asarray(abcd, dtype=np.complex128)
    x = nodes(N).astype(np.complex128)
    if b == 0:
        return x / d
    return 4.0 * b * x / np.pi


def lct(f, abcd, return_rho: bool = False):
    """XFT of each row of f (shape [count, N] or [N]).

    Returns Ghat = G e^{-rho} (equal to G for real parameters) with the same
    shape as f; with return_rho also rho (real, same shape)."""
    f_in = np.asarray(f)
    fs = _signals(f)
    count, N = fs.shape
    p, stride = _params(abcd, count)
    G = np.empty_like(fs)
    rho = np.empty((count, N), dtype=np.float64)
    rc = _load().oracle_lct(N, count, _dp(p), stride, _dp(fs.view(np.float64)),
                            _dp(G.view(np.float64)), _dp(rho))
    if rc != 0:
        raise RuntimeError("oracle_lct failed (%d)" % rc)
    G = G.reshape(f_in.shape)
    rho = rho.reshape(f_in.shape)
    return (G, rho) if return_rho else G


def lct_adjoint(g, abcd):
    """h = Lhat^H g for each row of g."""
    g_in = np.asarray(g)
    gs = _signals(g)
    count, N = gs.shape
    p, stride = _params(abcd, count)
    h = np.empty_like(gs)
    rc = _load().oracle_lct_adjoint(N, count, _dp(p), stride, _dp(gs.view(np.float64)),
                                    _dp(h.view(np.float64)))
    if rc != 0:
        raise RuntimeError("oracle_lct_adjoint failed (%d)" % rc)
    return h.reshape(g_in.shape)


def lct_grad_params(f, g, abcd) -> np.ndarray:
    """Dense-matrix gradient (dl/da, dl/db, dl/dd) per signal for real
    parameters with b != 0, given the cotangent g = dl/dRe G + i dl/dIm G.
    Returns shape [count, 3]."""
    fs = _signals(f)
    gs = _signals(g)
    count, N = fs.shape
    if gs.shape != fs.shape:
        raise ValueError("f and g must have the same shape")
    p, stride = _params(abcd, count)
    out = np.empty((count, 3), dtype=np.float64)
    rc = _load().oracle_lct_grad_params(N, count, _dp(p), stride, _dp(fs.view(np.float64)),
                                        _dp(gs.view(np.float64)), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle_lct_grad_params failed (%d)" % rc)
    return out


def lct_matrix(N: int, abcd) -> np.ndarray:
    """The dense matrix Lhat (N x N) of one parameter set."""
    p, _ = _params(abcd, 1)
    L = np.empty((N, N), dtype=np.complex128)
    rc = _load().oracle_lct_matrix(N, _dp(p), _dp(L.view(np.float64)))
    if rc != 0:
        raise RuntimeError("oracle_lct_matrix failed (%d)" % rc)
    return L


def abcd_of_z(z: complex):
    """LCT parameters of the fractional transform F_z of eq. (eqifft):
    matching its exponent with the LCT kernel of eq. (lctuno) gives
    a = d = (z + 1/z)/2, b = (1/z - z)/(2i), c = i (1/z - z)/2."""
    z = complex(z)
    a = (z + 1.0 / z) / 2.0
    b = (1.0 / z - z) / 2j
    c = 1j * (1.0 / z - z) / 2.0
    return np.array([a, b, c, a], dtype=np.complex128)


def frft_scale(z: complex) -> complex:
    """Scalar s(z) with F_z = s(z) * LCT(a(z), b(z), c(z), d(z)):
    sqrt(2/(1 - z^2)) * sqrt(2 pi i b(z)), both principal roots."""
    z = complex(z)
    b = abcd_of_z(z)[1]
    return complex(np.sqrt(2.0 / (1.0 - z * z)) * np.sqrt(2j * np.pi * b))


def frft(f, z: complex, return_rho: bool = False):
    """Discrete F_z (normalisation of eq. (eqifft)) through the XFT, at the
    output points y_j = 4 b(z) x_j / pi."""
    res = lct(f, abcd_of_z(z), return_rho=True)
    s = frft_scale(z)
    if return_rho:
        return res[0] * s, res[1]
    return res[0] * s


def frft_mehler(f, z: complex) -> np.ndarray:
    """F_z for complex z (|z| <= 1, z != +-1) on the real nodes y_j = x_j:
    the matrix of eq. (fasy) times the samples, eq. (primcuad) -- the Riemann
    sum of eq. (eqifft) that eq. (cuadtrfor) states.  Rows of f are signals."""
    f_in = np.asarray(f)
    fs = _signals(f)
    count, N = fs.shape
    z = complex(z)
    g = np.empty_like(fs)
    rc = _load().oracle_frft_mehler(N, count, z.real, z.imag, _dp(fs.view(np.float64)),
                                    _dp(g.view(np.float64)))
    if rc != 0:
        raise ValueError("oracle_frft_mehler: |z| <= 1 and z != +-1 required")
    return g.reshape(f_in.shape)
