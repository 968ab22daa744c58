"""Seeded synthetic inputs for the LCT workloads.

This module draws parameters and samples only; it holds none of the
transform's arithmetic.  Sample positions are passed in by the caller (the
tests take them from the oracle, the benchmark from the library's own input
grid query), so that the same generator serves both sides of every parity
check.

Workloads (shapes and distributions follow the paper's use cases: Gaussian
windows and chirps on the Hermite-node grid):

* ``config0``  one complex128 signal, N = 256, rotation angle 0.7:
  f(x) = exp(-x^2/2) (1 + 0.3 x + 0.1 x^3), plus the Hermite functions
  psi_0..psi_10 for the eigenvalue check (batch of 12).
* ``uniform``  generator G1, per signal
     a, d ~ U[-2, 2],  |b| ~ U[0.2, 2] with a fair random sign,  c = (a d - 1)/b,
     f(x) = exp(-x^2 / (2 s^2)) exp(i q x^2) + 1e-3 (n_r + i n_i)/sqrt(2),
     s ~ U[0.5, 3],  q ~ U[-1, 1],  n_r, n_i ~ N(0, 1).
  4096 x N=1024 (seed 1001) and 16384 x N=4096 (seed 1002, the throughput
  workload).
* ``ragged``   20000 instances, log2 N ~ U{6..16}; 9000 generic (G1), 5000
  fractional with complex z (|z| ~ U[0.3, 0.95], arg z ~ U[0, 2 pi)), 4000
  ordinary Fourier (a, b, c, d) = (0, 1, -1, 0), 2000 with b = 0
  (d ~ U[0.5, 2], a = 1/d, c ~ U[-2, 2]); kinds shuffled; inputs from G1.

Draw order (part of the definition, so that a subsample can be regenerated):
parameters for the whole batch first, then the signal noise in blocks of
NOISE_BLOCK signals, each block one ``standard_normal((blk, N, 2))`` call.
"""
from __future__ import annotations

import numpy as np

NOISE_BLOCK = 256

SEED_CONFIG0 = 1000
SEED_UNIFORM_1024 = 1001
SEED_UNIFORM_4096 = 1002
SEED_RAGGED = 1003
SEED_FIELDS = 1004

KIND_GENERIC, KIND_FRFT, KIND_FOURIER, KIND_B0 = 0, 1, 2, 3


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# config 0: the polynomial and the Hermite functions
# ----------------------------------------------------------------------------
def config0_signals(x: np.ndarray, n_hermite: int = 11) -> np.ndarray:
    """Rows: f(x) = exp(-x^2/2)(1 + 0.3x + 0.1x^3), then psi_0..psi_{n_hermite-1}
    (normalised Hermite functions, by their standard three-term recurrence)."""
    x = np.asarray(x, dtype=np.float64)
    rows = [np.exp(-x * x / 2.0) * (1.0 + 0.3 * x + 0.1 * x ** 3)]
    p_prev = np.zeros_like(x)
    p = np.pi ** -0.25 * np.exp(-x * x / 2.0)
    for n in range(n_hermite):
        rows.append(p.copy())
        p_next = np.sqrt(2.0 / (n + 1)) * x * p - np.sqrt(n / (n + 1.0)) * p_prev
        p_prev, p = p, p_next
    return np.asarray(rows, dtype=np.complex128)


CONFIG0_ANGLE = 0.7


def config0_params():
    t = CONFIG0_ANGLE
    return np.array([np.cos(t), np.sin(t), -np.sin(t), np.cos(t)], dtype=np.float64)


# ----------------------------------------------------------------------------
# G1: per-signal parameters and Gaussian-windowed random chirps
# ----------------------------------------------------------------------------
def g1_params(rng: np.random.Generator, count: int) -> np.ndarray:
    """[count, 4] real (a, b, c, d) with ad - bc = 1."""
    a = rng.uniform(-2.0, 2.0, count)
    d = rng.uniform(-2.0, 2.0, count)
    bmag = rng.uniform(0.2, 2.0, count)
    bsign = rng.integers(0, 2, count)
    b = np.where(bsign == 1, bmag, -bmag)
    c = (a * d - 1.0) / b
    return np.stack([a, b, c, d], axis=1)


def g1_shapes(rng: np.random.Generator, count: int):
    s = rng.uniform(0.5, 3.0, count)
    q = rng.uniform(-1.0, 1.0, count)
    return s, q


def g1_fill(rng: np.random.Generator, x: np.ndarray, s: np.ndarray, q: np.ndarray,
            out: np.ndarray) -> np.ndarray:
    """Write G1 signals for the rows of `out` ([count, N], complex64/128)."""
    x = np.asarray(x, dtype=np.float64)
    count, N = out.shape
    x2 = x * x
    for i0 in range(0, count, NOISE_BLOCK):
        i1 = min(count, i0 + NOISE_BLOCK)
        noise = rng.standard_normal((i1 - i0, N, 2))
        ss = s[i0:i1, None]
        qq = q[i0:i1, None]
        env = np.exp(-x2[None, :] / (2.0 * ss * ss))
        ph = qq * x2[None, :]
        re = env * np.cos(ph) + 1e-3 * noise[..., 0] / np.sqrt(2.0)
        im = env * np.sin(ph) + 1e-3 * noise[..., 1] / np.sqrt(2.0)
        out[i0:i1].real = re
        out[i0:i1].imag = im
    return out


def uniform_batch(x: np.ndarray, count: int, seed: int, dtype=np.complex64,
                  out: np.ndarray | None = None):
    """G1 batch on a common grid x (length N). Returns (params [count,4], f [count,N])."""
    rng = rng_for(seed)
    params = g1_params(rng, count)
    s, q = g1_shapes(rng, count)
    if out is None:
        out = np.empty((count, len(x)), dtype=dtype)
    g1_fill(rng, x, s, q, out)
    return params, out


# ----------------------------------------------------------------------------
# ragged mixed batch
# ----------------------------------------------------------------------------
RAGGED_COUNTS = {KIND_GENERIC: 9000, KIND_FRFT: 5000, KIND_FOURIER: 4000, KIND_B0: 2000}


def ragged_plan(count_scale: float = 1.0, seed: int = SEED_RAGGED, log2n_min: int = 6,
                log2n_max: int = 16):
    """Kinds, sizes and parameters of the ragged batch.

    Returns dict with 'kind' [M], 'log2n' [M], 'abcd' [M, 4] complex,
    'z' [M] complex (nan where not fractional), 's', 'q' (G1 shapes).
    count_scale shrinks the batch (counts are rounded, at least 1 each)."""
    rng = rng_for(seed)
    kinds = np.concatenate([np.full(max(1, int(round(n * count_scale))), k)
                            for k, n in RAGGED_COUNTS.items()])
    rng.shuffle(kinds)
    M = len(kinds)
    log2n = rng.integers(log2n_min, log2n_max + 1, M)
    abcd = np.zeros((M, 4), dtype=np.complex128)
    z = np.full(M, np.nan + 0j)
    g = g1_params(rng, M)
    zmag = rng.uniform(0.3, 0.95, M)
    zarg = rng.uniform(0.0, 2.0 * np.pi, M)
    d0 = rng.uniform(0.5, 2.0, M)
    c0 = rng.uniform(-2.0, 2.0, M)
    for i in range(M):
        k = kinds[i]
        if k == KIND_GENERIC:
            abcd[i] = g[i]
        elif k == KIND_FRFT:
            z[i] = zmag[i] * np.exp(1j * zarg[i])
        elif k == KIND_FOURIER:
            abcd[i] = (0.0, 1.0, -1.0, 0.0)
        else:
            abcd[i] = (1.0 / d0[i], 0.0, c0[i], d0[i])
    s, q = g1_shapes(rng, M)
    return {"kind": kinds, "log2n": log2n, "abcd": abcd, "z": z, "s": s, "q": q,
            "rng": rng}


def ragged_signal(x: np.ndarray, s: float, q: float, rng: np.random.Generator,
                  dtype=np.complex64) -> np.ndarray:
    """One G1 signal on grid x (the noise drawn from rng)."""
    out = np.empty((1, len(x)), dtype=dtype)
    return g1_fill(rng, x, np.array([s]), np.array([q]), out)[0]


# ----------------------------------------------------------------------------
# 2-D fields: Gaussian beam times a smooth random phase screen
# ----------------------------------------------------------------------------
def keys_upsample_matrix(n_out: int, n_in: int, a: float = -0.5) -> np.ndarray:
    """[n_out, n_in] bicubic (Keys kernel, parameter a) interpolation matrix,
    half-pixel centres (align_corners=False), edge samples replicated."""
    def kern(t):
        t = np.abs(t)
        return np.where(t <= 1, (a + 2) * t ** 3 - (a + 3) * t ** 2 + 1,
                        np.where(t < 2, a * t ** 3 - 5 * a * t ** 2 + 8 * a * t - 4 * a, 0.0))
    Wm = np.zeros((n_out, n_in))
    for i in range(n_out):
        u = (i + 0.5) * n_in / n_out - 0.5
        j0 = int(np.floor(u))
        for j in range(j0 - 1, j0 + 3):
            Wm[i, min(max(j, 0), n_in - 1)] += kern(u - j)
    return Wm


def fields_batch(x: np.ndarray, count: int = 8, seed: int = SEED_FIELDS, width: float = 6.0,
                 screen: int = 64):
    """count complex128 fields on the grid x (x) x: exp(-(x^2+y^2)/(2 w^2)) e^{i phi},
    phi = bicubic upsampling of a screen x screen N(0,1) array; per-axis (a,b,c,d)
    from G1.  Returns (fields [count, n, n], abcd_x, abcd_y)."""
    rng = rng_for(seed)
    p = g1_params(rng, 2)
    abcd_x, abcd_y = p[0], p[1]
    n = len(x)
    Wm = keys_upsample_matrix(n, screen)
    env = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / (2 * width * width))
    out = np.empty((count, n, n), dtype=np.complex128)
    for k in range(count):
        phi = Wm @ rng.standard_normal((screen, screen)) @ Wm.T
        out[k] = env * np.exp(1j * phi)
    return out, abcd_x, abcd_y
