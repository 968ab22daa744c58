"""Seeded input generators: determinism, ranges and the symplectic constraint."""
import numpy as np

import workloads as W


def test_g1_params_symplectic_and_ranges():
    p = W.g1_params(W.rng_for(1), 5000)
    a, b, c, d = p.T
    assert np.abs(a * d - b * c - 1).max() < 1e-12
    assert (np.abs(a) <= 2).all() and (np.abs(d) <= 2).all()
    assert (np.abs(b) >= 0.2).all() and (np.abs(b) <= 2).all()
    assert 0.4 < (b > 0).mean() < 0.6


def test_uniform_batch_deterministic_and_blockwise():
    x = np.linspace(-3, 3, 64)
    p1, f1 = W.uniform_batch(x, 600, seed=7, dtype=np.complex128)
    p2, f2 = W.uniform_batch(x, 600, seed=7, dtype=np.complex128)
    assert np.array_equal(p1, p2) and np.array_equal(f1, f2)
    # a signal's envelope is the Gaussian window plus 1e-3 noise
    rng = W.rng_for(7)
    W.g1_params(rng, 600)
    s, q = W.g1_shapes(rng, 600)
    env = np.exp(-x * x / (2 * s[5] ** 2))
    assert np.abs(np.abs(f1[5]) - env).max() < 1e-2


def test_config0_signals_are_hermite_functions():
    from scipy.special import eval_hermite
    from math import factorial
    x = np.linspace(-4, 4, 33)
    rows = W.config0_signals(x)
    assert rows.shape == (12, 33)
    for n in range(11):
        ref = eval_hermite(n, x) * np.exp(-x * x / 2) / np.sqrt(2.0 ** n * factorial(n) * np.sqrt(np.pi))
        assert np.abs(rows[n + 1] - ref).max() < 1e-12


def test_ragged_plan_counts_and_kinds():
    r = W.ragged_plan(count_scale=0.01)
    kinds = r["kind"]
    assert len(kinds) == 90 + 50 + 40 + 20
    assert set(np.unique(kinds)) == {0, 1, 2, 3}
    assert (r["log2n"] >= 6).all() and (r["log2n"] <= 16).all()
    b0 = kinds == W.KIND_B0
    assert np.all(r["abcd"][b0, 1] == 0)
    fr = kinds == W.KIND_FRFT
    zz = np.abs(r["z"][fr])
    assert (zz >= 0.3).all() and (zz <= 0.95).all()


def test_keys_upsampling_reproduces_linear_functions():
    """The Keys cubic (a = -0.5) reproduces polynomials up to degree 2 away
    from the edges; rows sum to one everywhere."""
    Wm = W.keys_upsample_matrix(256, 64)
    assert np.allclose(Wm.sum(axis=1), 1.0, atol=1e-12)
    src = np.arange(64, dtype=np.float64)
    u = (np.arange(256) + 0.5) * 64 / 256 - 0.5
    inner = (u > 2) & (u < 60)
    assert np.allclose((Wm @ src)[inner], u[inner], atol=1e-12)


def test_fields_batch_shape_and_envelope():
    x = np.linspace(-10, 10, 128)
    f, ax, ay = W.fields_batch(x, count=2)
    assert f.shape == (2, 128, 128)
    env = np.exp(-(x[:, None] ** 2 + x[None, :] ** 2) / 72.0)
    assert np.allclose(np.abs(f[0]), env)
    for p in (ax, ay):
        assert abs(p[0] * p[3] - p[1] * p[2] - 1) < 1e-12
