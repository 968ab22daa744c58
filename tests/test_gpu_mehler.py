"""GPU parity of the fractional transform for complex z on the real nodes
(Sec. 2, eqs. (fasy), (primcuad), (cuadtrfor)) against the oracle's dense
Riemann sum, through the C ABI (frft_mehler_execute).

* element by element against oracle.frft_mehler: complex128 to 1e-12 and
  complex64 to 1e-5 (relative L2 per signal), for powers of two and other N
  from 2 to the largest size, z inside the unit disc in every quadrant
  (Re z < 0 runs the reversed form), on the unit circle, 0 and purely
  imaginary, batches that leave the last CTA partly empty, in place;
* at the largest sizes, on sampled signals, and through the eigen-relation
  F_z psi_n = sqrt(2 pi) z^n psi_n of Mehler's formula, which holds at any N.
"""
import numpy as np
import pytest

import oracle as O
from oracle import closed_forms as C
from oracle import hermite as H
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402

TOL64, TOL32 = 1e-12, 1e-5
ZS = [0.5, 0.5j, -0.7 + 0.3j, 0.9 * np.exp(0.3j), 0.95 * np.exp(2.5j), 0.3 * np.exp(-1.2j), 0.0,
      np.exp(1.2j), -0.2 - 0.85j, np.exp(-2.0j)]


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    torch.cuda.set_device(0)


def apply(N, z, f, dtype=np.complex128, inplace=False):
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    x = torch.from_numpy(np.ascontiguousarray(f.astype(dtype))).cuda()
    out = x if inplace else torch.empty_like(x)
    lct.frft_mehler_execute(N, z, x, out, f.shape[0], code)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def signals(N, count, seed):
    x = O.nodes(N)
    rng = np.random.default_rng(seed)
    env = np.exp(-x * x / 8.0)
    f = env * (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N)))
    f[0] = C.config0_poly(x)
    return f


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("N", [2, 3, 5, 16, 64, 100, 256, 1000, 1024])
def test_matches_oracle_small(N, dtype):
    count = 37 if N <= 256 else 9
    f = signals(N, count, seed=N).astype(dtype)
    tol = TOL32 if dtype == np.complex64 else TOL64
    for z in ZS:
        ref = O.frft_mehler(f.astype(np.complex128), z)
        g = apply(N, z, f, dtype)
        assert rel_l2(g, ref).max() < tol, (N, z)


@pytest.mark.parametrize("dtype,N", [(np.complex64, 2048), (np.complex64, 3000), (np.complex64, 4096),
                                     (np.complex128, 2048), (np.complex128, 2500),
                                     (np.complex128, 4096)])
def test_matches_oracle_large(N, dtype):
    f = signals(N, 3, seed=N + 7).astype(dtype)
    tol = TOL32 if dtype == np.complex64 else TOL64
    for z in [0.6 + 0.5j, -0.3 - 0.9j, np.exp(1.0j)]:
        ref = O.frft_mehler(f.astype(np.complex128), z)
        assert rel_l2(apply(N, z, f, dtype), ref).max() < tol, (N, z)


def test_largest_complex64_sampled():
    """N = 8192 (M = 16384): a sampled batch of 5 of 300 signals against the oracle."""
    N = 8192
    f = signals(N, 300, seed=81).astype(np.complex64)
    z = -0.55 + 0.62j
    g = apply(N, z, f, np.complex64)
    rows = [0, 1, 150, 298, 299]
    ref = O.frft_mehler(f[rows].astype(np.complex128), z)
    assert rel_l2(g[rows], ref).max() < TOL32


@pytest.mark.parametrize("dtype,N", [(np.complex64, 8192), (np.complex128, 4096), (np.complex64, 6000)])
def test_eigen_relation_at_the_largest_sizes(N, dtype):
    """F_z psi_n = sqrt(2 pi) z^n psi_n (Mehler's formula), which the Riemann
    sum reaches to rounding at these N for resolved z."""
    x = O.nodes(N)
    psi = H.hermite_functions(10, x)
    tol = 1e-5 if dtype == np.complex64 else 1e-12
    for z in [0.7 * np.exp(2.0j), 0.4 + 0.8j, np.exp(0.9j)]:
        g = apply(N, z, psi.astype(np.complex128), dtype)
        for n in range(11):
            ref = np.sqrt(2 * np.pi) * complex(z) ** n * psi[n]
            assert np.linalg.norm(g[n] - ref) < tol * np.linalg.norm(psi[n]), (N, z, n)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_in_place_and_batch_one(dtype):
    N = 512
    f = signals(N, 5, seed=3).astype(dtype)
    tol = TOL32 if dtype == np.complex64 else TOL64
    z = -0.4 + 0.4j
    ref = O.frft_mehler(f.astype(np.complex128), z)
    assert rel_l2(apply(N, z, f, dtype, inplace=True), ref).max() < tol
    assert rel_l2(apply(N, z, f[:1], dtype), ref[:1]).max() < tol


def test_group_law_through_the_gpu():
    """F_{z1} F_{z2} = sqrt(2 pi) F_{z1 z2} holds for the continuous transform;
    the Riemann sums reproduce it for resolved z (complex128, N = 1024)."""
    N = 1024
    f = signals(N, 4, seed=5)
    z1, z2 = 0.8 * np.exp(0.7j), 0.7 * np.exp(-1.9j)
    lhs = apply(N, z1, apply(N, z2, f))
    rhs = np.sqrt(2 * np.pi) * apply(N, z1 * z2, f)
    assert rel_l2(lhs, rhs).max() < 1e-10
