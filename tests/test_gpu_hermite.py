"""GPU parity of the Hermite-zero discrete fractional transform (Sec. 2,
eq. (tmat)) against oracle B, through the C ABI.

* nodes (the zeros of H_N) and the basis U (signs of eq. (ortvec)) against
  the oracle's tridiagonal eigensolver;
* F_z f = sqrt(2 pi) U^T D(z) U f against the oracle's dense matrix, complex128
  to 1e-12 and complex64 to 1e-5 (relative L2 per signal);
* the transform's exact identities on the GPU output: unitarity up to
  sqrt(2 pi) for |z| = 1, the eigen-relation F_z v_n = sqrt(2 pi) z^n v_n, the
  group law F_{z1} F_{z2} = sqrt(2 pi) F_{z1 z2}, and the O(1/N) convergence
  to the continuous transform of Sec. 1.
"""
import numpy as np
import pytest

from oracle import closed_forms as C
from oracle import hermite as H
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402

TOL64, TOL32 = 1e-12, 1e-5


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
    lct.frft_hermite_execute(N, z, x, out, f.shape[0], code)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def signals(N, count, seed):
    x, _ = H.hermite_zero_basis(N)
    rng = np.random.default_rng(seed)
    env = np.exp(-x * x / 6.0)
    f = env * (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N)))
    f[0] = C.config0_poly(x)
    return f


@pytest.mark.parametrize("N", [2, 3, 17, 64, 256, 1024])
def test_nodes_and_basis_match_oracle(N):
    x, U = lct.frft_hermite_basis(N)
    xo, Uo = H.hermite_zero_basis(N)
    assert np.abs(x - xo).max() < 1e-12 * max(1.0, np.abs(xo).max())
    assert np.abs(U - Uo).max() < 1e-11
    assert np.abs(U.T @ U - np.eye(N)).max() < 1e-12


@pytest.mark.parametrize("N", [2, 5, 64, 256, 1024])
@pytest.mark.parametrize("z", [np.exp(-0.7j), 0.6 + 0.3j, 1.0, -1.0, 1j, 0.0])
def test_transform_matches_oracle_fp64(N, z):
    count = 35
    f = signals(N, count, seed=N)
    _, F = H.hermite_zero_frft(N, z)
    ref = f @ F.T
    got = apply(N, z, f)
    assert rel_l2(got, ref).max() < TOL64


@pytest.mark.parametrize("N", [64, 128, 300, 1024, 2048])
@pytest.mark.parametrize("z", [np.exp(-0.7j), 0.8 * np.exp(2.1j)])
def test_transform_matches_oracle_fp32(N, z):
    """complex64: CUDA cores below N = 128, else the tensor cores (split
    TF32, 64-signal x 256-column tiles: 70 signals and N = 300 leave partial
    tiles in both directions)."""
    f = signals(N, 70, seed=N + 1)
    _, F = H.hermite_zero_frft(N, z)
    ref = f.astype(np.complex64).astype(np.complex128) @ F.T
    got = apply(N, z, f, np.complex64)
    assert lct.frft_hermite_status() == 0
    assert rel_l2(got, ref).max() < TOL32


def test_in_place_and_batch_tail():
    N, z = 100, np.exp(0.4j)
    f = signals(N, 33, seed=3)          # one more than a 32-signal tile
    a = apply(N, z, f)
    b = apply(N, z, f, inplace=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("N", [64, 512])
def test_unitarity_on_the_gpu(N):
    """F_z^H F_z = 2 pi I for |z| = 1: the transform of the identity's rows."""
    z = np.exp(-1.1j)
    Ft = apply(N, z, np.eye(N, dtype=np.complex128))      # row k = F e_k = column k of F
    F = Ft.T
    assert np.abs(F.conj().T @ F - 2 * np.pi * np.eye(N)).max() < 1e-11


def test_eigenvectors_and_group_law_on_the_gpu():
    N = 256
    _, U = lct.frft_hermite_basis(N)
    z = 0.9 * np.exp(0.8j)
    rows = U[[0, 1, 5, 40, 200], :].astype(np.complex128)        # v_n = row n of U
    got = apply(N, z, rows)
    for r, n in enumerate([0, 1, 5, 40, 200]):
        assert np.abs(got[r] - np.sqrt(2 * np.pi) * z ** n * rows[r]).max() < 1e-12
    z1, z2 = 0.7 * np.exp(0.3j), np.exp(-1.2j)
    f = signals(N, 8, seed=9)
    lhs = apply(N, z1, apply(N, z2, f))
    rhs = np.sqrt(2 * np.pi) * apply(N, z1 * z2, f)
    assert rel_l2(lhs, rhs).max() < 1e-12


def test_convergence_to_the_continuous_transform():
    """Sec. 1: O(1/N) against the continuous F_z of the config-0 polynomial."""
    z = np.exp(-0.7j)
    scaled = []
    for N in [32, 64, 128, 256]:
        x, _ = lct.frft_hermite_basis(N, with_matrix=False)
        f = C.config0_poly(x)[None, :].astype(np.complex128)
        got = apply(N, z, f)[0]
        scaled.append(rel_l2(got, C.config0_poly_frft(z, x)) * N)
    scaled = np.array(scaled)
    assert scaled.max() / scaled.min() < 1.1


def test_bad_arguments():
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    for N, z, code in [(1, 0.5, lct.LCT_C128), (4097, 0.5, lct.LCT_C128)]:
        with pytest.raises(lct.LctError) as e:
            lct.frft_hermite_execute(N, z, x, x, 1, code)
        assert e.value.status == 2
    with pytest.raises(lct.LctError) as e:
        lct.frft_hermite_execute(8, 1.5, x, x, 1, lct.LCT_C128)
    assert e.value.status == 1
