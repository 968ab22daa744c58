"""GPU side of the sharded 2-D transform: the transpose kernel against numpy,
and lct2d_sharded on one GPU (world size 1: rows, transposes, columns, no
exchange) against the oracle's separable 2-D transform.  The exchange between
ranks is tested on CPU ranks (tests/test_multirank.py)."""
import numpy as np
import pytest

import oracle as O
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("rows,cols,vec,batch", [(100, 77, 1, 3), (32, 64, 1, 1), (3, 7, 5, 2),
                                                 (2, 128, 64, 1), (1, 1, 1, 1)])
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_transpose_kernel(rows, cols, vec, batch, dtype):
    rng = np.random.default_rng(rows * cols + vec)
    a = (rng.standard_normal((batch, rows, cols, vec)) + 1j * rng.standard_normal((batch, rows, cols, vec))).astype(dtype)
    x = torch.from_numpy(a).cuda()
    out = torch.empty_like(x)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    lct.lct_transpose(x, out, rows, cols, vec, batch, code)
    torch.cuda.synchronize()
    want = np.ascontiguousarray(a.transpose(0, 2, 1, 3))
    assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)


@pytest.mark.parametrize("dtype,tol", [(np.complex128, 1e-12), (np.complex64, 1e-5)])
def test_sharded_2d_on_one_gpu(dtype, tol):
    ny, nx = 128, 256
    rng = np.random.default_rng(3)
    y, x = O.nodes(ny), O.nodes(nx)
    f = np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / 18.0) * (
        rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx)))
    ax = (0.6, 1.3, (0.6 * -0.4 - 1) / 1.3, -0.4)
    ay = (-1.1, -0.7, (-1.1 * 0.9 - 1) / -0.7, 0.9)
    out = lct.lct2d_sharded(torch.from_numpy(f.astype(dtype)).cuda(), ax, ay)
    torch.cuda.synchronize()
    got = out.cpu().numpy()                          # [nx][ny]: the output transposed
    rows = O.lct(f.astype(dtype).astype(np.complex128), ax)
    ref = O.lct(np.ascontiguousarray(rows.T), ay)
    assert rel_l2(got.reshape(-1), ref.reshape(-1)) < tol
