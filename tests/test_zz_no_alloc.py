"""lct_execute_noalloc: the entry point for callers that cannot call
cudaMalloc (their device memory is reserved up front by their own pool, or
they must not take cudaMalloc's implicit device synchronisation).  It keeps
its FP64 intermediate in a static device array instead of allocating.

Checked on calls in a row with different shapes (so a later call runs on an
array an earlier one left filled) against the existing FP64 entry point (a
plan with LCT_PREC_PLAIN64 through lct_execute) and against the FP64 oracle,
including the b = 0 branch, where the first kernel applies the whole
transform and the DFT is skipped.  A repeated call must leave the device's
free memory and PyTorch's allocation count unchanged.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402

TOL64 = 1e-12      # complex128 in/out, FP64 arithmetic on both sides
TOL_C64 = 1e-6     # complex64 in/out: both sides round an FP64 result to FP32


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    O.build()
    torch.cuda.set_device(0)


def reference(N, abcd, f, dtype_code):
    x = torch.from_numpy(f).cuda()
    out = torch.empty_like(x)
    p = lct.Plan.create(N, *abcd, dtype=dtype_code).set_precision(lct.LCT_PREC_PLAIN64)
    try:
        p.execute(x, out, f.shape[0])
        torch.cuda.synchronize()
    finally:
        p.destroy()
    return out.cpu().numpy()


def noalloc(N, abcd, f, dtype_code):
    x = torch.from_numpy(f).cuda()
    out = torch.empty_like(x)
    lct.lct_execute_noalloc(N, *abcd, x, out, f.shape[0], dtype_code)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    (4096, (0.3, -1.2, (0.3 * 1.7 - 1) / -1.2, 1.7), 8, np.complex128, lct.LCT_C128, TOL64),
    (256, (np.cos(0.7), np.sin(0.7), -np.sin(0.7), np.cos(0.7)), 37, np.complex64, lct.LCT_C64, TOL_C64),
    (1024, (1.0 / 1.6, 0.0, 0.45, 1.6), 5, np.complex128, lct.LCT_C128, TOL64),       # b = 0
    (64, (1.0 / -0.8, 0.0, -1.1, -0.8), 3, np.complex64, lct.LCT_C64, TOL_C64),       # b = 0, d < 0
]


def test_calls_in_a_row_match_the_fp64_entry_point_and_the_oracle():
    for N, abcd, count, dt, code, tol in CASES:
        x = lct.lct_input_grid(N)
        _, f = W.uniform_batch(x, count, seed=N + count, dtype=dt)
        got = noalloc(N, abcd, f, code)
        assert rel_l2(got, reference(N, abcd, f, code)).max() < tol
        assert rel_l2(got, O.lct(f.astype(np.complex128), abcd)).max() < tol


def test_a_repeated_call_allocates_nothing():
    N, count = 2048, 64
    abcd = (0.9, 1.1, (0.9 * -0.4 - 1) / 1.1, -0.4)
    x = lct.lct_input_grid(N)
    _, f = W.uniform_batch(x, count, seed=11, dtype=np.complex64)
    xin = torch.from_numpy(f).cuda()
    out = torch.empty_like(xin)
    lct.lct_execute_noalloc(N, *abcd, xin, out, count, lct.LCT_C64)      # set-up done here
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_allocated()
    lct.lct_execute_noalloc(N, *abcd, xin, out, count, lct.LCT_C64)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == torch0
    assert rel_l2(out.cpu().numpy(), O.lct(f.astype(np.complex128), abcd)).max() < TOL_C64


def test_batch_zero_does_the_set_up_and_runs_nothing():
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    lct.lct_execute_noalloc(256, 1.0, 2.0, 0.5, 2.0, x, x, 0, lct.LCT_C64)
    torch.cuda.synchronize()
    assert torch.count_nonzero(x).item() == 0


def test_rejects_sizes_beyond_the_static_array():
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(lct.LctError) as e:        # batch * N above the array
        lct.lct_execute_noalloc(4096, 1.0, 2.0, 0.5, 2.0, x, x,
                                lct.LCT_NOALLOC_MAX_POINTS // 4096 + 1, lct.LCT_C64)
    assert e.value.status == 1
    with pytest.raises(lct.LctError) as e:        # N above the largest supported length
        lct.lct_execute_noalloc(8192, 1.0, 2.0, 0.5, 2.0, x, x, 1, lct.LCT_C64)
    assert e.value.status == 2
