"""Failure detection on the GPU without a GPU fault: a kernel waits on
purpose for an event that never happens (an mbarrier phase, a counter),
gives up after a short bound and reports LCT_ERR_TIMEOUT; the context stays
usable.  Host-side validation errors are covered in test_abi.py."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402

LCT_ERR_TIMEOUT = 9


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(which):
    assert lct.lct_selftest_timeout(which, 5.0) == LCT_ERR_TIMEOUT
    # the context is still usable: a transform right after matches the oracle
    N, count = 1024, 4
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=3, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N)
    try:
        xin = torch.from_numpy(f).cuda()
        out = torch.empty_like(xin)
        lct.lct_execute(p.handle, xin, out, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        G = out.cpu().numpy()
    finally:
        p.destroy()
    assert rel_l2(G, O.lct(f.astype(np.complex128), params)).max() < 1e-5


@pytest.mark.parametrize("batch_plan", [False, True])
def test_debug_mode_flags_nonfinite_output(batch_plan):
    """LCT_DEBUG / lct_set_debug: a NaN in the input reaches the output and
    lct_execute reports LCT_ERR_DEVICE (8), as does lct_backward for a NaN
    in its cotangent; finite data passes; off again, nothing is checked."""
    N, count = 256, 8
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=4, dtype=np.complex64)
    if batch_plan:
        p = lct.Plan.batch([N] * count, params, np.arange(count) * N)
    else:
        p = lct.Plan.create(N, *params[0])
    bad = f.copy()
    bad[3, 17] = np.nan
    try:
        lct.lct_set_debug(True)
        xin = torch.from_numpy(f).cuda()
        out = torch.empty_like(xin)
        lct.lct_execute(p.handle, xin, out, count)              # finite: no error
        xbad = torch.from_numpy(bad).cuda()
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute(p.handle, xbad, out, count)
        assert e.value.status == 8
        assert lct.lct_device_status(p.handle) == 0             # the word was cleared
        # lct_backward scans its grad_in the same way
        gin = torch.empty_like(xin)
        lct.lct_backward(p.handle, xin, xin, out, gin, None, count)    # finite: no error
        with pytest.raises(lct.LctError) as e:
            lct.lct_backward(p.handle, xbad, xin, out, gin, None, count)
        assert e.value.status == 8
        assert lct.lct_device_status(p.handle) == 0
        lct.lct_set_debug(False)
        lct.lct_execute(p.handle, xbad, out, count)             # not checked when off
        torch.cuda.synchronize()
        assert not np.isfinite(out.cpu().numpy()[3]).all()
    finally:
        lct.lct_set_debug(False)
        p.destroy()
