"""lct_execute_host: host buffers, chunked copy-in / transform / copy-out
pipeline.  The kernels are the device path's, so the results must be
bit-identical to lct_execute on device buffers; a sample is also checked
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
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


def device_result(plan, f):
    x = torch.from_numpy(f).cuda()
    out = torch.empty_like(x)
    plan.execute(x, out, f.shape[0])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def host_result(plan, f, pinned=True):
    if pinned:
        h_in = torch.from_numpy(f).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
    else:
        h_in = torch.from_numpy(f.copy())
        h_out = torch.empty_like(h_in)
    plan.execute_host(h_in, h_out, f.shape[0], torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert lct.lct_device_status(plan.handle) == 0
    return h_out.numpy()


@pytest.mark.parametrize("N,count,per_signal", [(4096, 5000, False), (4096, 5000, True),
                                                (256, 70000, True), (65536, 300, True)])
def test_host_equals_device(N, count, per_signal):
    """Several chunks (about 32 MiB each), a partial last chunk."""
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N + count, dtype=np.complex64)
    if per_signal:
        plan = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
    else:
        plan = lct.Plan.create(N, *params[0], dtype=lct.LCT_C64)
    try:
        ref_dev = device_result(plan, f)
        got = host_result(plan, f)
        got2 = host_result(plan, f[::-1].copy())          # a second call, other data
    finally:
        plan.destroy()
    assert np.array_equal(got, ref_dev)
    idx = np.unique(np.linspace(0, count - 1, 3 if N > 8192 else 6).astype(int))
    ref = O.lct(f[idx].astype(np.complex128), params[idx] if per_signal else params[0])
    assert rel_l2(got[idx], ref).max() < 1e-5
    if not per_signal:
        assert np.array_equal(got2, ref_dev[::-1])


def test_host_pageable_memory_and_fp64():
    N, count = 1024, 3000
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=9, dtype=np.complex128)
    plan = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C128)
    try:
        ref_dev = device_result(plan, f)
        got = host_result(plan, f, pinned=False)
    finally:
        plan.destroy()
    assert np.array_equal(got, ref_dev)


def test_host_staged_path_for_bulk_copy_variants():
    """Page-locked buffers are read in place by the plain-load kernels; a
    bulk-copy variant (1) keeps the chunked staging path: both bit-identical
    to the device run."""
    N, count = 4096, 5000
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=77, dtype=np.complex64)
    for variant in (0, 1):
        plan = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
        plan.set_variant(variant)
        try:
            ref_dev = device_result(plan, f)
            got = host_result(plan, f)
        finally:
            plan.destroy()
        assert np.array_equal(got, ref_dev), variant
