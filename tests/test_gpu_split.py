"""GPU parity of the tensor-core precisions (split BF16, split FP16, FP16)
against the FP64 oracle, through the C ABI.

Tolerances (relative L2 per signal, maximum over the checked signals):
  SPLIT_BF16, SPLIT_FP16   1e-5 (the split precision path's bound)
  FP16                     1e-2 (the plain FP16 path's bound)
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402

MODES = {
    "split_bf16": (lct.LCT_PREC_SPLIT_BF16, 1e-5),
    "split_fp16": (lct.LCT_PREC_SPLIT_FP16, 1e-5),
    "fp16": (lct.LCT_PREC_FP16, 1e-2),
}


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    torch.cuda.set_device(0)


def run(plan, f, batch=None):
    x = torch.from_numpy(np.ascontiguousarray(f.astype(np.complex64))).cuda()
    out = torch.empty_like(x)
    lct.lct_execute(plan, x, out, f.shape[0] if batch is None else batch)
    torch.cuda.synchronize()
    assert lct.lct_device_status(plan) == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("log2n", list(range(4, 13)))
def test_every_size_uniform_plan(mode, log2n):
    """One descriptor for the batch; the count leaves a partial last tile
    (4096/N signals per CTA)."""
    prec, tol = MODES[mode]
    N = 1 << log2n
    per_cta = 4096 // N
    count = 3 * per_cta + max(1, per_cta // 3) if per_cta > 1 else 5
    x = O.nodes(N)
    _, f = W.uniform_batch(x, count, seed=300 + log2n, dtype=np.complex64)
    abcd = (0.37, -1.3, (0.37 * 0.8 - 1) / -1.3, 0.8)
    p = lct.Plan.create(N, *abcd, dtype=lct.LCT_C64).set_precision(prec)
    try:
        G = run(p.handle, f)
    finally:
        p.destroy()
    idx = np.unique(np.linspace(0, count - 1, min(count, 40)).astype(int))
    ref = O.lct(f[idx].astype(np.complex128), abcd)
    assert rel_l2(G[idx], ref).max() < tol


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("N,count", [(64, 200), (1024, 77), (4096, 40)])
def test_per_signal_params_and_offsets(mode, N, count):
    """Batch plan: per-signal G1 parameters, signals stored in reverse order
    with a gap between them."""
    prec, tol = MODES[mode]
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N + 17, dtype=np.complex64)
    stride = N + 8
    offsets = (count - 1 - np.arange(count)) * stride
    buf = np.zeros(count * stride, dtype=np.complex64)
    for s in range(count):
        buf[offsets[s]:offsets[s] + N] = f[s]
    p = lct.Plan.batch([N] * count, params, offsets, dtype=lct.LCT_C64).set_precision(prec)
    try:
        xin = torch.from_numpy(buf).cuda()
        out = torch.zeros_like(xin)
        lct.lct_execute(p.handle, xin, out, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        ob = out.cpu().numpy()
    finally:
        p.destroy()
    G = np.stack([ob[o:o + N] for o in offsets])
    gaps = np.ones(count * stride, dtype=bool)
    for o in offsets:
        gaps[o:o + N] = False
    assert np.all(ob[gaps] == 0)                     # nothing written outside the signals
    ref = O.lct(f.astype(np.complex128), params)
    assert rel_l2(G, ref).max() < tol


@pytest.mark.parametrize("mode", list(MODES))
def test_magnitudes_far_apart_in_one_tile(mode):
    """Per-signal scaling: signals of very different size (and a zero signal)
    share a CTA at N = 256 (16 signals per CTA)."""
    prec, tol = MODES[mode]
    N, count = 256, 16
    x = O.nodes(N)
    _, f = W.uniform_batch(x, count, seed=5, dtype=np.complex128)
    scales = np.array([1e-30, 1e30, 1.0, 0.0, 1e-20, 3e20, 1e-3, 7.0,
                       1e10, 1e-10, 2.0, 0.5, 1e-35, 1e35, 1.0, 1.0])
    f = f * scales[:, None]
    abcd = (1.1, 0.6, (1.1 * 0.9 - 1) / 0.6, 0.9)
    p = lct.Plan.create(N, *abcd, dtype=lct.LCT_C64).set_precision(prec)
    try:
        G = run(p.handle, f.astype(np.complex64))
    finally:
        p.destroy()
    assert np.all(G[3] == 0)
    keep = scales != 0
    if prec == lct.LCT_PREC_SPLIT_BF16:
        keep &= (scales > 1e-30) & (scales < 1e30)   # BF16 has FP32's range, no rescaling
    assert np.all(np.isfinite(G[keep]))
    ref = O.lct(f[keep].astype(np.complex64).astype(np.complex128), abcd)
    assert rel_l2(G[keep], ref).max() < tol


@pytest.mark.parametrize("mode", list(MODES))
def test_complex_parameters_and_b_zero(mode):
    """Complex z fractional transform (Gaussian decay in the pre-chirp) and a
    b = 0 plan (no DFT; the diagonal kernel runs whatever the precision)."""
    prec, tol = MODES[mode]
    N, count = 1024, 9
    x = O.nodes(N)
    _, f = W.uniform_batch(x, count, seed=11, dtype=np.complex64)
    z = 0.8 * np.exp(0.9j)
    abcd = O.abcd_of_z(z)
    p = lct.Plan.create(N, *[complex(v) for v in abcd], dtype=lct.LCT_C64).set_precision(prec)
    try:
        G = run(p.handle, f)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), abcd)
    assert rel_l2(G, ref).max() < tol
    b0 = (0.5, 0.0, 1.3, 2.0)
    p = lct.Plan.create(N, *b0, dtype=lct.LCT_C64).set_precision(prec)
    try:
        G = run(p.handle, f)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), b0)
    assert rel_l2(G, ref).max() < 1e-5


@pytest.mark.parametrize("mode", list(MODES))
def test_full_size_16384x4096(mode):
    """The throughput workload: 16384 G1 signals of N = 4096 (per-signal
    parameters), checked on the 64 signals 0, 256, ..., 16128."""
    prec, tol = MODES[mode]
    N, count = 4096, 16384
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
    p.set_precision(prec)
    try:
        G = run(p.handle, f)
    finally:
        p.destroy()
    idx = np.arange(0, count, 256)
    ref = O.lct(f[idx].astype(np.complex128), params[idx])
    err = rel_l2(G[idx], ref)
    print("%s full-size rel L2: max %.3e median %.3e" % (mode, err.max(), np.median(err)))
    assert err.max() < tol


def test_tcgen05_split_bf16_n4096_complex_z_and_gapped_offsets():
    """Split BF16 at N = 4096 runs on the tcgen05 tensor cores: a complex-z
    fractional transform (decaying pre-chirp) and a batch plan with gaps
    between the signals (offsets not multiples of N), against the oracle."""
    N, count = 4096, 21
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=29, dtype=np.complex64)
    z = 0.7 * np.exp(-2.2j)
    abcd = O.abcd_of_z(z)
    p = lct.Plan.create(N, *[complex(v) for v in abcd], dtype=lct.LCT_C64)
    p.set_precision(lct.LCT_PREC_SPLIT_BF16)
    try:
        G = run(p.handle, f)
        assert lct.lct_device_status(p.handle) == 0
    finally:
        p.destroy()
    assert rel_l2(G, O.lct(f.astype(np.complex128), abcd)).max() < 1e-5
    offs = np.arange(count, dtype=np.int64) * (N + 6) + 2
    buf = np.zeros(offs[-1] + N + 5, dtype=np.complex64)
    for s in range(count):
        buf[offs[s]:offs[s] + N] = f[s]
    p = lct.Plan.batch([N] * count, params, offs, dtype=lct.LCT_C64)
    p.set_precision(lct.LCT_PREC_SPLIT_BF16)
    try:
        xin = torch.from_numpy(buf).cuda()
        out = torch.zeros_like(xin)
        lct.lct_execute(p.handle, xin, out, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        Gb = out.cpu().numpy()
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), params)
    for s in range(count):
        assert rel_l2(Gb[offs[s]:offs[s] + N], ref[s]) < 1e-5


@pytest.mark.parametrize("mode", ["split_fp16", "fp16"])
def test_tcgen05_fp16_scaling_at_n4096(mode):
    """The FP16 modes at N = 4096 run on tcgen05 with a per-signal
    power-of-two scale: signals from 1e-30 to 1e30 and a zero signal, each
    one CTA's work, stay inside the FP16 range."""
    prec, tol = MODES[mode]
    N = 4096
    scales = np.array([1e-30, 1e30, 1.0, 0.0, 1e-20, 3e20, 1e-3, 7.0, 1e10, 1e-10, 2.0])
    count = len(scales)
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=41, dtype=np.complex128)
    f = f * scales[:, None]
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
    p.set_precision(prec)
    try:
        G = run(p.handle, f.astype(np.complex64))
    finally:
        p.destroy()
    assert np.all(G[3] == 0)
    keep = scales != 0
    assert np.all(np.isfinite(G[keep]))
    ref = O.lct(f[keep].astype(np.complex64).astype(np.complex128), params[keep])
    assert rel_l2(G[keep], ref).max() < tol
