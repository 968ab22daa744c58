"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (relative L2 per signal, the maximum over signals must pass):
  FP64 paths (complex128, fused and plain)   1e-12
  FP32 fused path (complex64)                1e-5
  plain FP64 path with complex64 I/O         1e-6 (output rounded to FP32)
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
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


def to_dev(f, dtype):
    return torch.from_numpy(np.ascontiguousarray(f.astype(dtype))).cuda()


def run(plan, f, dtype, batch=None, inplace=False):
    x = to_dev(f, dtype)
    out = x if inplace else torch.empty_like(x)
    n = f.shape[0] if batch is None else batch
    lct.lct_execute(plan, x, out, n)
    torch.cuda.synchronize()
    assert lct.lct_device_status(plan) == 0
    return out.cpu().numpy()


def rot(t):
    return (np.cos(t), np.sin(t), -np.sin(t), np.cos(t))


# --------------------------------------------------------------------------
# config 0: N = 256, complex128, rotation 0.7, polynomial + psi_0..psi_10
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [lct.LCT_PREC_NATIVE, lct.LCT_PREC_PLAIN64])
def test_config0_fp64(prec):
    N = 256
    x = O.nodes(N)
    f = W.config0_signals(x)
    abcd = W.config0_params()
    p = lct.Plan.create(N, *abcd, dtype=lct.LCT_C128).set_precision(prec)
    try:
        G = run(p.handle, f, np.complex128)
    finally:
        p.destroy()
    ref = O.lct(f, abcd)
    assert rel_l2(G, ref).max() < TOL64


# --------------------------------------------------------------------------
# every supported N, both precisions, ragged batch counts
# --------------------------------------------------------------------------
@pytest.mark.parametrize("log2n", list(range(1, 17)))
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_every_size(log2n, dtype):
    N = 1 << log2n
    count = 37 if N <= 1024 else (5 if N <= 16384 else 2)   # ragged w.r.t. signals per CTA
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=100 + log2n, dtype=np.complex128)
    abcd = (0.37, -1.3, (0.37 * 0.8 - 1) / -1.3, 0.8)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.create(N, *abcd, dtype=code)
    try:
        G = run(p.handle, f.astype(dtype), dtype)
    finally:
        p.destroy()
    ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
    tol = TOL32 if dtype == np.complex64 else TOL64
    assert rel_l2(G, ref).max() < tol


# --------------------------------------------------------------------------
# per-signal parameters (batch plan), generator G1
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,count,seed", [(1024, 512, W.SEED_UNIFORM_1024), (4096, 48, 77)])
def test_uniform_batch_per_signal_params(N, count, seed):
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=seed, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
    try:
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), params)
    err = rel_l2(G, ref)
    assert err.max() < TOL32


@pytest.mark.parametrize("N,count", [(256, 100), (1024, 333), (4096, 700), (8192, 30), (16384, 9)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11])
def test_kernel_variants(N, count, variant):
    """Both fused variants (one CTA per group / persistent with bulk-async
    prefetch) on per-signal parameters, with a ragged last group."""
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N + variant, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N).set_variant(variant)
    try:
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    n_check = 24 if N <= 4096 else 3                  # oracle cost grows as N^2
    idx = np.unique(np.linspace(0, count - 1, n_check).astype(int))
    ref = O.lct(f[idx].astype(np.complex128), params[idx])
    assert rel_l2(G[idx], ref).max() < TOL32


@pytest.mark.parametrize("N,count", [(256, 40), (256, 33), (4096, 7)])
def test_tensor_map_variant_partial_groups_and_fallback(N, count):
    """Variant 8 (TMA tensor-map staged loads): a last group that ends
    inside its box (count not a multiple of the signals per CTA, zero-filled
    rows), and a batch whose N count is not a multiple of 256 rows of the
    tensor view (33 x 256 is, 7 x 4096 is; the gapped plan falls back)."""
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N + 8 * count, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N).set_variant(8)
    try:
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), params)
    assert rel_l2(G, ref).max() < TOL32
    # gapped offsets: not contiguous, so the plan runs variant 0 instead
    offs = np.arange(count, dtype=np.int64) * (N + 2)
    buf = np.zeros(offs[-1] + N, dtype=np.complex64)
    for s in range(count):
        buf[offs[s]:offs[s] + N] = f[s]
    p = lct.Plan.batch([N] * count, params, offs).set_variant(8)
    try:
        Gb = run(p.handle, buf[None, :], np.complex64, batch=count)[0]
    finally:
        p.destroy()
    for s in range(count):
        assert rel_l2(Gb[offs[s]:offs[s] + N], ref[s]) < TOL32


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("log2n", [13, 14, 15, 16])
@pytest.mark.parametrize("variant", [5, 7])
def test_large_n_variants(dtype, log2n, variant):
    """Large N: the cluster kernel (5, N >= 16384) and the two-pass kernels
    (7, N >= 8192) on per-signal parameters, both precisions."""
    if variant == 5 and log2n < 14:
        pytest.skip("cluster kernel starts at N = 16384")
    N, count = 1 << log2n, 3
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=log2n * 10 + variant, dtype=np.complex128)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code).set_variant(variant)
    try:
        G = run(p.handle, f.astype(dtype), dtype)
    finally:
        p.destroy()
    idx = [0, count - 1] if log2n == 16 else list(range(count))
    ref = O.lct(f[idx].astype(dtype).astype(np.complex128), params[idx])
    assert rel_l2(G[idx], ref).max() < (TOL32 if dtype == np.complex64 else TOL64)


def test_twopass_gapped_offsets():
    """The two-pass path on signals stored with gaps (odd offsets); the gaps
    stay untouched."""
    N, count = 8192, 520
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=77, dtype=np.complex64)
    stride = N + 3
    offs = np.arange(count, dtype=np.int64) * stride
    buf = np.zeros(count * stride, dtype=np.complex64)
    for s in range(count):
        buf[offs[s]:offs[s] + N] = f[s]
    p = lct.Plan.batch([N] * count, params, offs, dtype=lct.LCT_C64).set_variant(7)
    try:
        xin = torch.from_numpy(buf).cuda()
        out = torch.zeros_like(xin)
        lct.lct_execute(p.handle, xin, out, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        ob = out.cpu().numpy()
    finally:
        p.destroy()
    idx = [0, 1, 510, 511, 512, 513, 519]
    ref = O.lct(f[idx].astype(np.complex128), params[idx])
    G = np.stack([ob[offs[s]:offs[s] + N] for s in idx])
    assert rel_l2(G, ref).max() < TOL32
    mask = np.ones(len(buf), dtype=bool)
    for o in offs:
        mask[o:o + N] = False
    assert np.all(ob[mask] == 0)


def test_autotune_picks_a_valid_variant():
    N, count = 4096, 512
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=21, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N)
    try:
        xin = to_dev(f, np.complex64)
        out = torch.empty_like(xin)
        v = p.autotune(xin, out, count)
        assert v in (0, 1, 2, 3, 4, 5, 6, 8, 10, 11)
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    ref = O.lct(f[:8].astype(np.complex128), params[:8])
    assert rel_l2(G[:8], ref).max() < TOL32


def test_in_place_equals_out_of_place():
    N, count = 4096, 6
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=5, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N)
    try:
        a = run(p.handle, f, np.complex64)
        b = run(p.handle, f, np.complex64, inplace=True)
    finally:
        p.destroy()
    assert np.array_equal(a, b)


def test_plain64_complex64_io():
    N, count = 1024, 16
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=9, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N).set_precision(lct.LCT_PREC_PLAIN64)
    try:
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), params)
    assert rel_l2(G, ref).max() < 1e-6


# --------------------------------------------------------------------------
# N that is not a power of two: 7-smooth N by the mixed-radix kernel (chirp,
# DFT_N, chirp); other N by chirp - FFT_M - spectrum - inverse FFT_M - chirp
# (M >= 2N - 1) in one kernel (here 4095 = 3^2 5 7 13 and 8191, prime)
# --------------------------------------------------------------------------
NON_POW2 = [3, 5, 6, 7, 12, 100, 1000, 4095]


@pytest.mark.parametrize("N", NON_POW2 + [6000, 8191])
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_every_size_non_power_of_two(N, dtype):
    if dtype == np.complex128 and N > 4096:
        pytest.skip("complex128 takes N <= 4096 when N is not a power of two")
    count = 37 if N <= 1024 else 5
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=200 + N, dtype=np.complex128)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    for abcd in [(0.37, -1.3, (0.37 * 0.8 - 1) / -1.3, 0.8), None]:
        if abcd is None:       # per-signal parameters (batch plan)
            p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code)
            ref = O.lct(f.astype(dtype).astype(np.complex128), params)
        else:
            p = lct.Plan.create(N, *abcd, dtype=code)
            ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
        try:
            G = run(p.handle, f.astype(dtype), dtype)
        finally:
            p.destroy()
        assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64), (N, abcd is None)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_non_power_of_two_b_zero_frft_and_complex(dtype):
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    tol = TOL32 if dtype == np.complex64 else TOL64
    N = 300
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 4, seed=31, dtype=np.complex128)
    f = f.astype(dtype)
    f64 = f.astype(np.complex128)
    # b = 0
    abcd = (1 / 1.3, 0.0, -0.7, 1.3)
    p = lct.Plan.create(N, *abcd, dtype=code)
    try:
        assert rel_l2(run(p.handle, f, dtype), O.lct(f64, abcd)).max() < tol
    finally:
        p.destroy()
    # fractional transform, z inside and on the unit circle
    for z in [0.6 + 0.2j, np.exp(-0.9j)]:
        xin = to_dev(f, dtype)
        out = torch.empty_like(xin)
        lct.frft_execute(N, z, xin, out, f.shape[0], code)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), O.frft(f64, z)).max() < tol, z


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_ragged_mixed_powers_and_other_sizes(dtype):
    """Powers of two and other N, b = 0 and b != 0, in one ragged plan."""
    specs = [(None, 100, "lct", (0.5, 1.2, (0.5 * 0.4 - 1) / 1.2, 0.4)),
             (None, 1000, "lct", (-1.1, -0.6, (-1.1 * 1.3 - 1) / -0.6, 1.3)),
             (None, 256, "lct", (0.2, 0.9, (0.2 * -0.5 - 1) / 0.9, -0.5)),
             (None, 100, "b0", (1 / 0.8, 0.0, 0.6, 0.8)),
             (None, 7, "lct", (0.0, 1.0, -1.0, 0.0)),
             (None, 4095, "frft", 0.7 * np.exp(1.2j)),
             (None, 64, "b0", (1 / 1.5, 0.0, -0.2, 1.5)),
             (None, 100, "lct", (1.4, -1.8, (1.4 * 0.3 - 1) / -1.8, 0.3))]
    rng = np.random.default_rng(77)
    Ns, abcds, offs, sigs = [], [], [], []
    off = 3
    for _, N, kind, prm in specs:
        abcd = O.abcd_of_z(prm) if kind == "frft" else np.asarray(prm, dtype=np.complex128)
        x = O.nodes(N)
        f = np.exp(-x * x / 8) * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
        Ns.append(N)
        abcds.append(abcd)
        offs.append(off)
        sigs.append(f)
        off += N + 5
    buf = np.zeros(off, dtype=np.complex128)
    for o, f in zip(offs, sigs):
        buf[o:o + len(f)] = f
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.batch(Ns, np.array(abcds), offs, dtype=code)
    try:
        x = torch.from_numpy(buf.astype(dtype)).cuda()
        out = torch.zeros_like(x)
        lct.lct_execute(p.handle, x, out, len(Ns))
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        G = out.cpu().numpy()
    finally:
        p.destroy()
    tol = TOL32 if dtype == np.complex64 else TOL64
    for N, abcd, o, f in zip(Ns, abcds, offs, sigs):
        ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
        assert rel_l2(G[o:o + N], ref) < tol, (N, abcd)
    mask = np.ones(len(buf), dtype=bool)
    for N, o in zip(Ns, offs):
        mask[o:o + N] = False
    assert np.all(G[mask] == 0)


@pytest.mark.parametrize("N", [256, 4096])
def test_plain32_complex64(N):
    """The unfused FP32 baseline (FP32 chirps around cuFFT C2C)."""
    count = 16
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=19, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N).set_precision(lct.LCT_PREC_PLAIN32)
    try:
        G = run(p.handle, f, np.complex64)
    finally:
        p.destroy()
    ref = O.lct(f.astype(np.complex128), params)
    assert rel_l2(G, ref).max() < TOL32


def test_plain32_rejects_complex128():
    p = lct.Plan.create(256, 1.0, 2.0, 0.5, 2.0, dtype=lct.LCT_C128)
    try:
        with pytest.raises(lct.LctError) as e:
            p.set_precision(lct.LCT_PREC_PLAIN32)
        assert e.value.status == 10
    finally:
        p.destroy()


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("count", [1, 12, 16 * 160 + 3])
def test_small_and_packed_batches_n256(dtype, count):
    """N = 256 packs 16 signals per CTA; a batch that would fill fewer CTAs
    than the GPU has SMs runs one signal per CTA instead (12 signals: the
    complex128 latency case).  Both shapes against the oracle."""
    N = 256
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=23 + count, dtype=np.complex128)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code)
    try:
        G = run(p.handle, f.astype(dtype), dtype)
    finally:
        p.destroy()
    ref = O.lct(f.astype(dtype).astype(np.complex128), params)
    assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64)


# --------------------------------------------------------------------------
# b = 0 branch, complex parameters, fractional transform
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_b_zero(dtype):
    N = 512
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 7, seed=3, dtype=np.complex128)
    abcd = (1 / 1.7, 0.0, -0.9, 1.7)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.create(N, *abcd, dtype=code)
    try:
        G = run(p.handle, f.astype(dtype), dtype)
    finally:
        p.destroy()
    ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
    assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64)


@pytest.mark.parametrize("z", [0.5 + 0.3j, 0.9 * np.exp(2.0j), np.exp(-0.7j), 1.0, -1.0])
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_frft(z, dtype):
    N = 256
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 5, seed=11, dtype=np.complex128)
    f = f.astype(dtype)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    xin = to_dev(f, dtype)
    out = torch.empty_like(xin)
    lct.frft_execute(N, z, xin, out, f.shape[0], code)
    torch.cuda.synchronize()
    G = out.cpu().numpy()
    if abs(1 - z * z) == 0:
        ref = np.sqrt(2 * np.pi) * f.astype(np.complex128)     # F_{+-1} = sqrt(2 pi) I on y = x/z
    else:
        ref = O.frft(f.astype(np.complex128), z)
    assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64)


def test_complex_parameters_plan():
    N = 1024
    z = 0.6 * np.exp(1.2j)
    abcd = O.abcd_of_z(z)
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 4, seed=12, dtype=np.complex128)
    p = lct.Plan.create(N, *[complex(v) for v in abcd], dtype=lct.LCT_C128)
    try:
        G = run(p.handle, f, np.complex128)
        y, rho = lct.lct_output_grid(p.handle, 0, N)
    finally:
        p.destroy()
    ref, rho_o = O.lct(f, abcd, return_rho=True)
    assert rel_l2(G, ref).max() < TOL64
    assert np.allclose(rho, rho_o[0], rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# the throughput workload at full size, in the launch configuration the
# benchmark times: 16384 signals x N = 4096, complex64, per-signal params
# --------------------------------------------------------------------------
def test_full_size_uniform_4096():
    N, count = 4096, 16384
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=W.SEED_UNIFORM_4096, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N)
    try:
        xin = to_dev(f, np.complex64)
        out = torch.empty_like(xin)
        lct.lct_execute(p.handle, xin, out, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        # property at every signal: scaled Parseval ||G||^2 dy = ||f||^2 dx, dy = 4|b| dx / pi
        nf = torch.linalg.vector_norm(xin.to(torch.complex128), dim=1) ** 2
        ng = torch.linalg.vector_norm(out.to(torch.complex128), dim=1) ** 2
        b = torch.from_numpy(np.abs(params[:, 1])).cuda()
        ratio = (ng * 4 * b / np.pi / nf).cpu().numpy()
        assert np.abs(ratio - 1).max() < 2e-5
        idx = np.arange(0, count, 256)                           # 64 sampled signals
        G = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    finally:
        p.destroy()
    ref = O.lct(f[idx].astype(np.complex128), params[idx])
    assert rel_l2(G, ref).max() < TOL32


# --------------------------------------------------------------------------
# ragged batches: mixed N and kinds in one plan, one CUDA-graph launch
# --------------------------------------------------------------------------
def _ragged_case(specs, seed, gap=3):
    """specs: list of (log2n, kind, abcd or z). Returns N, abcd (complex),
    offsets (with gaps), packed input (complex64) and the per-signal inputs."""
    rng = np.random.default_rng(seed)
    Ns, abcds, offs, sigs = [], [], [], []
    off = 0
    for log2n, kind, par in specs:
        N = 1 << log2n
        if kind == "frft":
            abcd = O.abcd_of_z(par)
        else:
            abcd = np.asarray(par, dtype=np.complex128)
        x = O.nodes(N)
        f = (np.exp(-x * x / 8) * np.exp(0.3j * x * x)
             + 1e-3 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))).astype(np.complex64)
        Ns.append(N); abcds.append(abcd); offs.append(off); sigs.append(f)
        off += N + gap * 2                      # even gaps keep 16-byte alignment optional
    buf = np.zeros(off, dtype=np.complex64)
    for o, f in zip(offs, sigs):
        buf[o:o + len(f)] = f
    return np.array(Ns), np.array(abcds), np.array(offs), buf, sigs


RAGGED_SPECS = [
    (16, "lct", (0.4, 1.3, (0.4 * -0.7 - 1) / 1.3, -0.7)),
    (10, "frft", 0.6 * np.exp(1.1j)),
    (6, "lct", (0.0, 1.0, -1.0, 0.0)),
    (12, "b0", (1 / 1.4, 0.0, 0.7, 1.4)),
    (15, "lct", (-1.2, -0.5, (-1.2 * 0.9 - 1) / -0.5, 0.9)),
    (8, "frft", 0.35 * np.exp(-2.0j)),
    (12, "lct", (1.1, 0.8, (1.1 * 0.3 - 1) / 0.8, 0.3)),
    (10, "lct", (0.0, 1.0, -1.0, 0.0)),
    (7, "b0", (1 / 0.6, 0.0, -1.5, 0.6)),
    (14, "lct", (0.2, 1.9, (0.2 * 1.5 - 1) / 1.9, 1.5)),
    (12, "frft", 0.9 * np.exp(0.4j)),
    (9, "lct", (1.7, -1.1, (1.7 * 0.2 - 1) / -1.1, 0.2)),
]


@pytest.mark.parametrize("variant", [None, 9])
def test_ragged_mixed_sizes_and_kinds(variant):
    """variant None: the CUDA graph of one kernel per N; 9: one persistent
    launch over a largest-first work queue."""
    Ns, abcds, offs, buf, sigs = _ragged_case(RAGGED_SPECS, seed=31)
    p = lct.Plan.batch(Ns, abcds, offs, dtype=lct.LCT_C64)
    if variant is not None:
        p.set_variant(variant)
    try:
        x = torch.from_numpy(buf).cuda()
        out = torch.zeros_like(x)
        lct.lct_execute(p.handle, x, out, len(Ns))
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        G = out.cpu().numpy()
        # a second buffer pair: the graph is captured again for the new pointers
        x2 = torch.from_numpy(buf[::-1].copy()[::-1].copy()).cuda()
        out2 = torch.zeros_like(x2)
        lct.lct_execute(p.handle, x2, out2, len(Ns))
        torch.cuda.synchronize()
        G2 = out2.cpu().numpy()
    finally:
        p.destroy()
    assert np.array_equal(G, G2)
    for N, abcd, o, f in zip(Ns, abcds, offs, sigs):
        ref = O.lct(f.astype(np.complex128), abcd)
        assert rel_l2(G[o:o + N], ref) < TOL32, (N, abcd)
    # the gaps between signals are untouched
    mask = np.ones(len(buf), dtype=bool)
    for N, o in zip(Ns, offs):
        mask[o:o + N] = False
    assert np.all(G[mask] == 0)


SMALL_SPECS = [
    (1, "lct", (0.4, 1.3, (0.4 * -0.7 - 1) / 1.3, -0.7)),
    (2, "frft", 0.6 * np.exp(1.1j)),
    (3, "lct", (0.0, 1.0, -1.0, 0.0)),
    (1, "b0", (1 / 1.4, 0.0, 0.7, 1.4)),
    (4, "lct", (-1.2, -0.5, (-1.2 * 0.9 - 1) / -0.5, 0.9)),
    (5, "frft", 0.35 * np.exp(-2.0j)),
    (2, "b0", (1 / 0.6, 0.0, -1.5, 0.6)),
    (3, "lct", (1.7, -1.1, (1.7 * 0.2 - 1) / -1.1, 0.2)),
    (11, "b0", (1 / 0.9, 0.0, 0.3, 0.9)),
    (12, "b0", (1 / 1.9, 0.0, -0.3, 1.9)),
]


@pytest.mark.parametrize("dtype,variant", [(np.complex64, None), (np.complex128, None),
                                           (np.complex64, 9)])
def test_ragged_smallest_sizes_both_dtypes(dtype, variant):
    """Ragged plans with N = 2 .. 32 (several signals per CTA), b = 0 signals
    below and above the 2048-sample chunk of the diagonal launch, and -- in
    complex128 -- an N = 32768 signal on the persistent two-pass kernel."""
    specs = list(SMALL_SPECS)
    if dtype == np.complex128:
        specs.append((15, "lct", (0.9, -0.7, (0.9 * 0.4 - 1) / -0.7, 0.4)))
    Ns, abcds, offs, buf, sigs = _ragged_case(specs, seed=53)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    p = lct.Plan.batch(Ns, abcds, offs, dtype=code)
    if variant is not None:
        p.set_variant(variant)
    try:
        x = torch.from_numpy(buf.astype(dtype)).cuda()
        out = torch.zeros_like(x)
        lct.lct_execute(p.handle, x, out, len(Ns))
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        G = out.cpu().numpy()
    finally:
        p.destroy()
    tol = TOL32 if dtype == np.complex64 else TOL64
    for N, abcd, o, f in zip(Ns, abcds, offs, sigs):
        ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
        assert rel_l2(G[o:o + N], ref) < tol, (N, abcd)
    mask = np.ones(len(buf), dtype=bool)
    for N, o in zip(Ns, offs):
        mask[o:o + N] = False
    assert np.all(G[mask] == 0)


@pytest.mark.parametrize("variant", [None, 9])
def test_ragged_full_size_workload(variant):
    """The 20000-instance ragged workload (N = 2^6..2^16, four kinds), one
    graph launch (variant None) or one persistent launch (9); parity on a
    sample of signals, Parseval on all real ones."""
    r = W.ragged_plan()
    M = len(r["kind"])
    Ns = (1 << r["log2n"]).astype(np.int64)
    abcd = r["abcd"].copy()
    fr = r["kind"] == W.KIND_FRFT
    for s in np.nonzero(fr)[0]:
        abcd[s] = O.abcd_of_z(r["z"][s])
    offs = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)
    total = int(Ns.sum())
    buf = np.empty(total, dtype=np.complex64)
    rng = r["rng"]
    for s in range(M):
        x = O.nodes(int(Ns[s]))
        buf[offs[s]:offs[s] + Ns[s]] = W.ragged_signal(x, r["s"][s], r["q"][s], rng)
    p = lct.Plan.batch(Ns, abcd, offs, dtype=lct.LCT_C64)
    if variant is not None:
        p.set_variant(variant)
    try:
        xin = torch.from_numpy(buf).cuda()
        out = torch.empty_like(xin)
        lct.lct_execute(p.handle, xin, out, M)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        G = out.cpu().numpy()
    finally:
        p.destroy()
    # sample: the first three signals of every kind at every N = 2^6 .. 2^16
    # (the sizes from 8192 up hold most of the points; they run on the
    # two-pass and single-CTA kernels of the graph, complex-z FrFT included)
    checked = 0
    for kind in range(4):
        for log2n in range(6, 17):
            ids = np.nonzero((r["kind"] == kind) & (r["log2n"] == log2n))[0][:3]
            assert len(ids) == 3, (kind, log2n)
            N = 1 << log2n
            f = np.stack([buf[offs[s]:offs[s] + N] for s in ids]).astype(np.complex128)
            ref = O.lct(f, abcd[ids])
            for k, s in enumerate(ids):
                o = offs[s]
                assert rel_l2(G[o:o + N], ref[k]) < TOL32, (kind, N, int(s))
                checked += 1
    assert checked == 4 * 11 * 3
    # scaled Parseval for every real-parameter signal with b != 0
    for s in np.nonzero((r["kind"] == W.KIND_GENERIC) | (r["kind"] == W.KIND_FOURIER))[0]:
        o, N = offs[s], Ns[s]
        b = abs(abcd[s][1])
        lhs = np.sum(np.abs(G[o:o + N].astype(np.complex128)) ** 2) * 4 * b / np.pi
        rhs = np.sum(np.abs(buf[o:o + N].astype(np.complex128)) ** 2)
        assert abs(lhs / rhs - 1) < 2e-5


# 7-smooth sizes that are not powers of two take the mixed-radix kernel (one
# DFT of N); every radix (16, 8, 4, 2, 7, 5, 3) appears first, in the middle
# and last, and alone.
MIXED_SIZES = [3, 5, 6, 7, 9, 10, 12, 14, 15, 21, 24, 25, 27, 35, 48, 49, 96, 125, 243, 343, 384,
               625, 729, 1000, 1536, 2187, 2401, 3000, 3072, 3125, 4000, 6000, 6144, 6561, 7168,
               7776, 8000]


@pytest.mark.parametrize("N", MIXED_SIZES)
def test_mixed_radix_sizes(N):
    count = 13 if N <= 1024 else 3
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=900 + N, dtype=np.complex128)
    for dtype in [np.complex64, np.complex128]:
        if dtype == np.complex128 and N > 4096:
            continue
        code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
        fd = f.astype(dtype)
        ref = O.lct(fd.astype(np.complex128), params)
        p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code)
        try:
            G = run(p.handle, fd, dtype)
        finally:
            p.destroy()
        assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64), (N, dtype)
        abcd = (0.37, -1.3, (0.37 * 0.8 - 1) / -1.3, 0.8)
        p = lct.Plan.create(N, *abcd, dtype=code)
        try:
            G = run(p.handle, fd, dtype)
        finally:
            p.destroy()
        ref = O.lct(fd.astype(np.complex128), abcd)
        assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64), (N, dtype)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("N", [16, 32, 64, 512, 2048, 8192])
def test_schedule_variants_both_dtypes(N, dtype):
    """The autotuner's schedules (10: radix-8 passes; 11: one signal per CTA)
    in both dtypes, shared parameters, a partly empty last CTA."""
    count = 37 if N <= 2048 else 5
    x = O.nodes(N)
    _, f = W.uniform_batch(x, count, seed=N + 11, dtype=np.complex128)
    abcd = (0.9, -0.7, (0.9 * 1.2 - 1) / -0.7, 1.2)
    code = lct.LCT_C64 if dtype == np.complex64 else lct.LCT_C128
    ref = O.lct(f.astype(dtype).astype(np.complex128), abcd)
    for variant in (10, 11):
        p = lct.Plan.create(N, *abcd, dtype=code).set_variant(variant)
        try:
            G = run(p.handle, f.astype(dtype), dtype)
        finally:
            p.destroy()
        assert rel_l2(G, ref).max() < (TOL32 if dtype == np.complex64 else TOL64), (N, variant)


def test_ragged_groups_take_schedule_defaults():
    """Ragged groups of N = 256, 512, 1024 and 2048 run their default
    schedules (variants 10, 11, 11, 11) inside the graph, through the signal
    index lists."""
    specs = [256, 1024, 2048, 256, 1024, 2048, 512]
    rng = np.random.default_rng(5)
    Ns, abcds, offs, sigs = [], [], [], []
    off = 0
    for N in specs:
        b = rng.uniform(0.5, 2.0) * rng.choice([-1, 1])
        a, d = rng.uniform(-1.5, 1.5), rng.uniform(-1.5, 1.5)
        abcd = np.array([a, b, (a * d - 1) / b, d], dtype=np.complex128)
        x = O.nodes(N)
        f = np.exp(-x * x / 8) * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
        Ns.append(N)
        abcds.append(abcd)
        offs.append(off)
        sigs.append(f)
        off += N + 3
    buf = np.zeros(off, dtype=np.complex128)
    for o, f in zip(offs, sigs):
        buf[o:o + len(f)] = f
    p = lct.Plan.batch(Ns, np.array(abcds), offs, dtype=lct.LCT_C64)
    try:
        xin = torch.from_numpy(buf.astype(np.complex64)).cuda()
        out = torch.zeros_like(xin)
        lct.lct_execute(p.handle, xin, out, len(Ns))
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        ob = out.cpu().numpy()
    finally:
        p.destroy()
    for o, f, abcd in zip(offs, sigs, abcds):
        ref = O.lct(f.astype(np.complex64).astype(np.complex128), abcd)
        assert rel_l2(ob[o:o + len(f)], ref).max() < TOL32
