"""GPU parity of the backward pass (adjoint + parameter gradients), the
torch autograd wrappers, and the separable 2-D transform, against the CPU
oracle (adjoint and dense-matrix gradient) and finite differences.

Tolerances: complex128 adjoint 1e-12; complex64 adjoint 1e-5; parameter
gradients 1e-9 (complex128) and 1e-4 (complex64), relative to the largest
component."""
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


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def grad_rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [(64, np.complex128), (1024, np.complex128), (4096, np.complex64), (256, np.complex64)]


@pytest.mark.parametrize("N,dt", CASES)
@pytest.mark.parametrize("per_signal", [False, True])
def test_backward_matches_oracle(N, dt, per_signal):
    count = 6
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N, dtype=dt)
    rng = np.random.default_rng(N + 1)
    g = (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))).astype(dt)
    code = lct.LCT_C64 if dt == np.complex64 else lct.LCT_C128
    if per_signal:
        p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code)
        abcd = params
    else:
        abcd = params[0]
        p = lct.Plan.create(N, *abcd, dtype=code)
    try:
        xf, xg = cu(f), cu(g)
        G = torch.empty_like(xf)
        p.execute(xf, G, count)
        h = torch.empty_like(xf)
        gp = torch.zeros((count, 3) if per_signal else (3,), dtype=torch.float64, device="cuda")
        lct.lct_backward(p.handle, xg, xf, G, h, gp, count)
        torch.cuda.synchronize()
        assert lct.lct_device_status(p.handle) == 0
        h, gp, Gc = h.cpu().numpy(), gp.cpu().numpy(), G.cpu().numpy()
    finally:
        p.destroy()
    f64, g64 = f.astype(np.complex128), g.astype(np.complex128)
    ref_h = O.lct_adjoint(g64, abcd)
    tol = 1e-12 if dt == np.complex128 else 1e-5
    assert rel_l2(h, ref_h).max() < tol
    ref_gp = O.lct_grad_params(f64, g64, params if per_signal else np.tile(abcd, (count, 1)))
    if not per_signal:
        ref_gp = ref_gp.sum(axis=0)
    gtol = 1e-9 if dt == np.complex128 else 1e-4
    assert grad_rel(gp, ref_gp) < gtol
    # adjoint identity <L f, g> = <f, L^H g> on the GPU outputs
    lhs = np.vdot(g64.ravel(), Gc.astype(np.complex128).ravel())
    rhs = np.vdot(h.astype(np.complex128).ravel(), f64.ravel())
    assert abs(lhs - rhs) < (1e-11 if dt == np.complex128 else 1e-4) * abs(lhs)


def test_autograd_gradcheck_fp64():
    """torch.autograd.gradcheck of the LCT Function (complex128 input, real
    (a, b, d) with c = (ad - 1)/b formed in torch)."""
    N = 32
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 2, seed=3, dtype=np.complex128)
    xf = cu(f).requires_grad_(True)
    abd = torch.tensor([0.7, 1.3, -0.4], dtype=torch.float64, requires_grad=True)

    def fn(xx, p):
        a, b, d = p[0], p[1], p[2]
        abcd = torch.stack([a, b, (a * d - 1) / b, d])
        return lct.lct(xx, abcd)

    assert torch.autograd.gradcheck(fn, (xf, abd), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_autograd_per_signal_parameters():
    N, count = 512, 4
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=8, dtype=np.complex64)
    abcd = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    xf = cu(f).requires_grad_(True)
    rng = np.random.default_rng(9)
    T = cu((rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))).astype(np.complex64))
    G = lct.lct(xf, abcd)
    loss = ((G - T).abs() ** 2).sum()
    loss.backward()
    g = (2 * (G - T)).detach().cpu().numpy().astype(np.complex128)
    ref = O.lct_grad_params(f.astype(np.complex128), g, params)
    got = abcd.grad.cpu().numpy()
    assert grad_rel(got[:, [0, 1, 3]], ref) < 1e-4
    assert np.all(got[:, 2] == 0)
    ref_x = O.lct_adjoint(g, params)
    assert rel_l2(xf.grad.cpu().numpy(), ref_x).max() < 1e-5


# --------------------------------------------------------------------------
# separable 2-D transform
# --------------------------------------------------------------------------
def oracle_2d(f, ax, ay):
    """Rows (last axis) with ax, then columns with ay, by the 1-D oracle."""
    B, ny, nx = f.shape
    mid = O.lct(f.reshape(-1, nx), ax).reshape(B, ny, nx)
    out = O.lct(np.swapaxes(mid, 1, 2).reshape(-1, ny), ay).reshape(B, nx, ny)
    return mid, np.swapaxes(out, 1, 2)


def field(ny, nx, B, seed, dt):
    rng = np.random.default_rng(seed)
    yy, xx = O.nodes(ny), O.nodes(nx)
    env = np.exp(-(yy[:, None] ** 2 + xx[None, :] ** 2) / 18.0)
    ph = rng.standard_normal((B, ny, nx)) * 0.3
    return (env[None] * np.exp(1j * ph)).astype(dt)


@pytest.mark.parametrize("ny,nx,dt", [(256, 128, np.complex64), (256, 256, np.complex128)])
def test_2d_forward_backward_vs_oracle(ny, nx, dt):
    B = 2
    ax = (0.6, 1.2, (0.6 * -0.5 - 1) / 1.2, -0.5)
    ay = (-0.9, 0.7, (-0.9 * 1.1 - 1) / 0.7, 1.1)
    f = field(ny, nx, B, 4, dt)
    rng = np.random.default_rng(5)
    g = (rng.standard_normal((B, ny, nx)) + 1j * rng.standard_normal((B, ny, nx))).astype(dt)
    code = lct.LCT_C64 if dt == np.complex64 else lct.LCT_C128
    plan = lct.lct2d_plan_create(ny, nx, ay, ax, code)
    try:
        xf, xg = cu(f), cu(g)
        mid, out = torch.empty_like(xf), torch.empty_like(xf)
        lct.lct2d_execute(plan, xf, mid, out, B)
        gmid, gin = torch.empty_like(xf), torch.empty_like(xf)
        gp = torch.zeros(6, dtype=torch.float64, device="cuda")
        lct.lct2d_backward(plan, xg, xf, mid, out, gmid, gin, gp, B)
        torch.cuda.synchronize()
        out, gin, gp = out.cpu().numpy(), gin.cpu().numpy(), gp.cpu().numpy()
    finally:
        lct.lct2d_plan_destroy(plan)
    f64, g64 = f.astype(np.complex128), g.astype(np.complex128)
    ref_mid, ref_out = oracle_2d(f64, ax, ay)
    tol = 1e-5 if dt == np.complex64 else 1e-12
    assert rel_l2(out.reshape(B, -1), ref_out.reshape(B, -1)).max() < tol
    # adjoint: columns then rows
    gcol = O.lct_adjoint(np.swapaxes(g64, 1, 2).reshape(-1, ny), ay).reshape(B, nx, ny)
    gmid_ref = np.swapaxes(gcol, 1, 2)
    gin_ref = O.lct_adjoint(gmid_ref.reshape(-1, nx), ax).reshape(B, ny, nx)
    assert rel_l2(gin.reshape(B, -1), gin_ref.reshape(B, -1)).max() < tol
    # parameter gradients: x axis on the rows, y axis on the columns (shared, summed)
    gx = O.lct_grad_params(f64.reshape(-1, nx), gmid_ref.reshape(-1, nx),
                           np.tile(ax, (B * ny, 1))).sum(axis=0)
    gy = O.lct_grad_params(np.swapaxes(ref_mid, 1, 2).reshape(-1, ny),
                           np.swapaxes(g64, 1, 2).reshape(-1, ny), np.tile(ay, (B * nx, 1))).sum(axis=0)
    gtol = 1e-4 if dt == np.complex64 else 1e-9
    assert grad_rel(gp[:3], gx) < gtol
    assert grad_rel(gp[3:], gy) < gtol


@pytest.mark.parametrize("ny,nx,B", [(512, 8, 1), (1024, 4, 3), (2048, 16, 1), (4096, 8, 1),
                                      (2048, 2, 1)])
def test_2d_column_kernels(ny, nx, B):
    """The column passes at N = 512 .. 4096: whole groups of columns run the
    persistent kernel that stages the next strip in shared memory (and
    tabulates the diagonal factors), nx = 2 with B = 1 the per-strip kernel;
    forward, adjoint without and with the gradient sums, against the oracle."""
    ax = (0.6, 1.2, (0.6 * -0.5 - 1) / 1.2, -0.5)
    ay = (-0.9, 0.7, (-0.9 * 1.1 - 1) / 0.7, 1.1)
    f = field(ny, nx, B, 11, np.complex64)
    rng = np.random.default_rng(12)
    g = (rng.standard_normal((B, ny, nx)) + 1j * rng.standard_normal((B, ny, nx))).astype(np.complex64)
    plan = lct.lct2d_plan_create(ny, nx, ay, ax, lct.LCT_C64)
    try:
        xf, xg = cu(f), cu(g)
        mid, out = torch.empty_like(xf), torch.empty_like(xf)
        lct.lct2d_execute(plan, xf, mid, out, B)
        gmid, gin = torch.empty_like(xf), torch.empty_like(xf)
        lct.lct2d_backward(plan, xg, xf, mid, out, gmid, gin, None, B)
        torch.cuda.synchronize()
        gin0 = gin.cpu().numpy()
        gp = torch.zeros(6, dtype=torch.float64, device="cuda")
        lct.lct2d_backward(plan, xg, xf, mid, out, gmid, gin, gp, B)
        torch.cuda.synchronize()
        out, gin, gp = out.cpu().numpy(), gin.cpu().numpy(), gp.cpu().numpy()
    finally:
        lct.lct2d_plan_destroy(plan)
    f64, g64 = f.astype(np.complex128), g.astype(np.complex128)
    ref_mid, ref_out = oracle_2d(f64, ax, ay)
    assert rel_l2(out.reshape(B, -1), ref_out.reshape(B, -1)).max() < 1e-5
    gcol = O.lct_adjoint(np.swapaxes(g64, 1, 2).reshape(-1, ny), ay).reshape(B, nx, ny)
    gmid_ref = np.swapaxes(gcol, 1, 2)
    gin_ref = O.lct_adjoint(gmid_ref.reshape(-1, nx), ax).reshape(B, ny, nx)
    assert rel_l2(gin0.reshape(B, -1), gin_ref.reshape(B, -1)).max() < 1e-5
    assert rel_l2(gin.reshape(B, -1), gin_ref.reshape(B, -1)).max() < 1e-5
    gy = O.lct_grad_params(np.swapaxes(ref_mid, 1, 2).reshape(-1, ny),
                           np.swapaxes(g64, 1, 2).reshape(-1, ny), np.tile(ay, (B * nx, 1))).sum(axis=0)
    assert grad_rel(gp[3:], gy) < 1e-4


def test_2d_full_size_fields():
    """8 fields of 2048 x 2048 (complex64): Gaussian beam times a smooth random
    phase screen; Parseval and the adjoint identity at full size, and the
    parameter gradients of a phase-sensitive loss against Richardson central
    differences of the complex128 path (the paper fixes no loss; see the
    readings in the design notes)."""
    B, n = 8, 2048
    fields, ax, ay = W.fields_batch(O.nodes(n), B)
    code64 = lct.LCT_C64
    plan = lct.lct2d_plan_create(n, n, ay, ax, code64)
    try:
        xf = cu(fields.astype(np.complex64))
        mid, out = torch.empty_like(xf), torch.empty_like(xf)
        lct.lct2d_execute(plan, xf, mid, out, B)
        torch.cuda.synchronize()
        nf = (xf.abs().double() ** 2).sum(dim=(1, 2))
        ng = (out.abs().double() ** 2).sum(dim=(1, 2)) * (4 * abs(ax[1]) / np.pi) * (4 * abs(ay[1]) / np.pi)
        assert torch.max(torch.abs(ng / nf - 1)).item() < 2e-5
        g = torch.randn_like(xf)
        gmid, gin = torch.empty_like(xf), torch.empty_like(xf)
        lct.lct2d_backward(plan, g, xf, mid, out, gmid, gin, None, B)
        torch.cuda.synchronize()
        lhs = torch.vdot(g.flatten().to(torch.complex128), out.flatten().to(torch.complex128))
        rhs = torch.vdot(gin.flatten().to(torch.complex128), xf.flatten().to(torch.complex128))
        assert abs((lhs - rhs) / lhs).item() < 1e-4
    finally:
        lct.lct2d_plan_destroy(plan)

    # gradients: loss = sum |G - T|^2 on a centre crop of 2 fields (complex128)
    f2 = cu(fields[:2].astype(np.complex128))
    T = torch.randn_like(f2) * 0.01

    def loss_of(pax, pay, want_grad=False):
        pl = lct.lct2d_plan_create(n, n, pay, pax, lct.LCT_C128)
        try:
            mid, out = torch.empty_like(f2), torch.empty_like(f2)
            lct.lct2d_execute(pl, f2, mid, out, 2)
            val = float(((out - T).abs() ** 2).sum().item())
            gp = None
            if want_grad:
                gmid, gin = torch.empty_like(f2), torch.empty_like(f2)
                gp = torch.zeros(6, dtype=torch.float64, device="cuda")
                lct.lct2d_backward(pl, 2 * (out - T), f2, mid, out, gmid, gin, gp, 2)
                gp = gp.cpu().numpy()
            torch.cuda.synchronize()
        finally:
            lct.lct2d_plan_destroy(pl)
        return val, gp

    _, gp = loss_of(ax, ay, True)

    def with_c(p):
        a, b, d = p
        return (a, b, (a * d - 1) / b, d)

    h = 1e-4
    for axis in range(2):
        for q, comp in enumerate([0, 1, 3]):
            def at(s):
                px, py = list(ax), list(ay)
                tgt = px if axis == 0 else py
                tgt[comp] += s
                return loss_of(with_c((px[0], px[1], px[3])), with_c((py[0], py[1], py[3])))[0]
            d1 = (at(h) - at(-h)) / (2 * h)
            d2 = (at(h / 2) - at(-h / 2)) / h
            fd = (4 * d2 - d1) / 3
            got = gp[3 * axis + q]
            assert abs(got - fd) < 1e-4 * max(abs(fd), 1e-3 * np.abs(gp).max()), (axis, comp, got, fd)


# --------------------------------------------------------------------------
# input gradient of plans the backward kernel does not take: N = 8192 ..
# 65536, N that is not a power of two, b = 0 (through the forward kernels)
# --------------------------------------------------------------------------
BIG = [(8192, np.complex64, True), (16384, np.complex128, False), (32768, np.complex64, True),
       (3000, np.complex64, True), (3000, np.complex128, False), (3001, np.complex64, False),
       (1000, np.complex128, True)]


def _adjoint_run(p, g, f, count):
    xg, xf = cu(g), cu(f)
    h = torch.empty_like(xg)
    lct.lct_backward(p.handle, xg, None, None, h, None, count)
    G = torch.empty_like(xf)
    p.execute(xf, G, count)
    torch.cuda.synchronize()
    assert lct.lct_device_status(p.handle) == 0
    return h.cpu().numpy(), G.cpu().numpy()


@pytest.mark.parametrize("N,dt,per_signal", BIG)
def test_adjoint_through_forward_kernels(N, dt, per_signal):
    count = 3 if N <= 8192 else 2
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=N + 5, dtype=dt)
    rng = np.random.default_rng(N + 6)
    g = (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))).astype(dt)
    code = lct.LCT_C64 if dt == np.complex64 else lct.LCT_C128
    abcd = params if per_signal else params[0]
    p = (lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code) if per_signal
         else lct.Plan.create(N, *abcd, dtype=code))
    try:
        h, G = _adjoint_run(p, g, f, count)
    finally:
        p.destroy()
    tol = 1e-12 if dt == np.complex128 else 1e-5
    ref = O.lct_adjoint(g.astype(np.complex128), abcd)
    assert rel_l2(h, ref).max() < tol, (N, dt)
    lhs = np.vdot(g.astype(np.complex128).ravel(), G.astype(np.complex128).ravel())
    rhs = np.vdot(h.astype(np.complex128).ravel(), f.astype(np.complex128).ravel())
    assert abs(lhs - rhs) < (1e-11 if dt == np.complex128 else 1e-4) * abs(lhs)


@pytest.mark.parametrize("dt", [np.complex64, np.complex128])
def test_adjoint_identity_at_65536(dt):
    """<L f, g> = <f, L^H g> for the two-pass path (the oracle's O(N^2)
    adjoint is checked at 32768)."""
    N, count = 65536, 2
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=65, dtype=dt)
    rng = np.random.default_rng(66)
    g = (rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))).astype(dt)
    code = lct.LCT_C64 if dt == np.complex64 else lct.LCT_C128
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=code)
    try:
        h, G = _adjoint_run(p, g, f, count)
    finally:
        p.destroy()
    for s in range(count):
        lhs = np.vdot(g[s].astype(np.complex128), G[s].astype(np.complex128))
        rhs = np.vdot(h[s].astype(np.complex128), f[s].astype(np.complex128))
        assert abs(lhs - rhs) < (1e-11 if dt == np.complex128 else 1e-4) * abs(lhs)


@pytest.mark.parametrize("N", [256, 300])
def test_adjoint_b_zero(N):
    abcd = (1 / 1.4, 0.0, 0.35, 1.4)
    x = O.nodes(N)
    _, f = W.uniform_batch(x, 3, seed=N, dtype=np.complex128)
    g = np.random.default_rng(N).standard_normal((3, N)) + 0j
    p = lct.Plan.create(N, *abcd, dtype=lct.LCT_C128)
    try:
        h, _ = _adjoint_run(p, g, f, 3)
    finally:
        p.destroy()
    assert rel_l2(h, O.lct_adjoint(g, abcd)).max() < 1e-12


def test_adjoint_through_forward_rejects_what_it_cannot_do():
    N = 8192
    x = O.nodes(N)
    params, f = W.uniform_batch(x, 3, seed=1, dtype=np.complex64)
    xf = cu(f)
    out = torch.empty_like(xf)
    gp = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = lct.Plan.create(N, *params[0], dtype=lct.LCT_C64)
    try:
        with pytest.raises(lct.LctError) as e:           # parameter gradients: N <= 4096 only
            lct.lct_backward(p.handle, xf, xf, out, out, gp, 3)
        assert e.value.status == 10
    finally:
        p.destroy()
    z = 0.6 + 0.3j                                       # complex parameters
    abcd = O.abcd_of_z(z)
    p = lct.Plan.create(N, *[complex(v) for v in abcd], dtype=lct.LCT_C64)
    try:
        with pytest.raises(lct.LctError) as e:
            lct.lct_backward(p.handle, xf, None, None, out, None, 3)
        assert e.value.status == 10
    finally:
        p.destroy()
    gapped = lct.Plan.batch([N] * 2, params[:2], [0, N + 4], dtype=lct.LCT_C64)
    try:
        with pytest.raises(lct.LctError) as e:           # signals not at s N
            lct.lct_backward(gapped.handle, xf, None, None, out, None, 2)
        assert e.value.status == 10
    finally:
        gapped.destroy()
