"""Entry points called from several host threads at once, through the C ABI.

The kernel launchers cache per-device launch configurations (resident CTAs
per multiprocessor, shared-memory opt-ins) on their first launch; the
library serialises host-side submission so that concurrent first launches
are safe.  This file is collected before the other GPU tests of a session,
so these are the first launches of the process: eight threads start
together on their own streams, each on a different kernel family (bulk-copy
and paired fused variants, the persistent two-pass and ragged kernels, the
tcgen05 split path, the 2-D column kernel, the backward kernel and the
fractional transform through the nested lct_execute), and every result must
equal, bit for bit, the same work run afterwards on one thread.
"""
import threading

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0912_1379_gb300 as lct  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lct.build()
    torch.cuda.set_device(0)


def _batch_plan(N, count, seed, variant=None, precision=None):
    x = O.nodes(N)
    params, f = W.uniform_batch(x, count, seed=seed, dtype=np.complex64)
    p = lct.Plan.batch([N] * count, params, np.arange(count) * N, dtype=lct.LCT_C64)
    if variant is not None:
        p.set_variant(variant)
    if precision is not None:
        p.set_precision(precision)
    return p, torch.from_numpy(f.reshape(-1).copy()).cuda(), count


def _jobs(keep):
    """(name, inputs, run(out, stream)) for every kernel family; plans and
    buffers are appended to `keep` for clean-up."""
    jobs = []

    def plan_job(name, N, count, seed, variant=None, precision=None):
        p, x, c = _batch_plan(N, count, seed, variant, precision)
        keep.append(p)
        jobs.append((name, x, lambda out, s, p=p, x=x, c=c: lct.lct_execute(p.handle, x, out, c, s), p))

    plan_job("bulk-copy fused (variant 1)", 4096, 64, 501, variant=1)
    plan_job("paired fused (variant 3)", 4096, 64, 502, variant=3)
    plan_job("two-pass (variant 7)", 65536, 6, 503, variant=7)
    plan_job("tcgen05 split BF16", 4096, 32, 504, precision=lct.LCT_PREC_SPLIT_BF16)

    # ragged batch in one persistent launch
    Ns = [8192, 1024, 256, 64, 8192, 4096]
    rng = np.random.default_rng(505)
    abcds, sigs = [], []
    for N in Ns:
        params, f = W.uniform_batch(O.nodes(N), 1, seed=int(rng.integers(1 << 30)), dtype=np.complex64)
        abcds.append(params[0])
        sigs.append(f[0])
    offs = np.concatenate([[0], np.cumsum(Ns)[:-1]])
    pr = lct.Plan.batch(Ns, np.array(abcds), offs, dtype=lct.LCT_C64).set_variant(9)
    keep.append(pr)
    xr = torch.from_numpy(np.concatenate(sigs)).cuda()
    jobs.append(("ragged persistent (variant 9)", xr,
                 lambda out, s: lct.lct_execute(pr.handle, xr, out, len(Ns), s), pr))

    # separable 2-D transform (row kernel + interleaved-column kernel)
    n2, b2 = 256, 2
    ay = (0.4, 1.2, (0.4 * 0.5 - 1) / 1.2, 0.5)
    ax = (1.1, -0.7, (1.1 * 0.3 - 1) / -0.7, 0.3)
    p2 = lct.lct2d_plan_create(n2, n2, ay, ax, lct.LCT_C64)
    keep.append(("2d", p2))
    f2 = (rng.standard_normal((b2, n2, n2)) + 1j * rng.standard_normal((b2, n2, n2))).astype(np.complex64)
    x2 = torch.from_numpy(f2.reshape(-1).copy()).cuda()
    mid2 = torch.empty_like(x2)
    jobs.append(("2-D transform", x2, lambda out, s: lct.lct2d_execute(p2, x2, mid2, out, b2, s), None))

    # backward (adjoint kernel) of a uniform plan
    pb, xb, cb = _batch_plan(1024, 16, 506)
    keep.append(pb)
    fwd = torch.empty_like(xb)
    pb.execute(xb, fwd, cb)
    torch.cuda.synchronize()
    jobs.append(("backward", xb,
                 lambda out, s: lct.lct_backward(pb.handle, xb, xb, fwd, out, None, cb, s), pb))

    # fractional transform (runs lct_execute inside the entry point)
    _, ff = W.uniform_batch(O.nodes(4096), 16, seed=507, dtype=np.complex64)
    xf = torch.from_numpy(ff.reshape(-1).copy()).cuda()
    jobs.append(("fractional transform", xf,
                 lambda out, s: lct.frft_execute(4096, 0.8 * np.exp(0.7j), xf, out, 16, lct.LCT_C64, s), None))
    return jobs


def test_concurrent_first_launches_match_one_thread():
    keep = []
    try:
        jobs = _jobs(keep)
        torch.cuda.synchronize()
        outs = [torch.zeros_like(x) for _, x, _, _ in jobs]
        streams = [torch.cuda.Stream() for _ in jobs]
        start = threading.Barrier(len(jobs))
        errors = []

        def worker(k):
            try:
                start.wait(timeout=60)
                for _ in range(2):
                    jobs[k][2](outs[k], streams[k])
            except Exception as e:                       # reported after the join
                errors.append((jobs[k][0], repr(e)))

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(jobs))]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=300)
        assert not any(t.is_alive() for t in threads), "a thread did not finish"
        torch.cuda.synchronize()
        assert not errors, errors
        for name, _, _, p in jobs:
            if p is not None:
                assert lct.lct_device_status(p.handle) == 0, name
        # the same work on one thread, one stream
        for k, (name, x, run, _) in enumerate(jobs):
            ref = torch.zeros_like(x)
            run(ref, None)
            torch.cuda.synchronize()
            assert torch.equal(outs[k], ref), name
            assert torch.isfinite(torch.view_as_real(ref)).all(), name
            assert ref.abs().max().item() > 0, name
    finally:
        torch.cuda.synchronize()
        for item in keep:
            if isinstance(item, tuple):
                lct.lct2d_plan_destroy(item[1])
            else:
                item.destroy()
