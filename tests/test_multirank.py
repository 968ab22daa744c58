"""Multi-rank path on the CPU: two gloo ranks (world size 2) shard batches
with lct_partition (no collective on the data path) and, for shared
parameters, sum their parameter gradients with one all-reduce.  The FP64
oracle stands in for each rank's GPU, so the host logic -- partition
agreement, exact coverage, load balance, gradient reduction -- is tested
without a device."""
import os
import socket
import traceback

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_ragged():
    import oracle as O
    import workloads as W
    r = W.ragged_plan(count_scale=0.002, log2n_max=8)
    Ns = (1 << r["log2n"]).astype(np.int64)
    abcd = r["abcd"].copy()
    for s in np.nonzero(r["kind"] == W.KIND_FRFT)[0]:
        abcd[s] = O.abcd_of_z(r["z"][s])
    sigs = [W.ragged_signal(O.nodes(int(N)), r["s"][s], r["q"][s], r["rng"], dtype=np.complex128)
            for s, N in enumerate(Ns)]
    return Ns, abcd, sigs


def _worker(rank, port, errq):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=WORLD)
        import oracle as O
        import paper_0912_1379_gb300 as lct

        # 1. ragged batch: every rank derives the same assignment
        Ns, abcd, sigs = _small_ragged()
        owner, load = lct.lct_partition(Ns, WORLD, abcd)
        mine = torch.from_numpy(owner.astype(np.int64))
        all_owners = [torch.zeros_like(mine) for _ in range(WORLD)]
        dist.all_gather(all_owners, mine)
        assert all(torch.equal(all_owners[0], o) for o in all_owners)
        # loads within the largest single cost of each other (LPT bound)
        cost = np.where(abcd[:, 1] == 0, Ns, Ns * np.log2(Ns))
        assert load.max() - load.min() <= cost.max() + 1e-9
        assert abs(load.sum() - cost.sum()) < 1e-6 * cost.sum()
        # each rank transforms its own signals; rank 0 checks the union
        local = {int(s): O.lct(sigs[s], abcd[s]) for s in np.nonzero(owner == rank)[0]}
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, local)
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not set(part) & set(merged)            # no signal twice
                merged.update(part)
            assert sorted(merged) == list(range(len(Ns)))      # every signal once
            for s in range(len(Ns)):
                ref = O.lct(sigs[s], abcd[s])
                assert np.array_equal(merged[s], ref)

        # 2. shared parameters over a uniform batch: gradients summed by one all-reduce
        import workloads as W
        N, count = 128, 6
        x = O.nodes(N)
        params, f = W.uniform_batch(x, count, seed=21, dtype=np.complex128)
        abcd1 = params[0]
        rng = np.random.default_rng(5)
        g = rng.standard_normal((count, N)) + 1j * rng.standard_normal((count, N))
        owner2, _ = lct.lct_partition(np.full(count, N), WORLD)
        sel = np.nonzero(owner2 == rank)[0]
        part = np.zeros(3)
        if len(sel):
            part = O.lct_grad_params(f[sel], g[sel], abcd1).sum(axis=0)
        t = torch.from_numpy(part)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        full = O.lct_grad_params(f, g, abcd1).sum(axis=0)
        assert np.allclose(t.numpy(), full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
        dist.barrier()
        dist.destroy_process_group()
    except Exception:
        errq.put((rank, traceback.format_exc()))
        raise


def test_two_ranks_shard_and_reduce():
    import oracle as O
    import paper_0912_1379_gb300 as lct
    lct.build()
    O.build()
    ctx = mp.get_context("spawn")
    errq = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, errq)) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        if p.is_alive():
            p.kill()
    errors = []
    while not errq.empty():
        errors.append(errq.get())
    assert not errors, errors
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]


def test_partition_properties():
    """Host-only checks of lct_partition: determinism, one owner per signal,
    b = 0 signals cost N, ties keep the lowest rank, bad arguments."""
    import paper_0912_1379_gb300 as lct
    lct.build()
    Ns = np.array([4096, 64, 65536, 1024, 1024, 256, 32768, 16], dtype=np.int64)
    own, load = lct.lct_partition(Ns, 3)
    own2, load2 = lct.lct_partition(Ns, 3)
    assert np.array_equal(own, own2) and np.array_equal(load, load2)
    cost = Ns * np.log2(Ns)
    for r in range(3):
        assert np.isclose(load[r], cost[own == r].sum())
    assert own[np.argmax(Ns)] == 0                      # the largest signal goes first, to rank 0
    # world 1: everything on rank 0
    own1, load1 = lct.lct_partition(Ns, 1)
    assert np.all(own1 == 0) and np.isclose(load1[0], cost.sum())
    # b = 0 signals cost N
    abcd = np.array([[1.0, 2.0, 0.5, 2.0]] * len(Ns))
    abcd[2] = [0.5, 0.0, 1.0, 2.0]
    _, loadb = lct.lct_partition(Ns, 1, abcd)
    assert np.isclose(loadb[0], cost.sum() - cost[2] + Ns[2])
    with pytest.raises(lct.LctError):
        lct.lct_partition(np.array([70000]), 2)          # above 65536
    with pytest.raises(lct.LctError):
        lct.lct_partition(Ns, 0)


# --------------------------------------------------------------------------
# one 2-D field sharded over two ranks: rows, all-to-all, columns
# --------------------------------------------------------------------------
def _field(ny, nx, seed=7):
    import oracle as O
    rng = np.random.default_rng(seed)
    y, x = O.nodes(ny), O.nodes(nx)
    env = np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / 18.0)
    return env * (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx)))


AX = (0.6, 1.3, (0.6 * -0.4 - 1) / 1.3, -0.4)
AY = (-1.1, -0.7, (-1.1 * 0.9 - 1) / -0.7, 0.9)


def _cpu_rows(x, abcd):
    """Stand-in for the GPU row transform on a CPU rank: the FP64 oracle."""
    import oracle as O
    return torch.from_numpy(O.lct(x.numpy(), abcd))


def _cpu_transpose(x, rows, cols, vec):
    """Stand-in for lct_transpose on a CPU rank (same memory contract)."""
    a = x.numpy().reshape(rows, cols, vec).transpose(1, 0, 2)
    return torch.from_numpy(np.ascontiguousarray(a).reshape(x.shape))


def _sharded_worker(rank, port, errq):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=WORLD)
        import oracle as O
        from paper_0912_1379_gb300.sharded import lct2d_sharded
        ny, nx = 64, 128
        f = _field(ny, nx)
        R, C = ny // WORLD, nx // WORLD
        mine = torch.from_numpy(np.ascontiguousarray(f[rank * R:(rank + 1) * R]))
        out = lct2d_sharded(mine, AX, AY, row_transform=_cpu_rows, transpose=_cpu_transpose)
        assert tuple(out.shape) == (C, ny)
        parts = [torch.zeros_like(torch.view_as_real(out)) for _ in range(WORLD)]
        dist.all_gather(parts, torch.view_as_real(out.contiguous()))
        if rank == 0:
            got = np.concatenate([torch.view_as_complex(p).numpy() for p in parts])   # [nx][ny]
            rows = O.lct(f, AX)                     # 1-D transform of every row (along x)
            ref = O.lct(np.ascontiguousarray(rows.T), AY)   # then every column (along y), transposed
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err < 1e-13, err
        dist.barrier()
        dist.destroy_process_group()
    except Exception:
        errq.put((rank, traceback.format_exc()))
        raise


def test_two_ranks_sharded_2d_field():
    """The exchange of lct2d_sharded (row transform, transpose, all-to-all,
    transpose, column transform) on two gloo ranks, with the oracle and a
    host transpose standing in for each rank's GPU kernels; the gathered
    result equals the oracle's separable 2-D transform of the whole field."""
    import oracle as O
    import paper_0912_1379_gb300 as lct
    lct.build()
    O.build()
    ctx = mp.get_context("spawn")
    errq = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, port, errq)) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        if p.is_alive():
            p.kill()
    errors = []
    while not errq.empty():
        errors.append(errq.get())
    assert not errors, errors
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
