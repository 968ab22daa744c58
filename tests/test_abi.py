"""The C-ABI library on the CPU: it loads, exports every declared symbol, and
its host-side logic (validation, grids, exact phase constants) is right.
No compute call is made here (no GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import paper_0912_1379_gb300 as lct
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    lct.build()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "lct_execute" in names and "frft_execute" in names and "lct_plan_create" in names
    lib = ctypes.CDLL(lct.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_only_the_c_abi():
    """Hidden visibility: the internal launchers and host helpers are not
    exported; every exported C (unmangled) function is declared in include/."""
    lib = ctypes.CDLL(lct.library_path())
    for internal in ("lct_launch_fused", "lct_launch_twopass", "lct_launch_gen",
                     "lct_twiddle_table", "lct_make_desc_host"):
        assert not hasattr(lib, internal), internal
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", lct.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines()
                if len(ln.split()) == 3 and ln.split()[1] == "T"}
    c_names = {n for n in exported if not n.startswith("_")}
    assert c_names == set(declared_functions()), sorted(c_names ^ set(declared_functions()))


def test_status_strings():
    for s in range(len(lct.STATUS)):
        assert lct.lct_status_string(s) not in ("", "unknown status")


def test_input_grid_matches_oracle_nodes():
    for N in [2, 16, 1024, 65536]:
        x = lct.lct_input_grid(N)
        assert np.allclose(x, O.nodes(N), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("N", [0, 1, 9000, 65535, 131072, -4])
def test_bad_N(N):
    with pytest.raises(lct.LctError) as e:
        lct.lct_plan_create(N, 1.0, 2.0, 0.5, 2.0)
    assert e.value.status == 2


def test_not_symplectic_and_dtype():
    with pytest.raises(lct.LctError) as e:
        lct.lct_plan_create(64, 1.0, 2.0, 0.6, 2.0)
    assert e.value.status == 3
    with pytest.raises(lct.LctError) as e:
        lct.lct_plan_create(64, 1.0, 2.0, 0.5, 2.0, dtype=7)
    assert e.value.status == 4
    with pytest.raises(lct.LctError) as e:
        lct.lct_plan_create(64, float("nan"), 2.0, 0.5, 2.0)
    assert e.value.status == 1


def test_execute_validation_without_gpu():
    p = lct.lct_plan_create(64, 1.0, 2.0, 0.5, 2.0)
    try:
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute(p, 0, 0, 1, stream=0)
        assert e.value.status == 1
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute(p, 4, 4, 1, stream=0)          # not 8-byte aligned
        assert e.value.status == 5
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute(p, 64, 64, -1, stream=0)
        assert e.value.status == 1
        lct.lct_execute(p, 64, 64, 0, stream=0)             # batch 0: no-op, no device touched
    finally:
        lct.lct_plan_destroy(p)
    bp = lct.lct_plan_create_batch([64, 64], [[1, 2, 0.5, 2], [0, 1, -1, 0]], [0, 64])
    try:
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute(bp, 64, 64, 3, stream=0)
        assert e.value.status == 1
    finally:
        lct.lct_plan_destroy(bp)


def test_variant_selection_host_only():
    p = lct.lct_plan_create(1024, 1.0, 2.0, 0.5, 2.0)
    try:
        assert lct.lct_plan_get_variant(p) == 11          # measured default schedule at N = 1024
        lct.lct_plan_set_variant(p, 1)
        assert lct.lct_plan_get_variant(p) == 1
        lct.lct_plan_set_variant(p, 7)
        assert lct.lct_plan_get_variant(p) == 7
        lct.lct_plan_set_variant(p, 8)
        assert lct.lct_plan_get_variant(p) == 8
        lct.lct_plan_set_variant(p, 11)
        assert lct.lct_plan_get_variant(p) == 11
        for bad in (12, -1):
            with pytest.raises(lct.LctError) as e:
                lct.lct_plan_set_variant(p, bad)
            assert e.value.status == 1
    finally:
        lct.lct_plan_destroy(p)
    # default: two passes from N = 32768 up, else variant 0
    for N, want in [(16, 0), (32, 10), (256, 10), (512, 11), (2048, 11), (4096, 0), (16384, 0),
                    (32768, 7), (65536, 7)]:
        p = lct.lct_plan_create(N, 1.0, 2.0, 0.5, 2.0)
        try:
            assert lct.lct_plan_get_variant(p) == want
        finally:
            lct.lct_plan_destroy(p)
        # complex128 keeps variant 0 below the two-pass sizes
        p = lct.lct_plan_create(N, 1.0, 2.0, 0.5, 2.0, dtype=lct.LCT_C128)
        try:
            assert lct.lct_plan_get_variant(p) == (7 if N >= 32768 else 0)
        finally:
            lct.lct_plan_destroy(p)


def test_precision_selection_host_only():
    """Tensor-core precisions: complex64, one N in [16, 4096]; b = 0 plans
    (no DFT) accept them at any N; complex128 and ragged plans do not."""
    split = (lct.LCT_PREC_SPLIT_BF16, lct.LCT_PREC_SPLIT_FP16, lct.LCT_PREC_FP16)

    def status(N, abcd, dtype=lct.LCT_C64, prec=lct.LCT_PREC_SPLIT_BF16):
        p = lct.lct_plan_create(N, *abcd, dtype=dtype)
        try:
            lct.lct_plan_set_precision(p, prec)
            return 0
        except lct.LctError as e:
            return e.status
        finally:
            lct.lct_plan_destroy(p)

    gen = (1.0, 2.0, 0.5, 2.0)
    for prec in split:
        for N in (16, 32, 256, 2048, 4096):
            assert status(N, gen, prec=prec) == 0
        for N in (2, 8, 8192, 65536):
            assert status(N, gen, prec=prec) == 10
        assert status(1024, gen, dtype=lct.LCT_C128, prec=prec) == 10
        assert status(65536, (0.5, 0.0, 1.0, 2.0), prec=prec) == 0      # b = 0: diagonal
    assert status(1024, gen, prec=99) == 1
    rag = lct.Plan.batch([64, 128], np.array([gen, gen]), [0, 64], dtype=lct.LCT_C64)
    try:
        with pytest.raises(lct.LctError) as e:
            rag.set_precision(lct.LCT_PREC_SPLIT_FP16)
        assert e.value.status == 10
    finally:
        rag.destroy()


def test_execute_host_validation_without_gpu():
    """Host-buffer execution needs one N and contiguous signals; the checks
    come before any device work."""
    h = np.zeros(4 * 64, dtype=np.complex64)
    gen = np.array([1.0, 2.0, 0.5, 2.0])
    gapped = lct.Plan.batch([64] * 3, np.array([gen] * 3), [0, 70, 140], dtype=lct.LCT_C64)
    ragged = lct.Plan.batch([64, 128], np.array([gen] * 2), [0, 64], dtype=lct.LCT_C64)
    try:
        for plan, count in ((gapped, 3), (ragged, 2)):
            with pytest.raises(lct.LctError) as e:
                plan.execute_host(h.ctypes.data, h.ctypes.data, count, stream=0)
            assert e.value.status == 10
        with pytest.raises(lct.LctError) as e:
            gapped.execute_host(h.ctypes.data, h.ctypes.data, 2, stream=0)   # batch != count
        assert e.value.status == 1
        with pytest.raises(lct.LctError) as e:
            lct.lct_execute_host(gapped.handle, 0, h.ctypes.data, 3, stream=0)
        assert e.value.status == 1
    finally:
        gapped.destroy()
        ragged.destroy()


def test_selftest_timeout_arguments_without_gpu():
    for which, ms in [(2, 1.0), (-1, 1.0), (0, 0.0), (1, 2000.0), (0, float("nan"))]:
        assert lct.lct_selftest_timeout(which, ms, stream=0) == 1


@pytest.mark.parametrize("z", [0.0, 1.5, 2j, complex(float("nan"), 0)])
def test_frft_bad_z(z):
    with pytest.raises(lct.LctError) as e:
        lct.frft_execute(64, z, 64, 64, 1, stream=0)
    assert e.value.status == 1


@pytest.mark.parametrize("abcd", [(1.0, 2.0, 0.5, 2.0), (0.0, 1.0, -1.0, 0.0), (2.0, 0.0, 0.3, 0.5),
                                  (0.3 + 0.1j, 0.5 - 0.7j, None, 1.1 + 0.2j)])
def test_output_grid_matches_oracle(abcd):
    a, b, c, d = abcd
    if c is None:
        c = (a * d - 1) / b
    N = 128
    p = lct.Plan.create(N, a, b, c, d)
    try:
        y, rho = lct.lct_output_grid(p.handle, 0, N)
    finally:
        p.destroy()
    yo = O.output_grid(N, [a, b, c, d])
    f = np.ones(N, dtype=np.complex128)
    _, rho_o = O.lct(f, [a, b, c, d], return_rho=True)
    assert np.allclose(y, yo, rtol=1e-14, atol=1e-13)
    assert np.allclose(rho, rho_o, rtol=1e-12, atol=1e-12)


def _turns_err(q, exact, bits):
    """signed difference (in units of 2^-bits turns) between a fixed-point
    fraction q and an exact mpmath turn count, modulo one turn."""
    import mpmath
    mod = 1 << bits
    e = int(mpmath.floor((exact - mpmath.floor(exact)) * mod + mpmath.mpf(0.5))) % mod
    dlt = (q - e) % mod
    return dlt - mod if dlt >= mod // 2 else dlt


@pytest.mark.parametrize("N,abcd", [(256, (np.cos(0.7), np.sin(0.7), -np.sin(0.7), np.cos(0.7))),
                                    (65536, (1.7, 0.21, (1.7 * -1.3 - 1) / 0.21, -1.3)),
                                    (1024, (1.0, 100.0, 0.0, 1.0)),
                                    (64, (0.3, -1.9, (0.3 * 0.4 - 1) / -1.9, 0.4))])
def test_phase_constants_exact(N, abcd):
    """The 128-bit turn fractions equal the exactly computed phases of the
    FP64 parameters to better than 2^-100 turns (mpmath, 60 digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    a, b, c, d = abcd
    p = lct.lct_plan_create(N, a, b, c, d)
    try:
        in_hi, in_lo, out_hi, out_lo, out_c = lct.lct_plan_phase_turns(p)
    finally:
        lct.lct_plan_destroy(p)
    A, B, D = mpmath.mpf(a), mpmath.mpf(b), mpmath.mpf(d)
    t_in = A * mpmath.pi / (32 * B * N)               # a x^2/(2b) per m^2, in turns
    t_out = B * D / (2 * mpmath.pi * N)               # d y^2/(2b) per m^2, in turns
    assert abs(_turns_err((in_hi << 64) | in_lo, t_in, 128)) < 2 ** 28
    assert abs(_turns_err((out_hi << 64) | out_lo, t_out, 128)) < 2 ** 28
    # output constant: -(N-1)^2/(4N) + arg(dx / sqrt(2 pi i b)) / (2 pi)
    dx = mpmath.pi / mpmath.sqrt(2 * N)
    pre = dx / mpmath.sqrt(2j * mpmath.pi * B)
    t_c = -mpmath.mpf((N - 1) ** 2) / (4 * N) + mpmath.arg(pre) / (2 * mpmath.pi)
    assert abs(_turns_err(out_c, t_c, 64)) < 2 ** 14


# --------------------------------------------------------------------------
# N that is not a power of two (chirp-convolution kernel), host side
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,abcd", [(1000, (1.7, 0.21, (1.7 * -1.3 - 1) / 0.21, -1.3)),
                                    (4095, (0.3, -1.9, (0.3 * 0.4 - 1) / -1.9, 0.4)),
                                    (3, (1.0, 2.0, 0.5, 2.0))])
def test_phase_constants_non_power_of_two(N, abcd):
    """N that is not a power of two (mpmath, 60 digits).  7-smooth N (1000,
    3: the mixed-radix DFT) keeps the direct form: phi_in = a pi/(32 b N),
    phi_out = b d/(2 pi N), and the constant -(N-1)^2/(4N) + arg(dx/sqrt(2 pi
    i b)) turns.  Other N (4095 = 3^2 5 7 13: the chirp convolution) absorb
    the -1/(8N) turns of the convolution split in both chirps, and the
    constant is arg(dx/sqrt(2 pi i b)) alone."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    a, b, c, d = abcd
    p = lct.lct_plan_create(N, a, b, c, d)
    try:
        in_hi, in_lo, out_hi, out_lo, out_c = lct.lct_plan_phase_turns(p)
    finally:
        lct.lct_plan_destroy(p)
    m = N
    for q in (2, 3, 5, 7):
        while m % q == 0:
            m //= q
    smooth = m == 1
    A, B, D = mpmath.mpf(a), mpmath.mpf(b), mpmath.mpf(d)
    shift = 0 if smooth else mpmath.mpf(1) / (8 * N)
    t_in = A * mpmath.pi / (32 * B * N) - shift
    t_out = B * D / (2 * mpmath.pi * N) - shift
    assert abs(_turns_err((in_hi << 64) | in_lo, t_in, 128)) < 2 ** 28
    assert abs(_turns_err((out_hi << 64) | out_lo, t_out, 128)) < 2 ** 28
    dx = mpmath.pi / mpmath.sqrt(2 * N)
    pre = dx / mpmath.sqrt(2j * mpmath.pi * B)
    centre = -mpmath.mpf((N - 1) ** 2 % (4 * N)) / (4 * N) if smooth else 0
    assert abs(_turns_err(out_c, centre + mpmath.arg(pre) / (2 * mpmath.pi), 64)) < 2 ** 14


@pytest.mark.parametrize("N", [3, 100, 4095, 65535])
def test_input_grid_any_n(N):
    assert np.allclose(lct.lct_input_grid(N), O.nodes(N), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,dtype,ok", [(4095, lct.LCT_C128, True), (4097, lct.LCT_C128, False),
                                        (8191, lct.LCT_C64, True), (8193, lct.LCT_C64, False),
                                        (3, lct.LCT_C64, True), (65535, lct.LCT_C64, False),
                                        (1, lct.LCT_C64, False), (65537, lct.LCT_C64, False)])
def test_non_power_of_two_sizes_accepted(N, dtype, ok):
    if ok:
        lct.Plan.create(N, 1.0, 2.0, 0.5, 2.0, dtype=dtype).destroy()
        lct.Plan.batch([N, 64], [(1.0, 2.0, 0.5, 2.0)] * 2, [0, N], dtype=dtype).destroy()
    else:
        with pytest.raises(lct.LctError) as e:
            lct.Plan.create(N, 1.0, 2.0, 0.5, 2.0, dtype=dtype)
        assert e.value.status == 2


def test_non_power_of_two_precision_choices():
    p = lct.Plan.create(1000, 1.0, 2.0, 0.5, 2.0)
    try:
        for prec in (lct.LCT_PREC_PLAIN64, lct.LCT_PREC_PLAIN32, lct.LCT_PREC_SPLIT_BF16):
            with pytest.raises(lct.LctError) as e:
                p.set_precision(prec)
            assert e.value.status == 10
        p.set_precision(lct.LCT_PREC_NATIVE)
    finally:
        p.destroy()


def test_partition_costs_non_power_of_two():
    """A 7-smooth N costs one mixed-radix DFT (N ceil(log2 N)); another N two
    DFTs of M >= 2N - 1 (1001 = 7 11 13: M = 2048)."""
    owner, load = lct.lct_partition([1001, 1024], 2)
    assert sorted(load.tolist()) == [1024 * 10, 2 * 2048 * 11]
    owner, load = lct.lct_partition([1000, 3000], 2)
    assert sorted(load.tolist()) == [1000 * 10, 3000 * 12]


@pytest.mark.parametrize("N,z,dtype,status", [
    (1, 0.5, lct.LCT_C64, 2), (8193, 0.5, lct.LCT_C64, 2), (4097, 0.5, lct.LCT_C128, 2),
    (64, 1.0, lct.LCT_C64, 1), (64, -1.0, lct.LCT_C128, 1), (64, 1.2j, lct.LCT_C64, 1),
    (64, 0.8 + 0.7j, lct.LCT_C64, 1), (64, complex(float("nan"), 0.0), lct.LCT_C64, 1),
    (64, 0.5, 9, 4)])
def test_frft_mehler_validation_without_gpu(N, z, dtype, status):
    """Size, z and dtype are checked before any device call."""
    with pytest.raises(lct.LctError) as e:
        lct.frft_mehler_execute(N, z, 64, 64, 1, dtype=dtype, stream=0)
    assert e.value.status == status


def test_frft_mehler_batch_and_pointers_without_gpu():
    # batch 0 is a no-op after validation; a negative batch or a null
    # pointer is LCT_ERR_ARG, all without a device call
    for N, dtype in [(2, lct.LCT_C64), (8192, lct.LCT_C64), (4096, lct.LCT_C128), (3000, lct.LCT_C64)]:
        lct.frft_mehler_execute(N, 0.3 + 0.4j, 0, 0, 0, dtype=dtype, stream=0)
    for z in [np.exp(0.7j), -0.6j, 0.0]:
        lct.frft_mehler_execute(256, z, 0, 0, 0, stream=0)
    for batch, ptr in [(-1, 64), (1, 0)]:
        with pytest.raises(lct.LctError) as e:
            lct.frft_mehler_execute(64, 0.5, ptr, ptr, batch, stream=0)
        assert e.value.status == 1
