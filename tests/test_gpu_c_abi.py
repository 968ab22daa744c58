"""A C99 program drives the library through the C ABI alone (cudaMalloc'd
buffers, lct_execute on the default stream); its complex128 output matches
the FP64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import paper_0912_1379_gb300 as lct
from conftest import rel_l2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_c_program_executes_through_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = lct.build()
    libdir = os.path.dirname(lib)
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "abi_device")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c", "abi_device.c"),
           "-o", exe, "-L", libdir, "-llct", "-Wl,-rpath," + libdir,
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64"),
           "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = str(tmp_path / "result.bin")
    r = subprocess.run([exe, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout + r.stderr)
    raw = np.fromfile(out, dtype=np.float64)
    N, count = int(raw[0]), int(raw[1])
    abcd = raw[2:6]
    data = raw[6:].view(np.complex128)
    f = data[:N * count].reshape(count, N)
    g = data[N * count:].reshape(count, N)
    ref = O.lct(f, abcd)
    assert rel_l2(g, ref).max() < 1e-12
