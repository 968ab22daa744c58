"""Host checks of the tcgen05 descriptor encoders (umma_desc.h) used by the
tensor-core kernels, before anything runs on a GPU.

* shared-memory descriptor: start address, LBO and SBO (each >> 4, 14 bits)
  at bits 0, 16 and 32, the version 1 at bit 46, every other bit zero
  (no swizzle, base offset 0, LBO mode 0);
* instruction descriptor: F32 accumulator at bit 4, A and B formats at bits
  7 and 10, N >> 3 at bit 17, M >> 4 at bit 24, nothing else;
* tile layout: the offset the kernels store element (row, k) at is the
  address the descriptor of MMA k-step ks = k // 8 reads it from (start
  advanced by two core matrices per step), so the product sees the tile the
  kernel wrote.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("umma") / "umma_desc_check")
    src = os.path.join(ROOT, "tests", "c", "umma_desc_check.cpp")
    inc = os.path.join(ROOT, "paper_0912_1379_gb300", "csrc")
    r = subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", inc, src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return [ln.split() for ln in out.splitlines()]


def field(v, lo, width):
    return (v >> lo) & ((1 << width) - 1)


def test_smem_descriptor_fields(lines):
    rows = [ln for ln in lines if ln[0] == "S"]
    assert len(rows) == 45
    for _, s, l, b, d in rows:
        s, l, b, d = int(s), int(l), int(b), int(d)
        assert field(d, 0, 14) == (s >> 4) & 0x3FFF
        assert field(d, 16, 14) == (l >> 4) & 0x3FFF
        assert field(d, 32, 14) == (b >> 4) & 0x3FFF
        assert field(d, 46, 2) == 1
        rest = d & ~((0x3FFF) | (0x3FFF << 16) | (0x3FFF << 32) | (3 << 46))
        assert rest == 0


def test_instruction_descriptor_fields(lines):
    rows = [ln for ln in lines if ln[0] == "I"]
    assert len(rows) == 4
    for _, af, bf, m, n, d in rows:
        af, bf, m, n, d = map(int, (af, bf, m, n, d))
        assert field(d, 4, 2) == 1                 # F32 accumulator
        assert field(d, 7, 3) == af and field(d, 10, 3) == bf
        assert field(d, 15, 2) == 0                # both operands K-major
        assert field(d, 17, 6) == n >> 3
        assert field(d, 24, 5) == m >> 4
        known = (3 << 4) | (7 << 7) | (7 << 10) | (0x3F << 17) | (0x1F << 24)
        assert d & ~known == 0


def test_tile_offsets_match_descriptor_addressing(lines):
    """Element (r, k) of a K-major TF32 tile with 32 K values per row group:
    MMA k-step ks reads row r, K index k' (0..7) at
    start + 256 ks + (r // 8) SBO + (k' // 4) LBO + (r % 8) 16 + (k' % 4) 4
    with LBO = 128 and SBO = 1024."""
    rows = [ln for ln in lines if ln[0] == "O"]
    assert rows
    seen = set()
    for _, r, k, off in rows:
        r, k, off = int(r), int(k), int(off)
        ks, kp = divmod(k, 8)
        addr = 256 * ks + (r // 8) * 1024 + (kp // 4) * 128 + (r % 8) * 16 + (kp % 4) * 4
        assert off == addr
        assert off % 4 == 0 and off not in seen
        seen.add(off)
    assert max(seen) < 256 * 32 * 4            # inside a 256-row, 32-k tile
