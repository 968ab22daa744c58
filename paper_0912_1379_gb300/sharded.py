"""Separable 2-D LCT of one field sharded over several GPUs (one process per
GPU, torch.distributed): the fields that do not fit one GPU.

Rank r holds rows [r R, (r + 1) R) of the ny x nx field (R = ny / W, W ranks).
1. The 1-D transform with abcd_x along each of its R rows (lct_execute).
2. lct_transpose: [R][nx] -> [nx][R] = [W][C][R], C = nx / W, so that the
   block for rank q (its C columns) is contiguous.
3. all_to_all_single: rank r receives [W][C][R], block p holding rows
   [p R, (p + 1) R) of its own C columns.
4. lct_transpose with vectors of R samples: [W][C][R] -> [C][W][R] = [C][ny],
   every one of its columns now contiguous.
5. The 1-D transform with abcd_y along each of these C columns.
The result is column-distributed and stored transposed: rank r returns
out[c, y] = G[y, r C + c] for c < C.  Every step on the data is a kernel
of the library or the collective; nothing runs on the host.

row_transform and transpose may be given to run the same exchange with
other implementations of steps 1, 2, 4 and 5 (the multi-rank tests use it to
check the exchange on CPU ranks); by default they are the library's
lct_execute and lct_transpose on the current GPU.
"""
from __future__ import annotations

import numpy as np


def _gpu_rows(x, abcd):
    """1-D LCT along the last axis of the 2-D device tensor x (a new tensor)."""
    import torch
    from . import Plan, dtype_code
    rows, n = x.shape
    code = dtype_code(x.dtype)
    a, b, c, d = [float(v) for v in np.asarray(abcd, dtype=np.float64)]
    out = torch.empty_like(x)
    p = Plan.create(n, a, b, c, d, dtype=code)
    try:
        p.execute(x.contiguous(), out, rows)
    finally:
        # the plan's buffers are freed only after the work queued on the stream
        torch.cuda.current_stream().synchronize()
        p.destroy()
    return out


def _gpu_transpose(x, rows, cols, vec):
    import torch
    from . import dtype_code, lct_transpose
    out = torch.empty_like(x)
    lct_transpose(x.contiguous(), out, rows, cols, vec, 1, dtype_code(x.dtype))
    return out


def lct2d_sharded(field_rows, abcd_x, abcd_y, group=None, row_transform=None, transpose=None):
    """Sharded separable 2-D LCT (see the module docstring).  field_rows:
    this rank's [R, nx] rows of the field (complex tensor).  Returns this
    rank's [C, ny] slab of the output, out[c, y] = G[y, rank C + c]."""
    import torch
    import torch.distributed as dist
    row_transform = row_transform or _gpu_rows
    transpose = transpose or _gpu_transpose
    distributed = dist.is_available() and dist.is_initialized()
    W = dist.get_world_size(group) if distributed else 1
    R, nx = field_rows.shape
    if nx % W:
        raise ValueError("nx must be a multiple of the number of ranks")
    C, ny = nx // W, R * W
    a = row_transform(field_rows, abcd_x)                 # [R][nx]
    send = transpose(a, R, nx, 1).reshape(W, C * R)       # [nx][R] = [W][C][R]
    if W > 1:
        # one block per destination along dim 0; complex samples travel as
        # (re, im) pairs, which every backend takes
        recv = torch.empty_like(send)
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=group)
    else:
        recv = send
    cols = transpose(recv.reshape(W * C, R), W, C, R).reshape(C, ny)   # [C][W][R] = [C][ny]
    return row_transform(cols, abcd_y)
