"""Slab-decomposed 2D transform over several GPUs (one rank per GPU).

The paper computes its 2D FFT as row FFTs, a global transpose and column FFTs
(Section 5, Fig. 6), and names the multi-card form -- the transpose becoming
an exchange between cards -- as future work (Section 6).  Here each of the G
ranks of a torch.distributed group holds ``rows = ny / G`` consecutive rows of
every [ny][nx] slice and

1. transforms its rows (a 1D batch plan, the library's row kernels),
2. packs, for every rank s, the (rows x w) block of its rows lying in column
   slab s (w = nx / G) into one contiguous chunk (``fft_slab_pack``),
3. exchanges the chunks with one all-to-all (NCCL between GPUs),
4. assembles the received chunks into its column slab [batch][ny][w]
   (``fft_slab_unpack``), and
5. transforms the columns of that slab (a column-only plan).

The result stays distributed by columns: rank s holds columns
[s*w, (s+1)*w) of every transformed slice, in natural [ky][kx] order.  The
only collective is the exchange of step 3; everything else runs in the
library's kernels on the rank's own GPU.  The local steps are supplied by an
``ops`` object, so the same driver runs with the library (``LibraryOps``) or,
in the CPU tests, with stand-ins over gloo.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import fft as _fft


class LibraryOps:
    """The local steps on the rank's GPU through the library."""

    def __init__(self, nx: int, ny: int, batch: int, parts: int, inverse: bool):
        self.rows = ny // parts
        self.row_plan = _fft.Plan(nx, 1, batch * self.rows, inverse=inverse)
        self.col_plan = _fft.ColumnPlan(nx // parts, ny, batch, inverse=inverse)

    def rows_fft(self, x):
        return self.row_plan.execute(x)

    def pack(self, y, parts, batch, rows, nx):
        return _fft.slab_pack(y, parts, batch, rows, nx)

    def unpack(self, recv, parts, batch, rows, w):
        return _fft.slab_unpack(recv, parts, batch, rows, w)

    def cols_fft(self, z):
        return self.col_plan.execute(z)

    def empty_like(self, t):
        return torch.empty_like(t)


class SlabFFT2:
    """Unnormalised 2D DFT (sign -1 forward, +1 inverse) of ``batch``
    [ny][nx] slices distributed by row slabs over ``group``.

    Call with this rank's slab, a complex64 tensor of batch*(ny/G)*nx
    elements laid out [batch][ny/G][nx]; returns this rank's column slab
    [batch][ny][nx/G].  ny and nx must be multiples of G; the local plans
    follow the library's size rules (powers of two)."""

    def __init__(self, nx: int, ny: int, batch: int = 1, inverse: bool = False, group=None, ops=None):
        self.group = group
        self.parts = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        if ny % self.parts or nx % self.parts:
            raise ValueError(f"nx = {nx} and ny = {ny} must be multiples of the {self.parts} ranks")
        self.nx, self.ny, self.batch, self.inverse = int(nx), int(ny), int(batch), bool(inverse)
        self.rows = self.ny // self.parts
        self.w = self.nx // self.parts
        self.ops = ops if ops is not None else LibraryOps(self.nx, self.ny, self.batch, self.parts, self.inverse)

    def __call__(self, x_local):
        G, b, rows, w = self.parts, self.batch, self.rows, self.w
        if x_local.numel() != b * rows * self.nx:
            raise ValueError(f"this rank's slab must hold {b * rows * self.nx} elements")
        y = self.ops.rows_fft(x_local)                      # step 1
        send = self.ops.pack(y, G, b, rows, self.nx)        # step 2: [G][b][rows][w]
        recv = self.ops.empty_like(send)
        if G > 1:  # step 3: one contiguous chunk to and from every rank (real views of the complex data)
            dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=self.group)
        else:
            recv.copy_(send)
        z = self.ops.unpack(recv, G, b, rows, w)            # step 4: [b][ny][w]
        return self.ops.cols_fft(z)                         # step 5
