"""One reactor's particles shared among processes (Sec. 2.7, the paper's MPI scheme).

Every process holds the whole mesh and its own part of the particles.  After
each step a process's handle holds the deposit of its own particles; the
deposits (electrons, ions) and the charge the walls absorbed are summed over
the processes (one all-reduce), written back, and every process then solves
the same field in its next step.  Newborns are numbered in a residue class
per process (pic_set_id_stride) so ids stay unique.

Marshalling only: the step, the deposit and the solve run in the library;
this module moves the deposit through torch.distributed (gloo with host
arrays, NCCL with device arrays).
"""
from __future__ import annotations

import numpy as np

from . import pic

# deposit layout of one exchange: N_e, N_i ([nz][nr] each), then the 3 wall charges
def _size(h):
    return 2 * h.nz * h.nr + 3


def exchange_deposit(h, group=None) -> None:
    """Sum the deposit of handle h over the process group and write it back."""
    import torch
    import torch.distributed as dist

    ng = h.nz * h.nr
    if dist.get_backend(group) == "nccl":
        buf = torch.empty(_size(h), dtype=torch.float64, device="cuda")
        p = buf.data_ptr()
        st = pic.lib().pic_get_deposit(h.ptr, p, p + 8 * ng, p + 16 * ng, 1)
        pic._check(h, st)
        # the handle's stream is the caller's current stream (pic_init's default)
        dist.all_reduce(buf, group=group)
        pic._check(h, pic.lib().pic_set_deposit(h.ptr, p, p + 8 * ng, p + 16 * ng, 1))
        return
    d = pic.pic_get_deposit(h)
    buf = torch.from_numpy(np.concatenate([d["Ne"].ravel(), d["Ni"].ravel(), d["q"]]))
    dist.all_reduce(buf, group=group)
    a = buf.numpy()
    pic.pic_set_deposit(h, a[:ng], a[ng:2 * ng], a[2 * ng:])


def number_newborns(h, rank: int, world: int, first_free) -> None:
    """Newborns of process `rank` get ids first_free[s] + rank + world k."""
    pic.pic_set_id_stride(h, [int(first_free[0]) + rank, int(first_free[1]) + rank], world)


def step(h, nsteps: int, group=None) -> int:
    """nsteps steps, the deposit exchanged after each; the first non-OK status."""
    first = pic.PIC_OK
    for _ in range(nsteps):
        st = pic.pic_step(h, 1)
        if first == pic.PIC_OK and st != pic.PIC_OK:
            first = st
        exchange_deposit(h, group)
    return first
