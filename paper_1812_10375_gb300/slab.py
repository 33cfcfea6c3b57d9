"""Y-slab decomposition of one domain over several ranks: the host-side plan.

A domain of ny rows is split into contiguous slabs of rows, one per rank.
One step (Eqs. 1-18, with N energy sub-steps of Eq. 27) of the rows a rank
owns depends on the state (the post-collision populations f* and the
temperature T) of the rows within a fixed distance:

* rho^n and u^n of a row come from f* of the rows within 2 (streaming pulls
  from the adjacent rows; the pseudo-potential force of Eq. 6 reads psi of the
  adjacent rows, which again needs their streamed populations), and from T^n
  within 1 (psi depends on T through the EOS, Eq. 28);
* T^{n+1} of a row comes from T^n within 4 N rows and from rho^n, u^n within
  4 N rows: each of the 4 N RK4 stages at a row reads the previous stage at
  the adjacent rows and its own coefficients, which take lambda (from rho) and
  div u (Eq. 19) from the adjacent rows.

So with one exchange per step, before the step, a slab needs HALO(N) = 4 N + 2
rows of f* (and 4 N + 1 of T; the plan sends 4 N + 2 of both) from each
neighbour, and the new state of its own rows follows exactly; the rows of the
halo are recomputed by both neighbours.  The step also needs two global
scalars of the previous step, the mean density rho_ave of Eq. (9) and the
outlet velocity U of the convective top (Section 4.2), which every rank
obtains by a reduction over all slabs; the outlet memory of the top row (the
populations that entered it at the previous step) stays with the top rank.

This module holds no arithmetic of the method: the slab bounds, the halo
width, and the send/receive schedule of one exchange, with `exchange`
moving row blocks of host (numpy) arrays over torch.distributed
point-to-point calls on a gloo group.  A device-resident slab would follow
the same schedule with device tensors over NCCL; that path is not built.
"""
from __future__ import annotations

import numpy as np


def halo_rows(n_sub: int) -> int:
    """Rows of f* and T a slab needs beyond each of its edges for one step."""
    if n_sub < 1:
        raise ValueError("n_sub >= 1")
    return 4 * n_sub + 2


def slab_bounds(ny: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [a, b) owned by `rank`: contiguous, as even as possible, the
    lower ranks taking the remainder rows."""
    if not 0 <= rank < world or world > ny:
        raise ValueError("rank out of range or more ranks than rows")
    base, extra = divmod(ny, world)
    a = rank * base + min(rank, extra)
    return a, a + base + (1 if rank < extra else 0)


def check_plan(ny: int, world: int, n_sub: int) -> None:
    """Every slab must be at least one halo thick, so that a halo comes from
    the adjacent rank alone, and the top slab thicker than a halo, so that no
    other rank's halo reaches the top row and the outlet memory stays with the
    top rank."""
    h = halo_rows(n_sub)
    for r in range(world):
        a, b = slab_bounds(ny, world, r)
        if b - a < h or (r == world - 1 and world > 1 and b - a <= h):
            raise ValueError(f"slab {r} has {b - a} rows: too thin for the halo of {h}")


def exchange_plan(ny: int, world: int, rank: int, n_sub: int):
    """[(peer, send_rows, recv_rows)] of one exchange: row ranges [lo, hi) of
    the global lattice this rank sends to and receives from each neighbour."""
    check_plan(ny, world, n_sub)
    h = halo_rows(n_sub)
    a, b = slab_bounds(ny, world, rank)
    plan = []
    if rank > 0:
        pa, pb = slab_bounds(ny, world, rank - 1)
        plan.append((rank - 1, (a, a + h), (max(pa, a - h), a)))
    if rank < world - 1:
        na, nb = slab_bounds(ny, world, rank + 1)
        plan.append((rank + 1, (b - h, b), (b, min(nb, b + h))))
    return plan


def extended_bounds(ny: int, world: int, rank: int, n_sub: int) -> tuple[int, int]:
    """Rows [lo, hi) whose state a rank holds for one step: its slab and halos."""
    h = halo_rows(n_sub)
    a, b = slab_bounds(ny, world, rank)
    return max(0, a - h), min(ny, b + h)


def exchange(arrays, plan, dist, row_axis=None):
    """Send and receive the planned row blocks of every array (numpy, rows on
    axis row_axis[k], default the second-to-last axis) in place: the rows this
    rank sends are read from its arrays and the received rows overwrite the
    halo rows.  Lower ranks send first to avoid a deadlock with blocking
    point-to-point calls."""
    import torch
    axes = row_axis or [a.ndim - 2 for a in arrays]
    me = dist.get_rank()
    for peer, (s0, s1), (r0, r1) in plan:
        send = [torch.from_numpy(np.ascontiguousarray(np.take(a, range(s0, s1), axis=ax)))
                for a, ax in zip(arrays, axes)]
        recv = [torch.empty_like(torch.from_numpy(np.ascontiguousarray(np.take(a, range(r0, r1), axis=ax))))
                for a, ax in zip(arrays, axes)]
        order = (send, recv) if me < peer else (recv, send)
        for phase, blocks in enumerate(order):
            for t in blocks:
                if (phase == 0) == (me < peer):
                    dist.send(t, dst=peer)
                else:
                    dist.recv(t, src=peer)
        for a, ax, t in zip(arrays, axes, recv):
            idx = [slice(None)] * a.ndim
            idx[ax] = slice(r0, r1)
            a[tuple(idx)] = t.numpy()
