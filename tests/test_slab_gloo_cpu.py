"""Y-slab decomposition of one domain (paper_1812_10375_gb300.slab) on CPU
gloo ranks, against the single-domain FP64 oracle, bit for bit.

Each rank holds the state (f*, T) of its slab plus halo_rows(N) rows on
either side, received from its neighbours before every step by the planned
point-to-point exchange; every other row of its arrays is NaN.  It then takes
the oracle's step (which computes on whole arrays: the NaN rows cost time,
nothing else) and keeps its own rows.  A row outside the halo that an owned
row depended on would turn that row into NaN, so bit-for-bit agreement of
the owned rows with the undivided oracle shows that the exchange carries
everything one step needs.  The two global scalars of the step, the mean
density of Eq. (9) and the outlet velocity U of the convective top, come from
reductions over the ranks: the density rows of all slabs are gathered and
summed as the undivided oracle sums them (a reduction of per-rank partial
sums would round differently), U is broadcast by the rank owning row ny - 2.

Cases: a convective-top pool (gravity, nucleation sites, a 6-row heater) on 2
and 3 ranks with N = 1 and 2, and a closed box (top wall) on 2 ranks."""
import dataclasses
import os
import socket

import numpy as np
import pytest

from paper_1812_10375_gb300 import slab
from paper_1812_10375_gb300 import workloads as wl

STEPS = 40


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    pool = wl.pool(nx=40, ny=64, n_sites=2, heater_rows=6, superheat=0.12, seed=wl.BASE_SEED + 4)
    box = dataclasses.replace(pool, name="closed_box", top_bc="wall", T_top_over_Tc=wl.TS_OVER_TC - 0.02)
    return {"pool": pool, "box": box}


def _oracle(case, n_sub):
    """The undivided oracle domain of a case (the helpers' construction)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from helpers import coexistence, oracle_domain
    return oracle_domain(case, coexistence(), n_sub=n_sub)


def _rank_main(rank, world, port, name, n_sub, out_path):
    import torch.distributed as dist
    delta = int(os.environ.get("HLB_SLAB_HALO_DELTA", "0"))
    if delta:  # a deliberately thinner halo (test_a_thinner_halo_lets_nan_into_the_slab)
        halo = slab.halo_rows
        slab.halo_rows = lambda n: halo(n) + delta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = _cases()[name]
        d = _oracle(case, n_sub)
        ny = d.p.ny
        a, b = slab.slab_bounds(ny, world, rank)
        lo, hi = slab.extended_bounds(ny, world, rank, n_sub)
        plan = slab.exchange_plan(ny, world, rank, n_sub)
        keep = np.zeros(ny, bool)
        keep[lo:hi] = True

        def poison():
            d.fs[:, ~keep] = np.nan
            d.T[~keep] = np.nan

        poison()
        for _ in range(STEPS):
            # the state rows of the halos, from the neighbours
            slab.exchange([d.fs, d.T], plan, dist)
            with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
                d.step(1)
            poison()
            # global scalars of this step, for the next one
            rows = [None] * world
            dist.all_gather_object(rows, (a, b, d.rho[a:b].copy(), d.uy[ny - 2].copy() if a <= ny - 2 < b else None))
            rho = np.concatenate([r[2] for r in sorted(rows, key=lambda r: r[0])])
            mass = float(rho[d.fluid].sum())
            u_top = next(float(r[3].mean()) for r in rows if r[3] is not None)
            d.rho_ave = mass / d.n_fluid
            d.U = max(0.0, u_top)
        res = [None] * world
        dist.all_gather_object(res, (a, b, d.rho[a:b], d.ux[a:b], d.uy[a:b], d.T[a:b], d.fs[:, a:b],
                                     d.rho_ave, d.U))
        if rank == 0:
            np.savez(out_path, **{f"r{k}_{i}": np.asarray(v) for k, r in enumerate(res) for i, v in enumerate(r)})
    finally:
        dist.destroy_process_group()


def _run(world, name, n_sub, tmp_path):
    import multiprocessing as mp
    out = str(tmp_path / f"slab_{name}_{world}_{n_sub}.npz")
    port = _port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, n_sub, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    z = np.load(out)
    return [[z[f"r{k}_{i}"] for i in range(9)] for k in range(world)]


@pytest.mark.parametrize("world,name,n_sub", [(2, "pool", 1), (3, "pool", 1), (2, "pool", 2), (2, "box", 1)])
def test_slabs_reproduce_the_undivided_oracle_bit_for_bit(world, name, n_sub, tmp_path):
    ranks = _run(world, name, n_sub, tmp_path)
    ref = _oracle(_cases()[name], n_sub).step(STEPS)
    for a, b, rho, ux, uy, T, fs, rho_ave, U in ranks:
        a, b = int(a), int(b)
        assert np.isfinite(T).all() and np.isfinite(fs).all()
        assert np.array_equal(rho, ref.rho[a:b]), (a, b)
        assert np.array_equal(ux, ref.ux[a:b]) and np.array_equal(uy, ref.uy[a:b]), (a, b)
        assert np.array_equal(T, ref.T[a:b]), (a, b)
        assert np.array_equal(fs, ref.fs[:, a:b]), (a, b)
        assert float(rho_ave) == ref.rho_ave and float(U) == ref.U
    # the slabs tile the lattice
    assert [int(r[0]) for r in ranks] == [0] + [int(r[1]) for r in ranks[:-1]]
    assert int(ranks[-1][1]) == ref.p.ny


def test_plan_covers_the_lattice_and_refuses_thin_slabs():
    for ny, world, n_sub in ((64, 2, 1), (64, 3, 1), (64, 2, 2), (400, 8, 3), (97, 4, 2)):
        bounds = [slab.slab_bounds(ny, world, r) for r in range(world)]
        assert bounds[0][0] == 0 and bounds[-1][1] == ny
        assert all(bounds[k][1] == bounds[k + 1][0] for k in range(world - 1))
        assert max(b - a for a, b in bounds) - min(b - a for a, b in bounds) <= 1
        h = slab.halo_rows(n_sub)
        for r in range(world):
            for peer, (s0, s1), (r0, r1) in slab.exchange_plan(ny, world, r, n_sub):
                assert abs(peer - r) == 1 and s1 - s0 == h and r1 - r0 == h
                # what r receives from peer is what peer sends to r
                back = {p: s for p, s, _ in slab.exchange_plan(ny, world, peer, n_sub)}
                assert back[r] == (r0, r1)
    with pytest.raises(ValueError):
        slab.exchange_plan(17, 3, 0, 1)   # slabs of 5-6 rows, halo 6
    with pytest.raises(ValueError):
        slab.exchange_plan(12, 2, 0, 1)   # top slab exactly one halo thick


@pytest.mark.parametrize("n_sub", [1, 2])
def test_a_thinner_halo_lets_nan_into_the_slab(n_sub, tmp_path, monkeypatch):
    """The halo is no wider than it must be: one row fewer and a row the slab
    owns depends on a row nobody sent (a NaN reaches it, or its value
    differs from the undivided oracle's)."""
    monkeypatch.setenv("HLB_SLAB_HALO_DELTA", "-1")
    with pytest.raises(AssertionError):
        test_slabs_reproduce_the_undivided_oracle_bit_for_bit(2, "pool", n_sub, tmp_path)
