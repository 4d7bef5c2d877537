"""Domain decomposition of one box into z slabs, on CPU (no GPU).

paper_1606_02862_gb300.decomp.SlabStepper drives slabs through the staged
step and moves their messages (J guard planes, migrants, E and B planes)
around a ring.  Here the slabs are the FP64 oracle on an extended grid
(tests/_oracle_slab.py), so the decomposition itself is checked against the
undivided oracle box: the slabs must reproduce its fields and every
particle (by id) up to the order of FP64 sums at the slab faces.  The ring
runs in one process (LocalRing) and as two gloo ranks (DistRing), the form
NCCL takes between GPUs.
"""
import os
import socket

import numpy as np
import pytest
import torch

from paper_1606_02862_gb300 import decomp

TOL = 1e-11  # FP64; only the order of the current sums at the slab faces differs
STEPS = 6
N = (8, 8, 24)


def _workload(seed=3, ppc=2, u_th=0.25):
    from paper_1606_02862_gb300 import workloads as W

    nx, ny, nz = N
    rng = np.random.default_rng(seed)
    x = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    u = W.maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], 0.02 / ppc)
    E = rng.normal(0, 0.02, (3, nz, ny, nx))
    B = rng.normal(0, 0.02, (3, nz, ny, nx))
    return x, u, w, E, B


def _single(orc, steps):
    x, u, w, E, B = _workload()
    sp = orc.Species(-1.0, 1.0, 2, x, u, w)
    st = orc.State(*N, 0.5 / np.sqrt(3.0), E=E, B=B, species=[sp])
    st.step(steps)
    return st


def _slab(orc, layout, rank):
    from _oracle_slab import OracleSlab

    x, u, w, E, B = _workload()
    ids = np.arange(x.shape[0])
    sel = layout.owner(x[:, 2]) == rank
    xl, ul, wl = decomp.split_particles(layout, rank, x, u, w)
    z0, nzl = layout.extent(rank)
    return OracleSlab(orc, N[0], N[1], nzl, 0.5 / np.sqrt(3.0), [(-1.0, 1.0, 2, xl, ul, wl, ids[sel])],
                      E=E[:, z0:z0 + nzl], B=B[:, z0:z0 + nzl])


def _f64_buffers(kind, n):
    return torch.zeros(int(n), dtype=torch.float64)


def _check(st, pieces):
    """pieces: per slab (z0, E, B, J interior planes, ids, x, u)."""
    E = np.concatenate([p[1] for p in pieces], axis=1)
    B = np.concatenate([p[2] for p in pieces], axis=1)
    J = np.concatenate([p[3] for p in pieces], axis=1)
    for got, ref in ((E, st.E), (B, st.B), (J, st.J)):
        assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
    ids = np.concatenate([p[4] for p in pieces])
    x = np.concatenate([p[5] + np.array([0.0, 0.0, p[0]]) for p in pieces])
    u = np.concatenate([p[6] for p in pieces])
    o = np.argsort(ids)
    assert np.array_equal(ids[o], np.arange(st.species[0].x.shape[0]))
    assert np.max(np.abs(x[o] - st.species[0].x)) <= TOL * N[2]
    assert np.max(np.abs(u[o] - st.species[0].u)) <= TOL * np.max(np.abs(st.species[0].u))


def _pieces(layout, slabs):
    out = []
    for r, s in enumerate(slabs):
        ids, x, u = s.particles(0)
        out.append((layout.extent(r)[0], s.interior(s.E), s.interior(s.B), s.interior(s.J), ids, x, u))
    return out


def test_slab_layout_covers_the_box_in_whole_rows():
    for nz, world, LZ in ((256, 8, 4), (24, 2, 4), (24, 3, 4), (40, 3, 8), (16, 4, 4)):
        lay = decomp.SlabLayout(nz, world, LZ)
        ext = [lay.extent(r) for r in range(world)]
        assert ext[0][0] == 0 and sum(e[1] for e in ext) == nz
        for (z0, n), (z1, _) in zip(ext, ext[1:]):
            assert z0 + n == z1
        assert all(n % LZ == 0 and n >= 4 for _, n in ext)
        assert max(n for _, n in ext) - min(n for _, n in ext) <= LZ
        z = np.linspace(-nz, 2 * nz, 997)
        own = lay.owner(z)
        zz = np.mod(z, nz)
        for r, (z0, n) in enumerate(ext):
            assert np.all((zz[own == r] >= z0) & (zz[own == r] < z0 + n))
    with pytest.raises(ValueError):
        decomp.SlabLayout(24, 7, 4)  # 6 rows for 7 slabs
    with pytest.raises(ValueError):
        decomp.SlabLayout(26, 2, 4)


def test_split_particles_keeps_every_particle_once():
    x, u, w, _, _ = _workload()
    lay = decomp.SlabLayout(N[2], 3, 4)
    parts = [decomp.split_particles(lay, r, x, u, w) for r in range(3)]
    assert sum(p[0].shape[0] for p in parts) == x.shape[0]
    for r, (xl, ul, wl) in enumerate(parts):
        assert np.all((xl[:, 2] >= 0) & (xl[:, 2] < lay.extent(r)[1]))
        assert xl.shape[0] == ul.shape[0] == wl.shape[0]


@pytest.mark.parametrize("nslabs", [1, 2, 3])
def test_oracle_slabs_on_a_local_ring_match_the_undivided_box(orc, nslabs):
    lay = decomp.SlabLayout(N[2], nslabs, 4)
    slabs = [_slab(orc, lay, r) for r in range(nslabs)]
    stepper = decomp.SlabStepper(slabs, decomp.LocalRing(nslabs), _f64_buffers)
    stepper.prime()
    stepper.step(STEPS)
    st = _single(orc, STEPS)
    crossed = sum(len(s.particles(0)[0]) for s in slabs)
    assert crossed == st.species[0].x.shape[0]
    _check(st, _pieces(lay, slabs))


def test_a_dropped_exchange_is_caught(orc):
    """The comparison is sharp: two slabs that skip the J exchange (their
    faces' current never reaches the neighbour) differ from the undivided
    box."""
    from paper_1606_02862_gb300 import pic

    lay = decomp.SlabLayout(N[2], 2, 4)
    slabs = [_slab(orc, lay, r) for r in range(2)]
    stepper = decomp.SlabStepper(slabs, decomp.LocalRing(2), _f64_buffers)
    real = stepper.exchange
    stepper.exchange = lambda key: None if key == pic.FIELD_J else real(key)
    stepper.prime()
    stepper.step(2)
    with pytest.raises(AssertionError):
        _check(_single(orc, 2), _pieces(lay, slabs))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lay = decomp.SlabLayout(N[2], world, 4)
        slab = _slab(oracle, lay, rank)
        stepper = decomp.SlabStepper([slab], decomp.DistRing(dist), _f64_buffers)
        stepper.prime()
        stepper.step(STEPS)
        ids, x, u = slab.particles(0)
        mine = (lay.extent(rank)[0], slab.interior(slab.E), slab.interior(slab.B), slab.interior(slab.J),
                ids, x, u)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


def test_oracle_slabs_as_two_gloo_ranks_match_the_undivided_box(orc):
    import torch.multiprocessing as mp

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    pieces = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    _check(_single(orc, STEPS), pieces)
