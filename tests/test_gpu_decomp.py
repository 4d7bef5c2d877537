"""Domain decomposition of one box into z slabs on one GPU, through the C ABI.

Several libpic subdomain contexts (pic_set_subdomain), each one z slab of
the same box, are stepped stage by stage by decomp.SlabStepper, their
messages (J guard planes, migrant particles, E and B planes) moved between
them by device copies on one stream (decomp.LocalRing).  Every slab runs its
own kernels; nothing waits on another slab inside a kernel.  The slabs
together must follow the undivided periodic box:
  * against a one-context run of the same box, step after step (FP32 on
    both sides; only the order of the current sums at the slab faces and of
    the atomics differs): rel 1e-5 of the max norm on E, B, J and momenta,
    1e-5 cells on positions, every particle present once (ids);
  * against the FP64 oracle over one step from the same state (the mixed
    form's per-step tolerance).
"""
import numpy as np
import pytest

from _gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

N = (16, 16, 32)
SC = (4, 4, 4)
TOL = 1e-5


@pytest.fixture(autouse=True)
def _own_stream():
    """The slabs and the copies between them share one non-default stream."""
    torch = require_gpu()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        yield
    torch.cuda.synchronize()


def _state(seed=7, ppc=4, u_th=0.2):
    from paper_1606_02862_gb300 import workloads as W

    nx, ny, nz = N
    rng = np.random.default_rng(seed)
    x = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    u = W.maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], 0.01 / ppc)
    E = rng.normal(0, 0.01, (3, nz, ny, nx))
    B = rng.normal(0, 0.01, (3, nz, ny, nx))
    B[2] += 0.1
    return x, u, w, E, B


def _ordered(layout, x, u, w):
    """Particles grouped by slab (so that slab r's ids are a contiguous
    range of the one-context run's ids) and the first id of each slab."""
    own = layout.owner(x[:, 2])
    o = np.argsort(own, kind="stable")
    starts = np.searchsorted(own[o], np.arange(layout.world))
    return x[o], u[o], w[o], starts


def _single(x, u, w, E, B):
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    ctx = pic.Context([N], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)], sc=SC,
                      track_ids=True, use_graph=False)
    ctx.set_background(0, 0.01)
    ctx.load_particles(0, 0, x, u, w)
    ctx.write_fields(0, pic.FIELD_E, E)
    ctx.write_fields(0, pic.FIELD_B, B)
    return ctx


def _slabs(layout, x, u, w, E, B, starts):
    import torch

    from paper_1606_02862_gb300 import decomp, pic
    from paper_1606_02862_gb300 import workloads as W

    slabs = []
    for r in range(layout.world):
        z0, nzl = layout.extent(r)
        ctx = pic.Context([(N[0], N[1], nzl)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)],
                          sc=SC, track_ids=True, use_graph=False)
        slab = decomp.LibpicSlab(ctx, id_base=int(starts[r]))
        ctx.set_background(0, 0.01)
        xl, ul, wl = decomp.split_particles(layout, r, x, u, w)
        ctx.load_particles(0, 0, xl, ul, wl)
        ctx.write_fields(0, pic.FIELD_E, E[:, z0:z0 + nzl])
        ctx.write_fields(0, pic.FIELD_B, B[:, z0:z0 + nzl])
        slabs.append(slab)
    stepper = decomp.SlabStepper(slabs, decomp.LocalRing(layout.world), decomp.torch_buffers("cuda"))
    stepper.prime()
    torch.cuda.synchronize()
    return slabs, stepper


def _gather(layout, slabs):
    """Fields (E, B, J) and particles (ids, x, u; global z) of all slabs."""
    from paper_1606_02862_gb300 import pic

    F = {k: np.concatenate([s.ctx.read_fields(0, k) for s in slabs], axis=1)
         for k in (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J)}
    ids, xs, us = [], [], []
    for r, s in enumerate(slabs):
        p = s.ctx.read_particles(0, 0, ids=True)
        z0, nzl = layout.extent(r)
        assert np.all((p["x"][:, 2] >= 0.0) & (p["x"][:, 2] < nzl))
        x = p["x"].copy()
        x[:, 2] += z0
        ids.append(p["id"])
        xs.append(x)
        us.append(p["u"])
    ids = np.concatenate(ids)
    o = np.argsort(ids)
    return F, ids[o], np.concatenate(xs)[o], np.concatenate(us)[o]


def _compare(F, ids, x, u, refF, ref_ids, ref_x, ref_u, tol=TOL):
    errs = {}
    for k, ref in refF.items():
        errs[k] = float(np.max(np.abs(F[k] - ref)) / np.max(np.abs(ref)))
        assert errs[k] <= tol, (k, errs[k])
    assert np.array_equal(ids, ref_ids), "every particle once, with its id"
    Nv = np.array(N, dtype=float)
    d = x - ref_x
    d -= Nv * np.round(d / Nv)
    errs["x"] = float(np.max(np.abs(d)))
    errs["u"] = float(np.max(np.abs(u - ref_u)) / np.max(np.abs(ref_u)))
    assert errs["x"] <= tol and errs["u"] <= tol, errs
    return errs


def _single_state(ctx):
    from paper_1606_02862_gb300 import pic

    F = {k: ctx.read_fields(0, k) for k in (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J)}
    p = ctx.read_particles(0, 0, ids=True)
    o = np.argsort(p["id"])
    return F, p["id"][o], p["x"][o], p["u"][o]


@pytest.mark.parametrize("nslabs", [1, 2, 4])
def test_slabs_follow_the_undivided_box(nslabs):
    require_gpu()
    from paper_1606_02862_gb300 import decomp

    layout = decomp.SlabLayout(N[2], nslabs, SC[2])
    x, u, w, starts = _ordered(layout, *_state()[:3])
    E, B = _state()[3:]
    single = _single(x, u, w, E, B)
    slabs, stepper = _slabs(layout, x, u, w, E, B, starts)
    try:
        crossed = 0
        for step in range(6):
            single.step(1)
            stepper.step(1)
            got = _gather(layout, slabs)
            errs = _compare(*got, *_single_state(single))
            print(f"{nslabs} slabs, step {step + 1}:", errs)
        for s in slabs:
            s.ctx.sync()
        if nslabs > 1:  # particles did cross the slab faces
            ref_owner = layout.owner(x[:, 2])
            crossed = int(np.sum(layout.owner(got[2][:, 2]) != ref_owner))
            assert crossed > 0
    finally:
        single.close()
        for s in slabs:
            s.ctx.close()


def test_two_slabs_one_step_parity_with_the_oracle(orc):
    require_gpu()
    from paper_1606_02862_gb300 import decomp, pic
    from paper_1606_02862_gb300 import workloads as W

    layout = decomp.SlabLayout(N[2], 2, SC[2])
    x, u, w, starts = _ordered(layout, *_state(seed=8)[:3])
    E, B = _state(seed=8)[3:]
    single = _single(x, u, w, E, B)
    slabs, stepper = _slabs(layout, x, u, w, E, B, starts)
    try:
        # the oracle starts from the GPU's (FP32) state, read back in FP64
        F0, ids0, x0, u0 = _single_state(single)
        w0 = single.read_particles(0, 0, ids=True)
        w0 = w0["w"][np.argsort(w0["id"])]
        st = orc.State(*N, W.DT_HALF_COURANT, E=F0[pic.FIELD_E], B=F0[pic.FIELD_B],
                       species=[orc.Species(-1.0, 1.0, 2, x0, u0, w0)], rho_bg=0.01)
        st.step(1)
        stepper.step(1)
        F, ids, xg, ug = _gather(layout, slabs)
        errs = _compare(F, ids, xg, ug, {pic.FIELD_E: st.E, pic.FIELD_B: st.B, pic.FIELD_J: st.J}, ids0,
                        st.species[0].x, st.species[0].u)
        print("two slabs vs oracle:", errs)
    finally:
        single.close()
        for s in slabs:
            s.ctx.close()


def test_subdomain_misuse_is_rejected():
    require_gpu()
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    ctx = pic.Context([(16, 16, 16)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)],
                      sc=SC, use_graph=False)
    try:
        with pytest.raises(pic.PicError):
            ctx.halo_floats(pic.FIELD_E, 0)  # not a subdomain
        ctx.set_subdomain(True)
        with pytest.raises(pic.PicError):
            ctx.step(1)  # a slab steps by stages
        with pytest.raises(pic.PicError):
            ctx.step_stage(pic.STAGE_FRAMES)  # out of order
        import torch

        buf = torch.zeros(ctx.migrant_bytes(), dtype=torch.uint8, device="cuda")
        with pytest.raises(pic.PicError):
            ctx.migrants_accept(0, buf.data_ptr())  # only between PUSH and FRAMES
        with pytest.raises(pic.PicError):
            ctx.set_boundary(0, open_y=True)
        for st in range(5):
            ctx.step_stage(st)
        ctx.sync()
    finally:
        ctx.close()
    multi = pic.Context([(16, 16, 16), (16, 16, 16)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT,
                        [pic.Species(-1.0, 1.0, 2)], sc=SC)
    try:
        with pytest.raises(pic.PicError):
            multi.set_subdomain(True)  # a slab is a one-box context
    finally:
        multi.close()
