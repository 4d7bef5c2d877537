"""Open-y boundaries on the GPU (mixed form) against the FP64 oracle: the
damping absorber, the laser antenna, particle removal at the y faces and the
moving window, each through the C ABI, one step from the GPU's own state
(read back in FP64) at the per-step tolerance of the other parity tests, and
an antenna run in vacuum over many steps against the oracle's."""
import numpy as np
import pytest

from _gpu_helpers import compare_box, ctx_from, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu

TOL = dict(tol_field=1e-5, tol_x=1e-5, tol_u=1e-5)


def _plasma(nx=16, ny=32, nz=16, ppc=4, u_th=0.1, fields=1e-2, seed=0, y_range=None, shape=2):
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(4000 + seed)
    x = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    if y_range is not None:
        x = x[(x[:, 1] >= y_range[0]) & (x[:, 1] < y_range[1])]
    u = W.maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], 0.01 / ppc)
    E = rng.normal(0, fields, (3, nz, ny, nx))
    B = rng.normal(0, fields, (3, nz, ny, nx))
    box = W.BoxInit(nx, ny, nz, particles=[(x, u, w)], E=E, B=B, rho_bg=0.01)
    return W.Workload("open_y_test", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, shape)], [box])


def _step_and_compare(orc, ctx, wl, state_kw, tol=TOL):
    st, _ = oracle_state_from_gpu(orc, ctx, wl, 0, **state_kw)
    ctx.step(1)
    st.step(1)
    ids = [sp.ids for sp in st.species]
    errs = compare_box(st, ids, ctx, wl, 0, **tol)
    print("open-y parity errors:", errs)
    return st


@pytest.mark.parametrize("pre,shape", [(0, 2), (2, 2), (1, 3)])
def test_absorber_one_step(orc, pre, shape):
    require_gpu()
    wl = _plasma(shape=shape)
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        ctx.set_boundary(0, absorber_cells=8, absorber_sigma=0.5)
        ctx.step(pre)
        _step_and_compare(orc, ctx, wl, dict(absorber=(8, 0.5)))
    finally:
        ctx.close()


def test_open_y_particles_one_step(orc):
    """Fast particles near both y faces: the ones that cross leave on both sides."""
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    rng = np.random.default_rng(11)
    n = 600
    x = np.column_stack([rng.uniform(0, 16, n), np.where(rng.random(n) < 0.5, rng.uniform(0, 0.4, n),
                                                         rng.uniform(31.6, 32, n)), rng.uniform(0, 16, n)])
    u = rng.normal(0, 0.6, (n, 3))
    box = W.BoxInit(16, 32, 16, particles=[(x, u, np.full(n, 0.01))], rho_bg=0.0)
    wl = W.Workload("open_y_particles", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [box])
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        ctx.set_boundary(0, open_y=True)
        st = _step_and_compare(orc, ctx, wl, dict(open_y=True))
        gone = n - st.species[0].x.shape[0]
        assert gone > 50 and ctx.count_particles(0, 0) == n - gone
        ctx.step(3)
        st.step(3)
        assert ctx.count_particles(0, 0) == st.species[0].x.shape[0]
    finally:
        ctx.close()


@pytest.mark.parametrize("w0", [0.0, 5.0])
def test_antenna_one_step(orc, w0):
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = _plasma(ny=64, fields=1e-3, y_range=(24, 64))
    ant = dict(plane_y=12, E0=0.05, omega=2 * np.pi / 16, w0=w0, xc=8.0, zc=8.0, tau=8.0, t0=6.0)
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        ctx.set_boundary(0, open_y=True, absorber_cells=8, absorber_sigma=0.3)
        ctx.set_antenna(0, **ant)
        ctx.step(20)
        assert ctx.info(pic.INFO_STEPS) == 20
        a = orc.Antenna(ja=12, E0=0.05, omega=ant["omega"], w0=w0, xc=8.0, zc=8.0, tau=8.0, t0=6.0)
        kw = dict(absorber=(8, 0.3), open_y=True, antenna=a, t=20 * wl.dt)
        _step_and_compare(orc, ctx, wl, kw)
        # the pulse is on its way: Ex near the sheet is of order E0
        ex = ctx.read_fields(0, pic.FIELD_E)[0]
        assert 0.2 * 0.05 < np.max(np.abs(ex[:, 13:24, :])) < 2 * 0.05
    finally:
        ctx.close()


def test_antenna_vacuum_run_matches_oracle(orc):
    """A plane antenna in vacuum with absorbers, 400 steps: GPU (FP32 fields)
    against the oracle (FP64), both from zero fields."""
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    nx, ny, nz = 8, 128, 8
    box = W.BoxInit(nx, ny, nz, particles=[(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))])
    wl = W.Workload("antenna_vacuum", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [box])
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    om = 2 * np.pi / 12
    try:
        ctx.set_boundary(0, absorber_cells=24, absorber_sigma=1.0)
        ctx.set_antenna(0, plane_y=40, E0=1.0, omega=om, tau=30.0, t0=60.0)
        ctx.step(400)
        st = orc.State(nx, ny, nz, wl.dt, absorber=(24, 1.0),
                       antenna=orc.Antenna(ja=40, E0=1.0, omega=om, tau=30.0, t0=60.0))
        st.step(400)
        got = ctx.read_fields(0, pic.FIELD_E)
        err = np.max(np.abs(got - st.E)) / np.max(np.abs(st.E))
        print("antenna vacuum run, max |E_gpu - E_oracle| / max |E|:", err, "max |E|:", np.max(np.abs(st.E)))
        assert np.max(np.abs(st.E)) > 0.5
        assert err < 1e-4
    finally:
        ctx.close()


@pytest.mark.parametrize("shape", [2, 3])
def test_window_shift_then_step(orc, shape):
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    wl = _plasma(ny=32, shape=shape)
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        ctx.set_boundary(0, open_y=True, absorber_cells=4, absorber_sigma=0.2)
        ctx.step(3)
        st, _ = oracle_state_from_gpu(orc, ctx, wl, 0, absorber=(4, 0.2), open_y=True)
        n0 = ctx.count_particles(0, 0)
        ctx.shift_window(0, 8)
        st.shift_window(8)
        # right after the shift: a translation, so FP32 values are moved, not recomputed
        for which, ref in ((pic.FIELD_E, st.E), (pic.FIELD_B, st.B)):
            got = ctx.read_fields(0, which)
            assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref))
        assert ctx.count_particles(0, 0) == st.species[0].x.shape[0] < n0
        # fresh plasma in the top rows, the same particles on both sides
        rng = np.random.default_rng(21)
        xn = W.uniform_in_cells(rng, 16, 8, 16, 4) + [0.0, 24.0, 0.0]
        un = W.maxwellian(rng, xn.shape[0], 0.1)
        wn = np.full(xn.shape[0], 0.0025)
        ctx.load_particles(0, 0, xn, un, wn)
        sp = st.species[0]
        id0 = wl.boxes[0].particles[0][0].shape[0]  # ids run on in load order
        sp.x = np.vstack([sp.x, xn])
        sp.u = np.vstack([sp.u, un])
        sp.w = np.concatenate([sp.w, wn])
        sp.ids = np.concatenate([sp.ids, np.arange(id0, id0 + xn.shape[0])])
        got = ctx.read_particles(0, 0, ids=True)
        assert np.array_equal(np.sort(got["id"]), np.sort(sp.ids))
        order = np.argsort(sp.ids)
        sp.x, sp.u, sp.w, sp.ids = (np.ascontiguousarray(a[order]) for a in (sp.x, sp.u, sp.w, sp.ids))
        ctx.step(1)
        st.step(1)
        errs = compare_box(st, [sp.ids], ctx, wl, 0, **TOL)
        print("after shift + load + step:", errs)
        with pytest.raises(pic.PicError):
            ctx.shift_window(0, 6)  # not a multiple of the supercell edge along y
    finally:
        ctx.close()


def test_open_y_rejected_in_plain_form():
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = _plasma(nx=8, ny=8, nz=8)
    ctx = ctx_from(wl, precision=pic.PRECISION_FP64_PLAIN)
    try:
        with pytest.raises(pic.PicError):
            ctx.set_boundary(0, open_y=True)
        with pytest.raises(pic.PicError):
            ctx.set_antenna(0, plane_y=2, E0=1.0, omega=0.5)
    finally:
        ctx.close()


def _unmatched_near_faces(ctx, st, ny, excused, tol=1e-5):
    """Particles present on one side only (FP32 and FP64 may disagree on a
    face crossing by the rounding of the position): each must sit within tol
    cells of a y face of the box it is still in, i.e. on the plane the other
    side's copy crossed.  Returns the number newly found; `excused` keeps
    (species, id) of every one found so far, which are left out afterwards."""
    found = 0
    for si, sp in enumerate(st.species):
        p = ctx.read_particles(0, si, ids=True)
        gpu = dict(zip(p["id"].tolist(), p["x"][:, 1].tolist()))
        orc = dict(zip(sp.ids.tolist(), sp.x[:, 1].tolist()))
        for side, mine, other in (("gpu", gpu, orc), ("oracle", orc, gpu)):
            for i in set(mine) - set(other):
                if (si, i) in excused:
                    continue
                y = mine[i]
                assert min(abs(y), abs(y - ny)) <= tol, (side, si, i, y)
                excused.add((si, i))
                found += 1
    return found


def test_laser_window_run_matches_oracle(orc):
    """The open-boundary laser workload at reduced size through 70 steps with
    the window advanced by 4 cells whenever c t passes them (5 shifts) and the
    same fresh plasma loaded on both sides: every particle by id (one present
    on one side only must have crossed a y face within 1e-5 cells of it, the
    FP32/FP64 disagreement on that crossing), charge, field energy and E
    against the oracle run of the same recipe."""
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    wl = W.laser_window(nx=16, ny=96, nz=16, ppc=2, lam=16.0, a0=0.5, waist=6.0, duration=10.0,
                        ramp=(40, 70), absorber=12, antenna_y=16)
    b = wl.boxes[0]
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    a = wl.extra["antenna"]
    bd = wl.extra["boundary"]
    species = []
    next_id = []
    for sd, (x, u, w) in zip(wl.species, b.particles):
        osp = orc.Species(sd.q, sd.m, sd.shape, x, u, w)
        osp.ids = np.arange(x.shape[0])  # the library's ids: load order per species
        next_id.append(x.shape[0])
        species.append(osp)
    st = orc.State(b.nx, b.ny, b.nz, wl.dt, species=species, open_y=True,
                   absorber=(bd["absorber_cells"], bd["absorber_sigma"]),
                   antenna=orc.Antenna(ja=a["plane_y"], E0=a["E0"], omega=a["omega"], w0=a["w0"],
                                       xc=a["xc"], zc=a["zc"], tau=a["tau"], t0=a["t0"]))
    rng = np.random.default_rng(77)
    shifts = 0
    excused = set()
    try:
        for k in range(70):
            ctx.step(1)
            st.step(1)
            _unmatched_near_faces(ctx, st, b.ny, excused)
            if (k + 1) * wl.dt >= (shifts + 1) * 4:
                shifts += 1
                ctx.shift_window(0, 4)
                st.shift_window(4)
                _unmatched_near_faces(ctx, st, b.ny, excused)
                slab = W.window_slab(rng, b.nx, b.nz, b.ny - 4, b.ny, 2, wl.extra["density"],
                                     y_shift=float(4 * shifts))
                for si, (x, u, w) in enumerate(slab):
                    ctx.load_particles(0, si, x, u, w)
                    sp = st.species[si]
                    sp.x = np.vstack([sp.x, x])
                    sp.u = np.vstack([sp.u, u])
                    sp.w = np.concatenate([sp.w, w])
                    sp.ids = np.concatenate([sp.ids, np.arange(next_id[si], next_id[si] + x.shape[0])])
                    next_id[si] += x.shape[0]
        assert shifts == 5
        print("particles on one side only (all at a y face):", sorted(excused))
        for si in range(2):
            gone = sum(1 for s_, _ in excused if s_ == si)
            n_gpu, n_orc = ctx.count_particles(0, si), st.species[si].x.shape[0]
            assert abs(n_gpu - n_orc) <= gone, (si, n_gpu, n_orc, gone)
        d_gpu, d_orc = ctx.diagnostics(0), st.diagnostics()
        print("laser window run: gpu", d_gpu, "oracle", d_orc)
        assert abs(d_gpu[0] / d_orc[0] - 1) < 1e-3
        qw_max = max(abs(sp.q) * float(np.max(np.abs(sp.w))) for sp in st.species)
        # the particles found above, plus the FP32 rounding of every weight
        assert abs(d_gpu[2] - d_orc[2]) < 1e-6 * max(1.0, abs(d_orc[2])) + max(2, len(excused)) * qw_max
        E = ctx.read_fields(0, pic.FIELD_E)
        assert np.max(np.abs(E - st.E)) < 1e-3 * np.max(np.abs(st.E))
    finally:
        ctx.close()
