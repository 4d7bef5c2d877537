"""Parity at the full size of the headline workload, in the launch
configuration the benchmark times: 256^3 periodic cells, 134,217,728 TSC
electrons at 8 per cell (Maxwellian u_th = 0.05, density 0.01 on a fixed
background), 8x4x4 supercells with 256 threads each, the step replayed
from its CUDA graph, a sort pass every 4 steps.

The oracle cannot step the whole box in seconds, so it steps windows of
24^3 cells cut out of the GPU state (the fields and every particle inside),
periodic on the window.  A wrap of the window reaches at most 3 cells into
it in one step: a TSC particle's gather and deposit windows reach 2.5 cells
from it, the Yee update one cell per half step.  The comparison therefore
keeps the cells and the particles at least 5 cells inside the window.
One window straddles the periodic seam of the box on all three axes, where
the deposit goes through the guard images.  The first step after the load
(a sort pass of the push) and the next one (a stored-order pass) are both
compared, on random E, B written over the whole box (the recipe itself
starts from zero fields, which would leave the gather untested).

Then the 64^3 sub-run of the same recipe (2,097,152 particles, zero initial
fields): the oracle follows the GPU from the load for 4 steps (one sort
pass, three stored-order passes) and the state is compared at the end,
with the per-step tolerance times the number of steps.
"""
import numpy as np
import pytest

from _gpu_helpers import compare_box, ctx_from, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu

N = 256
PPC = 8
WIN = 24
MARGIN = 5
TOL = 1e-5
# window origins (x, y, z); the first straddles the seam on every axis
ORIGINS = [(N - 12, N - 12, N - 12), (100, 37, 200), (3, 181, 64)]


def _window_index(o):
    return [(o[a] + np.arange(WIN)) % N for a in range(3)]


def _cut_fields(F, o):
    ix, iy, iz = _window_index(o)
    return F[:, iz][:, :, iy][:, :, :, ix].copy()


def _select(cell, o):
    """Mask of the particles whose cell lies in the window at origin o."""
    m = np.ones(cell.shape[0], dtype=bool)
    for a in range(3):
        m &= ((cell[:, a] - o[a]) % N) < WIN
    return m


def _window_states(orc, dt, E, B, x, u, w, ids):
    """One oracle State per window, its particles carrying their ids."""
    cell = np.floor(x).astype(np.int32)
    out = []
    for o in ORIGINS:
        m = _select(cell, o)
        xl = np.mod(x[m] - np.asarray(o, dtype=np.float64), N)
        sp = orc.Species(q=-1.0, m=1.0, order=2, x=xl, u=u[m], w=w[m])
        sp.ids = ids[m]
        st = orc.State(WIN, WIN, WIN, dt, E=_cut_fields(E, o), B=_cut_fields(B, o), species=[sp],
                       rho_bg=0.01)
        inner = np.all((xl >= MARGIN) & (xl < WIN - MARGIN), axis=1)
        out.append((o, st, sp, inner))
    return out


def _step_and_compare(orc, ctx, wins, pic):
    """Step the oracle windows once; compare them with the GPU state the
    caller has stepped once.  Returns the GPU readback (x, u, w, ids)."""
    E = ctx.read_fields(0, pic.FIELD_E)
    B = ctx.read_fields(0, pic.FIELD_B)
    J = ctx.read_fields(0, pic.FIELD_J)
    p = ctx.read_particles(0, 0, ids=True)
    errs = []
    inner_sl = slice(MARGIN, WIN - MARGIN)
    want = np.zeros(p["id"].shape[0], dtype=bool)
    for o, st, sp, inner in wins:
        ids_in = sp.ids[inner]
        want[:] = False
        want[ids_in] = True
        st.step(1)
        e = {}
        for name, got_full, ref in (("E", E, st.E), ("B", B, st.B), ("J", J, st.J)):
            r = ref[:, inner_sl, inner_sl, inner_sl]
            g = _cut_fields(got_full, o)[:, inner_sl, inner_sl, inner_sl]
            scale = np.max(np.abs(r))
            assert scale > 0.0, name
            e[name] = float(np.max(np.abs(g - r)) / scale)
            assert e[name] <= TOL, (o, name, e[name])
        # the window's inner particles after the step, matched by id
        gm = want[p["id"]]
        gids = p["id"][gm]
        assert gids.shape[0] == ids_in.shape[0], "particles lost or duplicated"
        go = np.argsort(gids)
        oo = np.argsort(ids_in)
        assert np.array_equal(gids[go], ids_in[oo])
        xr = sp.x[inner][oo] + np.asarray(o, dtype=np.float64)
        d = p["x"][gm][go] - xr
        d -= N * np.round(d / N)
        e["x"] = float(np.max(np.abs(d)))
        ur = sp.u[inner][oo]
        e["u"] = float(np.max(np.abs(p["u"][gm][go] - ur)) / np.max(np.abs(ur)))
        assert e["x"] <= TOL and e["u"] <= TOL, (o, e)
        errs.append(e)
    print("full-size window errors:", errs)
    return E, B, p


def test_headline_full_size_sampled_windows(orc):
    require_gpu()
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    npart = N ** 3 * PPC
    x = np.empty((npart, 3))
    u = np.empty((npart, 3))
    w = np.empty(npart)
    assert W.fill_thermal(x, u, w, N, N, N, PPC, 0.05) == npart
    rng = np.random.default_rng(77)
    E0 = rng.normal(0.0, 0.01, (3, N, N, N))
    B0 = rng.normal(0.0, 0.01, (3, N, N, N))
    B0[2] += 0.1
    ctx = pic.Context([(N, N, N)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2, True, 0)],
                      sc=(8, 4, 4), threads_per_sc=256, use_graph=True, track_ids=True)
    try:
        ctx.set_background(0, 0.01)
        ctx.load_particles(0, 0, x, u, w)
        ctx.write_fields(0, pic.FIELD_E, E0)
        ctx.write_fields(0, pic.FIELD_B, B0)
        # step 1: a sort pass, from the loaded state (ids are the load order)
        wins = _window_states(orc, W.DT_HALF_COURANT, E0, B0, x, u, w, np.arange(npart, dtype=np.int64))
        del x, u, w, E0, B0
        ctx.step(1)
        E1, B1, p1 = _step_and_compare(orc, ctx, wins, pic)
        # step 2: a stored-order pass, from the GPU state after step 1
        wins = _window_states(orc, W.DT_HALF_COURANT, E1, B1, p1["x"], p1["u"], p1["w"], p1["id"])
        del E1, B1, p1
        ctx.step(1)
        _step_and_compare(orc, ctx, wins, pic)
        assert ctx.count_particles(0, 0) == npart
    finally:
        ctx.close()


def test_subrun_64_follows_the_oracle_for_four_steps(orc):
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    steps = 4
    wl = W.thermal_tsc(n=64)
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        st, ids = oracle_state_from_gpu(orc, ctx, wl, 0)
        ctx.step(steps)
        st.step(steps)
        tol = steps * TOL
        errs = compare_box(st, ids, ctx, wl, 0, tol_field=tol, tol_x=tol, tol_u=tol)
        print("64^3 sub-run errors after", steps, "steps:", errs)
    finally:
        ctx.close()
