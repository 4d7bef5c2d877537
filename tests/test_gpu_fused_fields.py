"""The fused two-buffer field update (pic_options.field_update
PIC_FIELD_UPDATE_FUSED, or chosen by the automatic mode) through the C ABI.
A pic_step of two or more steps updates the fields of each pair of steps
with k_yee_fused: E^n, B^n, J read from one buffer pair, E^{n+1},
B^{n+1} written to the other, and back on the second step of the pair.
Checked:
  * against the three in-place kernels (PIC_FIELD_UPDATE_IN_PLACE) from the
    same state:
    after the first pair E, B and every particle agree to FP32 rounding (rel
    1e-6 of the max norm, 1e-6 cells); J, whose fixed-point chunk sums round
    each term to 2^-21 of the chunk's largest and whose global sums run in
    atomic order, to 1e-5; after 3 and 7 steps all of them to 1e-5 (the
    per-step tolerance of the parity tests).  Boxes whose edges are not
    multiples of the fused tile (partial x and y tiles, a z chunk shorter
    than the others), several boxes in one launch, the PCS guard layout, and
    an open-y box with absorber and antenna;
  * against the FP64 oracle over one fused pair from a read-back state (the
    per-step tolerance of the other parity tests, twice);
  * PIC_INFO_FUSED_STEPS counts the fused steps: an odd last step and the
    in-place form take the in-place kernels;
  * the automatic choice (PIC_FIELD_UPDATE_AUTO, 0) settles on one form at
    the first step, reports it, and follows the forced in-place form within the
    parity tolerance.
"""
import numpy as np
import pytest

from _gpu_helpers import compare_box, ctx_from, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu

TOL, TOL_J = 1e-6, 1e-5


def _box(rng, nx, ny, nz, ppc=2, u_th=0.1, fields=1e-2):
    from paper_1606_02862_gb300 import workloads as W

    x = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    u = W.maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], 0.01 / ppc)
    E = rng.normal(0, fields, (3, nz, ny, nx))
    B = rng.normal(0, fields, (3, nz, ny, nx))
    B[2] += 0.1
    return W.BoxInit(nx, ny, nz, particles=[(x, u, w)], E=E, B=B, rho_bg=0.01)


def _workload(kind, seed=0):
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(7000 + seed)
    if kind == "uneven":  # x tiles of 32 + 16, y tiles of 8, z chunks of 24 + 16; a second box
        boxes, shape = [_box(rng, 48, 24, 40), _box(rng, 32, 16, 16)], 2
    elif kind == "pcs":  # guard layout 2
        boxes, shape = [_box(rng, 32, 16, 16)], 3
    elif kind == "cic":
        boxes, shape = [_box(rng, 16, 16, 8, ppc=4)], 1
    else:  # open y: absorber and antenna
        boxes, shape = [_box(rng, 16, 32, 16)], 2
    return W.Workload("fused_" + kind, W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, shape)], boxes)


def _ctx(wl, kind, field_update):
    from paper_1606_02862_gb300 import pic

    sc = (4, 4, 4) if kind == "cic" else (8, 4, 4)
    threads = 256 if kind == "pcs" else 128  # the PCS kernel is built for 8x4x4 with 256
    ctx = ctx_from(wl, sc=sc, threads_per_sc=threads, field_update=field_update)
    if kind == "open_y":
        ctx.set_boundary(0, open_y=True, absorber_cells=8, absorber_sigma=0.5)
        ctx.set_antenna(0, plane_y=12, E0=0.05, omega=0.7, tau=4.0, t0=2.0)
    assert ctx.info(pic.INFO_FUSED_STEPS) == 0
    return ctx


def _state(ctx, wl):
    from paper_1606_02862_gb300 import pic

    out = []
    for b in range(len(wl.boxes)):
        F = [ctx.read_fields(b, k) for k in (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J)]
        p = ctx.read_particles(b, 0, ids=True)
        o = np.argsort(p["id"])
        out.append((F, p["id"][o], p["x"][o], p["u"][o]))
    return out


def _agree(a, b, wl, tol=TOL):
    errs = {}
    for bi, ((Fa, ia, xa, ua), (Fb, ib, xb, ub)) in enumerate(zip(a, b)):
        for name, fa, fb in zip("EBJ", Fa, Fb):
            err = float(np.max(np.abs(fa - fb)) / max(np.max(np.abs(fb)), 1e-30))
            errs[f"{name}{bi}"] = err
            assert err <= (max(tol, TOL_J) if name == "J" else tol), (bi, name, err)
        assert np.array_equal(ia, ib), "the same particles"
        nb = wl.boxes[bi]
        N = np.array([nb.nx, nb.ny, nb.nz], dtype=float)
        d = xa - xb
        d -= N * np.round(d / N)
        errs[f"x{bi}"] = float(np.max(np.abs(d))) if d.size else 0.0
        errs[f"u{bi}"] = float(np.max(np.abs(ua - ub)) / max(np.max(np.abs(ub)), 1e-30)) if d.size else 0.0
        assert errs[f"x{bi}"] <= tol and errs[f"u{bi}"] <= tol, errs
    return errs


@pytest.mark.parametrize("kind", ["uneven", "pcs", "cic", "open_y"])
def test_fused_pairs_follow_the_in_place_update(kind):
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _workload(kind)
    fused, in_place = _ctx(wl, kind, pic.FIELD_UPDATE_FUSED), _ctx(wl, kind, pic.FIELD_UPDATE_IN_PLACE)
    try:
        done = 0
        for n in (2, 1, 4):  # a pair; one in-place step; two pairs
            fused.step(n)
            in_place.step(n)
            done += n
            errs = _agree(_state(fused, wl), _state(in_place, wl), wl, TOL if done == 2 else TOL_J)
            print(kind, f"after {done} steps:", errs)
        assert fused.info(pic.INFO_FUSED_STEPS) == 6
        assert in_place.info(pic.INFO_FUSED_STEPS) == 0
        assert fused.info(pic.INFO_STEPS) == in_place.info(pic.INFO_STEPS) == 7
        fused.step(3)  # a pair and an odd last step
        assert fused.info(pic.INFO_FUSED_STEPS) == 8
    finally:
        fused.close()
        in_place.close()


def test_fused_pair_against_the_oracle(orc):
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _workload("uneven", seed=1)
    ctx = _ctx(wl, "uneven", pic.FIELD_UPDATE_FUSED)
    try:
        ctx.step(1)  # a sort pass first, so that the pair has a stored-order pass
        states = [oracle_state_from_gpu(orc, ctx, wl, b) for b in range(len(wl.boxes))]
        ctx.step(2)
        assert ctx.info(pic.INFO_FUSED_STEPS) == 2
        for b, (st, ids) in enumerate(states):
            st.step(2)
            errs = compare_box(st, ids, ctx, wl, b, tol_field=2e-5, tol_x=2e-5, tol_u=2e-5)
            print("box", b, "fused pair vs oracle:", errs)
    finally:
        ctx.close()


def test_fused_graph_and_eager_agree():
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _workload("uneven", seed=2)
    outs = []
    for use_graph in (True, False):
        ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=128, use_graph=use_graph,
                       field_update=pic.FIELD_UPDATE_FUSED)
        try:
            ctx.step(4)
            assert ctx.info(pic.INFO_FUSED_STEPS) == 4
            outs.append(_state(ctx, wl))
        finally:
            ctx.close()
    _agree(outs[0], outs[1], wl, TOL_J)


def test_automatic_choice_settles_on_one_form():
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _workload("uneven", seed=3)
    auto = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=128)
    ref = _ctx(wl, "uneven", pic.FIELD_UPDATE_IN_PLACE)
    try:
        assert auto.info(pic.INFO_FIELD_UPDATE) == pic.FIELD_UPDATE_AUTO
        auto.step(4)
        ref.step(4)
        form = auto.info(pic.INFO_FIELD_UPDATE)
        assert form in (pic.FIELD_UPDATE_IN_PLACE, pic.FIELD_UPDATE_FUSED)
        assert auto.info(pic.INFO_FUSED_STEPS) == (4 if form == pic.FIELD_UPDATE_FUSED else 0)
        assert ref.info(pic.INFO_FIELD_UPDATE) == pic.FIELD_UPDATE_IN_PLACE
        print("automatic choice:", "fused" if form == pic.FIELD_UPDATE_FUSED else "in place",
              _agree(_state(auto, wl), _state(ref, wl), wl, TOL_J))
    finally:
        auto.close()
        ref.close()


def test_field_update_option_is_checked():
    require_gpu()
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    with pytest.raises(pic.PicError):
        pic.Context([(16, 16, 16)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)],
                    sc=(4, 4, 4), field_update=3)
    # a subdomain slab steps by stages: its field update is the in-place one
    ctx = pic.Context([(16, 16, 16)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)],
                      sc=(4, 4, 4), field_update=pic.FIELD_UPDATE_FUSED, use_graph=False)
    try:
        ctx.set_subdomain(True)
        assert ctx.info(pic.INFO_FIELD_UPDATE) == pic.FIELD_UPDATE_IN_PLACE
    finally:
        ctx.close()


def test_fused_pairs_across_a_window_shift():
    """The moving window shifts the first buffer pair between pic_step calls;
    the fused pairs then continue from it."""
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _workload("open_y", seed=4)
    fused, in_place = _ctx(wl, "open_y", pic.FIELD_UPDATE_FUSED), _ctx(wl, "open_y", pic.FIELD_UPDATE_IN_PLACE)
    try:
        for c in (fused, in_place):
            c.step(2)
            c.shift_window(0, 4)
            c.step(4)
        errs = _agree(_state(fused, wl), _state(in_place, wl), wl, TOL_J)
        print("window shift:", errs)
        assert fused.info(pic.INFO_FUSED_STEPS) == 6
    finally:
        fused.close()
        in_place.close()
