"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Single-step parity: the GPU state is read back in FP64 and handed to the
oracle, both advance one full PIC step (gather -> Boris -> move -> Esirkepov
-> Yee, Sec. 4), and E, B, J and every particle (matched by id) are
compared.  Tolerances:
  * plain FP64 form: 1e-11 relative to the max norm (only the order of the
    FP64 atomic sums differs from the oracle);
  * mixed form (FP32 fields, momenta and in-cell offsets): rel 1e-5 of the
    max norm on E, B, J and momenta, 1e-5 cells on positions.  FP32 carries
    ~6e-8 relative error per operation; the deposit forms DS = S1 - S0 from
    the displacement directly, so the current keeps that relative accuracy
    even for displacements of 1e-3 cells, and a cell's J sums O(100)
    particle terms, which keeps the error near 1e-6.
"""
import math

import numpy as np
import pytest

from _gpu_helpers import compare_box, ctx_from, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu

MIXED_TOL = dict(tol_field=1e-5, tol_x=1e-5, tol_u=1e-5)
PLAIN_TOL = dict(tol_field=1e-11, tol_x=1e-11, tol_u=1e-11)


def _thermal(n=(16, 16, 16), ppc=4, u_th=0.05, shape=2, seed=0, fields=1e-2, species=None):
    from paper_1606_02862_gb300 import workloads as W

    nx, ny, nz = n
    rng = np.random.default_rng(1000 + seed)
    x = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    u = W.maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], 0.01 / ppc)
    E = rng.normal(0, fields, (3, nz, ny, nx))
    B = rng.normal(0, fields, (3, nz, ny, nx))
    B[2] += 0.1
    parts = [(x, u, w)]
    sp = [W.SpeciesDef("e", -1.0, 1.0, shape)]
    if species == "ions":
        xi = W.uniform_in_cells(rng, nx, ny, nz, ppc)
        parts.append((xi, W.maxwellian(rng, xi.shape[0], u_th / 40.0), w.copy()))
        sp.append(W.SpeciesDef("p", 1.0, W.PROTON_MASS, shape))
    box = W.BoxInit(nx, ny, nz, particles=parts, E=E, B=B, rho_bg=0.0 if species else 0.01)
    return W.Workload("thermal_test", W.DT_HALF_COURANT, sp, [box])


def _one_step_parity(orc, wl, tol, pre_steps=0, **ctx_kw):
    """pre_steps GPU steps first, then one compared step.  With the default
    sort period of 4 the step after 0 pre-steps is a sort pass of the push
    and the step after 1 to 3 pre-steps pushes the lists in stored order."""
    require_gpu()
    ctx = ctx_from(wl, **ctx_kw)
    try:
        if pre_steps:
            ctx.step(pre_steps)
        states = []
        for bi in range(len(wl.boxes)):
            st, ids = oracle_state_from_gpu(orc, ctx, wl, bi)
            states.append((st, ids))
        ctx.step(1)
        errs = []
        for bi, (st, ids) in enumerate(states):
            st.step(1)
            errs.append(compare_box(st, ids, ctx, wl, bi, **tol))
        print("parity errors:", errs)
        return errs
    finally:
        ctx.close()


@pytest.mark.parametrize("shape", [1, 2])
def test_plain_fp64_one_step(orc, shape):
    from paper_1606_02862_gb300 import pic

    wl = _thermal(shape=shape, u_th=0.1)
    _one_step_parity(orc, wl, PLAIN_TOL, precision=pic.PRECISION_FP64_PLAIN)


@pytest.mark.parametrize("pre", [0, 2], ids=["sort_pass", "stored_order"])
@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("sc,threads", [((4, 4, 4), 64), ((4, 4, 4), 128), ((8, 8, 4), 128),
                                        ((8, 8, 4), 256), ((8, 4, 4), 128), ((8, 4, 4), 256),
                                        ((8, 8, 8), 256)])
def test_mixed_one_step(orc, shape, sc, threads, pre):
    wl = _thermal(n=(16, 24, 16), shape=shape, u_th=0.1)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=pre, sc=sc, threads_per_sc=threads)


@pytest.mark.parametrize("sort_every", [1, 3])
def test_mixed_sort_period(orc, sort_every):
    """Every step a sort pass (1), or passes 1 and 2 in stored order after
    a sort (3): the compared step is the one after two pre-steps."""
    wl = _thermal(n=(16, 16, 16), shape=2, u_th=0.1, species="ions")
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=2, sc=(8, 4, 4), threads_per_sc=256,
                     sort_every=sort_every)


def test_mixed_small_cic_workload(orc):
    """The 32^3, 2 ppc, CIC, B_z = 0.1 workload, u_th = 0.01."""
    from paper_1606_02862_gb300 import workloads as W

    _one_step_parity(orc, W.small_cic_32(), MIXED_TOL)


def test_mixed_two_species_relativistic(orc):
    wl = _thermal(n=(16, 16, 16), shape=2, u_th=0.8, species="ions", fields=0.05)
    _one_step_parity(orc, wl, MIXED_TOL, sc=(8, 8, 4), threads_per_sc=128)


def test_mixed_batched_uneven_boxes(orc):
    """Three boxes of different size and ppc advance in the same launches."""
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(7)
    boxes = []
    for n, ppc in (((8, 8, 8), 1), ((16, 8, 12), 6), ((12, 12, 12), 3)):
        x = W.uniform_in_cells(rng, *n, ppc)
        u = W.maxwellian(rng, x.shape[0], 0.1)
        boxes.append(W.BoxInit(*n, particles=[(x, u, np.full(x.shape[0], 0.01 / ppc))],
                               E=rng.normal(0, 0.01, (3, n[2], n[1], n[0])), rho_bg=0.01))
    wl = W.Workload("batched_test", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], boxes)
    _one_step_parity(orc, wl, MIXED_TOL)


def test_mixed_graph_and_eager_agree(orc):
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = _thermal(n=(16, 16, 16), shape=2)
    outs = []
    for use_graph in (True, False):
        ctx = ctx_from(wl, use_graph=use_graph)
        ctx.step(3)
        outs.append((ctx.read_fields(0, pic.FIELD_E), ctx.read_particles(0, 0, ids=True)))
        ctx.close()
    (e1, p1), (e2, p2) = outs
    assert np.max(np.abs(e1 - e2)) <= 1e-5 * np.max(np.abs(e2))
    o1, o2 = np.argsort(p1["id"]), np.argsort(p2["id"])
    assert np.max(np.abs(p1["u"][o1] - p2["u"][o2])) <= 1e-5 * np.max(np.abs(p2["u"]))


def test_mixed_edge_positions(orc):
    """Particles on cell faces, just below a face, on supercell and box
    seams, moving across them in every direction."""
    from paper_1606_02862_gb300 import workloads as W

    n = 8
    pts = []
    us = []
    for base in ([0.0, 0.0, 0.0], [3.999999, 4.0, 7.9999995], [7.5, 3.5, 0.5], [4.0, 4.0, 4.0]):
        for dirn in ([1, 1, 1], [-1, -1, -1], [1, -1, 0], [0, 0, -1]):
            pts.append(base)
            us.append(0.6 * np.array(dirn, dtype=float))
    x = np.array(pts)
    u = np.array(us)
    box = W.BoxInit(n, n, n, particles=[(x, u, np.full(x.shape[0], 0.05))], rho_bg=0.0)
    wl = W.Workload("edges", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [box])
    _one_step_parity(orc, wl, MIXED_TOL)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=1)


def test_mixed_empty_and_lopsided_boxes(orc):
    """An empty box and a box whose particles all sit in one supercell."""
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(9)
    x = rng.uniform(4.0, 8.0, (500, 3))
    u = W.maxwellian(rng, 500, 0.2)
    b1 = W.BoxInit(12, 12, 12, particles=[(x, u, np.full(500, 0.02))], rho_bg=0.0)
    b0 = W.BoxInit(8, 8, 8, particles=[(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))],
                   E=rng.normal(0, 0.01, (3, 8, 8, 8)))
    wl = W.Workload("lopsided", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [b0, b1])
    _one_step_parity(orc, wl, MIXED_TOL)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=1)


def test_plain_and_mixed_agree_after_one_step(orc):
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = _thermal(n=(16, 16, 16), shape=2)
    a = ctx_from(wl, precision=pic.PRECISION_FP64_PLAIN)
    b = ctx_from(wl)
    a.step(1)
    b.step(1)
    for which in (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J):
        fa, fb = a.read_fields(0, which), b.read_fields(0, which)
        assert np.max(np.abs(fa - fb)) <= 2e-5 * np.max(np.abs(fa))
    a.close()
    b.close()


def test_diagnostics_match_oracle(orc):
    require_gpu()
    wl = _thermal(n=(16, 16, 16), shape=2, u_th=0.1, species="ions")
    ctx = ctx_from(wl)
    ctx.step(2)
    st, _ = oracle_state_from_gpu(orc, ctx, wl, 0)
    got = ctx.diagnostics(0)
    want = st.diagnostics()
    assert abs(got[0] / want[0] - 1) < 1e-6
    assert abs(got[1] / want[1] - 1) < 1e-6
    assert abs(got[2] - want[2]) < 1e-9 * (1 + abs(want[2]))
    rho_scale = np.max(np.abs(st.rho()))
    assert abs(got[3] - want[3]) < 1e-5 * rho_scale
    ctx.close()


@pytest.mark.parametrize("pre", [0, 2], ids=["sort_pass", "stored_order"])
@pytest.mark.parametrize("shape", [1, 2])
def test_mixed_energy_conserving_gather(orc, shape, pre):
    """The energy-conserving gather variant (one order lower along each
    staggered axis) against the oracle's, two species with the variant on
    one of them."""
    from paper_1606_02862_gb300 import workloads as W

    wl = _thermal(n=(16, 16, 16), shape=shape, u_th=0.1, species="ions", fields=0.05)
    wl.species[0] = W.SpeciesDef("e", -1.0, 1.0, shape, True, True)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=pre, sc=(8, 4, 4), threads_per_sc=256)


@pytest.mark.parametrize("shape", [1, 2])
def test_plain_energy_conserving_gather(orc, shape):
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    wl = _thermal(shape=shape, u_th=0.1, fields=0.05)
    wl.species[0] = W.SpeciesDef("e", -1.0, 1.0, shape, True, True)
    _one_step_parity(orc, wl, PLAIN_TOL, precision=pic.PRECISION_FP64_PLAIN)


# ---------------------------------------------------------------- PCS shape

PCS_CONFIGS = [((4, 4, 4), 128), ((8, 4, 4), 256)]


@pytest.mark.parametrize("pre", [0, 2], ids=["sort_pass", "stored_order"])
@pytest.mark.parametrize("sc,threads", PCS_CONFIGS)
def test_mixed_pcs_one_step(orc, sc, threads, pre):
    """The PCS (cubic spline) shape: 4-node gather, 4-node common and 5-node
    general Esirkepov windows, 2-cell field guards."""
    wl = _thermal(n=(16, 24, 16), shape=3, u_th=0.1)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=pre, sc=sc, threads_per_sc=threads)


@pytest.mark.parametrize("other", [1, 2])
def test_mixed_pcs_with_cic_or_tsc_species(orc, other):
    """A CIC or TSC species in a context whose tiles carry the PCS guards
    (every tile index shifted by one), next to a PCS species."""
    from paper_1606_02862_gb300 import workloads as W

    wl = _thermal(n=(16, 16, 16), shape=other, u_th=0.3, species="ions", fields=0.05)
    wl.species[1] = W.SpeciesDef("p", 1.0, W.PROTON_MASS, 3)
    _one_step_parity(orc, wl, MIXED_TOL, sc=(8, 4, 4), threads_per_sc=256)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=2, sc=(8, 4, 4), threads_per_sc=256)


def test_mixed_pcs_energy_conserving_gather(orc):
    from paper_1606_02862_gb300 import workloads as W

    wl = _thermal(n=(16, 16, 16), shape=3, u_th=0.1, fields=0.05)
    wl.species[0] = W.SpeciesDef("e", -1.0, 1.0, 3, True, True)
    _one_step_parity(orc, wl, MIXED_TOL, pre_steps=1, sc=(4, 4, 4), threads_per_sc=128)


def test_mixed_pcs_edge_positions(orc):
    """Particles on and next to cell faces, supercell and box seams, moving
    across them: the 5-node general window."""
    from paper_1606_02862_gb300 import workloads as W

    n = 8
    pts, us = [], []
    for base in ([0.0, 0.0, 0.0], [3.999999, 4.0, 7.9999995], [7.5, 3.5, 0.5], [4.0, 4.0, 4.0],
                 [0.02, 7.97, 3.01]):
        for dirn in ([1, 1, 1], [-1, -1, -1], [1, -1, 0], [0, 0, -1]):
            pts.append(base)
            us.append(0.6 * np.array(dirn, dtype=float))
    box = W.BoxInit(n, n, n, particles=[(np.array(pts), np.array(us), np.full(len(pts), 0.05))], rho_bg=0.0)
    wl = W.Workload("pcs_edges", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 3)], [box])
    _one_step_parity(orc, wl, MIXED_TOL, sc=(4, 4, 4), threads_per_sc=128)


def test_pcs_diagnostics_match_oracle(orc):
    require_gpu()
    wl = _thermal(n=(16, 16, 16), shape=3, u_th=0.1)
    ctx = ctx_from(wl, sc=(4, 4, 4), threads_per_sc=128)
    ctx.step(3)
    st, _ = oracle_state_from_gpu(orc, ctx, wl, 0)
    got, want = ctx.diagnostics(0), st.diagnostics()
    assert abs(got[0] / want[0] - 1) < 1e-6 and abs(got[1] / want[1] - 1) < 1e-6
    assert abs(got[2] - want[2]) < 1e-9 * (1 + abs(want[2]))
    assert abs(got[3] - want[3]) < 1e-5 * np.max(np.abs(st.rho()))
    ctx.close()


def test_pcs_rejected_where_unsupported():
    from paper_1606_02862_gb300 import pic

    require_gpu()
    with pytest.raises(pic.PicError):  # the plain form has CIC and TSC only
        ctx_from(_thermal(n=(8, 8, 8), shape=3), precision=pic.PRECISION_FP64_PLAIN)
    with pytest.raises(pic.PicError):  # no PCS kernel for 8x8x4 supercells
        ctx_from(_thermal(n=(16, 16, 16), shape=3), sc=(8, 8, 4), threads_per_sc=256)
