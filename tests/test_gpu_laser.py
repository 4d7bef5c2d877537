"""The two-species workloads at reduced size: the laser-plasma ones
(a Gaussian pulse along y, a density ramp or an overdense foil, most
supercells empty) and the KHI-like shear flow of the paper's evaluation:
one-step parity with the FP64 oracle, and, for the laser cases, invariants
over a run in which the pulse drives the electrons relativistically."""
import numpy as np
import pytest

from _gpu_helpers import compare_box, ctx_from, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu


def _laser_small():
    from paper_1606_02862_gb300 import workloads as W

    # 32 x 128 x 32 cells, ramp over y in [40, 80), pulse at y = 24 with lambda = 16
    return W.laser_ramp(nx=32, ny=128, nz=32, ppc=2, lam=16.0, a0=3.0, waist=8.0, duration=10.0,
                        y_c=24.0, ramp=(40, 80), n_frac=0.5)


def _foil_small():
    from paper_1606_02862_gb300 import workloads as W

    # 16 x 128 x 16 cells, a 6-cell foil at y = 60, pulse centred 16 cells before it
    return W.foil_overdense(nx=16, ny=128, nz=16, ppc=4, lam=16.0, a0=10.0, waist=6.0, duration=8.0,
                            foil=(60, 66), n_e_over_nc=30.0, pulse_gap=16.0)


def _khi_small():
    from paper_1606_02862_gb300 import workloads as W

    return W.khi(n=16, ppc=4)


@pytest.mark.parametrize("make", [_laser_small, _foil_small, _khi_small], ids=["laser_ramp", "foil", "khi"])
def test_laser_workloads_one_step_parity(orc, make):
    require_gpu()
    wl = make()
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        st, ids = oracle_state_from_gpu(orc, ctx, wl, 0)
        ctx.step(1)
        st.step(1)
        errs = compare_box(st, ids, ctx, wl, 0, tol_field=1e-5, tol_x=1e-5, tol_u=1e-5)
        print("laser parity errors:", errs)
    finally:
        ctx.close()


@pytest.mark.parametrize("make", [_laser_small, _foil_small], ids=["laser_ramp", "foil"])
def test_laser_workloads_invariants(orc, make):
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = make()
    ctx = ctx_from(wl, sc=(8, 4, 4), threads_per_sc=256)
    try:
        b = wl.boxes[0]
        g = orc.grid(b.nx, b.ny, b.nz)
        n0 = [ctx.count_particles(0, s) for s in range(2)]
        q0 = ctx.diagnostics(0)[2]
        res0 = orc.div_e(g, ctx.read_fields(0, pic.FIELD_E)) - ctx.read_fields(0, pic.FIELD_RHO)
        ctx.step(30)
        for s in range(2):
            p = ctx.read_particles(0, s, ids=True)
            assert np.array_equal(np.sort(p["id"]), np.arange(n0[s]))
        d1 = ctx.diagnostics(0)
        assert abs(d1[2] - q0) <= 1e-9 * max(1.0, abs(q0))
        res1 = orc.div_e(g, ctx.read_fields(0, pic.FIELD_E)) - ctx.read_fields(0, pic.FIELD_RHO)
        # the pulse's own divergence is in res0; the step keeps div E - rho
        scale = max(np.max(np.abs(res0)), np.max(np.abs(ctx.read_fields(0, pic.FIELD_RHO))))
        assert np.max(np.abs(res1 - res0)) <= 2e-5 * scale
        p = ctx.read_particles(0, 0)
        assert np.max(np.linalg.norm(p["u"], axis=1)) > 0.5  # the pulse did push the electrons
    finally:
        ctx.close()
