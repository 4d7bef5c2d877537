"""Multi-step invariants of the CUDA path, and its error reporting.

Over many steps FP32 and FP64 thermal trajectories separate, so the checks
are the properties the method keeps at any step count: particle count and
identity (every id exactly once, frames never duplicate or drop a
particle), total weight and charge, positions inside the box, and Gauss's
law residual div E - rho unchanged (charge-conserving Esirkepov deposit +
Yee update) to FP32 roundoff.  Device-side conditions (frame pool or move
buffer exhausted) and bad input come back as status codes, never as a
fault.
"""
import numpy as np
import pytest

from _gpu_helpers import ctx_from, require_gpu

pytestmark = pytest.mark.gpu


def _wl(n=(16, 16, 16), ppc=4, u_th=0.3, shape=2, seed=3):
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    xe = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    xi = W.uniform_in_cells(rng, nx, ny, nz, ppc)
    w = np.full(xe.shape[0], 0.02 / ppc)
    parts = [(xe, W.maxwellian(rng, xe.shape[0], u_th), w),
             (xi, W.maxwellian(rng, xi.shape[0], u_th / 40), w.copy())]
    sp = [W.SpeciesDef("e", -1.0, 1.0, shape), W.SpeciesDef("p", 1.0, W.PROTON_MASS, shape)]
    return W.Workload("inv", W.DT_HALF_COURANT, sp, [W.BoxInit(nx, ny, nz, particles=parts)])


@pytest.mark.parametrize("sc,threads", [((4, 4, 4), 64), ((8, 8, 4), 128)])
def test_invariants_over_many_steps(sc, threads):
    from paper_1606_02862_gb300 import pic

    require_gpu()
    wl = _wl()
    ctx = ctx_from(wl, sc=sc, threads_per_sc=threads)
    d0 = ctx.diagnostics(0)
    rho0 = ctx.read_fields(0, pic.FIELD_RHO)
    E0 = ctx.read_fields(0, pic.FIELD_E)
    n0 = [ctx.count_particles(0, s) for s in range(2)]
    w0 = [ctx.read_particles(0, s)["w"].sum() for s in range(2)]
    ctx.step(40)
    N = np.array(wl.boxes[0].particles[0][0].shape)  # noqa: F841
    box = np.array([16, 16, 16], dtype=float)
    for s in range(2):
        p = ctx.read_particles(0, s, ids=True)
        assert p["x"].shape[0] == n0[s]
        assert np.array_equal(np.sort(p["id"]), np.arange(n0[s]))
        assert np.all(p["x"] >= 0) and np.all(p["x"] < box)
        assert abs(p["w"].sum() - w0[s]) <= 1e-12 * w0[s]
    d1 = ctx.diagnostics(0)
    assert abs(d1[2] - d0[2]) <= 1e-9 * max(1.0, abs(d0[2]))
    # div E - rho unchanged (compare the residual fields, not only their max)
    from oracle import oracle as orc

    g = orc.grid(16, 16, 16)
    res0 = orc.div_e(g, E0) - rho0
    res1 = orc.div_e(g, ctx.read_fields(0, pic.FIELD_E)) - ctx.read_fields(0, pic.FIELD_RHO)
    scale = np.max(np.abs(rho0))
    assert np.max(np.abs(res1 - res0)) <= 2e-5 * scale
    ctx.close()


def test_frame_pool_exhaustion_is_reported():
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    rng = np.random.default_rng(4)
    # one frame of particles at the +x face of supercell (0,0,0), all leaving
    x = np.column_stack([rng.uniform(3.8, 3.99, 64), rng.uniform(0.2, 3.8, 64), rng.uniform(0.2, 3.8, 64)])
    u = np.tile([3.0, 0.0, 0.0], (64, 1))
    wl = W.Workload("pool", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)],
                    [W.BoxInit(16, 16, 16, particles=[(x, u, np.full(64, 0.01))])])
    ctx = ctx_from(wl, pool_frames=1)
    with pytest.raises(pic.PicError) as ei:
        ctx.step(2)
    assert ei.value.status == 5  # PIC_ERR_FRAME_POOL
    with pytest.raises(pic.PicError) as ei:
        ctx.step(1)
    assert ei.value.status == 7  # PIC_ERR_STATE: poisoned
    ctx.close()


def test_move_buffer_overflow_is_reported():
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    rng = np.random.default_rng(5)
    wl = W.Workload("cap", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)],
                    [W.BoxInit(16, 16, 16)])
    ctx = ctx_from(wl, move_capacity=64)
    for x0 in (3.9, 7.9):  # two loads of 64: the move buffer stays at 64
        x = np.column_stack([np.full(64, x0), rng.uniform(0.2, 3.8, 64), rng.uniform(0.2, 3.8, 64)])
        ctx.load_particles(0, 0, x, np.tile([3.0, 0.0, 0.0], (64, 1)), np.full(64, 0.01))
    with pytest.raises(pic.PicError) as ei:
        ctx.step(1)
    assert ei.value.status == 8  # PIC_ERR_CAPACITY
    ctx.close()


def test_non_finite_input_is_rejected_and_context_survives():
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    for prec in (pic.PRECISION_MIXED, pic.PRECISION_FP64_PLAIN):
        wl = W.Workload("nan", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)],
                        [W.BoxInit(8, 8, 8)])
        ctx = ctx_from(wl, precision=prec)
        x = np.array([[1.0, 2.0, np.nan], [2.0, 2.0, 2.0]])
        with pytest.raises(pic.PicError) as ei:
            ctx.load_particles(0, 0, x, np.zeros((2, 3)))
        assert ei.value.status == 1
        assert ctx.count_particles(0, 0) == 0
        ctx.load_particles(0, 0, np.array([[1.0, 2.0, 3.0]]), np.zeros((1, 3)))
        ctx.step(2)
        assert ctx.count_particles(0, 0) == 1
        ctx.close()


def test_load_wraps_positions_and_reads_back_exactly():
    """Positions outside [0, N) wrap on load; read-back of a freshly loaded
    state reproduces the input to FP32 offset precision."""
    from paper_1606_02862_gb300 import workloads as W

    require_gpu()
    rng = np.random.default_rng(6)
    x = rng.uniform(-20, 40, (1000, 3))
    u = rng.normal(0, 0.1, (1000, 3))
    w = rng.uniform(0.5, 1.5, 1000)
    wl = W.Workload("wrap", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 1)],
                    [W.BoxInit(16, 8, 12, particles=[(x, u, w)])])
    ctx = ctx_from(wl)
    p = ctx.read_particles(0, 0, ids=True)
    o = np.argsort(p["id"])
    N = np.array([16, 8, 12], dtype=float)
    want = x - N * np.floor(x / N)
    d = p["x"][o] - want
    d -= N * np.round(d / N)
    assert np.max(np.abs(d)) < 1e-6
    assert np.max(np.abs(p["u"][o] - u)) < 1e-7 * np.max(np.abs(u)) + 1e-12
    assert np.max(np.abs(p["w"][o] - w)) < 1e-7
    ctx.close()
