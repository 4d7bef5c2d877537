"""The library's own tuner (pic_options sc = 0,0,0 / threads_per_sc = 0),
through the C ABI.

Before its first step a context left to the tuner times every supercell
shape and thread count the push kernel is built for on its loaded state and
moves into the fastest.  Checked here:
  * the configuration it reports (pic_info) is one the kernel supports and
    that fits the box, and several configurations were timed;
  * the move keeps the state: the first step after tuning matches the FP64
    oracle started from the state read back before it (the mixed form's
    per-step tolerance), every particle present once with its id;
  * a second context of the same kind of state takes the cached result
    (no configuration timed) and the same configuration;
  * threads_per_sc = 0 with a given supercell tunes the thread count only.
"""
import numpy as np
import pytest

from _gpu_helpers import compare_box, oracle_state_from_gpu, require_gpu

pytestmark = pytest.mark.gpu

SUPPORTED = {((4, 4, 4), 64), ((4, 4, 4), 128), ((4, 4, 4), 256), ((8, 4, 4), 128), ((8, 4, 4), 256),
             ((8, 8, 4), 128), ((8, 8, 4), 256), ((8, 8, 8), 256)}


def _wl(seed=31):
    from paper_1606_02862_gb300 import workloads as W

    n = (32, 16, 16)
    rng = np.random.default_rng(seed)
    x = W.uniform_in_cells(rng, *n, 4)
    u = W.maxwellian(rng, x.shape[0], 0.1)
    w = np.full(x.shape[0], 0.0025)
    E = rng.normal(0, 0.01, (3, n[2], n[1], n[0]))
    B = rng.normal(0, 0.01, (3, n[2], n[1], n[0]))
    box = W.BoxInit(*n, particles=[(x, u, w)], E=E, B=B, rho_bg=0.01)
    return W.Workload("tuned", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [box])


def test_tuned_context_reports_a_fitting_configuration_and_keeps_its_state(orc):
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _wl()
    ctx = pic.from_workload(wl, sc=(0, 0, 0), threads_per_sc=0, track_ids=True)
    try:
        assert ctx.config() == ((4, 4, 4), 128)  # before the first step
        st, ids = oracle_state_from_gpu(orc, ctx, wl, 0)
        ctx.step(1)  # tunes, then steps
        sc, threads = ctx.config()
        assert (sc, threads) in SUPPORTED
        assert all(g % e == 0 for g, e in zip((32, 16, 16), sc))
        assert ctx.info(pic.INFO_TUNE_TRIALS) >= 2
        st.step(1)
        errs = compare_box(st, ids, ctx, wl, 0, tol_field=1e-5, tol_x=1e-5, tol_u=1e-5)
        print("tuned", sc, threads, errs)
        ctx.step(3)  # and it keeps stepping
        assert ctx.count_particles(0, 0) == ids[0].size
    finally:
        ctx.close()
    again = pic.from_workload(_wl(seed=32), sc=(0, 0, 0), threads_per_sc=0)
    try:
        again.step(1)
        assert again.info(pic.INFO_TUNE_TRIALS) == 0  # same kind of state: the cached result
        assert again.config() == (sc, threads)
    finally:
        again.close()


def test_threads_only_tuning_keeps_the_supercell():
    require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _wl(seed=33)
    wl.boxes[0].particles = [(p[0], p[1], p[2] * 2.0) for p in wl.boxes[0].particles]
    ctx = pic.from_workload(wl, sc=(8, 4, 4), threads_per_sc=0, track_ids=True)
    try:
        ctx.step(2)
        sc, threads = ctx.config()
        assert sc == (8, 4, 4) and threads in (128, 256)
        assert ctx.count_particles(0, 0) == wl.boxes[0].particles[0][0].shape[0]
    finally:
        ctx.close()
