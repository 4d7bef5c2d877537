"""Pins of the oracle's open-y boundaries (damping absorber, laser antenna,
particle removal at the y faces, moving window) against what the Yee
equations and the definitions fix, independently of the oracle's own code:

  * the absorber leaves the interior untouched, is mirror symmetric, and
    takes a vacuum pulse out of the box with a reflection below 1e-6 in
    energy;
  * a plane current sheet radiates the same field to both sides, and the
    wave leaving it is the discrete plane-wave solution of the Yee scheme
    E0 env(t - d/v_g) cos(kappa d - omega (t - t0)), with kappa and v_g from
    the Yee dispersion relation -- a wrong sheet factor (cos(kappa/2), 8 %
    here), sign or plane fails it;
  * a particle that crosses a y face is gone after the step, the others stay;
  * a window shift is a translation: a shifted run equals the unshifted run
    of a box that is long enough, inside the region no boundary can reach.
"""
import numpy as np
import pytest

DT = 0.5 / np.sqrt(3.0)


def _pulse_state(orc, ny=160, absorber=None, centre=80.0):
    """A Gaussian vacuum pulse moving +y (Ex, Bz = -Ex at the Bz position and
    half a step earlier), 1D-like: 4 x ny x 4 cells."""
    st = orc.State(4, ny, 4, DT, absorber=absorber)
    y = np.arange(ny, dtype=float)
    k = 2 * np.pi / 8.0
    env = lambda yy: np.exp(-((yy - centre) / 8.0) ** 2)  # noqa: E731
    st.E[0] = (env(y) * np.cos(k * (y - centre)))[None, :, None]
    yb = y + 0.5 - 0.5 * DT
    st.B[2] = (-(env(yb) * np.cos(k * (yb - centre))))[None, :, None]
    return st


def test_absorber_leaves_interior_alone_and_is_mirror_symmetric(orc):
    A, sig, ny = 16, 0.7, 64
    g = orc.grid(4, ny, 4)
    E = np.ones((3, 4, ny, 4))
    B = np.ones((3, 4, ny, 4))
    orc.absorb_y(g, A, sig, E, B)
    # interior planes (no staggered position inside a layer) are untouched
    assert np.all(E[:, :, A + 1:ny - A, :] == 1.0) and np.all(B[:, :, A + 1:ny - A, :] == 1.0)
    # the factor falls monotonically towards both faces
    ex = E[0, 0, :, 0]
    assert np.all(np.diff(ex[:A + 1]) >= 0) and np.all(np.diff(ex[ny - A:]) <= 0)
    assert ex[0] == pytest.approx(np.exp(-sig)) and ex[A] == 1.0
    # mirror symmetry about the box centre: integer-y components at j <-> ny - j,
    # half-y components (Ey, Bx, Bz) at j + 1/2 <-> ny - j - 1/2
    for F, c, half in ((E, 0, False), (E, 1, True), (E, 2, False), (B, 0, True), (B, 1, False), (B, 2, True)):
        v = F[c, 0, :, 0]
        if half:
            assert np.allclose(v, v[::-1], rtol=0, atol=1e-15)
        else:
            assert np.allclose(v[1:], v[1:][::-1], rtol=0, atol=1e-15)
    # no damping: the identity
    E2, B2 = np.full((3, 4, ny, 4), 3.0), np.full((3, 4, ny, 4), -2.0)
    orc.absorb_y(g, A, 0.0, E2, B2)
    assert np.all(E2 == 3.0) and np.all(B2 == -2.0)


def test_absorber_takes_a_pulse_out_of_the_box(orc):
    A = 32
    st = _pulse_state(orc, absorber=(A, 1.0))
    ref = _pulse_state(orc)  # the same pulse, periodic, no absorber
    W0 = st.diagnostics()[0]
    worst = 0.0
    for n in range(int(200 / DT)):
        st.step(1)
        ref.step(1)
        if n < 36:
            # the Yee stencil carries a change at most one cell per step: what the
            # layers (y < 32, y >= 128) did has not reached 70 <= y < 90 yet
            assert np.array_equal(st.E[:, :, 70:90], ref.E[:, :, 70:90])
            assert np.array_equal(st.B[:, :, 70:90], ref.B[:, :, 70:90])
        if st.t > 120:  # a reflection off the layer would be back in the interior by now
            wi = 0.5 * np.sum(st.E[:, :, A:-A] ** 2 + st.B[:, :, A:-A] ** 2)
            worst = max(worst, wi / W0)
    assert worst < 1e-6
    assert st.diagnostics()[0] < 1e-9 * W0


def _antenna_run(orc, a, ny=400, steps=None):
    st = orc.State(4, ny, 4, DT, antenna=a)
    st.step(steps if steps is not None else int(round(a.t0 / DT)) + 20)
    return st


def test_plane_antenna_radiates_the_discrete_plane_wave(orc):
    lam = 8.0
    om = 2 * np.pi / lam
    kappa = 2 * np.arcsin(np.sin(om * DT / 2) / DT)  # Yee dispersion along y, dy = 1
    vg = np.cos(kappa / 2) / np.cos(om * DT / 2)      # d omega / d kappa
    j0, tau, t0 = 200, 60.0, 180.0
    a = orc.Antenna(ja=j0, E0=1.0, omega=om, tau=tau, t0=t0)
    st = _antenna_run(orc, a)
    ex = st.E[0, 0, :, 0]
    m = np.arange(1, 150)
    assert np.max(np.abs(ex[j0 + m] - ex[j0 - m])) <= 1e-13  # both sides alike
    assert np.max(np.abs(st.E[0] - st.E[0, :1, :, :1])) == 0.0  # a plane sheet: uniform in x, z
    d = np.arange(0, 40)
    pred = np.exp(-((st.t - t0 - d / vg) / tau) ** 2) * np.cos(kappa * d - om * (st.t - t0))
    assert np.max(np.abs(ex[j0 + d] - pred)) < 1e-2
    # the field leaving the sheet has amplitude E0: the envelope peak passes d = 24
    peak = 0.0
    st2 = orc.State(4, 400, 4, DT, antenna=a)
    for _ in range(int((t0 + 24 / vg + 2 * lam) / DT)):
        st2.step(1)
        peak = max(peak, abs(st2.E[0, 0, j0 + 24, 0]))
    assert 0.98 < peak <= 1.0 + 1e-3


def test_antenna_j0_rejects_an_unresolved_frequency(orc):
    with pytest.raises(ValueError):
        orc.antenna_j0(1.0, 2.0 / DT, DT)  # (dy/dt) sin(omega dt / 2) > 1
    # the plane-wave limit: a slow sheet radiates -K/2 to each side, K = J0 dy
    assert orc.antenna_j0(1.0, 1e-6, DT) == pytest.approx(-2.0, rel=1e-9)


def test_gaussian_antenna_profile_is_centred(orc):
    a = orc.Antenna(ja=10, E0=1.0, omega=2 * np.pi / 16, w0=3.0, xc=8.0, zc=8.0, tau=0.0, t0=0.0)
    g = orc.grid(16, 32, 16)
    J = np.zeros((3, 16, 32, 16))
    orc.antenna(g, a, DT, 0.0, J)
    jx = J[0, :, 10, :]
    assert np.count_nonzero(J[0]) == np.count_nonzero(jx) and not J[1].any() and not J[2].any()
    # Ex sits at x = i + 1/2: the profile is symmetric about x = 8 between i = 7 and i = 8
    i = np.arange(16) + 0.5
    k = np.arange(16)
    prof = np.exp(-((i[None, :] - 8.0) ** 2 + (k[:, None] - 8.0) ** 2) / 9.0)
    assert np.allclose(jx / jx[8, 7], prof / prof[8, 7], rtol=1e-12)


def test_open_y_removes_particles_that_cross_a_y_face(orc):
    ny = 16
    x = np.array([[4.5, 15.95, 4.5], [4.5, 0.03, 4.5], [4.5, 8.0, 4.5], [4.5, 15.9, 4.5]])
    u = np.array([[0.0, 0.9, 0.0], [0.0, -0.9, 0.0], [0.0, 0.9, 0.0], [0.0, -0.9, 0.0]])
    sp = orc.Species(-1.0, 1.0, 2, x, u, np.full(4, 0.1))
    sp.ids = np.arange(4)
    st = orc.State(8, ny, 8, DT, species=[sp], open_y=True)
    st.step(1)
    assert list(sp.ids) == [2, 3]
    assert np.all((sp.x[:, 1] >= 0) & (sp.x[:, 1] < ny))
    assert np.any(st.J[1] != 0.0)  # the leavers deposited before they went
    # periodic y: nobody leaves
    sp2 = orc.Species(-1.0, 1.0, 2, x, u, np.full(4, 0.1))
    st2 = orc.State(8, ny, 8, DT, species=[sp2])
    st2.step(1)
    assert sp2.x.shape[0] == 4


def test_window_shift_is_a_translation(orc):
    """Box A (ny = 64) shifted by 8 after 10 steps against box B (ny = 72, the
    same initial state in its first 64 planes): after the shift A's plane j is
    B's plane j + 8, exactly, wherever no face or wrap of either box can have
    reached in the steps taken (the light cone)."""
    rng = np.random.default_rng(3)
    nx, nz = 8, 8
    ny_a, ny_b, m = 64, 72, 8
    E = np.zeros((3, nz, ny_b, nx))
    E[:, :, 16:48, :] = rng.normal(0, 0.01, (3, nz, 32, nx))
    x = np.column_stack([rng.uniform(0, nx, 400), rng.uniform(20, 44, 400), rng.uniform(0, nz, 400)])
    u = rng.normal(0, 0.05, (400, 3))
    w = np.full(400, 0.01)

    def make(ny):
        sp = orc.Species(-1.0, 1.0, 2, x, u, w)
        sp.ids = np.arange(400)
        return orc.State(nx, ny, nz, DT, E=E[:, :, :ny, :].copy(), species=[sp], rho_bg=0.0), sp

    a, spa = make(ny_a)
    b, spb = make(ny_b)
    a.step(10)
    b.step(10)
    a.shift_window(m)
    a.step(6)
    b.step(6)
    # 16 steps at c dt < 0.3 cells: nothing from y < 16 or y > 48 reaches 24 .. 40
    sl_a, sl_b = slice(24 - m, 40 - m), slice(24, 40)
    assert np.max(np.abs(a.E[:, :, sl_a] - b.E[:, :, sl_b])) <= 1e-15
    assert np.max(np.abs(a.B[:, :, sl_a] - b.B[:, :, sl_b])) <= 1e-15
    # particles: the same ones, translated
    assert np.array_equal(np.sort(spa.ids), np.sort(spb.ids))
    oa, ob = np.argsort(spa.ids), np.argsort(spb.ids)
    assert np.allclose(spa.x[oa] + [0, m, 0], spb.x[ob], rtol=0, atol=1e-12)
    assert np.allclose(spa.u[oa], spb.u[ob], rtol=0, atol=1e-14)
    # a shift drops what falls out at the bottom and zeroes the planes entering at the top
    c, spc = make(ny_a)
    spc.x[:5, 1] = 3.0
    c.shift_window(m)
    assert spc.x.shape[0] == 395 and not c.E[:, :, ny_a - m:].any()
