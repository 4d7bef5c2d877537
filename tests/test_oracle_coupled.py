"""Pins of the oracle's full coupled step (gather -> Boris -> move ->
Esirkepov -> Yee, the PIC cycle of Sec. 2.1 and Sec. 4).

1. Cold plasma oscillation at k = 0: electrons on an identical lattice (one
   per cell, same offset in every cell, so the state stays exactly uniform),
   all with u = u0 x, over a fixed neutralising background.  Uniform E_x
   then obeys the leapfrog oscillator exactly (up to O(u0^2) relativistic
   terms): E^{n+1} - 2 E^n + E^{n-1} = -(omega_p dt)^2 E^n, so
   sin(omega dt / 2) = omega_p dt / 2 with omega_p^2 = n q^2 / m; a wrong
   current sign makes it grow instead.  Any three consecutive samples give
   cos(omega dt) = (E^{n+1} + E^{n-1}) / (2 E^n).
2. Gauss's law is kept: div E - rho does not change from step to step (the
   charge-conserving deposit plus the Yee update), for a thermal plasma.
3. Total charge is constant, and total energy is conserved to the accuracy
   of the explicit scheme over a short run.
"""
import math

import numpy as np
import pytest


def test_cold_plasma_frequency(orc):
    n = 4
    dens = 0.01
    dt = 0.5 / math.sqrt(3.0)
    u0 = 1e-3
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1) + np.array([0.3, 0.6, 0.45])
    u = np.tile([u0, 0.0, 0.0], (x.shape[0], 1))
    w = np.full(x.shape[0], dens)  # one particle per cell of volume 1
    sp = orc.Species(q=-1.0, m=1.0, order=2, x=x, u=u, w=w)
    st = orc.State(n, n, n, dt, species=[sp], rho_bg=dens)
    ex = []
    for _ in range(400):
        st.step(1)
        ex.append(st.E[0].mean())
        # exactly uniform state
        # (roundoff of the deposit sums only; E_x itself is ~1e-4)
        assert np.max(np.abs(st.E[0] - st.E[0].mean())) < 1e-15
        assert np.max(np.abs(st.E[1:])) < 1e-15 and np.max(np.abs(st.B)) < 1e-15
    ex = np.array(ex)
    wp = math.sqrt(dens)
    omega = 2.0 / dt * math.asin(wp * dt / 2.0)
    big = np.abs(ex[1:-1]) > 0.5 * np.max(np.abs(ex))
    cosw = (ex[2:] + ex[:-2])[big] / (2 * ex[1:-1][big])
    est = np.arccos(np.clip(cosw, -1, 1)) / dt
    assert np.max(np.abs(est / omega - 1.0)) < 1e-5
    # amplitude: the oscillator is neutral, no growth or damping
    assert abs(np.max(np.abs(ex[:200])) / np.max(np.abs(ex[200:])) - 1.0) < 1e-3
    # the first step: E^1 = -dt J^{1/2} with J = q n v
    gam = math.sqrt(1 + u0 * u0)
    assert abs(ex[0] - (-dt * (-1.0) * dens * u0 / gam)) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_gauss_law_residual_is_invariant(orc, order):
    n = 8
    dt = 0.5 / math.sqrt(3.0)
    rng = np.random.default_rng(60 + order)
    x = rng.uniform(0, n, (600, 3))
    u = rng.normal(0, 0.2, (600, 3))
    w = np.full(600, 0.05)
    xi = rng.uniform(0, n, (300, 3))
    ions = orc.Species(q=1.0, m=1836.0, order=order, x=xi, u=np.zeros((300, 3)), w=np.full(300, 0.1))
    ele = orc.Species(q=-1.0, m=1.0, order=order, x=x, u=u, w=w)
    E0 = rng.normal(0, 1e-3, (3, n, n, n))
    B0 = rng.normal(0, 1e-3, (3, n, n, n))
    st = orc.State(n, n, n, dt, E=E0, B=B0, species=[ele, ions])
    res0 = orc.div_e(st.g, st.E) - st.rho()
    q0 = st.diagnostics()[2]
    for _ in range(5):
        st.step(1)
        res = orc.div_e(st.g, st.E) - st.rho()
        assert np.max(np.abs(res - res0)) < 1e-13
        assert abs(st.diagnostics()[2] - q0) < 1e-12


def test_energy_is_conserved_over_a_short_run(orc):
    n = 8
    dt = 0.5 / math.sqrt(3.0)
    rng = np.random.default_rng(70)
    npart = 2 * n ** 3
    dens = 0.05
    x = rng.uniform(0, n, (npart, 3))
    u = rng.normal(0, 0.05, (npart, 3))
    ele = orc.Species(q=-1.0, m=1.0, order=2, x=x, u=u, w=np.full(npart, dens / 2))
    st = orc.State(n, n, n, dt, species=[ele], rho_bg=dens)
    st.step(1)
    e0 = st.diagnostics()
    st.step(30)
    e1 = st.diagnostics()
    tot0 = e0[0] + e0[1]
    tot1 = e1[0] + e1[1]
    assert abs(tot1 / tot0 - 1.0) < 0.03
    assert e1[0] > 0.0  # thermal noise does build a field
