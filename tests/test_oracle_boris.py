"""Pin of the oracle's Boris push and move against the closed form of the
discrete gyration in a uniform magnetic field (Boris 1970, named in Sec. 4).

With E = 0 and a uniform B, the Boris rotation turns the perpendicular
momentum by exactly theta = 2 atan(omega_c dt / (2 gamma)) per step, with
omega_c = |q| B / m, in the sense of the Lorentz force (counter-clockwise
about +B for an electron), and keeps |u| and gamma exactly.  The positions
x^{n+1} = x^n + dt u^{n+1/2} / gamma are then the vertices of a regular
polygon with side L = |u_perp| dt / gamma, inscribed in a circle of radius
R = L / (2 sin(theta / 2)), closing after 2 pi / theta steps, while the
parallel coordinate advances by dt u_par / gamma per step.

The particle has weight 0, so it deposits no current and the fields stay
uniform through the full coupled step.
"""
import math

import numpy as np
import pytest


def _run(orc, q, m, B0, u0, x0, dt, nsteps, order=2, n=16):
    B = np.zeros((3, n, n, n))
    B[2] = B0
    sp = orc.Species(q=q, m=m, order=order, x=np.array([x0]), u=np.array([u0]),
                     w=np.array([0.0]))
    st = orc.State(n, n, n, dt, B=B, species=[sp])
    xs = [sp.x[0].copy()]
    us = [sp.u[0].copy()]
    for _ in range(nsteps):
        st.step(1)
        xs.append(sp.x[0].copy())
        us.append(sp.u[0].copy())
    xs = np.array(xs)
    # unwrap the periodic positions
    d = np.diff(xs, axis=0)
    d -= n * np.round(d / n)
    xs = np.concatenate([xs[:1], xs[0] + np.cumsum(d, axis=0)])
    return xs, np.array(us), st


@pytest.mark.parametrize("q,m,B0", [(-1.0, 1.0, 0.1), (1.0, 1836.15, 50.0), (-1.0, 1.0, 2.0)])
def test_boris_gyration_closed_form(orc, q, m, B0):
    dt = 0.5 / math.sqrt(3.0)
    u0 = np.array([0.3, -0.1, 0.05]) * (1.0 if m == 1.0 else 30.0)
    x0 = np.array([8.2, 7.7, 3.1])
    nsteps = 120
    xs, us, _ = _run(orc, q, m, B0, u0, x0, dt, nsteps)

    gamma = math.sqrt(1.0 + u0 @ u0)
    theta = 2.0 * math.atan(abs(q) * B0 * dt / (2.0 * m * gamma))
    uperp = math.hypot(u0[0], u0[1])
    L = uperp * dt / gamma
    R = L / (2.0 * math.sin(theta / 2.0))

    # |u| and gamma are invariants of the rotation
    assert np.max(np.abs(np.linalg.norm(us, axis=1) - np.linalg.norm(u0))) < 1e-14 * (1 + np.linalg.norm(u0))
    # angle per step, sense of the Lorentz force: rotation about -q B
    ang = np.arctan2(us[:, 1], us[:, 0])
    dang = np.diff(ang)
    dang = (dang + np.pi) % (2 * np.pi) - np.pi
    sense = -np.sign(q) * np.sign(B0)
    assert np.max(np.abs(dang - sense * theta)) < 1e-12
    # parallel motion
    assert np.max(np.abs(np.diff(xs[:, 2]) - dt * u0[2] / gamma)) < 1e-12
    # polygon vertices on a circle of radius R about a fixed centre
    # centre from the closed form: x^n = c + R * (unit vector at angle phi_n)
    phi0 = math.atan2(u0[1], u0[0])
    # the chord x^{n+1} - x^n has direction phi0 + (n+1) theta*sense;
    # the vertex x^n sits at angle (phi0 + (n + 1/2) sense theta) - sense pi/2 from the centre
    a0 = phi0 + 0.5 * sense * theta - sense * math.pi / 2.0
    centre = xs[0, :2] - R * np.array([math.cos(a0), math.sin(a0)])
    for nn in range(nsteps + 1):
        an = a0 + nn * sense * theta
        want = centre + R * np.array([math.cos(an), math.sin(an)])
        assert np.allclose(xs[nn, :2], want, rtol=0, atol=1e-10 * max(1.0, R)), nn
    # the radius is the discrete one, not the continuum Larmor radius (they
    # differ by O(theta^2)); check the discrete value is the one realised
    rad = np.linalg.norm(xs[:, :2] - centre, axis=1)
    assert np.max(np.abs(rad - R)) < 1e-10 * max(1.0, R)


def test_boris_period_in_steps(orc):
    """Choose B so that theta = 2 pi / 40 exactly: after 40 steps the particle
    is back at its start (to roundoff)."""
    dt = 0.5 / math.sqrt(3.0)
    u0 = np.array([0.2, 0.0, 0.0])
    gamma = math.sqrt(1.0 + u0 @ u0)
    theta = 2.0 * math.pi / 40.0
    B0 = math.tan(theta / 2.0) * 2.0 * gamma / dt  # electron, m = 1
    xs, us, _ = _run(orc, -1.0, 1.0, B0, u0, np.array([8.0, 8.0, 8.0]), dt, 40, order=1)
    assert np.allclose(us[40], u0, rtol=0, atol=1e-13)
    assert np.allclose(xs[40], xs[0], rtol=0, atol=1e-11)
    assert not np.allclose(xs[20], xs[0], atol=1e-3)


def test_boris_electric_kick_is_exact_for_b0(orc):
    """With B = 0 the push is u^{n+1/2} = u^{n-1/2} + (q dt / m) E exactly."""
    E = np.array([0.01, -0.02, 0.03])
    u = np.array([0.5, 0.1, -0.2])
    out = orc.boris(-1.0, 1.0, 0.3, E, np.zeros(3), u)
    assert np.allclose(out, u - 0.3 * E, rtol=0, atol=1e-16)
