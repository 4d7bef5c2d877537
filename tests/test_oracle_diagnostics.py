"""Pins of the oracle's FP64 diagnostics against closed forms.

  * a uniform field E0 (and B0) over the whole box has energy
    (E0^2 + B0^2) / 2 times the box volume;
  * a particle with |u| = sqrt(3) has gamma = 2, so w m (gamma - 1) = w m;
  * for |u| << 1 the kinetic energy tends to w m |u|^2 / 2 with a relative
    correction of -|u|^2 / 4 (gamma - 1 = u^2/2 - u^4/8 + ...);
  * the charge density of one particle integrates to q w (partition of unity
    times 1 / V_cell, times V_cell), for every position and both shapes.
"""
import math

import numpy as np
import pytest


def test_field_energy_of_uniform_fields(orc):
    n = (6, 5, 4)
    h = (1.0, 0.5, 2.0)
    E = np.zeros((3, n[2], n[1], n[0]))
    B = np.zeros_like(E)
    E[1] = 0.3
    B[2] = -0.7
    st = orc.State(*n, 0.1, dx=h, E=E, B=B)
    vol = n[0] * n[1] * n[2] * h[0] * h[1] * h[2]
    assert abs(st.diagnostics()[0] - 0.5 * (0.09 + 0.49) * vol) < 1e-12


@pytest.mark.parametrize("m,w", [(1.0, 0.25), (1836.0, 3.0)])
def test_kinetic_energy_closed_forms(orc, m, w):
    u = np.array([[1.0, 1.0, 1.0]])  # |u| = sqrt(3), gamma = 2
    sp = orc.Species(q=-1.0, m=m, order=2, x=np.array([[1.0, 1.0, 1.0]]), u=u, w=np.array([w]))
    st = orc.State(4, 4, 4, 0.1, species=[sp])
    assert abs(st.diagnostics()[1] - w * m) < 1e-12 * w * m
    small = 1e-4
    sp.u[...] = [[small, 0.0, 0.0]]
    ek = st.diagnostics()[1]
    nonrel = 0.5 * w * m * small ** 2
    assert abs(ek / nonrel - 1.0 + 0.25 * small ** 2) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_rho_integrates_to_the_charge(orc, order):
    rng = np.random.default_rng(80 + order)
    n = 6
    h = (0.8, 1.1, 1.3)
    g = orc.grid(n, n, n, h)
    for x in rng.uniform(0, n, (20, 3)):
        rho = np.zeros((n, n, n))
        orc.deposit_rho(g, order, -2.0, np.array([x]), np.array([0.7]), rho)
        assert abs(rho.sum() * h[0] * h[1] * h[2] - (-2.0 * 0.7)) < 1e-13
