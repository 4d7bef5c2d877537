"""Pins of the oracle's particle shapes and field gather (Sec. 4 names TSC
and a product-of-1D-weights gather; CIC is the linear shape).

What fixes the values independently of the oracle's code:
  * B-spline identities: every shape sums to one over the integer grid points
    and reproduces the first moment (sum of n S(x - n) is x), for any x;
  * the support widths (2 points for CIC, 3 for TSC, 4 for PCS), the second
    moment of the B-spline of order n, (n + 1) / 12, and the textbook values
    at the centre and at the half-cell points;
  * a gather of a uniform field returns the field; a gather of a field that
    is linear in space, sampled at each component's staggered Yee position,
    returns the linear function at the particle (both shapes are symmetric
    splines and so reproduce linear functions exactly).
"""
import numpy as np
import pytest


@pytest.mark.parametrize("order", [1, 2, 3])
def test_partition_of_unity_and_first_moment(orc, order):
    rng = np.random.default_rng(1)
    for x in np.concatenate([rng.uniform(-5, 5, 200), [0.0, 0.5, -0.5, 1.0, 2.5]]):
        nodes = np.arange(np.floor(x) - 4, np.floor(x) + 5)
        s = np.array([orc.shape(order, x - n) for n in nodes])
        assert np.all(s >= 0.0)
        assert abs(s.sum() - 1.0) < 1e-15
        assert abs((nodes * s).sum() - x) < 1e-13
        assert np.count_nonzero(s) <= order + 1
        # second moment of the B-spline of order n: variance (n + 1) / 12
        if order > 1:
            assert abs((((x - nodes) ** 2) * s).sum() - (order + 1) / 12.0) < 1e-13


def test_textbook_values():
    import oracle as orc

    # CIC: linear tent of half-width 1
    assert orc.shape(1, 0.0) == 1.0 and orc.shape(1, 1.0) == 0.0 and orc.shape(1, -0.25) == 0.75
    # TSC (Hockney & Eastwood): 3/4 at the centre, 1/2 at half a cell, 1/8 at one cell, 0 at 3/2
    assert orc.shape(2, 0.0) == 0.75
    assert orc.shape(2, 0.5) == 0.5 and orc.shape(2, -0.5) == 0.5
    assert orc.shape(2, 1.0) == 0.125 and orc.shape(2, -1.0) == 0.125
    assert orc.shape(2, 1.5) == 0.0 and orc.shape(2, 2.0) == 0.0
    # PCS (the cubic B-spline): 2/3 at the centre, 1/6 at one cell, 1/48 at 3/2, 0 at 2
    assert orc.shape(3, 0.0) == pytest.approx(2.0 / 3.0, abs=1e-16)
    assert orc.shape(3, 1.0) == pytest.approx(1.0 / 6.0, abs=1e-16)
    assert orc.shape(3, -1.5) == pytest.approx(1.0 / 48.0, abs=1e-16)
    assert orc.shape(3, 0.5) == pytest.approx(23.0 / 48.0, abs=1e-16)
    assert orc.shape(3, 2.0) == 0.0 and orc.shape(3, -2.5) == 0.0
    # continuity of the spline and of its slope at |d| = 1/2
    eps = 1e-7
    assert abs(orc.shape(2, 0.5 - eps) - 0.5) < 1.01 * eps
    assert abs(orc.shape(2, 0.5 + eps) - 0.5) < 1.01 * eps
    d1 = (orc.shape(2, 0.5 - eps) - orc.shape(2, 0.5 - 2 * eps)) / eps
    d2 = (orc.shape(2, 0.5 + 2 * eps) - orc.shape(2, 0.5 + eps)) / eps
    assert abs(d1 - d2) < 1e-5


E_POS = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]
B_POS = [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]


def _field_from(fn, n, stagger):
    z, y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float),
                          np.arange(n, dtype=float), indexing="ij")
    out = np.zeros((3, n, n, n))
    for c in range(3):
        sx, sy, sz = stagger[c]
        out[c] = fn(c, x + sx, y + sy, z + sz)
    return out


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_uniform_field(orc, order):
    n = 8
    g = orc.grid(n, n, n)
    E = np.zeros((3, n, n, n))
    B = np.zeros((3, n, n, n))
    for c, v in enumerate([1.7, -0.3, 0.25]):
        E[c] = v
        B[c] = 2 * v - 1
    rng = np.random.default_rng(2)
    for x in rng.uniform(0, n, (50, 3)):
        Ep, Bp = orc.gather(g, order, E, B, x)
        assert np.allclose(Ep, [1.7, -0.3, 0.25], rtol=0, atol=1e-14)
        assert np.allclose(Bp, [2.4, -1.6, -0.5], rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_gather_linear_field_at_staggered_positions(orc, order):
    """A wrong staggering offset (1/2 cell) or a swapped axis moves the result
    by slope/2 or by (slope_a - slope_b) * coordinate and fails here."""
    n = 16
    g = orc.grid(n, n, n)
    coef = np.array([[0.3, 1.1, -0.7, 0.4], [-0.2, 0.5, 0.9, -1.3], [1.0, -0.6, 0.2, 0.8]])
    coefb = coef[::-1] * 0.5 + 0.1

    def lin(cf):
        return lambda c, x, y, z: cf[c, 0] + cf[c, 1] * x + cf[c, 2] * y + cf[c, 3] * z

    E = _field_from(lin(coef), n, E_POS)
    B = _field_from(lin(coefb), n, B_POS)
    rng = np.random.default_rng(3)
    for x in rng.uniform(4, 12, (60, 3)):  # away from the periodic seam
        Ep, Bp = orc.gather(g, order, E, B, x)
        want_e = coef[:, 0] + coef[:, 1:] @ x
        want_b = coefb[:, 0] + coefb[:, 1:] @ x
        assert np.allclose(Ep, want_e, rtol=0, atol=1e-12)
        assert np.allclose(Bp, want_b, rtol=0, atol=1e-12)


def test_gather_wraps_periodically(orc):
    n = 8
    g = orc.grid(n, n, n)
    rng = np.random.default_rng(4)
    E = rng.normal(size=(3, n, n, n))
    B = rng.normal(size=(3, n, n, n))
    for order in (1, 2):
        x = np.array([0.1, 7.95, 3.3])
        a = orc.gather(g, order, E, B, x)
        b = orc.gather(g, order, E, B, x + np.array([n, -n, 2 * n]))
        assert np.allclose(a[0], b[0], atol=1e-13) and np.allclose(a[1], b[1], atol=1e-13)
