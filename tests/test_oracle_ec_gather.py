"""Pins of the oracle's energy-conserving gather variant (one shape order
lower along each axis on which a field component is staggered):

  * closed forms for a quadratic field, from the second moments of the
    B-splines: sum_m S_n(x - m) m^2 = x^2 + (n + 1) / 12 for the smooth
    splines sampled symmetrically (TSC: + 1/4), x^2 + t (1 - t) for CIC
    (t the offset from the lower node), the nearest node's value for NGP.
    They tell which axes are reduced and by how much;
  * the energy identity that defines the variant: for a particle moving
    along one axis, the work of the grid current on the field,
    sum over cells of J.E V dt (Esirkepov's J), equals the line integral of
    the gathered field along the path, q w int E_gathered . dx -- exactly for
    this gather, and not for the momentum-conserving one.
"""
import numpy as np
import pytest

N = 32


def _grid(orc):
    return orc.grid(N, N, N)


def _field(fn):
    """(3, N, N, N) field with component c = fn(c, i, j, k) (array indices)."""
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return np.stack([fn(c, i, j, k) for c in range(3)]).astype(float)


def _frac(v):
    return v - np.floor(v)


@pytest.mark.parametrize("seed", range(4))
def test_quadratic_field_closed_forms_tsc(orc, seed):
    rng = np.random.default_rng(seed)
    g = _grid(orc)
    x = rng.uniform(10, 20, 3)
    # Ex at (i+1/2, j, k): Ex = x^2 along its staggered axis, Bx at (i, j+1/2, k+1/2): Bx = y^2
    E = _field(lambda c, i, j, k: (i + 0.5) ** 2 if c == 0 else 0.0 * i)
    B = _field(lambda c, i, j, k: (j + 0.5) ** 2 if c == 0 else 0.0 * i)
    Em, Bm = orc.gather(g, 2, E, B, x)
    Ee, Be = orc.gather(g, 2, E, B, x, ec=True)
    assert Em[0] == pytest.approx(x[0] ** 2 + 0.25, abs=1e-10)          # TSC along x
    assert Bm[0] == pytest.approx(x[1] ** 2 + 0.25, abs=1e-10)
    tx, ty = _frac(x[0] - 0.5), _frac(x[1] - 0.5)
    assert Ee[0] == pytest.approx(x[0] ** 2 + tx * (1 - tx), abs=1e-10)  # CIC along staggered x
    assert Be[0] == pytest.approx(x[1] ** 2 + ty * (1 - ty), abs=1e-10)  # CIC along staggered y
    # along an axis on which the component is not staggered, TSC in both variants
    E2 = _field(lambda c, i, j, k: j.astype(float) ** 2 if c == 0 else 0.0 * i)
    B2 = _field(lambda c, i, j, k: i.astype(float) ** 2 if c == 0 else 0.0 * i)
    Ee2, Be2 = orc.gather(g, 2, E2, B2, x, ec=True)
    assert Ee2[0] == pytest.approx(x[1] ** 2 + 0.25, abs=1e-10)
    assert Be2[0] == pytest.approx(x[0] ** 2 + 0.25, abs=1e-10)
    # Bz at (i+1/2, j+1/2, k) reduced along x and y, not z
    B3 = _field(lambda c, i, j, k: ((i + 0.5) ** 2 + (j + 0.5) ** 2 + k.astype(float) ** 2) if c == 2 else 0.0 * i)
    _, Be3 = orc.gather(g, 2, E2, B3, x, ec=True)
    assert Be3[2] == pytest.approx(x[0] ** 2 + tx * (1 - tx) + x[1] ** 2 + ty * (1 - ty) + x[2] ** 2 + 0.25,
                                   abs=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_cic_variant_is_nearest_grid_point_along_staggered_axes(orc, seed):
    rng = np.random.default_rng(10 + seed)
    g = _grid(orc)
    x = rng.uniform(10, 20, 3)
    E = _field(lambda c, i, j, k: (i + 0.5) ** 2 + 3.0 * j if c == 0 else 0.0 * i)
    B = np.zeros_like(E)
    Em, _ = orc.gather(g, 1, E, B, x)
    Ee, _ = orc.gather(g, 1, E, B, x, ec=True)
    t = _frac(x[0] - 0.5)
    assert Em[0] == pytest.approx(x[0] ** 2 + t * (1 - t) + 3.0 * x[1], abs=1e-10)
    # nearest half node of x is floor(x) + 1/2; CIC (linear-exact) along y
    assert Ee[0] == pytest.approx((np.floor(x[0]) + 0.5) ** 2 + 3.0 * x[1], abs=1e-10)


def test_uniform_field_is_exact_in_both_variants(orc):
    g = _grid(orc)
    E = np.empty((3, N, N, N))
    B = np.empty((3, N, N, N))
    for c in range(3):
        E[c] = 0.3 + c
        B[c] = -1.1 * (c + 1)
    for order in (1, 2):
        Ee, Be = orc.gather(g, order, E, B, [7.3, 11.5, 19.99], ec=True)
        assert np.allclose(Ee, [0.3, 1.3, 2.3], atol=1e-13) and np.allclose(Be, [-1.1, -2.2, -3.3], atol=1e-13)


def _line_integral(orc, g, order, E, B, x0, axis, D, ec):
    """int_0^1 E_axis(x0 + s D e_axis) D ds, split where the gathered
    component is not smooth (integer and half-integer positions along the
    axis) and integrated by 4-point Gauss-Legendre on each piece (exact for
    the piecewise polynomials of degree <= 7 that a gather of order <= 3 gives)."""
    a, b = x0[axis], x0[axis] + D
    lo, hi = min(a, b), max(a, b)
    cuts = [lo] + [k / 2.0 for k in range(int(np.floor(lo * 2)) + 1, int(np.ceil(hi * 2)))] + [hi]
    gx, gw = np.polynomial.legendre.leggauss(4)
    tot = 0.0
    for p, q in zip(cuts[:-1], cuts[1:]):
        for xi, wi in zip(gx, gw):
            pos = np.array(x0, dtype=float)
            pos[axis] = 0.5 * (p + q) + 0.5 * (q - p) * xi
            Ep, _ = orc.gather(g, order, E, B, pos, ec=ec)
            tot += 0.5 * (q - p) * wi * Ep[axis]
    return tot if D > 0 else -tot


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_energy_identity_for_motion_along_one_axis(orc, order, axis):
    """sum J.E over the cells (Esirkepov, q w = 1, dt = V = 1) equals the line
    integral of the energy-conserving gather along the path."""
    rng = np.random.default_rng(100 + 3 * order + axis)
    g = _grid(orc)
    E = rng.normal(size=(3, N, N, N))
    B = rng.normal(size=(3, N, N, N))
    for trial in range(6):
        x0 = rng.uniform(10, 20, 3)
        D = rng.uniform(-0.49, 0.49)
        x1 = x0.copy()
        x1[axis] += D
        J = np.zeros((3, N, N, N))
        orc.deposit_esirkepov(g, order, 1.0, 1.0, x0, x1, J)
        work = float(np.sum(J * E))
        ec = _line_integral(orc, g, order, E, B, x0, axis, D, ec=True)
        assert work == pytest.approx(ec, abs=1e-12 * max(1.0, abs(ec)))
        mc = _line_integral(orc, g, order, E, B, x0, axis, D, ec=False)
        if trial == 0:
            assert abs(work - mc) > 1e-6  # the momentum-conserving gather does not satisfy it
