"""Pins of the oracle's Esirkepov current deposition (Esirkepov 2001, the
"Esirkepov current solver" named in Sec. 4).

Independent facts the deposit must satisfy:
  * discrete continuity at every node, (rho^{n+1} - rho^n) / dt + div J = 0,
    with rho from the particle shape at the nodes (charge conservation, the
    defining property of the scheme);
  * the total current equals the particle current:
    sum over cells of J_d V = q w (x1_d - x0_d) dx_d / dt;
  * time reversal: the move x1 -> x0 deposits exactly minus x0 -> x1;
  * for CIC and a move that stays inside one cell, J_d through the one face
    it crosses is the charge flux of the linear cloud: q w v_d / V times the
    path average of the transverse CIC weights (Villasenor-Buneman), here
    integrated with Simpson's rule, exact for the quadratic integrand;
  * Esirkepov's decomposition is the average over the six orders of moving
    one axis at a time; that average, built here from 1D continuity alone,
    must equal the oracle's J for either shape.
"""
import itertools
import math

import numpy as np
import pytest

DT = 0.5 / math.sqrt(3.0)


def _deposit(orc, g, order, qw, x0, x1, dt=DT):
    J = np.zeros((3, g.nz, g.ny, g.nx))
    orc.deposit_esirkepov(g, order, qw, dt, x0, x1, J)
    return J


def _rho(orc, g, order, q, x, w):
    r = np.zeros((g.nz, g.ny, g.nx))
    orc.deposit_rho(g, order, q, np.ascontiguousarray(np.atleast_2d(x), dtype=float),
                    np.ascontiguousarray(np.atleast_1d(w), dtype=float), r)
    return r


def _moves(rng, n, count, maxd):
    x0 = rng.uniform(0, n, (count, 3))
    d = rng.uniform(-maxd, maxd, (count, 3))
    return x0, d


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.7, 1.3, 1.0)])
def test_continuity_random_moves(orc, order, h):
    n = 8
    g = orc.grid(n, n, n, h)
    rng = np.random.default_rng(10 + order)
    x0, d = _moves(rng, n, 40, 0.95)
    q, w = -1.0, 0.37
    for a, dd in zip(x0, d):
        b = a + dd
        J = _deposit(orc, g, order, q * w, a, b)
        r0 = _rho(orc, g, order, q, a % n, w)
        r1 = _rho(orc, g, order, q, b % n, w)
        res = (r1 - r0) / DT + orc.div_e(g, J)
        scale = abs(q * w) / (h[0] * h[1] * h[2] * DT)
        assert np.max(np.abs(res)) < 1e-13 * scale


@pytest.mark.parametrize("order", [1, 2, 3])
def test_total_current_is_particle_current(orc, order):
    n = 8
    h = (1.0, 0.9, 1.2)
    g = orc.grid(n, n, n, h)
    V = h[0] * h[1] * h[2]
    rng = np.random.default_rng(20 + order)
    x0, d = _moves(rng, n, 30, 0.9)
    qw = 0.81
    for a, dd in zip(x0, d):
        J = _deposit(orc, g, order, qw, a, a + dd)
        for c in range(3):
            assert abs(J[c].sum() * V - qw * dd[c] * h[c] / DT) < 1e-13


@pytest.mark.parametrize("order", [1, 2, 3])
def test_time_reversal(orc, order):
    n = 8
    g = orc.grid(n, n, n)
    rng = np.random.default_rng(30 + order)
    x0, d = _moves(rng, n, 20, 0.9)
    for a, dd in zip(x0, d):
        Jf = _deposit(orc, g, order, 1.0, a, a + dd)
        Jb = _deposit(orc, g, order, 1.0, a + dd, a)
        assert np.max(np.abs(Jf + Jb)) < 1e-13


def test_every_face_edge_and_corner_crossing(orc):
    """A particle near a cell corner moved in each of the 26 directions (and
    not at all): continuity and total current for both shapes."""
    n = 6
    g = orc.grid(n, n, n)
    for order in (1, 2, 3):
        for start in ([2.95, 3.02, 2.97], [3.5, 3.5, 3.5], [2.51, 2.49, 3.0]):
            for dirn in itertools.product((-1, 0, 1), repeat=3):
                a = np.array(start)
                b = a + 0.4 * np.array(dirn, dtype=float)
                J = _deposit(orc, g, order, 1.0, a, b)
                res = (_rho(orc, g, order, 1.0, b % n, 1.0) - _rho(orc, g, order, 1.0, a % n, 1.0)) / DT \
                    + orc.div_e(g, J)
                assert np.max(np.abs(res)) < 1e-12
                for c in range(3):
                    assert abs(J[c].sum() - 0.4 * dirn[c] / DT) < 1e-12
                if dirn == (0, 0, 0):
                    assert np.max(np.abs(J)) == 0.0


def test_cic_within_cell_equals_charge_flux(orc):
    """Villasenor-Buneman: for CIC and a move inside one cell, Jx is nonzero
    only at the x-face inside that cell, and equals q w vx / V times the
    average over the path of the transverse weights."""
    n = 6
    g = orc.grid(n, n, n)
    rng = np.random.default_rng(40)
    for _ in range(20):
        cell = rng.integers(1, n - 2, 3)
        a = cell + rng.uniform(0.05, 0.45, 3)
        b = cell + rng.uniform(0.55, 0.95, 3)
        if rng.random() < 0.5:
            a, b = b, a
        J = _deposit(orc, g, 1, 1.0, a, b)
        i, j, k = cell
        # transverse CIC weights along the path, Simpson's rule in t
        ts = np.array([0.0, 0.5, 1.0])
        sw = np.array([1.0, 4.0, 1.0]) / 6.0
        path = a[None, :] + ts[:, None] * (b - a)[None, :]
        fy = path[:, 1] - j
        fz = path[:, 2] - k
        wy = [1 - fy, fy]
        wz = [1 - fz, fz]
        vx = (b[0] - a[0]) / DT
        want = np.zeros((3, n, n, n))
        for dj in range(2):
            for dk in range(2):
                want[0, k + dk, j + dj, i] = vx * np.sum(sw * wy[dj] * wz[dk])
        assert np.max(np.abs(J[0] - want[0])) < 1e-13


@pytest.mark.parametrize("order", [1, 2, 3])
def test_equals_average_over_axis_orderings(orc, order):
    """Build J from 1D continuity alone: move one axis at a time; a move along
    d carries J_d(m_d + 1/2) = -(dx_d/dt) q w / V * prefix sum over m' <= m_d
    of (S_new(m') - S_old(m')) along d, times the current shapes on the two
    other axes.  Average over the 6 axis orders."""
    n = 10
    h = (1.0, 1.0, 1.0)
    g = orc.grid(n, n, n, h)
    rng = np.random.default_rng(50 + order)

    def shape_vec(xd, lo, count):
        return np.array([orc.shape(order, xd - (lo + m)) for m in range(count)])

    for _ in range(10):
        a = rng.uniform(3, 7, 3)
        b = a + rng.uniform(-0.9, 0.9, 3)
        lo = np.floor(a).astype(int) - 2
        cnt = 6
        S0 = [shape_vec(a[d], lo[d], cnt) for d in range(3)]
        S1 = [shape_vec(b[d], lo[d], cnt) for d in range(3)]
        Jw = np.zeros((3, cnt, cnt, cnt))  # window-local [c][k][j][i]
        for perm in itertools.permutations(range(3)):
            cur = [S0[0].copy(), S0[1].copy(), S0[2].copy()]
            for d in perm:
                flux = -np.cumsum(S1[d] - cur[d]) * h[d] / DT  # q w / V = 1
                e, f = [x for x in range(3) if x != d]
                # outer product in window axes order (x=i, y=j, z=k)
                vecs = [None, None, None]
                vecs[d] = flux
                vecs[e] = cur[e]
                vecs[f] = cur[f]
                Jw[d] += np.einsum("k,j,i->kji", vecs[2], vecs[1], vecs[0])
                cur[d] = S1[d].copy()
        Jw /= 6.0
        J = _deposit(orc, g, order, 1.0, a, b)
        Jwin = J[:, lo[2]:lo[2] + cnt, lo[1]:lo[1] + cnt, lo[0]:lo[0] + cnt]
        assert np.max(np.abs(Jwin - Jw)) < 1e-13
        assert abs(np.abs(J).sum() - np.abs(Jwin).sum()) < 1e-13


def test_rejects_moves_of_a_cell_or_more(orc):
    g = orc.grid(8, 8, 8)
    with pytest.raises(ValueError):
        _deposit(orc, g, 2, 1.0, [3.0, 3.0, 3.0], [4.0, 3.0, 3.0])
