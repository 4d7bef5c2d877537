"""Pin of the oracle's Yee field solver (Yee 1966, named in Sec. 4) against
the closed-form dispersion relation of the staggered leapfrog scheme.

In a periodic vacuum box a single discrete Fourier mode k is an exact
eigenmode of the scheme: on the staggered grid every centred difference
along axis d acts on it as i K_d with K_d = 2 sin(k_d dx_d / 2) / dx_d, and
the leapfrog in time as i Omega with Omega = 2 sin(omega dt / 2) / dt.  The
mode evolves as cos(k.r - omega t) with

    sin^2(omega dt / 2) / dt^2 = sum_d sin^2(k_d dx_d / 2) / dx_d^2,

for E perpendicular to K and B = K x E / Omega (at half-integer time; the
integer-time B the step starts from is cos(omega dt / 2) times that).  A
wrong sign, a swapped difference (i-1 for i+1) or a wrong staggering breaks
the relation or the amplitude.
"""
import math

import numpy as np
import pytest

E_POS = [(0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]
B_POS = [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)]


def _phase_grid(n, kvec, stagger, h):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float),
                          np.arange(nx, dtype=float), indexing="ij")
    return [kvec[0] * (x + s[0]) * h[0] + kvec[1] * (y + s[1]) * h[1] + kvec[2] * (z + s[2]) * h[2]
            for s in stagger]


def _mode(n, modes, h, dt):
    kvec = np.array([2 * math.pi * modes[d] / (n[d] * h[d]) for d in range(3)])
    K = np.array([2 * math.sin(kvec[d] * h[d] / 2) / h[d] for d in range(3)])
    Omega = math.sqrt(K @ K)
    omega = 2.0 / dt * math.asin(Omega * dt / 2.0)
    a = np.array([0.3, -1.0, 0.7])
    Ehat = np.cross(K, a)
    Ehat /= np.linalg.norm(Ehat)
    Bhat = np.cross(K, Ehat) / Omega
    return kvec, K, Omega, omega, Ehat, Bhat


@pytest.mark.parametrize("n,modes,h", [((16, 12, 8), (1, 1, 1), (1.0, 1.0, 1.0)),
                                       ((16, 16, 4), (3, -2, 1), (1.0, 1.0, 1.0)),
                                       ((12, 10, 8), (2, 1, -1), (1.0, 0.8, 1.25))])
def test_yee_vacuum_dispersion(orc, n, modes, h):
    nx, ny, nz = n
    courant = 1.0 / math.sqrt(sum(1.0 / hh ** 2 for hh in h))
    dt = 0.5 * courant
    kvec, K, Omega, omega, Ehat, Bhat = _mode(n, modes, h, dt)
    pe = _phase_grid(n, kvec, E_POS, h)
    pb = _phase_grid(n, kvec, B_POS, h)
    E = np.stack([Ehat[c] * np.cos(pe[c]) for c in range(3)])
    B = np.stack([Bhat[c] * math.cos(omega * dt / 2) * np.cos(pb[c]) for c in range(3)])
    st = orc.State(nx, ny, nz, dt, dx=h, E=E, B=B)
    nsteps = 1000
    st.step(nsteps)
    # project onto cos / sin of the mode
    num_c = sum(np.sum(st.E[c] * Ehat[c] * np.cos(pe[c])) for c in range(3))
    num_s = sum(np.sum(st.E[c] * Ehat[c] * np.sin(pe[c])) for c in range(3))
    den = sum(np.sum((Ehat[c] * np.cos(pe[c])) ** 2) for c in range(3))
    phase = math.atan2(num_s, num_c)
    want = (omega * nsteps * dt + math.pi) % (2 * math.pi) - math.pi
    err = (phase - want + math.pi) % (2 * math.pi) - math.pi
    assert abs(err) < 1e-10, (phase, want)
    # the mode keeps its shape and amplitude
    expect = np.stack([Ehat[c] * np.cos(pe[c] - omega * nsteps * dt) for c in range(3)])
    assert np.max(np.abs(st.E - expect)) < 1e-10
    assert abs(math.hypot(num_c, num_s) / den - 1.0) < 1e-10
    # the numerical phase velocity is below c and matches omega / |k|
    assert omega / np.linalg.norm(kvec) < 1.0


def test_yee_preserves_div_b_and_div_e_without_current(orc):
    n = 8
    rng = np.random.default_rng(5)
    st = orc.State(n, n, n, 0.25, E=rng.normal(size=(3, n, n, n)), B=np.zeros((3, n, n, n)))
    # B = curl of a random A has zero discrete divergence; build it with one Yee B update
    A = rng.normal(size=(3, n, n, n))
    orc.yee_b(st.g, -1.0, A, st.B)  # B = +curl A on the B positions
    g = st.g

    def div_b(B):
        # divergence at cell centres (i+1/2, j+1/2, k+1/2) of the face-centred B
        return ((np.roll(B[0], -1, axis=2) - B[0]) + (np.roll(B[1], -1, axis=1) - B[1]) +
                (np.roll(B[2], -1, axis=0) - B[2]))

    assert np.max(np.abs(div_b(st.B))) < 1e-12
    dive0 = orc.div_e(g, st.E)
    st.step(20)
    assert np.max(np.abs(div_b(st.B))) < 1e-12
    assert np.max(np.abs(orc.div_e(g, st.E) - dive0)) < 1e-12
