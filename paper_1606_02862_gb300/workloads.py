"""Seeded synthetic workloads for the explicit PIC step.

This module only draws and lays out initial conditions: particle positions,
momenta and weights, uniform fields, a Gaussian laser pulse.  It holds none
of the method's arithmetic (no shape function, gather, push, deposit or field
update), so both the CUDA path and the FP64 oracle may take their inputs from
it.  Every array is FP64 and comes from ``numpy.random.default_rng(seed)``
(PCG64).

Normalised units: c = 1, eps0 = 1, e = m_e = 1, dx = dy = dz = 1, so a
number density n gives the plasma frequency omega_p = sqrt(n q^2 / m) and the
critical density of a laser of wavelength lambda cells is
n_c = (2 pi / lambda)^2.  A macro-particle weight is w = n * V_cell / ppc.

Workloads (sizes as the benchmark table names them):
  small_cic_32      32^3 periodic, electrons 2 ppc, u_th = 0.01, B_z = 0.1, CIC
  thermal_tsc_256   256^3 periodic, electrons 8 ppc + neutralising background,
                    u_th = 0.05, TSC (and its 64^3 sub-run)
  laser_ramp        128 x 1024 x 128, electrons + protons 4 ppc each in a
                    linear density ramp, Gaussian laser pulse along y
  batched_uneven    64 periodic boxes, edges from {16, 24, ..., 96}, ppc from
                    1..16, u_th from [0.01, 0.1]
  foil_overdense    256 x 2048 x 256, a 20-cell foil of electrons + C6+ at
                    30 n_c, 16 ppc each, Gaussian laser a0 = 10
  khi_128           128^3, electrons + ions 16 ppc each, counter-streaming
                    shear slabs at +-0.2 c, TSC (the paper's evaluation size)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 160602862  # arXiv 1606.02862
COURANT_3D = 1.0 / math.sqrt(3.0)  # for dx = dy = dz = 1
DT_HALF_COURANT = 0.5 * COURANT_3D
PROTON_MASS = 1836.15267
C6_MASS = 12.0 * 1822.888486 - 6.0  # carbon-12 nucleus in electron masses


@dataclass
class SpeciesDef:
    name: str
    q: float
    m: float
    shape: int  # 1 = CIC, 2 = TSC
    mobile: bool = True
    ec: bool = False  # energy-conserving gather


@dataclass
class BoxInit:
    nx: int
    ny: int
    nz: int
    # per species: (x (n,3), u (n,3), w (n,)) float64
    particles: list = field(default_factory=list)
    E: np.ndarray | None = None  # (3, nz, ny, nx) or None = zero
    B: np.ndarray | None = None
    rho_bg: float = 0.0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nparticles(self) -> int:
        return int(sum(p[0].shape[0] for p in self.particles))


@dataclass
class Workload:
    name: str
    dt: float
    species: list
    boxes: list
    dx: tuple = (1.0, 1.0, 1.0)
    steps: int = 1
    note: str = ""
    extra: dict = field(default_factory=dict)  # open-y options of the first box, window recipe

    @property
    def nparticles(self) -> int:
        return sum(b.nparticles for b in self.boxes)

    @property
    def ncells(self) -> int:
        return sum(b.ncells for b in self.boxes)


# ----------------------------------------------------------------- loaders

def uniform_in_cells(rng, nx, ny, nz, ppc, y_lo=0, y_hi=None):
    """ppc positions drawn uniformly inside every cell of the y-slab
    [y_lo, y_hi); returns (n, 3) float64 in cell units."""
    y_hi = ny if y_hi is None else y_hi
    cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(y_lo, y_hi), np.arange(nx), indexing="ij")
    base = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    base = np.repeat(base, ppc, axis=0)
    x = base + rng.random(base.shape)
    # rng.random is in [0, 1); keep the sum strictly inside the box
    np.minimum(x, np.array([nx, ny, nz], dtype=np.float64) * (1.0 - 2.0 ** -52), out=x)
    return x


def maxwellian(rng, n, u_th, drift=(0.0, 0.0, 0.0)):
    """Each momentum component drawn independently from N(drift, u_th^2)."""
    return rng.normal(0.0, u_th, size=(n, 3)) + np.asarray(drift, dtype=np.float64)


def uniform_field(nx, ny, nz, comp, value):
    f = np.zeros((3, nz, ny, nx))
    f[comp] = value
    return f


def gaussian_pulse_y(nx, ny, nz, a0, lam, waist, duration, y_c, x_c=None, z_c=None):
    """Linearly polarised (E along x) Gaussian pulse travelling along +y:
    Ex = a0 w_L exp(-r^2/waist^2) exp(-(y-y_c)^2/duration^2) cos(k (y-y_c)),
    Bz = -Ex, each sampled at its own staggered Yee position.  waist and
    duration are 1/e field radii in cells; w_L = k = 2 pi / lam."""
    k = 2.0 * math.pi / lam
    x_c = nx / 2.0 if x_c is None else x_c
    z_c = nz / 2.0 if z_c is None else z_c

    def profile(xs, ys, zs):
        r2 = (xs - x_c) ** 2 + (zs - z_c) ** 2
        return a0 * k * np.exp(-r2 / waist ** 2) * np.exp(-((ys - y_c) ** 2) / duration ** 2) * \
            np.cos(k * (ys - y_c))

    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    E = np.zeros((3, nz, ny, nx))
    B = np.zeros((3, nz, ny, nx))
    E[0] = profile(x + 0.5, y, z)          # Ex at (i+1/2, j, k)
    B[2] = -profile(x + 0.5, y + 0.5, z)   # Bz at (i+1/2, j+1/2, k)
    return E, B


# ----------------------------------------------------------------- configs

def small_cic_32(n=32, ppc=2, seed_offset=0) -> Workload:
    """32^3 periodic, one electron species 2 ppc, Maxwellian u_th = 0.01,
    uniform B_z = 0.1, zero E, CIC; electron density 0.01 with a fixed
    neutralising background so the zero initial E satisfies Gauss's law."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    dens = 0.01
    x = uniform_in_cells(rng, n, n, n, ppc)
    u = maxwellian(rng, x.shape[0], 0.01)
    w = np.full(x.shape[0], dens / ppc)
    box = BoxInit(n, n, n, particles=[(x, u, w)], B=uniform_field(n, n, n, 2, 0.1), rho_bg=dens)
    return Workload("small_cic_32", DT_HALF_COURANT, [SpeciesDef("e", -1.0, 1.0, 1)], [box],
                    steps=100)


def thermal_tsc(n=256, ppc=8, u_th=0.05, seed_offset=1, ny=None, nz=None) -> Workload:
    """n^3 periodic, electrons ppc per cell, Maxwellian u_th, TSC, density
    0.01 plus a fixed neutralising background.  n = 64 is the sub-run the
    FP64 oracle can follow."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    dens = 0.01
    x = uniform_in_cells(rng, n, ny, nz, ppc)
    u = maxwellian(rng, x.shape[0], u_th)
    w = np.full(x.shape[0], dens / ppc)
    box = BoxInit(n, ny, nz, particles=[(x, u, w)], rho_bg=dens)
    return Workload(f"thermal_tsc_{n}", DT_HALF_COURANT, [SpeciesDef("e", -1.0, 1.0, 2)], [box],
                    steps=200)


def fill_thermal(x, u, w, nx, ny, nz, ppc, u_th, dens=0.01, seed_offset=1, slab=8, z_lo=0, z_hi=None):
    """Write the thermal_tsc recipe (ppc uniform positions per cell,
    Maxwellian u_th, weight dens / ppc) into preallocated (n,3), (n,3), (n,)
    float64 arrays, one z-slab at a time with its own PCG64 stream, so that a
    256^3 state (134M particles) never needs more than the output arrays.
    z_lo, z_hi (multiples of `slab`): only the planes [z_lo, z_hi), the same
    particles as that part of the whole box.  Returns the particle count
    written."""
    per_layer = nx * ny * ppc
    z_hi = nz if z_hi is None else z_hi
    if z_lo % slab or (z_hi % slab and z_hi != nz) or not 0 <= z_lo <= z_hi <= nz:
        raise ValueError("z range must be whole generator slabs")
    k = 0
    for z0 in range(z_lo, z_hi, slab):
        z1 = min(z_hi, z0 + slab)
        rng = np.random.default_rng([BASE_SEED + seed_offset, z0])
        cz, cy, cx = np.meshgrid(np.arange(z0, z1), np.arange(ny), np.arange(nx), indexing="ij")
        m = (z1 - z0) * per_layer
        xs = x[k:k + m]
        xs[:, 0] = np.repeat(cx.ravel(), ppc)
        xs[:, 1] = np.repeat(cy.ravel(), ppc)
        xs[:, 2] = np.repeat(cz.ravel(), ppc)
        xs += rng.random((m, 3))
        u[k:k + m] = rng.normal(0.0, u_th, size=(m, 3))
        w[k:k + m] = dens / ppc
        k += m
    np.minimum(x[:k], np.array([nx, ny, nz], dtype=np.float64) * (1.0 - 2.0 ** -52), out=x[:k])
    return k


def khi(n=128, ppc=16, drift=0.2, u_th=0.005, dens=0.01, seed_offset=5) -> Workload:
    """A Kelvin-Helmholtz-like shear flow in the configuration of the paper's
    evaluation (Sec. 4: 128^3 cells, electrons and ions at 16 particles per
    cell each, TSC): both species drift at +drift c along x for y in
    [n/4, 3n/4) and at -drift c elsewhere (two periodic shear layers), with
    thermal spread u_th (ions: u_th / sqrt(m_p)); quasi-neutral, zero
    initial fields.  The paper cites its setup without parameters; these are
    this workload's own choices."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    parts = []
    for m in (1.0, PROTON_MASS):
        x = uniform_in_cells(rng, n, n, n, ppc)
        sign = np.where((x[:, 1] >= n / 4) & (x[:, 1] < 3 * n / 4), 1.0, -1.0)
        gamma_drift = 1.0 / math.sqrt(1.0 - drift * drift)
        u = maxwellian(rng, x.shape[0], u_th / math.sqrt(m))
        u[:, 0] += sign * drift * gamma_drift
        parts.append((x, u, np.full(x.shape[0], dens / ppc)))
    box = BoxInit(n, n, n, particles=parts)
    sp = [SpeciesDef("e", -1.0, 1.0, 2), SpeciesDef("p", 1.0, PROTON_MASS, 2)]
    return Workload(f"khi_{n}", DT_HALF_COURANT, sp, [box], steps=1000)


def laser_ramp(nx=128, ny=1024, nz=128, ppc=4, seed_offset=2, lam=32.0, a0=3.0, waist=16.0,
               duration=40.0, y_c=80.0, ramp=(160, 360), n_frac=0.01) -> Workload:
    """Electron + proton species, ppc each, density rising linearly from 0 at
    y = ramp[0] to n_frac n_c at y = ramp[1], then flat; Gaussian pulse along
    y.  Weights follow the local density at each particle's cell row."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    nc = (2.0 * math.pi / lam) ** 2
    n0 = n_frac * nc
    y_lo = min(ramp[0], ny)
    xs = []
    for _sp in range(2):
        x = uniform_in_cells(rng, nx, ny, nz, ppc, y_lo=y_lo, y_hi=ny)
        row = np.floor(x[:, 1]) + 0.5
        dens = n0 * np.clip((row - ramp[0]) / (ramp[1] - ramp[0]), 0.0, 1.0)
        xs.append((x, dens / ppc))
    ue = maxwellian(rng, xs[0][0].shape[0], 0.001)
    ui = maxwellian(rng, xs[1][0].shape[0], 0.001 / math.sqrt(PROTON_MASS))
    E, B = gaussian_pulse_y(nx, ny, nz, a0, lam, waist, duration, y_c)
    box = BoxInit(nx, ny, nz, particles=[(xs[0][0], ue, xs[0][1]), (xs[1][0], ui, xs[1][1])],
                  E=E, B=B)
    sp = [SpeciesDef("e", -1.0, 1.0, 2), SpeciesDef("p", 1.0, PROTON_MASS, 2)]
    return Workload("laser_ramp", DT_HALF_COURANT, sp, [box], steps=1000)


def window_slab(rng, nx, nz, y0, y1, ppc, density, u_th=0.001, species_masses=(1.0, PROTON_MASS),
                y_shift=0.0):
    """Fresh plasma for rows y0 <= y < y1 of a moving window: for each species
    (masses in m_e), ppc particles per cell, weights following density(y) at
    each cell row's centre (y in the lab frame, y_shift + box y), thermal
    momenta u_th / sqrt(m).  Returns [(x, u, w), ...] in box coordinates."""
    out = []
    for m in species_masses:
        x = uniform_in_cells(rng, nx, y1 - y0, nz, ppc) + np.array([0.0, float(y0), 0.0])
        row = np.floor(x[:, 1]) + 0.5 + y_shift
        w = density(row) / ppc
        keep = w > 0.0
        x, w = x[keep], w[keep]
        out.append((x, maxwellian(rng, x.shape[0], u_th / math.sqrt(m)), w))
    return out


def laser_window(nx=128, ny=1024, nz=128, ppc=4, seed_offset=5, lam=32.0, a0=3.0, waist=16.0,
                 duration=40.0, ramp=(160, 360), n_frac=0.01, absorber=32, sigma=1.0,
                 antenna_y=40) -> Workload:
    """The laser-ramp setup with open y boundaries: damping layers of
    `absorber` cells at both y faces, particles leaving through them removed,
    the pulse injected by an antenna on the plane y = antenna_y (amplitude
    a0 omega, 1/e radius waist, 1/e half duration `duration`, peak at 2
    durations), and a moving window that the caller advances by whole
    supercell rows, loading fresh plasma (window_slab) at the top.  e- + p+
    at ppc each in a density rising linearly from 0 at y = ramp[0] to n_frac
    n_c at ramp[1], flat beyond."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    omega = 2.0 * math.pi / lam
    n0 = n_frac * omega ** 2

    def density(y):
        return n0 * np.clip((np.asarray(y) - ramp[0]) / (ramp[1] - ramp[0]), 0.0, 1.0)

    parts = window_slab(rng, nx, nz, 0, ny, ppc, density)
    box = BoxInit(nx, ny, nz, particles=parts)
    sp = [SpeciesDef("e", -1.0, 1.0, 2), SpeciesDef("p", 1.0, PROTON_MASS, 2)]
    wl = Workload("laser_window", DT_HALF_COURANT, sp, [box], steps=1000)
    wl.extra = {
        "boundary": dict(open_y=True, absorber_cells=absorber, absorber_sigma=sigma),
        "antenna": dict(plane_y=antenna_y, E0=a0 * omega, omega=omega, w0=waist, xc=nx / 2.0,
                        zc=nz / 2.0, tau=duration, t0=2.0 * duration),
        "density": density,
        "ppc": ppc,
        "seed": BASE_SEED + seed_offset,
    }
    return wl


def iter_batched_uneven(nboxes=64, seed_offset=3, sizes=tuple(range(16, 97, 8)), max_ppc=16,
                        dens=0.01):
    """Yield the boxes of batched_uneven one at a time: (n, ppc, u_th, x, u, w),
    from one PCG64 stream, so a caller never holds more than one box."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    for _ in range(nboxes):
        n = int(rng.choice(sizes))
        ppc = int(rng.integers(1, max_ppc + 1))
        u_th = float(rng.uniform(0.01, 0.1))
        x = uniform_in_cells(rng, n, n, n, ppc)
        u = maxwellian(rng, x.shape[0], u_th)
        w = np.full(x.shape[0], dens / ppc)
        yield n, ppc, u_th, x, u, w


def batched_uneven(nboxes=64, seed_offset=3, sizes=tuple(range(16, 97, 8)), max_ppc=16) -> Workload:
    """nboxes independent periodic cubic boxes; edge drawn uniformly from
    sizes, ppc from 1..max_ppc, u_th from U[0.01, 0.1]; electrons, TSC,
    density 0.01 plus background."""
    dens = 0.01
    boxes = [BoxInit(n, n, n, particles=[(x, u, w)], rho_bg=dens)
             for n, _ppc, _uth, x, u, w in iter_batched_uneven(nboxes, seed_offset, sizes, max_ppc, dens)]
    return Workload("batched_uneven", DT_HALF_COURANT, [SpeciesDef("e", -1.0, 1.0, 2)], boxes,
                    steps=500)


def foil_overdense(nx=256, ny=2048, nz=256, ppc=16, seed_offset=4, lam=32.0, a0=10.0,
                   waist=16.0, duration=40.0, foil=(512, 532), n_e_over_nc=30.0,
                   pulse_gap=100.0) -> Workload:
    """A foil y in [foil[0], foil[1]) of electrons at n_e_over_nc n_c and C6+
    at a sixth of that (neutral), ppc each, in vacuum; Gaussian pulse centred
    pulse_gap cells before the foil."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    nc = (2.0 * math.pi / lam) ** 2
    ne = n_e_over_nc * nc
    xe = uniform_in_cells(rng, nx, ny, nz, ppc, y_lo=foil[0], y_hi=foil[1])
    xi = uniform_in_cells(rng, nx, ny, nz, ppc, y_lo=foil[0], y_hi=foil[1])
    ue = maxwellian(rng, xe.shape[0], 0.001)
    ui = maxwellian(rng, xi.shape[0], 0.001 / math.sqrt(C6_MASS))
    E, B = gaussian_pulse_y(nx, ny, nz, a0, lam, waist, duration, foil[0] - pulse_gap)
    box = BoxInit(nx, ny, nz, particles=[(xe, ue, np.full(xe.shape[0], ne / ppc)),
                                         (xi, ui, np.full(xi.shape[0], ne / 6.0 / ppc))], E=E, B=B)
    sp = [SpeciesDef("e", -1.0, 1.0, 2), SpeciesDef("C6+", 6.0, C6_MASS, 2)]
    return Workload("foil_overdense", DT_HALF_COURANT, sp, [box], steps=2000)
