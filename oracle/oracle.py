"""FP64 CPU oracle of one explicit relativistic PIC step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product library never does: it
shares no code with the oracle, and the oracle shares none with it.

The arithmetic lives in ``pic_oracle.c`` (plain loops, FP64, one function per
algorithm the paper names in Sec. 4: Yee field solver, product-of-1D-weights
field gather, Boris pusher, Esirkepov current deposition, CIC / TSC shapes).
This file builds that C file with gcc, loads it with ctypes and strings the
functions together in the step order of the leapfrog cycle (Sec. 2.1 and
Sec. 4):

    gather E^n, B^n -> Boris -> move -> Esirkepov J^{n+1/2}
    -> B^{n+1/2} = B^n - dt/2 curl E^n -> E^{n+1} = E^n + dt (curl B - J)
    -> B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}

Arrays: fields are (3, nz, ny, nx) float64, x fastest; particle positions
are (n, 3) global coordinates in cell units in [0, N); momenta u = gamma v
are (n, 3); weights (n,).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpic_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_ARG = 1
ORC_ERR_DISPLACEMENT = 2


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("dz", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into a shared library (gcc, -O2, no fast-math and
    no FMA contraction, so that x86 and Arm hosts give identical results)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            gp = ctypes.POINTER(_Grid)
            L.orc_shape.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_shape.restype = ctypes.c_double
            L.orc_gather.argtypes = [gp, ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_int]
            L.orc_gather.restype = None
            L.orc_boris.argtypes = [ctypes.c_double] * 3 + [dp, dp, dp]
            L.orc_boris.restype = None
            L.orc_deposit_esirkepov.argtypes = [gp, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, dp, dp, dp]
            L.orc_deposit_esirkepov.restype = ctypes.c_int
            L.orc_push_deposit.argtypes = [gp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, dp, dp, dp, ctypes.c_int64,
                                           dp, dp, dp, ctypes.c_int, ctypes.c_int]
            L.orc_push_deposit.restype = ctypes.c_int
            L.orc_yee_b.argtypes = [gp, ctypes.c_double, dp, dp]
            L.orc_yee_b.restype = None
            L.orc_yee_e.argtypes = [gp, ctypes.c_double, dp, dp, dp]
            L.orc_yee_e.restype = None
            L.orc_yee_step.argtypes = [gp, ctypes.c_double, dp, dp, dp]
            L.orc_yee_step.restype = None
            L.orc_deposit_rho.argtypes = [gp, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                          dp, dp, dp]
            L.orc_deposit_rho.restype = None
            L.orc_div_e.argtypes = [gp, dp, dp]
            L.orc_div_e.restype = None
            L.orc_field_energy.argtypes = [gp, dp, dp]
            L.orc_field_energy.restype = ctypes.c_double
            L.orc_kinetic_energy.argtypes = [ctypes.c_double, ctypes.c_int64, dp, dp]
            L.orc_kinetic_energy.restype = ctypes.c_double
            L.orc_absorb_factor.argtypes = [ctypes.c_double] * 4
            L.orc_absorb_factor.restype = ctypes.c_double
            L.orc_absorb_y.argtypes = [gp, ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_absorb_y.restype = None
            L.orc_antenna_j0.argtypes = [ctypes.c_double] * 4 + [dp]
            L.orc_antenna_j0.restype = ctypes.c_int
            L.orc_antenna.argtypes = [gp, ctypes.c_int64] + [ctypes.c_double] * 9 + [dp]
            L.orc_antenna.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle wants C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def grid(nx, ny, nz, dx=(1.0, 1.0, 1.0)) -> _Grid:
    return _Grid(int(nx), int(ny), int(nz), float(dx[0]), float(dx[1]), float(dx[2]))


# ---------------------------------------------------------------- primitives

def shape(order: int, d: float) -> float:
    """1D assignment function S(d): order 1 = CIC, 2 = TSC (Hockney & Eastwood)."""
    return lib().orc_shape(int(order), float(d))


def gather(g: _Grid, order: int, E: np.ndarray, B: np.ndarray, x, ec: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """E and B interpolated to one position x (3,) in cell units; ec: the
    energy-conserving variant (one order lower along staggered axes)."""
    xp = _f64(x, (3,))
    Ep = np.zeros(3)
    Bp = np.zeros(3)
    lib().orc_gather(ctypes.byref(g), int(order), _ptr(E), _ptr(B), _ptr(xp), _ptr(Ep), _ptr(Bp),
                     int(bool(ec)))
    return Ep, Bp


def boris(q: float, m: float, dt: float, E, B, u) -> np.ndarray:
    """One relativistic Boris update of u = gamma v; returns the new u."""
    E = _f64(E, (3,))
    B = _f64(B, (3,))
    uu = _f64(u, (3,)).copy()
    lib().orc_boris(float(q), float(m), float(dt), _ptr(E), _ptr(B), _ptr(uu))
    return uu


def deposit_esirkepov(g: _Grid, order: int, qw: float, dt: float, x0, x1, J: np.ndarray) -> None:
    """Add one particle's Esirkepov current for the move x0 -> x1 into J."""
    a = _f64(x0, (3,))
    b = _f64(x1, (3,))
    rc = lib().orc_deposit_esirkepov(ctypes.byref(g), int(order), float(qw), float(dt),
                                     _ptr(a), _ptr(b), _ptr(J))
    if rc != ORC_OK:
        raise ValueError(f"oracle Esirkepov deposit rejected the move (code {rc})")


def deposit_rho(g: _Grid, order: int, q: float, x: np.ndarray, w: np.ndarray | None,
                rho: np.ndarray) -> None:
    lib().orc_deposit_rho(ctypes.byref(g), int(order), float(q), int(x.shape[0]), _ptr(x),
                          _ptr(w), _ptr(rho))


def div_e(g: _Grid, E: np.ndarray) -> np.ndarray:
    out = np.zeros((g.nz, g.ny, g.nx))
    lib().orc_div_e(ctypes.byref(g), _ptr(E), _ptr(out))
    return out


def absorb_factor(y: float, ny: float, A: float, sigma: float) -> float:
    """Damping factor of the y absorber at the (staggered) y position y."""
    return lib().orc_absorb_factor(float(y), float(ny), float(A), float(sigma))


def absorb_y(g: _Grid, A: float, sigma: float, E: np.ndarray, B: np.ndarray) -> None:
    lib().orc_absorb_y(ctypes.byref(g), float(A), float(sigma), _ptr(E), _ptr(B))


def antenna_j0(E0: float, omega: float, dt: float, dy: float = 1.0) -> float:
    """Sheet current density that radiates a wave of amplitude E0 on the grid."""
    out = np.zeros(1)
    if lib().orc_antenna_j0(float(E0), float(omega), float(dt), float(dy), _ptr(out)) != ORC_OK:
        raise ValueError("omega has no propagating wave on this grid")
    return float(out[0])


@dataclass
class Antenna:
    """Laser antenna on the node plane y = ja (Ex-polarised current sheet)."""
    ja: int
    E0: float
    omega: float
    w0: float = 0.0      # <= 0: plane sheet
    xc: float = 0.0
    zc: float = 0.0
    tau: float = 0.0     # <= 0: no temporal envelope
    t0: float = 0.0


def antenna(g: _Grid, a: Antenna, dt: float, t: float, J: np.ndarray) -> None:
    """Add the antenna's current at time t (the half step) into J."""
    rc = lib().orc_antenna(ctypes.byref(g), int(a.ja), float(a.E0), float(a.omega), float(a.w0),
                           float(a.xc), float(a.zc), float(a.tau), float(a.t0), float(dt), float(t),
                           _ptr(J))
    if rc != ORC_OK:
        raise ValueError("omega has no propagating wave on this grid")


def yee_b(g: _Grid, tau: float, E: np.ndarray, B: np.ndarray) -> None:
    lib().orc_yee_b(ctypes.byref(g), float(tau), _ptr(E), _ptr(B))


def yee_e(g: _Grid, dt: float, E: np.ndarray, B: np.ndarray, J: np.ndarray) -> None:
    lib().orc_yee_e(ctypes.byref(g), float(dt), _ptr(E), _ptr(B), _ptr(J))


# ---------------------------------------------------------------- full state

@dataclass
class Species:
    """One macro-particle species: charge q, mass m (in e and m_e), shape
    order (1 = CIC, 2 = TSC), mobile flag, its particle arrays, and the
    gather variant (ec: energy-conserving, one order lower along each
    staggered axis of a field component)."""
    q: float
    m: float
    order: int
    x: np.ndarray
    u: np.ndarray
    w: np.ndarray | None = None
    mobile: bool = True
    ec: bool = False

    def __post_init__(self):
        self.x = _f64(self.x).reshape(-1, 3).copy()
        self.u = _f64(self.u).reshape(-1, 3).copy()
        if self.w is not None:
            self.w = _f64(self.w).reshape(-1).copy()


@dataclass
class State:
    """One box: fields, species, and a fixed uniform background charge
    density rho_bg (it adds to rho and carries no current).  Periodic unless
    the open-y options are set:
      absorber = (A, sigma): damping layers of A cells at both y faces;
      open_y: particles that leave through a y face are removed;
      antenna: a laser antenna (Antenna) driven at the half steps;
    t is the time of E (advanced by dt per step)."""
    nx: int
    ny: int
    nz: int
    dt: float
    dx: tuple = (1.0, 1.0, 1.0)
    E: np.ndarray | None = None
    B: np.ndarray | None = None
    J: np.ndarray | None = None
    species: list = field(default_factory=list)
    rho_bg: float = 0.0
    absorber: tuple | None = None
    open_y: bool = False
    antenna: Antenna | None = None
    t: float = 0.0

    def __post_init__(self):
        shp = (3, self.nz, self.ny, self.nx)
        self.E = np.zeros(shp) if self.E is None else _f64(self.E, shp).copy()
        self.B = np.zeros(shp) if self.B is None else _f64(self.B, shp).copy()
        self.J = np.zeros(shp) if self.J is None else _f64(self.J, shp).copy()
        self.g = grid(self.nx, self.ny, self.nz, self.dx)

    def step(self, nsteps: int = 1) -> None:
        """Advance nsteps full PIC cycles in the order of the module docstring;
        with the open-y options: particles that left through a y face are
        removed after their deposit, the antenna current joins J before the
        field update, and the absorber damps E and B after it."""
        L = lib()
        for _ in range(nsteps):
            self.J[...] = 0.0
            for sp in self.species:
                if not sp.mobile:
                    continue
                rc = L.orc_push_deposit(ctypes.byref(self.g), float(self.dt), int(sp.order),
                                        float(sp.q), float(sp.m), _ptr(self.E), _ptr(self.B),
                                        _ptr(self.J), int(sp.x.shape[0]), _ptr(sp.x), _ptr(sp.u),
                                        _ptr(sp.w), int(bool(self.open_y)), int(bool(sp.ec)))
                if rc != ORC_OK:
                    raise ValueError(f"oracle push rejected a particle move (code {rc})")
                if self.open_y:
                    keep = (sp.x[:, 1] >= 0.0) & (sp.x[:, 1] < float(self.ny))
                    if not np.all(keep):
                        sp.x = np.ascontiguousarray(sp.x[keep])
                        sp.u = np.ascontiguousarray(sp.u[keep])
                        if sp.w is not None:
                            sp.w = np.ascontiguousarray(sp.w[keep])
                        if getattr(sp, "ids", None) is not None:
                            sp.ids = sp.ids[keep]
            if self.antenna is not None:
                antenna(self.g, self.antenna, self.dt, self.t + 0.5 * self.dt, self.J)
            L.orc_yee_step(ctypes.byref(self.g), float(self.dt), _ptr(self.E), _ptr(self.B),
                           _ptr(self.J))
            if self.absorber is not None:
                absorb_y(self.g, self.absorber[0], self.absorber[1], self.E, self.B)
            self.t += self.dt

    def shift_window(self, cells: int) -> None:
        """Moving window: the box moves `cells` cells towards +y.  Field values
        move down by `cells` planes and the planes that enter at the top are
        zero; particle y coordinates drop by `cells` and the particles that
        leave through the bottom are removed.  Fresh plasma for the top is
        the caller's to load."""
        m = int(cells)
        if not 0 < m < self.ny:
            raise ValueError("shift must be in (0, ny)")
        for F in (self.E, self.B, self.J):
            F[:, :, :self.ny - m, :] = F[:, :, m:, :].copy()
            F[:, :, self.ny - m:, :] = 0.0
        for sp in self.species:
            sp.x[:, 1] -= float(m)
            keep = sp.x[:, 1] >= 0.0
            sp.x = np.ascontiguousarray(sp.x[keep])
            sp.u = np.ascontiguousarray(sp.u[keep])
            if sp.w is not None:
                sp.w = np.ascontiguousarray(sp.w[keep])
            if getattr(sp, "ids", None) is not None:
                sp.ids = sp.ids[keep]

    def rho(self) -> np.ndarray:
        """Charge density at the nodes, background included."""
        r = np.full((self.nz, self.ny, self.nx), float(self.rho_bg))
        for sp in self.species:
            deposit_rho(self.g, sp.order, sp.q, sp.x, sp.w, r)
        return r

    def diagnostics(self) -> np.ndarray:
        """[field energy, kinetic energy, total charge, max |div E - rho|]."""
        L = lib()
        wf = L.orc_field_energy(ctypes.byref(self.g), _ptr(self.E), _ptr(self.B))
        wk = 0.0
        qtot = float(self.rho_bg) * self.nx * self.ny * self.nz * self.dx[0] * self.dx[1] * self.dx[2]
        for sp in self.species:
            wk += L.orc_kinetic_energy(float(sp.m), int(sp.u.shape[0]), _ptr(sp.u), _ptr(sp.w))
            wsum = float(sp.x.shape[0]) if sp.w is None else float(np.sum(sp.w))
            qtot += sp.q * wsum
        gauss = float(np.max(np.abs(div_e(self.g, self.E) - self.rho())))
        return np.array([wf, wk, qtot, gauss])
