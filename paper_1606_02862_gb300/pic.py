"""ctypes binding of libpic (include/pic.h): the same entry points, argument
marshalling only.  Every step of the PIC cycle runs in the library's CUDA
kernels; there is no Python or CPU fallback.  If the library is missing or
no GPU is present, the calls raise.

PyTorch supplies device memory (its caching allocator, through the
library's allocator callback) and the stream (the current torch stream),
when ``torch_memory=True``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpic.so")

PIC_OK = 0
STATUS_NAMES = {
    0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_CFL", 3: "PIC_ERR_OOM", 4: "PIC_ERR_CUDA",
    5: "PIC_ERR_FRAME_POOL", 6: "PIC_ERR_TIMEOUT", 7: "PIC_ERR_STATE", 8: "PIC_ERR_CAPACITY",
    9: "PIC_ERR_PARTICLE",
}
PRECISION_FP64_PLAIN = 0
PRECISION_MIXED = 1
FIELD_E, FIELD_B, FIELD_J, FIELD_RHO = 0, 1, 2, 3

# every symbol include/pic.h declares
EXPORTED = ("pic_create", "pic_set_background", "pic_set_boundary", "pic_set_antenna",
            "pic_shift_window", "pic_load_particles", "pic_write_fields",
            "pic_step", "pic_step_async", "pic_sync", "pic_read_fields", "pic_count_particles",
            "pic_read_particles", "pic_diagnostics", "pic_stage_timing", "pic_stage_times",
            "pic_info", "pic_set_subdomain", "pic_step_stage", "pic_halo_floats", "pic_halo_pack",
            "pic_halo_unpack", "pic_migrant_bytes", "pic_migrants_pack", "pic_migrants_accept",
            "pic_field_energy_noalloc", "pic_last_error", "pic_destroy")
STAGE_PUSH, STAGE_FRAMES, STAGE_B_FIRST, STAGE_E, STAGE_B_SECOND = range(5)
(INFO_GRAPH_ACTIVE, INFO_KERNELS_PER_STEP, INFO_POOL_FRAMES, INFO_FRAMES_USED, INFO_MOVE_CAPACITY,
 INFO_STEPS, INFO_HOST_DIRECT, INFO_SUPERCELL_X, INFO_SUPERCELL_Y, INFO_SUPERCELL_Z, INFO_THREADS,
 INFO_TUNE_TRIALS, INFO_FUSED_STEPS, INFO_FIELD_UPDATE) = range(14)
FIELD_UPDATE_AUTO, FIELD_UPDATE_IN_PLACE, FIELD_UPDATE_FUSED = 0, 1, 2


class PicError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


GATHER_MOMENTUM, GATHER_ENERGY = 0, 1


class SpeciesC(ctypes.Structure):
    _fields_ = [("charge", ctypes.c_double), ("mass", ctypes.c_double),
                ("shape", ctypes.c_int32), ("mobile", ctypes.c_int32),
                ("gather", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Boundary(ctypes.Structure):
    _fields_ = [("open_y", ctypes.c_int32), ("absorber_cells", ctypes.c_int32),
                ("absorber_sigma", ctypes.c_double)]


class AntennaC(ctypes.Structure):
    _fields_ = [("plane_y", ctypes.c_int32), ("reserved", ctypes.c_int32)] + \
        [(k, ctypes.c_double) for k in ("E0", "omega", "w0", "xc", "zc", "tau", "t0")]


class Subdomain(ctypes.Structure):
    _fields_ = [("enable", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("migrant_capacity", ctypes.c_int64), ("id_base", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("sc", ctypes.c_int32 * 3),
                ("threads_per_sc", ctypes.c_int32), ("track_ids", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("sort_every", ctypes.c_int32),
                ("field_update", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("pool_frames", ctypes.c_int64), ("move_capacity", ctypes.c_int64),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ud", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


_lib = None


def library(path: str = LIB_PATH):
    """Load libpic.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpic is not built ({path} missing): run "
                           "paper_1606_02862_gb300.build.build() (nvcc, sm_103a) first")
    L = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.pic_create.argtypes = [ctypes.POINTER(Grid), i32, ctypes.POINTER(ctypes.c_double),
                             ctypes.c_double, ctypes.POINTER(SpeciesC), i32,
                             ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.pic_set_background.argtypes = [vp, i32, ctypes.c_double]
    L.pic_set_boundary.argtypes = [vp, i32, ctypes.POINTER(Boundary)]
    L.pic_set_antenna.argtypes = [vp, i32, ctypes.POINTER(AntennaC)]
    L.pic_shift_window.argtypes = [vp, i32, i32]
    L.pic_load_particles.argtypes = [vp, i32, i32, i64, dp, dp, dp]
    L.pic_write_fields.argtypes = [vp, i32, i32, dp]
    L.pic_step.argtypes = [vp, i32]
    L.pic_step_async.argtypes = [vp, i32]
    L.pic_sync.argtypes = [vp]
    L.pic_read_fields.argtypes = [vp, i32, i32, dp]
    L.pic_count_particles.argtypes = [vp, i32, i32, ctypes.POINTER(i64)]
    L.pic_read_particles.argtypes = [vp, i32, i32, i64, dp, dp, dp, dp, ctypes.POINTER(i64)]
    L.pic_diagnostics.argtypes = [vp, i32, dp]
    L.pic_stage_timing.argtypes = [vp, i32]
    L.pic_stage_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
    L.pic_info.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.pic_set_subdomain.argtypes = [vp, i32, ctypes.POINTER(Subdomain)]
    L.pic_step_stage.argtypes = [vp, i32]
    L.pic_halo_floats.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i64)]
    L.pic_halo_pack.argtypes = [vp, i32, i32, i32, vp]
    L.pic_halo_unpack.argtypes = [vp, i32, i32, i32, vp]
    L.pic_migrant_bytes.argtypes = [vp, ctypes.POINTER(i64)]
    L.pic_migrants_pack.argtypes = [vp, i32, vp]
    L.pic_migrants_accept.argtypes = [vp, i32, vp]
    L.pic_field_energy_noalloc.argtypes = [vp, vp, i64, ctypes.c_double, vp, vp]
    L.pic_last_error.argtypes = [vp]
    L.pic_last_error.restype = ctypes.c_char_p
    L.pic_destroy.argtypes = [vp]
    L.pic_destroy.restype = None
    for name in EXPORTED:
        if name not in ("pic_last_error", "pic_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _f64(a, shape=None):
    """C-contiguous float64 host array (numpy, or a CPU torch tensor)."""
    if a is None:
        return None
    if hasattr(a, "detach") and hasattr(a, "numpy"):
        a = a.detach().numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


@dataclass
class Species:
    charge: float
    mass: float
    shape: int = 2
    mobile: bool = True
    gather: int = GATHER_MOMENTUM


class _TorchMemory:
    """Device allocator callbacks backed by torch's caching allocator."""

    def __init__(self):
        import torch

        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream()
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, _ud):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # noqa: BLE001 - an allocator failure must reach C as NULL
            return None

    def _free(self, ptr, _ud):
        self.torch.cuda.caching_allocator_delete(int(ptr))


class Context:
    """One libpic context: nboxes periodic boxes sharing dx, dt and species."""

    def __init__(self, grids, dx, dt, species, precision=PRECISION_MIXED, sc=(4, 4, 4),
                 threads_per_sc=None, track_ids=False, use_graph=True, pool_frames=0,
                 move_capacity=0, torch_memory=True, sort_every=0, field_update=FIELD_UPDATE_AUTO):
        """sc = (0, 0, 0) and/or threads_per_sc = 0 leave the configuration
        to the library's tuner (at the first step); threads_per_sc = None
        takes the supercell's default (256 threads from 256 cells on, else
        128); field_update picks the field update: the three in-place kernels,
        the fused two-buffer kernel for pairs of steps, or (the default) the
        faster of the two on this context's fields, timed at the first step."""
        if threads_per_sc is None:
            cells = int(sc[0]) * int(sc[1]) * int(sc[2])
            threads_per_sc = 256 if cells >= 256 else 128
        L = library()
        self._L = L
        self._ctx = ctypes.c_void_p()
        grids = [tuple(int(v) for v in g) for g in grids]
        self.grids = grids
        self.species = [s if isinstance(s, Species) else Species(*s) for s in species]
        self.dx = tuple(float(v) for v in dx)
        self.dt = float(dt)
        self.precision = precision
        garr = (Grid * len(grids))(*[Grid(*g) for g in grids])
        sarr = (SpeciesC * len(self.species))(*[SpeciesC(float(s.charge), float(s.mass), int(s.shape),
                                                         int(bool(s.mobile)), int(s.gather), 0)
                                                for s in self.species])
        dxa = (ctypes.c_double * 3)(*self.dx)
        o = Options()
        o.precision = int(precision)
        o.sc[0], o.sc[1], o.sc[2] = (int(v) for v in sc)
        o.threads_per_sc = int(threads_per_sc)
        o.track_ids = int(bool(track_ids))
        o.use_graph = int(bool(use_graph))
        o.sort_every = int(sort_every)
        o.field_update = int(field_update)
        o.pool_frames = int(pool_frames)
        o.move_capacity = int(move_capacity)
        self._mem = None
        if torch_memory:
            self._mem = _TorchMemory()
            o.dev_alloc = self._mem.alloc_fn
            o.dev_free = self._mem.free_fn
            o.stream = ctypes.c_void_p(self._mem.stream.cuda_stream or None)
        self._opts = o
        st = L.pic_create(garr, len(grids), dxa, self.dt, sarr, len(self.species), ctypes.byref(o),
                          ctypes.byref(self._ctx))
        if st != PIC_OK:
            raise PicError(st, "pic_create failed")

    # ------------------------------------------------------------ helpers
    def _check(self, st):
        if st != PIC_OK:
            msg = self._L.pic_last_error(self._ctx)
            raise PicError(st, msg.decode() if msg else "")

    def ncells(self, box):
        g = self.grids[box]
        return g[0] * g[1] * g[2]

    # ------------------------------------------------------------ ABI calls
    def set_background(self, box, rho_bg):
        self._check(self._L.pic_set_background(self._ctx, box, float(rho_bg)))

    def set_boundary(self, box, open_y=False, absorber_cells=0, absorber_sigma=0.0):
        """Open y faces: remove particles leaving through them, and/or damping
        layers of absorber_cells cells (factor exp(-sigma d^2) per step)."""
        b = Boundary(int(bool(open_y)), int(absorber_cells), float(absorber_sigma))
        self._check(self._L.pic_set_boundary(self._ctx, box, ctypes.byref(b)))

    def set_antenna(self, box, plane_y, E0=0.0, omega=0.0, w0=0.0, xc=0.0, zc=0.0, tau=0.0, t0=0.0):
        """Ex current-sheet laser antenna on the node plane y = plane_y (< 0: none)."""
        a = AntennaC(int(plane_y), 0, float(E0), float(omega), float(w0), float(xc), float(zc),
                     float(tau), float(t0))
        self._check(self._L.pic_set_antenna(self._ctx, box, ctypes.byref(a)))

    def shift_window(self, box, cells):
        """Moving window: box moves `cells` (a multiple of the supercell edge) towards +y."""
        self._check(self._L.pic_shift_window(self._ctx, box, int(cells)))

    def steps_taken(self):
        return self.info(INFO_STEPS)

    def config(self):
        """(supercell edges, threads per supercell) in use (mixed form)."""
        return ((self.info(INFO_SUPERCELL_X), self.info(INFO_SUPERCELL_Y), self.info(INFO_SUPERCELL_Z)),
                self.info(INFO_THREADS))

    def load_particles(self, box, species, x, u, w=None):
        x = _f64(x, (-1, 3))
        u = _f64(u, (-1, 3))
        w = _f64(w, (-1,))
        n = x.shape[0]
        if u.shape[0] != n or (w is not None and w.shape[0] != n):
            raise ValueError("x, u, w lengths differ")
        self._check(self._L.pic_load_particles(self._ctx, box, species, n, _p(x), _p(u), _p(w)))

    def load_particles_ptr(self, box, species, n, x_ptr, u_ptr, w_ptr=None):
        """Same as load_particles for host buffers given as raw addresses
        (e.g. pinned torch tensors' data_ptr())."""
        self._check(self._L.pic_load_particles(self._ctx, box, species, int(n), ctypes.c_void_p(x_ptr),
                                               ctypes.c_void_p(u_ptr),
                                               None if w_ptr is None else ctypes.c_void_p(w_ptr)))

    def write_fields(self, box, which, f):
        nz, ny, nx = self.grids[box][2], self.grids[box][1], self.grids[box][0]
        f = _f64(f, (3, nz, ny, nx))
        self._check(self._L.pic_write_fields(self._ctx, box, which, _p(f)))

    def step(self, n=1):
        self._check(self._L.pic_step(self._ctx, int(n)))

    def step_async(self, n=1):
        self._check(self._L.pic_step_async(self._ctx, int(n)))

    def sync(self):
        self._check(self._L.pic_sync(self._ctx))

    def read_fields(self, box, which):
        nx, ny, nz = self.grids[box]
        shape = (nz, ny, nx) if which == FIELD_RHO else (3, nz, ny, nx)
        out = np.empty(shape, dtype=np.float64)
        self._check(self._L.pic_read_fields(self._ctx, box, which, _p(out)))
        return out

    def count_particles(self, box, species):
        n = ctypes.c_int64()
        self._check(self._L.pic_count_particles(self._ctx, box, species, ctypes.byref(n)))
        return n.value

    def read_particles(self, box, species, ids=False):
        n = self.count_particles(box, species)
        x = np.empty((n, 3))
        u = np.empty((n, 3))
        w = np.empty(n)
        pid = np.empty(n, dtype=np.int64) if ids else None
        nout = ctypes.c_int64()
        self._check(self._L.pic_read_particles(self._ctx, box, species, n, _p(x), _p(u), _p(w),
                                               _p(pid), ctypes.byref(nout)))
        out = {"x": x, "u": u, "w": w}
        if ids:
            out["id"] = pid
        return out

    def read_particles_ptr(self, box, species, cap, x_ptr, u_ptr, w_ptr, id_ptr=None):
        """pic_read_particles into host buffers given as raw addresses (e.g.
        pinned torch tensors' data_ptr()); returns the count."""
        nout = ctypes.c_int64()
        vp = ctypes.c_void_p
        self._check(self._L.pic_read_particles(self._ctx, box, species, int(cap), vp(x_ptr), vp(u_ptr),
                                               vp(w_ptr), None if id_ptr is None else vp(id_ptr),
                                               ctypes.byref(nout)))
        return nout.value

    def read_fields_ptr(self, box, which, out_ptr):
        self._check(self._L.pic_read_fields(self._ctx, box, which, ctypes.c_void_p(out_ptr)))

    def diagnostics(self, box):
        out = np.zeros(4)
        self._check(self._L.pic_diagnostics(self._ctx, box, _p(out)))
        return out

    def stage_timing(self, enable=True):
        self._check(self._L.pic_stage_timing(self._ctx, int(bool(enable))))

    def stage_times(self):
        ms = np.zeros(4)
        n = ctypes.c_int64()
        self._check(self._L.pic_stage_times(self._ctx, _p(ms), ctypes.byref(n)))
        return ms, n.value

    def info(self, key):
        v = ctypes.c_int64()
        self._check(self._L.pic_info(self._ctx, int(key), ctypes.byref(v)))
        return v.value

    # ------------------------------------------------------------ z-slab subdomains
    def set_subdomain(self, enable=True, migrant_capacity=0, id_base=0):
        """Make box 0 one z slab of a decomposed box (pic_set_subdomain)."""
        sd = Subdomain(int(bool(enable)), 0, int(migrant_capacity), int(id_base))
        self._check(self._L.pic_set_subdomain(self._ctx, 0, ctypes.byref(sd)))

    def step_stage(self, stage):
        self._check(self._L.pic_step_stage(self._ctx, int(stage)))

    def halo_floats(self, which, side):
        n = ctypes.c_int64()
        self._check(self._L.pic_halo_floats(self._ctx, 0, int(which), int(side), ctypes.byref(n)))
        return n.value

    def halo_pack(self, which, side, buf_ptr):
        self._check(self._L.pic_halo_pack(self._ctx, 0, int(which), int(side), ctypes.c_void_p(buf_ptr)))

    def halo_unpack(self, which, side, buf_ptr):
        self._check(self._L.pic_halo_unpack(self._ctx, 0, int(which), int(side), ctypes.c_void_p(buf_ptr)))

    def migrant_bytes(self):
        n = ctypes.c_int64()
        self._check(self._L.pic_migrant_bytes(self._ctx, ctypes.byref(n)))
        return n.value

    def migrants_pack(self, side, buf_ptr):
        self._check(self._L.pic_migrants_pack(self._ctx, int(side), ctypes.c_void_p(buf_ptr)))

    def migrants_accept(self, side, buf_ptr):
        self._check(self._L.pic_migrants_accept(self._ctx, int(side), ctypes.c_void_p(buf_ptr)))

    def last_error(self):
        msg = self._L.pic_last_error(self._ctx)
        return msg.decode() if msg else ""

    def close(self):
        if self._ctx:
            self._L.pic_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def field_energy_noalloc(E_ptr, B_ptr, ncells, cell_volume, out_ptr, stream=None):
    """pic_field_energy_noalloc on device buffers given as raw addresses:
    writes the FP64 field energy to *out_ptr without allocating device memory."""
    L = library()
    st = L.pic_field_energy_noalloc(ctypes.c_void_p(E_ptr), ctypes.c_void_p(B_ptr), int(ncells),
                                    float(cell_volume), ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(stream) if stream else None)
    if st != PIC_OK:
        raise PicError(st, "pic_field_energy_noalloc failed")


def from_workload(wl, precision=PRECISION_MIXED, sc=(4, 4, 4), threads_per_sc=None, track_ids=False,
                  use_graph=True, **kw) -> Context:
    """Create a context for a workloads.Workload and load its initial state."""
    ctx = Context([(b.nx, b.ny, b.nz) for b in wl.boxes], wl.dx, wl.dt,
                  [Species(s.q, s.m, s.shape, s.mobile, GATHER_ENERGY if getattr(s, "ec", False)
                           else GATHER_MOMENTUM) for s in wl.species], precision=precision,
                  sc=sc, threads_per_sc=threads_per_sc, track_ids=track_ids, use_graph=use_graph,
                  **kw)
    extra = getattr(wl, "extra", None) or {}
    if "boundary" in extra:
        ctx.set_boundary(0, **extra["boundary"])
    if "antenna" in extra:
        ctx.set_antenna(0, **extra["antenna"])
    for bi, b in enumerate(wl.boxes):
        ctx.set_background(bi, b.rho_bg)
        for si, (x, u, w) in enumerate(b.particles):
            ctx.load_particles(bi, si, x, u, w)
        if b.E is not None:
            ctx.write_fields(bi, FIELD_E, b.E)
        if b.B is not None:
            ctx.write_fields(bi, FIELD_B, b.B)
    return ctx
