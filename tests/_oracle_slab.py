"""One z slab of a periodic box advanced by the FP64 oracle, in the form
paper_1606_02862_gb300.decomp.SlabStepper drives (test infrastructure).

The slab's fields live on an extended grid of nz + 2H planes (H = 3 ghost
planes below and above, more than a TSC particle's gather and deposit
reach plus a half-cell move), indexed periodically by the oracle over that
extended grid: every value the interior reads lies within H planes of it,
so the wrap only ever touches ghost planes, which the exchange overwrites
(E, B) or sends away (J) before anything reads them.  Messages are float64
torch tensors:
  E, B to side s: the H interior planes next to face s (the neighbour's
      ghosts); from side s: into the ghost planes of face s;
  J to side s: the ghost planes of face s (deposits into the neighbour's
      cells); from side s: added into the H interior planes next to face s;
  migrants to side s: [count, then (species, x, y, z past the face, ux,
      uy, uz, w, id) per particle] for the particles whose z left through
      face s.
"""
from __future__ import annotations

import ctypes

import numpy as np

H = 3
REC = 9


class OracleSlab:
    def __init__(self, orc, nx, ny, nz, dt, species, E=None, B=None, cap=4096):
        """species: list of (q, m, order, x, u, w, ids) in slab coordinates
        (z in [0, nz)); E, B: (3, nz, ny, nx) or None."""
        self.orc = orc
        self.nx, self.ny, self.nz, self.dt = nx, ny, nz, dt
        self.g = orc.grid(nx, ny, nz + 2 * H)
        shp = (3, nz + 2 * H, ny, nx)
        self.E, self.B, self.J = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        if E is not None:
            self.E[:, H:H + nz] = E
        if B is not None:
            self.B[:, H:H + nz] = B
        self.species = []
        for q, m, order, x, u, w, ids in species:
            x = np.array(x, dtype=np.float64).reshape(-1, 3)
            x[:, 2] += H
            sp = orc.Species(q, m, order, x, u, w)
            sp.ids = np.asarray(ids, dtype=np.int64).copy()
            self.species.append(sp)
        self.cap = cap
        self.out = [np.zeros(1 + cap * REC), np.zeros(1 + cap * REC)]

    # ---------------------------------------------------------------- stages
    def step_stage(self, stage):
        from paper_1606_02862_gb300 import pic

        from oracle.oracle import _ptr

        L = self.orc.lib()
        if stage == pic.STAGE_PUSH:
            self.J[...] = 0.0
            for o in self.out:
                o[0] = 0.0
            for si, sp in enumerate(self.species):
                rc = L.orc_push_deposit(ctypes.byref(self.g), float(self.dt), int(sp.order), float(sp.q),
                                        float(sp.m), _ptr(self.E), _ptr(self.B),
                                        _ptr(self.J), int(sp.x.shape[0]), _ptr(sp.x),
                                        _ptr(sp.u), _ptr(sp.w), 0, 0)
                assert rc == 0
                z = sp.x[:, 2]
                for side, sel in ((0, z < H), (1, z >= H + self.nz)):
                    idx = np.nonzero(sel)[0]
                    o = self.out[side]
                    n0 = int(o[0])
                    assert n0 + idx.size <= self.cap
                    zr = z[idx] - H if side == 0 else z[idx] - H - self.nz
                    w = sp.w[idx] if sp.w is not None else np.ones(idx.size)
                    rec = np.column_stack([np.full(idx.size, si), sp.x[idx, 0], sp.x[idx, 1], zr, sp.u[idx],
                                           w, sp.ids[idx]])
                    o[1 + n0 * REC:1 + (n0 + idx.size) * REC] = rec.ravel()
                    o[0] = n0 + idx.size
                keep = (z >= H) & (z < H + self.nz)
                self._keep(sp, keep)
        elif stage == pic.STAGE_B_FIRST or stage == pic.STAGE_B_SECOND:
            self.orc.yee_b(self.g, 0.5 * self.dt, self.E, self.B)
        elif stage == pic.STAGE_E:
            self.orc.yee_e(self.g, self.dt, self.E, self.B, self.J)

    @staticmethod
    def _keep(sp, keep):
        sp.x = np.ascontiguousarray(sp.x[keep])
        sp.u = np.ascontiguousarray(sp.u[keep])
        if sp.w is not None:
            sp.w = np.ascontiguousarray(sp.w[keep])
        sp.ids = sp.ids[keep]

    # ---------------------------------------------------------------- halos
    def _field(self, which):
        from paper_1606_02862_gb300 import pic

        return {pic.FIELD_E: self.E, pic.FIELD_B: self.B, pic.FIELD_J: self.J}[which]

    def _planes(self, which, side, pack):
        from paper_1606_02862_gb300 import pic

        ghosts = (which == pic.FIELD_J) == pack
        if ghosts:
            return slice(0, H) if side == 0 else slice(H + self.nz, 2 * H + self.nz)
        return slice(H, 2 * H) if side == 0 else slice(self.nz, H + self.nz)

    def halo_floats(self, which, side):
        return 3 * H * self.ny * self.nx

    def halo_pack(self, which, side, buf):
        buf.numpy()[:] = self._field(which)[:, self._planes(which, side, True)].ravel()

    def halo_unpack(self, which, side, buf):
        from paper_1606_02862_gb300 import pic

        F = self._field(which)
        sl = self._planes(which, side, False)
        v = buf.numpy().reshape(3, H, self.ny, self.nx)
        if which == pic.FIELD_J:
            F[:, sl] += v
        else:
            F[:, sl] = v

    # ---------------------------------------------------------------- migrants
    def migrant_bytes(self):
        return 1 + self.cap * REC

    def migrants_pack(self, side, buf):
        buf.numpy()[:] = self.out[side]

    def migrants_accept(self, side, buf):
        b = buf.numpy()
        n = int(b[0])
        rec = b[1:1 + n * REC].reshape(n, REC)
        for si, sp in enumerate(self.species):
            r = rec[rec[:, 0] == si]
            if r.size == 0:
                continue
            x = r[:, 1:4].copy()
            x[:, 2] += H if side == 0 else H + self.nz
            sp.x = np.ascontiguousarray(np.vstack([sp.x, x]))
            sp.u = np.ascontiguousarray(np.vstack([sp.u, r[:, 4:7]]))
            if sp.w is not None:
                sp.w = np.ascontiguousarray(np.concatenate([sp.w, r[:, 7]]))
            sp.ids = np.concatenate([sp.ids, r[:, 8].astype(np.int64)])

    # ---------------------------------------------------------------- results
    def interior(self, F):
        return F[:, H:H + self.nz]

    def particles(self, si):
        """(ids, x in slab coordinates, u) sorted by id."""
        sp = self.species[si]
        o = np.argsort(sp.ids)
        x = sp.x[o].copy()
        x[:, 2] -= H
        return sp.ids[o], x, sp.u[o]
