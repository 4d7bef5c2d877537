"""Helpers for the GPU parity tests: move a libpic state into the FP64
oracle and compare the two after the same number of steps."""
from __future__ import annotations

import numpy as np


def require_gpu():
    import pytest
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    return torch


def ctx_from(wl, **kw):
    from paper_1606_02862_gb300 import pic

    kw.setdefault("track_ids", True)
    return pic.from_workload(wl, **kw)


def oracle_state_from_gpu(orc, ctx, wl, box, **state_kw):
    """The GPU's current state of one box, read back in FP64, as an oracle
    State (particles of each species sorted by id, the ids attached to the
    oracle species as `ids`).  state_kw go to the State (open-y options, t)."""
    from paper_1606_02862_gb300 import pic

    b = wl.boxes[box]
    E = ctx.read_fields(box, pic.FIELD_E)
    B = ctx.read_fields(box, pic.FIELD_B)
    species = []
    ids = []
    for si, sd in enumerate(wl.species):
        p = ctx.read_particles(box, si, ids=True)
        order = np.argsort(p["id"])
        ids.append(p["id"][order])
        osp = orc.Species(q=sd.q, m=sd.m, order=sd.shape, x=p["x"][order], u=p["u"][order],
                          w=p["w"][order], mobile=sd.mobile, ec=getattr(sd, "ec", False))
        osp.ids = p["id"][order]
        species.append(osp)
    st = orc.State(b.nx, b.ny, b.nz, wl.dt, dx=wl.dx, E=E, B=B, species=species, rho_bg=b.rho_bg,
                   **state_kw)
    return st, ids


def rel_max(a, b):
    scale = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / scale)


def compare_box(orc_state, ids, ctx, wl, box, tol_field, tol_x, tol_u, check_j=True):
    """Fields (relative to the oracle's max norm), then every particle by id:
    periodic position difference in cells and momentum relative to max |u|."""
    from paper_1606_02862_gb300 import pic

    out = {}
    for name, which, ref in (("E", pic.FIELD_E, orc_state.E), ("B", pic.FIELD_B, orc_state.B),
                             ("J", pic.FIELD_J, orc_state.J)):
        if name == "J" and not check_j:
            continue
        got = ctx.read_fields(box, which)
        if np.max(np.abs(ref)) == 0.0:
            assert np.max(np.abs(got)) == 0.0, name
            out[name] = 0.0
            continue
        err = rel_max(got, ref)
        out[name] = err
        assert err <= tol_field, (name, err)
    b = wl.boxes[box]
    N = np.array([b.nx, b.ny, b.nz], dtype=float)
    for si, sp in enumerate(orc_state.species):
        p = ctx.read_particles(box, si, ids=True)
        order = np.argsort(p["id"])
        gid = p["id"][order]
        assert np.array_equal(gid, ids[si]), "particle ids changed"
        d = p["x"][order] - sp.x
        d -= N * np.round(d / N)
        ex = float(np.max(np.abs(d))) if d.size else 0.0
        umax = max(float(np.max(np.abs(sp.u))) if sp.u.size else 0.0, 1e-30)
        eu = float(np.max(np.abs(p["u"][order] - sp.u))) / umax if d.size else 0.0
        out[f"x{si}"] = ex
        out[f"u{si}"] = eu
        assert ex <= tol_x, (si, ex)
        assert eu <= tol_u, (si, eu)
        assert np.all(p["x"] >= 0.0) and np.all(p["x"] < N)
    return out
