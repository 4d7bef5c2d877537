"""Particle load and read-back from page-locked host memory.

When every host array of a pic_load_particles / pic_read_particles call lies
inside one page-locked allocation, the mixed form converts the particles in
place over the host link instead of staging them through device memory.
The two paths must give the same results: every particle (matched by id)
bit-identical after a load, and the same context read back into pinned and
into pageable arrays bit-identical element by element.  Where particles go
within a frame list depends on the order of device atomics, so two
contexts are compared by id, and after a few steps within the mixed form's
per-step tolerance.  A call with one pageable array among pinned ones
takes the staged path.
"""
import numpy as np
import pytest

from _gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


def _state(seed=5, n=(24, 16, 16), ppc=6):
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(seed)
    x = W.uniform_in_cells(rng, *n, ppc)
    u = W.maxwellian(rng, x.shape[0], 0.1)
    w = rng.uniform(0.5, 1.5, x.shape[0]) * 0.01
    return n, x, u, w


def _ctx(n):
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    ctx = pic.Context([n], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2, True, 0)],
                      sc=(8, 4, 4), threads_per_sc=256, track_ids=True)
    ctx.set_background(0, 0.01)
    return ctx


def _pinned(torch, a, dtype=None):
    t = torch.empty(a.shape, dtype=dtype or torch.float64, pin_memory=True)
    t.numpy()[...] = a
    return t


def _by_id(r):
    o = np.argsort(r[3])
    return tuple(v[o] for v in r)


def _read(torch, ctx, npart, pinned):
    if pinned:
        X = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
        U = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
        Wt = torch.empty((npart,), dtype=torch.float64, pin_memory=True)
        I = torch.empty((npart,), dtype=torch.int64, pin_memory=True)
        got = ctx.read_particles_ptr(0, 0, npart, X.data_ptr(), U.data_ptr(), Wt.data_ptr(), I.data_ptr())
        assert got == npart
        return X.numpy().copy(), U.numpy().copy(), Wt.numpy().copy(), I.numpy().copy()
    p = ctx.read_particles(0, 0, ids=True)
    return p["x"], p["u"], p["w"], p["id"]


@pytest.mark.parametrize("steps", [0, 3])
def test_pinned_load_and_read_match_the_staged_path(steps):
    from paper_1606_02862_gb300 import pic

    torch = require_gpu()
    n, x, u, w = _state()
    npart = x.shape[0]
    Xp, Up, Wp = _pinned(torch, x), _pinned(torch, u), _pinned(torch, w)
    a = _ctx(n)  # staged: pageable numpy arrays
    b = _ctx(n)  # direct: page-locked tensors
    try:
        a.load_particles(0, 0, x, u, w)
        b.load_particles_ptr(0, 0, npart, Xp.data_ptr(), Up.data_ptr(), Wp.data_ptr())
        assert a.info(pic.INFO_HOST_DIRECT) == 0 and b.info(pic.INFO_HOST_DIRECT) == 1
        if steps:
            a.step(steps)
            b.step(steps)
        ra = _by_id(_read(torch, a, npart, pinned=False))
        rb = _read(torch, b, npart, pinned=True)
        rc = _read(torch, b, npart, pinned=False)
        assert b.info(pic.INFO_HOST_DIRECT) == 2  # the pinned read converted in place
        for vb, vc in zip(rb, rc):  # one context, two read paths: element by element
            assert np.array_equal(vb, vc)
        rb = _by_id(rb)
        assert np.array_equal(rb[3], np.arange(npart)) and np.array_equal(ra[3], rb[3])
        if steps == 0:
            for va, vb in zip(ra[:3], rb[:3]):
                assert np.array_equal(va, vb)
        else:
            d = rb[0] - ra[0]
            d -= np.array(n) * np.round(d / np.array(n))
            assert np.max(np.abs(d)) <= 1e-5
            assert np.max(np.abs(rb[1] - ra[1])) <= 1e-5 * np.max(np.abs(ra[1]))
            assert np.array_equal(rb[2], ra[2])
            Ea, Eb = a.read_fields(0, 0), b.read_fields(0, 0)
            assert np.max(np.abs(Ea - Eb)) <= 1e-5 * np.max(np.abs(Ea))
    finally:
        a.close()
        b.close()


def test_mixed_pinned_and_pageable_arrays():
    from paper_1606_02862_gb300 import pic

    torch = require_gpu()
    n, x, u, w = _state(seed=6)
    npart = x.shape[0]
    Xp = _pinned(torch, x)
    u_c = np.ascontiguousarray(u)
    w_c = np.ascontiguousarray(w)
    a = _ctx(n)
    b = _ctx(n)
    try:
        a.load_particles(0, 0, x, u, w)
        # x page-locked, u and w pageable: the whole call takes the staged path
        b.load_particles_ptr(0, 0, npart, Xp.data_ptr(), u_c.ctypes.data, w_c.ctypes.data)
        assert b.info(pic.INFO_HOST_DIRECT) == 0
        ra = _by_id(_read(torch, a, npart, pinned=False))
        # read-back into a pinned x and pageable u, w, ids
        xo = torch.empty((npart, 3), dtype=torch.float64, pin_memory=True)
        uo = np.empty((npart, 3))
        wo = np.empty(npart)
        io = np.empty(npart, dtype=np.int64)
        got = b.read_particles_ptr(0, 0, npart, xo.data_ptr(), uo.ctypes.data, wo.ctypes.data, io.ctypes.data)
        assert got == npart and b.info(pic.INFO_HOST_DIRECT) == 0
        for va, vb in zip(ra, _by_id((xo.numpy(), uo, wo, io))):
            assert np.array_equal(va, vb)
    finally:
        a.close()
        b.close()


def test_pinned_subrange_of_a_larger_buffer():
    """Views into the middle of one pinned allocation load in place."""
    from paper_1606_02862_gb300 import pic

    torch = require_gpu()
    n, x, u, w = _state(seed=7)
    npart = x.shape[0]
    pad = 1000
    X = torch.empty((npart + 2 * pad, 3), dtype=torch.float64, pin_memory=True)
    U = torch.empty((npart + 2 * pad, 3), dtype=torch.float64, pin_memory=True)
    Wt = torch.empty((npart + 2 * pad,), dtype=torch.float64, pin_memory=True)
    X.numpy()[pad:pad + npart] = x
    U.numpy()[pad:pad + npart] = u
    Wt.numpy()[pad:pad + npart] = w
    a = _ctx(n)
    b = _ctx(n)
    try:
        a.load_particles(0, 0, x, u, w)
        b.load_particles_ptr(0, 0, npart, X[pad].data_ptr(), U[pad].data_ptr(), Wt[pad:].data_ptr())
        assert b.info(pic.INFO_HOST_DIRECT) == 1
        ra = _by_id(_read(torch, a, npart, pinned=False))
        rb = _by_id(_read(torch, b, npart, pinned=True))
        for va, vb in zip(ra, rb):
            assert np.array_equal(va, vb)
    finally:
        a.close()
        b.close()


def test_pinned_load_without_weights():
    """w = NULL (all ones) on the in-place path equals the staged path."""
    from paper_1606_02862_gb300 import pic

    torch = require_gpu()
    n, x, u, _ = _state(seed=8)
    npart = x.shape[0]
    Xp, Up = _pinned(torch, x), _pinned(torch, u)
    a = _ctx(n)
    b = _ctx(n)
    try:
        a.load_particles(0, 0, x, u)
        b.load_particles_ptr(0, 0, npart, Xp.data_ptr(), Up.data_ptr(), None)
        assert b.info(pic.INFO_HOST_DIRECT) == 1
        ra = _by_id(_read(torch, a, npart, pinned=False))
        rb = _by_id(_read(torch, b, npart, pinned=True))
        for va, vb in zip(ra, rb):
            assert np.array_equal(va, vb)
        assert np.all(rb[2] == 1.0)
    finally:
        a.close()
        b.close()


def test_pinned_field_read():
    """pic_read_fields into a page-locked array equals the staged read."""
    from paper_1606_02862_gb300 import pic

    torch = require_gpu()
    n, x, u, w = _state(seed=9)
    ctx = _ctx(n)
    try:
        ctx.load_particles(0, 0, x, u, w)
        ctx.step(2)
        nx, ny, nz = n
        for which in (pic.FIELD_E, pic.FIELD_B, pic.FIELD_J):
            before = ctx.info(pic.INFO_HOST_DIRECT)
            ref = ctx.read_fields(0, which)
            assert ctx.info(pic.INFO_HOST_DIRECT) == before
            out = torch.empty((3, nz, ny, nx), dtype=torch.float64, pin_memory=True)
            ctx.read_fields_ptr(0, which, out.data_ptr())
            assert ctx.info(pic.INFO_HOST_DIRECT) == before + 1
            assert np.array_equal(out.numpy(), ref)
    finally:
        ctx.close()
