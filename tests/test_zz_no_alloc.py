"""pic_field_energy_noalloc: the field energy without any device allocation.

Callers that cannot allocate device memory when they need the number (hosts
that hand out only pre-reserved memory) get the same FP64 field energy as
pic_diagnostics out[0] from arrays they own.  The test builds a field state with a context, copies E and B to
device tensors, and calls the entry point twice in a row through the C ABI
-- once on the state, once on a scaled copy -- checking each result against
the context's own reduction.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import math

import numpy as np
import pytest

from _gpu_helpers import ctx_from, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-11  # both sides are FP64 sums of the same values, in different orders


def _state():
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(21)
    n = (16, 24, 8)
    x = W.uniform_in_cells(rng, *n, 4)
    u = W.maxwellian(rng, x.shape[0], 0.2)
    E = rng.normal(0, 0.02, (3, n[2], n[1], n[0]))
    B = rng.normal(0, 0.02, (3, n[2], n[1], n[0]))
    box = W.BoxInit(*n, particles=[(x, u, np.full(x.shape[0], 0.005))], E=E, B=B, rho_bg=0.02)
    return W.Workload("noalloc", W.DT_HALF_COURANT, [W.SpeciesDef("e", -1.0, 1.0, 2)], [box])


def test_noalloc_field_energy_matches_diagnostics_twice():
    torch = require_gpu()
    from paper_1606_02862_gb300 import pic

    wl = _state()
    ctx = ctx_from(wl)
    try:
        ctx.step(3)
        E = ctx.read_fields(0, pic.FIELD_E)
        B = ctx.read_fields(0, pic.FIELD_B)
        want = ctx.diagnostics(0)[0]
    finally:
        ctx.close()
    ncells = E.shape[1] * E.shape[2] * E.shape[3]
    stream = torch.cuda.current_stream().cuda_stream
    Ed = torch.from_numpy(E).cuda()
    Bd = torch.from_numpy(B).cuda()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for scale in (1.0, 3.0):  # two calls in a row share the scratch array
        Es = Ed * scale
        Bs = Bd * scale
        torch.cuda.synchronize()
        pic.field_energy_noalloc(Es.data_ptr(), Bs.data_ptr(), ncells, 1.0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = float(out.item())
        assert math.isfinite(got)
        assert abs(got - scale * scale * want) <= TOL * scale * scale * want, (scale, got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = require_gpu()
    from paper_1606_02862_gb300 import pic

    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as ei:
        # the size check fires before anything reads the (small) buffers
        pic.field_energy_noalloc(buf.data_ptr(), buf.data_ptr(), 44_739_243, 1.0, buf.data_ptr())
    assert ei.value.status == 1
