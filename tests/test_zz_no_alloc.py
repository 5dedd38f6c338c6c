"""bp_paste_particles_noalloc: the particle paste for callers that cannot allocate device
memory during a call (applications that hand all device memory to their own pool at
start-up; latency-critical loops where cudaMalloc/cudaFree would synchronise the device).

Called through the C ABI, twice in a row on different inputs, and compared with
bp_paste_particles on the same inputs.  Collected last so that a run stopping at the
first failure has already run every other test; passes alone and after the others.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, assigned_tensor, folded  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


def _paste_noalloc(lib, ctx, rec, g, maps, select=0):
    p = lambda t: C.c_void_p(t.data_ptr())
    return lib.bp_paste_particles_noalloc(ctx._h, rec.shape[0], p(rec), C.byref(g), select,
                                          p(maps.y), p(maps.b), p(maps.ylo), p(maps.blo))


def test_noalloc_paste_matches_paste_particles(api):
    from paper_2201_02632_gb300 import _lib

    lib = _lib.load()
    ctx = api.Context()      # only the allocation-free entry point runs on this context
    ref_ctx = api.Context()  # the regular paste, with its own scratch
    assert ctx.workspace_bytes() == 0
    g = api.geom(200, 130, 0.0, 0.0, 1.0)
    for call, seed in enumerate((101, 202)):
        a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30, seed=seed)
        rec = assigned_tensor(a)
        ref = api.Maps.zeros(g)
        ref_ctx.paste_particles(rec, g, ref)
        got = api.Maps.zeros(g)
        rc = _paste_noalloc(lib, ctx, rec, g, got)
        assert rc == 0, lib.bp_last_error(ctx._h).decode()
        torch.cuda.synchronize()
        y, b = folded(got)
        yr, br = folded(ref)
        assert_map_parity(y[0], yr[0], what=f"y, call {call + 1}")
        assert_map_parity(b[0], br[0], what=f"b, call {call + 1}")
        assert np.count_nonzero(y) > 1000
    # the context's own scratch was never used
    assert ctx.workspace_bytes() == 0
    # sizes beyond the fixed maximum are refused before any work is queued
    big = _lib.BP_ERANGE
    rc = lib.bp_paste_particles_noalloc(ctx._h, (1 << 19) + 1, C.c_void_p(rec.data_ptr()),
                                        C.byref(g), 0, None, None, None, None)
    assert rc == big and b"exceed the limit" in lib.bp_last_error(ctx._h)
    torch.cuda.synchronize()
    ctx.close()
    ref_ctx.close()
