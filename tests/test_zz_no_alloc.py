"""bp_paste_particles_noalloc: the particle paste for callers that cannot allocate device
memory during a call (applications that hand all device memory to their own pool at
start-up; latency-critical loops where cudaMalloc/cudaFree would synchronise the device).

Called through the C ABI, twice in a row on different inputs, and compared with
bp_paste_particles on the same inputs, for the tensor-core deposit (tile 64) and the SIMT
deposit (tiles 64 and 32).  The device's free memory must not change across the calls (the
library's array and kernels are loaded when the context is created).  Sizes beyond the
fixed maximum return BP_ERANGE and leave the maps as they were.  Collected last so that a
run stopping at the first failure has already run every other test; passes alone and after
the others.
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


@pytest.mark.parametrize("kernel,tile", [("auto", 64), ("simt", 64), ("simt", 32)])
def test_noalloc_paste_matches_paste_particles(api, kernel, tile):
    from paper_2201_02632_gb300 import _lib

    lib = _lib.load()
    ctx = api.Context()      # only the allocation-free entry point runs on this context
    ref_ctx = api.Context()  # the regular paste, with its own scratch
    for c in (ctx, ref_ctx):
        c.set_deposit_kernel(kernel)
        c.set_tiling(pp_tile=tile)
    assert ctx.workspace_bytes() == 0
    g = api.geom(200, 130, 0.0, 0.0, 1.0)
    inputs = []
    for seed in (101, 202):
        a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30, seed=seed)
        rec = assigned_tensor(a)
        ref = api.Maps.zeros(g)
        ref_ctx.paste_particles(rec, g, ref)
        inputs.append((rec, ref, api.Maps.zeros(g)))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call, (rec, ref, got) in enumerate(inputs):
        rc = _paste_noalloc(lib, ctx, rec, g, got)
        assert rc == 0, lib.bp_last_error(ctx._h).decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the calls changed the device's free memory"
    for call, (rec, ref, got) in enumerate(inputs):
        y, b = folded(got)
        yr, br = folded(ref)
        assert_map_parity(y[0], yr[0], what=f"y, call {call + 1}")
        assert_map_parity(b[0], br[0], what=f"b, call {call + 1}")
        assert np.count_nonzero(y) > 1000
    # the context's own scratch was never used
    assert ctx.workspace_bytes() == 0
    ctx.close()
    ref_ctx.close()


def test_noalloc_paste_refuses_sizes_beyond_its_array(api):
    from paper_2201_02632_gb300 import _lib

    lib = _lib.load()
    ctx = api.Context()
    a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30, seed=303)
    rec = assigned_tensor(a)
    # more particles than the array holds: refused before any work is queued
    g = api.geom(200, 130, 0.0, 0.0, 1.0)
    rc = lib.bp_paste_particles_noalloc(ctx._h, (1 << 19) + 1, C.c_void_p(rec.data_ptr()),
                                        C.byref(g), 0, None, None, None, None)
    assert rc == _lib.BP_ERANGE and b"exceed the limit" in lib.bp_last_error(ctx._h)

    def refused(rec, g, what):
        maps = api.Maps.zeros(g)
        for t in (maps.y, maps.b, maps.ylo, maps.blo):
            t.normal_()
        before = [t.clone() for t in (maps.y, maps.b, maps.ylo, maps.blo)]
        rc = _paste_noalloc(lib, ctx, rec, g, maps)
        torch.cuda.synchronize()
        msg = lib.bp_last_error(ctx._h)
        assert rc == _lib.BP_ERANGE and what in msg, msg
        for t, t0 in zip((maps.y, maps.b, maps.ylo, maps.blo), before):
            assert torch.equal(t, t0)

    # more tiles than the array holds (65 x 65 tiles of 64 pixels > 4096)
    refused(rec, api.geom(65 * 64, 65 * 64, 0.0, 0.0, 1.0), b"tiles exceed the limit")
    # more (tile, particle) pairs than the array holds: 2^19 particles with 80-pixel kernels
    # on a 256^2 map touch at least 4 tiles of 64 pixels each (> 2^20 pairs)
    n = 1 << 19
    rng = np.random.default_rng(4)
    px = rng.uniform(60.0, 196.0, n)
    py = rng.uniform(60.0, 196.0, n)
    big = {"fx": (px - np.floor(px)).astype(np.float32), "fy": (py - np.floor(py)).astype(np.float32),
           "ix": np.floor(px).astype(np.int32), "iy": np.floor(py).astype(np.int32),
           "hp": np.full(n, 80.0, np.float32), "Y": np.ones(n, np.float32),
           "B": np.ones(n, np.float32), "kind": np.zeros(n, np.int32)}
    refused(assigned_tensor(big), api.geom(256, 256, 0.0, 0.0, 1.0), b"pairs exceed the limit")
    torch.cuda.synchronize()
    ctx.close()
