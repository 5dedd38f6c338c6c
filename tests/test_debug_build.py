"""The debug build (-DBP_DEBUG): device-side index checks in the particle paste's kernels that
skip a misplaced store and record the check's site in the context's debug word.

On the CPU: the debug variant builds and exports the same entry points as the release build,
and says it is a debug build.  On the GPU (a child process loads the debug library through
BP_LIB): the read-back reports a site the self-test records and clears it; pastes through
every deposit kernel (tensor cores with split work units, small particles, SIMT at tiles 64
and 32) and the pair list record no failed check; and the debug build's maps are bit-identical
to the release build's (the checks change no arithmetic)."""
import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2201_02632_gb300 import _lib
from paper_2201_02632_gb300 import build as B

ROOT = os.path.join(os.path.dirname(__file__), "..")


def _exports(path):
    lib = C.CDLL(path)
    return {n for n in _lib.EXPORTS if hasattr(lib, n)}, lib


def test_debug_build_exports_the_release_entry_points():
    dbg = B.build(debug=True)
    rel = B.build()
    e_dbg, ldbg = _exports(dbg)
    e_rel, lrel = _exports(rel)
    assert e_dbg == e_rel == set(_lib.EXPORTS)
    assert ldbg.bp_debug_build() == 1 and lrel.bp_debug_build() == 0


CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ".")
from paper_2201_02632_gb300 import api, _lib, inputs as I
from tests.gpu_common import assigned_tensor
import ctypes as C

def status(ctx):
    s = C.c_int(-1)
    assert ctx._L.bp_debug_status(ctx._h, C.byref(s)) == 0
    return s.value

ctx = api.Context()
out = {"debug_build": ctx._L.bp_debug_build()}
assert ctx._L.bp_debug_selftest(ctx._h, 777) == 0
out["selftest"] = [status(ctx), status(ctx)]
rng = np.random.default_rng(5)
n, nx, ny = 60000, 300, 200
hp = np.where(rng.random(n) < 0.75, rng.exponential(2.0, n), rng.uniform(8.0, 60.0, n))
hp[rng.random(n) < 0.02] = 0.0
a = I.deposit_inputs(rng.uniform(-10, nx + 10, n), rng.uniform(-10, ny + 10, n), hp,
                     rng.uniform(0, 1e-6, n), rng.normal(0, 1e-6, n), rng.integers(0, 2, n))
rec = assigned_tensor(a)
g = api.geom(nx, ny, 0.0, 0.0, 1.0)
maps = {}
for name, kernel, tile, span, unit in (("tc", "auto", 64, 0, 512), ("small", "auto", 64, 8, 0),
                                       ("simt64", "simt", 64, 0, 0), ("simt32", "simt", 32, 0, 0)):
    ctx.set_deposit_kernel(kernel)
    ctx.set_tiling(pp_tile=tile, pp_unit=unit)
    ctx.set_small_span(span)
    m = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, m)
    k, v = ctx.pp_pairs(rec, g, tile)
    torch.cuda.synchronize()
    maps[name] = [m.y.cpu().numpy(), m.ylo.cpu().numpy(), m.b.cpu().numpy(), m.blo.cpu().numpy()]
    out[name] = status(ctx)
np.savez(sys.argv[1], **{f"{k}_{i}": a for k, v in maps.items() for i, a in enumerate(v)})
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_debug_build_records_nothing_and_matches_release(tmp_path):
    dbg = B.build(debug=True)
    outs = {}
    for tag, path in (("debug", dbg), ("release", B.build())):
        f = tmp_path / f"{tag}.npz"
        r = subprocess.run([sys.executable, "-c", CHILD, str(f)], cwd=ROOT,
                           env=dict(os.environ, BP_LIB=path), capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[tag] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(f))
    d, dm = outs["debug"]
    rl, rm = outs["release"]
    assert d["debug_build"] == 1 and rl["debug_build"] == 0
    assert d["selftest"] == [777, 0] and rl["selftest"] == [777, 0]
    for name in ("tc", "small", "simt64", "simt32"):
        assert d[name] == 0, (name, d[name])
    assert sorted(dm.files) == sorted(rm.files)
    for k in dm.files:
        np.testing.assert_array_equal(dm[k], rm[k], err_msg=k)
