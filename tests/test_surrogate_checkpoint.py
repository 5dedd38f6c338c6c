"""Surrogate checkpoints: save then load gives back every array (weights, feature and
target normalisation, training hull, Adam moments) bit for bit and the step count, and a
file that is not a checkpoint, or is cut short, is refused.  On the GPU, a trained
surrogate reloaded from its checkpoint solves a catalogue to bit-identical models and
resumes training where it stopped."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300.surrogate import MAGIC, Surrogate


def _filled(device="cpu"):
    s = Surrogate.init(device, seed=3)
    g = torch.Generator().manual_seed(5)
    s.m = torch.randn(s.params.shape, generator=g).to(device)
    s.v = torch.rand(s.params.shape, generator=g).to(device)
    s.norm[6:9] = torch.tensor([0.25, -1.5, 3.0])
    s.step = 1234
    return s


def test_checkpoint_round_trip_is_exact(tmp_path):
    s = _filled()
    p = tmp_path / "s.bin"
    s.save(p)
    r = Surrogate.load(p, "cpu")
    for name in ("params", "norm", "hull", "m", "v"):
        a, b = getattr(s, name), getattr(r, name)
        assert a.dtype == b.dtype == torch.float32 and a.shape == b.shape, name
        assert torch.equal(a, b), name
    assert r.step == 1234
    # saving the reloaded surrogate writes the same bytes
    q = tmp_path / "r.bin"
    r.save(q)
    assert p.read_bytes() == q.read_bytes()


def test_checkpoint_refuses_other_files(tmp_path):
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"NOTASURR" + bytes(64))
    with pytest.raises(ValueError):
        Surrogate.load(bad, "cpu")
    s = _filled()
    good = tmp_path / "good.bin"
    s.save(good)
    data = good.read_bytes()
    assert data[:8] == MAGIC
    cut = tmp_path / "cut.bin"
    cut.write_bytes(data[: len(data) // 2])
    with pytest.raises((ValueError, struct_error())):
        Surrogate.load(cut, "cpu")


def struct_error():
    import struct

    return struct.error


@pytest.mark.gpu
def test_reloaded_surrogate_solves_identically_and_resumes(tmp_path):
    from paper_2201_02632_gb300 import api
    from paper_2201_02632_gb300 import inputs as I

    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c = api.Context()
    M, cc, z, prm = I.surrogate_halos(20000, seed=21)
    s = Surrogate.init("cuda", seed=1)
    s.fit(c, cuda(M), cuda(cc), cuda(z), cuda(prm), epochs=3, batch=2048)
    p = tmp_path / "trained.bin"
    s.save(p)
    r = Surrogate.load(p, "cuda")
    Mt, ct, zt, pt = I.surrogate_halos(500, seed=22)
    for mode in (4, 0):  # polished, and the gated FP32 acceptance
        ma, sa = s.solve(c, cuda(Mt), cuda(ct), cuda(zt), cuda(pt), polish_iter=mode,
                         raise_on_noconv=False)
        mb, sb = r.solve(c, cuda(Mt), cuda(ct), cuda(zt), cuda(pt), polish_iter=mode,
                         raise_on_noconv=False)
        assert torch.equal(sa, sb) and torch.equal(ma, mb), mode
    # one more epoch from the original and from the reloaded copy: the same parameters
    s.fit(c, cuda(M), cuda(cc), cuda(z), cuda(prm), epochs=1, batch=2048)
    r.fit(c, cuda(M), cuda(cc), cuda(z), cuda(prm), epochs=1, batch=2048)
    assert r.step == s.step
    assert torch.equal(r.params, s.params)
    torch.cuda.synchronize()
    c.close()
