"""Comparison helpers shared by the parity tests."""
import numpy as np

# Floating-point parity bar for maps: relative L2 over the map, and per-pixel relative
# error on pixels brighter than 1% of the map's maximum |value|.
MAP_REL_L2 = 1e-5
MAP_PIX_REL = 1e-4


def rel_l2(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref.ravel())
    return np.linalg.norm((got - ref).ravel()) / den if den > 0 else np.linalg.norm(got.ravel())


def max_rel_bright(got, ref, frac=0.01):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    m = np.abs(ref).max()
    if m == 0:
        return 0.0
    mask = np.abs(ref) > frac * m
    return float(np.max(np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])))


def assert_map_parity(got, ref, l2=MAP_REL_L2, pix=MAP_PIX_REL, what="map"):
    e2 = rel_l2(got, ref)
    ep = max_rel_bright(got, ref)
    assert e2 <= l2 and ep <= pix, f"{what}: rel L2 {e2:.3g} (<= {l2}), bright pixel {ep:.3g} (<= {pix})"
    return e2, ep
