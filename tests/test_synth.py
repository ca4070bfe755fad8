"""The seeded input generator: deterministic, and its C fill equals the
closed form evaluated in numpy."""
import numpy as np

import synth


def test_response_matches_closed_form():
    rng = np.random.default_rng(0)
    pa = rng.uniform(0, 100, (3, 3))
    pb = rng.uniform(0, 100, (4, 3))
    out = synth.response(pa, pb, 40, 3.5)
    d = np.linalg.norm(pa[:, None, :] - pb[None, :, :], axis=2)
    t = np.arange(40)[None, None, :] - (d / 3.5)[:, :, None]
    a = (np.pi * 0.1 * t) ** 2
    ref = np.exp(-d / 50.0)[:, :, None] * (1 - 2 * a) * np.exp(-a)
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())
    out32 = synth.response(pa, pb, 40, 3.5, dtype=np.float32)
    assert np.allclose(out32, ref, rtol=1e-7, atol=1e-8)


def test_workloads_are_deterministic():
    wl = synth.WORKLOADS["tiny"]
    g1, g2 = wl.geometry_obj(), wl.geometry_obj()
    assert np.array_equal(g1.grid, g2.grid)
    assert np.array_equal(wl.slip(g1), wl.slip(g2))
    wl = synth.WORKLOADS["batched"]
    geom = synth.geometry_plane(wl.Ns, 50, wl.No, wl.geom_seed)
    s = wl.slip(geom, B=4)
    dur = wl.durations(4)
    for b in range(4):
        assert np.all(s[b][:, dur[b]:] == 0)
    assert np.all(s >= 0) and s.max() > 0
