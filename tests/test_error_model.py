"""The reduced-precision error bars (helpers.BARS) against the rounding each
path makes: tests/error_model.py evaluates the FFT pipeline in FP64 with only
that path's roundings; every bar must lie between 1.5x (room for the FP32
arithmetic of the kernels) and 4x (not a loose bar) the modelled error on the
worst rupture of the tiny workload and of a compact-box case like those of
the GPU tests.  The model itself is pinned first: with no rounding it is the
oracle, and its rounding functions give the textbook values."""
import numpy as np
import pytest

import error_model as em
import oracle
import synth
from helpers import BARS

MODEL_PATH = {"stream_bf16": ["stream_bf16"], "stream_bf16_hilo": ["stream_bf16_hilo"],
              "stream_fp8": ["stream_fp8", "stream_fp8_bf16p"], "tensor_bf16": ["tensor_bf16"],
              "tensor_split": ["tensor_split"], "tensor_fp8": ["tensor_fp8", "tensor_fp8_hilo"]}


def cases():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    out = [(geom, wl.Nt, wl.slip(geom, B=3))]
    g = synth.geometry_box(24, 700, 6, 12)
    box = synth.Geometry(g.sub * 0.1, g.grid * 0.1, g.obs * 0.1, g.strike * 0.1, g.dip * 0.1, "box")
    s = np.random.default_rng(13).standard_normal((3, 24, 64))
    s[:, :, 32:] = 0
    out.append((box, 64, s))
    return out


@pytest.fixture(scope="module")
def prepared():
    res = []
    for geom, Nt, slip in cases():
        G = geom.greens_rows(0, geom.Ng, Nt, np.float32).astype(np.float64)
        P = geom.adjoint_cols(0, geom.Ng, Nt, np.float32).astype(np.float64)
        s = slip.astype(np.float32).astype(np.float64)
        qw = oracle.fft_window(G, P, s)
        res.append((G, P, s, qw[..., :Nt], np.linalg.norm(qw.reshape(qw.shape[0], -1), axis=1)))
    return res


def test_rounding_functions():
    # BF16: 8 significant bits, ties to even
    assert em.bf16(1.0 + 2.0 ** -8) == 1.0
    assert em.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert em.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    # e4m3: 448 is the largest finite value (saturation), 2^-9 the smallest subnormal
    assert em.e4m3(np.array([500.0, 448.0, 2.0 ** -9, 2.0 ** -10, 1.0625, 1.1875]))[0] == 448.0
    v = em.e4m3(np.array([448.0, 2.0 ** -9, 2.0 ** -10 + 2.0 ** -12, 1.0625, 1.1875, -13.5]))
    assert list(v) == [448.0, 2.0 ** -9, 2.0 ** -9, 1.0, 1.25, -14.0]


def test_retransform_matrix_of_the_model():
    """The model's retransform matrix maps the bins of m to those of D_t of
    its truncation, built from the oracle's DFT and D_t."""
    Nt = 32
    T = em.retransform_matrix(Nt)
    u = np.random.default_rng(1).standard_normal((4, 2 * Nt))
    m = np.fft.irfft(em.to_bins(u, Nt), n=2 * Nt)[:, :Nt]
    want = em.to_dofs(oracle.dft_real(oracle.dt_apply(m), 2 * Nt), Nt)
    assert np.max(np.abs(u @ T.T - want)) <= 1e-12 * np.max(np.abs(want))


def test_model_without_rounding_is_the_oracle(prepared):
    for G, P, s, q_ref, _ in prepared:
        q = em.model_waveforms(G, P, s, "exact")
        assert np.max(np.abs(q - q_ref)) <= 1e-10 * np.max(np.abs(q_ref))


@pytest.mark.parametrize("bar", sorted(BARS))
def test_bar_is_derived_from_the_path_rounding(prepared, bar):
    worst = 0.0
    for G, P, s, q_ref, wn in prepared:
        for path in MODEL_PATH[bar]:
            q = em.model_waveforms(G, P, s, path)
            e = np.linalg.norm((q - q_ref).reshape(q.shape[0], -1), axis=1) / wn
            worst = max(worst, float(e.max()))
    print(f"{bar}: modelled worst error / window {worst:.3g}, bar {BARS[bar]:.3g} ({BARS[bar] / worst:.2f}x)")
    assert 1.5 * worst <= BARS[bar] <= 4.0 * worst


def test_full_size_model_is_the_oracle():
    """The model without rounding, run over the full batched workload's grid
    in chunks (tests/golden/make_full_size_model.py, operator spectra by an
    FP64 DFT matrix), gives the FP64 oracle's stored waveforms of the same
    ruptures: the full-size bars come from a model of the same map."""
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    m = np.load(os.path.join(here, "model_batched.npz"))
    o = np.load(os.path.join(here, "oracle_batched.npz"))
    assert np.array_equal(m["index"], o["index"]) and np.array_equal(m["draw"], o["draw"])
    assert np.allclose(m["checksum"], o["checksum"], rtol=1e-12, atol=0.0)
    n = len(m["index"])
    rel = np.linalg.norm((m["q_exact"] - o["q"]).reshape(n, -1), axis=1) / np.linalg.norm(o["q"].reshape(n, -1), axis=1)
    assert rel.max() <= 1e-12, rel
    for k in ("rel_tensor_bf16", "rel_tensor_split"):
        assert m[k].shape == (n,) and np.all(m[k] > 0)
