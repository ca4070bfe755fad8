"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Bars per rupture (tests/helpers.assert_parity):
  FP32 class (FP32 pairs, and FP32 storage on inputs whose kept head is not
  dwarfed by the rest of the FFT window): the plain relative L2 error over the
  No x Nt samples <= 1e-5, every rupture.
  Reduced precision: ||q - q_ref|| <= TOL * ||q_win||, with q_win the 2
  Nt-sample window that Alg. 2 computes before Truncate (oracle.fft_window),
  the scale on which a finite-precision FFT evaluation errs:
        BF16 hi/lo storage  2e-5  (hi + lo keeps ~17 bits: <= 2^-18 per entry)
        BF16 storage        5e-3  (8 significant bits: <= 2^-9 per entry)
        FP8 e4m3 storage    1e-1  (4 significant bits: <= 2^-4 per entry)
  (helpers.BARS; tests/test_error_model.py derives each from the rounding the
  path makes.)  FP32 storage errs by up to ~1e-5 of that window too: on the tiny
  workload, whose rupture 0 keeps 1/393 of its window's norm in the kept head,
  that is 1.2e-4 of the head; the FP32 pair storage (fp32_hilo) takes the same
  rupture to ~1e-9.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BARS, assert_parity, make_context, oracle_reference, rel_l2, window_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402

TOL = {"fp32": 1e-5, "fp32_hilo": 1e-5, "bf16_hilo": BARS["stream_bf16_hilo"], "bf16": BARS["stream_bf16"],
       "fp8": BARS["stream_fp8"]}


@pytest.fixture(scope="module")
def tiny():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=3)
    q_ref, m_ref = oracle_reference(geom, wl.Nt, slip, seafloor=True)
    return wl, geom, slip, q_ref, m_ref


@pytest.fixture(scope="module")
def tiny_window(tiny):
    wl, geom, slip, _, _ = tiny
    G = geom.greens_rows(0, geom.Ng, wl.Nt)
    P = geom.adjoint_cols(0, geom.Ng, wl.Nt)
    return window_norms(G, P, slip)


def compact_box(Ns, Ng, No, seed, scale=0.1):
    """geometry_box shrunk by `scale` (a 20 x 10 km box for 0.1), so that the
    responses arrive inside short records."""
    g = synth.geometry_box(Ns, Ng, No, seed)
    return synth.Geometry(g.sub * scale, g.grid * scale, g.obs * scale,
                          g.strike * scale, g.dip * scale, "box")


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("Nt", [32, 64, 128, 256, 512])
def test_rfft_matches_oracle_dft(Nt):
    ctx = s2w.Context(4, 8, 2, Nt)
    x = np.random.default_rng(Nt).standard_normal((37, Nt))
    X = ctx.rfft(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = oracle.dft_real(x.astype(np.float32), 2 * Nt)
    assert rel_l2(X.real, ref.real) < 1e-6 and rel_l2(X.imag, ref.imag) < 1e-6


@pytest.mark.parametrize("Nt", [32, 256, 512])
def test_irfft_truncates_and_inverts(Nt):
    ctx = s2w.Context(4, 8, 2, Nt)
    rng = np.random.default_rng(Nt + 1)
    X = rng.standard_normal((19, Nt + 1)) + 1j * rng.standard_normal((19, Nt + 1))
    X[:, 0] = X[:, 0].real
    X[:, -1] = X[:, -1].real
    x = ctx.irfft(torch.tensor(X, dtype=torch.complex64, device="cuda")).cpu().numpy()
    ref = np.fft.irfft(X, n=2 * Nt)[:, :Nt]
    assert x.shape == (19, Nt)
    assert rel_l2(x, ref) < 1e-6
    # round trip on a signal supported on [0, Nt)
    s = rng.standard_normal((5, Nt))
    st = torch.tensor(s, dtype=torch.float32, device="cuda")
    back = ctx.irfft(ctx.rfft(st)).cpu().numpy()
    assert rel_l2(back, s) < 1e-6


# ---------------------------------------------------------------- end to end
@pytest.mark.parametrize("prec", ["fp32_hilo", "bf16_hilo", "bf16", "fp8"])
def test_tiny_workload_against_oracle(tiny, tiny_window, prec):
    wl, geom, slip, q_ref, _ = tiny
    # stream engine: these bars are for the storage precisions alone
    prec_p = "fp32_hilo" if prec == "fp32_hilo" else "fp32"
    ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, prec_p=prec_p, max_batch=3, chunk=256, engine="stream")
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_parity(q, q_ref, *tiny_window, tol=TOL[prec], label=f"tiny {prec}")
    ctx.sync()


def test_fp32_storage_errs_on_the_window_scale(tiny, tiny_window):
    """FP32 (complex64) spectra on the tiny workload: every rupture within
    1e-5 of its FFT window's norm, which for rupture 0 (kept head 1/393 of
    the window) is not 1e-5 of the head; the FP32 pairs meet 1e-5 of the head
    there with room to spare (the config's FP32 path)."""
    wl, geom, slip, q_ref, _ = tiny
    wn, kappa = tiny_window
    out = {}
    for prec in ("fp32", "fp32_hilo"):
        ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, prec_p=prec, max_batch=3, engine="stream")
        out[prec] = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
        ctx.sync()
    err = {k: np.linalg.norm((v - q_ref).reshape(3, -1), axis=1) for k, v in out.items()}
    head = np.linalg.norm(q_ref.reshape(3, -1), axis=1)
    print("fp32: rel", err["fp32"] / head, "window", err["fp32"] / wn, "kappa", kappa)
    print("fp32_hilo: rel", err["fp32_hilo"] / head)
    assert np.all(err["fp32"] <= 1e-5 * wn)
    assert np.all(err["fp32_hilo"] <= 1e-5 * head)
    assert err["fp32_hilo"][0] * 100 <= err["fp32"][0]


@pytest.mark.parametrize("prec", ["fp32", "fp32_hilo"])
def test_seafloor_field_against_oracle(tiny, prec):
    wl, geom, slip, q_ref, m_ref = tiny
    ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, prec_p=prec, max_batch=3)
    s = torch.tensor(slip, dtype=torch.float32, device="cuda")
    sf = torch.empty((3, geom.Ng, wl.Nt), dtype=torch.float32, device="cuda")
    q = ctx.waveforms(s, seafloor=sf).cpu().numpy()
    assert np.all(rel_l2(sf.cpu().numpy(), m_ref) <= 1e-5)
    if prec == "fp32_hilo":  # the seafloor output does not change the waveforms
        assert np.all(rel_l2(q, q_ref) <= 1e-5)
        assert np.array_equal(q, ctx.waveforms(s).cpu().numpy())


def test_bf16_p_storage(tiny, tiny_window):
    wl, geom, slip, q_ref, _ = tiny
    ctx = make_context(s2w, geom, wl.Nt, prec_p="bf16", max_batch=3, engine="stream")
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_parity(q, q_ref, *tiny_window, tol=TOL["bf16"], label="tiny P bf16")


def test_impulse_returns_green_column_and_composed_response(tiny):
    """An impulse on subfault j returns column j of the Green's function as the
    seafloor field, and (P * G)[:, j] as the waveforms when D_t is off."""
    wl, geom, _, _, _ = tiny
    j = 5
    s = np.zeros((1, geom.Ns, wl.Nt))
    s[0, j, 0] = 1.0
    ctx = make_context(s2w, geom, wl.Nt, dt_mode="none")
    sf = torch.empty((1, geom.Ng, wl.Nt), dtype=torch.float32, device="cuda")
    q = ctx.waveforms(torch.tensor(s, dtype=torch.float32, device="cuda"), seafloor=sf).cpu().numpy()
    G = geom.greens_rows(0, geom.Ng, wl.Nt)
    P = geom.adjoint_cols(0, geom.Ng, wl.Nt)
    assert rel_l2(sf.cpu().numpy()[0], G[:, j, :]) < 1e-5
    q_ref = oracle.bltt_apply(P, G[:, j, :])
    assert rel_l2(q[0], q_ref) < 1e-5


def test_linearity_and_causality(tiny):
    wl, geom, slip, _, _ = tiny
    ctx = make_context(s2w, geom, wl.Nt)
    dev = lambda a: torch.tensor(a[None], dtype=torch.float32, device="cuda")
    s1, s2 = slip[0], slip[1]
    q1 = ctx.waveforms(dev(s1)).cpu().numpy()[0].astype(np.float64)
    q2 = ctx.waveforms(dev(s2)).cpu().numpy()[0].astype(np.float64)
    q12 = ctx.waveforms(dev(2.0 * s1 - 0.5 * s2)).cpu().numpy()[0]
    assert rel_l2(q12, 2.0 * q1 - 0.5 * q2) < 1e-5
    n0 = 12
    s3 = s1.copy()
    s3[:, n0:] += np.random.default_rng(3).standard_normal(s3[:, n0:].shape)
    q3 = ctx.waveforms(dev(s3)).cpu().numpy()[0]
    d = q3 - q1
    assert np.linalg.norm(d[:, :n0]) <= 1e-5 * np.linalg.norm(d)


def test_time_shift(tiny, tiny_window):
    wl, geom, slip, _, _ = tiny
    ctx = make_context(s2w, geom, wl.Nt)
    tau = 4
    s = slip[1]
    sh = np.zeros_like(s)
    sh[:, tau:] = s[:, :-tau]
    dev = lambda a: torch.tensor(a[None], dtype=torch.float32, device="cuda")
    q = ctx.waveforms(dev(s)).cpu().numpy()[0]
    qs = ctx.waveforms(dev(sh)).cpu().numpy()[0]
    wn = tiny_window[0][1]
    assert np.linalg.norm(qs[:, tau:] - q[:, :-tau]) <= 2e-5 * wn
    assert np.linalg.norm(qs[:, :tau]) <= 1e-5 * wn


def test_host_device_batch_and_chunking_agree_bitwise(tiny):
    wl, geom, slip, _, _ = tiny
    ctx = make_context(s2w, geom, wl.Nt, max_batch=3, chunk=1024)
    ctx2 = make_context(s2w, geom, wl.Nt, max_batch=3, chunk=96, order=list(range(10, -1, -1)))
    s32 = slip.astype(np.float32)
    q_host = ctx.waveforms(s32)                                        # numpy: host path
    q_dev = ctx.waveforms(torch.tensor(s32, device="cuda")).cpu().numpy()
    q_ch = ctx2.waveforms(torch.tensor(s32, device="cuda")).cpu().numpy()
    q_one = np.stack([ctx.waveforms(s32[b:b + 1])[0] for b in range(3)])
    assert np.array_equal(q_host, q_dev)
    assert np.array_equal(q_dev, q_ch)
    assert np.array_equal(q_dev, q_one)


def test_stream_groups_of_ruptures():
    """The stream engine handles a call's ruptures in groups of 64; a
    70-rupture call equals the same ruptures one by one, bit for bit."""
    geom = compact_box(6, 500, 3, seed=70)
    Nt, B = 32, 70
    slip = np.random.default_rng(70).standard_normal((B, 6, Nt)).astype(np.float32)
    ctx = make_context(s2w, geom, Nt, max_batch=B)
    st = torch.tensor(slip, device="cuda")
    q = ctx.waveforms(st).cpu().numpy()
    q1 = np.stack([ctx.waveforms(st[b:b + 1]).cpu().numpy()[0] for b in (0, 63, 64, 69)])
    assert np.array_equal(q[[0, 63, 64, 69]], q1)
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    assert_parity(q, oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=1e-5, label="stream groups")


@pytest.mark.parametrize("prec", ["fp32", "fp32_hilo"])
@pytest.mark.parametrize("Ns,Ng,No,Nt", [(5, 1000, 3, 64), (1, 37, 1, 32), (1024, 300, 2, 32),
                                         (7, 2100, 5, 128)])
def test_ragged_shapes(Ns, Ng, No, Nt, prec):
    geom = compact_box(Ns, Ng, No, seed=Ns + Ng)
    slip = np.random.default_rng(1).standard_normal((2, Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    ctx = make_context(s2w, geom, Nt, prec_g=prec, prec_p=prec, max_batch=2, chunk=512)
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    assert_parity(q, q_ref, *window_norms(G, P, slip), tol=1e-5, label=f"ragged {Ns}x{Ng}x{No}x{Nt}")


def test_errors_and_empty_batch(tiny):
    wl, geom, slip, _, _ = tiny
    ctx = s2w.Context(geom.Ns, geom.Ng, geom.No, wl.Nt, max_batch=2)
    s = torch.tensor(slip[:1], dtype=torch.float32, device="cuda")
    with pytest.raises(s2w.S2WError) as e:
        ctx.waveforms(s)
    assert e.value.status == -3          # operators not loaded
    ctx.load_greens(0, geom.greens_rows(0, geom.Ng, wl.Nt, np.float32))
    with pytest.raises(s2w.S2WError):
        ctx.waveforms(s)                 # adjoint still missing
    ctx.load_adjoint(0, geom.adjoint_cols(0, geom.Ng, wl.Nt, np.float32))
    ctx.waveforms(s)
    q = torch.empty((0, geom.No, wl.Nt), device="cuda")
    ctx.waveforms(torch.empty((0, geom.Ns, wl.Nt), device="cuda"), q=q)   # B = 0
    with pytest.raises(s2w.S2WError) as e:
        ctx.waveforms(torch.zeros((3, geom.Ns, wl.Nt), device="cuda"))
    assert e.value.status == -1          # B > max_batch
    with pytest.raises(s2w.S2WError):
        ctx.load_greens(geom.Ng - 2, geom.greens_rows(0, 4, wl.Nt, np.float32))
    fp8 = s2w.Context(geom.Ns, geom.Ng, geom.No, wl.Nt, prec_g="fp8")
    with pytest.raises(s2w.S2WError):
        fp8.load_greens(100, geom.greens_rows(100, 356, wl.Nt, np.float32))  # unaligned
    ctx.sync()


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def plain_reference():
    """Paper-shaped plain workload (963 subfaults, 20,000 grid points, 64
    observations, 256 steps), one rupture: the FP64 oracle over grid chunks
    (Eq. distributed-composition), plus the norm of its 2 Nt-sample window."""
    wl = synth.WORKLOADS["plain"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=1)
    q_ref, q_win = None, None
    for g0 in range(0, wl.Ng, 1024):
        g1 = min(wl.Ng, g0 + 1024)
        G = geom.greens_rows(g0, g1, wl.Nt)
        P = geom.adjoint_cols(g0, g1, wl.Nt)
        w = oracle.fft_window(G, P, slip)
        q_win = w if q_win is None else q_win + w
    q_ref = q_win[..., :wl.Nt]
    wn = np.linalg.norm(q_win.reshape(1, -1), axis=1)
    kappa = wn / np.linalg.norm(q_ref.reshape(1, -1), axis=1)
    return wl, geom, slip, q_ref, wn, kappa


@pytest.mark.parametrize("prec_g,prec_p", [("fp32", "fp32"), ("fp32_hilo", "fp32_hilo"), ("bf16_hilo", "fp32"),
                                           ("bf16", "bf16"), ("fp8", "bf16")])
def test_plain_workload_full_size(plain_reference, prec_g, prec_p):
    """The whole waveform set of the plain workload against the FP64 oracle,
    in every storage precision, at the size and launch configuration that
    bench.py times (one rupture per call)."""
    wl, geom, slip, q_ref, wn, kappa = plain_reference
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt, prec_g=prec_g, prec_p=prec_p)
    for g0 in range(0, wl.Ng, 4096):
        g1 = min(wl.Ng, g0 + 4096)
        ctx.load_greens(g0, geom.greens_rows(g0, g1, wl.Nt, np.float32))
        ctx.load_adjoint(g0, geom.adjoint_cols(g0, g1, wl.Nt, np.float32))
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    tol = max(TOL[prec_g], TOL[prec_p])
    assert_parity(q, q_ref, wn, kappa, tol=tol, label=f"plain {prec_g}/{prec_p}")
    ctx.sync()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_spectra_loaders_match_time_domain_loaders(prec):
    """s2w_load_greens_spectra / s2w_load_adjoint_spectra with spectra formed
    by numpy (FP64 zero-padded rfft, rounded to complex64): mixed with the
    time-domain loader over row chunks, host and device sources; waveforms
    meet the same bars and agree with a context loaded in the time domain."""
    Ns, Ng, No, Nt, B = 24, 700, 6, 64, 3
    geom = compact_box(Ns, Ng, No, seed=41)
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    Ghat = np.ascontiguousarray(np.fft.rfft(G, n=2 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    Phat = np.ascontiguousarray(np.fft.rfft(P, n=2 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    ctx = s2w.Context(Ns, Ng, No, Nt, prec_g=prec, max_batch=B, engine="stream")
    ctx.load_greens_spectra(0, np.ascontiguousarray(Ghat[:, :300]))
    ctx.load_greens(300, geom.greens_rows(300, Ng, Nt, np.float32))
    ctx.load_adjoint_spectra(0, torch.tensor(Phat[:, :, :512], device="cuda"))
    ctx.load_adjoint(512, np.ascontiguousarray(geom.adjoint_cols(512, Ng, Nt, np.float32)))
    rng = np.random.default_rng(42)
    slip = rng.standard_normal((B, Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    q_ref = oracle.waveforms(G, P, slip)
    tol = {"fp32": 1e-5, "bf16": BARS["stream_bf16"]}[prec]
    assert_parity(q, q_ref, *window_norms(G, P, slip), tol=tol, label=f"spectra loaders {prec}")
    ct = make_context(s2w, geom, Nt, prec_g=prec, max_batch=B, engine="stream")
    qt = ct.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    wn, _ = window_norms(G, P, slip)
    assert np.all(np.linalg.norm((q - qt).reshape(B, -1), axis=1) <= 2 * tol * wn)


def test_spectra_loaders_feed_the_tensor_adjoint():
    """Spectra loaded directly also build the transposed copies of the
    tensor-engine adjoint (split precision)."""
    Ns, Ng, No, Nt, B = 16, 900, 5, 32, 4
    geom = compact_box(Ns, Ng, No, seed=43)
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    Ghat = np.ascontiguousarray(np.fft.rfft(G, n=2 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    Phat = np.ascontiguousarray(np.fft.rfft(P, n=2 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    ctx = s2w.Context(Ns, Ng, No, Nt, prec_g="bf16_hilo", max_batch=B, engine="tensor", tc_adjoint=True)
    ctx.load_greens_spectra(0, Ghat)
    ctx.load_adjoint_spectra(0, Phat)
    r = np.random.default_rng(44).standard_normal((B, No, Nt))
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    gw = oracle.fft_window_adjoint(G, P, r)
    err = np.linalg.norm((g - gw[..., Nt:]).reshape(B, -1), axis=1)
    assert np.all(err <= 3e-5 * np.linalg.norm(gw.reshape(B, -1), axis=1)), err


@pytest.mark.parametrize("engine,prec", [("stream", "fp32"), ("tensor", "bf16"), ("tensor", "bf16_hilo")])
def test_active_lengths_match_zero_filled_tails(engine, prec):
    """s2w_waveforms_active: samples past each rupture's active length are
    never read (they hold NaN here) and the result equals s2w_waveforms on
    zero-filled tails, bit for bit; lengths 0 and Nt included."""
    Ns, Ng, No, Nt = 24, 700, 6, 64
    lens = [0, 1, 17, 32, 63, 64]
    B = len(lens)
    geom = compact_box(Ns, Ng, No, seed=51)
    rng = np.random.default_rng(52)
    slip = rng.standard_normal((B, Ns, Nt)).astype(np.float32)
    zeroed, garbage = slip.copy(), slip.copy()
    for b, n in enumerate(lens):
        zeroed[b, :, n:] = 0
        garbage[b, :, n:] = np.nan
    ctx = make_context(s2w, geom, Nt, prec_g=prec, max_batch=B, engine=engine)
    q0 = ctx.waveforms(torch.tensor(zeroed, device="cuda")).cpu().numpy()
    q1 = ctx.waveforms_active(torch.tensor(garbage, device="cuda"), lens).cpu().numpy()
    assert np.array_equal(q0, q1)
    assert np.all(q0[0] == 0)
    q2 = ctx.waveforms_active(garbage, lens)  # host path
    assert np.array_equal(q0, q2)
    with pytest.raises(s2w.S2WError):
        ctx.waveforms_active(torch.tensor(zeroed, device="cuda"), [Nt + 1] + lens[1:])
    ctx.sync()


@pytest.mark.parametrize("prec,tol,dt_mode", [("fp32", 1e-5, "backward"), ("bf16_hilo", BARS["stream_bf16_hilo"], "backward"),
                                              ("fp32", 1e-5, "none")])
def test_single_pass_variant(prec, tol, dt_mode):
    """The single-pass ablation (L = 4 Nt, D_t folded into Phat, no
    retransform) meets the same bar as the two-pass path and agrees with it;
    its operators take (2 Nt + 1) / (Nt + 1) times the bytes."""
    Ns, Ng, No, Nt, B = 24, 700, 6, 64, 3
    geom = compact_box(Ns, Ng, No, seed=71)
    rng = np.random.default_rng(72)
    slip = rng.standard_normal((B, Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    c1 = make_context(s2w, geom, Nt, prec_g=prec, dt_mode=dt_mode, max_batch=B, engine="stream",
                      single_pass=True, chunk=256)
    c2 = make_context(s2w, geom, Nt, prec_g=prec, dt_mode=dt_mode, max_batch=B, engine="stream")
    q1 = c1.waveforms(st).cpu().numpy()
    q2 = c2.waveforms(st).cpu().numpy()
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip, dt_mode=dt_mode)
    wn, kappa = window_norms(G, P, slip, dt_mode)
    assert_parity(q1, q_ref, wn, kappa, tol=tol, label=f"single pass {prec} {dt_mode}")
    assert np.all(np.linalg.norm((q1 - q2).reshape(B, -1), axis=1) <= 2 * tol * wn)
    g1, _ = c1.operator_bytes()
    g2, _ = c2.operator_bytes()
    assert g1 * (Nt + 1) == g2 * (2 * Nt + 1)
    with pytest.raises(s2w.S2WError):
        c1.waveforms(st, seafloor=torch.empty((B, Ng, Nt), device="cuda"))
    with pytest.raises(s2w.S2WError):
        c1.adjoint(torch.zeros((B, No, Nt), device="cuda"))
    c1.sync()


def test_single_pass_spectral_loads():
    """Spectra of length 4 Nt handed to the single-pass variant directly."""
    Ns, Ng, No, Nt, B = 16, 500, 4, 32, 2
    geom = compact_box(Ns, Ng, No, seed=73)
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    Ghat = np.ascontiguousarray(np.fft.rfft(G, n=4 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    Phat = np.ascontiguousarray(np.fft.rfft(P, n=4 * Nt, axis=2).transpose(2, 0, 1)).astype(np.complex64)
    ctx = s2w.Context(Ns, Ng, No, Nt, max_batch=B, engine="stream", single_pass=True)
    ctx.load_greens_spectra(0, Ghat)
    ctx.load_adjoint_spectra(0, Phat)
    slip = np.random.default_rng(74).standard_normal((B, Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    assert_parity(q, oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=1e-5, label="single pass spectra")


@pytest.mark.parametrize("prec", ["fp32", "fp32_hilo"])
@pytest.mark.parametrize("Ns,Ng,No,Nt,B", [(96, 3000, 8, 256, 3), (60, 1500, 4, 128, 2), (33, 777, 5, 64, 2)])
def test_paper_geometry_full_length_slip(prec, Ns, Ng, No, Nt, B):
    """Ragged shapes on the paper-shaped geometry (subfaults on the dipping
    1000 x 100 km plane, grid and observations over its surface projection)
    with full-length von Karman ruptures (no zeroed tail, no shrunken box):
    every rupture within 1e-5 of the oracle in plain relative L2."""
    geom = synth.geometry_plane(Ns, Ng, No, seed=Ns + Nt)
    slip = synth.slip_von_karman(geom, B, Nt, seed=Ng, mw_range=(8.0, 9.0))
    ctx = make_context(s2w, geom, Nt, prec_g=prec, prec_p=prec, max_batch=B, chunk=1024)
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    assert_parity(q, oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=1e-5,
                  label=f"plane {prec} {Ns}x{Ng}x{No}x{Nt}")


def test_fp32_pairs_reject_what_they_do_not_support():
    geom = compact_box(8, 200, 2, seed=3)
    with pytest.raises(s2w.S2WError):   # both operators or neither
        s2w.Context(8, 200, 2, 32, prec_g="fp32_hilo", prec_p="fp32")
    with pytest.raises(s2w.S2WError):
        s2w.Context(8, 200, 2, 32, prec_g="fp32_hilo", prec_p="fp32_hilo", engine="tensor")
    ctx = make_context(s2w, geom, 32, prec_g="fp32_hilo", prec_p="fp32_hilo", max_batch=2)
    with pytest.raises(s2w.S2WError) as e:
        ctx.adjoint(torch.zeros((1, 2, 32), device="cuda"))
    assert e.value.status == -6
    g, p = ctx.operator_bytes()
    c32 = make_context(s2w, geom, 32, max_batch=2)
    g32, p32 = c32.operator_bytes()
    assert (g, p) == (2 * g32, 2 * p32)
    ctx.sync()
