"""Tensor-core engine (tcgen05, BF16 operands, FP32 accumulation) against the
FP64 oracle, through the C ABI.

Bar: ||q - q_ref|| <= TOL_TC * ||q_win|| per rupture (q_win: the 2 Nt-sample
FFT window, oracle.fft_window).  The engine rounds the operator spectra AND
the activations (slip and velocity spectra) to BF16 (8 significant bits,
<= 2^-9 relative per entry), so its bar is twice the BF16-storage bar.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BARS, assert_parity, make_context, window_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402

# bars derived from the roundings of each path (helpers.BARS,
# tests/test_error_model.py): BF16 operands and activations; the hi/lo split
# of every operand (three MMAs per K step); FP8 operator with FP16 activations
TOL_TC = BARS["tensor_bf16"]
TOL_SPLIT = BARS["tensor_split"]
TOL_F8 = BARS["tensor_fp8"]


def compact_box(Ns, Ng, No, seed, scale=0.1):
    g = synth.geometry_box(Ns, Ng, No, seed)
    return synth.Geometry(g.sub * scale, g.grid * scale, g.obs * scale,
                          g.strike * scale, g.dip * scale, "box")


def run_case(geom, Nt, B, seed=5, engine="tensor", chunk=4096, prec="bf16", tc_pair="auto", tc_bsub=0,
             tc_s2_chunks=0):
    rng = np.random.default_rng(seed)
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    ctx = make_context(s2w, geom, Nt, prec_g=prec, max_batch=B, chunk=chunk, engine=engine,
                       tc_pair=tc_pair, tc_bsub=tc_bsub, tc_s2_chunks=tc_s2_chunks)
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    return q, q_ref, window_norms(G, P, slip), ctx, slip


def test_tiny_workload_tensor_engine():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=3)
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt, prec_g="bf16", max_batch=3, engine="tensor")
    ctx.load_greens(0, geom.greens_rows(0, wl.Ng, wl.Nt, np.float32))
    ctx.load_adjoint(0, geom.adjoint_cols(0, wl.Ng, wl.Nt, np.float32))
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    assert_parity(q, oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=TOL_TC, label="tiny tensor")


@pytest.mark.parametrize("B", [1, 7])
def test_small_batches_tensor_engine(B):
    geom = compact_box(24, 700, 6, seed=3)
    q, q_ref, wn, _, _ = run_case(geom, 64, B)
    assert_parity(q, q_ref, *wn, tol=TOL_TC, label=f"tensor B={B}")


def test_full_width_batch_and_sub_batches():
    """B = 300: one sub-batch of 256 ruptures (N = 512, two MMAs per K step)
    and one of 44 (N = 96); 700 grid rows = 5 full M tiles + 60."""
    geom = compact_box(24, 700, 6, seed=4)
    q, q_ref, wn, ctx, slip = run_case(geom, 64, 300)
    assert_parity(q, q_ref, *wn, tol=TOL_TC, label="tensor B=300")
    # deterministic: same inputs, same bits
    q2 = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.array_equal(q, q2)
    # host buffers: the sub-batches' copies overlap the other sub-batches'
    # GEMMs on an internal stream; same kernels, same bits
    s32 = np.ascontiguousarray(slip, dtype=np.float32)
    assert np.array_equal(q, ctx.waveforms(s32))
    # ... with per-rupture active lengths (each sub-batch gets its own)
    lens = np.random.default_rng(41).integers(1, 65, size=300)
    cut = s32.copy()
    for b, n in enumerate(lens):
        cut[b, :, n:] = 0
    want = ctx.waveforms(torch.tensor(cut, device="cuda")).cpu().numpy()
    junk = cut.copy()
    for b, n in enumerate(lens):
        junk[b, :, n:] = 1e30  # never read
    assert np.array_equal(want, ctx.waveforms_active(junk, lens))
    ctx.sync()


def test_split_k_over_grid_chunks():
    """5,000 grid points: the stage-2 reduction dimension (2 x 5,000) spans
    three 4,096-element chunks whose partials are summed in fixed order."""
    geom = compact_box(16, 5000, 4, seed=6)
    q, q_ref, wn, _, _ = run_case(geom, 32, 20, chunk=2048)
    assert_parity(q, q_ref, *wn, tol=TOL_TC, label="tensor split-K")


def test_auto_engine_uses_tensor_path_for_batches_only():
    """AUTO: one rupture goes through the streaming kernels (activations kept
    FP32), a batch through the tensor engine; both meet their bars."""
    geom = compact_box(24, 700, 6, seed=7)
    Nt, B = 64, 5
    rng = np.random.default_rng(9)
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    ctx = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B)
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    ctx.profile_enable(True)
    q_batch = ctx.waveforms(st).cpu().numpy()
    q_one = ctx.waveforms(st[:1]).cpu().numpy()
    stages, _ = ctx.profile_read()
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    wn, kappa = window_norms(G, P, slip)
    assert_parity(q_batch, q_ref, wn, kappa, tol=TOL_TC, label="auto batch")
    assert_parity(q_one, q_ref[:1], wn[:1], kappa[:1], tol=5e-3, label="auto single")
    assert stages["contract_stage1"][1] == 2  # one tensor pass + one streaming pass


def test_tensor_engine_with_seafloor_output():
    """A call that asks for the seafloor field runs on the stream kernels
    (the tensor engine never materialises m); both calls meet the
    tensor-engine bar and the seafloor field matches the oracle's m."""
    geom = compact_box(24, 700, 6, seed=8)
    Nt, B = 64, 6
    rng = np.random.default_rng(10)
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    ctx = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B, engine="tensor")
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    sf = torch.empty((B, geom.Ng, Nt), dtype=torch.float32, device="cuda")
    q_sf = ctx.waveforms(st, seafloor=sf).cpu().numpy()
    q = ctx.waveforms(st).cpu().numpy()
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref, m_ref = oracle.waveforms(G, P, slip, return_seafloor=True)
    wn, kappa = window_norms(G, P, slip)
    assert_parity(q, q_ref, wn, kappa, tol=TOL_TC, label="tensor, GEMM retransform")
    assert_parity(q_sf, q_ref, wn, kappa, tol=TOL_TC, label="tensor ctx, stream call with seafloor")
    m = sf.cpu().numpy()
    err = np.linalg.norm((m - m_ref).reshape(B, -1), axis=1) / np.linalg.norm(m_ref.reshape(B, -1), axis=1)
    assert np.all(err <= TOL_TC), err


@pytest.mark.parametrize("Nt", [32, 128, 256])
def test_gemm_retransform_record_lengths(Nt):
    geom = compact_box(12, 300, 3, seed=Nt)
    q, q_ref, wn, _, _ = run_case(geom, Nt, 4)
    assert_parity(q, q_ref, *wn, tol=TOL_TC, label=f"tensor Nt={Nt}")


@pytest.mark.parametrize("prec", ["bf16", "bf16_hilo"])
@pytest.mark.parametrize("knob", [{"tc_bsub": 128}, {"tc_s2_chunks": 1}, {"tc_s2_chunks": 3},
                                  {"tc_s2_chunks": 16}])
def test_schedule_knobs(prec, knob):
    """The schedule options the autotuner searches (ruptures per GEMM pass,
    stage-2 K chunks) change only the order of FP32 accumulation: each meets
    the bar and agrees with the default schedule within the reordering bound
    of an FP32 sum of K terms, K u (K = 2 x 704 stage-2 products per output,
    u = 2^-24).  700 grid rows = 5.5 M tiles, B = 300 (two sub-batches)."""
    if prec == "bf16_hilo" and "tc_bsub" in knob:
        pytest.skip("split passes take 128 ruptures anyway")
    geom = compact_box(24, 700, 6, seed=12)
    tol = TOL_SPLIT if prec == "bf16_hilo" else TOL_TC
    q1, q_ref, wn, _, _ = run_case(geom, 64, 300, seed=13, prec=prec)
    q2, _, _, _, _ = run_case(geom, 64, 300, seed=13, prec=prec, **knob)
    assert_parity(q2, q_ref, *wn, tol=tol, label=f"{prec} {knob}")
    d = np.linalg.norm((q2 - q1).ravel()) / np.linalg.norm(q1.ravel())
    assert d < 2 * 704 * 2.0 ** -24, d


@pytest.mark.parametrize("prec", ["bf16", "bf16_hilo"])
@pytest.mark.parametrize("Ng,B", [(700, 48), (600, 300), (5000, 150)])
def test_two_sm_pairs_match_single_cta(prec, Ng, B):
    """Two-SM MMAs (a CTA pair per 256-row tile, each CTA staging half of the
    B tile) against the oracle and against one CTA per 128-row tile: 700 grid
    rows = 3 pairs with a partial last tile, 600 = 5 tiles (the last pair's
    second tile empty); B = 48 (N = 96), 300 (sub-batches with N = 512 and 96,
    and a 256-row stage 2), 150 (a 150-row stage 2 over grid chunks)."""
    geom = compact_box(24, Ng, 6, seed=Ng + B)
    chunk = 2048 if Ng > 4096 else 4096
    tol = TOL_SPLIT if prec == "bf16_hilo" else TOL_TC
    q1, q_ref, wn, _, _ = run_case(geom, 64, B, seed=B, prec=prec, chunk=chunk, tc_pair="off")
    q2, _, _, ctx, slip = run_case(geom, 64, B, seed=B, prec=prec, chunk=chunk, tc_pair="on")
    assert_parity(q2, q_ref, *wn, tol=tol, label=f"pair {prec} Ng={Ng} B={B}")
    # the same products in the same K order: equal to rounding of the accumulation
    d = np.linalg.norm((q2 - q1).ravel()) / np.linalg.norm(q1.ravel())
    assert d < 1e-6, d
    q3 = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.array_equal(q2, q3)


@pytest.mark.parametrize("B", [1, 5, 130])
def test_split_precision_tensor_engine(B):
    """BF16 hi/lo operator spectra with hi/lo slip and velocity spectra on the
    tensor engine (the FFT retransform stays FP32); B = 130 runs sub-batches
    of 128 and 2."""
    geom = compact_box(24, 700, 6, seed=31)
    q, q_ref, wn, _, _ = run_case(geom, 64, B, seed=32, prec="bf16_hilo")
    rel, win = assert_parity(q, q_ref, *wn, tol=TOL_SPLIT, label=f"tensor split B={B}")


def test_split_precision_tiny_workload_and_stream_agreement():
    """Tiny workload: the split tensor engine and the hi/lo stream engine (FP32
    activations) both meet the hi/lo bar and agree with each other."""
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=4)
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    q_ref = oracle.waveforms(G, P, slip)
    wn = window_norms(G, P, slip)
    out = {}
    for engine in ("tensor", "stream"):
        ctx = make_context(s2w, geom, wl.Nt, prec_g="bf16_hilo", max_batch=4, engine=engine)
        out[engine] = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
        ctx.sync()
        assert_parity(out[engine], q_ref, *wn, tol=TOL_SPLIT, label=f"tiny hi/lo {engine}")


@pytest.mark.parametrize("Nt", [32, 256])
def test_split_precision_record_lengths(Nt):
    geom = compact_box(12, 300, 3, seed=Nt + 1)
    q, q_ref, wn, _, _ = run_case(geom, Nt, 6, prec="bf16_hilo")
    assert_parity(q, q_ref, *wn, tol=TOL_SPLIT, label=f"tensor split Nt={Nt}")


@pytest.mark.parametrize("B", [3, 7, 300])
def test_fp8_operator_on_tensor_engine(B):
    """FP8 e4m3 stage-1 spectra on the tensor engine with the default
    activations (hi + lo e4m3 parts on two-SM tiles; FP16 below two M tiles),
    per-(bin, 256-row) scales in the epilogue.  Against the oracle at the
    FP8 bar, and against the FP8 stream engine (same quantised operator; they
    differ by the rounding of the activations)."""
    geom = compact_box(24, 700, 6, seed=61)
    Nt = 64
    rng = np.random.default_rng(62)
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    wn, kappa = window_norms(G, P, slip)
    out = {}
    for engine in ("tensor", "stream"):
        ctx = make_context(s2w, geom, Nt, prec_g="fp8", max_batch=B, chunk=256, engine=engine)
        out[engine] = ctx.waveforms(st).cpu().numpy()
        ctx.sync()
        assert_parity(out[engine], q_ref, wn, kappa, tol=TOL_F8, label=f"fp8 {engine} B={B}")
    d = np.linalg.norm((out["tensor"] - out["stream"]).reshape(B, -1), axis=1)
    assert np.all(d <= TOL_TC * wn), d / wn


@pytest.mark.parametrize("Ng,B", [(700, 48), (600, 300)])
def test_fp8_two_sm_pairs_match_single_cta(Ng, B):
    """FP8 A on the two-SM form (each CTA widens its own 128 rows; both CTAs'
    converters release the pair's MMAs) against the oracle at the FP8 bar and
    against one CTA per 128-row tile (same FP8 products, FP32 accumulation):
    600 rows leave the last pair's second tile empty, B = 300 runs N = 512
    and N = 96 sub-batches."""
    geom = compact_box(24, Ng, 6, seed=Ng + B + 1)
    q1, q_ref, wn, _, _ = run_case(geom, 64, B, seed=B + 1, prec="fp8", chunk=256, tc_pair="off")
    q2, _, _, ctx, slip = run_case(geom, 64, B, seed=B + 1, prec="fp8", chunk=256, tc_pair="on")
    assert_parity(q2, q_ref, *wn, tol=TOL_F8, label=f"fp8 pair Ng={Ng} B={B}")
    d = np.linalg.norm((q2 - q1).ravel()) / np.linalg.norm(q1.ravel())
    assert d < 1e-6, d
    q3 = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.array_equal(q2, q3)


@pytest.mark.parametrize("Ng,B", [(700, 3), (700, 48), (600, 300)])
def test_fp8_activations_on_tensor_engine(Ng, B):
    """FP8 operator x FP8 activations (tc_fp8_act: slip spectra rounded to
    e4m3 with one power-of-two scale per (bin, rupture); kind::f8f6f4 MMAs on
    two-SM tiles): against the oracle at the FP8 bar, and against the
    FP16-activation FP8 path within the activation rounding, <= 2^-4 relative
    per entry, as a fraction of the window norm (measured up to ~4e-2: the
    products' rounding errors do not cancel like the products do); B = 3 and
    48 pad N to 32 and 96 columns, B = 300 runs an N = 512 and an N = 96
    sub-batch."""
    geom = compact_box(24, Ng, 6, seed=Ng + B + 7)
    rng = np.random.default_rng(B + 7)
    Nt = 64
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    wn, kappa = window_norms(G, P, slip)
    out = {}
    for act in (False, True):
        ctx = make_context(s2w, geom, Nt, prec_g="fp8", max_batch=B, chunk=256, engine="tensor", tc_fp8_act=act)
        out[act] = ctx.waveforms(st).cpu().numpy()
        ctx.sync()
        assert_parity(out[act], q_ref, wn, kappa, tol=TOL_F8, label=f"fp8 act={act} B={B}")
    d = np.linalg.norm((out[True] - out[False]).reshape(B, -1), axis=1)
    assert np.all(d <= 2.0 ** -4 * wn), d / wn
    # deterministic
    q2 = ctx.waveforms(st).cpu().numpy()
    assert np.array_equal(out[True], q2)


@pytest.mark.parametrize("Ng,B", [(700, 3), (600, 300), (5000, 256), (700, 150)])
def test_fp8_hilo_activations_match_fp16_activations(Ng, B):
    """FP8 operator x FP8 activations as hi + lo e4m3 parts (tc_fp8_act = 2:
    two kind::f8f6f4 MMAs per K step on two-SM tiles; 64-byte swizzle up to
    N = 256, and at N = 512 (B = 256, the first sub-batch of B = 300, and
    B = 150, whose second column half holds 22 live ruptures) two 256-column
    units per tile with alternating accumulators): at
    the FP8 bar against the oracle, and within 2^-7 of the window norm of the
    FP16-activation path (the hi + lo pair keeps ~2^-8 of each entry, FP16
    2^-11; the operator's own e4m3 rounding is common to both)."""
    geom = compact_box(24, Ng, 6, seed=Ng + B + 9)
    rng = np.random.default_rng(B + 9)
    Nt = 64
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    st = torch.tensor(slip, dtype=torch.float32, device="cuda")
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q_ref = oracle.waveforms(G, P, slip)
    wn, kappa = window_norms(G, P, slip)
    out = {}
    for act in (0, 2):
        ctx = make_context(s2w, geom, Nt, prec_g="fp8", max_batch=B, chunk=256, engine="tensor", tc_fp8_act=act)
        out[act] = ctx.waveforms(st).cpu().numpy()
        ctx.sync()
        assert_parity(out[act], q_ref, wn, kappa, tol=TOL_F8, label=f"fp8 act={act} B={B}")
    d = np.linalg.norm((out[2] - out[0]).reshape(B, -1), axis=1)
    print("hi/lo vs FP16 activations, / window:", d / wn)
    assert np.all(d <= 2.0 ** -7 * wn), d / wn
    q2 = ctx.waveforms(st).cpu().numpy()
    assert np.array_equal(out[2], q2)


def test_fp8_activations_reject_other_precisions():
    geom = compact_box(8, 300, 2, seed=5)
    with pytest.raises(s2w.S2WError):
        make_context(s2w, geom, 32, prec_g="bf16", max_batch=4, tc_fp8_act=True)


@pytest.mark.parametrize("act", [0, 2])
def test_fp8_tensor_operand_range_is_scaled(act):
    """The FP8 path's B operand (FP16, or hi + lo e4m3) carries a power-of-two
    scale from its amax (the whole operand's, or each (bin, rupture)'s):
    slip scaled by 1e6 or 1e-6 (beyond / far inside the FP16 and e4m3 ranges)
    gives the scaled waveforms, finite and within the tensor path's bar (a
    non-power-of-two rescale reshuffles the BF16 rounding of the later
    stages, ~2e-3 of the window; an overflow or underflow would be O(1))."""
    geom = compact_box(24, 700, 6, seed=65)
    Nt, B = 64, 3
    rng = np.random.default_rng(66)
    slip = rng.standard_normal((B, geom.Ns, Nt))
    slip[:, :, Nt // 2:] = 0
    ctx = make_context(s2w, geom, Nt, prec_g="fp8", max_batch=B, chunk=256, engine="tensor", tc_fp8_act=act)
    q1 = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    wn, _ = window_norms(G, P, slip)
    for alpha in (1e6, 1e-6):
        qa = ctx.waveforms(torch.tensor(slip * alpha, dtype=torch.float32, device="cuda")).cpu().numpy()
        assert np.all(np.isfinite(qa))
        d = np.linalg.norm((qa / alpha - q1).reshape(B, -1), axis=1)
        assert np.all(d <= TOL_TC * wn), (alpha, d / wn)
    ctx.sync()
