"""CUDA-graph replay (s2w_waveforms_graph) and the engine autotuner
(s2w_autotune), through the C ABI.

A replayed graph runs the same kernels with the same launch shapes on the
same buffers as s2w_waveforms, so its output is compared bit for bit; the
autotuner only chooses among configurations that the other tests check
against the oracle, and its choices are checked for validity and for
parity of the path they select.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BARS, assert_parity, make_context, window_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402


def compact_box(Ns, Ng, No, seed, scale=0.1):
    g = synth.geometry_box(Ns, Ng, No, seed)
    return synth.Geometry(g.sub * scale, g.grid * scale, g.obs * scale,
                          g.strike * scale, g.dip * scale, "box")


def slips(B, Ns, Nt, seed):
    rng = np.random.default_rng(seed)
    s = rng.standard_normal((B, Ns, Nt))
    s[:, :, Nt // 2:] = 0
    return s


@pytest.mark.parametrize("prec,engine,B", [("fp32", "stream", 3), ("bf16", "tensor", 7), ("fp8", "stream", 2)])
def test_graph_replay_matches_direct_call(prec, engine, B):
    geom = compact_box(24, 700, 6, seed=21)
    Nt = 64
    ctx = make_context(s2w, geom, Nt, prec_g=prec, max_batch=B, engine=engine)
    s1 = torch.tensor(slips(B, geom.Ns, Nt, 1), dtype=torch.float32, device="cuda")
    s2 = torch.tensor(slips(B, geom.Ns, Nt, 2), dtype=torch.float32, device="cuda")
    ref1 = ctx.waveforms(s1).clone()
    ref2 = ctx.waveforms(s2).clone()
    x = s1.clone()
    q = torch.empty_like(ref1)
    ctx.waveforms_graph(x, q)  # captures
    assert torch.equal(q, ref1)
    x.copy_(s2)  # same buffers, new contents: replay sees them
    ctx.waveforms_graph(x, q)
    assert torch.equal(q, ref2)
    q.zero_()
    ctx.waveforms_graph(x, q)
    assert torch.equal(q, ref2)
    # another output buffer: re-captured
    q2 = torch.empty_like(ref1)
    x.copy_(s1)
    ctx.waveforms_graph(x, q2)
    assert torch.equal(q2, ref1)
    ctx.sync()


def test_graph_replay_parity_and_profile():
    """The replayed pipeline (the FP32 path with FP32-pair spectra) meets the
    FP32 bar on the tiny workload; the profiler counts one graph per replay
    with the kernels it holds."""
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=2)
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt, prec_g="fp32_hilo", prec_p="fp32_hilo", max_batch=2)
    ctx.load_greens(0, geom.greens_rows(0, wl.Ng, wl.Nt, np.float32))
    ctx.load_adjoint(0, geom.adjoint_cols(0, wl.Ng, wl.Nt, np.float32))
    x = torch.tensor(slip, dtype=torch.float32, device="cuda")
    q = torch.empty((2, wl.No, wl.Nt), dtype=torch.float32, device="cuda")
    ctx.profile_enable(True)
    for _ in range(3):
        ctx.waveforms_graph(x, q)
    stages, launches = ctx.profile_read()
    assert stages["graph"][1] == 3
    assert launches >= 3 * 3  # at least rfft, two contractions per replay
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    assert_parity(q.cpu().numpy(), oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=1e-5,
                  label="graph tiny fp32 pairs")
    assert torch.equal(q, ctx.waveforms(x))
    ctx.sync()


def test_graph_rejects_host_pointers():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    ctx = make_context(s2w, geom, wl.Nt, max_batch=1)
    x = np.zeros((1, wl.Ns, wl.Nt), np.float32)
    q = np.zeros((1, wl.No, wl.Nt), np.float32)
    with pytest.raises(RuntimeError):
        ctx.waveforms_graph(x, q)


def test_autotune_choices_and_selected_path():
    geom = compact_box(24, 700, 6, seed=22)
    Nt, B = 64, 40
    ctx = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B)
    t = ctx.autotune(B)
    print("autotune:", t)
    assert not t["from_cache"]
    assert t["ms_stream_per_rupture"] > 0
    assert t["probe_batch"] == B
    # B = 40 fits one pass: the forms probed are the three pair modes at 40 ruptures per pass
    assert [(f["bsub"], f["pair"]) for f in t["forms"]] == [(B, "auto"), (B, "off"), (B, "on")]
    assert all(f["ms"] > 0 for f in t["forms"])
    assert t["tc_pair"] in ("auto", "off", "on") and t["tc_bsub"] == B
    assert len(t["s2_chunks"]) >= 2 and all(c["ms"] > 0 for c in t["s2_chunks"])
    assert t["tc_s2_chunks"] in [c["chunks"] for c in t["s2_chunks"]]
    assert t["tc_min_batch"] >= 1
    sizes = [1, 2, 4, 8, 16, 32, 64]
    measured = [b for b, v in zip(sizes, t["ms_tensor_batch"]) if v > 0]
    assert measured == [b for b in sizes if b <= B]
    # whichever engine AUTO now takes for each batch size, it meets the bar
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    for nb in (1, 3, B):
        s = slips(nb, geom.Ns, Nt, 30 + nb)
        q = ctx.waveforms(torch.tensor(s, dtype=torch.float32, device="cuda")).cpu().numpy()
        assert_parity(q, oracle.waveforms(G, P, s), *window_norms(G, P, s), tol=BARS["tensor_bf16"], label=f"autotuned B={nb}")
    ctx.sync()


def test_autotune_split_keeps_short_accumulations():
    """With the BF16 hi/lo split the autotuner probes no stage-2 chunk count
    below the round-balance default (the first candidate): fewer chunks mean
    longer FP32 accumulations, which the split's error level shows."""
    geom = compact_box(24, 700, 6, seed=24)
    Nt, B = 64, 40
    ctx = make_context(s2w, geom, Nt, prec_g="bf16_hilo", prec_p="fp32", max_batch=B)
    t = ctx.autotune(B)
    probed = [c["chunks"] for c in t["s2_chunks"]]
    print("split autotune chunks:", t["s2_chunks"], "chosen", t["tc_s2_chunks"])
    assert probed and min(probed) == probed[0] and t["tc_s2_chunks"] >= probed[0]
    s = slips(B, geom.Ns, Nt, 31)
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    q = ctx.waveforms(torch.tensor(s, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_parity(q, oracle.waveforms(G, P, s), *window_norms(G, P, s), tol=BARS["tensor_split"], label="autotuned split")
    ctx.sync()


def test_autotune_without_tensor_engine():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    ctx = make_context(s2w, geom, wl.Nt, max_batch=4)  # FP32: stream engine only
    t = ctx.autotune(4)
    assert t["ms_stream_per_rupture"] > 0
    assert t["forms"] == [] and t["s2_chunks"] == []
    assert t["ms_tensor_batch"] == [0.0] * 7
    ctx.sync()


def test_autotune_cache_second_context(tmp_path):
    """The tuned schedule is written to the cache file; a second context for
    the same problem takes it from there without timing anything, and its
    waveforms equal the first context's bit for bit (same schedule, same
    kernels).  A third context given the same choices as explicit options
    computes the same bits without any tuning."""
    cache = str(tmp_path / "s2w_tune.txt")
    geom = compact_box(24, 700, 6, seed=23)
    Nt, B = 64, 40
    s = slips(B, geom.Ns, Nt, 77)
    x = torch.tensor(s, dtype=torch.float32, device="cuda")
    ctx1 = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B, tune_cache=cache)
    t1 = ctx1.autotune(B)
    assert not t1["from_cache"]
    text = open(cache).read()
    assert text.count("s2w-tune-1 ") == 1 and f"Ng=700" in text
    q1 = ctx1.waveforms(x).cpu().numpy()
    ctx1.sync()
    ctx2 = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B, tune_cache=cache)
    t2 = ctx2.autotune(B)
    assert t2["from_cache"]
    assert t2["forms"] == [] and t2["s2_chunks"] == [] and t2["ms_stream_per_rupture"] == 0.0
    for k in ("tc_bsub", "tc_pair", "tc_s2_chunks", "tc_min_batch"):
        assert t2[k] == t1[k], k
    q2 = ctx2.waveforms(x).cpu().numpy()
    ctx2.sync()
    assert np.array_equal(q1, q2)
    ctx3 = make_context(s2w, geom, Nt, prec_g="bf16", max_batch=B, tc_bsub=0, tc_pair=t1["tc_pair"],
                        tc_s2_chunks=t1["tc_s2_chunks"])
    q3 = ctx3.waveforms(x).cpu().numpy()
    ctx3.sync()
    assert np.array_equal(q1, q3)
    G = geom.greens_rows(0, geom.Ng, Nt)
    P = geom.adjoint_cols(0, geom.Ng, Nt)
    assert_parity(q2, oracle.waveforms(G, P, s), *window_norms(G, P, s), tol=BARS["tensor_bf16"], label="cached schedule")
    # a different problem (another batch) is not in the cache: measured and appended
    t4 = ctx2.autotune(B // 2)
    assert not t4["from_cache"]
    assert open(cache).read().count("s2w-tune-1 ") == 2


def test_graph_cache_alternating_buffers_and_eviction():
    """Ten output buffers used in turn (more than the eight graphs a context
    keeps): every replay or re-capture writes the direct call's result."""
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2)
    x = torch.tensor(wl.slip(geom, B=2), dtype=torch.float32, device="cuda")
    ref = ctx.waveforms(x).clone()
    qs = [torch.empty_like(ref) for _ in range(10)]
    for rnd in range(3):
        for q in qs:
            q.fill_(float("nan"))
            ctx.waveforms_graph(x, q)
            assert torch.equal(q, ref), rnd
    ctx.sync()
