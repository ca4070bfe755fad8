"""Adjoint / gradient path (s2w_adjoint and the torch.autograd.Function)
against the FP64 oracle, through the C ABI.

Bars per rupture, as for the forward path but on the adjoint's own window:
||g - g_ref|| <= TOL * ||g_win|| with g_win the full correlation window the
FFT evaluation forms before Truncate (oracle.fft_window_adjoint), and the
plain rel-L2 <= 1e-5 for FP32-class storage where that window is not
dominated by negative lags (window/head ratio <= 10).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import make_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402
from paper_2608_21763_gb300 import autograd as s2w_autograd  # noqa: E402

TOL = {"fp32": 1e-5, "bf16_hilo": 2e-5, "bf16": 5e-3, "fp8": 1e-1}


def compact_box(Ns, Ng, No, seed, scale=0.1):
    g = synth.geometry_box(Ns, Ng, No, seed)
    return synth.Geometry(g.sub * scale, g.grid * scale, g.obs * scale,
                          g.strike * scale, g.dip * scale, "box")


def adjoint_bars(g, G, P, r, tol, label, strict=1e-5, kappa_max=10.0):
    gw = oracle.fft_window_adjoint(G, P, r)
    Nt = G.shape[2]
    g_ref = gw[..., Nt:]
    B = g.shape[0]
    err = np.linalg.norm((g.astype(np.float64) - g_ref).reshape(B, -1), axis=1)
    wn = np.linalg.norm(gw.reshape(B, -1), axis=1)
    hn = np.linalg.norm(g_ref.reshape(B, -1), axis=1)
    rel, win, kappa = err / hn, err / wn, wn / hn
    print(f"{label}: rel-L2 {rel}, error / window norm {win}, kappa {kappa}")
    assert np.all(win <= tol), (label, win)
    if tol <= 1e-5:
        assert np.all(rel[kappa <= kappa_max] <= strict), (label, rel, kappa)
    return g_ref


@pytest.fixture(scope="module")
def tiny_ops():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    return wl, geom, G, P


@pytest.mark.parametrize("prec", ["fp32", "bf16_hilo", "bf16", "fp8"])
def test_adjoint_against_oracle(tiny_ops, prec):
    wl, geom, G, P = tiny_ops
    r = synth.random_waveforms(3, wl.No, wl.Nt, seed=4)
    ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, max_batch=3, chunk=256, engine="stream")
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    adjoint_bars(g, G, P, r, TOL[prec], f"adjoint tiny {prec}")


def test_adjoint_identity(tiny_ops):
    """<W s, r> = <s, W^T r> with both sides from the GPU (FP32)."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=3)
    r = synth.random_waveforms(3, wl.No, wl.Nt, seed=5)
    ctx = make_context(s2w, geom, wl.Nt, max_batch=3)
    q = ctx.waveforms(torch.tensor(s, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    for b in range(3):
        lhs, rhs = np.sum(q[b] * r[b]), np.sum(s[b] * g[b])
        assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(q[b]) * np.linalg.norm(r[b]) + 1e-5 * abs(lhs), (b, lhs, rhs)


def test_gradient_central_differences(tiny_ops):
    """GPU gradient of 0.5 ||W s - d||^2 (adjoint applied to the FP64
    residual) against central differences (h = 1e-3) of the FP64 oracle
    misfit along random unit directions."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=1)[0]
    d = synth.random_waveforms(1, wl.No, wl.Nt, seed=6)[0]
    r = oracle.waveforms(G, P, s) - d
    ctx = make_context(s2w, geom, wl.Nt)
    g = ctx.adjoint(torch.tensor(r[None], dtype=torch.float32, device="cuda")).cpu().numpy()[0].astype(np.float64)
    loss = lambda x: 0.5 * np.sum((oracle.waveforms(G, P, x) - d) ** 2)
    rng = np.random.default_rng(7)
    h = 1e-3
    for _ in range(4):
        e = rng.standard_normal(s.shape)
        e /= np.linalg.norm(e)
        fd = (loss(s + h * e) - loss(s - h * e)) / (2 * h)
        assert abs(fd - np.sum(g * e)) <= 1e-4 * max(abs(fd), np.linalg.norm(g) * 1e-3), (fd, np.sum(g * e))


def test_autograd_misfit_gradient(tiny_ops):
    """torch.autograd through the library: loss.backward() gives the misfit
    gradient; compared with the FP64 oracle gradient at the same slip and
    targets."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=2)
    d = synth.random_waveforms(2, wl.No, wl.Nt, seed=8)
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2)
    st = torch.tensor(s, dtype=torch.float32, device="cuda", requires_grad=True)
    dt = torch.tensor(d, dtype=torch.float32, device="cuda")
    loss = s2w_autograd.misfit(ctx, st, dt)
    loss.backward()
    g = st.grad.cpu().numpy()
    loss_ref, g_ref = oracle.gradient(G, P, s, d)
    assert abs(loss.item() - loss_ref.sum()) <= 1e-5 * loss_ref.sum()
    r = oracle.waveforms(G, P, s) - d
    adjoint_bars(g, G, P, r, 2e-5, "autograd misfit")  # residual carries the forward FP32 error too
    assert np.all(np.linalg.norm((g - g_ref).reshape(2, -1), axis=1) <=
                  1e-4 * np.linalg.norm(g_ref.reshape(2, -1), axis=1))


@pytest.mark.parametrize("Ns,Ng,No,Nt", [(5, 1000, 3, 64), (1, 37, 1, 32), (7, 2100, 5, 128)])
def test_adjoint_ragged_shapes(Ns, Ng, No, Nt):
    geom = compact_box(Ns, Ng, No, seed=Ns + Ng + 1)
    r = np.random.default_rng(2).standard_normal((2, No, Nt))
    ctx = make_context(s2w, geom, Nt, max_batch=2, chunk=512)
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    adjoint_bars(g, G, P, r, 1e-5, f"adjoint ragged {Ns}x{Ng}x{No}x{Nt}")


def test_adjoint_host_and_device_agree(tiny_ops):
    wl, geom, G, P = tiny_ops
    r = synth.random_waveforms(2, wl.No, wl.Nt, seed=9).astype(np.float32)
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2)
    g_host = ctx.adjoint(r)
    g_dev = ctx.adjoint(torch.tensor(r, device="cuda")).cpu().numpy()
    assert np.array_equal(g_host, g_dev)


def test_adjoint_plain_workload_full_size():
    """Gradient-shaped check at the paper shape: 963 subfaults, 20,000 grid
    points, 64 observations, 256 steps; the oracle gradient summed over grid
    chunks (Eq. distributed-composition, transposed)."""
    wl = synth.WORKLOADS["plain"]
    geom = wl.geometry_obj()
    r = synth.random_waveforms(1, wl.No, wl.Nt, seed=11)
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt)
    g_win = None
    for g0 in range(0, wl.Ng, 1024):
        g1 = min(wl.Ng, g0 + 1024)
        G = geom.greens_rows(g0, g1, wl.Nt)
        P = geom.adjoint_cols(g0, g1, wl.Nt)
        ctx.load_greens(g0, G.astype(np.float32))
        ctx.load_adjoint(g0, np.ascontiguousarray(P.astype(np.float32)))
        w = oracle.fft_window_adjoint(G, P, r)
        g_win = w if g_win is None else g_win + w
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    g_ref = g_win[..., wl.Nt:]
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    win = np.linalg.norm(g - g_ref) / np.linalg.norm(g_win)
    print(f"adjoint plain full size: rel-L2 {err}, error / window norm {win}")
    assert win <= 1e-5 and err <= 1e-5 * max(1.0, np.linalg.norm(g_win) / np.linalg.norm(g_ref)), (err, win)
    ctx.sync()


def test_misfit_gradient_entry_point(tiny_ops):
    """s2w_misfit_gradient (forward, residual, adjoint in the library)
    against the FP64 oracle misfit and gradient."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=3)
    d = synth.random_waveforms(3, wl.No, wl.Nt, seed=12)
    ctx = make_context(s2w, geom, wl.Nt, max_batch=3)
    g, loss = ctx.misfit_gradient(torch.tensor(s, dtype=torch.float32, device="cuda"),
                                  torch.tensor(d, dtype=torch.float32, device="cuda"))
    loss_ref, g_ref = oracle.gradient(G, P, s, d)
    assert np.allclose(loss.cpu().numpy(), loss_ref, rtol=1e-5)
    r = oracle.waveforms(G, P, s) - d
    adjoint_bars(g.cpu().numpy(), G, P, r, 2e-5, "misfit gradient")
    g_h, loss_h = ctx.misfit_gradient(s.astype(np.float32), d.astype(np.float32))
    assert np.array_equal(g_h, g.cpu().numpy()) and np.array_equal(loss_h, loss.cpu().numpy())


# tensor-engine adjoint (transposed operator copies, tcgen05 GEMMs)
TOL_TC_ADJ = {"bf16": 1e-2, "bf16_hilo": 3e-5}


@pytest.mark.parametrize("prec", ["bf16", "bf16_hilo"])
def test_tensor_adjoint_against_oracle(tiny_ops, prec):
    wl, geom, G, P = tiny_ops
    r = synth.random_waveforms(5, wl.No, wl.Nt, seed=21)
    ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, max_batch=5, engine="tensor", tc_adjoint=True)
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    adjoint_bars(g, G, P, r, TOL_TC_ADJ[prec], f"tensor adjoint tiny {prec}")


@pytest.mark.parametrize("tc_pair", ["off", "on"])
@pytest.mark.parametrize("Ns,Ng,No,Nt,B", [(5, 1000, 3, 64, 2), (24, 700, 6, 32, 130), (7, 2100, 5, 128, 9)])
def test_tensor_adjoint_shapes(Ns, Ng, No, Nt, B, tc_pair):
    """Ragged shapes: partial M tiles of the transposed operators, No far
    below its 32-column padding, and (B = 130) two sub-batches; with one CTA
    per 128-row tile and with two-SM CTA pairs where the shape allows."""
    geom = compact_box(Ns, Ng, No, seed=Ns + Ng + 3)
    r = np.random.default_rng(3).standard_normal((B, No, Nt))
    ctx = make_context(s2w, geom, Nt, prec_g="bf16_hilo", max_batch=B, chunk=512, engine="tensor",
                       tc_adjoint=True, tc_pair=tc_pair)
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    G = geom.greens_rows(0, Ng, Nt)
    P = geom.adjoint_cols(0, Ng, Nt)
    adjoint_bars(g, G, P, r, TOL_TC_ADJ["bf16_hilo"], f"tensor adjoint {Ns}x{Ng}x{No}x{Nt} B={B}")


def test_tensor_adjoint_identity_and_stream_agreement(tiny_ops):
    """<W s, r> = <s, W^T r> with both sides from the split tensor engine,
    and the tensor adjoint against the streaming adjoint of the same
    hi/lo operator."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=4)
    r = synth.random_waveforms(4, wl.No, wl.Nt, seed=22)
    ctx = make_context(s2w, geom, wl.Nt, prec_g="bf16_hilo", max_batch=4, engine="tensor", tc_adjoint=True)
    q = ctx.waveforms(torch.tensor(s, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    g = ctx.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    # each side carries its engine error on the scale of its FFT window
    qn = np.linalg.norm(oracle.fft_window(G, P, s).reshape(4, -1), axis=1)
    gw = oracle.fft_window_adjoint(G, P, r)
    wn = np.linalg.norm(gw.reshape(4, -1), axis=1)
    for b in range(4):
        lhs, rhs = np.sum(q[b] * r[b]), np.sum(s[b] * g[b])
        bound = 3e-5 * (qn[b] * np.linalg.norm(r[b]) + np.linalg.norm(s[b]) * wn[b])
        assert abs(lhs - rhs) <= bound, (b, lhs, rhs, bound)
    cs = make_context(s2w, geom, wl.Nt, prec_g="bf16_hilo", max_batch=4, engine="stream")
    g_s = cs.adjoint(torch.tensor(r, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.all(np.linalg.norm((g - g_s).reshape(4, -1), axis=1) <= 6e-5 * wn)
    ctx.sync()


def test_tensor_misfit_gradient(tiny_ops):
    """s2w_misfit_gradient with forward and adjoint on the split tensor
    engine against the FP64 oracle misfit and gradient, and autograd through
    the same context."""
    wl, geom, G, P = tiny_ops
    s = wl.slip(geom, B=3)
    d = synth.random_waveforms(3, wl.No, wl.Nt, seed=23)
    ctx = make_context(s2w, geom, wl.Nt, prec_g="bf16_hilo", max_batch=3, engine="tensor", tc_adjoint=True)
    g, loss = ctx.misfit_gradient(torch.tensor(s, dtype=torch.float32, device="cuda"),
                                  torch.tensor(d, dtype=torch.float32, device="cuda"))
    loss_ref, g_ref = oracle.gradient(G, P, s, d)
    assert np.allclose(loss.cpu().numpy(), loss_ref, rtol=5e-5)
    r = oracle.waveforms(G, P, s) - d
    adjoint_bars(g.cpu().numpy(), G, P, r, 6e-5, "tensor misfit gradient")
    st = torch.tensor(s, dtype=torch.float32, device="cuda", requires_grad=True)
    lt = s2w_autograd.misfit(ctx, st, torch.tensor(d, dtype=torch.float32, device="cuda"))
    lt.backward()
    assert torch.allclose(st.grad, g, rtol=0, atol=1e-6 * float(g.abs().max()))
    ctx.sync()
