"""Shared test helpers: build a library context from a synthetic geometry and
compute the FP64 oracle reference for the same inputs."""
import numpy as np

import oracle

# Error bars of the reduced-precision paths: ||q - q_ref|| <= bar * ||q_win||
# per rupture (q_win: the 2 Nt-sample FFT window).  Each is about twice the
# error that the path's own roundings produce in an otherwise exact FP64
# evaluation (tests/error_model.py) on the worst rupture of the tiny workload
# (8.6e-3 for the tensor BF16 path, 2.6e-3 for BF16 storage, 5.2e-2 for FP8,
# 5.9e-6 / 1.7e-5 for the hi/lo splits); tests/test_error_model.py checks
# that every bar lies between 1.5 and 4 times that modelled error.
BARS = {"stream_bf16": 5e-3, "stream_bf16_hilo": 2e-5, "stream_fp8": 1e-1,
        "tensor_bf16": 2e-2, "tensor_split": 3e-5, "tensor_fp8": 1e-1}


def make_context(s2w, geom, Nt, prec_g="fp32", prec_p="fp32", dt_mode="backward",
                 max_batch=1, chunk=4096, order=None, engine="auto", tc_adjoint=False,
                 single_pass=False, tc_pair="auto", tc_fp8_act=None, **opts):
    """Context with both operators loaded from the generator, in row chunks
    (optionally in a permuted chunk order)."""
    Ng = geom.Ng
    ctx = s2w.Context(geom.Ns, Ng, geom.No, Nt, prec_g=prec_g, prec_p=prec_p,
                      dt_mode=dt_mode, max_batch=max_batch, engine=engine,
                      tc_adjoint=tc_adjoint, single_pass=single_pass, tc_pair=tc_pair, tc_fp8_act=tc_fp8_act,
                      **opts)
    starts = list(range(0, Ng, chunk))
    if order is not None:
        starts = [starts[i] for i in order]
    for g0 in starts:
        g1 = min(Ng, g0 + chunk)
        ctx.load_greens(g0, geom.greens_rows(g0, g1, Nt, np.float32))
        ctx.load_adjoint(g0, np.ascontiguousarray(geom.adjoint_cols(g0, g1, Nt, np.float32)))
    return ctx


def oracle_reference(geom, Nt, slip, dt_mode="backward", chunk=1024, seafloor=False):
    """FP64 oracle q (and optionally m) through Eq. (distributed-composition)
    over grid chunks, with operators regenerated in FP64."""
    if seafloor:
        G = geom.greens_rows(0, geom.Ng, Nt)
        P = geom.adjoint_cols(0, geom.Ng, Nt)
        return oracle.waveforms(G, P, slip, dt_mode=dt_mode, return_seafloor=True)

    def chunks():
        for g0 in range(0, geom.Ng, chunk):
            g1 = min(geom.Ng, g0 + chunk)
            yield geom.greens_rows(g0, g1, Nt), geom.adjoint_cols(g0, g1, Nt)
    return oracle.waveforms_partitioned(chunks(), slip, dt_mode=dt_mode)


def rel_l2(a, ref):
    return oracle.rel_l2(np.asarray(a, dtype=np.float64), ref)


def window_norms(G, P, slip, dt_mode="backward"):
    """Per-rupture norm of the oracle's 2 Nt-sample FFT window (oracle.fft_window)
    and the window/head energy ratio kappa."""
    qw = oracle.fft_window(G, P, slip, dt_mode)
    if qw.ndim == 2:
        qw = qw[None]
    Nt = qw.shape[-1] // 2
    wn = np.linalg.norm(qw.reshape(qw.shape[0], -1), axis=1)
    hn = np.linalg.norm(qw[..., :Nt].reshape(qw.shape[0], -1), axis=1)
    return wn, wn / np.maximum(hn, 1e-300)


def assert_parity(q, q_ref, wnorm, kappa, tol, strict=1e-5, label=""):
    """Per rupture, the plain relative L2 error over all No x Nt samples and
    the error relative to the 2 Nt-sample FFT window (``window_norms``) are
    printed, then:
    FP32-class paths (tol <= 1e-5): plain rel-L2 <= strict (1e-5, the stated
        target) for EVERY rupture, whatever its window/head ratio kappa;
    reduced-precision paths: ||q - q_ref|| <= tol * ||q_win||, the path's
        stated bound on the scale its FFT evaluation works on."""
    q = np.asarray(q, dtype=np.float64)
    q_ref = np.asarray(q_ref, dtype=np.float64)
    if q.ndim == 2:
        q, q_ref = q[None], q_ref[None]
    err = np.linalg.norm((q - q_ref).reshape(q.shape[0], -1), axis=1)
    rel = err / np.maximum(np.linalg.norm(q_ref.reshape(q.shape[0], -1), axis=1), 1e-300)
    win = err / np.maximum(wnorm, 1e-300)
    print(f"{label}: rel-L2 {rel}, error / window norm {win}, kappa {kappa}")
    if tol <= 1e-5:
        assert np.all(rel <= strict), (label, rel, kappa)
    else:
        assert np.all(win <= tol), (label, win, tol)
    return rel, win
