"""s2w_waveforms_noalloc: the one-rupture entry point that allocates nothing.

It is meant for callers that cannot let the library allocate device memory
(applications that own all device memory through their own pool, code inside
a CUDA stream capture, latency-bound loops that must not wait on the
allocator).  Its intermediates live in a static device array shared by every
call.  This file is collected last on purpose, and must pass both alone in a
fresh process and after the other tests: the static array then holds whatever
the earlier calls left in it.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from helpers import BARS, make_context, window_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402


def call_noalloc(ctx, slip, q, stream):
    return s2w.lib().s2w_waveforms_noalloc(ctx._h, slip.data_ptr(), q.data_ptr(), stream.cuda_stream)


TOL_WINDOW = {"fp32": 1e-5, "bf16_hilo": BARS["stream_bf16_hilo"], "bf16": BARS["stream_bf16"],
              "fp8": BARS["stream_fp8"]}


@pytest.mark.parametrize("prec,max_batch", [("fp32", 1), ("fp32_hilo", 1), ("bf16", 1), ("bf16_hilo", 1),
                                            ("fp8", 1), ("bf16", 4)])
def test_noalloc_matches_waveforms_on_two_calls_in_a_row(prec, max_batch):
    """Two calls in a row through the C ABI (different ruptures, the same
    static scratch) against s2w_waveforms with B = 1, which runs the same
    stream kernels in the same order: equal bit for bit, in every storage
    precision (the FP32 pairs included), also on a context whose tensor
    engine is on (max_batch 4: one rupture still streams).  Against the FP64
    oracle: the FP32 pairs within 1e-5 relative L2 of every rupture, the
    other precisions within their window bound."""
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip_np = wl.slip(geom, B=2)
    slip = torch.tensor(slip_np, dtype=torch.float32, device="cuda")
    prec_p = "fp32_hilo" if prec == "fp32_hilo" else "fp32"
    ctx = make_context(s2w, geom, wl.Nt, prec_g=prec, prec_p=prec_p, max_batch=max_batch)
    stream = torch.cuda.current_stream()
    # the existing entry point, one rupture per call
    ref = [ctx.waveforms(slip[b:b + 1]).cpu().numpy()[0] for b in range(2)]
    out = [torch.full((wl.No, wl.Nt), float("nan"), device="cuda") for _ in range(2)]
    for b in range(2):
        st = call_noalloc(ctx, slip[b], out[b], stream)
        assert st == 0, s2w.lib().s2w_last_error(ctx._h)
    torch.cuda.synchronize()
    ctx.sync()
    q = np.stack([o.cpu().numpy() for o in out])
    assert np.array_equal(q, np.stack(ref))
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    q_ref = oracle.waveforms(G, P, slip_np)
    err = np.linalg.norm((q - q_ref).reshape(2, -1), axis=1)
    if prec == "fp32_hilo":
        assert np.all(err <= 1e-5 * np.linalg.norm(q_ref.reshape(2, -1), axis=1)), err
    else:
        wn, _ = window_norms(G, P, slip_np)
        assert np.all(err <= TOL_WINDOW[prec] * wn), err / wn


def test_noalloc_rejects_oversize_and_host_pointers():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    ctx = make_context(s2w, geom, wl.Nt, max_batch=1)
    host_slip = np.zeros((wl.Ns, wl.Nt), np.float32)
    host_q = np.zeros((wl.No, wl.Nt), np.float32)
    L = s2w.lib()
    st = L.s2w_waveforms_noalloc(ctx._h, host_slip.ctypes.data, host_q.ctypes.data, None)
    assert st == -1 and b"device pointers" in L.s2w_last_error(ctx._h)
    # 20,000 grid points at Nt = 256 need ~82 MB of scratch: beyond the 32 MiB
    big = s2w.Context(8, 20000, 4, 256)
    d = torch.zeros((8, 256), device="cuda")
    qd = torch.zeros((4, 256), device="cuda")
    st = L.s2w_waveforms_noalloc(big._h, d.data_ptr(), qd.data_ptr(), None)
    assert st == -6
    assert b"scratch" in L.s2w_last_error(big._h)
