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

import synth
from helpers import make_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402


def call_noalloc(ctx, slip, q, stream):
    return s2w.lib().s2w_waveforms_noalloc(ctx._h, slip.data_ptr(), q.data_ptr(), stream.cuda_stream)


def test_noalloc_matches_waveforms_on_two_calls_in_a_row():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = torch.tensor(wl.slip(geom, B=2), dtype=torch.float32, device="cuda")
    ctx = make_context(s2w, geom, wl.Nt, max_batch=1)
    stream = torch.cuda.current_stream()
    # the existing entry point, one rupture per call
    ref = [ctx.waveforms(slip[b:b + 1]).cpu().numpy()[0].astype(np.float64) for b in range(2)]
    # two calls in a row through the C ABI, different ruptures, same static scratch
    out = [torch.full((wl.No, wl.Nt), float("nan"), device="cuda") for _ in range(2)]
    for b in range(2):
        st = call_noalloc(ctx, slip[b], out[b], stream)
        assert st == 0, s2w.lib().s2w_last_error(ctx._h)
    torch.cuda.synchronize()
    ctx.sync()
    for b in range(2):
        q = out[b].cpu().numpy().astype(np.float64)
        # FP32 bar of the parity tests: 1e-5 relative L2 (the two entry points
        # run the same kernels, so the results should in fact agree exactly)
        err = np.linalg.norm(q - ref[b]) / np.linalg.norm(ref[b])
        assert err <= 1e-5, (b, err)


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
