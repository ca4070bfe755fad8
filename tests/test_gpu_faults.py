"""Failure detection without a GPU fault: the library's test hooks
(s2w_opts.fault, or the S2W_FAULT environment variable) make a kernel's
bounded wait run out, an operator load report an allocation failure, or a
launch report a failure.  Each must come back as a status code, and a fresh
context afterwards must work normally.  Nothing here traps, faults or hangs
the GPU: the injected wait is bounded (2 ms), after which the kernel latches
the timeout, drains its own copies and returns."""
import numpy as np
import pytest

import oracle
import synth
from helpers import assert_parity, make_context, window_norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402

TIMEOUT, OOM, STATE, CUDA = -5, -2, -3, -4


def tiny():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    return wl, geom, wl.slip(geom, B=2)


def check_fresh_context(wl, geom, slip):
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2, prec_g="fp32_hilo", prec_p="fp32_hilo")
    q = ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda")).cpu().numpy()
    ctx.sync()
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    assert_parity(q, oracle.waveforms(G, P, slip), *window_norms(G, P, slip), tol=1e-5, label="fresh context")


def test_expired_wait_is_reported_by_sync():
    wl, geom, slip = tiny()
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2, fault="wait", fault_wait_us=2000)
    x = torch.tensor(slip, dtype=torch.float32, device="cuda")
    q = torch.zeros((2, wl.No, wl.Nt), dtype=torch.float32, device="cuda")
    ctx.waveforms(x, q=q)   # enqueued: the stage-1 kernel's first stage never fills
    with pytest.raises(s2w.S2WError) as e:
        ctx.sync()
    assert e.value.status == TIMEOUT
    assert b"status bits" in s2w.lib().s2w_last_error(ctx._h)
    ctx.sync()              # the status word was cleared by the report
    ctx.close()
    check_fresh_context(wl, geom, slip)


def test_injected_load_failure_is_an_allocation_error():
    wl, geom, slip = tiny()
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt, max_batch=2, fault="oom_load")
    with pytest.raises(s2w.S2WError) as e:
        ctx.load_greens(0, geom.greens_rows(0, wl.Ng, wl.Nt, np.float32))
    assert e.value.status == OOM
    with pytest.raises(s2w.S2WError) as e:
        ctx.load_adjoint(0, geom.adjoint_cols(0, wl.Ng, wl.Nt, np.float32))
    assert e.value.status == OOM
    with pytest.raises(s2w.S2WError) as e:   # nothing was marked loaded
        ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda"))
    assert e.value.status == STATE
    ctx.sync()
    ctx.close()
    check_fresh_context(wl, geom, slip)


def test_injected_launch_failure_from_the_environment(monkeypatch):
    wl, geom, slip = tiny()
    monkeypatch.setenv("S2W_FAULT", "launch")
    ctx = make_context(s2w, geom, wl.Nt, max_batch=2)
    monkeypatch.delenv("S2W_FAULT")
    with pytest.raises(s2w.S2WError) as e:
        ctx.waveforms(torch.tensor(slip, dtype=torch.float32, device="cuda"))
    assert e.value.status == CUDA
    ctx.sync()   # nothing was enqueued, nothing latched
    ctx.close()
    check_fresh_context(wl, geom, slip)
