"""FP64 CPU oracle for the two-stage source-to-waveform map.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and
its Python binding never do, and share no code with it.

What it computes (paper, Sec. II):

* ``bltt_apply(F, x)``: one block lower-triangular Toeplitz matvec written as
  the direct temporal convolution of Eq. (time-domain-conv),
  ``y_i[n] = sum_j sum_{k=0}^{n} f_ij[k] x_j[n-k]``.  With ``F = G`` it is
  Eq. (elastic-response) ``m_n = sum_k F_{G,k} s_{n-k}``; with ``F = P`` it is
  Eq. (waveform-response) ``q_n = sum_k F_{q,k} v_{n-k}``.
* ``dt_apply(m)``: ``v = D_t m`` (Sec. II-B.2).  The paper does not print the
  stencil; the reading taken is the first-order backward difference
  ``v[n] = (m[n] - m[n-1]) / dt`` with ``m[-1] = 0`` (causal and lower
  triangular Toeplitz, so the composition stays block Toeplitz), dt = 1 s.
  ``dt_mode="none"`` skips it (the map is then two plain convolutions).
* ``waveforms(G, P, s)``: ``q = F_q D_t F_G s`` (Alg. 1, steps 2-4).
* ``waveforms_partitioned(chunks, s)``: Eq. (distributed-composition),
  ``q = sum_r F_q^(r) D_t F_G^(r) s`` over a partition of the seafloor grid,
  each chunk being ``(G[rows r], P[:, cols r])``.
* ``gradient(...)``: for the misfit ``L = 0.5 ||q(s) - d||^2``,
  ``dL/ds = F_G^T D_t^T F_q^T (q - d)``, each transpose written out directly.
* ``dft_real(x, L)``: the DFT of a real sequence zero-padded to length L, bins
  ``0..L/2`` (Alg. 2, ZeroPad then FFT, as the plain sum).

Parity pins (tests/test_oracle.py) tie every function to something other than
itself: explicit dense BLTT matrices, impulse responses, linearity, time-shift
invariance, causality, numpy's FFT, closed-form DFTs and the adjoint identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (gcc -O2, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, L, I, D = ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_double
        lib.oracle_bltt_apply.argtypes = [P, L, L, I, P, L, P]
        lib.oracle_bltt_transpose.argtypes = [P, L, L, I, P, L, P]
        lib.oracle_dt_apply.argtypes = [P, L, I, D, P]
        lib.oracle_dt_transpose.argtypes = [P, L, I, D, P]
        lib.oracle_dft_real.argtypes = [P, L, I, I, P, P]
        for f in (lib.oracle_bltt_apply, lib.oracle_bltt_transpose,
                  lib.oracle_dt_apply, lib.oracle_dt_transpose,
                  lib.oracle_dft_real):
            f.restype = None
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _batched(x, nin, nt):
    x = _f64(x)
    squeeze = x.ndim == 2
    if squeeze:
        x = x[None]
    assert x.shape[1:] == (nin, nt), (x.shape, nin, nt)
    return x, squeeze


def bltt_apply(F: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. (time-domain-conv).  F: [Nout][Nin][Nt], x: [B][Nin][Nt] or
    [Nin][Nt] -> y with the same leading shape and Nout channels."""
    F = _f64(F)
    nout, nin, nt = F.shape
    x, sq = _batched(x, nin, nt)
    y = np.empty((x.shape[0], nout, nt))
    _load().oracle_bltt_apply(F.ctypes.data, nout, nin, nt, x.ctypes.data,
                              x.shape[0], y.ctypes.data)
    return y[0] if sq else y


def bltt_transpose(F: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Transpose of ``bltt_apply``: ``x_j[n] = sum_i sum_{k<=Nt-1-n}
    f_ij[k] y_i[n+k]``."""
    F = _f64(F)
    nout, nin, nt = F.shape
    y, sq = _batched(y, nout, nt)
    x = np.empty((y.shape[0], nin, nt))
    _load().oracle_bltt_transpose(F.ctypes.data, nout, nin, nt, y.ctypes.data,
                                  y.shape[0], x.ctypes.data)
    return x[0] if sq else x


def dt_apply(m: np.ndarray, dt: float = 1.0) -> np.ndarray:
    """``v[n] = (m[n] - m[n-1]) / dt``, ``m[-1] = 0``, along the last axis."""
    m = _f64(m)
    v = np.empty_like(m)
    nt = m.shape[-1]
    _load().oracle_dt_apply(m.ctypes.data, m.size // nt, nt, dt, v.ctypes.data)
    return v


def dt_transpose(w: np.ndarray, dt: float = 1.0) -> np.ndarray:
    """``u[n] = (w[n] - w[n+1]) / dt``, ``w[Nt] = 0``, along the last axis."""
    w = _f64(w)
    u = np.empty_like(w)
    nt = w.shape[-1]
    _load().oracle_dt_transpose(w.ctypes.data, w.size // nt, nt, dt,
                                u.ctypes.data)
    return u


def dft_real(x: np.ndarray, L: int) -> np.ndarray:
    """Bins ``0..L/2`` of the DFT of each row of x zero-padded to length L."""
    x = _f64(x)
    n_in = x.shape[-1]
    assert n_in <= L and L % 2 == 0
    rows = x.size // n_in
    re = np.empty((rows, L // 2 + 1))
    im = np.empty_like(re)
    _load().oracle_dft_real(x.ctypes.data, rows, n_in, L, re.ctypes.data,
                            im.ctypes.data)
    return (re + 1j * im).reshape(x.shape[:-1] + (L // 2 + 1,))


def _stage_dt(m, dt_mode, dt):
    if dt_mode == "none":
        return m
    assert dt_mode == "backward", dt_mode
    return dt_apply(m, dt)


def _stage_dt_t(w, dt_mode, dt):
    if dt_mode == "none":
        return w
    return dt_transpose(w, dt)


def waveforms(G, P, s, dt_mode: str = "backward", dt: float = 1.0,
              return_seafloor: bool = False):
    """``q = F_q D_t F_G s`` for full operators G [Ng][Ns][Nt], P [No][Ng][Nt]
    and slip s [B][Ns][Nt] (or [Ns][Nt])."""
    m = bltt_apply(G, s)
    q = bltt_apply(P, _stage_dt(m, dt_mode, dt))
    return (q, m) if return_seafloor else q


def waveforms_partitioned(chunks, s, dt_mode: str = "backward",
                          dt: float = 1.0):
    """Eq. (distributed-composition): ``q = sum_r F_q^(r) D_t F_G^(r) s``.

    ``chunks`` yields ``(G_r, P_r)`` with ``G_r = G[I_r]`` ([n_r][Ns][Nt]) and
    ``P_r = P[:, I_r]`` ([No][n_r][Nt]) for a disjoint partition {I_r} of the
    grid points."""
    q = None
    for G_r, P_r in chunks:
        q_r = bltt_apply(P_r, _stage_dt(bltt_apply(G_r, s), dt_mode, dt))
        q = q_r if q is None else q + q_r
    return q


def gradient(G, P, s, d, dt_mode: str = "backward", dt: float = 1.0):
    """Misfit ``L = 0.5 ||q(s) - d||^2`` and ``dL/ds = F_G^T D_t^T F_q^T r``
    with ``r = q(s) - d``.  Returns (L per rupture, dL/ds)."""
    q = waveforms(G, P, s, dt_mode, dt)
    r = q - _f64(d)
    loss = 0.5 * np.sum(r.reshape(r.shape[0], -1) ** 2, axis=1) if r.ndim == 3 \
        else 0.5 * np.sum(r ** 2)
    w = bltt_transpose(P, r)
    g = bltt_transpose(G, _stage_dt_t(w, dt_mode, dt))
    return loss, g


def gradient_partitioned(chunks_fn, s, d, dt_mode: str = "backward",
                         dt: float = 1.0):
    """``gradient`` over a grid partition; ``chunks_fn()`` returns a fresh
    iterator of ``(G_r, P_r)`` (it is walked twice: forward, then adjoint)."""
    q = waveforms_partitioned(chunks_fn(), s, dt_mode, dt)
    r = q - _f64(d)
    loss = 0.5 * np.sum(r.reshape(r.shape[0], -1) ** 2, axis=1)
    g = None
    for G_r, P_r in chunks_fn():
        g_r = bltt_transpose(G_r, _stage_dt_t(bltt_transpose(P_r, r), dt_mode, dt))
        g = g_r if g is None else g + g_r
    return loss, g


def fft_window(G, P, s, dt_mode: str = "backward", dt: float = 1.0):
    """The 2 Nt-sample stage-2 output window that Alg. 2 forms before its
    final Truncate: with the seafloor motion truncated to Nt samples (Alg. 2
    step 5 of stage 1) and v = D_t m zero-padded to 2 Nt,
    ``q_win[n] = sum_i sum_k P[o,i,k] v_i[n-k]`` for n < 2 Nt, written as
    ``bltt_apply`` on zero-extended arrays.  Its first Nt samples are q.

    A finite-precision FFT evaluation is accurate relative to this window,
    not to its first Nt samples alone: when most of the window's energy lies
    past Nt (signals arriving at the end of the record), the kept head is
    small next to the rounding of the whole window."""
    G, P, s = _f64(G), _f64(P), _f64(s)
    m = bltt_apply(G, s)
    v = _stage_dt(m, dt_mode, dt)
    ext = lambda a: np.concatenate([a, np.zeros_like(a)], axis=-1)
    return bltt_apply(ext(P), ext(v))


def fft_window_adjoint(G, P, r, dt_mode: str = "backward", dt: float = 1.0):
    """Adjoint analogue of ``fft_window``: the full correlation window that
    an FFT evaluation of ``F_G^T D_t^T F_q^T r`` forms before its final
    Truncate, lags -Nt..Nt-1 (index n' = n + Nt):
    ``g_full[j][n] = sum_i sum_k G[i,j,k] u_i[n+k]`` with ``u = D_t^T w`` and
    ``w`` the kept (n >= 0) part of the stage-2 correlation.  Written as
    ``bltt_transpose`` on arrays extended by Nt leading zeros.  Its second
    half (n >= 0) is the gradient."""
    G, P, r = _f64(G), _f64(P), _f64(r)
    Nt = G.shape[2]
    pad_lag = lambda F: np.concatenate([F, np.zeros_like(F)], axis=-1)
    lead = lambda y: np.concatenate([np.zeros_like(y), y], axis=-1)
    w = bltt_transpose(P, r)
    u = _stage_dt_t(w, dt_mode, dt)
    return bltt_transpose(pad_lag(G), lead(u))


def rel_l2(a, ref) -> np.ndarray:
    """Relative L2 error per leading index: ||a - ref||_2 / ||ref||_2."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if a.ndim <= 2:
        return np.linalg.norm(a - ref) / np.linalg.norm(ref)
    d = (a - ref).reshape(a.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(r, axis=1)
