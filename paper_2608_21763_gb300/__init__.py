"""GB300-native source-to-waveform library (arXiv 2608.21763).

Python binding of ``libs2w.so`` (C ABI in ``include/s2w.h``).  This layer only
marshals arguments: every step of the waveform path runs in the library's
CUDA kernels.  PyTorch is used for device memory and streams; numpy arrays
(host memory) are accepted as well and go through the library's host-pointer
path (host -> device copy inside the call).

If ``libs2w.so`` cannot be built or loaded, importing ``lib()`` raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import layout  # noqa: F401  (size arithmetic, no library load)

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

PREC = {"fp32": 0, "bf16": 1, "bf16_hilo": 2, "fp8": 3, "fp32_hilo": 4}
ENGINE = {"auto": 0, "stream": 1, "tensor": 2}
DT_MODE = {"backward": 0, "none": 1}
PAIR = {"auto": 0, "on": 1, "off": 2}
PAIR_NAME = {v: k for k, v in PAIR.items()}
FAULT = {"none": 0, "wait": 1, "oom_load": 2, "launch": 3}
STATUS = {0: "S2W_OK", -1: "S2W_ERR_ARG", -2: "S2W_ERR_OOM", -3: "S2W_ERR_STATE",
          -4: "S2W_ERR_CUDA", -5: "S2W_ERR_TIMEOUT", -6: "S2W_ERR_UNSUPPORTED"}

# every entry point declared in include/s2w.h
EXPORTS = ("s2w_default_opts", "s2w_create", "s2w_destroy", "s2w_operator_bytes",
           "s2w_load_greens", "s2w_load_adjoint", "s2w_load_greens_spectra", "s2w_load_adjoint_spectra",
           "s2w_waveforms", "s2w_waveforms_active", "s2w_waveforms_noalloc",
           "s2w_adjoint", "s2w_misfit_gradient", "s2w_waveforms_graph", "s2w_autotune", "s2w_rfft",
           "s2w_irfft", "s2w_retransform_matrix", "s2w_profile_enable", "s2w_profile_read", "s2w_sync",
           "s2w_last_error", "s2w_status_string")
NUM_STAGES = 8
STAGE_NAMES = ("rfft_slip", "contract_stage1", "retransform", "contract_stage2",
               "reduce_irfft", "copies", "pack_operands", "graph")


class S2WError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * NUM_STAGES),
                ("count", ctypes.c_longlong * NUM_STAGES),
                ("launches", ctypes.c_longlong)]


class Tuning(ctypes.Structure):
    _fields_ = [("from_cache", ctypes.c_int), ("tc_min_batch", ctypes.c_int), ("tc_bsub", ctypes.c_int),
                ("tc_pair", ctypes.c_int), ("tc_s2_chunks", ctypes.c_int), ("probe_batch", ctypes.c_int),
                ("ms_stream_per_rupture", ctypes.c_float), ("form_bsub", ctypes.c_int * 6),
                ("form_pair", ctypes.c_int * 6), ("ms_form", ctypes.c_float * 6),
                ("s2_chunk_cand", ctypes.c_int * 4), ("ms_s2_chunks", ctypes.c_float * 4),
                ("ms_tensor_batch", ctypes.c_float * 7)]


class Opts(ctypes.Structure):
    _fields_ = [("prec_g", ctypes.c_int), ("prec_p", ctypes.c_int),
                ("dt_mode", ctypes.c_int), ("dt", ctypes.c_double),
                ("max_batch", ctypes.c_int), ("device", ctypes.c_int),
                ("engine", ctypes.c_int), ("tc_adjoint", ctypes.c_int),
                ("single_pass", ctypes.c_int), ("tc_pair", ctypes.c_int), ("tc_fp8_act", ctypes.c_int),
                ("tc_bsub", ctypes.c_int), ("tc_s2_chunks", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("fault", ctypes.c_int), ("fault_wait_us", ctypes.c_int)]


def lib_path() -> str:
    return os.path.join(_HERE, "libs2w.so")


def lib():
    """Load libs2w.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import _build
    path = _build.build()
    L = ctypes.CDLL(path)
    V, I, LL, P, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_size_t
    L.s2w_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.s2w_default_opts.restype = None
    L.s2w_create.argtypes = [I, I, I, I, ctypes.POINTER(Opts), ctypes.POINTER(V)]
    L.s2w_destroy.argtypes = [V]
    L.s2w_operator_bytes.argtypes = [V, ctypes.POINTER(SZ), ctypes.POINTER(SZ)]
    L.s2w_load_greens.argtypes = [V, I, I, P, V]
    L.s2w_load_adjoint.argtypes = [V, I, I, P, V]
    L.s2w_load_greens_spectra.argtypes = [V, I, I, P, V]
    L.s2w_load_adjoint_spectra.argtypes = [V, I, I, P, V]
    L.s2w_waveforms.argtypes = [V, P, I, P, P, V]
    L.s2w_waveforms_active.argtypes = [V, P, P, I, P, P, V]
    L.s2w_waveforms_noalloc.argtypes = [V, P, P, V]
    L.s2w_adjoint.argtypes = [V, P, I, P, V]
    L.s2w_misfit_gradient.argtypes = [V, P, P, I, P, P, V]
    L.s2w_waveforms_graph.argtypes = [V, P, I, P, V]
    L.s2w_autotune.argtypes = [V, I, ctypes.POINTER(Tuning), V]
    L.s2w_rfft.argtypes = [V, P, LL, P, V]
    L.s2w_irfft.argtypes = [V, P, LL, P, V]
    L.s2w_retransform_matrix.argtypes = [I, I, ctypes.c_double, I, ctypes.POINTER(ctypes.c_double)]
    L.s2w_profile_enable.argtypes = [V, I]
    L.s2w_profile_read.argtypes = [V, ctypes.POINTER(Profile)]
    L.s2w_sync.argtypes = [V]
    L.s2w_last_error.argtypes = [V]
    L.s2w_last_error.restype = ctypes.c_char_p
    L.s2w_status_string.argtypes = [I]
    L.s2w_status_string.restype = ctypes.c_char_p
    for name in ("s2w_create", "s2w_destroy", "s2w_operator_bytes", "s2w_load_greens",
                 "s2w_load_adjoint", "s2w_load_greens_spectra", "s2w_load_adjoint_spectra", "s2w_waveforms_active", "s2w_waveforms", "s2w_waveforms_noalloc", "s2w_adjoint", "s2w_misfit_gradient", "s2w_waveforms_graph",
                 "s2w_autotune", "s2w_rfft",
                 "s2w_irfft", "s2w_sync",
                 "s2w_profile_enable", "s2w_profile_read"):
        getattr(L, name).restype = I
    _lib = L
    return L


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous float32)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags.c_contiguous, "need C-contiguous float32"
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        assert a.dtype == torch.float32 and a.is_contiguous(), "need contiguous float32"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as_float(a):
    """complex64 array / tensor viewed as interleaved float32 (no copy)."""
    if isinstance(a, np.ndarray):
        assert a.dtype == np.complex64 and a.flags.c_contiguous, "need C-contiguous complex64"
        return a.view(np.float32)
    import torch
    assert a.dtype == torch.complex64 and a.is_contiguous(), "need contiguous complex64"
    return torch.view_as_real(a)


def _stream(stream, *arrays):
    """cudaStream_t for the call: explicit, else torch's current stream when a
    CUDA tensor is involved, else the legacy default stream."""
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


class Context:
    """One resident operator pair (Ghat, Phat) on one GPU.

    ``Context(Ns, Ng, No, Nt, prec_g="fp32", prec_p="fp32", dt_mode="backward",
    dt=1.0, max_batch=1, device=0, engine="auto", ...)``; load the operators with
    ``load_greens``/``load_adjoint`` (time-domain responses, any row chunking),
    then call ``waveforms``.  The keyword options mirror ``s2w_opts``
    (``include/s2w.h``); ``tune_cache`` is a file path, ``fault`` one of
    ``FAULT``'s names (a test hook).
    """

    def __init__(self, Ns, Ng, No, Nt, prec_g="fp32", prec_p="fp32",
                 dt_mode="backward", dt=1.0, max_batch=1, device=0, engine="auto",
                 tc_adjoint=False, single_pass=False, tc_pair="auto", tc_fp8_act=None, tc_bsub=0,
                 tc_s2_chunks=0, tune_cache=None, fault="none", fault_wait_us=5000):
        L = lib()
        o = Opts()
        L.s2w_default_opts(ctypes.byref(o))
        o.prec_g, o.prec_p = PREC[prec_g], PREC[prec_p]
        o.dt_mode, o.dt = DT_MODE[dt_mode], float(dt)
        o.max_batch, o.device = int(max_batch), int(device)
        o.engine = ENGINE[engine]
        o.tc_adjoint = int(bool(tc_adjoint))
        o.single_pass = int(bool(single_pass))
        o.tc_pair = PAIR[tc_pair]
        if tc_fp8_act is not None:  # 0 / False: FP16, 1 / True: e4m3, 2: hi + lo e4m3 (library default)
            o.tc_fp8_act = int(tc_fp8_act)
        o.tc_bsub = int(tc_bsub)
        o.tc_s2_chunks = int(tc_s2_chunks)
        cache = None if tune_cache is None else os.fsencode(tune_cache)
        o.tune_cache = cache
        o.fault = FAULT[fault]
        o.fault_wait_us = int(fault_wait_us)
        h = ctypes.c_void_p()
        st = L.s2w_create(Ns, Ng, No, Nt, ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise S2WError(st, L.s2w_last_error(None).decode())
        self._h = h
        self.Ns, self.Ng, self.No, self.Nt = Ns, Ng, No, Nt
        self.Nb = 2 * Nt + 1 if single_pass else Nt + 1
        self.prec_g, self.prec_p, self.max_batch, self.device = prec_g, prec_p, max_batch, device
        self.engine = engine

    def _check(self, st):
        if st != 0:
            raise S2WError(st, lib().s2w_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().s2w_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def operator_bytes(self):
        g, p = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(lib().s2w_operator_bytes(self._h, ctypes.byref(g), ctypes.byref(p)))
        return g.value, p.value

    def load_greens(self, g0, G, stream=None):
        """G: float32 [ng][Ns][Nt] time-domain rows g0..g0+ng-1 (host or device)."""
        assert G.shape[1:] == (self.Ns, self.Nt), G.shape
        self._check(lib().s2w_load_greens(self._h, int(g0), int(G.shape[0]), _ptr(G),
                                          _stream(stream, G)))

    def load_adjoint(self, g0, P, stream=None):
        """P: float32 [No][ng][Nt] time-domain columns g0..g0+ng-1."""
        assert P.shape[0] == self.No and P.shape[2] == self.Nt, P.shape
        self._check(lib().s2w_load_adjoint(self._h, int(g0), int(P.shape[1]), _ptr(P),
                                           _stream(stream, P)))

    def load_greens_spectra(self, g0, Ghat, stream=None):
        """Ghat: complex64 [Nt+1][ng][Ns], the zero-padded DFTs (length 2 Nt) of
        rows g0..g0+ng-1 of the stage-1 blocks (host or device)."""
        assert Ghat.shape[0] == self.Nb and Ghat.shape[2] == self.Ns, Ghat.shape
        self._check(lib().s2w_load_greens_spectra(self._h, int(g0), int(Ghat.shape[1]), _ptr(_as_float(Ghat)),
                                                  _stream(stream, Ghat)))

    def load_adjoint_spectra(self, g0, Phat, stream=None):
        """Phat: complex64 [Nt+1][No][ng], the zero-padded DFTs of columns
        g0..g0+ng-1 of the stage-2 blocks."""
        assert Phat.shape[0] == self.Nb and Phat.shape[1] == self.No, Phat.shape
        self._check(lib().s2w_load_adjoint_spectra(self._h, int(g0), int(Phat.shape[2]), _ptr(_as_float(Phat)),
                                                   _stream(stream, Phat)))

    def waveforms(self, slip, q=None, seafloor=None, stream=None):
        """q[b] = F_q D_t F_G slip[b].  slip: float32 [B][Ns][Nt] (torch CUDA
        tensor, or numpy for the host path).  Returns q (allocated like slip
        when not given)."""
        B = slip.shape[0]
        assert slip.shape[1:] == (self.Ns, self.Nt), slip.shape
        if q is None:
            if isinstance(slip, np.ndarray):
                q = np.empty((B, self.No, self.Nt), np.float32)
            else:
                import torch
                q = torch.empty((B, self.No, self.Nt), dtype=torch.float32, device=slip.device)
        self._check(lib().s2w_waveforms(self._h, _ptr(slip), int(B), _ptr(q), _ptr(seafloor),
                                        _stream(stream, slip, q, seafloor)))
        return q

    def adjoint(self, r, grad=None, stream=None):
        """grad[b] = F_G^T D_t^T F_q^T r[b]: the gradient of 0.5 ||q - d||^2
        with respect to slip when r = q - d.  r: float32 [B][No][Nt]."""
        B = r.shape[0]
        assert r.shape[1:] == (self.No, self.Nt), r.shape
        if grad is None:
            if isinstance(r, np.ndarray):
                grad = np.empty((B, self.Ns, self.Nt), np.float32)
            else:
                import torch
                grad = torch.empty((B, self.Ns, self.Nt), dtype=torch.float32, device=r.device)
        self._check(lib().s2w_adjoint(self._h, _ptr(r), int(B), _ptr(grad), _stream(stream, r, grad)))
        return grad

    def waveforms_active(self, slip, active_len, q=None, seafloor=None, stream=None):
        """s2w_waveforms with per-rupture active durations: slip[b][:, n] for
        n >= active_len[b] is taken as zero (never read)."""
        B = slip.shape[0]
        lens = np.ascontiguousarray(np.asarray(active_len, dtype=np.int32))
        assert lens.shape == (B,), lens.shape
        if q is None:
            if isinstance(slip, np.ndarray):
                q = np.empty((B, self.No, self.Nt), np.float32)
            else:
                import torch
                q = torch.empty((B, self.No, self.Nt), dtype=torch.float32, device=slip.device)
        self._check(lib().s2w_waveforms_active(self._h, _ptr(slip), lens.ctypes.data, int(B), _ptr(q),
                                               _ptr(seafloor), _stream(stream, slip, q, seafloor)))
        return q

    def waveforms_graph(self, slip, q, stream=None):
        """s2w_waveforms as a replayed CUDA graph (device tensors only; the
        first call with these buffers captures, later calls replay)."""
        self._check(lib().s2w_waveforms_graph(self._h, _ptr(slip), int(slip.shape[0]), _ptr(q),
                                              _stream(stream, slip, q)))
        return q

    def autotune(self, B, stream=None):
        """Choose the tensor engine's schedule (GEMM form, stage-2 chunk
        count, AUTO batch threshold) by timing it on the loaded operators, or
        from the context's tune cache.  Returns the choices and timings."""
        t = Tuning()
        st = stream
        if st is None:
            import torch
            st = torch.cuda.current_stream(self.device)
        self._check(lib().s2w_autotune(self._h, int(B), ctypes.byref(t), _stream(st)))
        forms = [{"bsub": t.form_bsub[k], "pair": PAIR_NAME[t.form_pair[k]], "ms": t.ms_form[k]}
                 for k in range(6) if t.form_bsub[k] > 0]
        chunks = [{"chunks": t.s2_chunk_cand[k], "ms": t.ms_s2_chunks[k]} for k in range(4) if t.s2_chunk_cand[k] > 0]
        return {"from_cache": bool(t.from_cache), "tc_min_batch": t.tc_min_batch, "tc_bsub": t.tc_bsub,
                "tc_pair": PAIR_NAME[t.tc_pair], "tc_s2_chunks": t.tc_s2_chunks, "probe_batch": t.probe_batch,
                "ms_stream_per_rupture": t.ms_stream_per_rupture, "forms": forms, "s2_chunks": chunks,
                "ms_tensor_batch": list(t.ms_tensor_batch)}

    def misfit_gradient(self, slip, d, grad=None, loss=None, stream=None):
        """Gradient of 0.5 ||q(slip[b]) - d[b]||^2 per rupture; returns
        (grad [B][Ns][Nt], loss [B])."""
        B = slip.shape[0]
        assert slip.shape[1:] == (self.Ns, self.Nt) and d.shape == (B, self.No, self.Nt)
        if isinstance(slip, np.ndarray):
            grad = np.empty((B, self.Ns, self.Nt), np.float32) if grad is None else grad
            loss = np.empty((B,), np.float32) if loss is None else loss
        else:
            import torch
            if grad is None:
                grad = torch.empty((B, self.Ns, self.Nt), dtype=torch.float32, device=slip.device)
            if loss is None:
                loss = torch.empty((B,), dtype=torch.float32, device=grad.device)
        self._check(lib().s2w_misfit_gradient(self._h, _ptr(slip), _ptr(d), int(B), _ptr(grad), _ptr(loss),
                                              _stream(stream, slip, d, grad)))
        return grad, loss

    def rfft(self, x, X=None, stream=None):
        """Zero-padded real FFT of device rows x [..., Nt] -> complex64 [..., Nt+1]."""
        import torch
        rows = x.numel() // self.Nt
        if X is None:
            X = torch.empty(x.shape[:-1] + (self.Nb,), dtype=torch.complex64, device=x.device)
        self._check(lib().s2w_rfft(self._h, _ptr(x), rows, X.data_ptr(), _stream(stream, x)))
        return X

    def irfft(self, X, x=None, stream=None):
        """First Nt samples of the length-2Nt real IFFT of device bins X [..., Nt+1]."""
        import torch
        rows = X.numel() // self.Nb
        if x is None:
            x = torch.empty(X.shape[:-1] + (self.Nt,), dtype=torch.float32, device=X.device)
        self._check(lib().s2w_irfft(self._h, X.data_ptr(), rows, _ptr(x), _stream(stream, x)))
        return x

    def profile_enable(self, on=True):
        self._check(lib().s2w_profile_enable(self._h, int(bool(on))))

    def profile_read(self):
        """Per-stage {name: (ms, count)} since profile_enable, and the total
        number of kernel launches made by the library."""
        p = Profile()
        self._check(lib().s2w_profile_read(self._h, ctypes.byref(p)))
        stages = {STAGE_NAMES[i]: (p.ms[i], p.count[i]) for i in range(NUM_STAGES)}
        return stages, p.launches

    def sync(self):
        self._check(lib().s2w_sync(self._h))
