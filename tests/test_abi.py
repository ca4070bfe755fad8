"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/s2w.h declares.  No kernel is launched."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2608_21763_gb300 as s2w

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "s2w.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(s2w_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_binding_exports():
    assert declared() == sorted(s2w.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = s2w.lib()._name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared() if f not in syms]
    assert not missing, missing


def test_library_is_built_for_sm_103a_only():
    """Every object is compiled with exactly one -gencode, sm_103a's, and
    the link uses the same one."""
    from paper_2608_21763_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    flags = _build.NVCC_FLAGS
    assert flags[:2] == _build.ARCH
    assert flags.count("-gencode") == 1 and not any(f.startswith("-arch") for f in flags)


def test_status_strings_and_default_opts():
    L = s2w.lib()
    assert L.s2w_status_string(0) == b"S2W_OK"
    assert L.s2w_status_string(-5) == b"S2W_ERR_TIMEOUT"
    o = s2w.Opts()
    L.s2w_default_opts(ctypes.byref(o))
    assert (o.prec_g, o.prec_p, o.dt_mode, o.dt, o.max_batch, o.device) == (0, 0, 0, 1.0, 1, 0)


def test_create_rejects_bad_shapes_before_touching_a_device():
    L = s2w.lib()
    h = ctypes.c_void_p()
    assert L.s2w_create(16, 64, 4, 48, None, ctypes.byref(h)) == -6   # Nt unsupported
    assert h.value is None
    assert b"Nt=48" in L.s2w_last_error(None)
    assert L.s2w_create(0, 64, 4, 32, None, ctypes.byref(h)) == -1
    assert L.s2w_create(2000, 64, 4, 32, None, ctypes.byref(h)) == -6  # Ns > 1024


def test_opts_layout_matches_the_header():
    """s2w_default_opts writes every field of s2w_opts: written into a buffer
    larger than the binding's Opts, it must stop exactly at Opts' end (a
    field missing from the binding would be written past it) and leave the
    defaults of the last fields (two-SM tiles: library choice; FP8 operators
    take hi + lo e4m3 activations; library sub-batch and stage-2 chunking;
    no tune cache; no injected fault)."""
    L = s2w.lib()
    n = ctypes.sizeof(s2w.Opts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    L.s2w_default_opts(ctypes.cast(buf, ctypes.POINTER(s2w.Opts)))
    assert all(b == 0xAB for b in buf[n:])
    o = s2w.Opts.from_buffer(buf)
    assert (o.tc_adjoint, o.single_pass, o.tc_pair, o.tc_fp8_act) == (0, 0, 0, 2)
    assert (o.tc_bsub, o.tc_s2_chunks, o.tune_cache, o.fault, o.fault_wait_us) == (0, 0, None, 0, 5000)


def test_create_rejects_bad_options_before_touching_a_device():
    L = s2w.lib()
    h = ctypes.c_void_p()
    for field, value, prec_g in [("tc_pair", 3, 1), ("tc_pair", -1, 1), ("tc_fp8_act", 3, 3),
                                 ("tc_fp8_act", 1, 1), ("tc_fp8_act", 1, 0), ("tc_bsub", 64, 1),
                                 ("tc_bsub", -1, 1), ("tc_s2_chunks", 17, 1), ("tc_s2_chunks", -1, 1),
                                 ("fault", 9, 0)]:
        o = s2w.Opts()
        L.s2w_default_opts(ctypes.byref(o))
        o.prec_g = prec_g
        setattr(o, field, value)
        assert L.s2w_create(16, 64, 4, 32, ctypes.byref(o), ctypes.byref(h)) == -1, (field, value, prec_g)
        assert h.value is None
        assert field.encode() in L.s2w_last_error(None)


def test_null_context_is_an_argument_error():
    L = s2w.lib()
    assert L.s2w_waveforms(None, None, 1, None, None, None) == -1
    assert L.s2w_sync(None) == -1
    assert L.s2w_destroy(None) == 0


def test_split_passes_take_at_most_128_ruptures():
    L = s2w.lib()
    h = ctypes.c_void_p()
    o = s2w.Opts()
    L.s2w_default_opts(ctypes.byref(o))
    o.prec_g, o.tc_bsub = s2w.PREC["bf16_hilo"], 256
    assert L.s2w_create(16, 64, 4, 32, ctypes.byref(o), ctypes.byref(h)) == -6
    assert b"tc_bsub=256" in L.s2w_last_error(None)


def test_fault_environment_variable_is_checked(monkeypatch):
    """S2W_FAULT selects a test hook at s2w_create; an unknown name is an
    argument error before any device is touched."""
    L = s2w.lib()
    h = ctypes.c_void_p()
    monkeypatch.setenv("S2W_FAULT", "segfault")
    assert L.s2w_create(16, 64, 4, 32, None, ctypes.byref(h)) == -1
    assert b"S2W_FAULT=segfault" in L.s2w_last_error(None)
    o = s2w.Opts()
    L.s2w_default_opts(ctypes.byref(o))
    o.fault, o.fault_wait_us = s2w.FAULT["wait"], 0
    monkeypatch.delenv("S2W_FAULT")
    assert L.s2w_create(16, 64, 4, 32, ctypes.byref(o), ctypes.byref(h)) == -1
    assert b"fault_wait_us" in L.s2w_last_error(None)
