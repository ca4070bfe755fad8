"""Write the rounding model's error for the tensor engine's BF16 and split
(hi/lo) paths on the sampled ruptures of the full-size batched workload
(963 x 60,000 x 64 x 256), from which the full-size parity test derives
those paths' bars (test infrastructure).

Calls only the rounding model (``tests/error_model.py``: the FFT pipeline of
Alg. 2 in FP64 with the roundings each path makes) and the seeded generator
``synth/``; nothing here touches the CUDA library.  For these paths every
rounding is per element or per signal, so the model runs over grid chunks
(in worker processes) and sums their stage-2 spectra.  Operator and slip
spectra are the zero-padded DFT as an FP64 product with the cos / sin
matrices of the bins.

The sampled ruptures and their draw are those of ``make_full_size_oracle.py``
(same indices, same checksums).  Output ``model_<workload>.npz``: q_exact
[n][No][Nt] (the model without rounding, which a CPU test compares with the
oracle's waveforms) and, per path, the relative L2 distance of the path's
modelled waveforms from q_exact, per rupture.

Run:  python tests/golden/make_full_size_model.py batched   (about half an hour on 8 cores)
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.dirname(HERE), HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import error_model  # noqa: E402
import synth  # noqa: E402
from make_full_size_oracle import SAMPLES, checksums, draw  # noqa: E402

PATHS = {"batched": ("tensor_bf16", "tensor_split")}


def dft_matrices(Nt: int):
    """cos and sin of the zero-padded length-2Nt DFT, [Nt][Nt + 1], angles
    reduced exactly as integers (n k mod 2Nt)."""
    L = 2 * Nt
    nk = np.outer(np.arange(Nt), np.arange(Nt + 1)) % L
    th = 2.0 * np.pi * nk / L
    return np.cos(th), np.sin(th)


def spectra(x: np.ndarray, C: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Bins 0..Nt of the zero-padded DFT of x [..][Nt] (FP64), shaped
    [..][Nb] but stored bins-outer, the layout of the model's per-bin
    products."""
    flat = x.reshape(-1, x.shape[-1]).T
    z = np.empty((C.shape[1], flat.shape[1]), np.complex128)  # [Nb][..]
    z.real = C.T @ flat
    z.imag = S.T @ flat
    np.negative(z.imag, out=z.imag)
    return z.reshape((C.shape[1],) + x.shape[:-1]).transpose(tuple(range(1, x.ndim)) + (0,))


_W = {}


def _init(name: str) -> None:
    wl, geom, slip, idx = draw(name)
    C, S = dft_matrices(wl.Nt)
    _W.update(name=name, wl=wl, geom=geom, C=C, S=S, T=error_model.retransform_matrix(wl.Nt),
              sh=spectra(slip[idx].astype(np.float64), C, S))


def _chunk(rows):
    """Stage-2 spectra of every path over grid rows [g0, g1)."""
    g0, g1 = rows
    w = _W
    Gh = spectra(synth.response(w["geom"].grid[g0:g1], w["geom"].sub, w["wl"].Nt, synth.GREEN_VEL_KMS),
                 w["C"], w["S"])
    Ph = spectra(w["geom"].adjoint_cols(g0, g1, w["wl"].Nt), w["C"], w["S"])
    return {p: error_model.model_spectra(Gh, Ph, w["sh"], p, w["T"]) for p in ("exact",) + PATHS[w["name"]]}


def make(name: str, chunk: int = 128, workers: int = 8) -> None:
    wl, _, slip, idx = draw(name)
    Nt, L = wl.Nt, 2 * wl.Nt
    paths = ("exact",) + PATHS[name]
    qh = {p: np.zeros((len(idx), wl.No, Nt + 1), np.complex128) for p in paths}
    jobs = [(g0, min(wl.Ng, g0 + chunk)) for g0 in range(0, wl.Ng, chunk)]
    t0 = time.time()
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"  # one BLAS thread per worker process
    with mp.get_context("spawn").Pool(workers, initializer=_init, initargs=(name,)) as pool:
        for n, part in enumerate(pool.imap_unordered(_chunk, jobs)):
            for p in paths:
                qh[p] += part[p]
            if n % 50 == 0:
                print(f"{name}: {n + 1} of {len(jobs)} chunks at {time.time() - t0:.0f} s", flush=True)
    q = {p: np.fft.irfft(qh[p], L, axis=-1)[..., :Nt] for p in paths}
    ref = np.linalg.norm(q["exact"].reshape(len(idx), -1), axis=1)
    rel = {f"rel_{p}": np.linalg.norm((q[p] - q["exact"]).reshape(len(idx), -1), axis=1) / ref
           for p in PATHS[name]}
    for k, v in rel.items():
        print(f"{name}: {k} max {v.max():.3g} median {np.median(v):.3g}", flush=True)
    np.savez_compressed(os.path.join(HERE, f"model_{name}.npz"), q_exact=q["exact"], index=np.array(idx),
                        draw=np.array(SAMPLES[name][:2]), checksum=checksums(slip[idx]), **rel)


if __name__ == "__main__":
    for n in sys.argv[1:] or list(PATHS):
        make(n)
