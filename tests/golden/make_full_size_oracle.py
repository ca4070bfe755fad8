"""Write the FP64 oracle's waveforms for sampled ruptures of the full-size
workloads, for the full-size parity tests and bench.py's accuracy block.

Calls only ``oracle/`` (the direct FP64 time-domain convolution) and the
seeded input generator ``synth/``; nothing here touches the CUDA library.

For each workload the ruptures are generated exactly as ``bench.py`` does
(one draw of ``pool * B`` ruptures; batch 0 is the first B), and the sampled
ruptures of batch 0 are evaluated with ``oracle.waveforms_partitioned`` over
grid chunks (Eq. distributed-composition).  Each rupture's subfaults whose
slip rate is zero at every step are left out of its sums: their terms are
exact zeros, so the sums are unchanged.  Output: ``oracle_<workload>.npz``
with q [n][No][Nt] (float64), the rupture indices within batch 0, the draw
size, and per-rupture slip checksums (sum |s| and sum s^2) that users of the
file compare against their own draw.

Run:  python tests/golden/make_full_size_oracle.py plain batched largest
(about 5 / 20 / 50 minutes on 8 cores).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

# workload -> (ruptures per batch, batches drawn, sampled indices of batch 0)
SAMPLES = {
    "plain": (1, 8, list(range(8))),           # bench: B = 1, a pool of 8 inputs; every one of them
    "batched": (256, 2, list(range(0, 256, 16))),
    "largest": (1024, 2, list(range(0, 1024, 64))),
}


def path(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.npz")


def draw(name: str):
    """The ruptures as bench.py draws them (float32, as the library gets
    them), and the sampled ones."""
    B, pool, idx = SAMPLES[name]
    wl = synth.WORKLOADS[name]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=pool * B).astype(np.float32)
    return wl, geom, slip, idx


def checksums(s: np.ndarray) -> np.ndarray:
    s = s.astype(np.float64)
    return np.stack([np.abs(s).sum(axis=(-2, -1)), (s * s).sum(axis=(-2, -1))], axis=-1)


def make(name: str, chunk: int = 2048) -> None:
    wl, geom, slip, idx = draw(name)
    q = np.zeros((len(idx), wl.No, wl.Nt))
    t0 = time.time()
    for k, b in enumerate(idx):
        s = slip[b].astype(np.float64)
        act = np.nonzero(np.any(s != 0, axis=1))[0]

        def chunks():
            for g0 in range(0, wl.Ng, chunk):
                g1 = min(wl.Ng, g0 + chunk)
                G = synth.response(geom.grid[g0:g1], geom.sub[act], wl.Nt, synth.GREEN_VEL_KMS)
                yield G, geom.adjoint_cols(g0, g1, wl.Nt)
        if act.size:
            q[k] = oracle.waveforms_partitioned(chunks(), s[act][None])[0]
        print(f"{name}: rupture {b} ({act.size} active subfaults) done at {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(path(name), q=q, index=np.array(idx), draw=np.array(SAMPLES[name][:2]),
                        checksum=checksums(slip[idx]), workload=np.array(name))


def load(name: str):
    """(q_ref, indices) of a workload's file, or None when it is absent."""
    p = path(name)
    if not os.path.exists(p):
        return None
    d = np.load(p)
    return d["q"], [int(i) for i in d["index"]], d["checksum"]


if __name__ == "__main__":
    for n in sys.argv[1:] or list(SAMPLES):
        make(n)
