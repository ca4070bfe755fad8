"""Write the FP64 oracle's misfit gradient for sampled ruptures of the
full-size differentiation workload (963 x 40,000 x 64 x 256, 64 ruptures per
call), for the full-size gradient parity test (test infrastructure).

Calls only ``oracle/`` (the direct FP64 time-domain convolution and its
transpose) and the seeded generator ``synth/``; nothing here touches the
CUDA library.  The ruptures are drawn as ``bench.py`` draws them (``pool * B``
ruptures, batch 0 first).  For each sampled rupture of batch 0 the slip
where the gradient is taken is s = float32(0.9 * s_true), as in the bench;
the targets are d = float32(q(s) / 0.9 + 5 % noise) (``synth.noisy_targets``
with seed 1000 + rupture index), q(s) the oracle's waveforms; then the
misfit 0.5 ||q(s) - d||^2 and its gradient F_G^T D_t^T F_q^T (q(s) - d) are
evaluated over grid chunks (Eq. distributed-composition and its
transpose).  Output ``gradient_<workload>.npz``: the rupture indices, the
draw, slip checksums of s_true, q [n][No][Nt] (float64, the oracle's
waveforms at s), d [n][No][Nt] (float32, as the library receives it), loss
[n] and g [n][Ns][Nt] (float64).

Run:  python tests/golden/make_full_size_gradient.py   (about 25 minutes on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import synth  # noqa: E402
from make_full_size_oracle import checksums  # noqa: E402

NAME = "gradient"
POOL = 2                     # bench.py draws pool * B ruptures for B > 16
INDEX = [0, 16, 32, 48]      # sampled ruptures of batch 0


def make(chunk: int = 512) -> None:
    wl = synth.WORKLOADS[NAME]
    geom = wl.geometry_obj()
    s_true = wl.slip(geom, B=POOL * wl.B).astype(np.float32)[INDEX]
    s = (s_true * np.float32(0.9)).astype(np.float32)
    s64 = s.astype(np.float64)
    t0 = time.time()

    def chunks():
        for g0 in range(0, wl.Ng, chunk):
            g1 = min(wl.Ng, g0 + chunk)
            yield (synth.response(geom.grid[g0:g1], geom.sub, wl.Nt, synth.GREEN_VEL_KMS),
                   geom.adjoint_cols(g0, g1, wl.Nt))

    q = oracle.waveforms_partitioned(chunks(), s64)
    print(f"forward done at {time.time() - t0:.0f} s", flush=True)
    d = np.stack([synth.noisy_targets(1000 + b, q[k:k + 1] / 0.9)[0] for k, b in enumerate(INDEX)])
    d = d.astype(np.float32)
    r = q - d.astype(np.float64)
    loss = 0.5 * np.sum(r.reshape(len(INDEX), -1) ** 2, axis=1)
    g = None
    for G_r, P_r in chunks():
        g_r = oracle.bltt_transpose(G_r, oracle.dt_transpose(oracle.bltt_transpose(P_r, r)))
        g = g_r if g is None else g + g_r
    print(f"adjoint done at {time.time() - t0:.0f} s; loss {loss}", flush=True)
    np.savez_compressed(os.path.join(HERE, f"gradient_{NAME}.npz"), index=np.array(INDEX),
                        draw=np.array([wl.B, POOL]), checksum=checksums(s_true), q=q, d=d, loss=loss, g=g)


if __name__ == "__main__":
    make()
