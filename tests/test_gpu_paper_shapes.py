"""The paper's per-GPU shapes (Table I, Sec. III-A) and its comparison method.

f3: the weak-scaling shape (480 subfaults x 37,758 grid points x 32
observations) and the 8-GPU strong-scaling shape (60 x 302,066 x 4; with 60
subfaults the stage-1 rows are short and the lane-group form of the stream
kernel runs), full size, one rupture, against the FP64 oracle on whole
waveforms of sampled observations.  P[o, i, :] is exactly zero in FP64 for
grid points beyond ~69 km of observation o (the Ricker envelope underflows),
so the oracle sums exactly the terms of the rows where it is not.

f4: the paper's direct baseline, two conv_transpose1d passes with D_t
between (bench.py --impl torch_conv), on the tiny workload against the
oracle (FP64 and FP32, TF32 off).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_21763_gb300 as s2w  # noqa: E402


def oracle_observation(wl, geom, slip0, o):
    """q_o [Nt] of rupture slip0 [Ns][Nt] through the rows where P[o] != 0."""
    Po = synth.response(geom.obs[o:o + 1], geom.grid, wl.Nt, synth.ADJ_VEL_KMS)[0]
    idx = np.nonzero(np.any(Po != 0, axis=1))[0]
    G = synth.response(geom.grid[idx], geom.sub, wl.Nt, synth.GREEN_VEL_KMS)
    m = oracle.bltt_apply(G, slip0[None].astype(np.float64))
    return oracle.bltt_apply(Po[idx][None], oracle.dt_apply(m))[0, 0], idx.size


@pytest.mark.parametrize("name,prec", [("paper_weak", "fp32"), ("paper_strong8", "fp32"),
                                       ("paper_strong8", "fp32_hilo")])
def test_paper_per_gpu_shapes(name, prec):
    wl = synth.WORKLOADS[name]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=1).astype(np.float32)
    ctx = s2w.Context(wl.Ns, wl.Ng, wl.No, wl.Nt, prec_g=prec, prec_p=prec)
    for g0 in range(0, wl.Ng, 8192):
        g1 = min(wl.Ng, g0 + 8192)
        ctx.load_greens(g0, geom.greens_rows(g0, g1, wl.Nt, np.float32))
        ctx.load_adjoint(g0, geom.adjoint_cols(g0, g1, wl.Nt, np.float32))
    q = ctx.waveforms(torch.tensor(slip, device="cuda")).cpu().numpy()[0].astype(np.float64)
    ctx.sync()
    ctx.close()
    rels = []
    for o in (0, wl.No - 1):
        q_ref, rows = oracle_observation(wl, geom, slip[0], o)
        rels.append(np.linalg.norm(q[o] - q_ref) / np.linalg.norm(q_ref))
        print(f"{name} {prec}: observation {o} ({rows} rows with P != 0): rel-L2 {rels[-1]:.3g}")
    assert max(rels) <= 1e-5, rels


@pytest.mark.parametrize("dtype,bar", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_torch_conv_baseline_on_the_tiny_workload(dtype, bar):
    import bench
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    slip = wl.slip(geom, B=3)
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    td = torch.float64 if dtype == "fp64" else torch.float32
    W1 = torch.tensor(G, dtype=td, device="cuda").permute(1, 0, 2).contiguous()
    W2 = torch.tensor(P, dtype=td, device="cuda").permute(1, 0, 2).contiguous()
    x = torch.tensor(slip, dtype=td, device="cuda")
    # a tile smaller than the grid: the tiled sums are exercised
    q = bench.torch_conv_forward(W1, W2, x, 256).cpu().numpy()
    assert bench.torch_conv_tile(wl.Ns, wl.Ng, wl.No, wl.Nt, 3) == 1024
    s = slip.astype(np.float32).astype(np.float64) if dtype == "fp32" else slip
    q_ref = oracle.waveforms(G, P, s)
    rel = np.linalg.norm((q - q_ref).reshape(3, -1), axis=1) / np.linalg.norm(q_ref.reshape(3, -1), axis=1)
    print(f"conv_transpose1d {dtype}: rel-L2 {rel}")
    assert np.all(rel <= bar), rel
