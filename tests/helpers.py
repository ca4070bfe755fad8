"""Shared test helpers: build a library context from a synthetic geometry and
compute the FP64 oracle reference for the same inputs."""
import numpy as np

import oracle


def make_context(s2w, geom, Nt, prec_g="fp32", prec_p="fp32", dt_mode="backward",
                 max_batch=1, chunk=4096, order=None):
    """Context with both operators loaded from the generator, in row chunks
    (optionally in a permuted chunk order)."""
    Ng = geom.Ng
    ctx = s2w.Context(geom.Ns, Ng, geom.No, Nt, prec_g=prec_g, prec_p=prec_p,
                      dt_mode=dt_mode, max_batch=max_batch)
    starts = list(range(0, Ng, chunk))
    if order is not None:
        starts = [starts[i] for i in order]
    for g0 in starts:
        g1 = min(Ng, g0 + chunk)
        ctx.load_greens(g0, geom.greens_rows(g0, g1, Nt, np.float32))
        ctx.load_adjoint(g0, np.ascontiguousarray(geom.adjoint_cols(g0, g1, Nt, np.float32)))
    return ctx


def oracle_reference(geom, Nt, slip, dt_mode="backward", chunk=1024, seafloor=False):
    """FP64 oracle q (and optionally m) through Eq. (distributed-composition)
    over grid chunks, with operators regenerated in FP64."""
    if seafloor:
        G = geom.greens_rows(0, geom.Ng, Nt)
        P = geom.adjoint_cols(0, geom.Ng, Nt)
        return oracle.waveforms(G, P, slip, dt_mode=dt_mode, return_seafloor=True)

    def chunks():
        for g0 in range(0, geom.Ng, chunk):
            g1 = min(geom.Ng, g0 + chunk)
            yield geom.greens_rows(g0, g1, Nt), geom.adjoint_cols(g0, g1, Nt)
    return oracle.waveforms_partitioned(chunks(), slip, dt_mode=dt_mode)


def rel_l2(a, ref):
    return oracle.rel_l2(np.asarray(a, dtype=np.float64), ref)
