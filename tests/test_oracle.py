"""Pins for the FP64 oracle: each function is checked against something other
than itself (a dense block-Toeplitz matrix, numpy's FFT, closed forms,
invariants of LTI maps, the adjoint identity), so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one test."""
import numpy as np
import pytest

import oracle
import synth


def dense_bltt(F):
    """The stacked block lower-triangular Toeplitz matrix of Sec. II-B.3,
    BLTT(F_0..F_{Nt-1}), acting on x = [x_0; x_1; ...; x_{Nt-1}] with
    x_n in R^{Nin}: block (n, n') = F_{n-n'} for n >= n', else 0."""
    nout, nin, nt = F.shape
    M = np.zeros((nt * nout, nt * nin))
    for n in range(nt):
        for n2 in range(n + 1):
            M[n * nout:(n + 1) * nout, n2 * nin:(n2 + 1) * nin] = F[:, :, n - n2]
    return M


def stack_time(x):
    """[C][Nt] -> time-stacked vector [x_0; x_1; ...] (block n = x[:, n])."""
    return x.T.reshape(-1)


def unstack_time(v, c):
    return v.reshape(-1, c).T


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(7)
    Ns, Ng, No, Nt = 3, 5, 2, 9
    G = rng.standard_normal((Ng, Ns, Nt))
    P = rng.standard_normal((No, Ng, Nt))
    s = rng.standard_normal((Ns, Nt))
    return G, P, s


def test_bltt_apply_matches_dense_block_toeplitz(small):
    G, P, s = small
    for F, x in ((G, s), (P, rng_like(P, 1))):
        y = oracle.bltt_apply(F, x)
        y_ref = unstack_time(dense_bltt(F) @ stack_time(x), F.shape[0])
        assert np.allclose(y, y_ref, rtol=0, atol=1e-13 * np.abs(y_ref).max())


def rng_like(F, seed):
    return np.random.default_rng(seed).standard_normal((F.shape[1], F.shape[2]))


def test_bltt_transpose_matches_dense_transpose(small):
    G, _, _ = small
    y = np.random.default_rng(3).standard_normal((G.shape[0], G.shape[2]))
    x = oracle.bltt_transpose(G, y)
    x_ref = unstack_time(dense_bltt(G).T @ stack_time(y), G.shape[1])
    assert np.allclose(x, x_ref, rtol=0, atol=1e-13 * np.abs(x_ref).max())


def test_batch_axis_is_independent(small):
    G, _, s = small
    s2 = np.stack([s, 2 * s[::-1], -s])
    y = oracle.bltt_apply(G, s2)
    for b in range(3):
        assert np.array_equal(y[b], oracle.bltt_apply(G, s2[b]))


@pytest.mark.parametrize("j,tau", [(0, 0), (2, 0), (1, 4)])
def test_impulse_returns_green_column(small, j, tau):
    """An impulse on subfault j at step tau returns column j of the Green's
    function, delayed by tau (Eq. elastic-response with s = e_j delta)."""
    G, _, _ = small
    Ns, Nt = G.shape[1], G.shape[2]
    s = np.zeros((Ns, Nt))
    s[j, tau] = 1.0
    m = oracle.bltt_apply(G, s)
    expect = np.zeros_like(m)
    expect[:, tau:] = G[:, j, :Nt - tau]
    assert np.array_equal(m, expect)


def test_dt_is_backward_difference_and_lower_toeplitz():
    rng = np.random.default_rng(11)
    m = rng.standard_normal((4, 10))
    v = oracle.dt_apply(m, dt=0.5)
    # library routine: numpy.diff with m[-1] = 0 prepended
    assert np.allclose(v, np.diff(m, prepend=0.0, axis=1) / 0.5, rtol=1e-15, atol=0)
    # D_t is itself BLTT(I/dt, -I/dt, 0, ...): lower triangular, lag-only
    F = np.zeros((4, 4, 10))
    F[np.arange(4), np.arange(4), 0] = 1 / 0.5
    F[np.arange(4), np.arange(4), 1] = -1 / 0.5
    assert np.allclose(v, oracle.bltt_apply(F, m), rtol=0, atol=1e-14)
    # transpose
    w = rng.standard_normal((4, 10))
    u = oracle.dt_transpose(w, dt=0.5)
    lhs = np.sum(v * w)
    rhs = np.sum(m * u)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    assert np.allclose(u, oracle.bltt_transpose(F, w), rtol=0, atol=1e-14)


def test_linearity(small):
    G, P, _ = small
    rng = np.random.default_rng(5)
    s1, s2 = rng.standard_normal((2,) + (G.shape[1], G.shape[2]))
    a, b = 1.7, -0.3
    lhs = oracle.waveforms(G, P, a * s1 + b * s2)
    rhs = a * oracle.waveforms(G, P, s1) + b * oracle.waveforms(G, P, s2)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


@pytest.mark.parametrize("tau", [1, 3])
def test_time_shift_invariance(small, tau):
    G, P, s = small
    Nt = s.shape[1]
    s_sh = np.zeros_like(s)
    s_sh[:, tau:] = s[:, :Nt - tau]
    q = oracle.waveforms(G, P, s)
    q_sh = oracle.waveforms(G, P, s_sh)
    assert np.allclose(q_sh[:, tau:], q[:, :Nt - tau], rtol=1e-13, atol=1e-13)
    assert np.all(q_sh[:, :tau] == 0)


def test_causality(small):
    G, P, s = small
    n0 = 5
    s2 = s.copy()
    s2[:, n0:] += np.random.default_rng(9).standard_normal(s[:, n0:].shape)
    q, q2 = oracle.waveforms(G, P, s), oracle.waveforms(G, P, s2)
    assert np.array_equal(q[:, :n0], q2[:, :n0])
    assert not np.array_equal(q[:, n0:], q2[:, n0:])


def test_composition_uses_dt_between_stages(small):
    """q = F_q D_t F_G s: the dense-matrix product with D_t in the middle."""
    G, P, s = small
    Ng, Nt = G.shape[0], G.shape[2]
    Dt = np.zeros((Ng, Ng, Nt))
    Dt[np.arange(Ng), np.arange(Ng), 0] = 1.0
    Dt[np.arange(Ng), np.arange(Ng), 1] = -1.0
    W = dense_bltt(P) @ dense_bltt(Dt) @ dense_bltt(G)
    q_ref = unstack_time(W @ stack_time(s), P.shape[0])
    q = oracle.waveforms(G, P, s)
    assert np.allclose(q, q_ref, rtol=0, atol=1e-12 * np.abs(q_ref).max())
    q_none = oracle.waveforms(G, P, s, dt_mode="none")
    W0 = dense_bltt(P) @ dense_bltt(G)
    assert np.allclose(q_none, unstack_time(W0 @ stack_time(s), P.shape[0]),
                       rtol=0, atol=1e-12 * np.abs(q_ref).max())


@pytest.mark.parametrize("parts", [[5], [1, 4], [2, 2, 1], [1, 1, 1, 1, 1]])
def test_partitioned_composition(small, parts):
    """Eq. (distributed-composition): summing per-partition results over any
    partition of the grid gives the same q."""
    G, P, s = small
    q = oracle.waveforms(G, P, s)
    edges = np.cumsum([0] + parts)
    chunks = [(G[a:b], P[:, a:b]) for a, b in zip(edges[:-1], edges[1:])]
    qp = oracle.waveforms_partitioned(chunks, s)
    assert np.allclose(qp, q, rtol=0, atol=1e-13 * np.abs(q).max())


def test_dft_real_matches_numpy_rfft():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 16))
    X = oracle.dft_real(x, 32)
    assert X.shape == (3, 17)
    assert np.allclose(X, np.fft.rfft(x, n=32), rtol=0, atol=1e-12)


def test_dft_real_closed_forms():
    L = 64
    l = np.arange(L // 2 + 1)
    x = np.zeros((1, 32))
    x[0, 5] = 1.0       # impulse at n0 -> exp(-2 pi i n0 l / L)
    assert np.allclose(oracle.dft_real(x, L)[0], np.exp(-2j * np.pi * 5 * l / L),
                       atol=1e-14)
    ones = np.ones((1, 32))  # box of length L/2: X[0] = 32, X[even l > 0] = 0
    X = oracle.dft_real(ones, L)[0]
    assert abs(X[0] - 32) < 1e-12
    assert np.allclose(X[2::2], 0, atol=1e-12)
    assert np.allclose(X[1::2], 2 / (1 - np.exp(-2j * np.pi * l[1::2] / L)),
                       atol=1e-11)


def test_fft_convolution_equals_direct_with_pad_2nt(small):
    """Alg. 2 with L = 2 Nt (ZeroPad, FFT, per-bin product over bins 0..Nt,
    IFFT, Truncate) reproduces Eq. (time-domain-conv): no circular wrap."""
    G, _, s = small
    Nt = s.shape[1]
    L = 2 * Nt
    Gh = oracle.dft_real(G, L)                       # [Ng][Ns][Nt+1]
    sh = oracle.dft_real(s, L)                       # [Ns][Nt+1]
    mh = np.einsum("ijl,jl->il", Gh, sh)
    m = np.fft.irfft(mh, n=L)[:, :Nt]
    assert np.allclose(m, oracle.bltt_apply(G, s), rtol=0, atol=1e-12)


def test_single_pass_needs_longer_pad(small):
    """Folding D_t and both stages into one per-bin product at L = 2 Nt
    aliases (support 3 Nt - 2 > L); with the truncate-and-retransform step, or
    with L >= 3 Nt - 1, it is exact."""
    G, P, s = small
    Nt = s.shape[1]
    q = oracle.waveforms(G, P, s)

    def one_pass(L):
        Gh, Ph, sh = (oracle.dft_real(a, L) for a in (G, P, s))
        dh = 1 - np.exp(-2j * np.pi * np.arange(L // 2 + 1) / L)
        qh = np.einsum("oil,il->ol", Ph, dh * np.einsum("ijl,jl->il", Gh, sh))
        return np.fft.irfft(qh, n=L)[:, :Nt]

    assert not np.allclose(one_pass(2 * Nt), q, atol=1e-9 * np.abs(q).max())
    L3 = 3 * Nt - 1 + (3 * Nt - 1) % 2      # smallest even L >= 3 Nt - 1
    assert np.allclose(one_pass(L3), q, atol=1e-11 * np.abs(q).max())


def test_adjoint_identity(small):
    """<W s, r> = <s, W^T r> for the composed map (FP64)."""
    G, P, s = small
    r = np.random.default_rng(4).standard_normal((P.shape[0], P.shape[2]))
    q = oracle.waveforms(G, P, s)
    wt = oracle.bltt_transpose(G, oracle.dt_transpose(oracle.bltt_transpose(P, r)))
    lhs, rhs = np.sum(q * r), np.sum(s * wt)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradient_central_differences(small):
    """The misfit is quadratic in s, so a central difference is exact up to
    rounding: (L(s+h e) - L(s-h e)) / 2h = <dL/ds, e>."""
    G, P, s = small
    rng = np.random.default_rng(8)
    d = rng.standard_normal((P.shape[0], P.shape[2]))
    loss, g = oracle.gradient(G, P, s[None], d[None])
    h = 1e-3
    for trial in range(3):
        e = rng.standard_normal(s.shape)
        e /= np.linalg.norm(e)
        lp, _ = oracle.gradient(G, P, (s + h * e)[None], d[None])
        lm, _ = oracle.gradient(G, P, (s - h * e)[None], d[None])
        fd = (lp[0] - lm[0]) / (2 * h)
        assert abs(fd - np.sum(g[0] * e)) <= 1e-9 * max(1.0, abs(fd))


def test_gradient_partitioned_matches_full(small):
    G, P, s = small
    d = np.random.default_rng(12).standard_normal((1, P.shape[0], P.shape[2]))
    loss, g = oracle.gradient(G, P, s[None], d)
    lp, gp = oracle.gradient_partitioned(
        lambda: [(G[:2], P[:, :2]), (G[2:], P[:, 2:])], s[None], d)
    assert np.allclose(lp, loss, rtol=1e-13)
    assert np.allclose(gp, g, rtol=0, atol=1e-13 * np.abs(g).max())


def test_oracle_on_tiny_workload_is_finite_and_nonzero():
    wl = synth.WORKLOADS["tiny"]
    geom = wl.geometry_obj()
    G = geom.greens_rows(0, wl.Ng, wl.Nt)
    P = geom.adjoint_cols(0, wl.Ng, wl.Nt)
    s = wl.slip(geom)
    q = oracle.waveforms(G, P, s)
    assert q.shape == (1, wl.No, wl.Nt)
    assert np.all(np.isfinite(q)) and np.abs(q).max() > 0


def test_fft_window_head_is_q_and_tail_is_linear_convolution(small):
    """oracle.fft_window: first Nt samples are q; the whole window is the
    linear convolution of P with the Nt-truncated v (numpy.convolve)."""
    G, P, s = small
    Nt = s.shape[1]
    qw = oracle.fft_window(G, P, s[None])
    assert qw.shape == (1, P.shape[0], 2 * Nt)
    assert np.allclose(qw[0, :, :Nt], oracle.waveforms(G, P, s), rtol=0, atol=1e-13)
    v = oracle.dt_apply(oracle.bltt_apply(G, s))
    ref = np.zeros((P.shape[0], 2 * Nt))
    for o in range(P.shape[0]):
        for i in range(P.shape[1]):
            # full linear convolution has 2 Nt - 1 samples; the last one is 0
            ref[o, :2 * Nt - 1] += np.convolve(P[o, i], v[i])
    assert np.allclose(qw[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_fft_window_adjoint_tail_is_gradient_and_full_correlation(small):
    """oracle.fft_window_adjoint: lags n >= 0 are F_G^T D_t^T F_q^T r; the
    whole window is the full cross-correlation (numpy.correlate) of the
    Green's functions with u = D_t^T F_q^T r."""
    G, P, _ = small
    Nt = G.shape[2]
    r = np.random.default_rng(21).standard_normal((1, P.shape[0], Nt))
    gw = oracle.fft_window_adjoint(G, P, r)
    assert gw.shape == (1, G.shape[1], 2 * Nt)
    g = oracle.bltt_transpose(G, oracle.dt_transpose(oracle.bltt_transpose(P, r)))
    assert np.allclose(gw[..., Nt:], g, rtol=0, atol=1e-13 * np.abs(g).max())
    u = oracle.dt_transpose(oracle.bltt_transpose(P, r))[0]
    ref = np.zeros((G.shape[1], 2 * Nt))
    for j in range(G.shape[1]):
        for i in range(G.shape[0]):
            # c[m] = sum_k G[k] u[m + k], m = -(Nt-1)..Nt-1  ->  index m + Nt
            c = np.correlate(u[i], G[i, j], mode="full")  # lags -(Nt-1)..(Nt-1)
            ref[j, 1:] += c
    assert np.allclose(gw[0], ref, rtol=0, atol=1e-12 * np.abs(ref).max())
