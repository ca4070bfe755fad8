"""Host-side FP64 arithmetic of the library, checked on the CPU: the
retransform matrix that the tensor engine applies between the stages (Alg. 2:
IFFT, Truncate, D_t, ZeroPad, FFT of one real signal's Nt + 1 bins), through
the C ABI (s2w_retransform_matrix touches no device).

Pins: the oracle's own D_t / D_t^T and zero-padded DFT, with numpy's inverse
real FFT as the IFFT step; without D_t the map is the projection
DFT . ZeroPad . Truncate . IDFT, hence idempotent."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2608_21763_gb300 as s2w

BACKWARD, NONE = 0, 1


def lib_matrix(Nt, dt_mode, dt, transpose):
    T = np.empty(4 * Nt * Nt, dtype=np.float64)
    st = s2w.lib().s2w_retransform_matrix(Nt, dt_mode, dt, transpose,
                                         T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == 0, s2w.lib().s2w_last_error(None)
    return T.reshape(2 * Nt, 2 * Nt)


def dofs_to_bins(u, Nt):
    """k = 0: Re bin 0, k = 1: Re bin Nt, k = 2l, 2l + 1: Re, Im bin l."""
    X = np.zeros(u.shape[:-1] + (Nt + 1,), dtype=np.complex128)
    X[..., 0] = u[..., 0]
    X[..., Nt] = u[..., 1]
    X[..., 1:Nt] = u[..., 2:2 * Nt:2] + 1j * u[..., 3:2 * Nt:2]
    return X


def bins_to_dofs(X, Nt):
    u = np.empty(X.shape[:-1] + (2 * Nt,))
    u[..., 0] = X[..., 0].real
    u[..., 1] = X[..., Nt].real
    u[..., 2:2 * Nt:2] = X[..., 1:Nt].real
    u[..., 3:2 * Nt:2] = X[..., 1:Nt].imag
    return u


@pytest.mark.parametrize("Nt", [32, 64, 256])
@pytest.mark.parametrize("dt_mode,dt", [(BACKWARD, 1.0), (BACKWARD, 0.25), (NONE, 1.0)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_retransform_matrix_matches_the_oracle_steps(Nt, dt_mode, dt, transpose):
    T = lib_matrix(Nt, dt_mode, dt, transpose)
    L = 2 * Nt
    u = np.random.default_rng(Nt + transpose).standard_normal((6, 2 * Nt))
    m = np.fft.irfft(dofs_to_bins(u, Nt), n=L)[:, :Nt]  # IFFT, then Truncate
    if dt_mode == NONE:
        v = m
    else:
        v = oracle.dt_transpose(m, dt) if transpose else oracle.dt_apply(m, dt)
    want = bins_to_dofs(oracle.dft_real(v, L), Nt)      # ZeroPad, then FFT
    got = u @ T.T
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("Nt", [32, 128])
def test_without_dt_the_retransform_is_a_projection(Nt):
    T = lib_matrix(Nt, NONE, 1.0, 0)
    assert np.allclose(T @ T, T, rtol=0, atol=1e-12 * np.abs(T).max())
    assert not np.allclose(T, np.eye(2 * Nt))  # truncation discards the tail


def test_retransform_matrix_rejects_bad_arguments():
    L = s2w.lib()
    T = (ctypes.c_double * 16)()
    assert L.s2w_retransform_matrix(48, BACKWARD, 1.0, 0, T) == -6
    assert L.s2w_retransform_matrix(32, 7, 1.0, 0, T) == -1
    assert L.s2w_retransform_matrix(32, BACKWARD, 0.0, 0, T) == -1
    assert L.s2w_retransform_matrix(32, BACKWARD, 1.0, 2, T) == -1
    assert L.s2w_retransform_matrix(32, BACKWARD, 1.0, 0, None) == -1


def test_embedding_second_row_is_a_pair_rotation_of_the_first():
    """The stage-2 GEMM stores only row 2t = (Re P, -Im P) of the real
    embedding of each adjoint spectrum and builds row 2t + 1 = (Im P, Re P)
    in shared memory by rotating each 32-bit BF16 pair by 16 bits and
    flipping bit 15 (the sign of the new low half).  That is exact because
    round-to-nearest-even is odd-symmetric, bf16(-x) = -bf16(x), signed
    zeros included: checked here on the bit patterns, with the pair's first
    element in the low half as the BF16x2 layout has it."""
    from error_model import bf16
    rng = np.random.default_rng(3)
    re = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                         [0.0, -0.0, 0.0, -0.0, 1.0 + 2.0 ** -8, -(1.0 + 3 * 2.0 ** -8), 3.0e38]])
    im = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                         [0.0, 0.0, -0.0, -0.0, -(1.0 + 2.0 ** -8), 1.0 + 3 * 2.0 ** -8, -3.0e38]])

    def bits(x):
        return (np.asarray(bf16(x), np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint32)

    row_a = bits(re) | (bits(-im) << np.uint32(16))       # (Re, -Im), as stored
    rot = ((row_a << np.uint32(16)) | (row_a >> np.uint32(16))) ^ np.uint32(0x8000)
    row_b = bits(im) | (bits(re) << np.uint32(16))        # (Im, Re), as the embedding needs
    assert np.array_equal(rot, row_b)


def _offblock_rank1_residual(M, rows_bin, cols_bin):
    """Relative residual of the best rank-one fit (alternating least squares)
    to the entries of M whose row and column belong to different bins."""
    off = rows_bin[:, None] != cols_bin[None, :]
    Moff = np.where(off, M, 0.0)
    u = np.ones(M.shape[0])
    v = np.ones(M.shape[1])
    for _ in range(100):
        v = (Moff * u[:, None]).sum(0) / np.maximum((off * u[:, None] ** 2).sum(0), 1e-300)
        u = (Moff * v[None, :]).sum(1) / np.maximum((off * v[None, :] ** 2).sum(1), 1e-300)
    return np.abs(np.where(off, M - np.outer(u, v), 0.0)).max() / np.abs(M).max()


@pytest.mark.parametrize("Nt", [32, 256])
def test_parity_blocks_of_the_retransform_are_block_diagonal_plus_rank_one(Nt):
    """With the degrees of freedom grouped by bin parity, the even-to-even
    and odd-to-odd blocks of the retransform matrix are a per-bin (2 x 2)
    block diagonal plus a rank-one term: the even bins of the zero-padded
    2Nt-point transform are the Nt-point transform of the kept samples, the
    odd bins that of the samples times exp(-i pi n / Nt); under either a
    circular (or anti-circular) difference is diagonal, and the causal D_t
    differs from it by the wrap-around term of sample 0 only.  The cross
    blocks are not
    of that form (the structure is what a GEMM with half the MMAs would
    use)."""
    T = lib_matrix(Nt, BACKWARD, 1.0, 0)
    bins = np.array([0, Nt] + [k // 2 for k in range(2, 2 * Nt)])
    ev = np.where(bins % 2 == 0)[0]
    od = np.where(bins % 2 == 1)[0]
    for r, c in ((ev, ev), (od, od)):
        assert _offblock_rank1_residual(T[np.ix_(r, c)], bins[r], bins[c]) <= 1e-12
    for r, c in ((ev, od), (od, ev)):
        assert _offblock_rank1_residual(T[np.ix_(r, c)], bins[r], bins[c]) > 1e-2
