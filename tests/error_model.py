"""Rounding models of the library's reduced-precision paths, for deriving
their error bars (test infrastructure; shares no code with the library).

Each model evaluates the same FFT pipeline as Alg. 2 in FP64 (numpy's FFT)
but rounds, round-to-nearest-even, exactly the operands that the path stores
or feeds to its MMAs in a narrower type, as the library's header documents:
  stream BF16 / BF16 hi-lo / FP8:   the operator spectra only;
  tensor BF16:  operator spectra, slip spectra, seafloor spectra (the stage-1
                epilogue writes BF16), the retransform matrix, velocity
                spectra, stage-2 operator;
  tensor split: every one of those as hi + lo BF16 parts, products formed as
                hi*hi + hi*lo + lo*hi (lo*lo dropped); the seafloor spectra
                stay FP32 and are split by the retransform;
  tensor FP8:   stage-1 operator as e4m3 with one scale per (bin, 256 grid
                rows), slip spectra as FP16 (an exact power-of-two rescale
                first), the rest as tensor BF16;
  tensor FP8 hi/lo: the same with the slip spectra as hi + lo e4m3 parts in
                one power-of-two frame per (bin, rupture) (amax <= 448).
The FP32 arithmetic of the kernels is not modelled: the bars are set at
about twice the modelled rounding error so that it fits beside it.
"""
import numpy as np


def bf16(x):
    """Round to BF16 (nearest even) through FP32, as the kernels round FP32
    values: add 0x7FFF plus the kept part's last bit to the FP32 pattern and
    clear the low 16 bits (no carry past bit 31 for finite values)."""
    f = np.array(x, np.float64).astype(np.float32)
    u = f.view(np.uint32)
    u += (u >> 16) & np.uint32(1)
    u += np.uint32(0x7FFF)
    u &= np.uint32(0xFFFF0000)
    return f.astype(np.float64)


def cplx(f, z):
    """f applied to the real and the imaginary parts (the memory layout of z kept)."""
    out = np.empty_like(z)
    out.real = f(z.real)
    out.imag = f(z.imag)
    return out


def bf16c(z):
    return cplx(bf16, z)


def hilo(z):
    """(hi, lo) BF16 parts of a complex array."""
    hi = bf16c(z)
    return hi, bf16c(z - hi)


def f16c(z):
    return cplx(lambda a: a.astype(np.float16).astype(np.float64), z)


def e4m3(x):
    """Round to e4m3 (3 mantissa bits, exponent bias 7, subnormals below
    2^-6, largest finite 448), nearest even, saturating."""
    a = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.maximum(a, 1e-300))), -6.0)
    q = 2.0 ** (e - 3)
    return np.sign(x) * np.minimum(np.round(a / q) * q, 448.0)


def fp8_rows(Gh):
    """Gh [Ng][Ns][Nb] complex rounded as e4m3 with scale amax / 448 per (bin,
    256 consecutive grid rows) over Re and Im."""
    out = np.empty_like(Gh)
    for g0 in range(0, Gh.shape[0], 256):
        blk = Gh[g0:g0 + 256]
        amax = np.maximum(np.abs(blk.real).max(axis=(0, 1)), np.abs(blk.imag).max(axis=(0, 1)))
        sc = np.where(amax > 0, amax / 448.0, 1.0)
        out[g0:g0 + 256] = (e4m3(blk.real / sc) + 1j * e4m3(blk.imag / sc)) * sc
    return out


def e4m3_hilo_cols(sh):
    """sh [B][Ns][Nb] as hi + lo e4m3 parts, both in the frame of the power of
    two that brings each (rupture, bin)'s largest |Re|, |Im| to <= 448."""
    out = np.empty_like(sh)
    for b in range(sh.shape[0]):
        for l in range(sh.shape[2]):
            x = sh[b, :, l]
            m = max(np.abs(x.real).max(), np.abs(x.imag).max())
            sc = 2.0 ** np.floor(np.log2(448.0 / m)) if m > 0 else 1.0
            xr, xi = x.real * sc, x.imag * sc
            hr, hi = e4m3(xr), e4m3(xi)
            out[b, :, l] = (hr + e4m3(xr - hr) + 1j * (hi + e4m3(xi - hi))) / sc
    return out


def retransform_matrix(Nt, dt=1.0):
    """The real 2Nt x 2Nt map of IFFT, Truncate, backward D_t, ZeroPad, FFT on
    one signal's degrees of freedom (Re bin 0, Re bin Nt, Re/Im bins 1..Nt-1),
    built column by column with numpy's FFT."""
    L = 2 * Nt
    K = 2 * Nt
    T = np.zeros((K, K))
    for k in range(K):
        u = np.zeros(K)
        u[k] = 1.0
        X = to_bins(u[None], Nt)[0]
        m = np.fft.irfft(X, n=L)[:Nt]
        v = (m - np.concatenate([[0.0], m[:-1]])) / dt
        T[:, k] = to_dofs(np.fft.rfft(v, n=L)[None], Nt)[0]
    return T


def to_bins(u, Nt):
    X = np.zeros(u.shape[:-1] + (Nt + 1,), dtype=np.complex128)
    X[..., 0] = u[..., 0]
    X[..., Nt] = u[..., 1]
    X[..., 1:Nt] = u[..., 2:2 * Nt:2] + 1j * u[..., 3:2 * Nt:2]
    return X


def to_dofs(X, Nt):
    u = np.empty(X.shape[:-1] + (2 * Nt,))
    u[..., 0] = X[..., 0].real
    u[..., 1] = X[..., Nt].real
    u[..., 2:2 * Nt:2] = X[..., 1:Nt].real
    u[..., 3:2 * Nt:2] = X[..., 1:Nt].imag
    return u


def ein1(g, s):
    """m[b][i][l] = sum_j g[i][j][l] s[b][j][l]: stage 1 per bin (BLAS over bins)."""
    return np.matmul(g.transpose(2, 0, 1), s.transpose(2, 1, 0)).transpose(2, 1, 0)


def ein2(p, v):
    """q[b][o][l] = sum_i p[o][i][l] v[b][i][l]: stage 2 per bin."""
    return np.matmul(p.transpose(2, 0, 1), v.transpose(2, 1, 0)).transpose(2, 1, 0)


def model_waveforms(G, P, slip, path):
    """q [B][No][Nt] of the FFT pipeline with `path`'s roundings (see the
    module docstring); G [Ng][Ns][Nt], P [No][Ng][Nt], slip [B][Ns][Nt], all
    FP32-representable inputs as the library receives them."""
    Nt = G.shape[2]
    L = 2 * Nt
    qh = model_spectra(np.fft.rfft(G, L, axis=-1), np.fft.rfft(P, L, axis=-1), np.fft.rfft(slip, L, axis=-1),
                       path, retransform_matrix(Nt))
    return np.fft.irfft(qh, L, axis=-1)[..., :Nt]


def model_spectra(Gh, Ph, sh, path, T):
    """Stage-2 spectra qh [B][No][Nb] of `path` from the operator spectra
    Gh [Ng][Ns][Nb], Ph [No][Ng][Nb], the slip spectra sh [B][Ns][Nb] and the
    retransform matrix T.  Except for the FP8 operator's per-(bin, 256-row)
    scales and the FP16 activations' global scale, every rounding is per
    element or per signal, so for the other paths the result over a grid is
    the sum of the results over its row chunks."""
    Nt = (Gh.shape[2] - 1)

    def split_prod(ein, a, b):  # hi*hi + hi*lo + lo*hi of BF16 parts (lo*lo dropped)
        ah, al = hilo(a)
        bh, bl = hilo(b)
        return ein(ah, bh + bl) + ein(al, bh)

    def retransform(mh, T_used):
        return to_bins(to_dofs(mh, Nt) @ T_used.T, Nt)

    if path in ("exact", "stream_bf16", "stream_bf16_hilo", "stream_fp8", "stream_fp8_bf16p"):
        if path == "stream_bf16":
            Gh, Ph = bf16c(Gh), bf16c(Ph)
        elif path == "stream_bf16_hilo":
            Gh = sum(hilo(Gh))
        elif path != "exact":
            Gh = fp8_rows(Gh)
            if path == "stream_fp8_bf16p":
                Ph = bf16c(Ph)
        mh = ein1(Gh, sh)
        vh = retransform(mh, T)
        return ein2(Ph, vh)
    if path == "tensor_bf16":
        mh = bf16c(ein1(bf16c(Gh), bf16c(sh)))
        vh = bf16c(retransform(mh, bf16(T)))
        return ein2(bf16c(Ph), vh)
    if path == "tensor_fp8":
        sc = 2.0 ** np.ceil(np.log2(np.abs(sh).max()))
        mh = bf16c(ein1(fp8_rows(Gh), f16c(sh / sc) * sc))
        vh = bf16c(retransform(mh, bf16(T)))
        return ein2(bf16c(Ph), vh)
    if path == "tensor_fp8_hilo":
        mh = bf16c(ein1(fp8_rows(Gh), e4m3_hilo_cols(sh)))
        vh = bf16c(retransform(mh, bf16(T)))
        return ein2(bf16c(Ph), vh)
    if path == "tensor_split":
        mh = split_prod(ein1, Gh, sh)
        Th, Tl = bf16(T), bf16(T - bf16(T))
        mh_h, mh_l = hilo(mh)
        d_h, d_l = to_dofs(mh_h, Nt), to_dofs(mh_l, Nt)
        vh = to_bins(d_h @ Th.T + d_h @ Tl.T + d_l @ Th.T, Nt)
        vh = sum(hilo(vh))
        return split_prod(ein2, Ph, vh)
    raise ValueError(path)
