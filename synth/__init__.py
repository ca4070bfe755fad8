"""Seeded synthetic inputs for the source-to-waveform path.

This module holds none of the method's arithmetic.  It builds the inputs that
both the FP64 oracle (``oracle/``) and the CUDA library are fed:

* geometry: subfault, seafloor-grid and observation coordinates (km);
* time-domain response operators ``G[i][j][k]`` (grid row i, subfault j, lag k)
  and ``P[o][i][k]`` (observation o, grid column i, lag k), standing in for the
  paper's elastic Green's functions F_{G,k} (Sec. II-B.1) and acoustic-gravity
  adjoint responses F_{q,k} (Sec. II-B.2);
* slip-rate histories ``s[b][j][n]`` (rupture b, subfault j, step n), standing
  in for FakeQuakes ruptures (Sec. II-A): a triangular source-time function on
  every subfault, with slip from a von Karman random field.

All draws come from ``numpy.random.default_rng(seed)``; the same seed gives the
same arrays on x86 and Arm.  Operators are filled by a small C routine
(``synth_ops.c``) because the largest ones hold billions of entries.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_ops.c")
_LIB = os.path.join(_HERE, "_synth_ops.so")
_lib = None

# Closed-form response parameters (Ricker pulse delayed by travel time).
GREEN_VEL_KMS = 3.5       # elastic stand-in: apparent speed (km/s)
ADJ_VEL_KMS = 0.2         # acoustic-gravity stand-in: apparent speed (km/s)
DECAY_KM = 50.0           # amplitude decay length exp(-d/50 km)
RICKER_F0 = 0.1           # Hz
RUPTURE_VEL_KMS = 2.8     # rupture-front speed used for onset times


def build(force: bool = False) -> str:
    """Compile ``synth_ops.c`` into ``_synth_ops.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_response.argtypes = [
            ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_long,
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
        lib.synth_response.restype = None
        _lib = lib
    return _lib


def response(pa: np.ndarray, pb: np.ndarray, Nt: int, vel: float,
             dtype=np.float64, dt: float = 1.0, decay: float = DECAY_KM,
             f0: float = RICKER_F0, out: np.ndarray | None = None) -> np.ndarray:
    """``out[a][b][k] = exp(-d_ab/decay) * ricker(k*dt - d_ab/vel; f0)``."""
    pa = np.ascontiguousarray(pa, dtype=np.float64)
    pb = np.ascontiguousarray(pb, dtype=np.float64)
    dtype = np.dtype(dtype)
    assert dtype in (np.float32, np.float64)
    shape = (pa.shape[0], pb.shape[0], Nt)
    if out is None:
        out = np.empty(shape, dtype=dtype)
    assert out.shape == shape and out.dtype == dtype and out.flags.c_contiguous
    _load().synth_response(pa.ctypes.data, pa.shape[0], pb.ctypes.data,
                           pb.shape[0], Nt, dt, vel, decay, f0,
                           int(dtype == np.float32), out.ctypes.data)
    return out


# --------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Geometry:
    sub: np.ndarray      # [Ns][3] subfault centres (x, y, z) km, z down
    grid: np.ndarray     # [Ng][3] seafloor grid points, z = 0
    obs: np.ndarray      # [No][3] observation points, z = 0
    strike: np.ndarray   # [Ns] along-strike coordinate of each subfault (km)
    dip: np.ndarray      # [Ns] down-dip coordinate of each subfault (km)
    kind: str

    @property
    def Ns(self):
        return self.sub.shape[0]

    @property
    def Ng(self):
        return self.grid.shape[0]

    @property
    def No(self):
        return self.obs.shape[0]

    def greens_rows(self, i0: int, i1: int, Nt: int, dtype=np.float64,
                    out=None) -> np.ndarray:
        """Time-domain elastic stand-in ``G[i][j][k]`` for grid rows i0..i1."""
        return response(self.grid[i0:i1], self.sub, Nt, GREEN_VEL_KMS,
                        dtype=dtype, out=out)

    def adjoint_cols(self, i0: int, i1: int, Nt: int, dtype=np.float64,
                     out=None) -> np.ndarray:
        """Time-domain adjoint stand-in ``P[o][i][k]`` for grid columns i0..i1."""
        return response(self.obs, self.grid[i0:i1], Nt, ADJ_VEL_KMS,
                        dtype=dtype, out=out)


def geometry_box(Ns: int, Ng: int, No: int, seed: int) -> Geometry:
    """Points uniform in a 200 x 100 km box; subfaults at 10 km depth."""
    rng = np.random.default_rng(seed)
    sx = rng.uniform(0, 200, Ns)
    sy = rng.uniform(0, 100, Ns)
    sub = np.stack([sx, sy, np.full(Ns, 10.0)], axis=1)
    grid = np.stack([rng.uniform(0, 200, Ng), rng.uniform(0, 100, Ng),
                     np.zeros(Ng)], axis=1)
    obs = np.stack([rng.uniform(0, 200, No), rng.uniform(0, 100, No),
                    np.zeros(No)], axis=1)
    return Geometry(sub, grid, obs, sx, sy, "box")


PLANE_LEN_KM = 1000.0
PLANE_WID_KM = 100.0
PLANE_DIP_DEG = 12.0
PLANE_TOP_KM = 5.0
GRID_PAD_KM = 50.0


def geometry_plane(Ns: int, Ng: int, No: int, seed: int) -> Geometry:
    """Subfaults on a 1000 x 100 km plane dipping 12 deg (top at 5 km depth);
    grid and observations uniform over its surface projection widened by
    50 km."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, PLANE_LEN_KM, Ns)            # along strike
    w = rng.uniform(0, PLANE_WID_KM, Ns)            # down dip
    dip = np.deg2rad(PLANE_DIP_DEG)
    sub = np.stack([u, w * np.cos(dip), PLANE_TOP_KM + w * np.sin(dip)], axis=1)
    ymax = PLANE_WID_KM * np.cos(dip)
    lo = (-GRID_PAD_KM, -GRID_PAD_KM)
    hi = (PLANE_LEN_KM + GRID_PAD_KM, ymax + GRID_PAD_KM)
    grid = np.stack([rng.uniform(lo[0], hi[0], Ng), rng.uniform(lo[1], hi[1], Ng),
                     np.zeros(Ng)], axis=1)
    obs = np.stack([rng.uniform(lo[0], hi[0], No), rng.uniform(lo[1], hi[1], No),
                    np.zeros(No)], axis=1)
    return Geometry(sub, grid, obs, u, w, "plane")


# --------------------------------------------------------------------------
# Slip-rate histories
# --------------------------------------------------------------------------
def _triangle(n: np.ndarray, t0: np.ndarray, rise: np.ndarray) -> np.ndarray:
    """Unit-area triangle on [t0, t0 + rise] sampled at integer steps n."""
    half = 0.5 * rise
    x = 1.0 - np.abs(n[None, :] - (t0 + half)[:, None]) / half[:, None]
    return np.maximum(x, 0.0) / half[:, None]


def slip_triangular(geom: Geometry, B: int, Nt: int, seed: int) -> np.ndarray:
    """Tiny-case ruptures: a triangular STF of 5-20 steps per subfault, onset at
    hypocentral distance / 2.8 km/s, amplitude from a seeded Gaussian draw.
    Returns float64 [B][Ns][Nt]."""
    rng = np.random.default_rng(seed)
    n = np.arange(Nt, dtype=np.float64)
    out = np.empty((B, geom.Ns, Nt))
    for b in range(B):
        h = geom.sub[rng.integers(geom.Ns)]
        t0 = np.linalg.norm(geom.sub - h, axis=1) / RUPTURE_VEL_KMS
        rise = rng.integers(5, 21, geom.Ns).astype(np.float64)
        amp = rng.standard_normal(geom.Ns)
        out[b] = amp[:, None] * _triangle(n, t0, rise)
    return out


VK_CORR_STRIKE_KM = 40.0
VK_CORR_DIP_KM = 15.0
VK_HURST = 0.75
SHEAR_MODULUS_PA = 30e9


def _von_karman_field(rng, nx: int, nw: int, dx: float) -> np.ndarray:
    """Zero-mean, unit-variance von Karman field on an nx x nw grid by FFT
    filtering of white noise, PSD ~ (1 + kx^2 ax^2 + kw^2 aw^2)^-(H+1)."""
    kx = 2 * np.pi * np.fft.fftfreq(nx, dx)
    kw = 2 * np.pi * np.fft.fftfreq(nw, dx)
    KX, KW = np.meshgrid(kx, kw, indexing="ij")
    psd = (1 + KX ** 2 * VK_CORR_STRIKE_KM ** 2
           + KW ** 2 * VK_CORR_DIP_KM ** 2) ** (-(VK_HURST + 1))
    noise = rng.standard_normal((nx, nw))
    f = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.sqrt(psd)))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def slip_von_karman(geom: Geometry, B: int, Nt: int, seed: int,
                    mw_range=(8.0, 9.0), durations=None) -> np.ndarray:
    """Stochastic ruptures on the dipping plane.

    Per rupture: a magnitude Mw ~ U(mw_range); a rupture box whose length and
    width follow magnitude scaling (clipped to the plane); a log-normal von
    Karman slip field (correlation 40/15 km, Hurst 0.75) with a 10 % cosine
    taper at the box edges, scaled so that M0 = mu * A * mean slip with
    M0 = 10^(1.5 Mw + 9.1) N m and mu = 30 GPa; a hypocentre inside the box;
    onsets at hypocentral distance / 2.8 km/s; triangular slip-rate functions
    whose rise time grows with sqrt(slip).  ``durations`` (one per rupture),
    when given, zeroes every sample at or after it.  Returns float64
    [B][Ns][Nt] in m/s.
    """
    rng = np.random.default_rng(seed)
    n = np.arange(Nt, dtype=np.float64)
    dx = 5.0
    nx = int(PLANE_LEN_KM / dx)
    nw = int(PLANE_WID_KM / dx)
    out = np.zeros((B, geom.Ns, Nt))
    u, w = geom.strike, geom.dip
    iu = np.clip((u / dx).astype(int), 0, nx - 1)
    iw = np.clip((w / dx).astype(int), 0, nw - 1)
    for b in range(B):
        mw = rng.uniform(*mw_range)
        length = min(PLANE_LEN_KM, 10 ** (-2.37 + 0.57 * mw))
        width = min(PLANE_WID_KM, 10 ** (-1.86 + 0.46 * mw))
        u0 = rng.uniform(0, PLANE_LEN_KM - length)
        w0 = rng.uniform(0, PLANE_WID_KM - width)
        field = np.exp(0.5 * _von_karman_field(rng, nx, nw, dx))[iu, iw]
        su = (u - u0) / length
        sw = (w - w0) / width
        inside = (su >= 0) & (su <= 1) & (sw >= 0) & (sw <= 1)

        def taper(t):
            e = 0.1
            return np.where(t < e, 0.5 - 0.5 * np.cos(np.pi * np.clip(t, 0, e) / e),
                            np.where(t > 1 - e,
                                     0.5 - 0.5 * np.cos(np.pi * np.clip(1 - t, 0, e) / e),
                                     1.0))
        slip = np.where(inside, field * taper(su) * taper(sw), 0.0)
        m0 = 10 ** (1.5 * mw + 9.1)
        mean_slip = m0 / (SHEAR_MODULUS_PA * length * width * 1e6)
        act = slip[inside]
        if act.size and act.mean() > 0:
            slip *= mean_slip / act.mean()
        hu = u0 + rng.uniform(0.2, 0.8) * length
        hw = w0 + rng.uniform(0.2, 0.8) * width
        dist = np.hypot(u - hu, w - hw)
        t0 = dist / RUPTURE_VEL_KMS
        rise = np.clip(4.0 * np.sqrt(slip), 3.0, 40.0)
        s = slip[:, None] * _triangle(n, t0, rise)
        if durations is not None:
            s[:, int(durations[b]):] = 0.0
        out[b] = s
    return out


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    Ns: int
    Ng: int
    No: int
    Nt: int
    B: int
    geometry: str          # "box" | "plane"
    geom_seed: int
    slip_seed: int
    slip_kind: str         # "triangular" | "von_karman"
    mw_range: tuple = (8.0, 9.0)
    uneven: bool = False   # durations ~ U{32..Nt}

    def geometry_obj(self) -> Geometry:
        f = geometry_box if self.geometry == "box" else geometry_plane
        return f(self.Ns, self.Ng, self.No, self.geom_seed)

    def durations(self, B: int | None = None):
        if not self.uneven:
            return None
        rng = np.random.default_rng(self.slip_seed + 1000003)
        return rng.integers(32, self.Nt + 1, B or self.B)

    def slip(self, geom: Geometry, B: int | None = None) -> np.ndarray:
        B = B or self.B
        if self.slip_kind == "triangular":
            return slip_triangular(geom, B, self.Nt, self.slip_seed)
        return slip_von_karman(geom, B, self.Nt, self.slip_seed,
                               self.mw_range, self.durations(B))


WORKLOADS = {
    # 16 subfaults, 1024 grid points, 4 observations, 32 steps, one rupture
    "tiny": Workload("tiny", 16, 1024, 4, 32, 1, "box", 1, 2, "triangular"),
    # paper shape (963 x 64 x 256) on a 20,000-point grid, one rupture, FP32
    "plain": Workload("plain", 963, 20000, 64, 256, 1, "plane", 10, 11,
                      "von_karman", (8.0, 9.0)),
    # 60,000-point grid, 256 ruptures with uneven active durations
    "batched": Workload("batched", 963, 60000, 64, 256, 256, "plane", 20, 21,
                        "von_karman", (7.5, 9.0), True),
    # 40,000-point grid, 64 ruptures, waveform-misfit gradient
    "gradient": Workload("gradient", 963, 40000, 64, 256, 64, "plane", 30, 31,
                         "von_karman", (8.0, 9.0)),
    # 150,000-point grid, 1024 ruptures
    "largest": Workload("largest", 963, 150000, 64, 256, 1024, "plane", 40, 41,
                        "von_karman", (7.0, 9.2)),
    # per-GPU shapes of the paper's runs (Table I, Table II), one rupture:
    # weak scaling, 480 subfaults x 37,758 grid points x 32 observations
    "paper_weak": Workload("paper_weak", 480, 37758, 32, 256, 1, "plane", 50, 51,
                           "von_karman", (8.0, 9.0)),
    # strong scaling on 8 GPUs, 60 x (2,416,530 / 8) x 4
    "paper_strong8": Workload("paper_strong8", 60, 302066, 4, 256, 1, "plane", 60, 61,
                              "von_karman", (8.0, 9.0)),
    # full Cascadia operator on 64 GPUs, 963 x (2,416,530 / 64) x 64
    "paper_csz64": Workload("paper_csz64", 963, 37758, 64, 256, 1, "plane", 70, 71,
                            "von_karman", (8.0, 9.0)),
}


def noisy_targets(rng_seed: int, q: np.ndarray, rel_noise: float = 0.05):
    """Targets d = q + N(0, (rel_noise * RMS(q))^2), per rupture."""
    rng = np.random.default_rng(rng_seed)
    rms = np.sqrt(np.mean(q.reshape(q.shape[0], -1) ** 2, axis=1))
    return q + rel_noise * rms[:, None, None] * rng.standard_normal(q.shape)


def random_waveforms(B: int, No: int, Nt: int, seed: int) -> np.ndarray:
    """Smooth random residual-like waveforms r[b][o][n] (for adjoint tests)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, No, Nt))
    k = np.exp(-0.5 * (np.arange(-8, 9) / 3.0) ** 2)
    return np.apply_along_axis(lambda v: np.convolve(v, k, "same"), 2, x)
