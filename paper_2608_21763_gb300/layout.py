"""Size arithmetic of the FFT representation (no GPU, no library load).

Alg. 2 zero-pads each length-Nt history to L = 2 Nt before the FFT; a real
signal of length L has L/2 + 1 = Nt + 1 independent bins, so the resident
response spectra hold Nt + 1 complex blocks per operator entry (Sec. II-C.1:
bins l = 0..Nt).  The library stores the stage-1 spectrum as
[bin][grid row][Ns_pad] and the stage-2 spectrum as [bin][observation][Ng_pad],
with the inner dimension padded to a multiple of ``PAD`` entries so that every
row starts on a 16-byte boundary for every storage type.
"""
from __future__ import annotations

import dataclasses

PAD = 8
COMPLEX_BYTES = {"fp64": 16, "fp32": 8, "bf16": 4, "bf16_hilo": 8, "fp8": 2}
FP8_ROW_BLOCK = 256     # one FP32 scale per (bin, 256 grid rows)


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


def fft_length(Nt: int) -> int:
    return 2 * Nt


def num_bins(Nt: int) -> int:
    return Nt + 1


@dataclasses.dataclass(frozen=True)
class Layout:
    Ns: int
    Ng: int
    No: int
    Nt: int

    @property
    def L(self):
        return fft_length(self.Nt)

    @property
    def Nb(self):
        return num_bins(self.Nt)

    @property
    def Ns_pad(self):
        return round_up(self.Ns, PAD)

    @property
    def Ng_pad(self):
        return round_up(self.Ng, PAD)

    def g_bytes(self, prec: str) -> int:
        b = self.Nb * self.Ng * self.Ns_pad * COMPLEX_BYTES[prec]
        if prec == "fp8":
            b += self.Nb * ((self.Ng + FP8_ROW_BLOCK - 1) // FP8_ROW_BLOCK) * 4
        return b

    def p_bytes(self, prec: str) -> int:
        return self.Nb * self.No * self.Ng_pad * COMPLEX_BYTES[prec]

    def seafloor_dim(self) -> int:
        """Entries of one seafloor space-time field m (Ng x Nt)."""
        return self.Ng * self.Nt


def paper_coefficient_bytes_per_gpu(Nf: int, Nm: int, Nq: int, Nt: int,
                                    gpus: int, complex_bytes: int = 16) -> float:
    """Unpadded resident spectra per GPU when the seafloor grid is split
    evenly: (Nt + 1) bins x complex x (Nm Nf + Nq Nm) / gpus."""
    return num_bins(Nt) * complex_bytes * (Nm * Nf + Nq * Nm) / gpus
