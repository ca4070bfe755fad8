"""Size arithmetic pinned to the figures the paper prints (tests/golden)."""
import os

from paper_2608_21763_gb300 import layout

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sizes.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("="))
            out[k] = float(v)
    return out


def test_resident_coefficients_match_paper():
    g = golden()
    b = layout.paper_coefficient_bytes_per_gpu(int(g["Nf"]), int(g["Nm"]),
                                               int(g["Nq"]), int(g["Nt"]),
                                               int(g["gpus"]))
    gib = b / 2 ** 30
    # the paper prints 148.51 GiB; Nt + 1 = 257 complex128 bins gives 148.50
    assert abs(gib - g["coeff_gib_per_gpu"]) < 0.02, gib
    # a wrong bin count (Nt or 2 Nt bins) would miss by far more
    assert abs(gib * 256 / 257 - g["coeff_gib_per_gpu"]) > 0.5
    assert abs(gib * 512 / 257 - g["coeff_gib_per_gpu"]) > 50


def test_seafloor_dimension_and_weak_scaling_sizes():
    g = golden()
    lay = layout.Layout(int(g["Nf"]), int(g["Nm"]), int(g["Nq"]), int(g["Nt"]))
    assert lay.seafloor_dim() == int(g["seafloor_spacetime_dim"])
    assert int(g["Nm"]) * 8 // 64 == int(g["weak_grid_8gpu"])
    assert round(g["Nm"] / 64) == int(g["weak_pts_per_gpu"])


def test_layout_padding():
    lay = layout.Layout(963, 20000, 64, 256)
    assert lay.L == 512 and lay.Nb == 257 and lay.Ns_pad == 968
    for prec, cb in layout.COMPLEX_BYTES.items():
        assert (lay.Ns_pad * cb) % 16 == 0, prec
