"""The workloads against tables the paper prints (fixtures in tests/golden/, each citing its
table): the strong-scaling meshes A-I."""
import os

from paper_2003_08746_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def _round_sig(x: float, sig: int) -> float:
    return float(f"{x:.{sig - 1}e}")


def test_paper_meshes_match_the_printed_table():
    """Axial x radial counts as printed, and axial x radial x 361 azimuthal points (first and
    last superposed, so 360 unique in the solver) round to the printed totals at the printed
    number of significant digits."""
    rows = _rows("paper_meshes.txt")
    assert [r[0] for r in rows] == sorted(W.PAPER_MESHES)
    for name, ni, nj, total in rows:
        ni, nj = int(ni), int(nj)
        assert W.PAPER_MESHES[name] == (ni, nj)
        mantissa = total.split("e")[0]
        sig = len(mantissa.replace(".", "").lstrip("0"))
        assert _round_sig(ni * nj * 361, sig) == float(total), (name, ni * nj * 361, total)
