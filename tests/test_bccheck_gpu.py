"""The Sec. 3.1 boundary benchmark on the GPU: against the oracle on a coarser
version of the set-up (same box, 200 x 200 cells), and against the paper's
"about 1%" on the paper's 400 x 400 grid."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def oracle_reflectivity(bc, n, t_end=30.0):
    w = W.bc_check_2d(bc, n=n)
    og = oracle.OracleGrid(w.grid)
    og.inject_axion(w.axions[0])
    a0 = np.abs(og.phi_cur).max()
    H0 = og.diagnostics()["H_phi"]
    og.step(int(round(t_end / w.grid.dt)))
    N = w.grid.pml_cells if bc == "pml" else 0
    amp = np.abs(og.phi_cur[0, N:w.grid.n[1] - N, N:w.grid.n[0] - N]).max() / a0
    return og.diagnostics()["H_phi"] / H0, amp


# FP32 split: the reflected energy and amplitude are what is left after the
# layer absorbed all but 0.03% of the energy (2% of the amplitude), so they are
# differences of FP32 fields of order 1; measured against the FP64 oracle they
# differ by 3e-6 (energy) and 5e-6 (amplitude) on the 200 x 200 grid, held
# here to 1e-4.
@pytest.mark.parametrize("bc,prec,tol", [("pml", "fp64", 1e-8), ("outflow", "fp64", 1e-8), ("pml", "fp32", 1e-4)])
def test_reflectivity_matches_oracle(bc, prec, tol):
    from paper_2406_16796_gb300 import bccheck

    got = bccheck.reflectivity(bc, precision=prec, n=200)
    e, a = oracle_reflectivity(bc, 200)
    assert got["energy"] == pytest.approx(e, rel=tol)
    assert got["amplitude"] == pytest.approx(a, rel=tol)
    assert got["kernel"] == ("general" if bc == "outflow" else "k_tm2d")


@pytest.mark.parametrize("bc", ["pml", "outflow"])
def test_reflectivity_about_one_percent_on_the_paper_grid(bc):
    from paper_2406_16796_gb300 import bccheck

    R = GOLDEN["bc_reflectivity"]["value"]
    got = bccheck.reflectivity(bc, n=400)
    assert got["energy"] < R
    assert 0.3 * R < got["amplitude"] < 4 * R
