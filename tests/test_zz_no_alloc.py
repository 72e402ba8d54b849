"""The allocation-free diagnostics entry point against the regular one.

axp_diagnostics_noalloc serves callers that cannot call cudaMalloc (their
fields live in memory another allocator owns): its reduction scratch is a
fixed array inside the library.  This file is collected last so that, if it
fails, a run stopping at the first failure has already run every other test.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2406_16796_gb300 import workloads as W

KEYS = ("H_phi", "H_g0", "H_g1", "P_g2a", "P_a2g", "W", "sum_xB1z2", "sum_B1z2", "gauss_l2")
ORDER = ("E0x", "E0y", "E0z", "B0x", "B0y", "B0z", "E1x", "E1y", "E1z", "B1x", "B1y", "B1z", "phi_cur", "phi_old")


@pytest.mark.gpu
def test_noalloc_diagnostics_match_regular_entry_point_on_two_calls():
    import torch

    from paper_2406_16796_gb300 import axp

    w = W.pulse_2d(nx=192, ny=96, m=0.5 * W.K0, g=1e-2)
    grid = w.grid.replace(pml_cells=10)
    g = axp.Grid(grid)
    g.inject_laser(w.lasers[0])
    g.step(20)
    for call in range(2):
        ref = g.diagnostics()  # the regular entry point (workspace scratch)
        host = {k: g.read(k) for k in ORDER}
        dev = {k: torch.tensor(v, dtype=torch.float64, device="cuda").contiguous() for k, v in host.items()}
        ptrs = [dev[k].data_ptr() for k in ORDER]
        torch.cuda.synchronize()
        got = axp.axp_diagnostics_noalloc(g.desc, ptrs, grid.B_ext, grid.E_ext, g.step_count,
                                          torch.cuda.current_stream().cuda_stream)
        assert got["step"] == ref["step"] == g.step_count
        for k in KEYS:
            # the two entry points partition the sums over blocks differently; W
            # (H_phi plus the cross energy sum(E0.E1 + B0.B1) dV) nearly cancels,
            # so its rounding is measured against the size of its terms, which
            # Cauchy-Schwarz bounds by H_phi + 2 sqrt(H_g0 H_g1)
            scale = ref["H_phi"] + 2.0 * np.sqrt(ref["H_g0"] * ref["H_g1"]) if k == "W" else abs(ref[k])
            assert abs(got[k] - ref[k]) <= 1e-12 * scale + 1e-300, (call, k, got[k], ref[k])
        assert ref["H_phi"] > 0 and ref["H_g1"] > 0
        g.step(15)
    g.close()


_REJECT = r"""
import sys
sys.path.insert(0, sys.argv[1])
from paper_2406_16796_gb300 import axp
from paper_2406_16796_gb300 import workloads as W
big = W.pulse_2d(nx=4096, ny=2049).grid
try:
    axp.axp_diagnostics_noalloc(axp.desc_of(big), [1] * 14, big.B_ext, big.E_ext, 0, 0)
except axp.AxpError as e:
    print("status", e.status)
else:
    print("accepted")
"""


def test_noalloc_rejects_grids_beyond_its_scratch():
    """A grid one row larger than the scratch allows is refused before any CUDA
    call.  The pointers are placeholders, so the check runs in a child process
    that sees no GPU at all: should the size check ever regress, the call fails
    at device lookup (AXP_E_CUDA) instead of launching on bad addresses."""
    from paper_2406_16796_gb300 import axp

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _REJECT, root], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split()[-2:] == ["status", str(axp.AXP_E_INVAL)], (r.stdout, r.stderr)
    assert "exceed the maximum" in r.stderr
