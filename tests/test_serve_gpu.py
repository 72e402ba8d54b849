"""The serving loop: continuous batching of 1D and 2D conversion requests.

Each request's result must be the same whether it was served alone or in the
mix: the batch and the group advance every request with per-cell arithmetic
that does not depend on the other requests, the tiling or the launch count,
so the comparison is exact.  One
1D and one 2D request also go to the FP64 oracle (conversion probability
within 1e-3, the FP32 split tolerance)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_16796_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_requests(count=36, seed=11, rate=400.0):
    """Seeded requests drawn like the serving stream, with sizes and step counts
    cut down so that the whole stream runs in seconds."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        m = W.K0 * math.exp(rng.uniform(math.log(1e-3), math.log(2.0)))
        g = math.exp(rng.uniform(math.log(1e-6), math.log(1e-3)))
        B0 = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        steps = int(rng.integers(100, 700))
        if rng.uniform() < 0.7:
            nx = int(round(math.exp(rng.uniform(math.log(64), math.log(9000)))))
            out.append(W.Request(t, 1, (nx, 1, 1), m, g, B0, steps))
        else:
            nx = 2 * int(round(math.exp(rng.uniform(math.log(128), math.log(300)))))
            out.append(W.Request(t, 2, (nx, nx // 2, 1), m, g, B0, steps))
    return out


def alone(r):
    """The request served by itself: a server holding only this request."""
    from paper_2406_16796_gb300 import serve

    srv = serve.Server(mem_1d_cells=max(64, r.n[0]), max_1d=1, mem_2d_bytes=1 << 30, max_2d=1, max_tiles=256)
    rec = srv.serve([W.Request(0.0, r.ndim, r.n, r.m, r.g, r.B0, r.steps)]).records[0]
    srv.close()
    return {"P_g2a": rec.P_g2a, "H_phi": rec.H_phi}


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_2406_16796_gb300 import serve

    reqs = small_requests()
    assert 5 <= sum(r.ndim == 2 for r in reqs) < len(reqs)
    # small pools so that requests queue for memory and share rounds
    srv = serve.Server(mem_1d_cells=20000, max_1d=64, mem_2d_bytes=48 << 20, max_2d=8, max_tiles=64,
                       round_s=0.002)
    st = srv.serve(reqs)
    srv.close()
    assert len(st.records) == len(reqs)
    assert st.max_live >= 4  # requests really overlapped on the device
    for rec in st.records:
        r = reqs[rec.index]
        assert rec.arrival <= rec.admitted <= rec.finished
        d = alone(r)
        assert rec.P_g2a == d["P_g2a"], (r, rec.P_g2a, d["P_g2a"])
        assert rec.H_phi == d["H_phi"]
    s = st.summary()
    assert s["requests"] == len(reqs) and s["p50_latency_s"] <= s["p99_latency_s"]
    assert s["gpu_launches"] > 0


def test_served_results_match_the_oracle():
    from paper_2406_16796_gb300 import serve

    reqs = [W.Request(0.0, 1, (1500, 1, 1), 0.4 * W.K0, 3e-4, 2.0, 600),
            W.Request(0.001, 2, (256, 128, 1), 0.3 * W.K0, 2e-4, 1.5, 300)]
    srv = serve.Server(mem_1d_cells=4096, max_1d=4, mem_2d_bytes=1 << 28, max_2d=4, max_tiles=64)
    st = srv.serve(reqs)
    srv.close()
    for rec in st.records:
        r = reqs[rec.index]
        w = W.request_workload(r, precision="fp64")
        og = oracle.OracleGrid(w.grid)
        og.inject_laser(w.lasers[0])
        og.step(r.steps)
        want = og.diagnostics()["P_g2a"]
        assert rec.P_g2a == pytest.approx(want, rel=1e-3), (r.ndim, rec.P_g2a, want)
