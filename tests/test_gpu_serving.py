"""Serving loop on the GPU: a short Poisson stream over a few topologies (one of them
partitioned), every solve reading and writing the requests' pinned host buffers in place
and starting from the diagonal multipliers computed inside the solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ilves_oracle as orc  # noqa: E402
from paper_2503_13075_gb300 import serving as sv  # noqa: E402

pytestmark = pytest.mark.gpu


def test_serving_stream_converges_and_matches_the_oracle():
    reqs, pool = sv.make_requests(60, rate_hz=4000.0, seed=12, n_topologies=4, lo=20, hi=9000)  # 59..6500 atoms
    eng = sv.Engine(hbm_budget_bytes=2 << 30, n_streams=4, max_batch=16, max_wait_s=0.001,
                    precision="mixed", warm_start="diag", tol=1e-12, device="cuda:0")
    eng.prewarm(pool)
    for r in reqs:
        eng.pin(r)
    stats = eng.serve(reqs)
    assert stats.completed == len(reqs) and stats.rejected == 0
    assert all(r.status == "ok" for r in reqs)
    for r in reqs:
        assert sv.max_relative_violation(r.x, r.atom_i, r.atom_j, r.d) <= 1e-12
    # the largest request against the oracle (positions within 1e-10 nm)
    big = max(reqs, key=lambda q: q.n_atoms)
    sysm = next(p for p in pool if p.n_atoms == big.n_atoms)
    ref = orc.solve_system(type(sysm)(sysm.name, big.x_old, big.x_unc, big.inv_mass, big.atom_i, big.atom_j, big.d),
                           tol=1e-12)
    assert np.abs(big.x - ref.x).max() <= 1e-10
