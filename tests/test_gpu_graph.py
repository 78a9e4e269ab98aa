"""ilves_solve inside a captured CUDA graph: the batched (persistent), the partitioned and
the overlapping-domain (cooperative, side stream) solves capture into one graph whose replays give, bit for
bit, the eager solve's results -- also after new inputs are copied into the captured
buffers (one replay per MD step).  The solve allocates nothing, so capture needs no
special mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_13075_gb300 import binding as B  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["trees", "trees_one_warp_teams", "protein_parted", "protein_domains"])
def test_solve_replays_from_a_cuda_graph(case):
    dev = torch.device("cuda:0")
    if case == "trees":
        s = wl.tree_batch(n_mol=256, seed=1012)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    elif case == "trees_one_warp_teams":  # both slot classes in every CTA, each with its pool
        s = wl.tree_batch(n_mol=2000, seed=1015)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, narrow_atoms=80)
        sc = t.schedule("mixed")
        assert 0 < sc["n_slots_wide"] < len(sc["slot_team"]) and sc["pool_wide"] < sc["pool_n"]
    elif case == "protein_domains":
        s = wl.protein_like(n_atoms=12000, seed=1014)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000, overlap=4)
        assert t.n_large == 1
    else:
        s = wl.protein_like(n_atoms=12000, seed=1013)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000)
        assert t.n_large == 1
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    xo, xu, w, d = f(s.x_old), f(s.x_unc), f(s.inv_mass), f(s.d)
    outs = (torch.empty_like(xu), torch.empty(s.n_constraints, dtype=torch.float64, device=dev),
            torch.empty(t.n_molecules, dtype=torch.int32, device=dev),
            torch.empty(t.n_molecules, dtype=torch.int32, device=dev))

    def solve():
        t.solve(xo, xu, w, d, precision="mixed", start="diag", x_out=outs[0], lambda_out=outs[1],
                iterations_out=outs[2], status_out=outs[3])

    solve()
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):  # warm-up on a side stream before capture
        solve()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        solve()
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, outs):
        assert torch.equal(a, b)
    assert int(outs[3].abs().max()) == 0
    # next step: new unconstrained positions copied into the captured input buffer
    rng = np.random.default_rng(5)
    x_unc2 = s.x_old + rng.normal(0.0, 0.003, size=s.x_old.shape)
    xu.copy_(f(x_unc2))
    g.replay()
    torch.cuda.synchronize()
    replayed = [o.clone() for o in outs]
    solve()  # eager on the same new inputs
    torch.cuda.synchronize()
    for a, b in zip(replayed, outs):
        assert torch.equal(a, b)
    assert int(outs[3].abs().max()) == 0
