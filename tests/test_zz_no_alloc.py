"""The allocation-free entry point ilves_solve_static_scratch against ilves_solve.

Callers that cannot allocate device memory while they solve (an MD engine that has
reserved the device memory pool for its own buffers, or a time-stepping pipeline that
must not call cudaMalloc / cudaFree because they can synchronise the device) use
ilves_solve_static_scratch.  It keeps the state of the CTA-per-molecule path in one
static device array instead of the topology's workspace.  These tests check, through
the C ABI, that two calls in a row give the results of ilves_solve within the parity
tolerances used by the other GPU tests -- after a solve of another topology has left its
own state in the array -- and that an oversized topology is rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_13075_gb300 import binding as B  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
X_TOL = 1e-10
LAM_RTOL = 1e-8


def _dev(s):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    return f(s.x_old), f(s.x_unc), f(s.inv_mass), f(s.d)


def _host(outs):
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def _same(ref, got):
    x0, l0, i0, s0 = ref
    x1, l1, i1, s1 = got
    assert np.array_equal(s0, s1) and np.array_equal(i0, i1)
    assert np.abs(x1 - x0).max(initial=0) <= X_TOL
    scale = np.abs(l0).max(initial=0)
    assert np.all(np.abs(l1 - l0) <= LAM_RTOL * np.abs(l0) + 1e-10 * scale)


def _case(case, seed):
    if case == "protein_like":
        s = wl.protein_like(n_atoms=20000 - 997 * (seed % 2), seed=seed)
        return s, B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    if case == "protein_domains":  # overlapping domains keep positions and corrections in the array
        s = wl.protein_like(n_atoms=20000 - 997 * (seed % 2), seed=seed)
        return s, B.Topology(s.n_atoms, s.atom_i, s.atom_j, overlap=4)
    # a batch where most molecules take the CTA-per-molecule path, some the warp path
    s = wl.tree_batch(n_mol=24 + seed % 5, seed=seed)
    return s, B.Topology(s.n_atoms, s.atom_i, s.atom_j, max_warp_constraints=40)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("case", ["protein_like", "protein_domains", "forced_large"])
def test_static_scratch_matches_solve(case, prec):
    s, topo = _case(case, 77 if case == "forced_large" else 1002)
    assert topo.n_large > 0
    assert 0 < topo.workspace_bytes() <= B.lib().ilves_static_scratch_bytes()
    dev_in = _dev(s)
    ref = _host(topo.solve(*dev_in, precision=prec))
    assert np.all(ref[3] == B.CONVERGED)
    # another topology's solve through the same array first, so it holds other state (and
    # other barrier counts) when the case under test starts: results must not depend on it
    s_o, topo_o = _case(case, 78 if case == "forced_large" else 1003)
    other = _host(topo_o.solve_static_scratch(*_dev(s_o), precision=prec))
    assert np.all(other[3] == B.CONVERGED)
    for _ in range(2):  # two calls in a row, each compared with ilves_solve
        got = _host(topo.solve_static_scratch(*dev_in, precision=prec))
        _same(ref, got)


def test_static_scratch_rejects_oversized_topology():
    s = wl.protein_like(n_atoms=100_000, seed=1002)
    topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    assert topo.workspace_bytes() > B.lib().ilves_static_scratch_bytes()
    with pytest.raises(B.IlvesError) as e:
        topo.solve_static_scratch(*_dev(s), precision="mixed")
    assert e.value.code == 6
