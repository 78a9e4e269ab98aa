"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bounds (stated for every result): max_k |sigma_k| / d_k^2 <= tol (1e-12) recomputed
in float64 from the returned positions; positions within 1e-10 nm of the oracle;
multipliers within 1e-8 relative (plus a small absolute floor); per-molecule
iterations equal to the oracle's +-1 and identical statuses.  Both precision modes
meet the same bounds (the mixed mode reaches them through the outer Newton loop).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ilves_oracle as orc  # noqa: E402
from paper_2503_13075_gb300 import binding as B  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "mixed", "mixed_df"]
TOL = 1e-12
X_TOL = 1e-10
LAM_RTOL = 1e-8


def to_dev(s):
    dev = torch.device("cuda:0")
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return f(s.x_old), f(s.x_unc), f(s.inv_mass), f(s.d)


def run(s, precision, topo=None, **kw):
    t = topo or B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    xo, xu, w, d = to_dev(s)
    x, lam, it, st = t.solve(xo, xu, w, d, precision=precision, **kw)
    torch.cuda.synchronize()
    return t, x.cpu().numpy(), lam.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def compare(s, ref, x, lam, it, st, tol=TOL, it_slack=1):
    assert np.array_equal(st, ref.status), (np.unique(st, return_counts=True), np.unique(ref.status, return_counts=True))
    ok = st == orc.CONVERGED
    assert np.abs(it[ok] - ref.iterations[ok]).max(initial=0) <= it_slack
    sig = orc.violation(x, s.atom_i.astype(np.int64), s.atom_j.astype(np.int64), s.d)
    conv_c = ok[ref.mol_of_constraint]
    assert (np.abs(sig[conv_c]) / s.d[conv_c] ** 2).max(initial=0) <= tol
    assert np.abs(x - ref.x).max(initial=0) <= X_TOL
    scale = np.abs(ref.lam).max(initial=0)
    assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * scale)


@pytest.fixture(scope="module")
def trees():
    s = wl.tree_batch(n_mol=256, seed=1001)
    return s, orc.solve_system(s, tol=TOL)


@pytest.fixture(scope="module")
def trees_full():
    s = wl.tree_batch()
    return s, orc.solve_system(s, tol=TOL)


@pytest.fixture(scope="module")
def small_trees():
    """1,300 trees of 20..100 atoms: more molecules than the GPU's 96-thread teams, all at
    most 100 atoms, so the automatic choice solves every one on a one-warp team."""
    s = wl.tree_batch(n_mol=1300, lo=20, hi=100, seed=1701)
    return s, orc.solve_system(s, tol=TOL)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("narrow", [0, 60, 100])
def test_narrow_teams(prec, narrow, small_trees, trees):
    """One-warp teams (the narrow class): all molecules of a batch of small trees
    (automatic choice), and both classes side by side in every CTA (explicit thresholds on
    the 20..200-atom batch; then each CTA's wide and narrow slots run at once)."""
    s, ref = small_trees if narrow == 0 else trees
    topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j, narrow_atoms=narrow)
    team = topo.schedule(prec)["mol_team"]
    assert np.all(team == 32) if narrow == 0 else (np.any(team == 32) and np.any(team == 96))
    for start in (None, "diag"):
        t, x, lam, it, st = run(s, prec, topo=topo, start=start)
        compare(s, ref, x, lam, it, st, it_slack=1 if start is None else 2)
    if narrow == 60:  # ILVES-F on both classes: same root, chord iterations within +-1
        ref_chord = orc.solve_system(s, tol=TOL, max_iter=60, method="chord")
        t, x, lam, it, st = run(s, prec, topo=topo, method="chord", max_iter=60)
        assert np.all(st == B.CONVERGED)
        assert np.abs(it - ref_chord.iterations).max() <= 1
        assert np.abs(x - ref.x).max() <= X_TOL
        # the float-float mode tests convergence on |r|^2 - d^2 evaluated in float-float
        # arithmetic (rounding errors of ~2^-48 |r|^2 in each of about six tail terms) from
        # displacements, and returns x_unc + displacement rounded to float64 (coordinates of
        # a few nm: up to ~1.5e-14 d^2 in |r|^2 - d^2); together below 2^-44 ~ 5.7e-14 of d^2.
        # The chord method's linear convergence stops just under the tolerance, so the float64
        # recomputation of its returned positions may exceed the tolerance by that much
        slack = 2.0 ** -44 if prec == "mixed_df" else 0.0
        assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= TOL + slack


@pytest.mark.parametrize("prec", PRECS)
def test_chain64(prec):
    s = wl.chain64()
    ref = orc.solve_system(s, tol=TOL)
    t, x, lam, it, st = run(s, prec)
    compare(s, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_tree_batch_256(prec, trees):
    s, ref = trees
    t, x, lam, it, st = run(s, prec)
    compare(s, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_tree_batch_full_4096(prec, trees_full):
    s, ref = trees_full
    t, x, lam, it, st = run(s, prec)
    compare(s, ref, x, lam, it, st)
    assert t.last_launch_count() >= 1


@pytest.mark.parametrize("prec", PRECS)
def test_protein_like_large_path(prec):
    s = wl.protein_like(n_atoms=20000, seed=1002)
    ref = orc.solve_system(s, tol=TOL)
    t, x, lam, it, st = run(s, prec)
    assert t.n_large == 1
    compare(s, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_warp_path_forced_to_large_path(prec):
    """The CTA-per-molecule path on ordinary molecules gives the same results."""
    s = wl.tree_batch(n_mol=20, seed=77)
    ref = orc.solve_system(s, tol=TOL)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, max_warp_constraints=10)
    assert t.n_large > 0
    _, x, lam, it, st = run(s, prec, topo=t)
    compare(s, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_two_atoms_closed_form(prec):
    s = wl.two_atoms(d=0.1, w1=1 / 1.008, w2=1 / 12.011, seed=3, sigma=0.01)
    t, x, lam, it, st = run(s, prec)
    rho = s.x_old[0] - s.x_old[1]
    sv = s.x_unc[0] - s.x_unc[1]
    a, b, c0 = rho @ rho, sv @ rho, sv @ sv - s.d[0] ** 2
    c = (b - np.sqrt(b * b - a * c0)) / a
    lam_cf = c / (2 * (s.inv_mass[0] + s.inv_mass[1]))
    assert st[0] == B.CONVERGED
    assert abs(lam[0] - lam_cf) <= 1e-11 * abs(lam_cf)


@pytest.mark.parametrize("prec", PRECS)
def test_permuted_atoms_and_constraints(prec):
    """Non-contiguous molecules (scattered atom ids) and shuffled constraints."""
    s = wl.tree_batch(n_mol=40, seed=8)
    rng = np.random.default_rng(2)
    pa = rng.permutation(s.n_atoms)
    inv = np.empty_like(pa)
    inv[pa] = np.arange(s.n_atoms)
    pc = rng.permutation(s.n_constraints)
    sw = rng.random(s.n_constraints) < 0.5
    s2 = wl.System("perm", s.x_old[pa], s.x_unc[pa], s.inv_mass[pa],
                   inv[np.where(sw, s.atom_j, s.atom_i)[pc]].astype(np.int32),
                   inv[np.where(sw, s.atom_i, s.atom_j)[pc]].astype(np.int32), s.d[pc])
    ref = orc.solve_system(s2, tol=TOL)
    t, x, lam, it, st = run(s2, prec)
    compare(s2, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(prec):
    dev = torch.device("cuda:0")
    # no constraints at all: x_out = x_unc
    t = B.Topology(4, [], [])
    xo = torch.zeros(4, 3, dtype=torch.float64, device=dev)
    xu = torch.rand(4, 3, dtype=torch.float64, device=dev)
    x, lam, it, st = t.solve(xo, xu, torch.ones(4, dtype=torch.float64, device=dev),
                             torch.zeros(0, dtype=torch.float64, device=dev), precision=prec)
    assert torch.equal(x, xu)
    # unconstrained atoms pass through; anchored atom (w = 0) stays put
    s = wl.chain64()
    xo_ = np.vstack([s.x_old, [[9.0, 9.0, 9.0]]])
    xu_ = np.vstack([s.x_unc, [[9.1, 9.0, 9.0]]])
    w_ = np.append(s.inv_mass, 1.0)
    w_[0] = 0.0
    s2 = wl.System("c", xo_, xu_, w_, s.atom_i, s.atom_j, s.d)
    ref = orc.solve_system(s2, tol=TOL)
    _, x, lam, it, st = run(s2, prec)
    compare(s2, ref, x, lam, it, st)
    assert np.array_equal(x[-1], xu_[-1]) and np.array_equal(x[0], xu_[0])
    # feasible input: 0 solves, lambda = 0
    s3 = wl.chain64()
    s3.x_unc = s3.x_old + np.array([0.2, 0.0, -0.1])
    _, x, lam, it, st = run(s3, prec)
    assert it[0] == 0 and st[0] == B.CONVERGED and np.all(lam == 0)
    # NaN input -> NONFINITE; unreachable tolerance -> MAX_ITER after exactly max_iter solves
    s4 = wl.chain64()
    s4.x_unc = s4.x_unc.copy()
    s4.x_unc[5, 1] = np.nan
    _, x, lam, it, st = run(s4, prec)
    assert st[0] == B.NONFINITE
    _, x, lam, it, st = run(wl.chain64(), prec, tol=1e-30, max_iter=6)
    assert st[0] == B.MAX_ITER and it[0] == 6
    # r . rho = 0 at lambda = 0: singular pivot
    s5 = wl.System("sing", np.array([[0.0, 0, 0], [0.1, 0, 0]]), np.array([[0.0, 0, 0], [0.0, 0.12, 0]]),
                   np.ones(2), np.array([0], np.int32), np.array([1], np.int32), np.array([0.1]))
    _, x, lam, it, st = run(s5, prec)
    assert st[0] == B.SINGULAR_PIVOT


@pytest.mark.parametrize("prec", PRECS)
def test_batched_encoding_limits(prec):
    """Molecules at the batched kernel's encoding limits (fewer than 256 constraints, at
    most 511 atoms) and just past them, which take the CTA-per-molecule path, in one
    topology; and long chains (deep elimination orders) on both paths."""
    sizes = [2, 3, 254, 255, 256, 257, 258, 400]
    s = wl.tree_molecules_of_sizes(sizes, seed=1030)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    assert sorted(t.molecules()[0].tolist()) == sorted(sizes)
    assert 3 <= t.n_large < len(sizes)  # trees of 257, 258, 400 atoms have 256+ constraints
    ref = orc.solve_system(s, tol=TOL)
    _, x, lam, it, st = run(s, prec, topo=t, start="diag")
    compare(s, ref, x, lam, it, st, it_slack=2)
    c = wl.chain_molecules([64, 128, 255, 256, 257, 300], seed=1031)
    tc = B.Topology(c.n_atoms, c.atom_i, c.atom_j)
    assert tc.n_large == 2  # 256 and 299 bonds
    ref = orc.solve_system(c, tol=TOL)
    _, x, lam, it, st = run(c, prec, topo=tc)
    compare(c, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
def test_warm_start_and_aliasing(prec, trees):
    s, ref = trees
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    xo, xu, w, d = to_dev(s)
    lam0 = torch.from_numpy(ref.lam.astype(np.float32)).cuda()
    xu2 = xu.clone()
    x, lam, it, st = t.solve(xo, xu2, w, d, precision=prec, lambda0=lam0, x_out=xu2)  # x_out aliases x_unc
    torch.cuda.synchronize()
    x, lam, it, st = x.cpu().numpy(), lam.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == B.CONVERGED)
    assert it.max() <= 2  # a float32 copy of the exact multipliers leaves ~1e-7 relative error
    assert np.abs(x - ref.x).max() <= X_TOL
    sig = orc.violation(x, s.atom_i.astype(np.int64), s.atom_j.astype(np.int64), s.d)
    assert (np.abs(sig) / s.d ** 2).max() <= TOL


def test_repeated_solves_are_deterministic(trees):
    s, ref = trees
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    for prec in PRECS:
        outs = [run(s, prec, topo=t)[1] for _ in range(3)]
        assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["chain64", "trees", "protein_parted"])
def test_chord_method_ilves_f(prec, case):
    """ILVES-F: same root as the Newton oracle; iterations within +-1 of the chord oracle."""
    if case == "chain64":
        s = wl.chain64()
        topo = None
    elif case == "trees":
        s = wl.tree_batch(n_mol=128, seed=1001)
        topo = None
    else:
        s = wl.protein_like(n_atoms=12000, seed=1002)
        topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000)
        assert topo.n_large == 1
    ref = orc.solve_system(s, tol=TOL)
    ref_chord = orc.solve_system(s, tol=TOL, max_iter=60, method="chord")
    t, x, lam, it, st = run(s, prec, topo=topo, method="chord", max_iter=60)
    assert np.all(st == B.CONVERGED)
    assert np.abs(it - ref_chord.iterations).max() <= 1
    assert np.abs(x - ref.x).max() <= X_TOL
    assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= TOL
    assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("part", [24, 64])
def test_partitioned_small_parts(prec, part):
    """Many small parts: most constraints couple to the separator block, whose entries
    receive the parts' Schur contributions (two per entry) plus in-line terms."""
    s = wl.protein_like(n_atoms=3000, seed=1010)
    ref = orc.solve_system(s, tol=TOL)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=500, part_constraints=part)
    assert t.n_large == 1
    _, x, lam, it, st = run(s, prec, topo=t)
    compare(s, ref, x, lam, it, st)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["trees", "cta_path", "protein_parted"])
def test_diag_start_inside_the_solve(prec, case):
    """ILVES_START_DIAG: the set-up pass computes the diagonal starting multipliers itself.
    With max_iter = 0 the solve returns them unchanged (lambda_out) with the positions
    they give, which must equal, bit for bit, a solve started from ilves_warm_start's
    diagonal guess; the converged solve meets the oracle bounds."""
    if case == "trees":
        s = wl.tree_batch(n_mol=128, seed=1003)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    elif case == "cta_path":
        s = wl.tree_batch(n_mol=20, seed=78)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, max_warp_constraints=10)
        assert t.n_large > 0
    else:
        s = wl.protein_like(n_atoms=12000, seed=1002)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000)
        assert t.n_large == 1
    xo, xu, w, d = to_dev(s)
    lam0 = B.warm_start(None, t, xo, xu, w, d)
    a = [v.cpu().numpy() for v in t.solve(xo, xu, w, d, precision=prec, lambda0=lam0, max_iter=0)]
    b = [v.cpu().numpy() for v in t.solve(xo, xu, w, d, precision=prec, start="diag", max_iter=0)]
    assert np.array_equal(b[1], lam0.cpu().numpy().astype(np.float64))
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    ref = orc.solve_system(s, tol=TOL)
    x, lam, it, st = [v.cpu().numpy() for v in t.solve(xo, xu, w, d, precision=prec, start="diag")]
    compare(s, ref, x, lam, it, st, it_slack=2)
    with pytest.raises(ValueError):
        t.solve(xo, xu, w, d, precision=prec, lambda0=lam0, start="diag")
    # the C ABI refuses a lambda0 together with the flag
    P = lambda v: v.data_ptr()
    xs = torch.empty_like(xu)
    code = B.lib().ilves_solve(t._h, P(xo), P(xu), P(w), P(d), 1e-12, 25, B.PRECISIONS[prec] | B.START_DIAG,
                               P(lam0), P(xs), None, None, None, None)
    assert code == 1  # ILVES_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["trees", "cta_path", "protein_parted", "protein_domains"])
def test_pinned_host_buffers(prec, case):
    """ilves_solve on page-locked host buffers (read and written in place by the kernels)
    gives bit for bit the results of the same solve on device buffers."""
    if case == "protein_domains":
        s = wl.protein_like(n_atoms=12000, seed=1008)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000, overlap=4)
        assert len(t.export_domains(0)["cons"]) > 10
    elif case == "trees":
        s = wl.tree_batch(n_mol=128, seed=1004)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    elif case == "cta_path":
        s = wl.tree_batch(n_mol=20, seed=79)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, max_warp_constraints=10)
        assert t.n_large > 0
    else:
        s = wl.protein_like(n_atoms=12000, seed=1005)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000)
        assert t.n_large == 1
    dev_out = [v.cpu().numpy() for v in t.solve(*to_dev(s), precision=prec, start="diag")]
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (s.x_old, s.x_unc, s.inv_mass, s.d)]
    outs = t.solve(*host, precision=prec, start="diag")
    torch.cuda.synchronize()
    assert all(o.device.type == "cpu" and o.is_pinned() for o in outs)
    for u, v in zip(dev_out, outs):
        assert np.array_equal(u, v.numpy())
    assert np.all(dev_out[3] == B.CONVERGED)
    with pytest.raises(ValueError):  # pageable host memory is refused
        t.solve(*[torch.from_numpy(np.ascontiguousarray(a)) for a in (s.x_old, s.x_unc, s.inv_mass, s.d)])


@pytest.mark.parametrize("prec", PRECS)
def test_chord_with_diag_start(prec):
    """ILVES-F from the diagonal start computed inside the solve: same root as the Newton
    oracle, within the parity bounds, on the batched and the partitioned paths."""
    for s, topo in ((wl.tree_batch(n_mol=96, seed=1006), None),
                    (wl.protein_like(n_atoms=12000, seed=1007), "parted")):
        t = (B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000) if topo
             else B.Topology(s.n_atoms, s.atom_i, s.atom_j))
        ref = orc.solve_system(s, tol=TOL)
        _, x, lam, it, st = run(s, prec, topo=t, method="chord", max_iter=60, start="diag")
        assert np.all(st == B.CONVERGED)
        assert np.abs(x - ref.x).max() <= X_TOL
        assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= TOL
        assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_partitioned_more_parts_than_resident_ctas(prec):
    """718 parts: more than three CTAs per SM can hold, so CTAs loop over several parts
    without shared-memory part copies, and the separator block (too large for shared
    memory) is solved from global memory by CTA 0 -- the fallback configuration."""
    s = wl.protein_like(n_atoms=30000, seed=1011)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000, part_constraints=48)
    assert t.n_large == 1
    ref = orc.solve_system(s, tol=TOL)
    _, x, lam, it, st = run(s, prec, topo=t, start="diag")
    compare(s, ref, x, lam, it, st, it_slack=2)


def test_partitioned_grid_barrier_wait_runs_out():
    """A bounded device wait that runs out: with ``wait_test`` the partitioned solve's grid
    barriers also count CTAs that never arrive.  Every CTA gives up after its spin budget,
    the kernel returns normally, the molecule reports WAIT_TIMEOUT, and the context stays
    usable for the next (ordinary) solve."""
    import time

    s = wl.protein_like(n_atoms=6000, seed=1020)
    for overlap in (0, 4):  # the Schur-complement and the overlapping-domain kernels
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=1000, wait_test=1, overlap=overlap)
        assert t.n_large == 1
        t0 = time.perf_counter()
        _, x, lam, it, st = run(s, "mixed", topo=t)
        assert time.perf_counter() - t0 < 20.0
        assert st.tolist() == [B.WAIT_TIMEOUT]
    ref = orc.solve_system(s, tol=TOL)
    t2 = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=1000)
    _, x, lam, it, st = run(s, "mixed", topo=t2)
    compare(s, ref, x, lam, it, st)


@pytest.fixture(scope="module")
def protein_full():
    s = wl.protein_like()
    return s, orc.solve_system(s, tol=TOL), B.Topology(s.n_atoms, s.atom_i, s.atom_j)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("start", [None, "diag"])
def test_protein_like_full_size(prec, start, protein_full):
    """The 100,001-atom protein-like system (114,987 constraints) as benchmarked: one
    partitioned cooperative solve, element by element against the oracle."""
    s, ref, t = protein_full
    assert t.n_large == 1 and t.n_molecules == 1
    _, x, lam, it, st = run(s, prec, topo=t, start=start)
    compare(s, ref, x, lam, it, st, it_slack=1 if start is None else 2)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["trees", "protein_parted"])
def test_hydroxyl_angle_distances(prec, case):
    """X-O-H triangle-closing distances (main text, h-angles) on top of all bonds (and the
    H-X-H distances of the protein-like system): parity with the oracle, zero and diagonal
    starts, on the batched and the partitioned paths."""
    if case == "trees":
        s = wl.tree_batch(n_mol=256, seed=1030, xoh=True)
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    else:
        s = wl.protein_like(n_atoms=12000, seed=1031, xoh=True)
        assert s.meta["n_xoh_constraints"] > 0
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000)
        assert t.n_large == 1
    ref = orc.solve_system(s, tol=TOL)
    for start in (None, "diag"):
        _, x, lam, it, st = run(s, prec, topo=t, start=start)
        compare(s, ref, x, lam, it, st, it_slack=1 if start is None else 2)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("overlap", [2, 4])
def test_overlapping_domains(prec, overlap):
    """Overlapping domains (supplement Sec. 3, Overlapping Partitioning Method): every domain
    of a cooperative launch solves its own system and keeps its owned corrections.  The
    quasi-Newton iteration reaches the Newton oracle's root within the parity bounds, in the
    iterations of the oracle's own overlapping-domain iteration (+-1 from a zero start)."""
    s = wl.protein_like(n_atoms=12000, seed=1040, xoh=True)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000, part_constraints=256,
                   overlap=overlap)
    assert t.n_large == 1 and t.export_layout(0)["n_parts"] > 10
    ref = orc.solve_system(s, tol=TOL)
    ref_opm = orc.solve_system(s, tol=TOL, overlap=overlap, part_constraints=256, part_min=2000)
    for start in (None, "diag"):
        _, x, lam, it, st = run(s, prec, topo=t, start=start)
        assert st.tolist() == [B.CONVERGED]
        if start is None:
            assert abs(int(it[0]) - int(ref_opm.iterations[0])) <= 1
        assert np.abs(x - ref.x).max() <= X_TOL
        assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= TOL
        assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())


@pytest.mark.parametrize("prec", PRECS)
def test_overlapping_domains_chord(prec):
    """ILVES-F over overlapping domains: each domain factorises A(x_old, x_old) on its
    constraints once; same root, iterations within +-1 of the oracle's."""
    s = wl.protein_like(n_atoms=8000, seed=1041)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, partition_min_constraints=2000, part_constraints=256, overlap=4)
    ref = orc.solve_system(s, tol=TOL)
    ref_c = orc.solve_system(s, tol=TOL, max_iter=80, method="chord", overlap=4, part_constraints=256, part_min=2000)
    _, x, lam, it, st = run(s, prec, topo=t, method="chord", max_iter=80)
    assert st.tolist() == [B.CONVERGED]
    assert abs(int(it[0]) - int(ref_c.iterations[0])) <= 1
    assert np.abs(x - ref.x).max() <= X_TOL
    assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())


@pytest.mark.parametrize("prec", PRECS)
def test_overlapping_domains_full_size(prec, protein_full):
    """The 100,001-atom system over overlapping domains (overlap 4, automatic part size):
    parity with the Newton oracle; the planner's domains are the oracle's, and the iteration
    count is within +-1 of the oracle's overlapping-domain iteration."""
    s, ref, _ = protein_full
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, overlap=4)
    D = t.export_domains(0)
    part = int(np.ceil(s.n_constraints / (len(D["cons"]))))
    _, x, lam, it, st = run(s, prec, topo=t)
    assert st.tolist() == [B.CONVERGED]
    assert np.abs(x - ref.x).max() <= X_TOL
    assert np.all(np.abs(lam - ref.lam) <= LAM_RTOL * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())
    if len(D["cons"]) == -(-s.n_constraints // 256):  # the default part size held
        ref_opm = orc.solve_system(s, tol=TOL, overlap=4, part_constraints=256, part_min=4096)
        assert abs(int(it[0]) - int(ref_opm.iterations[0])) <= 1


def test_autotune_keeps_the_fastest_converging_configuration():
    """ilves_autotune times candidate set-up options on the caller's inputs and keeps the
    fastest; the tuned topologies still meet the parity bounds.  Batched molecules tune slots,
    CTAs per SM and elimination order; a partitioned molecule also the Schur complement
    against overlapping domains."""
    s = wl.tree_batch(n_mol=512, seed=1050)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    tun = t.autotune(*to_dev(s), precision="mixed", start="diag", reps=3)
    assert tun["candidates"] >= 5 and 0 < tun["best_ms"] <= tun["before_ms"]
    assert t.tuning() == tun
    ref = orc.solve_system(s, tol=TOL)
    _, x, lam, it, st = run(s, "mixed", topo=t, start="diag")
    compare(s, ref, x, lam, it, st, it_slack=2)
    p = wl.protein_like(n_atoms=12000, seed=1051)
    tp = B.Topology(p.n_atoms, p.atom_i, p.atom_j, partition_min_constraints=2000)
    tun = tp.autotune(*to_dev(p), precision="mixed", start="diag", reps=3)
    assert tun["candidates"] >= 5 and tun["chosen"]["overlap"] in (0, 2, 3, 4, 6)
    assert tp.n_large == 1
    refp = orc.solve_system(p, tol=TOL)
    _, x, lam, it, st = run(p, "mixed", topo=tp, start="diag")
    assert st.tolist() == [B.CONVERGED]
    assert np.abs(x - refp.x).max() <= X_TOL
    assert np.all(np.abs(lam - refp.lam) <= LAM_RTOL * np.abs(refp.lam) + 1e-10 * np.abs(refp.lam).max())
