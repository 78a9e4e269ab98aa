"""Pins for the FP64 oracle: checks against facts other than the oracle itself.

Each test targets a family of plausible oracle mistakes:
  * two-atom closed form        -> factor-of-2 / mass-weighting / sign / root-choice errors
  * collinear chain closed form -> coupling signs s_k(a) s_l(a), wrong endpoint index
  * finite-difference Jacobian  -> transposed operands in A, G evaluated at the wrong x
  * quadratic convergence       -> any Jacobian error (inexact Newton converges linearly)
  * SHAKE cross-check           -> anything that changes the root on non-collinear geometry
  * brute-force root search     -> uniqueness of the root continuous with lambda = 0
  * invariants                  -> momentum / angular momentum / displacement span
  * pendulum worked example     -> the paper's printed energy errors (supplement Sec. 4)
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.special as ss

from oracle import ilves_oracle as orc
from paper_2503_13075_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------- helpers
def sigma_of_lambda(s, lam):
    """sigma(x(lambda)) by explicit loops over constraints (independent of the oracle)."""
    x = s.x_unc.copy()
    for k, (i, j) in enumerate(zip(s.atom_i, s.atom_j)):
        rho = s.x_old[i] - s.x_old[j]
        x[i] -= s.inv_mass[i] * 2.0 * rho * lam[k]
        x[j] += s.inv_mass[j] * 2.0 * rho * lam[k]
    out = np.empty(len(s.d))
    for k, (i, j) in enumerate(zip(s.atom_i, s.atom_j)):
        r = x[i] - x[j]
        out[k] = r.dot(r) - s.d[k] ** 2
    return out, x


def small_tree(seed, n):
    return wl.tree_molecules_of_sizes([n], seed=seed)


# ---------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("w1,w2", [(1.0, 1.0), (1 / 1.008, 1 / 12.011), (0.0, 1.0), (1 / 32.06, 1 / 1.008)])
def test_two_atom_closed_form(w1, w2):
    """|s - c rho|^2 = d^2 with c = 2 lambda (w1 + w2); the small root is the Newton root."""
    s = wl.two_atoms(d=0.1, w1=w1, w2=w2, seed=11, sigma=0.01)
    res = orc.solve_system(s)
    rho = s.x_old[0] - s.x_old[1]
    sv = s.x_unc[0] - s.x_unc[1]
    a, b, c0 = rho.dot(rho), sv.dot(rho), sv.dot(sv) - s.d[0] ** 2
    c = (b - math.sqrt(b * b - a * c0)) / a
    lam = c / (2.0 * (w1 + w2))
    assert res.status[0] == orc.CONVERGED
    assert abs(res.lam[0] - lam) <= 1e-12 * abs(lam)
    x_exp = s.x_unc.copy()
    x_exp[0] -= w1 * 2 * rho * lam
    x_exp[1] += w2 * 2 * rho * lam
    assert np.abs(res.x - x_exp).max() <= 1e-14
    # paper's multiplier convention: lambda_paper = -2 lambda / h^2 (g = -sigma/2, x_unc carries h^2)
    h = 0.002
    lam_paper = -2.0 * res.lam[0] / h**2
    Gp = -(s.x_old[0] - s.x_old[1])  # paper: dg/dq_a = -(q_a - q_b)
    x_paper = s.x_unc[0] - h * h * w1 * Gp * lam_paper
    assert np.allclose(x_paper, res.x[0], atol=1e-15)


def test_collinear_chain_closed_form():
    """All atoms and perturbations on one axis: r(lambda) is linear, lambda = B^-1 (s - d sign(rho))."""
    rng = np.random.default_rng(5)
    n = 12
    d = rng.uniform(0.1, 0.15, n - 1)
    xo = np.zeros((n, 3))
    xo[1:, 0] = np.cumsum(d)
    xu = xo.copy()
    xu[:, 0] += rng.normal(0, 0.004, n)
    w = 1.0 / rng.choice([1.008, 12.011, 15.999], n)
    ai = np.arange(n - 1, dtype=np.int32)
    aj = ai + 1
    # swap endpoints of a few constraints to exercise both signs
    flip = rng.random(n - 1) < 0.4
    ai2 = np.where(flip, aj, ai).astype(np.int32)
    aj2 = np.where(flip, ai, aj).astype(np.int32)
    res = orc.solve(xo, xu, w, ai2, aj2, d)
    rho = xo[ai2, 0] - xo[aj2, 0]
    svec = xu[ai2, 0] - xu[aj2, 0]
    B = np.zeros((n - 1, n - 1))
    for k in range(n - 1):
        for l in range(n - 1):
            for a in {ai2[k], aj2[k]} & {ai2[l], aj2[l]}:
                sk = 1.0 if a == ai2[k] else -1.0
                sl = 1.0 if a == ai2[l] else -1.0
                B[k, l] += 2.0 * rho[l] * sk * sl * w[a]
    lam = np.linalg.solve(B, svec - d * np.sign(rho))
    assert res.status[0] == orc.CONVERGED
    np.testing.assert_allclose(res.lam, lam, rtol=1e-9, atol=1e-14)


# ---------------------------------------------------------------------------- Jacobian
@pytest.mark.parametrize("seed,n", [(1, 8), (2, 25), (3, 40)])
def test_jacobian_matches_finite_differences(seed, n):
    """d sigma / d lambda = -A(x(lambda), x_old); sigma is quadratic so central differences are exact."""
    s = small_tree(seed, n)
    rng = np.random.default_rng(seed)
    lam = rng.normal(0, 1e-3, len(s.d))
    sig, x = sigma_of_lambda(s, lam)
    A = orc.newton_matrix(x, s.x_old, s.inv_mass, s.atom_i.astype(np.int64), s.atom_j.astype(np.int64)).toarray()
    h = 1e-4
    J = np.empty_like(A)
    for l in range(len(lam)):
        e = np.zeros_like(lam)
        e[l] = h
        J[:, l] = (sigma_of_lambda(s, lam + e)[0] - sigma_of_lambda(s, lam - e)[0]) / (2 * h)
    np.testing.assert_allclose(-J, A, atol=1e-9 * np.abs(A).max())
    # structurally symmetric (pattern of the line graph), numerically nonsymmetric
    assert np.array_equal(A != 0, A.T != 0)
    assert np.abs(A - A.T).max() > 0


def test_quadratic_convergence():
    """Newton: e_{l+1} / e_l^2 stays bounded (supplement Sec. 2.3, quadratic convergence)."""
    for s in (wl.chain64(), small_tree(9, 150)):
        h = orc.solve_system(s, tol=1e-15).history
        ratios = [h[l + 1] / h[l] ** 2 for l in range(len(h) - 1) if h[l + 1] > 1e-13]
        assert len(ratios) >= 2
        assert max(ratios) < 50.0, ratios
        assert h[-1] < 1e-13


# ---------------------------------------------------------------------------- independent solvers
def shake(s, tol=1e-13, max_sweeps=5000):
    """SHAKE: nonlinear Gauss-Seidel, one exact two-atom solve per constraint per sweep."""
    x = s.x_unc.copy()
    lam = np.zeros(len(s.d))
    for _ in range(max_sweeps):
        worst = 0.0
        for k, (i, j) in enumerate(zip(s.atom_i, s.atom_j)):
            rho = s.x_old[i] - s.x_old[j]
            r = x[i] - x[j]
            worst = max(worst, abs(r.dot(r) - s.d[k] ** 2) / s.d[k] ** 2)
            wsum = s.inv_mass[i] + s.inv_mass[j]
            a, b, c0 = rho.dot(rho), r.dot(rho), r.dot(r) - s.d[k] ** 2
            c = (b - math.sqrt(b * b - a * c0)) / a
            dl = c / (2 * wsum)
            x[i] -= s.inv_mass[i] * 2 * rho * dl
            x[j] += s.inv_mass[j] * 2 * rho * dl
            lam[k] += dl
        if worst <= tol:
            return x, lam
    raise AssertionError("SHAKE did not converge")


@pytest.mark.parametrize("maker", [wl.chain64, lambda: small_tree(21, 60), lambda: small_tree(22, 120)])
def test_shake_agreement(maker):
    """ILVES-M and SHAKE solve the same equations (supplement Sec. 2.3 / Sec. 3): same root."""
    s = maker()
    res = orc.solve_system(s, tol=1e-13)
    x_sh, lam_sh = shake(s)
    assert np.abs(res.x - x_sh).max() <= 1e-10
    np.testing.assert_allclose(res.lam, lam_sh, rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("seed", [31, 32])
def test_bruteforce_root_is_unique_near_zero(seed):
    """Tiny molecules: root finding from random starts lands on the oracle's root or far away."""
    s = small_tree(seed, 6)
    res = orc.solve_system(s)
    f = lambda lam: sigma_of_lambda(s, lam)[0]
    rng = np.random.default_rng(seed)
    scale = np.abs(res.lam).max()
    near = 0
    for _ in range(12):
        start = rng.normal(0, scale, len(s.d))
        sol = so.fsolve(f, start, xtol=1e-14, full_output=True)
        if sol[2] != 1:
            continue
        if np.abs(sol[0]).max() < 3 * scale:
            near += 1
            np.testing.assert_allclose(sol[0], res.lam, rtol=1e-7, atol=1e-12 * scale)
    assert near >= 3


# ---------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("maker", [wl.chain64, lambda: wl.tree_batch(n_mol=16, seed=3)])
def test_invariants(maker):
    s = maker()
    res = orc.solve_system(s)
    m = 1.0 / s.inv_mass
    dx = res.x - s.x_unc
    # momentum: sum_a m_a dx_a = 0 (each constraint force acts pairwise)
    scale = np.abs(m[:, None] * dx).sum()
    assert np.abs((m[:, None] * dx).sum(axis=0)).max() <= 1e-13 * scale
    # angular momentum about the origin with the x_old lever arms: forces are parallel to rho_k
    L = np.cross(s.x_old, m[:, None] * dx).sum(axis=0)
    assert np.abs(L).max() <= 1e-12 * np.abs(np.cross(s.x_old, m[:, None] * dx)).sum()
    # displacement lies in span(M^-1 G(x_old)^T): least squares returns the same lambda, ~0 residual
    G0 = orc.constraint_jacobian(s.x_old, s.atom_i.astype(np.int64), s.atom_j.astype(np.int64), s.n_atoms)
    B = -(np.repeat(s.inv_mass, 3)[:, None] * G0.T.toarray())
    lam_ls, *_ = np.linalg.lstsq(B, dx.ravel(), rcond=None)
    assert np.abs(B @ lam_ls - dx.ravel()).max() <= 1e-15 + 1e-12 * np.abs(dx).max()
    np.testing.assert_allclose(lam_ls, res.lam, rtol=1e-8, atol=1e-14)
    assert orc.max_relative_violation(res.x, s.atom_i, s.atom_j, s.d) <= 1e-12


def test_feasible_input_needs_no_solve():
    s = wl.chain64()
    s.x_unc = s.x_old + np.array([0.3, -0.2, 0.1])
    res = orc.solve_system(s)
    assert res.iterations[0] == 0 and res.status[0] == orc.CONVERGED
    assert np.all(res.lam == 0.0)


def test_relabelling_and_endpoint_swap():
    s = wl.tree_batch(n_mol=6, seed=4)
    res = orc.solve_system(s)
    rng = np.random.default_rng(0)
    pa = rng.permutation(s.n_atoms)  # new index of old atom a is inv[a]
    inv = np.empty_like(pa)
    inv[pa] = np.arange(s.n_atoms)
    pc = rng.permutation(s.n_constraints)
    swap = rng.random(s.n_constraints) < 0.5
    ai = np.where(swap, s.atom_j, s.atom_i)[pc]
    aj = np.where(swap, s.atom_i, s.atom_j)[pc]
    r2 = orc.solve(s.x_old[pa], s.x_unc[pa], s.inv_mass[pa], inv[ai], inv[aj], s.d[pc])
    np.testing.assert_allclose(r2.x, res.x[pa], atol=1e-13)
    np.testing.assert_allclose(r2.lam, res.lam[pc], rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------------------- degenerate cases
def test_edge_cases():
    empty = orc.solve(np.zeros((3, 3)), np.ones((3, 3)), np.ones(3), [], [], [])
    assert empty.iterations.size == 0 and np.all(empty.x == 1.0)
    # atoms outside any constraint pass through untouched
    s = wl.chain64()
    xo = np.vstack([s.x_old, [[5.0, 5.0, 5.0]]])
    xu = np.vstack([s.x_unc, [[5.1, 5.0, 5.0]]])
    r = orc.solve(xo, xu, np.append(s.inv_mass, 1.0), s.atom_i, s.atom_j, s.d)
    assert np.all(r.x[-1] == xu[-1]) and r.status[0] == orc.CONVERGED
    # non-finite input
    xu2 = s.x_unc.copy()
    xu2[3, 1] = np.nan
    assert orc.solve(s.x_old, xu2, s.inv_mass, s.atom_i, s.atom_j, s.d).status[0] == orc.NONFINITE
    # unreachable tolerance -> max_iter
    r = orc.solve_system(s, tol=1e-30, max_iter=7)
    assert r.status[0] == orc.MAX_ITER and r.iterations[0] == 7
    # r . rho = 0 at lambda = 0: singular Newton matrix
    xo = np.array([[0.0, 0, 0], [0.1, 0, 0]])
    xu = np.array([[0.0, 0, 0], [0.0, 0.12, 0]])
    r = orc.solve(xo, xu, np.ones(2), [0], [1], [0.1])
    assert r.status[0] == orc.SINGULAR


# ---------------------------------------------------------------------------- paper worked example
def _pendulum_max_rel_energy_error(steps_per_period, periods=2.0):
    """Leap-frog pendulum with the oracle as constraint solver (supplement Sec. 4 tables)."""
    m, l, g = 1.0, 1.0, 9.82
    pivot = np.array([0.0, l, 0.0])
    q = np.zeros(3)
    v0 = np.array([1.0, 0.0, 0.0])
    theta = math.acos(1.0 - v0.dot(v0) / (2.0 * g * l))
    period = 4.0 * math.sqrt(l / g) * ss.ellipk(math.sin(theta / 2.0) ** 2)
    h = period / steps_per_period
    f = np.array([0.0, -m * g, 0.0])
    vh = v0 - 0.5 * h * (f / m + v0.dot(v0) / l * (pivot - q) / l)  # v_{-1/2}
    e0 = 0.5 * m * v0.dot(v0) + m * g * q[1]
    x_old = np.stack([pivot, q])
    inv = np.array([0.0, 1.0 / m])
    worst = 0.0
    for _ in range(int(steps_per_period * periods)):
        x_unc = x_old.copy()
        x_unc[1] = x_old[1] + h * vh + h * h * f / m
        res = orc.solve(x_old, x_unc, inv, [0], [1], [l], tol=1e-12)
        assert res.status[0] == orc.CONVERGED
        v_new = (res.x[1] - x_old[1]) / h
        vk = 0.5 * (vh + v_new)
        n = (x_old[1] - pivot) / np.linalg.norm(x_old[1] - pivot)
        vk = vk - vk.dot(n) * n  # velocity at t_k tangent to the constraint
        e = 0.5 * m * vk.dot(vk) + m * g * x_old[1][1]
        worst = max(worst, abs(e - e0) / e0)
        vh, x_old = v_new, res.x
    return worst


def test_pendulum_energy_error_matches_paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "pendulum_energy.txt"))
    errs = []
    for spp, log2_err in rows:
        e = _pendulum_max_rel_energy_error(int(spp))
        errs.append(e)
        assert abs(math.log2(e) - log2_err) < 0.3, (spp, math.log2(e))
    # second order in h: halving h divides the error by ~4
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4


# ---------------------------------------------------------------------------- ILVES-F
@pytest.mark.parametrize("maker", [wl.chain64, lambda: wl.tree_batch(n_mol=30, seed=7)])
def test_chord_method_reaches_the_newton_root_linearly(maker):
    """ILVES-F (supplement Sec. 3): same equations, same root; linear convergence."""
    s = maker()
    newton = orc.solve_system(s, tol=1e-13)
    chord = orc.solve_system(s, tol=1e-13, max_iter=60, method="chord")
    assert np.all(chord.status == orc.CONVERGED)
    assert np.abs(chord.x - newton.x).max() <= 1e-10
    np.testing.assert_allclose(chord.lam, newton.lam, rtol=1e-7, atol=1e-14)
    assert chord.iterations.mean() > newton.iterations.mean()
    if s.n_molecules == 1:  # linear: successive error ratios stay bounded below 1
        h = [e for e in chord.history if e > 1e-12]
        ratios = [b / a for a, b in zip(h, h[1:])]
        assert max(ratios[1:]) < 0.5


@pytest.mark.parametrize("seed,n", [(41, 10), (42, 30)])
def test_chord_matrix_is_the_reference_jacobian(seed, n):
    """ILVES-F's constant matrix is A(x_old, x_old) (supplement Sec. 3): the Jacobian, negated,
    of lambda -> sigma(x_old - M^-1 G(x_old)^T lambda) at lambda = 0.  The Jacobian comes from
    central differences of this file's own loop evaluation (exact: the map is quadratic).  The
    matrix is symmetric and differs from the first Newton matrix A(x_unc, x_old); and the
    oracle's chord iterates are lambda_{l+1} = lambda_l + A0^-1 sigma(x(lambda_l)) with it."""
    s = small_tree(seed, n)
    ai, aj = s.atom_i.astype(np.int64), s.atom_j.astype(np.int64)
    at_ref = wl.System("ref", s.x_old, s.x_old.copy(), s.inv_mass, s.atom_i, s.atom_j, s.d)
    nc = len(s.d)
    h = 1e-4
    J = np.empty((nc, nc))
    for l in range(nc):
        e = np.zeros(nc)
        e[l] = h
        J[:, l] = (sigma_of_lambda(at_ref, e)[0] - sigma_of_lambda(at_ref, -e)[0]) / (2 * h)
    A0 = orc.chord_matrix(s.x_old, s.inv_mass, ai, aj).toarray()
    np.testing.assert_allclose(A0, -J, atol=1e-9 * np.abs(A0).max())
    assert np.abs(A0 - A0.T).max() <= 1e-15 * np.abs(A0).max()
    A_unc = orc.newton_matrix(s.x_unc, s.x_old, s.inv_mass, ai, aj).toarray()
    assert np.abs(A_unc - A0).max() > 1e-3 * np.abs(A0).max()
    lam = np.zeros(nc)
    for k in (1, 2, 3):
        sig, _ = sigma_of_lambda(s, lam)
        lam = lam + np.linalg.solve(-J, sig)
        got = orc.solve_system(s, tol=1e-30, max_iter=k, method="chord")
        assert got.status[0] == orc.MAX_ITER and got.iterations[0] == k
        np.testing.assert_allclose(got.lam, lam, rtol=1e-8, atol=1e-9 * np.abs(lam).max())


def test_molecules_are_numbered_by_smallest_atom():
    """Molecule ids follow the smallest atom of each component, whatever the constraint order:
    {6, 7, 8} listed first is molecule 2, {0, 2} molecule 0, {3, 4, 5} molecule 1; atom 1 is
    in no constraint.  Per-molecule outputs of the solve follow the same numbering."""
    ai = np.array([8, 7, 4, 2, 3])
    aj = np.array([7, 6, 5, 0, 4])
    mol, n = orc.molecules(9, ai, aj)
    assert n == 3 and mol.tolist() == [2, 2, 1, 0, 1]
    # molecule 0 feasible (no solve), molecules 1 and 2 perturbed; atom 1 passes through
    rng = np.random.default_rng(3)
    x_old = np.cumsum(rng.normal(0.0, 0.1, (9, 3)), axis=0)
    r = x_old[ai] - x_old[aj]
    d = np.sqrt(np.einsum("ij,ij->i", r, r))
    x_unc = x_old + rng.normal(0.0, 0.004, (9, 3))
    x_unc[[0, 2]] = x_old[[0, 2]] + 0.01  # a rigid shift keeps {0, 2} feasible
    res = orc.solve(x_old, x_unc, np.ones(9), ai, aj, d)
    assert res.mol_of_constraint.tolist() == [2, 2, 1, 0, 1]
    assert res.iterations[0] == 0 and res.iterations[1] > 0 and res.iterations[2] > 0
    assert np.array_equal(res.x[1], x_unc[1])


def test_average_relative_error_follows_the_paper_formula():
    """Main text, Results: (1 / (2 n N_s)) sum_k sum_i |d_i^2 - |q_a - q_b|^2| / d_i^2.  Three bonds
    (d = 1, 1, 2) at squared lengths 1.02, 0.99 and 4.04 in one step: (0.02 + 0.01 + 0.01) / 6."""
    x = np.zeros((6, 3))
    x[1, 0] = math.sqrt(1.02)
    x[2, 0], x[3, 0] = 10.0, 10.0 + math.sqrt(0.99)
    x[4, 0], x[5, 0] = 20.0, 20.0 + math.sqrt(4.04)
    ai, aj, d = np.array([0, 2, 4]), np.array([1, 3, 5]), np.array([1.0, 1.0, 2.0])
    assert orc.average_relative_error(x, ai, aj, d) == pytest.approx(0.04 / 6.0, rel=1e-12)
    assert orc.max_relative_violation(x, ai, aj, d) == pytest.approx(0.02, rel=1e-12)


# ---------------------------------------------------------------------------- overlapping domains
def _chain_indices(n):
    return np.arange(n - 1), np.arange(1, n)


def test_greedy_partition_of_a_chain_is_even():
    """On a path every boundary cuts one constraint, so the greedy partition (supplement
    Sec. 3) ends each part at the size nearest its target: equal parts when they divide."""
    ai, aj = _chain_indices(600)
    assert orc.greedy_partition(600, ai, aj, 6) == [0, 100, 200, 300, 400, 500, 600]


def test_greedy_partition_avoids_cuts_within_its_window():
    """A part boundary inside a 3-cycle cuts two constraints; the partition moves it to a
    single-cut position within maxDeviation of the target (cutPenalty 10 outweighs the size
    term)."""
    n = 200
    ai, aj = list(range(n - 1)), list(range(1, n))
    ai.append(99)  # triangle 99-100-101: a boundary at 100 or 101 cuts two constraints
    aj.append(101)
    b = orc.greedy_partition(n, np.array(ai), np.array(aj), 2)
    assert b == [0, 102, 200] or b == [0, 99, 200]


def test_overlapping_domains_of_a_chain():
    """Chain of 40 atoms in parts [0, 10), [10, 20), ...: with overlap I the domain of part
    [a, b) holds atoms [a - I, b + I) (clipped) and the constraints between them; the part
    owns the constraints (k, k + 1) with a <= k < b."""
    n, I = 40, 3
    ai, aj = _chain_indices(n)
    doms = orc.opm_domains(n, ai, aj, [0, 10, 20, 30, 40], I)
    for dpart, (cons, owned) in enumerate(doms):
        a, b = 10 * dpart, 10 * dpart + 10
        lo, hi = max(0, a - I), min(n, b + I)
        assert cons.tolist() == list(range(lo, hi - 1))
        assert cons[owned].tolist() == [k for k in range(a, b) if k < n - 1]


@pytest.mark.parametrize("overlap", [2, 4])
def test_opm_reaches_the_newton_root(overlap):
    """The overlapping-domain quasi-Newton iteration solves the same constraint equations: it
    converges to ILVES-M's root (supplement Sec. 3), in more iterations for a small overlap."""
    s = wl.protein_like(n_atoms=5000, seed=1003)
    ref = orc.solve_system(s, tol=1e-13)
    got = orc.solve_system(s, tol=1e-13, overlap=overlap, part_constraints=300, part_min=1000)
    assert np.all(got.status == orc.CONVERGED)
    assert np.abs(got.x - ref.x).max() <= 1e-10
    np.testing.assert_allclose(got.lam, ref.lam, rtol=1e-7, atol=1e-12 * np.abs(ref.lam).max())
    assert got.iterations[0] >= ref.iterations[0]


def test_opm_with_domains_covering_the_molecule_is_newton():
    """When every domain holds the whole molecule, each domain's local solve is the full
    Newton solve and the owned entries assemble A^-1 sigma: the iterates are Newton's."""
    s = wl.protein_like(n_atoms=1500, seed=1004)
    ref = orc.solve_system(s, tol=1e-13)
    got = orc.solve_system(s, tol=1e-13, overlap=10_000, part_constraints=400, part_min=500)
    assert np.array_equal(got.iterations, ref.iterations)
    np.testing.assert_allclose(got.history, ref.history, rtol=1e-6, atol=1e-15)
