"""FP64 CPU oracle for ILVES-M's per-step constraint solve (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
``--impl reference`` legs) may import this module.  The CUDA library never calls it,
and it shares no code with the CUDA path; the only common dependency is the seeded
input generator module, which contains none of the method's arithmetic.

What it computes (paper, supplement Sec. 2.2-2.3 and Sec. 4):

* Constraint function, Sec. 2.2 Eq. (bond constraint g_i): the library uses the
  scaled form  sigma_k(x) = |x_i - x_j|^2 - d_k^2  (= -2 g_k), whose Jacobian G(x)
  has the 3-blocks  +2 r_k  at atom i and  -2 r_k  at atom j,  r_k = x_i - x_j.
* Position map, Sec. 2.3 Eq. (phi_k): with h^2 absorbed into lambda,
  x(lambda) = x_unc - M^-1 G(x_old)^T lambda,  x_unc = q_k + h v_{k-1/2} + h^2 M^-1 f.
* Newton matrix, Sec. 2.3 Eq. (A(x, y)): A = G(x) M^-1 G(x_old)^T (the paper's
  -h^2 factor is absorbed by the same rescaling), sparse, structurally symmetric,
  numerically nonsymmetric.
* ILVES-M Newton iteration, Sec. 2.3 (Newton equations for the constraint equation):
  A(x(lambda_l), x_old) delta_l = sigma(x(lambda_l)),  lambda_{l+1} = lambda_l + delta_l
  (the paper writes z = -delta with its sign convention), started from lambda_0 = 0.
* ILVES-F (``method="chord"``), supplement Sec. 3: the simplified Newton / chord method
  with the constant symmetric matrix A(x_old, x_old), factorised once per solve.
* Overlapping Partitioning Method (``overlap=I > 0``), supplement Sec. 3: a molecule with
  at least ``part_min`` constraints is cut into parts by the greedy k-way partition of its
  atoms (``greedy_partition``); part d owns the constraints whose smaller atom it holds, its
  domain adds the atoms within I edges, and each Newton step replaces A^-1 sigma by the
  domains' local solves with A restricted to the constraints between domain atoms, keeping
  each domain's owned entries: a quasi-Newton iteration with the same root.
* Stopping rule, Sec. 4: stop when max_k |sigma_k| / d_k^2 <= tol or after max_iter
  linear solves.  The convergence test happens before each solve, so an already
  feasible x_unc needs 0 solves.

Each connected component of the constraint graph (a molecule) converges on its own
and reports its own iteration count and status.  Molecules are numbered by their
smallest atom index.  The paper's multipliers are lambda_paper = -2 lambda / h^2.

Steps that use library primitives: the sparse products G M^-1 G0^T (scipy.sparse
matmul) and the linear solve (scipy.sparse.linalg.splu, SuperLU with partial
pivoting).  No blocking, fusion or reordering beyond those calls.
"""
from __future__ import annotations

from dataclasses import dataclass

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

CONVERGED, MAX_ITER, SINGULAR, NONFINITE = 0, 1, 2, 3
STATUS_NAMES = {CONVERGED: "converged", MAX_ITER: "max_iter", SINGULAR: "singular", NONFINITE: "nonfinite"}


@dataclass
class OracleResult:
    x: np.ndarray  # (n_atoms, 3) constrained positions
    lam: np.ndarray  # (n_c,) multipliers, library convention
    iterations: np.ndarray  # (n_mol,) linear solves per molecule
    status: np.ndarray  # (n_mol,) CONVERGED / MAX_ITER / SINGULAR / NONFINITE
    mol_of_constraint: np.ndarray  # (n_c,) molecule id of each constraint
    history: list  # per Newton iterate l: max relative violation over molecules still active


def molecules(n_atoms, atom_i, atom_j):
    """Connected components of the constraint graph G (supplement Sec. 3).

    Returns (mol_of_constraint, n_mol); molecules are numbered by smallest atom index.
    Atoms without constraints belong to no molecule.
    """
    atom_i = np.asarray(atom_i, np.int64)
    atom_j = np.asarray(atom_j, np.int64)
    n_c = atom_i.size
    if n_c == 0:
        return np.zeros(0, np.int64), 0
    adj = sp.coo_matrix((np.ones(n_c), (atom_i, atom_j)), shape=(n_atoms, n_atoms))
    _, label = csg.connected_components(adj, directed=False)
    used = np.zeros(n_atoms, bool)
    used[atom_i] = True
    used[atom_j] = True
    # renumber labels in order of each component's smallest atom
    first = {}
    for a in np.flatnonzero(used):
        first.setdefault(int(label[a]), len(first))
    remap = np.array([first.get(int(lab), -1) for lab in range(label.max() + 1)])
    return remap[label[atom_i]], len(first)


def constraint_jacobian(x, atom_i, atom_j, n_atoms):
    """G(x): n_c x 3 n_atoms sparse, rows  +2 r_k at atom i,  -2 r_k at atom j (Sec. 2.2)."""
    n_c = atom_i.size
    r = x[atom_i] - x[atom_j]
    rows = np.repeat(np.arange(n_c), 6)
    cols = np.concatenate([3 * atom_i[:, None] + np.arange(3), 3 * atom_j[:, None] + np.arange(3)], axis=1).ravel()
    vals = np.concatenate([2.0 * r, -2.0 * r], axis=1).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_c, 3 * n_atoms))


def positions(lam, x_unc, inv_mass, G0):
    """x(lambda) = x_unc - M^-1 G(x_old)^T lambda  (Sec. 2.3 Eq. phi_k, h^2 absorbed)."""
    minv = np.repeat(inv_mass, 3)
    return x_unc - (minv * (G0.T @ lam)).reshape(-1, 3)


def violation(x, atom_i, atom_j, d):
    """sigma_k = |x_i - x_j|^2 - d_k^2."""
    r = x[atom_i] - x[atom_j]
    return np.einsum("ij,ij->i", r, r) - d * d


def newton_matrix(x, x_old, inv_mass, atom_i, atom_j):
    """A(x, x_old) = G(x) M^-1 G(x_old)^T  (Sec. 2.3 Eq. defining A)."""
    n_atoms = x.shape[0]
    G = constraint_jacobian(x, atom_i, atom_j, n_atoms)
    G0 = constraint_jacobian(x_old, atom_i, atom_j, n_atoms)
    Minv = sp.diags(np.repeat(inv_mass, 3))
    return (G @ Minv @ G0.T).tocsc()


def chord_matrix(x_old, inv_mass, atom_i, atom_j):
    """ILVES-F's constant matrix A(x_old, x_old) = G(x_old) M^-1 G(x_old)^T (supplement Sec. 3,
    the approximation of A(phi_k(lambda), q_k) by A(q_k, q_k)); symmetric."""
    return newton_matrix(x_old, x_old, inv_mass, atom_i, atom_j)


def greedy_partition(n_atoms, atom_i, atom_j, n_parts, max_dev=0.05, cut_penalty=10.0):
    """Greedy k-way partition of the constraint graph (supplement Sec. 3; maxDeviation 0.05,
    cutPenalty 10).  Atoms are taken in index order; part p starts at a0 and, with target =
    (atoms left) / (parts left), ends before atom e for the e in [a0 + target (1 - max_dev),
    a0 + target (1 + max_dev)] (at least a0 + 1, at most n_atoms - 1) that minimises
    cut_penalty * cut(e) + |(e - a0) - target|, cut(e) = number of constraints joining an
    atom of [a0, e) to an atom >= e (the first such e on ties).  Returns the part bounds
    (n_parts + 1 increasing atom indices from 0 to n_atoms; fewer if atoms run out)."""
    lo_a = np.minimum(atom_i, atom_j)
    hi_a = np.maximum(atom_i, atom_j)
    bounds = [0]
    a0 = 0
    for p in range(n_parts - 1):
        if a0 >= n_atoms:
            break
        target = (n_atoms - a0) / (n_parts - p)
        lo = max(a0 + 1, int(math.floor(a0 + target * (1.0 - max_dev))))
        hi = min(n_atoms - 1, int(math.ceil(a0 + target * (1.0 + max_dev))))
        best_e, best = min(n_atoms - 1, max(lo, a0 + 1)), float("inf")
        for e in range(lo, hi + 1):
            cut = int(np.count_nonzero((lo_a >= a0) & (lo_a < e) & (hi_a >= e)))
            score = cut_penalty * cut + abs((e - a0) - target)
            if score < best:
                best, best_e = score, e
        if best_e <= a0:
            break
        bounds.append(best_e)
        a0 = best_e
    bounds.append(n_atoms)
    return bounds


def opm_domains(n_atoms, atom_i, atom_j, bounds, overlap):
    """Domains of the Overlapping Partitioning Method (supplement Sec. 3) for one molecule with
    local atoms 0..n_atoms-1: per part d, (constraints between domain atoms ascending, owned
    flags), the domain being the part's atoms and every atom within `overlap` edges of them;
    part d owns a constraint when it holds the constraint's smaller atom."""
    adj = sp.coo_matrix((np.ones(len(atom_i)), (atom_i, atom_j)), shape=(n_atoms, n_atoms)).tocsr()
    adj = (adj + adj.T).tocsr()
    part = np.zeros(n_atoms, np.int64)
    for dpart in range(len(bounds) - 1):
        part[bounds[dpart]:bounds[dpart + 1]] = dpart
    out = []
    for dpart in range(len(bounds) - 1):
        dist = csg.dijkstra(adj, directed=False, unweighted=True, limit=overlap + 0.5, min_only=True,
                            indices=np.arange(bounds[dpart], bounds[dpart + 1]))
        inside = np.isfinite(dist)
        cons = np.flatnonzero(inside[atom_i] & inside[atom_j])
        owned = part[np.minimum(atom_i[cons], atom_j[cons])] == dpart
        out.append((cons, owned))
    return out


def _opm_delta(A, sigma, domains):
    """One quasi-Newton step of the Overlapping Partitioning Method: each domain solves its
    restriction of A delta = sigma and keeps its owned entries; None if a local system is
    singular."""
    delta = np.zeros_like(sigma)
    for cons, owned in domains:
        try:
            z = spla.splu(A[cons][:, cons].tocsc(), permc_spec="COLAMD").solve(sigma[cons])
        except RuntimeError:
            return None
        if not np.all(np.isfinite(z)):
            return None
        delta[cons[owned]] = z[owned]
    return delta


def solve(x_old, x_unc, inv_mass, atom_i, atom_j, d, tol=1e-12, max_iter=25, lambda0=None, method="newton",
          overlap=0, part_constraints=256, part_min=4096):
    """ILVES-M exact Newton (or ILVES-F, method="chord") on every molecule, or the
    overlapping-domain quasi-Newton (overlap > 0) on molecules of at least part_min
    constraints; see the module docstring."""
    x_old = np.asarray(x_old, np.float64).reshape(-1, 3)
    x_unc = np.asarray(x_unc, np.float64).reshape(-1, 3)
    inv_mass = np.asarray(inv_mass, np.float64)
    atom_i = np.asarray(atom_i, np.int64)
    atom_j = np.asarray(atom_j, np.int64)
    d = np.asarray(d, np.float64)
    n_atoms, n_c = x_old.shape[0], atom_i.size
    mol, n_mol = molecules(n_atoms, atom_i, atom_j)
    iters = np.zeros(n_mol, np.int64)
    status = np.full(n_mol, MAX_ITER, np.int64)
    if n_c == 0:
        return OracleResult(x_unc.copy(), np.zeros(0), iters, status, mol, [])
    G0 = constraint_jacobian(x_old, atom_i, atom_j, n_atoms)
    lam = np.zeros(n_c) if lambda0 is None else np.asarray(lambda0, np.float64).copy()
    # overlapping domains of the large molecules, in global constraint ids
    opm = {}
    if overlap > 0:
        for m in range(n_mol):
            cidx = np.flatnonzero(mol == m)
            if cidx.size < part_min:
                continue
            atoms = np.unique(np.concatenate([atom_i[cidx], atom_j[cidx]]))  # local atom = rank
            li = np.searchsorted(atoms, atom_i[cidx])
            lj = np.searchsorted(atoms, atom_j[cidx])
            n_parts = max(2, -(-cidx.size // part_constraints))
            bounds = greedy_partition(atoms.size, li, lj, n_parts)
            opm[m] = [(cidx[c], o) for c, o in opm_domains(atoms.size, li, lj, bounds, overlap)]
    chord_A0 = None
    active = np.ones(n_mol, bool)  # molecules still iterating
    history = []
    chord_lu = None
    if method == "chord":  # A(x_old, x_old), factorised once
        chord_A0 = chord_matrix(x_old, inv_mass, atom_i, atom_j)
        chord_lu = spla.splu(chord_A0, permc_spec="COLAMD")
    elif method != "newton":
        raise ValueError(method)
    for it in range(max_iter + 1):
        x = positions(lam, x_unc, inv_mass, G0)
        sigma = violation(x, atom_i, atom_j, d)
        rel = np.abs(sigma) / (d * d)
        mol_rel = np.zeros(n_mol)
        np.maximum.at(mol_rel, mol, np.where(np.isfinite(rel), rel, np.inf))
        if not active.any():
            break
        history.append(float(mol_rel[active].max()))
        bad = np.zeros(n_mol, bool)
        np.logical_or.at(bad, mol, ~np.isfinite(sigma))
        newly_bad = active & bad
        status[newly_bad] = NONFINITE
        iters[newly_bad] = it
        active &= ~bad
        done = active & (mol_rel <= tol)
        status[done] = CONVERGED
        iters[done] = it
        active &= ~done
        if not active.any() or it == max_iter:
            break
        # Newton step on the still-active molecules; finished ones keep lambda fixed
        row_active = active[mol]
        rhs = np.where(row_active, sigma, 0.0)
        if chord_lu is not None:  # blocks are independent: finished molecules get delta = 0
            delta = np.where(row_active, chord_lu.solve(rhs), 0.0)
            singular_mols = np.zeros(n_mol, bool)
        else:
            A = newton_matrix(x, x_old, inv_mass, atom_i, atom_j)
            A = _restrict(A, row_active)
            delta, singular_mols = _sparse_solve(A, rhs, mol, n_mol, row_active)
        for m, doms in opm.items():  # overlapping domains replace the exact step
            if not active[m]:
                continue
            dm = _opm_delta(chord_A0.tocsr() if chord_lu is not None else newton_matrix(x, x_old, inv_mass, atom_i,
                                                                                          atom_j).tocsr(), rhs, doms)
            rows = mol == m
            if dm is None:
                singular_mols[m] = True
            else:
                delta[rows] = dm[rows]
        if singular_mols.any():
            status[singular_mols] = SINGULAR
            iters[singular_mols] = it
            active &= ~singular_mols
            delta[singular_mols[mol]] = 0.0
        lam = lam + np.where(active[mol], delta, 0.0)
    iters[active] = max_iter
    x = positions(lam, x_unc, inv_mass, G0)
    return OracleResult(x, lam, iters, status, mol, history)


def _restrict(A, row_active):
    """Replace rows/cols of finished molecules by the identity (their delta is then 0)."""
    keep = sp.diags(row_active.astype(np.float64))
    eye = sp.diags((~row_active).astype(np.float64))
    return (keep @ A @ keep + eye).tocsc()


def _sparse_solve(A, rhs, mol, n_mol, row_active):
    """Solve A delta = rhs; molecules whose block is singular are reported, not solved."""
    singular = np.zeros(n_mol, bool)
    try:
        delta = spla.splu(A, permc_spec="COLAMD").solve(rhs)
        if np.all(np.isfinite(delta)):
            return delta, singular
    except RuntimeError:
        pass
    # locate the singular molecule(s) by solving block by block
    delta = np.zeros_like(rhs)
    order = np.argsort(mol, kind="stable")
    bounds = np.searchsorted(mol[order], np.arange(n_mol + 1))
    for m in range(n_mol):
        idx = order[bounds[m]:bounds[m + 1]]
        if idx.size == 0 or not row_active[idx[0]]:
            continue
        blk = A[idx][:, idx].tocsc()
        try:
            sol = spla.splu(blk).solve(rhs[idx])
            if not np.all(np.isfinite(sol)):
                raise RuntimeError
            delta[idx] = sol
        except RuntimeError:
            singular[m] = True
    return delta, singular


def solve_system(system, **kw):
    """Convenience wrapper taking a ``workloads.System``."""
    return solve(system.x_old, system.x_unc, system.inv_mass, system.atom_i, system.atom_j, system.d, **kw)


def average_relative_error(x, atom_i, atom_j, d):
    """Paper's reported accuracy metric (main text, Results): mean |d^2 - |r|^2| / d^2 / 2."""
    s = violation(np.asarray(x).reshape(-1, 3), np.asarray(atom_i), np.asarray(atom_j), np.asarray(d))
    return float(np.mean(np.abs(s) / (d * d)) / 2.0) if s.size else 0.0


def max_relative_violation(x, atom_i, atom_j, d):
    s = violation(np.asarray(x).reshape(-1, 3), np.asarray(atom_i), np.asarray(atom_j), np.asarray(d))
    return float(np.max(np.abs(s) / (d * d))) if s.size else 0.0
