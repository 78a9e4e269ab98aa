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


def solve(x_old, x_unc, inv_mass, atom_i, atom_j, d, tol=1e-12, max_iter=25, lambda0=None, method="newton"):
    """ILVES-M exact Newton (or ILVES-F, method="chord") on every molecule; see the module docstring."""
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
    active = np.ones(n_mol, bool)  # molecules still iterating
    history = []
    chord_lu = None
    if method == "chord":  # A(x_old, x_old), factorised once
        chord_lu = spla.splu(chord_matrix(x_old, inv_mass, atom_i, atom_j), permc_spec="COLAMD")
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
