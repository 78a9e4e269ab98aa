"""Seeded synthetic constrained-molecule workloads.

This module only *draws inputs*: topologies (which atom pairs are constrained),
target distances, inverse masses, feasible reference positions ``x_old`` and
perturbed unconstrained positions ``x_unc``.  It contains none of the solver's
arithmetic, so both the CUDA path and the CPU oracle may use it.

The shapes follow the systems the paper simulates (supplement Sec. 6, table of
simulated systems): lipid-like tree molecules of ~100 atoms with about one
constraint per atom, and protein-like single systems of ~1e5 atoms with bond
constraints plus H-X-H triangle-closing distances (``constraints=h-angles``,
main text Sec. "Results").  All bonds are constrained ("all-bonds").

Workloads (seed = 1000 + workload id unless given):

* ``chain64``       -- one unbranched carbon chain, 64 atoms / 63 bonds of 0.153 nm,
                       bond angle 111 deg, uniform dihedrals, perturbation N(0, 0.002 nm).
* ``tree_batch``    -- 4096 independent tree molecules of U{20..200} atoms, elements
                       H/C/N/O/S with p = .50/.30/.08/.10/.02, valence caps C4/N3/O2/S2,
                       H only as leaves; X-H bonds 0.100 nm, heavy-heavy U(0.122, 0.153);
                       perturbation N(0, 0.003 nm).
* ``protein_like``  -- one connected system of ~1e5 atoms: backbone chain with seeded
                       side chains, all bonds plus H-X-H distances on every CH3 / NH2 /
                       NH3 group (3-cycles and K4 cliques); perturbation N(0, 0.004 nm).
* ``chain_batch``   -- many chain64-distribution chains (learned warm start data).
* ``serving_sizes`` -- log-uniform request sizes for the serving loop.

Layout of every system: atoms of one molecule are contiguous, constraints of one
molecule are contiguous and ordered as the generator emitted them (bond to each
new atom when it is placed, angle distances right after their hydrogens).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "S": 32.06}
VALENCE = {"H": 1, "C": 4, "N": 3, "O": 2, "S": 2}
ELEMENTS = ("H", "C", "N", "O", "S")
ELEMENT_P = (0.50, 0.30, 0.08, 0.10, 0.02)
TETRA = np.deg2rad(109.4712206)  # ideal sp3 bond angle


@dataclass
class System:
    """A constrained system in the library's boundary layout (all float64 / int32)."""

    name: str
    x_old: np.ndarray  # (n_atoms, 3) feasible reference positions q_k [nm]
    x_unc: np.ndarray  # (n_atoms, 3) unconstrained update [nm]
    inv_mass: np.ndarray  # (n_atoms,)
    atom_i: np.ndarray  # (n_c,) int32
    atom_j: np.ndarray  # (n_c,) int32
    d: np.ndarray  # (n_c,) target distances [nm]
    mol_atom_ptr: np.ndarray = field(default=None)  # (n_mol+1,) generator's molecule ranges
    elements: list = field(default=None)
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.x_old.shape[0])

    @property
    def n_constraints(self) -> int:
        return int(self.atom_i.shape[0])

    @property
    def n_molecules(self) -> int:
        return 0 if self.mol_atom_ptr is None else int(len(self.mol_atom_ptr) - 1)


# ----------------------------------------------------------------------------------
# geometry helpers (placement only; plain floats for speed)
# ----------------------------------------------------------------------------------
def _unit(v):
    return v / np.linalg.norm(v)


def _perp(v, rng):
    a = rng.normal(size=3)
    a -= a.dot(v) * v
    return _unit(a)


def _direction(axis, e1, angle, dihedral):
    """Unit vector at `angle` from `axis`, rotated by `dihedral` about it (e1 = reference)."""
    e2 = np.cross(axis, e1)
    return np.cos(angle) * axis + np.sin(angle) * (np.cos(dihedral) * e1 + np.sin(dihedral) * e2)


_CT, _ST = math.cos(TETRA), math.sin(TETRA)


def _norm3(a, b, c):
    n = math.sqrt(a * a + b * b + c * c)
    return a / n, b / n, c / n


class _Builder:
    """Grows a tree-shaped molecule atom by atom with tetrahedral geometry.

    Each atom keeps an axis (unit vector towards its parent, or a random virtual
    parent for a root) and a perpendicular reference; its k-th child is placed at
    the tetrahedral angle from the axis with dihedral phase + 2*pi*k/3, so bonds at
    one atom never coincide.  A root's fourth child takes the virtual-parent slot.
    """

    def __init__(self, rng):
        self.rng = rng
        self.pos = []
        self.elem = []
        self.parent = []
        self.nchild = []
        self.axis = []
        self.ref = []
        self.phase = []
        self.bonds = []  # (parent, child, length)
        self._u = rng.random(size=4096).tolist()
        self._k = 0

    def _rand(self):
        if self._k == len(self._u):
            self._u = self.rng.random(size=4096).tolist()
            self._k = 0
        v = self._u[self._k]
        self._k += 1
        return v

    def root(self, element, at=(0.0, 0.0, 0.0)):
        g = self.rng.normal(size=6)
        ax = _norm3(g[0], g[1], g[2])
        d = g[3] * ax[0] + g[4] * ax[1] + g[5] * ax[2]
        ref = _norm3(g[3] - d * ax[0], g[4] - d * ax[1], g[5] - d * ax[2])
        self.pos.append(tuple(float(v) for v in at))
        self.elem.append(element)
        self.parent.append(-1)
        self.nchild.append(0)
        self.axis.append(ax)
        self.ref.append(ref)
        self.phase.append(2.0 * math.pi * self._rand())
        return len(self.pos) - 1

    def child(self, p, element, length):
        k = self.nchild[p]
        ax = self.axis[p]
        if self.parent[p] < 0 and k == 3:
            u = ax
        else:
            e1 = self.ref[p]
            e2 = (ax[1] * e1[2] - ax[2] * e1[1], ax[2] * e1[0] - ax[0] * e1[2], ax[0] * e1[1] - ax[1] * e1[0])
            dih = self.phase[p] + 2.0 * math.pi * k / 3.0
            c, s_ = math.cos(dih), math.sin(dih)
            u = tuple(_CT * ax[t] + _ST * (c * e1[t] + s_ * e2[t]) for t in range(3))
        self.nchild[p] += 1
        xp = self.pos[p]
        self.pos.append((xp[0] + length * u[0], xp[1] + length * u[1], xp[2] + length * u[2]))
        self.elem.append(element)
        self.parent.append(p)
        self.nchild.append(0)
        nax = (-u[0], -u[1], -u[2])
        self.axis.append(nax)
        d = ax[0] * nax[0] + ax[1] * nax[1] + ax[2] * nax[2]
        r = (ax[0] - d * nax[0], ax[1] - d * nax[1], ax[2] - d * nax[2])
        nr = math.sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2])
        if nr < 1e-8:  # axis parallel to the parent's: any perpendicular will do
            r = (nax[1] - nax[2], nax[2] - nax[0], nax[0] - nax[1])
            nr = math.sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2])
        self.ref.append((r[0] / nr, r[1] / nr, r[2] / nr))
        self.phase.append(2.0 * math.pi * self._rand())
        self.bonds.append((p, len(self.pos) - 1, length))
        return len(self.pos) - 1


def _bond_length(b, ea, eb):
    if ea == "H" or eb == "H":
        return 0.100
    return 0.122 + 0.031 * b._rand()


class _Slots:
    """Atoms with free valence; uniform choice and removal in O(1)."""

    def __init__(self):
        self.items, self.free, self.where = [], {}, {}

    def add(self, a, free):
        if free > 0:
            self.where[a] = len(self.items)
            self.items.append(a)
            self.free[a] = free

    def take(self, u):
        a = self.items[int(u * len(self.items))]
        self.free[a] -= 1
        if self.free[a] == 0:
            i = self.where.pop(a)
            last = self.items.pop()
            if last != a:
                self.items[i] = last
                self.where[last] = i
        return a

    def __len__(self):
        return len(self.items)


def _tree_molecule(rng, n_atoms):
    """One random tree molecule of exactly ``n_atoms`` atoms (elements, bonds, positions)."""
    elems = list(rng.choice(ELEMENTS, size=n_atoms, p=ELEMENT_P))
    heavy = [e for e in elems if e != "H"]
    n_h = n_atoms - len(heavy)
    if not heavy:
        heavy = ["C"]
        n_h -= 1
    # hydrogens beyond the available valence become carbons
    free = sum(VALENCE[e] for e in heavy) - 2 * (len(heavy) - 1)
    while n_h > free:
        heavy.append("C")
        n_h -= 1
        free += 2
    b = _Builder(rng)
    slots = _Slots()
    slots.add(b.root(heavy[0]), VALENCE[heavy[0]])
    for e in heavy[1:]:
        pa = slots.take(b._rand())
        c = b.child(pa, e, _bond_length(b, b.elem[pa], e))
        slots.add(c, VALENCE[e] - 1)
    for _ in range(n_h):
        pa = slots.take(b._rand())
        b.child(pa, "H", 0.100)
    return _renumber_dfs(b)


def _renumber_dfs(b):
    """Renumber atoms depth-first (hydrogens right after their parent), like MD topologies."""
    n = len(b.pos)
    kids = [[] for _ in range(n)]
    for p, c, _ in b.bonds:
        kids[p].append(c)
    order = []
    stack = [0]
    while stack:
        a = stack.pop()
        order.append(a)
        hs = [c for c in kids[a] if b.elem[c] == "H"]
        hv = [c for c in kids[a] if b.elem[c] != "H"]
        order.extend(hs)
        stack.extend(reversed(hv))
    new = [0] * n
    for i, a in enumerate(order):
        new[a] = i
    pos = np.asarray(b.pos, dtype=np.float64)[order]
    elem = [b.elem[a] for a in order]
    bonds = sorted(((new[p], new[c], ln) for p, c, ln in b.bonds), key=lambda t: t[1])
    return elem, bonds, pos


def _xoh_pairs(elem, bonds):
    """X-O-H triangle-closing pairs (main text, ``h-angles``): every oxygen bonded to exactly
    one hydrogen H and one heavy atom X contributes the X...H distance."""
    nb = [[] for _ in elem]
    for p, c, _ in bonds:
        nb[p].append(c)
        nb[c].append(p)
    out = []
    for a, e in enumerate(elem):
        if e != "O" or len(nb[a]) != 2:
            continue
        hs = [c for c in nb[a] if elem[c] == "H"]
        xs = [c for c in nb[a] if elem[c] != "H"]
        if len(hs) == 1 and len(xs) == 1:
            out.append((min(xs[0], hs[0]), max(xs[0], hs[0])))
    return out


def _with_xoh(mol):
    """A tree molecule (elements, bonds, positions) with its X-O-H distances appended."""
    elem, bonds, pos = mol
    return elem, list(bonds) + [(u, v, 0.0) for u, v in _xoh_pairs(elem, bonds)], pos


def _assemble(name, mols, rng, sigma, seed, box):
    """Concatenate molecules, place them in a box, perturb, and build boundary arrays."""
    xs, ii, jj, dd, el, ptr = [], [], [], [], [], [0]
    off = 0
    for elem, bonds, pos in mols:
        shift = rng.uniform(0.0, box, size=3) - pos.mean(axis=0)
        xs.append(pos + shift)
        for p, c, ln in bonds:
            ii.append(off + p)
            jj.append(off + c)
            dd.append(ln)
        el.extend(elem)
        off += len(elem)
        ptr.append(off)
    x_old = np.ascontiguousarray(np.concatenate(xs), dtype=np.float64)
    x_unc = x_old + rng.normal(0.0, sigma, size=x_old.shape)
    inv_mass = np.array([1.0 / MASS[e] for e in el], dtype=np.float64)
    return System(
        name=name,
        x_old=x_old,
        x_unc=np.ascontiguousarray(x_unc),
        inv_mass=inv_mass,
        atom_i=np.asarray(ii, dtype=np.int32),
        atom_j=np.asarray(jj, dtype=np.int32),
        d=np.asarray(dd, dtype=np.float64),
        mol_atom_ptr=np.asarray(ptr, dtype=np.int64),
        elements=el,
        seed=seed,
        meta={"perturbation_nm": sigma, "box_nm": box},
    )


def _exact_lengths(sys_: System) -> System:
    """Set each target distance to the exact |x_old_i - x_old_j| so x_old is feasible to rounding."""
    r = sys_.x_old[sys_.atom_i] - sys_.x_old[sys_.atom_j]
    sys_.d = np.sqrt(np.einsum("ij,ij->i", r, r))
    return sys_


# ----------------------------------------------------------------------------------
# public workloads
# ----------------------------------------------------------------------------------
def _chain(rng, n_atoms=64, bond=0.153, angle_deg=111.0):
    """Random walk with fixed bond length, fixed bond angle and uniform dihedrals."""
    theta = math.radians(180.0 - angle_deg)  # angle between successive bond vectors
    ct, st = math.cos(theta), math.sin(theta)
    g = rng.normal(size=6)
    dih = rng.uniform(0.0, 2.0 * math.pi, size=n_atoms).tolist()
    u = _norm3(g[0], g[1], g[2])
    dd = g[3] * u[0] + g[4] * u[1] + g[5] * u[2]
    e1 = _norm3(g[3] - dd * u[0], g[4] - dd * u[1], g[5] - dd * u[2])
    pos = [(0.0, 0.0, 0.0)]
    pos.append((bond * u[0], bond * u[1], bond * u[2]))
    for k in range(n_atoms - 2):
        e2 = (u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0])
        c, s_ = math.cos(dih[k]), math.sin(dih[k])
        un = _norm3(*(ct * u[t] + st * (c * e1[t] + s_ * e2[t]) for t in range(3)))
        dd = u[0] * un[0] + u[1] * un[1] + u[2] * un[2]
        e1 = _norm3(u[0] - dd * un[0], u[1] - dd * un[1], u[2] - dd * un[2])
        u = un
        x = pos[-1]
        pos.append((x[0] + bond * u[0], x[1] + bond * u[1], x[2] + bond * u[2]))
    elem = ["C"] * n_atoms
    bonds = [(k, k + 1, bond) for k in range(n_atoms - 1)]
    return elem, bonds, np.asarray(pos, dtype=np.float64)


def chain64(seed: int = 1000, sigma: float = 0.002) -> System:
    """One 64-atom carbon chain (63 bonds, 0.153 nm, 111 deg angles)."""
    rng = np.random.default_rng(seed)
    s = _assemble("chain64", [_chain(rng)], rng, sigma, seed, box=0.0)
    return _exact_lengths(s)


def chain_batch(n_chains: int, seed: int, sigma: float = 0.002, box: float = 20.0) -> System:
    """Many independent chain64-distribution chains."""
    rng = np.random.default_rng(seed)
    mols = [_chain(rng) for _ in range(n_chains)]
    return _exact_lengths(_assemble(f"chain_batch{n_chains}", mols, rng, sigma, seed, box))


def chain_molecules(sizes, seed: int, sigma: float = 0.002, box: float = 20.0) -> System:
    """Carbon chains of the given atom counts (the chain64 distribution: 0.153 nm bonds,
    111 deg angles, uniform dihedrals); long chains give deep elimination orders."""
    rng = np.random.default_rng(seed)
    mols = [_chain(rng, n_atoms=int(n)) for n in sizes]
    return _exact_lengths(_assemble("chains", mols, rng, sigma, seed, box))


def tree_batch(n_mol: int = 4096, lo: int = 20, hi: int = 200, seed: int = 1001,
               sigma: float = 0.003, box: float | None = None, xoh: bool = False) -> System:
    """Batch of independent random tree molecules with U{lo..hi} atoms each; with ``xoh``
    every hydroxyl adds its X-O-H triangle-closing distance (3-cycles in the graph)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=n_mol)
    mols = [_tree_molecule(rng, int(n)) for n in sizes]
    if xoh:
        mols = [_with_xoh(m) for m in mols]
    if box is None:  # ~100 atoms per nm^3, a condensed-phase density
        box = float(max(1.0, (sizes.sum() / 100.0) ** (1.0 / 3.0)))
    s = _assemble(f"tree_batch{n_mol}", mols, rng, sigma, seed, box)
    return _exact_lengths(s)


def tree_molecules_of_sizes(sizes, seed: int, sigma: float = 0.003, box: float = 10.0) -> System:
    """Tree molecules of the given atom counts (serving requests, edge cases)."""
    rng = np.random.default_rng(seed)
    mols = [_tree_molecule(rng, int(n)) for n in sizes]
    return _exact_lengths(_assemble("trees", mols, rng, sigma, seed, box))


def protein_like(n_atoms: int = 100_000, seed: int = 1002, sigma: float = 0.004, xoh: bool = False) -> System:
    """One connected protein-like system: backbone + side chains + H-X-H distances.

    Residue pattern: N(-H) - CA(-HA)(side chain) - C(=O).  Side chains are random
    heavy-atom subtrees (elements C/N/O/S in the tree-batch proportions) saturated
    with hydrogens, so terminal carbons become CH3 and terminal nitrogens NH2/NH3.
    Each CH3 and NH3 adds the three H-H distances of its hydrogens, each NH2 adds one.
    With ``xoh`` every hydroxyl (side-chain O with one H) also adds its X-O-H distance.
    """
    rng = np.random.default_rng(seed)
    b = _Builder(rng)
    heavy_p = np.array(ELEMENT_P[1:]) / sum(ELEMENT_P[1:])
    prev_c = None
    while len(b.pos) < n_atoms:
        if prev_c is None:
            n_at = b.root("N")
        else:
            n_at = b.child(prev_c, "N", float(rng.uniform(0.122, 0.153)))
        b.child(n_at, "H", 0.100)
        ca = b.child(n_at, "C", float(rng.uniform(0.122, 0.153)))
        b.child(ca, "H", 0.100)
        # side chain: 0..5 heavy atoms as a random subtree rooted at CA
        n_side = int(rng.integers(0, 6))
        side = [ca]
        freev = {ca: 1}
        for _ in range(n_side):
            cand = [a for a in side if freev[a] > 0]
            if not cand:
                break
            pa = cand[int(rng.integers(len(cand)))]
            e = str(rng.choice(ELEMENTS[1:], p=heavy_p))
            c = b.child(pa, e, _bond_length(b, b.elem[pa], e))
            freev[pa] -= 1
            freev[c] = VALENCE[e] - 1
            side.append(c)
        for a in list(side[1:]):
            # a share of terminal carbons become CH2-OH instead of methyls
            if b.elem[a] == "C" and b.nchild[a] == 0 and rng.random() < 0.3:
                o = b.child(a, "O", float(rng.uniform(0.122, 0.153)))
                freev[a] -= 1
                freev[o] = 1
                side.append(o)
        for a in side[1:]:
            # saturate with hydrogens; a terminal N carries NH2 or NH3 with equal odds
            nh = freev[a]
            if b.elem[a] == "N" and b.nchild[a] == 0:
                nh = 2 + int(rng.random() < 0.5)
            for _ in range(min(nh, 3)):
                b.child(a, "H", 0.100)
        c_at = b.child(ca, "C", float(rng.uniform(0.122, 0.153)))
        b.child(c_at, "O", float(rng.uniform(0.122, 0.153)))
        prev_c = c_at
    elem = b.elem
    pos = np.asarray(b.pos)
    # atoms are already in emission order (children after parents); bonds sorted by child
    bonds = sorted(((p, c, ln) for p, c, ln in b.bonds), key=lambda t: t[1])
    # H-X-H triangle-closing distances on CH3 / NH2 / NH3
    kids = [[] for _ in range(len(elem))]
    for p, c, _ in b.bonds:
        kids[p].append(c)
    extra = []
    for a, e in enumerate(elem):
        hs = [c for c in kids[a] if elem[c] == "H"]
        heavy_nb = len([c for c in kids[a] if elem[c] != "H"]) + (1 if b.parent[a] >= 0 else 0)
        if (e == "C" and len(hs) == 3 and heavy_nb == 1) or (e == "N" and len(hs) >= 2 and heavy_nb == 1):
            for u in range(len(hs)):
                for v in range(u + 1, len(hs)):
                    extra.append((hs[u], hs[v]))
    n_hxh = len(extra)
    if xoh:
        extra += _xoh_pairs(elem, bonds)
    cons = [(p, c, ln) for p, c, ln in bonds]
    # interleave each angle distance after the bond of its later hydrogen (keeps bands narrow)
    by_child = {}
    for h1, h2 in extra:
        by_child.setdefault(max(h1, h2), []).append((min(h1, h2), max(h1, h2), 0.0))
    merged = []
    for t in cons:
        merged.append(t)
        merged.extend(by_child.get(t[1], []))
    s = _assemble("protein_like", [(elem, merged, pos)], rng, sigma, seed, box=0.0)
    s = _exact_lengths(s)
    s.meta["n_angle_constraints"] = len(extra)
    s.meta["n_xoh_constraints"] = len(extra) - n_hxh
    return s


def benzene_batch(n_mol: int = 64, seed: int = 1005, sigma: float = 0.003, box: float = 6.0) -> System:
    """Benzene-like rings: six carbons in a planar hexagon (C-C 0.139 nm) with six
    hydrogens (C-H 0.109 nm); all 12 bonds constrained (6-cycles in the constraint graph,
    like the paper's pure-benzene system, supplement Sec. 6)."""
    rng = np.random.default_rng(seed)
    mols = []
    for _ in range(n_mol):
        q, _r = np.linalg.qr(rng.normal(size=(3, 3)))
        ang = np.arange(6) * np.pi / 3.0
        ring = np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], axis=1)
        pos = np.concatenate([0.139 * ring, (0.139 + 0.109) * ring]) @ q.T
        elem = ["C"] * 6 + ["H"] * 6
        bonds = [(k, (k + 1) % 6, 0.139) for k in range(6)] + [(k, k + 6, 0.109) for k in range(6)]
        bonds = [(min(a, b), max(a, b), ln) for a, b, ln in bonds]
        mols.append((elem, bonds, pos))
    return _exact_lengths(_assemble(f"benzene{n_mol}", mols, rng, sigma, seed, box))


def serving_sizes(n_req: int, seed: int, lo: int = 20, hi: int = 50_000) -> np.ndarray:
    """Log-uniform request sizes (atoms) for the serving loop."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_req)).astype(np.int64)


def two_atoms(d=0.1, w1=1.0, w2=1.0, seed=7, sigma=0.01) -> System:
    """Smallest case: one constraint between two atoms (closed-form lambda)."""
    rng = np.random.default_rng(seed)
    u = _unit(rng.normal(size=3))
    x_old = np.stack([np.zeros(3), d * u]) + rng.uniform(-1, 1, size=3)
    x_unc = x_old + rng.normal(0.0, sigma, size=x_old.shape)
    return System("two_atoms", x_old, x_unc, np.array([w1, w2], float),
                  np.array([0], np.int32), np.array([1], np.int32), np.array([d], float),
                  mol_atom_ptr=np.array([0, 2]), seed=seed)


def by_name(name: str, **kw) -> System:
    return {"chain64": chain64, "tree_batch": tree_batch, "protein_like": protein_like}[name](**kw)
