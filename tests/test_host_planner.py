"""Host-side checks of the C-ABI library: symbol exports, validation, symbolic LU.

These run without a GPU: topologies are planned with device = -2 (host only).
"""
import ctypes

import numpy as np
import pytest

from paper_2503_13075_gb300 import binding as B
from paper_2503_13075_gb300 import workloads as wl


def test_library_exports_every_header_symbol():
    L = B.lib()
    names = B.header_functions()
    assert "ilves_solve" in names and "ilves_setup_topology" in names
    for n in names:
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


@pytest.mark.parametrize("ai,aj,code", [([0], [5], 2), ([1], [1], 2), ([0, 1], [1, 0], 2), ([0, 2], [1, 1], 0)])
def test_topology_validation(ai, aj, code):
    if code == 0:
        t = B.Topology(3, ai, aj, plan_only=True)
        assert t.n_molecules == 1
    else:
        with pytest.raises(B.IlvesError) as e:
            B.Topology(3, ai, aj, plan_only=True)
        assert e.value.code == code


def test_invalid_arguments():
    with pytest.raises(B.IlvesError) as e:
        B.Topology(-1, [], [], plan_only=True)
    assert e.value.code == 1
    with pytest.raises(B.IlvesError) as e:
        B.Topology(4, [0], [1], ordering=7, plan_only=True)
    assert e.value.code == 1
    with pytest.raises(B.IlvesError) as e:  # the wait-test knob is bounded
        B.Topology(4, [0], [1], wait_test=65, plan_only=True)
    assert e.value.code == 1
    B.Topology(4, [0], [1], wait_test=1, plan_only=True)
    with pytest.raises(B.IlvesError) as e:  # the overlap depth is bounded
        B.Topology(4, [0], [1], overlap=17, plan_only=True)
    assert e.value.code == 1
    t = B.Topology(4, [0], [1], plan_only=True)  # a host-only plan cannot be tuned or solved
    tune = B.Tuning()
    assert B.lib().ilves_autotune(t._h, None, None, None, None, 1e-12, 1, 3, None, ctypes.byref(tune)) == 1
    assert t.tuning()["candidates"] == 0


def _line_graph(ai, aj):
    inc = {}
    for k, (i, j) in enumerate(zip(ai, aj)):
        inc.setdefault(int(i), []).append(k)
        inc.setdefault(int(j), []).append(k)
    adj = [set() for _ in ai]
    for ks in inc.values():
        for x in ks:
            adj[x].update(ks)
            adj[x].discard(x)
    return adj


def _check_molecule(topo, s, m, rng):
    pos_gid, level, ptr, idx = topo.export_molecule(m)
    nc = pos_gid.size
    up = [set(idx[ptr[p]:ptr[p + 1]].tolist()) for p in range(nc)]
    pos_of = {int(g): p for p, g in enumerate(pos_gid)}
    ai, aj = s.atom_i[pos_gid], s.atom_j[pos_gid]
    adj = _line_graph(ai, aj)  # in position numbering
    # 1. the pattern of A (line graph) is inside the filled pattern
    for p in range(nc):
        for q in adj[p]:
            lo, hi = min(p, q), max(p, q)
            assert hi in up[lo]
    # 2. every pivot's later neighbours form a clique of later pivots (elimination closure)
    for p in range(nc):
        u = sorted(up[p])
        assert all(q > p for q in u)
        for a_ in range(len(u)):
            for b_ in range(a_ + 1, len(u)):
                assert u[b_] in up[u[a_]]
    # 3. levels: sorted, and a pivot's later neighbours sit on higher levels
    assert np.all(np.diff(level) >= 0)
    for p in range(nc):
        for q in up[p]:
            assert level[q] > level[p]
    # 4. numeric: LU without pivoting of a random diagonally dominant matrix on A's pattern
    #    in this order has no entry outside the symbolic pattern
    if nc <= 300:
        A = np.zeros((nc, nc))
        for p in range(nc):
            for q in adj[p]:
                A[p, q] = rng.normal()
            A[p, p] = 10.0 + len(adj[p])
        U = A.copy()
        Lm = np.eye(nc)
        for k in range(nc):
            for i in range(k + 1, nc):
                if U[i, k] != 0.0:
                    Lm[i, k] = U[i, k] / U[k, k]
                    U[i, :] -= Lm[i, k] * U[k, :]
        allowed = np.eye(nc, dtype=bool)
        for p in range(nc):
            for q in up[p]:
                allowed[p, q] = allowed[q, p] = True
        nz = (np.abs(U) > 1e-12) | (np.abs(Lm) > 1e-12)
        assert not np.any(nz & ~allowed)
    return pos_of


@pytest.mark.parametrize("ordering,slack", [(0, 2), (1, 0), (2, 0), (2, 3)])
def test_symbolic_factorisation_chain_and_trees(ordering, slack):
    rng = np.random.default_rng(0)
    for s in (wl.chain64(), wl.tree_batch(n_mol=12, seed=17)):
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, ordering=ordering, degree_slack=slack, plan_only=True)
        atoms, cons, levels, first = t.molecules()
        assert t.n_molecules == s.n_molecules
        assert np.array_equal(first, s.mol_atom_ptr[:-1])
        assert np.array_equal(atoms, np.diff(s.mol_atom_ptr))
        for m in range(t.n_molecules):
            _check_molecule(t, s, m, rng)


def test_symbolic_factorisation_rings_and_cliques():
    """Protein-like fragment: CH3 groups form K4 cliques with their H-H distances."""
    rng = np.random.default_rng(1)
    s = wl.protein_like(n_atoms=600, seed=5)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True)
    assert t.n_molecules == 1
    _check_molecule(t, s, 0, rng)


def test_symbolic_factorisation_hydroxyl_triangles():
    """X-O-H distances (main text, h-angles) close 3-cycles through hydroxyl oxygens: tree
    molecules and a protein-like fragment with them keep a consistent symbolic LU."""
    rng = np.random.default_rng(2)
    s = wl.tree_batch(n_mol=24, seed=21, xoh=True)
    assert s.n_constraints > s.n_atoms - s.n_molecules  # some molecules carry triangles
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True)
    assert t.n_molecules == s.n_molecules
    for m in range(t.n_molecules):
        _check_molecule(t, s, m, rng)
    p = wl.protein_like(n_atoms=800, seed=6, xoh=True)
    assert p.meta["n_xoh_constraints"] > 0
    t = B.Topology(p.n_atoms, p.atom_i, p.atom_j, plan_only=True)
    _check_molecule(t, p, 0, rng)


def test_level_counts_are_small():
    """The rounds ordering keeps the level count near log scale (chain) / tree depth."""
    c = wl.chain64()
    t1 = B.Topology(c.n_atoms, c.atom_i, c.atom_j, ordering=1, plan_only=True)
    t0 = B.Topology(c.n_atoms, c.atom_i, c.atom_j, plan_only=True)
    assert t1.max_levels >= 30  # one pivot per step on a chain: ~n/2 levels
    assert t0.max_levels <= 8  # cyclic-reduction-like
    s = wl.tree_batch(n_mol=64, seed=3)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True)
    assert t.molecules()[2].mean() < 12


def test_free_atoms_and_empty():
    t = B.Topology(5, [], [], plan_only=True)
    assert t.n_molecules == 0
    t = B.Topology(6, [0, 4], [1, 5], plan_only=True)
    atoms, cons, levels, first = t.molecules()
    assert list(first) == [0, 4] and list(cons) == [1, 1]


def test_partitioned_molecule_structure():
    """Large molecules are cut into contiguous atom parts; separators (constraints between
    parts) come last, every pivot's later neighbours are later positions, and the
    symbolic closure holds across the whole molecule."""
    s = wl.protein_like(n_atoms=3000, seed=21)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, partition_min_constraints=1000,
                   part_constraints=200)
    assert t.n_large == 1
    pos_gid, level, ptr, idx = t.export_molecule(0)
    nc = pos_gid.size
    up = [set(idx[ptr[p]:ptr[p + 1]].tolist()) for p in range(nc)]
    for p in range(nc):
        u = sorted(up[p])
        assert all(q > p for q in u)
        for a_ in range(len(u)):
            for b_ in range(a_ + 1, len(u)):
                assert u[b_] in up[u[a_]]
    # the pattern of A is inside the filled pattern
    adj = _line_graph(s.atom_i[pos_gid], s.atom_j[pos_gid])
    for p in range(nc):
        for q in adj[p]:
            assert max(p, q) in up[min(p, q)]
    # segments (levels restart at every segment): each part's constraints lie inside one
    # contiguous block of atoms, blocks are disjoint, and the last segment (separators)
    # holds exactly the constraints that cross blocks
    ai, aj = s.atom_i[pos_gid], s.atom_j[pos_gid]
    starts = [0] + [p for p in range(1, nc) if level[p] < level[p - 1]] + [nc]
    assert len(starts) >= 5
    blocks = []
    for g in range(len(starts) - 2):
        seg_atoms = np.concatenate([ai[starts[g]:starts[g + 1]], aj[starts[g]:starts[g + 1]]])
        blocks.append((seg_atoms.min(), seg_atoms.max()))
    blocks.sort()
    for (lo0, hi0), (lo1, hi1) in zip(blocks, blocks[1:]):
        assert hi0 < lo1
    def block_of(a):
        return next((k for k, (lo, hi) in enumerate(blocks) if lo <= a <= hi), -1)
    for p in range(starts[-2], nc):  # separators cross blocks (or touch a block-less atom)
        assert block_of(ai[p]) != block_of(aj[p]) or block_of(ai[p]) == -1


def test_symbolic_factorisation_benzene_rings():
    """6-cycles (benzene-like rings): closure and pattern checks with fill."""
    rng = np.random.default_rng(4)
    s = wl.benzene_batch(n_mol=3)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True)
    assert t.n_molecules == 3 and t.n_fill > 0
    for m in range(3):
        _check_molecule(t, s, m, rng)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("n_mol,n_cta", [(600, 152), (37, 152), (1, 152), (300, 4)])
@pytest.mark.parametrize("narrow", [0, -1, 60, 140])
def test_warp_slot_schedule(prec, n_mol, n_cta, narrow):
    """Every batched molecule is queued exactly once (a slot of its class or its class's
    pool), fits its slot's slice, pool molecules fit every slice of their class, each
    CTA's slices fit the arena and its teams the CTA's threads, and a CTA's 96-thread slots
    come before its one-warp slots."""
    arena = 232448
    s = wl.tree_batch(n_mol=n_mol, seed=11)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, narrow_atoms=narrow)
    sc = t.schedule(prec, n_cta=n_cta, arena_bytes=arena)
    ms, mb, team = sc["mol_slot"], sc["mol_bytes"], sc["mol_team"]
    st, cta = sc["slot_team"], sc["slot_cta"]
    atoms = t.molecules()[0]
    ns = len(cta)
    assert ns >= 1 and np.all(mb > 0)
    # the class follows the size threshold (-1: no narrow class; 0: none for these batches
    # of 20-200 atoms)
    assert np.array_equal(team == 32, atoms <= (-1 if narrow <= 0 else narrow))
    assert np.all((team == 32) | (team == 96)) and np.all((st == 32) | (st == 96))
    queued = ms >= 0
    assert np.array_equal(np.bincount(ms[queued], minlength=ns), sc["slot_queue"])
    assert int((ms == -1).sum()) == sc["pool_n"]
    assert int(((ms == -1) & (team == 96)).sum()) == sc["pool_wide"]
    assert np.all(mb[queued] <= sc["slot_bytes"][ms[queued]])
    assert np.all(st[ms[queued]] == team[queued])  # queued in a slot of its class
    assert int((st == 96).sum()) == sc["n_slots_wide"]
    for cls in (96, 32):
        pool = (ms == -1) & (team == cls)
        if pool.any():
            assert (st == cls).any()
            assert mb[pool].max() <= sc["slot_bytes"][st == cls].min()
            q = queued & (team == cls)  # the pool holds the class's smallest molecules
            assert mb[pool].max() <= mb[q].min() if q.any() else True
    per_cta = np.bincount(cta, weights=sc["slot_bytes"], minlength=n_cta)
    assert per_cta.max() <= arena
    threads = np.bincount(cta, weights=st, minlength=n_cta)
    assert threads.max() == sc["block_threads"] <= 768
    assert np.bincount(cta).max() == sc["max_slots"]
    assert np.all(np.diff(cta) >= 0)  # slots are numbered CTA by CTA
    for c in range(cta.max() + 1):  # the used CTAs are a prefix; wide slots first
        tc = st[cta == c]
        assert tc.size > 0 and np.all(np.diff(tc) <= 0)
        assert (tc == 96).sum() <= 8


@pytest.mark.parametrize("seed", range(12))
def test_slot_schedule_random_batches(seed):
    """Random batches (2..250 atoms per molecule), thresholds, grids and arenas: every batched
    molecule lands in exactly one slot queue or pool of its own class, no CTA exceeds its
    arena, its threads or eight 96-thread slots, and 96-thread slots come first in a CTA."""
    rng = np.random.default_rng(900 + seed)
    sizes = rng.integers(2, 251, size=int(rng.integers(1, 400)))
    s = wl.tree_molecules_of_sizes(sizes.tolist(), seed=seed)
    narrow = int(rng.choice([0, -1, 40, 70, 100, 200]))
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, narrow_atoms=narrow)
    n_cta = int(rng.choice([1, 3, 17, 152, 304]))
    arena = int(rng.choice([232320, 115712]))
    for prec in ("fp64", "mixed", "mixed_df"):
        sc = t.schedule(prec, n_cta=n_cta, arena_bytes=arena)
        ms, team, st, cta = sc["mol_slot"], sc["mol_team"], sc["slot_team"], sc["slot_cta"]
        batched = team > 0
        assert np.all(ms[batched] >= -1) and np.all(ms[~batched] == -2)
        q = ms >= 0
        assert np.array_equal(np.bincount(ms[q], minlength=len(cta)), sc["slot_queue"])
        assert np.all(st[ms[q]] == team[q])
        assert int((batched & (ms == -1)).sum()) == sc["pool_n"]
        for cls in (96, 32):  # a class with batched molecules has slots
            assert not np.any(team == cls) or np.any(st == cls)
        if len(cta):
            assert cta.max() < n_cta and np.all(np.diff(cta) >= 0)
            assert np.bincount(cta, weights=sc["slot_bytes"]).max() <= arena
            assert np.bincount(cta, weights=st).max() <= 768
            for c in range(cta.max() + 1):
                tc = st[cta == c]
                assert tc.size and np.all(np.diff(tc) <= 0) and (tc == 96).sum() <= 8


def test_narrow_class_automatic_choice():
    """narrow_atoms = 0: one-warp teams for molecules of at most 100 atoms only in a batch of
    such molecules (>= 90 % of the batched atoms) larger than the GPU's 96-thread teams
    (8 per SM, 152 SMs); the schedule then gives them one-warp slots, up to 24 per CTA."""
    small = wl.tree_batch(n_mol=1300, lo=20, hi=100, seed=5)
    t = B.Topology(small.n_atoms, small.atom_i, small.atom_j, plan_only=True)
    sc = t.schedule("mixed")
    assert np.all(sc["mol_team"] == 32) and np.all(sc["slot_team"] == 32)
    assert sc["max_slots"] > 8 and sc["n_slots_wide"] == 0
    few = wl.tree_batch(n_mol=1000, lo=20, hi=100, seed=5)  # fewer molecules than wide teams
    t = B.Topology(few.n_atoms, few.atom_i, few.atom_j, plan_only=True)
    assert np.all(t.schedule("mixed")["mol_team"] == 96)
    mixed = wl.tree_batch(n_mol=1300, lo=20, hi=200, seed=5)  # mixed sizes: no narrow class
    t = B.Topology(mixed.n_atoms, mixed.atom_i, mixed.atom_j, plan_only=True)
    assert np.all(t.schedule("mixed")["mol_team"] == 96)
    # explicit threshold on the mixed batch: both classes, every CTA mixing them
    t = B.Topology(mixed.n_atoms, mixed.atom_i, mixed.atom_j, plan_only=True, narrow_atoms=60)
    sc = t.schedule("mixed")
    atoms = t.molecules()[0]
    assert np.array_equal(sc["mol_team"] == 32, atoms <= 60)
    assert 0 < sc["n_slots_wide"] < len(sc["slot_team"])


def test_batched_atoms_ordered_by_degree():
    """Batched molecules order their local atoms by decreasing number of constraints (ties
    in global order), as a permutation of the molecule's atoms; molecules on the
    CTA-per-molecule path keep the global order."""
    s = wl.tree_batch(n_mol=48, seed=31)
    deg = np.bincount(np.concatenate([s.atom_i, s.atom_j]), minlength=s.n_atoms)
    for forced_large in (False, True):
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True,
                       max_warp_constraints=10 if forced_large else 0)
        atoms, cons, _, first = t.molecules()
        for m in range(t.n_molecules):
            gid = t.export_layout(m)["atom_gid"]
            assert sorted(gid.tolist()) == list(range(first[m], first[m] + atoms[m]))
            if forced_large and cons[m] > 10:
                assert np.all(np.diff(gid) > 0)
                continue
            d = deg[gid]
            assert np.all(np.diff(d) <= 0)
            ties = np.diff(d) == 0
            assert np.all(np.diff(gid)[ties] > 0)


def test_partitioned_programs_layout():
    """A partitioned molecule gets a shared-memory program per part and one for the
    separator block; the parts' level counts are those of the exported elimination; no
    separator term reads an interior pivot (a separator constraint touches at most two
    parts, whose contributions fill its two slots); the slack tuning keeps the deepest part
    shallow."""
    s = wl.protein_like(n_atoms=20000, seed=1002)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, partition_min_constraints=2000)
    assert t.n_large == 1
    atoms, cons, _, _ = t.molecules()
    m = int(np.argmax(cons))
    L = t.export_layout(m)
    assert L["n_parts"] >= 50
    assert np.all(L["part_prog_bytes"] > 0) and np.all(L["part_prog_bytes"] % 16 == 0)
    assert L["part_prog_max"] > L["part_prog_bytes"].max()  # scratch behind the largest program
    assert L["sep_prog_bytes"] > 0 and L["sep_interior_terms"] == 0
    pos, level, _, _ = t.export_molecule(m)
    starts = [0] + [p for p in range(1, pos.size) if level[p] < level[p - 1]] + [pos.size]
    seg_levels = [int(level[a:b].max()) + 1 for a, b in zip(starts, starts[1:])]
    assert seg_levels[:-1] == L["part_levels"].tolist()
    assert seg_levels[-1] == L["sep_levels"]
    assert L["part_levels"].max() <= 12
    assert sorted(L["atom_gid"].tolist()) == list(range(s.n_atoms))


def test_partition_threshold_and_ring_atom_order():
    """A tree of exactly the partition threshold (constraints) is partitioned, one
    constraint fewer is not; benzene rings (fill in the factor) order their atoms carbons
    first (three constraints each), hydrogens after."""
    s = wl.tree_molecules_of_sizes([2001], seed=41)  # 2000 constraints
    for thresh, parted in ((2000, True), (2001, False)):
        t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, partition_min_constraints=thresh,
                       max_warp_constraints=0)
        L = t.export_layout(0)
        assert (L["n_parts"] > 1) == parted
        if parted:
            assert np.all(L["part_prog_bytes"] > 0) and L["sep_interior_terms"] == 0
    b = wl.benzene_batch(n_mol=8, seed=42)
    t = B.Topology(b.n_atoms, b.atom_i, b.atom_j, plan_only=True)
    deg = np.bincount(np.concatenate([b.atom_i, b.atom_j]), minlength=b.n_atoms)
    for m in range(t.n_molecules):
        gid = t.export_layout(m)["atom_gid"]
        assert gid.size == 12 and list(deg[gid]) == [3] * 6 + [1] * 6


@pytest.mark.parametrize("overlap,part", [(1, 256), (3, 256), (4, 180)])
def test_overlapping_domains_match_the_oracle(overlap, part):
    """The planner's overlapping domains (greedy partition, halo of `overlap` edges, owned
    constraints) are exactly the oracle's, which derives them independently."""
    from oracle import ilves_oracle as orc

    s = wl.protein_like(n_atoms=8000, seed=1006, xoh=True)
    t = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, overlap=overlap, part_constraints=part,
                   partition_min_constraints=2000)
    D = t.export_domains(0)
    ai, aj = s.atom_i.astype(np.int64), s.atom_j.astype(np.int64)
    atoms = np.unique(np.concatenate([ai, aj]))
    li, lj = np.searchsorted(atoms, ai), np.searchsorted(atoms, aj)
    b = orc.greedy_partition(atoms.size, li, lj, max(2, -(-len(ai) // part)))
    assert np.array_equal(np.asarray(b), D["atom_bounds"])
    doms = orc.opm_domains(atoms.size, li, lj, b, overlap)
    assert len(doms) == len(D["cons"])
    for (cons, owned), c2, o2 in zip(doms, D["cons"], D["owned"]):
        assert np.array_equal(cons, c2) and np.array_equal(owned, o2)
    owned_all = np.concatenate([c[o] for c, o in zip(D["cons"], D["owned"])])
    assert np.array_equal(np.sort(owned_all), np.arange(s.n_constraints))  # each owned once
    # the exact-Newton molecule export is refused for a molecule solved by domains
    with pytest.raises(B.IlvesError):
        t.export_molecule(0)


def test_overlapping_domains_fall_back_to_the_schur_path():
    """Domains that cannot all be resident at once (a random tree's 4-edge halos double
    them) leave the molecule on the Schur-complement path instead of failing set-up."""
    s = wl.tree_molecules_of_sizes([40000], seed=77)
    t4 = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, overlap=4)
    assert len(t4.export_domains(0)["cons"]) == 0 and t4.export_layout(0)["n_parts"] > 100
    t2 = B.Topology(s.n_atoms, s.atom_i, s.atom_j, plan_only=True, overlap=2)
    assert len(t2.export_domains(0)["cons"]) == t2.export_layout(0)["n_parts"] > 100
