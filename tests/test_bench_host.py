"""Host-side pieces of the benchmark (no GPU): algorithmic bytes and float64 flops of a
solve, and the traffic records of the committed profiles."""
import numpy as np

import bench


class _Sys:
    def __init__(self, n_atoms, n_constraints, n_molecules):
        self.n_atoms, self.n_constraints, self.n_molecules = n_atoms, n_constraints, n_molecules


def test_algorithmic_bytes():
    # 80 B per atom, 24 B per constraint, 8 B per molecule
    assert bench.algorithmic_bytes(_Sys(10, 9, 1)) == 80 * 10 + 24 * 9 + 8


def test_mixed_fp64_flops_counts_each_step():
    # one two-atom molecule, one constraint, I Newton solves
    na, nc = np.array([2]), np.array([1])
    for it in (0, 1, 3):
        for started in (False, True):
            upd = it + (1 if started else 0)
            want = 4 + 10 * (it + 1) + it + (12 + 6 * 2) * upd
            assert bench.mixed_fp64_flops(na, nc, np.array([it]), started) == want
    # additive over molecules
    two = bench.mixed_fp64_flops(np.array([2, 5]), np.array([1, 4]), np.array([3, 2]), True)
    one = bench.mixed_fp64_flops(np.array([2]), np.array([1]), np.array([3]), True)
    other = bench.mixed_fp64_flops(np.array([5]), np.array([4]), np.array([2]), True)
    assert two == one + other


def test_traffic_records_are_well_formed():
    """Every traffic record names a kernel, a mode, positive bytes and atoms, and a source
    digest of the kernel sources' form; a record applies only to its own kernel and mode."""
    import glob
    import os

    recs = []
    for path in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md")):
        for line in open(path):
            if line.startswith("traffic-record:"):
                kv = dict(tok.split("=", 1) for tok in line.split()[1:])
                recs.append(kv)
    assert recs
    for kv in recs:
        assert kv["kernel"] in ("k_solve_small", "k_solve_parted", "k_solve_opm")
        assert kv["mode"] in ("fp64", "mixed", "mixed_df")
        assert int(kv["dram_bytes"]) > 0 and int(kv["atoms"]) > 0
        assert len(kv["sources"]) == 16 and int(kv["sources"], 16) >= 0
    assert bench.measured_traffic("k_solve_small", "no-such-mode", 1000) == (None, None)


def test_serving_oracle_report():
    """The serving line's oracle sample: results equal to the oracle's give zero errors and
    equal statuses; a moved atom and a wrong status show up in the report."""
    import torch

    from oracle import ilves_oracle as orc
    from paper_2503_13075_gb300 import serving as sv
    from paper_2503_13075_gb300 import workloads as wl

    done = []
    for k, n in enumerate((20, 35, 60)):
        s = wl.tree_molecules_of_sizes([n], seed=400 + k)
        r = sv.Request(k, 0.0, s.n_atoms, s.atom_i, s.atom_j, s.x_old, s.x_unc, s.inv_mass, s.d)
        ref = orc.solve(s.x_old, s.x_unc, s.inv_mass, s.atom_i, s.atom_j, s.d, tol=1e-12)
        r.x, r.iterations, r.mol_status = ref.x.copy(), ref.iterations.astype(np.int32), ref.status.astype(np.int32)
        r.host = [None] * 7 + [torch.from_numpy(ref.lam.copy())]
        done.append(r)
    cpu, err = bench.serving_oracle(done, 1e-12, n_sample=3)
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0
    assert err["max_abs_x_nm"] == 0.0 and err["lambda_over_bound"] == 0.0
    assert err["max_abs_iterations_diff"] == 0 and err["statuses_equal"]
    done[1].x[3, 0] += 1e-9
    done[2].mol_status[0] = 1
    _, err = bench.serving_oracle(done, 1e-12, n_sample=3)
    assert abs(err["max_abs_x_nm"] - 1e-9) < 1e-12 and not err["statuses_equal"]
