"""Time stepping with the GPU solver (constrained leap-frog, supplement Sec. 2.3 and Sec. 4),
and ring topologies (cycles in the constraint graph, like the paper's benzene system).

* pendulum (supplement Sec. 4 tables): the GPU solve inside a leap-frog loop reproduces
  the paper's maximum relative energy errors 2^-10, 2^-12, 2^-14 at 100/200/400 steps
  per period, i.e. second order in h;
* a constrained chain under a harmonic angle-free force field keeps every bond at its
  length (1e-12) over many steps, and the GPU trajectory matches the oracle's;
* benzene-like rings: parity with the oracle in every precision and both methods.
"""
import math
import os

import numpy as np
import pytest
import scipy.special as ss

torch = pytest.importorskip("torch")

from oracle import ilves_oracle as orc  # noqa: E402
from paper_2503_13075_gb300 import binding as B  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_pendulum_max_energy_error(steps_per_period, precision, periods=2.0):
    m, l, g = 1.0, 1.0, 9.82
    pivot = np.array([0.0, l, 0.0])
    q = np.zeros(3)
    v0 = np.array([1.0, 0.0, 0.0])
    theta = math.acos(1.0 - v0.dot(v0) / (2.0 * g * l))
    period = 4.0 * math.sqrt(l / g) * ss.ellipk(math.sin(theta / 2.0) ** 2)
    h = period / steps_per_period
    f = np.array([0.0, -m * g, 0.0])
    vh = v0 - 0.5 * h * (f / m + v0.dot(v0) / l * (pivot - q) / l)
    e0 = 0.5 * m * v0.dot(v0) + m * g * q[1]
    topo = B.Topology(2, [0], [1])
    inv = _t(np.array([0.0, 1.0 / m]))
    d = _t(np.array([l]))
    x_old = np.stack([pivot, q])
    worst = 0.0
    for _ in range(int(steps_per_period * periods)):
        x_unc = x_old.copy()
        x_unc[1] = x_old[1] + h * vh + h * h * f / m
        x, lam, it, st = topo.solve(_t(x_old), _t(x_unc), inv, d, precision=precision)
        assert st.item() == 0
        x = x.cpu().numpy()
        v_new = (x[1] - x_old[1]) / h
        vk = 0.5 * (vh + v_new)
        n = (x_old[1] - pivot) / np.linalg.norm(x_old[1] - pivot)
        vk = vk - vk.dot(n) * n
        e = 0.5 * m * vk.dot(vk) + m * g * x_old[1][1]
        worst = max(worst, abs(e - e0) / e0)
        vh, x_old = v_new, x
    return worst


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_pendulum_energy_error_with_gpu_solver(precision):
    rows = np.loadtxt(os.path.join(GOLDEN, "pendulum_energy.txt"))
    errs = []
    for spp, log2_err in rows[:2]:  # 100 and 200 steps per period keep the test short
        e = gpu_pendulum_max_energy_error(int(spp), precision)
        errs.append(e)
        assert abs(math.log2(e) - log2_err) < 0.3, (spp, math.log2(e))
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_constrained_chain_md_matches_oracle():
    """Leap-frog with a soft pair force: bonds stay at length, GPU and oracle trajectories agree."""
    s = wl.chain64(seed=77)
    n = s.n_atoms
    rng = np.random.default_rng(1)
    h = 0.002
    v = rng.normal(0, 0.5, (n, 3))
    topo = B.Topology(n, s.atom_i, s.atom_j)
    w, d = _t(s.inv_mass), _t(s.d)

    def force(x):  # weak springs between atoms three apart (keeps the chain compact)
        f = np.zeros_like(x)
        r = x[3:] - x[:-3]
        f[3:] -= 50.0 * r
        f[:-3] += 50.0 * r
        return f

    xg = s.x_old.copy()
    xo = s.x_old.copy()
    vg = v.copy()
    vo = v.copy()
    for _ in range(40):
        for x, vel, which in ((xg, vg, "gpu"), (xo, vo, "oracle")):
            x_unc = x + h * vel + h * h * s.inv_mass[:, None] * force(x)
            if which == "gpu":
                xn, lam, it, st = topo.solve(_t(x), _t(x_unc), w, d, precision="mixed")
                assert st.item() == 0
                xn = xn.cpu().numpy()
            else:
                r = orc.solve(x, x_unc, s.inv_mass, s.atom_i, s.atom_j, s.d)
                xn = r.x
            vel[:] = (xn - x) / h
            x[:] = xn
        assert orc.max_relative_violation(xg, s.atom_i, s.atom_j, s.d) <= 1e-12
    assert np.abs(xg - xo).max() <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_df"])
@pytest.mark.parametrize("method", ["newton", "chord"])
def test_benzene_rings(prec, method):
    s = wl.benzene_batch(n_mol=64)
    ref = orc.solve_system(s, tol=1e-12)
    topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    x, lam, it, st = topo.solve(_t(s.x_old), _t(s.x_unc), _t(s.inv_mass), _t(s.d), precision=prec,
                                method=method, max_iter=60)
    x, lam, st = x.cpu().numpy(), lam.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0)
    assert np.abs(x - ref.x).max() <= 1e-10
    assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= 1e-12
    assert np.all(np.abs(lam - ref.lam) <= 1e-8 * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())
