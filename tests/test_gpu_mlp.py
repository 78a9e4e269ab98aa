"""GPU tests of the learned warm start through the C ABI, against the FP64 MLP oracle.

Bounds: features within 1e-4 absolute (float32 from truncated float64 inputs); network
output within 1e-3 relative to max |y| of the oracle's bfloat16 emulation; gradients
within 5e-3 of max |g| (float32 accumulation vs float64); a warm-started solve meets
the same parity bounds as the zero start, in no more iterations after training.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ilves_oracle as orc  # noqa: E402
from oracle import mlp_oracle as mo  # noqa: E402
from paper_2503_13075_gb300 import binding as B  # noqa: E402
from paper_2503_13075_gb300 import warmstart as ws  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def dev_inputs(s):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return f(s.x_old), f(s.x_unc), f(s.inv_mass), f(s.d)


@pytest.mark.parametrize("maker", [wl.chain64, lambda: wl.tree_batch(n_mol=40, seed=12)])
def test_features_match_oracle(maker):
    s = maker()
    topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    F, sc = B.features(topo, *dev_inputs(s))
    Fo, sco = mo.features(s.x_old, s.x_unc, s.inv_mass, s.atom_i, s.atom_j, s.d)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, atol=1e-4, rtol=1e-4)
    np.testing.assert_allclose(sc.cpu().numpy(), sco, rtol=1e-4)


def test_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(3)
    n = 1000  # several 16-row tiles and a ragged tail
    X = rng.normal(size=(n, 16)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    mlp = B.Mlp(max_batch=4096, seed=5)
    theta = mlp.get_params().astype(np.float64)
    assert np.allclose(theta, mlp.get_params())
    Xd = torch.from_numpy(X).to(DEV)
    y = mlp.forward(Xd).cpu().numpy()
    yo, _ = mo.forward(theta, X.astype(np.float64), bf16_mode=True)
    assert np.abs(y - yo).max() <= 1e-3 * np.abs(yo).max()
    g, loss = mlp.gradient(Xd, torch.from_numpy(t).to(DEV))
    lo, go = mo.loss_and_grad(theta, X.astype(np.float64), t.astype(np.float64), bf16_mode=True)
    g = g.cpu().numpy()
    assert abs(loss.item() - lo) <= 1e-3 * lo
    for name_off, size in ((0, 2048), (2048, 128), (2176, 16384), (18560, 128), (18688, 128), (18816, 1)):
        a, b = g[name_off:name_off + size], go[name_off:name_off + size]
        assert np.abs(a - b).max() <= 5e-3 * max(np.abs(go).max(), 1e-12), name_off


def test_training_reduces_loss_and_warm_start_keeps_parity():
    feat, y, ok = ws.chain_training_set(n_pairs=63 * 400, seed=2000)
    assert ok
    mlp = B.Mlp(max_batch=8192, seed=1)
    losses = ws.train(mlp, feat, y, epochs=15, batch=2048, lr=3e-3, lr_final=3e-4)
    assert losses[-1] < 0.5 * losses[0]
    # held-out chains: warm start from the network
    s = wl.chain_batch(50, seed=9000)
    ref = orc.solve_system(s, tol=1e-12)
    topo = B.Topology(s.n_atoms, s.atom_i, s.atom_j)
    xo, xu, w, d = dev_inputs(s)
    it0 = topo.solve(xo, xu, w, d, precision="mixed")[2].cpu().numpy()
    for guess in (mlp, None):  # network and diagonal (Jacobi) guess
        lam0 = B.warm_start(guess, topo, xo, xu, w, d)
        x, lam, it, st = topo.solve(xo, xu, w, d, precision="mixed", lambda0=lam0)
        x, lam, it, st = x.cpu().numpy(), lam.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()
        assert np.all(st == 0)
        assert np.abs(x - ref.x).max() <= 1e-10
        assert orc.max_relative_violation(x, s.atom_i, s.atom_j, s.d) <= 1e-12
        assert np.all(np.abs(lam - ref.lam) <= 1e-8 * np.abs(ref.lam) + 1e-10 * np.abs(ref.lam).max())
        if guess is mlp:
            assert it.mean() <= it0.mean()


def test_forward_on_hand_parameters():
    """The tensor-core forward pass on the hand-worked parameter set of the oracle pins
    (tests/test_mlp_oracle.py): every output is exact, across tile boundaries and a ragged
    tail (the three rows repeated 100 times)."""
    from tests.test_mlp_oracle import HAND_Y, hand_features, hand_params

    mlp = B.Mlp(max_batch=512, seed=7)
    mlp.set_params(hand_params().astype(np.float32))
    X = np.tile(hand_features(), (100, 1)).astype(np.float32)
    y = mlp.forward(torch.from_numpy(X).to(DEV)).cpu().numpy()
    assert mlp.check() == 0
    assert np.array_equal(y, np.tile(HAND_Y, 100).astype(np.float32))


def test_tensor_core_wait_runs_out():
    """A bounded device wait that runs out: in wait-test mode the forward kernel waits on a
    completion barrier nothing signals (no MMA in flight), gives up, frees its tensor memory
    and returns; ilves_mlp_check reports it.  A fresh network afterwards computes normally."""
    X = torch.zeros(128, 16, dtype=torch.float32, device=DEV)
    mlp = B.Mlp(max_batch=256, seed=8)
    mlp.set_wait_test(True)
    mlp.forward(X)
    assert mlp.check() >= 1
    code = B.lib().ilves_mlp_check(mlp._h, ctypes.byref(ctypes.c_int32()))
    assert code == 5  # ILVES_ERR_TIMEOUT
    m2 = B.Mlp(max_batch=256, seed=9)
    from tests.test_mlp_oracle import HAND_Y, hand_features, hand_params

    m2.set_params(hand_params().astype(np.float32))
    y = m2.forward(torch.from_numpy(hand_features().astype(np.float32)).to(DEV)).cpu().numpy()
    assert m2.check() == 0 and np.array_equal(y, HAND_Y.astype(np.float32))


def test_params_round_trip_and_save(tmp_path):
    mlp = B.Mlp(max_batch=64, seed=2)
    th = mo.init_params(11).astype(np.float32)
    mlp.set_params(th)
    assert np.array_equal(mlp.get_params(), th)
    mlp.save(tmp_path / "w.npy")
    m2 = B.Mlp(max_batch=64, seed=3)
    m2.load(tmp_path / "w.npy")
    assert np.array_equal(m2.get_params(), th)
