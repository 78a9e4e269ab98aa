"""Pins for the warm-start oracle (features, network, gradients) -- all CPU.

* central differences pin the analytic gradient (a dropped ReLU mask, a transposed
  weight or a missing 1/N fails it);
* geometric facts pin the features: feasible input -> zero violation features; a
  collinear chain has coupling cosine -1 on interior bonds; for one constraint the
  Jacobi guess y = f0 is the exact target to first order (pins the target scale);
* the bfloat16 rounding matches torch's conversion.
"""
import math

import numpy as np
import pytest

from oracle import ilves_oracle as orc
from oracle import mlp_oracle as mo
from paper_2503_13075_gb300 import workloads as wl


def test_param_count():
    assert mo.N_PARAMS == 16 * 128 + 128 + 128 * 128 + 128 + 128 + 1 == 18817


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    theta = mo.init_params(seed) * 0.5
    X = rng.normal(size=(24, 16))
    t = rng.normal(size=24)
    loss, g = mo.loss_and_grad(theta, X, t)
    h = 1e-6
    idx = rng.choice(mo.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [mo.N_PARAMS - 1, 2048, 2048 + 128 + 5]])  # b3, b1[0], a W2 entry
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mo.loss_and_grad(theta + e, X, t)[0] - mo.loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-9, -2.5e-3, 3.14159, 1e-30, 65504.0, 1 + 2**-7])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mo.bf16(v), ref)


def test_features_of_feasible_input_and_straight_chain():
    n = 8
    xo = np.zeros((n, 3))
    xo[:, 0] = 0.15 * np.arange(n)
    ai = np.arange(n - 1)
    aj = ai + 1
    d = np.full(n - 1, 0.15)
    w = np.ones(n)
    F, sc = mo.features(xo, xo + 0.3, w, ai, aj, d)
    assert np.allclose(F[:, [0, 1, 3]], 0.0, atol=1e-12)  # feasible, aligned, unperturbed
    # interior bond k = (k, k+1): neighbour (k-1, k) at atom i in slot 0, (k+1, k+2) at atom j in slot 2
    for k in range(1, n - 2):
        assert F[k, 5] == pytest.approx(-1.0) and F[k, 11] == pytest.approx(-1.0)
        assert F[k, 6] == pytest.approx(0.5) and F[k, 12] == pytest.approx(0.5)
        assert F[k, 8] == 0.0 and F[k, 14] == 0.0  # second slots empty on a chain
    assert np.all(sc > 0)


def test_jacobi_guess_is_first_order_exact_for_one_constraint():
    for sigma in (1e-3, 1e-4):
        s = wl.two_atoms(d=0.1, w1=1 / 12.011, w2=1 / 1.008, seed=4, sigma=sigma)
        F, sc = mo.features(s.x_old, s.x_unc, s.inv_mass, s.atom_i, s.atom_j, s.d)
        lam = orc.solve_system(s).lam
        y = lam[0] * sc[0]
        assert abs(y - F[0, 0]) <= 10 * F[0, 0] ** 2 + 1e-12


def test_neighbour_slots_follow_constraint_order():
    s = wl.tree_batch(n_mol=3, seed=9)
    nbr, nat = mo.neighbours(s.atom_i, s.atom_j)
    for k in range(len(s.d)):
        for q in range(4):
            l = nbr[k, q]
            if l < 0:
                continue
            a = nat[k, q]
            assert a == (s.atom_i[k] if q < 2 else s.atom_j[k])
            assert a in (s.atom_i[l], s.atom_j[l]) and l != k
        for side in (0, 1):
            ls = [l for l in nbr[k, 2 * side:2 * side + 2] if l >= 0]
            assert ls == sorted(ls)


# Hand-worked parameters: hidden unit h < 4 copies feature h, unit 4 copies -feature 0, b1[1] =
# 0.5; the second layer is the identity on units 0..4 with b2[2] = -0.25 and b2[3] = 0.5; the
# output weights are (1, 2, 1, -1, 0.5) and b3 = -1.  With H1 = relu(W1 x + b1) and
# H2 = relu(W2 H1 + b2) the output y = w3 . H2 + b3 of each row below is worked out by hand:
#   x = (1, -2, 0.5, -1):  H1 = (1, 0, 0.5, 0, 0),   H2 = (1, 0, 0.25, 0.5, 0),  y = -0.25
#   x = (-1, 0.25, 0, 0):  H1 = (0, 0.75, 0, 0, 1),  H2 = (0, 0.75, 0, 0.5, 1),  y = 0.5
#   x = (0.5, 1, 2, 0):    H1 = (0.5, 1.5, 2, 0, 0), H2 = (0.5, 1.5, 1.75, 0.5, 0), y = 3.75
# A missing ReLU in either hidden layer, a ReLU on the output, or a bias added twice or not at
# all changes at least one of them.  Every value is exact in bfloat16.
HAND_X = np.array([[1.0, -2.0, 0.5, -1.0], [-1.0, 0.25, 0.0, 0.0], [0.5, 1.0, 2.0, 0.0]])
HAND_Y = np.array([-0.25, 0.5, 3.75])


def hand_params():
    p = {name: np.zeros(shape) for name, shape in mo.SIZES}
    for h in range(4):
        p["W1"][h, h] = 1.0
    p["W1"][4, 0] = -1.0
    p["b1"][1] = 0.5
    for h in range(5):
        p["W2"][h, h] = 1.0
    p["b2"][2], p["b2"][3] = -0.25, 0.5
    p["w3"][:5] = [1.0, 2.0, 1.0, -1.0, 0.5]
    p["b3"][0] = -1.0
    return mo.pack(p)


def hand_features():
    X = np.zeros((len(HAND_X), mo.N_FEAT))
    X[:, :4] = HAND_X
    return X


@pytest.mark.parametrize("bf16_mode", [False, True])
def test_forward_pass_on_hand_parameters(bf16_mode):
    y, _ = mo.forward(hand_params(), hand_features(), bf16_mode=bf16_mode)
    assert np.array_equal(y, HAND_Y)
