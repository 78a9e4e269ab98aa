"""FP64 CPU oracle for the learned warm start (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` may import this module.
The paper starts Newton from lambda_0 = 0 (supplement Sec. 2.3); the warm start is an
addition of this project, so there is no passage to follow for the network itself.
What it computes:

Features (16 per constraint k with atoms i, j; s = x_unc,i - x_unc,j,
rho = x_old,i - x_old,j, W = w_i + w_j):
  f0 = (s.s - d^2) / d^2        initial relative violation
  f1 = s.rho / d^2 - 1          alignment of the update with the reference bond
  f2 = (w_i - w_j) / W          mass asymmetry
  f3 = |s - rho|^2 / d^2        perturbation size
  for each of 4 neighbour slots (line-graph neighbours sharing atom i: slots 0-1,
  sharing atom j: slots 2-3, ascending constraint id, missing -> zeros), neighbour l
  sharing atom a:
    (s_l.s_l - d_l^2) / d_l^2,  s_k(a) s_l(a) s.rho_l / (d d_l),  w_a / W
Target: y = lambda * scale with scale = 4 W (s.rho) / d^2, so lambda_0 = y / scale;
the "diagonal" (Jacobi) guess is y = f0.

Network: 16 -> 128 -> ReLU -> 128 -> ReLU -> 1, parameters packed as
[W1 (128x16, out x in), b1, W2 (128x128), b2, w3 (128), b3].  With ``bf16=True`` the
inputs, W1, W2 and the first hidden layer are rounded to bfloat16 (round to nearest
even) where the GPU kernels round them; gradients treat the rounding as identity.
Loss: mean squared error.
"""
from __future__ import annotations

import numpy as np

N_FEAT, N_HID = 16, 128
SIZES = [("W1", (N_HID, N_FEAT)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def neighbours(atom_i, atom_j):
    """Up to 2 neighbours per endpoint, ascending constraint id; (nbr, shared atom)."""
    n_c = len(atom_i)
    at = {}
    for k in range(n_c):
        at.setdefault(int(atom_i[k]), []).append(k)
        at.setdefault(int(atom_j[k]), []).append(k)
    nbr = -np.ones((n_c, 4), np.int64)
    nat = -np.ones((n_c, 4), np.int64)
    for k in range(n_c):
        for side, a in enumerate((int(atom_i[k]), int(atom_j[k]))):
            others = [l for l in sorted(at[a]) if l != k][:2]
            for q, l in enumerate(others):
                nbr[k, 2 * side + q] = l
                nat[k, 2 * side + q] = a
    return nbr, nat


def features(x_old, x_unc, inv_mass, atom_i, atom_j, d):
    """(features (n_c, 16), scale (n_c,)) by explicit loops over constraints."""
    x_old = np.asarray(x_old, np.float64).reshape(-1, 3)
    x_unc = np.asarray(x_unc, np.float64).reshape(-1, 3)
    n_c = len(atom_i)
    nbr, nat = neighbours(atom_i, atom_j)
    F = np.zeros((n_c, N_FEAT))
    scale = np.zeros(n_c)
    for k in range(n_c):
        i, j = int(atom_i[k]), int(atom_j[k])
        s = x_unc[i] - x_unc[j]
        rho = x_old[i] - x_old[j]
        d2 = d[k] * d[k]
        W = inv_mass[i] + inv_mass[j]
        F[k, 0] = (s @ s - d2) / d2
        F[k, 1] = (s @ rho) / d2 - 1.0
        F[k, 2] = (inv_mass[i] - inv_mass[j]) / W
        F[k, 3] = (s - rho) @ (s - rho) / d2
        scale[k] = 4.0 * W * (s @ rho) / d2
        for q in range(4):
            l = nbr[k, q]
            if l < 0:
                continue
            a = nat[k, q]
            il, jl = int(atom_i[l]), int(atom_j[l])
            sl_ = x_unc[il] - x_unc[jl]
            rl = x_old[il] - x_old[jl]
            dl2 = d[l] * d[l]
            sk = 1.0 if a == i else -1.0
            sl = 1.0 if a == il else -1.0
            F[k, 4 + 3 * q] = (sl_ @ sl_ - dl2) / dl2
            F[k, 5 + 3 * q] = sk * sl * (s @ rl) / (d[k] * d[l])
            F[k, 6 + 3 * q] = inv_mass[a] / W
    return F, scale


def forward(theta, X, bf16_mode=False):
    """Returns y and the cache needed by ``backward``."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    W1, W2 = p["W1"], p["W2"]
    if bf16_mode:
        X, W1, W2 = bf16(X), bf16(W1), bf16(W2)
    Z1 = X @ W1.T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    if bf16_mode:
        H1 = bf16(H1)
    Z2 = H1 @ W2.T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, dict(X=X, W1=W1, W2=W2, Z1=Z1, H1=H1, Z2=Z2, H2=H2, w3=p["w3"])


def loss_and_grad(theta, X, t, bf16_mode=False):
    """Mean squared error and its gradient with respect to the packed parameters."""
    y, c = forward(theta, X, bf16_mode)
    n = len(t)
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = c["H2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dZ2 = np.outer(dy, c["w3"]) * (c["Z2"] > 0)
    g["W2"] = dZ2.T @ c["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ c["W2"]) * (c["Z1"] > 0)
    g["W1"] = dZ1.T @ c["X"]
    g["b1"] = dZ1.sum(axis=0)
    return loss, pack(g)


def init_params(seed):
    """He-uniform weights, zero biases (same scheme as the library's initialiser)."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.uniform(-1, 1, (N_HID, N_FEAT)) * np.sqrt(6.0 / N_FEAT),
        "b1": np.zeros(N_HID),
        "W2": rng.uniform(-1, 1, (N_HID, N_HID)) * np.sqrt(6.0 / N_HID),
        "b2": np.zeros(N_HID),
        "w3": rng.uniform(-1, 1, N_HID) * np.sqrt(3.0 / N_HID),
        "b3": np.zeros(1),
    }
    return pack(p)
