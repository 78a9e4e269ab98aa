"""Training driver for the learned warm start (all arithmetic runs in the library).

Training data are (features, y) pairs where y = lambda * scale and lambda comes from the
plain FP64 solve (``ilves_solve`` with precision "fp64") of seeded chain or tree
molecules; features and scales come from ``ilves_mlp_features``.  Training calls
``ilves_mlp_train_step`` (tensor-core forward, float32 backward, Adam) on shuffled
mini-batches; this module only orchestrates.
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import workloads as wl


def _dev_inputs(s, dev):
    import torch

    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return f(s.x_old), f(s.x_unc), f(s.inv_mass), f(s.d)


def training_pairs(system, dev="cuda:0", tol=1e-12):
    """(features, target y, scale) tensors for every constraint of `system`."""
    topo = B.Topology(system.n_atoms, system.atom_i, system.atom_j)
    xo, xu, w, d = _dev_inputs(system, dev)
    _, lam, _, st = topo.solve(xo, xu, w, d, tol=tol, precision="fp64")
    feat, scale = B.features(topo, xo, xu, w, d)
    y = (lam * scale.double()).float()
    ok = (st == 0).all().item()
    return feat, y, scale, ok


def chain_training_set(n_pairs=500_000, seed=2000, dev="cuda:0"):
    """Chain64-distribution training pairs (63 per chain)."""
    n_chains = -(-n_pairs // 63)
    feat, y, _, ok = training_pairs(wl.chain_batch(n_chains, seed=seed), dev)
    return feat[:n_pairs], y[:n_pairs], ok


def tree_training_set(n_mol=4096, seed=3001, dev="cuda:0"):
    feat, y, _, ok = training_pairs(wl.tree_batch(n_mol=n_mol, seed=seed), dev)
    return feat, y, ok


def train(mlp, feat, y, epochs=20, batch=8192, lr=2e-3, lr_final=1e-4, seed=0):
    """Adam over shuffled mini-batches with a geometric learning-rate decay; returns losses."""
    import torch

    n = feat.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (-(-n // batch))
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    losses = []
    loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
    k = 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(feat.device)
        ep = []
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb = feat.index_select(0, idx).contiguous()
            yb = y.index_select(0, idx).contiguous()
            mlp.train_step(xb, yb, lr * decay**k, loss_out=loss)
            ep.append(loss.clone())
            k += 1
        losses.append(float(torch.stack(ep).mean().item()))
    return losses
