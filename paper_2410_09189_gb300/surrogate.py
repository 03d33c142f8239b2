"""Training utilities for the learned SCF seed (plumbing around the library's network calls).

The network, its features and targets, the loss, the gradient and Adam all run in the CUDA
library (``rmgtd.Net``); this module only records trajectories into device tensors, picks
mini-batches and sets the normalisation scales from training-set statistics.

Data: after every converged step j the context's rho_j and V_j (V_H + V_xc) are copied to
device tensors.  Sample j (2 <= j < nsteps) has features from (rho_j, rho_{j-1}, rho_{j-2})
and target (V_{j+1} - 2 V_j + V_{j-1}) / s_out: the residual of the paper's linear
extrapolation seed for step j + 1 (Algorithm 1).
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from . import rmgtd


def record(ctx: "rmgtd.Context", nsteps: int):
    """Propagate `nsteps` steps and keep rho and V_H + V_xc of every replica after each
    step (index 0 = the state before the first step).  Returns (rho, V, passes):
    float64 device tensors [nsteps + 1, nrep, Ng] and the SCF passes per step."""
    import torch

    nrep, Ng = ctx.nrep, ctx.Ng
    rho = torch.empty((nsteps + 1, nrep, Ng), dtype=torch.float64, device="cuda")
    V = torch.empty_like(rho)

    def grab(j):
        for r in range(nrep):
            ctx.field_into(rmgtd.FIELD_RHO, r, rho[j, r].data_ptr())
            ctx.field_into(rmgtd.FIELD_VHXC, r, V[j, r].data_ptr())

    grab(0)
    passes = []
    for j in range(1, nsteps + 1):
        st = ctx.step(1)
        passes.append(st["passes"].copy())
        grab(j)
    return rho, V, np.array(passes)


def scales(rho, V, steps) -> Dict[str, object]:
    """Feature scales s_0 = max |rho|, s_1, s_2 = RMS of the first and second differences,
    s_out = RMS of the extrapolation residual, over the training steps `steps`."""
    import torch

    j = torch.as_tensor(np.asarray(steps), device=rho.device)
    d1 = rho[j] - rho[j - 1]
    d2 = rho[j] - 2 * rho[j - 1] + rho[j - 2]
    t = V[j + 1] - 2 * V[j] + V[j - 1]
    rms = lambda a: float(torch.sqrt(torch.mean(a * a)).item())  # noqa: E731
    return {"in": [float(rho.abs().max().item()), rms(d1), rms(d2)], "out": rms(t)}


def samples(net: "rmgtd.Net", rho, V, steps):
    """Features X [len(steps) * nrep, 3, Ng] and targets T [len(steps) * nrep, Ng]
    (float32 device tensors) computed by the library's feature / target kernels."""
    import torch

    nrep, Ng = rho.shape[1], rho.shape[2]
    steps = list(steps)
    X = torch.empty((len(steps) * nrep, 3, Ng), dtype=torch.float32, device="cuda")
    T = torch.empty((len(steps) * nrep, Ng), dtype=torch.float32, device="cuda")
    for k, j in enumerate(steps):
        for r in range(nrep):
            i = k * nrep + r
            net.features(rho[j, r].data_ptr(), rho[j - 1, r].data_ptr(), rho[j - 2, r].data_ptr(),
                         X[i].data_ptr())
            net.targets(V[j + 1, r].data_ptr(), V[j, r].data_ptr(), V[j - 1, r].data_ptr(),
                        T[i].data_ptr())
    return X, T


def fit(net: "rmgtd.Net", X, T, iters: int, batch: int = 4, lr: float = 1e-3,
        decay_at: float = 0.7, seed: int = 0) -> List[float]:
    """Adam on random mini-batches (seeded); the learning rate drops 10x after a fraction
    `decay_at` of the iterations.  Returns the loss of every iteration."""
    import torch

    rng = np.random.default_rng(seed)
    n = X.shape[0]
    batch = min(batch, n, net.max_batch)
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=torch.float32, device="cuda")
    tb = torch.empty((batch,) + tuple(T.shape[1:]), dtype=torch.float32, device="cuda")
    hist = []
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(n, batch, replace=False), device="cuda")
        xb.copy_(X.index_select(0, idx))
        tb.copy_(T.index_select(0, idx))
        hist.append(net.backward(xb.data_ptr(), tb.data_ptr(), batch))
        net.adam(lr if it < decay_at * iters else 0.1 * lr)
    return hist


def seed_error(net: "rmgtd.Net", X, T, radius: int = 4):
    """RMS over interior points of the target (the paper's seed error, scaled) and of
    target - network output (the learned seed's error), averaged over the samples."""
    import torch

    n = net.n
    m = torch.zeros((n[2], n[1], n[0]), dtype=torch.bool, device="cuda")
    m[radius:n[2] - radius, radius:n[1] - radius, radius:n[0] - radius] = True
    m = m.reshape(-1)
    y = torch.empty((1, X.shape[2]), dtype=torch.float32, device="cuda")
    lin, learned = [], []
    for i in range(X.shape[0]):
        net.forward(X[i:i + 1].data_ptr(), y.data_ptr(), 1)
        t = T[i][m]
        lin.append(float(torch.sqrt(torch.mean(t * t)).item()))
        r = t - y[0][m]
        learned.append(float(torch.sqrt(torch.mean(r * r)).item()))
    return float(np.mean(lin)), float(np.mean(learned))


LAYERS = ((16, 3), (16, 16), (16, 16), (1, 16))   # (cout, cin) of the four layers


def init_params(seed: int, gain: float = 1.0) -> np.ndarray:
    """Seeded starting parameters: normal weights with std gain * sqrt(2 / (27 cin)), zero
    biases, and a zero last layer (so the untrained network is the paper's seed)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (co, ci) in enumerate(LAYERS):
        w = (np.zeros(co * ci * 27) if l == len(LAYERS) - 1
             else rng.standard_normal(co * ci * 27) * gain * np.sqrt(2.0 / (27 * ci)))
        parts += [w, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def train_on_trajectory(ctx: "rmgtd.Context", nsteps: int, iters: int, batch: int = 4,
                        lr: float = 1e-3, train_frac: float = 0.75, seed: int = 0,
                        init_seed: int = 7):
    """Record `nsteps` steps of `ctx`, train a network on the samples of the first
    `train_frac` of the trajectory and measure the seed errors on the rest.
    Returns (net, report)."""
    rho, V, passes = record(ctx, nsteps)
    J = np.arange(2, nsteps)
    ntr = int(train_frac * len(J))
    tr, te = J[:ntr], J[ntr:]
    sc = scales(rho, V, tr)
    net = rmgtd.Net(ctx.sys.n, max_batch=max(batch, ctx.nrep))
    net.set_scales(sc["in"], sc["out"])
    net.set_params(init_params(init_seed))
    Xtr, Ttr = samples(net, rho, V, tr)
    hist = fit(net, Xtr, Ttr, iters, batch=batch, lr=lr, seed=seed)
    Xte, Tte = samples(net, rho, V, te)
    lin, learned = seed_error(net, Xte, Tte)
    report = {"passes_recorded": float(passes.mean()), "scales": sc, "loss_first": hist[0],
              "loss_last": float(np.mean(hist[-50:])), "heldout_seed_rms_linear": lin,
              "heldout_seed_rms_learned": learned, "heldout_ratio": learned / lin,
              "train_samples": int(Xtr.shape[0]), "heldout_samples": int(Xte.shape[0])}
    return net, report
