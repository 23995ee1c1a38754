"""Training and evaluation of the learned step controller.

Data: the plain adaptive controller run with a step-doubling judge on every step
(`judge_every=1`, `record=True`) on open chains; each record holds the step features, the
spectral drift of the step and its judged local error.  The target is log(err / drift): the
network learns how the free drift indicator relates to the local error, so that the library's
learned rule can estimate the error of a step without the extra two half-steps of a judge.
Training runs on the GPU through the network's own gradient and Adam kernels.
"""
from __future__ import annotations

import numpy as np

from . import Lrei, Mlp, NFEAT


def generate(workloads, t_end=0.3, tols=(1e-7, 1e-9), precision="fp64"):
    """Run the plain controller with per-step judging; return (X, Y) training arrays."""
    import torch
    Xs, Ys = [], []
    for w in workloads:
        for tol in tols:
            L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, precision, w.r)
            dt = torch.complex128 if precision == "fp64" else torch.complex64
            L.set_state(torch.from_numpy(w.V).to("cuda", dt), w.lam)
            L.controller_config(judge_every=1, record=True, h0=0.01)
            L.step_adaptive(t_end, tol, 0)
            rows = L.controller_records()
            drift, err = rows[:, NFEAT + 1], rows[:, NFEAT + 2]
            ok = (err > 0) & (drift > 0)
            Xs.append(rows[ok, :NFEAT])
            Ys.append(np.log(err[ok] / drift[ok])[:, None])
            L.close()
    return np.concatenate(Xs).astype(np.float32), np.concatenate(Ys).astype(np.float32)


HIDDEN = 128   # width of both hidden layers (fixed by the library's network)


def init_params(n_in, n_out, seed=0, hidden=HIDDEN):
    """Glorot-uniform initial weights in the library's flat layout [W1|b1|W2|b2|W3|b3]."""
    rng = np.random.default_rng(seed)

    def glorot(o, i):
        lim = np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, size=(o, i))
    parts = [glorot(hidden, n_in), np.zeros(hidden), glorot(hidden, hidden), np.zeros(hidden),
             glorot(n_out, hidden), np.zeros(n_out)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def fit(X, Y, iters=3000, lr=2e-3, seed=0, batch=512):
    """Fit the controller network on the GPU with minibatch Adam; returns (net, train loss).

    Features and targets are standardised for training (raw features span many decades);
    the scalings are then folded into the first and last layers, so the returned network
    takes the raw features the step controller builds.
    """
    import torch
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    mu, sd = X.mean(0), X.std(0)
    sd = np.where(sd > 1e-6 * np.maximum(1.0, np.abs(mu)), sd, 1.0)
    ymu, ysd = Y.mean(0), Y.std(0)
    ysd = np.where(ysd > 1e-12, ysd, 1.0)
    n_in, n_out = X.shape[1], Y.shape[1]
    net = Mlp(n_in, n_out, init_params(n_in, n_out, seed))
    Xd = torch.from_numpy(((X - mu) / sd).astype(np.float32)).cuda()
    Yd = torch.from_numpy(((Y - ymu) / ysd).astype(np.float32)).cuda()
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = X.shape[0]
    for it in range(iters):
        if n > batch:
            idx = torch.randint(0, n, (batch,), device="cuda", generator=g)
            net.grads(Xd[idx], Yd[idx])
        else:
            net.grads(Xd, Yd)
        net.adam(lr=lr)
    # fold: W1' = W1 / sd, b1' = b1 - W1' mu; W3' = ysd W3, b3' = ysd b3 + ymu
    p = net.get_params().astype(np.float64)
    h = HIDDEN
    o = 0
    W1 = p[o:o + h * n_in].reshape(h, n_in); o += h * n_in
    b1 = p[o:o + h]; o += h
    o += h * h + h
    W3 = p[o:o + n_out * h].reshape(n_out, h); o3 = o; o += n_out * h
    b3 = p[o:o + n_out]
    W1n = W1 / sd[None, :]
    b1n = b1 - W1n @ mu
    q = p.copy()
    q[:h * n_in] = W1n.reshape(-1)
    q[h * n_in:h * n_in + h] = b1n
    q[o3:o3 + n_out * h] = (ysd[:, None] * W3).reshape(-1)
    q[o3 + n_out * h:o3 + n_out * h + n_out] = ysd * b3 + ymu
    net.set_params(q.astype(np.float32))
    loss, _ = net.grads(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(Y.astype(np.float32)).cuda())
    return net, loss
