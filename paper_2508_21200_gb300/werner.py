"""Werner-state initial data on top of the context API (Sec. 5, eq. werner-sol).

rho_W = p I/N + (1 - p) rho_hat_0 is full rank, but its q-LL / q-LLG flow stays
p I/N + (1 - p) rho_hat(t), where rho_hat solves the same equation from the low-rank
rho_hat_0 with kappa replaced by (1 - p) kappa.  So: create the context with
`shifted_kappa(kappa, p)`, set rho_hat_0 as the state, step as usual, and map the
context's observables with `observables`.  H and the magnetisations are traceless, so their
expectations scale by (1 - p); the spectrum and the purity pick up the identity part.
"""
from __future__ import annotations

import numpy as np


def shifted_kappa(kappa: float, p: float) -> float:
    """Damping of the low-rank part: (1 - p) kappa, for 0 <= p < 1."""
    if not (0.0 <= p < 1.0):
        raise ValueError("Werner weight p must lie in [0, 1)")
    return (1.0 - p) * kappa


def observables(obs_hat: dict, p: float, n: int) -> dict:
    """Observables of rho = p I/N + (1 - p) rho_hat from those of rho_hat (N = 2^n)."""
    N = float(1 << n)
    q = 1.0 - p
    out = dict(obs_hat)
    for k in ("energy", "mx", "my", "mz", "comm_norm"):
        out[k] = q * obs_hat[k]
    out["trace"] = p + q * obs_hat["trace"]
    out["purity"] = p * p / N + 2.0 * p * q / N * obs_hat["trace"] + q * q * obs_hat["purity"]
    for k in ("ritz", "lambda0"):
        if k in obs_hat:
            out[k] = p / N + q * np.asarray(obs_hat[k])
    return out
