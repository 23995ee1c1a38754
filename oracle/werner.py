"""Werner-state initial data through a shifted low-rank problem (oracle; test infrastructure only).

Paper: Sec. 5 "A full-rank state", eq. werner-sol.  rho_W = p I/2^n + (1 - p) rho_hat_0 is full
rank, but the q-LL and q-LLG flows from rho_W stay of the form p I/2^n + (1 - p) rho_hat(t), with
rho_hat the solution from rho_hat_0 of the same equation with kappa replaced by (1 - p) kappa
(the identity commutes with everything, and each commutator of the equation carries one factor
(1 - p) per rho).  Observables follow as Tr(A rho) = p/2^n Tr(A) + (1 - p) Tr(A rho_hat).
"""
from __future__ import annotations

import numpy as np

from . import dense_ei


def werner_state(V_hat, lam_hat, p: float):
    """Dense rho_W = p I/N + (1 - p) V diag(lam) V^*."""
    N = V_hat.shape[0]
    return p * np.eye(N) / N + (1.0 - p) * dense_ei.state(V_hat, lam_hat)


def evolve(V_hat, lam_hat, p: float, H, kappa: float, model: str, h: float, steps: int, scheme: str = "rk4"):
    """Low-rank factor of rho_hat(t): the EI scheme from rho_hat_0 with kappa -> (1 - p) kappa."""
    V, _ = dense_ei.integrate(V_hat, lam_hat, H, (1.0 - p) * kappa, model, h, steps, scheme)
    return V


def expectation(A, V_hat, lam_hat, p: float):
    """Tr(A rho) for rho = p I/N + (1 - p) rho_hat, rho_hat = V diag(lam) V^* (factored form)."""
    N = V_hat.shape[0]
    AV = A @ V_hat
    lowrank = np.sum(lam_hat * np.einsum("ij,ij->j", V_hat.conj(), AV))
    return p / N * np.trace(A) + (1.0 - p) * lowrank
