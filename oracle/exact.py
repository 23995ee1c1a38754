"""Closed-form references (oracle; test infrastructure only).  hbar = 1.

* Pure-state solution of q-LL (Sec. 1, eq. exact_q-LL), corrected reading:
  the printed e^{-i H~ t} rho_0 e^{+i H~ t} with H~ = (1 - i kappa) H is not
  Hermitian for kappa > 0; the Hermitian reading keeps the adjoint on the
  right factor, rho(t) = psi psi^* / |psi|^2 with psi = e^{-(i + kappa) H t} psi_0.
  The q-LLG pure-state solution is the same at rescaled time t / (1 + kappa^2)
  (Sec. 1; Sec. 5.3).
* kappa = 0: both equations reduce to rho' = i[rho, H], whose solution is
  rho(t) = e^{-iHt} rho_0 e^{iHt}.
Both are evaluated from a dense eigendecomposition of H.
"""
from __future__ import annotations

import numpy as np


def rank1_solution(psi0, H, kappa, t, model="qll"):
    if model == "qllg":
        t = t / (1.0 + kappa * kappa)
    w, U = np.linalg.eigh(H)
    c = U.conj().T @ psi0
    psi = U @ (np.exp(-(1j + kappa) * w * t) * c)
    psi = psi / np.linalg.norm(psi)
    return np.outer(psi, psi.conj())


def unitary_solution(rho0, H, t):
    w, U = np.linalg.eigh(H)
    E = U @ np.diag(np.exp(-1j * w * t)) @ U.conj().T
    return E @ rho0 @ E.conj().T
