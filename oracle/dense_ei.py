"""Dense eigenmode integration (EI) -- the plain definition the low-rank method reproduces.

Oracle; test infrastructure only.  hbar = 1.

Paper passages followed:
  * eq. q-LL:  rho' = i[rho, H] - kappa [rho, [rho, H]]                 (Sec. 1)
  * eq. q-LLG: rho' = i[rho, H] + i kappa [rho, rho'], solved through the
    eigendecomposition rho = V Lambda V^* (eq. eigendecom), X = V^* rho' V
    (eq. Xdef), the Sylvester-type equation (I+S)X - XS = D with
    D = i V^*[rho,H]V and S = -i kappa Lambda (eqs. q-LLG-3, Dmat), solved
    column-wise by X_{il} = D_{il} / (1 + s_i - s_l) (eq. x_ell_sol), and
    rho' = V X V^* (eq. q-LLG-final)                                    (Sec. 2)
  * EI projection: every stage matrix is replaced by V Lambda_0 V^*, with V
    the eigenvectors of its r largest eigenvalues and Lambda_0 the initial
    spectrum (Sec. 2, last paragraph; Sec. 3.7)
  * s-stage RK in the form of eq. rk:sstageform, with f evaluated at the
    projected stage matrices (Sec. 3.7)
  * Adams-Bashforth m-step form (Sec. 3.8), started with RK4 steps.

Readings where the paper is ambiguous: AB2 uses b = (3/2, -1/2) (the printed -3/2 is
a typo: the weights of a consistent 2-step AB method sum to one); the r
largest eigenvalues are taken by algebraic value, matched in decreasing order
to Lambda_0 sorted decreasingly.
"""
from __future__ import annotations

import numpy as np

# Butcher tableaus of the explicit RK schemes (Sec. 3.7): (A, b), A strictly lower triangular.
RK_TABLEAUS = {
    "rk1": (np.zeros((1, 1)), np.array([1.0])),
    # the paper's RK2 example: a21 = 1, b1 = b2 = 1/2
    "rk2": (np.array([[0.0, 0.0], [1.0, 0.0]]), np.array([0.5, 0.5])),
    # Kutta's third-order method
    "rk3": (np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [-1.0, 2.0, 0.0]]),
            np.array([1.0, 4.0, 1.0]) / 6.0),
    # classic fourth-order RK
    "rk4": (np.array([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0],
                      [0.0, 0.0, 1.0, 0.0]]),
            np.array([1.0, 2.0, 2.0, 1.0]) / 6.0),
}

# Adams-Bashforth weights b_1..b_m multiplying f(rho_k), f(rho_{k-1}), ... (Sec. 3.8)
AB_WEIGHTS = {
    "ab2": np.array([3.0, -1.0]) / 2.0,
    "ab3": np.array([23.0, -16.0, 5.0]) / 12.0,
    "ab4": np.array([55.0, -59.0, 37.0, -9.0]) / 24.0,
}


def comm(A, B):
    return A @ B - B @ A


def f_qll(rho, H, kappa):
    """Right-hand side of eq. q-LL."""
    c = comm(rho, H)
    return 1j * c - kappa * comm(rho, c)


def f_qllg(rho, H, kappa):
    """Right-hand side of eq. q-LLG through eqs. eigendecom, Dmat, x_ell_sol and q-LLG-final."""
    rho = 0.5 * (rho + rho.conj().T)
    w, U = np.linalg.eigh(rho)
    D = 1j * (U.conj().T @ comm(rho, H) @ U)          # eq. Dmat
    s = -1j * kappa * w                                 # diagonal of S = -i kappa Lambda
    X = D / (1.0 + s[:, None] - s[None, :])             # eq. x_ell_sol, column l divides by 1 + s - s_l
    return U @ X @ U.conj().T                           # eq. q-LLG-final


def rhs(rho, H, kappa, model):
    if model == "qll":
        return f_qll(rho, H, kappa)
    if model == "qllg":
        return f_qllg(rho, H, kappa)
    raise ValueError(model)


def spectral_projection(K, r):
    """Eigenvectors of the r largest eigenvalues of the Hermitian part of K, sorted decreasingly.

    Returns (V, mu): V is N x r with orthonormal columns, mu the r eigenvalues.
    """
    Kh = 0.5 * (K + K.conj().T)
    w, U = np.linalg.eigh(Kh)
    idx = np.argsort(-w, kind="stable")[:r]
    return U[:, idx], w[idx]


def state(V, lam0):
    return (V * lam0[None, :]) @ V.conj().T


def ei_rk_step(V, lam0, H, kappa, model, h, scheme="rk4"):
    """One projected EI-RK step (eq. rk:sstageform with the EI projection at each stage).

    Returns (V_next, mu): mu are the r largest eigenvalues of the unprojected rho_{k+1}.
    """
    A, b = RK_TABLEAUS[scheme]
    r = lam0.shape[0]
    K1 = state(V, lam0)
    F = [rhs(K1, H, kappa, model)]
    for j in range(1, len(b)):
        Kj = K1 + h * sum(A[j, l] * F[l] for l in range(j))
        Vj, _ = spectral_projection(Kj, r)
        F.append(rhs(state(Vj, lam0), H, kappa, model))
    rho_next = K1 + h * sum(b[l] * F[l] for l in range(len(b)))
    return spectral_projection(rho_next, r)


def ei_ab_step(V, lam0, H, kappa, model, h, hist_F, scheme="ab3"):
    """One projected EI-AB step.  hist_F holds f(rho_{k-1}), f(rho_{k-2}), ... (most recent first).

    Returns (V_next, mu, F_k) with F_k = f(rho_k) to be prepended to the history.
    """
    b = AB_WEIGHTS[scheme]
    r = lam0.shape[0]
    rho = state(V, lam0)
    Fk = rhs(rho, H, kappa, model)
    Fs = [Fk] + list(hist_F)
    rho_next = rho + h * sum(b[l] * Fs[l] for l in range(len(b)))
    Vn, mu = spectral_projection(rho_next, r)
    return Vn, mu, Fk


def observables(V, lam0, H, Mops):
    """Energy <H>, magnetisations <M_x>, <M_y>, <M_z>, purity Tr(rho^2) and trace Tr(rho) (Sec. 3.6)."""
    rho = state(V, lam0)
    out = {"energy": float(np.real(np.trace(H @ rho)))}
    for v in "xyz":
        out["m" + v] = float(np.real(np.trace(Mops[v] @ rho)))
    out["purity"] = float(np.real(np.trace(rho @ rho)))
    out["trace"] = float(np.real(np.trace(rho)))
    out["comm_norm"] = float(np.linalg.norm(comm(rho, H)))      # ||[rho, H]||_F, dense
    return out


def integrate(V0, lam0, H, kappa, model, h, steps, scheme="rk4", Mops=None, every=1):
    """Run `steps` EI steps; returns (V_final, list of (step, observables, mu)).

    AB schemes take their first m-1 steps with RK4 (a start-up of global order >= m-1).
    """
    V = V0
    traj = []
    mu = None
    if scheme.startswith("rk"):
        for k in range(steps):
            V, mu = ei_rk_step(V, lam0, H, kappa, model, h, scheme)
            if Mops is not None and ((k + 1) % every == 0 or k + 1 == steps):
                traj.append((k + 1, observables(V, lam0, H, Mops), mu))
        return V, traj
    m = len(AB_WEIGHTS[scheme])
    hist = []
    for k in range(steps):
        if k < m - 1:
            hist.insert(0, rhs(state(V, lam0), H, kappa, model))
            V, mu = ei_rk_step(V, lam0, H, kappa, model, h, "rk4")
        else:
            V, mu, Fk = ei_ab_step(V, lam0, H, kappa, model, h, hist[: m - 1], scheme)
            hist.insert(0, Fk)
        hist = hist[: m - 1]
        if Mops is not None and ((k + 1) % every == 0 or k + 1 == steps):
            traj.append((k + 1, observables(V, lam0, H, Mops), mu))
    return V, traj
