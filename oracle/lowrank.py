"""Plain low-rank LREI as the paper states it (oracle; test infrastructure only).  hbar = 1.

Passages followed, in the paper's order:
  * partial eigendecomposition rho = V~ Lambda~ V~^* (Sec. 3.1, eq. partial-eigendecom)
  * X blocks: X11 = cwd(D11, E11 + L11 + L11^*), X12 = cwd(D12, E12 + L12) with
    D11 = i(Lambda G - G Lambda), D12 = i Lambda V~^* H V^  (Sec. 3.3, eq. X-blocks-sol);
    for q-LL X11 and X12 of Sec. 4, eq. X-blocks-sol-qLL
  * products A V^ and V^ A through the Householder vectors u_k of V~:
    A P = A - beta (A u) u^*, P A = A - beta u (u^* A), Q = P_1 ... P_r,
    A V^ = last N-r columns of A Q, V^ A = Q [0; A]  (Sec. 3.4, eq. Householder-mat)
  * Z = V~ X11 + W, W = V^ X12^* so that f = Z V~^* + V~ W^*  (Sec. 3.5, eq. q-LLG-low-rank)
  * stage matrices in factored form sum_l (A_l V_l^* + V_l B_l^*)  (Sec. 3.7, eqs. K-expand,
    rho-expand) and their partial eigendecomposition by implicitly restarted Lanczos (ARPACK,
    via SciPy) on the operator g(x) = sum_l A_l (V_l^* x) + V_l (B_l^* x) with m = 2r + 1
    Lanczos vectors (eq. g-func)
  * LREI-AB: rho_{k+1} = rho_k + h sum_l b_l f(rho_{k-l+1}) in factored form (Sec. 3.8).
Shares no code with the GPU path (which uses the projector form of the complement and an
exact block Rayleigh-Ritz eigensolver).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla

from .dense_ei import RK_TABLEAUS, AB_WEIGHTS


def householder_vectors(V):
    """Householder vectors u_1..u_r reducing V to upper-triangular form (Sec. 3.4, eq. Householder-mat).

    Step k reflects the k-th column below row k onto alpha e_k with |alpha| = its norm and the
    phase of alpha opposite to that of the pivot (so that no cancellation occurs in u_k).
    Returns (us, R) with P_r ... P_1 V = [R; 0].
    """
    A = np.array(V, dtype=np.complex128, copy=True)
    N, r = A.shape
    us = []
    for k in range(r):
        x = A[k:, k]
        nx = np.linalg.norm(x)
        phase = x[0] / abs(x[0]) if abs(x[0]) > 0 else 1.0
        alpha = -phase * nx
        u = np.zeros(N, dtype=np.complex128)
        u[k:] = x
        u[k] -= alpha
        uu = np.vdot(u, u).real
        if uu > 0:
            beta = 2.0 / uu
            A = A - beta * np.outer(u, u.conj() @ A)
        us.append(u)
    return us, A[:r, :]


def apply_right(A, us):
    """A Q = A P_1 P_2 ... P_r using A P = A - beta (A u) u^* (Sec. 3.4)."""
    A = np.array(A, dtype=np.complex128, copy=True)
    for u in us:
        uu = np.vdot(u, u).real
        if uu == 0:
            continue
        w = A @ u
        A -= (2.0 / uu) * np.outer(w, u.conj())
    return A


def apply_left(us, B):
    """Q B = P_1 (P_2 (... (P_r B))) using P A = A - beta u (u^* A) (Sec. 3.4)."""
    B = np.array(B, dtype=np.complex128, copy=True)
    for u in reversed(us):
        uu = np.vdot(u, u).real
        if uu == 0:
            continue
        w = u.conj() @ B
        B -= (2.0 / uu) * np.outer(u, w)
    return B


def rhs_factors(V, lam, Hop, kappa, model):
    """Low-rank right-hand side f(rho) = Z V^* + V W^* at rho = V Lambda V^* (Secs. 3.3-3.5, 4).

    Returns (Z, W, G) with G = V^* H V.
    """
    N, r = V.shape
    HV = Hop @ V
    G = V.conj().T @ HV
    li = lam[:, None]
    lj = lam[None, :]
    if model == "qllg":
        D11 = 1j * (li * G - G * lj)
        X11 = D11 / (1.0 - 1j * kappa * li + 1j * kappa * lj)        # E11 + L11 + L11^*
    elif model == "qll":
        X11 = (1j * (li * G - G * lj) - kappa * (li ** 2 * G + G * lj ** 2)
               + 2.0 * kappa * li * G * lj)                          # eq. X-blocks-sol-qLL
    else:
        raise ValueError(model)
    us, _ = householder_vectors(V)
    A = HV.conj().T                                                  # V^* H = (H V)^*
    AVh = apply_right(A, us)[:, r:]                                  # V^* H V^
    if model == "qllg":
        D12 = 1j * lam[:, None] * AVh
        X12 = D12 / (1.0 - 1j * kappa * lam)[:, None]                # E12 + L12
    else:
        X12 = (1j - kappa * lam)[:, None] * (lam[:, None] * AVh)     # (iI - kappa Lambda) Lambda V^* H V^
    W = apply_left(us, np.vstack([np.zeros((r, r), dtype=np.complex128), X12.conj().T]))
    Z = V @ X11 + W
    return Z, W, G


def partial_eig(terms, N, r, tol=1e-14):
    """Top-r eigenpairs of sum_l (A_l V_l^* + V_l B_l^*) by ARPACK on g(x) (eq. g-func), m = 2r + 1.

    Returns (V, mu) sorted by decreasing eigenvalue.
    """
    def g(x):
        x = np.asarray(x).reshape(N, -1)
        y = np.zeros_like(x, dtype=np.complex128)
        for (A, Vl, Bl) in terms:
            y += A @ (Vl.conj().T @ x)
            if Bl is not None:
                y += Vl @ (Bl.conj().T @ x)
        return y

    ncv = 2 * r + 1
    if ncv >= N:
        # too small for ARPACK: apply g to the identity (same operator, dense eigensolve)
        K = g(np.eye(N, dtype=np.complex128))
        K = 0.5 * (K + K.conj().T)
        w, U = np.linalg.eigh(K)
        idx = np.argsort(-w, kind="stable")[:r]
        return U[:, idx], w[idx]
    op = sla.LinearOperator((N, N), matvec=g, matmat=g, dtype=np.complex128)
    v0 = np.ones(N, dtype=np.complex128) / np.sqrt(N)
    w, U = sla.eigsh(op, k=r, which="LA", ncv=ncv, tol=tol, v0=v0, maxiter=100000)
    w = np.real(w)
    idx = np.argsort(-w, kind="stable")
    return U[:, idx], w[idx]


def lrei_rk_step(V1, lam0, Hop, kappa, model, h, scheme="rk4"):
    """One LREI-RK step (Sec. 3.7): stages in factored form, partial eigendecomposition of each.

    Returns (V_next, mu).
    """
    A, b = RK_TABLEAUS[scheme]
    N, r = V1.shape
    Vs, Zs, Ws = [V1], [], []
    Z, W, _ = rhs_factors(V1, lam0, Hop, kappa, model)
    Zs.append(Z); Ws.append(W)

    def factored(coef):
        terms = []
        for l, c in enumerate(coef):
            Al = (V1 * lam0[None, :] if l == 0 else 0.0) + h * c * Zs[l]
            terms.append((Al, Vs[l], h * c * Ws[l] if c != 0 else None))
        return terms

    for j in range(1, len(b)):
        Vj, _ = partial_eig(factored(A[j, :j]), N, r)
        Vs.append(Vj)
        Z, W, _ = rhs_factors(Vj, lam0, Hop, kappa, model)
        Zs.append(Z); Ws.append(W)
    return partial_eig(factored(b), N, r)


def lrei_ab_step(V, lam0, Hop, kappa, model, h, hist, scheme="ab3"):
    """One LREI-AB step (Sec. 3.8).  hist = [(V_{k-1}, Z_{k-1}, W_{k-1}), ...] most recent first.

    Returns (V_next, mu, (V, Z, W)) -- the last item to be prepended to the history.
    """
    b = AB_WEIGHTS[scheme]
    N, r = V.shape
    Z, W, _ = rhs_factors(V, lam0, Hop, kappa, model)
    entries = [(V, Z, W)] + list(hist)
    terms = []
    for l in range(len(b)):
        Vl, Zl, Wl = entries[l]
        Al = (V * lam0[None, :] if l == 0 else 0.0) + h * b[l] * Zl
        terms.append((Al, Vl, h * b[l] * Wl))
    Vn, mu = partial_eig(terms, N, r)
    return Vn, mu, (V, Z, W)


def integrate(V0, lam0, Hop, kappa, model, h, steps, scheme="rk4", callback=None):
    """Run LREI steps; AB schemes start with RK4 steps.  callback(k, V, mu) after each step."""
    V = V0
    if scheme.startswith("rk"):
        for k in range(steps):
            V, mu = lrei_rk_step(V, lam0, Hop, kappa, model, h, scheme)
            if callback:
                callback(k + 1, V, mu)
        return V
    m = len(AB_WEIGHTS[scheme])
    hist = []
    for k in range(steps):
        if k < m - 1:
            Z, W, _ = rhs_factors(V, lam0, Hop, kappa, model)
            hist.insert(0, (V, Z, W))
            V, mu = lrei_rk_step(V, lam0, Hop, kappa, model, h, "rk4")
        else:
            V, mu, e = lrei_ab_step(V, lam0, Hop, kappa, model, h, hist[: m - 1], scheme)
            hist.insert(0, e)
        hist = hist[: m - 1]
        if callback:
            callback(k + 1, V, mu)
    return V


def observables(V, lam0, Hop, Mops):
    """<A> = Tr(Lambda_0 V^* (A V)) (Sec. 3.6, eq. measuerA), plus purity and trace from V^* V."""
    out = {"energy": float(np.real(np.sum(lam0 * np.einsum("bi,bi->i", V.conj(), Hop @ V))))}
    for v in "xyz":
        out["m" + v] = float(np.real(np.sum(lam0 * np.einsum("bi,bi->i", V.conj(), Mops[v] @ V))))
    S = V.conj().T @ V
    LS = lam0[:, None] * S
    out["purity"] = float(np.real(np.trace(LS @ LS)))
    out["trace"] = float(np.real(np.trace(LS)))
    # [rho, H] = V Lambda (H V)^* - (H V) Lambda V^* = B J B^* with B = [V, H V] and
    # J = [[0, Lambda], [-Lambda, 0]]; its Frobenius norm from the 2r x 2r Gram B^* B
    HV = Hop @ V
    Bm = np.hstack([V, HV])
    r = V.shape[1]
    J = np.zeros((2 * r, 2 * r), dtype=np.complex128)
    J[:r, r:] = np.diag(lam0)
    J[r:, :r] = -np.diag(lam0)
    Gb = Bm.conj().T @ Bm
    out["comm_norm"] = float(np.sqrt(max(np.real(np.trace(J @ Gb @ J.conj().T @ Gb)), 0.0)))
    return out
