"""Two-spin reduced density matrices and entanglement measures (oracle; test infrastructure only).

Paper: Sec. 3.6 (measurement of a two-spin reduced density matrix R_kl, the partial trace of
rho(t) over every spin but k and l, and entanglement measures computed from the 4 x 4 matrix:
concurrence, Wootters 1998; negativity, Vidal and Werner 2002).  The paper evaluates the 16
entries of R_kl as expectation values Tr(A rho) of sparse operators; `rdm_pauli` follows that
route (A = sigma_a on site k times sigma_b on site l, R = 1/4 sum_ab <A_ab> sigma_a x sigma_b),
`rdm_partial_trace` is the plain definition (a tensor partial trace of the dense rho), and the
tests pin one against the other.  Basis of R: |s_k s_l> with s = 0 for spin up, site k the
first factor, as in `model` (site i is Kronecker factor i from the left).
"""
from __future__ import annotations

import numpy as np

from . import model

_I2 = np.eye(2, dtype=np.complex128)
_PAULI4 = [_I2, model.SIGMA_X, model.SIGMA_Y, model.SIGMA_Z]


def rdm_partial_trace(rho, n: int, k: int, l: int):
    """R_kl = Tr over all sites but k, l of the dense N x N rho (the definition, Sec. 3.6)."""
    if k == l:
        raise ValueError("two distinct sites")
    t = np.asarray(rho).reshape((2,) * (2 * n))
    keep = [k, l]
    rest = [i for i in range(n) if i not in keep]
    # move kept row axes, kept column axes first; trace the rest pairwise
    order = keep + rest + [n + k, n + l] + [n + i for i in rest]
    t = np.transpose(t, order)
    m = len(rest)
    t = t.reshape(4, 1 << m, 4, 1 << m)
    return np.einsum("ajbj->ab", t)


def _site_pauli(a: int, site: int, n: int):
    """sigma_a on Kronecker factor `site` (a = 0 identity, 1 x, 2 y, 3 z), sparse."""
    import scipy.sparse as sp
    left = sp.identity(1 << site, dtype=np.complex128, format="csr")
    right = sp.identity(1 << (n - site - 1), dtype=np.complex128, format="csr")
    return sp.kron(sp.kron(left, sp.csr_matrix(_PAULI4[a])), right, format="csr")


def rdm_pauli(V, lam, n: int, k: int, l: int):
    """R_kl from 16 expectation values Tr(A rho) = Tr(Lambda V^*(A V)) of the factored state
    rho = V diag(lam) V^* (the paper's route, Sec. 3.6 eq. measuerA)."""
    V = np.asarray(V, dtype=np.complex128)
    lam = np.asarray(lam, dtype=np.float64)
    R = np.zeros((4, 4), dtype=np.complex128)
    for a in range(4):
        Pa = _site_pauli(a, k, n)
        for b in range(4):
            A = Pa @ _site_pauli(b, l, n)
            ev = np.sum(lam * np.einsum("ij,ij->j", V.conj(), A @ V))
            R += ev * np.kron(_PAULI4[a], _PAULI4[b])
    return R / 4.0


def concurrence(R) -> float:
    """Wootters' concurrence of a two-qubit state: C = max(0, l1 - l2 - l3 - l4) with l_i the
    decreasing square roots of the eigenvalues of R (Y x Y) conj(R) (Y x Y)."""
    YY = np.kron(model.SIGMA_Y, model.SIGMA_Y)
    Rt = YY @ np.conj(R) @ YY
    ev = np.linalg.eigvals(R @ Rt)
    s = np.sort(np.sqrt(np.clip(ev.real, 0.0, None)))[::-1]
    return float(max(0.0, s[0] - s[1] - s[2] - s[3]))


def negativity(R) -> float:
    """N = (||R^{T_B}||_1 - 1) / 2: the summed magnitudes of the negative eigenvalues of the
    partial transpose on the second spin (Vidal and Werner 2002)."""
    T = np.asarray(R).reshape(2, 2, 2, 2).transpose(0, 3, 2, 1).reshape(4, 4)
    w = np.linalg.eigvalsh(0.5 * (T + T.conj().T))
    return float(-np.sum(w[w < 0]))
