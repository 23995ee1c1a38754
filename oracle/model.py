"""Dense spin operators and the spin Hamiltonian (oracle; test infrastructure only).

Paper: Sec. 3.6 eq. spin_op (S_i^v as a Kronecker product with sigma_v/2 in
factor i) and Sec. 5 eq. H1 (exchange + Zeeman Hamiltonian).  hbar = 1.

Readings used here (where the paper leaves a choice open):
  * the exchange sum of eq. H1 runs once over each listed bond (i, j); an
    XXZ bond carries 2*Jxy*(S^x S^x + S^y S^y) + 2*Jz*S^z S^z, which for
    Jxy = Jz = J is the paper's 2J S_i . S_j;
  * the Zeeman term is B . sum_i S_i with B the field in energy units
    (B = g mu_B b of eq. H1 with hbar = 1; the sign of -mu b . S with
    mu = -mu_B g / hbar is +g mu_B b . S);
  * site i is Kronecker factor i from the left, so site 0 is the most
    significant bit of the basis index; bit 0 means spin up.

The matrices are built from Kronecker products on purpose: this is a
different mechanism from the GPU kernels' bit arithmetic, so agreement also
pins the bit order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"x": SIGMA_X, "y": SIGMA_Y, "z": SIGMA_Z}


def spin_op(v: str, i: int, n: int, sparse: bool = False):
    """S_i^v = I x ... x (1/2) sigma_v x ... x I with sigma_v in Kronecker factor i (eq. spin_op)."""
    op = 0.5 * PAULI[v]
    if sparse:
        left = sp.identity(1 << i, dtype=np.complex128, format="csr")
        right = sp.identity(1 << (n - i - 1), dtype=np.complex128, format="csr")
        return sp.kron(sp.kron(left, sp.csr_matrix(op)), right, format="csr")
    return np.kron(np.kron(np.eye(1 << i), op), np.eye(1 << (n - i - 1)))


def magnetization_op(v: str, n: int, sparse: bool = False):
    """M_v = (1/n) sum_i S_i^v (Sec. 3.6)."""
    M = None
    for i in range(n):
        t = spin_op(v, i, n, sparse)
        M = t if M is None else M + t
    return M / n


def hamiltonian(n: int, bonds, B=(0.0, 0.0, 0.0), sparse: bool = False, dmi=None):
    """Spin Hamiltonian of eq. H1: sum over bonds of the XXZ exchange, the Dzyaloshinskii-Moriya
    term 2 d_ij . (S_i x S_j) when `dmi` (one 3-vector per bond) is given, plus B . sum_i S_i."""
    N = 1 << n
    H = sp.csr_matrix((N, N), dtype=np.complex128) if sparse else np.zeros((N, N), dtype=np.complex128)
    for b in range(len(bonds)):
        i, j = int(bonds.site_i[b]), int(bonds.site_j[b])
        jxy, jz = float(bonds.jxy[b]), float(bonds.jz[b])
        for v, c in (("x", jxy), ("y", jxy), ("z", jz)):
            if c != 0.0:
                H = H + 2.0 * c * (spin_op(v, i, n, sparse) @ spin_op(v, j, n, sparse))
        if dmi is not None:
            d = np.asarray(dmi[b], dtype=np.float64)
            # (S_i x S_j)_x = S_i^y S_j^z - S_i^z S_j^y, and cyclically
            for c, (u, w) in zip(d, (("y", "z"), ("z", "x"), ("x", "y"))):
                if c != 0.0:
                    H = H + 2.0 * c * (spin_op(u, i, n, sparse) @ spin_op(w, j, n, sparse)
                                       - spin_op(w, i, n, sparse) @ spin_op(u, j, n, sparse))
    for v, c in zip("xyz", B):
        if c != 0.0:
            for i in range(n):
                H = H + c * spin_op(v, i, n, sparse)
    return H


def expectation(A, rho) -> float:
    """<A> = Tr(A rho) (Sec. 3.6)."""
    return float(np.real(np.trace(A @ rho)))


def hamiltonian_row(n: int, bonds, B, b: int) -> np.ndarray:
    """Row b of the Hamiltonian of eq. H1, as a dense length-2^n vector.

    Row b of a Kronecker product is the Kronecker product of the factors' rows
    (row bit of factor i = bit n-1-i of b), so each term's row is built from
    2-vectors.  Used to check single output rows at sizes where H cannot be formed.
    """
    bits = [(b >> (n - 1 - i)) & 1 for i in range(n)]
    N = 1 << n
    row = np.zeros(N, dtype=np.complex128)

    def term_row(ops):
        v = np.ones(1, dtype=np.complex128)
        for i in range(n):
            f = ops.get(i)
            v = np.kron(v, (f[bits[i], :] if f is not None else np.eye(2)[bits[i], :]))
        return v

    for k in range(len(bonds)):
        i, j = int(bonds.site_i[k]), int(bonds.site_j[k])
        for v_, c in (("x", float(bonds.jxy[k])), ("y", float(bonds.jxy[k])), ("z", float(bonds.jz[k]))):
            if c != 0.0:
                row += 2.0 * c * term_row({i: 0.5 * PAULI[v_], j: 0.5 * PAULI[v_]})
    for v_, c in zip("xyz", B):
        if c != 0.0:
            for i in range(n):
                row += c * term_row({i: 0.5 * PAULI[v_]})
    return row
