"""Two-spin reduced density matrices, concurrence and negativity on the GPU (Sec. 3.6).

Against the oracle's partial trace of the dense rho (n <= 8) and, at the benchmark size
(n = 20, r = 16), against its route through 16 Pauli-pair expectation values of the factored
state.  Tolerances: 1e-12 absolute on R entries and 1e-10 on the measures in FP64; 1e-6 and
1e-5 in complex64 bulk (the measures are eigenvalue functions of R, Lipschitz in R up to a
constant of order one).
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, reduced, werner

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei, LreiError  # noqa: E402

TOL_R = {"fp64": 1e-12, "mixed": 1e-6}
TOL_M = {"fp64": 1e-10, "mixed": 1e-5}


def _ctx(n, bonds, B, V, lam, precision="fp64", kappa=0.2, mdl="qll"):
    L = Lrei(n, bonds, B, kappa, mdl, precision, V.shape[1])
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    L.set_state(torch.from_numpy(np.ascontiguousarray(V)).to("cuda", dt), lam)
    return L


def _check(L, rho, n, pairs, precision):
    R, conc, neg = L.two_spin_rdm(pairs)
    for q, (k, l) in enumerate(pairs):
        Rr = reduced.rdm_partial_trace(rho, n, k, l)
        assert np.abs(R[q] - Rr).max() <= TOL_R[precision], (k, l, np.abs(R[q] - Rr).max())
        assert abs(conc[q] - reduced.concurrence(Rr)) <= TOL_M[precision], (k, l)
        assert abs(neg[q] - reduced.negativity(Rr)) <= TOL_M[precision], (k, l)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_all_pairs_of_a_random_state_after_steps(precision):
    w = li.workload(2, n=7, r=3)
    H = model.hamiltonian(w.n, w.bonds, w.B)
    L = _ctx(w.n, w.bonds, w.B, w.V, w.lam, precision, kappa=0.3)
    pairs = [(k, l) for k in range(w.n) for l in range(w.n) if k != l]
    _check(L, de.state(w.V, w.lam), w.n, pairs, precision)
    L.step(0.01, "rk4", 5)
    V, _ = de.integrate(w.V, w.lam, H, 0.3, "qll", 0.01, 5, "rk4")
    _check(L, de.state(V, w.lam), w.n, pairs, precision)


def test_named_entangled_states():
    # W: every pair has concurrence 2/n; GHZ: every pair is separable (C = N = 0); a singlet on
    # sites (1, 2) times up spins: C = 1, N = 1/2 for that pair, 0 for the others
    n = 5
    bonds, B = li.chain_bonds(n, False), (0.0, 0.0, 0.5)
    single = np.array([1.0])
    for psi, expect in ((li.w_state(n), 2.0 / n), (li.ghz_state(n), 0.0)):
        L = _ctx(n, bonds, B, psi[:, None], single)
        _, conc, neg = L.two_spin_rdm([(0, 1), (1, 3), (4, 2)])
        assert np.allclose(conc, expect, atol=1e-12)
        _check(L, np.outer(psi, psi.conj()), n, [(0, 1), (1, 3), (4, 2)], "fp64")
    up, dn = np.array([1.0, 0.0]), np.array([0.0, 1.0])
    singlet = (np.kron(up, dn) - np.kron(dn, up)) / np.sqrt(2)
    psi = np.kron(np.kron(up, singlet), np.kron(up, up))
    L = _ctx(n, bonds, B, psi[:, None], single)
    _, conc, neg = L.two_spin_rdm([(1, 2), (2, 1), (0, 1), (3, 4)])
    assert np.allclose(conc, [1, 1, 0, 0], atol=1e-12) and np.allclose(neg, [0.5, 0.5, 0, 0], atol=1e-12)


def test_werner_weight_mixes_in_the_identity():
    w = li.workload(2, n=6, r=2)
    L = _ctx(w.n, w.bonds, w.B, w.V, w.lam)
    L.set_werner(0.4)
    rho = werner.werner_state(w.V, w.lam, 0.4)
    _check(L, rho, w.n, [(0, 3), (5, 1), (2, 3)], "fp64")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_benchmark_size_against_pauli_expectations(precision):
    w = li.workload(3)           # n = 20, r = 16
    L = _ctx(w.n, w.bonds, w.B, w.V, w.lam, precision, kappa=w.kappa)
    L.step(w.dt, "rk4", 2)
    V, lam, _ = L.get_state()
    V = V.cpu().numpy().astype(np.complex128)
    # the state is the factor's Cholesky orthonormalisation
    Rc = np.linalg.cholesky(V.conj().T @ V).conj().T
    V = V @ np.linalg.inv(Rc)
    pairs = [(0, 1), (9, 10), (3, 17)]
    R, conc, neg = L.two_spin_rdm(pairs)
    for q, (k, l) in enumerate(pairs):
        Rr = reduced.rdm_pauli(V, lam, w.n, k, l)
        assert np.abs(R[q] - Rr).max() <= 10 * TOL_R[precision]
        assert abs(conc[q] - reduced.concurrence(Rr)) <= TOL_M[precision]
        assert abs(neg[q] - reduced.negativity(Rr)) <= TOL_M[precision]


def test_rejects_bad_pairs():
    w = li.workload(2, n=5, r=2)
    L = _ctx(w.n, w.bonds, w.B, w.V, w.lam)
    for pairs in ([(1, 1)], [(0, 5)], [(-1, 2)]):
        with pytest.raises(LreiError) as e:
            L.two_spin_rdm(pairs)
        assert e.value.code == -1
