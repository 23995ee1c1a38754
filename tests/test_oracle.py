"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: textbook
closed forms, the defining equations, conservation laws, exact solutions and
convergence orders.  A plausible slip in the oracle (a sign, a transposed
operand, a wrong bit order, a dropped term) fails at least one of them; the
planted-mistake tests at the end show this for a few.
"""
import json
import os

import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, lowrank as lr, exact

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "spin_closed_forms.json")))


def _bonds(pairs, jxy=1.0, jz=1.0):
    pairs = np.array(pairs, dtype=np.int32).reshape(-1, 2)
    m = pairs.shape[0]
    return li.Bonds(pairs[:, 0].copy(), pairs[:, 1].copy(), np.full(m, jxy), np.full(m, jz))


def _rand_state(n, r, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return li.haar_orthonormal(1 << n, r, rng), li.dirichlet_spectrum(r, rng)


# ---------------------------------------------------------------- Hamiltonian

def test_two_spin_spectrum_matches_textbook():
    g = GOLD["two_spin_bond"]
    H = model.hamiltonian(2, _bonds([(0, 1)], g["J"], g["J"]))
    w = np.sort(np.linalg.eigvalsh(H))
    assert np.allclose(w, sorted([g["singlet"], g["triplet"], g["triplet"], g["triplet"]]), atol=1e-14)


def test_two_spin_xxz_matrix_elements_and_bit_order():
    # |b> with b = 2*s0 + s1 (site 0 = most significant bit), bit 0 = up.
    jxy, jz, bz = 0.7, 1.3, 0.4
    H = model.hamiltonian(2, _bonds([(0, 1)], jxy, jz), (0.0, 0.0, bz))
    assert np.isclose(H[0, 0].real, jz / 2 + bz)      # up up
    assert np.isclose(H[3, 3].real, jz / 2 - bz)      # down down
    assert np.isclose(H[1, 1].real, -jz / 2)
    assert np.isclose(H[2, 2].real, -jz / 2)
    assert np.isclose(H[1, 2].real, jxy) and np.isclose(H[2, 1].real, jxy)
    assert abs(H[0, 3]) == 0 and abs(H[1, 3]) == 0


def test_single_spin_zeeman_and_msb_site():
    g = GOLD["single_spin_zeeman"]
    H = model.hamiltonian(1, _bonds(np.zeros((0, 2))), (0.0, 0.0, g["Bz"]))
    assert np.isclose(H[0, 0].real, g["up"]) and np.isclose(H[1, 1].real, g["down"])
    # site 0 is the MSB: S^z_0 on |100> (index 4, n=3) is -1/2, on |011> (index 3) +1/2
    Sz0 = model.spin_op("z", 0, 3)
    assert np.isclose(Sz0[4, 4].real, -0.5) and np.isclose(Sz0[3, 3].real, 0.5)


def test_heisenberg_ring4_ground_energy():
    g = GOLD["heisenberg_ring_4"]
    # our bond term is 2 J S.S, so E0 = 2 * (-2J)
    H = model.hamiltonian(4, li.chain_bonds(4, periodic=True, J=g["J"]))
    assert np.isclose(np.linalg.eigvalsh(H)[0], 2.0 * g["ground_energy_of_J_sum_SdotS"], atol=1e-12)


def test_hamiltonian_hermitian_and_conserves_total_sz():
    n = 5
    w = li.workload(2, n=n, r=2)
    H = model.hamiltonian(n, w.bonds, w.B)
    Sz = sum(model.spin_op("z", i, n) for i in range(n))
    assert np.abs(H - H.conj().T).max() == 0
    assert np.abs(H @ Sz - Sz @ H).max() < 1e-13


def test_named_states():
    assert li.af1_state(4)[0b0101] == 1 and li.af2_state(4)[0b1010] == 1
    Mz = model.magnetization_op("z", 4)
    up = li.basis_state(4, 0)
    assert np.isclose(np.vdot(up, Mz @ up).real, 0.5)
    assert np.isclose(np.vdot(li.af1_state(4), Mz @ li.af1_state(4)).real, 0.0)
    assert np.isclose(np.linalg.norm(li.w_state(5)), 1) and np.isclose(np.linalg.norm(li.ghz_state(5)), 1)


# ------------------------------------------------------------ right-hand side

@pytest.mark.parametrize("kappa", [0.0, 0.1, 1.0])
def test_qllg_rhs_solves_its_implicit_equation(kappa):
    n, r = 5, 3
    V, lam = _rand_state(n, r, 11)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.3))
    rho = de.state(V, lam)
    f = de.f_qllg(rho, H, kappa)
    res = f - 1j * de.comm(rho, H) - 1j * kappa * de.comm(rho, f)     # eq. q-LLG
    assert np.abs(res).max() < 1e-13


def test_qllg_pure_state_is_rescaled_qll():
    n, kappa = 5, 0.7
    psi = li.haar_orthonormal(1 << n, 1, np.random.Generator(np.random.PCG64(3)))[:, 0]
    rho = np.outer(psi, psi.conj())
    H = model.hamiltonian(n, li.chain_bonds(n, True), (0, 0, 0.5))
    assert np.abs(de.f_qllg(rho, H, kappa) - de.f_qll(rho, H, kappa) / (1 + kappa ** 2)).max() < 1e-13


def test_qll_is_first_order_truncation_of_qllg():
    n, r = 4, 2
    V, lam = _rand_state(n, r, 5)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    rho = de.state(V, lam)
    d = [np.abs(de.f_qllg(rho, H, k) - de.f_qll(rho, H, k)).max() for k in (1e-2, 5e-3)]
    assert 3.5 < d[0] / d[1] < 4.5      # difference is O(kappa^2)


@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_rhs_is_isospectral_and_dissipative(mdl):
    n, r, kappa = 5, 3, 0.4
    V, lam = _rand_state(n, r, 7)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    rho = de.state(V, lam)
    f = de.rhs(rho, H, kappa, mdl)
    assert np.abs(f - f.conj().T).max() < 1e-14
    for m in range(4):       # d/dt Tr rho^{m+1} = (m+1) Tr(rho^m f) = 0  (eq. spectrum_conservation)
        assert abs(np.trace(np.linalg.matrix_power(rho, m) @ f)) < 1e-13
    dE = np.trace(H @ f).real
    C = de.comm(rho, H)
    if mdl == "qll":
        assert np.isclose(dE, -kappa * np.linalg.norm(C) ** 2, rtol=1e-12)
    else:
        assert dE < 0


# ----------------------------------------------------- low-rank vs dense EI

@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_lowrank_rhs_equals_dense(mdl):
    n, r = 6, 3
    w = li.workload(2, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Hs = model.hamiltonian(n, w.bonds, w.B, sparse=True)
    Z, W, G = lr.rhs_factors(w.V, w.lam, Hs, 0.3, mdl)
    f = de.rhs(de.state(w.V, w.lam), H, 0.3, mdl)
    assert np.abs(Z @ w.V.conj().T + w.V @ W.conj().T - f).max() < 1e-13
    # W lies in the complement of V (Sec. 3.5: W = V^ X12^*)
    assert np.abs(w.V.conj().T @ W).max() < 1e-13


def test_householder_reflectors():
    n, r = 5, 4
    V, _ = _rand_state(n, r, 9)
    us, R = lr.householder_vectors(V)
    Q = lr.apply_left(us, np.eye(1 << n))
    assert np.abs(Q.conj().T @ Q - np.eye(1 << n)).max() < 1e-13
    # first r columns of Q span V: Q[:, :r] = V R^{-1} with R upper triangular unitary (diagonal phases)
    assert np.abs(np.triu(R, 1)).max() < 1e-13 and np.allclose(np.abs(np.diag(R)), 1.0)
    assert np.abs(Q[:, :r] @ R - V).max() < 1e-13
    # apply_right agrees with the explicit product
    A = np.random.default_rng(1).standard_normal((3, 1 << n))
    assert np.abs(lr.apply_right(A, us) - A @ Q).max() < 1e-13


@pytest.mark.parametrize("scheme", ["rk1", "rk2", "rk3", "rk4"])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_lrei_rk_equals_ei_rk(scheme, mdl):
    n, r = 6, 3
    w = li.workload(1, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Hs = model.hamiltonian(n, w.bonds, w.B, sparse=True)
    V1, mu1 = de.ei_rk_step(w.V, w.lam, H, 0.2, mdl, 0.02, scheme)
    V2, mu2 = lr.lrei_rk_step(w.V, w.lam, Hs, 0.2, mdl, 0.02, scheme)
    assert np.abs(de.state(V1, w.lam) - de.state(V2, w.lam)).max() < 1e-12
    assert np.abs(mu1 - mu2).max() < 1e-12


@pytest.mark.parametrize("scheme", ["ab2", "ab3", "ab4"])
def test_lrei_ab_equals_ei_ab(scheme):
    n, r, steps = 5, 2, 6
    w = li.workload(2, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Hs = model.hamiltonian(n, w.bonds, w.B, sparse=True)
    Vd, _ = de.integrate(w.V, w.lam, H, 0.1, "qllg", 0.01, steps, scheme)
    Vl = lr.integrate(w.V, w.lam, Hs, 0.1, "qllg", 0.01, steps, scheme)
    assert np.abs(de.state(Vd, w.lam) - de.state(Vl, w.lam)).max() < 1e-11


# -------------------------------------------------------- exact solutions

def _err_vs(exact_rho, V, lam):
    return np.abs(de.state(V, lam) - exact_rho).max()


def test_rank1_closed_form_satisfies_qll():
    n, kappa = 4, 0.5
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    psi0 = li.af1_state(n)
    t, dt = 0.3, 1e-5
    rp = exact.rank1_solution(psi0, H, kappa, t + dt)
    rm = exact.rank1_solution(psi0, H, kappa, t - dt)
    rho = exact.rank1_solution(psi0, H, kappa, t)
    fd = (rp - rm) / (2 * dt)
    assert np.abs(fd - de.f_qll(rho, H, kappa)).max() < 1e-8


def test_printed_rank1_form_is_not_hermitian():
    # The literal e^{-iH~t} rho0 e^{+iH~t} with H~ = (1 - i kappa) H is not Hermitian, so the
    # oracle reads the closed form as psi(t) = exp(-(i + kappa) H t) psi0 / norm instead.
    import scipy.linalg as sla
    n, kappa, t = 4, 0.5, 0.7
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    psi0 = li.af1_state(n)
    Ht = (1 - 1j * kappa) * H
    R = sla.expm(-1j * Ht * t) @ np.outer(psi0, psi0) @ sla.expm(1j * Ht * t)
    R = R / np.trace(R)
    assert np.abs(R - R.conj().T).max() > 1e-2


def _order(errs, hs):
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


@pytest.mark.parametrize("scheme,order", [("rk1", 1), ("rk2", 2), ("rk3", 3), ("rk4", 4)])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_rk_order_on_rank1_exact_solution(scheme, order, mdl):
    n, kappa, T = 4, 0.5, 0.2
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    psi0 = li.af1_state(n)
    ref = exact.rank1_solution(psi0, H, kappa, T, mdl)
    lam = np.array([1.0])
    hs = [0.02, 0.01, 0.005]
    errs = []
    for h in hs:
        V, _ = de.integrate(psi0[:, None], lam, H, kappa, mdl, h, int(round(T / h)), scheme)
        errs.append(_err_vs(ref, V, lam))
    assert abs(_order(errs, hs) - order) < 0.35


@pytest.mark.parametrize("scheme,order", [("ab2", 2), ("ab3", 3), ("ab4", 4)])
def test_ab_order_on_unitary_flow(scheme, order):
    n, T = 4, 0.16
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    V0, lam = _rand_state(n, 2, 21)
    ref = exact.unitary_solution(de.state(V0, lam), H, T)
    hs = [0.01, 0.005, 0.0025]
    errs = []
    for h in hs:
        V, _ = de.integrate(V0, lam, H, 0.0, "qll", h, int(round(T / h)), scheme)
        errs.append(_err_vs(ref, V, lam))
    assert abs(_order(errs, hs) - order) < 0.4


def test_rk4_unitary_limit():
    n, T, h = 5, 0.2, 0.01
    w = li.workload(2, n=n, r=3)
    H = model.hamiltonian(n, w.bonds, w.B)
    ref = exact.unitary_solution(de.state(w.V, w.lam), H, T)
    V, _ = de.integrate(w.V, w.lam, H, 0.0, "qll", h, int(round(T / h)), "rk4")
    assert _err_vs(ref, V, w.lam) < 1e-7


@pytest.mark.parametrize("mdl,kappa", [("qll", 0.0), ("qll", 0.5), ("qllg", 0.5)])
def test_mz_conserved_for_sz_commuting_state(mdl, kappa):
    # [H, S^z_tot] = 0 for XXZ + B_z; a state commuting with S^z_tot keeps <M_z> fixed for any kappa
    n = 5
    w = li.workload(2, n=n, r=2)
    H = model.hamiltonian(n, w.bonds, w.B)
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    V0 = np.stack([li.af2_state(n), li.af1_state(n)], axis=1)
    lam = np.array([0.75, 0.25])
    V, traj = de.integrate(V0, lam, H, kappa, mdl, 0.01, 30, "rk4", Mo)
    mz = [o["mz"] for (_, o, _) in traj]
    assert max(mz) - min(mz) < 1e-13


@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_ei_invariants_and_monotone_energy(mdl):
    n, r = 5, 3
    w = li.workload(1, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    V, traj = de.integrate(w.V, w.lam, H, 0.5, mdl, 0.02, 40, "rk4", Mo)
    E = [o["energy"] for (_, o, _) in traj]
    assert all(E[i + 1] <= E[i] + 1e-12 for i in range(len(E) - 1))
    rho = de.state(V, w.lam)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-15
    ev = np.sort(np.linalg.eigvalsh(rho))[::-1]
    assert np.abs(ev[:r] - w.lam).max() < 1e-13 and np.abs(ev[r:]).max() < 1e-13


def test_qll_initial_dissipation_rate():
    n, r, kappa, h = 4, 2, 0.3, 1e-4
    V, lam = _rand_state(n, r, 31)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    E0 = de.observables(V, lam, H, Mo)["energy"]
    V1, _ = de.ei_rk_step(V, lam, H, kappa, "qll", h)
    E1 = de.observables(V1, lam, H, Mo)["energy"]
    V2, _ = de.ei_rk_step(V, lam, H, kappa, "qll", -h)
    Em = de.observables(V2, lam, H, Mo)["energy"]
    C = de.comm(de.state(V, lam), H)
    assert np.isclose((E1 - Em) / (2 * h), -kappa * np.linalg.norm(C) ** 2, rtol=1e-6)


def test_lowrank_observables_match_dense():
    n, r = 6, 3
    w = li.workload(1, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Hs = model.hamiltonian(n, w.bonds, w.B, sparse=True)
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    a = de.observables(w.V, w.lam, H, Mo)
    b = lr.observables(w.V, w.lam, Hs, Mo)
    for k in a:
        assert abs(a[k] - b[k]) < 1e-13


def test_purity_equals_sum_of_squared_spectrum():
    # Tr(rho^2) = sum_i lambda_i^2 for rho = V diag(lambda) V^* with orthonormal V (Sec. 3.6: the
    # spectrum is conserved, so the purity is a function of Lambda_0 alone); also 1 for a pure state
    n, r = 6, 4
    w = li.workload(1, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    Hs = model.hamiltonian(n, w.bonds, w.B, sparse=True)
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    for obs in (de.observables(w.V, w.lam, H, Mo), lr.observables(w.V, w.lam, Hs, Mo)):
        assert abs(obs["purity"] - np.sum(w.lam ** 2)) < 1e-14
        assert abs(obs["trace"] - 1.0) < 1e-14
    psi = li.af1_state(n)[:, None]
    assert abs(de.observables(psi, np.array([1.0]), H, Mo)["purity"] - 1.0) < 1e-15


def test_commutator_norm_of_pure_state_is_twice_energy_variance():
    # for rho = psi psi^*: ||[rho, H]||_F^2 = 2 (<H^2> - <H>^2); zero for an eigenvector of H
    n = 6
    rng = np.random.default_rng(5)
    H = model.hamiltonian(n, li.chain_bonds(n, True), (0, 0, 0.3))
    Hs = model.hamiltonian(n, li.chain_bonds(n, True), (0, 0, 0.3), sparse=True)
    Mo = {v: model.magnetization_op(v, n) for v in "xyz"}
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    e1 = np.vdot(psi, H @ psi).real
    e2 = np.vdot(H @ psi, H @ psi).real
    lam = np.array([1.0])
    for obs in (de.observables(psi[:, None], lam, H, Mo), lr.observables(psi[:, None], lam, Hs, Mo)):
        assert abs(obs["comm_norm"] ** 2 - 2.0 * (e2 - e1 * e1)) < 1e-12 * e2
    w, U = np.linalg.eigh(H)
    for obs in (de.observables(U[:, [3]], lam, H, Mo), lr.observables(U[:, [3]], lam, Hs, Mo)):
        assert obs["comm_norm"] < 1e-12


def test_planted_purity_and_commutator_mistakes_are_caught():
    # the pins above fail for the plausible slips Tr(rho) in place of Tr(rho^2) and a commutator
    # taken with the wrong sign of one term (rho H + H rho)
    n, r = 5, 3
    w = li.workload(1, n=n, r=r)
    H = model.hamiltonian(n, w.bonds, w.B)
    rho = de.state(w.V, w.lam)
    assert abs(np.trace(rho).real - np.sum(w.lam ** 2)) > 1e-2
    psi = li.af1_state(n) + li.af2_state(n)
    psi /= np.linalg.norm(psi)
    P = np.outer(psi, psi.conj())
    e1 = np.vdot(psi, H @ psi).real
    e2 = np.vdot(H @ psi, H @ psi).real
    assert abs(np.linalg.norm(P @ H + H @ P) ** 2 - 2.0 * (e2 - e1 * e1)) > 1e-2


# ---------------------------------------------- planted mistakes are caught

def test_planted_sign_error_in_qllg_is_caught(monkeypatch):
    orig = de.f_qllg

    def wrong(rho, H, kappa):          # flips the sign of kappa inside the Sylvester denominators
        return orig(rho, H, -kappa)
    n, r, kappa = 4, 2, 0.5
    V, lam = _rand_state(n, r, 2)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    rho = de.state(V, lam)
    f = wrong(rho, H, kappa)
    res = f - 1j * de.comm(rho, H) - 1j * kappa * de.comm(rho, f)
    assert np.abs(res).max() > 1e-3


def test_planted_bit_order_error_is_caught():
    # a Hamiltonian built with site 0 as the LEAST significant bit breaks the MSB pin
    n = 3
    wrong_Sz0 = np.kron(np.kron(np.eye(4), 0.5 * model.SIGMA_Z), np.eye(1))
    assert not np.isclose(wrong_Sz0[4, 4].real, -0.5)


def test_planted_dropped_term_in_qll_is_caught():
    n, r, kappa = 4, 2, 0.4
    V, lam = _rand_state(n, r, 8)
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0, 0, 0.5))
    rho = de.state(V, lam)
    f_wrong = 1j * de.comm(rho, H)          # damping term dropped
    C = de.comm(rho, H)
    assert not np.isclose(np.trace(H @ f_wrong).real, -kappa * np.linalg.norm(C) ** 2, rtol=1e-3)


def test_hamiltonian_row_matches_dense():
    n = 5
    w = li.workload(2, n=n, r=2)
    H = model.hamiltonian(n, w.bonds, w.B)
    for b in (0, 7, 21, 31):
        assert np.abs(model.hamiltonian_row(n, w.bonds, w.B, b) - H[b]).max() == 0


# ------------------------------------------------------- controller network

def test_mlp_gradients_match_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(4)
    p = mlp.init_params(7, 2, rng, hidden=16)
    X = rng.standard_normal((5, 7))
    T = rng.standard_normal((5, 2))
    w = np.array([1.0, 0.3])
    g = mlp.grads(p, X, T, w)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.loss(p, X, T, w)
            flat[idx] = old - eps
            lm = mlp.loss(p, X, T, w)
            flat[idx] = old
            assert abs((lp - lm) / (2 * eps) - g[k].reshape(-1)[idx]) < 1e-8


def test_mlp_linear_limit_and_adam_first_step():
    from oracle import mlp
    rng = np.random.default_rng(5)
    p = mlp.init_params(3, 1, rng, hidden=8)
    # with tiny inputs and zero biases the network is linear: y = W3 W2 W1 x to first order
    X = 1e-6 * rng.standard_normal((4, 3))
    Y, _ = mlp.forward(p, X)
    assert np.allclose(Y, X @ (p["W3"] @ p["W2"] @ p["W1"]).T, rtol=1e-9, atol=1e-18)
    # Adam's first update is -lr * g / (|g| + eps) (bias corrections cancel)
    g = mlp.grads(p, rng.standard_normal((4, 3)), rng.standard_normal((4, 1)))
    q = {k: v.copy() for k, v in p.items()}
    mlp.adam_step(q, g, {}, lr=1e-2)
    for k in p:
        assert np.allclose(q[k] - p[k], -1e-2 * g[k] / (np.abs(g[k]) + 1e-8), atol=1e-15)


# ------------------------------------------- two-spin reduced density matrices (Sec. 3.6)

from oracle import reduced  # noqa: E402


def _pure(psi):
    psi = np.asarray(psi, dtype=np.complex128)
    psi = psi / np.linalg.norm(psi)
    return np.outer(psi, psi.conj()), psi[:, None], np.array([1.0])


def test_bell_and_product_states_textbook_measures():
    rho, _, _ = _pure([1, 0, 0, 1])                      # (|00> + |11>)/sqrt2
    R = reduced.rdm_partial_trace(rho, 2, 0, 1)
    assert np.allclose(R, rho)
    assert abs(reduced.concurrence(R) - 1.0) < 1e-12 and abs(reduced.negativity(R) - 0.5) < 1e-12
    rho, _, _ = _pure(np.kron([1, 1], [1, 2j]))          # a product state
    R = reduced.rdm_partial_trace(rho, 2, 0, 1)
    assert reduced.concurrence(R) < 1e-12 and reduced.negativity(R) < 1e-12


@pytest.mark.parametrize("p", [0.0, 0.2, 1 / 3, 0.5, 0.8, 1.0])
def test_werner_pair_closed_forms(p):
    # p |Psi-><Psi-| + (1 - p) I/4: C = max(0, (3p - 1)/2), N = max(0, (3p - 1)/4)
    psi = np.array([0, 1, -1, 0]) / np.sqrt(2)
    R = p * np.outer(psi, psi) + (1 - p) * np.eye(4) / 4
    assert abs(reduced.concurrence(R) - max(0.0, (3 * p - 1) / 2)) < 1e-12
    assert abs(reduced.negativity(R) - max(0.0, (3 * p - 1) / 4)) < 1e-12


def test_w_and_ghz_pairs():
    w = np.zeros(8); w[[1, 2, 4]] = 1                      # W state of 3 spins
    rho, _, _ = _pure(w)
    for k, l in ((0, 1), (0, 2), (1, 2)):
        R = reduced.rdm_partial_trace(rho, 3, k, l)
        assert abs(reduced.concurrence(R) - 2 / 3) < 1e-12 and reduced.negativity(R) > 0.1
    g = np.zeros(8); g[[0, 7]] = 1                         # GHZ: every pair is a classical mixture
    rho, _, _ = _pure(g)
    R = reduced.rdm_partial_trace(rho, 3, 0, 2)
    assert np.allclose(R, np.diag([0.5, 0, 0, 0.5]))
    assert reduced.concurrence(R) < 1e-12 and reduced.negativity(R) < 1e-12


@pytest.mark.parametrize("k,l", [(0, 5), (2, 3), (4, 1)])
def test_pauli_route_equals_partial_trace_on_low_rank_states(k, l):
    n, r = 6, 3
    rng = np.random.default_rng(11 + k)
    V = np.linalg.qr(rng.standard_normal((1 << n, r)) + 1j * rng.standard_normal((1 << n, r)))[0]
    lam = np.array([0.5, 0.3, 0.2])
    rho = (V * lam) @ V.conj().T
    R1 = reduced.rdm_partial_trace(rho, n, k, l)
    R2 = reduced.rdm_pauli(V, lam, n, k, l)
    assert np.abs(R1 - R2).max() < 1e-13
    assert abs(np.trace(R1) - 1) < 1e-13 and np.allclose(R1, R1.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(R1).min() > -1e-13
    # swapping the sites swaps the factors of the basis
    R3 = reduced.rdm_partial_trace(rho, n, l, k)
    assert np.abs(R3 - R1.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)).max() < 1e-13


def test_planted_dropped_partial_transpose_is_caught(monkeypatch):
    # plant the slip of forgetting the partial transpose in the oracle: the Bell pin fails
    rho, _, _ = _pure([1, 0, 0, 1])
    assert abs(reduced.negativity(rho) - 0.5) < 1e-12

    def negativity_without_transpose(R):
        w = np.linalg.eigvalsh(R)
        return float(-np.sum(w[w < 0]))
    monkeypatch.setattr(reduced, "negativity", negativity_without_transpose)
    assert abs(reduced.negativity(rho) - 0.5) > 0.4


# ------------------------------------------------------ Werner-state initial data (Sec. 5)

from oracle import werner  # noqa: E402



@pytest.mark.parametrize("mdl", ["qll", "qllg"])
@pytest.mark.parametrize("rank", [1, 2])
def test_werner_shift_equals_full_rank_evolution(mdl, rank):
    # the full-rank EI evolution of rho_W equals p I/N + (1 - p) rho_hat(t) with kappa -> (1-p) kappa
    n, p, kappa, h, steps = 4, 0.3, 0.5, 0.01, 12
    N = 1 << n
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0.0, 0.0, 0.5))
    rng = np.random.default_rng(7 + rank)
    if rank == 1:
        ghz = np.zeros(N, dtype=np.complex128); ghz[[0, N - 1]] = 1 / np.sqrt(2)
        V_hat, lam_hat = ghz[:, None], np.array([1.0])
    else:
        V_hat = np.linalg.qr(rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2)))[0]
        lam_hat = np.array([0.7, 0.3])
    rho_W = werner.werner_state(V_hat, lam_hat, p)
    w, U = np.linalg.eigh(rho_W)
    idx = np.argsort(-w, kind="stable")
    V_full, lam_full = U[:, idx], w[idx]
    V_full_t, _ = de.integrate(V_full, lam_full, H, kappa, mdl, h, steps, "rk4")
    rho_full = de.state(V_full_t, lam_full)
    V_hat_t = werner.evolve(V_hat, lam_hat, p, H, kappa, mdl, h, steps)
    rho_shift = werner.werner_state(V_hat_t, lam_hat, p)
    assert np.abs(rho_full - rho_shift).max() < 1e-12
    # and the observable shortcut
    Mz = model.magnetization_op("z", n)
    assert abs(werner.expectation(H, V_hat_t, lam_hat, p) - np.trace(H @ rho_full)) < 1e-12
    assert abs(werner.expectation(Mz, V_hat_t, lam_hat, p) - np.trace(Mz @ rho_full)) < 1e-12


def test_planted_unshifted_kappa_is_caught():
    # evolving rho_hat with the unshifted kappa misses the full-rank evolution
    n, p, kappa, h, steps = 4, 0.3, 0.5, 0.01, 12
    N = 1 << n
    H = model.hamiltonian(n, li.chain_bonds(n, False), (0.0, 0.0, 0.5))
    rng = np.random.default_rng(9)
    V_hat = np.linalg.qr(rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2)))[0]
    lam_hat = np.array([0.7, 0.3])
    rho_W = werner.werner_state(V_hat, lam_hat, p)
    w, U = np.linalg.eigh(rho_W)
    idx = np.argsort(-w, kind="stable")
    V_full_t, _ = de.integrate(U[:, idx], w[idx], H, kappa, "qll", h, steps, "rk4")
    rho_full = de.state(V_full_t, w[idx])
    V_bad, _ = de.integrate(V_hat, lam_hat, H, kappa, "qll", h, steps, "rk4")
    assert np.abs(rho_full - werner.werner_state(V_bad, lam_hat, p)).max() > 1e-6



# ------------------------------------------- Dzyaloshinskii-Moriya term of eq. H1 (NEXT-3)

def test_two_spin_dmi_z_closed_form():
    # 2J S1.S2 + 2D (S1 x S2)_z: triplet |uu>, |dd> at J/2; the Sz = 0 pair couples with
    # amplitude J + iD, so its energies are -J/2 +- sqrt(J^2 + D^2)
    J, D = 1.0, 0.4
    bonds = li.Bonds(np.array([0]), np.array([1]), np.array([J]), np.array([J]))
    H = model.hamiltonian(2, bonds, dmi=[(0.0, 0.0, D)])
    w = np.sort(np.linalg.eigvalsh(H))
    ref = np.sort([J / 2, J / 2, -J / 2 + np.hypot(J, D), -J / 2 - np.hypot(J, D)])
    assert np.abs(w - ref).max() < 1e-13
    assert abs(H[1, 2] - (J + 1j * D)) < 1e-14          # <ud|H|du>: bit 0 = up, site 0 = first factor


def test_dmi_hermitian_antisymmetric_and_sz_conservation():
    n = 4
    bonds = li.chain_bonds(n, True)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((len(bonds), 3))
    H = model.hamiltonian(n, bonds, (0.1, 0.0, 0.5), dmi=d)
    assert np.abs(H - H.conj().T).max() < 1e-14
    # swapping the two sites of every bond flips the sign of its DM term
    H0 = model.hamiltonian(n, bonds)
    swapped = li.Bonds(bonds.site_j, bonds.site_i, bonds.jxy, bonds.jz)
    Hs = model.hamiltonian(n, swapped, dmi=d)
    assert np.abs((Hs - H0) + (model.hamiltonian(n, bonds, dmi=d) - H0)).max() < 1e-13
    # a DM vector along z commutes with total S^z; one along x does not
    Sz = sum(model.spin_op("z", i, n) for i in range(n))
    dz = np.zeros_like(d); dz[:, 2] = d[:, 2]
    Hz = model.hamiltonian(n, bonds, dmi=dz)
    assert np.abs(Hz @ Sz - Sz @ Hz).max() < 1e-13
    dx = np.zeros_like(d); dx[:, 0] = 1.0
    Hx = model.hamiltonian(n, bonds, dmi=dx)
    assert np.abs(Hx @ Sz - Sz @ Hx).max() > 1e-2
    # sparse and dense builds agree
    assert np.abs(model.hamiltonian(n, bonds, (0.1, 0.0, 0.5), sparse=True, dmi=d).toarray() - H).max() < 1e-14
