"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative observable error |o - o_ref| / max(|o_ref|, s_o) <= 1e-10
for the FP64 path and <= 1e-6 for the mixed (complex64 bulk) path, with
s_M = 1/2 for magnetisations, s_E = sum_bonds(|Jxy| + |Jz|/2) + n|B|/2 for the
energy, 1 for purity and trace, and lambda0_max for Ritz values.
Element-wise kernel checks (H.V, the right-hand side) use 1e-13 (FP64) and
2e-6 (FP32) relative to the largest entry.
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, lowrank as lr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei, LreiError  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 1e-6}


def ctx_for(w, precision="fp64", kappa=None, model_=None, r_max=None):
    return Lrei(w.n, w.bonds, w.B, w.kappa if kappa is None else kappa, model_ or w.model, precision,
                r_max or max(w.r, 1))


def dev(V, precision="fp64"):
    return torch.from_numpy(np.ascontiguousarray(V)).to("cuda", torch.complex128 if precision == "fp64" else torch.complex64)


def scales(w):
    sE = float(np.sum(np.abs(w.bonds.jxy) + np.abs(w.bonds.jz) / 2) + w.n * np.linalg.norm(w.B) / 2)
    return {"energy": sE, "mx": 0.5, "my": 0.5, "mz": 0.5, "purity": 1.0, "trace": 1.0}


def obs_err(o, ref, w):
    s = scales(w)
    return max(abs(o[k] - ref[k]) / max(abs(ref[k]), s[k]) for k in s)


def dense_ops(w):
    H = model.hamiltonian(w.n, w.bonds, w.B)
    M = {v: model.magnetization_op(v, w.n) for v in "xyz"}
    return H, M


def gpu_rho(L):
    V, lam, _ = L.get_state()
    V = V.cpu().numpy().astype(np.complex128)
    # the stored factor is orthonormal to working precision; use its orthonormalisation
    R = np.linalg.cholesky(V.conj().T @ V).conj().T
    V = V @ np.linalg.inv(R)
    return de.state(V, lam), V, lam


# ------------------------------------------------------------------ H.V

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,r,cfg", [(3, 1, 1), (6, 3, 2), (9, 4, 1), (9, 16, 2), (10, 5, 2),
                                     # n >= 10: more than one 1024-row tile, bonds astride and above
                                     # the tiles, a periodic wrap (cfg 2)
                                     (10, 4, 2), (11, 8, 2), (12, 16, 1), (12, 8, 2), (13, 4, 2)])
def test_apply_h_matches_dense(precision, n, r, cfg):
    w = li.workload(cfg, n=n, r=r)
    L = ctx_for(w, precision, r_max=r)
    V = dev(w.V, precision)
    Y = torch.empty_like(V)
    L.apply_h(V, Y)
    H = model.hamiltonian(n, w.bonds, w.B, sparse=n > 10)
    ref = H @ V.cpu().numpy().astype(np.complex128)
    err = np.abs(Y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if precision == "fp64" else 2e-6), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_h_full_size_sampled_rows(precision):
    n, r = 20, 16
    w = li.workload(3, with_state=False)
    g = torch.Generator(device="cuda").manual_seed(7)
    V = torch.randn((1 << n, r), dtype=torch.complex128 if precision == "fp64" else torch.complex64, device="cuda",
                    generator=g)
    L = ctx_for(w, precision, r_max=r)
    Y = torch.empty_like(V)
    L.apply_h(V, Y)
    torch.cuda.synchronize()
    Vh = V.cpu().numpy().astype(np.complex128)
    Yh = Y.cpu().numpy()
    rows = [0, 1, 0b01010101010101010101, (1 << n) - 1, 123457, 777777, 1 << 19]
    for b in rows:
        ref = model.hamiltonian_row(n, w.bonds, w.B, b) @ Vh
        err = np.abs(Yh[b] - ref).max() / max(np.abs(ref).max(), 1e-30)
        assert err < (1e-13 if precision == "fp64" else 2e-6), (b, err)


# ------------------------------------------------------------- rhs (Z, W)

@pytest.mark.parametrize("mdl", ["qll", "qllg"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rhs_matches_dense_definition(mdl, precision):
    w = li.workload(2, n=6, r=3)
    L = ctx_for(w, precision, kappa=0.3, model_=mdl)
    L.set_state(dev(w.V, precision), w.lam)
    Z, W, G = L.rhs(0)
    rho, V, lam = gpu_rho(L)
    Zh, Wh = Z.cpu().numpy().astype(np.complex128), W.cpu().numpy().astype(np.complex128)
    Vs = L.get_state()[0].cpu().numpy().astype(np.complex128)
    f_gpu = Zh @ Vs.conj().T + Vs @ Wh.conj().T
    H, _ = dense_ops(w)
    f_ref = de.rhs(de.state(w.V, w.lam), H, 0.3, mdl)
    err = np.abs(f_gpu - f_ref).max() / np.abs(f_ref).max()
    assert err < (1e-12 if precision == "fp64" else 5e-6), err
    # G = V^* H V is Hermitian with trace-weighted energy Tr(Lambda G)
    assert abs(np.sum(lam * np.real(np.diag(G))) - np.real(np.trace(H @ de.state(w.V, w.lam)))) < (
        1e-12 if precision == "fp64" else 1e-5)


# ---------------------------------------------------------------- RK steps

@pytest.mark.parametrize("scheme", ["rk1", "rk2", "rk3", "rk4"])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_one_rk_step_matches_dense_ei(scheme, mdl):
    w = li.workload(1, n=6, r=3)
    H, _ = dense_ops(w)
    L = ctx_for(w, "fp64", kappa=0.4, model_=mdl)
    L.set_state(dev(w.V), w.lam)
    L.step(0.02, scheme, 1)
    Vd, mud = de.ei_rk_step(w.V, w.lam, H, 0.4, mdl, 0.02, scheme)
    rho, _, _ = gpu_rho(L)
    assert np.abs(rho - de.state(Vd, w.lam)).max() < 1e-12
    o = L.observables()
    assert np.abs(o["ritz"] - mud).max() < 1e-12 * w.lam.max()
    assert np.allclose(o["lambda0"], w.lam, atol=1e-14)


def _trajectory_check(w, precision, steps, every, scheme="rk4", kappa=None, mdl=None):
    kappa = w.kappa if kappa is None else kappa
    mdl = mdl or w.model
    H, M = dense_ops(w)
    L = ctx_for(w, precision, kappa=kappa, model_=mdl)
    L.set_state(dev(w.V, precision), w.lam)
    V = w.V
    hist = []
    worst, worst_mu = 0.0, 0.0
    m = {"ab2": 2, "ab3": 3, "ab4": 4}.get(scheme, 1)
    done = 0
    while done < steps:
        for _ in range(every):
            if scheme.startswith("rk"):
                V, mu = de.ei_rk_step(V, w.lam, H, kappa, mdl, w.dt, scheme)
            else:
                if done < m - 1:
                    hist.insert(0, de.rhs(de.state(V, w.lam), H, kappa, mdl))
                    V, mu = de.ei_rk_step(V, w.lam, H, kappa, mdl, w.dt, "rk4")
                else:
                    V, mu, Fk = de.ei_ab_step(V, w.lam, H, kappa, mdl, w.dt, hist[: m - 1], scheme)
                    hist.insert(0, Fk)
                hist = hist[: m - 1]
            done += 1
        L.step(w.dt, scheme, every)
        o = L.observables()
        ref = de.observables(V, w.lam, H, M)
        worst = max(worst, obs_err(o, ref, w))
        worst_mu = max(worst_mu, np.abs(o["ritz"] - mu).max() / w.lam.max())
    return worst, worst_mu


def test_config1_fp64_1000_steps_vs_dense_oracle():
    w = li.workload(1)       # open chain n=8, r=4, q-LL, kappa=0.1, RK4, dt=0.01, 1000 steps
    err, err_mu = _trajectory_check(w, "fp64", w.steps, 100)
    assert err <= TOL["fp64"], err
    assert err_mu <= TOL["fp64"], err_mu


def test_config1_mixed_vs_dense_oracle():
    w = li.workload(1)
    err, err_mu = _trajectory_check(w, "mixed", 300, 100)
    assert err <= TOL["mixed"], err
    assert err_mu <= TOL["mixed"], err_mu


@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_config2_shape_small_fp64(mdl):
    # periodic anisotropic chain (workload 2 recipe) shrunk to n=8 for the dense oracle
    w = li.workload(2, n=8, r=8)
    err, err_mu = _trajectory_check(w, "fp64", 60, 20, kappa=0.1, mdl=mdl)
    assert err <= TOL["fp64"] and err_mu <= TOL["fp64"], (err, err_mu)


@pytest.mark.parametrize("n,r", [(1, 1), (2, 1), (3, 2), (4, 4), (5, 3)])
def test_tiny_and_ragged_sizes(n, r):
    # N < tile rows (one ragged tile) and Krylov spaces wider than N (rank-deficient blocks)
    w = li.workload(1, n=n, r=r)
    err, err_mu = _trajectory_check(w, "fp64", 10, 5, kappa=0.3)
    assert err <= TOL["fp64"] and err_mu <= TOL["fp64"], (err, err_mu)


def test_pure_state_af1():
    n = 6
    w = li.workload(1, n=n, r=1, with_state=False)
    w.V = li.af1_state(n)[:, None]
    w.lam = np.array([1.0])
    err, err_mu = _trajectory_check(w, "fp64", 20, 10, kappa=0.5, mdl="qllg")
    assert err <= TOL["fp64"] and err_mu <= TOL["fp64"], (err, err_mu)


def test_eigenstate_is_stationary():
    # all spins up is an eigenstate of XXZ + B_z: the Krylov space is invariant (block breakdown)
    n = 6
    w = li.workload(1, n=n, r=1, with_state=False)
    V0 = li.basis_state(n, 0)[:, None]
    L = ctx_for(w, "fp64", kappa=0.3, r_max=1)
    L.set_state(dev(V0), np.array([1.0]))
    L.step(0.01, "rk4", 5)
    rho, _, _ = gpu_rho(L)
    assert np.abs(rho - np.outer(V0, V0.conj())).max() < 1e-13


def test_mixture_of_sz_eigenstates_keeps_mz():
    n = 6
    w = li.workload(2, n=n, r=2, with_state=False)
    V0 = np.stack([li.af2_state(n), li.af1_state(n)], axis=1)
    L = ctx_for(w, "fp64", kappa=0.5, model_="qllg", r_max=2)
    L.set_state(dev(V0), np.array([0.75, 0.25]))
    mz0 = L.observables()["mz"]
    L.step(0.01, "rk4", 30)
    assert abs(L.observables()["mz"] - mz0) < 1e-12


# -------------------------------------------------------------- error paths

def test_error_codes():
    w = li.workload(1, n=5, r=2)
    L = ctx_for(w, "fp64")
    with pytest.raises(LreiError) as e:
        L.step(0.01, "rk4", 1)
    assert e.value.code == -9                      # step before set_state
    with pytest.raises(LreiError) as e:
        L.set_state(dev(w.V), np.array([0.7, 0.2]))
    assert e.value.code == -4                      # trace != 1
    with pytest.raises(LreiError) as e:
        L.set_state(dev(w.V), np.array([1.2, -0.2]))
    assert e.value.code == -4                      # negative weight
    bad = w.V.copy()
    bad[3, 1] = np.nan
    with pytest.raises(LreiError) as e:
        L.set_state(dev(bad), w.lam)
    assert e.value.code == -3                      # non-finite input
    dup = np.stack([w.V[:, 0], w.V[:, 0]], axis=1)
    with pytest.raises(LreiError) as e:
        L.set_state(dev(dup), np.array([0.5, 0.5]))
    assert e.value.code == -5                      # rank-deficient V
    with pytest.raises(LreiError) as e:
        Lrei(w.n, w.bonds, (0.2, float("inf"), 0.5), 0.1, "qll", "fp64", 2)
    assert e.value.code == -3                      # non-finite field
    with pytest.raises(LreiError) as e:
        L.set_dmi(np.zeros(len(w.bonds) + 1))
    assert e.value.code == -1                      # one DM vector per bond
    with pytest.raises(LreiError) as e:
        Lrei(w.n, w.bonds, w.B, 0.1, "qll", "bf16x", 2)
    assert e.value.code == -2                      # the BF16-split precision is declared, not built


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rank_rule_drops_trailing_weight_and_bounds_the_change(precision):
    # rank rule of the plain controller: trailing weights of total w <= tol_r are dropped and the
    # rest renormalised; observables move by at most 2 w ||A||; the truncated state then evolves
    # like the dense oracle started from the truncated, renormalised state
    w = li.workload(2, n=8, r=6)
    lam = np.array([0.5, 0.3, 0.199, 5e-4, 3e-4, 2e-4])
    H, M = dense_ops(w)
    L = ctx_for(w, precision)
    L.set_state(dev(w.V, precision), lam)
    o_full = L.observables()
    k, wdrop = L.truncate_rank(1.05e-3)
    # a complex64 context holds the spectrum of its rounded initial state (within ~1e-8)
    tol_lam = 1e-15 if precision == "fp64" else 1e-7
    assert k == 3 and abs(wdrop - 1e-3) < tol_lam
    o = L.observables()
    lam3 = lam[:3] / (1.0 - wdrop)
    assert np.allclose(o["lambda0"], lam3, rtol=0, atol=tol_lam)
    normH = np.abs(np.linalg.eigvalsh(H)).max()
    assert abs(o["energy"] - o_full["energy"]) <= 2 * wdrop * normH + 1e-9
    for v in "xyz":
        assert abs(o["m" + v] - o_full["m" + v]) <= 2 * wdrop * 0.5 + 1e-9
    L.step(w.dt, "rk4", 10)
    V3, _ = de.integrate(w.V[:, :3], lam3, H, w.kappa, w.model, w.dt, 10, "rk4")
    assert obs_err(L.observables(), de.observables(V3, lam3, H, M), w) <= TOL[precision]
    assert L.truncate_rank(0.0) == (3, 0.0)                  # nothing below a zero tolerance


# ------------------------------------------------------ full-size properties

def test_full_size_mixed_vs_fp64_and_invariants():
    # n=20, r=16 (the benchmarked workload): mixed vs FP64 GPU and the method's invariants
    w = li.workload(3)
    Lm = ctx_for(w, "mixed")
    Ld = ctx_for(w, "fp64")
    Lm.set_state(dev(w.V, "mixed"), w.lam)
    Ld.set_state(dev(w.V), w.lam)
    o0 = Ld.observables()
    for _ in range(3):
        Lm.step(w.dt, "rk4", 1)
        Ld.step(w.dt, "rk4", 1)
    om, od = Lm.observables(), Ld.observables()
    s = scales(w)
    for k in s:
        assert abs(om[k] - od[k]) / max(abs(od[k]), s[k]) <= TOL["mixed"], (k, om[k], od[k])
    assert od["orth_err"] < 1e-12 and om["orth_err"] < 1e-5
    assert abs(od["trace"] - 1) < 1e-12
    assert od["energy"] <= o0["energy"] + 1e-12              # dissipation (kappa > 0)
    assert np.abs(od["ritz"] - w.lam).max() < 1e-6 * w.lam.max()


@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_config2_n16_fp64_vs_lowrank_oracle(mdl):
    # workload 2 at full size (n=16, r=8, periodic anisotropic chain) against the paper-literal
    # low-rank CPU version (Householder complement + ARPACK on g), two RK4 steps
    w = li.workload(2)
    Hs = model.hamiltonian(w.n, w.bonds, w.B, sparse=True)
    M = {v: model.magnetization_op(v, w.n, sparse=True) for v in "xyz"}
    L = ctx_for(w, "fp64", kappa=0.1, model_=mdl)
    L.set_state(dev(w.V), w.lam)
    V = w.V
    for _ in range(2):
        V, mu = lr.lrei_rk_step(V, w.lam, Hs, 0.1, mdl, w.dt, "rk4")
    L.step(w.dt, "rk4", 2)
    o = L.observables()
    ref = lr.observables(V, w.lam, Hs, M)
    assert obs_err(o, ref, w) <= TOL["fp64"]
    assert np.abs(o["ritz"] - mu).max() <= TOL["fp64"] * w.lam.max()


# ------------------------------------------------------------ Adams-Bashforth

@pytest.mark.parametrize("scheme", ["ab2", "ab3", "ab4"])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_ab_matches_dense_ei(scheme, mdl):
    # AB_m with an RK4 start-up (m-1 steps), periodic anisotropic chain, history kept across calls
    w = li.workload(2, n=7, r=3)
    err, err_mu = _trajectory_check(w, "fp64", 40, 8, scheme=scheme, kappa=0.1, mdl=mdl)
    assert err <= TOL["fp64"] and err_mu <= TOL["fp64"], (err, err_mu)


@pytest.mark.parametrize("scheme", ["ab2", "ab3", "ab4"])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
@pytest.mark.parametrize("dt", [0.005, 0.01])
def test_ab_mixed_matches_dense_ei(scheme, mdl, dt):
    # complex64 history blocks: nearly dependent (consecutive states differ by O(h)), orthonormalised
    # through measured Grams of the written residuals; checked after every step
    w = li.workload(2, n=8, r=4)
    w.dt = dt
    err, err_mu = _trajectory_check(w, "mixed", 60, 1, scheme=scheme, kappa=0.1, mdl=mdl)
    assert err <= TOL["mixed"] and err_mu <= TOL["mixed"], (err, err_mu)


def test_ab_history_resets_on_dt_change():
    w = li.workload(1, n=6, r=2)
    H, M = dense_ops(w)
    L = ctx_for(w, "fp64")
    L.set_state(dev(w.V), w.lam)
    L.step(0.01, "ab3", 4)
    L.step(0.02, "ab3", 3)     # new dt: history restarts with RK4 steps
    V, _ = de.integrate(w.V, w.lam, H, w.kappa, w.model, 0.01, 4, "ab3")
    V, _ = de.integrate(V, w.lam, H, w.kappa, w.model, 0.02, 3, "ab3")
    o, ref = L.observables(), de.observables(V, w.lam, H, M)
    assert obs_err(o, ref, w) <= TOL["fp64"]


# ------------------------------------------------------- Householder route

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_householder_compact_wy_factors(precision):
    # Q = I - U T U^H is unitary, Q[:, :r] = V diag(D) and Q^H V = [diag(D)^{-1}; 0] (Sec. 3.4)
    w = li.workload(2, n=6, r=4)
    L = ctx_for(w, precision)
    L.set_state(dev(w.V, precision), w.lam)
    U, T, D = L.householder()
    U = U.cpu().numpy().astype(np.complex128)
    V = L.get_state()[0].cpu().numpy().astype(np.complex128)
    N = 1 << w.n
    Q = np.eye(N) - U @ T @ U.conj().T
    tol = 1e-13 if precision == "fp64" else 3e-6
    assert np.abs(Q.conj().T @ Q - np.eye(N)).max() < tol
    assert np.abs(Q[:, :w.r] - V * D[None, :]).max() < tol
    # the top block of U is the unit lower-triangular LU factor (to rounding: U is formed as
    # ([I; 0] - V D) R^{-1}, so the entries above the diagonal are rounding residue)
    assert np.abs(np.triu(U[:w.r], 1)).max() < tol and np.allclose(np.diag(U[:w.r]), 1, atol=tol)
    assert np.abs(np.tril(T, -1)).max() < tol


@pytest.mark.parametrize("mdl", ["qll", "qllg"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_householder_route_equals_projector_and_oracle(mdl, precision):
    w = li.workload(2, n=7, r=3)
    L = ctx_for(w, precision, kappa=0.4, model_=mdl)
    L.set_state(dev(w.V, precision), w.lam)
    Z0, W0, G0 = L.rhs(0)
    Z1, W1, G1 = L.rhs(1)
    tol = 1e-12 if precision == "fp64" else 5e-6
    sc = np.abs(W0.cpu().numpy()).max()
    assert np.abs((W1 - W0).cpu().numpy()).max() < tol * sc
    assert np.abs((Z1 - Z0).cpu().numpy()).max() < tol * sc
    # against the paper-literal CPU version (Householder vectors applied column by column)
    Vs = L.get_state()[0].cpu().numpy().astype(np.complex128)
    Hs = model.hamiltonian(w.n, w.bonds, w.B, sparse=True)
    _, lam, _ = L.get_state()
    Zr, Wr, _ = lr.rhs_factors(Vs, lam, Hs, 0.4, mdl)
    assert np.abs(W1.cpu().numpy() - Wr).max() < tol * sc
    assert np.abs(Z1.cpu().numpy() - Zr).max() < tol * sc


# ------------------------------------------------------- tall-skinny Gram entry point

@pytest.mark.parametrize("precision,m", [("fp64", 1), ("fp64", 5), ("mixed", 3), ("mixed", 5)])
def test_gram_entry_point_matches_numpy(precision, m):
    # P = [B_0..B_{m-1}]^* B_{m-1} over N = 2048 rows (32 tiles of 64 rows, more CTAs than tiles)
    w = li.workload(2, n=11, r=8)
    L = ctx_for(w, precision)
    L.set_state(dev(w.V, precision), w.lam)
    rng = np.random.default_rng(5)
    B = [rng.standard_normal((1 << w.n, w.r)) + 1j * rng.standard_normal((1 << w.n, w.r)) for _ in range(m)]
    Bd = [dev(b, precision) for b in B]
    P = L.gram(Bd).cpu().numpy()
    Bh = [b.cpu().numpy().astype(np.complex128) for b in Bd]     # the values the kernel read
    ref = np.concatenate(Bh, axis=1).conj().T @ Bh[-1]
    tol = 1e-13 if precision == "fp64" else 2e-6
    assert np.abs(P - ref).max() <= tol * np.abs(ref).max()


# ------------------------------------------------------ checkpoint / resume

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["rk4", "ab3"])
def test_checkpoint_resume_is_bitwise(precision, scheme):
    # a context restored from a checkpoint continues bit for bit like the one that saved it
    w = li.workload(2, n=11, r=8)
    La = ctx_for(w, precision)
    La.set_state(dev(w.V, precision), w.lam)
    La.step(w.dt, scheme, 6)
    blob = La.checkpoint()
    La.step(w.dt, scheme, 5)
    Va, lam_a, ta = La.get_state()
    oa = La.observables()
    Lb = ctx_for(w, precision)
    Lb.restore(blob)
    Lb.step(w.dt, scheme, 5)
    Vb, lam_b, tb = Lb.get_state()
    ob = Lb.observables()
    assert torch.equal(Va, Vb)
    assert np.array_equal(lam_a, lam_b) and ta == tb
    for k in ("energy", "mx", "my", "mz", "purity", "trace", "comm_norm"):
        assert oa[k] == ob[k], k
    assert np.array_equal(oa["ritz"], ob["ritz"])
    # a context of another precision refuses the blob
    other = ctx_for(w, "mixed" if precision == "fp64" else "fp64")
    with pytest.raises(LreiError):
        other.restore(blob)


def test_eigensolver_sweep_limit_reports_no_convergence():
    # failure detection without a device fault: one FP64 Jacobi sweep cannot diagonalise the
    # r x r Rayleigh-Ritz matrix of a random state, so the step reports LREI_ERR_EIG_NOCONV
    w = li.workload(2, n=8, r=6)
    L = ctx_for(w, "fp64")
    L.set_state(dev(w.V), w.lam)
    L.set_eig_sweeps(1)
    with pytest.raises(LreiError) as e:
        L.step(w.dt, "rk4", 1)
    assert e.value.code == -6
    L.set_state(dev(w.V), w.lam)
    L.set_eig_sweeps(30)
    L.step(w.dt, "rk4", 1)                       # the context stays usable
    with pytest.raises(LreiError):
        L.set_eig_sweeps(0)


def test_eigensolver_counters_count_one_solve_per_stage():
    # each RK4 stage diagonalises its stage matrix once: one FP32 Jacobi (all k eigenpairs) and one
    # FP64 Jacobi (the r x r Rayleigh-Ritz), each taking at least one sweep
    from paper_2508_21200_gb300 import eig_counters
    w = li.workload(2, n=8, r=4)
    L = ctx_for(w, "mixed")
    L.set_state(dev(w.V, "mixed"), w.lam)
    L.step(w.dt, "rk4", 1)            # the graph is built and run once
    a = eig_counters()
    L.step(w.dt, "rk4", 3)
    b = eig_counters()
    d = {k: b[k] - a[k] for k in a}
    assert d["fp32_calls"] == 12 and d["fp64_calls"] == 12, d
    assert d["fp32_sweeps"] >= 12 and d["fp64_sweeps"] >= 12, d
