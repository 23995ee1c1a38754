"""Werner-state initial data through the library (Sec. 5, eq. werner-sol).

CPU: the binding's map from the low-rank part's observables to those of
rho_W = p I/N + (1 - p) rho_hat, against the dense rho_W of the oracle.
GPU: a context created with kappa -> (1 - p) kappa, stepped from rho_hat_0, reproduces the
oracle's full-rank evolution of rho_W.
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, werner


def test_werner_observable_map_of_the_binding():
    # the binding's host-side map from rho_hat's observables to rho_W's, against dense rho_W
    from paper_2508_21200_gb300 import werner as pw
    n, p = 5, 0.25
    N = 1 << n
    H = model.hamiltonian(n, li.chain_bonds(n, True), (0.0, 0.0, 0.7))
    M = {v: model.magnetization_op(v, n) for v in "xyz"}
    rng = np.random.default_rng(3)
    V = np.linalg.qr(rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3)))[0]
    lam = np.array([0.5, 0.3, 0.2])
    o_hat = de.observables(V, lam, H, M)
    rho_hat = de.state(V, lam)
    o_hat["comm_norm"] = np.linalg.norm(rho_hat @ H - H @ rho_hat)
    o_hat["lambda0"] = lam
    got = pw.observables(o_hat, p, n)
    rho = werner.werner_state(V, lam, p)
    want = {"energy": np.trace(H @ rho).real, "purity": np.trace(rho @ rho).real, "trace": np.trace(rho).real,
            "comm_norm": np.linalg.norm(rho @ H - H @ rho)}
    want.update({"m" + v: np.trace(M[v] @ rho).real for v in "xyz"})
    for k, v in want.items():
        assert abs(got[k] - v) < 1e-13, k
    assert np.allclose(np.sort(got["lambda0"]), np.sort(np.linalg.eigvalsh(rho))[-3:], atol=1e-13)
    assert pw.shifted_kappa(0.4, 0.25) == pytest.approx(0.3)
    with pytest.raises(ValueError):
        pw.shifted_kappa(0.4, 1.0)



@pytest.mark.gpu
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
def test_werner_evolution_on_gpu_matches_full_rank_oracle(mdl):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("needs a CUDA GPU")
    from paper_2508_21200_gb300 import Lrei
    from paper_2508_21200_gb300 import werner as pw
    n, p, kappa, h, steps = 6, 0.3, 0.5, 0.01, 10
    N = 1 << n
    bonds, B = li.chain_bonds(n, False), (0.0, 0.0, 0.5)
    H = model.hamiltonian(n, bonds, B)
    M = {v: model.magnetization_op(v, n) for v in "xyz"}
    rng = np.random.default_rng(21)
    V_hat = np.linalg.qr(rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2)))[0]
    lam_hat = np.array([0.7, 0.3])
    # oracle: the full-rank EI evolution of rho_W itself
    w, U = np.linalg.eigh(werner.werner_state(V_hat, lam_hat, p))
    idx = np.argsort(-w, kind="stable")
    Vt, _ = de.integrate(U[:, idx], w[idx], H, kappa, mdl, h, steps, "rk4")
    ref = de.observables(Vt, w[idx], H, M)
    # library: the low-rank part with the shifted damping
    L = Lrei(n, bonds, B, pw.shifted_kappa(kappa, p), mdl, "fp64", 2)
    L.set_state(torch.from_numpy(V_hat).cuda(), lam_hat)
    L.step(h, "rk4", steps)
    got = pw.observables(L.observables(), p, n)
    for k in ("energy", "mx", "my", "mz", "purity", "trace"):
        assert abs(got[k] - ref[k]) <= 1e-10 * max(abs(ref[k]), 0.5), (k, got[k], ref[k])
