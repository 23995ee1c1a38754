"""Werner-state initial data through the C ABI (Sec. 5, eq. werner-sol).

lrei_set_werner(p) makes the library evolve rho = p I/N + (1 - p) rho_hat: the steps use the
damping (1 - p) kappa on the stored low-rank rho_hat, and lrei_observables reports the
observables of rho itself.  The GPU test compares that with the oracle's full-rank EI
evolution of rho_W, which knows nothing of the shift.
"""
import ctypes

import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, werner


def test_set_werner_rejects_weights_outside_the_unit_interval():
    # argument checks happen before any device work (a NULL context is rejected first)
    from paper_2508_21200_gb300 import build
    try:
        path = build.ensure_built()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc in this environment
        pytest.skip(f"cannot build: {e}")
    lib = ctypes.CDLL(path)
    lib.lrei_set_werner.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.lrei_set_werner(None, 0.2) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("mdl,p", [("qll", 0.3), ("qllg", 0.3), ("qll", 0.0), ("qllg", 0.8)])
def test_werner_evolution_on_gpu_matches_full_rank_oracle(mdl, p):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("needs a CUDA GPU")
    from paper_2508_21200_gb300 import Lrei, LreiError
    n, kappa, h, steps = 6, 0.5, 0.01, 10
    N = 1 << n
    bonds, B = li.chain_bonds(n, False), (0.0, 0.0, 0.5)
    H = model.hamiltonian(n, bonds, B)
    M = {v: model.magnetization_op(v, n) for v in "xyz"}
    rng = np.random.default_rng(21)
    V_hat = np.linalg.qr(rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2)))[0]
    lam_hat = np.array([0.7, 0.3])
    # oracle: the full-rank EI evolution of rho_W itself
    rho_w = werner.werner_state(V_hat, lam_hat, p)
    w, U = np.linalg.eigh(rho_w)
    idx = np.argsort(-w, kind="stable")
    Vt, _ = de.integrate(U[:, idx], w[idx], H, kappa, mdl, h, steps, "rk4")
    ref = de.observables(Vt, w[idx], H, M)
    rho_t = de.state(Vt, w[idx])
    # library: the low-rank part, Werner weight set through the ABI
    L = Lrei(n, bonds, B, kappa, mdl, "fp64", 2)
    L.set_state(torch.from_numpy(V_hat).cuda(), lam_hat)
    L.set_werner(p)
    L.step(h, "rk4", steps)
    got = L.observables()
    for k in ("energy", "mx", "my", "mz", "purity", "trace", "comm_norm"):
        assert abs(got[k] - ref[k]) <= 1e-10 * max(abs(ref[k]), 0.5), (k, got[k], ref[k])
    top = np.sort(np.linalg.eigvalsh(rho_t))[::-1][:2]
    assert np.abs(np.sort(got["lambda0"])[::-1] - top).max() < 1e-10
    with pytest.raises(LreiError):
        L.set_werner(1.0)
