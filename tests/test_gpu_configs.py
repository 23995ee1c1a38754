"""The stated workloads run at their stated sizes on the GPU (through the C ABI).

Workload 2 (periodic anisotropic chain n=16, r=8, B_z=1, h=0.005, 500 steps) over its whole
matrix: kappa in {0.01, 0.1, 1} x {q-LL, q-LLG} x {RK4, AB3}, complex128 against complex64
bulk, the FP64 path against the paper-literal low-rank CPU oracle at the same size, and the
same recipe at n=9 against the dense EI oracle.  Workload 3 (n=20, r=16) for its stated 100
steps, complex64 bulk against FP64.  Tolerances as in test_gpu_parity: relative observable
error 1e-10 (FP64) and 1e-6 (complex64 bulk), Ritz values relative to lambda0_max.
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de, lowrank as lr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 1e-6}
KAPPAS = [0.01, 0.1, 1.0]
MODELS = ["qll", "qllg"]
SCHEMES = ["rk4", "ab3"]


def scales(w):
    sE = float(np.sum(np.abs(w.bonds.jxy) + np.abs(w.bonds.jz) / 2) + w.n * np.linalg.norm(w.B) / 2)
    return {"energy": sE, "mx": 0.5, "my": 0.5, "mz": 0.5, "purity": 1.0, "trace": 1.0}


def obs_err(o, ref, w):
    s = scales(w)
    return max(abs(o[k] - ref[k]) / max(abs(ref[k]), s[k]) for k in s)


def ctx(w, precision, kappa, mdl):
    L = Lrei(w.n, w.bonds, w.B, kappa, mdl, precision, w.r)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    L.set_state(torch.from_numpy(w.V).to("cuda", dt), w.lam)
    return L


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("mdl", MODELS)
@pytest.mark.parametrize("kappa", KAPPAS)
def test_config2_complex64_bulk_vs_complex128_500_steps(kappa, mdl, scheme):
    w = li.workload(2)
    Ld, Lm = ctx(w, "fp64", kappa, mdl), ctx(w, "mixed", kappa, mdl)
    worst, worst_mu = 0.0, 0.0
    for _ in range(w.steps // 100):
        Ld.step(w.dt, scheme, 100)
        Lm.step(w.dt, scheme, 100)
        od, om = Ld.observables(), Lm.observables()
        worst = max(worst, obs_err(om, od, w))
        worst_mu = max(worst_mu, float(np.abs(om["ritz"] - od["ritz"]).max() / w.lam.max()))
        assert abs(od["trace"] - 1.0) < 1e-12 and od["orth_err"] < 1e-12
        # the complex64 context's Lambda_0 is the spectrum of its own (rounded) initial state
        assert np.abs(od["lambda0"] - om["lambda0"]).max() <= TOL["mixed"] * w.lam.max()
    assert worst <= TOL["mixed"], worst
    assert worst_mu <= TOL["mixed"], worst_mu


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("mdl", MODELS)
@pytest.mark.parametrize("kappa", KAPPAS)
def test_config2_fp64_vs_lowrank_oracle_at_full_size(kappa, mdl, scheme):
    # n=16 against the paper-literal low-rank CPU version (Householder complement, ARPACK on g):
    # RK4 for two steps; AB3 for three (its two RK4 start-up steps and one AB3 step)
    w = li.workload(2)
    steps = 2 if scheme == "rk4" else 3
    Hs = model.hamiltonian(w.n, w.bonds, w.B, sparse=True)
    M = {v: model.magnetization_op(v, w.n, sparse=True) for v in "xyz"}
    mus = []
    V = lr.integrate(w.V, w.lam, Hs, kappa, mdl, w.dt, steps, scheme, callback=lambda k, V, mu: mus.append(mu))
    L = ctx(w, "fp64", kappa, mdl)
    L.step(w.dt, scheme, steps)
    o = L.observables()
    assert obs_err(o, lr.observables(V, w.lam, Hs, M), w) <= TOL["fp64"]
    assert np.abs(o["ritz"] - mus[-1]).max() <= TOL["fp64"] * w.lam.max()


_DENSE = {}


def _dense_reference(w, kappa, mdl, scheme, steps, every):
    key = (kappa, mdl, scheme, steps, every)
    if key not in _DENSE:
        H = model.hamiltonian(w.n, w.bonds, w.B)
        M = {v: model.magnetization_op(v, w.n) for v in "xyz"}
        _, traj = de.integrate(w.V, w.lam, H, kappa, mdl, w.dt, steps, scheme, Mops=M, every=every)
        _DENSE[key] = traj
    return _DENSE[key]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("mdl", MODELS)
@pytest.mark.parametrize("kappa", KAPPAS)
def test_config2_recipe_at_n9_vs_dense_oracle(kappa, mdl, scheme, precision):
    w = li.workload(2, n=9)          # same recipe (periodic, anisotropic, r=8, B_z=1, h=0.005)
    steps, every = 40, 10
    traj = _dense_reference(w, kappa, mdl, scheme, steps, every)
    L = ctx(w, precision, kappa, mdl)
    worst, worst_mu = 0.0, 0.0
    for k, ref, mu in traj:
        L.step(w.dt, scheme, every)
        o = L.observables()
        worst = max(worst, obs_err(o, ref, w))
        worst_mu = max(worst_mu, float(np.abs(o["ritz"] - mu).max() / w.lam.max()))
        if precision == "fp64":
            assert abs(o["comm_norm"] - ref["comm_norm"]) <= TOL["fp64"] * max(ref["comm_norm"], 1.0)
    assert worst <= TOL[precision], worst
    assert worst_mu <= TOL[precision], worst_mu


def test_config3_mixed_vs_fp64_for_100_steps():
    # the benchmarked workload (n=20, r=16, q-LL, kappa=0.1, RK4, h=0.01) for its stated 100 steps
    w = li.workload(3)
    Lm, Ld = ctx(w, "mixed", w.kappa, w.model), ctx(w, "fp64", w.kappa, w.model)
    E_prev = Ld.observables()["energy"]
    worst, worst_mu = 0.0, 0.0
    for _ in range(w.steps // 25):
        Lm.step(w.dt, "rk4", 25)
        Ld.step(w.dt, "rk4", 25)
        om, od = Lm.observables(), Ld.observables()
        worst = max(worst, obs_err(om, od, w))
        worst_mu = max(worst_mu, float(np.abs(om["ritz"] - od["ritz"]).max() / w.lam.max()))
        assert od["energy"] <= E_prev + 1e-12          # dissipation, kappa > 0
        E_prev = od["energy"]
        assert abs(od["trace"] - 1.0) < 1e-12 and od["orth_err"] < 1e-12 and om["orth_err"] < 1e-5
        assert abs(od["purity"] - np.sum(w.lam ** 2)) < 1e-12
    assert worst <= TOL["mixed"], worst
    assert worst_mu <= TOL["mixed"], worst_mu
