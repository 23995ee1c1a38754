"""Adaptive step control (plain rule and learned network) on the GPU, checked against the oracle.

Reference solutions come from the dense EI-RK4 oracle with a step 8x smaller than any step
the controllers take, so its own error is negligible at the tested tolerances.
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei, Mlp, NFEAT  # noqa: E402
from paper_2508_21200_gb300 import controller as ctl  # noqa: E402


def _reference(w, t_end, h=0.00125):
    H = model.hamiltonian(w.n, w.bonds, w.B)
    M = {v: model.magnetization_op(v, w.n) for v in "xyz"}
    steps = int(round(t_end / h))
    V, _ = de.integrate(w.V, w.lam, H, w.kappa, w.model, t_end / steps, steps, "rk4")
    return de.observables(V, w.lam, H, M)


def _err(o, ref):
    return max(abs(o[k] - ref[k]) for k in ("energy", "mx", "my", "mz"))


def _run(w, t_end, tol, controller, judge_every=8, net=None):
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, "fp64", w.r)
    L.set_state(torch.from_numpy(w.V).cuda(), w.lam)
    L.controller_config(judge_every=judge_every, record=False, h0=0.01)
    if net is not None:
        L.controller_attach(net)
    L.step_adaptive(t_end, tol, controller)
    o = L.observables()
    st = L.controller_stats()
    return o, st


def test_plain_controller_reaches_t_end_and_controls_error():
    w = li.workload(1, n=8, r=4)
    t_end = 0.4
    ref = _reference(w, t_end)
    errs = {}
    for tol in (1e-6, 1e-9):
        o, st = _run(w, t_end, tol, 0)
        assert abs(o["t"] - t_end) < 1e-12
        assert st["accepted"] > 0 and st["judged"] > 0
        errs[tol] = _err(o, ref)
    assert errs[1e-9] < 1e-7
    assert errs[1e-9] <= errs[1e-6] + 1e-12


def test_learned_controller_with_untrained_network_stays_safe():
    # a random network proposes poor steps; the plain judge must keep the error controlled
    w = li.workload(1, n=7, r=3)
    t_end = 0.3
    ref = _reference(w, t_end)
    net = Mlp(NFEAT, 1, ctl.init_params(NFEAT, 1, seed=3))
    o, st = _run(w, t_end, 1e-9, 1, net=net)
    assert abs(o["t"] - t_end) < 1e-12
    assert _err(o, ref) < 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tolerance_below_rounding_floor_terminates(precision):
    # a tolerance below what the stored factor can resolve is raised to the precision's floor
    # (1e-13 FP64, 1e-6 complex64) instead of shrinking the step without end
    w = li.workload(1, n=7, r=3)
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, precision, w.r)
    dt = torch.complex128 if precision == "fp64" else torch.complex64
    L.set_state(torch.from_numpy(w.V).to("cuda", dt), w.lam)
    L.controller_config(judge_every=1, record=False, h0=0.01)
    L.step_adaptive(0.05, 1e-16, 0)
    st = L.controller_stats()
    assert abs(L.observables()["t"] - 0.05) < 1e-12
    assert st["accepted"] >= 1 and st["rejected"] < 64


def test_records_have_features_and_judged_errors():
    w = li.workload(1, n=7, r=3)
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, "fp64", w.r)
    L.set_state(torch.from_numpy(w.V).cuda(), w.lam)
    L.controller_config(judge_every=1, record=True, h0=0.01)
    L.step_adaptive(0.1, 1e-8, 0)
    rows = L.controller_records()
    assert rows.shape[1] == NFEAT + 4 and rows.shape[0] >= L.controller_stats()["accepted"]
    assert np.all(rows[:, NFEAT + 2] >= 0)              # judged every step
    assert np.all(np.isfinite(rows))


def test_trained_network_gain_over_plain_rule():
    """Train on plain-controller data (n = 8..10), evaluate on a held-out chain (n = 9, other seed)
    over t in [0, 1].

    The gain is reported as RK4 steps (including judge and rejected steps) per unit simulated
    time, plain / learned, at the same tolerance; the learned run must also keep the error bound.
    """
    train_w = [li.workload(4, t, n=n, r=4, kappa=0.1) for t, n in ((1, 8), (2, 9), (3, 10))]
    X, Y = ctl.generate(train_w, t_end=0.2, tols=(1e-6, 1e-7))
    net, loss = ctl.fit(X, Y, iters=2000, lr=2e-3)
    assert loss < 0.5 * float(np.var(Y)) + 1e-6      # better than the mean (loss = half the mean square)
    w = li.workload(4, 9, n=9, r=4, kappa=0.1)
    t_end, tol = 1.0, 1e-8
    ref = _reference(w, t_end, h=0.005)
    o_p, st_p = _run(w, t_end, tol, 0, judge_every=8)
    o_l, st_l = _run(w, t_end, tol, 1, judge_every=8, net=net)
    assert _err(o_l, ref) < 1e-6 and _err(o_p, ref) < 1e-6
    gain = st_p["rk4_steps"] / st_l["rk4_steps"]
    print(f"learned controller: {st_l}  plain: {st_p}  gain {gain:.3f}")
    assert gain > 1.0
