"""Many trajectories in one launch (BASELINE workload 4 recipe, shrunk): a batch steps every
trajectory exactly as the trajectory steps alone (bit for bit: the same kernels in the same
order, reductions in a fixed order), and against the dense oracle where it is small enough.
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Batch, Lrei, LreiError  # noqa: E402


def _trajectories(count, precision):
    out = []
    for t in range(count):
        rng = li.rng_for(4, 1000 + t)
        n = int(rng.integers(6, 12))
        r = int(rng.integers(2, 9))
        kappa = float(10.0 ** rng.uniform(-3.0, 0.0))
        w = li.workload(4, 1000 + t, n=n, r=r, kappa=kappa)
        mdl = "qll" if t % 3 else "qllg"
        L = Lrei(w.n, w.bonds, w.B, w.kappa, mdl, precision, w.r)
        dt = torch.complex128 if precision == "fp64" else torch.complex64
        L.set_state(torch.from_numpy(w.V).to("cuda", dt), w.lam)
        out.append((w, mdl, L))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_trajectories_stepped_alone(precision):
    A = _trajectories(12, precision)
    B = _trajectories(12, precision)
    batch = Batch([L for _, _, L in A])
    batch.step(0.01, 7)
    for (w, mdl, La), (_, _, Lb) in zip(A, B):
        Lb.step(0.01, "rk4", 7)
        Va, _, ta = La.get_state()
        Vb, _, tb = Lb.get_state()
        assert torch.equal(Va, Vb) and abs(ta - tb) < 1e-15
        oa, ob = La.observables(), Lb.observables()
        assert oa["energy"] == ob["energy"] and np.array_equal(oa["ritz"], ob["ritz"])
    batch.close()


def test_batch_against_dense_oracle_and_autotuner():
    A = _trajectories(6, "fp64")
    batch = Batch([L for _, _, L in A])
    share, ms = batch.autotune(0.01, steps=1)
    assert share >= 1 and ms > 0
    for w, _, L in A:       # the autotuner advanced the trajectories: start over
        L.set_state(torch.from_numpy(w.V).cuda(), w.lam)
    batch.step(0.01, 5)
    for w, mdl, L in A:
        H = model.hamiltonian(w.n, w.bonds, w.B)
        M = {v: model.magnetization_op(v, w.n) for v in "xyz"}
        V, _ = de.integrate(w.V, w.lam, H, w.kappa, mdl, 0.01, 5, "rk4")
        ref = de.observables(V, w.lam, H, M)
        o = L.observables()
        sE = float(np.sum(np.abs(w.bonds.jxy) + np.abs(w.bonds.jz) / 2) + w.n * np.linalg.norm(w.B) / 2)
        for k, s in (("energy", sE), ("mx", 0.5), ("my", 0.5), ("mz", 0.5), ("purity", 1.0)):
            assert abs(o[k] - ref[k]) <= 1e-10 * max(abs(ref[k]), s), (k, w.n, w.r)
        assert abs(o["t"] - 0.05) < 1e-12


def test_batch_rejects_contexts_without_state():
    w = li.workload(1, n=6, r=2)
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, "fp64", w.r)
    with pytest.raises(LreiError) as e:
        Batch([L])
    assert e.value.code == -9
