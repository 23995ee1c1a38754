"""The per-step JSON-lines metrics harness on a small GPU run."""
import json

import numpy as np
import pytest

import lrei_inputs as li

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei  # noqa: E402
from paper_2508_21200_gb300.metrics import run_logged  # noqa: E402


def test_run_logged_writes_one_line_per_interval(tmp_path):
    w = li.workload(1, n=8, r=4)
    L = Lrei(w.n, w.bonds, w.B, w.kappa, w.model, "fp64", w.r)
    L.set_state(torch.from_numpy(w.V).cuda(), w.lam)
    path = tmp_path / "m.jsonl"
    recs = run_logged(L, w.dt, 7, str(path), every=3)
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert lines == recs and [r["step"] for r in lines] == [0, 3, 6, 7]
    assert np.allclose([r["t"] for r in lines], [0.0, 0.03, 0.06, 0.07], atol=1e-14)
    for r in lines:
        assert abs(r["trace"] - 1.0) < 1e-12 and r["orth_err"] < 1e-12 and r["rank"] == 4
        assert 0.0 <= r["ritz_drift"] < 1e-2
    # launches since the previous record: three steps launch more kernels than one
    assert lines[1]["kernel_launches"] > lines[3]["kernel_launches"] > 0
    # dissipation: the energy does not increase (kappa > 0)
    E = [r["energy"] for r in lines]
    assert all(b <= a + 1e-12 for a, b in zip(E, E[1:]))
