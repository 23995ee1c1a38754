"""The workload recipes under configs/ and the inputs drawn from them."""
import numpy as np
import pytest

import lrei_inputs as li


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5])
def test_recipe_fields(c):
    cfg = li.load_config(c)
    assert cfg["name"] == f"cfg{c}" and cfg["lattice"]["kind"] == "chain"
    for k in ("B", "model", "scheme", "dt", "steps"):
        assert k in cfg
    w = li.workload(c, with_state=False)
    assert w.dt == cfg["dt"] and w.steps == cfg["steps"] and w.model == cfg["model"] and w.B == tuple(cfg["B"])
    if "n" in cfg["lattice"]:
        assert w.n == cfg["lattice"]["n"] and w.r == cfg["r"] and w.kappa == cfg["kappa"]
    else:
        lo, hi = cfg["lattice"]["n_range"]
        assert lo <= w.n <= hi and cfg["r_range"][0] <= w.r <= cfg["r_range"][1]
        assert 10 ** cfg["kappa_log10_range"][0] <= w.kappa <= 10 ** cfg["kappa_log10_range"][1]


def test_workload_2_anisotropy_and_periodic_bonds():
    cfg = li.load_config(2)
    w = li.workload(2, with_state=False)
    assert len(w.bonds) == w.n and w.bonds.site_j[-1] == 0          # periodic: n bonds, the last wraps
    d = w.bonds.jz - w.bonds.jxy
    lo, hi = cfg["lattice"]["jz_aniso"]
    assert np.all(d >= lo) and np.all(d <= hi) and np.ptp(d) > 0


def test_workload_4_draws_differ_per_trajectory_and_repeat_per_seed():
    a, b = li.workload(4, 3, with_state=False), li.workload(4, 4, with_state=False)
    c = li.workload(4, 3, with_state=False)
    assert (a.n, a.r, a.kappa) == (c.n, c.r, c.kappa) and (a.n, a.r, a.kappa) != (b.n, b.r, b.kappa)
