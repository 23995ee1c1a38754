"""The full Hamiltonian of eq. H1 on the GPU: Dzyaloshinskii-Moriya vectors along z and a
transverse field, on chains and triangular lattices (Sec. 5), against the oracle's dense H.

The paper's example in its units: J = 1 meV, DMI 0.4 meV along z, b = 1 T along x, which is
B_x = g mu_B b = 0.116 meV with g = 2.  Tolerances as in test_gpu_parity (1e-13 / 2e-6 of the
largest entry for H.V; relative observable error 1e-10 / 1e-6 for trajectories).
"""
import numpy as np
import pytest

import lrei_inputs as li
from oracle import model, dense_ei as de

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2508_21200_gb300 import Lrei  # noqa: E402

B_PAPER = (0.116, 0.0, 0.0)
D_PAPER = 0.4


def _dense_h(n, bonds, B, dz):
    return model.hamiltonian(n, bonds, B, dmi=[(0.0, 0.0, d) for d in dz], sparse=n > 10)


def _dev(V, precision):
    return torch.from_numpy(np.ascontiguousarray(V)).to("cuda", torch.complex128 if precision == "fp64" else torch.complex64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n,r,B,periodic", [(5, 2, (0.3, -0.2, 0.5), True), (8, 4, B_PAPER, False),
                                             (10, 16, (0.1, 0.3, 1.0), True), (11, 8, B_PAPER, True),
                                             (12, 16, (0.0, 0.4, 0.0), False), (3, 1, (0.2, 0.1, 0.3), True)])
def test_apply_h_with_dmi_and_transverse_field(precision, n, r, B, periodic):
    rng = np.random.default_rng(n * 100 + r)
    bonds = li.chain_bonds(n, periodic)
    dz = rng.uniform(-0.5, 0.5, len(bonds))
    L = Lrei(n, bonds, B, 0.1, "qll", precision, r)
    L.set_dmi(dz)
    V = (rng.standard_normal((1 << n, r)) + 1j * rng.standard_normal((1 << n, r))) / np.sqrt(2)
    Vd = _dev(V, precision)
    Y = torch.empty_like(Vd)
    L.apply_h(Vd, Y)
    ref = _dense_h(n, bonds, B, dz) @ Vd.cpu().numpy().astype(np.complex128)
    err = np.abs(Y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if precision == "fp64" else 2e-6), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_triangular_lattice_apply_h(precision):
    # 3 x 4 periodic triangular lattice: 36 bonds over 12 sites, bit pairs far apart
    bonds = li.triangular_bonds(3, 4, True)
    n, r = 12, 16
    rng = np.random.default_rng(9)
    dz = np.full(len(bonds), D_PAPER)
    L = Lrei(n, bonds, B_PAPER, 0.5, "qllg", precision, r)
    L.set_dmi(dz)
    V = (rng.standard_normal((1 << n, r)) + 1j * rng.standard_normal((1 << n, r))) / np.sqrt(2)
    Vd = _dev(V, precision)
    Y = torch.empty_like(Vd)
    L.apply_h(Vd, Y)
    ref = _dense_h(n, bonds, B_PAPER, dz) @ Vd.cpu().numpy().astype(np.complex128)
    err = np.abs(Y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if precision == "fp64" else 2e-6), err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mdl", ["qll", "qllg"])
@pytest.mark.parametrize("scheme", ["rk4", "ab3"])
def test_trajectory_on_the_paper_hamiltonian(precision, mdl, scheme):
    # 2 x 3 periodic triangular lattice (n = 6) with the paper's DMI and transverse field, kappa = 0.5
    bonds = li.triangular_bonds(2, 3, True)
    n, r, kappa, h, steps = 6, 3, 0.5, 0.01, 30
    rng = li.rng_for(6, 0)
    V0 = li.haar_orthonormal(1 << n, r, rng)
    lam = li.dirichlet_spectrum(r, rng)
    dz = np.full(len(bonds), D_PAPER)
    H = model.hamiltonian(n, bonds, B_PAPER, dmi=[(0.0, 0.0, d) for d in dz])
    M = {v: model.magnetization_op(v, n) for v in "xyz"}
    L = Lrei(n, bonds, B_PAPER, kappa, mdl, precision, r)
    L.set_dmi(dz)
    L.set_state(_dev(V0, precision), lam)
    _, traj = de.integrate(V0, lam, H, kappa, mdl, h, steps, scheme, Mops=M, every=10)
    sE = float(np.sum(np.abs(bonds.jxy) + np.abs(bonds.jz) / 2 + np.abs(dz)) + n * np.linalg.norm(B_PAPER) / 2)
    s = {"energy": sE, "mx": 0.5, "my": 0.5, "mz": 0.5, "purity": 1.0, "trace": 1.0}
    tol = 1e-10 if precision == "fp64" else 1e-6
    for k, ref, mu in traj:
        L.step(h, scheme, 10)
        o = L.observables()
        err = max(abs(o[q] - ref[q]) / max(abs(ref[q]), s[q]) for q in s)
        assert err <= tol, (k, err)
        assert np.abs(o["ritz"] - mu).max() <= tol * lam.max()
