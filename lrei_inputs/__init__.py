"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the LREI method itself: it only draws
random numbers and lays out named basis states, bond lists and the five
workload recipes.  Both sides of every parity test receive the same arrays
from here.

Conventions (the paper's spin-1/2 Kronecker order, Sec. 3.6, eq. spin_op):
  * site i (0-based) is Kronecker factor i counted from the left, i.e. bit
    (n-1-i) of the basis index b (site 0 is the most significant bit);
  * bit value 0 is spin up (S^z = +1/2), 1 is spin down.

Seed recipe: workload c, trajectory t uses numpy Generator(PCG64(1000*c + t));
draw order is bond anisotropies, then the initial factor V, then Lambda.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np

__all__ = [
    "Bonds", "chain_bonds", "triangular_bonds", "haar_orthonormal", "dirichlet_spectrum",
    "basis_state", "af1_state", "af2_state", "ghz_state", "w_state",
    "Workload", "workload", "rng_for", "load_config",
]


@dataclasses.dataclass
class Bonds:
    """Exchange bonds (i, j) with coupling Jxy (S^+S^- part) and Jz (S^zS^z part)."""
    site_i: np.ndarray  # int32
    site_j: np.ndarray  # int32
    jxy: np.ndarray     # float64
    jz: np.ndarray      # float64

    def __len__(self):
        return int(self.site_i.shape[0])


def rng_for(config: int, traj: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * config + traj))


def chain_bonds(n: int, periodic: bool, J: float = 1.0, aniso: np.ndarray | None = None) -> Bonds:
    """Nearest-neighbour chain bonds; Jz = J + aniso[b] when an anisotropy list is given."""
    m = n if (periodic and n > 2) else n - 1
    si = np.arange(m, dtype=np.int32)
    sj = ((si + 1) % n).astype(np.int32)
    jxy = np.full(m, float(J))
    jz = np.full(m, float(J))
    if aniso is not None:
        jz = jz + np.asarray(aniso, dtype=np.float64)[:m]
    return Bonds(si, sj, jxy, jz)


def triangular_bonds(lx: int, ly: int, periodic: bool = True, J: float = 1.0) -> Bonds:
    """Nearest-neighbour bonds of an lx x ly triangular lattice (sites row by row, site = y lx + x):
    each site bonds to its right, upper and upper-right neighbours (the three lattice directions);
    with periodic boundaries the neighbours wrap around, duplicate pairs are listed once."""
    pairs = []
    seen = set()
    for y in range(ly):
        for x in range(lx):
            i = y * lx + x
            for dx, dy in ((1, 0), (0, 1), (1, 1)):
                xx, yy = x + dx, y + dy
                if periodic:
                    xx, yy = xx % lx, yy % ly
                elif xx >= lx or yy >= ly:
                    continue
                j = yy * lx + xx
                key = (min(i, j), max(i, j))
                if i != j and key not in seen:
                    seen.add(key)
                    pairs.append((i, j))
    si = np.array([p[0] for p in pairs], dtype=np.int32)
    sj = np.array([p[1] for p in pairs], dtype=np.int32)
    return Bonds(si, sj, np.full(len(pairs), float(J)), np.full(len(pairs), float(J)))


def haar_orthonormal(N: int, r: int, rng: np.random.Generator) -> np.ndarray:
    """N x r matrix with Haar-distributed orthonormal columns (complex Ginibre + QR, Mezzadri 2007)."""
    G = (rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    ph = d / np.abs(d)
    return np.ascontiguousarray(Q * ph[None, :])


def dirichlet_spectrum(r: int, rng: np.random.Generator, alpha: float = 1.0) -> np.ndarray:
    """Dirichlet(alpha) weights sorted in decreasing order (a trace-one positive spectrum)."""
    lam = rng.dirichlet(np.full(r, alpha))
    return np.sort(lam)[::-1].copy()


def basis_state(n: int, index: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[index] = 1.0
    return v


def _alternating(n: int, first: int) -> int:
    # bit string of length n read from site 0 (MSB) to site n-1 (LSB)
    idx = 0
    for i in range(n):
        bit = (first + i) & 1
        idx = (idx << 1) | bit
    return idx


def af1_state(n: int) -> np.ndarray:
    """|AF1>: the single basis state whose bit string is 0101... (site 0 first)."""
    return basis_state(n, _alternating(n, 0))


def af2_state(n: int) -> np.ndarray:
    """|AF2>: the single basis state whose bit string is 1010... (site 0 first)."""
    return basis_state(n, _alternating(n, 1))


def ghz_state(n: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    v[0] = v[(1 << n) - 1] = 1.0 / np.sqrt(2.0)
    return v


def w_state(n: int) -> np.ndarray:
    v = np.zeros(1 << n, dtype=np.complex128)
    for i in range(n):
        v[1 << (n - 1 - i)] = 1.0 / np.sqrt(n)
    return v


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    r: int
    bonds: Bonds
    B: tuple
    kappa: float
    model: str          # "qll" | "qllg"
    scheme: str         # "rk4", "ab3", ...
    dt: float
    steps: int
    V: np.ndarray | None = None
    lam: np.ndarray | None = None


CONFIG_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "configs")


def load_config(config: int) -> dict:
    """The recipe of workload `config` from configs/cfg<config>.json."""
    with open(os.path.join(CONFIG_DIR, f"cfg{config}.json")) as f:
        return json.load(f)


def workload(config: int, traj: int = 0, *, n: int | None = None, r: int | None = None,
             kappa: float | None = None, model: str | None = None, scheme: str | None = None,
             with_state: bool = True) -> Workload:
    """The synthetic workloads, from the recipes in configs/cfg1.json .. cfg5.json.

    1: open chain n=8, r=4, J=1, B_z=0.5, kappa=0.1, q-LL, RK4, dt=0.01, 1000 steps.
    2: periodic chain n=16, r=8, Jxy=1, Jz=1+U[-0.2,0.2] per bond, B_z=1, dt=0.005, 500 steps.
    3: open chain n=20, r=16, J=1, B_z=0.5, kappa=0.1, RK4, dt=0.01, 100 steps.
    4: open chains n in U{10..18}, r in U{2..16}, kappa log-uniform in [1e-3, 1], RK4, dt=0.01, 200 steps.
    5: open chain n=22, r=32, kappa=0.05, J=1, B_z=0.5, 50 steps (controller evaluation).
    Keyword overrides let tests shrink a workload while keeping its recipe.  Draw order per seed:
    n, r, kappa (where the recipe gives ranges), the bond anisotropies, then V, then Lambda.
    """
    if config not in (1, 2, 3, 4, 5):
        raise ValueError(f"unknown workload {config}")
    cfg = load_config(config)
    lat = cfg["lattice"]
    rng = rng_for(config, traj)
    if "n_range" in lat:
        lo, hi = lat["n_range"]
        nn = n or int(rng.integers(lo, hi + 1))
    else:
        nn = n or int(lat["n"])
    if "r_range" in cfg:
        lo, hi = cfg["r_range"]
        rr = r or int(rng.integers(lo, hi + 1))
    else:
        rr = int(cfg["r"])
    if "kappa_log10_range" in cfg:
        lo, hi = cfg["kappa_log10_range"]
        kap = kappa if kappa is not None else float(10.0 ** rng.uniform(lo, hi))
    else:
        kap = float(cfg["kappa"])
    aniso = None
    if lat.get("jz_aniso"):
        m = nn if (lat["periodic"] and nn > 2) else nn - 1
        aniso = rng.uniform(lat["jz_aniso"][0], lat["jz_aniso"][1], size=m)
    bonds = chain_bonds(nn, periodic=bool(lat["periodic"]), J=float(lat["jxy"]), aniso=aniso)
    B = tuple(float(x) for x in cfg["B"])
    mdl, sch, dt, steps = cfg["model"], cfg["scheme"], float(cfg["dt"]), int(cfg["steps"])
    rr = r or rr
    kap = kappa if kappa is not None else kap
    mdl = model or mdl
    sch = scheme or sch
    w = Workload(f"cfg{config}", nn, rr, bonds, B, kap, mdl, sch, dt, steps)
    if with_state:
        w.V = haar_orthonormal(1 << nn, rr, rng)
        w.lam = dirichlet_spectrum(rr, rng)
    return w
