"""Per-step metrics as JSON lines: a harness around a context's public calls.

`run_logged` steps a context and, every `every` steps, appends one JSON object per line to a
file: the step count, the time, the observables of lrei_observables (energy, magnetisations,
purity, trace, the factor's orthonormality error ||V*V - I||, the Hermiticity error of V*HV,
the commutator norm), the Ritz values' drift from the conserved spectrum,
max_i |mu_i - lambda0_i| / max_i lambda0_i, the wall time of the steps since the previous line,
and the kernels the library launched for the context since the previous line (the observables
read included).  Nothing here computes a step; it only reads
what the library returns.
"""
from __future__ import annotations

import json
import time

import numpy as np

_FIELDS = ("energy", "mx", "my", "mz", "purity", "trace", "orth_err", "herm_err", "comm_norm")


def metrics_line(L, step: int, wall_s: float) -> dict:
    """One record for the context's current state."""
    o = L.observables()
    lam = np.asarray(o["lambda0"], dtype=np.float64)
    ritz = np.asarray(o["ritz"], dtype=np.float64)
    rec = {"step": int(step), "t": float(o["t"])}
    rec.update({k: float(o[k]) for k in _FIELDS})
    rec["ritz_drift"] = float(np.abs(ritz - lam).max() / lam.max()) if lam.size and lam.max() > 0 else 0.0
    rec["rank"] = int(o["r"])
    rec["wall_s"] = float(wall_s)
    rec["kernel_launches"] = int(L.kernel_launches())
    return rec


def run_logged(L, dt: float, nsteps: int, path: str, scheme: str = "rk4", every: int = 1) -> list[dict]:
    """Step L by nsteps fixed steps of dt, writing a record of the start and of every `every`
    steps (and of the last) to `path` (appended).  Returns the records."""
    if every < 1 or nsteps < 0:
        raise ValueError("every >= 1 and nsteps >= 0")
    recs = [metrics_line(L, 0, 0.0)]
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        t0 = time.perf_counter()
        L.step(dt, scheme, k)
        wall = time.perf_counter() - t0
        done += k
        recs.append(metrics_line(L, done, wall))
    with open(path, "a") as f:
        for rec in recs:
            f.write(json.dumps(rec) + "\n")
    return recs
