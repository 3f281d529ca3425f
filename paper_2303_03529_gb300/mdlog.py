"""Per-step metrics of an MD run as JSON lines (no counterpart in the paper).

One line per logged step with the paper's three traces (total energy per
atom, temperature, RMS(q - n)), the chemical potential, the spin moments and
the wall time per step:

    {"step": 40, "E_tot_per_atom": -7.812, "T": 301.2, "rms_q_minus_n": 3.4e-05,
     "mu": -4.93, "m_total": 0.0, "m_abs_max": 0.0, "wall_s_per_step": 0.47}

`step_record` builds one record from the library's per-step statistics row
[E_tot (eV), T (K), RMS(q - n), mu (eV)] and the charges and spins q of the
evaluation (up block, then down block; per atom, or per atom and shell).
`run` steps a context and appends records to a file.  `spin_flip_events`
scans records for the marks a spin flip leaves: the residual jumps and the
moments change abruptly (the paper's Summary and Discussion names such
flips, a discontinuity of the potential, as a limit of collinear spins).
"""
from __future__ import annotations

import json
import time

import numpy as np


def spin_moments(q, n_atoms: int):
    """Per-atom moments m_I = q_up,I - q_dn,I (summed over shells when q is
    shell-resolved) from q = [up block; down block]."""
    q = np.asarray(q, dtype=np.float64)
    half = q.size // 2
    if half % n_atoms != 0:
        raise ValueError(f"q of length {q.size} does not fit {n_atoms} atoms")
    up = q[:half].reshape(n_atoms, -1).sum(axis=1)
    dn = q[half:].reshape(n_atoms, -1).sum(axis=1)
    return up - dn


def step_record(step: int, stats_row, n_atoms: int, q=None, wall_s_per_step=None) -> dict:
    e_tot, temp, rms, mu = (float(x) for x in stats_row[:4])
    rec = {"step": int(step), "E_tot_per_atom": e_tot / n_atoms, "T": temp,
           "rms_q_minus_n": rms, "mu": mu}
    if q is not None:
        m = spin_moments(q, n_atoms)
        rec["m_total"] = float(m.sum())
        rec["m_abs_max"] = float(np.abs(m).max())
    if wall_s_per_step is not None:
        rec["wall_s_per_step"] = float(wall_s_per_step)
    return rec


def run(ctx, nsteps: int, path, every: int = 1, spins: bool = True):
    """nsteps sXL-BOMD steps of a library context; after every `every`
    steps appends the record of the last one to the JSON-lines file at
    path.  Returns the records written."""
    if nsteps < 0 or every < 1:
        raise ValueError("nsteps >= 0 and every >= 1")
    out = []
    with open(path, "a") as f:
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            t0 = time.perf_counter()
            stats = ctx.step(k, stats=True)
            wall = (time.perf_counter() - t0) / k
            done += k
            q = ctx.charges() if spins else None
            rec = step_record(ctx.md_step(), stats[-1], ctx.nat, q, wall)
            f.write(json.dumps(rec) + "\n")
            out.append(rec)
    return out


def spin_flip_events(records, rms_factor: float = 10.0, moment_jump: float = 0.5):
    """Steps at which a spin flip shows in a sequence of records: the
    residual RMS(q - n) grows by more than rms_factor over the previous
    record, or the total or the largest atomic moment changes by more than
    moment_jump (electrons) between consecutive records.  Returns a list of
    (step, reason) pairs."""
    events = []
    for prev, cur in zip(records, records[1:]):
        step = cur["step"]
        if prev["rms_q_minus_n"] > 0 and cur["rms_q_minus_n"] > rms_factor * prev["rms_q_minus_n"]:
            events.append((step, "residual jump"))
        for key in ("m_total", "m_abs_max"):
            if key in cur and key in prev and abs(cur[key] - prev[key]) > moment_jump:
                events.append((step, f"{key} jump"))
    return events

