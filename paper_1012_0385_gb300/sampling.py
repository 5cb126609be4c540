"""Sampling times of the width W(L, t).

Eq. (sampling), paper sec. 2.2: t_0 = 30 and t_{i+1} = 1.05 t_i; the width
is recorded at floor(t_i) (double recurrence, duplicates dropped), optionally
preceded by t = 0, the flat start.  Up to 10^7 sweeps this gives t_0 and the
paper's 260 further sampling events.
"""
from __future__ import annotations

import math


def log_times(t_max: int, t0: int = 30, ratio: float = 1.05, include_zero: bool = True) -> list[int]:
    times = [0] if include_zero else []
    t = float(t0)
    while math.floor(t) <= t_max:
        v = int(math.floor(t))
        if not times or times[-1] != v:
            times.append(v)
        t *= ratio
    return times


def every(step: int, t_max: int, include_zero: bool = True) -> list[int]:
    """Uniform snapshots every `step` sweeps (e.g. the lattice every 100 MCS)."""
    return ([0] if include_zero else []) + list(range(step, t_max + 1, step))
