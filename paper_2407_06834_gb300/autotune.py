"""Autotuner cache: the fastest work tiling (points per item, points per
unit) and the spread / interpolation launch shape per arithmetic, per
problem class, found by nlh_plan_autotune and kept in a JSON file (one per
machine, next to the built library).

Problem class key: grid size n_os, stencil half-width m, window count L and
log2 of N; it is known before a plan is built, so a cached tiling goes
straight into the plan description.
"""
from __future__ import annotations

import json
import math
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("NLH_AUTOTUNE_CACHE", os.path.join(_HERE, "_build", "autotune.json"))
_lock = threading.Lock()


def key_of(n_os: int, m: int, L: int, N: int) -> str:
    return "n%d_m%d_L%d_N%d" % (n_os, m, L, int(math.log2(max(2, N))))


def _read() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _write(d: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def lookup(n_os: int, m: int, L: int, N: int):
    with _lock:
        return _read().get(key_of(n_os, m, L, N))


def tune_and_record(plan, stream=None) -> dict:
    """Tune `plan` in place and record the winner for its class."""
    info = plan.info()
    res = plan.autotune(stream=stream)
    with _lock:
        d = _read()
        d[key_of(info["n_os"], info["m"], info["L"], info["N"])] = {
            "max_items_pts": res["max_items_pts"], "unit_points": res["unit_points"],
            "team": res["team"], "ms": res["ms"]}
        _write(d)
    return res
