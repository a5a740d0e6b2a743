"""Compact volume quadrature rules on the reference tetrahedron (inputs).

``quadrature_rules.json`` holds, for N = 1..5, a fully symmetric rule of
degree 2N with positive weights and interior points, as rows (r, s, t, w) on
the reference tetrahedron (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1) whose
weights sum to its volume 4/3.  The rules were written once by
``synthetic/make_quadrature.py`` (a moment-equation solve; the paper's own
tabulated rules are not available).  Like a mesh, a rule is an input: the
oracle and the library each build their operators from it, and each side
checks it independently.
"""
from __future__ import annotations

import functools
import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "quadrature_rules.json")


@functools.lru_cache(maxsize=None)
def _doc():
    with open(PATH) as f:
        return json.load(f)


def compact_rule(N: int) -> np.ndarray:
    """(nq, 4) array of r, s, t, w of the compact degree-2N rule."""
    return np.array(_doc()["rules"][str(N)]["rstw"], dtype=np.float64)


def compact_rule_info(N: int) -> dict:
    r = _doc()["rules"][str(N)]
    return {"degree": r["degree"], "points": r["points"],
            "orbits": [o["kind"] for o in r["orbits"]]}
