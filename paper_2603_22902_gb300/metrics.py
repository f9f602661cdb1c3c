"""Measurements taken on exported fields (host side, numpy)."""
from __future__ import annotations

import numpy as np


def front_height(F, nx: int) -> float:
    """Height of the solid at the centre line of a drop freezing from the wall y = 0:
    sum_y f_s phi_0 over the four central columns, averaged (lattice units)."""
    cols = slice(nx // 2 - 2, nx // 2 + 2)
    return float(((1.0 - np.asarray(F["fl"])) * np.asarray(F["phi"])[0])[:, cols].sum(axis=0).mean())


def front_integral(F, nx: int) -> float:
    """Solid height averaged over the width: sum over the whole lattice of f_s phi_0,
    divided by nx (lattice units)."""
    return float(((1.0 - np.asarray(F["fl"])) * np.asarray(F["phi"])[0]).sum() / nx)
