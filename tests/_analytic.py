"""Closed-form references used by the oracle pins (no lattice-Boltzmann arithmetic)."""
import math


def neumann_kappa(ste: float) -> float:
    """Root of Ste / (exp(k^2) erf(k)) = k sqrt(pi): the one-phase Neumann problem
    (Section 4.1 transcendental equation with the liquid at the melting point)."""
    f = lambda k: ste / (math.exp(k * k) * math.erf(k)) - k * math.sqrt(math.pi)
    lo, hi = 1e-9, 3.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def neumann_front(ste: float, alpha: float, t: float) -> float:
    """Solid thickness s(t) = 2 kappa sqrt(alpha_s t)."""
    return 2.0 * neumann_kappa(ste) * math.sqrt(alpha * t)


def neumann_triangle(s12: float, s23: float, s13: float):
    """Angles (degrees) that the upper (phases 2-3) and lower (phases 2-1) arcs of a
    lens of phase 2 make with a flat 1-3 interface at the triple point, from the force
    balance of the three tensions (Neumann's triangle): s13 = s23 cos(a_u) + s12 cos(a_d)
    and s23 sin(a_u) = s12 sin(a_d).  Needs s23 <= s12 and a lens (s13 < s12 + s23)."""
    def resid(au):
        ad = math.asin(min(1.0, s23 * math.sin(au) / s12))
        return s23 * math.cos(au) + s12 * math.cos(ad) - s13
    lo, hi = 1e-12, 0.5 * math.pi
    for _ in range(200):                      # resid decreases in au on (0, pi/2]
        mid = 0.5 * (lo + hi)
        if resid(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    au = 0.5 * (lo + hi)
    return math.degrees(au), math.degrees(math.asin(s23 * math.sin(au) / s12))


def level_crossings(a, level=0.5):
    """Points (x, y) where the cell-centred field a[y, x] (cell centres at i + 1/2)
    crosses `level` along rows and columns, by linear interpolation."""
    ny, nx = len(a), len(a[0])
    pts = []
    for i in range(nx):
        for j in range(ny - 1):
            u, v = a[j][i] - level, a[j + 1][i] - level
            if u * v < 0.0:
                pts.append((i + 0.5, j + 0.5 + u / (u - v)))
    for j in range(ny):
        for i in range(nx - 1):
            u, v = a[j][i] - level, a[j][i + 1] - level
            if u * v < 0.0:
                pts.append((i + 0.5 + u / (u - v), j + 0.5))
    return pts


def fit_circle(pts):
    """Least-squares circle x^2 + y^2 + D x + E y + F = 0 through the points (Kasa's
    algebraic fit): centre (xc, yc) and radius."""
    import numpy as np
    p = np.asarray(pts, dtype=float)
    x, y = p[:, 0], p[:, 1]
    D, E, F = np.linalg.lstsq(np.c_[x, y, np.ones_like(x)], -(x * x + y * y), rcond=None)[0]
    xc, yc = -D / 2.0, -E / 2.0
    return xc, yc, math.sqrt(xc * xc + yc * yc - F)


def cap_angle(yc: float, R: float, y0: float, up: bool = True) -> float:
    """Angle (degrees) between a circular arc of centre height yc and radius R and the
    line y = y0 where they meet, measured inside the cap that lies above the line (up)
    or below it."""
    c = (y0 - yc) / R if up else (yc - y0) / R
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def neumann_kappa_superheated(ste: float, superheat: float) -> float:
    """Root of Ste / (exp(k^2) erf(k)) - superheat Ste / (exp(k^2) erfc(k)) = k sqrt(pi):
    the two-phase Neumann problem (Section 4.1 transcendental equation) with equal
    conductivities, diffusivities and densities in the solid and the liquid, and
    superheat = (T_0 - T_m) / (T_m - T_w)."""
    f = lambda k: (ste / (math.exp(k * k) * math.erf(k)) - superheat * ste / (math.exp(k * k) * math.erfc(k))
                   - k * math.sqrt(math.pi))
    lo, hi = 1e-9, 3.0
    for _ in range(200):                      # f decreases from +inf
        mid = 0.5 * (lo + hi)
        if f(mid) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
