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


def janus_wetting_lengths(theta13: float, theta23: float, s12: float = 1.0, s13: float = 1.0,
                          s23: float = 1.0, R: float = 1.0):
    """Equilibrium wetting lengths (L1 / R, L2 / R) of a Janus drop on a flat wall in 2D:
    liquids 1 (left) and 2 (right) of equal areas pi R^2 / 4 (the initial half disc of
    radius R, halved), in fluid 3, no gravity (Section 4.3, Table 2 analytic column).

    Equilibrium: every interface is a circular arc; at the wall each contact line obeys
    Young's law, with the 1-2 contact angle from the same wall energies,
    s12 cos theta_12 = s13 cos theta13 - s23 cos theta23 (angles measured inside liquid 1,
    liquid 1 and liquid 2); the three arcs meet at a triple junction where the tensions
    balance, s13 t13 + s23 t23 + s12 t12 = 0 (unit tangents pointing away from the
    junction).  Unknowns: the two outer contact points, the three curvatures and the three
    arc lengths (the 1-2 contact point is the origin); equations: the three arcs end at one
    point (4), the tension balance (2) and the two areas (2), solved by least squares from
    several starts.  The Laplace relation of the three curvatures then holds by itself."""
    import numpy as np
    from scipy.optimize import least_squares

    t13, t23 = math.radians(theta13), math.radians(theta23)
    c12 = (s13 * math.cos(t13) - s23 * math.cos(t23)) / s12
    t12 = math.acos(c12)
    area = math.pi * R * R / 4.0

    def arc(x0, a0, turn, length, n=4000):
        # start (x0, 0), initial direction angle a0, direction angle a0 + turn * s
        s = np.linspace(0.0, length, n)
        a = a0 + turn * s
        return x0 + (np.sin(a) - math.sin(a0)) / turn, (math.cos(a0) - np.cos(a)) / turn

    def polygon_area(x, y):
        return 0.5 * abs(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))

    def residual(v):
        xL, k1, l1, xR, k2, l2, k12, l12 = v
        k12 = k12 if abs(k12) > 1e-9 else 1e-9
        x1, y1 = arc(xL, t13, -k1, l1)                 # 1-3: from the left contact, bending right
        x2, y2 = arc(xR, math.pi - t23, k2, l2)        # 2-3: from the right contact, bending left
        x3, y3 = arc(0.0, math.pi - t12, k12, l12)     # 1-2: from the origin
        a1, a2, a3 = t13 - k1 * l1, math.pi - t23 + k2 * l2, math.pi - t12 + k12 * l12
        bal = -(s13 * np.array([math.cos(a1), math.sin(a1)]) + s23 * np.array([math.cos(a2), math.sin(a2)]) +
                s12 * np.array([math.cos(a3), math.sin(a3)]))
        A1 = polygon_area(np.r_[xL, 0.0, x3, x1[::-1]], np.r_[0.0, 0.0, y3, y1[::-1]])
        A2 = polygon_area(np.r_[0.0, xR, x2, x3[::-1]], np.r_[0.0, 0.0, y2, y3[::-1]])
        return np.r_[x1[-1] - x3[-1], y1[-1] - y3[-1], x2[-1] - x3[-1], y2[-1] - y3[-1], bal,
                     (A1 - area) / R ** 2, (A2 - area) / R ** 2]

    rng = np.random.default_rng(0)
    v0 = np.array([-1.0, 1.0, 2.0, 1.0, 1.0, 2.0, 0.1, 1.0]) * np.array([R, 1 / R, R, R, 1 / R, R, 1 / R, R])
    lo = np.array([-5 * R, 0.01 / R, 0.01 * R, 0.0, 0.01 / R, 0.01 * R, -5 / R, 0.01 * R])
    hi = np.array([0.0, 10 / R, 10 * R, 5 * R, 10 / R, 10 * R, 5 / R, 10 * R])
    best = None
    for trial in range(100):
        start = v0 if trial == 0 else np.clip(v0 * rng.uniform(0.5, 1.5, 8), lo + 1e-6, hi - 1e-6)
        r = least_squares(residual, start, bounds=(lo, hi), xtol=1e-14, ftol=1e-14, gtol=1e-14)
        if best is None or r.cost < best.cost:
            best = r
        if best.cost < 1e-22:
            break
    if best.cost > 1e-16:
        raise RuntimeError(f"Janus geometry did not converge (cost {best.cost:.3e})")
    xL, xR = best.x[0], best.x[3]
    return -xL / R, xR / R


def janus_contact_lengths(phi):
    """Wetting lengths (L1, L2) of a Janus drop on the bottom wall from the order
    parameters phi[3, ny, nx] (cell centres at i + 1/2, half-way wall at y = 0).  Along
    each of the two rows next to the wall: the 1-2 contact point is where phi_1 - phi_2
    changes sign under the drop (phi_3 < 1/2), nearest to the middle of the row; the outer
    contact points are the nearest crossings of phi_3 = 1/2 to its left and right (linear
    interpolation).  Each point is extrapolated linearly from the rows at y = 1/2 and 3/2
    to the wall at y = 0."""
    import numpy as np

    def row_points(p1, p2, p3):
        p1, p2, p3 = (np.asarray(a, dtype=float) for a in (p1, p2, p3))
        n = p1.size
        d = p1 - p2
        cands = [k for k in range(n - 1) if d[k] > 0.0 >= d[k + 1] and p3[k] < 0.5 and p3[k + 1] < 0.5]
        if not cands:
            raise ValueError("no 1-2 contact point")
        k = min(cands, key=lambda i: abs(i - n / 2.0))
        xc = k + 0.5 + d[k] / (d[k] - d[k + 1])
        g = p3 - 0.5
        left = next(i for i in range(k, 0, -1) if g[i - 1] >= 0.0 > g[i])
        right = next(i for i in range(k + 1, n - 1) if g[i] < 0.0 <= g[i + 1])
        xL = left - 0.5 + g[left - 1] / (g[left - 1] - g[left])
        xR = right + 0.5 + g[right] / (g[right] - g[right + 1])
        return xL, xc, xR

    r0 = row_points(phi[0][0], phi[1][0], phi[2][0])
    r1 = row_points(phi[0][1], phi[1][1], phi[2][1])
    xL, xc, xR = (1.5 * a - 0.5 * b for a, b in zip(r0, r1))
    return xc - xL, xR - xc


def brinkman_profile(H: float, y_chi, chi, g: float, nu: float, n: int = 64000):
    """Steady velocity u(y) of a unidirectional flow between walls at y = 0 and y = H
    driven by the body force g and damped by the penalty force of the flow LBE (Section 3:
    f = chi (u_s - u*), u = u* + f / 2, u_s = 0, so f = -k u with k = chi / (1 - chi / 2)):
    nu u'' - k(y) u + g = 0, u(0) = u(H) = 0.  chi(y) is interpolated linearly from the
    samples (y_chi, chi); the equation is solved by second-order finite differences on n
    intervals.  Returns (y, u) on the fine grid."""
    import numpy as np
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    y = np.linspace(0.0, H, n + 1)
    dy = y[1] - y[0]
    c = np.interp(y, y_chi, chi)
    k = c / (1.0 - 0.5 * c)
    m = n - 1
    A = sp.diags([np.full(m - 1, nu / dy ** 2), -2.0 * nu / dy ** 2 - k[1:-1], np.full(m - 1, nu / dy ** 2)],
                 [-1, 0, 1], format="csc")
    u = np.zeros(n + 1)
    u[1:-1] = spl.spsolve(A, -g * np.ones(m))
    return y, u
