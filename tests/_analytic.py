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
