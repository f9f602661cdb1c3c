"""Seeded synthetic inputs: case parameters and initial fields.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle.  It holds no lattice-Boltzmann arithmetic: it only lays out the
geometry of the paper's test problems (Section 4: tanh order-parameter
profiles of the film, the sessile drop, the compound drop and the pools) and
chooses parameters.  Random draws use splitmix64 (Steele, Lea, Flood 2014),
uniform doubles as (x >> 11) * 2**-53.

Coordinates: cell (i, j) has its centre at (i + 1/2, j + 1/2); a half-way wall
on the y-min side sits at y = 0.
"""
from __future__ import annotations

import copy
import dataclasses
import math
from typing import List

import numpy as np

PERIODIC, WALL, OUTFLOW = 0, 1, 2
ADIABATIC, DIRICHLET = 0, 1
XMIN, XMAX, YMIN, YMAX = 0, 1, 2, 3


@dataclasses.dataclass
class Case:
    """Parameters and initial fields of one problem."""

    name: str
    nx: int
    ny: int
    N: int
    phases: List[dict]          # rho_l, rho_s, mu_l, mu_s, lam_l, lam_s, cp_l, cp_s, latent
    sigma: np.ndarray           # [N, N]
    eps: float = 4.0
    mobility: float = 0.02
    T_sol: float = 0.0
    T_liq: float = 0.0
    rho_ref: float = 1.0
    cp_ref: float = 1.0
    u_solid: tuple = (0.0, 0.0)
    accel: tuple = (0.0, 0.0)
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    tbc: tuple = (ADIABATIC, ADIABATIC, ADIABATIC, ADIABATIC)
    T_wall: tuple = (0.0, 0.0, 0.0, 0.0)
    wet_cos: np.ndarray = None  # [4, N, N], antisymmetric per side
    phi: np.ndarray = None      # [N, ny, nx]
    T: np.ndarray = None        # [ny, nx]
    ux: np.ndarray = None
    uy: np.ndarray = None
    meta: dict = dataclasses.field(default_factory=dict)

    def __post_init__(self):
        self.sigma = np.asarray(self.sigma, dtype=np.float64)
        if self.wet_cos is None:
            self.wet_cos = np.zeros((4, self.N, self.N))
        if self.T is None:
            self.T = np.zeros((self.ny, self.nx))
        if self.ux is None:
            self.ux = np.zeros((self.ny, self.nx))
        if self.uy is None:
            self.uy = np.zeros((self.ny, self.nx))

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def copy(self) -> "Case":
        return copy.deepcopy(self)


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of splitmix64 started at `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = (np.uint64(seed & _M64) + k * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def phase(rho_l=1.0, rho_s=None, mu_l=0.1, mu_s=None, lam_l=0.1, lam_s=None,
          cp_l=1.0, cp_s=None, latent=0.0) -> dict:
    return dict(rho_l=rho_l, rho_s=rho_l if rho_s is None else rho_s,
                mu_l=mu_l, mu_s=mu_l if mu_s is None else mu_s,
                lam_l=lam_l, lam_s=lam_l if lam_s is None else lam_s,
                cp_l=cp_l, cp_s=cp_l if cp_s is None else cp_s, latent=latent)


def tanh_step(d, eps):
    """1/2 + 1/2 tanh(d / (eps/2)): 1 where d > 0 (Section 4 initial profiles)."""
    return 0.5 + 0.5 * np.tanh(d / (eps / 2.0))


def grid(nx, ny):
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    return np.meshgrid(x, y)  # X[ny, nx], Y[ny, nx]


def sigma_matrix(N, pairs):
    s = np.zeros((N, N))
    for (p, q), v in pairs.items():
        s[p, q] = s[q, p] = v
    return s


def wetting(N, side_angles):
    """wet_cos[4, N, N] from {side: {(p, q): theta_deg}} (cos antisymmetric)."""
    w = np.zeros((4, N, N))
    for side, pairs in side_angles.items():
        for (p, q), th in pairs.items():
            c = math.cos(math.radians(th))
            w[side, p, q] = c
            w[side, q, p] = -c
    return w


def latent_from_stefan(ste: float, cp_s: float = 1.0, dT_ref: float = 1.0) -> float:
    """Ste = c_p,s (T_m - T_w) / L with a fixed reference difference T_m - T_w = dT_ref."""
    return cp_s * dT_ref / ste


# --------------------------------------------------------------------------
# the paper's problems (Section 4) and the small cases of the tests
# --------------------------------------------------------------------------

def film(nx=16, ny=256, h0=128.0, ste=0.1, rho_ratio=0.9, T_wall=-1.0, T0=0.0,
         lam=0.1, mu=0.1, sigma=1e-3, eps=4.0, mobility=0.02, rho_gas=1.0) -> Case:
    """Film freezing (Section 4.1): liquid 0 < y < h0 under gas, cold bottom wall,
    outflow top, x periodic."""
    X, Y = grid(nx, ny)
    phi1 = tanh_step(h0 - Y, eps)
    phi = np.stack([phi1, 1.0 - phi1])
    phases = [phase(rho_l=1.0, rho_s=rho_ratio, mu_l=mu, lam_l=lam, latent=latent_from_stefan(ste)),
              phase(rho_l=rho_gas, mu_l=mu * rho_gas, lam_l=lam)]
    return Case(name=f"film_{nx}x{ny}", nx=nx, ny=ny, N=2, phases=phases,
                sigma=sigma_matrix(2, {(0, 1): sigma}), eps=eps, mobility=mobility,
                bc=(PERIODIC, PERIODIC, WALL, OUTFLOW), tbc=(ADIABATIC, ADIABATIC, DIRICHLET, ADIABATIC),
                T_wall=(0.0, 0.0, T_wall, 0.0), phi=phi, T=np.full((ny, nx), T0),
                meta=dict(h0=h0, ste=ste, rho_ratio=rho_ratio, T_wall=T_wall))


def sessile_drop(n=512, R=100.0, ste=0.1, rho_ratio=0.9, theta=90.0, T_wall=-1.0, T0=1.0,
                 rho_gas=0.01, mu_l=0.02, mu_gas=0.002, lam_l=0.1, lam_gas=0.01, cp_gas=100.0,
                 sigma=1e-3, eps=4.0, mobility=0.03, ny=None) -> Case:
    """Single droplet on a cold wall (Section 4.2): drop of radius R centred on the
    bottom wall, gas around it, x periodic, bottom Dirichlet + wetting, top adiabatic wall.

    Unstated parameters: the drop starts superheated at T0 = 1 (the paper's film
    setting), and the gas heat capacity makes rho_g c_g equal to rho_l c_l, because the
    total-enthalpy LBE with one rho_ref c_p,ref is unstable where rho c_p is far below it.
    The mobility is 0.03: at 0.02 (the film problem's value) the 512 x 512 drop stays
    bounded only to ~17 500 steps (the peak velocity then grows from ~1e-2 to 6e-2 and T
    undershoots the wall temperature), while at 0.03 and 0.05 every precision policy
    stays bounded through 20 000 steps."""
    nx, ny = n, (ny or n)
    X, Y = grid(nx, ny)
    r = np.sqrt((X - nx / 2.0) ** 2 + Y ** 2)
    phi1 = tanh_step(R - r, eps)
    phi = np.stack([phi1, 1.0 - phi1])
    phases = [phase(rho_l=1.0, rho_s=rho_ratio, mu_l=mu_l, lam_l=lam_l, latent=latent_from_stefan(ste)),
              phase(rho_l=rho_gas, mu_l=mu_gas, lam_l=lam_gas, cp_l=cp_gas)]
    return Case(name=f"sessile_drop_{nx}x{ny}", nx=nx, ny=ny, N=2, phases=phases,
                sigma=sigma_matrix(2, {(0, 1): sigma}), eps=eps, mobility=mobility,
                bc=(PERIODIC, PERIODIC, WALL, WALL), tbc=(ADIABATIC, ADIABATIC, DIRICHLET, ADIABATIC),
                T_wall=(0.0, 0.0, T_wall, 0.0), wet_cos=wetting(2, {YMIN: {(0, 1): theta}}),
                phi=phi, T=np.full((ny, nx), T0),
                meta=dict(R=R, ste=ste, rho_ratio=rho_ratio, theta=theta, T_wall=T_wall))


def compound_drop(n=1024, R_core=80.0, R_shell=160.0, ste=0.2, seed=3, noise=1e-3,
                  T_wall=-1.0, T0=1.0, sigma12=1e-3, sigma23=1.5e-3, sigma13=3e-3,
                  eps=4.0, mobility=0.03, ny=None) -> Case:
    """Encapsulated compound drop (Section 4.3, Table 3): liquid core (phase 1) inside a
    liquid shell (phase 2) on a cold wall in gas (phase 3).

    The mobility is 0.03, as in the single-droplet problem: at 0.02 the 1024 x 1024 run
    diverges before step 10 000 (FP64) or 17 500 (FP32), at 0.03 and 0.05 it stays bounded
    through 50 000 steps (peak velocity ~2e-2)."""
    nx, ny = n, (ny or n)
    X, Y = grid(nx, ny)
    r = np.sqrt((X - nx / 2.0) ** 2 + Y ** 2)
    phi1 = tanh_step(R_core - r, eps)
    phi2 = (1.0 - phi1) * tanh_step(R_shell - r, eps)
    if noise:
        xi = uniform(seed, 2 * nx * ny, -noise, noise).reshape(2, ny, nx)
        phi1 = np.clip(phi1 + xi[0], 0.0, 1.0)
        phi2 = np.clip(phi2 + xi[1], 0.0, 1.0)
        over = phi1 + phi2
        scale = 1.0 / np.maximum(over, 1.0)
        phi1, phi2 = phi1 * scale, phi2 * scale
    phi3 = 1.0 - phi1 - phi2
    phi = np.stack([phi1, phi2, np.maximum(phi3, 0.0)])
    lam1 = 0.1
    phases = [phase(rho_l=1.0, rho_s=1.1, mu_l=0.02, lam_l=lam1, latent=latent_from_stefan(ste)),
              phase(rho_l=0.9, rho_s=0.81, mu_l=0.02, lam_l=2.7 * lam1, latent=latent_from_stefan(ste)),
              phase(rho_l=0.01, mu_l=0.002, lam_l=0.1 * lam1, cp_l=100.0)]
    sig = sigma_matrix(3, {(0, 1): sigma12, (1, 2): sigma23, (0, 2): sigma13})
    return Case(name=f"compound_drop_{nx}x{ny}", nx=nx, ny=ny, N=3, phases=phases, sigma=sig,
                eps=eps, mobility=mobility,
                bc=(PERIODIC, PERIODIC, WALL, WALL), tbc=(ADIABATIC, ADIABATIC, DIRICHLET, ADIABATIC),
                T_wall=(0.0, 0.0, T_wall, 0.0), phi=phi, T=np.full((ny, nx), T0),
                meta=dict(R_core=R_core, R_shell=R_shell, ste=ste, seed=seed))


def periodic_drop(n=64, R=16.0, sigma=1e-3, rho_ratio=1.0, mu=0.1, eps=4.0, mobility=0.02,
                  N=2, rho_gas=1.0, ny=None, cx=None, cy=None) -> Case:
    """A drop in a fully periodic box, no phase change (Laplace-law problem)."""
    nx, ny = n, (ny or n)
    X, Y = grid(nx, ny)
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2)
    phi1 = tanh_step(R - r, eps)
    phis = [phi1, 1.0 - phi1] + [np.zeros_like(phi1)] * (N - 2)
    phases = [phase(rho_l=1.0, mu_l=mu), phase(rho_l=rho_gas, mu_l=mu * rho_gas)]
    phases += [phase(rho_l=1.0, mu_l=mu) for _ in range(N - 2)]
    sig = np.full((N, N), sigma)
    np.fill_diagonal(sig, 0.0)
    return Case(name=f"periodic_drop_{nx}x{ny}", nx=nx, ny=ny, N=N, phases=phases, sigma=sig,
                eps=eps, mobility=mobility, phi=np.stack(phis), meta=dict(R=R, sigma=sigma))


def liquid_lens(nx=64, ny=48, R=10.0, y_bot=12.0, y_top=30.0, s12=1e-2, s23=1e-2, s13=1e-2, mu=0.1,
                eps=4.0, mobility=0.03) -> Case:
    """A lens of phase 2 at a flat interface between phase 1 (a band y_bot < y < y_top)
    and phase 3, fully periodic, equal densities, no phase change: a triple junction,
    whose interfacial angles the balance of the three tensions fixes (Section 2; with
    equal tensions all three are 120 degrees, as in the three-phase pool of Section 4.2).
    The lens starts as a disc of radius R centred on the upper 1-3 interface."""
    c = periodic_drop(n=nx, ny=ny, R=R, sigma=s12, mu=mu, eps=eps, mobility=mobility, N=3)
    c.sigma = sigma_matrix(3, {(0, 1): s12, (1, 2): s23, (0, 2): s13})
    X, Y = grid(nx, ny)
    lens = tanh_step(R - np.sqrt((X - nx / 2.0) ** 2 + (Y - y_top) ** 2), eps)
    band = tanh_step(Y - y_bot, eps) * tanh_step(y_top - Y, eps)
    phi1 = (1.0 - lens) * band
    c.phi = np.stack([phi1, lens, 1.0 - phi1 - lens])
    c.name = f"liquid_lens_{nx}x{ny}"
    c.meta = dict(R=R, y_bot=y_bot, y_top=y_top, s12=s12, s23=s23, s13=s13)
    return c


def channel(T0=1.0, H=32, g=1e-6, mu=0.1, nx=4) -> Case:
    """A liquid filling a channel between walls at y = 0 and y = H (half-way bounce-back),
    x periodic, driven by a body force g along x; walls and fluid at temperature T0
    (T0 > T_m: liquid, T0 < T_m: frozen solid with rho_s = rho_l)."""
    c = Case(name=f"channel_{nx}x{H}", nx=nx, ny=H, N=2,
             phases=[phase(rho_l=1.0, rho_s=1.0, mu_l=mu, latent=latent_from_stefan(0.1)),
                     phase(rho_l=1.0, mu_l=mu)],
             sigma=sigma_matrix(2, {(0, 1): 1e-3}),
             bc=(PERIODIC, PERIODIC, WALL, WALL), tbc=(ADIABATIC, ADIABATIC, DIRICHLET, DIRICHLET),
             T_wall=(0.0, 0.0, T0, T0), accel=(g, 0.0),
             phi=np.stack([np.ones((H, nx)), np.zeros((H, nx))]), T=np.full((H, nx), T0),
             meta=dict(g=g, mu=mu))
    return c


def frozen_layer_channel(H=64, h=12.0, g=1e-6, mu=0.1, T0=-0.5, nx=4, eps=4.0, sigma=1e-3,
                         mobility=0.02) -> Case:
    """A frozen layer of phase-changing material (phase 0, y < h, tanh profile) under a
    channel of ambient fluid (phase 1, latent heat 0), walls at y = 0 and y = H (half-way
    bounce-back), x periodic, driven by a body force g along x.  Walls (Dirichlet) and
    fluid at T0 < T_m, so the layer stays solid; equal densities (also rho_s = rho_l) and
    viscosities, so nothing changes volume and the interface stays flat."""
    X, Y = grid(nx, H)
    phi0 = tanh_step(h - Y, eps)
    return Case(name=f"frozen_layer_{nx}x{H}", nx=nx, ny=H, N=2,
                phases=[phase(rho_l=1.0, rho_s=1.0, mu_l=mu, latent=latent_from_stefan(0.1)),
                        phase(rho_l=1.0, mu_l=mu)],
                sigma=sigma_matrix(2, {(0, 1): sigma}), eps=eps, mobility=mobility,
                bc=(PERIODIC, PERIODIC, WALL, WALL), tbc=(ADIABATIC, ADIABATIC, DIRICHLET, DIRICHLET),
                T_wall=(0.0, 0.0, T0, T0), accel=(g, 0.0), phi=np.stack([phi0, 1.0 - phi0]),
                T=np.full((H, nx), T0), meta=dict(g=g, mu=mu, h=h))


def flat_interface(nx=4, ny=64, h0=None, sigma=1e-3, eps=4.0, mobility=0.02) -> Case:
    """Two flat interfaces in a periodic column (an exact tanh equilibrium of the AC equation)."""
    X, Y = grid(nx, ny)
    h0 = ny / 4.0 if h0 is None else h0
    phi1 = tanh_step(h0 - np.abs(Y - ny / 2.0), eps)
    phases = [phase(), phase()]
    return Case(name=f"flat_{nx}x{ny}", nx=nx, ny=ny, N=2, phases=phases,
                sigma=sigma_matrix(2, {(0, 1): sigma}), eps=eps, mobility=mobility,
                phi=np.stack([phi1, 1.0 - phi1]), meta=dict(h0=h0))


def lateral_pool(n=64, eps=4.0, sigma=0.01, T_wall=-1.0, T0=0.0, ste=0.2, freeze=True,
                 rho_ratio1=1.0, rho_ratio2=1.0, mobility=0.02) -> Case:
    """Two laterally placed liquids under gas (Section 4.1, Fig. 4 initial fields), walls
    on all sides.  With freeze=False the bottom wall is warm (no phase change)."""
    nx = ny = n
    X, Y = grid(nx, ny)
    L = float(n)
    lower = tanh_step(L / 2.0 - Y, eps)
    phi1 = tanh_step(L / 2.0 - X, eps) * lower
    phi2 = tanh_step(X - L / 2.0, eps) * lower
    phi3 = 1.0 - phi1 - phi2
    lat = latent_from_stefan(ste)
    phases = [phase(rho_l=1.0, rho_s=rho_ratio1, mu_l=0.05, latent=lat),
              phase(rho_l=1.0, rho_s=rho_ratio2, mu_l=0.05, latent=lat),
              phase(rho_l=1.0, mu_l=0.05)]
    sig = np.full((3, 3), sigma)
    np.fill_diagonal(sig, 0.0)
    return Case(name=f"lateral_pool_{n}", nx=nx, ny=ny, N=3, phases=phases, sigma=sig, eps=eps,
                mobility=mobility, bc=(WALL, WALL, WALL, WALL),
                tbc=(ADIABATIC, ADIABATIC, DIRICHLET if freeze else ADIABATIC, ADIABATIC),
                T_wall=(0.0, 0.0, T_wall, 0.0), phi=np.stack([phi1, phi2, phi3]),
                T=np.full((ny, nx), T0))


def perturbed(case: Case, seed: int, amp_u: float = 1e-3, amp_T: float = 0.0) -> Case:
    """Same case with seeded uniform noise on the initial velocity (and temperature)."""
    c = case.copy()
    n = c.nx * c.ny
    r = uniform(seed, 3 * n, -1.0, 1.0).reshape(3, c.ny, c.nx)
    c.ux = c.ux + amp_u * r[0]
    c.uy = c.uy + amp_u * r[1]
    if amp_T:
        c.T = c.T + amp_T * r[2]
    c.name += f"_perturbed{seed}"
    return c


def sessile_cap(nx, ny, R, theta=90.0, ste=0.1, T_wall=-1.0, T0=1.0, name=None, **kw) -> Case:
    """A drop on the cold wall y = 0 as a circular cap meeting the wall at the contact
    angle theta (centre at y = -R cos(theta)), with the wall wetting at theta; other
    parameters as the single-droplet problem (sessile_drop)."""
    c = sessile_drop(n=nx, ny=ny, R=R, theta=theta, ste=ste, T_wall=T_wall, T0=T0, **kw)
    X, Y = grid(nx, ny)
    yc = -R * math.cos(math.radians(theta))
    r = np.sqrt((X - nx / 2.0) ** 2 + (Y - yc) ** 2)
    phi1 = tanh_step(R - r, c.eps)
    c.phi = np.stack([phi1, 1.0 - phi1])
    c.name = name or f"sessile_cap_{nx}x{ny}_th{theta:.0f}"
    c.meta.update(yc=yc)
    return c


def janus_drop(nx=300, ny=150, R=60.0, theta13=75.0, theta23=90.0, eps=5.0, sigma=0.01, mu=0.1,
               mobility=0.05) -> Case:
    """Janus compound drop on a flat substrate (Section 4.3, Table 2): a half disc of
    radius R on the bottom wall, its left half liquid 1 (phase 0), its right half liquid 2
    (phase 1), in a third fluid (phase 2), with the initial profiles of Section 4.3.
    Equal pairwise tensions, no phase change.

    Wall wetting of the bottom wall: theta13 and theta23 are the angles of liquids 1 and 2
    against the third fluid (measured inside the liquid); the 1-2 contact line takes the
    angle that Young's law gives with the same wall energies,
    sigma_12 cos theta_12 = sigma_13 cos theta_13 - sigma_23 cos theta_23.  The top wall is
    neutral (90 degrees) and x is periodic.  Proposed where the paper is silent or its
    values do not apply here: equal densities and viscosities (without gravity the
    equilibrium shape depends only on the tensions and the wall angles), viscosity mu,
    mobility 0.05."""
    X, Y = grid(nx, ny)
    x = X - nx / 2.0
    disc = tanh_step(R - np.sqrt(x ** 2 + Y ** 2), eps)
    phi1 = disc * tanh_step(-x, eps)
    phi2 = disc * tanh_step(x, eps)
    phi = np.stack([phi1, phi2, 1.0 - phi1 - phi2])
    c13, c23 = math.cos(math.radians(theta13)), math.cos(math.radians(theta23))
    c12 = (sigma * c13 - sigma * c23) / sigma
    w = np.zeros((4, 3, 3))
    for (p, q), cv in {(0, 2): c13, (1, 2): c23, (0, 1): c12}.items():
        w[YMIN, p, q] = cv
        w[YMIN, q, p] = -cv
    phases = [phase(rho_l=1.0, mu_l=mu), phase(rho_l=1.0, mu_l=mu), phase(rho_l=1.0, mu_l=mu)]
    sig = np.full((3, 3), sigma)
    np.fill_diagonal(sig, 0.0)
    return Case(name=f"janus_drop_{nx}x{ny}_th{theta23:.0f}", nx=nx, ny=ny, N=3, phases=phases, sigma=sig,
                eps=eps, mobility=mobility, bc=(PERIODIC, PERIODIC, WALL, WALL), wet_cos=w, phi=phi,
                T=np.zeros((ny, nx)), meta=dict(R=R, theta13=theta13, theta23=theta23, theta12=math.degrees(
                    math.acos(c12))))


BATCH_SIDES = (128, 192, 256, 384, 512)


def batch_sweep(n_cases=256, seed=4, sides=BATCH_SIDES) -> List[Case]:
    """The batched droplet sweep: n_cases independent sessile drops.  Per case, in draw
    order, four uniforms u0..u3 of the seeded stream: side = sides[floor(5 u0)],
    Ste = U[0.05, 0.5], theta = U[60, 150] deg, T_wall = U[-2, -0.5]; drop radius
    round(0.2 side) as a cap at theta."""
    u = uniform(seed, 4 * n_cases)
    cases = []
    for k in range(n_cases):
        side = sides[min(int(u[4 * k] * len(sides)), len(sides) - 1)]
        ste = 0.05 + 0.45 * u[4 * k + 1]
        theta = 60.0 + 90.0 * u[4 * k + 2]
        T_wall = -2.0 + 1.5 * u[4 * k + 3]
        c = sessile_cap(side, side, float(round(0.2 * side)), theta=theta, ste=ste, T_wall=T_wall,
                        name=f"batch{k:03d}_{side}")
        c.meta.update(side=side, ste=ste, theta=theta, T_wall=T_wall)
        cases.append(c)
    return cases


def small_batch() -> List[Case]:
    """Cases of uneven sizes, boundaries and parameters (all N = 2) for batch tests."""
    return [sessile_cap(48, 40, 14.0, theta=70.0, ste=0.2, T_wall=-1.5),
            film(nx=16, ny=64, h0=32.0),
            periodic_drop(n=37, R=9.0, ny=29),
            sessile_cap(70, 44, 16.0, theta=120.0, ste=0.08, T_wall=-0.7),
            sessile_cap(130, 33, 12.0, theta=95.0, ste=0.4, T_wall=-2.0)]


def impurity_freeze(n=512, ny=None, liquid_top=None, T_wall=-1.0, ste=0.2, lam_ratio=1.0, n_disks=24,
                    r_range=(6, 14), seed=5, T0=0.5, eps=4.0, mobility=0.02, sigma=1e-3) -> Case:
    """Freezing of a pool holding insoluble impurities (Section 4.4), N = 4: freezing
    liquid (phase 0) below y = liquid_top (3/4 of the height), a second fluid (phase 1)
    above, and n_disks seeded, non-overlapping disks of two impurity fluids (phases 2
    and 3, alternating) in the liquid, kept 2 eps from each other, the walls and the
    liquid surface.  Walls on all sides; cold Dirichlet bottom, adiabatic elsewhere.

    lam_ratio = lambda_s / lambda_l of phase 0.  Proposed where the paper is silent:
    upper fluid rho = 1 (as the film problem), impurity conductivities 3 and 1.5 times
    the liquid's, impurity viscosity 10 times, equal surface tensions, start at T0 = 0.5
    (above T_m = 0, so that no cell starts on the liquidus kink of eq. H)."""
    nx, ny = n, (ny or n)
    top = 0.75 * ny if liquid_top is None else liquid_top
    X, Y = grid(nx, ny)
    u = uniform(seed, 8 * n_disks * 64)
    disks, k, gap = [], 0, 2.0 * eps
    while len(disks) < n_disks and k + 3 <= len(u):
        r = r_range[0] + min(int(u[k] * (r_range[1] - r_range[0] + 1)), r_range[1] - r_range[0])
        cxd = r + gap + u[k + 1] * (nx - 2 * (r + gap))
        cyd = r + gap + u[k + 2] * (top - 2 * (r + gap))
        k += 3
        if all(math.hypot(cxd - a, cyd - b) >= r + rr + gap for a, b, rr in disks):
            disks.append((cxd, cyd, r))
    imp = [np.zeros((ny, nx)), np.zeros((ny, nx))]
    for j, (a, b, r) in enumerate(disks):
        imp[j % 2] += tanh_step(r - np.sqrt((X - a) ** 2 + (Y - b) ** 2), eps)
    rest = np.clip(1.0 - imp[0] - imp[1], 0.0, 1.0)
    liq = tanh_step(top - Y, eps)
    phi = np.stack([rest * liq, rest * (1.0 - liq), imp[0], imp[1]])
    lam1 = 0.1
    phases = [phase(rho_l=1.0, rho_s=0.95, mu_l=0.02, lam_l=lam1, lam_s=lam_ratio * lam1,
                    latent=latent_from_stefan(ste)),
              phase(rho_l=1.0, mu_l=0.02, lam_l=lam1),
              phase(rho_l=1.0, mu_l=0.2, lam_l=3.0 * lam1),
              phase(rho_l=1.0, mu_l=0.2, lam_l=1.5 * lam1)]
    sig = np.full((4, 4), sigma)
    np.fill_diagonal(sig, 0.0)
    return Case(name=f"impurity_freeze_{nx}x{ny}", nx=nx, ny=ny, N=4, phases=phases, sigma=sig, eps=eps,
                mobility=mobility, bc=(WALL, WALL, WALL, WALL),
                tbc=(ADIABATIC, ADIABATIC, DIRICHLET, ADIABATIC), T_wall=(0.0, 0.0, T_wall, 0.0),
                phi=phi, T=np.full((ny, nx), T0),
                meta=dict(T_wall=T_wall, ste=ste, lam_ratio=lam_ratio, disks=disks, seed=seed))
