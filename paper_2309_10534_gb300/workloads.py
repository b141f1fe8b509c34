"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds initial conditions (conserved-variable cell averages
in float64, SoA ``[nvar][ny][nx]``) and problem parameters.  It holds none of
the scheme's arithmetic; both the CUDA library and the CPU oracle consume
what it returns.  Random draws use numpy's PCG64 with an explicit seed.

Problems (paper Sec. 5 unless noted):
  * ``advection_1d``  -- density-perturbation advection, Sec. 5.1
  * ``advection_2d``  -- diagonal density advection, Sec. 5.5
  * ``sod``           -- Sod tube, Sec. 5.2 (b)
  * ``lax``           -- Lax tube, Sec. 5.2 (a)
  * ``riemann2d``     -- 2-D Riemann configuration 3, Sec. 5.6 (a), split point
                         a parameter
  * ``viscous_shock_tube`` -- Sec. 5.8
  * ``ensemble_1d``   -- many independent 1-D Riemann problems (seeded)
  * ``isentropic_vortex`` -- smooth periodic vortex (not in the paper; a
                         standard smooth 2-D Euler solution)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Setup:
    dim: int
    nx: int
    ny: int
    lx: float
    ly: float
    W: np.ndarray                      # conserved cell averages [nvar][ny][nx]
    bc: tuple = ("zerograd",) * 4      # x-low, x-high, y-low, y-high
    gamma: float = 1.4
    mu: float = 0.0
    Pr: float = 1.0
    tau: str = "euler"
    cfl: float = 0.5
    t_end: float = 0.0
    name: str = ""
    extra: dict = field(default_factory=dict)
    # state-setting boundary data (bc_in, bc_pre: conserved (rho, rho u,
    # rho v, E); shock_x0, shock_theta, shock_speed), passed to both sides
    bcstate: dict = field(default_factory=dict)
    # scheme parameters the workload prescribes (the paper's settings for
    # that test), passed to both sides
    scheme: dict = field(default_factory=dict)

    @property
    def dx(self):
        return self.lx / self.nx

    @property
    def dy(self):
        return self.ly / self.ny if self.dim == 2 else 1.0

    def problem_kwargs(self):
        return dict(lx=self.lx, ly=self.ly, bc=self.bc, gamma=self.gamma, mu=self.mu, Pr=self.Pr,
                    tau=self.tau, cfl=self.cfl, **self.bcstate, **self.scheme)


def conserved_1d(rho, u, p, gamma):
    rho = np.asarray(rho, dtype=np.float64)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def conserved_2d(rho, u, v, p, gamma):
    rho = np.asarray(rho, dtype=np.float64)
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def advection_1d(n, gamma=1.4):
    """rho = 1 + 0.2 sin(pi x), U = 1, p = 1 on [0, 2], periodic; exact cell
    averages (Sec. 5.1).  The exact solution at time t is the same profile
    shifted by t."""
    x = np.linspace(0.0, 2.0, n + 1)
    dx = 2.0 / n
    rho = 1.0 + 0.2 * (np.cos(np.pi * x[:-1]) - np.cos(np.pi * x[1:])) / (np.pi * dx)
    W = np.stack([rho, rho, 1.0 / (gamma - 1.0) + 0.5 * rho])[:, None, :]
    return Setup(1, n, 1, 2.0, 1.0, W, bc=("periodic",) * 4, gamma=gamma, tau="zero", t_end=2.0,
                 name="advection_1d")


def advection_1d_exact_rho(n, t):
    x = np.linspace(0.0, 2.0, n + 1)
    dx = 2.0 / n
    return 1.0 + 0.2 * (np.cos(np.pi * (x[:-1] - t)) - np.cos(np.pi * (x[1:] - t))) / (np.pi * dx)


def _sin_sum_cellavg(nx, ny, lx, ly, t):
    """Exact cell averages of sin(pi (x + y - t)) on a uniform grid."""
    x = np.linspace(0.0, lx, nx + 1) - t
    y = np.linspace(0.0, ly, ny + 1)
    dx, dy = lx / nx, ly / ny
    X0, Y0 = np.meshgrid(x[:-1], y[:-1])
    X1, Y1 = np.meshgrid(x[1:], y[1:])
    s = (np.sin(np.pi * (X1 + Y0)) - np.sin(np.pi * (X0 + Y0)) - np.sin(np.pi * (X1 + Y1))
         + np.sin(np.pi * (X0 + Y1)))
    return s / (np.pi ** 2 * dx * dy)


def advection_2d(n, gamma=1.4):
    """rho = 1 + 0.2 sin(pi (x + y)), U = V = 1, p = 1 on [0, 2]^2, periodic
    (Sec. 5.5); exact cell averages."""
    rho = 1.0 + 0.2 * _sin_sum_cellavg(n, n, 2.0, 2.0, 0.0)
    W = np.stack([rho, rho, rho, 1.0 / (gamma - 1.0) + rho])
    return Setup(2, n, n, 2.0, 2.0, W, bc=("periodic",) * 4, gamma=gamma, tau="zero", t_end=2.0,
                 name="advection_2d")


def advection_2d_exact_rho(n, t):
    return 1.0 + 0.2 * _sin_sum_cellavg(n, n, 2.0, 2.0, t)


def _riemann_1d(n, left, right, x0=0.5, gamma=1.4, length=1.0):
    """Exact cell averages of a piecewise-constant (rho, u, p) with a jump at x0."""
    edges = np.linspace(0.0, length, n + 1)
    frac_left = np.clip((x0 - edges[:-1]) / (edges[1:] - edges[:-1]), 0.0, 1.0)
    WL = conserved_1d(*left, gamma)
    WR = conserved_1d(*right, gamma)
    return (frac_left[None, :] * WL[:, None] + (1.0 - frac_left[None, :]) * WR[:, None])


def sod(n=400, gamma=1.4):
    """Sod tube: (1, 0, 1) | (0.125, 0, 0.1) at x = 0.5 on [0, 1], t = 0.2."""
    W = _riemann_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, gamma)[:, None, :]
    return Setup(1, n, 1, 1.0, 1.0, W, gamma=gamma, t_end=0.2, name="sod",
                 extra=dict(left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5))


def lax(n=100, gamma=1.4):
    """Lax tube: (0.445, 0.689, 3.528) | (0.5, 0, 0.571) at x = 0.5, t = 0.14."""
    left, right = (0.445, 0.689, 3.528), (0.5, 0.0, 0.571)
    W = _riemann_1d(n, left, right, 0.5, gamma)[:, None, :]
    return Setup(1, n, 1, 1.0, 1.0, W, gamma=gamma, t_end=0.14, name="lax",
                 extra=dict(left=left, right=right, x0=0.5))


def _sine_wave_tube(n, length, x0, left, amp, k, gamma):
    """Cell averages of (rho, u, p) = left for x < x0 and (1 + amp sin(k x),
    0, 1) beyond: a shock running into a density wave."""
    edges = np.linspace(0.0, length, n + 1)
    a, b = edges[:-1], edges[1:]
    h = b - a
    frac = np.clip((x0 - a) / h, 0.0, 1.0)           # fraction left of x0
    lo = np.minimum(np.maximum(a, x0), b)              # wave part [lo, b] (empty left of x0)
    wave_int = (b - lo) + amp * (np.cos(k * lo) - np.cos(k * b)) / k
    WL = conserved_1d(*left, gamma)
    rho = frac * left[0] + wave_int / h
    mom = frac * WL[1]
    E = frac * WL[2] + (1.0 - frac) * (1.0 / (gamma - 1.0))
    return np.stack([rho, mom, E])[:, None, :]


def shu_osher(n=400, gamma=1.4):
    """Shu-Osher shock / density-wave interaction (Sec. 5.3 (a)) on [0, 10]:
    (3.857134, 2.629369, 10.33333) for x < 1, (1 + 0.2 sin 5x, 0, 1) beyond,
    t = 1.8.  Right boundary: zero gradient (the wave there is at rest and
    no signal reaches it by t = 1.8)."""
    left = (3.857134, 2.629369, 10.33333)
    W = _sine_wave_tube(n, 10.0, 1.0, left, 0.2, 5.0, gamma)
    return Setup(1, n, 1, 10.0, 1.0, W, gamma=gamma, t_end=1.8, name="shu_osher")


def titarev_toro(n=1000, gamma=1.4):
    """Titarev-Toro shock / high-frequency wave interaction (Sec. 5.3 (b)) on
    [0, 10]: (1.515695, 0.523346, 1.805) for x < 0.5, (1 + 0.1 sin 20 pi x,
    0, 1) beyond, t = 5."""
    left = (1.515695, 0.523346, 1.805)
    W = _sine_wave_tube(n, 10.0, 0.5, left, 0.1, 20.0 * np.pi, gamma)
    return Setup(1, n, 1, 10.0, 1.0, W, gamma=gamma, t_end=5.0, name="titarev_toro")


def blast_wave(n=400, gamma=1.4):
    """Woodward-Colella interacting blast waves (Sec. 5.4) on [0, 1]: p = 1000,
    0.01, 100 on [0, 0.1), [0.1, 0.9), [0.9, 1], rho = 1, u = 0; reflecting
    ends, t = 0.038."""
    edges = np.linspace(0.0, 1.0, n + 1)
    a, b = edges[:-1], edges[1:]
    h = b - a
    f1 = np.clip((0.1 - a) / h, 0.0, 1.0)
    f3 = np.clip((b - 0.9) / h, 0.0, 1.0)
    f2 = 1.0 - f1 - f3
    E = (1000.0 * f1 + 0.01 * f2 + 100.0 * f3) / (gamma - 1.0)
    W = np.stack([np.ones(n), np.zeros(n), E])[:, None, :]
    return Setup(1, n, 1, 1.0, 1.0, W, bc=("reflect", "reflect", "zerograd", "zerograd"), gamma=gamma,
                 t_end=0.038, name="blast_wave")


RIEMANN_CONFIG3 = {
    # (rho, u, v, p) per quadrant, Sec. 5.6 (a)
    "ll": (0.138, 1.206, 1.206, 0.029),   # x < x0, y < y0
    "lr": (0.5323, 0.0, 1.206, 0.3),      # x >= x0, y < y0
    "ur": (1.5, 0.0, 0.0, 1.5),           # x >= x0, y >= y0
    "ul": (0.5323, 1.206, 0.0, 0.3),      # x < x0, y >= y0
}


RIEMANN_CONFIG6 = {
    # (rho, u, v, p) per quadrant, Sec. 5.6 (b): four contact discontinuities
    "ll": (1.0, -0.75, 0.5, 1.0),
    "lr": (3.0, -0.75, -0.5, 1.0),
    "ur": (1.0, -0.75, -0.5, 1.0),
    "ul": (2.0, 0.75, 0.5, 1.0),
}


def riemann2d(n=1024, ny=None, split=0.8, t_end=0.8, gamma=1.4, config=3, cfl=0.5):
    """Four-quadrant Riemann problem (configuration 3, or 6 with its split at
    0.5) on [0, 1]^2 with exact cell averages (area fractions of each
    quadrant)."""
    ny = n if ny is None else ny
    xe = np.linspace(0.0, 1.0, n + 1)
    ye = np.linspace(0.0, 1.0, ny + 1)
    fx = np.clip((split - xe[:-1]) / (xe[1:] - xe[:-1]), 0.0, 1.0)  # fraction with x < split
    fy = np.clip((split - ye[:-1]) / (ye[1:] - ye[:-1]), 0.0, 1.0)
    FX, FY = np.meshgrid(fx, fy)
    table = RIEMANN_CONFIG3 if config == 3 else RIEMANN_CONFIG6
    W = np.zeros((4, ny, n))
    for key, wx, wy in (("ll", FX, FY), ("lr", 1 - FX, FY), ("ur", 1 - FX, 1 - FY),
                        ("ul", FX, 1 - FY)):
        W += (wx * wy)[None] * conserved_2d(*table[key], gamma)[:, None, None]
    return Setup(2, n, ny, 1.0, 1.0, W, bc=("zerograd",) * 4, gamma=gamma, t_end=t_end, cfl=cfl,
                 name="riemann2d_config%d" % config, extra=dict(split=split))


def riemann2d_config6(n=400, t_end=0.6, cfl=0.8, gamma=1.4):
    """Configuration 6 (Sec. 5.6 (b)): split at (0.5, 0.5), t = 0.6, CFL 0.8."""
    return riemann2d(n, split=0.5, t_end=t_end, gamma=gamma, config=6, cfl=cfl)


def _area_left_of_line(x0, x1, y0, y1, a, c, sub=64):
    """Fraction of the cell [x0, x1] x [y0, y1] with x < a + c y: the exact
    integral over y of the clipped linear fraction, by the midpoint rule on
    sub-intervals split at the two kinks (exact: the integrand is linear
    between kinks)."""
    h = x1 - x0
    f = lambda y: np.clip((a + c * y - x0) / h, 0.0, 1.0)
    # kinks where the line crosses x0 and x1
    ys = [y0, y1]
    if c != 0.0:
        for xk in (x0, x1):
            yk = (xk - a) / c
            if y0 < yk < y1:
                ys.append(yk)
    ys = sorted(ys)
    tot = 0.0
    for ya, yb in zip(ys[:-1], ys[1:]):
        tot += 0.5 * (f(ya) + f(yb)) * (yb - ya)  # linear between kinks: trapezoid is exact
    return tot / (y1 - y0)


DMR_POST = (8.0, 4.125 * np.sqrt(3.0), -4.125, 116.5)  # (rho, u, v, p) behind the shock, Sec. 5.7
DMR_PRE = (1.4, 0.0, 0.0, 1.0)


def double_mach(nx=960, ny=240, t_end=0.2, cfl=0.5, gamma=1.4):
    """Double Mach reflection (Sec. 5.7) on [0, 4] x [0, 1]: a Mach 10 shock
    at 60 degrees to the x-axis through (1/6, 0), post-shock state behind
    it; inflow of the post-shock state on the left, zero gradient on the
    right, the post-shock state on the bottom for x < 1/6 and a reflecting
    wall beyond, the exact moving shock on the top.  Exact cell averages of
    the initial discontinuity."""
    x0, theta, us = 1.0 / 6.0, np.pi / 3.0, 10.0
    c = 1.0 / np.tan(theta)
    dx, dy = 4.0 / nx, 1.0 / ny
    frac = np.empty((ny, nx))
    for j in range(ny):
        for i in range(nx):
            xa, xb, ya, yb = i * dx, (i + 1) * dx, j * dy, (j + 1) * dy
            if xb <= x0 + c * ya:
                frac[j, i] = 1.0
            elif xa >= x0 + c * yb:
                frac[j, i] = 0.0
            else:
                frac[j, i] = _area_left_of_line(xa, xb, ya, yb, x0, c)
    Wpost = conserved_2d(*DMR_POST, gamma)
    Wpre = conserved_2d(*DMR_PRE, gamma)
    W = frac[None] * Wpost[:, None, None] + (1.0 - frac[None]) * Wpre[:, None, None]
    bcstate = dict(bc_in=tuple(float(x) for x in Wpost), bc_pre=tuple(float(x) for x in Wpre),
                   shock_x0=x0, shock_theta=theta, shock_speed=us)
    # Sec. 5.7: TENO-D GKS runs this problem only with C_T > 1e-5 in the
    # tangential reconstruction (no limit in the normal one)
    return Setup(2, nx, ny, 4.0, 1.0, W, bc=("inflow", "zerograd", "wall_after_x0", "moving_shock"),
                 gamma=gamma, cfl=cfl, t_end=t_end, name="double_mach", bcstate=bcstate,
                 scheme=dict(ct1_t=1e-4))


def viscous_shock_tube(nx=2048, ny=1024, Re=200.0, Pr=0.73, gamma=1.4, t_end=1.0, cfl=0.2):
    """Viscous shock tube (Sec. 5.8) on [0,1] x [0,0.5]: (120, 0, 120/gamma) |
    (1.2, 0, 1.2/gamma) at x = 0.5; no-slip adiabatic walls on the left,
    right and bottom, symmetry on the top; mu = 1/Re (constant)."""
    edges = np.linspace(0.0, 1.0, nx + 1)
    fl = np.clip((0.5 - edges[:-1]) / (edges[1:] - edges[:-1]), 0.0, 1.0)
    WL = conserved_2d(120.0, 0.0, 0.0, 120.0 / gamma, gamma)
    WR = conserved_2d(1.2, 0.0, 0.0, 1.2 / gamma, gamma)
    row = fl[None, :] * WL[:, None] + (1 - fl[None, :]) * WR[:, None]
    W = np.repeat(row[:, None, :], ny, axis=1)
    return Setup(2, nx, ny, 1.0, 0.5, W, bc=("noslip", "noslip", "noslip", "symmetry"),
                 gamma=gamma, mu=1.0 / Re, Pr=Pr, tau="ns", cfl=cfl, t_end=t_end,
                 name="viscous_shock_tube", extra=dict(Re=Re))


@dataclass
class Ensemble:
    ncells: np.ndarray     # int32 per problem
    offsets: np.ndarray    # int64 start of each problem in the packed array
    W: np.ndarray          # packed conserved variables [3][sum ncells]
    left: np.ndarray       # (rho, u, p) per problem
    right: np.ndarray
    gamma: float = 1.4
    t_end: float = 0.15
    cfl: float = 0.5


def ensemble_1d(count=4096, seed=2309, nmin=200, nmax=4000, gamma=1.4, t_end=0.15):
    """Independent 1-D Riemann problems on [0, 1] with the jump at 0.5:
    rho, p ~ log-uniform [0.1, 10] and u ~ uniform [-1, 1] per side, cell
    counts uniform in [nmin, nmax]; zero-gradient ends."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ncells = rng.integers(nmin, nmax + 1, size=count).astype(np.int32)
    lr = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(count, 2)))
    lp = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(count, 2)))
    lu = rng.uniform(-1.0, 1.0, size=(count, 2))
    left = np.stack([lr[:, 0], lu[:, 0], lp[:, 0]], axis=1)
    right = np.stack([lr[:, 1], lu[:, 1], lp[:, 1]], axis=1)
    offsets = np.zeros(count + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ncells)
    W = np.zeros((3, int(offsets[-1])))
    for k in range(count):
        W[:, offsets[k]:offsets[k + 1]] = _riemann_1d(int(ncells[k]), tuple(left[k]),
                                                      tuple(right[k]), 0.5, gamma)
    return Ensemble(ncells, offsets[:-1].copy(), W, left, right, gamma, t_end)


def isentropic_vortex(n=512, strength=5.0, center=(5.0, 5.0), length=10.0, gamma=1.4,
                      seed=None, amplitude=1e-3, quad=4, kmax=4):
    """Isentropic vortex on a periodic [0, L]^2 in a (1, 1) mean flow
    (standard smooth Euler test; not from the paper).  Cell averages by
    quad x quad Gauss-Legendre points per cell.  With ``seed`` the initial
    density gets a Gaussian-random perturbation at fixed (u, v, p): a
    periodic Gaussian random field whose Fourier coefficients for wave
    numbers 0 < max(|kx|, |ky|) <= kmax are independent standard normals,
    scaled to an RMS of ``amplitude`` over the cell averages.  It stays
    smooth on the grid (a white-noise field would make TENO-D's stencil
    choice, and so the discrete flow map, non-smooth at the noise level).
    The perturbation is returned in ``extra['delta_rho']``."""
    h = length / n
    gx, gw = np.polynomial.legendre.leggauss(quad)
    gx = 0.5 * gx
    gw = 0.5 * gw
    c = (np.arange(n) + 0.5) * h
    W = np.zeros((4, n, n))
    modes = []
    if seed is not None:
        rng = np.random.Generator(np.random.PCG64(seed))
        for kx in range(-kmax, kmax + 1):
            for ky in range(0, kmax + 1):
                if (ky == 0 and kx <= 0) or max(abs(kx), ky) == 0:
                    continue
                modes.append((kx, ky, rng.standard_normal(), rng.standard_normal()))
    drho = np.zeros((n, n))
    for a in range(quad):
        for b in range(quad):
            X, Y = np.meshgrid(c + gx[a] * h, c + gx[b] * h)
            dxr = X - center[0]
            dyr = Y - center[1]
            r2 = dxr * dxr + dyr * dyr
            du = strength / (2 * math.pi) * np.exp(0.5 * (1 - r2))
            u = 1.0 - du * dyr
            v = 1.0 + du * dxr
            T = 1.0 - (gamma - 1.0) * strength ** 2 / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
            rho = T ** (1.0 / (gamma - 1.0))
            p = rho * T
            W += gw[a] * gw[b] * conserved_2d(rho, u, v, p, gamma)
            for kx, ky, ca, cb in modes:
                ph = 2 * math.pi * (kx * X + ky * Y) / length
                drho += gw[a] * gw[b] * (ca * np.cos(ph) + cb * np.sin(ph))
    extra = {}
    if seed is not None:
        drho *= amplitude / math.sqrt(np.mean(drho * drho))
        rho = W[0]
        u = W[1] / rho
        v = W[2] / rho
        p = (gamma - 1.0) * (W[3] - 0.5 * rho * (u * u + v * v))
        W = conserved_2d(rho + drho, u, v, p, gamma)
        extra["delta_rho"] = drho
    return Setup(2, n, n, length, length, W, bc=("periodic",) * 4, gamma=gamma, tau="zero",
                 t_end=2.0, name="isentropic_vortex", extra=extra)


def random_smooth_2d(nx, ny, seed, gamma=1.4, amp=0.1, modes=3, kmax=3):
    """Seeded smooth periodic state (few Fourier modes per field, wave
    numbers 1..kmax per direction) for parity tests of the smooth branch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)

    def field_(base):
        f = np.full_like(X, base)
        for _ in range(modes):
            kx, ky = rng.integers(1, kmax + 1, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            f += amp * rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return f

    rho = field_(1.0)
    u = field_(0.3)
    v = field_(-0.2)
    p = field_(1.0)
    return conserved_2d(rho, u, v, p, gamma)


def random_rough_2d(nx, ny, seed, gamma=1.4):
    """Seeded piecewise-constant blocks plus noise: exercises every TENO-D
    branch.  Positive density and pressure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bx = rng.integers(2, 6)
    by = rng.integers(2, 6)
    rho = np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=(by, bx)))
    p = np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=(by, bx)))
    u = rng.uniform(-1, 1, size=(by, bx))
    v = rng.uniform(-1, 1, size=(by, bx))
    iy = (np.arange(ny) * by) // ny
    ix = (np.arange(nx) * bx) // nx

    def expand(a):
        return a[iy][:, ix] * (1.0 + 0.02 * rng.standard_normal((ny, nx)))

    return conserved_2d(expand(rho), expand(u) , expand(v), expand(p), gamma)
