"""Seeded synthetic inputs shaped like the test cases of arXiv 2103.02903.

This module only draws parameters and initial data; it holds none of the
multiresolution or lattice-Boltzmann arithmetic.  Both the CUDA path and the
CPU oracle consume what it returns:

* ``config``: a plain dict (scheme name, lattice velocity, relaxation rates,
  physical constants, domain, levels, threshold, boundary conditions);
* ``conserved``: the conserved moments sampled at the centres of the finest
  cells, float64 array ``[ncons, N_J]`` with x fastest (then y).

The paper's own initial states (Lax-Liu configurations, the obstacle set-up)
are not available, so the Riemann states are drawn from a seed; every draw
uses numpy's PCG64 generator.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

SCHEMES = {
    "d1q2_advection": 0,
    "d1q2_burgers": 1,
    "d1q3_shallow_water": 2,
    "d2q4x4_euler": 3,
    "d2q9_ns": 4,
    "d3q6_advection": 5,
}
DIM = {"d1q2_advection": 1, "d1q2_burgers": 1, "d1q3_shallow_water": 1,
       "d2q4x4_euler": 2, "d2q9_ns": 2, "d3q6_advection": 3}
NCONS = {"d1q2_advection": 1, "d1q2_burgers": 1, "d1q3_shallow_water": 2,
         "d2q4x4_euler": 4, "d2q9_ns": 3, "d3q6_advection": 1}
NPOP = {"d1q2_advection": 2, "d1q2_burgers": 2, "d1q3_shallow_water": 3,
        "d2q4x4_euler": 16, "d2q9_ns": 9, "d3q6_advection": 6}
BC = {"periodic": 0, "copy": 1, "bounce_back": 2, "anti_bounce_back": 3,
      "bounce_back_velocity": 4}


def base_config(scheme: str, **kw) -> Dict:
    cfg = dict(scheme=scheme, lambda_=1.0, s=[0.0] * 16, phys=[0.0] * 8,
               xmin=[0.0, 0.0, 0.0], xmax=[1.0, 1.0, 1.0], roots=[1, 1, 1],
               min_level=2, max_level=6, eps=1e-4, mu_bar=0,
               bc=["periodic"] * 6, cross_sign=1, obstacle=0)
    cfg.update(kw)
    return cfg


def finest_shape(cfg: Dict) -> Tuple[int, ...]:
    d = DIM[cfg["scheme"]]
    J = cfg["max_level"]
    return tuple(cfg["roots"][a] << J for a in range(d))


def cell_centres(cfg: Dict):
    """Physical centres of the finest cells, one array per axis (x fastest)."""
    d = DIM[cfg["scheme"]]
    shape = finest_shape(cfg)
    axes = []
    for a in range(d):
        n = shape[a]
        h = (cfg["xmax"][a] - cfg["xmin"][a]) / n
        axes.append(cfg["xmin"][a] + (np.arange(n) + 0.5) * h)
    if d == 1:
        return (axes[0],)
    if d == 2:
        X, Y = np.meshgrid(axes[0], axes[1], indexing="xy")
        return (X.ravel(), Y.ravel())
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")  # x fastest, then y, then z
    return (X.ravel(), Y.ravel(), Z.ravel())


def steps_to(cfg: Dict, T: float) -> int:
    """Number of steps of Algorithm 1 to reach time T (dt = dx / lambda)."""
    dx = (cfg["xmax"][0] - cfg["xmin"][0]) / (cfg["roots"][0] << cfg["max_level"])
    return int(math.ceil(T / (dx / cfg["lambda_"]) - 1e-12))


# --------------------------------------------------------------------------
# D1Q2 linear advection: indicator of [-1, 1] plus a Gaussian bump
# --------------------------------------------------------------------------

def advection_1d(seed: int = 0, max_level: int = 9, min_level: int = 2, eps: float = 1e-4):
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.uniform(-2.5, 2.5)
    cfg = base_config("d1q2_advection", lambda_=1.0, xmin=[-3.0, 0, 0], xmax=[3.0, 1, 1],
                      min_level=min_level, max_level=max_level, eps=eps, mu_bar=0,
                      bc=["periodic"] * 6)
    cfg["s"][0] = 1.0
    cfg["phys"][0] = 0.75
    (x,) = cell_centres(cfg)
    u = ((x >= -1.0) & (x <= 1.0)).astype(np.float64) + np.exp(-((x - c) / 0.2) ** 2)
    return cfg, u[None, :].copy()


# --------------------------------------------------------------------------
# D1Q2 Burgers and D1Q3 shallow water Riemann problems on [-1, 1]
# --------------------------------------------------------------------------

def burgers_1d(seed: int = 0, max_level: int = 12, min_level: int = 2, eps: float = 1e-4):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = float(rng.choice([1.0, 1.5, 1.75]))
    xi = rng.uniform(-1.0, 1.0, size=2)
    uL, uR = 2.0 * (1 + 0.01 * xi[0]), 1.0 * (1 + 0.01 * xi[1])
    cfg = base_config("d1q2_burgers", lambda_=3.0, xmin=[-1.0, 0, 0], xmax=[1.0, 1, 1],
                      min_level=min_level, max_level=max_level, eps=eps, mu_bar=0,
                      bc=["copy"] * 6)
    cfg["s"][0] = s
    (x,) = cell_centres(cfg)
    u = np.where(x < 0.0, uL, uR).astype(np.float64)
    return cfg, u[None, :].copy()


def shallow_water_1d(seed: int = 0, max_level: int = 12, min_level: int = 2, eps: float = 1e-4):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = float(rng.choice([1.0, 1.5, 1.75]))
    xi = rng.uniform(-1.0, 1.0, size=2)
    hL, hR = 2.0 * (1 + 0.01 * xi[0]), 1.0 * (1 + 0.01 * xi[1])
    cfg = base_config("d1q3_shallow_water", lambda_=3.0, xmin=[-1.0, 0, 0], xmax=[1.0, 1, 1],
                      min_level=min_level, max_level=max_level, eps=eps, mu_bar=0,
                      bc=["copy"] * 6)
    cfg["s"][0] = s
    cfg["phys"][0] = 1.0  # gravity
    (x,) = cell_centres(cfg)
    h = np.where(x < 0.0, hL, hR).astype(np.float64)
    q = np.zeros_like(h)
    return cfg, np.stack([h, q])


# --------------------------------------------------------------------------
# D2Q4^4 Euler four-quadrant Riemann problem on [0, 1]^2
# --------------------------------------------------------------------------

def euler_quadrant_states(rng, gamma=1.4, lam=5.0):
    """Four quadrant states (rho, u, v, p): rho, p ~ U[0.5, 1.5] and
    u, v ~ U[0.1, 0.5].  Drawing all four in [0.1, 1.5] gives density and
    pressure contrasts up to 15 for which the D2Q4^4 reference scheme itself
    (lambda = 5, s^q = 1.9 / 1.75) loses positivity within a few dozen steps,
    so the draw is narrowed to states it integrates to T = 0.25."""
    states = []
    for _ in range(4):
        while True:
            rho, p = rng.uniform(0.5, 1.5, size=2)
            u, v = rng.uniform(0.1, 0.5, size=2)
            if max(abs(u), abs(v)) + math.sqrt(gamma * p / rho) <= 0.8 * lam:
                break
        states.append((rho, u, v, p))
    return states  # order: UR, UL, LL, LR


def euler_2d(seed: int = 0, max_level: int = 10, min_level: int = 2, eps: float = 1e-3,
             mu_bar: int = 0):
    rng = np.random.Generator(np.random.PCG64(seed))
    gamma, lam = 1.4, 5.0
    st = euler_quadrant_states(rng, gamma, lam)
    cfg = base_config("d2q4x4_euler", lambda_=lam, xmin=[0.0, 0.0, 0.0], xmax=[1.0, 1.0, 1.0],
                      min_level=min_level, max_level=max_level, eps=eps, mu_bar=mu_bar,
                      bc=["copy"] * 6)
    cfg["s"][0:4] = [1.9, 1.75, 1.75, 1.75]
    cfg["s"][4:8] = [1.0, 1.0, 1.0, 1.0]
    cfg["phys"][0] = gamma
    X, Y = cell_centres(cfg)
    quad = np.where(X > 0.5, np.where(Y > 0.5, 0, 3), np.where(Y > 0.5, 1, 2))
    prim = np.array(st)[quad]  # [N, 4]
    rho, u, v, p = prim.T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return cfg, np.stack([rho, rho * u, rho * v, E]).astype(np.float64)


# --------------------------------------------------------------------------
# D2Q9 flow past a disc on [0, 2] x [0, 1]
# --------------------------------------------------------------------------

def ns_obstacle_2d(seed: int = 0, max_level: int = 10, min_level: int = 2, eps: float = 1e-4,
                   reynolds: float = 1200.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    rho0, u0, lam = 1.0, 0.05, 1.0
    radius = 0.05
    L = math.sqrt(math.pi) * radius
    mu = rho0 * u0 * L / reynolds
    cfg = base_config("d2q9_ns", lambda_=lam, xmin=[0.0, 0.0, 0.0], xmax=[2.0, 1.0, 1.0],
                      roots=[2, 1, 1], min_level=min_level, max_level=max_level, eps=eps, mu_bar=1,
                      bc=["bounce_back_velocity", "copy", "bounce_back_velocity",
                          "bounce_back_velocity", "periodic", "periodic"], obstacle=1)
    dx = 1.0 / (1 << max_level)
    dt = dx / lam
    cs2 = lam * lam / 3.0
    s2 = 1.0 / (0.5 + mu / (cs2 * dt * rho0))
    cfg["s"][0] = 1.5
    cfg["s"][1] = s2
    cfg["phys"][0:6] = [rho0, u0, 0.0, 0.3, 0.5, radius]
    X, Y = cell_centres(cfg)
    a = rng.standard_normal(4)
    dv = 1e-3 * u0 * sum(a[m - 1] * np.sin(m * math.pi * Y) * np.sin(m * math.pi * X / 2.0)
                         for m in range(1, 5))
    rho = np.full_like(X, rho0)
    return cfg, np.stack([rho, rho * u0 * np.ones_like(X), rho * dv]).astype(np.float64)


def vortices_2d(seed: int = 0, max_level: int = 8, min_level: int = 2, eps: float = 1e-4,
                n_vortices: int = 0, bc: str = "periodic"):
    """D2Q9 on the periodic unit square with 2-8 Gaussian (Lamb-Oseen) vortices:
    seeded centres, core radii in [0.02, 0.1], circulations +-U(0.5, 1) * 0.05
    (velocity scale 0.05, lambda = 1), rho = 1; minimum-image distances.
    ``bc`` other than periodic puts that condition on all four faces."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam, rho0, u0 = 1.0, 1.0, 0.05
    cfg = base_config("d2q9_ns", lambda_=lam, min_level=min_level, max_level=max_level, eps=eps,
                      mu_bar=1, bc=[bc] * 4 + ["periodic"] * 2)
    cfg["s"][0] = 1.5
    cfg["s"][1] = 1.8
    cfg["phys"][0:3] = [rho0, 0.0, 0.0]
    X, Y = cell_centres(cfg)
    nv = n_vortices or int(rng.integers(2, 9))
    ux = np.zeros_like(X)
    uy = np.zeros_like(X)
    for _ in range(nv):
        xc, yc = rng.uniform(0.0, 1.0, 2)
        R = rng.uniform(0.02, 0.1)
        gam = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.0) * u0 * 2.0 * math.pi * R
        dx = (X - xc + 0.5) % 1.0 - 0.5
        dy = (Y - yc + 0.5) % 1.0 - 0.5
        r2 = np.maximum(dx * dx + dy * dy, 1e-300)
        ut = gam / (2.0 * math.pi * r2) * (1.0 - np.exp(-r2 / (R * R)))
        ux += -dy * ut
        uy += dx * ut
    rho = np.full_like(X, rho0)
    return cfg, np.stack([rho, rho * ux, rho * uy]).astype(np.float64)


# --------------------------------------------------------------------------
# D3Q6 advection of a ball (Sec. 7.3)
# --------------------------------------------------------------------------

def advection_3d(seed: int = 0, max_level: int = 8, min_level: int = 2, eps: float = 1e-3, mu_bar: int = 2):
    """Indicator of a ball of radius 0.15 on the periodic cube [-0.5, 0.5]^3,
    advected with a constant velocity V: the test of Sec. 7.3 (lambda = 1,
    s1 = 1.4, s2 = 1, mu_bar = 2, eps = 1e-3).  The paper gives neither the
    domain nor V: the ball's centre is drawn within 0.05 of the origin and
    each component of V in [-0.25, 0.25] from the seed.  The equilibria
    u/6 +- V_a u/2 are non-negative only for |V_a| <= lambda / 3, and with
    s1 = 1.4 velocities near lambda / 2 make the scheme blow up within a few
    tens of steps.  J_min = 2 (the paper's 1 is below the library's smallest
    level)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.uniform(-0.05, 0.05, 3)
    V = rng.uniform(-0.25, 0.25, 3)
    s = [0.0] * 16
    s[0], s[1] = 1.4, 1.0
    phys = [0.0] * 8
    phys[0:3] = list(V)
    cfg = base_config("d3q6_advection", lambda_=1.0, xmin=[-0.5, -0.5, -0.5], xmax=[0.5, 0.5, 0.5],
                      min_level=min_level, max_level=max_level, eps=eps, mu_bar=mu_bar,
                      bc=["periodic"] * 6, s=s, phys=phys)
    X, Y, Z = cell_centres(cfg)
    u = (((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) <= 0.15 ** 2).astype(np.float64)
    return cfg, u[None, :]


def serving_batch(seed: int = 0, n: int = 256, levels=(6, 7, 8, 9, 10), eps=(1e-3, 1e-4),
                  precision: str = "fp16"):
    """Independent instances of a batched serving load: half D2Q9 periodic
    vortex flows, half D2Q4^4 four-quadrant Riemann problems, each with a
    finest level drawn from ``levels`` and a threshold from ``eps``.
    Returns a list of (config, conserved)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        J = int(rng.choice(levels))
        e = float(rng.choice(eps))
        s = int(rng.integers(0, 2 ** 31))
        if i % 2 == 0:
            cfg, u = vortices_2d(seed=s, max_level=J, eps=e)
        else:
            cfg, u = euler_2d(seed=s, max_level=J, eps=e)
        cfg["precision"] = precision
        out.append((cfg, u))
    return out


WORKLOADS = {
    "advection_1d": advection_1d,
    "burgers_1d": burgers_1d,
    "shallow_water_1d": shallow_water_1d,
    "euler_2d": euler_2d,
    "ns_obstacle_2d": ns_obstacle_2d,
    "vortices_2d": vortices_2d,
    "advection_3d": advection_3d,
}
