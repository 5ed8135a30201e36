"""Seeded synthetic problem data for the 2-D stochastic minimum-time problem.

This module is shared by the FP64 oracle tests, the GPU tests and ``bench.py``.
It holds only the *data* of a problem instance -- grid geometry, speed field,
target / obstacle mask, the boundary sectors Gamma_p and the discretised
control set -- never any step of the solution method (no interpolation, no
value iteration, no synthesis, no labelling).  Both the oracle and the CUDA
path receive these arrays as inputs.

Conventions (shared by every consumer):
  * n nodes per side on [-1, 1]^2, dx = 2/(n-1), node (i, j) sits at
    (-1 + i*dx, -1 + j*dx); arrays are row-major with i fastest, k = j*n + i.
  * speed: float32 (n*n), the scalar c(x) of the dynamics f(x, a) = c(x) a
    (Section 5, dynamics B).
  * drift: optional float32 (n*n*2), interleaved (bx, by), the control-free
    part b(x) of f(x, a) = b(x) + c(x) a (dynamics A and C of Section 5).
  * mask: uint8 (n*n): 0 free, 1 target (u = g = 0), 2 obstacle.
  * sector: int8 (n*n): the boundary subset Gamma_p a target node belongs
    to (0..N_P-1), -1 for every other node.
  * controls: float64 (N_A, 2): the points discretising the control set A.
  * general terms (Section 5.3), all optional: sigma_field float32 (n*n), the
    diffusion sigma(x) per node (replacing the constant sigma); diffusion 0 for
    sigma(x) I_2, 1 for sigma(x) a (a one-dimensional Wiener process along the
    control); cost_field float32 (n*n), l(x) per node (replacing the constant
    cost); control_cost float64 (N_A), m(a_m): the running cost is l(x) + m(a).
    sigma is in the units of the points x + h f +- sqrt(2h) sigma e_k, so the
    paper's sqrt(2 eps) I_2 is sigma = sqrt(eps).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

MASK_FREE = 0
MASK_TARGET = 1
MASK_OBSTACLE = 2


def node_coords(n: int) -> Tuple[np.ndarray, float]:
    """1-D node coordinates of the uniform grid on [-1, 1] and its step dx."""
    if n < 3:
        raise ValueError("n must be >= 3")
    dx = 2.0 / (n - 1)
    # (2i - (n-1)) / (n-1) is exactly antisymmetric about the centre node, so
    # symmetric data (discs, even speed fields) stay bit-symmetric.
    i = np.arange(n, dtype=np.float64)
    return (2.0 * i - (n - 1)) / (n - 1), dx


def mesh(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """2-D coordinate arrays X1, X2 of shape (n, n) indexed [j, i]."""
    x, _ = node_coords(n)
    X1, X2 = np.meshgrid(x, x, indexing="xy")
    return X1, X2


def control_set(n_controls: int, phase: float = 0.0) -> np.ndarray:
    """N_A unit directions a_j = (cos(2 pi j/N_A + phase), sin(...)), float64 (N_A, 2)."""
    if n_controls < 1:
        raise ValueError("n_controls must be >= 1")
    t = 2.0 * math.pi * np.arange(n_controls, dtype=np.float64) / n_controls + phase
    return np.stack([np.cos(t), np.sin(t)], axis=1)


# ----------------------------------------------------------------- speed fields

def speed_constant(n: int, c: float = 1.0) -> np.ndarray:
    return np.full(n * n, c, dtype=np.float32)


def speed_sine(n: int, amplitude: float = 0.5, freq: float = 2.0 * math.pi) -> np.ndarray:
    """c(x) = 1 + 0.5 sin(2 pi x1) sin(2 pi x2), evaluated in FP64, stored FP32."""
    X1, X2 = mesh(n)
    c = 1.0 + amplitude * np.sin(freq * X1) * np.sin(freq * X2)
    return c.astype(np.float32).reshape(-1)


def speed_halfplane(n: int, c_left: float = 1.0, c_right: float = 2.0) -> np.ndarray:
    """c(x) = c_left + (c_right - c_left) * chi{x1 >= 0} (Section 5, Table 0 case B)."""
    X1, _ = mesh(n)
    c = np.where(X1 >= 0.0, c_right, c_left)
    return c.astype(np.float32).reshape(-1)


def speed_fourier(n: int, rng: np.random.Generator, n_modes: int = 8,
                  lo: float = 0.2, hi: float = 1.8) -> np.ndarray:
    """Random Fourier speed field: clip(1 + 0.5 sum_m A_m cos(pi(k1 x1 + k2 x2) + phi_m), lo, hi).

    A_m ~ U[-1, 1], k1, k2 ~ U{1..4}, phi_m ~ U[0, 2 pi), all from ``rng``.
    """
    X1, X2 = mesh(n)
    amp = rng.uniform(-1.0, 1.0, n_modes)
    k1 = rng.integers(1, 5, n_modes)
    k2 = rng.integers(1, 5, n_modes)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_modes)
    s = np.zeros_like(X1)
    for m in range(n_modes):
        s += amp[m] * np.cos(math.pi * (k1[m] * X1 + k2[m] * X2) + phi[m])
    c = np.clip(1.0 + 0.5 * s, lo, hi)
    return c.astype(np.float32).reshape(-1)


# ------------------------------------------------------------- masks / sectors

def disc_target(n: int, centres: Sequence[Tuple[float, float]],
                radii: Sequence[float]) -> np.ndarray:
    """mask with 1 on nodes inside any closed disc |x - c| <= r, 0 elsewhere."""
    X1, X2 = mesh(n)
    m = np.zeros((n, n), dtype=bool)
    for (cx, cy), r in zip(centres, radii):
        m |= (X1 - cx) ** 2 + (X2 - cy) ** 2 <= r * r
    return m.astype(np.uint8).reshape(-1)


def square_boundary_target(n: int) -> np.ndarray:
    """mask with 1 on the nodes of the boundary of the square (exit problem)."""
    m = np.zeros((n, n), dtype=np.uint8)
    m[0, :] = m[-1, :] = m[:, 0] = m[:, -1] = 1
    return m.reshape(-1)


def add_rect_obstacles(n: int, mask: np.ndarray,
                       rects: Sequence[Tuple[float, float, float, float]]) -> np.ndarray:
    """Mark nodes inside axis-aligned rectangles (x0, y0, x1, y1) as obstacles (2),
    leaving target nodes untouched."""
    X1, X2 = mesh(n)
    out = mask.copy().reshape(n, n)
    for (x0, y0, x1, y1) in rects:
        inside = (X1 >= x0) & (X1 <= x1) & (X2 >= y0) & (X2 <= y1)
        out[inside & (out == MASK_FREE)] = MASK_OBSTACLE
    return out.reshape(-1)


def sectors_about_centres(n: int, mask: np.ndarray,
                          centres: Sequence[Tuple[float, float]],
                          n_patches: int) -> np.ndarray:
    """Split the target nodes into N_P angular sectors about the nearest disc centre.

    sector = floor(N_P * (atan2(y - cy, x - cx) + pi) / (2 pi)) mod N_P on target
    nodes, -1 elsewhere.  This is the partition of the target boundary into the
    subsets Gamma_p from which the patches are grown.
    """
    X1, X2 = mesh(n)
    sec = np.full((n, n), -1, dtype=np.int8)
    tgt = mask.reshape(n, n) == MASK_TARGET
    cs = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    d2 = np.stack([(X1 - c[0]) ** 2 + (X2 - c[1]) ** 2 for c in cs], axis=0)
    near = np.argmin(d2, axis=0)
    cx = cs[near, 0]
    cy = cs[near, 1]
    ang = np.arctan2(X2 - cy, X1 - cx)
    s = np.floor(n_patches * (ang + math.pi) / (2.0 * math.pi)).astype(np.int64) % n_patches
    sec[tgt] = s[tgt].astype(np.int8)
    return sec.reshape(-1)


def sectors_square_sides(n: int, mask: np.ndarray) -> np.ndarray:
    """Sectors 0..3 = bottom, right, top, left side of the square (corners go to
    the first side listed that contains them); -1 on non-target nodes."""
    sec = np.full((n, n), -1, dtype=np.int8)
    sec[:, 0] = 3
    sec[-1, :] = 2
    sec[:, -1] = 1
    sec[0, :] = 0
    sec[mask.reshape(n, n) != MASK_TARGET] = -1
    return sec.reshape(-1)


# ----------------------------------------------------------------- instances

@dataclasses.dataclass
class Instance:
    """One problem instance: the statement's data plus the discretisation knobs."""
    n: int
    controls: np.ndarray            # float64 (N_A, 2)
    speed: np.ndarray               # float32 (n*n)
    mask: np.ndarray                # uint8 (n*n)
    sector: np.ndarray              # int8 (n*n)
    h: float = 0.0                  # <= 0 means h = dx
    lam: float = 1.0                # discount rate lambda
    sigma: float = 0.0              # diffusion, displacement sqrt(2h)*sigma per axis
    coarse_n: int = 0               # 0: no coarse grid
    n_patches: int = 1
    cost: float = 1.0               # running cost l
    drift: Optional[np.ndarray] = None   # float32 (n*n*2) or None
    name: str = ""
    sigma_field: Optional[np.ndarray] = None    # float32 (n*n): sigma(x), or None
    diffusion: int = 0                          # 0: sigma(x) I_2, 1: sigma(x) a
    cost_field: Optional[np.ndarray] = None     # float32 (n*n): l(x), or None
    control_cost: Optional[np.ndarray] = None   # float64 (N_A): m(a_m), or None

    @property
    def dx(self) -> float:
        return 2.0 / (self.n - 1)

    @property
    def h_eff(self) -> float:
        return self.h if self.h > 0 else self.dx

    @property
    def n_controls(self) -> int:
        return int(self.controls.shape[0])


def disc_instance(n: int, sigma: float, *, n_controls: int = 32, lam: float = 1.0,
                  speed: Optional[np.ndarray] = None, radius: float = 0.1,
                  centre: Tuple[float, float] = (0.0, 0.0), coarse_n: int = 0,
                  n_patches: int = 16, h: float = 0.0, name: str = "") -> Instance:
    """Discounted problem with one target disc and projected (reflecting) outer boundary."""
    mask = disc_target(n, [centre], [radius])
    sec = sectors_about_centres(n, mask, [centre], n_patches)
    if speed is None:
        speed = speed_constant(n, 1.0)
    return Instance(n=n, controls=control_set(n_controls), speed=speed, mask=mask,
                    sector=sec, h=h, lam=lam, sigma=sigma, coarse_n=coarse_n,
                    n_patches=n_patches, name=name)


def plain_101() -> Instance:
    """The plain full-grid FP64 workload: 101^2 grid (dx = 0.02), c = 1, sigma = 0.05,
    lambda = 1, h = dx, 32 controls, target disc |x| <= 0.1."""
    return disc_instance(101, 0.05, n_controls=32, lam=1.0, n_patches=16,
                         name="plain-101x101-sigma0.05")


def patchy_1025(sigma: float, n: int = 1025, coarse_n: int = 129,
                n_patches: int = 16) -> Instance:
    """The patchy workload: c = 1 + 0.5 sin(2 pi x1) sin(2 pi x2), target disc |x| <= 0.1,
    32 controls, lambda = 1, h = dx, coarse 129^2, 16 sectors.  Smaller n (with
    (n-1) divisible by (coarse_n-1)) gives the same workload at test sizes."""
    return disc_instance(n, sigma, n_controls=32, lam=1.0, speed=speed_sine(n),
                         coarse_n=coarse_n, n_patches=n_patches,
                         name=f"patchy-{n}x{n}-sigma{sigma:g}")


def batched_instance(seed: int, n: Optional[int] = None) -> Instance:
    """One instance of the many-instance workload: n = 8k + 1 with k ~ U{8..64}
    (65 <= n <= 513, so the coarse grid (n-1)/4 + 1 nests with ratio 4),
    random Fourier speed clipped to [0.2, 1.8], 1-3 target discs of radius
    0.05-0.15, sigma ~ U[0, 0.1], lambda ~ U[0.5, 2], 32 controls, 4-16 patches."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    if n is None:
        n = int(rng.integers(8, 65)) * 8 + 1
    speed = speed_fourier(n, rng)
    k = int(rng.integers(1, 4))
    centres = [tuple(rng.uniform(-0.7, 0.7, 2)) for _ in range(k)]
    radii = list(rng.uniform(0.05, 0.15, k))
    mask = disc_target(n, centres, radii)
    n_p = int(rng.integers(4, 17))
    sec = sectors_about_centres(n, mask, centres, n_p)
    sigma = float(rng.uniform(0.0, 0.1))
    lam = float(rng.uniform(0.5, 2.0))
    coarse = min(129, (n - 1) // 4 + 1)
    while (n - 1) % (coarse - 1) != 0:
        coarse -= 1
    return Instance(n=n, controls=control_set(32), speed=speed, mask=mask, sector=sec,
                    lam=lam, sigma=sigma, coarse_n=coarse, n_patches=n_p,
                    name=f"batched-seed{seed}-n{n}")


def large_instance(seed: int = 5000, n: int = 4097, coarse_n: int = 129,
                   n_patches: int = 64, sigma: float = 0.01, n_obstacles: int = 6) -> Instance:
    """The large workload: n = 4097, random Fourier speed clipped to [0.2, 1.8],
    64 controls, sigma = 0.01, lambda = 1, h = dx, target disc |x| <= 0.1,
    6 seeded axis-aligned rectangular obstacles (sides 0.08-0.35, at least 0.25
    from the origin; speed 0 there, nodes held at the obstacle value), 64 sectors.
    Smaller n (with (n-1) divisible by (coarse_n-1)) gives the same recipe at
    test sizes."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    speed = speed_fourier(n, rng)
    mask = disc_target(n, [(0.0, 0.0)], [0.1])
    rects = []
    while len(rects) < n_obstacles:
        w, hh = rng.uniform(0.08, 0.35, 2)
        cx, cy = rng.uniform(-0.85, 0.85, 2)
        gx = max(abs(cx) - w / 2, 0.0)
        gy = max(abs(cy) - hh / 2, 0.0)
        if math.hypot(gx, gy) < 0.25:
            continue
        rects.append((cx - w / 2, cy - hh / 2, cx + w / 2, cy + hh / 2))
    mask = add_rect_obstacles(n, mask, rects)
    speed = speed.copy()
    speed[mask == MASK_OBSTACLE] = 0.0
    sec = sectors_about_centres(n, mask, [(0.0, 0.0)], n_patches)
    return Instance(n=n, controls=control_set(64), speed=speed, mask=mask, sector=sec,
                    lam=1.0, sigma=sigma, coarse_n=coarse_n, n_patches=n_patches,
                    name=f"large-seed{seed}-n{n}")


def warmstart_instance(seed: int, n: int = 257, coarse_n: int = 129) -> Instance:
    """One instance of the warm-start training / evaluation recipe: 257^2 fine grid
    with a 129^2 coarse grid, random Fourier speed clipped to [0.2, 1.8], 1-3
    target discs of radius 0.05-0.15, 0-4 seeded rectangular obstacles (sides
    0.1-0.4, speed 0, clear of the discs), sigma ~ U[0, 0.1], lambda ~ U[0.5, 2],
    32 controls, 4-16 patches."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    speed = speed_fourier(n, rng)
    k = int(rng.integers(1, 4))
    centres = [tuple(rng.uniform(-0.7, 0.7, 2)) for _ in range(k)]
    radii = list(rng.uniform(0.05, 0.15, k))
    mask = disc_target(n, centres, radii)
    rects = []
    n_obst = int(rng.integers(0, 5))
    while len(rects) < n_obst:
        w, hh = rng.uniform(0.1, 0.4, 2)
        cx, cy = rng.uniform(-0.8, 0.8, 2)
        r = (cx - w / 2, cy - hh / 2, cx + w / 2, cy + hh / 2)
        clear = all(math.hypot(max(abs(cx - c[0]) - w / 2, 0.0), max(abs(cy - c[1]) - hh / 2, 0.0)) > rad + 0.05
                    for c, rad in zip(centres, radii))
        if clear:
            rects.append(r)
    mask = add_rect_obstacles(n, mask, rects)
    speed = speed.copy()
    speed[mask == MASK_OBSTACLE] = 0.0
    n_p = int(rng.integers(4, 17))
    sec = sectors_about_centres(n, mask, centres, n_p)
    sigma = float(rng.uniform(0.0, 0.1))
    lam = float(rng.uniform(0.5, 2.0))
    return Instance(n=n, controls=control_set(32), speed=speed, mask=mask, sector=sec, lam=lam,
                    sigma=sigma, coarse_n=coarse_n, n_patches=n_p, name=f"warmstart-seed{seed}-n{n}")


def random_values(n: int, seed: int, lo: float = 0.0, hi: float = 1.0,
                  mask: Optional[np.ndarray] = None) -> np.ndarray:
    """A seeded random value field (float64, n*n) for operator-level tests; target
    nodes are set to 0 when a mask is given."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    u = rng.uniform(lo, hi, n * n)
    if mask is not None:
        u[mask == MASK_TARGET] = 0.0
    return u


# ------------------------------------------------ the problems of Section 5

def h_upper_bound(n: int, f_max: float, eps: float, theta: float = 0.9) -> float:
    """The time step with h f_max + sqrt(2 eps h) = theta dx (the bound of
    Section 4.1 that keeps every point in the first neighbouring cells)."""
    dx = 2.0 / (n - 1)
    if f_max <= 0.0:
        return (theta * dx) ** 2 / (2.0 * eps)
    b = math.sqrt(2.0 * eps)
    q = (-b + math.sqrt(b * b + 4.0 * f_max * theta * dx)) / (2.0 * f_max)
    return q * q


def boundary_instance(n: int, speed: np.ndarray, *, n_controls: int = 16, h: float = 0.0,
                      lam: float = 0.0, sigma: float = 0.0, drift: Optional[np.ndarray] = None,
                      coarse_n: int = 0, name: str = "", **general) -> Instance:
    """Exit-time problem of Section 5: target = the boundary of the square (u = g = 0
    there), the four sides as the boundary subsets Gamma_p, N_A unit directions,
    undiscounted unless lam > 0."""
    mask = square_boundary_target(n)
    return Instance(n=n, controls=control_set(n_controls), speed=speed, mask=mask,
                    sector=sectors_square_sides(n, mask), h=h, lam=lam, sigma=sigma,
                    coarse_n=coarse_n, n_patches=4, drift=drift, name=name, **general)


def speed_general(n: int) -> np.ndarray:
    """c(x) = 1 + max{x2, max{x1, 0}} (eq. nonomog)."""
    X1, X2 = mesh(n)
    return (1.0 + np.maximum(X2, np.maximum(X1, 0.0))).astype(np.float32).reshape(-1)


def upper_half(n: int) -> np.ndarray:
    """chi_{x2 >= 0} per node (float64)."""
    _, X2 = mesh(n)
    return (X2 >= 0.0).astype(np.float64).reshape(-1)


def general_instance(n: int, sigma_kind: int, cost_kind: int, *, eps: float = 0.1,
                     n_controls: int = 16, coarse_n: int = 0, h: float = 0.0) -> Instance:
    """The general nonlinear problems of Section 5.3: f = c(x) a with c of eq.
    nonomog, d_eps(x) = sqrt(2 eps) chi_{x2 >= 0}, diffusion sigma_1 = 0,
    sigma_2 = d_eps I_2 or sigma_3 = d_eps a (eq. s123), running cost l_1 = 1,
    l_2 = 1 + |x1 x2| or l_3 = l_2 + |a1 / (2 + a2)| (eq. l123); boundary target,
    no discount.  h defaults to the Section 4.1 bound with f_max = 2."""
    if sigma_kind not in (1, 2, 3) or cost_kind not in (1, 2, 3):
        raise ValueError("sigma_kind and cost_kind are 1, 2 or 3")
    if h <= 0.0:
        h = h_upper_bound(n, 2.0, eps)
    X1, X2 = mesh(n)
    gen = {}
    if sigma_kind > 1:
        gen["sigma_field"] = (math.sqrt(eps) * upper_half(n)).astype(np.float32)
        gen["diffusion"] = 0 if sigma_kind == 2 else 1
    if cost_kind > 1:
        gen["cost_field"] = (1.0 + np.abs(X1 * X2)).astype(np.float32).reshape(-1)
    if cost_kind == 3:
        a = control_set(n_controls)
        gen["control_cost"] = np.abs(a[:, 0] / (2.0 + a[:, 1]))
    return boundary_instance(n, speed_general(n), n_controls=n_controls, h=h, coarse_n=coarse_n,
                             name=f"general-l{cost_kind}-sigma{sigma_kind}-n{n}", **gen)


def degenerate_instance(n: int, *, eps: float = 0.1, n_controls: int = 16, coarse_n: int = 0,
                        h: float = 0.0) -> Instance:
    """Degenerate diffusion of Section 5.2: eps(x) = 0.1 chi_{x2 >= 0} (sigma(x) =
    sqrt(eps(x)) I_2 in the units above), speed c = 1 + chi_{x1 >= 0}, l = 1,
    boundary target, no discount."""
    if h <= 0.0:
        h = h_upper_bound(n, 2.0, eps)
    return boundary_instance(n, speed_halfplane(n, 1.0, 2.0), n_controls=n_controls, h=h,
                             coarse_n=coarse_n, name=f"degenerate-n{n}",
                             sigma_field=(math.sqrt(eps) * upper_half(n)).astype(np.float32))


def zermelo_fields(n: int, eta: float, theta: float) -> Tuple[np.ndarray, np.ndarray]:
    """f(x, a) = (R_theta x/|x| + (eta/2) a) / (1 + |x|^2) (dynamics C) as the drift
    b(x) = R_theta x/|x| / (1 + |x|^2) (0 at the origin) and the speed
    c(x) = (eta/2) / (1 + |x|^2)."""
    X1, X2 = mesh(n)
    r = np.hypot(X1, X2)
    q = 1.0 / (1.0 + r * r)
    inv = np.where(r > 0.0, 1.0 / np.where(r > 0.0, r, 1.0), 0.0)
    ct, st = math.cos(theta), math.sin(theta)
    bx = (ct * X1 - st * X2) * inv * q
    by = (st * X1 + ct * X2) * inv * q
    drift = np.stack([bx.reshape(-1), by.reshape(-1)], axis=1).astype(np.float32).reshape(-1)
    speed = (0.5 * eta * q).astype(np.float32).reshape(-1)
    return speed, drift


def zermelo_instance(n: int, *, eta: float = 1.0, eps: float = 0.1, theta: float = math.pi / 4,
                     n_controls: int = 16, coarse_n: int = 0, h: float = 0.0) -> Instance:
    """The Zermelo navigation problem of Section 5.2 (dynamics C) with uniform
    diffusion eps (sigma = sqrt(eps)), l = 1, boundary target, no discount.
    |f| <= 1 + eta/2; h defaults to the Section 4.1 bound."""
    speed, drift = zermelo_fields(n, eta, theta)
    if h <= 0.0:
        h = h_upper_bound(n, 1.0 + 0.5 * eta, max(eps, 1e-300)) if eps > 0 else 0.9 * (2.0 / (n - 1)) / (1.0 + 0.5 * eta)
    return boundary_instance(n, speed, n_controls=n_controls, h=h, sigma=math.sqrt(eps), drift=drift,
                             coarse_n=coarse_n, name=f"zermelo-eta{eta:g}-eps{eps:g}-n{n}")


TABLE0_ROWS = [("A", 0.0), ("A", 1e-2), ("B1", 0.0), ("B1", 1e-2), ("Bchi", 0.0), ("Bchi", 1e-2),
               ("C", 0.0), ("C", 1e-2)]


def table0_instance(dynamics: str, eps: float, n: int = 50, n_controls: int = 16,
                    theta: float = math.pi / 4) -> Instance:
    """One row of Table 0 on the n x n grid: dynamics A (b = (1, 0)), B1 (c = 1),
    Bchi (c = 1 + chi_{x1 >= 0}) or C (Zermelo, eta = 1), diffusion eps,
    boundary target, no discount, h = dx / 2."""
    h = 0.5 * 2.0 / (n - 1)
    drift = None
    if dynamics == "A":
        speed = speed_constant(n, 0.0)
        drift = np.tile(np.array([1.0, 0.0], np.float32), n * n)
    elif dynamics == "B1":
        speed = speed_constant(n, 1.0)
    elif dynamics == "Bchi":
        speed = speed_halfplane(n, 1.0, 2.0)
    elif dynamics == "C":
        speed, drift = zermelo_fields(n, 1.0, theta)
    else:
        raise ValueError(dynamics)
    return boundary_instance(n, speed, n_controls=n_controls, h=h, sigma=math.sqrt(eps), drift=drift,
                             name=f"table0-{dynamics}-eps{eps:g}-n{n}")

