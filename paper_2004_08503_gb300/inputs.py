"""Seeded synthetic initial data shaped like the paper's workloads.

This module serves both the GPU path's tests/benchmark and the oracle's tests.
It holds no step of the method: it only defines initial states as functions of
the node coordinates (x, y) the caller supplies, in conserved variables.  The
conversion from primitive data (rho, v, p) uses the ideal-gas relation
rho E = p/(gamma-1) + rho |v|^2 / 2 that defines those initial states.

Recipes (all float64):
  burgers_pulse      0.5 + sin(2 pi x) sin(2 pi y) + [0.3 <= x <= 0.6 and 0.3 <= y <= 0.6]
  four_quadrant      quadrant split at a seeded point in [0.3,0.7]^2; per quadrant
                     rho ~ U[0.1,1.5], v_x, v_y ~ U[-1,1], p ~ U[0.03,1.5]
                     (draw order x0, y0, then SW, SE, NW, NE each (rho, vx, vy, p));
                     x < x0 is west, x >= x0 east (likewise in y)
  riemann_config12   the paper's printed 2D Riemann data (Sec. 5.6) on [0,1]^2
  blast              rho = 1, v = 0, p = 1e-5 + 1e3 exp(-r^2/0.01^2), r from (1/2,1/2)
  vortex             steady isentropic vortex: T = 1 - A exp(-r^2/(2 s^2)), rho = T^(1/(g-1)),
                     p = rho T, swirl u_theta = r sqrt(g A/((g-1) s^2)) exp(-r^2/(4 s^2))
  sod_x              Sod data (rho,v,p) = (1,0,1) | (1/8,0,1/10) split at x = xs, y-invariant
  sine_advection     sin(2 pi x), y-invariant
  solid_body         Sec. 5.4 rotation data on [0,1]^2: disks of radius 0.15, r normalised by it;
                     bump (1 + cos(pi r))/4 at (0.25,0.5), cone 1 - r at (0.5,0.25), slotted
                     cylinder at (0.5,0.75): 1 where |x - 0.5| >= 0.025 or y >= 0.85, else 0;
                     zero outside the disks.  Rotation velocity (2 pi (1/2 - y), 2 pi (x - 1/2)).
  smooth_bump        cos(pi r/2)^6 on a disk of radius r0 around (xc, yc) (C^5), zero outside
  double_mach        Sec. 5.7 on [0,4] x [0,1]: a Mach 10 shock through (1/6, 0) inclined at 60 degrees
                     to the wall; pre-shock (rho, v, p) = (1.4, 0, 1), post-shock (8, 8.25 (cos 30,
                     -sin 30), 116.5); the shock line at time t is x = 1/6 + (y + 20 t)/sqrt(3)
  batch_shapes       seeded (elements per side, p) pairs of a batch of independent problems

Curved-mesh node coordinates (the caller maps the nodes of a Cartesian mesh; shared face nodes
of neighbouring elements get identical coordinates since they map the same point):
  warped_coords      x = X + eps Lx s, y = Y + eps Ly s, s = sin(2 pi X/Lx) sin(2 pi Y/Ly) on
                     [0,Lx] x [0,Ly] (a periodic displacement; eps <= 0.1 keeps det J > 0)
  rotated_coords     rotation of (X, Y) by theta about (xc, yc)
"""
import numpy as np

GAMMA = 1.4


def _cons(rho, vx, vy, p, gamma=GAMMA):
    return np.stack([rho, rho * vx, rho * vy, p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)])


def burgers_pulse(x, y):
    pulse = ((x >= 0.3) & (x <= 0.6) & (y >= 0.3) & (y <= 0.6)).astype(np.float64)
    return (0.5 + np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) + pulse)[None]


def sine_advection(x, y):
    return np.sin(2 * np.pi * x)[None] + 0.0 * y[None]


def four_quadrant_params(seed):
    rng = np.random.default_rng(seed)
    x0, y0 = rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7)
    quads = []
    for _ in range(4):  # SW, SE, NW, NE
        rho = rng.uniform(0.1, 1.5)
        vx = rng.uniform(-1.0, 1.0)
        vy = rng.uniform(-1.0, 1.0)
        p = rng.uniform(0.03, 1.5)
        quads.append((rho, vx, vy, p))
    return x0, y0, quads


def _quadrants(x, y, x0, y0, quads, gamma):
    east = x >= x0
    north = y >= y0
    q = np.where(north, 2, 0) + np.where(east, 1, 0)
    prim = np.array(quads)  # (4, 4)
    rho, vx, vy, p = (prim[q, k] for k in range(4))
    return _cons(rho, vx, vy, p, gamma)


def four_quadrant(x, y, seed, gamma=GAMMA):
    x0, y0, quads = four_quadrant_params(seed)
    return _quadrants(x, y, x0, y0, quads, gamma)


def riemann_config12(x, y, gamma=GAMMA):
    s = 3.0 / np.sqrt(17.0)
    quads = [(0.8, 0.0, 0.0, 1.0), (1.0, 0.0, s, 1.0), (1.0, s, 0.0, 1.0), (17.0 / 32.0, 0.0, 0.0, 0.4)]
    return _quadrants(x, y, 0.5, 0.5, quads, gamma)


def blast(x, y, gamma=GAMMA):
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    p = 1e-5 + 1e3 * np.exp(-r2 / 0.01 ** 2)
    one = np.ones_like(x)
    return _cons(one, 0.0 * x, 0.0 * x, p, gamma)


def vortex(x, y, gamma=GAMMA, amp=0.1, width=0.1, xc=0.5, yc=0.5):
    dx, dy = x - xc, y - yc
    r2 = dx * dx + dy * dy
    T = 1.0 - amp * np.exp(-r2 / (2 * width ** 2))
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    k = np.sqrt(gamma * amp / ((gamma - 1.0) * width ** 2)) * np.exp(-r2 / (4 * width ** 2))
    return _cons(rho, -dy * k, dx * k, p, gamma)


def sod_x(x, y, xs=0.0, gamma=GAMMA):
    left = x < xs
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return _cons(rho, 0.0 * x, 0.0 * x, p, gamma)


SOLID_BODY_VELOCITY = (np.pi, -2.0 * np.pi, -np.pi, 2.0 * np.pi)  # (bx0, bxy, by0, byx)


def solid_body(x, y):
    r0 = 0.15
    u = np.zeros_like(x, dtype=float)
    r = np.hypot(x - 0.25, y - 0.5) / r0
    u = np.where(r <= 1.0, 0.25 * (1.0 + np.cos(np.pi * np.minimum(r, 1.0))), u)
    r = np.hypot(x - 0.5, y - 0.25) / r0
    u = np.where(r <= 1.0, 1.0 - r, u)
    r = np.hypot(x - 0.5, y - 0.75) / r0
    cyl = np.where((np.abs(x - 0.5) >= 0.025) | (y >= 0.85), 1.0, 0.0)
    u = np.where(r <= 1.0, cyl, u)
    return u[None]


def smooth_bump(x, y, xc=0.5, yc=0.3, r0=0.2):
    r = np.minimum(np.hypot(x - xc, y - yc) / r0, 1.0)
    return (np.cos(0.5 * np.pi * r) ** 6)[None]


DMR_PRE = (1.4, 0.0, 0.0, 1.0)                                          # rho, vx, vy, p
DMR_POST = (8.0, 8.25 * np.cos(np.pi / 6), -8.25 * np.sin(np.pi / 6), 116.5)


def dmr_shock_x(y, t):
    """x of the incident shock at height y and time t (Sec. 5.7)."""
    return 1.0 / 6.0 + (y + 20.0 * t) / np.sqrt(3.0)


def dmr_cons(prim, gamma=GAMMA):
    rho, vx, vy, p = prim
    return np.array([rho, rho * vx, rho * vy, p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)])


def double_mach(x, y, gamma=GAMMA):
    post = x < dmr_shock_x(y, 0.0)
    rho = np.where(post, DMR_POST[0], DMR_PRE[0])
    vx = np.where(post, DMR_POST[1], DMR_PRE[1])
    vy = np.where(post, DMR_POST[2], DMR_PRE[2])
    p = np.where(post, DMR_POST[3], DMR_PRE[3])
    return _cons(rho, vx, vy, p, gamma)


def double_mach_boundaries(gamma=GAMMA):
    """Boundary data of Sec. 5.7 as split-side parameters: west inflow (post-shock), south
    post-shock up to x = 1/6 then a slip wall, north post-shock / pre-shock split at the moving
    shock; the east side is outflow."""
    post, pre = dmr_cons(DMR_POST, gamma), dmr_cons(DMR_PRE, gamma)
    return {
        "W": dict(s0=1e30, speed=0.0, a=post, b=post),
        "S": dict(s0=1.0 / 6.0, speed=0.0, a=post, b=None),
        "N": dict(s0=dmr_shock_x(1.0, 0.0), speed=20.0 / np.sqrt(3.0), a=post, b=pre),
    }


def constant_state(x, y, prim=(0.7, 0.3, -0.2, 0.9), gamma=GAMMA):
    one = np.ones_like(x)
    return _cons(prim[0] * one, prim[1] * one, prim[2] * one, prim[3] * one, gamma)


def batch_shapes(seed, count=512, sides=(8, 16, 32, 64), degrees=(2, 3, 4, 5, 6, 7)):
    rng = np.random.default_rng(seed)
    nel = rng.choice(np.array(sides), size=count)
    ps = rng.choice(np.array(degrees), size=count)
    return [(int(a), int(b)) for a, b in zip(nel, ps)]


def warped_coords(X, Y, eps=0.05, L=(1.0, 1.0)):
    s = np.sin(2.0 * np.pi * X / L[0]) * np.sin(2.0 * np.pi * Y / L[1])
    return X + eps * L[0] * s, Y + eps * L[1] * s


def rotated_coords(X, Y, theta, xc=0.5, yc=0.5):
    c, s = np.cos(theta), np.sin(theta)
    return xc + c * (X - xc) - s * (Y - yc), yc + s * (X - xc) + c * (Y - yc)
