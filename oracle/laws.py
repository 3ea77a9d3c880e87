"""Physical laws of the oracle (test infrastructure only), float64 numpy.

States are arrays of shape (nc, ...).  Every law provides
  flux(u)              -> (Fx, Fy), each (nc, ...)       flux F(u) of Eq. (cons-law)
  lam(uL, uR, nx, ny)  -> upper bound of the maximum wave speed lambda_max of the
                          1D Riemann problem Eq. (riemann-problem) with u^- = uL,
                          u^+ = uR along the unit normal (nx, ny) (Sec. 2.1.1)

Euler also provides the pressure (Eq. euler-eos), the entropy function
sigma = rho e / rho^gamma (s = log(sigma)/(gamma-1), Sec. 4.3) and psi_K.
"""
import numpy as np


class Advection:
    """Linear advection u_t + div(beta u) = 0 with constant beta (Sec. 3.3, constant case)."""

    nc = 1
    name = "advection"

    def __init__(self, beta=(1.0, 0.0)):
        self.bx, self.by = float(beta[0]), float(beta[1])

    def flux(self, u):
        return self.bx * u, self.by * u

    def lam(self, uL, uR, nx, ny):
        # The Riemann problem is linear with the single speed beta.n.
        return np.abs(self.bx * nx + self.by * ny) * np.ones_like(uL[0])


class AdvectionVar:
    """Linear advection u_t + div(beta(x) u) = 0 with the divergence-free affine velocity
    beta = (bx0 + bxy y, by0 + byx x) (Sec. 3.3; solid body rotation of Sec. 5.4 is
    bx0 = pi, bxy = -2 pi, by0 = -pi, byx = 2 pi).  Each component is constant along its own
    direction, so beta.n is continuous across every face of a Cartesian mesh."""

    nc = 1
    name = "advection_var"

    def __init__(self, bx0=0.0, bxy=0.0, by0=0.0, byx=0.0):
        self.bx0, self.bxy, self.by0, self.byx = float(bx0), float(bxy), float(by0), float(byx)

    def velocity(self, X, Y):
        return self.bx0 + self.bxy * Y, self.by0 + self.byx * X


class Burgers:
    """2D Burgers f(u) = u^2/2 (1,1) (Sec. 5.5, velocity vector (1,1))."""

    nc = 1
    name = "burgers"

    def flux(self, u):
        f = 0.5 * u * u
        return f, f.copy()

    def lam(self, uL, uR, nx, ny):
        # F.n = (nx+ny) u^2/2 is convex in u; its characteristic speed (nx+ny) u is
        # monotone, so the largest |speed| over the fan is attained at an end state.
        return np.abs(nx + ny) * np.maximum(np.abs(uL[0]), np.abs(uR[0]))


class Euler:
    """2D compressible Euler, conserved variables (rho, rho v_x, rho v_y, rho E) (Sec. 4.3)."""

    nc = 4
    name = "euler"

    def __init__(self, gamma=1.4):
        self.gamma = float(gamma)

    def pressure(self, u):
        """Eq. (euler-eos): p = (gamma-1) (rho E - |rho v|^2 / (2 rho))."""
        rho, mx, my, E = u
        return (self.gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)

    def flux(self, u):
        """Eq. (euler-flux): F = (rho v, rho v v^T + p I, rho H v), rho H = rho E + p."""
        rho, mx, my, E = u
        p = self.pressure(u)
        vx, vy = mx / rho, my / rho
        Fx = np.stack([mx, mx * vx + p, my * vx, (E + p) * vx])
        Fy = np.stack([my, mx * vy, my * vy + p, (E + p) * vy])
        return Fx, Fy

    def lam(self, uL, uR, nx, ny):
        """Guaranteed upper bound of lambda_max for 1 < gamma <= 5/3.

        The paper only asks for an upper bound (Sec. 2.1.1) and cites Guermond & Popov.
        This is their two-rarefaction estimate: the two-rarefaction pressure p_TR is an
        upper bound of the star pressure, and the extreme wave speeds grow with it.
        """
        g = self.gamma
        rL, rR = uL[0], uR[0]
        unL = (uL[1] * nx + uL[2] * ny) / rL
        unR = (uR[1] * nx + uR[2] * ny) / rR
        pL, pR = self.pressure(uL), self.pressure(uR)
        aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
        e = (g - 1.0) / (2.0 * g)
        num = np.maximum(aL + aR - 0.5 * (g - 1.0) * (unR - unL), 0.0)
        den = aL * pL ** (-e) + aR * pR ** (-e)
        pstar = (num / den) ** (1.0 / e)
        c = (g + 1.0) / (2.0 * g)
        lamL = unL - aL * np.sqrt(1.0 + c * np.maximum(pstar - pL, 0.0) / pL)
        lamR = unR + aR * np.sqrt(1.0 + c * np.maximum(pstar - pR, 0.0) / pR)
        return np.maximum(np.abs(lamL), np.abs(lamR))

    def sigma(self, u):
        """sigma = rho e rho^-gamma, with s = log(e^{1/(gamma-1)} / rho) = log(sigma)/(gamma-1)."""
        rho, mx, my, E = u
        rhoe = E - 0.5 * (mx * mx + my * my) / rho
        return rhoe * rho ** (-self.gamma)

    def entropy(self, u):
        """Specific entropy s of Sec. 4.3."""
        return np.log(self.sigma(u)) / (self.gamma - 1.0)

    def psi(self, u, K):
        """psi_K(u) = rho e - K rho^gamma.  For rho > 0: psi >= 0 <=> sigma(u) >= K <=> s >= s_min.

        psi is concave in the conserved variables (rho e is concave, rho^gamma convex).
        """
        rho, mx, my, E = u
        return E - 0.5 * (mx * mx + my * my) / rho - K * np.abs(rho) ** self.gamma

    def prim_to_cons(self, rho, vx, vy, p):
        return np.stack([rho, rho * vx, rho * vy, p / (self.gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)])
