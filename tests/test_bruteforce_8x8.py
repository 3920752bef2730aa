"""Brute-force direct check of the oracle on 8 x 8 grids: a second, independent statement of one
time step written with NumPy from the paper's equations as printed, in distribution space, with
no Chapman-Enskog reduction and no moment-space shortcut.  It builds the collision operators
Lambda = M^-1 S M and M^-1 (I - S/2) M densely per cell from the printed matrix M
(tests/golden/natural_moment_matrix.txt), evaluates the equilibria and sources of Secs. 3.1-3.3
with the material laws, mass flux and surface-tension force of Secs. 2.1-2.3, streams with
half-way bounce-back (Sec. 4), and is compared with every population of the C oracle after 1 and
10 steps.  The readings where the paper is silent (stencils, backward time differences, the
normal's threshold, wall ghosts, the velocity with 1/rho, K = w0 / (c^2 - cs^2)) are the same
ones, restated here."""
import os

import numpy as np
import pytest

import oracle
from paper_2408_15654_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CS2 = 1.0 / 3.0
CV = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
WV = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


class Brute:
    """The step of Secs. 2-4 on an (ny, nx) grid, all cells at once (arrays [9, ny, nx])."""

    def __init__(self, p):
        self.p = p
        self.M = np.loadtxt(os.path.join(GOLDEN, "natural_moment_matrix.txt"))
        self.Minv = np.linalg.inv(self.M)
        self.first = True

    # --- neighbours: periodic in x; in y periodic, or walls whose ghost row repeats the fluid row
    def shift(self, q, cx, cy):
        ny, nx = q.shape
        xs = (np.arange(nx) + cx) % nx
        ys = np.arange(ny) + cy
        ys = ys % ny if not self.p["walls"] else np.clip(ys, 0, ny - 1)
        return q[np.ix_(ys, xs)]

    def grad_lap(self, q):
        gx = sum(WV[i] * CV[i, 0] * self.shift(q, *CV[i]) for i in range(9)) / CS2
        gy = sum(WV[i] * CV[i, 1] * self.shift(q, *CV[i]) for i in range(9)) / CS2
        lap = 2.0 / CS2 * sum(WV[i] * (self.shift(q, *CV[i]) - q) for i in range(1, 9))
        return gx, gy, lap

    def operators(self, s):
        """Lambda and M^-1 (I - S/2) M for relaxation rates s[..., 9] (per cell)."""
        S = s[..., None] * np.eye(9)
        lam = self.Minv @ S @ self.M
        src = self.Minv @ (np.eye(9) - 0.5 * S) @ self.M
        return lam, src

    @staticmethod
    def diag(s5):
        s0, s1, s2, s3, s4 = s5
        return np.stack([s0, s1, s1, s2, s2, s2, s3, s3, s4], axis=-1)

    def equilibria(self, phi, psi, ux, uy, P, rho, Sx, Sy):
        p = self.p
        cu = CV[:, 0, None, None] * ux + CV[:, 1, None, None] * uy
        w = WV[:, None, None]
        feq = w * phi * (1 + cu / CS2)
        geq = w * psi * (1 + cu / CS2)
        # (rho u - S) u : (c c - cs2 I) / (2 cs4)
        jx, jy = rho * ux - Sx, rho * uy - Sy
        cxx = CV[:, 0, None, None] ** 2 - CS2
        cyy = CV[:, 1, None, None] ** 2 - CS2
        cxy = (CV[:, 0] * CV[:, 1])[:, None, None]
        quad = (jx * ux * cxx + jy * uy * cyy + (jx * uy + jy * ux) * cxy) / (2 * CS2 ** 2)
        lam = w * P / CS2
        lam[0] = p["rho0"] + (WV[0] - 1) * P / CS2
        heq = lam + w * ((CV[:, 0, None, None] * rho * ux + CV[:, 1, None, None] * rho * uy) / CS2 + quad)
        return feq, geq, heq

    def init(self, phi, psi, ux, uy, P):
        p = self.p
        shape = phi.shape
        ux, uy, P = (np.broadcast_to(np.asarray(a, float), shape).copy() for a in (ux, uy, P))
        rho = p["rhoB"] + (phi - p["phiB"]) / (p["phiA"] - p["phiB"]) * (p["rhoA"] - p["rhoB"])
        z = np.zeros(shape)
        self.f, self.g, self.h = self.equilibria(phi, psi, ux, uy, P, rho, z, z)
        self.first = True

    def step(self):
        p = self.p
        dphi = p["phiA"] - p["phiB"]
        f, g, h = self.f, self.g, self.h
        phi, psi = f.sum(0), g.sum(0)
        gpx, gpy, lap = self.grad_lap(phi)
        gsx, gsy, _ = self.grad_lap(psi)
        gn = np.hypot(gpx, gpy)
        big = gn > p["n_eps"]
        nx_ = np.where(big, gpx / np.where(big, gn, 1.0), 0.0)
        ny_ = np.where(big, gpy / np.where(big, gn, 1.0), 0.0)
        A = 4 * (p["phiA"] - phi) * (phi - p["phiB"]) / (p["W"] * dphi)
        B = 4 * psi * (p["phiA"] + p["phiB"] - 2 * phi) / (p["W"] * dphi)
        # material laws (Sec. 2.3), EOS (Eqs. EOS and EOSlinear), grad sigma by the chain rule
        lin = (phi - p["phiB"]) / dphi
        rho = lin * (p["rhoA"] - p["rhoB"]) + p["rhoB"]
        mu = lin * (p["muA"] - p["muB"]) + p["muB"]
        drho = (p["rhoA"] - p["rhoB"]) / dphi
        grx, gry = drho * gpx, drho * gpy
        if p["eos"] == "langmuir":
            sigma = p["sigma0"] * (1 + p["E0"] * np.log(1 - psi))
            dsig = -p["sigma0"] * p["E0"] / (1 - psi)
        else:
            sigma = p["sigma0"] * (1 - p["E0"] * psi)
            dsig = -p["sigma0"] * p["E0"] * np.ones_like(psi)
        gsigx, gsigy = dsig * gsx, dsig * gsy
        # surface tension, expanded form (Sec. 2.3), body force rho g, mass flux S
        capk = 3 * sigma / (2 * dphi ** 2) * (16 / p["W"] * (p["phiA"] - phi) * (phi - p["phiB"]) *
                                              (p["phiA"] + p["phiB"] - 2 * phi) - p["W"] * lap)
        mar = 3 * p["W"] / (2 * dphi ** 2)
        g2 = gpx ** 2 + gpy ** 2
        sdot = gsigx * gpx + gsigy * gpy
        Fx = capk * gpx + mar * (g2 * gsigx - sdot * gpx) + rho * p["gx"]
        Fy = capk * gpy + mar * (g2 * gsigy - sdot * gpy) + rho * p["gy"]
        Sx = p["M_phi"] * drho * (gpx - A * nx_)
        Sy = p["M_phi"] * drho * (gpy - A * ny_)
        # velocity (rho u = sum c h + F/2) and the time derivatives (backward, zero on the first step)
        ux = ((CV[:, 0, None, None] * h).sum(0) + 0.5 * Fx) / rho
        uy = ((CV[:, 1, None, None] * h).sum(0) + 0.5 * Fy) / rho
        if self.first:
            php, psp, uxp, uyp, Sxp, Syp = phi, psi, ux, uy, Sx, Sy
        else:
            php, psp, uxp, uyp, Sxp, Syp = self.hist
        rhop = (php - p["phiB"]) / dphi * (p["rhoA"] - p["rhoB"]) + p["rhoB"]
        dt_phix, dt_phiy = phi * ux - php * uxp, phi * uy - php * uyp
        dt_psix, dt_psiy = psi * ux - psp * uxp, psi * uy - psp * uyp
        Q = lambda r, a, b, sa, sb: r * a * b - 0.5 * (sa * b + a * sb)  # noqa: E731
        dxx = Q(rho, ux, ux, Sx, Sx) - Q(rhop, uxp, uxp, Sxp, Sxp)
        dyy = Q(rho, uy, uy, Sy, Sy) - Q(rhop, uyp, uyp, Syp, Syp)
        dxy = Q(rho, ux, uy, Sx, Sy) - Q(rhop, uxp, uyp, Sxp, Syp)
        dtr = (rho * (ux * ux + uy * uy) - (Sx * ux + Sy * uy)) - (rhop * (uxp * uxp + uyp * uyp) - (Sxp * uxp + Syp * uyp))
        # pressure (Eq. P) with K = w0 / (c^2 - cs2)
        K = WV[0] / (1 - CS2)
        ugr = ux * grx + uy * gry
        jSu = (rho * ux - Sx) * ux + (rho * uy - Sy) * uy
        P = CS2 / (1 - WV[0]) * (h[1:].sum(0) + 0.5 * ugr - WV[0] * jSu / (2 * CS2) + K * 0.5 * dtr)
        # equilibria and sources (Secs. 3.1-3.3)
        feq, geq, heq = self.equilibria(phi, psi, ux, uy, P, rho, Sx, Sy)
        w = WV[:, None, None]
        cX, cY = CV[:, 0, None, None], CV[:, 1, None, None]
        Fs = w * (cX * dt_phix + cY * dt_phiy) / CS2 + w * (cX * A * nx_ + cY * A * ny_)
        Gs = w * (cX * dt_psix + cY * dt_psiy) / CS2 + w * (cX * B * nx_ + cY * B * ny_)
        m2xx = dxx + CS2 * 2 * ux * grx
        m2yy = dyy + CS2 * 2 * uy * gry
        m2xy = dxy + CS2 * (ux * gry + uy * grx)
        cxx, cyy, cxy = cX ** 2 - CS2, cY ** 2 - CS2, cX * cY
        Hs = w * (ugr + (cX * Fx + cY * Fy) / CS2 + (m2xx * cxx + m2yy * cyy + 2 * m2xy * cxy) / (2 * CS2 ** 2))
        # collision: q* = q - Lambda (q - q_eq) + M^-1 (I - S/2) M Q
        sf = list(p["s_f"]); sf[1] = 1 / (p["M_phi"] / CS2 + 0.5)
        sg = list(p["s_g"]); sg[1] = 1 / (p["D"] / CS2 + 0.5)
        lf, srcf = self.operators(self.diag(np.array(sf)))
        lg, srcg = self.operators(self.diag(np.array(sg)))
        s2 = 1 / (mu / (rho * CS2) + 0.5)
        sh = [np.full(phi.shape, v, float) for v in p["s_h"]]
        sh[2] = s2
        if p["s_h"][4] <= 0:
            sh[4] = s2
        lh, srch = self.operators(self.diag(sh))  # per cell [ny, nx, 9, 9]
        fs = f - np.einsum("ij,jyx->iyx", lf, f - feq) + np.einsum("ij,jyx->iyx", srcf, Fs)
        gs = g - np.einsum("ij,jyx->iyx", lg, g - geq) + np.einsum("ij,jyx->iyx", srcg, Gs)
        hs = h - np.einsum("yxij,jyx->iyx", lh, h - heq) + np.einsum("yxij,jyx->iyx", srch, Hs)
        # pull streaming; half-way bounce-back at walls, moving-wall term for h with rho of the cell
        ny, nx = phi.shape
        nf, ng, nh = np.empty_like(f), np.empty_like(g), np.empty_like(h)
        for i in range(9):
            cx, cy = CV[i]
            for y in range(ny):
                ys = y - cy
                for x in range(nx):
                    xs = (x - cx) % nx
                    if p["walls"] and not (0 <= ys < ny):
                        o = OPP[i]
                        uw = p["u_bot"] if ys < 0 else p["u_top"]
                        nf[i, y, x], ng[i, y, x] = fs[o, y, x], gs[o, y, x]
                        nh[i, y, x] = hs[o, y, x] - 2 * WV[o] * rho[y, x] * (CV[o, 0] * uw) / CS2
                    else:
                        ys_ = ys % ny
                        nf[i, y, x], ng[i, y, x], nh[i, y, x] = fs[i, ys_, xs], gs[i, ys_, xs], hs[i, ys_, xs]
        self.f, self.g, self.h = nf, ng, nh
        self.hist = (phi, psi, ux, uy, Sx, Sy)
        self.first = False


def smooth_fields(nx, ny, seed, density_ratio):
    rng = np.random.default_rng(seed)
    x, y = W.grid(nx, ny)
    k = 2 * np.pi / nx
    a = rng.uniform(0, 2 * np.pi, 6)
    phi = 0.5 + 0.3 * np.sin(k * x + a[0]) * np.cos(k * y + a[1]) + 0.1 * np.cos(2 * k * x + a[2])
    psi = 0.25 + 0.1 * np.sin(k * x + a[3]) + 0.08 * np.cos(k * y + a[4])
    ux = 0.02 * np.sin(k * y + a[5])
    uy = 0.015 * np.cos(k * x + a[0])
    P = 1e-3 * np.sin(k * (x + y))
    return W.fields(phi, psi, ux=ux, uy=uy, P=P)


CASES = {
    "periodic_linear": dict(walls=False, eos="linear", rhoA=1.0, rhoB=1.0, s_h=(1.0, 1.1, 1.0, 1.2, 0.0)),
    "walls_langmuir": dict(walls=True, eos="langmuir", u_top=0.01, u_bot=-0.02, rhoA=1.0, rhoB=1.0,
                           s_h=(1.0, 1.1, 1.0, 1.2, 0.95)),
    "walls_density_ratio": dict(walls=True, eos="linear", u_top=0.01, u_bot=0.0, rhoA=1.0, rhoB=0.2,
                                gx=2e-5, gy=-1e-5, s_h=(1.0, 1.1, 1.0, 1.2, 0.0)),
    "periodic_density_ratio_langmuir": dict(walls=False, eos="langmuir", rhoA=0.5, rhoB=1.0, gy=-2e-5,
                                            s_h=(1.0, 0.9, 1.0, 1.15, 1.05)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_equals_brute_force_on_8x8(name):
    p = W.base_params(8, 8, muA=0.12, muB=0.07, W=4.0, M_phi=0.07, D=0.04, sigma0=2e-3, E0=0.4,
                      s_f=(1.0, 1.0, 1.2, 0.9, 1.1), s_g=(1.0, 1.0, 0.8, 1.3, 1.05))
    p.update(CASES[name])
    f0 = smooth_fields(8, 8, seed=len(name), density_ratio=p["rhoA"] != p["rhoB"])
    o = oracle.Sim(p)
    o.init(**f0)
    b = Brute(p)
    b.init(**{k: np.asarray(v, float) for k, v in f0.items()})
    for n in (1, 9):
        o.step(n)
        for _ in range(n):
            b.step()
        fo, go, ho = o.populations()
        for got, want, lab in ((fo, b.f, "f"), (go, b.g, "g"), (ho, b.h, "h")):
            err = np.abs(got - want).max()
            assert err <= 1e-13, (name, o.steps, lab, err)
    assert o.status == 0
