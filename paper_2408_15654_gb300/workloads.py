"""Seeded synthetic workloads: parameter sets and initial fields.

This module only builds inputs (initial phase field, surfactant, velocity and pressure on a grid,
plus the physical parameters in lattice units).  It contains none of the lattice-Boltzmann step,
so the CUDA library and the FP64 oracle can both be fed from it without sharing any arithmetic of
the method.

Lattice units throughout: dx = dt = 1, cells at integer coordinates (x, y), x in [0, nx),
y in [0, ny).  With walls, the walls sit half a cell outside the first and last rows
(y = -1/2 and y = ny - 1/2), so the channel height is H = ny.

Workloads (stand-ins for the paper's Sec. 4 benchmarks; the paper's comparison data is not used):
  stationary_drop    128 x 128 periodic drop, R = 32, linear EOS, interface-uniform psi
  surface_diffusion  256 x 256 periodic drop, R = 60, psi = 0.5 (1 + cos theta) on the interface,
                     sigma0 = 0 so the flow stays at rest (Sec. 4.1)
  shear_drop         drop between walls moving at +/-U (Sec. 4.4): 512 x 256 with R = 40 and
                     2048 x 1024 with R = 160, Re = 1, Ca = 0.2, Langmuir EOS E0 = 0.2, psi0 = 0.3
  convected_drop     a drop carried by an imposed uniform velocity (prescribed-velocity mode):
                     the convection test of Sec. 4 (100 x 100, R = 20, u = (0.05, 0), psi = phi,
                     M_phi = 1, D = 2 in lattice units)
  rising_bubble      the single rising bubble of Sec. 4 (density and viscosity ratio 10, Re = 35,
                     Pe = 10, Bo = 10, linear EOS)
  batch_instances    64 seeded drops of mixed sizes for the batched launch
  serving_requests   a seeded Poisson stream of sheared-drop jobs of mixed sizes, step counts and
                     storage modes, for the lattice server
"""
from __future__ import annotations

import math

import numpy as np

# Free relaxation rates (s0, s1, s2, s3, s4) of the moment-space collision.  The paper fixes only
# the transport rates (s1 of f and g from M_phi and D, s2 of h from mu / rho), which each
# implementation recomputes.  All other rates default to 1, except the fourth-order rate of the
# flow populations: 0 there means "s4 = s2", which keeps plane Couette flow exact.
_UNIT_RATES = (1.0, 1.0, 1.0, 1.0, 1.0)
_FLOW_RATES = (1.0, 1.0, 1.0, 1.0, 0.0)


def base_params(nx: int, ny: int, **kw) -> dict:
    """Defaults of every workload.  The unit normal n = grad phi / |grad phi| is taken wherever
    |grad phi| > n_eps = 1e-12, that is wherever grad phi is not zero, as the paper defines it.
    In single precision that makes some workloads sensitive to rounding: in a nearly flat bulk
    grad phi is itself of rounding size (about 1e-7 for phi of order 1) and its direction, which
    steers the sharpening terms A n and B n, flips from step to step.  Measured with the FP64
    oracle, a 6e-8 relative jitter of the initial fields moves phi by 1e-5 and psi by 2e-5
    (relative L2) in 3000 steps of a 256 x 128 sheared drop with n_eps = 1e-12, by 3e-9 and 1e-8
    with n_eps = 1e-4.  A larger threshold is no default: with n = 0 in the bulk, surfactant there
    is no longer swept onto the interface (Sec. 2.2)."""
    p = dict(
        nx=int(nx), ny=int(ny), walls=False, eos="linear", u_top=0.0, u_bot=0.0,
        phiA=1.0, phiB=0.0, rhoA=1.0, rhoB=1.0, muA=0.1, muB=0.1,
        W=4.0, M_phi=0.05, D=0.02, sigma0=1e-3, E0=0.5, gx=0.0, gy=0.0, rho0=1.0,
        n_eps=1e-12, s_f=_UNIT_RATES, s_g=_UNIT_RATES, s_h=_FLOW_RATES, velocity="solved",
    )
    for k, v in kw.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def grid(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def drop_phi(nx, ny, R, W, xc=None, yc=None, phiA=1.0, phiB=0.0):
    """Circular drop of phase A (inside) with the tanh profile of the equilibrium interface."""
    x, y = grid(nx, ny)
    xc = nx / 2 - 0.5 if xc is None else xc
    yc = ny / 2 - 0.5 if yc is None else yc
    r = np.hypot(x - xc, y - yc)
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * (R - r) / W)


def interface_weight(phi, phiA=1.0, phiB=0.0):
    """4 (phiA - phi)(phi - phiB) / (phiA - phiB)^2: 1 on the interface, 0 in the bulk."""
    return 4.0 * (phiA - phi) * (phi - phiB) / (phiA - phiB) ** 2


def polar_angle(nx, ny, xc=None, yc=None):
    x, y = grid(nx, ny)
    xc = nx / 2 - 0.5 if xc is None else xc
    yc = ny / 2 - 0.5 if yc is None else yc
    return np.arctan2(y - yc, x - xc)


def fields(phi, psi, ux=0.0, uy=0.0, P=0.0) -> dict:
    shape = np.shape(phi)
    f = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
    return dict(phi=f(phi), psi=f(psi), ux=f(ux), uy=f(uy), P=f(P))


def stationary_drop(nx=128, ny=128, R=32.0, W=4.0, psi0=0.3, sigma0=1e-3, E0=0.5, tau_h=0.8,
                    M_phi=0.05, D=0.02, eos="linear"):
    """Stationary drop in a periodic box; 1 / s2^h = tau_h fixes nu = (tau_h - 1/2) / 3."""
    mu = (tau_h - 0.5) / 3.0
    p = base_params(nx, ny, W=W, sigma0=sigma0, E0=E0, muA=mu, muB=mu, M_phi=M_phi, D=D, eos=eos)
    phi = drop_phi(nx, ny, R, W)
    psi = psi0 * interface_weight(phi)
    return p, fields(phi, psi)


def surface_diffusion(n=256, R=60.0, W=4.0, D=0.05, M_phi=0.05):
    """Cos-theta surfactant mode on a fixed circular interface; sigma0 = 0 keeps u = 0."""
    p = base_params(n, n, W=W, D=D, M_phi=M_phi, sigma0=0.0, E0=0.0)
    phi = drop_phi(n, n, R, W)
    theta = polar_angle(n, n)
    psi = 0.5 * (1.0 + np.cos(theta)) * interface_weight(phi)
    return p, fields(phi, psi)


def rising_bubble(R=60.0, W=4.0, E0=0.5, psi0=1.0, Re=35.0, Pe=10.0, Bo=10.0, M_phi=0.05):
    """Single rising bubble (Sec. 4): a bubble of fluid B (phi = phiB = 0; rhoB = rhoA/10,
    muB = muA/10) of radius R at (2R, 2R) in a 4R x 8R box, walls at rest below and above, periodic
    in x, gravity -y, linear EOS, psi = psi0 sech^2 on the interface.  Lattice units with the
    paper's diffusive scaling dt = dx^2 at dx = 0.25/R: the velocity scale sqrt(2 g R) = 0.7 (in
    the paper's units) becomes 0.175/R, and mu_A, sigma0 and D follow from Re, Bo and Pe.  The
    phase-field mobility is not given; M_phi = 0.05 as for the other workloads.  This flow is the
    most sensitive to the normal threshold n_eps: a 6e-8 relative jitter of the initial fields
    moves phi by 5e-5 (relative L2, 400 steps, R = 16) with the default n_eps = 1e-12, by 1-2e-5
    with 1e-5 and by 5e-9 with 1e-4."""
    nx, ny = int(round(4 * R)), int(round(8 * R))
    U = 0.175 / R
    g = U * U / (2.0 * R)
    muA = 2.0 * R * U / Re
    sigma0 = 4.0 * g * R * R / Bo
    p = base_params(nx, ny, walls=True, rhoA=1.0, rhoB=0.1, muA=muA, muB=0.1 * muA, sigma0=sigma0,
                    E0=E0, eos="linear", gy=-g, W=W, M_phi=M_phi, D=2.0 * R * U / Pe)
    phi = 1.0 - drop_phi(nx, ny, R, W, xc=nx / 2.0 - 0.5, yc=2.0 * R - 0.5)  # walls at y = -1/2, ny - 1/2
    return p, fields(phi, psi0 * interface_weight(phi))


def convected_drop(nx=100, ny=100, R=20.0, W=4.0, u=(0.05, 0.0), M_phi=1.0, D=2.0):
    """Drop carried by the imposed uniform velocity u in a periodic box (prescribed-velocity mode,
    no flow populations); psi starts equal to phi, as in the paper's convection test (Sec. 4:
    R = 0.2 in the unit box at dx = 0.01, u = (0.5, 0) at dt = 0.001, M_phi = 0.1, D = 0.2)."""
    p = base_params(nx, ny, W=W, M_phi=M_phi, D=D, sigma0=0.0, E0=0.0, velocity="prescribed")
    phi = drop_phi(nx, ny, R, W)
    return p, fields(phi, phi.copy(), ux=u[0], uy=u[1])


def shear_params(nx, ny, R, U=0.01, Re=1.0, Ca=0.2, rho=1.0):
    """Viscosity and clean-interface tension from Re = rho g R^2 / mu and Ca = mu g R / sigma0,
    with the shear rate g = 2 U / H and H = ny."""
    gdot = 2.0 * U / ny
    mu = rho * gdot * R * R / Re
    sigma0 = mu * gdot * R / Ca
    return mu, sigma0


def shear_drop(nx=512, ny=256, R=40.0, W=4.0, U=0.01, Re=1.0, Ca=0.2, E0=0.2, psi0=0.3,
               eos="langmuir", M_phi=0.05, D=0.02):
    """Drop between walls moving at +U (top) and -U (bottom), linear initial shear profile."""
    mu, sigma0 = shear_params(nx, ny, R, U, Re, Ca)
    p = base_params(nx, ny, walls=True, u_top=U, u_bot=-U, muA=mu, muB=mu, sigma0=sigma0,
                    E0=E0, eos=eos, W=W, M_phi=M_phi, D=D)
    phi = drop_phi(nx, ny, R, W)
    psi = psi0 * interface_weight(phi)
    _, y = grid(nx, ny)
    ux = -U + 2.0 * U * (y + 0.5) / ny
    return p, fields(phi, psi, ux=ux)


def shear_drop_large(nx=2048, ny=1024):
    """The 2048 x 1024 sheared drop: R scaled to 160 at the same W, Re and Ca."""
    return shear_drop(nx=nx, ny=ny, R=160.0)


def perturbed(params: dict, flds: dict, seed: int, amp_phi=0.02, amp_psi=0.01, amp_u=0.005,
              amp_P=1e-4) -> dict:
    """Add seeded smooth random perturbations (a few low Fourier modes) to every field, so that
    all terms of the step (including the time derivatives and off-axis gradients) are exercised.
    The surfactant stays non-negative and below 1."""
    rng = np.random.default_rng(seed)
    nx, ny = params["nx"], params["ny"]
    x, y = grid(nx, ny)

    def smooth():
        out = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(0, 3, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            out += rng.uniform(-1, 1) * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny) + ph)
        return out / 4.0

    f = dict(flds)
    f["phi"] = flds["phi"] + amp_phi * smooth()
    f["psi"] = np.clip(flds["psi"] + amp_psi * (1 + smooth()) * 0.5, 0.0, 0.9) if amp_psi else flds["psi"]
    f["ux"] = flds["ux"] + amp_u * smooth()
    f["uy"] = flds["uy"] + amp_u * smooth()
    f["P"] = flds["P"] + amp_P * smooth()
    return {k: np.ascontiguousarray(v) for k, v in f.items()}


BATCH_SIZES = ((128, 128), (256, 256), (512, 256), (1024, 512))


def batch_instances(count=64, seed=0):
    """Seeded mix of independent drop simulations of uneven sizes.

    Sizes uniform over BATCH_SIZES; R ~ U[10, 80] clamped to 0.35 min(nx, ny); psi0 ~ U[0, 0.6];
    linear EOS with E0 ~ U[0.1, 0.5]; wall speed U ~ U[0, 0.02] (walls at rest when U = 0); the
    other parameters as for the stationary drop."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny = BATCH_SIZES[rng.integers(0, len(BATCH_SIZES))]
        R = min(rng.uniform(10.0, 80.0), 0.35 * min(nx, ny))
        psi0 = rng.uniform(0.0, 0.6)
        E0 = rng.uniform(0.1, 0.5)
        U = rng.uniform(0.0, 0.02)
        p = base_params(nx, ny, walls=True, u_top=U, u_bot=-U, E0=E0, eos="linear")
        phi = drop_phi(nx, ny, R, p["W"])
        psi = psi0 * interface_weight(phi)
        _, y = grid(nx, ny)
        ux = -U + 2.0 * U * (y + 0.5) / ny
        out.append((p, fields(phi, psi, ux=ux)))
    return out


SERVING_SIDES = tuple(range(256, 2049, 64))


def serving_requests(count=200, rate=20.0, seed=0):
    """Seeded job stream for the lattice server: Poisson arrivals at `rate` per second; each job a
    sheared drop (as shear_drop) on a square grid of side ~ U{256, 320, ..., 2048} with
    R = 40 side / 512; steps ~ U[5000, 50000]; storage FP32 or FP16 with probability 1/2 each.
    Returns dicts with the arrival time `t` (seconds from the first), nx, ny, R, steps, storage;
    serving_job builds a job's parameters and fields."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        if k:
            t += rng.exponential(1.0 / rate)
        side = int(SERVING_SIDES[rng.integers(0, len(SERVING_SIDES))])
        steps = int(rng.integers(5000, 50001))
        storage = "fp16" if rng.random() < 0.5 else "fp32"
        out.append({"t": t, "nx": side, "ny": side, "R": 40.0 * side / 512.0, "steps": steps,
                    "storage": storage})
    return out


def serving_job(req: dict):
    """Parameters (with the request's storage mode) and initial fields of one server job."""
    p, f = shear_drop(nx=req["nx"], ny=req["ny"], R=req["R"])
    return dict(p, storage=req["storage"]), f
