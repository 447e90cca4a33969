"""Seeded synthetic inputs for the two-distribution D2Q9 multiphase lattice Boltzmann workloads.

This module is the one piece shared by the CUDA path, its tests, the bench and the FP64 oracle.
It holds *inputs only*: physical parameters (surface tension, interface width, densities,
kinematic viscosities, gravity, boundary types, step counts) and initial fields (order
parameter, velocity, pressure). It contains none of the scheme's arithmetic: the conversion of
(sigma, W) into the free-energy coefficients (beta, kappa) and of viscosities into relaxation
times is done separately by the library and by the oracle.

Conventions (lattice units, dx = dt = 1):
  * cell centres sit at integer coordinates (x, y), x in [0, nx), y in [0, ny);
    fields are row-major float32 arrays of shape (ny, nx);
  * the heavy phase A ("liquid") is phi = +phi_star, the light phase B ("gas") is phi = -phi_star;
  * a droplet is phi = phi_star * tanh(2 (R - r) / W), a liquid film of thickness h on the
    bottom wall is phi = phi_star * tanh(2 (h - y) / W); droplet plus film is their maximum.
    These are the planar/circular equilibrium profiles of the double-well free energy
    (Eq. 1, second form) with interface width W.

Workloads (all synthetic; the paper uses no dataset):
  c1  static droplet, 128x128 periodic, R=25, W=4, sigma=0.01, rho 1:0.1, tau=0.8, 1000 steps.
  c2  falling droplet, 256x1024, walls on y, R=40 at (128, 800), rho 1:0.01, dynamic-viscosity
      ratio 10 with nu_A=0.025, g=1e-6, sigma=0.005, W=4, 20k steps, diagnostics every 100.
  c3  droplet splashing on a thin film, 2048x512, walls on y, film h=20, D=200, rho 1:0.001,
      dynamic-viscosity ratio 40, Re=500 and We=8000 at U=0.04 (nu_A=0.016, sigma=4e-5), W=5,
      impact velocity -U inside the droplet, 10k steps.
  c4  256 independent static/falling droplets with ragged grid sizes (seed 1234), 2k steps.
  c5  Poisson stream of falling-droplet requests (seed 5678, 50 req/s).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

PERIODIC = 0
WALL = 1

# Default Cahn-Hilliard mobility (lattice units) used by every workload; the configurations
# quoted for this method fix no mobility.
THETA_M_DEFAULT = 0.1
TAU_F_DEFAULT = 0.8


@dataclasses.dataclass
class Physical:
    """Physical parameters of one simulation (inputs only)."""

    sigma: float            # surface tension
    W: float                # interface width
    phi_star: float = 1.0   # equilibrium order parameter
    theta_M: float = THETA_M_DEFAULT
    tau_f: float = TAU_F_DEFAULT
    nu_A: float = 0.1       # kinematic viscosity of the heavy phase A (phi = +phi_star)
    nu_B: float = 0.1       # kinematic viscosity of the light phase B (phi = -phi_star)
    rho_A: float = 1.0
    rho_B: float = 0.1
    gravity: float = 0.0    # magnitude of g; gravity points to -y
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    remove_Fa: int = 0      # 0: scheme as first stated, 1: additional interfacial force removed
    ch_conservative: int = 0  # 0: convective Cahn-Hilliard equation (as printed), 1: conservative form
    fs_form: int = 0        # 0: F_s = -phi grad(mu), 1: F_s = mu grad(phi)
    s_form: int = 0         # mass defect s: 0 by Eq. 5, 1 from the stored rho and div(rho u)
    f_form: int = 0         # order-parameter LBE: 0 mu-term equilibrium, 1 forced (equilibrium phi Gamma)


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    phys: Physical
    steps: int
    phi0: np.ndarray
    ux0: np.ndarray
    uy0: np.ndarray
    p0: np.ndarray
    diag_every: int = 100
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def with_flag(self, remove_Fa: int) -> "Workload":
        w = dataclasses.replace(self, phys=dataclasses.replace(self.phys, remove_Fa=int(remove_Fa)))
        return w


# --------------------------------------------------------------------------- profiles

def _grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def droplet_phi(nx, ny, xc, yc, R, W, phi_star=1.0, periodic_x=True, periodic_y=True):
    """phi_star * tanh(2 (R - r) / W) around (xc, yc); r uses the nearest periodic image."""
    x, y = _grid(nx, ny)
    dx = x - xc
    dy = y - yc
    if periodic_x:
        dx = dx - nx * np.round(dx / nx)
    if periodic_y:
        dy = dy - ny * np.round(dy / ny)
    r = np.sqrt(dx * dx + dy * dy)
    return phi_star * np.tanh(2.0 * (R - r) / W)


def film_phi(nx, ny, h, W, phi_star=1.0):
    x, y = _grid(nx, ny)
    return phi_star * np.tanh(2.0 * (h - y) / W)


def planar_slab_phi(nx, ny, x_lo, x_hi, W, phi_star=1.0):
    """Liquid slab x_lo < x < x_hi: two planar interfaces normal to x."""
    x, _ = _grid(nx, ny)
    d = np.minimum(x - x_lo, x_hi - x)
    return phi_star * np.tanh(2.0 * d / W)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _zeros(nx, ny):
    return np.zeros((ny, nx), dtype=np.float32)


def make(name, nx, ny, phys, steps, phi0, ux0=None, uy0=None, p0=None, diag_every=100, **meta):
    return Workload(name=name, nx=nx, ny=ny, phys=phys, steps=steps, phi0=_f32(phi0),
                    ux0=_f32(ux0) if ux0 is not None else _zeros(nx, ny),
                    uy0=_f32(uy0) if uy0 is not None else _zeros(nx, ny),
                    p0=_f32(p0) if p0 is not None else _zeros(nx, ny),
                    diag_every=diag_every, meta=dict(meta))


# --------------------------------------------------------------------------- configs

def static_droplet(nx=128, ny=128, R=25.0, W=4.0, sigma=0.01, ratio=10.0, tau=0.8, steps=1000,
                   remove_Fa=0, theta_M=THETA_M_DEFAULT, xc=None, yc=None):
    """c1: static droplet at the centre of a periodic box; tau_f = tau_g = tau in both phases."""
    nu = (tau - 0.5) / 3.0
    phys = Physical(sigma=sigma, W=W, theta_M=theta_M, tau_f=tau, nu_A=nu, nu_B=nu, rho_A=1.0,
                    rho_B=1.0 / ratio, gravity=0.0, bc_x=PERIODIC, bc_y=PERIODIC,
                    remove_Fa=remove_Fa)
    xc = nx / 2 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    phi0 = droplet_phi(nx, ny, xc, yc, R, W)
    return make("c1_static_droplet_%dx%d" % (nx, ny), nx, ny, phys, steps, phi0, R=R, xc=xc, yc=yc)


def falling_droplet(nx=256, ny=1024, R=40.0, yc=800.0, ratio=100.0, visc_ratio=10.0, nu_A=0.025,
                    gravity=1e-6, sigma=0.005, W=4.0, steps=20000, remove_Fa=0, diag_every=100,
                    theta_M=THETA_M_DEFAULT):
    """c2: droplet falling under gravity between no-slip walls at y=0 and y=ny-1, periodic in x.

    visc_ratio is the dynamic-viscosity ratio mu_A / mu_B."""
    rho_A, rho_B = 1.0, 1.0 / ratio
    nu_B = nu_A * rho_A / (visc_ratio * rho_B)
    phys = Physical(sigma=sigma, W=W, theta_M=theta_M, nu_A=nu_A, nu_B=nu_B, rho_A=rho_A,
                    rho_B=rho_B, gravity=gravity, bc_x=PERIODIC, bc_y=WALL, remove_Fa=remove_Fa)
    phi0 = droplet_phi(nx, ny, nx / 2, yc, R, W, periodic_y=False)
    return make("c2_falling_droplet_%dx%d" % (nx, ny), nx, ny, phys, steps, phi0,
                diag_every=diag_every, R=R, xc=nx / 2, yc=yc)


def splash(nx=2048, ny=512, D=200.0, h=None, U=0.04, Re=500.0, We=8000.0, ratio=1000.0,
           visc_ratio=40.0, W=5.0, steps=10000, remove_Fa=0, theta_M=THETA_M_DEFAULT):
    """c3: droplet of diameter D impacting a liquid film of thickness 0.1 D on the bottom wall.

    We = rho_A U^2 D / sigma and Re = U D / nu_A fix sigma and nu_A at U = 0.04."""
    rho_A, rho_B = 1.0, 1.0 / ratio
    h = 0.1 * D if h is None else h
    sigma = rho_A * U * U * D / We
    nu_A = U * D / Re
    nu_B = nu_A * rho_A / (visc_ratio * rho_B)
    phys = Physical(sigma=sigma, W=W, theta_M=theta_M, nu_A=nu_A, nu_B=nu_B, rho_A=rho_A,
                    rho_B=rho_B, gravity=0.0, bc_x=PERIODIC, bc_y=WALL, remove_Fa=remove_Fa)
    R = D / 2
    yc = h + R + W
    drop = droplet_phi(nx, ny, nx / 2, yc, R, W, periodic_y=False)
    film = film_phi(nx, ny, h, W)
    phi0 = np.maximum(drop, film)
    uy0 = np.where(drop >= 0.0, -U, 0.0)   # liquid fraction of the droplet >= 1/2
    return make("c3_splash_%dx%d" % (nx, ny), nx, ny, phys, steps, phi0, uy0=uy0,
                R=R, xc=nx / 2, yc=yc, h=h, U=U)


def paper_falling_droplet(steps=19000, remove_Fa=0):
    """The paper's second experiment at its own size: 150x450, Eo=17, sigma=0.002, D=32,
    rho_L=5, rho_G=1, W=3, nu_L=0.025 (g from Eo = g (rho_L - rho_G) D^2 / sigma)."""
    D, sigma, Eo = 32.0, 0.002, 17.0
    rho_A, rho_B = 5.0, 1.0
    g = Eo * sigma / ((rho_A - rho_B) * D * D)
    phys = Physical(sigma=sigma, W=3.0, nu_A=0.025, nu_B=0.025, rho_A=rho_A, rho_B=rho_B,
                    gravity=g, bc_x=PERIODIC, bc_y=WALL, remove_Fa=remove_Fa)
    nx, ny = 150, 450
    yc = ny - 2 * D
    phi0 = droplet_phi(nx, ny, nx / 2, yc, D / 2, 3.0, periodic_y=False)
    return make("paper_falling_droplet_150x450", nx, ny, phys, steps, phi0, R=D / 2, xc=nx / 2,
                yc=yc)


def paper_splash(Re=480.0, steps=3000, remove_Fa=0):
    """The paper's first experiment at its own size: droplet splashing on a thin film, 300x150,
    film height one tenth of the domain height, We = 960 with sigma = 1e-4, U = 0.04, D = 60;
    Re = 48 or 480 (nu_L = 0.05 or 0.005); W = 3, rho_L = 1, rho_G = 0.1.  The paper gives one
    viscosity: both phases take nu_L.  Walls on y, periodic in x; the drop touches the film and
    moves down at U."""
    nx, ny, D, U, sigma = 300, 150, 60.0, 0.04, 1e-4
    nu = U * D / Re
    h, W = 0.1 * ny, 3.0
    phys = Physical(sigma=sigma, W=W, nu_A=nu, nu_B=nu, rho_A=1.0, rho_B=0.1, gravity=0.0,
                    bc_x=PERIODIC, bc_y=WALL, remove_Fa=remove_Fa)
    R = D / 2
    yc = h + R + W
    drop = droplet_phi(nx, ny, nx / 2, yc, R, W, periodic_y=False)
    phi0 = np.maximum(drop, film_phi(nx, ny, h, W))
    uy0 = np.where(drop >= 0.0, -U, 0.0)
    return make("paper_splash_300x150_Re%g" % Re, nx, ny, phys, steps, phi0, uy0=uy0, R=R, xc=nx / 2,
                yc=yc, h=h, U=U, D=D)


def _round32(v):
    return max(32, int(round(v / 32.0)) * 32)


def ragged_batch(n=256, seed=1234, steps=2000, storage="fp32"):
    """c4: independent static/falling droplets; grid area ~ U[64^2, 512^2], aspect ~ U[1, 4]."""
    rng = np.random.default_rng(seed)
    out: List[Workload] = []
    for i in range(n):
        A = rng.uniform(64 * 64, 512 * 512)
        a = rng.uniform(1.0, 4.0)
        nx = _round32(math.sqrt(A * a))
        ny = max(64, int(round(A / nx)))
        falling = bool(rng.random() < 0.5)
        R = rng.uniform(8.0, 0.3 * min(nx, ny))
        ratio = float(rng.choice([10.0, 100.0, 1000.0]))
        sigma = rng.uniform(1e-3, 1e-2)
        W = 4.0
        rho_A, rho_B = 1.0, 1.0 / ratio
        phys = Physical(sigma=sigma, W=W, nu_A=0.1, nu_B=0.1, rho_A=rho_A, rho_B=rho_B,
                        gravity=1e-6 if falling else 0.0, bc_x=PERIODIC,
                        bc_y=WALL if falling else PERIODIC)
        yc = (0.7 * ny) if falling else ny / 2
        yc = min(yc, ny - R - 2 * W)
        phi0 = droplet_phi(nx, ny, nx / 2, yc, R, W, periodic_y=not falling)
        out.append(make("c4_%03d_%s_%dx%d" % (i, "falling" if falling else "static", nx, ny), nx,
                        ny, phys, steps, phi0, R=R, xc=nx / 2, yc=yc, storage=storage))
    return out


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    workload: Workload


def serving_stream(n=256, seed=5678, rate=50.0, step_scale=1.0, max_steps=None, size_scale=1):
    """c5: Poisson arrivals of falling-droplet requests.

    nx ~ U{128..1024 step 32}, ny = nx * a with a ~ U{2,3,4} clamped to [256, 4096],
    steps log-uniform in [2k, 50k] (times step_scale), density ratio log-uniform in [10, 1000].
    size_scale divides both grid sizes (rounded to 32) for bounded runs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out: List[Request] = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        nx = int(rng.integers(128 // 32, 1024 // 32 + 1)) * 32
        a = int(rng.integers(2, 5))
        ny = min(max(nx * a, 256), 4096)
        steps = math.exp(rng.uniform(math.log(2000.0), math.log(50000.0)))
        ratio = math.exp(rng.uniform(math.log(10.0), math.log(1000.0)))
        if size_scale > 1:
            nx = max(64, (nx // size_scale) // 32 * 32)
            ny = max(64, ny // size_scale)
        steps = max(1, int(round(steps * step_scale)))
        if max_steps is not None:
            steps = min(steps, max_steps)
        R = min(nx, ny) / 6.0
        rho_A, rho_B = 1.0, 1.0 / ratio
        nu_A = 0.025
        nu_B = nu_A * rho_A / (10.0 * rho_B)
        phys = Physical(sigma=0.005, W=4.0, nu_A=nu_A, nu_B=nu_B, rho_A=rho_A, rho_B=rho_B,
                        gravity=1e-6, bc_x=PERIODIC, bc_y=WALL)
        yc = 0.75 * ny
        phi0 = droplet_phi(nx, ny, nx / 2, yc, R, 4.0, periodic_y=False)
        w = make("c5_req%03d_%dx%d" % (i, nx, ny), nx, ny, phys, steps, phi0, R=R, xc=nx / 2,
                 yc=yc)
        out.append(Request(rid=i, arrival_s=t, workload=w))
    return out


def random_small(nx, ny, seed, bc_x=PERIODIC, bc_y=PERIODIC, remove_Fa=0, ratio=10.0,
                 gravity=0.0, u_amp=0.01, steps=50, sigma=0.01, W=4.0, nu_A=0.1, nu_B=0.1,
                 theta_M=THETA_M_DEFAULT, tau_f=TAU_F_DEFAULT):
    """Tiny seeded case for parity tests: one or two droplets plus a smooth random velocity."""
    rng = np.random.default_rng(seed)
    phi = np.full((ny, nx), -1.0)
    for _ in range(int(rng.integers(1, 3))):
        R = rng.uniform(0.15, 0.3) * min(nx, ny)
        xc = rng.uniform(0.3, 0.7) * nx
        yc = rng.uniform(0.3, 0.7) * ny
        d = droplet_phi(nx, ny, xc, yc, R, W, periodic_x=bc_x == PERIODIC,
                        periodic_y=bc_y == PERIODIC)
        phi = np.maximum(phi, d)
    x, y = _grid(nx, ny)
    kx = 2 * math.pi / nx
    ky = 2 * math.pi / ny
    a = rng.uniform(-1, 1, size=4)
    ux = u_amp * (a[0] * np.sin(ky * y + a[1]) + 0.3 * a[2] * np.cos(kx * x))
    uy = u_amp * (a[2] * np.sin(kx * x + a[3]) + 0.3 * a[0] * np.cos(ky * y))
    if bc_y == WALL:
        ux *= np.sin(math.pi * (y + 0.5) / ny)
        uy *= np.sin(math.pi * (y + 0.5) / ny)
    if bc_x == WALL:
        ux *= np.sin(math.pi * (x + 0.5) / nx)
        uy *= np.sin(math.pi * (x + 0.5) / nx)
    p = 1e-4 * rng.standard_normal((ny, nx)) * 0.0
    phys = Physical(sigma=sigma, W=W, theta_M=theta_M, tau_f=tau_f, nu_A=nu_A, nu_B=nu_B,
                    rho_A=1.0, rho_B=1.0 / ratio, gravity=gravity, bc_x=bc_x, bc_y=bc_y,
                    remove_Fa=remove_Fa)
    return make("small_%dx%d_s%d" % (nx, ny, seed), nx, ny, phys, steps, phi, ux, uy, p)


CONFIGS = {
    "c1": static_droplet,
    "c2": falling_droplet,
    "c3": splash,
}
