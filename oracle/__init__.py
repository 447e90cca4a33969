"""FP64 CPU oracle of the two-distribution multiphase lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY: this package is loaded by the tests, by the smoke check and by the
bench's CPU-baseline leg, never by the library.  It is the plain restatement of the scheme in
``lbm_oracle.c`` (see its header for the equations and their sources in the paper) plus a thin
ctypes wrapper.  It imports nothing from the CUDA library and the library imports nothing
from it; the two only share the seeded inputs of the ``workloads`` module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
WALL = 1
CS2 = 1.0 / 3.0

MU, S, FSX, FSY, DPX, DPY, GRAD_PHI_X, GRAD_PHI_Y, LAP_MU, TAU_G, DIVU, FAX, FAY = range(13)


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "beta", "kappa", "phi_star", "theta_M", "tau_f", "tau_g_A", "tau_g_B", "rho_A", "rho_B",
        "gravity")] + [(n, ctypes.c_int) for n in ("bc_x", "bc_y", "remove_Fa", "storage", "ch_conservative", "fs_form", "s_form", "f_form")]


class Diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong)] + [(n, ctypes.c_double) for n in (
        "sum_phi", "liquid_area", "centroid_x", "centroid_y", "vel_x", "vel_y", "spread_radius",
        "max_u", "p_liquid", "p_gas")] + [("finite", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


# -O3 with OpenMP over rows.  No -march=native: the oracle must give the same FP64 results on
# every host it runs on (x86_64 and aarch64), and no contraction into fused multiply-adds, which
# aarch64 compilers otherwise apply and x86_64 baseline code does not.
CFLAGS = ["-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object next to its source (gcc, OpenMP)."""
    with _lock:
        stamp = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.abspath(__file__)))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < stamp:
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.lbm_create_ref.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                                     ctypes.POINTER(vp)]
        L.lbm_create_ref.restype = ctypes.c_int
        L.lbm_destroy_ref.argtypes = [vp]
        L.lbm_init_fields_ref.argtypes = [vp, dp, dp, dp, dp]
        L.lbm_init_fields_ref.restype = ctypes.c_int
        L.lbm_step_ref.argtypes = [vp, ctypes.c_int]
        L.lbm_step_ref.restype = ctypes.c_int
        L.lbm_moments_ref.argtypes = [vp, dp, dp, dp, dp, dp]
        L.lbm_moments_ref.restype = ctypes.c_int
        L.lbm_diagnostics_ref.argtypes = [vp, ctypes.POINTER(Diag)]
        L.lbm_diagnostics_ref.restype = ctypes.c_int
        L.orc_field.argtypes = [vp, ctypes.c_int, dp]
        L.orc_field.restype = ctypes.c_int
        L.orc_get_state.argtypes = [vp, dp, dp]
        L.orc_set_state.argtypes = [vp, dp, dp]
        L.orc_collide.argtypes = [vp, dp, dp]
        L.orc_step_count.argtypes = [vp]
        L.orc_step_count.restype = ctypes.c_longlong
        L.orc_lap_iso.argtypes = [ctypes.c_int] * 4 + [dp, dp]
        L.orc_grad_iso.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp]
        L.orc_stream.argtypes = [ctypes.c_int] * 4 + [dp, dp]
        L.orc_node_equilibria.argtypes = [ctypes.POINTER(Params)] + [ctypes.c_double] * 6 + \
            [dp, dp, dp]
        L.orc_node_forcing.argtypes = [ctypes.c_double] * 6 + [dp]
        L.orc_params_from_sigma_W.argtypes = [ctypes.c_double] * 3 + [dp, dp]
        L.orc_tau_from_nu.argtypes = [ctypes.c_double]
        L.orc_tau_from_nu.restype = ctypes.c_double
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def params_from_sigma_W(sigma, W, phi_star=1.0):
    b = ctypes.c_double()
    k = ctypes.c_double()
    lib().orc_params_from_sigma_W(sigma, W, phi_star, ctypes.byref(b), ctypes.byref(k))
    return b.value, k.value


def tau_from_nu(nu):
    return lib().orc_tau_from_nu(nu)


def params_from_physical(phys) -> Params:
    """Scheme parameters of a ``workloads.Physical`` record (oracle's own conversion)."""
    beta, kappa = params_from_sigma_W(phys.sigma, phys.W, phys.phi_star)
    return Params(beta=beta, kappa=kappa, phi_star=phys.phi_star, theta_M=phys.theta_M,
                  tau_f=phys.tau_f, tau_g_A=tau_from_nu(phys.nu_A), tau_g_B=tau_from_nu(phys.nu_B),
                  rho_A=phys.rho_A, rho_B=phys.rho_B, gravity=phys.gravity, bc_x=phys.bc_x,
                  bc_y=phys.bc_y, remove_Fa=phys.remove_Fa, storage=0,
                  ch_conservative=phys.ch_conservative, fs_form=phys.fs_form, s_form=phys.s_form,
                  f_form=phys.f_form)


def set_threads(n: int):
    lib().orc_set_num_threads(int(n))


def num_threads() -> int:
    return lib().orc_num_threads()


class Sim:
    """One FP64 simulation.  Fields are (ny, nx) float64 arrays."""

    def __init__(self, nx, ny, params: Params):
        self.nx, self.ny = int(nx), int(ny)
        self.params = params
        h = ctypes.c_void_p()
        rc = lib().lbm_create_ref(self.nx, self.ny, ctypes.byref(params), ctypes.byref(h))
        if rc != 0:
            raise ValueError("lbm_create_ref failed (%d)" % rc)
        self._h = h

    @classmethod
    def from_workload(cls, w, init=True):
        s = cls(w.nx, w.ny, params_from_physical(w.phys))
        if init:
            s.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        return s

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().lbm_destroy_ref(h)
            self._h = None

    def init_fields(self, phi0, ux0=None, uy0=None, p0=None):
        a = [_f64(v) for v in (phi0, ux0, uy0, p0)]
        for v in a:
            if v is not None:
                assert v.shape == (self.ny, self.nx)
        rc = lib().lbm_init_fields_ref(self._h, *[_ptr(v) for v in a])
        if rc != 0:
            raise ValueError("init failed")

    def step(self, n=1):
        rc = lib().lbm_step_ref(self._h, int(n))
        if rc != 0:
            raise ValueError("step failed")

    @property
    def step_count(self):
        return lib().orc_step_count(self._h)

    def moments(self):
        out = {k: np.empty((self.ny, self.nx)) for k in ("phi", "rho", "ux", "uy", "p")}
        lib().lbm_moments_ref(self._h, *[_ptr(out[k]) for k in ("phi", "rho", "ux", "uy", "p")])
        return out

    def field(self, which):
        out = np.empty((self.ny, self.nx))
        rc = lib().orc_field(self._h, int(which), _ptr(out))
        if rc != 0:
            raise ValueError("unknown field")
        return out

    def diagnostics(self):
        d = Diag()
        lib().lbm_diagnostics_ref(self._h, ctypes.byref(d))
        return d.as_dict()

    def get_state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        lib().orc_get_state(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_state(self, f, g):
        lib().orc_set_state(self._h, _ptr(_f64(f)), _ptr(_f64(g)))

    def collide(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        lib().orc_collide(self._h, _ptr(f), _ptr(g))
        return f, g


def lap_iso(a, bc_x=PERIODIC, bc_y=PERIODIC):
    a = _f64(a)
    out = np.empty_like(a)
    lib().orc_lap_iso(a.shape[1], a.shape[0], bc_x, bc_y, _ptr(a), _ptr(out))
    return out


def grad_iso(a, bc_x=PERIODIC, bc_y=PERIODIC):
    a = _f64(a)
    gx = np.empty_like(a)
    gy = np.empty_like(a)
    lib().orc_grad_iso(a.shape[1], a.shape[0], bc_x, bc_y, _ptr(a), _ptr(gx), _ptr(gy))
    return gx, gy


def stream(pop, bc_x=PERIODIC, bc_y=PERIODIC):
    pop = _f64(pop)
    out = np.full_like(pop, np.nan)
    lib().orc_stream(pop.shape[2], pop.shape[1], bc_x, bc_y, _ptr(pop), _ptr(out))
    return out


def node_equilibria(params: Params, phi, mu, rho, p, ux, uy):
    feq = np.empty(9)
    geq = np.empty(9)
    G = np.empty(9)
    lib().orc_node_equilibria(ctypes.byref(params), phi, mu, rho, p, ux, uy, _ptr(feq), _ptr(geq),
                              _ptr(G))
    return feq, geq, G


def node_forcing(ux, uy, Fx, Fy, dpsix, dpsiy):
    S = np.empty(9)
    lib().orc_node_forcing(ux, uy, Fx, Fy, dpsix, dpsiy, _ptr(S))
    return S


def run(w, steps=None, remove_Fa=None):
    """Run a workload for ``steps`` (default: its own count); returns the Sim."""
    if remove_Fa is not None:
        w = w.with_flag(remove_Fa)
    s = Sim.from_workload(w)
    s.step(w.steps if steps is None else steps)
    return s
