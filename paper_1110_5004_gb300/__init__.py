"""GB300-native two-distribution D2Q9 multiphase lattice Boltzmann library (Python side).

Thin layer over the C ABI in ``include/lbm.h``: every step of the method runs in the CUDA
kernels of ``liblbm.so``; this module only marshals arguments.  PyTorch is used for device
buffers and streams when the caller passes tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (LBM_BF16_DEV, LBM_ERR_BUDGET, LBM_ERR_DIVERGED, LBM_FP16_DEV, LBM_FP32,
                   LBM_KERNEL_AUTO, LBM_KERNEL_RESIDENT, LBM_KERNEL_ROWS, LBM_KERNEL_TILES, LBM_PERIODIC, LBM_WALL,
                   LBMError, lbm_diag, lbm_params)

__all__ = ["Sim", "Batch", "LBMError", "params_from_physical", "lbm_params", "LBM_FP32",
           "LBM_FP16_DEV", "LBM_BF16_DEV", "LBM_PERIODIC", "LBM_WALL", "LBM_ERR_DIVERGED",
           "LBM_ERR_BUDGET", "LBM_KERNEL_AUTO", "LBM_KERNEL_ROWS", "LBM_KERNEL_TILES", "LBM_KERNEL_RESIDENT",
           "device_bytes"]


def lib():
    return _lib.load()


def _ptr(a):
    """Address of a host numpy array or a device torch tensor (float32, contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags.c_contiguous, "float32 C-contiguous array required"
        return a.ctypes.data
    # torch tensor
    assert a.dtype.__repr__().endswith("float32") and a.is_contiguous(), "float32 contiguous tensor required"
    return a.data_ptr()


def _bptr(a):
    """Address of any C-contiguous host numpy array or contiguous device torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "C-contiguous array required"
        return a.ctypes.data
    assert a.is_contiguous(), "contiguous tensor required"
    return a.data_ptr()


def _nbytes(a):
    return int(a.nbytes) if isinstance(a, np.ndarray) else int(a.numel() * a.element_size())


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream   # torch.cuda.Stream


def params_from_physical(phys, storage=LBM_FP32) -> lbm_params:
    """Scheme parameters of a ``workloads.Physical`` record, converted by the library."""
    b, k = ctypes.c_double(), ctypes.c_double()
    _lib.check(lib().lbm_params_from_sigma_W(phys.sigma, phys.W, phys.phi_star, ctypes.byref(b),
                                             ctypes.byref(k)))
    return lbm_params(beta=b.value, kappa=k.value, phi_star=phys.phi_star, theta_M=phys.theta_M,
                      tau_f=phys.tau_f, tau_g_A=lib().lbm_tau_from_nu(phys.nu_A),
                      tau_g_B=lib().lbm_tau_from_nu(phys.nu_B), rho_A=phys.rho_A,
                      rho_B=phys.rho_B, gravity=phys.gravity, bc_x=phys.bc_x, bc_y=phys.bc_y,
                      remove_Fa=phys.remove_Fa, storage=storage,
                      ch_conservative=phys.ch_conservative, fs_form=phys.fs_form, s_form=phys.s_form,
                      f_form=phys.f_form)


def device_bytes(nx, ny, storage=LBM_FP32) -> int:
    return int(lib().lbm_device_bytes(nx, ny, storage))


class Sim:
    """One simulation with device-resident state (owned by the library)."""

    def __init__(self, nx, ny, params: lbm_params, stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.params = params
        h = ctypes.c_void_p()
        _lib.check(lib().lbm_create(self.nx, self.ny, ctypes.byref(params), _stream_handle(stream),
                                    ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_workload(cls, w, storage=LBM_FP32, stream=None, init=True, tile=None, kernel=None):
        """A simulation of workload `w`.  `tile` (threads, rows) shapes the row march and selects it
        unless `kernel` says otherwise; `kernel` is one of the LBM_KERNEL_* values."""
        s = cls(w.nx, w.ny, params_from_physical(w.phys, storage), stream=stream)
        if tile is not None:
            s.set_tile(*tile)
        if kernel is not None or tile is not None:
            s.set_kernel(LBM_KERNEL_ROWS if kernel is None else kernel)
        if init:
            s.init_fields(w.phi0, w.ux0, w.uy0, w.p0)
        return s

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, threads=0, seg_rows=0):
        """Tile of the step kernel: threads per CTA (64, 128 or 256) and rows per CTA; 0 keeps
        the current value of either (a simulation starts with as many rows per CTA as fill one
        wave of resident CTAs)."""
        _lib.check(lib().lbm_set_tile(self._h, int(threads), int(seg_rows)))

    def set_kernel(self, kernel):
        """Step kernel: LBM_KERNEL_AUTO, LBM_KERNEL_ROWS, LBM_KERNEL_TILES or LBM_KERNEL_RESIDENT
        (bitwise the same results; the tile kernels need s_form 0 and f_form 0)."""
        _lib.check(lib().lbm_set_kernel(self._h, int(kernel)))

    @property
    def active_kernel(self):
        """lbm_active_kernel: the LBM_KERNEL_* value lbm_step runs (AUTO resolved)."""
        return _lib.check_value(lib().lbm_active_kernel(self._h))

    def set_wait_limit(self, timeout_ns, hold_tile=-1):
        """lbm_set_wait_limit: bound of the resident kernel's waits; hold_tile >= 0 makes that
        tile never announce a finished step (the test of the bound)."""
        _lib.check(lib().lbm_set_wait_limit(self._h, int(timeout_ns), int(hold_tile)))

    def step_status(self):
        """lbm_step_status: LBM_OK (0), or LBM_ERR_TIMEOUT if a resident launch gave up since the
        last read (returned, not raised)."""
        return int(lib().lbm_step_status(self._h))

    def set_stream(self, stream):
        _lib.check(lib().lbm_set_stream(self._h, _stream_handle(stream)))

    def init_fields(self, phi0, ux0=None, uy0=None, p0=None):
        _lib.check(lib().lbm_init_fields(self._h, _ptr(phi0), _ptr(ux0), _ptr(uy0), _ptr(p0)))

    def init_fields_packed(self, fields):
        """lbm_init_fields_packed: phi0, ux0, uy0, p0 in one (4, ny, nx) float32 block (host
        array or device tensor), copied in one transfer."""
        _lib.check(lib().lbm_init_fields_packed(self._h, _ptr(fields)))

    def moments_packed(self, out=None):
        """lbm_moments_packed: phi, rho, ux, uy, p into one (5, ny, nx) float32 block (a new
        host array, or the given host array / device tensor)."""
        if out is None:
            out = np.empty((5, self.ny, self.nx), np.float32)
        _lib.check(lib().lbm_moments_packed(self._h, _ptr(out)))
        return out

    def step(self, n=1):
        _lib.check(lib().lbm_step(self._h, int(n)))

    @property
    def step_count(self):
        return int(lib().lbm_step_count(self._h))

    @property
    def launch_count(self):
        return int(lib().lbm_launch_count(self._h))

    @property
    def device_bytes(self):
        return int(lib().lbm_sim_device_bytes(self._h))

    @property
    def checkpoint_bytes(self):
        return int(lib().lbm_checkpoint_bytes(self._h))

    def checkpoint(self, out=None):
        """The current state as a checkpoint: into `out` (a host array or a device tensor of at
        least checkpoint_bytes bytes) or a new uint8 host array."""
        n = self.checkpoint_bytes
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        _lib.check(lib().lbm_checkpoint(self._h, _bptr(out), _nbytes(out)))
        return out

    def restore(self, buf):
        """Replace the state (and step count) by a checkpoint of a same-sized simulation."""
        _lib.check(lib().lbm_restore(self._h, _bptr(buf), _nbytes(buf)))

    def moments(self, out=None):
        """phi, rho, ux, uy, p as (ny, nx) float32 host arrays (or into the given dict of
        host arrays / device tensors)."""
        names = ("phi", "rho", "ux", "uy", "p")
        if out is None:
            out = {k: np.empty((self.ny, self.nx), np.float32) for k in names}
        _lib.check(lib().lbm_moments(self._h, *[_ptr(out.get(k)) for k in names]))
        return out

    def interfacial_force(self, out=None):
        """The additional interfacial force F_a = -u s of the current state (Eq. 12), whether or
        not the scheme removes it: fax, fay as (ny, nx) float32 host arrays (or into the given
        dict of host arrays / device tensors)."""
        names = ("fax", "fay")
        if out is None:
            out = {k: np.empty((self.ny, self.nx), np.float32) for k in names}
        _lib.check(lib().lbm_interfacial_force(self._h, *[_ptr(out.get(k)) for k in names]))
        return out

    def diagnostics(self, raise_on_divergence=False):
        d = lbm_diag()
        rc = lib().lbm_diagnostics(self._h, ctypes.byref(d))
        if rc != 0 and (rc != LBM_ERR_DIVERGED or raise_on_divergence):
            _lib.check(rc)
        return d.as_dict()


class Batch:
    """Ragged batch: member simulations advance together, one persistent launch per step."""

    def __init__(self, budget_bytes=0, stream=None):
        h = ctypes.c_void_p()
        _lib.check(lib().lbm_batch_create(int(budget_bytes), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.members = {}

    def add(self, sim: Sim) -> int:
        slot = ctypes.c_int()
        _lib.check(lib().lbm_batch_add(self._h, sim.handle, ctypes.byref(slot)))
        self.members[slot.value] = sim
        return slot.value

    def try_add(self, sim: Sim):
        """Slot, or None when the budget is exhausted."""
        slot = ctypes.c_int()
        rc = lib().lbm_batch_add(self._h, sim.handle, ctypes.byref(slot))
        if rc == LBM_ERR_BUDGET:
            return None
        _lib.check(rc)
        self.members[slot.value] = sim
        return slot.value

    def remove(self, slot: int):
        _lib.check(lib().lbm_batch_remove(self._h, int(slot)))
        return self.members.pop(slot)

    def step(self, k=1):
        _lib.check(lib().lbm_batch_step(self._h, int(k)))

    def set_tile(self, threads=0, seg_rows=0):
        """Tile of the batch kernel for members without their own rows per CTA; 0 keeps the
        current value of either."""
        _lib.check(lib().lbm_batch_set_tile(self._h, int(threads), int(seg_rows)))

    @property
    def size(self):
        return int(lib().lbm_batch_size(self._h))

    @property
    def bytes(self):
        return int(lib().lbm_batch_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
