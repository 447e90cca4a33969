"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports every
function include/lbm.h declares, its host-only helpers agree with the oracle's independent
conversions, and invalid arguments are rejected before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as lbm
    return lbm.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    from paper_1110_5004_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def test_params_from_sigma_W_matches_oracle(L):
    import oracle
    for sigma, W, ps in ((0.01, 4.0, 1.0), (4e-5, 5.0, 1.0), (0.002, 3.0, 0.7)):
        b, k = ctypes.c_double(), ctypes.c_double()
        assert L.lbm_params_from_sigma_W(sigma, W, ps, ctypes.byref(b), ctypes.byref(k)) == 0
        ob, ok = oracle.params_from_sigma_W(sigma, W, ps)
        assert b.value == pytest.approx(ob, rel=1e-15) and k.value == pytest.approx(ok, rel=1e-15)
        assert L.lbm_tau_from_nu(sigma) == pytest.approx(oracle.tau_from_nu(sigma), rel=1e-15)
    b, k = ctypes.c_double(), ctypes.c_double()
    assert L.lbm_params_from_sigma_W(-1.0, 4.0, 1.0, ctypes.byref(b), ctypes.byref(k)) == -1
    assert b"positive" in L.lbm_last_error()


def test_c1_coefficients(L):
    """c1 (W = 4, sigma = 0.01, phi* = 1): kappa = 0.015, beta = 0.001875."""
    b, k = ctypes.c_double(), ctypes.c_double()
    L.lbm_params_from_sigma_W(0.01, 4.0, 1.0, ctypes.byref(b), ctypes.byref(k))
    assert k.value == pytest.approx(0.015) and b.value == pytest.approx(0.001875)


def _params(**kw):
    from paper_1110_5004_gb300 import lbm_params
    base = dict(beta=0.001875, kappa=0.015, phi_star=1.0, theta_M=0.1, tau_f=0.8, tau_g_A=0.8,
                tau_g_B=0.8, rho_A=1.0, rho_B=0.1, gravity=0.0, bc_x=0, bc_y=0, remove_Fa=0, storage=0)
    base.update(kw)
    return lbm_params(**base)


@pytest.mark.parametrize("nx,ny,kw,msg", [
    (2, 16, {}, b"too small"),
    (16, 3, {"bc_y": 1}, b"too small"),
    (16, 16, {"tau_f": 0.5}, b"relaxation"),
    (16, 16, {"tau_g_B": 0.4}, b"relaxation"),
    (16, 16, {"rho_B": 0.0}, b"densities"),
    (16, 16, {"kappa": -1.0}, b"positive"),
    (16, 16, {"theta_M": -0.1}, b"theta_M"),
    (16, 16, {"bc_x": 7}, b"bc_x"),
    (1 << 16, 1 << 16, {}, b"too large"),
    (16, 16, {"storage": 3}, b"storage"),
    (16, 16, {"ch_conservative": 2}, b"ch_conservative"),
    (16, 16, {"fs_form": -1}, b"fs_form"),
    (16, 16, {"s_form": 5}, b"s_form"),
    (16, 16, {"f_form": 2}, b"f_form"),
    (16, 16, {"f_form": 1, "storage": 1}, b"FP32"),
])
def test_invalid_arguments_rejected_on_host(L, nx, ny, kw, msg):
    h = ctypes.c_void_p()
    rc = L.lbm_create(nx, ny, ctypes.byref(_params(**kw)), None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert msg in L.lbm_last_error()


def test_null_handles(L):
    assert L.lbm_step(None, 1) == -1
    assert L.lbm_destroy(None) == 0
    assert L.lbm_step_count(None) == -1
    assert L.lbm_create(8, 8, None, None, None) == -1
    assert L.lbm_strerror(-4) == b"simulation diverged"
    assert L.lbm_checkpoint_bytes(None) == 0 and L.lbm_sim_device_bytes(None) == 0
    buf = (ctypes.c_ubyte * 64)()
    assert L.lbm_checkpoint(None, buf, 64) == -1
    assert L.lbm_restore(None, buf, 64) == -1
    assert L.lbm_interfacial_force(None, None, None) == -1 and L.lbm_moments(None, None, None, None, None, None) == -1


def test_params_layout_zero_defaults():
    """A zero-initialised lbm_params selects the paper's forms: convective Cahn-Hilliard
    (ch_conservative = 0), F_s = -phi grad(mu) (fs_form = 0), mass defect by Eq. 5 (s_form = 0);
    the struct is 10 doubles + 8 ints with no padding, as include/lbm.h declares it."""
    from paper_1110_5004_gb300 import lbm_params
    p = lbm_params()
    assert (p.ch_conservative, p.fs_form, p.s_form, p.f_form, p.remove_Fa) == (0, 0, 0, 0, 0)
    assert ctypes.sizeof(lbm_params) == 10 * 8 + 8 * 4


def test_device_bytes_accounting(L):
    # 2 x 19 FP32 planes (f, gbar, low half of f_0) + 6 field planes with a 32-element row
    # pitch + FP64 reduction scratch
    n = L.lbm_device_bytes(100, 10, 0)
    assert n == 2 * 19 * 10 * 128 * 4 + 6 * 10 * 128 * 4 + (10 * 12 + 16) * 8
