"""The allocation-free diagnostics entry point, called through the C ABI.

lbm_diagnostics_fields_noalloc serves callers that cannot call cudaMalloc (a host application
that owns the device-memory budget): it reduces fields the caller holds on the device with its
partial sums in a fixed device array of the library.  This test compares it with the
simulation's own lbm_diagnostics on two calls in a row (two different states), and checks the
size limit.  It sits in a file collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as m
    return m


def noalloc(L, fields, nx, ny, phi_star, step, stream, out):
    return L.lbm_diagnostics_fields_noalloc(fields["phi"].data_ptr(), fields["ux"].data_ptr(),
                                            fields["uy"].data_ptr(), fields["p"].data_ptr(), nx, ny,
                                            phi_star, step, stream, ctypes.byref(out))


def test_noalloc_diagnostics_match_simulation_diagnostics_twice(lbm):
    import torch
    from paper_1110_5004_gb300 import _lib
    L = lbm.lib()
    w = W.falling_droplet(nx=96, ny=160, R=20.0, yc=100.0, ratio=10.0, steps=0)
    stream = torch.cuda.current_stream()
    sim = lbm.Sim.from_workload(w, stream=stream)
    for call, steps in enumerate((40, 25)):
        sim.step(steps)
        fields = {k: torch.empty((w.ny, w.nx), device="cuda") for k in ("phi", "rho", "ux", "uy", "p")}
        sim.moments(fields)
        want = sim.diagnostics()
        got = _lib.lbm_diag()
        rc = noalloc(L, fields, w.nx, w.ny, w.phys.phi_star, sim.step_count, stream.cuda_stream, got)
        assert rc == 0, L.lbm_last_error()
        got = got.as_dict()
        assert got["step"] == want["step"] == sim.step_count
        for k in want:
            if k == "step":
                continue
            assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-15), (call, k)


def test_noalloc_rejects_too_many_rows(lbm):
    import torch
    from paper_1110_5004_gb300 import _lib
    L = lbm.lib()
    t = torch.zeros((8193, 4), device="cuda")
    fields = {k: t for k in ("phi", "ux", "uy", "p")}
    out = _lib.lbm_diag()
    rc = noalloc(L, fields, 4, 8193, 1.0, 0, None, out)
    assert rc == _lib.LBM_ERR_INVALID_ARG
    assert b"8192" in L.lbm_last_error()
    host = np.zeros((4, 4), np.float32)
    rc = L.lbm_diagnostics_fields_noalloc(host.ctypes.data, host.ctypes.data, host.ctypes.data,
                                          host.ctypes.data, 4, 4, 1.0, 0, None, ctypes.byref(out))
    assert rc == _lib.LBM_ERR_INVALID_ARG
