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


def assert_same_record(got, want, call):
    assert got["step"] == want["step"]
    for k in want:
        if k == "step":
            continue
        assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-15), (call, k)


# nx = 96 runs one column per thread of the row kernel; nx = 600 also runs its strided loop
# (more columns than its 256 threads).
@pytest.mark.parametrize("nx,ny", [(96, 160), (600, 90)])
def test_noalloc_diagnostics_match_simulation_diagnostics_twice(lbm, nx, ny):
    import torch
    from paper_1110_5004_gb300 import _lib
    L = lbm.lib()
    w = W.falling_droplet(nx=nx, ny=ny, R=20.0, yc=0.6 * ny, ratio=10.0, steps=0)
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
        assert_same_record(got, want, call)


def test_noalloc_device_record_on_a_side_stream_twice(lbm):
    """A device lbm_diag written asynchronously on a non-default stream, by two calls in a row
    that reuse the shared scratch; both records are read after one synchronisation."""
    import torch
    from paper_1110_5004_gb300 import _lib
    L = lbm.lib()
    w = W.falling_droplet(nx=300, ny=120, R=18.0, yc=70.0, ratio=10.0, steps=0)
    side = torch.cuda.Stream()
    sim = lbm.Sim.from_workload(w, stream=side)
    nrec = ctypes.sizeof(_lib.lbm_diag)
    recs = torch.zeros((2, nrec), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()   # the zero fill ran on the default stream
    wants, keep = [], []
    for call, steps in enumerate((30, 20)):
        sim.step(steps)
        with torch.cuda.stream(side):
            fields = {k: torch.empty((w.ny, w.nx), device="cuda") for k in ("phi", "rho", "ux", "uy", "p")}
        sim.moments(fields)
        wants.append(sim.diagnostics())
        rc = L.lbm_diagnostics_fields_noalloc(
            fields["phi"].data_ptr(), fields["ux"].data_ptr(), fields["uy"].data_ptr(), fields["p"].data_ptr(),
            w.nx, w.ny, w.phys.phi_star, sim.step_count, side.cuda_stream,
            ctypes.cast(recs[call].data_ptr(), ctypes.POINTER(_lib.lbm_diag)))
        assert rc == 0, L.lbm_last_error()
        keep.append(fields)
    side.synchronize()
    host = recs.cpu().numpy()
    for call in range(2):
        got = _lib.lbm_diag.from_buffer_copy(host[call].tobytes()).as_dict()
        assert got["step"] == wants[call]["step"]
        assert_same_record(got, wants[call], call)


def test_noalloc_at_the_row_limit(lbm):
    """ny = 8192, the size of the fixed scratch, is accepted and reduces like the simulation."""
    import torch
    from paper_1110_5004_gb300 import _lib
    L = lbm.lib()
    ny, nx = 8192, 40
    y = torch.arange(ny, device="cuda", dtype=torch.float32)[:, None]
    x = torch.arange(nx, device="cuda", dtype=torch.float32)[None, :]
    phi = torch.tanh((y - 3000.0) / 2.0) * torch.ones_like(x)
    ux = 1e-3 * torch.sin(x / 7.0) * torch.ones_like(y)
    uy = 1e-3 * torch.cos(y / 13.0) * torch.ones_like(x)
    p = 1e-4 * phi
    fields = {"phi": phi.contiguous(), "ux": ux.contiguous(), "uy": uy.contiguous(), "p": p.contiguous()}
    out = _lib.lbm_diag()
    rc = noalloc(L, fields, nx, ny, 1.0, 7, None, out)
    assert rc == 0, L.lbm_last_error()
    got = out.as_dict()
    ph = fields["phi"].double().cpu().numpy()
    c = np.clip((ph + 1.0) / 2.0, 0.0, 1.0)
    assert got["step"] == 7
    assert got["sum_phi"] == pytest.approx(ph.sum(), rel=1e-12, abs=1e-9)
    assert got["liquid_area"] == pytest.approx(c.sum(), rel=1e-12)
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    assert got["centroid_y"] == pytest.approx((c * yy).sum() / c.sum(), rel=1e-12)


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
