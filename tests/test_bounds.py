"""Out-of-bounds detection without a sanitizer: every row of a simulation's state is padded from
nx to a pitch of 32 cells, and no kernel may read or write those pad columns.  The pads of both
ping-pong buffers are filled with NaN patterns through the checkpoint interface; after each step
they must still hold the pattern (nothing wrote them) and the interior must equal a run without
poison bitwise (nothing read them: a NaN would spread).

Checkpoint payload (version 2): ny rows of pitch / 32 blocks; a block holds every population
plane of its 32 cells in turn (FP32: 19 planes of 32 floats; 16-bit: one plane of 32 floats,
then 17 planes of 32 halves); the s_form planes follow as 2 x ny x pitch floats."""
import dataclasses

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
HEADER = 64
POISON32 = np.uint32(0x7FC0DEAD)                          # a quiet NaN
POISON16 = {1: np.uint16(0x7E01), 2: np.uint16(0x7FC1)}   # FP16 / BF16 quiet NaNs


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_5004_gb300 import build
    build.build()
    import paper_1110_5004_gb300 as m
    return m


def views(buf, nx, ny, storage, s_form):
    """(32-bit planes, 16-bit planes, s_form planes) of a checkpoint's payload, each as a
    (planes, ny, pitch) view of the payload (the blocked population layout, unblocked by
    strides)."""
    pitch = (nx + 31) // 32 * 32
    nb = pitch // 32
    plane = ny * pitch
    payload = buf[HEADER:]
    n32 = 19 if storage == 0 else 1
    n16 = 0 if storage == 0 else 17
    blk = 4 * 32 * n32 + 2 * 32 * n16
    pop = payload[:ny * nb * blk].reshape(ny, nb, blk)
    off = ny * nb * blk
    extra = payload[off:off + 8 * plane * s_form].view(np.uint32).reshape(2 * s_form, ny, pitch)
    assert off + 8 * plane * s_form == payload.size
    return Unblocked(pop, n32, n16, 32), Unblocked(pop, n32, n16, 16), extra


class Unblocked:
    """Read/write access to the 32- or 16-bit planes of a blocked payload as [plane, y, x]."""

    def __init__(self, pop, n32, n16, bits):
        self.pop, self.n32, self.n16, self.bits = pop, n32, n16, bits
        ny, nb, _ = pop.shape
        self.shape = (n32 if bits == 32 else n16, ny, nb * 32)

    def _blocks(self):
        ny, nb, _ = self.pop.shape
        if self.bits == 32:
            return self.pop[:, :, :4 * 32 * self.n32].view(np.uint32).reshape(ny, nb, self.n32, 32)
        return self.pop[:, :, 4 * 32 * self.n32:].view(np.uint16).reshape(ny, nb, self.n16, 32)

    def get(self):
        b = self._blocks()
        return b.transpose(2, 0, 1, 3).reshape(self.shape)

    def set_columns_from(self, x0, value):
        """Write `value` into columns >= x0 of every plane and row (in place)."""
        b = self._blocks()
        ny, nb, npl, _ = b.shape
        for x in range(x0, nb * 32):
            b[:, x // 32, :, x % 32] = value


def poison(buf, nx, ny, storage, s_form):
    a32, a16, extra = views(buf, nx, ny, storage, s_form)
    a32.set_columns_from(nx, POISON32)
    extra[:, :, nx:] = POISON32
    if storage:
        a16.set_columns_from(nx, POISON16[storage])


def check(buf, ref, nx, ny, storage, s_form):
    g32, g16, gx = views(buf, nx, ny, storage, s_form)
    r32, r16, rx = views(ref, nx, ny, storage, s_form)
    g32, g16, r32, r16 = g32.get(), g16.get(), r32.get(), r16.get()
    assert (g32[:, :, nx:] == POISON32).all() and (gx[:, :, nx:] == POISON32).all(), "a pad was written"
    if storage:
        assert (g16[:, :, nx:] == POISON16[storage]).all(), "a pad was written"
    assert np.array_equal(g32[:, :, :nx], r32[:, :, :nx]) and np.array_equal(g16[:, :, :nx], r16[:, :, :nx])
    assert np.array_equal(gx[:, :, :nx], rx[:, :, :nx]), "a pad was read"


CASES = [
    # nx, ny, bc_x, bc_y, storage, s_form, tile
    (33, 21, W.PERIODIC, W.WALL, 0, 0, (64, 5)),
    (77, 40, W.WALL, W.WALL, 0, 1, (128, 16)),
    (130, 37, W.PERIODIC, W.PERIODIC, 0, 0, (64, 0)),
    (250, 29, W.WALL, W.PERIODIC, 0, 0, (256, 8)),
    (95, 33, W.PERIODIC, W.WALL, 1, 0, (128, 7)),
    (61, 26, W.WALL, W.WALL, 2, 1, (64, 9)),
]


@pytest.mark.parametrize("kernel", ["rows", "tiles"])
@pytest.mark.parametrize("nx,ny,bcx,bcy,st,sform,tile", CASES)
def test_pad_columns_never_touched(lbm, nx, ny, bcx, bcy, st, sform, tile, kernel):
    if kernel == "tiles" and sform:
        pytest.skip("the tile kernel runs s_form 0 only")
    w = W.random_small(nx, ny, seed=nx + ny, bc_x=bcx, bc_y=bcy, gravity=1e-5 if bcy == W.WALL else 0.0,
                       remove_Fa=1)
    w = dataclasses.replace(w, phys=dataclasses.replace(w.phys, s_form=sform))
    k = lbm.LBM_KERNEL_ROWS if kernel == "rows" else lbm.LBM_KERNEL_TILES
    sim = lbm.Sim.from_workload(w, tile=tile, storage=st, kernel=k)
    ref = lbm.Sim.from_workload(w, tile=tile, storage=st, kernel=k)
    # poison the pads of the current buffer, step once, then those of the other buffer
    for _ in range(2):
        c = sim.checkpoint()
        poison(c, nx, ny, st, sform)
        sim.restore(c)
        sim.step(1)
        ref.step(1)
    c = sim.checkpoint()
    poison(c, nx, ny, st, sform)
    sim.restore(c)
    for _ in range(6):
        sim.step(1)
        ref.step(1)
        check(sim.checkpoint(), ref.checkpoint(), nx, ny, st, sform)
    m = sim.moments()
    assert all(np.isfinite(v).all() for v in m.values())
