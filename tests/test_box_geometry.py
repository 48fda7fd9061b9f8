"""Host-side model of the shared-memory box geometry of the semi-Lagrangian
steps (k_sl_pipe) and the box foot points (k_footpoints_box): both place each
tile's box at the tile's own floor range (the box entry), and for every voxel
of every tile whose floor range fits the box, each of the 64 stencil taps the
kernel reads (box row and column from the voxel's floors, the tile origin and
the 16-byte chunk shift) lies inside the part of the box the copy writes, and
that slot holds the periodic grid sample the cubic stencil of the paper's
interpolation (Section 4.1) needs.  The tile, box and chunk constants are read
from the CUDA source, so the model follows the kernel's geometry.  No GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2008_12820_gb300", "csrc", "transport.cu")


def constants():
    s = open(SRC).read()
    pt = re.search(r"constexpr int PT3 = (\d+), PT2 = (\d+), PT1 = (\d+);", s)
    span = re.search(r"constexpr int BOX_SPAN = (\d+);", s)
    pitch = re.search(r"constexpr int BOX_PITCH = (\d+);", s)
    ch = re.search(r"constexpr int BOX_CH = (\d+);", s)
    assert pt and span and pitch and ch
    return dict(PT3=int(pt.group(1)), PT2=int(pt.group(2)), PT1=int(pt.group(3)), SPAN=int(span.group(1)),
                PITCH=int(pitch.group(1)), CH=int(ch.group(1)))


C = constants()
BS1, BS2, BS3 = C["PT1"] + 3 + C["SPAN"], C["PT2"] + 3 + C["SPAN"], C["PT3"] + 3 + C["SPAN"]


def floor_int(x):
    return np.clip(np.floor(x), -1e6, 1e6).astype(np.int64)


def box_contents(lo1, lo2, lo3, shape, chunked):
    """global (i1, i2, i3) held by each box slot [row, column]; -1 where the copy writes nothing"""
    n1, n2, n3 = shape
    box = -np.ones((BS1 * BS2, C["PITCH"], 3), np.int64)
    for row in range(BS1 * BS2):
        z, y = divmod(row, BS2)
        g1, g2 = (lo1 + z) % n1, (lo2 + y) % n2
        if chunked:
            for lch in range(C["CH"]):
                gx = ((lo3 & ~3) + 4 * lch) % n3
                assert gx % 4 == 0 and gx + 3 < n3          # whole 16-byte chunks inside the row
                box[row, 4 * lch:4 * lch + 4] = [(g1, g2, gx + k) for k in range(4)]
        else:
            for col in range(BS3):
                box[row, col] = (g1, g2, (lo3 + col) % n3)
    return box


def check_tiles(shape, disp, per_tile):
    """disp: [3][n1][n2][n3] displacement (index units) of each voxel's stencil
    origin; per_tile: floor range of the tile (the kernels' box entries) or of
    the whole field"""
    n1, n2, n3 = shape
    chunked = n3 % 4 == 0
    fl = floor_int(disp)
    lo_field, hi_field = fl.reshape(3, -1).min(1), fl.reshape(3, -1).max(1)
    fits = checked = 0
    for t1 in range(-(-n1 // C["PT1"])):
        for t2 in range(-(-n2 // C["PT2"])):
            for t3 in range(-(-n3 // C["PT3"])):
                sl = (slice(t1 * C["PT1"], (t1 + 1) * C["PT1"]), slice(t2 * C["PT2"], (t2 + 1) * C["PT2"]),
                      slice(t3 * C["PT3"], (t3 + 1) * C["PT3"]))
                f = fl[(slice(None),) + sl]
                lo, hi = (f.reshape(3, -1).min(1), f.reshape(3, -1).max(1)) if per_tile else (lo_field, hi_field)
                if np.any(hi - lo > C["SPAN"]) or np.any(lo <= -1000000) or np.any(hi >= 1000000):
                    continue                                   # the tile gathers from global memory
                fits += 1
                lo1, lo2, lo3 = t1 * C["PT1"] + lo[0] - 1, t2 * C["PT2"] + lo[1] - 1, t3 * C["PT3"] + lo[2] - 1
                box = box_contents(lo1, lo2, lo3, shape, chunked)
                sh = lo3 - (lo3 & ~3) if chunked else 0
                i1, i2, i3 = np.meshgrid(*(np.arange(s.start, min(s.stop, n)) for s, n in zip(sl, shape)),
                                         indexing="ij")
                f1, f2, f3 = f[0].ravel(), f[1].ravel(), f[2].ravel()
                i1, i2, i3 = i1.ravel(), i2.ravel(), i3.ravel()
                b1 = i1 - t1 * C["PT1"] + f1 - lo[0]
                b2 = i2 - t2 * C["PT2"] + f2 - lo[1]
                b3 = i3 - t3 * C["PT3"] + f3 - lo[2] + sh
                for a in range(4):
                    for b in range(4):
                        row = (b1 + a) * BS2 + (b2 + b)
                        assert row.min() >= 0 and row.max() < BS1 * BS2
                        for c in range(4):
                            col = b3 + c
                            assert col.min() >= 0 and col.max() < C["PITCH"]
                            want = np.stack([(i1 + f1 + a - 1) % n1, (i2 + f2 + b - 1) % n2,
                                             (i3 + f3 + c - 1) % n3], -1)
                            assert (box[row, col] == want).all()
                            checked += row.size
    return fits, checked


def smooth_disp(shape, amp, seed):
    rng = np.random.default_rng(seed)
    x = np.meshgrid(*(np.arange(n) * 2 * np.pi / n for n in shape), indexing="ij")
    return np.stack([amp * np.sin(x[0] + rng.uniform(0, 6)) * np.cos(x[1] + rng.uniform(0, 6))
                     + amp * rng.uniform(-1, 1) for _ in range(3)]).astype(np.float32)


@pytest.mark.parametrize("shape,amp,seed", [((24, 32, 40), 0.6, 1), ((16, 24, 33), 0.8, 2),
                                            ((12, 20, 36), 1.6, 3), ((9, 10, 64), 1.2, 4)])
def test_foot_point_boxes_cover_every_tap(shape, amp, seed):
    # k_footpoints_box: the predictor displacement -dt v/h with the tile's own floor range
    fits, checked = check_tiles(shape, smooth_disp(shape, amp, seed), per_tile=True)
    assert fits > 0 and checked > 0


@pytest.mark.parametrize("shape,amp,seed", [((24, 32, 40), 0.5, 5), ((20, 16, 33), 0.9, 6), ((32, 64, 64), 3.0, 7),
                                            ((32, 64, 64), 5.0, 7)])
def test_sl_step_boxes_cover_every_tap(shape, amp, seed):
    # k_sl_pipe: the foot-point displacement with each tile's own floor range
    disp = smooth_disp(shape, amp, seed)
    fits, checked = check_tiles(shape, disp, per_tile=True)
    assert fits > 0 and checked > 0
    if amp > 2:
        # displacements of several cells: a field-wide range would send every
        # tile to the gather path; per tile, all (amp 3) or some (amp 5) fit
        assert check_tiles(shape, disp, per_tile=False)[0] == 0
        ntiles = np.prod([-(-n // c) for n, c in zip(shape, (C["PT1"], C["PT2"], C["PT3"]))])
        assert (fits == ntiles) if amp < 4 else (0 < fits < ntiles)


def test_wide_or_nonfinite_ranges_leave_the_box_path():
    # a span beyond the box, or a clamped (non-finite) floor, never takes the box path,
    # and only the tile that holds it leaves
    assert np.all(floor_int(np.array([np.inf, -np.inf, 3e9])) == [1e6, -1e6, 1e6])
    shape = (8, 8, 32)
    disp = np.zeros((3,) + shape, np.float32)
    disp[0, 0, 0, 0] = C["SPAN"] + 1.5
    fits, _ = check_tiles(shape, disp, per_tile=False)
    assert fits == 0
    fits, _ = check_tiles(shape, disp, per_tile=True)
    ntiles = (8 // C["PT1"]) * (8 // C["PT2"]) * (32 // C["PT3"])
    assert fits == ntiles - 1
    # every displacement infinite: a span of 0 at the clamp, still not the box
    fits, _ = check_tiles(shape, np.full((3,) + shape, np.inf, np.float32), per_tile=True)
    assert fits == 0
