"""The frame-staggered item order of the persistent CG kernel (CPU only,
through the host test hook of the library).

The persistent kernel hands out tickets; an item waits only for the previous
phase of its own frame.  A launch can only hang if some item waits for an
item with a larger ticket.  These tests decode every ticket of small orders
and check that, for tables of independent frames, the order is a bijection
onto the items and every dependency points to smaller tickets:
  - a frame-iteration's update chunks come after all its normal-product tiles;
  - a frame's tiles at iteration k + 1 come after all its update chunks at k.
"""
import ctypes
import itertools

import pytest

from paper_1807_11830_gb300 import build as sense_build


@pytest.fixture(scope="module")
def lib():
    lib = ctypes.CDLL(sense_build.build())
    lib.sense_testing_staggered_item.restype = None
    lib.sense_testing_staggered_item.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.sense_testing_persistent_lag.restype = ctypes.c_int
    lib.sense_testing_persistent_lag.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    return lib


def decode(lib, units, p1, p2, lag):
    out = (ctypes.c_int * 3)()
    items = {}
    for t in range(units * (p1 + p2)):
        lib.sense_testing_staggered_item(t, units, p1, p2, lag, out)
        key = (out[0], out[1], out[2])
        assert key not in items, (t, key)
        items[key] = t
    return items


@pytest.mark.parametrize("frames,iters,tiles,chunks", [(1, 5, 4, 2), (3, 4, 5, 3), (20, 3, 32, 8), (7, 6, 2, 9)])
def test_cg_order_is_a_bijection_with_backward_waits(lib, frames, iters, tiles, chunks):
    units = frames * iters
    for lag in range(frames):  # every stagger the kernel accepts: 0 .. frames - 1
        items = decode(lib, units, tiles, chunks, lag)
        want = {(0, u, p) for u in range(units) for p in range(tiles)} | \
               {(1, u, p) for u in range(units) for p in range(chunks)}
        assert set(items) == want
        for u in range(units):
            last_tile = max(items[(0, u, p)] for p in range(tiles))
            first_chunk = min(items[(1, u, p)] for p in range(chunks))
            assert last_tile < first_chunk, (lag, u)  # update waits for the same frame-iteration's tiles
            if u + frames < units:  # the frame's next iteration waits for this update
                last_chunk = max(items[(1, u, p)] for p in range(chunks))
                assert last_chunk < min(items[(0, u + frames, p)] for p in range(tiles)), (lag, u)


def test_update_lands_lag_stages_after_its_tiles(lib):
    frames, iters, tiles, chunks, lag = 6, 3, 4, 2, 3
    items = decode(lib, frames * iters, tiles, chunks, lag)
    order = sorted(items, key=items.get)
    # between a frame-iteration's last tile and its first chunk lie exactly the tiles of the next `lag` units
    for u in range(frames * iters - lag):
        a = items[(0, u, tiles - 1)]
        b = items[(1, u, 0)]
        between = order[a + 1:b]
        assert {(kind, v) for kind, v, _ in between if kind == 0} == {(0, v) for v in range(u + 1, u + lag + 1)}


def test_lag_choice(lib):
    for frames, tiles, grid in itertools.product((1, 2, 5, 20, 400), (8, 32, 40), (152, 304, 456)):
        d = lib.sense_testing_persistent_lag(frames, tiles, grid)
        assert 0 <= d <= max(frames - 1, 0)
        if frames > 1:
            assert d == min(frames - 1, -(-grid // tiles) + 1)
