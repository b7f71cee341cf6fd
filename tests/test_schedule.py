"""Work items and the dependency lists of the persistent launch (host logic, no GPU).

An item of step k of the persistent launch may start once every item listed for it has finished
step k - 1.  The lists must therefore cover every item of the same lattice whose region meets
the rows and columns the item reads (its rows z0 - 2 .. z1 + 1 and columns x0 - 4 .. x0 + w + 3,
periodic in x: pull streaming, neighbour densities, the 16-byte aligned staging window), which is
also the set of items that read the region it overwrites.  Checked here by brute force.
"""
import numpy as np
import pytest

from paper_1808_05168_gb300 import capi


CASES = [
    ([(128, 32), (256, 64), (512, 128), (1024, 256)], 128, 64),
    ([(128, 32), (256, 64), (512, 128), (1024, 256)], 128, 256),
    ([(128, 32)], 32, 5),
    ([(128, 32)], 256, 32),
    ([(128, 32)], 64, 1),
    ([(16, 8), (64, 8)], 32, 3),
    ([(8, 4)], 128, 1),
    ([(64, 16), (96, 12)], 32, 2),
]


@pytest.mark.parametrize("shapes,tile,rows", CASES)
def test_items_partition_every_lattice(shapes, tile, rows):
    items, off, nbr = capi.lb_debug_schedule(shapes, tile, rows)
    for lat, (Lx, Lz) in enumerate(shapes):
        cover = np.zeros((Lz, Lx), np.int32)
        for m, x0, z0, z1 in items:
            if m == lat:
                cover[z0:z1, x0:min(x0 + tile, Lx)] += 1
        assert (cover == 1).all()
    # longest row chunks first, the items of one lattice contiguous
    chunk = [min(rows, shapes[m][1]) for m in items[:, 0]]
    assert chunk == sorted(chunk, reverse=True)
    lat_seq = [int(m) for m in items[:, 0]]
    assert sum(1 for a, b in zip(lat_seq, lat_seq[1:]) if a != b) == len(shapes) - 1


@pytest.mark.parametrize("shapes,tile,rows", CASES)
def test_dependency_lists_cover_the_read_halo(shapes, tile, rows):
    items, off, nbr = capi.lb_debug_schedule(shapes, tile, rows)
    n = len(items)
    assert off[0] == 0 and off[-1] == len(nbr) and (np.diff(off) >= 1).all()
    lists = [set(nbr[off[i]:off[i + 1]].tolist()) for i in range(n)]
    width = lambda m, x0: min(tile, shapes[m][0] - x0)
    for i, (lat, x0, z0, z1) in enumerate(items):
        Lx, Lz = shapes[lat]
        rows_read = set(range(max(0, z0 - 2), min(Lz - 1, z1 + 1) + 1))
        cols_read = {c % Lx for c in range(x0 - 4, x0 + width(lat, x0) + 4)}
        need = {j for j, (m, y0, v0, v1) in enumerate(items)
                if m == lat and rows_read & set(range(v0, v1)) and cols_read & set(range(y0, y0 + width(m, y0)))}
        assert i in lists[i]
        assert need <= lists[i], (i, sorted(need - lists[i]))
        assert all(items[j][0] == lat for j in lists[i])
    # symmetric: whoever item i waits for also waits for i
    for i in range(n):
        for j in lists[i]:
            assert i in lists[j]


def test_schedule_sizes_and_errors():
    ni, nn = capi.ctypes.c_int64(), capi.ctypes.c_int64()
    lx = np.array([64], np.int32)
    lz = np.array([16], np.int32)
    lib = capi.load()
    assert lib.lb_debug_schedule(1, capi._iptr(lx), capi._iptr(lz), 32, 4, None, 0, None, None, 0,
                                 capi.ctypes.byref(ni), capi.ctypes.byref(nn)) == capi.LB_ERR_SIZE
    assert ni.value == 8 and nn.value > 0
    assert lib.lb_debug_schedule(1, capi._iptr(lx), capi._iptr(lz), 0, 4, None, 0, None, None, 0,
                                 capi.ctypes.byref(ni), capi.ctypes.byref(nn)) == capi.LB_ERR_BAD_PARAM
