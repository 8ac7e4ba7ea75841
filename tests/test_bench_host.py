"""Host-side parts of the benchmark's roofline, on the CPU: the count of BULK cells behind the
bulk sweep's algorithmic bytes (the cells whose 18 D3Q19 neighbours all carry PDFs or lie beyond
a wall) against a cell-by-cell count, and the recorded ncu traffic tied to the sources it was
captured on."""
import itertools
import re

import numpy as np
import pytest

import bench
from paper_1712_07028_gb300 import lbm


def _bulk_one_by_one(fl, bc):
    """a liquid cell counts if each of its 18 neighbours is liquid or interface, the periodic
    image standing in across a periodic face and nothing being needed beyond any other face"""
    nz, ny, nx = fl.shape
    L = (nx, ny, nz)
    carries = (lbm.CELL_LIQUID, lbm.CELL_INTERFACE)
    n = 0
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if fl[z, y, x] != lbm.CELL_LIQUID:
            continue
        ok = True
        for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
            if abs(dx) + abs(dy) + abs(dz) not in (1, 2):
                continue
            c = [x + dx, y + dy, z + dz]
            beyond = False
            for k in range(3):
                if not 0 <= c[k] < L[k]:
                    if bc[k]:
                        c[k] %= L[k]
                    else:
                        beyond = True
            if not beyond and fl[c[2], c[1], c[0]] not in carries:
                ok = False
                break
        n += ok
    return n


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)])
def test_bulk_cell_count_matches_a_cell_by_cell_count(bc):
    import torch
    rng = np.random.default_rng(11 + sum(b << k for k, b in enumerate(bc)))
    types = np.array([lbm.CELL_LIQUID] * 12 + [lbm.CELL_INTERFACE, lbm.CELL_GAS, lbm.CELL_OBSTACLE], dtype=np.uint8)
    fl = rng.choice(types, size=(7, 6, 9))
    want = _bulk_one_by_one(fl, bc)
    assert 0 < want < int((fl == lbm.CELL_LIQUID).sum())   # the case tells counted from not counted
    assert bench._bulk_cells(torch, lbm, torch.from_numpy(fl), bc) == want


def test_bulk_cell_count_of_an_all_liquid_box_and_of_a_single_obstacle():
    import torch
    fl = np.full((5, 4, 6), lbm.CELL_LIQUID, dtype=np.uint8)
    for bc in ((0, 0, 0), (1, 1, 1)):
        assert bench._bulk_cells(torch, lbm, torch.from_numpy(fl), bc) == fl.size
    fl[2, 2, 3] = lbm.CELL_OBSTACLE   # itself and its 18 neighbours drop out
    assert bench._bulk_cells(torch, lbm, torch.from_numpy(fl), (0, 0, 0)) == fl.size - 19


def test_recorded_traffic_is_keyed_by_workload_and_source_hash():
    sha = bench._sweep_sha()
    assert re.fullmatch(r"[0-9a-f]{40}", sha) and sha == bench._sweep_sha()
    for key, rec in bench.NCU_TRAFFIC.items():
        name, storage = key.split("/")
        assert storage in ("f32", "f16dev", "bf16dev") and name
        assert re.fullmatch(r"[0-9a-f]{40}", rec["sha1"])
        assert isinstance(rec["bytes_per_launch"], int) and rec["bytes_per_launch"] > 0
