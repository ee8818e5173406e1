"""The lattice geometry of the measured workloads (the paper gives pictures only): bond counts,
coordination and the stated sector dimensions."""
import math
from collections import Counter

import workloads as wl


def test_ring_bonds():
    b1, b2 = wl.ring_bonds(28, 1), wl.ring_bonds(28, 2)
    assert len(b1) == 28 and len(b2) == 28 and not set(b1) & set(b2)
    deg = Counter([i for e in b1 for i in e])
    assert set(deg.values()) == {2}


def test_square_torus_bonds():
    for lx in (4, 6):
        b = wl.square_bonds(lx, lx)
        assert len(b) == 2 * lx * lx and len(set(map(frozenset, b))) == len(b)
        deg = Counter([i for e in b for i in e])
        assert set(deg.values()) == {4}


def test_honeycomb_bonds():
    b = wl.honeycomb_bonds(4, 3)
    assert len(b) == 36
    assert Counter(lab for _, _, lab in b) == {"x": 12, "y": 12, "z": 12}
    deg = Counter()
    for i, j, lab in b:
        assert (i % 2) != (j % 2)  # every bond joins an A site to a B site
        deg[(i, lab)] += 1
        deg[(j, lab)] += 1
    assert set(deg.values()) == {1} and len(deg) == 24 * 3  # one bond of each kind per site


def test_workload_sizes():
    assert wl.workload("hubbard_4x4_8u8d")["dim"] == math.comb(16, 8) ** 2 == 165_636_900
    assert wl.workload("heisenberg_6x6_sz0")["dim"] == math.comb(36, 18) == 9_075_135_300
    assert sum(math.comb(28, n) for n in wl.workload("j1j2_ring28_all_sectors")["sectors"]) == 1 << 28
    k = wl.workload("kitaev_24_tpq64")
    assert k["dim"] == 1 << 24 and k["n_starts"] == 64 and k["model"].n_sites == 24
