"""Seeded synthetic inputs shared by the CUDA library's tests/benchmark and the oracle.

This module holds only *inputs*: lattice geometry (which sites are bonded), coupling
constants, basis choices and seeded random vectors.  It contains none of the method's
arithmetic (no matrix elements, ranks, signs, Lanczos or TPQ steps), so both sides can
import it without sharing any of the computation they are checked on.

Model families follow section 2.3 of the paper ("Fermion Hubbard" and "Spin" models);
the lattices follow section 2.4 (chains, square lattice, honeycomb), with the cluster
shapes chosen here because the paper shows them only as figures.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

SPIN = 0
HUBBARD = 1

BASIS_FULL = 0
BASIS_SZ = 1
BASIS_NUMBER = 2


@dataclasses.dataclass
class ModelSpec:
    """A two-body lattice Hamiltonian as a plain term list.

    couplings: (i, j, J) with J a 3x3 matrix of J^{ab} S_i^a S_j^b (a, b = x, y, z)
    fields:    (i, (hx, hy, hz)) meaning - h . S_i
    hops:      (i, j, spin, t) meaning - t c+_{i s} c_{j s} - conj(t) c+_{j s} c_{i s}
    onsite_U:  (i, U) meaning U n_{i up} n_{i dn}
    density:   (i, j, V) meaning V n_i n_j
    chem_pot:  (i, mu) meaning - mu n_i
    basis:     BASIS_FULL, BASIS_SZ (n_a = number of up spins) or
               BASIS_NUMBER (n_a = N_up, n_b = N_dn)
    """

    kind: int
    n_sites: int
    basis: int = BASIS_FULL
    n_a: int = 0
    n_b: int = 0
    couplings: List[Tuple[int, int, np.ndarray]] = dataclasses.field(default_factory=list)
    fields: List[Tuple[int, Tuple[float, float, float]]] = dataclasses.field(default_factory=list)
    hops: List[Tuple[int, int, int, complex]] = dataclasses.field(default_factory=list)
    onsite_U: List[Tuple[int, float]] = dataclasses.field(default_factory=list)
    density: List[Tuple[int, int, float]] = dataclasses.field(default_factory=list)
    chem_pot: List[Tuple[int, float]] = dataclasses.field(default_factory=list)
    name: str = ""

    def with_basis(self, basis: int, n_a: int = 0, n_b: int = 0) -> "ModelSpec":
        return dataclasses.replace(self, basis=basis, n_a=n_a, n_b=n_b)

    @property
    def is_complex(self) -> bool:
        """True when H has complex matrix elements in the S^z / occupation basis."""
        for _, _, J in self.couplings:
            J = np.asarray(J, dtype=float)
            # S^x S^y, S^y S^x, S^y S^z, S^z S^y carry a single factor i
            if J[0, 1] != 0 or J[1, 0] != 0 or J[1, 2] != 0 or J[2, 1] != 0:
                return True
        for _, h in self.fields:
            if h[1] != 0:
                return True
        for _, _, _, t in self.hops:
            if complex(t).imag != 0:
                return True
        return False


# ----------------------------------------------------------------------------- lattices
def ring_bonds(n: int, dist: int = 1) -> List[Tuple[int, int]]:
    """Periodic chain: bonds (i, i + dist mod n), each listed once."""
    out = []
    seen = set()
    for i in range(n):
        j = (i + dist) % n
        key = (min(i, j), max(i, j))
        if i != j and key not in seen:
            seen.add(key)
            out.append((i, j))
    return out


def square_bonds(lx: int, ly: int) -> List[Tuple[int, int]]:
    """Periodic lx x ly square lattice, site x + lx*y, bonds to +x and +y, each listed once."""
    out = []
    seen = set()
    for y in range(ly):
        for x in range(lx):
            i = x + lx * y
            for (dx, dy) in ((1, 0), (0, 1)):
                j = ((x + dx) % lx) + lx * ((y + dy) % ly)
                key = (min(i, j), max(i, j))
                if i != j and key not in seen:
                    seen.add(key)
                    out.append((i, j))
    return out


def tilted_square_bonds(a0: Tuple[int, int], a1: Tuple[int, int]) -> Tuple[int, List[Tuple[int, int]]]:
    """Square-lattice cluster with periodic boundaries along the superlattice vectors a0, a1
    (section 2.4's a0W/a0L, a1W/a1L); returns (number of sites, nearest-neighbour bonds).
    Points are identified modulo the superlattice; sites are numbered in the order their
    classes are first met scanning x, then y, over a box that covers every class."""
    det = a0[0] * a1[1] - a0[1] * a1[0]
    n = abs(det)

    def cls(x, y):  # superlattice coordinates times det, reduced modulo det
        return ((x * a1[1] - y * a1[0]) % n, (a0[0] * y - a0[1] * x) % n)

    site, rep = {}, []
    r = abs(a0[0]) + abs(a0[1]) + abs(a1[0]) + abs(a1[1])
    for y in range(-r, r + 1):
        for x in range(-r, r + 1):
            c = cls(x, y)
            if c not in site:
                site[c] = len(rep)
                rep.append((x, y))
    assert len(rep) == n
    out, seen = [], set()
    for i, (x, y) in enumerate(rep):
        for dx, dy in ((1, 0), (0, 1)):
            j = site[cls(x + dx, y + dy)]
            key = (min(i, j), max(i, j))
            if i != j and key not in seen:
                seen.add(key)
                out.append(key)
    return n, out


def honeycomb_bonds(cx: int, cy: int) -> List[Tuple[int, int, str]]:
    """Periodic honeycomb of cx x cy two-site cells: A = 2(x + cx*y), B = A + 1.

    z-bond A(x,y)-B(x,y); x-bond A(x,y)-B(x-1,y); y-bond A(x,y)-B(x,y-1).
    Returns (i, j, label) with label in {'x', 'y', 'z'}; duplicate bonds (possible on
    clusters one cell wide) are kept only once.
    """
    out = []
    seen = set()

    def a(x, y):
        return 2 * ((x % cx) + cx * (y % cy))

    for y in range(cy):
        for x in range(cx):
            for lab, (bx, by) in (("z", (x, y)), ("x", (x - 1, y)), ("y", (x, y - 1))):
                i, j = a(x, y), a(bx, by) + 1
                key = (min(i, j), max(i, j), lab)
                if key not in seen:
                    seen.add(key)
                    out.append((i, j, lab))
    return out


# ----------------------------------------------------------------------------- models
def _iso(J: float) -> np.ndarray:
    return J * np.eye(3)


def heisenberg(n_sites: int, bonds: Sequence[Tuple[int, int]], J: float = 1.0, name: str = "") -> ModelSpec:
    return ModelSpec(kind=SPIN, n_sites=n_sites, couplings=[(i, j, _iso(J)) for i, j in bonds], name=name)


def heisenberg_ring(n: int, J: float = 1.0) -> ModelSpec:
    return heisenberg(n, ring_bonds(n), J, name=f"heisenberg_ring_{n}")


def j1j2_ring(n: int, J1: float = 1.0, J2: float = 0.5) -> ModelSpec:
    cp = [(i, j, _iso(J1)) for i, j in ring_bonds(n, 1)] + [(i, j, _iso(J2)) for i, j in ring_bonds(n, 2)]
    return ModelSpec(kind=SPIN, n_sites=n, couplings=cp, name=f"j1j2_ring_{n}")


def heisenberg_square(lx: int, ly: int, J: float = 1.0) -> ModelSpec:
    return heisenberg(lx * ly, square_bonds(lx, ly), J, name=f"heisenberg_square_{lx}x{ly}")


def kitaev_honeycomb(cx: int, cy: int, K: float = -1.0, h: float = 0.05) -> ModelSpec:
    axis = {"x": 0, "y": 1, "z": 2}
    cp = []
    for i, j, lab in honeycomb_bonds(cx, cy):
        J = np.zeros((3, 3))
        J[axis[lab], axis[lab]] = K
        cp.append((i, j, J))
    n = 2 * cx * cy
    fields = [(i, (h, h, h)) for i in range(n)] if h != 0 else []
    return ModelSpec(kind=SPIN, n_sites=n, couplings=cp, fields=fields, name=f"kitaev_honeycomb_{cx}x{cy}")


def hubbard(n_sites: int, bonds: Sequence[Tuple[int, int]], t: complex = 1.0, U: float = 8.0, name: str = "") -> ModelSpec:
    hops = [(i, j, s, t) for (i, j) in bonds for s in (0, 1)]
    onsite = [(i, U) for i in range(n_sites)] if U != 0 else []
    return ModelSpec(kind=HUBBARD, n_sites=n_sites, hops=hops, onsite_U=onsite, name=name)


def hubbard_square(lx: int, ly: int, t: float = 1.0, U: float = 8.0) -> ModelSpec:
    return hubbard(lx * ly, square_bonds(lx, ly), t, U, name=f"hubbard_square_{lx}x{ly}")


def hubbard_tilted8(t: float = 1.0, U: float = 8.0) -> ModelSpec:
    """The 8-site periodic square cluster of section 5.1 (a0 = (2, 2), a1 = (-2, 2))."""
    n, bonds = tilted_square_bonds((2, 2), (-2, 2))
    return hubbard(n, bonds, t, U, name="hubbard_tilted8")


def hubbard_ring(n: int, t: float = 1.0, U: float = 8.0) -> ModelSpec:
    return hubbard(n, ring_bonds(n), t, U, name=f"hubbard_ring_{n}")


# ----------------------------------------------------------------------------- random models
def random_spin_model(n: int, n_bonds: int, seed: int, complex_: bool = True, fields: bool = True) -> ModelSpec:
    """Random couplings J^{ab} and fields on random site pairs (for brute-force checks)."""
    rng = np.random.default_rng(seed)
    cp = []
    for _ in range(n_bonds):
        i, j = rng.choice(n, size=2, replace=False)
        J = rng.normal(size=(3, 3))
        if not complex_:
            J[0, 1] = J[1, 0] = J[1, 2] = J[2, 1] = 0.0
        cp.append((int(i), int(j), J))
    fl = []
    if fields:
        for i in range(n):
            h = rng.normal(size=3)
            if not complex_:
                h[1] = 0.0
            fl.append((i, tuple(float(x) for x in h)))
    return ModelSpec(kind=SPIN, n_sites=n, couplings=cp, fields=fl, name=f"random_spin_{n}_{seed}")


def random_xxz_model(n: int, n_bonds: int, seed: int) -> ModelSpec:
    """Random S^z-conserving couplings (J^xx = J^yy, J^xy = -J^yx, J^zz) and z fields."""
    rng = np.random.default_rng(seed)
    cp = []
    for _ in range(n_bonds):
        i, j = rng.choice(n, size=2, replace=False)
        a, b, c = rng.normal(size=3)
        J = np.array([[a, b, 0.0], [-b, a, 0.0], [0.0, 0.0, c]])
        cp.append((int(i), int(j), J))
    fl = [(i, (0.0, 0.0, float(rng.normal()))) for i in range(n)]
    return ModelSpec(kind=SPIN, n_sites=n, couplings=cp, fields=fl, name=f"random_xxz_{n}_{seed}")


def random_hubbard_model(n: int, n_hops: int, seed: int, complex_: bool = True) -> ModelSpec:
    rng = np.random.default_rng(seed)
    hops = []
    for _ in range(n_hops):
        i, j = rng.choice(n, size=2, replace=False)
        s = int(rng.integers(0, 2))
        t = complex(rng.normal(), rng.normal() if complex_ else 0.0)
        hops.append((int(i), int(j), s, t))
    U = [(i, float(rng.uniform(0, 8))) for i in range(n)]
    V = []
    for _ in range(max(1, n // 2)):
        i, j = rng.choice(n, size=2, replace=False)
        V.append((int(i), int(j), float(rng.normal())))
    mu = [(i, float(rng.normal())) for i in range(n)]
    return ModelSpec(kind=HUBBARD, n_sites=n, hops=hops, onsite_U=U, density=V, chem_pot=mu,
                     name=f"random_hubbard_{n}_{seed}")


# ----------------------------------------------------------------------------- vectors
def gaussian_vector(seed: int, dim: int, nvec: int = 1, complex_: bool = False) -> np.ndarray:
    """Seeded standard-normal start vectors, shape [dim, nvec] (row-major: rows, then starts)."""
    rng = np.random.default_rng(seed)
    if complex_:
        out = np.empty((dim, nvec), dtype=np.complex128)
        out.real = rng.standard_normal((dim, nvec))
        out.imag = rng.standard_normal((dim, nvec))
        return out
    return rng.standard_normal((dim, nvec))


# ----------------------------------------------------------------------------- named workloads
START_SEED = 123432  # the paper's seed offset for random initial vectors (appendix A)


def workload(name: str) -> dict:
    """The five measured workloads, by name, with their sizes and run parameters."""
    if name == "heisenberg_ring12_full":
        m = heisenberg_ring(12)
        return dict(model=m, steps=100, prec="fp64", dim=4096)
    if name == "hubbard_4x4_8u8d":
        m = hubbard_square(4, 4, 1.0, 8.0).with_basis(BASIS_NUMBER, 8, 8)
        return dict(model=m, steps=200, prec="fp64", dim=math.comb(16, 8) ** 2)
    if name == "kitaev_24_tpq64":
        m = kitaev_honeycomb(4, 3, -1.0, 0.05)
        return dict(model=m, steps=1000, n_starts=64, l=1.0, dim=1 << 24)
    if name == "kitaev_18_tpq64":
        # the same cluster family at 3x3 cells (2^18 rows): small enough for kernel profiling,
        # its 64-start blocks (134 MB c64, 268 MB c128) still exceed L2
        m = kitaev_honeycomb(3, 3, -1.0, 0.05)
        return dict(model=m, steps=1000, n_starts=64, l=1.0, dim=1 << 18)
    if name == "j1j2_ring28_all_sectors":
        m = j1j2_ring(28, 1.0, 0.5)
        return dict(model=m, steps=150, sectors=list(range(29)), dim=1 << 28)
    if name == "heisenberg_6x5_sz15":
        # the 6x5 torus in its S^z = 0 sector (155,117,520 rows): the same split-row kernels as
        # the 6x6 sector at a size for kernel profiling (a 1.24 GB fp64 vector, above L2)
        m = heisenberg_square(6, 5).with_basis(BASIS_SZ, 15)
        return dict(model=m, steps=100, prec="fp64", dim=math.comb(30, 15))
    if name == "hubbard_18_sz0_tpq":
        # section 5.2.1: the half-filled 18-site cluster (a0 = (3, 3), a1 = (-3, 3)), t = 1, U = 8,
        # S^z = 0 (N_up = N_dn = 9): dim (18 C 9)^2 = 2,363,904,400; one mTPQ start, l = 8 (the
        # Gershgorin bound of H / N_s: U * 9 + 72 possible hops, over 18 sites)
        n, bonds = tilted_square_bonds((3, 3), (-3, 3))
        m = hubbard(n, bonds, 1.0, 8.0, name="hubbard_tilted18").with_basis(BASIS_NUMBER, 9, 9)
        return dict(model=m, steps=1000, n_starts=1, l=8.0, prec="fp32", dim=math.comb(18, 9) ** 2)
    if name == "heisenberg_6x6_sz0":
        m = heisenberg_square(6, 6).with_basis(BASIS_SZ, 18)
        return dict(model=m, steps=100, prec="mixed", dim=math.comb(36, 18))
    raise KeyError(name)


WORKLOADS = ["heisenberg_ring12_full", "hubbard_4x4_8u8d", "kitaev_24_tpq64", "j1j2_ring28_all_sectors",
             "heisenberg_6x6_sz0", "kitaev_18_tpq64", "heisenberg_6x5_sz15", "hubbard_18_sz0_tpq"]
