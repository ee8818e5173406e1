"""Independent textbook constructions used to pin the oracle (tests only).

Dense Hamiltonians built from Kronecker products of Pauli matrices (spins) and from the
Jordan-Wigner representation of fermion operators, i.e. by a route that shares nothing
with the oracle's bit-level element evaluation.
"""
import numpy as np

# Pauli matrices in the textbook (up, down) ordering.
_SX = np.array([[0, 1], [1, 0]], dtype=complex)
_SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
_SZ = np.array([[1, 0], [0, -1]], dtype=complex)
# The oracle/library basis orders a site as (down = bit 0, up = bit 1): permute.
_P = np.array([[0, 1], [1, 0]], dtype=complex)
SPIN_OPS = [(_P @ s @ _P) / 2 for s in (_SX, _SY, _SZ)]


def site_op(A, k, n):
    """A acting on site k of n sites; site k is bit k of the basis index."""
    return np.kron(np.kron(np.eye(2 ** (n - 1 - k)), A), np.eye(2 ** k))


def dense_spin(spec):
    n = spec.n_sites
    H = np.zeros((2 ** n, 2 ** n), dtype=complex)
    S = [[site_op(SPIN_OPS[a], k, n) for a in range(3)] for k in range(n)]
    for i, j, J in spec.couplings:
        for a in range(3):
            for b in range(3):
                if J[a][b] != 0:
                    H += J[a][b] * S[i][a] @ S[j][b]
    for i, h in spec.fields:
        for a in range(3):
            H -= h[a] * S[i][a]
    return H


def fermion_ops(n_modes):
    """Annihilators c_m, m = 0..n_modes-1, with the string of Z on modes < m."""
    a = np.array([[0, 1], [0, 0]], dtype=complex)  # a|1> = |0>, basis (0, 1)
    Z = np.diag([1.0, -1.0]).astype(complex)
    I2 = np.eye(2, dtype=complex)
    ops = []
    for m in range(n_modes):
        M = np.ones((1, 1), dtype=complex)
        for p in reversed(range(n_modes)):  # kron from the highest bit down to bit 0
            f = a if p == m else (Z if p < m else I2)
            M = np.kron(M, f)
        ops.append(M)
    return ops


def dense_hubbard(spec, mode_of=None):
    """Mode order (up 0..n-1, down 0..n-1) unless mode_of(site, spin) is given."""
    n = spec.n_sites
    if mode_of is None:
        mode_of = lambda i, s: i + n * s  # noqa: E731
    c = fermion_ops(2 * n)
    cd = [x.conj().T for x in c]
    num = [cd[m] @ c[m] for m in range(2 * n)]
    D = 4 ** n
    H = np.zeros((D, D), dtype=complex)
    for i, j, s, t in spec.hops:
        p, q = mode_of(i, s), mode_of(j, s)
        H += -t * cd[p] @ c[q] - np.conj(t) * cd[q] @ c[p]
    for i, U in spec.onsite_U:
        H += U * num[mode_of(i, 0)] @ num[mode_of(i, 1)]
    for i, j, V in spec.density:
        ni = num[mode_of(i, 0)] + num[mode_of(i, 1)]
        nj = num[mode_of(j, 0)] + num[mode_of(j, 1)]
        H += V * ni @ nj
    for i, mu in spec.chem_pot:
        H -= mu * (num[mode_of(i, 0)] + num[mode_of(i, 1)])
    return H


def popcount(x):
    return bin(int(x)).count("1")


def spin_sector_indices(n, k):
    return np.array([s for s in range(2 ** n) if popcount(s) == k], dtype=np.int64)


def hubbard_sector_indices(n, na, nb):
    """Full-basis indices f = up + 2^n dn of the (na, nb) sector, ascending."""
    return np.array([f for f in range(4 ** n)
                     if popcount(f & (2 ** n - 1)) == na and popcount(f >> n) == nb], dtype=np.int64)
