"""Python access to the CPU oracle (hphi_oracle.cpp) -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain, slow, fp64 CPU restatement of the method, written independently of
the CUDA library; it exists only to check that library.  Only tests, the smoke check and
the benchmark's CPU-baseline leg may import this package.  It never imports the CUDA
library and the CUDA library never imports it.

Eigenvalues of the Lanczos tridiagonal matrix come from LAPACK (scipy), as in the paper,
which diagonalises T_n with dsyev (appendix A.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hphi_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host C++ compiler (g++, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("n_sites", ctypes.c_int), ("basis", ctypes.c_int),
        ("n_a", ctypes.c_int), ("n_b", ctypes.c_int),
        ("n_coup", ctypes.c_int), ("coup_ij", ctypes.c_void_p), ("coup_J", ctypes.c_void_p),
        ("n_field", ctypes.c_int), ("field_i", ctypes.c_void_p), ("field_h", ctypes.c_void_p),
        ("n_hop", ctypes.c_int), ("hop_ij", ctypes.c_void_p), ("hop_spin", ctypes.c_void_p), ("hop_t", ctypes.c_void_p),
        ("n_U", ctypes.c_int), ("U_i", ctypes.c_void_p), ("U_val", ctypes.c_void_p),
        ("n_V", ctypes.c_int), ("V_ij", ctypes.c_void_p), ("V_val", ctypes.c_void_p),
        ("n_mu", ctypes.c_int), ("mu_i", ctypes.c_void_p), ("mu_val", ctypes.c_void_p),
    ]


def _bind(L):
    """Argument and result types of the oracle library's exported functions."""
    P = ctypes.c_void_p
    u64, i64, i32, f64 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.or_dim.argtypes = [P, P]
    L.or_binom.argtypes = [i32, i32]; L.or_binom.restype = u64
    L.or_sector_list.argtypes = [i32, i32, P, i64]; L.or_sector_list.restype = i64
    L.or_rank.argtypes = [u64, i32]; L.or_rank.restype = u64
    L.or_unrank.argtypes = [u64, i32, i32]; L.or_unrank.restype = u64
    L.or_hop_sign.argtypes = [u64, u64, i32, i32, i32]
    L.or_apply_H.argtypes = [P, P, P, i32]
    L.or_apply_H_slice.argtypes = [P, P, P, i32, u64, u64]
    L.or_philox4x32_10.argtypes = [P, P, P]
    L.or_gauss_pair.argtypes = [u64, u64, P]
    L.or_random_at.argtypes = [u64, P, i64, i32, P]
    L.or_apply_H_rows_philox.argtypes = [P, P, i64, u64, i32, i32, i32, P]
    L.or_lanczos.argtypes = [P, P, i32, f64, P, P]
    L.or_lanczos_vector.argtypes = [P, P, i32, P, P, P, P]
    L.or_tpq.argtypes = [P, P, i32, f64, f64, P, P, P, P]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


class OracleModel:
    """ctypes view of a workloads.ModelSpec (keeps the backing arrays alive)."""

    def __init__(self, spec):
        self.spec = spec
        cp = spec.couplings
        self.coup_ij = np.array([[i, j] for i, j, _ in cp], dtype=np.int32).reshape(-1, 2)
        self.coup_J = np.array([np.asarray(J, dtype=np.float64).reshape(9) for _, _, J in cp], dtype=np.float64).reshape(-1, 9)
        self.field_i = np.array([i for i, _ in spec.fields], dtype=np.int32)
        self.field_h = np.array([list(h) for _, h in spec.fields], dtype=np.float64).reshape(-1, 3)
        self.hop_ij = np.array([[i, j] for i, j, _, _ in spec.hops], dtype=np.int32).reshape(-1, 2)
        self.hop_spin = np.array([s for _, _, s, _ in spec.hops], dtype=np.int32)
        self.hop_t = np.array([[complex(t).real, complex(t).imag] for *_, t in spec.hops], dtype=np.float64).reshape(-1, 2)
        self.U_i = np.array([i for i, _ in spec.onsite_U], dtype=np.int32)
        self.U_val = np.array([u for _, u in spec.onsite_U], dtype=np.float64)
        self.V_ij = np.array([[i, j] for i, j, _ in spec.density], dtype=np.int32).reshape(-1, 2)
        self.V_val = np.array([v for *_, v in spec.density], dtype=np.float64)
        self.mu_i = np.array([i for i, _ in spec.chem_pot], dtype=np.int32)
        self.mu_val = np.array([m for _, m in spec.chem_pot], dtype=np.float64)
        self.s = _Model(spec.kind, spec.n_sites, spec.basis, spec.n_a, spec.n_b,
                        len(cp), _ptr(self.coup_ij), _ptr(self.coup_J),
                        len(spec.fields), _ptr(self.field_i), _ptr(self.field_h),
                        len(spec.hops), _ptr(self.hop_ij), _ptr(self.hop_spin), _ptr(self.hop_t),
                        len(spec.onsite_U), _ptr(self.U_i), _ptr(self.U_val),
                        len(spec.density), _ptr(self.V_ij), _ptr(self.V_val),
                        len(spec.chem_pot), _ptr(self.mu_i), _ptr(self.mu_val))

    @property
    def ref(self):
        return ctypes.byref(self.s)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc == -2:
        raise OracleError(f"{what}: a term connects the basis to a configuration outside it")
    if rc < 0:
        raise OracleError(f"{what}: invalid model or arguments (rc={rc})")


def dim(spec) -> int:
    d = ctypes.c_uint64()
    _check(lib().or_dim(OracleModel(spec).ref, ctypes.byref(d)), "dim")
    return int(d.value)


def binom(n: int, k: int) -> int:
    return int(lib().or_binom(n, k))


def sector_list(n_bits: int, k: int) -> np.ndarray:
    cnt = binom(n_bits, k)
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    got = lib().or_sector_list(n_bits, k, _ptr(out), cnt)
    assert got == cnt
    return out[:cnt]


def rank(s: int, n_bits: int) -> int:
    return int(lib().or_rank(s, n_bits))


def unrank(r: int, n_bits: int, k: int) -> int:
    return int(lib().or_unrank(r, n_bits, k))


def hop_sign(up: int, dn: int, n: int, p: int, q: int) -> int:
    return int(lib().or_hop_sign(up, dn, n, p, q))


def _as_c128(v, d: int) -> np.ndarray:
    v = np.asarray(v)
    if v.ndim == 1:
        v = v.reshape(d, 1)
    return np.ascontiguousarray(v, dtype=np.complex128)


def apply_H(spec, v) -> np.ndarray:
    """w = H v; v: [dim] or [dim, nvec]; returns complex128 of v's shape."""
    om = OracleModel(spec)
    d = dim(spec)
    shape = np.shape(v)
    vc = _as_c128(v, d)
    w = np.zeros_like(vc)
    _check(lib().or_apply_H(om.ref, _ptr(vc), _ptr(w), vc.shape[1]), "apply_H")
    return w.reshape(shape)


def apply_H_slice(spec, v, r0: int, nrows: int) -> np.ndarray:
    om = OracleModel(spec)
    d = dim(spec)
    vc = _as_c128(v, d)
    w = np.zeros((nrows, vc.shape[1]), dtype=np.complex128)
    _check(lib().or_apply_H_slice(om.ref, _ptr(vc), _ptr(w), vc.shape[1], r0, nrows), "apply_H_slice")
    return w


def apply_H_rows_philox(spec, rows, seed: int, complex_: bool, nvec: int = 1, col: int = 0) -> np.ndarray:
    """Rows of H v where v [dim][nvec] is the Philox start vector of `seed` (column `col`)."""
    om = OracleModel(spec)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    out = np.zeros(len(rows), dtype=np.complex128)
    _check(lib().or_apply_H_rows_philox(om.ref, _ptr(rows), len(rows), seed, int(complex_), nvec, col, _ptr(out)),
           "apply_H_rows_philox")
    return out


def dense_H(spec) -> np.ndarray:
    """The full matrix <i|H|j>, built column by column from the oracle's H v."""
    d = dim(spec)
    return apply_H(spec, np.eye(d, dtype=np.complex128))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def random_at(seed: int, idx, complex_: bool) -> np.ndarray:
    """Elements idx of the Philox Gaussian start vector of `seed` (appendix A.2 / A.4's random
    coefficients): complex element e is the Box-Muller pair of Philox block e, real elements
    2p and 2p + 1 are the two numbers of block p."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.zeros(len(idx), dtype=np.complex128)
    lib().or_random_at(seed, _ptr(idx), len(idx), int(complex_), _ptr(out))
    return out if complex_ else out.real.copy()


def lanczos(spec, v0, m: int, brk: float = 1e-13):
    """Returns (alpha[steps], beta[steps]) with beta[k] = beta_{k+1} (section 3.4)."""
    om = OracleModel(spec)
    d = dim(spec)
    vc = _as_c128(v0, d)
    a = np.zeros(m)
    b = np.zeros(m)
    steps = lib().or_lanczos(om.ref, _ptr(vc), m, brk, _ptr(a), _ptr(b))
    _check(min(steps, 0), "lanczos")
    return a[:steps], b[:steps]


def ritz_values(alpha, beta, k: int | None = None) -> np.ndarray:
    """Eigenvalues of the Lanczos tridiagonal matrix T (LAPACK via scipy)."""
    from scipy.linalg import eigh_tridiagonal
    alpha = np.asarray(alpha, dtype=np.float64)
    n = len(alpha)
    e = np.asarray(beta[: n - 1], dtype=np.float64)
    w = eigh_tridiagonal(alpha, e, eigvals_only=True) if n > 1 else alpha.copy()
    return w if k is None else w[:k]


def ritz_vector(alpha, beta, which: int = 0) -> np.ndarray:
    from scipy.linalg import eigh_tridiagonal
    alpha = np.asarray(alpha, dtype=np.float64)
    n = len(alpha)
    if n == 1:
        return np.ones(1)
    w, v = eigh_tridiagonal(alpha, np.asarray(beta[: n - 1], dtype=np.float64))
    return v[:, which]


def lanczos_vector(spec, v0, alpha, beta, coef) -> np.ndarray:
    om = OracleModel(spec)
    d = dim(spec)
    vc = _as_c128(v0, d)
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    x = np.zeros(d, dtype=np.complex128)
    _check(lib().or_lanczos_vector(om.ref, _ptr(vc), len(a), _ptr(a), _ptr(b), _ptr(c), _ptr(x)), "lanczos_vector")
    return x


def tpq(spec, psi0, K: int, l: float, Ns: float | None = None, want_state: bool = False):
    """mTPQ records (section 3.5): u[k], h2[k], nrm[k] for the state of step k = 0..K-1."""
    om = OracleModel(spec)
    d = dim(spec)
    Ns = float(spec.n_sites if Ns is None else Ns)
    pc = _as_c128(psi0, d)
    u = np.zeros(K)
    h2 = np.zeros(K)
    nrm = np.zeros(K)
    out = np.zeros(d, dtype=np.complex128) if want_state else None
    _check(lib().or_tpq(om.ref, _ptr(pc), K, l, Ns, _ptr(u), _ptr(h2), _ptr(nrm), _ptr(out)), "tpq")
    return (u, h2, nrm, out) if want_state else (u, h2, nrm)


def _popcount(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.uint64)
    out = np.zeros(a.shape, dtype=np.int64)
    for b in range(64):
        out += ((a >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return out


def basis_configurations(spec):
    """Configuration of every basis index (section 3.1's ordering): spin -> s [dim];
    Hubbard -> (up [dim], dn [dim]) with index = dn_index * dim_up + up_index."""
    n = spec.n_sites
    if spec.kind == 0:
        if spec.basis == 0:
            return np.arange(1 << n, dtype=np.uint64)
        return sector_list(n, spec.n_a)
    if spec.basis == 0:
        lu = ld = np.arange(1 << n, dtype=np.uint64)
    else:
        lu, ld = sector_list(n, spec.n_a), sector_list(n, spec.n_b)
    up = np.tile(lu, len(ld))
    dn = np.repeat(ld, len(lu))
    return up, dn


def diag_observables(spec, psi):
    """Section 3.5's local estimate <psi|A|psi> / (<psi|psi> N_s) for the diagonal operators
    A = sum_i n_i,up n_i,dn (doubly occupied sites; 0 for spins), S^z_total and (S^z_total)^2.
    psi [dim] or [dim][nvec]; returns three arrays [nvec] (or scalars)."""
    p = np.asarray(psi)
    w = np.abs(p) ** 2
    if spec.kind == 0:
        s = basis_configurations(spec)
        dbl = np.zeros(len(s))
        m2 = 2 * _popcount(s) - spec.n_sites
    else:
        up, dn = basis_configurations(spec)
        dbl = _popcount(up & dn).astype(np.float64)
        m2 = _popcount(up) - _popcount(dn)
    m2 = m2.astype(np.float64)
    ww = w.sum(axis=0)
    ns = spec.n_sites
    if w.ndim == 2:
        dbl, m2 = dbl[:, None], m2[:, None]
    return ((w * dbl).sum(axis=0) / ww / ns, (w * m2).sum(axis=0) / 2 / ww / ns,
            (w * m2 * m2).sum(axis=0) / 4 / ww / ns)


def tpq_states(spec, psi0, K: int, l: float, Ns: float | None = None):
    """The normalised mTPQ states psi_0 .. psi_{K-1} of section 3.5, one multiplication by
    (l - H / N_s) and one normalisation per step; returns [K][dim]."""
    d = dim(spec)
    Ns = float(spec.n_sites if Ns is None else Ns)
    x = _as_c128(psi0, d)[:, 0].copy()
    x /= np.linalg.norm(x)
    out = np.zeros((K, d), dtype=np.complex128)
    for k in range(K):
        out[k] = x
        y = l * x - apply_H(spec, x) / Ns
        x = y / np.linalg.norm(y)
    return out


def inverse_iteration(spec, x0, E: float, delta: float, outer: int):
    """Section 3.4.1: y_{k+1} = (H - E + delta)^{-1} y_k, normalised, from y_0 = x0 (each
    solve by LAPACK on the dense matrix of the oracle's H)."""
    H = dense_H(spec)
    A = H - (E - delta) * np.eye(H.shape[0])
    y = np.asarray(x0, dtype=np.complex128).copy()
    y /= np.linalg.norm(y)
    for _ in range(outer):
        y = np.linalg.solve(A, y)
        y /= np.linalg.norm(y)
    return y


def lanczos_convergence_step(alpha, beta, eps: float, first: int = 5, every: int = 2):
    """Appendix C's stopping rule on a recurrence's alpha / beta: the first n (n = first,
    first + every, ...) at which T_n's first excited eigenvalue agrees with its value at the
    previous test to eps relative; None if no n within the data does."""
    prev = None
    for n in range(first, len(alpha) + 1, every):
        e1 = ritz_values(alpha[:n], beta[:n])[1]
        if prev is not None and abs(e1 - prev) <= eps * abs(e1):
            return n
        prev = e1
    return None


def lanczos_reorth(spec, v0, m: int, brk: float = 1e-13, want_vectors: bool = False):
    """Section 3.4's recurrence with full reorthogonalisation: after w = H v_k - beta_k v_{k-1}
    - alpha_k v_k, the components of w along every earlier v_j are removed (classical
    Gram-Schmidt, numpy inner products) before beta_{k+1} = |w|.  Returns (alpha, beta[, V])."""
    d = dim(spec)
    v = _as_c128(v0, d)[:, 0].copy()
    v /= np.linalg.norm(v)
    V = [v]
    a, b = [], []
    v_prev, b_prev = np.zeros_like(v), 0.0
    for _ in range(m):
        w = apply_H(spec, v) - b_prev * v_prev
        al = np.vdot(v, w).real
        w = w - al * v
        Vm = np.array(V)
        w = w - Vm.T @ (Vm.conj() @ w)
        be = np.linalg.norm(w)
        a.append(al)
        b.append(be)
        if not be > brk * max(1.0, abs(al)):
            break
        v_prev, v, b_prev = v, w / be, be
        V.append(v)
    out = (np.array(a), np.array(b))
    return out + (np.array(V),) if want_vectors else out
