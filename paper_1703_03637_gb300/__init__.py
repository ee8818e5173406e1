"""GB300-native Lanczos / microcanonical-TPQ library for two-body quantum lattice models.

Thin ctypes binding over the C ABI of include/hphi_gpu.h (libhphi_gpu.so, built from
csrc/ for sm_103a).  The binding only marshals arguments: every step of the method runs
in the library's CUDA kernels.  PyTorch provides device memory and the current stream.
If the library cannot be loaded, every entry point raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["Model", "load", "LibraryError", "FP64", "FP32", "philox4x32_10", "lib_path"]

SPIN_HALF, HUBBARD = 0, 1
BASIS_FULL, BASIS_SZ, BASIS_NUMBER = 0, 1, 2
FP64, FP32 = 0, 1
OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "BASIS_MISMATCH", -3: "OUT_OF_MEMORY", -4: "NOT_BUILT", -5: "CUDA", -7: "UNSUPPORTED"}

# C symbols declared in include/hphi_gpu.h
EXPORTS = [
    "hphi_create", "hphi_destroy", "hphi_last_error", "hphi_add_spin_coupling", "hphi_add_spin_field",
    "hphi_add_hopping", "hphi_add_onsite_U", "hphi_add_density", "hphi_add_chemical_potential", "hphi_set_basis",
    "hphi_build_sector", "hphi_dim", "hphi_is_complex", "hphi_basis_states", "hphi_basis_ranks", "hphi_apply_H",
    "hphi_random_vector", "hphi_philox4x32_10", "hphi_lanczos_run", "hphi_tpq_run", "hphi_apply_H_noalloc",
    "hphi_lanczos_run_sectors", "hphi_autotune", "hphi_set_window_bits", "hphi_set_sector_split",
    "hphi_release_workspace", "hphi_inverse_iteration",
]


class LibraryError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class LanczosParams(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("prec", ctypes.c_int), ("seed", ctypes.c_uint64), ("v0", ctypes.c_void_p),
                ("n_eig", ctypes.c_int), ("refine", ctypes.c_int), ("breakdown", ctypes.c_double),
                ("profile", ctypes.c_int), ("keep_basis", ctypes.c_int), ("v0_on_host", ctypes.c_int),
                ("eps", ctypes.c_double), ("ritz_out", ctypes.c_void_p), ("reorth", ctypes.c_int)]


class LanczosResult(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int), ("alpha", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("eig", ctypes.c_double * 8), ("e_refined", ctypes.c_double), ("residual", ctypes.c_double),
                ("variance", ctypes.c_double), ("device_ms", ctypes.c_float), ("hv_ms", ctypes.c_float),
                ("hv_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int), ("converged", ctypes.c_int)]


class InvitParams(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("shift", ctypes.c_double), ("outer", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("cg_tol", ctypes.c_double)]


class InvitResult(ctypes.Structure):
    _fields_ = [("e", ctypes.c_double), ("residual", ctypes.c_double), ("variance", ctypes.c_double),
                ("cg_steps", ctypes.c_int), ("device_ms", ctypes.c_float), ("kernel_launches", ctypes.c_int)]


class TuneResult(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int), ("best_dn_ept", ctypes.c_int), ("best_up_k", ctypes.c_int),
                ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float), ("worst_ms", ctypes.c_float),
                ("best_split_L", ctypes.c_int), ("best_split_K", ctypes.c_int), ("best_split_hi_cols", ctypes.c_int)]


class TpqParams(ctypes.Structure):
    _fields_ = [("n_starts", ctypes.c_int), ("steps", ctypes.c_int), ("l", ctypes.c_double), ("n_s", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("psi0", ctypes.c_void_p), ("prec", ctypes.c_int),
                ("profile", ctypes.c_int), ("obs_every", ctypes.c_int)]


class TpqResult(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("h2", ctypes.c_void_p), ("norm", ctypes.c_void_p), ("device_ms", ctypes.c_float),
                ("kernel_launches", ctypes.c_int), ("hv_ms", ctypes.c_float), ("hv_launches", ctypes.c_int),
                ("beta", ctypes.c_void_p), ("spec_heat", ctypes.c_void_p), ("doublon", ctypes.c_void_p),
                ("sz", ctypes.c_void_p), ("sz2", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libhphi_gpu.so (building it with nvcc first if it is stale or missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB_PATH
        if not os.path.exists(path):
            raise LibraryError(-5, f"CUDA library not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        P, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.hphi_create.argtypes = [ctypes.POINTER(P), I, I]
        L.hphi_destroy.argtypes = [P]
        L.hphi_destroy.restype = None
        L.hphi_last_error.argtypes = [P]
        L.hphi_last_error.restype = ctypes.c_char_p
        L.hphi_add_spin_coupling.argtypes = [P, I, I, P]
        L.hphi_add_spin_field.argtypes = [P, I, P]
        L.hphi_add_hopping.argtypes = [P, I, I, I, D, D]
        L.hphi_add_onsite_U.argtypes = [P, I, D]
        L.hphi_add_density.argtypes = [P, I, I, D]
        L.hphi_add_chemical_potential.argtypes = [P, I, D]
        L.hphi_set_basis.argtypes = [P, I, I, I]
        L.hphi_build_sector.argtypes = [P, ctypes.POINTER(I64), P]
        L.hphi_dim.argtypes = [P]
        L.hphi_dim.restype = I64
        L.hphi_is_complex.argtypes = [P]
        L.hphi_basis_states.argtypes = [P, I64, I64, P, P]
        L.hphi_basis_ranks.argtypes = [P, P, I64, P, P]
        L.hphi_apply_H.argtypes = [P, P, P, I, I, P]
        L.hphi_apply_H_noalloc.argtypes = [P, P, P, P]
        L.hphi_random_vector.argtypes = [P, P, I, I, U64, P]
        L.hphi_philox4x32_10.argtypes = [P, P, P, I64, P]
        L.hphi_lanczos_run.argtypes = [P, ctypes.POINTER(LanczosParams), ctypes.POINTER(LanczosResult), P]
        L.hphi_tpq_run.argtypes = [P, ctypes.POINTER(TpqParams), ctypes.POINTER(TpqResult), P]
        L.hphi_autotune.argtypes = [P, I, ctypes.POINTER(TuneResult), P]
        L.hphi_set_window_bits.argtypes = [P, I]
        L.hphi_set_sector_split.argtypes = [P, I, I, I, P]
        L.hphi_release_workspace.argtypes = [P]
        L.hphi_inverse_iteration.argtypes = [P, ctypes.POINTER(InvitParams), P, ctypes.POINTER(InvitResult), P]
        L.hphi_lanczos_run_sectors.argtypes = [P, P, I, ctypes.POINTER(LanczosParams), ctypes.POINTER(LanczosResult), P]
        _lib = L
        return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise LibraryError(-5, "no CUDA device: this library has no CPU path")
    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    if not t.is_cuda:
        raise LibraryError(-1, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise LibraryError(-1, "expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


class Model:
    """One lattice Hamiltonian with its basis, tables and solver workspace on the GPU."""

    def __init__(self, kind: int, n_sites: int):
        self._L = load()
        h = ctypes.c_void_p()
        rc = self._L.hphi_create(ctypes.byref(h), kind, n_sites)
        if rc:
            raise LibraryError(rc, self._L.hphi_last_error(None).decode())
        self._h = h
        self.kind, self.n_sites = kind, n_sites
        self.dim = None
        self.is_complex = None

    # ------------------------------------------------------------------ construction
    @classmethod
    def from_spec(cls, spec, build: bool = True) -> "Model":
        """Build from any object with the attributes of workloads.ModelSpec."""
        m = cls(spec.kind, spec.n_sites)
        for i, j, J in spec.couplings:
            m.add_spin_coupling(i, j, J)
        for i, h in spec.fields:
            m.add_spin_field(i, h)
        for i, j, s, t in spec.hops:
            m.add_hopping(i, j, s, t)
        for i, U in spec.onsite_U:
            m.add_onsite_U(i, U)
        for i, j, V in spec.density:
            m.add_density(i, j, V)
        for i, mu in spec.chem_pot:
            m.add_chemical_potential(i, mu)
        m.set_basis(spec.basis, spec.n_a, spec.n_b)
        if build:
            m.build()
        return m

    def _check(self, rc):
        if rc:
            raise LibraryError(rc, self._L.hphi_last_error(self._h).decode())

    def add_spin_coupling(self, i, j, J):
        a = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(9))
        self._check(self._L.hphi_add_spin_coupling(self._h, i, j, a.ctypes.data))

    def add_spin_field(self, i, h):
        a = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(3))
        self._check(self._L.hphi_add_spin_field(self._h, i, a.ctypes.data))

    def add_hopping(self, i, j, spin, t):
        t = complex(t)
        self._check(self._L.hphi_add_hopping(self._h, i, j, spin, t.real, t.imag))

    def add_onsite_U(self, i, U):
        self._check(self._L.hphi_add_onsite_U(self._h, i, float(U)))

    def add_density(self, i, j, V):
        self._check(self._L.hphi_add_density(self._h, i, j, float(V)))

    def add_chemical_potential(self, i, mu):
        self._check(self._L.hphi_add_chemical_potential(self._h, i, float(mu)))

    def set_basis(self, basis, a=0, b=0):
        self._check(self._L.hphi_set_basis(self._h, basis, a, b))

    def build(self) -> int:
        _torch()
        d = ctypes.c_int64()
        self._check(self._L.hphi_build_sector(self._h, ctypes.byref(d), _stream()))
        self.dim = int(d.value)
        self.is_complex = bool(self._L.hphi_is_complex(self._h))
        return self.dim

    def close(self):
        if getattr(self, "_h", None):
            self._L.hphi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ tensors
    def dtype(self, prec=FP64):
        torch = _torch()
        if self.is_complex:
            return torch.complex128 if prec == FP64 else torch.complex64
        return torch.float64 if prec == FP64 else torch.float32

    def empty(self, nvec=1, prec=FP64):
        torch = _torch()
        return torch.empty((self.dim, nvec), dtype=self.dtype(prec), device="cuda")

    def _prec_of(self, t):
        torch = _torch()
        if t.dtype in (torch.float64, torch.complex128):
            return FP64
        if t.dtype in (torch.float32, torch.complex64):
            return FP32
        raise LibraryError(-1, f"unsupported dtype {t.dtype}")

    # ------------------------------------------------------------------ operations
    def apply_H(self, v, w=None):
        """w = H v for v of shape [dim] or [dim, nvec] (CUDA tensor of the model's dtype)."""
        prec = self._prec_of(v)
        if v.dtype != self.dtype(prec):
            raise LibraryError(-1, f"vector dtype {v.dtype} does not match the model ({self.dtype(prec)})")
        nvec = 1 if v.dim() == 1 else v.shape[1]
        if v.shape[0] != self.dim:
            raise LibraryError(-1, "vector length differs from the basis dimension")
        if w is None:
            w = _torch().empty_like(v)
        self._check(self._L.hphi_apply_H(self._h, _dptr(v), _dptr(w), nvec, prec, _stream()))
        return w

    def autotune(self, prec=FP64) -> dict:
        """Time the H v launch configurations and keep the fastest (see hphi_autotune)."""
        _torch()
        r = TuneResult()
        self._check(self._L.hphi_autotune(self._h, prec, ctypes.byref(r), _stream()))
        return dict(n_candidates=r.n_candidates, dn_ept=r.best_dn_ept, up_k=r.best_up_k, best_ms=r.best_ms,
                    default_ms=r.default_ms, worst_ms=r.worst_ms, split_L=r.best_split_L, split_K=r.best_split_K,
                    split_hi_cols=r.best_split_hi_cols)

    def set_sector_split(self, prec=FP64, L: int = 0, K: int = 0):
        """Split-row spin path (see hphi_set_sector_split): L = -1 off, 0 default, else the low
        part's length; K = 0 widest tile, else rows per tile."""
        _torch()
        self._check(self._L.hphi_set_sector_split(self._h, prec, int(L), int(K), _stream()))

    def release_workspace(self):
        """Free the solver workspace (vectors and scratch kept between calls); tables stay."""
        _torch()
        self._check(self._L.hphi_release_workspace(self._h))

    def set_window_bits(self, bits: int):
        """Window passes of the many-vector H v: 0 automatic, -1 off, else the window's sites."""
        self._check(self._L.hphi_set_window_bits(self._h, int(bits)))

    def apply_H_noalloc(self, v, w):
        """w = H v through the allocation-free entry point (fp64, one vector, real Hubbard
        models with one hopping value per species).  v and w are caller-owned CUDA tensors of
        shape [dim]; the library allocates nothing during the call."""
        torch = _torch()
        if v.dtype != torch.float64 or w.dtype != torch.float64 or v.numel() != self.dim or w.numel() != self.dim:
            raise LibraryError(-1, "apply_H_noalloc takes float64 vectors of length dim")
        self._check(self._L.hphi_apply_H_noalloc(self._h, _dptr(v), _dptr(w), _stream()))
        return w

    def random_vector(self, seed: int, nvec: int = 1, prec=FP64):
        v = self.empty(nvec, prec)
        self._check(self._L.hphi_random_vector(self._h, _dptr(v), nvec, prec, seed, _stream()))
        return v

    def basis_states(self, r0: int = 0, n: int | None = None):
        torch = _torch()
        n = self.dim - r0 if n is None else n
        out = torch.empty(n, dtype=torch.int64, device="cuda")
        self._check(self._L.hphi_basis_states(self._h, r0, n, _dptr(out), _stream()))
        return out

    def basis_ranks(self, states):
        torch = _torch()
        states = states.to(device="cuda", dtype=torch.int64).contiguous()
        out = torch.empty_like(states)
        self._check(self._L.hphi_basis_ranks(self._h, _dptr(states), states.numel(), _dptr(out), _stream()))
        return out

    def lanczos(self, steps: int, prec=FP64, seed: int = 123432, v0=None, n_eig: int = 1, refine: bool = False,
                breakdown: float = 0.0, profile: bool = False, keep_basis: int = 0, v0_on_host: bool = False,
                eps: float = 0.0, ritz_out=None, reorth: bool = False):
        """Section 3.4 Lanczos; returns dict(alpha, beta, steps, eig, e_refined, residual, variance, ms,
        converged).  eps > 0: appendix C's convergence test, steps is then the limit.  ritz_out: a CUDA
        fp64 (complex128) tensor of length dim that receives the refined Ritz vector (refine=True).
        reorth: full reorthogonalisation against the kept Lanczos vectors (fp64 inner products).
        v0: start vector (a CUDA tensor, or any tensor moved to the device here); with v0_on_host
        it must be a host tensor, which the library copies in itself (hphi_lanczos_params.v0_on_host)."""
        torch = _torch()
        on_host = v0 is not None and v0_on_host
        if on_host:  # the library copies the host vector itself (no device copy is made here)
            if v0.is_cuda:
                raise LibraryError(-1, "v0_on_host: v0 must be a host tensor")
            want = torch.complex128 if self.is_complex else torch.float64
            if v0.dtype != want or not v0.is_contiguous() or v0.numel() != self.dim:
                raise LibraryError(-1, f"host v0 must be a contiguous {want} tensor of length dim")
            vptr = ctypes.c_void_p(v0.data_ptr())
        elif v0 is not None:
            v0 = v0.to(device="cuda", dtype=torch.complex128 if self.is_complex else torch.float64).contiguous()
            vptr = _dptr(v0)
        else:
            vptr = None
        a = np.zeros(steps)
        b = np.zeros(steps)
        if ritz_out is not None:
            want = torch.complex128 if self.is_complex else torch.float64
            if not (ritz_out.is_cuda and ritz_out.dtype == want and ritz_out.is_contiguous()
                    and ritz_out.numel() == self.dim):
                raise LibraryError(-1, f"ritz_out must be a contiguous CUDA {want} tensor of length dim")
        p = LanczosParams(steps, prec, seed, vptr, n_eig, int(refine), breakdown, int(profile), int(keep_basis),
                          int(on_host), float(eps), _dptr(ritz_out) if ritz_out is not None else None, int(reorth))
        r = LanczosResult()
        r.alpha = a.ctypes.data
        r.beta = b.ctypes.data
        self._check(self._L.hphi_lanczos_run(self._h, ctypes.byref(p), ctypes.byref(r), _stream()))
        n = r.steps_done
        return dict(alpha=a[:n], beta=b[:n], steps=n, eig=np.array(r.eig[:n_eig]), e_refined=r.e_refined,
                    residual=r.residual, variance=r.variance, ms=r.device_ms, hv_ms=r.hv_ms,
                    hv_launches=r.hv_launches, launches=r.kernel_launches, converged=bool(r.converged))

    def lanczos_sectors(self, n_up_list, steps: int, prec=FP64, seed: int = 123432, n_eig: int = 1,
                        refine: bool = False, breakdown: float = 0.0, keep_basis: int = 0, eps: float = 0.0):
        """Lanczos in several S^z sectors captured as one CUDA graph; one result dict per sector."""
        _torch()
        nu = np.ascontiguousarray(n_up_list, dtype=np.int32)
        ns = len(nu)
        al = [np.zeros(steps) for _ in range(ns)]
        be = [np.zeros(steps) for _ in range(ns)]
        res = (LanczosResult * ns)()
        for i in range(ns):
            res[i].alpha = al[i].ctypes.data
            res[i].beta = be[i].ctypes.data
        p = LanczosParams(steps, prec, seed, None, n_eig, int(refine), breakdown, 0, int(keep_basis), 0, float(eps),
                          None, 0)
        self._check(self._L.hphi_lanczos_run_sectors(self._h, nu.ctypes.data, ns, ctypes.byref(p), res, _stream()))
        out = []
        for i in range(ns):
            n = res[i].steps_done
            out.append(dict(n_up=int(nu[i]), alpha=al[i][:n], beta=be[i][:n], steps=n, eig=np.array(res[i].eig[:n_eig]),
                            e_refined=res[i].e_refined, residual=res[i].residual, variance=res[i].variance,
                            ms=res[i].device_ms, launches=res[i].kernel_launches, converged=bool(res[i].converged)))
        return out

    def inverse_iteration(self, x, energy: float, shift: float = 0.0, outer: int = 2, max_cg: int = 1000,
                          cg_tol: float = 0.0):
        """Section 3.4.1 inverse iteration by CG on the CUDA fp64 (complex128) tensor x, in place; returns
        dict(e, residual, variance, cg_steps, ms, launches)."""
        torch = _torch()
        want = torch.complex128 if self.is_complex else torch.float64
        if not (x.is_cuda and x.dtype == want and x.is_contiguous() and x.numel() == self.dim):
            raise LibraryError(-1, f"x must be a contiguous CUDA {want} tensor of length dim")
        p = InvitParams(float(energy), float(shift), int(outer), int(max_cg), float(cg_tol))
        r = InvitResult()
        self._check(self._L.hphi_inverse_iteration(self._h, ctypes.byref(p), _dptr(x), ctypes.byref(r), _stream()))
        return dict(e=r.e, residual=r.residual, variance=r.variance, cg_steps=r.cg_steps, ms=r.device_ms,
                    launches=r.kernel_launches)

    def tpq(self, n_starts: int, steps: int, l: float = 1.0, n_s: float = 0.0, prec=FP64, seed: int = 123432,
            psi0=None, profile: bool = False, obs_every: int = 0):
        """Section 3.5 mTPQ for n_starts interleaved starts; returns dict(u, h2, norm, beta, spec_heat, doublon,
        sz, sz2, ms, ...), arrays [steps, n_starts] (observables NaN where not measured)."""
        torch = _torch()
        if psi0 is not None:
            psi0 = psi0.to(device="cuda", dtype=torch.complex128 if self.is_complex else torch.float64).contiguous()
        out = {k: np.zeros((steps, n_starts)) for k in ("u", "h2", "norm", "beta", "spec_heat", "doublon", "sz", "sz2")}
        p = TpqParams(n_starts, steps, l, n_s, seed, _dptr(psi0) if psi0 is not None else None, prec, int(profile),
                      int(obs_every))
        r = TpqResult(out["u"].ctypes.data, out["h2"].ctypes.data, out["norm"].ctypes.data, 0.0, 0, 0.0, 0,
                      out["beta"].ctypes.data, out["spec_heat"].ctypes.data, out["doublon"].ctypes.data,
                      out["sz"].ctypes.data, out["sz2"].ctypes.data)
        self._check(self._L.hphi_tpq_run(self._h, ctypes.byref(p), ctypes.byref(r), _stream()))
        out.update(ms=r.device_ms, launches=r.kernel_launches, hv_ms=r.hv_ms, hv_launches=r.hv_launches)
        return out


def philox4x32_10(ctr, key):
    """Device Philox4x32-10 on arrays ctr [n, 4] and key [n, 2] (uint32); returns [n, 4] numpy uint32."""
    torch = _torch()
    L = load()
    c = torch.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).cuda()
    k = torch.as_tensor(np.ascontiguousarray(key, dtype=np.uint32).view(np.int32)).cuda()
    n = c.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    rc = L.hphi_philox4x32_10(_dptr(c), _dptr(k), _dptr(out), n, _stream())
    if rc:
        raise LibraryError(rc, L.hphi_last_error(None).decode())
    return out.cpu().numpy().view(np.uint32)
