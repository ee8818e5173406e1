"""Planted mistakes in the oracle, each caught by a pin of tests/test_oracle.py (CPU only).

A pin is worth the mistakes it catches.  Each case below plants one plausible mistake --
a dropped term, a wrong sign, a wrong index, a transposed operand -- in a copy of the oracle
(the C++ source compiled into a temporary library, or one Python function re-executed from
edited source), points the oracle package at the copy, and runs the pins that must now
fail.  The oracle itself is never modified; every copy lives in a temporary directory.
"""
import concurrent.futures
import ctypes
import os
import shutil
import subprocess
import types

import pytest

import oracle
from tests import test_oracle as T

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
CPP = os.path.join(ORACLE_DIR, "hphi_oracle.cpp")
PY = os.path.join(ORACLE_DIR, "__init__.py")

def _rows_philox_pin():
    import workloads as wl
    T.test_apply_H_rows_philox_matches_full_product(
        "heisenberg_4x3_sz6", lambda: wl.heisenberg_square(4, 3).with_basis(wl.BASIS_SZ, 6), 4)


# (name, text of the oracle, planted text, pins that must fail)
CPP_MUTANTS = [
    ("rank_wrong_binomial", "      r += binom(p, ones_left);\n", "      r += binom(p, ones_left - 1);\n",
     [lambda: T.test_rank_unrank_exhaustive(9), T.test_paper_sz0_basis_and_ranks]),
    ("unrank_off_by_one", "    if (r >= below) {\n", "    if (r > below) {\n",
     [lambda: T.test_rank_unrank_exhaustive(9)]),
    ("sector_filter", "    if (popcount64(s) == k) {\n", "    if (popcount64(s) >= k) {\n",
     [T.test_paper_sz0_basis_and_ranks]),
    ("sz_sign", "return cplx(b ? 0.5 : -0.5, 0.0); }", "return cplx(b ? -0.5 : 0.5, 0.0); }",
     [lambda: T.test_spin_elements_vs_kronecker(0)]),
    ("sy_transposed", "return b ? cplx(0.0, -0.5) : cplx(0.0, 0.5);", "return b ? cplx(0.0, 0.5) : cplx(0.0, -0.5);",
     [T.test_spin_field_y_sign, lambda: T.test_spin_elements_vs_kronecker(0)]),
    ("sx_dropped", "if (a == 0) return cplx(0.5, 0.0);", "if (a == 0) return cplx(0.0, 0.0);",
     [T.test_heisenberg_4ring_e0, lambda: T.test_spin_elements_vs_kronecker(0)]),
    ("field_sign", "el[ki ^ bi] += -h * ei;", "el[ki ^ bi] += h * ei;",
     [lambda: T.test_spin_elements_vs_kronecker(0)]),
    ("coupling_transposed", "m->coup_J[9 * t + 3 * a + b]", "m->coup_J[9 * t + 3 * b + a]",
     [lambda: T.test_spin_elements_vs_kronecker(0)]),
    ("jordan_wigner_sign_dropped",
     "  if (f->occ(q)) return 0;\n  const int sgn = (f->occupied_before(q) & 1) ? -1 : 1;\n",
     "  if (f->occ(q)) return 0;\n  const int sgn = 1;\n",
     [T.test_hop_sign_literal, lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("hopping_not_conjugated", "const cplx coef[2] = {-t, -std::conj(t)};", "const cplx coef[2] = {-t, -t};",
     [lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("onsite_U_sum_for_product", "(((up >> i) & 1u) * ((dn >> i) & 1u))", "(((up >> i) & 1u) + ((dn >> i) & 1u))",
     [T.test_two_site_hubbard_e0, lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("chemical_potential_sign", "    diag -= m->mu_val[k] *", "    diag += m->mu_val[k] *",
     [lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("lanczos_beta_term_dropped", "u[r] = u[r] - beta_k * vprev[r] - a_k * v[r];", "u[r] = u[r] - a_k * v[r];",
     [T.test_lanczos_ground_state_vs_dense]),
    ("second_pass_coefficient_index", "x[r] += coef[k + 1] * v[r];", "x[r] += coef[k] * v[r];",
     [T.test_lanczos_eigenvector_second_pass]),
    ("tpq_sign", "psi[r] = l * psi[r] - hp[r] / Ns;", "psi[r] = l * psi[r] + hp[r] / Ns;",
     [T.test_tpq_matches_matrix_power]),
    ("tpq_h2_scale", "h2_out[k - 1] = h2 / (Ns * Ns);", "h2_out[k - 1] = h2 / Ns;",
     [T.test_tpq_matches_matrix_power]),
    ("philox_weyl_constants_swapped", "const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;",
     "const uint32_t W0 = 0xBB67AE85u, W1 = 0x9E3779B9u;", [T.test_philox_known_answers]),
    ("box_muller_cos_sin_transposed", "  *g0 = rad * std::cos(ang);\n  *g1 = rad * std::sin(ang);\n",
     "  *g0 = rad * std::sin(ang);\n  *g1 = rad * std::cos(ang);\n", [T.test_start_vector_numbers]),
    ("real_pair_order_swapped", "*re = (e & 1) ? g1 : g0;", "*re = (e & 1) ? g0 : g1;",
     [T.test_start_vector_numbers]),
    ("sampled_rows_column_dropped", "start_element(seed, col * (uint64_t)nvec + (uint64_t)c,",
     "start_element(seed, col * (uint64_t)nvec,", [_rows_philox_pin]),
    ("binomial_divisor", "r = r * (unsigned)(n - k + i) / (unsigned)i;", "r = r * (unsigned)(n - k + i) / (unsigned)(i + 1);",
     [lambda: T.test_paper_dimension_statements("dim_13_6")]),
    ("density_term_squared", "diag += m->V_val[k] * ni * nj;", "diag += m->V_val[k] * ni * ni;",
     [lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("hop_operator_order", "  int sgn = annihilate(&f, q);\n  sgn *= create(&f, p);\n",
     "  int sgn = create(&f, p);\n  sgn *= annihilate(&f, q);\n",
     [T.test_hop_sign_literal, lambda: T.test_hubbard_elements_vs_jordan_wigner(0)]),
    ("lanczos_start_not_normalised", "++r) v[r] = v0[r] / nrm;", "++r) v[r] = v0[r];",
     [T.test_lanczos_ground_state_vs_dense]),
    ("lanczos_no_breakdown_stop", "    if (b_next <= brk * std::fmax(1.0, std::fabs(a_k))) break;\n", "",
     [T.test_lanczos_breakdown_on_one_state_sector]),
    ("hubbard_index_transposed", "return rank_same_popcount(dn, n) * dim_up + rank_same_popcount(up, n);",
     "return rank_same_popcount(up, n) * dim_dn + rank_same_popcount(dn, n);",
     [lambda: T.test_hubbard_sector_vs_jordan_wigner(2, 1)]),
    ("vector_block_column_dropped", "out[c] += el * v[col * nvec + c];", "out[c] += el * v[col * nvec];",
     [lambda: T.test_apply_H_vector_block_vs_independent_matrices(3)]),
    ("slice_offset_dropped", "const uint64_t r = r0 + (uint64_t)k;", "const uint64_t r = (uint64_t)k;",
     [T.test_apply_H_slice_rows]),
    ("tpq_norm_squared", "nrm_out[k - 1] = pn;", "nrm_out[k - 1] = pn * pn;", [T.test_tpq_matches_matrix_power]),
    ("popcount_counts_every_bit", "while (x) { c += (int)(x & 1u); x >>= 1; }", "while (x) { c += 1; x >>= 1; }",
     [T.test_paper_sz0_basis_and_ranks]),
]

# (name, function, text of oracle/__init__.py, planted text, pins that must fail)
PY_MUTANTS = [
    ("sz_half_dropped", "diag_observables", "(w * m2).sum(axis=0) / 2 / ww / ns", "(w * m2).sum(axis=0) / ww / ns",
     [T.test_diag_observables_spin_match_pauli_operators]),
    ("doublon_or_for_and", "diag_observables", "dbl = _popcount(up & dn).astype(np.float64)",
     "dbl = _popcount(up | dn).astype(np.float64)",
     [lambda: T.test_diag_observables_hubbard_match_fermion_operators("full")]),
    ("tpq_state_sign", "tpq_states", "y = l * x - apply_H(spec, x) / Ns", "y = l * x + apply_H(spec, x) / Ns",
     [T.test_tpq_states_are_normalised_matrix_powers]),
    ("inverse_iteration_forward", "inverse_iteration", "y = np.linalg.solve(A, y)", "y = A @ y",
     [T.test_inverse_iteration_converges_to_the_eigenvector]),
    ("convergence_on_ground_level", "lanczos_convergence_step", "e1 = ritz_values(alpha[:n], beta[:n])[1]",
     "e1 = ritz_values(alpha[:n], beta[:n])[0]", [T.test_lanczos_convergence_step_rule]),
    ("reorthogonalisation_dropped", "lanczos_reorth", "        w = w - Vm.T @ (Vm.conj() @ w)\n", "",
     [T.test_lanczos_reorth_keeps_the_basis_orthonormal]),
    ("hubbard_index_layout_transposed", "basis_configurations",
     "    up = np.tile(lu, len(ld))\n    dn = np.repeat(ld, len(lu))\n",
     "    up = np.repeat(lu, len(ld))\n    dn = np.tile(ld, len(lu))\n",
     [lambda: T.test_diag_observables_hubbard_match_fermion_operators("sector")]),
    ("ritz_beta_offset", "ritz_values", "e = np.asarray(beta[: n - 1], dtype=np.float64)",
     "e = np.asarray(beta[1:n], dtype=np.float64)", [T.test_lanczos_ground_state_vs_dense]),
    ("ritz_vector_wrong_column", "ritz_vector", "    return v[:, which]\n", "    return v[:, -1]\n",
     [T.test_lanczos_eigenvector_second_pass]),
]


def _plant(text, old, new, name):
    assert text.count(old) == 1, f"{name}: the planted site must occur exactly once in the oracle"
    return text.replace(old, new)


@pytest.fixture(scope="module")
def cpp_mutants(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(CPP).read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, old, new, _ in CPP_MUTANTS:
        cpp = d / f"{name}.cpp"
        cpp.write_text(_plant(src, old, new, name))
        jobs[name] = (str(cpp), str(d / f"lib{name}.so"))

    def compile_one(item):
        cpp, so = item
        subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", so, cpp], check=True)
        return so

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        out = dict(zip(jobs, ex.map(compile_one, jobs.values())))
    return out


def _expect_caught(pins, name):
    for pin in pins:
        with pytest.raises((AssertionError, oracle.OracleError)):
            pin()


@pytest.mark.parametrize("name,old,new,pins", CPP_MUTANTS, ids=[m[0] for m in CPP_MUTANTS])
def test_cpp_mutant_is_caught(cpp_mutants, monkeypatch, name, old, new, pins):
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(cpp_mutants[name])))
    _expect_caught(pins, name)


@pytest.mark.parametrize("name,func,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_is_caught(monkeypatch, name, func, old, new, pins):
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = PY
    exec(compile(_plant(open(PY).read(), old, new, name), PY, "exec"), mod.__dict__)
    monkeypatch.setattr(oracle, func, getattr(mod, func))
    _expect_caught(pins, name)


def test_unplanted_copy_passes_the_same_pins(tmp_path, monkeypatch):
    """The harness itself: an unmodified copy of the oracle, loaded the same way, passes."""
    so = str(tmp_path / "liboracle_copy.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", so, CPP], check=True)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(ctypes.CDLL(so)))
    T.test_rank_unrank_exhaustive(9)
    T.test_spin_elements_vs_kronecker(0)
    T.test_hubbard_elements_vs_jordan_wigner(0)
    T.test_lanczos_ground_state_vs_dense()
    T.test_tpq_matches_matrix_power()
    T.test_start_vector_numbers()
