"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test fixes one part of the oracle by a worked example printed in the paper, a
closed form, an independent textbook construction (Kronecker products / Jordan-Wigner
matrices in tests/_indep.py), brute force, or a published known-answer vector.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from tests import _indep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, *vals = line.split()
                out[k] = vals
    return out


# ----------------------------------------------------------------------------- basis
def test_paper_sz0_basis_and_ranks():
    g = _golden("paper_examples.txt")
    want = [int(x) for x in g["sz0_basis_4site"]]
    got = oracle.sector_list(4, 2).tolist()
    assert got == want
    assert [oracle.rank(s, 4) for s in want] == list(range(6))
    assert [oracle.unrank(r, 4, 2) for r in range(6)] == want


@pytest.mark.parametrize("key", ["dim_hubbard_18", "dim_13_6", "dim_13_9"])
def test_paper_dimension_statements(key):
    n, k, d = (int(x) for x in _golden("paper_examples.txt")[key])
    assert oracle.binom(n, k) ** 2 == d
    spec = wl.hubbard_ring(n).with_basis(wl.BASIS_NUMBER, k, k)
    assert oracle.dim(spec) == d


@pytest.mark.parametrize("n", [1, 2, 5, 9, 14])
def test_rank_unrank_exhaustive(n):
    for k in range(n + 1):
        lst = oracle.sector_list(n, k)
        assert len(lst) == math.comb(n, k)
        assert np.all(np.diff(lst.astype(np.int64)) > 0)
        for r, s in enumerate(lst.tolist()):
            assert _indep.popcount(s) == k
            assert oracle.rank(s, n) == r
            assert oracle.unrank(r, n, k) == s


def test_rank_unrank_36_bits_random():
    rng = np.random.default_rng(1)
    n, k = 36, 18
    D = math.comb(n, k)
    for r in rng.integers(0, D, size=2000).tolist() + [0, D - 1]:
        s = oracle.unrank(r, n, k)
        assert _indep.popcount(s) == k and s < (1 << n)
        assert oracle.rank(s, n) == r
    assert oracle.unrank(0, n, k) == (1 << k) - 1
    assert oracle.unrank(D - 1, n, k) == ((1 << k) - 1) << (n - k)


def test_paper_fermion_4ary_example():
    """Section 3.1: the 4-site configuration |0, up, dn, updn> is [0123]_4 = 27, one base-4
    digit per site (0 empty, 1 up, 2 down, 3 both; site 0 is the lowest digit).

    The digits of the paper's label give each site's up and down occupations.  On a model
    with distinct on-site U_i and chemical potentials mu_i, the oracle must put
    sum_i U_i n_i,up n_i,dn - mu_i n_i on the row of this configuration (row = dn * 2^N + up,
    its documented full-basis order), and an up-spin hop between sites 2 and 3 must connect
    that row to exactly one other: the configuration whose up electron moved from site 2 to
    site 3, with element -t (no modes lie between the two in the order up 0..3, dn 0..3).
    This pins the oracle's Hubbard diagonal, species assignment and row order against the
    paper's example."""
    g = [int(x) for x in _golden("paper_examples.txt")["fermion_4ary"]]
    label = g[4]
    digits = [(label >> (2 * site)) & 3 for site in range(4)]  # base-4 digits, site 0 first
    assert digits[::-1] == g[:4]                                 # the paper writes site 3 first
    n, t = 4, 0.75
    U = [1.0, 10.0, 100.0, 1000.0]
    mu = [0.001, 0.003, 0.009, 0.027]
    spec = wl.ModelSpec(kind=wl.HUBBARD, n_sites=n, onsite_U=list(enumerate(U)), chem_pot=list(enumerate(mu)),
                        hops=[(3, 2, 0, t)])
    want = sum(U[i] * (digits[i] == 3) - mu[i] * ((digits[i] & 1) + (digits[i] >> 1)) for i in range(n))
    up = sum(((d & 1) << i) for i, d in enumerate(digits))
    dn = sum((((d >> 1) & 1) << i) for i, d in enumerate(digits))
    assert (up, dn) == (0b0101, 0b0011)
    row = dn * (1 << n) + up
    H = oracle.dense_H(spec)
    assert abs(H[row, row].real - want) < 1e-12
    col = H[:, row].copy()
    col[row] = 0.0
    moved = dn * (1 << n) + (up ^ 0b1100)
    assert np.flatnonzero(np.abs(col) > 1e-15).tolist() == [moved]
    assert abs(col[moved] - (-t)) < 1e-15


# ----------------------------------------------------------------------------- spin H
def test_paper_xor_flip_example():
    """Section 3.3: (S+_0 S-_1 + S-_0 S+_1) = 2 (S^x S^x + S^y S^y) on bond (0, 1)."""
    g = _golden("paper_examples.txt")
    s_in, mask, s_out = (int(x) for x in g["xor_flip"])
    assert s_in ^ mask == s_out
    spec = wl.ModelSpec(kind=wl.SPIN, n_sites=4, couplings=[(0, 1, np.diag([2.0, 2.0, 0.0]))])
    H = oracle.dense_H(spec)
    col = H[:, s_in]
    assert abs(col[s_out] - 1.0) < 1e-15
    assert np.count_nonzero(np.abs(col) > 1e-15) == 1
    zero = int(g["xor_zero"][0])
    assert np.all(np.abs(H[:, zero]) < 1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spin_elements_vs_kronecker(seed):
    spec = wl.random_spin_model(5, 7, seed, complex_=True, fields=True)
    H = oracle.dense_H(spec)
    Href = _indep.dense_spin(spec)
    assert np.max(np.abs(H - Href)) < 1e-13


def test_spin_field_y_sign():
    """-h S^y on one site: <up|H|dn> = -h <up|S^y|dn> = -h (-i/2) = i h / 2."""
    h = 0.3
    spec = wl.ModelSpec(kind=wl.SPIN, n_sites=1, fields=[(0, (0.0, h, 0.0))])
    H = oracle.dense_H(spec)
    assert abs(H[1, 0] - 1j * h / 2) < 1e-15 and abs(H[0, 1] + 1j * h / 2) < 1e-15


@pytest.mark.parametrize("n,k", [(6, 3), (7, 2), (6, 0)])
def test_spin_sector_vs_kronecker(n, k):
    spec = wl.random_xxz_model(n, 9, seed=10 + n + k).with_basis(wl.BASIS_SZ, k)
    H = oracle.dense_H(spec)
    idx = _indep.spin_sector_indices(n, k)
    Href = _indep.dense_spin(spec.with_basis(wl.BASIS_FULL))[np.ix_(idx, idx)]
    assert H.shape == Href.shape
    assert np.max(np.abs(H - Href)) < 1e-13


@pytest.mark.parametrize("nvec", [3, 4])
def test_apply_H_vector_block_vs_independent_matrices(nvec):
    """A [dim][nvec] block (row-major: the nvec values of a row are adjacent) is multiplied
    column by column: against the Kronecker and Jordan-Wigner matrices, with different
    columns, so a column index dropped or mixed up fails."""
    for spec, dense in ((wl.random_spin_model(5, 7, 11, complex_=True, fields=True), _indep.dense_spin),
                        (wl.random_hubbard_model(3, 6, 12, complex_=True), _indep.dense_hubbard)):
        D = oracle.dim(spec)
        V = wl.gaussian_vector(20 + nvec, D, nvec, complex_=True)
        W = oracle.apply_H(spec, V)
        assert W.shape == (D, nvec)
        assert np.max(np.abs(W - dense(spec) @ V)) < 1e-12


def test_apply_H_slice_rows():
    """Rows [r0, r0 + n) of the product, for the CPU timing legs, equal those rows of the
    Kronecker matrix times v."""
    spec = wl.random_spin_model(6, 9, 13, complex_=True, fields=True)
    D = oracle.dim(spec)
    v = wl.gaussian_vector(31, D, 2, complex_=True)
    full = _indep.dense_spin(spec) @ v
    for r0, n in ((0, 5), (17, 23), (D - 9, 9)):
        assert np.max(np.abs(oracle.apply_H_slice(spec, v, r0, n) - full[r0:r0 + n])) < 1e-12


def test_sector_mismatch_is_reported():
    spec = wl.random_spin_model(4, 3, seed=3).with_basis(wl.BASIS_SZ, 2)
    with pytest.raises(oracle.OracleError):
        oracle.apply_H(spec, np.ones(6))


# ----------------------------------------------------------------------------- Hubbard H
@pytest.mark.parametrize("seed", [0, 1])
def test_hubbard_elements_vs_jordan_wigner(seed):
    spec = wl.random_hubbard_model(3, 6, seed, complex_=True)
    H = oracle.dense_H(spec)
    Href = _indep.dense_hubbard(spec)
    assert np.max(np.abs(H - Href)) < 1e-13


@pytest.mark.parametrize("na,nb", [(2, 1), (1, 1), (3, 0)])
def test_hubbard_sector_vs_jordan_wigner(na, nb):
    spec = wl.random_hubbard_model(3, 7, seed=5, complex_=True).with_basis(wl.BASIS_NUMBER, na, nb)
    H = oracle.dense_H(spec)
    idx = _indep.hubbard_sector_indices(3, na, nb)
    Href = _indep.dense_hubbard(spec.with_basis(wl.BASIS_FULL))[np.ix_(idx, idx)]
    assert np.max(np.abs(H - Href)) < 1e-13


def test_hubbard_interleaved_order_is_a_gauge():
    """The paper's per-site interleaving of up/down modes (section 3.1) orders the modes
    differently; the spectrum must not change."""
    spec = wl.random_hubbard_model(3, 6, seed=7, complex_=False)
    ev_ours = np.linalg.eigvalsh(oracle.dense_H(spec))
    ev_inter = np.linalg.eigvalsh(_indep.dense_hubbard(spec, mode_of=lambda i, s: 2 * i + s))
    assert np.max(np.abs(ev_ours - ev_inter)) < 1e-12


def test_hop_sign_literal():
    # modes: up 0..3 = 0..3, dn 0..3 = 4..7; <bra| c+_p c_q |ket>
    # bra has up sites {0, 2}; c+_2 c_0 (p=2, q=0): ket has up {0, 1}... choose explicitly
    # ket = up {0, 1}, bra = up {1, 2}: c_0 on ket: 0 occupied before -> +; c+_2 on up{1}: 1 before -> -
    assert oracle.hop_sign(0b0110, 0, 4, 2, 0) == -1
    assert oracle.hop_sign(0b0110, 0, 4, 0, 2) == 0  # bra must have mode p occupied


# ----------------------------------------------------------------------------- closed forms
def _e0(spec):
    return np.linalg.eigvalsh(oracle.dense_H(spec))[0]


def test_heisenberg_4ring_e0():
    assert abs(_e0(wl.heisenberg_ring(4)) - (-2.0)) < 1e-12


def test_two_site_hubbard_e0():
    t, U = 1.0, 8.0
    spec = wl.hubbard(2, [(0, 1)], t, U).with_basis(wl.BASIS_NUMBER, 1, 1)
    want = (U - math.sqrt(U * U + 16 * t * t)) / 2
    assert abs(_e0(spec) - want) < 1e-12


@pytest.mark.parametrize("na,nb,want", [(3, 3, -8.0), (2, 3, -7.0), (2, 2, -6.0), (1, 0, -2.0)])
def test_free_fermion_ring_band_sum(na, nb, want):
    # 6-site ring, U = 0: single-particle levels -2 cos(2 pi k / 6) = -2, -1, -1, 1, 1, 2
    spec = wl.hubbard_ring(6, 1.0, 0.0).with_basis(wl.BASIS_NUMBER, na, nb)
    assert abs(_e0(spec) - want) < 1e-12


def test_free_fermion_4x4_one_species_lanczos():
    """4x4 torus, 8 fermions of one species, U = 0: the sum of the 8 lowest levels of
    -2(cos kx + cos ky) is -4 - 2*(-... ) = -12."""
    lv = sorted(-2 * (math.cos(2 * math.pi * a / 4) + math.cos(2 * math.pi * b / 4)) for a in range(4) for b in range(4))
    want = sum(lv[:8])
    assert abs(want + 12.0) < 1e-12
    spec = wl.hubbard_square(4, 4, 1.0, 0.0).with_basis(wl.BASIS_NUMBER, 8, 0)
    v0 = wl.gaussian_vector(1, oracle.dim(spec))[:, 0]
    a, b = oracle.lanczos(spec, v0, 120)
    assert abs(oracle.ritz_values(a, b)[0] - want) < 1e-9


def test_majumdar_ghosh_point():
    n = 12
    spec = wl.j1j2_ring(n, 1.0, 0.5)
    e_sz0 = _e0(spec.with_basis(wl.BASIS_SZ, n // 2))
    assert abs(e_sz0 - (-3 * n / 8)) < 1e-10
    assert abs(_e0(spec.with_basis(wl.BASIS_SZ, n)) - n * 1.5 / 4) < 1e-12
    # one magnon: E(k) = N (J1 + J2)/4 + J1 (cos k - 1) + J2 (cos 2k - 1)
    ev = np.linalg.eigvalsh(oracle.dense_H(spec.with_basis(wl.BASIS_SZ, n - 1)))
    k = 2 * np.pi * np.arange(n) / n
    want = np.sort(n * 1.5 / 4 + (np.cos(k) - 1) + 0.5 * (np.cos(2 * k) - 1))
    assert np.max(np.abs(ev - want)) < 1e-12


def test_heisenberg_ring12_sector_minima():
    spec = wl.heisenberg_ring(12)
    mins = [_e0(spec.with_basis(wl.BASIS_SZ, k)) for k in range(13)]
    assert abs(mins[6] - (-5.387390917445)) < 1e-9
    assert abs(mins[0] - 3.0) < 1e-12 and abs(mins[12] - 3.0) < 1e-12
    for k in range(13):
        assert abs(mins[k] - mins[12 - k]) < 1e-10
    # ferromagnetic bound and monotonic in |Sz|
    for k in range(6):
        assert mins[k] >= mins[k + 1] - 1e-10


# ----------------------------------------------------------------------------- Lanczos
def test_lanczos_ground_state_vs_dense():
    spec = wl.heisenberg_ring(10).with_basis(wl.BASIS_SZ, 5)
    v0 = wl.gaussian_vector(3, oracle.dim(spec))[:, 0]
    a, b = oracle.lanczos(spec, v0, 80)
    H = oracle.dense_H(spec)
    ev = np.linalg.eigvalsh(H)
    assert abs(oracle.ritz_values(a, b)[0] - ev[0]) < 1e-10
    # first coefficients straight from the dense matrix
    v = v0 / np.linalg.norm(v0)
    hv = H @ v
    a0 = np.vdot(v, hv).real
    assert abs(a[0] - a0) < 1e-12
    assert abs(b[0] - np.linalg.norm(hv - a0 * v)) < 1e-12


def test_lanczos_shift_invariance():
    """Section 3.4: the Krylov space of H + a I equals that of H, so alpha shifts by a and
    beta is unchanged.  A uniform chemical potential at fixed particle number is such a
    shift (a = -mu (N_up + N_dn))."""
    base = wl.hubbard_ring(6, 1.0, 4.0).with_basis(wl.BASIS_NUMBER, 3, 2)
    mu = 0.7
    shifted = wl.ModelSpec(**{**base.__dict__, "chem_pot": [(i, mu) for i in range(6)]})
    v0 = wl.gaussian_vector(4, oracle.dim(base))[:, 0]
    a1, b1 = oracle.lanczos(base, v0, 30)
    a2, b2 = oracle.lanczos(shifted, v0, 30)
    assert np.max(np.abs((a2 - a1) - (-mu * 5))) < 1e-12
    assert np.max(np.abs(b2 - b1)) < 1e-12


def test_lanczos_breakdown_on_one_state_sector():
    spec = wl.j1j2_ring(8, 1.0, 0.5).with_basis(wl.BASIS_SZ, 8)
    a, b = oracle.lanczos(spec, np.ones(1), 10)
    assert len(a) == 1 and abs(a[0] - 8 * 1.5 / 4) < 1e-14 and b[0] < 1e-14


def test_lanczos_eigenvector_second_pass():
    spec = wl.heisenberg_ring(10).with_basis(wl.BASIS_SZ, 5)
    v0 = wl.gaussian_vector(5, oracle.dim(spec))[:, 0]
    a, b = oracle.lanczos(spec, v0, 60)
    e0 = oracle.ritz_values(a, b)[0]
    x = oracle.lanczos_vector(spec, v0, a, b, oracle.ritz_vector(a, b, 0))
    hx = oracle.apply_H(spec, x)
    xx = np.vdot(x, x).real
    erq = np.vdot(x, hx).real / xx
    assert abs(erq - e0) < 1e-9
    assert np.linalg.norm(hx - erq * x) / math.sqrt(xx) < 1e-5


# ----------------------------------------------------------------------------- TPQ
def test_tpq_matches_matrix_power():
    spec = wl.kitaev_honeycomb(2, 2, -1.0, 0.05)
    D = oracle.dim(spec)
    psi0 = wl.gaussian_vector(7, D, complex_=True)[:, 0]
    K, l = 12, 1.0
    u, h2, nrm, psiK = oracle.tpq(spec, psi0, K, l, want_state=True)
    H = _indep.dense_spin(spec)
    A = l * np.eye(D) - H / spec.n_sites
    ref = np.linalg.matrix_power(A, K) @ psi0
    ref /= np.linalg.norm(ref)
    assert np.max(np.abs(psiK - ref)) < 1e-12
    p = psi0 / np.linalg.norm(psi0)
    assert abs(u[0] - np.vdot(p, H @ p).real / spec.n_sites) < 1e-13
    assert abs(h2[0] - np.linalg.norm(H @ p) ** 2 / spec.n_sites ** 2) < 1e-13
    assert abs(nrm[0] - np.linalg.norm(A @ p)) < 1e-13


def test_kitaev_trace_h2_closed_form():
    """Tr H^2 / D = sum_bonds K^2/16 + sum_sites sum_a h_a^2 / 4 (distinct Pauli strings are
    trace-orthogonal), and Tr H = 0.  Pins the honeycomb geometry (12 bonds on 2x2 cells)."""
    K, h = -1.0, 0.05
    spec = wl.kitaev_honeycomb(2, 2, K, h)
    assert len(spec.couplings) == 12
    H = oracle.dense_H(spec)
    D = H.shape[0]
    assert abs(np.trace(H).real / D) < 1e-14
    want = 12 * K * K / 16 + 8 * 3 * h * h / 4
    assert abs(np.trace(H @ H).real / D - want) < 1e-12
    assert len(wl.kitaev_honeycomb(4, 3, K, h).couplings) == 36


def test_tpq_vs_canonical_ensemble():
    """The paper's own validation (section 5.1): TPQ energies at beta_k agree with the
    canonical ensemble from full diagonalization within the sample-to-sample spread."""
    spec = wl.kitaev_honeycomb(2, 2, -1.0, 0.05)
    Ns = spec.n_sites
    ev = np.linalg.eigvalsh(oracle.dense_H(spec))
    D = len(ev)
    K, l, R = 60, 1.0, 8
    us = []
    for r in range(R):
        psi0 = wl.gaussian_vector(100 + r, D, complex_=True)[:, 0]
        u, _, _ = oracle.tpq(spec, psi0, K, l)
        us.append(u)
    us = np.array(us)
    for k in (10, 30, 59):
        uk = us[:, k]
        beta = np.mean(2 * k / Ns / (l - uk))
        w = np.exp(-beta * (ev - ev[0]))
        e_can = np.sum(w * ev) / np.sum(w) / Ns
        assert abs(np.mean(uk) - e_can) < 4 * np.std(uk) + 2e-3


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    kat = _golden("philox4x32_10_kat.txt")
    for name, vals in kat.items():
        v = [int(x, 16) for x in vals]
        ctr, key, want = v[0:4], v[4:6], v[6:10]
        assert oracle.philox4x32_10(ctr, key).tolist() == want, name


def test_start_vector_numbers():
    """Start vectors (appendix A.2 / A.4: random coefficients; a seeded Gaussian): standard-normal
    moments, real elements 2p and 2p + 1 the two numbers of Philox block p and complex element p
    both of them; the mapping from Philox words pinned on the published known-answer block with
    counter (0, 0, 0, 0) through the textbook Box-Muller transform (numpy's log, cos, sin)."""
    idx = np.arange(200000, dtype=np.uint64)
    g = oracle.random_at(123432, idx, complex_=True)
    for part in (g.real, g.imag):
        assert abs(part.mean()) < 0.01 and abs(part.var() - 1.0) < 0.01
        assert abs(np.mean(part ** 4) - 3.0) < 0.05
    r = oracle.random_at(123432, idx[:200], complex_=False).real
    assert np.array_equal(r[0::2], g[:100].real) and np.array_equal(r[1::2], g[:100].imag)
    kat = _golden("philox4x32_10_kat.txt")
    v = [int(x, 16) for x in kat["zeros"]]
    assert v[0:6] == [0] * 6
    w = v[6:10]
    ua = (((((w[0] << 32) | w[1]) >> 11)) + 0.5) / 2.0 ** 53
    ub = (((((w[2] << 32) | w[3]) >> 11)) + 0.5) / 2.0 ** 53
    rad = np.sqrt(-2.0 * np.log(ua))
    got = oracle.random_at(0, np.array([0], dtype=np.uint64), complex_=True)[0]
    assert abs(got.real - rad * np.cos(2 * np.pi * ub)) < 1e-14 and abs(got.imag - rad * np.sin(2 * np.pi * ub)) < 1e-14
    pair = oracle.random_at(0, np.array([0, 1], dtype=np.uint64), complex_=False).real
    assert pair[0] == got.real and pair[1] == got.imag


def test_tpq_deferred_norm_identity():
    """The identity the GPU's mTPQ step uses instead of a third reduction: for a unit psi,
    |(l - H/N_s) psi|^2 = l^2 - 2 l u + <H^2>/N_s^2, with u = <psi|H|psi>/N_s (section 3.5).
    Checked on the oracle's own records, which take the norm directly."""
    spec = wl.kitaev_honeycomb(2, 2)
    psi0 = wl.gaussian_vector(17, oracle.dim(spec), 1, complex_=True)[:, 0]
    for l in (1.0, 1.5):
        u, h2, nrm = oracle.tpq(spec, psi0, 12, l)
        assert np.max(np.abs(nrm ** 2 - (l * l - 2.0 * l * u + h2))) < 1e-12


# ----------------------------------------------------------------------------- sampled rows
@pytest.mark.parametrize("name,mk", [
    ("heisenberg_4x3_sz6", lambda: wl.heisenberg_square(4, 3).with_basis(wl.BASIS_SZ, 6)),
    ("xxz_complex_sector", lambda: wl.random_xxz_model(11, 20, seed=8).with_basis(wl.BASIS_SZ, 5)),
    ("kitaev_2x2_full", lambda: wl.kitaev_honeycomb(2, 2)),
    ("hubbard_3x2_32", lambda: wl.hubbard_square(3, 2).with_basis(wl.BASIS_NUMBER, 3, 2)),
    ("hubbard_random_complex", lambda: wl.random_hubbard_model(5, 10, seed=4).with_basis(wl.BASIS_NUMBER, 2, 3)),
])
@pytest.mark.parametrize("nvec", [1, 4])
def test_apply_H_rows_philox_matches_full_product(name, mk, nvec):
    """The sampled-row product behind the full-size GPU checks regenerates each element of v
    from its Philox index: column c of a [dim][nvec] block is element r * nvec + c.  Rows of
    it must equal the plain product H v on the same vector built from the generator's
    element values (column c of the block, all rows)."""
    spec = mk()
    D = oracle.dim(spec)
    cplx = spec.is_complex
    seed = 4711 + nvec
    rows = np.unique(np.concatenate([[0, D - 1], np.random.default_rng(3).integers(0, D, size=200)]))
    for c in sorted({0, nvec - 1}):
        v = oracle.random_at(seed, np.arange(D, dtype=np.uint64) * nvec + c, cplx)
        full = oracle.apply_H(spec, v)
        got = oracle.apply_H_rows_philox(spec, rows.astype(np.uint64), seed, cplx, nvec, c)
        assert np.max(np.abs(got - full[rows])) <= 1e-13 * np.max(np.abs(full))
        if not cplx:
            assert np.max(np.abs(got.imag)) == 0.0


# ----------------------------------------------------------------------------- TPQ observables
def _num_ops(n):
    c = _indep.fermion_ops(2 * n)
    return [x.conj().T @ x for x in c]


@pytest.mark.parametrize("basis", ["full", "sector"])
def test_diag_observables_hubbard_match_fermion_operators(basis):
    """Doubly occupied sites and S^z_total of a Hubbard state against the Jordan-Wigner
    number operators (mode i + n s, full-basis index up + 2^n dn).  The sector (3, 2) has
    different up and down dimensions (4 and 6), so a transposed (up, down) index layout
    changes the result."""
    n = 4
    spec = wl.hubbard(n, [], U=1.0)
    num = _num_ops(n)
    Dop = sum(num[i] @ num[i + n] for i in range(n)).real
    Sz = sum(num[i] - num[i + n] for i in range(n)).real / 2
    if basis == "full":
        idx = np.arange(4 ** n)
    else:
        spec = spec.with_basis(wl.BASIS_NUMBER, 3, 2)
        idx = _indep.hubbard_sector_indices(n, 3, 2)
    psi = wl.gaussian_vector(5, len(idx), nvec=3, complex_=True)
    d, sz, sz2 = oracle.diag_observables(spec, psi)
    full = np.zeros((4 ** n, 3), dtype=complex)
    full[idx] = psi
    for c in range(3):
        x = full[:, c]
        nn = np.vdot(x, x).real
        assert abs(d[c] - np.vdot(x, Dop @ x).real / nn / n) < 1e-13
        assert abs(sz[c] - np.vdot(x, Sz @ x).real / nn / n) < 1e-13
        assert abs(sz2[c] - np.vdot(x, Sz @ Sz @ x).real / nn / n) < 1e-13
    if basis == "sector":
        assert np.allclose(sz, (3 - 2) / 2 / n, atol=1e-15) and np.allclose(sz2, 0.25 / n, atol=1e-15)
    # the oracle's own U term is the doublon operator
    HU = oracle.dense_H(spec)
    x = psi[:, 0]
    assert abs(d[0] - np.vdot(x, HU @ x).real / np.vdot(x, x).real / n) < 1e-13


def test_diag_observables_spin_match_pauli_operators():
    n = 7
    spec = wl.heisenberg_ring(n)
    Sz = sum(_indep.site_op(_indep.SPIN_OPS[2], k, n) for k in range(n)).real
    psi = wl.gaussian_vector(9, 2 ** n, nvec=2, complex_=True)
    d, sz, sz2 = oracle.diag_observables(spec, psi)
    assert np.all(d == 0)
    for c in range(2):
        x = psi[:, c]
        nn = np.vdot(x, x).real
        assert abs(sz[c] - np.vdot(x, Sz @ x).real / nn / n) < 1e-13
        assert abs(sz2[c] - np.vdot(x, Sz @ Sz @ x).real / nn / n) < 1e-13
    sec = spec.with_basis(wl.BASIS_SZ, 2)
    d, sz, sz2 = oracle.diag_observables(sec, wl.gaussian_vector(1, oracle.dim(sec)))
    assert abs(sz - (2 - n / 2) / n) < 1e-15 and abs(sz2 - (2 - n / 2) ** 2 / n) < 1e-15


def test_tpq_states_are_normalised_matrix_powers():
    spec = wl.hubbard_tilted8(U=8.0).with_basis(wl.BASIS_NUMBER, 2, 2)
    D = oracle.dim(spec)
    psi0 = wl.gaussian_vector(3, D)[:, 0]
    K, l = 6, 5.0
    st = oracle.tpq_states(spec, psi0, K, l)
    A = l * np.eye(D) - oracle.dense_H(spec) / spec.n_sites
    ref = psi0.astype(complex)
    for k in range(K):
        r = ref / np.linalg.norm(ref)
        assert np.max(np.abs(st[k] - r)) < 1e-13
        ref = A @ ref
    u, _, _ = oracle.tpq(spec, psi0, K, l)
    H = oracle.dense_H(spec)
    for k in range(K):
        assert abs(u[k] - np.vdot(st[k], H @ st[k]).real / spec.n_sites) < 1e-12


def test_tilted8_cluster_geometry():
    """Section 5.1's cluster: 8 sites, every site 4 distinct neighbours, 16 bonds; the
    periodic 4x4 cluster from the same construction has the square lattice's 32 bonds."""
    n, bonds = wl.tilted_square_bonds((2, 2), (-2, 2))
    assert n == 8 and len(bonds) == 16
    deg = np.zeros(n, dtype=int)
    for i, j in bonds:
        deg[i] += 1
        deg[j] += 1
    assert np.all(deg == 4)
    n16, b16 = wl.tilted_square_bonds((4, 0), (0, 4))
    assert n16 == 16 and len(b16) == 32
    # the 8-site cluster's free-fermion levels: -2t (cos kx + cos ky) over its 8 momenta
    spec = wl.hubbard_tilted8(U=0.0).with_basis(wl.BASIS_NUMBER, 1, 0)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_H(spec)))
    ks = [(kx, ky) for kx in range(4) for ky in range(4) if (2 * kx + 2 * ky) % 4 == 0 and (-2 * kx + 2 * ky) % 4 == 0]
    want = np.sort([-2 * (math.cos(math.pi * kx / 2) + math.cos(math.pi * ky / 2)) for kx, ky in ks])
    assert len(ks) == 8 and np.allclose(ev, want, atol=1e-12)


def test_inverse_iteration_converges_to_the_eigenvector():
    """Section 3.4.1 on a small sector: from a rough vector and an energy just above E_0, a few
    shifted solves reach numpy's ground state; E = E_0 + delta/2 keeps the operator definite."""
    spec = wl.heisenberg_ring(12).with_basis(wl.BASIS_SZ, 6)
    H = oracle.dense_H(spec).real
    ev, V = np.linalg.eigh(H)
    assert ev[1] - ev[0] > 0.1  # a non-degenerate ground state
    x0 = V[:, 0] + 0.3 * wl.gaussian_vector(4, len(ev))[:, 0] / math.sqrt(len(ev))
    y = oracle.inverse_iteration(spec, x0, ev[0] + 1e-3, 1e-2, outer=4)
    assert abs(abs(np.vdot(y, V[:, 0])) - 1.0) < 1e-12
    # the error shrinks by (E0 - E + delta) / (E1 - E + delta) per step
    y1 = oracle.inverse_iteration(spec, x0, ev[0] + 1e-3, 1e-2, outer=1)
    err0 = 1 - abs(np.vdot(x0 / np.linalg.norm(x0), V[:, 0])) ** 2
    err1 = 1 - abs(np.vdot(y1, V[:, 0])) ** 2
    assert err1 < err0 * ((1e-2 - 1e-3) / (ev[1] - ev[0] - 1e-3 + 1e-2)) ** 2 * 10


def _lanczos_diag(d, m):
    """Lanczos with full reorthogonalisation on diag(d) from the uniform vector, in plain numpy
    (the oracle's recurrence is pinned elsewhere)."""
    v0 = np.ones(len(d)) / math.sqrt(len(d))
    a, b, Q = [], [], [v0]
    q_prev, q, bk = np.zeros_like(v0), v0, 0.0
    for _ in range(m):
        w = d * q - bk * q_prev
        ak = q @ w
        w -= ak * q
        Qm = np.array(Q)
        w -= Qm.T @ (Qm @ w)
        bk = np.linalg.norm(w)
        a.append(ak)
        b.append(bk)
        q_prev, q = q, w / bk
        Q.append(q)
    return a, b


def test_lanczos_convergence_step_rule():
    """Appendix C's rule on recurrences with a known answer: T from a diagonal matrix converges;
    the rule returns an odd n >= 7 at which the first excited Ritz value has settled, and None
    when eps is unreachable.  In the second spectrum the ground level is isolated (settled
    after 9 steps) while the first excited level sits next to the bulk, so a rule that watched
    the ground level would stop with the first excited value still 0.06 off."""
    d = np.concatenate([[-3.0, -2.0], np.linspace(0, 1, 200)])
    a, b = _lanczos_diag(d, 40)
    n = oracle.lanczos_convergence_step(a, b, 1e-10)
    assert n is not None and n >= 7 and (n - 5) % 2 == 0
    e1n = oracle.ritz_values(a[:n], b[:n])[1]
    assert abs(e1n - (-2.0)) < 1e-8
    assert oracle.lanczos_convergence_step(a[:9], b[:9], 1e-300) is None
    d = np.concatenate([[-10.0, -1.05], np.linspace(-1, 1, 300)])
    a, b = _lanczos_diag(d, 80)
    n = oracle.lanczos_convergence_step(a, b, 1e-10)
    assert n is not None and n > 20 and (n - 5) % 2 == 0
    assert abs(oracle.ritz_values(a[:n], b[:n])[1] - (-1.05)) < 1e-8


def test_lanczos_reorth_keeps_the_basis_orthonormal():
    """Full reorthogonalisation: the Lanczos vectors stay orthonormal to rounding long after the
    plain recurrence has lost orthogonality, the first steps equal the plain recurrence's, and
    the Ritz values show no spurious copies of converged eigenvalues (each lowest Ritz value is
    a distinct eigenvalue of H)."""
    spec = wl.heisenberg_ring(10)
    D = oracle.dim(spec)
    v0 = oracle.random_at(11, np.arange(D, dtype=np.uint64), False)
    a, b, V = oracle.lanczos_reorth(spec, v0, 120, want_vectors=True)
    G = V.conj() @ V.T
    assert np.max(np.abs(G - np.eye(len(V)))) < 1e-12
    ap, bp = oracle.lanczos(spec, v0, 120)
    assert np.max(np.abs(a[:10] - ap[:10])) < 1e-12 and np.max(np.abs(b[:10] - bp[:10])) < 1e-12
    evs = np.linalg.eigvalsh(oracle.dense_H(spec).real)
    mult = lambda e, vals: int(np.sum(np.abs(vals - e) < 1e-7))  # noqa: E731
    rv = oracle.ritz_values(a, b)[:6]
    for e in rv:  # every low Ritz value is an eigenvalue, at most as often as its multiplicity
        assert np.min(np.abs(evs - e)) < 1e-9 and mult(e, rv) <= mult(e, evs)
    assert mult(evs[0], evs) == 1 and mult(evs[0], rv) == 1
    # the plain recurrence has spurious copies of the (non-degenerate) ground state by now
    rp = oracle.ritz_values(ap, bp)[:6]
    assert mult(evs[0], rp) >= 2


def test_tilted18_cluster_of_section_5_2_1():
    """The 18-site cluster (a0 = (3, 3), a1 = (-3, 3)): 36 bonds, coordination 4, the sector
    dimension (18 C 9)^2 quoted in section 5.2.1, and one-particle levels
    -2t (cos kx + cos ky) over the cluster's 18 momenta."""
    W = wl.workload("hubbard_18_sz0_tpq")
    spec = W["model"]
    assert spec.n_sites == 18 and oracle.dim(spec) == 2_363_904_400 == W["dim"]
    n, bonds = wl.tilted_square_bonds((3, 3), (-3, 3))
    assert len(bonds) == 36
    deg = np.bincount(np.array(bonds).ravel(), minlength=n)
    assert np.all(deg == 4)
    one = wl.hubbard(n, bonds, 1.0, 0.0).with_basis(wl.BASIS_NUMBER, 1, 0)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_H(one)))
    ks = [(kx, ky) for kx in range(6) for ky in range(6) if (3 * kx + 3 * ky) % 6 == 0 and (-3 * kx + 3 * ky) % 6 == 0]
    want = np.sort([-2 * (math.cos(math.pi * kx / 3) + math.cos(math.pi * ky / 3)) for kx, ky in ks])
    assert len(ks) == 18 and np.allclose(ev, want, atol=1e-12)
