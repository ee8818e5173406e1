// Reference oracle for the Lanczos / microcanonical-TPQ hot path of HPhi
// (Kawamura et al., "Quantum lattice model solver HPhi", Comput. Phys. Commun. 2017).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, deliberately literal CPU
// restatement of what the method computes.  It exists so that the CUDA library can be
// checked against something written independently from the paper.  It shares no code,
// header, table or constant with the CUDA library and must never be linked into it.
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
//
// Everything is computed in fp64 / complex<double>.  Matrix elements are evaluated one
// single-site operator at a time, fermion signs by literally counting occupied modes in
// front of the mode an operator acts on, and basis ranks by the counting definition
// "number of sector states smaller than s".  No blocking, fusion or reordering.
//
// Conventions (readings of the paper, each stated where it is used):
//  * spin-1/2 site i <-> bit i of the configuration, bit = 1 <-> spin up (section 3.3,
//    the 4-site example whose configurations are written with site 0 rightmost);
//  * S = sigma / 2; S^y|up> = (i/2)|down>, S^y|down> = (-i/2)|up>;
//  * spin Hamiltonian (section 2.3, "Spin" model): sum_bonds sum_ab J^{ab} S_i^a S_j^b
//    - sum_i h_i . S_i  (the paper writes the fields as -h S^z - Gamma S^x);
//  * fermion modes are ordered (up,0) .. (up,N-1), (down,0) .. (down,N-1); a creation or
//    annihilation operator on mode m picks up (-1)^(number of occupied modes before m);
//  * Hubbard Hamiltonian (section 2.3, "Fermion Hubbard"): - t c+_i c_j - conj(t) c+_j c_i
//    per listed hop and spin, U n_up n_dn per listed site, V n_i n_j per listed pair,
//    -mu n_i per listed chemical-potential site;
//  * basis index: spin full basis index = s; spin Sz sector index = rank of s among the
//    states with popcount(s) = n_up in ascending order (section 3.1); Hubbard index =
//    rank_dn(dn) * dim_up + rank_up(up).
//
// Parity status: every function here is pinned by the CPU tests in tests/ (closed forms,
// brute force, worked examples of the paper and published known-answer vectors).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

typedef std::complex<double> cplx;

extern "C" {

struct or_model {
  int kind;      // 0 = spin-1/2, 1 = Hubbard
  int n_sites;
  int basis;     // 0 = full, 1 = fixed Sz (spin) , 2 = fixed (N_up, N_dn) (Hubbard)
  int n_a;       // spin: number of up spins; Hubbard: N_up
  int n_b;       // Hubbard: N_dn
  int n_coup;  const int* coup_ij;  const double* coup_J;    // [n][2], [n][9] row-major J[a][b]
  int n_field; const int* field_i;  const double* field_h;   // [n], [n][3] (hx, hy, hz)
  int n_hop;   const int* hop_ij;   const int* hop_spin; const double* hop_t;  // [n][2],[n],[n][2] (re, im)
  int n_U;     const int* U_i;      const double* U_val;
  int n_V;     const int* V_ij;     const double* V_val;
  int n_mu;    const int* mu_i;     const double* mu_val;
};

}  // extern "C"

namespace {

// ---------------------------------------------------------------- combinatorics
uint64_t binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  // multiplicative formula; each intermediate is an exact binomial coefficient C(n-k+i, i)
  unsigned __int128 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (unsigned)(n - k + i) / (unsigned)i;
  return (uint64_t)r;
}

int popcount64(uint64_t x) {
  int c = 0;
  while (x) { c += (int)(x & 1u); x >>= 1; }
  return c;
}

// Rank of s among all n_bits-bit strings with the same popcount, ascending: the number
// of such strings that are smaller than s.  Counted position by position from the most
// significant bit: at each set bit p, every string that agrees with s above p, has 0 at
// p and places the remaining ones anywhere below p is smaller than s.
uint64_t rank_same_popcount(uint64_t s, int n_bits) {
  int ones_left = popcount64(s);
  uint64_t r = 0;
  for (int p = n_bits - 1; p >= 0; --p) {
    if ((s >> p) & 1u) {
      r += binom(p, ones_left);
      --ones_left;
    }
  }
  return r;
}

// Inverse of rank_same_popcount: the r-th (0-based) n_bits-bit string with k ones.
uint64_t unrank_same_popcount(uint64_t r, int n_bits, int k) {
  uint64_t s = 0;
  int ones_left = k;
  for (int p = n_bits - 1; p >= 0 && ones_left > 0; --p) {
    uint64_t below = binom(p, ones_left);  // strings with 0 at p (and the ones below p)
    if (r >= below) {
      s |= (uint64_t)1 << p;
      r -= below;
      --ones_left;
    }
  }
  return s;
}

// ---------------------------------------------------------------- basis
struct Basis {
  int kind, n, mode, na, nb;
  uint64_t dim_up = 0, dim_dn = 0, dim = 0;

  bool init(const or_model* m) {
    kind = m->kind; n = m->n_sites; mode = m->basis; na = m->n_a; nb = m->n_b;
    if (kind == 0) {
      if (n < 1 || n > 63) return false;
      if (mode == 0) dim = (uint64_t)1 << n;
      else if (mode == 1) { if (na < 0 || na > n) return false; dim = binom(n, na); }
      else return false;
      return true;
    }
    if (kind == 1) {
      if (n < 1 || n > 31) return false;
      if (mode == 0) { dim_up = dim_dn = (uint64_t)1 << n; }
      else if (mode == 2) {
        if (na < 0 || na > n || nb < 0 || nb > n) return false;
        dim_up = binom(n, na); dim_dn = binom(n, nb);
      } else return false;
      dim = dim_up * dim_dn;
      return true;
    }
    return false;
  }
  // spin: configuration of basis index r
  uint64_t spin_state(uint64_t r) const { return mode == 0 ? r : unrank_same_popcount(r, n, na); }
  // spin: index of configuration s, or UINT64_MAX if s is outside the basis
  uint64_t spin_index(uint64_t s) const {
    if (mode == 0) return s;
    if (popcount64(s) != na) return UINT64_MAX;
    return rank_same_popcount(s, n);
  }
  void hub_state(uint64_t r, uint64_t* up, uint64_t* dn) const {
    uint64_t ru = r % dim_up, rd = r / dim_up;
    if (mode == 0) { *up = ru; *dn = rd; return; }
    *up = unrank_same_popcount(ru, n, na);
    *dn = unrank_same_popcount(rd, n, nb);
  }
  uint64_t hub_index(uint64_t up, uint64_t dn) const {
    if (mode == 0) return dn * dim_up + up;
    if (popcount64(up) != na || popcount64(dn) != nb) return UINT64_MAX;
    return rank_same_popcount(dn, n) * dim_up + rank_same_popcount(up, n);
  }
};

// ---------------------------------------------------------------- spin matrix elements
// <b | S^a | b'> for one site, b = bra bit; returns the value and sets *b_ket to the only
// ket bit with a non-zero element.
cplx site_elem(int a, int b, int* b_ket) {
  if (a == 2) { *b_ket = b; return cplx(b ? 0.5 : -0.5, 0.0); }          // S^z diagonal
  *b_ket = 1 - b;                                                         // S^x, S^y flip
  if (a == 0) return cplx(0.5, 0.0);
  return b ? cplx(0.0, -0.5) : cplx(0.0, 0.5);                           // <up|S^y|dn> = -i/2
}

// Visits every non-zero element <s_r|H|s'> of row r of a spin model as f(col(s'), value).
// The nine operator strings S^a_i S^b_j of a coupling are summed per target configuration
// first, so strings that cancel (e.g. S^x S^x + S^y S^y on parallel spins) do not count as
// leaving the basis.  Returns false if a non-zero element reaches a configuration outside
// the basis.
template <class F>
bool spin_row_elems(const or_model* m, const Basis& B, uint64_t r, F f) {
  const uint64_t s = B.spin_state(r);
  bool ok = true;
  for (int t = 0; t < m->n_coup; ++t) {
    const int i = m->coup_ij[2 * t], j = m->coup_ij[2 * t + 1];
    const int bi = (int)((s >> i) & 1u), bj = (int)((s >> j) & 1u);
    cplx el[2][2] = {{0.0, 0.0}, {0.0, 0.0}};  // [flip i][flip j]
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) {
        const double J = m->coup_J[9 * t + 3 * a + b];
        if (J == 0.0) continue;
        int ki, kj;
        const cplx ei = site_elem(a, bi, &ki);
        const cplx ej = site_elem(b, bj, &kj);
        el[ki ^ bi][kj ^ bj] += J * ei * ej;
      }
    }
    for (int fi = 0; fi < 2; ++fi)
      for (int fj = 0; fj < 2; ++fj) {
        if (el[fi][fj] == cplx(0.0, 0.0)) continue;
        const uint64_t sk = s ^ ((uint64_t)fi << i) ^ ((uint64_t)fj << j);
        const uint64_t col = B.spin_index(sk);
        if (col == UINT64_MAX) { ok = false; continue; }
        f(col, el[fi][fj]);
      }
  }
  for (int q = 0; q < m->n_field; ++q) {
    const int i = m->field_i[q];
    const int bi = (int)((s >> i) & 1u);
    cplx el[2] = {0.0, 0.0};  // [flip i]
    for (int a = 0; a < 3; ++a) {
      const double h = m->field_h[3 * q + a];
      if (h == 0.0) continue;
      int ki;
      const cplx ei = site_elem(a, bi, &ki);
      el[ki ^ bi] += -h * ei;
    }
    for (int fi = 0; fi < 2; ++fi) {
      if (el[fi] == cplx(0.0, 0.0)) continue;
      const uint64_t col = B.spin_index(s ^ ((uint64_t)fi << i));
      if (col == UINT64_MAX) { ok = false; continue; }
      f(col, el[fi]);
    }
  }
  return ok;
}

// ---------------------------------------------------------------- fermion operators
// Occupation of mode q in the combined string: modes 0..n-1 are up, n..2n-1 are down.
struct Fock {
  uint64_t up, dn;
  int n;
  int occ(int q) const { return q < n ? (int)((up >> q) & 1u) : (int)((dn >> (q - n)) & 1u); }
  void set(int q, int val) {
    if (q < n) up = (up & ~((uint64_t)1 << q)) | ((uint64_t)val << q);
    else dn = (dn & ~((uint64_t)1 << (q - n))) | ((uint64_t)val << (q - n));
  }
  int occupied_before(int q) const {
    int c = 0;
    for (int p = 0; p < q; ++p) c += occ(p);
    return c;
  }
};

// Apply c_q to |f>: returns the sign (0 if the mode is empty) and updates f.
int annihilate(Fock* f, int q) {
  if (!f->occ(q)) return 0;
  const int sgn = (f->occupied_before(q) & 1) ? -1 : 1;
  f->set(q, 0);
  return sgn;
}
int create(Fock* f, int q) {
  if (f->occ(q)) return 0;
  const int sgn = (f->occupied_before(q) & 1) ? -1 : 1;
  f->set(q, 1);
  return sgn;
}

// <bra| c+_p c_q |ket> for p != q: the ket must equal bra with mode p emptied and mode q
// filled.  Computes that ket and the matrix element (+1, -1 or 0).
int hop_elem(uint64_t up, uint64_t dn, int n, int p, int q, uint64_t* kup, uint64_t* kdn) {
  Fock bra{up, dn, n};
  if (!bra.occ(p) || bra.occ(q)) return 0;
  Fock ket = bra;
  ket.set(p, 0);
  ket.set(q, 1);
  *kup = ket.up; *kdn = ket.dn;
  Fock f = ket;
  int sgn = annihilate(&f, q);
  sgn *= create(&f, p);
  return sgn;  // f now equals bra
}

// Visits every non-zero element of row r of a Hubbard model as f(col, value).
template <class F>
bool hub_row_elems(const or_model* m, const Basis& B, uint64_t r, F f) {
  uint64_t up, dn;
  B.hub_state(r, &up, &dn);
  const int n = B.n;
  bool ok = true;
  double diag = 0.0;
  for (int k = 0; k < m->n_U; ++k) {
    const int i = m->U_i[k];
    diag += m->U_val[k] * (double)(((up >> i) & 1u) * ((dn >> i) & 1u));
  }
  for (int k = 0; k < m->n_V; ++k) {
    const int i = m->V_ij[2 * k], j = m->V_ij[2 * k + 1];
    const double ni = (double)(((up >> i) & 1u) + ((dn >> i) & 1u));
    const double nj = (double)(((up >> j) & 1u) + ((dn >> j) & 1u));
    diag += m->V_val[k] * ni * nj;
  }
  for (int k = 0; k < m->n_mu; ++k) {
    const int i = m->mu_i[k];
    diag -= m->mu_val[k] * (double)(((up >> i) & 1u) + ((dn >> i) & 1u));
  }
  if (diag != 0.0) f(r, cplx(diag, 0.0));
  for (int k = 0; k < m->n_hop; ++k) {
    const int i = m->hop_ij[2 * k], j = m->hop_ij[2 * k + 1];
    const int off = m->hop_spin[k] ? n : 0;
    const cplx t(m->hop_t[2 * k], m->hop_t[2 * k + 1]);
    // - t c+_i c_j  and  - conj(t) c+_j c_i
    const int pq[2][2] = {{i + off, j + off}, {j + off, i + off}};
    const cplx coef[2] = {-t, -std::conj(t)};
    for (int d = 0; d < 2; ++d) {
      uint64_t kup, kdn;
      const int sgn = hop_elem(up, dn, n, pq[d][0], pq[d][1], &kup, &kdn);
      if (!sgn) continue;
      const uint64_t col = B.hub_index(kup, kdn);
      if (col == UINT64_MAX) { ok = false; continue; }
      f(col, coef[d] * (double)sgn);
    }
  }
  return ok;
}

bool row_times(const or_model* m, const Basis& B, uint64_t r, const cplx* v, int nvec, cplx* out) {
  for (int c = 0; c < nvec; ++c) out[c] = 0.0;
  auto acc = [&](uint64_t col, cplx el) {
    for (int c = 0; c < nvec; ++c) out[c] += el * v[col * nvec + c];
  };
  return B.kind == 0 ? spin_row_elems(m, B, r, acc) : hub_row_elems(m, B, r, acc);
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of two 32x32->64 multiplications on a 4-word counter with a 2-word key
// bumped by the Weyl constants after every round.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c[0];
    const uint64_t p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    const uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// Standard-normal pair of Philox block p of stream `seed` (Box & Muller 1958 on two 53-bit
// uniforms in the open interval (0, 1)).
void gauss_pair(uint64_t seed, uint64_t p, double* g0, double* g1) {
  const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  philox4x32_10(ctr, key, x);
  const uint64_t a = (((uint64_t)x[0] << 32) | x[1]) >> 11;
  const uint64_t b = (((uint64_t)x[2] << 32) | x[3]) >> 11;
  const double ua = ((double)a + 0.5) * (1.0 / 9007199254740992.0);
  const double ub = ((double)b + 0.5) * (1.0 / 9007199254740992.0);
  const double rad = std::sqrt(-2.0 * std::log(ua));
  const double ang = 2.0 * M_PI * ub;
  *g0 = rad * std::cos(ang);
  *g1 = rad * std::sin(ang);
}

// Element e of the start vector of `seed`: complex, g0 + i g1 of block e; real, g0 or g1
// (e even / odd) of block e / 2.
void start_element(uint64_t seed, uint64_t e, bool is_complex, double* re, double* im) {
  double g0, g1;
  if (is_complex) {
    gauss_pair(seed, e, &g0, &g1);
    *re = g0;
    *im = g1;
  } else {
    gauss_pair(seed, e / 2, &g0, &g1);
    *re = (e & 1) ? g1 : g0;
    *im = 0.0;
  }
}

}  // namespace

extern "C" {

// ----------------------------------------------------------------- basis queries
int or_dim(const or_model* m, uint64_t* dim) {
  Basis B;
  if (!B.init(m)) return -1;
  *dim = B.dim;
  return 0;
}

uint64_t or_binom(int n, int k) { return binom(n, k); }

// All n_bits-bit strings with popcount k in ascending order, by plain filtering of
// 0 .. 2^n_bits - 1 (the definition of the restricted space of section 3.1).
int64_t or_sector_list(int n_bits, int k, uint64_t* out, int64_t cap) {
  if (n_bits < 0 || n_bits > 40) return -1;
  int64_t cnt = 0;
  const uint64_t lim = (uint64_t)1 << n_bits;
  for (uint64_t s = 0; s < lim; ++s) {
    if (popcount64(s) == k) {
      if (cnt < cap) out[cnt] = s;
      ++cnt;
    }
  }
  return cnt;
}

uint64_t or_rank(uint64_t s, int n_bits) { return rank_same_popcount(s, n_bits); }
uint64_t or_unrank(uint64_t r, int n_bits, int k) { return unrank_same_popcount(r, n_bits, k); }

// Fermion sign of <bra| c+_p c_q |ket> with mode order (up 0..n-1, down 0..n-1).
int or_hop_sign(uint64_t up, uint64_t dn, int n, int p, int q) {
  uint64_t ku, kd;
  return hop_elem(up, dn, n, p, q, &ku, &kd);
}

// ----------------------------------------------------------------- H v
// w = H v on the whole basis.  v, w: complex128 [dim][nvec].  Returns 0, or -2 if a
// term connects the basis to a configuration outside it, -1 on a bad model.
int or_apply_H(const or_model* m, const double* v_ri, double* w_ri, int nvec) {
  Basis B;
  if (!B.init(m)) return -1;
  const cplx* v = reinterpret_cast<const cplx*>(v_ri);
  cplx* w = reinterpret_cast<cplx*>(w_ri);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : bad)
  for (int64_t r = 0; r < (int64_t)B.dim; ++r) {
    const bool ok = row_times(m, B, (uint64_t)r, v, nvec, w + (uint64_t)r * nvec);
    if (!ok) bad |= 1;
  }
  return bad ? -2 : 0;
}

// Rows [r0, r0 + nrows) of H v only (the vector v is still the whole basis).
int or_apply_H_slice(const or_model* m, const double* v_ri, double* w_ri, int nvec, uint64_t r0, uint64_t nrows) {
  Basis B;
  if (!B.init(m)) return -1;
  if (r0 + nrows > B.dim) return -1;
  const cplx* v = reinterpret_cast<const cplx*>(v_ri);
  cplx* w = reinterpret_cast<cplx*>(w_ri);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
  for (int64_t k = 0; k < (int64_t)nrows; ++k) {
    const uint64_t r = r0 + (uint64_t)k;
    const bool ok = row_times(m, B, r, v, nvec, w + (uint64_t)k * nvec);
    if (!ok) bad |= 1;
  }
  return bad ? -2 : 0;
}

// ----------------------------------------------------------------- Philox start vectors
void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

void or_gauss_pair(uint64_t seed, uint64_t p, double* g) { gauss_pair(seed, p, &g[0], &g[1]); }

// Element values of the Philox start vector at arbitrary indices.  Output complex128 [n].
void or_random_at(uint64_t seed, const uint64_t* idx, int64_t n, int is_complex, double* out_ri) {
  for (int64_t k = 0; k < n; ++k) start_element(seed, idx[k], is_complex != 0, &out_ri[2 * k], &out_ri[2 * k + 1]);
}

// Sampled rows of H v where v is the (unnormalised) Philox start vector of `seed`:
// every element a row needs is regenerated from its index, so the full vector never has
// to exist on the host.  rows: [nrows]; out: complex128 [nrows].
// Vector layout [dim][nvec]: element (row, c) is Philox element row * nvec + c; column c of
// H v is evaluated.
int or_apply_H_rows_philox(const or_model* m, const uint64_t* rows, int64_t nrows, uint64_t seed,
                           int is_complex, int nvec, int c, double* out_ri) {
  Basis B;
  if (!B.init(m)) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t k = 0; k < nrows; ++k) {
    cplx acc = 0.0;
    auto f = [&](uint64_t col, cplx el) {
      double g0, g1;
      start_element(seed, col * (uint64_t)nvec + (uint64_t)c, is_complex != 0, &g0, &g1);
      acc += el * cplx(g0, g1);
    };
    const bool ok = B.kind == 0 ? spin_row_elems(m, B, rows[k], f) : hub_row_elems(m, B, rows[k], f);
    out_ri[2 * k] = acc.real();
    out_ri[2 * k + 1] = acc.imag();
    if (!ok) bad |= 1;
  }
  return bad ? -2 : 0;
}

// ----------------------------------------------------------------- Lanczos (section 3.4)
// v0: complex128 [dim] start vector (normalised here).  Runs at most m steps of
//   alpha_k = (H v_k, v_k),  w = H v_k - beta_k v_{k-1} - alpha_k v_k,
//   beta_{k+1} = |w|,        v_{k+1} = w / |w|,
// with beta_0 = 0 and v_{-1} = 0.  Stops early when beta_{k+1} <= brk * max(1, |alpha_k|)
// (an invariant subspace has been found).  alpha[k] for k < steps, beta[k] = beta_{k+1}.
// Returns the number of steps taken, or a negative error.
int or_lanczos(const or_model* m, const double* v0_ri, int m_steps, double brk, double* alpha, double* beta) {
  Basis B;
  if (!B.init(m)) return -1;
  const uint64_t D = B.dim;
  std::vector<cplx> vprev(D, 0.0), v(D), u(D);
  const cplx* v0 = reinterpret_cast<const cplx*>(v0_ri);
  double nrm = 0.0;
  for (uint64_t r = 0; r < D; ++r) nrm += std::norm(v0[r]);
  nrm = std::sqrt(nrm);
  for (uint64_t r = 0; r < D; ++r) v[r] = v0[r] / nrm;
  double beta_k = 0.0;
  int steps = 0;
  for (int k = 0; k < m_steps; ++k) {
    const int rc = or_apply_H(m, reinterpret_cast<const double*>(v.data()), reinterpret_cast<double*>(u.data()), 1);
    if (rc) return rc;
    cplx a = 0.0;
    for (uint64_t r = 0; r < D; ++r) a += std::conj(v[r]) * u[r];
    const double a_k = a.real();
    double bb = 0.0;
    for (uint64_t r = 0; r < D; ++r) {
      u[r] = u[r] - beta_k * vprev[r] - a_k * v[r];
      bb += std::norm(u[r]);
    }
    const double b_next = std::sqrt(bb);
    alpha[k] = a_k;
    beta[k] = b_next;
    steps = k + 1;
    if (b_next <= brk * std::fmax(1.0, std::fabs(a_k))) break;
    for (uint64_t r = 0; r < D; ++r) {
      vprev[r] = v[r];
      v[r] = u[r] / b_next;
    }
    beta_k = b_next;
  }
  return steps;
}

// Second Lanczos pass (section 3.4: the eigenvector e = V_n e~ is rebuilt by running the
// same recurrence again and accumulating the Lanczos vectors with the Ritz coefficients).
// coef: [steps] real coefficients e~_k.  x_out: complex128 [dim].
int or_lanczos_vector(const or_model* m, const double* v0_ri, int steps, const double* alpha,
                      const double* beta, const double* coef, double* x_ri) {
  Basis B;
  if (!B.init(m)) return -1;
  const uint64_t D = B.dim;
  std::vector<cplx> vprev(D, 0.0), v(D), u(D);
  cplx* x = reinterpret_cast<cplx*>(x_ri);
  const cplx* v0 = reinterpret_cast<const cplx*>(v0_ri);
  double nrm = 0.0;
  for (uint64_t r = 0; r < D; ++r) nrm += std::norm(v0[r]);
  nrm = std::sqrt(nrm);
  for (uint64_t r = 0; r < D; ++r) { v[r] = v0[r] / nrm; x[r] = coef[0] * v[r]; }
  double beta_k = 0.0;
  for (int k = 0; k + 1 < steps; ++k) {
    const int rc = or_apply_H(m, reinterpret_cast<const double*>(v.data()), reinterpret_cast<double*>(u.data()), 1);
    if (rc) return rc;
    for (uint64_t r = 0; r < D; ++r) {
      const cplx wv = u[r] - beta_k * vprev[r] - alpha[k] * v[r];
      vprev[r] = v[r];
      v[r] = wv / beta[k];
      x[r] += coef[k + 1] * v[r];
    }
    beta_k = beta[k];
  }
  return 0;
}

// ----------------------------------------------------------------- mTPQ (section 3.5)
// psi0: complex128 [dim] (normalised here).  For k = 1 .. K:
//   phi = (l - H / Ns) psi_{k-1},  psi_k = phi / |phi|,
// recording, for the state psi_{k-1} that the k-th multiplication acts on,
//   u[k-1]  = <psi|H|psi> / Ns,   h2[k-1] = <psi|H^2|psi> / Ns^2 = |H psi|^2 / Ns^2,
//   nrm[k-1] = |phi|.
// psi_out (optional, complex128 [dim]) receives psi_K.
int or_tpq(const or_model* m, const double* psi0_ri, int K, double l, double Ns, double* u_out,
           double* h2_out, double* nrm_out, double* psi_out_ri) {
  Basis B;
  if (!B.init(m)) return -1;
  const uint64_t D = B.dim;
  std::vector<cplx> psi(D), hp(D);
  const cplx* p0 = reinterpret_cast<const cplx*>(psi0_ri);
  double nrm = 0.0;
  for (uint64_t r = 0; r < D; ++r) nrm += std::norm(p0[r]);
  nrm = std::sqrt(nrm);
  for (uint64_t r = 0; r < D; ++r) psi[r] = p0[r] / nrm;
  for (int k = 1; k <= K; ++k) {
    const int rc = or_apply_H(m, reinterpret_cast<const double*>(psi.data()), reinterpret_cast<double*>(hp.data()), 1);
    if (rc) return rc;
    cplx e = 0.0;
    double h2 = 0.0;
    for (uint64_t r = 0; r < D; ++r) {
      e += std::conj(psi[r]) * hp[r];
      h2 += std::norm(hp[r]);
    }
    double pn = 0.0;
    for (uint64_t r = 0; r < D; ++r) {
      psi[r] = l * psi[r] - hp[r] / Ns;
      pn += std::norm(psi[r]);
    }
    pn = std::sqrt(pn);
    for (uint64_t r = 0; r < D; ++r) psi[r] /= pn;
    u_out[k - 1] = e.real() / Ns;
    h2_out[k - 1] = h2 / (Ns * Ns);
    nrm_out[k - 1] = pn;
  }
  if (psi_out_ri) {
    cplx* po = reinterpret_cast<cplx*>(psi_out_ri);
    for (uint64_t r = 0; r < D; ++r) po[r] = psi[r];
  }
  return 0;
}

}  // extern "C"
