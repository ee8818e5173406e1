// Split-row H v for real spin models in a fixed-S^z sector (section 3.3's on-the-fly
// product over section 3.1's restricted basis), laid out for GB300's memory hierarchy.
//
// A sector configuration is s = (hi << L) | lo.  Ascending order sorts by hi first, so the
// rows of one high part are contiguous: row hi starts at hi_off[hi] and holds the C(L, q)
// low parts of popcount q = n_ones - popcount(hi) in ascending order.  In an S^z sector the
// only off-diagonal terms are exchange flips of two antiparallel spins, so
//   low-low bonds    act inside a row:        (hi, lo)  <- (hi, lo ^ m)
//   high-high bonds  combine whole rows:      row hi    <- row hi ^ m, same column
//   straddling bonds gather from one row:     (hi, lo)  <- (hi ^ 2^a, lo ^ 2^b)
// (section 4.3's point, terms acting on data that is already local, with the row as the
// local unit).  Two passes:
//   pass H  (k_sec_hi)  the high-high row combinations, stripe-major per popcount class so
//           one column stripe of every row of the class is the L2 working set; the plain
//           sums go to W (a scratch vector for Lanczos, else the output buffer itself).
//   pass R  (k_sec_lo)  stages K rows of one class in shared memory, applies the low-low
//           bonds from a per-class neighbour table, gathers the straddling bonds from the
//           partner rows (for one bond the column map lo -> rank(lo ^ 2^b) is increasing,
//           so a warp's gathers stay close together), adds the diagonal from integer bond
//           counts and a small table, adds W and runs the fused Lanczos / mTPQ / refine
//           epilogue.
// fp64 vectors run on the 64-bit fixed-point copy (integer sums, one conversion per
// element); fp32 vectors sum in fp32.
#include <math.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "epilogue.cuh"
#include "reduce.cuh"

namespace hphi {

// ====================================================================== host: analysis
namespace {

struct Bond {
  int i, j;    // i < j
  double c;    // element <s ^ m| H |s> for antiparallel bits i, j
};

struct Analysis {
  bool ok = false;
  std::string why;
  std::vector<Bond> bonds;
  std::vector<double> cls;        // distinct exchange coefficients
  std::vector<int> bond_cls;
  double unit = 0.0;              // fp64: cls[c] = mult[c] * unit
  std::vector<int> mult;
  bool int_ok = false;            // integer multiples found
  int qextra = 0;
  // the diagonal in units of `unit` is an integer everywhere (fp64 pass R then forms the whole
  // element as one exact int64 sum); maxdgi bounds its magnitude
  bool dint = false;
  double maxdgi = 0.0;
  // diagonal = c0 + sum_g gcoef[g] * count_g, count_g over pair bonds (both up) and sites (up)
  double c0 = 0.0;
  int n_dg = 0;
  double gcoef[2] = {0.0, 0.0};
  std::vector<std::pair<int, int>> gpairs[2];  // pair groups
  uint64_t gsites[2] = {0, 0};                 // site groups (linear terms)
  int gmax[2] = {0, 0};
};

uint64_t binom_u(int n, int k) {
  if (k < 0 || k > n || n < 0) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (unsigned)(n - k + i) / (unsigned)i;
  return (uint64_t)r;
}

Analysis analyse(const SecTerms& t) {
  Analysis a;
  const int N = t.n_sites;
  if (N < 2 || N > kSecMaxL + kSecMaxH) {
    a.why = "split-row path: 2..42 sites";
    return a;
  }
  // exchange bonds: each entry flips two sites with a real element, the same both ways
  std::map<std::pair<int, int>, double> bond;
  for (const SpinEntry& e : t.ents) {
    if (e.i == e.j || __builtin_popcountll(e.mask) != 2) {
      a.why = "split-row path: only two-site exchange terms";
      return a;
    }
    const double2 c = t.cls[e.cls];
    if (c.y != 0.0) {
      a.why = "split-row path: real couplings only";
      return a;
    }
    const int code0 = e.phases & 7, code1 = (e.phases >> 3) & 7, code2 = (e.phases >> 6) & 7,
              code3 = (e.phases >> 9) & 7;
    auto val = [&](int code) -> double {
      return code == 1 ? c.x : (code == 3 ? -c.x : 0.0);
    };
    if (code0 || code3 || (code1 != 0 && code1 != 1 && code1 != 3) || (code2 != 0 && code2 != 1 && code2 != 3)) {
      a.why = "split-row path: exchange of antiparallel spins with real elements only";
      return a;
    }
    if (val(code1) != val(code2)) {
      a.why = "split-row path: non-symmetric exchange element";
      return a;
    }
    const int i = std::min<int>(e.i, e.j), j = std::max<int>(e.i, e.j);
    bond[std::make_pair(i, j)] += val(code1);
  }
  for (auto& kv : bond) {
    if (kv.second == 0.0) continue;
    a.bonds.push_back(Bond{kv.first.first, kv.first.second, kv.second});
  }
  for (const Bond& b : a.bonds) {
    int c = -1;
    for (size_t k = 0; k < a.cls.size(); ++k)
      if (a.cls[k] == b.c) c = (int)k;
    if (c < 0) {
      a.cls.push_back(b.c);
      c = (int)a.cls.size() - 1;
    }
    a.bond_cls.push_back(c);
  }
  if ((int)a.cls.size() > kSecMaxCls) {
    a.why = "split-row path: too many distinct exchange couplings";
    return a;
  }
  // fp64: integer multiples of one power of two (a single class is its own unit)
  if (a.cls.size() <= 1) {
    a.unit = a.cls.empty() ? 1.0 : a.cls[0];
    a.mult.assign(a.cls.size(), 1);
    a.int_ok = true;
  } else {
    int g = 1 << 20;
    for (double c : a.cls) {
      int e;
      const double f = frexp(fabs(c), &e);  // c = f 2^e, f in [0.5, 1)
      uint64_t M = (uint64_t)ldexp(f, 53);
      int z = 0;
      while (M && !(M & 1)) { M >>= 1; ++z; }
      g = std::min(g, e - 53 + z);
    }
    a.unit = ldexp(1.0, g);
    a.int_ok = true;
    for (double c : a.cls) {
      const double m = ldexp(c, -g);
      if (fabs(m) > 65536.0 || m != floor(m)) a.int_ok = false;
      a.mult.push_back((int)m);
    }
  }
  long long msum = 0;
  for (size_t k = 0; k < a.bonds.size(); ++k) msum += a.int_ok ? std::abs(a.mult[a.bond_cls[k]]) : 1;
  // integer sums of msum terms of magnitude < 2^(56 - qextra) must stay below 2^63
  while (a.qextra < 40 && (double)msum * ldexp(1.0, 56 - a.qextra) >= ldexp(1.0, 63)) ++a.qextra;
  // diagonal: c0 + linear site groups + pair groups; a linear coefficient common to every site
  // is constant in the sector (it multiplies n_ones)
  a.c0 = t.c0;
  std::vector<double> lin(N, 0.0);
  for (const LinGroup& g : t.lin)
    for (int i = 0; i < N; ++i)
      if ((g.mask >> i) & 1ull) lin[i] += g.coef;
  // the most frequent per-site coefficient l0 is part of the constant (sum_i l0 b_i = l0 n_ones);
  // sites with another coefficient form count groups of lin[i] - l0
  double l0 = lin[0];
  int best = 0;
  for (int i = 0; i < N; ++i) {
    const int c = (int)std::count(lin.begin(), lin.end(), lin[i]);
    if (c > best) {
      best = c;
      l0 = lin[i];
    }
  }
  a.c0 += l0 * t.n_ones;
  int ng = 0;
  std::vector<double> vals;
  for (int i = 0; i < N; ++i)
    if (lin[i] != l0 && std::find(vals.begin(), vals.end(), lin[i]) == vals.end()) vals.push_back(lin[i]);
  for (double v : vals) {
    if (ng >= 2) {
      a.why = "split-row path: the diagonal has more than two coefficient groups";
      return a;
    }
    a.gcoef[ng] = v - l0;
    for (int i = 0; i < N; ++i)
      if (lin[i] == v) a.gsites[ng] |= 1ull << i;
    ++ng;
  }
  for (size_t k = 0; k < t.pcoef.size(); ++k) {
    if (t.pcoef[k] == 0.0) continue;
    if (ng >= 2) {
      a.why = "split-row path: the diagonal has more than two coefficient groups";
      return a;
    }
    a.gcoef[ng] = t.pcoef[k];
    for (const PairEntry& p : t.pairs)
      if (p.grp == (uint16_t)k) a.gpairs[ng].push_back(std::make_pair((int)p.i, (int)p.j));
    ++ng;
  }
  a.n_dg = ng;
  for (int g = 0; g < ng; ++g) {
    a.gmax[g] = (int)a.gpairs[g].size() + __builtin_popcountll(a.gsites[g]);
    if (a.gmax[g] > 255) {
      a.why = "split-row path: more than 255 diagonal terms in one group";
      return a;
    }
  }
  if ((a.gmax[0] + 1) * (a.gmax[1] + 1) > kSecDtab) {
    a.why = "split-row path: diagonal table too large";
    return a;
  }
  if (a.int_ok && a.unit != 0.0) {
    bool all_int = true;
    double mx = 0.0;
    for (int x = 0; x <= a.gmax[0] && all_int; ++x)
      for (int y = 0; y <= a.gmax[1]; ++y) {
        const double v = (a.c0 + a.gcoef[0] * x + a.gcoef[1] * y) / a.unit;
        if (v != floor(v) || fabs(v) > 1048576.0) {
          all_int = false;
          break;
        }
        mx = std::max(mx, fabs(v));
      }
    if (all_int) {
      a.dint = true;
      a.maxdgi = mx;
      // the element d q + S sums msum + maxdgi terms of magnitude < 2^(56 - qextra)
      while (a.qextra < 40 && ((double)msum + mx) * ldexp(1.0, 56 - a.qextra) >= ldexp(1.0, 63)) ++a.qextra;
    }
  }
  a.ok = true;
  return a;
}

constexpr int kTileBudget = 200000;  // shared-memory bytes of one row tile

// longest row of a class present in the sector for low-part length L
uint64_t longest_row(int N, int n_ones, int L) {
  const int H = N - L;
  uint64_t mx = 0;
  for (int p = 0; p <= H; ++p) {
    const int q = n_ones - p;
    if (q < 0 || q > L) continue;
    mx = std::max(mx, binom_u(L, q));
  }
  return mx;
}

bool split_ok(int N, int L) { return L >= 1 && L <= kSecMaxL && N - L >= 1 && N - L <= kSecMaxH; }

}  // namespace

bool sec_applicable(const SecTerms& t, int prec, std::string* why) {
  Analysis a = analyse(t);
  if (!a.ok) {
    if (why) *why = a.why;
    return false;
  }
  if (prec == HPHI_FP64 && !a.int_ok) {
    if (why) *why = "split-row path (fp64): couplings are not small integer multiples of one power of two";
    return false;
  }
  if (sec_default_L(t, prec == HPHI_FP64 ? 8 : 4) == 0) {
    if (why) *why = "split-row path: no split whose rows fit shared memory";
    return false;
  }
  if (why) why->clear();
  return true;
}

int sec_default_L(const SecTerms& t, int esz) {
  const int N = t.n_sites;
  for (int L = std::min(kSecMaxL, N - 1); L >= 1; --L) {
    if (!split_ok(N, L)) continue;
    const uint64_t r = longest_row(N, t.n_ones, L);
    if (r <= 65535 && r * (uint64_t)esz <= (uint64_t)kTileBudget) return L;
  }
  return 0;
}

bool sec_fits(const SecTerms& t, int L, int K, int esz) {
  if (!split_ok(t.n_sites, L) || K < 1) return false;
  const uint64_t r = longest_row(t.n_sites, t.n_ones, L);
  return r >= 1 && r <= 65535 && r * (uint64_t)esz * (uint64_t)K <= (uint64_t)kTileBudget;
}

int sec_default_K(const SecTerms& t, int L, int esz) {
  const uint64_t r = std::max<uint64_t>(1, longest_row(t.n_sites, t.n_ones, L));
  // 8-byte elements stop at 4 rows (8 int64 rows run out of registers)
  const int kmax = esz >= 8 ? 4 : 8;
  int K = 1;
  while (K < kmax && r * esz * (uint64_t)(2 * K) <= (uint64_t)kTileBudget) K *= 2;
  return K;
}

// ====================================================================== device tables
struct SecTables {
  SecDev dev{};
  std::vector<void*> bufs;
};

void sec_free(SecTables* t) {
  if (!t) return;
  for (void* p : t->bufs)
    if (p) cudaFree(p);
  delete t;
}

const SecDev& sec_dev(const SecTables* t) { return t->dev; }

namespace {

template <class X>
Status up(SecTables* T, const std::vector<X>& v, const X** out, cudaStream_t st) {
  void* p = nullptr;
  const size_t b = sizeof(X) * std::max<size_t>(1, v.size());
  cudaError_t e = cudaMalloc(&p, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return {e == cudaErrorMemoryAllocation ? HPHI_ERR_OUT_OF_MEMORY : HPHI_ERR_CUDA,
            std::string("split-row tables: cudaMalloc(") + std::to_string(b) + "): " + cudaGetErrorString(e)};
  }
  T->bufs.push_back(p);
  if (!v.empty()) HPHI_CUDA_TRY(cudaMemcpyAsync(p, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice, st));
  *out = reinterpret_cast<const X*>(p);
  return {};
}

}  // namespace

Status sec_build(const SecTerms& t, int L, int K, SecTables** out, cudaStream_t st) {
  *out = nullptr;
  Analysis a = analyse(t);
  if (!a.ok) return {HPHI_ERR_UNSUPPORTED, a.why};
  const int N = t.n_sites, n1 = t.n_ones;
  if (!split_ok(N, L)) return {HPHI_ERR_INVALID_ARG, "split-row path: low part of 1..20 bits, high part of 1..22"};
  if (K < 1 || K > 8 || (K & (K - 1))) return {HPHI_ERR_INVALID_ARG, "split-row path: tile rows K in {1, 2, 4, 8}"};
  const int H = N - L;
  const uint64_t nqmax = longest_row(N, n1, L);
  if (nqmax == 0) return {HPHI_ERR_INVALID_ARG, "split-row path: empty sector"};
  if (nqmax > 65535) return {HPHI_ERR_UNSUPPORTED, "split-row path: rows longer than 65,535 entries"};
  const uint32_t nL = 1u << L, nH = 1u << H;

  std::unique_ptr<SecTables, SecTablesDeleter> T(new SecTables());
  SecDev& d = T->dev;
  d.L = L;
  d.H = H;
  d.n_ones = n1;
  d.dim = (int64_t)binom_u(N, n1);
  d.K = K;
  d.nq_max = (int)nqmax;
  d.n_cls = (int)a.cls.size();
  d.one_cls = a.cls.size() <= 1 ? 1 : 0;
  for (size_t c = 0; c < a.cls.size(); ++c) {
    d.coef[c] = a.cls[c];
    d.mult[c] = a.int_ok ? a.mult[c] : 0;
  }
  d.unit = a.unit;
  d.qextra = a.qextra;
  d.dint = a.dint ? 1 : 0;

  // low side: popcount-grouped list and ranks
  std::vector<uint32_t> lo_rank(nL), lo_list(nL);
  {
    std::vector<uint32_t> cnt(L + 2, 0);
    for (int q = 0; q <= L; ++q) cnt[q + 1] = cnt[q] + (uint32_t)binom_u(L, q);
    for (int q = 0; q <= L + 1; ++q) d.lo_off[q] = cnt[q];
    std::vector<uint32_t> fill(cnt.begin(), cnt.end() - 1);
    for (uint32_t lo = 0; lo < nL; ++lo) {  // ascending, so each class comes out ascending
      const int q = __builtin_popcount(lo);
      lo_rank[lo] = fill[q] - cnt[q];
      lo_list[fill[q]++] = lo;
    }
  }
  // the low-part tables cover the classes present, q in [n1 - H, n1] within [0, L]
  const int qmin = std::max(0, n1 - H), qmax = std::min(L, n1);
  const uint32_t j0 = d.lo_off[qmin], nJ = d.lo_off[qmax + 1] - j0;
  d.jbase = j0;
  d.nJ = nJ;
  // bonds by group
  std::vector<int> llb, hhb, stb;
  for (size_t k = 0; k < a.bonds.size(); ++k) {
    const Bond& b = a.bonds[k];
    if (b.j < L) llb.push_back((int)k);
    else if (b.i >= L) hhb.push_back((int)k);
    else stb.push_back((int)k);
  }
  if ((int)stb.size() > kSecMaxStr) return {HPHI_ERR_UNSUPPORTED, "split-row path: too many straddling bonds"};
  // low neighbour table, class-sorted per entry
  std::vector<int> ll_sorted = llb;
  std::stable_sort(ll_sorted.begin(), ll_sorted.end(), [&](int x, int y) { return a.bond_cls[x] < a.bond_cls[y]; });
  int lo_slots = 0;
  std::vector<uint8_t> lo_cnt(nJ, 0);
  std::vector<uint16_t> lo_diag(nJ, 0);
  for (uint32_t j = 0; j < nJ; ++j) {
    const uint32_t lo = lo_list[j0 + j];
    int c = 0;
    for (int k : ll_sorted) {
      const Bond& b = a.bonds[k];
      if (((lo >> b.i) ^ (lo >> b.j)) & 1u) ++c;
    }
    if (c > 255) return {HPHI_ERR_UNSUPPORTED, "split-row path: more than 255 low-part neighbours"};
    lo_cnt[j] = (uint8_t)c;
    lo_slots = std::max(lo_slots, c);
  }
  // groups of four slots; slots past an entry's count point at the zero entry (index nq_max)
  const int G = std::max(1, (lo_slots + 3) / 4);
  std::vector<uint16_t> lo_nbr((size_t)G * nJ * 4, (uint16_t)nqmax);
  std::vector<uint8_t> lo_cls(d.one_cls ? 4 : (size_t)G * nJ * 4, 0);
  for (uint32_t j = 0; j < nJ; ++j) {
    const uint32_t lo = lo_list[j0 + j];
    int s = 0;
    for (int k : ll_sorted) {
      const Bond& b = a.bonds[k];
      if (!(((lo >> b.i) ^ (lo >> b.j)) & 1u)) continue;
      const uint32_t lo2 = lo ^ ((1u << b.i) | (1u << b.j));
      const size_t o = ((size_t)(s / 4) * nJ + j) * 4 + (s % 4);
      lo_nbr[o] = (uint16_t)lo_rank[lo2];  // same class: rank < C(L, q) <= 65535
      if (!d.one_cls) lo_cls[o] = (uint8_t)a.bond_cls[k];
      ++s;
    }
  }
  d.lo_groups = G;
  // straddling bonds (a = high site - L, b = low site) and one rank table per distinct low site
  std::vector<int> str_sites;
  d.n_str = (int)stb.size();
  for (int n = 0; n < d.n_str; ++n) {
    const Bond& b = a.bonds[stb[n]];
    d.str_a[n] = (uint8_t)(b.j - L);
    d.str_b[n] = (uint8_t)b.i;
    d.str_cls[n] = (uint8_t)a.bond_cls[stb[n]];
    auto it = std::find(str_sites.begin(), str_sites.end(), b.i);
    if (it == str_sites.end()) {
      str_sites.push_back(b.i);
      it = str_sites.end() - 1;
    }
    d.str_t[n] = (uint8_t)(it - str_sites.begin());
  }
  if ((int)str_sites.size() > kSecMaxStrSites) return {HPHI_ERR_UNSUPPORTED, "split-row path: too many straddling sites"};
  std::vector<uint16_t> str_rank((size_t)std::max<size_t>(1, str_sites.size()) * nJ, 0);
  for (size_t u = 0; u < str_sites.size(); ++u)
    for (uint32_t j = 0; j < nJ; ++j) {
      const uint32_t r = lo_rank[lo_list[j0 + j] ^ (1u << str_sites[u])];
      // ranks in classes that never receive a straddling gather may exceed 16 bits; unused
      str_rank[u * nJ + j] = (uint16_t)(r <= 65535 ? r : 0);
    }
  // diagonal counts: field g of 8 bits
  auto counts = [&](uint64_t s, int side) -> uint16_t {  // side 0: low part only, 1: high part only
    uint32_t packed = 0;
    for (int g = 0; g < a.n_dg; ++g) {
      int c = 0;
      for (const auto& pr : a.gpairs[g]) {
        const bool lo_pair = pr.second < L, hi_pair = pr.first >= L;
        if ((side == 0 && lo_pair) || (side == 1 && hi_pair)) c += (int)((s >> pr.first) & (s >> pr.second) & 1ull);
      }
      const uint64_t sites = a.gsites[g] & (side == 0 ? ((1ull << L) - 1ull) : ~((1ull << L) - 1ull));
      c += __builtin_popcountll(s & sites);
      packed |= (uint32_t)c << (8 * g);
    }
    return (uint16_t)packed;
  };
  for (uint32_t j = 0; j < nJ; ++j) lo_diag[j] = counts(lo_list[j0 + j], 0);
  // straddling S^z S^z pairs in layers: a pair joins the first layer of its group that has
  // no pair on the same low site yet (one low bit counts one pair per layer)
  d.n_sp = 0;
  d.n_sl = 0;
  std::vector<uint32_t> layer_bits;
  for (int g = 0; g < a.n_dg; ++g)
    for (const auto& pr : a.gpairs[g]) {
      if (pr.first < L && pr.second >= L) {
        if (d.n_sp >= kSecMaxSp) return {HPHI_ERR_UNSUPPORTED, "split-row path: too many straddling S^z S^z pairs"};
        const uint32_t bit = 1u << pr.first;
        int l = 0;
        while (l < d.n_sl && (d.sp_lg[l] != g || (layer_bits[l] & bit))) ++l;
        if (l == d.n_sl) {
          if (d.n_sl >= kSecMaxSl) return {HPHI_ERR_UNSUPPORTED, "split-row path: too many straddling pair layers"};
          d.sp_lg[d.n_sl++] = (uint8_t)g;
          layer_bits.push_back(0u);
        }
        layer_bits[l] |= bit;
        d.sp_a[d.n_sp] = (uint8_t)(pr.second - L);
        d.sp_b[d.n_sp] = (uint8_t)pr.first;
        d.sp_l[d.n_sp] = (uint8_t)l;
        ++d.n_sp;
      }
    }
  d.n_dg = a.n_dg;
  d.dstride = a.gmax[0] + 1;
  std::vector<double> dtab((size_t)(a.gmax[0] + 1) * (a.gmax[1] + 1));
  for (int x = 0; x <= a.gmax[0]; ++x)
    for (int y = 0; y <= a.gmax[1]; ++y) dtab[(size_t)x + (size_t)d.dstride * y] = a.c0 + a.gcoef[0] * x + a.gcoef[1] * y;
  d.dtab_n = (int)dtab.size();
  // high side: row offsets, neighbour lists, diagonal counts
  std::vector<uint64_t> hi_off(nH);
  {
    uint64_t run = 0;
    for (uint32_t hi = 0; hi < nH; ++hi) {
      hi_off[hi] = run;
      run += binom_u(L, n1 - __builtin_popcount(hi));
    }
    if (run != (uint64_t)d.dim) return {HPHI_ERR_CUDA, "split-row path: row offsets do not add up to the dimension"};
  }
  std::vector<int> hh_sorted = hhb;
  std::stable_sort(hh_sorted.begin(), hh_sorted.end(), [&](int x, int y) { return a.bond_cls[x] < a.bond_cls[y]; });
  int hi_slots = 0;
  std::vector<uint8_t> hi_cnt(nH, 0);
  std::vector<uint16_t> hi_diag(nH, 0);
  for (uint32_t hi = 0; hi < nH; ++hi) {
    int c = 0;
    for (int k : hh_sorted) {
      const Bond& b = a.bonds[k];
      if (((hi >> (b.i - L)) ^ (hi >> (b.j - L))) & 1u) ++c;
    }
    hi_cnt[hi] = (uint8_t)c;
    hi_slots = std::max(hi_slots, c);
    hi_diag[hi] = counts((uint64_t)hi << L, 1);
  }
  std::vector<uint32_t> hi_nbr((size_t)std::max(1, hi_slots) * nH, 0);
  for (uint32_t hi = 0; hi < nH; ++hi) {
    int s = 0;
    for (int k : hh_sorted) {
      const Bond& b = a.bonds[k];
      if (!(((hi >> (b.i - L)) ^ (hi >> (b.j - L))) & 1u)) continue;
      const uint32_t h2 = hi ^ ((1u << (b.i - L)) | (1u << (b.j - L)));
      hi_nbr[(size_t)s * nH + hi] = h2 | ((uint32_t)a.bond_cls[k] << 24);
      ++s;
    }
  }
  d.hi_slots = hi_slots;
  // classes present, high parts grouped by popcount
  std::vector<uint32_t> hi_cls;
  d.n_pc = 0;
  for (int p = 0; p <= H; ++p) {
    const int q = n1 - p;
    if (q < 0 || q > L) continue;
    d.pc_p[d.n_pc] = p;
    d.pc_row0[d.n_pc] = (uint32_t)hi_cls.size();
    for (uint32_t hi = 0; hi < nH; ++hi)
      if (__builtin_popcount(hi) == p) hi_cls.push_back(hi);
    ++d.n_pc;
  }
  d.pc_row0[d.n_pc] = (uint32_t)hi_cls.size();
  // row-pass tiles.  A row is read three times: staged by its own tile, and gathered by the
  // tiles of its straddling partners hi ^ 2^a (a in S, the high bits of the straddling bonds),
  // which lie one class above or below.  Blocks of high parts that agree outside S are closed
  // under those flips; a block runs class by class, so a row's partners are read while its
  // neighbouring classes run and it stays in L2 between the three reads.  Up to K rows of one
  // class per tile.
  std::vector<uint32_t> hi_seq, tiles;
  {
    uint32_t S = 0;
    for (int n = 0; n < d.n_str; ++n) S |= 1u << d.str_a[n];
    // blocks of at least 2^8 high parts, so that the classes of a block fill tiles of K rows
    for (int b = 0; b < H && __builtin_popcount(S) < std::min(H, 8); ++b) S |= 1u << b;
    const uint32_t nonS = (uint32_t)(nH - 1) & ~S;
    std::vector<uint32_t> sv;  // the 2^|S| settings of the bits of S
    for (uint32_t x = S;; x = (x - 1) & S) {
      sv.push_back(x);
      if (x == 0) break;
    }
    std::sort(sv.begin(), sv.end());
    std::vector<uint32_t> in_cls;
    for (uint32_t o = 0;; o = ((o | S) + 1) & nonS) {  // the settings of the other bits, ascending
      for (int i = 0; i < d.n_pc; ++i) {
        const int p = d.pc_p[i];
        in_cls.clear();
        for (uint32_t x : sv)
          if (__builtin_popcount(o | x) == p) in_cls.push_back(o | x);
        for (size_t r = 0; r < in_cls.size(); r += (size_t)K) {
          const size_t nk = std::min<size_t>((size_t)K, in_cls.size() - r);
          tiles.push_back((uint32_t)hi_seq.size() | ((uint32_t)(nk - 1) << 24));
          hi_seq.insert(hi_seq.end(), in_cls.begin() + (long)r, in_cls.begin() + (long)(r + nk));
        }
      }
      if (o == nonS) break;
    }
  }
  d.n_tiles = (int64_t)tiles.size();

  Status s;
  const std::vector<uint32_t> lo_used(lo_list.begin() + j0, lo_list.begin() + j0 + nJ);
  if ((s = up(T.get(), lo_used, &d.lo_list, st)).code) return s;
  {
    const uint16_t* p16 = nullptr;
    if ((s = up(T.get(), lo_nbr, &p16, st)).code) return s;
    d.lo_nbr4 = reinterpret_cast<const uint2*>(p16);
  }
  if ((s = up(T.get(), lo_cnt, &d.lo_cnt, st)).code) return s;
  {
    const uint8_t* p8 = nullptr;
    if ((s = up(T.get(), lo_cls, &p8, st)).code) return s;
    d.lo_cls4 = reinterpret_cast<const uint32_t*>(p8);
  }
  if ((s = up(T.get(), lo_diag, &d.lo_diag, st)).code) return s;
  if ((s = up(T.get(), hi_off, &d.hi_off, st)).code) return s;
  if ((s = up(T.get(), hi_nbr, &d.hi_nbr, st)).code) return s;
  if ((s = up(T.get(), hi_cnt, &d.hi_cnt, st)).code) return s;
  if ((s = up(T.get(), hi_diag, &d.hi_diag, st)).code) return s;
  if ((s = up(T.get(), str_rank, &d.str_rank, st)).code) return s;
  if ((s = up(T.get(), dtab, &d.dtab, st)).code) return s;
  if ((s = up(T.get(), hi_seq, &d.hi_seq, st)).code) return s;
  if ((s = up(T.get(), tiles, &d.tiles, st)).code) return s;
  if ((s = up(T.get(), hi_cls, &d.hi_cls, st)).code) return s;
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors die here
  *out = T.release();
  return {};
}

// ====================================================================== kernels
namespace {

constexpr int kHiWarps = kThreads / 32;
constexpr int kHiClaim = 4;  // items per warp per counter claim

template <class T> struct SecAcc;
template <> struct SecAcc<float> { using A = float; };
template <> struct SecAcc<long long> { using A = long long; };

// weight of exchange class c: fp32 the coefficient, fixed point the integer multiple
template <class T>
__device__ __forceinline__ T sec_w(const SecDev& d, int c);
template <>
__device__ __forceinline__ float sec_w<float>(const SecDev& d, int c) { return (float)d.coef[c]; }
template <>
__device__ __forceinline__ long long sec_w<long long>(const SecDev& d, int c) { return (long long)d.mult[c]; }

// pass H: W[row hi][col] = sum over active high-high bonds of w X[row hi'][col].  Warp items
// (class, stripe of 32 * EPT columns, row) run class by class and stripe by stripe, claimed in
// order from a counter, so the stripe of all rows of the class stays in L2 while it is used.
template <class T, int EPT, bool ONE>
__global__ void __launch_bounds__(kThreads) k_sec_hi(const SecDev d, const T* __restrict__ X, T* W,
                                                     const int* __restrict__ done,
                                                     unsigned long long* __restrict__ counter) {
  if (done != nullptr && *done) return;
  constexpr int SW = 32 * EPT;
  __shared__ long long s_item0[kSecMaxH + 2];
  __shared__ uint32_t s_nrow[kSecMaxH + 1], s_nq[kSecMaxH + 1], s_nstr[kSecMaxH + 1];
  __shared__ T s_w[kSecMaxCls];
  __shared__ unsigned long long s_claim;
  // per warp: the current batch of neighbour rows (first element, weight), read back as
  // shared-memory broadcasts by every lane
  __shared__ uint64_t s_src[kHiWarps][32];
  __shared__ T s_wt[kHiWarps][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    long long acc = 0;
    for (int i = 0; i < d.n_pc; ++i) {
      const int q = d.n_ones - d.pc_p[i];
      const uint32_t nrow = d.pc_row0[i + 1] - d.pc_row0[i];
      const uint32_t nq = d.lo_off[q + 1] - d.lo_off[q];
      const uint32_t ns = (nq + SW - 1) / SW;
      s_item0[i] = acc;
      s_nrow[i] = nrow;
      s_nq[i] = nq;
      s_nstr[i] = ns;
      acc += (long long)nrow * ns;
    }
    s_item0[d.n_pc] = acc;
  }
  if (tid < kSecMaxCls) s_w[tid] = tid < d.n_cls ? sec_w<T>(d, tid) : (T)0;
  __syncthreads();
  const long long total = s_item0[d.n_pc];
  const size_t nH = (size_t)1 << d.H;
  for (;;) {
    if (tid == 0) s_claim = atomicAdd(counter, (unsigned long long)(kHiWarps * kHiClaim));
    __syncthreads();
    const long long base = (long long)s_claim;
    __syncthreads();
    if (base >= total) break;
    for (int it = 0; it < kHiClaim; ++it) {
      const long long item = base + (long long)it * kHiWarps + warp;  // the CTA's warps on neighbouring rows
      if (item >= total) break;
      int pc = 0;
      while (item >= s_item0[pc + 1]) ++pc;
      const long long k = item - s_item0[pc];
      const uint32_t nrow = s_nrow[pc];
      const uint32_t sidx = (uint32_t)(k / nrow);
      const uint32_t r = (uint32_t)(k - (long long)sidx * nrow);
      const int nq = (int)s_nq[pc];
      const uint32_t hi = __ldg(d.hi_cls + d.pc_row0[pc] + r);
      const uint64_t o = __ldg(d.hi_off + hi);
      const int cnt = __ldg(d.hi_cnt + hi);
      const int col0 = (int)sidx * SW + lane;
      const bool full = (int)sidx * SW + SW <= nq;  // the whole stripe lies inside the row
      T acc[EPT];
#pragma unroll
      for (int j = 0; j < EPT; ++j) acc[j] = (T)0;
      for (int qb = 0; qb < cnt; qb += 32) {
        const int nn = min(32, cnt - qb);
        __syncwarp();  // the previous batch's entries have been read
        if (lane < nn) {
          const uint32_t e = __ldg(d.hi_nbr + (size_t)(qb + lane) * nH + hi);
          s_src[warp][lane] = __ldg(d.hi_off + (e & 0xffffffu));
          if constexpr (!ONE) s_wt[warp][lane] = s_w[e >> 24];
        }
        __syncwarp();
        for (int q0 = 0; q0 < nn; q0 += 4) {
          T x[4][EPT];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const bool on = q0 + t < nn;
            const T* p = X + s_src[warp][(q0 + t) & 31] + col0;
#pragma unroll
            for (int j = 0; j < EPT; ++j) x[t][j] = (on && (full || col0 + j * 32 < nq)) ? __ldg(p + j * 32) : (T)0;
          }
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const T wt = ONE ? (T)1 : ((q0 + t < nn) ? s_wt[warp][(q0 + t) & 31] : (T)0);
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
              if constexpr (ONE) acc[j] += x[t][j];
              else acc[j] += wt * x[t][j];
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        const int col = col0 + j * 32;
        if (col < nq) W[o + col] = acc[j];
      }
    }
  }
}

// a 128-bit integer as the nearest-ish fp64 (two roundings: relative error below 2^-52)
__device__ __forceinline__ double i128_to_double(__int128 v) {
  const long long hi = (long long)(v >> 64);
  const unsigned long long lo = (unsigned long long)v;
  return fma(__ll2double_rn(hi), 18446744073709551616.0, __ull2double_rn(lo));
}

// K consecutive values of an interleaved shared-memory tile with the widest aligned loads
template <class T, int K>
__device__ __forceinline__ void tile_load(const T* p, T* out) {
  if constexpr (sizeof(T) * K == 16 && sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
  } else if constexpr (sizeof(T) * K == 16 && sizeof(T) == 8) {
    const longlong2 t = *reinterpret_cast<const longlong2*>(p);
    out[0] = t.x; out[1] = t.y;
  } else if constexpr (sizeof(T) * K == 8 && sizeof(T) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    out[0] = t.x; out[1] = t.y;
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) out[m] = p[m];
  }
}

// pass R: K rows of one class in shared memory; low-low exchange from the grouped neighbour
// table, straddling exchange gathered from the partner rows, diagonal from packed counts, plus
// the pass-H sums Wh, then the fused epilogue.  X is the input (fp32) or its fixed-point copy.
// Every thread owns E elements of the tile at a time (E * K values); the straddling bonds run
// in an outer loop that is the same for all threads, so each bond's constants (low bit, rank
// table, partner row pointers, activating bit values) are read once per thread and used for
// all its elements, and the loads of the E elements are independent.
template <class T, int K, Epi E, int NT, bool ONE>
__global__ void __launch_bounds__(NT, (NT >= 1024) ? 1 : 2) k_sec_lo(const SecDev d, const T* __restrict__ X,
                                                                    const T* Wh, void* w, FusedArgs fa,
                                                                    const int* __restrict__ Ep,
                                                                    unsigned long long* __restrict__ claim) {
  using R = std::conditional_t<sizeof(T) == 4, float, double>;
  constexpr bool FIX = sizeof(T) == 8;
  constexpr int EL = (K >= 4) ? 1 : 4 / K;  // elements per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  R* s_dtab = reinterpret_cast<R*>(smem_raw + (((size_t)(d.nq_max + 1) * K * sizeof(T) + 15) / 16) * 16);
  int* s_dti = reinterpret_cast<int*>(s_dtab + d.dtab_n);  // fp64 with d.dint: the table in units
  __shared__ uint64_t s_roff[K];
  __shared__ uint32_t s_hrow[K];
  __shared__ uint32_t s_hdiag[K];
  __shared__ uint32_t s_spm[K][kSecMaxSl];
  __shared__ uint2 s_sb[kSecMaxStr];         // low bit | class << 16, offset of the bond's rank table
  __shared__ uint32_t s_need[kSecMaxStr];    // bit m: low-bit value that activates the bond in row m
  __shared__ const T* s_ptr[kSecMaxStr][K];  // partner row of row m through the bond
  __shared__ uint32_t s_hi0;
  __shared__ int s_nk;
  __shared__ unsigned long long s_t;
  __shared__ T s_w[kSecMaxCls];
  __shared__ double s_inv[1];
  __shared__ double s_red[(NT / 32) * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  const uint32_t nJ = d.nJ;
  // fixed point: element = q 2^eoff; a power-of-two unit 2^k folds into the scales (see
  // k_hub_up_q): hv = (dg 2^-k xr + (+-S)) 2^(eoff + k)
  const int eoff = FIX ? (*Ep + d.qextra - 1078) : 0;
  const long long ubits = __double_as_longlong(d.unit);
  const int uexp = (int)((ubits >> 52) & 0x7ff);
  const bool u_p2 = FIX && (ubits & 0xfffffffffffffll) == 0 && uexp > 0 && uexp < 0x7ff;
  const bool u_neg = ubits < 0;
  const int u_l2 = uexp - 1023;
  const int e2 = eoff + u_l2;
  const bool fold = u_p2 && eoff >= -1022 && eoff <= 1023 && e2 >= -1022 && e2 <= 1023 &&
                    (E == Epi::kStore || E == Epi::kLanczos1);
  const double s_eoff = fold ? __longlong_as_double((long long)(eoff + 1023) << 52) : 1.0;
  const double s_e2 = fold ? __longlong_as_double((long long)(e2 + 1023) << 52) : 1.0;
  const double r_k = fold ? __longlong_as_double((long long)(1023 - u_l2) << 52) : 1.0;
  for (int k = tid; k < d.dtab_n; k += NT) s_dtab[k] = (R)(d.dtab[k] * r_k);
  // integral diagonal (in units of `unit`): in the folded fp64 Lanczos step the element is one
  // exact int64 sum d q + (+-S), so its conversion is the only rounding, and <x, H x> adds the
  // exact products q (d q +- S) in 128 bits, moved to fp64 every 64 elements
  const bool dint = FIX && fold && d.dint && E == Epi::kLanczos1;
  if (dint)
    for (int k = tid; k < d.dtab_n; k += NT) s_dti[k] = (int)__double2ll_rn(d.dtab[k] * r_k);
  __int128 ia = 0;
  int ic = 0;
  if (tid < kSecMaxCls) s_w[tid] = tid < d.n_cls ? sec_w<T>(d, tid) : (T)0;
  if (tid < d.n_str)
    s_sb[tid] = make_uint2((uint32_t)d.str_b[tid] | ((uint32_t)d.str_cls[tid] << 16), (uint32_t)d.str_t[tid] * nJ);
  if (tid < K) tile[(size_t)d.nq_max * K + tid] = (T)0;  // the zero entry unused neighbour slots point at
  if constexpr (E == Epi::kTpq) {
    if (tid == 0) s_inv[0] = fa.scal[0];
  }
  EpiScalars es{0.0, 0.0};
  if constexpr (E == Epi::kLanczos1) {
    es.c1 = fa.scal[0];
    es.c2 = fa.scal[1];
  }
  const R coef0 = (R)d.coef[0];
  const int n_str = d.n_str;
  const uint32_t pad2 = (uint32_t)d.nq_max | ((uint32_t)d.nq_max << 16);
  constexpr int NQ = n_red<E>() > 0 ? n_red<E>() : 1;  // reduced quantities of the epilogue
  Red<FIX, NQ> red;
  red.zero();
  int pmx = 0;  // fp64 Lanczos: largest exponent field of the P values written (fa.pexp)

  // tiles are claimed in order from a counter, so the tiles in flight stay a narrow window of
  // the processing order (a fixed stride would let CTAs drift apart over thousands of tiles)
  for (;;) {
    __syncthreads();  // the previous tile's rows are no longer read
    if (tid == 0) s_t = atomicAdd(claim, 1ull);
    __syncthreads();
    const int64_t t = (int64_t)s_t;
    if (t >= d.n_tiles) break;
    if (tid < K) {
      const uint32_t tw = __ldg(d.tiles + t);
      const uint32_t start = tw & 0xffffffu;
      const int nk = (int)(tw >> 24) + 1;
      uint64_t roff = 0;
      uint32_t hd = 0, hi = 0;
      for (int l = 0; l < kSecMaxSl; ++l) s_spm[tid][l] = 0u;
      if (tid < nk) {
        hi = __ldg(d.hi_seq + start + tid);
        if (tid == 0) s_hi0 = hi;
        roff = __ldg(d.hi_off + hi);
        hd = __ldg(d.hi_diag + hi);
        for (int n = 0; n < d.n_sp; ++n)
          if ((hi >> d.sp_a[n]) & 1u) s_spm[tid][d.sp_l[n]] |= 1u << d.sp_b[n];
      }
      if (tid == 0) s_nk = nk;
      s_roff[tid] = roff;
      s_hrow[tid] = hi;
      s_hdiag[tid] = hd;
    }
    __syncthreads();
    const int nk = s_nk;
    // straddling bonds of this tile's rows, one bond per thread (read after the staging barrier)
    if (tid < n_str) {
      const uint32_t a = d.str_a[tid];
      uint32_t need = 0u;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        const uint32_t hi = s_hrow[m];
        // active when bit b of lo differs from bit a of hi
        need |= (1u - ((hi >> a) & 1u)) << m;
        s_ptr[tid][m] = X + (m < nk ? __ldg(d.hi_off + (hi ^ (1u << a))) : 0ull);
      }
      s_need[tid] = need;
    }
    const int q = d.n_ones - __popc(s_hi0);
    const uint32_t loff = d.lo_off[q] - d.jbase;  // the class in the tables of the present classes
    const int nq = (int)(d.lo_off[q + 1] - d.lo_off[q]);
    // stage the rows, tile[u * K + m] = X[row m][u], with kStage elements per thread in flight
    constexpr int kStage = (K >= 8) ? 1 : 8 / K;
    for (int u0 = tid; u0 < nq; u0 += NT * kStage) {
      T tmp[kStage][K];
#pragma unroll
      for (int e = 0; e < kStage; ++e) {
        const int u = u0 + e * NT;
#pragma unroll
        for (int m = 0; m < K; ++m) tmp[e][m] = (u < nq && m < nk) ? __ldg(X + s_roff[m] + u) : (T)0;
      }
#pragma unroll
      for (int e = 0; e < kStage; ++e) {
        const int u = u0 + e * NT;
        if (u < nq) {
#pragma unroll
          for (int m = 0; m < K; ++m) tile[u * K + m] = tmp[e][m];
        }
      }
    }
    __syncthreads();
    const uint32_t kmask = (1u << nk) - 1u;
    for (int u0 = tid; u0 < nq; u0 += NT * EL) {
      uint32_t lo[EL], jj[EL];
      int ng[EL];
      T acc[EL][K];
      int gmax = 0;
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int u = u0 + e * NT;
        const bool ok = u < nq;
        jj[e] = loff + (uint32_t)(ok ? u : 0);
        lo[e] = __ldg(d.lo_list + jj[e]);
        ng[e] = ok ? ((int)__ldg(d.lo_cnt + jj[e]) + 3) >> 2 : 0;
        gmax = max(gmax, ng[e]);
#pragma unroll
        for (int m = 0; m < K; ++m) acc[e][m] = (T)0;
      }
      // Lanczos: ask L2 for this thread's W and P elements now, so the epilogue's loads find
      // them there instead of in DRAM (measured 1 to 3 % faster on the 6x6 sector)
      if constexpr (E == Epi::kLanczos1) {
        const char* pin = reinterpret_cast<const char*>(fa.in ? fa.in : fa.out);
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const int u = u0 + e * NT;
          if (u < nq) {
#pragma unroll
            for (int m = 0; m < K; ++m) {
              if (m < nk) {
                const int64_t idx = (int64_t)s_roff[m] + u;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Wh + idx));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pin + idx * (int64_t)sizeof(T)));
              }
            }
          }
        }
      }
      // low-low exchange: four neighbours per table load, unused slots read the zero entry
      for (int g = 0; g < gmax; ++g) {
        uint2 rec[EL];
        uint32_t cw[EL];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const uint32_t o = (uint32_t)g * nJ + jj[e];  // < 2^28
          rec[e] = g < ng[e] ? __ldg(d.lo_nbr4 + o) : make_uint2(pad2, pad2);
          if constexpr (!ONE) cw[e] = g < ng[e] ? __ldg(d.lo_cls4 + o) : 0u;
        }
#pragma unroll
        for (int e = 0; e < EL; ++e) {
#pragma unroll
          for (int t4 = 0; t4 < 4; ++t4) {
            const uint32_t word = (t4 < 2) ? rec[e].x : rec[e].y;
            const uint32_t nb = (t4 & 1) ? (word >> 16) : (word & 0xffffu);
            T v[K];
            tile_load<T, K>(tile + nb * K, v);
#pragma unroll
            for (int m = 0; m < K; ++m) {
              if constexpr (ONE) acc[e][m] += v[m];
              else acc[e][m] += s_w[(cw[e] >> (8 * t4)) & (kSecMaxCls - 1)] * v[m];
            }
          }
        }
      }
      // straddling exchange, one bond at a time for all elements of the thread
      for (int n = 0; n < n_str; ++n) {
        const uint2 sb = s_sb[n];
        const uint32_t b = sb.x & 31u;
        const uint32_t need = s_need[n];
        const T wn = ONE ? (T)1 : s_w[(sb.x >> 16) & (kSecMaxCls - 1)];
        const T* pm[K];
#pragma unroll
        for (int m = 0; m < K; ++m) pm[m] = s_ptr[n][m];
        uint32_t col[EL], act[EL];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
          const uint32_t lb = (lo[e] >> b) & 1u;
          act[e] = (lb ? need : ~need) & kmask & (ng[e] >= 0 && u0 + e * NT < nq ? 0xffffffffu : 0u);
          col[e] = act[e] ? (uint32_t)__ldg(d.str_rank + sb.y + jj[e]) : 0u;
        }
#pragma unroll
        for (int e = 0; e < EL; ++e)
#pragma unroll
          for (int m = 0; m < K; ++m) {
            const T x = ((act[e] >> m) & 1u) ? __ldg(pm[m] + col[e]) : (T)0;
            if constexpr (ONE) acc[e][m] += x;
            else acc[e][m] += wn * x;
          }
      }
      // diagonal, pass-H sums and the epilogue
#pragma unroll
      for (int e = 0; e < EL; ++e) {
        const int u = u0 + e * NT;
        if (u >= nq) break;
        const uint32_t ld = __ldg(d.lo_diag + jj[e]);
#pragma unroll
        for (int m = 0; m < K; ++m) {
          if (m >= nk) break;
          uint32_t c = ld + s_hdiag[m];
          for (int l = 0; l < d.n_sl; ++l) c += (uint32_t)__popc(lo[e] & s_spm[m][l]) << (8 * d.sp_lg[l]);
          const int ci = (int)(c & 0xffu) + d.dstride * (int)(c >> 8);
          const int64_t idx = (int64_t)s_roff[m] + u;
          const T xq = tile[u * K + m];
          const T wv = Wh[idx];
          const R dg = s_dtab[ci];
          if constexpr (!FIX) {
            const R hv = ONE ? dg * xq + coef0 * (acc[e][m] + wv) : dg * xq + (acc[e][m] + wv);
            epilogue<float, E, NQ>(idx, 0, xq, 0.f, hv, 0.f, reinterpret_cast<float*>(w), fa, es, s_inv, red);
          } else {
            const long long S = acc[e][m] + wv;
            if constexpr (E == Epi::kLanczos1) {
              if (dint) {
                const long long hq = (long long)s_dti[ci] * xq + (u_neg ? -S : S);  // hv = hq 2^e2
                const double hvu = __ll2double_rn(hq);
                double* P = reinterpret_cast<double*>(fa.out);
                const double* Pin = fa.in ? reinterpret_cast<const double*>(fa.in) : P;
                const double pv = fma(es.c1 * s_e2, hvu, -(es.c2 * Pin[idx]));
                P[idx] = pv;
                pmx = max(pmx, (int)((__double_as_longlong(pv) >> 52) & 0x7ff));
                ia += (__int128)xq * (__int128)hq;
                if (++ic == 64) {
                  red.add(0, i128_to_double(ia), 1.0);
                  ia = 0;
                  ic = 0;
                }
                continue;
              }
            }
            const double xr = __ll2double_rn(xq);
            if (fold) {
              const double hvu = fma(dg, xr, __ll2double_rn(u_neg ? -S : S));  // hv = hvu 2^e2
              if constexpr (E == Epi::kStore) {
                reinterpret_cast<double*>(w)[idx] = hvu * s_e2;
              } else if constexpr (E == Epi::kLanczos1) {
                double* P = reinterpret_cast<double*>(fa.out);
                const double* Pin = fa.in ? reinterpret_cast<const double*>(fa.in) : P;
                const double pv = fma(es.c1 * s_e2, hvu, -(es.c2 * Pin[idx]));
                P[idx] = pv;
                pmx = max(pmx, (int)((__double_as_longlong(pv) >> 52) & 0x7ff));
                red.add(0, xr, hvu);
                red.tick();
              }
            } else {
              const double x = fix_to_double(xq, eoff);
              const double hv = fma((double)dg, x, d.unit * fix_to_double(S, eoff));
              if constexpr (E == Epi::kLanczos1) {  // the epilogue's Lanczos step, with the exponent kept
                double* P = reinterpret_cast<double*>(fa.out);
                const double* Pin = fa.in ? reinterpret_cast<const double*>(fa.in) : P;
                const double pv = es.c1 * hv - es.c2 * Pin[idx];
                P[idx] = pv;
                pmx = max(pmx, (int)((__double_as_longlong(pv) >> 52) & 0x7ff));
                red.add(0, x, hv);
                red.tick();
              } else {
                epilogue<double, E, NQ>(idx, 0, x, 0.0, hv, 0.0, reinterpret_cast<double*>(w), fa, es, s_inv, red);
              }
            }
          }
        }
      }
    }
  }
  if constexpr (FIX && E == Epi::kLanczos1) {
    if (ic) red.add(0, i128_to_double(ia), 1.0);
    if (fa.pexp != nullptr) {
      pmx = (int)__reduce_max_sync(0xffffffffu, (unsigned)pmx);
      if ((tid & 31) == 0 && pmx > 0) atomicMax(fa.pexp, pmx);
    }
  }
  if constexpr (E != Epi::kStore) {
    constexpr int nq = n_red<E>();
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int qq = 0; qq < nq; ++qq) {
      double x = red.get(qq);
      if (fold) x = (x * s_eoff) * s_e2;  // back from units of 2^(eoff + e2)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) s_red[wid * kMaxRedQ + qq] = x;
    }
    __syncthreads();
    if (tid < nq) {
      double x = 0.0;
      for (int k = 0; k < NT / 32; ++k) x += s_red[k * kMaxRedQ + tid];
      fa.partials[(size_t)blockIdx.x * kMaxRedQ + tid] = x;
    }
  }
}

// ---------------------------------------------------------------- launch helpers
size_t lo_smem(const SecDev& d, int esz) {  // the rows, their zero entry, the diagonal table(s)
  return (((size_t)(d.nq_max + 1) * d.K * esz + 15) / 16) * 16 + (size_t)d.dtab_n * esz +
         (esz == 8 && d.dint ? (size_t)d.dtab_n * 4 : 0);
}

// row-pass threads: 1024 (one CTA per SM) for tiles above ~110 KB, else 512
int lo_threads(const SecDev& d, int esz) { return lo_smem(d, esz) > 110000 ? 1024 : 512; }

template <class KernelT>
int occupancy_of(KernelT kern, int nt, size_t smem) {
  int n = 0;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, nt, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

template <class T, int K, Epi E, bool ONE>
Status launch_lo_t(const SecDev& d, const T* X, const T* Wh, void* w, const FusedArgs& fa, const int* Ep, int grid,
                   unsigned long long* claim, cudaStream_t st) {
  const size_t smem = lo_smem(d, (int)sizeof(T));
  HPHI_CUDA_TRY(cudaMemsetAsync(claim, 0, sizeof(unsigned long long), st));
#define HPHI_SECLO(NN)                                                                                        \
  HPHI_CUDA_TRY(cudaFuncSetAttribute(k_sec_lo<T, K, E, NN, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)smem));                                                             \
  k_sec_lo<T, K, E, NN, ONE><<<grid, NN, smem, st>>>(d, X, Wh, w, fa, Ep, claim);
  if (lo_threads(d, (int)sizeof(T)) == 1024) {
    HPHI_SECLO(1024)
  } else {
    HPHI_SECLO(512)
  }
#undef HPHI_SECLO
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

template <class T, int K, Epi E, bool ONE>
int lo_occupancy_t(const SecDev& d) {
  const size_t smem = lo_smem(d, (int)sizeof(T));
  return lo_threads(d, (int)sizeof(T)) == 1024 ? occupancy_of(k_sec_lo<T, K, E, 1024, ONE>, 1024, smem)
                                               : occupancy_of(k_sec_lo<T, K, E, 512, ONE>, 512, smem);
}

template <class T, Epi E>
Status launch_lo_k(const SecDev& d, const T* X, const T* Wh, void* w, const FusedArgs& fa, const int* Ep, int grid,
                   unsigned long long* claim, cudaStream_t st) {
  const bool one = d.one_cls != 0;
#define HPHI_SECK(KK)                                                                 \
  return one ? launch_lo_t<T, KK, E, true>(d, X, Wh, w, fa, Ep, grid, claim, st)      \
             : launch_lo_t<T, KK, E, false>(d, X, Wh, w, fa, Ep, grid, claim, st);
  switch (d.K) {
    case 8: HPHI_SECK(8)
    case 4: HPHI_SECK(4)
    case 2: HPHI_SECK(2)
    default: HPHI_SECK(1)
  }
#undef HPHI_SECK
}

template <class T, Epi E>
int lo_occupancy_k(const SecDev& d) {
  const bool one = d.one_cls != 0;
  switch (d.K) {
    case 8: return one ? lo_occupancy_t<T, 8, E, true>(d) : lo_occupancy_t<T, 8, E, false>(d);
    case 4: return one ? lo_occupancy_t<T, 4, E, true>(d) : lo_occupancy_t<T, 4, E, false>(d);
    case 2: return one ? lo_occupancy_t<T, 2, E, true>(d) : lo_occupancy_t<T, 2, E, false>(d);
    default: return one ? lo_occupancy_t<T, 1, E, true>(d) : lo_occupancy_t<T, 1, E, false>(d);
  }
}

template <class T>
Status launch_hi(const SecDev& d, const T* X, T* W, const int* done, unsigned long long* counter, cudaStream_t st) {
  HPHI_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  const int grid = num_sms() * 8;
  const bool one = d.one_cls != 0;
  // 1 KB row stripes per warp item (4 int64 / 8 fp32 columns per lane).  The kernel is bound by
  // instruction issue (64-bit adds, addresses, neighbour lists), so wider stripes spread each
  // neighbour's overhead over more columns: on the 6x6 sector 256-byte stripes measured 185 ms,
  // 512-byte 124 ms, and 1 KB about 2.5 % less again, although one stripe of the largest class
  // (360 MB) then far exceeds L2.
  // The autotuner may halve them (d.hi_cols): on the 6x6 sector a 1 KB stripe of the largest
  // class is 360 MB, so the partner reads partly come from DRAM.
  constexpr int EPT = sizeof(T) == 8 ? 4 : 8;
  if (d.hi_cols == EPT / 2) {
    if (one) k_sec_hi<T, EPT / 2, true><<<grid, kThreads, 0, st>>>(d, X, W, done, counter);
    else k_sec_hi<T, EPT / 2, false><<<grid, kThreads, 0, st>>>(d, X, W, done, counter);
  } else {
    if (one) k_sec_hi<T, EPT, true><<<grid, kThreads, 0, st>>>(d, X, W, done, counter);
    else k_sec_hi<T, EPT, false><<<grid, kThreads, 0, st>>>(d, X, W, done, counter);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

// scratch layout: fp64 [Q: dim int64][W: dim int64, Lanczos only][tail]; fp32 [W: dim float,
// Lanczos only][tail]; tail = 256 bytes: exponent (int) at 0 (and the QSlots ints at 4, 8,
// 192), pass-H counter (u64) at 64, pass-R tile counter (u64) at 128
size_t vec_bytes(const SecDev& d, int esz) { return (((size_t)d.dim * esz + 255) / 256) * 256; }

}  // namespace

size_t sec_scratch_bytes(const SecDev& d, int prec, Epi epi) {
  const int esz = prec == HPHI_FP64 ? 8 : 4;
  size_t b = 256;
  if (prec == HPHI_FP64) b += vec_bytes(d, 8);
  if (epi == Epi::kLanczos1) b += vec_bytes(d, esz);
  return b;
}

int* sec_exponent_slot(const SecDev& d, int prec, Epi epi, void* scratch) {
  return reinterpret_cast<int*>(static_cast<char*>(scratch) + sec_scratch_bytes(d, prec, epi) - 256);
}

// fp64: Q at the start of the scratch; tail ints: exponent of Q at 0, the exact exponents of
// the current / next vector at 4 and 8, the pass-1 exponent at 192
QSlots sec_qslots(const SecDev& d, int prec, Epi epi, void* scratch) {
  QSlots q;
  if (prec != HPHI_FP64 || scratch == nullptr) return q;
  char* tail = static_cast<char*>(scratch) + sec_scratch_bytes(d, prec, epi) - 256;
  q.Q = reinterpret_cast<long long*>(scratch);
  q.eq = reinterpret_cast<int*>(tail);
  q.ec[0] = reinterpret_cast<int*>(tail + 4);
  q.ec[1] = reinterpret_cast<int*>(tail + 8);
  q.ep = reinterpret_cast<int*>(tail + 192);
  q.extra = d.qextra;
  return q;
}

int sec_grid(const SecDev& d, int prec, Epi epi) {
  int occ = 1;
#define HPHI_SECOCC(TT)                                                      \
  switch (epi) {                                                             \
    case Epi::kStore: occ = lo_occupancy_k<TT, Epi::kStore>(d); break;       \
    case Epi::kLanczos1: occ = lo_occupancy_k<TT, Epi::kLanczos1>(d); break; \
    case Epi::kTpq: occ = lo_occupancy_k<TT, Epi::kTpq>(d); break;           \
    case Epi::kRefine: occ = lo_occupancy_k<TT, Epi::kRefine>(d); break;     \
  }
  if (prec == HPHI_FP64) { HPHI_SECOCC(long long) } else { HPHI_SECOCC(float) }
#undef HPHI_SECOCC
  return (int)std::max<int64_t>(1, std::min<int64_t>(d.n_tiles, (int64_t)num_sms() * occ));
}

Status launch_sec(const SecDev& d, int prec, const void* v, void* w, void* scratch, Epi epi, const FusedArgs& fa,
                  int grid, cudaStream_t st) {
  if (epi == Epi::kRefine && prec != HPHI_FP64) return {HPHI_ERR_INVALID_ARG, "refinement runs in fp64"};
  char* sc = static_cast<char*>(scratch);
  char* tail = sc + sec_scratch_bytes(d, prec, epi) - 256;
  int* Ep = reinterpret_cast<int*>(tail);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(tail + 64);
  unsigned long long* claim = reinterpret_cast<unsigned long long*>(tail + 128);
  // the output buffer receives the pass-H sums and is finished in place, except in Lanczos
  // steps, whose output (P) is also an input: their sums go to the scratch vector
  void* out = (epi == Epi::kStore) ? w : fa.out;
  if (prec == HPHI_FP64) {
    long long* Q = reinterpret_cast<long long*>(sc);
    long long* W = (epi == Epi::kLanczos1) ? reinterpret_cast<long long*>(sc + vec_bytes(d, 8))
                                           : reinterpret_cast<long long*>(out);
    Status s;
    if (fa.exp_ready != 2) {  // 2: the previous Lanczos pass 2 wrote Q and its exponent
      s = launch_quant_vec(reinterpret_cast<const double*>(v), Q, d.dim, Ep, fa.done, fa.exp_ready != 0, d.qextra, st);
      if (s.code) return s;
    }
    if (fa.pexp != nullptr) HPHI_CUDA_TRY(cudaMemsetAsync(fa.pexp, 0, sizeof(int), st));
    if ((s = launch_hi<long long>(d, Q, W, fa.done, counter, st)).code) return s;
    switch (epi) {
      case Epi::kStore: return launch_lo_k<long long, Epi::kStore>(d, Q, W, w, fa, Ep, grid, claim, st);
      case Epi::kLanczos1: return launch_lo_k<long long, Epi::kLanczos1>(d, Q, W, w, fa, Ep, grid, claim, st);
      case Epi::kTpq: return launch_lo_k<long long, Epi::kTpq>(d, Q, W, w, fa, Ep, grid, claim, st);
      case Epi::kRefine: return launch_lo_k<long long, Epi::kRefine>(d, Q, W, w, fa, Ep, grid, claim, st);
    }
  } else {
    const float* X = reinterpret_cast<const float*>(v);
    float* W = (epi == Epi::kLanczos1) ? reinterpret_cast<float*>(sc) : reinterpret_cast<float*>(out);
    Status s = launch_hi<float>(d, X, W, fa.done, counter, st);
    if (s.code) return s;
    switch (epi) {
      case Epi::kStore: return launch_lo_k<float, Epi::kStore>(d, X, W, w, fa, Ep, grid, claim, st);
      case Epi::kLanczos1: return launch_lo_k<float, Epi::kLanczos1>(d, X, W, w, fa, Ep, grid, claim, st);
      case Epi::kTpq: return launch_lo_k<float, Epi::kTpq>(d, X, W, w, fa, Ep, grid, claim, st);
      case Epi::kRefine: break;
    }
  }
  return {HPHI_ERR_INVALID_ARG, "split-row path: unsupported precision / epilogue"};
}

}  // namespace hphi
