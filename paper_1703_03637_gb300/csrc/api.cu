// C ABI of the library: model definition, term compilation (section 3.3), sector build
// (section 3.1) and the Lanczos (section 3.4) / mTPQ (section 3.5) drivers.  Host code
// only arranges work; every step of the method runs in the kernels of k_*.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <complex>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

using cplx = std::complex<double>;

namespace {

struct Coupling { int i, j; double J[9]; };
struct Field { int i; double h[3]; };
struct Hop { int i, j, spin; double tr, ti; };
struct Onsite { int i; double U; };
struct Density { int i, j; double V; };
struct Chem { int i; double mu; };

// device buffer owned by the model
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  hphi::Status ensure(size_t b) {
    if (b <= bytes && p) return {};
    release();
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return {e == cudaErrorMemoryAllocation ? HPHI_ERR_OUT_OF_MEMORY : HPHI_ERR_CUDA,
              std::string("cudaMalloc(") + std::to_string(b) + " bytes): " + cudaGetErrorString(e)};
    }
    bytes = b;
    return {};
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

template <class T>
hphi::Status upload(DBuf& b, const std::vector<T>& v, cudaStream_t st) {
  hphi::Status s = b.ensure(sizeof(T) * std::max<size_t>(v.size(), 1));
  if (s.code) return s;
  if (!v.empty()) HPHI_CUDA_TRY(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return {};
}

uint64_t binom_host(int n, int k) {
  if (k < 0 || k > n || n < 0) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (unsigned)(n - k + i) / (unsigned)i;
  return (uint64_t)r;
}

// canonical class coefficient: rotate by a power of i into {re > 0, im >= 0}; returns the
// phase code p with el = coef * i^(p-1)  (1: +1, 2: +i, 3: -1, 4: -i)
int canon(cplx el, cplx* coef) {
  cplx c = el;
  for (int k = 0; k < 4; ++k) {
    if (c.real() > 0 && c.imag() >= 0) {
      *coef = c;
      return k + 1;
    }
    c = c * cplx(0, -1);  // el = c * i^k
  }
  *coef = el;
  return 1;
}

// spin single-site element <b|S^a|b'>, b' the only ket bit with a non-zero value
cplx site_el(int a, int b, int* kb) {
  if (a == 2) { *kb = b; return cplx(b ? 0.5 : -0.5, 0); }
  *kb = 1 - b;
  if (a == 0) return cplx(0.5, 0);
  return b ? cplx(0, -0.5) : cplx(0, 0.5);
}

struct Workspace {
  DBuf vecA, vecB, x, partials, scal, work, basis;
  DBuf cgp, cgq;  // inverse iteration: CG direction and A p
};

}  // namespace

struct hphi_model {
  int kind = 0, n_sites = 0;
  int basis = HPHI_BASIS_FULL, a = 0, b = 0;
  std::vector<Coupling> coup;
  std::vector<Field> field;
  std::vector<Hop> hop;
  std::vector<Onsite> onsite;
  std::vector<Density> dens;
  std::vector<Chem> chem;
  bool built = false;
  bool cplx_model = false;
  int64_t dim = 0;
  std::string err;
  int device = 0;
  // device data
  DBuf d_entries, d_cls, d_lin, d_pairs, d_pcoef, d_hi_off, d_lo_rank, d_lo_list, d_lo_off;
  DBuf d_nbr_up, d_deg_up, d_nbr_dn, d_deg_dn, d_npos_up, d_npos_dn, d_counter;
  hphi::SpinDev sdev{};
  hphi::HubDev hdev{};
  Workspace ws;
  // sector sub-models of hphi_lanczos_run_sectors, rebuilt when the terms change
  uint64_t gen = 0, sub_gen = ~0ull;
  std::map<int, std::unique_ptr<hphi_model>> sub;
  // window passes of the batched-row kernel: the compiled entries, the size setting
  // (-1 off, 0 sized from L2, else the window's sites) and the plans built so far by size
  std::vector<hphi::SpinEntry> host_entries;
  int win_bits_opt = -1;
  struct WinCache {
    DBuf ents, dep;
    hphi::BatchPlan plan;
  };
  std::map<int, std::unique_ptr<WinCache>> win;
  // split-row path of real S^z-sector spin models: the compiled terms, whether each precision
  // may take the path, the split asked for per precision (-1 off, 0 default, else L) and
  // rows per tile (0 default), and the device tables built so far by (L, K)
  hphi::SecTerms sec_terms;
  bool sec_ok[2] = {false, false};
  std::string sec_why;
  int sec_L[2] = {0, 0}, sec_K[2] = {0, 0};
  int sec_hi_cols[2] = {0, 0};  // pass H columns per lane per precision (0: built-in)
  std::map<std::pair<int, int>, std::unique_ptr<hphi::SecTables, hphi::SecTablesDeleter>> sec_tab;
};

namespace {

std::mutex g_err_mu;
std::string g_err;

int fail(hphi_model* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_err = msg;
  }
  return code;
}

int fail(hphi_model* m, const hphi::Status& s) { return fail(m, s.code, s.msg); }

// ------------------------------------------------------------------ spin term compiler
struct ClassTable {
  std::vector<cplx> coefs;
  int get(cplx c) {
    for (size_t k = 0; k < coefs.size(); ++k)
      if (coefs[k] == c) return (int)k;
    coefs.push_back(c);
    return (int)coefs.size() - 1;
  }
};

hphi::Status compile_spin(hphi_model* m, cudaStream_t st) {
  const int N = m->n_sites;
  const bool sector = (m->basis == HPHI_BASIS_SZ);
  // diagonal decomposition: c0 + sum_i lin_i b_i + sum_pairs quad b_i b_j
  double c0 = 0.0;
  std::vector<double> lin(N, 0.0);
  std::map<std::pair<int, int>, double> quad;
  struct Pat { uint64_t mask; int i, j; cplx el[4]; };  // el indexed by b_i + 2 b_j
  std::vector<Pat> pats;
  bool cplx_model = false;

  // merge couplings on the same (unordered) pair
  std::map<std::pair<int, int>, std::array<std::array<cplx, 4>, 4>> bond_el;  // [pattern fi+2fj][b_i+2b_j]
  for (const Coupling& c : m->coup) {
    const int i = c.i, j = c.j;
    auto key = std::make_pair(i, j);
    auto& E = bond_el[key];
    for (int bi = 0; bi < 2; ++bi)
      for (int bj = 0; bj < 2; ++bj)
        for (int x = 0; x < 3; ++x)
          for (int y = 0; y < 3; ++y) {
            const double J = c.J[3 * x + y];
            if (J == 0.0) continue;
            int ki, kj;
            const cplx ei = site_el(x, bi, &ki), ej = site_el(y, bj, &kj);
            const int pat = (ki ^ bi) + 2 * (kj ^ bj);
            E[pat][bi + 2 * bj] += J * ei * ej;
          }
  }
  for (auto& kv : bond_el) {
    const int i = kv.first.first, j = kv.first.second;
    auto& E = kv.second;
    // diagonal pattern
    const double d00 = E[0][0].real(), d10 = E[0][1].real(), d01 = E[0][2].real(), d11 = E[0][3].real();
    c0 += d00;
    lin[i] += d10 - d00;
    lin[j] += d01 - d00;
    const double q = d11 - d10 - d01 + d00;
    if (q != 0.0) quad[std::make_pair(std::min(i, j), std::max(i, j))] += q;
    for (int pat = 1; pat < 4; ++pat) {
      Pat p{};
      p.mask = ((pat & 1) ? (1ull << i) : 0ull) | ((pat & 2) ? (1ull << j) : 0ull);
      p.i = i;
      p.j = j;
      bool any = false;
      for (int s = 0; s < 4; ++s) {
        p.el[s] = E[pat][s];
        if (p.el[s] != cplx(0, 0)) {
          any = true;
          if (p.el[s].imag() != 0.0) cplx_model = true;
          if (sector) {
            const int bi = s & 1, bj = s >> 1;
            const int dpop = ((pat & 1) ? (bi ? -1 : 1) : 0) + ((pat & 2) ? (bj ? -1 : 1) : 0);
            if (dpop != 0)
              return {HPHI_ERR_BASIS_MISMATCH, "coupling (" + std::to_string(i) + "," + std::to_string(j) +
                                                   ") does not conserve S^z, which the Sz basis requires"};
          }
        }
      }
      if (any) pats.push_back(p);
    }
  }
  // fields: merge per site
  std::map<int, std::array<std::array<cplx, 2>, 2>> site_el_m;  // [flip][b_i]
  for (const Field& f : m->field) {
    auto& E = site_el_m[f.i];
    for (int bi = 0; bi < 2; ++bi)
      for (int x = 0; x < 3; ++x) {
        if (f.h[x] == 0.0) continue;
        int ki;
        const cplx e = site_el(x, bi, &ki);
        E[ki ^ bi][bi] += -f.h[x] * e;
      }
  }
  for (auto& kv : site_el_m) {
    const int i = kv.first;
    auto& E = kv.second;
    c0 += E[0][0].real();
    lin[i] += E[0][1].real() - E[0][0].real();
    Pat p{};
    p.mask = 1ull << i;
    p.i = i;
    p.j = i;
    bool any = false;
    for (int s = 0; s < 4; ++s) {
      const int bi = s & 1;
      // a one-site pattern reads only b_i; index b_i + 2 b_i takes values 0 and 3
      p.el[s] = (s == 0 || s == 3) ? E[1][bi] : cplx(0, 0);
      if (p.el[s] != cplx(0, 0)) {
        any = true;
        if (p.el[s].imag() != 0.0) cplx_model = true;
        if (sector)
          return {HPHI_ERR_BASIS_MISMATCH,
                  "a transverse field on site " + std::to_string(i) + " does not conserve S^z, which the Sz basis requires"};
      }
    }
    if (any) pats.push_back(p);
  }
  // classes
  ClassTable ct;
  std::vector<hphi::SpinEntry> ents;
  for (const Pat& p : pats) {
    // split the four elements by class
    std::map<int, uint16_t> by_cls;
    for (int s = 0; s < 4; ++s) {
      if (p.el[s] == cplx(0, 0)) continue;
      cplx coef;
      const int code = canon(p.el[s], &coef);
      const int cls = ct.get(coef);
      by_cls[cls] |= (uint16_t)(code << (3 * s));
    }
    for (auto& kv : by_cls) {
      hphi::SpinEntry e{};
      e.mask = p.mask;
      e.i = (uint8_t)p.i;
      e.j = (uint8_t)p.j;
      e.phases = kv.second;
      e.cls = (uint16_t)kv.first;
      ents.push_back(e);
    }
  }
  if ((int)ct.coefs.size() > hphi::kMaxClasses) return {HPHI_ERR_UNSUPPORTED, "too many distinct coupling values"};
  if ((int)ents.size() > hphi::kMaxSpinEntries) return {HPHI_ERR_UNSUPPORTED, "too many off-diagonal terms"};
  std::stable_sort(ents.begin(), ents.end(), [](const hphi::SpinEntry& x, const hphi::SpinEntry& y) { return x.cls < y.cls; });
  int max_run = 0;
  for (size_t k = 0, run = 0; k < ents.size(); ++k) {
    run = (k > 0 && ents[k].cls == ents[k - 1].cls) ? run + 1 : 1;
    max_run = std::max(max_run, (int)run);
  }
  std::vector<double2> cls;
  for (const cplx& c : ct.coefs) cls.push_back(make_double2(c.real(), c.imag()));
  // linear groups by value
  std::vector<hphi::LinGroup> lg;
  for (int i = 0; i < N; ++i) {
    if (lin[i] == 0.0) continue;
    bool found = false;
    for (auto& g : lg)
      if (g.coef == lin[i]) { g.mask |= 1ull << i; found = true; break; }
    if (!found) lg.push_back(hphi::LinGroup{1ull << i, lin[i]});
  }
  if ((int)lg.size() > hphi::kMaxLin) return {HPHI_ERR_UNSUPPORTED, "too many distinct field values"};
  // pair groups by value
  std::vector<double> pc;
  std::vector<hphi::PairEntry> pe;
  for (auto& kv : quad) {
    if (kv.second == 0.0) continue;
    int g = -1;
    for (size_t k = 0; k < pc.size(); ++k)
      if (pc[k] == kv.second) g = (int)k;
    if (g < 0) { pc.push_back(kv.second); g = (int)pc.size() - 1; }
    pe.push_back(hphi::PairEntry{(uint8_t)kv.first.first, (uint8_t)kv.first.second, (uint16_t)g});
  }
  if ((int)pc.size() > hphi::kMaxPairGroups || (int)pe.size() > hphi::kMaxPairs)
    return {HPHI_ERR_UNSUPPORTED, "too many distinct S^z S^z couplings"};
  std::stable_sort(pe.begin(), pe.end(), [](const hphi::PairEntry& x, const hphi::PairEntry& y) { return x.grp < y.grp; });

  hphi::Status s;
  if ((s = upload(m->d_entries, ents, st)).code) return s;
  if ((s = upload(m->d_cls, cls, st)).code) return s;
  if ((s = upload(m->d_lin, lg, st)).code) return s;
  if ((s = upload(m->d_pairs, pe, st)).code) return s;
  if ((s = upload(m->d_pcoef, pc, st)).code) return s;
  hphi::SpinDev& d = m->sdev;
  d = hphi::SpinDev{};
  d.n_sites = N;
  d.sector = sector ? 1 : 0;
  d.n_entries = (int)ents.size();
  d.max_run = max_run;
  m->host_entries = ents;
  m->win.clear();
  d.n_classes = (int)cls.size();
  d.n_lin = (int)lg.size();
  d.n_pairs = (int)pe.size();
  d.n_pair_groups = (int)pc.size();
  d.c0 = c0;
  d.entries = m->d_entries.as<hphi::SpinEntry>();
  d.cls_coef = m->d_cls.as<double2>();
  d.lin = m->d_lin.as<hphi::LinGroup>();
  d.pairs = m->d_pairs.as<hphi::PairEntry>();
  d.pair_coef = m->d_pcoef.as<double>();
  m->cplx_model = cplx_model;
  m->sec_terms = hphi::SecTerms{};
  m->sec_tab.clear();
  m->sec_ok[0] = m->sec_ok[1] = false;
  if (sector && !cplx_model) {
    hphi::SecTerms& t = m->sec_terms;
    t.n_sites = N;
    t.n_ones = m->a;
    t.ents = ents;
    t.cls = cls;
    t.c0 = c0;
    t.lin = lg;
    t.pairs = pe;
    t.pcoef = pc;
  }
  return {};
}

// ------------------------------------------------------------------ Hubbard term compiler
hphi::Status compile_hub(hphi_model* m, cudaStream_t st) {
  const int N = m->n_sites;
  ClassTable ct;
  std::vector<hphi::HopEntry> hops[2];
  bool cplx_model = false;
  for (const Hop& h : m->hop) {
    const cplx t(h.tr, h.ti);
    if (h.ti != 0.0) cplx_model = true;
    hphi::HopEntry e{};
    e.i = (uint8_t)h.i;
    e.j = (uint8_t)h.j;
    e.mask = (1u << h.i) | (1u << h.j);
    const int lo = std::min(h.i, h.j), hi = std::max(h.i, h.j);
    e.between = (hi - lo > 1) ? (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u)) : 0u;
    e.cls = (uint16_t)ct.get(-t);
    hops[h.spin ? 1 : 0].push_back(e);
  }
  for (int s = 0; s < 2; ++s)
    std::stable_sort(hops[s].begin(), hops[s].end(), [](const hphi::HopEntry& x, const hphi::HopEntry& y) { return x.cls < y.cls; });
  std::vector<hphi::HopEntry> all = hops[0];
  all.insert(all.end(), hops[1].begin(), hops[1].end());
  if ((int)all.size() > hphi::kMaxHops) return {HPHI_ERR_UNSUPPORTED, "too many hopping terms"};
  if ((int)ct.coefs.size() > hphi::kMaxClasses) return {HPHI_ERR_UNSUPPORTED, "too many distinct hopping values"};
  // diagonal groups
  std::vector<double> Usite(N, 0.0), musite(N, 0.0);
  for (const Onsite& o : m->onsite) Usite[o.i] += o.U;
  for (const Chem& c : m->chem) musite[c.i] += -c.mu;
  std::vector<hphi::LinGroup> ul, ml;
  for (int i = 0; i < N; ++i) {
    if (Usite[i] != 0.0) {
      bool f = false;
      for (auto& g : ul) if (g.coef == Usite[i]) { g.mask |= 1ull << i; f = true; break; }
      if (!f) ul.push_back(hphi::LinGroup{1ull << i, Usite[i]});
    }
    if (musite[i] != 0.0) {
      bool f = false;
      for (auto& g : ml) if (g.coef == musite[i]) { g.mask |= 1ull << i; f = true; break; }
      if (!f) ml.push_back(hphi::LinGroup{1ull << i, musite[i]});
    }
  }
  std::map<std::pair<int, int>, double> vp;
  for (const Density& d : m->dens) vp[std::make_pair(std::min(d.i, d.j), std::max(d.i, d.j))] += d.V;
  std::vector<double> pc;
  std::vector<hphi::PairEntry> pe;
  for (auto& kv : vp) {
    if (kv.second == 0.0) continue;
    int g = -1;
    for (size_t k = 0; k < pc.size(); ++k) if (pc[k] == kv.second) g = (int)k;
    if (g < 0) { pc.push_back(kv.second); g = (int)pc.size() - 1; }
    pe.push_back(hphi::PairEntry{(uint8_t)kv.first.first, (uint8_t)kv.first.second, (uint16_t)g});
  }
  if ((int)ul.size() > hphi::kMaxLin || (int)ml.size() > hphi::kMaxLin || (int)pc.size() > hphi::kMaxPairGroups ||
      (int)pe.size() > hphi::kMaxPairs)
    return {HPHI_ERR_UNSUPPORTED, "too many distinct diagonal terms"};
  std::stable_sort(pe.begin(), pe.end(), [](const hphi::PairEntry& x, const hphi::PairEntry& y) { return x.grp < y.grp; });
  std::vector<double2> cls;
  for (const cplx& c : ct.coefs) cls.push_back(make_double2(c.real(), c.imag()));
  std::vector<hphi::LinGroup> lin_all = ul;
  lin_all.insert(lin_all.end(), ml.begin(), ml.end());
  hphi::Status s;
  if ((s = upload(m->d_entries, all, st)).code) return s;
  if ((s = upload(m->d_cls, cls, st)).code) return s;
  if ((s = upload(m->d_lin, lin_all, st)).code) return s;
  if ((s = upload(m->d_pairs, pe, st)).code) return s;
  if ((s = upload(m->d_pcoef, pc, st)).code) return s;
  hphi::HubDev& d = m->hdev;
  d = hphi::HubDev{};
  d.n_sites = N;
  d.n_up_hops = (int)hops[0].size();
  d.n_dn_hops = (int)hops[1].size();
  d.n_classes = (int)cls.size();
  d.n_ulin = (int)ul.size();
  d.n_mulin = (int)ml.size();
  d.n_pairs = (int)pe.size();
  d.n_pair_groups = (int)pc.size();
  d.c0 = 0.0;
  d.hops = m->d_entries.as<hphi::HopEntry>();
  d.cls_coef = m->d_cls.as<double2>();
  d.ulin = m->d_lin.as<hphi::LinGroup>();
  d.mulin = m->d_lin.as<hphi::LinGroup>() + ul.size();
  d.pairs = m->d_pairs.as<hphi::PairEntry>();
  d.pair_coef = m->d_pcoef.as<double>();
  m->cplx_model = cplx_model;
  return {};
}

// popcount-class tables over L bits: lo_rank, lo_list, lo_list_off
hphi::Status build_lo_tables(hphi_model* m, int L, cudaStream_t st) {
  std::vector<uint32_t> off(L + 2, 0);
  for (int p = 0; p <= L; ++p) off[p + 1] = off[p] + (uint32_t)binom_host(L, p);
  hphi::Status s;
  if ((s = upload(m->d_lo_off, off, st)).code) return s;
  if ((s = m->d_lo_rank.ensure(sizeof(uint32_t) << L)).code) return s;
  if ((s = m->d_lo_list.ensure(sizeof(uint32_t) << L)).code) return s;
  return hphi::build_popcount_tables(L, m->d_lo_rank.as<uint32_t>(), m->d_lo_list.as<uint32_t>(),
                                     m->d_lo_off.as<uint32_t>(), st);
}

// Two-pass Hubbard path: real model with one hopping value per species.  Builds the
// per-species neighbour tables on the device.
hphi::Status build_hub_fast(hphi_model* m, cudaStream_t st) {
  hphi::HubDev& d = m->hdev;
  d.fast = 0;
  if (m->cplx_model) return {};
  int cls[2] = {-1, -1};
  int cnt[2] = {0, 0};
  for (int sp = 0; sp < 2; ++sp) {
    for (const Hop& h : m->hop) {
      if ((h.spin ? 1 : 0) != sp) continue;
      ++cnt[sp];
    }
  }
  if (cnt[0] > 255 || cnt[1] > 255) return {};
  std::vector<hphi::HopEntry> host(cnt[0] + cnt[1]);
  if (!host.empty())
    HPHI_CUDA_TRY(cudaMemcpyAsync(host.data(), d.hops, sizeof(hphi::HopEntry) * host.size(), cudaMemcpyDeviceToHost, st));
  std::vector<double2> cc(std::max(1, d.n_classes));
  HPHI_CUDA_TRY(cudaMemcpyAsync(cc.data(), d.cls_coef, sizeof(double2) * cc.size(), cudaMemcpyDeviceToHost, st));
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < (int)host.size(); ++k) {
    const int sp = k < cnt[0] ? 0 : 1;
    if (cls[sp] < 0) cls[sp] = host[k].cls;
    else if (cls[sp] != host[k].cls) return {};  // several hopping values: generic path
  }
  const size_t tab = (size_t)4 * (d.dim_up * std::max(1, cnt[0]) + d.dim_dn * std::max(1, cnt[1]));
  if (tab > ((size_t)1 << 30)) return {};
  hphi::Status s;
  d.maxdeg_up = std::max(1, cnt[0]);
  d.maxdeg_dn = std::max(1, cnt[1]);
  d.c_up = cls[0] >= 0 ? cc[cls[0]].x : 0.0;
  d.c_dn = cls[1] >= 0 ? cc[cls[1]].x : 0.0;
  if ((s = m->d_nbr_up.ensure((size_t)4 * d.dim_up * d.maxdeg_up)).code) return s;
  if ((s = m->d_deg_up.ensure((size_t)d.dim_up)).code) return s;
  if ((s = m->d_nbr_dn.ensure((size_t)4 * d.dim_dn * d.maxdeg_dn)).code) return s;
  if ((s = m->d_deg_dn.ensure((size_t)d.dim_dn)).code) return s;
  if ((s = m->d_npos_up.ensure((size_t)d.dim_up)).code) return s;
  if ((s = m->d_npos_dn.ensure((size_t)d.dim_dn)).code) return s;
  d.nbr_up = m->d_nbr_up.as<uint32_t>();
  d.deg_up = m->d_deg_up.as<uint8_t>();
  d.npos_up = m->d_npos_up.as<uint8_t>();
  d.nbr_dn = m->d_nbr_dn.as<uint32_t>();
  d.deg_dn = m->d_deg_dn.as<uint8_t>();
  d.npos_dn = m->d_npos_dn.as<uint8_t>();
  if ((s = hphi::build_hub_neighbours(d, 0, m->d_nbr_up.as<uint32_t>(), m->d_deg_up.as<uint8_t>(),
                                      m->d_npos_up.as<uint8_t>(), st)).code)
    return s;
  if ((s = hphi::build_hub_neighbours(d, 1, m->d_nbr_dn.as<uint32_t>(), m->d_deg_dn.as<uint8_t>(),
                                      m->d_npos_dn.as<uint8_t>(), st)).code)
    return s;
  d.fast = 1;
  return {};
}

// ------------------------------------------------------------------ split-row spin path
// The split (L, K) precision prec runs with: the one asked for, else the default (largest
// low part whose rows fit one tile, widest tile that fits); (0, 0) when the path is off.
std::pair<int, int> sec_shape(const hphi_model* m, int prec) {
  const int pi = prec == HPHI_FP64 ? 0 : 1;
  if (!m->sec_ok[pi] || m->sec_L[pi] < 0) return {0, 0};
  const int esz = prec == HPHI_FP64 ? 8 : 4;
  const int L = m->sec_L[pi] > 0 ? m->sec_L[pi] : hphi::sec_default_L(m->sec_terms, esz);
  if (L <= 0) return {0, 0};
  const int K = m->sec_K[pi] > 0 ? m->sec_K[pi] : hphi::sec_default_K(m->sec_terms, L, esz);
  return {L, K};
}

// Builds (once) the tables of the shape prec runs with.  Never called inside a stream capture.
hphi::Status sec_ensure(hphi_model* m, int prec, cudaStream_t st) {
  const std::pair<int, int> sh = sec_shape(m, prec);
  if (sh.first == 0 || m->sec_tab.count(sh)) return {};
  hphi::SecTables* t = nullptr;
  hphi::Status s = hphi::sec_build(m->sec_terms, sh.first, sh.second, &t, st);
  if (s.code) return s;
  m->sec_tab[sh].reset(t);
  return {};
}

// Tables of the shape prec runs with, or null (path off, not applicable, or not built).
const hphi::SecDev* sec_find(hphi_model* m, int prec) {
  auto it = m->sec_tab.find(sec_shape(m, prec));
  return it == m->sec_tab.end() ? nullptr : &hphi::sec_dev(it->second.get());
}

hphi::Status sec_prepare(hphi_model* m, cudaStream_t st) {
  m->sec_why.clear();
  if (m->basis != HPHI_BASIS_SZ || m->cplx_model) {
    m->sec_why = "split-row path: real models in an S^z sector only";
    return {};
  }
  for (int prec : {HPHI_FP64, HPHI_FP32}) {
    std::string why;
    m->sec_ok[prec == HPHI_FP64 ? 0 : 1] = hphi::sec_applicable(m->sec_terms, prec, &why);
    if (!why.empty()) m->sec_why = why;
    hphi::Status s = sec_ensure(m, prec, st);
    if (s.code) return s;
  }
  return {};
}

hphi::Status build_sector_impl(hphi_model* m, cudaStream_t st) {
  HPHI_CUDA_TRY(cudaGetDevice(&m->device));
  hphi::Status s;
  if ((s = m->d_counter.ensure(256)).code) return s;
  const int N = m->n_sites;
  if (m->kind == HPHI_SPIN_HALF) {
    if ((s = compile_spin(m, st)).code) return s;
    hphi::SpinDev& d = m->sdev;
    if (m->basis == HPHI_BASIS_FULL) {
      if (N > 34) return {HPHI_ERR_UNSUPPORTED, "full spin basis limited to 34 sites"};
      d.dim = (int64_t)1 << N;
    } else {
      if (N > 40) return {HPHI_ERR_UNSUPPORTED, "Sz sectors limited to 40 sites"};
      const int L = (N + 1) / 2, H = N - L;
      if ((s = build_lo_tables(m, L, st)).code) return s;
      if ((s = m->d_hi_off.ensure(sizeof(uint64_t) << H)).code) return s;
      if ((s = hphi::build_hi_offsets(L, H, m->a, m->d_hi_off.as<uint64_t>(), st)).code) return s;
      d.t.L = L;
      d.t.H = H;
      d.t.n_ones = m->a;
      d.t.hi_off = m->d_hi_off.as<uint64_t>();
      d.t.lo_rank = m->d_lo_rank.as<uint32_t>();
      d.t.lo_list = m->d_lo_list.as<uint32_t>();
      d.t.lo_list_off = m->d_lo_off.as<uint32_t>();
      d.dim = (int64_t)binom_host(N, m->a);
    }
    d.counter = m->d_counter.as<unsigned long long>();
    m->dim = d.dim;
    if ((s = sec_prepare(m, st)).code) return s;
  } else {
    if ((s = compile_hub(m, st)).code) return s;
    hphi::HubDev& d = m->hdev;
    if (m->basis == HPHI_BASIS_FULL) {
      if (2 * N > 34) return {HPHI_ERR_UNSUPPORTED, "full Hubbard basis limited to 17 sites"};
      d.sector = 0;
      d.dim_up = d.dim_dn = (int64_t)1 << N;
    } else {
      if ((s = build_lo_tables(m, N, st)).code) return s;
      std::vector<uint32_t> off(N + 2, 0);
      for (int p = 0; p <= N; ++p) off[p + 1] = off[p] + (uint32_t)binom_host(N, p);
      d.sector = 1;
      d.n_up = m->a;
      d.n_dn = m->b;
      d.dim_up = (int64_t)binom_host(N, m->a);
      d.dim_dn = (int64_t)binom_host(N, m->b);
      d.rank = m->d_lo_rank.as<uint32_t>();
      d.list_up = m->d_lo_list.as<uint32_t>() + off[m->a];
      d.list_dn = m->d_lo_list.as<uint32_t>() + off[m->b];
    }
    d.dim = d.dim_up * d.dim_dn;
    d.counter = m->d_counter.as<unsigned long long>();
    m->dim = d.dim;
    if ((s = build_hub_fast(m, st)).code) return s;
  }
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));
  return {};
}

int check_built(hphi_model* m) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (!m->built) return fail(m, HPHI_ERR_NOT_BUILT, "hphi_build_sector has not run since the model last changed");
  return HPHI_OK;
}

const void* dev_model(hphi_model* m) {
  return m->kind == HPHI_HUBBARD ? static_cast<const void*>(&m->hdev) : static_cast<const void*>(&m->sdev);
}

int launch_grid(int64_t work) {
  const int64_t cap = (int64_t)hphi::hv_grid(1);
  int64_t g = (work + hphi::kThreads - 1) / hphi::kThreads;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

// Grid of an H v launch: every resident CTA slot of the kernel instance, clamped to the
// number of work items (Hubbard: (down row, chunk) items; spin: kThreads-element chunks).
bool use_hub_fast(hphi_model* m, int prec, int nvec, hphi::Epi epi) {
  return m->kind == HPHI_HUBBARD && hphi::hub_fast_ok(m->hdev, prec, m->cplx_model, nvec, epi);
}

bool use_batch(hphi_model* m, int nvec) { return m->kind == HPHI_SPIN_HALF && hphi::batch_applies(m->sdev, nvec); }

// Split-row tables when the split-row path applies to this launch (one real vector of an
// S^z-sector spin model), else null.  The path also needs its scratch (sec_scratch_bytes).
const hphi::SecDev* use_sec(hphi_model* m, int prec, int nvec, hphi::Epi epi) {
  if (m->kind != HPHI_SPIN_HALF || nvec != 1 || m->cplx_model) return nullptr;
  if (epi == hphi::Epi::kRefine && prec != HPHI_FP64) return nullptr;
  return sec_find(m, prec);
}

// Window plan of the batched-row kernel for nvec vectors in precision prec, or null for one
// pass in natural row order (windows off, one window holds every term, or no plan found).
// Built on first use for each window size and kept until the terms change.
const hphi::BatchPlan* batch_plan(hphi_model* m, int prec, int nvec) {
  if (!use_batch(m, nvec) || m->win_bits_opt < 0) return nullptr;
  const int wbits = m->win_bits_opt > 0 ? m->win_bits_opt : hphi::batch_window_bits(prec, m->cplx_model, nvec);
  if (wbits >= m->n_sites) return nullptr;
  auto it = m->win.find(wbits);
  if (it == m->win.end()) {
    std::unique_ptr<hphi_model::WinCache> wc(new (std::nothrow) hphi_model::WinCache());
    std::vector<hphi::SpinEntry> ordered;
    std::vector<uint32_t> dep;
    int off[hphi::kMaxPasses + 1] = {};
    int np = 0, max_run = 0;
    if (!wc || !hphi::batch_plan_windows(m->n_sites, wbits, m->host_entries, &ordered, &dep, off, &np, &max_run) ||
        upload(wc->ents, ordered, nullptr).code || upload(wc->dep, dep, nullptr).code ||
        cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      wc.reset();
    } else {
      wc->plan.n_pass = np;
      wc->plan.ents = wc->ents.as<hphi::SpinEntry>();
      wc->plan.dep = wc->dep.as<uint32_t>();
      for (int k = 0; k <= np; ++k) wc->plan.ent_off[k] = off[k];
      wc->plan.max_run = max_run;
    }
    it = m->win.emplace(wbits, std::move(wc)).first;
  }
  return it->second ? &it->second->plan : nullptr;
}

// kernels one hv_launch runs (for the launch counts the results report)
int hv_kernels(hphi_model* m, int prec, int nvec, hphi::Epi epi) {
  if (use_hub_fast(m, prec, nvec, epi)) return prec == HPHI_FP64 ? 4 : 2;  // (max-exponent, quantise,) D, U
  if (use_sec(m, prec, nvec, epi) && m->ws.work.p != nullptr &&
      m->ws.work.bytes >= hphi::sec_scratch_bytes(*use_sec(m, prec, nvec, epi), prec, epi))
    return prec == HPHI_FP64 ? 4 : 2;  // (max-exponent, quantise,) pass H, pass R
  if (use_batch(m, nvec)) {
    const hphi::BatchPlan* plan = epi == hphi::Epi::kLanczos1 ? nullptr : batch_plan(m, prec, nvec);
    const int passes = plan ? plan->n_pass : 1;
    return passes + (hphi::batch_scratch_bytes(m->sdev, plan, prec, m->cplx_model, nvec) ? 2 : 0);
  }
  if (m->kind == HPHI_SPIN_HALF) {
    // the quantised copy (max-exponent and quantise kernels) when the workspace holds it
    const size_t q = hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, nvec);
    return 1 + ((q != 0 && m->ws.work.p != nullptr && m->ws.work.bytes >= q) ? 2 : 0);
  }
  return 1;
}

// scratch an H v launch needs beyond its vectors (0: none)
size_t hv_scratch_bytes(hphi_model* m, int prec, int nvec, hphi::Epi epi) {
  if (use_hub_fast(m, prec, nvec, epi)) return hphi::hub_scratch_bytes(m->hdev, prec, epi);
  if (const hphi::SecDev* sd = use_sec(m, prec, nvec, epi)) return hphi::sec_scratch_bytes(*sd, prec, epi);
  if (use_batch(m, nvec))
    return hphi::batch_scratch_bytes(m->sdev, epi == hphi::Epi::kLanczos1 ? nullptr : batch_plan(m, prec, nvec), prec,
                                     m->cplx_model, nvec);
  if (m->kind == HPHI_SPIN_HALF) return hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, nvec);
  return 0;
}

// Scratch that only speeds a launch up (the quantised copy of the generic spin path): the
// workspace buffer if it can hold `need` bytes, else null (the launch then runs without it).
void* optional_scratch(hphi_model* m, size_t need) {
  if (need == 0) return nullptr;
  if (m->ws.work.ensure(need).code) {
    cudaGetLastError();
    return nullptr;
  }
  return m->ws.work.p;
}

// true when the split-row kernels run this launch: they apply and `scratch_bytes` of scratch
// (the workspace buffer) hold what they need
bool sec_runs(hphi_model* m, int prec, int nvec, hphi::Epi epi, size_t scratch_bytes) {
  const hphi::SecDev* sd = use_sec(m, prec, nvec, epi);
  return sd != nullptr && scratch_bytes >= hphi::sec_scratch_bytes(*sd, prec, epi);
}

int hv_grid_for(hphi_model* m, int nvec, int prec, hphi::Epi epi) {
  if (use_hub_fast(m, prec, nvec, epi)) return hphi::hub_up_grid(m->hdev, prec, epi);
  if (const hphi::SecDev* sd = use_sec(m, prec, nvec, epi)) {
    if (m->ws.work.p != nullptr && m->ws.work.bytes >= hphi::sec_scratch_bytes(*sd, prec, epi))
      return hphi::sec_grid(*sd, prec, epi);
  }
  if (use_batch(m, nvec)) return hphi::batch_grid(prec, m->cplx_model, nvec, epi, m->dim);
  const bool hub = m->kind == HPHI_HUBBARD;
  const int64_t cap = hphi::hv_resident_grid(hub, prec, m->cplx_model, epi);
  int64_t work;
  if (hub) work = ((m->hdev.dim_up * nvec + hphi::kThreads - 1) / hphi::kThreads) * m->hdev.dim_dn;
  else work = (m->dim * nvec + hphi::kThreads - 1) / hphi::kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(work, cap));
}

// One H v (or fused step) launch: the two-pass Hubbard kernels when they apply (they need
// a scratch vector for the fused steps), the batched-row kernel for many aligned vectors of
// a full-basis spin model (fp64 needs scratch), else the generic gather kernel.  Every
// kernel loops over its rows with any grid, so the grid of hv_grid_for suits each of them.
hphi::Status hv_launch(hphi_model* m, int prec, const void* v, void* w, int nvec, hphi::Epi epi,
                       const hphi::FusedArgs& fa, int grid, void* scratch, cudaStream_t st) {
  if (use_hub_fast(m, prec, nvec, epi) && (hphi::hub_scratch_bytes(m->hdev, prec, epi) == 0 || scratch != nullptr))
    return hphi::launch_hub_fast(m->hdev, prec, v, w, scratch, epi, fa, grid, st);
  if (scratch != nullptr && scratch == m->ws.work.p && sec_runs(m, prec, nvec, epi, m->ws.work.bytes)) {
    hphi::SecDev dd = *use_sec(m, prec, nvec, epi);
    dd.hi_cols = m->sec_hi_cols[prec == HPHI_FP64 ? 0 : 1];
    return hphi::launch_sec(dd, prec, v, w, scratch, epi, fa, grid, st);
  }
  if (use_batch(m, nvec) && hphi::batch_aligned(v, w)) {
    const hphi::BatchPlan* plan = epi == hphi::Epi::kLanczos1 ? nullptr : batch_plan(m, prec, nvec);
    if (scratch != nullptr || hphi::batch_scratch_bytes(m->sdev, plan, prec, m->cplx_model, nvec) == 0)
      return hphi::launch_batch(m->sdev, plan, prec, m->cplx_model, v, w, scratch, nvec, epi, fa, grid, st);
  }
  // spin models: scratch, when given, is at least spin_scratch_bytes (the caller sized it
  // with hv_scratch_bytes, whose batched-row figure has the same quantised-copy layout)
  void* sp = (m->kind == HPHI_SPIN_HALF && scratch != nullptr &&
              hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, nvec) != 0 &&
              m->ws.work.bytes >= hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, nvec) &&
              scratch == m->ws.work.p)
                 ? scratch
                 : nullptr;
  return hphi::launch_hv(m->kind == HPHI_HUBBARD, dev_model(m), prec, m->cplx_model, v, w, nvec, epi, fa, grid, sp,
                         st);
}

// Times one plain H v of the split-row path for every candidate split (L, K) -- the default
// low part and one or two bits fewer, each with every tile height that fits -- and keeps the
// fastest for precision prec.  Tables of the losing candidates are freed.
hphi::Status sec_autotune(hphi_model* m, int prec, hphi_tune_result* res, cudaStream_t st) {
  const int pi = prec == HPHI_FP64 ? 0 : 1;
  const int esz = prec == HPHI_FP64 ? 8 : 4;
  const int saved_L = m->sec_L[pi], saved_K = m->sec_K[pi];
  const int L0 = hphi::sec_default_L(m->sec_terms, esz);
  if (L0 <= 0) return {};
  std::vector<std::pair<int, int>> cand;
  for (int L = L0; L >= std::max(1, L0 - 2); --L) {
    if (m->n_sites - L > hphi::kSecMaxH) break;
    const int kmax = hphi::sec_default_K(m->sec_terms, L, esz);
    for (int K = 1; K <= kmax; K *= 2) cand.emplace_back(L, K);
  }
  hphi::Status s;
  if ((s = m->ws.vecA.ensure((size_t)esz * (size_t)m->dim)).code) return s;
  if ((s = m->ws.vecB.ensure((size_t)esz * (size_t)m->dim)).code) return s;
  if ((s = hphi::launch_random(m->ws.vecA.p, m->dim, false, prec == HPHI_FP64, 7, st)).code) return s;
  struct Ev {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Ev() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } tm;
  HPHI_CUDA_TRY(cudaEventCreate(&tm.a));
  HPHI_CUDA_TRY(cudaEventCreate(&tm.b));
  const std::pair<int, int> dflt = sec_shape(m, prec);
  m->sec_hi_cols[pi] = 0;  // the shapes are compared at the built-in pass-H columns
  float best = 1e30f, worst = 0.f, dms = 0.f;
  std::pair<int, int> best_sh = dflt;
  hphi::FusedArgs fa;
  for (const auto& sh : cand) {
    m->sec_L[pi] = sh.first;
    m->sec_K[pi] = sh.second;
    if ((s = sec_ensure(m, prec, st)).code) {
      if (s.code != HPHI_ERR_OUT_OF_MEMORY) break;
      s = {};
      continue;  // a candidate whose tables do not fit is skipped
    }
    const size_t need = hv_scratch_bytes(m, prec, 1, hphi::Epi::kStore);
    if ((s = m->ws.work.ensure(need)).code) break;
    const int grid = hv_grid_for(m, 1, prec, hphi::Epi::kStore);
    s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, m->ws.work.p, st);
    if (s.code) break;
    HPHI_CUDA_TRY(cudaEventRecord(tm.a, st));
    for (int rep = 0; rep < 2 && !s.code; ++rep)
      s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, m->ws.work.p, st);
    HPHI_CUDA_TRY(cudaEventRecord(tm.b, st));
    if (s.code) break;
    HPHI_CUDA_TRY(cudaEventSynchronize(tm.b));
    float ms = 0.f;
    HPHI_CUDA_TRY(cudaEventElapsedTime(&ms, tm.a, tm.b));
    ms /= 2.f;
    ++res->n_candidates;
    if (sh == dflt) dms = ms;
    worst = std::max(worst, ms);
    if (ms < best) {
      best = ms;
      best_sh = sh;
    }
    // keep only the tables of this precision's default and best so far, and of the shape the
    // other precision runs with
    const std::pair<int, int> other = sec_shape(m, pi == 0 ? HPHI_FP32 : HPHI_FP64);
    for (auto it = m->sec_tab.begin(); it != m->sec_tab.end();) {
      if (it->first != dflt && it->first != best_sh && it->first != other) it = m->sec_tab.erase(it);
      else ++it;
    }
  }
  if (s.code) {
    m->sec_L[pi] = saved_L;
    m->sec_K[pi] = saved_K;
    return s;
  }
  m->sec_L[pi] = best_sh.first;
  m->sec_K[pi] = best_sh.second;
  // pass H at half the columns per lane on the chosen shape (narrower stripes keep a large
  // class's stripe nearer L2's size, at more instructions per output)
  {
    const int full = prec == HPHI_FP64 ? 4 : 8;
    const int saved_cols = m->sec_hi_cols[pi];
    float ms_half = 1e30f;
    if ((s = sec_ensure(m, prec, st)).code == 0 &&
        (s = m->ws.work.ensure(hv_scratch_bytes(m, prec, 1, hphi::Epi::kStore))).code == 0) {
      const int grid = hv_grid_for(m, 1, prec, hphi::Epi::kStore);
      m->sec_hi_cols[pi] = full / 2;
      s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, m->ws.work.p, st);
      if (!s.code) HPHI_CUDA_TRY(cudaEventRecord(tm.a, st));
      for (int rep = 0; rep < 2 && !s.code; ++rep)
        s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, m->ws.work.p, st);
      if (!s.code) {
        HPHI_CUDA_TRY(cudaEventRecord(tm.b, st));
        HPHI_CUDA_TRY(cudaEventSynchronize(tm.b));
        HPHI_CUDA_TRY(cudaEventElapsedTime(&ms_half, tm.a, tm.b));
        ms_half /= 2.f;
        ++res->n_candidates;
        worst = std::max(worst, ms_half);
      }
    }
    if (s.code) {
      m->sec_hi_cols[pi] = saved_cols;
      return s;
    }
    if (ms_half < best) {
      best = ms_half;
      m->sec_hi_cols[pi] = full / 2;
    } else {
      m->sec_hi_cols[pi] = 0;
    }
    res->best_split_hi_cols = m->sec_hi_cols[pi] ? full / 2 : full;
  }
  res->best_split_L = best_sh.first;
  res->best_split_K = best_sh.second;
  res->best_ms = best;
  res->default_ms = dms;
  res->worst_ms = worst;
  return sec_ensure(m, prec, st);
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int hphi_create(hphi_model** out, int kind, int n_sites) {
  if (!out) return fail(nullptr, HPHI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (kind != HPHI_SPIN_HALF && kind != HPHI_HUBBARD) return fail(nullptr, HPHI_ERR_INVALID_ARG, "unknown model kind");
  if (n_sites < 1 || (kind == HPHI_SPIN_HALF && n_sites > 63) || (kind == HPHI_HUBBARD && n_sites > 24))
    return fail(nullptr, HPHI_ERR_INVALID_ARG, "n_sites out of range");
  hphi_model* m = new (std::nothrow) hphi_model();
  if (!m) return fail(nullptr, HPHI_ERR_OUT_OF_MEMORY, "host allocation failed");
  m->kind = kind;
  m->n_sites = n_sites;
  *out = m;
  return HPHI_OK;
}

void hphi_destroy(hphi_model* m) { delete m; }

const char* hphi_last_error(const hphi_model* m) {
  if (m) return m->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

int hphi_add_spin_coupling(hphi_model* m, int i, int j, const double J[9]) {
  if (!m || !J) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_SPIN_HALF) return fail(m, HPHI_ERR_INVALID_ARG, "spin coupling on a Hubbard model");
  if (i < 0 || j < 0 || i >= m->n_sites || j >= m->n_sites || i == j)
    return fail(m, HPHI_ERR_INVALID_ARG, "coupling sites out of range or equal");
  Coupling c{i, j, {}};
  for (int k = 0; k < 9; ++k) {
    if (!isfinite(J[k])) return fail(m, HPHI_ERR_INVALID_ARG, "non-finite coupling");
    c.J[k] = J[k];
  }
  m->coup.push_back(c);
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_add_spin_field(hphi_model* m, int i, const double h[3]) {
  if (!m || !h) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_SPIN_HALF) return fail(m, HPHI_ERR_INVALID_ARG, "spin field on a Hubbard model");
  if (i < 0 || i >= m->n_sites) return fail(m, HPHI_ERR_INVALID_ARG, "field site out of range");
  for (int k = 0; k < 3; ++k)
    if (!isfinite(h[k])) return fail(m, HPHI_ERR_INVALID_ARG, "non-finite field");
  m->field.push_back(Field{i, {h[0], h[1], h[2]}});
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_add_hopping(hphi_model* m, int i, int j, int spin, double t_re, double t_im) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_HUBBARD) return fail(m, HPHI_ERR_INVALID_ARG, "hopping on a spin model");
  if (i < 0 || j < 0 || i >= m->n_sites || j >= m->n_sites || i == j || (spin != 0 && spin != 1))
    return fail(m, HPHI_ERR_INVALID_ARG, "hopping sites/spin out of range");
  if (!isfinite(t_re) || !isfinite(t_im)) return fail(m, HPHI_ERR_INVALID_ARG, "non-finite hopping");
  m->hop.push_back(Hop{i, j, spin, t_re, t_im});
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_add_onsite_U(hphi_model* m, int i, double U) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_HUBBARD) return fail(m, HPHI_ERR_INVALID_ARG, "U on a spin model");
  if (i < 0 || i >= m->n_sites || !isfinite(U)) return fail(m, HPHI_ERR_INVALID_ARG, "bad onsite U");
  m->onsite.push_back(Onsite{i, U});
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_add_density(hphi_model* m, int i, int j, double V) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_HUBBARD) return fail(m, HPHI_ERR_INVALID_ARG, "V on a spin model");
  if (i < 0 || j < 0 || i >= m->n_sites || j >= m->n_sites || i == j || !isfinite(V))
    return fail(m, HPHI_ERR_INVALID_ARG, "bad density interaction");
  m->dens.push_back(Density{i, j, V});
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_add_chemical_potential(hphi_model* m, int i, double mu) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_HUBBARD) return fail(m, HPHI_ERR_INVALID_ARG, "mu on a spin model");
  if (i < 0 || i >= m->n_sites || !isfinite(mu)) return fail(m, HPHI_ERR_INVALID_ARG, "bad chemical potential");
  m->chem.push_back(Chem{i, mu});
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_set_basis(hphi_model* m, int basis, int a, int b) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind == HPHI_SPIN_HALF) {
    if (basis == HPHI_BASIS_FULL) { a = 0; b = 0; }
    else if (basis == HPHI_BASIS_SZ) {
      if (a < 0 || a > m->n_sites) return fail(m, HPHI_ERR_INVALID_ARG, "number of up spins out of range");
      b = 0;
    } else return fail(m, HPHI_ERR_INVALID_ARG, "spin models take HPHI_BASIS_FULL or HPHI_BASIS_SZ");
  } else {
    if (basis == HPHI_BASIS_FULL) { a = 0; b = 0; }
    else if (basis == HPHI_BASIS_NUMBER) {
      if (a < 0 || a > m->n_sites || b < 0 || b > m->n_sites)
        return fail(m, HPHI_ERR_INVALID_ARG, "particle numbers out of range");
    } else return fail(m, HPHI_ERR_INVALID_ARG, "Hubbard models take HPHI_BASIS_FULL or HPHI_BASIS_NUMBER");
  }
  m->basis = basis;
  m->a = a;
  m->b = b;
  m->built = false;
  ++m->gen;
  return HPHI_OK;
}

int hphi_build_sector(hphi_model* m, int64_t* dim_out, void* stream) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  m->built = false;
  hphi::Status s = build_sector_impl(m, (cudaStream_t)stream);
  if (s.code) return fail(m, s);
  m->built = true;
  if (dim_out) *dim_out = m->dim;
  return HPHI_OK;
}

int64_t hphi_dim(const hphi_model* m) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (!m->built) return HPHI_ERR_NOT_BUILT;
  return m->dim;
}

int hphi_is_complex(const hphi_model* m) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (!m->built) return HPHI_ERR_NOT_BUILT;
  return m->cplx_model ? 1 : 0;
}

int hphi_basis_states(hphi_model* m, int64_t r0, int64_t n, uint64_t* states, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (r0 < 0 || n < 0 || r0 + n > m->dim || (n > 0 && !states)) return fail(m, HPHI_ERR_INVALID_ARG, "row range");
  hphi::Status s = m->kind == HPHI_HUBBARD ? hphi::launch_hub_states(m->hdev, r0, n, states, (cudaStream_t)stream)
                                           : hphi::launch_spin_states(m->sdev, r0, n, states, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_basis_ranks(hphi_model* m, const uint64_t* states, int64_t n, int64_t* ranks, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (n < 0 || (n > 0 && (!states || !ranks))) return fail(m, HPHI_ERR_INVALID_ARG, "bad arrays");
  hphi::Status s = m->kind == HPHI_HUBBARD ? hphi::launch_hub_ranks(m->hdev, states, n, ranks, (cudaStream_t)stream)
                                           : hphi::launch_spin_ranks(m->sdev, states, n, ranks, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_apply_H(hphi_model* m, const void* v, void* w, int nvec, int prec, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!v || !w || nvec < 1 || nvec > hphi::kMaxNvec || (prec != HPHI_FP64 && prec != HPHI_FP32))
    return fail(m, HPHI_ERR_INVALID_ARG, "apply_H: bad vectors, nvec or precision");
  if (v == w) return fail(m, HPHI_ERR_INVALID_ARG, "apply_H: v and w must not overlap");
  hphi::FusedArgs fa;
  void* scratch = nullptr;
  const size_t need = hv_scratch_bytes(m, prec, nvec, hphi::Epi::kStore);
  if (need && m->kind == HPHI_SPIN_HALF && !use_batch(m, nvec)) {
    scratch = optional_scratch(m, need);
  } else if (need) {
    hphi::Status a = m->ws.work.ensure(need);
    if (a.code) return fail(m, a);
    scratch = m->ws.work.p;
  }
  hphi::Status s = hv_launch(m, prec, v, w, nvec, hphi::Epi::kStore, fa, hv_grid_for(m, nvec, prec, hphi::Epi::kStore),
                             scratch, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_release_workspace(hphi_model* m) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(m, HPHI_ERR_CUDA, std::string("release_workspace: ") + cudaGetErrorString(e));
  Workspace& ws = m->ws;
  for (DBuf* b : {&ws.vecA, &ws.vecB, &ws.x, &ws.partials, &ws.scal, &ws.work, &ws.basis, &ws.cgp, &ws.cgq})
    b->release();
  return HPHI_OK;
}

int hphi_set_window_bits(hphi_model* m, int bits) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (bits < -1 || bits > 32) return fail(m, HPHI_ERR_INVALID_ARG, "window bits: -1, 0 or 1..32");
  m->win_bits_opt = bits;
  return HPHI_OK;
}

int hphi_set_sector_split(hphi_model* m, int prec, int L, int K, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (prec != HPHI_FP64 && prec != HPHI_FP32) return fail(m, HPHI_ERR_INVALID_ARG, "set_sector_split: prec FP64 or FP32");
  if (L < -1 || L > hphi::kSecMaxL || K < 0 || K > 8 || (K & (K - 1)))
    return fail(m, HPHI_ERR_INVALID_ARG, "set_sector_split: L in -1..20, K in {0, 1, 2, 4, 8}");
  const int pi = prec == HPHI_FP64 ? 0 : 1;
  if (L >= 0 && !m->sec_ok[pi])
    return fail(m, HPHI_ERR_UNSUPPORTED,
                m->sec_why.empty() ? std::string("set_sector_split: the model does not take the split-row path")
                                   : m->sec_why);
  const int oldL = m->sec_L[pi], oldK = m->sec_K[pi];
  m->sec_L[pi] = L;
  m->sec_K[pi] = L < 0 ? 0 : K;
  m->sec_hi_cols[pi] = 0;
  if (L >= 0) {
    const int esz = prec == HPHI_FP64 ? 8 : 4;
    const std::pair<int, int> sh = sec_shape(m, prec);
    if (sh.first == 0 || !hphi::sec_fits(m->sec_terms, sh.first, sh.second, esz)) {
      m->sec_L[pi] = oldL;
      m->sec_K[pi] = oldK;
      return fail(m, HPHI_ERR_INVALID_ARG,
                  "set_sector_split: the high part must have 1..22 bits and K rows of the longest row must fit one "
                  "shared-memory tile");
    }
    hphi::Status s = sec_ensure(m, prec, (cudaStream_t)stream);
    if (s.code) {
      m->sec_L[pi] = oldL;
      m->sec_K[pi] = oldK;
      return fail(m, s);
    }
  }
  return HPHI_OK;
}

}  // extern "C"

namespace {
hphi::Status sector_model(hphi_model* m, int n_up, cudaStream_t st, hphi_model** out);

// A spin model in its full basis: tune the split-row shape of every S^z sector of at least
// 2^20 rows, the sectors hphi_lanczos_run_sectors runs (their sub-models keep the shapes).
// The result reports the candidates of all of them and the timings of the largest.
hphi::Status tune_sectors(hphi_model* m, int prec, hphi_tune_result* res, cudaStream_t st) {
  if (m->n_sites > 40) return {};
  int n_cand = 0;
  hphi_tune_result big{};
  int64_t big_dim = 0;
  for (int n_up = 0; n_up <= m->n_sites; ++n_up) {
    const int64_t d = (int64_t)binom_host(m->n_sites, n_up);
    if (d < ((int64_t)1 << 20)) continue;
    hphi_model* sub = nullptr;
    hphi::Status s = sector_model(m, n_up, st, &sub);
    if (s.code) return s;
    const int pi = prec == HPHI_FP64 ? 0 : 1;
    if (!sub->sec_ok[pi] || sub->sec_L[pi] < 0 || sub->cplx_model) continue;
    hphi_tune_result r{};
    if ((s = sec_autotune(sub, prec, &r, st)).code) return s;
    n_cand += r.n_candidates;
    if (d > big_dim) {
      big_dim = d;
      big = r;
    }
  }
  *res = big;
  res->n_candidates = n_cand;
  return {};
}
}  // namespace

extern "C" {

int hphi_autotune(hphi_model* m, int prec, hphi_tune_result* out, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (prec != HPHI_FP64 && prec != HPHI_FP32) return fail(m, HPHI_ERR_INVALID_ARG, "autotune: prec FP64 or FP32");
  hphi_tune_result res{};
  if (m->kind == HPHI_SPIN_HALF && m->basis == HPHI_BASIS_FULL && !m->cplx_model) {
    hphi::Status s = tune_sectors(m, prec, &res, (cudaStream_t)stream);
    if (s.code) return fail(m, s);
    if (out) *out = res;
    return HPHI_OK;
  }
  if (m->kind == HPHI_SPIN_HALF && m->sec_ok[prec == HPHI_FP64 ? 0 : 1] && m->sec_L[prec == HPHI_FP64 ? 0 : 1] >= 0 &&
      !m->cplx_model) {
    hphi::Status s = sec_autotune(m, prec, &res, (cudaStream_t)stream);
    if (s.code) return fail(m, s);
    if (out) *out = res;
    return HPHI_OK;
  }
  if (!use_hub_fast(m, prec, 1, hphi::Epi::kStore)) {
    if (out) *out = res;
    return HPHI_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t esz = prec == HPHI_FP64 ? 8 : 4;
  hphi::Status s;
  if ((s = m->ws.vecA.ensure(esz * (size_t)m->dim)).code) return fail(m, s);
  if ((s = m->ws.vecB.ensure(esz * (size_t)m->dim)).code) return fail(m, s);
  const size_t need = hphi::hub_scratch_bytes(m->hdev, prec, hphi::Epi::kStore);
  if (need && (s = m->ws.work.ensure(need)).code) return fail(m, s);
  void* scratch = need ? m->ws.work.p : nullptr;
  if ((s = hphi::launch_random(m->ws.vecA.p, m->dim, false, prec == HPHI_FP64, 7, st)).code) return fail(m, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    cudaGetLastError();
    return fail(m, HPHI_ERR_CUDA, "autotune: cudaEventCreate failed");
  }
  const int pi = prec == HPHI_FP64 ? 0 : 1;
  const int saved_ept = m->hdev.tuned_ept[pi], saved_k = m->hdev.tuned_k[pi];
  float best = 1e30f, worst = 0.f, dflt = 0.f;
  int best_ept = 0, best_k = 0;
  const int epts[] = {0, 1, 2, 4};
  const int ks[] = {0, 1, 2, 4};
  hphi::FusedArgs fa;
  for (int ept : epts) {
    for (int k : ks) {
      if ((ept == 0) != (k == 0)) continue;  // (0, 0) is the built-in default
      m->hdev.tuned_ept[pi] = ept;
      m->hdev.tuned_k[pi] = k;
      const int grid = hv_grid_for(m, 1, prec, hphi::Epi::kStore);
      s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, scratch, st);
      if (s.code) break;
      cudaEventRecord(a, st);
      for (int rep = 0; rep < 3 && !s.code; ++rep)
        s = hv_launch(m, prec, m->ws.vecA.p, m->ws.vecB.p, 1, hphi::Epi::kStore, fa, grid, scratch, st);
      cudaEventRecord(b, st);
      if (s.code) break;
      if (cudaEventSynchronize(b) != cudaSuccess) {
        s = {HPHI_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(cudaGetLastError())};
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      ms /= 3.f;
      ++res.n_candidates;
      if (ept == 0) dflt = ms;
      worst = std::max(worst, ms);
      if (ms < best) {
        best = ms;
        best_ept = ept;
        best_k = k;
      }
    }
    if (s.code) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s.code) {
    m->hdev.tuned_ept[pi] = saved_ept;
    m->hdev.tuned_k[pi] = saved_k;
    return fail(m, s);
  }
  m->hdev.tuned_ept[pi] = best_ept;
  m->hdev.tuned_k[pi] = best_k;
  res.best_dn_ept = best_ept;
  res.best_up_k = best_k;
  res.best_ms = best;
  res.default_ms = dflt;
  res.worst_ms = worst;
  if (out) *out = res;
  return HPHI_OK;
}

int hphi_apply_H_noalloc(hphi_model* m, const void* v, void* w, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!v || !w) return fail(m, HPHI_ERR_INVALID_ARG, "apply_H_noalloc: v and w must be device buffers");
  if (v == w) return fail(m, HPHI_ERR_INVALID_ARG, "apply_H_noalloc: v and w must not overlap");
  if (!use_hub_fast(m, HPHI_FP64, 1, hphi::Epi::kStore))
    return fail(m, HPHI_ERR_UNSUPPORTED,
                "apply_H_noalloc: only real Hubbard models with one hopping value per spin species (fp64, one vector)");
  hphi::Status s = hphi::launch_hub_store_noalloc(m->hdev, v, w, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_random_vector(hphi_model* m, void* v, int nvec, int prec, uint64_t seed, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!v || nvec < 1 || (prec != HPHI_FP64 && prec != HPHI_FP32)) return fail(m, HPHI_ERR_INVALID_ARG, "bad vector");
  hphi::Status s = hphi::launch_random(v, m->dim * nvec, m->cplx_model, prec == HPHI_FP64, seed, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(nullptr, HPHI_ERR_INVALID_ARG, "bad arrays");
  hphi::Status s = hphi::launch_philox_raw(ctr, key, out, n, (cudaStream_t)stream);
  return s.code ? fail(nullptr, s) : HPHI_OK;
}

}  // extern "C"

// ====================================================================== Lanczos driver
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// One Lanczos run, split so several runs can be captured as parallel branches of one graph:
// lz_prepare allocates (no launches), lz_enqueue issues every kernel in stream order
// (capturable), lz_collect copies the scalars back after the stream has run.
struct LzPlan {
  hphi_model* m = nullptr;
  int steps = 0, prec = 0, n_eig = 1;
  bool cplx = false, refine = false, profile = false, store = false;
  int64_t n_real = 0;
  size_t vbytes = 0;
  int grid = 1, rgrid = 1, vgrid = 1;
  double* partials = nullptr;
  void* scratch = nullptr;
  hphi::LzDev lz{};
  double* base = nullptr;
  size_t nsc = 0;
  int* flags = nullptr;
  double brk = 1e-13;
  double eps = 0.0;  // convergence test of appendix C (0: off)
  void* ritz_out = nullptr;
  bool cta = false;  // the whole recurrence in one thread-block cluster (small real spin models)
  bool reorth = false;  // full reorthogonalisation against the kept basis
  const double* v0 = nullptr;
  const double* v0_host = nullptr;  // start vector in host memory (copied in by start())
  uint64_t seed = 0;
  int launches = 0;
  std::vector<cudaEvent_t> ev;  // profile: events around every fused H v launch
  ~LzPlan() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

hphi::Status lz_prepare(hphi_model* m, const hphi_lanczos_params* p, LzPlan& L) {
  L.m = m;
  L.steps = p->steps;
  L.prec = p->prec;
  L.n_eig = std::max(1, std::min(8, p->n_eig));
  L.cplx = m->cplx_model;
  L.refine = p->refine != 0;
  L.profile = p->profile != 0;
  L.v0 = reinterpret_cast<const double*>(p->v0);
  if (p->v0_on_host && p->v0) {
    L.v0_host = L.v0;
    L.v0 = nullptr;
  }
  L.seed = p->seed;
  L.brk = p->breakdown > 0 ? p->breakdown : 1e-13;
  L.eps = p->eps > 0 ? p->eps : 0.0;
  L.ritz_out = p->ritz_out;
  L.reorth = p->reorth != 0;
  const int steps = L.steps, prec = L.prec;
  const size_t esz = (prec == HPHI_FP64 ? 8 : 4) * (L.cplx ? 2 : 1);
  L.n_real = m->dim * (L.cplx ? 2 : 1);
  const size_t vbytes = esz * (size_t)m->dim;
  Workspace& ws = m->ws;
  hphi::Status s;
  // the refinement's fp64 H x reuses buffer A, which must then hold an fp64 vector
  const size_t need_a = L.refine ? std::max(vbytes, (size_t)8 * (size_t)L.n_real) : vbytes;
  L.vbytes = vbytes;
  // keep the whole basis when asked, or when it fits comfortably (the refinement then needs
  // one streaming pass over it instead of a second Lanczos run)
  if (L.reorth || (L.refine && p->keep_basis >= 0)) {
    const size_t need = (size_t)(steps + 1) * vbytes;
    if (p->keep_basis == 1 || L.reorth) {
      L.store = true;
    } else {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) cudaGetLastError();
      // a basis buffer kept from an earlier run counts as free (ensure() reuses or replaces it)
      L.store = ws.basis.bytes >= need || need <= (size_t)(0.6 * (double)(free_b + ws.basis.bytes));
    }
    if (L.store && (s = ws.basis.ensure(need)).code) return s;
  }
  if ((s = ws.vecA.ensure(L.store ? (size_t)8 * (size_t)L.n_real : need_a)).code) return s;
  if (!L.store && (s = ws.vecB.ensure(vbytes)).code) return s;
  if ((L.refine || (L.v0_host && prec != HPHI_FP64)) && (s = ws.x.ensure(8 * (size_t)L.n_real)).code) return s;
  if (use_hub_fast(m, prec, 1, hphi::Epi::kLanczos1)) {
    size_t need = hphi::hub_scratch_bytes(m->hdev, prec, hphi::Epi::kLanczos1);
    if (L.refine) need = std::max(need, hphi::hub_scratch_bytes(m->hdev, HPHI_FP64, hphi::Epi::kRefine));
    if ((s = ws.work.ensure(need)).code) return s;
    L.scratch = ws.work.p;
  } else if (m->kind == HPHI_SPIN_HALF) {
    // split-row kernels (S^z sectors of real models): their scratch (fp64: the quantised copy;
    // Lanczos: one more vector for the high-part sums); generic fp64 kernels gather from a
    // quantised copy.  Without the memory the generic kernels' per-term sums run instead.
    size_t need = std::max(hv_scratch_bytes(m, prec, 1, hphi::Epi::kLanczos1),
                           hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, 1));
    if (L.refine)
      need = std::max(need, std::max(hv_scratch_bytes(m, HPHI_FP64, 1, hphi::Epi::kRefine),
                                     hphi::spin_scratch_bytes(m->sdev, HPHI_FP64, m->cplx_model, 1)));
    L.scratch = optional_scratch(m, need);
    if (L.scratch == nullptr) {
      size_t gen = hphi::spin_scratch_bytes(m->sdev, prec, m->cplx_model, 1);
      if (L.refine) gen = std::max(gen, hphi::spin_scratch_bytes(m->sdev, HPHI_FP64, m->cplx_model, 1));
      L.scratch = optional_scratch(m, gen);
    }
  }
  // small real spin models: both vectors in one thread-block cluster's shared memory, one
  // kernel for all steps
  L.cta = m->kind == HPHI_SPIN_HALF && !L.cplx && prec == HPHI_FP64 && !L.refine && !L.profile && L.eps == 0.0 &&
          !L.reorth && hphi::lz_cta_smem(m->sdev) > 0;
  // grids after the scratch: the split-row kernels run only when it holds what they need
  L.grid = hv_grid_for(m, 1, prec, hphi::Epi::kLanczos1);
  L.rgrid = hv_grid_for(m, 1, HPHI_FP64, hphi::Epi::kRefine);
  L.vgrid = launch_grid(L.n_real);
  const int pgrid = std::max(std::max(L.grid, L.rgrid), L.vgrid);
  size_t pdoubles = (size_t)pgrid * hphi::kMaxRedQ;
  if (L.reorth) pdoubles = std::max(pdoubles, hphi::ro_part_doubles(L.vgrid));
  if ((s = ws.partials.ensure(sizeof(double) * pdoubles)).code) return s;
  L.partials = ws.partials.as<double>();
  // scalars: alpha[m], beta[m], sig[m+1], coef[m], s[16], tri[16 + 5m], done, steps_done,
  // then ro[2 (m + 1)]
  L.nsc = 3 * (size_t)steps + 1 + steps + 16 + 16 + 5 * (size_t)steps + 4 + 2 * ((size_t)steps + 1);
  if ((s = ws.scal.ensure(sizeof(double) * L.nsc)).code) return s;
  L.base = ws.scal.as<double>();
  L.lz.alpha = L.base;
  L.lz.beta = L.lz.alpha + steps;
  L.lz.sig = L.lz.beta + steps;
  L.lz.coef = L.lz.sig + steps + 1;
  L.lz.s = L.lz.coef + steps;
  L.lz.tri = L.lz.s + 16;
  L.flags = reinterpret_cast<int*>(L.lz.tri + 16 + 5 * (size_t)steps);
  L.lz.done = L.flags;
  L.lz.steps_done = L.flags + 1;
  L.lz.ro = reinterpret_cast<double*>(L.flags + 4);  // after the flags' two doubles of room
  if (L.profile) {
    L.ev.assign(2 * (size_t)steps, nullptr);
    for (auto& e : L.ev) {
      const cudaError_t ce = cudaEventCreate(&e);
      if (ce != cudaSuccess) return {HPHI_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce)};
    }
  }
  return {};
}

// Lanczos recurrence of section 3.4 (m fused steps), the tridiagonal eigensolve and, if asked,
// the second pass with the fp64 Ritz vector and its Rayleigh quotient / residual.
hphi::Status lz_enqueue(LzPlan& L, cudaStream_t st) {
  hphi_model* m = L.m;
  Workspace& ws = m->ws;
  const int steps = L.steps, prec = L.prec;
  const bool cplx = L.cplx;
  hphi::Status s;
  L.launches = 0;
  HPHI_CUDA_TRY(cudaMemsetAsync(L.base, 0, sizeof(double) * L.nsc, st));
  // stored basis: V_k at slot k (C_k); otherwise two buffers A / B swapped every step
  auto slot = [&](int k) -> void* {
    return static_cast<char*>(ws.basis.p) + (size_t)k * L.vbytes;
  };
  void* c0 = L.store ? slot(0) : ws.vecA.p;
  void* p0 = L.store ? slot(1) : ws.vecB.p;
  // fp32 runs take a host start vector through the fp64 vector x, which lz_init reads before
  // the second pass clears it
  const double* v0_dev = L.v0 ? L.v0 : ((L.v0_host && prec != HPHI_FP64) ? ws.x.as<double>() : nullptr);
  auto start = [&]() -> hphi::Status {
    if (L.v0) return {};
    if (L.v0_host) {  // copied in again for the second pass
      void* dst = prec == HPHI_FP64 ? c0 : ws.x.p;
      HPHI_CUDA_TRY(cudaMemcpyAsync(dst, L.v0_host, 8 * (size_t)L.n_real, cudaMemcpyHostToDevice, st));
      return {};
    }
    ++L.launches;  // buffer A holds C_0 (regenerated bit-identically for the second pass)
    return hphi::launch_random(c0, m->dim, cplx, prec == HPHI_FP64, L.seed, st);
  };
  // fp64 fixed-point paths (two-pass Hubbard, split-row): pass 1 records the largest exponent
  // of the P it writes, and pass 2 writes the next step's quantised copy on a scale bounded
  // from it (k_lz_pass2) and finds the new vector's exact largest exponent, so the next step's
  // H v starts from a ready copy: no max-exponent scan, no quantisation pass
  int* emax = nullptr;
  hphi::QSlots qs;
  if (prec == HPHI_FP64 && L.scratch != nullptr && !cplx) {
    if (use_hub_fast(m, prec, 1, hphi::Epi::kLanczos1))
      qs = hphi::hub_qslots(m->hdev, L.scratch);
    else if (sec_runs(m, prec, 1, hphi::Epi::kLanczos1, ws.work.bytes))
      qs = hphi::sec_qslots(*use_sec(m, prec, 1, hphi::Epi::kLanczos1), prec, hphi::Epi::kLanczos1, L.scratch);
  }
  const bool qnext = qs.Q != nullptr;
  auto run_pass = [&](bool with_x) -> hphi::Status {
    hphi::Status q;
    L.launches += 2 + (3 + hv_kernels(m, prec, 1, hphi::Epi::kLanczos1)) * steps - (qnext ? 2 * (steps - 1) : 0);
    if ((q = hphi::launch_lz_init(prec, cplx, v0_dev, c0, p0, L.n_real, L.partials, L.vgrid, st)).code) return q;
    if ((q = hphi::launch_lz_init_fin(L.lz, L.partials, L.vgrid, st)).code) return q;
    if (with_x) HPHI_CUDA_TRY(cudaMemsetAsync(ws.x.p, 0, 8 * (size_t)L.n_real, st));
    void* C = c0;
    void* P = p0;
    for (int k = 0; k < steps; ++k) {
      hphi::FusedArgs fa;
      if (L.store) {
        // pass 1 reads v_{k-1} from its slot and writes u into slot k + 1 (slot 1 holds the
        // zero vector at k = 0); pass 2 finishes slot k + 1 in place
        C = slot(k);
        P = slot(k + 1);
        fa.in = (k == 0) ? slot(1) : slot(k - 1);
      }
      fa.out = P;
      fa.scal = L.lz.s;
      fa.partials = L.partials;
      fa.done = L.lz.done;
      fa.exp_ready = (qnext && k > 0) ? 2 : 0;
      fa.pexp = qnext ? qs.ep : nullptr;
      const bool timed = L.profile && !with_x;
      if (timed) HPHI_CUDA_TRY(cudaEventRecord(L.ev[2 * k], st));
      if ((q = hv_launch(m, prec, C, nullptr, 1, hphi::Epi::kLanczos1, fa, L.grid, L.scratch, st)).code) return q;
      if (timed) HPHI_CUDA_TRY(cudaEventRecord(L.ev[2 * k + 1], st));
      if ((q = hphi::launch_lz_fin1(L.lz, k, L.partials, L.grid, st)).code) return q;
      hphi::QNext qn{};
      if (qnext) {
        // the exact exponent of C_k: k_maxexp's slot (the copy's) at k = 0, else the one the
        // previous pass 2 found; this pass 2 finds C_{k+1}'s into the other slot
        emax = qs.ec[(k + 1) & 1];
        qn = hphi::QNext{qs.Q, qs.eq, qs.ep, k == 0 ? qs.eq : qs.ec[k & 1], qs.extra};
        HPHI_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(int), st));
      }
      if ((q = hphi::launch_lz_pass2(prec, cplx, L.lz, k, C, P, with_x ? ws.x.as<double>() : nullptr, L.n_real,
                                     L.partials, L.vgrid, emax, st, qnext ? &qn : nullptr)).code)
        return q;
      if (L.reorth && !with_x) {  // P is slot k + 1 of the kept basis; its norm replaces pass 2's
        L.launches += hphi::reorth_launches(k);
        if ((q = hphi::launch_reorth(prec, cplx, L.lz, k, slot(0), L.n_real,
                                     (int64_t)(L.vbytes / (prec == HPHI_FP64 ? 8 : 4)), P, L.partials, L.partials,
                                     L.vgrid, st)).code)
          return q;
      }
      if ((q = hphi::launch_lz_fin2(L.lz, k, L.brk, L.partials, L.vgrid, with_x, st)).code) return q;
      // appendix C: after five steps, then every two, unless the run already stopped
      if (!with_x && L.eps > 0.0 && k + 1 >= 5 && (k + 1 - 5) % 2 == 0 && k + 1 < steps) {
        ++L.launches;
        if ((q = hphi::launch_lz_conv(L.lz, L.eps, st)).code) return q;
      }
      if (!L.store) std::swap(C, P);
    }
    return {};
  };
  if ((s = start()).code) return s;
  if (L.cta) {
    L.launches += 3;
    if ((s = hphi::launch_lz_init(prec, cplx, v0_dev, c0, p0, L.n_real, L.partials, L.vgrid, st)).code) return s;
    if ((s = hphi::launch_lz_init_fin(L.lz, L.partials, L.vgrid, st)).code) return s;
    if ((s = hphi::launch_lz_cta(m->sdev, L.lz, steps, L.brk, static_cast<const double*>(c0), st)).code) return s;
  } else if ((s = run_pass(false)).code) {
    return s;
  }
  ++L.launches;
  // the replayed pass may skip steps whose Ritz coefficients change the unit Ritz vector by
  // less than the storage precision's rounding (fp64: 1e-15, fp32: 1e-8)
  const double tail_tol = prec == HPHI_FP64 ? 1e-30 : 1e-16;
  if ((s = hphi::launch_tridiag(L.lz, steps, L.n_eig, L.refine, tail_tol, st)).code) return s;
  if (!L.refine) return {};
  if (L.store) {
    // Ritz vector straight from the stored basis: one streaming pass
    ++L.launches;
    if ((s = hphi::launch_lz_combine(prec, L.lz, slot(0), L.n_real, (int64_t)(L.vbytes / (prec == HPHI_FP64 ? 8 : 4)),
                                     ws.x.as<double>(), L.vgrid, st)).code)
      return s;
  } else {
    if ((s = start()).code) return s;
    if ((s = run_pass(true)).code) return s;
  }
  L.launches += 3 + hv_kernels(m, HPHI_FP64, 1, hphi::Epi::kRefine);
  // fp64 H x into the (now free) buffer A, then E, variance and residual
  double* hx = ws.vecA.as<double>();
  hphi::FusedArgs fa;
  fa.out = hx;
  fa.partials = L.partials;
  if ((s = hv_launch(m, HPHI_FP64, ws.x.p, nullptr, 1, hphi::Epi::kRefine, fa, L.rgrid, L.scratch, st)).code) return s;
  if ((s = hphi::launch_refine_fin(L.lz, L.partials, L.rgrid, 0, st)).code) return s;
  if ((s = hphi::launch_refine_resid(cplx, ws.x.as<double>(), hx, L.n_real, L.lz, L.partials, L.vgrid, st)).code)
    return s;
  if ((s = hphi::launch_refine_fin(L.lz, L.partials, L.vgrid, 1, st)).code) return s;
  if (L.ritz_out)
    HPHI_CUDA_TRY(cudaMemcpyAsync(L.ritz_out, ws.x.p, 8 * (size_t)L.n_real, cudaMemcpyDeviceToDevice, st));
  return {};
}

hphi::Status lz_collect(LzPlan& L, hphi_lanczos_result* r, cudaStream_t st) {
  std::vector<double> host(L.nsc);
  HPHI_CUDA_TRY(cudaMemcpyAsync(host.data(), L.base, sizeof(double) * L.nsc, cudaMemcpyDeviceToHost, st));
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));
  const int* hf = reinterpret_cast<const int*>(host.data() + (reinterpret_cast<double*>(L.flags) - L.base));
  r->steps_done = hf[1];
  r->converged = host[(L.lz.s - L.base) + 8] > 0.0 ? 1 : 0;
  if (r->alpha) memcpy(r->alpha, host.data() + (L.lz.alpha - L.base), sizeof(double) * L.steps);
  if (r->beta) memcpy(r->beta, host.data() + (L.lz.beta - L.base), sizeof(double) * L.steps);
  for (int k = 0; k < 8; ++k) r->eig[k] = (k < L.n_eig) ? host[(L.lz.tri - L.base) + k] : 0.0;
  if (L.refine) {
    r->e_refined = host[(L.lz.tri - L.base) + 8];
    r->residual = host[(L.lz.tri - L.base) + 9];
    r->variance = host[(L.lz.tri - L.base) + 10];
  } else {
    r->e_refined = r->residual = r->variance = 0.0;
  }
  r->hv_ms = 0.f;
  r->hv_launches = 0;
  if (L.profile) {
    for (int k = 0; k < L.steps && k < r->steps_done; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, L.ev[2 * k], L.ev[2 * k + 1]) == cudaSuccess) r->hv_ms += t;
      else cudaGetLastError();  // clear the error so later calls do not report it
    }
    r->hv_launches = std::min(L.steps, r->steps_done);
  }
  r->kernel_launches = L.launches;
  return {};
}

// Runs `enqueue` captured into one CUDA graph (fork/join over `branches` streams if > 0) and
// launches it on st between the events of tm.
template <class F>
hphi::Status run_graph(cudaStream_t st, Timer& tm, int branches, F enqueue) {
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> bs(std::max(0, branches), nullptr);
  std::vector<cudaEvent_t> joins(bs.size(), nullptr);
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  hphi::Status s;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : joins)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (auto b : bs)
      if (b) cudaStreamDestroy(b);
    if (cap) cudaStreamDestroy(cap);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (size_t i = 0; e == cudaSuccess && i < bs.size(); ++i) {
    e = cudaStreamCreateWithFlags(&bs[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cleanup();
    return {HPHI_ERR_CUDA, std::string("graph setup: ") + cudaGetErrorString(e)};
  }
  if (bs.empty()) {
    s = enqueue(0, cap);
  } else {
    e = cudaEventRecord(fork, cap);
    for (size_t i = 0; e == cudaSuccess && i < bs.size() && !s.code; ++i) {
      e = cudaStreamWaitEvent(bs[i], fork, 0);
      if (e == cudaSuccess) s = enqueue((int)i, bs[i]);
      if (e == cudaSuccess && !s.code) e = cudaEventRecord(joins[i], bs[i]);
      if (e == cudaSuccess && !s.code) e = cudaStreamWaitEvent(cap, joins[i], 0);
    }
    if (e != cudaSuccess && !s.code) s = {HPHI_ERR_CUDA, std::string("graph fork/join: ") + cudaGetErrorString(e)};
  }
  e = cudaStreamEndCapture(cap, &graph);
  if (!s.code && e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e)};
  if (!s.code) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)};
  }
  if (!s.code) {
    e = cudaEventRecord(tm.a, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(tm.b, st);
    if (e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e)};
  }
  cleanup();
  return s;
}

hphi::Status lanczos_impl(hphi_model* m, const hphi_lanczos_params* p, hphi_lanczos_result* r, cudaStream_t st) {
  LzPlan L;
  hphi::Status s = lz_prepare(m, p, L);
  if (s.code) return s;
  Timer tm;
  HPHI_CUDA_TRY(cudaEventCreate(&tm.a));
  HPHI_CUDA_TRY(cudaEventCreate(&tm.b));
  if (L.profile || L.v0_host) {
    // profiled runs launch eagerly: events recorded inside a captured graph cannot be
    // queried with cudaEventElapsedTime; so do runs copying a host start vector
    HPHI_CUDA_TRY(cudaEventRecord(tm.a, st));
    if ((s = lz_enqueue(L, st)).code) return s;
    HPHI_CUDA_TRY(cudaEventRecord(tm.b, st));
  } else {
    s = run_graph(st, tm, 0, [&](int, cudaStream_t cs) { return lz_enqueue(L, cs); });
    if (s.code) return s;
  }
  if ((s = lz_collect(L, r, st)).code) return s;
  float ms = 0.f;
  HPHI_CUDA_TRY(cudaEventElapsedTime(&ms, tm.a, tm.b));
  r->device_ms = ms;
  return {};
}

// Sector sub-model (same terms, HPHI_BASIS_SZ with n_up up spins), built once per term set.
hphi::Status sector_model(hphi_model* m, int n_up, cudaStream_t st, hphi_model** out) {
  if (m->sub_gen != m->gen) {
    m->sub.clear();
    m->sub_gen = m->gen;
  }
  auto it = m->sub.find(n_up);
  if (it == m->sub.end()) {
    std::unique_ptr<hphi_model> sm(new (std::nothrow) hphi_model());
    if (!sm) return {HPHI_ERR_OUT_OF_MEMORY, "host allocation failed"};
    sm->kind = m->kind;
    sm->n_sites = m->n_sites;
    sm->coup = m->coup;
    sm->field = m->field;
    sm->basis = HPHI_BASIS_SZ;
    sm->a = n_up;
    hphi::Status s = build_sector_impl(sm.get(), st);
    if (s.code) return s;
    sm->built = true;
    it = m->sub.emplace(n_up, std::move(sm)).first;
  }
  *out = it->second.get();
  return {};
}

// All requested S^z sectors in one CUDA graph: each sector's Lanczos chain (fused steps,
// eigensolve, optional refinement) is one branch, so small sectors run beside large ones.
hphi::Status lanczos_sectors_impl(hphi_model* m, const int* n_up, int n_sec, const hphi_lanczos_params* p,
                                  hphi_lanczos_result* res, cudaStream_t st) {
  std::vector<hphi_model*> subs(n_sec, nullptr);
  hphi::Status s;
  for (int i = 0; i < n_sec; ++i)
    if ((s = sector_model(m, n_up[i], st, &subs[i])).code) return s;
  std::vector<std::unique_ptr<LzPlan>> plans;
  for (int i = 0; i < n_sec; ++i) {
    hphi_lanczos_params q = *p;
    q.seed = p->seed + (uint64_t)n_up[i];
    q.v0 = nullptr;
    q.profile = 0;
    plans.emplace_back(new LzPlan());
    if ((s = lz_prepare(subs[i], &q, *plans.back())).code) return s;
  }
  Timer tm;
  HPHI_CUDA_TRY(cudaEventCreate(&tm.a));
  HPHI_CUDA_TRY(cudaEventCreate(&tm.b));
  s = run_graph(st, tm, n_sec, [&](int i, cudaStream_t cs) { return lz_enqueue(*plans[i], cs); });
  if (s.code) return s;
  float ms = 0.f;
  for (int i = 0; i < n_sec; ++i)
    if ((s = lz_collect(*plans[i], &res[i], st)).code) return s;
  HPHI_CUDA_TRY(cudaEventElapsedTime(&ms, tm.a, tm.b));
  for (int i = 0; i < n_sec; ++i) res[i].device_ms = ms;
  return {};
}

hphi::Status tpq_impl(hphi_model* m, const hphi_tpq_params* p, hphi_tpq_result* r, cudaStream_t st) {
  const int nvec = p->n_starts;
  const int K = p->steps;
  const int prec = p->prec;
  const bool cplx = m->cplx_model;
  const size_t esz = (prec == HPHI_FP64 ? 8 : 4) * (cplx ? 2 : 1);
  const size_t vbytes = esz * (size_t)m->dim * nvec;
  Workspace& ws = m->ws;
  hphi::Status s;
  if ((s = ws.vecA.ensure(vbytes)).code) return s;
  if ((s = ws.vecB.ensure(vbytes)).code) return s;
  const size_t tneed = hv_scratch_bytes(m, prec, nvec, hphi::Epi::kTpq);
  if (tneed && (s = ws.work.ensure(tneed)).code) return s;
  void* tscratch = tneed ? ws.work.p : nullptr;
  const int grid = hv_grid_for(m, nvec, prec, hphi::Epi::kTpq);
  const int vgrid = launch_grid(m->dim * nvec);
  const int pgrid = std::max(grid, vgrid);
  if ((s = ws.partials.ensure(sizeof(double) * (size_t)pgrid * nvec * hphi::kMaxRedQ)).code) return s;
  const int obs_every = p->obs_every;
  const size_t nsc = 2 * (size_t)nvec + 6 * (size_t)K * nvec;
  if ((s = ws.scal.ensure(sizeof(double) * nsc)).code) return s;
  hphi::TpqDev tq;
  tq.n2 = ws.scal.as<double>();
  tq.inv = tq.n2 + nvec;
  tq.u = tq.inv + nvec;
  tq.h2 = tq.u + (size_t)K * nvec;
  tq.nrm = tq.h2 + (size_t)K * nvec;
  tq.doub = tq.nrm + (size_t)K * nvec;
  tq.sz = tq.doub + (size_t)K * nvec;
  tq.sz2 = tq.sz + (size_t)K * nvec;
  hphi::ObsDev od{};
  od.n_sites = m->n_sites;
  od.dim = m->dim;
  if (m->kind == HPHI_SPIN_HALF) {
    od.kind = m->basis == HPHI_BASIS_FULL ? 0 : 1;
    od.n_ones = m->a;
  } else {
    od.kind = 2;
    od.dim_up = m->hdev.dim_up;
    od.list_up = m->hdev.sector ? m->hdev.list_up : nullptr;
    od.list_dn = m->hdev.sector ? m->hdev.list_dn : nullptr;
  }
  double* partials = ws.partials.as<double>();
  const double ns = p->n_s > 0 ? p->n_s : (double)m->n_sites;
  const double inv_ns = 1.0 / ns;

  Timer tm;
  HPHI_CUDA_TRY(cudaEventCreate(&tm.a));
  HPHI_CUDA_TRY(cudaEventCreate(&tm.b));
  if (!p->psi0) {
    if ((s = hphi::launch_random(ws.vecA.p, m->dim * nvec, cplx, prec == HPHI_FP64, p->seed, st)).code) return s;
  }
  HPHI_CUDA_TRY(cudaEventRecord(tm.a, st));
  // profiled runs launch eagerly on st with an event pair around every H v launch group
  // (events recorded inside a captured graph cannot be timed)
  const bool prof = p->profile != 0;
  std::vector<cudaEvent_t> ev(prof ? 2 * (size_t)K : 0, nullptr);
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (cudaEvent_t x : v)
        if (x) cudaEventDestroy(x);
    }
  } ev_guard{ev};
  for (auto& x : ev) HPHI_CUDA_TRY(cudaEventCreate(&x));
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaSuccess;
  if (prof) {
    cap = st;
  } else {
    HPHI_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return {HPHI_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e)};
    }
  }
  auto body = [&]() -> hphi::Status {
    hphi::Status q;
    if ((q = hphi::launch_tpq_init(prec, cplx, p->psi0, ws.vecA.p, m->dim, nvec, partials, vgrid, cap)).code) return q;
    if ((q = hphi::launch_tpq_init_fin(tq, nvec, partials, vgrid, cap)).code) return q;
    void* X = ws.vecA.p;
    void* Xn = ws.vecB.p;
    for (int k = 0; k < K; ++k) {
      hphi::FusedArgs fa;
      fa.out = Xn;
      fa.scal = tq.inv;
      fa.partials = partials;
      fa.l = p->l;
      fa.inv_ns = inv_ns;
      if (prof) HPHI_CUDA_TRY(cudaEventRecord(ev[2 * (size_t)k], cap));
      if ((q = hv_launch(m, prec, X, nullptr, nvec, hphi::Epi::kTpq, fa, grid, tscratch, cap)).code) return q;
      if (prof) HPHI_CUDA_TRY(cudaEventRecord(ev[2 * (size_t)k + 1], cap));
      if ((q = hphi::launch_tpq_fin(tq, k, nvec, inv_ns, p->l, partials, grid, cap)).code) return q;
      if (obs_every > 0 && k % obs_every == 0) {  // observables of psi_k, still held in X
        if ((q = hphi::launch_tpq_obs(prec, cplx, od, X, nvec, partials, vgrid, cap)).code) return q;
        if ((q = hphi::launch_tpq_obs_fin(tq, k, nvec, inv_ns, partials, vgrid, cap)).code) return q;
      }
      std::swap(X, Xn);
    }
    return {};
  };
  s = body();
  if (!prof) {
    e = cudaStreamEndCapture(cap, &graph);
    if (s.code == 0 && e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e)};
    if (s.code == 0) {
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)};
    }
    if (s.code == 0) {
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) s = {HPHI_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e)};
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
  }
  if (s.code) return s;
  HPHI_CUDA_TRY(cudaEventRecord(tm.b, st));
  std::vector<double> host((obs_every > 0 ? 6 : 3) * (size_t)K * nvec);
  HPHI_CUDA_TRY(cudaMemcpyAsync(host.data(), tq.u, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, st));
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  HPHI_CUDA_TRY(cudaEventElapsedTime(&ms, tm.a, tm.b));
  const size_t kn = (size_t)K * nvec;
  if (r->u) memcpy(r->u, host.data(), sizeof(double) * kn);
  if (r->h2) memcpy(r->h2, host.data() + kn, sizeof(double) * kn);
  if (r->norm) memcpy(r->norm, host.data() + 2 * kn, sizeof(double) * kn);
  if (r->beta) {
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < nvec; ++c) {
        const size_t o = (size_t)k * nvec + c;
        r->beta[o] = (2.0 * k / ns) / (p->l - host[o]);  // host[o] = u_k of start c
      }
  }
  if (r->spec_heat) {  // C / N_s = beta^2 (<H^2> - <H>^2) / N_s = beta^2 N_s (h2_k - u_k^2)
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < nvec; ++c) {
        const size_t o = (size_t)k * nvec + c;
        const double b = (2.0 * k / ns) / (p->l - host[o]);
        r->spec_heat[o] = b * b * ns * (host[kn + o] - host[o] * host[o]);
      }
  }
  int n_obs = 0;
  for (double* dst : {r->doublon, r->sz, r->sz2}) {
    const size_t src = (3 + (size_t)n_obs++) * kn;
    if (!dst) continue;
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < nvec; ++c) {
        const size_t o = (size_t)k * nvec + c;
        dst[o] = (obs_every > 0 && k % obs_every == 0) ? host[src + o] : NAN;
      }
  }
  r->device_ms = ms;
  const int n_meas = obs_every > 0 ? (K + obs_every - 1) / obs_every : 0;
  r->kernel_launches = (p->psi0 ? 0 : 1) + 2 + (1 + hv_kernels(m, prec, nvec, hphi::Epi::kTpq)) * K + 2 * n_meas;
  r->hv_ms = 0.f;
  r->hv_launches = prof ? K : 0;
  for (int k = 0; prof && k < K; ++k) {
    float t = 0.f;
    HPHI_CUDA_TRY(cudaEventElapsedTime(&t, ev[2 * (size_t)k], ev[2 * (size_t)k + 1]));
    r->hv_ms += t;
  }
  return {};
}

// Inverse iteration of section 3.4.1 by CG, fp64.  x (the caller's vector) is b of the
// first solve and receives every normalised iterate; y, r, p, q are the four extra vectors.
hphi::Status invit_impl(hphi_model* m, const hphi_invit_params* p, void* xv, hphi_invit_result* r, cudaStream_t st) {
  const bool cplx = m->cplx_model;
  const int64_t n = m->dim * (cplx ? 2 : 1);
  const size_t vb = sizeof(double) * (size_t)n;
  Workspace& ws = m->ws;
  hphi::Status s;
  for (DBuf* b : {&ws.vecA, &ws.vecB, &ws.cgp, &ws.cgq})
    if ((s = b->ensure(vb)).code) return s;
  void* scratch = nullptr;
  const size_t need = hv_scratch_bytes(m, HPHI_FP64, 1, hphi::Epi::kStore);
  if (need && m->kind == HPHI_SPIN_HALF) {
    scratch = optional_scratch(m, need);
  } else if (need) {
    if ((s = ws.work.ensure(need)).code) return s;
    scratch = ws.work.p;
  }
  const int grid = hv_grid_for(m, 1, HPHI_FP64, hphi::Epi::kStore);
  const int vgrid = launch_grid(n);
  if ((s = ws.partials.ensure(sizeof(double) * (size_t)vgrid * hphi::kMaxRedQ)).code) return s;
  if ((s = ws.scal.ensure(sizeof(double) * 18)).code) return s;
  hphi::CgDev cg;
  cg.s = ws.scal.as<double>();
  cg.done = reinterpret_cast<int*>(cg.s + 16);
  cg.steps = cg.done + 1;
  double* x = static_cast<double*>(xv);
  double* y = ws.vecA.as<double>();
  double* rr = ws.vecB.as<double>();
  double* pp = ws.cgp.as<double>();
  double* q = ws.cgq.as<double>();
  double* partials = ws.partials.as<double>();
  const double delta = p->shift > 0 ? p->shift : 1e-4 * std::max(1.0, std::fabs(p->energy));
  const double tol = p->cg_tol > 0 ? p->cg_tol : 1e-12;
  double host_s[18] = {0.0};
  host_s[4] = delta - p->energy;
  host_s[5] = tol * tol;
  Timer tm;
  HPHI_CUDA_TRY(cudaEventCreate(&tm.a));
  HPHI_CUDA_TRY(cudaEventCreate(&tm.b));
  HPHI_CUDA_TRY(cudaEventRecord(tm.a, st));
  HPHI_CUDA_TRY(cudaMemcpyAsync(cg.s, host_s, sizeof(host_s), cudaMemcpyHostToDevice, st));
  int launches = 0;
  hphi::FusedArgs plain;  // H v without a flag
  hphi::FusedArgs flagged;
  flagged.done = cg.done;  // H p of a solve that has converged is skipped
  const int hvk = hv_kernels(m, HPHI_FP64, 1, hphi::Epi::kStore);
  int done_h = 0;
  for (int outer = 0; outer < p->outer; ++outer) {
    HPHI_CUDA_TRY(cudaMemsetAsync(cg.done, 0, sizeof(int), st));
    // start: y = b, r = b - A b, p = r
    plain.out = q;
    if ((s = hv_launch(m, HPHI_FP64, x, q, 1, hphi::Epi::kStore, plain, grid, scratch, st)).code) return s;
    if ((s = hphi::launch_cg_shift(cg, x, q, n, partials, vgrid, st)).code) return s;
    if ((s = hphi::launch_cg_update(cg, 0, x, y, rr, pp, q, n, partials, vgrid, st)).code) return s;
    if ((s = hphi::launch_cg_fin(cg, 0, partials, vgrid, st)).code) return s;
    launches += hvk + 3;
    for (int it = 0; it < p->max_cg; ++it) {
      flagged.out = q;
      if ((s = hv_launch(m, HPHI_FP64, pp, q, 1, hphi::Epi::kStore, flagged, grid, scratch, st)).code) return s;
      if ((s = hphi::launch_cg_shift(cg, pp, q, n, partials, vgrid, st)).code) return s;
      if ((s = hphi::launch_cg_fin(cg, 1, partials, vgrid, st)).code) return s;
      if ((s = hphi::launch_cg_update(cg, 1, nullptr, y, rr, pp, q, n, partials, vgrid, st)).code) return s;
      if ((s = hphi::launch_cg_fin(cg, 2, partials, vgrid, st)).code) return s;
      if ((s = hphi::launch_cg_dir(cg, rr, pp, n, vgrid, st)).code) return s;
      launches += hvk + 5;
      if (it % 16 == 15) {  // look at the flag now and then; the kernels skip work once it is set
        HPHI_CUDA_TRY(cudaMemcpyAsync(&done_h, cg.done, sizeof(int), cudaMemcpyDeviceToHost, st));
        HPHI_CUDA_TRY(cudaStreamSynchronize(st));
        if (done_h) break;
      }
    }
    // x = y / |y|
    if ((s = hphi::launch_cg_norm(cg, 0, y, x, n, partials, vgrid, st)).code) return s;
    if ((s = hphi::launch_cg_fin(cg, 3, partials, vgrid, st)).code) return s;
    if ((s = hphi::launch_cg_norm(cg, 1, y, x, n, partials, vgrid, st)).code) return s;
    launches += 3;
  }
  // Rayleigh quotient, variance and residual of the final unit vector
  plain.out = q;
  if ((s = hv_launch(m, HPHI_FP64, x, q, 1, hphi::Epi::kStore, plain, grid, scratch, st)).code) return s;
  if ((s = hphi::launch_cg_rq(cg, 0, x, q, n, partials, vgrid, st)).code) return s;
  if ((s = hphi::launch_cg_fin(cg, 4, partials, vgrid, st)).code) return s;
  if ((s = hphi::launch_cg_rq(cg, 1, x, q, n, partials, vgrid, st)).code) return s;
  if ((s = hphi::launch_cg_fin(cg, 5, partials, vgrid, st)).code) return s;
  launches += hvk + 4;
  HPHI_CUDA_TRY(cudaEventRecord(tm.b, st));
  HPHI_CUDA_TRY(cudaMemcpyAsync(host_s, cg.s, sizeof(host_s), cudaMemcpyDeviceToHost, st));
  HPHI_CUDA_TRY(cudaStreamSynchronize(st));
  float ms = 0.f;
  HPHI_CUDA_TRY(cudaEventElapsedTime(&ms, tm.a, tm.b));
  r->e = host_s[6];
  r->residual = host_s[7];
  r->variance = host_s[8];
  r->cg_steps = reinterpret_cast<const int*>(host_s + 16)[1];
  r->device_ms = ms;
  r->kernel_launches = launches;
  return {};
}

}  // namespace

extern "C" {

int hphi_lanczos_run(hphi_model* m, const hphi_lanczos_params* p, hphi_lanczos_result* r, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!p || !r) return fail(m, HPHI_ERR_INVALID_ARG, "params/result NULL");
  if (p->steps < 1 || p->steps > 4096 || (p->prec != HPHI_FP64 && p->prec != HPHI_FP32) || p->n_eig < 1 || p->n_eig > 8)
    return fail(m, HPHI_ERR_INVALID_ARG, "lanczos: steps in 1..4096, prec FP64/FP32, n_eig in 1..8");
  hphi::Status s = lanczos_impl(m, p, r, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_lanczos_run_sectors(hphi_model* m, const int* n_up_list, int n_sectors, const hphi_lanczos_params* p,
                             hphi_lanczos_result* results, void* stream) {
  if (!m) return HPHI_ERR_INVALID_ARG;
  if (m->kind != HPHI_SPIN_HALF) return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: spin models only");
  if (!n_up_list || !p || !results || n_sectors < 1 || n_sectors > 64)
    return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: 1..64 sectors, non-NULL lists");
  if (p->steps < 1 || p->steps > 4096 || (p->prec != HPHI_FP64 && p->prec != HPHI_FP32) || p->n_eig < 1 || p->n_eig > 8)
    return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: steps in 1..4096, prec FP64/FP32, n_eig in 1..8");
  if (p->v0) return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: start vectors are seeded per sector (v0 must be NULL)");
  for (int i = 0; i < n_sectors; ++i) {
    if (n_up_list[i] < 0 || n_up_list[i] > m->n_sites || m->n_sites > 40)
      return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: n_up out of range (or more than 40 sites)");
    for (int j = 0; j < i; ++j)
      if (n_up_list[j] == n_up_list[i]) return fail(m, HPHI_ERR_INVALID_ARG, "lanczos_run_sectors: repeated sector");
  }
  hphi::Status s = lanczos_sectors_impl(m, n_up_list, n_sectors, p, results, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_inverse_iteration(hphi_model* m, const hphi_invit_params* p, void* x, hphi_invit_result* r, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!p || !r || !x) return fail(m, HPHI_ERR_INVALID_ARG, "inverse_iteration: params, result and x must be non-NULL");
  if (p->outer < 1 || p->outer > 64 || p->max_cg < 1 || p->max_cg > 100000 || !isfinite(p->energy) ||
      !(p->shift >= 0.0) || !(p->cg_tol >= 0.0))
    return fail(m, HPHI_ERR_INVALID_ARG, "inverse_iteration: outer 1..64, max_cg 1..100000, finite energy, shift and tol >= 0");
  hphi::Status s = invit_impl(m, p, x, r, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

int hphi_tpq_run(hphi_model* m, const hphi_tpq_params* p, hphi_tpq_result* r, void* stream) {
  int rc = check_built(m);
  if (rc) return rc;
  if (!p || !r) return fail(m, HPHI_ERR_INVALID_ARG, "params/result NULL");
  const int nv = p->n_starts;
  if (nv < 1 || nv > hphi::kMaxNvec || (nv & (nv - 1)) != 0)
    return fail(m, HPHI_ERR_INVALID_ARG, "tpq: n_starts must be a power of two in 1..256");
  if (p->steps < 1 || (p->prec != HPHI_FP64 && p->prec != HPHI_FP32) || !isfinite(p->l) || p->obs_every < 0)
    return fail(m, HPHI_ERR_INVALID_ARG, "tpq: bad steps, precision, l or obs_every");
  hphi::Status s = tpq_impl(m, p, r, (cudaStream_t)stream);
  return s.code ? fail(m, s) : HPHI_OK;
}

}  // extern "C"
