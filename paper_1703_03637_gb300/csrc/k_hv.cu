// Matrix-free H v over the bit-string basis (section 3.3), fused with the Lanczos
// (section 3.4) and mTPQ (section 3.5) vector updates and their reductions.
//
// Gather form: each thread owns one output element (row r, vector c) and sums
//     w[r] = diag(s_r) v[r] + sum_patterns coef * phase * v[rank(s_r ^ mask)],
// so every write is coalesced and no atomics are needed.  The diagonal is an integer bit
// count per coefficient class (popcounts), then one multiply-add per class.  Off-diagonal
// patterns that share a coefficient up to a phase in {+1, +i, -1, -i} are summed first
// and multiplied once per class.  Fermion signs are popcount parities of the bits between
// the two hopping sites.  Reductions for the fused steps are per-thread partial sums
// (fp64, or error-free fp32 TwoSum chunks flushed to fp64) reduced per CTA in a fixed
// order and written to a partials array, so results are bit-reproducible run to run.
#include "basis.cuh"
#include "common.cuh"
#include "reduce.cuh"

namespace hphi {

namespace {

// Per-column CTA reduction in a fixed tree order; partials[(block * nvec + c) * kMaxRedQ + q].
template <bool F64>
__device__ void block_finish(const Red<F64>& red, int nq, int nvec, double* __restrict__ partials, double* sm) {
  const int tid = threadIdx.x;
  for (int q = 0; q < nq; ++q) sm[q * kThreads + tid] = red.get(q);
  __syncthreads();
  for (int off = kThreads / 2; off >= nvec; off >>= 1) {
    if (tid < off) {
      for (int q = 0; q < nq; ++q) sm[q * kThreads + tid] += sm[q * kThreads + tid + off];
    }
    __syncthreads();
  }
  if (tid < nvec) {
    for (int q = 0; q < nq; ++q) partials[((size_t)blockIdx.x * nvec + tid) * kMaxRedQ + q] = sm[q * kThreads + tid];
  }
}

// ------------------------------------------------------------------ element access
template <class S>
__device__ __forceinline__ void ld(const S* __restrict__ p, int64_t i, typename Traits<S>::R& re,
                                   typename Traits<S>::R& im) {
  if constexpr (Traits<S>::kCplx) {
    const S x = p[i];
    re = x.x;
    im = x.y;
  } else {
    re = p[i];
    im = 0;
  }
}

template <class S>
__device__ __forceinline__ void st(S* __restrict__ p, int64_t i, typename Traits<S>::R re, typename Traits<S>::R im) {
  if constexpr (Traits<S>::kCplx) {
    S x;
    x.x = re;
    x.y = im;
    p[i] = x;
  } else {
    p[i] = re;
  }
}

// acc += phase(code) * x, code: 1 (+1), 2 (+i), 3 (-1), 4 (-i)
template <class R>
__device__ __forceinline__ void acc_phase(int code, R xr, R xi, R& ar, R& ai) {
  switch (code) {
    case 1: ar += xr; ai += xi; break;
    case 2: ar -= xi; ai += xr; break;
    case 3: ar -= xr; ai -= xi; break;
    default: ar += xi; ai -= xr; break;
  }
}

// ------------------------------------------------------------------ epilogues
struct EpiScalars {
  double c1, c2;  // Lanczos pass 1
};

template <class S, Epi E>
__device__ __forceinline__ void epilogue(int64_t idx, int c, typename Traits<S>::R sr, typename Traits<S>::R si,
                                         typename Traits<S>::R hr, typename Traits<S>::R hi, S* __restrict__ w,
                                         const FusedArgs& fa, const EpiScalars& es, const double* s_inv,
                                         Red<Traits<S>::kF64>& red) {
  using R = typename Traits<S>::R;
  constexpr bool C = Traits<S>::kCplx;
  if constexpr (E == Epi::kStore) {
    st<S>(w, idx, hr, hi);
  } else if constexpr (E == Epi::kLanczos1) {
    // P <- sigma_k * (H C) - beta_k sigma_{k-1} * P ;  partial <C, H C>
    S* P = reinterpret_cast<S*>(fa.out);
    R pr, pi;
    ld<S>(P, idx, pr, pi);
    const R c1 = (R)es.c1, c2 = (R)es.c2;
    st<S>(P, idx, c1 * hr - c2 * pr, c1 * hi - c2 * pi);
    red.add(0, sr, hr);
    if constexpr (C) red.add(0, si, hi);
    red.tick();
  } else if constexpr (E == Epi::kTpq) {
    // X_{k+1} = (l X_k - H X_k / N_s) / |X_k| ; partials <X, HX>, |HX|^2, |X_{k+1}|^2
    S* Xn = reinterpret_cast<S*>(fa.out);
    const R inv = (R)s_inv[c], l = (R)fa.l, ins = (R)fa.inv_ns;
    const R nr = inv * (l * sr - hr * ins);
    const R ni = inv * (l * si - hi * ins);
    st<S>(Xn, idx, nr, ni);
    red.add(0, sr, hr);
    red.add(1, hr, hr);
    red.add(2, nr, nr);
    if constexpr (C) {
      red.add(0, si, hi);
      red.add(1, hi, hi);
      red.add(2, ni, ni);
    }
    red.tick();
  } else {  // kRefine: Hx stored; partials <x, Hx>, <x, x>, <Hx, Hx>
    st<S>(reinterpret_cast<S*>(fa.out), idx, hr, hi);
    red.add(0, sr, hr);
    red.add(1, sr, sr);
    red.add(2, hr, hr);
    if constexpr (C) {
      red.add(0, si, hi);
      red.add(1, si, si);
      red.add(2, hi, hi);
    }
    red.tick();
  }
}

template <Epi E> __host__ __device__ constexpr int n_red() {
  return E == Epi::kStore ? 0 : (E == Epi::kLanczos1 ? 1 : 3);
}

// ------------------------------------------------------------------ spin kernel
template <class S, Epi E>
__global__ void __launch_bounds__(kThreads) k_hv_spin(const SpinDev md, const S* __restrict__ v, S* __restrict__ w,
                                                      int nvec, int lg_nvec, FusedArgs fa) {
  using R = typename Traits<S>::R;
  constexpr bool C = Traits<S>::kCplx;
  constexpr bool F64 = Traits<S>::kF64;
  __shared__ SpinEntry s_ent[kMaxSpinEntries];
  __shared__ double2 s_cls[kMaxClasses];
  __shared__ LinGroup s_lin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  __shared__ double s_inv[kMaxNvec];
  __shared__ uint64_t s_hi[2];
  __shared__ double s_red[(E == Epi::kStore) ? 1 : kThreads * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  for (int k = tid; k < md.n_entries; k += kThreads) s_ent[k] = md.entries[k];
  for (int k = tid; k < md.n_classes; k += kThreads) s_cls[k] = md.cls_coef[k];
  for (int k = tid; k < md.n_lin; k += kThreads) s_lin[k] = md.lin[k];
  for (int k = tid; k < md.n_pairs; k += kThreads) s_pair[k] = md.pairs[k];
  for (int k = tid; k < md.n_pair_groups; k += kThreads) s_pcoef[k] = md.pair_coef[k];
  if constexpr (E == Epi::kTpq) {
    for (int k = tid; k < nvec; k += kThreads) s_inv[k] = fa.scal[k];
  }
  EpiScalars es{0.0, 0.0};
  if constexpr (E == Epi::kLanczos1) {
    es.c1 = fa.scal[0];
    es.c2 = fa.scal[1];
  }
  __syncthreads();

  Red<F64> red;
  red.zero();
  const int64_t total = md.dim * (int64_t)nvec;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  const uint64_t hmax = md.sector ? ((1ull << md.t.H) - 1ull) : 0ull;
  const int n_ent = md.n_entries;

  for (int64_t base = (int64_t)blockIdx.x * kThreads; base < total; base += stride) {
    const int64_t idx = base + tid;
    const bool act = idx < total;
    int64_t r;
    int c;
    if (lg_nvec >= 0) {
      r = idx >> lg_nvec;
      c = (int)(idx & (nvec - 1));
    } else {
      r = idx / nvec;
      c = (int)(idx - r * nvec);
    }
    uint64_t s = (uint64_t)r;
    if (md.sector) {
      __syncthreads();
      if (tid == 0) s_hi[0] = sector_find_hi(md.t, (uint64_t)(base / nvec), 0, hmax);
      if (tid == 1) {
        const int64_t last = (base + kThreads < total ? base + kThreads : total) - 1;
        s_hi[1] = sector_find_hi(md.t, (uint64_t)(last / nvec), 0, hmax);
      }
      __syncthreads();
      if (act) s = sector_state_in(md.t, (uint64_t)r, sector_find_hi(md.t, (uint64_t)r, s_hi[0], s_hi[1]));
    }
    if (!act) continue;

    // diagonal: integer bit counts per coefficient class
    R d = (R)md.c0;
    for (int g = 0; g < md.n_lin; ++g) d += (R)s_lin[g].coef * (R)__popcll(s & s_lin[g].mask);
    if (md.n_pairs) {
      int grp = s_pair[0].grp, cnt = 0;
      for (int p = 0; p < md.n_pairs; ++p) {
        const PairEntry pe = s_pair[p];
        if (pe.grp != grp) {
          d += (R)s_pcoef[grp] * (R)cnt;
          cnt = 0;
          grp = pe.grp;
        }
        cnt += (int)((s >> pe.i) & (s >> pe.j) & 1ull);
      }
      d += (R)s_pcoef[grp] * (R)cnt;
    }
    R sr, si;
    ld<S>(v, idx, sr, si);
    R hr = d * sr, hi = d * si;

    // off-diagonal XOR patterns, summed per coefficient class
    R ar = 0, ai = 0;
    int cur = n_ent ? s_ent[0].cls : 0;
    for (int e = 0; e < n_ent; ++e) {
      const SpinEntry en = s_ent[e];
      if (en.cls != cur) {
        const double2 cc = s_cls[cur];
        if constexpr (C) {
          hr += (R)cc.x * ar - (R)cc.y * ai;
          hi += (R)cc.x * ai + (R)cc.y * ar;
        } else {
          hr += (R)cc.x * ar;
        }
        ar = 0;
        ai = 0;
        cur = en.cls;
      }
      const int sel = (int)((s >> en.i) & 1ull) | ((int)((s >> en.j) & 1ull) << 1);
      const int code = (en.phases >> (3 * sel)) & 7;
      if (!code) continue;
      const uint64_t s2 = s ^ en.mask;
      const uint64_t r2 = md.sector ? sector_rank(md.t, s2) : s2;
      R xr, xi;
      ld<S>(v, (int64_t)r2 * nvec + c, xr, xi);
      if constexpr (C) {
        acc_phase<R>(code, xr, xi, ar, ai);
      } else {
        ar += (code == 1) ? xr : -xr;
      }
    }
    if (n_ent) {
      const double2 cc = s_cls[cur];
      if constexpr (C) {
        hr += (R)cc.x * ar - (R)cc.y * ai;
        hi += (R)cc.x * ai + (R)cc.y * ar;
      } else {
        hr += (R)cc.x * ar;
      }
    }
    epilogue<S, E>(idx, c, sr, si, hr, hi, w, fa, es, s_inv, red);
  }
  if constexpr (E != Epi::kStore) block_finish<F64>(red, n_red<E>(), nvec, fa.partials, s_red);
}

// ------------------------------------------------------------------ Hubbard kernel
template <class S, Epi E>
__global__ void __launch_bounds__(kThreads) k_hv_hub(const HubDev md, const S* __restrict__ v, S* __restrict__ w,
                                                     int nvec, int lg_nvec, FusedArgs fa) {
  using R = typename Traits<S>::R;
  constexpr bool C = Traits<S>::kCplx;
  constexpr bool F64 = Traits<S>::kF64;
  __shared__ HopEntry s_hop[kMaxHops];
  __shared__ double2 s_cls[kMaxClasses];
  __shared__ LinGroup s_ulin[kMaxLin];
  __shared__ LinGroup s_mlin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  __shared__ double s_inv[kMaxNvec];
  __shared__ double s_red[(E == Epi::kStore) ? 1 : kThreads * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  const int n_hops = md.n_up_hops + md.n_dn_hops;
  for (int k = tid; k < n_hops; k += kThreads) s_hop[k] = md.hops[k];
  for (int k = tid; k < md.n_classes; k += kThreads) s_cls[k] = md.cls_coef[k];
  for (int k = tid; k < md.n_ulin; k += kThreads) s_ulin[k] = md.ulin[k];
  for (int k = tid; k < md.n_mulin; k += kThreads) s_mlin[k] = md.mulin[k];
  for (int k = tid; k < md.n_pairs; k += kThreads) s_pair[k] = md.pairs[k];
  for (int k = tid; k < md.n_pair_groups; k += kThreads) s_pcoef[k] = md.pair_coef[k];
  if constexpr (E == Epi::kTpq) {
    for (int k = tid; k < nvec; k += kThreads) s_inv[k] = fa.scal[k];
  }
  EpiScalars es{0.0, 0.0};
  if constexpr (E == Epi::kLanczos1) {
    es.c1 = fa.scal[0];
    es.c2 = fa.scal[1];
  }
  __syncthreads();

  Red<F64> red;
  red.zero();
  const int64_t row_elems = md.dim_up * (int64_t)nvec;
  const int64_t nchunk = (row_elems + kThreads - 1) / kThreads;
  const int64_t n_items = nchunk * md.dim_dn;

  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t d = item / nchunk;
    const int64_t e = (item - d * nchunk) * kThreads + tid;
    if (e >= row_elems) continue;
    int64_t u;
    int c;
    if (lg_nvec >= 0) {
      u = e >> lg_nvec;
      c = (int)(e & (nvec - 1));
    } else {
      u = e / nvec;
      c = (int)(e - u * nvec);
    }
    const uint32_t up = md.sector ? __ldg(md.list_up + u) : (uint32_t)u;
    const uint32_t dn = md.sector ? __ldg(md.list_dn + d) : (uint32_t)d;
    const int64_t row_base = d * md.dim_up;
    const int64_t idx = (row_base + u) * nvec + c;

    // diagonal
    R dg = (R)md.c0;
    for (int g = 0; g < md.n_ulin; ++g) dg += (R)s_ulin[g].coef * (R)__popc(up & dn & (uint32_t)s_ulin[g].mask);
    for (int g = 0; g < md.n_mulin; ++g) {
      const uint32_t m = (uint32_t)s_mlin[g].mask;
      dg += (R)s_mlin[g].coef * (R)(__popc(up & m) + __popc(dn & m));
    }
    if (md.n_pairs) {
      int grp = s_pair[0].grp, cnt = 0;
      for (int p = 0; p < md.n_pairs; ++p) {
        const PairEntry pe = s_pair[p];
        if (pe.grp != grp) {
          dg += (R)s_pcoef[grp] * (R)cnt;
          cnt = 0;
          grp = pe.grp;
        }
        const int ni = (int)((up >> pe.i) & 1u) + (int)((dn >> pe.i) & 1u);
        const int nj = (int)((up >> pe.j) & 1u) + (int)((dn >> pe.j) & 1u);
        cnt += ni * nj;
      }
      dg += (R)s_pcoef[grp] * (R)cnt;
    }
    R sr, si;
    ld<S>(v, idx, sr, si);
    R hr = dg * sr, hi = dg * si;

    // hops: (i set, j empty) -> coef, (j set, i empty) -> conj(coef); sign from the bits between
    for (int part = 0; part < 2; ++part) {
      const int e0 = part ? md.n_up_hops : 0;
      const int e1 = part ? n_hops : md.n_up_hops;
      if (e0 == e1) continue;
      const uint32_t bits = part ? dn : up;
      R a_r = 0, a_i = 0, b_r = 0, b_i = 0;
      int cur = s_hop[e0].cls;
      for (int k = e0; k <= e1; ++k) {
        const bool last = (k == e1);
        if (last || s_hop[k].cls != cur) {
          const double2 cc = s_cls[cur];
          if constexpr (C) {
            // coef * a + conj(coef) * b
            hr += (R)cc.x * (a_r + b_r) - (R)cc.y * (a_i - b_i);
            hi += (R)cc.x * (a_i + b_i) + (R)cc.y * (a_r - b_r);
          } else {
            hr += (R)cc.x * a_r;
          }
          a_r = a_i = b_r = b_i = 0;
          if (last) break;
          cur = s_hop[k].cls;
        }
        const HopEntry h = s_hop[k];
        const uint32_t bi = (bits >> h.i) & 1u, bj = (bits >> h.j) & 1u;
        if (bi == bj) continue;
        const uint32_t b2 = bits ^ h.mask;
        const int64_t k2 = md.sector ? (int64_t)__ldg(md.rank + b2) : (int64_t)b2;
        const int64_t src = part ? ((k2 * md.dim_up + u) * nvec + c) : ((row_base + k2) * nvec + c);
        R xr, xi;
        ld<S>(v, src, xr, xi);
        const bool neg = (__popc(bits & h.between) & 1) != 0;
        if (neg) {
          xr = -xr;
          xi = -xi;
        }
        if constexpr (C) {
          if (bi) { a_r += xr; a_i += xi; }
          else { b_r += xr; b_i += xi; }
        } else {
          a_r += xr;
        }
      }
    }
    epilogue<S, E>(idx, c, sr, si, hr, hi, w, fa, es, s_inv, red);
  }
  if constexpr (E != Epi::kStore) block_finish<F64>(red, n_red<E>(), nvec, fa.partials, s_red);
}

template <class S, Epi E>
Status launch_t(bool hub, const void* md, const void* v, void* w, int nvec, const FusedArgs& fa, int grid,
                cudaStream_t st) {
  int lg = -1;
  if ((nvec & (nvec - 1)) == 0) {
    lg = 0;
    while ((1 << lg) < nvec) ++lg;
  }
  if (hub) {
    k_hv_hub<S, E><<<grid, kThreads, 0, st>>>(*reinterpret_cast<const HubDev*>(md), reinterpret_cast<const S*>(v),
                                             reinterpret_cast<S*>(w), nvec, lg, fa);
  } else {
    k_hv_spin<S, E><<<grid, kThreads, 0, st>>>(*reinterpret_cast<const SpinDev*>(md), reinterpret_cast<const S*>(v),
                                              reinterpret_cast<S*>(w), nvec, lg, fa);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

template <Epi E>
Status launch_e(bool hub, const void* md, int prec, bool cplx, const void* v, void* w, int nvec, const FusedArgs& fa,
                int grid, cudaStream_t st) {
  if (prec == HPHI_FP64) {
    return cplx ? launch_t<double2, E>(hub, md, v, w, nvec, fa, grid, st)
                : launch_t<double, E>(hub, md, v, w, nvec, fa, grid, st);
  }
  return cplx ? launch_t<float2, E>(hub, md, v, w, nvec, fa, grid, st)
              : launch_t<float, E>(hub, md, v, w, nvec, fa, grid, st);
}

}  // namespace

int hv_grid(int nvec) {
  (void)nvec;
  return num_sms() * 4;
}

Status launch_hv(bool hubbard, const void* md, int prec, bool cplx, const void* v, void* w, int nvec, Epi epi,
                 const FusedArgs& fa, int grid, cudaStream_t st) {
  switch (epi) {
    case Epi::kStore: return launch_e<Epi::kStore>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, st);
    case Epi::kLanczos1: return launch_e<Epi::kLanczos1>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, st);
    case Epi::kTpq: return launch_e<Epi::kTpq>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, st);
    case Epi::kRefine:
      if (prec != HPHI_FP64) return {HPHI_ERR_INVALID_ARG, "refinement runs in fp64"};
      return launch_e<Epi::kRefine>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, st);
  }
  return {HPHI_ERR_INVALID_ARG, "unknown epilogue"};
}

}  // namespace hphi
