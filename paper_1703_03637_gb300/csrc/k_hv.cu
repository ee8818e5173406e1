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
#include <type_traits>

#include "basis.cuh"
#include "common.cuh"
#include "reduce.cuh"
#include "epilogue.cuh"

namespace hphi {

namespace {

// ------------------------------------------------------------------ spin kernel
// One thread per output element.  Patterns are visited in unrolled batches of kBatch:
// the active test, rank and address of every pattern in a batch are computed first and
// the batch's loads are issued together (predicated on the phase code), so each thread
// keeps kBatch gathers in flight instead of one.  Class boundaries are the same for every
// thread (patterns are sorted by class), so class flushes never diverge.
constexpr int kBatch = 8;

//
// QT (fp64): the gathers read the input quantised to 64-bit integers, one scale per vector
// column (q = round(x 2^(1078 - E_c)), |q| < 2^56), so every class sum of at most 127 terms
// is an exact integer sum (two integer instructions a term instead of the per-term
// alignment of the fixed-point accumulator), converted to fp64 once per class.
template <class S, Epi E, bool QT = false>
__global__ void __launch_bounds__(kThreads) k_hv_spin(const SpinDev md, const S* __restrict__ v, S* __restrict__ w,
                                                      int nvec, int lg_nvec, FusedArgs fa,
                                                      const long long* __restrict__ Q, const int* __restrict__ Ec) {
  using R = typename Traits<S>::R;
  static_assert(!QT || Traits<S>::kF64, "quantised gathers are an fp64 path");
  using A = std::conditional_t<QT, IntAcc, typename SumAcc<R>::T>;
  using T = std::conditional_t<QT, long long, R>;  // gathered scalar
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
  __shared__ int64_t s_item;
  const uint64_t hmax = md.sector ? ((1ull << md.t.H) - 1ull) : 0ull;
  const int n_ent = md.n_entries;

  // plain H v: chunks of kThreads elements are handed out in order from a counter, so
  // resident CTAs stay on neighbouring rows and share the rows they gather through L2.
  // Fused steps keep the static assignment (chunk = CTA + k * grid): each CTA's partial sums
  // then cover the same elements in the same order every run (bit-reproducible reductions).
  constexpr bool kDyn = (E == Epi::kStore);
  int64_t next = blockIdx.x;
  for (;;) {
    if constexpr (kDyn) {
      __syncthreads();
      if (tid == 0) s_item = (int64_t)atomicAdd(md.counter, 1ull);
      __syncthreads();
      next = s_item;
    }
    const int64_t base = next * kThreads;
    if constexpr (!kDyn) next += gridDim.x;
    if (base >= total) break;
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
    const int eoff = QT ? Ec[c] - 1078 : 0;

    A ar, ai;
    ar.zero();
    ai.zero();
    int cur = n_ent ? s_ent[0].cls : 0;
    for (int e0 = 0; e0 < n_ent; e0 += kBatch) {
      T xr[kBatch], xi[kBatch];
      int code[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = e0 + j;
        code[j] = 0;
        xr[j] = 0;
        xi[j] = 0;
        if (k < n_ent) {
          const SpinEntry en = s_ent[k];
          const int sel = (int)((s >> en.i) & 1ull) | ((int)((s >> en.j) & 1ull) << 1);
          code[j] = (en.phases >> (3 * sel)) & 7;
          if (code[j]) {
            const uint64_t s2 = s ^ en.mask;
            const uint64_t r2 = md.sector ? sector_rank(md.t, s2) : s2;
            if constexpr (QT) {
              const int64_t o = (int64_t)r2 * nvec + c;
              if constexpr (C) {
                const longlong2 t = __ldg(reinterpret_cast<const longlong2*>(Q) + o);
                xr[j] = t.x;
                xi[j] = t.y;
              } else {
                xr[j] = __ldg(Q + o);
              }
            } else {
              ld<S>(v, (int64_t)r2 * nvec + c, xr[j], xi[j]);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = e0 + j;
        if (k < n_ent) {
          const int cls = s_ent[k].cls;
          if (cls != cur) {
            const double2 cc = s_cls[cur];
            R vr, vi;
            if constexpr (QT) {
              vr = fix_to_double(ar.value(), eoff);
              vi = C ? fix_to_double(ai.value(), eoff) : 0.0;
            } else {
              vr = (R)ar.value();
              vi = (R)ai.value();
            }
            if constexpr (C) {
              hr += (R)cc.x * vr - (R)cc.y * vi;
              hi += (R)cc.x * vi + (R)cc.y * vr;
            } else {
              hr += (R)cc.x * vr;
            }
            ar.zero();
            ai.zero();
            cur = cls;
          }
          if (code[j]) {
            if constexpr (C) acc_phase<A, T>(code[j], xr[j], xi[j], ar, ai);
            else ar.add(xr[j], code[j] != 1);
          }
        }
      }
    }
    if (n_ent) {
      const double2 cc = s_cls[cur];
      R vr, vi;
      if constexpr (QT) {
        vr = fix_to_double(ar.value(), eoff);
        vi = C ? fix_to_double(ai.value(), eoff) : 0.0;
      } else {
        vr = (R)ar.value();
        vi = (R)ai.value();
      }
      if constexpr (C) {
        hr += (R)cc.x * vr - (R)cc.y * vi;
        hi += (R)cc.x * vi + (R)cc.y * vr;
      } else {
        hr += (R)cc.x * vr;
      }
    }
    epilogue<S, E>(idx, c, sr, si, hr, hi, w, fa, es, s_inv, red);
  }
  if constexpr (E != Epi::kStore) block_finish<F64>(red, n_red<E>(), nvec, fa.partials, s_red);
}

// ------------------------------------------------------------------ Hubbard kernel
// Work item = (down-spin row d, chunk of kThreads consecutive (up, vector) elements).
// Down-spin hops depend only on d, so warp 0 builds the row's compacted neighbour list
// (source row, sign, direction, class) in shared memory once per item and every thread
// walks it uniformly in batches of kBatch coalesced loads.  Up-spin hops depend on each
// thread's up configuration and are visited in predicated batches of kBatch.
template <class S, Epi E>
__global__ void __launch_bounds__(kThreads) k_hv_hub(const HubDev md, const S* __restrict__ v, S* __restrict__ w,
                                                     int nvec, int lg_nvec, FusedArgs fa) {
  using R = typename Traits<S>::R;
  using A = typename SumAcc<R>::T;
  constexpr bool C = Traits<S>::kCplx;
  constexpr bool F64 = Traits<S>::kF64;
  __shared__ HopEntry s_hop[kMaxHops];
  __shared__ double2 s_cls[kMaxClasses];
  __shared__ LinGroup s_ulin[kMaxLin];
  __shared__ LinGroup s_mlin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  __shared__ double s_inv[kMaxNvec];
  __shared__ int64_t s_dl_src[kMaxHops];   // source element offset of neighbour row d'
  __shared__ uint32_t s_dl_meta[kMaxHops];  // bit 0 negative sign, bit 1 direction b, class << 2
  __shared__ int s_dl_n;
  __shared__ double s_red[(E == Epi::kStore) ? 1 : kThreads * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  const int n_up = md.n_up_hops, n_dn = md.n_dn_hops;
  const int n_hops = n_up + n_dn;
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

  __shared__ int64_t s_item;
  constexpr bool kDyn = (E == Epi::kStore);  // see k_hv_spin: fused steps stay static
  int64_t next = blockIdx.x;
  for (;;) {
    if constexpr (kDyn) {
      __syncthreads();
      if (tid == 0) s_item = (int64_t)atomicAdd(md.counter, 1ull);
      __syncthreads();
      next = s_item;
    }
    const int64_t item = next;
    if constexpr (!kDyn) next += gridDim.x;
    if (item >= n_items) break;
    const int64_t d = item / nchunk;
    const int64_t e = (item - d * nchunk) * kThreads + tid;
    const uint32_t dn = md.sector ? __ldg(md.list_dn + d) : (uint32_t)d;
    // neighbour list of row d (ordered, so classes stay grouped)
    __syncthreads();
    if (tid < 32) {
      int cnt = 0;
      for (int k0 = 0; k0 < n_dn; k0 += 32) {
        const int k = k0 + tid;
        bool on = false;
        int64_t src = 0;
        uint32_t meta = 0;
        if (k < n_dn) {
          const HopEntry h = s_hop[n_up + k];
          const uint32_t bi = (dn >> h.i) & 1u, bj = (dn >> h.j) & 1u;
          if (bi != bj) {
            on = true;
            const uint32_t b2 = dn ^ h.mask;
            const int64_t d2 = md.sector ? (int64_t)__ldg(md.rank + b2) : (int64_t)b2;
            src = d2 * md.dim_up * nvec;
            meta = (uint32_t)(__popc(dn & h.between) & 1) | ((bi ? 0u : 1u) << 1) | ((uint32_t)h.cls << 2);
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (on) {
          const int pos = cnt + __popc(bal & ((1u << tid) - 1u));
          s_dl_src[pos] = src;
          s_dl_meta[pos] = meta;
        }
        cnt += __popc(bal);
      }
      if (tid == 0) s_dl_n = cnt;
    }
    __syncthreads();
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

    // coef * a + conj(coef) * b for one class
    A ar, ai, br, bi_;
    ar.zero(); ai.zero(); br.zero(); bi_.zero();
    auto flush = [&](int cls) {
      const double2 cc = s_cls[cls];
      if constexpr (C) {
        const R a_r = (R)ar.value(), a_i = (R)ai.value(), b_r = (R)br.value(), b_i = (R)bi_.value();
        hr += (R)cc.x * (a_r + b_r) - (R)cc.y * (a_i - b_i);
        hi += (R)cc.x * (a_i + b_i) + (R)cc.y * (a_r - b_r);
        br.zero();
        bi_.zero();
      } else {
        hr += (R)cc.x * (R)ar.value();
      }
      ar.zero();
      ai.zero();
    };

    // up hops: predicated batches
    int cur = n_up ? s_hop[0].cls : 0;
    for (int k0 = 0; k0 < n_up; k0 += kBatch) {
      R xr[kBatch], xi[kBatch];
      uint32_t fl[kBatch];  // bit 0 active, bit 1 negative, bit 2 direction b
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j;
        fl[j] = 0;
        xr[j] = 0;
        xi[j] = 0;
        if (k < n_up) {
          const HopEntry h = s_hop[k];
          const uint32_t bi = (up >> h.i) & 1u, bj = (up >> h.j) & 1u;
          if (bi != bj) {
            const uint32_t b2 = up ^ h.mask;
            const int64_t u2 = md.sector ? (int64_t)__ldg(md.rank + b2) : (int64_t)b2;
            ld<S>(v, (row_base + u2) * nvec + c, xr[j], xi[j]);
            fl[j] = 1u | ((uint32_t)(__popc(up & h.between) & 1) << 1) | ((bi ? 0u : 1u) << 2);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j;
        if (k < n_up) {
          const int cls = s_hop[k].cls;
          if (cls != cur) {
            flush(cur);
            cur = cls;
          }
          if (fl[j] & 1u) {
            const bool neg = (fl[j] & 2u) != 0;
            if constexpr (C) {
              if (!(fl[j] & 4u)) { ar.add(xr[j], neg); ai.add(xi[j], neg); }
              else { br.add(xr[j], neg); bi_.add(xi[j], neg); }
            } else {
              ar.add(xr[j], neg);
            }
          }
        }
      }
    }
    if (n_up) flush(cur);

    // down hops: row-uniform compacted list, batches of coalesced loads
    const int ndl = s_dl_n;
    const int64_t off = u * nvec + c;
    cur = ndl ? (int)(s_dl_meta[0] >> 2) : 0;
    for (int q0 = 0; q0 < ndl; q0 += kBatch) {
      R xr[kBatch], xi[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        xr[j] = 0;
        xi[j] = 0;
        if (q0 + j < ndl) ld<S>(v, s_dl_src[q0 + j] + off, xr[j], xi[j]);
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int q = q0 + j;
        if (q < ndl) {
          const uint32_t meta = s_dl_meta[q];
          const int cls = (int)(meta >> 2);
          if (cls != cur) {
            flush(cur);
            cur = cls;
          }
          const bool neg = (meta & 1u) != 0;
          if constexpr (C) {
            if (!(meta & 2u)) { ar.add(xr[j], neg); ai.add(xi[j], neg); }
            else { br.add(xr[j], neg); bi_.add(xi[j], neg); }
          } else {
            ar.add(xr[j], neg);
          }
        }
      }
    }
    if (ndl) flush(cur);
    epilogue<S, E>(idx, c, sr, si, hr, hi, w, fa, es, s_inv, red);
  }
  if constexpr (E != Epi::kStore) block_finish<F64>(red, n_red<E>(), nvec, fa.partials, s_red);
}

template <class S, Epi E>
int occupancy_t(bool hub) {
  static int cache[2] = {0, 0};
  int& b = cache[hub ? 1 : 0];
  if (b == 0) {
    int n = 0;
    cudaError_t e = hub ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hv_hub<S, E>, kThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hv_spin<S, E>, kThreads, 0);
    if (e != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 2;
    }
    b = n;
  }
  return b;
}

template <Epi E>
int occupancy_e(bool hub, int prec, bool cplx) {
  if (prec == HPHI_FP64) return cplx ? occupancy_t<double2, E>(hub) : occupancy_t<double, E>(hub);
  return cplx ? occupancy_t<float2, E>(hub) : occupancy_t<float, E>(hub);
}

template <class S, Epi E>
Status launch_t(bool hub, const void* md, const void* v, void* w, int nvec, const FusedArgs& fa, int grid,
                void* scratch, cudaStream_t st) {
  int lg = -1;
  if ((nvec & (nvec - 1)) == 0) {
    lg = 0;
    while ((1 << lg) < nvec) ++lg;
  }
  unsigned long long* counter = hub ? reinterpret_cast<const HubDev*>(md)->counter
                                   : reinterpret_cast<const SpinDev*>(md)->counter;
  HPHI_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  if (hub) {
    k_hv_hub<S, E><<<grid, kThreads, 0, st>>>(*reinterpret_cast<const HubDev*>(md), reinterpret_cast<const S*>(v),
                                             reinterpret_cast<S*>(w), nvec, lg, fa);
  } else {
    const SpinDev& sd = *reinterpret_cast<const SpinDev*>(md);
    bool qt = false;
    if constexpr (Traits<S>::kF64) {
      if (spin_quantised(sd, HPHI_FP64, nvec) && scratch != nullptr) {
        constexpr int ncomp = Traits<S>::kCplx ? 2 : 1;
        long long* q = reinterpret_cast<long long*>(scratch);
        int* e = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(scratch) + (size_t)sd.dim * nvec * sizeof(S));
        Status qs = launch_quant_cols(reinterpret_cast<const double*>(v), sd.dim, nvec, ncomp, q, e, st);
        if (qs.code) return qs;
        k_hv_spin<S, E, true><<<grid, kThreads, 0, st>>>(sd, reinterpret_cast<const S*>(v), reinterpret_cast<S*>(w),
                                                         nvec, lg, fa, q, e);
        qt = true;
      }
    }
    if (!qt)
      k_hv_spin<S, E><<<grid, kThreads, 0, st>>>(sd, reinterpret_cast<const S*>(v), reinterpret_cast<S*>(w), nvec, lg,
                                                fa, nullptr, nullptr);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

template <Epi E>
Status launch_e(bool hub, const void* md, int prec, bool cplx, const void* v, void* w, int nvec, const FusedArgs& fa,
                int grid, void* scratch, cudaStream_t st) {
  if (prec == HPHI_FP64) {
    return cplx ? launch_t<double2, E>(hub, md, v, w, nvec, fa, grid, scratch, st)
                : launch_t<double, E>(hub, md, v, w, nvec, fa, grid, scratch, st);
  }
  return cplx ? launch_t<float2, E>(hub, md, v, w, nvec, fa, grid, scratch, st)
              : launch_t<float, E>(hub, md, v, w, nvec, fa, grid, scratch, st);
}

}  // namespace

int hv_grid(int nvec) {
  (void)nvec;
  return num_sms() * (2048 / kThreads);
}

int hv_resident_grid(bool hubbard, int prec, bool cplx, Epi epi) {
  int b = 2;
  switch (epi) {
    case Epi::kStore: b = occupancy_e<Epi::kStore>(hubbard, prec, cplx); break;
    case Epi::kLanczos1: b = occupancy_e<Epi::kLanczos1>(hubbard, prec, cplx); break;
    case Epi::kTpq: b = occupancy_e<Epi::kTpq>(hubbard, prec, cplx); break;
    case Epi::kRefine: b = occupancy_e<Epi::kRefine>(hubbard, HPHI_FP64, cplx); break;
  }
  return num_sms() * b;
}

bool spin_quantised(const SpinDev& md, int prec, int nvec) {
  return prec == HPHI_FP64 && md.max_run <= 127 && nvec >= 1 && nvec <= kMaxNvec && (nvec & (nvec - 1)) == 0;
}

size_t spin_scratch_bytes(const SpinDev& md, int prec, bool cplx, int nvec) {
  if (!spin_quantised(md, prec, nvec)) return 0;
  return (size_t)md.dim * nvec * 8 * (cplx ? 2 : 1) + sizeof(int) * (size_t)nvec;
}

Status launch_hv(bool hubbard, const void* md, int prec, bool cplx, const void* v, void* w, int nvec, Epi epi,
                 const FusedArgs& fa, int grid, void* scratch, cudaStream_t st) {
  switch (epi) {
    case Epi::kStore: return launch_e<Epi::kStore>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, scratch, st);
    case Epi::kLanczos1:
      return launch_e<Epi::kLanczos1>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, scratch, st);
    case Epi::kTpq: return launch_e<Epi::kTpq>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, scratch, st);
    case Epi::kRefine:
      if (prec != HPHI_FP64) return {HPHI_ERR_INVALID_ARG, "refinement runs in fp64"};
      return launch_e<Epi::kRefine>(hubbard, md, prec, cplx, v, w, nvec, fa, grid, scratch, st);
  }
  return {HPHI_ERR_INVALID_ARG, "unknown epilogue"};
}

// ------------------------------------------------------------------ one-cluster Lanczos
// The whole recurrence of section 3.4 in one thread-block cluster when both Lanczos vectors fit
// in the cluster's shared memory (real spin models up to kClMaxDim rows): no launch per step,
// no trip through HBM.  CTA c of the cluster owns rows [c R, (c + 1) R) of C and P in its shared
// memory; a thread owns rows of its CTA's slice.  H C gathers C[r'] from whichever CTA owns r'
// through distributed shared memory.  GB300 issues fp64 at 1/64 of its fp32 rate, so one SM
// alone would be bound by the fp64 work of the diagonal and exchange sums: the cluster spreads
// it over kClCtas SMs.  Per step: P = c1 H C - c2 P with the partial (C, H C), cluster barrier,
// alpha from the kClCtas partials (every CTA sums them in the same order), P -= gamma C with
// |P|^2, cluster barrier, beta, swap C and P.  The two partial slots alternate, so each
// barrier also ends the reads of the previous one.  Scalars follow k_lz_fin's conventions (C
// unnormalised, sigma = 1 / |C|), so k_tridiag reads the same arrays.
namespace {
constexpr int kClThreads = 256;

__device__ double cl_block_sum(double x, double* s_w) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // the previous sum has been read
  if (lane == 0) s_w[wid] = x;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < kClThreads / 32; ++k) t += s_w[k];  // same order in every thread
  return t;
}

// cluster barrier (all threads of all CTAs; shared-memory writes before it are visible after)
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of variable p of this CTA, as seen in CTA `rank` of the cluster
template <class T>
__device__ __forceinline__ T* cl_map(T* p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// sum over the cluster's CTAs of one shared double: lane c of every warp loads CTA c's value
// (one round trip of distributed shared memory for all of them) and the warp adds them in a
// fixed tree order, so every thread of every CTA gets the same bits
__device__ __forceinline__ double cl_gather_sum(double* p, int ncta) {
  const int lane = threadIdx.x & 31;
  double v = lane < ncta ? *cl_map(p, (unsigned)lane) : 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  // lanes may hold differently rounded sums; lane 0's is the same in every warp of every CTA,
  // and the loop's exit test must see one value everywhere
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__global__ void __launch_bounds__(kClThreads, 1) k_lz_cl(const SpinDev md, LzDev lz, int steps, double brk,
                                                         const double* __restrict__ C0, int R, int ncta) {
  extern __shared__ __align__(16) double sm_v[];  // [2][R]: this CTA's slices of the two vectors
  __shared__ double s_w[kClThreads / 32];
  __shared__ double s_part[2];                   // this CTA's partial of each alternating slot
  __shared__ SpinEntry s_ent[kMaxSpinEntries];
  __shared__ double s_cls[kMaxClasses];
  __shared__ LinGroup s_lin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  const int tid = threadIdx.x;
  const unsigned rank = cl_rank();
  const int64_t n = md.dim;
  const int64_t r0 = (int64_t)rank * R;
  const int64_t left = n - r0;
  const int nloc = left <= 0 ? 0 : (left < (int64_t)R ? (int)left : R);
  double* A = sm_v;
  double* B = sm_v + R;
  for (int i = tid; i < nloc; i += kClThreads) {
    A[i] = C0[r0 + i];
    B[i] = 0.0;
  }
  for (int k = tid; k < md.n_entries; k += kClThreads) s_ent[k] = md.entries[k];
  for (int k = tid; k < md.n_classes; k += kClThreads) s_cls[k] = md.cls_coef[k].x;
  for (int k = tid; k < md.n_lin; k += kClThreads) s_lin[k] = md.lin[k];
  for (int k = tid; k < md.n_pairs; k += kClThreads) s_pair[k] = md.pairs[k];
  for (int k = tid; k < md.n_pair_groups; k += kClThreads) s_pcoef[k] = md.pair_coef[k];
  // k_lz_init / its finaliser have set sigma_0, c1, c2 and the flags
  double sg = lz.sig[0];
  double c1 = lz.s[0], c2 = lz.s[1];
  int done = *lz.done;
  bool cur_a = true;  // C is A (else B)
  int k = 0;
  cl_sync();  // every CTA has staged its slice of C_0
  for (; k < steps && !done; ++k) {
    double* C = cur_a ? A : B;
    double* P = cur_a ? B : A;
    double xh = 0.0;
    for (int i = tid; i < nloc; i += kClThreads) {
      const uint64_t s = md.sector ? sector_state(md.t, (uint64_t)(r0 + i)) : (uint64_t)(r0 + i);
      // diagonal: integer bit counts per coefficient group, one multiply-add per group
      double d = md.c0;
      for (int g = 0; g < md.n_lin; ++g) d += s_lin[g].coef * (double)__popcll(s & s_lin[g].mask);
      if (md.n_pairs) {
        int grp = s_pair[0].grp, cnt = 0;
        for (int q = 0; q < md.n_pairs; ++q) {
          const PairEntry pe = s_pair[q];
          if (pe.grp != grp) {
            d += s_pcoef[grp] * (double)cnt;
            cnt = 0;
            grp = pe.grp;
          }
          cnt += (int)((s >> pe.i) & (s >> pe.j) & 1ull);
        }
        d += s_pcoef[grp] * (double)cnt;
      }
      const double x = C[i];
      double hv = d * x;
      // exchange: signed sums per coefficient class (entries are sorted by class), gathers in
      // batches of eight so their distributed-shared-memory loads overlap
      double acc = 0.0;
      int cur = md.n_entries ? s_ent[0].cls : 0;
      for (int e0 = 0; e0 < md.n_entries; e0 += 8) {
        double y[8];
        int sg8[8], cl8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          y[j] = 0.0;
          sg8[j] = 0;
          cl8[j] = cur;
          const int e = e0 + j;
          if (e < md.n_entries) {
            const SpinEntry en = s_ent[e];
            cl8[j] = en.cls;
            const int sel = (int)((s >> en.i) & 1ull) | ((int)((s >> en.j) & 1ull) << 1);
            const int code = (en.phases >> (3 * sel)) & 7;
            if (code) {
              const uint64_t s2 = s ^ en.mask;
              const int64_t r2 = md.sector ? (int64_t)sector_rank(md.t, s2) : (int64_t)s2;
              const unsigned owner = (unsigned)(r2 / R);
              y[j] = cl_map(C, owner)[r2 - (int64_t)owner * R];
              sg8[j] = code == 1 ? 1 : -1;  // real models: codes +1 / -1 only
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (cl8[j] != cur) {
            hv = fma(s_cls[cur], acc, hv);
            acc = 0.0;
            cur = cl8[j];
          }
          if (sg8[j] > 0) acc += y[j];
          else if (sg8[j] < 0) acc -= y[j];
        }
      }
      if (md.n_entries) hv = fma(s_cls[cur], acc, hv);
      xh = fma(x, hv, xh);
      P[i] = c1 * hv - c2 * P[i];
    }
    double t = cl_block_sum(xh, s_w);
    if (tid == 0) s_part[0] = t;
    cl_sync();  // P written everywhere (so C is no longer read), partials of alpha ready
    const double xs = cl_gather_sum(&s_part[0], ncta);
    const double a = xs * sg * sg;  // alpha_k = (H v_k, v_k)
    const double gm = a * sg;
    double pp = 0.0;
    for (int i = tid; i < nloc; i += kClThreads) {
      const double pv = fma(-gm, C[i], P[i]);
      P[i] = pv;
      pp = fma(pv, pv, pp);
    }
    t = cl_block_sum(pp, s_w);
    if (tid == 0) s_part[1] = t;
    cl_sync();  // the new vector complete everywhere, partials of beta ready
    const double ps = cl_gather_sum(&s_part[1], ncta);
    const double b = sqrt(ps);
    if (rank == 0 && tid == 0) {
      lz.alpha[k] = a;
      lz.beta[k] = b;
    }
    if (!(b > brk * fmax(1.0, fabs(a)))) {
      done = 1;
    } else {
      const double sn = 1.0 / b;
      c1 = sn;
      c2 = b * sg;
      sg = sn;
      if (rank == 0 && tid == 0) lz.sig[k + 1] = sn;
      cur_a = !cur_a;
    }
  }
  if (rank == 0 && tid == 0) {
    *lz.steps_done = k;
    *lz.done = 1;
  }
  cl_sync();  // no CTA leaves while another may still read its shared memory
}

constexpr int kClCtas = 16;       // CTAs per cluster (non-portable size; 8 if 16 cannot launch)
constexpr int64_t kClMaxDim = 32768;

}  // namespace

// dynamic shared memory of one cluster CTA, or 0 when the model does not take the path
size_t lz_cta_smem(const SpinDev& md) {
  if (md.dim > kClMaxDim) return 0;
  const int64_t R = (md.dim + kClCtas - 1) / kClCtas;
  return 2 * sizeof(double) * (size_t)R;
}

Status launch_lz_cta(const SpinDev& md, const LzDev& lz, int steps, double brk, const double* C0, cudaStream_t st) {
  for (int cs : {kClCtas, 8}) {
    const int R = (int)((md.dim + cs - 1) / cs);
    const size_t smem = 2 * sizeof(double) * (size_t)R;
    HPHI_CUDA_TRY(cudaFuncSetAttribute(k_lz_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (cs > 8) HPHI_CUDA_TRY(cudaFuncSetAttribute(k_lz_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_lz_cl, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    HPHI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_lz_cl, md, lz, steps, brk, C0, R, cs));
    return {};
  }
  return {HPHI_ERR_CUDA, "one-cluster Lanczos: no cluster of 16 or 8 CTAs can be scheduled"};
}

}  // namespace hphi
