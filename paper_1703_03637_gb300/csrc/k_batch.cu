// H v over rows of many vectors at once: the batched mTPQ starts of section 3.5 (and any
// apply_H with nvec in {32, 64, 128, 256}) on spin models in the full 2^N basis, N <= 32.
//
// The vectors are stored [row][column], so the nvec entries a term gathers from row s ^ mask
// are contiguous.  A row is handled by nvec / CPL lanes, lane l owning CPL consecutive
// columns (32 or 64 bytes: two or four 16-byte loads per neighbour); a warp takes
// 32 / (nvec / CPL) rows at once.  The per-term work (entry, phase code, neighbour row) is
// paid once per lane for CPL columns instead of once per column as in the generic kernel,
// and the loads are 16 bytes wide.
//
// fp64 runs the gathers on a copy of the input quantised to 64-bit integers with one scale
// per column (q = round(x 2^(1078 - E_c)), |q| < 2^56): the sum of a class run of at most 127
// terms is an exact integer sum, converted to fp64 once (the same trick as the two-pass
// Hubbard path, for the same reason: fp64 adds run at 1/64 of the fp32 rate on this part).
//
// Optional window passes (section 4.3's continuous memory access on one GPU): each pass takes
// the terms whose flipped sites lie in one cyclic window and visits the rows with that
// window's bits varying fastest, keeping its partial sums in the buffer the last pass writes.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "epilogue.cuh"
#include "reduce.cuh"

namespace hphi {

namespace {

// Launch shape per scalar type and epilogue, from a sweep on the 2^24-row, 64-vector Kitaev
// workload: kRegs = 32-bit registers of gathered values in flight per thread, kMinB =
// resident CTAs per SM the register budget is cut for, kLaneBytes = bytes of a row one lane
// gathers per term (at least).  The plain fp32 product keeps the most loads in flight, the
// fp32 mTPQ step a few less (its sums need registers), fp64 fewer still; fp64 lanes take
// 64 bytes (four columns).
template <class S, Epi E> struct BatchTune {
  static constexpr bool kF64 = Traits<S>::kF64;
  static constexpr int kRegs = kF64 ? 32 : (E == Epi::kStore ? 64 : (E == Epi::kTpq ? 48 : 32));
  static constexpr int kMinB = 2;
  static constexpr int kLaneBytes = kF64 ? 64 : 32;
};

template <class S, Epi E> struct BatchCpl {
  static constexpr int kMin = (int)(BatchTune<S, E>::kLaneBytes / sizeof(S));  // columns per lane
};

template <class T, int N> struct Regs {
  T re[N], im[N];
};

// CPL consecutive elements of type S as (re, im) scalars of type T; p is 32-byte aligned
// (kStream: evict-first, for the pass accumulator, which is read once per pass)
template <class S, int CPL, bool kStream = false, class T>
__device__ __forceinline__ void vload(const T* __restrict__ p, Regs<T, CPL>& o) {
  constexpr bool C = Traits<S>::kCplx;
  constexpr int nT = CPL * (C ? 2 : 1);
  constexpr int n16 = nT * (int)sizeof(T) / 16;
  union {
    uint4 u[n16];
    T t[nT];
  } b;
#pragma unroll
  for (int k = 0; k < n16; ++k)
    b.u[k] = kStream ? __ldcs(reinterpret_cast<const uint4*>(p) + k) : __ldg(reinterpret_cast<const uint4*>(p) + k);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    o.re[c] = C ? b.t[2 * c] : b.t[c];
    o.im[c] = C ? b.t[2 * c + 1] : T(0);
  }
}

template <class S, int CPL, bool kStream = false, class T>
__device__ __forceinline__ void vstore(T* __restrict__ p, const Regs<T, CPL>& o) {
  constexpr bool C = Traits<S>::kCplx;
  constexpr int nT = CPL * (C ? 2 : 1);
  constexpr int n16 = nT * (int)sizeof(T) / 16;
  union {
    uint4 u[n16];
    T t[nT];
  } b;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    if (C) {
      b.t[2 * c] = o.re[c];
      b.t[2 * c + 1] = o.im[c];
    } else {
      b.t[c] = o.re[c];
    }
  }
#pragma unroll
  for (int k = 0; k < n16; ++k) {
    if (kStream) __stcs(reinterpret_cast<uint4*>(p) + k, b.u[k]);
    else reinterpret_cast<uint4*>(p)[k] = b.u[k];
  }
}

// one pass over the rows: its entries, its visit order and its place in the sequence
struct PassArgs {
  const SpinEntry* ents;  // entries [e0, e1) of this pass
  int e0, e1;
  const uint32_t* dep;    // [4][256] visit-index byte -> row bits; null: natural order
  int first, last;        // the first pass adds the diagonal, the last runs the epilogue
  void* acc;              // row-owned accumulator between passes (null for one pass)
};

// column exponents: E[c] = the largest exponent field over the rows (real and imaginary
// parts) of column c; the [row][column] vector is read once, coalesced
__global__ void __launch_bounds__(kThreads) k_maxexp_cols(const double* __restrict__ X, int64_t rows, int rowlen,
                                                           int ncomp, int* __restrict__ E) {
  __shared__ int s_max[kMaxNvec];
  const int tid = threadIdx.x;
  for (int k = tid; k < rowlen; k += kThreads) s_max[k / ncomp] = 0;
  __syncthreads();
  const int per = rowlen < kThreads ? rowlen : kThreads;  // threads per row segment
  const int rpb = kThreads / per;                          // rows per CTA and iteration
  const int k0 = tid % per, rs = tid / per;
  for (int k = k0; k < rowlen; k += per) {
    int mx = 0;
    for (int64_t r = (int64_t)blockIdx.x * rpb + rs; r < rows; r += (int64_t)gridDim.x * rpb)
      mx = max(mx, (__double2hiint(__ldg(X + r * rowlen + k)) >> 20) & 0x7ff);
    atomicMax(&s_max[k / ncomp], mx);
  }
  __syncthreads();
  for (int c = tid; c < rowlen / ncomp; c += kThreads)
    if (s_max[c] > 0) atomicMax(E + c, s_max[c]);
}

// q = round(x 2^(1078 - E_c)): |q| < 2^56, one rounding per element (at most 2^-57 max_c |x|)
__global__ void __launch_bounds__(kThreads) k_quant_cols(const double* __restrict__ X, long long* __restrict__ Q,
                                                          int64_t n, int lg_rowlen, int lg_ncomp,
                                                          const int* __restrict__ Ec) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const int c = (int)((i & ((1ll << lg_rowlen) - 1)) >> lg_ncomp);
    const int E = Ec[c];
    const double x = __ldg(X + i);
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (hi >> 20) & 0x7ff;
    long long q = 0;
    if (ex != 0) {
      const long long M = ((long long)((hi & 0xfffff) | 0x100000) << 32) | (long long)lo;  // x = M 2^(ex-1075)
      const int sh = E - ex - 3;                                                           // q = M 2^-sh
      if (sh <= 0) q = M << (-sh);
      else if (sh < 62) q = (M + (1ll << (sh - 1))) >> sh;
      if (hi < 0) q = -q;
    }
    Q[i] = q;
  }
}

// QT (fp64 only): gathers read the quantised copy Q; class sums are exact int64 sums.
// Without QT, fp64 class sums are exact fixed-point sums of the fp64 terms (class runs
// longer than 127 terms) and fp32 sums are plain fp32.
template <class S, Epi E, int CPL, bool QT>
__global__ void __launch_bounds__(kThreads, BatchTune<S, E>::kMinB)
    k_hv_batch(const SpinDev md, const PassArgs pa, const S* __restrict__ v, S* __restrict__ w, int nvec,
               FusedArgs fa, const long long* __restrict__ Q, const int* __restrict__ Ec) {
  using R = typename Traits<S>::R;
  constexpr bool C = Traits<S>::kCplx;
  constexpr bool F64 = Traits<S>::kF64;
  static_assert(!QT || F64, "quantised gathers are an fp64 path");
  constexpr int kWarps = kThreads / 32;
  // terms in flight: kBatchRegs 32-bit registers of gathered values
  constexpr int kRegsPerTerm = CPL * (C ? 2 : 1) * (QT ? 2 : (int)sizeof(R) / 4);
  constexpr int kB = BatchTune<S, E>::kRegs / kRegsPerTerm > 1 ? BatchTune<S, E>::kRegs / kRegsPerTerm : 1;
  using T = std::conditional_t<QT, long long, R>;  // gathered scalar
  using A = std::conditional_t<QT, IntAcc, typename SumAcc<R>::T>;
  __shared__ SpinEntry s_ent[kMaxSpinEntries];
  __shared__ R s_cr[kMaxClasses], s_ci[kMaxClasses];
  __shared__ LinGroup s_lin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  __shared__ double s_inv[kMaxNvec];
  __shared__ double s_red[(E == Epi::kStore) ? 1 : kThreads * CPL];
  __shared__ uint32_t s_dep[4 * 256];
  __shared__ float2 s_phase[8];  // phase codes 0 (none), 1 (+1), 2 (+i), 3 (-1), 4 (-i) as (re, im)

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ne = pa.e1 - pa.e0;
  for (int k = tid; k < ne; k += kThreads) s_ent[k] = pa.ents[pa.e0 + k];
  if (tid < 8) s_phase[tid] = make_float2(tid == 1 ? 1.f : tid == 3 ? -1.f : 0.f, tid == 2 ? 1.f : tid == 4 ? -1.f : 0.f);
  const bool deposit = pa.dep != nullptr;
  if (deposit)
    for (int k = tid; k < 4 * 256; k += kThreads) s_dep[k] = pa.dep[k];
  for (int k = tid; k < md.n_classes; k += kThreads) {
    const double2 cc = md.cls_coef[k];
    s_cr[k] = (R)cc.x;
    s_ci[k] = (R)cc.y;
  }
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

  constexpr int kNQ = n_red<E>() > 0 ? n_red<E>() : 1;
  Red<F64, kNQ> red[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) red[q].zero();
  const int lpr = nvec / CPL;  // lanes per row: a power of two <= 32
  const int lg_lpr = __ffs(lpr) - 1;
  const int rpw = 32 >> lg_lpr;  // rows per warp
  const int slot = lane >> lg_lpr;
  const int c0 = (lane & (lpr - 1)) * CPL;
  int eoff[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) eoff[q] = QT ? Ec[c0 + q] - 1078 : 0;
  const int64_t step = (int64_t)gridDim.x * kWarps * rpw;
  const bool first = pa.first != 0, last = pa.last != 0;
  S* acc = reinterpret_cast<S*>(pa.acc);
  for (int64_t row = ((int64_t)blockIdx.x * kWarps + warp) * rpw + slot; row < md.dim; row += step) {
    const uint32_t t = (uint32_t)row;  // visit index
    const uint32_t s = deposit ? (s_dep[t & 255u] | s_dep[256 + ((t >> 8) & 255u)] |
                                  s_dep[512 + ((t >> 16) & 255u)] | s_dep[768 + (t >> 24)])
                               : t;
    const int64_t off = (int64_t)s * nvec + c0;
    Regs<R, CPL> h;
    if (!first) {
      vload<S, CPL, true>(reinterpret_cast<const R*>(acc + off), h);
    } else {
    // diagonal
    R d = (R)md.c0;
    for (int g = 0; g < md.n_lin; ++g) d += (R)s_lin[g].coef * (R)__popc(s & (uint32_t)s_lin[g].mask);
    if (md.n_pairs) {
      int grp = s_pair[0].grp, cnt = 0;
      for (int p = 0; p < md.n_pairs; ++p) {
        const PairEntry pe = s_pair[p];
        if (pe.grp != grp) {
          d += (R)s_pcoef[grp] * (R)cnt;
          cnt = 0;
          grp = pe.grp;
        }
        cnt += (int)((s >> pe.i) & (s >> pe.j) & 1u);
      }
      d += (R)s_pcoef[grp] * (R)cnt;
    }
    {
      Regs<R, CPL> x0;
      vload<S, CPL>(reinterpret_cast<const R*>(v + off), x0);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        h.re[q] = d * x0.re[q];
        h.im[q] = d * x0.im[q];
      }
    }
    }
    A ar[CPL], ai[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      ar[q].zero();
      ai[q].zero();
    }
    int cur = ne ? s_ent[0].cls : 0;
    auto flush = [&](int cls) {
      const R cr = s_cr[cls], ci = s_ci[cls];
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        R vr, vi;
        if constexpr (QT) {
          vr = fix_to_double(ar[q].value(), eoff[q]);
          vi = C ? fix_to_double(ai[q].value(), eoff[q]) : 0.0;
        } else {
          vr = (R)ar[q].value();
          vi = (R)ai[q].value();
        }
        if constexpr (C) {
          if (ci == R(0)) {  // real class coefficient (the same in every lane): half the fp64 work
            h.re[q] += cr * vr;
            h.im[q] += cr * vi;
          } else {
            h.re[q] += cr * vr - ci * vi;
            h.im[q] += cr * vi + ci * vr;
          }
        } else {
          h.re[q] += cr * vr;
        }
        ar[q].zero();
        ai[q].zero();
      }
    };
    for (int e0 = 0; e0 < ne; e0 += kB) {
      Regs<T, CPL> x[kB];
      int code[kB], cls[kB];
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        code[j] = 0;
        cls[j] = cur;
        if (e0 + j < ne) {
          const SpinEntry en = s_ent[e0 + j];
          const int sel = (int)((s >> en.i) & 1u) | ((int)((s >> en.j) & 1u) << 1);
          code[j] = (en.phases >> (3 * sel)) & 7;
          cls[j] = en.cls;
          if constexpr (F64) {
            // fp64 skips code-0 terms in the switch below: load only the live ones
            if (code[j]) {
              const int64_t o2 = (int64_t)(s ^ (uint32_t)en.mask) * nvec + c0;
              if constexpr (QT) vload<S, CPL>(Q + o2 * (C ? 2 : 1), x[j]);
              else vload<S, CPL>(reinterpret_cast<const R*>(v + o2), x[j]);
            }
          } else {
            // fp32 multiplies every term by its phase, (0, 0) for code 0: such a term reads
            // the row itself (already in L1) so that the value is defined and costs no DRAM
            const uint32_t t = code[j] ? (s ^ (uint32_t)en.mask) : s;
            vload<S, CPL>(reinterpret_cast<const R*>(v + ((int64_t)t * nvec + c0)), x[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        if (e0 + j < ne) {
          if (cls[j] != cur) {  // the same in every lane: the entries are shared
            flush(cur);
            cur = cls[j];
          }
          if constexpr (F64) {
            // the code is the same in every lane of a row, and a warp holds one row when
            // the row is 512 bytes or more, so the switch inside acc_phase rarely diverges
            // (branch-free selects cost three times the integer instructions)
            if (code[j]) {
#pragma unroll
              for (int q = 0; q < CPL; ++q) {
                if constexpr (C) acc_phase(code[j], x[j].re[q], x[j].im[q], ar[q], ai[q]);
                else ar[q].add(x[j].re[q], code[j] != 1);
              }
            }
          } else {
            const float2 ph = s_phase[code[j]];
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              if constexpr (C) {
                ar[q].s = fmaf(ph.x, x[j].re[q], fmaf(-ph.y, x[j].im[q], ar[q].s));
                ai[q].s = fmaf(ph.x, x[j].im[q], fmaf(ph.y, x[j].re[q], ai[q].s));
              } else {
                ar[q].s = fmaf(ph.x, x[j].re[q], ar[q].s);
              }
            }
          }
        }
      }
    }
    if (ne) flush(cur);
    if (!last) {
      vstore<S, CPL, true>(reinterpret_cast<R*>(acc + off), h);
    } else if constexpr (E == Epi::kStore) {
      vstore<S, CPL>(reinterpret_cast<R*>(w + off), h);
    } else {
      Regs<R, CPL> x0;  // read again (from L1 / L2) rather than held across the term loop
      vload<S, CPL>(reinterpret_cast<const R*>(v + off), x0);
      if constexpr (E == Epi::kTpq || E == Epi::kRefine) {
        // the same updates and sums as the shared epilogue, with the row's columns written
        // as 16-byte stores
        Regs<R, CPL> o;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          if constexpr (E == Epi::kTpq) {
            const R inv = (R)s_inv[c0 + q], l = (R)fa.l, ins = (R)fa.inv_ns;
            o.re[q] = inv * (l * x0.re[q] - h.re[q] * ins);
            o.im[q] = inv * (l * x0.im[q] - h.im[q] * ins);
            red[q].add(0, x0.re[q], h.re[q]);
            red[q].add(1, h.re[q], h.re[q]);
            if constexpr (C) {
              red[q].add(0, x0.im[q], h.im[q]);
              red[q].add(1, h.im[q], h.im[q]);
            }
          } else {
            o.re[q] = h.re[q];
            o.im[q] = h.im[q];
            red[q].add(0, x0.re[q], h.re[q]);
            red[q].add(1, x0.re[q], x0.re[q]);
            red[q].add(2, h.re[q], h.re[q]);
            if constexpr (C) {
              red[q].add(0, x0.im[q], h.im[q]);
              red[q].add(1, x0.im[q], x0.im[q]);
              red[q].add(2, h.im[q], h.im[q]);
            }
          }
          red[q].tick();
        }
        vstore<S, CPL>(reinterpret_cast<R*>(reinterpret_cast<S*>(fa.out) + off), o);
      } else {
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          epilogue<S, E, kNQ>(off + q, c0 + q, x0.re[q], x0.im[q], h.re[q], h.im[q], w, fa, es, s_inv, red[q]);
      }
    }
  }
  if constexpr (E != Epi::kStore) {
    if (!last) return;  // the same for the whole grid
    // per-column sums, one quantity at a time; the (warp, row slot) pairs are summed in a
    // fixed order, so the result does not depend on timing
    constexpr int nq = n_red<E>();
    const int nvw = kWarps * rpw;
    for (int k = 0; k < nq; ++k) {
#pragma unroll
      for (int q = 0; q < CPL; ++q) s_red[(warp * rpw + slot) * nvec + c0 + q] = red[q].get(k);
      __syncthreads();
      for (int c = tid; c < nvec; c += kThreads) {
        double t = 0.0;
        for (int vw = 0; vw < nvw; ++vw) t += s_red[vw * nvec + c];
        fa.partials[((size_t)blockIdx.x * nvec + c) * kMaxRedQ + k] = t;
      }
      __syncthreads();
    }
  }
}

int max_run_of(const SpinDev& md, const BatchPlan* plan) { return plan ? plan->max_run : md.max_run; }
bool quantised(int max_run, int prec) { return prec == HPHI_FP64 && max_run <= 127; }

template <class S, Epi E, int CPL, bool QT>
Status launch_q(const SpinDev& md, const BatchPlan* plan, const void* v, void* w, void* scratch, int nvec,
                const FusedArgs& fa, int grid, cudaStream_t st) {
  constexpr int ncomp = Traits<S>::kCplx ? 2 : 1;
  const long long* Q = nullptr;
  const int* Ec = nullptr;
  if constexpr (QT) {
    // scratch: [Q: the quantised input] [E: one exponent per column]
    const size_t vb = (size_t)md.dim * nvec * sizeof(S);
    long long* q = reinterpret_cast<long long*>(scratch);
    int* e = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(scratch) + vb);
    Status qs = launch_quant_cols(reinterpret_cast<const double*>(v), md.dim, nvec, ncomp, q, e, st);
    if (qs.code) return qs;
    Q = q;
    Ec = e;
  }
  const int np = plan ? plan->n_pass : 1;
  for (int p = 0; p < np; ++p) {
    PassArgs pa;
    pa.ents = plan ? plan->ents : md.entries;
    pa.e0 = plan ? plan->ent_off[p] : 0;
    pa.e1 = plan ? plan->ent_off[p + 1] : md.n_entries;
    pa.dep = plan ? plan->dep + (size_t)p * 1024 : nullptr;
    pa.first = p == 0;
    pa.last = p == np - 1;
    // the accumulator is the buffer the last pass writes row by row: w, or the epilogue's
    // output (the last pass reads a row's partial sum before it overwrites the row)
    pa.acc = np > 1 ? (E == Epi::kStore ? w : fa.out) : nullptr;
    k_hv_batch<S, E, CPL, QT><<<grid, kThreads, 0, st>>>(md, pa, reinterpret_cast<const S*>(v),
                                                         reinterpret_cast<S*>(w), nvec, fa, Q, Ec);
    HPHI_CUDA_TRY(cudaGetLastError());
  }
  return {};
}

// columns per lane for nvec vectors: the tuned load width, at most 32 lanes per row
template <class S, Epi E>
int cpl_for(int nvec) {
  return std::max(BatchCpl<S, E>::kMin, nvec / 32);
}

template <class S, Epi E, int CPL>
Status launch_c(const SpinDev& md, const BatchPlan* plan, int prec, const void* v, void* w, void* scratch, int nvec,
                const FusedArgs& fa, int grid, cudaStream_t st) {
  if constexpr (CPL < BatchCpl<S, E>::kMin) {
    return {HPHI_ERR_INVALID_ARG, "batched rows: columns per lane below the load width"};
  } else {
    if constexpr (Traits<S>::kF64) {
      if (quantised(max_run_of(md, plan), prec))
        return launch_q<S, E, CPL, true>(md, plan, v, w, scratch, nvec, fa, grid, st);
    }
    return launch_q<S, E, CPL, false>(md, plan, v, w, scratch, nvec, fa, grid, st);
  }
}

template <class S, Epi E>
Status launch_t(const SpinDev& md, const BatchPlan* plan, int prec, const void* v, void* w, void* scratch, int nvec,
                const FusedArgs& fa, int grid, cudaStream_t st) {
  switch (cpl_for<S, E>(nvec)) {
    case 2: return launch_c<S, E, 2>(md, plan, prec, v, w, scratch, nvec, fa, grid, st);
    case 4: return launch_c<S, E, 4>(md, plan, prec, v, w, scratch, nvec, fa, grid, st);
    case 8: return launch_c<S, E, 8>(md, plan, prec, v, w, scratch, nvec, fa, grid, st);
    default: return {HPHI_ERR_INVALID_ARG, "batched rows: unsupported nvec"};
  }
}

template <Epi E>
Status launch_e(const SpinDev& md, const BatchPlan* plan, int prec, bool cplx, const void* v, void* w, void* scratch,
                int nvec, const FusedArgs& fa, int grid, cudaStream_t st) {
  if (prec == HPHI_FP64)
    return cplx ? launch_t<double2, E>(md, plan, prec, v, w, scratch, nvec, fa, grid, st)
                : launch_t<double, E>(md, plan, prec, v, w, scratch, nvec, fa, grid, st);
  return cplx ? launch_t<float2, E>(md, plan, prec, v, w, scratch, nvec, fa, grid, st)
              : launch_t<float, E>(md, plan, prec, v, w, scratch, nvec, fa, grid, st);
}

template <class S, Epi E, int CPL>
int occupancy_c() {
  if constexpr (CPL < BatchCpl<S, E>::kMin) {
    return 1;
  } else {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hv_batch<S, E, CPL, Traits<S>::kF64>, kThreads, 0) !=
        cudaSuccess) {
      cudaGetLastError();
      n = 1;
    }
    return n < 1 ? 1 : n;
  }
}

template <class S, Epi E>
int occupancy_t(int nvec) {
  static int cache[4] = {0, 0, 0, 0};  // by columns per lane 2, 4, 8
  const int cpl = cpl_for<S, E>(nvec);
  int& b = cache[cpl == 2 ? 1 : cpl == 4 ? 2 : 3];
  if (b == 0) b = cpl == 2 ? occupancy_c<S, E, 2>() : cpl == 4 ? occupancy_c<S, E, 4>() : occupancy_c<S, E, 8>();
  return b;
}

template <Epi E>
int occupancy_e(int prec, bool cplx, int nvec) {
  if (prec == HPHI_FP64) return cplx ? occupancy_t<double2, E>(nvec) : occupancy_t<double, E>(nvec);
  return cplx ? occupancy_t<float2, E>(nvec) : occupancy_t<float, E>(nvec);
}

}  // namespace

int batch_window_bits(int prec, bool cplx, int nvec) {
  const double row = (double)nvec * (prec == HPHI_FP64 ? 8 : 4) * (cplx ? 2 : 1);
  int w = 0;
  while ((double)(1ll << (w + 1)) * row <= 32.0 * 1024 * 1024) ++w;
  return w;
}

bool batch_plan_windows(int n_sites, int wbits, const std::vector<SpinEntry>& ents,
                        std::vector<SpinEntry>* ordered, std::vector<uint32_t>* dep, int* ent_off, int* n_pass,
                        int* max_run) {
  *n_pass = 0;
  if (n_sites > 32 || wbits < 1 || wbits >= n_sites) return false;
  auto window = [&](int a) {
    uint64_t m = 0;
    for (int b = 0; b < wbits; ++b) m |= 1ull << ((a + b) % n_sites);
    return m;
  };
  // greedy: the cyclic window holding the most unassigned flip masks, until all are held
  std::vector<int> pass_of(ents.size(), -1);
  std::vector<uint64_t> chosen;
  size_t left = ents.size();
  while (left > 0) {
    if ((int)chosen.size() >= kMaxPasses) return false;
    int best_a = -1;
    size_t best_n = 0;
    for (int a = 0; a < n_sites; ++a) {
      const uint64_t m = window(a);
      size_t n = 0;
      for (size_t k = 0; k < ents.size(); ++k)
        if (pass_of[k] < 0 && (ents[k].mask & ~m) == 0) ++n;
      if (n > best_n) {
        best_n = n;
        best_a = a;
      }
    }
    if (best_a < 0) return false;  // a mask wider than the window
    const uint64_t m = window(best_a);
    for (size_t k = 0; k < ents.size(); ++k)
      if (pass_of[k] < 0 && (ents[k].mask & ~m) == 0) {
        pass_of[k] = (int)chosen.size();
        --left;
      }
    chosen.push_back(m);
  }
  if (chosen.size() < 2) return false;  // one window holds every term: the plain order does
  ordered->clear();
  dep->assign(chosen.size() * 1024, 0u);
  *max_run = 0;
  for (size_t p = 0; p < chosen.size(); ++p) {
    ent_off[p] = (int)ordered->size();
    for (size_t k = 0; k < ents.size(); ++k)  // input is class-sorted; keep that order
      if (pass_of[k] == (int)p) ordered->push_back(ents[k]);
    // visit index bit t -> row bit pos[t]: the window's bits first (fastest), then the rest
    int pos[32], n = 0;
    for (int b = 0; b < n_sites; ++b)
      if ((chosen[p] >> b) & 1ull) pos[n++] = b;
    for (int b = 0; b < n_sites; ++b)
      if (!((chosen[p] >> b) & 1ull)) pos[n++] = b;
    for (int byte = 0; byte < 4; ++byte)
      for (int val = 0; val < 256; ++val) {
        uint32_t r = 0;
        for (int t = 0; t < 8; ++t) {
          const int src = byte * 8 + t;
          if (((val >> t) & 1) && src < n_sites) r |= 1u << pos[src];
        }
        (*dep)[p * 1024 + byte * 256 + val] = r;
      }
  }
  ent_off[chosen.size()] = (int)ordered->size();
  for (size_t p = 0; p < chosen.size(); ++p) {
    int run = 0;
    for (int k = ent_off[p]; k < ent_off[p + 1]; ++k) {
      run = (k > ent_off[p] && (*ordered)[k].cls == (*ordered)[k - 1].cls) ? run + 1 : 1;
      *max_run = std::max(*max_run, run);
    }
  }
  *n_pass = (int)chosen.size();
  return true;
}

Status launch_quant_cols(const double* v, int64_t rows, int nvec, int ncomp, long long* Q, int* E, cudaStream_t st) {
  const int rowlen = nvec * ncomp;
  if ((rowlen & (rowlen - 1)) != 0 || nvec > kMaxNvec)
    return {HPHI_ERR_INVALID_ARG, "quantised copy: nvec must be a power of two up to 256"};
  int lg_row = 0;
  while ((1 << lg_row) < rowlen) ++lg_row;
  HPHI_CUDA_TRY(cudaMemsetAsync(E, 0, sizeof(int) * nvec, st));
  const int gv = (int)std::max<int64_t>(
      1, std::min<int64_t>((rows * rowlen + kThreads - 1) / kThreads, (int64_t)num_sms() * 8));
  k_maxexp_cols<<<gv, kThreads, 0, st>>>(v, rows, rowlen, ncomp, E);
  HPHI_CUDA_TRY(cudaGetLastError());
  k_quant_cols<<<gv, kThreads, 0, st>>>(v, Q, rows * rowlen, lg_row, ncomp == 2 ? 1 : 0, E);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

bool batch_applies(const SpinDev& md, int nvec) {
  return md.sector == 0 && md.n_sites <= 32 && (nvec == 32 || nvec == 64 || nvec == 128 || nvec == 256);
}

bool batch_aligned(const void* v, const void* w) { return (((uintptr_t)v | (uintptr_t)w) & 31u) == 0; }

size_t batch_scratch_bytes(const SpinDev& md, const BatchPlan* plan, int prec, bool cplx, int nvec) {
  if (!quantised(max_run_of(md, plan), prec)) return 0;
  return (size_t)md.dim * nvec * 8 * (cplx ? 2 : 1) + sizeof(int) * (size_t)nvec;
}

// One wave of resident CTAs (a grid-stride kernel given more CTAs than fit runs a second,
// mostly empty wave), and no more CTAs than there are rows for (one row per warp at least).
int batch_grid(int prec, bool cplx, int nvec, Epi epi, int64_t dim) {
  int b = 1;
  switch (epi) {
    case Epi::kStore: b = occupancy_e<Epi::kStore>(prec, cplx, nvec); break;
    case Epi::kLanczos1: b = occupancy_e<Epi::kLanczos1>(prec, cplx, nvec); break;
    case Epi::kTpq: b = occupancy_e<Epi::kTpq>(prec, cplx, nvec); break;
    case Epi::kRefine: b = occupancy_e<Epi::kRefine>(HPHI_FP64, cplx, nvec); break;
  }
  const int64_t need = (dim + kThreads / 32 - 1) / (kThreads / 32);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * b));
}

Status launch_batch(const SpinDev& md, const BatchPlan* plan, int prec, bool cplx, const void* v, void* w,
                    void* scratch, int nvec, Epi epi, const FusedArgs& fa, int grid, cudaStream_t st) {
  if (!batch_applies(md, nvec) || !batch_aligned(v, w))
    return {HPHI_ERR_INVALID_ARG, "batched rows: model, nvec or alignment not supported"};
  // several passes keep their partial sums in the buffer the last pass writes: not possible
  // for the Lanczos epilogue, which reads that buffer's previous contents
  if (plan && (plan->n_pass < 2 || epi == Epi::kLanczos1)) plan = nullptr;
  if (batch_scratch_bytes(md, plan, prec, cplx, nvec) != 0 && scratch == nullptr)
    return {HPHI_ERR_INVALID_ARG, "batched rows: fp64 needs a scratch buffer"};
  switch (epi) {
    case Epi::kStore: return launch_e<Epi::kStore>(md, plan, prec, cplx, v, w, scratch, nvec, fa, grid, st);
    case Epi::kLanczos1: return launch_e<Epi::kLanczos1>(md, plan, prec, cplx, v, w, scratch, nvec, fa, grid, st);
    case Epi::kTpq: return launch_e<Epi::kTpq>(md, plan, prec, cplx, v, w, scratch, nvec, fa, grid, st);
    case Epi::kRefine:
      if (prec != HPHI_FP64) break;
      return launch_e<Epi::kRefine>(md, plan, prec, cplx, v, w, scratch, nvec, fa, grid, st);
  }
  return {HPHI_ERR_INVALID_ARG, "batched rows: unsupported precision / epilogue"};
}

}  // namespace hphi
