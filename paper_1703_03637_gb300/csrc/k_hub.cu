// Two-pass H v for Hubbard models with real hopping and one hopping value per spin
// species (the half-filled square-lattice workloads): section 3.3's on-the-fly product,
// laid out for GB300's memory hierarchy.
//
// The amplitudes form a matrix X[d][u] (down-spin rank d, up-spin rank u).  Down-spin
// hops combine whole rows (W[d][:] = sum_q +-X[d'_q][:]) and up-spin hops act inside a row
// (sum_q +-X[d][u'_q]).  So:
//   pass D  walks column stripes in stripe-major order; the stripe of every row stays in
//           L2 while all rows of that stripe are combined, so X is read from HBM about once.
//           W receives the plain signed sums.
//   pass U  stages K whole rows of X in shared memory, applies the up-spin neighbour table
//           (built once per sector on the device) to all K rows at once, adds diag * X and
//           coef * W, and runs the fused Lanczos / mTPQ epilogue.
// fp64 sums use the exact fixed-point accumulator (integer pipes); fp32 sums are plain.
#include <mutex>
#include <string>

#include "common.cuh"
#include "epilogue.cuh"
#include "reduce.cuh"

namespace hphi {

// ------------------------------------------------------------------ allocation-free scratch
// Scratch of hphi_apply_H_noalloc: the int64 copy of the input, the int64 down-spin sums and
// the scale word of the fixed-point fp64 path (16 bytes per row + 256).  It is a file-scope
// device array, so every GPU that loads this library holds these 64 MiB until the process
// exits, and every call on a device shares it.  Host code must not use the symbol as a
// pointer: its device address comes from cudaGetSymbolAddress (noalloc_scratch below).
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// columns per thread in pass D (stripe = kThreads * EPT columns); the stripe of all rows is
// the L2 working set of pass D
// built-in pass-D columns per thread per precision (hphi_autotune replaces them per model)
#ifndef HPHI_DN_EPT32
#define HPHI_DN_EPT32 4
#endif
#ifndef HPHI_DN_EPT64
#define HPHI_DN_EPT64 1
#endif

// K consecutive values of a shared-memory row tile with the widest aligned accesses
template <class R, int K>
__device__ __forceinline__ void load_k(const R* p, R* out) {
  if constexpr (sizeof(R) * K == 16) {
    if constexpr (sizeof(R) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(p);
      out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
    } else {
      const double2 t = *reinterpret_cast<const double2*>(p);
      out[0] = t.x; out[1] = t.y;
    }
  } else if constexpr (sizeof(R) * K == 8 && sizeof(R) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    out[0] = t.x; out[1] = t.y;
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) out[m] = p[m];
  }
}

template <class R, int K>
__device__ __forceinline__ void store_k(R* p, const R* v) {
  if constexpr (sizeof(R) * K == 16) {
    if constexpr (sizeof(R) == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else if constexpr (sizeof(R) * K == 8 && sizeof(R) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int m = 0; m < K; ++m) p[m] = v[m];
  }
}
constexpr int kSmemBudget = 208000;  // shared-memory bytes for the row tile (plus ~21 KB static)

// neighbour table of one species, hop-slot major: nbr[q * n + k] is the q-th active hop
// target of state k (rank | sign << 31), so threads of consecutive states read
// consecutive words
__global__ void k_hub_nbr(const HubDev md, int species, uint32_t* __restrict__ nbr, uint8_t* __restrict__ deg,
                          uint8_t* __restrict__ npos) {
  const int64_t n = species ? md.dim_dn : md.dim_up;
  const int e0 = species ? md.n_up_hops : 0;
  const int ne = species ? md.n_dn_hops : md.n_up_hops;
  const uint32_t* list = species ? md.list_dn : md.list_up;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = md.sector ? list[k] : (uint32_t)k;
    // positive-sign targets first, then negative ones (hop order within each group)
    int cnt = 0, np = 0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < ne; ++q) {
        const HopEntry h = md.hops[e0 + q];
        if (((b >> h.i) ^ (b >> h.j)) & 1u) {
          const uint32_t sg = (uint32_t)(__popc(b & h.between) & 1);
          if ((int)sg != pass) continue;
          const uint32_t b2 = b ^ h.mask;
          const uint32_t r2 = md.sector ? md.rank[b2] : b2;
          nbr[(int64_t)cnt * n + k] = r2 | (sg << 31);
          ++cnt;
        }
      }
      if (pass == 0) np = cnt;
    }
    deg[k] = (uint8_t)cnt;
    npos[k] = (uint8_t)np;
  }
}

// difference of two accumulated sums (pass D keeps positive and negative terms apart)
__device__ __forceinline__ IntAcc diff_acc(const IntAcc& p, const IntAcc& n) {
  IntAcc r;
  r.s = p.s - n.s;
  return r;
}
__device__ __forceinline__ F32Acc diff_acc(const F32Acc& p, const F32Acc& n) {
  F32Acc r;
  r.s = p.s - n.s;
  return r;
}

// pass D: W[d][u] = sum over down-spin neighbours d' of d of +-X[d'][u].  Items run
// stripe-major (stripe = kThreads * EPT columns) so one stripe of all rows is the L2
// working set.  Each warp loads the row's neighbour list once (lane q holds entry q) and
// broadcasts it with shuffles, so the data loads of four neighbours issue back to back.
template <class R, int EPT>
__global__ void __launch_bounds__(kThreads) k_hub_dn(const HubDev md, const R* __restrict__ X, R* __restrict__ W,
                                                     const int* __restrict__ done,
                                                     unsigned long long* __restrict__ next_item) {
  using A = typename SumAcc<R>::T;
  if (done != nullptr && *done) return;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int SW = kThreads * EPT;
  const int64_t dim_up = md.dim_up, dim_dn = md.dim_dn;
  const int n_str = (int)((dim_up + SW - 1) / SW);
  const int64_t n_items = (int64_t)n_str * dim_dn;
  const int last_full = (int)(dim_up / SW);  // stripes [0, last_full) need no bounds checks
  // items are handed out in order from a counter, so all CTAs stay on neighbouring rows of
  // one stripe and the stripe of X they gather stays in L2 (static round-robin lets CTAs
  // drift over several stripes)
  __shared__ int64_t s_item;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = (int64_t)atomicAdd(next_item, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= n_items) break;
    const int s = (int)(item / dim_dn);
    const int64_t d = item - (int64_t)s * dim_dn;
    const int deg = md.deg_dn[d];
    const int npos = md.npos_dn[d];
    const int u0 = s * SW + tid;
    const bool full = s < last_full;
    // the list is sign-sorted: entries [0, npos) add, [npos, deg) subtract; each group is
    // summed without per-term sign handling and the two sums are subtracted once
    A accp[EPT], accn[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      accp[j].zero();
      accn[j].zero();
    }
    for (int qb = 0; qb < deg; qb += 32) {
      const int nq = (deg - qb < 32) ? (deg - qb) : 32;
      const uint32_t mine = (lane < nq) ? __ldg(md.nbr_dn + (int64_t)(qb + lane) * dim_dn + d) : 0u;
      for (int q0 = 0; q0 < nq; q0 += 4) {
        R x[4][EPT];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t e = __shfl_sync(0xffffffffu, mine, (q0 + t) & 31);
          const bool on = q0 + t < nq;
          const R* src = X + (int64_t)(e & 0x7fffffffu) * dim_up + u0;
#pragma unroll
          for (int j = 0; j < EPT; ++j) {
            x[t][j] = (R)0;
            if (on && (full || u0 + j * kThreads < dim_up)) x[t][j] = __ldg(src + j * kThreads);
          }
        }
        const int qn = qb + q0;  // list position of t = 0
        if (qn + 4 <= npos) {
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int j = 0; j < EPT; ++j) accp[j].add(x[t][j], false);
        } else if (qn >= npos) {
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int j = 0; j < EPT; ++j) accn[j].add(x[t][j], false);
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int j = 0; j < EPT; ++j) {
              if (qn + t < npos) accp[j].add(x[t][j], false);
              else accn[j].add(x[t][j], false);
            }
        }
      }
    }
    A acc[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) acc[j] = diff_acc(accp[j], accn[j]);
    R* dst = W + d * dim_up + u0;
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (full || u0 + j * kThreads < dim_up) __stcs(dst + j * kThreads, (R)acc[j].value());
    }
  }
}

// pass U: up-spin hops on K rows staged in shared memory, diag, + c_dn W, fused epilogue
template <class R, int K, Epi E, int NT>
__global__ void __launch_bounds__(NT) k_hub_up(const HubDev md, const R* __restrict__ X,
                                                       const R* __restrict__ W, R* __restrict__ w, FusedArgs fa) {
  using A = typename SumAcc<R>::T;
  constexpr bool F64 = sizeof(R) == 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* tile = reinterpret_cast<R*>(smem_raw);
  __shared__ LinGroup s_ulin[kMaxLin];
  __shared__ LinGroup s_mlin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ R s_uc[kMaxLin], s_mc[kMaxLin], s_pcoef[kMaxPairGroups];  // coefficients in R
  __shared__ double s_inv[1];
  __shared__ double s_red[(NT / 32) * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  for (int k = tid; k < md.n_ulin; k += NT) { s_ulin[k] = md.ulin[k]; s_uc[k] = (R)md.ulin[k].coef; }
  for (int k = tid; k < md.n_mulin; k += NT) { s_mlin[k] = md.mulin[k]; s_mc[k] = (R)md.mulin[k].coef; }
  for (int k = tid; k < md.n_pairs; k += NT) s_pair[k] = md.pairs[k];
  for (int k = tid; k < md.n_pair_groups; k += NT) s_pcoef[k] = (R)md.pair_coef[k];
  if constexpr (E == Epi::kTpq) {
    if (tid == 0) s_inv[0] = fa.scal[0];
  }
  EpiScalars es{0.0, 0.0};
  if constexpr (E == Epi::kLanczos1) {
    es.c1 = fa.scal[0];
    es.c2 = fa.scal[1];
  }
  const R c_up = (R)md.c_up, c_dn = (R)md.c_dn;
  const bool same_c = md.c_up == md.c_dn;
  __shared__ R s_dtab[33];
  const bool dtab = md.n_ulin == 1 && md.n_mulin == 0 && md.n_pairs == 0;
  if (dtab && tid <= 32) s_dtab[tid] = (R)(md.c0 + md.ulin[0].coef * (double)tid);
  __syncthreads();
  Red<F64> red;
  red.zero();
  const int64_t dim_up = md.dim_up, dim_dn = md.dim_dn;
  const int64_t n_tiles = (dim_dn + K - 1) / K;

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t d0 = t * K;
    const int nk = (int)((dim_dn - d0 < K) ? (dim_dn - d0) : K);
    __syncthreads();
    // tile[u * K + m] = X[d0 + m][u]: the K rows interleaved, so one vector load per
    // neighbour fetches the value of all K rows
    for (int64_t u = tid; u < dim_up; u += NT) {
      R vals[K];
#pragma unroll
      for (int m = 0; m < K; ++m) vals[m] = (m < nk) ? __ldg(X + (d0 + m) * dim_up + u) : (R)0;
      store_k<R, K>(tile + u * K, vals);
    }
    __syncthreads();
    uint32_t dn[K];
#pragma unroll
    for (int m = 0; m < K; ++m) dn[m] = (m < nk) ? (md.sector ? __ldg(md.list_dn + d0 + m) : (uint32_t)(d0 + m)) : 0u;
    for (int64_t u = tid; u < dim_up; u += NT) {
      const uint32_t up = md.sector ? __ldg(md.list_up + u) : (uint32_t)u;
      const int deg = md.deg_up[u];
      const uint32_t* nb = md.nbr_up + u;
      A acc[K];
#pragma unroll
      for (int m = 0; m < K; ++m) acc[m].zero();
      const int du = (int)dim_up;  // neighbour tables hold < 2^28 entries
      int q = 0;
      for (; q + 2 <= deg; q += 2) {
        const uint32_t e0 = __ldg(nb + q * du), e1 = __ldg(nb + (q + 1) * du);
        R v0[K], v1[K];
        load_k<R, K>(tile + (int)(e0 & 0x7fffffffu) * K, v0);
        load_k<R, K>(tile + (int)(e1 & 0x7fffffffu) * K, v1);
#pragma unroll
        for (int m = 0; m < K; ++m) {
          acc[m].add(v0[m], (e0 >> 31) != 0);
          acc[m].add(v1[m], (e1 >> 31) != 0);
        }
      }
      if (q < deg) {
        const uint32_t e0 = __ldg(nb + q * du);
        R v0[K];
        load_k<R, K>(tile + (int)(e0 & 0x7fffffffu) * K, v0);
#pragma unroll
        for (int m = 0; m < K; ++m) acc[m].add(v0[m], (e0 >> 31) != 0);
      }
#pragma unroll
      for (int m = 0; m < K; ++m) {
        if (m >= nk) break;
        const int64_t idx = (d0 + m) * dim_up + u;
        const R x = tile[u * K + m];
        // diagonal: integer counts times the class coefficients
        R dg;
        if (dtab) {
          dg = s_dtab[__popc(up & dn[m] & (uint32_t)s_ulin[0].mask)];
        } else {
        dg = (R)md.c0;
        for (int g = 0; g < md.n_ulin; ++g) dg += s_uc[g] * (R)__popc(up & dn[m] & (uint32_t)s_ulin[g].mask);
        for (int g = 0; g < md.n_mulin; ++g) {
          const uint32_t mk = (uint32_t)s_mlin[g].mask;
          dg += s_mc[g] * (R)(__popc(up & mk) + __popc(dn[m] & mk));
        }
        if (md.n_pairs) {
          int grp = s_pair[0].grp, cnt = 0;
          for (int p = 0; p < md.n_pairs; ++p) {
            const PairEntry pe = s_pair[p];
            if (pe.grp != grp) {
              dg += s_pcoef[grp] * (R)cnt;
              cnt = 0;
              grp = pe.grp;
            }
            const int ni = (int)((up >> pe.i) & 1u) + (int)((dn[m] >> pe.i) & 1u);
            const int nj = (int)((up >> pe.j) & 1u) + (int)((dn[m] >> pe.j) & 1u);
            cnt += ni * nj;
          }
          dg += s_pcoef[grp] * (R)cnt;
        }
        }
        R hv;
        if (same_c) {
          acc[m].add(W[idx], false);
          hv = dg * x + c_up * (R)acc[m].value();
        } else {
          hv = dg * x + c_up * (R)acc[m].value() + c_dn * W[idx];
        }
        epilogue<R, E>(idx, 0, x, (R)0, hv, (R)0, w, fa, es, s_inv, red);
      }
    }
  }
  if constexpr (E != Epi::kStore) {
    // fixed-order reduction: warp shuffles, then the warps' sums in warp order
    constexpr int nq = n_red<E>();
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < nq; ++q) {
      double x = red.get(q);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) s_red[wid * kMaxRedQ + q] = x;
    }
    __syncthreads();
    if (tid < nq) {
      double x = 0.0;
      for (int k = 0; k < NT / 32; ++k) x += s_red[k * kMaxRedQ + tid];
      fa.partials[(size_t)blockIdx.x * kMaxRedQ + tid] = x;
    }
  }
}

// ------------------------------------------------------------------ fp64 via fixed point
// fp64 vectors take the gather passes as 64-bit integers on one scale per vector:
// q = round(x * 2^(1078 - E)), E = the largest exponent field of x, so |q| < 2^56 and the
// signed sums of up to 127 terms are exact integer additions (two instructions a term on
// the integer pipes instead of one fp64 add each at 1/64 rate).  Each element is rounded
// once, by at most 2^-57 max|x|; the final sums convert back to fp64 exactly rounded.

__global__ void __launch_bounds__(kThreads) k_maxexp(const double* __restrict__ X, int64_t n, int* __restrict__ E,
                                                      const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  int mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    mx = max(mx, (__double2hiint(__ldg(X + i)) >> 20) & 0x7ff);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(E, mx);
}

// extra: headroom bits; q = round(x 2^(1078 - E - extra)), |q| < 2^(56 - extra)
__global__ void __launch_bounds__(kThreads) k_quant(const double* __restrict__ X, long long* __restrict__ Q, int64_t n,
                                                     const int* __restrict__ Ep, const int* __restrict__ done,
                                                     int extra) {
  if (done != nullptr && *done) return;
  const int E = *Ep + extra;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
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

// pass U on quantised rows: K int64 rows interleaved in shared memory; the diagonal term and
// the reductions take each element's value from the same quantised tile
template <int K, Epi E, int NT>
__global__ void __launch_bounds__(NT) k_hub_up_q(const HubDev md,
                                                         const long long* __restrict__ Q,
                                                         const long long* __restrict__ WQ, const int* __restrict__ Ep,
                                                         double* __restrict__ w, FusedArgs fa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  long long* tile = reinterpret_cast<long long*>(smem_raw);
  __shared__ LinGroup s_ulin[kMaxLin];
  __shared__ LinGroup s_mlin[kMaxLin];
  __shared__ PairEntry s_pair[kMaxPairs];
  __shared__ double s_pcoef[kMaxPairGroups];
  __shared__ double s_inv[1];
  __shared__ double s_red[(NT / 32) * kMaxRedQ];

  if (fa.done != nullptr && *fa.done) return;
  const int tid = threadIdx.x;
  for (int k = tid; k < md.n_ulin; k += NT) s_ulin[k] = md.ulin[k];
  for (int k = tid; k < md.n_mulin; k += NT) s_mlin[k] = md.mulin[k];
  for (int k = tid; k < md.n_pairs; k += NT) s_pair[k] = md.pairs[k];
  for (int k = tid; k < md.n_pair_groups; k += NT) s_pcoef[k] = md.pair_coef[k];
  if constexpr (E == Epi::kTpq) {
    if (tid == 0) s_inv[0] = fa.scal[0];
  }
  EpiScalars es{0.0, 0.0};
  if constexpr (E == Epi::kLanczos1) {
    es.c1 = fa.scal[0];
    es.c2 = fa.scal[1];
  }
  const int eoff = *Ep - 1078;
  const bool same_c = md.c_up == md.c_dn;
  // one hopping value of magnitude 2^k (t = 1 in particular): c * fix(a) = fix(+-a) 2^k,
  // an exponent shift instead of an fp64 multiply per element
  const long long cbits = __double_as_longlong(md.c_up);
  const int cexp = (int)((cbits >> 52) & 0x7ff);
  const bool c_p2 = same_c && (cbits & 0xfffffffffffffll) == 0 && cexp > 0 && cexp < 0x7ff;
  const bool c_neg = cbits < 0;
  const int c_l2 = cexp - 1023;
  // With such a hopping the element is computed in units of 2^e2, e2 = eoff + k:
  // hv = (dg 2^-k xr + (+-(acc + wq))) 2^e2 with xr = q as fp64, so the two per-element
  // power-of-two scalings fold into the diagonal table, the Lanczos coefficient and the
  // per-CTA partial sum (both scales must be normal numbers).
  const int e2 = eoff + c_l2;
  const bool fold = c_p2 && eoff >= -1022 && eoff <= 1023 && e2 >= -1022 && e2 <= 1023 &&
                    (E == Epi::kStore || E == Epi::kLanczos1);
  const double s_eoff = fold ? __longlong_as_double((long long)(eoff + 1023) << 52) : 1.0;
  const double s_e2 = fold ? __longlong_as_double((long long)(e2 + 1023) << 52) : 1.0;
  const double r_k = fold ? __longlong_as_double((long long)(1023 - c_l2) << 52) : 1.0;  // 2^-k
  // diagonal = c0 + U * popcount(up & dn & mask) in the common single-group case: table
  __shared__ double s_dtab[33];
  const bool dtab = md.n_ulin == 1 && md.n_mulin == 0 && md.n_pairs == 0;
  if (dtab && tid <= 32) s_dtab[tid] = (md.c0 + md.ulin[0].coef * (double)tid) * r_k;
  __syncthreads();
  Red<true> red;
  red.zero();
  int pmx = 0;  // Lanczos: largest exponent field of the P values written (fa.pexp)
  const int64_t dim_up = md.dim_up, dim_dn = md.dim_dn;
  const int64_t n_tiles = (dim_dn + K - 1) / K;
  const int du = (int)dim_up;

  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t d0 = t * K;
    const int nk = (int)((dim_dn - d0 < K) ? (dim_dn - d0) : K);
    __syncthreads();
    for (int64_t u = tid; u < dim_up; u += NT) {
#pragma unroll
      for (int m = 0; m < K; ++m) tile[u * K + m] = (m < nk) ? __ldg(Q + (d0 + m) * dim_up + u) : 0ll;
    }
    __syncthreads();
    uint32_t dn[K];
#pragma unroll
    for (int m = 0; m < K; ++m) dn[m] = (m < nk) ? (md.sector ? __ldg(md.list_dn + d0 + m) : (uint32_t)(d0 + m)) : 0u;
    for (int64_t u = tid; u < dim_up; u += NT) {
      const uint32_t up = md.sector ? __ldg(md.list_up + u) : (uint32_t)u;
      const int deg = md.deg_up[u];
      const uint32_t* nb = md.nbr_up + u;
      long long acc[K];
#pragma unroll
      for (int m = 0; m < K; ++m) acc[m] = 0;
      for (int q = 0; q < deg; ++q) {
        const uint32_t e = __ldg(nb + q * du);
        const long long* src = tile + (int)(e & 0x7fffffffu) * K;
        const bool neg = (e >> 31) != 0;
        if constexpr (K == 2) {
          const longlong2 v2 = *reinterpret_cast<const longlong2*>(src);
          acc[0] += neg ? -v2.x : v2.x;
          acc[1] += neg ? -v2.y : v2.y;
        } else {
#pragma unroll
          for (int m = 0; m < K; ++m) acc[m] += neg ? -src[m] : src[m];
        }
      }
#pragma unroll
      for (int m = 0; m < K; ++m) {
        if (m >= nk) break;
        const int64_t idx = (d0 + m) * dim_up + u;
        // the row's own value from the quantised tile: H v is then H applied to the
        // quantised vector (each element within 2^-57 max|x| of v, as in the gathers)
        const double xr = __ll2double_rn(tile[u * K + m]);
        double dg;  // (times 2^-k when folding)
        if (dtab) {
          dg = s_dtab[__popc(up & dn[m] & (uint32_t)s_ulin[0].mask)];
        } else {
        dg = md.c0;
        for (int g = 0; g < md.n_ulin; ++g) dg += s_ulin[g].coef * (double)__popc(up & dn[m] & (uint32_t)s_ulin[g].mask);
        for (int g = 0; g < md.n_mulin; ++g) {
          const uint32_t mk = (uint32_t)s_mlin[g].mask;
          dg += s_mlin[g].coef * (double)(__popc(up & mk) + __popc(dn[m] & mk));
        }
        if (md.n_pairs) {
          int grp = s_pair[0].grp, cnt = 0;
          for (int p = 0; p < md.n_pairs; ++p) {
            const PairEntry pe = s_pair[p];
            if (pe.grp != grp) {
              dg += s_pcoef[grp] * (double)cnt;
              cnt = 0;
              grp = pe.grp;
            }
            const int ni = (int)((up >> pe.i) & 1u) + (int)((dn[m] >> pe.i) & 1u);
            const int nj = (int)((up >> pe.j) & 1u) + (int)((dn[m] >> pe.j) & 1u);
            cnt += ni * nj;
          }
          dg += s_pcoef[grp] * (double)cnt;
        }
        if (fold) dg *= r_k;
        }
        const long long wq = __ldg(WQ + idx);
        if (fold) {
          const long long y = c_neg ? -(acc[m] + wq) : acc[m] + wq;
          const double hvu = fma(dg, xr, __ll2double_rn(y));  // hv = hvu 2^e2
          if constexpr (E == Epi::kStore) {
            w[idx] = hvu * s_e2;
          } else if constexpr (E == Epi::kLanczos1) {
            // P <- c1 hv - c2 P; partial <x, hv> in units of 2^(eoff + e2)
            double* P = reinterpret_cast<double*>(fa.out);
            const double* Pin = fa.in ? reinterpret_cast<const double*>(fa.in) : P;
            const double pv = fma(es.c1 * s_e2, hvu, -(es.c2 * Pin[idx]));
            P[idx] = pv;
            pmx = max(pmx, (int)((__double_as_longlong(pv) >> 52) & 0x7ff));
            red.add(0, xr, hvu);
            red.tick();
          }
        } else {
          const double x = fix_to_double(tile[u * K + m], eoff);
          double hv;
          if (c_p2) hv = fma(dg, x, fix_to_double(c_neg ? -(acc[m] + wq) : acc[m] + wq, eoff + c_l2));
          else if (same_c) hv = fma(dg, x, md.c_up * fix_to_double(acc[m] + wq, eoff));
          else hv = fma(dg, x, fma(md.c_up, fix_to_double(acc[m], eoff), md.c_dn * fix_to_double(wq, eoff)));
          if constexpr (E == Epi::kLanczos1) {  // the epilogue's Lanczos step, with the exponent kept
            double* P = reinterpret_cast<double*>(fa.out);
            const double* Pin = fa.in ? reinterpret_cast<const double*>(fa.in) : P;
            const double pv = es.c1 * hv - es.c2 * Pin[idx];
            P[idx] = pv;
            pmx = max(pmx, (int)((__double_as_longlong(pv) >> 52) & 0x7ff));
            red.add(0, x, hv);
            red.tick();
          } else {
            epilogue<double, E>(idx, 0, x, 0.0, hv, 0.0, w, fa, es, s_inv, red);
          }
        }
      }
    }
  }
  if constexpr (E == Epi::kLanczos1) {
    if (fa.pexp != nullptr) {
      pmx = (int)__reduce_max_sync(0xffffffffu, (unsigned)pmx);
      if ((tid & 31) == 0 && pmx > 0) atomicMax(fa.pexp, pmx);
    }
  }
  if constexpr (E != Epi::kStore) {
    constexpr int nq = n_red<E>();
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < nq; ++q) {
      double x = red.get(q);
      if (fold) x = (x * s_eoff) * s_e2;  // back from units of 2^(eoff + e2)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) s_red[wid * kMaxRedQ + q] = x;
    }
    __syncthreads();
    if (tid < nq) {
      double x = 0.0;
      for (int k = 0; k < NT / 32; ++k) x += s_red[k * kMaxRedQ + tid];
      fa.partials[(size_t)blockIdx.x * kMaxRedQ + tid] = x;
    }
  }
}

template <class R>
int pick_k(const HubDev& md) {
  const int64_t row = md.dim_up * (int64_t)sizeof(R);
  int k = 1;
  if (4 * row <= kSmemBudget) k = 4;
  else if (2 * row <= kSmemBudget) k = 2;
  if (md.up_k > 0 && md.up_k < k) k = (md.up_k >= 2) ? 2 : 1;
  return k;
}

int pick_kq(const HubDev& md) {
  int k = (2 * md.dim_up * 8 <= kSmemBudget) ? 2 : 1;
  if (md.up_k == 1) k = 1;
  return k;
}

// pass D launch with the tuned (or default) columns per thread
template <class R>
Status launch_dn(const HubDev& md, const R* X, R* W, const int* done, unsigned long long* counter, cudaStream_t st) {
  int ept = md.dn_ept > 0 ? md.dn_ept : (sizeof(R) == 8 ? HPHI_DN_EPT64 : HPHI_DN_EPT32);
  if (ept != 1 && ept != 2 && ept != 4) ept = 1;
  const int64_t sw = (int64_t)kThreads * ept;
  const int64_t items = ((md.dim_up + sw - 1) / sw) * md.dim_dn;
  const int gd = (int)std::min<int64_t>(items, (int64_t)num_sms() * 8);
  HPHI_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  if (ept == 4) k_hub_dn<R, 4><<<gd, kThreads, 0, st>>>(md, X, W, done, counter);
  else if (ept == 2) k_hub_dn<R, 2><<<gd, kThreads, 0, st>>>(md, X, W, done, counter);
  else k_hub_dn<R, 1><<<gd, kThreads, 0, st>>>(md, X, W, done, counter);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

// pass U threads: 1024 (one CTA per SM) for tiles above ~110 KB, else 512 so two CTAs per
// SM alternate between loading a tile and working on one
inline int up_threads(size_t tile_bytes) { return tile_bytes > 110000 ? 1024 : 512; }

template <class KernelT>
int occupancy_for(KernelT kern, int nt, size_t smem) {
  int n = 0;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, nt, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

template <class R, int K, Epi E>
int up_occupancy(const HubDev& md) {
  const size_t smem = (size_t)K * md.dim_up * sizeof(R);
  return up_threads(smem) == 1024 ? occupancy_for(k_hub_up<R, K, E, 1024>, 1024, smem)
                                  : occupancy_for(k_hub_up<R, K, E, 512>, 512, smem);
}

template <class R, int K, Epi E>
Status launch_up(const HubDev& md, const R* X, const R* W, R* w, const FusedArgs& fa, int grid, cudaStream_t st) {
  const size_t smem = (size_t)K * md.dim_up * sizeof(R);
  if (up_threads(smem) == 1024) {
    HPHI_CUDA_TRY(cudaFuncSetAttribute(k_hub_up<R, K, E, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    k_hub_up<R, K, E, 1024><<<grid, 1024, smem, st>>>(md, X, W, w, fa);
  } else {
    HPHI_CUDA_TRY(cudaFuncSetAttribute(k_hub_up<R, K, E, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget));
    k_hub_up<R, K, E, 512><<<grid, 512, smem, st>>>(md, X, W, w, fa);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

template <int K, Epi E>
int upq_occupancy(const HubDev& md) {
  const size_t smem = (size_t)K * md.dim_up * 8;
  return up_threads(smem) == 1024 ? occupancy_for(k_hub_up_q<K, E, 1024>, 1024, smem)
                                  : occupancy_for(k_hub_up_q<K, E, 512>, 512, smem);
}

// scratch layout of the quantised fp64 path: [Q: dim int64][WQ: dim int64][E: int]
size_t quant_scratch_bytes(const HubDev& md) { return (size_t)16 * md.dim + 256; }

template <Epi E>
Status launch_q(const HubDev& md, const void* v, void* w, void* scratch, const FusedArgs& fa, int grid_up,
                cudaStream_t st) {
  const double* X = reinterpret_cast<const double*>(v);
  long long* Q = reinterpret_cast<long long*>(scratch);
  long long* WQ = Q + md.dim;
  int* Ep = reinterpret_cast<int*>(WQ + md.dim);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(WQ + md.dim) + 1;
  const int gv = (int)std::max<int64_t>(1, std::min<int64_t>((md.dim + kThreads - 1) / kThreads, (int64_t)num_sms() * 8));
  if (!fa.exp_ready) {
    HPHI_CUDA_TRY(cudaMemsetAsync(Ep, 0, sizeof(int), st));
    k_maxexp<<<gv, kThreads, 0, st>>>(X, md.dim, Ep, fa.done);
    HPHI_CUDA_TRY(cudaGetLastError());
  }
  if (fa.exp_ready != 2) {  // 2: the previous Lanczos pass 2 wrote Q and its exponent
    k_quant<<<gv, kThreads, 0, st>>>(X, Q, md.dim, Ep, fa.done, 0);
    HPHI_CUDA_TRY(cudaGetLastError());
  }
  if (fa.pexp != nullptr) HPHI_CUDA_TRY(cudaMemsetAsync(fa.pexp, 0, sizeof(int), st));
  Status sd = launch_dn<long long>(md, Q, WQ, fa.done, counter, st);
  if (sd.code) return sd;
  double* out = reinterpret_cast<double*>(w);
  const int K = pick_kq(md);
  const size_t smem = (size_t)K * md.dim_up * 8;
  const bool big = up_threads(smem) == 1024;
#define HPHI_UPQ(KK, NN)                                                                                          \
  HPHI_CUDA_TRY(cudaFuncSetAttribute(k_hub_up_q<KK, E, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget)); \
  k_hub_up_q<KK, E, NN><<<grid_up, NN, smem, st>>>(md, Q, WQ, Ep, out, fa);
  if (K == 2) {
    if (big) { HPHI_UPQ(2, 1024) } else { HPHI_UPQ(2, 512) }
  } else {
    if (big) { HPHI_UPQ(1, 1024) } else { HPHI_UPQ(1, 512) }
  }
#undef HPHI_UPQ
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

int* hub_exponent_slot_impl(const HubDev& md, void* scratch) {
  return reinterpret_cast<int*>(reinterpret_cast<long long*>(scratch) + 2 * md.dim);
}

int upq_grid(const HubDev& md, Epi epi) {
  const int K = pick_kq(md);
  int occ = 1;
#define HPHI_OCCQ(KK)                                                          \
  switch (epi) {                                                               \
    case Epi::kStore: occ = upq_occupancy<KK, Epi::kStore>(md); break;         \
    case Epi::kLanczos1: occ = upq_occupancy<KK, Epi::kLanczos1>(md); break;   \
    case Epi::kTpq: occ = upq_occupancy<KK, Epi::kTpq>(md); break;             \
    case Epi::kRefine: occ = upq_occupancy<KK, Epi::kRefine>(md); break;       \
  }
  if (K == 2) { HPHI_OCCQ(2) } else { HPHI_OCCQ(1) }
#undef HPHI_OCCQ
  const int64_t tiles = (md.dim_dn + K - 1) / K;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * occ));
}

template <class R, Epi E>
Status launch_r(const HubDev& md, const void* v, void* w, void* scratch, const FusedArgs& fa, int grid_up,
                cudaStream_t st) {
  const R* X = reinterpret_cast<const R*>(v);
  // kStore writes the down-spin sums into w and finishes them in place; the fused steps
  // use the scratch vector
  R* W = (E == Epi::kStore) ? reinterpret_cast<R*>(w) : reinterpret_cast<R*>(scratch);
  // the item counter of pass D sits after the fp32 scratch vector (first bytes of scratch
  // when the scratch holds no vector)
  const size_t voff = (E == Epi::kStore) ? 0 : (((size_t)md.dim * sizeof(R) + 255) / 256) * 256;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + voff);
  Status sd = launch_dn<R>(md, X, W, fa.done, counter, st);
  if (sd.code) return sd;
  R* out = reinterpret_cast<R*>(w);
  switch (pick_k<R>(md)) {
    case 4: return launch_up<R, 4, E>(md, X, W, out, fa, grid_up, st);
    case 2: return launch_up<R, 2, E>(md, X, W, out, fa, grid_up, st);
    default: return launch_up<R, 1, E>(md, X, W, out, fa, grid_up, st);
  }
}

template <class R>
int up_grid_r(const HubDev& md, Epi epi) {
  int occ = 1;
  const int k = pick_k<R>(md);
#define HPHI_OCC(KK)                                                         \
  switch (epi) {                                                             \
    case Epi::kStore: occ = up_occupancy<R, KK, Epi::kStore>(md); break;       \
    case Epi::kLanczos1: occ = up_occupancy<R, KK, Epi::kLanczos1>(md); break; \
    case Epi::kTpq: occ = up_occupancy<R, KK, Epi::kTpq>(md); break;           \
    case Epi::kRefine: occ = up_occupancy<R, KK, Epi::kRefine>(md); break;     \
  }
  if (k == 4) { HPHI_OCC(4) } else if (k == 2) { HPHI_OCC(2) } else { HPHI_OCC(1) }
#undef HPHI_OCC
  const int64_t tiles = (md.dim_dn + k - 1) / k;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * occ));
}

// Device address of g_noalloc_scratch on the current device.  Looked up again on every call
// whose stream is not being captured (the lookup allocates nothing), so a device reset or
// another current context cannot leave a stale address behind; a capturing stream takes the
// address cached by the last such lookup on the device (a graph replays that address anyway).
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

Status noalloc_scratch(void** out, cudaStream_t st) {
  int dev = 0;
  HPHI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return {HPHI_ERR_UNSUPPORTED, "allocation-free path: device ordinal above 63"};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HPHI_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (cs == cudaStreamCaptureStatusNone || g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return {HPHI_ERR_CUDA, std::string("cudaGetSymbolAddress(allocation-free scratch): ") + cudaGetErrorString(e)};
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return {};
}

}  // namespace

HubDev with_shape(const HubDev& md, int prec);

size_t noalloc_capacity_bytes() { return kNoAllocScratchBytes; }

Status launch_hub_store_noalloc(const HubDev& md0, const void* v, void* w, cudaStream_t st) {
  const HubDev md = with_shape(md0, HPHI_FP64);
  const size_t need = quant_scratch_bytes(md);
  if (need > kNoAllocScratchBytes)
    return {HPHI_ERR_INVALID_ARG, "hphi_apply_H_noalloc: the basis needs " + std::to_string(need) +
                                      " bytes of scratch, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                                      " (at most " + std::to_string((kNoAllocScratchBytes - 256) / 16) + " rows)"};
  void* scratch = nullptr;
  Status s = noalloc_scratch(&scratch, st);
  if (s.code) return s;
  FusedArgs fa;  // plain H v: no reductions, no breakdown flag
  return launch_q<Epi::kStore>(md, v, w, scratch, fa, upq_grid(md, Epi::kStore), st);
}

Status launch_quant_vec(const double* X, long long* Q, int64_t n, int* Ep, const int* done, bool exp_ready, int extra,
                        cudaStream_t st) {
  const int gv = (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)num_sms() * 8));
  if (!exp_ready) {
    HPHI_CUDA_TRY(cudaMemsetAsync(Ep, 0, sizeof(int), st));
    k_maxexp<<<gv, kThreads, 0, st>>>(X, n, Ep, done);
    HPHI_CUDA_TRY(cudaGetLastError());
  }
  k_quant<<<gv, kThreads, 0, st>>>(X, Q, n, Ep, done, extra);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status build_hub_neighbours(const HubDev& md, int species, uint32_t* nbr, uint8_t* deg, uint8_t* npos,
                            cudaStream_t st) {
  const int64_t n = species ? md.dim_dn : md.dim_up;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)num_sms() * 8));
  k_hub_nbr<<<g, kThreads, 0, st>>>(md, species, nbr, deg, npos);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

bool hub_fast_ok(const HubDev& md, int prec, bool cplx, int nvec, Epi epi) {
  if (!md.fast || cplx || nvec != 1) return false;
  // fixed-point sums of at most 127 terms (|q| < 2^56) stay exact in 64 bits
  if (prec == HPHI_FP64 && md.maxdeg_up + md.maxdeg_dn > 126) return false;
  if (epi == Epi::kRefine && prec != HPHI_FP64) return false;
  const int64_t row = md.dim_up * (int64_t)(prec == HPHI_FP64 ? 8 : 4);
  return row <= kSmemBudget;
}

// the launch shape of one precision: the autotuner's choice, else the built-in default
HubDev with_shape(const HubDev& md, int prec) {
  HubDev t = md;
  const int i = prec == HPHI_FP64 ? 0 : 1;
  t.dn_ept = md.tuned_ept[i];
  t.up_k = md.tuned_k[i];
  return t;
}

int hub_up_grid(const HubDev& md0, int prec, Epi epi) {
  const HubDev md = with_shape(md0, prec);
  return prec == HPHI_FP64 ? upq_grid(md, epi) : up_grid_r<float>(md, epi);
}

int* hub_exponent_slot(const HubDev& md, void* scratch) { return hub_exponent_slot_impl(md, scratch); }

// Q at the start of the scratch; tail (after WQ) ints: exponent of Q at 0, work counter
// (u64) at 8, the exact exponents of the current / next vector at 16 and 20, pass-1's at 24
QSlots hub_qslots(const HubDev& md, void* scratch) {
  QSlots q;
  if (scratch == nullptr) return q;
  int* tail = hub_exponent_slot_impl(md, scratch);
  q.Q = reinterpret_cast<long long*>(scratch);
  q.eq = tail;
  q.ec[0] = tail + 4;
  q.ec[1] = tail + 5;
  q.ep = tail + 6;
  q.extra = 0;
  return q;
}

size_t hub_scratch_bytes(const HubDev& md, int prec, Epi epi) {
  if (prec == HPHI_FP64) return quant_scratch_bytes(md);
  return (epi == Epi::kStore ? 0 : (((size_t)4 * md.dim + 255) / 256) * 256) + 256;
}

Status launch_hub_fast(const HubDev& md0, int prec, const void* v, void* w, void* scratch, Epi epi,
                       const FusedArgs& fa, int grid_up, cudaStream_t st) {
  const HubDev md = with_shape(md0, prec);
  if (prec == HPHI_FP64) {
    switch (epi) {
      case Epi::kStore: return launch_q<Epi::kStore>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kLanczos1: return launch_q<Epi::kLanczos1>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kTpq: return launch_q<Epi::kTpq>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kRefine: return launch_q<Epi::kRefine>(md, v, w, scratch, fa, grid_up, st);
    }
  } else {
    switch (epi) {
      case Epi::kStore: return launch_r<float, Epi::kStore>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kLanczos1: return launch_r<float, Epi::kLanczos1>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kTpq: return launch_r<float, Epi::kTpq>(md, v, w, scratch, fa, grid_up, st);
      case Epi::kRefine: break;
    }
  }
  return {HPHI_ERR_INVALID_ARG, "two-pass Hubbard path: unsupported precision / epilogue"};
}

}  // namespace hphi
