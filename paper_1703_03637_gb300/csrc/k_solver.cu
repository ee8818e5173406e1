// Streaming Lanczos / mTPQ vector kernels, scalar finalisers and the fp64 tridiagonal
// eigensolver (sections 3.4, 3.5 and appendix A.3).
//
// Lanczos vectors are kept unnormalised: buffer C_k holds w_k with v_k = sigma_k C_k, so the
// normalisation v_{k+1} = w / |w| costs no extra pass (the next H v multiplies by sigma).
// Every reduction ends in a fixed-order fp64 sum over per-CTA partials.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "reduce.cuh"

namespace hphi {

namespace {

// ------------------------------------------------------------------ reductions
__device__ double block_sum(double x, double* sm) {
  const int tid = threadIdx.x;
  sm[tid] = x;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if (tid < off) sm[tid] += sm[tid + off];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

// sum over `grid` partial rows of quantity q of column c, fixed order
__device__ double sum_partials(const double* __restrict__ partials, int grid, int nvec, int c, int q, double* sm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < grid; b += kThreads) s += partials[((size_t)b * nvec + c) * kMaxRedQ + q];
  return block_sum(s, sm);
}

// ------------------------------------------------------------------ Lanczos start
// C <- (storage precision) v0 (if given); P <- 0; partial |C|^2.  Elements counted as reals.
template <class R>
__global__ void __launch_bounds__(kThreads) k_lz_init(const double* __restrict__ v0, R* __restrict__ C, R* __restrict__ P,
                                                       int64_t n_real, double* __restrict__ partials) {
  __shared__ double sm[kThreads];
  double acc = 0.0;
  // four elements per thread and iteration, one grid stride apart (coalesced, loads first)
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_real; i += 4 * stride) {
    R x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      x[u] = k < n_real ? (v0 != nullptr ? (R)v0[k] : C[k]) : (R)0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      if (k < n_real) {
        if (v0 != nullptr) C[k] = x[u];
        P[k] = (R)0;
        acc = fma((double)x[u], (double)x[u], acc);
      }
    }
  }
  const double t = block_sum(acc, sm);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxRedQ] = t;
}

// mode 0: after init (sigma_0); mode 1: after pass 1 (alpha_k); mode 2: after pass 2 (beta_{k+1});
// mode 3: after pass 2 of the replayed second pass (same recurrence; stops after the last step
// whose Ritz coefficient matters and leaves the first pass's step count alone)
__global__ void __launch_bounds__(kThreads) k_lz_fin(LzDev lz, int mode, int k, double brk,
                                                      const double* __restrict__ partials, int grid) {
  __shared__ double sm[kThreads];
  if (mode != 0 && *lz.done) return;
  const double sum = sum_partials(partials, grid, 1, 0, 0, sm);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    const double sg = (sum > 0.0) ? 1.0 / sqrt(sum) : 0.0;
    lz.sig[0] = sg;
    lz.s[0] = sg;    // c1 = sigma_0
    lz.s[1] = 0.0;   // c2 = beta_0 sigma_{-1} = 0
    *lz.done = (sum > 0.0) ? 0 : 1;
    *lz.steps_done = 0;
  } else if (mode == 1) {
    const double sg = lz.sig[k];
    const double a = sum * sg * sg;  // alpha_k = (H v_k, v_k)
    lz.alpha[k] = a;
    lz.s[2] = a * sg;                // gamma: P <- P - alpha_k v_k = P - gamma C_k
    lz.s[3] = lz.coef[k] * sg;       // Ritz coefficient of v_k (refinement pass)
  } else {
    const double b = sqrt(sum);      // beta_{k+1} = |w|
    const double a = lz.alpha[k];
    lz.beta[k] = b;
    *lz.steps_done = (mode == 2) ? k + 1 : (int)lz.s[5];
    if (!(b > brk * fmax(1.0, fabs(a))) || (mode == 3 && k >= (int)lz.s[4])) {
      *lz.done = 1;
    } else {
      const double sg = 1.0 / b;
      lz.sig[k + 1] = sg;
      lz.s[0] = sg;                  // c1 = sigma_{k+1}
      lz.s[1] = b * lz.sig[k];       // c2 = beta_{k+1} sigma_k
    }
  }
}

// P <- P - gamma C ; partial |P|^2 ; optionally x += xc * C (fp64 accumulator); optionally
// (emax) the largest exponent field of the new P, which the next step's quantisation needs
// q = round(p 2^(1078 - E)) by integer operations on the bits of p (|q| < 2^56 when the
// exponent field of p is at most E); the same rounding as the quantisation kernels
__device__ __forceinline__ long long quant_bits(double p, int E) {
  const int hi = __double2hiint(p);
  const unsigned lo = (unsigned)__double2loint(p);
  const int ex = (hi >> 20) & 0x7ff;
  long long q = 0;
  if (ex != 0) {
    const long long M = ((long long)((hi & 0xfffff) | 0x100000) << 32) | (long long)lo;  // p = M 2^(ex-1075)
    const int sh = E - ex - 3;                                                           // q = M 2^-sh
    if (sh <= 0) q = M << (-sh);
    else if (sh < 62) q = (M + (1ll << (sh - 1))) >> sh;
    if (hi < 0) q = -q;
  }
  return q;
}

// With Q: the next step's quantised copy is written here instead of by a separate pass.  Its
// exponent must be fixed before any element is seen, so it is a bound: |P - gamma C| <
// 2^(EP - 1022) + |gamma| 2^(EC - 1022), EP the largest exponent field pass 1 wrote, EC the
// exact one of C, so E = max(EP, EC + e_gamma - 1022) + 1 is at least the exponent field of
// every new element; the scale is then at most two bits coarser than the exact maximum's
// (each element moves by at most 2^-55 max|P| instead of 2^-57).
template <class R, bool X>
__global__ void __launch_bounds__(kThreads) k_lz_pass2(LzDev lz, const R* __restrict__ C, R* __restrict__ P,
                                                        double* __restrict__ x, int64_t n_real,
                                                        double* __restrict__ partials, int* __restrict__ emax,
                                                        QNext qn) {
  constexpr bool F64 = sizeof(R) == 8;
  __shared__ double sm[kThreads];
  if (*lz.done) return;
  const double g = lz.s[2];
  const R gr = (R)g;
  const double xc = X ? lz.s[3] : 0.0;
  int Eq = 0;
  if (F64 && qn.Q != nullptr) {
    const int eg = (int)((__double_as_longlong(g) >> 52) & 0x7ff);
    const int ec = *qn.ec_cur;
    int eb = *qn.ep;
    if (eg != 0 && ec != 0) eb = max(eb, ec + eg - 1022);
    eb = min(eb + 1, 2046);
    Eq = eb + qn.extra;
    if (blockIdx.x == 0 && threadIdx.x == 0) *qn.eq = eb;
  }
  Red<F64, 1> red;  // one reduced quantity, |P|^2
  red.zero();
  int mx = 0;
  // four elements per thread and iteration, one grid stride apart (coalesced, loads first)
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_real; i += 4 * stride) {
    R c[4], pp[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      c[u] = k < n_real ? C[k] : (R)0;
      pp[u] = k < n_real ? P[k] : (R)0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      if (k < n_real) {
        const R p = pp[u] - gr * c[u];
        P[k] = p;
        red.add(0, p, p);
        red.tick();
        if (X) x[k] = fma(xc, (double)c[u], x[k]);
        if constexpr (F64) {
          mx = max(mx, (int)((__double_as_longlong((double)p) >> 52) & 0x7ff));
          if (qn.Q != nullptr) qn.Q[k] = quant_bits((double)p, Eq);
        }
      }
    }
  }
  if (F64 && emax != nullptr) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(emax, mx);
  }
  const double t = block_sum(red.get(0), sm);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxRedQ] = t;
}

// ------------------------------------------------------------------ tridiagonal eigensolver
// Number of eigenvalues of T (diag a[0..n-1], off-diag b[0..n-2]) smaller than x, by the
// Sturm sequence of the LDL^T pivots.
__device__ int sturm_count(const double* __restrict__ a, const double* __restrict__ b, int n, double x, double pivmin) {
  int cnt = 0;
  double q = a[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = (a[i] - x) - (b[i - 1] * b[i - 1]) / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Gershgorin interval of T_n (widened by a few ulps) and the pivot floor of the Sturm count
struct TriBounds {
  double lo, hi, scale, pivmin;
};
__device__ TriBounds tri_bounds(const double* a, const double* b, int n) {
  double lo = a[0], hi = a[0], bmax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
    if (i + 1 < n) bmax = fmax(bmax, fabs(b[i]));
  }
  TriBounds t;
  t.scale = fmax(fabs(lo), fabs(hi));
  t.pivmin = fmax(1e-300, 2.2250738585072014e-308 * fmax(1.0, bmax * bmax));
  t.lo = lo - (2.2e-16 * t.scale + 1e-300);
  t.hi = hi + (2.2e-16 * t.scale + 1e-300);
  return t;
}

// eigenvalue j (ascending, j < n) of T_n by one warp: 33-section of the bracket until it is a
// few ulps wide; every lane returns it
__device__ double tri_eigenvalue(const double* a, const double* b, int n, int j, const TriBounds& t, int lane) {
  double x0 = t.lo, x1 = t.hi;
  for (int it = 0; it < 64; ++it) {
    if (x1 - x0 <= 4.0 * 2.2204460492503131e-16 * fmax(fabs(x0), fabs(x1)) + 1e-300) break;
    const double x = x0 + (x1 - x0) * (double)(lane + 1) / 33.0;
    const int cnt = sturm_count(a, b, n, x, t.pivmin);
    // points with cnt <= j lie left of eigenvalue j
    const unsigned left = __ballot_sync(0xffffffffu, cnt <= j);
    const int nl = __popc(left);  // points are increasing in lane order
    double nx0 = x0, nx1 = x1;
    const double xl = __shfl_sync(0xffffffffu, x, nl > 0 ? nl - 1 : 0);
    const double xr = __shfl_sync(0xffffffffu, x, nl < 32 ? nl : 31);
    if (nl > 0) nx0 = xl;
    if (nl < 32) nx1 = xr;
    x0 = nx0;
    x1 = nx1;
  }
  return 0.5 * (x0 + x1);
}

// Convergence test of appendix C, one warp, after the fused step that made T_n: the first
// excited eigenvalue of T_n against its value at the previous test; when they agree to eps
// (relative) the run is done (the remaining steps' kernels return at once).  s[6] previous
// value, s[7] tests so far, s[8] 1 when the test stopped the run.
__global__ void k_lz_conv(LzDev lz, double eps) {
  if (*lz.done) return;
  const int n = *lz.steps_done;
  const int lane = threadIdx.x & 31;
  if (n < 2) return;
  const TriBounds t = tri_bounds(lz.alpha, lz.beta, n);
  const double e1 = tri_eigenvalue(lz.alpha, lz.beta, n, 1, t, lane);
  if (lane != 0) return;
  if (lz.s[7] > 0.0 && fabs(e1 - lz.s[6]) <= eps * fabs(e1)) {
    *lz.done = 1;
    lz.s[8] = 1.0;
  }
  lz.s[6] = e1;
  lz.s[7] += 1.0;
}

// One warp per wanted eigenvalue (tri_eigenvalue).  Then (warp 0, lane 0, if asked) inverse
// iteration for the lowest eigenvector of T with partial-pivoting tridiagonal LU.
__global__ void k_tridiag(LzDev lz, int n_eig, int want_vec, double tail_tol, double* __restrict__ work) {
  const int n = *lz.steps_done;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* a = lz.alpha;
  const double* b = lz.beta;
  if (n <= 0) return;
  const TriBounds tb = tri_bounds(a, b, n);
  const double scale = tb.scale;
  if (warp < n_eig) {
    const int j = warp;
    if (j >= n) {
      if (lane == 0) lz.tri[j] = nan("");
    } else {
      const double e = tri_eigenvalue(a, b, n, j, tb, lane);
      if (lane == 0) lz.tri[j] = e;
    }
  }
  if (!want_vec) return;
  __syncthreads();
  if (threadIdx.x != 0) return;
  // inverse iteration: (T - lambda I) y = y_prev, LU with partial pivoting (two superdiagonals)
  const double lam = lz.tri[0];
  double* d = work;            // diagonal of U
  double* e1 = work + n;       // first superdiagonal of U
  double* e2 = work + 2 * n;   // second superdiagonal of U (from pivoting)
  double* l = work + 3 * n;    // multipliers
  int* piv = reinterpret_cast<int*>(work + 4 * n);
  double* y = lz.coef;
  const double eps = 2.2204460492503131e-16 * fmax(scale, 1e-300);
  // factor
  double dd = a[0] - lam, ee = (n > 1) ? b[0] : 0.0;
  for (int i = 0; i < n; ++i) {
    if (i == n - 1) {
      d[i] = (fabs(dd) < eps) ? eps : dd;
      e1[i] = 0.0;
      e2[i] = 0.0;
      piv[i] = 0;
      break;
    }
    const double sub = b[i];
    const double nd = a[i + 1] - lam;
    const double ne = (i + 2 < n) ? b[i + 1] : 0.0;
    if (fabs(dd) >= fabs(sub)) {
      const double piv_d = (fabs(dd) < eps) ? eps : dd;
      const double m = sub / piv_d;
      d[i] = piv_d; e1[i] = ee; e2[i] = 0.0; l[i] = m; piv[i] = 0;
      dd = nd - m * ee;
      ee = ne;
    } else {
      const double m = dd / sub;
      d[i] = sub; e1[i] = nd; e2[i] = ne; l[i] = m; piv[i] = 1;
      dd = ee - m * nd;
      ee = -m * ne;
    }
  }
  for (int i = 0; i < n; ++i) y[i] = 1.0;
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply L^{-1} with the recorded row swaps
    for (int i = 0; i + 1 < n; ++i) {
      if (piv[i]) {
        const double t = y[i];
        y[i] = y[i + 1];
        y[i + 1] = t - l[i] * y[i];
      } else {
        y[i + 1] -= l[i] * y[i];
      }
    }
    // back substitution with U
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      if (i + 1 < n) t -= e1[i] * y[i + 1];
      if (i + 2 < n) t -= e2[i] * y[i + 2];
      y[i] = t / d[i];
    }
    double nrm = 0.0, big = 0.0;
    for (int i = 0; i < n; ++i) {
      nrm += y[i] * y[i];
      if (fabs(y[i]) > fabs(big)) big = y[i];
    }
    const double sc = (big < 0 ? -1.0 : 1.0) / sqrt(nrm);
    for (int i = 0; i < n; ++i) y[i] *= sc;
  }
  // last step whose Ritz coefficients still matter: the replayed second pass can stop once
  // the remaining weight sum_{j > cut} y_j^2 is below tail_tol (the square of the relative
  // change it makes to the unit Ritz vector: below the rounding of the stored vectors)
  double tail = 0.0;
  int cut = n - 1;
  for (int i = n - 1; i >= 0; --i) {
    tail += y[i] * y[i];
    if (tail > tail_tol) {
      cut = i;
      break;
    }
  }
  lz.s[4] = (double)cut;
  lz.s[5] = (double)n;  // the first pass's step count, restored by the replay's finalisers
}

// ------------------------------------------------------------------ Ritz vector from a stored basis
// x = sum_{k < n} coef_k sigma_k V_k, V_k the unnormalised Lanczos vectors kept in HBM
// (stride_real reals apart); fp64 accumulation, one streaming read of the basis.
template <class R>
__global__ void __launch_bounds__(kThreads) k_lz_combine(LzDev lz, const R* __restrict__ V, int64_t n_real,
                                                          int64_t stride_real, double* __restrict__ x) {
  __shared__ double s_c[4096];
  const int n = *lz.steps_done;
  for (int k = threadIdx.x; k < n; k += kThreads) s_c[k] = lz.coef[k] * lz.sig[k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_real; i += (int64_t)gridDim.x * kThreads) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(s_c[k], (double)V[(int64_t)k * stride_real + i], acc);
    x[i] = acc;
  }
}

// ------------------------------------------------------------------ full reorthogonalisation
// After pass 2 of step k (kept basis: slot j holds C_j, v_j = sigma_j C_j; slot k + 1 holds the
// new P): P <- P - sum_{j <= k} <v_j, P> v_j = P - sum_j sigma_j^2 <C_j, P> C_j, every inner
// product and every update accumulated in fp64 (classical Gram-Schmidt against the whole kept
// basis), then |P|^2 for beta_{k+1}.  Inner products run kRoChunk vectors per pass over P.
constexpr int kRoChunk = 16;

template <class R, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_ro_dots(LzDev lz, const R* __restrict__ V, int64_t stride_real,
                                                       int64_t n_elem, int j0, int nj, const R* __restrict__ P,
                                                       double* __restrict__ part) {
  constexpr int W = CPLX ? 2 : 1;
  constexpr int NQ = W * kRoChunk;
  __shared__ double s_part[kThreads / 32][NQ];
  if (*lz.done) return;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_elem; i += (int64_t)gridDim.x * kThreads) {
    const double pr = (double)P[W * i], pi = CPLX ? (double)P[W * i + 1] : 0.0;
#pragma unroll
    for (int j = 0; j < kRoChunk; ++j) {
      if (j < nj) {
        const R* c = V + (int64_t)(j0 + j) * stride_real + W * i;
        const double cr = (double)c[0];
        if constexpr (CPLX) {
          const double ci = (double)c[1];
          acc[2 * j] = fma(cr, pr, fma(ci, pi, acc[2 * j]));        // Re conj(c) p
          acc[2 * j + 1] = fma(cr, pi, fma(-ci, pr, acc[2 * j + 1]));  // Im conj(c) p
        } else {
          acc[j] = fma(cr, pr, acc[j]);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = acc[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) s_part[wid][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += s_part[w][threadIdx.x];
    part[(size_t)blockIdx.x * NQ + threadIdx.x] = t;
  }
}

// coefficient of C_j: sigma_j^2 <C_j, P> (re, im)
__global__ void __launch_bounds__(kThreads) k_ro_fin(LzDev lz, int j0, int nj, int nq_per_vec,
                                                      const double* __restrict__ part, int grid) {
  __shared__ double sm[kThreads];
  if (*lz.done) return;
  const int NQ = nq_per_vec * kRoChunk;
  for (int q = 0; q < nj * nq_per_vec; ++q) {
    double t = 0.0;
    for (int b = threadIdx.x; b < grid; b += kThreads) t += part[(size_t)b * NQ + q];
    t = block_sum(t, sm);
    if (threadIdx.x == 0) {
      const int j = j0 + q / nq_per_vec;
      const double sg = lz.sig[j];
      lz.ro[2 * j + (q % nq_per_vec)] = sg * sg * t;
      if (nq_per_vec == 1) lz.ro[2 * j + 1] = 0.0;
    }
  }
}

template <class R, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_ro_update(LzDev lz, const R* __restrict__ V, int64_t stride_real,
                                                         int64_t n_elem, int k, R* __restrict__ P,
                                                         double* __restrict__ partials) {
  constexpr int W = CPLX ? 2 : 1;
  extern __shared__ double s_ro[];  // [2 (k + 1)]
  __shared__ double sm[kThreads];
  if (*lz.done) return;
  for (int j = threadIdx.x; j < 2 * (k + 1); j += kThreads) s_ro[j] = lz.ro[j];
  __syncthreads();
  double pp = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_elem; i += (int64_t)gridDim.x * kThreads) {
    double pr = (double)P[W * i], pi = CPLX ? (double)P[W * i + 1] : 0.0;
    for (int j = 0; j <= k; ++j) {
      const R* c = V + (int64_t)j * stride_real + W * i;
      const double cr = (double)c[0];
      if constexpr (CPLX) {
        const double ci = (double)c[1];
        const double ar = s_ro[2 * j], ai = s_ro[2 * j + 1];
        pr = fma(-ar, cr, fma(ai, ci, pr));
        pi = fma(-ar, ci, fma(-ai, cr, pi));
      } else {
        pr = fma(-s_ro[2 * j], cr, pr);
      }
    }
    const R qr = (R)pr;
    P[W * i] = qr;
    pp = fma((double)qr, (double)qr, pp);
    if constexpr (CPLX) {
      const R qi = (R)pi;
      P[W * i + 1] = qi;
      pp = fma((double)qi, (double)qi, pp);
    }
  }
  const double t = block_sum(pp, sm);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxRedQ] = t;
}

// ------------------------------------------------------------------ refinement
__global__ void k_refine_fin(LzDev lz, const double* __restrict__ partials, int grid, int which) {
  __shared__ double sm[kThreads];
  if (which == 0) {
    const double xh = sum_partials(partials, grid, 1, 0, 0, sm);
    const double xx = sum_partials(partials, grid, 1, 0, 1, sm);
    const double hh = sum_partials(partials, grid, 1, 0, 2, sm);
    if (threadIdx.x == 0) {
      const double e = xh / xx;
      lz.tri[8] = e;
      lz.tri[10] = hh / xx - e * e;
      lz.tri[11] = xx;
    }
  } else {
    const double rr = sum_partials(partials, grid, 1, 0, 0, sm);
    if (threadIdx.x == 0) lz.tri[9] = sqrt(rr / lz.tri[11]);
  }
}

__global__ void __launch_bounds__(kThreads) k_refine_resid(const double* __restrict__ x, const double* __restrict__ hx,
                                                            int64_t n_real, LzDev lz, double* __restrict__ partials) {
  __shared__ double sm[kThreads];
  const double e = lz.tri[8];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_real; i += (int64_t)gridDim.x * kThreads) {
    const double r = hx[i] - e * x[i];
    acc = fma(r, r, acc);
  }
  const double t = block_sum(acc, sm);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxRedQ] = t;
}

// ------------------------------------------------------------------ mTPQ
// X <- (storage precision) psi0 (if given); per-column partial |X|^2.  nvec divides kThreads.
template <class R, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_tpq_init(const double* __restrict__ psi0, R* __restrict__ X,
                                                        int64_t n_rows, int nvec, double* __restrict__ partials) {
  __shared__ double sm[kThreads];
  const int W = CPLX ? 2 : 1;
  const int64_t n_elem = n_rows * nvec;
  double acc = 0.0;
  const int c = threadIdx.x % nvec;
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * kThreads) {
    for (int w = 0; w < W; ++w) {
      const int64_t i = e * W + w;
      R x;
      if (psi0 != nullptr) {
        x = (R)psi0[i];
        X[i] = x;
      } else {
        x = X[i];
      }
      acc = fma((double)x, (double)x, acc);
    }
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int off = kThreads / 2; off >= nvec; off >>= 1) {
    if (threadIdx.x < off) sm[threadIdx.x] += sm[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < nvec) partials[((size_t)blockIdx.x * nvec + c) * kMaxRedQ] = sm[threadIdx.x];
}

// one CTA per column; mode 0: initial norms; mode 1: records of step k
__global__ void __launch_bounds__(kThreads) k_tpq_fin(TpqDev tq, int mode, int k, int nvec, double inv_ns, double l,
                                                       const double* __restrict__ partials, int grid) {
  __shared__ double sm[kThreads];
  const int c = blockIdx.x;
  if (mode == 0) {
    const double n2 = sum_partials(partials, grid, nvec, c, 0, sm);
    if (threadIdx.x == 0) {
      tq.n2[c] = n2;
      tq.inv[c] = 1.0 / sqrt(n2);
    }
    return;
  }
  const double xy = sum_partials(partials, grid, nvec, c, 0, sm);
  const double yy = sum_partials(partials, grid, nvec, c, 1, sm);
  if (threadIdx.x == 0) {
    const double n2 = tq.n2[c];
    const size_t o = (size_t)k * nvec + c;
    const double u = xy * inv_ns / n2, h2 = yy * inv_ns * inv_ns / n2;
    // |(l - H/N_s) psi_k|^2 for the unit psi_k; positive for l above the spectrum per site
    const double nn = fmax(l * l - 2.0 * l * u + h2, 2.2250738585072014e-308);
    tq.u[o] = u;
    tq.h2[o] = h2;
    tq.nrm[o] = sqrt(nn);
    tq.n2[c] = nn;
    tq.inv[c] = 1.0 / sqrt(nn);
  }
}

// Diagonal observables of the TPQ state (section 3.5: a local quantity at beta_k is its
// expectation in psi_k per site).  Per column: S0 = sum |x|^2, S1 = sum |x|^2 D(s),
// S2 = sum |x|^2 M(s), S3 = sum |x|^2 M(s)^2 with D the number of doubly occupied sites and
// M = 2 S^z_total (an integer) of configuration s.  nvec divides kThreads.
template <class R, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_tpq_obs(const ObsDev od, const R* __restrict__ X, int lg_nvec,
                                                       double* __restrict__ partials) {
  __shared__ double sm[kThreads];
  const int nvec = 1 << lg_nvec;
  const int64_t n_elem = od.dim << lg_nvec;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int c = threadIdx.x & (nvec - 1);
  for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * kThreads) {
    const int64_t row = e >> lg_nvec;
    double w;
    if constexpr (CPLX) {
      const double xr = (double)X[2 * e], xi = (double)X[2 * e + 1];
      w = fma(xr, xr, xi * xi);
    } else {
      const double x = (double)X[e];
      w = x * x;
    }
    int dbl = 0, m2 = 0;
    switch (od.kind) {
      case 0:  // spin, all 2^N configurations: s = row
        m2 = 2 * __popcll((unsigned long long)row) - od.n_sites;
        break;
      case 1:  // spin, fixed popcount
        m2 = 2 * od.n_ones - od.n_sites;
        break;
      default: {  // Hubbard: row = d * dim_up + u
        const int64_t d = row / od.dim_up;
        const int64_t u = row - d * od.dim_up;
        const uint32_t up = od.list_up ? __ldg(od.list_up + u) : (uint32_t)u;
        const uint32_t dn = od.list_dn ? __ldg(od.list_dn + d) : (uint32_t)d;
        dbl = __popc(up & dn);
        m2 = __popc(up) - __popc(dn);
      }
    }
    a0 += w;
    a1 = fma(w, (double)dbl, a1);
    a2 = fma(w, (double)m2, a2);
    a3 = fma(w, (double)(m2 * m2), a3);
  }
  const double acc[4] = {a0, a1, a2, a3};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __syncthreads();
    sm[threadIdx.x] = acc[q];
    __syncthreads();
    for (int off = kThreads / 2; off >= nvec; off >>= 1) {
      if (threadIdx.x < off) sm[threadIdx.x] += sm[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x < nvec) partials[((size_t)blockIdx.x * nvec + c) * kMaxRedQ + q] = sm[threadIdx.x];
  }
}

// one CTA per column: the per-site observables of record k
__global__ void __launch_bounds__(kThreads) k_tpq_obs_fin(TpqDev tq, int k, int nvec, double inv_ns,
                                                           const double* __restrict__ partials, int grid) {
  __shared__ double sm[kThreads];
  const int c = blockIdx.x;
  const double s0 = sum_partials(partials, grid, nvec, c, 0, sm);
  const double s1 = sum_partials(partials, grid, nvec, c, 1, sm);
  const double s2 = sum_partials(partials, grid, nvec, c, 2, sm);
  const double s3 = sum_partials(partials, grid, nvec, c, 3, sm);
  if (threadIdx.x == 0) {
    const size_t o = (size_t)k * nvec + c;
    tq.doub[o] = s1 / s0 * inv_ns;
    tq.sz[o] = 0.5 * s2 / s0 * inv_ns;
    tq.sz2[o] = 0.25 * s3 / s0 * inv_ns;
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers
Status launch_lz_init(int prec, bool cplx, const void* v0_f64, void* C, void* P, int64_t n_real, double* partials,
                      int grid, cudaStream_t st) {
  (void)cplx;
  if (prec == HPHI_FP64)
    k_lz_init<double><<<grid, kThreads, 0, st>>>(reinterpret_cast<const double*>(v0_f64), reinterpret_cast<double*>(C),
                                                 reinterpret_cast<double*>(P), n_real, partials);
  else
    k_lz_init<float><<<grid, kThreads, 0, st>>>(reinterpret_cast<const double*>(v0_f64), reinterpret_cast<float*>(C),
                                                reinterpret_cast<float*>(P), n_real, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_init_fin(const LzDev& lz, const double* partials, int grid, cudaStream_t st) {
  k_lz_fin<<<1, kThreads, 0, st>>>(lz, 0, 0, 0.0, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_fin1(const LzDev& lz, int k, const double* partials, int grid, cudaStream_t st) {
  k_lz_fin<<<1, kThreads, 0, st>>>(lz, 1, k, 0.0, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_pass2(int prec, bool cplx, const LzDev& lz, int k, const void* C, void* P, double* x, int64_t n_real,
                       double* partials, int grid, int* emax, cudaStream_t st, const QNext* qn) {
  (void)cplx;
  (void)k;
  QNext q{nullptr, nullptr, nullptr, nullptr, 0};
  if (qn != nullptr && prec == HPHI_FP64 && !cplx) q = *qn;
  if (prec == HPHI_FP64) {
    if (x)
      k_lz_pass2<double, true><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const double*>(C),
                                                          reinterpret_cast<double*>(P), x, n_real, partials, emax, q);
    else
      k_lz_pass2<double, false><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const double*>(C),
                                                           reinterpret_cast<double*>(P), x, n_real, partials, emax, q);
  } else {
    if (x)
      k_lz_pass2<float, true><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const float*>(C),
                                                         reinterpret_cast<float*>(P), x, n_real, partials, nullptr, q);
    else
      k_lz_pass2<float, false><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const float*>(C),
                                                          reinterpret_cast<float*>(P), x, n_real, partials, nullptr, q);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_fin2(const LzDev& lz, int k, double brk, const double* partials, int grid, bool replay,
                      cudaStream_t st) {
  k_lz_fin<<<1, kThreads, 0, st>>>(lz, replay ? 3 : 2, k, brk, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_conv(const LzDev& lz, double eps, cudaStream_t st) {
  k_lz_conv<<<1, 32, 0, st>>>(lz, eps);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tridiag(const LzDev& lz, int m_max, int n_eig, bool want_vec, double tail_tol, cudaStream_t st) {
  (void)m_max;
  k_tridiag<<<1, 32 * 8, 0, st>>>(lz, n_eig, want_vec ? 1 : 0, tail_tol, lz.tri + 16);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_lz_combine(int prec, const LzDev& lz, const void* V, int64_t n_real, int64_t stride_real, double* x,
                         int grid, cudaStream_t st) {
  if (prec == HPHI_FP64)
    k_lz_combine<double><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const double*>(V), n_real, stride_real, x);
  else
    k_lz_combine<float><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const float*>(V), n_real, stride_real, x);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

size_t ro_part_doubles(int grid) { return (size_t)grid * 2 * kRoChunk; }

Status launch_reorth(int prec, bool cplx, const LzDev& lz, int k, const void* V, int64_t n_real, int64_t stride_real,
                     void* P, double* part, double* partials, int grid, cudaStream_t st) {
  const int64_t n_elem = cplx ? n_real / 2 : n_real;
  const int nqv = cplx ? 2 : 1;
  const size_t smem = sizeof(double) * 2 * (size_t)(k + 1);
#define HPHI_RO(RR, CC)                                                                                              \
  for (int j0 = 0; j0 <= k; j0 += kRoChunk) {                                                                        \
    const int nj = std::min(kRoChunk, k + 1 - j0);                                                                   \
    k_ro_dots<RR, CC><<<grid, kThreads, 0, st>>>(lz, reinterpret_cast<const RR*>(V), stride_real, n_elem, j0, nj,    \
                                                 reinterpret_cast<const RR*>(P), part);                             \
    k_ro_fin<<<1, kThreads, 0, st>>>(lz, j0, nj, nqv, part, grid);                                                   \
  }                                                                                                                  \
  HPHI_CUDA_TRY(cudaFuncSetAttribute(k_ro_update<RR, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));  \
  k_ro_update<RR, CC><<<grid, kThreads, smem, st>>>(lz, reinterpret_cast<const RR*>(V), stride_real, n_elem, k,      \
                                                    reinterpret_cast<RR*>(P), partials);
  if (prec == HPHI_FP64) {
    if (cplx) { HPHI_RO(double, true) } else { HPHI_RO(double, false) }
  } else {
    if (cplx) { HPHI_RO(float, true) } else { HPHI_RO(float, false) }
  }
#undef HPHI_RO
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

int reorth_launches(int k) { return 2 * ((k + kRoChunk) / kRoChunk) + 1; }

Status launch_refine_fin(const LzDev& lz, const double* partials, int grid, int which, cudaStream_t st) {
  k_refine_fin<<<1, kThreads, 0, st>>>(lz, partials, grid, which);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_refine_resid(bool cplx, const double* x, const double* hx, int64_t n_real, const LzDev& lz,
                           double* partials, int grid, cudaStream_t st) {
  (void)cplx;
  k_refine_resid<<<grid, kThreads, 0, st>>>(x, hx, n_real, lz, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tpq_init(int prec, bool cplx, const void* psi0_f64, void* X, int64_t n_rows, int nvec, double* partials,
                       int grid, cudaStream_t st) {
  const double* p = reinterpret_cast<const double*>(psi0_f64);
  if (prec == HPHI_FP64) {
    if (cplx) k_tpq_init<double, true><<<grid, kThreads, 0, st>>>(p, reinterpret_cast<double*>(X), n_rows, nvec, partials);
    else k_tpq_init<double, false><<<grid, kThreads, 0, st>>>(p, reinterpret_cast<double*>(X), n_rows, nvec, partials);
  } else {
    if (cplx) k_tpq_init<float, true><<<grid, kThreads, 0, st>>>(p, reinterpret_cast<float*>(X), n_rows, nvec, partials);
    else k_tpq_init<float, false><<<grid, kThreads, 0, st>>>(p, reinterpret_cast<float*>(X), n_rows, nvec, partials);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tpq_init_fin(const TpqDev& tq, int nvec, const double* partials, int grid, cudaStream_t st) {
  k_tpq_fin<<<nvec, kThreads, 0, st>>>(tq, 0, 0, nvec, 0.0, 0.0, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tpq_fin(const TpqDev& tq, int k, int nvec, double inv_ns, double l, const double* partials, int grid,
                      cudaStream_t st) {
  k_tpq_fin<<<nvec, kThreads, 0, st>>>(tq, 1, k, nvec, inv_ns, l, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tpq_obs(int prec, bool cplx, const ObsDev& od, const void* X, int nvec, double* partials, int grid,
                      cudaStream_t st) {
  int lg = 0;
  while ((1 << lg) < nvec) ++lg;
  if ((1 << lg) != nvec || nvec > kThreads) return {HPHI_ERR_INVALID_ARG, "tpq observables: nvec a power of two <= 256"};
  if (prec == HPHI_FP64) {
    if (cplx) k_tpq_obs<double, true><<<grid, kThreads, 0, st>>>(od, reinterpret_cast<const double*>(X), lg, partials);
    else k_tpq_obs<double, false><<<grid, kThreads, 0, st>>>(od, reinterpret_cast<const double*>(X), lg, partials);
  } else {
    if (cplx) k_tpq_obs<float, true><<<grid, kThreads, 0, st>>>(od, reinterpret_cast<const float*>(X), lg, partials);
    else k_tpq_obs<float, false><<<grid, kThreads, 0, st>>>(od, reinterpret_cast<const float*>(X), lg, partials);
  }
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_tpq_obs_fin(const TpqDev& tq, int k, int nvec, double inv_ns, const double* partials, int grid,
                          cudaStream_t st) {
  k_tpq_obs_fin<<<nvec, kThreads, 0, st>>>(tq, k, nvec, inv_ns, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

}  // namespace hphi
