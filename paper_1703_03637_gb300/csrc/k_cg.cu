// Inverse iteration by conjugate gradients (section 3.4.1): y_{k+1} solves
// (H - E + delta) y_{k+1} = y_k, the shift delta > 0 keeping the operator positive definite
// when E lies at or just above the lowest eigenvalue, and the CG solve starting from y_k
// itself.  fp64 throughout; complex vectors run as real vectors of twice the length (H is
// Hermitian, so Re <u, A v> is the inner product CG needs).  Besides the caller's vector the
// solve keeps four: the iterate y, the residual r, the direction p and q = A p.
//
// Every kernel streams its vectors once with four elements per thread one grid stride apart
// and leaves one fp64 partial sum per CTA; a one-CTA finaliser turns the partials into the
// CG scalars on the device, so a whole solve is a fixed launch sequence.
#include "common.cuh"

namespace hphi {
namespace {

__device__ double cg_block_sum(double x, double* sm) {
  const int tid = threadIdx.x;
  __syncthreads();  // an earlier sum's result has been read by every thread
  sm[tid] = x;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if (tid < off) sm[tid] += sm[tid + off];
    __syncthreads();
  }
  return sm[0];
}

__device__ __forceinline__ void cg_partial(double acc, double* partials, int q) {
  __shared__ double sm[kThreads];
  const double t = cg_block_sum(acc, sm);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kMaxRedQ + q] = t;
}

// q <- q + c p (c = delta - E, so q = (H - E + delta) p after q = H p); partial <p, q>
__global__ void __launch_bounds__(kThreads) k_cg_shift(CgDev cg, const double* __restrict__ p, double* __restrict__ q,
                                                        int64_t n, double* __restrict__ partials) {
  if (*cg.done) return;
  const double c = cg.s[4];
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += 4 * stride) {
    double pv[4], qv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      pv[u] = k < n ? p[k] : 0.0;
      qv[u] = k < n ? q[k] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      if (k < n) {
        const double t = fma(c, pv[u], qv[u]);
        q[k] = t;
        acc = fma(pv[u], t, acc);
      }
    }
  }
  cg_partial(acc, partials, 0);
}

// mode 0: start of a solve: y <- b, r <- b - q (q = A b), p <- r; partials |r|^2, |b|^2
// mode 1: y += alpha p, r -= alpha q; partial |r|^2
__global__ void __launch_bounds__(kThreads) k_cg_update(CgDev cg, int mode, const double* __restrict__ b,
                                                         double* __restrict__ y, double* __restrict__ r,
                                                         double* __restrict__ p, const double* __restrict__ q,
                                                         int64_t n, double* __restrict__ partials) {
  if (*cg.done) return;
  const double al = cg.s[1];
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += 4 * stride) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t k = i + u * stride;
      if (k >= n) break;
      if (mode == 0) {
        const double bv = b[k];
        const double rv = bv - q[k];
        y[k] = bv;
        r[k] = rv;
        p[k] = rv;
        rr = fma(rv, rv, rr);
        bb = fma(bv, bv, bb);
      } else {
        const double pv = p[k];
        y[k] = fma(al, pv, y[k]);
        const double rv = fma(-al, q[k], r[k]);
        r[k] = rv;
        rr = fma(rv, rv, rr);
      }
    }
  }
  cg_partial(rr, partials, 0);
  if (mode == 0) cg_partial(bb, partials, 1);
}

// p <- r + beta p
__global__ void __launch_bounds__(kThreads) k_cg_dir(CgDev cg, const double* __restrict__ r, double* __restrict__ p,
                                                      int64_t n) {
  if (*cg.done) return;
  const double be = cg.s[2];
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) p[i] = fma(be, p[i], r[i]);
}

// x <- y / |y| (mode 0: partial |y|^2 first; mode 1: scale, the norm in s[9])
__global__ void __launch_bounds__(kThreads) k_cg_norm(CgDev cg, int mode, const double* __restrict__ y,
                                                       double* __restrict__ x, int64_t n,
                                                       double* __restrict__ partials) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  if (mode == 0) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) acc = fma(y[i], y[i], acc);
    cg_partial(acc, partials, 0);
    return;
  }
  const double sc = cg.s[9];
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) x[i] = y[i] * sc;
}

// Rayleigh quotient of x (unit) with hx = H x: partials <x, hx>, <hx, hx>; then |hx - e x|^2
__global__ void __launch_bounds__(kThreads) k_cg_rq(CgDev cg, int mode, const double* __restrict__ x,
                                                     const double* __restrict__ hx, int64_t n,
                                                     double* __restrict__ partials) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  if (mode == 0) {
    double xh = 0.0, hh = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
      xh = fma(x[i], hx[i], xh);
      hh = fma(hx[i], hx[i], hh);
    }
    cg_partial(xh, partials, 0);
    cg_partial(hh, partials, 1);
    return;
  }
  const double e = cg.s[6];
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
    const double d = fma(-e, x[i], hx[i]);
    rr = fma(d, d, rr);
  }
  cg_partial(rr, partials, 0);
}

__device__ double cg_sum(const double* __restrict__ partials, int grid, int q, double* sm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < grid; b += kThreads) s += partials[(size_t)b * kMaxRedQ + q];
  return cg_block_sum(s, sm);
}

// scalar steps of the solve, one CTA:
// 0 start (rr, |b|^2, done if r = 0)  1 alpha = rr / <p, q>  2 beta = rr' / rr, test
// 3 the norm of y  4 e and the variance  5 the residual
__global__ void __launch_bounds__(kThreads) k_cg_fin(CgDev cg, int mode, const double* __restrict__ partials,
                                                      int grid) {
  __shared__ double sm[kThreads];
  if ((mode == 1 || mode == 2) && *cg.done) return;
  const double s0 = cg_sum(partials, grid, 0, sm);
  const double s1 = (mode == 0 || mode == 4) ? cg_sum(partials, grid, 1, sm) : 0.0;
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    cg.s[0] = s0;
    cg.s[3] = s1;
    *cg.done = (s0 <= cg.s[5] * s1) ? 1 : 0;
  } else if (mode == 1) {
    if (!(s0 > 0.0)) {  // A is positive definite on a non-zero p: only p = 0 gives this
      *cg.done = 1;
      return;
    }
    cg.s[1] = cg.s[0] / s0;
  } else if (mode == 2) {
    cg.s[2] = s0 / cg.s[0];
    cg.s[0] = s0;
    *cg.steps += 1;
    if (s0 <= cg.s[5] * cg.s[3]) *cg.done = 1;
  } else if (mode == 3) {
    cg.s[9] = s0 > 0.0 ? 1.0 / sqrt(s0) : 0.0;
  } else if (mode == 4) {
    cg.s[6] = s0;          // <x|H|x>, x a unit vector
    cg.s[8] = s1 - s0 * s0;  // <H^2> - <H>^2
  } else {
    cg.s[7] = sqrt(s0);    // |H x - e x|
  }
}

}  // namespace

Status launch_cg_shift(const CgDev& cg, const double* p, double* q, int64_t n, double* partials, int grid,
                       cudaStream_t st) {
  k_cg_shift<<<grid, kThreads, 0, st>>>(cg, p, q, n, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_cg_update(const CgDev& cg, int mode, const double* b, double* y, double* r, double* p, const double* q,
                        int64_t n, double* partials, int grid, cudaStream_t st) {
  k_cg_update<<<grid, kThreads, 0, st>>>(cg, mode, b, y, r, p, q, n, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_cg_dir(const CgDev& cg, const double* r, double* p, int64_t n, int grid, cudaStream_t st) {
  k_cg_dir<<<grid, kThreads, 0, st>>>(cg, r, p, n);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_cg_norm(const CgDev& cg, int mode, const double* y, double* x, int64_t n, double* partials, int grid,
                      cudaStream_t st) {
  k_cg_norm<<<grid, kThreads, 0, st>>>(cg, mode, y, x, n, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_cg_rq(const CgDev& cg, int mode, const double* x, const double* hx, int64_t n, double* partials,
                    int grid, cudaStream_t st) {
  k_cg_rq<<<grid, kThreads, 0, st>>>(cg, mode, x, hx, n, partials);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_cg_fin(const CgDev& cg, int mode, const double* partials, int grid, cudaStream_t st) {
  k_cg_fin<<<1, kThreads, 0, st>>>(cg, mode, partials, grid);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

}  // namespace hphi
