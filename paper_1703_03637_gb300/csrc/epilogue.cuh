// Helpers shared by the H v kernels: per-column CTA reductions, element access, the exact
// fixed-point accumulator for fp64 gather sums and the fused Lanczos / mTPQ epilogues.
#pragma once

#include "common.cuh"
#include "reduce.cuh"

namespace hphi {

// Per-column CTA reduction in a fixed tree order; partials[(block * nvec + c) * kMaxRedQ + q].
// NT is the CTA size; sm holds NT * kMaxRedQ doubles.
template <bool F64, int NT = kThreads>
__device__ void block_finish(const Red<F64>& red, int nq, int nvec, double* __restrict__ partials, double* sm) {
  const int tid = threadIdx.x;
  for (int q = 0; q < nq; ++q) sm[q * NT + tid] = red.get(q);
  __syncthreads();
  for (int off = NT / 2; off >= nvec; off >>= 1) {
    if (tid < off) {
      for (int q = 0; q < nq; ++q) sm[q * NT + tid] += sm[q * NT + tid + off];
    }
    __syncthreads();
  }
  if (tid < nvec) {
    for (int q = 0; q < nq; ++q) partials[((size_t)blockIdx.x * nvec + tid) * kMaxRedQ + q] = sm[q * NT + tid];
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

// m * 2^eoff rounded to nearest even: the hardware int64 -> fp64 conversion (round to
// nearest even) and an exact power-of-two scale.  Measured on GB300, this runs three
// times faster than assembling the result's bits with 64-bit integer operations.
__device__ __forceinline__ double fix_to_double(long long m, int eoff) {
  const double d = __ll2double_rn(m);
  if (eoff >= -1022 && eoff <= 1023) return d * __longlong_as_double((long long)(eoff + 1023) << 52);
  return ldexp(d, eoff);
}

// ------------------------------------------------------------------ gather sums
// fp64 terms are summed in an exact-alignment fixed-point accumulator: every term's
// 53-bit significand is shifted to the running largest exponent and added as a 64-bit
// integer (2 guard bits), so the sum runs on the integer pipes, which GB300 issues at 64x
// the fp64 rate.  Truncation below the grid 2^(e_max - 1077) costs at most one unit per
// term, i.e. <= n 2^-54 |largest term|, the same order as fp64 summation's error bound.
// Terms below 2^-1022 (subnormals) are dropped.
struct FixAcc {
  long long m;   // signed sum of aligned significands, units of 2^(e - 1077)
  int e;         // biased exponent of the largest term so far (0: empty)
  int n;         // terms since the last overflow flush
  double spill;  // flushed part (only after 128 terms)
  bool sp;       // spill holds something
  __device__ __forceinline__ void zero() { m = 0; e = 0; n = 0; spill = 0.0; sp = false; }
  __device__ __forceinline__ double value() const {
    const double r = fix_to_double(m, e - 1077);
    return sp ? r + spill : r;
  }
  __device__ __forceinline__ void add(double x, bool neg) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ex = (hi >> 20) & 0x7ff;
    if (ex == 0) return;
    if (++n == 128) {  // keep |m| < 2^63: 127 terms of < 2^55 each
      spill = value();
      sp = true;
      m = 0;
      e = 0;
      n = 1;
    }
    long long mant = ((long long)((hi & 0xfffff) | 0x100000) << 34) | ((long long)lo << 2);
    if (ex > e) {
      const int d = ex - e;
      m = (d >= 63) ? 0 : (m >> d);
      e = ex;
    }
    const int sh = e - ex;
    mant = (sh >= 63) ? 0 : (mant >> sh);
    if ((hi < 0) != neg) m -= mant;
    else m += mant;
  }
};

struct F32Acc {
  float s;
  __device__ __forceinline__ void zero() { s = 0.f; }
  __device__ __forceinline__ float value() const { return s; }
  __device__ __forceinline__ void add(float x, bool neg) { s += neg ? -x : x; }
};

// exact sums of 64-bit fixed-point terms (the quantised fp64 path; no overflow below
// 128 terms of magnitude < 2^56)
struct IntAcc {
  long long s;
  __device__ __forceinline__ void zero() { s = 0; }
  __device__ __forceinline__ long long value() const { return s; }
  __device__ __forceinline__ void add(long long x, bool neg) { s += neg ? -x : x; }
};

template <class R> struct SumAcc;
template <> struct SumAcc<double> { using T = FixAcc; };
template <> struct SumAcc<float> { using T = F32Acc; };
template <> struct SumAcc<long long> { using T = IntAcc; };

// (ar, ai) += phase(code) * (xr, xi), code: 1 (+1), 2 (+i), 3 (-1), 4 (-i)
template <class A, class R>
__device__ __forceinline__ void acc_phase(int code, R xr, R xi, A& ar, A& ai) {
  switch (code) {
    case 1: ar.add(xr, false); ai.add(xi, false); break;
    case 2: ar.add(xi, true); ai.add(xr, false); break;
    case 3: ar.add(xr, true); ai.add(xi, true); break;
    default: ar.add(xi, false); ai.add(xr, true); break;
  }
}

// ------------------------------------------------------------------ epilogues
struct EpiScalars {
  double c1, c2;  // Lanczos pass 1
};

template <class S, Epi E, int NQ = kMaxRedQ>
__device__ __forceinline__ void epilogue(int64_t idx, int c, typename Traits<S>::R sr, typename Traits<S>::R si,
                                         typename Traits<S>::R hr, typename Traits<S>::R hi, S* __restrict__ w,
                                         const FusedArgs& fa, const EpiScalars& es, const double* s_inv,
                                         Red<Traits<S>::kF64, NQ>& red) {
  using R = typename Traits<S>::R;
  constexpr bool C = Traits<S>::kCplx;
  if constexpr (E == Epi::kStore) {
    st<S>(w, idx, hr, hi);
  } else if constexpr (E == Epi::kLanczos1) {
    // P <- sigma_k * (H C) - beta_k sigma_{k-1} * P ;  partial <C, H C>
    S* P = reinterpret_cast<S*>(fa.out);
    const S* Pin = fa.in ? reinterpret_cast<const S*>(fa.in) : P;
    R pr, pi;
    ld<S>(Pin, idx, pr, pi);
    const R c1 = (R)es.c1, c2 = (R)es.c2;
    st<S>(P, idx, c1 * hr - c2 * pr, c1 * hi - c2 * pi);
    red.add(0, sr, hr);
    if constexpr (C) red.add(0, si, hi);
    red.tick();
  } else if constexpr (E == Epi::kTpq) {
    // X_{k+1} = (l X_k - H X_k / N_s) / |X_k| ; partials <X, HX>, |HX|^2.  |X_{k+1}|^2 follows
    // from them (section 3.5's norm, deferred): l^2 - 2 l u_k + <H^2>_k.
    S* Xn = reinterpret_cast<S*>(fa.out);
    const R inv = (R)s_inv[c], l = (R)fa.l, ins = (R)fa.inv_ns;
    const R nr = inv * (l * sr - hr * ins);
    const R ni = inv * (l * si - hi * ins);
    st<S>(Xn, idx, nr, ni);
    red.add(0, sr, hr);
    red.add(1, hr, hr);
    if constexpr (C) {
      red.add(0, si, hi);
      red.add(1, hi, hi);
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
  return E == Epi::kStore ? 0 : (E == Epi::kLanczos1 ? 1 : (E == Epi::kTpq ? 2 : 3));
}

}  // namespace hphi
