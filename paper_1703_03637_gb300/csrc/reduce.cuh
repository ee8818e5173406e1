// Reduction accumulators shared by the fused H v kernels and the streaming vector kernels.
//
// fp64 storage: products accumulate with one fp64 fused multiply-add per element.
// fp32 storage: GB300 issues fp64 at 1/64 of the fp32 rate, so each thread accumulates its
// products in fp32 pairs -- TwoProduct by FMA and Knuth's TwoSum, then double-float folds --
// and converts to fp64 once; the per-thread sums meet in fp64 (per-CTA and across CTAs).  The
// result is accurate to about 1e-12 relative while costing about a dozen fp32 instructions
// per product.
#pragma once

#include "common.cuh"

namespace hphi {

// NQ: number of reduced quantities (kernels that know theirs keep fewer registers)
template <bool F64, int NQ = kMaxRedQ> struct Red;

template <int NQ> struct Red<true, NQ> {
  double s[NQ];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = 0.0;
  }
  __device__ __forceinline__ void add(int q, double a, double b) { s[q] = fma(a, b, s[q]); }
  __device__ __forceinline__ void tick() {}
  __device__ __forceinline__ double get(int q) const { return s[q]; }
};

// fp32 products accumulated in (hi, lo) pairs: TwoProduct by FMA and TwoSum (Knuth), exact per
// product; every 16 products the pair is folded into a second pair (h2, l2) by a double-float
// addition (TwoSum of the high parts, then a fast renormalisation; relative error about 2^-46
// per fold), and the fp64 value is formed once, in get().  The fold is fp32-only on purpose:
// the compiler if-converts the every-16th branch, so the fold's instructions issue on every
// product, and fp64 conversions there would saturate GB300's 1/64-rate fp64 pipe.
template <int NQ> struct Red<false, NQ> {
  float hi[NQ], lo[NQ], h2[NQ], l2[NQ];
  int n;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NQ; ++q) { hi[q] = 0.f; lo[q] = 0.f; h2[q] = 0.f; l2[q] = 0.f; }
    n = 0;
  }
  __device__ __forceinline__ void add(int q, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float t = __fadd_rn(hi[q], p);
    const float z = __fsub_rn(t, hi[q]);
    const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(t, z)), __fsub_rn(p, z));
    hi[q] = t;
    lo[q] = __fadd_rn(lo[q], __fadd_rn(err, e));
  }
  // (h2, l2) += (hi, lo); (hi, lo) = 0
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float s = __fadd_rn(h2[q], hi[q]);
      const float z = __fsub_rn(s, h2[q]);
      float e = __fadd_rn(__fsub_rn(h2[q], __fsub_rn(s, z)), __fsub_rn(hi[q], z));
      e = __fadd_rn(e, __fadd_rn(l2[q], lo[q]));
      const float h = __fadd_rn(s, e);
      l2[q] = __fsub_rn(e, __fsub_rn(h, s));
      h2[q] = h;
      hi[q] = 0.f;
      lo[q] = 0.f;
    }
    n = 0;
  }
  __device__ __forceinline__ void tick() {
    if (++n == 16) fold();
  }
  __device__ __forceinline__ double get(int q) const {
    return ((double)h2[q] + (double)l2[q]) + ((double)hi[q] + (double)lo[q]);
  }
};

}  // namespace hphi
