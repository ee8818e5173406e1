// Reduction accumulators shared by the fused H v kernels and the streaming vector kernels.
//
// fp64 storage: products accumulate with one fp64 fused multiply-add per element.
// fp32 storage: GB300 issues fp64 at 1/64 of the fp32 rate, so products are accumulated
// without rounding loss in fp32 (hi, lo) pairs -- TwoProduct by FMA and Knuth's TwoSum --
// and every 16 elements the pair is added to an fp64 total.  The result carries fp64
// accuracy while costing about ten fp32 instructions per product.
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

// fp32 products accumulated without loss in (hi, lo) pairs: TwoProduct by FMA and TwoSum
// (Knuth); every 16 elements the pair is added to an fp64 total.
template <int NQ> struct Red<false, NQ> {
  double tot[NQ];
  float hi[NQ], lo[NQ];
  int n;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NQ; ++q) { tot[q] = 0.0; hi[q] = 0.f; lo[q] = 0.f; }
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
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      tot[q] += (double)hi[q] + (double)lo[q];
      hi[q] = 0.f;
      lo[q] = 0.f;
    }
    n = 0;
  }
  __device__ __forceinline__ void tick() {
    if (++n == 16) flush();
  }
  __device__ __forceinline__ double get(int q) const { return tot[q] + ((double)hi[q] + (double)lo[q]); }
};

}  // namespace hphi
