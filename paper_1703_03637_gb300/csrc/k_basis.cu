// Sector tables, basis decode / rank for tests, and the Philox4x32-10 start-vector
// generator (integer work, bit-exact).
#include <math.h>

#include "basis.cuh"
#include "common.cuh"

namespace hphi {

namespace {

constexpr int kBinomN = 64;
// Pascal's triangle C(n, k), 0 <= k <= n < 64; written once per device.
__device__ uint64_t g_binom[kBinomN][kBinomN];

__device__ __forceinline__ uint64_t binom_dev(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  return g_binom[n][k];
}

__global__ void k_pascal() {
  // one thread: 4096 entries, each the sum of two earlier ones
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int n = 0; n < kBinomN; ++n) {
    for (int k = 0; k < kBinomN; ++k) {
      uint64_t v;
      if (k > n) v = 0;
      else if (k == 0 || k == n) v = 1;
      else v = g_binom[n - 1][k - 1] + g_binom[n - 1][k];
      g_binom[n][k] = v;
    }
  }
}

// Rank of x among the L-bit strings with the same popcount (combinatorial number system:
// the t-th set bit from the bottom, at position q, contributes C(q, t)).
__global__ void k_popcount_tables(int L, uint32_t* __restrict__ lo_rank, uint32_t* __restrict__ lo_list,
                                  const uint32_t* __restrict__ lo_list_off) {
  const uint64_t n = 1ull << L;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t r = 0;
    int t = 0;
    uint64_t y = x;
    while (y) {
      const int q = __ffsll((long long)y) - 1;
      ++t;
      r += binom_dev(q, t);
      y &= y - 1;
    }
    lo_rank[x] = (uint32_t)r;
    lo_list[lo_list_off[__popcll(x)] + r] = (uint32_t)x;
  }
}

// hi_off[hi] = number of (L + H)-bit strings with n_ones ones whose high part is < hi:
// at every set bit of hi (from the top), the strings that agree above it and have a 0
// there place their remaining ones freely below.
__global__ void k_hi_offsets(int L, int H, int n_ones, uint64_t* __restrict__ hi_off) {
  const uint64_t n = 1ull << H;
  for (uint64_t hi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; hi < n; hi += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t c = 0;
    int above = 0;
    for (int q = H - 1; q >= 0; --q) {
      if ((hi >> q) & 1ull) {
        c += binom_dev(q + L, n_ones - above);
        ++above;
      }
    }
    hi_off[hi] = c;
  }
}

__global__ void k_spin_states(const SpinDev md, int64_t r0, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = (uint64_t)(r0 + k);
    out[k] = md.sector ? sector_state(md.t, r) : r;
  }
}

__global__ void k_spin_ranks(const SpinDev md, const uint64_t* __restrict__ st, int64_t n, int64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t s = st[k];
    int64_t r;
    if (md.n_sites < 64 && (s >> md.n_sites) != 0) r = -1;
    else if (!md.sector) r = (int64_t)s;
    else r = (__popcll(s) == md.t.n_ones) ? (int64_t)sector_rank(md.t, s) : -1;
    out[k] = r;
  }
}

__global__ void k_hub_states(const HubDev md, int64_t r0, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = (uint64_t)(r0 + k);
    const uint64_t d = r / (uint64_t)md.dim_up, u = r % (uint64_t)md.dim_up;
    uint64_t up = u, dn = d;
    if (md.sector) {
      up = md.list_up[u];
      dn = md.list_dn[d];
    }
    out[k] = up | (dn << 32);
  }
}

__global__ void k_hub_ranks(const HubDev md, const uint64_t* __restrict__ st, int64_t n, int64_t* __restrict__ out,
                            int na, int nb) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t up = st[k] & 0xffffffffull, dn = st[k] >> 32;
    int64_t r;
    if ((up >> md.n_sites) != 0 || (dn >> md.n_sites) != 0) r = -1;
    else if (!md.sector) r = (int64_t)(dn * (uint64_t)md.dim_up + up);
    else if (__popcll(up) != na || __popcll(dn) != nb) r = -1;
    else r = (int64_t)md.rank[dn] * md.dim_up + (int64_t)md.rank[up];
    out[k] = r;
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round multiplies
// words 0 and 2 by the two Philox multipliers, swaps the halves crosswise and mixes in the
// round key; the key is advanced by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__global__ void k_philox_raw(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, uint32_t* __restrict__ out,
                             int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2], ctr[4 * k + 3]);
    const uint2 kk = make_uint2(key[2 * k], key[2 * k + 1]);
    const uint4 o = philox(c, kk);
    out[4 * k] = o.x; out[4 * k + 1] = o.y; out[4 * k + 2] = o.z; out[4 * k + 3] = o.w;
  }
}

// Standard-normal numbers (a seeded Gaussian start vector; appendix A.2 / A.4 draw every
// coefficient from a random number generator).  Philox block p (counter (p mod 2^32, p >> 32,
// 0, 0)) gives two 53-bit open-interval uniforms and, by Box-Muller, the pair
// g0 = sqrt(-2 ln u_a) cos(2 pi u_b), g1 = sqrt(-2 ln u_a) sin(2 pi u_b).  A complex element e
// is g0 + i g1 of block e; real elements 2p and 2p + 1 are g0 and g1 of block p, so no half
// of a pair is wasted (GB300 runs the fp64 logarithm and sine / cosine at 1/64 of its fp32
// rate).  One thread per block.
template <bool CPLX, bool F64>
__global__ void k_random(void* __restrict__ v, int64_t n_elem, uint64_t seed) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  const int64_t n_blk = CPLX ? n_elem : (n_elem + 1) / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_blk; p += (int64_t)gridDim.x * blockDim.x) {
    const uint4 o = philox(make_uint4((uint32_t)p, (uint32_t)((uint64_t)p >> 32), 0u, 0u), key);
    const uint64_t a = ((((uint64_t)o.x) << 32) | o.y) >> 11;
    const uint64_t b = ((((uint64_t)o.z) << 32) | o.w) >> 11;
    if (F64) {
      const double ua = ((double)a + 0.5) * (1.0 / 9007199254740992.0);
      const double ub = ((double)b + 0.5) * (1.0 / 9007199254740992.0);
      const double rad = sqrt(-2.0 * log(ua));
      double sn, cs;
      sincospi(2.0 * ub, &sn, &cs);
      const double g0 = rad * cs, g1 = rad * sn;
      if (CPLX) {
        reinterpret_cast<double2*>(v)[p] = make_double2(g0, g1);
      } else {
        double* x = reinterpret_cast<double*>(v);
        x[2 * p] = g0;
        if (2 * p + 1 < n_elem) x[2 * p + 1] = g1;
      }
    } else {
      // fp32 storage: the same two uniforms, rounded to fp32 (relative error 2^-24, also in
      // the tail near 0), through the transform in fp32 arithmetic; the result is rounded to
      // fp32 anyway.  ln u_a: logf of u_a below 1/2; above, log1pf(-(1 - u_a)) with 1 - u_a
      // formed from the integer complement (2^53 - 1 - a + 0.5) / 2^53, so u_a near 1 keeps
      // full relative accuracy
      const float two53 = 1.0f / 9007199254740992.0f, half53 = 1.0f / 18014398509481984.0f;
      const float ua = fmaf(__ull2float_rn(a), two53, half53);
      const float la = (a < (1ull << 52)) ? logf(ua) : log1pf(-fmaf(__ull2float_rn((1ull << 53) - 1ull - a), two53, half53));
      const float ub = fmaf(__ull2float_rn(b), two53, half53);
      const float rad = sqrtf(-2.0f * la);
      float sn, cs;
      sincospif(2.0f * ub, &sn, &cs);
      if (CPLX) {
        reinterpret_cast<float2*>(v)[p] = make_float2(rad * cs, rad * sn);
      } else {
        float* x = reinterpret_cast<float*>(v);
        x[2 * p] = rad * cs;
        if (2 * p + 1 < n_elem) x[2 * p + 1] = rad * sn;
      }
    }
  }
}

int grid_for(int64_t n) {
  const int64_t cap = (int64_t)num_sms() * 8;
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

Status build_popcount_tables(int L, uint32_t* lo_rank, uint32_t* lo_list, const uint32_t* lo_list_off,
                             cudaStream_t st) {
  k_pascal<<<1, 1, 0, st>>>();
  HPHI_CUDA_TRY(cudaGetLastError());
  k_popcount_tables<<<grid_for(1ll << L), kThreads, 0, st>>>(L, lo_rank, lo_list, lo_list_off);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status build_hi_offsets(int L, int H, int n_ones, uint64_t* hi_off, cudaStream_t st) {
  k_pascal<<<1, 1, 0, st>>>();
  HPHI_CUDA_TRY(cudaGetLastError());
  k_hi_offsets<<<grid_for(1ll << H), kThreads, 0, st>>>(L, H, n_ones, hi_off);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_spin_states(const SpinDev& md, int64_t r0, int64_t n, uint64_t* out, cudaStream_t st) {
  if (n <= 0) return {};
  k_spin_states<<<grid_for(n), kThreads, 0, st>>>(md, r0, n, out);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_spin_ranks(const SpinDev& md, const uint64_t* states, int64_t n, int64_t* out, cudaStream_t st) {
  if (n <= 0) return {};
  k_spin_ranks<<<grid_for(n), kThreads, 0, st>>>(md, states, n, out);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_hub_states(const HubDev& md, int64_t r0, int64_t n, uint64_t* out, cudaStream_t st) {
  if (n <= 0) return {};
  k_hub_states<<<grid_for(n), kThreads, 0, st>>>(md, r0, n, out);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_hub_ranks(const HubDev& md, const uint64_t* states, int64_t n, int64_t* out, cudaStream_t st) {
  if (n <= 0) return {};
  k_hub_ranks<<<grid_for(n), kThreads, 0, st>>>(md, states, n, out, md.n_up, md.n_dn);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_philox_raw(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return {};
  k_philox_raw<<<grid_for(n), kThreads, 0, st>>>(ctr, key, out, n);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

Status launch_random(void* v, int64_t n_elem, bool cplx, bool f64, uint64_t seed, cudaStream_t st) {
  if (n_elem <= 0) return {};
  const int g = grid_for(n_elem);
  if (cplx && f64) k_random<true, true><<<g, kThreads, 0, st>>>(v, n_elem, seed);
  else if (cplx) k_random<true, false><<<g, kThreads, 0, st>>>(v, n_elem, seed);
  else if (f64) k_random<false, true><<<g, kThreads, 0, st>>>(v, n_elem, seed);
  else k_random<false, false><<<g, kThreads, 0, st>>>(v, n_elem, seed);
  HPHI_CUDA_TRY(cudaGetLastError());
  return {};
}

}  // namespace hphi
