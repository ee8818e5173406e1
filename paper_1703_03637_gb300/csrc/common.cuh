// Shared declarations of the GB300 (sm_103a) Lanczos / mTPQ library: device-side model
// descriptions, scalar traits, block reductions and the internal launch interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hphi_gpu.h"

namespace hphi {

// ------------------------------------------------------------------ limits
constexpr int kThreads = 256;        // threads per CTA of every streaming kernel
constexpr int kMaxSpinEntries = 640;  // off-diagonal XOR patterns staged in shared memory
constexpr int kMaxClasses = 384;      // distinct coefficient classes
constexpr int kMaxLin = 64;           // linear diagonal groups (coef * popcount(s & mask))
constexpr int kMaxPairs = 512;        // bilinear diagonal pairs
constexpr int kMaxPairGroups = 128;
constexpr int kMaxHops = 512;         // Hubbard hop entries (both species)
constexpr int kMaxRedQ = 4;           // reduced quantities per fused kernel
constexpr int kMaxNvec = 256;

// ------------------------------------------------------------------ device model
// Off-diagonal spin pattern: w[s] += coef[cls] * phase(b_i + 2 b_j) * v[rank(s ^ mask)].
struct SpinEntry {
  uint64_t mask;
  uint8_t i, j;      // sites whose bra bits select the phase (j == i for one-site terms)
  uint16_t phases;   // four 3-bit codes: 0 none, 1 (+1), 2 (+i), 3 (-1), 4 (-i)
  uint16_t cls;
  uint16_t pad;
};
static_assert(sizeof(SpinEntry) == 16, "SpinEntry layout");

struct LinGroup {   // coef * popcount(bits & mask)
  uint64_t mask;
  double coef;
};

struct PairEntry {  // one bilinear diagonal pair, counted as b_i & b_j (spin) or n_i n_j (Hubbard)
  uint8_t i, j;
  uint16_t grp;
};

// Hubbard hop: bra bits (i set, j empty) -> coef[cls]; (j set, i empty) -> conj(coef[cls]);
// times (-1)^popcount(species bits & between).
struct HopEntry {
  uint32_t mask;
  uint32_t between;
  uint8_t i, j;
  uint16_t cls;
  uint32_t pad;
};
static_assert(sizeof(HopEntry) == 16, "HopEntry layout");

struct SectorTables {
  int L;                       // bits handled by the low table
  int H;                       // high bits (n_bits - L)
  int n_ones;                  // popcount of the sector
  const uint64_t* hi_off;      // [2^H] sector states whose high part is smaller
  const uint32_t* lo_rank;     // [2^L] rank among L-bit strings of the same popcount
  const uint32_t* lo_list;     // [2^L] L-bit strings grouped by popcount, ascending
  const uint32_t* lo_list_off; // [L + 2] start of each popcount group in lo_list
};

struct SpinDev {
  int n_sites;
  int sector;        // 0 full basis, 1 fixed popcount
  int64_t dim;
  int n_entries, n_classes, n_lin, n_pairs, n_pair_groups;
  double c0;
  const SpinEntry* entries;  // sorted by class
  const double2* cls_coef;
  const LinGroup* lin;
  const PairEntry* pairs;
  const double* pair_coef;   // [n_pair_groups]
  SectorTables t;
  unsigned long long* counter;  // work-item counter of the H v kernels (reset before each launch)
  int max_run;                  // longest run of entries of one class
};

struct HubDev {
  int n_sites;
  int sector;        // 0 full (2^N per species), 1 fixed (N_up, N_dn)
  int n_up, n_dn;    // particle numbers of the sector
  int64_t dim, dim_up, dim_dn;
  int n_up_hops, n_dn_hops, n_classes;
  int n_ulin, n_mulin, n_pairs, n_pair_groups;
  double c0;
  const HopEntry* hops;      // up hops first, then down hops; sorted by class in each part
  const double2* cls_coef;
  const LinGroup* ulin;      // U groups: coef * popcount(up & dn & mask)
  const LinGroup* mulin;     // one-body groups: coef * (popcount(up & mask) + popcount(dn & mask))
  const PairEntry* pairs;    // V n_i n_j
  const double* pair_coef;
  // species tables (rank / list over n_sites bits); null for the full basis
  const uint32_t* rank;      // [2^N]
  const uint32_t* list_up;   // [dim_up]
  const uint32_t* list_dn;   // [dim_dn]
  unsigned long long* counter;  // work-item counter of the generic kernel
  // two-pass path (real model, one hopping value per species): neighbour tables
  // nbr[k * maxdeg + q] = rank of the q-th hop target of species state k | sign << 31
  int fast;
  int dn_ept;                // pass D columns per thread (0: default)
  int up_k;                  // pass U rows per tile (0: largest that fits)
  int tuned_ept[2], tuned_k[2];  // autotuner choices per precision (HPHI_FP64, HPHI_FP32)
  int maxdeg_up, maxdeg_dn;
  double c_up, c_dn;         // the hopping coefficient of each species
  const uint32_t* nbr_up;
  const uint8_t* deg_up;
  const uint8_t* npos_up;    // entries [0, npos) carry sign +1, [npos, deg) sign -1
  const uint32_t* nbr_dn;
  const uint8_t* deg_dn;
  const uint8_t* npos_dn;
};

// ------------------------------------------------------------------ scalar traits
template <class T> struct Cx { T x, y; };

template <class S> struct Traits;
template <> struct Traits<double> {
  using R = double; static constexpr bool kCplx = false; static constexpr bool kF64 = true;
};
template <> struct Traits<float> {
  using R = float; static constexpr bool kCplx = false; static constexpr bool kF64 = false;
};
template <> struct Traits<double2> {
  using R = double; static constexpr bool kCplx = true; static constexpr bool kF64 = true;
};
template <> struct Traits<float2> {
  using R = float; static constexpr bool kCplx = true; static constexpr bool kF64 = false;
};

// ------------------------------------------------------------------ runtime helpers
struct Status {
  int code = HPHI_OK;
  std::string msg;
};

#define HPHI_CUDA_TRY(expr)                                                            \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                           \
      return ::hphi::Status{HPHI_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
    }                                                                                  \
  } while (0)

int num_sms();

// Launch interface (k_basis.cu) --------------------------------------------------------
Status build_popcount_tables(int L, uint32_t* lo_rank, uint32_t* lo_list, const uint32_t* lo_list_off,
                             cudaStream_t st);
Status build_hi_offsets(int L, int H, int n_ones, uint64_t* hi_off, cudaStream_t st);
Status launch_spin_states(const SpinDev& md, int64_t r0, int64_t n, uint64_t* out, cudaStream_t st);
Status launch_spin_ranks(const SpinDev& md, const uint64_t* states, int64_t n, int64_t* out, cudaStream_t st);
Status launch_hub_states(const HubDev& md, int64_t r0, int64_t n, uint64_t* out, cudaStream_t st);
Status launch_hub_ranks(const HubDev& md, const uint64_t* states, int64_t n, int64_t* out, cudaStream_t st);
Status launch_philox_raw(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t st);
Status launch_random(void* v, int64_t n_elem, bool cplx, bool f64, uint64_t seed, cudaStream_t st);

// H v and fused solver kernels (k_hv.cu) -----------------------------------------------
enum class Epi { kStore = 0, kLanczos1 = 1, kTpq = 2, kRefine = 3 };

struct FusedArgs {
  // Lanczos pass 1: P <- c1 * Y - c2 * P; partial sum of self * Y.
  // TPQ: Xn <- inv[c] * (l * X - Y / Ns); partial sums <X, Y>, |Y|^2 per column.
  // Refine: stores Y and reduces <x, Y>, <x, x>.
  void* out = nullptr;             // P (Lanczos) / X_{k+1} (TPQ) / Hx (refine)
  const void* in = nullptr;        // Lanczos: previous vector read by pass 1 (null: same as out)
  const double* scal = nullptr;    // device scalars read at kernel start
  double* partials = nullptr;      // [grid][nvec][kMaxRedQ]
  const int* done = nullptr;       // device flag: skip all work when set
  double l = 0.0, inv_ns = 0.0;
  int exp_ready = 0;               // fp64 two-pass Hubbard: the input's exponent is already in
                                   // the scratch slot (computed by the previous Lanczos pass 2)
};

// Launches w = H v (or a fused step) over all rows; grid chosen by the library.  Spin models
// in fp64 gather from a quantised copy of v when scratch (spin_scratch_bytes) is given.
Status launch_hv(bool hubbard, const void* md, int prec, bool cplx, const void* v, void* w, int nvec, Epi epi,
                 const FusedArgs& fa, int grid, void* scratch, cudaStream_t st);
bool spin_quantised(const SpinDev& md, int prec, int nvec);
size_t spin_scratch_bytes(const SpinDev& md, int prec, bool cplx, int nvec);
int hv_grid(int nvec);  // upper bound of any H v grid (partials sizing)

// Two-pass Hubbard path (k_hub.cu): neighbour tables, and H v = diag + up hops (row tiles
// in shared memory) + down hops (stripe-major row combinations into the scratch vector W).
Status build_hub_neighbours(const HubDev& md, int species, uint32_t* nbr, uint8_t* deg, uint8_t* npos,
                            cudaStream_t st);
bool hub_fast_ok(const HubDev& md, int prec, bool cplx, int nvec, Epi epi);
int hub_up_grid(const HubDev& md, int prec, Epi epi);
size_t hub_scratch_bytes(const HubDev& md, int prec, Epi epi);  // scratch the launch needs
// the fp64 input-exponent slot inside that scratch (see FusedArgs::exp_ready)
int* hub_exponent_slot(const HubDev& md, void* scratch);
// fp64 H v of the two-pass path with its scratch in a fixed device array (no allocation)
Status launch_hub_store_noalloc(const HubDev& md, const void* v, void* w, cudaStream_t st);
size_t noalloc_capacity_bytes();
Status launch_hub_fast(const HubDev& md, int prec, const void* v, void* w, void* scratch, Epi epi,
                       const FusedArgs& fa, int grid_up, cudaStream_t st);
// resident CTAs of the chosen kernel instance over the whole GPU (occupancy API)
int hv_resident_grid(bool hubbard, int prec, bool cplx, Epi epi);

// Batched-row H v (k_batch.cu): full-basis spin models on <= 32 sites, nvec in {32, 64,
// 128, 256}, vectors 32-byte aligned.  fp64 needs batch_scratch_bytes() of scratch.
// With a window plan the terms run in passes over bit windows (the rows of each pass are
// visited with the window's bits varying fastest, so the pass's gathers stay in L2).
constexpr int kMaxPasses = 8;
struct BatchPlan {
  int n_pass = 0;
  const SpinEntry* ents = nullptr;  // entries pass by pass, class-sorted within a pass
  const uint32_t* dep = nullptr;    // [n_pass][4][256]: byte b of the visit index -> row bits
  int ent_off[kMaxPasses + 1] = {};
  int max_run = 0;                  // longest class run within a pass
};
// Greedy cyclic windows of wbits sites covering every entry's flip mask; false when more
// than kMaxPasses windows would be needed.
bool batch_plan_windows(int n_sites, int wbits, const std::vector<SpinEntry>& ents,
                        std::vector<SpinEntry>* ordered, std::vector<uint32_t>* dep, int* ent_off, int* n_pass,
                        int* max_run);
// window size whose block of rows (input rows only) fills about a quarter of L2
int batch_window_bits(int prec, bool cplx, int nvec);
bool batch_applies(const SpinDev& md, int nvec);
// Q = the [rows][nvec] (x ncomp) fp64 block quantised to 64-bit integers, one scale per
// column: q = round(x 2^(1078 - E_c)), E_c the column's largest exponent field (into E)
Status launch_quant_cols(const double* v, int64_t rows, int nvec, int ncomp, long long* Q, int* E, cudaStream_t st);
bool batch_aligned(const void* v, const void* w);
size_t batch_scratch_bytes(const SpinDev& md, const BatchPlan* plan, int prec, bool cplx, int nvec);
int batch_grid(int prec, bool cplx, int nvec, Epi epi, int64_t dim);
Status launch_batch(const SpinDev& md, const BatchPlan* plan, int prec, bool cplx, const void* v, void* w,
                    void* scratch, int nvec, Epi epi, const FusedArgs& fa, int grid, cudaStream_t st);

// Streaming vector kernels and finalisers (k_solver.cu) -------------------------------
struct LzDev {           // device scalars of one Lanczos run
  double* alpha;         // [m]
  double* beta;          // [m]   beta[k] = beta_{k+1}
  double* sig;           // [m+1] sigma_k = 1 / |C_k|
  double* coef;          // [m]   Ritz coefficients (refinement pass)
  double* s;             // [16]  scratch scalars (c1, c2, gamma, xcoef, last replay step)
  int* done;             // [1]   breakdown flag
  int* steps_done;       // [1]
  double* tri;           // [8 + 3]  eigenvalues and refinement results
};

Status launch_lz_init(int prec, bool cplx, const void* v0_f64, void* C, void* P, int64_t n_real, double* partials,
                      int grid, cudaStream_t st);
Status launch_lz_init_fin(const LzDev& lz, const double* partials, int grid, cudaStream_t st);
Status launch_lz_fin1(const LzDev& lz, int k, const double* partials, int grid, cudaStream_t st);
// emax (fp64 only, may be null): atomicMax of the exponent fields of the new P
Status launch_lz_pass2(int prec, bool cplx, const LzDev& lz, int k, const void* C, void* P, double* x,
                       int64_t n_real, double* partials, int grid, int* emax, cudaStream_t st);
// replay: the refinement's second pass (stops after the last step with a significant Ritz
// coefficient, keeps the first pass's step count)
Status launch_lz_fin2(const LzDev& lz, int k, double brk, const double* partials, int grid, bool replay,
                      cudaStream_t st);
// tail_tol: Ritz-coefficient weight below which the replayed second pass may stop
Status launch_tridiag(const LzDev& lz, int m_max, int n_eig, bool want_vec, double tail_tol, cudaStream_t st);
Status launch_refine_fin(const LzDev& lz, const double* partials, int grid, int which, cudaStream_t st);
// x = sum_k coef_k sigma_k V_k over the stored Lanczos vectors (k < steps_done)
Status launch_lz_combine(int prec, const LzDev& lz, const void* V, int64_t n_real, int64_t stride_real, double* x,
                         int grid, cudaStream_t st);
Status launch_refine_resid(bool cplx, const double* x, const double* hx, int64_t n_real, const LzDev& lz,
                           double* partials, int grid, cudaStream_t st);

struct TpqDev {
  double* n2;            // [nvec] |X_k|^2 of the current state
  double* inv;           // [nvec] 1 / |X_k|
  double* u;             // [K][nvec]
  double* h2;            // [K][nvec]
  double* nrm;           // [K][nvec]
};
Status launch_tpq_init(int prec, bool cplx, const void* psi0_f64, void* X, int64_t n_rows, int nvec,
                       double* partials, int grid, cudaStream_t st);
Status launch_tpq_init_fin(const TpqDev& tq, int nvec, const double* partials, int grid, cudaStream_t st);
Status launch_tpq_fin(const TpqDev& tq, int k, int nvec, double inv_ns, double l, const double* partials, int grid,
                      cudaStream_t st);

}  // namespace hphi
