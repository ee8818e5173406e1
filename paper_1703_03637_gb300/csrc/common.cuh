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

// Split-row view of a fixed-S^z sector (section 3.1's split of a configuration into a high
// and a low part, used as the data layout of H v): s = (hi << L) | lo.  The rows with one
// value of hi are contiguous in the vector (ascending order sorts by hi first), start at
// hi_off[hi] and hold the C(L, q) low parts of popcount q = n_ones - popcount(hi).
// Exchange bonds fall into three groups: both sites low (act inside a row), both high (add
// whole rows), one of each ("straddling": row hi ^ 2^a, low part lo ^ 2^b).
constexpr int kSecMaxCls = 8;    // distinct exchange coefficients
constexpr int kSecMaxStr = 24;   // straddling exchange bonds
constexpr int kSecMaxStrSites = 16;  // distinct low sites of straddling bonds
constexpr int kSecMaxSp = 24;    // straddling S^z S^z pairs
constexpr int kSecMaxSl = 8;     // layers of straddling pairs
constexpr int kSecMaxL = 20;
constexpr int kSecMaxH = 22;
constexpr int kSecDtab = 2048;   // diagonal table entries

struct SecDev {
  int L, H, n_ones;
  int64_t dim;
  int K;                        // rows per tile of the row pass
  int hi_cols;                  // pass H columns per lane (0: the built-in 4 for int64, 8 for fp32)
  int nq_max;                   // longest row present
  // coefficients: exchange class c has coef[c]; the fp64 path sums integer multiples
  // mult[c] of one unit (coef[c] = mult[c] * unit) and scales once
  int n_cls;
  int one_cls;                  // every exchange bond has the same coefficient
  double coef[kSecMaxCls];
  int mult[kSecMaxCls];
  double unit;
  int qextra;                   // extra headroom bits of the quantised copy
  int dint;                     // the diagonal is an integer multiple of `unit` everywhere
  // low side
  // low-part tables cover the classes present: entry j - jbase for list position j, nJ of them
  uint32_t lo_off[kSecMaxL + 2];     // start of popcount class q in the list of all 2^L low parts
  uint32_t jbase, nJ;
  const uint32_t* lo_list;      // [nJ] low parts grouped by popcount, ascending
  // low neighbours in groups of four 16-bit slots: group g of entry j is lo_nbr4[g * nJ + j];
  // slot 4g + t holds the rank (in its class) of neighbour 4g + t, unused slots hold nq_max,
  // the index of a zero entry placed after the staged rows
  int lo_groups;
  const uint2* lo_nbr4;         // [lo_groups][nJ]
  const uint8_t* lo_cnt;        // [nJ] neighbours; entries are class-sorted
  const uint32_t* lo_cls4;      // [lo_groups][nJ] class byte of each slot (multi-class only)
  const uint16_t* lo_diag;      // [nJ] packed diagonal counts of the low part
  // high side
  const uint64_t* hi_off;       // [2^H] first row element of each high part
  int hi_slots;
  const uint32_t* hi_nbr;       // [hi_slots][2^H] neighbour high part | class << 24
  const uint8_t* hi_cnt;        // [2^H]
  const uint16_t* hi_diag;      // [2^H] packed diagonal counts of the high part
  // straddling exchange: high bit a, low bit b, class, index of b's rank table
  int n_str;
  uint8_t str_a[kSecMaxStr], str_b[kSecMaxStr], str_cls[kSecMaxStr], str_t[kSecMaxStr];
  const uint16_t* str_rank;     // [sites][nJ] rank (in its class) of lo ^ 2^b
  // straddling S^z S^z pairs: high bit a, low bit b, layer l.  Pairs of one layer have
  // distinct low bits, so per row the pairs whose high bit is set give one mask of low bits
  // per layer and the count is a popcount per layer; layer l counts into diagonal field sp_lg[l]
  int n_sp, n_sl;
  uint8_t sp_a[kSecMaxSp], sp_b[kSecMaxSp], sp_l[kSecMaxSp];
  uint8_t sp_lg[kSecMaxSl];
  // diagonal = dtab[n0 + d1 * n1] with n_g the packed counts (field g: 8 bits)
  int n_dg;                     // diagonal count groups (0, 1 or 2)
  int dstride;                  // d1
  int dtab_n;
  const double* dtab;           // [dtab_n]
  // row pass work: tiles of up to K rows of one class, in processing order
  int64_t n_tiles;
  const uint32_t* hi_seq;       // [2^H] high parts in processing order
  const uint32_t* tiles;        // [n_tiles] start in hi_seq | (rows - 1) << 24
  // high pass work: classes p ascending, stripes, rows of class p
  int n_pc;                     // classes present
  int pc_p[kSecMaxH + 1];       // popcount of each class present
  uint32_t pc_row0[kSecMaxH + 2];   // start of the class in hi_cls
  const uint32_t* hi_cls;       // [2^H] high parts grouped by popcount, ascending
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
  int exp_ready = 0;               // fp64 fixed-point paths (two-pass Hubbard, split-row): 0 scan
                                   // the input's exponent and quantise it; 1 the exponent is in the
                                   // scratch slot already (quantise only); 2 the quantised copy is
                                   // ready too (written by the previous Lanczos pass 2)
  int* pexp = nullptr;             // fp64 Lanczos pass 1 of those paths: atomicMax of the exponent
                                   // fields of the P values written (null: not tracked)
};

// The scratch slots through which a fp64 Lanczos pass 2 writes the next step's quantised copy:
// Q [dim] int64, its exponent slot, the pass-1 exponent slot and two slots for the exact
// exponent of the current / next vector (alternating by step).
struct QSlots {
  long long* Q = nullptr;
  int* eq = nullptr;               // exponent field E of Q's scale (q = round(x 2^(1078 - E - extra)))
  int* ep = nullptr;               // max exponent field of the pass-1 output P
  int* ec[2] = {nullptr, nullptr}; // exact max exponent field of C_k (k even / odd)
  int extra = 0;                   // extra headroom bits of the path
};
QSlots sec_qslots(const SecDev& d, int prec, Epi epi, void* scratch);
QSlots hub_qslots(const HubDev& md, void* scratch);

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

// fp64 -> 64-bit fixed point at one scale per vector (k_hub.cu): q = round(x 2^(1078 - E - extra)),
// E the largest exponent field of x (computed into *Ep unless exp_ready), |q| < 2^(56 - extra)
Status launch_quant_vec(const double* X, long long* Q, int64_t n, int* Ep, const int* done, bool exp_ready, int extra,
                        cudaStream_t st);

// Split-row spin-sector H v (k_sector.cu) ---------------------------------------------
// The compiled terms of a real S^z-sector spin model, as the term compiler produced them.
struct SecTerms {
  int n_sites = 0, n_ones = 0;
  std::vector<SpinEntry> ents;
  std::vector<double2> cls;
  double c0 = 0.0;
  std::vector<LinGroup> lin;
  std::vector<PairEntry> pairs;
  std::vector<double> pcoef;
};
struct SecTables;  // device tables of one split (L, K); defined in k_sector.cu
void sec_free(SecTables* t);
struct SecTablesDeleter {
  void operator()(SecTables* t) const { sec_free(t); }
};
// true when the model takes the split-row path (empty *why), else the reason
bool sec_applicable(const SecTerms& t, int prec, std::string* why);
// the split used when nothing else is asked: the largest L whose longest row fits one tile
// of K = 1 rows of element size esz (0: none fits)
int sec_default_L(const SecTerms& t, int esz);
// tile rows K for low-part length L at element size esz (largest power of two that fits)
int sec_default_K(const SecTerms& t, int L, int esz);
// K rows of the longest row of split L fit one tile at element size esz
bool sec_fits(const SecTerms& t, int L, int K, int esz);
Status sec_build(const SecTerms& t, int L, int K, SecTables** out, cudaStream_t st);
const SecDev& sec_dev(const SecTables* t);
size_t sec_scratch_bytes(const SecDev& d, int prec, Epi epi);
int sec_grid(const SecDev& d, int prec, Epi epi);
int* sec_exponent_slot(const SecDev& d, int prec, Epi epi, void* scratch);
Status launch_sec(const SecDev& d, int prec, const void* v, void* w, void* scratch, Epi epi, const FusedArgs& fa,
                  int grid, cudaStream_t st);

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
  double* ro;            // [2 (m + 1)] reorthogonalisation coefficients (re, im) of C_0 .. C_k
};

Status launch_lz_init(int prec, bool cplx, const void* v0_f64, void* C, void* P, int64_t n_real, double* partials,
                      int grid, cudaStream_t st);
Status launch_lz_init_fin(const LzDev& lz, const double* partials, int grid, cudaStream_t st);
Status launch_lz_fin1(const LzDev& lz, int k, const double* partials, int grid, cudaStream_t st);
// emax (fp64 only, may be null): atomicMax of the exponent fields of the new P
// qn (fp64, may be null): also writes the next step's quantised copy qn->Q on a scale bounded
// before the pass (see k_lz_pass2), its exponent into qn->eq; emax then receives the exact
// max exponent field of the new P (qn->ec for the next step)
struct QNext {
  long long* Q;
  int* eq;
  const int* ep;
  const int* ec_cur;
  int extra;
};
Status launch_lz_pass2(int prec, bool cplx, const LzDev& lz, int k, const void* C, void* P, double* x,
                       int64_t n_real, double* partials, int grid, int* emax, cudaStream_t st,
                       const QNext* qn = nullptr);
// replay: the refinement's second pass (stops after the last step with a significant Ritz
// coefficient, keeps the first pass's step count)
Status launch_lz_fin2(const LzDev& lz, int k, double brk, const double* partials, int grid, bool replay,
                      cudaStream_t st);
// the whole Lanczos recurrence in one thread-block cluster (real spin models of at most 32,768
// rows, both vectors in the cluster's shared memory): C0 holds C_0 (after k_lz_init / its
// finaliser); fills alpha, beta, sig, steps_done.  lz_cta_smem: bytes per CTA, 0 if the model
// does not take the path
size_t lz_cta_smem(const SpinDev& md);
Status launch_lz_cta(const SpinDev& md, const LzDev& lz, int steps, double brk, const double* C0, cudaStream_t st);
// full reorthogonalisation of the new P (slot k + 1 of the kept basis) against C_0 .. C_k,
// then the partial |P|^2 that launch_lz_fin2 reads; part holds ro_part_doubles(grid) doubles
size_t ro_part_doubles(int grid);
Status launch_reorth(int prec, bool cplx, const LzDev& lz, int k, const void* V, int64_t n_real, int64_t stride_real,
                     void* P, double* part, double* partials, int grid, cudaStream_t st);
int reorth_launches(int k);
// appendix C's test after a step: stop when T_n's first excited eigenvalue agrees with the
// previous test's to eps (relative)
Status launch_lz_conv(const LzDev& lz, double eps, cudaStream_t st);
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
  double* doub;          // [K][nvec] doubly occupied sites per site (observables on)
  double* sz;            // [K][nvec] S^z_total per site
  double* sz2;           // [K][nvec] (S^z_total)^2 per site
};

// device scalars of an inverse-iteration (CG) solve: s[0] |r|^2, s[1] alpha, s[2] beta,
// s[3] |b|^2, s[4] delta - E, s[5] tol^2, s[6] e, s[7] residual, s[8] variance, s[9] 1/|y|
struct CgDev {
  double* s;             // [16]
  int* done;             // [1] the current solve has converged
  int* steps;            // [1] CG iterations so far
};
Status launch_cg_shift(const CgDev& cg, const double* p, double* q, int64_t n, double* partials, int grid,
                       cudaStream_t st);
Status launch_cg_update(const CgDev& cg, int mode, const double* b, double* y, double* r, double* p, const double* q,
                        int64_t n, double* partials, int grid, cudaStream_t st);
Status launch_cg_dir(const CgDev& cg, const double* r, double* p, int64_t n, int grid, cudaStream_t st);
Status launch_cg_norm(const CgDev& cg, int mode, const double* y, double* x, int64_t n, double* partials, int grid,
                      cudaStream_t st);
Status launch_cg_rq(const CgDev& cg, int mode, const double* x, const double* hx, int64_t n, double* partials,
                    int grid, cudaStream_t st);
Status launch_cg_fin(const CgDev& cg, int mode, const double* partials, int grid, cudaStream_t st);

// what the diagonal-observable kernel needs to know of a row's configuration
struct ObsDev {
  int kind;                  // 0 spin (all 2^N), 1 spin (fixed popcount), 2 Hubbard
  int n_sites, n_ones;
  int64_t dim;
  int64_t dim_up;            // Hubbard: row = d * dim_up + u
  const uint32_t* list_up;   // Hubbard sector species lists (null: all 2^N)
  const uint32_t* list_dn;
};
Status launch_tpq_obs(int prec, bool cplx, const ObsDev& od, const void* X, int nvec, double* partials, int grid,
                      cudaStream_t st);
Status launch_tpq_obs_fin(const TpqDev& tq, int k, int nvec, double inv_ns, const double* partials, int grid,
                          cudaStream_t st);
Status launch_tpq_init(int prec, bool cplx, const void* psi0_f64, void* X, int64_t n_rows, int nvec,
                       double* partials, int grid, cudaStream_t st);
Status launch_tpq_init_fin(const TpqDev& tq, int nvec, const double* partials, int grid, cudaStream_t st);
Status launch_tpq_fin(const TpqDev& tq, int k, int nvec, double inv_ns, double l, const double* partials, int grid,
                      cudaStream_t st);

}  // namespace hphi
