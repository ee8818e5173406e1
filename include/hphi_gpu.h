/*
 * hphi_gpu.h -- C ABI of the GB300 (sm_103a) Lanczos / microcanonical-TPQ library for
 * two-body quantum lattice models, after Kawamura et al., "Quantum lattice model solver
 * HPhi", Comput. Phys. Commun. 217 (2017) 180.
 *
 * General rules for every entry point below
 *  - Status: every function returning int returns HPHI_OK (0) or a negative HPHI_ERR_*
 *    code; nothing is thrown across the ABI.  hphi_last_error() gives a message for the
 *    last failure on that model.
 *  - Ownership: the model handle, its term list, its basis tables and its solver
 *    workspace are allocated and freed by the library (cudaMalloc on the current device).
 *    Vectors passed to hphi_apply_H / hphi_random_vector are caller-owned DEVICE buffers;
 *    result arrays in the *_result structs are caller-owned HOST buffers.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work of a call is issued on it.  hphi_build_sector, hphi_lanczos_run and
 *    hphi_tpq_run synchronise the stream before returning (their results are host
 *    values); hphi_apply_H and hphi_random_vector are asynchronous.
 *  - Vector layout: row-major [dim][nvec]; row r is basis state r (section 3.1 order, see
 *    hphi_set_basis), nvec vectors interleaved per row.  Real models use double (or float
 *    for HPHI_FP32); complex models use interleaved (re, im) pairs.
 *  - Threading: a model may be used from one host thread at a time.
 */
#ifndef HPHI_GPU_H
#define HPHI_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hphi_model hphi_model;

/* Model kinds (section 2.3: "Spin" and "Fermion Hubbard" models). */
enum { HPHI_SPIN_HALF = 0, HPHI_HUBBARD = 1 };

/* Basis modes (section 3.1: full space, or the restricted space of fixed particle number /
 * fixed total S^z, enumerated in ascending bit-string order). */
enum { HPHI_BASIS_FULL = 0, HPHI_BASIS_SZ = 1, HPHI_BASIS_NUMBER = 2 };

/* Vector storage precision.  HPHI_FP64: fp64 storage and arithmetic.  HPHI_FP32: fp32
 * storage and fp32 H v, with every inner product accumulated to fp64. */
enum { HPHI_FP64 = 0, HPHI_FP32 = 1 };

enum {
  HPHI_OK = 0,
  HPHI_ERR_INVALID_ARG = -1,    /* bad argument, index out of range, wrong model kind      */
  HPHI_ERR_BASIS_MISMATCH = -2, /* a term does not conserve the chosen sector             */
  HPHI_ERR_OUT_OF_MEMORY = -3,  /* device allocation failed                               */
  HPHI_ERR_NOT_BUILT = -4,      /* hphi_build_sector has not run since the last change    */
  HPHI_ERR_CUDA = -5,           /* a CUDA runtime call failed (message has the details)   */
  HPHI_ERR_UNSUPPORTED = -7     /* valid request outside what this library implements     */
};

/* ---------------------------------------------------------------- model definition */

/* Creates an empty model.  kind: HPHI_SPIN_HALF (1 <= n_sites <= 63) or HPHI_HUBBARD
 * (1 <= n_sites <= 24 per spin species).  *out receives the handle. */
int hphi_create(hphi_model** out, int kind, int n_sites);

/* Frees the model and all device memory the library allocated for it.  NULL is ignored. */
void hphi_destroy(hphi_model* m);

/* Message of the last failure on m (or of the last failed hphi_create if m is NULL). */
const char* hphi_last_error(const hphi_model* m);

/* Spin model, section 2.3 ("Spin"): adds sum_{a,b} J[3a+b] S_i^a S_j^b with a, b in
 * {x, y, z}, i != j.  J is a row-major 3x3 host array.  Heisenberg: J = J0 * identity;
 * Kitaev gamma-bond: a single diagonal entry. */
int hphi_add_spin_coupling(hphi_model* m, int i, int j, const double J[9]);

/* Spin model, section 2.3: adds - (h[0] S_i^x + h[1] S_i^y + h[2] S_i^z)  (the paper's
 * -h S^z - Gamma S^x generalised to any direction). */
int hphi_add_spin_field(hphi_model* m, int i, const double h[3]);

/* Hubbard model, section 2.3 ("Fermion Hubbard"): adds - t c+_{i s} c_{j s} - conj(t)
 * c+_{j s} c_{i s}, i != j, spin s = 0 (up) or 1 (down).  Fermion sign convention: modes
 * are ordered (up 0 .. N-1, down 0 .. N-1) (Jordan-Wigner order). */
int hphi_add_hopping(hphi_model* m, int i, int j, int spin, double t_re, double t_im);

/* Hubbard: adds U n_{i up} n_{i dn}. */
int hphi_add_onsite_U(hphi_model* m, int i, double U);

/* Hubbard: adds V n_i n_j (i != j), n_i = n_{i up} + n_{i dn}. */
int hphi_add_density(hphi_model* m, int i, int j, double V);

/* Hubbard: adds - mu n_i. */
int hphi_add_chemical_potential(hphi_model* m, int i, double mu);

/* Selects the basis (section 3.1).  Spin: HPHI_BASIS_FULL (all 2^N configurations, row r
 * is configuration r, bit i = site i, bit 1 = up) or HPHI_BASIS_SZ with a = number of up
 * spins (rows = configurations with popcount a, ascending).  Hubbard: HPHI_BASIS_FULL
 * (row = dn * 2^N + up) or HPHI_BASIS_NUMBER with a = N_up, b = N_dn (row = rank(dn) *
 * C(N, a) + rank(up)).  Invalidates previously built tables. */
int hphi_set_basis(hphi_model* m, int basis, int a, int b);

/* Compiles the term list (section 3.3: diagonal folded into integer bit counts per
 * coefficient class; off-diagonal terms as XOR masks with phase tables), checks that
 * every term conserves the sector (HPHI_ERR_BASIS_MISMATCH otherwise), and builds the
 * split-half rank tables of the restricted space on the device (section 3.1).  *dim_out
 * (may be NULL) receives the dimension. */
int hphi_build_sector(hphi_model* m, int64_t* dim_out, void* stream);

/* Dimension of the built basis, or a negative status. */
int64_t hphi_dim(const hphi_model* m);

/* 1 if H has complex elements (J^{xy}-type couplings, h_y fields or complex hopping). */
int hphi_is_complex(const hphi_model* m);

/* Basis decode on the device: states[k] = configuration of row r0 + k, k < n (spin: the
 * bit string; Hubbard: up | (dn << 32)).  states: device uint64_t[n]. */
int hphi_basis_states(hphi_model* m, int64_t r0, int64_t n, uint64_t* states, void* stream);

/* Basis rank on the device: ranks[k] = row of configuration states[k] (same encoding as
 * hphi_basis_states), or -1 if it is outside the basis.  Device arrays of length n. */
int hphi_basis_ranks(hphi_model* m, const uint64_t* states, int64_t n, int64_t* ranks, void* stream);

/* ---------------------------------------------------------------- H v (section 3.3) */

/* w = H v for nvec interleaved vectors.  v, w: device buffers [dim][nvec] of the model's
 * scalar type in precision prec (HPHI_FP64 or HPHI_FP32); v and w must not overlap.
 * Matrix-free: every element is generated on the fly from the bit strings.  Scratch the
 * kernels need lives in the model's workspace, allocated on first use and kept: the two-pass
 * Hubbard path one vector; fp64 on spin models one vector of 64-bit integers (the quantised
 * input; for the generic kernel only if the device has room, else its per-term fixed-point
 * sums run instead). */
int hphi_apply_H(hphi_model* m, const void* v, void* w, int nvec, int prec, void* stream);

/* Allocation-free w = H v.  The paper has no counterpart: this is a service for callers
 * that must not allocate device memory while they run -- code that enqueues work from a
 * CUDA host callback or another context where cudaMalloc is not permitted, real-time loops
 * that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree, and
 * applications whose memory is fully pre-reserved by their own allocator.  It computes the
 * same product as hphi_apply_H for one fp64 vector (prec = HPHI_FP64, nvec = 1) of a real
 * Hubbard model with one hopping value per spin species, and allocates nothing: its
 * scratch (16 bytes per basis row + 256 bytes) is a fixed 64 MiB device array inside the
 * library, so the basis may have at most 4,194,288 rows; larger bases return
 * HPHI_ERR_INVALID_ARG with the limit in the message, other models HPHI_ERR_UNSUPPORTED.
 * v and w are caller-owned device buffers [dim] of double and must not overlap.  A call on a
 * stream that is not being captured looks up the array's device address afresh (after a
 * device reset or a context switch it is the current one); a call on a capturing stream uses
 * the address of the device's last uncaptured call, so make one uncaptured call on the device
 * before any stream capture.  Every call on a device shares the one array,
 * so calls whose GPU work overlaps (different streams or threads without ordering between
 * them) race and give wrong results; calls ordered on one stream are safe.  The array is
 * held by every GPU that loads the library until the process exits. */
int hphi_apply_H_noalloc(hphi_model* m, const void* v, void* w, void* stream);

/* Frees the solver workspace of m (the vectors and scratch that hphi_apply_H,
 * hphi_lanczos_run, hphi_tpq_run and hphi_autotune allocate on first use and keep); the terms,
 * basis tables and launch choices stay.  The next call allocates what it needs again.  Waits
 * for the device first (cudaDeviceSynchronize).  Useful between runs of different precision or
 * size on large bases, whose buffers would otherwise stay at their largest size.  No
 * counterpart in the paper. */
int hphi_release_workspace(hphi_model* m);

/* ---------------------------------------------------------------- autotuning */

typedef struct {
  int n_candidates;    /* launch configurations timed (0: nothing to tune for this model)      */
  int best_dn_ept;     /* chosen columns per thread of the down-spin pass                       */
  int best_up_k;       /* chosen rows per shared-memory tile of the up-spin pass                */
  float best_ms;       /* H v time of the chosen configuration                                  */
  float default_ms;    /* H v time of the built-in default                                      */
  float worst_ms;      /* H v time of the slowest candidate                                     */
  int best_split_L;    /* split-row spin path: chosen low-part length L (0: path not tuned)      */
  int best_split_K;    /* split-row spin path: chosen rows per shared-memory tile                */
  int best_split_hi_cols; /* split-row spin path: chosen high-pass columns per lane (4 or 2 int64,
                          8 or 4 fp32)                                                          */
} hphi_tune_result;

/* Times the launch configurations of the model's H v at precision prec (HPHI_FP64 or
 * HPHI_FP32) on a seeded vector and keeps the fastest for every later hphi_apply_H /
 * hphi_lanczos_run / hphi_tpq_run on this model.  The two-pass Hubbard path is tuned over
 * columns per thread of the down-spin pass x rows per tile of the up-spin pass.  Real spin
 * models in an S^z sector that take the split-row path (see hphi_set_sector_split) are tuned
 * over the split: the default low part and up to two bits fewer, each with every tile height
 * that fits, and then over the high pass's columns per lane on the chosen split.  A real spin model in its full basis has every S^z sector of at least 2^20 rows
 * tuned that way: hphi_lanczos_run_sectors keeps those sectors' shapes; the result then
 * counts the candidates of all of them and reports the timings of the largest.  Other models
 * report n_candidates = 0.  Uses the model's workspace (and the sectors' own); synchronises
 * the stream.  *out may be NULL.  No counterpart in the paper (its CPU code has no launch
 * shapes). */
int hphi_autotune(hphi_model* m, int prec, hphi_tune_result* out, void* stream);

/* Split-row H v of real spin models in an S^z sector, section 3.1's split of a configuration
 * into a high and a low part (the split-half search) turned into the data layout: the rows
 * of one high part are contiguous, K of them are staged in shared memory, exchange bonds
 * inside the low part act in the staged rows, bonds inside the high part add whole rows
 * (one stripe-ordered pass through L2), and the few bonds that straddle the split gather
 * from one partner row each.  It applies to one real vector (nvec = 1) when every exchange
 * term flips two antiparallel spins with one real element and the diagonal has at most two
 * coefficient groups beyond a constant (Heisenberg, XXZ and J1-J2 models on regular lattices);
 * fp64 also needs the exchange couplings to be small integer multiples of one power of two.
 * Other models use the generic gather kernel.  This call chooses the split used for prec:
 * L = -1 turns the path off (generic kernel), L = 0 restores the default (the largest low
 * part whose rows fit one shared-memory tile), 1..20 forces the low part's length; K = 0
 * picks the widest tile that fits, 1/2/4/8 forces the rows per tile.  The device tables of
 * the split are built here (a host loop over 2^L low and 2^(N-L) high parts, then an upload
 * on `stream`, which is synchronised).  Results agree with the generic kernel to rounding
 * (fp32) or exactly up to the final conversion (fp64 fixed-point sums).  Returns
 * HPHI_ERR_UNSUPPORTED (with the reason) for a model the path does not cover and
 * HPHI_ERR_INVALID_ARG when the forced split does not fit.  No counterpart in the paper. */
int hphi_set_sector_split(hphi_model* m, int prec, int L, int K, void* stream);

/* Window passes of the many-vector H v (full-basis spin models, nvec in {32, 64, 128, 256}):
 * section 4.3's continuous-memory-access idea on one GPU.  Each pass takes the terms whose
 * flipped sites lie in one cyclic window of `bits` sites and visits the rows with that
 * window's bits varying fastest, so a pass's gathers hit a block of rows small enough to
 * stay in L2 instead of reaching across the whole vector in HBM.  bits = -1 (the default)
 * runs one pass, 0 sizes the window so that a block of input rows fills about a quarter of
 * L2, 1..32 forces a window size (a window covering all sites means one pass).  At most 8
 * passes; a plan that needs more falls back to one pass.  The passes cut HBM traffic about
 * threefold on the 2^24-row Kitaev cluster but add instructions, and one pass is already
 * bound by instruction issue there, hence the default.  The Lanczos step (one vector) is not
 * affected.  Results agree with one pass up to floating-point summation order. */
int hphi_set_window_bits(hphi_model* m, int bits);

/* ---------------------------------------------------------------- start vectors */

/* Fills v (device, [dim][nvec], precision prec) with standard-normal numbers (a seeded
 * Gaussian start vector) from the counter-based generator Philox4x32-10 (Salmon et al.,
 * SC'11) and the Box-Muller transform: Philox block p uses counter (p mod 2^32, p >> 32, 0, 0)
 * and key (seed mod 2^32, seed >> 32); its words w0, w1 give the 53-bit uniform
 * u_a = ((((w0 << 32) | w1) >> 11) + 0.5) / 2^53 and w2, w3 likewise u_b, and the block's pair
 * is g0 = sqrt(-2 ln u_a) cos(2 pi u_b), g1 = sqrt(-2 ln u_a) sin(2 pi u_b).  The elements
 * e = r * nvec + c of a complex vector are g0 + i g1 of block e; those of a real vector are g0
 * (e even) and g1 (e odd) of block e / 2.  prec = HPHI_FP64 evaluates the transform in fp64;
 * HPHI_FP32 rounds the same uniforms to fp32 and evaluates it in fp32 arithmetic (values
 * within a few fp32 ulps of the fp64 numbers).  Appendix A.2 / A.4 draw every coefficient of
 * the initial vector from dSFMT, whose stream depends on the process count; this generator
 * depends on the seed and the element index only. */
int hphi_random_vector(hphi_model* m, void* v, int nvec, int prec, uint64_t seed, void* stream);

/* Raw Philox4x32-10 on the device: for k < n, out[4k..4k+3] = Philox(ctr[4k..4k+3],
 * key[2k..2k+1]).  All pointers are device arrays. */
int hphi_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, void* stream);

/* ---------------------------------------------------------------- Lanczos (section 3.4) */

typedef struct {
  int steps;           /* m: number of H v products (size of T_m); 1..4096               */
  int prec;            /* HPHI_FP64 or HPHI_FP32                                         */
  uint64_t seed;       /* start vector seed if v0 == NULL (hphi_random_vector, nvec = 1) */
  const void* v0;      /* optional device start vector [dim], always fp64 (complex128 for
                          complex models); it is normalised internally                   */
  int n_eig;           /* lowest eigenvalues of T_m to return, 1..8                      */
  int refine;          /* 1: rebuild the Ritz vector x of the lowest eigenvalue by a second
                          Lanczos pass (section 3.4) in fp64 and return the fp64 Rayleigh
                          quotient, residual |Hx - Ex| / |x| and variance (appendix A.3)   */
  double breakdown;    /* stop when beta_{k+1} <= breakdown * max(1, |alpha_k|); 0 -> 1e-13 */
  int profile;         /* 1: time every fused H v launch with CUDA events (hv_ms below)   */
  int keep_basis;      /* refinement source: 1 keep all m Lanczos vectors in device memory
                          and form x = V_m e~ in one streaming pass; -1 replay the recurrence
                          (section 3.4's second pass), stopping after the last step whose
                          Ritz coefficient still matters at the storage precision; 0 keep
                          them when they fit in 60% of the free device memory, else replay */
  int v0_on_host;      /* 1: v0 is a HOST array [dim] of fp64 (complex128 for complex models),
                          copied by the call into its own first Lanczos vector (for prec =
                          HPHI_FP32 through the model's fp64 work vector), so the caller needs no
                          device copy of it; the refinement's second pass copies it again.  Such
                          runs launch their kernels one by one instead of as one CUDA graph.
                          Pinned (page-locked) memory copies fastest.  0: v0 is a device array */
  double eps;          /* appendix C's convergence test (LanczosEps): after 5 steps and then
                          every 2, the first excited eigenvalue of T_n is found on the device
                          and the run stops when it agrees with the previous test's value to
                          eps relative; steps is then the limit.  0: run all steps       */
  void* ritz_out;      /* optional device fp64 [dim] (complex128 for complex models): with
                          refine = 1 receives the fp64 Ritz vector x of the lowest eigenvalue
                          (the start of hphi_inverse_iteration); NULL: not copied out     */
  int reorth;          /* 1: full reorthogonalisation: after every step the new vector is
                          orthogonalised against all kept Lanczos vectors (classical Gram-
                          Schmidt, every inner product and update in fp64); keeps the m + 1
                          vectors in device memory (HPHI_ERR_OUT_OF_MEMORY if they do not
                          fit) and costs (k + 1) extra vector reads at step k.  The paper's
                          recurrence (section 3.4) has none: 0, the default               */
} hphi_lanczos_params;

typedef struct {
  int steps_done;      /* steps actually taken (< steps only at breakdown)               */
  double* alpha;       /* caller host array [steps] or NULL: alpha_0 .. alpha_{m-1}      */
  double* beta;        /* caller host array [steps] or NULL: beta_1 .. beta_m            */
  double eig[8];       /* lowest n_eig eigenvalues of T_m, ascending                     */
  double e_refined;    /* refine = 1: <x|H|x> / <x|x> in fp64                            */
  double residual;     /* refine = 1: |H x - E x| / |x|                                   */
  double variance;     /* refine = 1: <H^2> - <H>^2 for x / |x|                            */
  float device_ms;     /* device time of the call's GPU work (CUDA events on the stream)  */
  float hv_ms;         /* profile = 1: summed device time of the fused H v launches       */
  int hv_launches;     /* number of fused H v launches timed in hv_ms                      */
  int kernel_launches; /* CUDA kernels this call launched                                   */
  int converged;       /* 1 when the eps test ended the run (steps_done < steps possible)  */
} hphi_lanczos_result;

/* Lanczos recurrence of section 3.4 (alpha_k = (H v_k, v_k), w = H v_k - beta_k v_{k-1} -
 * alpha_k v_k, beta_{k+1} = |w|, v_{k+1} = w / |w|) on the device, with the H v product
 * fused with the vector update and every reduction accumulated in fp64; then the lowest
 * eigenvalues of the tridiagonal T_m by Sturm bisection in fp64 on the device. */
int hphi_lanczos_run(hphi_model* m, const hphi_lanczos_params* p, hphi_lanczos_result* r, void* stream);

/* Lanczos in several S^z sectors at once (spin models; the model's own basis setting is not
 * used).  Sector i has n_up_list[i] up spins; its tables are built on first use and kept
 * until the terms change.  All sectors' runs -- fused steps, eigensolve and optional
 * refinement -- are captured into one CUDA graph as parallel branches and launched once, so
 * sectors of very different dimension (1 .. C(N, N/2)) run side by side.  Each sector's
 * start vector is hphi_random_vector with seed p->seed + n_up_list[i]; p->v0 must be NULL
 * and p->profile is ignored.  results: caller host array [n_sectors], each filled as by
 * hphi_lanczos_run (alpha / beta host arrays of p->steps entries, or NULL); device_ms is the
 * time of the whole graph.  1 <= n_sectors <= 64, sectors distinct, n_sites <= 40.  The
 * paper runs one sector per job; batching sectors is this library's. */
int hphi_lanczos_run_sectors(hphi_model* m, const int* n_up_list, int n_sectors, const hphi_lanczos_params* p,
                             hphi_lanczos_result* results, void* stream);

/* ---------------------------------------------------------------- inverse iteration (section 3.4.1) */

typedef struct {
  double energy;       /* E_n: the eigenvalue estimate (e.g. hphi_lanczos_result.eig[0])   */
  double shift;        /* delta > 0: the CG operator is H - E_n + delta, positive definite
                          when E_n is at most delta above the lowest eigenvalue;
                          0 -> 1e-4 * max(1, |E_n|)                                        */
  int outer;           /* inverse-iteration steps y_k -> y_{k+1}: 1..64                     */
  int max_cg;          /* CG iterations per solve: 1..100000                               */
  double cg_tol;       /* a solve stops when |r| <= cg_tol |b| (0 -> 1e-12)               */
} hphi_invit_params;

typedef struct {
  double e;            /* <x|H|x> of the final unit vector                                 */
  double residual;     /* |H x - e x|                                                       */
  double variance;     /* <x|H^2|x> - e^2                                                   */
  int cg_steps;        /* CG iterations run over all solves                                */
  float device_ms;     /* device time of the call                                           */
  int kernel_launches; /* CUDA kernels this call launched                                   */
} hphi_invit_result;

/* Inverse iteration by conjugate gradients (section 3.4.1): (H - E_n + delta) y_{k+1} = y_k,
 * y_0 = x, each solve starting from its right-hand side, y_{k+1} normalised into x.  x is a
 * device fp64 [dim] vector (complex128 for complex models) owned by the caller: in, the start
 * vector (the Lanczos eigenvector); out, the unit result.  Besides x the call keeps four more
 * vectors of the model's dimension in the model's workspace (released by
 * hphi_release_workspace).  Every product and reduction is fp64; a solve's scalars stay on
 * the device, and the host reads its convergence flag every 16 iterations.  Synchronises
 * the stream before returning. */
int hphi_inverse_iteration(hphi_model* m, const hphi_invit_params* p, void* x, hphi_invit_result* r, void* stream);

/* ---------------------------------------------------------------- mTPQ (section 3.5) */

typedef struct {
  int n_starts;        /* independent random initial vectors, run interleaved: 1..256   */
  int steps;           /* K: number of multiplications by (l - H / N_s)                  */
  double l;            /* the constant l                                                  */
  double n_s;          /* N_s (0 -> number of sites)                                       */
  uint64_t seed;       /* start vectors: hphi_random_vector(seed, nvec = n_starts)        */
  const void* psi0;    /* optional device [dim][n_starts] fp64 start block (complex128 for
                          complex models); normalised internally per start               */
  int prec;            /* HPHI_FP64 or HPHI_FP32 (fp32 storage, fp64 norms and energies)   */
  int profile;         /* 1: launch the steps one by one (no graph) and time every fused H v
                          launch group with CUDA events (hv_ms below)                      */
  int obs_every;       /* diagonal observables of psi_k for k % obs_every == 0 (0: none); one
                          extra read of the state per measured record                     */
} hphi_tpq_params;

typedef struct {
  double* u;           /* host [steps][n_starts]: u_k = <psi_k|H|psi_k> / N_s             */
  double* h2;          /* host [steps][n_starts]: <psi_k|H^2|psi_k> / N_s^2              */
  double* norm;        /* host [steps][n_starts]: |(l - H/N_s) psi_k|                     */
  float device_ms;     /* device time of the TPQ loop                                      */
  int kernel_launches; /* CUDA kernels this call launched                                   */
  float hv_ms;         /* profile = 1: summed device time of the fused H v launch groups   */
  int hv_launches;     /* number of fused H v launch groups timed in hv_ms                  */
  double* beta;        /* host [steps][n_starts] or NULL: inverse temperature of record k,
                          beta_k = (2k / N_s) / (l - u_k) (section 3.5)                     */
  double* spec_heat;   /* host [steps][n_starts] or NULL: specific heat per site,
                          beta_k^2 (<H^2>_k - <H>_k^2) / N_s = beta_k^2 N_s (h2 - u^2)      */
  double* doublon;     /* host [steps][n_starts] or NULL: <psi_k| sum_i n_i,up n_i,dn |psi_k>
                          / N_s (0 for spin models); NaN for records not measured          */
  double* sz;          /* host [steps][n_starts] or NULL: <S^z_total> / N_s, NaN if not measured */
  double* sz2;         /* host [steps][n_starts] or NULL: <(S^z_total)^2> / N_s, NaN if not
                          measured (times beta: the uniform susceptibility per site)      */
} hphi_tpq_result;

/* Microcanonical TPQ (section 3.5): psi_{k+1} = (l - H/N_s) psi_k / |(l - H/N_s) psi_k| for
 * all starts at once, one fused pass per step (H psi, the update, and the fp64 per-start
 * reductions <psi|H psi> and |H psi|^2); the norm |(l - H/N_s) psi_k|^2 = l^2 - 2 l u_k +
 * <H^2>_k follows from them, so l must lie above the spectrum per site (the method's
 * condition), which keeps that difference free of cancellation.  Record k describes psi_k, the state
 * the (k+1)-th multiplication acts on, for k = 0 .. steps-1; the inverse temperature is
 * beta_k = (2k / N_s) / (l - u_k).  With obs_every > 0 the diagonal observables of section 3.5's
 * estimate <A>_beta_k = <psi_k|A|psi_k> / N_s (doubly occupied sites, S^z_total, its square) are
 * reduced in fp64 from the stored state by one extra kernel per measured record. */
int hphi_tpq_run(hphi_model* m, const hphi_tpq_params* p, hphi_tpq_result* r, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HPHI_GPU_H */
