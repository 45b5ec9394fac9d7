/*
 * hfx.h -- C ABI of the GB300 exact-exchange (HFX) force and stress library.
 *
 * The library evaluates, for a periodic structure, the LRI exchange energy
 * of Eq. exx_expand (paper Sec. 2)
 *
 *   E = - sum_{A in cell} sum_{F,B,G} C^A_{AF} V_{AB} C^B_{BG}
 *                                     (D_AB D_FG + D_AG D_FB)
 *
 * with real, fixed D, together with the force part that comes from the
 * variation of C and V (F^X1, Eq. Fexx1) and the matching stress
 * (sigma^X1, Eq. stress).  The problem statement is the paper's: given C, V,
 * their nuclear gradients and a fixed D, return F^X1 and sigma^X1 (Sec. 2,
 * after Eq. HD_ES, and Sec. 3.1).  The blocks C, V and their gradients come
 * from the built-in block model evaluated at the caller's positions:
 *
 *   C_{I,(J,R)} = G_{s(I)s(J)} f(r) [+ G'_{s(I)s(J)} f(r) (d.e)/R_C]
 *   V_{I,(J,R)} = M_{s(I)s(J)} h(r)
 *   f(r) = (1 - (r/R_C)^2)^3 exp(-r^2/2) for r < R_C = 2 r_c, else 0
 *   h(r) = erfc(omega r) / (r + 1)
 *
 * where d = tau_J + R.L - tau_I, r = |d|, and on-site blocks (I = J, R = 0)
 * do not move (their gradients vanish, Sec. 3.1).  Items are screened in two
 * steps (Sec. 3.2, Algorithm 1): per-tensor Frobenius-norm filters, then a
 * Cauchy-Schwarz bound per item.
 *
 * Conventions for every entry point:
 *  - Every call returns an hfx_status; no C++ exception crosses the ABI.
 *  - Outputs are written only when the call returns HFX_OK.
 *  - A plan is bound to one CUDA stream and one device and is not thread
 *    safe; calls on one plan must be serialised by the caller.  Different
 *    plans may be created and evaluated from different host threads at the
 *    same time (each on its own stream); the library's shared state is only
 *    the kernels' attributes, set to the same values by every plan.
 *  - Units: positions and lattice in Angstrom; E in model units; F in E/A;
 *    sigma in E/A^3, row-major 3x3, symmetric within rounding for the
 *    isotropic model.
 *  - Failing CUDA calls give HFX_ERR_CUDA; allocation failures HFX_ERR_OOM;
 *    bad arguments (null pointers, non-finite numbers, out-of-range species
 *    or indices, singular lattice) HFX_ERR_INVALID.  hfx_last_error()
 *    returns a message for the last failing call on a plan.
 */
#ifndef HFX_H_
#define HFX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HFX_OK = 0,
  HFX_ERR_INVALID = 1,
  HFX_ERR_OOM = 2,
  HFX_ERR_CUDA = 3,
  HFX_ERR_TIMEOUT = 4,
  HFX_ERR_PAIRLIST_STALE = 5,
  HFX_ERR_UNSUPPORTED = 6
} hfx_status;

/* Arithmetic of the contraction.  HFX_FP64 runs every step in FP64.  The
 * other values select split-precision tensor-core contractions with FP32
 * accumulation and FP64 screening, force, stress and energy reduction:
 * every operand is written as 2 (BF16X3) or 3 (BF16X6) bf16 pieces and the
 * piece products above 2^-16 (BF16X3) or 2^-24 (BF16X6) of the operands'
 * scale are kept.  (Value 1 is not assigned.) */
enum { HFX_FP64 = 0, HFX_BF16X3 = 2, HFX_BF16X6 = 3 };

/* Exchange products of Eq. exx_expand: bit 0 = D_AB D_FG, bit 1 = D_AG D_FB. */
enum { HFX_TERM_AB_FG = 1, HFX_TERM_AG_FB = 2, HFX_TERMS_ALL = 3 };

typedef struct hfx_plan hfx_plan; /* opaque, owned by the library */

/* The structure (Eqs. 1-2: atom I of the cell plus lattice vector R). */
typedef struct {
  int n_atoms;            /* > 0 */
  const int* species;     /* [n_atoms], each in 0..n_species-1; host memory */
  double lattice[9];      /* rows a1, a2, a3 (Angstrom); det != 0 */
  const double* positions;/* [n_atoms*3] Cartesian (Angstrom); host memory */
} hfx_system;

/* The block model and the fixed density matrix (host memory; copied by
 * hfx_plan_create, so the caller may free it afterwards). */
typedef struct {
  int n_species;                  /* 1..16 */
  const int* n_ao;                /* [n_species], 1..32 orbitals per atom */
  const int* n_abf;               /* [n_species], 1..128 auxiliary functions */
  double r_c;                     /* > 0; C range R_C = 2 r_c (Angstrom) */
  double omega;                   /* > 0; screening of h(r) (1/Angstrom) */
  const double* const* G;         /* [s*n_species+t] -> n_abf(s)*n_ao(s)*n_ao(t), row-major */
  const double* const* M;         /* [s*n_species+t] -> n_abf(s)*n_abf(t); M_ts = M_st^T,
                                     M_ss symmetric (gives V_BA = V_AB^T, Sec. 3.1) */
  const double* const* G_aniso;   /* NULL, or like G: anisotropic C term */
  double aniso_dir[3];            /* unit vector e of the anisotropic term */
  long long n_d;                  /* number of D blocks */
  const int* d_index;             /* [n_d*5] rows (I, J, R1, R2, R3), any order, no duplicates */
  const long long* d_offset;      /* [n_d+1] element offsets into d_values */
  const double* d_values;         /* block k is n_ao(I)*n_ao(J) row-major; both orientations
                                     must be present with D_JI(-R) = D_IJ(R)^T */
} hfx_model;

typedef struct {
  /* Screening thresholds (Sec. 3.2): step 1 drops a C pair only if
   * ||C|| <= theta_C and ||grad C|| <= theta_dC (likewise V), and a D
   * block if ||D|| <= theta_D (Frobenius norms).  Step 2 drops an item
   * whose Cauchy-Schwarz bound is <= theta_CS.  0 disables a filter. */
  double theta_C, theta_dC, theta_V, theta_dV, theta_D, theta_CS;
  int precision;      /* HFX_FP64 (default) or a split-precision mode */
  int terms;          /* HFX_TERMS_ALL by default */
  double skin;        /* Verlet skin of the pair lists (Angstrom), default 0.5 */
  int freeze_lists;   /* 1: keep pair lists and the first call's screening
                         decisions; a move beyond skin/2 gives
                         HFX_ERR_PAIRLIST_STALE.  0: lists are rebuilt when
                         stale and screening is redone on every call. */
  /* Home atoms.  Eq. exx_expand sums over the atom A of the home cell; the
   * plan sums A over [home_begin, home_end) only, so that E, F and sigma
   * are that range's share and the shares of disjoint ranges add up to the
   * whole (the paper distributes the atom quartets over processes the same
   * way, Sec. 3.3).  home_begin = home_end = 0 (the default) takes every
   * atom; otherwise 0 <= home_begin < home_end <= n_atoms (HFX_ERR_INVALID
   * otherwise).  F still has n_atoms rows: a range's items move atoms
   * outside it too. */
  int home_begin, home_end;
  /* Home atoms per pass of the contraction.  The Y blocks are built once per
   * evaluation; the per-call operand stores of the two exchange products
   * then hold one pass of home atoms at a time, so this bounds the memory
   * they take (roughly proportional to it).  0 (the default) = 128; larger
   * values save a little launch overhead, smaller ones memory. */
  int home_chunk;
  /* 1: replay the evaluations of a frozen plan (freeze_lists = 1) from a
   * CUDA graph.  Once the first call has fixed the screening decisions and
   * sized every store, an evaluation is a fixed sequence of launches whose
   * inputs (positions, lattice) sit in device memory: the second call
   * records it (stream capture on a stream of the plan's own, since the
   * plan's stream may be the legacy default stream) and every later call
   * launches the graph on the plan's stream.
   * Per-stage timing (hfx_set_timing) evaluates without the graph;
   * hfx_plan_autotune records a new one.  0 (the default): launch every
   * kernel on each call. */
  int graph;
  void* stream;       /* cudaStream_t for every launch and copy; NULL = legacy default */
  int device;         /* CUDA device ordinal */
  /* Device memory of the plan.  NULL (the default) = cudaMalloc / cudaFree.
   * Otherwise alloc returns `bytes` of device memory on `device` for use on
   * `stream` (the plan's stream), at least 256-byte aligned, or NULL when it
   * cannot (the call then fails with HFX_ERR_OOM), and free gives back a
   * block alloc returned, with its size.  Both are called on the thread
   * that called into the plan: in hfx_plan_create, in evaluations that grow
   * a per-call store, and in hfx_plan_destroy (after the plan's stream has
   * drained).  A stream-ordered caching allocator, such as PyTorch's, fits;
   * alloc_ctx is passed through unchanged.  alloc and free are set
   * together or not at all. */
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* alloc_ctx;
  /* 1: a deterministic reduction (Sec. 2, the sums of Eq. Fexx1 and Eq.
   * stress over pairs).  Every sum that several CTAs add to (E, the virial,
   * the per-pair gradients g^C and g^V, and F) is kept as an exact 128-bit
   * fixed-point integer in units of 2^-64 instead of an FP64 atomic sum,
   * and rounded to FP64 once at the end.  Integer sums do not depend on
   * the order of the additions, and every contribution is computed in a
   * fixed order inside its CTA, so E, F and sigma are bit-identical from
   * run to run, for any launch shape the autotuner picks and any split into
   * passes of home atoms (results differ from the FP64 atomic sums by
   * their rounding, about 1e-15 relative).  Costs 16 bytes per pair
   * gradient component and atom force component of device memory and two
   * integer atomics per addition.  0 (the default): FP64 atomic sums,
   * repeatable to rounding order (about 1e-15). */
  int deterministic;
} hfx_options;

/* Counters of the last call (FLOPs are the algorithmic count of the
 * factorised contraction; times are CUDA-event times per stage in ms when
 * timing was requested via hfx_set_timing: ms_blocks the block norms,
 * ms_screen both screening steps and the item lists, ms_y the operand
 * stores shared by all passes and the Y blocks, ms_term1 the per-pass
 * operand stores and the first exchange product, ms_term2 the second
 * product, ms_reduce forces, stress and energy). */
typedef struct {
  long long c_pairs, v_pairs, d_blocks;        /* kept after step 1 */
  long long triplets, term1_pairs, term2_pairs; /* kept after step 2 */
  long long y_blocks;                           /* Y^{XZ} = sum_W C_XW D_WZ built */
  double flops_y, flops_term1, flops_term2, flops_total;
  double ms_blocks, ms_screen, ms_y, ms_term1, ms_term2, ms_reduce, ms_total;
  long long device_bytes;                       /* device memory held by the plan */
  long long kernel_launches;                    /* CUDA kernels this library launched during the call
                                                   (all threads: exact when one plan evaluates at a time) */
  int passes;                                   /* passes of home atoms (home_chunk) */
  int graph_replayed;                           /* 1 if the call launched the plan's CUDA graph */
  /* CUDA-event times (ms, with timing on) of the contraction kernels alone,
   * summed over the passes: the first product's kernel (ms_term1 without
   * the per-pass operand stores) and the second product's kernels. */
  double ms_term1_kernel, ms_term2_kernel;
  /* Error of this result against the reference set by hfx_set_reference
   * (-1 when none is set): |E - E_ref| / |E_ref|, and max|x - x_ref| /
   * max|x_ref| over the entries of F and of sigma. */
  double ref_err_E, ref_err_F, ref_err_sigma;
} hfx_stats;

/* Fill *opt with the defaults (all thresholds 1e-10, FP64, both terms,
 * skin 0.5, no freeze, default stream, device 0).  HFX_ERR_INVALID if
 * opt is NULL. */
hfx_status hfx_default_options(hfx_options* opt);

/* Validate the inputs, copy the model and D to the device, build the pair
 * lists (Eqs. 1-2 labels) and lookup tables.  On HFX_OK *out owns a plan
 * that hfx_plan_destroy frees.  All pointers are host pointers. */
hfx_status hfx_plan_create(const hfx_system* sys, const hfx_model* model,
                           const hfx_options* opt, hfx_plan** out);

/* Evaluate E, F^X1 (Eq. Fexx1) and sigma^X1 (Eq. stress) at the given
 * geometry (host pointers).  lattice: 9 doubles (rows); positions:
 * n_atoms*3 doubles.  E: 1 double, F: n_atoms*3 doubles, sigma: 9 doubles,
 * all written only on HFX_OK; stats may be NULL.  The call is synchronous
 * (it returns after the results are on the host). */
hfx_status hfx_energy_force_stress(hfx_plan* plan, const double* lattice, const double* positions,
                                   double* E, double* F, double* sigma, hfx_stats* stats);

/* Same as hfx_energy_force_stress with positions and results in device
 * memory of the plan's device: d_positions [n_atoms*3], d_out
 * [1 + 3*n_atoms + 9] receives E, F, sigma in that order.  lattice is a
 * host pointer.  The call returns after the work is enqueued and the
 * results are complete on the plan's stream. */
hfx_status hfx_energy_force_stress_device(hfx_plan* plan, const double* lattice,
                                          const double* d_positions, double* d_out,
                                          hfx_stats* stats);

/* Evaluation for callers that cannot allocate device memory while they
 * evaluate: hosts whose device memory belongs to their own pool after
 * start-up (an allocation by the library would take memory the pool counts
 * as its own), and real-time loops that forbid allocation after
 * initialisation (cudaMalloc and cudaFree can block for milliseconds and
 * synchronise the device).  hfx_energy_force_stress may grow the plan's
 * per-call block stores with cudaMalloc; this entry point computes the same
 * E, F and sigma (same arguments, host pointers) with that scratch taken from
 * one fixed array inside the library, HFX_NOALLOC_SCRATCH_BYTES = 64 MiB,
 * which every device that loads the library holds until the process exits.
 * It calls no cudaMalloc or cudaFree and no allocation hook of the plan.
 * Like hfx_energy_force_stress it reads the screening counts back to the
 * host in the middle of the call and synchronises the plan's stream, so it
 * cannot be recorded under a stream capture.
 *  - FP64 plans only (HFX_ERR_UNSUPPORTED otherwise).
 *  - A call whose pair lists, Y blocks or V blocks do not fit the array
 *    returns HFX_ERR_UNSUPPORTED with a message; nothing is written.
 *  - Atoms moved beyond skin/2 give HFX_ERR_PAIRLIST_STALE (rebuilding the
 *    lists allocates; call hfx_energy_force_stress once to rebuild them).
 *  - The first call on a device looks up the array's device address, with
 *    that device current, and keeps it for the life of the process; a
 *    cudaDeviceReset (or any teardown of the primary context) invalidates
 *    it, so do not reset a device that has called this entry point.
 *  - Every call on every plan of a device shares the one array, which keeps
 *    the last call's contents (each call writes what it reads before reading
 *    it, so nothing has to start at zero).  Calls that overlap on the GPU
 *    (different streams, threads or plans) race on the array.
 * The paper has no counterpart: this is a deployment variant of the
 * evaluation above. */
#define HFX_NOALLOC_SCRATCH_BYTES (64ull << 20)
hfx_status hfx_energy_force_stress_noalloc(hfx_plan* plan, const double* lattice, const double* positions,
                                           double* E, double* F, double* sigma);

/* Per-stage CUDA-event timing on (1) or off (0, default). */
hfx_status hfx_set_timing(hfx_plan* plan, int on);

/* Reference result for the error report in hfx_stats (for example the FP64
 * result of the same geometry when the plan runs a split precision): E (1
 * double), F (n_atoms*3), sigma (9), host memory, copied.  Every later call
 * that fills hfx_stats reports its relative errors against it.  E = F =
 * sigma = NULL clears it.  HFX_ERR_INVALID for a partial set or non-finite
 * values. */
hfx_status hfx_set_reference(hfx_plan* plan, const double* E, const double* F, const double* sigma);

/* Autotuner.  Times the evaluation of `positions` (host, [n_atoms*3], with
 * `lattice` as in hfx_energy_force_stress) for each launch configuration of
 * the plan that leaves the arithmetic unchanged, and keeps the fastest for
 * the plan's later calls.  Today that is the shape of the tcgen05 first
 * product's Y ring (rows f per slot and number of slots, bounded by shared
 * memory): the shapes of the block pairs decide which run length balances
 * the copy of Y rows against the U build; then, with the best shape, the
 * order in which its items are handed out (longest first, so that the SMs
 * finish together; by home atom, so that items running at the same time
 * share their V_AB and grad V_AB blocks in L2; or by the atom F of the item
 * (A,F), so that they share Y^{BF} blocks); then the 128-row tiles per CTA
 * of the tcgen05 Y build (two tiles share each K step's D blocks; one tile
 * runs more pipeline stages and two accumulators) and the shape of the Q2
 * GEMM (one or two tiles per CTA, or two tiles in one CTA per SM with a
 * deeper copy pipeline and two accumulators per tile), each kept if it is
 * faster.  Each candidate is timed as the
 * median of `reps` >= 1 evaluations (CUDA events) after one warm-up.
 * `report` (nullable) receives the choice and both times.  Plans without a
 * tunable kernel (FP64, or the warp-level first product) return HFX_OK
 * with candidates = 0.  On an error the plan keeps its initial choice. */
typedef struct {
  int candidates;          /* configurations timed, the initial one included */
  int t1_rows_per_slot;    /* chosen rows f per Y slot */
  int t1_slots;            /* chosen number of Y slots */
  double default_ms;       /* median evaluation time with the initial choice */
  double best_ms;          /* median evaluation time with the chosen one */
  int t1_home_order;       /* chosen order of the first product's items: 0 = longest
                              first, 1 = by home atom, 2 = by the atom F of the item (A,F) */
  int y_tiles_per_cta;     /* chosen 128-row tiles per CTA of the tcgen05 Y build (1 or 2) */
  int q2_tiles_per_cta;    /* chosen shape of the tcgen05 Q2 GEMM: 1 or 2 row tiles of 128 per CTA,
                              or 3 = two tiles, one CTA per SM with a deeper copy pipeline */
} hfx_tune_report;
hfx_status hfx_plan_autotune(hfx_plan* plan, const double* lattice, const double* positions, int reps,
                             hfx_tune_report* report);

/* Block preparation: the LRI coefficient fit of Eq. C_VA and its nuclear
 * gradient (Sec. 3.1, the equation after Eq. V_inverse), FP64 on the GPU,
 * for `batch` atom pairs (I, K) of one species pair.  Per pair p, with
 * n = n_abf(I) + n_abf(K) auxiliary functions (those of I first) and
 * w = n_ao(I) n_ao(K) AO pairs (i, k), all row-major and contiguous per pair:
 *   A   [batch][n][n]     two-centre Coulomb metric (V_II, V_IK; V_KI, V_KK),
 *                         symmetric positive definite (only its lower
 *                         triangle is read);
 *   B   [batch][n][w]     three-centre integrals (P_beta | phi_i phi_k);
 *   dA  [batch][3][n][n]  gradient of A in the position of K (c = x, y, z);
 *   dB  [batch][3][n][w]  gradient of B in the position of K.
 * Outputs (caller-allocated):
 *   X   [batch][n][w]     X = A^-1 B: the C^I rows, then the C^K rows;
 *   dX  [batch][3][n][w]  dX[c] = A^-1 (dB[c] - dA[c] X).
 * dA, dB and dX must be all NULL (X only) or all non-NULL.  Pointers are
 * host memory; the call copies them to device `device`, runs one CTA per
 * pair (Cholesky factor in shared memory) on a stream of its own, copies the
 * results back and returns when they are written.  It holds no state and
 * may run beside any plan.
 * Errors: HFX_ERR_INVALID for batch < 0, n < 1, w < 1, a NULL pointer or a
 * mixed NULL set, or a metric that is not positive definite (outputs are
 * then not written); HFX_ERR_UNSUPPORTED if n exceeds what the device's
 * shared memory holds (n <= 160 on GB300); HFX_ERR_OOM / HFX_ERR_CUDA as
 * elsewhere.  hfx_last_error(NULL) gives the message. */
hfx_status hfx_lri_fit(int batch, int n, int w, const double* A, const double* B, const double* dA,
                       const double* dB, double* X, double* dX, int device);

/* Free every resource of the plan.  NULL is accepted. */
hfx_status hfx_plan_destroy(hfx_plan* plan);

/* Static strings; never NULL. */
const char* hfx_status_string(hfx_status s);
const char* hfx_last_error(const hfx_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* HFX_H_ */
