/*
 * paradeisos.h -- C ABI of the GB300 (sm_103a) library for matrix-free exact
 * diagonalisation of the single-band Hubbard model with Paradeisos basis
 * ranking (Jia, Wang, Mendl, Moritz, Devereaux, arXiv 1707.03974).
 *
 * Conventions used by every entry point (Sec. II A and Sec. III of the paper):
 *   - site i of an L-site cluster is bit i of an occupation string;
 *   - a combined basis state is the 64-bit integer (up << L) | dn, the
 *     spin-down string in the L low bits;
 *   - the per-spin position of a string with n particles is its index in the
 *     ascending list of L-bit integers with n bits set (the "forward map",
 *     Eq. 3); the combined index is I = C(L, N_dn) * idx_up + idx_dn;
 *   - a vector over the basis is stored densely in combined-index order, i.e.
 *     as a row-major D_up x D_dn matrix.
 *
 * Memory: every vector, state or index pointer passed in is caller-owned DEVICE
 * memory on the handle's device (in the Python binding: torch tensors).  The
 * library never frees caller memory.  A handle owns only its own small tables
 * (binomial lookup table, per-spin strings and hop lists: O(sqrt D) entries),
 * allocated on the current device at creation.  Calls that take a `stream`
 * enqueue work on that CUDA stream (a cudaStream_t passed as void*, NULL = the
 * legacy default stream) and return without synchronising unless stated.
 * A handle may be used by one stream at a time.
 *
 * Errors: argument errors are returned synchronously.  Per-element problems
 * detected on the device (a string with the wrong popcount, an index >= D)
 * write the sentinel UINT64_MAX to that output element and set a sticky flag
 * on the handle, read (and cleared) by hubbard_last_error().  Device code never
 * traps or asserts.
 */
#ifndef PARADEISOS_H
#define PARADEISOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hb_basis *hb_handle;

typedef enum {
    HB_OK = 0,
    HB_ERR_INVALID_ARG = 1,   /* bad argument (range, duplicate bond, aliasing, null) */
    HB_ERR_OVERFLOW = 2,      /* D would not fit the index type */
    HB_ERR_INVALID_STATE = 3, /* rank: a string with the wrong popcount or bits >= L */
    HB_ERR_OUT_OF_RANGE = 4,  /* unrank: an index >= D */
    HB_ERR_NO_MEMORY = 5,     /* a table or the workspace does not fit */
    HB_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    HB_ERR_NOT_CONVERGED = 7, /* Lanczos hit maxit; best estimate returned */
    HB_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} hb_status;

typedef enum {
    HB_F64 = 0,  /* IEEE binary64 vectors */
    HB_F32 = 1,  /* IEEE binary32 vectors */
    HB_FX64 = 2  /* signed 64-bit fixed point: element q stands for q * 2^-F, F from
                    hubbard_fixed_point_bits(); |value| must stay below 1 on input to
                    H·v.  Sums of hops are exact integer sums, each coefficient class is
                    applied once per element with one rounding (2^-(F+1)); reductions
                    are exact 128-bit integer sums.  Needs at most 4 distinct hopping
                    amplitudes and at most 255 bonds (else HB_ERR_INVALID_ARG). */
} hb_dtype;

/* Human-readable name of a status code (static string). */
const char *hb_status_string(hb_status s);

/*
 * Create the Hubbard problem of Eq. 1 on one cluster and one (N_up, N_dn) sector.
 *   H = - sum_bonds t_b sum_sigma (c+_{i sigma} c_{j sigma} + h.c.) + U sum_i n_{i up} n_{i dn}
 * L       number of sites, 1 <= L <= 32.
 * bonds   host array [n_bonds][2] of site pairs (i, j), 0 <= i, j < L, i != j;
 *         each unordered pair at most once (a duplicate is HB_ERR_INVALID_ARG).
 *         Every bond contributes both hop directions.
 * t       host array [n_bonds] of hopping amplitudes t_b (matrix element -t_b
 *         times the fermion sign of Sec. II B).
 * N_up, N_dn  particle numbers, 0 <= N <= L.  D = C(L,N_up) C(L,N_dn) must be < 2^63.
 * out     receives the handle.  Tables are built on the current CUDA device,
 *         synchronously.  The per-spin hop lists are built lazily on first use
 *         of hubbard_apply / hubbard_row_entries / lanczos_ground_state.
 */
hb_status hubbard_basis_create(int L, int n_bonds, const int32_t *bonds, const double *t, double U,
                               int N_up, int N_dn, hb_handle *out);

/*
 * Create the Hubbard problem in one momentum sector (Sec. IV A, Eq. 4):
 *   H = sum_{k sigma} eps_k n_{k sigma} + (U/N) sum_{k,k',q} c+_{k+q up} c+_{k'-q dn} c_{k' dn} c_{k up}
 * on an Lx x Ly periodic cluster (Ly = 1: a ring of Lx sites), N = Lx Ly, 2 <= N <= 32,
 * eps_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky (-2t cos k on a ring).
 * Bit i of a spin string is the occupation of momentum k_i = 2 pi (mx/Lx, my/Ly),
 * i = mx + Lx my; states passed to paradeisos_rank / paradeisos_unrank are
 * (up << N) | dn over these bits.  The sector has total momentum
 * K = 2 pi (Kx/Lx, Ky/Ly), 0 <= Kx < Lx, 0 <= Ky < Ly; its states are indexed by the
 * spin-full maps of Sec. IV A with the tables C_i^m(k) and C~_i^m(k; N_dn) (Eq. 6),
 * i.e. in ascending order of (up << N) | dn.  An empty sector is HB_ERR_INVALID_ARG.
 * The handle works with hubbard_basis_dim (D = sector dimension), paradeisos_rank /
 * unrank, hubbard_apply (HB_F64, HB_F32, HB_FX64), hubbard_row_entries,
 * hubbard_set_U, hubbard_autotune (one launch shape: it only times it),
 * lanczos_step(_noalloc) and lanczos_ground_state; not with the batch or MLP calls.
 * All tables (moves of every spin string for every q) are built here, synchronously.
 */
hb_status hubbard_basis_create_k(int Lx, int Ly, double t, double tp, double U, int N_up, int N_dn, int Kx, int Ky,
                                 hb_handle *out);
hb_status hubbard_basis_destroy(hb_handle h);
/* D, D_up = C(L,N_up), D_dn = C(L,N_dn); any pointer may be NULL. */
hb_status hubbard_basis_dim(hb_handle h, uint64_t *D, uint64_t *D_up, uint64_t *D_dn);
/* Change U (the interaction of Eq. 1) without rebuilding any table. */
hb_status hubbard_set_U(hb_handle h, double U);
/* Number of fractional bits F of the HB_FX64 format of this handle, chosen at
 * creation so that 3 * max_r sum_c |H_rc| * 2^F < 2^62 (Lanczos vectors of norm
 * <= 1 and their images under H fit without overflow). */
hb_status hubbard_fixed_point_bits(hb_handle h, int32_t *F);
/* Element-wise conversion between HB_F64 and HB_FX64 vectors of length n
 * (round to nearest; the float64 values must satisfy |x| * 2^F < 2^62). */
hb_status hubbard_convert(hb_handle h, hb_dtype from, const void *x, hb_dtype to, void *y, uint64_t n, void *stream);

/*
 * Paradeisos forward map, batched (Eq. 3 and the combined index of Sec. III).
 * states  device [n] combined strings (up << L) | dn
 * idx     device [n] output combined indices; UINT64_MAX (and the sticky flag
 *         HB_ERR_INVALID_STATE) for a string whose popcounts differ from
 *         (N_up, N_dn) or that has bits at or above L in either half.
 */
hb_status paradeisos_rank(hb_handle h, const uint64_t *states, uint64_t *idx, uint64_t n, void *stream);

/*
 * Paradeisos backward map, batched (the backward-map procedure of Sec. III).
 * idx     device [n] combined indices
 * states  device [n] output strings (up << L) | dn; UINT64_MAX (and the sticky
 *         flag HB_ERR_OUT_OF_RANGE) for an index >= D.
 */
hb_status paradeisos_unrank(hb_handle h, const uint64_t *idx, uint64_t *states, uint64_t n, void *stream);

/*
 * y = H x, matrix-free (Eq. 1): diagonal U * popcount(up & dn) (Sec. II B) plus
 * every hop of both spins, each target located by the forward map.
 * dt      HB_F64, HB_F32 or HB_FX64 (fixed point, see hubbard_fixed_point_bits):
 *         element type of x and y (length D each).
 * x, y    device vectors; must not overlap (HB_ERR_INVALID_ARG).
 * Every launch configuration (hb_hv_config) gives bit-identical results for
 * HB_F64 and HB_FX64.  For HB_F32 the one-kernel configurations agree bit for
 * bit, and so do the split ones (hb_hv_config.split = 1).  The split float32
 * row pass sums the spin-down hops per (amplitude class, sign) and then scales
 * each sum by -t, so it agrees with the one-kernel form to float32 rounding.
 */
hb_status hubbard_apply(hb_handle h, hb_dtype dt, const void *x, void *y, void *stream);

/*
 * hubbard_apply with a timing hook: records ev_begin, then the row pass
 * (diagonal + spin-down hops) of the split form, ev_mid, the spin-up pass,
 * ev_end, all on `stream` (cudaEvent_t passed as void*).  In the one-kernel
 * form (and for momentum-sector handles) ev_mid and ev_end both follow the one
 * kernel.  Same arguments, results and errors as hubbard_apply otherwise.
 */
hb_status hubbard_apply_timed(hb_handle h, hb_dtype dt, const void *x, void *y, void *ev_begin, void *ev_mid,
                              void *ev_end, void *stream);

/* Launch configuration of the H·v kernel for one vector type (zeros = library default). */
typedef struct {
    int32_t rows_per_cta;     /* rows of x staged together in shared memory: 1, 2 or 4 (0 = widest that fits) */
    int32_t threads_per_cta;  /* multiple of 32, <= 1024 (0 = 1024) */
    int32_t visit_order;      /* 1: rows in reverse Cuthill-McKee order of the spin-up hop graph (default);
                                 0: storage order.  Only the visiting order changes, never the layout. */
    float ms;                 /* hubbard_autotune: time per H·v of the chosen configuration */
    int32_t split;            /* 0: one kernel for all terms; 1: a row pass (diagonal + spin-down hops, the
                                 fields above) then a spin-up pass over column blocks of x, so the blocks
                                 in flight stay in L2 (the fields below).  For HB_FX64 and HB_F32 the row
                                 pass reads the handle's warp-blocked spin-down table when it has one (at
                                 most 4 distinct hopping amplitudes, at most 255 bonds, D_dn + 8 <= 65535):
                                 HB_FX64 stages 1 or 2 rows, HB_F32 1, 2 or 4 */
    int32_t up_block;         /* split: columns per block, multiple of 32, <= up_threads (0 = 256) */
    int32_t up_threads;       /* split: threads per CTA, a multiple of up_block, <= 1024 (0 = 1024) */
    int32_t up_rows;          /* split: rows per thread, 1, 2 or 4 (0 = 1) */
} hb_hv_config;

hb_status hubbard_get_hv_config(hb_handle h, hb_dtype dt, hb_hv_config *cfg);
/* HB_ERR_INVALID_ARG for out-of-range fields; a row count that does not fit
 * shared memory falls back to the widest that does. */
hb_status hubbard_set_hv_config(hb_handle h, hb_dtype dt, const hb_hv_config *cfg);
/* Autotuner: times every candidate configuration (rows 1/2/4, threads
 * 256/512/1024, both visiting orders, one kernel or split; for the split form
 * the row pass and the spin-up pass (blocks 128/256/512, threads 512/1024,
 * rows 1/2/4) are tuned one after the other) as reps applications to the
 * caller's x (into y, which is overwritten and left unspecified), keeps the
 * fastest in the handle and returns it in *best (may be NULL).  Synchronises
 * `stream`. */
hb_status hubbard_autotune(hb_handle h, hb_dtype dt, const void *x, void *y, int32_t reps, hb_hv_config *best,
                           void *stream);

/*
 * Verification export of matrix rows row0 .. row0+nrows-1 in canonical form:
 * entries sorted by column, the diagonal included even when it is zero.
 * cols, vals  device [nrows][max_entries]; counts device [nrows].
 * A row with more than max_entries entries sets counts[r] = UINT32_MAX and
 * the sticky flag HB_ERR_INVALID_ARG.  (1 + 2 * n_bonds always suffices.)
 */
hb_status hubbard_row_entries(hb_handle h, uint64_t row0, uint32_t nrows, uint32_t max_entries,
                              uint64_t *cols, double *vals, uint32_t *counts, void *stream);

/* Sticky device-side error of the handle: synchronises the device, returns
 * HB_OK or the first per-element error recorded since the last call, and clears it. */
hb_status hubbard_last_error(hb_handle h);

/* ---------------- Lanczos ground state (the solver the paper cites in Sec. I) ---- */

typedef struct {
    int32_t maxit;        /* maximum Lanczos steps (>= 1) */
    int32_t reorth;       /* 0: three-term recurrence; 1: full reorthogonalisation
                             (classical Gram-Schmidt twice against all stored vectors) */
    int32_t vec_dtype;    /* hb_dtype of the Krylov vectors */
    int32_t check_every;  /* Ritz check every k steps (>= 1) */
    double tol;           /* stop when beta_j |s_last| <= tol * max(1, |theta|); <= 0: run maxit */
    uint64_t seed;        /* start vector when v0 == NULL: SplitMix64, element i = output i+1
                             of the stream seeded with `seed`, mapped to [-1, 1), normalised */
    int32_t fp64_finish;  /* with vec_dtype HB_F32: after the binary32 phase reaches its own
                             tolerance, form the Ritz vector and continue until tol is met,
                             in binary64 vectors (1) or HB_FX64 vectors (2) */
    int32_t f32_tol_exp;  /* binary32 phase ends when the residual <= 10^f32_tol_exp * max(1,|theta|)
                             or stops improving (default -5 when 0) */
    int32_t store_basis;  /* with vec_dtype HB_F32 and fp64_finish: K > 0 keeps the binary32 Krylov
                             vectors v_0 .. v_K in the workspace (K + 1 vectors of 4 D bytes), caps the
                             binary32 phase at K steps and forms its Ritz vector in one pass over them
                             instead of replaying the recurrence; 0: replay (three vectors) */
} hb_lanczos_opts;

typedef struct {
    double E0;                 /* lowest Ritz value */
    double residual;           /* beta_j |s_last| of the lowest Ritz pair */
    int32_t iterations;        /* total Lanczos steps (all phases) */
    int32_t iterations_f32;    /* steps taken in the binary32 phase */
    int32_t status;            /* hb_status of the solve */
    int32_t converged;         /* 1 if the tolerance was met */
    double seconds;            /* host wall time of the call */
} hb_lanczos_info;

/* Bytes of device workspace lanczos_ground_state needs for these options. */
hb_status lanczos_workspace_bytes(hb_handle h, const hb_lanczos_opts *opts, uint64_t *bytes);

/*
 * Lowest eigenvalue of H by Lanczos.  v0: device start vector of vec_dtype
 * (length D, need not be normalised) or NULL for the seeded random start.
 * workspace: caller-owned device buffer of at least lanczos_workspace_bytes.
 * alphas, betas: optional HOST arrays [maxit] receiving the recurrence
 * coefficients of the last phase (may be NULL).  Synchronises `stream`; returns
 * HB_ERR_NOT_CONVERGED (with E0 filled) if maxit is reached first.
 */
hb_status lanczos_ground_state(hb_handle h, const hb_lanczos_opts *opts, const void *v0,
                               void *workspace, uint64_t workspace_bytes,
                               double *alphas, double *betas, double *E0, hb_lanczos_info *info,
                               void *stream);

/* Bytes of device scratch (per-block partial sums of the reductions: three
 * 16-byte sums per block) lanczos_step needs. */
hb_status lanczos_step_scratch_bytes(hb_handle h, uint64_t *bytes);

/*
 * One step of the three-term Lanczos recurrence (the building block of
 * lanczos_ground_state, exposed for drivers that keep their own loop):
 *   w = H v - beta_prev * vprev;  alpha = <w, v>;  w -= alpha * v;  beta = ||w||;  w /= beta,
 * after which w holds the next Lanczos vector.  HB_FX64 and HB_F32 take two
 * vector passes: the first forms w with the sums <w,v>, <w,w>, <v,v> (exact
 * 128-bit integers, or float32 pairs with exact products), from which
 * beta^2 = <w,w> - 2 alpha <w,v> + alpha^2 <v,v> is evaluated (double-double /
 * float64 arithmetic); the second writes (w - alpha v) / beta.  HB_F64 keeps the
 * textbook three passes.
 * dt            element type of v, vprev, w (device vectors of length D; w must not
 *               overlap v or vprev).
 * vprev, beta_prev  previous vector and device scalar; both NULL on the first step.
 * alpha, beta   device doubles written by the step (float64 reductions as in
 *               lanczos_ground_state).
 * scratch       caller-owned device buffer of lanczos_step_scratch_bytes bytes.
 * ev_hv_begin, ev_hv_end  optional cudaEvent_t (as void*) recorded on `stream`
 *               just before and just after the H·v kernel (a timing hook; NULL to skip).
 * launches      optional host counter, incremented by the number of kernels enqueued
 *               (H·v: 1, or 2 in the split form; then 3, or 5 for HB_F64).
 * Asynchronous on `stream`.
 */
hb_status lanczos_step(hb_handle h, hb_dtype dt, const void *v, const void *vprev, void *w, const double *beta_prev,
                       double *alpha, double *beta, void *scratch, uint64_t scratch_bytes, void *ev_hv_begin,
                       void *ev_hv_end, uint32_t *launches, void *stream);

/*
 * lanczos_step without any allocation (the paper has no counterpart; this is a
 * deployment convenience).  Some callers cannot call cudaMalloc at the point
 * where they step the solver: a host program that hands out all device memory
 * through its own pool and forbids libraries from allocating behind its back,
 * a plug-in that runs inside another framework's memory budget, or a loop that
 * must not risk an allocation's latency or failure mid-run.  For them this
 * entry point takes the same arguments as lanczos_step minus the scratch
 * buffer: the reductions' partial sums live in a fixed device array inside the
 * library, 2048 doubles (16 KiB), which every GPU that loads the library holds
 * until the process exits.
 *   - The caller still owns and passes v, vprev, w and the scalars.
 *   - dt is HB_F64 or HB_F32.  HB_FX64 is refused with HB_ERR_INVALID_ARG: the
 *     fixed-point step keeps three 128-bit partial sums per reduction block
 *     (six doubles), which on a 152-SM GB300 is more than the array holds.
 *   - The handle's per-spin tables must already exist (any earlier
 *     hubbard_apply, hubbard_row_entries, lanczos_step or lanczos_ground_state
 *     on the handle builds them); otherwise HB_ERR_INVALID_STATE, because
 *     building them would allocate.  Momentum-sector handles build theirs at
 *     creation.
 *   - Call it with the handle's device current (else HB_ERR_INVALID_ARG,
 *     returned before anything is enqueued).
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current, so a device reset between calls leaves no
 *     stale address behind.  With CUDA's lazy module loading the first call on
 *     a device may make the driver load the library's device code, and that
 *     load can allocate; make the first call before any stream capture begins
 *     and before a strict memory budget takes effect.
 *   - A device whose reductions need more than 2048 partial sums (three per
 *     reduction block, four blocks per SM: more than 170 SMs) is rejected
 *     with HB_ERR_NO_MEMORY.
 *   - All calls on a device share the array, which keeps the last call's
 *     contents (nothing in it needs to start at zero: every slot is written
 *     before it is read).  Calls whose kernels overlap on the GPU race on it:
 *     serialise them (one stream, or events).
 * After the first call on a device, neither this call nor anything it calls
 * allocates or frees device memory.
 */
hb_status lanczos_step_noalloc(hb_handle h, hb_dtype dt, const void *v, const void *vprev, void *w,
                               const double *beta_prev, double *alpha, double *beta, void *ev_hv_begin,
                               void *ev_hv_end, uint32_t *launches, void *stream);

/*
 * float32 Lanczos (float64 scalars) to opts->tol, then the normalised Ritz
 * vector of E0, written to ritz (device float[D]) by replaying the recurrence
 * from the stored start vector with the recorded alpha, beta.  Workspace as
 * lanczos_workspace_bytes for vec_dtype HB_F32 with fp64_finish = 1.  Used to
 * produce training targets for the start-vector network.  Synchronises.
 */
hb_status lanczos_ritz_vector_f32(hb_handle h, const hb_lanczos_opts *opts, const void *v0, void *workspace,
                                  uint64_t workspace_bytes, float *ritz, double *E0, hb_lanczos_info *info,
                                  void *stream);

/* ---------------- batches of independent problems ---------------- */
/*
 * A batch groups handles (different clusters, sectors, U) that are applied and
 * solved together: their vectors are concatenated, instance k occupying
 * elements [offsets[k], offsets[k] + D_k) of a batch vector of offsets[n]
 * elements (offsets are multiples of 64 elements).  The handles must outlive
 * the batch and stay on one device; a batch is not a copy of their tables.
 * (Not in the paper: a throughput arrangement for many small problems.)
 */
typedef struct hb_batch *hb_batch_handle;
hb_status hubbard_batch_create(int n, const hb_handle *handles, hb_batch_handle *out);
hb_status hubbard_batch_destroy(hb_batch_handle b);
hb_status hubbard_batch_layout(hb_batch_handle b, uint64_t *offsets /* [n+1] */);
/* y = H_k x for every instance k in one launch (row groups of all instances
 * form one work list); dt HB_F64, HB_F32 or HB_FX64. */
hb_status hubbard_batch_apply(hb_batch_handle b, hb_dtype dt, const void *x, void *y, void *stream);
/* Launch configuration of the batched H·v (the fields of hb_hv_config):
 *   one kernel (split 0): rows_per_cta 1, 2 or 4 per item, threads_per_cta <= 512;
 *   split form (split 1, fixed point only, every instance with a warp-blocked
 *   table): a row pass (diagonal + spin-down hops, rows_per_cta 1 or 2) over all
 *   instances, then the spin-up pass over column blocks (up_block columns,
 *   up_threads <= 512 threads, up_rows rows per thread) of all instances.
 * HB_ERR_INVALID_ARG for out-of-range fields or a split the batch cannot take. */
hb_status hubbard_batch_get_config(hb_batch_handle b, hb_hv_config *cfg);
hb_status hubbard_batch_set_config(hb_batch_handle b, const hb_hv_config *cfg);
/* Autotuner of the batched H·v: the one-kernel form (rows per group 1/2/4,
 * threads 128/256/512) and, for fixed point, the split form (row pass rows 1/2,
 * threads 256/512, then seven spin-up shapes); keeps the fastest in the batch.
 * x and y are batch vectors (y overwritten). */
hb_status hubbard_batch_autotune(hb_batch_handle b, hb_dtype dt, const void *x, void *y, int32_t reps,
                                 hb_hv_config *best, void *stream);
hb_status lanczos_batch_workspace_bytes(hb_batch_handle b, const hb_lanczos_opts *opts, uint64_t *bytes);
/*
 * Lowest eigenvalue of every instance by the three-term Lanczos recurrence
 * (vec_dtype HB_F64 or HB_FX64; reorth and fp64_finish are not supported).
 * Instance k starts from the SplitMix64 vector of seed opts->seed + k.
 * All steps of all instances run in one persistent cooperative kernel: per
 * step, the H·v of every row group of every active instance fused with
 * w = H v - beta vprev and the step's reductions, a grid barrier, then alpha
 * and beta of every instance (fixed point: from exact 128-bit sums in
 * double-double) and the vector update, and another barrier (float64 takes a
 * third phase for its second reduction).  Every check_every steps the CTA
 * holding an instance's first element solves its tridiagonal on the device
 * (Sturm multisection, inverse iteration) and masks it once
 * beta_j |s_last| <= tol max(1, |theta|).  One launch runs up to 64 steps and
 * is replayed from a captured CUDA graph until all instances have converged
 * or maxit is reached; the final E0 and residuals come from the recorded
 * coefficients through hb_tridiag_lowest.  Every grid barrier's wait gives up
 * after 5 s (global timer, with a poll cap); the call then returns
 * HB_ERR_TIMEOUT and the context stays usable.  A device without cooperative
 * launch support gives HB_ERR_CUDA.
 * E0, info: HOST arrays [n].  Synchronises `stream`.
 */
hb_status lanczos_batch_ground_state(hb_batch_handle b, const hb_lanczos_opts *opts, void *workspace,
                                     uint64_t workspace_bytes, double *E0, hb_lanczos_info *info, void *stream);

/*
 * Self-test of the bounded waits of lanczos_batch_ground_state: runs its first
 * step with CTA withhold_cta leaving the kernel before its first arrival at a
 * grid barrier, and a wait limit of limit_ms (1 .. 10000).  The other CTAs'
 * waits give up, so the expected result is HB_ERR_TIMEOUT, after which the
 * batch and the device remain usable.  Same workspace as
 * lanczos_batch_ground_state.  Synchronises `stream`.
 */
hb_status lanczos_batch_wait_selftest(hb_batch_handle b, const hb_lanczos_opts *opts, void *workspace,
                                      uint64_t workspace_bytes, int32_t withhold_cta, uint32_t limit_ms,
                                      void *stream);

/* ---------------- dynamical response (the continued fraction named in Sec. I) ---------------- */

/*
 * float64 Lanczos (three-term recurrence) to opts->tol, then the normalised
 * float64 Ritz vector of E0 in ritz (device double[D]), rebuilt by replaying the
 * recurrence from a stored copy of the start vector with the recorded alpha,
 * beta.  Workspace: lanczos_workspace_bytes for vec_dtype HB_F64 (reorth 0)
 * plus 8 D bytes rounded up to a multiple of 256.  Synchronises `stream`.
 */
hb_status lanczos_ritz_vector_f64(hb_handle h, const hb_lanczos_opts *opts, const void *v0, void *workspace,
                                  uint64_t workspace_bytes, double *ritz, double *E0, hb_lanczos_info *info,
                                  void *stream);

/*
 * y = c_{k s} x (op 0) or y = c+_{k s} x (op 1) between two momentum-sector
 * handles of the same cluster (hubbard_basis_create_k): dst must be the sector
 * with one particle of spin s (0 up, 1 down) fewer (more) and total momentum
 * K - k_k (K + k_k).  Sign convention: the many-body state is the up creators in
 * descending momentum index followed by the down creators, so the operator
 * carries (-1)^(particles of spin s above bit k), times (-1)^(N_up) for s = down.
 * x: device vector of the source sector, y of the target (dt HB_F64 or HB_F32).
 * norm2: optional device double receiving ||y||^2.  Asynchronous on `stream`.
 */
hb_status hubbard_apply_c(hb_handle src, hb_handle dst, int op, int spin, int k, hb_dtype dt, const void *x, void *y,
                          double *norm2, void *stream);

/*
 * Host utility: the Lanczos continued fraction
 *   G(z) = norm2 / (z + E0 - alpha_0 - beta_0^2 / (z + E0 - alpha_1 - ... - beta_{n-2}^2 / (z + E0 - alpha_{n-1})))
 * at nz complex points z = z_re + i z_im (alpha[n], beta[n-1] from a Lanczos run
 * started at phi / ||phi||, norm2 = ||phi||^2).
 */
hb_status hb_continued_fraction(const double *alpha, const double *beta, int n, double norm2, double E0,
                                const double *z_re, const double *z_im, int nz, double *g_re, double *g_im);

/* ---------------- inversion-symmetric maps (Sec. IV B) ---------------- */

/*
 * Index maps of the inversion-symmetric subspace of n particles on an N-site
 * chain (F maps site i to N-1-i): one basis element per orbit {phi, F(phi)},
 * ordered by the classification tree of Sec. IV B (outermost unclassified bit
 * pair (N-1-d, d): class A (0,1) is a leaf ranked by the forward map of Eq. 3 on
 * its inner bits, class B (0,0) and class C (1,1) recurse; A before B before C;
 * subtree sizes S_i^m = C_{i-2}^{m-1} + S_{i-2}^m + S_{i-2}^{m-2}).
 * 1 <= N <= 32, 0 <= n <= N.  The handle owns two small tables on the current device.
 */
typedef struct hb_inv *hb_inv_handle;
hb_status paradeisos_inv_create(int N, int n, hb_inv_handle *out);
hb_status paradeisos_inv_destroy(hb_inv_handle h);
/* D = number of orbits = (C(N,n) + number of palindromes) / 2 */
hb_status paradeisos_inv_dim(hb_inv_handle h, uint64_t *D);
/* Orbit index of each string (either member of an orbit gives the same index).
 * A string with bits >= N or a popcount != n gives UINT64_MAX and the sticky
 * HB_ERR_INVALID_STATE.  states, idx: device [n_items]; asynchronous on stream. */
hb_status paradeisos_inv_rank(hb_inv_handle h, const uint64_t *states, uint64_t *idx, uint64_t n_items, void *stream);
/* Representative of each index (the member whose first unequal outer pair reads (0,1),
 * or the palindrome); an index >= D gives UINT64_MAX and HB_ERR_OUT_OF_RANGE. */
hb_status paradeisos_inv_unrank(hb_inv_handle h, const uint64_t *idx, uint64_t *states, uint64_t n_items, void *stream);
/* Sticky error of the handle (synchronises the device, returns and clears it). */
hb_status paradeisos_inv_last_error(hb_inv_handle h);

/* ---------------- measured ceilings of the device (measurement support) ---------------- */

/*
 * The H·v of Eq. 1 reads 16 bytes per basis state from HBM but z hop operands
 * per state through the SM's load path, so its rooflines include on-chip
 * rates.  hb_measure_ceilings runs one small probe kernel per unit flat out
 * on the current device and reports what it sustains (best of three launches,
 * CUDA events).  Rates count useful work: flops (an FMA is 2), integer adds,
 * or bytes delivered to registers.
 */
typedef struct {
    int32_t sm_count;
    double sm_clock_mhz;       /* SM cycles per global-timer nanosecond during the float32 probe */
    double fp64_fma_tflops;    /* float64 FMA */
    double fp32_fma_tflops;    /* float32 FMA */
    double int32_add_tops;     /* 32-bit integer adds (10^12 per second) */
    double int64_add_tops;     /* 64-bit integer adds (the fixed-point hop sums) */
    double smem_seq16_gbs;     /* shared memory, conflict-free 16-byte loads (a warp reads 512 contiguous bytes) */
    double smem_gather8_gbs;   /* shared memory, 8-byte loads at uniformly random addresses */
    double smem_gather16_gbs;  /* shared memory, 16-byte loads at uniformly random addresses */
    double smem_gather8_clk;   /* SM cycles per warp-wide random 8-byte gather (about its wavefronts) */
    double smem_gather16_clk;  /* SM cycles per warp-wide random 16-byte gather */
    double l1_gbs;             /* coalesced 16-byte global loads hitting L1 (16 KiB window per CTA) */
    double l2_gbs;             /* coalesced 16-byte global loads served by L2 (window of l2_window_bytes) */
    double hbm_read_gbs;       /* one streaming read pass over the buffer (0 if it is under 1 GiB) */
    uint64_t l2_window_bytes, hbm_window_bytes;
} hb_ceilings;

/* buffer: caller-owned device memory of buffer_bytes >= 64 MiB, 16-byte aligned,
 * overwritten (>= 1 GiB adds the HBM read probe).  Synchronises `stream`; takes
 * well under a second. */
hb_status hb_measure_ceilings(void *buffer, uint64_t buffer_bytes, hb_ceilings *out, void *stream);

/* ---------------- pinned host buffers (host <-> device copies) ---------------- */

/*
 * Page-locked host memory for the vectors a caller streams to and from the
 * device (the end-to-end path of the Lanczos step copies v in every step).
 * The buffer is an anonymous mapping of `bytes` rounded up to 2 MiB, advised
 * for transparent huge pages, placed (as a preference, before the first touch)
 * on the host NUMA node nearest the current device when the driver reports one
 * (cudaDevAttrHostNumaId), zero-filled, and registered with the CUDA driver
 * (cudaHostRegister), so copies run at the link's full rate whichever pages the
 * host chose.  *ptr is aligned to the host's transparent huge page size (at
 * least 2 MiB).  Owned by the caller: release it with
 * hb_host_free.  Errors: HB_ERR_INVALID_ARG (bytes == 0 or ptr null),
 * HB_ERR_NO_MEMORY (the mapping failed), HB_ERR_CUDA (registration failed;
 * nothing is left allocated).  Needs a CUDA device for the registration.
 */
hb_status hb_host_alloc(uint64_t bytes, void **ptr);
/* Unregisters and unmaps a buffer from hb_host_alloc (null: no-op).
 * HB_ERR_INVALID_ARG for any other pointer. */
hb_status hb_host_free(void *ptr);

/*
 * Host utility (no GPU needed): lowest eigenvalue theta of the symmetric
 * tridiagonal matrix with diagonal alpha[0..n) and off-diagonal beta[0..n-1),
 * by Sturm-sequence bisection, and the last component of its normalised
 * eigenvector by inverse iteration (the Ritz residual of Lanczos step n-1 is
 * beta[n-1] * |s_last|).  Used by lanczos_ground_state after every check.
 */
hb_status hb_tridiag_lowest(const double *alpha, const double *beta, int n, double *theta, double *s_last);

#ifdef __cplusplus
}
#endif
#endif /* PARADEISOS_H */
