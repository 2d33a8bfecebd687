/*
 * ttsn.h -- C ABI of libttsn, a GB300 (sm_103a) implementation of the
 * tensor-train discrete-ordinates (TT-S_N) step-then-truncate time step for
 * gray thermal radiation transport of arXiv 2503.18056 ("Thermal radiation
 * transport with tensor trains").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev are CUDA device pointers on the current device;
 *   pointers named *_host are host pointers.  No entry point takes ownership
 *   of a caller pointer: inputs are copied in, outputs are written into
 *   caller-allocated buffers.
 * - Every call is ordered on the CUDA stream given at creation (or passed to
 *   the kernel-level calls).  Calls that return host data (ranks, totals,
 *   step info, sweep counts) synchronise that stream before returning.
 * - Nothing throws across the ABI.  Each call returns a tt_status; on an error
 *   tt_last_error() returns a thread-local message describing it.  Device-side
 *   failures (eigensolver sweep limit, a bounded wait that ran out) are latched
 *   in a device status word and reported by the next call that synchronises.
 * - Floating-point data are IEEE binary64 ("double").  All arrays are
 *   row-major (C order).  A TT core k has shape (r_{k-1}, n_k, r_k) with
 *   r_0 = r_d = 1 and is stored contiguously with r_k fastest.
 */
#ifndef TTSN_H
#define TTSN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_MAX_D 8
#define TT_MAX_SOURCES 16

typedef struct tt_ctx* tt_handle;

typedef enum {
    TT_OK = 0,
    TT_WARN_RANK_CAPPED = 1,   /* a rank cap bound: the eps guarantee is void   */
    TT_ERR_ARG = -1,           /* invalid argument (message says which)         */
    TT_ERR_OOM = -2,           /* device allocation failed                      */
    TT_ERR_CUDA = -3,          /* a CUDA runtime call failed                    */
    TT_ERR_NOT_CONVERGED = -4, /* Jacobi eigensolver hit its sweep limit        */
    TT_ERR_TIMEOUT = -5,       /* a bounded device-side wait ran out            */
    TT_ERR_STATE = -6,         /* call not valid for this handle                */
    TT_ERR_TOO_LARGE = -7,     /* output buffer too small / size over a limit   */
    TT_ERR_NONFINITE = -8      /* a rounding met Inf/NaN (the run diverged, or a
                                  field held one); the TT is then undefined and
                                  the caller restores saved cores and T      */
} tt_status;

enum { TT_BC_PERIODIC = 0, TT_BC_VACUUM = 1, TT_BC_OUTFLOW = 2 };
enum { TT_FP64 = 0, TT_MIXED = 1 };
enum { TT_LAYOUT_GROUPED = 0, TT_LAYOUT_SPLIT = 1 };
enum { TT_FLUX_UPWIND = 0, TT_FLUX_RUSANOV = 1, TT_FLUX_HLL = 2, TT_FLUX_RUSANOV_TAU = 3 };
enum { TT_ROUND_GRAM = 0, TT_ROUND_RANDOMIZED = 1, TT_ROUND_TTSVD = 2 };
enum { TT_EIG_ONE_SIDED = 0, TT_EIG_TWO_SIDED = 1 };

/* step flags for tt_sn_step_ex */
enum {
    TT_STEP_NO_SOURCE = 1, /* transport only (no absorption/emission stage)   */
    TT_STEP_NO_ROUND = 2   /* keep the rank-grown TT (untruncated step)       */
};

/*
 * Problem description for tt_create (Sec. 2-3 of the paper).
 *
 * Grid: ndim in {1,2,3} axes with n[a] cells over [0, L[a]], cell-centred;
 * cells are numbered in C order of the (n[0], n[1], n[2]) array (axis 0
 * slowest), N_c = prod n[a].  Ordinates: the latitude-longitude grid of Sec. 3,
 * n_theta cells uniform in mu = cos(theta) on [-1, 1] and n_phi cells uniform
 * in phi on [0, 2 pi), ordinates at cell centres, dOmega = 4 pi/(n_theta n_phi).
 * Constants: speed of light c, radiation constant a_r.  Time step: dt if > 0,
 * otherwise cfl * min(L[a]/n[a]) / c (Sec. 3.1).  bc[a]: TT_BC_PERIODIC,
 * TT_BC_VACUUM (zero incoming intensity: zero ghost cells) or TT_BC_OUTFLOW
 * (ghost cells copy the boundary cell, a zero-gradient face), the same on
 * both faces of axis a (Sec. 4.5).
 * Fields (device pointers, N_c doubles each, copied in at creation):
 *   sigma_a = rho kappa_a, sigma_s = rho kappa_s (NULL = 0), cv = rho c_v,
 *   T0 = initial material temperature, Tr0 = initial radiation temperature
 *   (the intensity starts isotropic, I = c a_r Tr0^4 / 4 pi; NULL = T0).
 * Rounding (Sec. 4.2, App. A): relative Frobenius tolerance eps balanced over
 * the bonds, ranks capped at max_rank (<= 0: no cap); rounds_per_step = 1
 * rounds once after the source stage, 2 also rounds after transport.
 * precision: TT_FP64, or TT_MIXED for the precision form: the Gram sweeps
 * (left Grams, and the right-Gram products of all but the last core) and the
 * core updates A' = A P_A (the dominant contractions of App. A.4) run on the
 * BF16 tensor cores with exact split products (tt_gram_mixed,
 * tt_gemm_nt_mixed: about 2^-48 of the operands' scales per term);
 * eigensolves, rank decisions, the small R x R products, the quartic and the
 * temperature update stay FP64.
 * layout: TT_LAYOUT_GROUPED holds the intensity in the paper's three-core
 * layout (Eq. tensor_decomp, all spatial axes in one core so that arbitrary
 * material fields cost nothing): X (1, N_c, r1), Theta (r1, n_theta, r2),
 * Phi (r2, n_phi, 1).  TT_LAYOUT_SPLIT holds one core per spatial axis, then
 * Theta and Phi (the split-space alternative of Sec. 4.1 / Sec. 7; d = ndim +
 * 2 cores, core a of shape (r_a, n[a], r_{a+1})).  In the split layout every
 * transport term is a TT with D^-/+ on one spatial core, the emission field e
 * enters as one more TT term holding e exactly (ranks N_x[, N_z] at the
 * spatial bonds before rounding), and the initial intensity is held the same
 * way and rounded to eps at creation.  It needs uniform sigma_a and sigma_s
 * (TT_ERR_ARG otherwise: a varying absorption factor would multiply every
 * spatial rank) and takes neither fixed sources nor the adjoint tape
 * (TT_ERR_STATE).
 * flux: the interface flux of Sec. 3.1 with piecewise-constant states.
 * TT_FLUX_UPWIND (Eq. upwind; flux_param unused); TT_FLUX_RUSANOV (Eq.
 * rusanov_flux_toro with S+ = flux_param[0] * c, 0 <= flux_param[0]: 1 is
 * the paper's optically thin choice, 0 the central difference);
 * TT_FLUX_HLL (Eq. hll with the wave speeds that follow it and the optical
 * depth of Eq. tauc: flux_param[0] = beta > 0, flux_param[1] =
 * tau_threshold in (0, sqrt 2]; a vacuum face takes the boundary cell's own
 * opacity for Eq. tauc); TT_FLUX_RUSANOV_TAU (Eq. rusanov_flux_toro with the
 * speed informed by each face's optical depth, Sec. 3.1: S+ = c |n_a|
 * min(1, 1 / tau_c), tau_c from Eq. tauc with flux_param[0] = beta > 0; the
 * thick-limit speed c |n_a| / tau_c of the expansion after Eq. hll on thick
 * faces, upwinding on faces with tau_c <= 1).  Every flux adds 1 + 2 ndim
 * terms to the TT sum, so the ranks grow as with upwinding.  The adjoint tape
 * takes upwinding only.
 */
typedef struct {
    int ndim;
    int n[3];
    double L[3];
    int n_theta, n_phi;
    double c, a_r, cfl, dt;
    int bc[3];
    const double* sigma_a;
    const double* sigma_s;
    const double* cv;
    const double* T0;
    const double* Tr0;
    double eps;
    int max_rank;
    int rounds_per_step;
    int precision;
    int layout;
    int flux;
    double flux_param[2];
} tt_problem_desc;

/* Diagnostics of the last rounding performed by a call (host struct). */
typedef struct {
    int d;                         /* number of cores                          */
    int ranks[TT_MAX_D + 1];       /* r_0..r_d after the call                  */
    int grown[TT_MAX_D + 1];       /* ranks entering the last rounding         */
    double discarded[TT_MAX_D];    /* sqrt(sum of discarded sigma^2) per bond  */
    double norm;                   /* ||X||_F entering the last rounding       */
    int capped;                    /* 1 if max_rank bound at some bond         */
    int sweeps;                    /* most Jacobi sweeps used by one eigensolve */
} tt_step_info;

/*
 * tt_create: build a TT-S_N problem (Sec. 3, Sec. 4.1 layout) on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Returns TT_ERR_ARG on an
 * invalid description, TT_ERR_OOM if device memory runs out.
 */
tt_status tt_create(const tt_problem_desc* desc, void* stream, tt_handle* out);

/*
 * A caller-supplied device allocator: alloc returns
 * `bytes` of device memory usable on `stream` (a cudaStream_t) or NULL on
 * failure; free returns a block that alloc gave, with the same size and the
 * stream of its last use.  The library frees a block only after enqueuing the
 * work that uses it on that stream, so a stream-ordered (caching) allocator
 * may hand the block out again for later work on the same stream.  ctx is
 * passed through unchanged.
 */
typedef struct {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} tt_allocator;

/*
 * tt_create_ex: as tt_create, with every device buffer of the handle (cores,
 * workspaces, scratch, tape) taken from `alloc` instead of the CUDA
 * stream-ordered pool; alloc (nullable: as tt_create) is copied, and its ctx
 * and functions must stay valid until tt_destroy.  Kernel-level calls
 * (tt_gram, tt_dgemm, ...) keep using the pool.
 */
tt_status tt_create_ex(const tt_problem_desc* desc, void* stream, const tt_allocator* alloc,
                       tt_handle* out);

/*
 * tt_create_tt: a bare TT with d cores of mode sizes n[0..d-1] and ranks
 * ranks[0..d] (ranks[0] = ranks[d] = 1), all cores zero; used with
 * tt_set_cores / tt_round / tt_to_full.  Physics calls return TT_ERR_STATE.
 */
tt_status tt_create_tt(int d, const int* n, const int* ranks, void* stream, tt_handle* out);

/*
 * tt_sn_step: advance nsteps time steps (Sec. 3-4): upwind transport applied
 * as a TT sum of 1 + 2 ndim rank-one-masked terms (Sec. 4.3, Eq. upwind),
 * backward-Euler absorption/emission with the quartic temperature solve
 * (Sec. 3.2, Eq. couple_a/couple_b) assembled as a row scaling of the spatial
 * core plus one rank-one emission term (Sec. 4.4), Gram-SVD rounding to eps
 * (App. A.2), and the energy-conserving temperature update (Sec. 3.2).
 * info (nullable) receives the diagnostics of the last step.
 * Returns TT_WARN_RANK_CAPPED if max_rank bound in any step, and
 * TT_ERR_NONFINITE (stopping at that step) if a rounding meets Inf or NaN:
 * an unstable time step, or a non-finite field or state, would otherwise
 * round to the zero tensor without notice.
 */
tt_status tt_sn_step(tt_handle h, int nsteps, tt_step_info* info);

/*
 * tt_sn_step_ex: as tt_sn_step with flags (TT_STEP_NO_SOURCE,
 * TT_STEP_NO_ROUND) and optional forced ranks (host; NULL = use eps) that
 * replace the tolerance rule: d-1 ints for the one rounding of a step, or
 * 2(d-1) ints when rounds_per_step = 2 (post-transport rounding first), used
 * in every step of the call.
 */
tt_status tt_sn_step_ex(tt_handle h, int nsteps, int flags, const int* forced_ranks_host,
                        tt_step_info* info);

/*
 * tt_round: round the current TT in place with Algorithm 1 and the Gram-SVD
 * truncation (App. A.2) to relative tolerance eps, rank cap max_rank (<= 0:
 * none) or forced ranks (d-1 ints, host; NULL = eps rule).
 */
tt_status tt_round(tt_handle h, double eps, int max_rank, const int* forced_ranks_host,
                   tt_step_info* info);

/*
 * tt_energy: radiation energy density E_i = (1/c) sum_lp I_ilp dOmega_lp by
 * TT integration (Eq. tt_energy_density) into E_dev (N_c doubles, nullable),
 * the material temperature into T_dev (nullable), and totals_host[0] =
 * sum_i E_i dV, totals_host[1] = sum_i cv_i T_i dV (nullable).
 */
tt_status tt_energy(tt_handle h, double* E_dev, double* T_dev, double* totals_host);

/*
 * tt_to_full: expand the TT into out_dev (prod n_k doubles, C order of
 * (n_1, ..., n_d)); TT_ERR_TOO_LARGE if out_len is smaller.
 */
tt_status tt_to_full(tt_handle h, double* out_dev, size_t out_len);

/* tt_get_ranks: copy r_0..r_d into ranks_host (cap entries at most). */
tt_status tt_get_ranks(tt_handle h, int* ranks_host, int cap);

/* tt_get_dims: d and the mode sizes n_1..n_d (n_host holds TT_MAX_D ints). */
tt_status tt_get_dims(tt_handle h, int* d_host, int* n_host);

/*
 * tt_get_core: copy core k (0-based) into out_dev (r_{k-1} n_k r_k doubles);
 * TT_ERR_TOO_LARGE if out_len is smaller.  out_dev may be device memory or
 * host memory (pinned host memory copies at the host link's speed); the call
 * returns once the copy is complete.
 */
tt_status tt_get_core(tt_handle h, int k, double* out_dev, size_t out_len);

/*
 * tt_get_cores: borrowed device views of the cores: cores_dev[k] (host array
 * of d pointers) receives core k's device address, shapes_host[3k..3k+2] its
 * shape (r_{k-1}, n_k, r_k).  Synchronises the stream first; the views stay
 * valid until the next call that changes the TT (steps, rounding, set calls,
 * tt_destroy).  Use tt_get_core for an owned copy.
 */
tt_status tt_get_cores(tt_handle h, double** cores_dev, int* shapes_host);

/*
 * tt_set_cores: replace the TT by the d cores cores_dev[k] (shapes
 * (ranks[k], n_k, ranks[k+1])), copied in; ranks_host has d+1 entries.  The
 * cores may be in device memory or in host memory (pinned or pageable); the
 * call returns once they are copied, so the caller may reuse the buffers.
 */
tt_status tt_set_cores(tt_handle h, const double* const* cores_dev, const int* ranks_host);

/*
 * tt_set_inflow: a given incoming intensity on one face (Sec. 4.5 ghost cells
 * holding a Dirichlet value instead of zero): on face `side` (0: low, 1: high)
 * of a TT_BC_VACUUM axis the ghost cells hold the rank-one intensity
 * g(cell) theta(l) phi(p), g_dev N_c doubles in cell order (read on the face's
 * layer of cells), theta_dev n_theta and phi_dev n_phi doubles, copied in.
 * With the flux's face weights the known ghost enters the boundary cells'
 * stencil as one rank-one term per face for upwinding (two for Rusanov and
 * HLL), carried like a fixed source (tt_set_sources) that follows the
 * caller's own sources; together at most TT_MAX_SOURCES.  g_dev = NULL
 * removes the face's inflow.  TT_ERR_ARG for a bad axis/side, a face that is
 * not vacuum or too many terms; TT_ERR_STATE on a split-layout handle.  The
 * hohlraum problem of Sec. 5.1 is unit isotropic inflow on the low x and y
 * faces.
 */
tt_status tt_set_inflow(tt_handle h, int axis, int side, const double* g_dev, const double* theta_dev,
                        const double* phi_dev);

/*
 * tt_set_sketch: the Gaussian sketch TT of the randomized rounding (App. A.3):
 * d device cores omega_dev[k] of shape (ranks_host[k], n_k, ranks_host[k+1])
 * (ranks_host has d + 1 entries, the first and last 1), copied in; NULL
 * removes it.  The caller draws the numbers (any Gaussian generator); a
 * rounding to ranks l_k uses the cores' leading (l_{k-1}, n_k, l_k) blocks,
 * so l_k <= ranks_host[k].
 * tt_set_rounding: TT_ROUND_GRAM (default; the tolerance and cap rules of
 * tt_round / steps) or TT_ROUND_RANDOMIZED for the following roundings of the
 * handle (steps and tt_round): for every bond W = B^T Omega (backward sweep),
 * then A' = Q, an orthonormal basis of A W, and M_upd = Q^T A (Eq.
 * randfinal).  Its ranks are the forced ranks if a call gives them, else the
 * sketch's ranks (both capped by the bond); eps and max_rank are not used.
 * FP64 whatever the precision setting.  TT_ERR_STATE without a sketch.
 * TT_ROUND_TTSVD: the QR-based TT-SVD rounding of App. A.1 with the same
 * tolerance, forced-rank and cap rules as TT_ROUND_GRAM: a backward sweep of
 * QR factorisations makes cores d-1 .. 1 right-orthonormal, then each left
 * unfolding A = Q Rf is truncated by the SVD of Rf.  The QR factors come from
 * three passes of eigen-form Cholesky QR (the first shifted), the SVD of Rf
 * from the eigenpairs of its Jordan-Wielandt matrix, so singular values are
 * resolved to eps_mach of the largest (App. A.4), at several times the Gram
 * path's cost.  FP64 whatever the precision setting.  Neither non-Gram
 * method is open to a spatial shard or while an adjoint tape records
 * (TT_ERR_STATE), nor to captured steps.
 */
tt_status tt_set_sketch(tt_handle h, const double* const* omega_dev, const int* ranks_host);
tt_status tt_set_rounding(tt_handle h, int method);

/*
 * tt_set_eigensolver: how the Gram-SVD rounding (App. A.2) takes the
 * eigenpairs of its small positive semidefinite matrix K = W G_A W^T at each
 * bond.  TT_EIG_ONE_SIDED (default): pivoted Cholesky K = W_K^T W_K, then
 * one-sided Jacobi on the rows of W_K (tt_syev_psd).  TT_EIG_TWO_SIDED:
 * two-sided Jacobi on K (tt_syev).  Both keep small eigenvalues to relative
 * accuracy; the one-sided form does about half the FP64 work with one grid
 * barrier per round.  TT_ERR_ARG for another value; TT_ERR_STATE for a change
 * while captured steps are on.
 */
tt_status tt_set_eigensolver(tt_handle h, int method);

/*
 * tt_set_graph: captured steps (enable = 1) or host-driven steps (0, the
 * default).  With capture on, the first tt_sn_step / tt_sn_step_ex call
 * without flags and forced ranks records one whole step (transport, source,
 * rounding, temperature update) into a CUDA graph, and that call and every
 * later one replay it, nsteps replays per call with one synchronisation at
 * the end.  The step's sizes are decided on the device: the kernels of the
 * recorded step read the grown ranks, the right Grams' numerical ranks and
 * both rank decisions from a device size block (grids cover the rank cap),
 * so one recording serves every later step whatever its ranks; results are
 * the same bits as host-driven steps.  Takes the grouped layout, FP64,
 * rounds_per_step 1, Gram-SVD rounding, a rank cap (max_rank > 0), upwind or
 * Rusanov, no fixed sources or inflow faces, no tape, not a shard
 * (TT_ERR_STATE otherwise, also when a later setting breaks one of these).
 * The info of a call is its last step's; TT_WARN_RANK_CAPPED if the cap bound
 * in any replayed step; a step that meets a zero tensor returns TT_ERR_STATE
 * (the recorded step does not represent it).  Calls other than steps
 * synchronise first and see the device's ranks.
 */
tt_status tt_set_graph(tt_handle h, int enable);

/* tt_set_precision: TT_FP64 or TT_MIXED for the following roundings. */
tt_status tt_set_precision(tt_handle h, int precision);

/* tt_set_T: replace the material temperature (N_c doubles, device or host
 * memory; copied before the call returns). */
tt_status tt_set_T(tt_handle h, const double* T_dev);

/*
 * tt_set_sources: fixed external sources S = sum_k x_k (x) theta_k (x) phi_k,
 * k < count (0 <= count <= TT_MAX_SOURCES; 0 removes them), an inhomogeneous
 * term of the transport equation (Sec. 3) taken explicitly with the
 * streaming: every step's transport stage gives I* = L I + c dt S, and each
 * source is one more rank-one term of the TT sum (the grown ranks become
 * (1 + 2 ndim) r + count (+1 for the emission term)).  Device arrays, copied
 * in: x_dev count x N_c (cell order as the fields), theta_dev count x n_theta,
 * phi_dev count x n_phi, row-major.  Ends any adjoint tape; the adjoint form
 * does not take sources (tt_tape_begin returns TT_ERR_STATE while any are set).
 * Grouped layout only (TT_ERR_STATE on a split-layout handle).
 */
tt_status tt_set_sources(tt_handle h, int count, const double* x_dev, const double* theta_dev,
                         const double* phi_dev);

/* tt_sync: wait for the handle's stream and report any latched device status. */
tt_status tt_sync(tt_handle h);

/* tt_last_error: thread-local message for the last failing call ("" if none). */
const char* tt_last_error(void);

/* tt_destroy: free the handle and its device memory (NULL is a no-op). */
void tt_destroy(tt_handle h);

/* ---------------------------------------------------------------------------
 * Adjoint form: gradient of the boundary-escape energy with respect to
 * sigma_a by reverse mode through the step of Sec. 3.2 / 4.3-4.4 and the
 * rounding of App. A.
 *
 * Objective: Q = sum over the taped steps m of the radiation energy that
 * leaves through the faces of vacuum axes (Sec. 4.5) during the step,
 *   Q_m = sum_faces sum_{cells i on the face} sum_{l,p}
 *         dt dA (n_lp . n_out)^+ I^m_{ilp} dOmega_lp,
 * I^m the state after step m, dA the face area (product of the other axes'
 * cell widths), n_out the outward face normal.  Periodic axes have no faces.
 *
 * The gradient is that of the step map with each rounding's factors held
 * fixed at their taped values (P_A^T and M_upd of every bond: the rounded
 * cores are X_g P_1 and M_1 Theta_g P_2 and M_2 Phi_g).  It equals the
 * derivative of the untruncated scheme wherever the truncated directions
 * carry no perturbation, and differs from a finite difference of the rounded
 * map at the level of the discarded singular values.  The temperature solve
 * (quartic) is reversed by the implicit-function theorem.
 * ------------------------------------------------------------------------ */

/*
 * tt_tape_begin: start recording.  Every later tt_sn_step / tt_sn_step_ex step
 * (flags 0; FP64 precision, rounds_per_step 1, no scattering, else
 * TT_ERR_STATE) appends a record and adds its Q_m to the objective.  Records
 * hold the step's input state (cores and T) every checkpoint_every (>= 1)
 * steps and, when checkpoint_every == 1, the frozen factors of every step;
 * otherwise tt_sn_step_adjoint re-runs each segment from its checkpoint.
 * Device memory held: about (steps / checkpoint_every + checkpoint_every)
 * states.  Clears any earlier tape and zeroes Q.  tt_round, tt_set_cores,
 * tt_set_T and tt_set_precision end the tape (the recorded run is discarded).
 */
tt_status tt_tape_begin(tt_handle h, int checkpoint_every);

/* tt_tape_objective: Q so far (host double) and, if steps_host is non-null,
 * the number of taped steps.  Synchronises the handle's stream. */
tt_status tt_tape_objective(tt_handle h, double* Q_host, int* steps_host);

/*
 * tt_sn_step_adjoint: run the reverse sweep over the taped steps.
 * grad_sigma_a_dev (device, N_c doubles, cell order as tt_create's fields,
 * nullable) receives dQ/dsigma_a; Q_host (nullable) receives Q.  The handle's
 * state (cores, ranks, T) is left as it was after the last taped step; the
 * tape is released and recording stops.  TT_ERR_STATE without a tape or if a
 * replayed step's ranks differ from the taped ones.
 */
tt_status tt_sn_step_adjoint(tt_handle h, double* grad_sigma_a_dev, double* Q_host);

/* tt_tape_clear: stop recording and release the tape. */
tt_status tt_tape_clear(tt_handle h);

/* ---------------------------------------------------------------------------
 * Batched form: many independent problems of uneven sizes stepped together.
 * ------------------------------------------------------------------------ */
typedef struct tt_batch_ctx* tt_batch;

/*
 * tt_batch_create: one problem per descs[i] (as tt_create), each on a CUDA
 * stream the batch creates and owns, all on the current device.  threads
 * (<= 0: min(count, 32)) host threads advance problems concurrently in
 * tt_batch_step.
 */
tt_status tt_batch_create(const tt_problem_desc* descs, int count, int threads, tt_batch* out);

/*
 * tt_batch_step: advance every problem by nsteps time steps (as tt_sn_step);
 * infos (nullable) receives count step infos.  The first failing problem's
 * status is returned with its message.
 */
tt_status tt_batch_step(tt_batch b, int nsteps, tt_step_info* infos);

/* tt_batch_size: number of problems.  tt_batch_handle: borrowed handle of
 * problem i (valid until tt_batch_destroy; use it for tt_energy, tt_to_full,
 * tt_get_core ...).  tt_batch_sync: wait for every problem's stream. */
tt_status tt_batch_size(tt_batch b, int* count);
tt_status tt_batch_handle(tt_batch b, int i, tt_handle* out);
tt_status tt_batch_sync(tt_batch b);
void tt_batch_destroy(tt_batch b);

/*
 * tt_batch_set_graph: captured steps (tt_set_graph) for every problem of the
 * batch.  The first tt_batch_step then records one graph holding every
 * problem's step as a branch of its own, and each batch step is one launch
 * of it (the branches run concurrently, ordered with each problem's stream
 * by events), with one synchronisation per problem at the end of the call
 * instead of the rank read-backs inside every step.  TT_ERR_STATE if a
 * problem cannot be captured (see tt_set_graph); the batch is then left
 * unchanged.  Disabling drops the graph.
 */
tt_status tt_batch_set_graph(tt_batch b, int enable);

/* ---------------------------------------------------------------------------
 * Spatial sharding: the method partitioned over space across several
 * processes (one GPU each).  In the grouped layout (Sec. 4.1, Eq.
 * tensor_decomp) the spatial core X holds one row per cell; a shard holds the
 * rows of a slab of whole layers along axis 0 (cells with plane_begin <= c_0 <
 * plane_end), and the angular cores Theta, Phi are replicated.  One step then
 * needs exactly two exchanges:
 *   - the upwind stencil of Sec. 4.3 reads one ghost layer on each side of
 *     the slab (Sec. 4.5 ghost cells): a halo exchange of the rows of X in
 *     the slab's first and last layers with the neighbouring shards;
 *   - the Gram-SVD rounding of App. A.2 needs the left Gram matrix of the
 *     spatial core, G_A = X*^T X* = sum over shards of X*_s^T X*_s: an
 *     R x R all-reduce (sum).
 * Everything else is either local to the rows (the grown core, the source
 * stage and quartic of Sec. 3.2, the core update A' = A P_A, the energy
 * update) or computed identically on every shard from replicated data (the
 * right Grams, the eigensolves and rank decisions, the small products, the
 * angular cores), so all shards take the same rank decisions.
 * ------------------------------------------------------------------------ */

enum { TT_XCHG_SUM = 0, TT_XCHG_HALO = 1 };

/*
 * The exchange callback of a shard.  The library calls it from inside
 * tt_sn_step / tt_round / tt_energy with its stream already synchronised; the
 * callback must have finished writing before it returns.  buf_dev is device
 * memory of the handle; stream is the handle's cudaStream_t (for callers that
 * order their own work on it).  Return 0 on success, anything else aborts
 * the call with TT_ERR_STATE.
 *   kind TT_XCHG_SUM: buf_dev holds count doubles; replace them by their sum
 *     over all shards, the same bits on every shard (an all-reduce).
 *   kind TT_XCHG_HALO: buf_dev holds four blocks of count doubles, [send_lo |
 *     send_hi | recv_lo | recv_hi]; on the ring of shards ordered by plane
 *     (shard s - 1 below s, the last shard below the first), fill recv_lo
 *     with the send_hi block of the shard below and recv_hi with the send_lo
 *     block of the shard above (with one shard, its own blocks).  The library
 *     then replaces the ghost layer of a global vacuum face by zeros and of a
 *     global outflow face by the boundary layer itself, so the ring's
 *     wrap-around is what a periodic axis 0 needs.
 */
typedef int (*tt_exchange_fn)(void* ctx, int kind, double* buf_dev, size_t count, void* stream);

/*
 * tt_create_shard: as tt_create for the shard of layers [plane_begin,
 * plane_end) along axis 0 of the grid that desc describes (the whole grid:
 * desc's fields are device arrays of all N_c cells, of which the shard copies
 * its own).  exchange (with ctx passed through) carries the halo and the sum
 * described above; it must stay valid until tt_destroy.  The shard's TT is
 * X (1, N_s, r1), Theta, Phi with N_s = (plane_end - plane_begin) times the
 * cells of one layer, in the same C order; tt_to_full, tt_energy's E and T
 * and tt_get_core(0) cover the shard's cells, tt_energy's totals the whole
 * grid.  Grouped layout only; upwind and Rusanov fluxes (HLL's per-face
 * optical depths would need the neighbours' opacities); no fixed sources,
 * inflow faces, adjoint tape or randomized rounding (TT_ERR_STATE).
 * TT_ERR_ARG for an empty or out-of-range slab or a null callback.
 */
tt_status tt_create_shard(const tt_problem_desc* desc, void* stream, int plane_begin, int plane_end,
                          tt_exchange_fn exchange, void* ctx, tt_handle* out);

/* ---------------------------------------------------------------------------
 * Kernel-level calls (the building blocks of tt_round, exposed for testing and
 * for callers that hold their own TT data).  All ordered on `stream`.
 * ------------------------------------------------------------------------ */

/*
 * tt_dgemm: C = alpha op(A) op(B) + beta C in FP64 on the FP64 tensor pipe
 * (mma m8n8k4), row-major, op(X) = X if trans_x == 0 else X^T; op(A) is M x K,
 * op(B) is K x N, C is M x N with leading dimensions lda, ldb, ldc.
 */
tt_status tt_dgemm(int trans_a, int trans_b, int M, int N, int K, double alpha,
                   const double* A_dev, int lda, const double* B_dev, int ldb, double beta,
                   double* C_dev, int ldc, void* stream);

/*
 * tt_gram: G = A^T A for a tall row-major A (m x n, leading dimension lda), the
 * left Gram matrix of App. A.2 (G_A = A^T A).  Split over the m rows with a
 * fixed-order reduction, so the result is bitwise reproducible; G (n x n,
 * leading dimension ldg) is exactly symmetric.  Uses device scratch of
 * (number of row splits) * n * n doubles allocated by the library.
 */
tt_status tt_gram(int m, int n, const double* A_dev, int lda, double* G_dev, int ldg, void* stream);

/*
 * tt_wait_probe: self-test of the device-side failure detection.  The
 * library's persistent kernels (Jacobi eigensolver, pivoted Cholesky) wait at
 * grid-wide barriers with a bounded spin (~1 s) that latches a status word
 * instead of waiting forever.  This call runs one such wait that can never
 * complete (one CTA waiting for a second that is never launched) and returns
 * TT_ERR_TIMEOUT when the wait ran out and the kernel returned; the CUDA
 * context stays usable.  Any other status means the bounded wait is broken.
 */
tt_status tt_wait_probe(void* stream);

/*
 * tt_pchol: pivoted Cholesky factor of a symmetric positive semidefinite n x n
 * matrix G (leading dimension ldg), the factor of the right Gram matrix that
 * the one-sided truncation uses (W^T W = G_B, App. A.2): the pivot is the
 * largest remaining diagonal entry and the factorisation stops when it falls
 * to eps_mach times the largest initial diagonal entry.  W_dev (n x n,
 * row-major, leading dimension n) receives the rank_host rows of W (rows
 * beyond it are unspecified); G is not modified.  TT_ERR_TOO_LARGE if n x 8
 * bytes exceed the shared-memory limit of one CTA (n > 25600);
 * TT_ERR_NONFINITE if the diagonal of G holds Inf or NaN.
 */
tt_status tt_pchol(int n, const double* G_dev, int ldg, double* W_dev, void* stream, int* rank_host);

/*
 * tt_syev: eigendecomposition G = V diag(lam) V^T of a symmetric n x n matrix
 * (the "small symmetric eigensolves" of App. A.2) by cyclic parallel Jacobi in
 * FP64.  lam_dev receives the n eigenvalues in descending order; Vt_dev
 * (n x n, leading dimension ldv) receives the eigenvectors as ROWS (row j is
 * the eigenvector of lam[j]).  G is not modified.  sweeps_host (nullable)
 * receives the number of Jacobi sweeps; TT_ERR_NOT_CONVERGED if the sweep
 * limit was reached (results are then approximate).
 */
tt_status tt_syev(int n, const double* G_dev, int ldg, double* lam_dev, double* Vt_dev, int ldv,
                  void* stream, int* sweeps_host);

/*
 * tt_syev_ex: tt_syev with a sweep limit of max_sweeps (1 .. 40; tt_syev
 * uses 40).  A limit the iteration reaches returns TT_ERR_NOT_CONVERGED, as
 * a stand-in for an eigensolve that failed to converge; nothing else changes.
 * tt_set_max_sweeps: the same limit for the eigensolves of a handle's
 * roundings (default 40); a step whose eigensolve reaches it completes and
 * returns TT_ERR_NOT_CONVERGED, and the handle stays usable.  TT_ERR_ARG for
 * a limit outside 1 .. 40.
 */
tt_status tt_syev_ex(int n, const double* G_dev, int ldg, double* lam_dev, double* Vt_dev, int ldv,
                     int max_sweeps, void* stream, int* sweeps_host);

/*
 * tt_syev_psd: eigendecomposition K = V diag(lam) V^T of a symmetric positive
 * semidefinite n x n matrix (the Gram-type matrices of App. A.2) by pivoted
 * Cholesky K = W^T W followed by one-sided Jacobi on the rows of W (Demmel and
 * Veselic 1992): small eigenvalues keep the relative accuracy of two-sided
 * Jacobi at about half its work.  Same layout, ordering, sweep limit and
 * status codes as tt_syev_ex.  Eigenvalues below the factorisation's floor
 * (eps_mach max diag K) are returned as 0 with zero rows in Vt; an indefinite
 * K is factorised only down to its first non-positive pivot.
 */
tt_status tt_syev_psd(int n, const double* K_dev, int ldk, double* lam_dev, double* Vt_dev, int ldv,
                      int max_sweeps, void* stream, int* sweeps_host);
tt_status tt_set_max_sweeps(tt_handle h, int max_sweeps);

/*
 * tt_gram_mixed: G = A^T A (as tt_gram) on the BF16 tensor cores (tcgen05).
 * Each column of A is scaled by a power of two and cut into seven signed
 * 7-bit digits (exact in BF16); digit products are exact in FP32, summed
 * exactly over 512-row blocks in tensor memory, and accumulated in
 * double-float (about 48 bits); products of digit levels s + t >= 7 are
 * dropped.  Error about 2^-48 max|A_j| max|A_k| per row term.  Device scratch
 * (row splits x n x n doubles and the digit planes, 14 bytes per element of
 * A) is allocated per call.
 */
tt_status tt_gram_mixed(int m, int n, const double* A_dev, int lda, double* G_dev, int ldg,
                        void* stream);

/*
 * tt_gemm_nt_mixed: C = A B^T (A: M x K, B: N x K, C: M x N, row-major) with the
 * same exact split products on the tensor cores, each row of A and of B scaled
 * by its own power of two (error about 2^-48 max_k|A_ik| max_k|B_jk| per term).
 * An output with too few 128 x 64 tiles to occupy the GPU is computed split-K
 * over the contraction, the partial products added in a fixed order (results
 * do not depend on scheduling).  Device scratch (digit images, 14 bytes per
 * element of A and B, and the partials) is allocated per call.
 */
tt_status tt_gemm_nt_mixed(int M, int N, int K, const double* A_dev, int lda, const double* B_dev,
                           int ldb, double* C_dev, int ldc, void* stream);

/*
 * tt_gram_noalloc: the same G = A^T A as tt_gram, for callers that must not
 * allocate device memory (for example an application whose own allocator owns
 * all device memory, or a latency-critical loop that cannot afford the
 * synchronisation of cudaMalloc/cudaFree).  The paper has no counterpart; this
 * is a property of the library, not of the method.  It allocates nothing: its
 * split-K scratch is a fixed 8 MiB array in device global memory that every
 * GPU loading the library holds until the process exits, which limits n to
 * 1024 (larger n returns TT_ERR_TOO_LARGE with a message; use tt_gram).  The
 * caller passes A (m x n, leading dimension lda) and the output G (n x n,
 * leading dimension ldg).  The first call on each device looks up the array's
 * device address with that device current; make that first call before any
 * stream capture begins.  All calls share the array, so calls that overlap on
 * the GPU race on it and must be serialised by the caller.  Results equal
 * tt_gram's up to the order of the floating-point sums (the split-K factor may
 * be smaller) and are exactly symmetric and reproducible.  The split over rows
 * is capped so that its n x n partials fit the array (2^20 / n^2 splits): for
 * n > 724 only one fits and the call runs without a row split, one CTA per
 * upper-triangle tile, which is slower than tt_gram on tall A (measured on
 * GB300: 300,000 x 897 in 680 ms against 273 ms; 300,000 x 700, two splits,
 * 341 against 152 ms).
 */
tt_status tt_gram_noalloc(int m, int n, const double* A_dev, int lda, double* G_dev, int ldg,
                          void* stream);

/* ---------------------------------------------------------------------------
 * Autotuned products (no counterpart in the paper).  The FP64 products of the
 * rounding whose output tile grid (64 x 64 tiles) leaves SMs idle split their
 * contraction depth K over CTAs; how many splits pays depends on the GPU.
 * tt_autotune measures, for every bucket of (floor(log2 tiles) < 8,
 * floor(log2 K) from 6 to 14), the product's time at each split 1, 2, 4, ...,
 * 64 (up to K / 32) on a representative product of that bucket, keeps the
 * fastest (best of three runs), extends the deepest bucket's choice to deeper
 * products, and installs the table for every later product of the process,
 * host-driven and captured alike (both read the same table, so their results
 * stay the same bits).  table_out (nullable, host) receives the
 * TT_AUTOTUNE_ENTRIES entries, index floor(log2 tiles) * 22 + floor(log2 K);
 * 0 means the built-in rule.  Takes a few seconds and some 1.5 GB of device
 * memory while it runs; call it before creating handles or recording steps,
 * not concurrently with other library calls.  tt_set_autotune_table installs
 * a stored table (entries 0 .. 64; TT_ERR_ARG otherwise), and
 * tt_get_autotune_table copies the installed one (all zero until a table is
 * installed).
 * ------------------------------------------------------------------------ */
#define TT_AUTOTUNE_ENTRIES (8 * 22)
tt_status tt_autotune(void* stream, int* table_out);
tt_status tt_set_autotune_table(const int* table_host, int n);
tt_status tt_get_autotune_table(int* table_host, int n);

/* ---------------------------------------------------------------------------
 * Measurement calls (no counterpart in the paper; used by the benchmark to
 * attribute time to the phases of the step and to count kernel launches).
 * ------------------------------------------------------------------------ */

/* Phases of the step timed with CUDA events on the handle's stream.  Every
 * phase occurrence (and every step of tt_sn_step) is also an NVTX range named
 * after it ("transport", "gram_right", "eig", "gram_left", "small", "update",
 * "energy"; "tt_sn_step"), so a profiler can attribute kernels to phases. */
enum {
    TT_PH_TRANSPORT = 0,  /* grown cores: transport terms + source (Sec. 4.3-4.4)  */
    TT_PH_GRAM_RIGHT = 1, /* backward sweep: right Gram matrices (App. A, Alg. 1)  */
    TT_PH_EIG = 2,        /* Jacobi eigensolves and rank decisions                */
    TT_PH_GRAM_LEFT = 3,  /* left Gram G_A = A^T A of each bond (App. A.2)        */
    TT_PH_SMALL = 4,      /* R x R products: W G_A W^T, P_A, M_upd                */
    TT_PH_UPDATE = 5,     /* core updates A' = A P_A and M_upd x_1 G_{k+1}        */
    TT_PH_ENERGY = 6,     /* quadrature of the rounded TT + temperature update    */
    TT_NPHASES = 7
};

/*
 * tt_profile: enable (1, also resets the accumulators) or disable (0) phase
 * timing on the handle.  While enabled every phase is bracketed by CUDA events
 * on the handle's stream; totals are resolved at the synchronisation points
 * of each call.
 */
tt_status tt_profile(tt_handle h, int enable);

/*
 * tt_profile_read: accumulated totals of one phase since the last reset: GPU
 * time in ms, kernel launches, phase occurrences, algorithmic flops and
 * algorithmic DRAM bytes (each nullable).  The algorithmic counts are those of
 * the operation (e.g. m R (R+1) flops for a symmetric m x R Gram), not of the
 * kernels' implementation.
 */
tt_status tt_profile_read(tt_handle h, int phase, double* ms, long long* launches,
                          long long* calls, double* flops, double* bytes);

/* tt_kernel_launches: kernels launched by the library since the process started. */
unsigned long long tt_kernel_launches(void);

/*
 * tt_bench_fp64_mma: measured throughput of the FP64 tensor pipe (dependent
 * chains of mma.m8n8k4.f64 on every SM) in TFLOP/s, written to tflops_host.
 */
tt_status tt_bench_fp64_mma(double* tflops_host, void* stream);

/*
 * tt_bench_bf16_mma: measured throughput of warp-level BF16 tensor MMA
 * (dependent chains of mma.sync m16n8k16 with FP32 accumulation on every SM),
 * the instruction the mixed contractions use, in TFLOP/s.
 */
tt_status tt_bench_bf16_mma(double* tflops_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TTSN_H */
