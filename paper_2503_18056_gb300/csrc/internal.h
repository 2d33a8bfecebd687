// Internal declarations shared by the libttsn translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/ttsn.h"

namespace ttsn {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* get_error();

#define TT_CUDA_TRY(expr)                                                           \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            ::ttsn::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); \
            return (_e == cudaErrorMemoryAllocation) ? TT_ERR_OOM : TT_ERR_CUDA;    \
        }                                                                           \
    } while (0)

#define TT_TRY(expr)                         \
    do {                                     \
        tt_status _s = (expr);               \
        if (_s < 0) return _s;               \
    } while (0)

// Device status word values (latched by kernels, read by the host).
enum : int { DEV_OK = 0, DEV_NOT_CONVERGED = 1, DEV_TIMEOUT = 2 };

// ---------------------------------------------------------------- launch accounting
// Every kernel launch of the library goes through note_launch() so callers can
// count the library's launches inside a timed region (tt_kernel_launches).
void note_launch(unsigned n = 1);

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per kernel and never lower (the attribute is process-wide, so setting it
// per launch to the launch's own size races between host threads that step
// different problems concurrently).
tt_status ensure_max_dynamic_smem(const void* kernel);

// ---------------------------------------------------------------- device buffer
// A growable device buffer: capacity only grows; contents are not preserved
// across a grow unless `keep` is set.
struct DevBuf {
    double* p = nullptr;
    size_t cap = 0;  // in doubles
    // the allocator that provided p (null: cudaMallocAsync / cudaFree) and the
    // stream it was requested on; taken from the calling thread's current
    // allocator (AllocScope) when the buffer first allocates
    const tt_allocator* alloc = nullptr;
    cudaStream_t astream = nullptr;
    tt_status ensure(size_t n, cudaStream_t s, bool keep = false);
    void release();
};

// The device allocator a handle was created with, current on this thread for
// the duration of a call on that handle (null: the stream-ordered pool).
const tt_allocator* current_allocator();
struct AllocScope {
    const tt_allocator* prev;
    explicit AllocScope(const tt_allocator* a);
    ~AllocScope();
};

// ---------------------------------------------------------------- GEMM (gemm.cu)
// C = alpha op(A) op(B) + beta C, row-major FP64 on mma.m8n8k4.
// batch > 1: A, B, C advance by strideA/B/C per batch entry.
tt_status dgemm(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                const double* A, long lda, const double* B, long ldb, double beta, double* C,
                long ldc, int batch = 1, long strideA = 0, long strideB = 0, long strideC = 0);

// beta = 0 GEMM that splits K over CTAs (fixed-order reduction through
// scratch) when the M x N tile grid alone would leave most SMs idle and K is
// long; otherwise the plain dgemm.
tt_status dgemm_sk(cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
                   const double* A, long lda, const double* B, long ldb, double* C, long ldc,
                   DevBuf& scratch);

// Autotuned split table (gemm.cu): buckets of floor(log2 tiles) < 8 and
// floor(log2 K) < 22; autotune measures and installs it, autotune_install
// installs a stored one, autotune_read copies the installed one.
constexpr int AT_TILE_BUCKETS = 8, AT_K_BUCKETS = 22;
tt_status autotune(cudaStream_t s, int* table_out);
tt_status autotune_install(const int* table, int n);
void autotune_read(int* table);

// The split rules of dgemm_sk (split of K) and of the Gram (split of the
// rows, from the number of resident CTAs), shared by host and device.
__host__ __device__ void sk_split(int M, int N, int K, int* ks_out, int* kchunk_out);
__host__ __device__ int gram_split_rule(int m, int n, long resident);
// splits of a large Gram dealt in many waves (gram_split_rule)
constexpr int GRAM_MULTI_SPLITS = 64;

// Products of a captured step, their sizes read from device memory: desc =
// M, N, K, lda, ldb, ldc (Gram: n, n, m, lda, lda, ldg with A m x n), caps
// bound every size the step can reach.  mode 0: plain product into C; 1:
// dgemm_sk (split of K by sk_split, partials in P); 2: the Gram G = A^T A
// (row split by gram_split_rule, partials in P).  The same bits as the host
// path for the same sizes.  P holds pcap doubles, at least
// dyn_partials_need(mode, Mcap, Ncap, Kcap) (checked: TT_ERR_TOO_LARGE).
tt_status dgemm_dyn(cudaStream_t s, bool ta, bool tb, const int* desc, int Mcap, int Ncap, int Kcap,
                    double alpha, const double* A, const double* B, double* C, double* P, size_t pcap, int mode);
size_t dyn_partials_need(int mode, int Mcap, int Ncap, int Kcap);
long gram_resident();
// scale_rows with rows, cols, ldi, ldo = desc[0..3] (rows * cols <= total_cap)
void scale_rows_dyn(cudaStream_t s, const int* desc, long total_cap, const double* in, const double* v, int mode,
                    double* out);

// G = A^T A (A: m x n row-major, lda); split over rows with fixed-order reduction.
// `partials` is scratch grown as needed (ksplit * n * n doubles).
tt_status gram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
               DevBuf& partials);
// The same with caller-provided scratch of `scratch_doubles` entries (no allocation).
tt_status gram_with_scratch(cudaStream_t s, int m, int n, const double* A, long lda, double* G,
                            long ldg, double* scratch, size_t scratch_doubles);
size_t gram_scratch_doubles(int m, int n);
// The same Gram with a fixed scratch: the split-K factor is reduced so the
// partials fit in scratch_doubles (needs scratch_doubles >= n * n).
tt_status gram_fixed_scratch(cudaStream_t s, int m, int n, const double* A, long lda, double* G,
                             long ldg, double* scratch, size_t scratch_doubles);
// Measured FP64 tensor-pipe throughput (TFLOP/s).
tt_status bench_fp64_mma(cudaStream_t s, double* tflops);
// Measured BF16 mma.sync (m16n8k16, FP32 accumulate) throughput (TFLOP/s).
tt_status bench_bf16_mma(cudaStream_t s, double* tflops);

// Mixed-precision (exact BF16 digit products, double-float accumulation) left
// Gram G = A^T A and product C = A B^T (slice.cu).  scratch grows as needed.
size_t slgram_scratch_doubles(int m, int n);
// erow_out (nullable, m ints): also the row exponents of A that slgemm_nt
// takes as erowA for the same A, from the same read of A.
tt_status slgram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
                 DevBuf& scratch, int* status_dev = nullptr, int* erow_out = nullptr);
// The left Gram on tcgen05 tensor cores (7-digit split, exact 512-row level
// sums, TMEM accumulators): what slgram runs.  status_dev (nullable) latches
// DEV_TIMEOUT if a bounded wait ran out.
size_t tcgram_scratch_doubles(int m, int n);
tt_status tcgram(cudaStream_t s, int m, int n, const double* A, long lda, double* G, long ldg,
                 DevBuf& scratch, int* status_dev, int* erow_out = nullptr);
// planes (nullable): where A's digit images go (14 bytes per element of A,
// padded to 128 rows x 32 columns), e.g. a buffer that is free at the time;
// null puts them in scratch.  erowA (nullable): A's row exponents from
// slgram's erow_out for this A (null: computed here).
tt_status slgemm_nt(cudaStream_t s, long M, int N, int K, const double* A, long lda, const double* B,
                    long ldb, double* C, long ldc, DevBuf& scratch, int* status_dev = nullptr,
                    DevBuf* planes = nullptr, const int* erowA = nullptr);

// Row scaling: out[i][j] = in[i][j] * f(v[i]) for i < rows, j < cols, where
// mode 0: v, 1: sqrt(v), 2: 1/sqrt(v), 3: 1/v.  out may alias in.
void scale_rows(cudaStream_t s, int rows, int cols, const double* in, long ldi, const double* v,
                int mode, double* out, long ldo);
void fill(cudaStream_t s, double* p, size_t n, double value);
// out[j] = alpha sum_i A[i][j] v[i], A m x ncols (lda), m large: row-split with
// a fixed-order reduction; scratch grows as needed.
tt_status gemv_t(cudaStream_t s, long m, int ncols, double alpha, const double* A, long lda,
                 const double* v, double* out, DevBuf& scratch);
void copy2d(cudaStream_t s, int rows, int cols, const double* in, long ldi, double* out, long ldo);

// ---------------------------------------------------------------- QR-based rounding (ttsvd.cu)
// out[i][j] = Vt[i][j] / sqrt(lam[i] + shift), i, j < l, lam descending, with
// shift = l eps_mach max(lam[0], 0) + max(0, -lam[l-1]) formed on the device.
void shifted_scale_rows(cudaStream_t s, int l, const double* Vt, long ldv, const double* lam, double* out,
                        long ldo);
// out (cols x rows, ldo) = in^T (in rows x cols, ldi)
void transpose(cudaStream_t s, long rows, long cols, const double* in, long ldi, double* out, long ldo);
// Jordan-Wielandt form of Rf (q x l, contiguous): c_dev[0] = ||Rf||_F and
// J ((q + l) x (q + l)) = [[c I, Rf], [Rf^T, c I]].
void jw_build(cudaStream_t s, int q, int l, const double* Rf, double* c_dev, double* J);
// sig2[i] = max(lam[i] - c, 0)^2, i < pm (the squared singular values of Rf)
void jw_sigma2(cudaStream_t s, int pm, const double* lam, const double* c_dev, double* sig2);
// From the eigenvectors (rows of Vt, ld ldv) of the Jordan-Wielandt matrix:
// U (r x q) rows sqrt(2) u_i^T, M (r x l) rows sigma_i sqrt(2) v_i^T.
void jw_split(cudaStream_t s, int r, int q, int l, const double* lam, const double* c_dev, const double* Vt,
              long ldv, double* U, double* M);

// ---------------------------------------------------------------- eigensolver (jacobi.cu)
struct EigWork {
    DevBuf g0, g1;          // double-buffered matrix
    DevBuf lam_unsorted;
    DevBuf vt_unsorted;
    DevBuf abc;             // per-round pair entries (double-buffered)
    DevBuf cs;              // the round's rotation angles (c, s per pair)
    DevBuf psd;             // syev_psd: factor workspace, row norms, factor rank
    DevBuf ctrl_buf;
    int* d_ctrl = nullptr;  // barrier counters, sweep counters, status (in ctrl_buf)
    int ctrl_cap = 0;
    void release();
};
// Eigendecomposition of symmetric n x n G (ldg): lam descending (n), Vt rows = eigvecs.
// *status_dev receives DEV_* codes (or-ed in; DEV_NOT_CONVERGED after
// max_sweeps sweeps, 1 .. JACOBI_MAX_SWEEPS); sweeps written to sweeps_dev[0].
constexpr int JACOBI_MAX_SWEEPS = 40;
tt_status syev(cudaStream_t s, int n, const double* G, long ldg, double* lam, double* Vt,
               long ldv, EigWork& w, int* status_dev, int* sweeps_dev,
               int max_sweeps = JACOBI_MAX_SWEEPS);

// Eigendecomposition of a symmetric positive semidefinite K (n x n, ldk) as
// syev returns it, by pivoted Cholesky K = W^T W and one-sided Jacobi on the
// rows of W: eigenvalues with the relative accuracy of two-sided Jacobi at
// about half its work and one grid barrier per round.  Eigenpairs below the
// factorisation's floor (eps_mach max diag K) come back as 0 with a zero
// vector; Inf/NaN in K as NaN eigenvalues.
tt_status syev_psd(cudaStream_t s, int n, const double* K, long ldk, double* lam, double* Vt, long ldv,
                   EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps = JACOBI_MAX_SWEEPS);
tt_status syev_psd_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* K, double* lam, double* Vt,
                       EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps = JACOBI_MAX_SWEEPS);

// Pivoted Cholesky of a symmetric positive semidefinite n x n G (ldg): writes
// W (rows 0..rank-1 of an n x n row-major buffer) with W^T W = G up to the
// floor eps_mach max(diag G), Wc (n x n scratch, the transpose) and uses
// dwork (2 n doubles, the double-buffered residual diagonal).  The rank is
// written to kB_dev.
tt_status pchol(cudaStream_t s, int n, const double* G, long ldg, double* W, double* Wc,
                double* dwork, EigWork& w, int* status_dev, int* kB_dev);

// The same factorisations in a captured step, their size n read from n_dev
// (at most ncap; grids, shared memory and workspaces fit ncap): the same bits
// as pchol / syev for the same n.  pchol_dyn writes the rank to kB_dev.
tt_status pchol_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* G, double* W, double* Wc,
                    double* dwork, EigWork& w, int* status_dev, int* kB_dev);
tt_status syev_dyn(cudaStream_t s, const int* n_dev, int ncap, const double* G, double* lam, double* Vt,
                   EigWork& w, int* status_dev, int* sweeps_dev, int max_sweeps);
// truncation_decision with the bond's size from kB_dev (a negative size, a
// failed factorisation, counts as zero)
void truncation_decision_dyn(cudaStream_t s, const double* lamK, const int* kB_dev, double eps, int dm1,
                             int forced, int max_rank, double* delta2_dev, int* dec_i, double* dec_d);

// Captured steps of one handle (api.cu): graph_steps_begin checks the
// conditions and launches nsteps replays without waiting; graph_steps_end
// waits for them and reports like tt_sn_step (info: the last step's).
tt_status graph_steps_begin(tt_handle h, int nsteps);
tt_status graph_steps_end(tt_handle h, tt_step_info* info);
// The captured steps of many handles as one graph (a branch per handle) and
// its replays: evs holds n + 1 events (the handles' and the origin's).
tt_status graph_batch_build(tt_handle* hs, int n, cudaGraphExec_t* out, unsigned* launches);
tt_status graph_batch_launch(tt_handle* hs, int n, cudaGraphExec_t exec, unsigned launches, cudaStream_t origin,
                             cudaEvent_t* evs, int nsteps);

// Shared-memory limits of the factorisation kernels set ahead of a capture,
// and the control block a capture's factorisations use.
tt_status eig_prepare();
tt_status eig_reserve(EigWork& w, cudaStream_t s);

// Self-test of the bounded grid-barrier wait: a wait that can never complete
// runs out and latches DEV_TIMEOUT into *status_dev.
tt_status wait_probe(cudaStream_t s, EigWork& w, int* status_dev);

// ---------------------------------------------------------------- rounding helpers (jacobi.cu)
// Truncation decision for one bond (App. A, note on rank truncation).
// Inputs: lamK (kB, descending, eigenvalues of M^T M), kB; mode: eps rule with
// delta2 (if delta2 < 0 it is set from this bond: delta2 = eps^2 ||X||^2/(d-1)),
// or forced rank (>0), and max_rank cap (<=0 none).
// Output (device int/double array `dec`): dec_i[0] = r', dec_i[1] = capped,
// dec_d[0] = delta2 used, dec_d[1] = discarded tail (sum sigma^2), dec_d[2] = ||X||^2.
// singular_values: lamK holds squared singular values from an SVD (resolved
// to kB eps_mach of the largest singular value) rather than Gram eigenvalues.
void truncation_decision(cudaStream_t s, const double* lamK, int kB, double eps, int dm1,
                         int forced, int max_rank, double* delta2_dev, int* dec_i,
                         double* dec_d, bool singular_values = false);
// Count of eigenvalues above the floor n * eps_mach * lam_max (lam descending).
void count_above_floor(cudaStream_t s, const double* lam, int n, int* out_dev);

// ---------------------------------------------------------------- physics (transport.cu)
struct Angular {
    int n_theta, n_phi;
    double* mu = nullptr;   // device, n_theta
    double* sint = nullptr; // device, n_theta
    double* cphi = nullptr; // device, n_phi
    double* sphi = nullptr; // device, n_phi
    // per-term angular factors of the transport terms [I, (x,1), (x,2), (y,1),
    // (y,2), (z,1), (z,2)]: tfac (terms x n_theta), pfac (terms x n_phi);
    // upwind and HLL: the masked direction cosines n_a^+, n_a^-; Rusanov: n_a
    // and 1 (Sec. 4.3)
    double* tfac = nullptr;
    double* pfac = nullptr;
    double w, v;            // quadrature weights (uniform)
};

// Fixed external sources S = sum_k x_k (x) theta_k (x) phi_k (device arrays:
// x n x N_c, th n x N_theta, ph n x N_phi, q n = the quadrature of each
// angular profile, sum_lp theta_k[l] phi_k[p] dOmega_lp); n = 0: none.
struct Sources {
    int n = 0;
    const double* x = nullptr;
    const double* th = nullptr;
    const double* ph = nullptr;
    const double* q = nullptr;
};

// Build the grown angular cores for the TT sum of transport (+ source) terms.
// nterms = 1 + 2 ndim if transport else 1; then one block per external source
// (ext.n of them, transport only), and source adds one unit block.
// dd (nullable): a captured step's size block (DYN_* slots); r1, r2, R1, R2
// are then the largest values, sizing the grids.
void build_grown_angular(cudaStream_t s, const Angular& ang, int ndim, bool transport,
                         bool source, int r1, int r2, const double* Th, const double* Ph,
                         double* Thg, double* Phg, int R1, int R2, const Sources& ext = Sources(),
                         const int* dd = nullptr);
// thbar[a] = sum_l w thfac_j[l] sum_b Th[a,l,b] phibar_j[b] for the grown core
// blocks (first nterms*r1 entries), phibar_j[b] = sum_p v phfac_j[p] Ph[b,p].
void grown_thbar(cudaStream_t s, const Angular& ang, int ndim, bool transport, int r1, int r2,
                 const double* Th, const double* Ph, double* thbar, const int* dd = nullptr);
// Plain quadrature vector of a 3-core TT: thbar[a] = sum_l w sum_b Th[a,l,b] sum_p v Ph[b,p].
void plain_thbar(cudaStream_t s, const Angular& ang, int r1, int r2, const double* Th,
                 const double* Ph, double* thbar, const int* dd = nullptr);

// Slots of a captured step's size block (ints in device memory): the ranks
// the device decides, read by the kernels of the step instead of host sizes.
enum : int {
    DYN_R1 = 0, DYN_R2 = 1,    // ranks of the TT entering the step
    DYN_G1 = 2, DYN_G2 = 3,    // grown ranks
    DYN_KB0 = 4, DYN_KB1 = 5,  // pivoted-Cholesky ranks of the right Grams
    DYN_DEC0 = 8,              // bond 0 decision: rank, capped, non-finite, spare
    DYN_DEC1 = 12,             // bond 1 decision
    DYN_SWEEPS = 16,           // Jacobi sweeps of the two eigensolves
    DYN_STICKY = 20,           // flags over a run of replays: 1 capped, 2 non-finite, 4 degenerate
    DYN_DESC = 24,             // product descriptors, 8 ints each
    DYN_NDESC = 20,
    DYN_INTS = DYN_DESC + 8 * DYN_NDESC
};

// Boundary rule of axis 0 of a spatial shard (tt_create_shard): the ghost
// layers are halo rows stored after the shard's own rows (the layer below
// the slab, then the layer above it).
enum : int { BC_HALO = 3 };

struct Grid {
    int ndim;
    int n[3];
    double dx[3];
    int bc[3];
    long nc;
};
struct Fields {
    double *sigma_a, *sigma_s, *cv, *T, *E_star;
    double c, a_r, dt;
    // interface flux (Sec. 3.1): the two terms of each axis are
    // -nu [w_L(i+1/2) X_i + w_R(i+1/2) X_{i+1} - w_L(i-1/2) X_{i-1} - w_R(i-1/2) X_i]
    // with face weights (w_L1, w_R1, w_L2, w_R2) = wc (upwind, Rusanov) or, for
    // HLL, per cell from fw (nc x ndim x 8: lo face w_L1 w_R1 w_L2 w_R2, then
    // the hi face); flux == TT_FLUX_UPWIND keeps the plain differences
    int flux = TT_FLUX_UPWIND;
    double wc[4] = {1.0, 0.0, 0.0, 1.0};
    const double* fw = nullptr;
};
// Fused transport + source row kernel (Sec. 4.3-4.4).  Writes Xg (nc x R1,
// ld = ldg): transport blocks then (if source) scaled by s_i and the emission
// column.  Computes E* (the post-transport energy) into fields.E_star when
// source is set, from the cells' term dots X_i . thbar_j (ydots: nc x nterms
// doubles of scratch).  thbar: grown quadrature vector (nterms*r1 entries).
// External sources (transport only) add columns nterms r1 + k = s_i c dt x_k[i]
// and c dt x_k[i] q_k / c to E*; the emission column follows them.
void transport_source_rows(cudaStream_t s, const Grid& g, const Fields& f, bool transport,
                           bool source, int r1, const double* X, long ldx, const double* thbar,
                           double* Xg, long ldg, double* ydots, const Sources& ext = Sources(),
                           const int* dd = nullptr);
// E_i = X_i . thbar / c (r entries); if update_T: T_i += (E*_i - E_i) / cv_i.
void energy_rows(cudaStream_t s, long nc, int r, const double* X, long ldx, const double* thbar,
                 double c, double* E_out, const double* E_star, const double* cv, double* T,
                 bool update_T, const int* dd = nullptr);
// ---------------------------------------------------------------- split-space layout (split.cu)
// One core of the grown TT in the split layout (cores x[, y[, z]], theta,
// phi): the K transport terms (K = 0: none) summed by Sec. 4.1's addition,
// plus the emission term's block (ekind, shape ea x n x eb) after them.
enum { SPLIT_SPATIAL = 0, SPLIT_THETA = 1, SPLIT_PHI = 2 };
// Spatial stencil of the two transport terms of each axis in the split layout
// (uniform opacities, so the flux's face weights are the same on every face):
// term t of axis a is c[a][t][0] X_i + c[a][t][1] X_{i+1} - c[a][t][2] X_{i-1}.
struct StencilCo {
    double c[3][2][3];
};
enum { SPLIT_E_NONE = 0, SPLIT_E_IDENT_COL = 1, SPLIT_E_IDENT_ROW = 2, SPLIT_E_ONES = 3,
       SPLIT_E_FIELD = 4 };
struct SplitCoreSpec {
    int kind, axis, bc;    // core kind; spatial axis and its boundary rule
    int first, last;       // position in the train
    int K;                 // transport terms
    int ra, n, rb;         // input core (ra x n x rb)
    int Ra, Rb;            // grown core
    int ekind;             // emission block kind (SPLIT_E_*)
    double tscale;         // factor on the transport blocks
    double co[2][3];       // stencil of this core's axis (spatial cores)
};
// fac: K x n per-term factors of an angular core (theta: -nu_a times the mask,
// phi: the mask; row 0 = ones).  G may be null when K = 0.
void split_grow_core(cudaStream_t s, const SplitCoreSpec& c, const double* G, const double* fac,
                     double* out);
// Per-cell source stage of the split layout: E*_i from the K spatial
// contractions F (nc x K, term-major columns: the identity term, then the
// upwind differences of the (a, +/-) terms taken here on F), T-dagger from the
// quartic, e_i written to eblk[c0 st0 + c1 st1 + c2 st2] (cell coordinates),
// E*_i to f.E_star.
void split_source_cells(cudaStream_t s, const Grid& g, const Fields& f, const StencilCo& co,
                        bool transport, int K, const double* F, double* eblk, long st0, long st1,
                        long st2);
// HLL face weights (Sec. 3.1, Eq. hll with the wave speeds after it and the
// optical depth of Eq. tauc) of every cell's two faces per axis into fw
// (nc x ndim x 8), from sigma_a + sigma_s (ghost opacity: the wrapped cell on
// periodic axes, the cell itself on vacuum faces).
void hll_face_weights(cudaStream_t s, const Grid& g, const double* sigma_a, const double* sigma_s,
                      double beta, double tau_threshold, double* fw);
// The same layout for Eq. rusanov_flux_toro with S+ = c |n_a| min(1, 1 / tau_c).
void rusanov_tau_face_weights(cudaStream_t s, const Grid& g, const double* sigma_a, const double* sigma_s,
                              double beta, double* fw);
// Inflow face (axis, side) of a vacuum axis as a fixed-source column: x[i] =
// w g[i] / dx_a on the face's layer of cells (0 elsewhere), w = +w_L(i-1/2) of
// term t on the low face, -w_R(i+1/2) on the high face, so that c dt x is the
// known ghost's contribution -nu (-w_L g) or -nu (w_R g) to the boundary cells.
void inflow_source(cudaStream_t s, const Grid& g, const Fields& f, int axis, int side, int term,
                   const double* gface, double* x);
// Isotropic initial intensity I = c a_r Tr^4 / 4 pi into X (nc x 1).
void init_isotropic(cudaStream_t s, long nc, const double* Tr, double c, double a_r, double* X);
// Adjoint form (reverse mode with the rounding's projections frozen).
void source_adjoint_rows(cudaStream_t s, const Grid& g, const Fields& f, int r1, const double* X,
                         long ldx, const double* thbar, const double* Tin, const double* Xgb,
                         long ldgb, const double* Esb_in, const double* Tb_out, double* ybar,
                         double* Y, long ldy, double* Esb_out, double* Tb_in, double* sigb);
void stencil_adjoint_rows(cudaStream_t s, const Grid& g, const Fields& f, int r1, const double* ybar,
                          long ldy, double* Xb, long ldxb);
void grown_angular_adjoint(cudaStream_t s, const Angular& ang, int ndim, int r1, int r2,
                           const double* Thgb, const double* Phgb, int R1, int R2, double* Thb,
                           double* Phb);
// Adds the adjoint of quadrature vectors thbar_j (j in [j0, nterms)) to Thb/Phb;
// scratch holds 2 * nterms * r2 doubles.
void thbar_adjoint(cudaStream_t s, const Angular& ang, int nterms, int j0, int r1, int r2,
                   const double* Th, const double* Ph, const double* thbb, double* scratch,
                   double* Thb, double* Phb);
void escape_rows(cudaStream_t s, const Grid& g, double dt, int r, const double* X, long ldx,
                 const double* thbar_terms, double* qcell, double* Xb, long ldxb, bool add_grad);
void escape_thbb(cudaStream_t s, const Grid& g, double dt, int r, const double* X, long ldx,
                 double* thbb);
void energy_adjoint_rows(cudaStream_t s, long nc, int r, const double* thbar, double c,
                         const double* cv, const double* Tb, double* Xb, long ldxb, double* e1b,
                         double* Esb);
void sum_into(cudaStream_t s, long n, const double* x, double* out);
// totals[0] = sum E, totals[1] = sum cv T (deterministic two-pass reduction).
void energy_totals(cudaStream_t s, long nc, const double* E, const double* cv, const double* T,
                   double* totals_dev, double* scratch /* >= 2*1024 doubles */);

}  // namespace ttsn
