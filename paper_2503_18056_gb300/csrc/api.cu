// Host runtime and C ABI of libttsn (declared in include/ttsn.h).
//
// The step (arXiv 2503.18056, Sec. 3-4) on one CUDA stream:
//   1. transport_source_rows: grown spatial core X* = [X | -nu D X ... | e]
//      (Sec. 4.3 TT sum + Sec. 4.4 source), grown angular cores, E*;
//   2. Gram-SVD rounding (Algorithm 1 with the App. A.2 truncation):
//      backward sweep of right Grams G_B, their eigendecompositions, then per
//      bond the left Gram G_A = A^T A, the rank decision and the core update;
//   3. energy_rows: E^{m+1} from the rounded TT and the energy-conserving
//      temperature update (Sec. 3.2).
//
// Rounding per bond.  App. A.2 forms M = S_A V_A^T V_B S_B from two
// eigendecompositions and takes the SVD of M.  Here the same quantities come
// from one eigendecomposition: with any factor W of G_B (W^T W = G_B; a
// pivoted Cholesky factor stopped at the floor n eps_mach max diag, or
// equivalently S_B V_B^T), K = W G_A W^T has the eigenvalues of M^T M, so
// eig(K) = V~ S~^2 V~^T gives the singular values of M and
//   A'    = A P_A,   P_A^T = S~_r^{-1} V~_r^T W,
//   M_upd = P_A^T G_A = A'^T A,
// which equal App. A.2's A V_A S_A^{-1} U~ and (V_B S_B^{-1} V~ S~)^T in exact
// arithmetic.  Neither S_A^{-1} nor S_B^{-1} is formed, so tensor components
// whose left singular values fall below sqrt(eps_mach) of the largest (where
// App. A.4 notes Gram eigenvalues lose their precision) are kept instead of
// being discarded with the floored eigenpairs of G_A.
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace ttsn {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};
static thread_local unsigned long long t_launches = 0;  // this thread's launches (capture counts)
void note_launch(unsigned n) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}
void set_error(const std::string& msg) { g_err = msg; }
const char* get_error() { return g_err.c_str(); }

static thread_local const tt_allocator* g_alloc = nullptr;
const tt_allocator* current_allocator() { return g_alloc; }
AllocScope::AllocScope(const tt_allocator* a) : prev(g_alloc) { g_alloc = a; }
AllocScope::~AllocScope() { g_alloc = prev; }

namespace {
// One device allocation through allocator a (null: the stream-ordered pool).
cudaError_t dev_alloc(const tt_allocator* a, double** out, size_t bytes, cudaStream_t s) {
    if (!a) return cudaMallocAsync((void**)out, bytes, s);
    *out = static_cast<double*>(a->alloc(a->ctx, bytes, (void*)s));
    return *out ? cudaSuccess : cudaErrorMemoryAllocation;
}
void dev_free(const tt_allocator* a, double* p, size_t bytes, cudaStream_t s, bool async) {
    if (!p) return;
    if (a) {
        a->free(a->ctx, p, bytes, (void*)s);
    } else if (async) {
        cudaFreeAsync(p, s);
    } else {
        cudaFree(p);
    }
}
}  // namespace

tt_status DevBuf::ensure(size_t n, cudaStream_t s, bool keep) {
    if (n <= cap) return TT_OK;
    // a recorded step must not allocate: an allocation inside a capture
    // becomes a graph node that the next replay cannot repeat
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        set_error("captured step: a buffer would have to grow inside the recording (" +
                  std::to_string(n * 8) + " bytes)");
        return TT_ERR_STATE;
    }
    if (!p) {  // the first allocation fixes the allocator this buffer uses
        alloc = current_allocator();
        astream = s;
    }
    size_t want = std::max(n, cap + cap / 2);
    double* np = nullptr;
    cudaError_t e = dev_alloc(alloc, &np, want * sizeof(double), s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        want = n;
        e = dev_alloc(alloc, &np, want * sizeof(double), s);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            set_error(std::string("device allocation of ") + std::to_string(want * 8) +
                      " bytes failed: " + cudaGetErrorString(e));
            return TT_ERR_OOM;
        }
    }
    if (keep && p && cap) TT_CUDA_TRY(cudaMemcpyAsync(np, p, cap * sizeof(double), cudaMemcpyDeviceToDevice, s));
    dev_free(alloc, p, cap * sizeof(double), s, true);
    p = np;
    cap = want;
    astream = s;
    return TT_OK;
}

tt_status ensure_max_dynamic_smem(const void* kernel) {
    static std::mutex mu;
    static std::vector<const void*> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const void* k : done)
        if (k == kernel) return TT_OK;
    int dev = 0, optin = 0;
    TT_CUDA_TRY(cudaGetDevice(&dev));
    TT_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    TT_CUDA_TRY(cudaFuncGetAttributes(&fa, kernel));
    TT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes));
    done.push_back(kernel);
    return TT_OK;
}

void DevBuf::release() {
    dev_free(alloc, p, cap * sizeof(double), astream, false);
    p = nullptr;
    cap = 0;
    alloc = nullptr;
}

}  // namespace ttsn

using namespace ttsn;

namespace ttsn {
struct PlanConsts {
    int nterms;   // 1 + 2 ndim
    int nt, np;   // n_theta, n_phi
    long nc;
};

__device__ __forceinline__ void put_desc(int* dd, int slot, int M, int N, int K, int lda, int ldb, int ldc) {
    int* d = dd + DYN_DESC + 8 * slot;
    d[0] = M;
    d[1] = N;
    d[2] = K;
    d[3] = lda;
    d[4] = ldb;
    d[5] = ldc;
}

// stage 0: step begins (grown ranks, backward sweep, bond 0 Gram); 1: right
// Grams factored (bond 0 products); 2: bond 0 decided (its update, bond 1
// Gram and products); 3: bond 1 decided (its update; the new ranks become the
// TT's).  A bond that meets a zero factor or a zero decision marks the step
// degenerate (slot DYN_DEC0 + 3), which the host reports after the replay.
__global__ void plan_kernel(int stage, int* dd, PlanConsts pc) {
    const int nt = pc.nt, np = pc.np;
    if (stage == 0) {
        const int G1 = pc.nterms * dd[DYN_R1] + 1, G2 = pc.nterms * dd[DYN_R2] + 1;
        dd[DYN_G1] = G1;
        dd[DYN_G2] = G2;
        dd[DYN_DEC0 + 3] = 0;
        put_desc(dd, 0, G2, G2, np, np, np, G2);                   // GB1 = Phi* Phi*^T
        put_desc(dd, 1, G1 * nt, G2, G2, G2, G2, G2);              // bwd = Theta* GB1
        put_desc(dd, 2, G1, G1, nt * G2, nt * G2, nt * G2, G1);    // GB0 = bwd Theta*^T
        put_desc(dd, 3, G1, G1, (int)pc.nc, G1, G1, G1);           // G_A of X*
    } else if (stage == 1) {
        const int G1 = dd[DYN_G1], G2 = dd[DYN_G2];
        const int k0 = max(dd[DYN_KB0], 0), k1 = max(dd[DYN_KB1], 0);
        if (k0 == 0 || k1 == 0) dd[DYN_DEC0 + 3] = 1;
        put_desc(dd, 4, G1, k0, G1, G1, G1, k0);                   // T1 = G_A W^T
        put_desc(dd, 5, k0, k0, G1, G1, k0, k0);                   // K = W T1
        (void)G2;
    } else if (stage == 2) {
        const int G1 = dd[DYN_G1], G2 = dd[DYN_G2];
        const int k0 = max(dd[DYN_KB0], 0), k1 = max(dd[DYN_KB1], 0);
        const int r = dd[DYN_DEC0];
        if (r == 0) dd[DYN_DEC0 + 3] = 1;
        put_desc(dd, 6, r, k0, k0, k0, 0, 0);                      // scale_rows rows, cols, ldi, ldo
        put_desc(dd, 7, r, G1, k0, k0, G1, G1);                    // P_A^T = S^-1 V^T W
        put_desc(dd, 8, r, G1, G1, G1, G1, G1);                    // M_upd = P_A^T G_A
        put_desc(dd, 9, (int)pc.nc, r, G1, G1, G1, r);             // X' = X* P_A
        put_desc(dd, 10, r, nt * G2, G1, G1, nt * G2, nt * G2);    // next = M_upd Theta*
        put_desc(dd, 11, G2, G2, r * nt, G2, G2, G2);              // G_A of the next core
        put_desc(dd, 12, G2, k1, G2, G2, G2, k1);
        put_desc(dd, 13, k1, k1, G2, G2, k1, k1);
    } else {
        const int G2 = dd[DYN_G2];
        const int k1 = max(dd[DYN_KB1], 0);
        const int r0 = dd[DYN_DEC0], r = dd[DYN_DEC1];
        if (r == 0) dd[DYN_DEC0 + 3] = 1;
        put_desc(dd, 14, r, k1, k1, k1, 0, 0);
        put_desc(dd, 15, r, G2, k1, k1, G2, G2);
        put_desc(dd, 16, r, G2, G2, G2, G2, G2);
        put_desc(dd, 17, r0 * nt, r, G2, G2, G2, r);
        put_desc(dd, 18, r, np, G2, G2, np, np);
        dd[DYN_R1] = r0;
        dd[DYN_R2] = r;
        // what the host reports after a run of replays: capped, non-finite, degenerate
        const int nonfinite = dd[DYN_DEC0 + 2] | dd[DYN_DEC1 + 2] | (dd[DYN_KB0] < 0) | (dd[DYN_KB1] < 0);
        dd[DYN_STICKY] |= (dd[DYN_DEC0 + 1] | dd[DYN_DEC1 + 1]) | (nonfinite << 1) | (dd[DYN_DEC0 + 3] << 2);
    }
}

}  // namespace ttsn

// host-side slots of the pinned readback block
enum { HI_KB = 0, HI_DEC = 16, HI_STATUS = 20, HI_SWEEPS = 24, HI_N = 64 };
enum { HD_DEC = 0, HD_DELTA2 = 4, HD_TOT = 8, HD_Q = 12, HD_ONE = 14, HD_JWC = 15, HD_N = 16 };

struct tt_ctx {
    cudaStream_t stream = nullptr;
    bool physics = false;
    int d = 0;
    int n[TT_MAX_D] = {0};
    int r[TT_MAX_D + 1] = {0};
    DevBuf core[TT_MAX_D];
    DevBuf gcore[TT_MAX_D];
    int gr[TT_MAX_D + 1] = {0};

    // rounding workspace
    DevBuf GB[TT_MAX_D], lamB[TT_MAX_D], VtB[TT_MAX_D];
    DevBuf GA, Wc, T1, K, lamK, VtK, Vts, PAt, Mupd, tmp[2], partials, bwd, slscratch, erowA;
    int precision = TT_FP64;
    EigWork eig;
    DevBuf small_buf;          // holds d_dbl then d_int
    int* d_int = nullptr;      // device ints (HI_* layout)
    double* d_dbl = nullptr;   // device doubles (HD_* layout)
    int* h_int = nullptr;      // pinned host mirror
    double* h_dbl = nullptr;
    int sweeps_slot = 0;
    int max_sweeps = JACOBI_MAX_SWEEPS;  // Jacobi sweep limit (tt_set_max_sweeps)

    // phase profiler (CUDA events on the handle's stream)
    struct PhaseAcc {
        double ms = 0, flops = 0, bytes = 0;
        long long launches = 0, calls = 0;
    };
    struct Pending {
        int phase;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    PhaseAcc ph[TT_NPHASES];
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;

    // adjoint tape: one record per taped step.  Checkpoint records hold the
    // step's input state (X, Theta, Phi, T); with a checkpoint interval of one
    // every record also holds the frozen rounding factors (P_A^T and M_upd of
    // each bond), otherwise the reverse sweep re-runs each segment from its
    // checkpoint to refill them before applying the transposed operations.
    struct StepRec {
        int r1 = 0, r2 = 0, R1 = 0, R2 = 0, o1 = 0, o2 = 0;
        bool state = false, proj = false;
        DevBuf X, Th, Ph, T, P[2], M[2];
        void release_state() {
            X.release();
            Th.release();
            Ph.release();
            T.release();
            state = false;
        }
        void release_proj() {
            for (int k = 0; k < 2; ++k) {
                P[k].release();
                M[k].release();
            }
            proj = false;
        }
        void release() {
            release_state();
            release_proj();
        }
    };
    bool taping = false;               // steps append records
    int tape_every = 1;                // checkpoint interval in steps
    std::vector<StepRec*> tape;
    StepRec* replay_rec = nullptr;     // record a replayed step refills
    StepRec* cur_rec = nullptr;        // record the running step fills
    bool rec_state = false, rec_proj = false;
    // reverse-sweep workspace
    DevBuf aXb, aXbi, aThb, aThbi, aPhb, aPhbi, aTb, aTbi, aXgb, aThgb, aPhgb, aThtb, aybar, aY,
        aEsb, aEsbo, ae1b, asigb, athbb, ascr, atb1, atb2, aq, agv;

    // physics
    Grid grid{};
    Angular ang{};
    Fields fields{};
    DevBuf f_sigma_a, f_sigma_s, f_cv, f_T, f_Estar, f_E, thbar, red, ang_buf;
    DevBuf ydots;  // the cells' term dots X_i . thbar_j of the source stage
    DevBuf src_x, src_th, src_ph, src_q;  // fixed external sources (all kinds)
    int nsrc = 0;
    // the caller's own sources (tt_set_sources) and the inflow faces
    // (tt_set_inflow); src_* holds the user sources followed by the inflow
    // faces' rank-one terms
    DevBuf usr_x, usr_th, usr_ph;
    int nusr = 0;
    struct InflowFace {
        bool on = false;
        DevBuf g;
        std::vector<double> th, ph;
    } inflow[3][2];
    std::vector<double> h_tfac, h_pfac;  // host copies of the angular factor tables
    // randomized rounding (App. A.3): the caller's Gaussian sketch TT (cores
    // (L_{k-1}, n_k, L_k)), its leading blocks at a rounding's target ranks,
    // the right sketches W_k and the orthonormalisation workspace
    int round_method = TT_ROUND_GRAM;
    int eig_method = TT_EIG_ONE_SIDED;  // eigensolver of the rounding's K
    DevBuf sketch[TT_MAX_D], sk_sub[TT_MAX_D], sk_W[TT_MAX_D], sk_Y, sk_Q, sk_G, sk_lam, sk_Vt, sk_Vs;
    int sk_L[TT_MAX_D + 1] = {0};
    bool has_sketch = false;
    // QR-based rounding (TT-SVD, App. A.1): the right-orthonormalised cores,
    // the two basis buffers of the Cholesky-QR passes, the transposed core,
    // the small factor, its Jordan-Wielandt matrix and eigenpairs, U and S V^T
    DevBuf ts_core[TT_MAX_D], ts_Qa, ts_Qb, ts_Y, ts_R, ts_J, ts_lam, ts_Vt, ts_U, ts_M;
    // split-space layout (cores x[, y[, z]], theta, phi): per-term angular
    // factors (theta rows then phi rows, 1 + 2 ndim terms each), the uniform
    // absorption factor s, the spatial contractions F (nc x terms) and the
    // contraction chain's intermediates
    int layout = TT_LAYOUT_GROUPED;
    DevBuf split_fac, sp_F, sp_tmp[2];
    StencilCo split_co{};  // the flux's stencil per axis (uniform opacities)
    DevBuf f_fw;           // HLL face weights (grouped layout)
    double split_s = 1.0;
    bool split() const { return layout == TT_LAYOUT_SPLIT; }
    bool has_sigma_s = false;
    double eps = 0.0;
    int max_rank = 0;
    int rounds = 1;
    // caller's device allocator (tt_create_ex), copied; every buffer of the
    // handle comes from it when has_allocator is set
    tt_allocator allocator{};
    bool has_allocator = false;
    // spatial shard (tt_create_shard): layers [p0, p1) of axis 0 out of n0,
    // axis 0's global rule bc0, cells per layer, the caller's exchange; xch
    // holds the four exchange blocks (the ghost layers themselves follow the
    // own rows of core[0])
    // captured step (tt_set_graph): the step's launches recorded once into a
    // CUDA graph whose kernels read the device-decided sizes from dyn
    // (DYN_* slots), replayed every step without a host synchronisation
    bool graph_on = false;
    cudaGraphExec_t graph_exec = nullptr;
    unsigned graph_launches = 0;       // library kernels one replay runs
    bool ranks_stale = false;          // h->r lags the device after replays
    int cap1 = 0, cap2 = 0;            // rank caps of the two bonds
    DevBuf dyn_buf, dyn_part;          // size block (ints) and product partials
    int* dyn = nullptr;
    int* h_dyn = nullptr;              // pinned mirror, refreshed by every replay
    double* h_dyn_dec = nullptr;       // pinned decisions of the two bonds (8 doubles)
    struct Shard {
        bool on = false;
        int p0 = 0, p1 = 0, n0 = 0, bc0 = TT_BC_PERIODIC;
        long plane = 1;
        tt_exchange_fn fn = nullptr;
        void* ctx = nullptr;
    } shard;
    DevBuf xch;
    const tt_allocator* alloc_ptr() const { return has_allocator ? &allocator : nullptr; }
    double dV = 1.0;

    tt_status init_common(cudaStream_t s) {
        stream = s;
        // keep freed stream-ordered blocks cached in the device pool so capacity
        // growth does not return memory to the OS between steps
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        (void)cudaGetLastError();
        TT_TRY(small_buf.ensure((size_t)HD_N + (HI_N * sizeof(int) + 7) / 8, s));
        d_dbl = small_buf.p;
        d_int = reinterpret_cast<int*>(small_buf.p + HD_N);
        TT_CUDA_TRY(cudaMallocHost(&h_int, HI_N * sizeof(int)));
        TT_CUDA_TRY(cudaMallocHost(&h_dbl, HD_N * sizeof(double)));
        TT_CUDA_TRY(cudaMemsetAsync(d_int, 0, HI_N * sizeof(int), s));
        fill(s, d_dbl + HD_ONE, 1, 1.0);
        return TT_OK;
    }
    ~tt_ctx() {
        if (stream) cudaStreamSynchronize(stream);
        for (int k = 0; k < TT_MAX_D; ++k) {
            sketch[k].release();
            sk_sub[k].release();
            sk_W[k].release();
            ts_core[k].release();
            core[k].release();
            gcore[k].release();
            GB[k].release();
            lamB[k].release();
            VtB[k].release();
        }
        DevBuf* bufs[] = {&slscratch, &erowA, &GA, &Wc, &T1, &K, &lamK, &VtK, &Vts, &PAt, &Mupd, &tmp[0], &tmp[1],
                          &partials, &bwd, &f_sigma_a, &f_sigma_s, &f_cv, &f_T, &f_Estar, &f_E,
                          &thbar, &red, &ang_buf, &src_x, &src_th, &src_ph, &src_q,
                          &split_fac, &sp_F, &sp_tmp[0], &sp_tmp[1], &f_fw, &usr_x, &usr_th, &usr_ph,
                          &sk_Y, &sk_Q, &sk_G, &sk_lam, &sk_Vt, &sk_Vs, &xch, &dyn_buf, &dyn_part, &ydots,
                          &ts_Qa, &ts_Qb, &ts_Y, &ts_R, &ts_J, &ts_lam, &ts_Vt, &ts_U, &ts_M};
        for (DevBuf* b : bufs) b->release();
        for (auto& ax : inflow)
            for (auto& face : ax) face.g.release();
        eig.release();
        for (StepRec* r : tape) {
            r->release();
            delete r;
        }
        DevBuf* abufs[] = {&aXb, &aXbi, &aThb, &aThbi, &aPhb, &aPhbi, &aTb, &aTbi, &aXgb, &aThgb,
                           &aPhgb, &aThtb, &aybar, &aY, &aEsb, &aEsbo, &ae1b, &asigb, &athbb,
                           &ascr, &atb1, &atb2, &aq, &agv};
        for (DevBuf* b : abufs) b->release();
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : ev_pool) cudaEventDestroy(e);
        small_buf.release();
        if (h_int) cudaFreeHost(h_int);
        if (h_dbl) cudaFreeHost(h_dbl);
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (h_dyn) cudaFreeHost(h_dyn);
        if (h_dyn_dec) cudaFreeHost(h_dyn_dec);
    }
    size_t core_len(int k, const int* rr) const { return (size_t)rr[k] * n[k] * rr[k + 1]; }
};

namespace {

tt_status fail(tt_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

cudaEvent_t get_event(tt_ctx* h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// NVTX range names of the phases (TT_PH_* order): profilers attribute the
// kernels a phase launches to its range (e.g. ncu --nvtx --nvtx-include
// "gram_left/").  Without a profiler attached the push/pop calls return at once.
const char* const kPhaseNames[TT_NPHASES] = {"transport", "gram_right", "eig", "gram_left",
                                              "small", "update", "energy"};

// Brackets one phase occurrence with an NVTX range and, when profiling is on,
// with events; the algorithmic flops/bytes and the library launches in
// between are accumulated.
struct PhaseScope {
    tt_ctx* h;
    int phase;
    cudaEvent_t a = nullptr;
    unsigned long long l0;
    PhaseScope(tt_ctx* hh, int p, double flops, double bytes) : h(hh), phase(p) {
        nvtxRangePushA(kPhaseNames[p]);
        l0 = g_launches.load(std::memory_order_relaxed);
        if (!h->prof_on) return;
        a = get_event(h);
        cudaEventRecord(a, h->stream);
        h->ph[p].flops += flops;
        h->ph[p].bytes += bytes;
        h->ph[p].calls += 1;
    }
    ~PhaseScope() {
        if (h->prof_on && a) {
            cudaEvent_t b = get_event(h);
            cudaEventRecord(b, h->stream);
            h->ph[phase].launches += (long long)(g_launches.load(std::memory_order_relaxed) - l0);
            h->pending.push_back({phase, a, b});
        }
        nvtxRangePop();
    }
};

// Resolve finished event pairs (call after a stream synchronisation).
void resolve_profile(tt_ctx* h) {
    for (auto& p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->ph[p.phase].ms += ms;
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    h->pending.clear();
    (void)cudaGetLastError();
}

tt_status read_status(tt_ctx* h) {
    TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_STATUS, h->d_int + HI_STATUS, sizeof(int),
                                cudaMemcpyDeviceToHost, h->stream));
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    resolve_profile(h);
    const int st = h->h_int[HI_STATUS];
    if (st) TT_CUDA_TRY(cudaMemsetAsync(h->d_int + HI_STATUS, 0, sizeof(int), h->stream));
    if (st & DEV_TIMEOUT) return fail(TT_ERR_TIMEOUT, "device: a bounded grid barrier wait ran out");
    if (st & DEV_NOT_CONVERGED)
        return fail(TT_ERR_NOT_CONVERGED, "device: Jacobi eigensolver reached its sweep limit");
    return TT_OK;
}

int next_sweep_slot(tt_ctx* h) {
    const int slot = HI_SWEEPS + (h->sweeps_slot % (HI_N - HI_SWEEPS));
    h->sweeps_slot++;
    return slot;
}

// Set dst to a rank-one zero TT (the rounding of a zero tensor).
tt_status zero_tt(tt_ctx* h, DevBuf* dst, int* rr) {
    for (int k = 0; k < h->d; ++k) {
        TT_TRY(dst[k].ensure((size_t)h->n[k], h->stream));
        fill(h->stream, dst[k].p, (size_t)h->n[k], 0.0);
        rr[k] = 1;
    }
    rr[0] = rr[h->d] = 1;
    return TT_OK;
}

// Algorithm 1 (App. A) with the Gram truncation.  Reads cores src[k] with ranks
// R[0..d]; writes the rounded cores into dst (h->core) with ranks rr.
// Orthonormal basis of the columns of Y (m x l, row-major) into Q (m x k, k <=
// l): eigendecomposition of the Gram matrix Y^T Y, Q = Y V diag(lambda)^(-1/2)
// on the eigenpairs above the floor l eps_mach lambda_max; returns k (host).
tt_status eig_orthonormalise(tt_ctx* h, long m, int l, const double* Y, DevBuf& Q, int* k_out) {
    cudaStream_t s = h->stream;
    TT_TRY(h->sk_G.ensure((size_t)l * l, s));
    TT_TRY(h->sk_lam.ensure((size_t)l, s));
    TT_TRY(h->sk_Vt.ensure((size_t)l * l, s));
    TT_TRY(h->sk_Vs.ensure((size_t)l * l, s));
    TT_TRY(gram(s, (int)m, l, Y, l, h->sk_G.p, l, h->partials));
    // Y^T Y is positive semidefinite: the handle's eigensolver for such matrices
    if (h->eig_method == TT_EIG_ONE_SIDED)
        TT_TRY(syev_psd(s, l, h->sk_G.p, l, h->sk_lam.p, h->sk_Vt.p, l, h->eig, h->d_int + HI_STATUS,
                        h->d_int + next_sweep_slot(h), h->max_sweeps));
    else
        TT_TRY(syev(s, l, h->sk_G.p, l, h->sk_lam.p, h->sk_Vt.p, l, h->eig, h->d_int + HI_STATUS,
                    h->d_int + next_sweep_slot(h), h->max_sweeps));
    count_above_floor(s, h->sk_lam.p, l, h->d_int + HI_DEC);
    TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_DEC, h->d_int + HI_DEC, sizeof(int), cudaMemcpyDeviceToHost, s));
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    const int k = h->h_int[HI_DEC];
    *k_out = k;
    if (k == 0) return TT_OK;
    scale_rows(s, k, l, h->sk_Vt.p, l, h->sk_lam.p, 2, h->sk_Vs.p, l);  // rows v_j / sqrt(lambda_j)
    TT_TRY(Q.ensure((size_t)m * k, s));
    TT_TRY(dgemm(s, false, true, (int)m, k, l, 1.0, Y, l, h->sk_Vs.p, l, 0.0, Q.p, k));
    return TT_OK;
}

// Randomized rounding (App. A.3): backward sweep W_b = B_b^T Omega (the right
// part of bond b contracted with the sketch's leading blocks), then per bond
// A' = Q with Q an orthonormal basis of A W_b (eig-based Cholesky-QR applied
// twice, so that the basis is orthonormal to rounding for condition numbers
// up to ~1/sqrt(eps_mach)), M_upd = Q^T A, next core = M_upd x_1 G_{b+1}.
// Target ranks: forced[b] if given, else the sketch's rank, capped by both.
tt_status round_randomized(tt_ctx* h, DevBuf* src, const int* R, DevBuf* dst, int* rr,
                           const int* forced, tt_step_info* info) {
    cudaStream_t s = h->stream;
    const int d = h->d;
    const int* n = h->n;
    if (!h->has_sketch) return fail(TT_ERR_STATE, "randomized rounding: no sketch set (tt_set_sketch)");
    h->sweeps_slot = 0;
    TT_CUDA_TRY(cudaMemsetAsync(h->d_int + HI_SWEEPS, 0, (HI_N - HI_SWEEPS) * sizeof(int), s));
    if (info) {
        info->d = d;
        for (int k = 0; k <= d; ++k) info->grown[k] = R[k];
        info->capped = 0;
        info->norm = 0.0;
        for (int k = 0; k < TT_MAX_D; ++k) info->discarded[k] = 0.0;
    }
    int l[TT_MAX_D + 1];
    l[0] = l[d] = 1;
    for (int b = 0; b < d - 1; ++b) {
        int t = forced ? forced[b] : h->sk_L[b + 1];
        l[b + 1] = std::max(1, std::min(t, std::min(h->sk_L[b + 1], R[b + 1])));
    }
    // leading blocks of the sketch cores at the target ranks
    for (int k = 0; k < d; ++k) {
        TT_TRY(h->sk_sub[k].ensure((size_t)l[k] * n[k] * l[k + 1], s));
        copy2d(s, l[k] * n[k], l[k + 1], h->sketch[k].p, h->sk_L[k + 1], h->sk_sub[k].p, l[k + 1]);
    }
    {
        double fl = 2.0 * R[d - 1] * (double)n[d - 1] * l[d - 1];
        for (int c = d - 2; c >= 1; --c)
            fl += 2.0 * R[c] * (double)n[c] * R[c + 1] * l[c + 1] + 2.0 * R[c] * (double)n[c] * l[c + 1] * l[c];
        PhaseScope ps(h, TT_PH_GRAM_RIGHT, fl, 0.0);
        TT_TRY(h->sk_W[d - 2].ensure((size_t)R[d - 1] * l[d - 1], s));
        TT_TRY(dgemm_sk(s, false, true, R[d - 1], l[d - 1], n[d - 1], 1.0, src[d - 1].p, n[d - 1],
                        h->sk_sub[d - 1].p, n[d - 1], h->sk_W[d - 2].p, l[d - 1], h->partials));
        for (int c = d - 2; c >= 1; --c) {
            // T = G_c W_c (R_c n_c x l_{c+1}); W_{c-1} = T (R_c x n_c l_{c+1}) Omega_c^T
            TT_TRY(h->bwd.ensure((size_t)R[c] * n[c] * l[c + 1], s));
            TT_TRY(dgemm(s, false, false, R[c] * n[c], l[c + 1], R[c + 1], 1.0, src[c].p, R[c + 1],
                         h->sk_W[c].p, l[c + 1], 0.0, h->bwd.p, l[c + 1]));
            TT_TRY(h->sk_W[c - 1].ensure((size_t)R[c] * l[c], s));
            TT_TRY(dgemm_sk(s, false, true, R[c], l[c], n[c] * l[c + 1], 1.0, h->bwd.p, (long)n[c] * l[c + 1],
                            h->sk_sub[c].p, (long)n[c] * l[c + 1], h->sk_W[c - 1].p, l[c], h->partials));
        }
    }
    rr[0] = 1;
    const double* A = src[0].p;
    int rprev = 1, tmp_idx = 0;
    for (int b = 0; b <= d - 2; ++b) {
        const int Rk = R[b + 1], lb = l[b + 1];
        const long m = (long)rprev * n[b];
        // sketch Y = A W_b and its orthonormal basis
        TT_TRY(h->sk_Y.ensure((size_t)m * lb, s));
        {
            PhaseScope ps(h, TT_PH_GRAM_LEFT, 2.0 * m * (double)Rk * lb + 2.0 * m * (double)lb * lb, 0.0);
            TT_TRY(dgemm(s, false, false, (int)m, lb, Rk, 1.0, A, Rk, h->sk_W[b].p, lb, 0.0, h->sk_Y.p, lb));
        }
        int k1 = 0, k2 = 0;
        {
            PhaseScope ps(h, TT_PH_EIG, 4.0 * m * (double)lb * lb, 0.0);
            TT_TRY(eig_orthonormalise(h, m, lb, h->sk_Y.p, h->sk_Q, &k1));
            if (k1 == 0) return zero_tt(h, dst, rr);
            TT_TRY(eig_orthonormalise(h, m, k1, h->sk_Q.p, dst[b], &k2));
            if (k2 == 0) return zero_tt(h, dst, rr);
        }
        const int rk = k2;
        const long ncols = (long)n[b + 1] * R[b + 2];
        double* next;
        if (b == d - 2) {
            TT_TRY(dst[d - 1].ensure((size_t)rk * ncols, s));
            next = dst[d - 1].p;
        } else {
            TT_TRY(h->tmp[tmp_idx].ensure((size_t)rk * ncols, s));
            next = h->tmp[tmp_idx].p;
            tmp_idx ^= 1;
        }
        {
            PhaseScope ps(h, TT_PH_UPDATE, 2.0 * m * (double)rk * Rk + 2.0 * rk * (double)Rk * ncols, 0.0);
            // M_upd = Q^T A (rk x Rk), then the next core M_upd x_1 G_{b+1}
            TT_TRY(h->Mupd.ensure((size_t)rk * Rk, s));
            TT_TRY(dgemm_sk(s, true, false, rk, Rk, (int)m, 1.0, dst[b].p, rk, A, Rk, h->Mupd.p, Rk,
                            h->partials));
            TT_TRY(dgemm_sk(s, false, false, rk, (int)ncols, Rk, 1.0, h->Mupd.p, Rk, src[b + 1].p, ncols,
                            next, ncols, h->partials));
        }
        rr[b + 1] = rk;
        A = next;
        rprev = rk;
    }
    rr[d] = 1;
    if (info) {
        const int nslots = std::min(h->sweeps_slot, HI_N - HI_SWEEPS);
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_SWEEPS, h->d_int + HI_SWEEPS, nslots * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        int mx = 0;
        for (int i = 0; i < nslots; ++i) mx = std::max(mx, h->h_int[HI_SWEEPS + i]);
        info->sweeps = mx;
    }
    return TT_OK;
}

// Orthonormal basis Q (m x k) of the columns of Y (m x l, row-major) by three
// passes of eigen-form Cholesky QR: the first with the shift of
// shifted_scale_rows (no eigenvalue is inverted, whatever the condition of
// Y), the next two with the eigenvalue floor of eig_orthonormalise.  The
// basis ends in *Q (one of ts_Qa / ts_Qb, never Y's buffer); k = 0 for a zero Y.
tt_status orth_qr3(tt_ctx* h, long m, int l, const double* Y, DevBuf** Q, int* k_out) {
    cudaStream_t s = h->stream;
    TT_TRY(h->sk_G.ensure((size_t)l * l, s));
    TT_TRY(h->sk_lam.ensure((size_t)l, s));
    TT_TRY(h->sk_Vt.ensure((size_t)l * l, s));
    TT_TRY(h->sk_Vs.ensure((size_t)l * l, s));
    TT_TRY(gram(s, (int)m, l, Y, l, h->sk_G.p, l, h->partials));
    TT_TRY(syev(s, l, h->sk_G.p, l, h->sk_lam.p, h->sk_Vt.p, l, h->eig, h->d_int + HI_STATUS,
                h->d_int + next_sweep_slot(h), h->max_sweeps));
    shifted_scale_rows(s, l, h->sk_Vt.p, l, h->sk_lam.p, h->sk_Vs.p, l);
    TT_TRY(h->ts_Qa.ensure((size_t)m * l, s));
    TT_TRY(dgemm(s, false, true, (int)m, l, l, 1.0, Y, l, h->sk_Vs.p, l, 0.0, h->ts_Qa.p, l));
    int k2 = 0, k3 = 0;
    TT_TRY(eig_orthonormalise(h, m, l, h->ts_Qa.p, h->ts_Qb, &k2));
    if (k2 == 0) {
        *k_out = 0;
        return TT_OK;
    }
    TT_TRY(eig_orthonormalise(h, m, k2, h->ts_Qb.p, h->ts_Qa, &k3));
    *Q = &h->ts_Qa;
    *k_out = k3;
    return TT_OK;
}

// TT-SVD rounding (App. A.1; Oseledets 2011): a backward sweep makes cores
// d-1 .. 1 right-orthonormal (C_k^T = Q Rf: core k <- Q^T, core k-1 <- core
// k-1 Rf^T), then a forward sweep takes each left unfolding A = Q Rf, the SVD
// Rf = U S V^T from the Jordan-Wielandt eigenproblem, keeps r singular
// triplets by the tolerance rule of the Gram path (the same decision kernel
// on sigma^2), writes A' = Q U_r and carries S_r V_r^T into the next core.
// No Gram matrix of a core is factorised without the QR passes around it, so
// singular values are resolved to eps_mach of the largest (App. A.4).  FP64.
tt_status round_ttsvd(tt_ctx* h, DevBuf* src, const int* R, DevBuf* dst, int* rr, double eps, int max_rank,
                      const int* forced, tt_step_info* info) {
    cudaStream_t s = h->stream;
    const int d = h->d;
    const int* n = h->n;
    h->sweeps_slot = 0;
    TT_CUDA_TRY(cudaMemsetAsync(h->d_int + HI_SWEEPS, 0, (HI_N - HI_SWEEPS) * sizeof(int), s));
    if (info) {
        info->d = d;
        for (int k = 0; k <= d; ++k) info->grown[k] = R[k];
        info->capped = 0;
        info->norm = 0.0;
        for (int k = 0; k < TT_MAX_D; ++k) info->discarded[k] = 0.0;
    }
    int Rb[TT_MAX_D + 1];
    for (int k = 0; k <= d; ++k) Rb[k] = R[k];
    // ---- backward sweep: right-orthonormalise cores d-1 .. 1
    {
        PhaseScope ps(h, TT_PH_GRAM_RIGHT, 0.0, 0.0);
        for (int k = d - 1; k >= 1; --k) {
            const double* C = (k == d - 1) ? src[k].p : h->ts_core[k].p;
            const int rows = Rb[k];
            const long ncols = (long)n[k] * Rb[k + 1];
            TT_TRY(h->ts_Y.ensure((size_t)ncols * rows, s));
            transpose(s, rows, ncols, C, ncols, h->ts_Y.p, rows);
            DevBuf* Q = nullptr;
            int q = 0;
            TT_TRY(orth_qr3(h, ncols, rows, h->ts_Y.p, &Q, &q));
            if (q == 0) return zero_tt(h, dst, rr);
            TT_TRY(h->ts_R.ensure((size_t)q * rows, s));
            TT_TRY(dgemm_sk(s, true, false, q, rows, (int)ncols, 1.0, Q->p, q, h->ts_Y.p, rows, h->ts_R.p, rows,
                            h->partials));
            TT_TRY(h->ts_core[k].ensure((size_t)q * ncols, s));
            transpose(s, ncols, q, Q->p, q, h->ts_core[k].p, ncols);
            const long prow = (long)Rb[k - 1] * n[k - 1];
            TT_TRY(h->ts_core[k - 1].ensure((size_t)prow * q, s));
            TT_TRY(dgemm(s, false, true, (int)prow, q, rows, 1.0, src[k - 1].p, rows, h->ts_R.p, rows, 0.0,
                         h->ts_core[k - 1].p, q));
            Rb[k] = q;
        }
    }
    // ---- forward sweep: truncated SVDs of the left unfoldings
    h->h_dbl[HD_DELTA2] = -1.0;
    TT_CUDA_TRY(cudaMemcpyAsync(h->d_dbl + HD_DELTA2, h->h_dbl + HD_DELTA2, sizeof(double),
                                cudaMemcpyHostToDevice, s));
    rr[0] = 1;
    const double* A = h->ts_core[0].p;
    int rprev = 1, tmp_idx = 0;
    bool any_capped = false;
    for (int k = 0; k <= d - 2; ++k) {
        const int l = Rb[k + 1];
        const long m = (long)rprev * n[k];
        DevBuf* Q = nullptr;
        int q = 0;
        {
            PhaseScope ps(h, TT_PH_GRAM_LEFT, 0.0, 0.0);
            TT_TRY(orth_qr3(h, m, l, A, &Q, &q));
            if (q == 0) return zero_tt(h, dst, rr);
            TT_TRY(h->ts_R.ensure((size_t)q * l, s));
            TT_TRY(dgemm_sk(s, true, false, q, l, (int)m, 1.0, Q->p, q, A, l, h->ts_R.p, l, h->partials));
        }
        const int p = q + l, pm = std::min(q, l);
        {
            PhaseScope ps(h, TT_PH_EIG, 0.0, 0.0);
            TT_TRY(h->ts_J.ensure((size_t)p * p, s));
            TT_TRY(h->ts_lam.ensure((size_t)p, s));
            TT_TRY(h->ts_Vt.ensure((size_t)p * p, s));
            TT_TRY(h->lamK.ensure((size_t)pm, s));
            jw_build(s, q, l, h->ts_R.p, h->d_dbl + HD_JWC, h->ts_J.p);
            TT_TRY(syev(s, p, h->ts_J.p, p, h->ts_lam.p, h->ts_Vt.p, p, h->eig, h->d_int + HI_STATUS,
                        h->d_int + next_sweep_slot(h), h->max_sweeps));
            jw_sigma2(s, pm, h->ts_lam.p, h->d_dbl + HD_JWC, h->lamK.p);
            const int fk = forced ? forced[k] : 0;
            truncation_decision(s, h->lamK.p, pm, eps, d - 1, fk, max_rank, h->d_dbl + HD_DELTA2,
                                h->d_int + HI_DEC, h->d_dbl + HD_DEC, /*singular_values=*/true);
        }
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_DEC, h->d_int + HI_DEC, 4 * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_dbl + HD_DEC, h->d_dbl + HD_DEC, 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        if (h->h_int[HI_DEC + 2])
            return fail(TT_ERR_NONFINITE, "rounding: the tensor holds Inf or NaN (the run diverged or a field "
                                          "held one); restore saved cores and T before stepping again");
        const int rk = h->h_int[HI_DEC];
        if (h->h_int[HI_DEC + 1]) any_capped = true;
        if (info) {
            info->discarded[k] = sqrt(std::max(h->h_dbl[HD_DEC + 1], 0.0));
            if (k == 0) info->norm = sqrt(std::max(h->h_dbl[HD_DEC + 2], 0.0));
        }
        if (rk == 0) return zero_tt(h, dst, rr);
        const long ncols = (long)n[k + 1] * Rb[k + 2];
        double* next;
        {
            PhaseScope ps(h, TT_PH_UPDATE, 0.0, 0.0);
            TT_TRY(h->ts_U.ensure((size_t)rk * q, s));
            TT_TRY(h->ts_M.ensure((size_t)rk * l, s));
            jw_split(s, rk, q, l, h->ts_lam.p, h->d_dbl + HD_JWC, h->ts_Vt.p, p, h->ts_U.p, h->ts_M.p);
            // A' = Q U_r
            TT_TRY(dst[k].ensure((size_t)m * rk, s));
            TT_TRY(dgemm(s, false, true, (int)m, rk, q, 1.0, Q->p, q, h->ts_U.p, q, 0.0, dst[k].p, rk));
            // next core = S_r V_r^T x_1 (right-orthonormal core k+1)
            if (k == d - 2) {
                TT_TRY(dst[d - 1].ensure((size_t)rk * ncols, s));
                next = dst[d - 1].p;
            } else {
                TT_TRY(h->tmp[tmp_idx].ensure((size_t)rk * ncols, s));
                next = h->tmp[tmp_idx].p;
                tmp_idx ^= 1;
            }
            TT_TRY(dgemm_sk(s, false, false, rk, (int)ncols, l, 1.0, h->ts_M.p, l, h->ts_core[k + 1].p, ncols,
                            next, ncols, h->partials));
        }
        rr[k + 1] = rk;
        A = next;
        rprev = rk;
    }
    rr[d] = 1;
    if (info) {
        info->capped = any_capped ? 1 : 0;
        const int nslots = std::min(h->sweeps_slot, HI_N - HI_SWEEPS);
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_SWEEPS, h->d_int + HI_SWEEPS, nslots * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        int mx = 0;
        for (int i = 0; i < nslots; ++i) mx = std::max(mx, h->h_int[HI_SWEEPS + i]);
        info->sweeps = mx;
    }
    return any_capped ? TT_WARN_RANK_CAPPED : TT_OK;
}

tt_status shard_exchange(tt_ctx* h, int kind, double* buf, size_t count);

tt_status round_cores(tt_ctx* h, DevBuf* src, const int* R, DevBuf* dst, int* rr, double eps,
                      int max_rank, const int* forced, tt_step_info* info) {
    if (h->round_method == TT_ROUND_RANDOMIZED && h->d > 1)
        return round_randomized(h, src, R, dst, rr, forced, info);
    if (h->round_method == TT_ROUND_TTSVD && h->d > 1)
        return round_ttsvd(h, src, R, dst, rr, eps, max_rank, forced, info);
    cudaStream_t s = h->stream;
    const int d = h->d;
    const int* n = h->n;
    h->sweeps_slot = 0;
    TT_CUDA_TRY(cudaMemsetAsync(h->d_int + HI_SWEEPS, 0, (HI_N - HI_SWEEPS) * sizeof(int), s));
    if (info) {
        info->d = d;
        for (int k = 0; k <= d; ++k) info->grown[k] = R[k];
        info->capped = 0;
        info->norm = 0.0;
        for (int k = 0; k < TT_MAX_D; ++k) info->discarded[k] = 0.0;
    }
    if (d == 1) {  // nothing to round
        TT_TRY(dst[0].ensure((size_t)n[0], s));
        TT_CUDA_TRY(cudaMemcpyAsync(dst[0].p, src[0].p, n[0] * sizeof(double), cudaMemcpyDeviceToDevice, s));
        rr[0] = rr[1] = 1;
        return TT_OK;
    }
    // ---- backward sweep: right Grams GB[k] = B_k^T B_k for bond k
    {
        double fl = 2.0 * R[d - 1] * (double)R[d - 1] * n[d - 1];
        for (int k = d - 3; k >= 0; --k)
            fl += 2.0 * R[k + 1] * (double)n[k + 1] * R[k + 2] * (R[k + 2] + R[k + 1]);
        double by = 0;
        for (int k = 1; k < d; ++k) by += 8.0 * R[k] * (double)n[k] * R[k + 1];
        PhaseScope ps(h, TT_PH_GRAM_RIGHT, fl, by);
        const int Rl = R[d - 1];
        TT_TRY(h->GB[d - 2].ensure((size_t)Rl * Rl, s));
        TT_TRY(dgemm_sk(s, false, true, Rl, Rl, n[d - 1], 1.0, src[d - 1].p, n[d - 1], src[d - 1].p,
                        n[d - 1], h->GB[d - 2].p, Rl, h->partials));
        for (int k = d - 3; k >= 0; --k) {
            const int Ra = R[k + 1], nn = n[k + 1], Rb = R[k + 2];
            TT_TRY(h->bwd.ensure((size_t)Ra * nn * Rb, s));
            TT_TRY(h->GB[k].ensure((size_t)Ra * Ra, s));
            // precision form: both products on the tensor cores (GB[k+1] is
            // symmetric, so bwd = G_{k+1} GB[k+1] = G_{k+1} GB[k+1]^T); a small
            // R x R output over the long contraction n R' runs split-K
            if (h->precision == TT_MIXED) {
                TT_TRY(slgemm_nt(s, (long)Ra * nn, Rb, Rb, src[k + 1].p, Rb, h->GB[k + 1].p, Rb,
                                 h->bwd.p, Rb, h->slscratch, h->d_int + HI_STATUS));
                TT_TRY(slgemm_nt(s, Ra, Ra, nn * Rb, h->bwd.p, (long)nn * Rb, src[k + 1].p,
                                 (long)nn * Rb, h->GB[k].p, Ra, h->slscratch, h->d_int + HI_STATUS));
            } else {
                TT_TRY(dgemm(s, false, false, Ra * nn, Rb, Rb, 1.0, src[k + 1].p, Rb, h->GB[k + 1].p,
                             Rb, 0.0, h->bwd.p, Rb));
                TT_TRY(dgemm_sk(s, false, true, Ra, Ra, nn * Rb, 1.0, h->bwd.p, (long)nn * Rb,
                                src[k + 1].p, (long)nn * Rb, h->GB[k].p, Ra, h->partials));
            }
        }
    }
    {
        // W_k with W_k^T W_k = G_B (pivoted Cholesky): the one-sided truncation
        // needs only this factor of the right Gram matrix
        PhaseScope ps(h, TT_PH_EIG, 0.0, 0.0);
        for (int k = 0; k <= d - 2; ++k) {
            const int Rk = R[k + 1];
            TT_TRY(h->VtB[k].ensure((size_t)Rk * Rk, s));
            TT_TRY(h->Wc.ensure((size_t)Rk * Rk, s));
            TT_TRY(h->lamB[k].ensure((size_t)2 * Rk, s));
            TT_TRY(pchol(s, Rk, h->GB[k].p, Rk, h->VtB[k].p, h->Wc.p, h->lamB[k].p, h->eig,
                         h->d_int + HI_STATUS, h->d_int + HI_KB + k));
        }
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_KB, h->d_int + HI_KB, (d - 1) * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    int kBs[TT_MAX_D];
    for (int k = 0; k < d - 1; ++k) {
        kBs[k] = h->h_int[HI_KB + k];
        if (kBs[k] < 0)
            return fail(TT_ERR_NONFINITE, "rounding: a right Gram matrix holds Inf or NaN (the run diverged or "
                                          "a field held one); restore saved cores and T before stepping again");
    }

    // delta^2 is set from the first bond's ||X||^2
    h->h_dbl[HD_DELTA2] = -1.0;
    TT_CUDA_TRY(cudaMemcpyAsync(h->d_dbl + HD_DELTA2, h->h_dbl + HD_DELTA2, sizeof(double),
                                cudaMemcpyHostToDevice, s));
    rr[0] = 1;
    const double* A = src[0].p;
    int rprev = 1;
    int tmp_idx = 0;
    bool any_capped = false;
    for (int k = 0; k <= d - 2; ++k) {
        const int Rk = R[k + 1];
        const int kB = kBs[k];
        const long m = (long)rprev * n[k];
        if (kB == 0) return zero_tt(h, dst, rr);
        // G_A = A^T A
        TT_TRY(h->GA.ensure((size_t)Rk * Rk, s));
        {
            PhaseScope ps(h, TT_PH_GRAM_LEFT, (double)m * Rk * (Rk + 1.0), 8.0 * ((double)m * Rk + (double)Rk * Rk));
            if (h->precision == TT_MIXED) {
                // A's row exponents for the update below come from the same read
                TT_TRY(h->erowA.ensure((size_t)(m + 1) / 2, s));
                TT_TRY(slgram(s, (int)m, Rk, A, Rk, h->GA.p, Rk, h->partials, h->d_int + HI_STATUS,
                              reinterpret_cast<int*>(h->erowA.p)));
            }
            else
                TT_TRY(gram(s, (int)m, Rk, A, Rk, h->GA.p, Rk, h->partials));
            // a spatial shard holds some rows of the spatial core: its left
            // Gram is the sum of the shards' partial Grams
            if (k == 0 && h->shard.on) TT_TRY(shard_exchange(h, TT_XCHG_SUM, h->GA.p, (size_t)Rk * Rk));
        }
        {
            PhaseScope ps(h, TT_PH_SMALL, 2.0 * Rk * (double)Rk * kB + 2.0 * kB * (double)kB * Rk, 0.0);
            // W (kB x Rk, W^T W = G_B) from the backward sweep; K = W G_A W^T
            const double* Wk = h->VtB[k].p;
            TT_TRY(h->T1.ensure((size_t)Rk * kB, s));
            TT_TRY(h->K.ensure((size_t)kB * kB, s));
            TT_TRY(dgemm_sk(s, false, true, Rk, kB, Rk, 1.0, h->GA.p, Rk, Wk, Rk, h->T1.p, kB, h->partials));
            TT_TRY(dgemm_sk(s, false, false, kB, kB, Rk, 1.0, Wk, Rk, h->T1.p, kB, h->K.p, kB, h->partials));
        }
        TT_TRY(h->lamK.ensure((size_t)kB, s));
        TT_TRY(h->VtK.ensure((size_t)kB * kB, s));
        {
            PhaseScope ps(h, TT_PH_EIG, 0.0, 0.0);
            if (h->eig_method == TT_EIG_ONE_SIDED)
                TT_TRY(syev_psd(s, kB, h->K.p, kB, h->lamK.p, h->VtK.p, kB, h->eig, h->d_int + HI_STATUS,
                                h->d_int + next_sweep_slot(h), h->max_sweeps));
            else
                TT_TRY(syev(s, kB, h->K.p, kB, h->lamK.p, h->VtK.p, kB, h->eig, h->d_int + HI_STATUS,
                            h->d_int + next_sweep_slot(h), h->max_sweeps));
            const int fk = forced ? forced[k] : 0;
            truncation_decision(s, h->lamK.p, kB, eps, d - 1, fk, max_rank, h->d_dbl + HD_DELTA2,
                                h->d_int + HI_DEC, h->d_dbl + HD_DEC);
        }
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_DEC, h->d_int + HI_DEC, 4 * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_dbl + HD_DEC, h->d_dbl + HD_DEC, 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        if (h->h_int[HI_DEC + 2])
            return fail(TT_ERR_NONFINITE, "rounding: the tensor holds Inf or NaN (the run diverged or a field "
                                          "held one); restore saved cores and T before stepping again");
        const int rk = h->h_int[HI_DEC];
        if (h->h_int[HI_DEC + 1]) any_capped = true;
        if (info) {
            info->discarded[k] = sqrt(std::max(h->h_dbl[HD_DEC + 1], 0.0));
            if (k == 0) info->norm = sqrt(std::max(h->h_dbl[HD_DEC + 2], 0.0));
        }
        if (rk == 0) return zero_tt(h, dst, rr);
        const long ncols = (long)n[k + 1] * R[k + 2];
        {
            PhaseScope ps(h, TT_PH_SMALL, 2.0 * rk * (double)kB * Rk + 2.0 * rk * (double)Rk * Rk, 0.0);
            // P_A^T = S~^{-1} V~_r^T W  (rk x Rk)
            TT_TRY(h->Vts.ensure((size_t)rk * kB, s));
            scale_rows(s, rk, kB, h->VtK.p, kB, h->lamK.p, 2, h->Vts.p, kB);
            TT_TRY(h->PAt.ensure((size_t)rk * Rk, s));
            TT_TRY(dgemm_sk(s, false, false, rk, Rk, kB, 1.0, h->Vts.p, kB, h->VtB[k].p, Rk, h->PAt.p, Rk,
                            h->partials));
            // M_upd = P_A^T G_A = A'^T A  (rk x Rk): B'^T = A'^T A B^T, the orthogonal
            // projection of A B^T onto span(A'); equals App. A.2's (V_B S_B^{-1} V~ S~)^T
            // on the retained eigenspace of G_B without forming S_B^{-1}
            TT_TRY(h->Mupd.ensure((size_t)rk * Rk, s));
            TT_TRY(dgemm_sk(s, false, false, rk, Rk, Rk, 1.0, h->PAt.p, Rk, h->GA.p, Rk, h->Mupd.p, Rk,
                            h->partials));
        }
        if (h->cur_rec && h->rec_proj && k < 2) {
            tt_ctx::StepRec* rc = h->cur_rec;
            TT_TRY(rc->P[k].ensure((size_t)rk * Rk, s));
            TT_TRY(rc->M[k].ensure((size_t)rk * Rk, s));
            TT_CUDA_TRY(cudaMemcpyAsync(rc->P[k].p, h->PAt.p, (size_t)rk * Rk * sizeof(double), cudaMemcpyDeviceToDevice, s));
            TT_CUDA_TRY(cudaMemcpyAsync(rc->M[k].p, h->Mupd.p, (size_t)rk * Rk * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        // A' = A P_A -> dst[k]
        TT_TRY(dst[k].ensure((size_t)m * rk, s));
        {
            PhaseScope ps(h, TT_PH_UPDATE, 2.0 * m * (double)Rk * rk, 8.0 * ((double)m * Rk + (double)m * rk));
            if (h->precision == TT_MIXED)
                // A's digit images go to the left Gram's scratch, free until the next bond
                TT_TRY(slgemm_nt(s, m, rk, Rk, A, Rk, h->PAt.p, Rk, dst[k].p, rk, h->slscratch,
                                 h->d_int + HI_STATUS, &h->partials, reinterpret_cast<const int*>(h->erowA.p)));
            else
                TT_TRY(dgemm(s, false, true, (int)m, rk, Rk, 1.0, A, Rk, h->PAt.p, Rk, 0.0, dst[k].p, rk));
        }
        // next core = M_upd x_1 G_{k+1}
        double* next;
        if (k == d - 2) {
            TT_TRY(dst[d - 1].ensure((size_t)rk * ncols, s));
            next = dst[d - 1].p;
        } else {
            TT_TRY(h->tmp[tmp_idx].ensure((size_t)rk * ncols, s));
            next = h->tmp[tmp_idx].p;
            tmp_idx ^= 1;
        }
        {
            PhaseScope ps(h, TT_PH_UPDATE, 2.0 * rk * (double)Rk * ncols,
                          8.0 * ((double)Rk * ncols + (double)rk * ncols));
            TT_TRY(dgemm_sk(s, false, false, rk, (int)ncols, Rk, 1.0, h->Mupd.p, Rk, src[k + 1].p, ncols,
                            next, ncols, h->partials));
        }
        rr[k + 1] = rk;
        A = next;
        rprev = rk;
    }
    rr[d] = 1;
    if (info) {
        info->capped = any_capped ? 1 : 0;
        const int nslots = std::min(h->sweeps_slot, HI_N - HI_SWEEPS);
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_int + HI_SWEEPS, h->d_int + HI_SWEEPS, nslots * sizeof(int),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        int mx = 0;
        for (int i = 0; i < nslots; ++i) mx = std::max(mx, h->h_int[HI_SWEEPS + i]);
        info->sweeps = mx;
    }
    return any_capped ? TT_WARN_RANK_CAPPED : TT_OK;
}

// Build the grown TT (transport terms and/or source) from h->core into h->gcore.
// ---------------------------------------------------------------- split-space layout
// Ranks of the emission term's TT at bonds 0..d (Sec. 3.2 e (x) 1 (x) 1 with
// e held exactly: 1D a column; 2D [I_{N_x}][e]; 3D [I_{N_x}][e][I_{N_z}]).
void split_emission_ranks(const tt_ctx* h, int* er) {
    const int nd = h->grid.ndim, d = h->d;
    for (int k = 0; k <= d; ++k) er[k] = 1;
    if (nd >= 2) er[1] = h->grid.n[0];
    if (nd == 3) er[2] = h->grid.n[2];
}

// Core k's spec in a grown split TT with K transport terms (ranks r -> R)
// and, if emission, the emission term's block.
SplitCoreSpec split_spec(const tt_ctx* h, int k, int K, bool emission, const int* r, const int* R,
                         double tscale) {
    const int nd = h->grid.ndim;
    SplitCoreSpec c{};
    c.kind = k < nd ? SPLIT_SPATIAL : (k == nd ? SPLIT_THETA : SPLIT_PHI);
    c.axis = k < nd ? k : -1;
    c.bc = k < nd ? h->grid.bc[k] : TT_BC_PERIODIC;
    c.first = k == 0;
    c.last = k == h->d - 1;
    c.K = K;
    c.ra = r[k];
    c.n = h->n[k];
    c.rb = r[k + 1];
    c.Ra = R[k];
    c.Rb = R[k + 1];
    c.tscale = c.kind == SPLIT_PHI ? tscale : 1.0;
    if (k < nd)
        for (int t = 0; t < 2; ++t)
            for (int q = 0; q < 3; ++q) c.co[t][q] = h->split_co.c[k][t][q];
    c.ekind = SPLIT_E_NONE;
    if (emission) {
        if (k >= nd)
            c.ekind = SPLIT_E_ONES;
        else if (nd == 1 || k == 1)
            c.ekind = SPLIT_E_FIELD;
        else if (k == 0)
            c.ekind = SPLIT_E_IDENT_COL;
        else
            c.ekind = SPLIT_E_IDENT_ROW;  // 3D z core
    }
    return c;
}

// Where e_i of cell (c0, c1, c2) goes in the grown core that holds the field
// block (core 0 in 1D, core 1 otherwise): base pointer and coordinate strides.
double* split_eblock(tt_ctx* h, int K, const int* r, const int* R, long* st) {
    const int nd = h->grid.ndim;
    if (nd == 1) {  // first core (1 x N_x x R1), block column K r1
        st[0] = R[1];
        st[1] = st[2] = 0;
        return h->gcore[0].p + (long)K * r[1];
    }
    const long n1 = h->n[1];
    st[0] = n1 * R[2];
    st[1] = R[2];
    st[2] = 1;
    return h->gcore[1].p + ((long)K * r[1] * n1) * R[2] + (long)K * r[2];
}

// out (nc x P, cell-major) = the spatial cores of the current TT contracted
// with P right vectors of the last spatial bond (U: P x r_ndim, row-major),
// by one GEMM per spatial core from the right: Z <- G_k (r_{k-1} n_k x r_k) Z.
tt_status split_contract(tt_ctx* h, const double* U, int P, double* out) {
    cudaStream_t s = h->stream;
    const int nd = h->grid.ndim;
    long cols = P;
    const double* Z = U;
    bool zt = true;  // the first right factor is U^T
    int ti = 0;
    for (int k = nd - 1; k >= 0; --k) {
        const long rows = (long)h->r[k] * h->n[k];
        double* dst;
        if (k == 0) {
            dst = out;
        } else {
            TT_TRY(h->sp_tmp[ti].ensure((size_t)(rows * cols), s));
            dst = h->sp_tmp[ti].p;
            ti ^= 1;
        }
        TT_TRY(dgemm(s, false, zt, (int)rows, (int)cols, h->r[k + 1], 1.0, h->core[k].p, h->r[k + 1], Z,
                     zt ? h->r[k + 1] : cols, 0.0, dst, cols));
        Z = dst;
        zt = false;
        cols *= h->n[k];
    }
    return TT_OK;
}

// E-field of the current TT times c (F_i = sum_lp I_ilp dOmega) into sp_F.
tt_status split_energy_field(tt_ctx* h) {
    cudaStream_t s = h->stream;
    const int nd = h->grid.ndim;
    const int ra = h->r[nd], rb = h->r[nd + 1];
    TT_TRY(h->thbar.ensure((size_t)(ra + rb), s));
    plain_thbar(s, h->ang, ra, rb, h->core[nd].p, h->core[nd + 1].p, h->thbar.p);
    TT_TRY(h->sp_F.ensure((size_t)h->grid.nc, s));
    return split_contract(h, h->thbar.p, 1, h->sp_F.p);
}

// Grown split TT (transport terms and/or emission) from h->core into h->gcore.
tt_status split_apply_terms(tt_ctx* h, bool transport, bool source) {
    cudaStream_t s = h->stream;
    const int nd = h->grid.ndim, d = h->d;
    const int K = transport ? 1 + 2 * nd : 1;
    int er[TT_MAX_D + 1], R[TT_MAX_D + 1];
    split_emission_ranks(h, er);
    R[0] = R[d] = 1;
    for (int k = 1; k < d; ++k) R[k] = K * h->r[k] + (source ? er[k] : 0);
    double by = 0.0;
    for (int k = 0; k < d; ++k) by += 8.0 * ((double)h->core_len(k, h->r) + (double)R[k] * h->n[k] * R[k + 1]);
    PhaseScope ps(h, TT_PH_TRANSPORT, 0.0, by + (source ? 8.0 * 6.0 * h->grid.nc : 0.0));
    if (source) {
        // E* pieces: term j's angular cores integrated (U: K x r_ndim), then
        // the spatial cores contracted with each (F: nc x K)
        const int ra = h->r[nd], rb = h->r[nd + 1];
        TT_TRY(h->thbar.ensure((size_t)K * (ra + rb), s));
        grown_thbar(s, h->ang, nd, transport, ra, rb, h->core[nd].p, h->core[nd + 1].p, h->thbar.p);
        TT_TRY(h->sp_F.ensure((size_t)h->grid.nc * K, s));
        TT_TRY(split_contract(h, h->thbar.p, K, h->sp_F.p));
    }
    const double* thf = h->split_fac.p;
    const double* phf = thf + (size_t)(1 + 2 * nd) * h->ang.n_theta;
    for (int k = 0; k < d; ++k) {
        TT_TRY(h->gcore[k].ensure((size_t)R[k] * h->n[k] * R[k + 1], s));
        const SplitCoreSpec c = split_spec(h, k, K, source, h->r, R, source ? h->split_s : 1.0);
        split_grow_core(s, c, h->core[k].p, k == nd ? thf : phf, h->gcore[k].p);
    }
    if (source) {
        long st[3];
        double* eb = split_eblock(h, K, h->r, R, st);
        h->fields.T = h->f_T.p;
        h->fields.E_star = h->f_Estar.p;
        split_source_cells(s, h->grid, h->fields, h->split_co, transport, K, h->sp_F.p, eb, st[0], st[1],
                           st[2]);
    }
    TT_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k <= d; ++k) h->gr[k] = R[k];
    return TT_OK;
}

// One exchange of a spatial shard through the caller's callback, with the
// handle's stream drained first so the callback sees finished data.
tt_status shard_exchange(tt_ctx* h, int kind, double* buf, size_t count) {
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const int rc = h->shard.fn(h->shard.ctx, kind, buf, count, (void*)h->stream);
    if (rc != 0)
        return fail(TT_ERR_STATE, std::string("shard exchange callback failed (") +
                                      (kind == TT_XCHG_SUM ? "sum" : "halo") + ", returned " +
                                      std::to_string(rc) + ")");
    return TT_OK;
}

// The shard's spatial core with its ghost layers (Sec. 4.5): the layer below
// the slab and the layer above it are written after the nc own rows of
// core[0] (r1 columns).  The ring exchange supplies the neighbours' boundary
// layers; at a global face of axis 0 a vacuum ghost is zero and an outflow
// ghost copies the boundary layer (a periodic axis takes the ring's
// wrap-around).
tt_status shard_halo(tt_ctx* h, int r1) {
    cudaStream_t s = h->stream;
    const long nc = h->grid.nc;
    const size_t lay = (size_t)h->shard.plane * r1;
    TT_TRY(h->core[0].ensure((size_t)nc * r1 + 2 * lay, s, /*keep=*/true));
    TT_TRY(h->xch.ensure(4 * lay, s));
    double* send_lo = h->xch.p;
    double* send_hi = send_lo + lay;
    double* recv_lo = send_hi + lay;
    double* recv_hi = recv_lo + lay;
    double* X = h->core[0].p;
    TT_CUDA_TRY(cudaMemcpyAsync(send_lo, X, lay * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(send_hi, X + (size_t)nc * r1 - lay, lay * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    TT_TRY(shard_exchange(h, TT_XCHG_HALO, h->xch.p, lay));
    const bool glo = h->shard.p0 == 0, ghi = h->shard.p1 == h->shard.n0;
    const int bc = h->shard.bc0;
    if (glo && bc == TT_BC_VACUUM) fill(s, recv_lo, lay, 0.0);
    if (ghi && bc == TT_BC_VACUUM) fill(s, recv_hi, lay, 0.0);
    const double* lo = (glo && bc == TT_BC_OUTFLOW) ? send_lo : recv_lo;
    const double* hi = (ghi && bc == TT_BC_OUTFLOW) ? send_hi : recv_hi;
    TT_CUDA_TRY(cudaMemcpyAsync(X + (size_t)nc * r1, lo, lay * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(X + (size_t)nc * r1 + lay, hi, lay * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return TT_OK;
}

tt_status apply_terms(tt_ctx* h, bool transport, bool source) {
    if (h->split()) return split_apply_terms(h, transport, source);
    cudaStream_t s = h->stream;
    const int r1 = h->r[1], r2 = h->r[2];
    const int nterms = transport ? 1 + 2 * h->grid.ndim : 1;
    const int sc = source ? 1 : 0;
    Sources ext;
    if (transport && h->nsrc > 0) {
        ext.n = h->nsrc;
        ext.x = h->src_x.p;
        ext.th = h->src_th.p;
        ext.ph = h->src_ph.p;
        ext.q = h->src_q.p;
    }
    const int R1 = nterms * r1 + ext.n + sc, R2 = nterms * r2 + ext.n + sc;
    const long nc = h->grid.nc;
    const double fbytes = 8.0 * nc * ((source ? 4.0 : 0.0) + (h->has_sigma_s && source ? 1.0 : 0.0));
    PhaseScope ps(h, TT_PH_TRANSPORT, 0.0,
                  8.0 * nc * (double)(r1 + R1) + fbytes +
                      8.0 * ((double)R1 * h->ang.n_theta * R2 + (double)R2 * h->ang.n_phi));
    TT_TRY(h->gcore[0].ensure((size_t)nc * R1, s));
    TT_TRY(h->gcore[1].ensure((size_t)R1 * h->ang.n_theta * R2, s));
    TT_TRY(h->gcore[2].ensure((size_t)R2 * h->ang.n_phi, s));
    if (source) {
        TT_TRY(h->thbar.ensure((size_t)nterms * (r1 + r2), s));
        grown_thbar(s, h->ang, h->grid.ndim, transport, r1, r2, h->core[1].p, h->core[2].p,
                    h->thbar.p);
    }
    build_grown_angular(s, h->ang, h->grid.ndim, transport, source, r1, r2, h->core[1].p,
                        h->core[2].p, h->gcore[1].p, h->gcore[2].p, R1, R2, ext);
    h->fields.T = h->f_T.p;
    h->fields.E_star = h->f_Estar.p;
    if (h->shard.on && transport) TT_TRY(shard_halo(h, r1));
    if (source)  // a shard's halo layers carry dots too
        TT_TRY(h->ydots.ensure((size_t)(nc + (h->shard.on && transport ? 2 * h->shard.plane : 0)) * nterms, s));
    transport_source_rows(s, h->grid, h->fields, transport, source, r1, h->core[0].p, r1,
                          source ? h->thbar.p : nullptr, h->gcore[0].p, R1, h->ydots.p, ext);
    TT_CUDA_TRY(cudaGetLastError());
    h->gr[0] = 1;
    h->gr[1] = R1;
    h->gr[2] = R2;
    h->gr[3] = 1;
    return TT_OK;
}

void swap_grown_into_current(tt_ctx* h) {
    for (int k = 0; k < h->d; ++k) std::swap(h->core[k], h->gcore[k]);
    for (int k = 0; k <= h->d; ++k) h->r[k] = h->gr[k];
}

tt_status energy_update(tt_ctx* h) {
    cudaStream_t s = h->stream;
    if (h->split()) {
        PhaseScope ps(h, TT_PH_ENERGY, 0.0, 8.0 * h->grid.nc * 5.0);
        TT_TRY(split_energy_field(h));
        energy_rows(s, h->grid.nc, 1, h->sp_F.p, 1, h->d_dbl + HD_ONE, h->fields.c, nullptr,
                    h->f_Estar.p, h->f_cv.p, h->f_T.p, true);
        TT_CUDA_TRY(cudaGetLastError());
        return TT_OK;
    }
    const int r1 = h->r[1], r2 = h->r[2];
    TT_TRY(h->thbar.ensure((size_t)(r1 + r2), s));
    PhaseScope ps(h, TT_PH_ENERGY, 0.0, 8.0 * h->grid.nc * (r1 + 4.0));
    plain_thbar(s, h->ang, r1, r2, h->core[1].p, h->core[2].p, h->thbar.p);
    energy_rows(s, h->grid.nc, r1, h->core[0].p, r1, h->thbar.p, h->fields.c, nullptr,
                h->f_Estar.p, h->f_cv.p, h->f_T.p, true);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

// Escape energy of a state (cores X, Th, Ph with ranks o1, o2) added into
// d_dbl[HD_Q]: sum over vacuum boundary faces of dt dA (n . n_out)^+ I dOmega.
tt_status add_escape_energy(tt_ctx* h, const double* X, const double* Th, const double* Ph, int o1,
                            int o2) {
    cudaStream_t s = h->stream;
    const int nterms = 1 + 2 * h->grid.ndim;
    TT_TRY(h->atb1.ensure((size_t)nterms * (o1 + o2), s));
    TT_TRY(h->aq.ensure((size_t)h->grid.nc, s));
    grown_thbar(s, h->ang, h->grid.ndim, true, o1, o2, Th, Ph, h->atb1.p);
    escape_rows(s, h->grid, h->fields.dt, o1, X, o1, h->atb1.p, h->aq.p, nullptr, 0, false);
    sum_into(s, h->grid.nc, h->aq.p, h->d_dbl + HD_Q);
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status copy_dev(DevBuf& dst, const double* src, size_t n, cudaStream_t s) {
    TT_TRY(dst.ensure(std::max<size_t>(n, 1), s));
    TT_CUDA_TRY(cudaMemcpyAsync(dst.p, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return TT_OK;
}

tt_status step_once(tt_ctx* h, int flags, const int* forced, tt_step_info* info) {
    const bool src = !(flags & TT_STEP_NO_SOURCE);
    const bool rnd = !(flags & TT_STEP_NO_ROUND);
    const bool two = (h->rounds == 2) && src && rnd;
    tt_status result = TT_OK;
    int rr[TT_MAX_D + 1];
    h->cur_rec = nullptr;
    if (h->taping || h->replay_rec) {
        if (!src || !rnd || two || h->precision != TT_FP64 || h->has_sigma_s || !h->physics ||
            h->split())
            return fail(TT_ERR_STATE, "adjoint tape: only plain FP64 transport steps (grouped "
                                      "layout, one rounding, source on, no scattering) can be "
                                      "recorded");
        tt_ctx::StepRec* rc = h->replay_rec;
        if (h->taping) {
            rc = new tt_ctx::StepRec();
            h->tape.push_back(rc);
            h->rec_state = ((h->tape.size() - 1) % (size_t)h->tape_every) == 0;
            h->rec_proj = h->tape_every == 1;
        }
        rc->r1 = h->r[1];
        rc->r2 = h->r[2];
        if (h->rec_state) {
            cudaStream_t s = h->stream;
            TT_TRY(copy_dev(rc->X, h->core[0].p, (size_t)h->grid.nc * rc->r1, s));
            TT_TRY(copy_dev(rc->Th, h->core[1].p, (size_t)rc->r1 * h->ang.n_theta * rc->r2, s));
            TT_TRY(copy_dev(rc->Ph, h->core[2].p, (size_t)rc->r2 * h->ang.n_phi, s));
            TT_TRY(copy_dev(rc->T, h->f_T.p, (size_t)h->grid.nc, s));
            rc->state = true;
        }
        h->cur_rec = rc;
    }
    TT_TRY(apply_terms(h, true, src && !two));
    if (two) {
        tt_status st = round_cores(h, h->gcore, h->gr, h->core, rr, h->eps, h->max_rank, forced, info);
        if (forced) forced += h->d - 1;  // the second rounding takes the next d-1 entries
        if (st < 0) return st;
        if (st == TT_WARN_RANK_CAPPED) result = st;
        for (int k = 0; k <= h->d; ++k) h->r[k] = rr[k];
        TT_TRY(apply_terms(h, false, true));
    }
    if (rnd) {
        tt_status st = round_cores(h, h->gcore, h->gr, h->core, rr, h->eps, h->max_rank, forced, info);
        if (st < 0) return st;
        if (st == TT_WARN_RANK_CAPPED) result = st;
        for (int k = 0; k <= h->d; ++k) h->r[k] = rr[k];
    } else {
        swap_grown_into_current(h);
        if (info) {
            info->d = h->d;
            for (int k = 0; k <= h->d; ++k) info->grown[k] = h->r[k];
        }
    }
    if (src) TT_TRY(energy_update(h));
    if (h->cur_rec) {
        tt_ctx::StepRec* rc = h->cur_rec;
        h->cur_rec = nullptr;
        rc->R1 = h->gr[1];
        rc->R2 = h->gr[2];
        rc->o1 = h->r[1];
        rc->o2 = h->r[2];
        if (h->rec_proj) rc->proj = true;
        if (h->taping)
            TT_TRY(add_escape_energy(h, h->core[0].p, h->core[1].p, h->core[2].p, rc->o1, rc->o2));
    }
    if (info)
        for (int k = 0; k <= h->d; ++k) info->ranks[k] = h->r[k];
    return result;
}

// ---------------------------------------------------------------- captured steps
// One grouped FP64 step recorded into a CUDA graph.  The step's sizes (the
// grown ranks, the right Grams' numerical ranks, the two rank decisions) are
// decided on the device, so every kernel of the captured step reads them from
// the handle's size block (DYN_* slots) and every grid covers the largest
// sizes the rank cap allows; the products' descriptors (M, N, K and the
// leading dimensions) are filled by plan_kernel as the sizes become known.
// The launches are the host path's own kernels in the same order with the
// same split rules, so a replayed step gives the same bits as tt_sn_step.
// Whether the handle's steps can be captured: the grouped FP64 step with one
// Gram-SVD rounding, a rank cap (every buffer has its largest size from the
// start), no fixed sources or inflow faces, no adjoint tape, not a shard.
const char* graph_unsupported(const tt_ctx* h) {
    if (!h->physics || h->split()) return "captured steps need the grouped layout";
    if (h->precision != TT_FP64) return "captured steps are FP64";
    if (h->rounds != 1) return "captured steps round once per step";
    if (h->round_method != TT_ROUND_GRAM) return "captured steps use the Gram-SVD rounding";
    if (h->max_rank <= 0) return "captured steps need a rank cap (max_rank > 0)";
    if (h->nsrc > 0) return "captured steps take no fixed sources or inflow faces";
    if (h->taping) return "captured steps are not taped";
    if (h->shard.on) return "a spatial shard exchanges on the host and is not captured";
    if (h->fields.flux == TT_FLUX_HLL || h->fields.flux == TT_FLUX_RUSANOV_TAU)
        return "captured steps take upwind or uniform-speed Rusanov fluxes";
    return nullptr;
}

// The launches of one step, sized by the caps, reading sizes from h->dyn.
tt_status graph_step_body(tt_ctx* h) {
    cudaStream_t s = h->stream;
    const Grid& g = h->grid;
    const int nterms = 1 + 2 * g.ndim;
    const int nt = h->ang.n_theta, np = h->ang.n_phi;
    const int c1 = h->cap1, c2 = h->cap2;
    const int G1 = nterms * c1 + 1, G2 = nterms * c2 + 1;
    const long nc = g.nc;
    int* dd = h->dyn;
    const int* desc = dd + DYN_DESC;
    double* P = h->dyn_part.p;
    const size_t PC = h->dyn_part.cap;
    double* dec_d = h->dyn_buf.p + (DYN_INTS + 1) / 2;
    const PlanConsts pc{nterms, nt, np, nc};
    auto plan = [&](int stage) {
        note_launch();
        plan_kernel<<<1, 1, 0, s>>>(stage, dd, pc);
    };
    plan(0);
    // transport + source (Sec. 4.3-4.4): the grown cores
    grown_thbar(s, h->ang, g.ndim, true, c1, c2, h->core[1].p, h->core[2].p, h->thbar.p, dd);
    build_grown_angular(s, h->ang, g.ndim, true, true, c1, c2, h->core[1].p, h->core[2].p, h->gcore[1].p,
                        h->gcore[2].p, G1, G2, Sources(), dd);
    h->fields.T = h->f_T.p;
    h->fields.E_star = h->f_Estar.p;
    transport_source_rows(s, g, h->fields, true, true, c1, h->core[0].p, c1, h->thbar.p, h->gcore[0].p, G1,
                          h->ydots.p, Sources(), dd);
    // rounding (App. A.2, one-sided Gram truncation): backward sweep
    fill(s, h->d_dbl + HD_DELTA2, 1, -1.0);
    TT_TRY(dgemm_dyn(s, false, true, desc + 0, G2, G2, np, 1.0, h->gcore[2].p, h->gcore[2].p, h->GB[1].p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, false, desc + 8, G1 * nt, G2, G2, 1.0, h->gcore[1].p, h->GB[1].p, h->bwd.p, P, PC, 0));
    TT_TRY(dgemm_dyn(s, false, true, desc + 16, G1, G1, nt * G2, 1.0, h->bwd.p, h->gcore[1].p, h->GB[0].p, P, PC, 1));
    TT_TRY(pchol_dyn(s, dd + DYN_G1, G1, h->GB[0].p, h->VtB[0].p, h->Wc.p, h->lamB[0].p, h->eig,
                     h->d_int + HI_STATUS, dd + DYN_KB0));
    TT_TRY(pchol_dyn(s, dd + DYN_G2, G2, h->GB[1].p, h->VtB[1].p, h->Wc.p, h->lamB[1].p, h->eig,
                     h->d_int + HI_STATUS, dd + DYN_KB1));
    plan(1);
    // bond 0: G_A, K = W G_A W^T, eig(K), decision
    TT_TRY(dgemm_dyn(s, true, false, desc + 24, G1, G1, (int)nc, 1.0, h->gcore[0].p, h->gcore[0].p, h->GA.p, P, PC, 2));
    TT_TRY(dgemm_dyn(s, false, true, desc + 32, G1, G1, G1, 1.0, h->GA.p, h->VtB[0].p, h->T1.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, false, desc + 40, G1, G1, G1, 1.0, h->VtB[0].p, h->T1.p, h->K.p, P, PC, 1));
    TT_TRY((h->eig_method == TT_EIG_ONE_SIDED ? syev_psd_dyn : syev_dyn)(
        s, dd + DYN_KB0, G1, h->K.p, h->lamK.p, h->VtK.p, h->eig, h->d_int + HI_STATUS, dd + DYN_SWEEPS,
        h->max_sweeps));
    truncation_decision_dyn(s, h->lamK.p, dd + DYN_KB0, h->eps, 2, 0, h->max_rank, h->d_dbl + HD_DELTA2,
                            dd + DYN_DEC0, dec_d);
    plan(2);
    // bond 0 update: P_A^T, M_upd, X' = X* P_A, next core = M_upd x_1 Theta*
    scale_rows_dyn(s, desc + 48, (long)c1 * G1, h->VtK.p, h->lamK.p, 2, h->Vts.p);
    TT_TRY(dgemm_dyn(s, false, false, desc + 56, c1, G1, G1, 1.0, h->Vts.p, h->VtB[0].p, h->PAt.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, false, desc + 64, c1, G1, G1, 1.0, h->PAt.p, h->GA.p, h->Mupd.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, true, desc + 72, (int)nc, c1, G1, 1.0, h->gcore[0].p, h->PAt.p, h->core[0].p, P, PC, 0));
    TT_TRY(dgemm_dyn(s, false, false, desc + 80, c1, nt * G2, G1, 1.0, h->Mupd.p, h->gcore[1].p, h->tmp[0].p, P, PC, 1));
    // bond 1 on the next core (replicated rows r0 n_theta)
    TT_TRY(dgemm_dyn(s, true, false, desc + 88, G2, G2, c1 * nt, 1.0, h->tmp[0].p, h->tmp[0].p, h->GA.p, P, PC, 2));
    TT_TRY(dgemm_dyn(s, false, true, desc + 96, G2, G2, G2, 1.0, h->GA.p, h->VtB[1].p, h->T1.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, false, desc + 104, G2, G2, G2, 1.0, h->VtB[1].p, h->T1.p, h->K.p, P, PC, 1));
    TT_TRY((h->eig_method == TT_EIG_ONE_SIDED ? syev_psd_dyn : syev_dyn)(
        s, dd + DYN_KB1, G2, h->K.p, h->lamK.p, h->VtK.p, h->eig, h->d_int + HI_STATUS, dd + DYN_SWEEPS + 1,
        h->max_sweeps));
    truncation_decision_dyn(s, h->lamK.p, dd + DYN_KB1, h->eps, 2, 0, h->max_rank, h->d_dbl + HD_DELTA2,
                            dd + DYN_DEC1, dec_d + 4);
    plan(3);
    scale_rows_dyn(s, desc + 112, (long)c2 * G2, h->VtK.p, h->lamK.p, 2, h->Vts.p);
    TT_TRY(dgemm_dyn(s, false, false, desc + 120, c2, G2, G2, 1.0, h->Vts.p, h->VtB[1].p, h->PAt.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, false, desc + 128, c2, G2, G2, 1.0, h->PAt.p, h->GA.p, h->Mupd.p, P, PC, 1));
    TT_TRY(dgemm_dyn(s, false, true, desc + 136, c1 * nt, c2, G2, 1.0, h->tmp[0].p, h->PAt.p, h->core[1].p, P, PC, 0));
    TT_TRY(dgemm_dyn(s, false, false, desc + 144, c2, np, G2, 1.0, h->Mupd.p, h->gcore[2].p, h->core[2].p, P, PC, 1));
    // energy-conserving temperature update (Sec. 3.2) from the rounded TT
    plain_thbar(s, h->ang, c1, c2, h->core[1].p, h->core[2].p, h->thbar.p, dd);
    energy_rows(s, nc, c1, h->core[0].p, c1, h->thbar.p, h->fields.c, nullptr, h->f_Estar.p, h->f_cv.p,
                h->f_T.p, true, dd);
    // the sizes and decisions for the host, read after the next synchronisation
    TT_CUDA_TRY(cudaMemcpyAsync(h->h_dyn, dd, DYN_INTS * sizeof(int), cudaMemcpyDeviceToHost, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->h_dyn_dec, dec_d, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

// Every buffer a captured step touches at its largest size (nothing may
// allocate inside a capture).
tt_status graph_reserve(tt_ctx* h) {
    cudaStream_t s = h->stream;
    const Grid& g = h->grid;
    const long nterms = 1 + 2 * g.ndim;
    const long nt = h->ang.n_theta, np = h->ang.n_phi, nc = g.nc;
    const long c1 = h->cap1, c2 = h->cap2, G1 = nterms * c1 + 1, G2 = nterms * c2 + 1;
    const long Gm = std::max(G1, G2);
    // partials of the captured split products: the largest need over the
    // (mode, M, N, K) capacities of graph_step_body's products
    size_t part = 1;
    {
        const int c[][4] = {{1, (int)G2, (int)G2, (int)np},       {1, (int)G1, (int)G1, (int)(nt * G2)},
                            {2, (int)G1, (int)G1, (int)nc},       {1, (int)G1, (int)G1, (int)G1},
                            {1, (int)c1, (int)G1, (int)G1},       {1, (int)c1, (int)(nt * G2), (int)G1},
                            {2, (int)G2, (int)G2, (int)(c1 * nt)}, {1, (int)G2, (int)G2, (int)G2},
                            {1, (int)c2, (int)G2, (int)G2},       {1, (int)c2, (int)np, (int)G2}};
        for (const auto& q : c) part = std::max(part, dyn_partials_need(q[0], q[1], q[2], q[3]));
    }
    struct Need {
        DevBuf* b;
        long n;
    } need[] = {
        {&h->core[0], nc * c1}, {&h->core[1], c1 * nt * c2}, {&h->core[2], c2 * np},
        {&h->gcore[0], nc * G1}, {&h->gcore[1], G1 * nt * G2}, {&h->gcore[2], G2 * np},
        {&h->GB[0], G1 * G1}, {&h->GB[1], G2 * G2}, {&h->VtB[0], G1 * G1}, {&h->VtB[1], G2 * G2},
        {&h->lamB[0], 2 * G1}, {&h->lamB[1], 2 * G2}, {&h->Wc, Gm * Gm}, {&h->GA, Gm * Gm},
        {&h->T1, Gm * Gm}, {&h->K, Gm * Gm}, {&h->lamK, Gm}, {&h->VtK, Gm * Gm},
        {&h->Vts, Gm * Gm}, {&h->PAt, Gm * Gm}, {&h->Mupd, Gm * Gm}, {&h->bwd, G1 * nt * G2},
        {&h->tmp[0], c1 * nt * G2}, {&h->thbar, nterms * (c1 + c2) + 2}, {&h->ydots, nc * nterms},
        {&h->eig.g0, Gm * Gm}, {&h->eig.g1, Gm * Gm}, {&h->eig.vt_unsorted, Gm * Gm},
        {&h->eig.lam_unsorted, Gm}, {&h->eig.abc, 3 * (Gm + 1)}, {&h->eig.cs, Gm + 1},
        {&h->eig.psd, 3 * Gm + 2},
        {&h->dyn_part, (long)part},
    };
    for (auto& x : need) TT_TRY(x.b->ensure((size_t)std::max<long>(x.n, 1), s, /*keep=*/true));
    TT_TRY(eig_reserve(h->eig, s));
    TT_TRY(h->dyn_buf.ensure((size_t)(DYN_INTS + 1) / 2 + 16, s));
    h->dyn = reinterpret_cast<int*>(h->dyn_buf.p);
    if (!h->h_dyn) TT_CUDA_TRY(cudaMallocHost(&h->h_dyn, DYN_INTS * sizeof(int)));
    if (!h->h_dyn_dec) TT_CUDA_TRY(cudaMallocHost(&h->h_dyn_dec, 8 * sizeof(double)));
    return TT_OK;
}

// The host's ranks after replays: wait for the stream and take the device's.
tt_status refresh_ranks(tt_ctx* h) {
    if (!h->ranks_stale) return TT_OK;
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->ranks_stale = false;
    h->r[0] = h->r[3] = 1;
    h->r[1] = h->h_dyn[DYN_R1];
    h->r[2] = h->h_dyn[DYN_R2];
    h->gr[0] = h->gr[3] = 1;
    h->gr[1] = h->h_dyn[DYN_G1];
    h->gr[2] = h->h_dyn[DYN_G2];
    return TT_OK;
}

// The diagnostics of the last replayed step and the flags of all replays
// since the sticky slot was cleared (host mirror, after a sync).
tt_status graph_info(tt_ctx* h, tt_step_info* info, bool* capped) {
    const int* hd = h->h_dyn;
    const int sticky = hd[DYN_STICKY];
    *capped = (sticky & 1) != 0;
    if (sticky & 2)
        return fail(TT_ERR_NONFINITE, "rounding: the tensor holds Inf or NaN (the run diverged or a field "
                                      "held one); restore saved cores and T before stepping again");
    if (sticky & 4)
        return fail(TT_ERR_STATE, "captured step: the rounding met a zero tensor, which a captured step "
                                  "does not represent; restore saved cores and T and step without capture");
    if (info) {
        info->d = 3;
        info->ranks[0] = info->ranks[3] = 1;
        info->ranks[1] = hd[DYN_R1];
        info->ranks[2] = hd[DYN_R2];
        info->grown[0] = info->grown[3] = 1;
        info->grown[1] = hd[DYN_G1];
        info->grown[2] = hd[DYN_G2];
        for (int k = 0; k < TT_MAX_D; ++k) info->discarded[k] = 0.0;
        info->discarded[0] = sqrt(std::max(h->h_dyn_dec[1], 0.0));
        info->discarded[1] = sqrt(std::max(h->h_dyn_dec[5], 0.0));
        info->norm = sqrt(std::max(h->h_dyn_dec[2], 0.0));
        info->capped = *capped ? 1 : 0;
        info->sweeps = std::max(hd[DYN_SWEEPS], hd[DYN_SWEEPS + 1]);
    }
    return TT_OK;
}

// Record the step once (the first captured step), then replay.
tt_status graph_launch(tt_ctx* h) {
    cudaStream_t s = h->stream;
    if (!h->graph_exec) {
        TT_TRY(graph_reserve(h));
        // the size block starts from the host's ranks
        int init[2] = {h->r[1], h->r[2]};
        TT_CUDA_TRY(cudaMemcpyAsync(h->dyn + DYN_R1, init, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        TT_TRY(eig_prepare());
        const unsigned long long before = t_launches;
        cudaGraph_t graph = nullptr;
        // record on a stream of its own (the handle's stream may be the legacy
        // default stream, which cannot be captured); the graph is then
        // launched on the handle's stream
        cudaStream_t cap = nullptr;
        TT_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        h->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        tt_status st = TT_OK;
        if (e == cudaSuccess) {
            st = graph_step_body(h);
            e = cudaStreamEndCapture(cap, &graph);
        }
        h->stream = s;
        cudaStreamDestroy(cap);
        if (st < 0) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(TT_ERR_CUDA, std::string("captured step: stream capture failed: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->graph_exec = nullptr;
            return fail(TT_ERR_CUDA, std::string("captured step: instantiation failed: ") + cudaGetErrorString(e));
        }
        // the capture counted its launches; each replay runs them again
        h->graph_launches = (unsigned)(t_launches - before);
        g_launches.fetch_sub(h->graph_launches);
        t_launches -= h->graph_launches;
    } else if (!h->ranks_stale) {
        // the host changed the state (set_cores, a plain step): restart from its ranks
        int init[2] = {h->r[1], h->r[2]};
        TT_CUDA_TRY(cudaMemcpyAsync(h->dyn + DYN_R1, init, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    TT_CUDA_TRY(cudaGraphLaunch(h->graph_exec, s));
    note_launch(h->graph_launches);
    h->ranks_stale = true;
    return TT_OK;
}

// Before a run of replays: the capture conditions still hold (a setting may
// have changed since tt_set_graph) and the sticky flags are cleared.
tt_status graph_start(tt_ctx* h) {
    if (const char* why = graph_unsupported(h)) return fail(TT_ERR_STATE, std::string("captured step: ") + why);
    if (h->cap1 == 0) {
        const long nc = h->grid.nc;
        h->cap1 = (int)std::min<long>(h->max_rank, std::min<long>(nc, (long)h->ang.n_theta * h->ang.n_phi));
        h->cap2 = (int)std::min<long>(h->max_rank, h->ang.n_phi);
    }
    if (h->r[1] > h->cap1 || h->r[2] > h->cap2)
        return fail(TT_ERR_STATE, "captured step: the TT's ranks exceed the rank cap");
    if (!h->dyn) TT_TRY(graph_reserve(h));
    TT_CUDA_TRY(cudaMemsetAsync(h->dyn + DYN_STICKY, 0, sizeof(int), h->stream));
    return TT_OK;
}

// After a run of replays: wait, report the device status and the flags, fill info.
tt_status graph_finish(tt_ctx* h, tt_step_info* info) {
    TT_TRY(read_status(h));  // synchronises the stream
    h->ranks_stale = false;
    TT_TRY(refresh_ranks(h));
    h->r[1] = h->h_dyn[DYN_R1];
    h->r[2] = h->h_dyn[DYN_R2];
    h->gr[1] = h->h_dyn[DYN_G1];
    h->gr[2] = h->h_dyn[DYN_G2];
    bool capped = false;
    TT_TRY(graph_info(h, info, &capped));
    return capped ? TT_WARN_RANK_CAPPED : TT_OK;
}

tt_status check_handle(tt_handle h, bool need_physics) {
    if (!h) return fail(TT_ERR_ARG, "null handle");
    if (need_physics && !h->physics) return fail(TT_ERR_STATE, "handle is a bare TT (no problem attached)");
    // after captured steps the host's ranks follow the device's
    TT_TRY(refresh_ranks(h));
    return TT_OK;
}

// ---------------------------------------------------------------- adjoint form
// Reverse mode of the taped steps for the gradient of the escape energy
// Q = sum_m Q(I^m) with respect to sigma_a.  The rounding's factors are held
// fixed: X' = X_g P_1, C = M_1 Theta_g, Theta' = C P_2, Phi' = M_2 Phi_g (P_k
// the transpose of the stored P_A^T), so the rounding is reversed by four
// GEMMs with the stored factors.  The quartic of Sec. 3.2 is reversed by the
// implicit-function theorem inside the source kernel.

// Copy a state into the handle (cores with ranks r1, r2 and the temperature).
tt_status load_state(tt_ctx* h, const double* X, const double* Th, const double* Ph, const double* T,
                     int r1, int r2) {
    cudaStream_t s = h->stream;
    const size_t nx = (size_t)h->grid.nc * r1, nth = (size_t)r1 * h->ang.n_theta * r2,
                 nph = (size_t)r2 * h->ang.n_phi;
    TT_TRY(h->core[0].ensure(nx, s));
    TT_TRY(h->core[1].ensure(nth, s));
    TT_TRY(h->core[2].ensure(nph, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->core[0].p, X, nx * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->core[1].p, Th, nth * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->core[2].p, Ph, nph * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->f_T.p, T, (size_t)h->grid.nc * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    h->r[0] = 1;
    h->r[1] = r1;
    h->r[2] = r2;
    h->r[3] = 1;
    return TT_OK;
}

// One step reversed.  In: the adjoints of the step's output state (aXb: nc x o1,
// aThb: o1 x nt x o2, aPhb: o2 x np, aTb: nc) and the output cores; out: the
// adjoints of its input state (swapped into the same buffers), sigma_a's
// gradient accumulated in asigb.
tt_status reverse_step(tt_ctx* h, const tt_ctx::StepRec& rc, const double* Xo, const double* Tho,
                       const double* Pho) {
    cudaStream_t s = h->stream;
    const Grid& g = h->grid;
    const Angular& ang = h->ang;
    const long nc = g.nc;
    const int nt = ang.n_theta, np = ang.n_phi;
    const int nterms = 1 + 2 * g.ndim;
    const int r1 = rc.r1, r2 = rc.r2, R1 = rc.R1, R2 = rc.R2, o1 = rc.o1, o2 = rc.o2;
    const int nr = nterms * r1;
    const double c = h->fields.c;
    TT_TRY(h->atb1.ensure((size_t)nterms * (std::max(o1, r1) + std::max(o2, r2)), s));
    TT_TRY(h->atb2.ensure((size_t)nterms * (r1 + r2), s));
    TT_TRY(h->aq.ensure((size_t)nc, s));
    TT_TRY(h->athbb.ensure((size_t)nterms * std::max(o1, r1), s));
    TT_TRY(h->ascr.ensure((size_t)2 * nterms * std::max(o2, r2), s));
    TT_TRY(h->ae1b.ensure((size_t)nc, s));
    TT_TRY(h->aEsb.ensure((size_t)nc, s));
    TT_TRY(h->aEsbo.ensure((size_t)nc, s));
    TT_TRY(h->aTbi.ensure((size_t)nc, s));
    TT_TRY(h->aPhgb.ensure((size_t)R2 * np, s));
    TT_TRY(h->aThtb.ensure((size_t)o1 * nt * R2, s));
    TT_TRY(h->aThgb.ensure((size_t)R1 * nt * R2, s));
    TT_TRY(h->aXgb.ensure((size_t)nc * R1, s));
    TT_TRY(h->aThbi.ensure((size_t)r1 * nt * r2, s));
    TT_TRY(h->aPhbi.ensure((size_t)r2 * np, s));
    TT_TRY(h->aybar.ensure((size_t)nc * nr, s));
    TT_TRY(h->aY.ensure((size_t)nc * nr, s));
    TT_TRY(h->aXbi.ensure((size_t)nc * r1, s));

    // (1) this step's term of Q, a linear functional of the output cores
    grown_thbar(s, ang, g.ndim, true, o1, o2, Tho, Pho, h->atb1.p);
    escape_rows(s, g, h->fields.dt, o1, Xo, o1, h->atb1.p, h->aq.p, h->aXb.p, o1, true);
    fill(s, h->athbb.p, (size_t)nterms * o1, 0.0);
    escape_thbb(s, g, h->fields.dt, o1, Xo, o1, h->athbb.p);
    thbar_adjoint(s, ang, nterms, 1, o1, o2, Tho, Pho, h->athbb.p, h->ascr.p, h->aThb.p, h->aPhb.p);

    // (2) T' = T + (E* - E')/C_v with E' = X' . thbar'/c
    plain_thbar(s, ang, o1, o2, Tho, Pho, h->atb1.p);
    energy_adjoint_rows(s, nc, o1, h->atb1.p, c, h->f_cv.p, h->aTb.p, h->aXb.p, o1, h->ae1b.p,
                        h->aEsb.p);
    TT_TRY(gemv_t(s, nc, o1, 1.0, Xo, o1, h->ae1b.p, h->athbb.p, h->agv));
    thbar_adjoint(s, ang, 1, 0, o1, o2, Tho, Pho, h->athbb.p, h->ascr.p, h->aThb.p, h->aPhb.p);

    // (3) rounding with frozen factors, reversed
    TT_TRY(dgemm(s, true, false, R2, np, o2, 1.0, rc.M[1].p, R2, h->aPhb.p, np, 0.0, h->aPhgb.p, np));
    TT_TRY(dgemm(s, false, false, o1 * nt, R2, o2, 1.0, h->aThb.p, o2, rc.P[1].p, R2, 0.0,
                 h->aThtb.p, R2));
    TT_TRY(dgemm(s, true, false, R1, nt * R2, o1, 1.0, rc.M[0].p, R1, h->aThtb.p, (long)nt * R2,
                 0.0, h->aThgb.p, (long)nt * R2));
    TT_TRY(dgemm(s, false, false, (int)nc, R1, o1, 1.0, h->aXb.p, o1, rc.P[0].p, R1, 0.0,
                 h->aXgb.p, R1));

    // (4) grown angular cores (block-diagonal with the term factors), reversed
    fill(s, h->aThbi.p, (size_t)r1 * nt * r2, 0.0);
    fill(s, h->aPhbi.p, (size_t)r2 * np, 0.0);
    grown_angular_adjoint(s, ang, g.ndim, r1, r2, h->aThgb.p, h->aPhgb.p, R1, R2, h->aThbi.p,
                          h->aPhbi.p);

    // (5) source stage and the quartic, reversed per cell
    grown_thbar(s, ang, g.ndim, true, r1, r2, rc.Th.p, rc.Ph.p, h->atb2.p);
    source_adjoint_rows(s, g, h->fields, r1, rc.X.p, r1, h->atb2.p, rc.T.p, h->aXgb.p, R1,
                        h->aEsb.p, h->aTb.p, h->aybar.p, h->aY.p, nr, h->aEsbo.p, h->aTbi.p,
                        h->asigb.p);

    // (6) E* = y . thbar / c: the quadrature vectors' adjoint
    TT_TRY(gemv_t(s, nc, nr, 1.0 / c, h->aY.p, nr, h->aEsbo.p, h->athbb.p, h->agv));
    thbar_adjoint(s, ang, nterms, 0, r1, r2, rc.Th.p, rc.Ph.p, h->athbb.p, h->ascr.p, h->aThbi.p,
                  h->aPhbi.p);

    // (7) the transport stencil, transposed
    stencil_adjoint_rows(s, g, h->fields, r1, h->aybar.p, nr, h->aXbi.p, r1);
    TT_CUDA_TRY(cudaGetLastError());
    std::swap(h->aXb, h->aXbi);
    std::swap(h->aThb, h->aThbi);
    std::swap(h->aPhb, h->aPhbi);
    std::swap(h->aTb, h->aTbi);
    return TT_OK;
}

void clear_tape(tt_ctx* h) {
    for (tt_ctx::StepRec* r : h->tape) {
        r->release();
        delete r;
    }
    h->tape.clear();
    h->taping = false;
    h->replay_rec = nullptr;
    h->cur_rec = nullptr;
}

tt_status adjoint_run(tt_ctx* h, double* grad_dev, double* Q_host) {
    cudaStream_t s = h->stream;
    const long nc = h->grid.nc;
    const int M = (int)h->tape.size();
    if (M == 0) return fail(TT_ERR_STATE, "tt_sn_step_adjoint: no taped steps");
    const int every = std::max(1, h->tape_every);
    h->taping = false;
    // the final state, restored after the replays
    tt_ctx::StepRec fin;
    fin.r1 = h->r[1];
    fin.r2 = h->r[2];
    TT_TRY(copy_dev(fin.X, h->core[0].p, (size_t)nc * fin.r1, s));
    TT_TRY(copy_dev(fin.Th, h->core[1].p, (size_t)fin.r1 * h->ang.n_theta * fin.r2, s));
    TT_TRY(copy_dev(fin.Ph, h->core[2].p, (size_t)fin.r2 * h->ang.n_phi, s));
    TT_TRY(copy_dev(fin.T, h->f_T.p, (size_t)nc, s));
    tt_status st = TT_OK;
    do {
        // adjoint of the final state: zero
        if ((st = h->aXb.ensure((size_t)nc * fin.r1, s)) < 0) break;
        if ((st = h->aThb.ensure((size_t)fin.r1 * h->ang.n_theta * fin.r2, s)) < 0) break;
        if ((st = h->aPhb.ensure((size_t)fin.r2 * h->ang.n_phi, s)) < 0) break;
        if ((st = h->aTb.ensure((size_t)nc, s)) < 0) break;
        if ((st = h->asigb.ensure((size_t)nc, s)) < 0) break;
        fill(s, h->aXb.p, (size_t)nc * fin.r1, 0.0);
        fill(s, h->aThb.p, (size_t)fin.r1 * h->ang.n_theta * fin.r2, 0.0);
        fill(s, h->aPhb.p, (size_t)fin.r2 * h->ang.n_phi, 0.0);
        fill(s, h->aTb.p, (size_t)nc, 0.0);
        fill(s, h->asigb.p, (size_t)nc, 0.0);
        for (int seg_end = M; seg_end > 0 && st >= 0;) {
            const int seg_start = ((seg_end - 1) / every) * every;
            bool need = false;
            for (int m = seg_start; m < seg_end; ++m)
                need = need || !h->tape[m]->state || !h->tape[m]->proj;
            if (need) {  // re-run the segment from its checkpoint, refilling the records
                tt_ctx::StepRec* c0 = h->tape[seg_start];
                if ((st = load_state(h, c0->X.p, c0->Th.p, c0->Ph.p, c0->T.p, c0->r1, c0->r2)) < 0)
                    break;
                for (int m = seg_start; m < seg_end && st >= 0; ++m) {
                    tt_ctx::StepRec* rc = h->tape[m];
                    const int forced[2] = {rc->o1, rc->o2};
                    h->replay_rec = rc;
                    h->rec_state = !rc->state;
                    h->rec_proj = true;
                    st = step_once(h, 0, forced, nullptr);
                    h->replay_rec = nullptr;
                    if (st >= 0 && (h->r[1] != rc->o1 || h->r[2] != rc->o2))
                        st = fail(TT_ERR_STATE, "adjoint replay: ranks differ from the taped run");
                }
                if (st < 0) break;
            }
            for (int m = seg_end - 1; m >= seg_start && st >= 0; --m) {
                const tt_ctx::StepRec* out = (m + 1 < M) ? h->tape[m + 1] : &fin;
                st = reverse_step(h, *h->tape[m], out->X.p, out->Th.p, out->Ph.p);
            }
            if (every > 1)
                for (int m = seg_start; m < seg_end; ++m) {
                    if (m != seg_start) h->tape[m]->release_state();
                    h->tape[m]->release_proj();
                }
            seg_end = seg_start;
        }
        if (st < 0) break;
        if (grad_dev)
            TT_CUDA_TRY(cudaMemcpyAsync(grad_dev, h->asigb.p, (size_t)nc * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s));
    } while (false);
    tt_status st2 = load_state(h, fin.X.p, fin.Th.p, fin.Ph.p, fin.T.p, fin.r1, fin.r2);
    if (st >= 0 && Q_host) {
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_dbl + HD_Q, h->d_dbl + HD_Q, sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
    }
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    if (st >= 0 && Q_host) *Q_host = h->h_dbl[HD_Q];
    fin.release();
    clear_tape(h);
    return st < 0 ? st : st2;
}

}  // namespace

// ============================================================== C ABI

namespace ttsn {
// One captured step for many handles: a graph with one branch per handle
// (forked from and joined to an origin stream through events, each branch
// the handle's graph_step_body on a capture stream of its own), so a batch
// step is one graph launch.  The branches are independent and run
// concurrently; every branch's arithmetic is its handle's captured step.
tt_status graph_batch_build(tt_handle* hs, int n, cudaGraphExec_t* out, unsigned* launches) {
    *out = nullptr;
    *launches = 0;
    for (int i = 0; i < n; ++i) {
        TT_TRY(check_handle(hs[i], true));
        if (!hs[i]->graph_on) return fail(TT_ERR_STATE, "captured steps are off for a handle of the batch");
        TT_TRY(graph_start(hs[i]));
        TT_CUDA_TRY(cudaStreamSynchronize(hs[i]->stream));
    }
    TT_TRY(eig_prepare());
    cudaStream_t origin = nullptr;
    TT_CUDA_TRY(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    std::vector<cudaStream_t> caps(n, nullptr);
    std::vector<cudaStream_t> saved(n, nullptr);
    std::vector<cudaEvent_t> evs(n + 1, nullptr);
    tt_status st = TT_OK;
    cudaGraph_t graph = nullptr;
    auto cleanup = [&]() {
        for (int i = 0; i < n; ++i) {
            if (saved[i]) hs[i]->stream = saved[i];
            if (caps[i]) cudaStreamDestroy(caps[i]);
        }
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        cudaStreamDestroy(origin);
    };
    for (int i = 0; i < n && st == TT_OK; ++i) {
        if (cudaStreamCreateWithFlags(&caps[i], cudaStreamNonBlocking) != cudaSuccess) st = TT_ERR_CUDA;
        else if (cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming) != cudaSuccess) st = TT_ERR_CUDA;
    }
    if (st == TT_OK && cudaEventCreateWithFlags(&evs[n], cudaEventDisableTiming) != cudaSuccess) st = TT_ERR_CUDA;
    if (st != TT_OK) {
        cleanup();
        return fail(st, "batched captured step: stream or event creation failed");
    }
    const unsigned long long before = t_launches;
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(evs[n], origin);
    for (int i = 0; i < n && e == cudaSuccess && st == TT_OK; ++i) {
        e = cudaStreamWaitEvent(caps[i], evs[n], 0);  // the branch joins the capture
        if (e != cudaSuccess) break;
        saved[i] = hs[i]->stream;
        hs[i]->stream = caps[i];
        st = graph_step_body(hs[i]);
        hs[i]->stream = saved[i];
        saved[i] = nullptr;
        if (st == TT_OK) e = cudaEventRecord(evs[i], caps[i]);
        if (st == TT_OK && e == cudaSuccess) e = cudaStreamWaitEvent(origin, evs[i], 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(origin, &graph);
    if (e == cudaSuccess) e = ee;
    *launches = (unsigned)(t_launches - before);
    g_launches.fetch_sub(*launches);
    t_launches -= *launches;
    if (st == TT_OK && e == cudaSuccess) {
        e = cudaGraphInstantiate(out, graph, 0);
        if (e != cudaSuccess) *out = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cleanup();
    if (st < 0) return st;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(TT_ERR_CUDA, std::string("batched captured step: ") + cudaGetErrorString(e));
    }
    return TT_OK;
}

// nsteps replays of a batch graph on `origin`, ordered after every handle's
// earlier work and before its later work (events on the handles' streams).
tt_status graph_batch_launch(tt_handle* hs, int n, cudaGraphExec_t exec, unsigned launches, cudaStream_t origin,
                             cudaEvent_t* evs, int nsteps) {
    for (int i = 0; i < n; ++i) {
        tt_ctx* h = hs[i];
        TT_TRY(graph_start(h));
        if (!h->ranks_stale) {  // the host's state: the size blocks start from its ranks
            int init[2] = {h->r[1], h->r[2]};
            TT_CUDA_TRY(cudaMemcpyAsync(h->dyn + DYN_R1, init, 2 * sizeof(int), cudaMemcpyHostToDevice, h->stream));
            TT_CUDA_TRY(cudaStreamSynchronize(h->stream));  // init lives on this frame
        }
        TT_CUDA_TRY(cudaEventRecord(evs[i], h->stream));
        TT_CUDA_TRY(cudaStreamWaitEvent(origin, evs[i], 0));
    }
    for (int it = 0; it < nsteps; ++it) {
        TT_CUDA_TRY(cudaGraphLaunch(exec, origin));
        note_launch(launches);
    }
    TT_CUDA_TRY(cudaEventRecord(evs[n], origin));
    for (int i = 0; i < n; ++i) {
        TT_CUDA_TRY(cudaStreamWaitEvent(hs[i]->stream, evs[n], 0));
        hs[i]->ranks_stale = true;
    }
    return TT_OK;
}

tt_status graph_steps_begin(tt_handle h, int nsteps) {
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!h->graph_on) return fail(TT_ERR_STATE, "captured steps are off for this handle");
    TT_TRY(graph_start(h));
    for (int it = 0; it < nsteps; ++it) TT_TRY(graph_launch(h));
    return TT_OK;
}
tt_status graph_steps_end(tt_handle h, tt_step_info* info) {
    AllocScope alloc_scope_(h->alloc_ptr());
    return graph_finish(h, info);
}
}  // namespace ttsn

extern "C" {

const char* tt_last_error(void) { return get_error(); }

tt_status tt_create(const tt_problem_desc* desc, void* stream, tt_handle* out) {
    return tt_create_ex(desc, stream, nullptr, out);
}

namespace {
struct ShardArgs {
    int p0, p1;
    tt_exchange_fn fn;
    void* ctx;
};

tt_status create_impl(const tt_problem_desc* desc, void* stream, const tt_allocator* alloc,
                      const ShardArgs* sh, tt_handle* out) {
    if (!desc || !out) return fail(TT_ERR_ARG, "tt_create: null argument");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(TT_ERR_ARG, "tt_create_ex: allocator needs both alloc and free");
    *out = nullptr;
    const tt_problem_desc& D = *desc;
    if (D.ndim < 1 || D.ndim > 3) return fail(TT_ERR_ARG, "tt_create: ndim must be 1, 2 or 3");
    long nc = 1;
    for (int a = 0; a < D.ndim; ++a) {
        if (D.n[a] < 1) return fail(TT_ERR_ARG, "tt_create: n[a] must be >= 1");
        if (!(D.L[a] > 0.0)) return fail(TT_ERR_ARG, "tt_create: L[a] must be > 0");
        if (D.bc[a] != TT_BC_PERIODIC && D.bc[a] != TT_BC_VACUUM && D.bc[a] != TT_BC_OUTFLOW)
            return fail(TT_ERR_ARG, "tt_create: bc must be TT_BC_PERIODIC, TT_BC_VACUUM or TT_BC_OUTFLOW");
        nc *= D.n[a];
    }
    if (nc > (1L << 31)) return fail(TT_ERR_TOO_LARGE, "tt_create: more than 2^31 cells");
    // a shard keeps the layers [p0, p1) of axis 0: its own cells start at
    // cell p0 * plane of the global C order
    long plane = 1;
    for (int a = 1; a < D.ndim; ++a) plane *= D.n[a];
    long cell0 = 0;
    if (sh) {
        if (!sh->fn) return fail(TT_ERR_ARG, "tt_create_shard: null exchange callback");
        if (sh->p0 < 0 || sh->p1 > D.n[0] || sh->p0 >= sh->p1)
            return fail(TT_ERR_ARG, "tt_create_shard: need 0 <= plane_begin < plane_end <= n[0]");
        if (D.layout != TT_LAYOUT_GROUPED)
            return fail(TT_ERR_ARG, "tt_create_shard: shards hold the grouped layout's spatial rows");
        if (D.flux == TT_FLUX_HLL || D.flux == TT_FLUX_RUSANOV_TAU)
            return fail(TT_ERR_ARG, "tt_create_shard: fluxes with per-face optical depths (HLL, Rusanov with "
                                    "the optical-depth speed) are not sharded; use upwind or Rusanov");
        cell0 = (long)sh->p0 * plane;
        nc = (long)(sh->p1 - sh->p0) * plane;
    }
    if (D.n_theta < 1 || D.n_phi < 1) return fail(TT_ERR_ARG, "tt_create: n_theta, n_phi must be >= 1");
    if (!(D.c > 0.0) || D.a_r < 0.0) return fail(TT_ERR_ARG, "tt_create: need c > 0, a_r >= 0");
    if (!(D.dt > 0.0) && !(D.cfl > 0.0)) return fail(TT_ERR_ARG, "tt_create: need dt > 0 or cfl > 0");
    if (!D.sigma_a || !D.cv || !D.T0) return fail(TT_ERR_ARG, "tt_create: sigma_a, cv, T0 are required");
    if (D.eps < 0.0) return fail(TT_ERR_ARG, "tt_create: eps must be >= 0");
    if (D.rounds_per_step != 1 && D.rounds_per_step != 2)
        return fail(TT_ERR_ARG, "tt_create: rounds_per_step must be 1 or 2");
    if (D.precision != TT_FP64 && D.precision != TT_MIXED)
        return fail(TT_ERR_ARG, "tt_create: precision must be TT_FP64 or TT_MIXED");
    if (D.layout != TT_LAYOUT_GROUPED && D.layout != TT_LAYOUT_SPLIT)
        return fail(TT_ERR_ARG, "tt_create: layout must be TT_LAYOUT_GROUPED or TT_LAYOUT_SPLIT");
    if (D.flux != TT_FLUX_UPWIND && D.flux != TT_FLUX_RUSANOV && D.flux != TT_FLUX_HLL &&
        D.flux != TT_FLUX_RUSANOV_TAU)
        return fail(TT_ERR_ARG, "tt_create: flux must be TT_FLUX_UPWIND, TT_FLUX_RUSANOV, TT_FLUX_HLL or "
                                "TT_FLUX_RUSANOV_TAU");
    if (D.flux == TT_FLUX_RUSANOV_TAU && !(D.flux_param[0] > 0.0 && D.flux_param[0] < 1e300))
        return fail(TT_ERR_ARG, "tt_create: Rusanov with the optical-depth speed needs flux_param[0] = beta > 0");
    if (D.flux == TT_FLUX_RUSANOV && !(D.flux_param[0] >= 0.0 && D.flux_param[0] < 1e300))
        return fail(TT_ERR_ARG, "tt_create: Rusanov needs flux_param[0] = S+/c >= 0");
    if (D.flux == TT_FLUX_HLL && !(D.flux_param[0] > 0.0 && D.flux_param[0] < 1e300 &&
                                   D.flux_param[1] > 0.0 && D.flux_param[1] <= sqrt(2.0)))
        return fail(TT_ERR_ARG, "tt_create: HLL needs flux_param = (beta > 0, 0 < tau_threshold <= sqrt 2)");
    double sig_a_uniform = 0.0, sig_s_uniform = 0.0;
    if (D.layout == TT_LAYOUT_SPLIT) {
        // the absorption factor s multiplies every spatial rank unless it is
        // one number, so the split layout takes uniform sigma_a and sigma_s
        std::vector<double> hv((size_t)nc);
        for (int pass = 0; pass < 2; ++pass) {
            const double* src = pass == 0 ? D.sigma_a : D.sigma_s;
            if (!src) continue;
            if (cudaMemcpy(hv.data(), src, nc * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(TT_ERR_ARG, "tt_create: sigma_a / sigma_s are not readable device arrays");
            }
            for (long i = 1; i < nc; ++i)
                if (hv[i] != hv[0])
                    return fail(TT_ERR_ARG, "tt_create: the split layout needs uniform sigma_a and "
                                            "sigma_s (use the grouped layout for varying fields)");
            (pass == 0 ? sig_a_uniform : sig_s_uniform) = hv[0];
        }
    }

    tt_ctx* h = new tt_ctx();
    if (alloc) {
        h->allocator = *alloc;
        h->has_allocator = true;
    }
    AllocScope alloc_scope_(h->alloc_ptr());
    cudaStream_t s = (cudaStream_t)stream;
    tt_status st = h->init_common(s);
    if (st < 0) {
        delete h;
        return st;
    }
    h->physics = true;
    h->d = 3;
    h->n[0] = (int)nc;
    h->n[1] = D.n_theta;
    h->n[2] = D.n_phi;
    h->r[0] = h->r[1] = h->r[2] = h->r[3] = 1;
    h->eps = D.eps;
    h->max_rank = D.max_rank > 0 ? D.max_rank : 0;
    h->rounds = D.rounds_per_step;
    h->precision = D.precision;
    Grid& g = h->grid;
    g.ndim = D.ndim;
    g.nc = nc;
    double dxmin = 1e300;
    h->dV = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < D.ndim ? D.n[a] : 1;
        g.dx[a] = a < D.ndim ? D.L[a] / D.n[a] : 1.0;
        g.bc[a] = a < D.ndim ? D.bc[a] : TT_BC_PERIODIC;
        if (a < D.ndim) {
            dxmin = std::min(dxmin, g.dx[a]);
            h->dV *= g.dx[a];
        }
    }
    if (sh) {
        // the shard's slab: axis 0 reads its ghost layers from the halo
        h->shard.on = true;
        h->shard.p0 = sh->p0;
        h->shard.p1 = sh->p1;
        h->shard.n0 = D.n[0];
        h->shard.bc0 = D.bc[0];
        h->shard.plane = plane;
        h->shard.fn = sh->fn;
        h->shard.ctx = sh->ctx;
        g.n[0] = sh->p1 - sh->p0;
        g.bc[0] = BC_HALO;
    }
    Fields& f = h->fields;
    f.c = D.c;
    f.a_r = D.a_r;
    f.dt = D.dt > 0.0 ? D.dt : D.cfl * dxmin / D.c;

    auto copy_field = [&](DevBuf& b, const double* srcp) -> tt_status {
        TT_TRY(b.ensure((size_t)nc, s));
        TT_CUDA_TRY(cudaMemcpyAsync(b.p, srcp + cell0, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return TT_OK;
    };
#define TT_CREATE_TRY(expr)      \
    do {                         \
        tt_status _s2 = (expr);  \
        if (_s2 < 0) {           \
            delete h;            \
            return _s2;          \
        }                        \
    } while (0)
    TT_CREATE_TRY(copy_field(h->f_sigma_a, D.sigma_a));
    TT_CREATE_TRY(copy_field(h->f_cv, D.cv));
    TT_CREATE_TRY(copy_field(h->f_T, D.T0));
    if (D.sigma_s) {
        TT_CREATE_TRY(copy_field(h->f_sigma_s, D.sigma_s));
        h->has_sigma_s = true;
    }
    TT_CREATE_TRY(h->f_Estar.ensure((size_t)nc, s));
    TT_CREATE_TRY(h->f_E.ensure((size_t)nc, s));
    TT_CREATE_TRY(h->red.ensure(4096, s));
    f.sigma_a = h->f_sigma_a.p;
    f.sigma_s = h->has_sigma_s ? h->f_sigma_s.p : nullptr;
    f.cv = h->f_cv.p;
    f.T = h->f_T.p;
    f.E_star = h->f_Estar.p;
    // interface flux: face weights (w_L1, w_R1, w_L2, w_R2) of Eq. upwind /
    // Eq. rusanov_flux_toro, or per cell from Eq. hll (grouped layout)
    f.flux = D.flux;
    if (D.flux == TT_FLUX_RUSANOV) {
        const double sp = D.flux_param[0];
        f.wc[0] = 0.5;
        f.wc[1] = 0.5;
        f.wc[2] = 0.5 * sp;
        f.wc[3] = -0.5 * sp;
    }
    if (D.flux == TT_FLUX_HLL && D.layout == TT_LAYOUT_GROUPED) {
        TT_CREATE_TRY(h->f_fw.ensure((size_t)nc * D.ndim * 8, s));
        hll_face_weights(s, g, h->f_sigma_a.p, h->has_sigma_s ? h->f_sigma_s.p : nullptr, D.flux_param[0],
                         D.flux_param[1], h->f_fw.p);
        f.fw = h->f_fw.p;
    }
    if (D.flux == TT_FLUX_RUSANOV_TAU && D.layout == TT_LAYOUT_GROUPED) {
        TT_CREATE_TRY(h->f_fw.ensure((size_t)nc * D.ndim * 8, s));
        rusanov_tau_face_weights(s, g, h->f_sigma_a.p, h->has_sigma_s ? h->f_sigma_s.p : nullptr,
                                 D.flux_param[0], h->f_fw.p);
        f.fw = h->f_fw.p;
    }
    for (int a = 0; a < D.ndim; ++a) {
        // the split layout's uniform stencils (all faces alike, opacities uniform)
        double w[4] = {f.wc[0], f.wc[1], f.wc[2], f.wc[3]};
        if (D.flux == TT_FLUX_HLL) {
            const double sig = sig_a_uniform + sig_s_uniform, thr = D.flux_param[1];
            const double tau = sig > 0.0 ? D.flux_param[0] * g.dx[a] * sig : 0.0;
            const double A = tau >= thr ? sqrt((1.0 - exp(-tau * tau)) / (tau * tau))
                                        : sqrt(std::max(1.0 - 0.5 * tau * tau, 0.0));
            const double B = tau >= thr ? sqrt((1.0 - exp(-tau * tau * tau * tau)) / (tau * tau)) : tau;
            w[0] = w[3] = A * (1.0 + B) / (A + B);
            w[1] = w[2] = B * (1.0 - A) / (A + B);
        }
        if (D.flux == TT_FLUX_RUSANOV_TAU) {
            const double sig = sig_a_uniform + sig_s_uniform;
            const double tau = sig > 0.0 ? D.flux_param[0] * g.dx[a] * sig : 0.0;
            const double m = tau > 1.0 ? 1.0 / tau : 1.0;
            w[0] = w[1] = 0.5;
            w[2] = 0.5 * m;
            w[3] = -0.5 * m;
        }
        for (int t = 0; t < 2; ++t) {
            h->split_co.c[a][t][0] = w[2 * t] - w[2 * t + 1];
            h->split_co.c[a][t][1] = w[2 * t + 1];
            h->split_co.c[a][t][2] = w[2 * t];
        }
    }

    // angular grid (Sec. 3): mu and phi at cell centres, uniform weights
    Angular& A = h->ang;
    A.n_theta = D.n_theta;
    A.n_phi = D.n_phi;
    A.w = 2.0 / D.n_theta;
    A.v = 2.0 * M_PI / D.n_phi;
    const int KT = 1 + 2 * D.ndim;  // transport terms
    std::vector<double> hbuf(2 * D.n_theta + 2 * D.n_phi + (size_t)KT * (D.n_theta + D.n_phi));
    for (int l = 0; l < D.n_theta; ++l) {
        const double mu = -1.0 + (l + 0.5) * A.w;
        hbuf[l] = mu;
        hbuf[D.n_theta + l] = sqrt(1.0 - mu * mu);
    }
    for (int p = 0; p < D.n_phi; ++p) {
        const double ph = (p + 0.5) * A.v;
        hbuf[2 * D.n_theta + p] = cos(ph);
        hbuf[2 * D.n_theta + D.n_phi + p] = sin(ph);
    }
    {
        // per-term angular factors (Sec. 4.3): term 0 is I itself; term (a, 1)
        // and (a, 2) carry n_a^+ and n_a^- (upwind, HLL), n_a and 1 (Rusanov)
        // or n_a and |n_a| (Rusanov with the optical-depth speed), with
        // n_x = sin(theta) cos(phi), n_y = sin(theta) sin(phi), n_z = mu
        double* tf = hbuf.data() + 2 * D.n_theta + 2 * D.n_phi;
        double* pf = tf + (size_t)KT * D.n_theta;
        const bool rt = D.flux == TT_FLUX_RUSANOV_TAU;
        const bool rus = D.flux == TT_FLUX_RUSANOV || rt;
        for (int j = 0; j < KT; ++j) {
            const int axis = (j - 1) >> 1, second = (j - 1) & 1;
            const bool absn = rt && second;  // |n_a| = sin(theta) |cos phi|, sin(theta) |sin phi|, |mu|
            for (int l = 0; l < D.n_theta; ++l) {
                const double mu = hbuf[l], st = hbuf[D.n_theta + l];
                double v = 1.0;
                if (j > 0 && !(rus && second && !absn)) {
                    if (axis < 2)
                        v = st;
                    else if (absn)
                        v = std::fabs(mu);
                    else
                        v = rus ? mu : (second ? std::min(mu, 0.0) : std::max(mu, 0.0));
                }
                tf[(size_t)j * D.n_theta + l] = v;
            }
            for (int p = 0; p < D.n_phi; ++p) {
                const double cp = hbuf[2 * D.n_theta + p], sp = hbuf[2 * D.n_theta + D.n_phi + p];
                double v = 1.0;
                if (j > 0 && !(rus && second && !absn) && axis < 2) {
                    const double n = axis == 0 ? cp : sp;
                    v = absn ? std::fabs(n) : (rus ? n : (second ? std::min(n, 0.0) : std::max(n, 0.0)));
                }
                pf[(size_t)j * D.n_phi + p] = v;
            }
        }
    }
    {
        const double* tf = hbuf.data() + 2 * D.n_theta + 2 * D.n_phi;
        h->h_tfac.assign(tf, tf + (size_t)KT * D.n_theta);
        h->h_pfac.assign(tf + (size_t)KT * D.n_theta, tf + (size_t)KT * (D.n_theta + D.n_phi));
    }
    TT_CREATE_TRY(h->ang_buf.ensure(hbuf.size(), s));
    A.mu = h->ang_buf.p;
    A.sint = A.mu + D.n_theta;
    A.cphi = A.sint + D.n_theta;
    A.sphi = A.cphi + D.n_phi;
    A.tfac = A.sphi + D.n_phi;
    A.pfac = A.tfac + (size_t)KT * D.n_theta;
    if (cudaMemcpyAsync(h->ang_buf.p, hbuf.data(), hbuf.size() * sizeof(double),
                        cudaMemcpyHostToDevice, s) != cudaSuccess) {
        delete h;
        return fail(TT_ERR_CUDA, "tt_create: angular grid upload failed");
    }
    if (D.layout == TT_LAYOUT_SPLIT) {
        // cores x[, y[, z]], theta, phi
        h->layout = TT_LAYOUT_SPLIT;
        const int nd = D.ndim;
        h->d = nd + 2;
        for (int a = 0; a < nd; ++a) h->n[a] = D.n[a];
        h->n[nd] = D.n_theta;
        h->n[nd + 1] = D.n_phi;
        for (int k = 0; k <= h->d; ++k) h->r[k] = 1;
        // per-term angular factors of the split cores: theta carries -nu_a times
        // the term's theta factor, phi the term's phi factor (the tables above)
        const int K = 1 + 2 * nd;
        std::vector<double> fac((size_t)K * (D.n_theta + D.n_phi));
        double* thf = fac.data();
        double* phf = thf + (size_t)K * D.n_theta;
        const double* tf0 = hbuf.data() + 2 * D.n_theta + 2 * D.n_phi;
        const double* pf0 = tf0 + (size_t)K * D.n_theta;
        for (int j = 0; j < K; ++j) {
            const int axis = (j - 1) >> 1;
            const double nu = j == 0 ? 0.0 : f.c * f.dt / g.dx[axis];
            for (int l = 0; l < D.n_theta; ++l)
                thf[(size_t)j * D.n_theta + l] = j == 0 ? 1.0 : -nu * tf0[(size_t)j * D.n_theta + l];
            for (int p = 0; p < D.n_phi; ++p) phf[(size_t)j * D.n_phi + p] = pf0[(size_t)j * D.n_phi + p];
        }
        TT_CREATE_TRY(h->split_fac.ensure(fac.size(), s));
        if (cudaMemcpyAsync(h->split_fac.p, fac.data(), fac.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s) != cudaSuccess) {
            delete h;
            return fail(TT_ERR_CUDA, "tt_create: split factor upload failed");
        }
        h->split_s = 1.0 / (1.0 + f.c * f.dt * sig_a_uniform + f.c * f.dt * sig_s_uniform);
        // initial TT: the isotropic equilibrium intensity held exactly (the
        // emission term's block structure with I0 in the field block), then
        // rounded to the problem's tolerance and rank cap
        int er[TT_MAX_D + 1];
        split_emission_ranks(h, er);
        for (int k = 0; k < h->d; ++k) {
            TT_CREATE_TRY(h->gcore[k].ensure((size_t)er[k] * h->n[k] * er[k + 1], s));
            const SplitCoreSpec c = split_spec(h, k, 0, true, h->r, er, 1.0);
            split_grow_core(s, c, nullptr, nullptr, h->gcore[k].p);
        }
        init_isotropic(s, nc, D.Tr0 ? D.Tr0 : D.T0, D.c, D.a_r, h->gcore[nd == 1 ? 0 : 1].p);
        int rr[TT_MAX_D + 1];
        TT_CREATE_TRY(round_cores(h, h->gcore, er, h->core, rr, h->eps, h->max_rank, nullptr, nullptr));
        for (int k = 0; k <= h->d; ++k) h->r[k] = rr[k];
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            delete h;
            return fail(TT_ERR_CUDA, "tt_create: initialisation failed");
        }
        *out = h;
        return TT_OK;
    }
    // initial TT: isotropic equilibrium intensity with Tr0, rank (1, 1)
    TT_CREATE_TRY(h->core[0].ensure((size_t)nc, s));
    TT_CREATE_TRY(h->core[1].ensure((size_t)D.n_theta, s));
    TT_CREATE_TRY(h->core[2].ensure((size_t)D.n_phi, s));
    if (h->max_rank > 0) {
        // capacity reservation for the capped case: the largest cores and Gram
        // workspaces a step can need, so steps do not allocate while ranks grow
        const long cap1 = std::min<long>(h->max_rank, std::min<long>(nc, (long)D.n_theta * D.n_phi));
        const long cap2 = std::min<long>(h->max_rank, D.n_phi);
        const long nterms = 1 + 2 * D.ndim;
        const long R1 = nterms * cap1 + 1, R2 = nterms * cap2 + 1;
        TT_CREATE_TRY(h->core[0].ensure((size_t)(nc * cap1), s));
        TT_CREATE_TRY(h->core[1].ensure((size_t)(R1 * D.n_theta * R2), s));
        TT_CREATE_TRY(h->core[2].ensure((size_t)(R2 * D.n_phi), s));
        TT_CREATE_TRY(h->gcore[0].ensure((size_t)(nc * R1), s));
        TT_CREATE_TRY(h->gcore[1].ensure((size_t)(R1 * D.n_theta * R2), s));
        TT_CREATE_TRY(h->gcore[2].ensure((size_t)(R2 * D.n_phi), s));
        TT_CREATE_TRY(h->GA.ensure((size_t)(R1 * R1), s));
        TT_CREATE_TRY(h->partials.ensure(D.precision == TT_MIXED
                                              ? slgram_scratch_doubles((int)nc, (int)R1)
                                              : gram_scratch_doubles((int)nc, (int)R1), s));
        for (int k = 0; k < 2; ++k) {
            const long Rk = k == 0 ? R1 : R2;
            TT_CREATE_TRY(h->GB[k].ensure((size_t)(Rk * Rk), s));
            TT_CREATE_TRY(h->VtB[k].ensure((size_t)(Rk * Rk), s));
            TT_CREATE_TRY(h->lamB[k].ensure((size_t)(2 * Rk), s));
        }
        // rounding workspaces at their largest (bond 1 of a capped step)
        const size_t RR = (size_t)(R1 * R1);
        DevBuf* sq[] = {&h->Wc, &h->T1, &h->K, &h->VtK, &h->eig.g0, &h->eig.g1, &h->eig.vt_unsorted};
        for (DevBuf* b : sq) TT_CREATE_TRY(b->ensure(RR, s));
        TT_CREATE_TRY(h->lamK.ensure((size_t)R1, s));
        TT_CREATE_TRY(h->eig.lam_unsorted.ensure((size_t)R1, s));
        TT_CREATE_TRY(h->eig.abc.ensure((size_t)(3 * (R1 + 1)), s));
        TT_CREATE_TRY(h->eig.cs.ensure((size_t)(R1 + 1), s));
        TT_CREATE_TRY(h->Vts.ensure((size_t)(cap1 * R1), s));
        TT_CREATE_TRY(h->PAt.ensure((size_t)(cap1 * R1), s));
        TT_CREATE_TRY(h->Mupd.ensure((size_t)(cap1 * R1), s));
        TT_CREATE_TRY(h->bwd.ensure((size_t)(R1 * D.n_theta * R2), s));
        TT_CREATE_TRY(h->tmp[0].ensure((size_t)(cap1 * D.n_theta * R2), s));
        TT_CREATE_TRY(h->tmp[1].ensure((size_t)(cap1 * D.n_theta * R2), s));
        TT_CREATE_TRY(h->thbar.ensure((size_t)(nterms * (cap1 + cap2) + 2), s));
        TT_CREATE_TRY(h->ydots.ensure((size_t)(nc * nterms), s));
        if (D.precision == TT_MIXED) {
            TT_CREATE_TRY(h->slscratch.ensure((size_t)(nc + R1) / 2 + 2, s));
            TT_CREATE_TRY(h->erowA.ensure((size_t)(nc + 1) / 2, s));
        }
    }
    init_isotropic(s, nc, (D.Tr0 ? D.Tr0 : D.T0) + cell0, D.c, D.a_r, h->core[0].p);
    fill(s, h->core[1].p, D.n_theta, 1.0);
    fill(s, h->core[2].p, D.n_phi, 1.0);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        delete h;
        return fail(TT_ERR_CUDA, "tt_create: initialisation failed");
    }
#undef TT_CREATE_TRY
    *out = h;
    return TT_OK;
}

}  // namespace

tt_status tt_create_ex(const tt_problem_desc* desc, void* stream, const tt_allocator* alloc,
                       tt_handle* out) {
    set_error("");
    return create_impl(desc, stream, alloc, nullptr, out);
}

tt_status tt_create_shard(const tt_problem_desc* desc, void* stream, int plane_begin, int plane_end,
                          tt_exchange_fn exchange, void* ctx, tt_handle* out) {
    set_error("");
    const ShardArgs sh{plane_begin, plane_end, exchange, ctx};
    return create_impl(desc, stream, nullptr, &sh, out);
}

tt_status tt_create_tt(int d, const int* n, const int* ranks, void* stream, tt_handle* out) {
    set_error("");
    if (!out || !n || !ranks) return fail(TT_ERR_ARG, "tt_create_tt: null argument");
    *out = nullptr;
    if (d < 1 || d > TT_MAX_D) return fail(TT_ERR_ARG, "tt_create_tt: d out of range");
    if (ranks[0] != 1 || ranks[d] != 1) return fail(TT_ERR_ARG, "tt_create_tt: ranks[0] and ranks[d] must be 1");
    for (int k = 0; k < d; ++k) {
        if (n[k] < 1) return fail(TT_ERR_ARG, "tt_create_tt: mode sizes must be >= 1");
        if (ranks[k + 1] < 1) return fail(TT_ERR_ARG, "tt_create_tt: ranks must be >= 1");
    }
    tt_ctx* h = new tt_ctx();
    cudaStream_t s = (cudaStream_t)stream;
    tt_status st = h->init_common(s);
    if (st < 0) {
        delete h;
        return st;
    }
    h->d = d;
    for (int k = 0; k < d; ++k) h->n[k] = n[k];
    for (int k = 0; k <= d; ++k) h->r[k] = ranks[k];
    for (int k = 0; k < d; ++k) {
        st = h->core[k].ensure(h->core_len(k, h->r), s);
        if (st < 0) {
            delete h;
            return st;
        }
        fill(s, h->core[k].p, h->core_len(k, h->r), 0.0);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        delete h;
        return fail(TT_ERR_CUDA, "tt_create_tt: initialisation failed");
    }
    *out = h;
    return TT_OK;
}

tt_status tt_sn_step_ex(tt_handle h, int nsteps, int flags, const int* forced, tt_step_info* info) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (nsteps < 0) return fail(TT_ERR_ARG, "tt_sn_step: nsteps < 0");
    if (flags & ~(TT_STEP_NO_SOURCE | TT_STEP_NO_ROUND)) return fail(TT_ERR_ARG, "tt_sn_step: unknown flag");
    const int nforced = (h->rounds == 2 && !(flags & (TT_STEP_NO_SOURCE | TT_STEP_NO_ROUND))) ? 2 * (h->d - 1) : h->d - 1;
    if (forced)
        for (int k = 0; k < nforced; ++k)
            if (forced[k] < 1) return fail(TT_ERR_ARG, "tt_sn_step: forced ranks must be >= 1");
    tt_status result = TT_OK;
    if (h->graph_on && flags == 0 && !forced && nsteps > 0) {
        // captured steps: replay the recorded step, one synchronisation at the end
        TT_TRY(graph_start(h));
        for (int it = 0; it < nsteps; ++it) TT_TRY(graph_launch(h));
        return graph_finish(h, info);
    }
    for (int it = 0; it < nsteps; ++it) {
        nvtxRangePushA("tt_sn_step");
        tt_status st = step_once(h, flags, forced, info);
        nvtxRangePop();
        if (st < 0) return st;
        if (st == TT_WARN_RANK_CAPPED) result = st;
    }
    tt_status st = read_status(h);
    if (st < 0) return st;
    return result;
}


tt_status tt_set_graph(tt_handle h, int enable) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (enable) {
        if (const char* why = graph_unsupported(h)) return fail(TT_ERR_STATE, std::string("tt_set_graph: ") + why);
        h->graph_on = true;
    } else {
        h->graph_on = false;
    }
    return TT_OK;
}

tt_status tt_sn_step(tt_handle h, int nsteps, tt_step_info* info) {
    return tt_sn_step_ex(h, nsteps, 0, nullptr, info);
}

tt_status tt_tape_begin(tt_handle h, int checkpoint_every) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (checkpoint_every < 1) return fail(TT_ERR_ARG, "tt_tape_begin: checkpoint_every must be >= 1");
    if (h->shard.on) return fail(TT_ERR_STATE, "tt_tape_begin: a spatial shard has no adjoint tape");
    if (h->precision != TT_FP64 || h->rounds != 1 || h->has_sigma_s || h->d != 3 || h->nsrc > 0 ||
        h->split() || h->round_method != TT_ROUND_GRAM || h->fields.flux != TT_FLUX_UPWIND ||
        h->grid.bc[0] == TT_BC_OUTFLOW ||
        h->grid.bc[1] == TT_BC_OUTFLOW || h->grid.bc[2] == TT_BC_OUTFLOW)
        return fail(TT_ERR_STATE, "tt_tape_begin: the adjoint form needs the grouped layout, "
                                  "upwinding, periodic or vacuum faces, FP64 precision, one rounding "
                                  "per step, no scattering and no external sources");
    clear_tape(h);
    h->taping = true;
    h->tape_every = checkpoint_every;
    h->h_dbl[HD_Q] = 0.0;
    TT_CUDA_TRY(cudaMemcpyAsync(h->d_dbl + HD_Q, h->h_dbl + HD_Q, sizeof(double),
                                cudaMemcpyHostToDevice, h->stream));
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return TT_OK;
}

tt_status tt_tape_objective(tt_handle h, double* Q_host, int* steps_host) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!Q_host) return fail(TT_ERR_ARG, "tt_tape_objective: null Q");
    TT_CUDA_TRY(cudaMemcpyAsync(h->h_dbl + HD_Q, h->d_dbl + HD_Q, sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    *Q_host = h->h_dbl[HD_Q];
    if (steps_host) *steps_host = (int)h->tape.size();
    return TT_OK;
}

tt_status tt_sn_step_adjoint(tt_handle h, double* grad_sigma_a_dev, double* Q_host) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!h->taping && h->tape.empty()) return fail(TT_ERR_STATE, "tt_sn_step_adjoint: no tape");
    tt_status st = adjoint_run(h, grad_sigma_a_dev, Q_host);
    if (st < 0) return st;
    return read_status(h);
}

tt_status tt_tape_clear(tt_handle h) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    clear_tape(h);
    return TT_OK;
}

tt_status tt_round(tt_handle h, double eps, int max_rank, const int* forced, tt_step_info* info) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    clear_tape(h);  // a change of state outside a step ends the tape
    if (eps < 0.0) return fail(TT_ERR_ARG, "tt_round: eps < 0");
    if (forced)
        for (int k = 0; k < h->d - 1; ++k)
            if (forced[k] < 1) return fail(TT_ERR_ARG, "tt_round: forced ranks must be >= 1");
    // current TT becomes the rounding source
    for (int k = 0; k < h->d; ++k) std::swap(h->core[k], h->gcore[k]);
    for (int k = 0; k <= h->d; ++k) h->gr[k] = h->r[k];
    int rr[TT_MAX_D + 1];
    tt_status st = round_cores(h, h->gcore, h->gr, h->core, rr, eps, max_rank > 0 ? max_rank : 0,
                               forced, info);
    if (st < 0) return st;
    for (int k = 0; k <= h->d; ++k) h->r[k] = rr[k];
    if (info)
        for (int k = 0; k <= h->d; ++k) info->ranks[k] = h->r[k];
    tt_status st2 = read_status(h);
    if (st2 < 0) return st2;
    return st;
}

tt_status tt_energy(tt_handle h, double* E_dev, double* T_dev, double* totals_host) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    cudaStream_t s = h->stream;
    const long nc = h->grid.nc;
    double* E = E_dev ? E_dev : h->f_E.p;
    if (h->split()) {
        TT_TRY(split_energy_field(h));
        energy_rows(s, nc, 1, h->sp_F.p, 1, h->d_dbl + HD_ONE, h->fields.c, E, nullptr, nullptr,
                    nullptr, false);
    } else {
        const int r1 = h->r[1], r2 = h->r[2];
        TT_TRY(h->thbar.ensure((size_t)(r1 + r2), s));
        plain_thbar(s, h->ang, r1, r2, h->core[1].p, h->core[2].p, h->thbar.p);
        energy_rows(s, nc, r1, h->core[0].p, r1, h->thbar.p, h->fields.c, E, nullptr, nullptr,
                    nullptr, false);
    }
    if (T_dev)
        TT_CUDA_TRY(cudaMemcpyAsync(T_dev, h->f_T.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (totals_host) {
        energy_totals(s, nc, E, h->f_cv.p, h->f_T.p, h->red.p + 2048, h->red.p);
        if (h->shard.on) TT_TRY(shard_exchange(h, TT_XCHG_SUM, h->red.p + 2048, 2));
        TT_CUDA_TRY(cudaMemcpyAsync(h->h_dbl + HD_TOT, h->red.p + 2048, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
    }
    TT_CUDA_TRY(cudaGetLastError());
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    if (totals_host) {
        totals_host[0] = h->h_dbl[HD_TOT] * h->dV;
        totals_host[1] = h->h_dbl[HD_TOT + 1] * h->dV;
    }
    return TT_OK;
}

tt_status tt_to_full(tt_handle h, double* out_dev, size_t out_len) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!out_dev) return fail(TT_ERR_ARG, "tt_to_full: null output");
    cudaStream_t s = h->stream;
    const int d = h->d;
    size_t total = 1;
    for (int k = 0; k < d; ++k) total *= (size_t)h->n[k];
    if (out_len < total) return fail(TT_ERR_TOO_LARGE, "tt_to_full: output buffer too small");
    if (d == 1) {
        TT_CUDA_TRY(cudaMemcpyAsync(out_dev, h->core[0].p, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return TT_OK;
    }
    // right-to-left: T_k = core_k (r_k n_k x r_{k+1}) * T_{k+1} (r_{k+1} x prod n_{k+1:})
    long cols = h->n[d - 1];
    const double* T = h->core[d - 1].p;  // (r_{d-1} x n_{d-1})
    int ti = 0;
    for (int k = d - 2; k >= 0; --k) {
        const long rows = (long)h->r[k] * h->n[k];
        double* outp;
        if (k == 0) {
            outp = out_dev;
        } else {
            TT_TRY(h->tmp[ti].ensure((size_t)rows * cols, s));
            outp = h->tmp[ti].p;
            ti ^= 1;
        }
        TT_TRY(dgemm(s, false, false, (int)rows, (int)cols, h->r[k + 1], 1.0, h->core[k].p,
                     h->r[k + 1], T, cols, 0.0, outp, cols));
        T = outp;
        cols *= h->n[k];
    }
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    return TT_OK;
}

tt_status tt_get_ranks(tt_handle h, int* ranks_host, int cap) {
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!ranks_host) return fail(TT_ERR_ARG, "tt_get_ranks: null output");
    for (int k = 0; k <= h->d && k < cap; ++k) ranks_host[k] = h->r[k];
    return TT_OK;
}

tt_status tt_get_dims(tt_handle h, int* d_host, int* n_host) {
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (d_host) *d_host = h->d;
    if (n_host)
        for (int k = 0; k < h->d; ++k) n_host[k] = h->n[k];
    return TT_OK;
}

tt_status tt_get_core(tt_handle h, int k, double* out_dev, size_t out_len) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (k < 0 || k >= h->d) return fail(TT_ERR_ARG, "tt_get_core: k out of range");
    const size_t len = h->core_len(k, h->r);
    if (out_len < len) return fail(TT_ERR_TOO_LARGE, "tt_get_core: output buffer too small");
    // device or host destination (unified addressing infers the direction)
    TT_CUDA_TRY(cudaMemcpyAsync(out_dev, h->core[k].p, len * sizeof(double), cudaMemcpyDefault, h->stream));
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return TT_OK;
}

tt_status tt_get_cores(tt_handle h, double** cores_dev, int* shapes_host) {
    set_error("");
    TT_TRY(check_handle(h, false));
    if (!cores_dev || !shapes_host) return fail(TT_ERR_ARG, "tt_get_cores: null argument");
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < h->d; ++k) {
        cores_dev[k] = h->core[k].p;
        shapes_host[3 * k] = h->r[k];
        shapes_host[3 * k + 1] = h->n[k];
        shapes_host[3 * k + 2] = h->r[k + 1];
    }
    return TT_OK;
}

tt_status tt_set_cores(tt_handle h, const double* const* cores_dev, const int* ranks_host) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    clear_tape(h);  // a change of state outside a step ends the tape
    if (!cores_dev || !ranks_host) return fail(TT_ERR_ARG, "tt_set_cores: null argument");
    if (ranks_host[0] != 1 || ranks_host[h->d] != 1)
        return fail(TT_ERR_ARG, "tt_set_cores: ranks[0] and ranks[d] must be 1");
    for (int k = 1; k < h->d; ++k)
        if (ranks_host[k] < 1) return fail(TT_ERR_ARG, "tt_set_cores: ranks must be >= 1");
    for (int k = 0; k < h->d; ++k) {
        const size_t len = h->core_len(k, ranks_host);
        TT_TRY(h->core[k].ensure(len, h->stream));
        // device or host source (unified addressing infers the direction)
        TT_CUDA_TRY(cudaMemcpyAsync(h->core[k].p, cores_dev[k], len * sizeof(double), cudaMemcpyDefault,
                                    h->stream));
    }
    for (int k = 0; k <= h->d; ++k) h->r[k] = ranks_host[k];
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return TT_OK;
}

namespace {
// src_* = the caller's sources, then two rank-one terms per inflow face (one
// for upwinding, whose other face weight is zero): column x from
// inflow_source, angular profiles the term's angular factor times the face's,
// and every profile's quadrature q_k = (w sum_l theta_k)(v sum_p phi_k).
tt_status rebuild_sources(tt_ctx* h) {
    cudaStream_t s = h->stream;
    const long nc = h->grid.nc;
    const int nt = h->ang.n_theta, np = h->ang.n_phi;
    struct Item {
        int a, side, t;
    };
    std::vector<Item> items;
    for (int a = 0; a < h->grid.ndim; ++a)
        for (int side = 0; side < 2; ++side) {
            if (!h->inflow[a][side].on) continue;
            for (int t = 0; t < 2; ++t) {
                if (h->fields.flux == TT_FLUX_UPWIND && t != side) continue;  // w_L2 = w_R1 = 0
                items.push_back({a, side, t});
            }
        }
    const int count = h->nusr + (int)items.size();
    h->nsrc = 0;
    if (count > TT_MAX_SOURCES)
        return fail(TT_ERR_ARG, "sources plus inflow-face terms exceed TT_MAX_SOURCES");
    if (count == 0) return TT_OK;
    TT_TRY(h->src_x.ensure((size_t)count * nc, s));
    TT_TRY(h->src_th.ensure((size_t)count * nt, s));
    TT_TRY(h->src_ph.ensure((size_t)count * np, s));
    TT_TRY(h->src_q.ensure((size_t)count, s));
    std::vector<double> th((size_t)count * nt), ph((size_t)count * np), q(count);
    if (h->nusr > 0) {
        const int u = h->nusr;
        TT_CUDA_TRY(cudaMemcpyAsync(h->src_x.p, h->usr_x.p, (size_t)u * nc * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        TT_CUDA_TRY(cudaMemcpyAsync(th.data(), h->usr_th.p, (size_t)u * nt * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaMemcpyAsync(ph.data(), h->usr_ph.p, (size_t)u * np * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
    }
    for (size_t k = 0; k < items.size(); ++k) {
        const Item& it = items[k];
        const tt_ctx::InflowFace& face = h->inflow[it.a][it.side];
        const int col = h->nusr + (int)k, j = 1 + 2 * it.a + it.t;
        inflow_source(s, h->grid, h->fields, it.a, it.side, it.t, face.g.p, h->src_x.p + (size_t)col * nc);
        for (int l = 0; l < nt; ++l) th[(size_t)col * nt + l] = h->h_tfac[(size_t)j * nt + l] * face.th[l];
        for (int p = 0; p < np; ++p) ph[(size_t)col * np + p] = h->h_pfac[(size_t)j * np + p] * face.ph[p];
    }
    TT_CUDA_TRY(cudaGetLastError());
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < count; ++k) {
        double a = 0.0, b = 0.0;
        for (int l = 0; l < nt; ++l) a += th[(size_t)k * nt + l];
        for (int p = 0; p < np; ++p) b += ph[(size_t)k * np + p];
        q[k] = (h->ang.w * a) * (h->ang.v * b);
    }
    TT_CUDA_TRY(cudaMemcpyAsync(h->src_th.p, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->src_ph.p, ph.data(), ph.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TT_CUDA_TRY(cudaMemcpyAsync(h->src_q.p, q.data(), q.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    h->nsrc = count;
    return TT_OK;
}
}  // namespace

tt_status tt_set_sources(tt_handle h, int count, const double* x_dev, const double* theta_dev,
                         const double* phi_dev) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (count < 0 || count > TT_MAX_SOURCES)
        return fail(TT_ERR_ARG, "tt_set_sources: count out of range");
    if (count > 0 && (!x_dev || !theta_dev || !phi_dev))
        return fail(TT_ERR_ARG, "tt_set_sources: null source array");
    if (count > 0 && h->split())
        return fail(TT_ERR_STATE, "tt_set_sources: fixed sources need the grouped layout");
    if (count > 0 && h->shard.on)
        return fail(TT_ERR_STATE, "tt_set_sources: a spatial shard takes no fixed sources");
    clear_tape(h);  // a change of state outside a step ends the tape
    cudaStream_t s = h->stream;
    const long nc = h->grid.nc;
    const int nt = h->ang.n_theta, np = h->ang.n_phi;
    int inflow_terms = 0;
    for (auto& ax : h->inflow)
        for (auto& face : ax) inflow_terms += face.on ? 2 : 0;
    if (count + inflow_terms > TT_MAX_SOURCES)
        return fail(TT_ERR_ARG, "tt_set_sources: sources plus inflow-face terms exceed TT_MAX_SOURCES");
    h->nusr = 0;
    if (count > 0) {
        TT_TRY(h->usr_x.ensure((size_t)count * nc, s));
        TT_TRY(h->usr_th.ensure((size_t)count * nt, s));
        TT_TRY(h->usr_ph.ensure((size_t)count * np, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->usr_x.p, x_dev, (size_t)count * nc * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->usr_th.p, theta_dev, (size_t)count * nt * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->usr_ph.p, phi_dev, (size_t)count * np * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
        h->nusr = count;
    }
    return rebuild_sources(h);
}

tt_status tt_set_inflow(tt_handle h, int axis, int side, const double* g_dev, const double* theta_dev,
                        const double* phi_dev) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (axis < 0 || axis >= h->grid.ndim || (side != 0 && side != 1))
        return fail(TT_ERR_ARG, "tt_set_inflow: axis or side out of range");
    if (h->grid.bc[axis] != TT_BC_VACUUM)
        return fail(TT_ERR_ARG, "tt_set_inflow: the axis must have vacuum faces");
    if (g_dev && (!theta_dev || !phi_dev)) return fail(TT_ERR_ARG, "tt_set_inflow: null angular profile");
    if (g_dev && h->split())
        return fail(TT_ERR_STATE, "tt_set_inflow: inflow faces need the grouped layout");
    if (g_dev && h->shard.on)
        return fail(TT_ERR_STATE, "tt_set_inflow: a spatial shard takes no inflow faces");
    clear_tape(h);
    cudaStream_t s = h->stream;
    tt_ctx::InflowFace& face = h->inflow[axis][side];
    const bool was_on = face.on;
    face.on = false;
    if (g_dev) {
        int terms = h->nusr;
        for (auto& ax : h->inflow)
            for (auto& f2 : ax) terms += f2.on ? 2 : 0;
        if (terms + 2 > TT_MAX_SOURCES) {
            face.on = was_on;
            return fail(TT_ERR_ARG, "tt_set_inflow: sources plus inflow-face terms exceed TT_MAX_SOURCES");
        }
        const long nc = h->grid.nc;
        const int nt = h->ang.n_theta, np = h->ang.n_phi;
        TT_TRY(face.g.ensure((size_t)nc, s));
        TT_CUDA_TRY(cudaMemcpyAsync(face.g.p, g_dev, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
        face.th.resize(nt);
        face.ph.resize(np);
        TT_CUDA_TRY(cudaMemcpyAsync(face.th.data(), theta_dev, nt * sizeof(double), cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaMemcpyAsync(face.ph.data(), phi_dev, np * sizeof(double), cudaMemcpyDeviceToHost, s));
        TT_CUDA_TRY(cudaStreamSynchronize(s));
        face.on = true;
    }
    return rebuild_sources(h);
}

tt_status tt_set_sketch(tt_handle h, const double* const* omega_dev, const int* ranks_host) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (!omega_dev) {
        h->has_sketch = false;
        if (h->round_method == TT_ROUND_RANDOMIZED) h->round_method = TT_ROUND_GRAM;
        return TT_OK;
    }
    if (!ranks_host) return fail(TT_ERR_ARG, "tt_set_sketch: null ranks");
    const int d = h->d;
    if (ranks_host[0] != 1 || ranks_host[d] != 1) return fail(TT_ERR_ARG, "tt_set_sketch: end ranks must be 1");
    for (int k = 1; k < d; ++k)
        if (ranks_host[k] < 1) return fail(TT_ERR_ARG, "tt_set_sketch: ranks must be >= 1");
    for (int k = 0; k < d; ++k)
        if (!omega_dev[k]) return fail(TT_ERR_ARG, "tt_set_sketch: null core");
    cudaStream_t s = h->stream;
    for (int k = 0; k < d; ++k) {
        const size_t len = (size_t)ranks_host[k] * h->n[k] * ranks_host[k + 1];
        TT_TRY(h->sketch[k].ensure(len, s));
        TT_CUDA_TRY(cudaMemcpyAsync(h->sketch[k].p, omega_dev[k], len * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    for (int k = 0; k <= d; ++k) h->sk_L[k] = ranks_host[k];
    TT_CUDA_TRY(cudaStreamSynchronize(s));
    h->has_sketch = true;
    return TT_OK;
}

tt_status tt_set_eigensolver(tt_handle h, int method) {
    set_error("");
    TT_TRY(check_handle(h, false));
    if (method != TT_EIG_ONE_SIDED && method != TT_EIG_TWO_SIDED)
        return fail(TT_ERR_ARG, "tt_set_eigensolver: method must be TT_EIG_ONE_SIDED or TT_EIG_TWO_SIDED");
    if (h->graph_on && method != h->eig_method)
        return fail(TT_ERR_STATE, "tt_set_eigensolver: captured steps are on (tt_set_graph 0 first)");
    h->eig_method = method;
    return TT_OK;
}

tt_status tt_set_rounding(tt_handle h, int method) {
    set_error("");
    TT_TRY(check_handle(h, false));
    if (method != TT_ROUND_GRAM && method != TT_ROUND_RANDOMIZED && method != TT_ROUND_TTSVD)
        return fail(TT_ERR_ARG,
                    "tt_set_rounding: method must be TT_ROUND_GRAM, TT_ROUND_RANDOMIZED or TT_ROUND_TTSVD");
    if (method == TT_ROUND_RANDOMIZED && !h->has_sketch)
        return fail(TT_ERR_STATE, "tt_set_rounding: the randomized rounding needs a sketch (tt_set_sketch)");
    if (method != TT_ROUND_GRAM && h->shard.on)
        return fail(TT_ERR_STATE, "tt_set_rounding: a spatial shard rounds by Gram-SVD only");
    if (method != TT_ROUND_GRAM && h->graph_on)
        return fail(TT_ERR_STATE, "tt_set_rounding: captured steps use the Gram-SVD rounding (tt_set_graph 0 first)");
    if (method != TT_ROUND_GRAM && (h->taping || h->replay_rec))
        return fail(TT_ERR_STATE, "tt_set_rounding: the adjoint tape records Gram-SVD roundings");
    h->round_method = method;
    return TT_OK;
}

tt_status tt_set_precision(tt_handle h, int precision) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    clear_tape(h);  // a change of state outside a step ends the tape
    if (precision != TT_FP64 && precision != TT_MIXED)
        return fail(TT_ERR_ARG, "tt_set_precision: precision must be TT_FP64 or TT_MIXED");
    h->precision = precision;
    return TT_OK;
}

tt_status tt_set_T(tt_handle h, const double* T_dev) {
    set_error("");
    TT_TRY(check_handle(h, true));
    AllocScope alloc_scope_(h->alloc_ptr());
    clear_tape(h);  // a change of state outside a step ends the tape
    if (!T_dev) return fail(TT_ERR_ARG, "tt_set_T: null input");
    TT_CUDA_TRY(cudaMemcpyAsync(h->f_T.p, T_dev, h->grid.nc * sizeof(double), cudaMemcpyDefault, h->stream));
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return TT_OK;
}

tt_status tt_sync(tt_handle h) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return read_status(h);
}

void tt_destroy(tt_handle h) { delete h; }

tt_status tt_dgemm(int trans_a, int trans_b, int M, int N, int K, double alpha, const double* A,
                   int lda, const double* B, int ldb, double beta, double* C, int ldc,
                   void* stream) {
    set_error("");
    if (M < 0 || N < 0 || K < 0) return fail(TT_ERR_ARG, "tt_dgemm: negative size");
    if ((M && N && K) && (!A || !B || !C)) return fail(TT_ERR_ARG, "tt_dgemm: null pointer");
    return dgemm((cudaStream_t)stream, trans_a != 0, trans_b != 0, M, N, K, alpha, A, lda, B, ldb,
                 beta, C, ldc);
}

tt_status tt_gram(int m, int n, const double* A, int lda, double* G, int ldg, void* stream) {
    set_error("");
    if (m < 0 || n < 0) return fail(TT_ERR_ARG, "tt_gram: negative size");
    if (n == 0) return TT_OK;
    if (!G || (m > 0 && !A)) return fail(TT_ERR_ARG, "tt_gram: null pointer");
    if (lda < n || ldg < n) return fail(TT_ERR_ARG, "tt_gram: leading dimension smaller than n");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf scratch;
    tt_status st = gram(s, m, n, A, lda, G, ldg, scratch);
    if (scratch.p) cudaFreeAsync(scratch.p, s);
    if (st < 0) return st;
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status tt_gram_mixed(int m, int n, const double* A, int lda, double* G, int ldg, void* stream) {
    set_error("");
    if (m < 0 || n < 0) return fail(TT_ERR_ARG, "tt_gram_mixed: negative size");
    if (n == 0) return TT_OK;
    if (!G || (m > 0 && !A)) return fail(TT_ERR_ARG, "tt_gram_mixed: null pointer");
    if (lda < n || ldg < n) return fail(TT_ERR_ARG, "tt_gram_mixed: leading dimension smaller than n");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf scratch;
    tt_status st = slgram(s, m, n, A, lda, G, ldg, scratch);
    if (scratch.p) cudaFreeAsync(scratch.p, s);
    if (st < 0) return st;
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status tt_gemm_nt_mixed(int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                           double* C, int ldc, void* stream) {
    set_error("");
    if (M < 0 || N < 0 || K < 0) return fail(TT_ERR_ARG, "tt_gemm_nt_mixed: negative size");
    if (M == 0 || N == 0) return TT_OK;
    if (!C || (K > 0 && (!A || !B))) return fail(TT_ERR_ARG, "tt_gemm_nt_mixed: null pointer");
    if (lda < K || ldb < K || ldc < N) return fail(TT_ERR_ARG, "tt_gemm_nt_mixed: leading dimension too small");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf scratch;
    tt_status st = slgemm_nt(s, M, N, K, A, lda, B, ldb, C, ldc, scratch);
    if (scratch.p) cudaFreeAsync(scratch.p, s);
    if (st < 0) return st;
    TT_CUDA_TRY(cudaGetLastError());
    return TT_OK;
}

tt_status tt_wait_probe(void* stream) {
    set_error("");
    cudaStream_t s = (cudaStream_t)stream;
    EigWork w;
    int* d_small = nullptr;
    TT_CUDA_TRY(cudaMallocAsync((void**)&d_small, sizeof(int), s));
    TT_CUDA_TRY(cudaMemsetAsync(d_small, 0, sizeof(int), s));
    tt_status st = wait_probe(s, w, d_small);
    int hs = 0;
    cudaMemcpyAsync(&hs, d_small, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_small, s);
    w.release();
    if (st < 0) return st;
    if (e != cudaSuccess) return fail(TT_ERR_CUDA, std::string("tt_wait_probe: ") + cudaGetErrorString(e));
    if (hs & DEV_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_wait_probe: the bounded wait ran out (as designed)");
    return TT_OK;
}

tt_status tt_pchol(int n, const double* G, int ldg, double* W, void* stream, int* rank_host) {
    set_error("");
    if (n < 0) return fail(TT_ERR_ARG, "tt_pchol: negative size");
    if (rank_host) *rank_host = 0;
    if (n == 0) return TT_OK;
    if (!G || !W) return fail(TT_ERR_ARG, "tt_pchol: null pointer");
    if (ldg < n) return fail(TT_ERR_ARG, "tt_pchol: leading dimension smaller than n");
    cudaStream_t s = (cudaStream_t)stream;
    EigWork w;
    DevBuf scratch;  // Wc (n x n) and the double-buffered residual diagonal (2 n)
    int* d_small = nullptr;
    tt_status st = scratch.ensure((size_t)n * n + 2 * (size_t)n, s);
    if (st < 0) return st;
    TT_CUDA_TRY(cudaMallocAsync((void**)&d_small, 2 * sizeof(int), s));
    TT_CUDA_TRY(cudaMemsetAsync(d_small, 0, 2 * sizeof(int), s));
    st = pchol(s, n, G, ldg, W, scratch.p, scratch.p + (size_t)n * n, w, d_small, d_small + 1);
    int hs[2] = {0, 0};
    cudaMemcpyAsync(hs, d_small, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_small, s);
    scratch.release();
    w.release();
    if (st < 0) return st;
    if (e != cudaSuccess) return fail(TT_ERR_CUDA, std::string("tt_pchol: ") + cudaGetErrorString(e));
    if (hs[0] & DEV_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_pchol: grid barrier wait ran out");
    if (hs[1] < 0) return fail(TT_ERR_NONFINITE, "tt_pchol: Inf or NaN on the diagonal of G");
    if (rank_host) *rank_host = hs[1];
    return TT_OK;
}

tt_status tt_syev(int n, const double* G, int ldg, double* lam, double* Vt, int ldv, void* stream,
                  int* sweeps_host) {
    return tt_syev_ex(n, G, ldg, lam, Vt, ldv, JACOBI_MAX_SWEEPS, stream, sweeps_host);
}

static tt_status syev_entry(bool psd, int n, const double* G, int ldg, double* lam, double* Vt, int ldv, int max_sweeps,
                     void* stream, int* sweeps_host);

tt_status tt_syev_ex(int n, const double* G, int ldg, double* lam, double* Vt, int ldv, int max_sweeps,
                     void* stream, int* sweeps_host) {
    return syev_entry(false, n, G, ldg, lam, Vt, ldv, max_sweeps, stream, sweeps_host);
}

tt_status tt_syev_psd(int n, const double* K, int ldk, double* lam, double* Vt, int ldv, int max_sweeps,
                      void* stream, int* sweeps_host) {
    return syev_entry(true, n, K, ldk, lam, Vt, ldv, max_sweeps, stream, sweeps_host);
}

static tt_status syev_entry(bool psd, int n, const double* G, int ldg, double* lam, double* Vt, int ldv, int max_sweeps,
                     void* stream, int* sweeps_host) {
    set_error("");
    if (max_sweeps < 1 || max_sweeps > JACOBI_MAX_SWEEPS)
        return fail(TT_ERR_ARG, "tt_syev_ex: max_sweeps must be in 1 .. " + std::to_string(JACOBI_MAX_SWEEPS));
    if (n < 0) return fail(TT_ERR_ARG, "tt_syev: negative size");
    if (n == 0) return TT_OK;
    if (!G || !lam || !Vt) return fail(TT_ERR_ARG, "tt_syev: null pointer");
    if (ldg < n || ldv < n) return fail(TT_ERR_ARG, "tt_syev: leading dimension smaller than n");
    cudaStream_t s = (cudaStream_t)stream;
    EigWork w;
    int* d_small = nullptr;
    TT_CUDA_TRY(cudaMallocAsync((void**)&d_small, 2 * sizeof(int), s));
    TT_CUDA_TRY(cudaMemsetAsync(d_small, 0, 2 * sizeof(int), s));
    tt_status st = psd ? syev_psd(s, n, G, ldg, lam, Vt, ldv, w, d_small, d_small + 1, max_sweeps)
                       : syev(s, n, G, ldg, lam, Vt, ldv, w, d_small, d_small + 1, max_sweeps);
    int hs[2] = {0, 0};
    cudaMemcpyAsync(hs, d_small, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_small, s);
    w.release();
    if (st < 0) return st;
    if (e != cudaSuccess) return fail(TT_ERR_CUDA, std::string("tt_syev: ") + cudaGetErrorString(e));
    if (sweeps_host) *sweeps_host = hs[1];
    if (hs[0] & DEV_TIMEOUT) return fail(TT_ERR_TIMEOUT, "tt_syev: grid barrier wait ran out");
    if (hs[0] & DEV_NOT_CONVERGED) return fail(TT_ERR_NOT_CONVERGED, "tt_syev: sweep limit reached");
    return TT_OK;
}

tt_status tt_autotune(void* stream, int* table_out) {
    set_error("");
    static_assert(TT_AUTOTUNE_ENTRIES == AT_TILE_BUCKETS * AT_K_BUCKETS, "autotune table size");
    return autotune((cudaStream_t)stream, table_out);
}

tt_status tt_set_autotune_table(const int* table_host, int n) {
    set_error("");
    if (!table_host) return fail(TT_ERR_ARG, "tt_set_autotune_table: null table");
    return autotune_install(table_host, n);
}

tt_status tt_get_autotune_table(int* table_host, int n) {
    set_error("");
    if (!table_host || n < TT_AUTOTUNE_ENTRIES)
        return fail(TT_ERR_ARG, "tt_get_autotune_table: need a table of TT_AUTOTUNE_ENTRIES ints");
    autotune_read(table_host);
    return TT_OK;
}

tt_status tt_set_max_sweeps(tt_handle h, int max_sweeps) {
    set_error("");
    TT_TRY(check_handle(h, false));
    if (max_sweeps < 1 || max_sweeps > JACOBI_MAX_SWEEPS)
        return fail(TT_ERR_ARG, "tt_set_max_sweeps: max_sweeps must be in 1 .. " +
                                    std::to_string(JACOBI_MAX_SWEEPS));
    h->max_sweeps = max_sweeps;
    return TT_OK;
}

tt_status tt_profile(tt_handle h, int enable) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    resolve_profile(h);
    h->prof_on = enable != 0;
    if (enable)
        for (int p = 0; p < TT_NPHASES; ++p) h->ph[p] = tt_ctx::PhaseAcc();
    return TT_OK;
}

tt_status tt_profile_read(tt_handle h, int phase, double* ms, long long* launches,
                          long long* calls, double* flops, double* bytes) {
    set_error("");
    TT_TRY(check_handle(h, false));
    AllocScope alloc_scope_(h->alloc_ptr());
    if (phase < 0 || phase >= TT_NPHASES) return fail(TT_ERR_ARG, "tt_profile_read: bad phase");
    TT_CUDA_TRY(cudaStreamSynchronize(h->stream));
    resolve_profile(h);
    const auto& a = h->ph[phase];
    if (ms) *ms = a.ms;
    if (launches) *launches = a.launches;
    if (calls) *calls = a.calls;
    if (flops) *flops = a.flops;
    if (bytes) *bytes = a.bytes;
    return TT_OK;
}

unsigned long long tt_kernel_launches(void) { return g_launches.load(); }

tt_status tt_bench_fp64_mma(double* tflops_host, void* stream) {
    set_error("");
    if (!tflops_host) return fail(TT_ERR_ARG, "tt_bench_fp64_mma: null output");
    return bench_fp64_mma((cudaStream_t)stream, tflops_host);
}

tt_status tt_bench_bf16_mma(double* tflops_host, void* stream) {
    set_error("");
    if (!tflops_host) return fail(TT_ERR_ARG, "tt_bench_bf16_mma: null output");
    return bench_bf16_mma((cudaStream_t)stream, tflops_host);
}

}  // extern "C"
