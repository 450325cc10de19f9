// Handle layout shared by the host drivers (not part of the C-ABI).
#pragma once

#include <vector>

#include "helm_internal.h"

// One multigrid level of the preconditioning operator: coefficients and k^2 in both
// precisions, and the level's work vectors (b: right-hand side / restricted residual,
// u: iterate / coarse error, t: Jacobi ping-pong partner).
struct LevelDev {
    int n[3] = {1, 1, 1};
    size_t np = 0;
    DevOp<double> M64{};
    DevOp<float> M32{};
    double2 *coef64[3] = {nullptr, nullptr, nullptr};
    float2 *coef32[3] = {nullptr, nullptr, nullptr};
    double *k2_64 = nullptr;
    float *k2_32 = nullptr;
    double2 *b64 = nullptr, *u64 = nullptr, *t64 = nullptr;
    float2 *b32 = nullptr, *u32 = nullptr, *t32 = nullptr;
};

// Opt-in launch timing: when on, every kernel launch of the drivers is bracketed by two CUDA
// events on the handle's stream and tagged with its class and algorithmic bytes / flops.
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
    double bytes_pass;  // the same work counted pass by pass (each sweep, residual, transfer)
};
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<ProfRec> recs;
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void reset() { used = 0; recs.clear(); }
    ~Profiler() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

struct helm_handle {
    Profiler prof;
    int dim = 2;
    int n[3] = {1, 1, 1};
    size_t np = 0;
    helm_mg_params mg{};
    cudaStream_t stream = nullptr;
    bool stream_owned_sync = true;
    std::vector<void *> owned;  // every device allocation, freed at destroy

    // A = Z (Helmholtz operator, fine grid) in FP64 and (on demand) FP32
    DevOp<double> A64{};
    DevOp<float> A32{};
    double2 *coefA64[3] = {nullptr, nullptr, nullptr};
    float2 *coefA32[3] = {nullptr, nullptr, nullptr};
    double *k2A = nullptr;
    DevOpDF Adf{};  // A with float-pair coefficients (double-FP32 Arnoldi products)
    double2 *wts[3] = {nullptr, nullptr, nullptr};  // dual-volume weights per axis

    std::vector<LevelDev> lv;
    // first level handled by the fused coarse-tail kernel, per precision (-1: none); chosen so
    // the tail's vectors fit in shared memory
    int tail_top32 = -1, tail_top64 = -1;  // first level of the fused tail (-1: none), as built
    helm_tuning tune{};                      // kernel choices (see helm_set_tuning)
    int ctail_fit[2] = {0, 0};               // most coarsest levels a cluster tail of 8 / 16 blocks holds
    // initial shared-memory images of the cluster tail, keyed by first level * 32 + blocks
    // (device memory, also listed in owned)
    std::vector<std::pair<int, void *>> ctail_img;
    int nu_c = 0;
    double2 *minv64 = nullptr;
    float2 *minv32 = nullptr;

    // Krylov workspace (allocated on first use, grown on demand)
    int m_alloc = 0;
    helm_prec z_prec = HELM_C128;
    double2 *V = nullptr;      // (m+1) basis vectors, FP64
    void *Z = nullptr;         // m preconditioned vectors (c64 or c128)
    double2 *H = nullptr;      // (m+1) x m Hessenberg, column-major
    double2 *g = nullptr, *sn = nullptr, *y = nullptr, *h2 = nullptr;
    double *cs = nullptr;
    double2 *partials = nullptr;
    double2 *scal = nullptr;   // scalar scratch (norms, Bi-CGSTAB scalars)
    double *est_dev = nullptr;
    int *gs_flag = nullptr;   // DGKS decision of the current Arnoldi step (device); [2]: the cycle's stop flag
    double *tol_dev = nullptr;  // the solve's tolerance (device), for the stop flag
    int *gs_count = nullptr;  // re-orthogonalisations in the current solve (device)
    double *est_host = nullptr;  // pinned: residual estimate of every FGMRES step (stored by the rotation kernel)
    int est_host_len = 0;
    double2 *fnorm_dev = nullptr;  // ||f|| of the current solve (device scalar)
    // FGMRES steps: one event per step j, and a CUDA graph of step j captured on cap_stream
    std::vector<cudaEvent_t> step_ev;
    // delayed CGS2: inner products of a step (2 (m + 1)), normalisation norms alpha_j (m + 2),
    // update coefficients (2 m + 4); closing step of a cycle with jc columns: event and graph jc
    double2 *hv = nullptr, *alpha2 = nullptr, *dcoef = nullptr;
    unsigned *tickets = nullptr;  // last-block counters of the fused passes (0 between launches)
    // side stream of a step (the Givens rotation runs beside the update pass): fork and join
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<cudaEvent_t> close_ev;
    std::vector<cudaGraphExec_t> close_graph;
    std::vector<cudaGraphExec_t> step_graph;
    cudaStream_t cap_stream = nullptr;
    bool graphs_ok = true;
    bool capturing = false;
    cudaEvent_t ev_fn = nullptr, ev_beta = nullptr;  // ||f|| and ||r0|| read-backs
    // Bi-CGSTAB workspace
    bool bicg_alloc = false;
    double2 *br = nullptr, *brh = nullptr, *bp = nullptr, *bv = nullptr, *bs = nullptr, *bt = nullptr;
    void *by = nullptr, *bz = nullptr;
    // adjoint temporaries
    double2 *adj_rhs = nullptr, *adj_y = nullptr;
    std::vector<void *> krylov_owned;
};

// Launch-timing scope: records a start event now and, at destruction, a stop event plus the
// launch's class and algorithmic cost.  A no-op unless the handle's profiler is on.
// bytes: algorithmic DRAM bytes of the launch (each operand touched once); bytes_pass (< 0:
// equal to bytes): the bytes of the same work counted pass by pass, as separate sweep, residual
// and transfer launches would move them (differs for the temporally blocked kernels).
struct ProfScope {
    helm_handle *h;
    int cls;
    double bytes, flops, bytes_pass;
    cudaEvent_t a = nullptr;
    ProfScope(helm_handle *h_, int cls_, double bytes_, double flops_, double bytes_pass_ = -1.0)
        : h(h_), cls(cls_), bytes(bytes_), flops(flops_), bytes_pass(bytes_pass_ < 0 ? bytes_ : bytes_pass_) {
        if (h->prof.on) {
            a = h->prof.next();
            if (a) cudaEventRecord(a, h->stream);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = h->prof.next();
        if (!b) return;
        cudaEventRecord(b, h->stream);
        h->prof.recs.push_back(ProfRec{cls, a, b, bytes, flops, bytes_pass});
    }
};

helm_status helm_fail(helm_status st, const char *fmt, ...);
void helm_free_krylov(helm_handle *h);
// Allocates (or keeps) the handle's FGMRES workspace for restart length m.
helm_status helm_ensure_krylov(helm_handle *h, int m);
// Destroys the captured FGMRES step graphs (they are captured again on next use).
void helm_drop_graphs(helm_handle *h);

// Resumable flexible-GMRES solve (krylov.cu): fgmres_begin queues the first work, each
// fgmres_advance performs the phases whose event has fired (or waits, if block) until the
// solve is DONE; the outcome is in status.
struct FgmresRun {
    enum Phase { WAIT_FN, START, WAIT_BETA, IN_CYCLE, DONE };
    helm_handle *h = nullptr;
    const double2 *f = nullptr;
    double2 *x = nullptr;
    double tol = 0, fn = 0, est = 1, rel = 1;
    int m = 0, maxit = 0, it = 0, restarts = 0, jmax = 0, next = 0;
    helm_stats *st = nullptr;
    helm_status status = HELM_ERR_NOCONV;
    Phase phase = DONE;
};
helm_status fgmres_begin(helm_handle *h, FgmresRun &r, const double2 *f, double2 *x, double tol, int m, int maxit,
                         helm_stats *st);
helm_status fgmres_advance(FgmresRun &r, bool block);
template <typename R> cudaError_t precondition(helm_handle *h, const double2 *v, typename CT<R>::T *z);
// v a float-pair vector (float4 (re.hi, re.lo, im.hi, im.lo) per node)
template <typename R>
cudaError_t precondition_pair(helm_handle *h, const float4 *v, const double2 *alpha, typename CT<R>::T *z);
// The complex64 cycle applied to what level 0's right-hand-side buffer already holds (written
// there by the delayed-CGS2 update pass), and that buffer.
cudaError_t precondition_level0_c64(helm_handle *h, float2 *z);
float2 *level0_rhs_c64(helm_handle *h);
// First level of the fused coarse tail of a precision-R cycle under the handle's tuning (-1: none).
template <typename R> int tail_top(const helm_handle *h);
// First level of the cluster tail (2D complex64 cycles) under the handle's tuning (-1: none).
int ctail_top(const helm_handle *h);
// Whether the cluster tail of a cycle from zero runs as the deep-halo kernel under the handle's
// tuning (cluster_halo 3, a V-cycle of omega-Jacobi with at most two sweeps each way, levels that
// fit).
bool ctail_deep(const helm_handle *h);
// The initial shared-memory image of the cluster tail (deep: of the deep-halo kernel) for the
// current tuning (null: no tail, or not built and build false); built on the handle's stream,
// outside graph capture.
const void *ctail_image(helm_handle *h, bool build, bool deep);

// Lockstep engine of helm_solve_batch (batch_lockstep.cu): every phase of an FGMRES step is one
// launch over all problems.  lockstep_eligible tells whether the batch's configuration is one it
// runs (lockstep_why says why not).
struct BatchLockstep;
BatchLockstep *lockstep_create(const std::vector<helm_handle *> &handles);
void lockstep_destroy(BatchLockstep *L);
bool lockstep_eligible(BatchLockstep *L);
const char *lockstep_why(const BatchLockstep *L);
helm_status lockstep_solve(BatchLockstep *L, cudaStream_t user, const void *const *rhs, void *const *x, double tol,
                           int m, int maxit, helm_stats *stats);
