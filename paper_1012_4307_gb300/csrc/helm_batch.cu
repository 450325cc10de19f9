// Batched solves of many independent problems (energies, right-hand sides, grid sizes).
//
// Each problem owns a full handle (levels, Krylov workspace) on its own non-blocking stream.
// Two engines:
//   lockstep (batch_lockstep.cu): the problems advance their FGMRES steps together and every
//     phase of a step is one launch over all of them (complex64 V(2,2) Jacobi cycles with the
//     delayed-CGS2 Arnoldi on 2D grids with a common coarse tail);
//   streams: one host thread drives every problem's flexible-GMRES state machine round-robin:
//     it only ever polls events, so while one problem waits for its residual estimate the
//     others keep enqueueing, and kernels of different problems run concurrently on the GPU.
//     Every FGMRES step of every problem is replayed from a CUDA graph captured on first use,
//     so a step costs one graph launch on the host.  Problems are visited largest first.
// The default picks lockstep whenever the configuration allows it.
#include <algorithm>
#include <numeric>
#include <thread>
#include <vector>

#include "helm_handle.h"

struct helm_batch {
    std::vector<helm_handle *> h;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    cudaStream_t user = nullptr;
    int engine = HELM_BATCH_AUTO;     // requested engine
    int last = HELM_BATCH_AUTO;       // engine of the last solve
    BatchLockstep *ls = nullptr;
};

extern "C" void helm_destroy_batch(helm_batch *b) {
    if (!b) return;
    if (b->ls) {
        cudaDeviceSynchronize();
        lockstep_destroy(b->ls);
    }
    for (helm_handle *h : b->h) helm_destroy(h);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->start) cudaEventDestroy(b->start);
    delete b;
}

extern "C" helm_status helm_batch_handle(helm_batch *b, int i, helm_handle **out) {
    if (!b || !out) return helm_fail(HELM_ERR_ARG, "null argument");
    if (i < 0 || i >= (int)b->h.size()) return helm_fail(HELM_ERR_ARG, "problem index %d out of range", i);
    *out = b->h[i];
    return HELM_OK;
}

extern "C" helm_status helm_create_batch(int nprob, const helm_grid *grids, const double *theta, const double *r0,
                                         const double *const *k2, const helm_mg_params *mg, void *stream,
                                         helm_batch **out) {
    if (!out) return helm_fail(HELM_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (nprob < 1 || !grids || !theta || !r0 || !k2 || !mg) return helm_fail(HELM_ERR_ARG, "bad batch arguments");
    helm_batch *b = new (std::nothrow) helm_batch();
    if (!b) return helm_fail(HELM_ERR_NOMEM, "host allocation failed");
    b->user = (cudaStream_t)stream;
    if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
        helm_destroy_batch(b);
        return helm_fail(HELM_ERR_CUDA, "cudaEventCreate failed");
    }
    for (int i = 0; i < nprob; i++) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            if (s) cudaStreamDestroy(s);
            helm_destroy_batch(b);
            return helm_fail(HELM_ERR_CUDA, "stream/event creation failed for problem %d", i);
        }
        b->streams.push_back(s);
        b->done.push_back(e);
        helm_handle *h = nullptr;
        const double *lo = r0 + 6 * (size_t)i, *hi = lo + 3;
        helm_status st = helm_create(&grids[i], theta[i], lo, hi, k2[i], mg, s, &h);
        if (st != HELM_OK) {
            helm_destroy_batch(b);
            return st;
        }
        b->h.push_back(h);
    }
    *out = b;
    return HELM_OK;
}

extern "C" helm_status helm_batch_set_engine(helm_batch *b, int engine) {
    if (!b) return helm_fail(HELM_ERR_ARG, "null batch");
    if (engine != HELM_BATCH_AUTO && engine != HELM_BATCH_LOCKSTEP && engine != HELM_BATCH_STREAMS)
        return helm_fail(HELM_ERR_ARG, "unknown batch engine %d", engine);
    b->engine = engine;
    return HELM_OK;
}

extern "C" helm_status helm_batch_get_engine(const helm_batch *b, int *last) {
    if (!b || !last) return helm_fail(HELM_ERR_ARG, "null argument");
    *last = b->last;
    return HELM_OK;
}

extern "C" helm_status helm_solve_batch(helm_batch *b, const void *const *rhs, void *const *x, double tol, int restart,
                                        int maxit, helm_stats *stats) {
    if (!b || !rhs || !x) return helm_fail(HELM_ERR_ARG, "bad batch arguments");
    if (!(tol > 0.0) || maxit < 1 || restart < 1 || restart > 64) return helm_fail(HELM_ERR_ARG, "bad tol/restart/maxit");
    const int n = (int)b->h.size();
    for (int i = 0; i < n; i++)
        if (!rhs[i] || !x[i] || rhs[i] == x[i] || ((uintptr_t)rhs[i] | (uintptr_t)x[i]) % 16)
            return helm_fail(HELM_ERR_ARG, "rhs/x of problem %d invalid (null, overlapping or misaligned)", i);
    if (b->engine != HELM_BATCH_STREAMS) {
        if (!b->ls && !(b->ls = lockstep_create(b->h))) return helm_fail(HELM_ERR_NOMEM, "host allocation failed");
        if (lockstep_eligible(b->ls) && restart <= 63) {
            // the problems' own streams may still hold work (setup, tuning images)
            for (cudaStream_t s : b->streams)
                if (cudaStreamSynchronize(s) != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "cudaStreamSynchronize failed");
            b->last = HELM_BATCH_LOCKSTEP;
            std::vector<helm_stats> local(n);
            helm_stats *sp = stats ? stats : local.data();
            if (stats)
                for (int i = 0; i < n; i++)
                    if (!stats[i].history) stats[i].history_len = 0;
            return lockstep_solve(b->ls, b->user, rhs, x, tol, restart, maxit, sp);
        }
        if (b->engine == HELM_BATCH_LOCKSTEP)
            return helm_fail(HELM_ERR_ARG, "batch not eligible for the lockstep engine: %s%s", lockstep_why(b->ls),
                             restart > 63 ? " (restart above 63)" : "");
    }
    b->last = HELM_BATCH_STREAMS;
    // the problems' streams start after everything already queued on the caller's stream
    if (cudaEventRecord(b->start, b->user) != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "cudaEventRecord failed");
    for (cudaStream_t s : b->streams)
        if (cudaStreamWaitEvent(s, b->start, 0) != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "cudaStreamWaitEvent failed");
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->h[a]->np > b->h[c]->np; });
    std::vector<FgmresRun> runs(n);
    std::vector<helm_stats> local(n);
    for (int i : order) {
        helm_stats *st = stats ? &stats[i] : &local[i];
        if (stats && !stats[i].history) stats[i].history_len = 0;
        helm_status s0 = fgmres_begin(b->h[i], runs[i], (const double2 *)rhs[i], (double2 *)x[i], tol, restart, maxit, st);
        if (s0 != HELM_OK) return s0;
    }
    int active = n;
    while (active > 0) {
        int progressed = 0;
        active = 0;
        for (int i : order) {
            FgmresRun &r = runs[i];
            if (r.phase == FgmresRun::DONE) continue;
            const int it0 = r.it;
            const FgmresRun::Phase p0 = r.phase;
            const helm_status s0 = fgmres_advance(r, false);
            if (s0 != HELM_OK) return s0;
            if (r.it != it0 || r.phase != p0) progressed++;
            if (r.phase != FgmresRun::DONE) active++;
        }
        if (active > 0 && progressed == 0) std::this_thread::yield();
    }
    helm_status worst = HELM_OK;
    for (int i = 0; i < n; i++) {
        const helm_stats &st = stats ? stats[i] : local[i];
        if (stats) stats[i].status = runs[i].status;
        if (runs[i].status != HELM_OK && worst == HELM_OK) worst = runs[i].status;
        (void)st;
        // the caller's stream continues after every problem's last work
        if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->user, b->done[i], 0) != cudaSuccess)
            return helm_fail(HELM_ERR_CUDA, "joining problem %d to the caller's stream failed", i);
    }
    if (worst != HELM_OK) return helm_fail(worst, "%s in at least one batch problem", worst == HELM_ERR_NOCONV ? "no convergence" : "failure");
    return HELM_OK;
}
