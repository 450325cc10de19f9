// Cycle tuning: which kernels carry out Algorithm 1 on each level (temporally blocked tiles or
// separate sweep / residual / transfer launches, and how many coarse levels go into the fused
// single-block tail or the thread-block-cluster tail), and an autotuner that times the choices
// on the device.  The arithmetic
// of the cycle does not depend on the choice (up to FP32 rounding order).
#include <algorithm>
#include <vector>

#include "helm_internal.h"
#include "helm_handle.h"

#define CKR(...)                                                                                               \
    do {                                                                                                       \
        cudaError_t e_ = (__VA_ARGS__);                                                                        \
        if (e_ != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)

namespace {

// v[q] = a fixed pseudo-random complex value in [-1/2, 1/2)^2 (integer hash of q).
__global__ void k_fill_probe(size_t n, double2 *v) {
    pdl_enter();
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        unsigned long long x = (unsigned long long)q * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        x ^= x >> 31;
        x *= 0xBF58476D1CE4E5B9ull;
        x ^= x >> 29;
        const double a = (double)(x >> 40) * (1.0 / 16777216.0) - 0.5;
        const double b = (double)((x >> 16) & 0xFFFFFFull) * (1.0 / 16777216.0) - 0.5;
        v[q] = make_double2(a, b);
    }
}

bool tuning_valid(const helm_tuning &t) {
    if (t.tail_levels < -1 || t.tail_levels == 1) return false;
    if (t.cluster_levels < 0 || t.cluster_levels == 1) return false;
    if (t.cluster_ctas != 8 && t.cluster_ctas != 16) return false;
    if (t.cluster_halo != 1 && t.cluster_halo != 3) return false;
    for (int l = 0; l < HELM_MAX_LEVELS; l++)
        if (t.level_tile[l] < HELM_TILE_NONE || t.level_tile[l] >= HELM_TILE_COUNT) return false;
    return true;
}

}  // namespace

extern "C" helm_status helm_set_tuning(helm_handle *h, const helm_tuning *t) {
    if (!h || !t) return helm_fail(HELM_ERR_ARG, "null argument");
    if (!tuning_valid(*t))
        return helm_fail(HELM_ERR_ARG, "invalid tuning (tail or cluster levels, cluster blocks or halo, or a tile)");
    h->tune = *t;
    helm_drop_graphs(h);
    ctail_image(h, true, ctail_deep(h));
    return HELM_OK;
}

extern "C" helm_status helm_get_tuning(const helm_handle *h, helm_tuning *t) {
    if (!h || !t) return helm_fail(HELM_ERR_ARG, "null argument");
    *t = h->tune;
    return HELM_OK;
}

extern "C" helm_status helm_autotune(helm_handle *h, helm_prec prec, int reps, helm_tuning *best, double *best_ms) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    if (h->mg.kind == HELM_PC_NONE) return helm_fail(HELM_ERR_ARG, "handle has no preconditioner hierarchy");
    if (prec != HELM_C64 && prec != HELM_C128) return helm_fail(HELM_ERR_ARG, "bad precision");
    if (reps < 1) return helm_fail(HELM_ERR_ARG, "reps must be >= 1");
    const size_t np = h->np;
    const bool c64 = prec == HELM_C64;
    double2 *v = nullptr;
    void *z = nullptr;
    if (cudaMalloc((void **)&v, np * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&z, np * (c64 ? sizeof(float2) : sizeof(double2))) != cudaSuccess) {
        cudaFree(v);
        cudaGetLastError();
        return helm_fail(HELM_ERR_NOMEM, "autotune vectors");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    helm_status st = HELM_OK;
    const helm_tuning keep = h->tune;
    const bool prof = h->prof.on;
    h->prof.on = false;
    auto fail = [&](cudaError_t e, const char *what) {
        st = helm_fail(HELM_ERR_CUDA, "autotune %s: %s", what, cudaGetErrorString(e));
        return -1.0;
    };
    // milliseconds per preconditioner application under tuning t: reps applications captured in
    // a CUDA graph (the form in which the FGMRES steps run them), replayed, best of three
    // timings; a candidate whose capture fails (soft: a cluster shape the device cannot run) is
    // skipped
    auto time_it = [&](const helm_tuning &t, bool soft = false) -> double {
        h->tune = t;
        ctail_image(h, true, ctail_deep(h));
        cudaStream_t keep_s = h->stream;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        h->stream = h->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            pdl_capture_scope no_pdl;
            h->capturing = true;
            for (int r = 0; r < reps && e == cudaSuccess; r++)
                e = c64 ? precondition<float>(h, v, (float2 *)z) : precondition<double>(h, v, (double2 *)z);
            h->capturing = false;
            const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
            if (e == cudaSuccess) e = e2;
        }
        h->stream = keep_s;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            if (ge) cudaGraphExecDestroy(ge);
            if (soft) {
                cudaGetLastError();
                return -2.0;
            }
            return fail(e, "capture");
        }
        double bestt = 1e300;
        for (int w = 0; w < 2 && e == cudaSuccess; w++) e = cudaGraphLaunch(ge, h->stream);
        for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
            float ms = 0.f;
            if ((e = cudaEventRecord(e0, h->stream)) != cudaSuccess || (e = cudaGraphLaunch(ge, h->stream)) != cudaSuccess ||
                (e = cudaEventRecord(e1, h->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                break;
            bestt = std::min(bestt, (double)ms / reps);
        }
        cudaGraphExecDestroy(ge);
        if (e != cudaSuccess) return fail(e, "replay");
        return bestt;
    };
    helm_tuning cur = keep;
    double cur_ms = 0.0;
    const int last = (int)h->lv.size() - 1;
    const int built = c64 ? h->tail_top32 : h->tail_top64;
    const int max_tail = built < 0 ? 0 : last - built + 1;
    const bool blockable = c64 && h->dim == 2 && h->mg.smoother == HELM_SMOOTH_JACOBI && h->mg.nu1 == 2 &&
                           h->mg.nu2 == 2;
    // tail depth: none, or 2 .. max_tail coarsest levels
    auto tune_tail = [&]() {
        for (int tl = 0; tl <= max_tail && st == HELM_OK; tl++) {
            if (tl == 1 || tl == cur.tail_levels) continue;
            helm_tuning t = cur;
            t.tail_levels = tl;
            const double ms = time_it(t);
            if (ms >= 0 && ms < cur_ms) { cur = t; cur_ms = ms; }
        }
    };
    // cluster tail (2D complex64): off, or 2 .. the levels that fit, on 8 or 16 blocks, with one
    // or (where it applies) three halo rows
    auto tune_cluster = [&]() {
        if (!(c64 && h->dim == 2)) return;
        const helm_mg_params &m = h->mg;
        const bool vj2 = m.smoother == HELM_SMOOTH_JACOBI && m.gamma_f == 1 && m.gamma_c == 1 && m.nu1 <= 2 && m.nu2 <= 2;
        for (int k = 0; k < 2 && st == HELM_OK; k++) {
            const int nc = k ? 16 : 8;
            for (int cl = 2; cl <= h->ctail_fit[k] && st == HELM_OK; cl++) {
                int n[MAX_CT_LEVELS][3];
                DevOp<float> ops[MAX_CT_LEVELS];
                for (int q = 0; q < cl; q++) {
                    ops[q] = h->lv[last - cl + 1 + q].M32;
                    for (int a = 0; a < 3; a++) n[q][a] = ops[q].n[a];
                }
                unsigned off[MAX_CT_LEVELS][7], obc, oz;
                if (mg_ctail_max_clusters(nc, mg_ctail_layout(cl, n, nc, h->nu_c, off, &obc, &oz)) < 1) continue;
                const size_t deep_bytes = vj2 ? mg_chalo_bytes(cl, ops, h->nu_c, nc) : 0;
                for (int halo : {1, 3}) {
                    if (cl == cur.cluster_levels && nc == cur.cluster_ctas && halo == cur.cluster_halo) continue;
                    if (halo == 3 && (!deep_bytes || mg_chalo_max_clusters(nc, deep_bytes) < 1)) continue;
                    helm_tuning t = cur;
                    t.cluster_levels = cl;
                    t.cluster_ctas = nc;
                    t.cluster_halo = halo;
                    const double ms = time_it(t, true);
                    if (ms >= 0 && ms < cur_ms) { cur = t; cur_ms = ms; }
                }
            }
        }
        if (cur.cluster_levels > 0 && st == HELM_OK) {  // and without it
            helm_tuning t = cur;
            t.cluster_levels = 0;
            const double ms = time_it(t);
            if (ms >= 0 && ms < cur_ms) { cur = t; cur_ms = ms; }
        }
    };
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        st = helm_fail(HELM_ERR_CUDA, "autotune capture stream");
    } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = helm_fail(HELM_ERR_CUDA, "autotune events");
    } else {
        launch_pdl(k_fill_probe, (unsigned)std::min<size_t>(cdiv(np, 256), 152 * 8), 256, 0, h->stream, np, v);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) fail(e, "fill");
        if (st == HELM_OK) {
            if (cur.tail_levels < 0) cur.tail_levels = max_tail;
            cur_ms = time_it(cur);
        }
        if (st == HELM_OK) tune_tail();
        if (st == HELM_OK) tune_cluster();
        // per level above the tails, greedily from the finest: separate launches or a tile shape
        if (blockable) {
            h->tune = cur;
            const int top = tail_top<float>(h), ctop = ctail_top(h);
            int stop = last;
            if (top >= 0) stop = std::min(stop, top);
            if (ctop >= 0) stop = std::min(stop, ctop);
            stop = std::min(stop, HELM_MAX_LEVELS);
            for (int l = 0; l < stop && st == HELM_OK; l++) {
                for (int tile = HELM_TILE_NONE; tile < HELM_TILE_COUNT && st == HELM_OK; tile++) {
                    if (tile == cur.level_tile[l]) continue;
                    if (tile != HELM_TILE_NONE && !fused_jacobi2_ok(h->lv[l].n, h->dim, tile)) continue;
                    helm_tuning t = cur;
                    t.level_tile[l] = tile;
                    const double ms = time_it(t);
                    if (ms >= 0 && ms < cur_ms) { cur = t; cur_ms = ms; }
                }
            }
            if (st == HELM_OK) tune_tail();  // the levels' choices may move the best depths
            if (st == HELM_OK) tune_cluster();
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(v);
    cudaFree(z);
    h->prof.on = prof;
    h->tune = st == HELM_OK ? cur : keep;
    helm_drop_graphs(h);
    ctail_image(h, true, ctail_deep(h));
    if (st != HELM_OK) return st;
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return HELM_OK;
}
