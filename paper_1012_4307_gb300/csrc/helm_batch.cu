// Batched solves of many independent problems (energies, right-hand sides, grid sizes).
// Each problem owns a full handle (levels, Krylov workspace) on the batch's shared stream;
// problems are solved largest first so that the tail of the batch is short.
#include <algorithm>
#include <numeric>
#include <vector>

#include "helm_handle.h"

struct helm_batch {
    std::vector<helm_handle *> h;
    cudaStream_t stream = nullptr;
};

extern "C" helm_status helm_create_batch(int nprob, const helm_grid *grids, const double *theta, const double *r0,
                                         const double *const *k2, const helm_mg_params *mg, void *stream,
                                         helm_batch **out) {
    if (!out) return helm_fail(HELM_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (nprob < 1 || !grids || !theta || !r0 || !k2 || !mg) return helm_fail(HELM_ERR_ARG, "bad batch arguments");
    helm_batch *b = new (std::nothrow) helm_batch();
    if (!b) return helm_fail(HELM_ERR_NOMEM, "host allocation failed");
    b->stream = (cudaStream_t)stream;
    for (int i = 0; i < nprob; i++) {
        helm_handle *h = nullptr;
        const int d = grids[i].dim;
        const double *lo = r0 + 6 * (size_t)i, *hi = lo + 3;
        helm_status st = helm_create(&grids[i], theta[i], lo, hi, k2[i], mg, stream, &h);
        (void)d;
        if (st != HELM_OK) {
            helm_destroy_batch(b);
            return st;
        }
        b->h.push_back(h);
    }
    *out = b;
    return HELM_OK;
}

extern "C" helm_status helm_solve_batch(helm_batch *b, const void *const *rhs, void *const *x, double tol, int restart,
                                        int maxit, helm_stats *stats) {
    if (!b || !rhs || !x) return helm_fail(HELM_ERR_ARG, "bad batch arguments");
    const int n = (int)b->h.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->h[a]->np > b->h[c]->np; });
    helm_status worst = HELM_OK;
    for (int i : order) {
        helm_status st = krylov_solve(b->h[i], HELM_FGMRES, rhs[i], x[i], tol, restart, maxit, stats ? &stats[i] : nullptr);
        if (st == HELM_ERR_CUDA || st == HELM_ERR_ARG || st == HELM_ERR_NOMEM) return st;
        if (st != HELM_OK && worst == HELM_OK) worst = st;
    }
    return worst;
}

extern "C" void helm_destroy_batch(helm_batch *b) {
    if (!b) return;
    for (helm_handle *h : b->h) helm_destroy(h);
    delete b;
}
