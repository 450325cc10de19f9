// Lockstep engine of helm_solve_batch: many independent problems advance their flexible-GMRES
// steps together, and every phase of a step is ONE launch over all problems.
//
// A step j of the delayed-CGS2 FGMRES (the algorithm of fgmres_step_dcgs2 in krylov.cu, with a
// complex64 V(2,2) omega-Jacobi cycle of Algorithm 1 as the preconditioner) is, for all problems:
//   cycle: one temporally blocked pre-smoothing launch per level shape above the coarse tail,
//          largest first (each covers every problem that has a level of that shape); one
//          thread-block-cluster launch of the coarse tail (one cluster per problem); one
//          post-smoothing launch per shape, smallest first;
//   A z_j, the two-vector inner-product pass, its reduction + coefficient step, the Givens
//   rotation of column j - 1 (which also gathers every problem's residual estimate for one copy
//   to the host), and the update pass.
// That is 2 (shapes) + 6 launches per step whatever the number of problems, each with a table of
// per-problem pointers in device memory; the step is captured once as a CUDA graph and replayed.
// A problem leaves the lockstep when its estimate reaches the tolerance (its solution update and
// true-residual check run on its own), by clearing its flag in device memory: the batched kernels
// skip it from then on.  Every problem restarts at the same step count m, so a problem whose true
// residual is not yet small enough waits for the next common restart; its arithmetic is the same
// as that of its single solve with the tuning the engine installs (the cycle's kernels do not
// depend on the launch grouping), so results and iteration counts match krylov_solve bit for bit.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "helm_handle.h"

#define CKR(...)                                                                                               \
    do {                                                                                                       \
        cudaError_t e_ = (__VA_ARGS__);                                                                        \
        if (e_ != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)
#define CKE(...)                          \
    do {                                  \
        cudaError_t e_ = (__VA_ARGS__);   \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

namespace {

// The levels of one shape above the tail: one pre and one post launch per step.
struct Phase {
    int n[3] = {1, 1, 1};
    int tile = HELM_TILE_32x8;
    std::vector<std::pair<int, int>> members;  // (problem, level index)
    BLevel *pre = nullptr, *post = nullptr;
};

}  // namespace

struct BatchLockstep {
    int P = 0, m = 0, T = 0, nc = 16, nu_c = 0;
    int halo = 3;        // cluster tail: halo rows the problems' tunings ask for
    bool deep = false;   // ... and whether the deep-halo kernel runs
    std::vector<helm_handle *> h;
    std::vector<Phase> phases;                  // largest shape first
    DevOp<float> tail_ops[MAX_CT_LEVELS] = {};  // shapes of the tail levels
    BTail *tail = nullptr;
    BVec *vec = nullptr;
    unsigned *apply_first = nullptr, *upd_first = nullptr, *dot_first = nullptr;
    unsigned apply_blocks = 0, upd_blocks = 0;
    std::vector<unsigned> dot_blocks;  // per row j = 0 .. m (nv = j + 1)
    int *active = nullptr;             // device flags, one per problem
    double *tol_dev = nullptr;         // the solve's tolerance (device), for the batched rotation
    int *active_h = nullptr;           // pinned staging of the flags
    // (m + 1) x P gathered estimates, pinned host memory that the batched rotation kernel writes
    // directly (no copy node in the step graphs)
    double *est_h = nullptr;
    double2 *norm_h = nullptr;         // pinned: per problem ||f|| or ||r0||
    cudaStream_t s = nullptr, cap = nullptr;
    std::vector<cudaGraphExec_t> step_graph, close_graph;
    std::vector<cudaEvent_t> step_ev, close_ev;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    std::vector<cudaEvent_t> pev;   // per problem: end of its fanned-out restart work
    std::vector<void *> owned;
    std::vector<const void *> key;  // workspace pointers the tables were built for
    bool graphs_ok = true;
    bool capturing = false;
    std::string why;                // why the batch is not eligible ("" if it is)

    void drop_graphs() {
        for (auto *v : {&step_graph, &close_graph})
            for (cudaGraphExec_t &g : *v)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
    }
    void free_tables() {
        drop_graphs();
        for (void *p : owned) cudaFree(p);
        owned.clear();
        for (Phase &ph : phases) ph.pre = ph.post = nullptr;
        tail = nullptr;
        vec = nullptr;
        apply_first = upd_first = dot_first = nullptr;
        active = nullptr;
        tol_dev = nullptr;
        key.clear();
    }
    ~BatchLockstep() {
        free_tables();
        for (cudaEvent_t e : step_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : close_ev)
            if (e) cudaEventDestroy(e);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (ev_fork) cudaEventDestroy(ev_fork);
        for (cudaEvent_t e : pev)
            if (e) cudaEventDestroy(e);
        if (active_h) cudaFreeHost(active_h);
        if (est_h) cudaFreeHost(est_h);
        if (norm_h) cudaFreeHost(norm_h);
        if (s) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
    }
};

void lockstep_destroy(BatchLockstep *L) { delete L; }

namespace {

template <typename T> cudaError_t upload(BatchLockstep *L, T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    CKE(cudaMalloc((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T)));
    L->owned.push_back(*dst);
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool same_shape(const int a[3], const int b[3]) { return a[0] == b[0] && a[1] == b[1] && a[2] == b[2]; }

// Whether the lockstep engine can run the batch (sets L->why otherwise), and with commit its
// schedule: the tail depth T, the cluster size, and a tile per level shape above the tail.
bool plan(BatchLockstep *L, bool commit) {
    const int P = (int)L->h.size();
    L->why.clear();
    for (int p = 0; p < P; p++) {
        const helm_handle *h = L->h[p];
        const helm_mg_params &g = h->mg;
        if (h->dim != 2) { L->why = "a problem is not 2D"; return false; }
        if (g.kind == HELM_PC_NONE || g.prec != HELM_C64 || g.gs_arith != HELM_GS_DCGS2 ||
            g.smoother != HELM_SMOOTH_JACOBI || g.nu1 != 2 || g.nu2 != 2 || g.gamma_f != 1 || g.gamma_c != 1) {
            L->why = "the lockstep engine runs complex64 V(2,2) omega-Jacobi cycles with the delayed-CGS2 Arnoldi";
            return false;
        }
    }
    // reference: the problem with the most levels; its tuning proposes the tail and the tiles
    int ref = 0;
    for (int p = 1; p < P; p++)
        if (L->h[p]->lv.size() > L->h[ref]->lv.size()) ref = p;
    const helm_handle *R = L->h[ref];
    int T = R->tune.cluster_levels >= 2 ? R->tune.cluster_levels : 4;
    const int nc = R->tune.cluster_levels >= 2 ? R->tune.cluster_ctas : 16;
    for (int p = 0; p < P; p++) {
        const helm_handle *h = L->h[p];
        T = std::min(T, (int)h->lv.size());
        T = std::min(T, h->ctail_fit[nc == 16 ? 1 : 0]);
    }
    if (T < 2) { L->why = "no common coarse tail fits a thread-block cluster"; return false; }
    // every problem's last T levels have the reference's shapes and the same coarsest solve
    const int nr = (int)R->lv.size();
    for (int p = 0; p < P; p++) {
        const helm_handle *h = L->h[p];
        const int nl = (int)h->lv.size();
        if (h->nu_c != R->nu_c) { L->why = "coarsest grids differ"; return false; }
        for (int k = 0; k < T; k++)
            if (!same_shape(h->lv[nl - T + k].n, R->lv[nr - T + k].n)) {
                L->why = "the problems' coarse levels differ in shape";
                return false;
            }
    }
    // shapes above the tail, each with one tile valid for it
    std::map<std::pair<int, int>, int> tile_of;
    for (int l = 0; l < nr - T; l++) {
        int t = l < HELM_MAX_LEVELS ? R->tune.level_tile[l] : HELM_TILE_32x8;
        // the small tile pays off when a lone small level leaves most SMs idle; a launch over many
        // problems fills the GPU, where its larger halo share costs time
        if (t == HELM_TILE_8x8) t = HELM_TILE_16x8;
        if (t == HELM_TILE_NONE || t == HELM_TILE_WAVE || !fused_jacobi2_ok(R->lv[l].n, 2, t)) t = HELM_TILE_32x8;
        tile_of[{R->lv[l].n[0], R->lv[l].n[1]}] = t;
    }
    std::vector<Phase> phases;
    std::map<std::pair<int, int>, int> idx;
    for (int p = 0; p < P; p++) {
        const helm_handle *h = L->h[p];
        for (int l = 0; l < (int)h->lv.size() - T; l++) {
            const std::pair<int, int> key{h->lv[l].n[0], h->lv[l].n[1]};
            int t = tile_of.count(key) ? tile_of[key] : HELM_TILE_32x8;
            if (!fused_jacobi2_ok(h->lv[l].n, 2, t)) {
                t = HELM_TILE_32x8;
                if (!fused_jacobi2_ok(h->lv[l].n, 2, t)) { L->why = "a level does not fit the blocked smoother tiles"; return false; }
            }
            tile_of[key] = t;
            if (!idx.count(key)) {
                idx[key] = (int)phases.size();
                Phase ph;
                for (int a = 0; a < 3; a++) ph.n[a] = h->lv[l].n[a];
                phases.push_back(ph);
            }
            phases[idx[key]].members.push_back({p, l});
        }
    }
    if (!commit) return true;
    for (Phase &ph : phases) ph.tile = tile_of[{ph.n[0], ph.n[1]}];
    // largest shape first: every problem coarsens through its levels in that order
    std::stable_sort(phases.begin(), phases.end(),
                     [](const Phase &a, const Phase &b) { return (long)a.n[0] * a.n[1] > (long)b.n[0] * b.n[1]; });
    L->phases.swap(phases);
    L->T = T;
    L->nc = nc;
    L->halo = R->tune.cluster_halo;
    L->nu_c = R->nu_c;
    for (int k = 0; k < T; k++) L->tail_ops[k] = R->lv[nr - T + k].M32;
    return true;
}

// Installs the schedule as every handle's tuning (so that a single solve on a handle runs the
// same kernels) and builds the device tables for restart length m.
helm_status build(BatchLockstep *L, int m) {
    const int P = (int)L->h.size();
    for (int p = 0; p < P; p++) {
        helm_status st = helm_ensure_krylov(L->h[p], m);
        if (st != HELM_OK) return st;
    }
    std::vector<const void *> key;
    for (helm_handle *h : L->h) {
        key.push_back(h->V);
        key.push_back(h->Z);
    }
    key.push_back((const void *)(size_t)m);
    if (key == L->key && L->vec) return HELM_OK;
    L->free_tables();
    if (!plan(L, true)) return helm_fail(HELM_ERR_ARG, "batch not eligible for the lockstep engine: %s", L->why.c_str());
    // tunings (each builds the problem's cluster-tail image on its own stream)
    for (int p = 0; p < P; p++) {
        helm_handle *h = L->h[p];
        helm_tuning t = h->tune;
        t.cluster_levels = L->T;
        t.cluster_ctas = L->nc;
        t.cluster_halo = L->halo;
        t.tail_levels = 0;
        for (int l = 0; l < HELM_MAX_LEVELS; l++) t.level_tile[l] = HELM_TILE_32x8;
        for (const Phase &ph : L->phases)
            for (const auto &mb : ph.members)
                if (mb.first == p && mb.second < HELM_MAX_LEVELS) t.level_tile[mb.second] = ph.tile;
        helm_status st = helm_set_tuning(h, &t);
        if (st != HELM_OK) return st;
        if (p == 0) L->deep = ctail_deep(h);
        if (ctail_deep(h) != L->deep) return helm_fail(HELM_ERR_ARG, "the problems' cluster tails differ");
        if (!ctail_image(h, false, L->deep)) return helm_fail(HELM_ERR_NOMEM, "cluster-tail image of problem %d", p);
        CKR(cudaStreamSynchronize(h->stream));
    }
    CKR(cudaMalloc((void **)&L->active, P * sizeof(int)));
    L->owned.push_back(L->active);
    CKR(cudaMalloc((void **)&L->tol_dev, sizeof(double)));
    L->owned.push_back(L->tol_dev);
    CKR(cudaMemset(L->active, 0, P * sizeof(int)));
    for (Phase &ph : L->phases) {
        std::vector<BLevel> pre, post;
        for (const auto &mb : ph.members) {
            helm_handle *h = L->h[mb.first];
            const int l = mb.second;
            LevelDev &Lv = h->lv[l], &Lc = h->lv[l + 1];
            BLevel e{};
            e.op = Lv.M32;
            e.b = Lv.b32;
            e.t = Lv.t32;
            e.coarse = Lc.b32;
            e.active = L->active + mb.first;
            pre.push_back(e);
            e.coarse = Lc.u32;
            e.u = l == 0 ? (float2 *)h->Z : Lv.u32;
            e.ustride = l == 0 ? h->np : 0;
            post.push_back(e);
        }
        CKR(upload(L, &ph.pre, pre));
        CKR(upload(L, &ph.post, post));
    }
    std::vector<BTail> tail(P);
    std::vector<BVec> vec(P);
    std::vector<unsigned> af(P + 1, 0), uf(P + 1, 0), df((size_t)(m + 1) * (P + 1), 0);
    L->dot_blocks.assign(m + 1, 0);
    for (int p = 0; p < P; p++) {
        helm_handle *h = L->h[p];
        const int nl = (int)h->lv.size(), t0 = nl - L->T;
        BTail &E = tail[p];
        for (int k = 0; k < L->T; k++) {
            E.cx[k] = h->lv[t0 + k].coef32[0];
            E.cy[k] = h->lv[t0 + k].coef32[1];
            E.k2[k] = h->lv[t0 + k].k2_32;
        }
        E.minv = h->minv32;
        E.b_top = h->lv[t0].b32;
        E.u_top = t0 == 0 ? (float2 *)h->Z : h->lv[t0].u32;
        E.ustride = t0 == 0 ? h->np : 0;
        E.img = ctail_image(h, false, L->deep);
        E.active = L->active + p;
        BVec &V = vec[p];
        V.n = h->np;
        V.V = (float4 *)h->V;
        V.Z = (float2 *)h->Z;
        V.b0 = h->lv[0].b32;
        V.A = h->Adf;
        V.partials = h->partials;
        V.hv = h->hv;
        V.alpha2 = h->alpha2;
        V.H = h->H;
        V.dcoef = h->dcoef;
        V.g = h->g;
        V.sn = h->sn;
        V.fnorm = h->fnorm_dev;
        V.cs = h->cs;
        V.est = h->est_dev;
        V.tickets = h->tickets;
        V.ldh = m + 1;
        V.active = L->active + p;
        af[p + 1] = af[p] + apply_A_df_blocks(h->n);
        uf[p + 1] = uf[p] + (unsigned)gs_df_update_nblocks(h->np);
        for (int j = 0; j <= m; j++) {
            unsigned *row = &df[(size_t)j * (P + 1)];
            row[p + 1] = row[p] + (unsigned)(gs_df_dot2_nblocks(h->np, j + 1) * gs_df_dot2_groups(j + 1));
        }
    }
    L->apply_blocks = af[P];
    L->upd_blocks = uf[P];
    for (int j = 0; j <= m; j++) L->dot_blocks[j] = df[(size_t)j * (P + 1) + P];
    CKR(upload(L, &L->tail, tail));
    CKR(upload(L, &L->vec, vec));
    CKR(upload(L, &L->apply_first, af));
    CKR(upload(L, &L->upd_first, uf));
    CKR(upload(L, &L->dot_first, df));
    if (L->est_h) cudaFreeHost(L->est_h);
    L->est_h = nullptr;
    CKR(cudaMallocHost((void **)&L->est_h, (size_t)(m + 1) * P * sizeof(double)));
    if (!L->active_h) CKR(cudaMallocHost((void **)&L->active_h, P * sizeof(int)));
    if (!L->norm_h) CKR(cudaMallocHost((void **)&L->norm_h, P * sizeof(double2)));
    if (!L->s) CKR(cudaStreamCreateWithFlags(&L->s, cudaStreamNonBlocking));
    if (!L->cap) CKR(cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking));
    if (!L->ev_in) CKR(cudaEventCreateWithFlags(&L->ev_in, cudaEventDisableTiming));
    if (!L->ev_out) CKR(cudaEventCreateWithFlags(&L->ev_out, cudaEventDisableTiming));
    if (!L->ev_fork) CKR(cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming));
    if ((int)L->pev.size() != P) {
        for (cudaEvent_t e : L->pev)
            if (e) cudaEventDestroy(e);
        L->pev.assign(P, nullptr);
        for (auto &e : L->pev) CKR(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    for (cudaEvent_t e : L->step_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : L->close_ev) cudaEventDestroy(e);
    L->step_ev.assign(m, nullptr);
    L->close_ev.assign(m + 1, nullptr);
    for (auto &e : L->step_ev) CKR(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto &e : L->close_ev) CKR(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    L->step_graph.assign(m, nullptr);
    L->close_graph.assign(m + 1, nullptr);
    L->m = m;
    L->P = P;
    L->key = key;
    CKR(cudaDeviceSynchronize());
    return HELM_OK;
}

// Launch timing under helm_profile (problem 0's profiler; eager launches only): the class and
// the algorithmic bytes of a batched launch summed over the problems still active.
struct Prof {
    BatchLockstep *L;
    const std::vector<char> *act;
    bool on() const { return L->h[0]->prof.on && !L->capturing; }
};
double interior(const LevelDev &Lv) { return (double)(Lv.n[0] - 2) * (Lv.n[1] - 2); }

// One batched step j (stream work only, capturable).
cudaError_t record_step(BatchLockstep *L, const Prof &pf, int j, cudaStream_t s) {
    const int P = L->P;
    const float om = (float)L->h[0]->mg.omega;
    helm_handle *h0 = L->h[0];
    {
        pdl_cycle_scope pdl;
        for (const Phase &ph : L->phases) {
            double bytes = 0, pass = 0;
            if (pf.on())
                for (const auto &mb : ph.members)
                    if ((*pf.act)[mb.first]) {
                        const double ni = interior(L->h[mb.first]->lv[mb.second]);
                        bytes += ni * (8 + 8 + 8 + 2);
                        pass += ni * (20 + 28 + 22);
                    }
            ProfScope ps(h0, ph.n[0] == h0->lv[0].n[0] ? HELM_K_SMOOTH_FINE : HELM_K_SMOOTH_COARSE, bytes, 0, pass);
            CKE(launch_pre2_restrict_batch(ph.n, ph.tile, (int)ph.members.size(), ph.pre, om, s));
        }
        {
            ProfScope ps(h0, HELM_K_COARSE, 0, 0);
            if (L->deep) CKE(launch_mg_chalo_batch(L->T, L->tail_ops, L->nu_c, 2, 2, om, L->nc, P, L->tail, j, s));
            else CKE(launch_mg_ctail_batch(L->T, L->tail_ops, L->nu_c, 2, 2, 0, om, 1, 1, L->nc, P, L->tail, j, s));
        }
        for (auto it = L->phases.rbegin(); it != L->phases.rend(); ++it) {
            const Phase &ph = *it;
            double bytes = 0, pass = 0;
            if (pf.on())
                for (const auto &mb : ph.members)
                    if ((*pf.act)[mb.first]) {
                        const double ni = interior(L->h[mb.first]->lv[mb.second]);
                        bytes += ni * (8 + 8 + 8 + 2 + 8);
                        pass += ni * (18 + 2 * 28);
                    }
            ProfScope ps(h0, ph.n[0] == h0->lv[0].n[0] ? HELM_K_SMOOTH_FINE : HELM_K_SMOOTH_COARSE, bytes, 0, pass);
            CKE(launch_prolong_post2_batch(ph.n, ph.tile, (int)ph.members.size(), ph.post, om, j, s));
        }
        double bytes = 0;
        if (pf.on())
            for (int p = 0; p < P; p++)
                if ((*pf.act)[p]) bytes += interior(L->h[p]->lv[0]) * (8 + 8 + 16);
        ProfScope ps(h0, HELM_K_APPLY, bytes, 0);
        CKE(launch_apply_A_df_batch(P, L->vec, L->apply_first, L->apply_blocks, j, s));
    }
    auto vec_bytes = [&](double per_node) {
        double b = 0;
        if (pf.on())
            for (int p = 0; p < P; p++)
                if ((*pf.act)[p]) b += (double)L->h[p]->np * per_node;
        return b;
    };
    const unsigned *row = L->dot_first + (size_t)j * (P + 1);
    {
        ProfScope ps(h0, HELM_K_MDOT, vec_bytes(16.0 * (j + 2)), 0);
        CKE(launch_mdot2_pair_batch(P, L->vec, row, L->dot_blocks[j], j, 0, s));
    }
    {
        pdl_cycle_scope pdl;
        ProfScope ps(h0, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce_dcgs2_batch(P, L->vec, row, gs_df_dot2_groups(j + 1), j, j > 0 ? 2 : 1, s));
    }
    if (j > 0) {
        ProfScope ps(h0, HELM_K_SMALL, 0, 0);
        CKE(launch_givens_batch(P, L->vec, j - 1, L->est_h + (size_t)(j - 1) * P, pf.on() ? nullptr : L->tol_dev, s));
    }
    {
        ProfScope ps(h0, HELM_K_UPDATE_NORM, vec_bytes(16.0 * (j + 4) + 8.0), 0);
        CKE(launch_update2_pair_batch(P, L->vec, L->upd_first, L->upd_blocks, j, s));
    }
    return L->capturing ? cudaEventRecordWithFlags(L->step_ev[j], s, cudaEventRecordExternal)
                        : cudaEventRecord(L->step_ev[j], s);
}

// The closing step of a cycle with jc columns: finishes column jc - 1 and its estimate.
cudaError_t record_close(BatchLockstep *L, const Prof &pf, int jc, cudaStream_t s) {
    const int P = L->P;
    helm_handle *h0 = L->h[0];
    const unsigned *row = L->dot_first + (size_t)jc * (P + 1);
    {
        double b = 0;
        if (pf.on())
            for (int p = 0; p < P; p++)
                if ((*pf.act)[p]) b += (double)L->h[p]->np * 16.0 * (jc + 1);
        ProfScope ps(h0, HELM_K_MDOT, b, 0);
        CKE(launch_mdot2_pair_batch(P, L->vec, row, L->dot_blocks[jc], jc, 1, s));
    }
    {
        ProfScope ps(h0, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce_dcgs2_batch(P, L->vec, row, gs_df_dot2_groups(jc + 1), jc, 0, s));
        CKE(launch_givens_batch(P, L->vec, jc - 1, L->est_h + (size_t)(jc - 1) * P, pf.on() ? nullptr : L->tol_dev, s));
    }
    return L->capturing ? cudaEventRecordWithFlags(L->close_ev[jc], s, cudaEventRecordExternal)
                        : cudaEventRecord(L->close_ev[jc], s);
}

// Eagerly while timing launches, else by replaying a CUDA graph captured on first use.
template <typename F> cudaError_t run(BatchLockstep *L, const Prof &pf, cudaGraphExec_t &exec, F work) {
    if (pf.on() || !L->graphs_ok) return work(L->s);
    if (!exec) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            pdl_capture_scope no_pdl;
            L->capturing = true;
            e = work(L->cap);
            L->capturing = false;
            cudaError_t e2 = cudaStreamEndCapture(L->cap, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            exec = nullptr;
            L->graphs_ok = false;
            return work(L->s);
        }
    }
    return cudaGraphLaunch(exec, L->s);
}

bool event_ready(cudaEvent_t e, cudaError_t *err) {
    *err = cudaEventSynchronize(e);
    return *err == cudaSuccess;
}

// Per-problem stream work (restarts, solution updates) for the problems in list, each on its own
// stream so that their small launches overlap: ordered after everything queued on the engine's
// stream so far, and joined back into it.
template <typename F> cudaError_t fan_out(BatchLockstep *L, const std::vector<int> &list, F work) {
    if (list.empty()) return cudaSuccess;
    CKE(cudaEventRecord(L->ev_fork, L->s));
    for (int p : list) {
        cudaStream_t ps = L->h[p]->stream;
        CKE(cudaStreamWaitEvent(ps, L->ev_fork, 0));
        CKE(work(p, ps));
        CKE(cudaEventRecord(L->pev[p], ps));
        CKE(cudaStreamWaitEvent(L->s, L->pev[p], 0));
    }
    return cudaSuccess;
}

cudaError_t norm_into(helm_handle *h, const double2 *x, double2 *out, cudaStream_t s) {
    CKE(launch_mdot_norm(h->np, nullptr, h->np, 0, x, h->partials, nullptr, s));
    return launch_reduce(h->partials, blas_nblocks(h->np), 1, out, 2, nullptr, s);
}

}  // namespace

bool lockstep_eligible(BatchLockstep *L) { return plan(L, false); }
const char *lockstep_why(const BatchLockstep *L) { return L->why.c_str(); }

BatchLockstep *lockstep_create(const std::vector<helm_handle *> &handles) {
    BatchLockstep *L = new (std::nothrow) BatchLockstep();
    if (L) L->h = handles;
    return L;
}

// The lockstep solve: same contract as helm_solve_batch.  The caller's stream is joined in and
// out through events.
helm_status lockstep_solve(BatchLockstep *L, cudaStream_t user, const void *const *rhs, void *const *x, double tol,
                           int m, int maxit, helm_stats *stats) {
    helm_status st = build(L, m);
    if (st != HELM_OK) return st;
    const int P = L->P;
    cudaStream_t s = L->s;
    CKR(cudaEventRecord(L->ev_in, user));
    CKR(cudaStreamWaitEvent(s, L->ev_in, 0));
    CKR(cudaMemcpyAsync(L->tol_dev, &tol, sizeof(double), cudaMemcpyHostToDevice, s));  // staged before return
    struct Run {
        const double2 *f;
        double2 *x;
        double fn = 0, rel = 1, est = 1;
        int it = 0, restarts = 0, jmax = 0;
        helm_status status = HELM_ERR_NOCONV;
        bool done = false;
    };
    std::vector<Run> r(P);
    std::vector<char> act(P, 0);
    Prof pf{L, &act};
    helm_handle *h0 = L->h[0];
    cudaStream_t keep0 = h0->stream;
    h0->stream = s;  // launch timing records its events on the stream the work runs on
    struct Restore {
        helm_handle *h;
        cudaStream_t k;
        ~Restore() { h->stream = k; }
    } restore{h0, keep0};
    std::vector<int> all(P);
    for (int p = 0; p < P; p++) {
        r[p].f = (const double2 *)rhs[p];
        r[p].x = (double2 *)x[p];
        all[p] = p;
    }
    CKR(fan_out(L, all, [&](int p, cudaStream_t ps) -> cudaError_t {
        helm_handle *h = L->h[p];
        CKE(norm_into(h, r[p].f, h->fnorm_dev, ps));
        return cudaMemcpyAsync(L->norm_h + p, h->fnorm_dev, sizeof(double2), cudaMemcpyDeviceToHost, ps);
    }));
    CKR(cudaStreamSynchronize(s));
    for (int p = 0; p < P; p++) {
        Run &R = r[p];
        R.fn = L->norm_h[p].x;
        if (!std::isfinite(R.fn)) {
            R.status = HELM_ERR_NONFINITE;
            R.done = true;
        } else if (R.fn == 0.0) {
            CKR(cudaMemsetAsync(R.x, 0, L->h[p]->np * sizeof(double2), s));
            R.status = HELM_OK;
            R.rel = R.est = 0.0;
            R.done = true;
        }
    }
    for (;;) {
        // restart of every unfinished problem: r0 = f - A x, ||r0|| (FP64 true residual)
        std::vector<int> pend;
        for (int p = 0; p < P; p++)
            if (!r[p].done) pend.push_back(p);
        if (pend.empty()) break;
        CKR(fan_out(L, pend, [&](int p, cudaStream_t ps) -> cudaError_t {
            helm_handle *h = L->h[p];
            CKE(launch_residual<double, double2>(h->A64, 2, r[p].f, r[p].x, h->V, ps));
            CKE(norm_into(h, h->V, h->scal, ps));
            return cudaMemcpyAsync(L->norm_h + p, h->scal, sizeof(double2), cudaMemcpyDeviceToHost, ps);
        }));
        CKR(cudaStreamSynchronize(s));
        std::vector<int> cyc;
        for (int p : pend) {
            Run &R = r[p];
            const double beta = L->norm_h[p].x;
            R.rel = beta / R.fn;
            if (!std::isfinite(beta)) { R.status = HELM_ERR_NONFINITE; R.done = true; continue; }
            if (R.rel <= tol) { R.status = HELM_OK; R.done = true; continue; }
            if (R.it >= maxit) { R.status = HELM_ERR_NOCONV; R.done = true; continue; }
            cyc.push_back(p);
        }
        if (cyc.empty()) continue;
        int jmax = 0;
        for (int p = 0; p < P; p++) {
            act[p] = 0;
            L->active_h[p] = 0;
        }
        for (int p : cyc) {
            Run &R = r[p];
            R.restarts++;
            R.jmax = std::min(m, maxit - R.it);
            jmax = std::max(jmax, R.jmax);
            act[p] = 1;
            L->active_h[p] = 1;
        }
        // v_0 = r0 / beta as a float-pair vector; its complex64 copy is the first cycle's input
        CKR(fan_out(L, cyc, [&](int p, cudaStream_t ps) -> cudaError_t {
            helm_handle *h = L->h[p];
            CKE(launch_split_scale(h->np, h->V, h->scal, ps));
            CKE(launch_cycle_start(h->g, m + 1, h->scal, nullptr, nullptr, 0.0, ps));
            return launch_pair_to_c64(h->np, (const float4 *)h->V, nullptr, h->lv[0].b32, ps);
        }));
        CKR(cudaMemcpyAsync(L->active, L->active_h, P * sizeof(int), cudaMemcpyHostToDevice, s));
        auto unit = [&](int k) -> cudaError_t {
            if (k + 1 < jmax)
                return run(L, pf, L->step_graph[k + 1], [&](cudaStream_t ss) { return record_step(L, pf, k + 1, ss); });
            return run(L, pf, L->close_graph[jmax], [&](cudaStream_t ss) { return record_close(L, pf, jmax, ss); });
        };
        auto unit_event = [&](int k) { return k + 1 < jmax ? L->step_ev[k + 1] : L->close_ev[jmax]; };
        CKR(run(L, pf, L->step_graph[0], [&](cudaStream_t ss) { return record_step(L, pf, 0, ss); }));
        for (int k = 0; k < 3 && k < jmax; k++) CKR(unit(k));
        std::vector<int> live = cyc;
        for (int j = 0; j < jmax && !live.empty(); j++) {
            cudaError_t err;
            if (!event_ready(unit_event(j), &err)) return helm_fail(HELM_ERR_CUDA, "event: %s", cudaGetErrorString(err));
            std::vector<int> still, leave;
            for (int p : live) {
                Run &R = r[p];
                R.est = L->est_h[(size_t)j * P + p];
                R.it++;
                helm_stats *sp = stats ? &stats[p] : nullptr;
                if (sp && sp->history && R.it - 1 < sp->history_len) sp->history[R.it - 1] = R.est;
                const bool bad = !std::isfinite(R.est);
                if (bad || R.est <= tol || j + 1 >= R.jmax) {
                    // the problem leaves the lockstep, then x += Z y over its first j + 1
                    // columns.  On convergence the rotation that formed the estimate has already
                    // cleared its flag, so the steps queued behind it skip the problem; otherwise
                    // (a full cycle, a non-finite estimate, or launches timed one by one, where
                    // the rotation leaves the flags alone) the flag is cleared here, behind them
                    // (they only write columns and slots past j)
                    act[p] = 0;
                    if (pf.on() || !(R.est <= tol)) CKR(cudaMemsetAsync(L->active + p, 0, sizeof(int), s));
                    if (bad) {
                        R.status = HELM_ERR_NONFINITE;
                        R.done = true;
                        continue;
                    }
                    leave.push_back(p);
                    continue;
                }
                still.push_back(p);
            }
            // x += Z y of the problems that left at this step, side by side (the steps already
            // queued only write their columns and slots past j)
            CKR(fan_out(L, leave, [&](int p, cudaStream_t ps) -> cudaError_t {
                helm_handle *h = L->h[p];
                CKE(launch_backsolve(h->H, m + 1, j + 1, h->g, h->y, ps));
                return launch_combine<float2>(h->np, (const float2 *)h->Z, h->np, j + 1, h->y, h->alpha2, r[p].x, ps);
            }));
            live.swap(still);
            if (!live.empty() && j + 3 < jmax) CKR(unit(j + 3));
        }
    }
    CKR(cudaEventRecord(L->ev_out, s));
    CKR(cudaStreamWaitEvent(user, L->ev_out, 0));
    CKR(cudaStreamSynchronize(s));
    helm_status worst = HELM_OK;
    for (int p = 0; p < P; p++) {
        const Run &R = r[p];
        if (stats) {
            stats[p].iterations = R.it;
            stats[p].restarts = R.restarts;
            stats[p].rel_res = R.rel;
            stats[p].est_res = R.est;
            stats[p].status = R.status;
            stats[p].reorthogonalizations = R.it;
        }
        if (R.status != HELM_OK && worst == HELM_OK) worst = R.status;
    }
    if (worst != HELM_OK)
        return helm_fail(worst, "%s in at least one batch problem", worst == HELM_ERR_NOCONV ? "no convergence" : "failure");
    return HELM_OK;
}
