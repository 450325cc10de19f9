// Outer Krylov drivers on the device: flexible GMRES(m) and Bi-CGSTAB, right-preconditioned
// by one multigrid cycle (Algorithm 1) in FP32 or FP64, with every vector operation, every
// inner product, the Givens rotations and the least-squares back substitution in FP64 on the
// GPU.  The host only sequences launches and reads one residual estimate per iteration.
//
// Flexible GMRES: Saad, Iterative Methods for Sparse Linear Systems, Algorithm 9.6, with
// classical Gram-Schmidt (two fused passes: dot + norm, update + norm) and a second
// Gram-Schmidt pass whenever the DGKS test asks for it, in place of modified Gram-Schmidt;
// the Gram-Schmidt arithmetic is FP64 or double-FP32 (helm_gs_arith).  Bi-CGSTAB: van der
// Vorst (1992), right preconditioning, two preconditioner cycles per iteration as in
// Section 5 of the paper.
#include <math.h>
#include <string.h>

#include <chrono>

#include "helm_handle.h"

#define CKR(...)                                                                                           \
    do {                                                                                                   \
        cudaError_t e_ = (__VA_ARGS__);                                                                           \
        if (e_ != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_));   \
    } while (0)

// DGKS threshold: re-orthogonalise when one Gram-Schmidt pass removed more than 1 - 1/sqrt(2)
// of the vector's norm (Daniel, Gragg, Kaufman & Stewart, Math. Comp. 30, 1976).
static const double kDGKSEta = 0.70710678118654752;

static void free_krylov(helm_handle *h) {
    for (cudaGraphExec_t g : h->step_graph)
        if (g) cudaGraphExecDestroy(g);
    h->step_graph.clear();
    for (cudaGraphExec_t g : h->close_graph)
        if (g) cudaGraphExecDestroy(g);
    h->close_graph.clear();
    for (cudaEvent_t e : h->step_ev)
        if (e) cudaEventDestroy(e);
    h->step_ev.clear();
    for (cudaEvent_t e : h->close_ev)
        if (e) cudaEventDestroy(e);
    h->close_ev.clear();
    h->hv = h->alpha2 = h->dcoef = nullptr;
    h->tickets = nullptr;
    for (void *p : h->krylov_owned) cudaFree(p);
    h->krylov_owned.clear();
    h->V = nullptr; h->Z = nullptr; h->H = nullptr; h->g = h->sn = h->y = h->h2 = nullptr;
    h->cs = nullptr; h->partials = nullptr; h->scal = nullptr; h->est_dev = nullptr; h->tol_dev = nullptr;
    h->gs_flag = h->gs_count = nullptr;
    h->m_alloc = 0;
    h->bicg_alloc = false;
    h->br = h->brh = h->bp = h->bv = h->bs = h->bt = nullptr;
    h->by = h->bz = nullptr;
}

void helm_free_krylov(helm_handle *h) { free_krylov(h); }

void helm_drop_graphs(helm_handle *h) {
    for (auto *v : {&h->step_graph, &h->close_graph})
        for (cudaGraphExec_t &g : *v)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

template <typename T> static cudaError_t kalloc(helm_handle *h, T **p, size_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
    if (e == cudaSuccess) {
        h->krylov_owned.push_back(*p);
        e = cudaMemsetAsync(*p, 0, (count ? count : 1) * sizeof(T), h->stream);
    }
    return e;
}

static helm_prec z_precision(const helm_handle *h) {
    return h->mg.kind == HELM_PC_NONE ? HELM_C128 : h->mg.prec;
}

static helm_status ensure_ws(helm_handle *h, int m) {
    const helm_prec zp = z_precision(h);
    if (h->m_alloc >= m && h->z_prec == zp && h->V) return HELM_OK;
    // grow: release only the GMRES part; keep it simple by releasing everything
    free_krylov(h);
    const size_t np = h->np;
    const int nblk = blas_nblocks(np);
    cudaError_t e = cudaSuccess;
#define KA(ptr, cnt) if (e == cudaSuccess) e = kalloc(h, ptr, cnt)
    KA(&h->V, (size_t)(m + 1) * np);
    if (zp == HELM_C64) { float2 *z; KA(&z, (size_t)m * np); h->Z = z; }
    else { double2 *z; KA(&z, (size_t)m * np); h->Z = z; }
    KA(&h->H, (size_t)(m + 1) * m);
    KA(&h->g, (size_t)m + 1);
    KA(&h->sn, (size_t)m);
    KA(&h->y, (size_t)m);
    KA(&h->h2, (size_t)m + 1);
    KA(&h->cs, (size_t)m);
    KA(&h->partials, (size_t)nblk * std::max(65, 2 * m + 4));
    KA(&h->hv, (size_t)2 * m + 4);
    KA(&h->alpha2, (size_t)m + 2);
    KA(&h->dcoef, (size_t)2 * m + 4);
    KA(&h->tickets, 4);
    KA(&h->scal, 32);
    KA(&h->est_dev, (size_t)m + 4);
    KA(&h->tol_dev, 1);
    KA(&h->gs_flag, 4);
    h->gs_count = h->gs_flag + 1;
#undef KA
    if (e != cudaSuccess) {
        free_krylov(h);
        return helm_fail(e == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA, "Krylov workspace: %s",
                         cudaGetErrorString(e));
    }
    if (h->est_host_len < m + 8) {
        if (h->est_host) cudaFreeHost(h->est_host);
        h->est_host = nullptr;
        h->est_host_len = 0;
        CKR(cudaMallocHost((void **)&h->est_host, (size_t)(m + 8) * sizeof(double)));
        h->est_host_len = m + 8;
    }
    h->step_ev.assign((size_t)m, nullptr);
    for (int j = 0; j < m; j++) CKR(cudaEventCreateWithFlags(&h->step_ev[j], cudaEventDisableTiming));
    h->step_graph.assign((size_t)m, nullptr);
    h->close_ev.assign((size_t)m + 1, nullptr);
    for (int j = 0; j <= m; j++) CKR(cudaEventCreateWithFlags(&h->close_ev[j], cudaEventDisableTiming));
    h->close_graph.assign((size_t)m + 1, nullptr);
    if (!h->ev_fn) CKR(cudaEventCreateWithFlags(&h->ev_fn, cudaEventDisableTiming));
    if (!h->ev_beta) CKR(cudaEventCreateWithFlags(&h->ev_beta, cudaEventDisableTiming));
    if (!h->cap_stream) CKR(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (!h->side) CKR(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    if (!h->ev_fork) CKR(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (!h->ev_join) CKR(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    h->fnorm_dev = h->scal + 24;
    h->m_alloc = m;
    h->z_prec = zp;
    return HELM_OK;
}

helm_status helm_ensure_krylov(helm_handle *h, int m) { return ensure_ws(h, m); }

static helm_status ensure_bicg(helm_handle *h) {
    helm_status st = ensure_ws(h, 1);
    if (st != HELM_OK) return st;
    if (h->bicg_alloc) return HELM_OK;
    const size_t np = h->np;
    cudaError_t e = cudaSuccess;
    double2 **vv[6] = {&h->br, &h->brh, &h->bp, &h->bv, &h->bs, &h->bt};
    for (auto p : vv)
        if (e == cudaSuccess) e = kalloc(h, p, np);
    if (h->z_prec == HELM_C64) {
        float2 *a = nullptr, *b = nullptr;
        if (e == cudaSuccess) e = kalloc(h, &a, np);
        if (e == cudaSuccess) e = kalloc(h, &b, np);
        h->by = a; h->bz = b;
    } else {
        double2 *a = nullptr, *b = nullptr;
        if (e == cudaSuccess) e = kalloc(h, &a, np);
        if (e == cudaSuccess) e = kalloc(h, &b, np);
        h->by = a; h->bz = b;
    }
    if (e != cudaSuccess) return helm_fail(HELM_ERR_NOMEM, "Bi-CGSTAB workspace: %s", cudaGetErrorString(e));
    h->bicg_alloc = true;
    return HELM_OK;
}

// ||x||_2 -> out (device scalar, .x); optionally read back to the host.
// out = (||x||, 0) on the device; with host_out (pinned), *host_out = ||x|| too.
static cudaError_t dev_norm(helm_handle *h, const double2 *x, double2 *out, double *host_out = nullptr) {
    ProfScope ps(h, HELM_K_VECTOR, h->np * 16.0, h->np * 4.0);
    cudaError_t e = launch_mdot_norm(h->np, nullptr, h->np, 0, x, h->partials, nullptr, h->stream);
    if (e != cudaSuccess) return e;
    return launch_reduce(h->partials, blas_nblocks(h->np), 1, out, 2, nullptr, h->stream, host_out);
}

static cudaError_t dev_dot(helm_handle *h, const double2 *a, const double2 *b, double2 *out) {
    ProfScope ps(h, HELM_K_VECTOR, h->np * 32.0, h->np * 12.0);
    cudaError_t e = launch_mdot_norm(h->np, a, h->np, 1, b, h->partials, nullptr, h->stream);
    if (e != cudaSuccess) return e;
    return launch_reduce(h->partials, blas_nblocks(h->np), 1, out, 0, nullptr, h->stream);
}

static helm_status read_scalars(helm_handle *h, const void *dev, size_t bytes, void *host) {
    CKR(cudaMemcpyAsync(h->est_host, dev, bytes, cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    memcpy(host, h->est_host, bytes);
    return HELM_OK;
}

// Algorithmic cost of one FP64 apply over the interior (read x, k^2, write y; 5- or 7-point
// complex stencil: one complex multiply-add per neighbour and for the diagonal, plus the
// diagonal's assembly).
static double interior_pts(const helm_handle *h) {
    return (double)(h->n[0] - 2) * (h->n[1] - 2) * (h->dim == 3 ? (double)(h->n[2] - 2) : 1.0);
}
static double apply_flops(const helm_handle *h) { return interior_pts(h) * (h->dim == 3 ? 68.0 : 48.0); }

// Double-FP32 Arnoldi (gs_arith = DF): the basis vectors are float-pair vectors.
// z = precondition(v / alpha->x) in the workspace precision (alpha null: v); w = A z as a
// float-pair vector.
static cudaError_t precond_apply_pair(helm_handle *h, const float4 *v, const double2 *alpha, void *z, float4 *w) {
    cudaError_t e;
    const double ni = interior_pts(h);
    if (h->z_prec == HELM_C64) {
        e = precondition_pair<float>(h, v, alpha, (float2 *)z);
        if (e != cudaSuccess) return e;
        ProfScope ps(h, HELM_K_APPLY, ni * (8 + 8 + 16), 0);
        return launch_apply_A_df(h->Adf, h->dim, (const float2 *)z, w, h->stream);
    }
    e = precondition_pair<double>(h, v, alpha, (double2 *)z);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(h, HELM_K_APPLY, ni * (16 + 8 + 16), apply_flops(h));
        e = launch_apply<double, double2>(h->A64, h->dim, (const double2 *)z, (double2 *)w, h->stream);
        if (e != cudaSuccess) return e;
    }
    ProfScope ps(h, HELM_K_VECTOR, h->np * 32.0, 0);
    return launch_split_scale(h->np, w, nullptr, h->stream);
}

// Delayed CGS2 with a complex64 multigrid cycle: the update pass writes each new basis vector
// straight into level 0's right-hand side, unscaled (see fgmres_step_dcgs2).
static bool dcgs2_fold(const helm_handle *h) {
    return h->mg.gs_arith == HELM_GS_DCGS2 && h->z_prec == HELM_C64 && h->mg.kind != HELM_PC_NONE;
}

// z = cycle(level 0's right-hand side) in complex64; w = A z as a float-pair vector.  When the
// device flag gate is set at launch, the levels' smoothing, residual and transfer kernels (all but
// the fused coarse tails) and the apply do nothing.
static cudaError_t precond_apply_level0(helm_handle *h, float2 *z, float4 *w, const int *gate) {
    pdl_cycle_scope pdl;  // the apply follows the cycle's last kernel
    for (LevelDev &L : h->lv) L.M32.gate = gate;  // for these launches only
    cudaError_t e = precondition_level0_c64(h, z);
    for (LevelDev &L : h->lv) L.M32.gate = nullptr;
    if (e != cudaSuccess) return e;
    ProfScope ps(h, HELM_K_APPLY, interior_pts(h) * (8 + 8 + 16), 0);
    return launch_apply_A_df(h->Adf, h->dim, z, w, h->stream, gate);
}

// Device flag of the current FGMRES cycle: set by the rotation kernel when a residual estimate
// meets the tolerance, cleared at the start of every cycle.
static int *stop_flag(helm_handle *h) { return h->gs_flag + 2; }

// z = precondition(v) in the workspace precision; w = A z (FP64)
static cudaError_t precond_apply(helm_handle *h, const double2 *v, void *z, double2 *w) {
    cudaError_t e;
    const double ni = interior_pts(h);
    if (h->z_prec == HELM_C64) {
        e = precondition<float>(h, v, (float2 *)z);
        if (e != cudaSuccess) return e;
        ProfScope ps(h, HELM_K_APPLY, ni * (8 + 8 + 16), apply_flops(h));
        return launch_apply<double, float2>(h->A64, h->dim, (const float2 *)z, w, h->stream);
    }
    e = precondition<double>(h, v, (double2 *)z);
    if (e != cudaSuccess) return e;
    ProfScope ps(h, HELM_K_APPLY, ni * (16 + 8 + 16), apply_flops(h));
    return launch_apply<double, double2>(h->A64, h->dim, (const double2 *)z, w, h->stream);
}

#define CKE(...)                          \
    do {                                  \
        cudaError_t e_ = (__VA_ARGS__);   \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// One FGMRES step j of a restart cycle (Saad, Algorithm 9.6): z_j = cycle(v_j); w = A z_j;
// Gram-Schmidt of w against v_0..v_j into H[:, j] with the DGKS second pass; v_{j+1} = w / h;
// Givens rotations; the relative residual estimate |g_{j+1}| / ||f|| goes to est[j] and is
// copied to pinned host memory, then the step's event is recorded.  Stream work only (no host
// synchronisation), so a step can be captured into a CUDA graph and replayed.  A step only
// writes column j of H, v_{j+1}, z_j, the rotation j and g[j..j+1].
static cudaError_t fgmres_step(helm_handle *h, int j, int m) {
    const size_t np = h->np;
    const int ldh = m + 1;
    cudaStream_t s = h->stream;
    const size_t zsz = h->z_prec == HELM_C64 ? sizeof(float2) : sizeof(double2);
    // Gram-Schmidt passes in FP64, or in double-FP32 on float-pair basis vectors (same
    // partials layout)
    const bool df = h->mg.gs_arith == HELM_GS_DF;
    const int gblk = df ? gs_df_nblocks(np) : blas_nblocks(np);         // blocks of the dot pass
    const int ublk = df ? gs_df_update_nblocks(np) : blas_nblocks(np);  // blocks of the update pass
    const float4 *V4 = (const float4 *)h->V;
    auto gs_dot = [&](int nv, double2 *w, const int *gate) {
        return df ? launch_mdot_norm_pair(np, V4, np, nv, (const float4 *)w, h->partials, gate, s)
                  : launch_mdot_norm(np, h->V, np, nv, w, h->partials, gate, s);
    };
    auto gs_update = [&](int nv, const double2 *hh, double2 *w, const int *gate) {
        return df ? launch_update_norm_pair(np, V4, np, nv, hh, (float4 *)w, h->partials, gate, s)
                  : launch_update_norm(np, h->V, np, nv, hh, w, h->partials, gate, s);
    };
    double2 *vj = h->V + (size_t)j * np, *w = h->V + (size_t)(j + 1) * np;
    void *zj = (char *)h->Z + (size_t)j * np * zsz;
    if (df) CKE(precond_apply_pair(h, (const float4 *)vj, nullptr, zj, (float4 *)w));
    else CKE(precond_apply(h, vj, zj, w));
    double2 *hcol = h->H + (size_t)ldh * j;
    const double nv = j + 1;
    // Classical Gram-Schmidt with the DGKS re-orthogonalisation test:
    //   h = V^H w (and ||w||^2 into H[j+1][j]);  w -= V h, ||w'||;
    //   if ||w'|| < eta ||w||:  h' = V^H w, H[:, j] += h';  w -= V h', ||w''||.
    // The second pass runs only when the device flag is set (gated kernels).
    {
        // FP64 flops only when the FP64 units do them (double-FP32 work is not FP64-bound)
        ProfScope ps(h, HELM_K_MDOT, np * 16.0 * (nv + 1), df ? 0.0 : np * (8.0 * nv + 4.0));
        CKE(gs_dot(j + 1, w, nullptr));
    }
    {
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce(h->partials, gblk, j + 2, hcol, 0, nullptr, s));
    }
    {
        ProfScope ps(h, HELM_K_UPDATE_NORM, np * 16.0 * (nv + 2), df ? 0.0 : np * (8.0 * nv + 4.0));
        CKE(gs_update(j + 1, hcol, w, nullptr));
    }
    {
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce_decide(h->partials, ublk, hcol + j + 1, h->gs_flag, h->gs_count, kDGKSEta, s));
    }
    // Under launch timing (eager steps, never captured) the host reads the decision, so that
    // the gated pass's bytes are attributed exactly when it runs.
    double pass2 = 0.0;
    if (h->prof.on) {
        int flag = 0;
        CKE(cudaMemcpyAsync(&flag, h->gs_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CKE(cudaStreamSynchronize(s));
        pass2 = flag ? 1.0 : 0.0;
    }
    {
        ProfScope ps(h, HELM_K_MDOT, pass2 * np * 16.0 * (nv + 1), df ? 0.0 : pass2 * np * (8.0 * nv + 4.0));
        CKE(gs_dot(j + 1, w, h->gs_flag));
    }
    {
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce(h->partials, gblk, j + 1, h->h2, 0, h->gs_flag, s));
        CKE(launch_reduce(h->partials, gblk, j + 1, hcol, 1, h->gs_flag, s));
    }
    {
        ProfScope ps(h, HELM_K_UPDATE_NORM, pass2 * np * 16.0 * (nv + 2), df ? 0.0 : pass2 * np * (8.0 * nv + 4.0));
        CKE(gs_update(j + 1, h->h2, w, h->gs_flag));
    }
    {
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce(h->partials, ublk, 1, hcol + j + 1, 2, h->gs_flag, s));
    }
    {
        ProfScope ps(h, HELM_K_VECTOR, np * 32.0, df ? 0.0 : np * 2.0);
        if (df) CKE(launch_scale_inv_pair(np, (float4 *)w, hcol + j + 1, s));
        else CKE(launch_scale_inv(np, w, hcol + j + 1, w, s));
    }
    {
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_givens(h->H, ldh, j, h->cs, h->sn, h->g, h->fnorm_dev, h->est_dev, h->est_host, nullptr, nullptr, s));
    }
    // inside a capture the record must become an event node of the graph (external), so that
    // the host can wait on the event after every replay
    return h->capturing ? cudaEventRecordWithFlags(h->step_ev[j], s, cudaEventRecordExternal)
                        : cudaEventRecord(h->step_ev[j], s);
}

// Delayed CGS2 step j (gs_arith = DCGS2; float-pair basis).  Basis slot j holds x_j = alpha_j
// u_j, the once-orthogonalised vector of step j - 1 (not normalised: alpha_j = ||x_j|| is in
// alpha2[j], and the division by it is folded into the next consumers; slot 0 holds v_0).
//   z_j = cycle(x_j / alpha_j); w = A z_j                        (slot j + 1)
//   one pass: V_i^H x_j and V_i^H w for i <= j (k_mdot2_pair); their reduction, whose last
//   block forms the coefficients: finish column j - 1 of H (reorthogonalisation of u_j),
//   first-pass column j;
//   the Givens rotation of column j - 1 and its residual estimate est[j - 1] run on a side
//   stream beside the update pass
//   one pass: slot j <- v_j (final), slot j + 1 <- w orthogonalised once; its last block forms
//   alpha_{j+1} = ||w||
// Only column j - 1 of H, the first-pass column j, rotation j - 1, g[j-1..j], slots j and j + 1
// and z_j are written, so a step queued ahead of the host's decision never disturbs columns
// 0 .. j - 2 that a solution update may use.
static cudaError_t fgmres_step_dcgs2(helm_handle *h, int j, int m) {
    const size_t np = h->np;
    const int ldh = m + 1;
    cudaStream_t s = h->stream;
    const size_t zsz = h->z_prec == HELM_C64 ? sizeof(float2) : sizeof(double2);
    float4 *V4 = (float4 *)h->V;
    float4 *u = V4 + (size_t)j * np, *w = V4 + (size_t)(j + 1) * np;
    void *zj = (char *)h->Z + (size_t)j * np * zsz;
    const double nv = j + 1;
    // With a complex64 cycle, the previous update pass left x_j itself (not x_j / alpha_j) in
    // level 0's right-hand side, so z_j and w come out alpha_j times too large: the coefficient
    // step, the update pass and the solution update divide by alpha_j (the cycle and A are
    // linear), and no conversion launch is needed.
    const bool fold = dcgs2_fold(h), scaled = fold && j > 0;
    // steps queued behind a converged one (the host learns of it one or two steps later) skip
    // their work: the rotation that met the tolerance sets the flag.  Not while launches are
    // timed one by one (helm_profile), so that every timed launch does its full work.
    int *stop = h->prof.on ? nullptr : stop_flag(h);
    if (scaled) CKE(precond_apply_level0(h, (float2 *)zj, w, stop));
    else CKE(precond_apply_pair(h, u, j > 0 ? h->alpha2 + j : nullptr, zj, w));
    {
        ProfScope ps(h, HELM_K_MDOT, np * 16.0 * (nv + 1), 0);
        CKE(launch_mdot2_pair(np, V4, np, j + 1, u, w, h->partials, stop, s));
    }
    {
        // reduction and, in its last block, the coefficient step (its few blocks may be scheduled
        // while the dot pass drains)
        pdl_cycle_scope pdl;
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce_dcgs2(h->partials, gs_df_dot2_nblocks(np, j + 1), h->hv, h->tickets, j, h->alpha2, h->H, ldh,
                                h->dcoef, scaled ? 2 : 1, s));
    }
    const bool fork = j > 0 && !h->prof.on;
    if (j > 0) {
        // column j - 1 is final: its rotation on the side stream (inline while timing launches)
        cudaStream_t gs = fork ? h->side : s;
        if (fork) {
            CKE(cudaEventRecord(h->ev_fork, s));
            CKE(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        }
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_givens(h->H, ldh, j - 1, h->cs, h->sn, h->g, h->fnorm_dev, h->est_dev, h->est_host,
                          stop ? h->tol_dev : nullptr, stop, gs));
        if (fork) CKE(cudaEventRecord(h->ev_join, h->side));
    }
    {
        // the update and the norm of the new vector in one launch; launched programmatically, so
        // that its blocks are placed on the SMs while the few blocks of the reduction finish
        // (about 2 us per step; the same attribute on the dot pass, which follows the many-block
        // apply, spread its one-wave grid unevenly and cost 36 us per step)
        pdl_cycle_scope pdl;
        ProfScope ps(h, HELM_K_UPDATE_NORM, np * 16.0 * (nv + 3), 0);
        CKE(launch_update2_pair(np, V4, np, j, h->dcoef, h->partials, h->tickets + 1, h->alpha2 + j + 1,
                                fold ? level0_rhs_c64(h) : nullptr, stop, s));
    }
    if (fork) CKE(cudaStreamWaitEvent(s, h->ev_join, 0));
    return h->capturing ? cudaEventRecordWithFlags(h->step_ev[j], s, cudaEventRecordExternal)
                        : cudaEventRecord(h->step_ev[j], s);
}

// Closing step of a delayed-CGS2 cycle with jc columns: the inner products of x_jc with
// v_0 .. v_{jc-1} only finish column jc - 1 of H, then its rotation and est[jc - 1].
static cudaError_t fgmres_close_dcgs2(helm_handle *h, int jc, int m) {
    const size_t np = h->np;
    const int ldh = m + 1;
    cudaStream_t s = h->stream;
    const float4 *V4 = (const float4 *)h->V;
    {
        // the two-vector pass with x in both places: its first jc + 1 sums are V_i^H x, i < jc,
        // and x^H x (slot jc is x)
        ProfScope ps(h, HELM_K_MDOT, np * 16.0 * (jc + 1), 0);
        const float4 *x = V4 + (size_t)jc * np;
        CKE(launch_mdot2_pair(np, V4, np, jc + 1, x, x, h->partials, nullptr, s));
    }
    {
        // the reduction and, in its last block, the coefficient step that finishes column jc - 1
        // only (the batched engine runs the same two launches)
        ProfScope ps(h, HELM_K_SMALL, 0, 0);
        CKE(launch_reduce_dcgs2(h->partials, gs_df_dot2_nblocks(np, jc + 1), h->hv, h->tickets, jc, h->alpha2, h->H,
                                ldh, h->dcoef, 0, s));
        CKE(launch_givens(h->H, ldh, jc - 1, h->cs, h->sn, h->g, h->fnorm_dev, h->est_dev, h->est_host, nullptr,
                          nullptr, s));
    }
    return h->capturing ? cudaEventRecordWithFlags(h->close_ev[jc], s, cudaEventRecordExternal)
                        : cudaEventRecord(h->close_ev[jc], s);
}

// Runs a piece of stream work eagerly while launch timing is on, else by replaying a CUDA
// graph of it, captured on the handle's private stream on first use with this workspace.
template <typename F>
static cudaError_t run_graph(helm_handle *h, cudaGraphExec_t &exec, F work) {
    if (h->prof.on || !h->graphs_ok) return work();
    if (!exec) {
        cudaStream_t keep = h->stream;
        cudaGraph_t g = nullptr;
        h->stream = h->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            pdl_capture_scope no_pdl;
            h->capturing = true;
            e = work();
            h->capturing = false;
            cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
            if (e == cudaSuccess) e = e2;
        }
        h->stream = keep;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {  // run this handle eagerly from now on
            cudaGetLastError();
            exec = nullptr;
            h->graphs_ok = false;
            return work();
        }
    }
    return cudaGraphLaunch(exec, h->stream);
}

static bool use_dcgs2(const helm_handle *h) { return h->mg.gs_arith == HELM_GS_DCGS2; }

// Step j of the cycle (either Gram-Schmidt variant).
static cudaError_t run_step(helm_handle *h, int j, int m) {
    if (use_dcgs2(h)) return run_graph(h, h->step_graph[j], [&] { return fgmres_step_dcgs2(h, j, m); });
    return run_graph(h, h->step_graph[j], [&] { return fgmres_step(h, j, m); });
}

// The work that makes est[k] available in a cycle of jmax columns (delayed CGS2): step k + 1,
// or the closing step after the last column.
static cudaError_t run_unit(helm_handle *h, int k, int jmax, int m) {
    if (k + 1 < jmax) return run_step(h, k + 1, m);
    return run_graph(h, h->close_graph[jmax], [&] { return fgmres_close_dcgs2(h, jmax, m); });
}

static cudaEvent_t unit_event(helm_handle *h, int k, int jmax) {
    return k + 1 < jmax ? h->step_ev[k + 1] : h->close_ev[jmax];
}

// ---------------------------------------------------------------------------------- FGMRES
// The outer loop is a resumable state machine so that one host thread can drive many
// problems at once (helm_solve_batch): every phase enqueues stream work and then waits for
// one event, which fgmres_advance either blocks on or polls.
//   WAIT_FN     ||f|| read back                      -> START
//   START       r0 = f - A x, ||r0|| read back        -> WAIT_BETA
//   WAIT_BETA   converged / capped / new cycle        -> DONE or IN_CYCLE
//   IN_CYCLE    step j's estimate read back; step j+2 queued (one step of look-ahead; delayed
//               CGS2: unit j+3, two steps);
//               converged or cycle full: x += Z y     -> START
// Pinned host slots, written by the kernels that form the values (no copy in the stream; the
// host reads a slot once the phase's event has fired): est_host[0..m) step estimates,
// [m+2] ||f||, [m+4] ||r0||.

static bool event_ready(cudaEvent_t e, bool block, cudaError_t *err) {
    *err = cudaSuccess;
    if (block) {
        *err = cudaEventSynchronize(e);
        return *err == cudaSuccess;
    }
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) return true;
    if (q != cudaErrorNotReady) *err = q;
    return false;
}

helm_status fgmres_begin(helm_handle *h, FgmresRun &r, const double2 *f, double2 *x, double tol, int m, int maxit,
                         helm_stats *st) {
    helm_status s0 = ensure_ws(h, m);
    if (s0 != HELM_OK) return s0;
    r = FgmresRun{};
    r.h = h; r.f = f; r.x = x; r.tol = tol; r.m = m; r.maxit = maxit; r.st = st;
    r.status = HELM_ERR_NOCONV;
    r.phase = FgmresRun::WAIT_FN;
    cudaStream_t s = h->stream;
    CKR(cudaMemsetAsync(h->gs_flag, 0, 3 * sizeof(int), s));
    CKR(dev_norm(h, f, h->fnorm_dev, h->est_host + m + 2));
    CKR(cudaEventRecord(h->ev_fn, s));
    return HELM_OK;
}

static helm_status fgmres_finish(FgmresRun &r) {
    helm_handle *h = r.h;
    r.phase = FgmresRun::DONE;
    helm_status rs;
    if (r.st) {
        int cnt[2] = {0, 0};
        if ((rs = read_scalars(h, h->gs_flag, 2 * sizeof(int), cnt)) != HELM_OK) return rs;
        r.st->iterations = r.it;
        r.st->restarts = r.restarts;
        r.st->rel_res = r.rel;
        r.st->est_res = r.est;
        r.st->status = r.status;
        // delayed CGS2 reorthogonalises every basis vector
        r.st->reorthogonalizations = use_dcgs2(h) ? r.it : cnt[1];
    } else {
        CKR(cudaStreamSynchronize(h->stream));
    }
    return HELM_OK;
}

// Performs every phase whose wait is satisfied (all of them when block is true).  Returns
// HELM_OK while running or finished; r.phase == DONE and r.status hold the outcome.
helm_status fgmres_advance(FgmresRun &r, bool block) {
    helm_handle *h = r.h;
    cudaStream_t s = h->stream;
    const size_t np = h->np;
    const int m = r.m, ldh = m + 1;
    cudaError_t err;
    for (;;) {
        switch (r.phase) {
        case FgmresRun::DONE:
            return HELM_OK;
        case FgmresRun::WAIT_FN: {
            if (!event_ready(h->ev_fn, block, &err)) {
                if (err != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "event: %s", cudaGetErrorString(err));
                return HELM_OK;
            }
            r.fn = h->est_host[m + 2];
            if (!std::isfinite(r.fn)) {
                r.status = HELM_ERR_NONFINITE;
                return fgmres_finish(r);
            }
            if (r.fn == 0.0) {
                CKR(cudaMemsetAsync(r.x, 0, np * sizeof(double2), s));
                r.status = HELM_OK;
                r.rel = r.est = 0.0;
                return fgmres_finish(r);
            }
            r.phase = FgmresRun::START;
            break;
        }
        case FgmresRun::START: {
            // r0 = f - A x -> V_0, beta = ||r0|| (FP64 true residual)
            {
                ProfScope ps(h, HELM_K_APPLY, interior_pts(h) * (16 + 16 + 8 + 16),
                             apply_flops(h) + 2 * interior_pts(h));
                CKR(launch_residual<double, double2>(h->A64, h->dim, r.f, r.x, h->V, s));
            }
            CKR(dev_norm(h, h->V, h->scal, h->est_host + m + 4));
            CKR(cudaEventRecord(h->ev_beta, s));
            r.phase = FgmresRun::WAIT_BETA;
            break;
        }
        case FgmresRun::WAIT_BETA: {
            if (!event_ready(h->ev_beta, block, &err)) {
                if (err != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "event: %s", cudaGetErrorString(err));
                return HELM_OK;
            }
            const double beta = h->est_host[m + 4];
            r.rel = beta / r.fn;
            if (!std::isfinite(beta)) { r.status = HELM_ERR_NONFINITE; return fgmres_finish(r); }
            if (r.rel <= r.tol) { r.status = HELM_OK; return fgmres_finish(r); }
            if (r.it >= r.maxit) { r.status = HELM_ERR_NOCONV; return fgmres_finish(r); }
            r.restarts++;
            // v_0 = r0 / beta (as a float-pair vector for the double-FP32 Arnoldi)
            if (h->mg.gs_arith != HELM_GS_FP64) CKR(launch_split_scale(np, h->V, h->scal, s));
            else CKR(launch_scale_inv(np, h->V, h->scal, h->V, s));
            // g = beta e_1; the cycle's stop flag cleared and the tolerance it is tested against set
            CKR(launch_cycle_start(h->g, m + 1, h->scal, stop_flag(h), h->tol_dev, r.tol, s));
            r.jmax = std::min(m, r.maxit - r.it);
            r.next = 0;
            // One step of look-ahead: step j+1 is queued before the host waits for step j's
            // estimate, so the GPU never idles on the host.  If step j converges, step j+1 has
            // only written column j+1, v_{j+2}, z_{j+1} and g[j+1..j+2], none of which the back
            // substitution over the first j+1 columns reads.
            // Delayed CGS2: est[k] comes from the unit after step k (step k + 1, or the closing
            // step); units 0, 1 and 2 are queued behind step 0, and est[j] queues unit j + 3, so
            // the host has two steps' time to answer (a step queued ahead of the converged step
            // j writes no column, slot, rotation or g entry at or below j).
            if (use_dcgs2(h)) {
                CKR(run_step(h, 0, m));
                for (int k = 0; k < 3 && k < r.jmax; k++) CKR(run_unit(h, k, r.jmax, m));
            } else {
                CKR(run_step(h, 0, m));
                if (r.jmax > 1) CKR(run_step(h, 1, m));
            }
            r.phase = FgmresRun::IN_CYCLE;
            break;
        }
        case FgmresRun::IN_CYCLE: {
            const int j = r.next;
            const cudaEvent_t ev = use_dcgs2(h) ? unit_event(h, j, r.jmax) : h->step_ev[j];
            if (!event_ready(ev, block, &err)) {
                if (err != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "event: %s", cudaGetErrorString(err));
                return HELM_OK;
            }
            r.est = h->est_host[j];
            r.it++;
            if (r.st && r.st->history && r.it - 1 < r.st->history_len) r.st->history[r.it - 1] = r.est;
            if (!std::isfinite(r.est)) { r.status = HELM_ERR_NONFINITE; return fgmres_finish(r); }
            const int jdone = j + 1;
            if (r.est > r.tol && jdone < r.jmax) {
                r.next = jdone;
                if (use_dcgs2(h)) {
                    if (jdone + 2 < r.jmax) CKR(run_unit(h, jdone + 2, r.jmax, m));
                } else if (jdone + 1 < r.jmax) {
                    CKR(run_step(h, jdone + 1, m));
                }
                break;
            }
            // x += Z y with y = H^{-1} g over the first jdone columns
            {
                ProfScope ps(h, HELM_K_SMALL, 0, 0);
                CKR(launch_backsolve(h->H, ldh, jdone, h->g, h->y, s));
            }
            {
                const size_t zsz = h->z_prec == HELM_C64 ? sizeof(float2) : sizeof(double2);
                ProfScope ps(h, HELM_K_VECTOR, np * (32.0 + zsz * jdone), np * 8.0 * jdone);
                if (h->z_prec == HELM_C64)
                    CKR(launch_combine<float2>(np, (const float2 *)h->Z, np, jdone, h->y,
                                               dcgs2_fold(h) ? h->alpha2 : nullptr, r.x, s));
                else
                    CKR(launch_combine<double2>(np, (const double2 *)h->Z, np, jdone, h->y, nullptr, r.x, s));
            }
            r.phase = FgmresRun::START;
            break;
        }
        }
    }
}

static helm_status fgmres(helm_handle *h, const double2 *f, double2 *x, double tol, int m, int maxit,
                          helm_stats *st) {
    FgmresRun r;
    helm_status s0 = fgmres_begin(h, r, f, x, tol, m, maxit, st);
    if (s0 != HELM_OK) return s0;
    while (r.phase != FgmresRun::DONE)
        if ((s0 = fgmres_advance(r, true)) != HELM_OK) return s0;
    if (r.status == HELM_ERR_NONFINITE) return helm_fail(r.status, "non-finite residual in FGMRES");
    if (r.status == HELM_ERR_NOCONV)
        return helm_fail(r.status, "FGMRES: %d iterations, rel. residual %.3e > %.3e", r.it, r.rel, tol);
    return r.status;
}

static helm_status bicgstab(helm_handle *h, const double2 *f, double2 *x, double tol, int maxit, helm_stats *st) {
    helm_status s0 = ensure_bicg(h);
    if (s0 != HELM_OK) return s0;
    const size_t np = h->np;
    cudaStream_t s = h->stream;
    double2 *sc = h->scal;  // 0 rho 1 rho_old 2 alpha 3 omega 4 beta 5 rv 6 ts 7 tt 8 -alpha 9 -omega 10 one 11 flags
    double2 *nrm = h->scal + 16;
    double2 hv[2];
    helm_status rs;
    CKR(dev_norm(h, f, nrm));
    if ((rs = read_scalars(h, nrm, sizeof(double2), hv)) != HELM_OK) return rs;
    const double fn = hv[0].x;
    if (!std::isfinite(fn)) return helm_fail(HELM_ERR_NONFINITE, "||rhs|| is not finite");
    if (fn == 0.0) {
        CKR(cudaMemsetAsync(x, 0, np * sizeof(double2), s));
        CKR(cudaStreamSynchronize(s));
        if (st) { st->iterations = 0; st->restarts = 0; st->rel_res = 0; st->est_res = 0; st->status = HELM_OK; }
        return HELM_OK;
    }
    CKR(launch_residual<double, double2>(h->A64, h->dim, f, x, h->br, s));
    CKR(cudaMemcpyAsync(h->brh, h->br, np * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    CKR(cudaMemsetAsync(h->bp, 0, np * sizeof(double2), s));
    CKR(cudaMemsetAsync(h->bv, 0, np * sizeof(double2), s));
    CKR(launch_bicg_scalars(3, sc, s));
    CKR(dev_norm(h, h->br, nrm));
    if ((rs = read_scalars(h, nrm, sizeof(double2), hv)) != HELM_OK) return rs;
    double est = hv[0].x / fn;
    int it = 0;
    helm_status status = est <= tol ? HELM_OK : HELM_ERR_NOCONV;
    const bool c64 = h->z_prec == HELM_C64;
    while (status == HELM_ERR_NOCONV && it < maxit) {
        CKR(dev_dot(h, h->brh, h->br, sc + 0));                                   // rho
        CKR(launch_bicg_scalars(0, sc, s));                                       // beta
        CKR(launch_bicg_p(np, h->br, h->bv, sc, h->bp, s));                       // p
        CKR(precond_apply(h, h->bp, h->by, h->bv));                               // y = M p, v = A y
        CKR(dev_dot(h, h->brh, h->bv, sc + 5));                                   // <rh, v>
        CKR(launch_bicg_scalars(1, sc, s));                                       // alpha
        CKR(cudaMemcpyAsync(h->bs, h->br, np * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        CKR(launch_axpby(np, sc + 8, h->bv, sc + 10, h->bs, s));                  // s = r - alpha v
        CKR(dev_norm(h, h->bs, nrm));
        double2 hs[12];
        CKR(cudaMemcpyAsync(h->est_host, nrm, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CKR(cudaMemcpyAsync(h->est_host + 2, sc + 11, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CKR(cudaStreamSynchronize(s));
        memcpy(hs, h->est_host, 2 * sizeof(double2));
        it++;
        if (hs[1].x != 0.0) { status = HELM_ERR_BREAKDOWN; break; }
        est = hs[0].x / fn;
        if (!std::isfinite(est)) { status = HELM_ERR_NONFINITE; break; }
        if (est <= tol) {                                                         // x += alpha y
            if (c64) CKR(launch_axpy_mixed<float2>(np, sc + 2, (const float2 *)h->by, x, s));
            else CKR(launch_axpy_mixed<double2>(np, sc + 2, (const double2 *)h->by, x, s));
            status = HELM_OK;
            if (st && st->history && it - 1 < st->history_len) st->history[it - 1] = est;
            break;
        }
        CKR(precond_apply(h, h->bs, h->bz, h->bt));                               // z = M s, t = A z
        CKR(dev_dot(h, h->bt, h->bs, sc + 6));                                    // <t, s>
        CKR(dev_dot(h, h->bt, h->bt, sc + 7));                                    // <t, t>
        CKR(launch_bicg_scalars(2, sc, s));                                       // omega
        if (c64) {
            CKR(launch_axpy_mixed<float2>(np, sc + 2, (const float2 *)h->by, x, s));
            CKR(launch_axpy_mixed<float2>(np, sc + 3, (const float2 *)h->bz, x, s));
        } else {
            CKR(launch_axpy_mixed<double2>(np, sc + 2, (const double2 *)h->by, x, s));
            CKR(launch_axpy_mixed<double2>(np, sc + 3, (const double2 *)h->bz, x, s));
        }
        CKR(cudaMemcpyAsync(h->br, h->bs, np * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        CKR(launch_axpby(np, sc + 9, h->bt, sc + 10, h->br, s));                  // r = s - omega t
        CKR(dev_norm(h, h->br, nrm));
        CKR(cudaMemcpyAsync(h->est_host, nrm, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CKR(cudaMemcpyAsync(h->est_host + 2, sc + 11, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CKR(cudaStreamSynchronize(s));
        memcpy(hs, h->est_host, 2 * sizeof(double2));
        est = hs[0].x / fn;
        if (st && st->history && it - 1 < st->history_len) st->history[it - 1] = est;
        if (!std::isfinite(est)) { status = HELM_ERR_NONFINITE; break; }
        if (est <= tol) { status = HELM_OK; break; }
        if (hs[1].x != 0.0) { status = HELM_ERR_BREAKDOWN; break; }
    }
    // true residual
    CKR(launch_residual<double, double2>(h->A64, h->dim, f, x, h->br, s));
    CKR(dev_norm(h, h->br, nrm));
    if ((rs = read_scalars(h, nrm, sizeof(double2), hv)) != HELM_OK) return rs;
    const double rel = hv[0].x / fn;
    if (status == HELM_OK && !(rel <= tol * 10.0)) status = HELM_ERR_NOCONV;
    if (st) {
        st->iterations = it;
        st->restarts = 0;
        st->rel_res = rel;
        st->est_res = est;
        st->status = status;
    }
    if (status == HELM_ERR_BREAKDOWN) return helm_fail(status, "Bi-CGSTAB breakdown at iteration %d", it);
    if (status == HELM_ERR_NONFINITE) return helm_fail(status, "non-finite residual in Bi-CGSTAB");
    if (status == HELM_ERR_NOCONV) return helm_fail(status, "Bi-CGSTAB: %d iterations, rel. residual %.3e > %.3e", it, rel, tol);
    return status;
}

static helm_status check_vec(const void *p, const char *name) {
    if (!p) return helm_fail(HELM_ERR_ARG, "%s is null", name);
    if ((uintptr_t)p % 16) return helm_fail(HELM_ERR_ARG, "%s is not 16-byte aligned", name);
    return HELM_OK;
}

extern "C" helm_status krylov_solve(helm_handle *h, helm_krylov method, const void *rhs, void *x, double tol,
                                    int restart, int maxit, helm_stats *stats) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    helm_status st;
    if ((st = check_vec(rhs, "rhs")) != HELM_OK || (st = check_vec(x, "x")) != HELM_OK) return st;
    if (rhs == x) return helm_fail(HELM_ERR_ARG, "rhs and x must not overlap");
    if (!(tol > 0.0) || !std::isfinite(tol)) return helm_fail(HELM_ERR_ARG, "tol must be positive");
    if (maxit < 1) return helm_fail(HELM_ERR_ARG, "maxit must be >= 1");
    auto t0 = std::chrono::steady_clock::now();
    if (method == HELM_FGMRES) {
        if (restart < 1 || restart > 64) return helm_fail(HELM_ERR_ARG, "restart must be in 1..64");
        st = fgmres(h, (const double2 *)rhs, (double2 *)x, tol, restart, maxit, stats);
    } else if (method == HELM_BICGSTAB) {
        st = bicgstab(h, (const double2 *)rhs, (double2 *)x, tol, maxit, stats);
    } else {
        return helm_fail(HELM_ERR_ARG, "unknown Krylov method");
    }
    if (stats) {
        stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats->status = st;
    }
    return st;
}

// y = A^{-1} W^{-1} r into h->adj_y, r = rhs or conj(rhs): with A^T = W A W^{-1} (the ECS FD
// matrix is complex symmetric after weighting by the dual volumes W), lambda = W y solves
// A^T lambda = r with the forward operator and its preconditioner.
static helm_status adjoint_solve_y(helm_handle *h, const void *rhs, int conj_rhs, double tol, int restart, int maxit,
                                   helm_stats *stats) {
    if (!h->adj_rhs) {
        // allocated outside the Krylov workspace so that a workspace regrow keeps them valid
        CKR(cudaMalloc((void **)&h->adj_rhs, h->np * sizeof(double2)));
        h->owned.push_back(h->adj_rhs);
        CKR(cudaMalloc((void **)&h->adj_y, h->np * sizeof(double2)));
        h->owned.push_back(h->adj_y);
        CKR(cudaMemsetAsync(h->adj_rhs, 0, h->np * sizeof(double2), h->stream));
    }
    const double2 *w[3] = {h->wts[0], h->wts[1], h->wts[2]};
    CKR(launch_weight(h->np, h->n, h->dim, w, 1, (const double2 *)rhs, h->adj_rhs, h->stream, conj_rhs));
    CKR(cudaMemsetAsync(h->adj_y, 0, h->np * sizeof(double2), h->stream));
    return krylov_solve(h, HELM_FGMRES, h->adj_rhs, h->adj_y, tol, restart, maxit, stats);
}

extern "C" helm_status helm_solve_adjoint(helm_handle *h, const void *rhs, void *lambda, double tol, int restart,
                                          int maxit, helm_stats *stats) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    helm_status st;
    if ((st = check_vec(rhs, "rhs")) != HELM_OK || (st = check_vec(lambda, "lambda")) != HELM_OK) return st;
    if (rhs == lambda) return helm_fail(HELM_ERR_ARG, "rhs and lambda must not overlap");
    st = adjoint_solve_y(h, rhs, 0, tol, restart, maxit, stats);
    if (st != HELM_OK && st != HELM_ERR_NOCONV) return st;
    const double2 *w[3] = {h->wts[0], h->wts[1], h->wts[2]};
    CKR(cudaMemsetAsync(lambda, 0, h->np * sizeof(double2), h->stream));
    CKR(launch_weight(h->np, h->n, h->dim, w, 0, h->adj_y, (double2 *)lambda, h->stream));
    return st;
}

extern "C" helm_status helm_backward(helm_handle *h, const void *grad_u, const void *u, double *grad_k2,
                                     void *grad_f, double tol, int restart, int maxit, helm_stats *stats) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    helm_status st;
    if ((st = check_vec(grad_u, "grad_u")) != HELM_OK) return st;
    if (!grad_k2 && !grad_f) return helm_fail(HELM_ERR_ARG, "grad_k2 and grad_f are both null");
    if (grad_k2) {
        if ((st = check_vec(u, "u")) != HELM_OK) return st;
        if ((uintptr_t)grad_k2 % 8) return helm_fail(HELM_ERR_ARG, "grad_k2 is not 8-byte aligned");
    }
    if (grad_f && (st = check_vec(grad_f, "grad_f")) != HELM_OK) return st;
    const void *outs[2] = {grad_k2, grad_f};
    for (const void *o : outs)
        if (o && (o == grad_u || o == u)) return helm_fail(HELM_ERR_ARG, "outputs must not overlap grad_u or u");
    // A^T lambda = conj(grad_u)
    st = adjoint_solve_y(h, grad_u, 1, tol, restart, maxit, stats);
    if (st != HELM_OK && st != HELM_ERR_NOCONV) return st;
    const double2 *w[3] = {h->wts[0], h->wts[1], h->wts[2]};
    CKR(launch_adjoint_grads(h->np, h->n, h->dim, w, h->adj_y, (const double2 *)u, grad_k2, (double2 *)grad_f,
                             h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    return st;
}

extern "C" helm_status helm_mg_conv(helm_handle *h, const void *b, void *x, helm_prec prec, double tol, int maxcyc,
                                    int *ncycles, double *factor) {
    if (!h || !ncycles || !factor) return helm_fail(HELM_ERR_ARG, "null argument");
    if (h->mg.kind == HELM_PC_NONE) return helm_fail(HELM_ERR_ARG, "handle has no preconditioner hierarchy");
    if (maxcyc < 1 || !(tol > 0)) return helm_fail(HELM_ERR_ARG, "bad tol/maxcyc");
    helm_status st = ensure_ws(h, 1);
    if (st != HELM_OK) return st;
    const size_t np = h->np;
    cudaStream_t s = h->stream;
    const size_t esz = prec == HELM_C128 ? sizeof(double2) : sizeof(float2);
    CKR(cudaMemsetAsync(x, 0, np * esz, s));
    double2 *r = h->V + np, *b64 = h->V;  // V has >= 2 vectors
    if (prec == HELM_C64) CKR(launch_convert(np, (const float2 *)b, b64, s));
    else CKR(cudaMemcpyAsync(b64, b, np * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    double2 hv[2];
    CKR(dev_norm(h, b64, h->scal));
    if ((st = read_scalars(h, h->scal, sizeof(double2), hv)) != HELM_OK) return st;
    const double bn = hv[0].x;
    std::vector<double> res(1, bn);
    int c = 0;
    while (c < maxcyc) {
        if ((st = mg_vcycle(h, b, x, prec)) != HELM_OK) return st;
        c++;
        if (prec == HELM_C64) {
            float2 *r32 = h->lv[0].t32;
            CKR(launch_residual<float, float2>(h->lv[0].M32, h->dim, (const float2 *)b, (const float2 *)x, r32, s));
            CKR(launch_convert(np, (const float2 *)r32, r, s));
        } else {
            CKR(launch_residual<double, double2>(h->lv[0].M64, h->dim, (const double2 *)b, (const double2 *)x, r, s));
        }
        CKR(dev_norm(h, r, h->scal));
        if ((st = read_scalars(h, h->scal, sizeof(double2), hv)) != HELM_OK) return st;
        res.push_back(hv[0].x);
        if (!std::isfinite(hv[0].x)) return helm_fail(HELM_ERR_NONFINITE, "multigrid diverged to non-finite values");
        if (hv[0].x <= tol * bn) break;
    }
    const int k = std::min(c, 5);
    *ncycles = c;
    *factor = k > 0 && res[c - k] > 0 ? pow(res[c] / res[c - k], 1.0 / k) : 0.0;
    return HELM_OK;
}
