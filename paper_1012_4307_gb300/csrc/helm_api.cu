// C-ABI entry points of libhelm.so and the host-side drivers: grid/level setup (ECS contour of
// Section 3.1, FD coefficients of Section 3.2, operators of Section 5, rediscretised levels of
// Section 4.2), the multigrid recursion of Algorithm 1, and the flexible GMRES / Bi-CGSTAB
// loops whose vector work runs in the kernels of kernels_mg.cu and kernels_krylov.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <string>
#include <vector>

#include "helm_internal.h"
#include "helm_handle.h"

typedef std::complex<double> cd;

// ------------------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
thread_local bool g_pdl_off = false;
thread_local bool g_pdl_cycle = false;

helm_status helm_fail(helm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

extern "C" const char *helm_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *helm_version(void) { return "helm-gb300 1.0 (sm_103a)"; }

#define CKR(...)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (__VA_ARGS__);                                                               \
        if (e_ != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)
#define CKE(...)                            \
    do {                                    \
        cudaError_t e_ = (__VA_ARGS__);            \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

// ------------------------------------------------------------------------------ host setup
// Linear ECS contour of one axis (Section 3.1): z = x on [r0lo, r0hi], z = r0 + (x - r0)e^{i theta}
// beyond either end (a side whose r0 is outside [lo, hi] has no layer).
std::vector<cd> ecs_contour(int n, double lo, double hi, double theta, double r0lo, double r0hi) {
    std::vector<cd> z(n);
    const double h = (hi - lo) / (double)(n - 1);
    const cd rot = std::polar(1.0, theta);
    for (int j = 0; j < n; j++) {
        const double x = (j == n - 1) ? hi : lo + h * (double)j;
        if (x > r0hi) z[j] = r0hi + (x - r0hi) * rot;
        else if (x < r0lo) z[j] = r0lo + (x - r0lo) * rot;
        else z[j] = x;
    }
    return z;
}

// Per-node coefficient triples of a * (-d^2/dz^2) with all widths multiplied by e^{i ts}
// (Section 3.2 formula for unequal widths): cw = -2/((hm+hp) hm), ce = -2/((hm+hp) hp),
// cc = -(cw + ce).  Boundary entries are zero.
std::vector<cd> fd_triples(const std::vector<cd> &z, double ts, cd a) {
    const int n = (int)z.size();
    std::vector<cd> t(3 * (size_t)n, cd(0, 0));
    const cd rot = std::polar(1.0, ts);
    for (int j = 1; j < n - 1; j++) {
        const cd hm = (z[j] - z[j - 1]) * rot, hp = (z[j + 1] - z[j]) * rot;
        const cd cw = -2.0 / ((hm + hp) * hm), ce = -2.0 / ((hm + hp) * hp);
        t[3 * j] = a * cw;
        t[3 * j + 1] = -a * (cw + ce);
        t[3 * j + 2] = a * ce;
    }
    return t;
}

// Operator coefficients (a, bk, c, ts) of Section 5 for the preconditioner kind.
static void pc_coefficients(const helm_mg_params &p, cd &a, cd &bk, cd &c, double &ts) {
    a = 1.0; bk = -1.0; c = 0.0; ts = 0.0;
    switch (p.kind) {
    case HELM_PC_CSG: ts = p.theta_a; break;                           // M = Z on rotated widths
    case HELM_PC_CSL: bk = cd(p.beta1, p.beta2); break;                 // -Delta + (b1 + i b2) k^2
    case HELM_PC_QD: a = 1.0 / fabs(p.re_lambda0); bk = -a; c = cd(1.0, -1.0); break;  // (1-i) + Z/|l0|
    case HELM_PC_LAPLACE: bk = 0.0; break;                              // -Delta
    default: break;
    }
}

// Dense operator on the unknowns of a small grid and its inverse (Gauss-Jordan with partial
// pivoting, FP64).  Returns false if singular.
static bool dense_inverse(int dim, const int n[3], const std::vector<cd> *tri, const std::vector<double> &k2, cd bk,
                          cd c, std::vector<cd> &inv) {
    const int mx = n[0] - 2, my = n[1] - 2, mz = dim == 3 ? n[2] - 2 : 1;
    const int nu = mx * my * mz;
    std::vector<cd> A((size_t)nu * nu, cd(0, 0)), B((size_t)nu * nu, cd(0, 0));
    auto unk = [&](int i, int j, int k) { return (i - 1) + mx * ((j - 1) + my * (dim == 3 ? k - 1 : 0)); };
    for (int k = (dim == 3 ? 1 : 0); k < (dim == 3 ? n[2] - 1 : 1); k++)
        for (int j = 1; j < n[1] - 1; j++)
            for (int i = 1; i < n[0] - 1; i++) {
                const int r = unk(i, j, k);
                const size_t p = (size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * k);
                const int idx[3] = {i, j, k};
                cd d = bk * k2[p] + c;
                for (int ax = 0; ax < dim; ax++) {
                    const cd *t = &tri[ax][3 * (size_t)idx[ax]];
                    d += t[1];
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    lo[ax]--;
                    hi[ax]++;
                    if (lo[ax] >= 1) A[(size_t)r * nu + unk(lo[0], lo[1], lo[2])] += t[0];
                    if (hi[ax] <= n[ax] - 2) A[(size_t)r * nu + unk(hi[0], hi[1], hi[2])] += t[2];
                }
                A[(size_t)r * nu + r] += d;
            }
    for (int r = 0; r < nu; r++) B[(size_t)r * nu + r] = 1.0;
    for (int col = 0; col < nu; col++) {
        int piv = col;
        double best = std::abs(A[(size_t)col * nu + col]);
        for (int r = col + 1; r < nu; r++)
            if (std::abs(A[(size_t)r * nu + col]) > best) { best = std::abs(A[(size_t)r * nu + col]); piv = r; }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        if (piv != col)
            for (int c2 = 0; c2 < nu; c2++) {
                std::swap(A[(size_t)col * nu + c2], A[(size_t)piv * nu + c2]);
                std::swap(B[(size_t)col * nu + c2], B[(size_t)piv * nu + c2]);
            }
        const cd inv_p = 1.0 / A[(size_t)col * nu + col];
        for (int c2 = 0; c2 < nu; c2++) { A[(size_t)col * nu + c2] *= inv_p; B[(size_t)col * nu + c2] *= inv_p; }
        for (int r = 0; r < nu; r++) {
            if (r == col) continue;
            const cd f = A[(size_t)r * nu + col];
            if (f == cd(0, 0)) continue;
            for (int c2 = 0; c2 < nu; c2++) {
                A[(size_t)r * nu + c2] -= f * A[(size_t)col * nu + c2];
                B[(size_t)r * nu + c2] -= f * B[(size_t)col * nu + c2];
            }
        }
    }
    inv.swap(B);
    return true;
}

// ------------------------------------------------------------------------------ device alloc
template <typename T> static cudaError_t dalloc(T **p, size_t count, std::vector<void *> &owned) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
}

template <typename C> static cudaError_t upload_c(C **dst, const std::vector<cd> &src, std::vector<void *> &owned,
                                                  cudaStream_t s) {
    typedef decltype((*dst)->x) R;
    std::vector<C> tmp(src.size());
    for (size_t q = 0; q < src.size(); q++) tmp[q] = mk((R)src[q].real(), (R)src[q].imag());
    CKE(dalloc(dst, src.size(), owned));
    CKE(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(C), cudaMemcpyHostToDevice, s));
    return cudaStreamSynchronize(s);
}

template <typename R> static cudaError_t upload_r(R **dst, const std::vector<double> &src, std::vector<void *> &owned,
                                                  cudaStream_t s) {
    std::vector<R> tmp(src.begin(), src.end());
    CKE(dalloc(dst, src.size(), owned));
    CKE(cudaMemcpyAsync(*dst, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice, s));
    return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------------------ create
static bool coarsen_further(int dim, const int n[3], int coarsest_n) {
    bool small = true;
    for (int a = 0; a < dim; a++) {
        if (n[a] > coarsest_n) small = false;
        if ((n[a] - 1) % 2 != 0 || (n[a] + 1) / 2 < 3) return false;
    }
    return !small;
}

helm_status helm_validate_create(const helm_grid *grid, const double *r0_lo, const double *r0_hi, const double *k2,
                                 const helm_mg_params *mg) {
    if (!grid || !r0_lo || !r0_hi || !k2 || !mg) return helm_fail(HELM_ERR_ARG, "null argument");
    if (grid->dim != 2 && grid->dim != 3) return helm_fail(HELM_ERR_ARG, "dim must be 2 or 3 (got %d)", grid->dim);
    for (int a = 0; a < grid->dim; a++) {
        if (grid->n[a] < 3 || grid->n[a] > (1 << 16)) return helm_fail(HELM_ERR_ARG, "n[%d] = %d out of range", a, grid->n[a]);
        if (!(grid->hi[a] > grid->lo[a])) return helm_fail(HELM_ERR_ARG, "hi[%d] must exceed lo[%d]", a, a);
    }
    if (mg->kind < HELM_PC_NONE || mg->kind > HELM_PC_LAPLACE) return helm_fail(HELM_ERR_ARG, "unknown preconditioner");
    if (mg->kind == HELM_PC_QD && !(fabs(mg->re_lambda0) > 0.0)) return helm_fail(HELM_ERR_ARG, "QD needs re_lambda0 != 0");
    if (mg->nu1 < 0 || mg->nu2 < 0 || mg->nu1 > 64 || mg->nu2 > 64) return helm_fail(HELM_ERR_ARG, "nu1/nu2 out of range");
    if (mg->gamma_f < 1 || mg->gamma_c < 1 || mg->gamma_f > 4 || mg->gamma_c > 4)
        return helm_fail(HELM_ERR_ARG, "gamma_f/gamma_c must be in 1..4");
    if (!(mg->omega > 0.0 && mg->omega < 2.0)) return helm_fail(HELM_ERR_ARG, "omega must be in (0, 2)");
    if (mg->prec != HELM_C128 && mg->prec != HELM_C64) return helm_fail(HELM_ERR_ARG, "bad precision");
    if (mg->smoother != HELM_SMOOTH_JACOBI && mg->smoother != HELM_SMOOTH_RB) return helm_fail(HELM_ERR_ARG, "bad smoother");
    if (mg->coarsest_n < 3) return helm_fail(HELM_ERR_ARG, "coarsest_n must be >= 3");
    if (mg->gs_arith != HELM_GS_FP64 && mg->gs_arith != HELM_GS_DF && mg->gs_arith != HELM_GS_DCGS2)
        return helm_fail(HELM_ERR_ARG, "bad gs_arith");
    return HELM_OK;
}

helm_status helm_create_impl(const helm_grid *grid, double theta, const double *r0_lo, const double *r0_hi,
                             const std::vector<double> &k2h, const helm_mg_params *mg, cudaStream_t s,
                             helm_handle **out) {
    helm_handle *h = new (std::nothrow) helm_handle();
    if (!h) return helm_fail(HELM_ERR_NOMEM, "host allocation failed");
    h->dim = grid->dim;
    h->mg = *mg;
    h->stream = s;
    for (int a = 0; a < 3; a++) h->n[a] = a < grid->dim ? grid->n[a] : 1;
    h->np = (size_t)h->n[0] * h->n[1] * h->n[2];
    const int dim = h->dim;
    std::vector<std::vector<cd>> z(dim);
    for (int a = 0; a < dim; a++) z[a] = ecs_contour(grid->n[a], grid->lo[a], grid->hi[a], theta, r0_lo[a], r0_hi[a]);

    auto cleanup_fail = [&](helm_status st) { helm_destroy(h); return st; };
#define CKC(...)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                                                            \
        if (e_ != cudaSuccess) {                                                                            \
            helm_fail(e_ == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__,   \
                      cudaGetErrorString(e_));                                                              \
            return cleanup_fail(e_ == cudaErrorMemoryAllocation ? HELM_ERR_NOMEM : HELM_ERR_CUDA);         \
        }                                                                                                   \
    } while (0)

    // A = Z = L_h - k^2 on the fine grid (FP64), and dual-volume weights per axis
    for (int a = 0; a < 3; a++) {
        std::vector<cd> tri = a < dim ? fd_triples(z[a], 0.0, 1.0) : std::vector<cd>(3, cd(0, 0));
        CKC(upload_c(&h->coefA64[a], tri, h->owned, s));
        h->A64.coef[a] = h->coefA64[a];
        std::vector<cd> w(a < dim ? z[a].size() : 1, cd(1, 0));
        if (a < dim)
            for (size_t j = 1; j + 1 < z[a].size(); j++) w[j] = 0.5 * ((z[a][j] - z[a][j - 1]) + (z[a][j + 1] - z[a][j]));
        CKC(upload_c(&h->wts[a], w, h->owned, s));
    }
    for (int a = 0; a < 3; a++) h->A64.n[a] = h->n[a];
    // the same A with every FP64 coefficient stored as a float pair hi + lo (hi = nearest
    // float, lo = nearest float to the remainder) for the double-FP32 apply
    {
        auto fsplit = [](double v, float &hi, float &lo) {
            hi = (float)v;
            lo = (float)(v - (double)hi);
        };
        for (int a = 0; a < 3; a++) {
            std::vector<cd> tri = a < dim ? fd_triples(z[a], 0.0, 1.0) : std::vector<cd>(3, cd(0, 0));
            std::vector<float4> t4(tri.size());
            for (size_t q = 0; q < tri.size(); q++) {
                float rh, rl, ih, il;
                fsplit(tri[q].real(), rh, rl);
                fsplit(tri[q].imag(), ih, il);
                t4[q] = make_float4(rh, rl, ih, il);
            }
            float4 *d = nullptr;
            CKC(dalloc(&d, t4.size(), h->owned));
            CKC(cudaMemcpyAsync(d, t4.data(), t4.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
            CKC(cudaStreamSynchronize(s));
            h->Adf.coef[a] = d;
            h->Adf.n[a] = h->n[a];
        }
        std::vector<float2> k2s(k2h.size());
        for (size_t q = 0; q < k2h.size(); q++) fsplit(k2h[q], k2s[q].x, k2s[q].y);
        float2 *d = nullptr;
        CKC(dalloc(&d, k2s.size(), h->owned));
        CKC(cudaMemcpyAsync(d, k2s.data(), k2s.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
        CKC(cudaStreamSynchronize(s));
        h->Adf.k2 = d;
    }
    CKC(upload_r(&h->k2A, k2h, h->owned, s));
    h->A64.k2 = h->k2A;
    h->A64.bk = make_double2(-1.0, 0.0);
    h->A64.c = make_double2(0.0, 0.0);

    // preconditioner hierarchy (rediscretisation; k^2 injected; nodes z_c[I] = z_f[2I])
    cd a_s, bk_s, c_s;
    double ts;
    pc_coefficients(*mg, a_s, bk_s, c_s, ts);
    std::vector<std::vector<cd>> zl = z;
    std::vector<double> k2l = k2h;
    int nl[3] = {h->n[0], h->n[1], h->n[2]};
    for (int l = 0;; l++) {
        LevelDev L;
        for (int a = 0; a < 3; a++) L.n[a] = nl[a];
        L.np = (size_t)nl[0] * nl[1] * nl[2];
        std::vector<cd> tri[3];
        for (int a = 0; a < 3; a++) {
            tri[a] = a < dim ? fd_triples(zl[a], ts, a_s) : std::vector<cd>(3, cd(0, 0));
            CKC(upload_c(&L.coef64[a], tri[a], h->owned, s));
            CKC(upload_c(&L.coef32[a], tri[a], h->owned, s));
            L.M64.coef[a] = L.coef64[a];
            L.M32.coef[a] = L.coef32[a];
            L.M64.n[a] = L.M32.n[a] = nl[a];
        }
        CKC(upload_r(&L.k2_64, k2l, h->owned, s));
        CKC(upload_r(&L.k2_32, k2l, h->owned, s));
        L.M64.k2 = L.k2_64;
        L.M32.k2 = L.k2_32;
        L.M64.bk = make_double2(bk_s.real(), bk_s.imag());
        L.M64.c = make_double2(c_s.real(), c_s.imag());
        L.M32.bk = make_float2((float)bk_s.real(), (float)bk_s.imag());
        L.M32.c = make_float2((float)c_s.real(), (float)c_s.imag());
        if (dim == 2) {  // 1 / diagonal for the temporally blocked smoothers
            float2 *di = nullptr;
            CKC(dalloc(&di, L.np, h->owned));
            CKC(launch_diag_inv(L.M32, di, s));
            L.M32.dinv = di;
        }
        CKC(dalloc(&L.b64, L.np, h->owned)); CKC(dalloc(&L.u64, L.np, h->owned));
        CKC(dalloc(&L.t64, L.np, h->owned)); CKC(dalloc(&L.b32, L.np, h->owned));
        CKC(dalloc(&L.u32, L.np, h->owned)); CKC(dalloc(&L.t32, L.np, h->owned));
        CKC(cudaMemsetAsync(L.b64, 0, L.np * sizeof(double2), s)); CKC(cudaMemsetAsync(L.u64, 0, L.np * sizeof(double2), s));
        CKC(cudaMemsetAsync(L.t64, 0, L.np * sizeof(double2), s)); CKC(cudaMemsetAsync(L.b32, 0, L.np * sizeof(float2), s));
        CKC(cudaMemsetAsync(L.u32, 0, L.np * sizeof(float2), s)); CKC(cudaMemsetAsync(L.t32, 0, L.np * sizeof(float2), s));
        if (mg->kind == HELM_PC_NONE) {  // no hierarchy: level 0 only, no coarsest inverse
            h->lv.push_back(L);
            break;
        }
        const bool more = l + 1 < 20 && coarsen_further(dim, nl, mg->coarsest_n);
        if (!more) {
            // coarsest level: exact solve through a dense inverse (Algorithm 1 step (0))
            const size_t nu = (size_t)(nl[0] - 2) * (nl[1] - 2) * (dim == 3 ? nl[2] - 2 : 1);
            if (nu > 4096) {
                helm_fail(HELM_ERR_ARG, "coarsest grid has %zu unknowns (> 4096) for the dense exact solve; "
                          "use odd 2^k+1 sizes or a smaller coarsest_n", nu);
                h->lv.push_back(L);
                return cleanup_fail(HELM_ERR_ARG);
            }
            std::vector<cd> inv;
            if (!dense_inverse(dim, nl, tri, k2l, bk_s, c_s, inv)) {
                helm_fail(HELM_ERR_ARG, "coarsest operator (%d nodes per axis) is singular", nl[0]);
                h->lv.push_back(L);
                return cleanup_fail(HELM_ERR_ARG);
            }
            h->nu_c = (int)llround(sqrt((double)inv.size()));
            CKC(upload_c(&h->minv64, inv, h->owned, s));
            CKC(upload_c(&h->minv32, inv, h->owned, s));
            h->lv.push_back(L);
            break;
        }
        h->lv.push_back(L);
        int nc[3] = {1, 1, 1};
        for (int a = 0; a < dim; a++) nc[a] = (nl[a] + 1) / 2;
        std::vector<std::vector<cd>> zc(dim);
        for (int a = 0; a < dim; a++) {
            zc[a].resize(nc[a]);
            for (int j = 0; j < nc[a]; j++) zc[a][j] = zl[a][2 * j];
        }
        std::vector<double> k2c((size_t)nc[0] * nc[1] * nc[2]);
        for (int k = 0; k < nc[2]; k++)
            for (int j = 0; j < nc[1]; j++)
                for (int i = 0; i < nc[0]; i++)
                    k2c[(size_t)i + (size_t)nc[0] * ((size_t)j + (size_t)nc[1] * k)] =
                        k2l[(size_t)(2 * i) + (size_t)nl[0] * ((size_t)(2 * j) + (size_t)nl[1] * (dim == 3 ? 2 * k : 0))];
        zl.swap(zc);
        k2l.swap(k2c);
        for (int a = 0; a < 3; a++) nl[a] = nc[a];
    }
    // coarse tail: the longest run of levels ending at the coarsest with at most
    // TAIL_MAX_UNKNOWNS interior nodes each (and at most MAX_TAIL_LEVELS levels)
    if (mg->kind != HELM_PC_NONE) {
        const int nlev = (int)h->lv.size();
        for (int pass = 0; pass < 2; pass++) {
            const size_t es = pass == 0 ? sizeof(float2) : sizeof(double2);
            int top = nlev - 1;
            while (top > 0 && nlev - top < MAX_TAIL_LEVELS) {
                const LevelDev &L = h->lv[top - 1];
                const double ni = (double)(L.n[0] - 2) * (L.n[1] - 2) * (dim == 3 ? (double)(L.n[2] - 2) : 1.0);
                int n[MAX_TAIL_LEVELS][3];
                for (int l = top - 1; l < nlev; l++)
                    for (int a = 0; a < 3; a++) n[l - top + 1][a] = h->lv[l].n[a];
                if (ni > TAIL_MAX_UNKNOWNS || mg_tail_smem_bytes_nodes(dim, nlev - top + 1, n, h->nu_c, es) > TAIL_SMEM_BYTES)
                    break;
                top--;
            }
            // a lone coarsest level keeps its dense-solve kernel
            (pass == 0 ? h->tail_top32 : h->tail_top64) = nlev - top >= 2 ? top : -1;
        }
    }
    h->tune.tail_levels = -1;
    for (int l = 0; l < HELM_MAX_LEVELS; l++) h->tune.level_tile[l] = HELM_TILE_32x8;
    h->tune.cluster_levels = 0;
    h->tune.cluster_ctas = 16;
    h->tune.cluster_halo = 3;
    // how many coarsest levels a cluster tail can hold (2D only)
    if (mg->kind != HELM_PC_NONE && dim == 2) {
        const int nlev = (int)h->lv.size();
        for (int k = 0; k < 2; k++) {
            const int nc = k ? 16 : 8;
            int fit = 0;
            for (int nt = 2; nt <= std::min(nlev, MAX_CT_LEVELS); nt++) {
                int n[MAX_CT_LEVELS][3];
                for (int q = 0; q < nt; q++)
                    for (int a = 0; a < 3; a++) n[q][a] = h->lv[nlev - nt + q].n[a];
                unsigned off[MAX_CT_LEVELS][7], obc, oz;
                if (mg_ctail_layout(nt, n, nc, h->nu_c, off, &obc, &oz) <= CT_SMEM_BYTES) fit = nt;
            }
            h->ctail_fit[k] = fit;
        }
    }
    CKC(cudaStreamSynchronize(s));
    *out = h;
    return HELM_OK;
#undef CKC
}

extern "C" helm_status helm_create(const helm_grid *grid, double theta, const double *r0_lo, const double *r0_hi,
                                   const double *k2, const helm_mg_params *mg, void *stream, helm_handle **out) {
    if (!out) return helm_fail(HELM_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    helm_status st = helm_validate_create(grid, r0_lo, r0_hi, k2, mg);
    if (st != HELM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    size_t np = (size_t)grid->n[0] * grid->n[1] * (grid->dim == 3 ? grid->n[2] : 1);
    std::vector<double> k2h(np);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, k2) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return helm_fail(HELM_ERR_ARG, "k2 must be a device pointer");
    }
    CKR(cudaMemcpyAsync(k2h.data(), k2, np * sizeof(double), cudaMemcpyDeviceToHost, s));
    CKR(cudaStreamSynchronize(s));
    for (size_t q = 0; q < np; q++)
        if (!std::isfinite(k2h[q])) return helm_fail(HELM_ERR_NONFINITE, "k2 has a non-finite value at node %zu", q);
    try {
        return helm_create_impl(grid, theta, r0_lo, r0_hi, k2h, mg, s, out);
    } catch (const std::bad_alloc &) {
        return helm_fail(HELM_ERR_NOMEM, "host allocation failed during setup");
    }
}

extern "C" void helm_destroy(helm_handle *h) {
    if (!h) return;
    if (h->stream_owned_sync) cudaStreamSynchronize(h->stream);
    helm_free_krylov(h);
    for (void *p : h->owned) cudaFree(p);
    if (h->est_host) cudaFreeHost(h->est_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fn) cudaEventDestroy(h->ev_fn);
    if (h->ev_beta) cudaEventDestroy(h->ev_beta);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
}

extern "C" helm_status helm_profile(helm_handle *h, int enable) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    CKR(cudaStreamSynchronize(h->stream));
    h->prof.reset();
    h->prof.on = enable != 0;
    return HELM_OK;
}

extern "C" helm_status helm_profile_read(helm_handle *h, int ncls, int *launches, double *ms, double *bytes,
                                         double *flops, double *bytes_pass) {
    if (!h || !launches || !ms || !bytes || !flops || ncls < 1 || ncls > HELM_K_NCLASS)
        return helm_fail(HELM_ERR_ARG, "bad profile arguments");
    CKR(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < ncls; c++) {
        launches[c] = 0;
        ms[c] = bytes[c] = flops[c] = 0.0;
        if (bytes_pass) bytes_pass[c] = 0.0;
    }
    for (const ProfRec &r : h->prof.recs) {
        if (r.cls < 0 || r.cls >= ncls) continue;
        float t = 0.f;
        CKR(cudaEventElapsedTime(&t, r.a, r.b));
        launches[r.cls]++;
        ms[r.cls] += t;
        bytes[r.cls] += r.bytes;
        flops[r.cls] += r.flops;
        if (bytes_pass) bytes_pass[r.cls] += r.bytes_pass;
    }
    return HELM_OK;
}

extern "C" helm_status helm_levels(const helm_handle *h, int *nlev) {
    if (!h || !nlev) return helm_fail(HELM_ERR_ARG, "null argument");
    *nlev = (int)h->lv.size();
    return HELM_OK;
}

extern "C" helm_status helm_level_shape(const helm_handle *h, int level, int n[3]) {
    if (!h || !n || level < 0 || level >= (int)h->lv.size()) return helm_fail(HELM_ERR_ARG, "bad level");
    for (int a = 0; a < 3; a++) n[a] = h->lv[level].n[a];
    return HELM_OK;
}

// ------------------------------------------------------------------------------ Algorithm 1
template <typename R> struct LvBuf;
template <> struct LvBuf<double> {
    static double2 *b(LevelDev &L) { return L.b64; }
    static double2 *u(LevelDev &L) { return L.u64; }
    static double2 *t(LevelDev &L) { return L.t64; }
    static const DevOp<double> &op(LevelDev &L) { return L.M64; }
    static const double2 *minv(helm_handle *h) { return h->minv64; }
};
template <> struct LvBuf<float> {
    static float2 *b(LevelDev &L) { return L.b32; }
    static float2 *u(LevelDev &L) { return L.u32; }
    static float2 *t(LevelDev &L) { return L.t32; }
    static const DevOp<float> &op(LevelDev &L) { return L.M32; }
    static const float2 *minv(helm_handle *h) { return h->minv32; }
};

// Interior node count of a level.
static double interior(const LevelDev &L, int dim) {
    return (double)(L.n[0] - 2) * (L.n[1] - 2) * (dim == 3 ? (double)(L.n[2] - 2) : 1.0);
}

// smoothing steps on level l; *cur holds the iterate and may be swapped with *oth (Jacobi).
// Algorithmic bytes per sweep and unknown: read u, b, k^2, write u (3 complex + 1 real).
template <typename R>
static cudaError_t smooth(helm_handle *h, int l, int sweeps, const typename CT<R>::T *b, typename CT<R>::T **cur,
                          typename CT<R>::T **oth, bool zero) {
    LevelDev &L = h->lv[l];
    const DevOp<R> &op = LvBuf<R>::op(L);
    const R om = (R)h->mg.omega;
    const int cls = l == 0 ? HELM_K_SMOOTH_FINE : HELM_K_SMOOTH_COARSE;
    const double es = sizeof(typename CT<R>::T), rs = sizeof(R), ni = interior(L, h->dim);
    if (sweeps == 0) {
        if (zero) {
            ProfScope ps(h, HELM_K_VECTOR, L.np * es, 0);
            CKE(launch_zero(L.np, *cur, h->stream));
        }
        return cudaSuccess;
    }
    if (h->mg.smoother == HELM_SMOOTH_RB) {
        if (zero) {
            ProfScope ps(h, HELM_K_VECTOR, L.np * es, 0);
            CKE(launch_zero(L.np, *cur, h->stream));
        }
        for (int s = 0; s < sweeps; s++) {
            for (int colour = 0; colour < 2; colour++) {
                ProfScope ps(h, cls, 0.5 * ni * (3 * es + rs), 0);
                CKE(launch_rb<R>(op, h->dim, om, b, *cur, colour, h->stream));
            }
        }
        return cudaSuccess;
    }
    for (int s = 0; s < sweeps; s++) {
        const bool z0 = zero && s == 0;
        ProfScope ps(h, cls, ni * ((z0 ? 2 : 3) * es + rs), 0);
        CKE(launch_jacobi<R>(op, h->dim, om, b, z0 ? nullptr : *cur, *oth, h->stream));
        std::swap(*cur, *oth);
    }
    return cudaSuccess;
}

template <typename R>
static cudaError_t coarse_solve(helm_handle *h, LevelDev &L, const typename CT<R>::T *b, typename CT<R>::T *u) {
    const double es = sizeof(typename CT<R>::T), nu = h->nu_c;
    ProfScope ps(h, HELM_K_COARSE, nu * nu * es + 2 * nu * es, 8.0 * nu * nu);
    return launch_dense_solve<R>(L.n, h->dim, h->nu_c, LvBuf<R>::minv(h), b, u, h->stream);
}

// u <- MG(l, M_l, b, u, nu1, nu2, C, gf, gc).  'zero' means u = 0 on entry (not read).
// The result always ends in u.  Level l uses its own t buffer as the Jacobi partner; coarse
// levels use their own b (restricted residual) and u (error) buffers.
// First level of the fused tail under the handle's tuning (-1: no tail): the built (largest
// fitting) tail shortened to tune.tail_levels levels.
template <typename R> int tail_top(const helm_handle *h) {
    const int built = sizeof(R) == sizeof(float) ? h->tail_top32 : h->tail_top64;
    const int want = h->tune.tail_levels;
    if (built < 0 || want == 0) return -1;
    if (want < 0) return built;
    const int last = (int)h->lv.size() - 1;
    const int top = std::max(built, last - want + 1);
    return last - top + 1 >= 2 ? top : -1;
}
template int tail_top<float>(const helm_handle *);
template int tail_top<double>(const helm_handle *);

const void *ctail_image(helm_handle *h, bool build, bool deep) {
    const int top = ctail_top(h);
    if (top < 0) return nullptr;
    const int nc = h->tune.cluster_ctas, key = top * 32 + nc + (deep ? 1024 : 0);
    for (const auto &e : h->ctail_img)
        if (e.first == key) return e.second;
    if (!build) return nullptr;
    const int nt = (int)h->lv.size() - top;
    DevOp<float> ops[MAX_CT_LEVELS];
    for (int k = 0; k < nt; k++) ops[k] = h->lv[top + k].M32;
    void *img = nullptr;
    if ((deep ? build_mg_chalo_image(nt, ops, h->minv32, h->nu_c, nc, &img, h->stream)
              : build_mg_ctail_image(nt, ops, h->minv32, h->nu_c, nc, &img, h->stream)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    try {
        h->owned.push_back(img);
        h->ctail_img.push_back({key, img});
    } catch (...) {
        cudaFree(img);
        return nullptr;
    }
    return img;
}

bool ctail_deep(const helm_handle *h) {
    if (h->tune.cluster_halo != 3) return false;
    const int top = ctail_top(h);
    const helm_mg_params &m = h->mg;
    if (top < 0 || m.smoother != HELM_SMOOTH_JACOBI || m.gamma_f != 1 || m.gamma_c != 1 || m.nu1 > 2 || m.nu2 > 2)
        return false;
    const int nt = (int)h->lv.size() - top;
    DevOp<float> ops[MAX_CT_LEVELS];
    for (int k = 0; k < nt; k++) ops[k] = h->lv[top + k].M32;
    return mg_chalo_bytes(nt, ops, h->nu_c, h->tune.cluster_ctas) > 0;
}

int ctail_top(const helm_handle *h) {
    const int want = h->tune.cluster_levels;
    if (h->dim != 2 || want < 2 || h->mg.kind == HELM_PC_NONE) return -1;
    const int fit = h->ctail_fit[h->tune.cluster_ctas == 16 ? 1 : 0];
    const int nt = std::min(want, fit);
    if (nt < 2) return -1;
    return (int)h->lv.size() - nt;
}

template <typename R>
static cudaError_t cycle(helm_handle *h, int l, const typename CT<R>::T *b, typename CT<R>::T *u, bool zero, int gf,
                         int gc) {
    typedef typename CT<R>::T C;
    LevelDev &L = h->lv[l];
    const int last = (int)h->lv.size() - 1;
    if (l == last) return coarse_solve<R>(h, L, b, u);
    if constexpr (sizeof(R) == sizeof(float)) {
        if (l == ctail_top(h)) {
            // levels l..last in one launch of a thread-block cluster
            const int nt = last - l + 1;
            DevOp<float> ops[MAX_CT_LEVELS];
            double bytes = 0;
            for (int k = 0; k < nt; k++) {
                ops[k] = h->lv[l + k].M32;
                bytes += interior(h->lv[l + k], h->dim) * sizeof(float2) * 8.0;
            }
            ProfScope ps(h, HELM_K_COARSE, bytes + (double)h->nu_c * h->nu_c * sizeof(float2), 0);
            if (zero && ctail_deep(h)) {
                const void *img = ctail_image(h, !h->capturing, true);
                if (img)
                    return launch_mg_chalo(nt, ops, b, u, h->minv32, h->nu_c, h->mg.nu1, h->mg.nu2,
                                           (float)h->mg.omega, h->tune.cluster_ctas, img, h->stream);
            }
            return launch_mg_ctail(nt, ops, b, u, h->minv32, h->nu_c, h->mg.nu1, h->mg.nu2,
                                   h->mg.smoother == HELM_SMOOTH_RB, (float)h->mg.omega, zero ? 1 : 0, gf, gc,
                                   h->tune.cluster_ctas, ctail_image(h, !h->capturing, false), h->stream);
        }
    }
    if (l == tail_top<R>(h)) {
        // levels l..last in one fused single-block launch
        const int nt = last - l + 1;
        DevOp<R> ops[MAX_TAIL_LEVELS];
        typename CT<R>::T *bb[MAX_TAIL_LEVELS], *uu[MAX_TAIL_LEVELS], *tt[MAX_TAIL_LEVELS];
        double bytes = 0;
        for (int k = 0; k < nt; k++) {
            LevelDev &Lk = h->lv[l + k];
            ops[k] = LvBuf<R>::op(Lk);
            bb[k] = k == 0 ? const_cast<typename CT<R>::T *>(b) : LvBuf<R>::b(Lk);
            uu[k] = k == 0 ? u : LvBuf<R>::u(Lk);
            tt[k] = LvBuf<R>::t(Lk);
            bytes += interior(Lk, h->dim) * sizeof(typename CT<R>::T) * 8.0;
        }
        ProfScope ps(h, HELM_K_COARSE, bytes + (double)h->nu_c * h->nu_c * sizeof(typename CT<R>::T), 0);
        return launch_mg_tail<R>(h->dim, nt, ops, bb, uu, tt, LvBuf<R>::minv(h), h->nu_c, h->mg.nu1, h->mg.nu2,
                                 h->mg.smoother == HELM_SMOOTH_RB, (R)h->mg.omega, gf, gc, zero ? 1 : 0, h->stream);
    }
    const double es = sizeof(C), rs = sizeof(R), ni = interior(L, h->dim), nd = h->dim == 3 ? 8.0 : 4.0;
    if constexpr (sizeof(R) == sizeof(float)) {
        // temporal blocking: two pre-sweeps from zero + residual + FW in one launch (iterate to
        // this level's t), the coarse correction, then correction + two post-sweeps in one
        // launch (t -> u)
        const int tile = l < HELM_MAX_LEVELS ? h->tune.level_tile[l] : (int)HELM_TILE_NONE;
        if (zero && h->mg.smoother == HELM_SMOOTH_JACOBI && h->mg.nu1 == 2 && h->mg.nu2 == 2 &&
            fused_jacobi2_ok(L.n, h->dim, tile)) {
            LevelDev &Lc = h->lv[l + 1];
            {
                // fused: read b and 1/D, write u and the coarse residual; pass by pass: the
                // first sweep from zero (b, k^2 -> u), the second (u, b, k^2 -> u), the
                // residual with full weighting (u, b, k^2 -> coarse)
                ProfScope ps(h, l == 0 ? HELM_K_SMOOTH_FINE : HELM_K_SMOOTH_COARSE, ni * (es + es + es + es / nd), 0,
                             ni * ((2 * es + rs) + (3 * es + rs) + (2 * es + rs + es / nd)));
                CKE(launch_pre2_restrict(L.M32, tile, (float)h->mg.omega, b, L.t32, Lc.b32, h->stream));
            }
            float2 *ec = Lc.u32;
            if (l + 1 == last) {
                CKE(coarse_solve<R>(h, Lc, Lc.b32, ec));
            } else {
                for (int i = 1; i <= gc; i++) {
                    if (i == 1) CKE(cycle<R>(h, l + 1, Lc.b32, ec, true, gf, gc));
                    else CKE(cycle<R>(h, l + 1, Lc.b32, ec, false, gc, gf));
                }
            }
            // fused: read b, 1/D, u and the coarse correction, write u; pass by pass: the
            // prolongation with correction (u, coarse -> u) and two sweeps (u, b, k^2 -> u)
            ProfScope ps(h, l == 0 ? HELM_K_SMOOTH_FINE : HELM_K_SMOOTH_COARSE, ni * (es + es + es + es / nd + es), 0,
                         ni * ((2 * es + es / nd) + 2 * (3 * es + rs)));
            return launch_prolong_post2(L.M32, tile, (float)h->mg.omega, b, L.t32, u, ec, h->stream);
        }
    }
    C *cur = u, *oth = LvBuf<R>::t(L);
    CKE(smooth<R>(h, l, h->mg.nu1, b, &cur, &oth, zero));
    LevelDev &Lc = h->lv[l + 1];
    {
        ProfScope ps(h, HELM_K_RESTRICT, ni * (2 * es + rs + es / nd), 0);
        CKE(launch_residual_restrict<R>(LvBuf<R>::op(L), h->dim, b, cur, LvBuf<R>::b(Lc), h->stream));
    }
    C *ec = LvBuf<R>::u(Lc);
    if (l + 1 == last) {
        CKE(coarse_solve<R>(h, Lc, LvBuf<R>::b(Lc), ec));
    } else {
        for (int i = 1; i <= gc; i++) {
            if (i == 1) CKE(cycle<R>(h, l + 1, LvBuf<R>::b(Lc), ec, true, gf, gc));
            else CKE(cycle<R>(h, l + 1, LvBuf<R>::b(Lc), ec, false, gc, gf));
        }
    }
    {
        ProfScope ps(h, HELM_K_PROLONG, ni * (2 * es + es / nd), 0);
        CKE(launch_prolong_add<R>(L.n, h->dim, ec, cur, h->stream, LvBuf<R>::op(L).gate));
    }
    CKE(smooth<R>(h, l, h->mg.nu2, b, &cur, &oth, false));
    if (cur != u) CKE(cudaMemcpyAsync(u, cur, L.np * sizeof(C), cudaMemcpyDeviceToDevice, h->stream));
    return cudaSuccess;
}

// z = M^{-1}-approximation of v (one cycle from zero), v in FP64, z in precision R.
template <typename R>
cudaError_t precondition(helm_handle *h, const double2 *v, typename CT<R>::T *z) {
    pdl_cycle_scope pdl;
    const double es = sizeof(typename CT<R>::T);
    if (h->mg.kind == HELM_PC_NONE) {
        ProfScope ps(h, HELM_K_VECTOR, h->np * (16 + es), 0);
        return launch_convert(h->np, v, z, h->stream);
    }
    if (sizeof(R) == sizeof(double))
        return cycle<R>(h, 0, (const typename CT<R>::T *)v, z, true, h->mg.gamma_f, h->mg.gamma_c);
    {
        ProfScope ps(h, HELM_K_VECTOR, h->np * (16 + es), 0);
        CKE(launch_convert(h->np, v, LvBuf<R>::b(h->lv[0]), h->stream));
    }
    return cycle<R>(h, 0, LvBuf<R>::b(h->lv[0]), z, true, h->mg.gamma_f, h->mg.gamma_c);
}
template cudaError_t precondition<float>(helm_handle *, const double2 *, float2 *);
template cudaError_t precondition<double>(helm_handle *, const double2 *, double2 *);

// The same with v / alpha->x for a float-pair vector v (the double-FP32 Krylov basis; alpha
// null: no scaling): converted into level 0's right-hand side in precision R, then one cycle
// from zero.
template <typename R>
cudaError_t precondition_pair(helm_handle *h, const float4 *v, const double2 *alpha, typename CT<R>::T *z) {
    pdl_cycle_scope pdl;
    typedef typename CT<R>::T C;
    const double es = sizeof(C);
    C *dst = h->mg.kind == HELM_PC_NONE ? z : LvBuf<R>::b(h->lv[0]);
    {
        ProfScope ps(h, HELM_K_VECTOR, h->np * (16 + es), 0);
        if constexpr (sizeof(R) == sizeof(float)) CKE(launch_pair_to_c64(h->np, v, alpha, dst, h->stream));
        else CKE(launch_pair_to_c128(h->np, v, alpha, dst, h->stream));
    }
    if (h->mg.kind == HELM_PC_NONE) return cudaSuccess;
    return cycle<R>(h, 0, dst, z, true, h->mg.gamma_f, h->mg.gamma_c);
}
template cudaError_t precondition_pair<float>(helm_handle *, const float4 *, const double2 *, float2 *);
cudaError_t precondition_level0_c64(helm_handle *h, float2 *z) {
    pdl_cycle_scope pdl;
    return cycle<float>(h, 0, LvBuf<float>::b(h->lv[0]), z, true, h->mg.gamma_f, h->mg.gamma_c);
}
float2 *level0_rhs_c64(helm_handle *h) { return LvBuf<float>::b(h->lv[0]); }
template cudaError_t precondition_pair<double>(helm_handle *, const float4 *, const double2 *, double2 *);

static helm_status check_ptr(const void *p, size_t align, const char *name) {
    if (!p) return helm_fail(HELM_ERR_ARG, "%s is null", name);
    if ((uintptr_t)p % align) return helm_fail(HELM_ERR_ARG, "%s is not %zu-byte aligned", name, align);
    return HELM_OK;
}

extern "C" helm_status helm_apply(helm_handle *h, helm_op which, helm_prec prec, const void *x, void *y) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    const size_t al = prec == HELM_C128 ? 16 : 8;
    helm_status st;
    if ((st = check_ptr(x, al, "x")) != HELM_OK || (st = check_ptr(y, al, "y")) != HELM_OK) return st;
    if (x == y) return helm_fail(HELM_ERR_ARG, "x and y must not overlap");
    if (which != HELM_OP_A && which != HELM_OP_M) return helm_fail(HELM_ERR_ARG, "bad operator");
    if (prec == HELM_C128) {
        const DevOp<double> &op = which == HELM_OP_A ? h->A64 : h->lv[0].M64;
        CKR(launch_apply<double, double2>(op, h->dim, (const double2 *)x, (double2 *)y, h->stream));
    } else if (prec == HELM_C64) {
        if (which == HELM_OP_A) {
            if (!h->A32.k2) {
                // FP32 copy of A, built on first use
                std::vector<cd> tri;
                for (int a = 0; a < 3; a++) {
                    std::vector<double2> t(3 * (size_t)h->n[a]);
                    CKR(cudaMemcpy(t.data(), h->coefA64[a], t.size() * sizeof(double2), cudaMemcpyDeviceToHost));
                    tri.resize(t.size());
                    for (size_t q = 0; q < t.size(); q++) tri[q] = cd(t[q].x, t[q].y);
                    CKR(upload_c(&h->coefA32[a], tri, h->owned, h->stream));
                    h->A32.coef[a] = h->coefA32[a];
                    h->A32.n[a] = h->n[a];
                }
                h->A32.k2 = h->lv[0].k2_32;
                h->A32.bk = make_float2(-1.f, 0.f);
                h->A32.c = make_float2(0.f, 0.f);
            }
            CKR(launch_apply<float, float2>(h->A32, h->dim, (const float2 *)x, (float2 *)y, h->stream));
        } else {
            CKR(launch_apply<float, float2>(h->lv[0].M32, h->dim, (const float2 *)x, (float2 *)y, h->stream));
        }
    } else {
        return helm_fail(HELM_ERR_ARG, "bad precision");
    }
    return HELM_OK;
}

extern "C" helm_status mg_vcycle(helm_handle *h, const void *b, void *x, helm_prec prec) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    if (h->mg.kind == HELM_PC_NONE) return helm_fail(HELM_ERR_ARG, "handle has no preconditioner hierarchy");
    const size_t al = prec == HELM_C128 ? 16 : 8;
    helm_status st;
    if ((st = check_ptr(b, al, "b")) != HELM_OK || (st = check_ptr(x, al, "x")) != HELM_OK) return st;
    if (b == x) return helm_fail(HELM_ERR_ARG, "b and x must not overlap");
    if (prec == HELM_C128)
        CKR(cycle<double>(h, 0, (const double2 *)b, (double2 *)x, false, h->mg.gamma_f, h->mg.gamma_c));
    else if (prec == HELM_C64)
        CKR(cycle<float>(h, 0, (const float2 *)b, (float2 *)x, false, h->mg.gamma_f, h->mg.gamma_c));
    else
        return helm_fail(HELM_ERR_ARG, "bad precision");
    return HELM_OK;
}

extern "C" helm_status mg_precondition(helm_handle *h, const void *v, void *z, helm_prec prec) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    if (h->mg.kind == HELM_PC_NONE) return helm_fail(HELM_ERR_ARG, "handle has no preconditioner hierarchy");
    helm_status st;
    if ((st = check_ptr(v, 16, "v")) != HELM_OK ||
        (st = check_ptr(z, prec == HELM_C128 ? 16 : 8, "z")) != HELM_OK)
        return st;
    if (v == z) return helm_fail(HELM_ERR_ARG, "v and z must not overlap");
    if (prec == HELM_C128)
        CKR(precondition<double>(h, (const double2 *)v, (double2 *)z));
    else if (prec == HELM_C64)
        CKR(precondition<float>(h, (const double2 *)v, (float2 *)z));
    else
        return helm_fail(HELM_ERR_ARG, "bad precision");
    return HELM_OK;
}

extern "C" helm_status helm_grad_k2(helm_handle *h, const void *lambda, const void *u, double *grad) {
    if (!h) return helm_fail(HELM_ERR_ARG, "null handle");
    helm_status st;
    if ((st = check_ptr(lambda, 16, "lambda")) != HELM_OK || (st = check_ptr(u, 16, "u")) != HELM_OK ||
        (st = check_ptr(grad, 8, "grad")) != HELM_OK)
        return st;
    CKR(launch_grad_k2(h->np, h->n, h->dim, (const double2 *)lambda, (const double2 *)u, grad, h->stream));
    return HELM_OK;
}
