/*
 * helm_oracle.c -- plain, slow, FP64 CPU oracle for the matrix-free ECS Helmholtz
 * solver of bin Zubair, Reps & Vanroose, "A preconditioned iterative solver for the
 * scattering solutions of the Schroedinger equation" (arXiv 1012.4307).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load this file.  The GPU library shares no code, header, table or helper
 * with it, and never calls it.
 *
 * Everything is written as the paper states it, in the paper's order, with
 * `double complex` arithmetic and no blocking, fusion or reordering:
 *   - the ECS contour z(x) of Section 3.1 (linear f, so the layer widths are h e^{i theta});
 *   - the non-uniform three-point second difference of Section 3.2, summed over axes;
 *   - the preconditioner operators CSL / CSG / QD of Section 5 (eqs. for M_CSL, M_CSG,
 *     M_QD) written as  M = a * L_h(widths * e^{i ts}) + bk * k^2 + c;
 *   - omega-Jacobi and omega-red-black Jacobi smoothing, full-weighting restriction,
 *     bi/trilinear prolongation and rediscretised coarse operators (Section 4.2);
 *   - the multigrid recursion MG(l, A, b, u, nu1, nu2, C, gamma_f, gamma_c) (Algorithm 1);
 *   - flexible GMRES (the paper's Section 6 mentions (restarted) GMRES) and
 *     right-preconditioned Bi-CGSTAB with two preconditioner calls per iteration (Section 5).
 *
 * Readings taken where the paper is silent are listed at the function that takes them.
 * Storage: node arrays of n0*n1*n2 values including the Dirichlet boundary nodes,
 * index p = i + n0*(j + n1*k), x fastest.  Boundary values are zero and never read as
 * unknowns.  Complex vectors are C99 `double complex` (re, im pairs).
 *
 * Parity pins: every function here is pinned by a test in tests/test_oracle_pins.py against
 * something other than itself (closed forms, dense linear algebra, Lemma 3.1, exact lattice
 * Green's functions, textbook identities).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* One discrete operator  M = a * L_h + bk * diag(k^2) + c * I  on an ECS grid.
 * L_h is the negative FD Laplacian of Section 3.2 on the complex nodes z[axis][j], with
 * every mesh width multiplied by e^{i ts} (ts = theta_alpha for the complex-scaled grid
 * of Section 5, 0 otherwise).  k2 holds real k^2 values at every node. */
typedef struct {
    int dim;             /* 1, 2 or 3                                        */
    int n[3];            /* nodes per axis incl. the two Dirichlet nodes; 1 for unused axes */
    const cplx *z[3];    /* complex node coordinates per axis (length n[a]) */
    cplx a, bk, c;       /* operator coefficients                           */
    double ts;           /* extra rotation of all widths (CSG)              */
    const double *k2;    /* k^2 at every node (length n0*n1*n2)             */
} or_op;

static size_t npts(const or_op *op) { return (size_t)op->n[0] * op->n[1] * op->n[2]; }

/* ------------------------------------------------------------------------------------ */
/* Section 3.1: exterior complex scaling with a linear scaling function.  Real nodes
 * x_j = lo + j (hi-lo)/(n-1).  Inside [r0lo, r0hi] the contour is z = x; beyond r0hi it is
 * z = r0hi + (x - r0hi) e^{i theta}, and beyond r0lo (mirror image) z = r0lo + (x - r0lo)
 * e^{i theta}, so both layers have complex widths h e^{i theta}.  A side whose r0 lies
 * outside [lo, hi] has no layer (plain Dirichlet there). */
void or_contour(int n, double lo, double hi, double theta, double r0lo, double r0hi, cplx *z)
{
    double h = (hi - lo) / (double)(n - 1);
    cplx rot = cexp(I * theta);
    for (int j = 0; j < n; j++) {
        double x = lo + h * (double)j;
        if (j == n - 1) x = hi;
        if (x > r0hi)
            z[j] = r0hi + (x - r0hi) * rot;
        else if (x < r0lo)
            z[j] = r0lo + (x - r0lo) * rot;
        else
            z[j] = x;
    }
}

/* Section 3.2: the three coefficients of  -d^2u/dz^2  at node j from the formula for
 * unequal widths, with h_{j-1} = z_j - z_{j-1} and h_j = z_{j+1} - z_j (times e^{i ts}):
 *   d^2u/dz^2 ~ 2/(h_{j-1}+h_j) * ( u_{j-1}/h_{j-1} - (1/h_{j-1}+1/h_j) u_j + u_{j+1}/h_j ).
 * Returned as coefficients of -d^2/dz^2 (west, centre, east). */
static void fd_coef(const cplx *z, int j, double ts, cplx *w, cplx *ctr, cplx *e)
{
    cplx rot = cexp(I * ts);
    cplx hm = (z[j] - z[j - 1]) * rot;
    cplx hp = (z[j + 1] - z[j]) * rot;
    cplx s = 2.0 / (hm + hp);
    *w = -s / hm;
    *ctr = s * (1.0 / hm + 1.0 / hp);
    *e = -s / hp;
}

static int is_interior(const or_op *op, int i, int j, int k)
{
    if (i < 1 || i > op->n[0] - 2) return 0;
    if (op->dim >= 2 && (j < 1 || j > op->n[1] - 2)) return 0;
    if (op->dim >= 3 && (k < 1 || k > op->n[2] - 2)) return 0;
    return 1;
}

/* (M x)_p at one interior node p = (i, j, k). */
static cplx apply_at(const or_op *op, const cplx *x, int i, int j, int k)
{
    const int n0 = op->n[0], n1 = op->n[1];
    const size_t p = (size_t)i + (size_t)n0 * ((size_t)j + (size_t)n1 * k);
    const size_t stride[3] = {1, (size_t)n0, (size_t)n0 * n1};
    const int idx[3] = {i, j, k};
    cplx lap = 0;
    for (int ax = 0; ax < op->dim; ax++) {
        cplx w, ctr, e;
        fd_coef(op->z[ax], idx[ax], op->ts, &w, &ctr, &e);
        lap += w * x[p - stride[ax]] + ctr * x[p] + e * x[p + stride[ax]];
    }
    return op->a * lap + (op->bk * op->k2[p] + op->c) * x[p];
}

/* Diagonal entry of M at p: a * sum_axes centre coefficient + bk k^2_p + c. */
static cplx diag_at(const or_op *op, int i, int j, int k)
{
    const int n0 = op->n[0], n1 = op->n[1];
    const size_t p = (size_t)i + (size_t)n0 * ((size_t)j + (size_t)n1 * k);
    const int idx[3] = {i, j, k};
    cplx d = 0;
    for (int ax = 0; ax < op->dim; ax++) {
        cplx w, ctr, e;
        fd_coef(op->z[ax], idx[ax], op->ts, &w, &ctr, &e);
        d += ctr;
    }
    return op->a * d + op->bk * op->k2[p] + op->c;
}

#define FOR_NODES(op)                                   \
    for (int k = 0; k < (op)->n[2]; k++)                \
        for (int j = 0; j < (op)->n[1]; j++)            \
            for (int i = 0; i < (op)->n[0]; i++)

/* The same loop for bodies that write only their own node p from inputs the loop does not
 * write: its iterations are independent, so with -fopenmp (the all-cores build of the CPU
 * baseline) they are shared out over threads with bit-identical results; without -fopenmp the
 * pragma is ignored.  Reductions (dot products, norms, counts) are never shared out. */
#define FOR_NODES_INDEP(op)                             \
    _Pragma("omp parallel for collapse(2) schedule(static)") \
    FOR_NODES(op)

#define PIDX(op) ((size_t)i + (size_t)(op)->n[0] * ((size_t)j + (size_t)(op)->n[1] * k))

/* y = M x on interior nodes; boundary nodes of y are set to zero. */
void or_apply(const or_op *op, const cplx *x, cplx *y)
{
    FOR_NODES_INDEP(op) {
        size_t p = PIDX(op);
        y[p] = is_interior(op, i, j, k) ? apply_at(op, x, i, j, k) : 0;
    }
}

/* y = M^T x (plain transpose, no conjugation): (M^T x)_p = sum_q M_{qp} x_q.  Row q = p -/+ e
 * holds x_p with its east/west coefficient respectively. */
void or_apply_T(const or_op *op, const cplx *x, cplx *y)
{
    const size_t stride[3] = {1, (size_t)op->n[0], (size_t)op->n[0] * op->n[1]};
    FOR_NODES_INDEP(op) {
        size_t p = PIDX(op);
        if (!is_interior(op, i, j, k)) { y[p] = 0; continue; }
        const int idx[3] = {i, j, k};
        cplx acc = 0;
        for (int ax = 0; ax < op->dim; ax++) {
            cplx w, ctr, e;
            fd_coef(op->z[ax], idx[ax], op->ts, &w, &ctr, &e);
            acc += ctr * x[p];
            if (idx[ax] - 1 >= 1) {            /* row q = p - e_ax is an unknown */
                cplx wq, cq, eq;
                fd_coef(op->z[ax], idx[ax] - 1, op->ts, &wq, &cq, &eq);
                acc += eq * x[p - stride[ax]];
            }
            if (idx[ax] + 1 <= op->n[ax] - 2) {  /* row q = p + e_ax is an unknown */
                cplx wq, cq, eq;
                fd_coef(op->z[ax], idx[ax] + 1, op->ts, &wq, &cq, &eq);
                acc += wq * x[p + stride[ax]];
            }
        }
        y[p] = op->a * acc + (op->bk * op->k2[p] + op->c) * x[p];
    }
}

void or_diag(const or_op *op, cplx *d)
{
    FOR_NODES_INDEP(op) {
        size_t p = PIDX(op);
        d[p] = is_interior(op, i, j, k) ? diag_at(op, i, j, k) : 0;
    }
}

/* r = f - M u on interior nodes, zero on the boundary (Algorithm 1, step 2). */
void or_residual(const or_op *op, const cplx *f, const cplx *u, cplx *r)
{
    FOR_NODES_INDEP(op) {
        size_t p = PIDX(op);
        r[p] = is_interior(op, i, j, k) ? f[p] - apply_at(op, u, i, j, k) : 0;
    }
}

/* omega-Jacobi (Section 4.2): every unknown at once,
 *   u_p <- u_p + omega (f_p - (M u)_p) / M_pp,  using the old u everywhere. */
void or_jacobi(const or_op *op, double omega, int sweeps, const cplx *f, cplx *u)
{
    size_t np = npts(op);
    cplx *r = (cplx *)malloc(np * sizeof(cplx));
    for (int s = 0; s < sweeps; s++) {
        or_residual(op, f, u, r);
        FOR_NODES_INDEP(op) {
            if (!is_interior(op, i, j, k)) continue;
            size_t p = PIDX(op);
            u[p] += omega * r[p] / diag_at(op, i, j, k);
        }
    }
    free(r);
}

/* omega-red-black Jacobi (Section 4.2): first every "red" unknown, (i+j+k) even, is
 * relaxed as in Jacobi; then every "black" unknown, (i+j+k) odd, using the new red values.
 * The node indices are those of the level's own grid. */
void or_rbjacobi(const or_op *op, double omega, int sweeps, const cplx *f, cplx *u)
{
    for (int s = 0; s < sweeps; s++) {
        for (int colour = 0; colour < 2; colour++) {
            size_t np = npts(op);
            cplx *upd = (cplx *)calloc(np, sizeof(cplx));
            FOR_NODES_INDEP(op) {
                if (!is_interior(op, i, j, k) || ((i + j + k) & 1) != colour) continue;
                size_t p = PIDX(op);
                upd[p] = omega * (f[p] - apply_at(op, u, i, j, k)) / diag_at(op, i, j, k);
            }
            FOR_NODES_INDEP(op) {
                if (!is_interior(op, i, j, k) || ((i + j + k) & 1) != colour) continue;
                u[PIDX(op)] += upd[PIDX(op)];
            }
            free(upd);
        }
    }
}

/* Full-weighting restriction (Section 4.2, "full weighting averaging"): coarse node I takes
 * sum over offsets d in {-1,0,1}^dim of prod_ax w(d_ax) * r_f[2I + d], with w(0) = 1/2 and
 * w(+-1) = 1/4 (the (1,2,1)/4 stencil per axis).  Coarse boundary nodes are set to zero.
 * nf = fine nodes per axis (odd); coarse nodes per axis (nf+1)/2. */
void or_restrict(int dim, const int nf[3], const cplx *rf, cplx *rc)
{
    int nc[3] = {1, 1, 1};
    for (int a = 0; a < dim; a++) nc[a] = (nf[a] + 1) / 2;
    _Pragma("omp parallel for collapse(2) schedule(static)")
    for (int K = 0; K < nc[2]; K++)
        for (int J = 0; J < nc[1]; J++)
            for (int Ii = 0; Ii < nc[0]; Ii++) {
                size_t pc = (size_t)Ii + (size_t)nc[0] * ((size_t)J + (size_t)nc[1] * K);
                int ci[3] = {Ii, J, K};
                int inner = 1;
                for (int a = 0; a < dim; a++)
                    if (ci[a] < 1 || ci[a] > nc[a] - 2) inner = 0;
                if (!inner) { rc[pc] = 0; continue; }
                cplx acc = 0;
                for (int dk = (dim >= 3 ? -1 : 0); dk <= (dim >= 3 ? 1 : 0); dk++)
                    for (int dj = (dim >= 2 ? -1 : 0); dj <= (dim >= 2 ? 1 : 0); dj++)
                        for (int di = -1; di <= 1; di++) {
                            double w = (di == 0 ? 0.5 : 0.25);
                            if (dim >= 2) w *= (dj == 0 ? 0.5 : 0.25);
                            if (dim >= 3) w *= (dk == 0 ? 0.5 : 0.25);
                            int fi = 2 * Ii + di, fj = (dim >= 2 ? 2 * J + dj : 0),
                                fk = (dim >= 3 ? 2 * K + dk : 0);
                            size_t pf = (size_t)fi + (size_t)nf[0] * ((size_t)fj + (size_t)nf[1] * fk);
                            acc += w * rf[pf];
                        }
                rc[pc] = acc;
            }
}

/* Bi/trilinear prolongation and correction (Section 4.2, Algorithm 1 step 2):
 * u_f += I_{l+1}^l e_c.  Fine node q takes the average of the coarse nodes at
 * floor(q/2) and ceil(q/2) along every axis (a coincident node copies its coarse value,
 * an edge node averages 2, a face-centre 4, a cell-centre 8).  Only interior fine
 * nodes are corrected; coarse boundary values are the zero Dirichlet values. */
void or_prolong_add(int dim, const int nf[3], const cplx *ec, cplx *uf)
{
    int nc[3] = {1, 1, 1};
    int nfx[3] = {nf[0], dim >= 2 ? nf[1] : 1, dim >= 3 ? nf[2] : 1};
    for (int a = 0; a < dim; a++) nc[a] = (nf[a] + 1) / 2;
    _Pragma("omp parallel for collapse(2) schedule(static)")
    for (int k = 0; k < nfx[2]; k++)
        for (int j = 0; j < nfx[1]; j++)
            for (int i = 0; i < nfx[0]; i++) {
                int q[3] = {i, j, k};
                int inner = 1;
                for (int a = 0; a < dim; a++)
                    if (q[a] < 1 || q[a] > nfx[a] - 2) inner = 0;
                if (!inner) continue;
                int lo[3], hi[3];
                for (int a = 0; a < 3; a++) {
                    if (a < dim) { lo[a] = q[a] / 2; hi[a] = (q[a] + 1) / 2; }
                    else { lo[a] = 0; hi[a] = 0; }
                }
                cplx acc = 0;
                int cnt = 0;
                for (int ck = lo[2]; ck <= hi[2]; ck++)
                    for (int cj = lo[1]; cj <= hi[1]; cj++)
                        for (int ci = lo[0]; ci <= hi[0]; ci++) {
                            acc += ec[(size_t)ci + (size_t)nc[0] * ((size_t)cj + (size_t)nc[1] * ck)];
                            cnt++;
                        }
                uf[(size_t)i + (size_t)nfx[0] * ((size_t)j + (size_t)nfx[1] * k)] += acc / (double)cnt;
            }
}

/* ------------------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (textbook Gaussian elimination), column-major A (n x n),
 * overwritten by its factors; piv records row swaps.  Returns 0, or -1 if singular. */
int or_lu_factor(int n, cplx *A, int *piv)
{
    for (int c = 0; c < n; c++) {
        int best = c;
        double bv = cabs(A[c + (size_t)n * c]);
        for (int r = c + 1; r < n; r++)
            if (cabs(A[r + (size_t)n * c]) > bv) { bv = cabs(A[r + (size_t)n * c]); best = r; }
        piv[c] = best;
        if (bv == 0.0) return -1;
        if (best != c)
            for (int cc = 0; cc < n; cc++) {
                cplx t = A[c + (size_t)n * cc];
                A[c + (size_t)n * cc] = A[best + (size_t)n * cc];
                A[best + (size_t)n * cc] = t;
            }
        for (int r = c + 1; r < n; r++) {
            cplx l = A[r + (size_t)n * c] / A[c + (size_t)n * c];
            A[r + (size_t)n * c] = l;
            for (int cc = c + 1; cc < n; cc++) A[r + (size_t)n * cc] -= l * A[c + (size_t)n * cc];
        }
    }
    return 0;
}

void or_lu_solve(int n, const cplx *LU, const int *piv, cplx *b)
{
    for (int c = 0; c < n; c++)
        if (piv[c] != c) { cplx t = b[c]; b[c] = b[piv[c]]; b[piv[c]] = t; }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < r; c++) b[r] -= LU[r + (size_t)n * c] * b[c];
    for (int r = n - 1; r >= 0; r--) {
        for (int c = r + 1; c < n; c++) b[r] -= LU[r + (size_t)n * c] * b[c];
        b[r] /= LU[r + (size_t)n * r];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Multigrid hierarchy (Section 4.2: rediscretisation on the coarse grids).  Level l+1 has
 * (n+1)/2 nodes per axis.  Its complex nodes are the contour sampled at the coarse real
 * nodes, i.e. every other fine node (z_c[I] = z_f[2I]), and its operator uses the same
 * (a, bk, c, ts) on those nodes.  Reading (paper silent): k^2 on a coarse level is
 * injected, k2_c[I] = k2_f[2I]. */
#define OR_MAXLEV 16
typedef struct {
    int nlev;
    or_op op[OR_MAXLEV];
    cplx *zbuf[OR_MAXLEV][3];
    double *k2buf[OR_MAXLEV];
    /* coarsest level: dense LU of M_C on its unknowns */
    int nc_unk;
    cplx *lu;
    int *piv;
    size_t *unk_index;  /* unknown number -> node index on the coarsest grid */
    /* cycle parameters */
    int nu1, nu2, smoother; /* 0 = omega-Jacobi, 1 = omega-red-black Jacobi */
    double omega;
} or_mg;

static void level_unknowns(const or_op *op, size_t **idx, int *count)
{
    int cnt = 0;
    FOR_NODES(op) if (is_interior(op, i, j, k)) cnt++;
    *idx = (size_t *)malloc((size_t)(cnt ? cnt : 1) * sizeof(size_t));
    cnt = 0;
    FOR_NODES(op) if (is_interior(op, i, j, k)) (*idx)[cnt++] = PIDX(op);
    *count = cnt;
}

/* Should the level with operator op be coarsened once more?  Yes while some axis has more
 * than coarsest_n nodes and every axis has an even number of cells leaving >= 3 nodes. */
static int coarsen_further(const or_op *op, int coarsest_n)
{
    int small = 1;
    for (int a = 0; a < op->dim; a++) {
        if (op->n[a] > coarsest_n) small = 0;
        if ((op->n[a] - 1) % 2 != 0 || (op->n[a] + 1) / 2 < 3) return 0;
    }
    return !small;
}

/* Builds the hierarchy from the fine operator down to the first level with at most
 * coarsest_n nodes per axis, then factors the coarsest operator (Algorithm 1, "exact").
 * mg->nc_unk is -1 if the coarsest operator is singular. */
or_mg *or_mg_create(const or_op *fine, int coarsest_n, int nu1, int nu2, double omega, int smoother)
{
    or_mg *mg = (or_mg *)calloc(1, sizeof(or_mg));
    mg->nu1 = nu1; mg->nu2 = nu2; mg->omega = omega; mg->smoother = smoother;
    /* level 0: own copies of the fine nodes and k^2 */
    mg->op[0] = *fine;
    for (int a = 0; a < 3; a++) {
        mg->zbuf[0][a] = (cplx *)calloc((size_t)fine->n[a], sizeof(cplx));
        if (a < fine->dim) memcpy(mg->zbuf[0][a], fine->z[a], (size_t)fine->n[a] * sizeof(cplx));
        mg->op[0].z[a] = mg->zbuf[0][a];
    }
    mg->k2buf[0] = (double *)malloc(npts(fine) * sizeof(double));
    memcpy(mg->k2buf[0], fine->k2, npts(fine) * sizeof(double));
    mg->op[0].k2 = mg->k2buf[0];
    int l = 0;
    while (l + 1 < OR_MAXLEV && coarsen_further(&mg->op[l], coarsest_n)) {
        const or_op *f = &mg->op[l];
        or_op *c = &mg->op[l + 1];
        *c = *f;
        for (int a = 0; a < f->dim; a++) c->n[a] = (f->n[a] + 1) / 2;
        for (int a = 0; a < 3; a++) {
            mg->zbuf[l + 1][a] = (cplx *)calloc((size_t)c->n[a], sizeof(cplx));
            if (a < f->dim)
                for (int j = 0; j < c->n[a]; j++) mg->zbuf[l + 1][a][j] = f->z[a][2 * j];
            c->z[a] = mg->zbuf[l + 1][a];
        }
        mg->k2buf[l + 1] = (double *)malloc(npts(c) * sizeof(double));
        for (int k = 0; k < c->n[2]; k++)
            for (int j = 0; j < c->n[1]; j++)
                for (int i = 0; i < c->n[0]; i++) {
                    int fi = 2 * i, fj = (f->dim >= 2 ? 2 * j : 0), fk = (f->dim >= 3 ? 2 * k : 0);
                    mg->k2buf[l + 1][(size_t)i + (size_t)c->n[0] * ((size_t)j + (size_t)c->n[1] * k)] =
                        f->k2[(size_t)fi + (size_t)f->n[0] * ((size_t)fj + (size_t)f->n[1] * fk)];
                }
        c->k2 = mg->k2buf[l + 1];
        l++;
    }
    mg->nlev = l + 1;
    /* coarsest: dense M_C on its unknowns, assembled column by column from the apply */
    const or_op *C = &mg->op[mg->nlev - 1];
    level_unknowns(C, &mg->unk_index, &mg->nc_unk);
    int nu = mg->nc_unk;
    size_t np = npts(C);
    mg->lu = (cplx *)malloc((size_t)(nu ? nu : 1) * (nu ? nu : 1) * sizeof(cplx));
    mg->piv = (int *)malloc((size_t)(nu ? nu : 1) * sizeof(int));
    cplx *e = (cplx *)calloc(np, sizeof(cplx));
    cplx *col = (cplx *)calloc(np, sizeof(cplx));
    for (int c = 0; c < nu; c++) {
        e[mg->unk_index[c]] = 1;
        or_apply(C, e, col);
        e[mg->unk_index[c]] = 0;
        for (int r = 0; r < nu; r++) mg->lu[r + (size_t)nu * c] = col[mg->unk_index[r]];
    }
    free(e); free(col);
    if (or_lu_factor(nu, mg->lu, mg->piv) != 0) mg->nc_unk = -1;
    return mg;
}

void or_mg_destroy(or_mg *mg)
{
    if (!mg) return;
    for (int l = 0; l < mg->nlev; l++) {
        for (int a = 0; a < 3; a++) free(mg->zbuf[l][a]);
        free(mg->k2buf[l]);
    }
    free(mg->lu); free(mg->piv); free(mg->unk_index);
    free(mg);
}

int or_mg_levels(const or_mg *mg) { return mg->nlev; }
void or_mg_level_shape(const or_mg *mg, int l, int n[3]) { for (int a = 0; a < 3; a++) n[a] = mg->op[l].n[a]; }
int or_mg_ok(const or_mg *mg) { return mg->nc_unk >= 0; }

/* Algorithm 1, step (0) "exact": u = M_C^{-1} b on the coarsest grid (boundary zero). */
static void exact_solve(const or_mg *mg, const cplx *b, cplx *u)
{
    const or_op *C = &mg->op[mg->nlev - 1];
    int nu = mg->nc_unk;
    cplx *rhs = (cplx *)malloc((size_t)(nu ? nu : 1) * sizeof(cplx));
    for (int r = 0; r < nu; r++) rhs[r] = b[mg->unk_index[r]];
    or_lu_solve(nu, mg->lu, mg->piv, rhs);
    memset(u, 0, npts(C) * sizeof(cplx));
    for (int r = 0; r < nu; r++) u[mg->unk_index[r]] = rhs[r];
    free(rhs);
}

static void smooth(const or_mg *mg, int l, int sweeps, const cplx *b, cplx *u)
{
    if (mg->smoother == 1) or_rbjacobi(&mg->op[l], mg->omega, sweeps, b, u);
    else or_jacobi(&mg->op[l], mg->omega, sweeps, b, u);
}

/* Algorithm 1: u <- MG(l, A_l, b, u, nu1, nu2, C, gamma_f, gamma_c).
 *  (0) at the coarsest level C: exact solve.
 *  (1) nu1 pre-smoothing steps.
 *  (2) residual, restriction, approximate coarse error by gamma_c recursive calls from a zero
 *      start, the first with (gamma_f, gamma_c) and the later ones with the two indices
 *      swapped; prolongate and correct.  Reading: the boxed "If l = C" test means "if the
 *      next level l+1 is the coarsest", where the error is the exact coarse solution.
 *  (3) nu2 post-smoothing steps. */
static void mg_rec(const or_mg *mg, int l, const cplx *b, cplx *u, int gf, int gc)
{
    const or_op *A = &mg->op[l];
    if (l == mg->nlev - 1) { exact_solve(mg, b, u); return; }
    smooth(mg, l, mg->nu1, b, u);
    size_t np = npts(A);
    const or_op *Ac = &mg->op[l + 1];
    size_t npc = npts(Ac);
    cplx *r = (cplx *)malloc(np * sizeof(cplx));
    cplx *rc = (cplx *)malloc(npc * sizeof(cplx));
    cplx *ec = (cplx *)calloc(npc, sizeof(cplx));
    or_residual(A, b, u, r);
    or_restrict(A->dim, A->n, r, rc);
    if (l + 1 == mg->nlev - 1) {
        exact_solve(mg, rc, ec);
    } else {
        for (int i = 1; i <= gc; i++) {
            if (i == 1) mg_rec(mg, l + 1, rc, ec, gf, gc);
            else mg_rec(mg, l + 1, rc, ec, gc, gf);
        }
    }
    or_prolong_add(A->dim, A->n, ec, u);
    smooth(mg, l, mg->nu2, b, u);
    free(r); free(rc); free(ec);
}

/* One cycle on the finest level: u (in: initial guess, out: result). */
void or_mg_cycle(const or_mg *mg, const cplx *b, cplx *u, int gamma_f, int gamma_c)
{
    mg_rec(mg, 0, b, u, gamma_f, gamma_c);
}

/* ------------------------------------------------------------------------------------ */
/* Krylov solvers.  Inner product <a, b> = sum conj(a_p) b_p (Hermitian); norms are l2
 * over all nodes (boundary values are zero). */
static cplx dotc(size_t n, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (size_t p = 0; p < n; p++) s += conj(a[p]) * b[p];
    return s;
}
static double nrm2(size_t n, const cplx *a) { return sqrt(creal(dotc(n, a, a))); }

typedef struct {
    int iterations;        /* Krylov iterations (FGMRES inner steps / Bi-CGSTAB steps) */
    int restarts;
    int status;            /* 0 converged, 1 not converged, 2 breakdown             */
    double rel_res;        /* final true ||f - A x|| / ||f||                        */
    double *history;       /* optional: residual estimate per iteration (caller-owned) */
    int history_len;       /* capacity of history                                   */
} or_stats;

/* Apply the preconditioner: z = MG-cycle(v) from a zero start, or z = v without one. */
static void precond(const or_mg *mg, int gf, int gc, size_t np, const cplx *v, cplx *z)
{
    memset(z, 0, np * sizeof(cplx));
    if (mg) or_mg_cycle(mg, v, z, gf, gc);
    else memcpy(z, v, np * sizeof(cplx));
}

/* Flexible GMRES(m) with right preconditioning (Saad, Iterative Methods for Sparse Linear
 * Systems, Algorithm 9.6), modified Gram-Schmidt Arnoldi and complex Givens rotations.
 * Reading (paper silent on Krylov details): x0 is the caller's x; convergence when the
 * Arnoldi residual estimate |g_{j+1}| <= tol ||f||, confirmed by the true residual at the
 * end of each cycle; restart from the current x.  maxit bounds the total inner steps. */
int or_fgmres(const or_op *A, const or_mg *mg, int gf, int gc, const cplx *f, cplx *x,
              double tol, int m, int maxit, or_stats *st)
{
    size_t np = npts(A);
    cplx *V = (cplx *)calloc((size_t)(m + 1) * np, sizeof(cplx));
    cplx *Z = (cplx *)calloc((size_t)m * np, sizeof(cplx));
    cplx *w = (cplx *)malloc(np * sizeof(cplx));
    cplx *H = (cplx *)calloc((size_t)(m + 1) * m, sizeof(cplx));   /* column-major */
    double *cs = (double *)calloc((size_t)m, sizeof(double));
    cplx *sn = (cplx *)calloc((size_t)m, sizeof(cplx));
    cplx *g = (cplx *)calloc((size_t)m + 1, sizeof(cplx));
    cplx *y = (cplx *)calloc((size_t)m, sizeof(cplx));
    double fn = nrm2(np, f);
    int it = 0, status = 1;
    st->restarts = 0;
    if (fn == 0.0) { memset(x, 0, np * sizeof(cplx)); st->iterations = 0; st->rel_res = 0; st->status = 0; goto done; }
    for (;;) {
        or_residual(A, f, x, w);
        double beta = nrm2(np, w);
        if (beta <= tol * fn) { status = 0; break; }
        if (it >= maxit) break;
        _Pragma("omp parallel for schedule(static)")
        for (size_t p = 0; p < np; p++) V[p] = w[p] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0;
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m && it < maxit; j++) {
            cplx *vj = V + (size_t)j * np, *zj = Z + (size_t)j * np;
            precond(mg, gf, gc, np, vj, zj);
            or_apply(A, zj, w);
            for (int i = 0; i <= j; i++) {
                cplx h = dotc(np, V + (size_t)i * np, w);
                H[i + (size_t)(m + 1) * j] = h;
                _Pragma("omp parallel for schedule(static)")
                for (size_t p = 0; p < np; p++) w[p] -= h * V[(size_t)i * np + p];
            }
            double hn = nrm2(np, w);
            H[j + 1 + (size_t)(m + 1) * j] = hn;
            if (hn != 0.0)
                _Pragma("omp parallel for schedule(static)")
                for (size_t p = 0; p < np; p++) V[(size_t)(j + 1) * np + p] = w[p] / hn;
            /* previous rotations on column j */
            for (int i = 0; i < j; i++) {
                cplx a = H[i + (size_t)(m + 1) * j], b = H[i + 1 + (size_t)(m + 1) * j];
                H[i + (size_t)(m + 1) * j] = cs[i] * a + sn[i] * b;
                H[i + 1 + (size_t)(m + 1) * j] = -conj(sn[i]) * a + cs[i] * b;
            }
            /* new rotation zeroing H[j+1][j]:  G = [c s; -conj(s) c], c real */
            cplx a = H[j + (size_t)(m + 1) * j], b = H[j + 1 + (size_t)(m + 1) * j];
            double t = sqrt(creal(a) * creal(a) + cimag(a) * cimag(a) + creal(b) * creal(b) + cimag(b) * cimag(b));
            if (cabs(a) == 0.0) { cs[j] = 0.0; sn[j] = 1.0; }
            else { cs[j] = cabs(a) / t; sn[j] = (a / cabs(a)) * conj(b) / t; }
            H[j + (size_t)(m + 1) * j] = cs[j] * a + sn[j] * b;
            H[j + 1 + (size_t)(m + 1) * j] = 0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            it++;
            jdone = j + 1;
            double est = cabs(g[j + 1]) / fn;
            if (st->history && it - 1 < st->history_len) st->history[it - 1] = est;
            if (est <= tol || hn == 0.0) break;
        }
        /* y = H^{-1} g (upper triangular jdone x jdone), x += Z y */
        for (int r = jdone - 1; r >= 0; r--) {
            cplx s = g[r];
            for (int c = r + 1; c < jdone; c++) s -= H[r + (size_t)(m + 1) * c] * y[c];
            y[r] = s / H[r + (size_t)(m + 1) * r];
        }
        for (int c = 0; c < jdone; c++)
            _Pragma("omp parallel for schedule(static)")
            for (size_t p = 0; p < np; p++) x[p] += y[c] * Z[(size_t)c * np + p];
        st->restarts++;
    }
    or_residual(A, f, x, w);
    st->rel_res = nrm2(np, w) / fn;
    st->iterations = it;
    st->status = status;
done:
    free(V); free(Z); free(w); free(H); free(cs); free(sn); free(g); free(y);
    return st->status;
}

/* Right-preconditioned Bi-CGSTAB (van der Vorst 1992) with the two preconditioner calls per
 * iteration that Section 5 describes.  Convergence when ||r|| <= tol ||f|| for the
 * recursively updated residual, confirmed by the true residual.  Breakdown (rho = 0 or
 * <rhat, v> = 0 or omega = 0) ends with status 2. */
int or_bicgstab(const or_op *A, const or_mg *mg, int gf, int gc, const cplx *f, cplx *x,
                double tol, int maxit, or_stats *st)
{
    size_t np = npts(A);
    cplx *r = (cplx *)malloc(np * sizeof(cplx)), *rh = (cplx *)malloc(np * sizeof(cplx));
    cplx *p = (cplx *)calloc(np, sizeof(cplx)), *v = (cplx *)calloc(np, sizeof(cplx));
    cplx *y = (cplx *)malloc(np * sizeof(cplx)), *s = (cplx *)malloc(np * sizeof(cplx));
    cplx *z = (cplx *)malloc(np * sizeof(cplx)), *t = (cplx *)malloc(np * sizeof(cplx));
    double fn = nrm2(np, f);
    int status = 1, it = 0;
    st->restarts = 0;
    if (fn == 0.0) { memset(x, 0, np * sizeof(cplx)); status = 0; goto fin; }
    or_residual(A, f, x, r);
    memcpy(rh, r, np * sizeof(cplx));
    cplx rho_old = 1, alpha = 1, om = 1;
    if (nrm2(np, r) <= tol * fn) { status = 0; goto fin; }
    while (it < maxit) {
        cplx rho = dotc(np, rh, r);
        if (rho == 0) { status = 2; break; }
        cplx beta = (rho / rho_old) * (alpha / om);
        _Pragma("omp parallel for schedule(static)")
        for (size_t q = 0; q < np; q++) p[q] = r[q] + beta * (p[q] - om * v[q]);
        precond(mg, gf, gc, np, p, y);
        or_apply(A, y, v);
        cplx rv = dotc(np, rh, v);
        if (rv == 0) { status = 2; break; }
        alpha = rho / rv;
        _Pragma("omp parallel for schedule(static)")
        for (size_t q = 0; q < np; q++) s[q] = r[q] - alpha * v[q];
        it++;
        double sn = nrm2(np, s);
        if (sn <= tol * fn) {
            _Pragma("omp parallel for schedule(static)")
            for (size_t q = 0; q < np; q++) x[q] += alpha * y[q];
            if (st->history && it - 1 < st->history_len) st->history[it - 1] = sn / fn;
            status = 0;
            break;
        }
        precond(mg, gf, gc, np, s, z);
        or_apply(A, z, t);
        double tt = creal(dotc(np, t, t));
        if (tt == 0.0) { status = 2; break; }
        om = dotc(np, t, s) / tt;
        _Pragma("omp parallel for schedule(static)")
        for (size_t q = 0; q < np; q++) {
            x[q] += alpha * y[q] + om * z[q];
            r[q] = s[q] - om * t[q];
        }
        double rn = nrm2(np, r);
        if (st->history && it - 1 < st->history_len) st->history[it - 1] = rn / fn;
        if (rn <= tol * fn) { status = 0; break; }
        if (om == 0) { status = 2; break; }
        rho_old = rho;
    }
fin:
    or_residual(A, f, x, r);
    st->rel_res = fn == 0.0 ? 0.0 : nrm2(np, r) / fn;
    st->iterations = it;
    st->status = status;
    free(r); free(rh); free(p); free(v); free(y); free(s); free(z); free(t);
    return status;
}

/* mg-conv of Section 5: the geometric mean of the residual reduction over the last five of
 * repeated stand-alone cycles u <- MG(u) for M u = b, from u = 0.  Runs until the relative
 * residual is <= tol or maxcyc cycles; returns the number of cycles, writes the factor.
 * Reading (paper silent): tol is 1e-6 by default at the call site. */
int or_mg_conv(const or_mg *mg, int gf, int gc, const cplx *b, double tol, int maxcyc, double *factor,
               double *hist)
{
    const or_op *A = &mg->op[0];
    size_t np = npts(A);
    cplx *u = (cplx *)calloc(np, sizeof(cplx)), *r = (cplx *)malloc(np * sizeof(cplx));
    double bn = nrm2(np, b);
    double *res = (double *)malloc((size_t)(maxcyc + 1) * sizeof(double));
    res[0] = bn;
    int c = 0;
    while (c < maxcyc) {
        or_mg_cycle(mg, b, u, gf, gc);
        c++;
        or_residual(A, b, u, r);
        res[c] = nrm2(np, r);
        if (hist) hist[c - 1] = res[c] / bn;
        if (res[c] <= tol * bn) break;
    }
    int k = c < 5 ? c : 5;
    *factor = k > 0 ? pow(res[c] / res[c - k], 1.0 / k) : 0.0;
    free(u); free(r); free(res);
    return c;
}

/* Dual-volume weights of the FD scheme: W_p = prod_axes (h_{j-1} + h_j)/2 at interior
 * nodes (used to state the complex symmetry of W M; zero on the boundary). */
void or_weights(const or_op *op, cplx *wts)
{
    FOR_NODES_INDEP(op) {
        size_t p = PIDX(op);
        if (!is_interior(op, i, j, k)) { wts[p] = 0; continue; }
        const int idx[3] = {i, j, k};
        cplx w = 1;
        for (int ax = 0; ax < op->dim; ax++) {
            const cplx *z = op->z[ax];
            w *= 0.5 * ((z[idx[ax]] - z[idx[ax] - 1]) + (z[idx[ax] + 1] - z[idx[ax]]));
        }
        wts[p] = w;
    }
}
