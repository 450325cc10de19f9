// Re(lambda0) for the quadrant-definite preconditioner M_QD = (1 - i) I + Z / |Re lambda0|
// (Section 5; eq. (4.1) in table form), where lambda0 is the eigenvalue of Z = -Delta - k^2 with
// the smallest real part.  Section 6 closes with two ways to obtain it without an eigensolve of
// the multidimensional operator: from a one-dimensional counterpart, or roughly as minus the
// largest discrete k^2 for piecewise-constant wavenumbers.  Host code only (setup, no kernels).
//
// One-dimensional counterpart: for a separable k^2(x) = sum_a k2_a(x_a), the discrete Z is the
// Kronecker sum of the 1D operators T_a = L_a - diag(k2_a) (L_a the ECS three-point operator of
// Section 3.2 on axis a), so its eigenvalues are the sums of one eigenvalue of every T_a, and the
// smallest real part is the sum over axes of each T_a's smallest real part.
//
// Eigenvalues of the complex tridiagonal T_a: the diagonal similarity that makes the off-
// diagonal pairs equal (e_j = sqrt(T[j][j+1] T[j+1][j])) gives a complex symmetric tridiagonal
// matrix with the same eigenvalues; its eigenvalues come from the shifted QR iteration with
// complex orthogonal plane rotations (c^2 + s^2 = 1, which keep the matrix complex symmetric and
// tridiagonal; the complex-symmetric QR of Cullum and Willoughby, "Lanczos Algorithms for Large
// Symmetric Eigenvalue Computations", 1985), a Wilkinson shift from the trailing 2 x 2 block and
// deflation at the bottom: O(n) per step, O(n^2) in all.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "helm_internal.h"

typedef std::complex<double> cd;

helm_status helm_fail(helm_status st, const char *fmt, ...);

namespace {

// Eigenvalue of [[a, b], [b, c]] nearer to c.
cd wilkinson(cd a, cd b, cd c) {
    const cd d = 0.5 * (a - c);
    const cd r = std::sqrt(d * d + b * b);
    const cd e1 = 0.5 * (a + c) + r, e2 = 0.5 * (a + c) - r;
    return std::abs(e1 - c) < std::abs(e2 - c) ? e1 : e2;
}

// All eigenvalues of the complex symmetric tridiagonal matrix with diagonal d[0..n) and
// off-diagonal e[0..n-1) (e[i] couples i and i + 1).  Returns false if the iteration does not
// converge (or meets an isotropic rotation vector it cannot step around).
bool cs_tridiag_eigenvalues(std::vector<cd> d, std::vector<cd> e, std::vector<cd> &out) {
    out.clear();
    int n = (int)d.size();
    std::vector<cd> r0(n), r1(n), c(n), s(n);
    const double eps = 1e-15;
    int iters = 0;
    while (n > 0) {
        if (n == 1) {
            out.push_back(d[0]);
            break;
        }
        // deflate at the bottom when the last coupling is negligible
        if (std::abs(e[n - 2]) <= eps * (std::abs(d[n - 2]) + std::abs(d[n - 1]))) {
            out.push_back(d[n - 1]);
            n--;
            iters = 0;
            continue;
        }
        if (++iters > 60) return false;
        // shift: Wilkinson, with an exceptional perturbation now and then
        cd mu = wilkinson(d[n - 2], e[n - 2], d[n - 1]);
        if (iters % 20 == 0) mu += 0.1 * std::abs(e[n - 2]) * cd(1.0, 0.5);
        // T - mu I = Q R: rotations on rows (i, i + 1) zero the coupling below the diagonal;
        // R is upper triangular with two superdiagonals (r0 diagonal, r1 first superdiagonal;
        // the second is not needed for R Q's tridiagonal part)
        cd p = d[0] - mu, q = e[0];
        bool ok = true;
        for (int i = 0; i + 1 < n; i++) {
            const cd b = e[i];
            const cd r = std::sqrt(p * p + b * b);
            if (std::abs(r) <= 1e-300 * (std::abs(p) + std::abs(b) + 1e-300)) {
                ok = false;
                break;
            }
            c[i] = p / r;
            s[i] = b / r;
            r0[i] = r;
            const cd a1 = d[i + 1] - mu;
            r1[i] = c[i] * q + s[i] * a1;
            const cd b1 = i + 2 < n ? e[i + 1] : cd(0.0);
            p = -s[i] * q + c[i] * a1;
            q = c[i] * b1;
        }
        if (!ok) {
            // step around an isotropic vector with a perturbed shift on the next pass
            d[n - 1] += 1e-12 * (std::abs(d[n - 1]) + 1.0);
            continue;
        }
        r0[n - 1] = p;
        // T' = R Q + mu I (complex symmetric tridiagonal)
        for (int i = 0; i < n; i++) {
            const cd cprev = i > 0 ? c[i - 1] : cd(1.0);
            if (i + 1 < n) {
                d[i] = c[i] * cprev * r0[i] + s[i] * r1[i] + mu;
                e[i] = s[i] * r0[i + 1];
            } else {
                d[i] = cprev * r0[i] + mu;
            }
        }
    }
    return true;
}

}  // namespace

// Smallest real part over the eigenvalues of the 1D operator T = L - diag(k2) on the interior
// nodes of one axis (ECS contour of Section 3.1, FD of Section 3.2).
static helm_status axis_lambda0(int n, double lo, double hi, double theta, double r0lo, double r0hi,
                                const double *k2, double *out) {
    const std::vector<cd> z = ecs_contour(n, lo, hi, theta, r0lo, r0hi);
    const std::vector<cd> t = fd_triples(z, 0.0, cd(1.0));
    const int m = n - 2;
    std::vector<cd> d(m), e(m > 0 ? m - 1 : 0);
    for (int j = 1; j <= m; j++) {
        d[j - 1] = t[3 * (size_t)j + 1] - k2[j];
        // T[j][j+1] = ce_j, T[j+1][j] = cw_{j+1}: equal off-diagonals by a diagonal similarity
        if (j < m) e[j - 1] = std::sqrt(t[3 * (size_t)j + 2] * t[3 * (size_t)(j + 1)]);
    }
    std::vector<cd> ev;
    if (!cs_tridiag_eigenvalues(d, e, ev) || ev.empty())
        return helm_fail(HELM_ERR_NOCONV, "eigenvalues of the 1D operator (%d nodes) did not converge", n);
    double best = ev[0].real();
    for (const cd &v : ev) best = std::min(best, v.real());
    *out = best;
    return HELM_OK;
}

extern "C" helm_status helm_qd_lambda0(const helm_grid *grid, double theta, const double *r0_lo,
                                       const double *r0_hi, const double *const *k2_axis, int mode,
                                       double *re_lambda0) {
    if (!grid || !r0_lo || !r0_hi || !k2_axis || !re_lambda0) return helm_fail(HELM_ERR_ARG, "null argument");
    if (grid->dim != 2 && grid->dim != 3) return helm_fail(HELM_ERR_ARG, "dim must be 2 or 3 (got %d)", grid->dim);
    if (mode != HELM_LAMBDA0_AXES && mode != HELM_LAMBDA0_MAX_K2) return helm_fail(HELM_ERR_ARG, "unknown mode %d", mode);
    for (int a = 0; a < grid->dim; a++) {
        if (!k2_axis[a]) return helm_fail(HELM_ERR_ARG, "k2_axis[%d] is null", a);
        if (grid->n[a] < 3 || grid->n[a] > (1 << 16)) return helm_fail(HELM_ERR_ARG, "n[%d] = %d out of range", a, grid->n[a]);
        if (!(grid->hi[a] > grid->lo[a])) return helm_fail(HELM_ERR_ARG, "hi[%d] must exceed lo[%d]", a, a);
        for (int j = 1; j + 1 < grid->n[a]; j++)
            if (!std::isfinite(k2_axis[a][j])) return helm_fail(HELM_ERR_NONFINITE, "k2_axis[%d][%d] is not finite", a, j);
    }
    double sum = 0.0;
    for (int a = 0; a < grid->dim; a++) {
        double v = 0.0;
        if (mode == HELM_LAMBDA0_MAX_K2) {
            // -max k^2 over the interior nodes: the separable field's maximum is the sum of the
            // axes' maxima
            double mx = -INFINITY;
            for (int j = 1; j + 1 < grid->n[a]; j++) mx = std::max(mx, k2_axis[a][j]);
            v = -mx;
        } else {
            try {
                helm_status st = axis_lambda0(grid->n[a], grid->lo[a], grid->hi[a], theta, r0_lo[a], r0_hi[a],
                                              k2_axis[a], &v);
                if (st != HELM_OK) return st;
            } catch (const std::bad_alloc &) {
                return helm_fail(HELM_ERR_NOMEM, "host allocation failed");
            }
        }
        sum += v;
    }
    *re_lambda0 = sum;
    return HELM_OK;
}
