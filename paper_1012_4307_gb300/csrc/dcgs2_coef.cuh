// Delayed CGS2 (DCGS2) coefficient step, shared by the stand-alone kernel (kernels_krylov.cu)
// and the fused tail of the two-vector inner-product pass (kernels_gs_df.cu).
#pragma once

#include "helm_internal.h"

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// DCGS2 coefficients of step j (Swirydowicz, Langou, Ananthan, Yang & Thomas,
// "Low synchronization Gram-Schmidt and GMRES algorithms", 2020; Bielich et al. 2022).
// Basis slot j holds x = alpha u: the once-orthogonalised vector of step j - 1, not normalised
// (alpha = alpha2[j].x its norm; slot 0 holds the final v_0 and alpha = 1).  From
// hv[i] = V_i^H x (i <= j; hv[j] = x^H x) and, with has_w, hv[j + 1 + i] = V_i^H w (i <= j):
//   u = sum_{i<j} a_i v_i + nu v_j,  a_i = hv[i] / alpha,  nu = sqrt(hv[j] / alpha^2 - |a|^2)
//   (nu = 1 for j = 0, where slot 0 already holds the final v_0);
//   column j - 1 of H, first-pass entries plus alpha a, gets its final values and
//   H[j][j-1] = alpha nu;
//   column j: c_i = hv[j+1+i] (i < j), H[j][j] = v_j^H w = (hv[2j+1] / alpha - a^H c) / nu;
//   with s = H[j][j] / nu, the update pass forms v_j = (x - sum V_i (alpha a_i)) / (alpha nu)
//   and w' = w - x (s / alpha) - sum V_i (c_i - a_i s): coef[i] = alpha a_i,
//   coef[j+i] = c_i - a_i s, coef[2j] = (1 / (alpha nu), small), coef[2j+1] = s / alpha,
//   where small = 1 when ||alpha a|| <= 2^-18 alpha nu, else 0.
// has_w = 2: the slot j + 1 vector and its inner products come from the unscaled x
// (w' = A M^{-1} x = alpha w, the preconditioner being linear): they are divided by alpha
// here, and coef[2j+2] = (1 / alpha, 0) tells the update pass to scale w' the same way
// (has_w = 1: coef[2j+2] = (1, 0)).
// One warp (lane = threadIdx.x & 31); lane l handles i = l and l + 32 (j <= 64).
__device__ __forceinline__ void dcgs2_coef_warp(int j, int has_w, const double2 *hv, const double2 *alpha2,
                                                double2 *H, int ldh, double2 *coef) {
    const int lane = threadIdx.x & 31;
    const double al = j > 0 ? alpha2[j].x : 1.0, ra = 1.0 / al;
    const double rw = has_w == 2 ? ra : 1.0;
    double2 a[2], c[2];
    double s2 = 0.0, tr = 0.0, ti = 0.0;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int i = lane + 32 * k;
        a[k] = i < j ? hv[i] : make_double2(0.0, 0.0);
        c[k] = (has_w && i < j) ? cscale(hv[j + 1 + i], rw) : make_double2(0.0, 0.0);
        s2 += a[k].x * a[k].x + a[k].y * a[k].y;
        // conj(a) c
        tr += a[k].x * c[k].x + a[k].y * c[k].y;
        ti += a[k].x * c[k].y - a[k].y * c[k].x;
    }
    s2 = warp_sum_d(s2);
    tr = warp_sum_d(tr);
    ti = warp_sum_d(ti);
    double nu = 1.0;
    if (j > 0) {
        nu = sqrt(fmax((hv[j].x - s2) * (ra * ra), 1e-300));
        double2 *col = H + (size_t)ldh * (j - 1);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int i = lane + 32 * k;
            if (i < j) col[i] = cadd(col[i], a[k]);  // alpha a_i = hv[i]
        }
        if (lane == 0) col[j] = make_double2(al * nu, 0.0);
    }
    if (!has_w) return;
    const double2 t = make_double2((hv[2 * j + 1].x * rw - tr) * ra, (hv[2 * j + 1].y * rw - ti) * ra);
    const double rn = 1.0 / nu;
    const double2 hjj = cscale(t, rn);
    const double2 sf = cscale(hjj, rn);
    double2 *col = H + (size_t)ldh * j;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int i = lane + 32 * k;
        if (i < j) {
            col[i] = c[k];
            coef[i] = a[k];
            coef[j + i] = csub(c[k], cmul(cscale(a[k], ra), sf));
        }
    }
    if (lane == 0) {
        col[j] = hjj;
        // small correction (||alpha a|| <= 2^-18 alpha nu): the update may form sum V_i (alpha a_i)
        // in FP32
        const double xn = al * nu;
        coef[2 * j] = make_double2(rn * ra, s2 <= 0x1p-36 * xn * xn ? 1.0 : 0.0);
        coef[2 * j + 1] = cscale(sf, ra);
        coef[2 * j + 2] = make_double2(rw, 0.0);
    }
}

// Last-block-done reduction: every block of a pass has written its partials; the block that
// takes the last ticket (the others return false) reduces them in a fixed order (warp v sums
// value v: lanes over the blocks b = lane, lane + 32, ..., then a fixed shuffle tree) into
// out[0..nvals) and resets the ticket for the next launch.  Deterministic like the separate
// reduction kernel.
__device__ __forceinline__ bool last_block(unsigned *ticket, unsigned nblocks) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == nblocks - 1;
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}
__device__ __forceinline__ void reduce_partials_block(const double2 *partials, int G, int nvals, double2 *out,
                                                      bool sqrt_first) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = warp; v < nvals; v += nw) {
        double sx = 0.0, sy = 0.0;
        for (int b = lane; b < G; b += 32) {
            const double2 p = partials[(size_t)v * G + b];
            sx += p.x;
            sy += p.y;
        }
        sx = warp_sum_d(sx);
        sy = warp_sum_d(sy);
        if (lane == 0) out[v] = sqrt_first ? make_double2(sqrt(sx), 0.0) : make_double2(sx, sy);
    }
}
