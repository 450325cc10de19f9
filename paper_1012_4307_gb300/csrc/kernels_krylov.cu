// FP64 vector kernels of the outer Krylov solvers (flexible GMRES, Bi-CGSTAB) and the
// adjoint helpers.  All sums use a fixed grid (a function of the vector length only) and a
// fixed reduction tree, so repeated runs give bit-identical results.
//
// Classical Gram-Schmidt runs as two fused passes over the basis:
//   "dot"     h = V^H w and ||w||^2                 (k_mdot_norm, 8 basis vectors per block row)
//   "update"  w <- w - V h and ||w'||^2, same sweep (k_update_norm)
// followed by the DGKS test on the device (k_reduce_decide); the optional second pass reuses
// the same kernels, gated by the device flag, so the host never waits for the decision.
// On GB300 the FP64 units (about 2 FMA per SM per clock) bound these kernels, not DRAM.
#include "helm_internal.h"
#include "df_arith.h"
#include "dcgs2_coef.cuh"

namespace {

constexpr int NT = 256;           // threads per block
constexpr int MAXBLK = 152 * 4;   // grid cap (4 blocks per SM on 152 SMs)

__device__ __forceinline__ double2 shfl_down2(double2 v, int off) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, off);
    v.y = __shfl_down_sync(0xffffffffu, v.y, off);
    return v;
}

// Block-wide sums of NV complex values per thread (fixed tree: warp shuffles, then warps in
// order); thread t < NV returns sum t in out[t] (other threads: unspecified).
template <int NV>
__device__ __forceinline__ void block_sum(double2 (&v)[NV], double2 *out_shared) {
    __shared__ double2 red[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        double2 x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = cadd(x, shfl_down2(x, off));
        if (lane == 0) red[warp][i] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double2 s = red[0][threadIdx.x];
        for (int w = 1; w < NT / 32; w++) s = cadd(s, red[w][threadIdx.x]);
        out_shared[threadIdx.x] = s;
    }
}

// Pass "dot": partials[i * G + b] = sum_q conj(V_i[q]) w[q] for the CH vectors of chunk
// blockIdx.y (i < nv), and chunk 0 also partials[nv * G + b] = (sum |w[q]|^2, 0).
// Grid (G, max(1, ceil(nv / CH))).  Skipped entirely when *gate == 0.
template <int CH>
__global__ void __launch_bounds__(NT) k_mdot_norm(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                  const double2 *__restrict__ w, double2 *__restrict__ partials,
                                                  const int *__restrict__ gate) {
    pdl_enter();
    if (gate && *gate == 0) return;
    __shared__ double2 sums[CH + 1];
    const int i0 = blockIdx.y * CH;
    const int cnt = min(CH, nv - i0);
    const bool first = blockIdx.y == 0;
    double2 acc[CH + 1];
#pragma unroll
    for (int t = 0; t <= CH; t++) acc[t] = make_double2(0.0, 0.0);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 wq = w[q];
        if (first) acc[CH].x = fma(wq.x, wq.x, fma(wq.y, wq.y, acc[CH].x));
#pragma unroll
        for (int t = 0; t < CH; t++)
            if (t < cnt) acc[t] = cfmac(V[(size_t)(i0 + t) * ldv + q], wq, acc[t]);
    }
    block_sum<CH + 1>(acc, sums);
    const int G = gridDim.x;
    if constexpr (CH > 0)
        if (threadIdx.x < CH && (int)threadIdx.x < cnt) partials[(size_t)(i0 + threadIdx.x) * G + blockIdx.x] = sums[threadIdx.x];
    if (first && threadIdx.x == CH) partials[(size_t)nv * G + blockIdx.x] = sums[CH];
}

// Pass "update": w -= sum_{i < nv} V_i h_i, then partials[b] = (sum |w|^2, 0).  Gated.
__global__ void __launch_bounds__(NT) k_update_norm(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                    const double2 *__restrict__ h, double2 *__restrict__ w,
                                                    double2 *__restrict__ partials, const int *__restrict__ gate) {
    pdl_enter();
    if (gate && *gate == 0) return;
    __shared__ double2 hs[64];
    __shared__ double2 sums[1];
    for (int i = threadIdx.x; i < nv; i += NT) hs[i] = h[i];
    __syncthreads();
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        double2 wq = w[q];
#pragma unroll 8
        for (int i = 0; i < nv; i++) {
            const double2 v = V[(size_t)i * ldv + q];
            const double2 hh = hs[i];
            wq.x = fma(-v.x, hh.x, fma(v.y, hh.y, wq.x));
            wq.y = fma(-v.x, hh.y, fma(-v.y, hh.x, wq.y));
        }
        w[q] = wq;
        acc[0].x = fma(wq.x, wq.x, fma(wq.y, wq.y, acc[0].x));
    }
    block_sum<1>(acc, sums);
    if (threadIdx.x == 0) partials[blockIdx.x] = sums[0];
}

// out[i] = sum_b partials[i * nblk + b] in a fixed order for i = blockIdx.x; mode 0 '=',
// 1 '+=', 2 (sqrt(re), 0).  Gated.
__global__ void k_reduce(const double2 *__restrict__ partials, int nblk, double2 *__restrict__ out, int mode,
                         const int *__restrict__ gate, double *host_out) {
    pdl_enter();
    if (gate && *gate == 0) return;
    __shared__ double2 sums[1];
    const int i = blockIdx.x;
    double2 s[1] = {make_double2(0.0, 0.0)};
    for (int b = threadIdx.x; b < nblk; b += NT) s[0] = cadd(s[0], partials[(size_t)i * nblk + b]);
    block_sum<1>(s, sums);
    if (threadIdx.x == 0) {
        const double2 t = sums[0];
        double2 r;
        if (mode == 0) r = t;
        else if (mode == 1) r = cadd(out[i], t);
        else r = make_double2(sqrt(t.x), 0.0);
        out[i] = r;
        if (host_out) host_out[i] = r.x;
    }
}

// DGKS test after one classical Gram-Schmidt pass: the new norm ||w'|| = sqrt(sum partials)
// is written to *hnorm (which held ||w||^2 before the pass); re-orthogonalise (*flag = 1) when
// ||w'|| < eta ||w||, i.e. when the projection cancelled most of w.
__global__ void k_reduce_decide(const double2 *__restrict__ partials, int nblk, double2 *hnorm, int *flag, int *count,
                                double eta) {
    pdl_enter();
    __shared__ double2 sums[1];
    double2 s[1] = {make_double2(0.0, 0.0)};
    for (int b = threadIdx.x; b < nblk; b += NT) s[0] = cadd(s[0], partials[b]);
    block_sum<1>(s, sums);
    if (threadIdx.x == 0) {
        const double before = sqrt(hnorm->x), after = sqrt(sums[0].x);
        const int redo = !(after >= eta * before);
        *flag = redo;
        if (redo) *count += 1;
        *hnorm = make_double2(after, 0.0);
    }
}

__global__ void k_scale_inv(size_t n, const double2 *x, const double2 *__restrict__ scale, double2 *y) {
    pdl_enter();
    const double s = scale[0].x;
    const double r = s != 0.0 ? 1.0 / s : 0.0;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 v = x[q];
        y[q] = make_double2(v.x * r, v.y * r);
    }
}

template <typename CZ>
__global__ void k_combine(size_t n, const CZ *__restrict__ Z, size_t ldz, int nz, const double2 *__restrict__ y,
                          double2 *__restrict__ x) {
    pdl_enter();
    __shared__ double2 ys[64];
    for (int i = threadIdx.x; i < nz; i += NT) ys[i] = y[i];
    __syncthreads();
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        double2 acc = x[q];
        for (int c = 0; c < nz; c++) acc = cfma(ys[c], to_c(Z[(size_t)c * ldz + q], 0.0), acc);
        x[q] = acc;
    }
}

// x += Z y for complex64 Z: the sum over the basis in double-FP32 on the FP32 units (products
// of the exact FP32 z with y split into float pairs are error-free, sums use TwoSum), added to
// x in FP64 once per node.  The FP64 form above is bound by the FP64 units (4 FMA per vector
// and node).
// With alpha, column c >= 1 of Z holds alpha_c z_c (alpha_c = alpha[c].x) and its weight is
// y_c / alpha_c.
__global__ void __launch_bounds__(NT) k_combine_df(size_t n, const float2 *__restrict__ Z, size_t ldz, int nz,
                                                   const double2 *__restrict__ y, const double2 *__restrict__ alpha,
                                                   double2 *__restrict__ x) {
    pdl_enter();
    __shared__ float4 ys[64];  // (re hi, re lo, im hi, im lo)
    for (int i = threadIdx.x; i < nz; i += NT) {
        const double r = (alpha && i > 0) ? 1.0 / alpha[i].x : 1.0;
        const ff a = ff_split(y[i].x * r), b = ff_split(y[i].y * r);
        ys[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    __syncthreads();
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll 4
        for (int c = 0; c < nz; c++) {
            const float2 z = Z[(size_t)c * ldz + q];
            const float4 y4 = ys[c];
            const ff yr{y4.x, y4.y}, yi{y4.z, y4.w};
            float p, e;
            // re += zr yr - zi yi ; im += zr yi + zi yr
            ff_prod_f(yr, z.x, p, e); ff_acc_prod(sr, cr, p, e);
            ff_prod_f(yi, z.y, p, e); ff_acc_prod(sr, cr, -p, -e);
            ff_prod_f(yi, z.x, p, e); ff_acc_prod(si, ci, p, e);
            ff_prod_f(yr, z.y, p, e); ff_acc_prod(si, ci, p, e);
        }
        const double2 xq = x[q];
        x[q] = make_double2(xq.x + ((double)sr + (double)cr), xq.y + ((double)si + (double)ci));
    }
}

// Complex Givens rotations G = [c s; -conj(s) c] (c real) on column j of the Hessenberg
// matrix (column-major, leading dimension ldh); see Saad, Iterative Methods for Sparse Linear
// Systems, Section 6.5.9 for the real case.
// Called by one warp: the lanes stage column j of H (j + 2 entries) and the earlier rotations in
// shared memory, lane 0 applies the rotations in order and forms the new one, the lanes write the
// column back.  The arithmetic is that of a single thread walking the column in global memory.
// est_host (may be null): pinned host memory, where est[j] is also stored, so that the host reads
// the estimate once the step's event has fired, with no copy in the step (a device-to-host copy
// node cost about 7 us per step at the end of every replayed step graph).
// tol, stop (may be null): *stop = 1 when est[j] <= *tol or is not a number.
__device__ __forceinline__ void givens_body(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g,
                                            const double2 *fnorm_dev, double *est, double *est_host = nullptr,
                                            const double *tol = nullptr, int *stop = nullptr) {
    __shared__ double2 colS[66], snS[64];
    __shared__ double csS[64];
    const int lane = threadIdx.x & 31;
    double2 *col = H + (size_t)ldh * j;
    for (int i = lane; i <= j + 1; i += 32) colS[i] = col[i];
    for (int i = lane; i < j; i += 32) {
        csS[i] = cs[i];
        snS[i] = sn[i];
    }
    __syncwarp();
    if (lane == 0) {
        const double fnorm = fnorm_dev->x;
        for (int i = 0; i < j; i++) {
            const double2 a = colS[i], b = colS[i + 1];
            const double c = csS[i];
            const double2 s = snS[i];
            colS[i] = cadd(cscale(a, c), cmul(s, b));
            colS[i + 1] = csub(cscale(b, c), cmul(make_double2(s.x, -s.y), a));
        }
        const double2 a = colS[j], b = colS[j + 1];
        const double na = hypot(a.x, a.y);
        const double t = hypot(na, hypot(b.x, b.y));
        double c;
        double2 s;
        if (na == 0.0) {
            c = 0.0;
            s = make_double2(1.0, 0.0);
        } else {
            c = na / t;
            const double2 ua = make_double2(a.x / na, a.y / na);
            s = cscale(cmul(ua, make_double2(b.x, -b.y)), 1.0 / t);
        }
        cs[j] = c;
        sn[j] = s;
        colS[j] = cadd(cscale(a, c), cmul(s, b));
        colS[j + 1] = make_double2(0.0, 0.0);
        const double2 gj = g[j];
        g[j + 1] = cscale(cmul(make_double2(-s.x, s.y), gj), 1.0);
        g[j] = cscale(gj, c);
        est[j] = hypot(g[j + 1].x, g[j + 1].y) / fnorm;
        if (est_host) est_host[j] = est[j];
        if (stop && !(est[j] > *tol)) *stop = 1;
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += 32) col[i] = colS[i];
}

__global__ void k_givens(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g, const double2 *fnorm_dev,
                         double *est, double *est_host, const double *tol, int *stop) {
    pdl_enter();
    if (threadIdx.x >= 32 || blockIdx.x != 0) return;
    givens_body(H, ldh, j, cs, sn, g, fnorm_dev, est, est_host, tol, stop);
}

__global__ void k_cycle_start(double2 *g, int len, const double2 *beta, int *stop, double *tol_dev, double tol) {
    pdl_enter();
    for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = i == 0 ? *beta : make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        if (stop) *stop = 0;
        if (tol_dev) *tol_dev = tol;
    }
}

// Batched rotation of column j (block z = problem), and the gather of every problem's estimate
// est[j] into out[problem] (-1 for inactive problems); out is pinned host memory, which the host
// reads once the step's event has fired.  A problem whose estimate meets *tol (or is not a
// number) is made inactive at once, so that the steps already queued behind this one skip it
// (the host, reading the same estimate, takes it out of the lockstep).
__global__ void k_givens_b(const BVec *__restrict__ tab, int j, double *out, const double *tol) {
    pdl_enter();
    const BVec &P = tab[blockIdx.z];
    if (threadIdx.x >= 32) return;
    if (*P.active == 0) {
        if (threadIdx.x == 0) out[blockIdx.z] = -1.0;
        return;
    }
    givens_body(P.H, P.ldh, j, P.cs, P.sn, P.g, P.fnorm, P.est);
    if (threadIdx.x == 0) {
        const double e = P.est[j];
        out[blockIdx.z] = e;
        if (tol && !(e > *tol)) *P.active = 0;
    }
}

// The reduction of the two-vector inner-product pass (block v sums value v of the partials in
// the fixed order of k_reduce) followed, in the last block to finish, by the DCGS2 coefficient
// step of step j (see dcgs2_coef.cuh); the ticket returns to 0.
__device__ __forceinline__ void reduce_dcgs2_body(const double2 *__restrict__ partials, int nblk, double2 *hv,
                                                  unsigned *ticket, int j, const double2 *alpha2, double2 *H, int ldh,
                                                  double2 *coef, int has_w) {
    __shared__ double2 sums[1];
    const int i = blockIdx.x;
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (int b = threadIdx.x; b < nblk; b += NT) acc[0] = cadd(acc[0], partials[(size_t)i * nblk + b]);
    block_sum<1>(acc, sums);
    if (threadIdx.x == 0) hv[i] = sums[0];
    if (!last_block(ticket, gridDim.x)) return;
    if (threadIdx.x < 32) dcgs2_coef_warp(j, has_w, hv, alpha2, H, ldh, coef);
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void k_reduce_dcgs2(const double2 *__restrict__ partials, int nblk, double2 *hv, unsigned *ticket, int j,
                               const double2 *alpha2, double2 *H, int ldh, double2 *coef, int has_w) {
    pdl_enter();
    reduce_dcgs2_body(partials, nblk, hv, ticket, j, alpha2, H, ldh, coef, has_w);
}

// Batched reduction + coefficient step of step j (block z = problem; the problem's dot pass
// had first[z + 1] - first[z] blocks, i.e. that many / groups per value).
__global__ void k_reduce_dcgs2_b(const BVec *__restrict__ tab, const unsigned *__restrict__ first, int groups, int j,
                                 int has_w) {
    pdl_enter();
    const BVec &P = tab[blockIdx.z];
    if (*P.active == 0) return;
    const int nblk = (int)((first[blockIdx.z + 1] - first[blockIdx.z]) / groups);
    reduce_dcgs2_body(P.partials, nblk, P.hv, P.tickets, j, P.alpha2, P.H, P.ldh, P.dcoef, has_w);
}

// DCGS2 coefficient step as its own launch (one warp); see dcgs2_coef.cuh.
__global__ void k_dcgs2_coef(int j, int has_w, const double2 *__restrict__ hv, const double2 *__restrict__ alpha2,
                             double2 *__restrict__ H, int ldh, double2 *__restrict__ coef) {
    pdl_enter();
    dcgs2_coef_warp(j, has_w, hv, alpha2, H, ldh, coef);
}

// y = R^{-1} g for the k x k upper-triangular leading block R of H (column-major, leading
// dimension ldh): R and g are staged in shared memory by the whole block, then one warp
// eliminates column by column (y_r = g_r / R_rr, then g_i -= R_ir y_r for i < r, lanes over i),
// with the reciprocals 1 / R_rr formed beforehand in parallel.
__global__ void __launch_bounds__(NT) k_backsolve(const double2 *H, int ldh, int k, const double2 *g, double2 *y) {
    pdl_enter();
    extern __shared__ double2 bs_smem[];
    double2 *R = bs_smem, *gs = bs_smem + (size_t)k * k;
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
        const int c = q / k, r = q - c * k;
        R[q] = r <= c ? H[r + (size_t)ldh * c] : make_double2(0.0, 0.0);
    }
    for (int q = threadIdx.x; q < k; q += blockDim.x) gs[q] = g[q];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    // the reciprocal diagonal first, all lanes at once; the elimination then only multiplies
    for (int r = lane; r < k; r += 32) R[r + (size_t)k * r] = cinv(R[r + (size_t)k * r]);
    __syncwarp();
    for (int r = k - 1; r >= 0; r--) {
        const double2 yr = cmul(gs[r], R[r + (size_t)k * r]);
        for (int i = lane; i < r; i += 32) gs[i] = csub(gs[i], cmul(R[i + (size_t)k * r], yr));
        if (lane == 0) y[r] = yr;
        __syncwarp();
    }
}

// Bi-CGSTAB scalar block (device): 0 rho, 1 rho_old, 2 alpha, 3 omega, 4 beta, 5 <rh,v>,
// 6 <t,s>, 7 <t,t>, 8 -alpha, 9 -omega, 10 one, 11 flags (x: breakdown)
__global__ void k_bicg_scalars(int stage, double2 *sc) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double2 zero = make_double2(0.0, 0.0);
    auto isz = [](double2 v) { return v.x == 0.0 && v.y == 0.0; };
    if (stage == 0) {            // beta = (rho / rho_old) (alpha / omega)
        if (isz(sc[0]) || isz(sc[1]) || isz(sc[3])) { sc[11].x = 1.0; sc[4] = zero; return; }
        sc[4] = cmul(cmul(sc[0], cinv(sc[1])), cmul(sc[2], cinv(sc[3])));
    } else if (stage == 1) {     // alpha = rho / <rh, v>
        if (isz(sc[5])) { sc[11].x = 1.0; sc[2] = zero; sc[8] = zero; return; }
        sc[2] = cmul(sc[0], cinv(sc[5]));
        sc[8] = make_double2(-sc[2].x, -sc[2].y);
    } else if (stage == 2) {     // omega = <t, s> / <t, t>; rho_old = rho
        if (sc[7].x == 0.0) { sc[11].x = 1.0; sc[3] = zero; sc[9] = zero; return; }
        sc[3] = cscale(sc[6], 1.0 / sc[7].x);
        sc[9] = make_double2(-sc[3].x, -sc[3].y);
        sc[1] = sc[0];
        if (isz(sc[3])) sc[11].x = 1.0;
    } else {                     // init: rho_old = alpha = omega = 1, flags = 0
        sc[1] = sc[2] = sc[3] = sc[10] = make_double2(1.0, 0.0);
        sc[11] = zero;
    }
}

__global__ void k_bicg_p(size_t n, const double2 *__restrict__ r, const double2 *__restrict__ v,
                         const double2 *__restrict__ sc, double2 *__restrict__ p) {
    pdl_enter();
    const double2 beta = sc[4], om = sc[3];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 t = csub(p[q], cmul(om, v[q]));
        p[q] = cfma(beta, t, r[q]);
    }
}

__global__ void k_axpby(size_t n, const double2 *__restrict__ a, const double2 *__restrict__ x,
                        const double2 *__restrict__ b, double2 *__restrict__ y) {
    pdl_enter();
    const double2 av = a[0], bv = b[0];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT)
        y[q] = cfma(av, x[q], cmul(bv, y[q]));
}

template <typename CY>
__global__ void k_axpy_mixed(size_t n, const double2 *__restrict__ a, const CY *__restrict__ x, double2 *__restrict__ y) {
    pdl_enter();
    const double2 av = a[0];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT)
        y[q] = cfma(av, to_c(x[q], 0.0), y[q]);
}

// y = W x or W^{-1} x, W_p = prod_axes w_axis[a][i_a] on interior nodes (boundary left).
// y = w x (inverse: x / w) on interior nodes, w the product of the axes' dual volumes;
// conj_x: x is conjugated first.
__global__ void k_weight(int nx, int ny, int nz, int dim, const double2 *__restrict__ wx,
                         const double2 *__restrict__ wy, const double2 *__restrict__ wz, int inverse, int conj_x,
                         const double2 *__restrict__ x, double2 *__restrict__ y) {
    pdl_enter();
    const size_t n = (size_t)nx * ny * nz;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((size_t)nx * ny));
        if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || (dim == 3 && (k < 1 || k > nz - 2))) continue;
        double2 w = cmul(wx[i], wy[j]);
        if (dim == 3) w = cmul(w, wz[k]);
        if (inverse) w = cinv(w);
        double2 v = x[q];
        if (conj_x) v.y = -v.y;
        y[q] = cmul(w, v);
    }
}

// Gradients of a real loss after the adjoint solve: lambda = w y (w as in k_weight) at interior
// nodes; grad_k2 = Re(lambda u) (null: skipped) and grad_f = conj(lambda) (null: skipped),
// both 0 on the boundary.
__global__ void k_adjoint_grads(int nx, int ny, int nz, int dim, const double2 *__restrict__ wx,
                                const double2 *__restrict__ wy, const double2 *__restrict__ wz,
                                const double2 *__restrict__ y, const double2 *__restrict__ u,
                                double *__restrict__ grad_k2, double2 *__restrict__ grad_f) {
    pdl_enter();
    const size_t n = (size_t)nx * ny * nz;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((size_t)nx * ny));
        const bool in = !(i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || (dim == 3 && (k < 1 || k > nz - 2)));
        double2 lam = make_double2(0.0, 0.0);
        if (in) {
            double2 w = cmul(wx[i], wy[j]);
            if (dim == 3) w = cmul(w, wz[k]);
            lam = cmul(w, y[q]);
        }
        if (grad_k2) {
            const double2 b = u[q];
            grad_k2[q] = in ? (lam.x * b.x - lam.y * b.y) : 0.0;
        }
        if (grad_f) grad_f[q] = make_double2(lam.x, -lam.y);
    }
}

__global__ void k_grad_k2(int nx, int ny, int nz, int dim, const double2 *__restrict__ lam,
                          const double2 *__restrict__ u, double *__restrict__ grad) {
    pdl_enter();
    const size_t n = (size_t)nx * ny * nz;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((size_t)nx * ny));
        const bool in = !(i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || (dim == 3 && (k < 1 || k > nz - 2)));
        const double2 a = lam[q], b = u[q];
        grad[q] = in ? (a.x * b.x - a.y * b.y) : 0.0;
    }
}

unsigned stream_grid(size_t n) { return (unsigned)std::min<size_t>(cdiv(n, NT), (size_t)152 * 8); }

}  // namespace

int blas_nblocks(size_t n) { return (int)std::min<size_t>(cdiv(n, NT), (size_t)MAXBLK); }

cudaError_t launch_mdot_norm(size_t n, const double2 *V, size_t ldv, int nv, const double2 *w, double2 *partials,
                             const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    if (nv == 0) {  // the norm alone: one value per block to reduce, not CH + 1
        launch_pdl(k_mdot_norm<0>, dim3(blas_nblocks(n), 1), NT, 0, s, n, V, ldv, nv, w, partials, gate);
        return cudaGetLastError();
    }
    constexpr int CH = 8;
    dim3 g(blas_nblocks(n), std::max(1, (nv + CH - 1) / CH));
    launch_pdl(k_mdot_norm<CH>, g, NT, 0, s, n, V, ldv, nv, w, partials, gate);
    return cudaGetLastError();
}

cudaError_t launch_update_norm(size_t n, const double2 *V, size_t ldv, int nv, const double2 *h, double2 *w,
                               double2 *partials, const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    launch_pdl(k_update_norm, blas_nblocks(n), NT, 0, s, n, V, ldv, nv, h, w, partials, gate);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double2 *partials, int nblk, int nv, double2 *out, int mode, const int *gate,
                          cudaStream_t s, double *host_out) {
    launch_pdl(k_reduce, nv, NT, 0, s, partials, nblk, out, mode, gate, host_out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_decide(const double2 *partials, int nblk, double2 *hnorm, int *flag, int *count, double eta,
                                 cudaStream_t s) {
    launch_pdl(k_reduce_decide, 1, NT, 0, s, partials, nblk, hnorm, flag, count, eta);
    return cudaGetLastError();
}

cudaError_t launch_scale_inv(size_t n, const double2 *x, const double2 *scale, double2 *y, cudaStream_t s) {
    launch_pdl(k_scale_inv, stream_grid(n), NT, 0, s, n, x, scale, y);
    return cudaGetLastError();
}

template <typename CZ>
cudaError_t launch_combine(size_t n, const CZ *Z, size_t ldz, int nz, const double2 *y, const double2 *alpha,
                           double2 *x, cudaStream_t s) {
    if (nz > 64) return cudaErrorInvalidValue;
    if constexpr (sizeof(CZ) == sizeof(float2)) {
        launch_pdl(k_combine_df, stream_grid(n), NT, 0, s, n, (const float2 *)Z, ldz, nz, y, alpha, x);
    } else {
        if (alpha) return cudaErrorInvalidValue;
        launch_pdl(k_combine<CZ>, stream_grid(n), NT, 0, s, n, Z, ldz, nz, y, x);
    }
    return cudaGetLastError();
}
template cudaError_t launch_combine<float2>(size_t, const float2 *, size_t, int, const double2 *, const double2 *,
                                            double2 *, cudaStream_t);
template cudaError_t launch_combine<double2>(size_t, const double2 *, size_t, int, const double2 *, const double2 *,
                                             double2 *, cudaStream_t);

cudaError_t launch_givens(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g, const double2 *fnorm,
                          double *est, double *est_host, const double *tol, int *stop, cudaStream_t s) {
    if (stop && !tol) return cudaErrorInvalidValue;
    k_givens<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, g, fnorm, est, est_host, tol, stop);
    return cudaGetLastError();
}

cudaError_t launch_cycle_start(double2 *g, int len, const double2 *beta, int *stop, double *tol_dev, double tol,
                               cudaStream_t s) {
    if (len < 1) return cudaErrorInvalidValue;
    launch_pdl(k_cycle_start, 1, NT, 0, s, g, len, beta, stop, tol_dev, tol);
    return cudaGetLastError();
}

cudaError_t launch_reduce_dcgs2(const double2 *partials, int nblk, double2 *hv, unsigned *ticket, int j,
                                const double2 *alpha2, double2 *H, int ldh, double2 *coef, int has_w,
                                cudaStream_t s) {
    if (j < 0 || j > 64 || has_w < 0 || has_w > 2) return cudaErrorInvalidValue;
    launch_pdl(k_reduce_dcgs2, 2 * (j + 1), NT, 0, s, partials, nblk, hv, ticket, j, alpha2, H, ldh, coef, has_w);
    return cudaGetLastError();
}

cudaError_t launch_reduce_dcgs2_batch(int count, const BVec *tab, const unsigned *first, int groups, int j,
                                      int has_w, cudaStream_t s) {
    if (count < 1 || count > 65535 || j < 0 || j > 64 || groups < 1 || has_w < 0 || has_w > 2)
        return cudaErrorInvalidValue;
    launch_pdl(k_reduce_dcgs2_b, dim3(2 * (j + 1), 1, count), NT, 0, s, tab, first, groups, j, has_w);
    return cudaGetLastError();
}

cudaError_t launch_givens_batch(int count, const BVec *tab, int j, double *est_out, const double *tol, cudaStream_t s) {
    if (count < 1 || count > 65535 || j < 0 || j > 63) return cudaErrorInvalidValue;
    launch_pdl(k_givens_b, dim3(1, 1, count), 32, 0, s, tab, j, est_out, tol);
    return cudaGetLastError();
}

cudaError_t launch_dcgs2_coef(int j, int has_w, const double2 *hv, const double2 *alpha2, double2 *H, int ldh,
                              double2 *coef, cudaStream_t s) {
    if (j < 0 || j > 64) return cudaErrorInvalidValue;
    launch_pdl(k_dcgs2_coef, 1, 32, 0, s, j, has_w, hv, alpha2, H, ldh, coef);
    return cudaGetLastError();
}

cudaError_t launch_backsolve(const double2 *H, int ldh, int k, const double2 *g, double2 *y, cudaStream_t s) {
    if (k < 1 || k > 64 || ldh < k) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)((64 * 64 + 64) * sizeof(double2)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    launch_pdl(k_backsolve, 1, NT, (size_t)(k * k + k) * sizeof(double2), s, H, ldh, k, g, y);
    return cudaGetLastError();
}

cudaError_t launch_bicg_scalars(int stage, double2 *sc, cudaStream_t s) {
    launch_pdl(k_bicg_scalars, 1, 32, 0, s, stage, sc);
    return cudaGetLastError();
}

cudaError_t launch_bicg_p(size_t n, const double2 *r, const double2 *v, const double2 *sc, double2 *p,
                          cudaStream_t s) {
    launch_pdl(k_bicg_p, stream_grid(n), NT, 0, s, n, r, v, sc, p);
    return cudaGetLastError();
}

cudaError_t launch_axpby(size_t n, const double2 *a, const double2 *x, const double2 *b, double2 *y,
                         cudaStream_t s) {
    launch_pdl(k_axpby, stream_grid(n), NT, 0, s, n, a, x, b, y);
    return cudaGetLastError();
}

template <typename CY>
cudaError_t launch_axpy_mixed(size_t n, const double2 *a, const CY *x, double2 *y, cudaStream_t s) {
    launch_pdl(k_axpy_mixed<CY>, stream_grid(n), NT, 0, s, n, a, x, y);
    return cudaGetLastError();
}
template cudaError_t launch_axpy_mixed<float2>(size_t, const double2 *, const float2 *, double2 *, cudaStream_t);
template cudaError_t launch_axpy_mixed<double2>(size_t, const double2 *, const double2 *, double2 *, cudaStream_t);

cudaError_t launch_weight(size_t n, const int nodes[3], int dim, const double2 *w_axis[3], int inverse,
                          const double2 *x, double2 *y, cudaStream_t s, int conj_x) {
    launch_pdl(k_weight, stream_grid(n), NT, 0, s, nodes[0], nodes[1], dim == 3 ? nodes[2] : 1, dim, w_axis[0], w_axis[1],
                                           w_axis[2], inverse, conj_x, x, y);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grads(size_t n, const int nodes[3], int dim, const double2 *w_axis[3], const double2 *y,
                                 const double2 *u, double *grad_k2, double2 *grad_f, cudaStream_t s) {
    launch_pdl(k_adjoint_grads, stream_grid(n), NT, 0, s, nodes[0], nodes[1], dim == 3 ? nodes[2] : 1, dim, w_axis[0],
               w_axis[1], w_axis[2], y, u, grad_k2, grad_f);
    return cudaGetLastError();
}

cudaError_t launch_grad_k2(size_t n, const int nodes[3], int dim, const double2 *lam, const double2 *u,
                           double *grad, cudaStream_t s) {
    launch_pdl(k_grad_k2, stream_grid(n), NT, 0, s, nodes[0], nodes[1], dim == 3 ? nodes[2] : 1, dim, lam, u, grad);
    return cudaGetLastError();
}
