// FP64 vector kernels of the outer Krylov solvers (flexible GMRES, Bi-CGSTAB) and the
// adjoint helpers.  All sums use a fixed grid (a function of the vector length only) and a
// fixed reduction tree, so repeated runs give bit-identical results.
//
// Classical Gram-Schmidt with one re-orthogonalisation (CGS2) is done in three passes over
// the basis instead of four:
//   pass 1  h1 = V^H w                                   (k_mdot)
//   pass 2  w <- w - V h1, then h2 = V^H w, same sweep   (k_update_mdot)
//   pass 3  w <- w - V h2, then ||w||^2, same sweep      (k_update_norm)
// Every thread owns one node at a time and keeps one accumulator per basis vector in
// registers (MAXV buckets), so w is read once per pass and V once per pass from DRAM.
#include "helm_internal.h"

namespace {

constexpr int NT = 256;           // threads per block
constexpr int MAXBLK = 152 * 4;   // grid cap (4 blocks per SM on 152 SMs)

__device__ __forceinline__ double2 shfl_down2(double2 v, int off) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, off);
    v.y = __shfl_down_sync(0xffffffffu, v.y, off);
    return v;
}

// Reduce acc[0..nv) over the block; thread 0 of warp 0 writes partials[i * nblk + blockIdx.x].
template <int MAXV>
__device__ __forceinline__ void block_store(double2 (&acc)[MAXV], int nv, double2 *partials) {
    __shared__ double2 red[NT / 32][MAXV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < MAXV; i++) {
        if (i < nv) {
            double2 v = acc[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v = cadd(v, shfl_down2(v, off));
            if (lane == 0) red[warp][i] = v;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += NT) {
        double2 s = red[0][i];
        for (int w = 1; w < NT / 32; w++) s = cadd(s, red[w][i]);
        partials[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
}

template <int MAXV>
__global__ void __launch_bounds__(NT) k_mdot(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                             const double2 *__restrict__ w, double2 *__restrict__ partials) {
    double2 acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; i++) acc[i] = make_double2(0.0, 0.0);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 wq = w[q];
#pragma unroll
        for (int i = 0; i < MAXV; i++)
            if (i < nv) acc[i] = cfmac(V[(size_t)i * ldv + q], wq, acc[i]);
    }
    block_store<MAXV>(acc, nv, partials);
}

template <int MAXV>
__global__ void __launch_bounds__(NT) k_update_mdot(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                    const double2 *__restrict__ h, double2 *__restrict__ w,
                                                    double2 *__restrict__ partials) {
    __shared__ double2 hs[MAXV];
    for (int i = threadIdx.x; i < nv; i += NT) hs[i] = h[i];
    __syncthreads();
    double2 acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; i++) acc[i] = make_double2(0.0, 0.0);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        double2 wq = w[q];
#pragma unroll
        for (int i = 0; i < MAXV; i++)
            if (i < nv) {
                const double2 v = V[(size_t)i * ldv + q];
                const double2 hh = hs[i];
                wq = make_double2(wq.x - (v.x * hh.x - v.y * hh.y), wq.y - (v.x * hh.y + v.y * hh.x));
            }
        w[q] = wq;
#pragma unroll
        for (int i = 0; i < MAXV; i++)
            if (i < nv) acc[i] = cfmac(V[(size_t)i * ldv + q], wq, acc[i]);
    }
    block_store<MAXV>(acc, nv, partials);
}

template <int MAXV>
__global__ void __launch_bounds__(NT) k_update_norm(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                    const double2 *__restrict__ h, double2 *__restrict__ w,
                                                    double2 *__restrict__ partials) {
    __shared__ double2 hs[MAXV];
    for (int i = threadIdx.x; i < nv; i += NT) hs[i] = h[i];
    __syncthreads();
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        double2 wq = w[q];
#pragma unroll
        for (int i = 0; i < MAXV; i++)
            if (i < nv) {
                const double2 v = V[(size_t)i * ldv + q];
                const double2 hh = hs[i];
                wq = make_double2(wq.x - (v.x * hh.x - v.y * hh.y), wq.y - (v.x * hh.y + v.y * hh.x));
            }
        w[q] = wq;
        acc[0].x = fma(wq.x, wq.x, fma(wq.y, wq.y, acc[0].x));
    }
    block_store<1>(acc, 1, partials);
}

// out[i] = sum_b partials[i * nblk + b] in a fixed order; mode 0 '=', 1 '+=', 2 sqrt(re).
__global__ void k_reduce(const double2 *__restrict__ partials, int nblk, double2 *__restrict__ out, int mode) {
    __shared__ double2 red[NT / 32];
    const int i = blockIdx.x;
    double2 s = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblk; b += NT) s = cadd(s, partials[(size_t)i * nblk + b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = cadd(s, shfl_down2(s, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = red[0];
        for (int w = 1; w < NT / 32; w++) t = cadd(t, red[w]);
        if (mode == 0) out[i] = t;
        else if (mode == 1) out[i] = cadd(out[i], t);
        else out[i] = make_double2(sqrt(t.x), 0.0);
    }
}

__global__ void k_scale_inv(size_t n, const double2 *x, const double2 *__restrict__ scale, double2 *y) {
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
    __shared__ double2 ys[64];
    for (int i = threadIdx.x; i < nz; i += NT) ys[i] = y[i];
    __syncthreads();
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        double2 acc = x[q];
        for (int c = 0; c < nz; c++) acc = cfma(ys[c], to_c(Z[(size_t)c * ldz + q], 0.0), acc);
        x[q] = acc;
    }
}

// Complex Givens rotations G = [c s; -conj(s) c] (c real) on column j of the Hessenberg
// matrix (column-major, leading dimension ldh); see Saad, Iterative Methods for Sparse Linear
// Systems, Section 6.5.9 for the real case.
__global__ void k_givens(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g, double fnorm,
                         double *est) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 *col = H + (size_t)ldh * j;
    for (int i = 0; i < j; i++) {
        const double2 a = col[i], b = col[i + 1];
        const double c = cs[i];
        const double2 s = sn[i];
        col[i] = cadd(cscale(a, c), cmul(s, b));
        col[i + 1] = csub(cscale(b, c), cmul(make_double2(s.x, -s.y), a));
    }
    const double2 a = col[j], b = col[j + 1];
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
    col[j] = cadd(cscale(a, c), cmul(s, b));
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    g[j + 1] = cscale(cmul(make_double2(-s.x, s.y), gj), 1.0);
    g[j] = cscale(gj, c);
    est[0] = hypot(g[j + 1].x, g[j + 1].y) / fnorm;
}

__global__ void k_backsolve(const double2 *H, int ldh, int k, const double2 *g, double2 *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int r = k - 1; r >= 0; r--) {
        double2 s = g[r];
        for (int c = r + 1; c < k; c++) s = csub(s, cmul(H[r + (size_t)ldh * c], y[c]));
        y[r] = cmul(s, cinv(H[r + (size_t)ldh * r]));
    }
}

// Bi-CGSTAB scalar block (device): 0 rho, 1 rho_old, 2 alpha, 3 omega, 4 beta, 5 <rh,v>,
// 6 <t,s>, 7 <t,t>, 8 -alpha, 9 -omega, 10 one, 11 flags (x: breakdown)
__global__ void k_bicg_scalars(int stage, double2 *sc) {
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
    const double2 beta = sc[4], om = sc[3];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 t = csub(p[q], cmul(om, v[q]));
        p[q] = cfma(beta, t, r[q]);
    }
}

__global__ void k_axpby(size_t n, const double2 *__restrict__ a, const double2 *__restrict__ x,
                        const double2 *__restrict__ b, double2 *__restrict__ y) {
    const double2 av = a[0], bv = b[0];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT)
        y[q] = cfma(av, x[q], cmul(bv, y[q]));
}

template <typename CY>
__global__ void k_axpy_mixed(size_t n, const double2 *__restrict__ a, const CY *__restrict__ x, double2 *__restrict__ y) {
    const double2 av = a[0];
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT)
        y[q] = cfma(av, to_c(x[q], 0.0), y[q]);
}

// y = W x or W^{-1} x, W_p = prod_axes w_axis[a][i_a] on interior nodes (boundary left).
__global__ void k_weight(int nx, int ny, int nz, int dim, const double2 *__restrict__ wx,
                         const double2 *__restrict__ wy, const double2 *__restrict__ wz, int inverse,
                         const double2 *__restrict__ x, double2 *__restrict__ y) {
    const size_t n = (size_t)nx * ny * nz;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((size_t)nx * ny));
        if (i < 1 || i > nx - 2 || j < 1 || j > ny - 2 || (dim == 3 && (k < 1 || k > nz - 2))) continue;
        double2 w = cmul(wx[i], wy[j]);
        if (dim == 3) w = cmul(w, wz[k]);
        if (inverse) w = cinv(w);
        y[q] = cmul(w, x[q]);
    }
}

__global__ void k_grad_k2(int nx, int ny, int nz, int dim, const double2 *__restrict__ lam,
                          const double2 *__restrict__ u, double *__restrict__ grad) {
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

#define DISPATCH_MAXV(nv, KERNEL, ...)                                                         \
    do {                                                                                       \
        if ((nv) <= 8) KERNEL<8><<<blas_nblocks(n), NT, 0, s>>>(__VA_ARGS__);                  \
        else if ((nv) <= 16) KERNEL<16><<<blas_nblocks(n), NT, 0, s>>>(__VA_ARGS__);           \
        else if ((nv) <= 32) KERNEL<32><<<blas_nblocks(n), NT, 0, s>>>(__VA_ARGS__);           \
        else KERNEL<64><<<blas_nblocks(n), NT, 0, s>>>(__VA_ARGS__);                           \
    } while (0)

cudaError_t launch_mdot(size_t n, const double2 *V, size_t ldv, int nv, const double2 *w, double2 *partials,
                        cudaStream_t s) {
    if (nv > 64) return cudaErrorInvalidValue;
    DISPATCH_MAXV(nv, k_mdot, n, V, ldv, nv, w, partials);
    return cudaGetLastError();
}

cudaError_t launch_update_mdot(size_t n, const double2 *V, size_t ldv, int nv, const double2 *h, double2 *w,
                               double2 *partials, cudaStream_t s) {
    if (nv > 64) return cudaErrorInvalidValue;
    DISPATCH_MAXV(nv, k_update_mdot, n, V, ldv, nv, h, w, partials);
    return cudaGetLastError();
}

cudaError_t launch_update_norm(size_t n, const double2 *V, size_t ldv, int nv, const double2 *h, double2 *w,
                               double2 *partials, cudaStream_t s) {
    if (nv > 64) return cudaErrorInvalidValue;
    DISPATCH_MAXV(nv, k_update_norm, n, V, ldv, nv, h, w, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double2 *partials, int nblk, int nv, double2 *out, int mode, cudaStream_t s) {
    k_reduce<<<nv, NT, 0, s>>>(partials, nblk, out, mode);
    return cudaGetLastError();
}

cudaError_t launch_scale_inv(size_t n, const double2 *x, const double2 *scale, double2 *y, cudaStream_t s) {
    k_scale_inv<<<stream_grid(n), NT, 0, s>>>(n, x, scale, y);
    return cudaGetLastError();
}

template <typename CZ>
cudaError_t launch_combine(size_t n, const CZ *Z, size_t ldz, int nz, const double2 *y, double2 *x, cudaStream_t s) {
    if (nz > 64) return cudaErrorInvalidValue;
    k_combine<CZ><<<stream_grid(n), NT, 0, s>>>(n, Z, ldz, nz, y, x);
    return cudaGetLastError();
}
template cudaError_t launch_combine<float2>(size_t, const float2 *, size_t, int, const double2 *, double2 *, cudaStream_t);
template cudaError_t launch_combine<double2>(size_t, const double2 *, size_t, int, const double2 *, double2 *, cudaStream_t);

cudaError_t launch_givens(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g, double fnorm,
                          double *est, cudaStream_t s) {
    k_givens<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, g, fnorm, est);
    return cudaGetLastError();
}

cudaError_t launch_backsolve(const double2 *H, int ldh, int k, const double2 *g, double2 *y, cudaStream_t s) {
    k_backsolve<<<1, 32, 0, s>>>(H, ldh, k, g, y);
    return cudaGetLastError();
}

cudaError_t launch_bicg_scalars(int stage, double2 *sc, cudaStream_t s) {
    k_bicg_scalars<<<1, 32, 0, s>>>(stage, sc);
    return cudaGetLastError();
}

cudaError_t launch_bicg_p(size_t n, const double2 *r, const double2 *v, const double2 *sc, double2 *p,
                          cudaStream_t s) {
    k_bicg_p<<<stream_grid(n), NT, 0, s>>>(n, r, v, sc, p);
    return cudaGetLastError();
}

cudaError_t launch_axpby(size_t n, const double2 *a, const double2 *x, const double2 *b, double2 *y,
                         cudaStream_t s) {
    k_axpby<<<stream_grid(n), NT, 0, s>>>(n, a, x, b, y);
    return cudaGetLastError();
}

template <typename CY>
cudaError_t launch_axpy_mixed(size_t n, const double2 *a, const CY *x, double2 *y, cudaStream_t s) {
    k_axpy_mixed<CY><<<stream_grid(n), NT, 0, s>>>(n, a, x, y);
    return cudaGetLastError();
}
template cudaError_t launch_axpy_mixed<float2>(size_t, const double2 *, const float2 *, double2 *, cudaStream_t);
template cudaError_t launch_axpy_mixed<double2>(size_t, const double2 *, const double2 *, double2 *, cudaStream_t);

cudaError_t launch_weight(size_t n, const int nodes[3], int dim, const double2 *w_axis[3], int inverse,
                          const double2 *x, double2 *y, cudaStream_t s) {
    k_weight<<<stream_grid(n), NT, 0, s>>>(nodes[0], nodes[1], dim == 3 ? nodes[2] : 1, dim, w_axis[0], w_axis[1],
                                           w_axis[2], inverse, x, y);
    return cudaGetLastError();
}

cudaError_t launch_grad_k2(size_t n, const int nodes[3], int dim, const double2 *lam, const double2 *u,
                           double *grad, cudaStream_t s) {
    k_grad_k2<<<stream_grid(n), NT, 0, s>>>(nodes[0], nodes[1], dim == 3 ? nodes[2] : 1, dim, lam, u, grad);
    return cudaGetLastError();
}
