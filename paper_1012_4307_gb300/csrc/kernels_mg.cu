// Stencil and multigrid kernels for the ECS Helmholtz operators (sm_103a).
//
// Operator (Section 3.2 FD formula for unequal complex widths, summed over axes, with the
// operator coefficients of Section 5 folded in):
//   (M x)_p = sum_axes (cw x_{p-e} + cc x_p + ce x_{p+e}) + (bk k2_p + c) x_p.
// Multigrid components (Section 4.2): omega-Jacobi, omega-red-black Jacobi, full-weighting
// restriction fused with the residual, bi/trilinear prolongation fused with the correction,
// and the exact coarsest solve (Algorithm 1 step (0)) as a dense-inverse product.
//
// Layout: interleaved complex node arrays, x fastest, boundary included (never written).
// Threads: 2D blocks of 32 x 8 over (i, j); in 3D every thread marches a chunk of k planes
// keeping the x[p - nx ny], x[p], x[p + nx ny] column in registers.  Every launch covers the
// interior only, so no thread touches a boundary node's value except as a stencil neighbour.
#include "helm_internal.h"

namespace {

constexpr int BX = 32, BY = 8, KCHUNK = 8;

template <typename R> struct OpView {
    typedef typename CT<R>::T C;
    const C *__restrict__ cx;
    const C *__restrict__ cy;
    const C *__restrict__ cz;
    const R *__restrict__ k2;
    const C *__restrict__ dinv;
    C bk, c;
    int nx, ny, nz;
    const int *gate;  // see DevOp::gate
};

template <typename R> __host__ __device__ OpView<R> view(const DevOp<R> &op) {
    OpView<R> v;
    v.cx = op.coef[0]; v.cy = op.coef[1]; v.cz = op.coef[2];
    v.k2 = op.k2; v.dinv = op.dinv; v.bk = op.bk; v.c = op.c; v.gate = op.gate;
    v.nx = op.n[0]; v.ny = op.n[1]; v.nz = op.n[2];
    return v;
}

// Coefficient load: the read-only global path (ld.global.nc) for operators in global memory,
// a plain (generic) load when the operator's arrays may live in shared memory.
template <bool GLOBAL, typename T> __device__ __forceinline__ T ldc(const T *p) {
    if constexpr (GLOBAL) return __ldg(p);
    else return *p;
}

// Off-diagonal part of the stencil at p (neighbours along x and y; z handled by callers that
// march in k) and the diagonal entry.  GLOBAL: the coefficient arrays are in global memory.
template <typename R, int DIM, typename CX, bool GLOBAL = true>
__device__ __forceinline__ typename CT<R>::T stencil(const OpView<R> &o, const CX *__restrict__ x, size_t p,
                                                    int i, int j, int k, typename CT<R>::T xm_z,
                                                    typename CT<R>::T xc, typename CT<R>::T xp_z,
                                                    typename CT<R>::T &diag) {
    typedef typename CT<R>::T C;
    const size_t sy = (size_t)o.nx;
    C cw = ldc<GLOBAL>(&o.cx[3 * i]), cc = ldc<GLOBAL>(&o.cx[3 * i + 1]), ce = ldc<GLOBAL>(&o.cx[3 * i + 2]);
    C acc = cmul(cw, to_c(x[p - 1], R()));
    acc = cfma(ce, to_c(x[p + 1], R()), acc);
    C d = cc;
    cw = ldc<GLOBAL>(&o.cy[3 * j]); cc = ldc<GLOBAL>(&o.cy[3 * j + 1]); ce = ldc<GLOBAL>(&o.cy[3 * j + 2]);
    acc = cfma(cw, to_c(x[p - sy], R()), acc);
    acc = cfma(ce, to_c(x[p + sy], R()), acc);
    d = cadd(d, cc);
    if (DIM == 3) {
        cw = ldc<GLOBAL>(&o.cz[3 * k]); cc = ldc<GLOBAL>(&o.cz[3 * k + 1]); ce = ldc<GLOBAL>(&o.cz[3 * k + 2]);
        acc = cfma(cw, xm_z, acc);
        acc = cfma(ce, xp_z, acc);
        d = cadd(d, cc);
    }
    d = cadd(d, cadd(cscale(o.bk, o.k2[p]), o.c));
    diag = d;
    return cfma(d, xc, acc);
}

// (M x)_p for a point whose z neighbours are loaded here (used by the restriction kernel).
template <typename R, int DIM, typename CX, bool GLOBAL = true>
__device__ __forceinline__ typename CT<R>::T apply_point(const OpView<R> &o, const CX *__restrict__ x, int i, int j,
                                                        int k, typename CT<R>::T &diag) {
    typedef typename CT<R>::T C;
    const size_t sz = (size_t)o.nx * o.ny;
    const size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k);
    C xm = mk(R(0), R(0)), xp = mk(R(0), R(0));
    if (DIM == 3) { xm = to_c(x[p - sz], R()); xp = to_c(x[p + sz], R()); }
    return stencil<R, DIM, CX, GLOBAL>(o, x, p, i, j, k, xm, to_c(x[p], R()), xp, diag);
}

// Thread preamble: interior (i, j) and the k range of this thread.
#define INTERIOR_IJ(o)                                              \
    const int i = blockIdx.x * BX + threadIdx.x + 1;                \
    const int j = blockIdx.y * BY + threadIdx.y + 1;                \
    if (i > (o).nx - 2 || j > (o).ny - 2) return;                   \
    int k0 = 0, k1 = 1;                                             \
    if (DIM == 3) {                                                 \
        k0 = blockIdx.z * KCHUNK + 1;                               \
        k1 = min(k0 + KCHUNK, (o).nz - 1);                          \
    }                                                               \
    const size_t sz = (size_t)(o).nx * (o).ny;                      \
    size_t p = (size_t)i + (size_t)(o).nx * ((size_t)j + (size_t)(o).ny * k0);

template <typename R, int DIM, typename CX>
__global__ void __launch_bounds__(BX *BY) k_apply(OpView<R> o, const CX *__restrict__ x, typename CT<R>::T *__restrict__ y) {
    pdl_enter();
    typedef typename CT<R>::T C;
    INTERIOR_IJ(o);
    C xm = mk(R(0), R(0)), xc = to_c(x[p], R()), xp = mk(R(0), R(0));
    if (DIM == 3) xm = to_c(x[p - sz], R());
    for (int k = k0; k < k1; k++, p += sz) {
        if (DIM == 3) xp = to_c(x[p + sz], R());
        C d;
        y[p] = stencil<R, DIM>(o, x, p, i, j, k, xm, xc, xp, d);
        if (DIM == 3) { xm = xc; xc = xp; }
    }
}

template <typename R, int DIM, typename CB>
__global__ void __launch_bounds__(BX *BY) k_residual(OpView<R> o, const CB *__restrict__ b, const typename CT<R>::T *__restrict__ u,
                                                     typename CT<R>::T *__restrict__ r) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    typedef typename CT<R>::T C;
    INTERIOR_IJ(o);
    C xm = mk(R(0), R(0)), xc = u[p], xp = mk(R(0), R(0));
    if (DIM == 3) xm = u[p - sz];
    for (int k = k0; k < k1; k++, p += sz) {
        if (DIM == 3) xp = u[p + sz];
        C d;
        C mu = stencil<R, DIM>(o, u, p, i, j, k, xm, xc, xp, d);
        r[p] = csub(to_c(b[p], R()), mu);
        if (DIM == 3) { xm = xc; xc = xp; }
    }
}

// omega-Jacobi: every unknown from the previous iterate (ping-pong buffers).
template <typename R, int DIM, typename CB, bool ZERO>
__global__ void __launch_bounds__(BX *BY) k_jacobi(OpView<R> o, R omega, const CB *__restrict__ b, const typename CT<R>::T *__restrict__ u,
                                                   typename CT<R>::T *__restrict__ un) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    typedef typename CT<R>::T C;
    INTERIOR_IJ(o);
    if (ZERO) {
        for (int k = k0; k < k1; k++, p += sz) {
            C d;
            // diagonal only: the stencil of the zero vector
            d = cadd(cadd(__ldg(&o.cx[3 * i + 1]), __ldg(&o.cy[3 * j + 1])), cadd(cscale(o.bk, o.k2[p]), o.c));
            if (DIM == 3) d = cadd(d, __ldg(&o.cz[3 * k + 1]));
            un[p] = cscale(cmul(to_c(b[p], R()), cinv(d)), omega);
        }
        return;
    }
    C xm = mk(R(0), R(0)), xc = u[p], xp = mk(R(0), R(0));
    if (DIM == 3) xm = u[p - sz];
    for (int k = k0; k < k1; k++, p += sz) {
        if (DIM == 3) xp = u[p + sz];
        C d;
        C mu = stencil<R, DIM>(o, u, p, i, j, k, xm, xc, xp, d);
        C res = csub(to_c(b[p], R()), mu);
        un[p] = cadd(xc, cscale(cmul(res, cinv(d)), omega));
        if (DIM == 3) { xm = xc; xc = xp; }
    }
}

// 3D omega-Jacobi: k_jacobi's arithmetic in the same order, with the x and y coefficient
// triples loaded once per thread, the (z - 1, z, z + 1) column in registers, and the next plane's
// operands (four in-plane neighbours, z + 2, b, k^2) loaded while this plane is computed.
// KC: fine planes per thread (shorter chunks on small grids give more blocks).
template <typename R, typename CB, bool ZERO, int KC>
__global__ void __launch_bounds__(BX *BY) k_jacobi3(OpView<R> o, R omega, const CB *__restrict__ b,
                                                    const typename CT<R>::T *__restrict__ u,
                                                    typename CT<R>::T *__restrict__ un) {
    pdl_enter();
    const int gv = gate_value(o.gate);
    typedef typename CT<R>::T C;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    if (i > o.nx - 2 || j > o.ny - 2) return;
    const int k0 = blockIdx.z * KC + 1, k1 = min(k0 + KC, o.nz - 1);
    const size_t sz = (size_t)o.nx * o.ny;
    size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k0);
    const size_t sy = (size_t)o.nx;
    const C cwx = __ldg(&o.cx[3 * i]), ccx = __ldg(&o.cx[3 * i + 1]), cex = __ldg(&o.cx[3 * i + 2]);
    const C cwy = __ldg(&o.cy[3 * j]), ccy = __ldg(&o.cy[3 * j + 1]), cey = __ldg(&o.cy[3 * j + 2]);
    C bq = to_c(b[p], R());
    R kq = o.k2[p];
    if (gv) return;
    if (ZERO) {
        const C dxy = cadd(ccx, ccy);
        for (int k = k0; k < k1; k++, p += sz) {
            C bn = bq;
            R kn = kq;
            if (k + 1 < k1) {
                bn = to_c(b[p + sz], R());
                kn = o.k2[p + sz];
            }
            const C d = cadd(cadd(dxy, cadd(cscale(o.bk, kq), o.c)), __ldg(&o.cz[3 * k + 1]));
            un[p] = cscale(cmul(bq, cinv(d)), omega);
            bq = bn;
            kq = kn;
        }
        return;
    }
    C xm = u[p - sz], xc = u[p], xp = u[p + sz];
    C xw = u[p - 1], xe = u[p + 1], xs = u[p - sy], xn = u[p + sy];
    for (int k = k0; k < k1; k++, p += sz) {
        C xw2 = xw, xe2 = xe, xs2 = xs, xn2 = xn, xp2 = xp, bn = bq;
        R kn = kq;
        if (k + 1 < k1) {
            const size_t q = p + sz;
            xw2 = u[q - 1];
            xe2 = u[q + 1];
            xs2 = u[q - sy];
            xn2 = u[q + sy];
            xp2 = u[q + sz];
            bn = to_c(b[q], R());
            kn = o.k2[q];
        }
        C acc = cmul(cwx, xw);
        acc = cfma(cex, xe, acc);
        C d = ccx;
        acc = cfma(cwy, xs, acc);
        acc = cfma(cey, xn, acc);
        d = cadd(d, ccy);
        const C czw = __ldg(&o.cz[3 * k]), czc = __ldg(&o.cz[3 * k + 1]), cze = __ldg(&o.cz[3 * k + 2]);
        acc = cfma(czw, xm, acc);
        acc = cfma(cze, xp, acc);
        d = cadd(d, czc);
        d = cadd(d, cadd(cscale(o.bk, kq), o.c));
        const C mu = cfma(d, xc, acc);
        const C res = csub(bq, mu);
        un[p] = cadd(xc, cscale(cmul(res, cinv(d)), omega));
        xm = xc;
        xc = xp;
        xw = xw2; xe = xe2; xs = xs2; xn = xn2; xp = xp2; bq = bn; kq = kn;
    }
}

// one colour of omega-red-black Jacobi, in place: threads map to every other x node.
template <typename R, int DIM, typename CB>
__global__ void __launch_bounds__(BX *BY) k_rb(OpView<R> o, R omega, const CB *__restrict__ b, typename CT<R>::T *u, int colour) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    typedef typename CT<R>::T C;
    const int t = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    if (j > o.ny - 2) return;
    int k0 = 0, k1 = 1;
    if (DIM == 3) { k0 = blockIdx.z * KCHUNK + 1; k1 = min(k0 + KCHUNK, o.nz - 1); }
    const size_t sz = (size_t)o.nx * o.ny;
    for (int k = k0; k < k1; k++) {
        const int i = 2 * t + 1 + ((1 + j + k + colour) & 1);
        if (i > o.nx - 2) continue;
        const size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k);
        C xm = mk(R(0), R(0)), xp = mk(R(0), R(0));
        if (DIM == 3) { xm = u[p - sz]; xp = u[p + sz]; }
        C xc = u[p];
        C d;
        C mu = stencil<R, DIM>(o, u, p, i, j, k, xm, xc, xp, d);
        u[p] = cadd(xc, cscale(cmul(csub(to_c(b[p], R()), mu), cinv(d)), omega));
    }
}

// rc[I] = sum_{d in {-1,0,1}^DIM} prod w(d) (b - M u)[2I + d],  w(0) = 1/2, w(+-1) = 1/4.
template <typename R, int DIM, typename CB>
__global__ void __launch_bounds__(BX *BY) k_residual_restrict(OpView<R> o, const CB *__restrict__ b, const typename CT<R>::T *__restrict__ u,
                                                              typename CT<R>::T *__restrict__ rc, int ncx, int ncy, int ncz) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    typedef typename CT<R>::T C;
    const int I = blockIdx.x * BX + threadIdx.x + 1;
    const int J = blockIdx.y * BY + threadIdx.y + 1;
    if (I > ncx - 2 || J > ncy - 2) return;
    int K0 = 0, K1 = 1;
    if (DIM == 3) { K0 = blockIdx.z * KCHUNK + 1; K1 = min(K0 + KCHUNK, ncz - 1); }
    for (int K = K0; K < K1; K++) {
        C acc = mk(R(0), R(0));
        const int dk0 = DIM == 3 ? -1 : 0, dk1 = DIM == 3 ? 1 : 0;
        for (int dk = dk0; dk <= dk1; dk++) {
            const R wk = DIM == 3 ? (dk == 0 ? R(0.5) : R(0.25)) : R(1);
            const int k = DIM == 3 ? 2 * K + dk : 0;
#pragma unroll
            for (int dj = -1; dj <= 1; dj++) {
                const R wj = wk * (dj == 0 ? R(0.5) : R(0.25));
                const int j = 2 * J + dj;
#pragma unroll
                for (int di = -1; di <= 1; di++) {
                    const R w = wj * (di == 0 ? R(0.5) : R(0.25));
                    const int i = 2 * I + di;
                    const size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k);
                    C d;
                    C mu = apply_point<R, DIM>(o, u, i, j, k, d);
                    acc = cadd(acc, cscale(csub(to_c(b[p], R()), mu), w));
                }
            }
        }
        rc[(size_t)I + (size_t)ncx * ((size_t)J + (size_t)ncy * K)] = acc;
    }
}

// uf[q] += average of ec over coarse nodes floor(q/2), ceil(q/2) along every axis.
template <typename R, int DIM>
__global__ void __launch_bounds__(BX *BY) k_prolong_add(int nx, int ny, int nz, const typename CT<R>::T *__restrict__ ec,
                                                        typename CT<R>::T *__restrict__ uf,
                                                        const int *__restrict__ gate) {
    pdl_enter();
    if (gate && *gate) return;
    typedef typename CT<R>::T C;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    if (i > nx - 2 || j > ny - 2) return;
    const int ncx = (nx + 1) / 2, ncy = (ny + 1) / 2;
    int k0 = 0, k1 = 1;
    if (DIM == 3) { k0 = blockIdx.z * KCHUNK + 1; k1 = min(k0 + KCHUNK, nz - 1); }
    const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
    for (int k = k0; k < k1; k++) {
        const int kk0 = DIM == 3 ? k >> 1 : 0, kk1 = DIM == 3 ? (k + 1) >> 1 : 0;
        C acc = mk(R(0), R(0));
        int cnt = 0;
        for (int kk = kk0; kk <= kk1; kk++)
            for (int jj = j0; jj <= j1; jj++)
                for (int ii = i0; ii <= i1; ii++) {
                    acc = cadd(acc, ec[(size_t)ii + (size_t)ncx * ((size_t)jj + (size_t)ncy * kk)]);
                    cnt++;
                }
        const size_t p = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
        uf[p] = cadd(uf[p], cscale(acc, R(1) / R(cnt)));
    }
}

// 3D residual + full weighting, each fine residual computed once.  A block owns R3_TX x R3_TY
// coarse nodes in (x, y) and kc coarse planes (at most R3_KC); one thread per fine node of the region those
// coarse nodes weigh ((2 R3_TX + 1) x (2 R3_TY + 1)) marches the block's fine planes
// 2 K0 - 1 .. 2 K1 - 1 like k_jacobi3 (coefficients in registers, the u column (z - 1, z, z + 1)
// in registers, the next plane's operands loaded while this plane is computed) and stores its
// residual in a shared plane (two buffers); after one barrier per plane the coarse nodes' threads
// apply (1,2,1)/4 in x and y from the shared plane and accumulate (1,2,1)/4 in z in registers:
// an odd fine plane 2K + 1 completes coarse plane K and starts K + 1.  Fine nodes outside the
// grid's interior hold zero residuals.  Same arithmetic as k_residual_restrict, with the weights
// applied per axis.
constexpr int R3_TX = 16, R3_TY = 8, R3_KC = 8;
constexpr int R3_FW = 2 * R3_TX + 1, R3_FH = 2 * R3_TY + 1;  // fine region
constexpr int R3_NT = ((R3_FW * R3_FH + 31) / 32) * 32;       // threads: one per region node
template <typename R> constexpr size_t r3_smem_bytes() {
    return (size_t)2 * R3_FW * R3_FH * sizeof(typename CT<R>::T);
}

template <typename R, typename CB>
__global__ void __launch_bounds__(R3_NT, sizeof(R) == sizeof(float) ? 2 : 1)
    k_resrestrict3(OpView<R> o, const CB *__restrict__ b, const typename CT<R>::T *__restrict__ u,
                   typename CT<R>::T *__restrict__ rc, int ncx, int ncy, int ncz, int kc) {
    pdl_enter();
    const int gv = gate_value(o.gate);
    typedef typename CT<R>::T C;
    extern __shared__ __align__(16) unsigned char r3_smem[];
    C(*rbuf)[R3_FH][R3_FW] = reinterpret_cast<C(*)[R3_FH][R3_FW]>(r3_smem);
    const int nx = o.nx, ny = o.ny;
    const int I0 = 1 + blockIdx.x * R3_TX, J0 = 1 + blockIdx.y * R3_TY;
    const int K0 = 1 + blockIdx.z * kc, K1 = min(K0 + kc, ncz - 1);
    const int t = threadIdx.x, lx = t % R3_FW, ly = t / R3_FW;
    const int x = 2 * I0 - 1 + lx, y = 2 * J0 - 1 + ly;
    // region nodes inside the grid's interior compute residuals; the others hold zeros
    const bool res = t < R3_FW * R3_FH && x <= nx - 2 && y <= ny - 2;
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const int zs = 2 * K0 - 1, ze = 2 * K1 - 1;
    const C zero = mk(R(0), R(0));
    C cwx = zero, ccx = zero, cex = zero, cwy = zero, ccy = zero, cey = zero;
    C xm = zero, xc = zero, xp = zero, xw = zero, xe = zero, xs = zero, xn = zero, bq = zero;
    R kq = R(0);
    size_t p = (size_t)x + sy * y + sz * zs;
    if (res) {
        cwx = __ldg(&o.cx[3 * x]); ccx = __ldg(&o.cx[3 * x + 1]); cex = __ldg(&o.cx[3 * x + 2]);
        cwy = __ldg(&o.cy[3 * y]); ccy = __ldg(&o.cy[3 * y + 1]); cey = __ldg(&o.cy[3 * y + 2]);
        xm = u[p - sz]; xc = u[p]; xp = u[p + sz];
        xw = u[p - 1]; xe = u[p + 1]; xs = u[p - sy]; xn = u[p + sy];
        bq = to_c(b[p], R());
        kq = o.k2[p];
    }
    if (gv) return;  // the same value in every thread: no barrier is left waiting
    // the coarse node of this thread (threads below R3_TX * R3_TY), and its running z sum
    const int cx = t % R3_TX, cy = t / R3_TX, I = I0 + cx, J = J0 + cy;
    const bool own = t < R3_TX * R3_TY && I <= ncx - 2 && J <= ncy - 2;
    C acc = zero;
    for (int z = zs; z <= ze; z++, p += sz) {
        if (res) {
            C xw2 = xw, xe2 = xe, xs2 = xs, xn2 = xn, xp2 = xp, bn = bq;
            R kn = kq;
            if (z < ze) {
                const size_t q = p + sz;
                xw2 = u[q - 1];
                xe2 = u[q + 1];
                xs2 = u[q - sy];
                xn2 = u[q + sy];
                xp2 = u[q + sz];
                bn = to_c(b[q], R());
                kn = o.k2[q];
            }
            C a2 = cmul(cwx, xw);
            a2 = cfma(cex, xe, a2);
            C d = ccx;
            a2 = cfma(cwy, xs, a2);
            a2 = cfma(cey, xn, a2);
            d = cadd(d, ccy);
            const C czw = __ldg(&o.cz[3 * z]), czc = __ldg(&o.cz[3 * z + 1]), cze = __ldg(&o.cz[3 * z + 2]);
            a2 = cfma(czw, xm, a2);
            a2 = cfma(cze, xp, a2);
            d = cadd(d, czc);
            d = cadd(d, cadd(cscale(o.bk, kq), o.c));
            rbuf[z & 1][ly][lx] = csub(bq, cfma(d, xc, a2));
            xm = xc;
            xc = xp;
            xw = xw2; xe = xe2; xs = xs2; xn = xn2; xp = xp2; bq = bn; kq = kn;
        } else if (t < R3_FW * R3_FH) {
            rbuf[z & 1][ly][lx] = zero;
        }
        __syncthreads();
        if (own) {
            // (1,2,1)/4 along x on the three fine rows 2J - 1 .. 2J + 1, then along y
            const C(*rr)[R3_FW] = rbuf[z & 1];
            const int fx = 2 * cx, fy = 2 * cy;
            C a[3];
#pragma unroll
            for (int dy = 0; dy < 3; dy++) {
                const C *row = &rr[fy + dy][fx];
                a[dy] = cadd(cadd(row[0], row[2]), cscale(row[1], R(2)));
            }
            const C v = cadd(cadd(a[0], a[2]), cscale(a[1], R(2)));
            if (z & 1) {
                // fine plane 2K + 1 (K = (z - 1) / 2) completes coarse plane K and starts K + 1
                const int K = (z - 1) >> 1;
                if (K >= K0) rc[(size_t)I + (size_t)ncx * ((size_t)J + (size_t)ncy * K)] = cscale(cadd(acc, v), R(1.0 / 64.0));
                acc = v;
            } else {
                acc = cadd(acc, cscale(v, R(2)));
            }
        }
    }
}

// 3D prolongation + correction in closed form: uf[p] += 1/8 of the sum of ec at the eight corners
// (floor / ceil of i/2, j/2, k/2), coincident corners repeated, i.e. the average over the distinct
// coarse nodes of k_prolong_add.  Each thread marches kc fine planes.
template <typename R>
__global__ void __launch_bounds__(BX *BY) k_prolong3(int nx, int ny, int nz, const typename CT<R>::T *__restrict__ ec,
                                                     typename CT<R>::T *__restrict__ uf, int kc,
                                                     const int *__restrict__ gate) {
    pdl_enter();
    const int gv = gate_value(gate);
    typedef typename CT<R>::T C;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    if (i > nx - 2 || j > ny - 2) return;
    const int ncx = (nx + 1) / 2, ncy = (ny + 1) / 2;
    const int k0 = blockIdx.z * kc + 1, k1 = min(k0 + kc, nz - 1);
    const size_t csy = (size_t)ncx, csz = (size_t)ncx * ncy;
    const size_t c00 = (size_t)(i >> 1) + csy * (j >> 1), c10 = (size_t)((i + 1) >> 1) + csy * (j >> 1);
    const size_t c01 = (size_t)(i >> 1) + csy * ((j + 1) >> 1), c11 = (size_t)((i + 1) >> 1) + csy * ((j + 1) >> 1);
    // S(c): the four in-plane corners' sum on coarse plane c; fine plane k takes S(k >> 1) and
    // S((k + 1) >> 1), so every coarse plane is summed once and the next one is loaded while the
    // current fine plane is written
    auto corner_sum = [&](int c) {
        const size_t z = csz * c;
        return cadd(cadd(ec[c00 + z], ec[c10 + z]), cadd(ec[c01 + z], ec[c11 + z]));
    };
    C sa = corner_sum(k0 >> 1), sb = corner_sum((k0 + 1) >> 1);
    size_t p = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k0);
    C uq = uf[p];
    if (gv) return;
    for (int k = k0; k < k1; k++, p += (size_t)nx * ny) {
        C sn = sb, un = uq;
        if (k + 1 < k1) {
            un = uf[p + (size_t)nx * ny];
            if (((k + 2) >> 1) != ((k + 1) >> 1)) sn = corner_sum((k + 2) >> 1);
        }
        uf[p] = cadd(uq, cscale(cadd(sa, sb), R(0.125)));
        // next fine plane: (k + 1) >> 1 is this plane's upper coarse plane
        sa = sb;
        sb = sn;
        uq = un;
    }
}

// Exact coarsest solve as u = Minv b on the unknowns (interior nodes in natural order); one
// warp per row, fixed-order lane partial sums reduced by shuffles.
template <typename R>
__global__ void k_dense_solve(int nx, int ny, int nz, int dim, int nu, const typename CT<R>::T *__restrict__ minv,
                              const typename CT<R>::T *__restrict__ b, typename CT<R>::T *__restrict__ u) {
    pdl_enter();
    typedef typename CT<R>::T C;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nu) return;
    const int mx = nx - 2, my = ny - 2;
    C acc = mk(R(0), R(0));
    for (int c = lane; c < nu; c += 32) {
        const int ci = c % mx, cj = (c / mx) % my, ck = dim == 3 ? c / (mx * my) : -1;
        const size_t q = (size_t)(ci + 1) + (size_t)nx * ((size_t)(cj + 1) + (size_t)ny * (ck + 1));
        acc = cfma(minv[(size_t)warp * nu + c], b[q], acc);
    }
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) {
        const int ri = warp % mx, rj = (warp / mx) % my, rk = dim == 3 ? warp / (mx * my) : -1;
        u[(size_t)(ri + 1) + (size_t)nx * ((size_t)(rj + 1) + (size_t)ny * (rk + 1))] = acc;
    }
    (void)nz;
}

template <typename CI, typename CO>
__global__ void k_convert(size_t n, const CI *__restrict__ in, CO *__restrict__ out) {
    pdl_enter();
    typedef decltype(out->x) RO;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        out[q] = to_c(in[q], RO());
}

template <typename C> __global__ void k_zero(size_t n, C *x) {
    pdl_enter();
    typedef decltype(x->x) R;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        x[q] = mk(R(0), R(0));
}

// ------------------------------------------------------------------------------ temporal blocking
// 2D omega-Jacobi with two sweeps, several sweeps per shared-memory tile.  Each block owns a
// tile of TCX x TCY coarse nodes and the fine nodes x in [2 I0 - 1, 2 I0 + 2 TCX - 1) (same in
// y), and works on the fine region R3 = [2 I0 - 3, 2 I0 + 2 TCX + 1], the owned nodes plus a
// 3-node halo: two sweeps and a residual each consume one halo layer.  Nodes outside the
// interior of the grid are held at zero (Dirichlet).  Same arithmetic as k_jacobi /
// k_residual_restrict / k_prolong_add, in one launch per phase of the cycle instead of three.
// The tile shape is a template parameter; the host picks one per level (tuning).
// Threads of a block of the blocked kernels for a region of n nodes: the fewest passes over the
// region with at most 512 threads, then the fewest warps for that many passes (a fixed 256 left a
// nearly empty last pass on some tiles: 777 = 3 x 256 + 9).
constexpr int tile_threads(int n) { return ((n + (n + 511) / 512 - 1) / ((n + 511) / 512) + 31) / 32 * 32; }

template <int TCX, int TCY> struct Tile {
    static constexpr int RW = 2 * TCX + 5, RH = 2 * TCY + 5;  // R3 extent
    static constexpr int NT = tile_threads(RW * RH);           // threads per block
    struct Coef {
        float2 x[RW][3], y[RH][3];
    };
    struct Pre {
        Coef tc;
        float2 b[RH][RW];
        float2 di[RH][RW];  // 1 / diagonal
        float2 u1[RH][RW];  // first sweep, later the residual
        float2 u2[RH][RW];
    };
    struct Post {
        Coef tc;
        float2 b[RH][RW];
        float2 di[RH][RW];  // 1 / diagonal
        float2 u3[RH][RW];
        float2 u4[RH][RW];
    };
};

// Loads the operator's coefficient triples of the region's columns and rows.
template <int RW, int RH, typename TC>
__device__ __forceinline__ void tile_coef(const OpView<float> &o, int X0, int Y0, TC &tc) {
    for (int q = threadIdx.x; q < RW * 3; q += blockDim.x) {
        const int sx = q / 3, t = q % 3, x = X0 + sx;
        tc.x[sx][t] = (x >= 1 && x <= o.nx - 2) ? o.cx[3 * x + t] : make_float2(0.f, 0.f);
    }
    for (int q = threadIdx.x; q < RH * 3; q += blockDim.x) {
        const int sy = q / 3, t = q % 3, y = Y0 + sy;
        tc.y[sy][t] = (y >= 1 && y <= o.ny - 2) ? o.cy[3 * y + t] : make_float2(0.f, 0.f);
    }
}

// (M u)_s and the diagonal at region node (sx, sy) from shared-memory u (row stride RW).
template <int RW, typename TC>
__device__ __forceinline__ float2 tile_stencil(const TC &tc, const float2 (*u)[RW], int sx, int sy, float k2,
                                               float2 bk, float2 c, float2 &d) {
    float2 acc = cmul(tc.x[sx][0], u[sy][sx - 1]);
    acc = cfma(tc.x[sx][2], u[sy][sx + 1], acc);
    acc = cfma(tc.y[sy][0], u[sy - 1][sx], acc);
    acc = cfma(tc.y[sy][2], u[sy + 1][sx], acc);
    d = cadd(cadd(tc.x[sx][1], tc.y[sy][1]), cadd(cscale(bk, k2), c));
    return cfma(d, u[sy][sx], acc);
}

// Off-diagonal part of (M u)_s at region node (sx, sy).
template <int RW, typename TC>
__device__ __forceinline__ float2 tile_offdiag(const TC &tc, const float2 (*u)[RW], int sx, int sy) {
    float2 acc = cmul(tc.x[sx][0], u[sy][sx - 1]);
    acc = cfma(tc.x[sx][2], u[sy][sx + 1], acc);
    acc = cfma(tc.y[sy][0], u[sy - 1][sx], acc);
    return cfma(tc.y[sy][2], u[sy + 1][sx], acc);
}
// One omega-Jacobi update at region node (sx, sy): u + omega ((b - offdiag) / d - u).
template <int RW, typename TC>
__device__ __forceinline__ float2 tile_jacobi(const TC &tc, const float2 (*u)[RW], const float2 (*b)[RW],
                                              const float2 (*di)[RW], int sx, int sy, float omega) {
    const float2 uc = u[sy][sx];
    const float2 t = cmul(csub(b[sy][sx], tile_offdiag<RW>(tc, u, sx, sy)), di[sy][sx]);
    return cadd(uc, cscale(csub(t, uc), omega));
}

// f(sx, sy) for every node of an RW x RH region, ST threads, node q = tid + ST k in row-major
// order (the region coordinates advance incrementally).
template <int RW, int RH, int ST, typename F>
__device__ __forceinline__ void for_region(F f) {
    constexpr int N = RW * RH, DX = ST % RW, DY = ST / RW;
    int sx = threadIdx.x % RW, sy = threadIdx.x / RW;
    for (int q = threadIdx.x; q < N; q += ST) {
        f(sx, sy);
        sx += DX;
        sy += DY;
        if (sx >= RW) {
            sx -= RW;
            sy++;
        }
    }
}

// Diagonal of M at region node (sx, sy) from the staged coefficients and k^2.
template <typename TC>
__device__ __forceinline__ float2 tile_diag(const TC &tc, int sx, int sy, float k2, float2 bk, float2 c) {
    return cadd(cadd(tc.x[sx][1], tc.y[sy][1]), cadd(cscale(bk, k2), c));
}

// u = two omega-Jacobi sweeps from u = 0 for M u = b, written on the owned fine nodes; then
// rc = FW(b - M u) on the owned coarse nodes.  Blocks whose region lies inside the grid's
// interior skip the per-node boundary tests.
// (bx, by): the tile of coarse nodes this block owns.
template <int TCX, int TCY>
__device__ __forceinline__ void pre2_restrict_tile(const OpView<float> &o, float omega, const float2 *__restrict__ b,
                                                   float2 *__restrict__ u, float2 *__restrict__ rc, int ncx, int ncy,
                                                   int bx, int by, const int *gate = nullptr) {
    typedef Tile<TCX, TCY> TL;
    constexpr int RW = TL::RW, RH = TL::RH;
    extern __shared__ __align__(16) unsigned char pre_smem[];
    __shared__ int gate_s;  // the gate flag, published by the first block barrier
    if (threadIdx.x == 0) gate_s = gate_value(gate);
    typename TL::Pre &T = *reinterpret_cast<typename TL::Pre *>(pre_smem);
    const int I0 = 1 + bx * TCX, J0 = 1 + by * TCY;
    const int X0 = 2 * I0 - 3, Y0 = 2 * J0 - 3;
    const int nx = o.nx, ny = o.ny;
    const bool full = X0 >= 1 && X0 + RW - 1 <= nx - 2 && Y0 >= 1 && Y0 + RH - 1 <= ny - 2;
    auto inside = [&](int x, int y) { return full || (x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2); };
    // the coefficients are first used by the second sweep: one barrier publishes them with b,
    // 1 / D and the first sweep
    tile_coef<RW, RH>(o, X0, Y0, T.tc);
    // load b and 1 / D; sweep 1 from zero (pointwise): u1 = omega b / D
    for_region<RW, RH, TL::NT>([&](int sx, int sy) {
        const int x = X0 + sx, y = Y0 + sy;
        float2 bv = make_float2(0.f, 0.f), dv = make_float2(0.f, 0.f);
        if (inside(x, y)) {
            const size_t p = (size_t)x + (size_t)nx * y;
            bv = b[p];
            dv = o.dinv[p];
        }
        T.b[sy][sx] = bv;
        T.di[sy][sx] = dv;
        T.u1[sy][sx] = cscale(cmul(bv, dv), omega);
    });
    __syncthreads();
    if (gate_s) return;
    // sweep 2 on R3 shrunk by one
    for_region<RW, RH, TL::NT>([&](int sx, int sy) {
        float2 v = make_float2(0.f, 0.f);
        if (sx >= 1 && sx < RW - 1 && sy >= 1 && sy < RH - 1 && inside(X0 + sx, Y0 + sy))
            v = tile_jacobi<RW>(T.tc, T.u1, T.b, T.di, sx, sy, omega);
        T.u2[sy][sx] = v;
    });
    __syncthreads();
    // owned fine nodes of the smoothed iterate, and the residual on R3 shrunk by two
    for_region<RW, RH, TL::NT>([&](int sx, int sy) {
        const int x = X0 + sx, y = Y0 + sy;
        const bool in = inside(x, y);
        if (in && sx >= 2 && sx < 2 + 2 * TCX && sy >= 2 && sy < 2 + 2 * TCY) u[(size_t)x + (size_t)nx * y] = T.u2[sy][sx];
        float2 r = make_float2(0.f, 0.f);
        if (in && sx >= 2 && sx < RW - 2 && sy >= 2 && sy < RH - 2) {
            const float2 d = cinv_fast(T.di[sy][sx]);
            r = csub(csub(T.b[sy][sx], tile_offdiag<RW>(T.tc, T.u2, sx, sy)), cmul(d, T.u2[sy][sx]));
        }
        T.u1[sy][sx] = r;
    });
    __syncthreads();
    // full weighting on the owned coarse nodes: fine node 2I is region node 2(I - I0) + 3
    for (int q = threadIdx.x; q < TCX * TCY; q += blockDim.x) {
        const int cx = q % TCX, cy = q / TCX, I = I0 + cx, J = J0 + cy;
        if (I > ncx - 2 || J > ncy - 2) continue;
        const int sx = 2 * cx + 3, sy = 2 * cy + 3;
        const float2 *r0 = &T.u1[sy - 1][sx], *r1 = &T.u1[sy][sx], *r2 = &T.u1[sy + 1][sx];
        // (1,2,1)/4 along x on each of the three rows, then (1,2,1)/4 along y
        const float2 a0 = cadd(cadd(r0[-1], r0[1]), cscale(r0[0], 2.f));
        const float2 a1 = cadd(cadd(r1[-1], r1[1]), cscale(r1[0], 2.f));
        const float2 a2 = cadd(cadd(r2[-1], r2[1]), cscale(r2[0], 2.f));
        rc[(size_t)I + (size_t)ncx * J] = cscale(cadd(cadd(a0, a2), cscale(a1, 2.f)), 0.0625f);
    }
}

template <int TCX, int TCY>
__global__ void __launch_bounds__(Tile<TCX, TCY>::NT, 4) k_pre2_restrict(OpView<float> o, float omega, const float2 *__restrict__ b,
                                                       float2 *__restrict__ u, float2 *__restrict__ rc, int ncx,
                                                       int ncy) {
    pdl_enter();
    pre2_restrict_tile<TCX, TCY>(o, omega, b, u, rc, ncx, ncy, blockIdx.x, blockIdx.y, o.gate);
}

// u_out <- two omega-Jacobi sweeps of (u_in + P ec), on the owned fine nodes.  u_in and u_out
// are different arrays: blocks read their halo of u_in while other blocks write u_out.
// Bilinear interpolation in closed form: P ec at fine node (x, y) is the mean of the four
// coarse values at (floor/ceil(x/2), floor/ceil(y/2)), coincident ones repeated.
template <int TCX, int TCY>
__device__ __forceinline__ void prolong_post2_tile(const OpView<float> &o, float omega, const float2 *__restrict__ b,
                                                   const float2 *__restrict__ u_in, float2 *__restrict__ u,
                                                   const float2 *__restrict__ ec, int ncx, int ncy, int bx, int by,
                                                   const int *gate = nullptr) {
    typedef Tile<TCX, TCY> TL;
    constexpr int RW = TL::RW, RH = TL::RH;
    extern __shared__ __align__(16) unsigned char post_smem[];
    __shared__ int gate_s;  // the gate flag, published by the first block barrier
    if (threadIdx.x == 0) gate_s = gate_value(gate);
    typename TL::Post &T = *reinterpret_cast<typename TL::Post *>(post_smem);
    const int I0 = 1 + bx * TCX, J0 = 1 + by * TCY;
    const int X0 = 2 * I0 - 3, Y0 = 2 * J0 - 3;
    const int nx = o.nx, ny = o.ny;
    const bool full = X0 >= 1 && X0 + RW - 1 <= nx - 2 && Y0 >= 1 && Y0 + RH - 1 <= ny - 2;
    auto inside = [&](int x, int y) { return full || (x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2); };
    // the coefficients are first used by the first sweep: one barrier publishes them with b,
    // 1 / D and u + P ec, whose coarse values each node reads itself (the four corner nodes
    // floor/ceil(x / 2), floor/ceil(y / 2) of an interior fine node lie in the coarse grid)
    tile_coef<RW, RH>(o, X0, Y0, T.tc);
    // u3 = u + P ec on the region
    for_region<RW, RH, TL::NT>([&](int sx, int sy) {
        const int x = X0 + sx, y = Y0 + sy;
        float2 bv = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
        float2 dv = make_float2(0.f, 0.f);
        if (inside(x, y)) {
            const size_t p = (size_t)x + (size_t)nx * y;
            bv = b[p];
            dv = o.dinv[p];
            const size_t ya = (size_t)ncx * (y >> 1), yb = (size_t)ncx * ((y + 1) >> 1);
            const int xa = x >> 1, xb = (x + 1) >> 1;
            const float2 e = cadd(cadd(ec[ya + xa], ec[ya + xb]), cadd(ec[yb + xa], ec[yb + xb]));
            v = cadd(u_in[p], cscale(e, 0.25f));
        }
        T.b[sy][sx] = bv;
        T.di[sy][sx] = dv;
        T.u3[sy][sx] = v;
    });
    __syncthreads();
    if (gate_s) return;
    // sweep 1 on R3 shrunk by one
    for_region<RW, RH, TL::NT>([&](int sx, int sy) {
        float2 v = make_float2(0.f, 0.f);
        if (sx >= 1 && sx < RW - 1 && sy >= 1 && sy < RH - 1 && inside(X0 + sx, Y0 + sy))
            v = tile_jacobi<RW>(T.tc, T.u3, T.b, T.di, sx, sy, omega);
        T.u4[sy][sx] = v;
    });
    __syncthreads();
    // sweep 2 on the owned fine nodes
    for (int q = threadIdx.x; q < 4 * TCX * TCY; q += blockDim.x) {
        const int sx = 2 + q % (2 * TCX), sy = 2 + q / (2 * TCX), x = X0 + sx, y = Y0 + sy;
        if (!inside(x, y)) continue;
        u[(size_t)x + (size_t)nx * y] = tile_jacobi<RW>(T.tc, T.u4, T.b, T.di, sx, sy, omega);
    }
}

template <int TCX, int TCY>
__global__ void __launch_bounds__(Tile<TCX, TCY>::NT, 4) k_prolong_post2(OpView<float> o, float omega, const float2 *__restrict__ b,
                                                       const float2 *__restrict__ u_in, float2 *__restrict__ u,
                                                       const float2 *__restrict__ ec, int ncx, int ncy) {
    pdl_enter();
    prolong_post2_tile<TCX, TCY>(o, omega, b, u_in, u, ec, ncx, ncy, blockIdx.x, blockIdx.y, o.gate);
}

// Batched forms (many problems, one launch): blockIdx.z picks the table entry, whose level has
// the same nodes in every entry of one launch; entries whose problem is inactive return at once.
template <int TCX, int TCY>
__global__ void __launch_bounds__(Tile<TCX, TCY>::NT, 4) k_pre2_restrict_b(const BLevel *__restrict__ tab, float omega) {
    pdl_enter();
    const BLevel &E = tab[blockIdx.z];
    if (*E.active == 0) return;
    const OpView<float> o = view(E.op);
    pre2_restrict_tile<TCX, TCY>(o, omega, E.b, E.t, E.coarse, (o.nx + 1) / 2, (o.ny + 1) / 2, blockIdx.x, blockIdx.y);
}

template <int TCX, int TCY>
__global__ void __launch_bounds__(Tile<TCX, TCY>::NT, 4) k_prolong_post2_b(const BLevel *__restrict__ tab, float omega, int j) {
    pdl_enter();
    const BLevel &E = tab[blockIdx.z];
    if (*E.active == 0) return;
    const OpView<float> o = view(E.op);
    prolong_post2_tile<TCX, TCY>(o, omega, E.b, E.t, E.u + (size_t)j * E.ustride, E.coarse, (o.nx + 1) / 2,
                                 (o.ny + 1) / 2, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------------------ coarse tail
// The coarse levels of a cycle (a few thousand unknowns or fewer) are launch- and latency-
// bound when every sweep is its own grid.  k_mg_tail runs Algorithm 1 from the tail's top
// level down to the exact coarsest solve and back inside ONE thread block, with every level's
// b, u, t in shared memory (the host picks the tail depth so they fit): the top level's
// right-hand side is copied in, its result copied out (interior nodes only).  Phases are
// block-wide loops (warps over grid rows, lanes over x) separated by __syncthreads().  Same
// arithmetic as the per-level kernels.
constexpr int TAIL_THREADS = 512;

template <typename R> struct TailLevelDev {
    OpView<R> o;
    typename CT<R>::T *b, *u, *t;
};

template <typename R> struct TailArgs {
    TailLevelDev<R> lv[MAX_TAIL_LEVELS];
    int nlev, nu_c, nu1, nu2, rb;
    R omega;
    const typename CT<R>::T *minv;
    typename CT<R>::T *bc;  // compact right-hand side of the coarsest solve (shared memory)
};

// f(i, j, k) for every interior node of a level; warps take rows (j, k), lanes take i.
template <int DIM, typename F>
__device__ __forceinline__ void for_interior(int nx, int ny, int nz, F f) {
    const int mx = nx - 2, my = ny - 2, rows = my * (DIM == 3 ? nz - 2 : 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < rows; r += nw) {
        const int j = 1 + (DIM == 3 ? r % my : r);
        const int k = DIM == 3 ? 1 + r / my : 0;
        for (int i = 1 + lane; i <= mx; i += 32) f(i, j, k);
    }
}

template <typename R, int DIM>
__device__ void tail_smooth(const TailArgs<R> &A, const TailLevelDev<R> &L, int sweeps, typename CT<R>::T **cur,
                            typename CT<R>::T **oth, bool zero) {
    typedef typename CT<R>::T C;
    const OpView<R> &o = L.o;
    const size_t sz = (size_t)o.nx * o.ny;
    auto at = [&](int i, int j, int k) { return (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k); };
    if (zero && (sweeps == 0 || A.rb)) {
        C *u = *cur;
        for_interior<DIM>(o.nx, o.ny, o.nz, [&](int i, int j, int k) { u[at(i, j, k)] = mk(R(0), R(0)); });
        __syncthreads();
    }
    for (int s = 0; s < sweeps; s++) {
        if (A.rb) {
            for (int colour = 0; colour < 2; colour++) {
                C *u = *cur;
                for_interior<DIM>(o.nx, o.ny, o.nz, [&](int i, int j, int k) {
                    if (((i + j + k) & 1) != colour) return;
                    const size_t p = at(i, j, k);
                    C xm = mk(R(0), R(0)), xp = mk(R(0), R(0));
                    if (DIM == 3) { xm = u[p - sz]; xp = u[p + sz]; }
                    const C xc = u[p];
                    C d;
                    const C mu = stencil<R, DIM, C, false>(o, u, p, i, j, k, xm, xc, xp, d);
                    u[p] = cadd(xc, cscale(cmul(csub(L.b[p], mu), cinv(d)), A.omega));
                });
                __syncthreads();
            }
        } else {
            const bool z0 = zero && s == 0;
            const C *u = *cur;
            C *un = *oth;
            for_interior<DIM>(o.nx, o.ny, o.nz, [&](int i, int j, int k) {
                const size_t p = at(i, j, k);
                if (z0) {
                    C d = cadd(cadd(o.cx[3 * i + 1], o.cy[3 * j + 1]), cadd(cscale(o.bk, o.k2[p]), o.c));
                    if (DIM == 3) d = cadd(d, o.cz[3 * k + 1]);
                    un[p] = cscale(cmul(L.b[p], cinv(d)), A.omega);
                } else {
                    C xm = mk(R(0), R(0)), xp = mk(R(0), R(0));
                    if (DIM == 3) { xm = u[p - sz]; xp = u[p + sz]; }
                    const C xc = u[p];
                    C d;
                    const C mu = stencil<R, DIM, C, false>(o, u, p, i, j, k, xm, xc, xp, d);
                    un[p] = cadd(xc, cscale(cmul(csub(L.b[p], mu), cinv(d)), A.omega));
                }
            });
            __syncthreads();
            C *t = *cur;
            *cur = *oth;
            *oth = t;
        }
    }
}

// Exact coarsest solve u = Minv b: gather b's unknowns (natural order) into a compact array,
// one warp per row of Minv (coalesced, 8 loads in flight per lane), scatter the rows.
template <typename R, int DIM>
__device__ void tail_dense(const TailArgs<R> &A, const TailLevelDev<R> &L) {
    typedef typename CT<R>::T C;
    const int mx = L.o.nx - 2, my = L.o.ny - 2, nu = A.nu_c;
    auto node = [&](int c) {
        const int i = 1 + c % mx, j = 1 + (c / mx) % my, k = DIM == 3 ? 1 + c / (mx * my) : 0;
        return (size_t)i + (size_t)L.o.nx * ((size_t)j + (size_t)L.o.ny * k);
    };
    for (int c = threadIdx.x; c < nu; c += blockDim.x) A.bc[c] = L.b[node(c)];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int row = warp; row < nu; row += nwarp) {
        const C *mrow = A.minv + (size_t)row * nu;
        C acc = mk(R(0), R(0));
#pragma unroll 8
        for (int c = lane; c < nu; c += 32) acc = cfma(mrow[c], A.bc[c], acc);
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) L.u[node(row)] = acc;
    }
    __syncthreads();
}

// Level LVL of the tail (compile-time depth, so no device recursion and no stack growth).
template <typename R, int DIM, int LVL>
__device__ void tail_cycle(const TailArgs<R> &A, bool zero, int gf, int gc) {
    typedef typename CT<R>::T C;
    constexpr int l = LVL;
    const TailLevelDev<R> &L = A.lv[l];
    if (l == A.nlev - 1) {
        tail_dense<R, DIM>(A, L);
        return;
    }
    if constexpr (LVL + 1 < MAX_TAIL_LEVELS) {
    C *cur = L.u, *oth = L.t;
    tail_smooth<R, DIM>(A, L, A.nu1, &cur, &oth, zero);
    const TailLevelDev<R> &Lc = A.lv[l + 1];
    // residual + full weighting into the next level's right-hand side
    {
        const C *uc = cur;
        for_interior<DIM>(Lc.o.nx, Lc.o.ny, Lc.o.nz, [&](int I, int J, int K) {
            C acc = mk(R(0), R(0));
            for (int dk = (DIM == 3 ? -1 : 0); dk <= (DIM == 3 ? 1 : 0); dk++) {
                const R wk = DIM == 3 ? (dk == 0 ? R(0.5) : R(0.25)) : R(1);
                const int k = DIM == 3 ? 2 * K + dk : 0;
#pragma unroll
                for (int dj = -1; dj <= 1; dj++) {
                    const R wj = wk * (dj == 0 ? R(0.5) : R(0.25));
                    const int j = 2 * J + dj;
#pragma unroll
                    for (int di = -1; di <= 1; di++) {
                        const R w = wj * (di == 0 ? R(0.5) : R(0.25));
                        const int i = 2 * I + di;
                        const size_t p = (size_t)i + (size_t)L.o.nx * ((size_t)j + (size_t)L.o.ny * k);
                        C d;
                        const C mu = apply_point<R, DIM, C, false>(L.o, uc, i, j, k, d);
                        acc = cadd(acc, cscale(csub(L.b[p], mu), w));
                    }
                }
            }
            Lc.b[(size_t)I + (size_t)Lc.o.nx * ((size_t)J + (size_t)Lc.o.ny * K)] = acc;
        });
        __syncthreads();
    }
    if (l + 1 == A.nlev - 1) {
        tail_dense<R, DIM>(A, Lc);
    } else {
        for (int i = 1; i <= gc; i++) {
            if (i == 1) tail_cycle<R, DIM, LVL + 1>(A, true, gf, gc);
            else tail_cycle<R, DIM, LVL + 1>(A, false, gc, gf);
        }
    }
    // prolongation + correction
    {
        const int nx = L.o.nx, ny = L.o.ny, ncx = Lc.o.nx, ncy = Lc.o.ny;
        C *uf = cur;
        for_interior<DIM>(nx, ny, L.o.nz, [&](int i, int j, int k) {
            const int kk0 = DIM == 3 ? k >> 1 : 0, kk1 = DIM == 3 ? (k + 1) >> 1 : 0;
            C acc = mk(R(0), R(0));
            int cnt = 0;
            for (int kk = kk0; kk <= kk1; kk++)
                for (int jj = j >> 1; jj <= (j + 1) >> 1; jj++)
                    for (int ii = i >> 1; ii <= (i + 1) >> 1; ii++) {
                        acc = cadd(acc, Lc.u[(size_t)ii + (size_t)ncx * ((size_t)jj + (size_t)ncy * kk)]);
                        cnt++;
                    }
            const size_t p = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
            uf[p] = cadd(uf[p], cscale(acc, R(1) / R(cnt)));
        });
        __syncthreads();
    }
    tail_smooth<R, DIM>(A, L, A.nu2, &cur, &oth, false);
    if (cur != L.u) {
        const C *src = cur;
        for_interior<DIM>(L.o.nx, L.o.ny, L.o.nz, [&](int i, int j, int k) {
            const size_t p = (size_t)i + (size_t)L.o.nx * ((size_t)j + (size_t)L.o.ny * k);
            L.u[p] = src[p];
        });
        __syncthreads();
    }
    }  // LVL + 1 < MAX_TAIL_LEVELS
}

// Dynamic shared memory: [compact coarsest rhs | per level: b, u, t | per level: coefficient
// triples, k^2].  A.lv[0].b / u hold the
// caller's global top-level vectors; zero != 0 means the top-level iterate starts at 0.
template <typename R, int DIM>
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(TailArgs<R> A, int gf, int gc, int zero) {
    pdl_enter();
    typedef typename CT<R>::T C;
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ TailArgs<R> S;
    if (threadIdx.x == 0) {
        S = A;
        C *p = (C *)tail_smem;
        S.bc = p;
        p += (A.nu_c + 1) & ~1;
        for (int l = 0; l < A.nlev; l++) {
            const size_t np = (size_t)A.lv[l].o.nx * A.lv[l].o.ny * (DIM == 3 ? A.lv[l].o.nz : 1);
            S.lv[l].b = p; p += np;
            S.lv[l].u = p; p += np;
            S.lv[l].t = p; p += np;
        }
        // then every level's coefficient triples and k^2 (read by every phase)
        for (int l = 0; l < A.nlev; l++) {
            OpView<R> &o = S.lv[l].o;
            const size_t np = (size_t)o.nx * o.ny * (DIM == 3 ? o.nz : 1);
            o.cx = p; p += 3 * o.nx;
            o.cy = p; p += 3 * o.ny;
            if (DIM == 3) { o.cz = p; p += 3 * o.nz; }
            o.k2 = (const R *)p;
            p = (C *)((unsigned char *)p + ((np * sizeof(R) + 15) & ~(size_t)15));
        }
    }
    __syncthreads();
    {
        const TailLevelDev<R> &last = S.lv[S.nlev - 1];
        const C *end = last.t + (size_t)last.o.nx * last.o.ny * (DIM == 3 ? last.o.nz : 1);
        const size_t total = end - (const C *)tail_smem;
        for (size_t q = threadIdx.x; q < total; q += blockDim.x) ((C *)tail_smem)[q] = mk(R(0), R(0));
        for (int l = 0; l < S.nlev; l++) {
            const OpView<R> &g = A.lv[l].o, &o = S.lv[l].o;
            const size_t np = (size_t)g.nx * g.ny * (DIM == 3 ? g.nz : 1);
            for (int q = threadIdx.x; q < 3 * g.nx; q += blockDim.x) const_cast<C *>(o.cx)[q] = g.cx[q];
            for (int q = threadIdx.x; q < 3 * g.ny; q += blockDim.x) const_cast<C *>(o.cy)[q] = g.cy[q];
            if (DIM == 3)
                for (int q = threadIdx.x; q < 3 * g.nz; q += blockDim.x) const_cast<C *>(o.cz)[q] = g.cz[q];
            for (size_t q = threadIdx.x; q < np; q += blockDim.x) const_cast<R *>(o.k2)[q] = g.k2[q];
        }
    }
    __syncthreads();
    const OpView<R> &o = A.lv[0].o;
    for_interior<DIM>(o.nx, o.ny, o.nz, [&](int i, int j, int k) {
        const size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k);
        S.lv[0].b[p] = A.lv[0].b[p];
        if (!zero) S.lv[0].u[p] = A.lv[0].u[p];
    });
    __syncthreads();
    tail_cycle<R, DIM, 0>(S, zero != 0, gf, gc);
    for_interior<DIM>(o.nx, o.ny, o.nz, [&](int i, int j, int k) {
        const size_t p = (size_t)i + (size_t)o.nx * ((size_t)j + (size_t)o.ny * k);
        A.lv[0].u[p] = S.lv[0].u[p];
    });
}

// Planes per thread of a 3D z-marching kernel: kmax, halved while the grid would have fewer than
// `target` blocks (small levels: more, shorter chains instead of a few long ones).
static int z_chunk(size_t tiles_xy, int planes, int kmax, size_t target) {
    int kc = kmax;
    while (kc > 1 && tiles_xy * cdiv(planes, kc) < target) kc /= 2;
    return kc;
}

dim3 grid_for(const int n[3], int dim) {
    return dim3(cdiv(n[0] - 2, BX), cdiv(n[1] - 2, BY), dim == 3 ? cdiv(n[2] - 2, KCHUNK) : 1);
}

}  // namespace

// ------------------------------------------------------------------------------ launchers
template <typename R, typename CX>
cudaError_t launch_apply(const DevOp<R> &op, int dim, const CX *x, typename CT<R>::T *y, cudaStream_t s) {
    dim3 g = grid_for(op.n, dim), b(BX, BY);
    if (dim == 3) launch_pdl(k_apply<R, 3, CX>, g, b, 0, s, view(op), x, y);
    else launch_pdl(k_apply<R, 2, CX>, g, b, 0, s, view(op), x, y);
    return cudaGetLastError();
}

template <typename R, typename CB>
cudaError_t launch_residual(const DevOp<R> &op, int dim, const CB *bb, const typename CT<R>::T *u,
                            typename CT<R>::T *r, cudaStream_t s) {
    dim3 g = grid_for(op.n, dim), b(BX, BY);
    if (dim == 3) launch_pdl(k_residual<R, 3, CB>, g, b, 0, s, view(op), bb, u, r);
    else launch_pdl(k_residual<R, 2, CB>, g, b, 0, s, view(op), bb, u, r);
    return cudaGetLastError();
}

template <typename R, typename CB>
cudaError_t launch_jacobi(const DevOp<R> &op, int dim, R omega, const CB *bb, const typename CT<R>::T *u_in,
                          typename CT<R>::T *u_out, cudaStream_t s) {
    dim3 g = grid_for(op.n, dim), b(BX, BY);
    if (dim == 3) {
        const int kc = z_chunk((size_t)g.x * g.y, op.n[2] - 2, KCHUNK, 152 * 10);
        g.z = cdiv(op.n[2] - 2, kc);
        if (u_in == nullptr) {
            switch (kc) {
            case 8: launch_pdl(k_jacobi3<R, CB, true, 8>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            case 4: launch_pdl(k_jacobi3<R, CB, true, 4>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            case 2: launch_pdl(k_jacobi3<R, CB, true, 2>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            default: launch_pdl(k_jacobi3<R, CB, true, 1>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            }
        } else {
            switch (kc) {
            case 8: launch_pdl(k_jacobi3<R, CB, false, 8>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            case 4: launch_pdl(k_jacobi3<R, CB, false, 4>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            case 2: launch_pdl(k_jacobi3<R, CB, false, 2>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            default: launch_pdl(k_jacobi3<R, CB, false, 1>, g, b, 0, s, view(op), omega, bb, u_in, u_out); break;
            }
        }
    } else if (u_in == nullptr) {
        launch_pdl(k_jacobi<R, 2, CB, true>, g, b, 0, s, view(op), omega, bb, u_in, u_out);
    } else {
        launch_pdl(k_jacobi<R, 2, CB, false>, g, b, 0, s, view(op), omega, bb, u_in, u_out);
    }
    return cudaGetLastError();
}

template <typename R, typename CB>
cudaError_t launch_rb(const DevOp<R> &op, int dim, R omega, const CB *bb, typename CT<R>::T *u, int colour,
                      cudaStream_t s) {
    dim3 g(cdiv((op.n[0] - 1) / 2, BX), cdiv(op.n[1] - 2, BY), dim == 3 ? cdiv(op.n[2] - 2, KCHUNK) : 1), b(BX, BY);
    if (dim == 3) launch_pdl(k_rb<R, 3, CB>, g, b, 0, s, view(op), omega, bb, u, colour);
    else launch_pdl(k_rb<R, 2, CB>, g, b, 0, s, view(op), omega, bb, u, colour);
    return cudaGetLastError();
}

template <typename R, typename CB>
cudaError_t launch_residual_restrict(const DevOp<R> &op, int dim, const CB *bb, const typename CT<R>::T *u,
                                     typename CT<R>::T *rc, cudaStream_t s) {
    int nc[3] = {(op.n[0] + 1) / 2, (op.n[1] + 1) / 2, dim == 3 ? (op.n[2] + 1) / 2 : 1};
    if (dim == 3 && (size_t)op.n[0] * op.n[1] < ((size_t)1 << 31)) {  // 32-bit in-plane offsets
        constexpr size_t smem = r3_smem_bytes<R>();
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_resrestrict3<R, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        dim3 g(cdiv(nc[0] - 2, R3_TX), cdiv(nc[1] - 2, R3_TY), 1);
        const int kc = z_chunk((size_t)g.x * g.y, nc[2] - 2, R3_KC, 152 * 4);
        g.z = cdiv(nc[2] - 2, kc);
        launch_pdl(k_resrestrict3<R, CB>, g, R3_NT, smem, s, view(op), bb, u, rc, nc[0], nc[1], nc[2], kc);
        return cudaGetLastError();
    }
    dim3 g = grid_for(nc, dim), b(BX, BY);
    if (dim == 3) launch_pdl(k_residual_restrict<R, 3, CB>, g, b, 0, s, view(op), bb, u, rc, nc[0], nc[1], nc[2]);
    else launch_pdl(k_residual_restrict<R, 2, CB>, g, b, 0, s, view(op), bb, u, rc, nc[0], nc[1], nc[2]);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prolong_add(const int nf[3], int dim, const typename CT<R>::T *ec, typename CT<R>::T *uf,
                               cudaStream_t s, const int *gate) {
    dim3 g = grid_for(nf, dim), b(BX, BY);
    if (dim == 3) {
        const int kc = z_chunk((size_t)g.x * g.y, nf[2] - 2, KCHUNK, 152 * 10);
        g.z = cdiv(nf[2] - 2, kc);
        launch_pdl(k_prolong3<R>, g, b, 0, s, nf[0], nf[1], nf[2], ec, uf, kc, gate);
    } else {
        launch_pdl(k_prolong_add<R, 2>, g, b, 0, s, nf[0], nf[1], 1, ec, uf, gate);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_dense_solve(const int n[3], int dim, int nu, const typename CT<R>::T *minv,
                               const typename CT<R>::T *b, typename CT<R>::T *u, cudaStream_t s) {
    const int threads = 256, warps = threads / 32;
    launch_pdl(k_dense_solve<R>, cdiv(nu, warps), threads, 0, s, n[0], n[1], dim == 3 ? n[2] : 1, dim, nu, minv, b, u);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mg_tail(int dim, int nlev, const DevOp<R> *ops, typename CT<R>::T *const *b,
                           typename CT<R>::T *const *u, typename CT<R>::T *const *t, const typename CT<R>::T *minv,
                           int nu_c, int nu1, int nu2, int rb, R omega, int gf, int gc, int zero, cudaStream_t s) {
    if (nlev < 2 || nlev > MAX_TAIL_LEVELS) return cudaErrorInvalidValue;
    TailArgs<R> A{};
    for (int l = 0; l < nlev; l++) {
        A.lv[l].o = view(ops[l]);
        if (dim != 3) A.lv[l].o.nz = 1;
        A.lv[l].b = b[l];
        A.lv[l].u = u[l];
        A.lv[l].t = t[l];
    }
    A.nlev = nlev;
    A.nu_c = nu_c;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.rb = rb;
    A.omega = omega;
    A.minv = minv;
    const size_t bytes = mg_tail_smem_bytes(dim, nlev, ops, nu_c, sizeof(typename CT<R>::T));
    if (bytes > TAIL_SMEM_BYTES) return cudaErrorInvalidValue;
    static bool attr_set[2] = {false, false};
    if (!attr_set[dim == 3]) {
        cudaError_t e = dim == 3 ? cudaFuncSetAttribute(k_mg_tail<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TAIL_SMEM_BYTES)
                                 : cudaFuncSetAttribute(k_mg_tail<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TAIL_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[dim == 3] = true;
    }
    if (dim == 3) launch_pdl(k_mg_tail<R, 3>, 1, TAIL_THREADS, bytes, s, A, gf, gc, zero);
    else launch_pdl(k_mg_tail<R, 2>, 1, TAIL_THREADS, bytes, s, A, gf, gc, zero);
    return cudaGetLastError();
}
template cudaError_t launch_mg_tail<float>(int, int, const DevOp<float> *, float2 *const *, float2 *const *,
                                           float2 *const *, const float2 *, int, int, int, int, float, int, int, int,
                                           cudaStream_t);
template cudaError_t launch_mg_tail<double>(int, int, const DevOp<double> *, double2 *const *, double2 *const *,
                                            double2 *const *, const double2 *, int, int, int, int, double, int, int,
                                            int, cudaStream_t);

// Tile shapes (coarse nodes per block) of the temporally blocked kernels, by tile index (the
// wavefront, HELM_TILE_WAVE, has none).
static const int kTiles[HELM_TILE_COUNT][2] = {{32, 8}, {16, 16}, {16, 8}, {64, 4}, {0, 0}, {8, 8}};

bool fused_jacobi2_ok(const int n[3], int dim, int tile) {
    if (tile == HELM_TILE_WAVE) return wave_jacobi2_ok(n, dim);
    if (tile < 0 || tile >= HELM_TILE_COUNT) return false;
    if (dim != 2 || (n[0] - 1) % 2 || (n[1] - 1) % 2) return false;
    const int ncx = (n[0] + 1) / 2, ncy = (n[1] + 1) / 2;
    // the last tile's owned range must reach the last interior node: a tile row or column
    // that ends exactly at the grid's edge would leave node n - 2 unowned
    return ncx >= 3 && ncy >= 3 && (ncx - 2) % kTiles[tile][0] != 0 && (ncy - 2) % kTiles[tile][1] != 0;
}

template <int TCX, int TCY>
static cudaError_t pre2_t(const DevOp<float> &op, float omega, const float2 *b, float2 *u_out, float2 *rc,
                          cudaStream_t s) {
    const int ncx = (op.n[0] + 1) / 2, ncy = (op.n[1] + 1) / 2;
    constexpr size_t smem = sizeof(typename Tile<TCX, TCY>::Pre);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pre2_restrict<TCX, TCY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g(cdiv(ncx - 2, TCX), cdiv(ncy - 2, TCY));
    launch_pdl(k_pre2_restrict<TCX, TCY>, g, Tile<TCX, TCY>::NT, smem, s, view(op), omega, b, u_out, rc, ncx, ncy);
    return cudaGetLastError();
}

template <int TCX, int TCY>
static cudaError_t post2_t(const DevOp<float> &op, float omega, const float2 *b, const float2 *u_in, float2 *u_out,
                           const float2 *ec, cudaStream_t s) {
    const int ncx = (op.n[0] + 1) / 2, ncy = (op.n[1] + 1) / 2;
    constexpr size_t smem = sizeof(typename Tile<TCX, TCY>::Post);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_prolong_post2<TCX, TCY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g(cdiv(ncx - 2, TCX), cdiv(ncy - 2, TCY));
    launch_pdl(k_prolong_post2<TCX, TCY>, g, Tile<TCX, TCY>::NT, smem, s, view(op), omega, b, u_in, u_out, ec, ncx,
               ncy);
    return cudaGetLastError();
}

cudaError_t launch_pre2_restrict(const DevOp<float> &op, int tile, float omega, const float2 *b, float2 *u_out,
                                 float2 *rc, cudaStream_t s) {
    if (!fused_jacobi2_ok(op.n, 2, tile) || (tile != HELM_TILE_WAVE && !op.dinv)) return cudaErrorInvalidValue;
    switch (tile) {
    case HELM_TILE_WAVE: return launch_pre2_wave(op, omega, b, u_out, rc, s);
    case 0: return pre2_t<32, 8>(op, omega, b, u_out, rc, s);
    case 1: return pre2_t<16, 16>(op, omega, b, u_out, rc, s);
    case 2: return pre2_t<16, 8>(op, omega, b, u_out, rc, s);
    case HELM_TILE_8x8: return pre2_t<8, 8>(op, omega, b, u_out, rc, s);
    default: return pre2_t<64, 4>(op, omega, b, u_out, rc, s);
    }
}

cudaError_t launch_prolong_post2(const DevOp<float> &op, int tile, float omega, const float2 *b, const float2 *u_in,
                                 float2 *u_out, const float2 *ec, cudaStream_t s) {
    if (!fused_jacobi2_ok(op.n, 2, tile) || (tile != HELM_TILE_WAVE && !op.dinv)) return cudaErrorInvalidValue;
    switch (tile) {
    case HELM_TILE_WAVE: return launch_post2_wave(op, omega, b, u_in, u_out, ec, s);
    case 0: return post2_t<32, 8>(op, omega, b, u_in, u_out, ec, s);
    case 1: return post2_t<16, 16>(op, omega, b, u_in, u_out, ec, s);
    case 2: return post2_t<16, 8>(op, omega, b, u_in, u_out, ec, s);
    case HELM_TILE_8x8: return post2_t<8, 8>(op, omega, b, u_in, u_out, ec, s);
    default: return post2_t<64, 4>(op, omega, b, u_in, u_out, ec, s);
    }
}

template <int TCX, int TCY>
static cudaError_t pre2_b_t(int n0, int n1, int count, const BLevel *tab, float omega, cudaStream_t s) {
    const int ncx = (n0 + 1) / 2, ncy = (n1 + 1) / 2;
    constexpr size_t smem = sizeof(typename Tile<TCX, TCY>::Pre);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_pre2_restrict_b<TCX, TCY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g(cdiv(ncx - 2, TCX), cdiv(ncy - 2, TCY), count);
    launch_pdl(k_pre2_restrict_b<TCX, TCY>, g, Tile<TCX, TCY>::NT, smem, s, tab, omega);
    return cudaGetLastError();
}

template <int TCX, int TCY>
static cudaError_t post2_b_t(int n0, int n1, int count, const BLevel *tab, float omega, int j, cudaStream_t s) {
    const int ncx = (n0 + 1) / 2, ncy = (n1 + 1) / 2;
    constexpr size_t smem = sizeof(typename Tile<TCX, TCY>::Post);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_prolong_post2_b<TCX, TCY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 g(cdiv(ncx - 2, TCX), cdiv(ncy - 2, TCY), count);
    launch_pdl(k_prolong_post2_b<TCX, TCY>, g, Tile<TCX, TCY>::NT, smem, s, tab, omega, j);
    return cudaGetLastError();
}

cudaError_t launch_pre2_restrict_batch(const int n[3], int tile, int count, const BLevel *tab, float omega,
                                       cudaStream_t s) {
    if (count < 1 || count > 65535 || tile == HELM_TILE_WAVE || !fused_jacobi2_ok(n, 2, tile)) return cudaErrorInvalidValue;
    switch (tile) {
    case 0: return pre2_b_t<32, 8>(n[0], n[1], count, tab, omega, s);
    case 1: return pre2_b_t<16, 16>(n[0], n[1], count, tab, omega, s);
    case 2: return pre2_b_t<16, 8>(n[0], n[1], count, tab, omega, s);
    case HELM_TILE_8x8: return pre2_b_t<8, 8>(n[0], n[1], count, tab, omega, s);
    default: return pre2_b_t<64, 4>(n[0], n[1], count, tab, omega, s);
    }
}

cudaError_t launch_prolong_post2_batch(const int n[3], int tile, int count, const BLevel *tab, float omega, int j,
                                       cudaStream_t s) {
    if (count < 1 || count > 65535 || tile == HELM_TILE_WAVE || !fused_jacobi2_ok(n, 2, tile)) return cudaErrorInvalidValue;
    switch (tile) {
    case 0: return post2_b_t<32, 8>(n[0], n[1], count, tab, omega, j, s);
    case 1: return post2_b_t<16, 16>(n[0], n[1], count, tab, omega, j, s);
    case 2: return post2_b_t<16, 8>(n[0], n[1], count, tab, omega, j, s);
    case HELM_TILE_8x8: return post2_b_t<8, 8>(n[0], n[1], count, tab, omega, j, s);
    default: return post2_b_t<64, 4>(n[0], n[1], count, tab, omega, j, s);
    }
}

template <typename CI, typename CO>
cudaError_t launch_convert(size_t n, const CI *in, CO *out, cudaStream_t s) {
    launch_pdl(k_convert<CI, CO>, (unsigned)std::min<size_t>(cdiv(n, 256), 152 * 16), 256, 0, s, n, in, out);
    return cudaGetLastError();
}

template <typename C> cudaError_t launch_zero(size_t n, C *x, cudaStream_t s) {
    launch_pdl(k_zero<C>, (unsigned)std::min<size_t>(cdiv(n, 256), 152 * 16), 256, 0, s, n, x);
    return cudaGetLastError();
}

#define INST_R(R)                                                                                               \
    template cudaError_t launch_residual<R, CT<R>::T>(const DevOp<R> &, int, const CT<R>::T *, const CT<R>::T *, \
                                                       CT<R>::T *, cudaStream_t);                               \
    template cudaError_t launch_jacobi<R, CT<R>::T>(const DevOp<R> &, int, R, const CT<R>::T *, const CT<R>::T *, \
                                                     CT<R>::T *, cudaStream_t);                                 \
    template cudaError_t launch_rb<R, CT<R>::T>(const DevOp<R> &, int, R, const CT<R>::T *, CT<R>::T *, int,     \
                                                 cudaStream_t);                                                 \
    template cudaError_t launch_residual_restrict<R, CT<R>::T>(const DevOp<R> &, int, const CT<R>::T *,          \
                                                                const CT<R>::T *, CT<R>::T *, cudaStream_t);    \
    template cudaError_t launch_prolong_add<R>(const int *, int, const CT<R>::T *, CT<R>::T *, cudaStream_t,      \
                                               const int *);                                                   \
    template cudaError_t launch_dense_solve<R>(const int *, int, int, const CT<R>::T *, const CT<R>::T *,        \
                                                CT<R>::T *, cudaStream_t);
INST_R(float)
INST_R(double)
template cudaError_t launch_apply<double, double2>(const DevOp<double> &, int, const double2 *, double2 *, cudaStream_t);
template cudaError_t launch_apply<double, float2>(const DevOp<double> &, int, const float2 *, double2 *, cudaStream_t);
template cudaError_t launch_apply<float, float2>(const DevOp<float> &, int, const float2 *, float2 *, cudaStream_t);
template cudaError_t launch_convert<double2, float2>(size_t, const double2 *, float2 *, cudaStream_t);
template cudaError_t launch_convert<float2, double2>(size_t, const float2 *, double2 *, cudaStream_t);
template cudaError_t launch_convert<double2, double2>(size_t, const double2 *, double2 *, cudaStream_t);
template cudaError_t launch_convert<float2, float2>(size_t, const float2 *, float2 *, cudaStream_t);
template cudaError_t launch_zero<double2>(size_t, double2 *, cudaStream_t);
template cudaError_t launch_zero<float2>(size_t, float2 *, cudaStream_t);

// ------------------------------------------------------------------------------ 1 / diagonal
namespace {
__global__ void k_diag_inv(OpView<float> o, float2 *__restrict__ dinv) {
    pdl_enter();
    const size_t n = (size_t)o.nx * o.ny;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % o.nx), y = (int)(p / o.nx);
        float2 v = make_float2(0.f, 0.f);
        if (x >= 1 && x <= o.nx - 2 && y >= 1 && y <= o.ny - 2) {
            const float2 d = cadd(cadd(o.cx[3 * x + 1], o.cy[3 * y + 1]), cadd(cscale(o.bk, o.k2[p]), o.c));
            v = cinv_fast(d);
        }
        dinv[p] = v;
    }
}
}  // namespace

cudaError_t launch_diag_inv(const DevOp<float> &op, float2 *dinv, cudaStream_t s) {
    const size_t n = (size_t)op.n[0] * op.n[1];
    launch_pdl(k_diag_inv, (unsigned)std::min<size_t>(cdiv(n, 256), 152 * 8), 256, 0, s, view(op), dinv);
    return cudaGetLastError();
}
