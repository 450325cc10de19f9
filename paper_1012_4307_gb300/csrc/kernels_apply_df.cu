// w = A z for the Helmholtz operator A = L_h - k^2 (Section 3.2 stencil) with a complex64 z
// (the output of the complex64 multigrid preconditioner), computed in double-FP32 arithmetic
// on the FP32 units.  A's coefficients and k^2 are stored pre-split as float pairs; z is exact
// in FP32, so each product a * z is error-free up to the dropped a.lo * z rounding (2^-48
// relative); the sum over the stencil is kept with TwoSum and written as a float-pair vector
// (float4 (re.hi, re.lo, im.hi, im.lo) per node), the form the double-FP32 Gram-Schmidt reads.
// Same operands as k_apply<double, 2|3, float2> in kernels_mg.cu, which does the work with FP64
// fused multiply-adds.
#include "helm_internal.h"
#include "df_arith.h"

namespace {

constexpr int BX = 32, BY = 8, KCHUNK = 8;

// acc += a * z with a = (re.hi, re.lo, im.hi, im.lo) and a float complex z.
__device__ __forceinline__ void cmac(float4 a, float2 z, float &sr, float &cr, float &si, float &ci) {
    const ff ar{a.x, a.y}, ai{a.z, a.w};
    float p, e;
    ff_prod_f(ar, z.x, p, e);
    ff_acc_prod(sr, cr, p, e);
    ff_prod_f(ai, z.y, p, e);
    ff_acc_prod(sr, cr, -p, -e);
    ff_prod_f(ar, z.y, p, e);
    ff_acc_prod(si, ci, p, e);
    ff_prod_f(ai, z.x, p, e);
    ff_acc_prod(si, ci, p, e);
}

// The first term of the sums: (sr, cr) and (si, ci) start as its exact products (what adding
// them to zero accumulators with TwoSum gives, up to the sign of a zero).
__device__ __forceinline__ void cmac_first(float4 a, float2 z, float &sr, float &cr, float &si, float &ci) {
    const ff ar{a.x, a.y}, ai{a.z, a.w};
    float p, e;
    ff_prod_f(ar, z.x, sr, cr);
    ff_prod_f(ai, z.y, p, e);
    ff_acc_prod(sr, cr, -p, -e);
    ff_prod_f(ar, z.y, si, ci);
    ff_prod_f(ai, z.x, p, e);
    ff_acc_prod(si, ci, p, e);
}

// (bx, by, bz): this block's tile of interior nodes.  GATED: gv != 0 (a gate flag's value)
// returns once the first operands have been loaded, writing nothing (the 2D form then loads a
// node's operands before its arithmetic; without the gate they are loaded as the arithmetic
// uses them, which keeps the batched kernel at 32 registers).
template <int DIM, bool GATED>
__device__ __forceinline__ void apply_A_df_tile(const DevOpDF &o, const float2 *__restrict__ z, float4 *__restrict__ y,
                                                int bx, int by, int bz, int gv = 0) {
    const int nx = o.n[0], ny = o.n[1], nz = o.n[2];
    const int i = bx * BX + threadIdx.x + 1;
    const int j = by * BY + threadIdx.y + 1;
    if (i > nx - 2 || j > ny - 2) return;
    int k0 = 0, k1 = 1;
    if (DIM == 3) {
        k0 = bz * KCHUNK + 1;
        k1 = min(k0 + KCHUNK, nz - 1);
    }
    const size_t sy = (size_t)nx, sz = (size_t)nx * ny;
    const float4 cxw = o.coef[0][3 * i], cxc = o.coef[0][3 * i + 1], cxe = o.coef[0][3 * i + 2];
    const float4 cyw = o.coef[1][3 * j], cyc = o.coef[1][3 * j + 1], cye = o.coef[1][3 * j + 2];
    const ff dxy_r = ff_add(ff{cxc.x, cxc.y}, ff{cyc.x, cyc.y}), dxy_i = ff_add(ff{cxc.z, cxc.w}, ff{cyc.z, cyc.w});
    if constexpr (DIM == 3) {
        // march in z with the column (z - 1, z, z + 1) in registers and the next plane's
        // operands loaded while this plane is processed (same arithmetic order as the 2D branch)
        size_t p = (size_t)i + sy * ((size_t)j + (size_t)ny * k0);
        float2 zm = z[p - sz], zc = z[p];
        float2 zw = z[p - 1], ze = z[p + 1], zs = z[p - sy], zn = z[p + sy], zp = z[p + sz];
        float2 kk = o.k2[p];
        if (GATED && gv) return;
        for (int k = k0; k < k1; k++, p += sz) {
            float2 zw2 = zw, ze2 = ze, zs2 = zs, zn2 = zn, zp2 = zp, kk2 = kk;
            if (k + 1 < k1) {
                const size_t q = p + sz;
                zw2 = z[q - 1];
                ze2 = z[q + 1];
                zs2 = z[q - sy];
                zn2 = z[q + sy];
                zp2 = z[q + sz];
                kk2 = o.k2[q];
            }
            float sr, cr, si, ci;
            cmac_first(cxw, zw, sr, cr, si, ci);
            cmac(cxe, ze, sr, cr, si, ci);
            cmac(cyw, zs, sr, cr, si, ci);
            cmac(cye, zn, sr, cr, si, ci);
            ff dr = dxy_r, di = dxy_i;
            const float4 czw = o.coef[2][3 * k], czc = o.coef[2][3 * k + 1], cze = o.coef[2][3 * k + 2];
            cmac(czw, zm, sr, cr, si, ci);
            cmac(cze, zp, sr, cr, si, ci);
            dr = ff_add(dr, ff{czc.x, czc.y});
            di = ff_add(di, ff{czc.z, czc.w});
            dr = ff_add(dr, ff{-kk.x, -kk.y});
            cmac(make_float4(dr.hi, dr.lo, di.hi, di.lo), zc, sr, cr, si, ci);
            const ff yr = ff_norm(sr, cr), yi = ff_norm(si, ci);
            y[p] = make_float4(yr.hi, yr.lo, yi.hi, yi.lo);
            zm = zc;
            zc = zp;
            zw = zw2; ze = ze2; zs = zs2; zn = zn2; zp = zp2; kk = kk2;
        }
    } else {
        for (int k = k0; k < k1; k++) {
            const size_t p = (size_t)i + sy * ((size_t)j + (size_t)ny * k);
            float sr, cr, si, ci;
            ff dr = dxy_r, di = dxy_i;
            float2 zc;
            if constexpr (GATED) {
                const float2 zw = z[p - 1], ze = z[p + 1], zs = z[p - sy], zn = z[p + sy];
                const float2 kk = o.k2[p];
                zc = z[p];
                if (gv) return;
                cmac_first(cxw, zw, sr, cr, si, ci);
                cmac(cxe, ze, sr, cr, si, ci);
                cmac(cyw, zs, sr, cr, si, ci);
                cmac(cye, zn, sr, cr, si, ci);
                dr = ff_add(dr, ff{-kk.x, -kk.y});  // diagonal: sum of centre coefficients - k^2
            } else {
                cmac_first(cxw, z[p - 1], sr, cr, si, ci);
                cmac(cxe, z[p + 1], sr, cr, si, ci);
                cmac(cyw, z[p - sy], sr, cr, si, ci);
                cmac(cye, z[p + sy], sr, cr, si, ci);
                const float2 kk = o.k2[p];
                dr = ff_add(dr, ff{-kk.x, -kk.y});
                zc = z[p];
            }
            cmac(make_float4(dr.hi, dr.lo, di.hi, di.lo), zc, sr, cr, si, ci);
            const ff yr = ff_norm(sr, cr), yi = ff_norm(si, ci);
            y[p] = make_float4(yr.hi, yr.lo, yi.hi, yi.lo);
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(BX *BY) k_apply_A_df(DevOpDF o, const float2 *__restrict__ z, float4 *__restrict__ y,
                                                       const int *__restrict__ gate) {
    pdl_enter();
    const int gv = gate_value(gate);
    apply_A_df_tile<DIM, true>(o, z, y, blockIdx.x, blockIdx.y, blockIdx.z, gv);
}

// Batched 2D apply of step j over many problems: problem e takes the flat blocks
// [first[e], first[e + 1]) (its tiles, x fastest); z = its complex64 slot j, y = basis slot j + 1.
__global__ void __launch_bounds__(BX *BY) k_apply_A_df_b(const BVec *__restrict__ tab, const unsigned *__restrict__ first,
                                                         int count, int j) {
    pdl_enter();
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const BVec &P = tab[lo];
    if (*P.active == 0) return;
    const int t = (int)(blockIdx.x - first[lo]), tx = (P.A.n[0] - 2 + BX - 1) / BX;
    apply_A_df_tile<2, false>(P.A, P.Z + (size_t)j * P.n, P.V + (size_t)(j + 1) * P.n, t % tx, t / tx, 0);
}

}  // namespace

// Flat blocks of one problem's batched 2D apply.
unsigned apply_A_df_blocks(const int n[3]) { return cdiv(n[0] - 2, BX) * cdiv(n[1] - 2, BY); }

cudaError_t launch_apply_A_df_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                    cudaStream_t s) {
    if (count < 1 || j < 0 || j > 63 || nblocks < (unsigned)count) return cudaErrorInvalidValue;
    launch_pdl(k_apply_A_df_b, dim3(nblocks), dim3(BX, BY), 0, s, tab, first, count, j);
    return cudaGetLastError();
}

cudaError_t launch_apply_A_df(const DevOpDF &op, int dim, const float2 *z, float4 *y, cudaStream_t s,
                              const int *gate) {
    dim3 g(cdiv(op.n[0] - 2, BX), cdiv(op.n[1] - 2, BY), dim == 3 ? cdiv(op.n[2] - 2, KCHUNK) : 1), b(BX, BY);
    if (dim == 3) launch_pdl(k_apply_A_df<3>, g, b, 0, s, op, z, y, gate);
    else launch_pdl(k_apply_A_df<2>, g, b, 0, s, op, z, y, gate);
    return cudaGetLastError();
}
