// Register-wavefront variants of the temporally blocked V(2,2) omega-Jacobi kernels (2D,
// complex64): the same two launches per level as k_pre2_restrict / k_prolong_post2 (two sweeps
// from zero + residual + full weighting; prolongation + two sweeps) with the same arithmetic,
// but without shared memory or block barriers.  One warp owns a strip of WV_CX coarse columns
// (2 WV_CX fine columns; lane = fine column, with a halo of 3 columns on each side) and a band of
// WV_TJ coarse rows, and marches down the fine rows with the stages pipelined: at row y it forms
// the first sweep at y, the second sweep at y - 1, the residual at y - 2 and, on coincident
// rows, the full weighting of coarse row (y - 3) / 2.  x-neighbours come from warp shuffles,
// y-neighbours from a sliding window of rows held in registers.
#include "helm_internal.h"

namespace {

// Operator view: per-axis coefficient triples (cw, cc, ce) per node, k^2, and the diagonal
// shift (bk k^2 + c); the same operator as DevOp<float>.
struct WaveOp {
    const float2 *cx, *cy;
    const float *k2;
    float2 bk, c;
    int nx, ny;
    const int *gate;  // see DevOp::gate
};

constexpr int WV_CX = 13;  // coarse columns per warp (26 owned fine columns of 32 lanes)
constexpr int WV_TJ = 8;   // coarse rows per warp
constexpr int WV_WARPS = 4;

__device__ __forceinline__ float2 shfl_up_c(float2 v) {  // value of lane - 1 (lane 0: own)
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_dn_c(float2 v) {  // value of lane + 1 (lane 31: own)
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

struct RowCoef {
    float2 w, c, e;  // y coefficients of a row (zero outside the interior)
};

__device__ __forceinline__ RowCoef row_coef(const WaveOp &o, int y) {
    RowCoef r;
    const float2 z = make_float2(0.f, 0.f);
    const bool in = y >= 1 && y <= o.ny - 2;
    r.w = in ? o.cy[3 * y] : z;
    r.c = in ? o.cy[3 * y + 1] : z;
    r.e = in ? o.cy[3 * y + 2] : z;
    return r;
}

// Inputs of one row at the lane's column: b, k^2 (zero outside the interior) and the row's y
// coefficients.
struct RowIn {
    float2 b;
    float k2;
    RowCoef ry;
};
__device__ __forceinline__ RowIn load_row_in(const WaveOp &o, const float2 *__restrict__ b, int x, bool xin, int y) {
    RowIn r;
    r.ry = row_coef(o, y);
    const bool in = xin && y >= 1 && y <= o.ny - 2;
    const size_t p = (size_t)(in ? x : 1) + (size_t)o.nx * (size_t)(in ? y : 1);  // in range either way
    r.b = in ? b[p] : make_float2(0.f, 0.f);
    r.k2 = in ? o.k2[p] : 0.f;
    return r;
}

// (M u)(x, y) from the row's values (u, its x-neighbours uw, ue, the rows above and below un,
// us) and the coefficients; d = the diagonal.
__device__ __forceinline__ float2 wave_apply(float2 cxw, float2 cxe, const RowCoef &ry, float2 d, float2 u, float2 uw,
                                             float2 ue, float2 un, float2 us) {
    float2 acc = cmul(cxw, uw);
    acc = cfma(cxe, ue, acc);
    acc = cfma(ry.w, un, acc);
    acc = cfma(ry.e, us, acc);
    return cfma(d, u, acc);
}

__device__ __forceinline__ void wave_geometry(int ncx, int ncy, int &I0, int &J0, bool &live) {
    const int wid = blockIdx.x * WV_WARPS + (threadIdx.x >> 5);
    const int nsx = (ncx - 2 + WV_CX - 1) / WV_CX;
    const int sx = wid % nsx, sy = wid / nsx;
    I0 = 1 + sx * WV_CX;
    J0 = 1 + sy * WV_TJ;
    live = J0 <= ncy - 2;  // warp-uniform
}

// Pre-smoothing: u = two sweeps from zero (owned fine nodes), rc = FW(b - M u) (owned coarse).
__global__ void __launch_bounds__(32 * WV_WARPS) k_pre2_wave(WaveOp o, float omega, const float2 *__restrict__ b,
                                                             float2 *__restrict__ u, float2 *__restrict__ rc, int ncx,
                                                             int ncy) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    int I0, J0;
    bool live;
    wave_geometry(ncx, ncy, I0, J0, live);
    if (!live) return;
    const int lane = threadIdx.x & 31, nx = o.nx, ny = o.ny;
    const int x = 2 * I0 - 4 + lane;
    const bool xin = x >= 1 && x <= nx - 2;
    const float2 z = make_float2(0.f, 0.f);
    const float2 cxw = xin ? o.cx[3 * x] : z, cxc = xin ? o.cx[3 * x + 1] : z, cxe = xin ? o.cx[3 * x + 2] : z;
    const bool own_x = lane >= 3 && lane <= 28 && xin;                        // owned fine column
    const bool fw_x = own_x && ((x & 1) == 0) && (x >> 1) <= ncx - 2;          // coarse column x / 2
    const int y0 = 2 * J0 - 3, y1 = 2 * J0 + 2 * WV_TJ + 1;                    // rows marched
    const int own_y0 = 2 * J0 - 1, own_y1 = 2 * J0 + 2 * WV_TJ - 1;            // owned fine rows
    // sliding windows (index 0 = the oldest row)
    float2 u1[3] = {z, z, z}, bb[3] = {z, z, z}, dd[3] = {z, z, z}, iv[3] = {z, z, z};
    RowCoef ry[3] = {{z, z, z}, {z, z, z}, {z, z, z}};
    float2 u2[3] = {z, z, z}, ax[3] = {z, z, z};
    // row inputs are loaded two rows ahead of their use
    RowIn pf[2];
    pf[0] = load_row_in(o, b, x, xin, y0);
    pf[1] = load_row_in(o, b, x, xin, y0 + 1);
    for (int y = y0; y <= y1; y++) {
        const RowIn cur = pf[0];
        pf[0] = pf[1];
        pf[1] = load_row_in(o, b, x, xin, y + 2);
        // shift windows; row y enters at index 2
        u1[0] = u1[1]; u1[1] = u1[2];
        bb[0] = bb[1]; bb[1] = bb[2];
        dd[0] = dd[1]; dd[1] = dd[2];
        iv[0] = iv[1]; iv[1] = iv[2];
        ry[0] = ry[1]; ry[1] = ry[2];
        ry[2] = cur.ry;
        const bool in = xin && y >= 1 && y <= ny - 2;
        float2 bv = z, dv = z, inv = z, v1 = z;
        if (in) {
            bv = cur.b;
            dv = cadd(cadd(cxc, ry[2].c), cadd(cscale(o.bk, cur.k2), o.c));
            inv = cscale(cinv_fast(dv), omega);
            v1 = cmul(bv, inv);  // first sweep from zero
        }
        bb[2] = bv; dd[2] = dv; iv[2] = inv; u1[2] = v1;
        // second sweep at row y - 1 (window index 1)
        {
            const int yy = y - 1;
            const float2 w1 = shfl_up_c(u1[1]), e1 = shfl_dn_c(u1[1]);
            float2 v2 = z;
            if (xin && yy >= 1 && yy <= ny - 2) {
                const float2 mu = wave_apply(cxw, cxe, ry[1], dd[1], u1[1], w1, e1, u1[0], u1[2]);
                v2 = cadd(u1[1], cmul(csub(bb[1], mu), iv[1]));
            }
            u2[0] = u2[1]; u2[1] = u2[2]; u2[2] = v2;
            if (own_x && yy >= own_y0 && yy < own_y1 && yy <= ny - 2 && yy >= 1) u[(size_t)x + (size_t)nx * yy] = v2;
        }
        // residual at row y - 2 (windows: u2 index 1, b/d/coef index 0), filtered along x
        {
            const int yy = y - 2;
            const float2 w2 = shfl_up_c(u2[1]), e2 = shfl_dn_c(u2[1]);
            float2 r = z;
            if (xin && yy >= 1 && yy <= ny - 2)
                r = csub(bb[0], wave_apply(cxw, cxe, ry[0], dd[0], u2[1], w2, e2, u2[0], u2[2]));
            // (1, 2, 1) along x
            const float2 rw = shfl_up_c(r), re = shfl_dn_c(r);
            ax[0] = ax[1]; ax[1] = ax[2];
            ax[2] = cadd(cadd(rw, re), cscale(r, 2.f));
        }
        // full weighting of coarse row (y - 3) / 2: rows y - 4, y - 3, y - 2 of the filtered residual
        {
            const int yc = y - 3;
            if (((yc & 1) == 0) && fw_x) {
                const int J = yc >> 1;
                if (J >= J0 && J < J0 + WV_TJ && J <= ncy - 2)
                    rc[(size_t)(x >> 1) + (size_t)ncx * J] = cscale(cadd(cadd(ax[0], ax[2]), cscale(ax[1], 2.f)), 0.0625f);
            }
        }
    }
}

// Post-smoothing: u_out = two sweeps of (u_in + P ec) on the owned fine nodes (halo 2).
__global__ void __launch_bounds__(32 * WV_WARPS) k_post2_wave(WaveOp o, float omega, const float2 *__restrict__ b,
                                                              const float2 *__restrict__ u_in, float2 *__restrict__ u,
                                                              const float2 *__restrict__ ec, int ncx, int ncy) {
    pdl_enter();
    if (o.gate && *o.gate) return;
    int I0, J0;
    bool live;
    wave_geometry(ncx, ncy, I0, J0, live);
    if (!live) return;
    const int lane = threadIdx.x & 31, nx = o.nx, ny = o.ny;
    const int x = 2 * I0 - 4 + lane;
    const bool xin = x >= 1 && x <= nx - 2;
    const float2 z = make_float2(0.f, 0.f);
    const float2 cxw = xin ? o.cx[3 * x] : z, cxc = xin ? o.cx[3 * x + 1] : z, cxe = xin ? o.cx[3 * x + 2] : z;
    const bool own_x = lane >= 3 && lane <= 28 && xin;
    const int own_y0 = 2 * J0 - 1, own_y1 = 2 * J0 + 2 * WV_TJ - 1;
    const int y0 = own_y0 - 2, y1 = own_y1 + 1;  // the sweeps need two rows of halo
    const int xa = x >> 1, xb = (x + 1) >> 1;  // coarse columns of the interpolation
    const bool ca = xa >= 0 && xa < ncx, cb = xb >= 0 && xb < ncx;
    float2 u3[3] = {z, z, z}, bb[3] = {z, z, z}, dd[3] = {z, z, z}, iv[3] = {z, z, z}, u4[3] = {z, z, z};
    RowCoef ry[3] = {{z, z, z}, {z, z, z}, {z, z, z}};
    // row inputs (b, k^2, the iterate, and the interpolated correction) two rows ahead
    struct PostIn {
        RowIn r;
        float2 u, e;
    };
    auto load_post = [&](int yy) {
        PostIn q;
        q.r = load_row_in(o, b, x, xin, yy);
        q.u = z;
        q.e = z;
        if (xin && yy >= 1 && yy <= ny - 2) {
            q.u = u_in[(size_t)x + (size_t)nx * yy];
            const int ya = yy >> 1, yb = (yy + 1) >> 1;
            const float2 e00 = ca ? ec[(size_t)xa + (size_t)ncx * ya] : z, e01 = cb ? ec[(size_t)xb + (size_t)ncx * ya] : z;
            const float2 e10 = ca ? ec[(size_t)xa + (size_t)ncx * yb] : z, e11 = cb ? ec[(size_t)xb + (size_t)ncx * yb] : z;
            q.e = cadd(cadd(e00, e01), cadd(e10, e11));
        }
        return q;
    };
    PostIn pf[2];
    pf[0] = load_post(y0);
    pf[1] = load_post(y0 + 1);
    for (int y = y0; y <= y1; y++) {
        const PostIn cur = pf[0];
        pf[0] = pf[1];
        pf[1] = load_post(y + 2);
        u3[0] = u3[1]; u3[1] = u3[2];
        bb[0] = bb[1]; bb[1] = bb[2];
        dd[0] = dd[1]; dd[1] = dd[2];
        iv[0] = iv[1]; iv[1] = iv[2];
        ry[0] = ry[1]; ry[1] = ry[2];
        ry[2] = cur.r.ry;
        const bool in = xin && y >= 1 && y <= ny - 2;
        float2 bv = z, dv = z, inv = z, v3 = z;
        if (in) {
            bv = cur.r.b;
            dv = cadd(cadd(cxc, ry[2].c), cadd(cscale(o.bk, cur.r.k2), o.c));
            inv = cscale(cinv_fast(dv), omega);
            v3 = cadd(cur.u, cscale(cur.e, 0.25f));
        }
        bb[2] = bv; dd[2] = dv; iv[2] = inv; u3[2] = v3;
        // first post-sweep at row y - 1
        {
            const int yy = y - 1;
            const float2 w3 = shfl_up_c(u3[1]), e3 = shfl_dn_c(u3[1]);
            float2 v4 = z;
            if (xin && yy >= 1 && yy <= ny - 2) {
                const float2 mu = wave_apply(cxw, cxe, ry[1], dd[1], u3[1], w3, e3, u3[0], u3[2]);
                v4 = cadd(u3[1], cmul(csub(bb[1], mu), iv[1]));
            }
            u4[0] = u4[1]; u4[1] = u4[2]; u4[2] = v4;
        }
        // second post-sweep at row y - 2, stored on the owned nodes
        {
            const int yy = y - 2;
            const float2 w4 = shfl_up_c(u4[1]), e4 = shfl_dn_c(u4[1]);
            if (own_x && yy >= own_y0 && yy < own_y1 && yy >= 1 && yy <= ny - 2) {
                const float2 mu = wave_apply(cxw, cxe, ry[0], dd[0], u4[1], w4, e4, u4[0], u4[2]);
                u[(size_t)x + (size_t)nx * yy] = cadd(u4[1], cmul(csub(bb[0], mu), iv[0]));
            }
        }
    }
}

}  // namespace

bool wave_jacobi2_ok(const int n[3], int dim) {
    if (dim != 2 || (n[0] - 1) % 2 || (n[1] - 1) % 2) return false;
    const int ncx = (n[0] + 1) / 2, ncy = (n[1] + 1) / 2;
    // a strip or band that ends exactly at the grid's last interior coarse node would leave
    // fine node n - 2 unowned
    return ncx >= 3 && ncy >= 3 && (ncx - 2) % WV_CX != 0 && (ncy - 2) % WV_TJ != 0;
}

static unsigned wave_blocks(const int n[3]) {
    const int ncx = (n[0] + 1) / 2, ncy = (n[1] + 1) / 2;
    const int warps = ((ncx - 2 + WV_CX - 1) / WV_CX) * ((ncy - 2 + WV_TJ - 1) / WV_TJ);
    return (unsigned)((warps + WV_WARPS - 1) / WV_WARPS);
}

cudaError_t launch_pre2_wave(const DevOp<float> &op, float omega, const float2 *b, float2 *u_out, float2 *rc,
                             cudaStream_t s) {
    if (!wave_jacobi2_ok(op.n, 2)) return cudaErrorInvalidValue;
    const WaveOp v{op.coef[0], op.coef[1], op.k2, op.bk, op.c, op.n[0], op.n[1], op.gate};
    const int ncx = (op.n[0] + 1) / 2, ncy = (op.n[1] + 1) / 2;
    return launch_pdl(k_pre2_wave, wave_blocks(op.n), 32 * WV_WARPS, 0, s, v, omega, b, u_out, rc, ncx, ncy);
}

cudaError_t launch_post2_wave(const DevOp<float> &op, float omega, const float2 *b, const float2 *u_in, float2 *u_out,
                              const float2 *ec, cudaStream_t s) {
    if (!wave_jacobi2_ok(op.n, 2)) return cudaErrorInvalidValue;
    const WaveOp v{op.coef[0], op.coef[1], op.k2, op.bk, op.c, op.n[0], op.n[1], op.gate};
    const int ncx = (op.n[0] + 1) / 2, ncy = (op.n[1] + 1) / 2;
    return launch_pdl(k_post2_wave, wave_blocks(op.n), 32 * WV_WARPS, 0, s, v, omega, b, u_in, u_out, ec, ncx, ncy);
}
