// Gram-Schmidt passes of flexible GMRES in double-FP32 ("double-float") arithmetic on the FP32
// units, with the Krylov basis stored as float pairs.
//
// Why: on GB300 the FP64 pipe retires about 2 fused multiply-adds per SM per clock, 64 times
// fewer than FP32, so FP64 inner products over the Krylov basis are bound by FP64 issue, not
// by DRAM.  Here each basis vector is a "float-pair vector": node q holds the float4
// (re.hi, re.lo, im.hi, im.lo), an unevaluated sum hi + lo per component (16 bytes per node,
// the size of a double2).  Vectors enter that form once (an FP64 vector is split exactly
// with integer instructions: hi = the leading 24 significand bits, lo = the next 29 rounded
// to 24, 47 bits kept) and the double-float kernels write it directly, so the inner loops do
// no conversion: products are error-free with FMA (Dekker/Ogita-Rump-Oishi TwoProduct), sums
// use Knuth's TwoSum, and inner products are rounded to FP64 once per block.  A product's
// relative error is about 2^-46 and a sum's about 2^-48: FP64-class accuracy at FP32
// throughput.  Magnitudes below 2^-126 are flushed (their contribution to products with
// unit-norm basis vectors is far below the FP64 rounding of the results).
//
// Same partials layout and gate as k_mdot_norm / k_update_norm in kernels_krylov.cu.
#include "helm_internal.h"
#include "df_arith.h"
#include "dcgs2_coef.cuh"

namespace {

constexpr int NT = 256;

__device__ __forceinline__ ff shfl_down_ff(ff v, int off) {
    v.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    v.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return v;
}


// Block sums of NV double-float values per thread (fixed tree); thread t < NV gets sum t as
// an FP64 number in out[t].
// For NV a power of two (2 .. 32) the warp stage is a transposing butterfly: at offsets 16, 8,
// ... a lane keeps half of its values, sends the other half to the lane at that offset and adds
// what it receives, so the values per lane halve at every level (NV - 1 + the plain levels
// additions per lane instead of 5 NV); after log2(NV) levels lane l holds a partial sum of value
// idx(l), and the remaining levels sum equal indices.  Otherwise one shuffle tree per value.
template <int NV>
__device__ __forceinline__ void block_sum_ff(ff (&v)[NV], double *out) {
    __shared__ ff red[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (NV >= 2 && NV <= 32 && (NV & (NV - 1)) == 0) {
        int idx = 0;
#pragma unroll
        for (int o = 16, m = NV; o > 0; o >>= 1) {
            if (m > 1) {
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < m / 2; i++) {
                    const ff keep = upper ? v[i + m / 2] : v[i];
                    ff send = upper ? v[i] : v[i + m / 2];
                    send.hi = __shfl_xor_sync(0xffffffffu, send.hi, o);
                    send.lo = __shfl_xor_sync(0xffffffffu, send.lo, o);
                    v[i] = ff_add(keep, send);
                }
                if (upper) idx += m / 2;
                m /= 2;
            } else {
                ff r = v[0];
                r.hi = __shfl_xor_sync(0xffffffffu, r.hi, o);
                r.lo = __shfl_xor_sync(0xffffffffu, r.lo, o);
                v[0] = ff_add(v[0], r);
            }
        }
        if ((lane & (32 / NV - 1)) == 0) red[warp][idx] = v[0];
    } else {
#pragma unroll
        for (int i = 0; i < NV; i++) {
            ff x = v[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x = ff_add(x, shfl_down_ff(x, off));
            if (lane == 0) red[warp][i] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        ff s = red[0][threadIdx.x];
        for (int w = 1; w < NT / 32; w++) s = ff_add(s, red[w][threadIdx.x]);
        out[threadIdx.x] = ff_to_double(s);
    }
}

__device__ __forceinline__ ff ff_re(float4 v) { return ff{v.x, v.y}; }
__device__ __forceinline__ ff ff_im(float4 v) { return ff{v.z, v.w}; }

// partials[i * G + b] = sum conj(V_i) w (i in this block row's chunk), chunk 0 also
// partials[nv * G + b] = (||w||^2, 0).  V and w hold float pairs; no splitting is needed.
template <int CH>
__global__ void __launch_bounds__(NT) k_mdot_norm_pair(size_t n, const float4 *__restrict__ V, size_t ldv, int nv,
                                                       const float4 *__restrict__ w, double2 *__restrict__ partials,
                                                       const int *__restrict__ gate) {
    pdl_enter();
    if (gate && *gate == 0) return;
    __shared__ double sums[2 * CH + 1];
    const int i0 = blockIdx.y * CH;
    const int cnt = min(CH, nv - i0);
    const bool first = blockIdx.y == 0;
    float sr[CH], cr[CH], si[CH], ci[CH];
    float sn = 0.f, cn = 0.f;
#pragma unroll
    for (int t = 0; t < CH; t++) sr[t] = cr[t] = si[t] = ci[t] = 0.f;
    const size_t stride = (size_t)gridDim.x * NT;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // software pipeline: the next node's operands are loaded while this node is processed
    size_t q = blockIdx.x * (size_t)NT + threadIdx.x;
    float4 wcur = zero4, vcur[CH];
#pragma unroll
    for (int t = 0; t < CH; t++) vcur[t] = zero4;
    if (q < n) {
        wcur = w[q];
#pragma unroll
        for (int t = 0; t < CH; t++)
            if (t < cnt) vcur[t] = V[(size_t)(i0 + t) * ldv + q];
    }
    for (; q < n; q += stride) {
        const size_t qn = q + stride;
        float4 wnext = zero4, vnext[CH];
#pragma unroll
        for (int t = 0; t < CH; t++) vnext[t] = zero4;
        if (qn < n) {
            wnext = w[qn];
#pragma unroll
            for (int t = 0; t < CH; t++)
                if (t < cnt) vnext[t] = V[(size_t)(i0 + t) * ldv + qn];
        }
        const ff wx = ff_re(wcur), wy = ff_im(wcur);
        float p, e;
        if (first) {
            ff_two_prod(wx, wx, p, e);
            ff_acc_prod(sn, cn, p, e);
            ff_two_prod(wy, wy, p, e);
            ff_acc_prod(sn, cn, p, e);
        }
#pragma unroll
        for (int t = 0; t < CH; t++) {
            if (t < cnt) {
                const ff vx = ff_re(vcur[t]), vy = ff_im(vcur[t]);
                // conj(v) w = (vx wx + vy wy) + i (vx wy - vy wx)
                ff_two_prod(vx, wx, p, e);
                ff_acc_prod(sr[t], cr[t], p, e);
                ff_two_prod(vy, wy, p, e);
                ff_acc_prod(sr[t], cr[t], p, e);
                ff_two_prod(vx, wy, p, e);
                ff_acc_prod(si[t], ci[t], p, e);
                ff_two_prod(vy, wx, p, e);
                ff_acc_prod(si[t], ci[t], -p, -e);
            }
        }
        wcur = wnext;
#pragma unroll
        for (int t = 0; t < CH; t++) vcur[t] = vnext[t];
    }
    ff vals[2 * CH + 1];
#pragma unroll
    for (int t = 0; t < CH; t++) {
        vals[2 * t] = ff_norm(sr[t], cr[t]);
        vals[2 * t + 1] = ff_norm(si[t], ci[t]);
    }
    vals[2 * CH] = ff_norm(sn, cn);
    block_sum_ff<2 * CH + 1>(vals, sums);
    __syncthreads();
    const int G = gridDim.x;
    if ((int)threadIdx.x < cnt)
        partials[(size_t)(i0 + threadIdx.x) * G + blockIdx.x] = make_double2(sums[2 * threadIdx.x], sums[2 * threadIdx.x + 1]);
    if (first && threadIdx.x == 0) partials[(size_t)nv * G + blockIdx.x] = make_double2(sums[2 * CH], 0.0);
}

// w -= sum_i V_i h_i in double-float (h in FP64, split once per block), the result kept as a
// float pair; partials[b] = (||w||^2, 0).
__global__ void __launch_bounds__(NT) k_update_norm_pair(size_t n, const float4 *__restrict__ V, size_t ldv, int nv,
                                                         const double2 *__restrict__ h, float4 *__restrict__ w,
                                                         double2 *__restrict__ partials, const int *__restrict__ gate) {
    pdl_enter();
    if (gate && *gate == 0) return;
    __shared__ float4 hs[64];  // (re.hi, re.lo, im.hi, im.lo)
    __shared__ double sums[1];
    for (int i = threadIdx.x; i < nv; i += NT) {
        const ff a = ff_split(h[i].x), b = ff_split(h[i].y);
        hs[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    __syncthreads();
    float sn = 0.f, cn = 0.f;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float4 wq = w[q];
        // four independent double-float accumulators per component (basis vectors i mod 4),
        // started from w in the first, so the TwoSum chains overlap; the basis values of the
        // next group of four are loaded while the current group is processed
        float sx[4] = {wq.x, 0.f, 0.f, 0.f}, cx[4] = {wq.y, 0.f, 0.f, 0.f};
        float sy[4] = {wq.z, 0.f, 0.f, 0.f}, cy[4] = {wq.w, 0.f, 0.f, 0.f};
        float4 cur[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cur[u] = u < nv ? V[(size_t)u * ldv + q] : zero4;
        for (int i0 = 0; i0 < nv; i0 += 4) {
            float4 nxt[4];
#pragma unroll
            for (int u = 0; u < 4; u++) nxt[u] = i0 + 4 + u < nv ? V[(size_t)(i0 + 4 + u) * ldv + q] : zero4;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (i0 + u < nv) {
                    const ff vx = ff_re(cur[u]), vy = ff_im(cur[u]);
                    const float4 hh = hs[i0 + u];
                    const ff hx = {hh.x, hh.y}, hy = {hh.z, hh.w};
                    float p, e;
                    // w -= v h:  re -= vx hx - vy hy ;  im -= vx hy + vy hx
                    ff_two_prod(vx, hx, p, e);
                    ff_acc_prod(sx[u], cx[u], -p, -e);
                    ff_two_prod(vy, hy, p, e);
                    ff_acc_prod(sx[u], cx[u], p, e);
                    ff_two_prod(vx, hy, p, e);
                    ff_acc_prod(sy[u], cy[u], -p, -e);
                    ff_two_prod(vy, hx, p, e);
                    ff_acc_prod(sy[u], cy[u], -p, -e);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) cur[u] = nxt[u];
        }
        const ff rx = ff_add(ff_add(ff_norm(sx[0], cx[0]), ff_norm(sx[1], cx[1])),
                             ff_add(ff_norm(sx[2], cx[2]), ff_norm(sx[3], cx[3])));
        const ff ry = ff_add(ff_add(ff_norm(sy[0], cy[0]), ff_norm(sy[1], cy[1])),
                             ff_add(ff_norm(sy[2], cy[2]), ff_norm(sy[3], cy[3])));
        w[q] = make_float4(rx.hi, rx.lo, ry.hi, ry.lo);
        float p, e;
        ff_two_prod(rx, rx, p, e);
        ff_acc_prod(sn, cn, p, e);
        ff_two_prod(ry, ry, p, e);
        ff_acc_prod(sn, cn, p, e);
    }
    ff vals[1] = {ff_norm(sn, cn)};
    block_sum_ff<1>(vals, sums);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(sums[0], 0.0);
}

// ---------------------------------------------------------------- delayed CGS2 (DCGS2)
// partials[i * G + b] = V_i^H x and partials[(nv + i) * G + b] = V_i^H w for i < nv: one pass
// over the basis for two right-hand vectors (x is itself basis slot nv - 1).  V^H x decides
// the final basis vector (the reorthogonalisation) and is double-FP32; V^H w only forms the
// first-pass Hessenberg column, whose error the next step's double-FP32 reorthogonalisation
// measures and adds to H (the update that uses it is double-FP32, so A z_j stays exactly
// expanded in the basis), so it is formed from the hi parts in FP32.
// bx: this block's index among the nblk blocks that cover the vector (one launch, or one
// problem's share of a batched launch).
// gv != 0 (a gate flag's value): stop after the first loads (the partials are then meaningless).
template <int CH>
__device__ __forceinline__ void mdot2_body(size_t n, const float4 *__restrict__ V, size_t ldv, int nv,
                                           const float4 *__restrict__ x, const float4 *__restrict__ w,
                                           double2 *__restrict__ partials, int bx, int nblk, int gv = 0) {
    __shared__ double sums[4 * CH];
    // block (b, y) = bx = b * ngroups + y: the blocks that read the same stretch of x and w run
    // side by side, so that all but the first of them find it in L2
    const int ngroups = (nv + CH - 1) / CH;
    const int yb = bx % ngroups, xb = bx / ngroups, G = nblk / ngroups;
    const int i0 = yb * CH;
    const int cnt = min(CH, nv - i0);
    float s[CH][4];   // V^H x: [basis][re.s, re.c, im.s, im.c]
    float f[CH][2];   // V^H w in FP32: [basis][re, im]
#pragma unroll
    for (int t = 0; t < CH; t++) {
#pragma unroll
        for (int k = 0; k < 4; k++) s[t][k] = 0.f;
        f[t][0] = f[t][1] = 0.f;
    }
    for (size_t q = xb * (size_t)NT + threadIdx.x; q < n; q += (size_t)G * NT) {
        const float4 xq = x[q], wq = w[q];
        float4 vq[CH];
#pragma unroll
        for (int t = 0; t < CH; t++) vq[t] = t < cnt ? V[(size_t)(i0 + t) * ldv + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (gv) break;
        const ff xr = ff_re(xq), xi = ff_im(xq);
#pragma unroll
        for (int t = 0; t < CH; t++) {
            if (t < cnt) {
                const ff vr = ff_re(vq[t]), vi = ff_im(vq[t]);
                float p, e;
                // conj(v) x = (vr xr + vi xi) + i (vr xi - vi xr)
                ff_two_prod(vr, xr, p, e); ff_acc_prod(s[t][0], s[t][1], p, e);
                ff_two_prod(vi, xi, p, e); ff_acc_prod(s[t][0], s[t][1], p, e);
                ff_two_prod(vr, xi, p, e); ff_acc_prod(s[t][2], s[t][3], p, e);
                ff_two_prod(vi, xr, p, e); ff_acc_prod(s[t][2], s[t][3], -p, -e);
                f[t][0] = __fmaf_rn(vq[t].x, wq.x, __fmaf_rn(vq[t].z, wq.z, f[t][0]));
                f[t][1] = __fmaf_rn(vq[t].x, wq.z, __fmaf_rn(-vq[t].z, wq.x, f[t][1]));
            }
        }
    }
    ff vals[4 * CH];
#pragma unroll
    for (int t = 0; t < CH; t++) {
        vals[2 * t] = ff_norm(s[t][0], s[t][1]);
        vals[2 * t + 1] = ff_norm(s[t][2], s[t][3]);
        vals[2 * (CH + t)] = ff{f[t][0], 0.f};
        vals[2 * (CH + t) + 1] = ff{f[t][1], 0.f};
    }
    block_sum_ff<4 * CH>(vals, sums);
    __syncthreads();
    if ((int)threadIdx.x < 2 * cnt) {
        const int r = threadIdx.x / cnt, t = threadIdx.x % cnt;
        partials[((size_t)r * nv + i0 + t) * G + xb] =
            make_double2(sums[(r * CH + t) * 2], sums[(r * CH + t) * 2 + 1]);
    }
}

template <int CH>
__global__ void __launch_bounds__(NT, 6) k_mdot2_pair(size_t n, const float4 *__restrict__ V, size_t ldv, int nv,
                                                   const float4 *__restrict__ x, const float4 *__restrict__ w,
                                                   double2 *__restrict__ partials, const int *__restrict__ gate) {
    pdl_enter();
    const int gv = gate_value(gate);
    mdot2_body<CH>(n, V, ldv, nv, x, w, partials, blockIdx.x, gridDim.x, gv);
}

// Index of the entry whose block range [first[e], first[e + 1]) holds block b (count entries).
__device__ __forceinline__ int batch_entry(const unsigned *first, int count, unsigned b) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched two-vector pass of step j over many problems: problem e takes blocks
// [first[e], first[e + 1]) (its one-launch grid); x = slot j and w = slot j + 1 of its basis.
// close: the closing step of a cycle with j columns (w = x = slot j).
template <int CH>
__global__ void __launch_bounds__(NT, 6) k_mdot2_pair_b(const BVec *__restrict__ tab, const unsigned *__restrict__ first,
                                                     int count, int j, int close) {
    pdl_enter();
    const int e = batch_entry(first, count, blockIdx.x);
    const BVec &P = tab[e];
    if (*P.active == 0) return;
    const float4 *V = P.V;
    const float4 *x = V + (size_t)j * P.n;
    mdot2_body<CH>(P.n, V, P.n, j + 1, x, close ? x : x + P.n, P.partials, (int)(blockIdx.x - first[e]),
                   (int)(first[e + 1] - first[e]));
}

// One pass of the DCGS2 update for step j with coefficients coef (see k_dcgs2_coef):
//   x <- (x - sum_{i<j} V_i A_i) r             (x = basis slot j: its final vector v_j)
//   w <- w rw - x_old s - sum_{i<j} V_i C_i    (w = slot j + 1: once orthogonalised, not
//                                                normalised)
// with A = coef[0..j), C = coef[j..2j), r = coef[2j].x, s = coef[2j + 1], rw = coef[2j + 2].x;
// partials[b] = (||w||^2, 0); with b_out, b_out = the new w rounded to complex64.
// With a ticket, the last block to finish also reduces the norm partials into
// *alpha_out = (||w||, 0).
// coef[2j].y != 0 marks a small correction, ||A|| <= 2^-18 ||x - sum V_i A_i|| (decided by the
// coefficient step): sum V_i A_i is then formed in FP32 from the high parts and subtracted from
// x in double-FP32; its rounding error, about 2^-24 ||A||, stays below 2^-42 of the result.
// Otherwise both sums are double-FP32.
template <bool SMALL_A>
__device__ __forceinline__ void update2_nodes(size_t n, float4 *__restrict__ V, size_t ldv, int j,
                                              const float4 *cA, const float4 *cC, ff rinv, ff sr, ff si, ff rw,
                                              float2 *__restrict__ b_out, float &sn, float &cn, int bx, int nblk) {
    float4 *x = V + (size_t)j * ldv, *w = V + (size_t)(j + 1) * ldv;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // The dot pass before this one sweeps the nodes upwards, so L2 holds the top of every
    // vector it read: this pass sweeps downwards and starts on those lines, and it ends at
    // the bottom, where the next step's dot pass starts.
    const size_t stride = (size_t)nblk * NT, base = bx * (size_t)NT + threadIdx.x;
    for (size_t round = (n + stride - 1) / stride; round-- > 0;) {
        const size_t q = round * stride + base;
        if (q >= n) continue;
        const float4 xq = x[q], wq = w[q];
        const ff xr = ff_re(xq), xi = ff_im(xq);
        // (sum, compensation) accumulators per component: v over the basis, started from x; w in
        // two, the basis terms (started from w rw) and the term x s; basis values loaded four at
        // a time, the next four while the current four are processed
        float vs[4] = {xq.x, xq.y, xq.z, xq.w};
        float ws[2][4];
        float fa[2] = {0.f, 0.f};  // small correction: FP32 (re, im)
        float p, e;
        // w rw (rw = 1 / alpha_j when w came from the unscaled slot j, else exactly 1)
        ff_two_prod(ff_re(wq), rw, ws[0][0], ws[0][1]);
        ff_two_prod(ff_im(wq), rw, ws[0][2], ws[0][3]);
        ws[1][0] = ws[1][1] = ws[1][2] = ws[1][3] = 0.f;
        // w -= x s: re -= xr sr - xi si ; im -= xr si + xi sr
        ff_two_prod(xr, sr, p, e); ff_acc_prod(ws[1][0], ws[1][1], -p, -e);
        ff_two_prod(xi, si, p, e); ff_acc_prod(ws[1][0], ws[1][1], p, e);
        ff_two_prod(xr, si, p, e); ff_acc_prod(ws[1][2], ws[1][3], -p, -e);
        ff_two_prod(xi, sr, p, e); ff_acc_prod(ws[1][2], ws[1][3], -p, -e);
        float4 cur[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cur[u] = u < j ? V[(size_t)u * ldv + q] : zero4;
        // basis vector i (value vq)
        auto step = [&](int i, const float4 vq) {
            float *va = vs, *wa = ws[0];
            const ff vr = ff_re(vq), vi = ff_im(vq);
            const float4 a4 = cA[i], c4 = cC[i];
            const ff cr = ff_re(c4), ci = ff_im(c4);
            // v -= V_i a ; w -= V_i c   (complex products)
            if (SMALL_A) {
                float *f = fa;
                f[0] = __fmaf_rn(vq.x, a4.x, __fmaf_rn(-vq.z, a4.z, f[0]));
                f[1] = __fmaf_rn(vq.x, a4.z, __fmaf_rn(vq.z, a4.x, f[1]));
            } else {
                const ff ar = ff_re(a4), ai = ff_im(a4);
                ff_two_prod(vr, ar, p, e); ff_acc_prod(va[0], va[1], -p, -e);
                ff_two_prod(vi, ai, p, e); ff_acc_prod(va[0], va[1], p, e);
                ff_two_prod(vr, ai, p, e); ff_acc_prod(va[2], va[3], -p, -e);
                ff_two_prod(vi, ar, p, e); ff_acc_prod(va[2], va[3], -p, -e);
            }
            ff_two_prod(vr, cr, p, e); ff_acc_prod(wa[0], wa[1], -p, -e);
            ff_two_prod(vi, ci, p, e); ff_acc_prod(wa[0], wa[1], p, e);
            ff_two_prod(vr, ci, p, e); ff_acc_prod(wa[2], wa[3], -p, -e);
            ff_two_prod(vi, cr, p, e); ff_acc_prod(wa[2], wa[3], -p, -e);
        };
        int i0 = 0;
        // groups whose successor is also full: no bounds tests
        for (; i0 + 8 <= j; i0 += 4) {
            float4 nxt[4];
#pragma unroll
            for (int u = 0; u < 4; u++) nxt[u] = V[(size_t)(i0 + 4 + u) * ldv + q];
#pragma unroll
            for (int u = 0; u < 4; u++) step(i0 + u, cur[u]);
#pragma unroll
            for (int u = 0; u < 4; u++) cur[u] = nxt[u];
        }
        for (; i0 < j; i0 += 4) {
            float4 nxt[4];
#pragma unroll
            for (int u = 0; u < 4; u++) nxt[u] = i0 + 4 + u < j ? V[(size_t)(i0 + 4 + u) * ldv + q] : zero4;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (i0 + u < j) step(i0 + u, cur[u]);
#pragma unroll
            for (int u = 0; u < 4; u++) cur[u] = nxt[u];
        }
        // v_j = v r
        ff vr, vi;
        if (SMALL_A) {
            vr = ff_add(xr, ff{-fa[0], 0.f});
            vi = ff_add(xi, ff{-fa[1], 0.f});
        } else {
            vr = ff_norm(vs[0], vs[1]);
            vi = ff_norm(vs[2], vs[3]);
        }
        ff_two_prod(vr, rinv, p, e);
        const ff or_ = ff_norm(p, e);
        ff_two_prod(vi, rinv, p, e);
        const ff oi = ff_norm(p, e);
        x[q] = make_float4(or_.hi, or_.lo, oi.hi, oi.lo);
        const ff wr = ff_add(ff_norm(ws[0][0], ws[0][1]), ff_norm(ws[1][0], ws[1][1]));
        const ff wi = ff_add(ff_norm(ws[0][2], ws[0][3]), ff_norm(ws[1][2], ws[1][3]));
        w[q] = make_float4(wr.hi, wr.lo, wi.hi, wi.lo);
        if (b_out) b_out[q] = make_float2(wr.hi, wi.hi);  // complex64 copy (hi = the rounded pair)
        ff_two_prod(wr, wr, p, e);
        ff_acc_prod(sn, cn, p, e);
        ff_two_prod(wi, wi, p, e);
        ff_acc_prod(sn, cn, p, e);
    }
}

// bx: this block among the nblk blocks of the vector (see mdot2_body).  gate (may be null): when
// the flag is set, leave the vectors as they are (zero norm partials; the ticket protocol still
// runs, so the ticket returns to 0).
__device__ __forceinline__ void update2_body(size_t n, float4 *__restrict__ V, size_t ldv, int j,
                                             const double2 *__restrict__ coef, double2 *__restrict__ partials,
                                             unsigned *ticket, double2 *alpha_out, float2 *__restrict__ b_out, int bx,
                                             int nblk, const int *gate) {
    __shared__ float4 cA[64], cC[64];
    __shared__ float4 sc[2];  // (r hi, lo, small-correction flag, 0), s
    __shared__ float2 rws;    // scale of the incoming w: coef[2j+2].x as a float pair
    __shared__ int skip;      // the gate flag
    __shared__ double sums[1];
    for (int i = threadIdx.x; i < j; i += NT) {
        const ff a = ff_split(coef[i].x), b = ff_split(coef[i].y);
        cA[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
        const ff c = ff_split(coef[j + i].x), d = ff_split(coef[j + i].y);
        cC[i] = make_float4(c.hi, c.lo, d.hi, d.lo);
    }
    if (threadIdx.x == 0) {
        const double2 rc = coef[2 * j];
        const ff r = ff_split(rc.x);
        sc[0] = make_float4(r.hi, r.lo, rc.y != 0.0 ? 1.f : 0.f, 0.f);
        const ff a = ff_split(coef[2 * j + 1].x), b = ff_split(coef[2 * j + 1].y);
        sc[1] = make_float4(a.hi, a.lo, b.hi, b.lo);
        const ff rw = ff_split(coef[2 * j + 2].x);
        rws = make_float2(rw.hi, rw.lo);
        skip = gate_value(gate);
    }
    __syncthreads();
    const ff rinv = ff_re(sc[0]), sr = ff_re(sc[1]), si = ff_im(sc[1]), rw{rws.x, rws.y};
    float sn = 0.f, cn = 0.f;
    if (skip) {
    } else if (sc[0].z != 0.f) {
        update2_nodes<true>(n, V, ldv, j, cA, cC, rinv, sr, si, rw, b_out, sn, cn, bx, nblk);
    } else {
        update2_nodes<false>(n, V, ldv, j, cA, cC, rinv, sr, si, rw, b_out, sn, cn, bx, nblk);
    }
    ff vals[1] = {ff_norm(sn, cn)};
    block_sum_ff<1>(vals, sums);
    if (threadIdx.x == 0) partials[bx] = make_double2(sums[0], 0.0);
    if (!ticket || !last_block(ticket, nblk)) return;
    reduce_partials_block(partials, nblk, 1, alpha_out, true);
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void __launch_bounds__(NT, 4) k_update2_pair(size_t n, float4 *__restrict__ V, size_t ldv, int j,
                                                     const double2 *__restrict__ coef, double2 *__restrict__ partials,
                                                     unsigned *ticket, double2 *alpha_out, float2 *__restrict__ b_out,
                                                     const int *__restrict__ gate) {
    pdl_enter();
    update2_body(n, V, ldv, j, coef, partials, ticket, alpha_out, b_out, blockIdx.x, gridDim.x, gate);
}

// Batched update pass of step j: problem e takes blocks [first[e], first[e + 1]); its ticket
// tickets[1] and alpha_out alpha2[j + 1], the new slot written into its level 0's right-hand side.
__global__ void __launch_bounds__(NT, 4) k_update2_pair_b(const BVec *__restrict__ tab, const unsigned *__restrict__ first,
                                                       int count, int j) {
    pdl_enter();
    const int e = batch_entry(first, count, blockIdx.x);
    const BVec &P = tab[e];
    if (*P.active == 0) return;
    update2_body(P.n, P.V, P.n, j, P.dcoef, P.partials, P.tickets + 1, P.alpha2 + j + 1, P.b0,
                 (int)(blockIdx.x - first[e]), (int)(first[e + 1] - first[e]), nullptr);
}

// 1 / beta.x as a float pair, one FP64 division per block.
__device__ __forceinline__ ff block_inv(const double2 *beta) {
    __shared__ float2 rs;
    if (threadIdx.x == 0) {
        const ff r = ff_split(1.0 / beta->x);
        rs = make_float2(r.hi, r.lo);
    }
    __syncthreads();
    return ff{rs.x, rs.y};
}

// w <- w / beta.x in double-float (w a float pair vector).
__global__ void __launch_bounds__(NT) k_scale_inv_pair(size_t n, float4 *__restrict__ w, const double2 *__restrict__ beta) {
    pdl_enter();
    const ff r = block_inv(beta);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float4 v = w[q];
        float p, e;
        ff_two_prod(ff_re(v), r, p, e);
        const ff a = ff_norm(p, e);
        ff_two_prod(ff_im(v), r, p, e);
        const ff b = ff_norm(p, e);
        w[q] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

// In place: the FP64 vector x (as double2) becomes the float-pair vector x / beta.x.
__global__ void __launch_bounds__(NT) k_split_scale(size_t n, void *x, const double2 *__restrict__ beta) {
    pdl_enter();
    __shared__ double rinv;
    if (threadIdx.x == 0) rinv = beta ? 1.0 / beta->x : 1.0;
    __syncthreads();
    const double r = rinv;
    double2 *in = (double2 *)x;
    float4 *out = (float4 *)x;
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 v = in[q];
        const ff a = ff_split(v.x * r), b = ff_split(v.y * r);
        out[q] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

// Float pairs to complex64 or complex128, divided by alpha->x (alpha null: no scaling).
__device__ __forceinline__ double block_recip(const double2 *alpha) {
    __shared__ double r;
    if (threadIdx.x == 0) r = alpha ? 1.0 / alpha->x : 1.0;
    __syncthreads();
    return r;
}
__global__ void __launch_bounds__(NT) k_pair_to_c64(size_t n, const float4 *__restrict__ v, const double2 *alpha,
                                                    float2 *__restrict__ z) {
    pdl_enter();
    const float r = (float)block_recip(alpha);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float4 a = v[q];
        z[q] = make_float2(__fmul_rn(__fadd_rn(a.x, a.y), r), __fmul_rn(__fadd_rn(a.z, a.w), r));
    }
}
__global__ void __launch_bounds__(NT) k_pair_to_c128(size_t n, const float4 *__restrict__ v, const double2 *alpha,
                                                     double2 *__restrict__ z) {
    pdl_enter();
    const double r = block_recip(alpha);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const float4 a = v[q];
        z[q] = make_double2(((double)a.x + (double)a.y) * r, ((double)a.z + (double)a.w) * r);
    }
}

}  // namespace

// Block counts (fixed for a given n).  The dot pass reduces 2 CH + 1 double-floats per block,
// so it keeps about 8 nodes per thread; the update pass reduces one value and uses the same
// grid as the FP64 kernels, which keeps enough warps resident to hide DRAM latency behind
// the TwoSum dependency chains.
int gs_df_nblocks(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>(cdiv(n, (size_t)NT * 8), (size_t)152 * 4)); }
// The update passes run one full wave: 152 SMs x the blocks of k_update2_pair that fit on an
// SM (by its registers), so that no SM gets a second, partial round of blocks.
int gs_df_update_nblocks(size_t n) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_update2_pair, NT, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 2;
        }
        per_sm = b;
    }
    return (int)std::max<size_t>(1, std::min<size_t>(cdiv(n, NT), (size_t)152 * per_sm));
}

constexpr int DF_CH = 4;  // basis vectors per block row of the dot pass

cudaError_t launch_mdot_norm_pair(size_t n, const float4 *V, size_t ldv, int nv, const float4 *w, double2 *partials,
                                  const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    dim3 g(gs_df_nblocks(n), std::max(1, (nv + DF_CH - 1) / DF_CH));
    launch_pdl(k_mdot_norm_pair<DF_CH>, g, NT, 0, s, n, V, ldv, nv, w, partials, gate);
    return cudaGetLastError();
}

cudaError_t launch_update_norm_pair(size_t n, const float4 *V, size_t ldv, int nv, const double2 *h, float4 *w,
                                    double2 *partials, const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    launch_pdl(k_update_norm_pair, gs_df_update_nblocks(n), NT, 0, s, n, V, ldv, nv, h, w, partials, gate);
    return cudaGetLastError();
}

constexpr int DF_CH2 = 2;  // basis vectors per block row of the two-vector dot pass (2: 40 registers, 6 blocks per SM)

// The two-vector dot pass runs one wave: G blocks per block row of DF_CH2 basis vectors, with
// G x (block rows) at most the blocks that are resident at once (152 SMs x the blocks that fit
// on an SM), so that each block sums a long stretch of nodes and its block reduction is rare.
int gs_df_dot2_nblocks(size_t n, int nv) {
    static int slots = 0;
    if (slots == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mdot2_pair<DF_CH2>, NT, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 2;
        }
        slots = 152 * b;
    }
    const int groups = std::max(1, (nv + DF_CH2 - 1) / DF_CH2);
    return std::max(1, std::min(gs_df_nblocks(n), slots / groups));
}

cudaError_t launch_mdot2_pair(size_t n, const float4 *V, size_t ldv, int nv, const float4 *x, const float4 *w,
                              double2 *partials, const int *gate, cudaStream_t s) {
    if (nv < 1 || nv > 64) return cudaErrorInvalidValue;
    const unsigned g = (unsigned)gs_df_dot2_nblocks(n, nv) * (unsigned)((nv + DF_CH2 - 1) / DF_CH2);
    launch_pdl(k_mdot2_pair<DF_CH2>, dim3(g), NT, 0, s, n, V, ldv, nv, x, w, partials, gate);
    return cudaGetLastError();
}

cudaError_t launch_update2_pair(size_t n, float4 *V, size_t ldv, int j, const double2 *coef, double2 *partials,
                                unsigned *ticket, double2 *alpha_out, float2 *b_out, const int *gate, cudaStream_t s) {
    if (j < 0 || j > 64) return cudaErrorInvalidValue;
    launch_pdl(k_update2_pair, gs_df_update_nblocks(n), NT, 0, s, n, V, ldv, j, coef, partials, ticket, alpha_out,
               b_out, gate);
    return cudaGetLastError();
}

cudaError_t launch_mdot2_pair_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                    int close, cudaStream_t s) {
    if (count < 1 || j < 0 || j > 63 || nblocks < (unsigned)count) return cudaErrorInvalidValue;
    launch_pdl(k_mdot2_pair_b<DF_CH2>, dim3(nblocks), NT, 0, s, tab, first, count, j, close);
    return cudaGetLastError();
}

cudaError_t launch_update2_pair_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                      cudaStream_t s) {
    if (count < 1 || j < 0 || j > 63 || nblocks < (unsigned)count) return cudaErrorInvalidValue;
    launch_pdl(k_update2_pair_b, dim3(nblocks), NT, 0, s, tab, first, count, j);
    return cudaGetLastError();
}

int gs_df_dot2_groups(int nv) { return std::max(1, (nv + DF_CH2 - 1) / DF_CH2); }

static unsigned pair_grid(size_t n) { return (unsigned)std::max<size_t>(1, std::min<size_t>(cdiv(n, NT), 152 * 8)); }

cudaError_t launch_scale_inv_pair(size_t n, float4 *w, const double2 *beta, cudaStream_t s) {
    launch_pdl(k_scale_inv_pair, pair_grid(n), NT, 0, s, n, w, beta);
    return cudaGetLastError();
}
cudaError_t launch_split_scale(size_t n, void *x, const double2 *beta, cudaStream_t s) {
    launch_pdl(k_split_scale, pair_grid(n), NT, 0, s, n, x, beta);
    return cudaGetLastError();
}
cudaError_t launch_pair_to_c64(size_t n, const float4 *v, const double2 *alpha, float2 *z, cudaStream_t s) {
    launch_pdl(k_pair_to_c64, pair_grid(n), NT, 0, s, n, v, alpha, z);
    return cudaGetLastError();
}
cudaError_t launch_pair_to_c128(size_t n, const float4 *v, const double2 *alpha, double2 *z, cudaStream_t s) {
    launch_pdl(k_pair_to_c128, pair_grid(n), NT, 0, s, n, v, alpha, z);
    return cudaGetLastError();
}
