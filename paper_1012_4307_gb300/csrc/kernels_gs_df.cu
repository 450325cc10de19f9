// Gram-Schmidt passes of flexible GMRES with FP64 vectors in memory but the arithmetic done
// in double-FP32 ("double-float") on the FP32 units.
//
// Why: on GB300 the FP64 pipe retires about 2 fused multiply-adds per SM per clock, 64 times
// fewer than FP32, so FP64 inner products over the Krylov basis are bound by FP64 issue, not
// by DRAM.  Here every FP64 operand is split exactly into hi + lo floats with integer
// instructions (hi = the leading 24 significand bits, lo = the next 29 rounded to 24, i.e. a
// 47-bit representation), products are formed error-free with FMA (Dekker/Ogita-Rump-Oishi
// TwoProduct), sums with Knuth's TwoSum, and the result is rounded back to FP64 once per
// node (update) or once per block (dot).  Relative error of a product is about 2^-46 and of a
// sum about 2^-48, i.e. FP64-class accuracy at FP32 throughput, which moves these kernels to
// the DRAM bound.  Inputs below 2^-126 in magnitude are flushed (their contribution to
// products with unit-norm basis vectors is far below the FP64 rounding of the result).
//
// Same contracts as k_mdot_norm / k_update_norm in kernels_krylov.cu (partials layout, gate).
#include "helm_internal.h"
#include "df_arith.h"

namespace {

constexpr int NT = 256;

__device__ __forceinline__ ff shfl_down_ff(ff v, int off) {
    v.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    v.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return v;
}


// Block sums of NV double-float values per thread (fixed tree); thread t < NV gets sum t as
// an FP64 number in out[t].
template <int NV>
__device__ __forceinline__ void block_sum_ff(ff (&v)[NV], double *out) {
    __shared__ ff red[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        ff x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x = ff_add(x, shfl_down_ff(x, off));
        if (lane == 0) red[warp][i] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        ff s = red[0][threadIdx.x];
        for (int w = 1; w < NT / 32; w++) s = ff_add(s, red[w][threadIdx.x]);
        out[threadIdx.x] = ff_to_double(s);
    }
}

// partials[i * G + b] = sum conj(V_i) w (i in this block row's chunk), chunk 0 also
// partials[nv * G + b] = (||w||^2, 0).
template <int CH>
__global__ void __launch_bounds__(NT) k_mdot_norm_df(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                     const double2 *__restrict__ w, double2 *__restrict__ partials,
                                                     const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ double sums[2 * CH + 1];
    const int i0 = blockIdx.y * CH;
    const int cnt = min(CH, nv - i0);
    const bool first = blockIdx.y == 0;
    float sr[CH], cr[CH], si[CH], ci[CH];
    float sn = 0.f, cn = 0.f;
#pragma unroll
    for (int t = 0; t < CH; t++) sr[t] = cr[t] = si[t] = ci[t] = 0.f;
    // software pipeline: the next node's operands are loaded while this node is processed
    const size_t stride = (size_t)gridDim.x * NT;
    const double2 zero2 = make_double2(0.0, 0.0);
    size_t q = blockIdx.x * (size_t)NT + threadIdx.x;
    double2 wcur = zero2, vcur[CH];
#pragma unroll
    for (int t = 0; t < CH; t++) vcur[t] = zero2;
    if (q < n) {
        wcur = w[q];
#pragma unroll
        for (int t = 0; t < CH; t++)
            if (t < cnt) vcur[t] = V[(size_t)(i0 + t) * ldv + q];
    }
    for (; q < n; q += stride) {
        const size_t qn = q + stride;
        double2 wnext = zero2, vnext[CH];
#pragma unroll
        for (int t = 0; t < CH; t++) vnext[t] = zero2;
        if (qn < n) {
            wnext = w[qn];
#pragma unroll
            for (int t = 0; t < CH; t++)
                if (t < cnt) vnext[t] = V[(size_t)(i0 + t) * ldv + qn];
        }
        const double2 wq = wcur;
        const ff wx = ff_split(wq.x), wy = ff_split(wq.y);
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
                const double2 vq = vcur[t];
                const ff vx = ff_split(vq.x), vy = ff_split(vq.y);
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

// w -= sum_i V_i h_i in double-float, rounded to FP64 once per node; partials[b] = (||w||^2, 0).
__global__ void __launch_bounds__(NT) k_update_norm_df(size_t n, const double2 *__restrict__ V, size_t ldv, int nv,
                                                       const double2 *__restrict__ h, double2 *__restrict__ w,
                                                       double2 *__restrict__ partials, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ float4 hs[64];  // (re.hi, re.lo, im.hi, im.lo)
    __shared__ double sums[1];
    for (int i = threadIdx.x; i < nv; i += NT) {
        const ff a = ff_split(h[i].x), b = ff_split(h[i].y);
        hs[i] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    __syncthreads();
    float sn = 0.f, cn = 0.f;
    const double2 zero2 = make_double2(0.0, 0.0);
    for (size_t q = blockIdx.x * (size_t)NT + threadIdx.x; q < n; q += (size_t)gridDim.x * NT) {
        const double2 wq = w[q];
        const ff wx = ff_split(wq.x), wy = ff_split(wq.y);
        // four independent double-float accumulators per component (basis vectors i mod 4),
        // started from w in the first, so the TwoSum chains overlap; the basis values of the
        // next group of four are loaded while the current group is processed
        float sx[4] = {wx.hi, 0.f, 0.f, 0.f}, cx[4] = {wx.lo, 0.f, 0.f, 0.f};
        float sy[4] = {wy.hi, 0.f, 0.f, 0.f}, cy[4] = {wy.lo, 0.f, 0.f, 0.f};
        double2 cur[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cur[u] = u < nv ? V[(size_t)u * ldv + q] : zero2;
        for (int i0 = 0; i0 < nv; i0 += 4) {
            double2 nxt[4];
#pragma unroll
            for (int u = 0; u < 4; u++) nxt[u] = i0 + 4 + u < nv ? V[(size_t)(i0 + 4 + u) * ldv + q] : zero2;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (i0 + u < nv) {
                    const ff vx = ff_split(cur[u].x), vy = ff_split(cur[u].y);
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
        const double2 out = make_double2(ff_to_double(rx), ff_to_double(ry));
        w[q] = out;
        float p, e;
        const ff ox = ff_split(out.x), oy = ff_split(out.y);
        ff_two_prod(ox, ox, p, e);
        ff_acc_prod(sn, cn, p, e);
        ff_two_prod(oy, oy, p, e);
        ff_acc_prod(sn, cn, p, e);
    }
    ff vals[1] = {ff_norm(sn, cn)};
    block_sum_ff<1>(vals, sums);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(sums[0], 0.0);
}

}  // namespace

// Block counts (fixed for a given n).  The dot pass reduces 2 CH + 1 double-floats per block,
// so it keeps about 8 nodes per thread; the update pass reduces one value and uses the same
// grid as the FP64 kernels, which keeps enough warps resident to hide DRAM latency behind
// the long split / TwoSum dependency chains.
int gs_df_nblocks(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>(cdiv(n, (size_t)NT * 8), (size_t)152 * 4)); }
int gs_df_update_nblocks(size_t n) { return blas_nblocks(n); }

constexpr int DF_CH = 4;  // basis vectors per block row of the dot pass

cudaError_t launch_mdot_norm_df(size_t n, const double2 *V, size_t ldv, int nv, const double2 *w, double2 *partials,
                                const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    dim3 g(gs_df_nblocks(n), std::max(1, (nv + DF_CH - 1) / DF_CH));
    k_mdot_norm_df<DF_CH><<<g, NT, 0, s>>>(n, V, ldv, nv, w, partials, gate);
    return cudaGetLastError();
}

cudaError_t launch_update_norm_df(size_t n, const double2 *V, size_t ldv, int nv, const double2 *h, double2 *w,
                                  double2 *partials, const int *gate, cudaStream_t s) {
    if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
    k_update_norm_df<<<gs_df_update_nblocks(n), NT, 0, s>>>(n, V, ldv, nv, h, w, partials, gate);
    return cudaGetLastError();
}
