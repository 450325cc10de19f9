// Coarse levels of a 2D complex64 V-cycle of omega-Jacobi sweeps (Algorithm 1 with
// gamma_f = gamma_c = 1, at most two pre- and two post-sweeps, zero initial guess) in ONE launch
// of a thread-block cluster, with deep halos: one exchange per level on the way down and one on
// the way up.
//
// As in the cluster tail of kernels_ctail.cu, block r of the cluster owns the nested slab of
// interior rows B_l[r] .. B_l[r+1]-1 of every level l, and every level lives in the blocks'
// shared memory.  Here each block also keeps the DH = 3 rows on either side of its slab (its
// window): b, the diagonal of M, its reciprocal and the y coefficients are stored there, and the
// iterates are recomputed there, so a level's whole way down (pre-sweeps, residual, full
// weighting) and its whole way up (prolongation, post-sweeps) each run on local shared memory
// with block barriers only.  The exchanges: the full weighting stores each coarse right-hand-side value into every
// block whose window holds its row, and the last post-sweep stores each result value likewise
// (into a separate array, which the finer level's prolongation reads); a cluster barrier then
// publishes them.  Rows of a window are recomputed by every block that holds them, from the
// same operands with the same operations as their owner, so they equal the owner's values bit
// for bit: the result is the general cluster tail's.
//
// Depths (rows around the slab a step covers): with nu1 pre-sweeps, sweep k covers nu1 + 2 - k
// and the residual 1 (the full weighting of an owned coarse row J reads the fine rows 2J - 1 ..
// 2J + 1, within one row of the fine slab); with nu2 post-sweeps, the prolongation covers nu2
// and sweep k covers nu2 - k.  The prolongation onto those rows reads coarse rows within the
// coarse window.  Per cycle: one cluster barrier before the first exchange (split: arrive after
// the initial fill, wait before the exchange), one per level on the way down, one for the
// coarsest solve and one per level below the top on the way up; the general tail takes about
// seven per level.
#include <cooperative_groups.h>

#include <algorithm>

#include "helm_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int CH_THREADS = CT_BLOCK_THREADS;
constexpr int DH = 3;  // rows of a block's window on either side of its slab

struct HLevel {
    const float2 *cx, *cy;  // global coefficient triples (3 nx, 3 ny)
    const float *k2;        // global k^2 (nx ny)
    float2 bk, c;
    int nx, ny;
    int B[MAX_CT_BLOCKS + 1];
    // byte offsets in shared memory (same in every block): right-hand side, iterate, second
    // iterate / residual, result copy for the finer level, diagonal of M and its reciprocal
    // (cinv_fast, formed once), x and y coefficients
    unsigned ob, ou, ot, oe, od, oi, ocx, ocy;
};

struct HArgs {
    HLevel lv[MAX_CT_LEVELS];
    int nlev, nu_c, nu1, nu2;
    unsigned total;        // bytes of dynamic shared memory
    float omega;
    const float2 *minv;    // nu_c x nu_c, row-major (global)
    const float2 *b_top;   // top level's right-hand side (global)
    float2 *u_top;         // top level's result (global)
    unsigned obc, ominv;   // compact coarsest right-hand side; staged rows of minv
    int mrow;              // rows of minv per warp staged (0: read from global memory)
    const float4 *img;     // initial shared memory of every block (rank r at r * total / 16)
};

struct Ctx {
    unsigned char *sm;
    int rank, nc;
};

// The launch arguments, copied into shared memory once per block (the phases read them there).
__shared__ HArgs ch_args;

// A level as a phase uses it: this block's slab [j0, j1), and full = the coarsest level, which
// every block holds whole (row j at slot j); other levels hold the window, row j at slot
// j - j0 + DH.
struct HL {
    int nx, ny, j0, j1;
    unsigned ob, ou, ot, oe, od, oi, ocx, ocy;
    float2 bk, c;
    const int *B;
    bool full;
};
__device__ __forceinline__ HL hl_of(const Ctx &X, const HArgs *A, int l) {
    const HLevel &L = A->lv[l];
    HL v;
    v.nx = L.nx;
    v.ny = L.ny;
    v.j0 = L.B[X.rank];
    v.j1 = L.B[X.rank + 1];
    v.ob = L.ob; v.ou = L.ou; v.ot = L.ot; v.oe = L.oe; v.od = L.od; v.oi = L.oi; v.ocx = L.ocx; v.ocy = L.ocy;
    v.bk = L.bk;
    v.c = L.c;
    v.B = L.B;
    v.full = l == A->nlev - 1;
    return v;
}

// The block's dynamic shared memory, addressed through the array itself (shared-space loads and
// 32-bit offsets in the phases; the initial fill takes a generic pointer, see hd_init).
extern __shared__ __align__(16) unsigned char ch_smem[];
__device__ __forceinline__ float2 *sarr(unsigned off) { return reinterpret_cast<float2 *>(ch_smem + off); }

__device__ __forceinline__ int slot(const HL &L, int j) { return L.full ? j : j - L.j0 + DH; }
__device__ __forceinline__ float2 *hrow(const Ctx &, const HL &L, unsigned off, int j) {
    return sarr(off) + slot(L, j) * L.nx;
}
// Row j of the array at off in block c's shared memory (a window row of c).
__device__ __forceinline__ float2 *hrow_at(const Ctx &X, const HL &L, unsigned off, int j, int c) {
    const int s = L.full ? j : j - L.B[c] + DH;
    float2 *p = sarr(off) + s * L.nx;
    return c == X.rank ? p : cg::this_cluster().map_shared_rank(p, c);
}

// v at (j, i) of the array at off, for a row j this block owns: into its own slot and into every
// other block whose window holds row j (every block on the coarsest level).  Stores into another
// block's shared memory do not wait; the next cluster barrier publishes them.
__device__ __forceinline__ void share(const Ctx &X, const HL &L, unsigned off, int j, int i, float2 v) {
    hrow(X, L, off, j)[i] = v;
    // no other window holds a row more than DH rows inside the slab
    if (!L.full && j >= L.j0 + DH && j < L.j1 - DH) return;
    if (L.full) {
        for (int c = 0; c < X.nc; c++)
            if (c != X.rank) hrow_at(X, L, off, j, c)[i] = v;
        return;
    }
    for (int c = X.rank - 1; c >= 0 && L.B[c + 1] + DH > j; c--) hrow_at(X, L, off, j, c)[i] = v;
    for (int c = X.rank + 1; c < X.nc && L.B[c] - DH <= j; c++) hrow_at(X, L, off, j, c)[i] = v;
}

// put(j, i, get(j, i)) for every interior node of the rows [ja, jb) (clipped to 1 .. ny - 2).
// Each thread takes U nodes per pass and computes them all before it stores any, so that their
// loads and arithmetic overlap (get only reads, and a node's put writes nothing another node's
// get reads).  The row of node index q is (q + 1/2) / m rounded down in FP32 (exact for
// q < 2^21).
template <int U = 2, typename G, typename S>
__device__ __forceinline__ void for_rows(const HL &L, int ja, int jb, G get, S put) {
    ja = max(ja, 1);
    jb = min(jb, L.ny - 1);
    const int m = L.nx - 2, total = (jb - ja) * m, step = blockDim.x;
    const float rm = 1.0f / (float)m;
    for (int q0 = threadIdx.x; q0 < total; q0 += U * step) {
        int jj[U], ii[U];
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int q = q0 + u * step, r = __float2int_rz(((float)q + 0.5f) * rm);
            jj[u] = ja + r;
            ii[u] = 1 + q - r * m;
            v[u] = q < total ? get(jj[u], ii[u]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (q0 + u * step < total) put(jj[u], ii[u], v[u]);
    }
}

__device__ __forceinline__ float2 hdinv(const HL &L, int j, int i) { return sarr(L.oi)[slot(L, j) * L.nx + i]; }

// (M u)(j, i) from the window rows j - 1, j, j + 1 of the array at u; d = the diagonal.  The
// operations and their order are those of the general cluster tail.
__device__ __forceinline__ float2 happly(const Ctx &, const HL &L, unsigned u, int j, int i, float2 &d) {
    const float2 *cx = sarr(L.ocx), *cy = sarr(L.ocy);
    const int s = slot(L, j);
    const float2 *uc = sarr(u) + s * L.nx;
    const float2 *un = uc - L.nx, *us = uc + L.nx;
    d = sarr(L.od)[s * L.nx + i];
    float2 acc = cmul(cx[3 * i], uc[i - 1]);
    acc = cfma(cx[3 * i + 2], uc[i + 1], acc);
    acc = cfma(cy[3 * s], un[i], acc);
    acc = cfma(cy[3 * s + 2], us[i], acc);
    return cfma(d, uc[i], acc);
}

// Level l's way down: nu1 sweeps from zero and the residual on the window, then the full
// weighting into level l + 1's right-hand side (owned coarse rows, shared), then a cluster
// barrier.  Level 0's waits for every block's initial fill before its first exchange.
__device__ __noinline__ void hd_down(Ctx X, int l) {
    const HArgs *A = &ch_args;
    const HL L = hl_of(X, A, l), Lc = hl_of(X, A, l + 1);
    const float om = A->omega;
    const int nu1 = A->nu1;
    if (L.j0 < L.j1) {
        unsigned src = L.ou;
        for (int k = 1; k <= nu1; k++) {
            const int dep = nu1 + 2 - k;
            const unsigned dst = ((nu1 - k) & 1) ? L.ot : L.ou;  // the last sweep ends in u
            auto store = [&](int j, int i, float2 v) { hrow(X, L, dst, j)[i] = v; };
            if (k == 1)
                for_rows(L, L.j0 - dep, L.j1 + dep,
                         [&](int j, int i) { return cscale(cmul(hrow(X, L, L.ob, j)[i], hdinv(L, j, i)), om); }, store);
            else
                for_rows(L, L.j0 - dep, L.j1 + dep, [&](int j, int i) {
                    const float2 b = hrow(X, L, L.ob, j)[i];
                    float2 d;
                    const float2 mu = happly(X, L, src, j, i, d);
                    return cadd(hrow(X, L, src, j)[i], cscale(cmul(csub(b, mu), hdinv(L, j, i)), om));
                }, store);
            __syncthreads();
            src = dst;
        }
        // residual within one row of the slab into t (u is zero when nu1 = 0)
        for_rows(L, L.j0 - 1, L.j1 + 1, [&](int j, int i) {
            float2 d;
            const float2 mu = happly(X, L, L.ou, j, i, d);
            return csub(hrow(X, L, L.ob, j)[i], mu);
        }, [&](int j, int i, float2 v) { hrow(X, L, L.ot, j)[i] = v; });
        __syncthreads();
    }
    if (l == 0) cg::this_cluster().barrier_wait();
    for_rows(Lc, Lc.j0, Lc.j1, [&](int J, int I) {
        const float2 *r0 = hrow(X, L, L.ot, 2 * J - 1), *r1 = hrow(X, L, L.ot, 2 * J), *r2 = hrow(X, L, L.ot, 2 * J + 1);
        const int x = 2 * I;
        const float2 a0 = cadd(cadd(r0[x - 1], r0[x + 1]), cscale(r0[x], 2.f));
        const float2 a1 = cadd(cadd(r1[x - 1], r1[x + 1]), cscale(r1[x], 2.f));
        const float2 a2 = cadd(cadd(r2[x - 1], r2[x + 1]), cscale(r2[x], 2.f));
        return cscale(cadd(cadd(a0, a2), cscale(a1, 2.f)), 0.0625f);
    }, [&](int J, int I, float2 v) { share(X, Lc, Lc.ob, J, I, v); });
    cg::this_cluster().sync();
}

// Exact coarsest solve: every block holds the whole right-hand side, computes its share of the
// rows of Minv b (one warp per row) and stores each value into every block's copy of the result.
__device__ __noinline__ void hd_dense(Ctx X) {
    const HArgs *A = &ch_args;
    const HL L = hl_of(X, A, A->nlev - 1);
    float2 *bc = sarr(A->obc);
    const int mx = L.nx - 2, nu = A->nu_c;
    for (int c = threadIdx.x; c < nu; c += blockDim.x) bc[c] = hrow(X, L, L.ob, 1 + c / mx)[1 + c % mx];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = X.rank * nw + warp, k = 0; r < nu; r += X.nc * nw, k++) {
        const float2 *mrow = A->mrow ? sarr(A->ominv) + (warp * A->mrow + k) * nu : A->minv + (size_t)r * nu;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = lane; c < nu; c += 32) acc = cfma(mrow[c], bc[c], acc);
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) share(X, L, L.ou, 1 + r / mx, 1 + r % mx, acc);
    }
    cg::this_cluster().sync();
}

// Level l's way up: the prolongation of level l + 1's result added to the iterate on the
// window, nu2 sweeps, the last one on the owned rows only; its values go to the top level's
// global result, or (shared) into the result copy the finer level reads, then a cluster barrier.
__device__ __noinline__ void hd_up(Ctx X, int l) {
    const HArgs *A = &ch_args;
    const HL L = hl_of(X, A, l), Lc = hl_of(X, A, l + 1);
    const float om = A->omega;
    const int nu2 = A->nu2;
    const unsigned e = Lc.full ? Lc.ou : Lc.oe;
    auto result = [&](int j, int i, float2 v) {
        if (l == 0) A->u_top[(size_t)i + (size_t)L.nx * j] = v;
        else share(X, L, L.oe, j, i, v);
    };
    if (L.j0 < L.j1) {
        // in place: a node's prolongation reads only its own iterate
        for_rows(L, L.j0 - nu2, L.j1 + nu2, [&](int j, int i) {
            const float2 *ea = hrow(X, Lc, e, j >> 1), *eb = hrow(X, Lc, e, (j + 1) >> 1);
            const int ia = i >> 1, ib = (i + 1) >> 1;
            const float2 ev = cadd(cadd(ea[ia], ea[ib]), cadd(eb[ia], eb[ib]));
            return cadd(hrow(X, L, L.ou, j)[i], cscale(ev, 0.25f));
        }, [&](int j, int i, float2 v) { hrow(X, L, L.ou, j)[i] = v; });
        __syncthreads();
        unsigned src = L.ou;
        for (int k = 1; k <= nu2; k++) {
            const int dep = nu2 - k;
            const unsigned dst = src == L.ou ? L.ot : L.ou;
            for_rows(L, L.j0 - dep, L.j1 + dep, [&](int j, int i) {
                const float2 b = hrow(X, L, L.ob, j)[i];
                float2 d;
                const float2 mu = happly(X, L, src, j, i, d);
                return cadd(hrow(X, L, src, j)[i], cscale(cmul(csub(b, mu), hdinv(L, j, i)), om));
            }, [&](int j, int i, float2 v) {
                if (k < nu2) hrow(X, L, dst, j)[i] = v;
                else result(j, i, v);
            });
            if (k < nu2) __syncthreads();
            src = dst;
        }
        if (nu2 == 0) for_rows(L, L.j0, L.j1, [&](int j, int i) { return hrow(X, L, L.ou, j)[i]; }, result);
    }
    if (l > 0) cg::this_cluster().sync();
}

// The block's initial shared memory: zeros, the x coefficients, the window's y coefficients and
// diagonal of M (bk k^2 + c + the two centre coefficients, as the general tail forms it) on
// every level above the coarsest, and the block's rows of the coarsest inverse.  X.sm may point
// to global memory (the image k_chalo_image builds once).
__device__ __noinline__ void hd_init(Ctx X, const HArgs *A) {
    for (unsigned q = threadIdx.x; q < A->total / 16; q += blockDim.x) ((float4 *)X.sm)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int l = 0; l + 1 < A->nlev; l++) {
        const HL L = hl_of(X, A, l);
        const HLevel &G = A->lv[l];
        float2 *cx = (float2 *)(X.sm + L.ocx), *cy = (float2 *)(X.sm + L.ocy);
        for (int q = threadIdx.x; q < 3 * L.nx; q += blockDim.x) cx[q] = G.cx[q];
        const int ja = max(L.j0 - DH, 1), jb = min(L.j1 + DH, L.ny - 1);
        for (int q = threadIdx.x; q < 3 * (jb - ja); q += blockDim.x) cy[3 * slot(L, ja) + q] = G.cy[3 * ja + q];
    }
    __syncthreads();
    for (int l = 0; l + 1 < A->nlev; l++) {
        const HL L = hl_of(X, A, l);
        const HLevel &G = A->lv[l];
        const float2 *cx = (const float2 *)(X.sm + L.ocx), *cy = (const float2 *)(X.sm + L.ocy);
        float2 *dg = (float2 *)(X.sm + L.od), *di = (float2 *)(X.sm + L.oi);
        const int ja = max(L.j0 - DH, 1), jb = min(L.j1 + DH, L.ny - 1);
        for (int q = threadIdx.x; q < (jb - ja) * L.nx; q += blockDim.x) {
            const int r = q / L.nx, i = q - r * L.nx, s = slot(L, ja + r);
            const float k2 = G.k2[(size_t)(ja + r) * L.nx + i];
            const float2 d = cadd(cadd(cx[3 * i + 1], cy[3 * s + 1]), cadd(cscale(L.bk, k2), L.c));
            dg[(size_t)s * L.nx + i] = d;
            di[(size_t)s * L.nx + i] = cinv_fast(d);
        }
    }
    if (A->mrow) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, nu = A->nu_c;
        float2 *dst = (float2 *)(X.sm + A->ominv);
        for (int r = X.rank * nw + warp, k = 0; r < nu; r += X.nc * nw, k++)
            for (int c = lane; c < nu; c += 32) dst[(size_t)(warp * A->mrow + k) * nu + c] = A->minv[(size_t)r * nu + c];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CH_THREADS, 1) k_chalo_image(const __grid_constant__ HArgs A0, unsigned char *img) {
    Ctx X{img + (size_t)blockIdx.x * A0.total, (int)blockIdx.x, (int)gridDim.x};
    hd_init(X, &A0);
}

// The cycle once the launch arguments are in shared memory and the image in the block's
// shared memory: the top level's right-hand side on the window (global), then down, the
// coarsest solve, and up.
__device__ __forceinline__ void hd_cycle(Ctx X) {
    const HArgs *A = &ch_args;
    const HL T = hl_of(X, A, 0);
    const float2 *bt = A->b_top;
    if (T.j0 < T.j1)
        for_rows<4>(T, T.j0 - DH, T.j1 + DH, [&](int j, int i) { return bt[(size_t)i + (size_t)T.nx * j]; },
                    [&](int j, int i, float2 v) { hrow(X, T, T.ob, j)[i] = v; });
    // this block's initial fill is complete: other blocks may store into it once all arrived
    cg::this_cluster().barrier_arrive();
    __syncthreads();
    const int nlev = A->nlev;
    for (int l = 0; l + 1 < nlev; l++) hd_down(X, l);
    hd_dense(X);
    for (int l = nlev - 2; l >= 0; l--) hd_up(X, l);
}

__device__ __forceinline__ void copy_args(HArgs &As, const HArgs &A0) {
    const int *src = reinterpret_cast<const int *>(&A0);
    int *dst = reinterpret_cast<int *>(&As);
    for (int q = threadIdx.x; q < (int)(sizeof(HArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
}

__device__ __forceinline__ void copy_image(const Ctx &X, const HArgs *A) {
    const float4 *src = A->img + (size_t)X.rank * (A->total / 16);
    float4 *dst = reinterpret_cast<float4 *>(ch_smem);
    block_copy16(dst, src, A->total / 16);
    __syncthreads();
}

__global__ void __launch_bounds__(CH_THREADS, 1) k_mg_chalo(const __grid_constant__ HArgs A0) {
    pdl_trigger();
    cg::cluster_group cl = cg::this_cluster();
    Ctx X{ch_smem, (int)cl.block_rank(), (int)cl.num_blocks()};
    copy_args(ch_args, A0);
    __syncthreads();
    copy_image(X, &ch_args);
    // the image is not written by earlier kernels; b_top is
    pdl_wait();
    hd_cycle(X);
}

// Batched: cluster z runs problem z's tail (the whole cluster returns when it is inactive) from
// its own image, right-hand side and result.
__global__ void __launch_bounds__(CH_THREADS, 1) k_mg_chalo_b(const __grid_constant__ HArgs A0,
                                                           const BTail *__restrict__ tab, int j) {
    pdl_trigger();
    const BTail &E = tab[blockIdx.z];
    if (*E.active == 0) return;
    HArgs &As = ch_args;
    cg::cluster_group cl = cg::this_cluster();
    Ctx X{ch_smem, (int)cl.block_rank(), (int)cl.num_blocks()};
    copy_args(As, A0);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int l = 0; l < As.nlev; l++) {
            As.lv[l].cx = E.cx[l];
            As.lv[l].cy = E.cy[l];
            As.lv[l].k2 = E.k2[l];
        }
        As.minv = E.minv;
        As.b_top = E.b_top;
        As.u_top = E.u_top + (size_t)j * E.ustride;
        As.img = (const float4 *)E.img;
    }
    __syncthreads();
    copy_image(X, &As);
    pdl_wait();
    hd_cycle(X);
}

}  // namespace

// Shared-memory layout (identical in every block): per level above the coarsest b, u, t, e, the
// diagonal of M and its reciprocal, each (rmax + 2 DH) rows of nx complex64 (rmax = the most rows a block
// owns; no e on the top level, whose result goes to global memory), the x coefficients (3 nx)
// and the window's y coefficients (3 (rmax + 2 DH)); the coarsest level's b and u whole (ny x nx
// each); the compact coarsest right-hand side; the block's staged rows of the coarsest inverse.
// ~0 when the levels are not nested.
size_t mg_chalo_layout(int nlev, const int (*n)[3], int nc, int nu_c, unsigned (*off)[8], unsigned *obc,
                       unsigned *ominv) {
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    int B[MAX_CT_LEVELS][MAX_CT_BLOCKS + 1];
    if (nlev < 2 || nlev > MAX_CT_LEVELS || !mg_ctail_bounds(nlev, n, nc, B)) return ~(size_t)0;
    size_t p = 0;
    for (int l = 0; l < nlev; l++) {
        const int nx = n[l][0];
        if (l == nlev - 1) {
            const size_t vec = al((size_t)n[l][1] * nx * sizeof(float2));
            off[l][0] = (unsigned)p; p += vec;  // b
            off[l][1] = (unsigned)p; p += vec;  // u
            for (int k = 2; k < 8; k++) off[l][k] = 0;
            continue;
        }
        int rmax = 0;
        for (int r = 0; r < nc; r++) rmax = std::max(rmax, B[l][r + 1] - B[l][r]);
        const int W = rmax + 2 * DH;
        const size_t vec = al((size_t)W * nx * sizeof(float2));
        off[l][0] = (unsigned)p; p += vec;                                  // b
        off[l][1] = (unsigned)p; p += vec;                                  // u
        off[l][2] = (unsigned)p; p += vec;                                  // t
        off[l][3] = (unsigned)p; p += l > 0 ? vec : 0;                      // e
        off[l][4] = (unsigned)p; p += vec;                                  // diagonal
        off[l][5] = (unsigned)p; p += vec;                                  // its reciprocal
        off[l][6] = (unsigned)p; p += al((size_t)3 * nx * sizeof(float2));  // x coefficients
        off[l][7] = (unsigned)p; p += al((size_t)3 * W * sizeof(float2));   // y coefficients
    }
    *obc = (unsigned)p;
    p += al((size_t)nu_c * sizeof(float2));
    *ominv = (unsigned)p;
    p += al(mg_ctail_minv_stage_bytes(nc, nu_c));
    return p;
}

// The launch arguments over nlev levels on nc blocks (0 bytes: not possible).
static size_t chalo_args(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, HArgs &A) {
    if (nlev < 2 || nlev > MAX_CT_LEVELS || (nc != 8 && nc != 16)) return 0;
    int n[MAX_CT_LEVELS][3];
    for (int l = 0; l < nlev; l++)
        for (int a = 0; a < 3; a++) n[l][a] = ops[l].n[a];
    unsigned off[MAX_CT_LEVELS][8], obc = 0, ominv = 0;
    const size_t bytes = mg_chalo_layout(nlev, n, nc, nu_c, off, &obc, &ominv);
    if (bytes > CT_SMEM_BYTES) return 0;
    int B[MAX_CT_LEVELS][MAX_CT_BLOCKS + 1];
    if (!mg_ctail_bounds(nlev, n, nc, B)) return 0;
    A = HArgs{};
    for (int l = 0; l < nlev; l++) {
        HLevel &L = A.lv[l];
        L.cx = ops[l].coef[0];
        L.cy = ops[l].coef[1];
        L.k2 = ops[l].k2;
        L.bk = ops[l].bk;
        L.c = ops[l].c;
        L.nx = n[l][0];
        L.ny = n[l][1];
        for (int r = 0; r <= MAX_CT_BLOCKS; r++) L.B[r] = B[l][std::min(r, nc)];
        L.ob = off[l][0]; L.ou = off[l][1]; L.ot = off[l][2]; L.oe = off[l][3]; L.od = off[l][4];
        L.oi = off[l][5]; L.ocx = off[l][6]; L.ocy = off[l][7];
    }
    A.nlev = nlev;
    A.nu_c = nu_c;
    A.minv = minv;
    A.obc = obc;
    A.ominv = ominv;
    A.mrow = mg_ctail_minv_stage_bytes(nc, nu_c) ? mg_ctail_minv_rows(nc, nu_c) : 0;
    A.total = (unsigned)bytes;
    return bytes;
}

size_t mg_chalo_bytes(int nlev, const DevOp<float> *ops, int nu_c, int nc) {
    HArgs A;
    return chalo_args(nlev, ops, nullptr, nu_c, nc, A);
}

cudaError_t build_mg_chalo_image(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, void **out,
                                 cudaStream_t s) {
    *out = nullptr;
    HArgs A;
    const size_t bytes = chalo_args(nlev, ops, minv, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    void *img = nullptr;
    cudaError_t e = cudaMalloc(&img, bytes * nc);
    if (e != cudaSuccess) return e;
    k_chalo_image<<<nc, CH_THREADS, 0, s>>>(A, (unsigned char *)img);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        cudaFree(img);
        return e;
    }
    *out = img;
    return cudaSuccess;
}

template <typename K>
static cudaError_t ch_attrs(K kernel, int nc, bool *done) {
    if (*done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM_BYTES);
    if (e == cudaSuccess && nc > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) *done = true;
    return e;
}

static cudaError_t ch_launch_cfg(cudaLaunchConfig_t &cfg, cudaLaunchAttribute (&at)[2], int nc, int count,
                                 size_t bytes, cudaStream_t s) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(nc, 1, count);
    cfg.blockDim = dim3(CH_THREADS, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cudaSuccess;
}

cudaError_t launch_mg_chalo(int nlev, const DevOp<float> *ops, const float2 *b_top, float2 *u_top, const float2 *minv,
                            int nu_c, int nu1, int nu2, float omega, int nc, const void *img, cudaStream_t s) {
    if (!img || nu1 < 0 || nu1 > 2 || nu2 < 0 || nu2 > 2) return cudaErrorInvalidValue;
    HArgs A;
    const size_t bytes = chalo_args(nlev, ops, minv, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.omega = omega;
    A.b_top = b_top;
    A.u_top = u_top;
    A.img = (const float4 *)img;
    static bool attr[2] = {false, false};
    cudaError_t e = ch_attrs(k_mg_chalo, nc, &attr[nc == 16]);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[2];
    ch_launch_cfg(cfg, at, nc, 1, bytes, s);
    return cudaLaunchKernelEx(&cfg, k_mg_chalo, A);
}

cudaError_t launch_mg_chalo_batch(int nlev, const DevOp<float> *ops, int nu_c, int nu1, int nu2, float omega, int nc,
                                  int count, const BTail *tab, int j, cudaStream_t s) {
    if (count < 1 || count > 65535 || nu1 < 0 || nu1 > 2 || nu2 < 0 || nu2 > 2) return cudaErrorInvalidValue;
    HArgs A;
    const size_t bytes = chalo_args(nlev, ops, nullptr, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.omega = omega;
    static bool attr[2] = {false, false};
    cudaError_t e = ch_attrs(k_mg_chalo_b, nc, &attr[nc == 16]);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[2];
    ch_launch_cfg(cfg, at, nc, count, bytes, s);
    return cudaLaunchKernelEx(&cfg, k_mg_chalo_b, A, tab, j);
}

int mg_chalo_max_clusters(int nc, size_t bytes) {
    static bool attr[2] = {false, false};
    if (ch_attrs(k_mg_chalo, nc, &attr[nc == 16]) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[2];
    ch_launch_cfg(cfg, at, nc, 1, bytes, nullptr);
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_mg_chalo, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
