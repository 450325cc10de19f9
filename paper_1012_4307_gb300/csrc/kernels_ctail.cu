// Coarse levels of a 2D complex64 cycle (Algorithm 1) in ONE launch of a thread-block cluster.
//
// The coarse levels (129 x 129 nodes and below on the benchmark grids) hold too little work to
// fill the GPU, so as separate launches each costs a launch latency plus a few dependent
// phases, and on one thread block they are bound by one SM's issue rate.  Here a cluster of
// NC thread blocks (8 or 16 SMs) keeps every level's b, u, t, diagonal and coefficients in its
// distributed shared memory.  Block r owns the interior rows B_l[r] .. B_l[r+1]-1 of level l,
// the slabs nested across levels (B_{l+1}[r] = (B_l[r] + 1) / 2), so that the full weighting of
// an owned coarse row and the prolongation onto an owned fine row only touch rows that the
// block owns or the two rows next to its slab.  Each block keeps those two rows as halo rows
// of u and t; whoever writes the first or last row of its slab also stores the value into the
// neighbouring slab's halo (a store to distributed shared memory, which does not wait), and the
// cluster barrier between phases publishes it.  Every read inside a phase is then a local
// shared-memory read; a dependent read of another block's shared memory costs about as much as
// a whole cluster barrier.  Same arithmetic as the per-level kernels in kernels_mg.cu:
// omega-Jacobi (ping-pong) or omega-red-black sweeps, residual and full weighting, bilinear
// prolongation, exact coarsest solve by the dense inverse.
#include <cooperative_groups.h>

#include <algorithm>

#include "helm_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int CT_THREADS = CT_BLOCK_THREADS;

struct CLevel {
    const float2 *cx, *cy;  // global coefficient triples (3 nx, 3 ny)
    const float *k2;        // global k^2 (nx ny)
    float2 bk, c;
    int nx, ny;
    int B[MAX_CT_BLOCKS + 1];     // block r owns interior rows B[r] .. B[r+1]-1 (possibly none)
    unsigned ob, ou, ot, ok, oi, ocx, ocy;  // byte offsets in shared memory (same in every block);
                                            // ok: the diagonal of M at the owned nodes, oi: its
                                            // reciprocal (cinv_fast, formed once)
};

struct CArgs {
    CLevel lv[MAX_CT_LEVELS];
    int nlev, nu_c, nu1, nu2, rb, zero, gf, gc;
    unsigned total;  // bytes of dynamic shared memory
    float omega;
    const float2 *minv;  // nu_c x nu_c, row-major (global)
    const float2 *b_top;  // top level's right-hand side (global)
    float2 *u_top;        // top level's result; initial guess when !zero (global)
    unsigned obc;         // compact coarsest right-hand side
    unsigned ominv;       // this block's rows of minv (mrow per warp), staged in the prologue
    int mrow;             // 0: minv is read from global memory in the dense phase
    const float4 *img;    // initial shared memory of every block (rank r at r * total / 16), or null
};

struct Ctx {
    unsigned char *sm;
    int rank, nc;
};

// A level as the phases use it: the scalars in registers (a phase's shared-memory stores could
// alias the launch arguments, which live in shared memory too, and would force reloads), this
// block's slab [j0, j1), and the slab bounds of every block (B, in shared memory) for the rare
// accesses to other blocks' rows.
struct LV {
    int nx, j0, j1;
    unsigned ob, ou, ot, ok, oi, ocx, ocy;
    float2 bk, c;
    const int *B;
};
__device__ __forceinline__ LV lv_of(const Ctx &X, const CLevel &L) {
    LV v;
    v.nx = L.nx;
    v.j0 = L.B[X.rank];
    v.j1 = L.B[X.rank + 1];
    v.ob = L.ob; v.ou = L.ou; v.ot = L.ot; v.ok = L.ok; v.oi = L.oi; v.ocx = L.ocx; v.ocy = L.ocy;
    v.bk = L.bk;
    v.c = L.c;
    v.B = L.B;
    return v;
}

// Row j of the level array at offset off in a block's slot layout: slot j - B[c] + 1, so slot
// 0 and slot rows + 1 are the halo rows (a boundary row's halo is never written: zeros).
// This block's row j, for j0 - 1 <= j <= j1:
__device__ __forceinline__ float2 *lrow(const Ctx &X, const LV &L, unsigned off, int j) {
    return (float2 *)(X.sm + off) + (size_t)(j - L.j0 + 1) * L.nx;
}
// block c's row j (another block's through distributed shared memory)
__device__ __forceinline__ float2 *crow(const Ctx &X, const LV &L, unsigned off, int j, int c) {
    if (c == X.rank) return lrow(X, L, off, j);
    float2 *p = (float2 *)(X.sm + off) + (size_t)(j - L.B[c] + 1) * L.nx;
    return cg::this_cluster().map_shared_rank(p, (unsigned)c);
}
__device__ __forceinline__ int owner_of(const LV &L, int nc, int j) {
    int c = 0;
    while (c + 1 < nc && L.B[c + 1] <= j) c++;
    return c;
}

// u(j, i) = v for row j owned by block `owner`, and the same value into every other block whose
// window of rows (B[c] - 1 .. B[c+1]) holds row j: the blocks just above the owner's slab whose
// slabs end at row j (empty ones, then the nearest non-empty one) when j is the owner's first
// row, and likewise below when j is its last row.
__device__ __forceinline__ void put(const Ctx &X, const LV &L, unsigned off, int j, int i, float2 v, int owner) {
    const bool own = owner == X.rank;
    const int b0 = own ? L.j0 : L.B[owner], b1 = own ? L.j1 : L.B[owner + 1];
    crow(X, L, off, j, owner)[i] = v;
    if (j == b0)
        for (int p = owner - 1; p >= 0 && L.B[p + 1] == j; p--) crow(X, L, off, j, p)[i] = v;
    if (j == b1 - 1)
        for (int q = owner + 1; q < X.nc && L.B[q] == j + 1; q++) crow(X, L, off, j, q)[i] = v;
}

__device__ __forceinline__ void csync() { cg::this_cluster().sync(); }

// f(j, i) for every owned interior node, one node per thread and pass (consecutive threads
// along a row).  The row of pass index q is (q + 1/2) / m rounded down in FP32: exact for
// q < 2^21, far above any slab.
template <typename F>
__device__ __forceinline__ void for_owned(const Ctx &X, const LV &L, F f) {
    const int m = L.nx - 2, total = (L.j1 - L.j0) * m;
    const float rm = 1.0f / (float)m;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int r = __float2int_rz(((float)q + 0.5f) * rm);
        f(L.j0 + r, 1 + q - r * m);
    }
}

// The diagonal of M at an owned node, formed once per launch (bk k^2 + c + the two centre
// coefficients) and kept in shared memory.
__device__ __forceinline__ float2 diag_at(const Ctx &X, const LV &L, int j, int i) {
    return ((const float2 *)(X.sm + L.ok))[(size_t)(j - L.j0) * L.nx + i];
}
__device__ __forceinline__ float2 dinv_at(const Ctx &X, const LV &L, int j, int i) {
    return ((const float2 *)(X.sm + L.oi))[(size_t)(j - L.j0) * L.nx + i];
}

// (M u)(j, i) from this block's rows of the array at offset u (j - 1 and j + 1 may be halo
// rows); d = the diagonal.
__device__ __forceinline__ float2 apply_at(const Ctx &X, const LV &L, unsigned u, int j, int i, float2 &d) {
    const float2 *cx = (const float2 *)(X.sm + L.ocx), *cy = (const float2 *)(X.sm + L.ocy);
    const int li = j - L.j0;
    const float2 *un = lrow(X, L, u, j - 1), *uc = lrow(X, L, u, j), *us = lrow(X, L, u, j + 1);
    d = diag_at(X, L, j, i);
    float2 acc = cmul(cx[3 * i], uc[i - 1]);
    acc = cfma(cx[3 * i + 2], uc[i + 1], acc);
    acc = cfma(cy[3 * li], un[i], acc);
    acc = cfma(cy[3 * li + 2], us[i], acc);
    return cfma(d, uc[i], acc);
}

// The phases of the cycle.  Each is one out-of-line function over a level index, so that the
// kernel's code stays small (inlining every phase at every depth multiplies it by the levels
// and smoothing steps and runs out of the instruction cache); each ends with a cluster barrier.

// nu sweeps on level l from *cur (partner *oth); zero: u = 0 on entry.  Returns the new pair.
__device__ __noinline__ uint2 ph_smooth(Ctx X, const CArgs *A, int l, int nu, uint2 co, bool zero) {
    const LV L = lv_of(X, A->lv[l]);
    const float om = A->omega;
    const bool rb = A->rb != 0;
    if (zero && (nu == 0 || rb)) {
        const unsigned u = co.x;
        for_owned(X, L, [&](int j, int i) { put(X, L, u, j, i, make_float2(0.f, 0.f), X.rank); });
        csync();
    }
    for (int s = 0; s < nu; s++) {
        if (rb) {
            for (int colour = 0; colour < 2; colour++) {
                // in place: this colour's neighbours (the other colour) are not written here
                const unsigned u = co.x;
                for_owned(X, L, [&](int j, int i) {
                    if (((i + j) & 1) != colour) return;
                    float2 d;
                    const float2 mu = apply_at(X, L, u, j, i, d);
                    const float2 uc = lrow(X, L, u, j)[i], b = lrow(X, L, L.ob, j)[i];
                    put(X, L, u, j, i, cadd(uc, cscale(cmul(csub(b, mu), dinv_at(X, L, j, i)), om)), X.rank);
                });
                csync();
            }
        } else {
            const bool z0 = zero && s == 0;
            const unsigned src = co.x, dst = co.y;
            for_owned(X, L, [&](int j, int i) {
                const float2 b = lrow(X, L, L.ob, j)[i];
                float2 v;
                if (z0) {
                    v = cscale(cmul(b, dinv_at(X, L, j, i)), om);
                } else {
                    float2 d;
                    const float2 mu = apply_at(X, L, src, j, i, d);
                    v = cadd(lrow(X, L, src, j)[i], cscale(cmul(csub(b, mu), dinv_at(X, L, j, i)), om));
                }
                put(X, L, dst, j, i, v, X.rank);
            });
            csync();
            co = make_uint2(dst, src);
        }
    }
    return co;
}

// Residual of level l (iterate u) into r, then full weighting into level l + 1's b (the fine
// rows 2J-1 .. 2J+1 of an owned coarse row J are owned or halo rows: nested slabs).
__device__ __noinline__ void ph_restrict(Ctx X, const CArgs *A, int l, unsigned u, unsigned r) {
    const LV L = lv_of(X, A->lv[l]), Lc = lv_of(X, A->lv[l + 1]);
    for_owned(X, L, [&](int j, int i) {
        float2 d;
        const float2 mu = apply_at(X, L, u, j, i, d);
        put(X, L, r, j, i, csub(lrow(X, L, L.ob, j)[i], mu), X.rank);
    });
    csync();
    for_owned(X, Lc, [&](int J, int I) {
        const float2 *r0 = lrow(X, L, r, 2 * J - 1), *r1 = lrow(X, L, r, 2 * J), *r2 = lrow(X, L, r, 2 * J + 1);
        const int x = 2 * I;
        const float2 a0 = cadd(cadd(r0[x - 1], r0[x + 1]), cscale(r0[x], 2.f));
        const float2 a1 = cadd(cadd(r1[x - 1], r1[x + 1]), cscale(r1[x], 2.f));
        const float2 a2 = cadd(cadd(r2[x - 1], r2[x + 1]), cscale(r2[x], 2.f));
        lrow(X, Lc, Lc.ob, J)[I] = cscale(cadd(cadd(a0, a2), cscale(a1, 2.f)), 0.0625f);
    });
    csync();
}

// Bilinear prolongation of level l + 1's u (coarse rows j/2 and (j+1)/2: owned or halo rows of
// the coarse slab), added to level l's iterate u.
__device__ __noinline__ void ph_prolong(Ctx X, const CArgs *A, int l, unsigned u) {
    const LV L = lv_of(X, A->lv[l]), Lc = lv_of(X, A->lv[l + 1]);
    for_owned(X, L, [&](int j, int i) {
        const float2 *ea = lrow(X, Lc, Lc.ou, j >> 1), *eb = lrow(X, Lc, Lc.ou, (j + 1) >> 1);
        const int ia = i >> 1, ib = (i + 1) >> 1;
        const float2 e = cadd(cadd(ea[ia], ea[ib]), cadd(eb[ia], eb[ib]));
        put(X, L, u, j, i, cadd(lrow(X, L, u, j)[i], cscale(e, 0.25f)), X.rank);
    });
    csync();
}

__device__ __noinline__ void ph_copy(Ctx X, const CArgs *A, int l, unsigned dst, unsigned src) {
    const LV L = lv_of(X, A->lv[l]);
    for_owned(X, L, [&](int j, int i) { put(X, L, dst, j, i, lrow(X, L, src, j)[i], X.rank); });
    csync();
}

// Exact coarsest solve: every block gathers the whole right-hand side, computes its share of
// the rows of Minv b (one warp per row) and stores each result in the owning block's u (and
// the halos that hold its row).
__device__ __noinline__ void ph_dense(Ctx X, const CArgs *A, int l) {
    const LV L = lv_of(X, A->lv[l]);
    float2 *bc = (float2 *)(X.sm + A->obc);
    const int mx = L.nx - 2, nu = A->nu_c;
    for (int c = threadIdx.x; c < nu; c += blockDim.x) {
        const int i = 1 + c % mx, j = 1 + c / mx;
        bc[c] = crow(X, L, L.ob, j, owner_of(L, X.nc, j))[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = X.rank * nw + warp, k = 0; r < nu; r += X.nc * nw, k++) {
        const float2 *mrow = A->mrow ? (const float2 *)(X.sm + A->ominv) + (size_t)(warp * A->mrow + k) * nu
                                     : A->minv + (size_t)r * nu;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = lane; c < nu; c += 32) acc = cfma(mrow[c], bc[c], acc);
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
            const int j = 1 + r / mx;
            put(X, L, L.ou, j, 1 + r % mx, acc, owner_of(L, X.nc, j));
        }
    }
    csync();
}

// This block's rows of the coarsest inverse into shared memory (the rows ph_dense gives each
// warp), before the kernel waits on its predecessor.
__device__ __noinline__ void ph_stage_minv(Ctx X, const CArgs *A) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, nu = A->nu_c;
    float2 *dst = (float2 *)(X.sm + A->ominv);
    for (int r = X.rank * nw + warp, k = 0; r < nu; r += X.nc * nw, k++)
        for (int c = lane; c < nu; c += 32) dst[(size_t)(warp * A->mrow + k) * nu + c] = A->minv[(size_t)r * nu + c];
}

// Level LVL of the cycle (compile-time depth); the result ends in the level's u.
template <int LVL>
__device__ __noinline__ void ct_cycle(Ctx X, const CArgs *A, bool zero, int gf, int gc) {
    const CLevel &L = A->lv[LVL];
    if (LVL == A->nlev - 1) {
        ph_dense(X, A, LVL);
        return;
    }
    if constexpr (LVL + 1 < MAX_CT_LEVELS) {
        uint2 co = ph_smooth(X, A, LVL, A->nu1, make_uint2(L.ou, L.ot), zero);
        ph_restrict(X, A, LVL, co.x, co.y);
        if (LVL + 1 == A->nlev - 1) {
            ph_dense(X, A, LVL + 1);
        } else {
            // first visit from zero with (gf, gc), later ones from the iterate with (gc, gf)
            for (int k = 1; k <= gc; k++) ct_cycle<LVL + 1>(X, A, k == 1, k == 1 ? gf : gc, k == 1 ? gc : gf);
        }
        ph_prolong(X, A, LVL, co.x);
        co = ph_smooth(X, A, LVL, A->nu2, co, false);
        if (co.x != L.ou) ph_copy(X, A, LVL, L.ou, co.x);
    }
}

// The block's shared memory before the cycle: zeros, the staged coefficients, the diagonal
// bk k^2 + c + centre coefficients of the owned rows and the block's rows of the coarsest
// inverse.  X.sm may point to global memory (the image that k_ctail_image builds once).
__device__ __noinline__ void ct_init(Ctx X, const CArgs *A) {
    for (unsigned q = threadIdx.x; q < A->total / 16; q += blockDim.x) ((float4 *)X.sm)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int l = 0; l < A->nlev; l++) {
        const CLevel &L = A->lv[l];
        const int j0 = L.B[X.rank], j1 = L.B[X.rank + 1];
        float2 *cx = (float2 *)(X.sm + L.ocx), *cy = (float2 *)(X.sm + L.ocy);
        for (int q = threadIdx.x; q < 3 * L.nx; q += blockDim.x) cx[q] = L.cx[q];
        for (int q = threadIdx.x; q < 3 * (j1 - j0); q += blockDim.x) cy[q] = L.cy[3 * j0 + q];
    }
    __syncthreads();
    for (int l = 0; l < A->nlev; l++) {
        const CLevel &L = A->lv[l];
        const int j0 = L.B[X.rank], j1 = L.B[X.rank + 1];
        const float2 *cx = (const float2 *)(X.sm + L.ocx), *cy = (const float2 *)(X.sm + L.ocy);
        float2 *dg = (float2 *)(X.sm + L.ok), *di = (float2 *)(X.sm + L.oi);
        for (int q = threadIdx.x; q < (j1 - j0) * L.nx; q += blockDim.x) {
            const int li = q / L.nx, i = q - li * L.nx;
            const float k2 = L.k2[(size_t)j0 * L.nx + q];
            const float2 d = cadd(cadd(cx[3 * i + 1], cy[3 * li + 1]), cadd(cscale(L.bk, k2), L.c));
            dg[q] = d;
            di[q] = cinv_fast(d);
        }
    }
    if (A->mrow) ph_stage_minv(X, A);
    __syncthreads();
}

// Builds the initial shared memory of every block of the cluster tail in global memory (one
// block per rank, no cluster): the tail then starts with one copy instead of three dependent
// rounds of loads.
__global__ void __launch_bounds__(CT_THREADS, 1) k_ctail_image(const __grid_constant__ CArgs A0, unsigned char *img) {
    Ctx X{img + (size_t)blockIdx.x * A0.total, (int)blockIdx.x, (int)gridDim.x};
    ct_init(X, &A0);
}

__global__ void __launch_bounds__(CT_THREADS, 1) k_mg_ctail(const __grid_constant__ CArgs A0) {
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char ct_smem[];
    __shared__ CArgs As;
    cg::cluster_group cl = cg::this_cluster();
    Ctx X{ct_smem, (int)cl.block_rank(), (int)cl.num_blocks()};
    {
        const int *src = reinterpret_cast<const int *>(&A0);
        int *dst = reinterpret_cast<int *>(&As);
        for (int q = threadIdx.x; q < (int)(sizeof(CArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    const CArgs *A = &As;
    if (A0.img) {
        const float4 *src = A0.img + (size_t)X.rank * (A0.total / 16);
        block_copy16((float4 *)ct_smem, src, A0.total / 16);
        __syncthreads();
    } else {
        __syncthreads();
        ct_init(X, A);
    }
    const LV T = lv_of(X, A->lv[0]);
    // the operator data above is not written by earlier kernels; b_top and u_top are
    pdl_wait();
    // every block's initial fill precedes any store into its halos
    csync();
    for_owned(X, T, [&](int j, int i) {
        const size_t p = (size_t)i + (size_t)T.nx * j;
        lrow(X, T, T.ob, j)[i] = A->b_top[p];
        if (!A->zero) put(X, T, T.ou, j, i, A->u_top[p], X.rank);
    });
    csync();
    ct_cycle<0>(X, A, A->zero != 0, A->gf, A->gc);
    for_owned(X, T, [&](int j, int i) { A->u_top[(size_t)i + (size_t)T.nx * j] = lrow(X, T, T.ou, j)[i]; });
}

// Batched cluster tail: cluster z runs problem z's tail (blockIdx.z is shared by every block of
// a cluster, so a cluster returns as a whole when its problem is inactive).  The launch
// arguments A0 are the levels' common layout; the problem's pointers come from its table entry,
// and its blocks start from the problem's prebuilt image.
__global__ void __launch_bounds__(CT_THREADS, 1) k_mg_ctail_b(const __grid_constant__ CArgs A0,
                                                           const BTail *__restrict__ tab, int j) {
    pdl_trigger();
    const BTail &E = tab[blockIdx.z];
    if (*E.active == 0) return;
    extern __shared__ __align__(16) unsigned char ct_smem[];
    __shared__ CArgs As;
    cg::cluster_group cl = cg::this_cluster();
    Ctx X{ct_smem, (int)cl.block_rank(), (int)cl.num_blocks()};
    {
        const int *src = reinterpret_cast<const int *>(&A0);
        int *dst = reinterpret_cast<int *>(&As);
        for (int q = threadIdx.x; q < (int)(sizeof(CArgs) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
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
    const CArgs *A = &As;
    {
        const float4 *src = A->img + (size_t)X.rank * (A->total / 16);
        block_copy16((float4 *)ct_smem, src, A->total / 16);
        __syncthreads();
    }
    const LV T = lv_of(X, A->lv[0]);
    pdl_wait();
    csync();
    for_owned(X, T, [&](int j, int i) {
        const size_t p = (size_t)i + (size_t)T.nx * j;
        lrow(X, T, T.ob, j)[i] = A->b_top[p];
        if (!A->zero) put(X, T, T.ou, j, i, A->u_top[p], X.rank);
    });
    csync();
    ct_cycle<0>(X, A, A->zero != 0, A->gf, A->gc);
    for_owned(X, T, [&](int j, int i) { A->u_top[(size_t)i + (size_t)T.nx * j] = lrow(X, T, T.ou, j)[i]; });
}

}  // namespace

bool mg_ctail_bounds(int nlev, const int (*n)[3], int nc, int (*B)[MAX_CT_BLOCKS + 1]) {
    if (nc < 1 || nc > MAX_CT_BLOCKS) return false;
    for (int l = 0; l < nlev; l++) {
        if (n[l][1] < 3 || n[l][1] % 2 == 0) return false;
        if (l + 1 < nlev && n[l + 1][1] != (n[l][1] + 1) / 2) return false;
    }
    const int rows = (n[0][1] - 2 + nc - 1) / nc;
    for (int r = 0; r <= nc; r++) B[0][r] = std::min(1 + r * rows, n[0][1] - 1);
    for (int l = 1; l < nlev; l++)
        for (int r = 0; r <= nc; r++) B[l][r] = (B[l - 1][r] + 1) / 2;
    return true;
}

int mg_ctail_minv_rows(int nc, int nu_c) { return (nu_c + nc * (CT_THREADS / 32) - 1) / (nc * (CT_THREADS / 32)); }
size_t mg_ctail_minv_stage_bytes(int nc, int nu_c) {
    const size_t b = (size_t)(CT_THREADS / 32) * mg_ctail_minv_rows(nc, nu_c) * nu_c * sizeof(float2);
    return b <= 64 * 1024 ? b : 0;
}

// Shared-memory layout of the cluster tail (identical in every block): per level b, u, t
// ((rmax + 2) rows x nx complex64 each: the owned rows between two halo rows; rmax = the most
// rows a block owns), the diagonal of M and its reciprocal (rmax x nx complex64 each), x
// coefficients (3 nx), y coefficients of the owned rows (3 rmax); then the compact coarsest
// right-hand side and the block's staged rows of the coarsest inverse (ominv).  Levels that are not nested (odd ny,
// halved) get a size no launch accepts.
size_t mg_ctail_layout(int nlev, const int (*n)[3], int nc, int nu_c, unsigned (*off)[7], unsigned *obc,
                       unsigned *ominv) {
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    int B[MAX_CT_LEVELS][MAX_CT_BLOCKS + 1];
    if (nlev < 1 || nlev > MAX_CT_LEVELS || !mg_ctail_bounds(nlev, n, nc, B)) return ~(size_t)0;
    size_t p = 0;
    for (int l = 0; l < nlev; l++) {
        const int nx = n[l][0];
        int rmax = 0;
        for (int r = 0; r < nc; r++) rmax = std::max(rmax, B[l][r + 1] - B[l][r]);
        const size_t vec = al((size_t)(rmax + 2) * nx * sizeof(float2));
        off[l][0] = (unsigned)p; p += vec;                                             // b
        off[l][1] = (unsigned)p; p += vec;                                             // u
        off[l][2] = (unsigned)p; p += vec;                                             // t
        off[l][3] = (unsigned)p; p += al((size_t)rmax * nx * sizeof(float2));          // diagonal
        off[l][4] = (unsigned)p; p += al((size_t)rmax * nx * sizeof(float2));          // its reciprocal
        off[l][5] = (unsigned)p; p += al((size_t)3 * nx * sizeof(float2));             // x coefficients
        off[l][6] = (unsigned)p; p += al((size_t)3 * rmax * sizeof(float2));           // y coefficients
    }
    *obc = (unsigned)p;
    p += al((size_t)nu_c * sizeof(float2));
    *ominv = (unsigned)p;
    p += al(mg_ctail_minv_stage_bytes(nc, nu_c));
    return p;
}

// The launch arguments of a cluster tail over nlev levels on nc blocks (0 bytes: not possible).
static size_t ct_args(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, CArgs &A) {
    if (nlev < 2 || nlev > MAX_CT_LEVELS || (nc != 8 && nc != 16)) return 0;
    int n[MAX_CT_LEVELS][3];
    for (int l = 0; l < nlev; l++)
        for (int a = 0; a < 3; a++) n[l][a] = ops[l].n[a];
    unsigned off[MAX_CT_LEVELS][7], obc = 0, ominv = 0;
    const size_t bytes = mg_ctail_layout(nlev, n, nc, nu_c, off, &obc, &ominv);
    if (bytes > CT_SMEM_BYTES) return 0;
    int B[MAX_CT_LEVELS][MAX_CT_BLOCKS + 1];
    if (!mg_ctail_bounds(nlev, n, nc, B)) return 0;
    A = CArgs{};
    for (int l = 0; l < nlev; l++) {
        CLevel &L = A.lv[l];
        L.cx = ops[l].coef[0];
        L.cy = ops[l].coef[1];
        L.k2 = ops[l].k2;
        L.bk = ops[l].bk;
        L.c = ops[l].c;
        L.nx = n[l][0];
        L.ny = n[l][1];
        for (int r = 0; r <= MAX_CT_BLOCKS; r++) L.B[r] = B[l][std::min(r, nc)];
        L.ob = off[l][0]; L.ou = off[l][1]; L.ot = off[l][2]; L.ok = off[l][3]; L.oi = off[l][4];
        L.ocx = off[l][5]; L.ocy = off[l][6];
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

cudaError_t build_mg_ctail_image(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, void **out,
                                 cudaStream_t s) {
    *out = nullptr;
    CArgs A;
    const size_t bytes = ct_args(nlev, ops, minv, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    void *img = nullptr;
    cudaError_t e = cudaMalloc(&img, bytes * nc);
    if (e != cudaSuccess) return e;
    k_ctail_image<<<nc, CT_THREADS, 0, s>>>(A, (unsigned char *)img);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        cudaFree(img);
        return e;
    }
    *out = img;
    return cudaSuccess;
}

cudaError_t launch_mg_ctail(int nlev, const DevOp<float> *ops, const float2 *b_top, float2 *u_top,
                            const float2 *minv, int nu_c, int nu1, int nu2, int rb, float omega, int zero, int gf,
                            int gc, int nc, const void *img, cudaStream_t s) {
    CArgs A;
    const size_t bytes = ct_args(nlev, ops, minv, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.rb = rb;
    A.zero = zero;
    A.omega = omega;
    A.b_top = b_top;
    A.u_top = u_top;
    A.gf = gf;
    A.gc = gc;
    A.img = (const float4 *)img;
    static bool attr[2] = {false, false};
    const int ai = nc == 16;
    if (!attr[ai]) {
        cudaError_t e = cudaFuncSetAttribute(k_mg_ctail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM_BYTES);
        if (e == cudaSuccess && nc > 8) e = cudaFuncSetAttribute(k_mg_ctail, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr[ai] = true;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_mg_ctail, A);
}

// Batched tail over count problems whose tail levels have the shapes of ops (every problem's
// own pointers and prebuilt image in tab); one cluster of nc blocks per problem.
cudaError_t launch_mg_ctail_batch(int nlev, const DevOp<float> *ops, int nu_c, int nu1, int nu2, int rb, float omega,
                                  int gf, int gc, int nc, int count, const BTail *tab, int j, cudaStream_t s) {
    if (count < 1 || count > 65535) return cudaErrorInvalidValue;
    CArgs A;
    const size_t bytes = ct_args(nlev, ops, nullptr, nu_c, nc, A);
    if (!bytes) return cudaErrorInvalidValue;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.rb = rb;
    A.zero = 1;
    A.omega = omega;
    A.gf = gf;
    A.gc = gc;
    static bool attr[2] = {false, false};
    const int ai = nc == 16;
    if (!attr[ai]) {
        cudaError_t e = cudaFuncSetAttribute(k_mg_ctail_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM_BYTES);
        if (e == cudaSuccess && nc > 8) e = cudaFuncSetAttribute(k_mg_ctail_b, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr[ai] = true;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nc, 1, count);
    cfg.blockDim = dim3(CT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, k_mg_ctail_b, A, tab, j);
}

// Clusters of nc blocks with the given shared memory that the device can run at once (0: the
// configuration cannot be launched).
int mg_ctail_max_clusters(int nc, size_t bytes) {
    if (cudaFuncSetAttribute(k_mg_ctail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT_SMEM_BYTES) != cudaSuccess ||
        (nc > 8 && cudaFuncSetAttribute(k_mg_ctail, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(nc, 1, 1);
    cfg.blockDim = dim3(CT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_mg_ctail, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
