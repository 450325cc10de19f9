// Coarse levels of a 2D complex64 cycle (Algorithm 1) in ONE launch of a thread-block cluster.
//
// The coarse levels (129 x 129 nodes and below on the benchmark grids) hold too little work to
// fill the GPU, so as separate launches each costs a launch latency plus a few dependent
// phases, and on one thread block they are bound by one SM's issue rate.  Here a cluster of
// NC thread blocks (8 or 16 SMs) keeps every level's b, u, t, k^2 and coefficients in its
// distributed shared memory: each block owns a slab of interior rows of every level, reads
// the neighbouring slabs' boundary rows, and writes the coarsest solve's results, through
// distributed shared memory (cooperative_groups::cluster_group::map_shared_rank), and the
// phases of the cycle are separated by cluster barriers.  Same arithmetic as the per-level
// kernels in kernels_mg.cu: omega-Jacobi (ping-pong) or omega-red-black sweeps, residual and
// full weighting, bilinear prolongation, exact coarsest solve by the dense inverse.
#include <cooperative_groups.h>

#include <algorithm>

#include "helm_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int CT_THREADS = 512;

struct CLevel {
    const float2 *cx, *cy;  // global coefficient triples (3 nx, 3 ny)
    const float *k2;        // global k^2 (nx ny)
    float2 bk, c;
    int nx, ny, rows;       // rows: interior rows per block (the last block may own fewer)
    unsigned ob, ou, ot, ok, ocx, ocy;  // byte offsets in shared memory (same in every block)
};

struct CArgs {
    CLevel lv[MAX_CT_LEVELS];
    int nlev, nu_c, nu1, nu2, rb, zero, gf, gc;
    unsigned total;  // bytes of dynamic shared memory
    float omega;
    const float2 *minv;  // nu_c x nu_c, row-major (global)
    const float2 *b_top;  // top level's right-hand side (global)
    float2 *u_top;        // top level's result; initial guess when !zero (global)
    unsigned obc, ozero;  // compact coarsest right-hand side; a row of zeros
};

struct Ctx {
    unsigned char *sm;
    int rank, nc;
};

__device__ __forceinline__ int own_j0(const CLevel &L, int rank) { return 1 + rank * L.rows; }
__device__ __forceinline__ int own_j1(const CLevel &L, int rank) { return min(1 + (rank + 1) * L.rows, L.ny - 1); }

// Row j (0 .. ny-1) of the level array at offset off: in this block's or the owning block's
// shared memory; the boundary rows read as zeros.
__device__ __forceinline__ float2 *row(const Ctx &X, const CArgs &A, const CLevel &L, unsigned off, int j) {
    if (j <= 0 || j >= L.ny - 1) return (float2 *)(X.sm + A.ozero);
    const int owner = (j - 1) / L.rows, li = (j - 1) - owner * L.rows;
    float2 *p = (float2 *)(X.sm + off) + (size_t)li * L.nx;
    if (owner == X.rank) return p;
    return cg::this_cluster().map_shared_rank(p, (unsigned)owner);
}
__device__ __forceinline__ float2 *lrow(const Ctx &X, const CLevel &L, unsigned off, int j) {
    return (float2 *)(X.sm + off) + (size_t)(j - own_j0(L, X.rank)) * L.nx;
}

__device__ __forceinline__ void csync() { cg::this_cluster().sync(); }

// f(j, i) for every owned interior node: warps over owned rows, lanes over i.
template <typename F>
__device__ __forceinline__ void for_owned(const Ctx &X, const CLevel &L, F f) {
    const int j0 = own_j0(L, X.rank), j1 = own_j1(L, X.rank);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = j0 + warp; j < j1; j += nw)
        for (int i = 1 + lane; i <= L.nx - 2; i += 32) f(j, i);
}

__device__ __forceinline__ float2 diag_at(const Ctx &X, const CLevel &L, int j, int i) {
    const float2 *cx = (const float2 *)(X.sm + L.ocx), *cy = (const float2 *)(X.sm + L.ocy);
    const int li = j - own_j0(L, X.rank);
    const float k2 = ((const float *)(X.sm + L.ok))[(size_t)li * L.nx + i];
    return cadd(cadd(cx[3 * i + 1], cy[3 * li + 1]), cadd(cscale(L.bk, k2), L.c));
}

// (M u)(j, i) with u's rows j-1, j, j+1 given; d = the diagonal.
__device__ __forceinline__ float2 apply_at(const Ctx &X, const CLevel &L, int j, int i, const float2 *un,
                                           const float2 *uc, const float2 *us, float2 &d) {
    const float2 *cx = (const float2 *)(X.sm + L.ocx), *cy = (const float2 *)(X.sm + L.ocy);
    const int li = j - own_j0(L, X.rank);
    d = diag_at(X, L, j, i);
    float2 acc = cmul(cx[3 * i], uc[i - 1]);
    acc = cfma(cx[3 * i + 2], uc[i + 1], acc);
    acc = cfma(cy[3 * li], un[i], acc);
    acc = cfma(cy[3 * li + 2], us[i], acc);
    return cfma(d, uc[i], acc);
}

__device__ void zero_level(const Ctx &X, const CLevel &L, unsigned off) {
    for_owned(X, L, [&](int j, int i) { lrow(X, L, off, j)[i] = make_float2(0.f, 0.f); });
}

// nu sweeps on level L; *cur holds the iterate (offset), *oth the partner; zero: u = 0 on entry.
__device__ void ct_smooth(const Ctx &X, const CArgs &A, const CLevel &L, int nu, unsigned *cur, unsigned *oth,
                          bool zero) {
    if (zero && (nu == 0 || A.rb)) {
        zero_level(X, L, *cur);
        csync();
    }
    for (int s = 0; s < nu; s++) {
        if (A.rb) {
            for (int colour = 0; colour < 2; colour++) {
                const unsigned u = *cur;
                // the rows of this colour's neighbours are not written in this phase
                const int j0 = own_j0(L, X.rank), j1 = own_j1(L, X.rank);
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
                for (int j = j0 + warp; j < j1; j += nw) {
                    const float2 *un = row(X, A, L, u, j - 1), *us = row(X, A, L, u, j + 1);
                    float2 *uc = lrow(X, L, u, j);
                    const float2 *b = lrow(X, L, L.ob, j);
                    for (int i = 1 + lane; i <= L.nx - 2; i += 32) {
                        if (((i + j) & 1) != colour) continue;
                        float2 d;
                        const float2 mu = apply_at(X, L, j, i, un, uc, us, d);
                        uc[i] = cadd(uc[i], cscale(cmul(csub(b[i], mu), cinv(d)), A.omega));
                    }
                }
                csync();
            }
        } else {
            const bool z0 = zero && s == 0;
            const unsigned src = *cur, dst = *oth;
            const int j0 = own_j0(L, X.rank), j1 = own_j1(L, X.rank);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int j = j0 + warp; j < j1; j += nw) {
                const float2 *un = z0 ? nullptr : row(X, A, L, src, j - 1);
                const float2 *us = z0 ? nullptr : row(X, A, L, src, j + 1);
                const float2 *uc = lrow(X, L, src, j);
                const float2 *b = lrow(X, L, L.ob, j);
                float2 *out = lrow(X, L, dst, j);
                for (int i = 1 + lane; i <= L.nx - 2; i += 32) {
                    if (z0) {
                        out[i] = cscale(cmul(b[i], cinv(diag_at(X, L, j, i))), A.omega);
                    } else {
                        float2 d;
                        const float2 mu = apply_at(X, L, j, i, un, uc, us, d);
                        out[i] = cadd(uc[i], cscale(cmul(csub(b[i], mu), cinv(d)), A.omega));
                    }
                }
            }
            csync();
            *cur = dst;
            *oth = src;
        }
    }
}

// Exact coarsest solve: every block gathers the whole right-hand side, computes its share of
// the rows of Minv b (one warp per row) and stores each result in the owning block's u.
__device__ void ct_dense(const Ctx &X, const CArgs &A, const CLevel &L) {
    float2 *bc = (float2 *)(X.sm + A.obc);
    const int mx = L.nx - 2, nu = A.nu_c;
    for (int c = threadIdx.x; c < nu; c += blockDim.x) {
        const int i = 1 + c % mx, j = 1 + c / mx;
        bc[c] = row(X, A, L, L.ob, j)[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = X.rank * nw + warp; r < nu; r += X.nc * nw) {
        const float2 *mrow = A.minv + (size_t)r * nu;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = lane; c < nu; c += 32) acc = cfma(mrow[c], bc[c], acc);
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) row(X, A, L, L.ou, 1 + r / mx)[1 + r % mx] = acc;
    }
    csync();
}

// Level LVL of the cycle (compile-time depth); the result ends in the level's u.
template <int LVL>
__device__ void ct_cycle(const Ctx &X, const CArgs &A, bool zero, int gf, int gc) {
    const CLevel &L = A.lv[LVL];
    if (LVL == A.nlev - 1) {
        ct_dense(X, A, L);
        return;
    }
    if constexpr (LVL + 1 < MAX_CT_LEVELS) {
        unsigned cur = L.ou, oth = L.ot;
        ct_smooth(X, A, L, A.nu1, &cur, &oth, zero);
        const CLevel &Lc = A.lv[LVL + 1];
        // residual into the free partner array, then full weighting into the coarse b
        {
            const int j0 = own_j0(L, X.rank), j1 = own_j1(L, X.rank);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int j = j0 + warp; j < j1; j += nw) {
                const float2 *un = row(X, A, L, cur, j - 1), *us = row(X, A, L, cur, j + 1);
                const float2 *uc = lrow(X, L, cur, j), *b = lrow(X, L, L.ob, j);
                float2 *r = lrow(X, L, oth, j);
                for (int i = 1 + lane; i <= L.nx - 2; i += 32) {
                    float2 d;
                    r[i] = csub(b[i], apply_at(X, L, j, i, un, uc, us, d));
                }
            }
        }
        csync();
        for_owned(X, Lc, [&](int J, int I) {
            const float2 *r0 = row(X, A, L, oth, 2 * J - 1), *r1 = row(X, A, L, oth, 2 * J),
                         *r2 = row(X, A, L, oth, 2 * J + 1);
            const int x = 2 * I;
            const float2 a0 = cadd(cadd(r0[x - 1], r0[x + 1]), cscale(r0[x], 2.f));
            const float2 a1 = cadd(cadd(r1[x - 1], r1[x + 1]), cscale(r1[x], 2.f));
            const float2 a2 = cadd(cadd(r2[x - 1], r2[x + 1]), cscale(r2[x], 2.f));
            lrow(X, Lc, Lc.ob, J)[I] = cscale(cadd(cadd(a0, a2), cscale(a1, 2.f)), 0.0625f);
        });
        csync();
        if (LVL + 1 == A.nlev - 1) {
            ct_dense(X, A, Lc);
        } else {
            for (int k = 1; k <= gc; k++) {
                if (k == 1) ct_cycle<LVL + 1>(X, A, true, gf, gc);
                else ct_cycle<LVL + 1>(X, A, false, gc, gf);
            }
        }
        // bilinear prolongation of the coarse result, added to the iterate
        for_owned(X, L, [&](int j, int i) {
            const float2 *ea = row(X, A, Lc, Lc.ou, j >> 1), *eb = row(X, A, Lc, Lc.ou, (j + 1) >> 1);
            const int ia = i >> 1, ib = (i + 1) >> 1;
            const float2 e = cadd(cadd(ea[ia], ea[ib]), cadd(eb[ia], eb[ib]));
            float2 *uc = lrow(X, L, cur, j);
            uc[i] = cadd(uc[i], cscale(e, 0.25f));
        });
        csync();
        ct_smooth(X, A, L, A.nu2, &cur, &oth, false);
        if (cur != L.ou) {
            const unsigned src = cur;
            for_owned(X, L, [&](int j, int i) { lrow(X, L, L.ou, j)[i] = lrow(X, L, src, j)[i]; });
            csync();
        }
    }
}

__global__ void __launch_bounds__(CT_THREADS) k_mg_ctail(CArgs A) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char ct_smem[];
    cg::cluster_group cl = cg::this_cluster();
    Ctx X{ct_smem, (int)cl.block_rank(), (int)cl.num_blocks()};
    // zero all of it (boundary columns and the zero row stay zero), stage k^2 and coefficients
    for (unsigned q = threadIdx.x; q < A.total / 16; q += blockDim.x) ((float4 *)ct_smem)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int l = 0; l < A.nlev; l++) {
        const CLevel &L = A.lv[l];
        const int j0 = own_j0(L, X.rank), j1 = own_j1(L, X.rank);
        float2 *cx = (float2 *)(ct_smem + L.ocx), *cy = (float2 *)(ct_smem + L.ocy);
        float *k2 = (float *)(ct_smem + L.ok);
        for (int q = threadIdx.x; q < 3 * L.nx; q += blockDim.x) cx[q] = L.cx[q];
        for (int q = threadIdx.x; q < 3 * (j1 - j0); q += blockDim.x) cy[q] = L.cy[3 * j0 + q];
        for (int q = threadIdx.x; q < (j1 - j0) * L.nx; q += blockDim.x) k2[q] = L.k2[(size_t)j0 * L.nx + q];
    }
    const CLevel &T = A.lv[0];
    for_owned(X, T, [&](int j, int i) {
        const size_t p = (size_t)i + (size_t)T.nx * j;
        lrow(X, T, T.ob, j)[i] = A.b_top[p];
        if (!A.zero) lrow(X, T, T.ou, j)[i] = A.u_top[p];
    });
    csync();
    ct_cycle<0>(X, A, A.zero != 0, A.gf, A.gc);
    for_owned(X, T, [&](int j, int i) { A.u_top[(size_t)i + (size_t)T.nx * j] = lrow(X, T, T.ou, j)[i]; });
    csync();  // no block leaves while another may still read its shared memory
}

}  // namespace

// Shared-memory layout of the cluster tail (identical in every block): per level b, u, t
// (rows x nx complex64 each), k^2 (rows x nx floats), x coefficients (3 nx), y coefficients of
// the owned rows (3 rows); then the compact coarsest right-hand side and a zero row.
size_t mg_ctail_layout(int nlev, const int (*n)[3], int nc, int nu_c, unsigned (*off)[6], unsigned *obc,
                       unsigned *ozero) {
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    size_t p = 0;
    int maxnx = 0;
    for (int l = 0; l < nlev; l++) {
        const int nx = n[l][0], ny = n[l][1], rows = (ny - 2 + nc - 1) / nc;
        maxnx = std::max(maxnx, nx);
        const size_t vec = al((size_t)rows * nx * sizeof(float2));
        off[l][0] = (unsigned)p; p += vec;                                             // b
        off[l][1] = (unsigned)p; p += vec;                                             // u
        off[l][2] = (unsigned)p; p += vec;                                             // t
        off[l][3] = (unsigned)p; p += al((size_t)rows * nx * sizeof(float));           // k^2
        off[l][4] = (unsigned)p; p += al((size_t)3 * nx * sizeof(float2));             // x coefficients
        off[l][5] = (unsigned)p; p += al((size_t)3 * rows * sizeof(float2));           // y coefficients
    }
    *obc = (unsigned)p;
    p += al((size_t)nu_c * sizeof(float2));
    *ozero = (unsigned)p;
    p += al((size_t)maxnx * sizeof(float2));
    return p;
}

cudaError_t launch_mg_ctail(int nlev, const DevOp<float> *ops, const float2 *b_top, float2 *u_top,
                            const float2 *minv, int nu_c, int nu1, int nu2, int rb, float omega, int zero, int gf,
                            int gc, int nc, cudaStream_t s) {
    if (nlev < 2 || nlev > MAX_CT_LEVELS || (nc != 8 && nc != 16)) return cudaErrorInvalidValue;
    int n[MAX_CT_LEVELS][3];
    for (int l = 0; l < nlev; l++)
        for (int a = 0; a < 3; a++) n[l][a] = ops[l].n[a];
    unsigned off[MAX_CT_LEVELS][6], obc = 0, ozero = 0;
    const size_t bytes = mg_ctail_layout(nlev, n, nc, nu_c, off, &obc, &ozero);
    if (bytes > CT_SMEM_BYTES) return cudaErrorInvalidValue;
    CArgs A{};
    for (int l = 0; l < nlev; l++) {
        CLevel &L = A.lv[l];
        L.cx = ops[l].coef[0];
        L.cy = ops[l].coef[1];
        L.k2 = ops[l].k2;
        L.bk = ops[l].bk;
        L.c = ops[l].c;
        L.nx = n[l][0];
        L.ny = n[l][1];
        L.rows = (n[l][1] - 2 + nc - 1) / nc;
        L.ob = off[l][0]; L.ou = off[l][1]; L.ot = off[l][2]; L.ok = off[l][3]; L.ocx = off[l][4]; L.ocy = off[l][5];
    }
    A.nlev = nlev;
    A.nu_c = nu_c;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.rb = rb;
    A.zero = zero;
    A.omega = omega;
    A.minv = minv;
    A.b_top = b_top;
    A.u_top = u_top;
    A.obc = obc;
    A.ozero = ozero;
    A.total = (unsigned)bytes;
    A.gf = gf;
    A.gc = gc;
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
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = nc;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mg_ctail, A);
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
