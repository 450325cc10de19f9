// Internal declarations shared by the libhelm translation units (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/helm.h"

// ------------------------------------------------------------------------------ complex
template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
    return mk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a)*b
template <typename C> __host__ __device__ __forceinline__ C cfmac(C a, C b, C acc) {
    return mk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
// 1 / a = conj(a) / |a|^2 (one real division)
template <typename C> __host__ __device__ __forceinline__ C cinv(C a) {
    const auto d = a.x * a.x + a.y * a.y;
    const auto r = decltype(d)(1) / d;
    return mk(a.x * r, -a.y * r);
}
// 1 / a for complex64 with the fast approximate reciprocal (__fdividef, about 2 ulp): used
// where the result only enters a complex64 smoother update.
__device__ __forceinline__ float2 cinv_fast(float2 a) {
    const float r = __fdividef(1.0f, a.x * a.x + a.y * a.y);
    return make_float2(a.x * r, -a.y * r);
}
// dst[q] = src[q] for q < n (src global and unchanged during the kernel, dst this block's
// shared memory): each thread issues eight loads before it stores, so that a block's copy takes
// a few memory round trips instead of one per float4 a thread moves.
__device__ __forceinline__ void block_copy16(float4 *dst, const float4 *__restrict__ src, unsigned n) {
    constexpr int U = 8;
    for (unsigned q0 = threadIdx.x; q0 < n; q0 += U * blockDim.x) {
        float4 r[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned q = q0 + u * blockDim.x;
            r[u] = q < n ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned q = q0 + u * blockDim.x;
            if (q < n) dst[q] = r[u];
        }
    }
}
__device__ __forceinline__ float2 to_c(float2 v, float) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(float2 v, double) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double) { return v; }

// ------------------------------------------------------------------------------ operator
// One discrete operator on one level:
//   (M x)_p = sum_axes (cw x_{p-e} + cc x_p + ce x_{p+e}) + (bk k2_p + c) x_p,
// with the operator scale a already folded into the per-axis coefficient triples
// coef[ax][3*j + {0,1,2}] = (cw, cc, ce) at node j of axis ax.
template <typename R> struct DevOp {
    typedef typename CT<R>::T C;
    int n[3];
    const C *coef[3];
    const R *k2;
    C bk, c;
    // 2D complex64 levels: 1 / (diagonal of M) at every node (0 off the interior), formed once
    // by launch_diag_inv for the temporally blocked smoothers; null otherwise
    const C *dinv = nullptr;
    // device flag (null: none): when it is set at launch, this level's smoothing, residual and
    // transfer kernels return at once (the fused coarse-tail kernels do not test it).  Set only
    // while the launches of an FGMRES step that may be queued behind a converged one are made.
    const int *gate = nullptr;
};

// The Helmholtz operator A = L_h - k^2 with coefficients and k^2 stored as float pairs
// (hi + lo, see df_arith.h): coef[ax][3*j + t] = (re.hi, re.lo, im.hi, im.lo), k2[p] = (hi, lo).
struct DevOpDF {
    int n[3];
    const float4 *coef[3];
    const float2 *k2;
};
// y = A z in double-FP32 arithmetic, z complex64, y a float-pair vector (interior written).
// gate (may be null): nothing is written when the device flag is set at launch.
cudaError_t launch_apply_A_df(const DevOpDF &op, int dim, const float2 *z, float4 *y, cudaStream_t s,
                             const int *gate = nullptr);

// Programmatic dependent launch.  Every kernel of the library begins with pdl_wait() (it returns
// once the kernel before it in the stream has finished and its writes are visible; a no-op when
// the kernel was launched without the attribute) and pdl_trigger() (the next kernel may be
// scheduled as soon as all of this kernel's blocks have started, so its launch overlaps this
// kernel's tail).  launch_pdl() launches with the attribute, except while the calling thread
// captures a CUDA graph (pdl_capture_scope): measured on GB300, replayed graphs of the FGMRES
// steps ran about 4% slower with programmatic edges, while eager launch sequences (the cycle
// alone) ran about 10% faster with them.
// Launches under pdl_cycle_scope keep the attribute inside captured graphs too: the multigrid
// cycle's (short, latency-bound kernels, each letting the next one's blocks be scheduled while it
// drains), and in a delayed-CGS2 step the reduction (a few blocks, placed while the dot pass
// drains) and the update pass after it (placed while the reduction's few blocks finish).
extern thread_local bool g_pdl_off, g_pdl_cycle;
constexpr bool kPdlCycleInGraphs = true;
struct pdl_capture_scope {
    bool keep;
    pdl_capture_scope() : keep(g_pdl_off) { g_pdl_off = true; }
    ~pdl_capture_scope() { g_pdl_off = keep; }
};
struct pdl_cycle_scope {
    bool keep;
    pdl_cycle_scope() : keep(g_pdl_cycle) { g_pdl_cycle = kPdlCycleInGraphs; }
    ~pdl_cycle_scope() { g_pdl_cycle = keep; }
};
inline bool pdl_enabled() { return !g_pdl_off || g_pdl_cycle; }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}
// Value of a gate flag (0 when there is none).  Kernels load it first and test it only after
// they have issued their first loads, so that its latency overlaps theirs.
__device__ __forceinline__ int gate_value(const int *g) { return g ? *g : 0; }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Host setup shared by the translation units (helm_api.cu): the linear ECS contour of one axis
// (Section 3.1) and its per-node FD coefficient triples (cw, cc, ce) of a * (-d^2/dz^2) with every
// width multiplied by e^{i ts} (Section 3.2).
std::vector<std::complex<double>> ecs_contour(int n, double lo, double hi, double theta, double r0lo, double r0hi);
std::vector<std::complex<double>> fd_triples(const std::vector<std::complex<double>> &z, double ts,
                                             std::complex<double> a);

// Kernel launch geometry helpers
static inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------------------ launchers
// All return cudaGetLastError() of their launch.  R = float or double; dim = 2 or 3.
// Vectors are full node arrays (boundary included).
template <typename R, typename CX>
cudaError_t launch_apply(const DevOp<R> &op, int dim, const CX *x, typename CT<R>::T *y, cudaStream_t s);
template <typename R, typename CB>
cudaError_t launch_residual(const DevOp<R> &op, int dim, const CB *b, const typename CT<R>::T *u,
                            typename CT<R>::T *r, cudaStream_t s);
// u_out = u_in + omega (b - M u_in) / diag(M); u_in == nullptr means u_in = 0.
template <typename R, typename CB>
cudaError_t launch_jacobi(const DevOp<R> &op, int dim, R omega, const CB *b, const typename CT<R>::T *u_in,
                          typename CT<R>::T *u_out, cudaStream_t s);
// one colour of omega-red-black Jacobi, in place; colour 0 = (i+j+k) even.
template <typename R, typename CB>
cudaError_t launch_rb(const DevOp<R> &op, int dim, R omega, const CB *b, typename CT<R>::T *u, int colour,
                      cudaStream_t s);
// rc = FW(b - M u) on the coarse grid (fine nodes op.n, coarse nodes (n+1)/2).
template <typename R, typename CB>
cudaError_t launch_residual_restrict(const DevOp<R> &op, int dim, const CB *b, const typename CT<R>::T *u,
                                     typename CT<R>::T *rc, cudaStream_t s);
// uf += P ec (fine nodes nf).
template <typename R>
cudaError_t launch_prolong_add(const int nf[3], int dim, const typename CT<R>::T *ec, typename CT<R>::T *uf,
                               cudaStream_t s, const int *gate = nullptr);
// u = Minv b on the interior unknowns of the coarsest grid (nodes n), natural order.
template <typename R>
cudaError_t launch_dense_solve(const int n[3], int dim, int nu, const typename CT<R>::T *minv,
                               const typename CT<R>::T *b, typename CT<R>::T *u, cudaStream_t s);
// Temporal blocking (2D, complex64, omega-Jacobi with two pre- and two post-sweeps):
//   pre:  u_out = two sweeps from u = 0, rc = FW(b - M u_out)   (one launch)
//   post: u_out = two sweeps of (u_in + P ec)                     (one launch; u_in != u_out)
// tile: index of the tile shape (HELM_TILE_* in helm.h).  fused_jacobi2_ok tells whether a
// level's grid fits the tiling with that tile.
bool fused_jacobi2_ok(const int n[3], int dim, int tile);
// Register-wavefront versions (kernels_wave.cu; tile HELM_TILE_WAVE): same contracts.
bool wave_jacobi2_ok(const int n[3], int dim);
cudaError_t launch_pre2_wave(const DevOp<float> &op, float omega, const float2 *b, float2 *u_out, float2 *rc,
                             cudaStream_t s);
cudaError_t launch_post2_wave(const DevOp<float> &op, float omega, const float2 *b, const float2 *u_in, float2 *u_out,
                              const float2 *ec, cudaStream_t s);
// dinv = 1 / (diagonal of M) at every node of a 2D level (0 off the interior)
cudaError_t launch_diag_inv(const DevOp<float> &op, float2 *dinv, cudaStream_t s);
cudaError_t launch_pre2_restrict(const DevOp<float> &op, int tile, float omega, const float2 *b, float2 *u_out,
                                 float2 *rc, cudaStream_t s);
cudaError_t launch_prolong_post2(const DevOp<float> &op, int tile, float omega, const float2 *b, const float2 *u_in,
                                 float2 *u_out, const float2 *ec, cudaStream_t s);

// Fused coarse tail: Algorithm 1 on levels 0..nlev-1 of the given arrays (level 0 = the
// tail's top, nlev - 1 = the coarsest, solved with minv) inside one thread block.  zero: the
// top-level iterate u[0] starts at 0 (not read).  Levels with at most TAIL_MAX_UNKNOWNS
// interior nodes, MAX_TAIL_LEVELS at most, go to the tail.
constexpr int MAX_TAIL_LEVELS = 4;
constexpr int TAIL_MAX_UNKNOWNS = 4096;
constexpr size_t TAIL_SMEM_BYTES = 200 * 1024;  // b, u, t of every tail level in shared memory
// Dynamic shared memory of the fused tail: the coarsest solve's compact right-hand side
// (nu_c values, rounded up to even), b, u, t of every tail level, then every tail level's
// coefficient triples and k^2 (each k^2 array padded to 16 bytes).
inline size_t mg_tail_smem_bytes_nodes(int dim, int nlev, const int (*n)[3], int nu_c, size_t es) {
    size_t bytes = (size_t)((nu_c + 1) & ~1) * es;
    for (int l = 0; l < nlev; l++) {
        const size_t np = (size_t)n[l][0] * n[l][1] * (dim == 3 ? n[l][2] : 1);
        bytes += 3 * es * np;                                                  // b, u, t
        bytes += 3 * es * (size_t)(n[l][0] + n[l][1] + (dim == 3 ? n[l][2] : 0));  // coefficients
        bytes += (np * (es / 2) + 15) & ~(size_t)15;                           // k^2
    }
    return bytes;
}
template <typename R>
inline size_t mg_tail_smem_bytes(int dim, int nlev, const DevOp<R> *ops, int nu_c, size_t es) {
    int n[MAX_TAIL_LEVELS][3];
    for (int l = 0; l < nlev && l < MAX_TAIL_LEVELS; l++)
        for (int a = 0; a < 3; a++) n[l][a] = ops[l].n[a];
    return mg_tail_smem_bytes_nodes(dim, nlev < MAX_TAIL_LEVELS ? nlev : MAX_TAIL_LEVELS, n, nu_c, es);
}
template <typename R>
cudaError_t launch_mg_tail(int dim, int nlev, const DevOp<R> *ops, typename CT<R>::T *const *b,
                           typename CT<R>::T *const *u, typename CT<R>::T *const *t, const typename CT<R>::T *minv,
                           int nu_c, int nu1, int nu2, int rb, R omega, int gf, int gc, int zero, cudaStream_t s);
// Cluster tail (kernels_ctail.cu): the coarsest nlev levels of a 2D complex64 cycle in one
// launch of a cluster of nc = 8 or 16 thread blocks, every level in distributed shared memory
// (rows split into slabs).  b_top / u_top: the first of those levels' right-hand side and result
// (global; u_top is the initial guess unless zero).
constexpr int MAX_CT_LEVELS = 6;
constexpr int MAX_CT_BLOCKS = 16;      // blocks per cluster at most
constexpr int CT_BLOCK_THREADS = 512;  // threads per block of a cluster tail
constexpr size_t CT_SMEM_BYTES = 200 * 1024;
// Nested row slabs of the tail levels: block r owns the interior rows B[l][r] .. B[l][r+1]-1 of
// level l (level 0 in runs of ceil((ny - 2) / nc) rows, B[l+1][r] = (B[l][r] + 1) / 2).  False
// unless every level has odd ny and the next has (ny + 1) / 2.
bool mg_ctail_bounds(int nlev, const int (*n)[3], int nc, int (*B)[MAX_CT_BLOCKS + 1]);
// Rows of the coarsest inverse each warp stages in the dense phase, and their shared-memory
// bytes (0 when above 64 KB: the rows are then read from global memory).
int mg_ctail_minv_rows(int nc, int nu_c);
size_t mg_ctail_minv_stage_bytes(int nc, int nu_c);
size_t mg_ctail_layout(int nlev, const int (*n)[3], int nc, int nu_c, unsigned (*off)[7], unsigned *obc,
                       unsigned *ominv);
// img: the blocks' initial shared memory from build_mg_ctail_image for the same levels and nc
// (null: each launch builds it itself); *out is device memory the caller frees.
cudaError_t launch_mg_ctail(int nlev, const DevOp<float> *ops, const float2 *b_top, float2 *u_top,
                            const float2 *minv, int nu_c, int nu1, int nu2, int rb, float omega, int zero, int gf,
                            int gc, int nc, const void *img, cudaStream_t s);
cudaError_t build_mg_ctail_image(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, void **out,
                                 cudaStream_t s);
int mg_ctail_max_clusters(int nc, size_t bytes);
// Deep-halo cluster tail (kernels_chalo.cu): the same levels for a V-cycle of omega-Jacobi with
// nu1, nu2 <= 2 sweeps from a zero guess, each block keeping three rows beyond its slab so that
// each level needs one cluster barrier down and one up.  img (required): the blocks' initial
// shared memory from build_mg_chalo_image.  mg_chalo_bytes: its shared memory per block (0: the
// levels do not fit).
size_t mg_chalo_layout(int nlev, const int (*n)[3], int nc, int nu_c, unsigned (*off)[8], unsigned *obc,
                       unsigned *ominv);
size_t mg_chalo_bytes(int nlev, const DevOp<float> *ops, int nu_c, int nc);
cudaError_t build_mg_chalo_image(int nlev, const DevOp<float> *ops, const float2 *minv, int nu_c, int nc, void **out,
                                 cudaStream_t s);
cudaError_t launch_mg_chalo(int nlev, const DevOp<float> *ops, const float2 *b_top, float2 *u_top, const float2 *minv,
                            int nu_c, int nu1, int nu2, float omega, int nc, const void *img, cudaStream_t s);
int mg_chalo_max_clusters(int nc, size_t bytes);

// ------------------------------------------------------------------------------ batched launches
// One launch covers the same phase of many problems (helm_solve_batch): a batched kernel reads
// the table entry of blockIdx.z (or of the block range that holds blockIdx.x) and returns at
// once when that problem's *active is 0.  Tables live in device memory.
//
// A level of one problem at one cycle phase (all entries of a launch have the same level shape):
//   pre:  t = two sweeps from zero for M u = b, coarse = FW(b - M t)
//   post: (u + j ustride) = two sweeps of (t + P coarse)
struct BLevel {
    DevOp<float> op;   // the level's complex64 operator (dinv set)
    const float2 *b;   // right-hand side
    float2 *t;         // pre: smoothed iterate (written); post: iterate (read)
    float2 *u;         // post: result base
    size_t ustride;    // post: the result is u + j * ustride (level 0: the j-th preconditioned vector)
    float2 *coarse;    // pre: next level's right-hand side (written); post: next level's result (read)
    const int *active;
};
// A problem's cluster tail (levels of equal shapes in every entry; image: the problem's prebuilt
// initial shared memory for that tail).
struct BTail {
    const float2 *cx[MAX_CT_LEVELS], *cy[MAX_CT_LEVELS];
    const float *k2[MAX_CT_LEVELS];
    const float2 *minv;
    const float2 *b_top;
    float2 *u_top;      // result base: the result is u_top + j * ustride
    size_t ustride;     // nonzero when the tail's top is the finest level (the j-th preconditioned vector)
    const void *img;
    const int *active;
};
// A problem's Krylov state for the batched delayed-CGS2 FGMRES step kernels.
struct BVec {
    size_t n;            // nodes
    float4 *V;           // float-pair basis, slot stride n
    float2 *Z;           // complex64 preconditioned vectors, slot stride n
    float2 *b0;          // level 0's complex64 right-hand side (the next cycle's input)
    DevOpDF A;           // A in double-FP32
    double2 *partials, *hv, *alpha2, *H, *dcoef, *g, *sn;
    const double2 *fnorm;
    double *cs, *est;
    unsigned *tickets;
    int ldh;
    int *active;  // the problem's flag (the batched rotation clears it on convergence)
};
cudaError_t launch_pre2_restrict_batch(const int n[3], int tile, int count, const BLevel *tab, float omega,
                                       cudaStream_t s);
cudaError_t launch_prolong_post2_batch(const int n[3], int tile, int count, const BLevel *tab, float omega, int j,
                                       cudaStream_t s);
cudaError_t launch_mg_ctail_batch(int nlev, const DevOp<float> *ops, int nu_c, int nu1, int nu2, int rb, float omega,
                                  int gf, int gc, int nc, int count, const BTail *tab, int j, cudaStream_t s);
cudaError_t launch_mg_chalo_batch(int nlev, const DevOp<float> *ops, int nu_c, int nu1, int nu2, float omega, int nc,
                                  int count, const BTail *tab, int j, cudaStream_t s);
// Flat blocks of one problem's batched 2D apply; problem e takes [first[e], first[e + 1]).
unsigned apply_A_df_blocks(const int n[3]);
cudaError_t launch_apply_A_df_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                    cudaStream_t s);
// Block rows of the two-vector dot pass over nv basis vectors (its grid is gs_df_dot2_nblocks x
// this); problem e's dot-pass blocks of step j are [first[e], first[e + 1]) of the launch.
int gs_df_dot2_groups(int nv);
// close: the closing step of a cycle with j columns (x and w both slot j)
cudaError_t launch_mdot2_pair_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                    int close, cudaStream_t s);
// has_w: 2 (w came from the unscaled slot j), 1 (w from slot 0), 0 (closing step: no new column)
cudaError_t launch_reduce_dcgs2_batch(int count, const BVec *tab, const unsigned *first, int groups, int j,
                                      int has_w, cudaStream_t s);
cudaError_t launch_update2_pair_batch(int count, const BVec *tab, const unsigned *first, unsigned nblocks, int j,
                                      cudaStream_t s);
// Rotation of column j of every active problem; est_out[e] = its est[j] (-1 if inactive).
// tol (device, may be null): problems whose estimate meets it are made inactive
cudaError_t launch_givens_batch(int count, const BVec *tab, int j, double *est_out, const double *tol, cudaStream_t s);

template <typename CI, typename CO>
cudaError_t launch_convert(size_t n, const CI *in, CO *out, cudaStream_t s);
template <typename C>
cudaError_t launch_zero(size_t n, C *x, cudaStream_t s);

// FP64 vector kernels on full node arrays (boundary values are zero, so sums over all nodes
// equal sums over unknowns).
// Number of blocks of every reduction over n nodes (fixed per n, so sums are reproducible).
int blas_nblocks(size_t n);
// Gram-Schmidt passes (gate: device int; the kernel returns at once when *gate == 0).
// partials[i * G + b] = sum conj(V_i) w (i < nv) and partials[nv * G + b] = (||w||^2, 0),
// G = blas_nblocks(n).
cudaError_t launch_mdot_norm(size_t n, const double2 *V, size_t ldv, int nv, const double2 *w, double2 *partials,
                             const int *gate, cudaStream_t s);
// w -= sum_i V_i h_i, then partials[b] = (||w||^2, 0)   (h on device)
cudaError_t launch_update_norm(size_t n, const double2 *V, size_t ldv, int nv, const double2 *h, double2 *w,
                               double2 *partials, const int *gate, cudaStream_t s);
// out[i] (mode 0: =, 1: +=, 2: (sqrt(re), 0)) = fixed-order sum of partials of vector i; with
// host_out (pinned host memory), host_out[i] = the real part of out[i] as well
cudaError_t launch_reduce(const double2 *partials, int nblk, int nv, double2 *out, int mode, const int *gate,
                          cudaStream_t s, double *host_out = nullptr);
// Same two passes in double-FP32 arithmetic on float-pair vectors (kernels_gs_df.cu): node q
// of such a vector is the float4 (re.hi, re.lo, im.hi, im.lo).  Dot-pass partials use
// G = gs_df_nblocks(n) blocks per vector, update-pass partials gs_df_update_nblocks(n).
int gs_df_nblocks(size_t n);         // dot pass
int gs_df_dot2_nblocks(size_t n, int nv);  // two-vector dot pass over nv basis vectors
int gs_df_update_nblocks(size_t n);  // update pass
cudaError_t launch_mdot_norm_pair(size_t n, const float4 *V, size_t ldv, int nv, const float4 *w, double2 *partials,
                                  const int *gate, cudaStream_t s);
cudaError_t launch_update_norm_pair(size_t n, const float4 *V, size_t ldv, int nv, const double2 *h, float4 *w,
                                    double2 *partials, const int *gate, cudaStream_t s);
// Delayed CGS2 (one dot and one update pass per Arnoldi step, float pairs):
//   dot:    partials[i*G+b] = V_i^H x, partials[(nv+i)*G+b] = V_i^H w  (i < nv, G = gs_df_dot2_nblocks)
//   coef:   one-thread FP64 step of the method (kernels_krylov.cu)
//   update: slot j <- final v_j, slot j+1 <- once-orthogonalised w; partials[b] = ||w||^2
//           (G = gs_df_update_nblocks)
// The update pass with a ticket (a device counter at 0 between launches) writes (||w||, 0) to
// alpha_out from its last block; without one (null) it only writes partials.  The dot pass's
// partials go to launch_reduce_dcgs2: one block per value, and the last block to finish runs the
// coefficient step of step j (ticket as above); w_scaled: w and its inner products are
// alpha_j times the true ones (the preconditioner was applied to the unscaled slot j).
// The update pass scales w by coef[2j+2].x and, with b_out, also writes the new slot j + 1 as
// complex64 (the next step's preconditioner input).
// gate (may be null): a device flag; when it is set at launch, the dot pass writes nothing and the
// update pass leaves the vectors as they are (its norm partials are zero and its ticket protocol
// still runs) -- used to skip FGMRES steps queued ahead of a converged one.
cudaError_t launch_mdot2_pair(size_t n, const float4 *V, size_t ldv, int nv, const float4 *x, const float4 *w,
                              double2 *partials, const int *gate, cudaStream_t s);
// has_w as in launch_reduce_dcgs2_batch
cudaError_t launch_reduce_dcgs2(const double2 *partials, int nblk, double2 *hv, unsigned *ticket, int j,
                                const double2 *alpha2, double2 *H, int ldh, double2 *coef, int has_w,
                                cudaStream_t s);
cudaError_t launch_dcgs2_coef(int j, int has_w, const double2 *hv, const double2 *alpha2, double2 *H, int ldh,
                              double2 *coef, cudaStream_t s);
cudaError_t launch_update2_pair(size_t n, float4 *V, size_t ldv, int j, const double2 *coef, double2 *partials,
                                unsigned *ticket, double2 *alpha_out, float2 *b_out, const int *gate, cudaStream_t s);
// w <- w / beta->x (float pairs)
cudaError_t launch_scale_inv_pair(size_t n, float4 *w, const double2 *beta, cudaStream_t s);
// in place: the double2 vector x becomes the float-pair vector x / beta->x (beta null: 1)
cudaError_t launch_split_scale(size_t n, void *x, const double2 *beta, cudaStream_t s);
// float pairs / alpha->x -> complex64 / complex128 (alpha null: no scaling)
cudaError_t launch_pair_to_c64(size_t n, const float4 *v, const double2 *alpha, float2 *z, cudaStream_t s);
cudaError_t launch_pair_to_c128(size_t n, const float4 *v, const double2 *alpha, double2 *z, cudaStream_t s);
// *hnorm: ||w||^2 in, ||w'|| out; *flag = (||w'|| < eta ||w||); *count += flag
cudaError_t launch_reduce_decide(const double2 *partials, int nblk, double2 *hnorm, int *flag, int *count, double eta,
                                 cudaStream_t s);
// y = x * (1 / scale[0].x)
cudaError_t launch_scale_inv(size_t n, const double2 *x, const double2 *scale, double2 *y, cudaStream_t s);
// x += sum_c y_c Z_c  (Z c64 or c128, ldz stride); with alpha (c64 only) the weights are
// y_c / alpha[c].x for c >= 1 (columns that hold alpha_c z_c)
template <typename CZ>
cudaError_t launch_combine(size_t n, const CZ *Z, size_t ldz, int nz, const double2 *y, const double2 *alpha,
                           double2 *x, cudaStream_t s);

// FGMRES small dense work on the device (one warp): rotations of column j, new rotation,
// residual estimate |g_{j+1}| / fnorm->x written to est[j] and, when est_host is not null, to
// est_host[j] (pinned host memory).  With stop not null, *stop = 1 when est[j] <= *tol (or is not
// a number): the host's own convergence test, taken on the device so that the steps already
// queued behind this one skip their vector passes.
cudaError_t launch_givens(double2 *H, int ldh, int j, double *cs, double2 *sn, double2 *g, const double2 *fnorm,
                          double *est, double *est_host, const double *tol, int *stop, cudaStream_t s);
// Start of an FGMRES cycle: g = (beta, 0, ..., 0) (len entries, beta = *beta), *stop = 0 and
// *tol_dev = tol.
cudaError_t launch_cycle_start(double2 *g, int len, const double2 *beta, int *stop, double *tol_dev, double tol,
                               cudaStream_t s);
// y = H(0:k,0:k)^{-1} g(0:k)  (upper triangular back substitution)
cudaError_t launch_backsolve(const double2 *H, int ldh, int k, const double2 *g, double2 *y, cudaStream_t s);

// Bi-CGSTAB vector updates (FP64)
// p = r + beta (p - omega v), beta and omega from dev scalars
cudaError_t launch_bicg_p(size_t n, const double2 *r, const double2 *v, const double2 *sc, double2 *p,
                          cudaStream_t s);
// generic: y = a*x + b*y with device complex scalars a, b (pointers into a scalar block)
cudaError_t launch_axpby(size_t n, const double2 *a, const double2 *x, const double2 *b, double2 *y,
                         cudaStream_t s);
template <typename CY>
cudaError_t launch_axpy_mixed(size_t n, const double2 *a, const CY *x, double2 *y, cudaStream_t s);
// scalar kernels of Bi-CGSTAB (device-side scalar algebra, no host round trip)
cudaError_t launch_bicg_scalars(int stage, double2 *sc, cudaStream_t s);

// adjoint helpers
// y = w x or x / w (inverse) with w the product of the axes' dual volumes, on interior nodes;
// conj_x: conj(x) in place of x
cudaError_t launch_weight(size_t n, const int nodes[3], int dim, const double2 *w_axis[3], int inverse,
                          const double2 *x, double2 *y, cudaStream_t s, int conj_x = 0);
// lambda = w y; grad_k2 = Re(lambda u), grad_f = conj(lambda) (either may be null)
cudaError_t launch_adjoint_grads(size_t n, const int nodes[3], int dim, const double2 *w_axis[3], const double2 *y,
                                 const double2 *u, double *grad_k2, double2 *grad_f, cudaStream_t s);
cudaError_t launch_grad_k2(size_t n, const int nodes[3], int dim, const double2 *lam, const double2 *u,
                           double *grad, cudaStream_t s);
