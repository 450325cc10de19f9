// Allocation-free variant of helm_mg_conv.
//
// helm_mg_conv creates its work vectors (a copy of b in FP64, the residual, the reduction
// partials) in the handle's Krylov workspace, which is allocated with cudaMalloc on first use.
// helm_mg_conv_noalloc runs the same cycles and the same residual-norm reduction kernels, but
// carves those work vectors out of one file-scope __device__ array, so it never allocates:
// not device memory, not pinned host memory (its scalar read-backs go to pageable memory).
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "helm_handle.h"

// Scratch shared by every call on a device; held by each GPU that loads the library until the
// process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device by the first call
// (with that device current) and kept for the life of the process.  In host code the symbol's
// name is only a host-side stand-in; a kernel may only be handed the looked-up address.  A
// cudaDeviceReset invalidates the kept address, as it does every handle's memory.
static void *g_scratch_addr[64];
static std::mutex g_scratch_mutex;

static helm_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return helm_fail(HELM_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return helm_fail(HELM_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HELM_OK;
}

#define CKR(...)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (__VA_ARGS__);                                                                   \
        if (e_ != cudaSuccess) return helm_fail(HELM_ERR_CUDA, "%s: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
    } while (0)

extern "C" helm_status helm_mg_conv_noalloc(helm_handle *h, const void *b, void *x, helm_prec prec, double tol,
                                            int maxcyc, int *ncycles, double *factor) {
    if (!h || !b || !x || !ncycles || !factor) return helm_fail(HELM_ERR_ARG, "null argument");
    if (h->mg.kind == HELM_PC_NONE) return helm_fail(HELM_ERR_ARG, "handle has no preconditioner hierarchy");
    if (prec != HELM_C128 && prec != HELM_C64) return helm_fail(HELM_ERR_ARG, "bad precision");
    if (maxcyc < 1 || !(tol > 0)) return helm_fail(HELM_ERR_ARG, "bad tol/maxcyc");
    const size_t np = h->np;
    const int nblk = blas_nblocks(np);
    // layout: b in FP64 | residual | reduction partials | one scalar, each 256-byte aligned
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t off_r = up(np * sizeof(double2));
    const size_t off_p = off_r + up(np * sizeof(double2));
    const size_t off_s = off_p + up((size_t)nblk * sizeof(double2));
    const size_t need = off_s + sizeof(double2);
    if (need > HELM_NOALLOC_SCRATCH_BYTES)
        return helm_fail(HELM_ERR_ARG, "grid of %zu nodes needs %zu bytes of scratch; the allocation-free entry point "
                         "holds %zu (at most about %zu nodes)", np, need, (size_t)HELM_NOALLOC_SCRATCH_BYTES,
                         (size_t)(HELM_NOALLOC_SCRATCH_BYTES / (2 * sizeof(double2))) - 1024);
    void *base = nullptr;
    helm_status st = scratch_address(&base);
    if (st != HELM_OK) return st;
    unsigned char *sc = (unsigned char *)base;
    double2 *b64 = (double2 *)sc, *r = (double2 *)(sc + off_r), *partials = (double2 *)(sc + off_p);
    double2 *scal = (double2 *)(sc + off_s);
    cudaStream_t s = h->stream;
    const size_t esz = prec == HELM_C128 ? sizeof(double2) : sizeof(float2);
    // the array keeps the previous call's contents: the residual's boundary nodes must be zero
    CKR(cudaMemsetAsync(r, 0, np * sizeof(double2), s));
    CKR(cudaMemsetAsync(x, 0, np * esz, s));
    if (prec == HELM_C64) CKR(launch_convert(np, (const float2 *)b, b64, s));
    else CKR(cudaMemcpyAsync(b64, b, np * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    auto norm = [&](const double2 *v, double *out) -> helm_status {
        CKR(launch_mdot_norm(np, nullptr, np, 0, v, partials, nullptr, s));
        CKR(launch_reduce(partials, nblk, 1, scal, 2, nullptr, s));
        double2 host;
        CKR(cudaMemcpyAsync(&host, scal, sizeof(double2), cudaMemcpyDeviceToHost, s));
        CKR(cudaStreamSynchronize(s));
        *out = host.x;
        return HELM_OK;
    };
    double bn = 0;
    if ((st = norm(b64, &bn)) != HELM_OK) return st;
    std::vector<double> res(1, bn);
    res.reserve((size_t)maxcyc + 1);
    int c = 0;
    while (c < maxcyc) {
        if ((st = mg_vcycle(h, b, x, prec)) != HELM_OK) return st;
        c++;
        if (prec == HELM_C64) {
            float2 *r32 = h->lv[0].t32;
            CKR(launch_residual<float, float2>(h->lv[0].M32, h->dim, (const float2 *)b, (const float2 *)x, r32, s));
            CKR(launch_convert(np, (const float2 *)r32, r, s));
        } else {
            CKR(launch_residual<double, double2>(h->lv[0].M64, h->dim, (const double2 *)b, (const double2 *)x, r, s));
        }
        double rn = 0;
        if ((st = norm(r, &rn)) != HELM_OK) return st;
        res.push_back(rn);
        if (!std::isfinite(rn)) return helm_fail(HELM_ERR_NONFINITE, "multigrid diverged to non-finite values");
        if (rn <= tol * bn) break;
    }
    const int k = std::min(c, 5);
    *ncycles = c;
    *factor = k > 0 && res[c - k] > 0 ? pow(res[c] / res[c - k], 1.0 / k) : 0.0;
    return HELM_OK;
}
