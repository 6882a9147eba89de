// mi_noalloc.cu -- hard-binned MI of one transform without allocating memory.
//
// Some callers cannot allocate device memory at the point where they need
// the metric: plug-ins living inside a framework whose caching allocator owns
// the GPU's memory (a cudaMalloc of their own fails once the pool holds it,
// or fragments it), services that budget their GPU memory up front and forbid
// allocations on the request path, and loops that cannot afford cudaMalloc's
// implicit device-wide synchronisation.  This file gives them mi_eval_noalloc:
// it uses the caller's device volumes in place and keeps every intermediate
// in one file-scope static device array of fixed size, which each GPU that
// loads the library holds until the process exits.  It calls no cudaMalloc,
// cudaFree or allocating library routine.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/mi.h"
#include "mi_internal.h"

namespace {

// Scratch layout: histogram (256 x 256 u32), then flags (2 int, padded to
// 256 bytes), then results (4 nq + 1 <= 33 doubles, padded).
constexpr size_t kHistBytes = (size_t)MI_NOALLOC_MAX_BINS * MI_NOALLOC_MAX_BINS * sizeof(uint32_t);
constexpr size_t kFlagsOffset = kHistBytes;
constexpr size_t kOutOffset = kHistBytes + 256;
constexpr size_t kScratchBytes = kOutOffset + 512;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

mi_status fail(mi_status st, const char *msg) {
    mi::set_thread_error(msg);
    return st;
}

mi_status fail_cuda(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return fail(MI_ECUDA, buf);
}

bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

mi_status check_volume(const mi_volume *v, const char *name, int dev, int *depth) {
    char buf[256];
    if (!v || !v->data) {
        snprintf(buf, sizeof buf, "%s volume or its data is NULL", name);
        return fail(MI_EINVAL, buf);
    }
    if (v->dtype != MI_U8 && v->dtype != MI_U16) {
        snprintf(buf, sizeof buf, "%s volume must be uint8 or uint16 for mi_eval_noalloc", name);
        return fail(MI_EUNSUPPORTED, buf);
    }
    for (int a = 0; a < 3; ++a) {
        if (v->dims[a] < 2 || !(v->spacing_mm[a] > 0.0f) || !isfinite(v->spacing_mm[a])) {
            snprintf(buf, sizeof buf, "%s volume dims must be >= 2 and spacings finite and > 0", name);
            return fail(MI_EINVAL, buf);
        }
    }
    const int full = v->dtype == MI_U8 ? 8 : 16;
    if (v->bit_depth < 0 || v->bit_depth > full) {
        snprintf(buf, sizeof buf, "%s volume bit_depth out of range", name);
        return fail(MI_EINVAL, buf);
    }
    *depth = v->bit_depth == 0 ? full : v->bit_depth;
    if (!on_device(v->data, dev)) {
        snprintf(buf, sizeof buf, "%s volume data must be device memory of the current device", name);
        return fail(MI_EINVAL, buf);
    }
    return MI_OK;
}

}  // namespace

extern "C" mi_status mi_eval_noalloc(const mi_volume *fixed, const mi_volume *moving, int bins,
                                     const float *transform, const float *q, int nq, double *out_mi, void *stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "no current CUDA device");
    if (dev < 0 || dev >= kMaxDevices) return fail(MI_EUNSUPPORTED, "device ordinal beyond 63");
    // ---- arguments ---------------------------------------------------------
    if (bins < MI_MIN_BINS || bins > MI_NOALLOC_MAX_BINS)
        return fail(MI_EINVAL, "mi_eval_noalloc: bins must be in 2..256 (the static scratch holds 256 x 256 counters)");
    int fdepth = 0, mdepth = 0;
    mi_status st;
    if ((st = check_volume(fixed, "fixed", dev, &fdepth)) != MI_OK) return st;
    if ((st = check_volume(moving, "moving", dev, &mdepth)) != MI_OK) return st;
    const long long nvf = (long long)fixed->dims[0] * fixed->dims[1] * fixed->dims[2];
    const long long nvm = (long long)moving->dims[0] * moving->dims[1] * moving->dims[2];
    if (nvf > MI_NOALLOC_MAX_VOXELS)
        return fail(MI_EINVAL, "mi_eval_noalloc: the fixed volume may hold at most 2^25 voxels "
                               "(the on-chip 16-bit counters drain into a table sized for that)");
    if (nvm > MI_NOALLOC_MAX_MOVING_VOXELS)
        return fail(MI_EINVAL, "mi_eval_noalloc: the moving volume must hold fewer than 2^31 voxels "
                               "(its neighbour offsets are 32-bit)");
    if (nq < 1 || nq > MI_MAX_Q || !q) return fail(MI_EINVAL, "nq must be in 1..8 and q non-NULL");
    if (!transform || !out_mi) return fail(MI_EINVAL, "transform and out_mi must be non-NULL");
    mi::QSet Q;
    memset(&Q, 0, sizeof Q);
    Q.nq = nq;
    Q.form = MI_TSALLIS_ADDITIVE;
    for (int i = 0; i < nq; ++i) {
        const float v = q[i];
        if (!(v > 0.0f) || !isfinite(v) || (v != 1.0f && fabsf(v - 1.0f) < 1e-6f))
            return fail(MI_EINVAL, "q values must be finite, > 0 and not within 1e-6 of 1 (use 1 for Shannon)");
        Q.q[i] = v;
    }
    for (int i = 0; i < 9; ++i)
        if (!isfinite(transform[i])) return fail(MI_EINVAL, "transform is not finite");
    int32_t q16[12];
    if (!mi::host_affine_q16(transform, fixed->dims, fixed->spacing_mm, moving->dims, moving->spacing_mm, q16))
        return fail(MI_ERANGE, "affine does not fit 16.16 fixed point");
    // ---- set-up, once per device (this device is current) ------------------
    unsigned char *scratch;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress of the static scratch");
            int n = 0;
            e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return fail_cuda(e, "reading the SM count");
            g_scratch_addr[dev] = (unsigned char *)p;
            g_sms[dev] = n;
        }
        scratch = g_scratch_addr[dev];
        sms = g_sms[dev];
    }
    // ---- work: the histogram and flags are cleared inside the launcher -----
    cudaStream_t s = (cudaStream_t)stream;
    const long long rows = (long long)fixed->dims[1] * fixed->dims[2];
    long long ctas = rows / (32 * 8);
    if (ctas > sms) ctas = sms;
    if (ctas < 1) ctas = 1;
    uint32_t *hist = (uint32_t *)scratch;
    int *flags = (int *)(scratch + kFlagsOffset);
    double *out = (double *)(scratch + kOutOffset);
    e = mi::launch_noalloc_eval(fixed->data, fixed->dtype, fdepth, moving->data, moving->dtype, mdepth, fixed->dims,
                                moving->dims, bins, q16, Q, hist, flags, out, (int)ctas, s);
    if (e != cudaSuccess) return fail_cuda(e, "mi_eval_noalloc kernels");
    int hflags[2] = {0, 0};
    if ((e = cudaMemcpyAsync(out_mi, out, (size_t)nq * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess)
        return fail_cuda(e, "copying results");
    if ((e = cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail_cuda(e, "reading flags");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail_cuda(e, "mi_eval_noalloc");
    if (hflags[1]) return fail(MI_ECUDA, "internal: 16-bit counter drain failed");
    if (hflags[0]) return fail(MI_EEMPTY, "the overlap is empty (MI is NaN)");
    return MI_OK;
}
