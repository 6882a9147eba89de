// mi_api.cu -- the C ABI of include/mi.h: contexts, validation, the
// parameter -> affine builder, path selection (plain / batched), CUDA-graph
// replay of the batched launch and the variant autotuner.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mi.h"
#include "mi_internal.h"

using namespace mi;

namespace {

thread_local std::string g_create_error;

// ---------------------------------------------------------------------------
// Device / pinned buffers
// ---------------------------------------------------------------------------

// mi_fault_alloc: successful device allocations left before a simulated failure (-1: disarmed).
std::atomic<int> g_fault_alloc{-1};

// True if this allocation is the one to fail (and disarms the hook).
bool fault_alloc_now() {
    int v = g_fault_alloc.load();
    while (v >= 0)
        if (g_fault_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(bytes, 256);
        if (fault_alloc_now()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    template <class T>
    T *as() const {
        return (T *)p;
    }
};

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(bytes, 256);
        cudaError_t e = cudaMallocHost(&p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    }
    template <class T>
    T *as() const {
        return (T *)p;
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// Parameters -> affine (FP64, order of operations fixed so the 16.16
// quantisation is reproducible; no fused multiply-add in this file's host code)
// ---------------------------------------------------------------------------

void mul3(const double x[9], const double y[9], double z[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc = acc + x[3 * r + k] * y[3 * k + c];
            z[3 * r + c] = acc;
        }
}

// Elementary rotation about `axis` by `rad`, or its derivative w.r.t. the angle.
void elem_rot(int axis, double rad, bool deriv, double m[9]) {
    const double c = cos(rad), s = sin(rad);
    for (int e = 0; e < 9; ++e) m[e] = 0.0;
    const int a = (axis + 1) % 3, b = (axis + 2) % 3;  // the rotated plane (a, b)
    if (!deriv) m[4 * axis] = 1.0;
    m[3 * a + a] = deriv ? -s : c;
    m[3 * a + b] = deriv ? -c : -s;
    m[3 * b + a] = deriv ? c : s;
    m[3 * b + b] = deriv ? -s : c;
}

const double kRadPerDeg = 3.14159265358979323846 / 180.0;

// Rotation of the unit quaternion (w, x, y, z) whose vector part is the parameter v; |v| >= 1 is
// first scaled onto the unit sphere (w = 0).  Expressions written in the order the quantised
// matrix depends on.  dR (optional, 3 x 9): dR/dv_p through w = sqrt(1 - |v|^2) inside the ball,
// through the normalisation v / |v| outside.
void versor_rotation(const double v[3], double R[9], double *dR) {
    double x = v[0], y = v[1], z = v[2];
    const double n2 = x * x + y * y + z * z;
    const bool on_sphere = n2 >= 1.0;
    const double len = on_sphere ? sqrt(n2) : 1.0;
    double w = 0.0;
    if (on_sphere) {
        x = x / len;
        y = y / len;
        z = z / len;
    } else {
        w = sqrt(1.0 - n2);
    }
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
    if (!dR) return;
    const double u[3] = {x, y, z};
    for (int p = 0; p < 3; ++p) {
        // the quaternion's change per unit change of v_p
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = on_sphere ? ((c == p ? 1.0 : 0.0) - u[c] * u[p]) / len : (c == p ? 1.0 : 0.0);
        const double dw = on_sphere ? 0.0 : -v[p] / w;
        double *g = dR + 9 * p;
        g[0] = -4.0 * (y * d[1] + z * d[2]);
        g[1] = 2.0 * (x * d[1] + y * d[0] - w * d[2] - z * dw);
        g[2] = 2.0 * (x * d[2] + z * d[0] + w * d[1] + y * dw);
        g[3] = 2.0 * (x * d[1] + y * d[0] + w * d[2] + z * dw);
        g[4] = -4.0 * (x * d[0] + z * d[2]);
        g[5] = 2.0 * (y * d[2] + z * d[1] - w * d[0] - x * dw);
        g[6] = 2.0 * (x * d[2] + z * d[0] - w * d[1] - y * dw);
        g[7] = 2.0 * (y * d[2] + z * d[1] + w * d[0] + x * dw);
        g[8] = -4.0 * (x * d[0] + y * d[1]);
    }
}

// [A | b] (row-major 3x4) for one transform, and optionally J = d[A|b]/dparam (12 x 9).
// rot: MI_ROT_EULER_DEG or MI_ROT_VERSOR; scale: MI_SCALE_FACTOR or MI_SCALE_OFFSET (sigma = 1 + s).
void build_affine(const float prm[9], const int nf[3], const float sfp[3], const int nm[3], const float smp[3],
                  double out[12], double *jac, int rot = MI_ROT_EULER_DEG, int scale = MI_SCALE_FACTOR) {
    double tr[3], rad[3], sc[3], sf[3], sm[3], cf[3], cm[3], vq[3];
    for (int a = 0; a < 3; ++a) {
        tr[a] = (double)prm[a];
        rad[a] = (double)prm[3 + a] * kRadPerDeg;
        vq[a] = (double)prm[3 + a];
        sc[a] = scale == MI_SCALE_OFFSET ? 1.0 + (double)prm[6 + a] : (double)prm[6 + a];
        sf[a] = (double)sfp[a];
        sm[a] = (double)smp[a];
        cf[a] = sf[a] * ((double)(nf[a] - 1) * 0.5);
        cm[a] = sm[a] * ((double)(nm[a] - 1) * 0.5);
    }
    double rx[9], ry[9], rz[9], rzy[9], R[9], dRv[27];
    if (rot == MI_ROT_VERSOR) {
        versor_rotation(vq, R, jac ? dRv : nullptr);
    } else {
        elem_rot(0, rad[0], false, rx);
        elem_rot(1, rad[1], false, ry);
        elem_rot(2, rad[2], false, rz);
        mul3(rz, ry, rzy);
        mul3(rzy, rx, R);
    }
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double rs = R[3 * a + c] * sc[c];
            out[4 * a + c] = (rs * sf[c]) / sm[a];
            acc = acc + rs * cf[c];
        }
        out[4 * a + 3] = ((cm[a] + tr[a]) - acc) / sm[a];
    }
    if (!jac) return;
    for (int e = 0; e < 108; ++e) jac[e] = 0.0;
    for (int a = 0; a < 3; ++a) jac[9 * (4 * a + 3) + a] = 1.0 / sm[a];
    for (int p = 0; p < 3; ++p) {
        double dx[9], dy[9], dz[9], t1[9], dR[9];
        double unit = kRadPerDeg;  // Euler angles are differentiated per degree
        if (rot == MI_ROT_VERSOR) {
            for (int e = 0; e < 9; ++e) dR[e] = dRv[9 * p + e];
            unit = 1.0;
        } else {
            elem_rot(0, rad[0], p == 0, dx);
            elem_rot(1, rad[1], p == 1, dy);
            elem_rot(2, rad[2], p == 2, dz);
            mul3(dz, dy, t1);
            mul3(t1, dx, dR);
        }
        for (int a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double d = dR[3 * a + c] * unit * sc[c];
                jac[9 * (4 * a + c) + 3 + p] = d * sf[c] / sm[a];
                acc += d * cf[c];
            }
            jac[9 * (4 * a + 3) + 3 + p] = -acc / sm[a];
        }
    }
    for (int p = 0; p < 3; ++p)
        for (int a = 0; a < 3; ++a) {
            jac[9 * (4 * a + p) + 6 + p] = R[3 * a + p] * sf[p] / sm[a];
            jac[9 * (4 * a + 3) + 6 + p] = -R[3 * a + p] * cf[p] / sm[a];
        }
}

// The general affine (12 parameters [M | t], row-major): R diag(sigma) of build_affine replaced by M, with the
// same order of operations.  J (12 x 12, optional) = d[A|b]/d[M|t] is constant.
void build_affine_matrix(const float prm[12], const int nf[3], const float sfp[3], const int nm[3],
                         const float smp[3], double out[12], double *jac) {
    double sf[3], sm[3], cf[3], cm[3];
    for (int a = 0; a < 3; ++a) {
        sf[a] = (double)sfp[a];
        sm[a] = (double)smp[a];
        cf[a] = sf[a] * ((double)(nf[a] - 1) * 0.5);
        cm[a] = sm[a] * ((double)(nm[a] - 1) * 0.5);
    }
    for (int a = 0; a < 3; ++a) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double m = (double)prm[4 * a + c];
            out[4 * a + c] = (m * sf[c]) / sm[a];
            acc = acc + m * cf[c];
        }
        out[4 * a + 3] = ((cm[a] + (double)prm[4 * a + 3]) - acc) / sm[a];
    }
    if (!jac) return;
    for (int e = 0; e < 144; ++e) jac[e] = 0.0;
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c) {
            jac[12 * (4 * a + c) + 4 * a + c] = sf[c] / sm[a];
            jac[12 * (4 * a + 3) + 4 * a + c] = -cf[c] / sm[a];
        }
        jac[12 * (4 * a + 3) + 4 * a + 3] = 1.0 / sm[a];
    }
}

// [A | b] of one transform in the context's conventions; jac (12 x nparams) optional.
void build_affine_opt(const mi_options &o, const float *prm, const int nf[3], const float sf[3], const int nm[3],
                      const float sm[3], double out[12], double *jac) {
    if (o.transform == MI_TRANSFORM_AFFINE)
        build_affine_matrix(prm, nf, sf, nm, sm, out, jac);
    else
        build_affine(prm, nf, sf, nm, sm, out, jac, o.rotation, o.scale);
}

bool quantise_q16(const double aff[12], int32_t q[12]) {
    for (int e = 0; e < 12; ++e) {
        const double s = aff[e] * 65536.0;
        if (!(fabs(s) <= 2147483647.0)) return false;
        const long long r = llround(s);
        if (r > 2147483647LL || r < -2147483647LL - 1) return false;
        q[e] = (int32_t)r;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

struct Pair {
    int nf[3], nm[3];
    float sf[3], sm[3];
    int bins;
    int fdepth, mdepth;
    int mdtype;  // stored moving type: 0 u8, 1 u16
    long long nvf, nvm;
    DevBuf fbins, mov, movp;    // hard path (movp: x-paired moving volume)
    cudaArray_t arr = nullptr;  // the pairs as a 3D array, read through tex
    cudaTextureObject_t tex = 0;
    cudaArray_t arrq = nullptr;  // 2 x 2 (y, z) quads as a 3D array, read through texq
    cudaTextureObject_t texq = 0;
    cudaArray_t arrg = nullptr;  // z-pair atlas (moving depth <= 12), read by 2D gathers through texg
    cudaTextureObject_t texg = 0;
    DevBuf zoff;                 // per moving plane: float2 atlas offset + 1 - 2^23
    DevBuf rowinfo;             // row-bound layout table (bins entries)
    DevBuf srow, scol, sbin;    // random sampling: per-row lists of the sampled fixed voxels
    int rows_words = 0;
    DevBuf pfbins, pmov, pmovx;  // Parzen path (pmovx: pmov extended by one plane per axis)
    cudaArray_t parr = nullptr;  // float4 quads of pmovx as a 3D array, read through ptex
    cudaTextureObject_t ptex = 0;
    ~Pair() {
        if (tex) cudaDestroyTextureObject(tex);
        if (arr) cudaFreeArray(arr);
        if (texq) cudaDestroyTextureObject(texq);
        if (arrq) cudaFreeArray(arrq);
        if (texg) cudaDestroyTextureObject(texg);
        if (arrg) cudaFreeArray(arrg);
        if (ptex) cudaDestroyTextureObject(ptex);
        if (parr) cudaFreeArray(parr);
    }
};

struct Choice {
    int variant = -1, threads = 0, ctas = 0;
    Tile tile{5, 4};  // lanes per row 2^5 (one row per warp step), 4 slabs per sweep
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    ~GraphEntry() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

}  // namespace

struct mi_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    mi_options opt;
    std::string err;
    std::vector<std::unique_ptr<Pair>> pairs;
    DevBuf d_pairs;     // PairDev[npairs]
    int max_bins = 0;
    int max_rows_words = 0;
    int max_zplanes = 0;      // moving planes of the largest pair (gather offsets in shared memory)
    bool all_gather = true;   // every pair has a z-pair atlas (gather variants allowed)
    // per-q FP64 tables, keyed by the float bits of q
    std::map<uint32_t, std::unique_ptr<DevBuf>> tables;
    // call scratch
    DevBuf d_aff, d_items, d_mi, d_h, d_cnt, d_hist, d_flags, d_ticket, d_dump, d_cols, d_part;
    HostBuf h_aff, h_items, h_out, h_read;
    // Parzen: the pairs' descriptors (device array), per-call pair indices and row offsets, scratch
    DevBuf p_pairs, p_pair_of, p_row_start;
    int p_bmax = 0, p_nxmax = 0;
    DevBuf p_aff, p_jac, p_hist, p_cnt, p_marg, p_ment, p_mterm, p_jsum, p_w, p_mom, p_grad;
    // autotune and graph caches
    std::map<std::tuple<int, int, int>, Choice> tuned;  // (path, pair-or--1, n bucket)
    std::map<std::string, std::unique_ptr<GraphEntry>> graphs;
    // profiling: events around the main kernels of the last call
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int last_launches = 0;
    bool timed = false;

    // floats per transform: 9 parameters, or the 12 of a general affine [M | t]
    int nparams() const { return opt.transform == MI_TRANSFORM_AFFINE ? 12 : 9; }

    mi_status fail(mi_status st, const std::string &msg) {
        err = msg;
        return st;
    }
    mi_status cuda_fail(cudaError_t e, const char *what) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? MI_ENOMEM : MI_ECUDA;
    }
};

namespace {

#define MI_CU(call, what)                                    \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return ctx->cuda_fail(e__, what); \
    } while (0)

// Per-call device guard: make the context's device current, restore on exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

mi_status validate_volume(const mi_volume *v, const char *name, bool parzen, std::string &err) {
    char buf[256];
    if (!v || !v->data) {
        snprintf(buf, sizeof buf, "%s volume or its data is NULL", name);
        err = buf;
        return MI_EINVAL;
    }
    if (v->dtype != MI_U8 && v->dtype != MI_U16 && v->dtype != MI_F32) {
        snprintf(buf, sizeof buf, "%s volume has unknown dtype %d", name, v->dtype);
        err = buf;
        return MI_EINVAL;
    }
    long long nv = 1;
    for (int a = 0; a < 3; ++a) {
        if (v->dims[a] < 2) {
            snprintf(buf, sizeof buf, "%s volume dims[%d] = %d (must be >= 2)", name, a, v->dims[a]);
            err = buf;
            return MI_EINVAL;
        }
        nv *= v->dims[a];
        if (!(v->spacing_mm[a] > 0.0f) || !isfinite(v->spacing_mm[a])) {
            snprintf(buf, sizeof buf, "%s volume spacing_mm[%d] must be finite and > 0", name, a);
            err = buf;
            return MI_EINVAL;
        }
    }
    if (nv >= (1LL << 31)) {
        snprintf(buf, sizeof buf, "%s volume has %lld voxels (limit 2^31 - 1)", name, nv);
        err = buf;
        return MI_EINVAL;
    }
    const int maxd = v->dtype == MI_U8 ? 8 : 16;
    if (v->dtype != MI_F32 && (v->bit_depth < 0 || v->bit_depth > maxd)) {
        snprintf(buf, sizeof buf, "%s volume bit_depth %d out of range 0..%d", name, v->bit_depth, maxd);
        err = buf;
        return MI_EINVAL;
    }
    (void)parzen;
    return MI_OK;
}

int effective_depth(const mi_volume *v) {
    if (v->dtype == MI_F32) return 16;
    const int full = v->dtype == MI_U8 ? 8 : 16;
    return v->bit_depth == 0 ? full : v->bit_depth;
}

size_t dtype_size(int dt) { return dt == MI_U8 ? 1 : (dt == MI_U16 ? 2 : 4); }

// Copy a caller volume (host or device) into a fresh device buffer.
mi_status upload_volume(mi_ctx *ctx, const mi_volume *v, DevBuf &dst) {
    const size_t bytes = (size_t)v->dims[0] * v->dims[1] * v->dims[2] * dtype_size(v->dtype);
    MI_CU(dst.ensure(bytes), "allocating a volume");
    MI_CU(cudaMemcpyAsync(dst.p, v->data, bytes, is_device_ptr(v->data) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          ctx->stream),
          "copying a volume to the device");
    return MI_OK;
}

// Random sampling (mi_options.sample_fraction in (0, 1)): per fixed row, the x indices and fixed
// bins (fb: the hard or the Parzen bins) of its sampled voxels, as row offsets + lists.
mi_status build_samples(mi_ctx *ctx, Pair &P, const uint8_t *fb, cudaStream_t s) {
    const double frac = (double)ctx->opt.sample_fraction;
    if (!(frac > 0.0 && frac < 1.0)) return MI_OK;
    if (P.nf[0] > 65536) return ctx->fail(MI_EUNSUPPORTED, "random sampling needs fixed rows of at most 65536 voxels");
    const uint32_t thr = (uint32_t)floor(frac * 4294967296.0);
    const long long R = (long long)P.nf[1] * P.nf[2];
    DevBuf dcnt;
    MI_CU(dcnt.ensure((size_t)R * 4), "allocating sample counts");
    MI_CU(launch_sample_count(P.nf[0], R, ctx->opt.sample_seed, thr, dcnt.as<uint32_t>(), s), "sample counts");
    std::vector<uint32_t> cnt((size_t)R), ptr((size_t)R + 1);
    MI_CU(cudaMemcpyAsync(cnt.data(), dcnt.p, (size_t)R * 4, cudaMemcpyDeviceToHost, s), "sample counts D2H");
    MI_CU(cudaStreamSynchronize(s), "sample counts");
    unsigned long long acc = 0;
    for (long long r = 0; r < R; ++r) {
        ptr[(size_t)r] = (uint32_t)acc;
        acc += cnt[(size_t)r];
    }
    ptr[(size_t)R] = (uint32_t)acc;
    MI_CU(P.srow.ensure(((size_t)R + 1) * 4), "allocating sample rows");
    MI_CU(P.scol.ensure(std::max<size_t>((size_t)acc * 2, 2)), "allocating sample columns");
    MI_CU(P.sbin.ensure(std::max<size_t>((size_t)acc, 1)), "allocating sample bins");
    MI_CU(cudaMemcpyAsync(P.srow.p, ptr.data(), ((size_t)R + 1) * 4, cudaMemcpyHostToDevice, s), "sample rows");
    MI_CU(launch_sample_fill(P.nf[0], R, ctx->opt.sample_seed, thr, fb, P.srow.as<uint32_t>(), P.scol.as<uint16_t>(),
                             P.sbin.as<uint8_t>(), s),
          "sample lists");
    MI_CU(cudaStreamSynchronize(s), "sample lists");
    return MI_OK;
}

mi_status add_pair(mi_ctx *ctx, const mi_volume *fx, const mi_volume *mv, int bins) {
    std::string e;
    const bool parzen = ctx->opt.kernel == MI_PARZEN;
    mi_status st;
    if ((st = validate_volume(fx, "fixed", parzen, e)) != MI_OK) return ctx->fail(st, e);
    if ((st = validate_volume(mv, "moving", parzen, e)) != MI_OK) return ctx->fail(st, e);
    {
        // both paths gather the moving volume through 3D textures of its dims (nx, ny, nz)
        int tw = 0, th = 0, td = 0;
        cudaDeviceGetAttribute(&tw, cudaDevAttrMaxTexture3DWidth, ctx->device);
        cudaDeviceGetAttribute(&th, cudaDevAttrMaxTexture3DHeight, ctx->device);
        cudaDeviceGetAttribute(&td, cudaDevAttrMaxTexture3DDepth, ctx->device);
        if (mv->dims[0] > tw || mv->dims[1] > th || mv->dims[2] > td)
            return ctx->fail(MI_EUNSUPPORTED, "moving volume dims exceed the device's 3D texture extent (" +
                                                  std::to_string(tw) + " x " + std::to_string(th) + " x " +
                                                  std::to_string(td) + ")");
    }
    if (parzen) {
        if (bins < MI_MIN_PARZEN_BINS || bins > 128)
            return ctx->fail(MI_EINVAL, "Parzen bins must be in " + std::to_string(MI_MIN_PARZEN_BINS) + "..128");
        if (fx->dims[0] > MI_MAX_PARZEN_NX)
            return ctx->fail(MI_EUNSUPPORTED, "Parzen fixed rows are limited to " + std::to_string(MI_MAX_PARZEN_NX) +
                                                  " voxels (nx)");
        // the moving volume extended by one plane per axis is indexed with 32-bit offsets
        if ((long long)(mv->dims[0] + 1) * (mv->dims[1] + 1) * (mv->dims[2] + 1) >= (1LL << 31))
            return ctx->fail(MI_EUNSUPPORTED, "the Parzen moving volume is limited to (nx+1)(ny+1)(nz+1) < 2^31");
    } else if (bins < MI_MIN_BINS || bins > MI_MAX_BINS) {
        return ctx->fail(MI_EINVAL, "bins must be in 2..256, got " + std::to_string(bins));
    }
    auto P = std::make_unique<Pair>();
    for (int a = 0; a < 3; ++a) {
        P->nf[a] = fx->dims[a];
        P->nm[a] = mv->dims[a];
        P->sf[a] = fx->spacing_mm[a];
        P->sm[a] = mv->spacing_mm[a];
    }
    P->bins = bins;
    P->fdepth = effective_depth(fx);
    P->mdepth = effective_depth(mv);
    P->nvf = (long long)P->nf[0] * P->nf[1] * P->nf[2];
    P->nvm = (long long)P->nm[0] * P->nm[1] * P->nm[2];
    cudaStream_t s = ctx->stream;
    DevBuf rawf, rawm;
    if ((st = upload_volume(ctx, fx, rawf)) != MI_OK) return st;
    if ((st = upload_volume(ctx, mv, rawm)) != MI_OK) return st;
    if (parzen) {
        MI_CU(P->pfbins.ensure((size_t)P->nvf), "allocating Parzen fixed bins");
        MI_CU(launch_parzen_prep_fixed(rawf.p, fx->dtype, P->fdepth, P->nvf, bins, P->pfbins.as<uint8_t>(), s),
              "Parzen fixed bins");
        MI_CU(P->pmov.ensure((size_t)P->nvm * 4), "allocating the normalised moving volume");
        MI_CU(launch_parzen_prep_moving(rawm.p, mv->dtype, P->mdepth, P->nvm, P->pmov.as<float>(), s),
              "normalising the moving volume");
        MI_CU(P->pmovx.ensure((size_t)(P->nm[0] + 1) * (P->nm[1] + 1) * (P->nm[2] + 1) * 4),
              "allocating the extended moving volume");
        MI_CU(launch_parzen_extend(P->pmov.as<float>(), P->nm, P->pmovx.as<float>(), s), "extending the moving volume");
        if ((st = build_samples(ctx, *P, P->pfbins.as<uint8_t>(), s)) != MI_OK) return st;
        {
            const cudaExtent ext = make_cudaExtent(P->nm[0], P->nm[1], P->nm[2]);  // (y, z) quads
            DevBuf quads;
            MI_CU(quads.ensure(ext.width * ext.height * ext.depth * 16), "allocating the Parzen quads");
            MI_CU(launch_parzen_quads(P->pmovx.as<float>(), P->nm, quads.p, s), "building the Parzen quads");
            cudaChannelFormatDesc cd = cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindFloat);
            MI_CU(cudaMalloc3DArray(&P->parr, &cd, ext), "allocating the Parzen quad array");
            cudaMemcpy3DParms cp;
            memset(&cp, 0, sizeof cp);
            cp.srcPtr = make_cudaPitchedPtr(quads.p, ext.width * 16, ext.width, ext.height);
            cp.dstArray = P->parr;
            cp.extent = ext;
            cp.kind = cudaMemcpyDeviceToDevice;
            MI_CU(cudaMemcpy3DAsync(&cp, s), "filling the Parzen quad array");
            cudaResourceDesc rd;
            memset(&rd, 0, sizeof rd);
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = P->parr;
            cudaTextureDesc td;
            memset(&td, 0, sizeof td);
            td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            MI_CU(cudaCreateTextureObject(&P->ptex, &rd, &td, nullptr), "creating the Parzen quad texture");
            MI_CU(cudaStreamSynchronize(s), "building the Parzen quads");
        }
        P->mdtype = 1;
    } else {
        // fixed: float -> 16-bit first, then bins
        int fdt = fx->dtype;
        const void *fsrc = rawf.p;
        DevBuf conv;
        if (fdt == MI_F32) {
            MI_CU(conv.ensure((size_t)P->nvf * 2), "allocating a conversion buffer");
            MI_CU(launch_f32_to_u16(rawf.as<float>(), P->nvf, conv.as<uint16_t>(), s), "converting the fixed volume");
            fsrc = conv.p;
            fdt = MI_U16;
        }
        MI_CU(P->fbins.ensure((size_t)P->nvf), "allocating fixed bins");
        MI_CU(launch_bin_fixed(fsrc, fdt, P->fdepth, P->nvf, bins, P->fbins.as<uint8_t>(), s), "binning the fixed volume");
        // row-bound layout: a row whose bin holds at most 65535 fixed voxels can never count past 16 bits
        {
            DevBuf dF;
            std::vector<unsigned long long> F(bins);
            MI_CU(dF.ensure((size_t)bins * 8), "allocating bin counts");
            MI_CU(launch_fixed_hist(P->fbins.as<uint8_t>(), P->nvf, bins, dF.as<unsigned long long>(), s), "bin counts");
            MI_CU(cudaMemcpyAsync(F.data(), dF.p, (size_t)bins * 8, cudaMemcpyDeviceToHost, s), "bin counts D2H");
            MI_CU(cudaStreamSynchronize(s), "bin counts");
            std::vector<uint32_t> info(bins);
            const uint32_t S = (uint32_t)bins + 1;
            uint32_t off = 0;
            for (int r = 0; r < bins; ++r)
                if (F[r] > 65535) {
                    info[r] = off << 6 | 32u;
                    off += S;
                }
            int k = 0;
            for (int r = 0; r < bins; ++r)
                if (F[r] <= 65535) {
                    info[r] = (off + (uint32_t)(k / 2) * S) << 6 | (uint32_t)(k % 2 ? 16 : 0);
                    ++k;
                }
            off += (uint32_t)((k + 1) / 2) * S;
            P->rows_words = (int)off;
            MI_CU(P->rowinfo.ensure((size_t)bins * 4), "allocating the row table");
            MI_CU(cudaMemcpyAsync(P->rowinfo.p, info.data(), (size_t)bins * 4, cudaMemcpyHostToDevice, s), "row table");
            MI_CU(cudaStreamSynchronize(s), "row table");
        }
        if ((st = build_samples(ctx, *P, P->fbins.as<uint8_t>(), s)) != MI_OK) return st;
        if (mv->dtype == MI_F32) {
            MI_CU(P->mov.ensure((size_t)P->nvm * 2), "allocating the moving volume");
            MI_CU(launch_f32_to_u16(rawm.as<float>(), P->nvm, P->mov.as<uint16_t>(), s), "converting the moving volume");
            P->mdtype = 1;
        } else {
            MI_CU(P->mov.ensure((size_t)P->nvm * dtype_size(mv->dtype)), "allocating the moving volume");
            MI_CU(cudaMemcpyAsync(P->mov.p, rawm.p, (size_t)P->nvm * dtype_size(mv->dtype), cudaMemcpyDeviceToDevice, s),
                  "copying the moving volume");
            P->mdtype = mv->dtype == MI_U8 ? 0 : 1;
            MI_CU(launch_clamp_depth(P->mov.p, P->mdtype, P->mdepth, P->nvm, s), "clamping the moving volume");
        }
        const size_t npairs = (size_t)P->nm[0] * (P->nm[1] + 1) * (P->nm[2] + 1);
        MI_CU(P->movp.ensure(npairs * (P->mdtype == 0 ? 2 : 4)), "allocating the paired moving volume");
        MI_CU(launch_make_pairs(P->mov.p, P->mdtype, P->nm, P->movp.p, s), "pairing the moving volume");
        // the same pairs (without the padding row / plane) as a 3D array for the texture path
        const size_t esz = P->mdtype == 0 ? 2 : 4;
        cudaChannelFormatDesc cd = cudaCreateChannelDesc((int)esz * 8, 0, 0, 0, cudaChannelFormatKindUnsigned);
        MI_CU(cudaMalloc3DArray(&P->arr, &cd, make_cudaExtent(P->nm[0], P->nm[1], P->nm[2])), "allocating the 3D array");
        cudaMemcpy3DParms cp;
        memset(&cp, 0, sizeof cp);
        cp.srcPtr = make_cudaPitchedPtr(P->movp.p, (size_t)P->nm[0] * esz, P->nm[0], P->nm[1] + 1);
        cp.dstArray = P->arr;
        cp.extent = make_cudaExtent(P->nm[0], P->nm[1], P->nm[2]);
        cp.kind = cudaMemcpyDeviceToDevice;
        MI_CU(cudaMemcpy3DAsync(&cp, s), "filling the 3D array");
        cudaResourceDesc rd;
        memset(&rd, 0, sizeof rd);
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = P->arr;
        cudaTextureDesc td;
        memset(&td, 0, sizeof td);
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        MI_CU(cudaCreateTextureObject(&P->tex, &rd, &td, nullptr), "creating the texture object");
        // 2 x 2 (y, z) quads (uchar4 / ushort4), read at integer texel coordinates
        {
            const int cb = P->mdtype == 0 ? 8 : 16;
            const size_t qsz = (size_t)cb / 2;  // bytes per quad
            const cudaExtent qext = make_cudaExtent(P->nm[0], P->nm[1], P->nm[2]);
            DevBuf quads;
            MI_CU(quads.ensure(qext.width * qext.height * qext.depth * qsz), "allocating the quads");
            MI_CU(launch_make_quads(P->mov.p, P->mdtype, P->nm, quads.p, s), "building the quads");
            cudaChannelFormatDesc cq = cudaCreateChannelDesc(cb, cb, cb, cb, cudaChannelFormatKindUnsigned);
            MI_CU(cudaMalloc3DArray(&P->arrq, &cq, qext), "allocating the quad array");
            cudaMemcpy3DParms cq3;
            memset(&cq3, 0, sizeof cq3);
            cq3.srcPtr = make_cudaPitchedPtr(quads.p, qext.width * qsz, qext.width, qext.height);
            cq3.dstArray = P->arrq;
            cq3.extent = qext;
            cq3.kind = cudaMemcpyDeviceToDevice;
            MI_CU(cudaMemcpy3DAsync(&cq3, s), "filling the quad array");
            rd.res.array.array = P->arrq;
            MI_CU(cudaCreateTextureObject(&P->texq, &rd, &td, nullptr), "creating the quad texture object");
            MI_CU(cudaStreamSynchronize(s), "building the quads");
        }
        // z-pair atlas for moving depths <= 12: plane z is the tile at ((z / ph) nx, (z % ph) ny) of a 2D
        // image no larger than the device's gather extent; a gather at (ix + 1 + ox, iy + 1 + oy) returns
        // the plane's 2 x 2 footprint with each texel's z + 1 neighbour packed beside it
        if (P->mdepth <= 12) {
            int gw = 0, gh = 0;
            cudaDeviceGetAttribute(&gw, cudaDevAttrMaxTexture2DGatherWidth, ctx->device);
            cudaDeviceGetAttribute(&gh, cudaDevAttrMaxTexture2DGatherHeight, ctx->device);
            const int nx = P->nm[0], ny = P->nm[1], nz = P->nm[2];
            const int ph = std::min(nz, gh / ny);
            const int cols = ph > 0 ? (nz + ph - 1) / ph : 0;
            if (ph > 0 && (long long)cols * nx <= gw) {
                const int W = cols * nx, H = ph * ny;
                DevBuf img;
                MI_CU(img.ensure((size_t)W * H * 4), "allocating the z-pair atlas");
                MI_CU(launch_make_zpairs(P->mov.p, P->mdtype, P->nm, ph, W, H, img.as<uint32_t>(), s),
                      "building the z-pair atlas");
                cudaChannelFormatDesc cg = cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindUnsigned);
                MI_CU(cudaMallocArray(&P->arrg, &cg, W, H, cudaArrayTextureGather), "allocating the z-pair array");
                MI_CU(cudaMemcpy2DToArrayAsync(P->arrg, 0, 0, img.p, (size_t)W * 4, (size_t)W * 4, H,
                                               cudaMemcpyDeviceToDevice, s),
                      "filling the z-pair array");
                rd.res.array.array = P->arrg;
                MI_CU(cudaCreateTextureObject(&P->texg, &rd, &td, nullptr), "creating the z-pair texture object");
                std::vector<float2> off(nz);
                for (int z = 0; z < nz; ++z) {
                    off[z].x = (float)((z / ph) * nx + 1) - 8388608.0f;
                    off[z].y = (float)((z % ph) * ny + 1) - 8388608.0f;
                }
                MI_CU(P->zoff.ensure((size_t)nz * sizeof(float2)), "allocating the plane offsets");
                MI_CU(cudaMemcpyAsync(P->zoff.p, off.data(), (size_t)nz * sizeof(float2), cudaMemcpyHostToDevice, s),
                      "plane offsets");
                MI_CU(cudaStreamSynchronize(s), "building the z-pair atlas");
            }
        }
    }
    MI_CU(cudaStreamSynchronize(s), "preparing the volumes");
    ctx->max_bins = std::max(ctx->max_bins, bins);
    ctx->max_rows_words = std::max(ctx->max_rows_words, P->rows_words);
    ctx->max_zplanes = std::max(ctx->max_zplanes, P->nm[2]);
    if (!P->texg) ctx->all_gather = false;
    ctx->pairs.push_back(std::move(P));
    return MI_OK;
}

mi_status upload_pairs(mi_ctx *ctx) {
    std::vector<PairDev> pd(ctx->pairs.size());
    for (size_t i = 0; i < ctx->pairs.size(); ++i) {
        const Pair &P = *ctx->pairs[i];
        PairDev &d = pd[i];
        memset(&d, 0, sizeof d);
        d.fbins = P.fbins.as<uint8_t>();
        d.mov = P.mov.p;
        d.movp = P.movp.p;
        d.texp = P.tex;
        d.texq = P.texq;
        d.texg = P.texg;
        d.zoff = P.zoff.as<float2>();
        d.rowinfo = P.rowinfo.as<uint32_t>();
        d.srow = P.srow.p ? P.srow.as<uint32_t>() : nullptr;
        d.scol = P.scol.as<uint16_t>();
        d.sbin = P.sbin.as<uint8_t>();
        d.rows_words = P.rows_words;
        for (int a = 0; a < 3; ++a) {
            d.nf[a] = P.nf[a];
            d.nm[a] = P.nm[a];
        }
        d.bins = P.bins;
        d.mdepth = P.mdepth;
        d.mdtype = P.mdtype;
    }
    MI_CU(ctx->d_pairs.ensure(pd.size() * sizeof(PairDev)), "allocating pair descriptors");
    MI_CU(cudaMemcpyAsync(ctx->d_pairs.p, pd.data(), pd.size() * sizeof(PairDev), cudaMemcpyHostToDevice, ctx->stream),
          "uploading pair descriptors");
    MI_CU(cudaStreamSynchronize(ctx->stream), "uploading pair descriptors");
    return MI_OK;
}

// The Parzen kernels' view of one pair.
ParzenPair parzen_pair(const mi_ctx *ctx, const Pair &P) {
    ParzenPair pp;
    memset(&pp, 0, sizeof pp);
    pp.fbins = P.pfbins.as<uint8_t>();
    pp.mov = P.pmov.as<float>();
    pp.movx = P.pmovx.as<float>();
    pp.texq = P.ptex;
    pp.srow = P.srow.p ? P.srow.as<uint32_t>() : nullptr;
    pp.scol = P.scol.as<uint16_t>();
    pp.sbin = P.sbin.as<uint8_t>();
    for (int a = 0; a < 3; ++a) {
        pp.nf[a] = P.nf[a];
        pp.nm[a] = P.nm[a];
    }
    pp.B = P.bins;
    (void)ctx;
    return pp;
}

mi_status upload_parzen_pairs(mi_ctx *ctx) {
    std::vector<ParzenPair> pd;
    for (auto &p : ctx->pairs) {
        pd.push_back(parzen_pair(ctx, *p));
        ctx->p_bmax = std::max(ctx->p_bmax, p->bins);
        ctx->p_nxmax = std::max(ctx->p_nxmax, p->nf[0]);
    }
    MI_CU(ctx->p_pairs.ensure(pd.size() * sizeof(ParzenPair)), "allocating Parzen pair descriptors");
    MI_CU(cudaMemcpyAsync(ctx->p_pairs.p, pd.data(), pd.size() * sizeof(ParzenPair), cudaMemcpyHostToDevice, ctx->stream),
          "uploading Parzen pair descriptors");
    MI_CU(cudaStreamSynchronize(ctx->stream), "uploading Parzen pair descriptors");
    return MI_OK;
}

PairDev host_pairdev(const Pair &P) {
    PairDev d;
    memset(&d, 0, sizeof d);
    d.fbins = P.fbins.as<uint8_t>();
    d.mov = P.mov.p;
    d.movp = P.movp.p;
    d.texp = P.tex;
    d.texq = P.texq;
    d.texg = P.texg;
    d.zoff = P.zoff.as<float2>();
    d.rowinfo = P.rowinfo.as<uint32_t>();
    d.srow = P.srow.p ? P.srow.as<uint32_t>() : nullptr;
    d.scol = P.scol.as<uint16_t>();
    d.sbin = P.sbin.as<uint8_t>();
    d.rows_words = P.rows_words;
    for (int a = 0; a < 3; ++a) {
        d.nf[a] = P.nf[a];
        d.nm[a] = P.nm[a];
    }
    d.bins = P.bins;
    d.mdepth = P.mdepth;
    d.mdtype = P.mdtype;
    return d;
}

mi_status create_common(mi_ctx **out, const mi_volume *fixed, const mi_volume *moving, const int *bins, int npairs,
                        const mi_options *opt) {
    if (!out) {
        g_create_error = "out is NULL";
        return MI_EINVAL;
    }
    *out = nullptr;
    auto ctx = std::make_unique<mi_ctx>();
    if (opt)
        ctx->opt = *opt;
    else
        mi_options_default(&ctx->opt);
    if (npairs < 1 || !fixed || !moving || !bins) {
        g_create_error = "need at least one (fixed, moving, bins) pair";
        return MI_EINVAL;
    }
    if (ctx->opt.kernel != MI_HARD && ctx->opt.kernel != MI_PARZEN) {
        g_create_error = "opt.kernel must be MI_HARD or MI_PARZEN";
        return MI_EINVAL;
    }
    if (!(ctx->opt.sample_fraction >= 0.0f && ctx->opt.sample_fraction <= 1.0f)) {
        g_create_error = "opt.sample_fraction must lie in [0, 1]";
        return MI_EINVAL;
    }
    if ((ctx->opt.rotation != MI_ROT_EULER_DEG && ctx->opt.rotation != MI_ROT_VERSOR) ||
        (ctx->opt.scale != MI_SCALE_FACTOR && ctx->opt.scale != MI_SCALE_OFFSET)) {
        g_create_error = "opt.rotation / opt.scale out of range";
        return MI_EINVAL;
    }
    if (ctx->opt.transform != MI_TRANSFORM_PARAMS && ctx->opt.transform != MI_TRANSFORM_AFFINE) {
        g_create_error = "opt.transform must be MI_TRANSFORM_PARAMS or MI_TRANSFORM_AFFINE";
        return MI_EINVAL;
    }
    if (ctx->opt.hist_variant < MI_HV_AUTO || ctx->opt.hist_variant > MI_HV_U16_GATHER) {
        g_create_error = "opt.hist_variant out of range";
        return MI_EINVAL;
    }
    if (ctx->opt.block_threads != 0 && ctx->opt.block_threads != 512 && ctx->opt.block_threads != 1024) {
        g_create_error = "opt.block_threads must be 0, 512 or 1024";
        return MI_EINVAL;
    }
    if (ctx->opt.tile_rows != 0 && ctx->opt.tile_rows != 1 && ctx->opt.tile_rows != 2 && ctx->opt.tile_rows != 4 &&
        ctx->opt.tile_rows != 32) {
        g_create_error = "opt.tile_rows must be 0, 1, 2, 4 or 32";
        return MI_EINVAL;
    }
    if (ctx->opt.tile_slabs < 0 || ctx->opt.tile_slabs > kMaxSlabs) {
        g_create_error = "opt.tile_slabs must be in 0..16";
        return MI_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return MI_ECUDA;
    }
    int dev = ctx->opt.device;
    if (dev < 0) cudaGetDevice(&dev);
    if (dev >= ndev) {
        g_create_error = "opt.device out of range";
        return MI_EINVAL;
    }
    ctx->device = dev;
    DeviceGuard guard(dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        g_create_error = std::string("creating a stream: ") + cudaGetErrorString(e);
        return MI_ECUDA;
    }
    ctx->stream = ctx->own_stream;
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "creating events";
        return MI_ECUDA;
    }
    for (int p = 0; p < npairs; ++p) {
        mi_status st = add_pair(ctx.get(), &fixed[p], &moving[p], bins[p]);
        if (st != MI_OK) {
            g_create_error = "pair " + std::to_string(p) + ": " + ctx->err;
            return st;
        }
    }
    if (ctx->opt.kernel == MI_PARZEN) {
        mi_status st = upload_parzen_pairs(ctx.get());
        if (st != MI_OK) {
            g_create_error = ctx->err;
            return st;
        }
    }
    if (ctx->opt.kernel == MI_HARD) {
        mi_status st = upload_pairs(ctx.get());
        if (st != MI_OK) {
            g_create_error = ctx->err;
            return st;
        }
        MI_CU(ctx->d_flags.ensure(2 * sizeof(int)), "allocating flags");
        MI_CU(ctx->d_ticket.ensure(2 * sizeof(int)), "allocating the ticket");  // ticket, sweep phase
    }
    *out = ctx.release();
    return MI_OK;
}

// ---------------------------------------------------------------------------
// q sets and tables
// ---------------------------------------------------------------------------

uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

// Reads `bytes` of caller device memory into host memory in the context's stream order: an
// asynchronous copy into pinned staging, then a wait on that stream alone (no legacy-stream copy).
mi_status read_from_device(mi_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return MI_OK;
    MI_CU(ctx->h_read.ensure(bytes), "pinned staging");
    MI_CU(cudaMemcpyAsync(ctx->h_read.p, src, bytes, cudaMemcpyDeviceToHost, ctx->stream), "reading device input");
    MI_CU(cudaStreamSynchronize(ctx->stream), "reading device input");
    memcpy(dst, ctx->h_read.p, bytes);
    return MI_OK;
}

mi_status read_q(mi_ctx *ctx, const float *q, int nq, float out[kMaxQ]) {
    if (nq < 1 || nq > kMaxQ) return ctx->fail(MI_EINVAL, "nq must be in 1..8");
    if (!q) return ctx->fail(MI_EINVAL, "q is NULL");
    if (is_device_ptr(q)) {
        mi_status st = read_from_device(ctx, out, q, nq * sizeof(float));
        if (st != MI_OK) return st;
    } else {
        memcpy(out, q, nq * sizeof(float));
    }
    for (int i = 0; i < nq; ++i) {
        const float v = out[i];
        if (!(v > 0.0f) || !isfinite(v)) return ctx->fail(MI_EINVAL, "q values must be finite and > 0");
        if (v != 1.0f && fabsf(v - 1.0f) < 1e-6f)
            return ctx->fail(MI_EINVAL, "q within 1e-6 of 1 is ill-conditioned; use q = 1 for Shannon");
    }
    return MI_OK;
}

mi_status make_qset(mi_ctx *ctx, const float *qv, int nq, QSet &Q) {
    memset(&Q, 0, sizeof Q);
    Q.nq = nq;
    Q.form = ctx->opt.tsallis_form;
    Q.bits = ctx->opt.log_bits ? 1 : 0;
    for (int i = 0; i < nq; ++i) {
        Q.q[i] = qv[i];
        if (ctx->opt.kernel == MI_HARD) {
            auto it = ctx->tables.find(fbits(qv[i]));
            if (it == ctx->tables.end()) {
                auto buf = std::make_unique<DevBuf>();
                MI_CU(buf->ensure(sizeof(double) * kTab), "allocating an entropy table");
                MI_CU(launch_table(buf->as<double>(), qv[i], ctx->stream), "building an entropy table");
                it = ctx->tables.emplace(fbits(qv[i]), std::move(buf)).first;
            }
            Q.tab[i] = it->second->as<double>();
        }
    }
    return MI_OK;
}

// Transforms from the caller (host or device) into a host vector.
mi_status read_transforms(mi_ctx *ctx, const float *tr, int n, std::vector<float> &out) {
    const int np = ctx->nparams();
    out.resize((size_t)n * np);
    if (n == 0) return MI_OK;
    if (!tr) return ctx->fail(MI_EINVAL, "transforms is NULL");
    if (is_device_ptr(tr)) {
        mi_status st = read_from_device(ctx, out.data(), tr, (size_t)n * np * sizeof(float));
        if (st != MI_OK) return st;
    } else {
        memcpy(out.data(), tr, (size_t)n * np * sizeof(float));
    }
    for (size_t i = 0; i < out.size(); ++i)
        if (!isfinite(out[i])) return ctx->fail(MI_EINVAL, "transform " + std::to_string(i / np) + " is not finite");
    return MI_OK;
}

mi_status build_q16(mi_ctx *ctx, const Pair &P, const float *prm, int32_t *q16, int t) {
    double aff[12];
    build_affine_opt(ctx->opt, prm, P.nf, P.sf, P.nm, P.sm, aff, nullptr);
    if (!quantise_q16(aff, q16))
        return ctx->fail(MI_ERANGE, "transform " + std::to_string(t) + ": affine does not fit 16.16 fixed point");
    return MI_OK;
}

// Copy n*each bytes of an internal device result to the caller's pointer (host or device).
mi_status deliver(mi_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (!dst || bytes == 0) return MI_OK;
    MI_CU(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream),
          "copying results");
    return MI_OK;
}

// ---------------------------------------------------------------------------
// Variant selection
// ---------------------------------------------------------------------------

bool variant_fits(int variant, int bins, int threads, long long nvox, int rows_words, int zmax) {
    const int kind = hv_kind(variant);
    const bool u16 = kind == HV_U16 || kind == HV_U16_MATCH;
    if (u16 && nvox > (long long)(kOvfSlots / 2) * kDrainT) return false;
    return hard_smem_bytes(variant, bins, threads, rows_words, zmax) <= 227 * 1024;
}

// Walks the tile shape may take for a variant: quad and gather fetches walk the warp's 32 rows as one
// voxel stream (lpr_log2 0) or 1, 2 or 4 rows per step (lanes per row 2^5, 2^4, 2^3); the others one
// row at a time.
std::vector<int> tile_lpr(mi_ctx *ctx, int variant) {
    if (hv_fetch(variant) < FM_QUAD) return {5};
    switch (ctx->opt.tile_rows) {
        case 1: return {5};
        case 2: return {4};
        case 4: return {3};
        case 32: return {0};  // the warp's 32 rows as one voxel stream
        default: return {0, 5, 4};
    }
}

std::vector<Choice> candidates(mi_ctx *ctx, int bins, long long nvox_max) {
    std::vector<Choice> c;
    const int fixed_v = ctx->opt.hist_variant;
    for (int v = 0; v < HV_COUNT; ++v) {
        if (fixed_v >= 0 && v != fixed_v) continue;
        if (hv_fetch(v) == FM_GATHER && !ctx->all_gather) continue;  // moving depth > 12 somewhere
        for (int th : {512, 1024}) {
            if (ctx->opt.block_threads > 0 && th != ctx->opt.block_threads) continue;
            if (!variant_fits(v, bins, th, nvox_max, ctx->max_rows_words, ctx->max_zplanes)) continue;
            const int per_sm = batched_ctas_per_sm(v, bins, th, ctx->max_rows_words, ctx->max_zplanes);
            if (per_sm < 1) continue;
            for (int lpr : tile_lpr(ctx, v)) {
                Choice ch;
                ch.variant = v;
                ch.threads = th;
                ch.ctas = per_sm * ctx->sms;
                ch.tile.lpr_log2 = lpr;
                ch.tile.slabs = ctx->opt.tile_slabs > 0 ? ctx->opt.tile_slabs : 4;
                c.push_back(ch);
            }
        }
    }
    return c;
}

// ---------------------------------------------------------------------------
// Plain path: many CTAs per transform, global histograms, then the entropy kernel
// ---------------------------------------------------------------------------

mi_status run_plain(mi_ctx *ctx, int pair, const int32_t *d_aff, int n, const QSet &Q, const Outputs &O,
                    const Choice &ch, uint32_t *keep_hist) {
    const Pair &P = *ctx->pairs[pair];
    const PairDev hp = host_pairdev(P);
    const PairDev *dp = ctx->d_pairs.as<PairDev>() + pair;
    const size_t B2 = (size_t)P.bins * P.bins;
    int chunk = (int)std::max<size_t>(1, (64u << 20) / (B2 * 4));
    chunk = std::min(chunk, 4096);
    MI_CU(cudaEventRecord(ctx->ev0, ctx->stream), "event");
    ctx->last_launches = 0;
    for (int t0 = 0; t0 < n; t0 += chunk) {
        const int m = std::min(chunk, n - t0);
        uint32_t *hist = keep_hist ? keep_hist + (size_t)t0 * B2 : nullptr;
        if (!hist) {
            MI_CU(ctx->d_hist.ensure((size_t)m * B2 * 4), "allocating histograms");
            hist = ctx->d_hist.as<uint32_t>();
        }
        // CTAs per transform: fill the GPU, but keep at least 8 row batches of 32 rows per CTA
        const long long rows = (long long)P.nf[1] * P.nf[2];
        const int per_sm =
            std::max(1, batched_ctas_per_sm(ch.variant, P.bins, ch.threads, P.rows_words, P.nm[2]));
        long long ctas = ((long long)ctx->sms * per_sm + m - 1) / m;
        ctas = std::min<long long>(ctas, std::max<long long>(1, rows / (32 * 8)));
        MI_CU(launch_plain_hist(dp, hp, d_aff + (size_t)t0 * 12, m, hist, ch.variant, ch.threads, (int)std::max(1LL, ctas),
                                ch.tile, O.flags, ctx->stream),
              "plain histogram kernel");
        if (O.mi || O.h || O.count) {
            Outputs Oc = O;
            if (Oc.mi) Oc.mi += (size_t)t0 * Q.nq;
            if (Oc.h) Oc.h += (size_t)t0 * Q.nq * 3;
            if (Oc.count) Oc.count += t0;
            Oc.dump = nullptr;
            if (m < ctx->sms) {
                // few transforms: the reduction of each histogram is split over several CTAs
                MI_CU(ctx->d_cols.ensure((size_t)m * P.bins * 4), "allocating column sums");
                MI_CU(ctx->d_part.ensure((size_t)m * entropy_parts(P.bins) * (1 + 2 * kMaxQ) * 8),
                      "allocating partial sums");
                MI_CU(launch_entropy_split(hist, m, P.bins, Q, Oc, ctx->d_cols.as<uint32_t>(), ctx->d_part.as<double>(),
                                           ctx->stream),
                      "entropy kernels");
                ctx->last_launches += 2;
            } else {
                MI_CU(launch_entropy(hist, m, P.bins, Q, Oc, ctx->stream), "entropy kernel");
                ctx->last_launches += 1;
            }
        }
        ctx->last_launches += 1;
    }
    MI_CU(cudaEventRecord(ctx->ev1, ctx->stream), "event");
    return MI_OK;
}

// ---------------------------------------------------------------------------
// Batched path: persistent kernel over a work queue, replayed as a CUDA graph
// ---------------------------------------------------------------------------

// Event record that also fires when replayed from a captured graph (external
// event node while the stream is capturing, a plain record otherwise).
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

mi_status launch_batched_once(mi_ctx *ctx, int nitems, const QSet &Q, const Outputs &O, const Choice &ch,
                              bool record = false) {
    MI_CU(cudaMemsetAsync(ctx->d_ticket.p, 0, 2 * sizeof(int), ctx->stream), "resetting the work queue");
    if (record) MI_CU(record_event(ctx->ev0, ctx->stream), "event");
    MI_CU(launch_batched(ctx->d_pairs.as<PairDev>(), ctx->d_aff.as<int32_t>(), ctx->d_items.as<Item>(), nitems,
                         ctx->d_ticket.as<int>(), ctx->max_bins, ctx->max_rows_words, ctx->max_zplanes, ch.variant,
                         ch.threads, ch.ctas, ch.tile, Q, O, ctx->stream),
          "batched kernel");
    if (record) MI_CU(record_event(ctx->ev1, ctx->stream), "event");
    return MI_OK;
}

// On-disk autotune cache: one line per tuned shape, "<key>\t<variant> <threads> <ctas> <lpr_log2> <slabs>".
// The file is named by mi_autotune_cache() or, until that is called, by the MI_AUTOTUNE_CACHE
// environment variable; without a name nothing is read or written.  A cached choice is used only if it
// is still one of the current candidates (so a changed library or device never replays a stale one).
std::mutex g_cache_mutex;
std::string g_cache_path;
bool g_cache_path_set = false;

std::string cache_path() {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    if (!g_cache_path_set) {
        const char *e = getenv("MI_AUTOTUNE_CACHE");
        return e ? std::string(e) : std::string();
    }
    return g_cache_path;
}

uint64_t fnv1a(const std::string &s) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

// Everything the candidates and their timings depend on: the device, the library, the pairs' geometry,
// types and bins, the call's transform-count bucket and the options that restrict the candidates.
std::string tune_key(mi_ctx *ctx, int bucket, int nq) {
    cudaDeviceProp pr;
    std::string dev = "?";
    if (cudaGetDeviceProperties(&pr, ctx->device) == cudaSuccess) dev = pr.name;
    cudaGetLastError();
    std::string pairs;
    for (auto &p : ctx->pairs) {
        char b[160];
        snprintf(b, sizeof b, "%d,%d,%d/%d,%d,%d/%d/%d/%d/%d/%d;", p->nf[0], p->nf[1], p->nf[2], p->nm[0], p->nm[1],
                 p->nm[2], p->mdtype, p->mdepth, p->bins, p->rows_words, p->srow.p ? 1 : 0);
        pairs += b;
    }
    char k[512];
    snprintf(k, sizeof k, "%s|%s|sms%d|n%zu|%016llx|b%d|q%d|hv%d|th%d|tr%d|ts%d", mi_version(), dev.c_str(), ctx->sms,
             ctx->pairs.size(), (unsigned long long)fnv1a(pairs), bucket, nq, ctx->opt.hist_variant,
             ctx->opt.block_threads, ctx->opt.tile_rows, ctx->opt.tile_slabs);
    for (char *c = k; *c; ++c)
        if (*c == '\t' || *c == '\n') *c = ' ';
    return k;
}

bool cache_lookup(const std::string &path, const std::string &key, const std::vector<Choice> &cands, Choice &out) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char *tab = strchr(line, '\t');
        if (!tab || std::string(line, tab - line) != key) continue;
        int v, th, ctas, lpr, slabs;
        if (sscanf(tab + 1, "%d %d %d %d %d", &v, &th, &ctas, &lpr, &slabs) != 5) continue;
        for (const Choice &c : cands)
            if (c.variant == v && c.threads == th && c.ctas == ctas && c.tile.lpr_log2 == lpr && c.tile.slabs == slabs) {
                out = c;  // the last matching line wins
                found = true;
            }
    }
    fclose(f);
    return found;
}

void cache_store(const std::string &path, const std::string &key, const Choice &c) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;  // the cache is an aid: a read-only location only costs the tuning time
    fprintf(f, "%s\t%d %d %d %d %d\n", key.c_str(), c.variant, c.threads, c.ctas, c.tile.lpr_log2, c.tile.slabs);
    fclose(f);
}

// Autotune: time every candidate on the first items of this call (up to three
// waves, so that effects that build up across waves, such as CTAs drifting to
// different parts of the volumes, show in the timing).
mi_status autotune(mi_ctx *ctx, int nitems, const QSet &Q, const Outputs &O, Choice &best,
                   const std::vector<Choice> &cands) {
    if (cands.empty()) return ctx->fail(MI_EUNSUPPORTED, "no histogram variant fits this bin count and volume size");
    if (cands.size() == 1 || !ctx->opt.autotune) {
        best = cands.front();
        // heuristic: plain shared atomics (32-bit counters where they fit), 1024 threads
        for (const Choice &c : cands)
            if ((c.variant == HV_U32 || (c.variant == HV_U16 && best.variant != HV_U32)) && c.threads == 1024) best = c;
        if (best.variant < 0) best = cands.front();
        return MI_OK;
    }
    // Two stages: every candidate is timed on one wave of items (after a warm-up of a few items, which
    // loads its kernel), then the three fastest on three waves; time per item decides.
    cudaEvent_t e0, e1;
    MI_CU(cudaEventCreate(&e0), "event");
    MI_CU(cudaEventCreate(&e1), "event");
    Outputs Ot = O;
    Ot.dump = nullptr;
    auto time_per_item = [&](const Choice &c, int items, float &ms) -> mi_status {
        Choice cc = c;
        cudaEventRecord(e0, ctx->stream);
        mi_status st = launch_batched_once(ctx, items, Q, Ot, cc);
        if (st != MI_OK) return st;
        cudaEventRecord(e1, ctx->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return ctx->cuda_fail(e, "autotuning");
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)items;
        return MI_OK;
    };
    std::vector<std::pair<float, size_t>> first;  // (ms per item on one wave, candidate)
    mi_status st = MI_OK;
    for (size_t i = 0; i < cands.size() && st == MI_OK; ++i) {
        Choice cc = cands[i];
        if ((st = launch_batched_once(ctx, std::min(nitems, 8), Q, Ot, cc)) != MI_OK) break;  // warm-up
        float ms = 0;
        if ((st = time_per_item(cands[i], std::min(nitems, cands[i].ctas), ms)) == MI_OK) first.push_back({ms, i});
    }
    std::sort(first.begin(), first.end());
    float best_ms = 1e30f;
    best = cands.front();
    for (size_t k = 0; k < first.size() && k < 3 && st == MI_OK; ++k) {
        const Choice &c = cands[first[k].second];
        float ms = 0;
        if ((st = time_per_item(c, std::min(nitems, 3 * c.ctas), ms)) != MI_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

mi_status run_batched(mi_ctx *ctx, int nitems, const QSet &Q, const Outputs &O, const Choice &ch, bool use_graph,
                      const std::string &key, const void *h_aff_src, size_t aff_bytes, const void *h_items_src,
                      size_t item_bytes) {
    // inputs go through pinned staging so that a captured graph can replay the copies
    MI_CU(ctx->h_aff.ensure(aff_bytes), "pinned staging");
    MI_CU(ctx->h_items.ensure(item_bytes), "pinned staging");
    memcpy(ctx->h_aff.p, h_aff_src, aff_bytes);
    memcpy(ctx->h_items.p, h_items_src, item_bytes);
    if (!use_graph) {
        MI_CU(cudaMemcpyAsync(ctx->d_aff.p, ctx->h_aff.p, aff_bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D");
        MI_CU(cudaMemcpyAsync(ctx->d_items.p, ctx->h_items.p, item_bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D");
        return launch_batched_once(ctx, nitems, Q, O, ch, true);
    }
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        // set kernel attributes outside of capture
        batched_ctas_per_sm(ch.variant, ctx->max_bins, ch.threads, ctx->max_rows_words, ctx->max_zplanes);
        cudaGraph_t g;
        MI_CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed), "begin capture");
        cudaMemcpyAsync(ctx->d_aff.p, ctx->h_aff.p, aff_bytes, cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(ctx->d_items.p, ctx->h_items.p, item_bytes, cudaMemcpyHostToDevice, ctx->stream);
        mi_status st = launch_batched_once(ctx, nitems, Q, O, ch, true);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        if (st != MI_OK) return st;
        if (e != cudaSuccess) return ctx->cuda_fail(e, "end capture");
        auto ge = std::make_unique<GraphEntry>();
        e = cudaGraphInstantiate(&ge->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return ctx->cuda_fail(e, "instantiating the graph");
        if (ctx->graphs.size() > 32) ctx->graphs.clear();
        it = ctx->graphs.emplace(key, std::move(ge)).first;
    }
    MI_CU(cudaGraphLaunch(it->second->exec, ctx->stream), "graph launch");
    return MI_OK;
}

// ---------------------------------------------------------------------------
// Shared evaluation core for mi_eval / mi_eval_q16 / mi_batch_eval / mi_hist
// ---------------------------------------------------------------------------

struct EvalReq {
    std::vector<int32_t> q16;  // n x 12 (host) -- or device affines below
    const int32_t *d_q16 = nullptr;
    std::vector<int> pair_of;  // n (empty = all pair 0)
    int n = 0;
    int path = MI_PATH_AUTO;
    uint32_t *dump = nullptr;  // device histograms (mi_hist)
};

mi_status eval_core(mi_ctx *ctx, const EvalReq &R, const float *qv, int nq, double *out_mi, double *out_h,
                    int64_t *out_count) {
    const int n = R.n;
    QSet Q;
    mi_status st = make_qset(ctx, qv, nq, Q);
    if (st != MI_OK) return st;
    MI_CU(ctx->d_mi.ensure((size_t)n * nq * 8), "allocating outputs");
    MI_CU(ctx->d_h.ensure((size_t)n * nq * 3 * 8), "allocating outputs");
    MI_CU(ctx->d_cnt.ensure((size_t)n * 8), "allocating outputs");
    MI_CU(ctx->d_aff.ensure((size_t)n * 12 * 4), "allocating affines");
    MI_CU(cudaMemsetAsync(ctx->d_flags.p, 0, 2 * sizeof(int), ctx->stream), "resetting flags");
    Outputs O;
    O.mi = ctx->d_mi.as<double>();
    O.h = ctx->d_h.as<double>();
    O.count = ctx->d_cnt.as<long long>();
    O.dump = R.dump;
    O.flags = ctx->d_flags.as<int>();
    const bool multi = ctx->pairs.size() > 1;
    int path = R.path;
    if (path == MI_PATH_AUTO) path = (multi || n >= ctx->sms) ? MI_PATH_BATCHED : MI_PATH_PLAIN;
    if (multi && path == MI_PATH_PLAIN) return ctx->fail(MI_EINVAL, "multi-pair contexts use the batched path");
    long long nvox_max = 0;
    for (auto &p : ctx->pairs) nvox_max = std::max(nvox_max, p->nvf);
    std::vector<Choice> cands = candidates(ctx, ctx->max_bins, nvox_max);
    if (cands.empty()) return ctx->fail(MI_EUNSUPPORTED, "no histogram variant fits this bin count and volume size");
    if (path == MI_PATH_PLAIN) {
        const int32_t *d_aff = R.d_q16;
        if (!d_aff) {
            MI_CU(cudaMemcpyAsync(ctx->d_aff.p, R.q16.data(), (size_t)n * 48, cudaMemcpyHostToDevice, ctx->stream), "H2D");
            d_aff = ctx->d_aff.as<int32_t>();
        }
        auto key = std::make_tuple((int)MI_PATH_PLAIN, 0, 0);
        Choice ch;
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            ch = it->second;
        } else {
            // heuristic (the plain form is not autotuned): the first of these kinds that fits, with
            // 1024 threads and the stream walk where the fetch allows it
            const int order[] = {HV_U32_GATHER, HV_ROWS_GATHER, HV_U16_GATHER, HV_U32_QUAD, HV_ROWS_QUAD,
                                 HV_U16_QUAD, HV_U32, HV_U16};
            ch = cands.front();
            bool found = false;
            for (int v : order) {
                if (v == HV_U32_GATHER || v == HV_U32_QUAD || v == HV_U32)
                    if (ctx->max_bins > 181) continue;
                for (const Choice &c : cands)
                    if (c.variant == v && c.threads == 1024 && (c.tile.lpr_log2 == 0 || hv_fetch(v) < FM_QUAD)) {
                        ch = c;
                        found = true;
                        break;
                    }
                if (found) break;
            }
            ctx->tuned[key] = ch;
        }
        st = run_plain(ctx, 0, d_aff, n, Q, O, ch, R.dump);
        if (st != MI_OK) return st;
        ctx->timed = true;
    } else {
        // work items sorted by cost (voxels of the pair), largest first
        std::vector<Item> items(n);
        for (int t = 0; t < n; ++t) items[t] = Item{R.pair_of.empty() ? 0 : R.pair_of[t], t};
        if (multi)
            std::stable_sort(items.begin(), items.end(), [&](const Item &a, const Item &b) {
                return ctx->pairs[a.pair]->nvf > ctx->pairs[b.pair]->nvf;
            });
        MI_CU(ctx->d_items.ensure((size_t)n * sizeof(Item)), "allocating items");
        std::vector<int32_t> q16h;
        const int32_t *h_aff = R.q16.data();
        if (R.d_q16) {
            q16h.resize((size_t)n * 12);
            if ((st = read_from_device(ctx, q16h.data(), R.d_q16, (size_t)n * 48)) != MI_OK) return st;
            h_aff = q16h.data();
        }
        const int bucket = n >= 4 * ctx->sms ? 2 : (n >= ctx->sms ? 1 : 0);
        auto key = std::make_tuple((int)MI_PATH_BATCHED, -1, bucket);
        Choice ch;
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            ch = it->second;
        } else {
            const std::string cpath = ctx->opt.autotune && cands.size() > 1 ? cache_path() : std::string();
            const std::string ckey = cpath.empty() ? std::string() : tune_key(ctx, bucket, nq);
            if (cpath.empty() || !cache_lookup(cpath, ckey, cands, ch)) {
                // tuning needs the inputs on the device
                MI_CU(cudaMemcpyAsync(ctx->d_aff.p, h_aff, (size_t)n * 48, cudaMemcpyHostToDevice, ctx->stream),
                      "H2D");
                MI_CU(cudaMemcpyAsync(ctx->d_items.p, items.data(), (size_t)n * sizeof(Item), cudaMemcpyHostToDevice,
                                      ctx->stream),
                      "H2D");
                st = autotune(ctx, n, Q, O, ch, cands);
                if (st != MI_OK) return st;
                MI_CU(cudaMemsetAsync(ctx->d_flags.p, 0, 2 * sizeof(int), ctx->stream), "resetting flags");
                if (!cpath.empty()) cache_store(cpath, ckey, ch);
            }
            ctx->tuned[key] = ch;
        }
        const bool use_graph = ctx->opt.use_graphs && !R.dump && ctx->stream != nullptr;
        // staging buffers are sized before the key is formed: a graph replays copies from their addresses
        MI_CU(ctx->h_aff.ensure((size_t)n * 48), "pinned staging");
        MI_CU(ctx->h_items.ensure((size_t)n * sizeof(Item)), "pinned staging");
        char kb[512];
        int off = snprintf(kb, sizeof kb, "b:%d:%d:%d:%d:%d:%d:%d:%p:%p:%p:%p:%p:%p:%p:%d:%d", n, nq, ch.variant,
                           ch.threads, ch.ctas, ch.tile.lpr_log2, ch.tile.slabs, ctx->d_aff.p, ctx->d_items.p,
                           ctx->d_mi.p, ctx->d_h.p, ctx->d_cnt.p, ctx->h_aff.p, ctx->h_items.p, Q.form, Q.bits);
        for (int i = 0; i < nq && off < (int)sizeof kb - 40; ++i)
            off += snprintf(kb + off, sizeof kb - off, ":%08x:%p", fbits(Q.q[i]), (const void *)Q.tab[i]);
        st = run_batched(ctx, n, Q, O, ch, use_graph, kb, h_aff, (size_t)n * 48, items.data(), (size_t)n * sizeof(Item));
        if (st != MI_OK) return st;
        ctx->timed = true;
        ctx->last_launches = 1;
    }
    if ((st = deliver(ctx, out_mi, ctx->d_mi.p, (size_t)n * nq * 8)) != MI_OK) return st;
    if ((st = deliver(ctx, out_h, ctx->d_h.p, (size_t)n * nq * 3 * 8)) != MI_OK) return st;
    if ((st = deliver(ctx, out_count, ctx->d_cnt.p, (size_t)n * 8)) != MI_OK) return st;
    int flags[2] = {0, 0};
    MI_CU(cudaMemcpyAsync(flags, ctx->d_flags.p, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream), "reading flags");
    MI_CU(cudaStreamSynchronize(ctx->stream), "evaluation");
    if (flags[1]) return ctx->fail(MI_ECUDA, "internal: 16-bit counter drain failed (flags " + std::to_string(flags[1]) + ")");
    if (flags[0]) return ctx->fail(MI_EEMPTY, "at least one transform has an empty overlap (its MI is NaN)");
    return MI_OK;
}

// ---------------------------------------------------------------------------
// Parzen
// ---------------------------------------------------------------------------

// Parzen MI (and, with out_grad, its gradient) for n transforms; pair_of (n entries) names each
// transform's pair in a multi-pair context (NULL: pair 0).  One launch per kernel for all pairs.
mi_status parzen_core(mi_ctx *ctx, const std::vector<float> &prm, int n, const float *qv, int nq, double *out_mi,
                      double *out_grad, const std::vector<int> *pair_of = nullptr, int64_t *out_count = nullptr) {
    const int Bmax = ctx->p_bmax;
    const size_t BM2 = (size_t)Bmax * Bmax;
    QSet Q;
    mi_status st = make_qset(ctx, qv, nq, Q);
    if (st != MI_OK) return st;
    const int np = ctx->nparams();
    const bool multi = pair_of != nullptr;
    std::vector<ParzenAffine> pa(n);
    std::vector<double> jac((size_t)n * 12 * np);
    std::vector<long long> row_start(multi ? n + 1 : 0);
    long long total_rows = 0;
    for (int t = 0; t < n; ++t) {
        const int pi = multi ? (*pair_of)[t] : 0;
        if (pi < 0 || pi >= (int)ctx->pairs.size()) return ctx->fail(MI_EINVAL, "pair index out of range");
        const Pair &P = *ctx->pairs[pi];
        double aff[12];
        double *J = &jac[(size_t)t * 12 * np];
        build_affine_opt(ctx->opt, &prm[(size_t)t * np], P.nf, P.sf, P.nm, P.sm, aff, J);
        for (int e = 0; e < 12; ++e) {
            const double sc = aff[e] * 4294967296.0;
            if (!(fabs(sc) < 4503599627370496.0))  // |x| < 2^20 keeps every int64 product below 2^63
                return ctx->fail(MI_ERANGE, "transform " + std::to_string(t) + ": affine out of range");
            pa[t].A[e] = llround(sc);
        }
        // re-centre: u = A (i - c) + (A c + b), so the constant row becomes dA c + db
        for (int a = 0; a < 3; ++a)
            for (int p = 0; p < np; ++p) {
                double acc = J[np * (4 * a + 3) + p];
                for (int c = 0; c < 3; ++c) acc += J[np * (4 * a + c) + p] * (0.5 * (double)(P.nf[c] - 1));
                J[np * (4 * a + 3) + p] = acc;
            }
        if (multi) row_start[t] = total_rows;
        total_rows += (long long)P.nf[1] * P.nf[2];
    }
    if (multi) row_start[n] = total_rows;
    cudaStream_t s = ctx->stream;
    // the launch shapes follow the largest pair (most fixed rows), with the largest bin count
    int big = 0;
    for (size_t i = 1; i < ctx->pairs.size(); ++i)
        if ((long long)ctx->pairs[i]->nf[1] * ctx->pairs[i]->nf[2] >
            (long long)ctx->pairs[big]->nf[1] * ctx->pairs[big]->nf[2])
            big = (int)i;
    ParzenPair rep = parzen_pair(ctx, *ctx->pairs[multi ? big : 0]);
    rep.B = Bmax;
    ParzenLaunch L;
    L.p0 = parzen_pair(ctx, *ctx->pairs[0]);
    L.d_pairs = ctx->p_pairs.as<ParzenPair>();
    L.d_pair_of = nullptr;
    L.d_row_start = nullptr;
    L.n = n;
    L.Bmax = Bmax;
    L.nx_max = ctx->p_nxmax;
    L.sampled = ctx->pairs[0]->srow.p != nullptr;
    L.total_rows = total_rows;
    const int actas = out_grad ? parzen_adj_ctas(rep, n, nq, ctx->sms) : 1;
    const int cblocks = parzen_cell_blocks(Bmax);
    if (multi) {
        MI_CU(ctx->p_pair_of.ensure((size_t)n * sizeof(int)), "alloc");
        MI_CU(ctx->p_row_start.ensure((size_t)(n + 1) * sizeof(long long)), "alloc");
        MI_CU(cudaMemcpyAsync(ctx->p_pair_of.p, pair_of->data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s),
              "H2D");
        MI_CU(cudaMemcpyAsync(ctx->p_row_start.p, row_start.data(), (size_t)(n + 1) * sizeof(long long),
                              cudaMemcpyHostToDevice, s),
              "H2D");
        L.d_pair_of = ctx->p_pair_of.as<int>();
        L.d_row_start = ctx->p_row_start.as<long long>();
    }
    MI_CU(ctx->p_aff.ensure((size_t)n * sizeof(ParzenAffine)), "alloc");
    MI_CU(ctx->p_jac.ensure((size_t)n * 12 * np * 8), "alloc");
    MI_CU(ctx->p_hist.ensure((size_t)n * BM2 * 8), "alloc");
    MI_CU(ctx->p_cnt.ensure((size_t)n * 8), "alloc");
    MI_CU(ctx->p_marg.ensure((size_t)n * 2 * Bmax * 8), "alloc");
    MI_CU(ctx->p_ment.ensure((size_t)n * nq * 2 * 8), "alloc");
    MI_CU(ctx->p_mterm.ensure((size_t)n * nq * 2 * Bmax * 8), "alloc");
    MI_CU(ctx->p_jsum.ensure((size_t)n * nq * cblocks * 8), "alloc");
    MI_CU(ctx->p_w.ensure((size_t)n * nq * BM2 * 4), "alloc");
    MI_CU(ctx->p_mom.ensure((size_t)n * nq * actas * 12 * 8), "alloc");
    MI_CU(ctx->p_grad.ensure((size_t)n * nq * np * 8), "alloc");
    MI_CU(ctx->d_mi.ensure((size_t)n * nq * 8), "alloc");
    MI_CU(cudaMemcpyAsync(ctx->p_aff.p, pa.data(), (size_t)n * sizeof(ParzenAffine), cudaMemcpyHostToDevice, s), "H2D");
    MI_CU(cudaMemcpyAsync(ctx->p_jac.p, jac.data(), (size_t)n * 12 * np * 8, cudaMemcpyHostToDevice, s), "H2D");
    const ParzenAffine *d_aff = ctx->p_aff.as<ParzenAffine>();
    auto *cnt = ctx->p_cnt.as<unsigned long long>();
    auto *hist = ctx->p_hist.as<unsigned long long>();
    MI_CU(cudaEventRecord(ctx->ev0, s), "event");
    MI_CU(launch_parzen_hist(L, d_aff, ctx->sms, hist, cnt, s), "Parzen histogram");
    MI_CU(launch_parzen_weights(hist, cnt, L, Q, ctx->p_marg.as<double>(), ctx->p_ment.as<double>(),
                                ctx->p_mterm.as<double>(), ctx->p_jsum.as<double>(), ctx->d_mi.as<double>(),
                                ctx->p_w.as<float>(), s),
          "Parzen entropies");
    if (out_grad)
        MI_CU(launch_parzen_adjoint(L, d_aff, ctx->p_jac.as<double>(), np, nq, actas, ctx->p_w.as<float>(), cnt,
                                    ctx->p_mom.as<double>(), ctx->p_grad.as<double>(), s),
              "Parzen adjoint");
    MI_CU(cudaEventRecord(ctx->ev1, s), "event");
    ctx->timed = true;
    ctx->last_launches = 4 + (out_grad ? (nq + 3) / 4 + 1 : 0);
    if ((st = deliver(ctx, out_mi, ctx->d_mi.p, (size_t)n * nq * 8)) != MI_OK) return st;
    if (out_grad && (st = deliver(ctx, out_grad, ctx->p_grad.p, (size_t)n * nq * np * 8)) != MI_OK) return st;
    if (out_count && (st = deliver(ctx, out_count, cnt, (size_t)n * 8)) != MI_OK) return st;
    std::vector<unsigned long long> hc(n);
    MI_CU(cudaMemcpyAsync(hc.data(), cnt, (size_t)n * 8, cudaMemcpyDeviceToHost, s), "reading counts");
    MI_CU(cudaStreamSynchronize(s), "Parzen evaluation");
    for (int t = 0; t < n; ++t)
        if (hc[t] == 0) return ctx->fail(MI_EEMPTY, "at least one transform has an empty overlap (its MI is NaN)");
    return MI_OK;
}

// The pair indices of mi_batch_eval / mi_batch_grad (host or device memory), checked.
mi_status read_pair_of(mi_ctx *ctx, const int *pair_of_transform, int n, std::vector<int> &out) {
    out.resize(n);
    if (is_device_ptr(pair_of_transform)) {
        mi_status st = read_from_device(ctx, out.data(), pair_of_transform, (size_t)n * 4);
        if (st != MI_OK) return st;
    } else {
        memcpy(out.data(), pair_of_transform, (size_t)n * 4);
    }
    for (int t = 0; t < n; ++t)
        if (out[t] < 0 || out[t] >= (int)ctx->pairs.size()) return ctx->fail(MI_EINVAL, "pair index out of range");
    return MI_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

void mi_options_default(mi_options *opt) {
    if (!opt) return;
    opt->kernel = MI_HARD;
    opt->tsallis_form = MI_TSALLIS_ADDITIVE;
    opt->log_bits = 0;
    opt->hist_variant = MI_HV_AUTO;
    opt->path = MI_PATH_AUTO;
    opt->use_graphs = 1;
    opt->autotune = 1;
    opt->device = -1;
    opt->block_threads = 0;
    opt->rotation = MI_ROT_EULER_DEG;
    opt->scale = MI_SCALE_FACTOR;
    opt->sample_fraction = 0.0f;
    opt->sample_seed = 0u;
    opt->transform = MI_TRANSFORM_PARAMS;
    opt->tile_rows = 0;
    opt->tile_slabs = 0;
}

const char *mi_version(void) { return "gb300-mi 0.1 (sm_103a)"; }

int mi_transform_size(const mi_ctx *ctx) { return ctx ? ctx->nparams() : -1; }

void mi_fault_alloc(int after) { g_fault_alloc.store(after < 0 ? -1 : after); }

mi_status mi_fault_drain_cap(int cap) {
    if (cap < 0) return MI_EINVAL;
    return set_drain_cap(cap) == cudaSuccess ? MI_OK : MI_ECUDA;
}

mi_status mi_create(mi_ctx **out, const mi_volume *fixed, const mi_volume *moving, int bins, const mi_options *opt) {
    return create_common(out, fixed, moving, &bins, 1, opt);
}

mi_status mi_batch_create(mi_ctx **out, const mi_volume *fixed, const mi_volume *moving, const int *bins, int npairs,
                          const mi_options *opt) {
    mi_options o;
    if (opt)
        o = *opt;
    else
        mi_options_default(&o);
    return create_common(out, fixed, moving, bins, npairs, &o);
}

void mi_destroy(mi_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
        ctx->graphs.clear();
        ctx->tables.clear();
        ctx->pairs.clear();
        if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
        ctx->own_stream = nullptr;
        if (ctx->ev0) cudaEventDestroy(ctx->ev0);
        if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    }
    delete ctx;
}

const char *mi_last_error(const mi_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

mi_status mi_set_stream(mi_ctx *ctx, void *stream) {
    if (!ctx) return MI_EINVAL;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    ctx->graphs.clear();
    return MI_OK;
}

mi_status mi_eval(mi_ctx *ctx, const float *transforms, int n, const float *q, int nq, double *out_mi, double *out_h,
                  int64_t *out_count) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (n < 0) return ctx->fail(MI_EINVAL, "n < 0");
    float qv[kMaxQ];
    mi_status st = read_q(ctx, q, nq, qv);
    if (st != MI_OK) return st;
    if (n == 0) return MI_OK;
    if (!out_mi) return ctx->fail(MI_EINVAL, "out_mi is NULL");
    if (ctx->pairs.size() != 1) return ctx->fail(MI_EINVAL, "mi_eval needs a single-pair context (use mi_batch_eval)");
    std::vector<float> prm;
    if ((st = read_transforms(ctx, transforms, n, prm)) != MI_OK) return st;
    if (ctx->opt.kernel == MI_PARZEN) {
        if (out_h) return ctx->fail(MI_EUNSUPPORTED, "out_h (hard-histogram entropies) is a hard-path output");
        return parzen_core(ctx, prm, n, qv, nq, out_mi, nullptr, nullptr, out_count);
    }
    EvalReq R;
    R.n = n;
    R.path = ctx->opt.path;
    R.q16.resize((size_t)n * 12);
    for (int t = 0; t < n; ++t)
        if ((st = build_q16(ctx, *ctx->pairs[0], &prm[(size_t)t * ctx->nparams()], &R.q16[(size_t)t * 12], t)) != MI_OK) return st;
    return eval_core(ctx, R, qv, nq, out_mi, out_h, out_count);
}

mi_status mi_eval_q16(mi_ctx *ctx, const int32_t *affines, int n, const float *q, int nq, double *out_mi, double *out_h,
                      int64_t *out_count) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (n < 0) return ctx->fail(MI_EINVAL, "n < 0");
    if (ctx->opt.kernel != MI_HARD) return ctx->fail(MI_EUNSUPPORTED, "mi_eval_q16 is a hard-path entry point");
    float qv[kMaxQ];
    mi_status st = read_q(ctx, q, nq, qv);
    if (st != MI_OK) return st;
    if (n == 0) return MI_OK;
    if (!out_mi) return ctx->fail(MI_EINVAL, "out_mi is NULL");
    if (!affines) return ctx->fail(MI_EINVAL, "affines is NULL");
    EvalReq R;
    R.n = n;
    R.path = ctx->opt.path;
    if (is_device_ptr(affines)) {
        R.d_q16 = affines;
    } else {
        R.q16.assign(affines, affines + (size_t)n * 12);
    }
    return eval_core(ctx, R, qv, nq, out_mi, out_h, out_count);
}

mi_status mi_batch_eval(mi_ctx *ctx, const int *pair_of_transform, const float *transforms, int n, const float *q,
                        int nq, double *out_mi, double *out_h, int64_t *out_count) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (n < 0) return ctx->fail(MI_EINVAL, "n < 0");
    float qv[kMaxQ];
    mi_status st = read_q(ctx, q, nq, qv);
    if (st != MI_OK) return st;
    if (n == 0) return MI_OK;
    if (!out_mi || !pair_of_transform) return ctx->fail(MI_EINVAL, "out_mi or pair_of_transform is NULL");
    std::vector<float> prm;
    if ((st = read_transforms(ctx, transforms, n, prm)) != MI_OK) return st;
    if (ctx->opt.kernel == MI_PARZEN) {
        if (out_h || out_count) return ctx->fail(MI_EUNSUPPORTED, "out_h / out_count are hard-path outputs");
        std::vector<int> po;
        if ((st = read_pair_of(ctx, pair_of_transform, n, po)) != MI_OK) return st;
        return parzen_core(ctx, prm, n, qv, nq, out_mi, nullptr, &po);
    }
    EvalReq R;
    R.n = n;
    R.path = MI_PATH_BATCHED;
    R.pair_of.resize(n);
    if (is_device_ptr(pair_of_transform)) {
        if ((st = read_from_device(ctx, R.pair_of.data(), pair_of_transform, (size_t)n * 4)) != MI_OK) return st;
    } else {
        memcpy(R.pair_of.data(), pair_of_transform, (size_t)n * 4);
    }
    R.q16.resize((size_t)n * 12);
    for (int t = 0; t < n; ++t) {
        const int p = R.pair_of[t];
        if (p < 0 || p >= (int)ctx->pairs.size()) return ctx->fail(MI_EINVAL, "pair index out of range");
        if ((st = build_q16(ctx, *ctx->pairs[p], &prm[(size_t)t * ctx->nparams()], &R.q16[(size_t)t * 12], t)) != MI_OK) return st;
    }
    return eval_core(ctx, R, qv, nq, out_mi, out_h, out_count);
}

mi_status mi_grad(mi_ctx *ctx, const float *transforms, int n, const float *q, int nq, double *out_mi,
                  double *out_grad) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (ctx->opt.kernel != MI_PARZEN)
        return ctx->fail(MI_EUNSUPPORTED, "mi_grad needs a MI_PARZEN context (the hard histogram is not differentiable)");
    if (n < 0) return ctx->fail(MI_EINVAL, "n < 0");
    float qv[kMaxQ];
    mi_status st = read_q(ctx, q, nq, qv);
    if (st != MI_OK) return st;
    if (n == 0) return MI_OK;
    if (!out_mi || !out_grad) return ctx->fail(MI_EINVAL, "out_mi or out_grad is NULL");
    if (ctx->pairs.size() != 1) return ctx->fail(MI_EINVAL, "mi_grad needs a single-pair context (use mi_batch_grad)");
    std::vector<float> prm;
    if ((st = read_transforms(ctx, transforms, n, prm)) != MI_OK) return st;
    return parzen_core(ctx, prm, n, qv, nq, out_mi, out_grad);
}

mi_status mi_batch_grad(mi_ctx *ctx, const int *pair_of_transform, const float *transforms, int n, const float *q,
                        int nq, double *out_mi, double *out_grad) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (ctx->opt.kernel != MI_PARZEN)
        return ctx->fail(MI_EUNSUPPORTED, "mi_batch_grad needs a MI_PARZEN context (the hard histogram is not differentiable)");
    if (n < 0) return ctx->fail(MI_EINVAL, "n < 0");
    float qv[kMaxQ];
    mi_status st = read_q(ctx, q, nq, qv);
    if (st != MI_OK) return st;
    if (n == 0) return MI_OK;
    if (!out_mi || !out_grad || !pair_of_transform)
        return ctx->fail(MI_EINVAL, "out_mi, out_grad or pair_of_transform is NULL");
    std::vector<float> prm;
    if ((st = read_transforms(ctx, transforms, n, prm)) != MI_OK) return st;
    std::vector<int> po;
    if ((st = read_pair_of(ctx, pair_of_transform, n, po)) != MI_OK) return st;
    return parzen_core(ctx, prm, n, qv, nq, out_mi, out_grad, &po);
}

mi_status mi_hist(mi_ctx *ctx, int pair, const float *transforms, const int32_t *affines, int n, int path,
                  uint32_t *out_counts) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (ctx->opt.kernel != MI_HARD) return ctx->fail(MI_EUNSUPPORTED, "mi_hist is a hard-path entry point");
    if (pair < 0 || pair >= (int)ctx->pairs.size()) return ctx->fail(MI_EINVAL, "pair index out of range");
    if (n < 0 || (!transforms == !affines)) return ctx->fail(MI_EINVAL, "give exactly one of transforms and affines");
    if (path != MI_PATH_PLAIN && path != MI_PATH_BATCHED) return ctx->fail(MI_EINVAL, "path must be PLAIN or BATCHED");
    if (ctx->pairs.size() != 1 && path == MI_PATH_PLAIN) return ctx->fail(MI_EINVAL, "plain path needs a single pair");
    if (n == 0) return MI_OK;
    if (!out_counts) return ctx->fail(MI_EINVAL, "out_counts is NULL");
    const Pair &P = *ctx->pairs[pair];
    EvalReq R;
    R.n = n;
    R.path = path;
    R.q16.resize((size_t)n * 12);
    mi_status st;
    if (transforms) {
        std::vector<float> prm;
        if ((st = read_transforms(ctx, transforms, n, prm)) != MI_OK) return st;
        for (int t = 0; t < n; ++t)
            if ((st = build_q16(ctx, P, &prm[(size_t)t * ctx->nparams()], &R.q16[(size_t)t * 12], t)) != MI_OK) return st;
    } else if (is_device_ptr(affines)) {
        if ((st = read_from_device(ctx, R.q16.data(), affines, (size_t)n * 48)) != MI_OK) return st;
    } else {
        R.q16.assign(affines, affines + (size_t)n * 12);
    }
    if (ctx->pairs.size() > 1) R.pair_of.assign(n, pair);
    const size_t B2 = (size_t)P.bins * P.bins;
    MI_CU(ctx->d_dump.ensure((size_t)n * B2 * 4), "allocating histograms");
    R.dump = ctx->d_dump.as<uint32_t>();
    const float one = 1.0f;
    st = eval_core(ctx, R, &one, 1, nullptr, nullptr, nullptr);
    if (st != MI_OK && st != MI_EEMPTY) return st;
    mi_status st2 = deliver(ctx, out_counts, R.dump, (size_t)n * B2 * 4);
    if (st2 != MI_OK) return st2;
    MI_CU(cudaStreamSynchronize(ctx->stream), "copying histograms");
    return MI_OK;
}

mi_status mi_affine(mi_ctx *ctx, int pair, const float *transforms, int n, double *out_affine, int32_t *out_q16,
                    double *out_jacobian) {
    if (!ctx) return MI_EINVAL;
    if (pair < 0 || pair >= (int)ctx->pairs.size()) return ctx->fail(MI_EINVAL, "pair index out of range");
    if (n < 0 || (n > 0 && !transforms)) return ctx->fail(MI_EINVAL, "bad transforms");
    const Pair &P = *ctx->pairs[pair];
    mi_status st = MI_OK;
    const int np = ctx->nparams();
    for (int t = 0; t < n; ++t) {
        double aff[12], jac[144];
        build_affine_opt(ctx->opt, transforms + (size_t)t * np, P.nf, P.sf, P.nm, P.sm, aff,
                         out_jacobian ? jac : nullptr);
        if (out_affine) memcpy(out_affine + (size_t)t * 12, aff, sizeof aff);
        if (out_jacobian) memcpy(out_jacobian + (size_t)t * 12 * np, jac, sizeof(double) * 12 * np);
        if (out_q16) {
            int32_t q[12];
            if (!quantise_q16(aff, q)) {
                st = ctx->fail(MI_ERANGE, "transform " + std::to_string(t) + ": affine does not fit 16.16 fixed point");
                memset(q, 0, sizeof q);
            }
            memcpy(out_q16 + (size_t)t * 12, q, sizeof q);
        }
    }
    return st;
}

mi_status mi_fixed_bins(mi_ctx *ctx, int pair, uint8_t *out) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (pair < 0 || pair >= (int)ctx->pairs.size() || !out) return ctx->fail(MI_EINVAL, "bad pair or output");
    const Pair &P = *ctx->pairs[pair];
    const DevBuf &src = ctx->opt.kernel == MI_PARZEN ? P.pfbins : P.fbins;
    mi_status st = deliver(ctx, out, src.p, (size_t)P.nvf);
    if (st != MI_OK) return st;
    MI_CU(cudaStreamSynchronize(ctx->stream), "copying bins");
    return MI_OK;
}

mi_status mi_resample(mi_ctx *ctx, int pair, const int32_t *affine, void *out) {
    if (!ctx) return MI_EINVAL;
    DeviceGuard guard(ctx->device);
    if (ctx->opt.kernel != MI_HARD) return ctx->fail(MI_EUNSUPPORTED, "mi_resample is a hard-path entry point");
    if (pair < 0 || pair >= (int)ctx->pairs.size() || !out || !affine) return ctx->fail(MI_EINVAL, "bad arguments");
    const Pair &P = *ctx->pairs[pair];
    int32_t q[12];
    if (is_device_ptr(affine)) {
        mi_status st = read_from_device(ctx, q, affine, 48);
        if (st != MI_OK) return st;
    } else {
        memcpy(q, affine, 48);
    }
    MI_CU(ctx->d_aff.ensure(48), "alloc");
    MI_CU(cudaMemcpyAsync(ctx->d_aff.p, q, 48, cudaMemcpyHostToDevice, ctx->stream), "H2D");
    const size_t bytes = (size_t)P.nvf * (P.mdtype == 0 ? 1 : 2);
    DevBuf tmp;
    void *dst = out;
    if (!is_device_ptr(out)) {
        MI_CU(tmp.ensure(bytes), "alloc");
        dst = tmp.p;
    }
    MI_CU(launch_resample(ctx->d_pairs.as<PairDev>() + pair, host_pairdev(P), ctx->d_aff.as<int32_t>(), dst, ctx->stream),
          "resample kernel");
    if (dst != out) MI_CU(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H");
    MI_CU(cudaStreamSynchronize(ctx->stream), "resampling");
    return MI_OK;
}

mi_status mi_last_kernel_ms(mi_ctx *ctx, float *ms, int *launches) {
    if (!ctx || !ms) return MI_EINVAL;
    if (!ctx->timed) return ctx->fail(MI_EINVAL, "no timed call yet");
    DeviceGuard guard(ctx->device);
    MI_CU(cudaEventSynchronize(ctx->ev1), "event");
    MI_CU(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1), "event elapsed time");
    if (launches) *launches = ctx->last_launches;
    return MI_OK;
}

static const Choice *selected_choice(mi_ctx *ctx, int n) {
    const int path = ctx->opt.path == MI_PATH_AUTO ? ((ctx->pairs.size() > 1 || n >= ctx->sms) ? MI_PATH_BATCHED : MI_PATH_PLAIN)
                                                   : ctx->opt.path;
    const int bucket = path == MI_PATH_BATCHED ? (n >= 4 * ctx->sms ? 2 : (n >= ctx->sms ? 1 : 0)) : 0;
    auto it = ctx->tuned.find(std::make_tuple(path, path == MI_PATH_BATCHED ? -1 : 0, bucket));
    return it == ctx->tuned.end() ? nullptr : &it->second;
}

int mi_selected_variant(mi_ctx *ctx, int pair, int n) {
    if (!ctx) return -1;
    (void)pair;
    const Choice *c = selected_choice(ctx, n);
    return c ? c->variant : -1;
}

void mi_autotune_cache(const char *path) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_cache_path = path ? path : "";
    g_cache_path_set = true;
}

mi_status mi_selected_config(mi_ctx *ctx, int n, int out[5]) {
    if (!ctx || !out) return MI_EINVAL;
    const Choice *c = selected_choice(ctx, n);
    if (!c) {
        for (int i = 0; i < 5; ++i) out[i] = -1;
        return MI_OK;
    }
    out[0] = c->variant;
    out[1] = c->threads;
    out[2] = c->ctas;
    out[3] = c->tile.lpr_log2 == 0 ? 32 : 32 >> c->tile.lpr_log2;
    out[4] = c->tile.slabs;
    return MI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Helpers for the allocation-free entry point in mi_noalloc.cu
// ---------------------------------------------------------------------------
namespace mi {

bool host_affine_q16(const float prm[9], const int nf[3], const float sf[3], const int nm[3], const float sm[3],
                     int32_t q16[12]) {
    double aff[12];
    build_affine(prm, nf, sf, nm, sm, aff, nullptr);
    return quantise_q16(aff, q16);
}

void set_thread_error(const char *msg) { g_create_error = msg; }

}  // namespace mi
