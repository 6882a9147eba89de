// mi_parzen.cu -- differentiable (Parzen-window) mutual information on sm_103a.
//
// Soft joint histogram: each overlap voxel adds beta0 (one bin) along the
// fixed axis and a cubic B-spline beta3 centred at m~ = m (B - 4) + 2 along
// the moving axis, m the FP32 trilinear value of the normalised moving volume
// at the real moving index u = A i + b.  Positions are 32.32 fixed point
// (int64) from the FP64 affine: the gradient jumps where a sample crosses a
// trilinear cell boundary, so cell and overlap decisions are taken on
// near-exact positions rather than FP32 ones.  Shannon MI (Eq. 1-2) and Tsallis MI
// follow from the normalised histogram P in FP64.  The gradient of MI with
// respect to the 9 transform parameters (the optimiser's input, Eq. 3 and
// the gradient-descent loop of the Introduction) is the adjoint:
//   dMI/dtheta = -(B-4)/N sum_x s(x) grad m(u_x) . du_x/dtheta,
//   s(x) = sum_k W(fb(x), k) beta3'(k - m~_x),   W = dMI/dP,
// with N and the overlap held fixed.  du/dtheta = J [i j k 1]^T is linear in
// the voxel index, so each thread accumulates the 12 moments
// sum s grad_a m * (i, j, k, 1) per q and the host Jacobian J (12 x 9)
// contracts them at the end.
//
// Kernels: k_pfix / k_pmov (once per context), k_parzen_hist (forward),
// k_parzen_marg + k_parzen_cells + k_parzen_final (FP64 entropies and W),
// k_parzen_adj + k_parzen_grad (adjoint).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "mi_internal.h"

namespace mi {
namespace {

// The dynamic shared memory a launch of fn needs, allowed on the current device (set before every
// launch: a device reset would clear it).
cudaError_t allow_smem(const void *fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Resident CTAs per SM (at least 1) of fn at a launch shape, asked of the driver once per process and
// device (it depends on nothing else); allow_smem(fn, smem) must have succeeded.
std::mutex g_launch_mu;
std::map<std::tuple<int, const void *, int, size_t>, int> g_per_sm;

int resident_per_sm(const void *fn, int threads, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_launch_mu);
    const auto key = std::make_tuple(dev, fn, threads, smem);
    auto it = g_per_sm.find(key);
    if (it != g_per_sm.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        return 1;
    }
    g_per_sm.emplace(key, nb);
    return nb;
}

constexpr unsigned kFull = 0xffffffffu;

inline int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

// Fixed bin floor(f (B - 4)) + 2: exact integer quotient for integer volumes.
template <typename T>
__global__ void k_pfix_int(const T *__restrict__ in, long long n, int depth, int B, uint8_t *__restrict__ out) {
    const unsigned long long vmax = (1ull << depth) - 1ull;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        unsigned long long v = in[x];
        v = v > vmax ? vmax : v;
        out[x] = (uint8_t)((v * (unsigned long long)(B - 4)) / vmax + 2ull);
    }
}

__global__ void k_pfix_f32(const float *__restrict__ in, long long n, int B, uint8_t *__restrict__ out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double f = (double)in[x];
        if (!(f == f)) f = 0.0;
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        out[x] = (uint8_t)((int)floor(f * (double)(B - 4)) + 2);
    }
}

// Normalised moving intensity: v / (2^d - 1) (rounded once to FP32), floats clamped to [0, 1].
template <typename T>
__global__ void k_pmov_int(const T *__restrict__ in, long long n, int depth, float *__restrict__ out) {
    const double vmax = (double)((1ull << depth) - 1ull);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double v = (double)in[x];
        out[x] = (float)(v > vmax ? 1.0 : v / vmax);
    }
}

__global__ void k_pmov_f32(const float *__restrict__ in, long long n, float *__restrict__ out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        float v = in[x];
        if (!(v == v)) v = 0.0f;
        out[x] = fminf(fmaxf(v, 0.0f), 1.0f);
    }
}

// FP32 trilinear value and gradient (w.r.t. the moving index) at a 32.32
// index u inside [0, n-1]^3, read from the extended volume (dims n + 1 per
// axis): the cell is the integer part of u and the weight its fraction, also
// on the last plane, where the extension makes the value v[n-1] and the
// derivative v[n-1] - v[n-2] (those of the last cell of the volume).
struct MG {
    float m, gx, gy, gz;
};

// m0 = n0 + 1 and m01 = (n0 + 1)(n1 + 1): element offsets fit 32 bits (the extended volume holds fewer
// than 2^31 elements, checked when the context is created).
template <bool GRAD>
__device__ __forceinline__ MG trilinear_x(const float *__restrict__ movx, int m0, int m01, long long Ux,
                                          long long Uy, long long Uz) {
    constexpr float k2m32 = 2.3283064365386963e-10f;  // 2^-32
    const int cx = (int)(Ux >> 32), cy = (int)(Uy >> 32), cz = (int)(Uz >> 32);
    const float wx = __uint2float_rn((unsigned)Ux) * k2m32, wy = __uint2float_rn((unsigned)Uy) * k2m32,
                wz = __uint2float_rn((unsigned)Uz) * k2m32;
    const float *p = movx + (cx + m0 * cy + m01 * cz);
    const float v000 = __ldg(p), v001 = __ldg(p + 1), v010 = __ldg(p + m0), v011 = __ldg(p + m0 + 1);
    const float v100 = __ldg(p + m01), v101 = __ldg(p + m01 + 1), v110 = __ldg(p + m01 + m0),
                v111 = __ldg(p + m01 + m0 + 1);
    const float d00 = v001 - v000, d01 = v011 - v010, d10 = v101 - v100, d11 = v111 - v110;
    const float a00 = fmaf(wx, d00, v000), a01 = fmaf(wx, d01, v010);
    const float a10 = fmaf(wx, d10, v100), a11 = fmaf(wx, d11, v110);
    const float b0 = fmaf(wy, a01 - a00, a00), b1 = fmaf(wy, a11 - a10, a10);
    MG r;
    r.m = fmaf(wz, b1 - b0, b0);
    if (GRAD) {
        r.gz = b1 - b0;
        const float y0 = a01 - a00, y1 = a11 - a10;
        r.gy = fmaf(wz, y1 - y0, y0);
        const float e0 = fmaf(wy, d01 - d00, d00), e1 = fmaf(wy, d11 - d10, d10);
        r.gx = fmaf(wz, e1 - e0, e0);
    } else {
        r.gx = r.gy = r.gz = 0.0f;
    }
    return r;
}

// The trilinear value (no gradient) through the texture of 2 x 2 (y, z) quads of the extended volume:
// two fetches at integer texel coordinates, columns cx and cx + 1, return the eight neighbours, so the
// value equals trilinear_x's.  Column cx + 1 = n0 lies past the texture only where the position sits
// on the last x plane, whose fraction wx is then 0: the clamped texel is read with weight 0 (the
// derivative along x there needs the extension's column, so the gradient reads the volume itself).
// Neighbouring lanes step along x, so one lane's second column is mostly the next lane's first.
__device__ __forceinline__ float trilinear_qv(unsigned long long tex, long long Ux, long long Uy, long long Uz) {
    constexpr float k2m32 = 2.3283064365386963e-10f;  // 2^-32
    const int cx = (int)(Ux >> 32), cy = (int)(Uy >> 32), cz = (int)(Uz >> 32);
    const float wx = __uint2float_rn((unsigned)Ux) * k2m32, wy = __uint2float_rn((unsigned)Uy) * k2m32,
                wz = __uint2float_rn((unsigned)Uz) * k2m32;
    float v000, v001, v010, v011, v100, v101, v110, v111;  // v[z][y][x] offsets
    asm("tex.3d.v4.f32.s32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
        : "=f"(v000), "=f"(v010), "=f"(v100), "=f"(v110)
        : "l"(tex), "r"(cx), "r"(cy), "r"(cz));
    asm("tex.3d.v4.f32.s32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
        : "=f"(v001), "=f"(v011), "=f"(v101), "=f"(v111)
        : "l"(tex), "r"(cx + 1), "r"(cy), "r"(cz));
    const float d00 = v001 - v000, d01 = v011 - v010, d10 = v101 - v100, d11 = v111 - v110;
    const float a00 = fmaf(wx, d00, v000), a01 = fmaf(wx, d01, v010);
    const float a10 = fmaf(wx, d10, v100), a11 = fmaf(wx, d11, v110);
    const float b0 = fmaf(wy, a01 - a00, a00), b1 = fmaf(wy, a11 - a10, a10);
    return fmaf(wz, b1 - b0, b0);
}

// Overlap interval of one fixed row, exactly: the i in [lo, hi] with
// 0 <= U_a(i) <= (n_a - 1) 2^32 for a = x, y, z, where U_a(i) = A[4a] i +
// A[4a+1] j + A[4a+2] k + A[4a+3] (32.32 integers), and U at i = lo.
struct Clip64 {
    int lo, hi;
    long long u0, u1, u2;
};

__device__ __forceinline__ long long floor_div(long long a, long long b) {
    long long q = a / b;
    if (a % b != 0 && ((a < 0) != (b < 0))) --q;
    return q;
}

__device__ __forceinline__ long long ceil_div(long long a, long long b) { return -floor_div(-a, b); }

__device__ Clip64 clip_row64(const long long *A, long long j, long long k, int nf0, int n0, int n1, int n2) {
    long long lo = 0, hi = nf0 - 1, b[3];
    const int nm[3] = {n0, n1, n2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b[a] = A[4 * a + 1] * j + A[4 * a + 2] * k + A[4 * a + 3];
        const long long st = A[4 * a], umax = (long long)(nm[a] - 1) << 32;
        if (st > 0) {
            lo = max(lo, ceil_div(-b[a], st));
            hi = min(hi, floor_div(umax - b[a], st));
        } else if (st < 0) {
            lo = max(lo, ceil_div(umax - b[a], st));
            hi = min(hi, floor_div(-b[a], st));
        } else if (b[a] < 0 || b[a] > umax) {
            hi = -1;
        }
    }
    Clip64 c;
    c.lo = 1;
    c.hi = 0;
    c.u0 = c.u1 = c.u2 = 0;
    if (lo <= hi) {
        c.lo = (int)lo;
        c.hi = (int)hi;
        c.u0 = b[0] + A[0] * lo;
        c.u1 = b[1] + A[4] * lo;
        c.u2 = b[2] + A[8] * lo;
    }
    return c;
}

// Cubic B-spline weights of the four bins k0-1 .. k0+2 around m~ = k0 + t.
__device__ __forceinline__ void bspline_w(float t, float w[4]) {
    const float s = 1.0f - t, t2 = t * t, t3 = t2 * t, s3 = s * s * s;
    w[0] = s3 * (1.0f / 6.0f);
    w[1] = fmaf(0.5f, t3, 2.0f / 3.0f - t2);
    w[2] = fmaf(0.5f, s3, 2.0f / 3.0f - s * s);
    w[3] = t3 * (1.0f / 6.0f);
}

// beta3'(k - m~) for the same four bins.
__device__ __forceinline__ void bspline_dw(float t, float d[4]) {
    const float s = 1.0f - t;
    d[0] = 0.5f * s * s;
    d[1] = t * fmaf(-1.5f, t, 2.0f);
    d[2] = s * fmaf(1.5f, s, -2.0f);
    d[3] = -0.5f * t * t;
}

// ---------------------------------------------------------------------------
// Forward: soft histogram (unnormalised sums of weights) and overlap count
// ---------------------------------------------------------------------------

// Weights are quantised to 2^-32 with the largest one absorbing the rounding
// residue, so every voxel adds exactly 2^32 (the B-spline partition of unity)
// and the integer sums are exact and independent of the order of the atomics:
// the soft histogram, MI and gradient are bitwise reproducible.  A weight is
// added as its two 16-bit halves into two 32-bit shared words per cell, with
// fire-and-forget atomics (no returned value, so no latency on the voxel's
// path).  A histogram copy sums at most 2^16 voxels, each adding at most once
// to a cell, so neither word can overflow (2^16 x (2^16 - 1) < 2^32); at the
// end the cell's 64-bit count, low + (high << 16) summed over the CTA's
// copies, goes to the global histogram.
constexpr int kParzenMaxVox = 65536;  // also the longest fixed row (MI_MAX_PARZEN_NX)
constexpr int kParzenBankSkew = 7;    // row stride of the forward's shared histogram, mod 32
constexpr bool kParzenFwdTex = true;   // forward gathers through the quad texture (the adjoint loads
                                       // the extended volume's eight neighbours, whose L1 serves it best)
constexpr int kParzenRowsPerStep = 1;  // rows a warp of the forward works on at a time

// Row stride of the shared tables: the least SB >= B + 1 with SB = kParzenBankSkew (mod 32).
__host__ __device__ inline int parzen_stride(int B) { return B + 1 + ((kParzenBankSkew - (B + 1)) % 32 + 32) % 32; }

// Histogram copies per CTA of the forward: with C copies, lane l adds to copy l mod C (copy i starts
// i (2 B SB + 32 / C) words in, so that one cell's copies fall in different banks), which divides by C
// the lanes of a warp that hit one cell in one atomic instruction.  A CTA has 1024 threads (64
// registers each: the whole register file) whatever C is, so an SM keeps 32 warps at every bin count.
// C is the largest power of two up to 8 whose copies take at most 160 KB, or 1: the rest of the SM's
// 256 KB of L1 caches the moving volume's texture gathers (6 copies at 64 bins, 213 KB, made the call
// 29 % slower than 4); so 8 copies up to 45 bins, 4 at 64, 2 at 96, 1 at 128.
constexpr int kParzenFwdMaxCopies = 8;
constexpr int kParzenFwdThreads = 1024;
constexpr int kParzenFwdSmemWords = 160 * 1024 / 4;
__host__ __device__ inline int parzen_copy_offset(int B, int copies) {
    return 2 * B * parzen_stride(B) + (copies > 1 ? 32 / copies : 0);
}
__host__ __device__ inline int parzen_fwd_copies_in(int B, int words) {
    int c = kParzenFwdMaxCopies;
    while (c > 1 && c * parzen_copy_offset(B, c) > words) c >>= 1;
    return c;
}
__host__ inline size_t parzen_fwd_smem(int B, int copies) {
    return (size_t)copies * parzen_copy_offset(B, copies) * sizeof(uint32_t);
}
__host__ inline int parzen_fwd_copies(int B) { return parzen_fwd_copies_in(B, kParzenFwdSmemWords); }

// MULTI: transforms on several pairs (descriptors read from `pairs`); otherwise every transform is on
// the pair P0 passed by value, whose fields stay kernel parameters.  The shared memory (smem_words
// words) is sized for the copies of the largest pair's bins; a transform of a pair with fewer bins
// uses as many copies as fit there.
template <int RPW, bool SAMPLED, bool MULTI>
__global__ void __launch_bounds__(kParzenFwdThreads)
    k_parzen_hist(ParzenPair P0, const ParzenPair *__restrict__ pairs, const int *__restrict__ pair_of,
                  const long long *__restrict__ row_start, int n, const ParzenAffine *__restrict__ aff,
                  long long rows_per_cta, long long total_rows, int Bmax, int smem_words,
                  unsigned long long *__restrict__ ghist, unsigned long long *__restrict__ gcount) {
    // Low-half sums [B x SB], then high-half sums.  The row stride SB >= B + 1 is 7 mod 32, so the
    // bank of cell (fixed bin b, moving bin k) is (k + 7 b) mod 32: the cells of neighbouring voxels,
    // which differ by a bin or two on either axis, fall in different banks.  Column B absorbs the
    // zero weight of bin B (m~ = B - 2 exactly).
    // The rows of all transforms form one sequence (transform t owns rows row_begin(t) ..
    // row_begin(t + 1) - 1, its pair's rows); CTA b takes rows_per_cta of them from b rows_per_cta
    // on, one transform segment at a time, and flushes its histogram after each segment into the
    // transform's slot of Bmax^2 cells (the first B^2 of them, row-major with row stride B).
    extern __shared__ uint32_t sh32[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    __shared__ long long A[12];
    const long long R0 = (long long)P0.nf[1] * P0.nf[2];  // rows per transform of a single pair
    const long long c0 = (long long)blockIdx.x * rows_per_cta;
    const long long c1 = c0 + rows_per_cta < total_rows ? c0 + rows_per_cta : total_rows;
    // a warp works on RPW rows at a time, G = 32 / RPW neighbouring voxels of each: the lanes that
    // add to one cell at once are then at most the G of a row (neighbouring voxels mostly share
    // cells, and same-address shared atomics queue), while each row's gathers stay coalesced
    constexpr int G = 32 / RPW;
    const int sub = lane / G, pos = lane % G;
    // the transform owning row c0
    int t = 0;
    if (MULTI) {
        int lo_t = 0, hi_t = n - 1;
        while (lo_t < hi_t) {  // last t with row_start[t] <= c0
            const int mid = (lo_t + hi_t + 1) >> 1;
            if (row_start[mid] <= c0) lo_t = mid; else hi_t = mid - 1;
        }
        t = lo_t;
    } else {
        t = (int)(c0 / R0);
    }
    bool first = true;
    for (long long s0 = c0; s0 < c1; ++t) {
        const ParzenPair P = MULTI ? pairs[pair_of[t]] : P0;
        const int B = P.B, B2 = B * B, SB = parzen_stride(B), NP = B * SB;
        const int NC = parzen_fwd_copies_in(B, smem_words);  // copies in use
        const int CP = parzen_copy_offset(B, NC);            // offset between copies
        uint32_t *lo16 = sh32 + (lane & (NC - 1)) * CP, *hi16 = lo16 + NP;
        const int nf0 = P.nf[0], nf1 = P.nf[1];
        const int n0 = P.nm[0], n1 = P.nm[1], n2 = P.nm[2];
        const long long R = (long long)nf1 * P.nf[2];
        const long long tb = MULTI ? row_start[t] : (long long)t * R0;
        const float Bm4 = (float)(B - 4);
        const long long r0 = s0 - tb, r1 = c1 - tb < R ? c1 - tb : R;
        if (!first) __syncthreads();  // the previous segment's flush has read the copies
        first = false;
        for (int c = threadIdx.x; c < NC * CP; c += blockDim.x) sh32[c] = 0u;
        if (threadIdx.x < 12) A[threadIdx.x] = aff[t].A[threadIdx.x];
        __syncthreads();
        const long long DG0 = G * A[0], DG1 = G * A[4], DG2 = G * A[8];
        unsigned int cnt = 0;  // overlap voxels counted by this lane
        // one voxel at 32.32 index U with fixed bin bf: its four quantised B-spline weights
        auto add_voxel = [&](long long U0, long long U1, long long U2, int bf) {
            const float mv = kParzenFwdTex ? trilinear_qv(P.texq, U0, U1, U2)
                                           : trilinear_x<false>(P.movx, P.nm[0] + 1, (P.nm[0] + 1) * (P.nm[1] + 1),
                                                                U0, U1, U2).m;
            const float mt = fmaf(fminf(fmaxf(mv, 0.0f), 1.0f), Bm4, 2.0f);
            const int k0 = (int)mt;
            float w[4];
            bspline_w(mt - (float)k0, w);
            // every quantised weight is below 2^32 (at most (2/3) 2^32)
            const uint32_t q0 = __float2uint_rn(w[0] * 4294967296.0f);
            const uint32_t q2 = __float2uint_rn(w[2] * 4294967296.0f);
            const uint32_t q3 = __float2uint_rn(w[3] * 4294967296.0f);
            const uint32_t q1 = 0u - q0 - q2 - q3;  // 2^32 - (q0 + q2 + q3)
            const int c = bf * SB + (k0 - 1);
            atomicAdd(lo16 + c, q0 & 0xffffu);
            atomicAdd(hi16 + c, q0 >> 16);
            atomicAdd(lo16 + c + 1, q1 & 0xffffu);
            atomicAdd(hi16 + c + 1, q1 >> 16);
            atomicAdd(lo16 + c + 2, q2 & 0xffffu);
            atomicAdd(hi16 + c + 2, q2 >> 16);
            atomicAdd(lo16 + c + 3, q3 & 0xffffu);
            atomicAdd(hi16 + c + 3, q3 >> 16);
        };
        // warp w takes rows r0 + w + nwarps n; a group of 32 of them is clipped at once (lane l: row l)
        for (long long g = r0 + warp; g < r1; g += 32LL * nwarps) {
            Clip64 mine;
            mine.lo = 1;
            mine.hi = 0;
            mine.u0 = mine.u1 = mine.u2 = 0;
            const long long rl = g + (long long)nwarps * lane;
            if (rl < r1) mine = clip_row64(A, rl % nf1, rl / nf1, nf0, n0, n1, n2);
            if constexpr (SAMPLED) {  // random sampling: each row's sampled voxels inside its interval
                for (int s = 0; s < 32; ++s) {
                    const long long r = g + (long long)nwarps * s;
                    if (r >= r1) break;  // warp-uniform
                    const int lo = __shfl_sync(kFull, mine.lo, s), hi = __shfl_sync(kFull, mine.hi, s);
                    if (lo > hi) continue;
                    const long long ub0 = __shfl_sync(kFull, mine.u0, s), ub1 = __shfl_sync(kFull, mine.u1, s),
                                    ub2 = __shfl_sync(kFull, mine.u2, s);
                    const uint32_t e0 = __ldg(P.srow + r), e1 = __ldg(P.srow + r + 1);
                    for (uint32_t eb = e0; eb < e1; eb += 32) {
                        const uint32_t e = eb + lane;
                        const int i = e < e1 ? (int)__ldg(P.scol + e) : -1;
                        if (e < e1 && i >= lo && i <= hi) {
                            const long long d = i - lo;
                            add_voxel(ub0 + A[0] * d, ub1 + A[4] * d, ub2 + A[8] * d, (int)__ldg(P.sbin + e));
                            ++cnt;
                        }
                    }
                }
            } else {
                for (int s = 0; s < 32; s += RPW) {
                    if (g + (long long)nwarps * s >= r1) break;  // warp-uniform: the rest of the group is past r1
                    const int src = s + sub;
                    const long long r = g + (long long)nwarps * src;
                    int lo = __shfl_sync(kFull, mine.lo, src), hi = __shfl_sync(kFull, mine.hi, src);
                    if (r >= r1) hi = lo - 1;
                    const int len = hi - lo + 1 > 0 ? hi - lo + 1 : 0;
                    if (pos == 0) cnt += (unsigned)len;
                    const int nsteps = __reduce_max_sync(kFull, (unsigned)((len + G - 1) / G));
                    long long U0 = __shfl_sync(kFull, mine.u0, src) + A[0] * pos;
                    long long U1 = __shfl_sync(kFull, mine.u1, src) + A[4] * pos;
                    long long U2 = __shfl_sync(kFull, mine.u2, src) + A[8] * pos;
                    const uint8_t *__restrict__ frow = P.fbins + (size_t)(r < r1 ? r : r0) * nf0;
                    for (int k = 0; k < nsteps; ++k) {
                        const int i = lo + k * G + pos;
                        if (i <= hi) add_voxel(U0, U1, U2, (int)__ldg(frow + i));
                        U0 += DG0;
                        U1 += DG1;
                        U2 += DG2;
                    }
                }
            }
        }
        cnt = __reduce_add_sync(kFull, cnt);
        __syncthreads();
        unsigned long long *gh = ghist + (size_t)t * Bmax * Bmax;
        for (int c = threadIdx.x; c < B2; c += blockDim.x) {
            const int cp = (c / B) * SB + c % B;
            unsigned long long v = 0;
            for (int i = 0; i < NC; ++i)
                v += (unsigned long long)sh32[i * CP + cp] + ((unsigned long long)sh32[i * CP + NP + cp] << 16);
            if (v) atomicAdd(gh + c, v);
        }
        if (lane == 0 && cnt) atomicAdd(gcount + t, (unsigned long long)cnt);
        s0 = tb + R;  // another transform may follow: its segment starts from empty copies
    }
}

__global__ void k_parzen_quads(const float *__restrict__ movx, int n0, int n1, int n2, float4 *__restrict__ out) {
    const long long m0 = n0 + 1, m01 = m0 * (n1 + 1), n = (long long)n0 * n1 * n2;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const long long x = o % n0, y = (o / n0) % n1, z = o / ((long long)n0 * n1);
        const float *p = movx + x + m0 * y + m01 * z;
        out[o] = make_float4(p[0], p[m0], p[m01], p[m01 + m0]);
    }
}

__global__ void k_parzen_extend(const float *__restrict__ mov, int n0, int n1, int n2, float *__restrict__ out) {
    const long long m0 = n0 + 1, m1 = n1 + 1, n = m0 * m1 * (n2 + 1);
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % m0), y = (int)((o / m0) % m1), z = (int)(o / (m0 * m1));
        // per axis: an index inside the volume, or the linear continuation 2 v[n-1] - v[n-2]
        int xi[2], yi[2], zi[2];
        double xc[2], yc[2], zc[2];
        const int nx = x < n0 ? 1 : 2, ny = y < n1 ? 1 : 2, nz = z < n2 ? 1 : 2;
        xi[0] = x < n0 ? x : n0 - 1, xc[0] = x < n0 ? 1.0 : 2.0, xi[1] = n0 - 2, xc[1] = -1.0;
        yi[0] = y < n1 ? y : n1 - 1, yc[0] = y < n1 ? 1.0 : 2.0, yi[1] = n1 - 2, yc[1] = -1.0;
        zi[0] = z < n2 ? z : n2 - 1, zc[0] = z < n2 ? 1.0 : 2.0, zi[1] = n2 - 2, zc[1] = -1.0;
        double v = 0.0;
        for (int c = 0; c < nz; ++c)
            for (int b = 0; b < ny; ++b)
                for (int a = 0; a < nx; ++a)
                    v += xc[a] * yc[b] * zc[c] * (double)mov[xi[a] + (long long)n0 * (yi[b] + (long long)n1 * zi[c])];
        out[o] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// Entropies and W = dMI/dP in FP64
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// block-wide sum of one double (all threads get the result); s_tmp holds >= 32 doubles
__device__ double block_sum(double v, double *s_tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) s_tmp[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += s_tmp[w];
    return s;
}

// Entropy contribution of one probability p > 0 for exponent q.
__device__ __forceinline__ double ent_term(double p, float qf) {
    return qf == 1.0f ? -p * log(p) : pow(p, (double)qf);
}

__device__ __forceinline__ double finish_entropy(double sum, float qf, int bits) {
    if (qf == 1.0f) return bits ? sum / log(2.0) : sum;
    return (1.0 - sum) / ((double)qf - 1.0);
}

// One CTA per transform: marginals P_F (rows), P_M (cols), their entropies per q, and the row and
// column factors of W per q (mterm: n x nq x 2B): ln P for q = 1, dS_q/dP = -q P^(q-1) / (q - 1)
// otherwise.  marg: n x 2B (P_F then P_M); ment: n x nq x 2 (S_F, S_M).
// B of transform t: its pair's bin count (a multi-pair call), else the single pair's.
__device__ __forceinline__ int bins_of(const ParzenPair *pairs, const int *pair_of, int t) {
    return pairs[pair_of ? pair_of[t] : 0].B;
}

__global__ void k_parzen_marg(const unsigned long long *__restrict__ ghist, const unsigned long long *__restrict__ gcount,
                              const ParzenPair *__restrict__ pairs, const int *__restrict__ pair_of, int Bmax, QSet Q,
                              double *__restrict__ marg, double *__restrict__ ment, double *__restrict__ mterm) {
    __shared__ double s_tmp[32];
    const int t = blockIdx.x;
    const int B = bins_of(pairs, pair_of, t);
    const double N = (double)gcount[t] * 4294967296.0;  // total weight: 2^32 per overlap voxel
    const unsigned long long *h = ghist + (size_t)t * Bmax * Bmax;
    double *pf = marg + (size_t)t * 2 * Bmax, *pm = pf + B;
    for (int r = threadIdx.x; r < B; r += blockDim.x) {
        unsigned long long sr = 0, sc = 0;
        for (int c = 0; c < B; ++c) {
            sr += h[(size_t)r * B + c];
            sc += h[(size_t)c * B + r];
        }
        pf[r] = N > 0 ? (double)sr / N : 0.0;
        pm[r] = N > 0 ? (double)sc / N : 0.0;
    }
    __syncthreads();
    for (int iq = 0; iq < Q.nq; ++iq) {
        const float qf = Q.q[iq];
        const double q = (double)qf;
        double *mt = mterm + ((size_t)t * Q.nq + iq) * 2 * Bmax;
        double a = 0.0, b = 0.0;
        for (int r = threadIdx.x; r < B; r += blockDim.x) {
            if (pf[r] > 0.0) a += ent_term(pf[r], qf);
            if (pm[r] > 0.0) b += ent_term(pm[r], qf);
            for (int h = 0; h < 2; ++h) {
                const double v = h ? pm[r] : pf[r];
                mt[h * B + r] = !(v > 0.0) ? 0.0 : qf == 1.0f ? log(v) : -q * pow(v, q - 1.0) / (q - 1.0);
            }
        }
        a = block_sum(a, s_tmp);
        b = block_sum(b, s_tmp);
        if (threadIdx.x == 0) {
            ment[((size_t)t * Q.nq + iq) * 2 + 0] = finish_entropy(a, Q.q[iq], Q.bits);
            ment[((size_t)t * Q.nq + iq) * 2 + 1] = finish_entropy(b, Q.q[iq], Q.bits);
        }
    }
}

// Grid (cells / 256, n): per-block joint entropy partial sums (jpart: n x nq x
// gridDim.x, reduced in a fixed order later) and W (n x nq x B^2, FP32).  One
// ln p per cell serves every q: the Shannon term -p ln p, p^q = exp(q ln p)
// for the Tsallis ones, and dS_q/dp = -q p^q / (p (q - 1)).
__global__ void __launch_bounds__(256)
    k_parzen_cells(const unsigned long long *__restrict__ ghist, const unsigned long long *__restrict__ gcount,
                   const ParzenPair *__restrict__ pairs, const int *__restrict__ pair_of, int Bmax, QSet Q,
                   const double *__restrict__ mterm, const double *__restrict__ ment, double *__restrict__ jpart,
                   float *__restrict__ wout) {
    __shared__ double s_tmp[32];
    const int t = blockIdx.y;
    const int B = bins_of(pairs, pair_of, t), B2 = B * B, BM2 = Bmax * Bmax;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double N = (double)gcount[t] * 4294967296.0;
    const double lnb = Q.bits ? log(2.0) : 1.0;
    double p = 0.0, lp = 0.0;
    if (c < B2 && N > 0) {
        p = (double)ghist[(size_t)t * BM2 + c] / N;
        if (p > 0.0) lp = log(p);
    }
    for (int iq = 0; iq < Q.nq; ++iq) {
        const float qf = Q.q[iq];
        const double q = (double)qf;
        const double pq = p > 0.0 && qf != 1.0f ? exp(q * lp) : 0.0;
        double e = p > 0.0 ? (qf == 1.0f ? -p * lp : pq) : 0.0;
        e = block_sum(e, s_tmp);
        if (threadIdx.x == 0) jpart[((size_t)t * Q.nq + iq) * gridDim.x + blockIdx.x] = e;
        if (c < B2) {
            double w = 0.0;
            if (p > 0.0) {
                const double *mt = mterm + ((size_t)t * Q.nq + iq) * 2 * Bmax;
                const double fr = mt[c / B], mc = mt[B + c % B];
                if (qf == 1.0f) {
                    w = (lp - fr - mc - 1.0) / lnb;
                } else {
                    const double dSJ = -q * pq / (p * (q - 1.0));
                    w = fr + mc - dSJ;
                    if (Q.form == 1) {
                        const double SF = ment[((size_t)t * Q.nq + iq) * 2 + 0];
                        const double SM = ment[((size_t)t * Q.nq + iq) * 2 + 1];
                        w += (1.0 - q) * (fr * SM + SF * mc);
                    }
                }
            }
            wout[((size_t)t * Q.nq + iq) * BM2 + c] = (float)w;
        }
    }
}

// MI per q: S_F + S_M - S_FM (+ (1 - q) S_F S_M for the pseudo-additive form).
__global__ void k_parzen_final(int n, const unsigned long long *__restrict__ gcount, QSet Q,
                               const double *__restrict__ ment, const double *__restrict__ jpart, int nparts,
                               double *__restrict__ mi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n * Q.nq) return;
    double js = 0.0;
    for (int b = 0; b < nparts; ++b) js += jpart[(size_t)x * nparts + b];
    const int t = x / Q.nq, iq = x % Q.nq;
    if (gcount[t] == 0) {
        mi[x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const float qf = Q.q[iq];
    const double SF = ment[(size_t)x * 2 + 0], SM = ment[(size_t)x * 2 + 1];
    const double SJ = finish_entropy(js, qf, Q.bits);
    double I = SF + SM - SJ;
    if (qf != 1.0f && Q.form == 1) I += (1.0 - (double)qf) * SF * SM;
    mi[x] = I;
}

// ---------------------------------------------------------------------------
// Adjoint: moments M[q][a][c] = sum_x s_q(x) d_a m(u_x) x_c, x = (i - ci, j - cj, k - ck, 1)
// ---------------------------------------------------------------------------

// Where an adjoint launch keeps the W table of its q values: in the shared memory of one 512-thread
// CTA an SM when it fits, else in global memory read by 256-thread CTAs (two an SM).  Either gives 16
// warps an SM at 128 registers a thread; the larger CTA measured 4 % faster at 64 bins (fewer, larger
// row shares), and one float a cell 1.5 % faster than (W[k], W[k + 1]) pairs read as two 8-byte words.
enum { kWGlobal = 0, kWShared = 1 };

template <int NQ, bool SAMPLED, bool MULTI, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB)
    k_parzen_adj(ParzenPair P0, const ParzenPair *__restrict__ pairs, const int *__restrict__ pair_of, int Bmax,
                 const ParzenAffine *__restrict__ aff, int nq_total, int q0, const float *__restrict__ wtab,
                 int w_mode, double *__restrict__ mom) {
    // mom: n x nq_total x gridDim.x x 12 per-CTA partial moments (no atomics: fixed-order reduction later)
    // NQ x B x SB weights in shared memory (w_mode kWShared); the row stride SB >= B + 1 is 7 mod 32, so
    // neighbouring voxels' cells, a bin or two apart on either axis, are read from different banks.
    // W of transform t is its slot of Bmax^2 entries per q (the first B^2 used, row stride B).
    extern __shared__ float sw[];
    const int t = blockIdx.y;
    const ParzenPair P = MULTI ? pairs[pair_of[t]] : P0;
    const int B = P.B, SB = parzen_stride(B);
    __shared__ long long A[12];
    __shared__ float s_red[TPB / 32][NQ * 12];
    if (threadIdx.x < 12) A[threadIdx.x] = aff[t].A[threadIdx.x];
    const size_t BM2 = (size_t)Bmax * Bmax;
    const float *W = wtab + ((size_t)t * nq_total + q0) * BM2;
    int RS = B, QS = (int)BM2;  // row stride and per-q stride of the table in use
    if (w_mode == kWShared) {
        for (int c = threadIdx.x; c < NQ * B * B; c += blockDim.x) {
            const int qq = c / (B * B), cc = c % (B * B);
            sw[qq * B * SB + (cc / B) * SB + cc % B] = W[(size_t)qq * BM2 + cc];
        }
        RS = SB;
        QS = B * SB;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const int n0 = P.nm[0], n1 = P.nm[1], n2 = P.nm[2];
    const long long R = (long long)nf1 * P.nf[2];
    const float Bm4 = (float)(B - 4);
    const long long D0 = 32 * A[0], D1 = 32 * A[4], D2 = 32 * A[8];
    // moments are taken about the fixed-volume centre, where the rotation and
    // scale columns of du/dtheta have no constant part (no cancellation)
    const float ci = 0.5f * (float)(nf0 - 1), cj = 0.5f * (float)(nf1 - 1), ck = 0.5f * (float)(P.nf[2] - 1);
    float M[NQ][12];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int e = 0; e < 12; ++e) M[q][e] = 0.0f;
    // warp w of CTA b takes rows (b nwarps + w) + gridDim.x nwarps n; a group of 32 is clipped at once
    const long long rstep = (long long)gridDim.x * nwarps;
    for (long long g = (long long)blockIdx.x * nwarps + warp; g < R; g += 32 * rstep) {
        Clip64 mine;
        mine.lo = 1;
        mine.hi = 0;
        mine.u0 = mine.u1 = mine.u2 = 0;
        const long long rl = g + rstep * lane;
        if (rl < R) mine = clip_row64(A, rl % nf1, rl / nf1, nf0, n0, n1, n2);
        for (int s = 0; s < 32; ++s) {
            const long long r = g + rstep * s;
            if (r >= R) break;  // warp-uniform
            const int lo = __shfl_sync(kFull, mine.lo, s), hi = __shfl_sync(kFull, mine.hi, s);
            if (lo > hi) continue;
            long long U0 = __shfl_sync(kFull, mine.u0, s) + A[0] * lane;
            long long U1 = __shfl_sync(kFull, mine.u1, s) + A[4] * lane;
            long long U2 = __shfl_sync(kFull, mine.u2, s) + A[8] * lane;
            const float j = (float)(r % nf1) - cj, k = (float)(r / nf1) - ck;
            const uint8_t *__restrict__ frow = P.fbins + (size_t)r * nf0;
            // along the row j and k are constant: per row, S0[q][a] = sum s d_a m, and the moments in
            // j, k and 1 follow from it at the row's end; sum s d_a m (i - ci) goes to M directly
            float S0[NQ][3];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int a = 0; a < 3; ++a) S0[q][a] = 0.0f;
            // one voxel (x index i, fixed bin bf) at 32.32 index U: its share of S0 and M
            auto acc_voxel = [&](long long V0, long long V1, long long V2, int i, int bf) {
                const MG g3 = trilinear_x<true>(P.movx, P.nm[0] + 1, (P.nm[0] + 1) * (P.nm[1] + 1), V0, V1, V2);
                const float ic = (float)i - ci;
                // d_a m and d_a m (i - ci), shared by every q
                const float hx = g3.gx * ic, hy = g3.gy * ic, hz = g3.gz * ic;
                const float mt = fmaf(fminf(fmaxf(g3.m, 0.0f), 1.0f), Bm4, 2.0f);
                const int k0 = (int)mt;
                float d[4];
                bspline_dw(mt - (float)k0, d);
                if (k0 + 2 >= B) d[3] = 0.0f;
                const int cb = bf * RS + (k0 - 1);
                const int i3 = k0 + 2 < B ? cb + 3 : cb;  // in range; weight 0 when clamped
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    float sv;
                    if (w_mode == kWShared) {
                        const float *Wq = sw + (size_t)q * QS;
                        sv = Wq[cb] * d[0] + Wq[cb + 1] * d[1] + Wq[cb + 2] * d[2] + Wq[i3] * d[3];
                    } else {
                        const float *Wq = W + (size_t)q * QS;
                        sv = Wq[cb] * d[0] + Wq[cb + 1] * d[1] + Wq[cb + 2] * d[2] + Wq[i3] * d[3];
                    }
                    M[q][0] = fmaf(sv, hx, M[q][0]);
                    S0[q][0] = fmaf(sv, g3.gx, S0[q][0]);
                    M[q][4] = fmaf(sv, hy, M[q][4]);
                    S0[q][1] = fmaf(sv, g3.gy, S0[q][1]);
                    M[q][8] = fmaf(sv, hz, M[q][8]);
                    S0[q][2] = fmaf(sv, g3.gz, S0[q][2]);
                }
            };
            if constexpr (SAMPLED) {  // random sampling: the row's sampled voxels inside [lo, hi]
                const long long ub0 = U0 - A[0] * lane, ub1 = U1 - A[4] * lane, ub2 = U2 - A[8] * lane;
                const uint32_t e0 = __ldg(P.srow + r), e1 = __ldg(P.srow + r + 1);
                for (uint32_t eb = e0; eb < e1; eb += 32) {
                    const uint32_t e = eb + lane;
                    const int i = e < e1 ? (int)__ldg(P.scol + e) : -1;
                    if (e < e1 && i >= lo && i <= hi) {
                        const long long dd = i - lo;
                        acc_voxel(ub0 + A[0] * dd, ub1 + A[4] * dd, ub2 + A[8] * dd, i, (int)__ldg(P.sbin + e));
                    }
                }
            } else {
                for (int base = lo; base <= hi; base += 32) {
                    const int i = base + lane;
                    if (i <= hi) acc_voxel(U0, U1, U2, i, (int)__ldg(frow + i));
                    U0 += D0;
                    U1 += D1;
                    U2 += D2;
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    M[q][4 * a + 1] = fmaf(S0[q][a], j, M[q][4 * a + 1]);
                    M[q][4 * a + 2] = fmaf(S0[q][a], k, M[q][4 * a + 2]);
                    M[q][4 * a + 3] += S0[q][a];
                }
        }
    }
    // warp reduction in FP32, then the 8 warps in FP64 into global memory
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int e = 0; e < 12; ++e) {
            float v = M[q][e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0) s_red[warp][q * 12 + e] = v;
        }
    __syncthreads();
    if (threadIdx.x < NQ * 12) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += (double)s_red[w][threadIdx.x];
        const int q = threadIdx.x / 12, e = threadIdx.x % 12;
        mom[(((size_t)t * nq_total + q0 + q) * gridDim.x + blockIdx.x) * 12 + e] = s;
    }
}

// grad[t][q][p] = -(B - 4) / N sum_e mom[t][q][e] J[t][e][p], J (12 x np) taken about the fixed centre
__global__ void k_parzen_grad(int n, int nq, int np, const ParzenPair *__restrict__ pairs,
                              const int *__restrict__ pair_of, int nparts, const unsigned long long *__restrict__ gcount,
                              const double *__restrict__ mom, const double *__restrict__ jac, double *__restrict__ grad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n * nq * np) return;
    const int p = x % np, tq = x / np, t = tq / nq;
    const int B = bins_of(pairs, pair_of, t);
    const double N = (double)gcount[t];
    if (N <= 0) {
        grad[x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double s = 0.0;
    for (int e = 0; e < 12; ++e) {
        double me = 0.0;
        for (int b = 0; b < nparts; ++b) me += mom[((size_t)tq * nparts + b) * 12 + e];
        s += me * jac[((size_t)t * 12 + e) * np + p];
    }
    grad[x] = -(double)(B - 4) / N * s;
}

}  // namespace

cudaError_t launch_parzen_prep_fixed(const void *data, int dtype, int depth, long long n, int B, uint8_t *out,
                                     cudaStream_t s) {
    if (dtype == 0)
        k_pfix_int<uint8_t><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)data, n, depth, B, out);
    else if (dtype == 1)
        k_pfix_int<uint16_t><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)data, n, depth, B, out);
    else
        k_pfix_f32<<<grid_for(n, 256), 256, 0, s>>>((const float *)data, n, B, out);
    return cudaGetLastError();
}

cudaError_t launch_parzen_prep_moving(const void *data, int dtype, int depth, long long n, float *out, cudaStream_t s) {
    if (dtype == 0)
        k_pmov_int<uint8_t><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)data, n, depth, out);
    else if (dtype == 1)
        k_pmov_int<uint16_t><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)data, n, depth, out);
    else
        k_pmov_f32<<<grid_for(n, 256), 256, 0, s>>>((const float *)data, n, out);
    return cudaGetLastError();
}

int parzen_ctas(const ParzenPair &P, int n, int sms) {
    const long long rows = (long long)P.nf[1] * P.nf[2];
    // about 4 CTAs per SM over all transforms, at least one row batch of 8 warps each
    long long per_t = (4LL * sms + n - 1) / n;
    long long max_rows = (rows + 7) / 8;
    if (per_t > max_rows) per_t = max_rows;
    if (per_t < 1) per_t = 1;
    return (int)per_t;
}

// W table of an adjoint launch over g q values at B bins: in shared memory when it fits beside the
// CTA's 3 KB of static shared memory (every B at up to three q, B <= 96 at four), else global memory.
static int parzen_adj_wmode(int B, int g) {
    return (size_t)g * B * parzen_stride(B) * sizeof(float) <= 220 * 1024 ? kWShared : kWGlobal;
}
static size_t parzen_adj_smem(int B, int g) {
    return parzen_adj_wmode(B, g) == kWShared ? (size_t)g * B * parzen_stride(B) * sizeof(float) : 0;
}
static int parzen_adj_threads(int B, int g) { return parzen_adj_wmode(B, g) == kWShared ? 512 : 256; }

template <int NQ, bool SAMPLED>
static int adj_blocks_per_sm(size_t smem, int tpb) {
    const void *fn = tpb == 512 ? (const void *)k_parzen_adj<NQ, SAMPLED, false, 512>
                                : (const void *)k_parzen_adj<NQ, SAMPLED, false, 256>;
    if (allow_smem(fn, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return resident_per_sm(fn, tpb, smem);
}

int parzen_adj_ctas(const ParzenPair &P, int n, int nq, int sms) {
    // every CTA of the adjoint does about the same work, so the grid is cut to whole waves of the
    // CTAs that fit at once (those of the first q group's instance): the nearest whole number of
    // waves to the usual ~4 CTAs per SM, then the most CTAs per transform that fill it
    const int g = nq < 4 ? nq : 4;
    const size_t smem = parzen_adj_smem(P.B, g);
    const int tpb = parzen_adj_threads(P.B, g);
    int per_sm = 1;
    switch (g) {
        case 1: per_sm = P.srow ? adj_blocks_per_sm<1, true>(smem, tpb) : adj_blocks_per_sm<1, false>(smem, tpb); break;
        case 2: per_sm = P.srow ? adj_blocks_per_sm<2, true>(smem, tpb) : adj_blocks_per_sm<2, false>(smem, tpb); break;
        case 3: per_sm = P.srow ? adj_blocks_per_sm<3, true>(smem, tpb) : adj_blocks_per_sm<3, false>(smem, tpb); break;
        default: per_sm = P.srow ? adj_blocks_per_sm<4, true>(smem, tpb) : adj_blocks_per_sm<4, false>(smem, tpb);
    }
    const long long cap = (long long)per_sm * sms, c0 = parzen_ctas(P, n, sms);
    long long waves = ((long long)n * c0 + cap / 2) / cap;
    if (waves < 1) waves = 1;
    long long c = waves * cap / n;
    const long long max_c = ((long long)P.nf[1] * P.nf[2] + tpb / 32 - 1) / (tpb / 32);  // a row per warp
    if (c > max_c) c = max_c;
    if (c < 1) c = 1;
    return (int)c;
}

int parzen_cell_blocks(int B) { return (B * B + 255) / 256; }

cudaError_t launch_parzen_extend(const float *mov, const int nm[3], float *out, cudaStream_t s) {
    const long long n = (long long)(nm[0] + 1) * (nm[1] + 1) * (nm[2] + 1);
    k_parzen_extend<<<grid_for(n, 256), 256, 0, s>>>(mov, nm[0], nm[1], nm[2], out);
    return cudaGetLastError();
}

cudaError_t launch_parzen_quads(const float *movx, const int nm[3], void *out, cudaStream_t s) {
    const long long n = (long long)nm[0] * nm[1] * nm[2];
    k_parzen_quads<<<grid_for(n, 256), 256, 0, s>>>(movx, nm[0], nm[1], nm[2], (float4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_parzen_hist(const ParzenLaunch &L, const ParzenAffine *d_aff, int sms, unsigned long long *d_hist,
                               unsigned long long *d_count, cudaStream_t s) {
    const int n = L.n;
    if (n <= 0) return cudaSuccess;
    const size_t BM2 = (size_t)L.Bmax * L.Bmax;
    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)n * BM2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_count, 0, (size_t)n * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    // shared memory for the largest pair's bins (a smaller pair's copies fit in the same space)
    const int copies = parzen_fwd_copies(L.Bmax);
    const size_t smem = parzen_fwd_smem(L.Bmax, copies);
    const bool multi = L.d_pair_of != nullptr;
    const void *fn = multi ? (L.sampled ? (const void *)k_parzen_hist<kParzenRowsPerStep, true, true>
                                        : (const void *)k_parzen_hist<kParzenRowsPerStep, false, true>)
                           : (L.sampled ? (const void *)k_parzen_hist<kParzenRowsPerStep, true, false>
                                        : (const void *)k_parzen_hist<kParzenRowsPerStep, false, false>);
    if ((e = allow_smem(fn, smem)) != cudaSuccess) return e;
    // rows per CTA: at most kParzenMaxVox voxels per copy, so that the 16-bit halves cannot overflow
    // (a row of nx voxels, or of at most nx sampled entries, is walked 32 lanes at a time, so copy i,
    // fed by the lanes l = i mod C, takes at most 32 / C of every 32; the longest row of all
    // pairs bounds it, and a pair with fewer bins than the largest uses at least C copies); CTAs do
    // equal shares of the rows of all transforms, as many as fill a whole number of waves of the CTAs
    // resident at once
    const long long TR = L.total_rows;
    long long cap = kParzenMaxVox / ((32 / copies) * ((L.nx_max + 31) / 32));
    if (cap < 1) cap = 1;
    const int per_sm = resident_per_sm(fn, kParzenFwdThreads, smem);
    const long long wave = (long long)per_sm * (sms > 0 ? sms : 1);
    long long nch = (TR + cap - 1) / cap;
    nch = (nch + wave - 1) / wave * wave;
    if (nch > TR) nch = TR;
    long long rpc = (TR + nch - 1) / nch, total = TR;
    dim3 grid((unsigned)((TR + rpc - 1) / rpc));
    int nn = n, bmax = L.Bmax, words = (int)(smem / sizeof(uint32_t));
    void *args[] = {(void *)&L.p0,  (void *)&L.d_pairs, (void *)&L.d_pair_of, (void *)&L.d_row_start,
                    (void *)&nn,    (void *)&d_aff,     (void *)&rpc,         (void *)&total,
                    (void *)&bmax,  (void *)&words,     (void *)&d_hist,      (void *)&d_count};
    return cudaLaunchKernel(fn, grid, dim3(kParzenFwdThreads), args, smem, s);
}

cudaError_t launch_parzen_weights(const unsigned long long *d_hist, const unsigned long long *d_count,
                                  const ParzenLaunch &L, const QSet &Q, double *marg, double *ment, double *mterm,
                                  double *jpart, double *d_mi, float *d_w, cudaStream_t s) {
    cudaError_t e;
    const int n = L.n;
    k_parzen_marg<<<n, 256, 0, s>>>(d_hist, d_count, L.d_pairs, L.d_pair_of, L.Bmax, Q, marg, ment, mterm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nb = parzen_cell_blocks(L.Bmax);
    dim3 grid(nb, n);
    k_parzen_cells<<<grid, 256, 0, s>>>(d_hist, d_count, L.d_pairs, L.d_pair_of, L.Bmax, Q, mterm, ment, jpart, d_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_parzen_final<<<(n * Q.nq + 127) / 128, 128, 0, s>>>(n, d_count, Q, ment, jpart, nb, d_mi);
    return cudaGetLastError();
}

cudaError_t launch_parzen_adjoint(const ParzenLaunch &L, const ParzenAffine *d_aff, const double *d_jac, int np, int nq,
                                  int ctas, const float *d_w, const unsigned long long *d_count, double *d_mom,
                                  double *d_grad, cudaStream_t s) {
    cudaError_t e;
    const int n = L.n;
    dim3 grid(ctas, n);
    for (int q0 = 0; q0 < nq; q0 += 4) {
        const int g = nq - q0 < 4 ? nq - q0 : 4;
        const size_t smem = parzen_adj_smem(L.Bmax, g);
        const int wmode = parzen_adj_wmode(L.Bmax, g), tpb = parzen_adj_threads(L.Bmax, g);
#define MI_ADJ_T(NQV, SV, MV, TV)                                                                              \
    do {                                                                                                       \
        if ((e = allow_smem((const void *)k_parzen_adj<NQV, SV, MV, TV>, smem)) != cudaSuccess) return e;      \
        k_parzen_adj<NQV, SV, MV, TV><<<grid, TV, smem, s>>>(L.p0, L.d_pairs, L.d_pair_of, L.Bmax, d_aff, nq, q0, \
                                                             d_w, wmode, d_mom);                               \
    } while (0)
#define MI_ADJ_S(NQV, SV, MV)            \
    do {                                 \
        if (tpb == 512)                  \
            MI_ADJ_T(NQV, SV, MV, 512);  \
        else                             \
            MI_ADJ_T(NQV, SV, MV, 256);  \
    } while (0)
#define MI_ADJ(NQV)                              \
    do {                                         \
        if (L.d_pair_of) {                       \
            if (L.sampled)                       \
                MI_ADJ_S(NQV, true, true);       \
            else                                 \
                MI_ADJ_S(NQV, false, true);      \
        } else {                                 \
            if (L.sampled)                       \
                MI_ADJ_S(NQV, true, false);      \
            else                                 \
                MI_ADJ_S(NQV, false, false);     \
        }                                        \
    } while (0)
        switch (g) {
            case 1: MI_ADJ(1); break;
            case 2: MI_ADJ(2); break;
            case 3: MI_ADJ(3); break;
            default: MI_ADJ(4); break;
        }
#undef MI_ADJ
#undef MI_ADJ_S
#undef MI_ADJ_T
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_parzen_grad<<<(n * nq * np + 127) / 128, 128, 0, s>>>(n, nq, np, L.d_pairs, L.d_pair_of, ctas, d_count, d_mom,
                                                            d_jac, d_grad);
    return cudaGetLastError();
}

}  // namespace mi
