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

#include "mi_internal.h"

namespace mi {
namespace {

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

// FP32 trilinear value and gradient (w.r.t. the moving index) at u inside
// [0, n-1]^3; cell c = min(floor(u), n - 2), weight u - c.
struct MG {
    float m, gx, gy, gz;
};

// Cell and weight of a 32.32 fixed-point coordinate U in [0, (n - 1) 2^32].
__device__ __forceinline__ int cell_of(long long U, int n, float &w) {
    const int c = min((int)(U >> 32), n - 2);
    w = (float)(U - ((long long)c << 32)) * 2.3283064365386963e-10f;  // 2^-32
    return c;
}

template <bool GRAD>
__device__ __forceinline__ MG trilinear(const float *__restrict__ mov, int n0, int n1, int n2, long long Ux,
                                        long long Uy, long long Uz) {
    float wx, wy, wz;
    const int cx = cell_of(Ux, n0, wx), cy = cell_of(Uy, n1, wy), cz = cell_of(Uz, n2, wz);
    const int sy = n0, sz = n0 * n1;
    const float *p = mov + (cx + n0 * (cy + n1 * cz));
    const float v000 = __ldg(p), v001 = __ldg(p + 1), v010 = __ldg(p + sy), v011 = __ldg(p + sy + 1);
    const float v100 = __ldg(p + sz), v101 = __ldg(p + sz + 1), v110 = __ldg(p + sz + sy), v111 = __ldg(p + sz + sy + 1);
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

__device__ __forceinline__ bool inside_u(long long Ux, long long Uy, long long Uz, int n0, int n1, int n2) {
    return Ux >= 0 && Uy >= 0 && Uz >= 0 && Ux <= ((long long)(n0 - 1) << 32) && Uy <= ((long long)(n1 - 1) << 32) &&
           Uz <= ((long long)(n2 - 1) << 32);
}

// ---------------------------------------------------------------------------
// Forward: soft histogram (unnormalised sums of weights) and overlap count
// ---------------------------------------------------------------------------

// Weights are quantised to 2^-32 with the largest one absorbing the rounding
// residue, so every voxel adds exactly 2^32 (the B-spline partition of unity)
// and the integer sums are exact and independent of the order of the atomics:
// the soft histogram, MI and gradient are bitwise reproducible.  Each shared
// cell is a 64-bit count kept as two 32-bit words (64-bit shared atomics are
// several times slower): a weight (< 2^32) is added to the low word, and the
// add that wraps it -- detected exactly once, from the returned old value --
// adds 1 to the high word.
__device__ __forceinline__ void add64(uint32_t *lo, uint32_t *hi, int c, uint32_t w) {
    const uint32_t old = atomicAdd(lo + c, w);
    if (old + w < old) atomicAdd(hi + c, 1u);
}

__global__ void __launch_bounds__(256)
    k_parzen_hist(ParzenPair P, const ParzenAffine *__restrict__ aff, unsigned long long *__restrict__ ghist,
                  unsigned long long *__restrict__ gcount) {
    // low words [B x (B + 1)], then high words: rows padded by one word so the
    // bank is (fixed bin + moving bin) mod 32 rather than the moving bin alone
    extern __shared__ uint32_t sh32[];
    const int t = blockIdx.y, B = P.B, B2 = B * B, SB = B + 1, NP = B * SB;
    uint32_t *lo = sh32, *hi = sh32 + NP;
    __shared__ long long A[12];
    if (threadIdx.x < 12) A[threadIdx.x] = aff[t].A[threadIdx.x];
    for (int c = threadIdx.x; c < 2 * NP; c += blockDim.x) sh32[c] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const int n0 = P.nm[0], n1 = P.nm[1], n2 = P.nm[2];
    const long long R = (long long)nf1 * P.nf[2];
    const float Bm4 = (float)(B - 4);
    unsigned int cnt = 0;
    for (long long r = (long long)blockIdx.x * nwarps + warp; r < R; r += (long long)gridDim.x * nwarps) {
        const long long j = r % nf1, k = r / nf1;
        const long long b0 = A[1] * j + A[2] * k + A[3];
        const long long b1 = A[5] * j + A[6] * k + A[7];
        const long long b2 = A[9] * j + A[10] * k + A[11];
        const uint8_t *__restrict__ frow = P.fbins + (size_t)r * nf0;
        for (int i = lane; i < nf0; i += 32) {
            const long long ux = b0 + A[0] * i, uy = b1 + A[4] * i, uz = b2 + A[8] * i;
            if (!inside_u(ux, uy, uz, n0, n1, n2)) continue;
            ++cnt;
            const MG g = trilinear<false>(P.mov, n0, n1, n2, ux, uy, uz);
            const float mt = fmaf(fminf(fmaxf(g.m, 0.0f), 1.0f), Bm4, 2.0f);
            const int k0 = (int)mt;
            float w[4];
            bspline_w(mt - (float)k0, w);
            // every quantised weight is at most (2/3) 2^32, so it fits the 32-bit low word
            const uint32_t q0 = (uint32_t)__float2ull_rn(w[0] * 4294967296.0f);
            const uint32_t q2 = (uint32_t)__float2ull_rn(w[2] * 4294967296.0f);
            const uint32_t q3 = (uint32_t)__float2ull_rn(w[3] * 4294967296.0f);
            const uint32_t q1 = (uint32_t)(4294967296ull - q0 - q2 - q3);
            const int c = (int)__ldg(frow + i) * SB + (k0 - 1);
            add64(lo, hi, c + 0, q0);
            add64(lo, hi, c + 1, q1);
            add64(lo, hi, c + 2, q2);
            if (q3) add64(lo, hi, c + 3, q3);  // q3 == 0 whenever k0 + 3 > B (t = 0 there)
        }
    }
    __syncthreads();
    unsigned long long *gh = ghist + (size_t)t * B2;
    for (int c = threadIdx.x; c < B2; c += blockDim.x) {
        const int cp = (c / B) * SB + c % B;
        const unsigned long long v = ((unsigned long long)hi[cp] << 32) | lo[cp];
        if (v) atomicAdd(gh + c, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0 && cnt) atomicAdd(gcount + t, (unsigned long long)cnt);
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

// One CTA per transform: marginals P_F (rows), P_M (cols) and their entropies per q.
// marg: n x 2B (P_F then P_M); ment: n x nq x 2 (S_F, S_M).
__global__ void k_parzen_marg(const unsigned long long *__restrict__ ghist, const unsigned long long *__restrict__ gcount,
                              int B, QSet Q, double *__restrict__ marg, double *__restrict__ ment) {
    __shared__ double s_tmp[32];
    const int t = blockIdx.x;
    const double N = (double)gcount[t] * 4294967296.0;  // total weight: 2^32 per overlap voxel
    const unsigned long long *h = ghist + (size_t)t * B * B;
    double *pf = marg + (size_t)t * 2 * B, *pm = pf + B;
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
        double a = 0.0, b = 0.0;
        for (int r = threadIdx.x; r < B; r += blockDim.x) {
            if (pf[r] > 0.0) a += ent_term(pf[r], Q.q[iq]);
            if (pm[r] > 0.0) b += ent_term(pm[r], Q.q[iq]);
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
// gridDim.x, reduced in a fixed order later) and W (n x nq x B^2, FP32).
__global__ void __launch_bounds__(256)
    k_parzen_cells(const unsigned long long *__restrict__ ghist, const unsigned long long *__restrict__ gcount, int B,
                   QSet Q, const double *__restrict__ marg, const double *__restrict__ ment, double *__restrict__ jpart,
                   float *__restrict__ wout) {
    __shared__ double s_tmp[32];
    const int t = blockIdx.y, B2 = B * B;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const double N = (double)gcount[t] * 4294967296.0;
    const double lnb = Q.bits ? log(2.0) : 1.0;
    double p = 0.0, pfr = 0.0, pmc = 0.0;
    if (c < B2 && N > 0) {
        p = (double)ghist[(size_t)t * B2 + c] / N;
        pfr = marg[(size_t)t * 2 * B + c / B];
        pmc = marg[(size_t)t * 2 * B + B + c % B];
    }
    for (int iq = 0; iq < Q.nq; ++iq) {
        const float qf = Q.q[iq];
        double e = p > 0.0 ? ent_term(p, qf) : 0.0;
        e = block_sum(e, s_tmp);
        if (threadIdx.x == 0) jpart[((size_t)t * Q.nq + iq) * gridDim.x + blockIdx.x] = e;
        if (c < B2) {
            double w = 0.0;
            if (p > 0.0) {
                if (qf == 1.0f) {
                    w = (log(p) - log(pfr) - log(pmc) - 1.0) / lnb;
                } else {
                    const double q = (double)qf;
                    const double dSF = -q * pow(pfr, q - 1.0) / (q - 1.0);
                    const double dSM = -q * pow(pmc, q - 1.0) / (q - 1.0);
                    const double dSJ = -q * pow(p, q - 1.0) / (q - 1.0);
                    w = dSF + dSM - dSJ;
                    if (Q.form == 1) {
                        const double SF = ment[((size_t)t * Q.nq + iq) * 2 + 0];
                        const double SM = ment[((size_t)t * Q.nq + iq) * 2 + 1];
                        w += (1.0 - q) * (dSF * SM + SF * dSM);
                    }
                }
            }
            wout[((size_t)t * Q.nq + iq) * B2 + c] = (float)w;
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

template <int NQ>
__global__ void __launch_bounds__(256)
    k_parzen_adj(ParzenPair P, const ParzenAffine *__restrict__ aff, int nq_total, int q0,
                 const float *__restrict__ wtab, int w_in_smem, double *__restrict__ mom) {
    // mom: n x nq_total x gridDim.x x 12 per-CTA partial moments (no atomics: fixed-order reduction later)
    extern __shared__ float sw[];  // NQ x B x (B + 1) weights (rows padded by one word) when they fit
    const int t = blockIdx.y, B = P.B, B2 = B * B;
    __shared__ long long A[12];
    __shared__ float s_red[8][NQ * 12];
    if (threadIdx.x < 12) A[threadIdx.x] = aff[t].A[threadIdx.x];
    const float *W = wtab + ((size_t)t * nq_total + q0) * B2;
    int RS = B, QS = B2;  // row stride and per-q stride of the table in use
    if (w_in_smem) {
        for (int c = threadIdx.x; c < NQ * B2; c += blockDim.x) {
            const int qq = c / B2, cc = c % B2;
            sw[qq * B * (B + 1) + (cc / B) * (B + 1) + cc % B] = W[c];
        }
        W = sw;
        RS = B + 1;
        QS = B * (B + 1);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const int n0 = P.nm[0], n1 = P.nm[1], n2 = P.nm[2];
    const long long R = (long long)nf1 * P.nf[2];
    const float Bm4 = (float)(B - 4);
    // moments are taken about the fixed-volume centre, where the rotation and
    // scale columns of du/dtheta have no constant part (no cancellation)
    const float ci = 0.5f * (float)(nf0 - 1), cj = 0.5f * (float)(nf1 - 1), ck = 0.5f * (float)(P.nf[2] - 1);
    float M[NQ][12];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int e = 0; e < 12; ++e) M[q][e] = 0.0f;
    for (long long r = (long long)blockIdx.x * nwarps + warp; r < R; r += (long long)gridDim.x * nwarps) {
        const long long jl = r % nf1, kl = r / nf1;
        const long long b0 = A[1] * jl + A[2] * kl + A[3];
        const long long b1 = A[5] * jl + A[6] * kl + A[7];
        const long long b2 = A[9] * jl + A[10] * kl + A[11];
        const float j = (float)jl - cj, k = (float)kl - ck;
        const uint8_t *__restrict__ frow = P.fbins + (size_t)r * nf0;
        for (int i = lane; i < nf0; i += 32) {
            const long long ux = b0 + A[0] * i, uy = b1 + A[4] * i, uz = b2 + A[8] * i;
            if (!inside_u(ux, uy, uz, n0, n1, n2)) continue;
            const MG g = trilinear<true>(P.mov, n0, n1, n2, ux, uy, uz);
            const float ic = (float)i - ci;
            const float mt = fmaf(fminf(fmaxf(g.m, 0.0f), 1.0f), Bm4, 2.0f);
            const int k0 = (int)mt;
            float d[4];
            bspline_dw(mt - (float)k0, d);
            if (k0 + 2 >= B) d[3] = 0.0f;
            const int base = (int)__ldg(frow + i) * RS + (k0 - 1);
            const int i3 = k0 + 2 < B ? base + 3 : base;  // in range; weight 0 when clamped
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float *Wq = W + (size_t)q * QS;
                const float s = Wq[base] * d[0] + Wq[base + 1] * d[1] + Wq[base + 2] * d[2] + Wq[i3] * d[3];
                const float sx = s * g.gx, sy = s * g.gy, sz = s * g.gz;
                M[q][0] = fmaf(sx, ic, M[q][0]);
                M[q][1] = fmaf(sx, j, M[q][1]);
                M[q][2] = fmaf(sx, k, M[q][2]);
                M[q][3] += sx;
                M[q][4] = fmaf(sy, ic, M[q][4]);
                M[q][5] = fmaf(sy, j, M[q][5]);
                M[q][6] = fmaf(sy, k, M[q][6]);
                M[q][7] += sy;
                M[q][8] = fmaf(sz, ic, M[q][8]);
                M[q][9] = fmaf(sz, j, M[q][9]);
                M[q][10] = fmaf(sz, k, M[q][10]);
                M[q][11] += sz;
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

// grad[t][q][p] = -(B - 4) / N sum_e mom[t][q][e] J[t][e][p], J taken about the fixed centre
__global__ void k_parzen_grad(int n, int nq, int B, int nparts, const unsigned long long *__restrict__ gcount,
                              const double *__restrict__ mom, const double *__restrict__ jac, double *__restrict__ grad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n * nq * 9) return;
    const int p = x % 9, tq = x / 9, t = tq / nq;
    const double N = (double)gcount[t];
    if (N <= 0) {
        grad[x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double s = 0.0;
    for (int e = 0; e < 12; ++e) {
        double me = 0.0;
        for (int b = 0; b < nparts; ++b) me += mom[((size_t)tq * nparts + b) * 12 + e];
        s += me * jac[((size_t)t * 12 + e) * 9 + p];
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

int parzen_cell_blocks(int B) { return (B * B + 255) / 256; }

cudaError_t launch_parzen_hist(const ParzenPair &P, const ParzenAffine *d_aff, int n, int ctas,
                               unsigned long long *d_hist, unsigned long long *d_count, cudaStream_t s) {
    const size_t B2 = (size_t)P.B * P.B;
    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)n * B2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_count, 0, (size_t)n * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    const size_t smem = 2 * (size_t)P.B * (P.B + 1) * sizeof(uint32_t);
    if ((e = cudaFuncSetAttribute(k_parzen_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    dim3 grid(ctas, n);
    k_parzen_hist<<<grid, 256, smem, s>>>(P, d_aff, d_hist, d_count);
    return cudaGetLastError();
}

cudaError_t launch_parzen_weights(const unsigned long long *d_hist, const unsigned long long *d_count, int n, int B,
                                  const QSet &Q, double *marg, double *ment, double *jpart, double *d_mi, float *d_w,
                                  cudaStream_t s) {
    cudaError_t e;
    k_parzen_marg<<<n, 256, 0, s>>>(d_hist, d_count, B, Q, marg, ment);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nb = parzen_cell_blocks(B);
    dim3 grid(nb, n);
    k_parzen_cells<<<grid, 256, 0, s>>>(d_hist, d_count, B, Q, marg, ment, jpart, d_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_parzen_final<<<(n * Q.nq + 127) / 128, 128, 0, s>>>(n, d_count, Q, ment, jpart, nb, d_mi);
    return cudaGetLastError();
}

cudaError_t launch_parzen_adjoint(const ParzenPair &P, const ParzenAffine *d_aff, const double *d_jac, int n, int nq,
                                  int ctas, const float *d_w, const unsigned long long *d_count, double *d_mom,
                                  double *d_grad, cudaStream_t s) {
    cudaError_t e;
    const size_t B2 = (size_t)P.B * P.B;
    dim3 grid(ctas, n);
    for (int q0 = 0; q0 < nq; q0 += 4) {
        const int g = nq - q0 < 4 ? nq - q0 : 4;
        const size_t wbytes = (size_t)g * P.B * (P.B + 1) * sizeof(float);
        const int in_smem = wbytes <= 96 * 1024;
        const size_t smem = in_smem ? wbytes : 0;
#define MI_ADJ(NQV)                                                                                         \
    do {                                                                                                    \
        if ((e = cudaFuncSetAttribute(k_parzen_adj<NQV>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                      (int)smem)) != cudaSuccess)                                           \
            return e;                                                                                       \
        k_parzen_adj<NQV><<<grid, 256, smem, s>>>(P, d_aff, nq, q0, d_w, in_smem, d_mom);                   \
    } while (0)
        switch (g) {
            case 1: MI_ADJ(1); break;
            case 2: MI_ADJ(2); break;
            case 3: MI_ADJ(3); break;
            default: MI_ADJ(4); break;
        }
#undef MI_ADJ
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_parzen_grad<<<(n * nq * 9 + 127) / 128, 128, 0, s>>>(n, nq, P.B, ctas, d_count, d_mom, d_jac, d_grad);
    return cudaGetLastError();
}

}  // namespace mi
