// mi_hard.cu -- hard-binned mutual information on sm_103a.
//
// Per transform T and fixed voxel i: the 16.16 moving index U = A i + b
// (exact integers), the overlap test, an 8-neighbour integer trilinear
// resample of the moving volume, the moving bin, and one increment of the
// joint histogram h[fixed bin][moving bin] (the paper's full, all-voxel
// histogram, Discussion).  The entropies of Eq. (1) and the MI of Eq. (2)
// (and Tsallis entropies for every q from the same histogram) are reduced in
// FP64 from the exact counts.
//
// Kernels:
//   k_bin_fixed       fixed volume -> uint8 bins, once per context
//   k_hist<...>       plain form: many CTAs per transform, privatised shared
//                     histograms flushed to a global histogram per transform
//   k_entropy         plain form: one CTA per transform reduces the global histogram
//   k_batched<...>    batched form: persistent CTAs pull (pair, transform)
//                     items from an atomic ticket; one CTA builds the whole
//                     histogram of an item in shared memory and reduces it in place
//   k_resample        v(T(x)) on the fixed grid
//
// Row clipping: along a fixed row (j, k) the moving index is linear in i, so
// the overlap is one interval [lo, hi] of i, found per row (float estimate,
// then exact 64-bit checks).  Inside it every U_a lies in [0, (n_a-1) 2^16],
// so the per-voxel arithmetic is exact in 32 bits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mi_internal.h"

namespace mi {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kEmptyKey = 0xffffffffu;

// ---------------------------------------------------------------------------
// Small kernels run once per context
// ---------------------------------------------------------------------------

__global__ void k_f32_to_u16(const float *__restrict__ in, long long n, uint16_t *__restrict__ out) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double v = (double)in[x];
        if (!(v == v)) v = 0.0;
        double s = rint(v * 65535.0);  // round half to even
        s = s < 0.0 ? 0.0 : (s > 65535.0 ? 65535.0 : s);
        out[x] = (uint16_t)s;
    }
}

template <typename T>
__global__ void k_clamp_depth(T *__restrict__ data, long long n, uint32_t vmax) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        uint32_t v = data[x];
        if (v > vmax) data[x] = (T)vmax;
    }
}

// bin(v) = (min(v, 2^d - 1) * bins) >> d
template <typename T>
__global__ void k_bin_fixed(const T *__restrict__ in, long long n, int depth, int bins, uint8_t *__restrict__ out) {
    const uint32_t vmax = (uint32_t)((1ull << depth) - 1ull);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        uint32_t v = in[x];
        v = v > vmax ? vmax : v;
        out[x] = (uint8_t)(((uint64_t)v * (uint32_t)bins) >> depth);
    }
}

// tab[c] = c ln c (q == 1) or c^q, FP64, c < kTab; tab[0] = 0.
__global__ void k_table(double *__restrict__ tab, float qf) {
    const double q = (double)qf;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < kTab; c += gridDim.x * blockDim.x) {
        double d = (double)c;
        tab[c] = c == 0 ? 0.0 : (qf == 1.0f ? d * log(d) : pow(d, q));
    }
}

// ---------------------------------------------------------------------------
// Per-voxel sampling
// ---------------------------------------------------------------------------

// Stage lerp with an 8-bit weight: (a (256 - f) + b f + 128) >> 8 written as
// a + floor(((b - a) f + 128) / 256), identical for integers (arithmetic shift).
__device__ __forceinline__ int lerp8(int a, int b, int f) { return a + (((b - a) * f + 128) >> 8); }

template <typename MovT>
__device__ __forceinline__ int sample_hard(const MovT *__restrict__ mov, int n0, int n1, int n2, int ux, int uy,
                                           int uz) {
    const int ix = ux >> 16, iy = uy >> 16, iz = uz >> 16;
    const int fx = (ux >> 8) & 255, fy = (uy >> 8) & 255, fz = (uz >> 8) & 255;
    // the upper neighbour is clamped on the last plane, where its weight is 0
    const int sx = ix < n0 - 1 ? 1 : 0;
    const int sy = iy < n1 - 1 ? n0 : 0;
    const int sz = iz < n2 - 1 ? n0 * n1 : 0;
    const MovT *p = mov + (ix + n0 * (iy + n1 * iz));
    const int v000 = __ldg(p), v001 = __ldg(p + sx), v010 = __ldg(p + sy), v011 = __ldg(p + sy + sx);
    const int v100 = __ldg(p + sz), v101 = __ldg(p + sz + sx), v110 = __ldg(p + sz + sy),
              v111 = __ldg(p + sz + sy + sx);
    const int e00 = lerp8(v000, v001, fx), e01 = lerp8(v010, v011, fx);
    const int e10 = lerp8(v100, v101, fx), e11 = lerp8(v110, v111, fx);
    const int g0 = lerp8(e00, e01, fy), g1 = lerp8(e10, e11, fy);
    return lerp8(g0, g1, fz);
}

// The same resample from the padded x-paired moving volume: element (x, y, z)
// holds v[x] in its low half and v[min(x + 1, n0 - 1)] in its high half
// (uint16 pairs of a uint8 volume, uint32 pairs of a uint16 volume), and the
// volume carries one extra y row and one extra z plane repeating the last
// ones, so the three neighbour offsets are constants (n0, n0 (n1 + 1)) and a
// voxel takes 4 loads.  On the last plane of an axis the weight of the upper
// neighbour is 0, so the repeated values change nothing.
// Each stage lerp is (a (256 - f) + b f + 128) >> 8.
__device__ __forceinline__ int lerp8g(int a, int b, int f, int g) { return (a * g + b * f + 128) >> 8; }

template <typename PairT>
__device__ __forceinline__ int sample_hard_pair(const PairT *__restrict__ movp, int sy, int sz, int n0, int n01p,
                                                int ux, int uy, int uz) {
    constexpr int HB = (int)sizeof(PairT) * 4;  // bits per half
    constexpr uint32_t LO = (1u << HB) - 1u;
    const int fx = (int)__byte_perm((unsigned)ux, 0u, 0x4441), fy = (int)__byte_perm((unsigned)uy, 0u, 0x4441),
              fz = (int)__byte_perm((unsigned)uz, 0u, 0x4441);
    const int gx = 256 - fx, gy = 256 - fy, gz = 256 - fz;
    const int idx = (ux >> 16) + n0 * (uy >> 16) + n01p * (uz >> 16);
    const PairT *p = movp + idx;
    const uint32_t a = __ldg(p), b = __ldg(p + sy), c = __ldg(p + sz), d = __ldg(p + sz + sy);
    const int e00 = lerp8g((int)(a & LO), (int)(a >> HB), fx, gx), e01 = lerp8g((int)(b & LO), (int)(b >> HB), fx, gx);
    const int e10 = lerp8g((int)(c & LO), (int)(c >> HB), fx, gx), e11 = lerp8g((int)(d & LO), (int)(d >> HB), fx, gx);
    const int g0 = lerp8g(e00, e01, fy, gy), g1 = lerp8g(e10, e11, fy, gy);
    return lerp8g(g0, g1, fz, gz);
}

// The same resample with the four x-pairs fetched through the texture path
// from a 3D array of pairs (block-linear layout, point sampling at texel
// centres, clamped addressing: exact integer texels).
template <typename PairT>
__device__ __forceinline__ int sample_hard_tex(unsigned long long tex, int ux, int uy, int uz) {
    constexpr int HB = (int)sizeof(PairT) * 4;
    constexpr uint32_t LO = (1u << HB) - 1u;
    const int fx = (int)__byte_perm((unsigned)ux, 0u, 0x4441), fy = (int)__byte_perm((unsigned)uy, 0u, 0x4441),
              fz = (int)__byte_perm((unsigned)uz, 0u, 0x4441);
    const int gx = 256 - fx, gy = 256 - fy, gz = 256 - fz;
    const float x = (float)(ux >> 16) + 0.5f, y = (float)(uy >> 16) + 0.5f, z = (float)(uz >> 16) + 0.5f;
    const uint32_t a = tex3D<PairT>(tex, x, y, z), b = tex3D<PairT>(tex, x, y + 1.0f, z);
    const uint32_t c = tex3D<PairT>(tex, x, y, z + 1.0f), d = tex3D<PairT>(tex, x, y + 1.0f, z + 1.0f);
    const int e00 = lerp8g((int)(a & LO), (int)(a >> HB), fx, gx), e01 = lerp8g((int)(b & LO), (int)(b >> HB), fx, gx);
    const int e10 = lerp8g((int)(c & LO), (int)(c >> HB), fx, gx), e11 = lerp8g((int)(d & LO), (int)(d >> HB), fx, gx);
    const int g0 = lerp8g(e00, e01, fy, gy), g1 = lerp8g(e10, e11, fy, gy);
    return lerp8g(g0, g1, fz, gz);
}

// The same resample from 2 x 2 (y, z) quads through the texture path.  A fetch
// at integer texel coordinates (ix, iy, iz) returns v(ix, iy, iz),
// v(ix, iy + 1, iz), v(ix, iy, iz + 1), v(ix, iy + 1, iz + 1) in four
// registers, already unpacked, so a voxel takes two fetches (columns ix and
// ix + 1).  Column ix + 1 lies past the volume only when ix = nx - 1, which
// inside the overlap means a fraction of 0: the clamped texel's weight is 0.
// Neighbouring lanes of a warp step along x, so the column one lane fetches
// second is, under most transforms, the one the next lane fetches first: the
// two requests of a warp step touch about one texel per voxel, and each texel
// is wanted within one step (with (x, y) quads each texel is also wanted as
// the upper plane of the next fixed slice, long after the L1 has evicted it).
__device__ __forceinline__ void tex_quad(unsigned long long tex, int x, int y, int z, uint32_t &a, uint32_t &b,
                                         uint32_t &c, uint32_t &d) {
    asm("tex.3d.v4.u32.s32 {%0, %1, %2, %3}, [%4, {%5, %6, %7, %7}];"
        : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
        : "l"(tex), "r"(x), "r"(y), "r"(z));
}

// The 8 neighbours of the sample at 16.16 index (ux, uy, uz) in quad_lerp's order: t[0..3] =
// (x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1) of plane iz, t[4..7] the same of plane iz + 1.
__device__ __forceinline__ void quad_fetch(unsigned long long tex, unsigned ux, unsigned uy, unsigned uz,
                                           uint32_t (&t)[8]) {
    const int ix = (int)(ux >> 16), iy = (int)(uy >> 16), iz = (int)(uz >> 16);
    tex_quad(tex, ix, iy, iz, t[0], t[2], t[4], t[6]);
    tex_quad(tex, ix + 1, iy, iz, t[1], t[3], t[5], t[7]);
}

// Trilinear value from the 8 neighbours: x, then y, then z stages.
__device__ __forceinline__ int quad_lerp(unsigned ux, unsigned uy, unsigned uz, const uint32_t (&t)[8]) {
    const int fx = (int)__byte_perm(ux, 0u, 0x4441), fy = (int)__byte_perm(uy, 0u, 0x4441),
              fz = (int)__byte_perm(uz, 0u, 0x4441);
    const int gx = 256 - fx, gy = 256 - fy, gz = 256 - fz;
    const int e00 = lerp8g((int)t[0], (int)t[1], fx, gx), e01 = lerp8g((int)t[2], (int)t[3], fx, gx);
    const int e10 = lerp8g((int)t[4], (int)t[5], fx, gx), e11 = lerp8g((int)t[6], (int)t[7], fx, gx);
    const int g0 = lerp8g(e00, e01, fy, gy), g1 = lerp8g(e10, e11, fy, gy);
    return lerp8g(g0, g1, fz, gz);
}

// The 8 neighbours of the sample at 16.16 index (ux, uy, uz) in one gather from the z-pair atlas:
// the float coordinates ix + 1 + ox, iy + 1 + oy (exact integers, so the gather's 2 x 2 footprint
// starts at texel (ix, iy) of plane iz's tile) are formed from the bit pattern 2^23 + ix plus the
// plane's stored offset ox + 1 - 2^23.  The gather returns (ix, iy + 1), (ix + 1, iy + 1),
// (ix + 1, iy), (ix, iy), each holding v(x, y, z) in bits 0..11 and v(x, y, z + 1) in bits 20..31
// (moving depth <= 12); unpacked, the eight values take quad_lerp's stages.  (Lerping both planes at
// once in 20-bit fields of 64-bit products took fewer instructions but measured 6 % slower.)  On the
// last plane of an axis the upper neighbour's weight is 0, so the texel beyond the tile edge (the next
// tile, or a clamped one) changes nothing.
__device__ __forceinline__ int gather_value(unsigned long long tex, const float2 *zoff, unsigned ux, unsigned uy,
                                            unsigned uz) {
    const float2 o = zoff[uz >> 16];
    const float u = __int_as_float((int)__funnelshift_r(ux, 0x4B00u, 16)) + o.x;
    const float v = __int_as_float((int)__funnelshift_r(uy, 0x4B00u, 16)) + o.y;
    const uint4 t = tex2Dgather<uint4>((cudaTextureObject_t)tex, u, v, 0);
    const uint32_t n[8] = {t.w & 0xFFFu, t.z & 0xFFFu, t.x & 0xFFFu, t.y & 0xFFFu,
                           t.w >> 20, t.z >> 20, t.x >> 20, t.y >> 20};
    return quad_lerp(ux, uy, uz, n);
}

// Builds the z-pair atlas (see launch_make_zpairs).
template <typename T>
__global__ void k_make_zpairs(const T *__restrict__ in, int n0, int n1, int n2, int ph, int W,
                              uint32_t *__restrict__ out) {
    const long long plane = (long long)n0 * n1, n = plane * n2;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % n0);
        const int y = (int)((o / n0) % n1);
        const int z = (int)(o / plane);
        const int z1 = min(z + 1, n2 - 1);
        const long long src = (long long)y * n0 + x;
        const uint32_t v = (uint32_t)in[plane * z + src] | ((uint32_t)in[plane * z1 + src] << 20);
        const long long ox = (long long)(z / ph) * n0 + x, oy = (long long)(z % ph) * n1 + y;
        out[oy * W + ox] = v;
    }
}

// Builds the 2 x 2 (y, z) quads: out has dims (n0, n1, n2); element (x, y, z) holds v(x, y, z),
// v(x, y + 1, z), v(x, y, z + 1), v(x, y + 1, z + 1), upper indices clamped to the last ones.
template <typename T, typename QT>
__global__ void k_make_quads(const T *__restrict__ in, int n0, int n1, int n2, QT *__restrict__ out) {
    const long long plane = (long long)n0 * n1, n = plane * n2;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % n0);
        const int y = (int)((o / n0) % n1);
        const int z = (int)(o / plane);
        const int y1 = min(y + 1, n1 - 1), z1 = min(z + 1, n2 - 1);
        QT q;
        q.x = in[plane * z + (long long)y * n0 + x];
        q.y = in[plane * z + (long long)y1 * n0 + x];
        q.z = in[plane * z1 + (long long)y * n0 + x];
        q.w = in[plane * z1 + (long long)y1 * n0 + x];
        out[o] = q;
    }
}

// Builds the padded x-paired volume: out has dims (n0, n1 + 1, n2 + 1).
template <typename T, typename PairT>
__global__ void k_make_pairs(const T *__restrict__ in, int n0, int n1, int n2, PairT *__restrict__ out) {
    constexpr int HB = (int)sizeof(PairT) * 4;
    const long long n = (long long)n0 * (n1 + 1) * (n2 + 1);
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % n0);
        const int y = min((int)((o / n0) % (n1 + 1)), n1 - 1);
        const int z = min((int)(o / ((long long)n0 * (n1 + 1))), n2 - 1);
        const long long src = x + (long long)n0 * (y + (long long)n1 * z);
        out[o] = (PairT)((uint32_t)in[src] | ((uint32_t)in[x < n0 - 1 ? src + 1 : src] << HB));
    }
}

// Overlap interval [lo, hi] of fixed row (j, k) and the 16.16 moving index at i = lo.
struct RowClip {
    int lo, hi, u0, u1, u2;
};

__device__ __forceinline__ bool inside_at(const long long base[3], const int st[3], const long long umax[3], int i) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long U = base[a] + (long long)st[a] * i;
        if (U < 0 || U > umax[a]) return false;
    }
    return true;
}

__device__ RowClip clip_row(const int *q, int j, int k, int nf0, const int nm[3]) {
    long long base[3], umax[3];
    int st[3];
    int lo = 0, hi = nf0 - 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        base[a] = (long long)q[4 * a + 1] * j + (long long)q[4 * a + 2] * k + (long long)q[4 * a + 3];
        umax[a] = (long long)(nm[a] - 1) << 16;
        st[a] = q[4 * a];
        if (st[a] == 0) {
            if (base[a] < 0 || base[a] > umax[a]) { lo = nf0; hi = -1; }
        } else {
            // estimate of the real interval {i : 0 <= base + st i <= umax}; within one voxel of the truth
            const float fb = (float)base[a], fs = (float)st[a], fm = (float)umax[a];
            float e0 = -fb / fs, e1 = (fm - fb) / fs;
            float a0 = fminf(e0, e1), a1 = fmaxf(e0, e1);
            a0 = fminf(fmaxf(a0, -2.0f), (float)nf0 + 1.0f);
            a1 = fminf(fmaxf(a1, -2.0f), (float)nf0 + 1.0f);
            lo = max(lo, (int)ceilf(a0));
            hi = min(hi, (int)floorf(a1));
        }
    }
    // exact fix-up: the interval of a linear function is contiguous
    while (lo <= hi && !inside_at(base, st, umax, lo)) ++lo;
    while (lo > 0 && lo <= nf0 && inside_at(base, st, umax, lo - 1)) --lo;
    while (hi >= lo && !inside_at(base, st, umax, hi)) --hi;
    while (hi >= lo && hi < nf0 - 1 && inside_at(base, st, umax, hi + 1)) ++hi;
    if (hi < lo && lo < nf0 && inside_at(base, st, umax, lo)) {
        hi = lo;
        while (hi < nf0 - 1 && inside_at(base, st, umax, hi + 1)) ++hi;
    }
    RowClip r;
    r.lo = lo;
    r.hi = hi;
    r.u0 = r.u1 = r.u2 = 0;
    if (lo <= hi) {
        r.u0 = (int)(base[0] + (long long)st[0] * lo);
        r.u1 = (int)(base[1] + (long long)st[1] * lo);
        r.u2 = (int)(base[2] + (long long)st[2] * lo);
    }
    return r;
}

// ---------------------------------------------------------------------------
// Shared-memory histogram policies
// ---------------------------------------------------------------------------

// Shared histograms address cell (bf, bm) through rows padded by one word:
// with a row stride of S = B + 1 words the bank is (row + column) mod 32,
// so cells clustered in a few moving bins (the Rician background occupies
// bins 0..15 of both volumes) still spread over the banks.

// 32-bit counters: one shared atomic per voxel (or per group of equal cells in a warp).
template <bool MATCH>
struct HistU32 {
    uint32_t *h;
    int B, S;  // bins, padded row stride in words
    __device__ void load_info(const uint32_t *) {}
    __device__ void zero() {
        for (int c = threadIdx.x; c < B * S; c += blockDim.x) h[c] = 0;
    }
    __device__ __forceinline__ void add(int bf, int bm, bool valid) {
        const int idx = bf * S + bm;
        if (!MATCH) {
            if (valid) atomicAdd(&h[idx], 1u);
        } else {
            const unsigned vm = __ballot_sync(kFull, valid);
            if (valid) {
                const unsigned peers = __match_any_sync(vm, idx);
                if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[idx], (unsigned)__popc(peers));
            }
        }
    }
    __device__ __forceinline__ uint32_t count(int bf, int bm) const { return h[bf * S + bm]; }
};

// 16-bit counters, two per word: the word at (row r, column bm) holds cell
// (r, bm) in its low half and cell (r + H, bm) in its high half, H = ceil(B/2),
// so the two halves of a word belong to fixed bins far apart and rarely
// collide.  A counter whose value reaches kDrainT is drained whole into a
// shared hash table of 32-bit overflow counts by a compare-and-swap; the
// adder that observed it does the drain, so a counter never exceeds
// kDrainT + (threads x 32) < 2^16.  The true count is the 16-bit value plus
// the overflow entry (flagged in a bitmap).  Overflow entries are keyed by
// the cell id bf * B + bm.
// Iteration cap of the drain's compare-and-swap loop (a failure-handling test hook lowers it; at 0
// every drain gives up at once and flags the error).
__device__ int g_drain_cap = 1 << 16;

template <bool MATCH>
struct HistU16 {
    uint32_t *w;      // H x S words
    uint32_t *okey;   // kOvfSlots keys
    uint32_t *ocnt;   // kOvfSlots counts
    uint32_t *bmap;   // (B^2 + 31) / 32 words
    int *flags;
    int B, S, H;
    __device__ void load_info(const uint32_t *) {}
    __device__ void zero() {
        const int nw = H * S, nb = (B * B + 31) >> 5;
        for (int c = threadIdx.x; c < nw; c += blockDim.x) w[c] = 0;
        for (int c = threadIdx.x; c < kOvfSlots; c += blockDim.x) {
            okey[c] = kEmptyKey;
            ocnt[c] = 0;
        }
        for (int c = threadIdx.x; c < nb; c += blockDim.x) bmap[c] = 0;
    }
    __device__ __forceinline__ static uint32_t slot_of(uint32_t key) { return (key * 2654435761u) >> 20; }
    __device__ void ovf_add(uint32_t key, uint32_t amount) {
        uint32_t s = slot_of(key) & (kOvfSlots - 1);
        for (int probe = 0; probe < kOvfSlots; ++probe) {
            const uint32_t k = ((volatile uint32_t *)okey)[s];
            if (k == key) {
                atomicAdd(&ocnt[s], amount);
                return;
            }
            if (k == kEmptyKey) {
                const uint32_t prev = atomicCAS(&okey[s], kEmptyKey, key);
                if (prev == kEmptyKey || prev == key) {
                    atomicAdd(&ocnt[s], amount);
                    if (prev == kEmptyKey) atomicOr(&bmap[key >> 5], 1u << (key & 31));
                    return;
                }
            }
            s = (s + 1) & (kOvfSlots - 1);
        }
        atomicOr(&flags[1], 1);  // cannot happen while N <= kOvfSlots / 2 * kDrainT
    }
    __device__ void drain(uint32_t idx, uint32_t sh, uint32_t key) {
        volatile uint32_t *vw = w;
        const int cap = g_drain_cap;
        // each failed attempt means another update of this word succeeded; bounded for safety
        for (int it = 0; it < cap; ++it) {
            const uint32_t cur = vw[idx];
            const uint32_t hv = (cur >> sh) & 0xffffu;
            if (hv < (uint32_t)kDrainT) return;
            if (atomicCAS(&w[idx], cur, cur - (hv << sh)) == cur) {
                ovf_add(key, hv);
                return;
            }
        }
        atomicOr(&flags[1], 2);
    }
    __device__ __forceinline__ void inc(int bf, int bm, uint32_t n) {
        const bool hi = bf >= H;
        const uint32_t idx = (uint32_t)((hi ? bf - H : bf) * S + bm), sh = hi ? 16u : 0u;
        const uint32_t old = atomicAdd(&w[idx], n << sh);
        if (((old >> sh) & 0xffffu) + n >= (uint32_t)kDrainT) drain(idx, sh, (uint32_t)(bf * B + bm));
    }
    __device__ __forceinline__ void add(int bf, int bm, bool valid) {
        if (!MATCH) {
            if (valid) inc(bf, bm, 1u);
        } else {
            const unsigned vm = __ballot_sync(kFull, valid);
            if (valid) {
                const unsigned peers = __match_any_sync(vm, bf * B + bm);
                if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) inc(bf, bm, (unsigned)__popc(peers));
            }
        }
    }
    __device__ __forceinline__ uint32_t count(int bf, int bm) const {
        const bool hi = bf >= H;
        uint32_t v = (w[(hi ? bf - H : bf) * S + bm] >> (hi ? 16 : 0)) & 0xffffu;
        const int c = bf * B + bm;
        if (bmap[c >> 5] & (1u << (c & 31))) {
            uint32_t s = slot_of((uint32_t)c) & (kOvfSlots - 1);
            for (int probe = 0; probe < kOvfSlots; ++probe) {
                const uint32_t k = okey[s];
                if (k == (uint32_t)c) return v + ocnt[s];
                if (k == kEmptyKey) break;
                s = (s + 1) & (kOvfSlots - 1);
            }
        }
        return v;
    }
};

// Row-bound layout.  A cell count can never exceed the number of fixed voxels
// in its row's bin, F[r] (each fixed voxel contributes at most once per
// transform), and F is known when the context is built.  Rows with
// F[r] <= 65535 ("narrow") share words two at a time as 16-bit halves; the
// others ("wide") get 32-bit words.  No counter can overflow, so increments
// are fire-and-forget atomics with no return value and no drain.  rowinfo[r]
// = word offset of row r << 6 | wide << 5 | shift (0 or 16: the half of a
// narrow row); rows are padded to S = B + 1 words.
struct HistRows {
    uint32_t *w;
    uint32_t *info;  // B entries, copied into shared memory per item
    int B, S, nwords;
    __device__ void load_info(const uint32_t *rowinfo) {
        for (int r = threadIdx.x; r < B; r += blockDim.x) info[r] = __ldg(rowinfo + r);
    }
    __device__ void zero() {
        for (int c = threadIdx.x; c < nwords; c += blockDim.x) w[c] = 0;
    }
    __device__ __forceinline__ void add(int bf, int bm, bool valid) {
        if (valid) {
            const uint32_t inf = info[bf];
            // 1 << (inf & 31): the funnel shift takes its count modulo 32
            atomicAdd(&w[(inf >> 6) + bm], __funnelshift_l(0u, 1u, inf));
        }
    }
    __device__ __forceinline__ uint32_t count(int bf, int bm) const {
        const uint32_t inf = info[bf];
        const uint32_t v = w[(inf >> 6) + bm] >> (inf & 31u);
        return (inf & 32u) ? v : (v & 0xffffu);
    }
};

// Global 32-bit histogram, row-major bins x bins (plain path's entropy reduction).
struct HistGlobal {
    const uint32_t *h;
    int B;
    __device__ __forceinline__ uint32_t count(int bf, int bm) const { return __ldg(h + bf * B + bm); }
};

// Shared-memory layout of a CTA: [histogram words][ovf keys][ovf counts][bitmap] [rows][cols] [FP64 scratch].
__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmemLayout {
    size_t hist, okey, ocnt, bmap, rinfo, rows, cols, red, zoff, total;
};

// zmax: planes of the largest moving volume (the gather variants keep one float2 offset per plane).
__host__ __device__ inline SmemLayout smem_layout(int variant, int bins, int threads, int rows_words, int zmax) {
    SmemLayout L;
    const size_t B2 = (size_t)bins * bins;
    const int kind = hv_kind(variant);
    const bool u16 = kind == HV_U16 || kind == HV_U16_MATCH;
    const size_t S = (size_t)bins + 1, H = ((size_t)bins + 1) / 2;
    size_t o = 0;
    L.hist = o;
    if (kind == HV_ROWS)
        o += (size_t)rows_words * 4;
    else
        o += u16 ? H * S * 4 : (size_t)bins * S * 4;
    L.okey = o;
    if (u16) o += (size_t)kOvfSlots * 4;
    L.ocnt = o;
    if (u16) o += (size_t)kOvfSlots * 4;
    L.bmap = o;
    if (u16) o += ((B2 + 31) / 32) * 4;
    L.rinfo = o;
    if (kind == HV_ROWS) o += (size_t)bins * 4;
    L.rows = o;
    o += (size_t)bins * 4;
    L.cols = o;
    o += (size_t)bins * 4;
    o = align_up(o, 16);
    L.red = o;
    o += (size_t)(3 * 32 + 3 * kMaxQ + 1) * 8;
    L.zoff = o;
    if (hv_fetch(variant) == FM_GATHER) o += (size_t)zmax * 8;
    L.total = o;
    (void)threads;
    return L;
}

template <int HV>
struct HistOf;
template <>
struct HistOf<HV_U32> { using T = HistU32<false>; };
template <>
struct HistOf<HV_U32_MATCH> { using T = HistU32<true>; };
template <>
struct HistOf<HV_U16> { using T = HistU16<false>; };
template <>
struct HistOf<HV_U16_MATCH> { using T = HistU16<true>; };
template <>
struct HistOf<HV_ROWS> { using T = HistRows; };

template <int HV>
__device__ typename HistOf<HV>::T make_hist(unsigned char *smem, const SmemLayout &L, int B, int *flags,
                                            int rows_words = 0) {
    typename HistOf<HV>::T H;
    H.B = B;
    H.S = B + 1;
    if constexpr (HV == HV_U16 || HV == HV_U16_MATCH) {
        H.H = (B + 1) / 2;
        H.w = (uint32_t *)(smem + L.hist);
        H.okey = (uint32_t *)(smem + L.okey);
        H.ocnt = (uint32_t *)(smem + L.ocnt);
        H.bmap = (uint32_t *)(smem + L.bmap);
        H.flags = flags;
    } else if constexpr (HV == HV_ROWS) {
        H.w = (uint32_t *)(smem + L.hist);
        H.info = (uint32_t *)(smem + L.rinfo);
        H.nwords = rows_words;
        (void)flags;
    } else {
        H.h = (uint32_t *)(smem + L.hist);
        (void)flags;
        (void)rows_words;
    }
    return H;
}

// ---------------------------------------------------------------------------
// Voxel loop: warps take batches of 32 fixed rows; lane l clips row rb + l,
// then the warp walks the 32 clipped rows 32 voxels at a time.
// ---------------------------------------------------------------------------

// Row order: the CTA walks blocks of nwarps adjacent fixed rows (block blk
// holds rows blk * nwarps + w) and warp w takes row w of each block, so at any
// time the warps of a CTA sample neighbouring moving lines (row j's upper y
// neighbours are row j + 1's samples).  Blocks are first_block + n *
// block_stride, n = 0, 1, ...  A warp clips its next 32 rows at once (lane l
// takes the warp's l-th upcoming row, exactly in 64 bits), then walks them one
// by one, 32 voxels at a time, with each row's interval broadcast by shuffles.
// Blocks first_block + n * block_stride, n = 0, 1, ..., below n_end are
// visited (the batched kernel passes one slab of blocks at a time).
// The interpolated moving value at a 16.16 index, through the variant's fetch path.
template <int FM, typename PairT>
__device__ __forceinline__ int sample_value(const PairDev &P, const float2 *zoff, unsigned U0, unsigned U1,
                                            unsigned U2) {
    if constexpr (FM == FM_GATHER) {
        return gather_value(P.texg, zoff, U0, U1, U2);
    } else if constexpr (FM == FM_QUAD) {
        uint32_t t[8];
        quad_fetch(P.texq, U0, U1, U2, t);
        return quad_lerp(U0, U1, U2, t);
    } else if constexpr (FM == FM_TEX) {
        return sample_hard_tex<PairT>(P.texp, (int)U0, (int)U1, (int)U2);
    } else {
        const int n0 = P.nm[0], sz = n0 * (P.nm[1] + 1);
        return sample_hard_pair<PairT>((const PairT *)P.movp, n0, sz, n0, sz, (int)U0, (int)U1, (int)U2);
    }
}

// A clipped row [lo, hi] under random sampling: its sampled voxels only, 32 at a time; U at an
// entry's x index i is u_lo + st (i - lo), exact inside the interval.
template <int FM, typename PairT, class Hist>
__device__ __forceinline__ void sampled_row(const PairDev &P, const float2 *zoff, long long r, int lo, int hi,
                                            unsigned ub0, unsigned ub1, unsigned ub2, int st0, int st1, int st2,
                                            Hist &H) {
    const int lane = threadIdx.x & 31;
    const int bins = P.bins, mdepth = P.mdepth;
    const uint32_t k0 = __ldg(P.srow + r), k1 = __ldg(P.srow + r + 1);
    for (uint32_t kb = k0; kb < k1; kb += 32) {
        const uint32_t k = kb + lane;
        int i = 0;
        bool valid = false;
        if (k < k1) {
            i = (int)__ldg(P.scol + k);
            valid = i >= lo && i <= hi;
        }
        int bf = 0, bm = 0;
        if (valid) {
            const unsigned d = (unsigned)(i - lo);
            const int v = sample_value<FM, PairT>(P, zoff, ub0 + (unsigned)st0 * d, ub1 + (unsigned)st1 * d,
                                                  ub2 + (unsigned)st2 * d);
            bm = (v * bins) >> mdepth;
            bf = (int)__ldg(P.sbin + k);
        }
        H.add(bf, bm, valid);
    }
}

template <typename PairT, int FM, class Hist>
__device__ void accumulate_rows(const PairDev &P, const int *q, const float2 *zoff, long long first_block,
                                long long block_stride, long long n_end, Hist &H) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const long long R = (long long)nf1 * P.nf[2];
    const int n0 = P.nm[0], sy = n0, sz = n0 * (P.nm[1] + 1);
    const int st0 = q[0], st1 = q[4], st2 = q[8];
    const int bins = P.bins, mdepth = P.mdepth;
    const PairT *__restrict__ movp = (const PairT *)P.movp;
    for (long long n0b = 0;; n0b += 32) {
        // blocks of this group: lane l gets block first_block + (n0b + l) * block_stride
        if (first_block + n0b * block_stride >= n_end) break;
        RowClip mine;
        mine.lo = 0;
        mine.hi = -1;
        mine.u0 = mine.u1 = mine.u2 = 0;
        const long long nl = first_block + (n0b + lane) * block_stride;
        if (nl < n_end) {
            const long long rl = nl * nwarps + warp;
            if (rl < R) mine = clip_row(q, (int)(rl % nf1), (int)(rl / nf1), nf0, P.nm);
        }
        for (int s = 0; s < 32; ++s) {
            const long long n = first_block + (n0b + s) * block_stride;
            if (n >= n_end) break;  // warp-uniform
            const long long r = n * nwarps + warp;
            if (r >= R) break;  // warp-uniform: only the last block may be partial
            const int lo = __shfl_sync(kFull, mine.lo, s), hi = __shfl_sync(kFull, mine.hi, s);
            if (lo > hi) continue;
            const unsigned ub0 = (unsigned)__shfl_sync(kFull, mine.u0, s), ub1 = (unsigned)__shfl_sync(kFull, mine.u1, s),
                           ub2 = (unsigned)__shfl_sync(kFull, mine.u2, s);
            if (P.srow != nullptr) {  // random sampling: the row's sampled voxels only
                sampled_row<FM, PairT>(P, zoff, r, lo, hi, ub0, ub1, ub2, st0, st1, st2, H);
                continue;
            }
            // unsigned: lanes past the row end may step outside the int range; only in-range lanes use them
            unsigned U0 = ub0 + (unsigned)st0 * lane, U1 = ub1 + (unsigned)st1 * lane, U2 = ub2 + (unsigned)st2 * lane;
            const uint8_t *__restrict__ frow = P.fbins + (size_t)r * nf0;
            for (int i = lo + lane; i - lane <= hi; i += 32) {
                const bool valid = i <= hi;
                int bf = 0, bm = 0;
                if (valid) {
                    int v;
                    if constexpr (FM == FM_TEX)
                        v = sample_hard_tex<PairT>(P.texp, (int)U0, (int)U1, (int)U2);
                    else if constexpr (FM == FM_LDG)
                        v = sample_hard_pair<PairT>(movp, sy, sz, n0, sz, (int)U0, (int)U1, (int)U2);
                    else
                        v = sample_value<FM, PairT>(P, zoff, U0, U1, U2);
                    bm = (v * bins) >> mdepth;
                    bf = (int)__ldg(frow + i);
                }
                H.add(bf, bm, valid);
                U0 += 32u * (unsigned)st0;
                U1 += 32u * (unsigned)st1;
                U2 += 32u * (unsigned)st2;
            }
        }
    }
}

// Row-group walk (quad and gather fetches, every fixed voxel).  Rows are clipped 32 at a time as in
// accumulate_rows; then each warp step covers G = 32 >> lpr_log2 adjacent rows of the batch with
// L = 1 << lpr_log2 lanes each (lane = row-in-group * L + column), so a row whose overlap is not a
// multiple of 32 wastes at most L - 1 lanes in its last step, and one clip broadcast serves G rows.
// Steps in which every lane of every row is inside its interval run without predicates; the last
// ones (up to the longest row of the group) are predicated.  The fixed bin of the next full step is
// loaded one step ahead.
template <int FM, class Hist>
__device__ void accumulate_groups(const PairDev &P, const int *q, const float2 *zoff, long long first_block,
                                  long long block_stride, long long n_end, int lpr_log2, Hist &H) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const long long R = (long long)nf1 * P.nf[2];
    const int st0 = q[0], st1 = q[4], st2 = q[8];
    const int bins = P.bins, mdepth = P.mdepth;
    const int lpr = 1 << lpr_log2, gsz = 32 >> lpr_log2;
    const int sub = lane >> lpr_log2, col = lane & (lpr - 1);
    const unsigned d0 = (unsigned)st0 << lpr_log2, d1 = (unsigned)st1 << lpr_log2, d2 = (unsigned)st2 << lpr_log2;
    for (long long n0b = 0;; n0b += 32) {
        if (first_block + n0b * block_stride >= n_end) break;
        RowClip mine;
        mine.lo = 0;
        mine.hi = -1;
        mine.u0 = mine.u1 = mine.u2 = 0;
        const long long nl = first_block + (n0b + lane) * block_stride;
        if (nl < n_end) {
            const long long rl = nl * nwarps + warp;
            if (rl < R) mine = clip_row(q, (int)(rl % nf1), (int)(rl / nf1), nf0, P.nm);
        }
        for (int s0 = 0; s0 < 32; s0 += gsz) {
            if (first_block + (n0b + s0) * block_stride >= n_end) break;  // warp-uniform
            const int s = s0 + sub;
            const int lo = __shfl_sync(kFull, mine.lo, s), hi = __shfl_sync(kFull, mine.hi, s);
            const int len = hi >= lo ? hi - lo + 1 : 0;  // rows past the end were clipped empty
            const int kfull = (int)__reduce_min_sync(kFull, (unsigned)(len >> lpr_log2));
            const int kall = (int)__reduce_max_sync(kFull, (unsigned)((len + lpr - 1) >> lpr_log2));
            if (kall == 0) continue;
            const unsigned ub0 = (unsigned)__shfl_sync(kFull, mine.u0, s), ub1 = (unsigned)__shfl_sync(kFull, mine.u1, s),
                           ub2 = (unsigned)__shfl_sync(kFull, mine.u2, s);
            const long long r = (first_block + (n0b + s) * block_stride) * nwarps + warp;
            // unsigned: lanes past their row's end may step outside the int range; only in-range lanes use them
            unsigned U0 = ub0 + (unsigned)st0 * col, U1 = ub1 + (unsigned)st1 * col, U2 = ub2 + (unsigned)st2 * col;
            const uint8_t *__restrict__ fp = P.fbins + (len > 0 ? (size_t)r * nf0 + lo + col : 0);
            int k = 0;
            int bf_next = kfull > 0 ? (int)__ldg(fp) : 0;
#pragma unroll 2
            for (; k < kfull; ++k) {
                const int bf = bf_next;
                fp += lpr;
                if (k + 1 < kfull) bf_next = (int)__ldg(fp);
                H.add(bf, (sample_value<FM, uint32_t>(P, zoff, U0, U1, U2) * bins) >> mdepth, true);
                U0 += d0;
                U1 += d1;
                U2 += d2;
            }
            for (; k < kall; ++k) {
                const bool valid = (k << lpr_log2) + col < len;
                int bf = 0, bm = 0;
                if (valid) {
                    bm = (sample_value<FM, uint32_t>(P, zoff, U0, U1, U2) * bins) >> mdepth;
                    bf = (int)__ldg(fp);
                }
                H.add(bf, bm, valid);
                fp += lpr;
                U0 += d0;
                U1 += d1;
                U2 += d2;
            }
        }
    }
}

// Stream walk (quad and gather fetches, every fixed voxel).  A warp clips its next 32 rows at once
// (lane s takes row s of the batch), then walks their overlap intervals as one stream of voxels: lane
// l takes stream positions l, l + 32, ...  An exclusive scan of the interval lengths gives each row's
// start in the stream; a lane crossing the end of its row moves to the next non-empty one and
// re-reads that row's 16.16 index and fixed-bin offset by shuffles from the row's clipping lane.
// Between row ends the warp runs segments of full steps (the most steps before any lane leaves its
// row, one warp-wide minimum) exactly like the row walk's predicate-free loop; only the batch's last
// step is partial (instead of every row's).  U = u_lo + st (i - lo) inside a row's interval is exact
// in 32 bits.
template <int FM, class Hist>
__device__ void accumulate_stream(const PairDev &P, const int *q, const float2 *zoff, long long first_block,
                                  long long block_stride, long long n_end, Hist &H) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const long long R = (long long)nf1 * P.nf[2];
    const int st0 = q[0], st1 = q[4], st2 = q[8];
    const int bins = P.bins, mdepth = P.mdepth;
    const unsigned d0 = 32u * (unsigned)st0, d1 = 32u * (unsigned)st1, d2 = 32u * (unsigned)st2;
    for (long long n0b = 0;; n0b += 32) {
        if (first_block + n0b * block_stride >= n_end) break;
        RowClip mine;
        mine.lo = 0;
        mine.hi = -1;
        mine.u0 = mine.u1 = mine.u2 = 0;
        long long rl = 0;
        const long long nl = first_block + (n0b + lane) * block_stride;
        if (nl < n_end) {
            rl = nl * nwarps + warp;
            if (rl < R) mine = clip_row(q, (int)(rl % nf1), (int)(rl / nf1), nf0, P.nm);
        }
        const int len = mine.hi >= mine.lo ? mine.hi - mine.lo + 1 : 0;
        int incl = len;  // inclusive scan: the end of this lane's row in the stream
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        // offset of the row's first overlap voxel in the fixed bins (rows past the end are empty)
        const long long rowoff = len > 0 ? rl * nf0 + mine.lo : 0;
        int s = -1, e = 0;  // this lane's row and that row's end in the stream
        unsigned U0 = 0, U1 = 0, U2 = 0;
        const uint8_t *__restrict__ fp = P.fbins;
        for (int g0 = 0; g0 < total;) {
            const int g = g0 + lane;
            bool moved = false;  // warp-uniform
            while (__any_sync(kFull, g < total && g >= e)) {
                if (g < total && g >= e) ++s;
                e = __shfl_sync(kFull, incl, s & 31);
                moved = true;
            }
            if (moved) {  // lanes that stayed re-read their own row: no change
                const int sc = s & 31;
                const int start = e - __shfl_sync(kFull, len, sc);
                const unsigned dd = (unsigned)(g - start);
                U0 = (unsigned)__shfl_sync(kFull, mine.u0, sc) + (unsigned)st0 * dd;
                U1 = (unsigned)__shfl_sync(kFull, mine.u1, sc) + (unsigned)st1 * dd;
                U2 = (unsigned)__shfl_sync(kFull, mine.u2, sc) + (unsigned)st2 * dd;
                fp = P.fbins + (__shfl_sync(kFull, rowoff, sc) + (long long)dd);
            }
            if (g0 + 32 <= total) {
                // a segment of full steps in which no lane leaves its row: predicate-free, two steps per
                // trip, the next step's fixed bin loaded one step ahead
                int nfree = (int)__reduce_min_sync(kFull, (unsigned)((e - g + 31) >> 5));
                nfree = min(nfree, (total - g0) >> 5);
                int bf_next = (int)__ldg(fp);
#pragma unroll 2
                for (int k = 0; k < nfree; ++k) {
                    const int bf = bf_next;
                    fp += 32;
                    if (k + 1 < nfree) bf_next = (int)__ldg(fp);
                    H.add(bf, (sample_value<FM, uint32_t>(P, zoff, U0, U1, U2) * bins) >> mdepth, true);
                    U0 += d0;
                    U1 += d1;
                    U2 += d2;
                }
                g0 += 32 * nfree;
            } else {  // the batch's last, partial step
                const bool valid = g < total;
                int bf = 0, bm = 0;
                if (valid) {
                    bf = (int)__ldg(fp);
                    bm = (sample_value<FM, uint32_t>(P, zoff, U0, U1, U2) * bins) >> mdepth;
                }
                H.add(bf, bm, valid);
                g0 = total;
            }
        }
    }
}

// The voxel walk of a variant: quad and gather fetches over every fixed voxel take the stream walk
// (lpr_log2 == 0) or the row-group walk, the others (and random sampling) the one-row-at-a-time walk.
template <typename PairT, int FM, class Hist>
__device__ __forceinline__ void walk_rows(const PairDev &P, const int *q, const float2 *zoff, long long first_block,
                                          long long block_stride, long long n_end, int lpr_log2, Hist &H) {
    if constexpr (FM == FM_QUAD || FM == FM_GATHER) {
        if (P.srow == nullptr) {
            if (lpr_log2 == 0)
                accumulate_stream<FM>(P, q, zoff, first_block, block_stride, n_end, H);
            else
                accumulate_groups<FM>(P, q, zoff, first_block, block_stride, n_end, lpr_log2, H);
            return;
        }
    }
    accumulate_rows<PairT, FM>(P, q, zoff, first_block, block_stride, n_end, H);
}

// Copies the per-plane atlas offsets of pair P into shared memory (gather fetches only).
template <int FM>
__device__ __forceinline__ void load_zoff(const PairDev &P, float2 *s_zoff) {
    if constexpr (FM == FM_GATHER) {
        for (int z = threadIdx.x; z < P.nm[2]; z += blockDim.x) s_zoff[z] = P.zoff[z];
    }
}

// ---------------------------------------------------------------------------
// Entropy reduction of one histogram by one CTA (Eq. 1, Eq. 2, Tsallis)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double term(uint32_t v, int iq, const QSet &Q) {
    if (v < (uint32_t)kTab) return __ldg(Q.tab[iq] + v);
    const double d = (double)v;
    return Q.q[iq] == 1.0f ? d * log(d) : pow(d, (double)Q.q[iq]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide FP64 sum of three values; every thread gets the results.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    __syncthreads();
    if (lane == 0) {
        s_red[3 * warp + 0] = a;
        s_red[3 * warp + 1] = b;
        s_red[3 * warp + 2] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
    for (int w = 0; w < nwarps; ++w) {
        a += s_red[3 * w + 0];
        b += s_red[3 * w + 1];
        c += s_red[3 * w + 2];
    }
}

// Entropies and MI of transform t from the overlap count N and, per q, the sums over the fixed
// marginal, the moving marginal and the joint cells (res[3 q + 0..2]) of c ln c (q == 1) or c^q:
// H = ln N - S / N (Eq. 1), S_q = (1 - N^-q S) / (q - 1), MI = H_F + H_M - H_FM (Eq. 2) plus
// (1 - q) S_q(F) S_q(M) in the pseudo-additive form.  One thread.
__device__ void write_mi(double N, const double *res, const QSet &Q, long long t, const Outputs &O) {
    const int nq = Q.nq;
    if (O.count) O.count[t] = (long long)N;
    if (N <= 0.0 && O.flags) atomicOr(&O.flags[0], 1);
    for (int iq = 0; iq < nq; ++iq) {
        const float qf = Q.q[iq];
        const double SF = res[3 * iq + 0], SM = res[3 * iq + 1], SJ = res[3 * iq + 2];
        double hf, hm, hj;
        if (N <= 0.0) {
            hf = hm = hj = __longlong_as_double(0x7ff8000000000000ll);
        } else if (qf == 1.0f) {
            const double lnN = log(N);
            hf = lnN - SF / N;
            hm = lnN - SM / N;
            hj = lnN - SJ / N;
            if (Q.bits) {
                const double l2 = log(2.0);
                hf /= l2;
                hm /= l2;
                hj /= l2;
            }
        } else {
            const double q = (double)qf, Nq = pow(N, -q);
            hf = (1.0 - Nq * SF) / (q - 1.0);
            hm = (1.0 - Nq * SM) / (q - 1.0);
            hj = (1.0 - Nq * SJ) / (q - 1.0);
        }
        double I = hf + hm - hj;
        if (qf != 1.0f && Q.form == 1) I += (1.0 - (double)qf) * hf * hm;
        if (O.mi) O.mi[t * nq + iq] = I;
        if (O.h) {
            O.h[(t * nq + iq) * 3 + 0] = hf;
            O.h[(t * nq + iq) * 3 + 1] = hm;
            O.h[(t * nq + iq) * 3 + 2] = hj;
        }
    }
}

// Entropies of one histogram by one CTA.  Pass 1: marginals (row sums by
// warps, column sums by shared atomics) and N.  Then one pass per q over the
// non-zero cells and the marginals, with one FP64 accumulator triple live at a
// time: sum c ln c (q == 1) or sum c^q (count-indexed tables for c < kTab).
template <class Hist>
__device__ void reduce_entropies(const Hist &H, int B, const QSet &Q, uint32_t *s_rows, uint32_t *s_cols,
                                 double *s_red, long long t, const Outputs &O) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nq = Q.nq;
    double *s_res = s_red + 3 * 32;  // 3 nq + 1 results after the per-warp scratch
    for (int c = tid; c < B; c += blockDim.x) s_cols[c] = 0;
    __syncthreads();
    for (int r = warp; r < B; r += nwarps) {
        uint32_t rsum = 0;
        for (int c = lane; c < B; c += 32) {
            const uint32_t v = H.count(r, c);
            if (v) {
                rsum += v;
                atomicAdd(&s_cols[c], v);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(kFull, rsum, o);
        if (lane == 0) s_rows[r] = rsum;
    }
    __syncthreads();
    {
        double n0 = 0.0, z1 = 0.0, z2 = 0.0;
        for (int r = tid; r < B; r += blockDim.x) n0 += (double)s_rows[r];
        block_sum3(n0, z1, z2, s_red);
        if (tid == 0) s_res[3 * kMaxQ] = n0;
    }
    for (int iq = 0; iq < nq; ++iq) {
        double aj = 0.0, af = 0.0, am = 0.0;
        for (int r = warp; r < B; r += nwarps)
            for (int c = lane; c < B; c += 32) {
                const uint32_t v = H.count(r, c);
                if (v) aj += term(v, iq, Q);
            }
        for (int r = tid; r < B; r += blockDim.x) {
            const uint32_t vf = s_rows[r], vm = s_cols[r];
            if (vf) af += term(vf, iq, Q);
            if (vm) am += term(vm, iq, Q);
        }
        block_sum3(af, am, aj, s_red);
        if (tid == 0) {
            s_res[3 * iq + 0] = af;
            s_res[3 * iq + 1] = am;
            s_res[3 * iq + 2] = aj;
        }
    }
    __syncthreads();
    if (tid == 0) write_mi(s_res[3 * kMaxQ], s_res, Q, t, O);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Plain form
// ---------------------------------------------------------------------------

template <typename PairT, int HV, int FM>
__global__ void __launch_bounds__(1024, 1)
    k_hist(const PairDev *__restrict__ pairs, const int32_t *__restrict__ aff, uint32_t *__restrict__ ghist,
           int *flags, Tile tile) {
    extern __shared__ __align__(16) unsigned char smem[];
    const PairDev P = pairs[0];
    const int t = blockIdx.y;
    const int B = P.bins;
    const SmemLayout L = smem_layout(HV, B, blockDim.x, P.rows_words, P.nm[2]);
    __shared__ int q[12];
    if (threadIdx.x < 12) q[threadIdx.x] = aff[(size_t)t * 12 + threadIdx.x];
    float2 *s_zoff = (float2 *)(smem + L.zoff);
    load_zoff<FM>(P, s_zoff);
    auto H = make_hist<HV>(smem, L, B, flags, P.rows_words);
    H.load_info(P.rowinfo);
    H.zero();
    __syncthreads();
    const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    walk_rows<PairT, FM>(P, q, s_zoff, blockIdx.x, gridDim.x, ((long long)P.nf[1] * P.nf[2] + nwarps - 1) / nwarps,
                         tile.lpr_log2, H);
    __syncthreads();
    uint32_t *gh = ghist + (size_t)t * B * B;
    for (int r = threadIdx.x >> 5; r < B; r += nwarps)
        for (int c = lane; c < B; c += 32) {
            const uint32_t v = H.count(r, c);
            if (v) atomicAdd(gh + r * B + c, v);
        }
}

// Shared memory of k_entropy: [rows B u32][cols B u32][FP64 scratch, 16-byte aligned].
__host__ __device__ inline size_t entropy_red_offset(int B) { return align_up((size_t)B * 8, 16); }
__host__ __device__ inline size_t entropy_smem_bytes(int B, int threads) {
    return entropy_red_offset(B) + (size_t)(3 * 32 + 3 * kMaxQ + 1) * 8;
}

__global__ void __launch_bounds__(1024, 1)
    k_entropy(const uint32_t *__restrict__ ghist, int B, QSet Q, Outputs O) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long t = blockIdx.x;
    HistGlobal H{ghist + (size_t)t * B * B, B};
    reduce_entropies(H, B, Q, (uint32_t *)smem, (uint32_t *)(smem + (size_t)B * 4),
                     (double *)(smem + entropy_red_offset(B)), t, O);
}

// The same reduction split over `parts` CTAs per transform, for calls with few transforms (the plain
// form's one-transform calls), where one CTA per transform would leave the GPU idle.  CTA (p, t) takes
// rows p, p + parts, ... of histogram t: their sums (the fixed marginal) and terms, the joint terms of
// their cells and their part of the column sums (the moving marginal, into cols[t], zeroed by the
// caller).  part[(t parts + p) (1 + 2 kMaxQ)]: the count, then per q the joint and fixed-marginal sums.
constexpr int kPartStride = 1 + 2 * kMaxQ;

__global__ void __launch_bounds__(256)
    k_entropy_part(const uint32_t *__restrict__ ghist, int B, QSet Q, uint32_t *__restrict__ cols,
                   double *__restrict__ part, int parts) {
    __shared__ uint32_t s_cols[256];
    __shared__ double s_red[3 * 32];
    const int t = blockIdx.y, p = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const uint32_t *h = ghist + (size_t)t * B * B;
    for (int c = tid; c < B; c += blockDim.x) s_cols[c] = 0;
    __syncthreads();
    double n = 0.0, aj[kMaxQ], af[kMaxQ];
#pragma unroll
    for (int iq = 0; iq < kMaxQ; ++iq) aj[iq] = af[iq] = 0.0;
    for (int r = p + parts * warp; r < B; r += parts * nwarps) {
        uint32_t rsum = 0;
        for (int c = lane; c < B; c += 32) {
            const uint32_t v = __ldg(h + (size_t)r * B + c);
            if (v) {
                rsum += v;
                atomicAdd(&s_cols[c], v);
#pragma unroll
                for (int iq = 0; iq < kMaxQ; ++iq)
                    if (iq < Q.nq) aj[iq] += term(v, iq, Q);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(kFull, rsum, o);
        if (lane == 0 && rsum) {
            n += (double)rsum;
#pragma unroll
            for (int iq = 0; iq < kMaxQ; ++iq)
                if (iq < Q.nq) af[iq] += term(rsum, iq, Q);
        }
    }
    __syncthreads();
    for (int c = tid; c < B; c += blockDim.x)
        if (s_cols[c]) atomicAdd(cols + (size_t)t * B + c, s_cols[c]);
    double *out = part + ((size_t)t * parts + p) * kPartStride;
    double z = 0.0;
    block_sum3(n, z, z, s_red);
    if (tid == 0) out[0] = n;
    for (int iq = 0; iq < Q.nq; ++iq) {
        double a = aj[iq], b = af[iq];
        z = 0.0;
        block_sum3(a, b, z, s_red);
        if (tid == 0) {
            out[1 + 2 * iq] = a;
            out[2 + 2 * iq] = b;
        }
    }
}

// Finishes the split reduction: the moving-marginal terms from cols[t], the parts' sums, then MI.
__global__ void __launch_bounds__(256)
    k_entropy_final(const uint32_t *__restrict__ cols, const double *__restrict__ part, int parts, int B, QSet Q,
                    Outputs O) {
    __shared__ double s_red[3 * 32];
    __shared__ double s_res[3 * kMaxQ + 1];
    const int t = blockIdx.x, tid = threadIdx.x;
    for (int iq = 0; iq < Q.nq; ++iq) {
        double am = 0.0, z0 = 0.0, z1 = 0.0;
        for (int c = tid; c < B; c += blockDim.x) {
            const uint32_t v = cols[(size_t)t * B + c];
            if (v) am += term(v, iq, Q);
        }
        block_sum3(am, z0, z1, s_red);
        if (tid == 0) {
            double sj = 0.0, sf = 0.0;
            for (int p = 0; p < parts; ++p) {
                const double *in = part + ((size_t)t * parts + p) * kPartStride;
                sj += in[1 + 2 * iq];
                sf += in[2 + 2 * iq];
            }
            s_res[3 * iq + 0] = sf;
            s_res[3 * iq + 1] = am;
            s_res[3 * iq + 2] = sj;
        }
    }
    if (tid == 0) {
        double N = 0.0;
        for (int p = 0; p < parts; ++p) N += part[((size_t)t * parts + p) * kPartStride];
        write_mi(N, s_res, Q, t, O);
    }
}

// ---------------------------------------------------------------------------
// Batched form: persistent CTAs, one (pair, transform) item per CTA at a time
// ---------------------------------------------------------------------------

template <int HV, int FM>
__global__ void __launch_bounds__(1024, 1)
    k_batched(const PairDev *__restrict__ pairs, const int32_t *__restrict__ aff, const Item *__restrict__ items,
              int nitems, int *ticket, int max_bins, int rows_words, int zmax, Tile tile, QSet Q, Outputs O) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_slab;
    __shared__ int q[12];
    const SmemLayout L = smem_layout(HV, max_bins, blockDim.x, rows_words, zmax);
    float2 *s_zoff = (float2 *)(smem + L.zoff);
    const int nwarps = blockDim.x >> 5;
    const int slabs = tile.slabs;
    int *phase = ticket + 1;  // the slab most recently started by any CTA
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const Item I = items[it];
        const PairDev P = pairs[I.pair];
        const int B = P.bins;
        if (threadIdx.x < 12) q[threadIdx.x] = aff[(size_t)I.t * 12 + threadIdx.x];
        load_zoff<FM>(P, s_zoff);
        auto H = make_hist<HV>(smem, L, B, O.flags, P.rows_words);
        H.load_info(P.rowinfo);
        H.zero();
        __syncthreads();
        // The sweep is cut into `slabs` slabs of row blocks, done in any order (counts do not depend
        // on it).  Each slab goes to the first remaining one at or after the slab most recently
        // started by any CTA, so CTAs working on different transforms keep to neighbouring slabs
        // of the volumes and their working set stays in L2.  No CTA waits for another.
        const long long NB = ((long long)P.nf[1] * P.nf[2] + nwarps - 1) / nwarps;
        const long long SB = (NB + slabs - 1) / slabs;
        unsigned left = (1u << slabs) - 1u;
        while (left) {
            if (threadIdx.x == 0) {
                int k = *(volatile int *)phase;
                k = k < 0 || k >= slabs ? 0 : k;
                while (!((left >> k) & 1u)) k = k + 1 == slabs ? 0 : k + 1;
                s_slab = k;
                *(volatile int *)phase = k;
            }
            __syncthreads();
            const int k = s_slab;
            left &= ~(1u << k);
            const long long b0 = (long long)k * SB, b1 = b0 + SB < NB ? b0 + SB : NB;
            if (b0 < b1) {
                // quads and gathers are unpacked by the texture unit: one instance
                if (FM == FM_QUAD || FM == FM_GATHER || P.mdtype == 1)
                    walk_rows<uint32_t, FM>(P, q, s_zoff, b0, 1, b1, tile.lpr_log2, H);
                else
                    walk_rows<uint16_t, FM>(P, q, s_zoff, b0, 1, b1, tile.lpr_log2, H);
            }
            __syncthreads();  // s_slab is rewritten for the next slab
        }
        __syncthreads();
        if (O.dump) {
            uint32_t *dh = O.dump + (size_t)I.t * B * B;
            for (int r = threadIdx.x >> 5; r < B; r += nwarps)
                for (int c = threadIdx.x & 31; c < B; c += 32) dh[r * B + c] = H.count(r, c);
        }
        reduce_entropies(H, P.bins, Q, (uint32_t *)(smem + L.rows), (uint32_t *)(smem + L.cols),
                         (double *)(smem + L.red), I.t, O);
    }
}

// ---------------------------------------------------------------------------
// Resampling v(T(x)) on the fixed grid
// ---------------------------------------------------------------------------

template <typename MovT>
__global__ void k_resample(const PairDev *__restrict__ pairs, const int32_t *__restrict__ aff, MovT *__restrict__ out) {
    const PairDev P = pairs[0];
    const long long n = (long long)P.nf[0] * P.nf[1] * P.nf[2];
    int q[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) q[e] = aff[e];
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        const long long i = x % P.nf[0], j = (x / P.nf[0]) % P.nf[1], k = x / ((long long)P.nf[0] * P.nf[1]);
        long long U[3];
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            U[a] = (long long)q[4 * a] * i + (long long)q[4 * a + 1] * j + (long long)q[4 * a + 2] * k + q[4 * a + 3];
            in = in && U[a] >= 0 && U[a] <= ((long long)(P.nm[a] - 1) << 16);
        }
        out[x] = in ? (MovT)sample_hard<MovT>((const MovT *)P.mov, P.nm[0], P.nm[1], P.nm[2], (int)U[0], (int)U[1],
                                               (int)U[2])
                    : (MovT)0;
    }
}

inline int grid_for(long long n, int threads) {
    long long g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t hard_smem_bytes(int variant, int bins, int threads, int rows_words, int zmax) {
    return smem_layout(variant, bins, threads, rows_words, zmax).total;
}

// MurmurHash3's 32-bit finalizer: xor-shift 16, multiply 0x85ebca6b, xor-shift 13, multiply 0xc2b2ae35,
// xor-shift 16 (mod 2^32).
__host__ __device__ inline uint32_t fmix32(uint32_t k) {
    k ^= k >> 16;
    k *= 0x85ebca6bu;
    k ^= k >> 13;
    k *= 0xc2b2ae35u;
    k ^= k >> 16;
    return k;
}

// One thread per fixed row: how many of its voxels are sampled (hseed = fmix32(seed)).
__global__ void k_sample_count(int n0, long long R, uint32_t hseed, uint32_t thr, uint32_t *__restrict__ counts) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R; r += (long long)gridDim.x * blockDim.x) {
        uint32_t c = 0;
        const uint32_t x0 = (uint32_t)(r * n0);
        for (int i = 0; i < n0; ++i) c += fmix32((x0 + (uint32_t)i) ^ hseed) < thr ? 1u : 0u;
        counts[r] = c;
    }
}

// One thread per fixed row: its sampled voxels' x indices (ascending) and fixed bins.
__global__ void k_sample_fill(int n0, long long R, uint32_t hseed, uint32_t thr, const uint8_t *__restrict__ fbins,
                              const uint32_t *__restrict__ row_ptr, uint16_t *__restrict__ cols,
                              uint8_t *__restrict__ bins) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R; r += (long long)gridDim.x * blockDim.x) {
        uint32_t o = row_ptr[r];
        const uint32_t x0 = (uint32_t)(r * n0);
        for (int i = 0; i < n0; ++i)
            if (fmix32((x0 + (uint32_t)i) ^ hseed) < thr) {
                cols[o] = (uint16_t)i;
                bins[o] = fbins[(size_t)r * n0 + i];
                ++o;
            }
    }
}

__global__ void k_fixed_hist(const uint8_t *__restrict__ fb, long long n, int bins, unsigned long long *__restrict__ out) {
    __shared__ unsigned int h[256];
    for (int c = threadIdx.x; c < 256; c += blockDim.x) h[c] = 0;
    __syncthreads();
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
        atomicAdd(&h[fb[x]], 1u);
    __syncthreads();
    for (int c = threadIdx.x; c < bins; c += blockDim.x)
        if (h[c]) atomicAdd(out + c, (unsigned long long)h[c]);
}

cudaError_t launch_sample_count(int n0, long long R, uint32_t seed, uint32_t threshold, uint32_t *counts,
                                cudaStream_t s) {
    k_sample_count<<<grid_for(R, 256), 256, 0, s>>>(n0, R, fmix32(seed), threshold, counts);
    return cudaGetLastError();
}

cudaError_t launch_sample_fill(int n0, long long R, uint32_t seed, uint32_t threshold, const uint8_t *fbins,
                               const uint32_t *row_ptr, uint16_t *cols, uint8_t *bins, cudaStream_t s) {
    k_sample_fill<<<grid_for(R, 256), 256, 0, s>>>(n0, R, fmix32(seed), threshold, fbins, row_ptr, cols, bins);
    return cudaGetLastError();
}

cudaError_t launch_fixed_hist(const uint8_t *fbins, long long n, int bins, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)bins * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long g = (n + 255) / 256;
    if (g > 1024) g = 1024;
    k_fixed_hist<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(fbins, n, bins, out);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_u16(const float *in, long long n, uint16_t *out, cudaStream_t s) {
    k_f32_to_u16<<<grid_for(n, 256), 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_clamp_depth(void *data, int dtype, int depth, long long n, cudaStream_t s) {
    const uint32_t vmax = (uint32_t)((1ull << depth) - 1ull);
    if (dtype == 0) {
        if (depth >= 8) return cudaSuccess;
        k_clamp_depth<uint8_t><<<grid_for(n, 256), 256, 0, s>>>((uint8_t *)data, n, vmax);
    } else {
        if (depth >= 16) return cudaSuccess;
        k_clamp_depth<uint16_t><<<grid_for(n, 256), 256, 0, s>>>((uint16_t *)data, n, vmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_make_pairs(const void *mov, int dtype, const int nm[3], void *out, cudaStream_t s) {
    const long long n = (long long)nm[0] * (nm[1] + 1) * (nm[2] + 1);
    if (dtype == 0)
        k_make_pairs<uint8_t, uint16_t><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)mov, nm[0], nm[1], nm[2],
                                                                          (uint16_t *)out);
    else
        k_make_pairs<uint16_t, uint32_t><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)mov, nm[0], nm[1], nm[2],
                                                                           (uint32_t *)out);
    return cudaGetLastError();
}

cudaError_t launch_make_zpairs(const void *mov, int dtype, const int nm[3], int ph, int W, int H, uint32_t *out,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)W * H * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)nm[0] * nm[1] * nm[2];
    if (dtype == 0)
        k_make_zpairs<uint8_t><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)mov, nm[0], nm[1], nm[2], ph, W, out);
    else
        k_make_zpairs<uint16_t><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)mov, nm[0], nm[1], nm[2], ph, W, out);
    return cudaGetLastError();
}

cudaError_t launch_make_quads(const void *mov, int dtype, const int nm[3], void *out, cudaStream_t s) {
    const long long n = (long long)nm[0] * nm[1] * nm[2];
    if (dtype == 0)
        k_make_quads<uint8_t, uchar4><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)mov, nm[0], nm[1], nm[2],
                                                                        (uchar4 *)out);
    else
        k_make_quads<uint16_t, ushort4><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)mov, nm[0], nm[1], nm[2],
                                                                          (ushort4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_bin_fixed(const void *data, int dtype, int depth, long long n, int bins, uint8_t *out,
                             cudaStream_t s) {
    if (dtype == 0)
        k_bin_fixed<uint8_t><<<grid_for(n, 256), 256, 0, s>>>((const uint8_t *)data, n, depth, bins, out);
    else
        k_bin_fixed<uint16_t><<<grid_for(n, 256), 256, 0, s>>>((const uint16_t *)data, n, depth, bins, out);
    return cudaGetLastError();
}

cudaError_t launch_table(double *tab, float q, cudaStream_t s) {
    k_table<<<kTab / 256, 256, 0, s>>>(tab, q);
    return cudaGetLastError();
}

// Every variant as (public value, counter kind, fetch mode): those that read x-pairs (whose element
// type follows the moving type) and those whose texels the texture unit unpacks (one instance each).
#define MI_VARIANTS_PAIRED(X)                                                                       \
    X(HV_U32, HV_U32, FM_LDG) X(HV_U32_MATCH, HV_U32_MATCH, FM_LDG) X(HV_U16, HV_U16, FM_LDG)        \
    X(HV_U16_MATCH, HV_U16_MATCH, FM_LDG) X(HV_TEX + HV_U32, HV_U32, FM_TEX)                        \
    X(HV_TEX + HV_U32_MATCH, HV_U32_MATCH, FM_TEX) X(HV_TEX + HV_U16, HV_U16, FM_TEX)                \
    X(HV_TEX + HV_U16_MATCH, HV_U16_MATCH, FM_TEX) X(HV_ROWS, HV_ROWS, FM_LDG)                      \
    X(HV_ROWS_TEX, HV_ROWS, FM_TEX)
#define MI_VARIANTS_TEXEL(X)                                                                        \
    X(HV_ROWS_QUAD, HV_ROWS, FM_QUAD) X(HV_U32_QUAD, HV_U32, FM_QUAD) X(HV_U16_QUAD, HV_U16, FM_QUAD) \
    X(HV_ROWS_GATHER, HV_ROWS, FM_GATHER) X(HV_U32_GATHER, HV_U32, FM_GATHER)                       \
    X(HV_U16_GATHER, HV_U16, FM_GATHER)
#define MI_VARIANTS(X) MI_VARIANTS_PAIRED(X) MI_VARIANTS_TEXEL(X)

template <typename MT>
static const void *plain_fn_of(int variant) {
    switch (variant) {
#define MI_PLAIN_CASE(V, K, F) \
    case V: return (const void *)k_hist<MT, K, F>;
        MI_VARIANTS_PAIRED(MI_PLAIN_CASE)
#undef MI_PLAIN_CASE
        default: return nullptr;
    }
}

static const void *plain_fn(int variant, int mdtype) {
    switch (variant) {
#define MI_PLAIN_CASE(V, K, F) \
    case V: return (const void *)k_hist<uint32_t, K, F>;
        MI_VARIANTS_TEXEL(MI_PLAIN_CASE)
#undef MI_PLAIN_CASE
        default: return mdtype == 0 ? plain_fn_of<uint16_t>(variant) : plain_fn_of<uint32_t>(variant);
    }
}

cudaError_t launch_plain_hist(const PairDev *d_pair, const PairDev &h_pair, const int32_t *d_aff, int n,
                              uint32_t *d_hist, int variant, int threads, int ctas, Tile tile, int *d_flags,
                              cudaStream_t s) {
    const size_t B2 = (size_t)h_pair.bins * h_pair.bins;
    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)n * B2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const size_t smem = smem_layout(variant, h_pair.bins, threads, h_pair.rows_words, h_pair.nm[2]).total;
    const void *fn = plain_fn(variant, h_pair.mdtype);
    if (!fn) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    void *args[] = {(void *)&d_pair, (void *)&d_aff, (void *)&d_hist, (void *)&d_flags, (void *)&tile};
    return cudaLaunchKernel(fn, dim3(ctas, n), dim3(threads), args, smem, s);
}

cudaError_t launch_entropy(const uint32_t *d_hist, int n, int bins, const QSet &Q, const Outputs &O, cudaStream_t s) {
    const int threads = 1024;
    const size_t smem = entropy_smem_bytes(bins, threads);
    cudaError_t e = set_smem(k_entropy, smem);
    if (e != cudaSuccess) return e;
    k_entropy<<<n, threads, smem, s>>>(d_hist, bins, Q, O);
    return cudaGetLastError();
}

int entropy_parts(int bins) { return bins >= 256 ? 32 : (bins / 8 > 1 ? bins / 8 : 1); }

cudaError_t launch_entropy_split(const uint32_t *d_hist, int n, int bins, const QSet &Q, const Outputs &O,
                                 uint32_t *d_cols, double *d_part, cudaStream_t s) {
    const int parts = entropy_parts(bins);
    cudaError_t e = cudaMemsetAsync(d_cols, 0, (size_t)n * bins * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_entropy_part<<<dim3(parts, n), 256, 0, s>>>(d_hist, bins, Q, d_cols, d_part, parts);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_entropy_final<<<n, 256, 0, s>>>(d_cols, d_part, parts, bins, Q, O);
    return cudaGetLastError();
}

static const void *batched_fn(int variant) {
    switch (variant) {
#define MI_BATCHED_CASE(V, K, F) \
    case V: return (const void *)k_batched<K, F>;
        MI_VARIANTS(MI_BATCHED_CASE)
#undef MI_BATCHED_CASE
        default: return nullptr;
    }
}

int batched_ctas_per_sm(int variant, int max_bins, int threads, int rows_words, int zmax) {
    const size_t smem = smem_layout(variant, max_bins, threads, rows_words, zmax).total;
    const void *fn = batched_fn(variant);
    if (!fn) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_batched(const PairDev *d_pairs, const int32_t *d_aff, const Item *d_items, int nitems,
                           int *d_ticket, int max_bins, int rows_words, int zmax, int variant, int threads, int ctas,
                           Tile tile, const QSet &Q, const Outputs &O, cudaStream_t s) {
    const size_t smem = smem_layout(variant, max_bins, threads, rows_words, zmax).total;
    const void *fn = batched_fn(variant);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&d_pairs, (void *)&d_aff, (void *)&d_items, (void *)&nitems, (void *)&d_ticket,
                    (void *)&max_bins, (void *)&rows_words, (void *)&zmax, (void *)&tile, (void *)&Q, (void *)&O};
    return cudaLaunchKernel(fn, dim3(ctas), dim3(threads), args, smem, s);
}

cudaError_t launch_resample(const PairDev *d_pair, const PairDev &h_pair, const int32_t *d_aff, void *out,
                            cudaStream_t s) {
    const long long n = (long long)h_pair.nf[0] * h_pair.nf[1] * h_pair.nf[2];
    if (h_pair.mdtype == 0)
        k_resample<uint8_t><<<grid_for(n, 256), 256, 0, s>>>(d_pair, d_aff, (uint8_t *)out);
    else
        k_resample<uint16_t><<<grid_for(n, 256), 256, 0, s>>>(d_pair, d_aff, (uint16_t *)out);
    return cudaGetLastError();
}

cudaError_t set_drain_cap(int cap) { return cudaMemcpyToSymbol(g_drain_cap, &cap, sizeof cap); }

}  // namespace mi

// ===========================================================================
// Allocation-free variant of the plain path (entry point in mi_noalloc.cu):
// the fixed volume is binned on the fly from its raw values, the histogram
// lives in caller-provided scratch (a static device array), and the entropy
// terms are evaluated directly in FP64 instead of from count-indexed tables.
// ===========================================================================

namespace mi {
namespace {

struct RawPair {
    const void *fix;
    const void *mov;
    int nf[3], nm[3];
    int bins, fdepth, mdepth;
};

struct Q12 {
    int q[12];
};

// sample_hard on a volume used as given: each of the 8 neighbours is clamped to vmax = 2^d - 1 as it
// is read, as the context path clamps every voxel when it copies the volume.
template <typename MovT>
__device__ __forceinline__ int sample_hard_raw(const MovT *__restrict__ mov, int n0, int n1, int n2, int ux, int uy,
                                               int uz, int vmax) {
    const int ix = ux >> 16, iy = uy >> 16, iz = uz >> 16;
    const int fx = (ux >> 8) & 255, fy = (uy >> 8) & 255, fz = (uz >> 8) & 255;
    const int sx = ix < n0 - 1 ? 1 : 0;
    const int sy = iy < n1 - 1 ? n0 : 0;
    const int sz = iz < n2 - 1 ? n0 * n1 : 0;
    const MovT *p = mov + (ix + n0 * (iy + n1 * iz));
    const int v000 = min((int)__ldg(p), vmax), v001 = min((int)__ldg(p + sx), vmax);
    const int v010 = min((int)__ldg(p + sy), vmax), v011 = min((int)__ldg(p + sy + sx), vmax);
    const int v100 = min((int)__ldg(p + sz), vmax), v101 = min((int)__ldg(p + sz + sx), vmax);
    const int v110 = min((int)__ldg(p + sz + sy), vmax), v111 = min((int)__ldg(p + sz + sy + sx), vmax);
    const int e00 = lerp8(v000, v001, fx), e01 = lerp8(v010, v011, fx);
    const int e10 = lerp8(v100, v101, fx), e11 = lerp8(v110, v111, fx);
    const int g0 = lerp8(e00, e01, fy), g1 = lerp8(e10, e11, fy);
    return lerp8(g0, g1, fz);
}

template <typename FixT, typename MovT, class Hist>
__device__ void accumulate_rows_raw(const RawPair &P, const int *q, long long first_batch, long long batch_stride,
                                    Hist &H) {
    const int lane = threadIdx.x & 31;
    const int nf0 = P.nf[0], nf1 = P.nf[1];
    const long long R = (long long)nf1 * P.nf[2];
    const int n0 = P.nm[0], n1 = P.nm[1], n2 = P.nm[2];
    const int st0 = q[0], st1 = q[4], st2 = q[8];
    const int bins = P.bins, mdepth = P.mdepth, fdepth = P.fdepth;
    const uint32_t fvmax = (uint32_t)((1ull << fdepth) - 1ull);
    const MovT *__restrict__ mov = (const MovT *)P.mov;
    for (long long rb = first_batch * 32; rb < R; rb += batch_stride * 32) {
        RowClip mine;
        mine.lo = 0;
        mine.hi = -1;
        mine.u0 = mine.u1 = mine.u2 = 0;
        const long long r = rb + lane;
        if (r < R) mine = clip_row(q, (int)(r % nf1), (int)(r / nf1), nf0, P.nm);
        for (int s = 0; s < 32; ++s) {
            const int lo = __shfl_sync(kFull, mine.lo, s), hi = __shfl_sync(kFull, mine.hi, s);
            if (lo > hi) continue;
            const int U0 = __shfl_sync(kFull, mine.u0, s), U1 = __shfl_sync(kFull, mine.u1, s),
                      U2 = __shfl_sync(kFull, mine.u2, s);
            const FixT *__restrict__ frow = (const FixT *)P.fix + (size_t)(rb + s) * nf0;
            for (int i0 = lo; i0 <= hi; i0 += 32) {
                const int i = i0 + lane;
                const bool valid = i <= hi;
                int bf = 0, bm = 0;
                if (valid) {
                    const int d = i - lo;
                    // volumes are read in place; each value is clamped to its bit depth as it is read
                    const int v = sample_hard_raw<MovT>(mov, n0, n1, n2, U0 + st0 * d, U1 + st1 * d, U2 + st2 * d,
                                                        (int)((1u << mdepth) - 1u));
                    bm = (v * bins) >> mdepth;
                    uint32_t fv = (uint32_t)__ldg(frow + i);
                    fv = fv > fvmax ? fvmax : fv;
                    bf = (int)((fv * (uint32_t)bins) >> fdepth);
                }
                H.add(bf, bm, valid);
            }
        }
    }
}

template <typename FixT, typename MovT>
__global__ void __launch_bounds__(1024, 1) k_hist_raw(RawPair P, Q12 A, uint32_t *__restrict__ ghist, int *flags) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = P.bins;
    const SmemLayout L = smem_layout(HV_U16_MATCH, B, blockDim.x, 0, 0);
    __shared__ int q[12];
    if (threadIdx.x < 12) q[threadIdx.x] = A.q[threadIdx.x];
    auto H = make_hist<HV_U16_MATCH>(smem, L, B, flags);
    H.zero();
    __syncthreads();
    const int nwarps = blockDim.x >> 5;
    accumulate_rows_raw<FixT, MovT>(P, q, (long long)blockIdx.x * nwarps + (threadIdx.x >> 5),
                                    (long long)gridDim.x * nwarps, H);
    __syncthreads();
    for (int r = threadIdx.x >> 5; r < B; r += nwarps)
        for (int c = threadIdx.x & 31; c < B; c += 32) {
            const uint32_t v = H.count(r, c);
            if (v) atomicAdd(ghist + r * B + c, v);
        }
}

// Entropy term of one count, evaluated directly in FP64: c ln c or c^q.
__device__ __forceinline__ double term_direct(uint32_t v, float qf) {
    const double d = (double)v;
    return qf == 1.0f ? d * log(d) : pow(d, (double)qf);
}

// One CTA: marginals, FP64 sums per q and MI from a global histogram.
// out: nq MI values, then nq x 3 entropies, then the overlap count (as a double).
__global__ void __launch_bounds__(1024, 1)
    k_entropy_direct(const uint32_t *__restrict__ ghist, int B, QSet Q, double *__restrict__ out, int *flags) {
    __shared__ uint32_t s_rows[256], s_cols[256];
    __shared__ double s_red[3 * 32];
    __shared__ double s_res[3 * kMaxQ + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int c = tid; c < B; c += blockDim.x) s_cols[c] = 0;
    __syncthreads();
    for (int r = warp; r < B; r += nwarps) {
        uint32_t rsum = 0;
        for (int c = lane; c < B; c += 32) {
            const uint32_t v = __ldg(ghist + r * B + c);
            if (v) {
                rsum += v;
                atomicAdd(&s_cols[c], v);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(kFull, rsum, o);
        if (lane == 0) s_rows[r] = rsum;
    }
    __syncthreads();
    {
        double n0 = 0.0, z1 = 0.0, z2 = 0.0;
        for (int r = tid; r < B; r += blockDim.x) n0 += (double)s_rows[r];
        block_sum3(n0, z1, z2, s_red);
        if (tid == 0) s_res[3 * kMaxQ] = n0;
    }
    for (int iq = 0; iq < Q.nq; ++iq) {
        double aj = 0.0, af = 0.0, am = 0.0;
        for (int c = tid; c < B * B; c += blockDim.x) {
            const uint32_t v = __ldg(ghist + c);
            if (v) aj += term_direct(v, Q.q[iq]);
        }
        for (int r = tid; r < B; r += blockDim.x) {
            if (s_rows[r]) af += term_direct(s_rows[r], Q.q[iq]);
            if (s_cols[r]) am += term_direct(s_cols[r], Q.q[iq]);
        }
        block_sum3(af, am, aj, s_red);
        if (tid == 0) {
            s_res[3 * iq + 0] = af;
            s_res[3 * iq + 1] = am;
            s_res[3 * iq + 2] = aj;
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double N = s_res[3 * kMaxQ];
        out[4 * Q.nq] = N;
        if (N <= 0.0) atomicOr(&flags[0], 1);
        for (int iq = 0; iq < Q.nq; ++iq) {
            const float qf = Q.q[iq];
            const double SF = s_res[3 * iq + 0], SM = s_res[3 * iq + 1], SJ = s_res[3 * iq + 2];
            double hf, hm, hj;
            if (N <= 0.0) {
                hf = hm = hj = __longlong_as_double(0x7ff8000000000000ll);
            } else if (qf == 1.0f) {
                const double lnN = log(N);
                hf = lnN - SF / N;
                hm = lnN - SM / N;
                hj = lnN - SJ / N;
                if (Q.bits) {
                    const double l2 = log(2.0);
                    hf /= l2;
                    hm /= l2;
                    hj /= l2;
                }
            } else {
                const double qd = (double)qf, Nq = pow(N, -qd);
                hf = (1.0 - Nq * SF) / (qd - 1.0);
                hm = (1.0 - Nq * SM) / (qd - 1.0);
                hj = (1.0 - Nq * SJ) / (qd - 1.0);
            }
            double I = hf + hm - hj;
            if (qf != 1.0f && Q.form == 1) I += (1.0 - (double)qf) * hf * hm;
            out[iq] = I;
            out[Q.nq + 3 * iq + 0] = hf;
            out[Q.nq + 3 * iq + 1] = hm;
            out[Q.nq + 3 * iq + 2] = hj;
        }
    }
}

}  // namespace

cudaError_t launch_noalloc_eval(const void *fix, int fdtype, int fdepth, const void *mov, int mdtype, int mdepth,
                                const int nf[3], const int nm[3], int bins, const int32_t q16[12], const QSet &Q,
                                uint32_t *hist, int *flags, double *out, int ctas, cudaStream_t s) {
    RawPair P;
    P.fix = fix;
    P.mov = mov;
    for (int a = 0; a < 3; ++a) {
        P.nf[a] = nf[a];
        P.nm[a] = nm[a];
    }
    P.bins = bins;
    P.fdepth = fdepth;
    P.mdepth = mdepth;
    Q12 A;
    for (int e = 0; e < 12; ++e) A.q[e] = q16[e];
    const int threads = 1024;
    const size_t smem = smem_layout(HV_U16_MATCH, bins, threads, 0, 0).total;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)bins * bins * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
#define MI_RAW(FT, MT)                                                                     \
    do {                                                                                   \
        if ((e = set_smem(k_hist_raw<FT, MT>, smem)) != cudaSuccess) return e;            \
        k_hist_raw<FT, MT><<<ctas, threads, smem, s>>>(P, A, hist, flags);                 \
    } while (0)
    if (fdtype == 0 && mdtype == 0) MI_RAW(uint8_t, uint8_t);
    else if (fdtype == 0) MI_RAW(uint8_t, uint16_t);
    else if (mdtype == 0) MI_RAW(uint16_t, uint8_t);
    else MI_RAW(uint16_t, uint16_t);
#undef MI_RAW
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_entropy_direct<<<1, 1024, 0, s>>>(hist, bins, Q, out, flags);
    return cudaGetLastError();
}

}  // namespace mi
