// mi_internal.h -- types and launchers shared by the library's CUDA sources.
// Not installed; the public boundary is include/mi.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mi {

constexpr int kMaxQ = 8;
constexpr int kTab = 65536;        // count-indexed FP64 tables cover counts < kTab
constexpr int kDrainT = 1 << 14;   // 16-bit counters are drained once they reach 2^14
constexpr int kOvfSlots = 4096;    // drain table entries (each entry holds >= kDrainT counts)

// One volume pair as the hard-path kernels see it.
struct PairDev {
    const uint8_t *fbins;  // fixed volume pre-binned to uint8, x fastest
    const void *mov;       // moving volume, uint8 or uint16, clamped to its bit depth
    const void *movp;      // x-paired copy (v[x], v[x+1]), uint16 / uint32, dims (nx, ny + 1, nz + 1)
    unsigned long long texp;  // the same pairs as a 3D texture (point sampling, clamped), dims (nx, ny, nz)
    unsigned long long texq;  // 2 x 2 quads (y, z), (y + 1, z), (y, z + 1), (y + 1, z + 1) as a 3D texture
    unsigned long long texg;  // z-pair texels v(x, y, z) | v(x, y, z + 1) << 20 in a 2D atlas, read by gathers
                              // (moving depth <= 12 only; 0 when not built)
    const float2 *zoff;       // per moving plane z: atlas offset of the plane + 1 - 2^23, (x, y)
    const uint32_t *rowinfo;  // row-bound layout: per fixed bin, word offset << 6 | wide << 5 | shift (0 or 16)
    const uint32_t *srow;     // random sampling (else null): row r's sampled voxels are entries srow[r]..srow[r+1]-1
    const uint16_t *scol;     //   of scol (their x index, ascending)
    const uint8_t *sbin;      //   and sbin (their fixed bin)
    int nf[3];             // fixed dims (x, y, z)
    int nm[3];             // moving dims
    int bins;
    int mdepth;            // moving bit depth
    int mdtype;            // 0 = uint8, 1 = uint16
    int rows_words;        // words of the row-bound layout of this pair
};

// q values of one call with their count-indexed FP64 tables
// tab[i][c] = c ln c (q == 1) or c^q (q != 1), c < kTab.
struct QSet {
    int nq;
    int form;   // 0 additive, 1 pseudo-additive Tsallis MI
    int bits;   // Shannon in bits
    int pad;
    float q[kMaxQ];
    const double *tab[kMaxQ];
};

// Per-transform outputs (device pointers; any may be null).
struct Outputs {
    double *mi;          // n x nq
    double *h;           // n x nq x 3
    long long *count;    // n
    uint32_t *dump;      // n x bins^2 histograms (test hook), single-pair only
    int *flags;          // [0] empty overlap seen, [1] drain table overflow
};

// Work item of the batched kernel.
struct Item {
    int pair;
    int t;   // transform index (row of the affine array and of the outputs)
};

// Histogram variants (match the public MI_HV_* values).  0..3: counter kinds
// with LDG gathers of x-pairs, 4..7: the same with texture-path gathers of
// x-pairs, 8 / 9: the row-bound layout with LDG / texture x-pairs, 10..12:
// the row-bound, 32-bit and 16-bit kinds with texture gathers of 2 x 2 (y, z) quads.
// 13..15: the row-bound, 32-bit and 16-bit kinds with one texture gather of 2 x 2 z-pair texels.
enum { HV_U32 = 0, HV_U32_MATCH = 1, HV_U16 = 2, HV_U16_MATCH = 3, HV_TEX = 4, HV_ROWS = 8, HV_ROWS_TEX = 9,
       HV_ROWS_QUAD = 10, HV_U32_QUAD = 11, HV_U16_QUAD = 12, HV_ROWS_GATHER = 13, HV_U32_GATHER = 14,
       HV_U16_GATHER = 15, HV_COUNT = 16 };
// How a variant fetches the moving volume.
enum { FM_LDG = 0, FM_TEX = 1, FM_QUAD = 2, FM_GATHER = 3 };
__host__ __device__ inline int hv_kind(int v) {
    if (v < HV_ROWS) return v % HV_TEX;
    if (v == HV_U32_QUAD || v == HV_U32_GATHER) return HV_U32;
    if (v == HV_U16_QUAD || v == HV_U16_GATHER) return HV_U16;
    return HV_ROWS;
}
__host__ __device__ inline int hv_fetch(int v) {
    if (v >= HV_ROWS_GATHER) return FM_GATHER;
    if (v >= HV_ROWS_QUAD) return FM_QUAD;
    return ((v >= HV_TEX && v < HV_ROWS) || v == HV_ROWS_TEX) ? FM_TEX : FM_LDG;
}
// Tile shape of the voxel walk (quad and gather fetches): a warp step covers 32 >> lpr_log2 adjacent
// fixed rows with 1 << lpr_log2 lanes each (lpr_log2 in 3..5), or, with lpr_log2 == 0, the warp walks
// its 32 clipped rows as one stream of voxels; the batched kernel cuts each sweep into `slabs` slabs
// of row blocks (1..16).
struct Tile {
    int lpr_log2;
    int slabs;
};
constexpr int kMaxSlabs = 16;

// Shared memory needed by a hard-path CTA of `threads` threads for `bins` bins
// (rows_words: words of the row-bound layout, used by HV_ROWS*).
// (zmax: moving planes of the largest pair, for the gather variants' per-plane offsets.)
size_t hard_smem_bytes(int variant, int bins, int threads, int rows_words, int zmax);
// Random voxel sampling: voxel x takes part iff fmix32(x ^ fmix32(seed)) < threshold.
// Per fixed row, the number of sampled voxels (counts: R entries), then the lists themselves
// (row_ptr: the exclusive prefix sums, R + 1 entries; cols / bins: row_ptr[R] entries).
cudaError_t launch_sample_count(int n0, long long R, uint32_t seed, uint32_t threshold, uint32_t *counts,
                                cudaStream_t s);
cudaError_t launch_sample_fill(int n0, long long R, uint32_t seed, uint32_t threshold, const uint8_t *fbins,
                               const uint32_t *row_ptr, uint16_t *cols, uint8_t *bins, cudaStream_t s);
// Per-bin voxel counts of a binned fixed volume (bins u64, zeroed here).
cudaError_t launch_fixed_hist(const uint8_t *fbins, long long n, int bins, unsigned long long *out, cudaStream_t s);

// ---- launchers (all asynchronous on `s`) ---------------------------------
cudaError_t launch_f32_to_u16(const float *in, long long n, uint16_t *out, cudaStream_t s);
cudaError_t launch_clamp_depth(void *data, int dtype, int depth, long long n, cudaStream_t s);
// Padded x-paired moving volume, dims (n0, n1 + 1, n2 + 1).
cudaError_t launch_make_pairs(const void *mov, int dtype, const int nm[3], void *out, cudaStream_t s);
// Iteration cap of the 16-bit counter drain on the current device (default 2^16; test hook).
cudaError_t set_drain_cap(int cap);
// 2 x 2 (y, z) quads of the moving volume, dims (n0, n1, n2): element (x, y, z) holds
// v(x, y, z), v(x, y + 1, z), v(x, y, z + 1), v(x, y + 1, z + 1), upper indices
// clamped to the last ones (uchar4 for uint8, ushort4 for uint16 volumes).
cudaError_t launch_make_quads(const void *mov, int dtype, const int nm[3], void *out, cudaStream_t s);
// z-pair atlas of the moving volume (depth <= 12): out is a W x H uint32 image (zeroed here) in which
// plane z occupies the nm[0] x nm[1] tile at ((z / ph) nm[0], (z % ph) nm[1]) and texel (x, y) of that
// tile holds v(x, y, z) | v(x, y, min(z + 1, nm[2] - 1)) << 20.
cudaError_t launch_make_zpairs(const void *mov, int dtype, const int nm[3], int ph, int W, int H, uint32_t *out,
                               cudaStream_t s);
cudaError_t launch_bin_fixed(const void *data, int dtype, int depth, long long n, int bins, uint8_t *out,
                             cudaStream_t s);
cudaError_t launch_table(double *tab, float q, cudaStream_t s);
// Plain path: n transforms, grid (ctas, n); histograms in global memory (n x bins^2 u32, zeroed here).
cudaError_t launch_plain_hist(const PairDev *d_pair, const PairDev &h_pair, const int32_t *d_aff, int n,
                              uint32_t *d_hist, int variant, int threads, int ctas, Tile tile, int *d_flags,
                              cudaStream_t s);
cudaError_t launch_entropy(const uint32_t *d_hist, int n, int bins, const QSet &Q, const Outputs &O,
                           cudaStream_t s);
// The same reduction split over entropy_parts(bins) CTAs per transform (for few transforms).
// Scratch: d_cols n x bins u32 (zeroed here), d_part n x entropy_parts(bins) x (1 + 2 kMaxQ) FP64.
int entropy_parts(int bins);
cudaError_t launch_entropy_split(const uint32_t *d_hist, int n, int bins, const QSet &Q, const Outputs &O,
                                 uint32_t *d_cols, double *d_part, cudaStream_t s);
// Batched path: persistent CTAs pull items from *d_ticket (reset by the caller).
cudaError_t launch_batched(const PairDev *d_pairs, const int32_t *d_aff, const Item *d_items, int nitems,
                           int *d_ticket, int max_bins, int rows_words, int zmax, int variant, int threads, int ctas,
                           Tile tile, const QSet &Q, const Outputs &O, cudaStream_t s);
int batched_ctas_per_sm(int variant, int max_bins, int threads, int rows_words, int zmax);
cudaError_t launch_resample(const PairDev *d_pair, const PairDev &h_pair, const int32_t *d_aff, void *out,
                            cudaStream_t s);

// ---- Parzen (differentiable) path ----------------------------------------
struct ParzenPair {
    const uint8_t *fbins;   // Parzen fixed bins floor(f (B-4)) + 2
    const float *mov;       // normalised moving intensities in [0, 1]
    const float *movx;      // the same extended by one plane per axis, dims (n0 + 1, n1 + 1, n2 + 1)
    unsigned long long texq;  // 2 x 2 (y, z) quads of movx as a float4 3D texture, dims (n0, n1, n2)
    const uint32_t *srow;   // random sampling (else null): row r's sampled voxels are entries srow[r]..srow[r+1]-1
    const uint16_t *scol;   //   of scol (their x index, ascending)
    const uint8_t *sbin;    //   and sbin (their Parzen fixed bin)
    int nf[3];
    int nm[3];
    int B;
    int pad;
};

struct ParzenAffine {       // per transform: the FP64 host affine [A | b] in 32.32 fixed point
    long long A[12];        // llround(x * 2^32); exact integer positions, so the trilinear cell and
};                          // overlap decisions match the FP64 definition except within ~1e-7 voxel

cudaError_t launch_parzen_prep_fixed(const void *data, int dtype, int depth, long long n, int B, uint8_t *out,
                                     cudaStream_t s);
cudaError_t launch_parzen_prep_moving(const void *data, int dtype, int depth, long long n, float *out,
                                      cudaStream_t s);
// About 4 CTAs per SM over n transforms, as CTAs per transform (the adjoint's starting point), and
// blocks of the per-cell kernel.
int parzen_ctas(const ParzenPair &P, int n, int sms);
// CTAs per transform of the adjoint for nq q values: whole waves of its resident CTAs.
int parzen_adj_ctas(const ParzenPair &P, int n, int nq, int sms);
// The extended moving volume: out has dims (n0 + 1, n1 + 1, n2 + 1); on the extra planes each axis
// continues linearly (v[n] = 2 v[n - 1] - v[n - 2]), so that the trilinear cell of an index on the
// last plane can be its integer part: the value there is v[n - 1] and the derivative along the axis
// is v[n - 1] - v[n - 2], those of the last cell.
cudaError_t launch_parzen_extend(const float *mov, const int nm[3], float *out, cudaStream_t s);
// (y, z) quads of the extended volume: out (float4) has dims (n0, n1, n2); element (x, y, z) holds
// movx at (x, y, z), (x, y + 1, z), (x, y, z + 1), (x, y + 1, z + 1).
cudaError_t launch_parzen_quads(const float *movx, const int nm[3], void *out, cudaStream_t s);
int parzen_cell_blocks(int B);
// One Parzen call over n transforms: the pairs as a device array, transform t evaluated on pair
// d_pair_of[t] (NULL: every transform on pair 0) whose fixed rows start at d_row_start[t] in the
// sequence of all transforms' rows (NULL: t R of pair 0; n + 1 entries).  Per-transform tables take
// slots sized for the largest bin count Bmax (histograms and W: Bmax^2 per transform and q; marginals
// 2 Bmax), the first B^2 used with row stride B.  nx_max: the longest fixed row of the pairs.
struct ParzenLaunch {
    ParzenPair p0;  // pair 0 (single-pair calls pass it by value)
    const ParzenPair *d_pairs;
    const int *d_pair_of;
    const long long *d_row_start;
    int n;
    int Bmax;
    int nx_max;
    bool sampled;
    long long total_rows;
};

// Soft histograms (n x Bmax^2 u64 sums of 2^-32-quantised weights, zeroed here) and overlap counts (n).
// sms: the device's SM count (the grid is sized in whole waves).
cudaError_t launch_parzen_hist(const ParzenLaunch &L, const ParzenAffine *d_aff, int sms, unsigned long long *d_hist,
                               unsigned long long *d_count, cudaStream_t s);
// MI per q (n x nq) and the weight tables W (n x nq x Bmax^2, FP32) from the soft histograms.
// Scratch: marg (n x 2 Bmax), ment (n x nq x 2), mterm (n x nq x 2 Bmax), jpart (n x nq x
// parzen_cell_blocks(Bmax)) FP64.
cudaError_t launch_parzen_weights(const unsigned long long *d_hist, const unsigned long long *d_count,
                                  const ParzenLaunch &L, const QSet &Q, double *marg, double *ment, double *mterm,
                                  double *jpart, double *d_mi, float *d_w, cudaStream_t s);
// Gradient: per-CTA moments (scratch n x nq x ctas x 12 FP64) and dMI/dtheta (n x nq x np FP64);
// d_jac: n x 12 x np (d[A|b]/dparam about the fixed centre), np = 9 or 12.
cudaError_t launch_parzen_adjoint(const ParzenLaunch &L, const ParzenAffine *d_aff, const double *d_jac, int np, int nq,
                                  int ctas, const float *d_w, const unsigned long long *d_count, double *d_mom,
                                  double *d_grad, cudaStream_t s);

// ---- allocation-free evaluation (mi_noalloc.cu) ---------------------------
// Plain-path variant that bins the fixed volume on the fly and keeps its
// histogram (bins^2 u32), flags (2 int) and results (4 nq + 1 doubles) in
// caller-provided device memory.
cudaError_t launch_noalloc_eval(const void *fix, int fdtype, int fdepth, const void *mov, int mdtype, int mdepth,
                                const int nf[3], const int nm[3], int bins, const int32_t q16[12], const QSet &Q,
                                uint32_t *hist, int *flags, double *out, int ctas, cudaStream_t s);
// The context path's parameter -> 16.16 affine builder (false if an entry does not fit).
bool host_affine_q16(const float prm[9], const int nf[3], const float sf[3], const int nm[3], const float sm[3],
                     int32_t q16[12]);
// Message returned by mi_last_error(NULL) on this thread.
void set_thread_error(const char *msg);

}  // namespace mi
