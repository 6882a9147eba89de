/*
 * mi.h -- C ABI of the GB300 mutual-information library.
 *
 * The library evaluates the registration metric of Vianna & Murta,
 * "Analysis of Generalized Entropies in Mutual Information Medical Image
 * Registration": Shannon mutual information, Eq. (1)-(2), and Tsallis mutual
 * information, between a fixed volume u(x) and a moving volume resampled
 * under a transform, v(T(x)) (Fig. 1 block diagram; the metric F_m whose
 * argmax over T is the registration, Eq. (3)).  T has 9 parameters from the
 * three families the paper studies (Introduction): translation, rotation,
 * scale; or, optionally, the 12 of a general affine (Methodology).  All voxels contribute to one full joint histogram (Discussion),
 * and one histogram serves Shannon and every Tsallis q (Discussion).
 *
 * Conventions that the paper leaves open and this library fixes:
 *  - Volumes: x fastest, index = x + nx (y + ny z).  Integer volumes carry a
 *    bit depth d; values above 2^d - 1 are clamped to 2^d - 1 on load.
 *    Float volumes hold values in [0, 1]; the hard-binned path converts them
 *    once to 16-bit integers (round-half-even of v * 65535, depth 16).
 *  - Binning: an integer value v of depth d lies in bin (v * bins) >> d.
 *  - Transform parameters, 9 floats per transform: tx ty tz (mm), rx ry rz
 *    (degrees; or a unit-ball versor, mi_options.rotation), sx sy sz (scale
 *    factors, 1 = identity; or zero-centred offsets, mi_options.scale).  A fixed physical
 *    point p = s_f * i (i the voxel index) maps to
 *    p_m = R diag(s) (p - c_f) + c_m + t, R = Rz(rz) Ry(ry) Rx(rx), c the
 *    volume centres s * (n - 1) / 2; the moving index is p_m / s_m (a general
 *    affine replaces R diag(s) by its matrix M, MI_TRANSFORM_AFFINE).  In index
 *    space u = A i + b; [A | b] is quantised to 16.16 fixed point as
 *    llround(x * 65536) (computed in FP64 on the host with the order of
 *    operations fixed, so the quantised matrix is reproducible).
 *  - Hard path: U = A i + b exactly in integers; a voxel counts iff
 *    0 <= U_a <= (n_a - 1) * 65536 on every axis (overlap only); trilinear
 *    interpolation with 8-bit weights w = (U & 0xFFFF) >> 8 and stage lerp
 *    (a (256 - w) + b w + 128) >> 8, x then y then z.  Joint counts are exact.
 *  - Entropies: natural log (nats) unless opt.log_bits; Tsallis
 *    S_q = (1 - sum p^q) / (q - 1); q == 1 means Shannon.  Tsallis MI is
 *    S_q(F) + S_q(M) - S_q(F,M) (MI_TSALLIS_ADDITIVE, the literal extension
 *    of Eq. (2)) or adds (1 - q) S_q(F) S_q(M) (MI_TSALLIS_PSEUDO_ADDITIVE).
 *    Marginals are the row / column sums of the overlap histogram.  Sums are
 *    accumulated in FP64 on the GPU.
 *  - Parzen (differentiable) path: fixed bin floor(f (B - 4)) + 2 of the
 *    normalised intensity f; moving term a cubic B-spline at
 *    m~ = m (B - 4) + 2, m the FP32 trilinear value at the real moving index;
 *    gradient with the overlap held fixed.
 *
 * Memory: every pointer argument may be host memory (pageable or pinned) or
 * CUDA device memory of the context's device; the library inspects each one.
 * The context copies the volumes into device memory it owns, so the caller's
 * volume buffers may be freed once mi_create returns.  Work is ordered on
 * the context's stream (its own non-blocking stream unless mi_set_stream
 * names another) and every call returns once its results are in the caller's
 * buffers (the call synchronises that stream).
 *
 * Errors: every call returns an mi_status; mi_last_error gives a message.
 * A context is not thread-safe; distinct contexts are independent.
 */
#ifndef MI_H
#define MI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MI_OK = 0,
    MI_EINVAL = 1,        /* invalid argument (message says which)             */
    MI_ENOMEM = 2,        /* device or host allocation failed                  */
    MI_ECUDA = 3,         /* a CUDA call failed                                */
    MI_EEMPTY = 4,        /* some transform had an empty overlap (its MI NaN)  */
    MI_EUNSUPPORTED = 5,  /* valid but not supported (e.g. mi_grad, hard mode) */
    MI_ERANGE = 6         /* an affine entry does not fit 16.16 fixed point    */
} mi_status;

typedef enum { MI_U8 = 0, MI_U16 = 1, MI_F32 = 2 } mi_dtype;

typedef struct {
    const void *data;     /* x fastest, contiguous                              */
    int dtype;            /* mi_dtype                                           */
    int dims[3];          /* nx, ny, nz; each >= 2; nx*ny*nz < 2^31             */
    int bit_depth;        /* u8: 1..8, u16: 1..16, 0 = full width; f32: ignored */
    float spacing_mm[3];  /* > 0                                                */
} mi_volume;

enum { MI_HARD = 0, MI_PARZEN = 1 };
enum { MI_TSALLIS_ADDITIVE = 0, MI_TSALLIS_PSEUDO_ADDITIVE = 1 };
/* Histogram privatisation variants of the hard path (-1 = autotuned). */
enum {
    MI_HV_AUTO = -1,
    MI_HV_U32 = 0,        /* 32-bit shared counters, one atomic per voxel        */
    MI_HV_U32_MATCH = 1,  /* 32-bit counters, warp-aggregated (match.any)        */
    MI_HV_U16 = 2,        /* 16-bit packed counters drained at 2^14              */
    MI_HV_U16_MATCH = 3,  /* 16-bit packed counters, warp-aggregated             */
    /* the same four with the moving volume read through the texture path */
    MI_HV_U32_TEX = 4,
    MI_HV_U32_MATCH_TEX = 5,
    MI_HV_U16_TEX = 6,
    MI_HV_U16_MATCH_TEX = 7,
    /* row-bound layout: 32-bit counters only for fixed bins holding more than
       65535 fixed voxels, 16-bit halves for the rest (provably never overflow);
       fits when those rows are few */
    MI_HV_ROWS = 8,
    MI_HV_ROWS_TEX = 9,
    /* the moving volume as 2 x 2 (y, z) quads read through the texture path:
       two fetches per voxel (columns x and x + 1) instead of four, twice the
       moving-volume memory */
    MI_HV_ROWS_QUAD = 10,
    MI_HV_U32_QUAD = 11,
    MI_HV_U16_QUAD = 12,
    /* moving depth <= 12 only: one 2D texture gather per voxel from an atlas of
       the moving planes whose 32-bit texels pack v(x, y, z) with v(x, y, z + 1),
       so the 2 x 2 footprint holds all 8 trilinear neighbours */
    MI_HV_ROWS_GATHER = 13,
    MI_HV_U32_GATHER = 14,
    MI_HV_U16_GATHER = 15
};
/* Meaning of the rotation parameters (transform[3..5]):
 *  MI_ROT_EULER_DEG  R = Rz(rz) Ry(ry) Rx(rx), right-handed, degrees;
 *  MI_ROT_VERSOR     the unit-ball parameterisation of the paper's rotation
 *                    maps (Results): v = (v1, v2, v3) is the vector part of
 *                    the unit quaternion (sqrt(1 - |v|^2), v), a turn by
 *                    2 asin|v| about v; |v| >= 1 is normalised onto the sphere
 *                    (a half turn).  Gradients are d/dv (the normalised
 *                    direction's outside the ball).
 * Meaning of the scale parameters (transform[6..8]):
 *  MI_SCALE_FACTOR   sigma = s (1 = identity);
 *  MI_SCALE_OFFSET   sigma = 1 + s (0 = identity), the paper's zero-centred
 *                    scale maps (Results). */
enum { MI_ROT_EULER_DEG = 0, MI_ROT_VERSOR = 1 };
enum { MI_SCALE_FACTOR = 0, MI_SCALE_OFFSET = 1 };

/* What a transform's floats are (mi_options.transform):
 *  MI_TRANSFORM_PARAMS  9 parameters: tx, ty, tz (mm), three rotation and
 *                       three scale parameters as above.
 *  MI_TRANSFORM_AFFINE  12 parameters, the general affine of the
 *                       Methodology's 12 degrees of freedom (the affine
 *                       family of the Introduction adds skew to translation,
 *                       rotation and scale): [M | t] row-major
 *                       (M00 M01 M02 t0 M10 M11 M12 t1 M20 M21 M22 t2), M
 *                       dimensionless and t in mm.  The moving physical point
 *                       is M (p - c_f) + c_m + t, p the fixed physical point
 *                       and c_f, c_m the volume centres, exactly as the
 *                       9-parameter form with R diag(sigma) replaced by M;
 *                       identity: M = I, t = 0.  mi.rotation and mi.scale do
 *                       not apply.  Gradients are d MI / d [M | t] in the
 *                       same order.
 * P below is the count (9 or 12); mi_transform_size returns it. */
enum { MI_TRANSFORM_PARAMS = 0, MI_TRANSFORM_AFFINE = 1 };

/* Evaluation path of mi_eval. */
enum { MI_PATH_AUTO = 0, MI_PATH_PLAIN = 1, MI_PATH_BATCHED = 2 };

#define MI_MAX_Q 8     /* q values per call          */
#define MI_MAX_BINS 256
#define MI_MIN_BINS 2
#define MI_MIN_PARZEN_BINS 8
#define MI_MAX_PARZEN_NX 65536  /* longest fixed row of a MI_PARZEN context */

typedef struct {
    int kernel;        /* MI_HARD (default) or MI_PARZEN                            */
    int tsallis_form;  /* MI_TSALLIS_ADDITIVE (default) or MI_TSALLIS_PSEUDO_ADDITIVE */
    int log_bits;      /* 0: nats (default); 1: Shannon entropies in bits          */
    int hist_variant;  /* MI_HV_AUTO (default) or a fixed MI_HV_* variant          */
    int path;          /* MI_PATH_AUTO (default), MI_PATH_PLAIN, MI_PATH_BATCHED    */
    int use_graphs;    /* 1 (default): replay the batched launch as a CUDA graph   */
    int autotune;      /* 1 (default): time the variants once per shape and cache  */
    int device;        /* CUDA device ordinal; -1 (default) = the current device   */
    int block_threads; /* hard-path CTA size: 0 (default) = autotuned, or 512 / 1024 */
    int rotation;      /* MI_ROT_EULER_DEG (default) or MI_ROT_VERSOR               */
    int scale;         /* MI_SCALE_FACTOR (default) or MI_SCALE_OFFSET              */
    float sample_fraction;    /* 0 (default) = every fixed voxel; in (0, 1) = a random
                                 subset of that fraction (see below)                   */
    unsigned int sample_seed; /* seed of that subset                                    */
    int transform;     /* MI_TRANSFORM_PARAMS (default) or MI_TRANSFORM_AFFINE       */
    int tile_rows;     /* hard path, quad and gather variants: adjacent fixed rows one
                          warp step covers (32 / tile_rows lanes each), 1, 2 or 4; or
                          32: a warp walks its 32 clipped rows as one stream of voxels
                          (one partial step per 32 rows); 0 (default) = autotuned     */
    int tile_slabs;    /* batched kernel: slabs per sweep of the fixed rows (CTAs on
                          different transforms keep to neighbouring slabs): 0 (default)
                          = 4, or 1..16                                                */
} mi_options;

/* Random voxel sampling (mi_options.sample_fraction in (0, 1), hard and
 * Parzen forms; the Discussion's comparison with ITK Mattes, which samples the
 * image at random, against MICUDA's every-voxel histogram).  A fixed voxel with
 * linear index x takes part iff fmix32(x ^ fmix32(seed)) < floor(fraction *
 * 2^32), fmix32 being the 32-bit finalizer of MurmurHash3.  The subset is
 * fixed when the context is created, so the metric stays a deterministic
 * function of the transform, and only the sampled voxels are visited.
 * Requires nx <= 65536 (MI_EUNSUPPORTED otherwise). */

typedef struct mi_ctx mi_ctx;

/* Fills *opt with the defaults listed above. */
void mi_options_default(mi_options *opt);

/* Library version string (static storage). */
const char *mi_version(void);

/*
 * Creates a context for one (fixed, moving) pair and a bin count
 * (MI_MIN_BINS..MI_MAX_BINS; MI_MIN_PARZEN_BINS..128 for MI_PARZEN, whose
 * fixed volume must have nx <= MI_MAX_PARZEN_NX, else MI_EUNSUPPORTED).  The metric
 * is F_m(u(x), v(T(x))) of Fig. 1; the pair's geometry (dims, spacing) fixes
 * the parameter-to-affine map.  The moving volume is gathered through 3D
 * textures: its dims must fit the device's 3D texture extent
 * (cudaDevAttrMaxTexture3DWidth / Height / Depth), else MI_EUNSUPPORTED.
 * opt may be NULL (defaults).  On success *out
 * owns device copies of both volumes (the fixed one pre-binned) and must be
 * released with mi_destroy.  On failure *out is NULL and mi_last_error(NULL)
 * describes the error on this thread.
 */
mi_status mi_create(mi_ctx **out, const mi_volume *fixed, const mi_volume *moving, int bins,
                    const mi_options *opt);

/*
 * Creates one context over npairs volume pairs of uneven sizes, types and
 * bin counts (bins[p] per pair).  The paper evaluates the metric over whole
 * grids of transforms of one pair at a time (Methodology: 3D parameter-space
 * maps, e.g. 51^3 translations); batching many transforms, and many pairs,
 * into one launch is this library's addition for that workload.  Hard
 * contexts (MI_HARD) are evaluated by mi_batch_eval in one persistent launch
 * with a per-pair work queue; Parzen contexts (MI_PARZEN, bins 8..128 per
 * pair) by mi_batch_eval (MI) and mi_batch_grad (MI and gradient), one
 * launch per kernel for all pairs.
 */
mi_status mi_batch_create(mi_ctx **out, const mi_volume *fixed, const mi_volume *moving, const int *bins,
                          int npairs, const mi_options *opt);

/* Releases every resource of the context (NULL is ignored). */
void mi_destroy(mi_ctx *ctx);

/* P, the number of floats per transform of ctx (9, or 12 for
 * MI_TRANSFORM_AFFINE); -1 if ctx is NULL. */
int mi_transform_size(const mi_ctx *ctx);

/* Message of the last failed call on ctx, or of the last failed create on
 * this thread when ctx is NULL.  Valid until the next call on ctx. */
const char *mi_last_error(const mi_ctx *ctx);

/* Orders all later work of ctx on the CUDA stream `stream` (a cudaStream_t of
 * the context's device; NULL = back to the context's own stream).  CUDA-graph
 * replay is skipped on the legacy default stream, which cannot be captured. */
mi_status mi_set_stream(mi_ctx *ctx, void *stream);

/*
 * MI for n transforms (n x P floats, parameters above) and nq exponents q
 * (1 <= nq <= MI_MAX_Q; q > 0; q == 1 is Shannon, Eq. (1)-(2); other q are
 * Tsallis; q within 1e-6 of 1 but not 1 is rejected).  One joint histogram
 * per transform serves every q (Discussion).
 * out_mi:    n x nq doubles (row = transform).
 * out_h:     n x nq x 3 doubles (H_F, H_M, H_FM per q), or NULL.
 * out_count: n int64 overlap voxel counts, or NULL.
 * A transform whose overlap is empty gets NaN and the call returns MI_EEMPTY
 * after finishing every other transform.  In MI_PARZEN mode this returns the
 * Parzen MI (no gradient) and out_count the voxels inside each overlap (the
 * voxels its soft histogram sums); out_h must be NULL there (MI_EUNSUPPORTED).
 * n == 0 is a no-op.
 */
mi_status mi_eval(mi_ctx *ctx, const float *transforms, int n, const float *q, int nq, double *out_mi,
                  double *out_h, int64_t *out_count);

/* As mi_eval, with the 16.16 affines [A | b] (n x 12 int32, row-major 3x4)
 * given directly instead of parameters: the index-space form of the Fig. 1
 * Transform block (any affine, e.g. one built by the caller for a map of the
 * Methodology), quantised as the hard path's fixed-point coordinates are.
 * Hard path, pair 0. */
mi_status mi_eval_q16(mi_ctx *ctx, const int32_t *affines, int n, const float *q, int nq, double *out_mi,
                      double *out_h, int64_t *out_count);

/*
 * Batched evaluation over the pairs of a mi_batch_create context (the
 * Methodology's parameter-space maps, many transforms per call):
 * transform t (n x P parameters) is evaluated on pair pair_of_transform[t]
 * (n ints, host or device memory).  Outputs as in mi_eval (out_h and
 * out_count are hard-path outputs; NULL for a Parzen context).
 */
mi_status mi_batch_eval(mi_ctx *ctx, const int *pair_of_transform, const float *transforms, int n,
                        const float *q, int nq, double *out_mi, double *out_h, int64_t *out_count);

/*
 * Parzen MI and its gradient dMI/dtheta over the P parameters (MI_PARZEN
 * contexts only): cubic-B-spline soft joint histogram of the moving
 * intensity against the box-binned fixed intensity, differentiated through
 * the trilinear resampling and the transform (the optimiser's gradient,
 * Introduction; registration as argmax, Eq. (3)).
 * out_mi: n x nq; out_grad: n x nq x P (d MI / d param, Euler angles per
 * degree).
 */
mi_status mi_grad(mi_ctx *ctx, const float *transforms, int n, const float *q, int nq, double *out_mi,
                  double *out_grad);

/*
 * mi_grad over the pairs of a MI_PARZEN mi_batch_create context: transform t
 * on pair pair_of_transform[t]; out_mi n x nq, out_grad n x nq x P.  Every
 * kernel of the forward, the entropies and the adjoint runs once for all
 * pairs (each pair with its own bin count).
 */
mi_status mi_batch_grad(mi_ctx *ctx, const int *pair_of_transform, const float *transforms, int n, const float *q,
                        int nq, double *out_mi, double *out_grad);

/*
 * Test hook: the joint histogram (row = fixed bin, bins x bins uint32 per
 * transform) of n transforms of pair `pair`, computed by the plain path
 * (path = MI_PATH_PLAIN) or copied out of the batched kernel's on-chip
 * histogram (MI_PATH_BATCHED).  Exactly one of transforms (n x P) and
 * affines (n x 12 16.16) is non-NULL.
 */
mi_status mi_hist(mi_ctx *ctx, int pair, const float *transforms, const int32_t *affines, int n, int path,
                  uint32_t *out_counts);

/* Test hook: the FP64 affine [A | b] (n x 12), its 16.16 quantisation (n x 12)
 * and its Jacobian d[A|b]/dparam (n x 12 x P) for pair `pair` and n x P
 * transforms; any output may be NULL.  Host computation only. */
mi_status mi_affine(mi_ctx *ctx, int pair, const float *transforms, int n, double *out_affine,
                    int32_t *out_q16, double *out_jacobian);

/* Test hook: the pre-binned fixed volume of pair `pair` (nvox uint8). */
mi_status mi_fixed_bins(mi_ctx *ctx, int pair, uint8_t *out);

/* v(T(x)) of pair `pair` on the fixed grid for one 16.16 affine, same type as
 * the stored moving volume (uint16 for float input), 0 outside the overlap. */
mi_status mi_resample(mi_ctx *ctx, int pair, const int32_t *affine, void *out);

/* The histogram variant the autotuner chose (or was told) for pair `pair`,
 * for the given number of transforms per call; -1 if none yet. */
int mi_selected_variant(mi_ctx *ctx, int pair, int n);

/* Autotune cache (process-wide): the batched path's autotuner records each
 * tuned shape in the text file `path` (one line per shape: a key naming the
 * device, the library version, the pairs' dims, types, bit depths and bins,
 * the transform-count bucket and the options that restrict the candidates,
 * then the choice) and, for a shape already in the file, takes the recorded
 * choice instead of timing the candidates -- as long as that choice is still
 * a candidate.  path NULL or "" disables it.  Until this is called the path
 * comes from the environment variable MI_AUTOTUNE_CACHE (unset: disabled).
 * A file that cannot be opened only costs the tuning time. */
void mi_autotune_cache(const char *path);

/* The whole configuration chosen (autotuned or set) for calls of n transforms:
 * out[0..4] = histogram variant, threads per CTA, CTAs, fixed rows per warp
 * step, slabs per sweep (all -1 if none chosen yet). */
mi_status mi_selected_config(mi_ctx *ctx, int n, int out[5]);

/* Test hook (failure handling): after `after` further successful device
 * allocations by the library in this process, the next one fails as if the
 * device were out of memory (the caller sees MI_ENOMEM), and the hook disarms
 * itself; after < 0 disarms it.  It lets callers check that every entry point
 * fails cleanly and leaves its context usable.  Host-side only: no GPU fault
 * is raised. */
void mi_fault_alloc(int after);

/* Test hook (failure handling): the iteration cap of the one retry loop in
 * the kernels, the compare-and-swap that drains a 16-bit counter
 * (MI_HV_U16* variants), on the current device; default 65536.  With 0 every
 * drain gives up at once: the kernel flags the error and finishes, and the
 * call reports MI_ECUDA.  Returns MI_EINVAL for cap < 0, MI_ECUDA if the
 * device write fails. */
mi_status mi_fault_drain_cap(int cap);

/* Profiling hook: device time in milliseconds of the main histogram kernel(s)
 * of the last completed mi_eval / mi_eval_q16 / mi_batch_eval / mi_grad call,
 * measured with CUDA events recorded on the context's stream around those
 * launches (inside the replayed graph for the batched path).  *launches
 * receives the number of kernels the call launched (NULL ok). */
mi_status mi_last_kernel_ms(mi_ctx *ctx, float *ms, int *launches);

/*
 * Allocation-free evaluation.  The paper has no counterpart: this is a
 * deployment aid for callers that may not allocate device memory where they
 * need the metric -- plug-ins inside a framework whose caching allocator owns
 * the GPU's memory (a cudaMalloc of their own fails once the pool holds it,
 * or fragments it), services that fix their GPU memory budget up front, loops
 * that cannot afford cudaMalloc's implicit device-wide synchronisation.  It
 * computes the same hard-binned MI as mi_eval (plain path) for ONE transform
 * (9 parameters in the default conventions -- Euler degrees, scale factors --
 * host memory) and nq q values (host memory) without creating a context and
 * without calling cudaMalloc, cudaFree or any allocating routine.
 *  - fixed, moving: uint8 or uint16 volumes already in device memory of the
 *    current device, used in place (no copy); values above 2^d - 1 are
 *    clamped as they are read, as mi_eval clamps them on load.
 *  - bins: 2..MI_NOALLOC_MAX_BINS; the fixed volume may hold at most
 *    MI_NOALLOC_MAX_VOXELS voxels and the moving volume at most
 *    MI_NOALLOC_MAX_MOVING_VOXELS.  Larger sizes return MI_EINVAL.
 *  - out_mi: nq doubles, host or device memory.  stream: a cudaStream_t
 *    (NULL = legacy default stream); the call synchronises it.
 *  - Intermediates live in one static device array of about 257 KiB that every
 *    GPU loading the library holds until the process exits.  The call clears
 *    the histogram part before use; the array keeps the last call's contents.
 *    All calls share it, so calls that overlap on the GPU (several streams or
 *    threads at once) race: serialise them.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current.
 *  - Shannon entropies in nats and the additive Tsallis form.  Errors as for
 *    mi_eval; the message is read with mi_last_error(NULL).
 */
#define MI_NOALLOC_MAX_BINS 256
#define MI_NOALLOC_MAX_VOXELS (1LL << 25)
#define MI_NOALLOC_MAX_MOVING_VOXELS ((1LL << 31) - 1)
mi_status mi_eval_noalloc(const mi_volume *fixed, const mi_volume *moving, int bins, const float *transform,
                          const float *q, int nq, double *out_mi, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MI_H */
