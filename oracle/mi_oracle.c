/*
 * mi_oracle.c -- plain, slow, obviously correct CPU reference for Shannon and
 * Tsallis mutual information between a fixed 3D volume and a moving volume
 * resampled under a 9-parameter transform (translation, rotation, scale) or
 * a general 12-parameter affine.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The CUDA library shares no
 * code, header, table or constant with it, and neither includes the other.
 *
 * Arithmetic: exact 64-bit integers for fixed-point coordinates, integer
 * interpolation and histogram counts; FP64 for every entropy and for the
 * whole Parzen (differentiable) form.  Build with -ffp-contract=off so that
 * the transform builder rounds the same way on every host.
 *
 * The paper prints Eq. (1) (Shannon entropy), Eq. (2) (mutual information)
 * and Eq. (3) (registration as argmax over T); it names Tsallis entropy and
 * the translation / rotation / scale families (Introduction) and a full,
 * all-voxel histogram (Discussion) but leaves the rest open.  The readings
 * used here are tagged R1..R17 where they are applied:
 *   R1 binning (v * bins) >> depth               R2 parameter -> affine
 *   R3 16.16 fixed-point coordinate, overlap     R4 integer trilinear
 *   R5 counts over the overlap only              R6 natural logarithm
 *   R7 Tsallis entropy and Tsallis MI forms      R8 Parzen soft histogram
 *   R9 Parzen gradient (adjoint of R8)           R14 unit-ball (versor) rotation
 *   R15 zero-centred scale parameters            R16 random voxel sampling
 *   R17 general affine [M | t] (12 parameters)
 *
 * Every function here is pinned by tests that do not re-type its formula:
 * hand-enumerated 4x4x4 cases, exact permutations, closed forms, limits,
 * finite differences and brute force.  Parity is pinned for every function
 * except where the function's comment says "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U8 0
#define ORC_U16 1
#define ORC_F32 2

#define ORC_OK 0
#define ORC_ERANGE 1
#define ORC_EINVAL 2
#define ORC_ENOMEM 3

/* ------------------------------------------------------------------------ */
/* Volume access                                                             */
/* ------------------------------------------------------------------------ */

static int64_t orc_nvox(const int n[3]) {
    return (int64_t)n[0] * (int64_t)n[1] * (int64_t)n[2];
}

static int64_t orc_index(const int n[3], int64_t i, int64_t j, int64_t k) {
    return i + (int64_t)n[0] * (j + (int64_t)n[1] * k); /* x fastest */
}

static uint32_t orc_get_u(const void *data, int dtype, int64_t idx) {
    if (dtype == ORC_U8) return ((const uint8_t *)data)[idx];
    return ((const uint16_t *)data)[idx];
}

/* Value of an integer voxel read at bit depth d: values above 2^d - 1 are
 * clamped to 2^d - 1 on load (the bit depth declares them impossible). */
static uint32_t orc_get_clamped(const void *data, int dtype, int depth, int64_t idx) {
    uint32_t v = orc_get_u(data, dtype, idx);
    uint32_t vmax = (uint32_t)((((uint64_t)1) << depth) - 1u);
    return v > vmax ? vmax : v;
}

/*
 * Hard-mode conversion of a float volume with values in [0, 1] to 16-bit
 * integers (depth 16): round-half-even of v * 65535 in FP64, clamped; NaN -> 0.
 * This lets the integer resampling of R4 apply to float volumes too.
 */
void orc_f32_to_u16(const float *in, int64_t nvox, uint16_t *out) {
    for (int64_t x = 0; x < nvox; x++) {
        double v = (double)in[x];
        if (!(v == v)) v = 0.0;
        double s = nearbyint(v * 65535.0);
        if (s < 0.0) s = 0.0;
        if (s > 65535.0) s = 65535.0;
        out[x] = (uint16_t)s;
    }
}

/* ------------------------------------------------------------------------ */
/* R1 binning                                                                */
/* ------------------------------------------------------------------------ */

/*
 * R1: the paper uses "all the voxels" and "a full histogram" (Discussion)
 * without a bin rule.  Reading: an integer value v of bit depth d lies in bin
 * (v * bins) >> d; values at or above 2^d are clamped to 2^d - 1 first.  With
 * bins = 2^d this is one bin per grey level, the paper's full histogram.
 */
int orc_bin_of(uint32_t v, int bins, int depth) {
    uint64_t vmax = (((uint64_t)1) << depth) - 1u;
    uint64_t w = v;
    if (w > vmax) w = vmax;
    return (int)((w * (uint64_t)bins) >> depth);
}

void orc_bin_volume(const void *data, int dtype, int depth, int64_t nvox, int bins,
                    uint8_t *out) {
    for (int64_t x = 0; x < nvox; x++) out[x] = (uint8_t)orc_bin_of(orc_get_u(data, dtype, x), bins, depth);
}

/* ------------------------------------------------------------------------ */
/* R2 parameters -> affine                                                   */
/* ------------------------------------------------------------------------ */

static void orc_mat3_mul(const double a[9], const double b[9], double c[9]) {
    for (int r = 0; r < 3; r++)
        for (int col = 0; col < 3; col++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s = s + a[3 * r + k] * b[3 * k + col];
            c[3 * r + col] = s;
        }
}

static double orc_deg2rad(double deg) { return deg * (3.14159265358979323846 / 180.0); }

/* Rotation about x, y, z by angles in radians; d = 1 gives the derivative
 * of the matrix with respect to its angle instead. */
static void orc_rot_x(double a, int d, double m[9]) {
    double c = cos(a), s = sin(a);
    double r[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    double dr[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
    memcpy(m, d ? dr : r, sizeof r);
}
static void orc_rot_y(double a, int d, double m[9]) {
    double c = cos(a), s = sin(a);
    double r[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    double dr[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
    memcpy(m, d ? dr : r, sizeof r);
}
static void orc_rot_z(double a, int d, double m[9]) {
    double c = cos(a), s = sin(a);
    double r[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    double dr[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
    memcpy(m, d ? dr : r, sizeof r);
}

/*
 * R2: the paper's Transform block (Fig. 1) maps the moving image to v(T(x))
 * with parameters from the three families it studies (Introduction,
 * Methodology): translation in mm, rotation, scale.  Reading:
 *   p      = s_f * i                     physical fixed point (mm), i = index
 *   c_f    = s_f * (n_f - 1) / 2         fixed centre; c_m likewise
 *   p_m    = R * diag(sigma) * (p - c_f) + c_m + t
 *   R      = Rz(rz) * Ry(ry) * Rx(rx), right-handed, angles in degrees
 *   u      = p_m / s_m                   moving index
 * so u = A i + b with A = diag(1/s_m) R diag(sigma) diag(s_f) and
 * b = diag(1/s_m) (c_m + t - R diag(sigma) c_f).
 * Parameter order: tx ty tz (mm), rx ry rz (degrees), sx sy sz (factors).
 * Output: out[4*a + c], row a of [A | b] (c = 3 is the offset), FP64.
 * If dout is not NULL it receives d out[e] / d param[p] at dout[9*e + p].
 * Floating-point order: R = (Rz*Ry)*Rx with each entry summed over k = 0,1,2
 * from 0.0, left to right; A[a][c] = ((R[a][c] * sigma[c]) * s_f[c]) / s_m[a];
 * b[a] = ((c_m[a] + t[a]) - sum_c (R[a][c]*sigma[c]) * c_f[c]) / s_m[a] with
 * the same summation order; no fused multiply-add anywhere.
 */
/*
 * R14, the unit-ball rotation (the rotation maps of the Results, whose points
 * outside radius 1 land on the sphere): the three rotation parameters are the
 * vector part v of a unit quaternion (w, v), w = sqrt(1 - |v|^2); |v| >= 1 is
 * first normalised onto the sphere (w = 0, a half turn).  R is the rotation
 * matrix of that quaternion (a turn by 2 asin|v| about v).  Order of
 * operations: n2 = (x*x + y*y) + z*z; outside, x = x / sqrt(n2) and so on;
 * R[0] = 1 - 2*(y*y + z*z), R[1] = 2*(x*y - w*z), R[2] = 2*(x*z + w*y),
 * R[3] = 2*(x*y + w*z), R[4] = 1 - 2*(x*x + z*z), R[5] = 2*(y*z - w*x),
 * R[6] = 2*(x*z - w*y), R[7] = 2*(y*z + w*x), R[8] = 1 - 2*(x*x + y*y).
 * dR (may be NULL) receives dR/dv_p at dR[9*p + e].
 */
static void orc_versor(const double v[3], double R[9], double *dR) {
    double x = v[0], y = v[1], z = v[2], w;
    const double n2 = x * x + y * y + z * z;
    const int outside = n2 >= 1.0;
    const double nrm = outside ? sqrt(n2) : 1.0;
    if (outside) {
        x = x / nrm;
        y = y / nrm;
        z = z / nrm;
        w = 0.0;
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
    /* partial derivatives of the nine entries with respect to x, y, z, w */
    const double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    const double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double q[3] = {x, y, z};
    for (int p = 0; p < 3; p++) {
        /* d(x, y, z, w)/d v_p: inside (e_p, -v_p / w); outside (e_p - q q_p) / |v| and 0 */
        double dq[3], dw = 0.0;
        for (int c = 0; c < 3; c++) dq[c] = outside ? ((c == p) - q[c] * q[p]) / nrm : (double)(c == p);
        if (!outside) dw = -v[p] / w;
        for (int e = 0; e < 9; e++) dR[9 * p + e] = Dx[e] * dq[0] + Dy[e] * dq[1] + Dz[e] * dq[2] + Dw[e] * dw;
    }
}

void orc_affine_mode(const float prm[9], const int nf[3], const float sf_in[3], const int nm[3],
                     const float sm_in[3], int rot_mode, int scale_mode, double out[12], double *dout);

void orc_affine(const float prm[9], const int nf[3], const float sf_in[3], const int nm[3],
                const float sm_in[3], double out[12], double *dout) {
    orc_affine_mode(prm, nf, sf_in, nm, sm_in, 0, 0, out, dout);
}

/* The same with the rotation parameters as Euler angles in degrees (rot_mode
 * 0) or the unit-ball versor of R14 (1), and the scale parameters as factors
 * sigma (scale_mode 0) or zero-centred offsets s, sigma = 1 + s (1, R15). */
void orc_affine_mode(const float prm[9], const int nf[3], const float sf_in[3], const int nm[3],
                     const float sm_in[3], int rot_mode, int scale_mode, double out[12], double *dout) {
    double t[3], ang[3], sig[3], sf[3], sm[3], cf[3], cm[3], vv[3];
    for (int a = 0; a < 3; a++) {
        t[a] = (double)prm[a];
        ang[a] = orc_deg2rad((double)prm[3 + a]);
        vv[a] = (double)prm[3 + a];
        sig[a] = scale_mode ? 1.0 + (double)prm[6 + a] : (double)prm[6 + a];
        sf[a] = (double)sf_in[a];
        sm[a] = (double)sm_in[a];
        cf[a] = sf[a] * ((double)(nf[a] - 1) * 0.5);
        cm[a] = sm[a] * ((double)(nm[a] - 1) * 0.5);
    }
    double Rx[9], Ry[9], Rz[9], Rzy[9], R[9], dRv[27];
    if (rot_mode) {
        orc_versor(vv, R, dout ? dRv : NULL);
    } else {
        orc_rot_x(ang[0], 0, Rx);
        orc_rot_y(ang[1], 0, Ry);
        orc_rot_z(ang[2], 0, Rz);
        orc_mat3_mul(Rz, Ry, Rzy);
        orc_mat3_mul(Rzy, Rx, R);
    }
    for (int a = 0; a < 3; a++) {
        double s = 0.0;
        for (int c = 0; c < 3; c++) {
            double rs = R[3 * a + c] * sig[c];
            out[4 * a + c] = (rs * sf[c]) / sm[a];
            s = s + rs * cf[c];
        }
        out[4 * a + 3] = ((cm[a] + t[a]) - s) / sm[a];
    }
    if (!dout) return;
    memset(dout, 0, sizeof(double) * 12 * 9);
    /* translation: d b_a / d t_a = 1 / s_m[a] */
    for (int a = 0; a < 3; a++) dout[9 * (4 * a + 3) + a] = 1.0 / sm[a];
    /* rotation: dR/d(deg) = (pi/180) * (Rz Ry Rx with one factor differentiated),
     * or the versor's dR/dv_p */
    for (int p = 0; p < 3; p++) {
        double dX[9], dY[9], dZ[9], M1[9], dR[9];
        double k = orc_deg2rad(1.0);
        if (rot_mode) {
            memcpy(dR, dRv + 9 * p, sizeof dR);
            k = 1.0;
        } else {
            orc_rot_x(ang[0], p == 0, dX);
            orc_rot_y(ang[1], p == 1, dY);
            orc_rot_z(ang[2], p == 2, dZ);
            orc_mat3_mul(dZ, dY, M1);
            orc_mat3_mul(M1, dX, dR);
        }
        for (int a = 0; a < 3; a++) {
            double s = 0.0;
            for (int c = 0; c < 3; c++) {
                double drs = dR[3 * a + c] * k * sig[c];
                dout[9 * (4 * a + c) + 3 + p] = drs * sf[c] / sm[a];
                s += drs * cf[c];
            }
            dout[9 * (4 * a + 3) + 3 + p] = -s / sm[a];
        }
    }
    /* scale: only column c = p of R diag(sigma) depends on sigma_p */
    for (int p = 0; p < 3; p++)
        for (int a = 0; a < 3; a++) {
            dout[9 * (4 * a + p) + 6 + p] = R[3 * a + p] * sf[p] / sm[a];
            dout[9 * (4 * a + 3) + 6 + p] = -R[3 * a + p] * cf[p] / sm[a];
        }
}

/* R17: the general affine of the Methodology's 12 degrees of freedom (the
 * affine family of the Introduction: translation, rotation, scale and skew).
 * prm = [M | t] row-major, M 3x3 and t in mm; the moving physical point is
 * M (p - c_f) + c_m + t, the 9-parameter form's R diag(sigma) replaced by M.
 * Index space: A = diag(1/s_m) M diag(s_f), b = diag(1/s_m) (c_m + t - M c_f),
 * evaluated in the same order as orc_affine_mode.  dout (12 x 12) is
 * d[A|b]/dprm, prm index 4a + c as in [M | t]. */
void orc_affine_matrix(const float prm[12], const int nf[3], const float sf_in[3], const int nm[3],
                       const float sm_in[3], double out[12], double *dout) {
    double sf[3], sm[3], cf[3], cm[3];
    for (int a = 0; a < 3; a++) {
        sf[a] = (double)sf_in[a];
        sm[a] = (double)sm_in[a];
        cf[a] = sf[a] * ((double)(nf[a] - 1) * 0.5);
        cm[a] = sm[a] * ((double)(nm[a] - 1) * 0.5);
    }
    for (int a = 0; a < 3; a++) {
        double s = 0.0;
        for (int c = 0; c < 3; c++) {
            double m = (double)prm[4 * a + c];
            out[4 * a + c] = (m * sf[c]) / sm[a];
            s = s + m * cf[c];
        }
        out[4 * a + 3] = ((cm[a] + (double)prm[4 * a + 3]) - s) / sm[a];
    }
    if (!dout) return;
    memset(dout, 0, sizeof(double) * 12 * 12);
    for (int a = 0; a < 3; a++) {
        /* row a of [A | b] depends on row a of [M | t] only */
        for (int c = 0; c < 3; c++) {
            dout[12 * (4 * a + c) + 4 * a + c] = sf[c] / sm[a];
            dout[12 * (4 * a + 3) + 4 * a + c] = -cf[c] / sm[a];
        }
        dout[12 * (4 * a + 3) + 4 * a + 3] = 1.0 / sm[a];
    }
}

/* R3: each of the 12 entries of [A | b] is quantised to 16.16 fixed point as
 * llround(x * 65536); returns ORC_ERANGE if one does not fit int32. */
int orc_affine_q16(const double aff[12], int32_t q[12]) {
    for (int e = 0; e < 12; e++) {
        double s = aff[e] * 65536.0;
        if (!(fabs(s) <= 2147483647.0)) return ORC_ERANGE;
        long long r = llround(s);
        if (r > 2147483647LL || r < -2147483647LL - 1) return ORC_ERANGE;
        q[e] = (int32_t)r;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* R3 + R4: fixed-point coordinate and integer trilinear resampling          */
/* ------------------------------------------------------------------------ */

/* R4 stage lerp with an 8-bit weight f in [0, 255]: (a (256 - f) + b f + 128) >> 8 */
static uint32_t orc_lerp8(uint32_t a, uint32_t b, uint32_t f) {
    return (a * (256u - f) + b * f + 128u) >> 8;
}

/*
 * R3: U_a = A_a0 i + A_a1 j + A_a2 k + b_a in exact 64-bit arithmetic
 * (16.16 moving index).  The voxel is inside the overlap iff
 * 0 <= U_a <= (n_a - 1) * 65536 on all three axes; outside voxels are left
 * out of the histogram.  R4: the cell is ix = U >> 16, its 8-bit weight
 * fx = (U & 0xFFFF) >> 8 (truncated), the upper neighbour is clamped to
 * n - 1 (its weight is then 0).  Lerp along x for the four (y, z) pairs,
 * then along y, then along z.  Returns 0 and leaves *val alone outside.
 */
static int orc_sample_hard(const void *mov, int mdtype, int mdepth, const int nm[3], const int32_t q[12],
                           int64_t i, int64_t j, int64_t k, uint32_t *val) {
    int64_t U[3];
    for (int a = 0; a < 3; a++) {
        U[a] = (int64_t)q[4 * a + 0] * i + (int64_t)q[4 * a + 1] * j + (int64_t)q[4 * a + 2] * k +
               (int64_t)q[4 * a + 3];
        if (U[a] < 0 || U[a] > (int64_t)(nm[a] - 1) * 65536) return 0;
    }
    int64_t c0[3], c1[3];
    uint32_t f[3];
    for (int a = 0; a < 3; a++) {
        c0[a] = U[a] >> 16;
        c1[a] = c0[a] + 1 <= nm[a] - 1 ? c0[a] + 1 : nm[a] - 1;
        f[a] = (uint32_t)((U[a] & 0xFFFF) >> 8);
    }
    uint32_t v[2][2][2]; /* v[z][y][x] */
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++)
                v[dz][dy][dx] = orc_get_clamped(mov, mdtype, mdepth,
                                                orc_index(nm, dx ? c1[0] : c0[0], dy ? c1[1] : c0[1], dz ? c1[2] : c0[2]));
    uint32_t ex[2][2];
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++) ex[dz][dy] = orc_lerp8(v[dz][dy][0], v[dz][dy][1], f[0]);
    uint32_t ey[2];
    for (int dz = 0; dz < 2; dz++) ey[dz] = orc_lerp8(ex[dz][0], ex[dz][1], f[1]);
    *val = orc_lerp8(ey[0], ey[1], f[2]);
    return 1;
}

/* v(T(x)) on the fixed grid (value 0 outside the overlap); same type as the moving volume. */
void orc_resample(const void *mov, int mdtype, int mdepth, const int nm[3], const int nf[3], const int32_t q[12],
                  void *out) {
    for (int64_t k = 0; k < nf[2]; k++)
        for (int64_t j = 0; j < nf[1]; j++)
            for (int64_t i = 0; i < nf[0]; i++) {
                uint32_t val = 0;
                orc_sample_hard(mov, mdtype, mdepth, nm, q, i, j, k, &val);
                int64_t o = orc_index(nf, i, j, k);
                if (mdtype == ORC_U8) ((uint8_t *)out)[o] = (uint8_t)val;
                else ((uint16_t *)out)[o] = (uint16_t)val;
            }
}

/*
 * R5: joint histogram h[bf * bins + bm] of (fixed bin, moving bin) over the
 * voxels inside the overlap -- the paper's "full histogram" over all voxels
 * (Discussion).  Row = fixed bin.  Returns the overlap count N.
 */
/*
 * R16, random sampling (the Discussion's open question: ITK Mattes samples
 * the image at random, MICUDA uses every voxel): a fixed voxel with linear
 * index x takes part iff fmix32((uint32) x ^ fmix32(seed)) < threshold, where
 * fmix32 is the 32-bit finalizer of MurmurHash3 (xor-shift by 16, multiply by
 * 0x85ebca6b, xor-shift by 13, multiply by 0xc2b2ae35, xor-shift by 16, all
 * mod 2^32) and threshold = floor(fraction * 2^32) for 0 < fraction < 1.  The
 * subset is fixed per seed (a property of the fixed volume, as in Mattes'
 * method), so the metric stays a deterministic function of the transform.
 */
uint32_t orc_fmix32(uint32_t k) {
    k ^= k >> 16;
    k *= 0x85ebca6bu;
    k ^= k >> 13;
    k *= 0xc2b2ae35u;
    k ^= k >> 16;
    return k;
}

int orc_sampled(int64_t x, uint32_t seed, uint32_t threshold) {
    return orc_fmix32((uint32_t)x ^ orc_fmix32(seed)) < threshold;
}

uint32_t orc_sample_threshold(double fraction) {
    if (!(fraction > 0.0 && fraction < 1.0)) return 0;
    return (uint32_t)floor(fraction * 4294967296.0);
}

/* Joint histogram over the overlap, restricted to the sampled fixed voxels
 * when threshold > 0 (R16); every voxel when threshold == 0. */
int64_t orc_joint_hist_s(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                         const int nm[3], const int32_t q[12], int bins, uint32_t seed, uint32_t threshold,
                         uint64_t *hist);

int64_t orc_joint_hist(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                       const int nm[3], const int32_t q[12], int bins, uint64_t *hist) {
    return orc_joint_hist_s(fbins, nf, mov, mdtype, mdepth, nm, q, bins, 0u, 0u, hist);
}

int64_t orc_joint_hist_s(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                         const int nm[3], const int32_t q[12], int bins, uint32_t seed, uint32_t threshold,
                         uint64_t *hist) {
    memset(hist, 0, sizeof(uint64_t) * (size_t)bins * (size_t)bins);
    int64_t n = 0;
    for (int64_t k = 0; k < nf[2]; k++)
        for (int64_t j = 0; j < nf[1]; j++)
            for (int64_t i = 0; i < nf[0]; i++) {
                uint32_t val;
                if (threshold && !orc_sampled(orc_index(nf, i, j, k), seed, threshold)) continue;
                if (!orc_sample_hard(mov, mdtype, mdepth, nm, q, i, j, k, &val)) continue;
                int bf = fbins[orc_index(nf, i, j, k)];
                int bm = orc_bin_of(val, bins, mdepth);
                hist[(size_t)bf * (size_t)bins + (size_t)bm] += 1;
                n++;
            }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Entropies (Eq. 1, Eq. 2, R6, R7)                                          */
/* ------------------------------------------------------------------------ */

/* Neumaier compensated summation, FP64. */
typedef struct { double s, c; } orc_sum;
static void orc_sum_add(orc_sum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double orc_sum_get(const orc_sum *a) { return a->s + a->c; }

/*
 * Entropy of the distribution p_i = c_i / N from counts (integers or, for the
 * Parzen form, non-negative reals).
 * q == 1: Shannon, Eq. (1): H = -sum p ln p = ln N - (1/N) sum c ln c, with
 *         0 ln 0 = 0 (R6: natural log, nats; bits = nats / ln 2).
 * q != 1: Tsallis (R7, the paper names it but prints no formula; standard
 *         definition): S_q = (1 - sum p^q) / (q - 1) = (1 - N^-q sum c^q)/(q - 1),
 *         zero cells left out.
 */
static double orc_entropy_counts(const double *c, int64_t m, double N, double q) {
    orc_sum s = {0, 0};
    if (q == 1.0) {
        for (int64_t x = 0; x < m; x++)
            if (c[x] > 0) orc_sum_add(&s, c[x] * log(c[x]));
        return log(N) - orc_sum_get(&s) / N;
    }
    for (int64_t x = 0; x < m; x++)
        if (c[x] > 0) orc_sum_add(&s, pow(c[x], q));
    return (1.0 - pow(N, -q) * orc_sum_get(&s)) / (q - 1.0);
}

/*
 * Marginal and joint entropies and MI for each q from one histogram (the
 * paper computes Shannon and Tsallis from the same histogram, Discussion).
 * Marginals are the row sums (fixed) and column sums (moving) of the overlap
 * histogram (R5).
 * MI, Eq. (2): I = H(F) + H(M) - H(F,M).
 * Tsallis MI (R7): form 0, additive: I_q = S_q(F) + S_q(M) - S_q(F,M);
 *                  form 1, pseudo-additive: I_q = S_q(F) + S_q(M)
 *                        + (1 - q) S_q(F) S_q(M) - S_q(F,M).
 * bits != 0 divides the Shannon entropies by ln 2.  Outputs per q:
 * mi[iq], h[3*iq + 0..2] = (H_F, H_M, H_FM).  N = 0 gives NaN.
 */
int orc_entropies(const double *hist, int bins, const double *qs, int nq, int form, int bits,
                  double *mi, double *h) {
    size_t B = (size_t)bins;
    double *rows = calloc(B, sizeof(double)), *cols = calloc(B, sizeof(double));
    if (!rows || !cols) { free(rows); free(cols); return ORC_ENOMEM; }
    double N = 0;
    for (size_t r = 0; r < B; r++)
        for (size_t c = 0; c < B; c++) {
            double v = hist[r * B + c];
            rows[r] += v;
            cols[c] += v;
            N += v;
        }
    for (int iq = 0; iq < nq; iq++) {
        double q = qs[iq];
        double hf, hm, hfm;
        if (N <= 0) {
            hf = hm = hfm = NAN;
        } else {
            hf = orc_entropy_counts(rows, (int64_t)B, N, q);
            hm = orc_entropy_counts(cols, (int64_t)B, N, q);
            hfm = orc_entropy_counts(hist, (int64_t)(B * B), N, q);
            if (q == 1.0 && bits) {
                hf /= log(2.0);
                hm /= log(2.0);
                hfm /= log(2.0);
            }
        }
        double I = hf + hm - hfm;
        if (q != 1.0 && form == 1) I += (1.0 - q) * hf * hm;
        if (mi) mi[iq] = I;
        if (h) {
            h[3 * iq + 0] = hf;
            h[3 * iq + 1] = hm;
            h[3 * iq + 2] = hfm;
        }
    }
    free(rows);
    free(cols);
    return ORC_OK;
}

/*
 * One hard-binned MI evaluation per transform, parallel across transforms
 * (each transform is computed serially and independently).
 * prm: n x 9 parameters (R2); qs: nq exponents (1 = Shannon).
 * Outputs: mi n x nq, h n x nq x 3 (NULL ok), count n (NULL ok).
 * Returns ORC_ERANGE if an affine does not fit 16.16.
 */
int orc_mi_eval(const uint8_t *fbins, const int nf[3], const float sf[3], const void *mov, int mdtype,
                int mdepth, const int nm[3], const float sm[3], int bins, const float *prm, int n,
                const double *qs, int nq, int form, int bits, int nthreads, double *mi, double *h,
                int64_t *count) {
    int err = ORC_OK;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int t = 0; t < n; t++) {
        double aff[12];
        int32_t q[12];
        orc_affine(prm + 9 * (size_t)t, nf, sf, nm, sm, aff, NULL);
        if (orc_affine_q16(aff, q) != ORC_OK) {
#pragma omp atomic write
            err = ORC_ERANGE;
            continue;
        }
        size_t B2 = (size_t)bins * (size_t)bins;
        uint64_t *hh = malloc(B2 * sizeof(uint64_t));
        double *hd = malloc(B2 * sizeof(double));
        if (!hh || !hd) {
            free(hh);
            free(hd);
#pragma omp atomic write
            err = ORC_ENOMEM;
            continue;
        }
        int64_t N = orc_joint_hist(fbins, nf, mov, mdtype, mdepth, nm, q, bins, hh);
        for (size_t x = 0; x < B2; x++) hd[x] = (double)hh[x];
        orc_entropies(hd, bins, qs, nq, form, bits, mi + (size_t)t * nq, h ? h + (size_t)t * nq * 3 : NULL);
        if (count) count[t] = N;
        free(hh);
        free(hd);
    }
    return err;
}

/* Same, from 16.16 affines given directly (n x 12 int32), over the sampled
 * fixed voxels (R16) when threshold > 0. */
int orc_mi_eval_q16_s(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                      const int nm[3], int bins, const int32_t *q, int n, const double *qs, int nq, int form,
                      int bits, int nthreads, uint32_t seed, uint32_t threshold, double *mi, double *h,
                      int64_t *count);

int orc_mi_eval_q16(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                    const int nm[3], int bins, const int32_t *q, int n, const double *qs, int nq, int form,
                    int bits, int nthreads, double *mi, double *h, int64_t *count) {
    return orc_mi_eval_q16_s(fbins, nf, mov, mdtype, mdepth, nm, bins, q, n, qs, nq, form, bits, nthreads, 0u, 0u,
                             mi, h, count);
}

int orc_mi_eval_q16_s(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                      const int nm[3], int bins, const int32_t *q, int n, const double *qs, int nq, int form,
                      int bits, int nthreads, uint32_t seed, uint32_t threshold, double *mi, double *h,
                      int64_t *count) {
    int err = ORC_OK;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int t = 0; t < n; t++) {
        size_t B2 = (size_t)bins * (size_t)bins;
        uint64_t *hh = malloc(B2 * sizeof(uint64_t));
        double *hd = malloc(B2 * sizeof(double));
        if (!hh || !hd) {
            free(hh);
            free(hd);
#pragma omp atomic write
            err = ORC_ENOMEM;
            continue;
        }
        int64_t N = orc_joint_hist_s(fbins, nf, mov, mdtype, mdepth, nm, q + 12 * (size_t)t, bins, seed, threshold, hh);
        for (size_t x = 0; x < B2; x++) hd[x] = (double)hh[x];
        orc_entropies(hd, bins, qs, nq, form, bits, mi + (size_t)t * nq, h ? h + (size_t)t * nq * 3 : NULL);
        if (count) count[t] = N;
        free(hh);
        free(hd);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* R8 / R9: Parzen (differentiable) form                                     */
/* ------------------------------------------------------------------------ */

/* Centred cubic B-spline and its derivative. */
double orc_beta3(double x) {
    double a = fabs(x);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}
double orc_dbeta3(double x) {
    double a = fabs(x), s = x < 0 ? -1.0 : 1.0;
    if (a < 1.0) return s * (-2.0 * a + 1.5 * a * a);
    if (a < 2.0) return s * (-0.5 * (2.0 - a) * (2.0 - a));
    return 0.0;
}

/* Normalised intensity in [0, 1]: integer v / (2^d - 1); float clamped. */
static double orc_norm_value(const void *data, int dtype, int depth, int64_t idx) {
    if (dtype == ORC_F32) {
        double v = ((const float *)data)[idx];
        if (!(v == v)) v = 0.0;
        return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    }
    double vmax = (double)((((uint64_t)1) << depth) - 1u);
    double v = (double)orc_get_u(data, dtype, idx);
    return v > vmax ? 1.0 : v / vmax;
}

/*
 * R8 fixed bin of the Parzen form: floor(f (B - 4)) + 2 with f the normalised
 * intensity, i.e. bins 2 .. B-2.  Integer volumes use the exact integer
 * quotient (v (B - 4)) div (2^d - 1); float volumes the FP64 product.
 */
int orc_parzen_fixed_bin(const void *data, int dtype, int depth, int64_t idx, int B) {
    if (dtype == ORC_F32) {
        double f = orc_norm_value(data, dtype, depth, idx);
        return (int)floor(f * (double)(B - 4)) + 2;
    }
    uint64_t vmax = (((uint64_t)1) << depth) - 1u;
    uint64_t v = orc_get_u(data, dtype, idx);
    if (v > vmax) v = vmax;
    return (int)((v * (uint64_t)(B - 4)) / vmax) + 2;
}

/*
 * FP64 trilinear value and gradient (with respect to the moving index u) of
 * the normalised moving volume at a real moving index u inside
 * [0, n-1]^3.  The cell is c = min(floor(u), n - 2), weight u - c, so the
 * value is continuous and the gradient is that of the cell on the upper side
 * of u (of the lower cell on the top face).
 */
static void orc_trilinear(const void *mov, int mdtype, int mdepth, const int nm[3], const double u[3],
                          double *m, double g[3]) {
    int64_t c[3];
    double w[3];
    for (int a = 0; a < 3; a++) {
        double fl = floor(u[a]);
        if (fl > nm[a] - 2) fl = nm[a] - 2;
        if (fl < 0) fl = 0;
        c[a] = (int64_t)fl;
        w[a] = u[a] - fl;
    }
    double v[2][2][2];
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++)
                v[dz][dy][dx] = orc_norm_value(mov, mdtype, mdepth, orc_index(nm, c[0] + dx, c[1] + dy, c[2] + dz));
    double val = 0, gx = 0, gy = 0, gz = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double wx = dx ? w[0] : 1 - w[0], wy = dy ? w[1] : 1 - w[1], wz = dz ? w[2] : 1 - w[2];
                double sx = dx ? 1 : -1, sy = dy ? 1 : -1, sz = dz ? 1 : -1;
                val += wx * wy * wz * v[dz][dy][dx];
                gx += sx * wy * wz * v[dz][dy][dx];
                gy += wx * sy * wz * v[dz][dy][dx];
                gz += wx * wy * sz * v[dz][dy][dx];
            }
    *m = val;
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

/* Entropy of a normalised distribution P (FP64), zero cells left out. */
static double orc_entropy_p(const double *p, int64_t m, double q) {
    orc_sum s = {0, 0};
    if (q == 1.0) {
        for (int64_t x = 0; x < m; x++)
            if (p[x] > 0) orc_sum_add(&s, -p[x] * log(p[x]));
        return orc_sum_get(&s);
    }
    for (int64_t x = 0; x < m; x++)
        if (p[x] > 0) orc_sum_add(&s, pow(p[x], q));
    return (1.0 - orc_sum_get(&s)) / (q - 1.0);
}

/*
 * R8: Parzen soft joint histogram, normalised:
 *   P(i, k) = (1/N) sum_x beta0(i - fb(x)) beta3(k - m~(T x)),
 * fb(x) the fixed bin above (a box kernel: one bin per voxel), m~ = m (B - 4) + 2
 * with m the FP64 trilinear value of the normalised moving volume at the real
 * moving index u = A x + b (FP64), N the overlap count, the overlap being
 * 0 <= u_a <= n_a - 1 on all axes.  MI per q from P as in orc_entropies.
 * R9: the gradient differentiates P with N and the overlap held fixed:
 *   dMI/dtheta = sum_x (dMI/dm~_x) (B - 4) grad m(u_x) . du_x/dtheta,
 *   dMI/dm~_x  = -(1/N) sum_k W(fb(x), k) beta3'(k - m~_x),
 *   W(i, k)    = dMI/dP(i, k) with P_F(i) = sum_k P and P_M(k) = sum_i P:
 *     Shannon: ln P - ln P_F - ln P_M - 1
 *     Tsallis: dS(F) + dS(M) [+ (1-q)(dS(F) S(M) + S(F) dS(M)) if form 1] - dS(FM),
 *              dS(X) = -q X^(q-1) / (q - 1) at the cell's X,
 *   and W = 0 on cells with P = 0 (no voxel moves them: beta3' vanishes there).
 * du/dtheta comes from daff (12 x npar, d [A|b] / d theta: npar = 9 from
 * orc_affine / orc_affine_mode, 12 from orc_affine_matrix).
 * If mask is not NULL, the voxel set is the mask (instead of the overlap)
 * and sample coordinates are clamped into the volume: this is the function
 * the gradient differentiates, used for finite-difference checks.
 * Outputs: mi[nq], grad[nq*npar] (NULL ok), count (NULL ok), phist (B*B, NULL ok).
 */
int orc_parzen(const void *fix, int fdtype, int fdepth, const int nf[3], const void *mov, int mdtype, int mdepth,
               const int nm[3], const double aff[12], const double *daff, int npar, int B, const double *qs, int nq,
               int form, int bits, const uint8_t *mask, double *mi, double *grad, int64_t *count, double *phist) {
    if (B < 8 || npar < 1 || npar > 12) return ORC_EINVAL;
    size_t BB = (size_t)B * (size_t)B;
    int64_t nvf = orc_nvox(nf);
    double *P = calloc(BB, sizeof(double));
    double *PF = calloc((size_t)B, sizeof(double)), *PM = calloc((size_t)B, sizeof(double));
    double *W = calloc(BB, sizeof(double));
    if (!P || !PF || !PM || !W) { free(P); free(PF); free(PM); free(W); return ORC_ENOMEM; }
    int64_t N = 0;
    /* pass 1: soft histogram */
    for (int64_t k = 0; k < nf[2]; k++)
        for (int64_t j = 0; j < nf[1]; j++)
            for (int64_t i = 0; i < nf[0]; i++) {
                int64_t idx = orc_index(nf, i, j, k);
                double u[3];
                int inside = 1;
                for (int a = 0; a < 3; a++) {
                    u[a] = aff[4 * a + 0] * (double)i + aff[4 * a + 1] * (double)j + aff[4 * a + 2] * (double)k +
                           aff[4 * a + 3];
                    if (!(u[a] >= 0.0 && u[a] <= (double)(nm[a] - 1))) inside = 0;
                }
                if (mask) {
                    if (!mask[idx]) continue;
                    for (int a = 0; a < 3; a++) u[a] = u[a] < 0 ? 0 : (u[a] > nm[a] - 1 ? nm[a] - 1 : u[a]);
                } else if (!inside) {
                    continue;
                }
                double m, g[3];
                orc_trilinear(mov, mdtype, mdepth, nm, u, &m, g);
                double mt = m * (double)(B - 4) + 2.0;
                int fb = orc_parzen_fixed_bin(fix, fdtype, fdepth, idx, B);
                /* beta3 vanishes beyond distance 2, so bins outside floor(mt) -+ 2 add nothing */
                int k0 = (int)floor(mt);
                for (int kk = k0 - 2; kk <= k0 + 2; kk++) {
                    if (kk < 0 || kk >= B) continue;
                    double w = orc_beta3((double)kk - mt);
                    if (w != 0.0) P[(size_t)fb * B + kk] += w;
                }
                N++;
            }
    if (count) *count = N;
    if (phist)
        for (size_t x = 0; x < BB; x++) phist[x] = N > 0 ? P[x] / (double)N : NAN;
    if (N == 0) {
        for (int iq = 0; iq < nq; iq++) {
            mi[iq] = NAN;
            if (grad)
                for (int p = 0; p < npar; p++) grad[npar * iq + p] = NAN;
        }
        free(P); free(PF); free(PM); free(W);
        return ORC_OK;
    }
    for (size_t x = 0; x < BB; x++) P[x] /= (double)N;
    for (int r = 0; r < B; r++)
        for (int c = 0; c < B; c++) {
            PF[r] += P[(size_t)r * B + c];
            PM[c] += P[(size_t)r * B + c];
        }
    double lnb = bits ? log(2.0) : 1.0;
    for (int iq = 0; iq < nq; iq++) {
        double q = qs[iq];
        double hf = orc_entropy_p(PF, B, q), hm = orc_entropy_p(PM, B, q), hfm = orc_entropy_p(P, (int64_t)BB, q);
        if (q == 1.0) { hf /= lnb; hm /= lnb; hfm /= lnb; }
        double I = hf + hm - hfm;
        if (q != 1.0 && form == 1) I += (1.0 - q) * hf * hm;
        mi[iq] = I;
        if (!grad) continue;
        for (int r = 0; r < B; r++)
            for (int c = 0; c < B; c++) {
                double p = P[(size_t)r * B + c];
                double w = 0.0;
                if (p > 0.0) {
                    if (q == 1.0) {
                        w = (log(p) - log(PF[r]) - log(PM[c]) - 1.0) / lnb;
                    } else {
                        double dSF = -q * pow(PF[r], q - 1.0) / (q - 1.0);
                        double dSM = -q * pow(PM[c], q - 1.0) / (q - 1.0);
                        double dSJ = -q * pow(p, q - 1.0) / (q - 1.0);
                        w = dSF + dSM - dSJ;
                        if (form == 1) w += (1.0 - q) * (dSF * hm + hf * dSM);
                    }
                }
                W[(size_t)r * B + c] = w;
            }
        /* pass 2: adjoint */
        double G[12] = {0};
        for (int64_t k = 0; k < nf[2]; k++)
            for (int64_t j = 0; j < nf[1]; j++)
                for (int64_t i = 0; i < nf[0]; i++) {
                    int64_t idx = orc_index(nf, i, j, k);
                    double u[3];
                    int inside = 1;
                    for (int a = 0; a < 3; a++) {
                        u[a] = aff[4 * a + 0] * (double)i + aff[4 * a + 1] * (double)j + aff[4 * a + 2] * (double)k +
                               aff[4 * a + 3];
                        if (!(u[a] >= 0.0 && u[a] <= (double)(nm[a] - 1))) inside = 0;
                    }
                    if (mask) {
                        if (!mask[idx]) continue;
                        for (int a = 0; a < 3; a++) u[a] = u[a] < 0 ? 0 : (u[a] > nm[a] - 1 ? nm[a] - 1 : u[a]);
                    } else if (!inside) {
                        continue;
                    }
                    double m, g[3];
                    orc_trilinear(mov, mdtype, mdepth, nm, u, &m, g);
                    double mt = m * (double)(B - 4) + 2.0;
                    int fb = orc_parzen_fixed_bin(fix, fdtype, fdepth, idx, B);
                    double s = 0.0;
                    int k0 = (int)floor(mt);
                    for (int kk = k0 - 2; kk <= k0 + 2; kk++)
                        if (kk >= 0 && kk < B) s += W[(size_t)fb * B + kk] * orc_dbeta3((double)kk - mt);
                    double dmt = -s / (double)N * (double)(B - 4);
                    double x4[4] = {(double)i, (double)j, (double)k, 1.0};
                    for (int p = 0; p < npar; p++) {
                        double d = 0.0;
                        for (int a = 0; a < 3; a++) {
                            double du = 0.0;
                            for (int c = 0; c < 4; c++) du += daff[npar * (4 * a + c) + p] * x4[c];
                            d += g[a] * du;
                        }
                        G[p] += dmt * d;
                    }
                }
        for (int p = 0; p < npar; p++) grad[npar * iq + p] = G[p];
    }
    free(P); free(PF); free(PM); free(W);
    (void)nvf;
    return ORC_OK;
}

/* Overlap mask of the Parzen form at an affine (FP64 bounds of R8). */
void orc_overlap_mask(const int nf[3], const int nm[3], const double aff[12], uint8_t *mask) {
    for (int64_t k = 0; k < nf[2]; k++)
        for (int64_t j = 0; j < nf[1]; j++)
            for (int64_t i = 0; i < nf[0]; i++) {
                int inside = 1;
                for (int a = 0; a < 3; a++) {
                    double u = aff[4 * a + 0] * (double)i + aff[4 * a + 1] * (double)j + aff[4 * a + 2] * (double)k +
                               aff[4 * a + 3];
                    if (!(u >= 0.0 && u <= (double)(nm[a] - 1))) inside = 0;
                }
                mask[orc_index(nf, i, j, k)] = (uint8_t)inside;
            }
}
