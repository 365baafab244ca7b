/* CPU oracle for the CityGaussian rendering hot path.  TEST INFRASTRUCTURE ONLY.
 *
 * This is the plain, slow, single-threaded statement of what the GPU library must
 * compute.  Only the test-suite, the package's smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code with the
 * CUDA library.
 *
 * What it computes (paper: CityGaussian, arXiv 2404.01133):
 *   - Eq. 1 (Sec. 3.1): c(x) = sum_k alpha_k c_k G2D_k(x) prod_{t<k} (1 - alpha_t G2D_t(x)),
 *     with G2D_k = proj(G_k, kappa, tau) and the Gaussians sorted in depth order.
 *     The per-Gaussian projection, SH colour and the compositing thresholds follow the
 *     3DGS conventions the paper defers to (Sec. 3.1): alpha = min(0.99, o exp(power)),
 *     entries with alpha < 1/255 are skipped, a pixel stops before the entry that would
 *     take its transmittance below 1e-4, ties in depth go to the lower index.
 *   - Differentiable rendering (Sec. 3.1): the analytic gradient of the above.
 *   - Sec. 3.2.2 and Eqs. 2 and 4: foreground normalisation, contraction, the uniform block
 *     grid over the contracted cube, stable grouping by block, the block of a camera pose
 *     (oracle_partition.inc).
 *   - Eq. 3 (Sec. 3.2.2): the SSIM loss of two renders (oracle_ssim.inc).
 *   - Sec. 3.3.1: nested detail levels per block from a significance ranking (opacity x
 *     volume, optionally weighted by per-pixel hit counts), oracle_levels.inc.
 *   - Eq. 7 (Sec. 3.3.2): MAD block bounds; block frustum test by projecting the corners
 *     in front of the camera; the camera's own block is always kept; the level of a
 *     block comes from the minimum corner distance; fusion by concatenation.
 *
 * Precision.  REAL is float (the parity build, liboracle_f32) or double (the build used
 * for finite-difference pins, liboracle_f64).  The key path -- everything that turns
 * floating point into an integer the GPU must reproduce (near/degenerate culls, radius,
 * tile rect, depth bits) -- is always evaluated in FP32 by project_one_f.  Compositing
 * decisions (skip, stop) are taken in REAL.  The falloff exp(power) is the exponential
 * rounded once to REAL (the FP64 exponential, then one rounding): the paper fixes no
 * precision for it, and a correctly rounded value is the plain definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

#ifndef REAL
#define REAL float
#endif

typedef struct {
    float R[9];        /* world -> camera rotation, row major, OpenCV axes */
    float t[3];        /* world -> camera translation: x_cam = R x + t */
    float campos[3];   /* camera centre in world coordinates */
    float fx, fy, cx, cy;
    int32_t width, height;
} orc_camera;

typedef struct {
    int32_t tile;      /* tile side in pixels */
    float near_z;      /* near plane (camera-space z) */
    float bg[3];       /* background colour */
} orc_config;

#define T float
#define SUF _f
#include "oracle_project.inc"
#undef T
#undef SUF
#define T REAL
#define SUF _r
#include "oracle_project.inc"
#undef T
#undef SUF

/* flag bits returned per Gaussian by orc_project */
#define F_CULL_NEAR 1
#define F_CULL_DET 2
#define F_CLAMP_X 4
#define F_CLAMP_Y 8
#define F_CLAMP_R 16
#define F_CLAMP_G 32
#define F_CLAMP_B 64

static uint64_t fnv(uint64_t h, uint64_t v)
{
    for (int i = 0; i < 8; i++) { h ^= (v >> (8 * i)) & 0xff; h *= 1099511628211ull; }
    return h;
}

/* ------------------------------------------------------------------------------------- */
/* Real spherical harmonics, orthonormal on the unit sphere, index l^2 + l + m, with the   */
/* Condon-Shortley phase: Y_{l,m} = sqrt2 Re Y_l^m (m > 0), sqrt2 Im Y_l^|m| (m < 0).      */
/* Polynomials in the components of the unit view direction (x, y, z).                     */
/* ------------------------------------------------------------------------------------- */
static void sh_consts(REAL k[10])
{
    const double pi = 3.14159265358979323846;
    k[0] = (REAL)(0.5 * sqrt(1.0 / pi));          /* Y00 */
    k[1] = (REAL)(sqrt(3.0 / (4.0 * pi)));        /* l = 1 */
    k[2] = (REAL)(0.5 * sqrt(15.0 / pi));         /* l = 2, m = +-2 (xy), +-1 */
    k[3] = (REAL)(0.25 * sqrt(5.0 / pi));         /* l = 2, m = 0 */
    k[4] = (REAL)(0.25 * sqrt(15.0 / pi));        /* l = 2, m = 2 (xx - yy) */
    k[5] = (REAL)(0.25 * sqrt(35.0 / (2.0 * pi)));/* l = 3, m = +-3 */
    k[6] = (REAL)(0.5 * sqrt(105.0 / pi));        /* l = 3, m = -2 */
    k[7] = (REAL)(0.25 * sqrt(21.0 / (2.0 * pi)));/* l = 3, m = +-1 */
    k[8] = (REAL)(0.25 * sqrt(7.0 / pi));         /* l = 3, m = 0 */
    k[9] = (REAL)(0.25 * sqrt(105.0 / pi));       /* l = 3, m = 2 */
}

/* Y[0..15] at direction (x, y, z); dY[k][3] its partial derivatives in x, y, z. */
static void sh_basis(REAL x, REAL y, REAL z, int deg, REAL* Y, REAL (*dY)[3])
{
    REAL k[10];
    sh_consts(k);
    REAL xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    Y[0] = k[0];
    if (dY) { dY[0][0] = dY[0][1] = dY[0][2] = 0; }
    if (deg < 1) return;
    Y[1] = -k[1] * y;
    Y[2] = k[1] * z;
    Y[3] = -k[1] * x;
    if (dY) {
        for (int i = 1; i < 4; i++) dY[i][0] = dY[i][1] = dY[i][2] = 0;
        dY[1][1] = -k[1]; dY[2][2] = k[1]; dY[3][0] = -k[1];
    }
    if (deg < 2) return;
    Y[4] = k[2] * xy;
    Y[5] = -k[2] * yz;
    Y[6] = k[3] * ((2 * zz - xx) - yy);
    Y[7] = -k[2] * xz;
    Y[8] = k[4] * (xx - yy);
    if (dY) {
        dY[4][0] = k[2] * y;  dY[4][1] = k[2] * x;  dY[4][2] = 0;
        dY[5][0] = 0;         dY[5][1] = -k[2] * z; dY[5][2] = -k[2] * y;
        dY[6][0] = k[3] * (-2 * x); dY[6][1] = k[3] * (-2 * y); dY[6][2] = k[3] * (4 * z);
        dY[7][0] = -k[2] * z; dY[7][1] = 0;         dY[7][2] = -k[2] * x;
        dY[8][0] = k[4] * (2 * x); dY[8][1] = k[4] * (-2 * y); dY[8][2] = 0;
    }
    if (deg < 3) return;
    Y[9] = (-k[5] * y) * (3 * xx - yy);
    Y[10] = k[6] * (xy * z);
    Y[11] = (-k[7] * y) * ((4 * zz - xx) - yy);
    Y[12] = (k[8] * z) * ((2 * zz - 3 * xx) - 3 * yy);
    Y[13] = (-k[7] * x) * ((4 * zz - xx) - yy);
    Y[14] = (k[9] * z) * (xx - yy);
    Y[15] = (-k[5] * x) * (xx - 3 * yy);
    if (dY) {
        dY[9][0] = -k[5] * (6 * xy);           dY[9][1] = -k[5] * (3 * xx - 3 * yy);  dY[9][2] = 0;
        dY[10][0] = k[6] * yz;                 dY[10][1] = k[6] * xz;                 dY[10][2] = k[6] * xy;
        dY[11][0] = -k[7] * (-2 * xy);         dY[11][1] = -k[7] * ((4 * zz - xx) - 3 * yy);
        dY[11][2] = -k[7] * (8 * yz);
        dY[12][0] = k[8] * (-6 * xz);          dY[12][1] = k[8] * (-6 * yz);
        dY[12][2] = k[8] * ((6 * zz - 3 * xx) - 3 * yy);
        dY[13][0] = -k[7] * ((4 * zz - 3 * xx) - yy);  dY[13][1] = -k[7] * (-2 * xy);
        dY[13][2] = -k[7] * (8 * xz);
        dY[14][0] = k[9] * (2 * xz);           dY[14][1] = k[9] * (-2 * yz);          dY[14][2] = k[9] * (xx - yy);
        dY[15][0] = -k[5] * (3 * xx - 3 * yy); dY[15][1] = -k[5] * (-6 * xy);         dY[15][2] = 0;
    }
}

void orc_sh_basis(int64_t n, const REAL* dirs, int32_t deg, REAL* out /*[n][16]*/, REAL* dout /*[n][16][3] or NULL*/)
{
    for (int64_t i = 0; i < n; i++) {
        REAL Y[16] = {0}, dY[16][3] = {{0}};
        sh_basis(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], deg, Y, dY);
        for (int k = 0; k < 16; k++) {
            out[16 * i + k] = Y[k];
            if (dout)
                for (int a = 0; a < 3; a++) dout[(16 * i + k) * 3 + a] = dY[k][a];
        }
    }
}

/* View-dependent colour c_k from the SH features f_k in R^{3x16} (Sec. 3.1):
 * raw = sum_k Y_k(dir) f_k + 0.5, clamped at 0 per channel.  Returns clamp bits. */
static int colour(const REAL mean[3], const REAL* campos, const REAL* sh, int64_t i, int deg,
                  REAL rgb[3], REAL dirv[3], REAL* len_out, REAL raw[3])
{
    REAL d0 = mean[0] - campos[0], d1 = mean[1] - campos[1], d2 = mean[2] - campos[2];
    REAL len = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
    dirv[0] = d0 / len; dirv[1] = d1 / len; dirv[2] = d2 / len;
    if (len_out) *len_out = len;
    REAL Y[16];
    sh_basis(dirv[0], dirv[1], dirv[2], deg, Y, NULL);
    int nc = (deg + 1) * (deg + 1);
    int clamp = 0;
    for (int ch = 0; ch < 3; ch++) {
        REAL acc = Y[0] * sh[(i * nc + 0) * 3 + ch];
        for (int k = 1; k < nc; k++) acc = acc + Y[k] * sh[(i * nc + k) * 3 + ch];
        acc = acc + (REAL)0.5;
        raw[ch] = acc;
        if (acc < 0) { rgb[ch] = 0; clamp |= (F_CLAMP_R << ch); }
        else rgb[ch] = acc;
    }
    return clamp;
}

/* ------------------------------------------------------------------------------------- */
/* Projection of every Gaussian (Eq. 1's proj) plus the tile rect of step 7.               */
/* Returns the number of (tile, Gaussian) entries, i.e. the sum of tiles_touched.          */
/* ------------------------------------------------------------------------------------- */
int64_t orc_project(int64_t n, const REAL* mean_opac, const REAL* scale, const REAL* quat, const REAL* sh,
                    int32_t sh_degree, const orc_camera* cam, const orc_config* cfg,
                    float* depth, int32_t* radius, int32_t* rect, int64_t* tiles_touched,
                    REAL* xy, REAL* cov2d, REAL* conic, REAL* rgb, int32_t* flags)
{
    camt_f cf; camt_r cr;
    make_cam_f(cam, cfg->near_z, &cf);
    make_cam_r(cam, cfg->near_z, &cr);
    const int B = cfg->tile;
    int64_t total = 0;
    for (int64_t i = 0; i < n; i++) {
        int fl = 0;
        /* key path in FP32 */
        float mf[3] = {(float)mean_opac[4 * i], (float)mean_opac[4 * i + 1], (float)mean_opac[4 * i + 2]};
        float sf[3] = {(float)scale[4 * i], (float)scale[4 * i + 1], (float)scale[4 * i + 2]};
        float qf[4] = {(float)quat[4 * i], (float)quat[4 * i + 1], (float)quat[4 * i + 2], (float)quat[4 * i + 3]};
        proj_f pf;
        int cul = project_one_f(mf, sf, qf, &cf, &pf);
        depth[i] = pf.tz;
        radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        tiles_touched[i] = 0;
        for (int a = 0; a < 2; a++) xy[2 * i + a] = 0;
        for (int a = 0; a < 3; a++) { cov2d[3 * i + a] = 0; conic[3 * i + a] = 0; rgb[3 * i + a] = 0; }
        if (cul == 1) fl |= F_CULL_NEAR;
        if (cul == 2) fl |= F_CULL_DET;
        if (cul) { flags[i] = fl; continue; }
        if (pf.clampx) fl |= F_CLAMP_X;
        if (pf.clampy) fl |= F_CLAMP_Y;
        /* 6-7. radius r = ceil(3 sqrt(lambda_max)); pixel centres with |i-u| <= r, |j-v| <= r */
        float r = ceil(3.0f * sqrt(pf.lam1));
        radius[i] = (int32_t)r;
        float W1 = (float)(cam->width - 1), H1 = (float)(cam->height - 1);
        float x0 = ceil(pf.u - r), x1 = floor(pf.u + r);
        float y0 = ceil(pf.v - r), y1 = floor(pf.v + r);
        if (x0 < 0.0f) x0 = 0.0f;
        if (y0 < 0.0f) y0 = 0.0f;
        if (x1 > W1) x1 = W1;
        if (y1 > H1) y1 = H1;
        if (x0 <= x1 && y0 <= y1) {
            int32_t tx0 = (int32_t)x0 / B, tx1 = (int32_t)x1 / B + 1;
            int32_t ty0 = (int32_t)y0 / B, ty1 = (int32_t)y1 / B + 1;
            rect[4 * i] = tx0; rect[4 * i + 1] = ty0; rect[4 * i + 2] = tx1; rect[4 * i + 3] = ty1;
            tiles_touched[i] = (int64_t)(tx1 - tx0) * (ty1 - ty0);
        }
        total += tiles_touched[i];
        /* values in REAL */
        REAL mr[3] = {mean_opac[4 * i], mean_opac[4 * i + 1], mean_opac[4 * i + 2]};
        REAL sr[3] = {scale[4 * i], scale[4 * i + 1], scale[4 * i + 2]};
        REAL qr[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
        proj_r pr;
        project_one_r(mr, sr, qr, &cr, &pr);
        xy[2 * i] = pr.u; xy[2 * i + 1] = pr.v;
        cov2d[3 * i] = pr.A; cov2d[3 * i + 1] = pr.B; cov2d[3 * i + 2] = pr.C;
        for (int a = 0; a < 3; a++) conic[3 * i + a] = pr.conic[a];
        REAL dirv[3], raw[3];
        fl |= colour(mr, cr.campos, sh, i, sh_degree, &rgb[3 * i], dirv, NULL, raw);
        flags[i] = fl;
    }
    return total;
}

/* ------------------------------------------------------------------------------------- */
/* Duplication into (tile | depth bits, index) pairs, in index order and row-major tile   */
/* order inside each rect.  Returns the count, or -1 if cap is exceeded.                   */
/* ------------------------------------------------------------------------------------- */
int64_t orc_emit_keys(int64_t n, const float* depth, const int32_t* rect, const int64_t* tiles_touched,
                      int32_t tiles_x, uint64_t* keys, uint32_t* vals, int64_t cap)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        if (tiles_touched[i] == 0) continue;
        uint32_t dbits;
        memcpy(&dbits, &depth[i], 4);
        for (int32_t ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ty++)
            for (int32_t tx = rect[4 * i]; tx < rect[4 * i + 2]; tx++) {
                if (k >= cap) return -1;
                uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                keys[k] = (tile << 32) | dbits;
                vals[k] = (uint32_t)i;
                k++;
            }
    }
    return k;
}

typedef struct { uint64_t key; uint32_t val; } kv_t;
static int kv_cmp(const void* a, const void* b)
{
    const kv_t* x = (const kv_t*)a; const kv_t* y = (const kv_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

/* Total order on (tile, depth bits, index): "sorted in depth order" per tile, ties by index. */
void orc_sort_pairs(int64_t k, uint64_t* keys, uint32_t* vals)
{
    kv_t* t = (kv_t*)malloc(sizeof(kv_t) * (size_t)(k > 0 ? k : 1));
    for (int64_t i = 0; i < k; i++) { t[i].key = keys[i]; t[i].val = vals[i]; }
    qsort(t, (size_t)k, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < k; i++) { keys[i] = t[i].key; vals[i] = t[i].val; }
    free(t);
}

/* [start, end) per tile of the sorted list; (0, 0) for a tile with no entries. */
void orc_tile_ranges(int64_t k, const uint64_t* keys, int32_t n_tiles, int64_t* ranges)
{
    for (int32_t t = 0; t < n_tiles; t++) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t i = 0; i < k; i++) {
        int64_t t = (int64_t)(keys[i] >> 32);
        if (t < 0 || t >= n_tiles) continue;
        if (i == 0 || (int64_t)(keys[i - 1] >> 32) != t) ranges[2 * t] = i;
        ranges[2 * t + 1] = i + 1;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Compositing, Eq. 1, one pixel at a time over its tile's sorted list.                    */
/* ------------------------------------------------------------------------------------- */
/* Decision margins for the parity comparison (not part of Eq. 1).  Another FP32 evaluation of
 * the same pair -- the power assembled in a different rounding order (from per-entry factors
 * pre-scaled by log2 e), the falloff by a hardware base-2 exponential, the transmittance by one
 * fused multiply-add -- agrees with this one only up to bounded rounding, so a pixel whose
 * discrete decisions (the sign test, the 1/255 skip, the 1e-4 stop) lie within twice these
 * bounds of their thresholds may legitimately take the other branch: it is flagged ambiguous.
 *   power:  |d power| <= AMB_POW_U * u * S, S = |A'dx^2/2| + |B'dx dy| + |C'dy^2/2|, u = 2^-24:
 *           here each term takes two product roundings, the sums and the final difference
 *           one each (at most 4u S); the other order takes at most three and a half per term
 *           (the factor's scaling by log2 e, its two products, half a unit for log2 e itself)
 *           and two fused sums (at most 5.5u S);
 *   alpha:  |d(o exp(power))| / (o exp(power)) <= |d power| + AMB_EXP2_REL + 4u (the
 *           exponential's relative error and the roundings of the exponential and the opacity
 *           product on either side);
 *   T:      relative error of the transmittance after k blends <= sum over blends of
 *           alpha e_alpha / (1 - alpha) + 3u (a relative error e_alpha of alpha is amplified by
 *           alpha / (1 - alpha) in 1 - alpha; the product rounds once or twice); a clamped
 *           alpha (o exp(power) above 0.99 by more than its margin) is exactly 0.99. */
#define AMB_U 5.9604644775390625e-8      /* 2^-24 */
#define AMB_POW_U 10.0
#define AMB_EXP2_REL 4.76837158203125e-7 /* 2^-21: bound assumed for the device's ex2.approx */

typedef struct {
    REAL alpha, G, T;        /* per blended entry: alpha, exp(power), transmittance before it */
    int clamped;             /* o exp(power) > 0.99 */
    int64_t g;               /* Gaussian index */
    REAL dx, dy;
} contrib_t;

/* Walk one pixel's list.  Fills the blended contributors (if out != NULL) and returns their
 * count; *stop_pos = list position one past the last blended entry (n_contrib),
 * *visited = entries evaluated (up to and including the stopping one). */
static int64_t pixel_walk(const int64_t* list, int64_t len, REAL px, REAL py, const REAL* xy, const REAL* conic,
                          const REAL* mean_opac, const REAL* rgb, REAL C[3], REAL* Tout, int64_t* stop_pos,
                          int64_t* visited, int* amb, uint64_t* hash, contrib_t* out)
{
    const REAL thr = (REAL)1 / (REAL)255;
    const REAL tmin = (REAL)0.0001;
    REAL Tr = 1;
    double eT = 0.0; /* relative error bound of Tr (decision margins only) */
    C[0] = C[1] = C[2] = 0;
    int64_t nb = 0, last = 0, vis = 0;
    for (int64_t p = 0; p < len; p++) {
        int64_t g = list[p];
        vis = p + 1;
        REAL dx = xy[2 * g] - px, dy = xy[2 * g + 1] - py;
        REAL a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
        REAL power = (REAL)-0.5 * ((a * dx) * dx + (c * dy) * dy) - (b * dx) * dy;
        double epow = 0.0, ea = 0.0;
        if (amb) {
            double ddx = (double)dx, ddy = (double)dy;
            epow = AMB_POW_U * AMB_U *
                   (fabs(0.5 * (double)a * ddx * ddx) + fabs((double)b * ddx * ddy) + fabs(0.5 * (double)c * ddy * ddy));
            ea = epow + AMB_EXP2_REL + 4.0 * AMB_U;
            if (fabs((double)power) <= 2.0 * epow) *amb = 1;
        }
        if (power > 0) { if (hash) *hash = fnv(*hash, 1); continue; }
        REAL o = mean_opac[4 * g + 3];
        /* G = exp(power) correctly rounded to REAL: the FP64 exponential, rounded once (in the
         * FP32 build its result is the nearest float to e^power except where e^power lies
         * within an FP64 rounding error of a float rounding boundary) */
        REAL G = (REAL)exp((double)power);
        REAL og = o * G;
        if (amb && fabs((double)og - 1.0 / 255.0) <= 2.0 * ea * (double)og) *amb = 1;
        REAL alpha = og < (REAL)0.99 ? og : (REAL)0.99;
        if (alpha < thr) { if (hash) *hash = fnv(*hash, 2); continue; }
        REAL Tn = Tr * ((REAL)1 - alpha);
        double eTn = 0.0;
        if (amb) {
            const double ealpha = (double)og * (1.0 - 2.0 * ea) > 0.99 ? 0.0 : ea;
            eTn = eT + (double)alpha * ealpha / (1.0 - (double)alpha) + 3.0 * AMB_U;
            if (fabs((double)Tn - 1e-4) <= 2.0 * eTn * (double)Tn) *amb = 1;
        }
        if (Tn < tmin) { if (hash) *hash = fnv(*hash, 3); break; }
        eT = eTn;
        if (hash) *hash = fnv(*hash, og > (REAL)0.99 ? 5 : 4);
        if (out) {
            out[nb].alpha = alpha; out[nb].G = G; out[nb].T = Tr; out[nb].clamped = og > (REAL)0.99;
            out[nb].g = g; out[nb].dx = dx; out[nb].dy = dy;
        }
        REAL w = alpha * Tr;
        for (int ch = 0; ch < 3; ch++) C[ch] = C[ch] + rgb[3 * g + ch] * w;
        Tr = Tn;
        last = p + 1;
        nb++;
    }
    *Tout = Tr;
    *stop_pos = last;
    *visited = vis;
    return nb;
}

/* Renders every pixel of every tile whose tile_mask entry is non-zero (all when NULL).
 * vals[] hold Gaussian indices in sorted order; ranges[] the per-tile [start, end).
 * Outputs image [3][H][W], final_T [H][W], n_contrib [H][W], n_visited [H][W],
 * ambiguous [H][W] (a skip/stop decision within the margins above) and a hash of every
 * decision taken.  Returns the number of evaluated pairs. */
int64_t orc_composite(int64_t n, const REAL* xy, const REAL* conic, const REAL* mean_opac, const REAL* rgb,
                      const uint32_t* vals, const int64_t* ranges, int32_t W, int32_t H, const orc_config* cfg,
                      const uint8_t* tile_mask, REAL* image, REAL* final_T, int32_t* n_contrib,
                      int32_t* n_visited, uint8_t* ambiguous, uint64_t* hash_out)
{
    (void)n;
    const int B = cfg->tile;
    const int tiles_x = (W + B - 1) / B, tiles_y = (H + B - 1) / B;
    int64_t pairs = 0;
    uint64_t hash = 1469598103934665603ull;
    int64_t cap = 0;
    for (int t = 0; t < tiles_x * tiles_y; t++) {
        int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > cap) cap = len;
    }
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    for (int ty = 0; ty < tiles_y; ty++)
        for (int tx = 0; tx < tiles_x; tx++) {
            int t = ty * tiles_x + tx;
            if (tile_mask && !tile_mask[t]) continue;
            int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
            for (int64_t p = s; p < e; p++) list[p - s] = vals[p];
            for (int j = ty * B; j < (ty + 1) * B && j < H; j++)
                for (int i = tx * B; i < (tx + 1) * B && i < W; i++) {
                    REAL C[3], Tr;
                    int64_t stop, vis;
                    int amb = 0;
                    pixel_walk(list, e - s, (REAL)i, (REAL)j, xy, conic, mean_opac, rgb, C, &Tr, &stop, &vis,
                               &amb, &hash, NULL);
                    int64_t pix = (int64_t)j * W + i;
                    for (int ch = 0; ch < 3; ch++) image[(int64_t)ch * H * W + pix] = C[ch] + Tr * (REAL)cfg->bg[ch];
                    final_T[pix] = Tr;
                    n_contrib[pix] = (int32_t)stop;
                    if (n_visited) n_visited[pix] = (int32_t)vis;
                    if (ambiguous) ambiguous[pix] = (uint8_t)amb;
                    pairs += vis;
                }
        }
    free(list);
    if (hash_out) *hash_out = hash;
    return pairs;
}

/* Brute force: every pixel over ALL non-culled Gaussians sorted by (depth, index), with no
 * binning.  Equal to orc_composite when every opacity < 1/(255 e^-4.5). */
typedef struct { float d; int64_t i; } di_t;
static int di_cmp(const void* a, const void* b)
{
    const di_t* x = (const di_t*)a; const di_t* y = (const di_t*)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return x->i < y->i ? -1 : (x->i > y->i);
}
void orc_composite_brute(int64_t n, const REAL* xy, const REAL* conic, const REAL* mean_opac, const REAL* rgb,
                         const float* depth, const int32_t* flags, int32_t W, int32_t H, const orc_config* cfg,
                         REAL* image, REAL* final_T)
{
    di_t* ord = (di_t*)malloc(sizeof(di_t) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (!(flags[i] & (F_CULL_NEAR | F_CULL_DET))) { ord[m].d = depth[i]; ord[m].i = i; m++; }
    qsort(ord, (size_t)m, sizeof(di_t), di_cmp);
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t k = 0; k < m; k++) list[k] = ord[k].i;
    for (int j = 0; j < H; j++)
        for (int i = 0; i < W; i++) {
            REAL C[3], Tr;
            int64_t stop, vis;
            pixel_walk(list, m, (REAL)i, (REAL)j, xy, conic, mean_opac, rgb, C, &Tr, &stop, &vis, NULL, NULL, NULL);
            int64_t pix = (int64_t)j * W + i;
            for (int ch = 0; ch < 3; ch++) image[(int64_t)ch * H * W + pix] = C[ch] + Tr * (REAL)cfg->bg[ch];
            final_T[pix] = Tr;
        }
    free(list);
    free(ord);
}

/* ------------------------------------------------------------------------------------- */
/* Backward of compositing: dL/d(u, v), dL/d(conic), dL/d(opacity), dL/d(rgb) per Gaussian. */
/* For pixel value P = sum_i alpha_i T_i c_i + T_end bg:                                    */
/*   dP/dc_i = alpha_i T_i,  dP/dalpha_i = T_i c_i - S_i / (1 - alpha_i),                  */
/*   S_i = sum_{m > i} alpha_m T_m c_m + T_end bg.                                          */
/* ------------------------------------------------------------------------------------- */
void orc_composite_backward(int64_t n, const REAL* xy, const REAL* conic, const REAL* mean_opac, const REAL* rgb,
                            const uint32_t* vals, const int64_t* ranges, int32_t W, int32_t H, const orc_config* cfg,
                            const uint8_t* tile_mask, const REAL* dL_dimage, REAL* g_xy, REAL* g_conic,
                            REAL* g_opac, REAL* g_rgb)
{
    const int B = cfg->tile;
    const int tiles_x = (W + B - 1) / B, tiles_y = (H + B - 1) / B;
    for (int64_t i = 0; i < 2 * n; i++) g_xy[i] = 0;
    for (int64_t i = 0; i < 3 * n; i++) { g_conic[i] = 0; g_rgb[i] = 0; }
    for (int64_t i = 0; i < n; i++) g_opac[i] = 0;
    int64_t cap = 0;
    for (int t = 0; t < tiles_x * tiles_y; t++) {
        int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > cap) cap = len;
    }
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
    contrib_t* cb = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)(cap > 0 ? cap : 1));
    for (int ty = 0; ty < tiles_y; ty++)
        for (int tx = 0; tx < tiles_x; tx++) {
            int t = ty * tiles_x + tx;
            if (tile_mask && !tile_mask[t]) continue;
            int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
            for (int64_t p = s; p < e; p++) list[p - s] = vals[p];
            for (int j = ty * B; j < (ty + 1) * B && j < H; j++)
                for (int i = tx * B; i < (tx + 1) * B && i < W; i++) {
                    REAL C[3], Tend;
                    int64_t stop, vis;
                    int64_t m = pixel_walk(list, e - s, (REAL)i, (REAL)j, xy, conic, mean_opac, rgb, C, &Tend,
                                           &stop, &vis, NULL, NULL, cb);
                    int64_t pix = (int64_t)j * W + i;
                    REAL gp[3];
                    for (int ch = 0; ch < 3; ch++) gp[ch] = dL_dimage[(int64_t)ch * H * W + pix];
                    REAL S[3];
                    for (int ch = 0; ch < 3; ch++) S[ch] = Tend * (REAL)cfg->bg[ch];
                    for (int64_t q = m - 1; q >= 0; q--) {
                        const contrib_t* c = &cb[q];
                        int64_t g = c->g;
                        REAL dalpha = 0;
                        for (int ch = 0; ch < 3; ch++) {
                            REAL cc = rgb[3 * g + ch];
                            g_rgb[3 * g + ch] += gp[ch] * c->alpha * c->T;
                            dalpha += gp[ch] * (c->T * cc - S[ch] / ((REAL)1 - c->alpha));
                        }
                        for (int ch = 0; ch < 3; ch++) S[ch] += c->alpha * c->T * rgb[3 * g + ch];
                        if (c->clamped) continue;
                        REAL o = mean_opac[4 * g + 3];
                        g_opac[g] += dalpha * c->G;
                        REAL dpow = dalpha * o * c->G;
                        REAL a = conic[3 * g], b = conic[3 * g + 1], cc = conic[3 * g + 2];
                        REAL dx = c->dx, dy = c->dy;
                        g_conic[3 * g] += dpow * (REAL)-0.5 * dx * dx;
                        g_conic[3 * g + 1] += dpow * -(dx * dy);
                        g_conic[3 * g + 2] += dpow * (REAL)-0.5 * dy * dy;
                        g_xy[2 * g] += dpow * -(a * dx + b * dy);
                        g_xy[2 * g + 1] += dpow * -(cc * dy + b * dx);
                    }
                }
        }
    free(cb);
    free(list);
}

/* ------------------------------------------------------------------------------------- */
/* Backward of the projection and colour: chains the 2D gradients to the mean, scale,      */
/* quaternion (through its normalisation), opacity and SH coefficients.  Gradients are     */
/* ADDED into the outputs.  Discrete decisions (culls, guard-band clamp, colour clamp)     */
/* pass no gradient.                                                                       */
/* ------------------------------------------------------------------------------------- */
void orc_project_backward(int64_t n, const REAL* mean_opac, const REAL* scale, const REAL* quat, const REAL* sh,
                          int32_t sh_degree, const orc_camera* cam, const orc_config* cfg, const int64_t* tiles_touched,
                          const REAL* g_xy, const REAL* g_conic, const REAL* g_opac_in, const REAL* g_rgb,
                          REAL* g_mean, REAL* g_scale, REAL* g_quat, REAL* g_opac, REAL* g_sh)
{
    camt_r cr;
    make_cam_r(cam, cfg->near_z, &cr);
    const REAL* W = cr.R;
    int nc = (sh_degree + 1) * (sh_degree + 1);
    for (int64_t i = 0; i < n; i++) {
        if (tiles_touched[i] == 0) continue;
        REAL mr[3] = {mean_opac[4 * i], mean_opac[4 * i + 1], mean_opac[4 * i + 2]};
        REAL sr[3] = {scale[4 * i], scale[4 * i + 1], scale[4 * i + 2]};
        REAL qr[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
        proj_r p;
        project_one_r(mr, sr, qr, &cr, &p);
        g_opac[i] += g_opac_in[i];

        /* colour -> SH coefficients and view direction */
        REAL rgbv[3], dirv[3], raw[3], len;
        int cl = colour(mr, cr.campos, sh, i, sh_degree, rgbv, dirv, &len, raw);
        REAL Y[16], dY[16][3];
        sh_basis(dirv[0], dirv[1], dirv[2], sh_degree, Y, dY);
        REAL gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ch++) {
            if (cl & (F_CLAMP_R << ch)) continue;
            REAL gc = g_rgb[3 * i + ch];
            for (int k = 0; k < nc; k++) {
                g_sh[(i * nc + k) * 3 + ch] += Y[k] * gc;
                for (int a = 0; a < 3; a++) gdir[a] += gc * sh[(i * nc + k) * 3 + ch] * dY[k][a];
            }
        }
        REAL dd = (dirv[0] * gdir[0] + dirv[1] * gdir[1]) + dirv[2] * gdir[2];
        REAL gm[3];
        for (int a = 0; a < 3; a++) gm[a] = (gdir[a] - dirv[a] * dd) / len;

        /* conic (C/D, -B/D, A/D), D = AC - B^2 -> Sigma2D entries (A, B, C).  The partials are
         * written over the common denominator D^2 (1/D - AC/D^2 = -B^2/D^2), which avoids the
         * cancellation of the unsimplified form. */
        REAL A = p.A, Bv = p.B, C = p.C, D2 = p.det * p.det;
        REAL ga_ = g_conic[3 * i], gb_ = g_conic[3 * i + 1], gc_ = g_conic[3 * i + 2];
        REAL dA = (-ga_ * C * C + gb_ * Bv * C - gc_ * Bv * Bv) / D2;
        REAL dB = (2 * ga_ * Bv * C - gb_ * (A * C + Bv * Bv) + 2 * gc_ * A * Bv) / D2;
        REAL dC = (-ga_ * Bv * Bv + gb_ * A * Bv - gc_ * A * A) / D2;

        /* Sigma2D = T S T^T:  dL/dS_ij and dL/dT */
        const REAL* Tm = p.Tm;
        const REAL* S = p.S3;
        REAL gS[9];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                gS[a * 3 + b] = dA * Tm[a] * Tm[b] + dB * Tm[a] * Tm[3 + b] + dC * Tm[3 + a] * Tm[3 + b];
        REAL ST0[3], ST1[3];
        for (int a = 0; a < 3; a++) {
            ST0[a] = S[a * 3 + 0] * Tm[0] + S[a * 3 + 1] * Tm[1] + S[a * 3 + 2] * Tm[2];
            ST1[a] = S[a * 3 + 0] * Tm[3] + S[a * 3 + 1] * Tm[4] + S[a * 3 + 2] * Tm[5];
        }
        REAL gT[6];
        for (int a = 0; a < 3; a++) {
            gT[a] = 2 * dA * ST0[a] + dB * ST1[a];
            gT[3 + a] = 2 * dC * ST1[a] + dB * ST0[a];
        }
        /* T = J W */
        REAL gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
        for (int a = 0; a < 3; a++) {
            gJ00 += gT[a] * W[0 * 3 + a];
            gJ02 += gT[a] * W[2 * 3 + a];
            gJ11 += gT[3 + a] * W[1 * 3 + a];
            gJ12 += gT[3 + a] * W[2 * 3 + a];
        }
        /* J and the screen mean -> camera-space mean */
        REAL fx = cr.fx, fy = cr.fy, tx = p.tx, ty = p.ty, tz = p.tz;
        REAL tz2 = tz * tz, tz3 = tz2 * tz;
        REAL gtx = 0, gty = 0, gtz = 0;
        gtz += gJ00 * (-fx / tz2);
        gtz += gJ11 * (-fy / tz2);
        if (!p.clampx) { gtx += gJ02 * (-fx / tz2); gtz += gJ02 * (2 * fx * tx / tz3); }
        else { REAL lim = tx / tz > 0 ? p.limx : -p.limx; gtz += gJ02 * (fx * lim / tz2); }
        if (!p.clampy) { gty += gJ12 * (-fy / tz2); gtz += gJ12 * (2 * fy * ty / tz3); }
        else { REAL lim = ty / tz > 0 ? p.limy : -p.limy; gtz += gJ12 * (fy * lim / tz2); }
        REAL gu = g_xy[2 * i], gv = g_xy[2 * i + 1];
        gtx += gu * fx / tz;
        gtz += gu * (-fx * tx / tz2);
        gty += gv * fy / tz;
        gtz += gv * (-fy * ty / tz2);
        for (int a = 0; a < 3; a++) gm[a] += W[0 * 3 + a] * gtx + W[1 * 3 + a] * gty + W[2 * 3 + a] * gtz;
        for (int a = 0; a < 3; a++) g_mean[3 * i + a] += gm[a];

        /* Sigma3D = M M^T, M = Rq diag(s) */
        REAL gM[9];
        for (int a = 0; a < 3; a++)
            for (int k = 0; k < 3; k++) {
                REAL acc = 0;
                for (int b = 0; b < 3; b++) acc += (gS[a * 3 + b] + gS[b * 3 + a]) * p.M[b * 3 + k];
                gM[a * 3 + k] = acc;
            }
        REAL gR[9];
        for (int k = 0; k < 3; k++) {
            REAL acc = 0;
            for (int a = 0; a < 3; a++) acc += gM[a * 3 + k] * p.Rq[a * 3 + k];
            g_scale[3 * i + k] += acc;
            for (int a = 0; a < 3; a++) gR[a * 3 + k] = gM[a * 3 + k] * sr[k];
        }
        REAL w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
        REAL gq[4];
        gq[0] = 2 * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
        gq[1] = 2 * (y * gR[1] + z * gR[2] + y * gR[3] - 2 * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2 * x * gR[8]);
        gq[2] = 2 * (-2 * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2 * y * gR[8]);
        gq[3] = 2 * (-2 * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2 * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
        REAL qd = w * gq[0] + x * gq[1] + y * gq[2] + z * gq[3];
        for (int a = 0; a < 4; a++) g_quat[4 * i + a] += (gq[a] - p.qn[a] * qd) / p.qlen;
    }
}

/* L1 loss (Sec. 3.2.3, the L1 part): mean |img - target| and its gradient sign(.)/count. */
void orc_l1(int64_t count, const REAL* img, const REAL* target, REAL* grad, double* loss)
{
    double acc = 0;
    for (int64_t i = 0; i < count; i++) {
        REAL d = img[i] - target[i];
        acc += fabs((double)d);
        grad[i] = d > 0 ? (REAL)1 / (REAL)count : (d < 0 ? (REAL)-1 / (REAL)count : 0);
    }
    *loss = acc / (double)count;
}

/* ------------------------------------------------------------------------------------- */
/* Block bounds by median absolute deviation, Eq. 7, per axis, in FP64; stored rounded    */
/* outward to FP32.  Median of an even count = mean of the two middle values.             */
/* ------------------------------------------------------------------------------------- */
static int dcmp(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y);
}
static double median_sorted(const double* v, int64_t m)
{
    if (m % 2) return v[m / 2];
    return (v[m / 2 - 1] + v[m / 2]) * 0.5;
}
static float round_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}
static float round_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}
void orc_block_bounds(int32_t n_blocks, int32_t n_levels, const int64_t* level_offset, const int64_t* level_count,
                      const float* mean_opac, double n_mad, float* aabb)
{
    for (int32_t b = 0; b < n_blocks; b++) {
        int64_t off = level_offset[(int64_t)b * n_levels], m = level_count[(int64_t)b * n_levels];
        if (m <= 0) { for (int a = 0; a < 6; a++) aabb[6 * b + a] = 0; continue; }
        double* v = (double*)malloc(sizeof(double) * (size_t)m);
        for (int ax = 0; ax < 3; ax++) {
            for (int64_t k = 0; k < m; k++) v[k] = (double)mean_opac[4 * (off + k) + ax];
            qsort(v, (size_t)m, sizeof(double), dcmp);
            double mn = v[0], mx = v[m - 1];
            double med = median_sorted(v, m);
            for (int64_t k = 0; k < m; k++) v[k] = fabs(v[k] - med);
            qsort(v, (size_t)m, sizeof(double), dcmp);
            double mad = median_sorted(v, m);
            double lo = med - n_mad * mad, hi = med + n_mad * mad;
            if (mn > lo) lo = mn;
            if (mx < hi) hi = mx;
            aabb[6 * b + ax] = round_down(lo);
            aabb[6 * b + 3 + ax] = round_up(hi);
        }
        free(v);
    }
}

/* ------------------------------------------------------------------------------------- */
/* Block-wise LoD selection and frustum culling (Sec. 3.3.2), in FP64.                     */
/* level[b] = -1 (culled or empty), else 0 (finest) .. n_levels - 1.                        */
/* ------------------------------------------------------------------------------------- */
void orc_lod_select(int32_t n_blocks, int32_t n_levels, const int64_t* level_count, const float* aabb,
                    const float* cell, const orc_camera* cam, float near_z, const double* dist, int8_t* level)
{
    double R[9], t[3], cp[3];
    for (int i = 0; i < 9; i++) R[i] = (double)cam->R[i];
    for (int i = 0; i < 3; i++) { t[i] = (double)cam->t[i]; cp[i] = (double)cam->campos[i]; }
    double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    double Wd = cam->width, Hd = cam->height, nz = near_z;
    for (int32_t b = 0; b < n_blocks; b++) {
        if (level_count[(int64_t)b * n_levels] <= 0) { level[b] = -1; continue; }
        const float* bb = &aabb[6 * b];
        int any_front = 0;
        double xmin = 0, xmax = 0, ymin = 0, ymax = 0, dmin = 0;
        for (int c = 0; c < 8; c++) {
            double p[3] = {(double)bb[(c & 1) ? 3 : 0], (double)bb[(c & 2) ? 4 : 1], (double)bb[(c & 4) ? 5 : 2]};
            double d0 = p[0] - cp[0], d1 = p[1] - cp[1], d2 = p[2] - cp[2];
            double dist_c = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
            if (c == 0 || dist_c < dmin) dmin = dist_c;
            double tx = ((R[0] * p[0] + R[1] * p[1]) + R[2] * p[2]) + t[0];
            double ty = ((R[3] * p[0] + R[4] * p[1]) + R[5] * p[2]) + t[1];
            double tz = ((R[6] * p[0] + R[7] * p[1]) + R[8] * p[2]) + t[2];
            if (!(tz > nz)) continue;
            double u = (fx * tx) / tz + cx, v = (fy * ty) / tz + cy;
            if (!any_front) { xmin = xmax = u; ymin = ymax = v; any_front = 1; }
            else {
                if (u < xmin) xmin = u;
                if (u > xmax) xmax = u;
                if (v < ymin) ymin = v;
                if (v > ymax) ymax = v;
            }
        }
        int visible = any_front && xmax > -0.5 && xmin < Wd - 0.5 && ymax > -0.5 && ymin < Hd - 0.5;
        const float* ce = &cell[4 * b];
        int inside = cp[0] >= (double)ce[0] && cp[0] < (double)ce[1] && cp[1] >= (double)ce[2] && cp[1] < (double)ce[3];
        if (!visible && !inside) { level[b] = -1; continue; }
        int lv = dmin < dist[0] ? 0 : (dmin < dist[1] ? 1 : 2);
        if (lv > n_levels - 1) lv = n_levels - 1;
        level[b] = (int8_t)lv;
    }
}

/* Fusion by concatenation (Sec. 3.2.3, 3.3.2): the global indices of the selected
 * (block, level) segments in block order.  Returns the count. */
int64_t orc_concat(int32_t n_blocks, int32_t n_levels, const int64_t* level_offset, const int64_t* level_count,
                   const int8_t* level, int64_t* out_idx)
{
    int64_t m = 0;
    for (int32_t b = 0; b < n_blocks; b++) {
        if (level[b] < 0) continue;
        int64_t off = level_offset[(int64_t)b * n_levels + level[b]];
        int64_t cnt = level_count[(int64_t)b * n_levels + level[b]];
        for (int64_t k = 0; k < cnt; k++) out_idx[m++] = off + k;
    }
    return m;
}

/* Point-wise level selection, the baseline Sec. 3.3.2 compares against (Table 5): each
 * Gaussian takes the level of its own distance to the camera centre (FP32,
 * dist = sqrt((dx*dx + dy*dy) + dz*dz), level 0 if dist < d1, 1 if < d2, else 2, clamped)
 * and is kept iff its rank in its block's finest level is below that level's count (levels
 * are nested prefixes).  No block culling.  Writes global indices in block order. */
int64_t orc_pointwise_select(int32_t n_blocks, int32_t n_levels, const int64_t* level_offset,
                             const int64_t* level_count, const float* mean_opac, const orc_camera* cam,
                             const double* dist, int64_t* out_idx)
{
    const float d1 = (float)dist[0], d2 = (float)dist[1];
    int64_t m = 0;
    for (int32_t b = 0; b < n_blocks; b++) {
        int64_t off = level_offset[(int64_t)b * n_levels], cnt = level_count[(int64_t)b * n_levels];
        for (int64_t r = 0; r < cnt; r++) {
            int64_t g = off + r;
            float e0 = mean_opac[4 * g] - cam->campos[0];
            float e1 = mean_opac[4 * g + 1] - cam->campos[1];
            float e2 = mean_opac[4 * g + 2] - cam->campos[2];
            float d = sqrtf((e0 * e0 + e1 * e1) + e2 * e2);
            int lv = d < d1 ? 0 : (d < d2 ? 1 : 2);
            if (lv > n_levels - 1) lv = n_levels - 1;
            if (r < level_count[(int64_t)b * n_levels + lv]) out_idx[m++] = g;
        }
    }
    return m;
}

#include "oracle_partition.inc"
#include "oracle_levels.inc"
#include "oracle_ssim.inc"

int32_t orc_real_bytes(void) { return (int32_t)sizeof(REAL); }
