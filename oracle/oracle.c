/*
 * oracle.c -- plain, slow FP64 CPU oracle of the spectral-cube ray caster.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  The product (the CUDA library and its
 * Python binding) never calls it, links it or shares a line of code with it.
 *
 * Everything is computed in double precision from the caller's inputs (the
 * float32 cube, camera and colour map promoted exactly to double), following
 * the paper's definitions in their own order:
 *
 *   ray generation ............ Appendix A (parallel and perspective projection)
 *   ray loop .................. Algorithm 1 (init; for i = 1..N: fetch, filter,
 *                               transferFunction, loc += step; setFragment)
 *   MIP ....................... Eq. 1, Algorithm 2 (MIP_0, ">=": last max wins)
 *   spectral-position colour .. Algorithm 4 (MIP_1: colour from maxloc.z)
 *   alpha compositing ......... Eq. 2, Algorithm 3 (AVIP_0, exit when alpha > 0.99)
 *   average ................... Eq. 3 (zeroth moment: orthographic ray sum)
 *   line ratio ................ Algorithm 14 (Method 2: per-sample ratio, then MIP_0)
 *   in-ray smoothing .......... Algorithm 8 (box along the ray), Algorithm 9 (taps
 *                               along each data axis, chained x, y, z)
 *   Gaussian smoothing ........ Eqs. 5-6 (sampled Gaussian, separable per axis),
 *                               binomial b_n = [1,1]^{*n} and Algorithm 9
 *   adjoint of compositing .... reverse mode over a stored per-sample tape
 *
 * Readings where the paper is silent, ambiguous or garbled (the paper fixes none of
 * these; each is the plainest reading of the passage cited beside the function that
 * takes it): voxel (i,j,k) sits at the point (i,j,k) and the box is
 * [-0.5, n-0.5]^3; samples lie at the mid-points t0 + (k + 1/2) h of a ray
 * clipped to the box, N = floor((t1 - t0) / h); indices clamp to the edge; a NaN
 * sample is replaced by DATAMIN, which is the colour map's domain low `lo`;
 * v_hat = clamp((v - lo)/(hi - lo), 0, 1); the colour map is interpolated
 * linearly between its 256 knots; compositing is written in the premultiplied
 * form C += T a c, T *= (1 - a), alpha = 1 - T (equal to the paper's recurrence).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MIP 0
#define OR_AVG 1
#define OR_COMPOSITE 2
#define OR_SPECTRAL 3
#define OR_RATIO 4
#define OR_MOMENT1 5
#define OR_COMPOSITE_SPECTRAL 6 /* Algorithm 5, AVIP_1: compositing, colour from the sample's spectral position */
#define OR_MIP_RGB 7            /* Algorithm 6: maximum, colour from the maximum's position (r, g, b) = (z, y, x) */
#define OR_COMPOSITE_RGB 8      /* Algorithm 7, AVIP_RGB: compositing, colour from the sample's position */
#define OR_RATIO_MIP 9          /* Algorithms 12-13, line ratio Method 1: maximum of each cube, then their ratio */

#define OR_NEAREST 0
#define OR_TRILINEAR 1

/* fragility bits: a discrete decision of this ray lies within eps of its switch point */
#define FRAG_COUNT 1     /* N = floor(len / h) near an integer                */
#define FRAG_ROUND 2     /* a nearest-sample coordinate near a rounding edge  */
#define FRAG_RATIO 4     /* a ratio denominator near its threshold            */
#define FRAG_EXIT 8      /* accumulated alpha near the early-exit threshold   */
#define FRAG_TIE 16      /* the running maximum is near-tied at another channel */

typedef struct {
    double eye[3], right[3], up[3], fwd[3];
    double tan_half_fovy, ortho_half_h;
    int ortho, W, H;
} ocam;

typedef struct {
    const double *v;
    int n[3]; /* nx, ny, nz */
} ovol;

static ocam make_cam(const double *c14, int ortho, int W, int H)
{
    ocam c;
    for (int a = 0; a < 3; ++a) {
        c.eye[a] = c14[a];
        c.right[a] = c14[3 + a];
        c.up[a] = c14[6 + a];
        c.fwd[a] = c14[9 + a];
    }
    c.tan_half_fovy = c14[12];
    c.ortho_half_h = c14[13];
    c.ortho = ortho;
    c.W = W;
    c.H = H;
    return c;
}

/* Appendix A: pixel (px, py) -> ray origin o and unit direction d.
 * Screen coordinates of the pixel centre: xs = 2(px+1/2)/W - 1, ys = 1 - 2(py+1/2)/H
 * (row 0 at the top).  Parallel: rays share the direction fwd and start on the
 * image plane through the eye.  Perspective: rays leave the eye through the pixel. */
static void pixel_ray(const ocam *c, int px, int py, double o[3], double d[3])
{
    double xs = 2.0 * (px + 0.5) / c->W - 1.0;
    double ys = 1.0 - 2.0 * (py + 0.5) / c->H;
    double aspect = (double)c->W / (double)c->H;
    if (c->ortho) {
        double hw = c->ortho_half_h * aspect, hh = c->ortho_half_h;
        double nf = sqrt(c->fwd[0] * c->fwd[0] + c->fwd[1] * c->fwd[1] + c->fwd[2] * c->fwd[2]);
        for (int a = 0; a < 3; ++a) {
            o[a] = c->eye[a] + xs * hw * c->right[a] + ys * hh * c->up[a];
            d[a] = c->fwd[a] / nf;
        }
    } else {
        double u[3];
        double tx = xs * c->tan_half_fovy * aspect, ty = ys * c->tan_half_fovy;
        for (int a = 0; a < 3; ++a)
            u[a] = c->fwd[a] + tx * c->right[a] + ty * c->up[a];
        double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int a = 0; a < 3; ++a) {
            o[a] = c->eye[a];
            d[a] = u[a] / nu;
        }
    }
}

static double dist_to_int(double x) { return fabs(x - floor(x + 0.5)); }

/* Clip the ray to the closed box [-0.5, n-0.5]^3 (slab method), keep t >= 0, and
 * count the samples N = floor((t1 - t0)/h) of Algorithm 1's loop.  Returns N
 * (0 for a miss) and the start parameter t0. */
static int clip_ray(const int n[3], const double o[3], const double d[3], double h,
                    double *t0_out, double eps, int *frag)
{
    double tmin = -INFINITY, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = -0.5, hi = n[a] - 0.5;
        if (d[a] == 0.0) {
            /* a ray lying on a face of the box: inside or outside is a rounding decision */
            if (frag && eps > 0.0 && (fabs(o[a] - lo) < eps || fabs(o[a] - hi) < eps))
                *frag |= FRAG_COUNT;
            if (o[a] < lo || o[a] > hi)
                return 0;
            continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        double tn = ta < tb ? ta : tb, tf = ta < tb ? tb : ta;
        if (tn > tmin) tmin = tn;
        if (tf < tmax) tmax = tf;
    }
    double t0 = tmin > 0.0 ? tmin : 0.0;
    *t0_out = t0;
    if (!(tmax > t0))
        return 0;
    double q = (tmax - t0) / h;
    /* an exactly integral quotient comes from exactly representable geometry
     * (axis-aligned views), which every implementation evaluates exactly */
    if (frag && eps > 0.0 && dist_to_int(q) < eps && dist_to_int(q) > 0.0 && q >= 0.5)
        *frag |= FRAG_COUNT;
    return (int)floor(q);
}

static inline double vox(const ovol *V, long x, long y, long z)
{
    if (x < 0) x = 0;
    if (y < 0) y = 0;
    if (z < 0) z = 0;
    if (x > V->n[0] - 1) x = V->n[0] - 1;
    if (y > V->n[1] - 1) y = V->n[1] - 1;
    if (z > V->n[2] - 1) z = V->n[2] - 1;
    return V->v[((size_t)z * V->n[1] + (size_t)y) * V->n[0] + (size_t)x];
}

/* Algorithm 1's fetch "val <- cube[loc]": nearest voxel (round half up, clamped). */
static double sample_nearest(const ovol *V, const double p[3], double eps, int *frag)
{
    long i[3];
    for (int a = 0; a < 3; ++a) {
        double q = p[a] + 0.5;
        i[a] = (long)floor(q);
        if (frag && eps > 0.0 && dist_to_int(q) < eps)
            *frag |= FRAG_ROUND;
    }
    return vox(V, i[0], i[1], i[2]);
}

/* Trilinear interpolation, written as its definition: the sum over the 8 corners
 * of the cell holding p of corner value x product of 1-D hat weights. */
static double sample_trilinear(const ovol *V, const double p[3])
{
    long i[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(p[a]);
        i[a] = (long)fl;
        f[a] = p[a] - fl;
    }
    double acc = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
                acc += w * vox(V, i[0] + cx, i[1] + cy, i[2] + cz);
            }
    return acc;
}

/* Colour map lookup (Section 2.1): v_hat in [0,1] -> RGBA, linear between knots. */
static void lut_eval(const double *L, double vhat, double out[4])
{
    double u = 255.0 * vhat;
    long i0 = (long)floor(u);
    if (i0 > 254) i0 = 254;
    if (i0 < 0) i0 = 0;
    double f = u - (double)i0;
    for (int ch = 0; ch < 4; ++ch)
        out[ch] = (1.0 - f) * L[4 * i0 + ch] + f * L[4 * (i0 + 1) + ch];
}

static double normalise(double v, double lo, double hi)
{
    double x = (v - lo) / (hi - lo);
    return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
}

typedef struct {
    int mode, interp;
    double h, lo, hi, s, term_alpha, ratio_floor, eps_pos, eps_val, eps_exit;
    const double *lut;
    int filter;        /* 0 none, 1 intensity clipping (Algorithm 10), 2 domain scaling (Algorithm 11) */
    double tmin, tmax; /* the filters' minimum and maximum thresholds */
    int alpha_thr;     /* spectral / first-moment colouring: alpha 0 up to tmin, 1 above */
    int smooth;        /* 0 none, 1 box along the ray (Algorithm 8), 2 per-axis taps (Algorithm 9) */
    int arm;           /* box: neighbours visited on each side (filterArm) */
    int ntap;          /* taps: fetches on each side of the sample per axis */
    double c0;         /* taps: weight of the value entering each axis pass */
    const double *toff, *tw; /* taps: offsets (voxels) and weights, ntap each */
} oparams;

#define OR_FILTER_NONE 0
#define OR_FILTER_CLIP 1
#define OR_FILTER_SCALE 2

/* The per-sample filter of Algorithm 1 ("val <- filter(val)"): Algorithm 10 replaces a
 * value below the minimum or above the maximum threshold by DATAMIN; Algorithm 11 does
 * the same and maps the kept range onto [0, 1].  A value within eps of a threshold is a
 * rounding decision. */
static double filter_value(const oparams *P, double v, int *frag)
{
    if (P->filter == OR_FILTER_NONE)
        return v;
    if (frag && P->eps_val > 0.0 && (fabs(v - P->tmin) < P->eps_val || fabs(v - P->tmax) < P->eps_val))
        *frag |= FRAG_ROUND;
    if (P->filter == OR_FILTER_CLIP) {
        if (v < P->tmin)
            v = P->lo;
        if (v > P->tmax)
            v = P->lo;
        return v;
    }
    const double ratio = 1.0 / (P->tmax - P->tmin);
    if (v > P->tmax)
        return P->lo;
    if (v < P->tmin)
        return P->lo;
    return (v - P->tmin) * ratio;
}

/* Alpha of the first-moment-inspired colourings (spectral, first moment): the value's
 * position in the colour-map domain, or -- with the threshold option (the remedy for
 * faint images the paper's discussion gives) -- transparent up to tmin, opaque above. */
static double colour_alpha(const oparams *P, double v, int *frag)
{
    if (!P->alpha_thr)
        return normalise(v, P->lo, P->hi);
    if (frag && P->eps_val > 0.0 && fabs(v - P->tmin) < P->eps_val)
        *frag |= FRAG_ROUND;
    return v > P->tmin ? 1.0 : 0.0;
}

/* A trilinear sample is NaN when any corner of its cell is; at a cell face next to a
 * NaN voxel, which cell the position falls in -- and so whether the sample is NaN --
 * is a rounding decision.  Flag samples within eps of such a face. */
static void nan_face_check(const ovol *V, const double p[3], double v, double eps, int *frag)
{
    for (int a = 0; a < 3; ++a) {
        if (dist_to_int(p[a]) >= eps)
            continue;
        double q[3] = {p[0], p[1], p[2]};
        q[a] = p[a] + eps;
        int n1 = isnan(sample_trilinear(V, q));
        q[a] = p[a] - eps;
        int n2 = isnan(sample_trilinear(V, q));
        if (n1 != isnan(v) || n2 != isnan(v))
            *frag |= FRAG_ROUND;
    }
}

/* Fetch counter (Section 6 counts texture fetches per ray step); counts only while enabled. */
static int g_count_fetches = 0;
static long long g_fetches = 0;

void oracle_fetch_counter(int enable) { g_count_fetches = enable; g_fetches = 0; }
long long oracle_fetches(void) { return g_fetches; }

static double fetch(const ovol *V, int interp, const double p[3], double eps, int *frag)
{
    if (g_count_fetches) {
#pragma omp atomic
        ++g_fetches;
    }
    if (interp == OR_NEAREST)
        return sample_nearest(V, p, eps, frag);
    double v = sample_trilinear(V, p);
    if (frag && eps > 0.0)
        nan_face_check(V, p, v, eps, frag);
    return v;
}

#define OR_SMOOTH_NONE 0
#define OR_SMOOTH_BOX 1
#define OR_SMOOTH_TAPS 2

/* Algorithm 1's "val <- smooth(val)" (Section 4.1-4.2), applied to one cube's sample at
 * p on a ray of unit direction d.
 *
 * Box (Algorithm 8): the sample plus arm neighbours on each side along the ray, one
 * voxel apart (p +- i d, i = 1..arm), summed and scaled by 1/(2 arm + 1).
 *
 * Taps (Algorithm 9): one pass per data axis, x then y then z.  A pass starts from the
 * value it is given (the raw sample for the x pass, the previous pass's result after
 * that), weights it by c0 and adds w_j times the cube at p +- off_j along its axis.
 * Every tap is a plain fetch of the cube, so a sample costs 1 + 6 ntap fetches. */
static double smooth_fetch(const ovol *V, const oparams *P, const double p[3], const double d[3], int *frag)
{
    double val = fetch(V, P->interp, p, P->eps_pos, frag);
    if (P->smooth == OR_SMOOTH_BOX) {
        for (int i = 1; i <= P->arm; ++i) {
            double fwd[3], back[3];
            for (int a = 0; a < 3; ++a) {
                fwd[a] = p[a] + i * d[a];
                back[a] = p[a] - i * d[a];
            }
            val += fetch(V, P->interp, fwd, P->eps_pos, frag);
            val += fetch(V, P->interp, back, P->eps_pos, frag);
        }
        val *= 1.0 / (2.0 * P->arm + 1.0);
    } else if (P->smooth == OR_SMOOTH_TAPS) {
        for (int axis = 0; axis < 3; ++axis) {
            double out = val * P->c0;
            for (int j = 0; j < P->ntap; ++j) {
                double q[3] = {p[0], p[1], p[2]};
                q[axis] = p[axis] + P->toff[j];
                out += fetch(V, P->interp, q, P->eps_pos, frag) * P->tw[j];
                q[axis] = p[axis] - P->toff[j];
                out += fetch(V, P->interp, q, P->eps_pos, frag) * P->tw[j];
            }
            val = out;
        }
    }
    return val;
}

/* The sample's z coordinate as used by spectral-position colouring: the channel of
 * the voxel for nearest sampling, the continuous coordinate for trilinear. */
static double sample_z(const ovol *V, int interp, const double p[3])
{
    if (interp == OR_NEAREST) {
        long k = (long)floor(p[2] + 0.5);
        if (k < 0) k = 0;
        if (k > V->n[2] - 1) k = V->n[2] - 1;
        return (double)k;
    }
    return p[2];
}

/* A position's texture coordinate along an axis of n voxels, (p + 1/2) / n in [0, 1]. */
static double tex_coord(double p, int n)
{
    double t = (p + 0.5) / (double)n;
    return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

/* The sample's position as colouring uses it: the voxel for nearest sampling, the point
 * itself for trilinear (sample_z's rule on every axis). */
static void sample_pos(const ovol *V, int interp, const double p[3], double q[3])
{
    for (int a = 0; a < 3; ++a) {
        if (interp == OR_NEAREST) {
            long k = (long)floor(p[a] + 0.5);
            if (k < 0) k = 0;
            if (k > V->n[a] - 1) k = V->n[a] - 1;
            q[a] = (double)k;
        } else {
            q[a] = p[a];
        }
    }
}

static int channel_of(double z, int nz)
{
    long k = (long)floor(z + 0.5);
    if (k < 0) k = 0;
    if (k > nz - 1) k = nz - 1;
    return (int)k;
}

/* One ray of Algorithm 1 with the selected transfer function. */
static void render_ray(const ovol *V, const ovol *V2, const ocam *c, const oparams *P, int px, int py,
                       double rgba[4], double *scalar, int *index, int *nsamp, int *frag)
{
    double o[3], d[3], t0;
    rgba[0] = rgba[1] = rgba[2] = rgba[3] = 0.0;
    *scalar = 0.0;
    *index = -1;
    *nsamp = 0;
    pixel_ray(c, px, py, o, d);
    int N = clip_ray(V->n, o, d, P->h, &t0, P->eps_pos, frag);
    if (N <= 0)
        return;

    double m = -INFINITY, zmax = 0.0;        /* MIP / MIP_1 state */
    double sum = 0.0;                        /* average state */
    double sw = 0.0, szw = 0.0;              /* first-moment state: sum of weights, of z * weight */
    double top = -INFINITY;                  /* largest v - lo over the samples */
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};  /* compositing state */
    double mpos[3] = {0.0, 0.0, 0.0};        /* MIP_RGB: position of the maximum */
    double m1 = -INFINITY, m2 = -INFINITY;   /* line ratio Method 1: maximum of each cube */
    double *vals = NULL, *zs = NULL;         /* kept for the near-tie check */
    int track = (P->mode == OR_MIP || P->mode == OR_SPECTRAL || P->mode == OR_RATIO || P->mode == OR_MIP_RGB) &&
                P->eps_val > 0.0;
    if (track) {
        vals = (double *)malloc(sizeof(double) * (size_t)N);
        zs = (double *)malloc(sizeof(double) * (size_t)N);
    }
    int done = 0;
    double near_ratio = -INFINITY; /* largest value a near-threshold sample could take */
    for (int k = 0; k < N; ++k) {
        double t = t0 + (k + 0.5) * P->h;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double v;
        if (P->mode == OR_RATIO_MIP) {
            /* Algorithm 13: each cube's running maximum (">"; a NaN sample is DATAMIN) */
            double c1 = filter_value(P, smooth_fetch(V, P, p, d, frag), frag);
            double c2 = filter_value(P, smooth_fetch(V2, P, p, d, frag), frag);
            if (isnan(c1)) c1 = P->lo;
            if (isnan(c2)) c2 = P->lo;
            if (c1 > m1) m1 = c1;
            if (c2 > m2) m2 = c2;
            ++done;
            continue;
        }
        if (P->mode == OR_RATIO) {
            /* Algorithm 14: val = cube2/cube1 where cube1 > 0 (threshold f), else DATAMIN */
            double c1 = filter_value(P, smooth_fetch(V, P, p, d, frag), frag);
            double c2 = filter_value(P, smooth_fetch(V2, P, p, d, frag), frag);
            v = (c1 > P->ratio_floor) ? c2 / c1 : P->lo;
            if (frag && P->eps_val > 0.0 && fabs(c1 - P->ratio_floor) < P->eps_val) {
                double alt = (c1 > P->ratio_floor) ? P->lo : c2 / c1; /* the other branch */
                double vv = isnan(v) ? P->lo : v, aa = isnan(alt) ? P->lo : alt;
                double hi2 = vv > aa ? vv : aa;
                if (hi2 > near_ratio) near_ratio = hi2;
            }
        } else {
            v = smooth_fetch(V, P, p, d, frag);
            if (isnan(v))
                v = P->lo; /* NaN sample -> DATAMIN */
            v = filter_value(P, v, frag);
        }
        if (isnan(v))
            v = P->lo; /* NaN sample (or ratio) -> DATAMIN */
        ++done;
        switch (P->mode) {
        case OR_MIP:
        case OR_RATIO:
        case OR_SPECTRAL:
        case OR_MIP_RGB:
            /* Eq. 1 / Algorithms 2, 4 and 6: c_i = v_i if v_i >= c_{i-1} */
            if (v >= m) {
                m = v;
                zmax = sample_z(V, P->interp, p);
                sample_pos(V, P->interp, p, mpos);
            }
            if (track) {
                vals[k] = v;
                zs[k] = sample_z(V, P->interp, p);
            }
            break;
        case OR_AVG:
            sum += v;
            break;
        case OR_MOMENT1: {
            /* Eq. 4 along the ray: weights are the intensity above DATAMIN (NaN and
             * values at or below DATAMIN weigh nothing), positions the sample's z */
            double w = v - P->lo;
            if (w > top)
                top = w;
            if (w < 0.0)
                w = 0.0;
            sw += w;
            szw += sample_z(V, P->interp, p) * w;
            sum += v;
            break;
        }
        case OR_COMPOSITE:
        case OR_COMPOSITE_SPECTRAL:
        case OR_COMPOSITE_RGB: {
            /* Algorithm 3 in premultiplied form: a = clamp(s * A_lut(v_hat), 0, 1); the
             * colour from the value (Algorithm 3), from the sample's spectral position
             * through the colour map (Algorithm 5), or from its position (Algorithm 7) */
            double col[4];
            lut_eval(P->lut, normalise(v, P->lo, P->hi), col);
            double a = P->s * col[3];
            a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
            if (P->mode != OR_COMPOSITE) {
                double q[3];
                sample_pos(V, P->interp, p, q);
                if (P->mode == OR_COMPOSITE_SPECTRAL) {
                    double cz[4];
                    lut_eval(P->lut, tex_coord(q[2], V->n[2]), cz);
                    col[0] = cz[0];
                    col[1] = cz[1];
                    col[2] = cz[2];
                } else {
                    col[0] = tex_coord(q[2], V->n[2]);
                    col[1] = tex_coord(q[1], V->n[1]);
                    col[2] = tex_coord(q[0], V->n[0]);
                }
            }
            for (int ch = 0; ch < 3; ++ch)
                C[ch] += T * a * col[ch];
            T *= (1.0 - a);
            double A = 1.0 - T;
            if (frag && P->eps_exit > 0.0 && fabs(A - P->term_alpha) < P->eps_exit)
                *frag |= FRAG_EXIT;
            if (A > P->term_alpha)
                k = N; /* early ray termination */
            break;
        }
        }
    }
    *nsamp = done;
    double col[4];
    switch (P->mode) {
    case OR_MIP:
    case OR_RATIO:
        *scalar = m;
        *index = channel_of(zmax, V->n[2]);
        lut_eval(P->lut, normalise(m, P->lo, P->hi), rgba);
        break;
    case OR_SPECTRAL: {
        /* Algorithm 4: colour from the spectral position of the maximum, alpha from its value */
        double tz = (zmax + 0.5) / (double)V->n[2];
        lut_eval(P->lut, tz < 0.0 ? 0.0 : (tz > 1.0 ? 1.0 : tz), col);
        rgba[0] = col[0];
        rgba[1] = col[1];
        rgba[2] = col[2];
        rgba[3] = colour_alpha(P, m, frag);
        *scalar = m;
        *index = channel_of(zmax, V->n[2]);
        break;
    }
    case OR_AVG:
        *scalar = sum / (double)N;
        lut_eval(P->lut, normalise(*scalar, P->lo, P->hi), rgba);
        break;
    case OR_COMPOSITE:
    case OR_COMPOSITE_SPECTRAL:
    case OR_COMPOSITE_RGB:
        rgba[0] = C[0];
        rgba[1] = C[1];
        rgba[2] = C[2];
        rgba[3] = 1.0 - T;
        *scalar = 1.0 - T;
        break;
    case OR_MIP_RGB:
        /* Algorithm 6: (r, g, b) = the maximum's (z, y, x) as texture coordinates */
        rgba[0] = tex_coord(mpos[2], V->n[2]);
        rgba[1] = tex_coord(mpos[1], V->n[1]);
        rgba[2] = tex_coord(mpos[0], V->n[0]);
        rgba[3] = colour_alpha(P, m, frag);
        *scalar = m;
        *index = channel_of(zmax, V->n[2]);
        break;
    case OR_RATIO_MIP:
        /* Algorithm 13: the colour of maxval2 / maxval1 where maxval1 > 0 (the floor),
         * else transparent black */
        if (m1 > P->ratio_floor) {
            *scalar = m2 / m1;
            lut_eval(P->lut, normalise(*scalar, P->lo, P->hi), rgba);
        } else {
            *scalar = P->lo;
        }
        if (frag && P->eps_val > 0.0 && fabs(m1 - P->ratio_floor) < P->eps_val)
            *frag |= FRAG_RATIO;
        break;
    case OR_MOMENT1:
        /* the intensity-weighted mean position (the velocity field of a moment-1 map),
         * coloured like spectral colouring, alpha from the mean intensity; nothing above
         * DATAMIN: transparent, no channel */
        if (sw > 0.0) {
            double m1 = szw / sw;
            double tz = (m1 + 0.5) / (double)V->n[2];
            lut_eval(P->lut, tz < 0.0 ? 0.0 : (tz > 1.0 ? 1.0 : tz), col);
            rgba[0] = col[0];
            rgba[1] = col[1];
            rgba[2] = col[2];
            rgba[3] = colour_alpha(P, sum / (double)N, frag);
            *scalar = m1;
            *index = channel_of(m1, V->n[2]);
            /* the channel is a rounding of m1: fragile within 1e-3 of a half channel;
             * and a total weight at rounding level makes the moment itself a rounding
             * decision (interpolated values within rounding of DATAMIN) */
            if (frag && P->eps_val > 0.0 && (fabs(m1 - floor(m1) - 0.5) < 1e-3 || sw < P->eps_val))
                *frag |= FRAG_ROUND;
        } else if (frag && P->eps_val > 0.0 && top > -P->eps_val) {
            *frag |= FRAG_ROUND; /* no weight, but a sample within rounding of DATAMIN */
        }
        break;
    }
    if (frag && P->mode == OR_RATIO && near_ratio >= m - P->eps_val)
        *frag |= FRAG_RATIO;
    if (track) {
        /* another sample within eps of the maximum: which one wins is a rounding
         * decision.  It matters if it changes the channel (index) or, for spectral
         * colouring, the z position that sets the hue. */
        int ch = channel_of(zmax, V->n[2]);
        for (int k = 0; k < N; ++k) {
            /* exact ties (e.g. two DATAMIN samples, equal voxel values) are resolved
             * identically by any implementation of ">="; only near ties are fragile */
            if (!(vals[k] >= m - P->eps_val) || vals[k] == m)
                continue;
            int differs = (P->mode == OR_MIP_RGB) ? 1
                          : (P->mode == OR_SPECTRAL) ? (zs[k] != zmax) : (channel_of(zs[k], V->n[2]) != ch);
            if (differs)
                *frag |= FRAG_TIE;
        }
        free(vals);
        free(zs);
    }
}

/* Render the pixels listed in pix (row-major pixel ids), or every pixel when pix is NULL.
 * Outputs are indexed by list position.  Any output pointer may be NULL. */
int oracle_render3(const double *cube, const double *cube2, int nx, int ny, int nz,
                   const double *cam14, int ortho, int W, int H,
                   int mode, int interp, double step, double lo, double hi,
                   const double *lut, double opacity_scale, double term_alpha, double ratio_floor,
                   const long *pix, long npix, double eps_pos, double eps_val, double eps_exit,
                   double *out_rgba, double *out_scalar, int *out_index, int *out_nsamples,
                   unsigned char *out_fragile, int filter, double tmin, double tmax, int alpha_thr,
                   int smooth, int arm, int ntap, double c0, const double *toff, const double *tw)
{
    if (!cube || nx <= 0 || ny <= 0 || nz <= 0 || W <= 0 || H <= 0 || !(step > 0.0) || !lut)
        return 1;
    if (mode < OR_MIP || mode > OR_RATIO_MIP)
        return -1;
    if ((mode == OR_RATIO || mode == OR_RATIO_MIP) && !cube2)
        return 1;
    ovol V = {cube, {nx, ny, nz}}, V2 = {cube2, {nx, ny, nz}};
    ocam c = make_cam(cam14, ortho, W, H);
    if (filter < OR_FILTER_NONE || filter > OR_FILTER_SCALE || (filter != OR_FILTER_NONE && !(tmin <= tmax)) ||
        (filter == OR_FILTER_SCALE && !(tmin < tmax)) || (alpha_thr != 0 && alpha_thr != 1))
        return -1;
    if (smooth < OR_SMOOTH_NONE || smooth > OR_SMOOTH_TAPS || (smooth == OR_SMOOTH_BOX && arm < 0) ||
        (smooth == OR_SMOOTH_TAPS && (ntap < 0 || (ntap > 0 && (!toff || !tw)))))
        return -1;
    oparams P = {mode, interp, step, lo, hi, opacity_scale, term_alpha, ratio_floor, eps_pos, eps_val, eps_exit, lut,
                 filter, tmin, tmax, alpha_thr, smooth, arm, ntap, c0, toff, tw};
    long n = pix ? npix : (long)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (long q = 0; q < n; ++q) {
        long id = pix ? pix[q] : q;
        int px = (int)(id % W), py = (int)(id / W);
        double rgba[4], sc;
        int idx, ns, fr = 0;
        render_ray(&V, &V2, &c, &P, px, py, rgba, &sc, &idx, &ns, &fr);
        if (out_rgba)
            for (int ch = 0; ch < 4; ++ch)
                out_rgba[4 * q + ch] = rgba[ch];
        if (out_scalar) out_scalar[q] = sc;
        if (out_index) out_index[q] = idx;
        if (out_nsamples) out_nsamples[q] = ns;
        if (out_fragile) out_fragile[q] = (unsigned char)fr;
    }
    return 0;
}

/* The same without smoothing (Algorithm 1 with smooth(val) = val). */
int oracle_render2(const double *cube, const double *cube2, int nx, int ny, int nz,
                   const double *cam14, int ortho, int W, int H,
                   int mode, int interp, double step, double lo, double hi,
                   const double *lut, double opacity_scale, double term_alpha, double ratio_floor,
                   const long *pix, long npix, double eps_pos, double eps_val, double eps_exit,
                   double *out_rgba, double *out_scalar, int *out_index, int *out_nsamples,
                   unsigned char *out_fragile, int filter, double tmin, double tmax, int alpha_thr)
{
    return oracle_render3(cube, cube2, nx, ny, nz, cam14, ortho, W, H, mode, interp, step, lo, hi, lut,
                          opacity_scale, term_alpha, ratio_floor, pix, npix, eps_pos, eps_val, eps_exit, out_rgba,
                          out_scalar, out_index, out_nsamples, out_fragile, filter, tmin, tmax, alpha_thr,
                          OR_SMOOTH_NONE, 0, 0, 1.0, NULL, NULL);
}

/* The same without a filter (Algorithm 1 with filter(val) = val). */
int oracle_render(const double *cube, const double *cube2, int nx, int ny, int nz,
                  const double *cam14, int ortho, int W, int H,
                  int mode, int interp, double step, double lo, double hi,
                  const double *lut, double opacity_scale, double term_alpha, double ratio_floor,
                  const long *pix, long npix, double eps_pos, double eps_val, double eps_exit,
                  double *out_rgba, double *out_scalar, int *out_index, int *out_nsamples,
                  unsigned char *out_fragile)
{
    return oracle_render2(cube, cube2, nx, ny, nz, cam14, ortho, W, H, mode, interp, step, lo, hi, lut,
                          opacity_scale, term_alpha, ratio_floor, pix, npix, eps_pos, eps_val, eps_exit, out_rgba,
                          out_scalar, out_index, out_nsamples, out_fragile, OR_FILTER_NONE, 0.0, 0.0, 0);
}

/* Sample count of every ray (the loop bound N of Algorithm 1), without sampling. */
long long oracle_count_samples(int nx, int ny, int nz, const double *cam14, int ortho, int W, int H,
                               double step, int *out_n)
{
    int n[3] = {nx, ny, nz};
    ocam c = make_cam(cam14, ortho, W, H);
    long long total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (long q = 0; q < (long)W * H; ++q) {
        double o[3], d[3], t0;
        pixel_ray(&c, (int)(q % W), (int)(q / W), o, d);
        int N = clip_ray(n, o, d, step, &t0, 0.0, NULL);
        if (out_n) out_n[q] = N;
        total += N;
    }
    return total;
}

/* Positions and fetched values of every sample of one ray (diagnostics and ties). */
int oracle_ray_trace(const double *cube, int nx, int ny, int nz, const double *cam14, int ortho,
                     int W, int H, int interp, double step, int px, int py, int maxn,
                     double *out_pos, double *out_val)
{
    ovol V = {cube, {nx, ny, nz}};
    ocam c = make_cam(cam14, ortho, W, H);
    double o[3], d[3], t0;
    pixel_ray(&c, px, py, o, d);
    int N = clip_ray(V.n, o, d, step, &t0, 0.0, NULL);
    for (int k = 0; k < N && k < maxn; ++k) {
        double t = t0 + (k + 0.5) * step;
        double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        for (int a = 0; a < 3; ++a)
            out_pos[3 * k + a] = p[a];
        out_val[k] = fetch(&V, interp, p, 0.0, NULL);
    }
    return N;
}

/* The fetch of Algorithm 1 at arbitrary points (pts[n][3], index space). */
int oracle_sample_points(const double *cube, int nx, int ny, int nz, int interp, const double *pts, long n,
                         double *out)
{
    ovol V = {cube, {nx, ny, nz}};
    for (long q = 0; q < n; ++q)
        out[q] = fetch(&V, interp, pts + 3 * q, 0.0, NULL);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Smoothing (Section 4.2)
 * ------------------------------------------------------------------------- */

/* Eq. 5 sampled on the integer taps k = -r..r of one axis (isotropic), normalised to sum 1. */
void oracle_gauss_weights(double sigma, int r, double *w)
{
    double s = 0.0;
    for (int k = -r; k <= r; ++k) {
        w[k + r] = exp(-(double)k * k / (2.0 * sigma * sigma));
        s += w[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k)
        w[k] /= s;
}

/* Binomial filter b_n = [1,1]^{*n}: n autoconvolutions of [1,1], by Pascal's rule,
 * then normalised by 2^n.  w has n+1 entries. */
void oracle_binomial_weights(int n, double *w)
{
    for (int m = 0; m <= n; ++m)
        w[m] = 0.0;
    w[0] = 1.0;
    for (int it = 0; it < n; ++it)
        for (int m = it + 1; m >= 1; --m)
            w[m] += w[m - 1];
    double s = ldexp(1.0, n);
    for (int m = 0; m <= n; ++m)
        w[m] /= s;
}

/* Collapse a symmetric discrete kernel w[-r..r] into fetches at fractional offsets
 * whose linear interpolation between neighbouring taps reproduces it (the
 * "linear sampling" merge the paper uses for Algorithm 9): the centre tap stays,
 * taps (2j-1, 2j) merge into one weight w_a + w_b at offset (a w_a + b w_b)/(w_a + w_b).
 * Returns the number of merged one-sided fetches; off[0] = 0, wt[0] = centre weight. */
int oracle_linear_sampling_merge(const double *w, int r, double *off, double *wt)
{
    off[0] = 0.0;
    wt[0] = w[r];
    int m = 0;
    for (int a = 1; a <= r; a += 2) {
        double wa = w[r + a], wb = (a + 1 <= r) ? w[r + a + 1] : 0.0;
        ++m;
        wt[m] = wa + wb;
        off[m] = (wa + wb) > 0.0 ? (a * wa + (a + 1) * wb) / (wa + wb) : (double)a;
    }
    return m;
}

static inline long clampl(long i, long n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

/* Separable 3-D convolution with the 1-D kernel w[-r..r] on each axis in turn
 * (x, then y, then z), clamp-to-edge boundary, all passes in double. */
int oracle_smooth_separable(const double *in, int nx, int ny, int nz, const double *w, int r, double *out)
{
    size_t n = (size_t)nx * ny * nz;
    double *a = (double *)malloc(n * sizeof(double)), *b = (double *)malloc(n * sizeof(double));
    if (!a || !b) {
        free(a);
        free(b);
        return 1;
    }
#pragma omp parallel for collapse(2)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = -r; k <= r; ++k)
                    s += w[k + r] * in[((size_t)z * ny + y) * nx + clampl(x + k, nx)];
                a[((size_t)z * ny + y) * nx + x] = s;
            }
#pragma omp parallel for collapse(2)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = -r; k <= r; ++k)
                    s += w[k + r] * a[((size_t)z * ny + clampl(y + k, ny)) * nx + x];
                b[((size_t)z * ny + y) * nx + x] = s;
            }
#pragma omp parallel for collapse(2)
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int k = -r; k <= r; ++k)
                    s += w[k + r] * b[((size_t)clampl(z + k, nz) * ny + y) * nx + x];
                out[((size_t)z * ny + y) * nx + x] = s;
            }
    free(a);
    free(b);
    return 0;
}

/* The same convolution written directly as the triple sum over the 3-D kernel
 * w[i] w[j] w[k] (Eq. 5 is separable), evaluated at the listed voxels only. */
int oracle_smooth_points(const double *in, int nx, int ny, int nz, const double *w, int r,
                         const long *vox_ids, long npts, double *out)
{
#pragma omp parallel for schedule(static)
    for (long q = 0; q < npts; ++q) {
        long id = vox_ids[q];
        long x = id % nx, y = (id / nx) % ny, z = id / ((long)nx * ny);
        double s = 0.0;
        for (int k = -r; k <= r; ++k)
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i)
                    s += w[k + r] * w[j + r] * w[i + r] *
                         in[((size_t)clampl(z + k, nz) * ny + clampl(y + j, ny)) * nx + clampl(x + i, nx)];
        out[q] = s;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Reduced-precision storage: round-to-nearest-even of a float32 value to
 * bfloat16 (1-8-7) and to IEEE binary16 (1-5-10), returned as the float32 it
 * represents.  Written from the two formats' definitions.
 * ------------------------------------------------------------------------- */
void oracle_round_bf16(const float *in, long n, float *out)
{
    for (long i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], 4);
        if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan: keep (quiet the nan) */
            if (u & 0x007fffffu) u |= 0x00400000u;
            u &= 0xffff0000u;
        } else {
            uint32_t lsb = (u >> 16) & 1u;
            u = (u + 0x7fffu + lsb) & 0xffff0000u;
        }
        memcpy(&out[i], &u, 4);
    }
}

void oracle_round_f16(const float *in, long n, float *out)
{
    for (long i = 0; i < n; ++i) {
        double x = (double)in[i];
        if (isnan(x) || isinf(x)) {
            out[i] = in[i];
            continue;
        }
        double ax = fabs(x);
        if (ax >= 65520.0) { /* rounds to infinity */
            out[i] = (float)(x > 0 ? INFINITY : -INFINITY);
            continue;
        }
        int e;
        frexp(ax, &e); /* ax = m 2^e, m in [0.5, 1) */
        int ulp_exp = e - 11; /* 11 significant bits */
        if (ulp_exp < -24) ulp_exp = -24; /* subnormal spacing 2^-24 */
        double q = ldexp(ax, -ulp_exp);
        double fl = floor(q), rem = q - fl;
        if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0))
            fl += 1.0;
        double r = ldexp(fl, ulp_exp);
        out[i] = (float)copysign(r, x);
    }
}

/* ---------------------------------------------------------------------------
 * Adjoint of the compositing render (Algorithm 3), by reverse mode over a tape of
 * every sample of the ray (no checkpointing: a different algorithm from the GPU's).
 * Loss gradient in: g[H*W*4] = dL/d(C_r, C_g, C_b, alpha).  Accumulates (+=) into
 * grad_vol[nz*ny*nx], grad_lut[256*4] and grad_s.  Clamp kinks take the
 * pass-through derivative on the closed interval (0 <= x <= 1).  The early-exit
 * index is treated as fixed.
 * ------------------------------------------------------------------------- */
typedef struct {
    double p[3];
    int nan;
    double x;      /* (v - lo)/(hi - lo) before the clamp */
    double vhat;
    double col[4];
    double alpha;  /* s * A_lut before the clamp */
    double a;
    double T;      /* transmittance before this sample */
} tape_t;

int oracle_render_grad(const double *cube, int nx, int ny, int nz, const double *cam14, int ortho,
                       int W, int H, int interp, double step, double lo, double hi,
                       const double *lut, double s, double term_alpha, const double *g,
                       double *out_rgba, double *grad_vol, double *grad_lut, double *grad_s)
{
    ovol V = {cube, {nx, ny, nz}};
    ocam c = make_cam(cam14, ortho, W, H);
    double gs_total = 0.0;
    double *glut_all = (double *)calloc(1024, sizeof(double));
#pragma omp parallel
    {
        double glut[1024];
        double gs = 0.0;
        memset(glut, 0, sizeof(glut));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < (long)W * H; ++q) {
            int px = (int)(q % W), py = (int)(q / W);
            double o[3], d[3], t0;
            pixel_ray(&c, px, py, o, d);
            int N = clip_ray(V.n, o, d, step, &t0, 0.0, NULL);
            double T = 1.0, C[3] = {0, 0, 0};
            tape_t *tp = N > 0 ? (tape_t *)malloc(sizeof(tape_t) * (size_t)N) : NULL;
            int K = 0;
            for (int k = 0; k < N; ++k) {
                tape_t *e = &tp[k];
                double t = t0 + (k + 0.5) * step;
                for (int a = 0; a < 3; ++a)
                    e->p[a] = o[a] + t * d[a];
                double v = fetch(&V, interp, e->p, 0.0, NULL);
                e->nan = isnan(v);
                if (e->nan) v = lo;
                e->x = (v - lo) / (hi - lo);
                e->vhat = e->x < 0 ? 0 : (e->x > 1 ? 1 : e->x);
                lut_eval(lut, e->vhat, e->col);
                e->alpha = s * e->col[3];
                e->a = e->alpha < 0 ? 0 : (e->alpha > 1 ? 1 : e->alpha);
                e->T = T;
                for (int ch = 0; ch < 3; ++ch)
                    C[ch] += T * e->a * e->col[ch];
                T *= (1.0 - e->a);
                K = k + 1;
                if (1.0 - T > term_alpha)
                    break;
            }
            if (out_rgba) {
                out_rgba[4 * q + 0] = C[0];
                out_rgba[4 * q + 1] = C[1];
                out_rgba[4 * q + 2] = C[2];
                out_rgba[4 * q + 3] = 1.0 - T;
            }
            const double *gq = g + 4 * q;
            double gT = -gq[3]; /* alpha_out = 1 - T_K */
            for (int k = K - 1; k >= 0; --k) {
                tape_t *e = &tp[k];
                /* C += T_k a_k col_k ; T_{k+1} = T_k (1 - a_k) */
                double ga = 0.0, gcol[4] = {0, 0, 0, 0};
                for (int ch = 0; ch < 3; ++ch) {
                    ga += gq[ch] * e->T * e->col[ch];
                    gcol[ch] = gq[ch] * e->T * e->a;
                }
                ga += -gT * e->T;
                double gTk = gT * (1.0 - e->a);
                for (int ch = 0; ch < 3; ++ch)
                    gTk += gq[ch] * e->a * e->col[ch];
                gT = gTk;
                /* a = clamp(alpha) ; alpha = s * A_lut */
                double galpha = (e->alpha >= 0.0 && e->alpha <= 1.0) ? ga : 0.0;
                gs += galpha * e->col[3];
                gcol[3] = galpha * s;
                /* colour map: col = (1-f) L[i0] + f L[i0+1], u = 255 v_hat */
                double u = 255.0 * e->vhat;
                long i0 = (long)floor(u);
                if (i0 > 254) i0 = 254;
                if (i0 < 0) i0 = 0;
                double f = u - (double)i0;
                double gvhat = 0.0;
                for (int ch = 0; ch < 4; ++ch) {
                    glut[4 * i0 + ch] += (1.0 - f) * gcol[ch];
                    glut[4 * (i0 + 1) + ch] += f * gcol[ch];
                    gvhat += 255.0 * gcol[ch] * (lut[4 * (i0 + 1) + ch] - lut[4 * i0 + ch]);
                }
                if (e->nan || !grad_vol)
                    continue;
                double gx = (e->x >= 0.0 && e->x <= 1.0) ? gvhat : 0.0;
                double gv = gx / (hi - lo);
                if (gv == 0.0)
                    continue;
                if (interp == OR_NEAREST) {
                    long i[3];
                    for (int a = 0; a < 3; ++a)
                        i[a] = clampl((long)floor(e->p[a] + 0.5), V.n[a]);
#pragma omp atomic
                    grad_vol[((size_t)i[2] * ny + i[1]) * nx + i[0]] += gv;
                } else {
                    long i[3];
                    double fr[3];
                    for (int a = 0; a < 3; ++a) {
                        double fl = floor(e->p[a]);
                        i[a] = (long)fl;
                        fr[a] = e->p[a] - fl;
                    }
                    for (int cz = 0; cz < 2; ++cz)
                        for (int cy = 0; cy < 2; ++cy)
                            for (int cx = 0; cx < 2; ++cx) {
                                double w = (cx ? fr[0] : 1 - fr[0]) * (cy ? fr[1] : 1 - fr[1]) *
                                           (cz ? fr[2] : 1 - fr[2]);
                                size_t vid = ((size_t)clampl(i[2] + cz, nz) * ny + clampl(i[1] + cy, ny)) * nx +
                                             clampl(i[0] + cx, nx);
#pragma omp atomic
                                grad_vol[vid] += w * gv;
                            }
                }
            }
            free(tp);
        }
#pragma omp critical
        {
            for (int j = 0; j < 1024; ++j)
                glut_all[j] += glut[j];
            gs_total += gs;
        }
    }
    if (grad_lut)
        for (int j = 0; j < 1024; ++j)
            grad_lut[j] += glut_all[j];
    if (grad_s)
        *grad_s += gs_total;
    free(glut_all);
    return 0;
}

int oracle_abi_version(void) { return 1; }
