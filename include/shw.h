/*
 * shw.h -- C ABI of the GB300 spectral-cube ray caster (libshw.so).
 *
 * The library renders 3-D float spectral cubes (two spatial axes x, y and one
 * spectral axis z) by per-pixel ray casting, as in "Real-time colouring and
 * filtering with graphics shaders" (Vohl et al. 2017): every ray takes samples
 * at a fixed step (Algorithm 1) and folds them with one transfer function --
 * maximum intensity (Eq. 1, Algorithm 2), average (Eq. 3), front-to-back alpha
 * compositing through an RGBA colour map (Eq. 2, Algorithm 3), spectral-position
 * colouring (Algorithm 4) or the per-sample ratio of two cubes (Algorithm 14); also the
 * first moment (Eq. 4), AVIP_1 / MIP_RGB / AVIP_RGB (Algorithms 5-7), the line ratio's
 * Method 1 (Algorithms 12-13), per-sample clipping and domain scaling (Algorithms 10-11)
 * and in-ray box / per-axis tap smoothing (Algorithms 8-9) -- and smooths cubes with a
 * separable 3-D Gaussian (Eqs. 5-6, Algorithm 9).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Cube layout: C-contiguous float32 [nz][ny][nx], x fastest, z = spectral.
 *   Voxel (i, j, k) sits at the point (i, j, k) of index space; the cube's box
 *   is [-0.5, n-0.5] on each axis; reads outside clamp to the nearest edge voxel.
 * - Rays: pixel (px, py) of a W x H image (row 0 at the top) has screen
 *   coordinates xs = 2(px+1/2)/W - 1, ys = 1 - 2(py+1/2)/H (Appendix A).
 *   Parallel projection: origin eye + xs*ortho_half_h*(W/H)*right + ys*ortho_half_h*up,
 *   direction fwd/|fwd|.  Perspective: origin eye, direction
 *   normalize(fwd + xs*tan_half_fovy*(W/H)*right + ys*tan_half_fovy*up).
 *   The ray is clipped to the box and to t >= 0 giving [t0, t1]; it takes
 *   N = floor((t1 - t0)/step) samples at t0 + (k + 1/2)*step, k = 0..N-1.
 * - Normalisation: v_hat = clamp((v - lo)/(hi - lo), 0, 1); the colour map is
 *   256 RGBA knots interpolated linearly at u = 255*v_hat.  A sample that is NaN
 *   counts as DATAMIN = lo.
 * - Pointers named *device* are CUDA device (or managed) memory owned by the
 *   caller; the library never frees them and keeps none after a call returns
 *   (a batch plan excepted, see shw_batch_plan_create).  Pointers named *host*
 *   are read during the call only.
 * - Every launch is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *   default stream).  A call returns SHW_OK once its work is enqueued, or an
 *   error before enqueuing anything.  Device-side faults of the CUDA runtime
 *   surface as SHW_ECUDA from a later call or from shw_sync_status.
 * - No call falls back to a CPU implementation.
 */
#ifndef SHW_H
#define SHW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHW_ABI_VERSION 5
#define SHW_LUT_SIZE 256
#define SHW_MAX_SMOOTH_RADIUS 16
#define SHW_MAX_SMOOTH_ARM 16   /* in-ray box smoothing: neighbours on each side */
#define SHW_MAX_SMOOTH_TAPS 4   /* in-ray tap smoothing: fetches on each side per axis */
#define SHW_BRICK 32        /* brick edge of the reduced-precision storage, voxels */
#define SHW_BRICK_APRON 1   /* replicated border kept around every brick, voxels */

typedef enum {
    SHW_OK = 0,
    SHW_EINVAL = 1,        /* a NULL pointer, a non-positive size, an unknown enum ... */
    SHW_EUNSUPPORTED = 2,  /* a valid request this build does not handle (size limits) */
    SHW_ECUDA = 3,         /* the CUDA runtime reported an error */
    SHW_ENOMEM = 4,        /* a caller buffer is too small, or a plan allocation failed */
    SHW_ETIMEOUT = 5,      /* a kernel's bounded wait for its own asynchronous copy gave up (shw_sync_status) */
    SHW_EDEVICE = 6,       /* no usable CUDA device */
    SHW_EBOUNDS = 7        /* a bounds-checked build (SHW_CHECKED) found an index outside its array
                              (shw_sync_status; the access was clamped into the array) */
} shw_status;

typedef enum {
    SHW_MIP = 0,        /* Eq. 1 / Algorithm 2: running maximum, ">=" (the last maximum wins) */
    SHW_AVG = 1,        /* Eq. 3: mean of the samples (zeroth moment / N on a spectral-axis view) */
    SHW_COMPOSITE = 2,  /* Eq. 2 / Algorithm 3: front-to-back compositing through the colour map */
    SHW_SPECTRAL = 3,   /* Algorithm 4: colour from the spectral position of the maximum */
    SHW_RATIO = 4,      /* Algorithm 14: per-sample cube2/cube1, then maximum */
    SHW_MOMENT1 = 5,    /* Eq. 4 along the ray: sum(z w) / sum(w), w = max(v - lo, 0), z the sample's
                           height (its channel when nearest); colour from (M1 + 1/2) / nz, alpha
                           from the mean intensity; a ray with no weight is transparent, channel -1 */
    SHW_COMPOSITE_SPECTRAL = 6, /* Algorithm 5 (AVIP_1): compositing, each sample coloured by the map at
                                   its spectral position (z + 1/2) / nz, opacity as SHW_COMPOSITE */
    SHW_MIP_RGB = 7,        /* Algorithm 6: maximum; (r, g, b) = the maximum's (z, y, x) as texture
                               coordinates (p + 1/2) / n, alpha from its value */
    SHW_COMPOSITE_RGB = 8,  /* Algorithm 7 (AVIP_RGB): compositing, each sample coloured by its (z, y, x) */
    SHW_RATIO_MIP = 9       /* Algorithms 12-13 (line ratio, Method 1): each cube's maximum; the colour of
                               max2 / max1 where max1 > ratio_floor, else transparent black (scalar
                               DATAMIN); needs vol2 like SHW_RATIO; channel output -1 */
    /* Modes 5..9 are not in batch plans (SHW_EUNSUPPORTED); positions follow spectral
       colouring's rule: the voxel for nearest sampling, the point for trilinear. */
} shw_mode;

typedef enum { SHW_NEAREST = 0, SHW_TRILINEAR = 1 } shw_interp;

typedef enum {
    SHW_F32 = 0,        /* linear float32 [nz][ny][nx] */
    SHW_BF16_BRICK = 1, /* bricks written by shw_pack_bricks, bfloat16 */
    SHW_F16_BRICK = 2,  /* bricks written by shw_pack_bricks, IEEE binary16 */
    SHW_F32_PAIR = 3,   /* the two co-registered cubes of a line ratio interleaved: float32
                           [nz][ny][nx][2], element 0 the first cube (the ratio's denominator),
                           element 1 the second; 8-byte aligned.  Only SHW_RATIO and SHW_RATIO_MIP
                           render it (vol2 = NULL; other modes SHW_EUNSUPPORTED), without in-ray
                           smoothing; results equal the two-cube render bit for bit.  Written by
                           shw_smooth_zip */
    SHW_BF16_PAIR_BRICK = 4, /* the pair storage as bricks: 32-bit elements, the low half the first
                                cube's bfloat16, the high half the second's; written by
                                shw_pack_bricks from an SHW_F32_PAIR buffer; the line ratios only */
    SHW_F16_PAIR_BRICK = 5,  /* the same with IEEE binary16 halves */
    SHW_BF16 = 6,       /* linear bfloat16 [nz][ny][nx] (raw 16-bit values, rounded to nearest even),
                           written by shw_pack_bricks.  Only the staged marcher renders the linear
                           16-bit storages: trilinear sampling, no in-ray smoothing, data 16-byte
                           aligned, nx * element bytes a multiple of 16, fewer than 2^31 voxels;
                           other requests SHW_EUNSUPPORTED */
    SHW_F16 = 7,        /* the same with IEEE binary16 */
    SHW_BF16_PAIR = 8,  /* the line ratios' two cubes as linear 16-bit pairs: 32-bit elements
                           [nz][ny][nx], the low half the first cube's bfloat16, the high half the
                           second's; written by shw_pack_bricks from an SHW_F32_PAIR buffer;
                           SHW_RATIO and SHW_RATIO_MIP only, with the limits of SHW_BF16 */
    SHW_F16_PAIR = 9    /* the same with IEEE binary16 halves */
} shw_storage;

/* A cube.  data: device.  For SHW_F32 it is the linear float32 array; for the
 * brick and 16-bit storages it is the buffer filled by shw_pack_bricks for the same dims. */
typedef struct {
    const void *data;
    int32_t nx, ny, nz;
    int32_t storage; /* shw_storage */
} shw_volume;

/* A camera in index space (Appendix A).  right, up and fwd should be unit and
 * mutually orthogonal; fwd is normalised by the library for parallel rays. */
typedef struct {
    float eye[3], right[3], up[3], fwd[3];
    float tan_half_fovy; /* perspective: tan of half the vertical field of view */
    float ortho_half_h;  /* parallel: half height of the view window, voxels */
    int32_t ortho;       /* 1 = parallel projection, 0 = perspective */
    int32_t width, height;
} shw_camera;

typedef struct {
    int32_t mode;          /* shw_mode */
    int32_t interp;        /* shw_interp */
    float step;            /* sample spacing along the ray, voxels, > 0 */
    float lo, hi;          /* colour-map domain; lo is also DATAMIN; hi > lo */
    const float *lut;      /* device, [256][4] RGBA float32 */
    float opacity_scale;   /* COMPOSITE: a = clamp(opacity_scale * A_lut(v_hat), 0, 1) (k of Algorithm 3) */
    float term_alpha;      /* COMPOSITE: stop after the sample that makes alpha > term_alpha (0.99) */
    float ratio_floor;     /* RATIO: a sample's ratio is cube2/cube1 where cube1 > ratio_floor, else DATAMIN */
    int32_t ckpt_interval; /* COMPOSITE checkpoints for the adjoint: samples between checkpoints (64) */
    int32_t filter;        /* shw_filter: per-sample filter applied before the transfer function (after a
                              NaN sample became DATAMIN; for SHW_RATIO, to each cube's sample) */
    float min_threshold;   /* the filter's minimum threshold; also the alpha threshold (below) */
    float max_threshold;   /* the filter's maximum threshold (>= min_threshold; > for SHW_FILTER_SCALE) */
    int32_t alpha_threshold; /* SHW_SPECTRAL / SHW_MOMENT1: 0 = alpha from the value; 1 = alpha 0 when the
                                value that sets it is <= min_threshold, else 1 (the paper's remedy for
                                faint first-moment-style images) */
    int32_t smooth;          /* shw_smooth_kind: per-sample smoothing of each fetched value, before the
                                filter (Algorithm 1's "smooth"; Sections 4.1-4.2) */
    int32_t smooth_arm;      /* SHW_SMOOTH_BOX: neighbours on each side, 0..SHW_MAX_SMOOTH_ARM */
    int32_t smooth_ntaps;    /* SHW_SMOOTH_TAPS: fetches on each side of the sample per axis,
                                0..SHW_MAX_SMOOTH_TAPS */
    float smooth_c0;         /* SHW_SMOOTH_TAPS: weight of the value entering each axis pass */
    float smooth_offset[SHW_MAX_SMOOTH_TAPS]; /* SHW_SMOOTH_TAPS: fetch offsets along the axis, voxels,
                                                 |offset| <= 64 (first smooth_ntaps used) */
    float smooth_weight[SHW_MAX_SMOOTH_TAPS]; /* SHW_SMOOTH_TAPS: weight of each of the two fetches at
                                                 +-offset (first smooth_ntaps used) */
} shw_render_params;

/* In-ray smoothing of every fetched sample (the cube lookups of Algorithm 1; both cubes
 * for the line ratios).  Reads beyond the cube clamp to the edge voxel like every fetch.
 * Only the general marcher applies it: batch plans and the adjoint reject it
 * (SHW_EUNSUPPORTED). */
typedef enum {
    SHW_SMOOTH_NONE = 0,
    SHW_SMOOTH_BOX = 1, /* Algorithm 8: (v(p) + sum_{i=1..arm} v(p + i u) + v(p - i u)) / (2 arm + 1),
                           u the ray's unit direction (neighbours one voxel apart along the ray);
                           2 arm + 1 fetches per sample.  With a step of exactly 1/2 voxel and a
                           single cube the neighbours are the ray's own samples, and the box runs
                           as running sums (about 2 fetches per sample; equal to the direct sums to
                           FP32 rounding); SHW_DEBUG_BOX_DIRECT (shw_set_debug_flags) selects the
                           direct fetches */
    SHW_SMOOTH_TAPS = 2 /* Algorithm 9 once per data axis e = x, then y, then z, each pass starting from
                           the previous pass's value (the raw sample for x):
                           val <- c0 val + sum_j w_j (v(p + off_j e) + v(p - off_j e));
                           1 + 6 ntaps fetches per sample (Section 6's 3(N-1)/2 + 1 for an N-tap
                           kernel merged by linear sampling, e.g. Algorithm 9's 9-tap: ntaps = 2) */
} shw_smooth_kind;

typedef enum {
    SHW_FILTER_NONE = 0,
    SHW_FILTER_CLIP = 1,  /* Algorithm 10: a value below min_threshold or above max_threshold -> DATAMIN */
    SHW_FILTER_SCALE = 2  /* Algorithm 11: outside [min, max] -> DATAMIN, else (v - min) / (max - min) */
} shw_filter;

/* ---- library information (host only, no GPU needed) ---------------------- */

int32_t shw_abi_version(void);
const char *shw_status_string(int32_t status);
/* sizeof of the ABI structs: which = 0 shw_volume, 1 shw_camera, 2 shw_render_params,
 * 3 shw_batch_item, 4 shw_batch_info. */
size_t shw_struct_size(int32_t which);
/* Number of kernels this library has launched in this process (all devices). */
uint64_t shw_launch_count(void);

/* Wait for `stream` and report any error the CUDA runtime has latched, then the
 * library's device error word of the current device (SHW_ETIMEOUT; the word is cleared).
 * A library built with -DSHW_CHECKED (paper_1707_00442_gb300.build.build_checked) also
 * checks every index its kernels take without clamping -- the interior fast paths of the
 * samplers, the staged marcher's shared-memory reads, the plane sweep's offsets and planes,
 * the smoothing's output planes -- clamps a violating one into its array and records it:
 * this call then reports SHW_EBOUNDS (and clears the record). */
shw_status shw_sync_status(void *stream);

/* ---- smoothing (Section 4.2) ---------------------------------------------- */

/* Separable 3-D Gaussian smoothing (Eq. 5 isotropic; Eq. 6 links sigma to the
 * FWHM): out = in convolved with w (x) w (x) w, where
 * w_k = exp(-k^2 / (2 sigma^2)) / sum_j exp(-j^2 / (2 sigma^2)), k = -radius..radius,
 * clamp-to-edge boundary.  in, out: device float32 [nz][ny][nx], must not overlap.
 * sigma > 0, 0 <= radius <= SHW_MAX_SMOOTH_RADIUS.  One kernel; no scratch memory. */
shw_status shw_smooth(const float *in, float *out, int32_t nx, int32_t ny, int32_t nz,
                      float sigma, int32_t radius, void *stream);

/* The same with caller-given 1-D weights w_host[2*radius+1] (host; used as given,
 * not renormalised), e.g. the binomial b_n filters of Section 4.2. */
shw_status shw_smooth_weights(const float *in, float *out, int32_t nx, int32_t ny, int32_t nz,
                              const float *w_host, int32_t radius, void *stream);

/* Smoothing into the interleaved storage of the line ratios: out_pair[v] = (first[v],
 * smooth(in)[v]) for every voxel v, smooth(in) exactly as shw_smooth(in, sigma, radius)
 * computes it.  in, first: device float32 [nz][ny][nx] (first is typically the other cube,
 * already smoothed; in == first is allowed); out_pair: device float32 [nz][ny][nx][2],
 * 8-byte aligned, overlapping neither input.  One kernel: in and first are read once,
 * out_pair is written once. */
shw_status shw_smooth_zip(const float *in, const float *first, float *out_pair, int32_t nx, int32_t ny,
                          int32_t nz, float sigma, int32_t radius, void *stream);

/* ---- fetch tables of in-ray tap smoothing (Section 4.2, Algorithm 9) ------ */

/* Fold a symmetric 1-D kernel into the fetches of SHW_SMOOTH_TAPS by linear sampling
 * (Section 4.2, the trick behind Algorithm 9's 9-tap kernel): the centre keeps w[r]; taps
 * a and a+1 (a = 1, 3, 5, ...) become one interpolated fetch of weight w[r+a] + w[r+a+1]
 * at offset (a w[r+a] + (a+1) w[r+a+1]) / (w[r+a] + w[r+a+1]) (a lone last tap keeps its
 * own offset and weight).  w_host: host, 2*radius+1 finite values, w[r+k] == w[r-k];
 * 0 <= radius <= 64.  Outputs (host): *c0, offsets[j], weights[j] for j < *nfetch =
 * ceil(radius/2); capacity = slots in offsets and weights (SHW_ENOMEM if too few).
 * Computed in double precision on the host; no GPU is needed. */
shw_status shw_linear_sampling_taps(const double *w_host, int32_t radius, double *c0, double *offsets,
                                    double *weights, int32_t capacity, int32_t *nfetch);

/* The N-tap binomial filter of Section 4.2 folded as above: b_n = [1, 1] convolved with
 * itself n = ntaps - 1 + 2*drop times (Pascal's row n), without its `drop` outer taps on
 * each side, renormalised to sum 1.  ntaps odd >= 1, drop >= 0, n <= 62
 * (SHW_EUNSUPPORTED beyond).  ntaps = 5, 9, 13 with drop = 0 are b_4, b_8, b_12;
 * ntaps = 9, drop = 2 gives the offsets 1.3846153846, 3.2307692308 and coefficients
 * 0.2270270270, 0.3162162162, 0.0702702703 that Algorithm 9 prints.  Host only. */
shw_status shw_binomial_taps(int32_t ntaps, int32_t drop, double *c0, double *offsets, double *weights,
                             int32_t capacity, int32_t *nfetch);

/* ---- reduced-precision storage (bricks and linear 16-bit cubes) ------------ */

/* Bytes of the buffer of a reduced-precision storage for a cube of these dims.  Bricks:
 * ceil(n/32) bricks per axis, each (32+2)^3 elements of 2 bytes (a 1-voxel apron on every
 * face), 4-byte elements for the pair bricks.  Linear 16-bit storages: nx*ny*nz elements of
 * 2 bytes (4 for SHW_BF16_PAIR / SHW_F16_PAIR).  Returns 0 for invalid arguments. */
size_t shw_bricked_bytes(int32_t nx, int32_t ny, int32_t nz, int32_t storage);

/* Round a float32 cube to a reduced-precision storage, to nearest even.  Bricks: brick
 * (bx, by, bz) starts at element ((bz*nby + by)*nbx + bx) * 34^3 and stores, at
 * ((lz*34 + ly)*34 + lx), the voxel (32 bx + lx - 1, 32 by + ly - 1, 32 bz + lz - 1)
 * clamped to the cube.  Linear 16-bit storages: element v holds voxel v.
 * in: device float32 [nz][ny][nx], or for the pair storages the SHW_F32_PAIR buffer
 * [nz][ny][nx][2] (8-byte aligned); out: device, 2-byte aligned (4 for pairs),
 * out_bytes >= shw_bricked_bytes. */
shw_status shw_pack_bricks(const float *in, int32_t nx, int32_t ny, int32_t nz, int32_t storage,
                           void *out, size_t out_bytes, void *stream);

/* ---- rendering (Sections 2-4) -------------------------------------------- */

/* Render one image.  vol2: the second cube for SHW_RATIO / SHW_RATIO_MIP (same dims and
 * storage), else NULL; NULL also when vol holds both cubes as SHW_F32_PAIR.  Outputs (device, any may be NULL except out_rgba):
 *   out_rgba   [H][W][4] float32: MIP/AVG/RATIO/RATIO_MIP: colourMap(v_hat(result));
 *              SPECTRAL: (colourMap_rgb(t_z), v_hat(max)), t_z = (z_max + 1/2)/nz;
 *              MOMENT1, MIP_RGB: as described with their modes;
 *              COMPOSITE and its coloured forms: premultiplied (C_r, C_g, C_b, 1 - T).
 *   out_scalar [H][W] float32: the maximum / mean / ratio maximum / 1 - T / first moment /
 *              max2 / max1 (RATIO_MIP; DATAMIN where max1 fails the floor).
 *   out_index  [H][W] int32: channel round(z) of the maximum (MIP, SPECTRAL, RATIO, MIP_RGB) or of
 *              the first moment (MOMENT1, -1 with no weight); -1 otherwise.
 *   out_nsamples [H][W] int32: samples the ray processed.
 * A ray that misses the box (or has N = 0) writes zeros and index -1.
 * ckpt: COMPOSITE only, device buffer of ckpt_bytes >= shw_ckpt_bytes(...), or NULL:
 * the transmittance every ckpt_interval samples, read by shw_render_backward.
 * Scheduling state: views that are not spectral-axis sweeps run as persistent CTAs that
 * take tiles from a device work counter, one of 1024 per device handed out in turn and
 * zeroed on `stream` at each call.  So at most 1024 renders may be enqueued and not yet
 * finished at once across all streams of a device, and a call made while `stream` is being
 * captured into a CUDA graph is refused with SHW_EUNSUPPORTED (a replayed capture would
 * keep its counter while later calls reuse it); batch plans are the graph-launched form. */
shw_status shw_render(const shw_volume *vol, const shw_volume *vol2, const shw_camera *cam,
                      const shw_render_params *p, float *out_rgba, float *out_scalar,
                      int32_t *out_index, int32_t *out_nsamples, void *ckpt, size_t ckpt_bytes,
                      void *stream);

/* Size of the checkpoint buffer for a COMPOSITE render of this volume/camera. */
size_t shw_ckpt_bytes(const shw_volume *vol, const shw_camera *cam, const shw_render_params *p);

/* ---- adjoint of compositing ----------------------------------------------- */

/* Reverse-mode gradient of a COMPOSITE render (Eq. 2 / Algorithm 3 in premultiplied
 * form) with respect to the voxels, the colour map and the opacity scale.
 * vol, cam, p: exactly those of the forward shw_render call that filled `ckpt`
 * (p->mode = SHW_COMPOSITE, 1 <= p->ckpt_interval <= 64; vol->storage = SHW_F32).
 * grad_rgba: device [H][W][4] float32, dL/d(C_r, C_g, C_b, alpha) of the forward's out_rgba.
 * Each segment of ckpt_interval samples is recomputed from its checkpoint, then
 * reversed.  Gradients ACCUMULATE (+=) into the device buffers grad_vol
 * [nz][ny][nx], grad_lut [256][4] and grad_scale [1]; any of them may be NULL.
 * Accumulation uses atomics, so the low bits of the result may vary run to run.
 * The early-exit sample of each ray is treated as fixed; at a clamp boundary the
 * gradient passes (closed interval). */
shw_status shw_render_backward(const shw_volume *vol, const shw_camera *cam, const shw_render_params *p,
                               const float *grad_rgba, const void *ckpt, size_t ckpt_bytes, float *grad_vol,
                               float *grad_lut, float *grad_scale, void *stream);

/* ---- test and diagnosis switches (no paper counterpart) -------------------- */

/* Process-wide switches for tests that compare two paths of the library or exercise its
 * failure handling; all off by default, and no caller needs them for normal use.  Each
 * call replaces every flag and returns the previous set.  The switches change which
 * kernel serves a request, never what it computes (the fault switches excepted). */
#define SHW_DEBUG_NO_AXIS_SWEEP 0x1u  /* orthographic spectral-axis views take the general marcher */
#define SHW_DEBUG_SMOOTH_PLAIN  0x2u  /* smoothing takes its kernel without tensor copies */
#define SHW_DEBUG_BOX_DIRECT    0x4u  /* in-ray box smoothing by direct fetches, never the lattice sums */
#define SHW_DEBUG_NO_STAGING    0x8u  /* general views take the gather marcher, not the staged one */
#define SHW_DEBUG_FAULT_ALLOC   0x10u /* batch-plan device allocations fail (SHW_ENOMEM) */
#define SHW_DEBUG_FAULT_GRAPH   0x20u /* batch-plan graph capture fails (SHW_ECUDA) */
#define SHW_DEBUG_REQUIRE_STAGING 0x80u /* a render of a float32 cube or pair storage that neither the
                                           spectral-axis sweep nor the staged marcher serves is
                                           refused (SHW_EUNSUPPORTED) instead of taking the gather
                                           marcher */
#define SHW_DEBUG_FAULT_TIMEOUT 0x40u /* smoothing launched while set (its tensor-copy form: radius 1..8,
                                         nx a multiple of 4) leaves the copy of each z chunk's second
                                         plane unissued and bounds its waits at about 1 ms: every CTA
                                         gives up at that plane, waits for its other copies and returns;
                                         shw_sync_status then reports SHW_ETIMEOUT and the output is
                                         incomplete.  Later calls run normally */
uint32_t shw_set_debug_flags(uint32_t flags);

/* ---- batched rendering of many sub-cubes ----------------------------------- */

/* Survey pipelines cut a sub-cube around each of many detected sources (Section 1).
 * A plan renders all of them with ONE graph launch: a persistent kernel per kind of
 * item (float32 cubes, bricks), captured in a CUDA graph; every (item, image tile) is a
 * work item, CTAs pop work items from a device counter, tiles of the largest items
 * first.  Each image is the same as shw_render of that item with the shared parameters. */

typedef struct shw_batch_plan shw_batch_plan; /* opaque */

#define SHW_BATCH_NO_TUNE 1 /* skip the autotuner: 16 x 16 tiles, 4 CTAs per SM, 32^3 bricks when packing */
#define SHW_BATCH_RETUNE 2  /* re-run the autotuner even if this batch signature is cached */
#define SHW_BATCH_PACK_BF16 4 /* the plan rounds every SHW_F32 item into bfloat16 bricks that it
                                 allocates and owns, with the brick edge (16 or 32 voxels) that the
                                 autotuner picks; each image is that of shw_render on the item's
                                 shw_pack_bricks storage (the values and the arithmetic do not
                                 depend on the edge).  Items of other storages render as given */
#define SHW_BATCH_PACK_F16 8  /* the same with IEEE binary16 */
#define SHW_BATCH_BRICK_16 16 /* with a PACK flag: 16^3 bricks, the edge not tuned */
#define SHW_BATCH_BRICK_32 32 /* with a PACK flag: 32^3 bricks, the edge not tuned */

typedef struct {
    shw_volume vol;  /* the sub-cube: SHW_F32 or 16-bit bricks, < 2^31 voxels; bricks (the caller's, or
                        the plan's own at either edge) < 2^31 stored elements, else SHW_EUNSUPPORTED */
    shw_camera cam;  /* its view; its image is cam.width x cam.height */
    float *out_rgba; /* device [H][W][4] float32, 16-byte aligned; written by every shw_render_batch */
    int32_t mode;    /* SHW_MIP, SHW_AVG, SHW_COMPOSITE or SHW_SPECTRAL (SHW_RATIO: SHW_EUNSUPPORTED) */
} shw_batch_item;

typedef struct {
    int32_t n_items, n_work;     /* items, work items (tiles) */
    int32_t tile, ctas_per_sm;   /* the chosen tile edge (pixels) and persistent CTAs per SM */
    int32_t grid, tuned;         /* CTAs of each kernel; 1 if the autotuner ran for this plan */
    int32_t brick;               /* edge of the plan's own bricks (16 or 32); 0 when it packs none */
    int32_t n_candidates;        /* configurations the autotuner times: tile x CTAs per SM, and
                                    x brick edge when the plan packs bricks and the edge is free */
    int32_t cand_tile[16], cand_ctas_per_sm[16], cand_brick[16];
    float tune_ms[16];           /* measured time of each candidate (-1 when not tuned) */
    int64_t packed_bytes;        /* device bytes of the plan's own bricks */
} shw_batch_info;

/* Build a plan for n items sharing the parameters p (p->mode is ignored: each item
 * has its own; interp, step, lo, hi, lut, opacity_scale, term_alpha are shared).
 * Allocates device memory for the item table, the work list and the counters, and
 * captures the launch into a CUDA graph: one persistent kernel for the float32 items and
 * one for the brick items, one after the other (a kernel for both would hold the
 * registers of both paths).  With SHW_BATCH_PACK_BF16 or _F16 it also
 * allocates the 16-bit bricks of its float32 items (the layout of shw_pack_bricks with
 * 32 replaced by the edge E and 34 by E + 2) and fills them on `stream`; the float32
 * cubes are not read after that.  Unless SHW_BATCH_NO_TUNE, the first plan of a batch
 * signature (mean size class, image size, storages, modes, packing) times every
 * candidate configuration on `stream` -- rendering into the items' outputs -- and keeps
 * the fastest; later plans of the same signature reuse the choice.  Tuning the brick
 * edge packs the items at both edges, so for a moment the plan holds both copies.
 * The plan keeps the item pointers (cubes, outputs, colour map) until destroyed.
 * Errors: SHW_EINVAL (also: both PACK flags, both BRICK flags, or a BRICK flag without a
 * PACK flag), SHW_EUNSUPPORTED, SHW_ENOMEM (allocation), SHW_ECUDA (capture),
 * SHW_EDEVICE.  SHW_DEBUG_FAULT_ALLOC / SHW_DEBUG_FAULT_GRAPH make the allocation or the
 * capture fail (host-side fault injection, see shw_set_debug_flags). */
shw_status shw_batch_plan_create(shw_batch_plan **plan, const shw_batch_item *items, int32_t n,
                                 const shw_render_params *p, int32_t flags, void *stream);

/* Render every item of the plan: one graph launch on `stream` (same device as the plan).
 * Launches of one plan must not overlap: they share the plan's work counter. */
shw_status shw_render_batch(shw_batch_plan *plan, void *stream);

shw_status shw_batch_plan_info(const shw_batch_plan *plan, shw_batch_info *info);

/* The same items rendered one launch each, in order, by a loop inside the library: each is
 * shw_render(&item.vol, NULL, &item.cam, p with mode = item.mode, item.out_rgba, NULL, NULL,
 * NULL, NULL, 0, stream).  The unbatched path a plan is measured against (no host language
 * overhead between launches).  Returns the first non-OK status (earlier items stay enqueued). */
shw_status shw_render_items(const shw_batch_item *items, int32_t n, const shw_render_params *p, void *stream);

/* Waits for the device to finish outstanding work, then frees the plan. */
shw_status shw_batch_plan_destroy(shw_batch_plan *plan);

/* ---- batched rendering without device allocation -------------------------- */

/* The paper has no counterpart of this call.  It exists for callers that cannot
 * let a library allocate device memory -- a host program that owns every byte of
 * the GPU through its own pool or budget (for example a plugin inside a
 * visualisation application), or an interactive loop that must never stall in an
 * allocator.  It renders the same images as a batch plan (16 x 16 tiles, 4 CTAs per
 * SM, no autotuning) but keeps the item table, the work list and the work counters
 * in a fixed device array that is part of the library: every GPU that loads
 * libshw.so holds SHW_NOALLOC_SCRATCH_BYTES of it until the process exits.  The
 * call makes no cudaMalloc/cudaFree or other allocating call; the caller passes the
 * inputs and outputs as for shw_batch_plan_create.
 *  - Capacity: 256 + 128 * n + 8 * (total 16 x 16 tiles of all images) bytes must fit
 *    in SHW_NOALLOC_SCRATCH_BYTES, else SHW_EUNSUPPORTED and nothing is enqueued.
 *  - The first call on a device looks up the array's device address (with that
 *    device current) and caches it.  A call made while `stream` is being captured into
 *    a CUDA graph is refused with SHW_EUNSUPPORTED: the call copies the item table and
 *    the work list from host memory it owns only while it runs.
 *  - That copy is from ordinary (pageable) host memory, so the call returns only after
 *    the work already enqueued on `stream` has finished and the table has been handed
 *    to the copy engine: the host waits for the stream, though no allocator is touched.
 *  - Every call reuses the one array per device and overwrites the previous call's
 *    contents (the counters are cleared on `stream` first).  Calls whose work can
 *    overlap on the GPU -- on different streams without ordering -- race with each
 *    other; calls on one stream are ordered.
 *  - Other errors as for shw_batch_plan_create. */
#define SHW_NOALLOC_SCRATCH_BYTES (8u << 20)
shw_status shw_render_batch_noalloc(const shw_batch_item *items, int32_t n, const shw_render_params *p,
                                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SHW_H */
