// render_slab.cuh -- the staged marcher: ray casting (Algorithm 1) through shared-memory
// slabs of the cube filled by tensor copies.
//
// The gather marcher (render_impl.cuh) fetches each interpolation cell's 8 corners from
// global memory per ray; its warps wait on those dependent loads most of the time.  Here a
// CTA owns a 16 x 16 pixel tile and its rays advance together through the cube in slabs:
//   - one producer warp computes, from the tile's four corner rays, which cells the tile's
//     rays can touch in the next few planes along the tile's major axis (the slab), and
//     stages that footprint into a shared-memory ring with cp.async.bulk.tensor copies of
//     8-row chunks (mbarrier completion, every wait bounded);
//   - eight consumer warps, one ray per thread in 8 x 4 warp tiles, interpolate from the
//     staged slab with the same fixed-point positions and the same arithmetic as the
//     gather marcher, so every output is bit-identical to it;
//   - the slab's depth is chosen per slab so its footprint fills one stage: thick slabs
//     where the tile's rays are close together, thin ones where they have spread out.
// Staging is only a cache: a sample whose cell lies outside the staged box (a footprint
// wider than the box, a slab the producer skipped) reads global memory like the gather
// marcher, and samples whose corners need edge clamping (the ray's head and tail) always
// do.  So the geometry of the footprints decides the speed, never the result.
#pragma once

#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "render_impl.cuh"
#include "tma.cuh"

namespace shw {

constexpr int kSlabTW = 16, kSlabTH = 16;            // pixel tile of one CTA
constexpr int kSlabWarps = 8;                        // consumer warps; warp w covers 8 x 4 pixels
constexpr int kSlabThreads = 32 * (kSlabWarps + 1);  // + the producer warp
constexpr int kSlabStages = 3;                       // ring depth
constexpr int kSlabStageBytes = 32 * 1024;           // bytes of one stage (a multiple of 128)
constexpr int kSlabRows = 8;                         // rows of one tensor copy (a chunk)
constexpr int kSlabMinBlocks = 2;
// bounded waits: kSlabWaitPolls x kSlabSleepNs is about a second
constexpr int kSlabWaitPolls = 1 << 20;
constexpr uint32_t kSlabSleepNs = 1000;

enum : int { kStageSlab = 0, kStageTile = 1, kStageTileEnd = 2, kStageExit = 3 };

// What the producer tells the consumers about one stage (written before the stage's "full"
// barrier is armed, read after it completes).
struct SlabHdr {
    int type, tile;
    int major, dir;     // the slab axis (0 x, 1 y, 2 z); +1: rays advance towards larger cells
    int s_lo, s_len;    // the slab: cells [s_lo, s_lo + s_len) along the major axis
    int ox, oy, oz;     // cell coordinates of the staged box's first element
    int ex1, ey1, ez1;  // a cell c is staged with c + 1 when (unsigned)(c - o) < e1 on every axis
    int sy, sz;         // element strides of y and z in the stage
    int wide;           // y- and z-major: the box rows are the wide chunk width (else the narrow one)
    int pad;
};
static_assert(sizeof(SlabHdr) == 64, "stage header");

// Element policies: the stored element, its size, and its value(s) in FP32.
struct ElemF32 {
    using raw = float;
    static constexpr bool kPair = false;
    __device__ __forceinline__ static float cvt(float r) { return r; }
};
struct ElemF32Pair {
    using raw = float2;
    static constexpr bool kPair = true;
    __device__ __forceinline__ static float2 cvt(float2 r) { return r; }
};
template <typename T>
struct ElemH {
    using raw = unsigned short;
    static constexpr bool kPair = false;
    __device__ __forceinline__ static float cvt(unsigned short r) { return to_f32<T>(r); }
};
template <typename T>
struct ElemHPair {
    using raw = unsigned;
    static constexpr bool kPair = true;
    __device__ __forceinline__ static float2 cvt(unsigned r) { return pair_to_f32<T>(r); }
};

// Chunk widths.  A chunk's rows lie one row pitch apart in the stage; pitches of 20, 28 and
// 40 words put 8 consecutive rows on different shared-memory banks, so the lanes of a warp,
// whose rays cover a few neighbouring rows, rarely collide.  y- and z-major slabs take the
// narrow width when their footprint fits it, else the wide one (x-major: one width).  Widths
// are 16-byte multiples and 8 rows a 128-byte multiple, as the tensor copies require.
template <class EP>
struct SlabGeom {
    static constexpr int kBytes = (int)sizeof(typename EP::raw);
    static constexpr int kAlign = 16 / kBytes;  // elements per 16 bytes (x alignment of a copy)
    // narrow and wide chunk widths (elements).  The 8-byte elements of the float32 pair
    // storage take one width of 32 (256-byte rows): a 16-pixel tile's x footprint at the
    // survey magnification is 21-30 cells, and rows of 14 / 20 made most slabs overflow
    // their box into global loads (line ratio 2.97 ms; 24 / 32: 2.16; 32: 2.13; wider rows
    // only thin the slabs)
    static constexpr int kBXn = kBytes == 8 ? 32 : (kBytes == 2 ? 80 : 112) / kBytes;
    static constexpr int kBXw = kBytes == 8 ? 32 : (kBytes == 2 ? 112 : 160) / kBytes;
    static constexpr int kBXx = 80 / kBytes;                         // x-major chunk width
    static constexpr int kStageElems = kSlabStageBytes / kBytes;
    static_assert((kBXn * kBytes) % 16 == 0 && (kBXw * kBytes) % 16 == 0 && (kBXx * kBytes) % 16 == 0,
                  "16-byte rows");
    static_assert((kSlabRows * kBXn * kBytes) % 128 == 0 && (kSlabRows * kBXw * kBytes) % 128 == 0 &&
                      (kSlabRows * kBXx * kBytes) % 128 == 0,
                  "chunks start on 128 bytes");
};

// ---- producer geometry (FP32; only the speed depends on it) -------------------------

// The ray of pixel centre (px + 1/2, py + 1/2) as origin o and (unnormalised) direction u
// (Appendix A); pixels beyond the image are allowed (the tile's outer corners).
__device__ __forceinline__ void corner_ray(const shw_camera &c, int px, int py, float o[3], float u[3])
{
    const float W = (float)c.width, H = (float)c.height;
    const float xs = (float)(2 * px + 1 - c.width) / W, ys = (float)(c.height - 2 * py - 1) / H;
    const float aspect = W / H;
    if (c.ortho) {
        const float sx = xs * c.ortho_half_h * aspect, sy = ys * c.ortho_half_h;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = c.eye[k] + sx * c.right[k] + sy * c.up[k];
            u[k] = c.fwd[k];
        }
    } else {
        const float tx = xs * c.tan_half_fovy * aspect, ty = ys * c.tan_half_fovy;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = c.eye[k];
            u[k] = c.fwd[k] + tx * c.right[k] + ty * c.up[k];
        }
    }
}

// A tile's four corner rays (pixel centres of its corner pixels) and its major axis: the
// axis the summed directions advance along fastest.
struct TileRays {
    float o[4][3], u[4][3];
    int major, dir;
};

__device__ __forceinline__ TileRays tile_rays(const shw_camera &c, int px0, int py0)
{
    TileRays t;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        corner_ray(c, px0 + (i & 1) * (kSlabTW - 1), py0 + (i >> 1) * (kSlabTH - 1), t.o[i], t.u[i]);
    float s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = t.u[0][k] + t.u[1][k] + t.u[2][k] + t.u[3][k];
    // y or z when either advances at least a quarter as fast as x: x-major boxes hold only a
    // few x planes per chunk, so their slabs stay thin
    const float ax = fabsf(s[0]), ay = fabsf(s[1]), az = fabsf(s[2]);
    t.major = ax > 4.0f * fmaxf(ay, az) ? 0 : (ay > az ? 1 : 2);
    const float sm = t.major == 0 ? s[0] : (t.major == 1 ? s[1] : s[2]);
    t.dir = sm > 0.0f ? 1 : -1;
    return t;
}

// The corner rays as lines over the major axis M: lateral coordinate a of corner ray i at
// plane m is A[i][a] + B[i][a] m.  False unless every corner advances along M with the
// tile's sign and a slope of at most kSlabMaxSlope on the other axes.
constexpr float kSlabMaxSlope = 8.0f;
template <int M>
struct TileLines {
    float A[4][3], B[4][3];
};

template <int M>
__device__ __forceinline__ bool tile_lines(const TileRays &r, TileLines<M> &t)
{
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float um = r.u[i][M];
        ok = ok && um != 0.0f && (um > 0.0f) == (r.dir > 0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float b = (k == M) ? 1.0f : r.u[i][k] / um;
            ok = ok && fabsf(b) <= kSlabMaxSlope;
            t.B[i][k] = b;
            t.A[i][k] = (k == M) ? 0.0f : r.o[i][k] - r.o[i][M] * b;
        }
    }
    return ok;
}

// Lateral cells [lo, hi] on axis a of the samples whose major coordinate lies in [m0, m1]
// (both corners of each interpolation cell included), clipped to the interior [0, n - 1].
template <int M, int AX>
__device__ __forceinline__ void lateral_cells(const TileLines<M> &t, float m0, float m1, int n, int &lo, int &hi)
{
    float pmin = INFINITY, pmax = -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float p0 = fmaf(t.B[i][AX], m0, t.A[i][AX]), p1 = fmaf(t.B[i][AX], m1, t.A[i][AX]);
        pmin = fminf(pmin, fminf(p0, p1));
        pmax = fmaxf(pmax, fmaxf(p0, p1));
    }
    const float eps = 0.02f + 1e-5f * fmaxf(fabsf(pmin), fabsf(pmax));
    const float l = floorf(pmin - eps), h = floorf(pmax + eps) + 1.0f;
    lo = (int)fmaxf(l, 0.0f);
    hi = (int)fminf(h, (float)(n - 1));
}

// One candidate slab: cells [c0, c1] along the major axis and the staged box that holds
// every cell its samples can touch (both corners of each interpolation cell).
// Stage layouts (elements): z- and x-major [z][y][x], y-major [y][z][x]; the row axis (y,
// or z for y-major) goes in chunks of kSlabRows rows, the x extent is one chunk width.
struct SlabPlan {
    SlabHdr h;
    int np, nc;  // planes and row chunks of the staged box
    bool empty;  // no interior cell of the cube can be touched
    bool fits;   // the whole footprint fits one stage (before clipping)
};

template <class EP, int M>
__device__ __forceinline__ SlabPlan plan_slab(const TileLines<M> &t, int dir, int c0, int c1, int nx, int ny, int nz)
{
    using G = SlabGeom<EP>;
    SlabPlan p;
    const float m0 = (float)c0, m1 = (float)(c1 + 1);
    SlabHdr &h = p.h;
    h.type = kStageSlab;
    h.major = M;
    h.dir = dir;
    h.s_lo = c0;
    h.s_len = c1 - c0 + 1;
    if constexpr (M == 0) {
        // x-major: the slab's planes along x inside one chunk width; rows y, planes z
        constexpr int qmax = G::kStageElems / (kSlabRows * G::kBXx);
        int ylo, yhi, zlo, zhi;
        lateral_cells<M, 1>(t, m0, m1, ny, ylo, yhi);
        lateral_cells<M, 2>(t, m0, m1, nz, zlo, zhi);
        p.empty = ylo > yhi || zlo > zhi;
        const int x0 = c0 & ~(G::kAlign - 1);
        p.nc = (yhi - ylo + kSlabRows) / kSlabRows;
        p.np = zhi - zlo + 1;
        p.fits = c1 + 1 <= x0 + G::kBXx - 1 && p.np * p.nc <= qmax;
        if (p.np * p.nc > qmax) {
            p.nc = min(p.nc, qmax);
            p.np = max(1, qmax / max(p.nc, 1));
        }
        h.ox = x0;
        h.oy = ylo;
        h.oz = zlo;
        h.ex1 = G::kBXx - 1;
        h.ey1 = p.nc * kSlabRows - 1;
        h.ez1 = p.np - 1;
        h.sy = G::kBXx;
        h.sz = p.nc * kSlabRows * G::kBXx;
        h.wide = 0;
    } else {
        // y- or z-major: planes along the major axis, x within one chunk width (narrow when
        // the footprint fits it), rows on the remaining axis (z for y-major, y for z-major)
        constexpr int R = (M == 2) ? 1 : 2;
        int xlo, xhi, rlo, rhi;
        lateral_cells<M, 0>(t, m0, m1, nx, xlo, xhi);
        lateral_cells<M, R>(t, m0, m1, R == 1 ? ny : nz, rlo, rhi);
        p.empty = xlo > xhi || rlo > rhi;
        const int x0 = xlo & ~(G::kAlign - 1);
        h.wide = xhi - x0 + 1 > G::kBXn;
        const int bx = h.wide ? G::kBXw : G::kBXn;
        const int qmax = G::kStageElems / (kSlabRows * bx);
        p.nc = (rhi - rlo + kSlabRows) / kSlabRows;
        p.np = c1 + 2 - c0;
        p.fits = p.np * p.nc <= qmax;
        if (!p.fits) p.nc = max(1, qmax / p.np);
        h.ox = x0;
        h.ex1 = bx - 1;
        if constexpr (M == 2) {
            h.oy = rlo;
            h.oz = c0;
            h.ey1 = p.nc * kSlabRows - 1;
            h.ez1 = p.np - 1;
            h.sy = bx;
            h.sz = p.nc * kSlabRows * bx;
        } else {
            h.oy = c0;
            h.oz = rlo;
            h.ey1 = p.np - 1;
            h.ez1 = p.nc * kSlabRows - 1;
            h.sy = p.nc * kSlabRows * bx;
            h.sz = bx;
        }
    }
    return p;
}

// ---- consumer side: samples through a staged slab -----------------------------------

// Algorithm 1's per-sample tail for one value (the filter, NaN as DATAMIN, the transfer
// function) and for the two cubes of the line ratios (Algorithms 13 and 14); the same
// operations as the gather marcher's interior loops.
// FILT: a per-sample filter is set (without one, filter_value returns its argument).
template <int MODE, bool FILT, class St>
__device__ __forceinline__ bool take_value(St &st, const RenderArgs &a, float v, int k)
{
    if constexpr (FILT) {
        v = filter_value(isnan(v) ? a.lo : v, a);
        v = isnan(v) ? a.lo : v;  // a NaN sample counts as DATAMIN
    } else {
        v = isnan(v) ? a.lo : v;
    }
    return st.update(v, k);
}

template <int MODE, bool FILT, class St>
__device__ __forceinline__ bool take_pair(St &st, const RenderArgs &a, float2 c, int k)
{
    const float c1 = FILT ? filter_value(c.x, a) : c.x, c2 = FILT ? filter_value(c.y, a) : c.y;
    if constexpr (MODE == SHW_RATIO_MIP) {
        st.update2(isnan(c1) ? a.lo : c1, isnan(c2) ? a.lo : c2);
        return false;
    } else {
        float v = (c1 > a.ratio_floor) ? __fdiv_rn(c2, c1) : a.lo;
        v = isnan(v) ? a.lo : v;
        return st.update(v, k);
    }
}

// The interior samples k.. (< kb) of one ray that lie in the slab of h (major axis M), in
// order; stops at the first sample a later slab holds.  Corners come from the stage when the
// cell is staged, else from global memory (no clamping: interior cells), for every sample:
// with half-voxel steps some lane of a warp enters a new cell at nearly every sample, so a
// per-lane cell cache would only add its checks (survey renders 2-5 % faster without it).
// True if the transfer function stopped the ray (k is then the count of samples processed).
// BX: the chunk width of this slab's box when fixed at compile time (the row pitch of x- and
// z-major boxes, the plane pitch of y-major ones), so that half of the 8 corner loads take
// immediate offsets; 0: both pitches from the header.
template <int MODE, class EP, int M, bool FILT, int BX, class S, class St>
__device__ __forceinline__ bool slab_march(const S &s, const RenderArgs &a, St &st, long long &X, long long &Y,
                                           long long &Z, long long DX, long long DY, long long DZ, int &k, int kb,
                                           const SlabHdr &h, const typename EP::raw *stage)
{
    using raw = typename EP::raw;
    using val = decltype(EP::cvt(raw{}));
    // the box's y and z pitches (elements); one of them the chunk width
    const int sy = (BX > 0 && M != 1) ? BX : h.sy, sz = (BX > 0 && M == 1) ? BX : h.sz;
    if constexpr (kChecked) SHW_CHECK(sy == h.sy && sz == h.sz);
    for (; k < kb; ++k) {
        const int cx = fx_cell(X), cy = fx_cell(Y), cz = fx_cell(Z);
        const int cm = M == 0 ? cx : (M == 1 ? cy : cz);
        // a sample outside the slab waits for a later one (one behind every slab -- never seen
        // on the survey views -- is marched at the tile's end with the interior left over)
        const int rel = cm - h.s_lo;
        if ((unsigned)rel >= (unsigned)h.s_len) return false;
        val c[8];
        {
            // a y- or z-major box starts at the slab's first cell and holds one plane more than
            // the slab along its axis: a sample in the slab is inside the box on that axis
            const int lx = cx - h.ox, ly = M == 1 ? rel : cy - h.oy, lz = M == 2 ? rel : cz - h.oz;
            const bool inbox = (unsigned)lx < (unsigned)h.ex1 && (M == 1 || (unsigned)ly < (unsigned)h.ey1) &&
                               (M == 2 || (unsigned)lz < (unsigned)h.ez1);
            if (inbox) {
                int off = lx + ly * sy + lz * sz;
                if constexpr (kChecked) {  // the cell's far corner lies in the stage
                    const bool ok = off >= 0 && off + sz + sy + 1 < SlabGeom<EP>::kStageElems;
                    SHW_CHECK(ok);
                    if (!ok) off = 0;
                }
                const raw *q = stage + off;
                const raw *qy = q + sy, *qz = q + sz, *qyz = qz + sy;
                c[0] = EP::cvt(q[0]);
                c[1] = EP::cvt(q[1]);
                c[2] = EP::cvt(qy[0]);
                c[3] = EP::cvt(qy[1]);
                c[4] = EP::cvt(qz[0]);
                c[5] = EP::cvt(qz[1]);
                c[6] = EP::cvt(qyz[0]);
                c[7] = EP::cvt(qyz[1]);
            } else if constexpr (EP::kPair) {
                s.template corners2<false>(cx, cy, cz, c);
            } else {
                s.template corners<false>(cx, cy, cz, c);
            }
        }
        const float fx = fx_frac(X), fy = fx_frac(Y), fz = fx_frac(Z);
        bool stop;
        if constexpr (EP::kPair)
            stop = take_pair<MODE, FILT>(st, a, trilerp_pair(c, fx, fy, fz), k);
        else
            stop = take_value<MODE, FILT>(st, a, trilerp(c, fx, fy, fz), k);
        X = fx_step(X, DX);
        Y = fx_step(Y, DY);
        Z = fx_step(Z, DZ);
        if (stop) {
            ++k;
            return true;
        }
    }
    return false;
}

// ---- the kernel ----------------------------------------------------------------------

// Wait for phase `parity` of `bar`, every lane polling (each lane's own acquire orders its
// later shared-memory reads).  Gives up after `polls` sleeping polls (about a second by
// default), recording a time-out in the error word, or as soon as another warp of the CTA
// has given up.
__device__ __forceinline__ bool slab_wait(uint64_t *bar, uint32_t parity, volatile int *quit, unsigned *err,
                                          int polls)
{
    for (int it = 0; it < polls; ++it) {
        if (__all_sync(0xffffffffu, mbar_try_wait_sleep(bar, parity, kSlabSleepNs))) return true;
        if (*quit) return false;
    }
    if ((threadIdx.x & 31) == 0 && err) atomicOr(err, kErrWaitTimeout);
    *quit = 1;
    return false;
}

// Tile t of the launch in centre-out order (rows, then columns within a row, from the
// tile under the projected cube centre): the longest rays start first.
__device__ __forceinline__ void slab_tile(int t, const RenderArgs &a, int &tx, int &ty)
{
    const int rr = t / a.tiles_x, cr = t - rr * a.tiles_x;
    ty = centre_out(rr, a.cty, a.tiles_y);
    tx = centre_out(cr, a.ctx, a.tiles_x);
}

struct SlabArgs {
    unsigned *ctr;  // the launch's tile counter
    unsigned *err;  // the library's device error word
    int ntiles;
    int polls;      // bound of every wait (sleeping polls)
};

struct SlabShared {
    SlabHdr hdr[kSlabStages];
    uint64_t full[kSlabStages], empty[kSlabStages];
    int quit;
};

// The producer warp's ring: stage take / publish with every wait bounded.
struct SlabRing {
    SlabShared &sh;
    const SlabArgs &sa;
    int posts = 0;
    // the next stage, once every consumer warp has released its previous contents (-1: give up)
    __device__ __forceinline__ int take()
    {
        const int st = posts % kSlabStages;
        if (posts >= kSlabStages &&
            !slab_wait(&sh.empty[st], (uint32_t)(((posts / kSlabStages) - 1) & 1), &sh.quit, sa.err, sa.polls))
            return -1;
        return st;
    }
    // a stage that carries only its header
    __device__ __forceinline__ bool post_plain(int type, int tile)
    {
        const int st = take();
        if (st < 0) return false;
        if ((threadIdx.x & 31) == 0) {
            SlabHdr h{};
            h.type = type;
            h.tile = tile;
            sh.hdr[st] = h;
            mbar_arrive(&sh.full[st]);
        }
        __syncwarp();
        ++posts;
        return true;
    }
};

// The slabs of one tile along major axis M, front to back.  Lane l weighs a slab of l + 1
// cells from the current cell; the thickest whose staged box fits a stage wins (one cell,
// its box clipped to a stage, when none fits), and empty runs are skipped.  False if a
// wait gave up.
template <class EP, int M>
__device__ __forceinline__ bool produce_tile(const TileRays &r, bool persp, const CUtensorMap *map_n,
                                             const CUtensorMap *map_w, const RenderArgs &a, int tile,
                                             unsigned char *stages, SlabRing &ring)
{
    using G = SlabGeom<EP>;
    TileLines<M> L;
    if (!tile_lines<M>(r, L)) return true;  // no slabs: the consumers read global memory
    const int lane = threadIdx.x & 31, dir = r.dir;
    const int n_m = M == 0 ? a.nx : (M == 1 ? a.ny : a.nz);
    int lo_c = 0, hi_c = n_m - 2;  // interior cells along the major axis
    if (persp) {
        // perspective: every ray starts at the eye, and every sample lies beyond it
        const int e = (int)fminf(fmaxf(floorf(r.o[0][M]), -1.0f), (float)n_m);
        if (dir > 0)
            lo_c = max(lo_c, e);
        else
            hi_c = min(hi_c, e);
    }
    int cur = dir > 0 ? lo_c : hi_c;
    while (cur >= lo_c && cur <= hi_c) {
        const int len = lane + 1;
        const int c0 = dir > 0 ? cur : max(cur - len + 1, lo_c);
        const int c1 = dir > 0 ? min(cur + len - 1, hi_c) : cur;
        const SlabPlan p = plan_slab<EP, M>(L, dir, c0, c1, a.nx, a.ny, a.nz);
        const unsigned em = __ballot_sync(0xffffffffu, p.empty);
        if (em & 1u) {  // nothing to stage next: skip the longest empty run weighed
            cur += dir * __shfl_sync(0xffffffffu, c1 - c0 + 1, 31 - __clz(em));
            continue;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, p.fits && !p.empty);
        const int pick = fm ? 31 - __clz(fm) : 0;
        const int span = __shfl_sync(0xffffffffu, c1 - c0 + 1, pick);
        const int np = __shfl_sync(0xffffffffu, p.np, pick), nc = __shfl_sync(0xffffffffu, p.nc, pick);
        const int ox = __shfl_sync(0xffffffffu, p.h.ox, pick), oy = __shfl_sync(0xffffffffu, p.h.oy, pick);
        const int oz = __shfl_sync(0xffffffffu, p.h.oz, pick);
        const bool wide = __shfl_sync(0xffffffffu, p.h.wide, pick) != 0;
        const int chunk = kSlabRows * (M == 0 ? G::kBXx : (wide ? G::kBXw : G::kBXn)) * G::kBytes;  // bytes of one copy
        const CUtensorMap *map = wide ? map_w : map_n;
        const int st = ring.take();
        if (st < 0) return false;
        if (lane == pick) {
            SlabHdr h = p.h;
            h.tile = tile;
            ring.sh.hdr[st] = h;
            mbar_arrive_expect_tx(&ring.sh.full[st], (uint32_t)(np * nc * chunk));
        }
        __syncwarp();
        unsigned char *base = stages + (size_t)st * kSlabStageBytes;
        for (int q = lane; q < np * nc; q += 32) {
            const int pl = q / nc, rr = q - pl * nc;
            void *dst = base + (size_t)(pl * nc + rr) * chunk;
            if (!tma_dst_ok(dst, ring.sa.err)) continue;  // never taken: stages and chunks are 128-byte multiples
            if constexpr (M == 1)
                tma_load_3d(dst, map, ox, oy + pl, oz + kSlabRows * rr, &ring.sh.full[st]);
            else
                tma_load_3d(dst, map, ox, oy + kSlabRows * rr, oz + pl, &ring.sh.full[st]);
        }
        __syncwarp();
        ++ring.posts;
        cur += dir * span;
    }
    return true;
}

// The producer warp: takes tiles from the counter and stages, for each, the slabs its rays
// cross, front to back.  Every stage carries a header: a tile's start, one slab, a tile's
// end, or the end of the launch.
template <class EP>
__device__ void slab_producer(const CUtensorMap *maps, const shw_camera &cam, const RenderArgs &a, const SlabArgs &sa,
                              unsigned char *stages, SlabShared &sh)
{
    const int lane = threadIdx.x & 31;
    SlabRing ring{sh, sa};
    bool ok = true;
    while (ok) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(sa.ctr, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned)sa.ntiles) {
            ring.post_plain(kStageExit, 0);
            break;
        }
        if (!ring.post_plain(kStageTile, (int)t)) break;
        int tx, ty;
        slab_tile((int)t, a, tx, ty);
        const TileRays r = tile_rays(cam, tx * kSlabTW, ty * kSlabTH);
        const bool persp = !cam.ortho;
        // maps: x-major; y-major narrow, wide; z-major narrow, wide
        if (r.major == 0)
            ok = produce_tile<EP, 0>(r, persp, &maps[0], &maps[0], a, (int)t, stages, ring);
        else if (r.major == 1)
            ok = produce_tile<EP, 1>(r, persp, &maps[1], &maps[2], a, (int)t, stages, ring);
        else
            ok = produce_tile<EP, 2>(r, persp, &maps[3], &maps[4], a, (int)t, stages, ring);
        if (ok) ok = ring.post_plain(kStageTileEnd, (int)t);
    }
    // the CTA may not exit while a tensor copy into its shared memory is in flight: wait
    // (bounded) for the last stages posted
    if (lane == 0) {
        for (int i = max(0, ring.posts - kSlabStages); i < ring.posts; ++i)
            for (int it = 0; it < sa.polls && !mbar_try_wait_sleep(&sh.full[i % kSlabStages],
                                                                   (uint32_t)((i / kSlabStages) & 1), kSlabSleepNs);
                 ++it) {
            }
    }
    __syncwarp();
}

// A consumer warp: one ray per thread of its 8 x 4 pixels of the current tile.  On a tile's
// start a ray is set up exactly as in the gather marcher and takes its clamped head samples
// from global memory; each slab then advances it through the interior samples the slab
// holds; at the tile's end it finishes any interior samples left (global memory), its
// clamped tail, and writes its outputs.
template <int MODE, class EP, class S>
__device__ void slab_consumer(const S &s, const shw_camera &cam, const RenderArgs &a, const SlabArgs &sa,
                              const unsigned char *stages, SlabShared &sh)
{
    using St = typename StateOf<MODE>::type;
    using raw = typename EP::raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = (warp & 1) * 8 + (lane & 7), ly = (warp >> 1) * 4 + (lane >> 3);
    volatile int *quit = &sh.quit;
    RayFx r;
    St st;
    CacheOf<S> cc;
    long long X = 0, Y = 0, Z = 0, pix = 0;
    int N = 0, k = 0, kb = 0, done = 0;
    bool has = false, live = false;
    for (int posts = 0;; ++posts) {
        const int si = posts % kSlabStages;
        if (!slab_wait(&sh.full[si], (uint32_t)((posts / kSlabStages) & 1), quit, sa.err, sa.polls)) return;
        const SlabHdr h = sh.hdr[si];
        if (h.type == kStageExit) return;
        if (h.type == kStageTile) {
            int tx, ty;
            slab_tile(h.tile, a, tx, ty);
            const int px = tx * kSlabTW + lx, py = ty * kSlabTH + ly;
            has = px < a.width && py < a.height;
            pix = (long long)py * a.width + px;
            const bool hit = has && !quick_miss(cam, px, py, s.nx, s.ny, s.nz) &&
                             setup_ray(cam, px, py, s.nx, s.ny, s.nz, a.step, r);
            N = hit ? min(r.N, a.nmax) : 0;
            st = St{};
            done = 0;
            live = N > 0;
            if (live) {
                int ka;
                interior_range(r, s.nx, s.ny, s.nz, N, ka, kb);
                init_ray_state<MODE, SHW_TRILINEAR>(st, s, a, r, pix, a.lut);
                X = r.P[0];
                Y = r.P[1];
                Z = r.P[2];
                cc.ix = cc.iy = cc.iz = -4;  // no cell yet
                // the clamped head [0, ka)
                if (march<true, MODE, SHW_TRILINEAR>(s, s, a, st, cc, cc, X, Y, Z, r.D[0], r.D[1], r.D[2], 0, ka,
                                                     done))
                    live = false;
                k = ka;
            }
        } else if (h.type == kStageSlab) {
            if (live && k < kb) {
                const raw *stg = reinterpret_cast<const raw *>(stages + (size_t)si * kSlabStageBytes);
                const long long DX = r.D[0], DY = r.D[1], DZ = r.D[2];
                bool stop;
                using G = SlabGeom<EP>;
#define SHW_SLAB_MARCH(MM, FF, BB) \
    stop = slab_march<MODE, EP, MM, FF, BB>(s, a, st, X, Y, Z, DX, DY, DZ, k, kb, h, stg)
                if (a.filter == SHW_FILTER_NONE) {  // the chunk width as a compile-time pitch
                    if (h.major == 0) SHW_SLAB_MARCH(0, false, G::kBXx);
                    else if (h.major == 1) {
                        if (h.wide) SHW_SLAB_MARCH(1, false, G::kBXw);
                        else SHW_SLAB_MARCH(1, false, G::kBXn);
                    } else {
                        if (h.wide) SHW_SLAB_MARCH(2, false, G::kBXw);
                        else SHW_SLAB_MARCH(2, false, G::kBXn);
                    }
                } else {
                    if (h.major == 0) SHW_SLAB_MARCH(0, true, 0);
                    else if (h.major == 1) SHW_SLAB_MARCH(1, true, 0);
                    else SHW_SLAB_MARCH(2, true, 0);
                }
#undef SHW_SLAB_MARCH
                if (stop) {
                    live = false;
                    done = k;
                }
            }
        } else if (has) {  // the tile's end
            if (live) {
                bool stop = false;
                if (k < kb) {  // interior samples no slab held
                    stop = march_interior<MODE>(s, s, a, st, X, Y, Z, r.D[0], r.D[1], r.D[2], k, kb, done);
                    cc.ix = -4;
                }
                // the clamped tail [kb, N)
                if (!stop) march<true, MODE, SHW_TRILINEAR>(s, s, a, st, cc, cc, X, Y, Z, r.D[0], r.D[1], r.D[2], kb,
                                                            N, done);
                live = false;
            }
            if (N <= 0) r.P[0] = r.P[1] = r.P[2] = r.D[0] = r.D[1] = r.D[2] = 0;
            emit_ray<MODE, SHW_TRILINEAR>(a, pix, N, r.P, r.D, st, done);
            has = false;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.empty[si]);
    }
}

// Persistent CTAs: a producer warp and kSlabWarps consumer warps; the ring of stages,
// their headers and barriers in dynamic shared memory.
// The tensor maps of one launch: x-major chunks; y-major narrow and wide; z-major narrow and wide.
struct SlabMaps {
    CUtensorMap m[5];
};

template <int MODE, class EP, class S>
__global__ void __launch_bounds__(kSlabThreads, kSlabMinBlocks)
    slab_kernel(const __grid_constant__ SlabMaps maps, S s, shw_camera cam, RenderArgs a, SlabArgs sa)
{
    extern __shared__ __align__(128) unsigned char slab_smem[];
    unsigned char *stages = slab_smem;
    SlabShared &sh = *reinterpret_cast<SlabShared *>(slab_smem + (size_t)kSlabStages * kSlabStageBytes);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kSlabStages; ++i) {
            mbar_init(&sh.full[i], 1);
            mbar_init(&sh.empty[i], kSlabWarps);
        }
        sh.quit = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if ((threadIdx.x >> 5) == kSlabWarps)
        slab_producer<EP>(maps.m, cam, a, sa, stages, sh);
    else
        slab_consumer<MODE, EP>(s, cam, a, sa, stages, sh);
}

constexpr size_t kSlabSmemBytes = (size_t)kSlabStages * kSlabStageBytes + sizeof(SlabShared);

// ---- host side ---------------------------------------------------------------------

// One mode's launch: persistent CTAs, as many as fit on the device at once (at most one per tile).
template <int MODE, class EP, class S>
shw_status slab_launch_one(const SlabMaps &maps, const S &s, const shw_camera &cam, const RenderArgs &a,
                           const SlabArgs &sa, cudaStream_t st)
{
    auto kern = slab_kernel<MODE, EP, S>;
    static int per_sm = -1;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemBytes) != cudaSuccess) {
        cudaGetLastError();
        return SHW_ECUDA;
    }
    if (per_sm < 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kSlabThreads, kSlabSmemBytes) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        per_sm = n;
    }
    const int nsm = sm_count();
    if (per_sm <= 0 || nsm <= 0) return SHW_ECUDA;
    const long long grid = std::min<long long>((long long)per_sm * nsm, sa.ntiles);
    kern<<<(unsigned)std::max<long long>(grid, 1), kSlabThreads, kSlabSmemBytes, st>>>(maps, s, cam, a, sa);
    return after_launch();
}

// The launch for one storage: the tensor maps (x-major chunks; y- and z-major chunks, narrow
// and wide), the tile order and counter, then the mode's kernel.  SHW_EUNSUPPORTED if the
// driver refuses a map.
template <class EP, class S>
shw_status slab_launch(int mode, const S &s, const void *base, const shw_camera &cam, const RenderArgs &a0,
                       cudaStream_t st)
{
    using G = SlabGeom<EP>;
    SlabMaps maps;
    if (!encode_tmap_3d(&maps.m[0], base, G::kBytes, s.nx, s.ny, s.nz, G::kBXx, kSlabRows, 1) ||
        !encode_tmap_3d(&maps.m[1], base, G::kBytes, s.nx, s.ny, s.nz, G::kBXn, 1, kSlabRows) ||
        !encode_tmap_3d(&maps.m[2], base, G::kBytes, s.nx, s.ny, s.nz, G::kBXw, 1, kSlabRows) ||
        !encode_tmap_3d(&maps.m[3], base, G::kBytes, s.nx, s.ny, s.nz, G::kBXn, kSlabRows, 1) ||
        !encode_tmap_3d(&maps.m[4], base, G::kBytes, s.nx, s.ny, s.nz, G::kBXw, kSlabRows, 1))
        return SHW_EUNSUPPORTED;
    RenderArgs a = a0;
    a.tiles_x = ceil_div(cam.width, kSlabTW);
    a.tiles_y = ceil_div(cam.height, kSlabTH);
    float cpx, cpy;
    project_centre(cam, s.nx, s.ny, s.nz, cpx, cpy);
    a.ctx = (int)fminf(fmaxf(cpx / kSlabTW, 0.0f), (float)(a.tiles_x - 1));
    a.cty = (int)fminf(fmaxf(cpy / kSlabTH, 0.0f), (float)(a.tiles_y - 1));
    SlabArgs sa;
    sa.ntiles = a.tiles_x * a.tiles_y;
    sa.err = device_error_word();
    sa.polls = kSlabWaitPolls;
    sa.ctr = work_counter(st);
    if (!sa.ctr) return SHW_ECUDA;
    if constexpr (EP::kPair) {
        switch (mode) {
        case SHW_RATIO: return slab_launch_one<SHW_RATIO, EP>(maps, s, cam, a, sa, st);
        case SHW_RATIO_MIP: return slab_launch_one<SHW_RATIO_MIP, EP>(maps, s, cam, a, sa, st);
        default: return SHW_EUNSUPPORTED;
        }
    } else {
        switch (mode) {
        case SHW_MIP:
            // without a channel output only the maximum's value matters
            if (a.index == nullptr) return slab_launch_one<kMipValue, EP>(maps, s, cam, a, sa, st);
            return slab_launch_one<SHW_MIP, EP>(maps, s, cam, a, sa, st);
        case SHW_AVG: return slab_launch_one<SHW_AVG, EP>(maps, s, cam, a, sa, st);
        case SHW_COMPOSITE: return slab_launch_one<SHW_COMPOSITE, EP>(maps, s, cam, a, sa, st);
        case SHW_SPECTRAL: return slab_launch_one<SHW_SPECTRAL, EP>(maps, s, cam, a, sa, st);
        case SHW_MOMENT1: return slab_launch_one<SHW_MOMENT1, EP>(maps, s, cam, a, sa, st);
        case SHW_COMPOSITE_SPECTRAL: return slab_launch_one<SHW_COMPOSITE_SPECTRAL, EP>(maps, s, cam, a, sa, st);
        case SHW_MIP_RGB: return slab_launch_one<SHW_MIP_RGB, EP>(maps, s, cam, a, sa, st);
        case SHW_COMPOSITE_RGB: return slab_launch_one<SHW_COMPOSITE_RGB, EP>(maps, s, cam, a, sa, st);
        default: return SHW_EUNSUPPORTED;
        }
    }
}

// host: the staged marcher (render_slab.cu); SHW_EUNSUPPORTED when the request is not one
// it serves: not trilinear, in-ray smoothing, a line ratio on two separate cubes, a storage
// it does not read, x rows that are not 16-byte multiples, 2^31 voxels or more.
shw_status render_slab(int mode, int interp, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                       cudaStream_t st);
// the linear 16-bit storages (render_slab_h16.cu)
shw_status render_slab_h16(int mode, const shw_volume &v, const shw_camera &cam, const RenderArgs &a,
                           cudaStream_t st);

}  // namespace shw
