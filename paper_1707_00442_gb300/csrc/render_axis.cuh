// render_axis.cuh -- orthographic views down the spectral axis as a plane sweep.
//
// A parallel ray down z is a spectrum: this view is the moment-map view of
// Section 2.2 (Eq. 3 is its zeroth moment).  All its rays take their samples at
// the same z, so a CTA sweeps the cube plane by plane for a 64 x 16 pixel tile:
//   - one producer thread stages the tile's footprint of each z plane into shared
//     memory with cp.async.bulk.tensor, through a ring of stages, a group of planes
//     (stages) per "full" and "empty" mbarrier phase (AxRing; every wait bounded);
//   - 16 consumer warps own two rays per thread, as a pair; each ray turns each plane
//     into one bilinear value (4 shared loads), in the same order of operations as the
//     general trilinear interpolation, and each warp releases the group's stages;
//   - the samples that fall between two planes (the same for every ray) are one
//     lerp each, fed to the same transfer-function state as the general marcher.
// When the step is exactly 1/Q voxel every interior cell holds Q samples at the same
// fractions, and runs of cells go through a loop unrolled over the ring, so stage
// addresses and barrier phases are compile-time constants.
// The cube is read from HBM about once, in coalesced boxes, and the results are
// bit-identical to the general marcher's.
#pragma once

#include <cmath>
#include <type_traits>

#include "render_impl.cuh"
#include "tma.cuh"

namespace shw {

constexpr int kAxTX = 64, kAxTY = 16;  // pixel tile of one CTA
constexpr int kAxSmemLimit = 100 * 1024;
constexpr int kAxMaxQ = 4;  // periodic stepping: at most this many samples per cell

// The ring: `stages` plane buffers, consumed in groups of `group` planes that complete on one
// barrier phase (each consumer warp waits and releases once per group).  A plane's fixed
// chain in each warp (wait, loads, dependent lerps, release) bounded the sweep, so the
// fixed box, whose 16 stages fit the shared-memory budget, takes groups of 8 (MIP of the
// 1 GiB cube 0.386 ms with one plane per phase, 0.261 ms with eight); the first moment, whose
// per-sample work is longest, does best with groups of 4 of 8 stages, as do runtime-sized boxes.
template <int MODE, bool FIX>
struct AxRing {
    static constexpr bool kDeep = FIX && MODE != SHW_MOMENT1;
    static constexpr int stages = kDeep ? 16 : 8, group = kDeep ? 8 : 4;
    static_assert((stages & (stages - 1)) == 0 && (group & (group - 1)) == 0 && stages % group == 0,
                  "groups tile a power-of-two ring");
};
// host: the stages of the kernel a request takes
inline int axis_stages(int mode, bool fix) { return (fix && mode != SHW_MOMENT1) ? 16 : 8; }

// W consumer warps share the tile's 16 rows: each thread owns 32 / W rays, in pairs (one row
// each, the pair's rays 32 columns apart), plus one producer warp.  Sixteen warps of two rays
// hide more of each warp's per-plane chain (wait, loads, dependent lerps) than eight warps of
// four, for every mode.
template <int W>
struct AxCfg {
    static constexpr int warps = W, pairs = kAxTY / W, rays = 2 * pairs, threads = 32 * (W + 1);
    static_assert(W * pairs == kAxTY, "the warps split the tile's rows evenly");
};
template <int MODE>
constexpr int axis_warps()
{
    return 16;
}

// The fixed staged box: enough for a 64 x 16 tile at up to one voxel per pixel,
// axis-aligned (extent 63 x 15, plus the alignment and rounding margins).
// fixed box: a 64 x kAxTY tile at up to one voxel per pixel, plus the margins of render_axis
constexpr int kFixBW = 72, kFixBH = kAxTY + 5;
constexpr int kFixStride = (kFixBW * kFixBH + 31) & ~31;  // floats per stage, 128-byte multiple

// bounded waits that sleep between polls: kAxWaitPolls x kAxSleepNs is about a second
constexpr int kAxWaitPolls = 1 << 20;
constexpr uint32_t kAxSleepNs = 1000;

template <int MODE>
struct AxisStateOf {
    using type = typename StateOf<MODE>::type;
};
template <>
struct AxisStateOf<kMipValue> {
    using type = MaxValState;
};

struct AxisArgs {
    int bw, bh;        // staged box per plane, elements (bw a multiple of 4)
    int stage_stride;  // floats from one stage to the next: bw * bh rounded up to 32 (128 bytes)
    int nx, ny, nz;
    int tiles_x;
    float cx, ax, bx;  // pixel (px, py) -> x = cx + ax px + bx py (FP32, for the box only)
    float cy, ay, by;
    unsigned *err;
};

__device__ __forceinline__ float bilerp(float v00, float v01, float v10, float v11, float fx, float fy)
{
    return lerp(lerp(v00, v01, fx), lerp(v10, v11, fx), fy);
}

// the float `off` bytes past p
__device__ __forceinline__ float at(const char *p, int off) { return *reinterpret_cast<const float *>(p + off); }

// b - a per lane as one packed FMA (a * -1 + b rounds once, like the subtraction)
__device__ __forceinline__ float2 sub2(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.0f, -1.0f), b); }

// lerp of two independent pairs with their own weights (packed FP32x2, same rounding)
__device__ __forceinline__ float2 lerp2v(float2 a, float2 b, float2 t) { return __ffma2_rn(t, sub2(b, a), a); }

// ray i of consumer thread (lane, warp): pair i / 2 is one row, its two rays 32 columns apart
__device__ __forceinline__ int ray_px(int txi, int lane, int i) { return txi * kAxTX + lane + 32 * (i & 1); }
template <int P>
__device__ __forceinline__ int ray_py(int tyi, int warp, int i)
{
    return tyi * kAxTY + P * warp + (i >> 1);
}

template <int MODE, class St>
__device__ __forceinline__ void axis_emit(const RenderArgs &a, long long pix, bool hit, int N, long long PZ,
                                          long long DZ, bool nearest, const St &st, int done)
{
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float scalar = 0.0f;
    int index = -1;
    if (hit) {
        if constexpr (MODE == SHW_MIP || MODE == kMipValue || MODE == SHW_SPECTRAL) {
            const long long Zm = PZ + (long long)st.kmax * DZ;
            index = clampi(fx_round(Zm), 0, a.nz - 1);
            scalar = st.m;
            const float vh = normalise(st.m, a.lo, a.inv_range);
            if constexpr (MODE == SHW_SPECTRAL) {
                const float zmax = nearest ? (float)index : __ll2float_rn(Zm) * 2.3283064365386963e-10f;
                const float tz = __saturatef((zmax + 0.5f) / (float)a.nz);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, colour_alpha(st.m, a));
            } else {
                out = lut_eval(a.lut, vh);
            }
        } else if constexpr (MODE == SHW_AVG) {
            scalar = __fdiv_rn(st.sum, (float)N);
            out = lut_eval(a.lut, normalise(scalar, a.lo, a.inv_range));
        } else if constexpr (MODE == SHW_MOMENT1) {
            if (st.sw > 0.0f) {
                const float m1 = __fdiv_rn(st.szw, st.sw);
                scalar = m1;
                index = clampi(__float2int_rd(m1 + 0.5f), 0, a.nz - 1);
                const float tz = __saturatef((m1 + 0.5f) / (float)a.nz);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, colour_alpha(__fdiv_rn(st.sv, (float)N), a));
            }
        } else {
            out = make_float4(st.cr, st.cg, st.cb, 1.0f - st.T);
            scalar = 1.0f - st.T;
        }
    } else {
        done = 0;
    }
    if constexpr (MODE == SHW_COMPOSITE)
        if (a.ckpt_K != nullptr) a.ckpt_K[pix] = done;
    a.rgba[pix] = out;
    if (a.scalar) a.scalar[pix] = scalar;
    if (a.index) a.index[pix] = index;
    if (a.nsamples) a.nsamples[pix] = done;
}

// MODE: a transfer function, or kMipValue.  UP: rays advance towards +z.  FIX: the
// staged box is kFixBW x kFixBH (else A.bw x A.bh).  W: consumer warps.
template <int MODE, int INTERP, bool UP, bool FIX, int W = axis_warps<MODE>()>
__global__ void __launch_bounds__(AxCfg<W>::threads, MODE == SHW_COMPOSITE ? 1 : 2)
    axis_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ vol, shw_camera cam, RenderArgs a,
                AxisArgs A)
{
    constexpr int R = AxCfg<W>::rays, P = AxCfg<W>::pairs;
    constexpr int S = AxRing<MODE, FIX>::stages, G = AxRing<MODE, FIX>::group;
    extern __shared__ __align__(128) float sm[];  // [stages][bh][bw]
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ long long s_pz, s_dz;
    __shared__ int s_n, s_any, s_x0, s_y0, s_bad, s_nidle;
    __shared__ volatile int s_quit;  // 1: every ray has stopped, or a wait gave up

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool consumer = warp < W;
    const int tile = blockIdx.x, tyi = tile / A.tiles_x, txi = tile - tyi * A.tiles_x;
    const int bw = FIX ? kFixBW : A.bw, bh = FIX ? kFixBH : A.bh;
    const int stride = FIX ? kFixStride : A.stage_stride;

    if (tid == 0) {
        s_any = 0;
        s_nidle = 0;
        s_quit = 0;
        // staged box: the tile's footprint widened by 2 voxels, x start 16-byte aligned
        const float qx0 = (float)(txi * kAxTX), qx1 = (float)min(txi * kAxTX + kAxTX - 1, a.width - 1);
        const float qy0 = (float)(tyi * kAxTY), qy1 = (float)min(tyi * kAxTY + kAxTY - 1, a.height - 1);
        float xmin = INFINITY, ymin = INFINITY;
        for (int c = 0; c < 4; ++c) {
            const float qx = (c & 1) ? qx1 : qx0, qy = (c & 2) ? qy1 : qy0;
            xmin = fminf(xmin, A.cx + A.ax * qx + A.bx * qy);
            ymin = fminf(ymin, A.cy + A.ay * qx + A.by * qy);
        }
        s_x0 = ((int)floorf(xmin) - 2) & ~3;
        s_y0 = (int)floorf(ymin) - 2;
        s_bad = 0;
        for (int s = 0; s < S; ++s) s_bad |= !tma_dst_ok(sm + s * stride, A.err);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_barrier_init();
    }

    // the consumer's rays; every ray that meets the cube shares one z sequence
    long long X[R], Y[R];
    int hitmask = 0, N = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        X[i] = Y[i] = 0;
        const int px = ray_px(txi, lane, i), py = ray_py<P>(tyi, warp, i);
        RayFx r;
        if (consumer && px < a.width && py < a.height && setup_ray(cam, px, py, A.nx, A.ny, A.nz, a.step, r) &&
            min(r.N, a.nmax) > 0) {
            hitmask |= 1 << i;
            N = min(r.N, a.nmax);
            X[i] = r.P[0];
            Y[i] = r.P[1];
            if ((hitmask & ((1 << i) - 1)) == 0) {
                s_pz = r.P[2];  // every hit writes the same values (plain stores, any winner)
                s_dz = r.D[2];
            }
        }
    }
    __syncthreads();
    if (hitmask != 0) {
        s_n = N;
        s_any = 1;
    }
    __syncthreads();
    if (s_bad) return;  // reported in the error word; nothing was issued
    if (s_any == 0) {   // no ray of this tile meets the cube
        if (consumer)
            for (int i = 0; i < R; ++i) {
                const int px = ray_px(txi, lane, i), py = ray_py<P>(tyi, warp, i);
                if (px < a.width && py < a.height)
                    axis_emit<MODE>(a, (long long)py * a.width + px, false, 0, 0, 0, INTERP == SHW_NEAREST,
                                    typename AxisStateOf<MODE>::type{}, 0);
            }
        return;
    }
    const int NS = s_n;
    const long long PZ = s_pz, DZ = s_dz;
    const int x0b = s_x0, y0b = s_y0;

    // the planes in the order the sweep needs them
    const int nz = A.nz;
    const int cz_first = clampi(fx_cell(PZ), -1, nz - 1);
    const int cz_last = clampi(fx_cell(PZ + (long long)(NS - 1) * DZ), -1, nz - 1);
    const int p_first = UP ? max(cz_first, 0) : min(cz_first + 1, nz - 1);
    const int p_last = UP ? min(cz_last + 1, nz - 1) : max(cz_last, 0);
    const int nplanes = (UP ? p_last - p_first : p_first - p_last) + 1;

    if (!consumer) {
        // producer: one thread keeps the ring full, a group of G planes at a time -- planes
        // j .. j + G - 1 (j a multiple of G) go to stages s .. s + G - 1 and complete on stage
        // s's barrier, so each consumer warp waits and releases once per group
        if (lane != 0) return;
        const uint32_t plane_bytes = (uint32_t)(bw * bh * 4);
        int issued = 0;
        for (int j = 0; j < nplanes; j += G) {
            const int s = j & (S - 1);
            if (j >= S) {  // wait until every consumer warp has released the group j - S
                const uint32_t par = (uint32_t)(((j / S) - 1) & 1);
                bool ok = false, quit = false;
                for (int it = 0; it < kAxWaitPolls && !ok && !quit; ++it) {
                    ok = mbar_try_wait_sleep(&empty[s], par, kAxSleepNs);
                    quit = !ok && s_quit != 0;
                }
                if (!ok) {
                    if (!quit) {
                        atomicOr(A.err, kErrWaitTimeout);
                        s_quit = 1;
                    }
                    break;
                }
            }
            const int cnt = min(G, nplanes - j);
            mbar_arrive_expect_tx(&full[s], (uint32_t)cnt * plane_bytes);
            for (int e = 0; e < cnt; ++e) {
                int pz = UP ? p_first + j + e : p_first - j - e;
                check_range(pz, 0, nz - 1);
                tma_load_3d(sm + (s + e) * stride, &tmap, x0b, y0b, pz, &full[s]);
            }
            issued = j + cnt;
        }
        // every copy issued lands before this CTA may exit (the groups still in the ring)
        for (int j = (max(issued - S, 0) + G - 1) & ~(G - 1); j < issued; j += G)
            mbar_wait(&full[j & (S - 1)], (uint32_t)((j / S) & 1), A.err);
        return;
    }

    // consumer: byte offsets of each ray's corners in the staged box, or in the global
    // plane for a ray outside the box (a ray that misses the cube reads stage element 0)
    int o00[R], o01[R], o10[R], o11[R], inbox = 0;
    float2 fx2[P], fy2[P];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ix = clampi(fx_cell(X[i]), -1, A.nx - 1), iy = clampi(fx_cell(Y[i]), -1, A.ny - 1);
        int gx0 = max(ix, 0), gx1 = min(ix + 1, A.nx - 1), gy0 = max(iy, 0), gy1 = min(iy + 1, A.ny - 1);
        if constexpr (INTERP == SHW_NEAREST) {
            gx0 = gx1 = clampi(fx_round(X[i]), 0, A.nx - 1);
            gy0 = gy1 = clampi(fx_round(Y[i]), 0, A.ny - 1);
        }
        if (i & 1) {
            fx2[i >> 1].y = fx_frac(X[i]);
            fy2[i >> 1].y = fx_frac(Y[i]);
        } else {
            fx2[i >> 1].x = fx_frac(X[i]);
            fy2[i >> 1].x = fx_frac(Y[i]);
        }
        const int c0 = gx0 - x0b, c1 = gx1 - x0b, r0 = gy0 - y0b, r1 = gy1 - y0b;
        if (!((hitmask >> i) & 1)) {
            inbox |= 1 << i;
            o00[i] = o01[i] = o10[i] = o11[i] = 0;
        } else if (c0 >= 0 && c1 < bw && r0 >= 0 && r1 < bh) {
            inbox |= 1 << i;
            o00[i] = 4 * (r0 * bw + c0);
            o01[i] = 4 * (r0 * bw + c1);
            o10[i] = 4 * (r1 * bw + c0);
            o11[i] = 4 * (r1 * bw + c1);
        } else {
            o00[i] = 4 * (gy0 * A.nx + gx0);
            o01[i] = 4 * (gy0 * A.nx + gx1);
            o10[i] = 4 * (gy1 * A.nx + gx0);
            o11[i] = 4 * (gy1 * A.nx + gx1);
        }
    }
    if constexpr (kChecked) {  // every offset inside the staged box, or inside the plane
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const long long lim = ((inbox >> i) & 1) ? 4ll * bw * bh : 4ll * A.nx * A.ny;
            const int lo = min(min(o00[i], o01[i]), min(o10[i], o11[i]));
            const int hi = max(max(o00[i], o01[i]), max(o10[i], o11[i]));
            const bool ok = lo >= 0 && (long long)hi + 4 <= lim;
            SHW_CHECK(ok);
            if (!ok) o00[i] = o01[i] = o10[i] = o11[i] = 0;
        }
    }
    const bool all_inbox = inbox == (1 << R) - 1;
    const size_t plane_elems = (size_t)A.nx * A.ny;

    // wait until stage s holds its next plane (phase parity ph); false if the sweep must
    // end.  The result is the same on every lane of the warp.
    auto wait_full = [&](int s, uint32_t ph) -> bool {
        bool ok = __all_sync(0xffffffffu, mbar_try_wait_sleep(&full[s], ph, kAxSleepNs));
        for (int it = 1; !ok && it < kAxWaitPolls; ++it) {
            if (__any_sync(0xffffffffu, s_quit != 0)) return false;
            ok = __all_sync(0xffffffffu, mbar_try_wait_sleep(&full[s], ph, kAxSleepNs));
        }
        if (!ok) {
            if (lane == 0) atomicOr(A.err, kErrWaitTimeout);
            s_quit = 1;
        }
        return ok;
    };
    // one plane's value for each ray pair (bilinear, or the nearest voxel) from stage s,
    // which holds the sweep's plane jp
    auto load_plane = [&](int s, int jp, float2 pv[P]) {
        const char *t = reinterpret_cast<const char *>(sm + s * stride);
        if (all_inbox) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int u = 2 * q, w = 2 * q + 1;
                if constexpr (INTERP == SHW_NEAREST) {
                    pv[q] = make_float2(at(t, o00[u]), at(t, o00[w]));
                } else {
                    // x first on rows y0 and y1, then y: the general interpolation's order
                    const float2 r0 = lerp2v(make_float2(at(t, o00[u]), at(t, o00[w])),
                                             make_float2(at(t, o01[u]), at(t, o01[w])), fx2[q]);
                    const float2 r1 = lerp2v(make_float2(at(t, o10[u]), at(t, o10[w])),
                                             make_float2(at(t, o11[u]), at(t, o11[w])), fx2[q]);
                    pv[q] = lerp2v(r0, r1, fy2[q]);
                }
            }
        } else {
            int pz = UP ? p_first + jp : p_first - jp;
            check_range(pz, 0, A.nz - 1);
            const char *g = reinterpret_cast<const char *>(vol + (size_t)pz * plane_elems);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const char *b = ((inbox >> i) & 1) ? t : g;
                const float fxi = (i & 1) ? fx2[i >> 1].y : fx2[i >> 1].x;
                const float fyi = (i & 1) ? fy2[i >> 1].y : fy2[i >> 1].x;
                float v;
                if constexpr (INTERP == SHW_NEAREST)
                    v = at(b, o00[i]);
                else
                    v = bilerp(at(b, o00[i]), at(b, o01[i]), at(b, o10[i]), at(b, o11[i]), fxi, fyi);
                if (i & 1)
                    pv[i >> 1].y = v;
                else
                    pv[i >> 1].x = v;
            }
        }
    };
    // hand stage s back to the producer once the whole warp has read it
    auto release = [&](int s) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    };

    typename AxisStateOf<MODE>::type st[R];
    int done[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        done[i] = NS;
        if constexpr (MODE == SHW_COMPOSITE) {
            const long long pix = (long long)ray_py<P>(tyi, warp, i) * a.width + ray_px(txi, lane, i);
            st[i].lut = a.lut;
            st[i].lo = a.lo;
            st[i].inv_range = a.inv_range;
            st[i].s = a.opacity_scale;
            st[i].term = a.term_alpha;
            st[i].ckpt = (a.ckpt_T != nullptr && ((hitmask >> i) & 1)) ? a.ckpt_T + pix : nullptr;
            st[i].ckpt_stride = (long long)a.width * a.height;
            st[i].I = a.ckpt_interval;
            st[i].nckpt = a.nckpt;
        }
        if constexpr (MODE == SHW_MOMENT1) {
            st[i].Z = PZ;
            st[i].DZ = DZ;
            st[i].lo = a.lo;
            st[i].nz = a.nz;
            st[i].nearest = INTERP == SHW_NEAREST;
        }
    }
    // COMPOSITE: rays still taking samples (a ray that misses counts as stopped)
    int live = hitmask;
    bool idle = __all_sync(0xffffffffu, hitmask == 0);
    if (idle && lane == 0 && atomicAdd(&s_nidle, 1) + 1 == W) s_quit = 1;
    // COMPOSITE: every 16 cells a warp whose rays have all stopped turns idle; when the
    // last warp does, the sweep ends
    int ncell = 0;
    auto after_cells = [&](int n) {
        if constexpr (MODE == SHW_COMPOSITE) {
            ncell += n;
            if (!idle && ncell >= 16) {
                ncell = 0;
                idle = __all_sync(0xffffffffu, live == 0);
                if (idle && lane == 0 && atomicAdd(&s_nidle, 1) + 1 == W) s_quit = 1;
            }
        }
    };

    // sample k of both rays of pair q, values v2 (NANCHK: NaN counts as DATAMIN)
    auto take2 = [&](int q, float2 v2, int k, auto nanchk) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = 2 * q + e;
            float v = e ? v2.y : v2.x;
            if (decltype(nanchk)::value) v = isnan(v) ? a.lo : v;
            if constexpr (MODE == SHW_COMPOSITE) {
                if (((live >> i) & 1) && st[i].update(v, k)) {
                    live &= ~(1 << i);
                    done[i] = k + 1;
                }
            } else {
                st[i].update(v, k);
            }
        }
    };
    using NanCheck = std::integral_constant<bool, true>;
    using NoNanCheck = std::integral_constant<bool, false>;
    // the value of a pair at fraction f (f2 = (f, f)) between its planes: lo2 and
    // d2 = hi - lo (nearest: d2 holds hi, and floor(z + 1/2) is the upper plane iff
    // frac >= 1/2)
    auto value2p = [&](float2 f2, float2 lo2, float2 d2) -> float2 {
        if constexpr (INTERP == SHW_NEAREST)
            return (f2.x >= 0.5f) ? d2 : lo2;
        else
            return __ffma2_rn(f2, d2, lo2);  // lerp(lo, hi, f) per ray
    };
    auto value2 = [&](float f, float2 lo2, float2 d2) -> float2 { return value2p(make_float2(f, f), lo2, d2); };
    // lo2 and d2 of every pair from the near (held) and far plane values; true if no
    // sample between them can be NaN
    auto setup_cell = [&](const float2 va_[P], const float2 vb_[P], float2 lo2[P], float2 d2[P]) -> bool {
        bool finite = true;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            lo2[q] = UP ? va_[q] : vb_[q];
            const float2 hi2 = UP ? vb_[q] : va_[q];
            if constexpr (INTERP == SHW_NEAREST) {
                d2[q] = hi2;
                finite = finite && !isnan(lo2[q].x) && !isnan(lo2[q].y) && !isnan(hi2.x) && !isnan(hi2.y);
            } else {
                d2[q] = sub2(hi2, lo2[q]);
                // hi - lo finite: both ends finite and every lerp between them finite
                finite = finite && fabsf(d2[q].x) < INFINITY && fabsf(d2[q].y) < INFINITY;
            }
        }
        return finite;
    };
    // the QQ samples k0 .. k0 + QQ - 1 of one interior cell, at fractions fq2 (each
    // duplicated into both lanes of a pair)
    auto cell_q = [&](const float2 va_[P], const float2 vb_[P], int k0, auto QC, const float2 fq2[kAxMaxQ]) {
        constexpr int QQ = decltype(QC)::value;
        float2 lo2[P], d2[P];
        if (setup_cell(va_, vb_, lo2, d2)) {
#pragma unroll
            for (int s = 0; s < QQ; ++s)
#pragma unroll
                for (int q = 0; q < P; ++q) take2(q, value2p(fq2[s], lo2[q], d2[q]), k0 + s, NoNanCheck{});
        } else {
#pragma unroll
            for (int s = 0; s < QQ; ++s)
#pragma unroll
                for (int q = 0; q < P; ++q) take2(q, value2p(fq2[s], lo2[q], d2[q]), k0 + s, NanCheck{});
        }
    };

    // planes consumed: plane j sits in stage j % S; the group of G planes from j (a multiple
    // of G) completes on stage j % S's barrier (phase parity (j / S) % 2), waited for at its
    // first plane and released after its last
    int j = 0;
    float2 va[P];  // values of the plane held (the near plane of the current cell)
#pragma unroll
    for (int q = 0; q < P; ++q) va[q] = make_float2(0.0f, 0.0f);
    bool alive = wait_full(0, 0u);
    if (alive) {
        if (!idle) load_plane(0, 0, va);
        j = 1;
    }
    // one more plane (the far plane of the current cell) through the ring, any stage
    auto next_plane = [&](float2 vb[P]) -> bool {
        const int s = j & (S - 1);
        if ((j & (G - 1)) == 0 && !wait_full(s, (uint32_t)((j / S) & 1))) return false;
        if (!idle) load_plane(s, j, vb);
        if ((j & (G - 1)) == G - 1) release(s - (G - 1));
        ++j;
        return true;
    };

    const long long zend = PZ + (long long)NS * DZ;  // Z just past the last sample
    // periodic stepping: a step of exactly 1/Q voxel (Q <= kAxMaxQ) puts Q samples in
    // every cell, at the same fractions in every cell
    const long long adz = UP ? DZ : -DZ;
    const int Q = (adz > 0 && ((1ll << 32) % adz) == 0 && (1ll << 32) / adz <= kAxMaxQ) ? (int)((1ll << 32) / adz)
                                                                                        : 0;
    long long Z = PZ;
    int k = 0, c = cz_first, held = p_first;
    // nb interior cells of QQ samples each, starting with cell c at sample k
    auto run_cells = [&](auto QC, int nb) {
        constexpr int QQ = decltype(QC)::value;
        float2 fq2[kAxMaxQ];
#pragma unroll
        for (int s = 0; s < kAxMaxQ; ++s) {
            const float f = fx_frac(Z + (long long)s * DZ);
            fq2[s] = make_float2(f, f);
        }
        while (nb > 0 && alive) {
            // (compositing keeps the plain loop: its per-sample work dwarfs the ring
            // bookkeeping, and unrolling it costs occupancy)
            if (MODE != SHW_COMPOSITE && (j & (S - 1)) == 0 && nb >= S) {
                // a whole turn of the ring: stages 0 .. S-1 in order
                const uint32_t ph = (uint32_t)((j / S) & 1);
#pragma unroll
                for (int u = 0; u < S; ++u) {
                    float2 vb[P];
                    if ((u & (G - 1)) == 0 && !wait_full(u, ph)) {
                        alive = false;
                        break;
                    }
                    if (!idle) load_plane(u, j + u, vb);
                    if ((u & (G - 1)) == G - 1) release(u - (G - 1));
                    if (!idle) cell_q(va, vb, k + u * QQ, QC, fq2);
#pragma unroll
                    for (int q = 0; q < P; ++q) va[q] = vb[q];
                }
                if (!alive) break;
                j += S;
                nb -= S;
                k += S * QQ;
                c += UP ? S : -S;
                after_cells(S);
            } else {
                float2 vb[P];
                if (!next_plane(vb)) {
                    alive = false;
                    break;
                }
                if (!idle) cell_q(va, vb, k, QC, fq2);
#pragma unroll
                for (int q = 0; q < P; ++q) va[q] = vb[q];
                --nb;
                k += QQ;
                c += UP ? 1 : -1;
                after_cells(1);
            }
            if (MODE == SHW_COMPOSITE && idle && s_quit != 0) alive = false;  // the sweep is over
        }
        Z = PZ + (long long)k * DZ;
        held = UP ? c : c + 1;  // the far plane of the last cell of the run
    };
    while (alive && k < NS) {
        // a run of interior cells (planes c and c + 1 both in the cube), each entered at
        // its first sample and holding Q samples before the end
        if (Q > 0 && c != cz_first && c >= 0 && c <= nz - 2) {
            const int nb = min(UP ? nz - 1 - c : c + 1, (NS - k) / Q);
            if (nb > 0) {
                if (Q == 2)
                    run_cells(std::integral_constant<int, 2>{}, nb);
                else if (Q == 1)
                    run_cells(std::integral_constant<int, 1>{}, nb);
                else  // Q divides 2^32: 4
                    run_cells(std::integral_constant<int, 4>{}, nb);
                continue;
            }
        }
        // one cell, sample by sample: planes max(c, 0) and min(c + 1, nz - 1); the far
        // one in sweep order
        const int far = UP ? min(c + 1, nz - 1) : max(c, 0);
        float2 vb[P];
#pragma unroll
        for (int q = 0; q < P; ++q) vb[q] = va[q];
        if (far != held) {
            if (!next_plane(vb)) break;
            held = far;
        }
        // the samples of cell c: Z below (c + 1) << 32 going up, at or above c << 32 going
        // down, and before zend
        long long zb;
        if (UP)
            zb = (c >= nz - 1) ? zend : min((long long)(c + 1) << 32, zend);
        else
            zb = (c < 0) ? zend + 1 : max((long long)c << 32, zend + 1);
        if (!idle) {
            float2 lo2[P], d2[P];
            setup_cell(va, vb, lo2, d2);
            for (; UP ? Z < zb : Z >= zb; Z += DZ, ++k) {
                const float f = fx_frac(Z);
#pragma unroll
                for (int q = 0; q < P; ++q) take2(q, value2(f, lo2[q], d2[q]), k, NanCheck{});
            }
        } else {
            // an idle warp only keeps releasing stages: skip the cell's samples
            for (; UP ? Z < zb : Z >= zb; Z += DZ) ++k;
        }
#pragma unroll
        for (int q = 0; q < P; ++q) va[q] = vb[q];
        c += UP ? 1 : -1;
        after_cells(1);
        if (MODE == SHW_COMPOSITE && idle && s_quit != 0) break;  // every warp is idle: the sweep is over
    }

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int px = ray_px(txi, lane, i), py = ray_py<P>(tyi, warp, i);
        if (px < a.width && py < a.height)
            axis_emit<MODE>(a, (long long)py * a.width + px, (hitmask >> i) & 1, N, PZ, DZ, INTERP == SHW_NEAREST,
                            st[i], done[i]);
    }
}

// Launch the sweep for one (mode, interp, direction); FIX selects the fixed box.
// mode may be kMipValue.  Returns SHW_EUNSUPPORTED for a mode it has no kernel for.
// Instantiated once per FIX, each in its own translation unit.
template <bool FIX>
shw_status launch_axis(int mode, int interp, bool up, const CUtensorMap &map, const float *data,
                       const shw_camera &c, const RenderArgs &a, const AxisArgs &A, unsigned grid, size_t smem,
                       cudaStream_t st)
{
#define SHW_AX(M, I, U)                                                                                 \
    do {                                                                                                \
        /* static + dynamic shared memory may pass the 48 KB default: always opt in */                \
        cudaFuncSetAttribute(axis_kernel<M, I, U, FIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)smem);                                                                \
        axis_kernel<M, I, U, FIX><<<grid, AxCfg<axis_warps<M>()>::threads, smem, st>>>(map, data, c, a, A);  \
    } while (0)
#define SHW_AXI(M, I)           \
    if (up) SHW_AX(M, I, true); \
    else SHW_AX(M, I, false);
#define SHW_AXC(M)                              \
    case M:                                     \
        if (interp == SHW_NEAREST) {            \
            SHW_AXI(M, SHW_NEAREST)             \
        } else {                                \
            SHW_AXI(M, SHW_TRILINEAR)           \
        }                                       \
        break;
    switch (mode) {
        SHW_AXC(kMipValue)
        SHW_AXC(SHW_MIP)
        SHW_AXC(SHW_AVG)
        SHW_AXC(SHW_COMPOSITE)
        SHW_AXC(SHW_SPECTRAL)
        SHW_AXC(SHW_MOMENT1)
    default:
        return SHW_EUNSUPPORTED;
    }
#undef SHW_AXC
#undef SHW_AXI
#undef SHW_AX
    return after_launch();
}

extern template shw_status launch_axis<true>(int, int, bool, const CUtensorMap &, const float *, const shw_camera &,
                                             const RenderArgs &, const AxisArgs &, unsigned, size_t, cudaStream_t);
extern template shw_status launch_axis<false>(int, int, bool, const CUtensorMap &, const float *, const shw_camera &,
                                              const RenderArgs &, const AxisArgs &, unsigned, size_t, cudaStream_t);

}  // namespace shw
