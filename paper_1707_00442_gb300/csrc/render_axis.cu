// render_axis.cu -- orthographic views down the spectral axis as a plane sweep.
//
// A parallel ray down z is a spectrum: this view is the moment-map view of
// Section 2.2 (Eq. 3 is its zeroth moment).  All its rays take their samples at
// the same z, so a CTA sweeps the cube plane by plane for a 64 x 16 pixel tile:
//   - one producer thread stages the tile's footprint of each z plane into shared
//     memory with cp.async.bulk.tensor, through a ring of stages with a "full" and an
//     "empty" mbarrier each (every wait bounded);
//   - eight consumer warps own four rays per thread; each ray turns each plane into
//     one bilinear value (4 shared loads), in the same order of operations as the
//     general trilinear interpolation, and releases the stage per warp;
//   - the samples that fall between two planes (the same for every ray) are one
//     lerp each, fed to the same transfer-function state as the general marcher.
// The cube is read from HBM about once, in coalesced boxes, and the results are
// bit-identical to the general marcher's.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "render_impl.cuh"
#include "tma.cuh"

namespace shw {

constexpr int kAxWarps = 8;                      // consumer warps
constexpr int kAxRays = 4;                       // rays per consumer thread
constexpr int kAxTX = 64, kAxTY = 2 * kAxWarps;  // pixel tile of one CTA
constexpr int kAxThreads = 32 * (kAxWarps + 1);  // consumers + one producer warp
constexpr int kAxMaxStages = 8;
constexpr int kAxSmemLimit = 96 * 1024;

struct AxisArgs {
    int bw, bh;        // staged box per plane, elements (bw a multiple of 4)
    int stage_stride;  // floats from one stage to the next: bw * bh rounded up to 32 (128 bytes)
    int stages;        // ring depth, 2..kAxMaxStages
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

// ray i of consumer thread (lane, warp): two columns 32 apart, two adjacent rows
__device__ __forceinline__ int ray_px(int txi, int lane, int i) { return txi * kAxTX + lane + 32 * (i & 1); }
__device__ __forceinline__ int ray_py(int tyi, int warp, int i) { return tyi * kAxTY + 2 * warp + (i >> 1); }

template <int MODE>
__device__ __forceinline__ void axis_emit(const RenderArgs &a, long long pix, bool hit, int N, long long PZ,
                                          long long DZ, int INTERP_NEAREST, const typename StateOf<MODE>::type &st,
                                          int done)
{
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    float scalar = 0.0f;
    int index = -1;
    if (hit) {
        if constexpr (MODE == SHW_MIP || MODE == SHW_SPECTRAL) {
            const long long Zm = PZ + (long long)st.kmax * DZ;
            index = clampi(fx_round(Zm), 0, a.nz - 1);
            scalar = st.m;
            const float vh = normalise(st.m, a.lo, a.inv_range);
            if constexpr (MODE == SHW_SPECTRAL) {
                const float zmax = INTERP_NEAREST ? (float)index : __ll2float_rn(Zm) * 2.3283064365386963e-10f;
                const float tz = fminf(fmaxf((zmax + 0.5f) / (float)a.nz, 0.0f), 1.0f);
                const float4 c = lut_eval(a.lut, tz);
                out = make_float4(c.x, c.y, c.z, vh);
            } else {
                out = lut_eval(a.lut, vh);
            }
        } else if constexpr (MODE == SHW_AVG) {
            scalar = __fdiv_rn(st.sum, (float)N);
            out = lut_eval(a.lut, normalise(scalar, a.lo, a.inv_range));
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

template <int MODE, int INTERP>
__global__ void __launch_bounds__(kAxThreads, 2)
    axis_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ vol, shw_camera cam, RenderArgs a,
                AxisArgs A)
{
    constexpr int R = kAxRays;
    extern __shared__ __align__(128) float sm[];  // [stages][bh][bw]
    __shared__ __align__(8) uint64_t full[kAxMaxStages], empty[kAxMaxStages];
    __shared__ long long s_pz, s_dz;
    __shared__ int s_n, s_any, s_x0, s_y0, s_bad, s_nidle;
    __shared__ volatile int s_quit;  // 1: every ray has stopped, or a wait gave up

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool consumer = warp < kAxWarps;
    const int tile = blockIdx.x, tyi = tile / A.tiles_x, txi = tile - tyi * A.tiles_x;
    const int S = A.stages;

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
        for (int s = 0; s < S; ++s) s_bad |= !tma_dst_ok(sm + s * A.stage_stride, A.err);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kAxWarps);
        }
        fence_barrier_init();
    }

    // the consumer's rays; every ray that meets the cube shares one z sequence
    long long X[R], Y[R];
    int hitmask = 0, N = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        X[i] = Y[i] = 0;
        const int px = ray_px(txi, lane, i), py = ray_py(tyi, warp, i);
        RayFx r;
        if (consumer && px < a.width && py < a.height && setup_ray(cam, px, py, A.nx, A.ny, A.nz, a.step, r) &&
            min(r.N, a.nmax) > 0) {
            hitmask |= 1 << i;
            N = min(r.N, a.nmax);
            X[i] = r.P[0];
            Y[i] = r.P[1];
            if (i == 0 || (hitmask & ((1 << i) - 1)) == 0) {
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
                const int px = ray_px(txi, lane, i), py = ray_py(tyi, warp, i);
                if (px < a.width && py < a.height)
                    axis_emit<MODE>(a, (long long)py * a.width + px, false, 0, 0, 0, INTERP == SHW_NEAREST,
                                    typename StateOf<MODE>::type{}, 0);
            }
        return;
    }
    const int NS = s_n;
    const long long PZ = s_pz, DZ = s_dz;
    const int bw = A.bw, bh = A.bh, x0b = s_x0, y0b = s_y0;
    const int stride = A.stage_stride;

    // the planes in the order the sweep needs them
    const int nz = A.nz;
    const int cz_first = clampi(fx_cell(PZ), -1, nz - 1);
    const int cz_last = clampi(fx_cell(PZ + (long long)(NS - 1) * DZ), -1, nz - 1);
    const bool up = DZ > 0;
    const int p_first = up ? max(cz_first, 0) : min(cz_first + 1, nz - 1);
    const int p_last = up ? min(cz_last + 1, nz - 1) : max(cz_last, 0);
    const int nplanes = (up ? p_last - p_first : p_first - p_last) + 1;

    if (!consumer) {
        // producer: one thread keeps the ring full
        if (lane != 0) return;
        const uint32_t stage_bytes = (uint32_t)(bw * bh * 4);
        int issued = 0;
        for (int j = 0; j < nplanes; ++j) {
            const int s = j % S;
            if (j >= S) {  // wait until every consumer warp has released plane j - S
                const uint32_t par = (uint32_t)(((j / S) - 1) & 1);
                bool ok = false, quit = false;
                for (int it = 0; it < kWaitSpins && !ok && !quit; ++it) {
                    ok = mbar_try_wait(&empty[s], par);
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
            mbar_arrive_expect_tx(&full[s], stage_bytes);
            tma_load_3d(sm + s * stride, &tmap, x0b, y0b, up ? p_first + j : p_first - j, &full[s]);
            issued = j + 1;
        }
        // every copy issued lands before this CTA may exit
        for (int j = max(issued - S, 0); j < issued; ++j) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), A.err);
        return;
    }

    // consumer: offsets of each ray's corners in the staged box, or in the global plane
    // for a ray outside the box
    int o00[R], o01[R], o10[R], o11[R], inbox = 0;
    float fx[R], fy[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int ix = clampi(fx_cell(X[i]), -1, A.nx - 1), iy = clampi(fx_cell(Y[i]), -1, A.ny - 1);
        int gx0 = max(ix, 0), gx1 = min(ix + 1, A.nx - 1), gy0 = max(iy, 0), gy1 = min(iy + 1, A.ny - 1);
        if constexpr (INTERP == SHW_NEAREST) {
            gx0 = gx1 = clampi(fx_round(X[i]), 0, A.nx - 1);
            gy0 = gy1 = clampi(fx_round(Y[i]), 0, A.ny - 1);
        }
        fx[i] = fx_frac(X[i]);
        fy[i] = fx_frac(Y[i]);
        const int c0 = gx0 - x0b, c1 = gx1 - x0b, r0 = gy0 - y0b, r1 = gy1 - y0b;
        if (c0 >= 0 && c1 < bw && r0 >= 0 && r1 < bh) {
            inbox |= 1 << i;
            o00[i] = r0 * bw + c0;
            o01[i] = r0 * bw + c1;
            o10[i] = r1 * bw + c0;
            o11[i] = r1 * bw + c1;
        } else {
            o00[i] = gy0 * A.nx + gx0;
            o01[i] = gy0 * A.nx + gx1;
            o10[i] = gy1 * A.nx + gx0;
            o11[i] = gy1 * A.nx + gx1;
        }
    }
    const size_t plane_elems = (size_t)A.nx * A.ny;

    int j = 0;  // planes consumed
    // one plane's value for each ray (bilinear, or the nearest voxel); false if the sweep must end
    auto consume = [&](float pv[R], bool idle) -> bool {
        const int s = j % S;
        const uint32_t par = (uint32_t)((j / S) & 1);
        bool ok = false, quit = false;
        for (int it = 0; it < kWaitSpins && !ok && !quit; ++it) {
            ok = mbar_try_wait(&full[s], par);
            quit = !ok && s_quit != 0;
        }
        if (!ok && !quit) {
            atomicOr(A.err, kErrWaitTimeout);
            s_quit = 1;
        }
        if (!__all_sync(0xffffffffu, ok)) return false;  // the warp leaves together
        if (!idle) {
            const float *t = sm + s * stride;
            const float *g = vol + (size_t)(up ? p_first + j : p_first - j) * plane_elems;
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (!((hitmask >> i) & 1)) continue;
                if constexpr (INTERP == SHW_NEAREST) {
                    pv[i] = ((inbox >> i) & 1) ? t[o00[i]] : __ldg(g + o00[i]);
                } else if ((inbox >> i) & 1) {
                    pv[i] = bilerp(t[o00[i]], t[o01[i]], t[o10[i]], t[o11[i]], fx[i], fy[i]);
                } else {
                    pv[i] = bilerp(__ldg(g + o00[i]), __ldg(g + o01[i]), __ldg(g + o10[i]), __ldg(g + o11[i]), fx[i],
                                   fy[i]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        ++j;
        return true;
    };

    typename StateOf<MODE>::type st[R];
    int done[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        done[i] = 0;
        if constexpr (MODE == SHW_COMPOSITE) {
            const long long pix = (long long)ray_py(tyi, warp, i) * a.width + ray_px(txi, lane, i);
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
    }
    int live = hitmask;  // rays still taking samples
    bool idle = __all_sync(0xffffffffu, live == 0);
    if (idle && lane == 0 && atomicAdd(&s_nidle, 1) + 1 == kAxWarps) s_quit = 1;

    float va[R];  // value of the plane held (the near plane of the current cell)
#pragma unroll
    for (int i = 0; i < R; ++i) va[i] = 0.0f;
    bool alive = consume(va, idle);
    long long Z = PZ;
    int k = 0, c = cz_first, held = p_first, ncell = 0;
    while (alive && k < NS) {
        // planes of cell c are max(c, 0) and min(c + 1, nz - 1); the far one in sweep order
        const int far = up ? min(c + 1, nz - 1) : max(c, 0);
        float vb[R];
#pragma unroll
        for (int i = 0; i < R; ++i) vb[i] = va[i];
        if (far != held) {
            if (!consume(vb, idle)) break;
            held = far;
        }
        if (!idle) {
            float lov[R], dv[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                lov[i] = up ? va[i] : vb[i];
                const float hiv = up ? vb[i] : va[i];
                dv[i] = (INTERP == SHW_NEAREST) ? hiv : hiv - lov[i];
            }
            // the samples of cell c: Z below (c + 1) << 32 going up, at or above c << 32 going down
            const bool open_end = up ? (c >= nz - 1) : (c < 0);
            const long long zb = up ? ((long long)(c + 1) << 32) : ((long long)c << 32);
            for (; k < NS; ++k, Z += DZ) {
                if (!open_end && (up ? Z >= zb : Z < zb)) break;
                const float f = fx_frac(Z);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if (!((live >> i) & 1)) continue;
                    float v;
                    if constexpr (INTERP == SHW_NEAREST)
                        v = (f >= 0.5f) ? dv[i] : lov[i];  // floor(z + 1/2) is the upper plane iff frac >= 1/2
                    else
                        v = __fmaf_rn(f, dv[i], lov[i]);  // lerp(lo, hi, f), as in the general interpolation
                    v = isnan(v) ? a.lo : v;
                    done[i] = k + 1;
                    if (st[i].update(v, k)) live &= ~(1 << i);
                }
            }
        } else {
            // an idle warp only keeps releasing stages: skip the cell's samples
            const bool open_end = up ? (c >= nz - 1) : (c < 0);
            const long long zb = up ? ((long long)(c + 1) << 32) : ((long long)c << 32);
            for (; k < NS; ++k, Z += DZ)
                if (!open_end && (up ? Z >= zb : Z < zb)) break;
        }
#pragma unroll
        for (int i = 0; i < R; ++i) va[i] = vb[i];
        c += up ? 1 : -1;
        if (MODE == SHW_COMPOSITE && !idle && (++ncell & 15) == 0) {
            idle = __all_sync(0xffffffffu, live == 0);
            if (idle && lane == 0 && atomicAdd(&s_nidle, 1) + 1 == kAxWarps) s_quit = 1;
        }
        if (idle && s_quit != 0) break;  // every warp is idle: the sweep is over
    }

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int px = ray_px(txi, lane, i), py = ray_py(tyi, warp, i);
        if (px < a.width && py < a.height)
            axis_emit<MODE>(a, (long long)py * a.width + px, (hitmask >> i) & 1, N, PZ, DZ, INTERP == SHW_NEAREST,
                            st[i], done[i]);
    }
}

// The sweep applies to a float32 cube seen orthographically down +-z with the image
// plane spanned by x and y (the moment-map view), for single-cube modes.
static bool axis_eligible(const shw_volume &v, const shw_camera &c, int mode)
{
    if (std::getenv("SHW_NO_AXIS_SWEEP")) return false;
    return v.storage == SHW_F32 && mode != SHW_RATIO && c.ortho && c.fwd[0] == 0.0f && c.fwd[1] == 0.0f &&
           c.fwd[2] != 0.0f && c.right[2] == 0.0f && c.up[2] == 0.0f && v.nx % 4 == 0 && aligned(v.data, 16) &&
           (long long)v.nx * v.ny < (1ll << 31);
}

shw_status render_axis(int mode, int interp, const shw_volume &v, const shw_camera &c, const RenderArgs &a0,
                       cudaStream_t st)
{
    if (!axis_eligible(v, c, mode)) return SHW_EUNSUPPORTED;
    // pixel -> (x, y) is affine for a parallel projection (Appendix A)
    const double W = c.width, H = c.height, aspect = W / H;
    const double hw = (double)c.ortho_half_h * aspect, hh = c.ortho_half_h;
    const double ax = 2.0 * hw * c.right[0] / W, bx = -2.0 * hh * c.up[0] / H;
    const double ay = 2.0 * hw * c.right[1] / W, by = -2.0 * hh * c.up[1] / H;
    const double cx = c.eye[0] + hw * c.right[0] * (1.0 - W) / W + hh * c.up[0] * (H - 1.0) / H;
    const double cy = c.eye[1] + hw * c.right[1] * (1.0 - W) / W + hh * c.up[1] * (H - 1.0) / H;
    const double ext_x = (kAxTX - 1) * std::fabs(ax) + (kAxTY - 1) * std::fabs(bx);
    const double ext_y = (kAxTX - 1) * std::fabs(ay) + (kAxTY - 1) * std::fabs(by);
    AxisArgs A{};
    A.bw = ((int)std::ceil(ext_x) + 8 + 3) & ~3;
    A.bh = (int)std::ceil(ext_y) + 6;
    if (A.bw > 256 || A.bh > 256) return SHW_EUNSUPPORTED;  // the tensor copy's box limit
    A.stage_stride = (A.bw * A.bh + 31) & ~31;               // TMA destinations must start on 128 bytes
    A.stages = std::min(kAxMaxStages, (int)(kAxSmemLimit / ((size_t)A.stage_stride * 4)));
    if (A.stages < 2) return SHW_EUNSUPPORTED;
    const size_t smem = (size_t)A.stages * A.stage_stride * 4;
    A.nx = v.nx;
    A.ny = v.ny;
    A.nz = v.nz;
    A.cx = (float)cx;
    A.ax = (float)ax;
    A.bx = (float)bx;
    A.cy = (float)cy;
    A.ay = (float)ay;
    A.by = (float)by;
    A.err = device_error_word();
    A.tiles_x = ceil_div(c.width, kAxTX);
    const long long tiles = (long long)A.tiles_x * ceil_div(c.height, kAxTY);
    const float *data = static_cast<const float *>(v.data);
    CUtensorMap map;
    if (!encode_tmap_3d_f32(&map, data, v.nx, v.ny, v.nz, A.bw, A.bh)) return SHW_EUNSUPPORTED;
    RenderArgs a = a0;
#define SHW_AX(M, I)                                                                                    \
    do {                                                                                                \
        /* static + dynamic shared memory may pass the 48 KB default: always opt in */                \
        cudaFuncSetAttribute(axis_kernel<M, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        axis_kernel<M, I><<<(unsigned)tiles, kAxThreads, smem, st>>>(map, data, c, a, A);              \
    } while (0)
#define SHW_AXC(M)                                         \
    case M:                                                \
        if (interp == SHW_NEAREST) SHW_AX(M, SHW_NEAREST); \
        else SHW_AX(M, SHW_TRILINEAR);                     \
        break;
    switch (mode) {
        SHW_AXC(SHW_MIP)
        SHW_AXC(SHW_AVG)
        SHW_AXC(SHW_COMPOSITE)
        SHW_AXC(SHW_SPECTRAL)
    default:
        return SHW_EUNSUPPORTED;
    }
#undef SHW_AXC
#undef SHW_AX
    return after_launch();
}

}  // namespace shw
