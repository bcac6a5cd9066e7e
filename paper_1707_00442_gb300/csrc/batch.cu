// batch.cu -- many sub-cubes of uneven sizes rendered by one persistent launch
// captured in a CUDA graph.
//
// Upcoming surveys produce sub-cubes for the many hundreds of galaxies they
// detect (Section 1); rendering each with its own launch wastes most of the GPU on
// launch latency and tail effects.  A plan lays out every (item, image tile) as a
// work item, ordered longest-first (an LPT schedule: big cubes' tiles first, small
// ones fill the tail); a persistent grid of CTAs pops work items from an atomic
// counter -- no CTA ever waits on another -- and renders each tile with the same
// per-ray code as shw_render.  The counter resets and the launches are captured once
// into a CUDA graph, so a batch render is a single graph launch.  Float32 cubes and
// bricks are rendered by two kernels (one work list each, run one after the other in
// the same graph): a kernel for both kinds would hold the registers of both paths.  An
// autotuner times the candidate tile shapes and CTAs-per-SM -- and, for plans that round
// their float32 items into 16-bit bricks of their own, the brick edge (16 or 32 voxels)
// -- at plan creation and caches the winner per batch signature.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "batch_kernel.cuh"

namespace shw {

bool valid_volume(const shw_volume *v);
bool valid_camera(const shw_camera *c);
long long max_samples(const shw_volume *v, float step);
size_t bricked_bytes_edge(int nx, int ny, int nz, int edge);

// Brick items are addressed with 32-bit element offsets: a storage of 2^31 elements or more
// (a cube of about 1280^3 voxels) is not taken in a batch.  edge: 0 for the caller's
// storage, else the edge of the plan's own bricks.
static bool bricks_fit_int(const shw_volume &v, int edge)
{
    const size_t bytes =
        edge ? bricked_bytes_edge(v.nx, v.ny, v.nz, edge) : shw_bricked_bytes(v.nx, v.ny, v.nz, v.storage);
    return bytes / 2 < ((size_t)1 << 31);
}
shw_status pack_bricks_edge(const float *in, int nx, int ny, int nz, int storage, int edge, void *out,
                            cudaStream_t st);

BatchKernel batch_kernel_for(int tile, int interp, int kind)
{
    if (kind == 16) return batch_kernel_b16(tile, interp);
    if (kind == 32) return batch_kernel_b32(tile, interp);
    if (tile == 8) return interp == SHW_NEAREST ? batch_kernel<8, SHW_NEAREST, 0> : batch_kernel<8, SHW_TRILINEAR, 0>;
    return interp == SHW_NEAREST ? batch_kernel<16, SHW_NEAREST, 0> : batch_kernel<16, SHW_TRILINEAR, 0>;
}

// One kernel's share of a batch: the items of one kind (0: float32, else the brick
// edge), `n` work items from `off` in the work list, counter `counter`.
struct WorkGroup {
    int kind, off, n, counter;
};

// Work items (item, tile) of every image, the largest items' tiles first (LPT), split by
// kind: float32 items first, then bricks.  Fills `work` and `groups` (empty kinds left out);
// false when there are 2^31 work items or more.
static bool group_work(const BatchItemDev *items, const std::vector<int> &order, int tile, int brick_kind,
                       std::vector<int2> &work, std::vector<WorkGroup> &groups)
{
    std::vector<int2> by_kind[2];
    for (int i : order) {
        const BatchItemDev &it = items[i];
        const int nt = ceil_div(it.cam.width, tile) * ceil_div(it.cam.height, tile);
        std::vector<int2> &w = by_kind[it.storage == SHW_F32 ? 0 : 1];
        for (int t = 0; t < nt; ++t) w.push_back(make_int2(i, t));
    }
    work.clear();
    groups.clear();
    if (by_kind[0].size() + by_kind[1].size() > (size_t)0x7fffffff) return false;
    for (int k = 0; k < 2; ++k) {
        if (by_kind[k].empty()) continue;
        groups.push_back({k == 0 ? 0 : brick_kind, (int)work.size(), (int)by_kind[k].size(), (int)groups.size()});
        work.insert(work.end(), by_kind[k].begin(), by_kind[k].end());
    }
    return true;
}

struct TileChoice {
    int tile, ctas_per_sm;
};
static const TileChoice kTileChoices[] = {{16, 2}, {16, 4}, {16, 8}, {8, 8}, {8, 16}, {8, 32}};
constexpr int kNumTileChoices = (int)(sizeof(kTileChoices) / sizeof(kTileChoices[0]));
constexpr int kDefaultTileChoice = 1;  // {16, 4}

// one configuration the autotuner times; brick: edge of the plan's own bricks (0: none)
struct Candidate {
    int tile, ctas_per_sm, brick;
};

// process-wide cache of tuned choices, keyed by the batch signature
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

}  // namespace shw

using namespace shw;

struct shw_batch_plan {
    int device = 0;
    int n_items = 0, nwork = 0, tile = 16, ctas_per_sm = 4, grid = 0, interp = SHW_TRILINEAR;
    int sms = 0;
    BatchItemDev *d_items = nullptr;
    int2 *d_work = nullptr;
    int *d_counter = nullptr;
    BatchShared sh{};
    std::vector<BatchItemDev> items;
    std::vector<int> order;  // items sorted by estimated cost, descending
    std::vector<Candidate> cands;
    std::vector<WorkGroup> groups;  // one kernel per kind of item, in launch order
    // bricks the plan packs itself (SHW_BATCH_PACK_*): one buffer per edge (16, 32)
    int brick = 0, pack_storage = 0;
    std::vector<const float *> src;  // each packed item's float32 cube, else nullptr
    void *d_packed[2] = {nullptr, nullptr};
    size_t packed_bytes[2] = {0, 0};
    std::vector<size_t> pack_off[2];
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    shw_batch_info info{};
};

static void plan_free(shw_batch_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->d_items) cudaFree(pl->d_items);
    if (pl->d_work) cudaFree(pl->d_work);
    if (pl->d_counter) cudaFree(pl->d_counter);
    for (void *b : pl->d_packed)
        if (b) cudaFree(b);
    delete pl;
}

// host-side fault injection (shw_set_debug_flags)
static bool fault(uint32_t flag) { return debug(flag); }

// (re)build the work list for a tile size: tiles of the biggest items first
static shw_status build_work(shw_batch_plan *pl, int tile)
{
    for (BatchItemDev &it : pl->items) it.tiles_x = ceil_div(it.cam.width, tile);
    std::vector<int2> work;
    if (!group_work(pl->items.data(), pl->order, tile, pl->brick == 16 ? 16 : 32, work, pl->groups))
        return SHW_EUNSUPPORTED;
    pl->nwork = (int)work.size();
    if (pl->d_work) cudaFree(pl->d_work);
    pl->d_work = nullptr;
    if (fault(SHW_DEBUG_FAULT_ALLOC) || cudaMalloc(&pl->d_work, work.size() * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        pl->d_work = nullptr;
        return SHW_ENOMEM;
    }
    if (cudaMemcpy(pl->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
        return SHW_ECUDA;
    if (cudaMemcpy(pl->d_items, pl->items.data(), pl->items.size() * sizeof(BatchItemDev), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return SHW_ECUDA;
    pl->tile = tile;
    return SHW_OK;
}

static int edge_slot(int edge) { return edge == 16 ? 0 : 1; }

// The plan's bricks of one edge: allocated and filled on `st` the first time they are asked for.
static shw_status pack_edge(shw_batch_plan *pl, int edge, cudaStream_t st)
{
    const int k = edge_slot(edge);
    if (pl->d_packed[k]) return SHW_OK;
    std::vector<size_t> &off = pl->pack_off[k];
    off.assign(pl->n_items, 0);
    size_t total = 0;
    for (int i = 0; i < pl->n_items; ++i) {
        if (!pl->src[i]) continue;
        const BatchItemDev &it = pl->items[i];
        off[i] = total;
        total += (bricked_bytes_edge(it.nx, it.ny, it.nz, edge) + 255) & ~(size_t)255;
    }
    if (fault(SHW_DEBUG_FAULT_ALLOC) || cudaMalloc(&pl->d_packed[k], total) != cudaSuccess) {
        cudaGetLastError();
        pl->d_packed[k] = nullptr;
        return SHW_ENOMEM;
    }
    pl->packed_bytes[k] = total;
    for (int i = 0; i < pl->n_items; ++i) {
        if (!pl->src[i]) continue;
        const BatchItemDev &it = pl->items[i];
        const shw_status s = pack_bricks_edge(pl->src[i], it.nx, it.ny, it.nz, pl->pack_storage, edge,
                                              static_cast<unsigned char *>(pl->d_packed[k]) + off[i], st);
        if (s != SHW_OK) return s;
    }
    return SHW_OK;
}

// Point the packed items at their bricks of one edge (build_work copies the table).
static void use_edge(shw_batch_plan *pl, int edge)
{
    const int k = edge_slot(edge);
    for (int i = 0; i < pl->n_items; ++i) {
        if (!pl->src[i]) continue;
        BatchItemDev &it = pl->items[i];
        it.data = static_cast<unsigned char *>(pl->d_packed[k]) + pl->pack_off[k][i];
        it.storage = pl->pack_storage;
        it.brick = edge;
        it.nbx = ceil_div(it.nx, edge);
        it.nby = ceil_div(it.ny, edge);
    }
    pl->brick = edge;
}

// Enqueue one render of the batch on `st`: clear the counters, then one persistent kernel
// per kind of item.  note: count the kernels as launched (not while capturing).
static shw_status enqueue_groups(const std::vector<WorkGroup> &groups, const BatchItemDev *d_items,
                                 const int2 *d_work, int *d_counter, BatchShared sh, int tile, int interp, int grid,
                                 cudaStream_t st, bool note)
{
    if (cudaMemsetAsync(d_counter, 0, 2 * sizeof(int), st) != cudaSuccess) return SHW_ECUDA;
    for (const WorkGroup &g : groups) {
        sh.nwork = g.n;
        batch_kernel_for(tile, interp, g.kind)<<<grid, tile * tile, 0, st>>>(d_items, d_work + g.off,
                                                                             d_counter + g.counter, sh);
        if (note) note_launch();
        if (cudaGetLastError() != cudaSuccess) return SHW_ECUDA;
    }
    return SHW_OK;
}

static shw_status launch_direct(shw_batch_plan *pl, int ctas_per_sm, cudaStream_t st)
{
    return enqueue_groups(pl->groups, pl->d_items, pl->d_work, pl->d_counter, pl->sh, pl->tile, pl->interp,
                          pl->sms * ctas_per_sm, st, true);
}

static shw_status capture(shw_batch_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
    if (fault(SHW_DEBUG_FAULT_GRAPH)) return SHW_ECUDA;
    if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SHW_ECUDA;
    pl->grid = pl->sms * pl->ctas_per_sm;
    // (an error here is reported by the end of the capture)
    enqueue_groups(pl->groups, pl->d_items, pl->d_work, pl->d_counter, pl->sh, pl->tile, pl->interp, pl->grid,
                   pl->cap, false);
    cudaError_t e = cudaStreamEndCapture(pl->cap, &pl->graph);
    if (e != cudaSuccess || !pl->graph) {
        cudaGetLastError();
        return SHW_ECUDA;
    }
    if (cudaGraphInstantiate(&pl->exec, pl->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return SHW_ECUDA;
    }
    return SHW_OK;
}

static std::string signature(const shw_batch_plan *pl)
{
    // size class of the work: log2 of the mean item voxel count and image area, storages, modes,
    // the packing storage and the brick edges tried
    double vox = 0.0, pix = 0.0;
    int smask = 0, mmask = 0;
    for (const auto &it : pl->items) {
        vox += (double)it.nx * it.ny * it.nz;
        pix += (double)it.cam.width * it.cam.height;
        smask |= 1 << it.storage;
        mmask |= 1 << it.mode;
    }
    const int n = std::max(1, pl->n_items);
    int emask = 0;
    for (const Candidate &c : pl->cands) emask |= c.brick;
    char buf[192];
    std::snprintf(buf, sizeof buf, "i%d v%d p%d n%d s%d m%d sm%d k%d e%d", pl->interp,
                  (int)std::lround(std::log2(vox / n + 1)), (int)std::lround(std::log2(pix / n + 1)),
                  (int)std::lround(std::log2((double)n)), smask, mmask, pl->sms, pl->pack_storage, emask);
    return buf;
}

static shw_status autotune(shw_batch_plan *pl, cudaStream_t st, int *best_out)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SHW_ECUDA;
    int best = -1;
    float best_ms = 1e30f;
    for (int c = 0; c < (int)pl->cands.size(); ++c) {
        const Candidate &cd = pl->cands[c];
        shw_status s = SHW_OK;
        if (cd.brick && cd.brick != pl->brick) {
            s = pack_edge(pl, cd.brick, st);
            if (s == SHW_OK) use_edge(pl, cd.brick);
        }
        if (s == SHW_OK) s = build_work(pl, cd.tile);
        if (s != SHW_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s;
        }
        s = launch_direct(pl, cd.ctas_per_sm, st);  // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && s == SHW_OK; ++rep) {
            cudaEventRecord(e0, st);
            s = launch_direct(pl, cd.ctas_per_sm, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = SHW_ECUDA;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (s != SHW_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return s;
        }
        pl->info.tune_ms[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_out = best;
    return SHW_OK;
}

extern "C" {

shw_status shw_batch_plan_create(shw_batch_plan **out, const shw_batch_item *items, int32_t n,
                                 const shw_render_params *p, int32_t flags, void *stream)
{
    NvtxRange nvtx_range("shw_batch_plan_create");
    if (!out) return SHW_EINVAL;
    *out = nullptr;
    if (!items || n <= 0 || !p || !p->lut || !aligned(p->lut, 16)) return SHW_EINVAL;
    if (p->interp != SHW_NEAREST && p->interp != SHW_TRILINEAR) return SHW_EINVAL;
    if (p->filter != SHW_FILTER_NONE || p->alpha_threshold != 0 || p->smooth != SHW_SMOOTH_NONE)
        return SHW_EUNSUPPORTED;  // not in batch plans
    if (!std::isfinite(p->step) || !(p->step > 0.0f) || !(p->hi > p->lo) || !std::isfinite(p->lo) ||
        !std::isfinite(p->hi) || !std::isfinite(p->opacity_scale) || !std::isfinite(p->term_alpha))
        return SHW_EINVAL;
    const int pack = flags & (SHW_BATCH_PACK_BF16 | SHW_BATCH_PACK_F16);
    const int fixed = flags & (SHW_BATCH_BRICK_16 | SHW_BATCH_BRICK_32);
    if (pack == (SHW_BATCH_PACK_BF16 | SHW_BATCH_PACK_F16) || fixed == (SHW_BATCH_BRICK_16 | SHW_BATCH_BRICK_32) ||
        (fixed && !pack))
        return SHW_EINVAL;
    int n_own = 0;  // float32 items the plan packs
    for (int i = 0; i < n; ++i) {
        const shw_batch_item &b = items[i];
        if (!valid_volume(&b.vol) || !valid_camera(&b.cam) || !b.out_rgba || !aligned(b.out_rgba, 16))
            return SHW_EINVAL;
        if (b.mode != SHW_MIP && b.mode != SHW_AVG && b.mode != SHW_COMPOSITE && b.mode != SHW_SPECTRAL)
            return (b.mode >= SHW_RATIO && b.mode <= SHW_RATIO_MIP) ? SHW_EUNSUPPORTED : SHW_EINVAL;
        if ((long long)b.vol.nx * b.vol.ny * b.vol.nz >= (1LL << 31)) return SHW_EUNSUPPORTED;
        if (b.vol.storage >= SHW_F32_PAIR) return SHW_EUNSUPPORTED;  // the line ratios' storages
        if (max_samples(&b.vol, p->step) > (1LL << 30)) return SHW_EINVAL;
        if (b.vol.storage != SHW_F32 && !bricks_fit_int(b.vol, 0)) return SHW_EUNSUPPORTED;
        if (pack && b.vol.storage == SHW_F32 && (!bricks_fit_int(b.vol, 16) || !bricks_fit_int(b.vol, 32)))
            return SHW_EUNSUPPORTED;
        n_own += (pack && b.vol.storage == SHW_F32) ? 1 : 0;
    }
    // brick edges to try: 16 needs its own kernel, which reads only the plan's bricks, so
    // a plan that also holds bricks packed by the caller (edge 32) keeps 32
    std::vector<int> edges;
    if (n_own == 0) {
        edges.push_back(0);
    } else if (fixed == SHW_BATCH_BRICK_16) {
        if (n_own != n) return SHW_EUNSUPPORTED;
        edges.push_back(16);
    } else if (fixed == SHW_BATCH_BRICK_32 || n_own != n) {
        edges.push_back(32);
    } else {
        edges.push_back(16);
        edges.push_back(32);
    }
    shw_batch_plan *pl = new (std::nothrow) shw_batch_plan();
    if (!pl) return SHW_ENOMEM;
    if (cudaGetDevice(&pl->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return SHW_EDEVICE;
    }
    pl->n_items = n;
    pl->interp = p->interp;
    pl->sh.lut = reinterpret_cast<const float4 *>(p->lut);
    pl->sh.step = p->step;
    pl->sh.lo = p->lo;
    pl->sh.inv_range = 1.0f / (p->hi - p->lo);
    pl->sh.opacity_scale = p->opacity_scale;
    pl->sh.term_alpha = p->term_alpha;
    pl->pack_storage = n_own ? (pack == SHW_BATCH_PACK_BF16 ? SHW_BF16_BRICK : SHW_F16_BRICK) : 0;
    for (int e : edges)
        for (const TileChoice &t : kTileChoices) pl->cands.push_back({t.tile, t.ctas_per_sm, e});
    pl->items.resize(n);
    pl->src.assign(n, nullptr);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        const shw_batch_item &b = items[i];
        BatchItemDev &d = pl->items[i];
        std::memset(&d, 0, sizeof d);
        d.data = b.vol.data;
        d.rgba = reinterpret_cast<float4 *>(b.out_rgba);
        d.nx = b.vol.nx;
        d.ny = b.vol.ny;
        d.nz = b.vol.nz;
        d.storage = b.vol.storage;
        d.mode = b.mode;
        d.nbx = ceil_div(b.vol.nx, kBrick);
        d.nby = ceil_div(b.vol.ny, kBrick);
        d.brick = kBrick;
        d.nmax = (int)max_samples(&b.vol, p->step);
        d.cam = b.cam;
        if (n_own && b.vol.storage == SHW_F32) pl->src[i] = static_cast<const float *>(b.vol.data);
        // expected work: pixels x mean chord (~ cube size) in samples
        cost[i] = (double)b.cam.width * b.cam.height * std::cbrt((double)b.vol.nx * b.vol.ny * b.vol.nz) / p->step;
    }
    pl->order.resize(n);
    for (int i = 0; i < n; ++i) pl->order[i] = i;
    std::stable_sort(pl->order.begin(), pl->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

    if (fault(SHW_DEBUG_FAULT_ALLOC) || cudaMalloc(&pl->d_items, sizeof(BatchItemDev) * n) != cudaSuccess ||
        cudaMalloc(&pl->d_counter, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        plan_free(pl);
        return SHW_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) {
        plan_free(pl);
        return SHW_ECUDA;
    }
    cudaStream_t st = as_stream(stream);
    const std::string sig = signature(pl);
    // untuned: {16, 4} with the last edge tried (32 unless 16 is fixed)
    const int ncand = (int)pl->cands.size();
    int choice = ncand - kNumTileChoices + kDefaultTileChoice;
    bool tuned = false;
    if (!(flags & SHW_BATCH_NO_TUNE)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto itc = g_tune_cache.find(sig);
        if (itc != g_tune_cache.end() && itc->second >= 0 && itc->second < ncand && !(flags & SHW_BATCH_RETUNE)) {
            choice = itc->second;
        } else {
            int best = -1;
            shw_status s = autotune(pl, st, &best);
            if (s != SHW_OK) {
                plan_free(pl);
                return s;
            }
            choice = best;
            tuned = true;
            g_tune_cache[sig] = best;
        }
    }
    const Candidate &cc = pl->cands[choice];
    shw_status s = SHW_OK;
    if (cc.brick) {
        // the chosen edge's bricks (already there if the autotuner packed them); the other
        // edge's copy, if any, is released
        s = pack_edge(pl, cc.brick, st);
        if (s == SHW_OK) {
            use_edge(pl, cc.brick);
            const int other = 1 - edge_slot(cc.brick);
            if (pl->d_packed[other]) {
                cudaFree(pl->d_packed[other]);
                pl->d_packed[other] = nullptr;
                pl->packed_bytes[other] = 0;
            }
        }
    }
    pl->ctas_per_sm = cc.ctas_per_sm;
    if (s == SHW_OK) s = build_work(pl, cc.tile);
    if (s == SHW_OK) s = capture(pl);
    // the bricks are written on `stream`; the graph may be replayed on any stream
    if (s == SHW_OK && cc.brick && cudaStreamSynchronize(st) != cudaSuccess) s = SHW_ECUDA;
    if (s != SHW_OK) {
        plan_free(pl);
        return s;
    }
    shw_batch_info &inf = pl->info;
    inf.n_items = n;
    inf.n_work = pl->nwork;
    inf.tile = pl->tile;
    inf.ctas_per_sm = pl->ctas_per_sm;
    inf.grid = pl->grid;
    inf.tuned = tuned ? 1 : 0;
    inf.brick = cc.brick;
    inf.packed_bytes = cc.brick ? (int64_t)pl->packed_bytes[edge_slot(cc.brick)] : 0;
    inf.n_candidates = ncand;
    for (int c = 0; c < ncand && c < 16; ++c) {
        inf.cand_tile[c] = pl->cands[c].tile;
        inf.cand_ctas_per_sm[c] = pl->cands[c].ctas_per_sm;
        inf.cand_brick[c] = pl->cands[c].brick;
        if (!tuned) inf.tune_ms[c] = -1.0f;
    }
    *out = pl;
    return SHW_OK;
}

shw_status shw_render_batch(shw_batch_plan *plan, void *stream)
{
    NvtxRange nvtx_range("shw_render_batch");
    if (!plan || !plan->exec) return SHW_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return SHW_EINVAL;
    if (cudaGraphLaunch(plan->exec, as_stream(stream)) != cudaSuccess) return SHW_ECUDA;
    for (size_t g = 0; g < plan->groups.size(); ++g) note_launch();  // one kernel per kind of item
    return SHW_OK;
}

shw_status shw_render_items(const shw_batch_item *items, int32_t n, const shw_render_params *p, void *stream)
{
    NvtxRange nvtx_range("shw_render_items");
    if (!items || n <= 0 || !p) return SHW_EINVAL;
    for (int i = 0; i < n; ++i) {
        shw_render_params q = *p;
        q.mode = items[i].mode;
        const shw_status s = shw_render(&items[i].vol, nullptr, &items[i].cam, &q, items[i].out_rgba, nullptr, nullptr,
                                        nullptr, nullptr, 0, stream);
        if (s != SHW_OK) return s;
    }
    return SHW_OK;
}

shw_status shw_batch_plan_info(const shw_batch_plan *plan, shw_batch_info *info)
{
    if (!plan || !info) return SHW_EINVAL;
    *info = plan->info;
    return SHW_OK;
}

shw_status shw_batch_plan_destroy(shw_batch_plan *plan)
{
    if (!plan) return SHW_EINVAL;
    cudaDeviceSynchronize();  // no launch of this plan may still be running
    cudaGetLastError();
    plan_free(plan);
    return SHW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched rendering without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host application
// that owns every byte of the GPU through its own pool or budget (a plugin inside
// a visualisation program), or an interactive loop that must never stall in the
// allocator.  For them the batch kernel above also runs from a fixed scratch
// array that is part of the library image: every GPU that loads the library holds
// these SHW_NOALLOC_SCRATCH_BYTES until the process exits.  Host code must not
// take the array's address directly (in host code its name is only a stand-in for
// the device symbol), so each device's address is fetched once with
// cudaGetSymbolAddress while that device is current.

namespace shw {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SHW_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr size_t kNoallocCounterBytes = 256;  // the two work counters live in the first aligned slot
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[kNoallocMaxDevices] = {};
static int g_noalloc_sms[kNoallocMaxDevices] = {};

}  // namespace shw

extern "C" shw_status shw_render_batch_noalloc(const shw_batch_item *items, int32_t n, const shw_render_params *p,
                                               void *stream)
{
    NvtxRange nvtx_range("shw_render_batch_noalloc");
    if (!items || n <= 0 || !p || !p->lut || !aligned(p->lut, 16)) return SHW_EINVAL;
    if (p->interp != SHW_NEAREST && p->interp != SHW_TRILINEAR) return SHW_EINVAL;
    if (p->filter != SHW_FILTER_NONE || p->alpha_threshold != 0 || p->smooth != SHW_SMOOTH_NONE)
        return SHW_EUNSUPPORTED;  // not in batch plans
    if (!std::isfinite(p->step) || !(p->step > 0.0f) || !(p->hi > p->lo) || !std::isfinite(p->lo) ||
        !std::isfinite(p->hi) || !std::isfinite(p->opacity_scale) || !std::isfinite(p->term_alpha))
        return SHW_EINVAL;
    constexpr int tile = 16, ctas_per_sm = 4;
    std::vector<double> cost(n);
    long long nwork = 0;
    for (int i = 0; i < n; ++i) {
        const shw_batch_item &b = items[i];
        if (!valid_volume(&b.vol) || !valid_camera(&b.cam) || !b.out_rgba || !aligned(b.out_rgba, 16))
            return SHW_EINVAL;
        if (b.mode != SHW_MIP && b.mode != SHW_AVG && b.mode != SHW_COMPOSITE && b.mode != SHW_SPECTRAL)
            return (b.mode >= SHW_RATIO && b.mode <= SHW_RATIO_MIP) ? SHW_EUNSUPPORTED : SHW_EINVAL;
        if ((long long)b.vol.nx * b.vol.ny * b.vol.nz >= (1LL << 31)) return SHW_EUNSUPPORTED;
        if (b.vol.storage >= SHW_F32_PAIR) return SHW_EUNSUPPORTED;  // the line ratios' storages
        if (max_samples(&b.vol, p->step) > (1LL << 30)) return SHW_EINVAL;
        if (b.vol.storage != SHW_F32 && !bricks_fit_int(b.vol, 0)) return SHW_EUNSUPPORTED;
        nwork += (long long)ceil_div(b.cam.width, tile) * ceil_div(b.cam.height, tile);
        cost[i] = (double)b.cam.width * b.cam.height * std::cbrt((double)b.vol.nx * b.vol.ny * b.vol.nz) / p->step;
    }
    const size_t items_off = kNoallocCounterBytes;
    const size_t work_off = items_off + sizeof(BatchItemDev) * (size_t)n;
    const size_t bytes = work_off + sizeof(int2) * (size_t)nwork;
    if (nwork > 0x7fffffffLL || bytes > SHW_NOALLOC_SCRATCH_BYTES) return SHW_EUNSUPPORTED;  // beyond the fixed scratch

    // the table below is copied from host memory this call owns only while it runs, so a
    // capture (whose replays would read it after the call returned) is refused
    const int cs = capture_state(as_stream(stream));
    if (cs != 0) return cs > 0 ? SHW_EUNSUPPORTED : SHW_ECUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SHW_EDEVICE;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) return SHW_EUNSUPPORTED;
    unsigned char *scratch = nullptr;
    int sms = 0;
    {
        // once per device, with that device current: the scratch array's device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return SHW_ECUDA;
            }
            int nsm = 0;
            if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
                cudaGetLastError();
                return SHW_EDEVICE;
            }
            g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
            g_noalloc_sms[dev] = nsm;
        }
        scratch = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }

    // the item table and the work list (largest items' tiles first), staged on the host
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<unsigned char> host(bytes - items_off);
    BatchItemDev *hitems = reinterpret_cast<BatchItemDev *>(host.data());
    int2 *hwork = reinterpret_cast<int2 *>(host.data() + (work_off - items_off));
    for (int i = 0; i < n; ++i) {
        const shw_batch_item &b = items[i];
        BatchItemDev d;
        std::memset(&d, 0, sizeof d);
        d.data = b.vol.data;
        d.rgba = reinterpret_cast<float4 *>(b.out_rgba);
        d.nx = b.vol.nx;
        d.ny = b.vol.ny;
        d.nz = b.vol.nz;
        d.storage = b.vol.storage;
        d.mode = b.mode;
        d.nbx = ceil_div(b.vol.nx, kBrick);
        d.nby = ceil_div(b.vol.ny, kBrick);
        d.brick = kBrick;
        d.nmax = (int)max_samples(&b.vol, p->step);
        d.cam = b.cam;
        d.tiles_x = ceil_div(b.cam.width, tile);
        std::memcpy(hitems + i, &d, sizeof d);
    }
    // one work list per kind of item (float32, bricks), each largest items first
    std::vector<int2> work;
    std::vector<WorkGroup> groups;
    if (!group_work(hitems, order, tile, kBrick, work, groups) || (long long)work.size() != nwork)
        return SHW_EUNSUPPORTED;
    std::memcpy(hwork, work.data(), work.size() * sizeof(int2));
    BatchShared sh{};
    sh.lut = reinterpret_cast<const float4 *>(p->lut);
    sh.step = p->step;
    sh.lo = p->lo;
    sh.inv_range = 1.0f / (p->hi - p->lo);
    sh.opacity_scale = p->opacity_scale;
    sh.term_alpha = p->term_alpha;

    cudaStream_t st = as_stream(stream);
    // the array keeps the previous call's contents: the two counters (the first slot) are
    // cleared on the stream by enqueue_groups, after the table's copy is enqueued
    if (cudaMemcpyAsync(scratch + items_off, host.data(), host.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SHW_ECUDA;
    return enqueue_groups(groups, reinterpret_cast<const BatchItemDev *>(scratch + items_off),
                          reinterpret_cast<const int2 *>(scratch + work_off), reinterpret_cast<int *>(scratch), sh,
                          tile, p->interp, sms * ctas_per_sm, st, true);
}

