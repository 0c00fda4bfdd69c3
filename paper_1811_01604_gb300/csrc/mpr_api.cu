// mpr_api.cu -- host side of the C ABI declared in include/mpr.h.
//
// A context owns a Batch: one or more grids ("entries") laid out as red/black planes
// (see mpr_internal.cuh) plus their gap lists, per-entry control state and the sweep
// work lists.  The main fill is a batch of one entry; the e(T, L) table of Eq. 5 is a
// batch of KT all-free lattices that run together.  Sweeps are driven by CUDA graphs
// of S sweeps (half-sweep A, half-sweep B, control) replayed until every entry of the
// relaxation has stopped.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mpr.h"
#include "mpr_internal.cuh"
#include "mpr_net_internal.cuh"

using namespace mpr;

namespace {
extern std::atomic<unsigned long long> g_launches;
}
void mpr::count_launches(unsigned long long n, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return;
    g_launches += n;
}

namespace {

constexpr int kMaxGraphSweeps = 64;       // longest captured chunk of sweeps
constexpr int kDefaultGraphSweeps = 8;    // sweeps per captured chunk unless autotuned
constexpr int kScratch = 2048;            // doubles of reduction scratch
constexpr int kFan = 8;                   // auxiliary streams of a batch's per-grid set-up work
constexpr int kMaxChains = 128;           // independent chains of one grid (mpr_predict_chains)
constexpr uint32_t kChainStride = 1u << 24; // chain word offset between forked chains

struct GridIn {
    int W, H;
    const float* z;       // device, may be null for all-free lattices
    const uint8_t* mask;  // device, may be null for all-free lattices
    uint32_t chain;
    double T;
    double zmin, scale;
    uint32_t row_off = 0;  // rows of a larger grid above this block (Philox counters)
};

struct Batch {
    int n_ent = 0;
    std::vector<EntryDesc> ents;
    EntryDesc* d_ents = nullptr;
    float2* d_lat = nullptr;
    size_t lat_elems = 0;
    uint32_t* d_gaps = nullptr;
    float* d_acc = nullptr;
    size_t n_gaps = 0;
    BlockWork* d_work[2] = {nullptr, nullptr};
    int nblk[2] = {0, 0};
    Part* d_part[2] = {nullptr, nullptr};
    Ctl* d_ctl = nullptr;
    double* d_ehist = nullptr;
    int ehist_stride = 0;
    int* d_active = nullptr;               // one counter per sweep of a captured chunk
    int* d_chunks = nullptr;               // chunks run by the device-side relaxation loop
    int gsweeps = kDefaultGraphSweeps;     // sweeps per captured chunk (loop condition once per chunk)
    double* d_scratch = nullptr;
    double* d_H = nullptr;                 // one exact energy per entry
    bool f64 = false;                      // lattice of double2 and d_acc of doubles (MPR_PREC_F64)
    // tile path (fused sweeps over shared-memory tiles, two lattice buffers)
    bool tiled = false;
    float2* d_lat2 = nullptr;
    TileDesc* d_tiles = nullptr;           // raster order per grid (index = TileDesc::t)
    TileDesc* d_tiles_ord = nullptr;       // the same, each grid's heaviest first (relaxation order)
    unsigned* d_tdone = nullptr;           // per tile: sweeps completed
    int* d_live = nullptr;                 // grids still relaxing during a relaxation launch
    int ntiles = 0;
    TileCnt* d_cnts = nullptr;
    uint16_t* d_lists = nullptr;
    float* d_tacc = nullptr;
    unsigned long long* d_gsum = nullptr;   // per grid and slot: fixed-point energy change, acceptance count
    unsigned* d_sched = nullptr;            // item counter, blocks-out counter, a flag nothing sets
    unsigned* d_ticket = nullptr;
    CUtensorMap* d_maps = nullptr;
    int* d_err = nullptr;
    int tcfg = 0;                          // compiled tile configuration in use
    const uint8_t* mask_base = nullptr;    // masks of the grids (concatenated), or null
    int all_free = 0;
    std::map<std::tuple<int, int, int, int, float>, cudaGraphExec_t> graphs;
};

}  // namespace

struct GridInfo {                          // host view of one grid of a context
    int W = 0, H = 0;
    long long site0 = 0;                   // offset in the concatenated [H][W] buffers
    double zmin = 0, zmax = 0, scale = 0;  // Eq. 1
    long long n_samples = 0;
    double e_s = 0;                        // Eq. 4
    long long n_sp = 0;
    double T = 0;
};

struct StripInfo {                         // a context that holds one row strip of a larger grid
    bool on = false;
    int row0 = 0, H_global = 0;            // grid row of the block's row 0, grid height
    int h0 = 0, h1 = 0;                    // rows of other strips above / below the own rows
    double pair_sum = 0, pair_cnt = 0;     // Eq. 4 terms of the own sample pairs
    double P_total = 0;                    // gap sites of the whole grid
};

struct mpr_ctx {
    cudaStream_t st = nullptr;
    StripInfo strip;
    int* d_stop = nullptr;                 // row strips: the control step's stop flag
    cudaStream_t cap = nullptr;            // private stream for graph capture
    mpr_params prm{};
    std::vector<GridInfo> g;               // one per grid
    long long n_sites = 0;                 // total sites of all grids
    float* d_z = nullptr;                  // concatenated inputs
    uint8_t* d_mask = nullptr;
    float* d_out = nullptr;                // concatenated staging for outputs
    bool T_set = false;
    Batch b;
    int* h_active = nullptr;               // pinned
    std::string err;
    int nfan = 0;                          // auxiliary streams in use (batches of 2 or more grids)
    cudaStream_t fan[kFan] = {};
    cudaEvent_t fan_ev[kFan + 1] = {};     // one per auxiliary stream, and the fork
};

namespace {

std::atomic<unsigned long long> g_launches{0};
std::mutex g_table_mu;
std::map<std::string, std::pair<std::vector<double>, std::vector<double>>> g_tables;

mpr_status fail(mpr_ctx* c, mpr_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MPR_ENOMEM : MPR_ECUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

// Device memory of the library's contexts comes from a stream-ordered memory pool per
// device owned by the library.  The pool keeps what is freed (release threshold:
// unlimited), so building and releasing contexts of similar sizes -- a serving loop over
// maps -- reuses that memory instead of going back to the driver; mpr_release_memory()
// hands it back.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t device_pool(cudaMemPool_t* pool) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *pool = g_pools[dev];
    return cudaSuccess;
}

// n elements of T from the pool, usable in the order of stream st
template <class T>
cudaError_t dalloc(T** p, size_t n, cudaStream_t st) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync((void**)p, n * sizeof(T), pool, st);
}

// returns p to the pool in the order of stream st (null is ignored)
void dfree(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// Pinned host slots of 4 ints for the contexts' small read-backs, cut from arenas that
// live as long as the process: building and freeing contexts in a serving loop then
// allocates and frees no pinned memory.
constexpr int kPinSlotInts = 4, kPinSlotsPerArena = 256;
std::mutex g_pin_mu;
std::vector<int*> g_pin_free;

// A batch's per-grid copies (inputs in, estimates out) go round-robin over up to kFan
// auxiliary streams that first wait for the context's stream; the context's stream then
// waits for all of them, so the grids' copies overlap instead of queueing one after
// another.  A single grid keeps everything on the context's stream.  Streams and events
// are made on first use and released by mpr_free.
cudaError_t fan_begin(mpr_ctx* ctx, int n) {
    if (n < 2 && !ctx->nfan) return cudaSuccess;
    if (!ctx->nfan) {
        const int k = std::min(kFan, n);
        cudaError_t e = cudaEventCreateWithFlags(&ctx->fan_ev[kFan], cudaEventDisableTiming);
        for (int i = 0; i < k && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&ctx->fan[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fan_ev[i], cudaEventDisableTiming);
            if (e == cudaSuccess) ctx->nfan = i + 1;
        }
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(ctx->fan_ev[kFan], ctx->st);
    for (int i = 0; i < ctx->nfan && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ctx->fan[i], ctx->fan_ev[kFan], 0);
    return e;
}
cudaStream_t fan_stream(const mpr_ctx* ctx, int i) { return ctx->nfan ? ctx->fan[i % ctx->nfan] : ctx->st; }
cudaError_t fan_end(mpr_ctx* ctx) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < ctx->nfan && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ctx->fan_ev[i], ctx->fan[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->st, ctx->fan_ev[i], 0);
    }
    return e;
}
void fan_release(mpr_ctx* ctx) {
    for (int i = 0; i < ctx->nfan; ++i) {
        cudaStreamDestroy(ctx->fan[i]);
        cudaEventDestroy(ctx->fan_ev[i]);
    }
    if (ctx->fan_ev[kFan]) cudaEventDestroy(ctx->fan_ev[kFan]);
    ctx->nfan = 0;
}

cudaError_t pinned_slot(int** out) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        int* arena = nullptr;
        const cudaError_t e = cudaMallocHost((void**)&arena, sizeof(int) * kPinSlotInts * kPinSlotsPerArena);
        if (e != cudaSuccess) return e;
        for (int i = kPinSlotsPerArena - 1; i >= 0; --i) g_pin_free.push_back(arena + i * kPinSlotInts);
    }
    *out = g_pin_free.back();
    g_pin_free.pop_back();
    return cudaSuccess;
}

void release_pinned_slot(int* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

void batch_free(Batch& b, cudaStream_t st) {
    for (auto& kv : b.graphs) cudaGraphExecDestroy(kv.second);
    b.graphs.clear();
    dfree(b.d_ents, st);
    dfree(b.d_lat, st);
    dfree(b.d_gaps, st);
    dfree(b.d_acc, st);
    for (int c = 0; c < 2; ++c) {
        dfree(b.d_work[c], st);
        dfree(b.d_part[c], st);
    }
    dfree(b.d_ctl, st);
    dfree(b.d_ehist, st);
    dfree(b.d_active, st);
    dfree(b.d_chunks, st);
    dfree(b.d_scratch, st);
    dfree(b.d_H, st);
    dfree(b.d_lat2, st);
    dfree(b.d_tiles, st);
    dfree(b.d_tiles_ord, st);
    dfree(b.d_tdone, st);
    dfree(b.d_live, st);
    dfree(b.d_cnts, st);
    dfree(b.d_lists, st);
    dfree(b.d_tacc, st);
    dfree(b.d_gsum, st);
    dfree(b.d_sched, st);
    dfree(b.d_ticket, st);
    dfree(b.d_maps, st);
    dfree(b.d_err, st);
    b = Batch();
}

// (Re)builds the tile tables of a batch for compiled configuration cfg: tile
// descriptors (raster order, and each grid's heaviest first), gap lists, per-tile
// accumulators and completion counters, per-grid totals and tickets, tensor maps.
mpr_status build_tiles(mpr_ctx* ctx, Batch& b, int cfg) {
    cudaStream_t st = ctx->st;
    if (cfg < 0 || cfg >= tile_config_count()) return fail(ctx, MPR_EINVAL, "tile configuration");
    const TileGeom g = tile_geom(cfg);
    dfree(b.d_tiles, st);
    dfree(b.d_tiles_ord, st);
    dfree(b.d_tdone, st);
    dfree(b.d_cnts, st);
    dfree(b.d_lists, st);
    dfree(b.d_tacc, st);
    dfree(b.d_gsum, st);
    dfree(b.d_sched, st);
    dfree(b.d_ticket, st);
    b.d_tiles = nullptr; b.d_tiles_ord = nullptr; b.d_tdone = nullptr; b.d_cnts = nullptr;
    b.d_lists = nullptr; b.d_tacc = nullptr; b.d_gsum = nullptr; b.d_sched = nullptr; b.d_ticket = nullptr;
    for (auto& kv : b.graphs) cudaGraphExecDestroy(kv.second);
    b.graphs.clear();
    std::vector<TileDesc> tiles;          // per grid ceil(H/th) x ceil(W/tw), row-major
    for (int e = 0; e < b.n_ent; ++e) {
        EntryDesc& E = b.ents[e];
        E.tile0 = (int)tiles.size();
        for (int y0 = 0; y0 < E.H; y0 += g.th)
            for (int x0 = 0; x0 < E.W; x0 += g.tw)
                tiles.push_back(TileDesc{e, y0, x0, 0, 0, 0, (int)tiles.size(), 0});
        E.ntiles = (int)tiles.size() - E.tile0;
    }
    CU(cudaMemcpyAsync(b.d_ents, b.ents.data(), b.n_ent * sizeof(EntryDesc), cudaMemcpyHostToDevice, st));
    b.ntiles = (int)tiles.size();
    CU(dalloc(&b.d_tiles, tiles.size(), st));
    CU(cudaMemcpyAsync(b.d_tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, st));
    CU(dalloc(&b.d_tiles_ord, tiles.size(), st));
    CU(dalloc(&b.d_tdone, tiles.size(), st));
    CU(dalloc(&b.d_cnts, tiles.size(), st));
    CU(dalloc(&b.d_lists, tiles.size() * (size_t)g.list, st));
    CU(dalloc(&b.d_tacc, tiles.size() * (size_t)g.acc, st));
    CU(dalloc(&b.d_gsum, (size_t)2 * kSlots * b.n_ent, st));
    CU(cudaMemsetAsync(b.d_gsum, 0, sizeof(unsigned long long) * 2 * kSlots * b.n_ent, st));
    CU(dalloc(&b.d_sched, 3, st));
    CU(cudaMemsetAsync(b.d_sched, 0, sizeof(unsigned) * 3, st));
    CU(dalloc(&b.d_ticket, (size_t)kSlots * b.n_ent, st));
    CU(cudaMemsetAsync(b.d_ticket, 0, sizeof(unsigned) * kSlots * b.n_ent, st));
    CU(launch_tile_lists(cfg, b.d_tiles, b.ntiles, b.d_ents, b.mask_base, b.all_free, b.d_lists,
                         b.d_cnts, st));
    // the relaxation's order (heaviest tiles first), from the counts just listed
    unsigned* d_hist = nullptr;
    CU(dalloc(&d_hist, (size_t)256 * b.n_ent, st));
    CU(launch_tile_order(b.d_tiles, b.ntiles, b.d_ents, b.n_ent, cfg, d_hist, b.d_tiles_ord, st));
    dfree(d_hist, st);
    if (b.d_ctl) CU(launch_tile_sync(b.d_tiles, b.ntiles, b.d_ctl, b.n_ent, b.d_tdone, st));
    CU(make_tile_maps(cfg, b.ents.data(), b.n_ent, b.d_lat, b.d_lat2, b.d_maps, st));
    tile_sweep_blocks(cfg);               // kernel attributes are set outside any capture
    CU(cudaGetLastError());
    b.tcfg = cfg;
    return MPR_OK;
}

// After the host changed the control state: every tile's completion counter and every
// grid's launch base follow the grids' sweep counters.
mpr_status sync_tiles(mpr_ctx* ctx, Batch& b) {
    if (!b.tiled) return MPR_OK;
    CU(launch_tile_sync(b.d_tiles, b.ntiles, b.d_ctl, b.n_ent, b.d_tdone, ctx->st));
    return MPR_OK;
}

// Lays out, packs and indexes a batch of grids.  all_free: every site is a gap.
mpr_status reset_relax(mpr_ctx* ctx, Batch& b);
mpr_status run_sweeps(mpr_ctx* ctx, Batch& b, int n, int mode, double a_fixed, bool acc);
mpr_status read_ctl(mpr_ctx* ctx, Batch& b, std::vector<Ctl>& out);

// same_grid: every entry is a chain of one grid (all read the grid at mask_base, site0 = 0).
mpr_status batch_build(mpr_ctx* ctx, Batch& b, const std::vector<GridIn>& grids, int all_free,
                       const uint8_t* mask_base, bool same_grid = false) {
    cudaStream_t st = ctx->st;
    b.f64 = ctx->prm.precision == MPR_PREC_F64;
    b.tiled = ctx->prm.exec_mode != MPR_EXEC_LIST && !b.f64 && ctx->prm.q == 0.5;
    const size_t wide = b.f64 ? 2 : 1;     // float2 slots per lattice element, floats per average
    const uint32_t k0 = (uint32_t)ctx->prm.seed, k1 = (uint32_t)(ctx->prm.seed >> 32);
    b.n_ent = (int)grids.size();
    b.ents.assign(b.n_ent, EntryDesc{});
    size_t lat = 0;
    long long site0 = 0;
    for (int e = 0; e < b.n_ent; ++e) {
        EntryDesc& E = b.ents[e];
        E.W = grids[e].W;
        E.H = grids[e].H;
        // >= W/2 + 3 columns, and at least one TMA box wide and high
        E.pitch = (std::max(E.W / 2 + 4, tile_max_cols()) + 31) & ~31;
        E.prows = std::max(E.H + 2, tile_max_rows());
        const size_t plane = (size_t)E.prows * E.pitch;
        E.plane[0] = (long long)lat;
        E.plane[1] = (long long)(lat + plane);
        lat += 2 * plane;
        E.chain = grids[e].chain;
        E.row_off = grids[e].row_off;
        E.q = ctx->prm.q;
        E.cQ = std::cos(kTwoPi * E.q);
        E.sQ = std::sin(kTwoPi * E.q);
        E.ngp = (double)E.W * (E.H - 1) + (double)E.H * (E.W - 1);
        E.site0 = same_grid ? 0 : site0;
        site0 += (long long)E.W * E.H;
    }
    b.lat_elems = lat;
    CU(dalloc(&b.d_lat, lat * wide, st));
    CU(cudaMemsetAsync(b.d_lat, 0, lat * wide * sizeof(float2), st));
    // gap lists: per-row counts of both colours (2 H ints per entry, all entries in one
    // buffer), scanned in place into row offsets; one read-back of the totals sizes the gap
    // buffer, then every entry's list is scattered from its own offsets.  Each entry's
    // pack, counts and scan on one stream of the batch's fan.
    std::vector<size_t> roff((size_t)b.n_ent + 1, 0);
    for (int e = 0; e < b.n_ent; ++e) roff[e + 1] = roff[e] + (size_t)2 * b.ents[e].H;
    int* d_rows = nullptr;
    int* d_tot = nullptr;
    CU(dalloc(&d_rows, roff[b.n_ent], st));
    CU(dalloc(&d_tot, (size_t)2 * b.n_ent, st));
    // several entries: each step one launch for all of them, from a table of set-up
    // records and an early copy of the entry table (layout fields; the gap counts follow)
    SetupRec* d_recs = nullptr;
    long long max_sites = 0;
    int max_rows = 0;
    CU(dalloc(&b.d_ents, b.n_ent, st));
    if (b.n_ent > 1) {
        std::vector<SetupRec> recs((size_t)b.n_ent);
        for (int e = 0; e < b.n_ent; ++e) {
            const EntryDesc& E = b.ents[e];
            recs[e] = SetupRec{grids[e].z, grids[e].mask, grids[e].zmin, grids[e].scale, (long long)E.W * E.H,
                               (int)roff[e], 0, 0};
            max_sites = std::max(max_sites, recs[e].n);
            max_rows = std::max(max_rows, E.H);
        }
        CU(dalloc(&d_recs, (size_t)b.n_ent, st));
        CU(cudaMemcpyAsync(d_recs, recs.data(), sizeof(SetupRec) * b.n_ent, cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(b.d_ents, b.ents.data(), b.n_ent * sizeof(EntryDesc), cudaMemcpyHostToDevice, st));
        CU(launch_pack_batch(b.d_ents, d_recs, b.n_ent, max_sites, b.d_lat, k0, k1, all_free, b.f64, st));
        CU(launch_gap_count_batch(b.d_ents, d_recs, b.n_ent, max_rows, all_free, d_rows, st));
        CU(launch_scan_rows_batch(b.d_ents, d_recs, b.n_ent, d_rows, d_tot, st));
    } else {
        CU(launch_pack(&b.ents[0], grids[0].z, grids[0].mask, grids[0].zmin, grids[0].scale, b.d_lat,
                       k0, k1, all_free, b.f64, st));
        CU(launch_gap_count(&b.ents[0], grids[0].mask, all_free, d_rows, st));
        CU(launch_scan_rows(d_rows, b.ents[0].H, 2, d_tot, st));
    }
    std::vector<int> tot((size_t)2 * b.n_ent);
    CU(cudaMemcpyAsync(tot.data(), d_tot, sizeof(int) * tot.size(), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    size_t ng = 0;
    for (int e = 0; e < b.n_ent; ++e) {
        EntryDesc& E = b.ents[e];
        E.ngap[0] = tot[2 * e];
        E.ngap[1] = tot[2 * e + 1];
        E.P = E.ngap[0] + E.ngap[1];
        E.gbase[0] = (long long)ng;
        E.gbase[1] = (long long)(ng + E.ngap[0]);
        ng += (size_t)E.P;
    }
    b.n_gaps = ng;
    CU(dalloc(&b.d_gaps, ng, st));
    CU(dalloc(&b.d_acc, ng * wide, st));
    if (b.n_ent > 1) {
        // the gap bases are in the host table now
        CU(cudaMemcpyAsync(b.d_ents, b.ents.data(), b.n_ent * sizeof(EntryDesc), cudaMemcpyHostToDevice, st));
        CU(launch_gap_scatter_batch(b.d_ents, d_recs, b.n_ent, max_rows, all_free, d_rows, b.d_gaps, st));
    } else {
        CU(launch_gap_scatter(&b.ents[0], grids[0].mask, all_free, d_rows, b.d_gaps, st));
    }
    dfree(d_rows, st);
    dfree(d_tot, st);
    dfree(d_recs, st);
    // sweep work lists
    const int chunk = kSweepThreads * kSweepItems;
    for (int c = 0; c < 2; ++c) {
        std::vector<BlockWork> w;
        for (int e = 0; e < b.n_ent; ++e) {
            EntryDesc& E = b.ents[e];
            E.blk0[c] = (int)w.size();
            const int nb = (E.ngap[c] + chunk - 1) / chunk;
            E.nblk[c] = nb;
            for (int i = 0; i < nb; ++i) w.push_back(BlockWork{e, i * chunk});
        }
        b.nblk[c] = (int)w.size();
        CU(dalloc(&b.d_work[c], w.size(), st));
        CU(dalloc(&b.d_part[c], w.size(), st));
        if (!w.empty())
            CU(cudaMemcpyAsync(b.d_work[c], w.data(), w.size() * sizeof(BlockWork),
                               cudaMemcpyHostToDevice, st));
    }
    CU(cudaMemcpyAsync(b.d_ents, b.ents.data(), b.n_ent * sizeof(EntryDesc), cudaMemcpyHostToDevice, st));
    if (b.tiled) {
        CU(dalloc(&b.d_lat2, lat, st));
        CU(cudaMemcpyAsync(b.d_lat2, b.d_lat, lat * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        CU(dalloc(&b.d_maps, (size_t)2 * b.n_ent, st));
        CU(dalloc(&b.d_err, 1, st));
        CU(cudaMemsetAsync(b.d_err, 0, sizeof(int), st));
        CU(dalloc(&b.d_live, 1, st));
        b.mask_base = mask_base;
        b.all_free = all_free;
        const mpr_status ts = build_tiles(ctx, b, ctx->prm.tile_cfg);
        if (ts != MPR_OK) return ts;
    }
    std::vector<Ctl> ctl(b.n_ent);
    for (int e = 0; e < b.n_ent; ++e) {
        std::memset(&ctl[e], 0, sizeof(Ctl));
        ctl[e].T = grids[e].T;
        ctl[e].a = 1.0;
        ctl[e].k = -1.0;
        ctl[e].half_qd = (float)(0.5 * kTwoPi * b.ents[e].q / 1.0);
        ctl[e].neg_inv_T = grids[e].T > 0.0 ? (float)(-1.0 / grids[e].T) : 0.0f;
    }
    CU(dalloc(&b.d_ctl, b.n_ent, st));
    for (auto& cc : ctl) ctl_set_go(cc);
    CU(cudaMemcpyAsync(b.d_ctl, ctl.data(), b.n_ent * sizeof(Ctl), cudaMemcpyHostToDevice, st));
    {
        const mpr_status ss = sync_tiles(ctx, b);
        if (ss != MPR_OK) return ss;
    }
    b.ehist_stride = ctx->prm.i_max + 2;
    CU(dalloc(&b.d_ehist, (size_t)b.n_ent * b.ehist_stride, st));
    CU(cudaMemsetAsync(b.d_ehist, 0, sizeof(double) * (size_t)b.n_ent * b.ehist_stride, st));
    CU(dalloc(&b.d_active, kMaxGraphSweeps, st));
    CU(dalloc(&b.d_chunks, 1, st));
    CU(dalloc(&b.d_scratch, kScratch + 8, st));
    CU(dalloc(&b.d_H, (size_t)b.n_ent, st));
    CU(cudaStreamSynchronize(st));
    return MPR_OK;
}

SweepArgs sweep_args(const mpr_ctx* ctx, const Batch& b, bool use_ctl_a, double a_fixed,
                     bool skip_stopped, bool acc) {
    SweepArgs A;
    std::memset(&A, 0, sizeof A);
    A.ents = b.d_ents;
    A.lat = b.d_lat;
    A.gaps = b.d_gaps;
    A.acc = acc ? b.d_acc : nullptr;
    A.ctl = b.d_ctl;
    for (int c = 0; c < 2; ++c) {
        A.part[c] = b.d_part[c];
        A.work[c] = b.d_work[c];
        A.nblk[c] = b.nblk[c];
    }
    A.use_ctl_a = use_ctl_a ? 1 : 0;
    A.half_qd_fixed = (float)(0.5 * kTwoPi * ctx->prm.q / a_fixed);
    A.skip_stopped = skip_stopped ? 1 : 0;
    A.or_mode = ctx->prm.or_mode;
    A.f64 = b.f64 ? 1 : 0;
    A.genq = ctx->prm.q != 0.5 ? 1 : 0;
    A.half_qd_fixed64 = 0.5 * kTwoPi * ctx->prm.q / a_fixed;
    A.rk = round_keys(ctx->prm.seed);
    return A;
}

// Limit of the tile kernels' waits between blocks, and the test switch that makes one
// wait expire (process-wide; mpr_debug_wait_limit).
std::atomic<unsigned long long> g_wait_ns{4000000000ull};
std::atomic<int> g_stall{0};
// Timestamp buffer of the sweep kernel (mpr_debug_trace): device words, their count.
std::atomic<unsigned long long*> g_trace{nullptr};
std::atomic<unsigned long long> g_trace_words{0};

// Timing of the sweep kernel (mpr_sweep_timing_start / _read): CUDA events around every
// tile-path sweep launch, on the context's stream, while enabled.
struct SweepTiming {
    std::mutex mu;
    bool on = false;
    double ms = 0.0;
    unsigned long long launches = 0;
    double site_sweeps = 0.0;    // sum over grids of sweeps x sites
    double gap_updates = 0.0;    // sum over grids of sweeps x gap sites
};
SweepTiming g_timing;

TileArgs tile_args(const mpr_ctx* ctx, const Batch& b, int mode, double a_fixed, bool acc, int nsweeps) {
    const mpr_params& p = ctx->prm;
    const bool relax = mode == CTL_RELAX;
    TileArgs T;
    std::memset(&T, 0, sizeof T);
    T.ents = b.d_ents;
    T.lat[0] = b.d_lat;
    T.lat[1] = b.d_lat2;
    T.maps = b.d_maps;
    T.err = b.d_err;
    T.desc = relax ? b.d_tiles_ord : b.d_tiles;
    T.lists = b.d_lists;
    T.acc = acc ? b.d_tacc : nullptr;
    T.ctl = b.d_ctl;
    T.gsum = b.d_gsum;
    T.ticket = b.d_ticket;
    T.sched = b.d_sched;
    T.tdone = b.d_tdone;
    T.live = b.d_live;
    T.ehist = b.d_ehist;
    T.ehist_stride = b.ehist_stride;
    T.ntiles = b.ntiles;
    T.n_ent = b.n_ent;
    T.nsweeps = nsweeps;
    T.cfg = b.tcfg;
    T.relax = relax ? 1 : 0;
    T.half_qd_fixed = (float)(0.5 * kTwoPi * p.q / a_fixed);
    T.or_mode = p.or_mode;
    T.rk = round_keys(p.seed);
    T.mode = mode;
    T.A_targ = p.A_targ;
    T.k_a = p.k_a;
    T.n_f = p.n_f;
    T.n_fit = p.n_fit;
    T.i_max = p.i_max;
    T.wait_ns = g_wait_ns.load();
    T.stall = g_stall.load();
    const unsigned long long words = g_trace_words.load();
    if (g_trace.load() && words >= 2ull * kTraceCtl) {
        T.trace = g_trace.load();
        T.trace_items = (words - 2ull * kTraceCtl) / kTraceWords;
    }
    return T;
}

// Sweeps per launch of the tile kernel (work items are counted in 32 bits).
int tile_launch_cap(const Batch& b) {
    const long long room = ((1LL << 31) - 65536LL) / std::max(1, b.ntiles);
    return (int)std::max(1LL, std::min<long long>(room, 1LL << 30));
}

// One launch of n tile sweeps on stream s, timed with CUDA events while the sweep timing
// is enabled (*ev_ms gets the launch's duration after the caller synchronised s).
mpr_status launch_tile_phase(mpr_ctx* ctx, Batch& b, cudaStream_t s, int n, int mode, double a_fixed,
                             bool acc, cudaEvent_t ev[2]) {
    const TileArgs T = tile_args(ctx, b, mode, a_fixed, acc, n);
    if (ev) CU(cudaEventRecord(ev[0], s));
    CU(launch_tile_sweep(T, ctx->prm.trig_mode, s));
    if (ev) CU(cudaEventRecord(ev[1], s));
    return MPR_OK;
}

mpr_status enqueue_sweeps(mpr_ctx* ctx, Batch& b, cudaStream_t s, int n, int mode, double a_fixed,
                          bool acc, bool count_active) {
    const bool relax = mode == CTL_RELAX;
    const SweepArgs A = sweep_args(ctx, b, relax, a_fixed, relax, acc);
    const mpr_params& p = ctx->prm;
    if (b.tiled) {
        const int cap = tile_launch_cap(b);
        for (int done = 0; done < n;) {
            const int k = std::min(cap, n - done);
            const mpr_status ls = launch_tile_phase(ctx, b, s, k, mode, a_fixed, acc, nullptr);
            if (ls != MPR_OK) return ls;
            done += k;
        }
        return MPR_OK;
    }
    if (count_active) CU(cudaMemsetAsync(b.d_active, 0, sizeof(int) * b.gsweeps, s));
    for (int i = 0; i < n; ++i) {
        CU(launch_half_sweep(A, 0, p.trig_mode, s));
        CU(launch_half_sweep(A, 1, p.trig_mode, s));
        CU(launch_control(b.d_ctl, b.d_part, b.d_ents, b.n_ent, mode, p.A_targ, p.k_a, p.n_f,
                          p.n_fit, p.i_max, b.d_ehist, b.ehist_stride,
                          count_active ? b.d_active + (i % b.gsweeps) : nullptr, b.f64, s));
    }
    return MPR_OK;
}

// The condition of the device-side relaxation loop, run after each chunk of S sweeps:
// continue while any grid is still relaxing (the control step of the chunk's last sweep
// counted them) and fewer than cap chunks have run.  Every grid stops by itself within
// i_max sweeps and cap covers that, so the loop ends even if a count went wrong.
__global__ void k_relax_loop_cond(cudaGraphConditionalHandle h, const int* __restrict__ active_last,
                                  int* __restrict__ chunks, int cap) {
    const int n = *chunks + 1;
    *chunks = n;
    cudaGraphSetConditional(h, (*active_last > 0 && n < cap) ? 1u : 0u);
}

// Relaxation graph: a WHILE node whose body is one chunk of S sweeps followed by the loop
// condition, so the whole relaxation runs without a host round trip per chunk.
// The stream the list path captures its graphs on, created on first use.
cudaError_t capture_stream(mpr_ctx* ctx) {
    if (ctx->cap) return cudaSuccess;
    return cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
}

mpr_status build_relax_graph(mpr_ctx* ctx, Batch& b, int S, int cap, double a_fixed, bool acc,
                             cudaGraphExec_t* out) {
    CU(capture_stream(ctx));
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    mpr_status s = MPR_OK;
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s = enqueue_sweeps(ctx, b, ctx->cap, S, CTL_RELAX, a_fixed, acc, true);
            if (s == MPR_OK) {
                k_relax_loop_cond<<<1, 1, 0, ctx->cap>>>(h, b.d_active + (S - 1), b.d_chunks, cap);
                e = cudaGetLastError();
            }
            cudaGraph_t captured = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(ctx->cap, &captured);
            if (e == cudaSuccess) e = ce;
        }
    }
    if (s == MPR_OK && e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (s != MPR_OK) return s;
    CU(e);
    return MPR_OK;
}

// List path: runs n sweeps through a cached CUDA graph of b.gsweeps sweeps (plus a tail);
// relaxation (n ignored) through the device-side loop of build_relax_graph.  The tile path
// runs each phase as one persistent launch (run_tile_sweeps).
mpr_status run_tile_sweeps(mpr_ctx* ctx, Batch& b, int n, int mode, double a_fixed, bool acc);

mpr_status run_sweeps(mpr_ctx* ctx, Batch& b, int n, int mode, double a_fixed, bool acc) {
    if (b.tiled) return run_tile_sweeps(ctx, b, n, mode, a_fixed, acc);
    const int S = b.gsweeps;
    const bool relax = mode == CTL_RELAX;
    if (n <= 0 && !relax) return MPR_OK;
    auto key = std::make_tuple(mode, acc ? 1 : 0, S, ctx->prm.trig_mode, (float)a_fixed);
    cudaGraphExec_t exec = nullptr;
    const int cap_chunks = (int)std::min<long long>((long long)ctx->prm.i_max / S + 4, 1LL << 30);
    if (relax) {
        auto it = b.graphs.find(key);
        if (it == b.graphs.end()) {
            const mpr_status s = build_relax_graph(ctx, b, S, cap_chunks, a_fixed, acc, &exec);
            if (s != MPR_OK) return s;
            b.graphs[key] = exec;
        } else {
            exec = it->second;
        }
    } else if (n >= S) {
        auto it = b.graphs.find(key);
        if (it == b.graphs.end()) {
            CU(capture_stream(ctx));
            CU(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
            mpr_status s = enqueue_sweeps(ctx, b, ctx->cap, S, mode, a_fixed, acc, relax);
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(ctx->cap, &g);
            if (s != MPR_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            CU(ce);
            cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            CU(ie);
            b.graphs[key] = exec;
        } else {
            exec = it->second;
        }
    }
    if (relax) {
        // chunks until no entry is still relaxing (each stops itself on the slope test or
        // on i_max), decided on the device; the host reads the chunk count once at the end
        CU(cudaMemsetAsync(b.d_chunks, 0, sizeof(int), ctx->st));
        CU(cudaGraphLaunch(exec, ctx->st));
        CU(cudaMemcpyAsync(ctx->h_active, b.d_chunks, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
        const int chunks = *ctx->h_active;
        count_launches((unsigned long long)chunks * ((b.tiled ? 1ull : 3ull) * S + 1ull), nullptr);
        if (chunks >= cap_chunks) {
            // the cap ends the loop only if some grid was still relaxing after i_max sweeps
            std::vector<Ctl> c;
            const mpr_status rs = read_ctl(ctx, b, c);
            if (rs != MPR_OK) return rs;
            for (const Ctl& x : c)
                if (!x.stop) return fail(ctx, MPR_ETIMEOUT, "relaxation did not stop within i_max sweeps");
        }
        return MPR_OK;
    }
    int done = 0;
    for (; exec && done + S <= n; done += S) {
        CU(cudaGraphLaunch(exec, ctx->st));
        count_launches((b.tiled ? 1ull : 3ull) * S, nullptr);
    }
    return enqueue_sweeps(ctx, b, ctx->st, n - done, mode, a_fixed, acc, false);
}

// Tile path: a whole phase is one launch of the persistent sweep kernel.  The relaxation
// is one launch of up to i_max + 1 sweeps that ends as soon as every grid has stopped (the
// control steps count down the grids still relaxing); a fixed-window phase of n sweeps is
// one launch.  (More launches only if a phase has more sweeps than one launch can count.)
// The host then reads the error flag, and the count of grids still relaxing, once.
mpr_status run_tile_sweeps(mpr_ctx* ctx, Batch& b, int n, int mode, double a_fixed, bool acc) {
    const bool relax = mode == CTL_RELAX;
    if (!relax && n <= 0) return MPR_OK;
    const int cap = tile_launch_cap(b);
    const long long total = relax ? (long long)ctx->prm.i_max + 1 : (long long)n;
    bool timing = false;
    {
        std::lock_guard<std::mutex> lk(g_timing.mu);
        timing = g_timing.on;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (timing) {
        CU(cudaEventCreate(&ev[0]));
        CU(cudaEventCreate(&ev[1]));
    }
    std::vector<Ctl> c0;
    if (timing && relax) {
        const mpr_status rs = read_ctl(ctx, b, c0);
        if (rs != MPR_OK) return rs;
    }
    if (relax) CU(launch_count_live(b.d_ctl, b.n_ent, b.d_live, ctx->st));
    mpr_status s = MPR_OK;
    long long done = 0;
    while (s == MPR_OK && done < total) {
        const int k = (int)std::min<long long>(cap, total - done);
        s = launch_tile_phase(ctx, b, ctx->st, k, mode, a_fixed, acc, timing ? ev : nullptr);
        if (s != MPR_OK) break;
        done += k;
        int* h = ctx->h_active;
        cudaError_t e = cudaMemcpyAsync(h, b.d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
        if (e == cudaSuccess && relax) e = cudaMemcpyAsync(h + 1, b.d_live, sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
        if (e != cudaSuccess) { s = fail(ctx, MPR_ECUDA, std::string("tile sweeps: ") + cudaGetErrorString(e)); break; }
        if (timing) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            double site_sweeps = 0.0, gap_updates = 0.0;
            std::vector<Ctl> c1;
            if (relax) s = read_ctl(ctx, b, c1);
            for (int g = 0; g < b.n_ent && s == MPR_OK; ++g) {
                const double sw = relax ? (double)(c1[g].sweep - c0[g].sweep) : (double)k;
                site_sweeps += sw * (double)b.ents[g].W * (double)b.ents[g].H;
                gap_updates += sw * (double)b.ents[g].P;
            }
            if (relax && s == MPR_OK) c0 = c1;
            std::lock_guard<std::mutex> lk(g_timing.mu);
            g_timing.ms += ms;
            g_timing.launches += 1;
            g_timing.site_sweeps += site_sweeps;
            g_timing.gap_updates += gap_updates;
        }
        if (h[0]) { s = fail(ctx, MPR_ETIMEOUT, "a bounded wait of the sweep kernel expired"); break; }
        if (relax && h[1] <= 0) break;
        if (relax && done >= total) s = fail(ctx, MPR_ETIMEOUT, "relaxation did not stop within i_max sweeps");
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    return s;
}

// Recomputes Eq. 2 for every entry and makes it the tracked energy.
mpr_status read_ctl(mpr_ctx* ctx, Batch& b, std::vector<Ctl>& out);

// Lattice buffer that holds entry e's current state (the tile path alternates buffers).
float2* lat_cur(const Batch& b, const Ctl& c) { return (b.tiled && c.cur) ? b.d_lat2 : b.d_lat; }

mpr_status reset_tracked_energy(mpr_ctx* ctx, Batch& b) {
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, b, c);
    if (s != MPR_OK) return s;
    if (b.n_ent >= 2) {
        // every grid in one launch (each with the single-grid launch's blocks and order)
        int max_w = 1, max_h = 1;
        for (const EntryDesc& E : b.ents) {
            max_w = std::max(max_w, E.W);
            max_h = std::max(max_h, E.H);
        }
        double* d_part = nullptr;
        CU(dalloc(&d_part, (size_t)b.n_ent * kScratch, ctx->st));
        CU(launch_energy_batch(b.d_ents, b.n_ent, max_w, max_h, b.d_lat, b.d_lat2, b.d_ctl, b.tiled ? 1 : 0,
                               d_part, kScratch, b.d_H, b.f64, ctx->st));
        dfree(d_part, ctx->st);
    } else {
        CU(launch_energy(&b.ents[0], lat_cur(b, c[0]), b.d_scratch, kScratch, b.d_H, b.f64, ctx->st));
    }
    CU(launch_set_tracked_energy(b.d_ctl, b.d_H, b.n_ent, ctx->st));
    return MPR_OK;
}

mpr_status read_ctl(mpr_ctx* ctx, Batch& b, std::vector<Ctl>& out) {
    out.resize(b.n_ent);
    CU(cudaMemcpyAsync(out.data(), b.d_ctl, sizeof(Ctl) * b.n_ent, cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

// Resets the relaxation state of every entry (Algorithm 2 steps 2.1, 2.3, 2.4).
mpr_status reset_relax(mpr_ctx* ctx, Batch& b) {
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, b, c);
    if (s != MPR_OK) return s;
    for (int e = 0; e < b.n_ent; ++e) {
        c[e].i = 0;
        c[e].k = -1.0;
        c[e].a = 1.0;
        c[e].stop = b.ents[e].P == 0 ? 1 : 0;
        c[e].converged = 0;
        c[e].esum = 0.0;
        c[e].nsamp = 0;
        c[e].half_qd = (float)(0.5 * kTwoPi * b.ents[e].q / 1.0);
    }
    for (auto& cc : c) ctl_set_go(cc);
    CU(cudaMemcpyAsync(b.d_ctl, c.data(), sizeof(Ctl) * b.n_ent, cudaMemcpyHostToDevice, ctx->st));
    return reset_tracked_energy(ctx, b);
}

std::string table_key(const mpr_params& p, int W, int H) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "%d|%d|%llu|%.17g|%.17g|%.17g|%d|%d|%d|%d|%d|%.17g|%d|%.17g|%.17g|%d|%d",
                  W, H, (unsigned long long)p.seed, p.q, p.A_targ, p.k_a, p.n_f, p.n_fit, p.i_max,
                  p.or_mode, p.trig_mode, p.a_eq, p.KT, p.T_min, p.T_max, p.M_T, p.precision);
    return buf;
}

// Eq. 5 tables: for each requested lattice shape, KT all-free lattices (one per T_k),
// all shapes in one batch; relaxed by Algorithm 2 step 5 at their own T_k, then M_T
// sweeps at a_eq averaging the specific energy.
mpr_status build_tables(mpr_ctx* ctx, const std::vector<std::pair<int, int>>& shapes,
                        std::vector<std::vector<double>>& Tk, std::vector<std::vector<double>>& ek) {
    const mpr_params& p = ctx->prm;
    std::vector<double> T(p.KT);
    for (int k = 0; k < p.KT; ++k)
        T[k] = p.T_min * std::pow(p.T_max / p.T_min, (double)k / (double)(p.KT - 1));
    std::vector<GridIn> g;
    for (size_t sh = 0; sh < shapes.size(); ++sh)
        for (int k = 0; k < p.KT; ++k)
            g.push_back(GridIn{shapes[sh].first, shapes[sh].second, nullptr, nullptr,
                               0x80000000u + (uint32_t)(sh * p.KT + k), T[k], 0.0, 0.0});
    Batch tb;
    mpr_status s = batch_build(ctx, tb, g, 1, nullptr);
    if (s == MPR_OK) s = reset_relax(ctx, tb);
    if (s == MPR_OK) s = run_sweeps(ctx, tb, 0, CTL_RELAX, 1.0, false);
    if (s == MPR_OK) s = run_sweeps(ctx, tb, p.M_T, CTL_SAMPLE, p.a_eq, false);
    std::vector<Ctl> c;
    if (s == MPR_OK) s = read_ctl(ctx, tb, c);
    if (s == MPR_OK) {
        Tk.assign(shapes.size(), T);
        ek.assign(shapes.size(), std::vector<double>(p.KT));
        for (size_t sh = 0; sh < shapes.size(); ++sh)
            for (int k = 0; k < p.KT; ++k) {
                const Ctl& x = c[sh * p.KT + k];
                ek[sh][k] = x.nsamp ? x.esum / x.nsamp : 0.0;
            }
    }
    batch_free(tb, ctx->st);
    return s;
}

// Shape of the unconditional lattices used for a grid's table: the grid's sides capped
// at T_cap; in batches of several grids also rounded down to a power of two (at least
// 32) so that grids of similar size share one table.
std::pair<int, int> table_shape(const mpr_params& p, int W, int H, bool batch) {
    auto side = [&](int v) {
        int t = p.T_cap > 0 ? std::min(v, p.T_cap) : v;
        if (batch && t >= 32) {
            int q = 32;
            while (q * 2 <= t) q *= 2;
            t = q;
        }
        return t;
    };
    return {side(W), side(H)};
}

// T-hat = argmin_T |e_s - e(T, L)|: first bracketing interval from the lowest T,
// linear in T inside it; otherwise the closest table point.
double invert_T(const std::vector<double>& Tk, const std::vector<double>& ek, double e_s) {
    const int K = (int)Tk.size();
    if (e_s <= ek[0]) return Tk[0];
    for (int k = 0; k + 1 < K; ++k)
        if (ek[k] <= e_s && e_s < ek[k + 1])
            return Tk[k] + (e_s - ek[k]) * (Tk[k + 1] - Tk[k]) / (ek[k + 1] - ek[k]);
    int best = 0;
    for (int k = 1; k < K; ++k)
        if (std::fabs(e_s - ek[k]) < std::fabs(e_s - ek[best])) best = k;
    return Tk[best];
}

}  // namespace

extern "C" {

void mpr_default_params(mpr_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->seed = 0;
    p->q = 0.5;
    p->A_targ = 0.3;
    p->k_a = 3.0;
    p->n_f = 5;
    p->n_fit = 20;
    p->i_max = 10000;
    p->M = 100;
    p->or_mode = MPR_OR_CONSERVING;
    p->trig_mode = MPR_TRIG_ACCURATE;
    p->a_eq = 1.0;
    p->KT = 16;
    p->T_min = 1e-4;
    p->T_max = 1.0;
    p->T_cap = 1024;
    p->M_T = 100;
    p->exec_mode = MPR_EXEC_AUTO;
    p->chain = 0;
    p->tile_cfg = 0;
}

const char* mpr_status_string(mpr_status s) {
    switch (s) {
        case MPR_OK: return "MPR_OK";
        case MPR_EINVAL: return "MPR_EINVAL";
        case MPR_ENOMEM: return "MPR_ENOMEM";
        case MPR_ECUDA: return "MPR_ECUDA";
        case MPR_ENODATA: return "MPR_ENODATA";
        case MPR_ENOPAIRS: return "MPR_ENOPAIRS";
        case MPR_ETIMEOUT: return "MPR_ETIMEOUT";
        case MPR_ENOTEQUIL: return "MPR_ENOTEQUIL";
        case MPR_ESTATE: return "MPR_ESTATE";
    }
    return "MPR_UNKNOWN";
}

const char* mpr_last_error(const mpr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void mpr_free(mpr_ctx* ctx) {
    if (!ctx) return;
    // the work already enqueued finishes before its buffers and graphs go (the frees are
    // stream-ordered on the caller's stream)
    cudaStreamSynchronize(ctx->st);
    for (int i = 0; i < ctx->nfan; ++i) cudaStreamSynchronize(ctx->fan[i]);   // an early return may leave work there
    batch_free(ctx->b, ctx->st);
    dfree(ctx->d_z, ctx->st);
    dfree(ctx->d_mask, ctx->st);
    dfree(ctx->d_out, ctx->st);
    dfree(ctx->d_stop, ctx->st);
    release_pinned_slot(ctx->h_active);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    fan_release(ctx);
    delete ctx;
}

static mpr_status check_params(const mpr_params* p, std::string& why) {
    if (!(p->q > 0.0 && p->q <= 0.5)) { why = "q must lie in (0, 1/2]"; return MPR_EINVAL; }
    if (p->q != 0.5 && (p->exec_mode == MPR_EXEC_TILE || p->or_mode == MPR_OR_LITERAL)) {
        why = "q < 1/2 runs the LIST kernels with the conserving or no reflection";
        return MPR_EINVAL;
    }
    if (!(p->A_targ >= 0.0 && p->A_targ <= 1.0)) { why = "A_targ must lie in [0, 1]"; return MPR_EINVAL; }
    if (!(p->k_a > 0.0)) { why = "k_a must be > 0"; return MPR_EINVAL; }
    if (p->n_f < 1 || p->n_fit < 2 || p->i_max < 0 || p->M < 1) { why = "n_f >= 1, n_fit >= 2, i_max >= 0, M >= 1"; return MPR_EINVAL; }
    if (p->i_max > 100000000) { why = "i_max too large"; return MPR_EINVAL; }
    if (p->or_mode != MPR_OR_CONSERVING && p->or_mode != MPR_OR_LITERAL && p->or_mode != MPR_OR_NONE) {
        why = "or_mode";
        return MPR_EINVAL;
    }
    if (p->trig_mode != MPR_TRIG_ACCURATE && p->trig_mode != MPR_TRIG_FAST) { why = "trig_mode"; return MPR_EINVAL; }
    if (!(p->a_eq >= 1.0)) { why = "a_eq must be >= 1"; return MPR_EINVAL; }
    if (p->tile_cfg < 0 || p->tile_cfg >= tile_config_count()) { why = "tile_cfg"; return MPR_EINVAL; }
    if (p->exec_mode != MPR_EXEC_AUTO && p->exec_mode != MPR_EXEC_LIST && p->exec_mode != MPR_EXEC_TILE) { why = "exec_mode"; return MPR_EINVAL; }
    if (p->KT < 2 || !(p->T_min > 0.0) || !(p->T_max > p->T_min) || p->M_T < 1 || p->T_cap < 0) { why = "table parameters"; return MPR_EINVAL; }
    if (p->precision != MPR_PREC_F32 && p->precision != MPR_PREC_F64) { why = "precision"; return MPR_EINVAL; }
    if (p->precision == MPR_PREC_F64 && (p->exec_mode == MPR_EXEC_TILE || p->trig_mode != MPR_TRIG_ACCURATE)) {
        why = "MPR_PREC_F64 runs the LIST kernels with accurate transcendentals";
        return MPR_EINVAL;
    }
    return MPR_OK;
}

// Copies the grids in, maps them (Eq. 1), builds the lattice batch and computes Eq. 4.
static mpr_status init_grids(mpr_ctx** out, int n, const float* const* z, const uint8_t* const* mask,
                             const int* W, const int* H, const mpr_params* params, void* stream) {
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    if (n < 1 || !z || !mask || !W || !H) return MPR_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!z[i] || !mask[i] || W[i] < 1 || H[i] < 1 || H[i] > 65535 || (W[i] + 1) / 2 > 65535)
            return MPR_EINVAL;
    mpr_ctx* ctx = new mpr_ctx();
    if (params) ctx->prm = *params; else mpr_default_params(&ctx->prm);
    std::string why;
    if (check_params(&ctx->prm, why) != MPR_OK) { delete ctx; return MPR_EINVAL; }
    ctx->st = (cudaStream_t)stream;
    ctx->g.resize(n);
    long long site0 = 0;
    for (int i = 0; i < n; ++i) {
        ctx->g[i].W = W[i];
        ctx->g[i].H = H[i];
        ctx->g[i].site0 = site0;
        site0 += (long long)W[i] * H[i];
    }
    ctx->n_sites = site0;
    auto bail = [&](mpr_status s) { mpr_free(ctx); return s; };
#define CUI(call) do { if ((call) != cudaSuccess) { cudaGetLastError(); return bail(MPR_ECUDA); } } while (0)
    CUI(pinned_slot(&ctx->h_active));
    const size_t N = (size_t)site0;
    if (dalloc(&ctx->d_z, N, ctx->st) != cudaSuccess || dalloc(&ctx->d_mask, N, ctx->st) != cudaSuccess ||
        dalloc(&ctx->d_out, N, ctx->st) != cudaSuccess) { cudaGetLastError(); return bail(MPR_ENOMEM); }
    // Eq. 1 extremes, per grid (each grid's input copies and extremes on one stream of the
    // batch's fan)
    unsigned* d_keys = nullptr;
    unsigned long long* d_ns = nullptr;
    CUI(dalloc(&d_keys, (size_t)2 * n, ctx->st));
    CUI(dalloc(&d_ns, (size_t)n, ctx->st));
    std::vector<unsigned> keys((size_t)2 * n);
    for (int i = 0; i < n; ++i) {                 // identities of the min / max keys
        keys[2 * i] = 0xFFFFFFFFu;
        keys[2 * i + 1] = 0u;
    }
    CUI(cudaMemcpyAsync(d_keys, keys.data(), sizeof(unsigned) * 2 * n, cudaMemcpyHostToDevice, ctx->st));
    CUI(cudaMemsetAsync(d_ns, 0, sizeof(unsigned long long) * n, ctx->st));
    // set-up records of the grids (several grids: each step is one launch for all of them)
    std::vector<SetupRec> recs((size_t)n);
    long long max_sites = 0;
    for (int i = 0; i < n; ++i) {
        recs[i] = SetupRec{ctx->d_z + ctx->g[i].site0, ctx->d_mask + ctx->g[i].site0, 0.0, 0.0,
                           (long long)W[i] * H[i], 0, 0, 0};
        max_sites = std::max(max_sites, recs[i].n);
    }
    SetupRec* d_recs = nullptr;
    if (n > 1) {
        CUI(dalloc(&d_recs, (size_t)n, ctx->st));
        CUI(cudaMemcpyAsync(d_recs, recs.data(), sizeof(SetupRec) * n, cudaMemcpyHostToDevice, ctx->st));
    }
    CUI(fan_begin(ctx, n));
    for (int i = 0; i < n; ++i) {
        const size_t ni = (size_t)W[i] * H[i];
        const cudaStream_t si = fan_stream(ctx, i);
        CUI(cudaMemcpyAsync(ctx->d_z + ctx->g[i].site0, z[i], ni * sizeof(float), cudaMemcpyDefault, si));
        CUI(cudaMemcpyAsync(ctx->d_mask + ctx->g[i].site0, mask[i], ni, cudaMemcpyDefault, si));
        if (n == 1)
            CUI(launch_minmax(ctx->d_z + ctx->g[i].site0, ctx->d_mask + ctx->g[i].site0,
                              (long long)W[i] * H[i], d_keys + 2 * i, d_ns + i, si));
    }
    CUI(fan_end(ctx));
    if (n > 1) CUI(launch_minmax_batch(d_recs, n, max_sites, d_keys, d_ns, ctx->st));
    std::vector<unsigned long long> ns((size_t)n);
    CUI(cudaMemcpyAsync(keys.data(), d_keys, sizeof(unsigned) * 2 * n, cudaMemcpyDeviceToHost, ctx->st));
    CUI(cudaMemcpyAsync(ns.data(), d_ns, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx->st));
    CUI(cudaStreamSynchronize(ctx->st));
    dfree(d_keys, ctx->st);
    dfree(d_ns, ctx->st);
    auto unkey = [](unsigned k) {
        const unsigned b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
        float f;
        std::memcpy(&f, &b, sizeof f);
        return (double)f;
    };
    std::vector<GridIn> gi(n);
    for (int i = 0; i < n; ++i) {
        GridInfo& G = ctx->g[i];
        G.n_samples = (long long)ns[i];
        if (ns[i] < 2) return bail(MPR_ENODATA);
        G.zmin = unkey(keys[2 * i]);
        G.zmax = unkey(keys[2 * i + 1]);
        if (!(G.zmax > G.zmin) || !std::isfinite(G.zmin) || !std::isfinite(G.zmax)) return bail(MPR_ENODATA);
        G.scale = kTwoPi / (G.zmax - G.zmin);
        gi[i] = GridIn{W[i], H[i], ctx->d_z + G.site0, ctx->d_mask + G.site0,
                       ctx->prm.chain + (uint32_t)i, 0.0, G.zmin, G.scale};
    }
    {
        const mpr_status bs = batch_build(ctx, ctx->b, gi, 0, ctx->d_mask);
        if (bs != MPR_OK) return bail(bs);
    }
    // Eq. 4, per grid: each grid's per-block partials in its own slots of one buffer (one
    // block per row, at most 1024), read back once and added in block order on the host
    std::vector<size_t> poff((size_t)n + 1, 0);
    for (int i = 0; i < n; ++i) poff[i + 1] = poff[i] + (size_t)std::min(std::max(H[i], 1), 1024);
    double* d_ps = nullptr;
    unsigned long long* d_pc = nullptr;
    CUI(dalloc(&d_ps, poff[n], ctx->st));
    CUI(dalloc(&d_pc, poff[n], ctx->st));
    if (n == 1) {
        GridInfo& G = ctx->g[0];
        int np = 0;
        CUI(launch_sample_energy(&ctx->b.ents[0], ctx->d_z + G.site0, ctx->d_mask + G.site0, G.scale,
                                 ctx->prm.q, d_ps, d_pc, &np, ctx->prm.precision == MPR_PREC_F64, ctx->st));
        if ((size_t)np != poff[1]) return bail(MPR_ECUDA);
    } else {
        int max_parts = 0;
        for (int i = 0; i < n; ++i) {
            recs[i].scale = ctx->g[i].scale;
            recs[i].poff = (int)poff[i];
            recs[i].nparts = (int)(poff[i + 1] - poff[i]);
            max_parts = std::max(max_parts, recs[i].nparts);
        }
        CUI(cudaMemcpyAsync(d_recs, recs.data(), sizeof(SetupRec) * n, cudaMemcpyHostToDevice, ctx->st));
        CUI(launch_sample_energy_batch(ctx->b.d_ents, d_recs, n, max_parts, ctx->prm.q, d_ps, d_pc,
                                       ctx->prm.precision == MPR_PREC_F64, ctx->st));
    }
    std::vector<double> ps(poff[n]);
    std::vector<unsigned long long> pc(poff[n]);
    CUI(cudaMemcpyAsync(ps.data(), d_ps, sizeof(double) * poff[n], cudaMemcpyDeviceToHost, ctx->st));
    CUI(cudaMemcpyAsync(pc.data(), d_pc, sizeof(unsigned long long) * poff[n], cudaMemcpyDeviceToHost, ctx->st));
    CUI(cudaStreamSynchronize(ctx->st));
    dfree(d_ps, ctx->st);
    dfree(d_pc, ctx->st);
    dfree(d_recs, ctx->st);
    for (int i = 0; i < n; ++i) {
        GridInfo& G = ctx->g[i];
        double sum = 0.0;
        unsigned long long cnt = 0;
        for (size_t k = poff[i]; k < poff[i + 1]; ++k) { sum += ps[k]; cnt += pc[k]; }
        G.n_sp = (long long)cnt;
        G.e_s = cnt ? -sum / (double)cnt : 0.0;
    }
#undef CUI
    *out = ctx;
    return MPR_OK;
}

mpr_status mpr_init(mpr_ctx** out, const float* z, const uint8_t* mask, int W, int H,
                    const mpr_params* params, void* cuda_stream) {
    return init_grids(out, 1, &z, &mask, &W, &H, params, cuda_stream);
}

mpr_status mpr_init_batch(mpr_ctx** out, int n, const float* const* z, const uint8_t* const* mask,
                          const int* W, const int* H, const mpr_params* params, void* cuda_stream) {
    return init_grids(out, n, z, mask, W, H, params, cuda_stream);
}

int mpr_batch_size(const mpr_ctx* ctx) { return ctx ? (int)ctx->g.size() : 0; }

static mpr_status set_T_all(mpr_ctx* ctx, const std::vector<double>& T) {
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    for (size_t i = 0; i < c.size(); ++i) {
        c[i].T = T[i];
        c[i].neg_inv_T = (float)(-1.0 / T[i]);
        ctx->g[i].T = T[i];
    }
    for (auto& cc : c) ctl_set_go(cc);
    CU(cudaMemcpyAsync(ctx->b.d_ctl, c.data(), sizeof(Ctl) * c.size(), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    ctx->T_set = true;
    return MPR_OK;
}

mpr_status mpr_set_T(mpr_ctx* ctx, double T) {
    if (!ctx) return MPR_EINVAL;
    if (!(T > 0.0) || !std::isfinite(T)) return fail(ctx, MPR_EINVAL, "T must be positive");
    return set_T_all(ctx, std::vector<double>(ctx->g.size(), T));
}

// T-hat of e_s from the e(T, L) tables of the given lattice shapes (built, all together, for
// the shapes not cached yet).
static mpr_status temperatures_for(mpr_ctx* ctx, const std::vector<std::pair<int, int>>& shapes,
                                   const std::vector<double>& e_s, std::vector<double>& T) {
    const mpr_params& p = ctx->prm;
    std::vector<std::pair<int, int>> need;
    for (const auto& sh : shapes) {
        std::lock_guard<std::mutex> lk(g_table_mu);
        if (!g_tables.count(table_key(p, sh.first, sh.second)) &&
            std::find(need.begin(), need.end(), sh) == need.end())
            need.push_back(sh);
    }
    if (!need.empty()) {
        std::vector<std::vector<double>> Tk, ek;
        mpr_status s = build_tables(ctx, need, Tk, ek);
        if (s != MPR_OK) return s;
        std::lock_guard<std::mutex> lk(g_table_mu);
        for (size_t i = 0; i < need.size(); ++i)
            g_tables[table_key(p, need[i].first, need[i].second)] = std::make_pair(Tk[i], ek[i]);
    }
    T.resize(shapes.size());
    for (size_t i = 0; i < shapes.size(); ++i) {
        std::pair<std::vector<double>, std::vector<double>> tab;
        {
            std::lock_guard<std::mutex> lk(g_table_mu);
            tab = g_tables[table_key(p, shapes[i].first, shapes[i].second)];
        }
        T[i] = invert_T(tab.first, tab.second, e_s[i]);
    }
    return MPR_OK;
}

mpr_status mpr_estimate_T(mpr_ctx* ctx, double* T_hat, double* e_s) {
    if (!ctx) return MPR_EINVAL;
    const mpr_params& p = ctx->prm;
    const bool batch = ctx->g.size() > 1;
    if (ctx->strip.on) return fail(ctx, MPR_ESTATE, "a row strip takes its temperature from mpr_strip_temperature");
    for (const GridInfo& G : ctx->g)
        if (G.n_sp == 0) return fail(ctx, MPR_ENOPAIRS, "no nearest-neighbour sample pairs");
    std::vector<std::pair<int, int>> shapes;
    std::vector<double> es;
    for (const GridInfo& G : ctx->g) {
        shapes.push_back(table_shape(p, G.W, G.H, batch));
        es.push_back(G.e_s);
    }
    std::vector<double> T;
    mpr_status s = temperatures_for(ctx, shapes, es, T);
    if (s != MPR_OK) return s;
    s = set_T_all(ctx, T);
    if (s != MPR_OK) return s;
    if (T_hat) *T_hat = T[0];
    if (e_s) *e_s = ctx->g[0].e_s;
    return MPR_OK;
}

mpr_status mpr_sweep(mpr_ctx* ctx, int n, double a, mpr_sweep_stats* out) {
    if (!ctx) return MPR_EINVAL;
    if (n < 0 || !(a >= 1.0)) return fail(ctx, MPR_EINVAL, "n >= 0 and a >= 1 required");
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    mpr_status s = reset_tracked_energy(ctx, ctx->b);
    if (s == MPR_OK) s = run_sweeps(ctx, ctx->b, n, CTL_FIXED, a, false);
    std::vector<Ctl> c;
    if (s == MPR_OK) s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    if (out) {
        out->sweeps = n;
        out->acceptance = c[0].A_last;
        out->e = c[0].e_last;
    }
    return MPR_OK;
}

mpr_status mpr_equilibrate(mpr_ctx* ctx, mpr_equil_stats* out) {
    if (!ctx) return MPR_EINVAL;
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    mpr_status s = reset_relax(ctx, ctx->b);
    if (s == MPR_OK) s = run_sweeps(ctx, ctx->b, 0, CTL_RELAX, 1.0, false);
    std::vector<Ctl> c;
    if (s == MPR_OK) s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    if (out) {
        out->sweeps = c[0].i;
        out->a = c[0].a;
        out->k = c[0].k;
        out->A_last = c[0].A_last;
        out->e_last = c[0].e_last;
        out->converged = c[0].converged;
    }
    for (size_t i = 0; i < c.size(); ++i)
        if (!c[i].converged && ctx->b.ents[i].P > 0) return MPR_ENOTEQUIL;
    return MPR_OK;
}

// M equilibrium sweeps of every grid, then each grid's zhat into out[g] (host or device).
static mpr_status predict_all(mpr_ctx* ctx, int M, float* const* out) {
    Batch& b = ctx->b;
    if (b.tiled)
        CU(cudaMemsetAsync(b.d_tacc, 0, sizeof(float) * (size_t)b.ntiles * tile_geom(b.tcfg).acc, ctx->st));
    else
        CU(cudaMemsetAsync(b.d_acc, 0, sizeof(float) * (b.f64 ? 2 : 1) * std::max<size_t>(b.n_gaps, 1), ctx->st));
    mpr_status s = run_sweeps(ctx, b, M, CTL_FIXED, ctx->prm.a_eq, true);
    if (s != MPR_OK) return s;
    CU(cudaMemcpyAsync(ctx->d_out, ctx->d_z, (size_t)ctx->n_sites * sizeof(float),
                       cudaMemcpyDeviceToDevice, ctx->st));
    if (b.tiled) {
        // one launch over the tiles of every grid, each grid's (z_min, z_max) from zr
        std::vector<double2> zr(ctx->g.size());
        for (size_t i = 0; i < ctx->g.size(); ++i) zr[i] = make_double2(ctx->g[i].zmin, ctx->g[i].zmax);
        double2* d_zr = nullptr;
        CU(dalloc(&d_zr, zr.size(), ctx->st));
        CU(cudaMemcpyAsync(d_zr, zr.data(), sizeof(double2) * zr.size(), cudaMemcpyHostToDevice, ctx->st));
        CU(launch_tile_predict_out(b.tcfg, b.d_tiles, b.d_cnts, b.d_lists, b.d_tacc, b.d_ents, 0, b.ntiles, M,
                                   ctx->prm.q, 0.0, 0.0, d_zr, 1, 0, ctx->d_out, ctx->st));
        dfree(d_zr, ctx->st);
    } else {
        for (size_t i = 0; i < ctx->g.size(); ++i) {
            const GridInfo& G = ctx->g[i];
            CU(launch_predict_out(&b.ents[i], b.d_lat, b.d_gaps, b.d_acc, M, ctx->prm.q, G.zmin,
                                  G.zmax, ctx->d_out + G.site0, b.f64, ctx->st));
        }
    }
    CU(fan_begin(ctx, (int)ctx->g.size()));
    for (size_t i = 0; i < ctx->g.size(); ++i) {
        const GridInfo& G = ctx->g[i];
        CU(cudaMemcpyAsync(out[i], ctx->d_out + G.site0, (size_t)G.W * G.H * sizeof(float),
                           cudaMemcpyDefault, fan_stream(ctx, (int)i)));
    }
    CU(fan_end(ctx));
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

mpr_status mpr_predict(mpr_ctx* ctx, int M, float* zhat) {
    if (!ctx || !zhat) return MPR_EINVAL;
    if (ctx->g.size() != 1) return fail(ctx, MPR_EINVAL, "mpr_predict serves one grid; use mpr_predict_batch");
    if (M < 1) return fail(ctx, MPR_EINVAL, "M >= 1 required");
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    return predict_all(ctx, M, &zhat);
}

// Independent-chain realizations (not in the paper, whose estimator is one chain): the
// grid's current state (normally equilibrated by mpr_equilibrate) is forked into K chains,
// chain k with Philox chain word chain + k * 2^24 (k = 0 continues the grid's own chain),
// all starting at the same sweep counter; the K chains run burn_in sweeps that are not
// averaged (to decorrelate from the shared start), then M_per_chain equilibrium sweeps, as
// one batch (one launch per sweep for all chains); zhat is the mean of the back-transformed
// angles of all K * M_per_chain realizations.  K = 1, burn_in = 0 is mpr_predict.  The
// grid's own state is left as it was.
mpr_status mpr_predict_chains(mpr_ctx* ctx, int K, int burn_in, int M_per_chain, float* zhat) {
    if (!ctx || !zhat) return MPR_EINVAL;
    if (ctx->g.size() != 1) return fail(ctx, MPR_EINVAL, "mpr_predict_chains serves one grid");
    if (K < 1 || K > kMaxChains) return fail(ctx, MPR_EINVAL, "1 <= K <= 128 chains");
    if (M_per_chain < 1 || burn_in < 0) return fail(ctx, MPR_EINVAL, "M_per_chain >= 1, burn_in >= 0 required");
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    Batch& b = ctx->b;
    if (!b.tiled) return fail(ctx, MPR_EINVAL, "independent chains run on the tile path");
    std::vector<Ctl> c0;
    mpr_status s = read_ctl(ctx, b, c0);
    if (s != MPR_OK) return s;
    const GridInfo& G = ctx->g[0];
    std::vector<GridIn> gi((size_t)K);
    for (int k = 0; k < K; ++k)
        gi[k] = GridIn{G.W, G.H, ctx->d_z + G.site0, ctx->d_mask + G.site0,
                       b.ents[0].chain + (uint32_t)k * kChainStride, G.T, G.zmin, G.scale};
    Batch ab;
    s = batch_build(ctx, ab, gi, 0, ctx->d_mask + G.site0, true);
    if (s == MPR_OK) s = build_tiles(ctx, ab, b.tcfg);
    if (s == MPR_OK) {
        // fork: every chain starts from the grid's current state and control state
        const size_t state = (size_t)2 * b.ents[0].prows * b.ents[0].pitch;
        const float2* src = lat_cur(b, c0[0]) + b.ents[0].plane[0];
        std::vector<Ctl> ck((size_t)K, c0[0]);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < K && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(ab.d_lat + ab.ents[k].plane[0], src, state * sizeof(float2),
                                cudaMemcpyDeviceToDevice, ctx->st);
            ck[k].cur = 0;
            ck[k].cur_base = 0;
            ck[k].sweep_base = ck[k].sweep;
        }
        for (auto& cc : ck) ctl_set_go(cc);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ab.d_ctl, ck.data(), sizeof(Ctl) * K, cudaMemcpyHostToDevice, ctx->st);
        if (e == cudaSuccess && sync_tiles(ctx, ab) != MPR_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess)
            e = cudaMemsetAsync(ab.d_tacc, 0, sizeof(float) * (size_t)ab.ntiles * tile_geom(ab.tcfg).acc,
                                ctx->st);
        if (e != cudaSuccess) s = fail(ctx, MPR_ECUDA, std::string("chain fork: ") + cudaGetErrorString(e));
    }
    if (s == MPR_OK && burn_in > 0) s = run_sweeps(ctx, ab, burn_in, CTL_FIXED, ctx->prm.a_eq, false);
    if (s == MPR_OK) s = run_sweeps(ctx, ab, M_per_chain, CTL_FIXED, ctx->prm.a_eq, true);
    if (s == MPR_OK) {
        cudaError_t e = cudaMemcpyAsync(ctx->d_out + G.site0, ctx->d_z + G.site0,
                                        (size_t)G.W * G.H * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st);
        const int nt = ab.ents[0].ntiles;
        if (e == cudaSuccess)
            e = launch_tile_predict_out(ab.tcfg, ab.d_tiles, ab.d_cnts, ab.d_lists, ab.d_tacc, ab.d_ents, 0,
                                        nt, M_per_chain, ctx->prm.q, G.zmin, G.zmax, nullptr, K, nt,
                                        ctx->d_out + G.site0, ctx->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(zhat, ctx->d_out + G.site0, (size_t)G.W * G.H * sizeof(float),
                                cudaMemcpyDefault, ctx->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
        if (e != cudaSuccess) s = fail(ctx, MPR_ECUDA, std::string("chain average: ") + cudaGetErrorString(e));
    }
    cudaStreamSynchronize(ctx->st);
    batch_free(ab, ctx->st);
    return s;
}

mpr_status mpr_predict_batch(mpr_ctx* ctx, int M, float* const* zhat) {
    if (!ctx || !zhat) return MPR_EINVAL;
    for (size_t i = 0; i < ctx->g.size(); ++i)
        if (!zhat[i]) return MPR_EINVAL;
    if (M < 1) return fail(ctx, MPR_EINVAL, "M >= 1 required");
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    return predict_all(ctx, M, zhat);
}

mpr_status mpr_fill(mpr_ctx* ctx, float* zhat, mpr_equil_stats* stats) {
    if (!ctx || !zhat) return MPR_EINVAL;
    if (ctx->g.size() != 1) return fail(ctx, MPR_EINVAL, "mpr_fill serves one grid; use mpr_fill_batch");
    mpr_status s = MPR_OK;
    if (!ctx->T_set) s = mpr_estimate_T(ctx, nullptr, nullptr);
    if (s != MPR_OK) return s;
    mpr_status eq = mpr_equilibrate(ctx, stats);
    if (eq != MPR_OK && eq != MPR_ENOTEQUIL) return eq;
    s = predict_all(ctx, ctx->prm.M, &zhat);
    return s != MPR_OK ? s : eq;
}

mpr_status mpr_fill_batch(mpr_ctx* ctx, float* const* zhat) {
    if (!ctx || !zhat) return MPR_EINVAL;
    mpr_status s = MPR_OK;
    if (!ctx->T_set) s = mpr_estimate_T(ctx, nullptr, nullptr);
    if (s != MPR_OK) return s;
    mpr_status eq = mpr_equilibrate(ctx, nullptr);
    if (eq != MPR_OK && eq != MPR_ENOTEQUIL) return eq;
    s = mpr_predict_batch(ctx, ctx->prm.M, zhat);
    return s != MPR_OK ? s : eq;
}

// Warm start: the network's initial gap state for every grid, run on runs of consecutive
// grids of one shape (contiguous in the concatenated buffers) as one batch.
mpr_status mpr_warmstart_init(mpr_ctx* ctx, mpr_net* net) {
    if (!ctx || !net) return MPR_EINVAL;
    Batch& b = ctx->b;
    if (b.f64) return fail(ctx, MPR_EINVAL, "the warm start writes an FP32 lattice");
    if (ctx->prm.q != 0.5) return fail(ctx, MPR_EINVAL, "the warm start writes theta = phi / 2 (q = 1/2)");
    float2* lat1 = b.tiled ? b.d_lat2 : nullptr;
    const int n = (int)ctx->g.size();
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && j - i < 4096 && ctx->g[j].W == ctx->g[i].W && ctx->g[j].H == ctx->g[i].H) ++j;
        std::vector<double> zmin, zmax;
        for (int k = i; k < j; ++k) {
            zmin.push_back(ctx->g[k].zmin);
            zmax.push_back(ctx->g[k].zmax);
        }
        const GridInfo& G = ctx->g[i];
        const mpr_status s = mprnet_warmstart(net, ctx->d_z + G.site0, ctx->d_mask + G.site0, j - i, G.H, G.W,
                                              zmin.data(), zmax.data(), b.d_ents + i, b.d_lat, lat1, ctx->st);
        if (s != MPR_OK) return fail(ctx, s, std::string("warm start: ") + mprnet_error(net));
        i = j;
    }
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

mpr_status mpr_batch_info(mpr_ctx* ctx, int g, double* T, double* e_s, int* sweeps, int* converged,
                          double* zmin, double* zmax) {
    if (!ctx || g < 0 || g >= (int)ctx->g.size()) return MPR_EINVAL;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    const GridInfo& G = ctx->g[g];
    if (T) *T = G.T;
    if (e_s) *e_s = G.e_s;
    if (sweeps) *sweeps = c[g].i;
    if (converged) *converged = c[g].converged;
    if (zmin) *zmin = G.zmin;
    if (zmax) *zmax = G.zmax;
    return MPR_OK;
}

mpr_status mpr_batch_info_all(mpr_ctx* ctx, int n, double* T, double* e_s, int* sweeps, int* converged,
                              double* zmin, double* zmax) {
    if (!ctx || n != (int)ctx->g.size()) return MPR_EINVAL;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    for (int g = 0; g < n; ++g) {
        const GridInfo& G = ctx->g[g];
        if (T) T[g] = G.T;
        if (e_s) e_s[g] = G.e_s;
        if (sweeps) sweeps[g] = c[g].i;
        if (converged) converged[g] = c[g].converged;
        if (zmin) zmin[g] = G.zmin;
        if (zmax) zmax[g] = G.zmax;
    }
    return MPR_OK;
}

mpr_status mpr_get_state(mpr_ctx* ctx, float* phi, uint32_t* sweep) {
    if (!ctx || !phi) return MPR_EINVAL;
    const size_t n = (size_t)ctx->g[0].W * ctx->g[0].H;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    CU(launch_get_state(&ctx->b.ents[0], lat_cur(ctx->b, c[0]), ctx->d_out, ctx->b.f64, ctx->st));
    CU(cudaMemcpyAsync(phi, ctx->d_out, n * sizeof(float), cudaMemcpyDefault, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    if (sweep) *sweep = c[0].sweep;
    return MPR_OK;
}

mpr_status mpr_get_state64(mpr_ctx* ctx, double* phi, uint32_t* sweep) {
    if (!ctx || !phi) return MPR_EINVAL;
    const size_t n = (size_t)ctx->g[0].W * ctx->g[0].H;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    double* d = nullptr;
    CU(dalloc(&d, n, ctx->st));
    cudaError_t e = launch_get_state64(&ctx->b.ents[0], lat_cur(ctx->b, c[0]), d, ctx->b.f64, ctx->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi, d, n * sizeof(double), cudaMemcpyDefault, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    dfree(d, ctx->st);
    CU(e);
    if (sweep) *sweep = c[0].sweep;
    return MPR_OK;
}

mpr_status mpr_get_state_batch(mpr_ctx* ctx, int g, float* phi) {
    if (!ctx || !phi || g < 0 || g >= (int)ctx->g.size()) return MPR_EINVAL;
    const GridInfo& G = ctx->g[g];
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    CU(launch_get_state(&ctx->b.ents[g], lat_cur(ctx->b, c[g]), ctx->d_out + G.site0, ctx->b.f64, ctx->st));
    CU(cudaMemcpyAsync(phi, ctx->d_out + G.site0, (size_t)G.W * G.H * sizeof(float), cudaMemcpyDefault, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

mpr_status mpr_set_state(mpr_ctx* ctx, const float* phi, uint32_t sweep) {
    if (!ctx || !phi) return MPR_EINVAL;
    const size_t n = (size_t)ctx->g[0].W * ctx->g[0].H;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    CU(cudaMemcpyAsync(ctx->d_out, phi, n * sizeof(float), cudaMemcpyDefault, ctx->st));
    CU(launch_set_state(&ctx->b.ents[0], lat_cur(ctx->b, c[0]), ctx->b.d_gaps, ctx->d_out, ctx->b.f64, ctx->st));
    c[0].sweep = sweep;
    c[0].sweep_base = sweep;
    c[0].cur_base = c[0].cur;
    for (auto& cc : c) ctl_set_go(cc);
    CU(cudaMemcpyAsync(ctx->b.d_ctl, c.data(), sizeof(Ctl), cudaMemcpyHostToDevice, ctx->st));
    s = sync_tiles(ctx, ctx->b);
    if (s != MPR_OK) return s;
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

mpr_status mpr_get_info(mpr_ctx* ctx, double* H_exact, double* H_tracked, double* zmin,
                        double* zmax, double* T, double* e_s) {
    if (!ctx) return MPR_EINVAL;
    std::vector<Ctl> c;
    mpr_status s = read_ctl(ctx, ctx->b, c);
    if (s != MPR_OK) return s;
    if (H_exact) {
        double* d = ctx->b.d_scratch + kScratch;
        CU(launch_energy(&ctx->b.ents[0], lat_cur(ctx->b, c[0]), ctx->b.d_scratch, kScratch, d, ctx->b.f64, ctx->st));
        CU(cudaMemcpyAsync(H_exact, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    if (H_tracked) *H_tracked = c[0].H;
    if (zmin) *zmin = ctx->g[0].zmin;
    if (zmax) *zmax = ctx->g[0].zmax;
    if (T) *T = ctx->g[0].T;
    if (e_s) *e_s = ctx->g[0].e_s;
    return MPR_OK;
}

// Autotuner: times a few sweeps of every compiled tile configuration on the context's own
// grids (from a snapshot of the state, restored afterwards, so the chain is unchanged),
// keeps the fastest, and sizes the captured chunk of sweeps from its time.
mpr_status mpr_autotune(mpr_ctx* ctx, int* tile_cfg, int* graph_sweeps, double* ms_per_sweep) {
    if (!ctx) return MPR_EINVAL;
    Batch& b = ctx->b;
    if (!b.tiled) return fail(ctx, MPR_ESTATE, "autotuning applies to the tile kernels");
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    // snapshot: both lattice buffers and the control state
    const size_t bytes = b.lat_elems * sizeof(float2);
    float2* snap0 = nullptr;
    float2* snap1 = nullptr;
    CU(dalloc(&snap0, b.lat_elems, ctx->st));
    CU(dalloc(&snap1, b.lat_elems, ctx->st));
    CU(cudaMemcpyAsync(snap0, b.d_lat, bytes, cudaMemcpyDeviceToDevice, ctx->st));
    CU(cudaMemcpyAsync(snap1, b.d_lat2, bytes, cudaMemcpyDeviceToDevice, ctx->st));
    std::vector<Ctl> c0;
    mpr_status s = read_ctl(ctx, b, c0);
    if (s != MPR_OK) return s;
    const int n_try = 6;
    int best = b.tcfg;
    double best_ms = 1e30;
    for (int cfg = 0; cfg < tile_config_count() && s == MPR_OK; ++cfg) {
        s = build_tiles(ctx, b, cfg);
        if (s != MPR_OK) break;
        double ms = 0.0;
        s = mpr_time_sweeps(ctx, 2, 4.0, &ms);                 // warm-up
        if (s == MPR_OK) s = mpr_time_sweeps(ctx, n_try, 4.0, &ms);
        if (s == MPR_OK && ms < best_ms) { best_ms = ms; best = cfg; }
        CU(cudaMemcpyAsync(b.d_lat, snap0, bytes, cudaMemcpyDeviceToDevice, ctx->st));
        CU(cudaMemcpyAsync(b.d_lat2, snap1, bytes, cudaMemcpyDeviceToDevice, ctx->st));
        for (auto& cc : c0) ctl_set_go(cc);
        CU(cudaMemcpyAsync(b.d_ctl, c0.data(), sizeof(Ctl) * c0.size(), cudaMemcpyHostToDevice, ctx->st));
        s = sync_tiles(ctx, b);
        if (s != MPR_OK) return s;
        CU(cudaStreamSynchronize(ctx->st));
    }
    dfree(snap0, ctx->st);
    dfree(snap1, ctx->st);
    if (s != MPR_OK) return s;
    if (best != b.tcfg) {
        s = build_tiles(ctx, b, best);
        if (s != MPR_OK) return s;
    }
    // sweeps per captured chunk of the list path's graphs (the tile path runs each phase as
    // one launch): at least ~60 us of sweeping per chunk, so that the chunk's condition
    // launch (a few us) costs under ~5 %
    int S = (int)std::lround(0.06 / std::max(best_ms, 1e-6));
    S = std::min(kMaxGraphSweeps, std::max(4, S));
    if (S != b.gsweeps) {
        for (auto& kv : b.graphs) cudaGraphExecDestroy(kv.second);
        b.graphs.clear();
        b.gsweeps = S;
    }
    if (tile_cfg) *tile_cfg = b.tcfg;
    if (graph_sweeps) *graph_sweeps = b.gsweeps;
    if (ms_per_sweep) *ms_per_sweep = best_ms;
    return MPR_OK;
}

uint64_t mpr_kernel_launches(void) { return (uint64_t)g_launches.load(); }

mpr_status mpr_time_sweeps(mpr_ctx* ctx, int n, double a, double* ms_per_sweep) {
    if (!ctx || n < 1 || !(a >= 1.0) || !ms_per_sweep) return MPR_EINVAL;
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    CU(cudaEventRecord(e0, ctx->st));
    mpr_status s = enqueue_sweeps(ctx, ctx->b, ctx->st, n, CTL_FIXED, a, false, false);
    if (s != MPR_OK) return s;
    CU(cudaEventRecord(e1, ctx->st));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_sweep = (double)ms / (double)n;
    return MPR_OK;
}

void mpr_debug_trace(uint64_t* buf, uint64_t words) {
    g_trace_words = buf ? (unsigned long long)words : 0ull;
    g_trace = buf ? reinterpret_cast<unsigned long long*>(buf) : nullptr;
}

void mpr_debug_wait_limit(uint64_t ns, int stall) {
    g_wait_ns = ns ? (unsigned long long)ns : 4000000000ull;
    g_stall = stall ? 1 : 0;
}

void mpr_sweep_timing_start(void) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    g_timing.on = true;
    g_timing.ms = 0.0;
    g_timing.launches = 0;
    g_timing.site_sweeps = 0.0;
    g_timing.gap_updates = 0.0;
}

void mpr_sweep_timing_read(int stop, double* ms, uint64_t* launches, double* site_sweeps,
                           double* gap_updates) {
    std::lock_guard<std::mutex> lk(g_timing.mu);
    if (ms) *ms = g_timing.ms;
    if (launches) *launches = g_timing.launches;
    if (site_sweeps) *site_sweeps = g_timing.site_sweeps;
    if (gap_updates) *gap_updates = g_timing.gap_updates;
    if (stop) g_timing.on = false;
}

mpr_status mpr_release_memory(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPR_ECUDA;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) return MPR_OK;
    return cudaMemPoolTrimTo(g_pools[dev], 0) == cudaSuccess ? MPR_OK : MPR_ECUDA;
}

mpr_status mpr_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, size_t n,
                      void* cuda_stream) {
    if ((!ctr || !out) && n) return MPR_EINVAL;
    if (n == 0) return MPR_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint4* d_in = nullptr;
    uint4* d_out = nullptr;
    if (dalloc(&d_in, n, st) != cudaSuccess) return MPR_ENOMEM;
    if (dalloc(&d_out, n, st) != cudaSuccess) { dfree(d_in, st); return MPR_ENOMEM; }
    mpr_status s = MPR_OK;
    if (cudaMemcpyAsync(d_in, ctr, n * sizeof(uint4), cudaMemcpyDefault, st) != cudaSuccess ||
        launch_philox(d_in, (uint32_t)seed, (uint32_t)(seed >> 32), d_out, n, st) != cudaSuccess ||
        cudaMemcpyAsync(out, d_out, n * sizeof(uint4), cudaMemcpyDefault, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        s = MPR_ECUDA;
    dfree(d_in, st);
    dfree(d_out, st);
    return s;
}

// ---------------------------------------------------------------- row strips of one grid
// A grid too large for one GPU is cut into bands of rows, one per process (the checkerboard
// of Sect. 3.3 cut by rows).  A strip's context holds the block of rows [row0, row0 + Hb)
// of the W x H_global grid: its own rows and, where another strip continues the grid, the
// one row of that strip above (h0 = 1) and below (h1 = 1), frozen in the block and
// refreshed from its owner after every half-sweep.  row0 is even, so the block's colours
// are the grid's, and the Philox site index of block site (y, x) is (row0 + y) W + x: the
// strips together draw exactly the random numbers of the whole grid.

static bool strip_geometry(int W, int Hb, int row0, int H_global, int* h0, int* h1) {
    if (W < 1 || Hb < 1 || row0 < 0 || (row0 & 1) || H_global < 1 || H_global > 65535 ||
        row0 + Hb > H_global || (W + 1) / 2 > 65535 || (long long)W * H_global >= (1LL << 31))
        return false;
    *h0 = row0 > 0 ? 1 : 0;
    *h1 = row0 + Hb < H_global ? 1 : 0;
    return Hb >= *h0 + *h1 + 1;
}

static double unkey_value(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    float f;
    std::memcpy(&f, &b, sizeof f);
    return (double)f;
}

mpr_status mpr_strip_extremes(const float* z, const uint8_t* mask, int W, int Hb, int row0, int H_global,
                              double* out, void* cuda_stream) {
    int h0 = 0, h1 = 0;
    if (!z || !mask || !out || !strip_geometry(W, Hb, row0, H_global, &h0, &h1)) return MPR_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned* d_keys = nullptr;
    unsigned long long* d_ns = nullptr;
    if (dalloc(&d_keys, 2, st) != cudaSuccess) return MPR_ENOMEM;
    if (dalloc(&d_ns, 1, st) != cudaSuccess) { dfree(d_keys, st); return MPR_ENOMEM; }
    unsigned keys[2] = {0u, 0u};
    unsigned long long ns = 0;
    const long long off = (long long)h0 * W;
    cudaError_t e = cudaMemsetAsync(d_keys, 0xFF, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_keys + 1, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ns, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_minmax(z + off, mask + off, (long long)(Hb - h0 - h1) * W, d_keys, d_ns, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(keys, d_keys, sizeof keys, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d_ns, sizeof ns, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_keys, st);
    dfree(d_ns, st);
    if (e != cudaSuccess) { cudaGetLastError(); return MPR_ECUDA; }
    out[0] = ns ? unkey_value(keys[0]) : INFINITY;
    out[1] = ns ? unkey_value(keys[1]) : -INFINITY;
    out[2] = (double)ns;
    return MPR_OK;
}

mpr_status mpr_strip_init(mpr_ctx** out, const float* z, const uint8_t* mask, int W, int Hb, int row0,
                          int H_global, double zmin, double zmax, const mpr_params* params, void* cuda_stream) {
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    int h0 = 0, h1 = 0;
    if (!z || !mask || !strip_geometry(W, Hb, row0, H_global, &h0, &h1)) return MPR_EINVAL;
    if (!(zmax > zmin) || !std::isfinite(zmin) || !std::isfinite(zmax)) return MPR_ENODATA;
    mpr_ctx* ctx = new mpr_ctx();
    if (params) ctx->prm = *params; else mpr_default_params(&ctx->prm);
    std::string why;
    if (ctx->prm.exec_mode == MPR_EXEC_TILE || check_params(&ctx->prm, why) != MPR_OK) {
        delete ctx;
        return MPR_EINVAL;
    }
    ctx->prm.exec_mode = MPR_EXEC_LIST;              // the half-sweep kernels carry the row offset
    ctx->st = (cudaStream_t)cuda_stream;
    ctx->g.resize(1);
    GridInfo& G = ctx->g[0];
    G.W = W;
    G.H = Hb;
    G.site0 = 0;
    G.zmin = zmin;
    G.zmax = zmax;
    G.scale = kTwoPi / (zmax - zmin);
    ctx->n_sites = (long long)W * Hb;
    auto bail = [&](mpr_status s) { mpr_free(ctx); return s; };
#define CUS(call) do { if ((call) != cudaSuccess) { cudaGetLastError(); return bail(MPR_ECUDA); } } while (0)
    CUS(pinned_slot(&ctx->h_active));
    const size_t N = (size_t)ctx->n_sites;
    if (dalloc(&ctx->d_z, N, ctx->st) != cudaSuccess || dalloc(&ctx->d_mask, N, ctx->st) != cudaSuccess ||
        dalloc(&ctx->d_out, N, ctx->st) != cudaSuccess || dalloc(&ctx->d_stop, 1, ctx->st) != cudaSuccess) {
        cudaGetLastError();
        return bail(MPR_ENOMEM);
    }
    CUS(cudaMemcpyAsync(ctx->d_z, z, N * sizeof(float), cudaMemcpyDefault, ctx->st));
    CUS(cudaMemcpyAsync(ctx->d_mask, mask, N, cudaMemcpyDefault, ctx->st));
    // Eq. 4 terms of the strip's own sample pairs (a pair belongs to the strip of its upper
    // or left site), before the neighbouring strips' rows are frozen in the mask copy
    {
        EntryDesc t{};
        t.W = W;
        t.H = Hb - h0;
        double* d_ps = nullptr;
        unsigned long long* d_pc = nullptr;
        CUS(dalloc(&d_ps, 1024, ctx->st));
        CUS(dalloc(&d_pc, 1024, ctx->st));
        int np = 0;
        const long long off = (long long)h0 * W;
        CUS(launch_sample_energy(&t, ctx->d_z + off, ctx->d_mask + off, G.scale, ctx->prm.q, d_ps, d_pc, &np,
                                 ctx->prm.precision == MPR_PREC_F64, ctx->st, Hb - h0 - h1));
        std::vector<double> ps(np);
        std::vector<unsigned long long> pc(np);
        CUS(cudaMemcpyAsync(ps.data(), d_ps, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->st));
        CUS(cudaMemcpyAsync(pc.data(), d_pc, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost, ctx->st));
        CUS(cudaStreamSynchronize(ctx->st));
        dfree(d_ps, ctx->st);
        dfree(d_pc, ctx->st);
        for (int k = 0; k < np; ++k) {
            ctx->strip.pair_sum += ps[k];
            ctx->strip.pair_cnt += (double)pc[k];
        }
    }
    // the neighbouring strips' rows: never updated here (their values come from their owners)
    if (h0) CUS(cudaMemsetAsync(ctx->d_mask, 1, (size_t)W, ctx->st));
    if (h1) CUS(cudaMemsetAsync(ctx->d_mask + (size_t)(Hb - 1) * W, 1, (size_t)W, ctx->st));
#undef CUS
    GridIn gi{W, Hb, ctx->d_z, ctx->d_mask, ctx->prm.chain, 0.0, zmin, G.scale};
    gi.row_off = (uint32_t)row0;
    const mpr_status bs = batch_build(ctx, ctx->b, std::vector<GridIn>{gi}, 0, ctx->d_mask);
    if (bs != MPR_OK) return bail(bs);
    ctx->strip.on = true;
    ctx->strip.row0 = row0;
    ctx->strip.H_global = H_global;
    ctx->strip.h0 = h0;
    ctx->strip.h1 = h1;
    *out = ctx;
    return MPR_OK;
}

static mpr_status strip_ctx(mpr_ctx* ctx) {
    if (!ctx) return MPR_EINVAL;
    if (!ctx->strip.on) return fail(ctx, MPR_ESTATE, "not a row-strip context (mpr_strip_init)");
    return MPR_OK;
}

mpr_status mpr_strip_pairs(mpr_ctx* ctx, double* sum_cos, double* n_pairs) {
    const mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (sum_cos) *sum_cos = ctx->strip.pair_sum;
    if (n_pairs) *n_pairs = ctx->strip.pair_cnt;
    return MPR_OK;
}

mpr_status mpr_strip_temperature(mpr_ctx* ctx, double e_s, double* T_hat) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (!std::isfinite(e_s)) return fail(ctx, MPR_EINVAL, "e_s must be finite");
    std::vector<double> T;
    s = temperatures_for(ctx, {table_shape(ctx->prm, ctx->g[0].W, ctx->strip.H_global, false)}, {e_s}, T);
    if (s == MPR_OK) s = set_T_all(ctx, T);
    if (s != MPR_OK) return s;
    ctx->g[0].e_s = e_s;
    if (T_hat) *T_hat = T[0];
    return MPR_OK;
}

mpr_status mpr_strip_energy(mpr_ctx* ctx, double* H_part) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (!H_part) return MPR_EINVAL;
    double* d = ctx->b.d_scratch + kScratch;
    CU(launch_energy(&ctx->b.ents[0], ctx->b.d_lat, ctx->b.d_scratch, kScratch, d, ctx->b.f64, ctx->st,
                     ctx->strip.h0, ctx->g[0].H - ctx->strip.h1));
    CU(cudaMemcpyAsync(H_part, d, sizeof(double), cudaMemcpyDefault, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

long long mpr_strip_gaps(const mpr_ctx* ctx) {
    return ctx && ctx->strip.on ? (long long)ctx->b.ents[0].P : -1;
}

mpr_status mpr_strip_begin(mpr_ctx* ctx, int phase, double H_total, double P_total) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (!ctx->T_set) return fail(ctx, MPR_ESTATE, "temperature not set");
    if (phase != 0 && phase != 1) return fail(ctx, MPR_EINVAL, "phase 0 (relaxation) or 1 (equilibrium)");
    if (!(P_total >= 0.0) || P_total >= 2147483648.0) return fail(ctx, MPR_EINVAL, "0 <= P_total < 2^31");
    Batch& b = ctx->b;
    ctx->strip.P_total = P_total;
    std::vector<Ctl> c;
    s = read_ctl(ctx, b, c);
    if (s != MPR_OK) return s;
    if (phase == 0) {                        // Algorithm 2 steps 2.1, 2.3, 2.4, and the energy of the grid
        c[0].i = 0;
        c[0].k = -1.0;
        c[0].a = 1.0;
        c[0].stop = P_total > 0.0 ? 0 : 1;
        c[0].converged = 0;
        c[0].esum = 0.0;
        c[0].nsamp = 0;
        c[0].half_qd = (float)(0.5 * kTwoPi * b.ents[0].q / 1.0);
        c[0].H = H_total;
        for (auto& cc : c) ctl_set_go(cc);
        CU(cudaMemcpyAsync(b.d_ctl, c.data(), sizeof(Ctl), cudaMemcpyHostToDevice, ctx->st));
    } else {                                 // step 6: the angle sums start at zero
        CU(cudaMemsetAsync(b.d_acc, 0, sizeof(float) * (b.f64 ? 2 : 1) * std::max<size_t>(b.n_gaps, 1), ctx->st));
    }
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

mpr_status mpr_strip_half_sweep(mpr_ctx* ctx, int color, int phase, double* totals) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if ((color != 0 && color != 1) || (phase != 0 && phase != 1) || !totals)
        return fail(ctx, MPR_EINVAL, "color 0 or 1, phase 0 or 1, totals required");
    Batch& b = ctx->b;
    const bool relax = phase == 0;
    const SweepArgs A = sweep_args(ctx, b, relax, ctx->prm.a_eq, relax, !relax);
    CU(launch_half_sweep(A, color, ctx->prm.trig_mode, ctx->st));
    CU(launch_strip_partials(b.d_part[color], b.nblk[color], color, totals, b.f64, ctx->st));
    return MPR_OK;
}

mpr_status mpr_strip_control(mpr_ctx* ctx, const double* totals, int phase, int* stop) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if ((phase != 0 && phase != 1) || !totals) return fail(ctx, MPR_EINVAL, "phase 0 or 1, totals required");
    Batch& b = ctx->b;
    const mpr_params& p = ctx->prm;
    const double W = ctx->g[0].W, Hg = ctx->strip.H_global;
    const double ngp = W * (Hg - 1.0) + Hg * (W - 1.0);
    CU(launch_strip_control(b.d_ctl, &b.ents[0], ctx->strip.P_total, ngp, totals, phase == 0 ? CTL_RELAX : CTL_FIXED,
                            p.A_targ, p.k_a, p.n_f, p.n_fit, p.i_max, b.d_ehist, ctx->d_stop, ctx->st));
    if (stop) {
        CU(cudaMemcpyAsync(ctx->h_active, ctx->d_stop, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
        *stop = phase == 0 ? ctx->h_active[0] : 0;
    }
    return MPR_OK;
}

size_t mpr_strip_row_bytes(const mpr_ctx* ctx) {
    if (!ctx || !ctx->strip.on) return 0;
    return (size_t)2 * ctx->b.ents[0].pitch * (ctx->b.f64 ? sizeof(double2) : sizeof(float2));
}

mpr_status mpr_strip_row(mpr_ctx* ctx, int which, void* buf) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (!buf || which < 0 || which > 3) return fail(ctx, MPR_EINVAL, "which in 0..3 and a buffer required");
    const int Hb = ctx->g[0].H, h0 = ctx->strip.h0, h1 = ctx->strip.h1;
    if ((which == 2 && !h0) || (which == 3 && !h1)) return fail(ctx, MPR_EINVAL, "no neighbouring strip there");
    const int y = which == 0 ? h0 : which == 1 ? Hb - 1 - h1 : which == 2 ? 0 : Hb - 1;
    const EntryDesc& E = ctx->b.ents[0];
    const size_t el = ctx->b.f64 ? sizeof(double2) : sizeof(float2);
    const size_t wide = ctx->b.f64 ? 2 : 1;
    const size_t row = (size_t)E.pitch * el;
    for (int c = 0; c < 2; ++c) {
        char* lat = reinterpret_cast<char*>(ctx->b.d_lat + (size_t)(E.plane[c] + (long long)(y + 1) * E.pitch) * wide);
        char* other = static_cast<char*>(buf) + (size_t)c * row;
        if (which <= 1) CU(cudaMemcpyAsync(other, lat, row, cudaMemcpyDefault, ctx->st));
        else CU(cudaMemcpyAsync(lat, other, row, cudaMemcpyDefault, ctx->st));
    }
    return MPR_OK;
}

mpr_status mpr_strip_predict(mpr_ctx* ctx, int M, float* zhat) {
    mpr_status s = strip_ctx(ctx);
    if (s != MPR_OK) return s;
    if (!zhat || M < 1) return fail(ctx, MPR_EINVAL, "M >= 1 and zhat required");
    Batch& b = ctx->b;
    const GridInfo& G = ctx->g[0];
    CU(cudaMemcpyAsync(ctx->d_out, ctx->d_z, (size_t)ctx->n_sites * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    CU(launch_predict_out(&b.ents[0], b.d_lat, b.d_gaps, b.d_acc, M, ctx->prm.q, G.zmin, G.zmax, ctx->d_out, b.f64,
                          ctx->st));
    CU(cudaMemcpyAsync(zhat, ctx->d_out, (size_t)ctx->n_sites * sizeof(float), cudaMemcpyDefault, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return MPR_OK;
}

}  // extern "C"
