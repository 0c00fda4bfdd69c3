// mpr_tile.cu -- fused sweeps over shared-memory tiles with halos, many sweeps per launch.
//
// One work item is one sweep of one TH x TW tile of one grid.  The block that runs it
// copies the tile plus a halo of two sites of both colour planes from the sweep's source
// lattice buffer into shared memory, updates colour A (Algorithm 1) on the tile and on a
// one-site ring around it, then colour B on the tile, and writes the tile's interior to
// the other lattice buffer.  The ring updates duplicate what the neighbouring tiles compute
// for their own interior: every update is a deterministic function of its neighbours and
// of its Philox counter {site, sweep, chain, 0}, so the duplicates are bitwise identical
// and each tile's B pass sees exactly the post-A values of a whole-grid half-sweep.
// Reading one buffer and writing the other keeps every tile's halo at the pre-sweep state;
// consecutive sweeps alternate the buffers.
//
// Per tile, the gap sites are listed once at set-up, by pairs of plane columns of one region
// row (u16 (r << 8) | (qp << 2) | members, k_tile_lists): colour A inside the tile, then
// colour A on the ring, then colour B inside the tile, contiguous in a 16-byte aligned slot
// that is copied into shared memory together with the region.  The two sites of a pair
// share one Philox block.  Accumulators for the equilibrium average follow the interior
// entries (two slots per full pair, one per single site; A, then B).
//
// The sweep's accepted energy change (each site's rounded to a whole number of kDEUnit)
// and acceptance count go into per-grid, per-sweep 64-bit integer totals, whose sum does
// not depend on the order in which tiles finish;
// the block that completes a sweep's tiles of a grid (atomic ticket) runs the Algorithm 2
// control step for that grid in place, so no separate control launch is needed and the
// results are bitwise reproducible.  A whole phase of Algorithm 2 (the relaxation, or the
// M equilibrium sweeps) is one launch (k_tile_sweep).
#include <algorithm>
#include <vector>

#include "mpr_internal.cuh"

namespace mpr {

namespace {


template <int TH, int TW>
struct Geo {
    static constexpr int RH = TH + 4;                 // region rows (halo 2)
    static constexpr int RW = TW / 2 + 4;             // region plane columns
    static constexpr int RP = RW / 2;                 // region plane column pairs
    // pairs of plane columns (2 qp, 2 qp + 1) holding gap sites: colour A inside the tile
    // and on its ring, colour B inside the tile
    static constexpr int CAPA = TH * TW / 4 + TH + TW + 2;
    static constexpr int CAPB = TH * TW / 4;
    static constexpr int LIST = (CAPA + CAPB + 7) / 8 * 8;   // u16 entries per tile (16-byte slots)
    static constexpr int ACC = TH * TW;               // accumulator floats per tile: 2 per pair
    static_assert(TH % 2 == 0 && TW % 8 == 0, "tile origin parity, quads of columns, 16-byte stores");
    static_assert(RH <= 64 && RP <= 64, "entry encoding (r << 8) | (qp << 2) | members");

    static_assert(RW * 8 % 16 == 0, "TMA box rows must be a multiple of 16 bytes");
    static_assert((2 * RH * RW * 8) % 128 == 0, "list slots stay 16-byte aligned");
};

// Lists the gap sites of each tile (one warp per tile) in region coordinates, by pairs of
// plane columns: entry (r << 8) | (qp << 2) | members, where bit m of `members` marks
// plane column q = 2 qp + m of region row r as a gap site of the part's kind.  The two
// sites of a pair have the same colour and lie in one quad of grid columns (the tile origin
// is a multiple of 4), so they share one Philox block.  The interior parts list their full
// pairs (both bits) first, then the pairs with only site 0, then those with only site 1, so
// that the warps of a block take entries of one kind together; the ring part has one entry
// per site.  A pair never mixes interior and
// ring sites (the interior starts on an even plane column and spans an even number of them).
template <int TH, int TW>
__global__ void k_tile_lists(TileDesc* __restrict__ tiles, int ntiles,
                             const EntryDesc* __restrict__ ents, const uint8_t* __restrict__ mask,
                             int all_free, uint16_t* __restrict__ lists, TileCnt* __restrict__ cnts) {
    using G = Geo<TH, TW>;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const TileDesc td = tiles[t];
    const EntryDesc E = ents[td.entry];
    const uint8_t* m = mask ? mask + E.site0 : nullptr;
    uint16_t* out = lists + (long long)t * G::LIST;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;                                  // entries written so far
    int counts[3] = {0, 0, 0}, full[2] = {0, 0};
    // part 0: colour A, interior; part 1: colour A, ring; part 2: colour B, interior; each in
    // three rounds: full pairs, pairs of site 0 only, pairs of site 1 only
    for (int part = 0; part < 3; ++part) {
        const int c = part == 2 ? 1 : 0;
        const int n0 = n;
        for (int round = 0; round < 3; ++round) {
            if (round == 1 && part != 1) full[part >> 1] = n - n0;
            for (int base = 0; base < G::RH * G::RP; base += 32) {
                const int idx = base + lane;
                unsigned members = 0u;
                int r = 0, qp = 0;
                if (idx < G::RH * G::RP) {
                    r = idx / G::RP;
                    qp = idx - r * G::RP;
                    const int y = td.y0 - 2 + r;
                    const int s = c ^ (r & 1);
#pragma unroll
                    for (int mm = 0; mm < 2; ++mm) {
                        const int x = td.x0 + 2 * (2 * qp + mm) - 4 + s;
                        const bool in_grid = y >= 0 && y < E.H && x >= 0 && x < E.W;
                        const bool interior = y >= td.y0 && y < td.y0 + TH && x >= td.x0 && x < td.x0 + TW;
                        const bool ring = !interior && y >= td.y0 - 1 && y <= td.y0 + TH && x >= td.x0 - 1 &&
                                          x <= td.x0 + TW;
                        const bool gap = in_grid && (all_free || !m[(long long)y * E.W + x]);
                        if (gap && (part == 1 ? ring : interior)) members |= 1u << mm;
                    }
                }
                // interior: full pairs, then pairs of site 0 only, then of site 1 only; ring:
                // one entry per site (sites 0, then sites 1)
                unsigned emit;
                if (part == 1) emit = round < 2 ? members & (1u << round) : 0u;
                else emit = members == (round == 0 ? 3u : round == 1 ? 1u : 2u) ? members : 0u;
                const bool take = emit != 0u;
                const unsigned b = __ballot_sync(0xffffffffu, take);
                if (take) out[n + __popc(b & lt)] = (uint16_t)((r << 8) | (qp << 2) | (int)emit);
                n += __popc(b);
            }
        }
        counts[part] = n - n0;
    }
    if (lane == 0) {
        TileCnt c;
        c.nA_int = (uint16_t)counts[0];
        c.nA_ring = (uint16_t)counts[1];
        c.nB = (uint16_t)counts[2];
        c.nA_full = (uint16_t)full[0];
        c.nB_full = (uint16_t)full[1];
        c._pad = 0;
        cnts[t] = c;
        tiles[t].nA_int = counts[0];
        tiles[t].nA_ring = counts[1];
        tiles[t].nB = counts[2];
        tiles[t].nfull = full[0] | (full[1] << 16);
    }
}

// ---------------------------------------------------------------- TMA and mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}
// Tiled bulk copy of a 3-D box (x = plane column, y = padded row, z = colour plane).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from global to shared memory.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"((unsigned long long)src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Orders this thread's generic-proxy shared-memory writes before later async-proxy reads.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity), "r"(100000u) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_try(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < 3000u; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- waits between blocks
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bench support (mpr_debug_trace): thread 0 stamps the phases of its work items and the
// control steps with the global timer, when the launch carries a trace buffer.  The item
// stamps are compiled into a separate instantiation of the sweep kernel (TRACE), which
// runs only while a trace buffer is set: in the kernel that runs otherwise they cost
// about 1.5 % of a sweep.
__device__ __forceinline__ void trace_item(const TileArgs& A, unsigned w, int k) {
    if (A.trace && w < A.trace_items) A.trace[(unsigned long long)w * kTraceWords + k] = gtimer();
}
__device__ __forceinline__ void trace_block(const TileArgs& A, unsigned w) {
    if (A.trace && w < A.trace_items) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        A.trace[(unsigned long long)w * kTraceWords + 5] =
            (unsigned long long)blockIdx.x | ((unsigned long long)smid << 32);
    }
}
__device__ __forceinline__ void trace_ctl(const TileArgs& A, uint32_t sig, int k) {
    if (A.trace)
        A.trace[A.trace_items * kTraceWords + 2ull * (sig % (uint32_t)kTraceCtl) + (unsigned)k] = gtimer();
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    return (int)ld_relaxed(reinterpret_cast<const unsigned*>(p));
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// with a preceding relaxed load that observed a release store: acquire
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// orders this thread's generic-proxy global accesses with its later async-proxy (TMA) ones
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// One thread spins until ready() holds.  It gives up, with the launch's error flag set,
// as soon as another block has set the flag or once the wait outlives A.wait_ns.
template <class F>
__device__ __forceinline__ bool bounded_wait(const TileArgs& A, F ready) {
    if (ready()) return true;
    const unsigned long long t0 = gtimer();
    for (unsigned k = 1;; ++k) {
        if (ready()) return true;
        if ((k & 7u) == 0u) {
            if (ld_relaxed(A.err) != 0) return false;
            if (gtimer() - t0 > A.wait_ns) {
                atomicExch(A.err, 1);
                return false;
            }
        }
    }
}

// Control state in 8-byte words through L2 (other blocks rewrite it during a launch).
static_assert(sizeof(Ctl) % 8 == 0 && offsetof(Ctl, sweep) % 8 == 0 &&
                  offsetof(Ctl, go_hqd) == offsetof(Ctl, sweep) + 4 &&
                  offsetof(Ctl, sweep) + 8 == sizeof(Ctl),
              "the sweep counter and its window are published as one word, last");
__device__ __forceinline__ Ctl ctl_load(const Ctl* p) {
    Ctl c;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&c);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(Ctl) / 8); ++i) dst[i] = __ldcg(src + i);
    return c;
}
// Every field but the last word, then the word {sweep, go_hqd} with release semantics: a
// block that acquires the new counter sees the whole control step.
__device__ __forceinline__ void ctl_publish(Ctl* p, const Ctl& c) {
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(p);
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&c);
    constexpr int kLast = (int)(offsetof(Ctl, sweep) / 8);
#pragma unroll
    for (int i = 0; i < kLast; ++i) __stcg(dst + i, src[i]);
    st_release(dst + kLast, src[kLast]);
}
// The published word {sweep, go_hqd} of a grid, in one load.
struct CtlGo {
    uint32_t sweep;
    float go_hqd;
};
__device__ __forceinline__ CtlGo ctl_go(const Ctl* p) {
    const unsigned long long v = ld_relaxed(reinterpret_cast<const unsigned long long*>(&p->sweep));
    return CtlGo{(uint32_t)v, __uint_as_float((uint32_t)(v >> 32))};
}

// Per-item parameters staged in shared memory by the issuing thread, in 16-byte groups
// so that each thread picks up what it needs with a few vector loads.
struct __align__(16) TileParams {
    int t, y0, x0, W;                     // tile (-1: no item), origin, grid width
    uint32_t chain, sweep;                // Philox counter words 2 and 1
    float half_qd, neg_inv_T;             // proposal half-angle scale, -1/T
    int nA_int, nA_ring, nB, e;           // list counts, grid
    int nfull, H, pitch, cur;             // full pairs (A | B << 16), grid height, row pitch, source buffer
    long long pl0, pl1;                   // plane offsets of the grid in the lattice buffers
};

// What the issuing thread keeps of the grid of the last item it looked at (constant
// during a launch).
struct GridCache {
    int e, W, H, pitch;
    int tile0, tpr, ntr, ntiles;          // first tile, tiles per row and per column, count
    uint32_t chain, sweep_base;
    int cur_base;
    float neg_inv_T;
    long long pl0, pl1;
    int stopped;                          // its relaxation has ended (seen in this launch)
    unsigned skips;                       // items of stopped grids skipped by this block
    uint32_t seen;                        // a sweep counter of the grid this thread acquired
    float seen_hqd;                       // relaxation: the window of sweep `seen`
};

// Thread 0 of a block, after a barrier that follows every warp's flush of the block's
// totals for grid e at sweep sig: n more tiles of that sweep are done.  The block that
// completes the sweep's tiles runs the grid's Algorithm 2 control step from the totals --
// after the control step of sweep sig - 1, which a fixed-window launch may still be
// running -- and publishes it.
template <bool TRACE>
__device__ void tile_ticket(const TileArgs& A, int e, uint32_t sig, int n) {
    const int slot = e * kSlots + (int)(sig & (uint32_t)(kSlots - 1));
    fence_acq_rel();                          // the block's flushes (after a barrier) before the ticket
    const unsigned prev = atomicAdd(A.ticket + slot, (unsigned)n);
    if (prev + (unsigned)n != (unsigned)A.ents[e].ntiles) return;
    if (TRACE) trace_ctl(A, sig, 0);
    fence_acq_rel();                          // every block's flushes before the totals are read
    Ctl* cp = A.ctl + e;
    // a fixed-window launch may still be running the control step of sweep sig - 1; in the
    // relaxation this thread acquired it before staging the sweep's tiles
    if (!A.relax && !bounded_wait(A, [&] { return ld_acquire(&cp->sweep) == sig; })) return;
    Ctl c = ctl_load(cp);                                     // in flight with the exchanges
    const long long f = (long long)atomicExch(A.gsum + 2 * slot, 0ull);
    const unsigned long long na = atomicExch(A.gsum + 2 * slot + 1, 0ull);
    atomicExch(A.ticket + slot, 0u);
    control_step(c, A.ents[e], (double)f * kDEUnit, na, A.mode, A.A_targ, A.k_a, A.n_f, A.n_fit,
                 A.i_max, A.ehist + (long long)e * A.ehist_stride, 1);
    ctl_publish(cp, c);
    if (TRACE) trace_ctl(A, sig, 1);
    if (A.relax && c.stop) atomicSub(A.live, 1);
}

// Persistent fused sweeps: A.nsweeps sweeps of every tile of every grid in one launch.
// Work item w is sweep s = w / ntiles of tile A.desc[w % ntiles]; blocks take items from a
// global counter in increasing order (the last block to leave resets it), so faster blocks
// take more items.  An item starts once what it reads is final:
//  * relaxation (Algorithm 2 step 5): sweep s of a grid needs the window that the control
//    step of sweep s - 1 chose, and runs only if that step did not end the relaxation, so
//    its items wait for that control step (which follows every tile of sweep s - 1);
//  * fixed window: tile t at sweep s needs the interiors of t and its 8 neighbours after
//    sweep s - 1 (its halo is two sites wide), and writes the buffer those tiles read at
//    sweep s - 1, so it waits for the 9 tiles' completion counters to pass s - 1; sweeps
//    overlap wherever the tiles allow.
// Items are taken in increasing order and depend only on items before them, so the
// smallest unfinished item can always run: the launch cannot deadlock, whatever the
// number of resident blocks.  Every wait is bounded (A.wait_ns); an expired wait sets the
// error flag and every block leaves after its copies have landed.
// Thread 0 stages an item: a TMA box of both colour planes plus the bulk-copied gap list,
// completing on the block's mbarrier.  Each thread keeps its energy change (fixed point)
// and acceptance count summed over the block's consecutive items of one grid and sweep;
// before the block moves on to another grid or sweep, the warps add them to that sweep's
// slot of the grid's totals and thread 0 adds the block's tile count to the slot's
// ticket.  The block that completes a sweep's tiles runs the grid's control step.
// The interior rows of both planes go back to the other lattice buffer as 16-byte stores.
template <int TH, int TW, int TRIG, bool ACC, int NT, int MB, bool TRACE = false>
__global__ void __launch_bounds__(NT, MB)
k_tile_sweep(const TileArgs A) {
    static_assert(TW % 8 == 0, "write-back in 16-byte vectors");
    using G = Geo<TH, TW>;
    extern __shared__ __align__(128) unsigned char dsm[];
    float2(*sm)[G::RH][G::RW] = reinterpret_cast<float2(*)[G::RH][G::RW]>(dsm);
    uint16_t* list = reinterpret_cast<uint16_t*>(dsm + 2 * G::RH * G::RW * sizeof(float2));
    __shared__ TileParams sp;
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) TileDesc dnext;
    __shared__ GridCache gc;
    __shared__ int s_fail, s_flush, s_ke, s_kn, s_last, s_pub_t;
    __shared__ uint32_t s_ksig, s_pub_sig;
    __shared__ unsigned s_w0;
    __shared__ unsigned s_wcur;           // the staged item (trace)
    unsigned w1 = 0u;                     // thread 0: the item after s_w0 (an atomic in flight)
    __shared__ long long s_fx[NT];
    __shared__ unsigned s_nat[NT];
    constexpr uint32_t kBytes = 2u * G::RH * G::RW * sizeof(float2);
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = (unsigned)A.ntiles;
    const unsigned nitems = (unsigned)A.nsweeps * ntiles;

    // thread 0 only: item s_w0 is next (its descriptor is on its way into dnext), w1 the
    // one after (taken from the counter an item ahead and kept in a register, so staging
    // never waits on the atomic)
    auto fetch_desc = [&](unsigned w) {
        const TileDesc* src = A.desc + (w % ntiles);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(&dnext)), "l"(src) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(&dnext) + 16u),
                     "l"(reinterpret_cast<const char*>(src) + 16) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto load_grid = [&](int e) {
        const EntryDesc& E = A.ents[e];
        const Ctl* cp = A.ctl + e;
        gc.e = e;
        gc.W = E.W;
        gc.H = E.H;
        gc.pitch = E.pitch;
        gc.tile0 = E.tile0;
        gc.tpr = (E.W + TW - 1) / TW;
        gc.ntr = (E.H + TH - 1) / TH;
        gc.ntiles = E.ntiles;
        gc.chain = E.chain;
        gc.pl0 = E.plane[0];
        gc.pl1 = E.plane[1];
        gc.sweep_base = __ldcg(&cp->sweep_base);
        gc.cur_base = __ldcg(&cp->cur_base);
        gc.neg_inv_T = __ldcg(&cp->neg_inv_T);
        gc.stopped = A.relax ? ld_relaxed(&cp->stop) : 0;     // stays set once set
        gc.seen = gc.sweep_base;
        gc.seen_hqd = -1.0f;                                  // none yet
    };
    // thread 0, fixed window: publishes that the last item's tile has finished its sweep (its
    // interior is in the other buffer and it no longer reads its source buffer).  Deferred
    // until after the next copy has been issued, unless that copy must wait for a tile.
    auto publish = [&]() {
        if (s_pub_t >= 0) {
            // the release is cumulative: it covers the block's write-back stores, ordered
            // before it by the barrier that precedes this call
            st_release(A.tdone + s_pub_t, s_pub_sig);
            s_pub_t = -1;
        }
    };
    // stages the next item to run into sp, or sets sp.t = -1 when there is none (all items
    // taken, every grid's relaxation ended, or an expired wait)
    auto issue = [&]() {
        for (;;) {
            const unsigned w = s_w0;
            if (w >= nitems) { sp.t = -1; return; }
            if (TRACE) trace_item(A, w, 0);
            asm volatile("cp.async.wait_all;" ::: "memory");          // the descriptor of w
            const TileDesc d = dnext;
            const unsigned wn = w1;
            s_w0 = wn;
            if (wn < nitems) fetch_desc(wn);
            w1 = atomicAdd(A.sched, 1u);
            const int e = d.entry;
            if (e != gc.e) load_grid(e);
            const unsigned s = w / ntiles;
            const uint32_t sig = gc.sweep_base + s;
            Ctl* cp = A.ctl + e;
            float half_qd = A.half_qd_fixed;
            bool ok = true;
            if (A.relax) {
                if (gc.stopped) {                                     // this grid has stopped
                    // and every grid? (looked at every 16th skipped item)
                    if ((++gc.skips & 15u) == 0u && ld_relaxed(A.live) <= 0) { sp.t = -1; return; }
                    continue;
                }
                if (sig == gc.seen && gc.seen_hqd > 0.0f) {
                    // this thread already acquired the control step of sweep sig - 1 (and it
                    // did not end the relaxation): nothing to wait for or load again
                    half_qd = gc.seen_hqd;
                } else {
                    // ready once the control step of sweep sig - 1 is published, or the
                    // grid's relaxation has ended: one word says both, and the window
                    // (every block polls the same word, so gently)
                    CtlGo g{0u, 0.0f};
                    ok = bounded_wait(A, [&] {
                        g = ctl_go(cp);
                        if ((int)(g.sweep - sig) >= 0 || g.go_hqd < 0.0f) return true;
                        __nanosleep(64);
                        return false;
                    });
                    fence_acq_rel();
                    if (ok && g.go_hqd < 0.0f) {                      // this grid has stopped
                        gc.stopped = 1;
                        continue;
                    }
                    half_qd = g.go_hqd;
                    if (ok) {                                         // kept for the sweep's other tiles
                        gc.seen = sig;
                        gc.seen_hqd = half_qd;
                    }
                }
            } else if (s > 0 && (int)(gc.seen - sig) < 0) {
                // the halo: tile t and its 8 neighbours have finished sweep sig - 1; and the
                // slot of sweep sig was emptied by the control step of sweep sig - kSlots.
                // (Nothing to wait for once this thread has acquired a sweep counter >= sig:
                // the control step of sweep sig - 1 follows every tile of that sweep.)
                const int i = d.t - gc.tile0, ty = i / gc.tpr, tx = i - ty * gc.tpr;
                const uint32_t slot_free = sig - (uint32_t)(kSlots - 1);
                auto ready = [&] {
                    unsigned v[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        const int yy = ty + k / 3 - 1, xx = tx + k % 3 - 1;
                        v[k] = (yy >= 0 && yy < gc.ntr && xx >= 0 && xx < gc.tpr)
                                   ? ld_relaxed(A.tdone + gc.tile0 + yy * gc.tpr + xx) : sig;
                    }
                    const unsigned cs = ld_relaxed(&cp->sweep);
                    if ((int)(cs - gc.seen) > 0) gc.seen = cs;        // acquired by the fence below
                    bool r = (int)(cs - slot_free) >= 0;
#pragma unroll
                    for (int k = 0; k < 9; ++k) r = r && (int)(v[k] - sig) >= 0;
                    return r;
                };
                if (!ready()) {
                    publish();                  // this block's last tile may be one of the nine
                    ok = bounded_wait(A, [&] {
                        if (ready()) return true;
                        __nanosleep(32);
                        return false;
                    });
                }
                fence_acq_rel();
            }
            if (!ok) { sp.t = -1; return; }
            const int cur = gc.cur_base ^ (int)(s & 1u);
            fence_proxy_async_global();                               // writes of other blocks before the copy
            TileParams P;
            P.t = d.t;
            P.y0 = d.y0;
            P.x0 = d.x0;
            P.W = gc.W;
            P.chain = gc.chain;
            P.sweep = sig;
            P.half_qd = half_qd;
            P.neg_inv_T = gc.neg_inv_T;
            P.nA_int = d.nA_int;
            P.nA_ring = d.nA_ring;
            P.nB = d.nB;
            P.e = e;
            P.nfull = d.nfull;
            P.H = gc.H;
            P.pitch = gc.pitch;
            P.cur = cur;
            P.pl0 = gc.pl0;
            P.pl1 = gc.pl1;
            sp = P;
            if (TRACE) {
                s_wcur = w;
                trace_item(A, w, 1);
                trace_block(A, w);
            }
            const uint32_t lbytes = ((uint32_t)(d.nA_int + d.nA_ring + d.nB) * 2u + 15u) & ~15u;
            mbar_expect_tx(&bar, kBytes + lbytes);
            tma_load_3d(&sm[0][0][0], A.maps + 2 * e + cur, &bar, d.x0 >> 1, d.y0 - 1, 0);
            if (lbytes) bulk_load(list, A.lists + (long long)d.t * G::LIST, lbytes, &bar);
            return;
        }
    };
    // thread 0, after an item of grid e at sweep sig: does the next item belong to another
    // grid or sweep (or is there none)?  Then the block hands in its totals first.
    auto next_differs = [&](int e, uint32_t sig) {
        const unsigned w = s_w0;
        if (w >= nitems) return true;
        asm volatile("cp.async.wait_all;" ::: "memory");
        const int ne = dnext.entry;
        if (ne != gc.e) load_grid(ne);
        return ne != e || gc.sweep_base + w / ntiles != sig;
    };
    auto flush_partials = [&](int e, uint32_t sig) {
        long long w = s_fx[threadIdx.x];
        unsigned long long wn = s_nat[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, o);
            wn += __shfl_xor_sync(0xffffffffu, wn, o);
        }
        if (lane == 0) {
            const int slot = e * kSlots + (int)(sig & (uint32_t)(kSlots - 1));
            if (w) atomicAdd(A.gsum + 2 * slot, (unsigned long long)w);
            if (wn) atomicAdd(A.gsum + 2 * slot + 1, wn);
        }
        s_fx[threadIdx.x] = 0;
        s_nat[threadIdx.x] = 0u;
    };

    if (threadIdx.x == 0) {
        // test support: a wait that must expire (before block 0 takes any item, so that it
        // happens whatever the order in which the blocks start)
        if (A.stall && blockIdx.x == 0) (void)bounded_wait(A, [&] { return ld_relaxed(A.sched + 2) != 0u; });
        mbar_init(&bar, 1);
        fence_barrier_init();
        s_fail = 0;
        s_flush = 0;
        s_ke = -1;
        s_kn = 0;
        s_pub_t = -1;
        gc.e = -1;
        gc.skips = 0u;
        s_w0 = atomicAdd(A.sched, 1u);
        w1 = atomicAdd(A.sched, 1u);
        if (s_w0 < nitems) fetch_desc(s_w0);
    }
    s_fx[threadIdx.x] = 0;
    s_nat[threadIdx.x] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) issue();

    for (int it = 0;; ++it) {
        const uint32_t parity = (uint32_t)it & 1u;
        if (it > 0) {
            __syncthreads();                                      // B0: write-back and flushes issued
            if (threadIdx.x == 0) {
                if (TRACE) trace_item(A, s_wcur, 4);
                // the previous item is done (a relaxation's items wait for control steps,
                // not for tiles: their counters are set when the launch ends)
                if (!A.relax) {
                    s_pub_t = sp.t;
                    s_pub_sig = sp.sweep + 1u;
                }
                if (s_flush) {
                    publish();
                    tile_ticket<TRACE>(A, s_ke, s_ksig, s_kn);
                    s_ke = -1;
                    s_kn = 0;
                }
                issue();
                publish();
            }
        }
        if (threadIdx.x == 0 && sp.t >= 0 && !mbar_wait_try(&bar, parity)) {
            atomicExch(A.err, 1);
            s_fail = 1;
        }
        __syncthreads();                                          // B1: the tile is in shared memory
        const int4 g0 = *reinterpret_cast<const int4*>(&sp.t);
        const int t = g0.x;
        if (t < 0) break;
        if (s_fail) {
            // give the late copy a second bounded wait to land before the block's shared
            // memory goes away (no other copy is in flight at B1), then leave
            if (threadIdx.x == 0) (void)mbar_wait_try(&bar, parity);
            break;
        }
        (void)mbar_test(&bar, parity);                            // each thread acquires the copy
        if (TRACE && threadIdx.x == 0) trace_item(A, s_wcur, 2);
        const int y0 = g0.y, x0 = g0.z, W = g0.w;
        const int4 g1 = *reinterpret_cast<const int4*>(&sp.chain);
        const int4 g2 = *reinterpret_cast<const int4*>(&sp.nA_int);
        const uint32_t chain = (uint32_t)g1.x, sweep = (uint32_t)g1.y;
        const float half_qd = __int_as_float(g1.z), kx = accept_scale<TRIG>(__int_as_float(g1.w));
        const int nA_int = g2.x, nA = g2.x + g2.y, nB = g2.z, e = g2.w;
        float* __restrict__ acc = ACC ? A.acc + (long long)t * G::ACC : nullptr;
        if (threadIdx.x == 0) {
            if (s_ke < 0) {
                s_ke = e;
                s_ksig = sweep;
            }
            ++s_kn;
        }

        // colour A on the tile and its ring, then colour B on the tile; energy changes in
        // fixed point per site, summed in 32 bits (at most kDEMaxSites32 sites a thread)
        static_assert(2 * ((G::LIST + NT - 1) / NT) <= kDEMaxSites32, "32-bit energy partial");
        int dE = 0;
        unsigned nacc = 0;
        const int nfull = *reinterpret_cast<const int*>(&sp.nfull);
        const uint32_t quads = (uint32_t)((W + 3) >> 2), quad0 = (uint32_t)(x0 >> 2) - 1u;
        const int sitesA = (nfull & 0xFFFF) + nA_int;     // accumulator slots of colour A
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int c = pass;                           // colour being updated
            const int n = pass ? nB : nA;
            const int nf = pass ? (nfull >> 16) : (nfull & 0xFFFF);
            const uint16_t* lst = pass ? list + nA : list;
            float* __restrict__ pacc = ACC ? acc + (pass ? sitesA : 0) : nullptr;
            float2(*own)[G::RW] = sm[c];
            float2(*oth)[G::RW] = sm[c ^ 1];
            // Algorithm 1 on plane column q of region row r with the pair's uniforms (ru:
            // proposal, ra: acceptance); own: an interior site (its energy change and
            // acceptance count, and its running angle sum in slot aidx)
            auto update = [&](int r, int q, uint32_t ru, uint32_t ra, bool own_site, int aidx) {
                // the running angle sum is loaded first, so that its latency hides behind
                // the update (from L2: another block may have written it in this launch)
                float acc_old = 0.0f;
                if (ACC && own_site) acc_old = __ldcg(pacc + aidx);
                const int s = c ^ (r & 1);
                const float2 nu = oth[r - 1][q], nd = oth[r + 1][q];
                const float2 nl = oth[r][q - 1 + s], nr = oth[r][q + s];
                const float C = (nu.x + nd.x) + (nl.x + nr.x);
                const float S = (nu.y + nd.y) + (nl.y + nr.y);
                float2 v = own[r][q];
                const float hq = (u24f(ru) - 0.5f) * half_qd;
                bool accepted;
                float Fx = 0.0f, Fy = 0.0f;
                if (A.or_mode == OR_LITERAL) literal_field(nu, nd, nl, nr, Fx, Fy);
                const float d = hybrid_update<TRIG>(v, C, S, Fx, Fy, hq, u24f(ra), kx, A.or_mode, accepted);
                own[r][q] = v;
                if (own_site) {
                    dE += de_fixed(d);
                    nacc += accepted ? 1u : 0u;
                    if (ACC) __stcg(pacc + aidx, acc_old + angle_upper(v.x, v.y));
                }
            };
            // the pair's Philox block: counter {quad, sweep, chain, colour}
            auto block = [&](int r, int qp) {
                const uint32_t quad = (uint32_t)(y0 - 2 + r) * quads + quad0 + (uint32_t)qp;
                return philox10(make_uint4(quad, sweep, chain, (uint32_t)c), A.rk);
            };
            // pairs of two gap sites: both updates from one block (interior sites only)
            for (int k = threadIdx.x; k < nf; k += NT) {
                const int ent = lst[k];
                const int r = ent >> 8, qp = (ent >> 2) & 63;
                const uint4 rnd = block(r, qp);
                update(r, 2 * qp, rnd.x, rnd.y, true, 2 * k);
                update(r, 2 * qp + 1, rnd.z, rnd.w, true, 2 * k + 1);
            }
            // single sites: the ring belongs to other tiles, its sites count nowhere
            for (int k = nf + threadIdx.x; k < n; k += NT) {
                const int ent = lst[k];
                const int r = ent >> 8, qp = (ent >> 2) & 63, mm = (ent >> 1) & 1;
                const uint4 rnd = block(r, qp);
                update(r, 2 * qp + mm, mm ? rnd.z : rnd.x, mm ? rnd.w : rnd.y, pass || k < nA_int, nf + k);
            }
            if (pass == 0) __syncthreads();               // B2: colour A done
        }
        s_fx[threadIdx.x] += dE;
        s_nat[threadIdx.x] += nacc;
        if (threadIdx.x == 0) s_flush = next_differs(e, sweep) ? 1 : 0;
        fence_proxy_async_smem();                         // this thread's stage writes before the next copy into it
        __syncthreads();                                  // B3: colour B done
        if (TRACE && threadIdx.x == 0) trace_item(A, s_wcur, 3);
        const int4 g3 = *reinterpret_cast<const int4*>(&sp.nfull);
        // interior rows of both colours to the other buffer (samples included), 16 bytes
        // per thread and step, one warp per row; rows and columns beyond the grid skipped
        {
            const int rows = min(TH, g3.y - y0);
            const int pc = (x0 >> 1) + 2;
            const int nv = (min(TW / 2, g3.z - pc) & ~1) >> 1;        // 16-byte vectors per row
            const long long pl0 = sp.pl0, pl1 = sp.pl1;
            float2* __restrict__ dst = g3.w ? A.lat[0] : A.lat[1];
            constexpr int V = TW / 4;
#pragma unroll
            for (int i = threadIdx.x; i < 2 * TH * V; i += NT) {
                const int c = i / (TH * V), rr = (i / V) % TH, v = i % V;
                if (rr < rows && v < nv) {
                    const float4 val = *reinterpret_cast<const float4*>(&sm[c][rr + 2][2 + 2 * v]);
                    *reinterpret_cast<float4*>(dst + (c ? pl1 : pl0) + (long long)(y0 + rr + 1) * g3.z +
                                               pc + 2 * v) = val;
                }
            }
        }
        if (s_flush) flush_partials(e, sweep);
    }
    // an error or the end of the relaxation can leave totals that were not handed in
    __syncthreads();
    {
        const int ke = s_ke;
        if (ke >= 0 && s_kn > 0) {
            flush_partials(ke, s_ksig);
            __syncthreads();
            if (threadIdx.x == 0) tile_ticket<TRACE>(A, ke, s_ksig, s_kn);
        }
    }
    // leave: the last block out resets the counters for the next launch and records every
    // grid's sweep counter and buffer as the next launch's base (every block has stopped
    // taking items, and every control step has run, by the time it counts itself out)
    if (threadIdx.x == 0) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __threadfence();
        s_last = atomicAdd(A.sched + 1, 1u) == gridDim.x - 1u ? 1 : 0;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last) {
        for (int e = threadIdx.x; e < A.n_ent; e += NT) {
            Ctl* cp = A.ctl + e;
            cp->sweep_base = ld_relaxed(&cp->sweep);
            cp->cur_base = ld_relaxed(&cp->cur);
        }
        if (A.relax)
            for (int j = threadIdx.x; j < A.ntiles; j += NT) {
                const TileDesc& d = A.desc[j];
                A.tdone[d.t] = ld_relaxed(&A.ctl[d.entry].sweep);
            }
        if (threadIdx.x == 0) {
            atomicExch(A.sched, 0u);
            atomicExch(A.sched + 1, 0u);
        }
    }
}

// Tile order of the relaxation: each grid's tiles heaviest first, in 256 buckets of the
// listed gap count (the order inside a bucket is arbitrary: every update depends only on
// its neighbours and its counter, and the totals are order-independent, so no result
// depends on it).  Handing out the heavy tiles first makes a sweep's tail out of light
// tiles, which matters where every sweep waits for the previous one's control step.
__device__ __forceinline__ int work_bucket(const TileDesc& d, int maxw) {
    // site updates: one per entry, two for a full pair
    const int w = d.nA_int + d.nA_ring + d.nB + (d.nfull & 0xFFFF) + (d.nfull >> 16);
    return 255 - min(255, (int)((long long)w * 256 / (maxw + 1)));
}
__global__ void k_tile_hist(const TileDesc* __restrict__ tiles, int ntiles, int maxw, unsigned* hist) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const TileDesc d = tiles[t];
    atomicAdd(hist + d.entry * 256 + work_bucket(d, maxw), 1u);
}
__global__ void k_tile_scan(unsigned* hist, const EntryDesc* __restrict__ ents, int n_ent) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ent) return;
    unsigned run = (unsigned)ents[e].tile0;
    for (int b = 0; b < 256; ++b) {
        const unsigned c = hist[e * 256 + b];
        hist[e * 256 + b] = run;
        run += c;
    }
}
__global__ void k_tile_scatter(const TileDesc* __restrict__ tiles, int ntiles, int maxw, unsigned* hist,
                               TileDesc* __restrict__ ord) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const TileDesc d = tiles[t];
    ord[atomicAdd(hist + d.entry * 256 + work_bucket(d, maxw), 1u)] = d;
}

__global__ void k_tile_sync(const TileDesc* __restrict__ tiles, int ntiles, Ctl* ctl, int n_ent,
                            unsigned* __restrict__ tdone) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ntiles) tdone[i] = ctl[tiles[i].entry].sweep;
    if (i < n_ent) {
        ctl[i].sweep_base = ctl[i].sweep;
        ctl[i].cur_base = ctl[i].cur;
    }
}

__global__ void k_count_live(const Ctl* __restrict__ ctl, int n_ent, int* live) {
    __shared__ int n;
    if (threadIdx.x == 0) n = 0;
    __syncthreads();
    int m = 0;
    for (int e = threadIdx.x; e < n_ent; e += blockDim.x) m += ctl[e].stop ? 0 : 1;
    if (m) atomicAdd(&n, m);
    __syncthreads();
    if (threadIdx.x == 0) *live = n;
}

// zhat at the gap sites of every tile (same mean and inverse map as the list path).  With
// K > 1 the angle sums of K chains of the same grid are added: chain c's copy of tile t is
// tile t + c * chain_tiles (every chain has the same tiles and lists).  zr, when given, holds
// each entry's (z_min, z_max), so that one launch serves the tiles of many grids.
template <int TH, int TW>
__global__ void k_tile_predict_out(const TileDesc* __restrict__ tiles, const TileCnt* __restrict__ cnts,
                                   const uint16_t* __restrict__ lists, const float* __restrict__ acc,
                                   const EntryDesc* __restrict__ ents, int M, double q, double zmin,
                                   double zmax, const double2* __restrict__ zr, int K, int chain_tiles,
                                   float* __restrict__ zhat) {
    using G = Geo<TH, TW>;
    const int tile = blockIdx.x;
    const TileDesc td = tiles[tile];
    const EntryDesc E = ents[td.entry];
    const TileCnt cnt = cnts[tile];
    if (zr) {
        zmin = zr[td.entry].x;
        zmax = zr[td.entry].y;
    }
    const uint16_t* list = lists + (long long)tile * G::LIST;
    const float* a = acc + (long long)tile * G::ACC;
    const long long cstride = (long long)chain_tiles * G::ACC;
    const int nA = cnt.nA_int + cnt.nA_ring;
    const double f = (zmax - zmin) / (kTwoPi * q * (double)M * (double)K);
    // interior entries of both colours (as in the sweep: full pairs in slots 2k, 2k + 1,
    // single sites of part p in slot nf_p + k, colour B after colour A's slots)
    const int sitesA = cnt.nA_full + cnt.nA_int;
    for (int k = threadIdx.x; k < cnt.nA_int + cnt.nB; k += blockDim.x) {
        const bool isA = k < cnt.nA_int;
        const int kk = isA ? k : k - cnt.nA_int;           // entry within its part
        const int nf = isA ? cnt.nA_full : cnt.nB_full;
        const int ent = isA ? list[k] : list[nA + kk];
        const int r = ent >> 8, qp = (ent >> 2) & 63;
        const int s = (isA ? 0 : 1) ^ (r & 1);
        const int y = td.y0 - 2 + r;
        const int base = isA ? 0 : sitesA;
        for (int mm = 0; mm < 2; ++mm) {
            if (!((ent >> mm) & 1)) continue;
            const int slot = base + (kk < nf ? 2 * kk + mm : nf + kk);
            const int x = td.x0 + 2 * (2 * qp + mm) - 4 + s;
            double sum = (double)a[slot];
            for (int c = 1; c < K; ++c) sum += (double)a[c * cstride + slot];
            double v = zmin + sum * f;
            v = v < zmin ? zmin : (v > zmax ? zmax : v);
            zhat[E.site0 + (long long)y * E.W + x] = (float)v;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- compiled configurations
// The tile shapes the library is built with; the autotuner picks one per batch.
//   id  TH  TW  threads  blocks/SM register budget
//    0  16 128     128    8
//    1  32  64     128    8
//    2  32 128     256    4
#define MPR_TILE_CONFIGS(X) \
    X(0, 16, 128, 128, 8)  \
    X(1, 32, 64, 128, 8)   \
    X(2, 32, 128, 256, 4)

template <int TH, int TW>
struct Cfg {
    using G = Geo<TH, TW>;
    static constexpr int SMEM = 2 * G::RH * G::RW * 8 + G::LIST * 2;
};

#define MPR_CFG_GEOM(id, th, tw, nt, mb) \
    case id: g = TileGeom{th, tw, Geo<th, tw>::RH, Geo<th, tw>::RW, Geo<th, tw>::LIST, Geo<th, tw>::ACC, nt}; break;
TileGeom tile_geom(int cfg) {
    TileGeom g{0, 0, 0, 0, 0, 0, 0};
    switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_GEOM) default: break; }
    return g;
}
int tile_config_count() { return 3; }
int tile_max_rows() { return 32 + 4; }
int tile_max_cols() { return 128 / 2 + 4; }

// Tensor maps of every entry's two lattice buffers, viewed as 3-D boxes
// {plane column, padded row, colour} of the configuration's region size: 8-byte elements,
// zero fill out of bounds.
cudaError_t make_tile_maps(int cfg, const EntryDesc* ents, int n_ent, float2* lat0, float2* lat1,
                           CUtensorMap* d_maps, cudaStream_t st) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const TileGeom g = tile_geom(cfg);
    std::vector<CUtensorMap> maps((size_t)2 * n_ent);
    for (int e = 0; e < n_ent; ++e) {
        const EntryDesc& E = ents[e];
        for (int b = 0; b < 2; ++b) {
            float2* base = (b ? lat1 : lat0) + E.plane[0];
            const cuuint64_t dims[3] = {(cuuint64_t)E.pitch, (cuuint64_t)E.prows, 2};
            const cuuint64_t strides[2] = {(cuuint64_t)E.pitch * 8, (cuuint64_t)E.prows * E.pitch * 8};
            const cuuint32_t box[3] = {(cuuint32_t)g.rw, (cuuint32_t)g.rh, 2};
            const cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = encode(&maps[2 * e + b], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims,
                                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
    }
    return cudaMemcpyAsync(d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice, st);
}

// Opts the sweep kernels of every configuration into their dynamic shared memory (more
// than the default 48 KB) and returns the persistent grid size of configuration cfg:
// blocks per SM at its footprint times the SMs.  Called from set-up code, never under
// stream capture.
template <int TH, int TW, int NT, int MB>
int blocks_for() {
    constexpr int sm = Cfg<TH, TW>::SMEM;
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_FAST, true, NT, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_FAST, false, NT, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, MB, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, MB, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per, k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, MB>, NT, sm);
    return std::max(1, sms * std::max(1, per));
}

#define MPR_CFG_BLOCKS(id, th, tw, nt, mb) \
    case id: blocks[id] = blocks_for<th, tw, nt, mb>(); break;
int tile_sweep_blocks(int cfg) {
    static int blocks[8] = {0};
    if (cfg < 0 || cfg >= tile_config_count()) return 0;
    if (!blocks[cfg]) {
        switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_BLOCKS) default: break; }
    }
    return blocks[cfg];
}

#define MPR_CFG_LISTS(id, th, tw, nt, mb) \
    case id: k_tile_lists<th, tw><<<(ntiles * 32 + 127) / 128, 128, 0, st_>>>(tiles, ntiles, ents, mask, all_free, lists, cnts); break;
cudaError_t launch_tile_lists(int cfg, TileDesc* tiles, int ntiles, const EntryDesc* ents,
                              const uint8_t* mask, int all_free, uint16_t* lists, TileCnt* cnts,
                              cudaStream_t st_) {
    if (ntiles == 0) return cudaSuccess;
    count_launches(1, st_);
    switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_LISTS) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

// Streaming multiprocessors of the current device (looked up once, like the block counts).
int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(1, n);
    }
    return sms;
}

template <int TH, int TW, int NT, int MB>
void sweep_for(const TileArgs& a, int trig, cudaStream_t st) {
    constexpr int sm = Cfg<TH, TW>::SMEM;
    // persistent: at most the resident blocks, and no more than the launch's items.  With
    // fewer tiles per sweep than resident blocks, at most as many blocks per SM as a sweep
    // has tiles per SM (rounded up): blocks take items in order, so with the full grid the
    // tiles of one sweep land on a random subset of the blocks and pile up to 4 on some
    // SMs while others idle, and a sweep lasts as long as its most crowded SM.
    const long long items = (long long)a.ntiles * a.nsweeps;
    const int sms = device_sms();
    const int per_sweep = sms * std::max(1, (a.ntiles + sms - 1) / sms);
    const int nb = (int)std::min<long long>(items, std::min(per_sweep, tile_sweep_blocks(a.cfg)));
    const bool acc = a.acc != nullptr;
    if (a.trace && trig == TRIG_ACCURATE) {            // bench support: the stamped kernel
        if (acc) k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, MB, true><<<nb, NT, sm, st>>>(a);
        else k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, MB, true><<<nb, NT, sm, st>>>(a);
    } else if (trig == TRIG_FAST) {
        if (acc) k_tile_sweep<TH, TW, TRIG_FAST, true, NT, MB><<<nb, NT, sm, st>>>(a);
        else k_tile_sweep<TH, TW, TRIG_FAST, false, NT, MB><<<nb, NT, sm, st>>>(a);
    } else {
        if (acc) k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, MB><<<nb, NT, sm, st>>>(a);
        else k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, MB><<<nb, NT, sm, st>>>(a);
    }
}
#define MPR_CFG_SWEEP(id, th, tw, nt, mb) \
    case id: sweep_for<th, tw, nt, mb>(a, trig, st); break;
cudaError_t launch_tile_sweep(const TileArgs& a, int trig, cudaStream_t st) {
    if (a.ntiles == 0 || a.nsweeps <= 0) return cudaSuccess;
    // items are counted in 32 bits, with room for the blocks' claims past the end
    if ((long long)a.ntiles * a.nsweeps + 4LL * tile_sweep_blocks(a.cfg) >= (1LL << 32))
        return cudaErrorInvalidValue;
    count_launches(1, st);
    switch (a.cfg) { MPR_TILE_CONFIGS(MPR_CFG_SWEEP) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const TileDesc* tiles, int ntiles, const EntryDesc* ents, int n_ent,
                              int cfg, unsigned* hist, TileDesc* ord, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    const int maxw = 2 * tile_geom(cfg).list;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * 256 * (size_t)n_ent, st);
    if (e != cudaSuccess) return e;
    count_launches(3, st);
    k_tile_hist<<<(ntiles + 255) / 256, 256, 0, st>>>(tiles, ntiles, maxw, hist);
    k_tile_scan<<<(n_ent + 127) / 128, 128, 0, st>>>(hist, ents, n_ent);
    k_tile_scatter<<<(ntiles + 255) / 256, 256, 0, st>>>(tiles, ntiles, maxw, hist, ord);
    return cudaGetLastError();
}

cudaError_t launch_tile_sync(const TileDesc* tiles, int ntiles, Ctl* ctl, int n_ent, unsigned* tdone,
                             cudaStream_t st) {
    const int n = std::max(ntiles, n_ent);
    if (n == 0) return cudaSuccess;
    count_launches(1, st);
    k_tile_sync<<<(n + 255) / 256, 256, 0, st>>>(tiles, ntiles, ctl, n_ent, tdone);
    return cudaGetLastError();
}

cudaError_t launch_count_live(const Ctl* ctl, int n_ent, int* live, cudaStream_t st) {
    count_launches(1, st);
    k_count_live<<<1, 256, 0, st>>>(ctl, n_ent, live);
    return cudaGetLastError();
}

#define MPR_CFG_OUT(id, th, tw, nt, mb) \
    case id: k_tile_predict_out<th, tw><<<ntiles, 256, 0, st>>>( \
        tiles + tile0, cnts + tile0, lists + (long long)tile0 * g.list, acc + (long long)tile0 * g.acc, \
        ents, M, q, zmin, zmax, zr, K, chain_tiles, zhat); break;
cudaError_t launch_tile_predict_out(int cfg, const TileDesc* tiles, const TileCnt* cnts,
                                    const uint16_t* lists, const float* acc, const EntryDesc* ents,
                                    int tile0, int ntiles, int M, double q, double zmin, double zmax,
                                    const double2* zr, int K, int chain_tiles, float* zhat, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    count_launches(1, st);
    const TileGeom g = tile_geom(cfg);
    switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_OUT) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

}  // namespace mpr
