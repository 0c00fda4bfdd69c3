// mpr_tile.cu -- fused full sweep over shared-memory tiles with halos.
//
// One block owns a TH x TW tile of one grid.  It copies the tile plus a halo of two
// sites of both colour planes from the current lattice buffer into shared memory,
// updates colour A (Algorithm 1) on the tile and on a one-site ring around it, then
// colour B on the tile, and writes the tile's interior to the other lattice buffer.
// The ring updates duplicate what the neighbouring tiles compute for their own interior:
// every update is a deterministic function of its neighbours and of its Philox counter
// {site, sweep, chain, 0}, so the duplicates are bitwise identical and each tile's B
// pass sees exactly the post-A values of a whole-grid half-sweep.  Reading one buffer
// and writing the other keeps every tile's halo at the pre-sweep state.
//
// Per tile, the gap sites are listed once at set-up (u16 (r << 7) | q in the tile's
// local region coordinates): colour-A sites inside the tile, then colour-A sites on the
// ring, then colour-B sites inside the tile, contiguous in a 16-byte aligned slot that is
// copied into shared memory together with the region.  Accumulators for the equilibrium average
// use the same order (A interior, then B).
//
// The sweep's accepted energy change and acceptance count are reduced per tile; the
// last tile of a grid to finish (atomic ticket) adds the tiles' partials in tile order
// and runs the Algorithm 2 control step for that grid in place, so no separate control
// launch is needed and the sums are bitwise reproducible.
#include <algorithm>
#include <vector>

#include "mpr_internal.cuh"

namespace mpr {

namespace {


template <int TH, int TW>
struct Geo {
    static constexpr int RH = TH + 4;                 // region rows (halo 2)
    static constexpr int RW = TW / 2 + 4;             // region plane columns
    static constexpr int CAPA = ((TH + 2) * (TW + 2) + 1) / 2;
    static constexpr int CAPB = TH * TW / 2;
    static constexpr int LIST = (CAPA + CAPB + 7) / 8 * 8;   // u16 entries per tile (16-byte slots)
    static constexpr int ACC = TH * TW;               // accumulator floats per tile
    static_assert(TH % 2 == 0 && TW % 4 == 0, "tile origin parity and 16-byte alignment");
    static_assert(RW <= 128 && RH <= 512, "entry encoding");

    static_assert(RW * 8 % 16 == 0, "TMA box rows must be a multiple of 16 bytes");
    static_assert((2 * RH * RW * 8) % 128 == 0, "list slots stay 16-byte aligned");
};

// Lists the gap sites of each tile (one warp per tile), row-major in region coordinates.
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
    int counts[3] = {0, 0, 0};
    // list 0: colour A, interior; list 1: colour A, ring; list 2: colour B, interior
    for (int which = 0; which < 3; ++which) {
        const int c = which == 2 ? 1 : 0;
        int n = 0;
        uint16_t* dst = out + (which == 0 ? 0 : which == 1 ? counts[0] : counts[0] + counts[1]);
        for (int base = 0; base < G::RH * G::RW; base += 32) {
            const int idx = base + lane;
            bool take = false;
            int r = 0, q = 0;
            if (idx < G::RH * G::RW) {
                r = idx / G::RW;
                q = idx - r * G::RW;
                const int y = td.y0 - 2 + r;
                const int s = c ^ (r & 1);
                const int x = td.x0 + 2 * q - 4 + s;
                const bool in_grid = y >= 0 && y < E.H && x >= 0 && x < E.W;
                const bool interior = y >= td.y0 && y < td.y0 + TH && x >= td.x0 && x < td.x0 + TW;
                const bool ring = !interior && y >= td.y0 - 1 && y <= td.y0 + TH && x >= td.x0 - 1 &&
                                  x <= td.x0 + TW;
                const bool gap = in_grid && (all_free || !m[(long long)y * E.W + x]);
                take = gap && (which == 1 ? ring : interior);
            }
            const unsigned b = __ballot_sync(0xffffffffu, take);
            if (take) dst[n + __popc(b & lt)] = (uint16_t)((r << 7) | q);
            n += __popc(b);
        }
        counts[which] = n;
    }
    if (lane == 0) {
        TileCnt c;
        c.nA_int = (uint16_t)counts[0];
        c.nA_ring = (uint16_t)counts[1];
        c.nB = (uint16_t)counts[2];
        c._pad = 0;
        cnts[t] = c;
        tiles[t].nA_int = counts[0];
        tiles[t].nA_ring = counts[1];
        tiles[t].nB = counts[2];
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

// Per-tile parameters staged in shared memory by the issuing thread, in 16-byte groups
// so that each thread picks up what it needs with a few vector loads.
struct __align__(16) TileParams {
    int t, y0, x0, W;                     // tile, origin, grid width
    uint32_t chain, sweep;                // Philox counter words 2 and 1
    float half_qd, neg_inv_T;             // proposal half-angle scale, -1/T
    int nA_int, nA_ring, nB, e;           // list counts, grid
    int ntiles, H, pitch, cur;            // grid's tile count and height, row pitch, source buffer
    long long pl0, pl1;                   // plane offsets of the grid in the lattice buffers
};

// Energy changes are summed across the tiles of a grid in 64-bit fixed point (2^-28 units):
// integer addition is associative, so the total does not depend on which block updated
// which tile or in which order.  |dH| <= 8 per site keeps any grid of < 2^31 sites far
// from overflow.
constexpr float kFixScale = 268435456.0f;             // 2^28
constexpr double kFixUnit = 1.0 / 268435456.0;

// Thread 0 of a block, after a barrier that follows every warp's flush for grid e: n more
// tiles of e are done (release/acquire through the fences around the ticket).  The block
// completing e's tiles runs e's control step from the fixed-point totals and clears them.
__device__ __forceinline__ void tile_ticket(const TileArgs& A, int e, int n) {
    __threadfence();
    const unsigned prev = atomicAdd(A.ticket + e, (unsigned)n);
    if (prev + (unsigned)n == (unsigned)A.ents[e].ntiles) {
        __threadfence();
        const long long f = (long long)atomicExch(A.gsum + 2 * e, 0ull);
        const unsigned long long nacc_e = atomicExch(A.gsum + 2 * e + 1, 0ull);
        Ctl c = A.ctl[e];
        control_step(c, A.ents[e], (double)f * kFixUnit, nacc_e, A.mode, A.A_targ, A.k_a, A.n_f,
                     A.n_fit, A.i_max, A.ehist + (long long)e * A.ehist_stride, 1);
        A.ctl[e] = c;
        A.ticket[e] = 0u;
        if (A.active && !c.stop) atomicAdd(A.active, 1);
    }
}

// Persistent fused sweep.  Blocks take tiles from a global counter (the last block to
// leave resets it for the next launch), so faster blocks take more tiles and no block
// idles while others finish.  Thread 0 stages a tile: a TMA box of both colour planes
// plus the bulk-copied gap list, completing on the stage's mbarrier.  With two stages the
// next tile is staged as soon as the current one is in shared memory, a whole tile
// ahead; with one stage, after the previous tile has been written back.
// Each thread keeps its energy change (fixed point) and acceptance count summed over the
// block's tiles of one grid; when the block moves on to another grid or runs out of
// tiles, the warps add them to the grid's totals and thread 0 adds the block's tile count
// to the grid's ticket.  The block that completes a grid's tiles runs the grid's
// Algorithm 2 control step from the totals.
// The interior rows of both planes go back to the other lattice buffer as 16-byte
// stores, which frees the stage at once.
template <int TH, int TW, int TRIG, bool ACC, int NT, int STAGES, int MB>
__global__ void __launch_bounds__(NT, MB)
k_tile_sweep(const TileArgs A) {
    static_assert(STAGES == 1 || STAGES == 2, "one or two stages");
    static_assert(TW % 8 == 0, "write-back in 16-byte vectors");
    using G = Geo<TH, TW>;
    extern __shared__ __align__(128) unsigned char dsm[];
    float2(*stage)[2][G::RH][G::RW] = reinterpret_cast<float2(*)[2][G::RH][G::RW]>(dsm);
    uint16_t(*slist)[G::LIST] =
        reinterpret_cast<uint16_t(*)[G::LIST]>(dsm + STAGES * 2 * G::RH * G::RW * sizeof(float2));
    __shared__ TileParams sp[STAGES];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ int s_fail;
    __shared__ TileParams cp_;                                 // thread 0's grid cache
    __shared__ const CUtensorMap* cmap;
    __shared__ int cstop;
    constexpr uint32_t kBytes = 2u * G::RH * G::RW * sizeof(float2);
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) mbar_init(&bar[i], 1);
        fence_barrier_init();
        s_fail = 0;
    }
    __syncthreads();

    // Thread 0 only: tile indices come from the counter two tiles ahead and descriptors
    // one tile ahead (an asynchronous copy into shared memory), so that staging a tile
    // never waits on the counter or on a global load; the parameters of the grid being
    // staged are reloaded only when the grid changes (tiles are taken in increasing
    // order and a grid's tiles are contiguous; they are constant during a launch).
    int ce = -1, i0 = A.ntiles, i1 = A.ntiles;
    __shared__ __align__(16) TileDesc dnext;
    auto fetch_desc = [&](int i) {
        const TileDesc* src = A.tiles + i;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(&dnext)), "l"(src) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(&dnext) + 16u),
                     "l"(reinterpret_cast<const char*>(src) + 16) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (threadIdx.x == 0) {
        i0 = (int)atomicAdd(A.sched, 1u);
        i1 = (int)atomicAdd(A.sched, 1u);
        if (i0 < A.ntiles) fetch_desc(i0);
    }
    auto load_entry = [&](int e) {
        const EntryDesc& E = A.ents[e];
        const Ctl& c = A.ctl[e];
        cp_.W = E.W;
        cp_.H = E.H;
        cp_.chain = E.chain;
        cp_.sweep = c.sweep;
        cp_.half_qd = A.use_ctl_a ? c.half_qd : A.half_qd_fixed;
        cp_.neg_inv_T = c.neg_inv_T;
        cp_.e = e;
        cp_.ntiles = E.ntiles;
        cp_.pl0 = E.plane[0];
        cp_.pl1 = E.plane[1];
        cp_.pitch = E.pitch;
        cp_.cur = c.cur;
        cstop = A.skip_stopped ? c.stop : 0;
        cmap = A.maps + 2 * e + c.cur;
        ce = e;
    };
    // stages the next tile whose grid is still relaxing into stage st, or marks the stage
    // empty (t = ntiles) when the counter is exhausted
    auto issue = [&](int st) {
        TileParams& P = sp[st];
        for (;;) {
            if (i0 >= A.ntiles) { P.t = A.ntiles; return; }
            asm volatile("cp.async.wait_all;" ::: "memory");          // the descriptor of i0
            const TileDesc d = dnext;
            const int cur_t = i0;
            i0 = i1;                                                  // taken a tile ago
            if (i0 < A.ntiles) fetch_desc(i0);
            i1 = (int)atomicAdd(A.sched, 1u);                         // needed two tiles from now
            if (d.entry != ce) load_entry(d.entry);
            if (!cstop) {
                cp_.t = cur_t;
                cp_.y0 = d.y0;
                cp_.x0 = d.x0;
                cp_.nA_int = d.nA_int;
                cp_.nA_ring = d.nA_ring;
                cp_.nB = d.nB;
                P = cp_;
                const uint32_t lbytes = ((uint32_t)(d.nA_int + d.nA_ring + d.nB) * 2u + 15u) & ~15u;
                mbar_expect_tx(&bar[st], kBytes + lbytes);
                tma_load_3d(&stage[st][0][0][0], cmap, &bar[st], d.x0 >> 1, d.y0 - 1, 0);
                if (lbytes)
                    bulk_load(&slist[st][0], A.lists + (long long)cur_t * G::LIST, lbytes, &bar[st]);
                return;
            }
        }
    };

    // each thread's totals over the block's tiles of grid s_acc_e (kept in shared memory)
    __shared__ long long s_fx[NT];
    __shared__ unsigned s_nat[NT];
    __shared__ int s_acc_e, ntile_e, pend_e, pend_n;         // thread 0 writes; ticket bookkeeping
    s_fx[threadIdx.x] = 0;
    s_nat[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        s_acc_e = -1;
        ntile_e = 0;
        pend_e = -1;
        pend_n = 0;
    }
    __syncthreads();
    auto flush_partials = [&](int e) {
        long long w = s_fx[threadIdx.x];
        unsigned long long wn = s_nat[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, o);
            wn += __shfl_xor_sync(0xffffffffu, wn, o);
        }
        if (lane == 0) {
            if (w) atomicAdd(A.gsum + 2 * e, (unsigned long long)w);
            if (wn) atomicAdd(A.gsum + 2 * e + 1, wn);
        }
        s_fx[threadIdx.x] = 0;
        s_nat[threadIdx.x] = 0u;
    };
    // thread 0, after a barrier that follows every warp's flush for grid e: n more tiles of
    // e are done; the block completing e's tiles runs e's control step
    auto take_ticket = [&](int e, int n) { tile_ticket(A, e, n); };

    if (threadIdx.x == 0) issue(0);
    for (int it = 0;; ++it) {
        const int st = STAGES == 1 ? 0 : (it & 1);
        const uint32_t parity = (uint32_t)(STAGES == 1 ? it : (it >> 1)) & 1u;
        if (STAGES == 1 && it > 0) {
            __syncthreads();                                      // B0: the write-back has read the stage
            if (threadIdx.x == 0) issue(0);
        }
        // the previous grid's ticket (its flushes were ordered by the last B2/B3), while the
        // copy is in flight
        if (threadIdx.x == 0 && pend_e >= 0) {
            take_ticket(pend_e, pend_n);
            pend_e = -1;
        }
        if (threadIdx.x == 0 && sp[st].t < A.ntiles && !mbar_wait_try(&bar[st], parity)) {
            atomicExch(A.err, 1);
            s_fail = 1;
        }
        __syncthreads();                                          // B1: the tile is in stage st
        const int4 g0 = *reinterpret_cast<const int4*>(&sp[st].t);
        const int t = g0.x;
        if (t >= A.ntiles) break;
        if (s_fail) {
            // give the late copy a second bounded wait to land before the block's shared
            // memory goes away (no other copy is in flight at B1), then leave
            if (threadIdx.x == 0) (void)mbar_wait_try(&bar[st], parity);
            break;
        }
        (void)mbar_test(&bar[st], parity);                        // each thread acquires the copy
        // stage st ^ 1 was written back before B1: stage the next tile into it now
        if (STAGES == 2 && threadIdx.x == 0) issue(st ^ 1);
        const int y0 = g0.y, x0 = g0.z, W = g0.w;
        const int4 g1 = *reinterpret_cast<const int4*>(&sp[st].chain);
        const int4 g2 = *reinterpret_cast<const int4*>(&sp[st].nA_int);
        const uint32_t chain = (uint32_t)g1.x, sweep = (uint32_t)g1.y;
        const float half_qd = __int_as_float(g1.z), kx = accept_scale<TRIG>(__int_as_float(g1.w));
        const int nA_int = g2.x, nA = g2.x + g2.y, nB = g2.z, e = g2.w;
        float2(*sm)[G::RH][G::RW] = stage[st];
        const uint16_t* list = slist[st];
        float* __restrict__ acc = ACC ? A.acc + (long long)t * G::ACC : nullptr;
        {
            const int acc_e = s_acc_e;                        // rewritten only after B2
            if (e != acc_e) {                                 // the block moves on to grid e
                if (acc_e >= 0) flush_partials(acc_e);
                if (threadIdx.x == 0) {
                    pend_e = acc_e;
                    pend_n = ntile_e;
                    ntile_e = 0;
                }
            }
        }

        // colour A on the tile and its ring, then colour B on the tile
        float dE = 0.0f;
        unsigned nacc = 0;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int c = pass;                           // colour being updated
            const int n = pass ? nB : nA;
            const uint16_t* lst = pass ? list + nA : list;
            float2(*own)[G::RW] = sm[c];
            float2(*oth)[G::RW] = sm[c ^ 1];
            for (int k = threadIdx.x; k < n; k += NT) {
                // the ring belongs to other tiles: its sites count nowhere
                const bool own_site = pass || k < nA_int;
                const int aidx = pass ? nA_int + k : k;
                // the running angle sum is loaded first, so that its latency hides behind
                // the update
                float acc_old = 0.0f;
                if (ACC && own_site) acc_old = acc[aidx];
                const int ent = lst[k];
                const int r = ent >> 7, q = ent & 127;
                const int s = c ^ (r & 1);
                const float2 nu = oth[r - 1][q], nd = oth[r + 1][q];
                const float2 nl = oth[r][q - 1 + s], nr = oth[r][q + s];
                const float C = (nu.x + nd.x) + (nl.x + nr.x);
                const float S = (nu.y + nd.y) + (nl.y + nr.y);
                float2 v = own[r][q];
                const int y = y0 - 2 + r, x = x0 + 2 * q - 4 + s;
                const uint32_t site = (uint32_t)y * (uint32_t)W + (uint32_t)x;
                const uint4 rnd = philox10(make_uint4(site, sweep, chain, 0u), A.rk);
                const float hq = (u24f(rnd.x) - 0.5f) * half_qd;
                bool accepted;
                float Fx = 0.0f, Fy = 0.0f;
                if (A.or_mode == OR_LITERAL) literal_field(nu, nd, nl, nr, Fx, Fy);
                const float d = hybrid_update<TRIG>(v, C, S, Fx, Fy, hq, u24f(rnd.y), kx, A.or_mode, accepted);
                own[r][q] = v;
                if (own_site) {
                    dE += d;
                    nacc += accepted ? 1u : 0u;
                    if (ACC) acc[aidx] = acc_old + angle_upper(v.x, v.y);
                }
            }
            if (pass == 0) {
                __syncthreads();                          // B2: colour A done (and any flush)
                if (threadIdx.x == 0) s_acc_e = e;
            }
        }
        // the tile's energy change in fixed point: deterministic whatever the tile order
        s_fx[threadIdx.x] += __float2ll_rn(dE * kFixScale);
        s_nat[threadIdx.x] += nacc;
        if (threadIdx.x == 0) ++ntile_e;
        fence_proxy_async_smem();                     // this thread's stage writes before the next copy into it
        __syncthreads();                              // B3: colour B done
        const int4 g3 = *reinterpret_cast<const int4*>(&sp[st].ntiles);
        // interior rows of both colours to the other buffer (samples included), 16 bytes
        // per thread and step, one warp per row; rows and columns beyond the grid skipped
        {
            const int rows = min(TH, g3.y - y0);
            const int pc = (x0 >> 1) + 2;
            const int nv = (min(TW / 2, g3.z - pc) & ~1) >> 1;        // 16-byte vectors per row
            const long long pl0 = sp[st].pl0, pl1 = sp[st].pl1;
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
    }
    // leave: hand in the last grid's totals and tiles, then the last block out resets the
    // tile counter for the next launch (every block has stopped taking tiles by the time
    // it counts itself out)
    const int acc_e = s_acc_e;
    if (acc_e >= 0) flush_partials(acc_e);
    __syncthreads();
    if (threadIdx.x == 0 && acc_e >= 0) take_ticket(acc_e, ntile_e);
    if (threadIdx.x == 0) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __threadfence();
        if (atomicAdd(A.sched + 1, 1u) == gridDim.x - 1u) {
            atomicExch(A.sched, 0u);
            atomicExch(A.sched + 1, 0u);
        }
    }
}

// zhat at the gap sites of every tile (same mean and inverse map as the list path).  With
// K > 1 the angle sums of K chains of the same grid are added: chain c's copy of tile t is
// tile t + c * chain_tiles (every chain has the same tiles and lists).
template <int TH, int TW>
__global__ void k_tile_predict_out(const TileDesc* __restrict__ tiles, const TileCnt* __restrict__ cnts,
                                   const uint16_t* __restrict__ lists, const float* __restrict__ acc,
                                   const EntryDesc* __restrict__ ents, int M, double q, double zmin,
                                   double zmax, int K, int chain_tiles, float* __restrict__ zhat) {
    using G = Geo<TH, TW>;
    const int tile = blockIdx.x;
    const TileDesc td = tiles[tile];
    const EntryDesc E = ents[td.entry];
    const TileCnt cnt = cnts[tile];
    const uint16_t* list = lists + (long long)tile * G::LIST;
    const float* a = acc + (long long)tile * G::ACC;
    const long long cstride = (long long)chain_tiles * G::ACC;
    const int nA = cnt.nA_int + cnt.nA_ring;
    const double f = (zmax - zmin) / (kTwoPi * q * (double)M * (double)K);
    for (int k = threadIdx.x; k < cnt.nA_int + cnt.nB; k += blockDim.x) {
        const bool isA = k < cnt.nA_int;
        const int ent = isA ? list[k] : list[nA + (k - cnt.nA_int)];
        const int r = ent >> 7, qq = ent & 127;
        const int s = (isA ? 0 : 1) ^ (r & 1);
        const int y = td.y0 - 2 + r, x = td.x0 + 2 * qq - 4 + s;
        double sum = (double)a[k];
        for (int c = 1; c < K; ++c) sum += (double)a[c * cstride + k];
        double v = zmin + sum * f;
        v = v < zmin ? zmin : (v > zmax ? zmax : v);
        zhat[E.site0 + (long long)y * E.W + x] = (float)v;
    }
}

}  // namespace

// Heaviest tiles first.  The persistent blocks take tiles in index order, so with each
// grid's tiles sorted by descending gap count the last tiles handed out are the lightest
// and the blocks finish close together (cloud-like gaps make some tiles several times
// heavier than others).  Stable, so equal tiles keep raster order; per grid, so a grid's
// tiles stay contiguous.  Every update depends only on its neighbours and its counter, so
// the order changes no result.
void order_tiles_by_work(TileDesc* tiles, const EntryDesc* ents, int n_ent) {
    for (int e = 0; e < n_ent; ++e) {
        TileDesc* t0 = tiles + ents[e].tile0;
        std::stable_sort(t0, t0 + ents[e].ntiles, [](const TileDesc& a, const TileDesc& b) {
            return a.nA_int + a.nA_ring + a.nB > b.nA_int + b.nA_ring + b.nB;
        });
    }
}

// ---------------------------------------------------------------- compiled configurations
// The tile shapes the library is built with; the autotuner picks one per batch.
//   id  TH  TW  threads  stages  blocks/SM register budget
//    0  16 128     128       1    8
//    1  32  64     128       1    8
//    2  32 128     256       1    4
#define MPR_TILE_CONFIGS(X) \
    X(0, 16, 128, 128, 1, 8)  \
    X(1, 32, 64, 128, 1, 8)   \
    X(2, 32, 128, 256, 1, 4)

template <int TH, int TW, int NT, int ST>
struct Cfg {
    using G = Geo<TH, TW>;
    static constexpr int SMEM = ST * 2 * G::RH * G::RW * 8 + ST * G::LIST * 2;
};

#define MPR_CFG_GEOM(id, th, tw, nt, st, mb) \
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
template <int TH, int TW, int NT, int ST, int MB>
int blocks_for() {
    constexpr int sm = Cfg<TH, TW, NT, ST>::SMEM;
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, ST, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, ST, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_FAST, true, NT, ST, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_tile_sweep<TH, TW, TRIG_FAST, false, NT, ST, MB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per, k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, ST, MB>, NT, sm);
    return std::max(1, sms * std::max(1, per));
}

#define MPR_CFG_BLOCKS(id, th, tw, nt, st, mb) \
    case id: blocks[id] = blocks_for<th, tw, nt, st, mb>(); break;
int tile_sweep_blocks(int cfg) {
    static int blocks[8] = {0};
    if (cfg < 0 || cfg >= tile_config_count()) return 0;
    if (!blocks[cfg]) {
        switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_BLOCKS) default: break; }
    }
    return blocks[cfg];
}

#define MPR_CFG_LISTS(id, th, tw, nt, st, mb) \
    case id: k_tile_lists<th, tw><<<(ntiles * 32 + 127) / 128, 128, 0, st_>>>(tiles, ntiles, ents, mask, all_free, lists, cnts); break;
cudaError_t launch_tile_lists(int cfg, TileDesc* tiles, int ntiles, const EntryDesc* ents,
                              const uint8_t* mask, int all_free, uint16_t* lists, TileCnt* cnts,
                              cudaStream_t st_) {
    if (ntiles == 0) return cudaSuccess;
    count_launches(1, st_);
    switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_LISTS) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

template <int TH, int TW, int NT, int ST, int MB>
void sweep_for(const TileArgs& a, int trig, cudaStream_t st) {
    constexpr int sm = Cfg<TH, TW, NT, ST>::SMEM;
    const int nb = std::min(a.ntiles, tile_sweep_blocks(a.cfg));
    const bool acc = a.acc != nullptr;
    if (trig == TRIG_FAST) {
        if (acc) k_tile_sweep<TH, TW, TRIG_FAST, true, NT, ST, MB><<<nb, NT, sm, st>>>(a);
        else k_tile_sweep<TH, TW, TRIG_FAST, false, NT, ST, MB><<<nb, NT, sm, st>>>(a);
    } else {
        if (acc) k_tile_sweep<TH, TW, TRIG_ACCURATE, true, NT, ST, MB><<<nb, NT, sm, st>>>(a);
        else k_tile_sweep<TH, TW, TRIG_ACCURATE, false, NT, ST, MB><<<nb, NT, sm, st>>>(a);
    }
}
#define MPR_CFG_SWEEP(id, th, tw, nt, st_, mb) \
    case id: sweep_for<th, tw, nt, st_, mb>(a, trig, st); break;
cudaError_t launch_tile_sweep(const TileArgs& a, int trig, cudaStream_t st) {
    if (a.ntiles == 0) return cudaSuccess;
    count_launches(1, st);
    switch (a.cfg) { MPR_TILE_CONFIGS(MPR_CFG_SWEEP) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

#define MPR_CFG_OUT(id, th, tw, nt, st_, mb) \
    case id: k_tile_predict_out<th, tw><<<ntiles, 256, 0, st>>>( \
        tiles + tile0, cnts + tile0, lists + (long long)tile0 * g.list, acc + (long long)tile0 * g.acc, \
        ents, M, q, zmin, zmax, K, chain_tiles, zhat); break;
cudaError_t launch_tile_predict_out(int cfg, const TileDesc* tiles, const TileCnt* cnts,
                                    const uint16_t* lists, const float* acc, const EntryDesc* ents,
                                    int tile0, int ntiles, int M, double q, double zmin, double zmax,
                                    int K, int chain_tiles, float* zhat, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    count_launches(1, st);
    const TileGeom g = tile_geom(cfg);
    switch (cfg) { MPR_TILE_CONFIGS(MPR_CFG_OUT) default: return cudaErrorInvalidValue; }
    return cudaGetLastError();
}

}  // namespace mpr
