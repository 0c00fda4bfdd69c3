// mpr_net_tc.cu -- 3x3 convolutions of the warm-start network on the 5th-generation tensor
// cores: implicit GEMM with tcgen05.mma (bf16 x bf16 -> fp32 in tensor memory), operands
// brought in by TMA.
//
// GEMM view: M = output pixels in spatial tiles of 8 rows x 16 columns (128 rows of A),
// N = output channels (tile BN), K = 9 taps x Kt channels (Kt = C rounded up to 64).  One
// pipeline stage is one 64-wide K chunk (tap, channel block): A is a 4-D TMA box
// {64 channels, 16 x, 8 y, 1 image} of the NHWC input at the tap's offset -- pixels outside
// the image and channels beyond C arrive as zeros, which is the convolution's zero padding
// -- and B is a {64, BN} box of the K-major weights.  Both land in the canonical K-major
// layout with the 128-byte swizzle (rows of 128 B, 8-row groups 1024 B apart).
//
// Warp roles of a persistent CTA (one per SM):
//   warps 0-3  epilogue: tcgen05.ld of the accumulator rows (TMEM lanes 0-127), bias, ReLU,
//              bf16 stores (optionally also into a channel slice of a concatenation buffer,
//              nearest-upsampled 2x) or fp32 stores;
//   warp 4     lane 0 issues the TMA loads of each stage on its "full" barrier;
//   warp 5     allocates tensor memory; lane 0 issues the MMAs (4 x K=16 per stage),
//              releases stages with tcgen05.commit and signals finished accumulators.
// The accumulator is double-buffered in tensor memory, so the epilogue of one tile runs
// while the next tile accumulates.  Every barrier wait is bounded: on expiry the kernel
// records an error, stops issuing work, lets its tensor-core work drain and releases its
// tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpr_net_kernels.cuh"

namespace mprnet {
namespace {

constexpr int kEpiWarps = 4;
constexpr int kProdWarp = 4, kMmaWarp = 5;
constexpr int kThreads = 6 * 32;
constexpr int kBM = 128, kTY = 8, kTX = 16;   // M tile: 8 rows x 16 columns of pixels
constexpr long long kSpin = 1LL << 24;        // bounded barrier polls (each with a short sleep)

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false (and the error flag set) on expiry.
// The first polls spin on try_wait (which itself suspends the thread in hardware for a
// while); only a wait that lasts longer backs off with a sleep between polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, volatile int* abort_flag) {
    for (long long i = 0; i < kSpin; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
        if (i >= 1024) __nanosleep(64);
    }
    atomicExch(err, 1);
    *abort_flag = 1;
    return false;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// ---- tcgen05 -----------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B
// apart (stride byte offset), leading byte offset unused for this layout (1), descriptor
// version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// The same for the 64-byte swizzle (rows of 64 B, 8-row groups 512 B apart; mode 4 = 64 B).
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// Instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B bf16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct Tc {
    static constexpr int A_BYTES = kBM * 128;
    static constexpr int B_BYTES = BN * 128;
    static constexpr int STAGE = A_BYTES + B_BYTES;                  // multiple of 1024
    static constexpr int STAGES = (200 * 1024 / STAGE) > 8 ? 8 : (200 * 1024 / STAGE);
    static constexpr int ACC_STRIDE = BN == 96 ? 128 : BN;           // TMEM columns per buffer
    static constexpr int TMEM_COLS = 2 * ACC_STRIDE;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int SMEM = BAR_OFF + 256 + 1024;                // + barriers + alignment slack
};

// Halo variant (small N): M tile 16 rows x 8 columns, 32-channel blocks with the 64-byte
// swizzle.  Per channel block three TMA boxes {32, 8, 18, 1} (the tile's rows -1..16 at
// column offsets dx - 1 = -1, 0, 1) serve all nine taps: tap (dy, dx) is copy dx shifted by
// dy rows of 8 pixels = dy * 512 bytes, again an aligned canonical operand.  The layer's
// weights (K = 9 x C, unpadded) stay resident in shared memory.
constexpr int kHY = 16, kHX = 8;
constexpr int kHaloRows = (kHY + 2) * kHX;                 // 144 rows of 64 B per copy
constexpr int kHaloCopy = kHaloRows * 64;                  // 9216 B = 9 x 1024
constexpr int kHaloStage = 3 * kHaloCopy;
constexpr int kHaloStages = 5;
constexpr int kHaloBmax = 80 * 1024;                       // resident weights at most
// RES: the layer's weights resident (at most kHaloBmax); otherwise each stage also carries
// the block's weights for the nine taps (9 x BN rows of 64 B).
template <int BN, bool RES>
struct Th {
    static constexpr int ACC_STRIDE = BN;
    static constexpr int TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;
    static constexpr int B_STAGE = RES ? 0 : 9 * BN * 64;
    static constexpr int STAGE = kHaloStage + B_STAGE;                 // multiple of 1024
    static constexpr int STAGES = RES ? kHaloStages : (196 * 1024) / STAGE;
    static constexpr int A_OFF = RES ? kHaloBmax : 0;
    static constexpr int BAR_OFF = A_OFF + STAGES * STAGE;
    static constexpr int SMEM = BAR_OFF + 256 + 1024;
};

// Epilogue of one 16-column slice of an accumulator row (one pixel per thread): bias, ReLU,
// bf16 stores (primary, concatenation buffer, optional fused 2 x 2 average pooling) or fp32
// stores.  TX: tile width in pixels, so the pixel below is lane ^ TX.  All lanes call it.
template <int TX>
__device__ __forceinline__ void epi16(const TcConv& c, const float* v, int n, int b, int y, int x, bool valid,
                                      long long p) {
    if (c.out) {
        uint32_t pk[8];
        float r[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float x0 = v[2 * i], x1 = v[2 * i + 1];
            if (c.bias) { x0 += c.bias[n + 2 * i]; x1 += c.bias[n + 2 * i + 1]; }
            if (c.relu) { x0 = fmaxf(x0, 0.f); x1 = fmaxf(x1, 0.f); }
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            pk[i] = *reinterpret_cast<const uint32_t*>(&h);
            r[2 * i] = __low2float(h);
            r[2 * i + 1] = __high2float(h);
        }
        if (c.pool) {                       // ((a + b) + c) + d over the 2 x 2 block, then / 4
            uint32_t pp[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float o[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float a = r[2 * i + h];
                    const float bb = __shfl_xor_sync(0xffffffffu, a, 1);
                    const float cc = __shfl_xor_sync(0xffffffffu, a, TX);
                    const float dd = __shfl_xor_sync(0xffffffffu, a, TX ^ 1);
                    o[h] = 0.25f * (((a + bb) + cc) + dd);
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(o[0], o[1]);
                pp[i] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            if (valid && !(y & 1) && !(x & 1)) {
                const long long q = ((long long)b * (c.H >> 1) + (y >> 1)) * (c.W >> 1) + (x >> 1);
                uint4* d = reinterpret_cast<uint4*>(c.pool + q * c.N + n);
                d[0] = make_uint4(pp[0], pp[1], pp[2], pp[3]);
                d[1] = make_uint4(pp[4], pp[5], pp[6], pp[7]);
            }
        }
        if (!valid) return;
        const uint4 lo = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        const uint4 hi = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        uint4* dst = reinterpret_cast<uint4*>(c.out + p * c.N + n);
        dst[0] = lo;
        dst[1] = hi;
        if (c.out2) {
            if (c.up2) {
#pragma unroll
                for (int sy = 0; sy < 2; ++sy)
#pragma unroll
                    for (int sx = 0; sx < 2; ++sx) {
                        const long long p2 = ((long long)b * 2 * c.H + 2 * y + sy) * (2LL * c.W) + 2 * x + sx;
                        uint4* d2 = reinterpret_cast<uint4*>(c.out2 + p2 * c.ld2 + c.off2 + n);
                        d2[0] = lo;
                        d2[1] = hi;
                    }
            } else {
                uint4* d2 = reinterpret_cast<uint4*>(c.out2 + p * c.ld2 + c.off2 + n);
                d2[0] = lo;
                d2[1] = hi;
            }
        }
    } else {
        if (!valid) return;
        const ConvOutF32& o = c.of;
        float* dst = n < o.C0 ? o.dst0 + p * o.C0 + n : o.dst1 + p * o.C1 + (n - o.C0);
        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float4 w = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            if (o.accumulate) {
                const float4 qv = d4[i];
                w.x += qv.x; w.y += qv.y; w.z += qv.z; w.w += qv.w;
            }
            d4[i] = w;
        }
    }
}

// Common set-up: barriers, tensor memory; returns the TMEM base.
struct Bars {
    uint32_t base;
    int stages;
    __device__ uint32_t full(int s) const { return base + 8u * s; }
    __device__ uint32_t empty(int s) const { return base + 8u * (stages + s); }
    __device__ uint32_t accf(int b) const { return base + 8u * (2 * stages + b); }
    __device__ uint32_t acce(int b) const { return base + 8u * (2 * stages + 2 + b); }
    __device__ uint32_t done() const { return base + 8u * (2 * stages + 4); }
    __device__ uint32_t bres() const { return base + 8u * (2 * stages + 5); }
    __device__ uint32_t* slot(uint8_t* smem_bar) const { return (uint32_t*)(smem_bar + 8 * (2 * stages + 6)); }
};

__device__ __forceinline__ void setup(const Bars& B, const CUtensorMap* ma, const CUtensorMap* mb, uint32_t* slot,
                                      volatile int* abort_flag, int tmem_cols) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < B.stages; ++s) {
            mbar_init(B.full(s), 1);
            mbar_init(B.empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(B.accf(b), 1);
            mbar_init(B.acce(b), kEpiWarps * 32);
        }
        mbar_init(B.done(), 1);
        mbar_init(B.bres(), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)ma) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)mb) : "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void teardown(uint32_t tmem, int tmem_cols) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
    }
}

// MMA-issuing lane: drains every MMA it issued before the CTA releases tensor memory.
__device__ __forceinline__ void drain(const Bars& B) {
    tc_commit(B.done());
    for (long long i = 0; i < kSpin && !mbar_test(B.done(), 0); ++i) __nanosleep(32);
}

// Epilogue warps: for each finished accumulator, TX-wide tiles of TY rows.
template <int BN, int TY, int TX, int ACC>
__device__ __forceinline__ void epilogue(const TcConv& c, const Bars& B, uint32_t tmem, long long ntiles, int NT,
                                         int TYn, int TXn, int* err, volatile int* abort_flag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = warp * 32 + lane;                      // TMEM lane = accumulator row
    long long tc = 0;
    for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tc) {
        const int buf = (int)(tc & 1);
        if (!mbar_wait(B.accf(buf), (uint32_t)(tc >> 1) & 1u, err, abort_flag)) break;
        tc_fence_after();
        long long q = t;
        const int n0 = (int)(q % NT) * BN; q /= NT;
        const int x = (int)(q % TXn) * TX + (row % TX); q /= TXn;
        const int y = (int)(q % TYn) * TY + row / TX;
        const int b = (int)(q / TYn);
        const bool valid = y < c.H && x < c.W;
        const long long p = ((long long)b * c.H + y) * c.W + x;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + buf * ACC;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc_ld16(taddr + c0, v);
            epi16<TX>(c, v, n0 + c0, b, y, x, valid, p);
        }
        tc_fence_before();
        mbar_arrive(B.acce(buf));
    }
}

// Tensor-core implicit-GEMM convolution, general tile (maps: A = input NHWC {C, W, H, B},
// box {64, 16, 8, 1}; B = K-major weights {Kpad, N}, box {64, BN}; both 128-byte swizzled).
template <int BN>
__global__ void __launch_bounds__(kThreads, 1) k_conv_tma(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB,
                                                          const TcConv c, int* __restrict__ err) {
    using C = Tc<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = saddr(smem);
    const Bars B{sbase + C::BAR_OFF, C::STAGES};
    uint32_t* tmem_slot = B.slot(smem + C::BAR_OFF);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int TYn = (c.H + kTY - 1) / kTY, TXn = (c.W + kTX - 1) / kTX;
    const int NT = c.N / BN;
    const long long ntiles = (long long)c.B * TYn * TXn * NT;
    const int KB = (c.C + 63) / 64;                  // 64-channel blocks per tap
    const int KC = 9 * KB;

    setup(B, &mapA, &mapB, tmem_slot, abort_flag, C::TMEM_COLS);
    const uint32_t tmem = *tmem_slot;

    if (warp == kProdWarp) {
        if (lane == 0) {                                   // TMA producer
            long long it = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                long long q = t;
                const int n0 = (int)(q % NT) * BN; q /= NT;
                const int x0 = (int)(q % TXn) * kTX; q /= TXn;
                const int y0 = (int)(q % TYn) * kTY;
                const int b = (int)(q / TYn);
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc, ++it) {
                    const int s = (int)(it % C::STAGES);
                    if (it >= C::STAGES &&
                        !mbar_wait(B.empty(s), (uint32_t)((it / C::STAGES) - 1) & 1u, err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int tap = kc / KB, cb = kc - tap * KB;
                    const int dy = tap / 3 - 1, dx = tap - (tap / 3) * 3 - 1;
                    const uint32_t sa = sbase + s * C::STAGE;
                    mbar_expect_tx(B.full(s), C::STAGE);
                    tma_load_4d(sa, &mapA, B.full(s), cb * 64, x0 + dx, y0 + dy, b);
                    tma_load_2d(sa + C::A_BYTES, &mapB, B.full(s), kc * 64, n0);
                }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {                                   // MMA issue
            constexpr uint32_t idesc = idesc_bf16(kBM, BN);
            long long it = 0, tc = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tc) {
                const int buf = (int)(tc & 1);
                if (tc >= 2 && !mbar_wait(B.acce(buf), (uint32_t)((tc >> 1) - 1) & 1u, err, abort_flag)) break;
                tc_fence_after();
                const uint32_t d = tmem + buf * C::ACC_STRIDE;
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc, ++it) {
                    const int s = (int)(it % C::STAGES);
                    if (!mbar_wait(B.full(s), (uint32_t)(it / C::STAGES) & 1u, err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + s * C::STAGE, sb = sa + C::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma(d, sdesc(sa + kk * 32), sdesc(sb + kk * 32), idesc, (kc | kk) != 0);
                    tc_commit(B.empty(s));
                }
                if (!ok) break;
                tc_commit(B.accf(buf));
            }
            drain(B);
        }
        __syncwarp();
    } else {
        epilogue<BN, kTY, kTX, C::ACC_STRIDE>(c, B, tmem, ntiles, NT, TYn, TXn, err, abort_flag);
    }
    teardown(tmem, C::TMEM_COLS);
}

// Halo-tile convolution for N = BN in {32, 64} (maps: A box {32, 8, 18, 1}; B box {32, BN}).
template <int BN, bool RES>
__global__ void __launch_bounds__(kThreads, 1) k_conv_halo(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           const TcConv c, int* __restrict__ err) {
    using C = Th<BN, RES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = saddr(smem);
    const Bars B{sbase + C::BAR_OFF, C::STAGES};
    uint32_t* tmem_slot = B.slot(smem + C::BAR_OFF);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int TYn = (c.H + kHY - 1) / kHY, TXn = (c.W + kHX - 1) / kHX;
    const long long ntiles = (long long)c.B * TYn * TXn;
    const int KB = c.C / 32;                           // 32-channel blocks (C % 32 == 0)

    setup(B, &mapA, &mapB, tmem_slot, abort_flag, C::TMEM_COLS);
    const uint32_t tmem = *tmem_slot;

    if (warp == kProdWarp) {
        if (lane == 0) {
            // the layer's weights, once: chunk kc = tap * KB + cb (32 wide) at kc * BN * 64
            if (RES) {
                mbar_expect_tx(B.bres(), (uint32_t)(9 * KB * BN * 64));
                for (int kc = 0; kc < 9 * KB; ++kc) tma_load_2d(sbase + kc * BN * 64, &mapB, B.bres(), kc * 32, 0);
            }
            long long it = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                long long q = t;
                const int x0 = (int)(q % TXn) * kHX; q /= TXn;
                const int y0 = (int)(q % TYn) * kHY;
                const int b = (int)(q / TYn);
                bool ok = true;
                for (int cb = 0; cb < KB; ++cb, ++it) {
                    const int s = (int)(it % C::STAGES);
                    if (it >= C::STAGES &&
                        !mbar_wait(B.empty(s), (uint32_t)((it / C::STAGES) - 1) & 1u, err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = sbase + C::A_OFF + s * C::STAGE;
                    mbar_expect_tx(B.full(s), C::STAGE);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        tma_load_4d(sa + dx * kHaloCopy, &mapA, B.full(s), cb * 32, x0 + dx - 1, y0 - 1, b);
                    if (!RES)                              // this block's weights of the nine taps
                        for (int tap = 0; tap < 9; ++tap)
                            tma_load_2d(sa + kHaloStage + tap * BN * 64, &mapB, B.full(s), tap * c.C + cb * 32, 0);
                }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kBM, BN);
            long long it = 0, tc = 0;
            bool ok = !RES || mbar_wait(B.bres(), 0, err, abort_flag);
            for (long long t = blockIdx.x; ok && t < ntiles && !*abort_flag; t += gridDim.x, ++tc) {
                const int buf = (int)(tc & 1);
                if (tc >= 2 && !mbar_wait(B.acce(buf), (uint32_t)((tc >> 1) - 1) & 1u, err, abort_flag)) break;
                tc_fence_after();
                const uint32_t d = tmem + buf * C::ACC_STRIDE;
                for (int cb = 0; cb < KB; ++cb, ++it) {
                    const int s = (int)(it % C::STAGES);
                    if (!mbar_wait(B.full(s), (uint32_t)(it / C::STAGES) & 1u, err, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + C::A_OFF + s * C::STAGE;
#pragma unroll 1
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap - dy * 3;
                        const uint32_t a0 = sa + dx * kHaloCopy + dy * 512;
                        const uint32_t b0 = RES ? sbase + (tap * KB + cb) * BN * 64 : sa + kHaloStage + tap * BN * 64;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            tc_mma(d, sdesc64(a0 + kk * 32), sdesc64(b0 + kk * 32), idesc, (cb | tap | kk) != 0);
                    }
                    tc_commit(B.empty(s));
                }
                if (!ok) break;
                tc_commit(B.accf(buf));
            }
            drain(B);
        }
        __syncwarp();
    } else {
        epilogue<BN, kHY, kHX, C::ACC_STRIDE>(c, B, tmem, ntiles, 1, TYn, TXn, err, abort_flag);
    }
    teardown(tmem, C::TMEM_COLS);
}

// Weights in K-major order for the tensor-core kernel, k = tap * Kt + channel, zero for
// channels >= the convolution's input channels (Kt = that count rounded up to 64):
//   forward (flip = 0): wt[co][t * Kt + ci] = w[t][ci][co]            (N = Cout)
//   data gradient (1):  wt[ci][t * Kt + co] = w[8 - t][ci][co]        (N = Cin)
__global__ void k_wt_kmajor(const bf16* __restrict__ w, int Cin, int Cout, int flip, int Kt, bf16* __restrict__ wt) {
    const int N = flip ? Cin : Cout, Kc = flip ? Cout : Cin;
    const long long Kpad = 9LL * Kt;
    const long long n_el = (long long)N * Kpad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_el; i += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(i / Kpad), k = (int)(i - (long long)n * Kpad);
        const int t = k / Kt, cc = k - t * Kt;
        bf16 v = __float2bfloat16(0.f);
        if (cc < Kc) v = flip ? w[((long long)(8 - t) * Cin + n) * Cout + cc] : w[((long long)t * Cin + cc) * Cout + n];
        wt[i] = v;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return enc;
}

bool encode_maps(const TcConv& c, int bn, bool halo, CUtensorMap* ma, CUtensorMap* mb) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    const cuuint32_t cw = halo ? 32 : 64;                  // channels per box row
    const CUtensorMapSwizzle sw = halo ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    const cuuint64_t da[4] = {(cuuint64_t)c.C, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.B};
    const cuuint64_t sa[3] = {(cuuint64_t)c.C * 2, (cuuint64_t)c.W * c.C * 2, (cuuint64_t)c.H * c.W * c.C * 2};
    const cuuint32_t ba[4] = {cw, (cuuint32_t)(halo ? kHX : kTX), (cuuint32_t)(halo ? kHY + 2 : kTY), 1};
    const cuuint32_t e4[4] = {1, 1, 1, 1};
    if (enc(ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)c.in, da, sa, ba, e4, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const long long Kpad = 9LL * tc_layer_kt(c.C, c.N);
    const cuuint64_t db[2] = {(cuuint64_t)Kpad, (cuuint64_t)c.N};
    const cuuint64_t sb[1] = {(cuuint64_t)Kpad * 2};
    const cuuint32_t bb[2] = {cw, (cuuint32_t)bn};
    return enc(mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)c.wt, db, sb, bb, e4, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

template <int BN>
cudaError_t launch_tma(const TcConv& c, int* err, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Tc<BN>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap ma, mb;
    if (!encode_maps(c, BN, false, &ma, &mb)) return cudaErrorInvalidValue;
    const long long tiles = (long long)c.B * ((c.H + kTY - 1) / kTY) * ((c.W + kTX - 1) / kTX) * (c.N / BN);
    const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
    if (grid <= 0) return cudaSuccess;
    k_conv_tma<BN><<<grid, kThreads, Tc<BN>::SMEM, st>>>(ma, mb, c, err);
    return cudaGetLastError();
}

template <int BN, bool RES>
cudaError_t launch_halo(const TcConv& c, int* err, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_conv_halo<BN, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, Th<BN, RES>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap ma, mb;
    if (!encode_maps(c, BN, true, &ma, &mb)) return cudaErrorInvalidValue;
    const long long tiles = (long long)c.B * ((c.H + kHY - 1) / kHY) * ((c.W + kHX - 1) / kHX);
    const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
    if (grid <= 0) return cudaSuccess;
    k_conv_halo<BN, RES><<<grid, kThreads, Th<BN, RES>::SMEM, st>>>(ma, mb, c, err);
    return cudaGetLastError();
}

}  // namespace

int tc_kt(int C) { return (C + 63) / 64 * 64; }

// halo tiles: N in {32, 64} and whole 32-channel blocks; weights resident when they fit
static bool halo_ok(int C, int N) { return (N == 32 || N == 64) && C % 32 == 0; }
static bool halo_resident(int C, int N) { return halo_ok(C, N) && 9LL * C * N * 2 <= kHaloBmax; }

int tc_layer_kt(int C, int N) { return halo_ok(C, N) ? C : tc_kt(C); }

cudaError_t tc_weights(const bf16* w, int Cin, int Cout, int flip, bf16* wt, cudaStream_t st) {
    const int Kt = flip ? tc_layer_kt(Cout, Cin) : tc_layer_kt(Cin, Cout);
    const long long n = (long long)(flip ? Cin : Cout) * 9 * Kt;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_wt_kmajor<<<(int)blocks, 256, 0, st>>>(w, Cin, Cout, flip, Kt, wt);
    return cudaGetLastError();
}

bool tc_supported(int C, int N) {
    return C % 8 == 0 && C >= 8 && (N == 32 || N == 64 || N == 96 || N == 128 || N == 192 || N == 256 || N == 384);
}

cudaError_t conv3x3_tma(const TcConv& c, int* err, cudaStream_t st) {
    if (!tc_supported(c.C, c.N) || c.B < 1 || c.H < 1 || c.W < 1) return cudaErrorInvalidValue;
    if (c.out2 && (c.ld2 % 8 || c.off2 % 8)) return cudaErrorInvalidValue;
    if (c.pool && (!c.out || c.H % 2 || c.W % 2)) return cudaErrorInvalidValue;
    if (halo_resident(c.C, c.N)) return c.N == 32 ? launch_halo<32, true>(c, err, st) : launch_halo<64, true>(c, err, st);
    if (halo_ok(c.C, c.N)) return c.N == 32 ? launch_halo<32, false>(c, err, st) : launch_halo<64, false>(c, err, st);
    switch (c.N) {
        case 32: return launch_tma<32>(c, err, st);
        case 64: return launch_tma<64>(c, err, st);
        case 96: case 192: return launch_tma<96>(c, err, st);
        case 128: case 384: return launch_tma<128>(c, err, st);
        case 256: return launch_tma<256>(c, err, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mprnet
