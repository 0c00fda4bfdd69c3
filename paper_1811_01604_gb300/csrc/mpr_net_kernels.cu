// mpr_net_kernels.cu -- the weight gradient of the warm-start network's 3x3 convolutions
// (a reduction over pixels on mma.sync, bf16 inputs, fp32 accumulation).
#include "mpr_net_kernels.cuh"

namespace mprnet {
namespace {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte asynchronous copy; src_bytes = 0 fills the destination with zeros.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr(dst)), "l"(src),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                        const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                          const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(saddr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1) : "r"(saddr(p)));
}
// D = A (16x16, row) * B (16x8, col) + D, bf16 inputs, fp32 accumulators
__device__ __forceinline__ void mma16816(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Address of 8 consecutive channels [c, c + 8) of the virtual input at pixel (b, y, x)
// (zero bytes when (y, x) lies outside the image).
__device__ __forceinline__ const bf16* in_ptr(const ConvIn& in, int b, int y, int x, int H, int W,
                                              int c, int* bytes) {
    if (y < 0 || y >= H || x < 0 || x >= W) {
        *bytes = 0;
        return in.src0;
    }
    *bytes = 16;
    if (c < in.C0) return in.src0 + (((long long)b * H + y) * W + x) * in.C0 + c;
    const int c1 = c - in.C0;
    if (in.up1) {
        const int Hh = (H + 1) >> 1, Wh = (W + 1) >> 1;
        return in.src1 + (((long long)b * Hh + (y >> 1)) * Wh + (x >> 1)) * in.C1 + c1;
    }
    return in.src1 + (((long long)b * H + y) * W + x) * in.C1 + c1;
}

// Weight gradient: block tile 64 (k = tap * Cin + ci) x 64 (co), reduction over a chunk of
// pixels in steps of 32; 8 warps: 2 along k x 4 along co (32 x 16 each).
constexpr int WK = 64, WC = 64, WP = 32, WPIX = 4096;   // WPIX pixels per block
__global__ void __launch_bounds__(256) k_conv3x3_wgrad(const ConvIn in, int B, int H, int W, int Cin,
                                                       const bf16* __restrict__ gr, int Cout,
                                                       float* __restrict__ dW) {
    __shared__ __align__(16) bf16 Xs[2][WP][WK + 8];      // [pixel][k]
    __shared__ __align__(16) bf16 Gs[2][WP][WC + 8];      // [pixel][co]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wk = warp & 1, wc = warp >> 1;
    const int k0 = blockIdx.x * WK, c0 = blockIdx.y * WC;
    const long long P = (long long)B * H * W;
    const long long pbeg = (long long)blockIdx.z * WPIX;
    const long long pend = pbeg + WPIX < P ? pbeg + WPIX : P;
    const int HW = H * W;
    const int K = 9 * Cin;
    auto load = [&](long long pb, int s) {
        // X tile: 32 pixels x 64 k in 8-channel pieces: 256 pieces, one per thread
        {
            const int r = tid >> 3, piece = tid & 7;
            const long long p = pb + r;
            const int k = k0 + piece * 8;
            int bytes = 0;
            const bf16* src = in.src0;
            if (p < pend && k < K) {
                const int tap = k / Cin, ci = k - tap * Cin;
                const int b = (int)(p / HW), rr = (int)(p - (long long)b * HW);
                const int y = rr / W, x = rr - (rr / W) * W;
                src = in_ptr(in, b, y + tap / 3 - 1, x + tap % 3 - 1, H, W, ci, &bytes);
            }
            cp16(&Xs[s][r][piece * 8], src, bytes);
        }
        // G tile: 32 pixels x 64 co
        {
            const int r = tid >> 3, piece = tid & 7;
            const long long p = pb + r;
            const int c = c0 + piece * 8;
            const bool ok = p < pend && c < Cout;
            cp16(&Gs[s][r][piece * 8], gr + (ok ? p * Cout + c : 0), ok ? 16 : 0);
        }
    };
    float acc[2][2][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    const int steps = (int)((pend - pbeg + WP - 1) / WP);
    if (steps > 0) {
        load(pbeg, 0);
        cp_commit();
    }
    for (int st = 0; st < steps; ++st) {
        const int s = st & 1;
        if (st + 1 < steps) load(pbeg + (long long)(st + 1) * WP, s ^ 1);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < WP; kk += 16) {          // reduction index = pixel
            uint32_t af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                // A = X^T (m = k, reduction = pixel); smem rows are pixels, so transpose:
                // lanes 0-7: pixel rows kk..kk+7, m cols 0-7; 8-15: same rows, m 8-15;
                // 16-23: pixel rows kk+8.., m 0-7; 24-31: pixel rows kk+8.., m 8-15
                const int prow = kk + (lane & 7) + (lane >> 4) * 8;
                const int mcol = wk * 32 + i * 16 + ((lane >> 3) & 1) * 8;
                ldsm_x4_t(af[i][0], af[i][1], af[i][2], af[i][3], &Xs[s][prow][mcol]);
            }
            uint32_t b0, b1, b2, b3;
            {
                const int prow = kk + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int ncol = wc * 16 + (lane >> 4) * 8;
                ldsm_x4_t(b0, b1, b2, b3, &Gs[s][prow][ncol]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                mma16816(acc[i][0], af[i][0], af[i][1], af[i][2], af[i][3], b0, b1);
                mma16816(acc[i][1], af[i][0], af[i][1], af[i][2], af[i][3], b2, b3);
            }
        }
        __syncthreads();
    }
    cp_wait<0>();
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + wk * 32 + i * 16 + h * 8 + g;
            if (k >= K) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int c = c0 + wc * 16 + j * 8 + 2 * t;
                if (c >= Cout) continue;
                atomicAdd(dW + (long long)k * Cout + c, acc[i][j][2 * h]);
                atomicAdd(dW + (long long)k * Cout + c + 1, acc[i][j][2 * h + 1]);
            }
        }
}

}  // namespace

cudaError_t conv3x3_wgrad(const ConvIn& in, int B, int H, int W, int Cin, const bf16* g, int Cout,
                          float* dW, cudaStream_t st) {
    const long long P = (long long)B * H * W;
    if ((P + WPIX - 1) / WPIX > 65535) return cudaErrorInvalidValue;      // grid.z limit
    const dim3 grid((unsigned)((9 * Cin + WK - 1) / WK), (unsigned)((Cout + WC - 1) / WC),
                    (unsigned)((P + WPIX - 1) / WPIX));
    k_conv3x3_wgrad<<<grid, 256, 0, st>>>(in, B, H, W, Cin, g, Cout, dW);
    return cudaGetLastError();
}

}  // namespace mprnet
