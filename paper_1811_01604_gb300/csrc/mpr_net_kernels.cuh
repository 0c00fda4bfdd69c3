// mpr_net_kernels.cuh -- BF16 tensor-core kernels of the warm-start network.
//
// Activations are NHWC bf16, weights [tap = 3 ky + kx][C_in][C_out] bf16 (C_out contiguous),
// gradients fp32.  Every 3x3 convolution (stride 1, zero padding 1) is an implicit GEMM
// over M = pixels, N = output channels, K = 9 C_in.  Forward and data-gradient convolutions
// run on the 5th-generation tensor cores (tcgen05, TMA-fed; conv3x3_tma); the weight
// gradient (training only) is a reduction over pixels computed with mma.sync m16n8k16
// (bf16 x bf16 -> fp32) on fragments loaded by ldmatrix from cp.async-filled shared memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mprnet {

typedef __nv_bfloat16 bf16;

// A convolution input: the channel-wise concatenation of src0 (C0 channels, full
// resolution) and src1 (C1 channels, at half resolution and upsampled by nearest
// neighbour if up1, else full resolution).  C0 and C1 are multiples of 32 (C1 may be 0).
struct ConvIn {
    const bf16* src0;
    int C0;
    const bf16* src1;
    int C1;
    int up1;
};

// An fp32 output split by channel ranges: channels [0, C0) to dst0, [C0, C0 + C1) to dst1
// (each NHWC with its own channel count); accumulate adds to the destination.
struct ConvOutF32 {
    float* dst0;
    int C0;
    float* dst1;
    int C1;
    int accumulate;
};

struct ConvArgs {
    ConvIn in;
    int B, H, W;                 // spatial size of input and output
    int Cin;                     // C0 + C1
    const bf16* w;               // [9 * Cin][Cout]
    int Cout;
    const float* bias;           // forward: [Cout] or null
    int relu;                    // forward: apply ReLU
    bf16* out_bf16;              // forward output [B][H][W][Cout]
    ConvOutF32 out_f32;          // backward output (used when out_bf16 is null)
};

// dW[tap][ci][co] += sum_p in(p + tap)[ci] * g[p][co] over all pixels (in: ConvIn with the
// forward layer's input, g: bf16 [B][H][W][Cout]).  dW fp32, accumulated with atomics.
cudaError_t conv3x3_wgrad(const ConvIn& in, int B, int H, int W, int Cin, const bf16* g, int Cout,
                          float* dW, cudaStream_t st);

// ---- tensor-core (tcgen05 + TMA) path: forward and data-gradient convolutions ----
// K-major weights: wt[n][k], k = tap * Kt + c, zero for c >= C, with C the input channels of
// the convolution, N its output channels and Kt = tc_layer_kt(C, N) (C itself for the
// halo-tile kernel, else C rounded up to 64).  flip = 0: forward weights of w[9][Cin][Cout]
// (n = co, C = Cin); flip = 1: data-gradient weights (n = ci, C = Cout, tap reflected).
int tc_kt(int C);
int tc_layer_kt(int C, int N);
cudaError_t tc_weights(const bf16* w, int Cin, int Cout, int flip, bf16* wt, cudaStream_t st);
// Channel counts the kernel instantiates: C any multiple of 8; N in {32, 64, 96, 128, 192,
// 256, 384}.
bool tc_supported(int C, int N);

// One tensor-core convolution.  in: NHWC bf16 [B][H][W][C] (16-byte aligned).  bf16 output
// (out non-null): out[p][N] = relu?(conv + bias), and if out2: the same values also at
// out2[p'][off2 + n] with channel stride ld2, where p' is p itself or, with up2, each of the
// 2 x 2 pixels of a 2H x 2W image that p covers under nearest upsampling; if pool: the 2 x 2
// average of the stored bf16 values, ((a + b) + c) + d then times 1/4, at [B][H/2][W/2][N]
// (H, W even).  fp32 output (out null): `of` as in ConvOutF32.
struct TcConv {
    const bf16* in;
    int C;
    int B, H, W;
    int N;
    const bf16* wt;
    const float* bias;
    int relu;
    bf16* out;
    bf16* out2;
    int ld2, off2, up2;
    bf16* pool;
    ConvOutF32 of;
};
// A barrier wait that expires sets *err (device int) to 1.
cudaError_t conv3x3_tma(const TcConv& c, int* err, cudaStream_t st);

}  // namespace mprnet
