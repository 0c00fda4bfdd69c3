/*
 * mpr_net.h -- C ABI of the learned warm start of libmpr.so.
 *
 * The warm start replaces the uniform random initial state of the gap sites in
 * Algorithm 2 (the conditional hybrid Monte Carlo then runs unchanged: the same
 * relaxation with the energy-slope stopping test, the same M equilibrium sweeps).
 * It is not part of the paper's method; a good initial state only shortens the
 * relaxation.
 *
 * Network: a 4-level convolutional encoder-decoder (U-Net style) on the grid.
 *  - Input per site (NHWC, 32 channels, 3 used): (cos theta, sin theta, 1) at
 *    sample sites and (0, 0, 0) at gap sites, with theta = q phi, q = 1/2, and phi
 *    the data-to-angle map of Eq. 1 (zmin, zmax of the grid's samples).
 *  - Encoder: two 3x3 convolutions + ReLU per level, channels 32, 64, 128, 256;
 *    2x2 average pooling between levels.  Decoder: nearest 2x upsampling,
 *    concatenation with the encoder output of the same level, two 3x3
 *    convolutions + ReLU (128, 64, 32); a 1x1 head to (u, v).
 *  - Prediction: theta_0 = direction of (u, max(v, 0)) in [0, pi), phi_0 = 2 theta_0.
 *  - Loss (training), mean over the batch's gap sites: 1 - cos(theta_0 - theta_t)
 *    with theta_t = phi_t / 2 of an equilibrium state of the MCMC.
 *  - Precision: bf16 weights and activations, fp32 accumulation (tensor cores),
 *    fp32 master weights, gradients, head and loss.  Adam (beta 0.9, 0.999, eps 1e-8).
 *  - Parameters: one fp32 vector; per convolution (order e0a e0b e1a e1b e2a e2b
 *    e3a e3b d2a d2b d1a d1b d0a d0b) W[9][C_in][C_out] (tap = 3 dy + dx) then
 *    b[C_out]; then the head Wh[32][2], bh[2].
 *
 * Conventions: as in mpr.h.  z (float), mask (uint8, 1 = sample) and phi_target
 * (float, radians in [0, 2 pi)) are [B][H][W] device arrays (B images of one
 * shape, contiguous); zmin, zmax are B doubles (host or device).  H and W are
 * positive multiples of 8 x stride (see mpr_net_create_strided), 1 <= B <= 4096.  All work is enqueued on the stream
 * given at creation; calls that return host values synchronise it.  A network is
 * not thread-safe.  Its activation workspace grows to the largest B x H x W frame
 * seen (training needs more than inference) and serves every smaller frame.
 */
#ifndef MPR_NET_H_
#define MPR_NET_H_

#include <stdint.h>

#include "mpr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpr_net mpr_net;

/* A new network with He-initialised weights drawn from seed (host PRNG).
   ENOMEM / ECUDA on device failure; *net is NULL then. */
mpr_status mpr_net_create(mpr_net** net, uint64_t seed, void* cuda_stream);
/* The same at stride 1, 2, 4 or 8 (mpr_net_create is stride 1).  At stride S the network works
   on a frame S times coarser along each axis: frame pixel (Y, X) stands for the S x S
   block of sites (S Y + dy, S X + dx); its input channels are the block means of the
   per-site input above, every gap site of the block takes the pixel's prediction, and
   the training loss stays the mean over the gap SITES of 1 - cos(theta_0 - theta_t).
   The network costs S^2 times less; the MCMC that follows refines the fine scale.
   EINVAL for another stride. */
mpr_status mpr_net_create_strided(mpr_net** net, uint64_t seed, int stride, void* cuda_stream);
/* The network's stride (0 for NULL). */
int mpr_net_stride(const mpr_net* net);
void mpr_net_free(mpr_net* net);
const char* mpr_net_last_error(const mpr_net* net);

/* Number of fp32 parameters (the layout above). */
long long mpr_net_num_params(const mpr_net* net);
/* Copy the fp32 parameters out / in (host or device, num_params floats).  set
   also refreshes the bf16 copy and resets the Adam state. */
mpr_status mpr_net_get_params(mpr_net* net, float* params);
mpr_status mpr_net_set_params(mpr_net* net, const float* params);
/* Accumulated gradient (num_params floats) and its reset. */
mpr_status mpr_net_get_grads(mpr_net* net, float* grads);
mpr_status mpr_net_zero_grads(mpr_net* net);

/* Forward pass, loss and backward pass on a batch; the gradient is ADDED to the
   network's gradient buffer.  *loss (host, may be NULL: no synchronisation) is the
   mean loss over the batch's gap sites (0 if there are none). */
mpr_status mpr_net_loss_grad(mpr_net* net, const float* z, const uint8_t* mask, const float* phi_target,
                             const double* zmin, const double* zmax, int B, int H, int W, double* loss);
/* One Adam step with learning rate lr on the accumulated gradient, which it clears. */
mpr_status mpr_net_adam_step(mpr_net* net, float lr);
/* mpr_net_loss_grad followed by mpr_net_adam_step. */
mpr_status mpr_net_train_step(mpr_net* net, const float* z, const uint8_t* mask, const float* phi_target,
                              const double* zmin, const double* zmax, int B, int H, int W, float lr,
                              double* loss);
/* Network output (u, v) per frame pixel: uv is float [B][H/S][W/S][2] at stride S
   (host or device). */
mpr_status mpr_net_forward(mpr_net* net, const float* z, const uint8_t* mask, const double* zmin,
                           const double* zmax, int B, int H, int W, float* uv);

/* Writes the warm-start state theta_0 into the gap sites of every grid of a
   context (replacing their random initial state; samples are untouched).  Grids of
   any shape (the network runs on the grid padded to multiples of 8, padding read
   as gaps).  Call after mpr_init / mpr_init_batch and before mpr_equilibrate or
   mpr_fill.  EINVAL for NULL arguments. */
mpr_status mpr_warmstart_init(mpr_ctx* ctx, mpr_net* net);

/* Test support (layer-by-layer checks): copies one internal tensor of the network, as the
   last mpr_net_forward / mpr_net_loss_grad call left it, to out (host or device), count
   elements; returns after the copy.  kind, index and layout (frame H x W = the call's grid
   divided by the stride; level l of a layer: H >> l x W >> l):
     MPR_NET_T_INPUT  the input, bf16 [B][H][W][32] (index ignored)
     MPR_NET_T_ACT    output of convolution index (0..13, ReLU applied), bf16 [B][Hl][Wl][C_out]
     MPR_NET_T_POOL   2 x 2 average of the output of convolution 2 index + 1 (index 0..2),
                      bf16 [B][H >> (index + 1)][W >> (index + 1)][C_out of that convolution]
     MPR_NET_T_DACT   loss gradient w.r.t. the output of convolution index, before the ReLU
                      gate, fp32 [B][Hl][Wl][C_out] (after mpr_net_loss_grad only)
     MPR_NET_T_OUT    head output (u, v), fp32 [B][H][W][2] (index ignored)
   MPR_EINVAL if count is not the tensor's element count, MPR_ESTATE if the tensor does not
   exist after the last call.  No counterpart in the paper (the network is this library's). */
enum { MPR_NET_T_INPUT = 0, MPR_NET_T_ACT = 1, MPR_NET_T_POOL = 2, MPR_NET_T_DACT = 3, MPR_NET_T_OUT = 4 };
mpr_status mpr_net_tensor(mpr_net* net, int kind, int index, void* out, long long count);

/* Test support: one 3x3 convolution (zero padding 1) of the network on caller
   device buffers.  in: bf16 [B][H][W][Cin], w: bf16 [9][Cin][Cout], bias: fp32
   [Cout] or NULL, out: bf16 [B][H][W][Cout] = relu?(conv(in) + bias).  Cin, Cout
   positive multiples of 32. */
mpr_status mpr_net_conv3x3(const uint16_t* in, int B, int H, int W, int Cin, const uint16_t* w,
                           const float* bias, int Cout, int relu, uint16_t* out, void* cuda_stream);
/* Its two gradients for an output gradient gout (bf16 [B][H][W][Cout]):
   din = fp32 [B][H][W][Cin] (overwritten), dw = fp32 [9][Cin][Cout] (added to);
   w_scratch: bf16 [9][Cin][Cout] device scratch. */
mpr_status mpr_net_conv3x3_bwd(const uint16_t* in, const uint16_t* gout, int B, int H, int W, int Cin,
                               const uint16_t* w, int Cout, float* din, float* dw, uint16_t* w_scratch,
                               void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPR_NET_H_ */
