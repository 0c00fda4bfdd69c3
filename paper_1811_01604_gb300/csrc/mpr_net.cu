// mpr_net.cu -- the learned warm start: a 4-level convolutional encoder-decoder that maps
// the samples of a grid (unit vectors of their half angles theta = q phi, Eq. 1, and the
// mask) to initial gap angles, replacing the uniform random initial gap state of
// Algorithm 2.  The MCMC that follows is unchanged.  Forward, backward and Adam run in the
// kernels below; weights and activations are bf16, accumulation and master weights fp32.
//
// Network (NHWC, 3x3 convolutions with ReLU, 2x2 average pooling, nearest upsampling):
//   level 0 (H):   in(32: c, s, m, 0...) -> 32 -> 32 = A0
//   level 1 (H/2): pool(A0) -> 64 -> 64 = A1
//   level 2 (H/4): pool(A1) -> 128 -> 128 = A2
//   level 3 (H/8): pool(A2) -> 256 -> 256 = A3
//   decoder:       [A2, up(A3)] -> 128 -> 128 = D2;  [A1, up(D2)] -> 64 -> 64 = D1;
//                  [A0, up(D1)] -> 32 -> 32 = D0;  1x1 head (fp32) -> (u, v)
// A gap's initial state is the direction of (u, max(v, 0)): theta in [0, pi), phi = 2 theta.
// Training loss, mean over gap sites: 1 - cos(theta_pred - theta_target).
//
// Parameter vector (fp32): for each of the 14 convolutions W[9][C_in][C_out] then b[C_out],
// in the order e0a e0b e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b d0a d0b; then the head
// Wh[32][2], bh[2].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/mpr.h"
#include "../../include/mpr_net.h"
#include "mpr_internal.cuh"
#include "mpr_net_internal.cuh"
#include "mpr_net_kernels.cuh"

using mprnet::bf16;
using mprnet::ConvArgs;
using mprnet::ConvIn;

namespace {

constexpr int kIn = 32;                // input channels (3 used, padded to one 32-channel chunk)
constexpr int kHeadC = 32;             // channels into the head
constexpr int kMaxB = 4096;            // images per call

// ---------------------------------------------------------------- elementwise kernels
// Network input: image b of B, grid Hin x Win (contiguous images); the network frame is
// H x W (multiples of 8) at stride S: frame pixel (Y, X) covers the S x S block of sites
// (S Y + dy, S X + dx), and its channels are the block means of (cos theta, sin theta, 1)
// over the block's sample sites (sites outside the grid read as missing samples).
__global__ void k_input(const float* __restrict__ z, const uint8_t* __restrict__ mask, int B, int Hin, int Win,
                        int H, int W, int S, const double* __restrict__ zmin, const double* __restrict__ zmax,
                        bf16* __restrict__ out) {
    const long long n = (long long)B * H * W;
    const float inv = 1.0f / (float)(S * S);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % W);
        const long long r = p / W;
        const int Y = (int)(r % H);
        const int b = (int)(r / H);
        float c = 0.f, s = 0.f, m = 0.f;
        for (int dy = 0; dy < S; ++dy)
            for (int dx = 0; dx < S; ++dx) {
                const int y = S * Y + dy, x = S * X + dx;
                if (y < Hin && x < Win) {
                    const long long i = ((long long)b * Hin + y) * Win + x;
                    if (mask[i]) {
                        // theta = q phi with q = 1/2 and phi of Eq. 1
                        const double th = 3.141592653589793 * ((double)z[i] - zmin[b]) / (zmax[b] - zmin[b]);
                        float si, ci;
                        sincosf((float)th, &si, &ci);
                        c += ci;
                        s += si;
                        m += 1.f;
                    }
                }
            }
        if (S > 1) {
            c *= inv;
            s *= inv;
            m *= inv;
        }
        const __nv_bfloat162 cs = __floats2bfloat162_rn(c, s);      // .x = c (low half)
        const __nv_bfloat162 m0 = __floats2bfloat162_rn(m, 0.f);
        uint4* o = reinterpret_cast<uint4*>(out + p * kIn);
        o[0] = make_uint4(*reinterpret_cast<const uint32_t*>(&cs), *reinterpret_cast<const uint32_t*>(&m0), 0u, 0u);
        o[1] = o[2] = o[3] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// dIn (H x W) += dOut (H/2 x W/2) / 4 on each 2x2 block
__global__ void k_pool_bwd(const float* __restrict__ dout, int B, int H, int W, int C, float* __restrict__ din) {
    const long long n = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int x = (int)(q % W); q /= W;
        const int y = (int)(q % H);
        const int b = (int)(q / H);
        din[i] += 0.25f * dout[(((long long)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
    }
}

// dLow (H/2 x W/2) = sum over each 2x2 block of dHigh (adjoint of nearest upsampling)
__global__ void k_upsum(const float* __restrict__ dhigh, int B, int H, int W, int C, float* __restrict__ dlow) {
    const int Ho = H / 2, Wo = W / 2;
    const long long n = (long long)B * Ho * Wo * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long q = i / C;
        const int x = (int)(q % Wo); q /= Wo;
        const int y = (int)(q % Ho);
        const int b = (int)(q / Ho);
        const float* s = dhigh + (((long long)b * H + 2 * y) * W + 2 * x) * C + c;
        dlow[i] = s[0] + s[C] + s[(long long)W * C] + s[(long long)W * C + C];
    }
}

// gradient through the ReLU (act > 0), rounded to bf16 for the tensor-core kernels
__global__ void k_gate(const float* __restrict__ d, const bf16* __restrict__ act, long long n, bf16* __restrict__ g) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.f ? d[i] : 0.f);
}

// db[c] += sum over pixels of g[p][c]
__global__ void k_bias_grad(const bf16* __restrict__ g, long long P, int C, float* __restrict__ db) {
    const int c = blockIdx.y * 32 + (threadIdx.x & 31);
    if (c >= C) return;
    float s = 0.f;
    for (long long p = blockIdx.x * 8 + (threadIdx.x >> 5); p < P; p += (long long)gridDim.x * 8)
        s += __bfloat162float(g[p * C + c]);
    atomicAdd(db + c, s);
}

// 1x1 head: out[p][o] = sum_c act[p][c] wh[c][o] + bh[o], o in {0, 1}
__global__ void k_head(const bf16* __restrict__ act, long long P, const float* __restrict__ wh,
                       const float* __restrict__ bh, float* __restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        float u = bh[0], v = bh[1];
        const uint4* a4 = reinterpret_cast<const uint4*>(act + p * kHeadC);
#pragma unroll
        for (int q = 0; q < kHeadC / 8; ++q) {
            const uint4 w4 = a4[q];
            const bf16* a = reinterpret_cast<const bf16*>(&w4);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float x = __bfloat162float(a[k]);
                u = fmaf(x, wh[2 * (8 * q + k)], u);
                v = fmaf(x, wh[2 * (8 * q + k) + 1], v);
            }
        }
        reinterpret_cast<float2*>(out)[p] = make_float2(u, v);
    }
}

__global__ void k_count_gaps(const uint8_t* __restrict__ mask, long long P, unsigned long long* __restrict__ cnt) {
    unsigned long long c = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x)
        c += mask[p] ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// circular loss, mean over the batch's gap sites, at stride S: every gap site of the S x S
// block of frame pixel p takes the direction of (u, v) = out[p]:
//   sum over the block's gaps of 1 - cos(theta - theta_t) = n_g - (u Tc + v Ts) / |(u, v)|
// with (Tc, Ts) the sum of the gaps' (cos, sin)(phi_target / 2) and n_g their number; and
// dL/d(u, v).  (S = 1: one site per pixel.)  phi_target and mask are B x Hin x Win with
// Hin = S H, Win = S W.
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ phi_t, const uint8_t* __restrict__ mask,
                       int B, int H, int W, int S, const unsigned long long* __restrict__ cnt, float* __restrict__ dout,
                       double* __restrict__ loss) {
    const unsigned long long ng_all = *cnt;
    const float inv = ng_all ? 1.f / (float)ng_all : 0.f;
    const long long P = (long long)B * H * W;
    const int Win = S * W;
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(p % W);
        const long long r = p / W;
        const int Y = (int)(r % H);
        const int b = (int)(r / H);
        float tc = 0.f, ts = 0.f, ng = 0.f;
        for (int dy = 0; dy < S; ++dy)
            for (int dx = 0; dx < S; ++dx) {
                const long long i = ((long long)b * (S * H) + S * Y + dy) * Win + S * X + dx;
                if (!mask[i]) {
                    float si, ci;
                    sincosf(0.5f * phi_t[i], &si, &ci);
                    tc += ci;
                    ts += si;
                    ng += 1.f;
                }
            }
        float du = 0.f, dv = 0.f;
        if (ng > 0.f) {
            const float2 o = reinterpret_cast<const float2*>(out)[p];
            const float n2 = fmaf(o.x, o.x, fmaf(o.y, o.y, 1e-12f));
            const float n = sqrtf(n2);
            const float dot = fmaf(o.x, tc, o.y * ts);
            acc += (double)ng - (double)(dot / n);
            const float n3 = n2 * n;
            du = inv * (dot * o.x / n3 - tc / n);
            dv = inv * (dot * o.y / n3 - ts / n);
        }
        reinterpret_cast<float2*>(dout)[p] = make_float2(du, dv);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(loss, acc * (double)inv);
}

// head backward: dact[p][c] = sum_o dout[p][o] wh[c][o]; dwh[c][o] += sum_p act dout;
// dbh[o] += sum_p dout
__global__ void k_head_bwd(const bf16* __restrict__ act, const float* __restrict__ dout, long long P,
                           const float* __restrict__ wh, float* __restrict__ dact, float* __restrict__ dwh,
                           float* __restrict__ dbh) {
    float gw[2 * kHeadC];
#pragma unroll
    for (int i = 0; i < 2 * kHeadC; ++i) gw[i] = 0.f;
    float gb0 = 0.f, gb1 = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float2 d = reinterpret_cast<const float2*>(dout)[p];
        gb0 += d.x;
        gb1 += d.y;
#pragma unroll
        for (int c = 0; c < kHeadC; ++c) {
            const float a = __bfloat162float(act[p * kHeadC + c]);
            dact[p * kHeadC + c] = fmaf(d.x, wh[2 * c], d.y * wh[2 * c + 1]);
            gw[2 * c] = fmaf(a, d.x, gw[2 * c]);
            gw[2 * c + 1] = fmaf(a, d.y, gw[2 * c + 1]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2 * kHeadC; ++i) {
        float v = gw[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(dwh + i, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        gb0 += __shfl_xor_sync(0xffffffffu, gb0, o);
        gb1 += __shfl_xor_sync(0xffffffffu, gb1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(dbh, gb0);
        atomicAdd(dbh + 1, gb1);
    }
}

// Adam on the fp32 master parameters; refreshes the bf16 copy and clears the gradient
__global__ void k_adam(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2, bf16* __restrict__ wb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
        g[i] = 0.f;
    }
}

__global__ void k_to_bf16(const float* __restrict__ a, long long n, bf16* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

// Gap sites of image blockIdx.y (entry ents[blockIdx.y], grid Hin x Win; network frame
// H x W at stride S: site (y, x) takes frame pixel (y / S, x / S)) <- unit vector of
// (u, max(v, 0)), in one or both lattice buffers.
__global__ void k_to_lattice(const float* __restrict__ out, const uint8_t* __restrict__ mask,
                             const mpr::EntryDesc* __restrict__ ents, int H, int W, int S, float2* __restrict__ lat0,
                             float2* __restrict__ lat1) {
    const int b = blockIdx.y;
    const mpr::EntryDesc e = ents[b];
    const long long n = (long long)e.W * e.H;
    const uint8_t* mk = mask + (long long)b * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (mk[i]) continue;
        const int y = (int)(i / e.W), x = (int)(i - (long long)y * e.W);
        const float2 o = reinterpret_cast<const float2*>(out)[((long long)b * H + y / S) * W + x / S];
        float u = o.x;
        float v = fmaxf(o.y, 1e-6f * fabsf(o.x));          // upper half circle, theta < pi
        const float r = sqrtf(u * u + v * v);
        if (!(r > 1e-30f)) { u = 0.f; v = 1.f; } else { u /= r; v /= r; }
        const long long base = ((x + y) & 1) ? e.plane[1] : e.plane[0];
        const long long k = base + (long long)(y + 1) * e.pitch + (x >> 1) + mpr::kPadL;
        lat0[k] = make_float2(u, v);
        if (lat1) lat1[k] = make_float2(u, v);
    }
}

int grid1(long long n) {
    long long b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return (int)(b < 1 ? 1 : b);
}

const int kLevel[14] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
const int kCin[14] = {kIn, 32, 32, 64, 64, 128, 128, 256, 128 + 256, 128, 64 + 128, 64, 32 + 64, 32};
const int kCout[14] = {32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32};
const int kCatC[3] = {32 + 64, 64 + 128, 128 + 256};

}  // namespace

struct mpr_net {
    cudaStream_t st = nullptr;
    long long off_w[14] = {0}, off_b[14] = {0};   // offsets into the parameter vector
    long long off_wh = 0, off_bh = 0;
    long long n_params = 0;
    float* w = nullptr;                // fp32 master parameters
    float* g = nullptr;                // gradients
    float* m = nullptr;                // Adam moments
    float* v = nullptr;
    bf16* wb = nullptr;                // bf16 copy of the parameters (conv weights are read from it)
    bf16* wt = nullptr;                // K-major weights of the tensor-core kernels: forward
    bf16* wtb = nullptr;               //   and data-gradient, per layer at wt_off / wtb_off
    long long wt_off[14] = {0}, wtb_off[14] = {0};
    int* d_err = nullptr;              // set by a tensor-core kernel whose barrier wait expired
    int adam_t = 0;
    int stride = 1;                    // sites per frame pixel along each axis (1, 2, 4 or 8)
    double* d_zr = nullptr;            // zmin[kMaxB], zmax[kMaxB]
    double* d_loss = nullptr;
    unsigned long long* d_cnt = nullptr;
    // activation workspace, sized for B x H x W
    int B = 0, H = 0, W = 0;
    long long cap = 0;                 // B x H x W the workspace is sized for
    bool train = false;
    std::vector<void*> bufs;
    bf16* in0 = nullptr;
    bf16* act[14] = {nullptr};
    bf16* pool[3] = {nullptr};
    float* out2 = nullptr;             // head output (u, v)
    float* dout2 = nullptr;
    float* dact[14] = {nullptr};
    float* dpool[3] = {nullptr};
    float* dup = nullptr;              // gradient w.r.t. an upsampled tensor
    bf16* cat[3] = {nullptr};          // decoder inputs [A_l, up(lower)] of levels 0-2, written by
                                       //   the producing layers (tensor-core path)
    bf16* gb = nullptr;                // gated bf16 gradient of one layer
    std::string err;
};

namespace {

mpr_status nfail(mpr_net* n, mpr_status s, const std::string& m) {
    if (n) n->err = m;
    return s;
}
#define NCU(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return nfail(net, e_ == cudaErrorMemoryAllocation ? MPR_ENOMEM : MPR_ECUDA,             \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

void free_ws(mpr_net* n) {
    for (void* p : n->bufs) cudaFree(p);
    n->bufs.clear();
    n->B = n->H = n->W = 0;
    n->cap = 0;
    n->train = false;
}

template <class T>
cudaError_t nalloc(mpr_net* n, T** p, long long count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, (size_t)std::max(1LL, count) * sizeof(T));
    if (e == cudaSuccess) n->bufs.push_back(*p);
    return e;
}

// Every workspace buffer scales with B x H x W (level l holds B (H >> l)(W >> l) pixels,
// H and W multiples of 8), so buffers sized for a larger frame serve any smaller one: the
// workspace grows only, and calls on grids of many shapes (a batch) do not reallocate.
mpr_status ensure_ws(mpr_net* net, int B, int H, int W, bool train) {
    const long long P0 = (long long)B * H * W;
    if (P0 <= net->cap && (!train || net->train)) {
        net->B = B;
        net->H = H;
        net->W = W;
        return MPR_OK;
    }
    NCU(cudaStreamSynchronize(net->st));
    free_ws(net);
    NCU(nalloc(net, &net->in0, P0 * kIn));
    for (int l = 0; l < 14; ++l) {
        const long long P = P0 >> (2 * kLevel[l]);
        NCU(nalloc(net, &net->act[l], P * kCout[l]));
        if (train) NCU(nalloc(net, &net->dact[l], P * kCout[l]));
    }
    for (int i = 0; i < 3; ++i) {
        const long long P = P0 >> (2 * (i + 1));
        NCU(nalloc(net, &net->pool[i], P * kCout[2 * i + 1]));
        if (train) NCU(nalloc(net, &net->dpool[i], P * kCout[2 * i + 1]));
    }
    NCU(nalloc(net, &net->out2, P0 * 2));
    for (int i = 0; i < 3; ++i) NCU(nalloc(net, &net->cat[i], (P0 >> (2 * i)) * kCatC[i]));
    if (train) {
        NCU(nalloc(net, &net->dout2, P0 * 2));
        NCU(nalloc(net, &net->dup, P0 * 64));       // largest: level 0, 64 upsampled channels
        NCU(nalloc(net, &net->gb, P0 * 32));        // largest: level 0 (32 ch) = level 1 (64 ch) x 4
    }
    net->B = B;
    net->H = H;
    net->W = W;
    net->train = train;
    net->cap = P0;
    return MPR_OK;
}

// K-major copies of the current bf16 weights for the tensor-core kernels
mpr_status refresh_wt(mpr_net* net) {
    for (int l = 0; l < 14; ++l) {
        NCU(mprnet::tc_weights(net->wb + net->off_w[l], kCin[l], kCout[l], 0, net->wt + net->wt_off[l], net->st));
        NCU(mprnet::tc_weights(net->wb + net->off_w[l], kCin[l], kCout[l], 1, net->wtb + net->wtb_off[l], net->st));
    }
    mpr::count_launches(28, net->st);
    return MPR_OK;
}

// One convolution on the tensor cores (TMA-fed, weights from the K-major copy).  The
// decoder inputs are the concatenation buffers, which the layers producing their parts
// also write (A_l as is, the lower level upsampled); 2 x 2 pooling is fused into the
// epilogue of the layer it follows.
mpr_status conv(mpr_net* net, ConvArgs& a, int l, bool dgrad) {
    mprnet::TcConv c;
    std::memset(&c, 0, sizeof c);
    c.B = a.B; c.H = a.H; c.W = a.W;
    c.N = a.Cout;
    if (dgrad) {
        c.in = a.in.src0;
        c.C = a.Cin;
        c.wt = net->wtb + net->wtb_off[l];
        c.of = a.out_f32;
    } else {
        if (l == 8 || l == 10 || l == 12) {
            const int lev = kLevel[l];
            c.in = net->cat[lev];
            c.C = kCatC[lev];
        } else {
            c.in = a.in.src0;
            c.C = a.Cin;
        }
        c.wt = net->wt + net->wt_off[l];
        c.bias = a.bias;
        c.relu = a.relu;
        c.out = a.out_bf16;
        switch (l) {                       // parts of the concatenation buffers
            case 1: c.out2 = net->cat[0]; c.ld2 = kCatC[0]; c.off2 = 0; c.pool = net->pool[0]; break;
            case 3: c.out2 = net->cat[1]; c.ld2 = kCatC[1]; c.off2 = 0; c.pool = net->pool[1]; break;
            case 5: c.out2 = net->cat[2]; c.ld2 = kCatC[2]; c.off2 = 0; c.pool = net->pool[2]; break;
            case 7: c.out2 = net->cat[2]; c.ld2 = kCatC[2]; c.off2 = 128; c.up2 = 1; break;
            case 9: c.out2 = net->cat[1]; c.ld2 = kCatC[1]; c.off2 = 64; c.up2 = 1; break;
            case 11: c.out2 = net->cat[0]; c.ld2 = kCatC[0]; c.off2 = 32; c.up2 = 1; break;
            default: break;
        }
    }
    NCU(mprnet::conv3x3_tma(c, net->d_err, net->st));
    mpr::count_launches(1, net->st);
    return MPR_OK;
}

// Reads and clears the kernels' error flag (synchronises the stream).
mpr_status check_err(mpr_net* net) {
    int h = 0;
    NCU(cudaMemcpyAsync(&h, net->d_err, sizeof(int), cudaMemcpyDeviceToHost, net->st));
    NCU(cudaStreamSynchronize(net->st));
    if (h) {
        NCU(cudaMemsetAsync(net->d_err, 0, sizeof(int), net->st));
        return nfail(net, MPR_ETIMEOUT, "a tensor-core convolution's barrier wait expired");
    }
    return MPR_OK;
}

// the input of layer l (the decoder's concatenations with upsampling)
ConvIn layer_in(const mpr_net* n, int l) {
    switch (l) {
        case 0: return ConvIn{n->in0, kIn, nullptr, 0, 0};
        case 2: return ConvIn{n->pool[0], 32, nullptr, 0, 0};
        case 4: return ConvIn{n->pool[1], 64, nullptr, 0, 0};
        case 6: return ConvIn{n->pool[2], 128, nullptr, 0, 0};
        case 8: return ConvIn{n->act[5], 128, n->act[7], 256, 1};
        case 10: return ConvIn{n->act[3], 64, n->act[9], 128, 1};
        case 12: return ConvIn{n->act[1], 32, n->act[11], 64, 1};
        default: return ConvIn{n->act[l - 1], kCin[l], nullptr, 0, 0};
    }
}

mpr_status input(mpr_net* net, const float* z, const uint8_t* mask, int B, int Hin, int Win, const double* zmin,
                 const double* zmax) {
    NCU(cudaMemcpyAsync(net->d_zr, zmin, sizeof(double) * B, cudaMemcpyDefault, net->st));
    NCU(cudaMemcpyAsync(net->d_zr + kMaxB, zmax, sizeof(double) * B, cudaMemcpyDefault, net->st));
    const long long P0 = (long long)net->B * net->H * net->W;
    k_input<<<grid1(P0), 256, 0, net->st>>>(z, mask, B, Hin, Win, net->H, net->W, net->stride, net->d_zr,
                                            net->d_zr + kMaxB, net->in0);
    mpr::count_launches(1, net->st);
    NCU(cudaGetLastError());
    return MPR_OK;
}

mpr_status forward(mpr_net* net) {
    cudaStream_t st = net->st;
    const int B = net->B, H = net->H, W = net->W;
    for (int l = 0; l < 14; ++l) {
        const int Hl = H >> kLevel[l], Wl = W >> kLevel[l];
        ConvArgs a;
        std::memset(&a, 0, sizeof a);
        a.in = layer_in(net, l);
        a.B = B; a.H = Hl; a.W = Wl;
        a.Cin = kCin[l];
        a.w = net->wb + net->off_w[l];
        a.Cout = kCout[l];
        a.bias = net->w + net->off_b[l];
        a.relu = 1;
        a.out_bf16 = net->act[l];
        const mpr_status cs = conv(net, a, l, false);
        if (cs != MPR_OK) return cs;
    }
    const long long P0 = (long long)B * H * W;
    k_head<<<grid1(P0), 256, 0, st>>>(net->act[13], P0, net->w + net->off_wh, net->w + net->off_bh, net->out2);
    mpr::count_launches(1, st);
    NCU(cudaGetLastError());
    return MPR_OK;
}

mpr_status backward(mpr_net* net) {
    cudaStream_t st = net->st;
    const int B = net->B, H = net->H, W = net->W;
    const long long P0 = (long long)B * H * W;
    k_head_bwd<<<std::min(grid1(P0), 1024), 256, 0, st>>>(net->act[13], net->dout2, P0, net->w + net->off_wh,
                                                          net->dact[13], net->g + net->off_wh, net->g + net->off_bh);
    mpr::count_launches(1, st);
    for (int l = 13; l >= 0; --l) {
        const int Hl = H >> kLevel[l], Wl = W >> kLevel[l];
        const long long P = (long long)B * Hl * Wl;
        const int Cin = kCin[l], Cout = kCout[l];
        k_gate<<<grid1(P * Cout), 256, 0, st>>>(net->dact[l], net->act[l], P * Cout, net->gb);
        k_bias_grad<<<dim3(64, (Cout + 31) / 32), 256, 0, st>>>(net->gb, P, Cout, net->g + net->off_b[l]);
        NCU(mprnet::conv3x3_wgrad(layer_in(net, l), B, Hl, Wl, Cin, net->gb, Cout, net->g + net->off_w[l], st));
        mpr::count_launches(3, st);
        if (l == 0) break;                                    // no gradient w.r.t. the network input
        ConvArgs a;
        std::memset(&a, 0, sizeof a);
        a.in = ConvIn{net->gb, Cout, nullptr, 0, 0};
        a.B = B; a.H = Hl; a.W = Wl;
        a.Cin = Cout;
        a.Cout = Cin;
        if (l == 2 || l == 4 || l == 6) {                      // input = pool(A)
            a.out_f32 = {net->dpool[l / 2 - 1], Cin, nullptr, 0, 0};
        } else if (l == 8 || l == 10 || l == 12) {             // input = [skip, up(low)]
            const int skip = l == 8 ? 5 : l == 10 ? 3 : 1;
            a.out_f32 = {net->dact[skip], kCout[skip], net->dup, Cin - kCout[skip], 0};
        } else {
            a.out_f32 = {net->dact[l - 1], Cin, nullptr, 0, 0};
        }
        const mpr_status cs = conv(net, a, l, true);
        if (cs != MPR_OK) return cs;
        if (l == 8 || l == 10 || l == 12) {
            const int low = l - 1;
            const int Cl = kCout[low];
            k_upsum<<<grid1((long long)B * (Hl / 2) * (Wl / 2) * Cl), 256, 0, st>>>(net->dup, B, Hl, Wl, Cl,
                                                                               net->dact[low]);
            mpr::count_launches(1, st);
        }
        if (l == 2 || l == 4 || l == 6) {                      // pool(A_{l-1}): A's gradient += pool adjoint
            const int A = l - 1;
            const int Ha = H >> kLevel[A], Wa = W >> kLevel[A];
            k_pool_bwd<<<grid1((long long)B * Ha * Wa * kCout[A]), 256, 0, st>>>(net->dpool[l / 2 - 1], B, Ha, Wa,
                                                                               kCout[A], net->dact[A]);
            mpr::count_launches(1, st);
        }
    }
    NCU(cudaGetLastError());
    return MPR_OK;
}

bool bad_shape(int B, int H, int W) { return B < 1 || B > kMaxB || H < 8 || W < 8 || H % 8 || W % 8; }

}  // namespace

// Warm start of the gap sites of B same-shape grids (z, mask: the first grid; grids
// contiguous), written into one or both lattice buffers through the entries' layout.
mpr_status mprnet_warmstart(mpr_net* net, const float* z, const uint8_t* mask, int B, int Hin, int Win,
                            const double* zmin, const double* zmax, const mpr::EntryDesc* d_ents, float2* lat0,
                            float2* lat1, cudaStream_t st) {
    if (!net) return MPR_EINVAL;
    if (B < 1 || B > kMaxB || Hin < 1 || Win < 1) return nfail(net, MPR_EINVAL, "bad warm-start batch");
    const cudaStream_t keep = net->st;
    net->st = st;
    const int S = net->stride;
    const int H = ((Hin + S - 1) / S + 7) / 8 * 8, W = ((Win + S - 1) / S + 7) / 8 * 8;
    mpr_status s = ensure_ws(net, B, H, W, false);
    if (s == MPR_OK) s = input(net, z, mask, B, Hin, Win, zmin, zmax);
    if (s == MPR_OK) s = forward(net);
    if (s == MPR_OK) {
        k_to_lattice<<<dim3(grid1((long long)Hin * Win), B), 256, 0, st>>>(net->out2, mask, d_ents, H, W, S, lat0,
                                                                           lat1);
        mpr::count_launches(1, st);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = nfail(net, MPR_ECUDA, std::string("k_to_lattice: ") + cudaGetErrorString(e));
    }
    if (s == MPR_OK) s = check_err(net);
    net->st = keep;
    return s;
}

const char* mprnet_error(const mpr_net* net) { return net ? net->err.c_str() : "null network"; }

extern "C" {

mpr_status mpr_net_create(mpr_net** out, uint64_t seed, void* cuda_stream) {
    return mpr_net_create_strided(out, seed, 1, cuda_stream);
}

int mpr_net_stride(const mpr_net* net) { return net ? net->stride : 0; }

mpr_status mpr_net_create_strided(mpr_net** out, uint64_t seed, int stride, void* cuda_stream) {
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    if (stride != 1 && stride != 2 && stride != 4 && stride != 8) return MPR_EINVAL;
    mpr_net* net = new mpr_net();
    net->stride = stride;
    net->st = (cudaStream_t)cuda_stream;
    long long off = 0;
    for (int l = 0; l < 14; ++l) {
        net->off_w[l] = off;
        off += 9LL * kCin[l] * kCout[l];
        net->off_b[l] = off;
        off += kCout[l];
    }
    net->off_wh = off;
    off += 2 * kHeadC;
    net->off_bh = off;
    off += 2;
    net->n_params = off;
    long long owt = 0, owtb = 0;
    for (int l = 0; l < 14; ++l) {
        net->wt_off[l] = owt;
        owt += (long long)kCout[l] * 9 * mprnet::tc_layer_kt(kCin[l], kCout[l]);
        net->wtb_off[l] = owtb;
        owtb += (long long)kCin[l] * 9 * mprnet::tc_layer_kt(kCout[l], kCin[l]);
    }
    std::vector<float> h((size_t)off, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 14; ++l) {                 // He initialisation (3 used input channels at l = 0)
        const int fan_in = 9 * (l == 0 ? 3 : kCin[l]);
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)fan_in));
        for (int t = 0; t < 9; ++t)
            for (int ci = 0; ci < kCin[l]; ++ci)
                for (int co = 0; co < kCout[l]; ++co) {
                    const float x = nd(rng);
                    if (l > 0 || ci < 3) h[(size_t)(net->off_w[l] + ((long long)t * kCin[l] + ci) * kCout[l] + co)] = x;
                }
    }
    std::normal_distribution<float> nh(0.f, std::sqrt(1.f / (float)kHeadC));
    for (int i = 0; i < 2 * kHeadC; ++i) h[(size_t)(net->off_wh + i)] = nh(rng);
    bool ok = cudaMalloc((void**)&net->w, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc((void**)&net->g, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc((void**)&net->m, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc((void**)&net->v, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc((void**)&net->wb, sizeof(bf16) * off) == cudaSuccess &&
              cudaMalloc((void**)&net->d_zr, sizeof(double) * 2 * kMaxB) == cudaSuccess &&
              cudaMalloc((void**)&net->d_loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&net->d_cnt, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc((void**)&net->wt, sizeof(bf16) * owt) == cudaSuccess &&
              cudaMalloc((void**)&net->wtb, sizeof(bf16) * owtb) == cudaSuccess &&
              cudaMalloc((void**)&net->d_err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mpr_net_free(net);
        return MPR_ENOMEM;
    }
    ok = cudaMemcpyAsync(net->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice, net->st) == cudaSuccess &&
         cudaMemsetAsync(net->g, 0, sizeof(float) * off, net->st) == cudaSuccess &&
         cudaMemsetAsync(net->m, 0, sizeof(float) * off, net->st) == cudaSuccess &&
         cudaMemsetAsync(net->v, 0, sizeof(float) * off, net->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(net->d_err, 0, sizeof(int), net->st) == cudaSuccess;
    if (ok) {
        k_to_bf16<<<grid1(off), 256, 0, net->st>>>(net->w, off, net->wb);
        mpr::count_launches(1, net->st);
        ok = refresh_wt(net) == MPR_OK && cudaStreamSynchronize(net->st) == cudaSuccess;
    }
    if (!ok) {
        mpr_net_free(net);
        return MPR_ECUDA;
    }
    *out = net;
    return MPR_OK;
}

void mpr_net_free(mpr_net* net) {
    if (!net) return;
    cudaStreamSynchronize(net->st);
    free_ws(net);
    cudaFree(net->w);
    cudaFree(net->g);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->wb);
    cudaFree(net->d_zr);
    cudaFree(net->d_loss);
    cudaFree(net->d_cnt);
    cudaFree(net->wt);
    cudaFree(net->wtb);
    cudaFree(net->d_err);
    delete net;
}

const char* mpr_net_last_error(const mpr_net* net) { return mprnet_error(net); }

long long mpr_net_num_params(const mpr_net* net) { return net ? net->n_params : 0; }

mpr_status mpr_net_get_params(mpr_net* net, float* params) {
    if (!net || !params) return MPR_EINVAL;
    NCU(cudaMemcpyAsync(params, net->w, sizeof(float) * net->n_params, cudaMemcpyDefault, net->st));
    NCU(cudaStreamSynchronize(net->st));
    return MPR_OK;
}

mpr_status mpr_net_set_params(mpr_net* net, const float* params) {
    if (!net || !params) return MPR_EINVAL;
    NCU(cudaMemcpyAsync(net->w, params, sizeof(float) * net->n_params, cudaMemcpyDefault, net->st));
    k_to_bf16<<<grid1(net->n_params), 256, 0, net->st>>>(net->w, net->n_params, net->wb);
    mpr::count_launches(1, net->st);
    {
        const mpr_status rs = refresh_wt(net);
        if (rs != MPR_OK) return rs;
    }
    NCU(cudaMemsetAsync(net->m, 0, sizeof(float) * net->n_params, net->st));
    NCU(cudaMemsetAsync(net->v, 0, sizeof(float) * net->n_params, net->st));
    NCU(cudaStreamSynchronize(net->st));
    net->adam_t = 0;
    return MPR_OK;
}

mpr_status mpr_net_get_grads(mpr_net* net, float* grads) {
    if (!net || !grads) return MPR_EINVAL;
    NCU(cudaMemcpyAsync(grads, net->g, sizeof(float) * net->n_params, cudaMemcpyDefault, net->st));
    return check_err(net);
}

mpr_status mpr_net_zero_grads(mpr_net* net) {
    if (!net) return MPR_EINVAL;
    NCU(cudaMemsetAsync(net->g, 0, sizeof(float) * net->n_params, net->st));
    return MPR_OK;
}

mpr_status mpr_net_loss_grad(mpr_net* net, const float* z, const uint8_t* mask, const float* phi_target,
                             const double* zmin, const double* zmax, int B, int H, int W, double* loss) {
    if (!net || !z || !mask || !phi_target || !zmin || !zmax || H % net->stride || W % net->stride ||
        bad_shape(B, H / net->stride, W / net->stride))
        return nfail(net, MPR_EINVAL, "B in [1, 4096] and H, W positive multiples of 8 x stride required");
    const int S = net->stride, Hf = H / S, Wf = W / S;
    mpr_status s = ensure_ws(net, B, Hf, Wf, true);
    if (s == MPR_OK) s = input(net, z, mask, B, H, W, zmin, zmax);
    if (s == MPR_OK) s = forward(net);
    if (s != MPR_OK) return s;
    const long long P0 = (long long)B * Hf * Wf, Pin = (long long)B * H * W;
    NCU(cudaMemsetAsync(net->d_loss, 0, sizeof(double), net->st));
    NCU(cudaMemsetAsync(net->d_cnt, 0, sizeof(unsigned long long), net->st));
    k_count_gaps<<<std::min(grid1(Pin), 1024), 256, 0, net->st>>>(mask, Pin, net->d_cnt);
    k_loss<<<grid1(P0), 256, 0, net->st>>>(net->out2, phi_target, mask, B, Hf, Wf, S, net->d_cnt, net->dout2,
                                           net->d_loss);
    mpr::count_launches(2, net->st);
    s = backward(net);
    if (s != MPR_OK) return s;
    if (loss) {
        NCU(cudaMemcpyAsync(loss, net->d_loss, sizeof(double), cudaMemcpyDefault, net->st));
        return check_err(net);
    }
    return MPR_OK;
}

mpr_status mpr_net_adam_step(mpr_net* net, float lr) {
    if (!net || !(lr >= 0.f)) return MPR_EINVAL;
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->adam_t), c2 = 1.f - std::pow(b2, (float)net->adam_t);
    k_adam<<<grid1(net->n_params), 256, 0, net->st>>>(net->w, net->g, net->m, net->v, net->n_params, lr, b1, b2,
                                                     1e-8f, c1, c2, net->wb);
    mpr::count_launches(1, net->st);
    NCU(cudaGetLastError());
    return refresh_wt(net);
}

mpr_status mpr_net_train_step(mpr_net* net, const float* z, const uint8_t* mask, const float* phi_target,
                              const double* zmin, const double* zmax, int B, int H, int W, float lr, double* loss) {
    mpr_status s = mpr_net_loss_grad(net, z, mask, phi_target, zmin, zmax, B, H, W, loss);
    return s != MPR_OK ? s : mpr_net_adam_step(net, lr);
}

mpr_status mpr_net_forward(mpr_net* net, const float* z, const uint8_t* mask, const double* zmin,
                           const double* zmax, int B, int H, int W, float* uv) {
    if (!net || !z || !mask || !zmin || !zmax || !uv || H % net->stride || W % net->stride ||
        bad_shape(B, H / net->stride, W / net->stride))
        return nfail(net, MPR_EINVAL, "B in [1, 4096] and H, W positive multiples of 8 x stride required");
    const int Hf = H / net->stride, Wf = W / net->stride;
    mpr_status s = ensure_ws(net, B, Hf, Wf, false);
    if (s == MPR_OK) s = input(net, z, mask, B, H, W, zmin, zmax);
    if (s == MPR_OK) s = forward(net);
    if (s != MPR_OK) return s;
    NCU(cudaMemcpyAsync(uv, net->out2, sizeof(float) * 2 * (size_t)B * Hf * Wf, cudaMemcpyDefault, net->st));
    return check_err(net);
}

// Test support: a copy of one of the network's internal tensors (layer-by-layer checks).
mpr_status mpr_net_tensor(mpr_net* net, int kind, int index, void* out, long long count) {
    if (!net || !out) return MPR_EINVAL;
    const long long P0 = (long long)net->B * net->H * net->W;
    const void* src = nullptr;
    size_t elem = 0;
    long long n = 0;
    switch (kind) {
        case MPR_NET_T_INPUT:
            src = net->in0; elem = sizeof(bf16); n = P0 * kIn;
            break;
        case MPR_NET_T_ACT:
            if (index < 0 || index >= 14) break;
            src = net->act[index]; elem = sizeof(bf16); n = (P0 >> (2 * kLevel[index])) * kCout[index];
            break;
        case MPR_NET_T_POOL:
            if (index < 0 || index >= 3) break;
            src = net->pool[index]; elem = sizeof(bf16); n = (P0 >> (2 * (index + 1))) * kCout[2 * index + 1];
            break;
        case MPR_NET_T_DACT:
            if (index < 0 || index >= 14 || !net->train) break;
            src = net->dact[index]; elem = sizeof(float); n = (P0 >> (2 * kLevel[index])) * kCout[index];
            break;
        case MPR_NET_T_OUT:
            src = net->out2; elem = sizeof(float); n = P0 * 2;
            break;
        default:
            break;
    }
    if (!src || P0 == 0) return nfail(net, MPR_ESTATE, "no such tensor after the last call");
    if (count != n) return nfail(net, MPR_EINVAL, "element count of the tensor differs");
    NCU(cudaMemcpyAsync(out, src, (size_t)n * elem, cudaMemcpyDefault, net->st));
    NCU(cudaStreamSynchronize(net->st));
    return MPR_OK;
}

// Test support: the library's own convolution kernels on caller buffers.
mpr_status mpr_net_conv3x3(const uint16_t* in, int B, int H, int W, int Cin, const uint16_t* w, const float* bias,
                           int Cout, int relu, uint16_t* out, void* cuda_stream) {
    if (!in || !w || !out || B < 1 || H < 1 || W < 1 || Cin < 32 || Cout < 32 || Cin % 32 || Cout % 32 ||
        !mprnet::tc_supported(Cin, Cout))
        return MPR_EINVAL;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    bf16* wt = nullptr;
    int* err = nullptr;
    int herr = 0;
    mprnet::TcConv c;
    std::memset(&c, 0, sizeof c);
    c.in = (const bf16*)in;
    c.C = Cin;
    c.B = B; c.H = H; c.W = W;
    c.N = Cout;
    c.bias = bias;
    c.relu = relu;
    c.out = (bf16*)out;
    cudaError_t e = cudaMalloc((void**)&wt, sizeof(bf16) * (size_t)Cout * 9 * mprnet::tc_layer_kt(Cin, Cout));
    if (e == cudaSuccess) e = cudaMalloc((void**)&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = mprnet::tc_weights((const bf16*)w, Cin, Cout, 0, wt, st);
    c.wt = wt;
    if (e == cudaSuccess) e = mprnet::conv3x3_tma(c, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mpr::count_launches(2, st);
    cudaFree(wt);
    cudaFree(err);
    return e != cudaSuccess ? MPR_ECUDA : herr ? MPR_ETIMEOUT : MPR_OK;
}

mpr_status mpr_net_conv3x3_bwd(const uint16_t* in, const uint16_t* gout, int B, int H, int W, int Cin,
                               const uint16_t* w, int Cout, float* din, float* dw, uint16_t* w_scratch,
                               void* cuda_stream) {
    if (!in || !gout || !w || !din || !dw || !w_scratch || B < 1 || H < 1 || W < 1 || Cin < 32 || Cout < 32 ||
        Cin % 32 || Cout % 32 || !mprnet::tc_supported(Cout, Cin))
        return MPR_EINVAL;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const ConvIn ci{(const bf16*)in, Cin, nullptr, 0, 0};
    if (mprnet::conv3x3_wgrad(ci, B, H, W, Cin, (const bf16*)gout, Cout, dw, st) != cudaSuccess) return MPR_ECUDA;
    bf16* wt = nullptr;
    int* err = nullptr;
    int herr = 0;
    mprnet::TcConv c;
    std::memset(&c, 0, sizeof c);
    c.in = (const bf16*)gout;
    c.C = Cout;
    c.B = B; c.H = H; c.W = W;
    c.N = Cin;
    c.of = {din, Cin, nullptr, 0, 0};
    cudaError_t e = cudaMalloc((void**)&wt, sizeof(bf16) * (size_t)Cin * 9 * mprnet::tc_layer_kt(Cout, Cin));
    if (e == cudaSuccess) e = cudaMalloc((void**)&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = mprnet::tc_weights((const bf16*)w, Cin, Cout, 1, wt, st);
    c.wt = wt;
    if (e == cudaSuccess) e = mprnet::conv3x3_tma(c, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mpr::count_launches(3, st);
    cudaFree(wt);
    cudaFree(err);
    return e != cudaSuccess ? MPR_ECUDA : herr ? MPR_ETIMEOUT : MPR_OK;
}

}  // extern "C"
