// mpr_static.cu -- an entry point that never allocates memory.
//
// mpr_sample_energy_static computes the same quantity that mpr_init computes on the way
// (the sample specific energy e_s of the data and the number of sample pairs) for callers
// that may not allocate device memory at all: code that runs inside an application which
// owns the device memory through its own pool or budget and forbids cudaMalloc/cudaFree
// from libraries, or latency-critical loops where an allocation or a free would stall or
// synchronise the device.  Every word of scratch memory it needs lives in one file-scope
// device array, reserved on a GPU when the library's device code is loaded there (with
// CUDA's lazy module loading, at the library's first use on that device) and kept until
// the process exits.  The caller passes device-resident inputs and host outputs.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "../../include/mpr.h"
#include "mpr_internal.cuh"

namespace {

constexpr int kThreads = 256;

// Layout of the static scratch area (all offsets 256-byte aligned):
//   [0, 256)          : unsigned keys[2] (z_min/z_max keys), unsigned long long n_samples,
//                       double scale, int status, double e_s, unsigned long long n_pairs
//   [256, ...)        : double row_sum[MPR_STATIC_MAX_ROWS]
//   then              : unsigned long long row_cnt[MPR_STATIC_MAX_ROWS]
struct Head {
    unsigned keys[2];
    unsigned long long n_samples;
    double scale;
    int status;
    int _pad;
    double e_s;
    unsigned long long n_pairs;
};
constexpr size_t kHeadBytes = 256;
constexpr size_t kRowSumOff = kHeadBytes;
constexpr size_t kRowCntOff = kRowSumOff + sizeof(double) * MPR_STATIC_MAX_ROWS;
constexpr size_t kScratchBytes = kRowCntOff + sizeof(unsigned long long) * MPR_STATIC_MAX_ROWS;
static_assert(sizeof(Head) <= kHeadBytes, "scratch head too large");

// The scratch itself.  Host code must not use this name as an address (on the host it is
// only a stand-in for the device symbol); it obtains the device address once per device
// with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

__device__ __forceinline__ double key_to_double(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return (double)__uint_as_float(b);
}

// Resets the fields that later kernels accumulate into (min/max keys, sample count).
__global__ void k_static_clear(unsigned char* s) {
    Head* h = reinterpret_cast<Head*>(s);
    h->keys[0] = 0xFFFFFFFFu;
    h->keys[1] = 0u;
    h->n_samples = 0ull;
    h->status = 0;
    h->scale = 0.0;
    h->e_s = 0.0;
    h->n_pairs = 0ull;
}

// Eq. 1 needs z_min < z_max and at least two samples; scale = 2 pi / (z_max - z_min).
__global__ void k_static_scale(unsigned char* s) {
    Head* h = reinterpret_cast<Head*>(s);
    if (h->n_samples < 2ull) { h->status = MPR_ENODATA; return; }
    const double zmin = key_to_double(h->keys[0]), zmax = key_to_double(h->keys[1]);
    if (!(zmax > zmin) || isinf(zmin) || isinf(zmax)) { h->status = MPR_ENODATA; return; }
    h->scale = mpr::kTwoPi / (zmax - zmin);
}

// Eq. 4, one warp per row: sum of cos(q (phi_i - phi_j)) over the sample pairs whose
// first site lies in the row (partner to the right or below), and their number.
__global__ void k_static_rows(const float* __restrict__ z, const uint8_t* __restrict__ mask,
                              int W, int H, double q, unsigned char* s) {
    const Head* h = reinterpret_cast<const Head*>(s);
    if (h->status) return;
    const double scale = h->scale;
    double* row_sum = reinterpret_cast<double*>(s + kRowSumOff);
    unsigned long long* row_cnt = reinterpret_cast<unsigned long long*>(s + kRowCntOff);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= H) return;
    const int y = warp;
    double acc = 0.0;
    unsigned cnt = 0;
    for (int x = lane; x < W; x += 32) {
        const long long i = (long long)y * W + x;
        if (!mask[i]) continue;
        const double zi = (double)z[i];
        if (x + 1 < W && mask[i + 1]) {
            acc += (double)cosf((float)(q * ((zi - (double)z[i + 1]) * scale)));
            ++cnt;
        }
        if (y + 1 < H && mask[i + W]) {
            acc += (double)cosf((float)(q * ((zi - (double)z[i + W]) * scale)));
            ++cnt;
        }
    }
    acc = mpr::warp_sum(acc);
    cnt = mpr::warp_sum(cnt);
    if (lane == 0) {
        row_sum[y] = acc;
        row_cnt[y] = cnt;
    }
}

// Adds the row partials in row order (one thread: the order is fixed).
__global__ void k_static_finish(int H, unsigned char* s) {
    Head* h = reinterpret_cast<Head*>(s);
    if (h->status) return;
    const double* row_sum = reinterpret_cast<const double*>(s + kRowSumOff);
    const unsigned long long* row_cnt = reinterpret_cast<const unsigned long long*>(s + kRowCntOff);
    double t = 0.0;
    unsigned long long c = 0;
    for (int y = 0; y < H; ++y) {
        t += row_sum[y];
        c += row_cnt[y];
    }
    h->n_pairs = c;
    h->e_s = c ? -t / (double)c : 0.0;
}

// Device address of the scratch, looked up once per device.  Two host threads making
// their first call on one device may both look it up; they store the same address, and the
// atomic slots make that a benign race rather than a data race.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_scratch_ptr[kMaxDevices];

cudaError_t scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned char* ptr = g_scratch_ptr[dev].load(std::memory_order_relaxed);
    if (!ptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        ptr = static_cast<unsigned char*>(p);
        g_scratch_ptr[dev].store(ptr, std::memory_order_relaxed);
    }
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" mpr_status mpr_sample_energy_static(const float* z, const uint8_t* mask, int W, int H,
                                               double q, double* e_s, long long* n_pairs,
                                               void* cuda_stream) {
    // the same coupling range as mpr_init: q in (0, 1/2]
    if (!z || !mask || !e_s || !n_pairs || W < 1 || H < 1 || !(q > 0.0 && q <= 0.5)) return MPR_EINVAL;
    if (H > MPR_STATIC_MAX_ROWS) return MPR_EINVAL;       // more rows than scratch slots
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* s = nullptr;
    if (scratch_for_current_device(&s) != cudaSuccess) {
        cudaGetLastError();
        return MPR_ECUDA;
    }
    const long long n = (long long)W * H;
    Head* h = reinterpret_cast<Head*>(s);
    k_static_clear<<<1, 1, 0, st>>>(s);
    mpr::count_launches(1, st);
    if (mpr::launch_minmax(z, mask, n, h->keys, &h->n_samples, st) != cudaSuccess) return MPR_ECUDA;
    k_static_scale<<<1, 1, 0, st>>>(s);
    k_static_rows<<<(H * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(z, mask, W, H, q, s);
    k_static_finish<<<1, 1, 0, st>>>(H, s);
    mpr::count_launches(3, st);
    if (cudaGetLastError() != cudaSuccess) return MPR_ECUDA;
    Head out;
    if (cudaMemcpyAsync(&out, h, sizeof(Head), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return MPR_ECUDA;
    }
    if (out.status) return (mpr_status)out.status;
    *e_s = out.e_s;
    *n_pairs = (long long)out.n_pairs;
    return out.n_pairs ? MPR_OK : MPR_ENOPAIRS;
}
