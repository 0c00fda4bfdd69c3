// mpr_internal.cuh -- device data layout, helpers and launcher declarations of libmpr.
//
// Lattice layout (one "entry" = one W x H grid with its own chain):
//   The checkerboard of Sect. 3.3 splits the grid into colour 0 ((x+y) even) and
//   colour 1.  Each colour is packed into a plane of float2 unit vectors
//   (cos(q phi), sin(q phi)), row y, column j = x >> 1, with one padding row above
//   and below and a padding column on the left.  Padding slots hold (0, 0), so an
//   out-of-grid neighbour contributes nothing to the local field: no boundary
//   branches in the sweep.  For q = 1/2 the state space phi in [0, 2pi) is the
//   upper half circle sin(q phi) >= 0.
//   Padded index of (y, j): (y + 1) * pitch + (j + 1).  For a site of colour c in
//   row y, s = c ^ (y & 1) gives x = 2j + s and its neighbours in the other plane at
//   k - pitch, k + pitch, k - 1 + s, k + s.
//   Gap sites of each colour are listed row-major as (y << 16) | j.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpr {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kSweepThreads = 256;
constexpr int kSweepItems = 2;                    // gap sites per thread per launch chunk
constexpr uint32_t kInitSweep = 0xFFFFFFFFu;      // Philox sweep word of the initial state

struct EntryDesc {            // immutable during a run
    int W, H, pitch, _pad0;
    long long plane[2];       // float2 offset of plane c's padded origin
    long long gbase[2];       // offset of colour c's gap list
    int ngap[2];
    uint32_t chain;           // realization id (Philox counter word 2)
    int P;                    // ngap[0] + ngap[1]
    double ngp;               // number of nearest-neighbour pairs, W(H-1) + H(W-1)
    long long site0;          // offset of the grid in concatenated [H][W] buffers
    int blk0[2];              // first sweep block of this entry in colour c's work list
    int nblk[2];              // number of sweep blocks of this entry per colour
};

struct Ctl {                  // mutable per-entry control state (Algorithm 2)
    double T;                 // temperature
    double a;                 // window factor
    double k;                 // last slope of the specific energy
    double H;                 // energy tracked by the sweeps
    double A_last, e_last;
    double esum;              // sum of e over sampling sweeps (table mode)
    int i;                    // relaxation counter
    int stop;                 // relaxation finished (or nothing to do)
    int converged;
    uint32_t sweep;           // global sweep counter (Philox counter word 1)
    int nsamp;
    int status;               // 0, or a device-side error code
};

struct Part {                 // one sweep block's energy change and acceptance count
    double dH;
    unsigned nacc;
    unsigned _pad;
};

struct BlockWork {            // one sweep block: entry and first gap index of its chunk
    int entry;
    int first;
};

struct SweepArgs {
    const EntryDesc* ents;
    float2* lat;
    const uint32_t* gaps;
    float* acc;               // per gap site sum of q*phi (prediction), or nullptr
    Ctl* ctl;
    Part* part[2];            // per colour, one per sweep block
    const BlockWork* work[2]; // per colour
    int nblk[2];
    int use_ctl_a;            // window from Ctl::a (relaxation) or fixed
    float half_qd_fixed;      // q * pi / a for the fixed window
    int skip_stopped;         // skip entries whose relaxation has ended
    int or_on;
    uint32_t key0, key1;      // Philox key
};

// Control-kernel modes.
enum { CTL_RELAX = 0, CTL_FIXED = 1, CTL_SAMPLE = 2 };

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
    // Philox4x32-10, Salmon et al. (SC'11): 10 rounds, Weyl key schedule.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u24f(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

// sin and cos of |x| <= pi/4 by their Taylor series (coefficients 1/n!), to degree 9
// and 10: truncation error below 2e-9, far under FP32 rounding.
__device__ __forceinline__ void sincos_quarter(float x, float* s, float* c) {
    const float x2 = x * x;
    float ps = 2.7557319e-6f;                 //  1/9!
    ps = fmaf(ps, x2, -1.9841270e-4f);        // -1/7!
    ps = fmaf(ps, x2, 8.3333333e-3f);         //  1/5!
    ps = fmaf(ps, x2, -1.6666667e-1f);        // -1/3!
    *s = fmaf(ps * x2, x, x);
    float pc = -2.7557319e-7f;                // -1/10!
    pc = fmaf(pc, x2, 2.4801587e-5f);         //  1/8!
    pc = fmaf(pc, x2, -1.3888889e-3f);        // -1/6!
    pc = fmaf(pc, x2, 4.1666667e-2f);         //  1/4!
    pc = fmaf(pc, x2, -0.5f);                 // -1/2!
    *c = fmaf(pc, x2, 1.0f);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned warp_sum(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Kernel launches enqueued by the library (direct launches and graph replays); launches
// recorded into a graph under capture are counted when the graph is replayed instead.
void count_launches(unsigned long long n, cudaStream_t st);

// ---------------------------------------------------------------- launchers
// init (mpr_init.cu)
cudaError_t launch_minmax(const float* z, const uint8_t* mask, long long n, unsigned* keys,
                          unsigned long long* nsamples, cudaStream_t st);
cudaError_t launch_pack(const EntryDesc* e_host, const float* z, const uint8_t* mask,
                        double zmin, double scale, float2* lat, uint32_t key0, uint32_t key1,
                        int all_free, cudaStream_t st);
cudaError_t launch_gap_count(const EntryDesc* e_host, const uint8_t* mask, int all_free,
                             int* row_counts, cudaStream_t st);
cudaError_t launch_scan_rows(int* row_counts, int nrows, int narrays, int* totals,
                             cudaStream_t st);
cudaError_t launch_gap_scatter(const EntryDesc* e_host, const uint8_t* mask, int all_free,
                               const int* row_offsets, uint32_t* gaps, cudaStream_t st);
// Eq. 4 partial sums: per block (sum of cosines, pair count) into part[block] (grid <= 1024).
cudaError_t launch_sample_energy(const EntryDesc* e_host, const float* z, const uint8_t* mask,
                                 double scale, double q, double* part_sum,
                                 unsigned long long* part_cnt, int* nparts, cudaStream_t st);
cudaError_t launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, size_t n,
                          cudaStream_t st);

// sweeps (mpr_sweep.cu)
cudaError_t launch_half_sweep(const SweepArgs& a, int color, int trig, cudaStream_t st);
cudaError_t launch_control(Ctl* ctl, Part* const part[2], const EntryDesc* ents, int n_ent,
                           int mode, double A_targ, double k_a, int n_f, int n_fit, int i_max,
                           double* ehist, int ehist_stride, int* active, cudaStream_t st);
// Eq. 2 of one grid: per-block partials then a fixed-order sum into *out (deterministic).
cudaError_t launch_energy(const EntryDesc* e_host, const float2* lat, double* scratch,
                          int scratch_len, double* out, cudaStream_t st);
cudaError_t launch_sum(const double* v, int n, double* out, cudaStream_t st);
cudaError_t launch_set_tracked_energy(Ctl* ctl, const double* H, int n_ent, cudaStream_t st);
cudaError_t launch_predict_out(const EntryDesc* e_host, const float2* lat, const uint32_t* gaps,
                               const float* acc, int M, double q, double zmin, double zmax,
                               float* zhat, cudaStream_t st);
cudaError_t launch_get_state(const EntryDesc* e_host, const float2* lat, float* phi,
                             cudaStream_t st);
cudaError_t launch_set_state(const EntryDesc* e_host, float2* lat, const uint32_t* gaps,
                             const float* phi, cudaStream_t st);

}  // namespace mpr
