// mpr_init.cu -- set-up kernels: Eq. 1 map, lattice packing, gap lists, Eq. 4.
//
// These run once per grid (Algorithm 2, steps 2-4.1); the hot path is in mpr_sweep.cu.
#include <algorithm>

#include "mpr_internal.cuh"

namespace mpr {
namespace {

constexpr int kThreads = 256;

// Order-preserving map of a float to an unsigned key (for atomicMin/atomicMax).
__device__ __forceinline__ unsigned float_key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// z_min, z_max and the number of samples over one grid (Eq. 1 needs the extremes); block
// bid of nb (integer keys and counts: any partition gives the same result).
__device__ __forceinline__ void minmax_body(const float* __restrict__ z, const uint8_t* __restrict__ mask,
                                            long long n, unsigned* keys, unsigned long long* nsamples,
                                            int bid, int nb) {
    unsigned kmin = 0xFFFFFFFFu, kmax = 0u, cnt = 0u;
    for (long long i = bid * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) {
        if (mask[i]) {
            const unsigned k = float_key(z[i]);
            kmin = min(kmin, k);
            kmax = max(kmax, k);
            ++cnt;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) {
        if (cnt) {
            atomicMin(&keys[0], kmin);
            atomicMax(&keys[1], kmax);
            atomicAdd(nsamples, (unsigned long long)cnt);
        }
    }
}
__global__ void k_minmax(const float* __restrict__ z, const uint8_t* __restrict__ mask,
                         long long n, unsigned* keys, unsigned long long* nsamples) {
    minmax_body(z, mask, n, keys, nsamples, blockIdx.x, gridDim.x);
}
__global__ void k_minmax_batch(const SetupRec* __restrict__ recs, unsigned* keys, unsigned long long* nsamples) {
    const SetupRec& r = recs[blockIdx.y];
    minmax_body(r.z, r.mask, r.n, keys + 2 * blockIdx.y, nsamples + blockIdx.y, blockIdx.x, gridDim.x);
}

// Packs one grid into its two colour planes.  Samples get the Eq. 1 angle; gap sites
// get phi = 2 pi u with u from the Philox stream {site, 0xFFFFFFFF, chain, 0}
// (Algorithm 2, step 2.2).  Stored as (cos(q phi), sin(q phi)).
// FP32 lattice: theta rounded to float, then sincosf; FP64 lattice: sincos of the double theta.
// sin is clamped at 0: theta = pi rounds above pi in FP32; stay on the upper half circle.
__device__ __forceinline__ void unit_at(double theta, float2& v) {
    float s, co;
    sincosf((float)theta, &s, &co);
    v = make_float2(co, fmaxf(s, 0.0f));
}
__device__ __forceinline__ void unit_at(double theta, double2& v) {
    double s, co;
    sincos(theta, &s, &co);
    v = make_double2(co, fmax(s, 0.0));
}

template <typename V>
__device__ __forceinline__ void pack_body(const EntryDesc& e, const float* __restrict__ z,
                                          const uint8_t* __restrict__ mask, double zmin, double scale,
                                          V* __restrict__ lat, uint32_t key0, uint32_t key1, int all_free,
                                          int bid, int nb) {
    const long long n = (long long)e.W * e.H;
    for (long long i = bid * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) {
        const int y = (int)(i / e.W), x = (int)(i - (long long)y * e.W);
        const int c = (x + y) & 1;
        double theta;
        if (!all_free && mask[i]) {
            const double phi = ((double)z[i] - zmin) * scale;          // Eq. 1
            theta = e.q * phi;
        } else {
            const uint32_t site = (uint32_t)i + e.row_off * (uint32_t)e.W;   // in the whole grid
            const uint4 r = philox10(make_uint4(site, kInitSweep, e.chain, 0u), key0, key1);
            theta = kTwoPi * e.q * (double)u24f(r.x);                  // q * 2 pi u
        }
        const long long base = c ? e.plane[1] : e.plane[0];
        unit_at(theta, lat[base + (long long)(y + 1) * e.pitch + (x >> 1) + kPadL]);
    }
}
template <typename V>
__global__ void k_pack(EntryDesc e, const float* __restrict__ z, const uint8_t* __restrict__ mask,
                       double zmin, double scale, V* __restrict__ lat, uint32_t key0,
                       uint32_t key1, int all_free) {
    pack_body(e, z, mask, zmin, scale, lat, key0, key1, all_free, blockIdx.x, gridDim.x);
}
template <typename V>
__global__ void k_pack_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                             V* __restrict__ lat, uint32_t key0, uint32_t key1, int all_free) {
    const EntryDesc e = ents[blockIdx.y];
    const SetupRec& r = recs[blockIdx.y];
    pack_body(e, r.z, r.mask, r.zmin, r.scale, lat, key0, key1, all_free, blockIdx.x, gridDim.x);
}

// Number of gap sites of each colour in each row: row_counts[c * H + y].  One warp per row.
__device__ __forceinline__ void gap_count_body(const EntryDesc& e, const uint8_t* __restrict__ mask,
                                               int all_free, int* __restrict__ row_counts) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= e.H) return;
    const int y = warp;
    int cnt[2] = {0, 0};
    for (int x0 = 0; x0 < e.W; x0 += 32) {
        const int x = x0 + lane;
        const bool gap = x < e.W && (all_free || !mask[(long long)y * e.W + x]);
        const unsigned b = __ballot_sync(0xffffffffu, gap);
        // lanes with (x + y) even are colour 0
        const unsigned even = ((x0 + y) & 1) ? 0xAAAAAAAAu : 0x55555555u;
        cnt[0] += __popc(b & even);
        cnt[1] += __popc(b & ~even);
    }
    if (lane == 0) {
        row_counts[y] = cnt[0];
        row_counts[e.H + y] = cnt[1];
    }
}
__global__ void k_gap_count(EntryDesc e, const uint8_t* __restrict__ mask, int all_free,
                            int* __restrict__ row_counts) {
    gap_count_body(e, mask, all_free, row_counts);
}
__global__ void k_gap_count_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                                  int all_free, int* __restrict__ row_counts) {
    const EntryDesc e = ents[blockIdx.y];
    gap_count_body(e, recs[blockIdx.y].mask, all_free, row_counts + recs[blockIdx.y].roff);
}

// In-place exclusive scan of narrays consecutive arrays of nrows ints (one block each);
// totals[a] receives the sum of array a.
__device__ __forceinline__ void scan_body(int* __restrict__ a, int nrows, int* __restrict__ total) {
    __shared__ int part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (nrows + nt - 1) / nt;
    const int b = min(nrows, t * chunk), e = min(nrows, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < nt; o <<= 1) {            // Hillis-Steele inclusive scan
        const int add = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    int run = t ? part[t - 1] : 0;
    for (int i = b; i < e; ++i) {
        const int c = a[i];
        a[i] = run;
        run += c;
    }
    if (t == nt - 1) *total = part[t];
}
__global__ void k_scan_rows(int* __restrict__ v, int nrows, int* __restrict__ totals) {
    scan_body(v + (long long)blockIdx.x * nrows, nrows, totals + blockIdx.x);
}
// array 2 i + c of the batch: colour c of grid i
__global__ void k_scan_rows_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                                  int* __restrict__ v, int* __restrict__ totals) {
    const int i = blockIdx.x >> 1, c = blockIdx.x & 1, H = ents[i].H;
    scan_body(v + recs[i].roff + (long long)c * H, H, totals + blockIdx.x);
}

// Writes the gap lists, row-major, as (y << 16) | j.  One warp per row.
__device__ __forceinline__ void gap_scatter_body(const EntryDesc& e, const uint8_t* __restrict__ mask,
                                                 int all_free, const int* __restrict__ row_off,
                                                 uint32_t* __restrict__ gaps) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= e.H) return;
    const int y = warp;
    int pos0 = row_off[y], pos1 = row_off[e.H + y];
    const unsigned lt = (1u << lane) - 1u;
    for (int x0 = 0; x0 < e.W; x0 += 32) {
        const int x = x0 + lane;
        const bool gap = x < e.W && (all_free || !mask[(long long)y * e.W + x]);
        const unsigned b = __ballot_sync(0xffffffffu, gap);
        const unsigned even = ((x0 + y) & 1) ? 0xAAAAAAAAu : 0x55555555u;
        const int c = (x + y) & 1;
        const unsigned mine = c ? (b & ~even) : (b & even);
        if (gap) {
            const long long at = c ? e.gbase[1] + pos1 : e.gbase[0] + pos0;
            gaps[at + __popc(mine & lt)] = ((uint32_t)y << 16) | (uint32_t)(x >> 1);
        }
        pos0 += __popc(b & even);
        pos1 += __popc(b & ~even);
    }
}
__global__ void k_gap_scatter(EntryDesc e, const uint8_t* __restrict__ mask, int all_free,
                              const int* __restrict__ row_off, uint32_t* __restrict__ gaps) {
    gap_scatter_body(e, mask, all_free, row_off, gaps);
}
__global__ void k_gap_scatter_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                                    int all_free, const int* __restrict__ row_off, uint32_t* __restrict__ gaps) {
    const EntryDesc e = ents[blockIdx.y];
    gap_scatter_body(e, recs[blockIdx.y].mask, all_free, row_off + recs[blockIdx.y].roff, gaps);
}

// Eq. 4: sum over nearest-neighbour sample pairs (each once: right and down partner) of
// cos(q (phi_i - phi_j)), with phi_i - phi_j = (z_i - z_j) * 2pi / (z_max - z_min).
// Each block writes its partial sums; they are added in block order afterwards.
__device__ __forceinline__ void sample_energy_body(const EntryDesc& e, const float* __restrict__ z,
                                                   const uint8_t* __restrict__ mask, float qs,
                                                   double* part_sum, unsigned long long* part_cnt, int y_end,
                                                   int bid, int nb) {
    // Eq. 4 pairs (each unordered sample pair once: right and down neighbours), rows
    // block-strided and columns thread-strided (no index division).  The cosine argument
    // q (z_i - z_j) 2 pi / (z_max - z_min) is formed in FP32 (one rounding of the scale,
    // one of the difference, one of the product: ~1e-7 rad), each row's terms are summed
    // in FP32 and the rows in FP64.
    __shared__ double ssum[kThreads / 32];
    __shared__ unsigned long long scnt[kThreads / 32];
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int y = bid; y < y_end; y += nb) {
        const float* __restrict__ zr = z + (long long)y * e.W;
        const uint8_t* __restrict__ mr = mask + (long long)y * e.W;
        const bool down = y + 1 < e.H;
        float row = 0.0f;
        unsigned rc = 0;
        for (int x = threadIdx.x; x < e.W; x += blockDim.x) {
            if (!mr[x]) continue;
            const float zi = zr[x];
            if (x + 1 < e.W && mr[x + 1]) {
                row += cosf(qs * (zi - zr[x + 1]));
                ++rc;
            }
            if (down && mr[x + e.W]) {
                row += cosf(qs * (zi - zr[x + e.W]));
                ++rc;
            }
        }
        acc += (double)row;
        cnt += rc;
    }
    acc = warp_sum(acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) {
        ssum[threadIdx.x >> 5] = acc;
        scnt[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < kThreads / 32; ++w) { t += ssum[w]; c += scnt[w]; }
        part_sum[bid] = t;
        part_cnt[bid] = c;
    }
}
__global__ void k_sample_energy(EntryDesc e, const float* __restrict__ z,
                                const uint8_t* __restrict__ mask, float qs,
                                double* part_sum, unsigned long long* part_cnt, int y_end) {
    sample_energy_body(e, z, mask, qs, part_sum, part_cnt, y_end, blockIdx.x, gridDim.x);
}
// grid i: its own partial count (blocks beyond it return), the same rows per block as the
// single-grid launch
__global__ void k_sample_energy_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                                      double q, double* part_sum, unsigned long long* part_cnt) {
    const SetupRec& r = recs[blockIdx.y];
    if ((int)blockIdx.x >= r.nparts) return;
    const EntryDesc e = ents[blockIdx.y];
    sample_energy_body(e, r.z, r.mask, (float)(q * r.scale), part_sum + r.poff, part_cnt + r.poff, e.H,
                       blockIdx.x, r.nparts);
}

// Eq. 4 in FP64 (MPR_PREC_F64): the same pairs and partials, the cosine argument
// q (z_i - z_j) 2 pi / (z_max - z_min) and every sum in double.
__device__ __forceinline__ void sample_energy64_body(const EntryDesc& e, const float* __restrict__ z,
                                                     const uint8_t* __restrict__ mask, double qs,
                                                     double* part_sum, unsigned long long* part_cnt, int y_end,
                                                     int bid, int nb) {
    __shared__ double ssum[kThreads / 32];
    __shared__ unsigned long long scnt[kThreads / 32];
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int y = bid; y < y_end; y += nb) {
        const float* __restrict__ zr = z + (long long)y * e.W;
        const uint8_t* __restrict__ mr = mask + (long long)y * e.W;
        const bool down = y + 1 < e.H;
        for (int x = threadIdx.x; x < e.W; x += blockDim.x) {
            if (!mr[x]) continue;
            const double zi = (double)zr[x];
            if (x + 1 < e.W && mr[x + 1]) {
                acc += cos(qs * (zi - (double)zr[x + 1]));
                ++cnt;
            }
            if (down && mr[x + e.W]) {
                acc += cos(qs * (zi - (double)zr[x + e.W]));
                ++cnt;
            }
        }
    }
    acc = warp_sum(acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) {
        ssum[threadIdx.x >> 5] = acc;
        scnt[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c = 0;
        for (int w = 0; w < kThreads / 32; ++w) { t += ssum[w]; c += scnt[w]; }
        part_sum[bid] = t;
        part_cnt[bid] = c;
    }
}
__global__ void k_sample_energy64(EntryDesc e, const float* __restrict__ z,
                                  const uint8_t* __restrict__ mask, double qs,
                                  double* part_sum, unsigned long long* part_cnt, int y_end) {
    sample_energy64_body(e, z, mask, qs, part_sum, part_cnt, y_end, blockIdx.x, gridDim.x);
}
__global__ void k_sample_energy64_batch(const EntryDesc* __restrict__ ents, const SetupRec* __restrict__ recs,
                                        double q, double* part_sum, unsigned long long* part_cnt) {
    const SetupRec& r = recs[blockIdx.y];
    if ((int)blockIdx.x >= r.nparts) return;
    const EntryDesc e = ents[blockIdx.y];
    sample_energy64_body(e, r.z, r.mask, q * r.scale, part_sum + r.poff, part_cnt + r.poff, e.H,
                         blockIdx.x, r.nparts);
}

__global__ void k_philox(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1,
                         uint4* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = philox10(ctr[i], k0, k1);
}

int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_minmax(const float* z, const uint8_t* mask, long long n, unsigned* keys,
                          unsigned long long* nsamples, cudaStream_t st) {
    count_launches(1, st);
    k_minmax<<<grid_for(n), kThreads, 0, st>>>(z, mask, n, keys, nsamples);
    return cudaGetLastError();
}

cudaError_t launch_pack(const EntryDesc* e, const float* z, const uint8_t* mask, double zmin,
                        double scale, float2* lat, uint32_t key0, uint32_t key1, int all_free,
                        bool f64, cudaStream_t st) {
    count_launches(1, st);
    const int g = grid_for((long long)e->W * e->H);
    if (f64)
        k_pack<double2><<<g, kThreads, 0, st>>>(*e, z, mask, zmin, scale, reinterpret_cast<double2*>(lat),
                                               key0, key1, all_free);
    else
        k_pack<float2><<<g, kThreads, 0, st>>>(*e, z, mask, zmin, scale, lat, key0, key1, all_free);
    return cudaGetLastError();
}

cudaError_t launch_gap_count(const EntryDesc* e, const uint8_t* mask, int all_free,
                             int* row_counts, cudaStream_t st) {
    const int blocks = (e->H * 32 + kThreads - 1) / kThreads;
    count_launches(1, st);
    k_gap_count<<<blocks, kThreads, 0, st>>>(*e, mask, all_free, row_counts);
    return cudaGetLastError();
}

cudaError_t launch_scan_rows(int* row_counts, int nrows, int narrays, int* totals,
                             cudaStream_t st) {
    count_launches(1, st);
    k_scan_rows<<<narrays, 1024, 0, st>>>(row_counts, nrows, totals);
    return cudaGetLastError();
}

cudaError_t launch_gap_scatter(const EntryDesc* e, const uint8_t* mask, int all_free,
                               const int* row_offsets, uint32_t* gaps, cudaStream_t st) {
    const int blocks = (e->H * 32 + kThreads - 1) / kThreads;
    count_launches(1, st);
    k_gap_scatter<<<blocks, kThreads, 0, st>>>(*e, mask, all_free, row_offsets, gaps);
    return cudaGetLastError();
}

cudaError_t launch_sample_energy(const EntryDesc* e, const float* z, const uint8_t* mask,
                                 double scale, double q, double* part_sum,
                                 unsigned long long* part_cnt, int* nparts, bool f64, cudaStream_t st,
                                 int y_end) {
    if (y_end < 0 || y_end > e->H) y_end = e->H;
    const int g = y_end < 1 ? 1 : (y_end < 1024 ? y_end : 1024);
    *nparts = g;
    count_launches(1, st);
    if (f64) k_sample_energy64<<<g, kThreads, 0, st>>>(*e, z, mask, q * scale, part_sum, part_cnt, y_end);
    else k_sample_energy<<<g, kThreads, 0, st>>>(*e, z, mask, (float)(q * scale), part_sum, part_cnt, y_end);
    return cudaGetLastError();
}

cudaError_t launch_minmax_batch(const SetupRec* recs, int n, long long max_sites, unsigned* keys,
                                unsigned long long* nsamples, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    count_launches(1, st);
    k_minmax_batch<<<dim3(std::min(grid_for(max_sites), 608), n), kThreads, 0, st>>>(recs, keys, nsamples);
    return cudaGetLastError();
}

cudaError_t launch_pack_batch(const EntryDesc* ents, const SetupRec* recs, int n, long long max_sites,
                              float2* lat, uint32_t key0, uint32_t key1, int all_free, bool f64,
                              cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    count_launches(1, st);
    const dim3 g(std::min(grid_for(max_sites), 608), n);
    if (f64)
        k_pack_batch<double2><<<g, kThreads, 0, st>>>(ents, recs, reinterpret_cast<double2*>(lat), key0, key1,
                                                      all_free);
    else
        k_pack_batch<float2><<<g, kThreads, 0, st>>>(ents, recs, lat, key0, key1, all_free);
    return cudaGetLastError();
}

cudaError_t launch_gap_count_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_rows,
                                   int all_free, int* row_counts, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    count_launches(1, st);
    k_gap_count_batch<<<dim3((max_rows * 32 + kThreads - 1) / kThreads, n), kThreads, 0, st>>>(ents, recs, all_free,
                                                                                               row_counts);
    return cudaGetLastError();
}

cudaError_t launch_scan_rows_batch(const EntryDesc* ents, const SetupRec* recs, int n, int* row_counts,
                                   int* totals, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    count_launches(1, st);
    k_scan_rows_batch<<<2 * n, 1024, 0, st>>>(ents, recs, row_counts, totals);
    return cudaGetLastError();
}

cudaError_t launch_gap_scatter_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_rows,
                                     int all_free, const int* row_offsets, uint32_t* gaps, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    count_launches(1, st);
    k_gap_scatter_batch<<<dim3((max_rows * 32 + kThreads - 1) / kThreads, n), kThreads, 0, st>>>(
        ents, recs, all_free, row_offsets, gaps);
    return cudaGetLastError();
}

cudaError_t launch_sample_energy_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_parts,
                                       double q, double* part_sum, unsigned long long* part_cnt, bool f64,
                                       cudaStream_t st) {
    if (n < 1 || max_parts < 1) return cudaSuccess;
    count_launches(1, st);
    if (f64) k_sample_energy64_batch<<<dim3(max_parts, n), kThreads, 0, st>>>(ents, recs, q, part_sum, part_cnt);
    else k_sample_energy_batch<<<dim3(max_parts, n), kThreads, 0, st>>>(ents, recs, q, part_sum, part_cnt);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, size_t n,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    count_launches(1, st);
    k_philox<<<grid_for((long long)n), kThreads, 0, st>>>(ctr, k0, k1, out, n);
    return cudaGetLastError();
}

}  // namespace mpr
