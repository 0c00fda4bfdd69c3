// mpr_sweep.cu -- the hot path: checkerboard half-sweeps of the hybrid update
// (Algorithm 1 with the over-relaxation of Eq. 6), the per-sweep control of
// Algorithm 2 step 5, the energy (Eq. 2), and the equilibrium averaging with the
// inverse of Eq. 1 (Algorithm 2 steps 6-7).
#include "mpr_internal.cuh"

namespace mpr {
namespace {

// Half-sweep: every gap site of one colour (all entries), Algorithm 1.
// Blocks come from a work list (entry, first gap) so that grids of any size share a launch.
template <int TRIG, bool ACC, bool GQ>
__global__ void __launch_bounds__(kSweepThreads)
k_half_sweep(const SweepArgs A, const int color) {
    const BlockWork w = (color ? A.work[1] : A.work[0])[blockIdx.x];
    const EntryDesc* __restrict__ E = A.ents + w.entry;
    const Ctl* ctl = A.ctl + w.entry;
    if (A.skip_stopped && ctl->stop) return;
    const float half_qd = A.use_ctl_a ? (float)(0.5 * kTwoPi * E->q / ctl->a) : A.half_qd_fixed;
    const float cQ = (float)E->cQ, sQ = (float)E->sQ;
    const float kx = accept_scale<TRIG>((float)(-1.0 / ctl->T));
    const uint32_t sweep = ctl->sweep;
    const int n = color ? E->ngap[1] : E->ngap[0], pitch = E->pitch, W = E->W;
    const uint32_t chain = E->chain;
    const int row_off = (int)E->row_off;
    const long long gb = color ? E->gbase[1] : E->gbase[0];
    const uint32_t* __restrict__ gl = A.gaps + gb;
    float2* __restrict__ own = A.lat + (color ? E->plane[1] : E->plane[0]);
    const float2* __restrict__ oth = A.lat + (color ? E->plane[0] : E->plane[1]);
    float* __restrict__ acc = ACC ? A.acc + gb : nullptr;

    static_assert(kSweepItems <= kDEMaxSites32, "32-bit energy partial");
    int dE = 0;                                   // fixed point, whole kDEUnit per site
    unsigned nacc = 0;
#pragma unroll
    for (int it = 0; it < kSweepItems; ++it) {
        const int g = w.first + it * kSweepThreads + (int)threadIdx.x;
        if (g < n) {
            const uint32_t ent = __ldg(gl + g);
            const int y = (int)(ent >> 16), j = (int)(ent & 0xFFFFu);
            const int s = color ^ (y & 1);
            const long long k = (long long)(y + 1) * pitch + j + kPadL;
            const float2 nu = oth[k - pitch], nd = oth[k + pitch];
            const float2 nl = oth[k - 1 + s], nr = oth[k + s];
            const float C = (nu.x + nd.x) + (nl.x + nr.x);
            const float S = (nu.y + nd.y) + (nl.y + nr.y);
            float2 v = own[k];
            const uint4 rnd = philox10(make_uint4(quad_index(W, y + row_off, 2 * j + s), sweep, chain,
                                                  (uint32_t)color), A.rk);
            const bool second = (j & 1) != 0;                    // floor(x / 2) odd
            const float hq = (u24f(second ? rnd.z : rnd.x) - 0.5f) * half_qd;
            const float ur = u24f(second ? rnd.w : rnd.y);
            bool accepted;
            float Fx = 0.0f, Fy = 0.0f;
            if (A.or_mode == OR_LITERAL) literal_field(nu, nd, nl, nr, Fx, Fy);
            dE += de_fixed(hybrid_update<TRIG, GQ>(v, C, S, Fx, Fy, hq, ur, kx, A.or_mode, accepted,
                                                   cQ, sQ));
            nacc += accepted ? 1u : 0u;
            own[k] = v;
            if (ACC) acc[g] += angle_upper(v.x, v.y);
        }
    }
    // energy change (exact integer sums) and acceptance count of the block
    __shared__ long long s_dE[kSweepThreads / 32];
    __shared__ unsigned s_na[kSweepThreads / 32];
    long long dEw = dE;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dEw += __shfl_xor_sync(0xffffffffu, dEw, o);
    nacc = warp_sum(nacc);
    if ((threadIdx.x & 31) == 0) {
        s_dE[threadIdx.x >> 5] = dEw;
        s_na[threadIdx.x >> 5] = nacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        unsigned na = 0;
#pragma unroll
        for (int i = 0; i < kSweepThreads / 32; ++i) { t += s_dE[i]; na += s_na[i]; }
        Part p;
        p.dH = (double)t * kDEUnit;
        p.nacc = na;
        p._pad = 0;
        (color ? A.part[1] : A.part[0])[blockIdx.x] = p;
    }
}

// The half-sweep in FP64 (MPR_PREC_F64): the same work list, counters and partials, on a
// lattice of double2 vectors with FP64 arithmetic throughout.
template <bool ACC, bool GQ>
__global__ void __launch_bounds__(kSweepThreads)
k_half_sweep64(const SweepArgs A, const int color) {
    const BlockWork w = (color ? A.work[1] : A.work[0])[blockIdx.x];
    const EntryDesc* __restrict__ E = A.ents + w.entry;
    const Ctl* ctl = A.ctl + w.entry;
    if (A.skip_stopped && ctl->stop) return;
    const double half_qd = A.use_ctl_a ? 0.5 * kTwoPi * E->q / ctl->a : A.half_qd_fixed64;
    const double cQ = E->cQ, sQ = E->sQ;
    const double neg_inv_T = -1.0 / ctl->T;
    const uint32_t sweep = ctl->sweep;
    const int n = color ? E->ngap[1] : E->ngap[0], pitch = E->pitch, W = E->W;
    const uint32_t chain = E->chain;
    const int row_off = (int)E->row_off;
    const long long gb = color ? E->gbase[1] : E->gbase[0];
    const uint32_t* __restrict__ gl = A.gaps + gb;
    double2* __restrict__ lat = reinterpret_cast<double2*>(A.lat);
    double2* __restrict__ own = lat + (color ? E->plane[1] : E->plane[0]);
    const double2* __restrict__ oth = lat + (color ? E->plane[0] : E->plane[1]);
    double* __restrict__ acc = ACC ? reinterpret_cast<double*>(A.acc) + gb : nullptr;

    double dE = 0.0;
    unsigned nacc = 0;
#pragma unroll
    for (int it = 0; it < kSweepItems; ++it) {
        const int g = w.first + it * kSweepThreads + (int)threadIdx.x;
        if (g < n) {
            const uint32_t ent = __ldg(gl + g);
            const int y = (int)(ent >> 16), j = (int)(ent & 0xFFFFu);
            const int s = color ^ (y & 1);
            const long long k = (long long)(y + 1) * pitch + j + kPadL;
            const double2 nu = oth[k - pitch], nd = oth[k + pitch];
            const double2 nl = oth[k - 1 + s], nr = oth[k + s];
            const double C = (nu.x + nd.x) + (nl.x + nr.x);
            const double S = (nu.y + nd.y) + (nl.y + nr.y);
            double2 v = own[k];
            const uint4 rnd = philox10(make_uint4(quad_index(W, y + row_off, 2 * j + s), sweep, chain,
                                                  (uint32_t)color), A.rk);
            const bool second = (j & 1) != 0;                    // floor(x / 2) odd
            const double hq = ((double)u24f(second ? rnd.z : rnd.x) - 0.5) * half_qd;
            const double ur = (double)u24f(second ? rnd.w : rnd.y);
            bool accepted;
            double Fx = 0.0, Fy = 0.0;
            if (A.or_mode == OR_LITERAL) literal_field64(nu, nd, nl, nr, Fx, Fy);
            dE += hybrid_update64<GQ>(v, C, S, Fx, Fy, hq, ur, neg_inv_T, A.or_mode, accepted,
                                      cQ, sQ);
            nacc += accepted ? 1u : 0u;
            own[k] = v;
            if (ACC) acc[g] += atan2(v.y, v.x);
        }
    }
    __shared__ double s_dE[kSweepThreads / 32];
    __shared__ unsigned s_na[kSweepThreads / 32];
    dE = warp_sum(dE);
    nacc = warp_sum(nacc);
    if ((threadIdx.x & 31) == 0) {
        s_dE[threadIdx.x >> 5] = dE;
        s_na[threadIdx.x >> 5] = nacc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned na = 0;
#pragma unroll
        for (int i = 0; i < kSweepThreads / 32; ++i) { t += s_dE[i]; na += s_na[i]; }
        Part p;
        p.dH = t;
        p.nacc = na;
        p._pad = 0;
        (color ? A.part[1] : A.part[0])[blockIdx.x] = p;
    }
}

// Per-sweep control, one block per entry.  The block first adds the sweep blocks'
// partials of this entry in a fixed order (bitwise reproducible), then thread 0 runs
//   CTL_RELAX : Algorithm 2 step 5 after one sweep (window 5.2, energy 5.3, slope 5.4, 5.5)
//   CTL_FIXED : bookkeeping of a fixed-window sweep (energy, acceptance, counter)
//   CTL_SAMPLE: as FIXED, and accumulate e for the e(T, L) table average
constexpr int kCtlThreads = 128;
__global__ void __launch_bounds__(kCtlThreads)
k_control(Ctl* ctl, Part* part0, Part* part1, const EntryDesc* __restrict__ ents, int mode,
          double A_targ, double k_a, int n_f, int n_fit, int i_max, double* ehist,
          int ehist_stride, int* active, int f64_parts) {
    __shared__ double s_dH[kCtlThreads];
    __shared__ unsigned long long s_na[kCtlThreads];
    __shared__ long long s_fx[kCtlThreads];
    const int e = blockIdx.x;
    const EntryDesc E = ents[e];
    // FP32 partials are whole numbers of kDEUnit: added as integers (exact); FP64 ones as
    // doubles in a fixed order
    const bool fixed = !f64_parts;
    double dH = 0.0;
    long long fx = 0;
    unsigned long long na = 0;
    for (int c = 0; c < 2; ++c) {
        const Part* p = c ? part1 + E.blk0[1] : part0 + E.blk0[0];
        const int nb = c ? E.nblk[1] : E.nblk[0];
        for (int b = threadIdx.x; b < nb; b += kCtlThreads) {
            if (fixed) fx += de_units(p[b].dH);
            else dH += p[b].dH;
            na += p[b].nacc;
        }
    }
    s_fx[threadIdx.x] = fx;
    s_dH[threadIdx.x] = dH;
    s_na[threadIdx.x] = na;
    __syncthreads();
    for (int o = kCtlThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_dH[threadIdx.x] += s_dH[threadIdx.x + o];
            s_fx[threadIdx.x] += s_fx[threadIdx.x + o];
            s_na[threadIdx.x] += s_na[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    dH = fixed ? (double)s_fx[0] * kDEUnit : s_dH[0];
    na = s_na[0];
    Ctl c = ctl[e];
    control_step(c, E, dH, na, mode, A_targ, k_a, n_f, n_fit, i_max,
                 ehist + (long long)e * ehist_stride, 0);
    ctl[e] = c;
    if (active && !c.stop) atomicAdd(active, 1);
}

// Eq. 2 over all bonds of one grid: each colour-0 site with its four colour-1 neighbours
// (padding contributes 0).  cos(theta_i - theta_j) = c_i c_j + s_i s_j.  One partial per block.
__device__ __forceinline__ double bond_sum(float2 v, float2 a, float2 b, float2 l, float2 r) {
    return (double)fmaf(v.x, a.x, v.y * a.y) + (double)fmaf(v.x, b.x, v.y * b.y) +
           (double)fmaf(v.x, l.x, v.y * l.y) + (double)fmaf(v.x, r.x, v.y * r.y);
}
__device__ __forceinline__ double bond_sum(double2 v, double2 a, double2 b, double2 l, double2 r) {
    return fma(v.x, a.x, v.y * a.y) + fma(v.x, b.x, v.y * b.y) + fma(v.x, l.x, v.y * l.y) +
           fma(v.x, r.x, v.y * r.y);
}

template <typename V>
__device__ __forceinline__ void energy_body(const EntryDesc& e, const V* __restrict__ lat, double* part, int y_a,
                                            int y_b, int bid, int nb) {
    __shared__ double sw[8];
    const int Wc = (e.W + 1) >> 1;
    const long long n = (long long)(y_b - y_a) * Wc;
    const V* p0 = lat + e.plane[0];
    const V* p1 = lat + e.plane[1];
    double acc = 0.0;
    for (long long t = bid * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)nb * blockDim.x) {
        const int yr = (int)(t / Wc), j = (int)(t - (long long)yr * Wc), y = y_a + yr;
        const int s = y & 1;                                     // colour 0: s = y & 1
        if (2 * j + s >= e.W) continue;
        const long long k = (long long)(y + 1) * e.pitch + j + kPadL;
        acc -= bond_sum(p0[k], p1[k - e.pitch], p1[k + e.pitch], p1[k - 1 + s], p1[k + s]);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
        part[bid] = t;
    }
}
template <typename V>
__global__ void k_energy(EntryDesc e, const V* __restrict__ lat, double* part, int y_a, int y_b) {
    energy_body(e, lat, part, y_a, y_b, blockIdx.x, gridDim.x);
}

// Blocks of the energy launch of a grid of W x H sites (the single-grid launch's count).
__host__ __device__ __forceinline__ int energy_blocks(int W, int H, int scratch_len) {
    const long long n = (long long)H * ((W + 1) >> 1);
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)(b < scratch_len ? b : scratch_len);
}
template <typename V>
__global__ void k_energy_batch(const EntryDesc* __restrict__ ents, const V* __restrict__ lat0,
                               const V* __restrict__ lat1, const Ctl* __restrict__ ctl, int tiled, double* scratch,
                               int scratch_len) {
    const EntryDesc e = ents[blockIdx.y];
    const int nb = energy_blocks(e.W, e.H, scratch_len);
    if ((int)blockIdx.x >= nb) return;
    const V* lat = (tiled && ctl[blockIdx.y].cur) ? lat1 : lat0;
    energy_body(e, lat, scratch + (long long)blockIdx.y * scratch_len, 0, e.H, blockIdx.x, nb);
}

// Fixed-order sum of n doubles (one block).
__device__ __forceinline__ void sum_body(const double* __restrict__ v, int n, double* out) {
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) t += v[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}
__global__ void k_sum(const double* __restrict__ v, int n, double* out) { sum_body(v, n, out); }
__global__ void k_sum_batch(const EntryDesc* __restrict__ ents, const double* __restrict__ v, int scratch_len,
                            double* out) {
    const EntryDesc& e = ents[blockIdx.x];
    sum_body(v + (long long)blockIdx.x * scratch_len, energy_blocks(e.W, e.H, scratch_len), out + blockIdx.x);
}

__global__ void k_set_tracked_energy(Ctl* ctl, const double* H, int n_ent) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_ent) ctl[e].H = H[e];
}

// Row strips: the half-sweep blocks' energy changes and acceptance counts of one colour,
// added in block order (one thread: the order is fixed).
__global__ void k_strip_partials(const Part* __restrict__ part, int nblk, int color, double* out,
                                 int f64_parts) {
    double dH = 0.0, na = 0.0;
    long long fx = 0;                                       // FP32: exact integer sum
    for (int b = 0; b < nblk; ++b) {
        if (f64_parts) dH += part[b].dH;
        else fx += de_units(part[b].dH);
        na += (double)part[b].nacc;
    }
    if (!f64_parts) dH = (double)fx * kDEUnit;
    out[0] = color ? out[0] + dH : dH;
    out[1] = color ? out[1] + na : na;
}

// Row strips: one control step from the totals of every strip; e carries the whole grid's
// gap count and bond count.
__global__ void k_strip_control(Ctl* ctl, EntryDesc e, const double* __restrict__ tot, int mode,
                                double A_targ, double k_a, int n_f, int n_fit, int i_max, double* ehist,
                                int* stop) {
    Ctl c = ctl[0];
    control_step(c, e, tot[0], (unsigned long long)tot[1], mode, A_targ, k_a, n_f, n_fit, i_max, ehist, 0);
    ctl[0] = c;
    if (stop) *stop = c.stop;
}

// Algorithm 2 step 7: zhat = G^-1(mean phi) at gap sites (G affine, so this equals the
// mean of the back-transformed realizations).  Sample sites are copied beforehand.
template <typename A>
__global__ void k_predict_out(EntryDesc e, const uint32_t* __restrict__ gaps,
                              const A* __restrict__ acc, int M, double q, double zmin,
                              double zmax, float* __restrict__ zhat) {
    const int P = e.ngap[0] + e.ngap[1];
    const double f = (zmax - zmin) / (kTwoPi * q * (double)M);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P; g += gridDim.x * blockDim.x) {
        const int c = g < e.ngap[0] ? 0 : 1;
        const long long gi = c ? e.gbase[1] + (g - e.ngap[0]) : e.gbase[0] + g;
        const uint32_t ent = gaps[gi];
        const int y = (int)(ent >> 16), j = (int)(ent & 0xFFFFu);
        const int x = 2 * j + (c ^ (y & 1));
        double v = zmin + (double)acc[gi] * f;
        v = v < zmin ? zmin : (v > zmax ? zmax : v);
        zhat[(long long)y * e.W + x] = (float)v;
    }
}

// phi = 2 theta, theta the angle of (cos, sin) in [0, pi], for every site of one grid:
// FP32 vectors to float by the polynomial angle, anything to double by atan2 in FP64.
// phi = theta / q (inv_q = 1/q; 2 exactly for q = 1/2).
__device__ __forceinline__ void put_angle(float2 v, double inv_q, float& out) {
    out = (float)inv_q * angle_upper(v.x, fmaxf(v.y, 0.0f));
}
__device__ __forceinline__ void put_angle(float2 v, double inv_q, double& out) {
    out = inv_q * atan2(fmax((double)v.y, 0.0), (double)v.x);
}
__device__ __forceinline__ void put_angle(double2 v, double inv_q, double& out) { out = inv_q * atan2(fmax(v.y, 0.0), v.x); }
__device__ __forceinline__ void put_angle(double2 v, double inv_q, float& out) {
    double d;
    put_angle(v, inv_q, d);
    out = (float)d;
}

template <typename V, typename O>
__global__ void k_get_state(EntryDesc e, const V* __restrict__ lat, O* __restrict__ phi) {
    const long long n = (long long)e.W * e.H;
    const double inv_q = 1.0 / e.q;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / e.W), x = (int)(i - (long long)y * e.W);
        const long long base = ((x + y) & 1) ? e.plane[1] : e.plane[0];
        put_angle(lat[base + (long long)(y + 1) * e.pitch + (x >> 1) + kPadL], inv_q, phi[i]);
    }
}

// (cos theta, sin theta) of theta = q phi.
__device__ __forceinline__ void unit_q(float phi, double q, float2& v) {
    float s, co;
    sincosf((float)q * phi, &s, &co);
    v = make_float2(co, fmaxf(s, 0.0f));
}
__device__ __forceinline__ void unit_q(float phi, double q, double2& v) {
    double s, co;
    sincos(q * (double)phi, &s, &co);
    v = make_double2(co, fmax(s, 0.0));
}

// Writes gap sites from phi (samples untouched).
template <typename V>
__global__ void k_set_state(EntryDesc e, V* __restrict__ lat, const uint32_t* __restrict__ gaps,
                            const float* __restrict__ phi) {
    const int P = e.ngap[0] + e.ngap[1];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P; g += gridDim.x * blockDim.x) {
        const int c = g < e.ngap[0] ? 0 : 1;
        const long long gi = c ? e.gbase[1] + (g - e.ngap[0]) : e.gbase[0] + g;
        const uint32_t ent = gaps[gi];
        const int y = (int)(ent >> 16), j = (int)(ent & 0xFFFFu);
        const int x = 2 * j + (c ^ (y & 1));
        const long long base = c ? e.plane[1] : e.plane[0];
        unit_q(phi[(long long)y * e.W + x], e.q, lat[base + (long long)(y + 1) * e.pitch + j + kPadL]);
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_half_sweep(const SweepArgs& a, int color, int trig, cudaStream_t st) {
    const int nb = a.nblk[color];
    if (nb == 0) return cudaSuccess;
    const bool acc = a.acc != nullptr;
    count_launches(1, st);
    const dim3 g(nb), b(kSweepThreads);
    if (a.f64) {
        if (a.genq) {
            if (acc) k_half_sweep64<true, true><<<g, b, 0, st>>>(a, color);
            else k_half_sweep64<false, true><<<g, b, 0, st>>>(a, color);
        } else {
            if (acc) k_half_sweep64<true, false><<<g, b, 0, st>>>(a, color);
            else k_half_sweep64<false, false><<<g, b, 0, st>>>(a, color);
        }
    } else if (a.genq) {
        if (trig == TRIG_FAST) {
            if (acc) k_half_sweep<TRIG_FAST, true, true><<<g, b, 0, st>>>(a, color);
            else k_half_sweep<TRIG_FAST, false, true><<<g, b, 0, st>>>(a, color);
        } else {
            if (acc) k_half_sweep<TRIG_ACCURATE, true, true><<<g, b, 0, st>>>(a, color);
            else k_half_sweep<TRIG_ACCURATE, false, true><<<g, b, 0, st>>>(a, color);
        }
    } else if (trig == TRIG_FAST) {
        if (acc) k_half_sweep<TRIG_FAST, true, false><<<g, b, 0, st>>>(a, color);
        else k_half_sweep<TRIG_FAST, false, false><<<g, b, 0, st>>>(a, color);
    } else {
        if (acc) k_half_sweep<TRIG_ACCURATE, true, false><<<g, b, 0, st>>>(a, color);
        else k_half_sweep<TRIG_ACCURATE, false, false><<<g, b, 0, st>>>(a, color);
    }
    return cudaGetLastError();
}

cudaError_t launch_control(Ctl* ctl, Part* const part[2], const EntryDesc* ents, int n_ent,
                           int mode, double A_targ, double k_a, int n_f, int n_fit, int i_max,
                           double* ehist, int ehist_stride, int* active, bool f64, cudaStream_t st) {
    count_launches(1, st);
    k_control<<<n_ent, kCtlThreads, 0, st>>>(ctl, part[0], part[1], ents, mode, A_targ, k_a, n_f,
                                             n_fit, i_max, ehist, ehist_stride, active, f64 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_energy(const EntryDesc* e_host, const float2* lat, double* scratch,
                          int scratch_len, double* out, bool f64, cudaStream_t st, int y_a, int y_b) {
    if (y_b < 0 || y_b > e_host->H) y_b = e_host->H;
    if (y_a < 0) y_a = 0;
    if (y_a > y_b) y_a = y_b;
    const long long n = (long long)(y_b - y_a) * ((e_host->W + 1) >> 1);
    int g = grid_for(n > 0 ? n : 1, 256);
    if (g > scratch_len) g = scratch_len;
    count_launches(1, st);
    if (f64) k_energy<double2><<<g, 256, 0, st>>>(*e_host, reinterpret_cast<const double2*>(lat), scratch, y_a, y_b);
    else k_energy<float2><<<g, 256, 0, st>>>(*e_host, lat, scratch, y_a, y_b);
    count_launches(1, st);
    k_sum<<<1, 256, 0, st>>>(scratch, g, out);
    return cudaGetLastError();
}

cudaError_t launch_energy_batch(const EntryDesc* ents, int n, int max_cols, int max_rows, const float2* lat0,
                                const float2* lat1, const Ctl* ctl, int tiled, double* scratch,
                                int scratch_len, double* out, bool f64, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    const dim3 g(energy_blocks(max_cols, max_rows, scratch_len), n);
    count_launches(2, st);
    if (f64)
        k_energy_batch<double2><<<g, 256, 0, st>>>(ents, reinterpret_cast<const double2*>(lat0),
                                                   reinterpret_cast<const double2*>(lat1), ctl, tiled, scratch,
                                                   scratch_len);
    else
        k_energy_batch<float2><<<g, 256, 0, st>>>(ents, lat0, lat1, ctl, tiled, scratch, scratch_len);
    k_sum_batch<<<n, 256, 0, st>>>(ents, scratch, scratch_len, out);
    return cudaGetLastError();
}

cudaError_t launch_strip_partials(const Part* part, int nblk, int color, double* out, bool f64,
                                  cudaStream_t st) {
    count_launches(1, st);
    k_strip_partials<<<1, 1, 0, st>>>(part, nblk, color, out, f64 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_strip_control(Ctl* ctl, const EntryDesc* e_host, double P, double ngp, const double* tot,
                                 int mode, double A_targ, double k_a, int n_f, int n_fit, int i_max,
                                 double* ehist, int* stop_dev, cudaStream_t st) {
    EntryDesc e = *e_host;
    e.P = (int)P;
    e.ngp = ngp;
    count_launches(1, st);
    k_strip_control<<<1, 1, 0, st>>>(ctl, e, tot, mode, A_targ, k_a, n_f, n_fit, i_max, ehist, stop_dev);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double* v, int n, double* out, cudaStream_t st) {
    count_launches(1, st);
    k_sum<<<1, 256, 0, st>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_set_tracked_energy(Ctl* ctl, const double* H, int n_ent, cudaStream_t st) {
    count_launches(1, st);
    k_set_tracked_energy<<<(n_ent + 255) / 256, 256, 0, st>>>(ctl, H, n_ent);
    return cudaGetLastError();
}

cudaError_t launch_predict_out(const EntryDesc* e_host, const float2*, const uint32_t* gaps,
                               const float* acc, int M, double q, double zmin, double zmax,
                               float* zhat, bool f64, cudaStream_t st) {
    const long long P = (long long)e_host->ngap[0] + e_host->ngap[1];
    if (P == 0) return cudaSuccess;
    count_launches(1, st);
    const int g = grid_for(P, 256);
    if (f64)
        k_predict_out<double><<<g, 256, 0, st>>>(*e_host, gaps, reinterpret_cast<const double*>(acc), M, q,
                                                 zmin, zmax, zhat);
    else
        k_predict_out<float><<<g, 256, 0, st>>>(*e_host, gaps, acc, M, q, zmin, zmax, zhat);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const EntryDesc* e_host, const float2* lat, float* phi, bool f64,
                             cudaStream_t st) {
    count_launches(1, st);
    const int g = grid_for((long long)e_host->W * e_host->H, 256);
    if (f64) k_get_state<double2, float><<<g, 256, 0, st>>>(*e_host, reinterpret_cast<const double2*>(lat), phi);
    else k_get_state<float2, float><<<g, 256, 0, st>>>(*e_host, lat, phi);
    return cudaGetLastError();
}

cudaError_t launch_get_state64(const EntryDesc* e_host, const float2* lat, double* phi, bool f64,
                               cudaStream_t st) {
    count_launches(1, st);
    const int g = grid_for((long long)e_host->W * e_host->H, 256);
    if (f64) k_get_state<double2, double><<<g, 256, 0, st>>>(*e_host, reinterpret_cast<const double2*>(lat), phi);
    else k_get_state<float2, double><<<g, 256, 0, st>>>(*e_host, lat, phi);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const EntryDesc* e_host, float2* lat, const uint32_t* gaps,
                             const float* phi, bool f64, cudaStream_t st) {
    const long long P = (long long)e_host->ngap[0] + e_host->ngap[1];
    if (P == 0) return cudaSuccess;
    count_launches(1, st);
    const int g = grid_for(P, 256);
    if (f64) k_set_state<double2><<<g, 256, 0, st>>>(*e_host, reinterpret_cast<double2*>(lat), gaps, phi);
    else k_set_state<float2><<<g, 256, 0, st>>>(*e_host, lat, gaps, phi);
    return cudaGetLastError();
}

}  // namespace mpr
