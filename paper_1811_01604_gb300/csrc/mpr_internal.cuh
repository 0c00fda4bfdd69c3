// mpr_internal.cuh -- device data layout, helpers and launcher declarations of libmpr.
//
// Lattice layout (one "entry" = one W x H grid with its own chain):
//   The checkerboard of Sect. 3.3 splits the grid into colour 0 ((x+y) even) and
//   colour 1.  Each colour is packed into a plane of float2 unit vectors
//   (cos(q phi), sin(q phi)), row y, column j = x >> 1, with one padding row above
//   and below and kPadL padding columns on the left (two, so that tiles whose first
//   grid column is a multiple of 4 start on a 16-byte boundary).  Padding slots hold
//   (0, 0), so an out-of-grid neighbour contributes nothing to the local field: no
//   boundary branches in the sweep.  For q = 1/2 the state space phi in [0, 2pi) is
//   the upper half circle sin(q phi) >= 0.
//   Padded index of (y, j): (y + 1) * pitch + (j + kPadL).  For a site of colour c in
//   row y, s = c ^ (y & 1) gives x = 2j + s and its neighbours in the other plane at
//   k - pitch, k + pitch, k - 1 + s, k + s.
//   Gap sites of each colour are listed row-major as (y << 16) | j.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpr {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kPadL = 2;                          // zero columns left of column j = 0
constexpr int kSweepThreads = 256;
constexpr int kSweepItems = 2;                    // gap sites per thread per launch chunk
constexpr uint32_t kInitSweep = 0xFFFFFFFFu;      // Philox sweep word of the initial state

// Control modes (Algorithm 2 step 5 / fixed window / table sampling).
enum { CTL_RELAX = 0, CTL_FIXED = 1, CTL_SAMPLE = 2 };

struct EntryDesc {            // immutable during a run
    int W, H, pitch;
    uint32_t row_off;         // rows of a larger grid above this block (its Philox counters)
    long long plane[2];       // float2 offset of plane c's padded origin
    long long gbase[2];       // offset of colour c's gap list
    int ngap[2];
    uint32_t chain;           // realization id (Philox counter word 2)
    int P;                    // ngap[0] + ngap[1]
    double ngp;               // number of nearest-neighbour pairs, W(H-1) + H(W-1)
    long long site0;          // offset of the grid in concatenated [H][W] buffers
    int blk0[2];              // first sweep block of this entry in colour c's work list
    int nblk[2];              // number of sweep blocks of this entry per colour
    int tile0;                // first tile of this entry (tile path)
    int ntiles;               // number of tiles of this entry
    int prows;                // rows allocated per plane: max(H + 2, tallest tile box)
    int _pad2;
    double q;                 // coupling of Eq. 2: theta = q phi in [0, 2 pi q)
    double cQ, sQ;            // cos and sin of Q = 2 pi q, the end of the range of theta
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
    int nsamp;
    int status;               // 0, or a device-side error code
    int cur;                  // tile path: which of the two lattice buffers holds the state
    float half_qd;            // q * pi / a as float (proposal half-angle scale)
    float neg_inv_T;          // -1/T as float
    // tile path: sweep counter and buffer at the start of the current multi-sweep launch
    // (sweep s of a launch has counter sweep_base + s and reads buffer cur_base ^ (s & 1));
    // written by the host with every change of `sweep` and by the last block of a launch
    uint32_t sweep_base;
    int cur_base;
    // global sweep counter (Philox counter word 1) and, in the same 8-byte word, the
    // window of that sweep, or -1 once the relaxation has stopped (ctl_set_go): the tile
    // path publishes this word last, with release semantics, after the other fields, so a
    // block learns with one load whether sweep `sweep` runs and with which window
    uint32_t sweep;
    float go_hqd;
};

// Keeps go_hqd in step with half_qd and stop (after every change of either).
__host__ __device__ inline void ctl_set_go(Ctl& c) { c.go_hqd = c.stop ? -1.0f : c.half_qd; }

struct Part {                 // one sweep block's energy change and acceptance count
    double dH;                // FP32 paths: a whole number of kDEUnit (exactly representable)
    unsigned nacc;
    unsigned _pad;
};

// Tile path (mpr_tile.cu): tiles of TH x TW grid sites in one of the compiled
// configurations (tile_geom).
struct TileGeom {
    int th, tw;               // tile rows and columns (grid sites)
    int rh, rw;               // TMA box: rows and plane columns of the region (halo 2)
    int list;                 // u16 list entries per tile slot
    int acc;                  // accumulator floats per tile
    int nt;                   // threads per block
};

// A tile's gap list has three parts: colour A inside the tile, colour A on the one-site
// ring around it, colour B inside the tile.  An entry is a pair of plane columns of one
// region row; the interior parts list the pairs whose two sites are both gaps first ("full":
// two updates from one Philox block), then the pairs with one gap site; the ring part has
// one entry per site.
struct TileDesc {             // one tile: its grid, origin, and gap-list counts (set-up)
    int entry;
    int y0, x0;
    int nA_int;               // entries: colour A inside the tile
    int nA_ring;              // entries: colour A on the one-site ring
    int nB;                   // entries: colour B inside the tile
    int t;                    // the tile's own index (its lists and accumulators)
    int nfull;                // full pairs: colour A in bits 0-15, colour B in bits 16-31
};

struct TileCnt {              // entries listed for one tile (as in TileDesc)
    uint16_t nA_int;
    uint16_t nA_ring;
    uint16_t nB;
    uint16_t nA_full;
    uint16_t nB_full;
    uint16_t _pad;
};

// Philox4x32-10 round keys (k + r * Weyl constant, r = 0..9) computed once on the host, so
// the kernels XOR them in straight from the parameter bank instead of stepping the key
// schedule for every site.
struct RoundKeys {
    uint32_t k0[10], k1[10];
};
inline RoundKeys round_keys(uint64_t seed) {
    RoundKeys rk;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return rk;
}

constexpr int kSlots = 8;     // per grid: ring of per-sweep totals and tickets (tile path)

struct TileArgs {
    const EntryDesc* ents;
    float2* lat[2];           // the two lattice buffers (sweep s reads cur_base ^ (s & 1))
    const CUtensorMap* maps;  // per entry: maps of buffer 0 and buffer 1 (64-byte aligned)
    int* err;                 // set to 1 if a bounded wait gave up
    const TileDesc* desc;     // tiles in the order they are handed out (TileDesc::t = index)
    const uint16_t* lists;    // per tile index: its gap list slot
    float* acc;               // per-tile accumulators, or nullptr
    Ctl* ctl;
    unsigned long long* gsum; // per grid and slot: energy change (fixed point, 2^-28), acceptance count
    unsigned* ticket;         // per grid and slot: tiles done, zero between uses
    unsigned* sched;          // work-item counter and blocks-done counter, zero between launches
    unsigned* tdone;          // per tile index: sweeps completed (absolute counter)
    int* live;                // relaxation: grids still relaxing
    double* ehist;
    int ehist_stride;
    int ntiles;
    int n_ent;
    int nsweeps;              // sweeps of this launch
    int cfg;                  // compiled tile configuration
    int relax;                // Algorithm 2 step 5 (window from Ctl, grids stop) or a fixed window
    float half_qd_fixed;
    int or_mode;              // over-relaxation: OR_CONSERVING, OR_LITERAL or OR_NONE
    RoundKeys rk;             // Philox round keys of the seed
    int mode;
    double A_targ, k_a;
    int n_f, n_fit, i_max;
    unsigned long long wait_ns;   // limit of every inter-block wait
    int stall;                // test support: block 0 first waits on a flag that nothing sets
    unsigned long long* trace;        // bench support: per-item timestamps (mpr_debug_trace), or nullptr
    unsigned long long trace_items;   // items the trace holds before its control-step area
};
constexpr int kTraceWords = 6;        // per work item of the trace
constexpr int kTraceCtl = 4096;       // control steps of the trace (by sweep counter modulo this)

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
    int or_mode;              // over-relaxation: OR_CONSERVING, OR_LITERAL or OR_NONE
    int f64;                  // lattice of double2 and FP64 arithmetic (MPR_PREC_F64)
    int genq;                 // q < 1/2: the arc tests and turns of hybrid_update<., true>
    double half_qd_fixed64;   // q * pi / a for the fixed window, FP64 path
    RoundKeys rk;             // Philox round keys of the seed
};


// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
    // Philox4x32-10, Salmon et al. (SC'11): 10 rounds, Weyl key schedule.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product per multiplier gives both halves
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same with precomputed round keys.
__device__ __forceinline__ uint4 philox10(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[r], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ float u24f(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

// Random numbers of a sweep's site update: Philox4x32-10 at the counter
// {y ceil(W/4) + floor(x/4), sweep, chain, colour}.  Of the four columns 4 floor(x/4) .. +3
// of row y, two sites have the colour; the one with floor(x/2) even takes words (0, 1), the
// other words (2, 3): proposal uniform first, acceptance uniform second.
__device__ __forceinline__ uint32_t quad_index(int W, int y, int x) {
    return (uint32_t)y * (uint32_t)((W + 3) >> 2) + (uint32_t)(x >> 2);
}

// The FP32 paths add energy changes in fixed point: each site's change is rounded to a
// whole number of kDEUnit = 2^-17 where it is computed, and those integers are summed.
// Integer sums are exact and associative, so a sweep's total is the same whichever
// kernel, tile shape, thread count or strip decomposition produced it.  The rounding is
// one FP32 addition: for |d| < 32, d + 96 lies in [64, 128), where FP32 numbers are spaced
// 2^-17 apart, so the sum is d rounded to nearest (even) and its bit pattern minus that of
// 96 is the rounded value in units.  |dH| <= 16 per update (8 from the proposal, 8 more
// from the printed reflection), so one site is below 2^21 units and 511 sites fit in a
// 32-bit partial.
constexpr double kDEUnit = 1.0 / 131072.0;
constexpr int kDEMaxSites32 = 511;
__device__ __forceinline__ int de_fixed(float d) { return __float_as_int(__fadd_rn(d, 96.0f)) - 0x42C00000; }
// a total held as a double (a whole number of units below 2^53) back to its integer
__device__ __forceinline__ long long de_units(double d) { return __double2ll_rn(d * 131072.0); }

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

// theta = atan2(s, c) for a point (c, s) of the closed upper half plane (s >= 0), in
// [0, pi]: reduction to x = min(|c|, s) / max(|c|, s) in [0, 1]; atan(x) = x P(x^2) with P
// of degree 7 fitted by csrc/fit_atan.py (least squares on Chebyshev nodes refined by
// Lawson's iteration towards the minimax fit; the FP32 evaluation is within 1.8e-7 of
// atan on [0, 1]); then pi/2 - a above the diagonal and pi - a for c < 0.  With the
// 2-ulp quotient the result is within 4e-7 rad of the exact angle.  (0, 0) gives 0.
__device__ __forceinline__ float angle_upper(float c, float s) {
    const float ac = fabsf(c);
    const float lo = fminf(ac, s), hi = fmaxf(ac, s);
    const float x = hi > 0.0f ? __fdividef(lo, hi) : 0.0f;
    const float t = x * x;
    float p = -4.781315569e-03f;
    p = fmaf(p, t, 2.456034347e-02f);
    p = fmaf(p, t, -5.990952626e-02f);
    p = fmaf(p, t, 9.943124652e-02f);
    p = fmaf(p, t, -1.402956843e-01f);
    p = fmaf(p, t, 1.997140646e-01f);
    p = fmaf(p, t, -3.333209753e-01f);
    p = fmaf(p, t, 9.999999404e-01f);
    float a = p * x;
    a = s > ac ? 1.5707963267948966f - a : a;
    return c < 0.0f ? 3.1415926535897932f - a : a;
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

// ---------------------------------------------------------------- the site update
enum { TRIG_ACCURATE = 0, TRIG_FAST = 1 };

// Over-relaxation modes (the values of mpr_params::or_mode).
enum { OR_CONSERVING = 0, OR_LITERAL = 1, OR_NONE = 2 };

// One gap-site update (Algorithm 1) in unit-vector form, theta = q phi (q = 1/2: in [0, pi)).
//   v        current (cos theta, sin theta) of the site
//   C, S     local field: sums of the neighbours' cos/sin
//   Fx, Fy   OR_LITERAL only: sum of the neighbours' (cos phi_j, sin phi_j) = (cos 2 theta_j,
//            sin 2 theta_j), the field of the reflection as Eq. 6 prints it
//   hq       half the proposal rotation, q * 2 pi (u - 1/2) / a / 2
//   r        acceptance uniform
//   kx       -1/T (TRIG_ACCURATE: the test uses expf) or -log2(e)/T (TRIG_FAST: ex2.approx)
//   or_mode  OR_CONSERVING (reflection about the MPR field), OR_LITERAL, OR_NONE
// Returns the energy change of the update (the reflection's, which is 0 unless OR_LITERAL,
// plus the proposal's if accepted) and writes the new vector.  The conserving path is
// written without branches: both outcomes of each test are computed and selected.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// theta of (c, s) in [0, Q), Q = 2 pi q <= pi: on the upper half circle (theta = 0
// included) and before (cQ, sQ), i.e. sin(Q - theta) > 0.
__device__ __forceinline__ bool in_arc(float c, float s, float cQ, float sQ) {
    return (s > 0.0f || (s == 0.0f && c > 0.0f)) && (s == 0.0f || fmaf(sQ, c, -(cQ * s)) > 0.0f);
}
__device__ __forceinline__ bool in_arc(double c, double s, double cQ, double sQ) {
    return (s > 0.0 || (s == 0.0 && c > 0.0)) && (s == 0.0 || fma(sQ, c, -(cQ * s)) > 0.0);
}

// GQ (q < 1/2): theta lives on the arc [0, Q); the reflection is kept only inside it, and
// the proposal's modulo 2 pi in phi is a turn by -Q above the arc or +Q below it (the step
// is at most pi q / a <= Q / 2, so one turn lands inside); dH is then taken from the new
// vector.  Without GQ (q = 1/2, Q = pi) the arc is the upper half circle and the turn a
// negation, written out below without the general tests.
template <int TRIG, bool GQ = false>
__device__ __forceinline__ float hybrid_update(float2& v, float C, float S, float Fx, float Fy, float hq,
                                               float r, float kx, int or_mode, bool& accepted,
                                               float cQ = -1.0f, float sQ = 0.0f) {
    float c = v.x, s = v.y;
    float dE_or = 0.0f;
    if (or_mode == OR_LITERAL) {
        // Eq. 6 as printed: phi' = 2 Psi - phi (mod 2 pi), Psi the direction of (Fx, Fy);
        // theta' = Psi - theta (mod pi).  It moves the local energy; that change is counted.
        const float F2 = fmaf(Fx, Fx, Fy * Fy);
        if (F2 > 1e-12f) {
            const float inv = rsqrtf(F2);
            const float cp = Fx * inv, sp = Fy * inv;
            float cl = fmaf(cp, c, sp * s), sl = fmaf(sp, c, -(cp * s));
            if (sl < 0.0f || (sl == 0.0f && cl < 0.0f)) {
                cl = -cl;
                sl = -sl;
            }
            dE_or = fmaf(c, C, s * S) - fmaf(cl, C, sl * S);     // local energy is -R cos(theta - psi)
            c = cl;
            s = sl;
        }
    }
    // R cos(theta - psi) and R sin(theta - psi), psi the direction of the field
    const float along = fmaf(c, C, s * S);
    const float perp0 = fmaf(s, C, -(c * S));
    // Eq. 6 (energy-conserving reading): reflect theta about psi; keep it only if the
    // image stays in [0, pi), i.e. sin > 0 or theta = 0 (the point theta = pi is excluded).
    // No reflection when the field vanishes (R^2 <= 1e-12).
    const float R2 = fmaf(C, C, S * S);
    // reflection factor 2 (v.n)/|n|^2; a 2-ulp quotient moves the image by ~2e-7 rad
    const float f = __fdividef(2.0f * along, R2);
    const float cr = fmaf(f, C, -c), sr = fmaf(f, S, -s);
    const bool refl = or_mode == OR_CONSERVING && R2 > 1e-12f &&
                      (GQ ? in_arc(cr, sr, cQ, sQ) : (sr > 0.0f || (sr == 0.0f && cr > 0.0f)));
    c = refl ? cr : c;
    s = refl ? sr : s;
    const float perp = refl ? -perp0 : perp0;     // the reflection keeps `along`, flips `perp`
    // proposal: rotate by 2*hq (steps 2-3); 1 - cos and sin of the rotation from the half angle
    float sh, ch;
    if (TRIG == TRIG_FAST) {
        __sincosf(hq, &sh, &ch);
    } else {
        sincos_quarter(hq, &sh, &ch);
    }
    const float sn = 2.0f * sh * ch;
    const float hh = 2.0f * sh * sh;
    // step 4: dH = R [cos(theta - psi) - cos(theta + 2hq - psi)]
    const float dH0 = fmaf(hh, along, sn * perp);
    const float c20 = c - fmaf(c, hh, s * sn);
    const float s20 = s - fmaf(s, hh, -(c * sn));
    float c2, s2, dH;
    if (GQ) {
        const bool inside = in_arc(c20, s20, cQ, sQ);
        const bool below = !inside && s20 < 0.0f && c20 > 0.0f;
        const float sb = below ? sQ : -sQ;                     // sin of the turn +-Q
        c2 = inside ? c20 : fmaf(c20, cQ, -(s20 * sb));
        s2 = inside ? s20 : fmaf(c20, sb, s20 * cQ);
        dH = inside ? dH0 : along - fmaf(c2, C, s2 * S);
    } else {
        // modulo 2 pi in phi is a half turn in theta: negate the vector, dH -> 2 along - dH
        const bool wrap = s20 < 0.0f || (s20 == 0.0f && c20 < 0.0f);
        c2 = wrap ? -c20 : c20;
        s2 = wrap ? -s20 : s20;
        dH = wrap ? 2.0f * along - dH0 : dH0;
    }
    // steps 5-6: accept if min(1, exp(-dH/T)) > r
    const float ap = (TRIG == TRIG_FAST) ? ex2_approx(dH * kx) : expf(dH * kx);
    accepted = (dH <= 0.0f) || (ap > r);
    c = accepted ? c2 : c;
    s = accepted ? s2 : s;
    // one Newton step back to unit length (rounding drift of reflections and rotations)
    const float g = fmaf(-0.5f, fmaf(c, c, s * s), 1.5f);
    v = make_float2(c * g, s * g);
    return (accepted ? dH : 0.0f) + dE_or;
}

// The same update in FP64 (MPR_PREC_F64): the steps and the unit-vector form above, with
// exact division, the reflection about the field for any nonzero field, and the library's
// double sin, cos and exp.
//   neg_inv_T  -1/T
template <bool GQ = false>
__device__ __forceinline__ double hybrid_update64(double2& v, double C, double S, double Fx, double Fy,
                                                  double hq, double r, double neg_inv_T, int or_mode,
                                                  bool& accepted, double cQ = -1.0, double sQ = 0.0) {
    double c = v.x, s = v.y;
    double dE_or = 0.0;
    if (or_mode == OR_LITERAL) {
        const double F2 = fma(Fx, Fx, Fy * Fy);
        if (F2 > 0.0) {
            const double inv = 1.0 / sqrt(F2);
            const double cp = Fx * inv, sp = Fy * inv;
            double cl = fma(cp, c, sp * s), sl = fma(sp, c, -(cp * s));
            if (sl < 0.0 || (sl == 0.0 && cl < 0.0)) {
                cl = -cl;
                sl = -sl;
            }
            dE_or = fma(c, C, s * S) - fma(cl, C, sl * S);
            c = cl;
            s = sl;
        }
    }
    const double along = fma(c, C, s * S);
    const double perp0 = fma(s, C, -(c * S));
    const double R2 = fma(C, C, S * S);
    bool refl = false;
    if (or_mode == OR_CONSERVING && R2 > 0.0) {
        const double f = 2.0 * along / R2;
        const double cr = fma(f, C, -c), sr = fma(f, S, -s);
        refl = GQ ? in_arc(cr, sr, cQ, sQ) : (sr > 0.0 || (sr == 0.0 && cr > 0.0));
        if (refl) {
            c = cr;
            s = sr;
        }
    }
    const double perp = refl ? -perp0 : perp0;
    double sh, ch;
    sincos(hq, &sh, &ch);
    const double sn = 2.0 * sh * ch;
    const double hh = 2.0 * sh * sh;
    const double dH0 = fma(hh, along, sn * perp);
    const double c20 = c - fma(c, hh, s * sn);
    const double s20 = s - fma(s, hh, -(c * sn));
    double c2, s2, dH;
    if (GQ) {
        const bool inside = in_arc(c20, s20, cQ, sQ);
        const bool below = !inside && s20 < 0.0 && c20 > 0.0;
        const double sb = below ? sQ : -sQ;
        c2 = inside ? c20 : fma(c20, cQ, -(s20 * sb));
        s2 = inside ? s20 : fma(c20, sb, s20 * cQ);
        dH = inside ? dH0 : along - fma(c2, C, s2 * S);
    } else {
        const bool wrap = s20 < 0.0 || (s20 == 0.0 && c20 < 0.0);
        c2 = wrap ? -c20 : c20;
        s2 = wrap ? -s20 : s20;
        dH = wrap ? 2.0 * along - dH0 : dH0;
    }
    accepted = (dH <= 0.0) || (exp(dH * neg_inv_T) > r);
    c = accepted ? c2 : c;
    s = accepted ? s2 : s;
    const double g = fma(-0.5, fma(c, c, s * s), 1.5);
    v = make_double2(c * g, s * g);
    return (accepted ? dH : 0.0) + dE_or;
}

// The field of Eq. 6 as printed (OR_LITERAL): sum of the four neighbours' (cos 2 theta,
// sin 2 theta) from their unit vectors (cos theta, sin theta).
__device__ __forceinline__ void literal_field(float2 a, float2 b, float2 c, float2 d, float& Fx, float& Fy) {
    Fx = (fmaf(a.x, a.x, -a.y * a.y) + fmaf(b.x, b.x, -b.y * b.y)) +
         (fmaf(c.x, c.x, -c.y * c.y) + fmaf(d.x, d.x, -d.y * d.y));
    Fy = 2.0f * ((a.x * a.y + b.x * b.y) + (c.x * c.y + d.x * d.y));
}

__device__ __forceinline__ void literal_field64(double2 a, double2 b, double2 c, double2 d, double& Fx,
                                                double& Fy) {
    Fx = (fma(a.x, a.x, -a.y * a.y) + fma(b.x, b.x, -b.y * b.y)) +
         (fma(c.x, c.x, -c.y * c.y) + fma(d.x, d.x, -d.y * d.y));
    Fy = 2.0 * ((a.x * a.y + b.x * b.y) + (c.x * c.y + d.x * d.y));
}

// The exponent scale kx of hybrid_update for a temperature given as -1/T.
template <int TRIG>
__device__ __forceinline__ float accept_scale(float neg_inv_T) {
    return TRIG == TRIG_FAST ? neg_inv_T * 1.4426950408889634f : neg_inv_T;
}

// ---------------------------------------------------------------- Algorithm 2 control
// One sweep's bookkeeping for one grid, given the sweep's accepted energy change dH and
// acceptance count na.  flip_cur: the sweep wrote the other lattice buffer (tile path).
//   CTL_RELAX : step 5 (window 5.2, energy 5.3, slope 5.4 every n_f sweeps, counter 5.5)
//   CTL_FIXED : energy, acceptance and sweep counter of a fixed-window sweep
//   CTL_SAMPLE: as FIXED, and e accumulated for the e(T, L) table average
__device__ __forceinline__ void control_step(Ctl& c, const EntryDesc& E, double dH,
                                             unsigned long long na, int mode, double A_targ,
                                             double k_a, int n_f, int n_fit, int i_max,
                                             double* eh, int flip_cur) {
    if (mode == CTL_RELAX) {
        if (c.stop) return;
        c.H += dH;
        const double A = E.P ? (double)na / (double)E.P : 0.0;
        if (A < A_targ) {                                                  // 5.2
            c.a = 1.0 + (double)(c.i + 1) / k_a;
            c.half_qd = (float)(0.5 * kTwoPi * E.q / c.a);
        }
        const double en = c.H / E.ngp;                                     // 5.3
        eh[c.i + 1] = en;
        if (c.i >= n_fit && c.i % n_f == 0) {                              // 5.4
            const double* w = eh + (c.i + 2 - n_fit);
            const double tbar = 0.5 * (double)(n_fit - 1);
            // least-squares slope of the last n_fit values; the history is read in chunks
            // of 8 independent loads and added in index order
            double ebar = 0.0;
            for (int t0 = 0; t0 < n_fit; t0 += 8) {
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = t0 + j < n_fit ? w[t0 + j] : 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (t0 + j < n_fit) ebar += v[j];
            }
            ebar /= (double)n_fit;
            double num = 0.0, den = 0.0;
            for (int t0 = 0; t0 < n_fit; t0 += 8) {
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = t0 + j < n_fit ? w[t0 + j] : 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (t0 + j < n_fit) {
                        const double dt = (double)(t0 + j) - tbar;
                        num += dt * (v[j] - ebar);
                        den += dt * dt;
                    }
                }
            }
            c.k = num / den;
        }
        c.i += 1;                                                          // 5.5
        c.sweep += 1u;
        c.A_last = A;
        c.e_last = en;
        if (flip_cur) c.cur ^= 1;
        if (!(c.k < 0.0 && c.i <= i_max)) {
            c.stop = 1;
            c.converged = c.k >= 0.0 ? 1 : 0;
        }
        ctl_set_go(c);
        return;
    }
    c.H += dH;
    c.A_last = E.P ? (double)na / (double)E.P : 0.0;
    c.e_last = c.H / E.ngp;
    if (mode == CTL_SAMPLE) {
        c.esum += c.e_last;
        c.nsamp += 1;
    }
    c.sweep += 1u;
    if (flip_cur) c.cur ^= 1;
    ctl_set_go(c);
}

// ---------------------------------------------------------------- launchers
// init (mpr_init.cu)
cudaError_t launch_minmax(const float* z, const uint8_t* mask, long long n, unsigned* keys,
                          unsigned long long* nsamples, cudaStream_t st);
// f64: the lattice holds double2 vectors (same element offsets, twice the bytes).
cudaError_t launch_pack(const EntryDesc* e_host, const float* z, const uint8_t* mask,
                        double zmin, double scale, float2* lat, uint32_t key0, uint32_t key1,
                        int all_free, bool f64, cudaStream_t st);
cudaError_t launch_gap_count(const EntryDesc* e_host, const uint8_t* mask, int all_free,
                             int* row_counts, cudaStream_t st);
cudaError_t launch_scan_rows(int* row_counts, int nrows, int narrays, int* totals,
                             cudaStream_t st);
cudaError_t launch_gap_scatter(const EntryDesc* e_host, const uint8_t* mask, int all_free,
                               const int* row_offsets, uint32_t* gaps, cudaStream_t st);
// Eq. 4 partial sums: per block (sum of cosines, pair count) into part[block] (grid <= 1024).
// f64: cosine arguments and row sums in FP64.
// y_end: only pairs whose upper or left site lies in rows [0, y_end) (a strip's own rows;
// e_host->H otherwise).
cudaError_t launch_sample_energy(const EntryDesc* e_host, const float* z, const uint8_t* mask,
                                 double scale, double q, double* part_sum,
                                 unsigned long long* part_cnt, int* nparts, bool f64, cudaStream_t st,
                                 int y_end = -1);
cudaError_t launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, size_t n,
                          cudaStream_t st);

// The same set-up steps for every grid of a batch in one launch each (grid i of the launch
// = blockIdx.y): a device table of SetupRec (and of the batch's EntryDesc where the step
// needs the lattice layout).  Per grid the work and its partition are those of the
// single-grid launchers above, so the results are the same bit for bit.
struct SetupRec {
    const float* z;           // the grid's data (device; null for all-free lattices)
    const uint8_t* mask;      // 1 = sample (device; null for all-free lattices)
    double zmin, scale;       // Eq. 1
    long long n;              // sites
    int roff;                 // first of its 2 H row counts (gap lists)
    int poff, nparts;         // its Eq. 4 partials: first, count
};
cudaError_t launch_minmax_batch(const SetupRec* recs, int n, long long max_sites, unsigned* keys,
                                unsigned long long* nsamples, cudaStream_t st);
cudaError_t launch_pack_batch(const EntryDesc* ents, const SetupRec* recs, int n, long long max_sites,
                              float2* lat, uint32_t key0, uint32_t key1, int all_free, bool f64,
                              cudaStream_t st);
cudaError_t launch_gap_count_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_rows,
                                   int all_free, int* row_counts, cudaStream_t st);
cudaError_t launch_scan_rows_batch(const EntryDesc* ents, const SetupRec* recs, int n, int* row_counts,
                                   int* totals, cudaStream_t st);
cudaError_t launch_gap_scatter_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_rows,
                                     int all_free, const int* row_offsets, uint32_t* gaps, cudaStream_t st);
cudaError_t launch_sample_energy_batch(const EntryDesc* ents, const SetupRec* recs, int n, int max_parts,
                                       double q, double* part_sum, unsigned long long* part_cnt, bool f64,
                                       cudaStream_t st);

// tile path (mpr_tile.cu)
TileGeom tile_geom(int cfg);
int tile_config_count();
int tile_max_rows();
int tile_max_cols();
int tile_sweep_blocks(int cfg);
cudaError_t make_tile_maps(int cfg, const EntryDesc* ents, int n_ent, float2* lat0, float2* lat1,
                           CUtensorMap* d_maps, cudaStream_t st);
cudaError_t launch_tile_lists(int cfg, TileDesc* tiles, int ntiles, const EntryDesc* ents,
                              const uint8_t* mask, int all_free, uint16_t* lists, TileCnt* cnts,
                              cudaStream_t st);
cudaError_t launch_tile_sweep(const TileArgs& a, int trig, cudaStream_t st);
// ord <- the tiles of every grid, heaviest first (grids contiguous, in entry order); hist:
// n_ent * 256 unsigned of scratch.  Needs the gap counts of every tile filled in.
cudaError_t launch_tile_order(const TileDesc* tiles, int ntiles, const EntryDesc* ents, int n_ent,
                              int cfg, unsigned* hist, TileDesc* ord, cudaStream_t st);
// tdone[t] <- the sweep counter of tile t's grid; and every grid's launch base <- its
// current sweep counter and buffer
cudaError_t launch_tile_sync(const TileDesc* tiles, int ntiles, Ctl* ctl, int n_ent, unsigned* tdone,
                             cudaStream_t st);
// *live <- number of grids whose relaxation has not stopped
cudaError_t launch_count_live(const Ctl* ctl, int n_ent, int* live, cudaStream_t st);
// K > 1: the angle sums of K chains of one grid, chain c's tiles at tile + c * chain_tiles.
// zr (device, one (z_min, z_max) per entry) replaces zmin, zmax when not null.
cudaError_t launch_tile_predict_out(int cfg, const TileDesc* tiles, const TileCnt* cnts,
                                    const uint16_t* lists, const float* acc, const EntryDesc* ents,
                                    int tile0, int ntiles, int M, double q, double zmin, double zmax,
                                    const double2* zr, int K, int chain_tiles, float* zhat, cudaStream_t st);

// sweeps (mpr_sweep.cu)
cudaError_t launch_half_sweep(const SweepArgs& a, int color, int trig, cudaStream_t st);
cudaError_t launch_control(Ctl* ctl, Part* const part[2], const EntryDesc* ents, int n_ent,
                           int mode, double A_targ, double k_a, int n_f, int n_fit, int i_max,
                           double* ehist, int ehist_stride, int* active, bool f64, cudaStream_t st);
// Eq. 2 of one grid: per-block partials then a fixed-order sum into *out (deterministic).
// [y_a, y_b): only the bonds of the colour-0 sites of these rows (every bond has one
// colour-0 end); the whole grid by default.
cudaError_t launch_energy(const EntryDesc* e_host, const float2* lat, double* scratch,
                          int scratch_len, double* out, bool f64, cudaStream_t st, int y_a = 0,
                          int y_b = -1);
// The same for every grid of a batch in two launches: grid i reads lattice buffer 1 where
// tiled and ctl[i].cur are set, else buffer 0; its partials go to scratch + i scratch_len
// (the single-grid launch's blocks and order), its H to out[i].
cudaError_t launch_energy_batch(const EntryDesc* ents, int n, int max_cols, int max_rows, const float2* lat0,
                                const float2* lat1, const Ctl* ctl, int tiled, double* scratch,
                                int scratch_len, double* out, bool f64, cudaStream_t st);
// Row strips: out[0] (color 0: =, color 1: +=) the colour's accepted energy change, out[1]
// its acceptance count, summed over the half-sweep blocks in block order (FP32 partials as
// exact integer sums of kDEUnit).
cudaError_t launch_strip_partials(const Part* part, int nblk, int color, double* out, bool f64,
                                  cudaStream_t st);
// Row strips: one control step of entry 0 from the totals {dH, n_acc} of all strips, with
// the whole grid's gap count P and bond count ngp; *stop_dev <- the relaxation has ended.
cudaError_t launch_strip_control(Ctl* ctl, const EntryDesc* e_host, double P, double ngp, const double* tot,
                                 int mode, double A_targ, double k_a, int n_f, int n_fit, int i_max,
                                 double* ehist, int* stop_dev, cudaStream_t st);
cudaError_t launch_sum(const double* v, int n, double* out, cudaStream_t st);
cudaError_t launch_set_tracked_energy(Ctl* ctl, const double* H, int n_ent, cudaStream_t st);
// f64: acc holds doubles (same element offsets).
cudaError_t launch_predict_out(const EntryDesc* e_host, const float2* lat, const uint32_t* gaps,
                               const float* acc, int M, double q, double zmin, double zmax,
                               float* zhat, bool f64, cudaStream_t st);
cudaError_t launch_get_state(const EntryDesc* e_host, const float2* lat, float* phi, bool f64,
                             cudaStream_t st);
cudaError_t launch_get_state64(const EntryDesc* e_host, const float2* lat, double* phi, bool f64,
                               cudaStream_t st);
cudaError_t launch_set_state(const EntryDesc* e_host, float2* lat, const uint32_t* gaps,
                             const float* phi, bool f64, cudaStream_t st);

}  // namespace mpr
