/*
 * mpr_oracle.c -- plain, slow FP64 reference of the MPR gap-filling method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only on seeded inputs.
 *
 * Paper: Zukovic, Borovsky, Lach, Hristopulos, "GPU-accelerated Simulation of
 * Massive Spatial Data based on the Modified Planar Rotator Model".
 *
 * Every function follows the paper's definition or algorithm step by step, in
 * double precision, with no blocking or reordering.  Readings of points the
 * paper leaves open are marked READING and listed in the design notes:
 *   R-OR   over-relaxation: reflection about the MPR local field, kept only
 *          when the reflected angle stays in [0, 2pi) (Eq. 6 reading).
 *   R-ES   sample specific energy: each unordered sample pair counted once.
 *   R-NGP  N_GP = W(H-1) + H(W-1); H sums over all nearest-neighbour bonds.
 *   R-SG   SG slope = least-squares linear slope of the last n_fit energies.
 *   R-RNG  Philox4x32-10, key = 64-bit seed.  In a sweep, site (x, y) of colour
 *          k = (x + y) & 1 draws from the counter {y ceil(W/4) + floor(x/4),
 *          sweep, chain, k}: of the four columns 4 floor(x/4) .. +3 of row y two
 *          sites have colour k; the one with floor(x/2) even takes words
 *          (o0, o1), the other (o2, o3); u = (first >> 8) 2^-24 is the
 *          proposal uniform, r = (second >> 8) 2^-24 the acceptance uniform.
 *          Initial gap angles: counter {y W + x, 0xFFFFFFFF, chain, 0}, o0.
 *   R-TAB  e(T,L): K_T log-spaced temperatures, all-free lattices started
 *          from U(0,2pi), Algorithm 2 step 5 relaxation, then M_T sweeps at
 *          the step-6 window; T-hat by piecewise-linear interpolation in T.
 *   R-WRAP proposals wrap modulo 2pi into [0, 2pi).
 *   R-CH   independent chains: the equilibrated state forked into K chains with
 *          chain words chain + k 2^24, all from the same sweep counter; the
 *          estimate averages all K * M_per_chain realizations.
 *   R-Q    couplings q in (0, 1/2] (Eq. 2 bounds q by 1/2): every step is written
 *          for a general q; the reflection is kept only inside [0, 2pi).
 *
 * Parity unpinned: the default values of the run-length parameters (A_targ,
 * k_a, n_f, n_fit, i_max, M) and of the table (K_T, T range, lattice size,
 * M_T).  The paper defers them to earlier work; they change how long the
 * chains run, not the law they sample, and no closed form fixes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO_PI 6.283185307179586476925286766559

enum { ORC_OR_CONSERVING = 0, ORC_OR_LITERAL = 1, ORC_OR_NONE = 2 };

/* Parameters of Algorithm 2, step 1.1, plus the readings above. */
typedef struct {
    uint64_t seed;
    double q;        /* coupling, Sect. 2.2 (q = 1/2 in the paper) */
    double A_targ;   /* target acceptance ratio */
    double k_a;      /* rate of the window factor a */
    int n_f;         /* equilibrium check period */
    int n_fit;       /* number of energies in the slope fit */
    int i_max;       /* cap on relaxation sweeps */
    int M;           /* equilibrium realizations */
    int or_mode;     /* ORC_OR_* */
    double a_eq;     /* window factor of step 6 (the paper uses 1) */
    int KT;          /* number of table temperatures */
    double T_min, T_max;
    int T_W, T_H;    /* size of the unconditional lattices */
    int M_T;         /* sweeps averaged per table temperature */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds of two     */
/* 32x32->64 multiplications with the Weyl-sequence key schedule.            */
/* The paper draws its random numbers from this generator (Sect. 3.3).       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n counters (4 words each) -> n output blocks; key from a 64-bit seed. */
void orc_philox_batch(const uint32_t* ctr, uint64_t seed, uint32_t* out, long n)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (long i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* 24-bit uniform in [0,1): exactly representable in FP32 and FP64. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* READING R-RNG: the two uniforms of a sweep's update of site (x, y) (y counted in the
 * whole grid) of a W-wide grid. */
static void site_randoms(uint64_t seed, int W, int x, int y, uint32_t sweep, uint32_t chain,
                         double* u, double* r)
{
    const uint32_t quads = (uint32_t)((W + 3) / 4);
    const uint32_t color = (uint32_t)((x + y) & 1);
    uint32_t ctr[4] = { (uint32_t)y * quads + (uint32_t)(x / 4), sweep, chain, color };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    const int second = (x / 2) & 1;
    *u = u24(o[second ? 2 : 0]);
    *r = u24(o[second ? 3 : 1]);
}

/* Initial gap angle uniform of site index i (READING R-RNG). */
static double init_uniform(uint64_t seed, uint32_t i, uint32_t chain)
{
    uint32_t ctr[4] = { i, 0xFFFFFFFFu, chain, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return u24(o[0]);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: linear map of the sample values to angles in [0, 2pi].            */
/* mask[i] = 1 marks a sample site, 0 a gap (prediction) site.              */
/* Returns the number of samples; phi of gap sites is left untouched.       */
/* ------------------------------------------------------------------------ */
long orc_map(const float* z, const uint8_t* mask, int W, int H, double* phi,
             double* zmin_out, double* zmax_out)
{
    long n = (long)W * H, ns = 0;
    double zmin = INFINITY, zmax = -INFINITY;
    for (long i = 0; i < n; ++i) {
        if (!mask[i]) continue;
        double v = (double)z[i];
        if (v < zmin) zmin = v;
        if (v > zmax) zmax = v;
        ++ns;
    }
    *zmin_out = zmin;
    *zmax_out = zmax;
    if (ns < 2 || !(zmax > zmin)) return ns;
    for (long i = 0; i < n; ++i) {
        if (!mask[i]) continue;
        double t = (double)z[i] - zmin;
        t = t * ORC_TWO_PI;
        phi[i] = t / (zmax - zmin);
    }
    return ns;
}

/* Inverse of Eq. 1 (Algorithm 2, step 6.3). */
double orc_unmap(double phi, double zmin, double zmax)
{
    return zmin + phi * (zmax - zmin) / ORC_TWO_PI;
}

/* ------------------------------------------------------------------------ */
/* Eq. 4: sample specific energy over nearest-neighbour sample pairs        */
/* (READING R-ES: each unordered pair once, so e_s lies in [-1, 1]).        */
/* ------------------------------------------------------------------------ */
double orc_sample_energy(const double* phi, const uint8_t* mask, int W, int H, double q,
                         long long* nsp_out)
{
    double sum = 0.0;
    long long nsp = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            if (!mask[i]) continue;
            if (x + 1 < W && mask[i + 1]) { sum += cos(q * (phi[i] - phi[i + 1])); ++nsp; }
            if (y + 1 < H && mask[i + W]) { sum += cos(q * (phi[i] - phi[i + W])); ++nsp; }
        }
    *nsp_out = nsp;
    return nsp ? -sum / (double)nsp : 0.0;
}

/* Eq. 2 with J = 1: H = -sum over nearest-neighbour bonds cos(q(phi_i-phi_j)). */
double orc_energy(const double* phi, int W, int H, double q)
{
    double h = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            if (x + 1 < W) h -= cos(q * (phi[i] - phi[i + 1]));
            if (y + 1 < H) h -= cos(q * (phi[i] - phi[i + W]));
        }
    return h;
}

/* READING R-NGP: number of nearest-neighbour pairs of a W x H open grid. */
long orc_n_gp(int W, int H) { return (long)W * (H - 1) + (long)H * (W - 1); }

/* Contribution of one site with angle v to Eq. 2, given its neighbours. */
double orc_local_energy(double v, const double* nb, int nnb, double q)
{
    double e = 0.0;
    for (int j = 0; j < nnb; ++j) e -= cos(q * (v - nb[j]));
    return e;
}

/* ------------------------------------------------------------------------ */
/* Eq. 6, over-relaxation.                                                   */
/* CONSERVING (READING R-OR): psi = atan2(sum sin(q phi_j), sum cos(q phi_j))*/
/*   is the direction of the MPR local field; the reflection q phi* =        */
/*   2 psi - q phi leaves the local energy unchanged.  It is applied only    */
/*   if phi* lies in [0, 2pi); otherwise, or if the field vanishes, the      */
/*   angle is kept.  The map is an involution with unit Jacobian.            */
/* LITERAL: the printed formula (the q = 1 reflection, then mod 2pi).        */
/* ------------------------------------------------------------------------ */
double orc_over_relax(double phi, const double* nb, int nnb, double q, int mode)
{
    if (mode == ORC_OR_NONE) return phi;
    if (mode == ORC_OR_LITERAL) {
        double s = 0.0, c = 0.0;
        for (int j = 0; j < nnb; ++j) { s += sin(nb[j]); c += cos(nb[j]); }
        if (s == 0.0 && c == 0.0) return phi;
        double v = fmod(2.0 * atan2(s, c) - phi, ORC_TWO_PI);
        if (v < 0.0) v += ORC_TWO_PI;
        if (v >= ORC_TWO_PI) v -= ORC_TWO_PI;
        return v;
    }
    double s = 0.0, c = 0.0;
    for (int j = 0; j < nnb; ++j) { s += sin(q * nb[j]); c += cos(q * nb[j]); }
    if (s == 0.0 && c == 0.0) return phi;
    double psi = atan2(s, c);
    double v = (2.0 * psi - q * phi) / q;
    if (v >= 0.0 && v < ORC_TWO_PI) return v;
    return phi;
}

/* Angles of the in-grid nearest neighbours of (x, y) (open boundaries). */
static int gather_nb(const double* phi, int W, int H, int x, int y, double nb[4])
{
    int n = 0;
    long i = (long)y * W + x;
    if (x > 0) nb[n++] = phi[i - 1];
    if (x + 1 < W) nb[n++] = phi[i + 1];
    if (y > 0) nb[n++] = phi[i - W];
    if (y + 1 < H) nb[n++] = phi[i + W];
    return n;
}

/* Decision flags recorded per site (for parity checks). */
enum { ORC_F_REFLECTED = 1, ORC_F_WRAPPED = 2, ORC_F_ACCEPTED = 4, ORC_F_VISITED = 8 };

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on one gap site: over-relaxation, restricted Metropolis       */
/* proposal phi'' = phi' + 2pi(u-1/2)/a (mod 2pi), energy change against     */
/* the current neighbours, acceptance if min(1, exp(-dH/T)) > r.             */
/* ------------------------------------------------------------------------ */
static int update_site(double* phi, int W, int H, int x, int y, double a, double T, double q,
                       uint64_t seed, uint32_t chain, uint32_t sweep, int or_mode,
                       double* margin, int row0)
{
    long i = (long)y * W + x;
    double nb[4];
    int nnb = gather_nb(phi, W, H, x, y, nb);
    double u, r;
    site_randoms(seed, W, x, row0 + y, sweep, chain, &u, &r);
    int flags = ORC_F_VISITED;

    double p1 = orc_over_relax(phi[i], nb, nnb, q, or_mode);          /* step 1 */
    if (p1 != phi[i]) flags |= ORC_F_REFLECTED;
    double p2 = p1 + ORC_TWO_PI * (u - 0.5) / a;                       /* steps 2-3 */
    if (p2 < 0.0 || p2 >= ORC_TWO_PI) flags |= ORC_F_WRAPPED;
    while (p2 < 0.0) p2 += ORC_TWO_PI;
    while (p2 >= ORC_TWO_PI) p2 -= ORC_TWO_PI;
    double dH = orc_local_energy(p2, nb, nnb, q) - orc_local_energy(p1, nb, nnb, q); /* 4 */
    double ap = exp(-dH / T);                                           /* step 5 */
    if (ap > 1.0) ap = 1.0;
    if (margin) *margin = ap - r;
    if (ap > r) { phi[i] = p2; flags |= ORC_F_ACCEPTED; }              /* step 6.1 */
    else phi[i] = p1;                                                   /* step 6.2 */
    return flags;
}

/* One hybrid sweep: Algorithm 1 over the gap sites of sub-grid A ((x+y) even)
 * and then of sub-grid B (checkerboard decomposition, Sect. 3.3).  Sites of
 * one colour depend only on the other colour, so row-major order within a
 * colour is as good as any.  Returns the number of accepted proposals.
 * flags/margins (optional, W*H) record each visited site's decisions. */
long orc_sweep(double* phi, const uint8_t* mask, int W, int H, double a, double T, double q,
               uint64_t seed, uint32_t chain, uint32_t sweep, int or_mode,
               uint8_t* flags, double* margins)
{
    long nacc = 0;
    for (int color = 0; color < 2; ++color)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                if (((x + y) & 1) != color) continue;
                long i = (long)y * W + x;
                if (mask[i]) continue;                 /* samples stay frozen */
                double m = 0.0;
                int f = update_site(phi, W, H, x, y, a, T, q, seed, chain, sweep, or_mode, &m, 0);
                if (f & ORC_F_ACCEPTED) ++nacc;
                if (flags) flags[i] = (uint8_t)f;
                if (margins) margins[i] = m;
            }
    return nacc;
}

/* ------------------------------------------------------------------------ */
/* Row strips of one grid: the checkerboard of Sect. 3.3 cut into bands of   */
/* rows.  A block holds rows [row0, row0 + Hb) of a W-wide grid: rows        */
/* [y_a, y_b) of the block are the strip's own, the rows beside them (other  */
/* strips' rows) serve as neighbours only, and the block's first and last    */
/* rows are the grid's edges where the block has no row beyond them.         */
/* ------------------------------------------------------------------------ */

/* Algorithm 1 on the gap sites of colour `color` ((x + row0 + y) & 1, the grid's colour) in
 * rows [y_a, y_b) of a block: the same updates orc_sweep makes to these sites in the whole
 * grid, with the grid's Philox counters (row row0 + y).  Returns the accepted proposals. */
long orc_sweep_rows(double* phi, const uint8_t* mask, int W, int Hb, int row0, int y_a, int y_b,
                    int color, double a, double T, double q, uint64_t seed, uint32_t chain,
                    uint32_t sweep, int or_mode)
{
    long nacc = 0;
    for (int y = y_a; y < y_b; ++y)
        for (int x = 0; x < W; ++x) {
            if (((x + row0 + y) & 1) != color) continue;
            long i = (long)y * W + x;
            if (mask[i]) continue;
            int f = update_site(phi, W, Hb, x, y, a, T, q, seed, chain, sweep, or_mode, NULL, row0);
            if (f & ORC_F_ACCEPTED) ++nacc;
        }
    return nacc;
}

/* Eq. 2 over the bonds whose upper or left end lies in rows [y_a, y_b) of a block (each
 * bond of the grid belongs to exactly one strip this way). */
double orc_energy_rows(const double* phi, int W, int Hb, int y_a, int y_b, double q)
{
    double E = 0.0;
    for (int y = y_a; y < y_b; ++y)
        for (int x = 0; x < W; ++x) {
            long i = (long)y * W + x;
            if (x + 1 < W) E -= cos(q * (phi[i] - phi[i + 1]));
            if (y + 1 < Hb) E -= cos(q * (phi[i] - phi[i + W]));
        }
    return E;
}

/* Algorithm 2 step 2.2: gap angles drawn from U(0, 2pi). */
void orc_init_gaps(double* phi, const uint8_t* mask, int W, int H, uint64_t seed, uint32_t chain)
{
    for (long i = 0; i < (long)W * H; ++i) {
        if (mask[i]) continue;
        phi[i] = ORC_TWO_PI * init_uniform(seed, (uint32_t)i, chain);
    }
}

/* READING R-SG: least-squares slope of e[0..n-1] against the sweep index. */
double orc_sg_slope(const double* e, int n)
{
    double tbar = 0.5 * (double)(n - 1), ebar = 0.0;
    for (int t = 0; t < n; ++t) ebar += e[t];
    ebar /= (double)n;
    double num = 0.0, den = 0.0;
    for (int t = 0; t < n; ++t) {
        num += ((double)t - tbar) * (e[t] - ebar);
        den += ((double)t - tbar) * ((double)t - tbar);
    }
    return num / den;
}

typedef struct {
    int sweeps;      /* relaxation sweeps performed (final i) */
    double a;        /* final window factor */
    double k;        /* final slope */
    double A_last;   /* acceptance ratio of the last sweep */
    double e_last;   /* specific energy after the last sweep */
} orc_equil_out;

/* State of the Algorithm 2 step 5 loop: counter i, slope k, window a, last acceptance A,
 * history of e (e[0] before the first sweep, >= i_max + 2 values). */
typedef struct {
    int i;
    double k, a, A;
    double* e;
} orc_relax;

/* Steps 5.2-5.5 after one sweep in which nacc of the P gap sites accepted their proposal,
 * e_next being the specific energy after it.  Returns 1 while the loop goes on (k < 0 and
 * i <= i_max), 0 when it ends. */
int orc_relax_step(orc_relax* s, long nacc, long P, double e_next, const orc_params* p)
{
    s->A = (double)nacc / (double)P;
    if (s->A < p->A_targ) s->a = 1.0 + (double)(s->i + 1) / p->k_a;   /* 5.2 */
    s->e[s->i + 1] = e_next;                                           /* 5.3 */
    if (s->i >= p->n_fit && s->i % p->n_f == 0)
        s->k = orc_sg_slope(&s->e[s->i + 2 - p->n_fit], p->n_fit);     /* 5.4 */
    s->i += 1;                                                         /* 5.5 */
    return s->k < 0.0 && s->i <= p->i_max;
}

static long count_gaps(const uint8_t* mask, long n)
{
    long p = 0;
    for (long i = 0; i < n; ++i) p += mask[i] ? 0 : 1;
    return p;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 step 5: non-equilibrium relaxation.  *sweep is the global     */
/* sweep counter of this chain (the RNG counter); it advances by one per     */
/* sweep.  ehist (optional, >= i_max + 2 values) receives e(i), i >= 1.      */
/* ------------------------------------------------------------------------ */
int orc_equilibrate(double* phi, const uint8_t* mask, int W, int H, double T,
                    const orc_params* p, uint32_t chain, uint32_t* sweep,
                    orc_equil_out* out, double* ehist)
{
    long P = count_gaps(mask, (long)W * H);
    double ngp = (double)orc_n_gp(W, H);
    int cap = p->i_max + 2;
    double* e = ehist ? ehist : (double*)calloc((size_t)cap, sizeof(double));
    orc_relax s;
    s.i = 0;                         /* step 2.1 */
    s.k = -1.0;                      /* step 2.3 */
    s.a = 1.0;                       /* step 2.4 */
    s.A = 0.0;
    s.e = e;
    e[0] = orc_energy(phi, W, H, p->q) / ngp;
    int go = P > 0 && s.i <= p->i_max;
    while (go) {
        long nacc = orc_sweep(phi, mask, W, H, s.a, T, p->q, p->seed, chain, (*sweep)++,
                              p->or_mode, NULL, NULL);                  /* 5.1 */
        go = orc_relax_step(&s, nacc, P, orc_energy(phi, W, H, p->q) / ngp, p);
    }
    if (out) {
        out->sweeps = s.i; out->a = s.a; out->k = s.k; out->A_last = s.A; out->e_last = e[s.i];
    }
    if (!ehist) free(e);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 steps 6-7: M sweeps at window a_eq, back-transform of each   */
/* realization with the inverse of Eq. 1, and their mean at the gap sites.  */
/* Sample sites return their data value.                                     */
/* ------------------------------------------------------------------------ */
int orc_predict(double* phi, const uint8_t* mask, const float* z, int W, int H, double T,
                const orc_params* p, uint32_t chain, uint32_t* sweep, double zmin, double zmax,
                int M, double* zhat)
{
    long n = (long)W * H;
    double* sum = (double*)calloc((size_t)n, sizeof(double));
    for (int j = 0; j < M; ++j) {
        orc_sweep(phi, mask, W, H, p->a_eq, T, p->q, p->seed, chain, (*sweep)++, p->or_mode,
                  NULL, NULL);                                           /* 6.2 */
        for (long i = 0; i < n; ++i)
            if (!mask[i]) sum[i] += orc_unmap(phi[i], zmin, zmax);       /* 6.3 */
    }
    for (long i = 0; i < n; ++i) zhat[i] = mask[i] ? (double)z[i] : sum[i] / (double)M;
    free(sum);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Independent chains (READING R-CH; the paper's estimator is one chain).    */
/* The state phi is forked into K chains; chain k (Philox chain word        */
/* chain + k 2^24; k = 0 is the chain itself) starts at sweep counter        */
/* sweep0, runs burn_in sweeps of step 6.2 that are not averaged, then       */
/* repeats steps 6.2-6.3 for M_per_chain sweeps; zhat is the mean of the     */
/* back-transformed angles of all K * M_per_chain realizations.  phi is      */
/* left unchanged.                                                           */
/* ------------------------------------------------------------------------ */
int orc_predict_chains(const double* phi, const uint8_t* mask, const float* z, int W, int H,
                       double T, const orc_params* p, uint32_t chain, uint32_t sweep0,
                       double zmin, double zmax, int K, int burn_in, int M_per_chain,
                       double* zhat)
{
    long n = (long)W * H;
    double* sum = (double*)calloc((size_t)n, sizeof(double));
    double* work = (double*)malloc((size_t)n * sizeof(double));
    for (int k = 0; k < K; ++k) {
        const uint32_t chain_k = chain + (uint32_t)k * (1u << 24);
        uint32_t sweep = sweep0;
        memcpy(work, phi, (size_t)n * sizeof(double));
        for (int j = 0; j < burn_in; ++j)
            orc_sweep(work, mask, W, H, p->a_eq, T, p->q, p->seed, chain_k, sweep++, p->or_mode,
                      NULL, NULL);
        for (int j = 0; j < M_per_chain; ++j) {
            orc_sweep(work, mask, W, H, p->a_eq, T, p->q, p->seed, chain_k, sweep++, p->or_mode,
                      NULL, NULL);
            for (long i = 0; i < n; ++i)
                if (!mask[i]) sum[i] += orc_unmap(work[i], zmin, zmax);
        }
    }
    const double m = (double)K * (double)M_per_chain;
    for (long i = 0; i < n; ++i) zhat[i] = mask[i] ? (double)z[i] : sum[i] / m;
    free(work);
    free(sum);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 5 table (READING R-TAB): e(T_k, L) from unconditional simulations of  */
/* an all-free T_W x T_H lattice, one chain per temperature.                 */
/* ------------------------------------------------------------------------ */
void orc_T_grid(const orc_params* p, double* Tk)
{
    for (int k = 0; k < p->KT; ++k)
        Tk[k] = (p->KT == 1) ? p->T_min
                             : p->T_min * pow(p->T_max / p->T_min, (double)k / (double)(p->KT - 1));
}

int orc_e_table(const orc_params* p, double* Tk, double* ek, int* sweeps_k)
{
    int W = p->T_W, H = p->T_H;
    long n = (long)W * H;
    double ngp = (double)orc_n_gp(W, H);
    uint8_t* free_mask = (uint8_t*)calloc((size_t)n, 1);
    double* phi = (double*)malloc((size_t)n * sizeof(double));
    orc_T_grid(p, Tk);
    for (int k = 0; k < p->KT; ++k) {
        uint32_t chain = 0x80000000u + (uint32_t)k, sweep = 0;
        orc_init_gaps(phi, free_mask, W, H, p->seed, chain);
        orc_equil_out eo;
        orc_equilibrate(phi, free_mask, W, H, Tk[k], p, chain, &sweep, &eo, NULL);
        double acc = 0.0;
        for (int j = 0; j < p->M_T; ++j) {
            orc_sweep(phi, free_mask, W, H, p->a_eq, Tk[k], p->q, p->seed, chain, sweep++,
                      p->or_mode, NULL, NULL);
            acc += orc_energy(phi, W, H, p->q) / ngp;
        }
        ek[k] = acc / (double)p->M_T;
        if (sweeps_k) sweeps_k[k] = eo.sweeps;
    }
    free(phi);
    free(free_mask);
    return 0;
}

/* T-hat = argmin_T |e_s - e(T, L)| (Sect. 2.3) on the piecewise-linear       */
/* interpolant of the table, scanning from the lowest temperature.           */
double orc_invert_T(const double* Tk, const double* ek, int K, double e_s)
{
    if (e_s <= ek[0]) return Tk[0];
    for (int k = 0; k + 1 < K; ++k)
        if (ek[k] <= e_s && e_s < ek[k + 1])
            return Tk[k] + (e_s - ek[k]) * (Tk[k + 1] - Tk[k]) / (ek[k + 1] - ek[k]);
    /* no bracketing interval: the table point closest in energy */
    int best = 0;
    for (int k = 1; k < K; ++k)
        if (fabs(e_s - ek[k]) < fabs(e_s - ek[best])) best = k;
    return Tk[best];
}

typedef struct {
    double zmin, zmax, e_s, T_hat;
    long long n_sp;
    long n_gap;
    orc_equil_out eq;
} orc_fill_out;

/* ------------------------------------------------------------------------ */
/* Algorithm 2 end to end.  T_fixed > 0 skips the temperature inference and */
/* uses the given value.  eq_sweeps >= 0 replaces the slope test by a fixed */
/* number of relaxation sweeps (window control unchanged).  Returns 0, or   */
/* 1 (fewer than two samples / constant data), 2 (no sample pairs).         */
/* ------------------------------------------------------------------------ */
int orc_fill(const float* z, const uint8_t* mask, int W, int H, const orc_params* p,
             double T_fixed, int eq_sweeps, double* zhat, double* phi_out, orc_fill_out* out)
{
    long n = (long)W * H;
    double* phi = (double*)calloc((size_t)n, sizeof(double));
    double zmin, zmax;
    long ns = orc_map(z, mask, W, H, phi, &zmin, &zmax);               /* step 3 */
    if (ns < 2 || !(zmax > zmin)) { free(phi); return 1; }
    long long nsp = 0;
    double e_s = orc_sample_energy(phi, mask, W, H, p->q, &nsp);       /* step 4.1 */
    double T = T_fixed;
    if (!(T_fixed > 0.0)) {
        if (nsp == 0) { free(phi); return 2; }
        double* Tk = (double*)malloc((size_t)p->KT * sizeof(double));
        double* ek = (double*)malloc((size_t)p->KT * sizeof(double));
        orc_e_table(p, Tk, ek, NULL);
        T = orc_invert_T(Tk, ek, p->KT, e_s);                          /* step 4.2 */
        free(Tk);
        free(ek);
    }
    uint32_t chain = 0, sweep = 0;
    orc_init_gaps(phi, mask, W, H, p->seed, chain);                     /* step 2.2 */
    orc_equil_out eo;
    memset(&eo, 0, sizeof eo);
    if (eq_sweeps < 0) {
        orc_equilibrate(phi, mask, W, H, T, p, chain, &sweep, &eo, NULL); /* step 5 */
    } else {
        /* fixed-length relaxation with the step-5 window control */
        long P = count_gaps(mask, n);
        double a = 1.0, A = 0.0;
        for (int i = 0; i < eq_sweeps; ++i) {
            long nacc = orc_sweep(phi, mask, W, H, a, T, p->q, p->seed, chain, sweep++,
                                  p->or_mode, NULL, NULL);
            A = P ? (double)nacc / (double)P : 0.0;
            if (A < p->A_targ) a = 1.0 + (double)(i + 1) / p->k_a;
        }
        eo.sweeps = eq_sweeps; eo.a = a; eo.k = 0.0; eo.A_last = A;
        eo.e_last = orc_energy(phi, W, H, p->q) / (double)orc_n_gp(W, H);
    }
    orc_predict(phi, mask, z, W, H, T, p, chain, &sweep, zmin, zmax, p->M, zhat); /* 6-7 */
    if (phi_out) memcpy(phi_out, phi, (size_t)n * sizeof(double));
    if (out) {
        out->zmin = zmin; out->zmax = zmax; out->e_s = e_s; out->T_hat = T;
        out->n_sp = nsp; out->n_gap = count_gaps(mask, n); out->eq = eo;
    }
    free(phi);
    return 0;
}
