/*
 * mpr.h -- C ABI of the GB300 MPR gap-filling library (libmpr.so).
 *
 * Method: Zukovic, Borovsky, Lach, Hristopulos, "GPU-accelerated Simulation of
 * Massive Spatial Data based on the Modified Planar Rotator Model".  A grid
 * G = G_S u G_P holds sample values Z_s at the sample sites G_S; the library
 * returns estimates Z_p at the prediction (gap) sites G_P (Sect. 2.1) by
 * conditional hybrid Monte Carlo of the MPR model (Eq. 2), following
 * Algorithm 2: data-to-angle map (Eq. 1), temperature inference by specific
 * energy matching (Eqs. 4-5), relaxation with the hybrid update of Algorithm 1
 * until the energy slope test passes, M equilibrium sweeps and the inverse map.
 *
 * Conventions shared by every entry point
 *  - Grids are row-major [H][W] (x fastest).  mask[i] = 1 marks a sample site,
 *    0 a gap site.  z values at gap sites are ignored.
 *  - Pointers may be host or device memory (CUDA unified addressing decides);
 *    inputs are copied at the call, outputs are written before the call returns.
 *    The caller owns every buffer it passes; the context owns all others.
 *  - All device work is enqueued on the stream given to mpr_init (a
 *    cudaStream_t passed as void*, NULL = legacy default stream).  A call that
 *    returns a value to the host synchronises that stream first.
 *  - Errors are returned as mpr_status; nothing is thrown across the ABI.
 *    mpr_last_error(ctx) gives a one-line description of the last failure.
 *  - A context is not thread-safe: use one context per host thread / stream.
 *  - The coupling q of Eq. 2 is the paper's 1/2 by default; any q in (0, 1/2] is
 *    accepted (the paper bounds q by 1/2 and fixes it there), q < 1/2 on the LIST
 *    kernels with the conserving or no reflection.  Angles are kept as unit vectors
 *    (cos q phi, sin q phi), q phi in [0, 2 pi q).
 */
#ifndef MPR_H_
#define MPR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpr_ctx mpr_ctx;

typedef enum {
    MPR_OK = 0,
    MPR_EINVAL = 1,      /* invalid argument (sizes, NULL pointer, parameter out of range) */
    MPR_ENOMEM = 2,      /* a device or pinned-host allocation failed */
    MPR_ECUDA = 3,       /* a CUDA runtime call failed */
    MPR_ENODATA = 4,     /* fewer than two samples, or z_max == z_min: Eq. 1 is undefined */
    MPR_ENOPAIRS = 5,    /* no nearest-neighbour sample pair: Eq. 4 is undefined */
    MPR_ETIMEOUT = 6,    /* a bounded device-side wait expired; the device state is unreliable */
    MPR_ENOTEQUIL = 7,   /* i_max reached with slope k < 0; results are valid but flagged */
    MPR_ESTATE = 8       /* call out of order (e.g. sweeps before a temperature is set) */
} mpr_status;

/* over-relaxation (Eq. 6) variants */
/* Over-relaxation (Eq. 6).  CONSERVING: reflection about the MPR local field, kept only
   inside [0, 2 pi) -- the energy-conserving reading, the default.  LITERAL: the formula as
   printed, phi' = 2 atan2(sum sin phi_j, sum cos phi_j) - phi (mod 2 pi), the q = 1
   reflection; it does not conserve the MPR energy (its energy change is counted in the
   tracked energy) and breaks detailed balance, and is kept for the study of that.  NONE:
   Metropolis steps only. */
enum { MPR_OR_CONSERVING = 0, MPR_OR_LITERAL = 1, MPR_OR_NONE = 2 };
/* transcendental functions of the sweep kernel (Sect. 3.3.2, precision study) */
enum { MPR_TRIG_ACCURATE = 0, MPR_TRIG_FAST = 1 };
/* sweep kernels: AUTO (= TILE), LIST (one launch per half-sweep over gap lists, in place),
   TILE (one fused launch per sweep over shared-memory tiles, two lattice buffers).
   Both are replayed as CUDA graphs and give bitwise identical lattices. */
enum { MPR_EXEC_AUTO = 0, MPR_EXEC_LIST = 1, MPR_EXEC_TILE = 2 };
/* Arithmetic of the lattice and the sweeps (Sect. 4, the single- versus double-precision
   comparison).  F32: unit vectors, field sums, proposal and Metropolis test in FP32 (energy
   sums, control and table in FP64).  F64: the lattice is stored as FP64 unit vectors and
   every step of Algorithm 1, the Eq. 4 sample energy, Eq. 2 and the equilibrium averages
   run in FP64 (sin, cos, exp and atan2 of the CUDA math library in double), on the LIST
   kernels only: exec_mode must be AUTO or LIST and trig_mode ACCURATE (mpr_init returns
   MPR_EINVAL otherwise); as in any LIST context mpr_autotune returns MPR_ESTATE and
   mpr_predict_chains MPR_EINVAL; mpr_warmstart_init returns MPR_EINVAL.  Outputs stay
   float (mpr_get_state64 reads the FP64 angles). */
enum { MPR_PREC_F32 = 0, MPR_PREC_F64 = 1 };

/*
 * Simulation parameters (Algorithm 2, step 1.1) and the readings of what the
 * paper leaves open.  Fill with mpr_default_params() and override.
 */
typedef struct {
    uint64_t seed;     /* Philox4x32-10 key; a sweep's update of site (x, y) of colour
                          k = (x + y) & 1 uses the counter {y ceil(W/4) + floor(x/4), sweep,
                          chain, k}, words 0-1 if floor(x/2) is even, else 2-3 */
    double q;          /* coupling of Eq. 2, in (0, 1/2] (default 1/2); q < 1/2 needs exec_mode
                          AUTO or LIST and or_mode CONSERVING or NONE, else MPR_EINVAL */
    double A_targ;     /* target Metropolis acceptance ratio (default 0.3) */
    double k_a;        /* a(i+1) = 1 + (i+1)/k_a when A < A_targ (default 3) */
    int n_f;           /* slope test every n_f sweeps (default 5) */
    int n_fit;         /* energies in the slope fit (default 20, >= 2) */
    int i_max;         /* cap on relaxation sweeps (default 10000) */
    int M;             /* equilibrium realizations for mpr_predict's default (default 100) */
    int or_mode;       /* MPR_OR_CONSERVING (default), MPR_OR_LITERAL or MPR_OR_NONE */
    int trig_mode;     /* MPR_TRIG_ACCURATE (default) or MPR_TRIG_FAST */
    double a_eq;       /* window factor in the equilibrium phase (paper: 1) */
    int KT;            /* temperatures in the e(T,L) table (default 16, >= 2) */
    double T_min;      /* table range (default 1e-4 .. 1) */
    double T_max;
    int T_cap;         /* table lattice side = min(W, T_cap) x min(H, T_cap); 0 = W x H (default 1024) */
    int M_T;           /* sweeps averaged per table temperature (default 100) */
    int exec_mode;     /* MPR_EXEC_* (default AUTO) */
    uint32_t chain;    /* realization id of this context's chain (default 0) */
    int tile_cfg;      /* compiled tile shape of the TILE kernels, 0 .. 2 (default 0; see mpr_autotune) */
    int precision;     /* MPR_PREC_F32 (default) or MPR_PREC_F64 */
} mpr_params;

typedef struct {
    int sweeps;          /* sweeps performed by the call */
    double acceptance;   /* Metropolis acceptance ratio of the last sweep */
    double e;            /* specific energy H/N_GP after the last sweep (Eq. 5 normalisation) */
} mpr_sweep_stats;

typedef struct {
    int sweeps;          /* relaxation sweeps i at exit (Algorithm 2 step 5) */
    double a;            /* window factor at exit */
    double k;            /* last energy slope */
    double A_last;       /* acceptance ratio of the last sweep */
    double e_last;       /* specific energy after the last sweep */
    int converged;       /* 1 if the loop ended on k >= 0, 0 if on i > i_max */
} mpr_equil_stats;

/* Fills *p with the defaults listed above. */
void mpr_default_params(mpr_params* p);

/* Returns a static string naming a status code. */
const char* mpr_status_string(mpr_status s);

/*
 * Algorithm 2 steps 2-3 and the set-up of the device lattice.
 * z: float[H][W] data, mask: uint8[H][W] (1 = sample).  W, H >= 1, W/2 < 65536,
 * H < 65536.  Maps samples to angles by Eq. 1, draws the gap angles from
 * U(0, 2pi) (step 2.2) and builds the red/black lattice and gap lists.
 * On success *ctx owns all device state; release it with mpr_free.
 * Errors: MPR_EINVAL, MPR_ENODATA, MPR_ENOMEM, MPR_ECUDA (no context is returned).
 */
mpr_status mpr_init(mpr_ctx** ctx, const float* z, const uint8_t* mask, int W, int H,
                    const mpr_params* params, void* cuda_stream);

/*
 * Algorithm 2 step 4: sample specific energy e_s (Eq. 4, each sample pair once),
 * the table e(T_k, L) of Eq. 5 from unconditional simulations of all-free
 * lattices (one chain per temperature, all in one batched run, cached per
 * lattice shape and parameters in the process), and T-hat = argmin |e_s - e(T,L)|
 * by piecewise-linear interpolation in T.  Sets the context temperature.
 * T_hat and e_s may be NULL.  Errors: MPR_ENOPAIRS, MPR_ECUDA, MPR_ETIMEOUT.
 */
mpr_status mpr_estimate_T(mpr_ctx* ctx, double* T_hat, double* e_s);

/* Sets the temperature directly (T > 0), skipping mpr_estimate_T. */
mpr_status mpr_set_T(mpr_ctx* ctx, double T);

/*
 * n >= 0 hybrid sweeps (Algorithm 1 on sub-grid A, then on sub-grid B) at a
 * fixed window factor a >= 1, advancing the sweep counter.  out may be NULL.
 */
mpr_status mpr_sweep(mpr_ctx* ctx, int n, double a, mpr_sweep_stats* out);

/*
 * Algorithm 2 step 5 from the current state: i = 0, k = -1, a = 1; sweep while
 * k < 0 and i <= i_max, with the window update of step 5.2 and the slope test of
 * step 5.4 (least-squares slope of the last n_fit specific energies, every n_f
 * sweeps once i >= n_fit).  Returns MPR_ENOTEQUIL if it stopped on i_max.  The loop runs
 * on the device; the host waits once, at the end.  TILE kernels: the whole loop is one
 * launch of the persistent sweep kernel, in which the block that completes a sweep's tiles
 * runs the grid's control step and the next sweep's tiles start once it has published its
 * window (every wait bounded: MPR_ETIMEOUT if one expires); the launch ends when every grid
 * has stopped.  LIST kernels: a CUDA graph whose conditional node repeats chunks of sweeps
 * while any grid is still relaxing (at most i_max / chunk + 4 chunks); sweeps of a chunk
 * that start after a grid has stopped leave it unchanged.
 */
mpr_status mpr_equilibrate(mpr_ctx* ctx, mpr_equil_stats* out);

/*
 * Algorithm 2 steps 6-7: M >= 1 sweeps at window a_eq, accumulating every gap
 * angle, then zhat = G^-1(mean angle) at gaps and zhat = z at samples.
 * zhat: float[H][W] (host or device).  TILE kernels: the M sweeps are one launch, in which
 * a tile starts its next sweep as soon as it and its eight neighbouring tiles have finished
 * the previous one, so consecutive sweeps overlap.
 */
mpr_status mpr_predict(mpr_ctx* ctx, int M, float* zhat);

/*
 * Independent-chain realizations (the paper's estimator is one chain: M consecutive
 * sweeps, Algorithm 2 step 6).  The grid's current state -- normally the one
 * mpr_equilibrate left -- is forked into K chains (1 <= K <= 128).  Chain k draws from
 * the grid's Philox counters with chain word chain + k * 2^24: k = 0 continues the grid's
 * own chain, and every chain starts at the grid's current sweep counter.  The K chains run
 * burn_in >= 0 sweeps that are not averaged (they decorrelate the forks from their shared
 * start), then M_per_chain >= 1 sweeps, all at window a_eq and together (one launch per
 * sweep for all chains), accumulating every gap angle; zhat = G^-1(mean over all
 * K * M_per_chain angles) at gaps and z at samples.  K = 1 with burn_in = 0 gives exactly
 * mpr_predict(ctx, M_per_chain).  The grid's own state and sweep counter are left
 * unchanged.  Single-grid contexts on the tile path; zhat: float[H][W] (host or device).
 * Needs K lattice copies of device memory.
 */
mpr_status mpr_predict_chains(mpr_ctx* ctx, int K, int burn_in, int M_per_chain, float* zhat);

/*
 * Algorithm 2 end to end: mpr_estimate_T (unless a temperature was set),
 * mpr_equilibrate, mpr_predict(params.M).  stats may be NULL.
 * Returns MPR_OK or MPR_ENOTEQUIL on success.
 */
mpr_status mpr_fill(mpr_ctx* ctx, float* zhat, mpr_equil_stats* stats);

/*
 * Batched form: n >= 1 grids of their own sizes in one context.  Every grid gets its own
 * map (Eq. 1), e_s (Eq. 4), temperature, window factor and slope test (Algorithm 2), and
 * its own Philox chain id (params.chain + g); the sweeps of all grids run in the same
 * kernel launches.  z[g], mask[g]: float/uint8 [H[g]][W[g]] (host or device).
 * mpr_estimate_T, mpr_set_T, mpr_sweep and mpr_equilibrate act on every grid (their
 * returned statistics describe grid 0); in a batch of several grids the e(T, L) table of a
 * grid is built on a lattice whose sides are the grid's, capped at T_cap and rounded down
 * to a power of two, so that grids of similar size share one table.
 */
mpr_status mpr_init_batch(mpr_ctx** ctx, int n, const float* const* z, const uint8_t* const* mask,
                          const int* W, const int* H, const mpr_params* params, void* cuda_stream);

/* Number of grids of the context. */
int mpr_batch_size(const mpr_ctx* ctx);

/* Algorithm 2 steps 6-7 for every grid: M sweeps, zhat[g] = float[H[g]][W[g]]. */
mpr_status mpr_predict_batch(mpr_ctx* ctx, int M, float* const* zhat);

/* mpr_fill for every grid (estimate_T unless set, equilibrate, predict_batch(params.M)).
   Returns MPR_ENOTEQUIL if any grid stopped on i_max. */
mpr_status mpr_fill_batch(mpr_ctx* ctx, float* const* zhat);

/* Per-grid results: temperature, e_s, relaxation sweeps, converged flag, map extremes
   (any pointer may be NULL). */
mpr_status mpr_batch_info(mpr_ctx* ctx, int g, double* T, double* e_s, int* sweeps, int* converged,
                          double* zmin, double* zmax);

/* The same for all n grids of the batch in one read of the control state (one host
   synchronisation instead of one per grid): each non-NULL pointer is an array of n = the
   batch size.  EINVAL if n differs from the batch size. */
mpr_status mpr_batch_info_all(mpr_ctx* ctx, int n, double* T, double* e_s, int* sweeps, int* converged,
                              double* zmin, double* zmax);

/*
 * Autotuner of the TILE kernels: times a few sweeps of every compiled tile shape on the
 * context's own grids (starting from a snapshot of the state, which is restored, so the
 * chains are not advanced), keeps the fastest, and sizes the chunk of sweeps of the LIST
 * kernels' captured graphs to about 60 us of sweeping, at least 4 and at most 64.  Needs a
 * temperature.  Outputs (may be NULL): chosen tile configuration, that chunk size, time of
 * one sweep in ms.
 */
mpr_status mpr_autotune(mpr_ctx* ctx, int* tile_cfg, int* graph_sweeps, double* ms_per_sweep);

/* Releases the context and everything it owns.  NULL is allowed. */
void mpr_free(mpr_ctx* ctx);

/* Text of the last error recorded on ctx (never NULL). */
const char* mpr_last_error(const mpr_ctx* ctx);

/*
 * State access (checkpoint / resume and per-sweep parity checks).
 * phi: float[H][W] angles in [0, 2pi] (sample sites hold their mapped angle);
 * sweep: the global sweep counter used by the Philox streams.
 * mpr_set_state writes only gap sites.
 */
mpr_status mpr_get_state(mpr_ctx* ctx, float* phi, uint32_t* sweep);
mpr_status mpr_set_state(mpr_ctx* ctx, const float* phi, uint32_t sweep);
/* Grid g of a batch context: its current angles phi (float[H_g][W_g], as above). */
mpr_status mpr_get_state_batch(mpr_ctx* ctx, int g, float* phi);
/* As mpr_get_state into double[H][W] (host or device): phi = 2 atan2(sin, cos) of the
   stored unit vector in FP64.  In MPR_PREC_F32 contexts the FP32 vectors are widened
   first.  sweep may be NULL. */
mpr_status mpr_get_state64(mpr_ctx* ctx, double* phi, uint32_t* sweep);

/*
 * Energy bookkeeping: H_exact recomputes Eq. 2 over all bonds; H_tracked is the
 * value carried incrementally by the sweeps (sum of accepted energy changes).
 * zmin/zmax/T/e_s report the context's map and temperature (any may be NULL).
 */
mpr_status mpr_get_info(mpr_ctx* ctx, double* H_exact, double* H_tracked, double* zmin,
                        double* zmax, double* T, double* e_s);

/*
 * Benchmark support: enqueues n sweeps at window a >= 1 (the kernels of the context's
 * exec_mode, launched directly, no graph: one launch of n sweeps on the TILE kernels),
 * times them with CUDA events on the context stream and returns the mean duration of one
 * sweep in milliseconds.  Advances the state and the sweep counter like mpr_sweep.
 */
mpr_status mpr_time_sweeps(mpr_ctx* ctx, int n, double a, double* ms_per_sweep);

/*
 * Diagnostics: number of kernels this library has enqueued in the process so far
 * (direct launches plus the kernels of every replayed CUDA graph).
 */
uint64_t mpr_kernel_launches(void);

/*
 * Benchmark support: timing of the TILE sweep kernel.  mpr_sweep_timing_start() resets
 * the process-wide record and enables it: from then on every launch of the sweep kernel
 * (every phase of mpr_equilibrate, mpr_predict, mpr_sweep, ...) is bracketed by CUDA events
 * on its context's stream, and the library adds up, after the call's own synchronisation,
 * the launches' durations (ms), their number, and the sweeps they performed as
 * sum over grids of (sweeps x sites) and (sweeps x gap sites).  mpr_sweep_timing_read
 * reports the record (any pointer may be NULL) and, if stop != 0, disables it.  The
 * relaxation's sweeps are counted from the grids' sweep counters, which costs one extra
 * read of the control state per phase while enabled.
 */
void mpr_sweep_timing_start(void);
void mpr_sweep_timing_read(int stop, double* ms, uint64_t* launches, double* site_sweeps,
                           double* gap_updates);

/*
 * Test support for the bounded waits of the TILE sweep kernel (process-wide, applies to
 * launches made after the call).  ns: limit of every wait between blocks in nanoseconds
 * (0 = the default, 4 s).  stall != 0: block 0 of every sweep launch first waits for a flag
 * that nothing sets, so that the wait expires after ns: the launch sets its error flag,
 * every block leaves after its copies have landed, and the call returns MPR_ETIMEOUT with
 * the GPU still usable (the context's state is then unreliable: free it).
 */
void mpr_debug_wait_limit(uint64_t ns, int stall);

/*
 * Benchmark support: where the TILE sweep kernel's time goes (process-wide, applies to
 * launches made after the call; not for concurrent use by several host threads).
 * buf: device memory of `words` 64-bit words, cleared by the caller, or NULL to stop.
 * Thread 0 of every block writes %globaltimer (ns) stamps into it: for the work item w of
 * a launch (w = sweep within the launch x tiles + position in the launch's tile order),
 * words 6w .. 6w + 5 are: item taken (before any wait), copy issued, copy landed, both
 * colours updated, write-back issued, and blockIdx.x | SM id << 32; items beyond
 * K = (words - 8192) / 6 are not stamped.  The 8192 words after item K - 1 hold, for the
 * Algorithm 2 control step of sweep counter c, words 2 (c mod 4096) and + 1: the ticket that
 * completed the sweep's tiles, and the control step published.  While a buffer is set,
 * launches with accurate transcendentals run a separately compiled copy of the sweep
 * kernel that writes the stamps (MPR_TRIG_FAST launches stamp nothing); results do not
 * change.  words < 8192 disables the trace.
 */
void mpr_debug_trace(uint64_t* buf, uint64_t words);

/*
 * Memory of released contexts.  Contexts take their device memory from a stream-ordered
 * pool per device owned by the library, which keeps what mpr_free releases so that the
 * next context of a similar size allocates without going back to the driver (no
 * counterpart in the paper; it serves repeated fills).  This call returns the kept,
 * unused memory of the current device's pool to the driver; live contexts are not
 * affected.  Returns MPR_OK (also when no pool exists yet) or MPR_ECUDA.
 */
mpr_status mpr_release_memory(void);

/*
 * Allocation-free sample energy.  The paper has no counterpart to this entry point: it
 * exists for callers that are not allowed to allocate device memory, such as a host
 * application that owns the GPU's memory through its own pool or budget and forbids
 * cudaMalloc/cudaFree inside libraries, or a latency-critical loop where an allocation
 * would stall or synchronise the device.
 *
 * Computes what mpr_init computes before any sweep: e_s of Eq. 4 (each nearest-neighbour
 * sample pair once) over the samples mapped by Eq. 1, and the number of sample pairs.
 * z: float[H][W] and mask: uint8[H][W] (1 = sample) must be device-accessible memory;
 * e_s and n_pairs are host pointers, written before the call returns (the call
 * synchronises the stream).  H may not exceed MPR_STATIC_MAX_ROWS (MPR_EINVAL otherwise).
 *
 * It allocates nothing and calls no allocating routine.  Its scratch is one fixed
 * device array of about 256 KB (16 bytes per row plus a 256-byte header), held until the
 * process exits.  The array is reserved on a GPU when the library's device code is loaded
 * there; under CUDA's lazy module loading (the default) that happens at the library's
 * first use on that device, so a caller that must not see any allocation makes one call
 * (or any other library call) on each device at start-up.  The first call on each device
 * also looks up that array's device address (cudaGetSymbolAddress, with the device
 * current); make that first call before any stream capture.  Every call
 * shares the one array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Each call clears the fields it
 * accumulates into before use, so one call's leftovers never reach the next.
 * Returns MPR_OK, MPR_EINVAL, MPR_ENODATA (fewer than two samples or constant data),
 * MPR_ENOPAIRS (no sample pair; e_s = 0) or MPR_ECUDA.
 */
#define MPR_STATIC_MAX_ROWS 16384
mpr_status mpr_sample_energy_static(const float* z, const uint8_t* mask, int W, int H, double q,
                                    double* e_s, long long* n_pairs, void* cuda_stream);

/*
 * Row strips of one grid (several processes, one GPU each, fill one grid too large for one
 * GPU; no counterpart in the paper, whose single GPU sweeps the whole checkerboard of
 * Sect. 3.3).  The grid's rows are cut into bands, one per process.  A strip's context
 * holds the block of rows [row0, row0 + Hb) of the W x H_global grid: its own rows, plus
 * one row of the strip above (when row0 > 0) and one of the strip below (when
 * row0 + Hb < H_global), which it never updates and which the caller refreshes from their
 * owners after every half-sweep (mpr_strip_row).  row0 must be even (so every strip but
 * the first begins at an odd grid row): the block's colours are then the grid's, and the
 * Philox counters of block site (y, x) are those of grid site (x, row0 + y), so the
 * strips together make exactly the updates of a single context on the whole grid.  Strip
 * contexts run the LIST kernels (exec_mode AUTO or LIST).  Reductions across strips (sums,
 * minimum, maximum) are the caller's (e.g. torch.distributed).  The order of one fill:
 *   mpr_strip_extremes on every strip -> global z_min, z_max (Eq. 1) -> mpr_strip_init;
 *   mpr_strip_pairs -> e_s = -sum / count over all strips (Eq. 4) -> mpr_strip_temperature;
 *   exchange the boundary rows; mpr_strip_energy and mpr_strip_gaps summed ->
 *   mpr_strip_begin(phase 0); per sweep: for colour 0, 1: mpr_strip_half_sweep, exchange;
 *   sum the totals; mpr_strip_control (until *stop);
 *   mpr_strip_begin(phase 1); M sweeps as above with phase 1; mpr_strip_predict.
 * z, mask: float / uint8 [Hb][W] of the block (device memory for mpr_strip_extremes, host
 * or device for mpr_strip_init); the gap sites of the other strips' rows are not read.
 */
/* Minimum, maximum and number of the samples in the strip's own rows: out[3] (host). */
mpr_status mpr_strip_extremes(const float* z, const uint8_t* mask, int W, int Hb, int row0, int H_global,
                              double* out, void* cuda_stream);
/* A strip's context, with the whole grid's Eq. 1 extremes.  EINVAL for an odd row0, a block
   outside the grid or one without an own row, the TILE kernels, or a grid of 2^31 sites or
   more; ENODATA unless zmax > zmin. */
mpr_status mpr_strip_init(mpr_ctx** ctx, const float* z, const uint8_t* mask, int W, int Hb, int row0,
                          int H_global, double zmin, double zmax, const mpr_params* params, void* cuda_stream);
/* Eq. 4 terms of the strip's sample pairs (those whose upper or left site is its own): the
   sum of cos(q (phi_i - phi_j)) and the pair count. */
mpr_status mpr_strip_pairs(mpr_ctx* ctx, double* sum_cos, double* n_pairs);
/* T-hat of the whole grid's e_s, from the e(T, L) table of the whole grid's shape (every
   strip computes the same value); sets the context's temperature. */
mpr_status mpr_strip_temperature(mpr_ctx* ctx, double e_s, double* T_hat);
/* Eq. 2 over the bonds of the strip's colour-0 sites (every bond has one colour-0 end): the
   strips' values add up to the grid's energy.  The neighbouring rows must be current. */
mpr_status mpr_strip_energy(mpr_ctx* ctx, double* H_part);
/* Gap sites of the strip's own rows (-1 for another context). */
long long mpr_strip_gaps(const mpr_ctx* ctx);
/* phase 0: Algorithm 2 steps 2.1-2.4 with the grid's energy H_total and gap count P_total;
   phase 1: the equilibrium angle sums start at zero (step 6). */
mpr_status mpr_strip_begin(mpr_ctx* ctx, int phase, double H_total, double P_total);
/* Algorithm 1 on the strip's gap sites of one colour (phase 0: at the relaxation's window;
   phase 1: at a_eq, adding every angle to the sums).  totals: double[2] of device memory;
   colour 0 sets, colour 1 adds, the strip's accepted energy change and acceptance count. */
mpr_status mpr_strip_half_sweep(mpr_ctx* ctx, int color, int phase, double* totals);
/* One control step (phase 0: Algorithm 2 step 5.2-5.5; phase 1: the energy bookkeeping and
   sweep counter of a fixed-window sweep) from totals summed over every strip (device
   double[2]), with the whole grid's gap and bond counts.  stop (host, may be NULL: no
   synchronisation): the relaxation has ended. */
mpr_status mpr_strip_control(mpr_ctx* ctx, const double* totals, int phase, int* stop);
/* Boundary rows, both colours: which = 0 copies the first own row to buf, 1 the last own
   row; 2 copies buf into the row of the strip above, 3 into the row of the strip below.
   buf (host or device) holds mpr_strip_row_bytes(ctx) bytes; enqueued on the stream. */
size_t mpr_strip_row_bytes(const mpr_ctx* ctx);
mpr_status mpr_strip_row(mpr_ctx* ctx, int which, void* buf);
/* Step 7 for the strip: zhat float[Hb][W] of the block (host or device); its own rows hold
   the estimates (gap sites) and the data (samples). */
mpr_status mpr_strip_predict(mpr_ctx* ctx, int M, float* zhat);

/*
 * Test support: Philox4x32-10 on the device.  ctr: uint32[n][4], out: uint32[n][4]
 * (host or device), key = (seed lo, seed hi).
 */
mpr_status mpr_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, size_t n,
                      void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MPR_H_ */
