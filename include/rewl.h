/*
 * rewl.h -- C ABI of librewl: two-dimensional replica-exchange Wang-Landau
 * (REWL) sampling of the joint density of states g(E,M) of the periodic L x L
 * Ising model on one GPU (sm_103a).
 *
 * The method is that of Valentim et al., "Exploring Replica-Exchange
 * Wang-Landau sampling in higher-dimensional parameter space"
 * (arXiv:1508.02748): Wang-Landau walkers doing single-spin-flip trials with
 * the acceptance of Eq. 1 and the g/H update of Sec. 2, in overlapping
 * windows of (E, M) (Sec. 2, Fig. 1b), exchanging configurations between
 * neighbouring windows with the acceptance of Eq. 2, all advancing to the
 * next modification factor together once every histogram is flat (80%
 * criterion, Sec. 3), and finally joined into one g(E,M) by the
 * marginal/derivative matching of Eqs. 3-4 (Sec. 2, one axis at a time).
 *
 * Conventions shared by every call:
 *   - Every call returns int: REWL_OK (0) or a negative REWL_E_* code; no
 *     exception crosses the ABI.  rewl_last_error() gives a message.
 *   - Bins: e = (E + 2N)/4 in [0, N], m = (M + N)/2 in [0, N], N = L*L.  A
 *     window is the integer rectangle [e0, e1] x [m0, m1].  Window index
 *     win = b * n_win_E + a for the a-th window along E and b-th along M.
 *     Walker index w = win * walkers_per_window + k.
 *   - Device memory: the caller passes one device buffer (the workspace) of
 *     at least rewl_workspace_size() bytes to rewl_create and keeps it alive
 *     until rewl_destroy; the library allocates no device memory of its own
 *     and never frees the workspace.  The handle itself is host memory owned
 *     by the library (freed by rewl_destroy).
 *   - Host pointers (host_*) are plain host memory owned by the caller; the
 *     calls that take them copy synchronously.
 *   - All device work is queued on the stream given to rewl_create (NULL =
 *     the legacy default stream); every call returns after that work is
 *     complete.
 *   - A handle is not thread-safe.
 */
#ifndef REWL_H
#define REWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REWL_OK 0
#define REWL_E_INVALID (-1)     /* bad argument or configuration */
#define REWL_E_CUDA (-2)        /* a CUDA call failed (message has the CUDA error) */
#define REWL_E_TIMEOUT (-3)     /* a bounded device wait gave up */
#define REWL_E_UNREACHABLE (-4) /* a walker could not be driven into its window */
#define REWL_E_OVERFLOW (-5)    /* a histogram entry would pass INT32_MAX */
#define REWL_E_BUDGET (-6)      /* rewl_run_iteration: cycle budget used, not flat yet */
#define REWL_E_JOIN (-7)        /* pieces cannot be joined (no common bins) */
#define REWL_E_CAPACITY (-8)    /* output or workspace buffer too small */

/* ln g arithmetic of the sampling tables.  The exact formats keep, per bin,
 * the value at the start of the current iteration (the base) and the
 * iteration's visit count H; ln g = base + H ln f is formed exactly where it
 * is needed, and the visits enter the base when the iteration ends.  With
 * ln f = 2^-k (enforced: see lnf_init) every ln g is a dyadic rational, so
 * both exact formats follow the sequential chain of Sec. 2 bit for bit. */
#define REWL_FP64 0             /* base as a double per bin */
#define REWL_F32X2 1            /* base as a compensated pair of floats (hi, lo) per bin */
#define REWL_F32 2              /* ln g as one float per bin, rounded at every visit: increments
                                   below half an ulp of ln g are lost (precision-study
                                   demonstration; always runs on the thread sampler) */

/* Where the warp sampler keeps a walker's screen and visit counts during a
 * launch (rewl_config.table_mode); every choice gives the same trajectory. */
#define REWL_TABLES_AUTO 0      /* staged when the window's bins fit in shared memory, else global */
#define REWL_TABLES_GLOBAL 1    /* global memory (L1-cached) */
#define REWL_TABLES_STAGED 2    /* all of the walker's bins in shared memory for the launch (REWL_E_CUDA
                                   at launch when they do not fit) */

/* How the warp sampler holds a walker's lattice during a launch
 * (rewl_config.lattice_mode); every choice gives the same trajectory. */
#define REWL_LATTICE_AUTO 0     /* a register when N <= 64, else shared memory */
#define REWL_LATTICE_REGISTER 1 /* one 64-bit register per lane (N <= 64 only, else REWL_E_INVALID) */
#define REWL_LATTICE_SHARED 2   /* one 32-bit word per row in shared memory (two for L > 32) */

/* Sampling kernels (same trajectory, different mapping onto the GPU). */
#define REWL_SAMPLER_WARP 0     /* 8/16/32 lanes per walker, 3/4/5 trials resolved per step */
#define REWL_SAMPLER_THREAD 1   /* one thread per walker, one trial per step */

/* What rewl_get_lng returns. */
#define REWL_LNG_JOINED 0       /* (N+1) x (N+1) doubles, [e][m], sum g = 2^N */
#define REWL_LNG_MARGINAL_E 1   /* N+1 doubles: ln sum_m g(e, m) of the joined table (Eq. 3) */
/* Flag OR-ed into `what` of rewl_get_lng / rewl_get_lng_jackknife: the
 * rescaling rule of each join step.  The paper rescales the surface at
 * g(E_mat, M) (the sentence before Eq. 4), which admits two readings.  Default: one constant per piece,
 * the difference of the two pieces' E marginals (Eq. 3) at E_mat (M
 * marginals at M_mat when joining rows along M).  With this flag: one
 * constant per M slice of the piece, ln g_i(E_mat, M) - ln g_j(E_mat, M),
 * where both pieces have that bin, else the marginal constant (per E slice
 * at M_mat along M). */
#define REWL_JOIN_PER_SLICE 0x100

typedef struct rewl_s rewl_t;   /* opaque */

/* Run configuration (the paper's statement of the problem, Sec. 2-3). */
typedef struct rewl_config {
    uint32_t struct_size;       /* sizeof(rewl_config) */
    int32_t L;                  /* lattice side, 4 <= L <= 64; N = L*L spins */
    int32_t n_win_E;            /* windows along E (Sec. 2, Fig. 1b) */
    int32_t n_win_M;            /* windows along M (Sec. 2: "splitting both") */
    double overlap_E;           /* overlap fraction of adjacent windows, [0, 1) */
    double overlap_M;
    int32_t walkers_per_window; /* independent walkers per window (Sec. 2), >= 1 */
    int32_t precision;          /* REWL_FP64, REWL_F32X2 or REWL_F32 */
    double lnf_init;            /* ln f of the first iteration: a power of two >= 2^-60
                                   (else REWL_E_INVALID; 1 in the workloads) */
    double lnf_final;           /* run ends after the first flat iteration with ln f <= this */
    double lnf_factor;          /* ln f <- ln f * factor, a power of two below 1; 0.5 is
                                   f -> sqrt(f) (Sec. 2) */
    double flatness;            /* min H >= flatness * mean H (0.8, Sec. 3); six decimals */
    uint64_t exchange_interval; /* trials per walker between exchange sweeps (Sec. 2) */
    int32_t check_every;        /* cycles between flatness checks, >= 1 */
    int32_t walkers_per_block;  /* sampling-kernel tiling (0 = automatic) */
    int32_t sampler;            /* REWL_SAMPLER_WARP (default) or REWL_SAMPLER_THREAD */
    int32_t lanes_per_walker;   /* warp sampler: 8, 16 or 32 lanes per walker (0 = automatic) */
    uint64_t seed;              /* Philox key of every random draw */
    uint64_t drive_budget;      /* steps allowed to drive a walker into its window */
    int32_t table_mode;         /* warp sampler: where a launch reads and writes S and H
                                   (REWL_TABLES_*; the trajectory is the same in each) */
    int32_t lattice_mode;       /* warp sampler: how a launch holds the lattice (REWL_LATTICE_*;
                                   the trajectory is the same in each) */
} rewl_config;

/* Snapshot of a run. */
typedef struct rewl_status {
    int32_t iteration;          /* completed iterations (flat events) */
    int32_t done;               /* 1 once the final iteration is flat */
    double lnf;                 /* ln f of the current iteration */
    uint64_t cycles;            /* sample/exchange cycles run */
    uint64_t trials;            /* trials per walker run so far */
    uint64_t exch_attempts;     /* exchange attempts (both walkers in the overlap) */
    uint64_t exch_accepts;
    int32_t n_flat;             /* walkers found flat at the last check */
    int32_t n_walkers;          /* walkers of non-empty windows */
    int32_t error;              /* device error word (0 = none) */
    int32_t reserved;
} rewl_status;

/* Bytes of device workspace a configuration needs.  Returns REWL_E_INVALID
 * for an invalid configuration. */
int rewl_workspace_size(const rewl_config *cfg, size_t *bytes);

/* Creates a run: window geometry (equal-sized overlapping windows; windows
 * with no possible (E, M) bin are left empty and get no walkers), initial
 * spins, and the drive of every walker into its window.
 *   host_init_spins: NULL to draw i.i.d. +-1 spins from the seed, else
 *     n_walkers * N bytes (0 = down, 1 = up), walker-major, site = i*L + j.
 *   d_workspace: device buffer of >= rewl_workspace_size() bytes, 256-byte
 *     aligned, owned by the caller.
 *   stream: a cudaStream_t (NULL = default stream).
 * Errors: REWL_E_INVALID, REWL_E_CAPACITY (workspace too small),
 * REWL_E_UNREACHABLE (drive budget exhausted), REWL_E_CUDA. */
int rewl_create(const rewl_config *cfg, const uint8_t *host_init_spins, void *d_workspace,
                size_t workspace_bytes, void *stream, rewl_t **out);

/* Runs n_cycles cycles.  One cycle: every walker does exchange_interval
 * trials (Eq. 1 and the Sec. 2 update), one exchange sweep (Eq. 2) of the
 * phase cycle mod 4 (E-even, E-odd, M-even, M-odd pairs of adjacent
 * windows), and every check_every cycles a flatness check over all walkers;
 * when every walker is flat the iteration ends (H reset, ln f * factor) or,
 * if ln f <= lnf_final, the run is done.  Cycles after done do nothing.
 * status may be NULL. */
int rewl_run_cycles(rewl_t *h, uint64_t n_cycles, rewl_status *status);

/* Runs cycles until an iteration ends (or the run is done): REWL_OK; or
 * until max_cycles cycles ran without that: REWL_E_BUDGET. */
int rewl_run_iteration(rewl_t *h, uint64_t max_cycles, rewl_status *status);

/* Parts of one cycle for rewl_enqueue_cycle. */
#define REWL_PART_SAMPLE 1      /* the exchange_interval trials of every walker */
#define REWL_PART_REST 2        /* exchange sweep, flatness check (every check_every cycles), counters */
#define REWL_PART_SAMPLE_PLAIN 4 /* the same trials in the plain form (see rewl_run_cycles_plain);
                                    not together with REWL_PART_SAMPLE */
#define REWL_PLAIN_STREAMS 4    /* streams the plain form spreads its launches over */

/* Queues one cycle, or the given parts of it in order SAMPLE then REST, on
 * the run's stream and returns without waiting: the asynchronous form of
 * rewl_run_cycles(h, 1, NULL) for callers that synchronise or time the
 * stream themselves (a cycle is counted when its REST part is queued).
 * Errors are those of queueing (REWL_E_INVALID, REWL_E_CUDA); device errors
 * surface at the next synchronous call. */
int rewl_enqueue_cycle(rewl_t *h, int parts);

/* The same cycles as rewl_run_cycles, with the same result bit for bit (the
 * chain of every walker does not depend on how it is scheduled), executed in
 * the plain unbatched form the batched sampler is measured against: each
 * walker's exchange_interval trials are a launch of their own (one thread of
 * the one-thread-per-walker kernel, whatever sampler the run was created
 * with), spread round-robin over REWL_PLAIN_STREAMS library-owned streams
 * forked from and joined back into the run's stream; the exchange, flatness
 * check and advance follow as separate launches; no CUDA graph.  The walkers
 * of one exchange interval are independent (Sec. 2), so the order of their
 * launches is free.  status may be NULL.  Errors as rewl_run_cycles. */
int rewl_run_cycles_plain(rewl_t *h, uint64_t n_cycles, rewl_status *status);

/* Single steps (also used inside the cycle): n trials per walker; one
 * exchange sweep of the current phase; one flatness check with advance. */
int rewl_sweep(rewl_t *h, uint64_t n_trials);
int rewl_exchange(rewl_t *h);
int rewl_check(rewl_t *h, int32_t *all_flat);

int rewl_get_status(rewl_t *h, rewl_status *status);

/* Window rectangles: n_windows x 5 int32 (e0, e1, m0, m1, non-empty). */
int rewl_get_windows(rewl_t *h, int32_t *host_out, size_t capacity);

/* Walker state: n_walkers x 4 int64 (e, m, trials, last flat verdict) and
 * optionally spins n_walkers x N bytes (0/1, site = i*L + j). */
int rewl_get_walkers(rewl_t *h, int64_t *host_state, uint8_t *host_spins);

/* Per-walker tables, walker-major, each window_bins = (e1-e0+1)(m1-m0+1)
 * entries in [e][m] order: ln g as double (exact formats: base + max(H, 0)
 * ln f, formed in double) and H as int32 (-1 = never visited).  Either
 * pointer may be NULL.  capacity counts entries per array. */
int rewl_get_tables(rewl_t *h, double *host_lng, int32_t *host_H, size_t capacity);
/* Overwrites the tables (tests set up join and flatness cases with it): the
 * exact formats store base = ln g - max(H, 0) ln f with the current ln f
 * (host_H NULL: the H on the device) and refresh the screens the sampler
 * decides with.  count must equal the number of entries get returns. */
int rewl_set_tables(rewl_t *h, const double *host_lng, const int32_t *host_H, size_t count);

/* Order-independent 64-bit digest of every walker's tables on the device:
 * the bit patterns of each entry's ln g (as rewl_get_tables gives it) and H,
 * mixed with the entry's index and summed modulo 2^64.  Runs whose tables
 * hold the same values have the same digest whatever their format; used to
 * compare table sets too large to copy to the host. */
int rewl_tables_digest(rewl_t *h, uint64_t *digest);

/* Final merge of each window's walkers, join (Eqs. 3-4, E then M) and
 * normalisation to sum g = 2^N, all on the device, copied to host_out.
 * what = REWL_LNG_JOINED or REWL_LNG_MARGINAL_E, optionally OR
 * REWL_JOIN_PER_SLICE (the rescaling rule).  *needed gets the entry
 * count; REWL_E_CAPACITY if capacity is smaller.  host_ematch (n_win_M x
 * (n_win_E - 1) int32) and host_mmatch (n_win_M - 1) receive the matching
 * points (-1 where unused) and may be NULL.  REWL_E_JOIN when two adjacent
 * pieces share no visited bin. */
int rewl_get_lng(rewl_t *h, int what, double *host_out, size_t capacity, size_t *needed,
                 int32_t *host_ematch, int32_t *host_mmatch);

/* Jackknife over the walkers of each window (Sec. 2 proposes it for error
 * bars from a single production run, the walkers being independent): replicate k
 * (k = 0..W-1) is the merge / join / normalisation of rewl_get_lng without
 * walker k of every window; host_mean gets the mean of the W replicates and
 * host_err sqrt((W-1)/W * sum_k (replicate_k - mean)^2), per entry, for
 * what = REWL_LNG_JOINED ((N+1)^2 entries) or REWL_LNG_MARGINAL_E (N+1).
 * Entries missing from any replicate: mean -inf, error NaN.  Needs
 * walkers_per_window >= 2.  Errors as rewl_get_lng. */
int rewl_get_lng_jackknife(rewl_t *h, int what, double *host_mean, double *host_err, size_t capacity,
                           size_t *needed);

/* Checkpoint / resume.  rewl_save writes the whole state of a run
 * (configuration, walkers' spins, bins and trial counters, ln g and H tables,
 * iteration, ln f, exchange and cycle counters) to the host file `path`.
 * rewl_load restores it into a new handle on a caller-provided workspace of
 * at least rewl_workspace_size() bytes for the saved configuration
 * (rewl_checkpoint_config reads that configuration from the file first).
 * Every random draw is a Philox counter of the trial or exchange index, so a
 * restored run continues exactly as the saved one would have.  The file is
 * host-endian and tied to this library version.  Errors: REWL_E_INVALID
 * (I/O, wrong file), REWL_E_CAPACITY, REWL_E_CUDA. */
int rewl_save(rewl_t *h, const char *path);
int rewl_checkpoint_config(const char *path, rewl_config *cfg);
int rewl_load(const char *path, void *d_workspace, size_t workspace_bytes, void *stream, rewl_t **out);

/* Message of the last failing call on h (never NULL). */
const char *rewl_last_error(const rewl_t *h);

/* Releases the handle (not the workspace). */
int rewl_destroy(rewl_t *h);

/* A batch: several runs (any L, geometry or precision) advanced together.
 * rewl_batch_create builds one CUDA graph whose parallel branches hold each
 * run's cycle kernels on a stream of its own, so the runs sample concurrently
 * on the GPU and one graph launch advances all of them by K cycles, K the
 * least common multiple of their check_every (at most 64).  Each run keeps
 * its own workspace and its trajectory is exactly the one it has when run
 * alone.  The runs must each stand at a multiple of their own check_every
 * cycles, must not be used on their own while the batch exists, and stay
 * owned by the caller (rewl_batch_destroy does not destroy them).
 *   runs: host array of n run handles (n >= 1); stream: the stream the
 *   batch's graph is launched on (not NULL).
 * rewl_batch_run_cycles runs n_cycles (a multiple of K) on every run and
 * returns when they are done.  Errors: REWL_E_INVALID, REWL_E_CUDA. */
typedef struct rewl_batch_s rewl_batch_t;
int rewl_batch_create(rewl_t *const *runs, int n, void *stream, rewl_batch_t **out);
int rewl_batch_cycles_per_launch(const rewl_batch_t *b, uint64_t *k);
int rewl_batch_run_cycles(rewl_batch_t *b, uint64_t n_cycles);
/* Queues one graph launch (K cycles of every run) on the batch stream and
 * returns without waiting (for callers that time or overlap the stream). */
int rewl_batch_enqueue(rewl_batch_t *b);
int rewl_batch_destroy(rewl_batch_t *b);

/* Joined ln g(E,M) of tables already on the device, with no memory
 * allocated by the call.  The paper has no counterpart: this serves callers
 * that may not call cudaMalloc -- a process whose device memory is all owned
 * by an external allocator (a framework's caching pool), or one that fixes
 * its memory budget up front -- but own their inputs and output.  The call
 * synchronises on `stream` before it returns.
 *   cfg: the configuration the tables were sampled with (geometry, walkers).
 *   d_lng, d_H: device pointers, n_walkers x window_bins entries each,
 *     walker-major, [e][m] within a walker (the layout rewl_get_tables
 *     returns): ln g as double, H as int32 (-1 = never visited).
 *   d_out: device pointer to (N+1) x (N+1) doubles, [e][m]: the merged,
 *     joined (Eqs. 3-4) and normalised (sum g = 2^N) table, -inf where no
 *     walker visited; the same result as rewl_get_lng(REWL_LNG_JOINED).
 *   stream: cudaStream_t (NULL = default); returns after the work is done.
 * Working memory comes from one fixed 8 MiB __device__ array in the library
 * (held on every GPU that loads it until the process exits); a geometry whose
 * join needs more gets REWL_E_CAPACITY (roughly L <= 16 fits).  The first call
 * on a device looks the array up (cudaGetSymbolAddress) with that device
 * current: make it before any stream capture.  All calls share the array and
 * it keeps the last call's contents; calls that overlap on the GPU race and
 * must be serialised by the caller.  Errors: REWL_E_INVALID, REWL_E_CAPACITY,
 * REWL_E_JOIN, REWL_E_CUDA; rewl_noalloc_last_error() gives the calling
 * thread's last message. */
int rewl_join_noalloc(const rewl_config *cfg, const double *d_lng, const int32_t *d_H, double *d_out,
                      void *stream);
const char *rewl_noalloc_last_error(void);

/* Measured rates of the GPU the library runs on (rewl_measure_peaks): the
 * denominators of the sampling kernels' roofline.  The paper has no
 * counterpart (it ran on CPUs). */
typedef struct rewl_peaks {
    double lop3_ops_per_s;      /* lane operations per second: independent lop3.b32 (integer logic) */
    double iadd_ops_per_s;      /* independent add.u32 */
    double imad_ops_per_s;      /* independent mad.lo.u32 */
    double ffma_ops_per_s;      /* independent fma.rn.f32 */
    double dep_iadd_cycles;     /* SM cycles per add of one chain of dependent adds */
    double smem_bytes_per_s;    /* shared-memory read bandwidth of the whole GPU (16-byte loads) */
    double l2_bytes_per_s;      /* L2 read bandwidth (64 MiB resident, L1 bypassed) */
    int32_t sms;                /* streaming multiprocessors */
    int32_t reserved;
} rewl_peaks;
/* Runs the microbenchmarks on `stream` (cudaStream_t) and fills *out.
 * d_scratch: caller-owned device memory, 256-byte aligned, at least 64 MiB +
 * 4 KiB (the L2 buffer); its contents are overwritten.  Each rate is one
 * CUDA-event-timed launch after an untimed one; the SM clock is whatever the
 * GPU runs at meanwhile (sample it beside the call).  Errors: REWL_E_INVALID
 * (null or short scratch), REWL_E_CUDA. */
int rewl_measure_peaks(void *d_scratch, size_t scratch_bytes, void *stream, rewl_peaks *out);

/* Relative difference of two density-of-states tables (Eq. 5, Sec. 3:
 * the comparison of a serial WL and a REWL result):
 * d_out[i] = |g_a - g_b| / ((g_a + g_b) / 2) computed from d_lng_a[i] =
 * ln g_a and d_lng_b[i] = ln g_b (same normalisation, e.g. two outputs of
 * rewl_get_lng); 2 where exactly one entry is -inf (empty), NaN where both
 * are.  All three are device pointers to n doubles, owned by the caller;
 * d_out may alias neither input.  Runs on `stream` and waits for it.
 * Errors: REWL_E_INVALID (null pointer with n > 0), REWL_E_CUDA. */
int rewl_relative_difference(const double *d_lng_a, const double *d_lng_b, double *d_out, uint64_t n,
                             void *stream);

/* Device Philox4x32-10 (the generator every random draw of the library uses;
 * Salmon et al., SC'11): d_out[4i..4i+3] = Philox(d_ctr[4i..4i+3], key).
 * d_ctr, d_out: device pointers to 4n uint32; key: host pointer to 2 uint32. */
int rewl_philox(const uint32_t *d_ctr, const uint32_t *key, uint32_t *d_out, uint64_t n,
                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* REWL_H */
