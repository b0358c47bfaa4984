/*
 * ising.h - C ABI of the GB300 (sm_103a) multi-spin-coded checkerboard
 * Metropolis sweep of the 2D Ising model, after Block, Virnau, Preis,
 * "Multi-GPU Accelerated Multi-Spin Monte Carlo Simulations of the 2D Ising
 * Model" (arXiv:1007.3726).
 *
 * Model (Sec. 3, Eq. 1): spins S = +1 / -1 on an L x L square lattice with
 * periodic boundaries, H = -J sum_<ij> S_i S_j - H sum_i S_i with J = 1; the
 * paper's case is H = 0 (a field is optional, see ising_set_field).
 * Dynamics (Sec. 3): Metropolis, checkerboard order: step A updates the sites
 * with (x + y) even, then step B the sites with (x + y) odd; a sweep is A then
 * B.  A move with dE <= 0 is always accepted; dE = 4 or 8 is accepted when the
 * site's 32-bit Philox4x32-10 draw u satisfies u < floor(2^32 exp(-dE/T))
 * (Sec. 3 precomputed factors, Eq. 3 with the strict "<").
 * Storage (Sec. 4 multi-spin coding, Sec. 5.2 "one bit per spin"): rows of
 * 32- or 64-bit words, bit b of word w of row y is site x = w * bits + b,
 * a set bit is S = +1.
 *
 * Random-number contract (replaces the LCG array of Sec. 5.3): in step p of
 * sweep t (t counts the lattice's sweeps since creation), the site (x, y) with
 * (x + y) & 1 == p has index j = y * L/2 + x/2 and takes word (j & 3) of
 * Philox4x32-10 with counter (g mod 2^32, g >> 32, t, stream_id << 1 | p),
 * g = j >> 2, and key (seed mod 2^32, seed >> 32).  The hot start gives the
 * site n = y * L + x the value +1 iff bit (n & 31) of word ((n >> 5) & 3) of
 * Philox4x32-10 with counter (n >> 7 mod 2^32, n >> 39, 0xFFFFFFFF,
 * stream_id << 1) is set.  Results are therefore fixed bit for bit by
 * (L, T, seed, stream_id, initial state, number of sweeps), independent of how
 * the sweeps are split into calls, of the word width and of the launch shape.
 *
 * Observables: M = sum S, E = -sum_(x,y) S(x,y) [S(x+1,y) + S(x,y+1)] (every
 * bond once) as exact int64 after every recorded sweep; FP64 moments, Binder
 * cumulant U4 = 1 - <m^4> / (3 <m^2>^2) (Sec. 3, Eq. 2) and susceptibility.
 *
 * Conventions for every function:
 *   - No exception or abort crosses this ABI; each call returns an
 *     ising_status, and ising_last_error() gives the calling thread's last
 *     message.
 *   - A handle must not be used by two host threads at once; distinct handles
 *     are independent.
 *   - Host pointers are owned by the caller and only read or written during
 *     the call.  Device memory of a handle is owned by the handle.
 *   - Work is queued on the handle's CUDA stream (given at creation; NULL is
 *     the legacy default stream).  Calls that return host data synchronise
 *     that stream.
 *   - A CUDA error makes the handle sticky-failed: every later call on it
 *     returns ISING_ERR_STATE until ising_destroy.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ISING_API __attribute__((visibility("default")))
#else
#define ISING_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ising_lattice ising_lattice; /* opaque; owned by the caller until ising_destroy */

typedef enum {
    ISING_OK = 0,
    ISING_ERR_INVALID = 1, /* bad argument; nothing was changed or allocated */
    ISING_ERR_OOM = 2,     /* device or pinned host allocation failed */
    ISING_ERR_CUDA = 3,    /* a CUDA call failed; the handle is now failed */
    ISING_ERR_TIMEOUT = 4, /* a bounded device wait expired; the handle is now failed */
    ISING_ERR_STATE = 5,   /* the handle failed earlier; only ising_destroy is allowed */
    ISING_ERR_CANCELLED = 6 /* a served request was cancelled before it finished */
} ising_status;

typedef enum {
    ISING_COLD_UP = 0,     /* every spin +1 */
    ISING_COLD_DOWN = 1,   /* every spin -1 */
    ISING_HOT = 2,         /* i.i.d. +-1, p = 1/2, from Philox (see above) */
    ISING_FROM_BUFFER = 3, /* host int8 array of L*L values +1/-1, row-major */
    ISING_FROM_PACKED = 4  /* host array of packed words in the storage layout above */
} ising_init;

typedef struct {
    uint64_t L;             /* linear size; a multiple of 64, 64 <= L <= 2^20 */
    double T;               /* temperature (k_B = J = 1); finite and > 0 */
    uint64_t seed;          /* Philox key */
    uint32_t stream_id;     /* independent chain index under one seed; < 2^31 */
    ising_init init;        /* initial state */
    const void *init_data;  /* host data for FROM_BUFFER (int8) / FROM_PACKED (words); else NULL */
    uint32_t word_bits;     /* 32, 64, or 0 = automatic (64 when L >= 2^16, else 32) */
    uint64_t first_sweep;   /* sweeps already applied to the initial state (resuming a saved
                               lattice: the next sweep uses Philox counter word 2 = first_sweep) */
    double H;               /* external field of Sec. 3, Eq. 1 (finite; 0 = the paper's case).
                               A nonzero field runs the field update of ising_sweep; the
                               recorded E stays the bond energy -sum S_i S_j (the field
                               energy is -H M) */
} ising_params;

typedef struct {
    uint64_t sweeps_done;   /* sweeps applied since creation */
    uint64_t n_samples;     /* samples recorded so far */
    int64_t M, E;           /* magnetisation and energy of the current state */
    double mean_m, mean_abs_m, mean_m2, mean_m4; /* m = M / N over all samples */
    double mean_e, mean_e2;                      /* e = E / N */
    double U4;              /* 1 - <m^4> / (3 <m^2>^2)   (Sec. 3, Eq. 2) */
    double chi;             /* N (<m^2> - <|m|>^2) / T */
    double C;               /* N (<e^2> - <e>^2) / T^2 */
} ising_obs;

/*
 * Creates a lattice on the current CUDA device: validates *params, computes
 * the two thresholds in FP64 on the host (Sec. 3), allocates the packed
 * lattice (L*L/8 bytes) and its per-sweep accumulators, writes the initial
 * state and counts its M and E.  cuda_stream is a cudaStream_t (or NULL).
 * On failure *out is NULL and nothing stays allocated.
 */
ISING_API ising_status ising_create(const ising_params *params, void *cuda_stream, ising_lattice **out);

/*
 * Applies nsweeps sweeps (step A then step B each, Sec. 3; two dependent
 * launches per sweep, the global synchronisation of Sec. 5.2).  A sample
 * (M, E) is recorded after every sweep whose global count sweeps_done becomes
 * a multiple of record_every (0 = record nothing); samples accumulate on the
 * handle for ising_measure.  If M_out and E_out are not NULL they receive the
 * samples of this call in order, at most cap of them (ISING_ERR_INVALID when
 * cap is smaller than the number this call records; nothing runs then), and
 * the call waits for the GPU.  Otherwise the call returns once the work is
 * queued.  ISING_ERR_INVALID if sweeps_done + nsweeps would reach 2^32 - 1.
 */
ISING_API ising_status ising_sweep(ising_lattice *h, uint64_t nsweeps, uint32_t record_every,
                         int64_t *M_out, int64_t *E_out, uint64_t cap);

/* ---- field and temperature changes ---------------------------------------- */

/*
 * In a field H (Sec. 3, Eq. 1) flipping S with c anti-aligned neighbours
 * (neighbour sum n = S (4 - 2c)) changes the energy by dE = 2 S (n + H); the
 * move is taken when dE <= 0, else when the site's draw u < floor(2^32
 * exp(-dE/T)).  Writes the acceptance of the ten classes, index 5 i + c with
 * i = 0 for S = -1 and 1 for S = +1: always[k] = 1 where dE <= 0 (thr[k] = 0
 * there), else thr[k].  H = 0 gives thr8 at c = 0 and thr4 at c = 1.
 * ISING_ERR_INVALID for T not finite and positive or H not finite.
 */
ISING_API ising_status ising_field_thresholds(double T, double H, uint32_t thr[10], uint8_t always[10]);
/*
 * Change the temperature / the field of a lattice from its next sweep on
 * (annealing, field sweeps).  Sweeps already queued keep the old values.  The
 * moments of ising_measure use the current T.  A batch keeps the values the
 * lattices had when it was created.
 */
ISING_API ising_status ising_set_temperature(ising_lattice *h, double T);
ISING_API ising_status ising_set_field(ising_lattice *h, double H);
/* The current T and H of a lattice (either pointer may be NULL). */
ISING_API ising_status ising_get_params(const ising_lattice *h, double *T, double *H);

/*
 * Waits for the handle's stream and fills *out: counters, the current M and E,
 * and FP64 moments of all samples recorded so far, summed in sample order on
 * the host.  With no samples the moments are 0.
 */
ISING_API ising_status ising_measure(ising_lattice *h, ising_obs *out);

/* As ising_measure, but the moments use samples first_sample, first_sample+1,
 * ... only (the equilibration samples before are dropped); n_samples counts
 * the samples used. */
ISING_API ising_status ising_measure_from(ising_lattice *h, uint64_t first_sample, ising_obs *out);

/* Releases everything the handle owns.  NULL is a no-op; always returns ISING_OK
 * unless freeing reported a CUDA error. */
ISING_API ising_status ising_destroy(ising_lattice *h);

/* ---- helpers (tests, checkpointing, serving) ---------------------------- */

/* Copies rows [row0, row0 + nrows) of the current state to out (host, nrows*L
 * int8 values +1/-1, row-major).  Waits for the GPU. */
ISING_API ising_status ising_get_spins(ising_lattice *h, uint64_t row0, uint64_t nrows, int8_t *out);

/* Copies the packed words of the whole lattice to out (host, L * L/8 bytes, the
 * storage layout above with the handle's word width).  Waits for the GPU. */
ISING_API ising_status ising_get_packed(ising_lattice *h, void *out, size_t bytes);

/* Copies recorded samples first .. first + count - 1 (fewer if fewer exist;
 * *n_out tells how many) to the host arrays M and E.  Waits for the GPU. */
ISING_API ising_status ising_get_samples(ising_lattice *h, uint64_t first, uint64_t count, int64_t *M,
                                         int64_t *E, uint64_t *n_out);

/* Full popcount recount of the current state on the GPU (independent of the
 * values fused into the sweep).  Waits for the GPU. */
ISING_API ising_status ising_recount(ising_lattice *h, int64_t *M, int64_t *E);

/* Word width (32 or 64), L, and sweeps done of a handle. */
ISING_API ising_status ising_info(const ising_lattice *h, uint32_t *word_bits, uint64_t *L,
                        uint64_t *sweeps_done);

/* Memory check (a stand-in for a device memory checker): every lattice
 * allocation carries 256 guard bytes of 0xA5 before and after the lattice.
 * Sets *intact to 1 while both guards are unchanged, 0 if any kernel wrote
 * past the lattice.  Waits for the handle's stream. */
ISING_API ising_status ising_check_guards(ising_lattice *h, uint32_t *intact);
/* Device address of the packed lattice and its size in bytes (owned by the handle). */
ISING_API ising_status ising_device_spins(const ising_lattice *h, void **dptr, size_t *bytes);

/* The two Metropolis thresholds floor(2^32 exp(-4/T)) and floor(2^32 exp(-8/T))
 * in FP64 (Sec. 3); ISING_ERR_INVALID for T not finite and positive.  A T whose
 * factor rounds to 1.0 gives 2^32 - 1. */
ISING_API ising_status ising_thresholds(double T, uint32_t *thr4, uint32_t *thr8);

/* Thread-local text of the last failure on this thread ("" if none). */
ISING_API const char *ising_last_error(void);

/* ---- launch configuration and autotuning ------------------------------- */

/*
 * A launch configuration of the half-sweep kernel (Sec. 5.2 leaves block and
 * thread counts to the implementation).  Every valid configuration gives
 * bit-identical lattices and samples; they differ only in speed.
 *   proc_bits      32 or 64: lattice bits one thread updates per row (any
 *                  storage word width can be processed either way)
 *   regcap         0: compiler's register choice, 1: <= 40, 2: <= 32 per thread
 *   block          threads per block: 128, 256 or 512
 *   rows_per_item  rows one thread walks down per work item (divides L, <= 64)
 *   grid           blocks, 0 = as many as can be resident at once
 *   insert         0, 1 or 2: how a compare's result (u < thr4, u < thr8)
 *                  becomes a mask bit: 0 a predicated OR on the integer
 *                  pipes; 1 a predicated FP32 add of 4^k into one exact
 *                  per-8-site counter of both compares; 2 the same into
 *                  separate P4 and P8 counters (FP32 adds issue on the FMA
 *                  pipe that the Philox multiplies leave idle)
 * proc_bits = 8 selects instead the one-CTA form for lattices one thread block
 * holds (L a power of two, 64 <= L <= 1024): the whole lattice stays in shared
 * memory and every sweep of an ising_sweep call runs in one launch, with a
 * block barrier as the synchronisation between steps A and B.  Then block is
 * its size, rows_per_item the threads that share one 32-bit word (1, 2 or 4),
 * grid the CTAs: 1, or a thread-block cluster of 2, 4 or 8 CTAs that split
 * the rows and read their neighbours' boundary rows from distributed shared
 * memory, with a cluster barrier between the steps; regcap = insert = 0.  It is
 * the default for L <= 512 (the warp-specialised cluster form below at L = 64,
 * 128 and 256, a cluster of 8 at 512).  At L = 64, 128 and 256, block 1024 with
 * one thread per word selects the warp-specialised form: consumer threads keep
 * the lattice in registers and update it (one word each at L = 64, a vertical
 * run of two or four words at L = 128 and 256), producer groups draw the
 * acceptance masks of later steps into a ring of tagged entries in the
 * consumers' shared memory, and mbarriers hand the ring slots back.  With grid
 * 1 (L = 64 only) producers and consumers share one CTA; with grid 2, 4 or 8
 * the first CTA of a cluster holds the consumers and the other CTAs the
 * producers, which store through distributed shared memory.  Every wait is
 * bounded: when one runs out the call returns ISING_ERR_TIMEOUT and the handle
 * is failed (the environment variable ISING_TINY_HOLD_STEP = 1 + a step index
 * withholds that step's masks, for failure-detection tests only).  A call of
 * more than 2^30 sweeps runs as several launches of at most 2^30 sweeps each
 * (ISING_TINY_MAX_SWEEPS lowers that bound, for tests only).  In a field (H != 0) it uses one
 * thread per word whatever rows_per_item says, and the warp-specialised
 * configurations run the one-CTA or cluster field kernel with block 512; the
 * step kernels are then replaced by the field step kernel.
 * persistent = 1 (with proc_bits 32 or 64, insert 0, grid 0; regcap 0, 1 or
 * 2 = the compiler's choice, <= 40 or <= 64 registers)
 * runs every sweep of an ising_sweep call in one cooperative launch of that
 * step shape, all blocks resident, with a grid-wide barrier between steps A
 * and B instead of a kernel boundary; for lattices the autotuner's scratch holds
 * whole (L <= 65536).  In a field the field step kernel runs instead.
 * persistent = 0 otherwise.
 */
typedef struct {
    uint32_t proc_bits, regcap, block, rows_per_item, grid, insert;
    uint32_t persistent;
} ising_launch;

/* The handle's current configuration. */
ISING_API ising_status ising_get_launch(const ising_lattice *h, ising_launch *out);
/* Replaces it (ISING_ERR_INVALID if not valid for the handle's L). */
ISING_API ising_status ising_set_launch(ising_lattice *h, const ising_launch *cfg);
/* Writes up to cap candidate configurations for lattices of size L to out and
 * returns how many there are in total (out may be NULL to count). */
ISING_API uint32_t ising_launch_candidates(uint64_t L, ising_launch *out, uint32_t cap);
/*
 * Times every candidate (reps timed step pairs each, after one untimed pair;
 * a one-CTA candidate: one launch of 8 reps sweeps after a one-sweep launch)
 * on a scratch copy of up to 256 MiB of the handle's rows, installs the
 * fastest on the handle, remembers it for later handles of the same L and
 * word width on this device, and returns it with its mean time per step in
 * microseconds.  The lattice itself is not changed.  Waits for the GPU.
 */
ISING_API ising_status ising_autotune(ising_lattice *h, uint32_t reps, ising_launch *best,
                                      double *best_us_per_step);

/*
 * ising_bench_mix - the integer-mix microbenchmark: how fast this GPU generates
 * the sweep's Philox4x32-10 draws alone (the random numbers of Sec. 5.3's role,
 * in the counter-based form of this library), timed with CUDA events on
 * cuda_stream over one launch of one full wave of resident 512-thread blocks,
 * after one untimed warm-up launch.  Each thread makes the eight calls (32
 * draws) of a 64-bit word, words_per_thread times (1 .. 2^20), in form
 *   0  ten full Philox rounds per call (2 widening multiplies and 2
 *      three-input XORs per round);
 *   1  the half-sweep's own form of the calls (rounds 1-2 partly hoisted);
 *   2  form 1 plus the acceptance masks (two compares and bit insertions per
 *      draw), i.e. the word update without its lattice logic and memory.
 * Outputs: *ms the launch's time, *draws_per_ns the draws per nanosecond.
 * Allocates (and frees) one word per thread of device memory; waits for the
 * GPU.  Errors: ISING_ERR_INVALID for a bad form or size, ISING_ERR_CUDA.
 */
ISING_API ising_status ising_bench_mix(uint32_t form, uint32_t words_per_thread, double *ms,
                                       double *draws_per_ns, void *cuda_stream);

/* ---- many lattices in one persistent launch ----------------------------- */

/*
 * A batch runs many lattices of uneven size in one persistent, cooperative
 * kernel launch.  Each lattice is cut into strips of rows held in shared
 * memory for the whole launch; strips of one lattice on different CTAs swap
 * their boundary rows after every checkerboard step through border arrays in
 * global memory (the border exchange of Sec. 6.1, between CTAs of one GPU),
 * and each strip waits only for its two neighbours.  Lattices, samples and
 * final states are bit-identical to ising_sweep on each handle: the batch
 * changes where and when sites are updated, never how.
 *
 * Options (zero = default):
 *   block          threads per CTA, 128, 256 or 512 (512)
 *   ctas_per_sm    resident CTAs per SM the plan is made for (2); each CTA gets
 *                  that share of the SM's shared memory
 *   rows_per_item  rows one thread walks per item (4)
 *   insert         as in ising_launch (0)
 *   use_graph      1: capture one run in a CUDA graph on the first run and
 *                  replay it afterwards
 *   wait_ms        limit of one wait for a neighbour strip (2000 ms); when it
 *                  runs out the launch stops, ising_batch_run returns
 *                  ISING_ERR_TIMEOUT and the handles become failed
 *   hold_strip     failure-detection testing only: 1 + index of a strip that
 *                  never announces its steps, so that its neighbours' waits
 *                  run out (0 = none)
 */
typedef struct ising_batch ising_batch;
typedef struct {
    uint32_t block, ctas_per_sm, rows_per_item, insert, use_graph;
    double wait_ms;
    uint32_t hold_strip;
} ising_batch_opts;

/* Plans a batch of n distinct handles on one device; each run advances handle
 * i by nsweeps[i] sweeps (1 .. 2^30) and records samples every record_every
 * sweeps as ising_sweep does.  ISING_ERR_INVALID if the lattices do not fit in
 * the GPU's shared memory at once.  The batch takes each lattice's temperature
 * and field when it is created (lattices in a field use the ten-class update of
 * ising_field_thresholds).  The handles must outlive the batch. */
ISING_API ising_status ising_batch_create(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                          uint32_t record_every, const ising_batch_opts *opts,
                                          ising_batch **out);
/* Performs `runs` runs one after another (one launch each); waits for the GPU
 * after each and appends the samples to the handles. */
ISING_API ising_status ising_batch_run(ising_batch *b, uint32_t runs);
/* CTAs, threads per CTA, strips and dynamic shared memory of the plan. */
ISING_API ising_status ising_batch_info(const ising_batch *b, uint32_t *grid, uint32_t *block,
                                        uint32_t *strips, size_t *smem_bytes);
ISING_API ising_status ising_batch_destroy(ising_batch *b);
/* Times a few batch configurations (threads per CTA, CTAs per SM, rows per
 * item) on probe runs of about probe_sweeps sweeps (0 = 20) and writes the
 * fastest into *best (its other fields are kept from *best on entry); the
 * lattices are saved before and restored after, the handles' counters and
 * samples are untouched.  best_ms receives the probe run's time. */
ISING_API ising_status ising_batch_tune(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                        uint32_t probe_sweeps, ising_batch_opts *best, double *best_ms);
/* One run of a batch made with default options, then destroyed. */
ISING_API ising_status ising_sweep_batch(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                         uint32_t record_every);

/* ---- request server: continuous batching --------------------------------- */

/*
 * A server accepts simulation requests at any time from any thread.  A worker
 * thread admits them in arrival order while their device memory fits the
 * budget; admitted lattices stay resident.  Each launch is one persistent
 * batch (above) over the resident lattices that fit it, each advancing by up
 * to epoch_sweeps sweeps; the lattices that ran go behind those that waited
 * (round robin), finished requests leave and free their memory, and new ones
 * join at the next launch.  A request's samples and final state are exactly
 * those of ising_sweep on the same parameters alone.
 */
typedef struct ising_server ising_server;
typedef struct {
    uint64_t hbm_budget_bytes;  /* device memory of resident lattices (0 = 64 GiB) */
    uint32_t epoch_sweeps;      /* sweeps per lattice per launch at most (0 = 1000) */
    uint32_t max_active;        /* lattices per launch at most (0 = as shared memory allows) */
    uint32_t keep_samples;      /* 1: keep each request's M/E samples for ising_server_samples */
    ising_batch_opts batch;     /* launch options (block 0 = 256 threads, 4 CTAs per SM) */
} ising_server_opts;
typedef struct {
    ising_params params;        /* FROM_BUFFER / FROM_PACKED data must stay valid until admission */
    uint64_t nsweeps;           /* 1 .. 2^32 - 2 */
    uint32_t record_every;
    uint64_t tag;               /* returned in the result */
} ising_request;
typedef struct {
    uint64_t id, tag;
    ising_status status;        /* ISING_OK; ISING_ERR_OOM if larger than the budget;
                                   ISING_ERR_CANCELLED; or why the launch failed */
    ising_obs obs;              /* final counters and moments of all its samples */
    double t_submit, t_admit, t_first_run, t_finish;  /* seconds since the server started */
    uint64_t epochs;            /* launches it took part in */
} ising_result;
typedef struct {
    uint64_t submitted, admitted, completed, failed, cancelled, queued, resident;
    uint64_t epochs, mem_used, peak_mem, attempts;
    double busy_seconds;        /* time inside launches */
    double now;                 /* seconds since the server started */
} ising_server_counters;

/* Starts a server (and its worker thread) on the current device. */
ISING_API ising_status ising_server_create(const ising_server_opts *opts, ising_server **out);
/* Queues a request (thread-safe, does not block on the GPU); *id identifies it. */
ISING_API ising_status ising_server_submit(ising_server *s, const ising_request *req, uint64_t *id);
/* Cancels a queued or running request; a running one stops at its next launch boundary. */
ISING_API ising_status ising_server_cancel(ising_server *s, uint64_t id);
/* Takes up to cap finished results, waiting up to wait_s seconds for the first. */
ISING_API ising_status ising_server_poll(ising_server *s, ising_result *out, uint32_t cap, uint32_t *n,
                                         double wait_s);
/* With keep_samples: the M/E samples of a polled, finished request (M or E NULL
 * queries *n); taking them releases them. */
ISING_API ising_status ising_server_samples(ising_server *s, uint64_t id, int64_t *M, int64_t *E,
                                            uint64_t cap, uint64_t *n);
ISING_API ising_status ising_server_stats(ising_server *s, ising_server_counters *out);
/* Stops the worker; unfinished requests are dropped. */
ISING_API ising_status ising_server_destroy(ising_server *s);

/* ---- one lattice over several GPUs: row strips ------------------------------ */

/*
 * The row-strip form of the super-lattice decomposition of Sec. 6.1: each rank
 * holds global rows [row0, row0 + nrows) of an L x L lattice in a device
 * buffer d_rows of (nrows + 2) rows in the storage layout above: a halo row
 * (the global row above the strip), the strip, a halo row (the row below).
 * Before every checkerboard step the caller fills the two halos with the
 * neighbouring ranks' boundary rows ("copy neighbor borders to GPU memory",
 * Sec. 6.1); ising_strip_step then updates the strip rows of parity p for
 * sweep t with the same per-site Philox draws as the whole lattice, so the
 * strips together equal ising_sweep bit for bit for any split.  With p == 1
 * and d_counts (2 device counters) not NULL, the step adds the strip's +1
 * spins and the anti-aligned bonds of its parity-1 sites after the step; the
 * sums over all ranks give M = 2 up - L^2 and E = 2 anti - 2 L^2.  Neither
 * call allocates memory; both are queued on cuda_stream.
 */
ISING_API ising_status ising_strip_init(void *d_rows, uint64_t L, uint32_t word_bits, uint64_t row0,
                                        uint64_t nrows, ising_init init, uint64_t seed, uint32_t stream_id,
                                        void *cuda_stream);
ISING_API ising_status ising_strip_step(void *d_rows, uint64_t L, uint32_t word_bits, uint64_t row0,
                                        uint64_t nrows, double T, uint64_t seed, uint32_t stream_id, uint32_t t,
                                        uint32_t p, unsigned long long *d_counts, void *cuda_stream);

/* M and E (Sec. 3, Eq. 1 with J = 1, H = 0) of a whole L x L lattice from the
 * summed step-B counts of its strips: n_up spins +1 and n_anti anti-aligned
 * bonds (of the 2 L^2) give M = 2 n_up - L^2 and E = 2 n_anti - 2 L^2.
 * Any L in [2, 2^20] (the counts may come from strips stepped elsewhere);
 * ISING_ERR_INVALID for null outputs, such an L or counts beyond the lattice. */
ISING_API ising_status ising_strip_observables(uint64_t L, uint64_t n_up, uint64_t n_anti, int64_t *M,
                                               int64_t *E);

/*
 * ising_sweep_noalloc - the sweep for callers that cannot allocate memory.
 * The paper has no counterpart; this entry point exists for callers that own
 * all of their device memory (a serving process whose HBM budget is reserved
 * up front in its own pool, a host application that lends device buffers to
 * plug-ins and forbids them the CUDA allocator, a loop that must not take the
 * device-wide synchronisation a cudaMalloc or cudaFree may bring).  It
 * allocates nothing: no cudaMalloc, cudaFree, pinned host memory or other
 * allocating call.
 *
 * It runs nsweeps sweeps t0 .. t0 + nsweeps - 1 (the same arithmetic and the
 * same results as ising_sweep on a handle whose sweeps_done is t0) on a lattice
 * the caller owns: d_spins is the caller's device array of L * L / 8 bytes in
 * the storage layout above with word_bits-bit words, updated in place.  It
 * must be memory of the current device (cudaMalloc'd or managed) and 16-byte
 * aligned, since the kernels read it in units of up to 128 bits whatever the
 * storage width; anything else fails with ISING_ERR_INVALID before any work.
 * Lattices that ising_sweep runs in one launch (one CTA or one cluster,
 * L <= 512 by default) run the same way here; larger ones take two step
 * launches per sweep.  The
 * samples (M, E) of the sweeps whose count t + 1 is a multiple of
 * record_every (0 = none) go to the caller's host arrays M_out / E_out (cap
 * entries each) and the call then waits for cuda_stream; with no sample the
 * call returns once the work is queued.
 *
 * Scratch: the per-sweep counters live in a fixed device array compiled into
 * the library, ISING_NOALLOC_MAX_RECORDS samples plus two slots (1 MiB) that every GPU which
 * loads the library holds until the process exits.  A call that would record
 * more samples fails with ISING_ERR_INVALID before any work; split it.  All
 * calls share that array and it keeps the previous call's contents (the call
 * clears what it uses), so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and corrupt each other's samples:
 * serialise them.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.
 */
#define ISING_NOALLOC_MAX_RECORDS 65536
ISING_API ising_status ising_sweep_noalloc(void *d_spins, uint64_t L, uint32_t word_bits, double T,
                                           uint64_t seed, uint32_t stream_id, uint64_t t0,
                                           uint64_t nsweeps, uint32_t record_every,
                                           int64_t *M_out, int64_t *E_out, uint64_t cap,
                                           void *cuda_stream);

/*
 * Optional device allocator for every later allocation of the library (for
 * example PyTorch's caching allocator).  alloc(bytes, stream, ctx) returns a
 * device pointer or NULL (reported as ISING_ERR_OOM); release(ptr, stream,
 * ctx) frees it.  Passing NULL functions restores cudaMalloc / cudaFree.  Must
 * not be changed while handles created under another allocator are alive.
 */
typedef void *(*ising_alloc_fn)(size_t bytes, void *cuda_stream, void *ctx);
typedef void (*ising_free_fn)(void *ptr, void *cuda_stream, void *ctx);
ISING_API ising_status ising_set_allocator(ising_alloc_fn alloc, ising_free_fn release, void *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */
