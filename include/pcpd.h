/*
 * pcpd.h -- C ABI of libpcpd.so: the bit-sliced Monte Carlo sweep of the 1+1-d pair contact
 * process with diffusion (PCPD) on an NVIDIA GB300 (sm_103a).
 *
 * The method is the one of Schram, "Reaction-diffusion model Monte Carlo simulations on the
 * GPU" (arXiv 1301.6082): reactions AA0/0AA -> AAA at rate (1-p)(1-d)/2 each, AA -> 00 at
 * rate p(1-d), A0 <-> 0A at rate d on a periodic lattice (Sec. 2, Eq. (1)), with the bond
 * decision tree of Alg. 1, evaluated branch-free on multispin words (Sec. 4, Alg. 2), and the
 * density rho(t) recorded at chosen times (Sec. 5.3).  This library fixes a parallel update
 * schedule: at every sub-step a random phase phi tiles the ring with K = floor(L/3)
 * non-overlapping 3-site windows, each making one bond attempt per sample; MCS time t is
 * reached after ceil(t*L/K) sub-steps (1 MCS = L attempts per sample).
 *
 * Samples are bit-sliced: one independent sample per bit, 32 samples per "group".
 * Canonical lattice layout (every host or device buffer that holds a lattice):
 *     uint32_t words[G][L], G = samples/32; bit j of words[g][i] = occupation of sample
 *     32*g + j at site i.
 * Random numbers: Philox4x32-10 keyed by the seed and counted by (sub-step, window, group,
 * tag|block), so results do not depend on how the work is split or batched.
 *
 * Conventions for every function returning int: 0 (PCPD_OK) on success, else one of the
 * PCPD_E* codes, with a message available from pcpd_last_error() (thread-local).  No
 * function keeps a pointer it was passed beyond the call unless stated.  Handles are not
 * thread-safe; distinct handles may be used from distinct threads.  Nothing in this library
 * falls back to the CPU: without a usable CUDA device every entry that computes fails with
 * PCPD_ENODEV.
 */
#ifndef PCPD_H
#define PCPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PCPD_OK = 0,
    PCPD_EINVAL = 1,   /* bad argument (range, order, NULL, size) */
    PCPD_ENOMEM = 2,   /* a device or host allocation failed */
    PCPD_ECUDA = 3,    /* a CUDA call failed; the message names it */
    PCPD_ETIMEOUT = 4, /* a device-side wait ran out of its iteration budget */
    PCPD_ESTATE = 5,   /* call out of order (e.g. record time already passed) */
    PCPD_ENODEV = 6    /* no usable sm_100-family CUDA device */
};

enum { PCPD_INIT_FULL = 0, PCPD_INIT_EMPTY = 1, PCPD_INIT_HALF = 2 };

typedef struct pcpd pcpd_t;

/* Creation parameters.  Zero-initialise and set what you need. */
typedef struct pcpd_params {
    uint32_t L;          /* lattice sites, 3 <= L < 2^30 */
    uint32_t samples;    /* independent samples, a positive multiple of 32, <= 2^22 */
    double p;            /* annihilation parameter of Eq. (1), in [0, 1] */
    double d;            /* diffusion parameter of Eq. (1), in [0, 1] */
    uint64_t seed;       /* Philox key */
    int init;            /* PCPD_INIT_FULL (default 0), PCPD_INIT_EMPTY or PCPD_INIT_HALF */
    void *stream;        /* cudaStream_t for all device work; NULL = a stream owned by the handle */
    void *dev_lattice;   /* optional caller-owned device buffer of >= 2*G*L*4 bytes, 256-byte
                            aligned, used for the lattice and its second buffer; NULL = the
                            handle allocates (and frees) its own */
    size_t dev_bytes;    /* size of dev_lattice in bytes (ignored when dev_lattice is NULL) */
    int per_sample;      /* non-zero: also keep per-sample counts at every record */
    /* plan override, 0 = automatic.  No plan changes a result bit.  Automatic: columns that
       fit one CTA's shared memory are whole-column tiles; longer columns are cut into tiles
       sized for two 256-thread CTAs per SM with tau = 64 (batch and server members: every
       tile, whole-column or not, sized for two CTAs of at most 256 threads per SM, so that a
       launch of any mix of members runs two CTAs per SM). */
    uint32_t plan_threads;   /* threads per CTA (multiple of 32 in [64, 512]) */
    uint32_t plan_seg_sites; /* core sites per tile for lattices that do not fit one CTA (at
                                most; every tile, the last included, must be at least a halo
                                long: a short last tile evens the tiles out, a length below
                                the halo is refused) */
    uint32_t plan_tau;       /* sub-steps per tile residency (temporal block) */
    int autotune;            /* non-zero and no plan_* override: use the plan pcpd_autotune
                                picks for this (L, samples), tuning on first use */
    int jit;                 /* specialise the sweep for this instance's two thresholds by
                                compiling it at run time (same bits, ~15% faster): 1 = yes,
                                -1 = no, 0 = automatically for lattices of >= 2^22 words */
    uint32_t tuple;          /* reacting tuple size n: 0 or 2 = PCPD (pairs, 3-site windows),
                                3 = TCPD (triplets), 4 = QCPD (quadruplets); windows of n+1
                                sites, K = floor(L/(n+1)) per sub-step, annihilation empties
                                the n-tuple (see pcpd_substep_of_time_n) */
    uint32_t group0;         /* first 32-sample group of this instance inside a larger
                                ensemble of the same seed and rates: the instance holds
                                groups group0 .. group0 + samples/32 - 1 and draws exactly
                                the random numbers those groups draw in a run of the whole
                                ensemble, so instances that split one ensemble's groups
                                between them (e.g. one per GPU; the paper runs one system
                                per workgroup, Sec. 3) together reproduce that run bit for
                                bit.  A multiple of 4 (whole 128-sample phase groups), with
                                group0 + samples/32 <= 2^26; 0 = a standalone instance. */
} pcpd_params;

/* Create a simulation of `samples` PCPD samples on a ring of L sites, initialised fully
 * occupied, using the handle's own stream and memory.  Returns NULL on error (see
 * pcpd_last_error()).  Initial state: Sec. 2's decay runs start fully occupied. */
pcpd_t *pcpd_create(uint32_t L, uint32_t samples, double p, double d, uint64_t seed);

/* Create from parameters.  On success *out receives the handle.  The lattice is initialised
 * (full, empty, or i.i.d. Bernoulli(1/2) bits from the seed) on the handle's stream. */
int pcpd_create_ex(const pcpd_params *prm, pcpd_t **out);

/* Advance every sample by steps_mcs Monte Carlo steps (t_now -> t_now + steps_mcs) and
 * record the occupation at each MCS time in record_times_mcs[0..n_times).  Time unit: Alg. 1
 * (Sec. 2) advances time by 1/L per attempted update, so one MCS is L attempts per sample;
 * with K windows per sub-step, MCS time t is reached after ceil(t*L/K) sub-steps.  Times
 * strictly increasing, each in (t_now, t_now + steps_mcs]; a time equal to t_now is allowed only as
 * the first entry and records the current state.  Work is enqueued on the handle's stream;
 * the call returns without waiting for it.  n_times may be 0 (record_times_mcs may then be
 * NULL).  Errors: PCPD_EINVAL (times out of order or range, sub-step count >= 2^32),
 * PCPD_ECUDA. */
int pcpd_run(pcpd_t *h, uint64_t steps_mcs, const uint64_t *record_times_mcs, size_t n_times);

/* Number of records taken so far (all pcpd_run calls). */
size_t pcpd_num_records(const pcpd_t *h);

/* Copy the first n_times records (waits for the handle's stream): the particle density
 * rho(t) whose decay the paper analyses (Sec. 5.3), rho_out[r] = counts[r] / (L * samples)
 * (nullable), counts_out[r] = occupied (site, sample) pairs (nullable); pcpd_record_times:
 * times_out[r] = the record's MCS time.  PCPD_EINVAL if n_times exceeds
 * pcpd_num_records(). */
int pcpd_density(const pcpd_t *h, double *rho_out, uint64_t *counts_out, size_t n_times);
int pcpd_record_times(const pcpd_t *h, uint64_t *times_out, size_t n_times);

/* Occupied nearest-neighbour pairs (i, i+1 mod L), summed over samples, of the first n_times
 * records: the pair density rho_pair = pairs / (L * samples), which the paper analyses beside
 * the particle density (Sec. 5.3).  Waits. */
int pcpd_pair_counts(const pcpd_t *h, uint64_t *counts_out, size_t n_times);

/* The pair density itself (Sec. 5.3): rho_pair_out[r] = pair counts[r] / (L * samples) for the
 * first n_times records.  Waits.  PCPD_EINVAL if n_times exceeds pcpd_num_records(). */
int pcpd_pair_density(const pcpd_t *h, double *rho_pair_out, size_t n_times);

/* Per-sample counts of record r into out[samples] (uint32, sample order 0..samples-1).
 * Needs per_sample at creation; else PCPD_ESTATE. */
int pcpd_sample_counts(const pcpd_t *h, size_t r, uint32_t *out);

/* Checkpoint and resume.  The paper is silent on both; resuming is exact here because every
 * random word is addressed by (seed, sub-step, window, group, block), so the state of a run is
 * just its lattice and its sub-step counter.
 * Copy the current lattice to host memory in the canonical layout (G*L words).  Waits. */
int pcpd_get_lattice(const pcpd_t *h, uint32_t *host_out);

/* Replace the lattice by host_in (canonical layout) and set the clock to `substep` completed
 * sub-steps (MCS time = the largest t with ceil(t*L/K) <= substep).  Records are cleared.
 * Resuming from a saved (lattice, sub-step) pair reproduces the uninterrupted run exactly. */
int pcpd_set_lattice(pcpd_t *h, const uint32_t *host_in, uint64_t substep);

/* The same two copies enqueued on the handle's stream without waiting: the host buffer must
 * stay valid (and unchanged, for set) until the stream has passed the copy (pcpd_sync, or any
 * call that waits).  With page-locked host memory the copies overlap other work on the GPU.
 * pcpd_get_lattice_async reports an engine time-out only at the next waiting call. */
int pcpd_get_lattice_async(const pcpd_t *h, uint32_t *host_out);
int pcpd_set_lattice_async(pcpd_t *h, const uint32_t *host_in, uint64_t substep);

/* Advance by exactly n_substeps sub-steps with no records (splice tests, fine control). */
int pcpd_run_substeps(pcpd_t *h, uint64_t n_substeps);

/* Current clock: completed sub-steps and MCS time. */
uint64_t pcpd_substep(const pcpd_t *h);
uint64_t pcpd_time_mcs(const pcpd_t *h);

/* The tile plan a handle runs with (see pcpd_params.plan_*). */
typedef struct pcpd_plan_info {
    uint32_t ring;       /* 1: tiles are whole columns (shared-memory resident for the run) */
    uint32_t gpi;        /* columns per tile (RING) */
    uint32_t threads;    /* threads per CTA */
    uint32_t core;       /* core sites per tile */
    uint32_t halo;       /* halo sites per side (SEGMENT; (W-1)*tau + W + 1, W = tuple + 1) */
    uint32_t tau;        /* sub-steps per tile residency */
    uint32_t n_seg;      /* tiles per column */
    uint32_t tiles;      /* tiles per epoch */
    uint32_t grid;       /* persistent CTAs */
    uint32_t jit;        /* 1: runs a sweep compiled for this instance's thresholds */
    size_t smem_bytes;   /* dynamic shared memory per CTA */
} pcpd_plan_info;

int pcpd_get_plan(const pcpd_t *h, pcpd_plan_info *out);

/* Block until all work enqueued for the handle has finished. */
int pcpd_sync(pcpd_t *h);

/* Release everything the handle owns.  NULL-safe. */
void pcpd_destroy(pcpd_t *h);

/* Message for the last error on this thread ("" if none). */
const char *pcpd_last_error(void);

/* Debug builds (libpcpd_debug.so, compiled with -DPCPD_DEBUG) check every shared- and
 * global-memory index the kernels form; a failed check skips the access and records a code
 * (1 window site, 2 tile load into shared memory, 3 tile load from the lattice, 4 tile store,
 * 5 paper-scheme word, 6 record read past a tile).  pcpd_debug_check() waits for the device,
 * returns the first recorded code (0: none; always 0 in release builds; ~0 if the device could
 * not be read) and clears it.  pcpd_debug_build() is 1 in debug builds.  Debug builds never
 * compile the runtime-specialised sweep. */
int pcpd_debug_build(void);
unsigned int pcpd_debug_check(void);

/* Number of CUDA kernels this library has launched in this process so far (all handles,
 * all threads).  Lets a caller count the device work of a region. */
unsigned long long pcpd_kernel_launches(void);

/* Integer thresholds of the rates of Eq. (1): T_D = min(2^32, floor(d*2^32)),
 * T_DA = min(2^32, T_D + floor(p*(1-d)*2^32)), IEEE double, no contraction.  A sample with
 * draw u diffuses if u < T_D, else annihilates an occupied bond if u < T_DA, else fissions. */
int pcpd_thresholds(double p, double d, uint64_t *t_d, uint64_t *t_da);

/* Sub-step at which MCS time t is reached on a ring of L sites: ceil(t*L/floor(L/3)). */
uint64_t pcpd_substep_of_time(uint32_t L, uint64_t t);

/* The same for the n-tuple processes (tuple as in pcpd_params): ceil(t*L/floor(L/(n+1)));
 * 0 for an invalid tuple or L shorter than one window. */
uint64_t pcpd_substep_of_time_n(uint32_t L, uint32_t tuple, uint64_t t);

/* ---- device-level entry points used by the tests (all pointers are device pointers,
 * stream may be NULL for the default stream; the call waits for completion) ---- */

/* Philox4x32-10 (Salmon et al., SC'11) on n counters ctr[n][4] under key = seed -> out[n][4]. */
int pcpd_dev_philox(const uint32_t *ctr, uint64_t seed, uint32_t *out, size_t n, void *stream);

/* The bit-plane threshold compare (the exact form of the dyadic masks of Sec. 4.2-4.3): for
 * each of n items, words[n][33] = (O, P31, ..., P0); lane j's draw is
 * u_j = sum_m bit_j(P_m) 2^m.  Writes masks[n][3] = (D: u < T_D, A: T_D <= u < T_DA, O),
 * using the early-exit MSB-first compare of the sweep kernels. */
int pcpd_dev_rate_masks(const uint32_t *words, uint64_t t_d, uint64_t t_da, uint32_t *masks,
                        size_t n, void *stream);

/* Autotuner: time candidate tile plans (threads per CTA -- i.e. windows per thread --, the
 * temporal block tau, the tile size and so the shared-memory residency) on trial_substeps
 * sub-steps of the instance prm describes, and return in *best (a copy of *prm with the
 * plan_* fields set) the fastest, with its rate in attempted updates/s (nullable).  Every
 * plan gives bit-identical results, so the choice only affects speed.  The winner is cached
 * per (L, samples) in the process and, if the environment variable PCPD_TUNE_CACHE names a
 * file, appended to it and read back by later processes.  Allocates and frees trial handles. */
int pcpd_autotune(const pcpd_params *prm, uint32_t trial_substeps, pcpd_params *best,
                  double *best_rate);

/* Failure-path test: runs the sweep engine on a one-item work list whose predecessor is
 * never scheduled, with a dependency-wait budget of spin_limit_cycles GPU clock cycles
 * (1 .. 2^34).  The bounded wait must give up, record the timeout in the engine's error word
 * and end the CTA; the call then returns PCPD_ETIMEOUT and the CUDA context stays usable.
 * Any other return code means the failure path did not behave as designed. */
int pcpd_dev_timeout_test(unsigned long long spin_limit_cycles);

/* ---- batched heterogeneous instances in one persistent launch ----
 * Independent systems run side by side, each with its own seed (the paper runs one system
 * per workgroup, Sec. 3); here any number of instances with different L, samples, p, d,
 * seeds, step counts and record times share one launch of the sweep engine through a
 * device work queue.  Results are bit-identical to running each instance alone. */
typedef struct pcpd_batch pcpd_batch_t;

/* Create an empty batch whose work runs on `stream` (cudaStream_t; NULL = its own). */
int pcpd_batch_create(void *stream, pcpd_batch_t **out);

/* Add an instance (pcpd_params as for pcpd_create_ex; its stream and dev_lattice fields are
 * ignored) to run for steps_mcs MCS from its initial state, with records at
 * record_times_mcs[0..n_times) (strictly increasing, in (0, steps_mcs]; copied).  Device
 * memory for the instance is allocated here.  *index_out (nullable) receives its index. */
int pcpd_batch_add(pcpd_batch_t *b, const pcpd_params *prm, uint64_t steps_mcs,
                   const uint64_t *record_times_mcs, size_t n_times, size_t *index_out);

/* Run every instance to its end: one persistent launch per 128 instances (the launches run
 * one after another; one batch may run at a time per process).  Waits for completion.
 * Errors: PCPD_EINVAL, PCPD_ESTATE (ran already), PCPD_ECUDA, PCPD_ETIMEOUT. */
int pcpd_batch_run(pcpd_batch_t *b);

/* Number of instances added. */
size_t pcpd_batch_size(const pcpd_batch_t *b);

/* Runtime-specialised kernels for members that share a threshold pair (T_D, T_DA) and window
 * width, e.g. the seeds of one p in a near-critical sweep: such members run in launches of
 * their own with the engine compiled for their pair (as a lone instance's long run is), the
 * rest on the generic kernel.  mode > 0: for every pair two or more members share; 0 (the
 * default): when those members' work reaches 2e13 attempted updates (the compile, about 1.5 s
 * once per process and pair, then pays); < 0: never.  Changes no result bit.  Call before
 * pcpd_batch_run; pcpd_batch_jit_launches reports how many launches of the last run used a
 * runtime-compiled kernel (0 where no runtime compiler is available). */
int pcpd_batch_set_jit(pcpd_batch_t *b, int mode);
size_t pcpd_batch_jit_launches(const pcpd_batch_t *b);

/* Record counts of instance i (occupied (site, sample) pairs, n <= its n_times). */
int pcpd_batch_counts(const pcpd_batch_t *b, size_t i, uint64_t *counts_out, size_t n);

/* Pair counts (see pcpd_pair_counts) of instance i. */
int pcpd_batch_pair_counts(const pcpd_batch_t *b, size_t i, uint64_t *counts_out, size_t n);

/* Final lattice of instance i, canonical layout (G*L words).  Waits. */
int pcpd_batch_lattice(const pcpd_batch_t *b, size_t i, uint32_t *host_out);

/* Release the batch and all its instances.  NULL-safe. */
void pcpd_batch_destroy(pcpd_batch_t *b);

/* ---- serving: continuous batching of simulation requests ----
 * A host thread of the library owns the GPU work.  Requests wait in FIFO order until a slot
 * (at most max_active on the GPU) and the device-memory budget allow their admission; each
 * round then advances every active request by at most chunk_attempts attempted updates in
 * one engine launch, so the requests' work overlaps on the device, while each request's
 * lattice and clock (its random-number counter) stay on the device between rounds.  A
 * finished request frees its slot and memory for the queue.  Results are bit-identical to
 * the same request run alone. */
typedef struct pcpd_server pcpd_server_t;

typedef struct pcpd_server_config {
    size_t hbm_budget_bytes;   /* device memory for admitted requests (lattices, records) */
    uint32_t max_active;       /* requests on the GPU at once, 1..128 */
    uint64_t chunk_attempts;   /* attempted updates per request per round (> 0) */
    void *stream;              /* cudaStream_t for the server's work; NULL = its own */
} pcpd_server_config;

typedef struct pcpd_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t rounds;           /* engine rounds run */
    double busy_seconds;       /* wall time inside rounds */
    unsigned long long attempts;  /* attempted site updates done */
    uint64_t active, queued;   /* now */
    size_t mem_used_bytes;     /* now */
} pcpd_server_stats;

/* Start a server (its thread begins waiting for requests). */
int pcpd_server_start(const pcpd_server_config *cfg, pcpd_server_t **out);

/* Queue a request (pcpd_params as for pcpd_create_ex; stream/dev_lattice ignored) for
 * steps_mcs MCS with records at record_times_mcs[0..n_times) (strictly increasing, in
 * (0, steps_mcs]; copied).  keep_lattice != 0 keeps the final lattice for pcpd_server_result.
 * Thread-safe.  *id_out receives the request id. */
int pcpd_server_submit(pcpd_server_t *sv, const pcpd_params *prm, uint64_t steps_mcs,
                       const uint64_t *record_times_mcs, size_t n_times, int keep_lattice,
                       uint64_t *id_out);

/* Cancel a request.  A queued request fails at once ("cancelled"); one on the GPU fails at the
 * end of the current round, when none of its work is in flight, and its memory goes back to
 * the budget.  PCPD_ESTATE if it has already finished, PCPD_EINVAL for an unknown id. */
int pcpd_server_cancel(pcpd_server_t *sv, uint64_t id);

/* State of a request: 0 queued, 1 on the GPU, 2 done, 3 failed. */
int pcpd_server_poll(pcpd_server_t *sv, uint64_t id, int *state_out);

/* Wait for request id and copy its first n record counts (nullable), its final lattice
 * (canonical layout, nullable; needs keep_lattice), its latency from submission to result
 * (nullable) and the part of it spent queued before admission (nullable). */
int pcpd_server_result(pcpd_server_t *sv, uint64_t id, uint64_t *counts_out, size_t n,
                       uint32_t *lattice_out, double *latency_s, double *queue_s);

/* Wait until every submitted request has finished or failed. */
int pcpd_server_wait_idle(pcpd_server_t *sv);

int pcpd_server_get_stats(pcpd_server_t *sv, pcpd_server_stats *out);

/* Stop the thread; requests not finished fail with "server stopped".  NULL-safe. */
void pcpd_server_stop(pcpd_server_t *sv);

/* ---- the paper's own GPU scheme (Sec. 3-4, Alg. 2), as a variant ----
 * Kept beside the window schedule above so that both can be run and compared.  Each of
 * `systems` independent systems is a ring of L = 32 * n_loc * S_w sites worked on by a group
 * of S_w threads (the paper's workgroup of S_w workitems); the 32 bits of a word are 32
 * segments of the same ring, L/32 sites apart ("connected lattices", Sec. 4).
 * Layout of a system's lattice (host and device): uint32_t words[n_loc][S_w]; bit b of
 * words[l][w] is site b*(L/32) + w*n_loc + l.  Systems follow one another.
 * One step: a local site l* drawn for the whole system, then in every (w, b) the bond
 * (s, s+1), s = b*(L/32) + w*n_loc + l*, is updated as in Alg. 2: the pair swaps with
 * probability d; otherwise an occupied pair annihilates with probability p, else puts a
 * particle on s+2 or s-1 with probability 1/2 each (all mod L).  One step = 32*S_w attempts
 * per system; one MCS = n_loc steps.  The diffusion draw of a bit is an m-bit value compared
 * with T_d = d*2^m (d must be a multiple of 2^-m, Sec. 4.2); the annihilation draw ANDs
 * n_dec decorrelation words with one comparison against T_c = floor(p*2^n_dec*2^32) that is
 * shared by all 32 bits of a word (the correlated draw with decorrelation of Sec. 4.3;
 * p*2^n_dec <= 1).  Random words (Philox4x32-10 keyed by the seed): each workitem w of
 * system s has its own stream, word k being word k mod 4 of the block counted by
 * (w, B mod 2^32, s, 4<<28 | B>>32), B = floor(k/4); step t takes the n_w = m + n_dec + 2
 * words n_w*t .. n_w*t + n_w - 1 (diffusion planes, decorrelation words, the broadcast word,
 * the fission word).  l* of step t: floor(x * n_loc / 2^32), x = word t mod 4 of the block
 * (0, floor(t/4), s, 5<<28). */
typedef struct pcpd_paper pcpd_paper_t;

typedef struct pcpd_paper_params {
    uint32_t n_loc;      /* local words per thread, >= 4 */
    uint32_t S_w;        /* threads per system, a multiple of 32 in [32, 1024] */
    uint32_t systems;    /* independent systems, 1 .. 2^24 */
    double p;            /* annihilation probability, 0 <= p*2^n_dec <= 1 */
    double d;            /* diffusion probability, a multiple of 2^-m in [0, 1] */
    uint32_t m;          /* diffusion planes, 0 .. 16 */
    uint32_t n_dec;      /* decorrelation words, 0 .. 16 */
    uint64_t seed;       /* Philox key */
    int init;            /* PCPD_INIT_FULL (0) or PCPD_INIT_EMPTY */
    void *stream;        /* cudaStream_t; NULL = a stream owned by the handle */
    uint32_t plan_spc;   /* systems per CTA (0 = automatic; changes no result bit) */
    int generic;         /* non-zero: run the kernel that reads m and n_dec at run time
                            (same bits; for tests) */
} pcpd_paper_params;

/* T_d = d*2^m and T_c = min(2^32, floor(p*2^n_dec*2^32)) (IEEE double); PCPD_EINVAL if d is
 * not a multiple of 2^-m, p*2^n_dec is outside [0, 1], or m or n_dec exceeds 16. */
int pcpd_paper_thresholds(double p, double d, uint32_t m, uint32_t n_dec, uint32_t *t_d,
                          uint64_t *t_c);

/* Create: every system's lattice resides in one CTA's shared memory during a launch, so
 * n_loc*S_w*4 bytes must fit (about 227 KB: L up to ~1.8e6 sites).  Device lattice
 * systems*n_loc*S_w words, filled (FULL) or empty. */
int pcpd_paper_create(const pcpd_paper_params *prm, pcpd_paper_t **out);

/* Advance every system by n_steps steps and record the occupied sites (summed over systems,
 * and per system) at each absolute step in record_steps[0..n_rec): strictly increasing, in
 * (now, now + n_steps]; the current step is allowed as the first entry.  The final step
 * count must stay below 2^32.  Enqueued on the handle's stream (copies record_steps first). */
int pcpd_paper_run(pcpd_paper_t *h, uint64_t n_steps, const uint64_t *record_steps, size_t n_rec);

size_t pcpd_paper_num_records(const pcpd_paper_t *h);
uint64_t pcpd_paper_step(const pcpd_paper_t *h);

/* First n records: counts_out[n] (sum over systems, nullable) and per_system_out[n][systems]
 * (nullable).  Waits. */
int pcpd_paper_counts(const pcpd_paper_t *h, uint64_t *counts_out, uint32_t *per_system_out, size_t n);

/* Copy the lattice (systems*n_loc*S_w words, layout above) out / in.  set_lattice also sets
 * the step counter and clears the records.  Both wait. */
int pcpd_paper_get_lattice(const pcpd_paper_t *h, uint32_t *host_out);
int pcpd_paper_set_lattice(pcpd_paper_t *h, const uint32_t *host_in, uint64_t step);

/* Launch shape: systems per CTA, threads per CTA, CTAs, dynamic shared memory per CTA. */
int pcpd_paper_get_plan(const pcpd_paper_t *h, uint32_t *systems_per_cta, uint32_t *threads,
                        uint32_t *grid, size_t *smem_bytes);

int pcpd_paper_sync(pcpd_paper_t *h);
void pcpd_paper_destroy(pcpd_paper_t *h);

/* ---- allocation-free sweep ----
 * Advance a caller-owned lattice by n_substeps sub-steps without allocating any memory.
 * The paper has no counterpart: this is an entry point for callers that cannot let a
 * library allocate -- a host application whose device memory is all owned by its own pool
 * or arena, or a latency-critical loop that cannot afford cudaMalloc/cudaFree, which can
 * synchronize the whole device and can fail on a fragmented heap.  The caller passes the
 * lattice in and out; the library's scratch (one epoch flag per tile, a work counter and an
 * error word) is a fixed array of 16384 + 64 words inside the library, present on every GPU
 * that loads it until the process exits.
 *   lat_in   device, canonical layout [samples/32][L] uint32, 4-byte aligned: the state after
 *            substep_begin sub-steps.  It is also used as work space: its contents are
 *            undefined afterwards.
 *   lat_out  device, same layout, not overlapping lat_in: receives the state after
 *            substep_begin + n_substeps sub-steps (bit-identical to pcpd_run_substeps).
 *   L, samples, p, d, seed   as for pcpd_create; stream: cudaStream_t or NULL.
 * The call is synchronous: it waits on `stream` after every launch to read the error word
 * into host memory.  Errors: PCPD_EINVAL (bad sizes or pointers, or more
 * tiles per epoch than the scratch holds -- about 16384 columns of up to ~50k sites, fewer
 * for longer columns), PCPD_ENODEV, PCPD_ECUDA, PCPD_ETIMEOUT.  After any error the contents
 * of both lattices are undefined (a run may stop between two launches, with the newest state
 * in either buffer).
 * Every call shares the one scratch array and clears it first; calls that overlap on the GPU
 * (from several threads or streams at once) race on it and must not be made.  Every call
 * looks up the array's device address on the current device (cudaGetSymbolAddress, which
 * allocates nothing), so the call stays valid after a cudaDeviceReset. */
int pcpd_sweep_noalloc(uint32_t *lat_in, uint32_t *lat_out, uint32_t L, uint32_t samples, double p,
                       double d, uint64_t seed, uint64_t substep_begin, uint64_t n_substeps,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PCPD_H */
