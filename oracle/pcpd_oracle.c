/*
 * pcpd_oracle.c -- plain, slow, scalar CPU oracle for the bit-sliced PCPD sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file: only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (the paper: Schram, arXiv 1301.6082):
 *   - the PCPD reactions of Eq. (1) with the bond-level decision tree of Alg. 1 (Sec. 2);
 *   - on the parallel schedule of non-overlapping 3-site windows with a random phase per
 *     sub-step (the reading of Sec. 3's "same local site" schedule that this project uses);
 *   - with one rate draw u per sample and window, compared with integer thresholds
 *     floor(rate * 2^32), the exact generalisation of the dyadic masks of Sec. 4.2-4.3;
 *   - random bits from Philox4x32-10 (Salmon et al., SC'11), keyed by seed and counted by
 *     (sub-step, window, group, tag|block);
 *   - and, separately, Alg. 1 itself (random-sequential updates) as a statistical reference.
 *
 * Every sample is simulated one at a time on a byte per site.  All 32 bit planes of u are
 * always computed (no early exit).  Parallelism over 32-sample groups with pthreads only
 * splits independent work; it changes no arithmetic and integer sums are order-free.
 *
 * Pins: every function is checked in tests/test_oracle_*.py against something other than
 * itself (a third-party Philox, closed forms, invariants, exact master equations).
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (see oracle/oracle.py).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_DYN 0u
#define ORC_TAG_PHASE 1u
#define ORC_TAG_INIT 2u
#define ORC_TAG_RS 3u
#define ORC_TWO32 4294967296ull

/* ---------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  One round: (x0,x1,x2,x3) -> (hi(M1*x2)^x1^k0, lo(M1*x2), hi(M0*x0)^x3^k1,
 * lo(M0*x0)); the key is bumped by the Weyl constants after every round; ten rounds.
 * ------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void orc_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Batch form for tests: n counters (row-major [n][4]) -> n outputs [n][4]. */
void orc_philox_batch(const uint32_t *ctrs, uint64_t seed, uint32_t *outs, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i)
        orc_block(seed, ctrs[4 * i], ctrs[4 * i + 1], ctrs[4 * i + 2], ctrs[4 * i + 3],
                  outs + 4 * i);
}

/* ---------------------------------------------------------------------------------------
 * Thresholds, the integer form of the rates of Eq. (1): P(diffuse) = d, P(annihilate) =
 * p(1-d), P(fission) = (1-p)(1-d).  Double precision, evaluated exactly as written, no
 * contraction: T_D = min(2^32, floor(d*2^32)), T_A = floor(p*(1-d)*2^32),
 * T_DA = min(2^32, T_D + T_A).  Random-sequential form (Alg. 1): T_P = min(2^32, floor(p*2^32)).
 * ------------------------------------------------------------------------------------- */
static uint64_t orc_floor_scaled(double x)
{
    double f = floor(x);
    if (f <= 0.0) return 0;
    if (f >= 4294967296.0) return ORC_TWO32;
    return (uint64_t)f;
}

int orc_thresholds(double p, double d, uint64_t *t_d, uint64_t *t_da, uint64_t *t_p)
{
    if (!(p >= 0.0 && p <= 1.0 && d >= 0.0 && d <= 1.0)) return 1;
    uint64_t td = orc_floor_scaled(d * 4294967296.0);
    double scaled_a = p * (1.0 - d);
    scaled_a = scaled_a * 4294967296.0;
    uint64_t ta = orc_floor_scaled(scaled_a);
    uint64_t tda = td + ta;
    if (tda > ORC_TWO32) tda = ORC_TWO32;
    if (t_d) *t_d = td;
    if (t_da) *t_da = tda;
    if (t_p) *t_p = orc_floor_scaled(p * 4294967296.0);
    return 0;
}

/* Time: after n sub-steps a sample has had n*K attempts, K = floor(L/W) windows of W sites
 * (W = 3 for the PCPD, W = n+1 for n-tuples); MCS time t (t*L attempts) is reached at
 * sub-step ceil(t*L/K). */
uint64_t orc_substep_of_time_w(uint32_t L, uint32_t W, uint64_t t)
{
    unsigned __int128 K = L / W;
    unsigned __int128 num = (unsigned __int128)t * L;
    return (uint64_t)((num + K - 1) / K);
}

uint64_t orc_substep_of_time(uint32_t L, uint64_t t)
{
    return orc_substep_of_time_w(L, 3u, t);
}

/* Random phase of sub-step n for phase group h: phi = floor(x0 * L / 2^32). */
uint32_t orc_phase(uint64_t seed, uint32_t L, uint32_t h, uint32_t n)
{
    uint32_t out[4];
    orc_block(seed, 0u, n, h, ORC_TAG_PHASE << 28, out);
    return (uint32_t)(((uint64_t)out[0] * (uint64_t)L) >> 32);
}

/* ---------------------------------------------------------------------------------------
 * Lattice state of the oracle: one byte per (sample, site), state[s*L + i] in {0,1}.
 * Initial states: 0 = full, 1 = empty, 2 = random half (bit j of the INIT word of group g
 * at site i is the occupation of sample 32g+j).  The state holds groups g0, g0+1, ...
 * ------------------------------------------------------------------------------------- */
int orc_init(uint8_t *state, uint32_t L, uint32_t S, int mode, uint64_t seed, uint32_t g0)
{
    if (S % 32u) return 1;
    for (uint32_t s = 0; s < S; ++s) {
        for (uint32_t i = 0; i < L; ++i) {
            uint8_t v;
            if (mode == 0) v = 1;
            else if (mode == 1) v = 0;
            else if (mode == 2) {
                uint32_t out[4];
                orc_block(seed, i, 0u, g0 + s / 32u, ORC_TAG_INIT << 28, out);
                v = (uint8_t)((out[0] >> (s % 32u)) & 1u);
            } else return 1;
            state[(uint64_t)s * L + i] = v;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * One window update for one sample: Alg. 1's decision tree (Eq. (1) rates through R3's
 * thresholds) on the tuple the orientation picks, for n-tuples (n = 2 is the PCPD; n = 3, 4
 * the TCPD and QCPD of R14).  site[0..n] are the W = n+1 consecutive sites of the window.
 *   o = 0: tuple site[0..n-1], diffusion bond (site[0], site[1]), fission target site[n]
 *          (Alg. 1 "fission high")
 *   o = 1: tuple site[1..n], diffusion bond (site[1], site[2]), fission target site[0]
 *          (Alg. 1 "fission low")
 * u < T_D: diffusion swaps the bond; else if all n tuple sites are occupied: u < T_DA empties
 * them, otherwise the target becomes occupied.  For n = 2: bond (a, b) -> target c, or bond
 * (b, c) -> target a.  Returns the change in particle number (one of +1, -n, 0).
 * ------------------------------------------------------------------------------------- */
static int orc_window(uint8_t *row, const uint32_t *site, uint32_t n, uint32_t o, uint64_t u,
                      uint64_t t_d, uint64_t t_da)
{
    const uint32_t first = o ? 1u : 0u;          /* the tuple's first site */
    const uint32_t target = o ? 0u : n;
    int before = 0;
    for (uint32_t j = 0; j <= n; ++j) before += row[site[j]];
    if (u < t_d) {
        uint8_t tmp = row[site[first]];
        row[site[first]] = row[site[first + 1]];
        row[site[first + 1]] = tmp;
    } else {
        uint32_t occupied = 0;   /* occupied sites of the tuple */
        for (uint32_t j = 0; j < n; ++j) occupied += row[site[first + j]];
        if (occupied == n) {
            if (u < t_da) {
                for (uint32_t j = 0; j < n; ++j) row[site[first + j]] = 0;
            } else {
                row[site[target]] = 1;
            }
        }
    }
    int after = 0;
    for (uint32_t j = 0; j <= n; ++j) after += row[site[j]];
    return after - before;
}

typedef struct {
    uint32_t L, S;
    uint32_t n;            /* tuple size: 2 PCPD, 3 TCPD, 4 QCPD; windows of n+1 sites */
    uint64_t t_d, t_da, seed;
    uint8_t *state;
    uint64_t n_begin, n_end;
    const uint64_t *rec_sub;
    uint32_t n_rec;
    uint64_t *rec_total;   /* [n_rec], summed over all threads under a mutex */
    uint64_t *rec_pairs;   /* [n_rec] occupied nearest-neighbour pairs, or NULL */
    uint32_t *rec_sample;  /* [n_rec][S] or NULL */
    uint64_t *events;      /* [3]: diffusion swaps that moved a particle, annihilations, fissions */
    pthread_mutex_t *mu;
    uint32_t g_begin, g_end;
    uint32_t g0;           /* group index of the state's first group (keys and phase groups) */
    int bad;               /* set if a window changed N by something other than +1, -n, 0 */
} orc_job;

/* Record r: occupied sites, and occupied nearest-neighbour pairs (i, i+1 mod L) -- the pair
 * density the paper analyses beside the particle density (Sec. 5.3). */
static void orc_count(orc_job *jb, uint32_t g, uint32_t r, uint64_t *tot, uint64_t *pairs)
{
    for (uint32_t j = 0; j < 32; ++j) {
        uint32_t s = 32u * g + j;
        const uint8_t *row = jb->state + (uint64_t)s * jb->L;
        uint32_t cnt = 0, pc = 0;
        for (uint32_t i = 0; i < jb->L; ++i) {
            cnt += row[i];
            pc += row[i] & row[(i + 1u) % jb->L];
        }
        tot[r] += cnt;
        pairs[r] += pc;
        if (jb->rec_sample) jb->rec_sample[(uint64_t)r * jb->S + s] = cnt;
    }
}

static void *orc_worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    const uint32_t L = jb->L, n_tup = jb->n, W = n_tup + 1u, K = L / W;
    uint64_t *tot = (uint64_t *)calloc(jb->n_rec ? jb->n_rec : 1, sizeof(uint64_t));
    uint64_t *prs = (uint64_t *)calloc(jb->n_rec ? jb->n_rec : 1, sizeof(uint64_t));
    uint64_t ev[3] = {0, 0, 0};
    for (uint32_t g = jb->g_begin; g < jb->g_end; ++g) {
        const uint32_t gk = jb->g0 + g;        /* the group's index in the full instance */
        const uint32_t h = (32u * gk) / 128u;  /* phase group: 128 samples */
        uint32_t r = 0;
        while (r < jb->n_rec && jb->rec_sub[r] < jb->n_begin) ++r;
        for (uint64_t n = jb->n_begin;; ++n) {
            /* records of the state after n sub-steps */
            while (r < jb->n_rec && jb->rec_sub[r] == n) { orc_count(jb, g, r, tot, prs); ++r; }
            if (n == jb->n_end) break;
            const uint32_t phi = orc_phase(jb->seed, L, h, (uint32_t)n);
            for (uint32_t k = 0; k < K; ++k) {
                /* 33 words: O and planes P31..P0 (blocks 0..8) */
                uint32_t words[36];
                for (uint32_t b = 0; b < 9; ++b)
                    orc_block(jb->seed, (uint32_t)n, k, gk, (ORC_TAG_DYN << 28) | b, words + 4 * b);
                const uint32_t O = words[0];
                /* plane P_m is words[32 - m] for m = 31..0 */
                uint32_t site[8];
                for (uint32_t q = 0; q < W; ++q)
                    site[q] = (uint32_t)(((uint64_t)phi + (uint64_t)W * k + q) % L);
                for (uint32_t j = 0; j < 32; ++j) {
                    uint64_t u = 0;
                    for (int m = 31; m >= 0; --m)
                        u |= (uint64_t)((words[32 - m] >> j) & 1u) << m;
                    const uint32_t o = (O >> j) & 1u;
                    uint8_t *row = jb->state + (uint64_t)(32u * g + j) * L;
                    const uint32_t first = o ? 1u : 0u;
                    const int moved = row[site[first]] != row[site[first + 1]];
                    int dn = orc_window(row, site, n_tup, o, u, jb->t_d, jb->t_da);
                    if (dn != 0 && dn != 1 && dn != -(int)n_tup) jb->bad = 1;
                    if (dn == -(int)n_tup) ev[1]++;
                    else if (dn == 1) ev[2]++;
                    else if (u < jb->t_d && moved) ev[0]++;
                }
            }
        }
    }
    pthread_mutex_lock(jb->mu);
    for (uint32_t r = 0; r < jb->n_rec; ++r) {
        jb->rec_total[r] += tot[r];
        if (jb->rec_pairs) jb->rec_pairs[r] += prs[r];
    }
    if (jb->events) for (int e = 0; e < 3; ++e) jb->events[e] += ev[e];
    pthread_mutex_unlock(jb->mu);
    free(tot);
    free(prs);
    return NULL;
}

/*
 * Run the window schedule from the state after n_begin sub-steps to the state after n_end.
 * The state holds the S/32 groups g0, g0+1, ... of an instance (g0 = 0 for all of it).
 * rec_sub: sorted sub-step indices in [n_begin, n_end]; the state after rec_sub[r] sub-steps
 * is counted into rec_total[r] (+= over all samples), rec_sample[r][s] (if non-NULL) and the
 * occupied nearest-neighbour pairs into rec_pairs[r] (if non-NULL).
 * events (nullable, [3]) accumulates moving swaps, annihilations and fissions.
 * tuple: n = 2 (PCPD; 0 means 2), 3 (TCPD) or 4 (QCPD): windows of n+1 sites (R14).
 * Returns 0, or 1 on bad arguments, or 2 if the particle-number invariant failed.
 */
int orc_run(uint32_t L, uint32_t S, uint64_t t_d, uint64_t t_da, uint64_t seed,
            uint8_t *state, uint64_t n_begin, uint64_t n_end, const uint64_t *rec_sub,
            uint32_t n_rec, uint64_t *rec_total, uint32_t *rec_sample, uint64_t *events,
            int n_threads, uint32_t g0, uint64_t *rec_pairs, uint32_t tuple)
{
    if (tuple == 0) tuple = 2u;
    if (tuple < 2u || tuple > 4u || L < tuple + 1u || S % 32u || n_end < n_begin || n_end > 0xFFFFFFFFull)
        return 1;
    const uint32_t G = S / 32u;
    if (n_threads < 1) n_threads = 1;
    if ((uint32_t)n_threads > G) n_threads = (int)G;
    for (uint32_t r = 0; r < n_rec; ++r) {
        rec_total[r] = 0;
        if (rec_pairs) rec_pairs[r] = 0;
    }
    if (events) events[0] = events[1] = events[2] = 0;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    orc_job *jobs = (orc_job *)calloc((size_t)n_threads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        orc_job *jb = &jobs[t];
        jb->L = L; jb->S = S; jb->n = tuple; jb->t_d = t_d; jb->t_da = t_da; jb->seed = seed;
        jb->state = state; jb->n_begin = n_begin; jb->n_end = n_end;
        jb->rec_sub = rec_sub; jb->n_rec = n_rec; jb->rec_total = rec_total;
        jb->rec_sample = rec_sample; jb->events = events; jb->mu = &mu;
        jb->rec_pairs = rec_pairs;
        jb->g_begin = (uint32_t)((uint64_t)G * t / n_threads);
        jb->g_end = (uint32_t)((uint64_t)G * (t + 1) / n_threads);
        jb->g0 = g0;
        pthread_create(&th[t], NULL, orc_worker, jb);
    }
    int bad = 0;
    for (int t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        bad |= jobs[t].bad;
    }
    free(jobs);
    free(th);
    return bad ? 2 : 0;
}

/* ---------------------------------------------------------------------------------------
 * Alg. 1, random-sequential: attempt m of sample s draws the Philox block
 * (m lo, m hi, s, TAG_RS<<28).  Site i = floor(x0*L/2^32); diffuse iff x1 < T_D; else, on
 * an occupied pair (i, i+1), annihilate iff x2 < T_P, else fission to i-1 iff x3 < 2^31,
 * otherwise to i+2.  One attempt is 1/L MCS.  Records at MCS times (state after t*L
 * attempts).  attempt_begin is the global attempt index of the first attempt.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    uint32_t L, S;
    uint64_t t_d, t_p, seed;
    uint8_t *state;
    uint64_t a_begin, a_end;
    const uint64_t *rec_att;
    uint32_t n_rec;
    uint64_t *rec_total;
    uint32_t *rec_sample;
    pthread_mutex_t *mu;
    uint32_t s_begin, s_end;
} orc_rs_job;

static void *orc_rs_worker(void *arg)
{
    orc_rs_job *jb = (orc_rs_job *)arg;
    const uint32_t L = jb->L;
    uint64_t *tot = (uint64_t *)calloc(jb->n_rec ? jb->n_rec : 1, sizeof(uint64_t));
    for (uint32_t s = jb->s_begin; s < jb->s_end; ++s) {
        uint8_t *q = jb->state + (uint64_t)s * L;
        uint32_t r = 0;
        while (r < jb->n_rec && jb->rec_att[r] < jb->a_begin) ++r;
        for (uint64_t m = jb->a_begin;; ++m) {
            while (r < jb->n_rec && jb->rec_att[r] == m) {
                uint32_t cnt = 0;
                for (uint32_t i = 0; i < L; ++i) cnt += q[i];
                tot[r] += cnt;
                if (jb->rec_sample) jb->rec_sample[(uint64_t)r * jb->S + s] = cnt;
                ++r;
            }
            if (m == jb->a_end) break;
            uint32_t x[4];
            orc_block(jb->seed, (uint32_t)m, (uint32_t)(m >> 32), s, ORC_TAG_RS << 28, x);
            const uint32_t i = (uint32_t)(((uint64_t)x[0] * L) >> 32);
            const uint32_t i1 = (i + 1u) % L;
            if ((uint64_t)x[1] < jb->t_d) {
                uint8_t tmp = q[i];
                q[i] = q[i1];
                q[i1] = tmp;
            } else if (q[i] == 1 && q[i1] == 1) {
                if ((uint64_t)x[2] < jb->t_p) {
                    q[i] = 0;
                    q[i1] = 0;
                } else if (x[3] < 0x80000000u) {
                    q[(i + L - 1u) % L] = 1;
                } else {
                    q[(i + 2u) % L] = 1;
                }
            }
        }
    }
    pthread_mutex_lock(jb->mu);
    for (uint32_t r = 0; r < jb->n_rec; ++r) jb->rec_total[r] += tot[r];
    pthread_mutex_unlock(jb->mu);
    free(tot);
    return NULL;
}

int orc_rs_run(uint32_t L, uint32_t S, uint64_t t_d, uint64_t t_p, uint64_t seed,
               uint8_t *state, uint64_t a_begin, uint64_t a_end, const uint64_t *rec_att,
               uint32_t n_rec, uint64_t *rec_total, uint32_t *rec_sample, int n_threads)
{
    if (L < 3 || S == 0 || a_end < a_begin) return 1;
    if (n_threads < 1) n_threads = 1;
    if ((uint32_t)n_threads > S) n_threads = (int)S;
    for (uint32_t r = 0; r < n_rec; ++r) rec_total[r] = 0;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    orc_rs_job *jobs = (orc_rs_job *)calloc((size_t)n_threads, sizeof(orc_rs_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        orc_rs_job *jb = &jobs[t];
        jb->L = L; jb->S = S; jb->t_d = t_d; jb->t_p = t_p; jb->seed = seed;
        jb->state = state; jb->a_begin = a_begin; jb->a_end = a_end;
        jb->rec_att = rec_att; jb->n_rec = n_rec; jb->rec_total = rec_total;
        jb->rec_sample = rec_sample; jb->mu = &mu;
        jb->s_begin = (uint32_t)((uint64_t)S * t / n_threads);
        jb->s_end = (uint32_t)((uint64_t)S * (t + 1) / n_threads);
        pthread_create(&th[t], NULL, orc_rs_worker, jb);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return 0;
}

/* Canonical packing: word [g][i] bit j <-> state[(32g+j)*L + i]. */
void orc_pack(const uint8_t *state, uint32_t L, uint32_t S, uint32_t *words)
{
    for (uint32_t g = 0; g < S / 32u; ++g)
        for (uint32_t i = 0; i < L; ++i) {
            uint32_t w = 0;
            for (uint32_t j = 0; j < 32; ++j)
                w |= (uint32_t)(state[(uint64_t)(32u * g + j) * L + i] & 1u) << j;
            words[(uint64_t)g * L + i] = w;
        }
}

void orc_unpack(const uint32_t *words, uint32_t L, uint32_t S, uint8_t *state)
{
    for (uint32_t g = 0; g < S / 32u; ++g)
        for (uint32_t i = 0; i < L; ++i)
            for (uint32_t j = 0; j < 32; ++j)
                state[(uint64_t)(32u * g + j) * L + i] =
                    (uint8_t)((words[(uint64_t)g * L + i] >> j) & 1u);
}

/* ---------------------------------------------------------------------------------------
 * The paper's own GPU scheme (Sec. 3-4, Alg. 2), as a variant.  One system (a lattice of
 * L = 32 * n_loc * S_w sites) per workgroup of S_w workitems; bit b of workitem w's local
 * word i holds site b*(L/32) + w*n_loc + i ("connected lattices", Sec. 4).  Every step
 * draws one local site i* for the whole system and every workitem updates, for all 32 bits
 * at once, the bond (s, s+1) with s = b*(L/32) + w*n_loc + i*, fission going to s-1 or s+2
 * (all mod L).  Each RNG() of Alg. 2 returns the next word of the workitem's own random
 * stream; a step takes n_w = m + n_dec + 2 words in this order: m planes of the diffusion
 * draw (bit b diffuses iff its m-bit value, MSB first, is below T_d = d*2^m), n_dec
 * decorrelation words (ANDed), one word compared with T_c = floor(p*2^n_dec*2^32) and
 * broadcast to all bits (the correlated annihilation draw), one fission-direction word (bit
 * 1: high, s+2).  A bit annihilates iff no diffusion, an occupied pair, all decorrelation
 * bits 1 and the broadcast draw true.  One step = 32*S_w attempts; MCS time t is step
 * t*n_loc.
 * Random streams (Philox4x32-10 keyed by the seed): word k of workitem w's stream in system
 * sys is word k mod 4 of the block counted by (w, B mod 2^32, sys, TAG_PAPER<<28 | B>>32),
 * B = floor(k/4); step t takes words n_w*t .. n_w*t + n_w - 1.  The local site of step t is
 * floor(x * n_loc / 2^32), x = word t mod 4 of the block (0, floor(t/4), sys,
 * TAG_PAPER_SITE<<28).  state: bytes [systems][L] of systems sys0, sys0+1, ...;
 * rec_sys (nullable): per-system counts [n_rec][systems].
 * ------------------------------------------------------------------------------------- */
#define ORC_TAG_PAPER 4u
#define ORC_TAG_PAPER_SITE 5u

/* Word k of workitem w's stream in system sys. */
static uint32_t orc_paper_word(uint64_t seed, uint32_t w, uint32_t sys, uint64_t k)
{
    uint32_t x[4];
    const uint64_t B = k / 4u;
    orc_block(seed, w, (uint32_t)B, sys, (ORC_TAG_PAPER << 28) | (uint32_t)(B >> 32), x);
    return x[k % 4u];
}

int orc_paper_run(uint32_t n_loc, uint32_t S_w, uint32_t systems, uint32_t m, uint32_t t_d,
                  uint32_t n_dec, uint64_t t_c, uint64_t seed, uint8_t *state, uint64_t step_begin,
                  uint64_t step_end, const uint64_t *rec_step, uint32_t n_rec, uint64_t *rec_total,
                  uint32_t sys0, uint32_t *rec_sys)
{
    if (n_loc < 4 || S_w == 0 || m > 16 || (t_d > (1u << m)) || n_dec > 16 ||
        step_end > 0xFFFFFFFFull || step_end < step_begin)
        return 1;
    const uint64_t L = 32ull * n_loc * S_w;
    const uint32_t nw = m + n_dec + 2;   /* words per workitem and step */
    for (uint32_t r = 0; r < n_rec; ++r) rec_total[r] = 0;
    uint32_t words[36];
    for (uint32_t sys = 0; sys < systems; ++sys) {
        uint8_t *q = state + (uint64_t)sys * L;
        const uint32_t gsys = sys0 + sys;
        uint32_t r = 0;
        while (r < n_rec && rec_step[r] < step_begin) ++r;
        for (uint64_t st = step_begin;; ++st) {
            while (r < n_rec && rec_step[r] == st) {
                uint64_t c = 0;
                for (uint64_t i = 0; i < L; ++i) c += q[i];
                rec_total[r] += c;
                if (rec_sys) rec_sys[(uint64_t)r * systems + sys] = (uint32_t)c;
                ++r;
            }
            if (st == step_end) break;
            uint32_t xs[4];
            orc_block(seed, 0u, (uint32_t)(st / 4u), gsys, ORC_TAG_PAPER_SITE << 28, xs);
            const uint32_t istar = (uint32_t)(((uint64_t)xs[st % 4u] * n_loc) >> 32);
            for (uint32_t w = 0; w < S_w; ++w) {
                for (uint32_t i = 0; i < nw; ++i)
                    words[i] = orc_paper_word(seed, w, gsys, (uint64_t)nw * st + i);
                const uint32_t corr = ((uint64_t)words[m + n_dec] < t_c) ? 1u : 0u;
                const uint32_t fis = words[m + n_dec + 1];
                for (uint32_t b = 0; b < 32; ++b) {
                    uint32_t u = 0;
                    for (uint32_t k = 0; k < m; ++k) u = (u << 1) | ((words[k] >> b) & 1u);
                    const int diffuse = u < t_d;
                    uint32_t dec = 1u;
                    for (uint32_t k = 0; k < n_dec; ++k) dec &= (words[m + k] >> b) & 1u;
                    const uint64_t s0 = (uint64_t)b * (L / 32) + (uint64_t)w * n_loc + istar;
                    const uint64_t s1 = (s0 + 1) % L, sl = (s0 + L - 1) % L, sh = (s0 + 2) % L;
                    if (diffuse) {
                        uint8_t t = q[s0];
                        q[s0] = q[s1];
                        q[s1] = t;
                    } else if (q[s0] && q[s1]) {
                        if (dec && corr) {
                            q[s0] = 0;
                            q[s1] = 0;
                        } else if ((fis >> b) & 1u) {
                            q[sh] = 1;
                        } else {
                            q[sl] = 1;
                        }
                    }
                }
            }
        }
    }
    return 0;
}
