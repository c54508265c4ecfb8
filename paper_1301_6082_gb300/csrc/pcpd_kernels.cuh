// pcpd_kernels.cuh -- device code of the bit-sliced PCPD sweep (sm_103a).
//
// The PCPD of Eq. (1) (Sec. 2) on a periodic lattice, one independent sample per bit of a
// 32-bit word (multispin coding, Sec. 4).  Each sub-step draws a random phase phi and tiles
// the ring with K = floor(L/3) non-overlapping windows (phi+3k, phi+3k+1, phi+3k+2); each
// window makes one bond attempt per sample with Alg. 1's decision tree, evaluated as
// branch-free bit logic in the spirit of Alg. 2.  Per-sample rate decisions compare a 32-bit
// draw u with integer thresholds floor(rate*2^32), bit-sliced over 32 random "planes" and
// evaluated most-significant plane first with an early exit -- the exact generalisation of
// the dyadic AND/OR masks of Sec. 4.2-4.3.  Random words come from Philox4x32-10 (Salmon et
// al., SC'11) keyed by the seed and counted by (sub-step, window, group, tag|block).  The
// triplet and quadruplet processes (TCPD, QCPD) use the same draws on windows of 4 and 5
// sites (window_update_n).
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace pcpdk {

// Debug builds (-DPCPD_DEBUG) check every shared- and global-memory index the kernels form;
// a failed check records its code (the first one wins) and skips the access, and the host
// reads the code through pcpd_debug_check().  Release builds compile the checks away.
#ifdef PCPD_DEBUG
__device__ unsigned int g_debug_err;
__device__ __forceinline__ bool debug_in_bounds(unsigned long long i, unsigned long long n,
                                                unsigned int code) {
  if (i < n) return true;
  atomicCAS(&g_debug_err, 0u, code);
  return false;
}
#define PCPD_IN_BOUNDS(i, n, code) pcpdk::debug_in_bounds((i), (n), (code))
#else
#define PCPD_IN_BOUNDS(i, n, code) true
#endif
constexpr unsigned int kDbgWindow = 1u, kDbgLoadDst = 2u, kDbgLoadSrc = 3u, kDbgStore = 4u,
                       kDbgPaper = 5u, kDbgRecord = 6u;

constexpr uint32_t kTagDyn = 0u;
constexpr uint32_t kTagPhase = 1u;
constexpr uint32_t kTagInit = 2u;

// Philox4x32 round multipliers and Weyl key increments (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Ten Philox4x32 rounds in place on (x0..x3) under key (k0, k1).
__device__ __forceinline__ void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                              uint32_t &x3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)x0 * kPhiloxM0;
    const uint64_t p1 = (uint64_t)x2 * kPhiloxM1;
    x0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    x1 = (uint32_t)p1;
    x2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    x3 = (uint32_t)p0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
}

// Round keys of Philox4x32-10 for one seed: key r = (k0 + r*W0, k1 + r*W1), r = 0..9.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys make_round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0 + (uint32_t)r * kPhiloxW0;
    rk.k1[r] = k1 + (uint32_t)r * kPhiloxW1;
  }
  return rk;
}

// Ten Philox4x32 rounds with the keys taken from a RoundKeys table (kernel constants).  The
// 64-bit products are formed as separate high and low 32-bit multiplies (same values; measured
// slightly faster on GB300 than the wide multiply).
__device__ __forceinline__ void philox4x32_10_rk(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                                 uint32_t &x3, const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t h0 = __umulhi(x0, kPhiloxM0), l0 = x0 * kPhiloxM0;
    const uint32_t h1 = __umulhi(x2, kPhiloxM1), l1 = x2 * kPhiloxM1;
    x0 = h1 ^ x1 ^ rk.k0[r];
    x1 = l1;
    x2 = h0 ^ x3 ^ rk.k1[r];
    x3 = l0;
  }
}

// Thresholds of one instance, pre-split for the plane compare.  A threshold T in [0, 2^32]:
// `full` = T == 2^32 (every draw is below it), else `t` = T.
// lo_d / lo_da: the lowest plane that still matters for T (T's bits below it are all zero,
// so a lane whose prefix equals T's is already known to satisfy u >= T); 32 when no plane
// matters (T = 0 or T = 2^32).
struct Thresholds {
  uint32_t td, tda;
  uint32_t td_full, tda_full;
  uint32_t lo_d, lo_da;
  uint32_t tmD[32], tmA[32];   // tm[m] = all ones if bit m of T is set, else 0
};

// Compare state of 32 lanes against one threshold: `lt` = decided u < T, `eq` = undecided
// (u's planes so far equal T's bits); lanes in neither are decided u >= T.
struct Cmp {
  uint32_t lt, eq;
};

__device__ __forceinline__ Cmp cmp_init(uint32_t t, uint32_t full) {
  Cmp c;
  c.lt = full ? 0xFFFFFFFFu : 0u;
  c.eq = (full || t == 0u) ? 0u : 0xFFFFFFFFu;
  return c;
}

// Fold the K planes m_hi, m_hi-1, ..., m_hi-K+1 (words w[0..K-1]) into the compare state.
// Within the group: eq_g = AND over planes of (P == T bit), and lt_g = (planes < T's bits)
// by a borrow chain run least-significant plane first, b' = (~P & t) | (~(P ^ t) & b) --
// each a single three-input logic operation with T's bit mask t as a kernel constant.
// Then lt |= eq & lt_g and eq &= eq_g: lanes still equal above the group are decided by it.
template <int K>
__device__ __forceinline__ void cmp_group(Cmp &c, const uint32_t (&w)[K], const uint32_t *tm,
                                          int m_hi) {
  uint32_t eq = c.eq, b = 0u;
#pragma unroll
  for (int q = 0; q < K; ++q) eq &= ~(w[q] ^ tm[m_hi - q]);
#pragma unroll
  for (int q = K - 1; q >= 0; --q) {
    const uint32_t t = tm[m_hi - q], P = w[q];
    b = (~P & t) | (~(P ^ t) & b);
  }
  c.lt |= c.eq & b;
  c.eq = eq;
}

// The same fold with the threshold T a compile-time constant (a specialised build of the
// engine for one (T_D, T_DA) pair): each plane's bit selects its operation, so two planes
// merge into one logic operation where the compiler can.
template <uint32_t T, int K>
__device__ __forceinline__ void cmp_group_ct(Cmp &c, const uint32_t (&w)[K], int m_hi) {
  uint32_t eq = c.eq, b = 0u;
#pragma unroll
  for (int q = 0; q < K; ++q) eq &= ((T >> (m_hi - q)) & 1u) ? w[q] : ~w[q];
#pragma unroll
  for (int q = K - 1; q >= 0; --q) {
    const uint32_t P = w[q];
    b = ((T >> (m_hi - q)) & 1u) ? (~P | b) : (~P & b);
  }
  c.lt |= c.eq & b;
  c.eq = eq;
}

// True while some lane is undecided after the planes down to m_lo and T has a set bit below
// m_lo (if T's lower bits are all zero, a lane equal so far is already known u >= T).
__device__ __forceinline__ bool cmp_open2(const Cmp &c, uint32_t lo, int m_lo) {
  return c.eq != 0u && (uint32_t)m_lo > lo;
}

// Rate masks of one (sub-step n, window k, group g): D = lanes with u < T_D (diffuse),
// A = lanes with T_D <= u < T_DA (annihilate an occupied bond), O = orientation bits.
// Block b of the counter (n, k, g, b) holds (O, P31, P30, P29) for b = 0 and
// (P_{32-4b} .. P_{29-4b}) for b >= 1; block 8 holds P0 in its first word.
struct Masks {
  uint32_t D, A, O;
};

// One window (a, b, c) for 32 samples of the PCPD (Alg. 1's tree on the bond the orientation picks,
// written as bit logic like Alg. 2).  Lane with o=0: bond (a,b), fission target c; o=1: bond
// (b,c), target a.  ltD = lanes with u < T_D: swap the bond; ltA = lanes with u < T_DA, which
// contains ltD: those that do not swap clear an occupied bond; the rest (u >= T_DA) fill the
// target next to an occupied bond.  A swapping lane ignores the clear, so the clear can be
// written with ltA rather than ltA & ~ltD (one operation fewer, same bits).
__device__ __forceinline__ void window_update(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t O,
                                              uint32_t ltD, uint32_t ltA) {
  const uint32_t q = (O & c) | (~O & a);         // partner of b
  const uint32_t t = (O & a) | (~O & c);         // fission target
  const uint32_t xb = b & ~(ltA & q);            // b after an annihilation
  const uint32_t xq = q & ~(ltA & b);            // partner after an annihilation
  const uint32_t nb = (ltD & q) | (~ltD & xb);   // a diffusion swaps b and its partner
  const uint32_t nq = (ltD & b) | (~ltD & xq);
  const uint32_t nt = t | (b & q & ~ltA);        // fission fills the target
  a = (O & nt) | (~O & nq);
  c = (O & nq) | (~O & nt);
  b = nb;
}

// One window of W = n+1 sites for 32 samples of the n-tuple process (R14; n = 3 TCPD, 4 QCPD):
// lane with o=0: tuple (s_0..s_{n-1}), diffusion bond (s_0, s_1), fission target s_n; o=1:
// tuple (s_1..s_n), bond (s_1, s_2), target s_0.  D: swap the bond; A: empty a full tuple;
// otherwise (F) fill the target next to a full tuple.  (W = 3 is window_update above.)
template <int W>
__device__ __forceinline__ void window_update_n(uint32_t (&s)[W], const Masks &m) {
  constexpr int n = W - 1;
  uint32_t mid = s[1];
#pragma unroll
  for (int j = 2; j < n; ++j) mid &= s[j];
  const uint32_t occ = mid & ((m.O & s[n]) | (~m.O & s[0]));   // the tuple is full
  const uint32_t ann = m.A & occ;
  const uint32_t fis = occ & ~(m.D | m.A);
  const uint32_t d0 = m.D & ~m.O, d1 = m.D & m.O;               // bond (s0,s1) / (s1,s2)
  const uint32_t n0 = (d0 & s[1]) | (~d0 & s[0]);
  const uint32_t n1 = (d0 & s[0]) | (d1 & s[2]) | (~m.D & s[1]);
  const uint32_t n2 = (d1 & s[1]) | (~d1 & s[2]);
  s[0] = n0;
  s[1] = n1;
  s[2] = n2;
  // a reacting lane did not diffuse, so these act on the lane's original sites
  s[0] &= ~(ann & ~m.O);
#pragma unroll
  for (int j = 1; j < n; ++j) s[j] &= ~ann;
  s[n] &= ~(ann & m.O);
  s[n] |= fis & ~m.O;
  s[0] |= fis & m.O;
}

// Random phase of sub-step n for phase group h: floor(x0 * L / 2^32).
__device__ __forceinline__ uint32_t phase_of(uint32_t n, uint32_t h, uint32_t L, uint32_t k0,
                                             uint32_t k1) {
  uint32_t x0 = 0u, x1 = n, x2 = h, x3 = kTagPhase << 28;
  philox4x32_10(x0, x1, x2, x3, k0, k1);
  return (uint32_t)(((uint64_t)x0 * L) >> 32);
}

// ---------------------------------------------------------------------------------------
// Tiles.  A CTA owns a tile of 32-sample group columns in shared memory:
//  RING: whole columns (tile = L sites each, periodic indexing);
//  SEGMENT: core sites [s0, s0+core) of one column plus a halo of H sites on each side
//  (temporal blocking): the windows of each sub-step are computed wherever all three sites
//  are still valid, and the valid region shrinks by at most 2 sites per side per sub-step,
//  so after tau <= H/2 sub-steps the core is exact.  Windows inside the halo are recomputed
//  redundantly; counter-based random numbers make the recomputation identical.
// ---------------------------------------------------------------------------------------
constexpr int kPhiChunk = 256;

// Count occupied sites of tile words [y0, y1) of group g into record r: the total into
// rec_total[r], occupied nearest-neighbour pairs (y, y+1) into rec_pairs[r] -- the pair
// density analysed beside the particle density in Sec. 5.3 -- and, if rec_sample is set,
// sample 32g+j's count into rec_sample[r*S + 32g + j].  ring_len != 0: the words are a whole
// ring of that length and the last site pairs with the first; otherwise word y1 (one past the
// range) must be valid.  s_red: 34 zeroed shared words, left zeroed.
__device__ __forceinline__ void tile_count(const uint32_t *sm, uint32_t y0, uint32_t y1,
                                           unsigned long long *rec_total, uint32_t *rec_sample,
                                           unsigned long long *rec_pairs, uint32_t S, uint32_t r,
                                           uint32_t g, uint32_t ring_len, unsigned int *s_red) {
  unsigned int local = 0, pairs = 0;
  for (uint32_t y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
    const uint32_t w = sm[y];
    uint32_t yn = y + 1u;
    if (ring_len && yn == ring_len) yn = 0u;
    local += __popc(w);
    pairs += __popc(w & sm[yn]);
  }
  local = __reduce_add_sync(0xFFFFFFFFu, local);
  pairs = __reduce_add_sync(0xFFFFFFFFu, pairs);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_red[32], local);
    atomicAdd(&s_red[33], pairs);
  }
  if (rec_sample) {
    unsigned int cnt[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) cnt[j] = 0;
    for (uint32_t y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
      const uint32_t w = sm[y];
#pragma unroll
      for (int j = 0; j < 32; ++j) cnt[j] += (w >> j) & 1u;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const unsigned int v = __reduce_add_sync(0xFFFFFFFFu, cnt[j]);
      if ((threadIdx.x & 31) == 0) atomicAdd(&s_red[j], v);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&rec_total[r], (unsigned long long)s_red[32]);
    if (rec_pairs) atomicAdd(&rec_pairs[r], (unsigned long long)s_red[33]);
  }
  if (rec_sample && threadIdx.x < 32)
    atomicAdd(&rec_sample[(size_t)r * S + 32u * g + threadIdx.x], s_red[threadIdx.x]);
  __syncthreads();
  for (uint32_t t = threadIdx.x; t <= 33u; t += blockDim.x) s_red[t] = 0;
  __syncthreads();
}

// Per-sub-step geometry of the windows a tile computes.  Candidate i is window k(i) with
// first site at tile index y(i); RING: k = i, y = (phi + W*i) mod L; SEGMENT: k = k_lo + i
// (mod K) and y = y_first + W*i, plus the idle gap L - W*K once k wraps from K-1 to 0.
struct Geometry {
  uint32_t phi, n_cand, k_lo, gap;
  int y_first;
  uint32_t lo, hi;
};

// Window k and the tile indexes of its W sites (RING: each reduced mod L).
template <bool RING, int W>
__device__ __forceinline__ bool candidate(const Geometry &G, uint32_t i, uint32_t L, uint32_t K,
                                          uint32_t &k, uint32_t (&idx)[W]) {
  if (i >= G.n_cand) return false;
  if (RING) {
    k = i;
    uint32_t a = G.phi + (uint32_t)W * i;   // phi < L and W*i < W*K <= L
    if (a >= L) a -= L;
    idx[0] = a;
#pragma unroll
    for (int j = 1; j < W; ++j) {
      a += 1u;
      if (a >= L) a -= L;
      idx[j] = a;
    }
    return true;
  } else {
    k = G.k_lo + i;
    int y = G.y_first + W * (int)i;
    if (k >= K) {
      k -= K;
      y += (int)G.gap;
    }
    if (y < (int)G.lo || y + (W - 1) >= (int)G.hi) return false;
#pragma unroll
    for (int j = 0; j < W; ++j) idx[j] = (uint32_t)(y + j);
    return true;
  }
}

// Every window draws blocks 0-2 (O and planes 31..21) up front: with 32 lanes per item a
// block-by-block early exit would make the whole warp wait for its slowest lane.  The few
// windows still undecided after plane 21 (about 3% for generic thresholds) are deferred to a
// per-CTA list and finished after the first pass of the sub-step with blocks 3..8, so their
// extra blocks run on compacted lanes.  Entries keep the candidate index, O and the compare
// state.
constexpr int kQ3Cap = 1024;  // per CTA; overflow is processed in place
constexpr int kQFields = 6;   // i, O, ltD, eqD, ltA, eqA

__host__ __device__ constexpr size_t sweep_queue_words(int nwarps) {
  return (void)nwarps, (size_t)kQFields * kQ3Cap;
}

// Finish an item from block 3 on: draw blocks 3.. until both compares are closed.
__device__ __forceinline__ void finish_from3(uint32_t k, uint32_t n, uint32_t g,
                                             const RoundKeys &rk, const Thresholds &T,
                                             Cmp &cD, Cmp &cA) {
#pragma unroll
  for (int b = 3; b <= 8; ++b) {
    const int m_prev = 33 - 4 * b;
    if (!cmp_open2(cD, T.lo_d, m_prev) && !cmp_open2(cA, T.lo_da, m_prev)) break;
    uint32_t x0 = n, x1 = k, x2 = g, x3 = (kTagDyn << 28) | (uint32_t)b;
    philox4x32_10_rk(x0, x1, x2, x3, rk);
    if (b < 8) {
      const uint32_t w[4] = {x0, x1, x2, x3};
      cmp_group<4>(cD, w, T.tmD, 32 - 4 * b);
      cmp_group<4>(cA, w, T.tmA, 32 - 4 * b);
    } else {
      const uint32_t w[1] = {x0};
      cmp_group<1>(cD, w, T.tmD, 0);
      cmp_group<1>(cA, w, T.tmA, 0);
    }
  }
}

template <int W>
__device__ __forceinline__ void apply_window(uint32_t *sm, const uint32_t (&idx)[W], uint32_t O,
                                             uint32_t ltD, uint32_t ltA, uint32_t lim) {
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (!PCPD_IN_BOUNDS(idx[j], lim, kDbgWindow)) return;
  (void)lim;
  if constexpr (W == 3) {
    uint32_t a = sm[idx[0]], b = sm[idx[1]], c = sm[idx[2]];
    window_update(a, b, c, O, ltD, ltA);
    sm[idx[0]] = a;
    sm[idx[1]] = b;
    sm[idx[2]] = c;
  } else {
    uint32_t s[W];
#pragma unroll
    for (int j = 0; j < W; ++j) s[j] = sm[idx[j]];
    Masks m;
    m.D = ltD;
    m.A = ltA & ~ltD;   // T_D <= u < T_DA
    m.O = O;
    window_update_n<W>(s, m);
#pragma unroll
    for (int j = 0; j < W; ++j) sm[idx[j]] = s[j];
  }
}

// Initial lattice: mode 0 full, 1 empty, 2 i.i.d. Bernoulli(1/2) bits (Philox tag INIT,
// counter (i, 0, g_base + g, INIT<<28), first word; g_base = the instance's first group).
__global__ void k_init(uint32_t *lat, uint32_t L, uint32_t pitch, uint32_t G, int mode, uint32_t k0,
                       uint32_t k1, uint32_t g_base) {
  const size_t total = (size_t)G * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const uint32_t g = (uint32_t)(idx / L), i = (uint32_t)(idx % L);
    uint32_t v;
    if (mode == 0) v = 0xFFFFFFFFu;
    else if (mode == 1) v = 0u;
    else {
      uint32_t x0 = i, x1 = 0u, x2 = g_base + g, x3 = kTagInit << 28;
      philox4x32_10(x0, x1, x2, x3, k0, k1);
      v = x0;
    }
    lat[(size_t)g * pitch + i] = v;
  }
}

// Record of the current state (no sub-step): one CTA per group.
__global__ void k_count(const uint32_t *lat, uint32_t L, uint32_t pitch, uint32_t S,
                        unsigned long long *rec_total, uint32_t *rec_sample,
                        unsigned long long *rec_pairs) {
  const uint32_t g = blockIdx.x;
  const uint32_t *col = lat + (size_t)g * pitch;
  unsigned int local = 0, pairs = 0;
  unsigned int cnt[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) cnt[j] = 0;
  for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
    const uint32_t w = col[i];
    local += __popc(w);
    pairs += __popc(w & col[i + 1u == L ? 0u : i + 1u]);
    if (rec_sample) {
#pragma unroll
      for (int j = 0; j < 32; ++j) cnt[j] += (w >> j) & 1u;
    }
  }
  local = __reduce_add_sync(0xFFFFFFFFu, local);
  pairs = __reduce_add_sync(0xFFFFFFFFu, pairs);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(rec_total, (unsigned long long)local);
    if (rec_pairs) atomicAdd(rec_pairs, (unsigned long long)pairs);
  }
  if (rec_sample) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const unsigned int v = __reduce_add_sync(0xFFFFFFFFu, cnt[j]);
      if ((threadIdx.x & 31) == 0) atomicAdd(&rec_sample[32u * g + j], v);
    }
  }
}

// Test entry: Philox on explicit counters.
__global__ void k_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    uint32_t x0 = ctr[4 * i], x1 = ctr[4 * i + 1], x2 = ctr[4 * i + 2], x3 = ctr[4 * i + 3];
    philox4x32_10(x0, x1, x2, x3, k0, k1);
    out[4 * i] = x0;
    out[4 * i + 1] = x1;
    out[4 * i + 2] = x2;
    out[4 * i + 3] = x3;
  }
}

// Test entry: the MSB-first plane compare on explicit words (O, P31..P0) per item, with
// the grouping and exit rule of the sweep (planes 31..21 first, then blocks 3..8).
__global__ void k_rate_masks(const uint32_t *words, Thresholds T, uint32_t *masks, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t *w = words + 33 * i;   // w[1 + q] = plane 31 - q
    Cmp cD = cmp_init(T.td, T.td_full), cA = cmp_init(T.tda, T.tda_full);
    {
      const uint32_t g11[11] = {w[1], w[2], w[3], w[4], w[5], w[6], w[7], w[8], w[9], w[10], w[11]};
      cmp_group<11>(cD, g11, T.tmD, 31);
      cmp_group<11>(cA, g11, T.tmA, 31);
    }
#pragma unroll
    for (int b = 3; b <= 8; ++b) {
      const int m_prev = 33 - 4 * b;
      if (!cmp_open2(cD, T.lo_d, m_prev) && !cmp_open2(cA, T.lo_da, m_prev)) break;
      const int m0 = 32 - 4 * b;
      if (b < 8) {
        const uint32_t g[4] = {w[32 - m0], w[33 - m0], w[34 - m0], w[35 - m0]};
        cmp_group<4>(cD, g, T.tmD, m0);
        cmp_group<4>(cA, g, T.tmA, m0);
      } else {
        const uint32_t g[1] = {w[32]};
        cmp_group<1>(cD, g, T.tmD, 0);
        cmp_group<1>(cA, g, T.tmA, 0);
      }
    }
    masks[3 * i] = cD.lt;
    masks[3 * i + 1] = cA.lt & ~cD.lt;
    masks[3 * i + 2] = w[0];
  }
}

}  // namespace pcpdk
