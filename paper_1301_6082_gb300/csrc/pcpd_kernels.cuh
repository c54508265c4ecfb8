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
// al., SC'11) keyed by the seed and counted by (window, sub-step, group, tag|block).
#pragma once
#include <cstdint>

namespace pcpdk {

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

// Thresholds of one instance, pre-split for the plane compare.  A threshold T in [0, 2^32]:
// `full` = T == 2^32 (every draw is below it), else `t` = T.
struct Thresholds {
  uint32_t td, tda;
  uint32_t td_full, tda_full;
};

// Less/greater state of the MSB-first compare of 32 lanes against one threshold: lanes in
// `lt` are decided u < T, lanes in `gt` decided u >= T, the rest match T's bits so far.
__device__ __forceinline__ void cmp_plane(uint32_t &lt, uint32_t &gt, uint32_t plane, bool tbit) {
  if (tbit) lt |= ~(gt | plane);   // T bit 1: an undecided lane with bit 0 is below T
  else      gt |= plane & ~lt;     // T bit 0: an undecided lane with bit 1 is above T
}

// True while some lane is undecided against T after the planes down to `m` (inclusive) and T
// still has a non-zero bit below m (if all of T's lower bits are zero, a lane whose prefix
// equals T's is already known to satisfy u >= T).
__device__ __forceinline__ bool cmp_open(uint32_t lt, uint32_t gt, uint32_t t, bool full, int m) {
  const uint32_t low = (m == 0) ? 0u : (t & ((1u << m) - 1u));
  return !full && low != 0u && ((lt | gt) != 0xFFFFFFFFu);
}

// Rate masks of one (window k, sub-step n, group g): D = lanes with u < T_D (diffuse),
// A = lanes with T_D <= u < T_DA (annihilate an occupied bond), O = orientation bits.
// Block b of the counter (k, n, g, b) holds (O, P31, P30, P29) for b = 0 and
// (P_{32-4b} .. P_{29-4b}) for b >= 1; block 8 holds P0 in its first word.
struct Masks {
  uint32_t D, A, O;
};

__device__ __forceinline__ Masks rate_masks(uint32_t k, uint32_t n, uint32_t g, uint32_t k0,
                                            uint32_t k1, const Thresholds &T) {
  uint32_t ltD = T.td_full ? 0xFFFFFFFFu : 0u, gtD = (!T.td_full && T.td == 0u) ? 0xFFFFFFFFu : 0u;
  uint32_t ltA = T.tda_full ? 0xFFFFFFFFu : 0u, gtA = (!T.tda_full && T.tda == 0u) ? 0xFFFFFFFFu : 0u;
  uint32_t O;
  {
    uint32_t x0 = k, x1 = n, x2 = g, x3 = (kTagDyn << 28) | 0u;
    philox4x32_10(x0, x1, x2, x3, k0, k1);
    O = x0;
    if (!T.td_full) {
      cmp_plane(ltD, gtD, x1, (T.td >> 31) & 1u);
      cmp_plane(ltD, gtD, x2, (T.td >> 30) & 1u);
      cmp_plane(ltD, gtD, x3, (T.td >> 29) & 1u);
    }
    if (!T.tda_full) {
      cmp_plane(ltA, gtA, x1, (T.tda >> 31) & 1u);
      cmp_plane(ltA, gtA, x2, (T.tda >> 30) & 1u);
      cmp_plane(ltA, gtA, x3, (T.tda >> 29) & 1u);
    }
  }
#pragma unroll
  for (int b = 1; b <= 8; ++b) {
    const int m_prev = 33 - 4 * b;  // lowest plane consumed so far
    if (!cmp_open(ltD, gtD, T.td, T.td_full, m_prev) &&
        !cmp_open(ltA, gtA, T.tda, T.tda_full, m_prev))
      break;
    uint32_t x0 = k, x1 = n, x2 = g, x3 = (kTagDyn << 28) | (uint32_t)b;
    philox4x32_10(x0, x1, x2, x3, k0, k1);
    const int m0 = 32 - 4 * b;  // plane of x0
    if (!T.td_full) {
      cmp_plane(ltD, gtD, x0, (T.td >> m0) & 1u);
      if (b < 8) {
        cmp_plane(ltD, gtD, x1, (T.td >> (m0 - 1)) & 1u);
        cmp_plane(ltD, gtD, x2, (T.td >> (m0 - 2)) & 1u);
        cmp_plane(ltD, gtD, x3, (T.td >> (m0 - 3)) & 1u);
      }
    }
    if (!T.tda_full) {
      cmp_plane(ltA, gtA, x0, (T.tda >> m0) & 1u);
      if (b < 8) {
        cmp_plane(ltA, gtA, x1, (T.tda >> (m0 - 1)) & 1u);
        cmp_plane(ltA, gtA, x2, (T.tda >> (m0 - 2)) & 1u);
        cmp_plane(ltA, gtA, x3, (T.tda >> (m0 - 3)) & 1u);
      }
    }
  }
  Masks r;
  r.D = ltD;
  r.A = ltA & ~ltD;
  r.O = O;
  return r;
}

// One window (a, b, c) for 32 samples (Alg. 1's tree on the bond the orientation picks,
// written as bit logic like Alg. 2).  Lane with o=0: bond (a,b), fission target c; o=1: bond
// (b,c), target a.  D: swap the bond; A: clear an occupied bond; otherwise (F) fill the
// target next to an occupied bond.
__device__ __forceinline__ void window_update(uint32_t &a, uint32_t &b, uint32_t &c,
                                              const Masks &m) {
  const uint32_t q = (m.O & c) | (~m.O & a);   // partner of b
  const uint32_t t = (m.O & a) | (~m.O & c);   // fission target
  const uint32_t F = ~(m.D | m.A);
  const uint32_t nb = (m.D & q) | (~m.D & b & ~(m.A & q));
  const uint32_t nq = (m.D & b) | (~m.D & q & ~(m.A & b));
  const uint32_t nt = t | (F & b & q);
  a = (m.O & nt) | (~m.O & nq);
  c = (m.O & nq) | (~m.O & nt);
  b = nb;
}

// Random phase of sub-step n for phase group h: floor(x0 * L / 2^32).
__device__ __forceinline__ uint32_t phase_of(uint32_t n, uint32_t h, uint32_t L, uint32_t k0,
                                             uint32_t k1) {
  uint32_t x0 = 0u, x1 = n, x2 = h, x3 = kTagPhase << 28;
  philox4x32_10(x0, x1, x2, x3, k0, k1);
  return (uint32_t)(((uint64_t)x0 * L) >> 32);
}

// ---------------------------------------------------------------------------------------
// Tile sweep.  One CTA owns a tile of one 32-sample group's column in shared memory:
//  RING: the whole column (tile = L sites, periodic indexing);
//  SEGMENT: core sites [s0, s0+core) plus a halo of H sites on each side (temporal
//  blocking): the windows of each sub-step are computed wherever all three sites are still
//  valid, and the valid region shrinks by at most 2 sites per side per sub-step, so after
//  tau <= H/2 sub-steps the core is exact.  Windows inside the halo are recomputed
//  redundantly; counter-based random numbers make the recomputation identical.
// ---------------------------------------------------------------------------------------
struct SweepParams {
  const uint32_t *src;          // lattice [G][L] before the sub-steps
  uint32_t *dst;                // lattice [G][L] after (may equal src in RING mode)
  uint32_t L, K, G, S;
  uint32_t core;                // core sites per tile (RING: L)
  uint32_t halo;                // H (RING: 0)
  uint32_t k0, k1;              // Philox key
  Thresholds T;
  uint32_t n_begin, n_end;      // sub-steps [n_begin, n_end)
  const uint32_t *rec_sub;      // records: state after rec_sub[r] sub-steps, in (n_begin, n_end]
  uint32_t n_rec;
  unsigned long long *rec_total;  // [n_rec] += occupied pairs
  uint32_t *rec_sample;           // [n_rec][S] += per-sample counts, or nullptr
};

constexpr int kPhiChunk = 256;

// Count occupied sites of tile words [y0, y1) into record r.
__device__ __forceinline__ void tile_count(const uint32_t *sm, uint32_t y0, uint32_t y1,
                                           const SweepParams &P, uint32_t r, uint32_t g,
                                           unsigned int *s_red) {
  unsigned int local = 0;
  for (uint32_t y = y0 + threadIdx.x; y < y1; y += blockDim.x) local += __popc(sm[y]);
  local = __reduce_add_sync(0xFFFFFFFFu, local);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_red[32], local);
  if (P.rec_sample) {
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
  if (threadIdx.x == 0) atomicAdd(&P.rec_total[r], (unsigned long long)s_red[32]);
  if (P.rec_sample && threadIdx.x < 32)
    atomicAdd(&P.rec_sample[(size_t)r * P.S + 32u * g + threadIdx.x], s_red[threadIdx.x]);
  __syncthreads();
  for (uint32_t t = threadIdx.x; t <= 32u; t += blockDim.x) s_red[t] = 0;
  __syncthreads();
}

template <bool RING>
__global__ void __launch_bounds__(1024, 1) k_sweep_tile(const SweepParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_phi[kPhiChunk];
  __shared__ unsigned int s_red[33];

  const uint32_t g = blockIdx.y;
  const uint32_t L = P.L, K = P.K;
  const uint32_t s0 = RING ? 0u : blockIdx.x * P.core;
  const uint32_t core_len = RING ? L : min(P.core, L - s0);
  const uint32_t H = RING ? 0u : P.halo;
  const uint32_t tile_len = core_len + 2u * H;
  const uint32_t base = RING ? 0u : (uint32_t)(((uint64_t)s0 + L - H) % L);
  const uint32_t h = (32u * g) / 128u;

  const uint32_t *src = P.src + (size_t)g * L;
  for (uint32_t y = threadIdx.x; y < tile_len; y += blockDim.x) {
    uint32_t x = base + y;
    if (x >= L) x -= L;
    smem[y] = src[x];
  }
  for (uint32_t t = threadIdx.x; t <= 32u; t += blockDim.x) s_red[t] = 0;
  __syncthreads();

  uint32_t lo = 0, hi = tile_len;   // valid region of the tile (SEGMENT mode)
  uint32_t r = 0;                   // next record
  for (uint32_t n = P.n_begin; n < P.n_end; ++n) {
    const uint32_t j = (n - P.n_begin) % kPhiChunk;
    if (j == 0) {
      for (uint32_t t = threadIdx.x; t < kPhiChunk; t += blockDim.x)
        s_phi[t] = phase_of(n + t, h, L, P.k0, P.k1);
      __syncthreads();
    }
    const uint32_t phi = s_phi[j];
    if (RING) {
      for (uint32_t k = threadIdx.x; k < K; k += blockDim.x) {
        uint32_t ia = phi + 3u * k;
        if (ia >= L) ia -= L;
        uint32_t ib = ia + 1u;
        if (ib >= L) ib -= L;
        uint32_t ic = ib + 1u;
        if (ic >= L) ic -= L;
        uint32_t a = smem[ia], b = smem[ib], c = smem[ic];
        const Masks m = rate_masks(k, n, g, P.k0, P.k1, P.T);
        window_update(a, b, c, m);
        smem[ia] = a;
        smem[ib] = b;
        smem[ic] = c;
      }
    } else {
      // window coordinate of tile position y: w(y) = (base + y - phi) mod L; a window starts
      // at every w = 3k < 3K.  Candidates: from the window holding position lo onwards.
      const uint32_t w_lo = (uint32_t)(((uint64_t)base + lo + L - phi) % L);
      const uint32_t k_lo = (w_lo < 3u * K) ? w_lo / 3u : 0u;
      const uint32_t n_cand = (hi - lo) / 3u + 2u;
      for (uint32_t i = threadIdx.x; i < n_cand; i += blockDim.x) {
        uint32_t k = k_lo + i;
        if (k >= K) k -= K;
        const uint32_t y = (uint32_t)(((uint64_t)phi + 3ull * k + 2ull * L - base) % L);
        if (y < lo || y + 2u >= hi) continue;
        uint32_t a = smem[y], b = smem[y + 1u], c = smem[y + 2u];
        const Masks m = rate_masks(k, n, g, P.k0, P.k1, P.T);
        window_update(a, b, c, m);
        smem[y] = a;
        smem[y + 1u] = b;
        smem[y + 2u] = c;
      }
      // shrink the valid region by the windows that straddle its edges
      if (w_lo < 3u * K && (w_lo % 3u) != 0u) lo += 3u - (w_lo % 3u);
      const uint32_t w_hi = (uint32_t)(((uint64_t)base + hi - 1u + L - phi) % L);
      if (w_hi < 3u * K && (w_hi % 3u) != 2u) hi -= 1u + (w_hi % 3u);
    }
    __syncthreads();
    if (r < P.n_rec && P.rec_sub[r] == n + 1u) {
      tile_count(smem, H, H + core_len, P, r, g, s_red);
      ++r;
    }
  }

  uint32_t *dst = P.dst + (size_t)g * L;
  for (uint32_t i = threadIdx.x; i < core_len; i += blockDim.x) dst[s0 + i] = smem[H + i];
}

// Initial lattice: mode 0 full, 1 empty, 2 i.i.d. Bernoulli(1/2) bits (Philox tag INIT,
// counter (i, 0, g, INIT<<28), first word).
__global__ void k_init(uint32_t *lat, uint32_t L, uint32_t G, int mode, uint32_t k0, uint32_t k1) {
  const size_t total = (size_t)G * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    uint32_t v;
    if (mode == 0) v = 0xFFFFFFFFu;
    else if (mode == 1) v = 0u;
    else {
      const uint32_t g = (uint32_t)(idx / L), i = (uint32_t)(idx % L);
      uint32_t x0 = i, x1 = 0u, x2 = g, x3 = kTagInit << 28;
      philox4x32_10(x0, x1, x2, x3, k0, k1);
      v = x0;
    }
    lat[idx] = v;
  }
}

// Record of the current state (no sub-step): one CTA per group.
__global__ void k_count(const uint32_t *lat, uint32_t L, uint32_t S,
                        unsigned long long *rec_total, uint32_t *rec_sample) {
  const uint32_t g = blockIdx.x;
  const uint32_t *col = lat + (size_t)g * L;
  unsigned int local = 0;
  unsigned int cnt[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) cnt[j] = 0;
  for (uint32_t i = threadIdx.x; i < L; i += blockDim.x) {
    const uint32_t w = col[i];
    local += __popc(w);
    if (rec_sample) {
#pragma unroll
      for (int j = 0; j < 32; ++j) cnt[j] += (w >> j) & 1u;
    }
  }
  local = __reduce_add_sync(0xFFFFFFFFu, local);
  if ((threadIdx.x & 31) == 0) atomicAdd(rec_total, (unsigned long long)local);
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

// Test entry: the MSB-first plane compare on explicit words (O, P31..P0) per item.
__global__ void k_rate_masks(const uint32_t *words, Thresholds T, uint32_t *masks, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t *w = words + 33 * i;
    uint32_t ltD = T.td_full ? 0xFFFFFFFFu : 0u, gtD = (!T.td_full && T.td == 0u) ? 0xFFFFFFFFu : 0u;
    uint32_t ltA = T.tda_full ? 0xFFFFFFFFu : 0u, gtA = (!T.tda_full && T.tda == 0u) ? 0xFFFFFFFFu : 0u;
    // same block structure and exit rule as rate_masks, with the words read from memory
    for (int b = 0; b <= 8; ++b) {
      if (b > 0) {
        const int m_prev = 33 - 4 * b;
        if (!cmp_open(ltD, gtD, T.td, T.td_full, m_prev) &&
            !cmp_open(ltA, gtA, T.tda, T.tda_full, m_prev))
          break;
      }
      const int first = (b == 0) ? 31 : 32 - 4 * b;
      const int cnt = (b == 0) ? 3 : (b < 8 ? 4 : 1);
      for (int q = 0; q < cnt; ++q) {
        const int m = first - q;
        const uint32_t plane = w[32 - m];
        if (!T.td_full) cmp_plane(ltD, gtD, plane, (T.td >> m) & 1u);
        if (!T.tda_full) cmp_plane(ltA, gtA, plane, (T.tda >> m) & 1u);
      }
    }
    masks[3 * i] = ltD;
    masks[3 * i + 1] = ltA & ~ltD;
    masks[3 * i + 2] = w[0];
  }
}

}  // namespace pcpdk
