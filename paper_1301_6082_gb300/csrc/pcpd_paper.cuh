// pcpd_paper.cuh -- the paper's own GPU scheme (Sec. 3-4, Alg. 2), kept as a variant of
// the sweep beside the window schedule of pcpd_kernels.cuh.
//
// One system per group of S_w threads (the paper's workgroup of S_w workitems, Sec. 3): a
// ring of L = 32 * n_loc * S_w sites whose 32 bits per word are 32 far-apart segments of the
// same lattice ("connected lattices", Sec. 4): bit b of thread w's local word l is site
//     s = b * (L/32) + w * n_loc + l.
// Every step draws one local site l* for the whole system, and every thread updates the bond
// (s, s+1) at l* for all 32 bits at once, with fission to s-1 or s+2.  The sites a thread
// touches lie in its own column except at the column ends, where they belong to the next or
// previous thread's column; past the system's last (first) column they are the next (previous)
// bit of column 0 (S_w - 1), which is a one-bit rotation of that word.
//
// Each RNG() of Alg. 2 returns the next word of the thread's own random stream.  A step
// takes n_w = m + n_dec + 2 words, in this order: m diffusion planes (a bit diffuses iff its
// m-bit value, most significant plane first, is below T_d = d * 2^m: the dyadic masks of
// Sec. 4.2), n_dec decorrelation words ANDed together (Sec. 4.3), one word compared with
// T_c = floor(p * 2^n_dec * 2^32) whose outcome is broadcast to all 32 bits (the correlated
// annihilation draw of Sec. 4.3), and one fission-direction word (bit 1: to s+2).  Word k of
// the stream of thread w in system sys is word k mod 4 of the Philox4x32-10 block counted by
// (w, B mod 2^32, sys, TAG_PAPER<<28 | B>>32), B = floor(k/4); step t takes words n_w*t ..
// n_w*t + n_w - 1, so four consecutive steps starting at a multiple of 4 use exactly n_w
// whole blocks.  The local site of step t is floor(x * n_loc / 2^32), x = word t mod 4 of the
// block (0, floor(t/4), sys, TAG_PAPER_SITE<<28).
//
// GB300 layout: the system's n_loc * S_w words stay in shared memory for the whole launch,
// word (l, w) at l * S_w + w, so a step's four loads and stores per thread are consecutive
// across the warp (bank-conflict free, the shared-memory analogue of the paper's coalesced
// 4*S_w-byte rows).  A thread touches another thread's column only in a step whose local
// site is within one word of a column end (l* = 0, n_loc-2 or n_loc-1); the S_w threads of a
// system meet just before and just after such a step and nowhere else (one warp: __syncwarp;
// a system of several warps has its CTA to itself and uses the CTA barrier, or, in CTAs of
// more than 256 threads, a named barrier per system), so most steps run without a barrier.
#pragma once
#include "pcpd_kernels.cuh"

namespace pcpdk {

constexpr uint32_t kTagPaper = 4u;
constexpr uint32_t kTagPaperSite = 5u;

struct PaperParams {
  uint32_t *lat;                          // [systems][n_loc][S_w] words (device)
  const unsigned long long *rec_step;     // this launch's record steps, strictly increasing
  unsigned long long *rec_total;          // [n_rec]: occupied sites summed over systems
  uint32_t *rec_sys;                      // [n_rec][systems] or null
  RoundKeys rk;                           // Philox round keys of the seed
  uint32_t n_loc, S_w, systems, spc;      // spc: systems per CTA
  uint32_t m, t_d, d_full, n_dec;         // d_full: T_d == 2^m (every bit diffuses)
  uint32_t tc, tc_full;                   // T_c < 2^32, or tc_full: the draw always passes
  uint32_t step_begin, step_end;          // steps [step_begin, step_end) of this launch
  uint32_t n_rec;
  uint32_t systems_total;                 // row length of rec_sys
};

// The S_w threads of one system meet.  One warp: __syncwarp.  NAMED = false: the CTA holds a
// single system (or systems of one warp each) and uses the CTA barrier; NAMED = true: several
// multi-warp systems share the CTA and each uses named barrier 1 + its slot.  A named barrier
// with a run-time id reserves all 16 of the CTA's hardware barriers (4 CTAs per SM at most),
// so only the kernels that need it have one.
template <bool NAMED>
__device__ __forceinline__ void paper_barrier(uint32_t id, uint32_t nthreads) {
  if (nthreads == 32u)
    __syncwarp();
  else if (!NAMED)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint32_t pick4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t i) {
  return i == 0u ? c0 : i == 1u ? c1 : i == 2u ? c2 : c3;
}

// Occupied sites of the thread's column, summed over the system, added to record slot r.
__device__ __forceinline__ void paper_record(const PaperParams &P, const uint32_t *lat,
                                             uint32_t w, uint32_t sys, uint32_t r) {
  uint32_t c = 0u;
  for (uint32_t l = 0; l < P.n_loc; ++l) c += __popc(lat[l * P.S_w + w]);
  c = __reduce_add_sync(~0u, c);
  if ((threadIdx.x & 31u) == 0u) {
    atomicAdd(P.rec_total + r, (unsigned long long)c);
    if (P.rec_sys) atomicAdd(P.rec_sys + (size_t)r * P.systems_total + sys, c);
  }
}

// Alg. 2 on one bond as bit logic, in the thread's frame (bit b of every value is a site of
// bit b's segment): swap (b0, b1) under D; else an occupied pair annihilates under A, else
// puts a particle on c2 = s+2 (F = 1) or on a = s-1 (F = 0).
__device__ __forceinline__ void paper_bond(uint32_t &a, uint32_t &b0, uint32_t &b1,
                                           uint32_t &c2, uint32_t D, uint32_t A, uint32_t F) {
  const uint32_t pair = b0 & b1;
  const uint32_t n0 = (D & b1) | (~D & b0);
  const uint32_t n1 = (D & b0) | (~D & b1);
  const uint32_t react = ~D & pair;
  const uint32_t ann = react & A;
  const uint32_t fis = react & ~ann;
  b0 = n0 & ~ann;
  b1 = n1 & ~ann;
  c2 |= fis & F;
  a |= fis & ~F;
}

// A step whose four sites reach into a neighbouring column (l* = 0, n_loc-2 or n_loc-1):
// word indexes with the wrap to the next/previous thread and the bit rotation at the seam.
__device__ __forceinline__ void paper_step_cross(uint32_t *lat, uint32_t n_loc, uint32_t S_w,
                                                 uint32_t w, uint32_t w_lo, uint32_t rot_lo,
                                                 uint32_t w_hi, uint32_t rot_hi, uint32_t ls,
                                                 uint32_t D, uint32_t A, uint32_t F) {
  const uint32_t i_a = (ls == 0u) ? (n_loc - 1u) * S_w + w_lo : (ls - 1u) * S_w + w;
  const uint32_t r_a = (ls == 0u) ? rot_lo : 0u;
  const uint32_t i_0 = ls * S_w + w;
  const uint32_t i_1 = (ls + 1u < n_loc) ? (ls + 1u) * S_w + w : w_hi;
  const uint32_t r_1 = (ls + 1u < n_loc) ? 0u : rot_hi;
  const uint32_t i_2 = (ls + 2u < n_loc) ? (ls + 2u) * S_w + w : (ls + 2u - n_loc) * S_w + w_hi;
  const uint32_t r_2 = (ls + 2u < n_loc) ? 0u : rot_hi;
  const uint32_t words = n_loc * S_w;
  if (!PCPD_IN_BOUNDS(i_a, words, kDbgPaper) || !PCPD_IN_BOUNDS(i_0, words, kDbgPaper) ||
      !PCPD_IN_BOUNDS(i_1, words, kDbgPaper) || !PCPD_IN_BOUNDS(i_2, words, kDbgPaper))
    return;
  (void)words;
  uint32_t a = __funnelshift_l(lat[i_a], lat[i_a], r_a);
  uint32_t b0 = lat[i_0];
  uint32_t b1 = __funnelshift_r(lat[i_1], lat[i_1], r_1);
  uint32_t c2 = __funnelshift_r(lat[i_2], lat[i_2], r_2);
  paper_bond(a, b0, b1, c2, D, A, F);
  lat[i_a] = __funnelshift_r(a, a, r_a);
  lat[i_0] = b0;
  lat[i_1] = __funnelshift_l(b1, b1, r_1);
  lat[i_2] = __funnelshift_l(c2, c2, r_2);
}

template <bool B>
struct PaperEdge {
  static constexpr bool value = B;
};

// M, ND >= 0: plane and decorrelation counts fixed at compile time (every word position in
// a 4-step group is then a constant); M < 0: read from P.  MAXT: largest CTA the kernel
// serves; CTAs of up to 256 threads get a register budget that keeps 6 of them per SM.
// NAMED: per-system named barriers (see paper_barrier).
template <int M, int ND, int MAXT, bool NAMED>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 6 : 1) k_paper_sweep(const PaperParams P) {
  extern __shared__ uint32_t s_lat[];
  const uint32_t S_w = P.S_w, n_loc = P.n_loc;
  const uint32_t slot = threadIdx.x / S_w, w = threadIdx.x - slot * S_w;
  const uint32_t sys = blockIdx.x * P.spc + slot;
  if (sys >= P.systems) return;  // S_w is a multiple of 32: whole warps of an absent system
  const uint32_t bar = 1u + slot;
  const uint32_t words = n_loc * S_w;
  uint32_t *lat = s_lat + (size_t)slot * words;
  uint32_t *glat = P.lat + (size_t)sys * words;
  // thread w loads, updates (outside the barrier-guarded steps) and stores only column w
  for (uint32_t i = w; i < words; i += S_w) lat[i] = __ldcg(glat + i);

  const uint32_t m = M >= 0 ? (uint32_t)M : P.m;
  const uint32_t nd = M >= 0 ? (uint32_t)ND : P.n_dec;
  const uint32_t nw = m + nd + 2u;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t w_lo = (w == 0u) ? S_w - 1u : w - 1u, rot_lo = (w == 0u) ? 1u : 0u;
  const uint32_t w_hi = (w == S_w - 1u) ? 0u : w + 1u, rot_hi = (w == S_w - 1u) ? 1u : 0u;
  const uint32_t begin = P.step_begin, end = P.step_end;
  // record slots: r, and the step of the next one (steps inside the loop are < 2^32 - 1)
  uint32_t r = 0u;
  uint32_t next_rec = P.n_rec ? (uint32_t)P.rec_step[0] : 0xFFFFFFFFu;
  uint32_t s0 = 0u, s1 = 0u, s2 = 0u, s3 = 0u;  // local-site words of this lane's group
  uint32_t q0 = begin >> 2;

  // The thread's stream blocks differ only in B: x0 = w, x2 = sys are fixed, and x3 = tag|B>>32
  // changes once per 2^32 blocks.  What depends on (w, sys, B>>32) alone is computed once:
  // then a block needs 16 of its 20 multiplies (rounds 1-3 share most of their products).
  const uint32_t A0 = __umulhi(sys, kPhiloxM1) ^ P.rk.k0[0];   // round-1 x0 = A0 ^ (uint32_t)B
  const uint32_t E = (w * kPhiloxM0) ^ P.rk.k1[1];             // round-2 x2 = hi(M0 x0) ^ E
  uint32_t C2 = 0u, C3h = 0u, C3l = 0u, hb_cached = 0u;
  auto prefix = [&](uint32_t hb) {
    const uint32_t x2p = __umulhi(w, kPhiloxM0) ^ P.rk.k1[0] ^ ((kTagPaper << 28) | hb);
    const uint32_t C1 = __umulhi(x2p, kPhiloxM1) ^ (sys * kPhiloxM1) ^ P.rk.k0[1];   // round-2 x0
    C2 = x2p * kPhiloxM1;                                                           // round-2 x1
    C3h = __umulhi(C1, kPhiloxM0) ^ P.rk.k1[2];
    C3l = C1 * kPhiloxM0;                                                           // round-3 x3
    hb_cached = hb;
  };
  prefix(0u);

  // one group of 4 steps (4q .. 4q+3); EDGE: the group may extend past [begin, end);
  // HASREC: a record step may fall inside (else the group has no branch and the compiler can
  // interleave its four steps)
  auto group = [&](uint32_t q, auto edge, auto hasrec) {
    constexpr bool EDGE = decltype(edge)::value;
    constexpr bool HASREC = decltype(hasrec)::value;
    constexpr bool FAST = !EDGE;   // blocks from the shared prefix (one value of B>>32)
    const uint32_t qi = (q - q0) & 31u;
    if (qi == 0u) {
      // lane i draws the local sites of the 4 steps of group q + i
      uint32_t x0 = 0u, x1 = q + lane, x2 = sys, x3 = kTagPaperSite << 28;
      philox4x32_10_rk(x0, x1, x2, x3, P.rk);
      s0 = x0, s1 = x1, s2 = x2, s3 = x3;
    }
    const unsigned long long B0 = (unsigned long long)q * nw;  // first block of the group
    uint32_t c0 = 0u, c1 = 0u, c2 = 0u, c3 = 0u;
#pragma unroll
    for (uint32_t j = 0; j < 4u; ++j) {
      const uint32_t st = 4u * q + j;
      uint32_t lt = 0u, eq = ~0u, dec = ~0u, corr = 0u, fis = 0u;
#pragma unroll
      for (uint32_t i = 0; i < nw; ++i) {
        const uint32_t k = j * nw + i;
        if ((k & 3u) == 0u) {
          const unsigned long long B = B0 + (k >> 2);
          if (FAST) {
            const uint32_t x0p = A0 ^ (uint32_t)B;
            const uint32_t x2pp = __umulhi(x0p, kPhiloxM0) ^ E;
            const uint32_t x3pp = x0p * kPhiloxM0;
            uint32_t x0 = __umulhi(x2pp, kPhiloxM1) ^ C2 ^ P.rk.k0[2];
            uint32_t x1 = x2pp * kPhiloxM1;
            uint32_t x2 = C3h ^ x3pp;
            uint32_t x3 = C3l;
#pragma unroll
            for (int rr = 3; rr < 10; ++rr) {
              const uint32_t h0 = __umulhi(x0, kPhiloxM0), l0 = x0 * kPhiloxM0;
              const uint32_t h1 = __umulhi(x2, kPhiloxM1), l1 = x2 * kPhiloxM1;
              x0 = h1 ^ x1 ^ P.rk.k0[rr];
              x1 = l1;
              x2 = h0 ^ x3 ^ P.rk.k1[rr];
              x3 = l0;
            }
            c0 = x0, c1 = x1, c2 = x2, c3 = x3;
          } else {
            uint32_t x0 = w, x1 = (uint32_t)B, x2 = sys, x3 = (kTagPaper << 28) | (uint32_t)(B >> 32);
            philox4x32_10_rk(x0, x1, x2, x3, P.rk);
            c0 = x0, c1 = x1, c2 = x2, c3 = x3;
          }
        }
        const uint32_t u = pick4(c0, c1, c2, c3, k & 3u);
        if ((int)i < (int)m) {
          // plane i carries bit (m-1-i) of each lane's draw; compare with T_d, MSB first
          const uint32_t tb = 0u - ((P.t_d >> (m - 1u - i)) & 1u);
          lt |= eq & ~u & tb;
          eq &= ~(u ^ tb);
        } else if ((int)i < (int)(m + nd)) {
          dec &= u;
        } else if (i == m + nd) {
          corr = (P.tc_full || u < P.tc) ? ~0u : 0u;
        } else {
          fis = u;
        }
      }
      if (EDGE && (st < begin || st >= end)) continue;
      if (HASREC && st == next_rec) {
        paper_record(P, lat, w, sys, r);
        ++r;
        next_rec = r < P.n_rec ? (uint32_t)P.rec_step[r] : 0xFFFFFFFFu;
      }
      const uint32_t x = __shfl_sync(~0u, pick4(s0, s1, s2, s3, j), qi);
      const uint32_t ls = (uint32_t)(((unsigned long long)x * n_loc) >> 32);
      const uint32_t D = P.d_full ? ~0u : lt, A = dec & corr;
      if (!PCPD_IN_BOUNDS(ls, n_loc, kDbgPaper)) continue;
      if (ls != 0u && ls + 2u < n_loc) {
        // the common case: all four sites in the thread's own column, no rotation
        uint32_t *p = lat + ls * S_w + w;
        uint32_t a = p[0u - S_w], b0 = p[0], b1 = p[S_w], cc = p[2u * S_w];
        paper_bond(a, b0, b1, cc, D, A, fis);
        p[0u - S_w] = a;
        p[0] = b0;
        p[S_w] = b1;
        p[2u * S_w] = cc;
      } else {
        paper_barrier<NAMED>(bar, S_w);
        paper_step_cross(lat, n_loc, S_w, w, w_lo, rot_lo, w_hi, rot_hi, ls, D, A, fis);
        paper_barrier<NAMED>(bar, S_w);
      }
    }
  };

  if (begin < end) {
    const uint32_t q1 = (end - 1u) >> 2;
    const bool head = (begin & 3u) != 0u || q0 == q1;
    uint32_t q = q0;
    if (head) group(q++, PaperEdge<true>{}, PaperEdge<true>{});
    const uint32_t q_full_end = ((end & 3u) == 0u) ? q1 + 1u : q1;  // groups entirely inside
    for (; q < q_full_end; ++q) {
      const unsigned long long B0 = (unsigned long long)q * nw;
      const uint32_t hb = (uint32_t)(B0 >> 32);
      if (hb != (uint32_t)((B0 + nw - 1u) >> 32)) {   // B>>32 changes inside the group
        group(q, PaperEdge<true>{}, PaperEdge<true>{});
        continue;
      }
      if (hb != hb_cached) prefix(hb);
      if ((next_rec >> 2) == q) group(q, PaperEdge<false>{}, PaperEdge<true>{});
      else group(q, PaperEdge<false>{}, PaperEdge<false>{});
    }
    if (q <= q1) group(q, PaperEdge<true>{}, PaperEdge<true>{});
  }
  if (r < P.n_rec && P.rec_step[r] == (unsigned long long)end) paper_record(P, lat, w, sys, r);
  for (uint32_t i = w; i < words; i += S_w) __stcg(glat + i, lat[i]);
}

}  // namespace pcpdk
