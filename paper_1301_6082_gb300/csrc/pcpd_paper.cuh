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
// Random words per thread and step, in stream order: m diffusion planes (a bit diffuses iff
// its m-bit value, most significant plane first, is below T_d = d * 2^m: the dyadic masks of
// Sec. 4.2), n_dec decorrelation words ANDed together (Sec. 4.3), one word compared with
// T_c = floor(p * 2^n_dec * 2^32) whose outcome is broadcast to all 32 bits (the correlated
// annihilation draw of Sec. 4.3), and one fission-direction word (bit 1: to s+2).  They are
// Philox4x32-10 blocks j = 0, 1, ... of the counter (w, step, system, TAG_PAPER<<28 | j);
// the local site is floor(x0 * n_loc / 2^32) of (0, step, system, TAG_PAPER_SITE<<28).
//
// GB300 layout: the system's n_loc * S_w words stay in shared memory for the whole launch,
// word (l, w) at l * S_w + w, so a step's four loads and stores per thread are consecutive
// across the warp (bank-conflict free, the shared-memory analogue of the paper's coalesced
// 4*S_w-byte rows).  Between steps the S_w threads of a system meet at a named barrier (one
// warp: __syncwarp), so systems in one CTA run independently.
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

// The S_w threads of one system meet (id: 1 + the system's slot in the CTA).
__device__ __forceinline__ void paper_barrier(uint32_t id, uint32_t nthreads) {
  if (nthreads == 32u)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Per-thread masks of one step: D (diffuse), A (annihilate if the bond is an occupied pair and
// D is clear: decorrelation AND broadcast draw), F (fission direction, 1 = high).
// M, ND >= 0: plane and decorrelation counts fixed at compile time; M < 0: read from P.
template <int M, int ND>
__device__ __forceinline__ void paper_masks(const PaperParams &P, uint32_t w, uint32_t st,
                                            uint32_t sys, uint32_t &D, uint32_t &A,
                                            uint32_t &F) {
  const uint32_t m = M >= 0 ? (uint32_t)M : P.m;
  const uint32_t nd = M >= 0 ? (uint32_t)ND : P.n_dec;
  const uint32_t nw = m + nd + 2u;
  uint32_t lt = 0u, eq = ~0u, dec = ~0u, corr = 0u, fis = 0u;
#pragma unroll
  for (uint32_t j = 0; 4u * j < nw; ++j) {
    uint32_t x0 = w, x1 = st, x2 = sys, x3 = (kTagPaper << 28) | j;
    philox4x32_10_rk(x0, x1, x2, x3, P.rk);
    const uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
    for (uint32_t q = 0; q < 4u; ++q) {
      const int k = (int)(4u * j + q), im = (int)m, ind = (int)nd;
      const uint32_t u = xs[q];
      if (k < im) {
        // plane k carries bit (m-1-k) of each lane's draw; compare with T_d, MSB first
        const uint32_t tb = 0u - ((P.t_d >> (im - 1 - k)) & 1u);
        lt |= eq & ~u & tb;
        eq &= ~(u ^ tb);
      } else if (k < im + ind) {
        dec &= u;
      } else if (k == im + ind) {
        corr = (P.tc_full || u < P.tc) ? ~0u : 0u;
      } else if (k == im + ind + 1) {
        fis = u;
      }
    }
  }
  D = P.d_full ? ~0u : lt;
  A = dec & corr;
  F = fis;
}

template <int M, int ND>
__global__ void __launch_bounds__(1024) k_paper_sweep(const PaperParams P) {
  extern __shared__ uint32_t s_lat[];
  const uint32_t S_w = P.S_w, n_loc = P.n_loc;
  const uint32_t slot = threadIdx.x / S_w, w = threadIdx.x - slot * S_w;
  const uint32_t sys = blockIdx.x * P.spc + slot;
  if (sys >= P.systems) return;  // S_w is a multiple of 32: whole warps of an absent system
  const uint32_t bar = 1u + slot;
  const uint32_t words = n_loc * S_w;
  uint32_t *lat = s_lat + (size_t)slot * words;
  uint32_t *glat = P.lat + (size_t)sys * words;
  for (uint32_t i = w; i < words; i += S_w) lat[i] = __ldcg(glat + i);
  paper_barrier(bar, S_w);

  const uint32_t lane = threadIdx.x & 31u;
  // neighbour columns and the bit rotation at the system's seam
  const uint32_t w_lo = (w == 0u) ? S_w - 1u : w - 1u, rot_lo = (w == 0u) ? 1u : 0u;
  const uint32_t w_hi = (w == S_w - 1u) ? 0u : w + 1u, rot_hi = (w == S_w - 1u) ? 1u : 0u;
  uint32_t site_cache = 0u;
  uint32_t r = 0u;
  for (uint32_t st = P.step_begin;; ++st) {
    if (r < P.n_rec && P.rec_step[r] == (unsigned long long)st) {
      uint32_t c = 0u;
      for (uint32_t l = 0; l < n_loc; ++l) c += __popc(lat[l * S_w + w]);
      c = __reduce_add_sync(~0u, c);
      if (lane == 0u) {
        atomicAdd(P.rec_total + r, (unsigned long long)c);
        if (P.rec_sys) atomicAdd(P.rec_sys + (size_t)r * P.systems_total + sys, c);
      }
      ++r;
      paper_barrier(bar, S_w);  // counting reads neighbour-written words of the next step
    }
    if (st == P.step_end) break;
    const uint32_t q = (st - P.step_begin) & 31u;
    if (q == 0u) {
      // lane i draws the local site of step st + i; the warp reads them one per step
      uint32_t x0 = 0u, x1 = st + lane, x2 = sys, x3 = kTagPaperSite << 28;
      philox4x32_10_rk(x0, x1, x2, x3, P.rk);
      site_cache = (uint32_t)(((unsigned long long)x0 * n_loc) >> 32);
    }
    const uint32_t ls = __shfl_sync(~0u, site_cache, q);

    uint32_t D, A, F;
    paper_masks<M, ND>(P, w, st, sys, D, A, F);

    // word indexes and seam rotations of sites s-1, s, s+1, s+2
    const uint32_t i_a = (ls == 0u) ? (n_loc - 1u) * S_w + w_lo : (ls - 1u) * S_w + w;
    const uint32_t r_a = (ls == 0u) ? rot_lo : 0u;
    const uint32_t i_0 = ls * S_w + w;
    const uint32_t i_1 = (ls + 1u < n_loc) ? (ls + 1u) * S_w + w : w_hi;
    const uint32_t r_1 = (ls + 1u < n_loc) ? 0u : rot_hi;
    const uint32_t i_2 = (ls + 2u < n_loc) ? (ls + 2u) * S_w + w : (ls + 2u - n_loc) * S_w + w_hi;
    const uint32_t r_2 = (ls + 2u < n_loc) ? 0u : rot_hi;
    // in the thread's frame bit b of every value is the site of bit b's segment
    uint32_t a = __funnelshift_l(lat[i_a], lat[i_a], r_a);
    uint32_t b0 = lat[i_0];
    uint32_t b1 = __funnelshift_r(lat[i_1], lat[i_1], r_1);
    uint32_t c2 = __funnelshift_r(lat[i_2], lat[i_2], r_2);

    // Alg. 2 as bit logic: swap under D; else an occupied pair annihilates under A, else
    // fissions to s+2 (F = 1) or s-1 (F = 0).
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

    lat[i_a] = __funnelshift_r(a, a, r_a);
    lat[i_0] = b0;
    lat[i_1] = __funnelshift_l(b1, b1, r_1);
    lat[i_2] = __funnelshift_l(c2, c2, r_2);
    paper_barrier(bar, S_w);
  }
  for (uint32_t i = w; i < words; i += S_w) __stcg(glat + i, lat[i]);
}

}  // namespace pcpdk
