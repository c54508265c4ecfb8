// pcpd_engine.cuh -- persistent work-queue sweep: one launch runs any number of PCPD
// instances (different L, samples, p, d, seeds, step counts) as a stream of tile items.
//
// Item = (instance, epoch e, tile).  A tile is either a group of whole columns (RING: gpi
// 32-sample groups that fit in shared memory, updated with periodic indexing) or one
// segment of one column with a halo of H = (W-1)*tau + W + 1 sites on each side (SEGMENT,
// temporal blocking: windows of W sites shrink the valid region by at most W-1 sites per side
// per sub-step; the extra sites keep the one after the core valid for pair records).  Epoch e
// covers sub-steps [n_begin + e*tau, ... + tau).  W = 3 for the PCPD, n+1 for the n-tuple
// processes (TCPD, QCPD).
// Items are popped in list order from a device counter by persistent CTAs; an item of epoch
// e > 0 first waits (bounded, acquire) until the tiles it reads -- itself and, for segments,
// its two neighbours -- have completed epoch e-1.  Epoch e reads lattice buffer e&1 and
// writes buffer (e+1)&1, so a neighbour still reading epoch e-1's halo is never overwritten.
// Counter-based random numbers (keyed by instance seed, group, sub-step, window) make every
// schedule, batching and tiling give the same bits as a lone run.
#pragma once
#ifndef PCPD_JIT_SOURCE
#include "pcpd_kernels.cuh"
#endif

// Threshold compare of the sweep: generic (thresholds read as kernel constants) or, in a
// build specialised for one (T_D, T_DA) pair (PCPD_JIT_TD / PCPD_JIT_TDA defined, both in
// (0, 2^32)), with the thresholds as compile-time constants.  Same arithmetic, same bits.
#ifdef PCPD_JIT_TD
#define PCPD_CMP_D(c, w, K, m_hi) cmp_group_ct<(uint32_t)(PCPD_JIT_TD), K>(c, w, m_hi)
#define PCPD_CMP_A(c, w, K, m_hi) cmp_group_ct<(uint32_t)(PCPD_JIT_TDA), K>(c, w, m_hi)
#define PCPD_LO_D (__ffs((int)(PCPD_JIT_TD)) - 1u)
#define PCPD_LO_DA (__ffs((int)(PCPD_JIT_TDA)) - 1u)
#else
#define PCPD_CMP_D(c, w, K, m_hi) cmp_group<K>(c, w, D.T.tmD, m_hi)
#define PCPD_CMP_A(c, w, K, m_hi) cmp_group<K>(c, w, D.T.tmA, m_hi)
#define PCPD_LO_D (D.T.lo_d)
#define PCPD_LO_DA (D.T.lo_da)
#endif

namespace pcpdk {

struct InstDesc {
  uint32_t L, K, G, S;
  uint32_t pitch;            // words between consecutive columns in the device buffers
  uint32_t k0, k1;           // Philox key (for the phase draw)
  uint32_t ring, gpi;        // RING tiles hold gpi whole columns (gpi in {1,2,4})
  uint32_t core, halo, tau;  // SEGMENT geometry; tau = sub-steps per epoch (both modes)
  uint32_t n_seg;            // segments per column (1 for RING)
  uint32_t n_begin, n_end;   // sub-steps of this launch
  uint32_t n_rec;            // records in (n_begin, n_end]
  uint32_t W;                // window width: tuple size + 1 (3 PCPD, 4 TCPD, 5 QCPD)
  uint32_t g_base;           // global index of the instance's first group (a multiple of 4)
  uint32_t *buf0, *buf1;     // state at n_begin is in buf0
  const uint32_t *rec_sub;   // [n_rec] sub-step of each record (increasing)
  unsigned long long *rec_total;  // [n_rec]
  uint32_t *rec_sample;      // [n_rec][S] or nullptr
  unsigned long long *rec_pairs;  // [n_rec] occupied nearest-neighbour pairs, or nullptr
  uint32_t *done;            // [tiles per epoch] epochs completed in this launch
  RoundKeys rk;
  Thresholds T;
};
static_assert(sizeof(InstDesc) % 4 == 0, "descriptor is copied as words");

// Batched launches read instance descriptors from this table (constant memory: every
// operand the hot loop takes from a descriptor -- round keys, threshold masks -- is then a
// constant-bank operand).  One batched launch at a time may use it.
constexpr int kMaxBatchInst = 128;
__constant__ InstDesc c_inst[kMaxBatchInst];

struct BatchParams {
  InstDesc single;                  // the instance of a single-instance launch
  const unsigned long long *items;  // packed items (batched); nullptr = single, implicit order
  uint32_t n_items;
  uint32_t tiles_per_epoch;          // implicit order only
  uint32_t *counter;                 // next item, 0 at launch
  uint32_t *err;                     // 0 = ok; sticky error code otherwise
  uint32_t tile_words;               // shared-memory words for tiles (list follows)
  unsigned long long spin_limit;     // clock cycles an item may wait for a dependency
};

// Threads per CTA of the sweep (at most): 16 warps with up to 128 registers each ran the
// L = 65536 tiles 3-8% faster than 32 warps held to 64 registers (same bits).
constexpr uint32_t kSweepThreads = 512;

constexpr uint32_t kErrDepTimeout = 1u;
constexpr uint32_t kErrLoadTimeout = 2u;

__host__ __device__ inline unsigned long long pack_item(uint32_t inst, uint32_t epoch, uint32_t tile) {
  return ((unsigned long long)inst << 48) | ((unsigned long long)(epoch & 0xFFFFFFu) << 24) |
         (unsigned long long)(tile & 0xFFFFFFu);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- TMA bulk copies (global -> shared), completion on an mbarrier ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// A contiguous span of words can go by TMA if both ends are 16-byte aligned.
__device__ __forceinline__ bool tma_ok(const uint32_t *dst, const uint32_t *src, uint32_t words) {
  return words >= 4u && (words & 3u) == 0u && (((uintptr_t)dst | (uintptr_t)src) & 15u) == 0u;
}

// Per-item tile work (the body of the tile sweep, generalised to gpi columns), for windows
// of W sites.
template <bool RING, int W>
__device__ __forceinline__ void run_item(const InstDesc &D, uint32_t *smem, uint32_t *q3,
                                         uint32_t g0, uint32_t sg, uint32_t e, uint32_t *s_phi,
                                         unsigned int *s_red, unsigned int *s_q3n) {
  const uint32_t L = D.L, K = D.K;
  const uint32_t gpi = RING ? D.gpi : 1u;
  const uint32_t s0 = RING ? 0u : sg * D.core;
  const uint32_t core_len = RING ? L : min(D.core, L - s0);
  const uint32_t H = RING ? 0u : D.halo;
  const uint32_t tile_len = core_len + 2u * H;
  const uint32_t win_lim = RING ? L : tile_len;   // a window's sites index its column's region
  const uint32_t base = RING ? 0u : (uint32_t)(((uint64_t)s0 + L - H) % L);
  const uint32_t h = (D.g_base + g0) >> 2;   // one 128-sample phase group for all gpi columns
  const uint32_t n_a = D.n_begin + e * D.tau;   // < n_end < 2^32
  // the epoch's end in 64 bits: n_a + tau may pass 2^32 near the end of the counter range
  const uint32_t n_b = (uint32_t)min((unsigned long long)n_a + D.tau, (unsigned long long)D.n_end);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  // the round keys in registers: a batch descriptor sits at a run-time index of a constant table
  const RoundKeys rk = D.rk;

  // first record after n_a
  uint32_t r = 0;
  {
    uint32_t lo_r = 0, hi_r = D.n_rec;
    while (lo_r < hi_r) {
      const uint32_t mid = (lo_r + hi_r) >> 1;
      if (D.rec_sub[mid] <= n_a) lo_r = mid + 1;
      else hi_r = mid;
    }
    r = lo_r;
  }

  Geometry G;
  G.lo = 0;
  G.hi = tile_len;
  G.gap = L - (uint32_t)W * K;
  const uint32_t n_cand_ring = gpi * K;
  for (uint32_t n = n_a; n < n_b; ++n) {
    const uint32_t j = (n - n_a) % kPhiChunk;
    if (j == 0) {
      for (uint32_t t = threadIdx.x; t < kPhiChunk; t += blockDim.x)
        s_phi[t] = phase_of(n + t, h, L, D.k0, D.k1);
    }
    if (threadIdx.x == 0) *s_q3n = 0;
    __syncthreads();
    G.phi = s_phi[j];
    uint32_t w_lo = 0;
    if (RING) {
      G.n_cand = K;
    } else {
      w_lo = base + G.lo + L - G.phi;
      if (w_lo >= L) w_lo -= L;
      if (w_lo >= L) w_lo -= L;
      if (w_lo < (uint32_t)W * K) {
        G.k_lo = w_lo / (uint32_t)W;
        G.y_first = (int)G.lo - (int)(w_lo - (uint32_t)W * G.k_lo);
      } else {
        G.k_lo = 0u;
        G.y_first = (int)G.lo + (int)(L - w_lo);
      }
      G.n_cand = (G.hi - G.lo) / (uint32_t)W + 2u;
    }
    const uint32_t n_cand = RING ? n_cand_ring : G.n_cand;

    // ---- first pass: blocks 0-2 for every window; undecided windows are deferred ----
    // SEGMENT tiles advance each thread's window index and first site incrementally (the index
    // wraps from K-1 to 0 at most once per sub-step, adding the idle gap to the site) and test
    // the site range with one unsigned compare; candidates past n_cand land beyond the range
    const uint32_t stride = blockDim.x;
    uint32_t seg_k = G.k_lo + warp * 32u + lane;
    int seg_y = G.y_first + W * (int)(warp * 32u + lane);
    if (!RING && seg_k >= K) {
      seg_k -= K;
      seg_y += (int)G.gap;
    }
    const uint32_t span = G.hi - G.lo - (uint32_t)(W - 1);   // first sites [lo, hi - W + 1)
    for (uint32_t i0 = warp * 32u; i0 < n_cand; i0 += stride) {
      const uint32_t i = i0 + lane;
      uint32_t col = 0, ii = i;
      if (RING) {
        col = (uint32_t)(i >= K) + (uint32_t)(i >= 2u * K) + (uint32_t)(i >= 3u * K);
        ii = i - col * K;
      }
      uint32_t k = 0, idx[W] = {};
      bool valid;
      if (RING) {
        valid = i < n_cand && candidate<RING, W>(G, ii, L, K, k, idx);
      } else {
        k = seg_k;
        valid = (uint32_t)(seg_y - (int)G.lo) < span;
#pragma unroll
        for (int j2 = 0; j2 < W; ++j2) idx[j2] = (uint32_t)(seg_y + j2);
        seg_k += stride;
        seg_y += W * (int)stride;
        if (seg_k >= K) {
          seg_k -= K;
          seg_y += (int)G.gap;
        }
      }
      uint32_t *sm = smem + col * L;
      const uint32_t g = D.g_base + g0 + col;   // the group's index in the Philox counter
      Cmp cD = cmp_init(D.T.td, D.T.td_full), cA = cmp_init(D.T.tda, D.T.tda_full);
      uint32_t O;
      {
        // the window index enters through a counter word that round 1 XORs rather than
        // multiplies: the products that depend on (n, g) alone stay out of the window loop
        uint32_t x0 = n, x1 = k, x2 = g, x3 = kTagDyn << 28;
        uint32_t y0 = n, y1 = k, y2 = g, y3 = (kTagDyn << 28) | 1u;
        uint32_t z0 = n, z1 = k, z2 = g, z3 = (kTagDyn << 28) | 2u;
        philox4x32_10_rk(x0, x1, x2, x3, rk);
        philox4x32_10_rk(y0, y1, y2, y3, rk);
        philox4x32_10_rk(z0, z1, z2, z3, rk);
        O = x0;
        const uint32_t w[11] = {x1, x2, x3, y0, y1, y2, y3, z0, z1, z2, z3};   // planes 31..21
        PCPD_CMP_D(cD, w, 11, 31);
        PCPD_CMP_A(cA, w, 11, 31);
      }
      const bool open = cmp_open2(cD, PCPD_LO_D, 21) || cmp_open2(cA, PCPD_LO_DA, 21);
      if (valid && !open) apply_window<W>(sm, idx, O, cD.lt, cA.lt, win_lim);
      if (valid && open) {
        const uint32_t p3 = atomicAdd(s_q3n, 1u);
        if (p3 < (uint32_t)kQ3Cap) {
          q3[0 * kQ3Cap + p3] = i;
          q3[1 * kQ3Cap + p3] = O;
          q3[2 * kQ3Cap + p3] = cD.lt;
          q3[3 * kQ3Cap + p3] = cD.eq;
          q3[4 * kQ3Cap + p3] = cA.lt;
          q3[5 * kQ3Cap + p3] = cA.eq;
        } else {  // list full: finish here
          finish_from3(k, n, g, rk, D.T, cD, cA);
          apply_window<W>(sm, idx, O, cD.lt, cA.lt, win_lim);
        }
      }
    }
    __syncthreads();
    // ---- second pass: blocks 3..8 for the few windows still open ----
    const uint32_t nq3 = min(*s_q3n, (uint32_t)kQ3Cap);
    for (uint32_t t = threadIdx.x; t < nq3; t += blockDim.x) {
      const uint32_t i = q3[0 * kQ3Cap + t];
      const uint32_t O = q3[1 * kQ3Cap + t];
      Cmp cD, cA;
      cD.lt = q3[2 * kQ3Cap + t];
      cD.eq = q3[3 * kQ3Cap + t];
      cA.lt = q3[4 * kQ3Cap + t];
      cA.eq = q3[5 * kQ3Cap + t];
      uint32_t col = 0, ii = i;
      if (RING) {
        col = (uint32_t)(i >= K) + (uint32_t)(i >= 2u * K) + (uint32_t)(i >= 3u * K);
        ii = i - col * K;
      }
      uint32_t k = 0, idx[W] = {};
      candidate<RING, W>(G, ii, L, K, k, idx);
      finish_from3(k, n, D.g_base + g0 + col, rk, D.T, cD, cA);
      apply_window<W>(smem + col * L, idx, O, cD.lt, cA.lt, win_lim);
    }
    if (!RING) {
      const uint32_t lo_before = G.lo;
      if (w_lo < (uint32_t)W * K) {
        const uint32_t rem = w_lo - (uint32_t)W * G.k_lo;
        if (rem) G.lo += (uint32_t)W - rem;
      }
      uint32_t w_hi = w_lo + (G.hi - 1u - lo_before);
      if (w_hi >= L) w_hi -= L;
      if (w_hi < (uint32_t)W * K) {
        const uint32_t rem = w_hi % (uint32_t)W;
        if (rem != (uint32_t)W - 1u) G.hi -= 1u + rem;
      }
    }
    __syncthreads();
    if (r < D.n_rec && D.rec_sub[r] == n + 1u) {
      // a segment's pair record reads the site after its core: it must lie inside the tile
      if (!RING) (void)PCPD_IN_BOUNDS(H + core_len, tile_len, kDbgRecord);
      for (uint32_t c = 0; c < gpi; ++c)
        tile_count(smem + c * L, H, H + core_len, D.rec_total, D.rec_sample, D.rec_pairs, D.S, r, g0 + c,
                   RING ? L : 0u, s_red);
      ++r;
    }
  }
}

template <bool BATCH>
__device__ __forceinline__ const InstDesc &descriptor(const BatchParams &B, uint32_t i);
template <>
__device__ __forceinline__ const InstDesc &descriptor<false>(const BatchParams &B, uint32_t) {
  return B.single;
}
template <>
__device__ __forceinline__ const InstDesc &descriptor<true>(const BatchParams &, uint32_t i) {
  return c_inst[i];
}

// WFIX: the window width of every instance of the launch (3, 4 or 5), or 0 to read it from
// each instance's descriptor.
template <bool BATCH, int WFIX>
__device__ __forceinline__ void sweep_body(const BatchParams &B) {
  extern __shared__ __align__(128) uint32_t smem[];
  __shared__ uint32_t s_phi[kPhiChunk];
  __shared__ unsigned int s_red[34];
  __shared__ unsigned int s_q3n;
  __shared__ unsigned long long s_item;
  __shared__ int s_abort;
  __shared__ __align__(8) unsigned long long s_mbar;

  uint32_t *q3 = smem + B.tile_words;
  uint32_t parity = 0;
  if (threadIdx.x == 0) mbar_init(&s_mbar);
  for (uint32_t t = threadIdx.x; t <= 33u; t += blockDim.x) s_red[t] = 0;
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long it = ~0ull;
      if (*(volatile uint32_t *)B.err == 0u) {
        const uint32_t q = atomicAdd(B.counter, 1u);
        if (q < B.n_items)
          it = B.items ? B.items[q] : pack_item(0u, q / B.tiles_per_epoch, q % B.tiles_per_epoch);
      }
      s_item = it;
      s_abort = 0;
    }
    __syncthreads();
    const unsigned long long item = s_item;
    if (item == ~0ull) break;
    const uint32_t inst = (uint32_t)(item >> 48);
    const uint32_t e = (uint32_t)((item >> 24) & 0xFFFFFFu);
    const uint32_t tile = (uint32_t)(item & 0xFFFFFFu);
    const InstDesc &D = descriptor<BATCH>(B, inst);
    const bool ring = D.ring != 0u;
    const uint32_t cg = tile / D.n_seg, sg = tile - cg * D.n_seg;
    const uint32_t g0 = cg * (ring ? D.gpi : 1u);
    const uint32_t L = D.L;
    const uint32_t gpi = ring ? D.gpi : 1u;
    const uint32_t *src = (e & 1u) ? D.buf1 : D.buf0;
    uint32_t *dst = (e & 1u) ? D.buf0 : D.buf1;

    // wait until the tiles this one reads have finished epoch e-1
    if (threadIdx.x == 0 && e > 0u) {
      uint32_t deps[3] = {tile, tile, tile};
      if (!ring && D.n_seg > 1u) {
        deps[1] = cg * D.n_seg + (sg == 0u ? D.n_seg - 1u : sg - 1u);
        deps[2] = cg * D.n_seg + (sg + 1u == D.n_seg ? 0u : sg + 1u);
      }
      const long long t0 = clock64();
      for (int q = 0; q < 3 && !s_abort; ++q) {
        while (ld_acquire(D.done + deps[q]) < e) {
          if (*(volatile uint32_t *)B.err != 0u) { s_abort = 1; break; }
          if ((unsigned long long)(clock64() - t0) > B.spin_limit) {
            atomicCAS(B.err, 0u, kErrDepTimeout);
            s_abort = 1;
            break;
          }
          __nanosleep(256);
        }
      }
    }
    __syncthreads();
    if (s_abort) break;

    // ---- load the tile: TMA for aligned spans, L2-coherent loads otherwise ----
    const uint32_t s0 = ring ? 0u : sg * D.core;
    const uint32_t core_len = ring ? L : min(D.core, L - s0);
    const uint32_t H = ring ? 0u : D.halo;
    const uint32_t tile_len = core_len + 2u * H;
    const uint32_t base = ring ? 0u : (uint32_t)(((uint64_t)s0 + L - H) % L);
    // spans: (smem offset, global column offset, words); at most 2 per column
    uint32_t tma_bytes = 0;
    for (uint32_t c = 0; c < gpi; ++c) {
      const uint32_t *col = src + (size_t)(g0 + c) * D.pitch;
      uint32_t *sm = smem + c * L;
      const uint32_t len1 = min(tile_len, L - base);
      const uint32_t off[2] = {0u, len1};
      const uint32_t gof[2] = {base, 0u};
      const uint32_t len[2] = {len1, tile_len - len1};
      for (int sp = 0; sp < 2; ++sp) {
        if (len[sp] == 0u) continue;
        if (!PCPD_IN_BOUNDS((unsigned long long)c * L + off[sp] + len[sp] - 1u, B.tile_words, kDbgLoadDst) ||
            !PCPD_IN_BOUNDS((unsigned long long)gof[sp] + len[sp] - 1u, D.pitch, kDbgLoadSrc))
          continue;
        if (tma_ok(sm + off[sp], col + gof[sp], len[sp])) {
          if (threadIdx.x == 0) {
            if (tma_bytes == 0u) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_bytes += 4u * len[sp];
          }
        } else {
          for (uint32_t y = threadIdx.x; y < len[sp]; y += blockDim.x) sm[off[sp] + y] = __ldcg(col + gof[sp] + y);
        }
      }
    }
    if (threadIdx.x == 0 && tma_bytes) {
      mbar_expect_tx(&s_mbar, tma_bytes);
      for (uint32_t c = 0; c < gpi; ++c) {
        const uint32_t *col = src + (size_t)(g0 + c) * D.pitch;
        uint32_t *sm = smem + c * L;
        const uint32_t len1 = min(tile_len, L - base);
        const uint32_t off[2] = {0u, len1};
        const uint32_t gof[2] = {base, 0u};
        const uint32_t len[2] = {len1, tile_len - len1};
        for (int sp = 0; sp < 2; ++sp) {
          if (len[sp] == 0u || !tma_ok(sm + off[sp], col + gof[sp], len[sp])) continue;
          if (!PCPD_IN_BOUNDS((unsigned long long)c * L + off[sp] + len[sp] - 1u, B.tile_words, kDbgLoadDst) ||
              !PCPD_IN_BOUNDS((unsigned long long)gof[sp] + len[sp] - 1u, D.pitch, kDbgLoadSrc))
            continue;
          uint32_t done_w = 0;
          while (done_w < len[sp]) {   // chunks of at most 32 KB
            const uint32_t w = min(len[sp] - done_w, 8192u);
            tma_load_1d(sm + off[sp] + done_w, col + gof[sp] + done_w, 4u * w, &s_mbar);
            done_w += w;
          }
        }
      }
      const long long t0 = clock64();
      while (!mbar_try_wait(&s_mbar, parity)) {
        if ((unsigned long long)(clock64() - t0) > B.spin_limit) {
          atomicCAS(B.err, 0u, kErrLoadTimeout);
          s_abort = 1;
          // give the copies in flight a second bounded chance to land before the CTA exits
          const long long t1 = clock64();
          while (!mbar_try_wait(&s_mbar, parity) &&
                 (unsigned long long)(clock64() - t1) < B.spin_limit) {
          }
          break;
        }
      }
    }
    if (threadIdx.x == 0 && tma_bytes) parity ^= 1u;
    __syncthreads();
    if (s_abort) break;   // a timed-out copy may still land in shared memory: stop here

#ifdef PCPD_JIT_W
    // a build specialised for one window width
    if (ring) run_item<true, PCPD_JIT_W>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
    else run_item<false, PCPD_JIT_W>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
#else
    if constexpr (WFIX != 0) {
      if (ring) run_item<true, WFIX>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
      else run_item<false, WFIX>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
    } else if (D.W == 4u) {
      if (ring) run_item<true, 4>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
      else run_item<false, 4>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
    } else if (D.W == 5u) {
      if (ring) run_item<true, 5>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
      else run_item<false, 5>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
    } else {
      if (ring) run_item<true, 3>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
      else run_item<false, 3>(D, smem, q3, g0, sg, e, s_phi, s_red, &s_q3n);
    }
#endif

    // ---- store the core and publish the epoch ----
    for (uint32_t c = 0; c < gpi; ++c) {
      uint32_t *col = dst + (size_t)(g0 + c) * D.pitch + s0;
      const uint32_t *sm = smem + c * L + H;
      if (!PCPD_IN_BOUNDS((unsigned long long)c * L + H + core_len - 1u, B.tile_words, kDbgStore) ||
          !PCPD_IN_BOUNDS((unsigned long long)s0 + core_len - 1u, D.pitch, kDbgStore))
        continue;
      for (uint32_t y = threadIdx.x; y < core_len; y += blockDim.x) __stcg(col + y, sm[y]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(D.done + tile, e + 1u);
    }
  }
  // parity is per-thread-0 state; nothing else to release (no TMEM, no outstanding copies
  // except after a timed-out wait, which ends the CTA after the error is recorded)
}

template <bool BATCH, int WFIX>
__global__ void __launch_bounds__(kSweepThreads, 1) k_sweep_persistent(const BatchParams B) {
  sweep_body<BATCH, WFIX>(B);
}

}  // namespace pcpdk
