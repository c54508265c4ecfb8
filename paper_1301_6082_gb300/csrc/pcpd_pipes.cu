// pcpd_pipes.cu -- lane rates of the integer pipes the PCPD sweep runs on (libpcpd_pipes.so,
// declared in include/pcpd_pipes.h).
//
// The sweep is integer bit work: Philox4x32-10's 32x32->64-bit products, three-input logic
// for the XORs of Philox, the threshold compares (Sec. 4.2-4.3) and the window logic (Alg. 2).
// Its roofline is therefore set by the SM's integer pipes, whose rates this library measures:
// each kernel runs one CTA per SM, every thread advancing 8 independent dependency chains of
// one operation written as inline PTX (so the compiler cannot fold or drop them), and the
// elapsed SM clock cycles are read with clock64 around the timed loop.  The result is in
// lane-operations per SM per clock, independent of the clock frequency.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <utility>
#include <vector>

#include "../../include/pcpd_pipes.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// one source register each: the rest are immediates (no register read)
__device__ __forceinline__ uint32_t lop3_xor_imm(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, 0x5bd1e995, 0x96;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t mad_lo_imm(uint32_t a) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, 0xD2511F53, 0x9E3779B9;" : "=r"(d) : "r"(a));
  return d;
}
__device__ __forceinline__ uint32_t mul_hi_imm(uint32_t a) {
  uint32_t d;
  asm volatile("mul.hi.u32 %0, %1, 0xD2511F53;" : "=r"(d) : "r"(a));
  return d;
}
__device__ __forceinline__ uint64_t mul_wide_imm(uint32_t a) {
  uint64_t d;
  asm volatile("mul.wide.u32 %0, %1, 0xD2511F53;" : "=l"(d) : "r"(a));
  return d;
}
__device__ __forceinline__ uint32_t add3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("{\n\t.reg .u32 t;\n\tadd.u32 t, %1, %2;\n\tadd.u32 %0, t, %3;\n\t}"
               : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Philox4x32-10 (Salmon et al., SC'11): multipliers and Weyl increments of the published
// definition.
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u, kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t k0,
                                       uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)x0 * kM0, p1 = (uint64_t)x2 * kM1;
    const uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
    const uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
    x0 = h1 ^ x1 ^ k0;
    x1 = l1;
    x2 = h0 ^ x3 ^ k1;
    x3 = l0;
    k0 += kW0;
    k1 += kW1;
  }
}

// One CTA per SM.  cycles[blockIdx] = clock64 cycles of the timed loop; sink keeps results live.
template <int OP>
__global__ void k_pipe(uint32_t iters, uint32_t seed, unsigned long long *cycles, uint32_t *sink) {
  uint32_t x[kChains], y[kChains];
  uint64_t w[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    x[j] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (uint32_t)(j + 1) + blockIdx.x;
    y[j] = x[j] ^ 0x5bd1e995u;
    w[j] = ((uint64_t)y[j] << 32) | x[j];
  }
  const uint32_t M = 0xD2511F53u ^ (seed & 0x10u);
  __syncthreads();
  const long long t0 = clock64();
  if constexpr (OP == PCPD_PIPE_PHILOX) {
    // three independent blocks per iteration (the sweep draws up to three per window); every
    // counter word changes with the iteration, so no round can be hoisted out of the loop
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it) {
      const uint32_t c = it * 0x9E3779B9u + threadIdx.x;
      uint32_t a0 = c, a1 = it, a2 = c ^ blockIdx.x, a3 = it + 0u;
      uint32_t b0 = c, b1 = it, b2 = c ^ blockIdx.x, b3 = it + 1u;
      uint32_t c0 = c, c1 = it, c2 = c ^ blockIdx.x, c3 = it + 2u;
      philox(a0, a1, a2, a3, seed, ~seed);
      philox(b0, b1, b2, b3, seed, ~seed);
      philox(c0, c1, c2, c3, seed, ~seed);
      acc ^= a0 ^ a1 ^ a2 ^ a3 ^ b0 ^ b1 ^ b2 ^ b3 ^ c0 ^ c1 ^ c2 ^ c3;
    }
    x[0] ^= acc;
  } else {
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if constexpr (OP == PCPD_PIPE_LOP3) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = lop3_xor(x[j], x[(j + 1) % kChains], x[(j + 2) % kChains]);
        } else if constexpr (OP == PCPD_PIPE_LOP3_2R) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = lop3_xor_imm(x[j], x[(j + 1) % kChains]);
        } else if constexpr (OP == PCPD_PIPE_IMAD_LO) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = mad_lo(x[j], M, x[(j + 1) % kChains]);
        } else if constexpr (OP == PCPD_PIPE_IMAD_LO_1R) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = mad_lo_imm(x[j]);
        } else if constexpr (OP == PCPD_PIPE_IMAD_HI) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = mul_hi_imm(x[j]);
        } else if constexpr (OP == PCPD_PIPE_IMAD_WIDE) {   // each product's halves feed the next
#pragma unroll
          for (int j = 0; j < kChains; ++j) {
            w[j] = mul_wide_imm(x[j]);
            x[j] = lop3_xor_imm((uint32_t)w[j], (uint32_t)(w[j] >> 32));
          }
        } else if constexpr (OP == PCPD_PIPE_IADD) {
#pragma unroll
          for (int j = 0; j < kChains; ++j) x[j] = add3(x[j], x[(j + 1) % kChains], x[(j + 2) % kChains]);
        } else if constexpr (OP == PCPD_PIPE_MIX_LO_LOP3) {   // 8 multiply-add chains beside 8 logic chains
#pragma unroll
          for (int j = 0; j < kChains; ++j) {
            x[j] = mad_lo(x[j], M, x[(j + 1) % kChains]);
            y[j] = lop3_xor(y[j], y[(j + 1) % kChains], y[(j + 2) % kChains]);
          }
        } else if constexpr (OP == PCPD_PIPE_MIX_LIGHT) {   // the same with one or two register sources
#pragma unroll
          for (int j = 0; j < kChains; ++j) {
            x[j] = mad_lo_imm(x[j]);
            y[j] = lop3_xor_imm(y[j], y[(j + 1) % kChains]);
          }
        } else if constexpr (OP == PCPD_PIPE_MIX_WIDE_LOP3) {   // widening products beside logic chains
#pragma unroll
          for (int j = 0; j < kChains; ++j) {
            w[j] = mul_wide_imm(x[j]);
            x[j] = lop3_xor_imm((uint32_t)w[j], (uint32_t)(w[j] >> 32));
            y[j] = lop3_xor_imm(y[j], y[(j + 1) % kChains]);
          }
        }
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) r ^= x[j] ^ y[j] ^ (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
  if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

using PipeKernel = void (*)(uint32_t, uint32_t, unsigned long long *, uint32_t *);

template <int... OPS>
PipeKernel pick(int op, std::integer_sequence<int, OPS...>) {
  PipeKernel k = nullptr;
  ((op == OPS ? (k = k_pipe<OPS>, 0) : 0), ...);
  return k;
}

PipeKernel kernel_of(int op) { return pick(op, std::make_integer_sequence<int, PCPD_PIPE_COUNT>{}); }

// Operations one thread performs per loop iteration, in the unit of the result.
double ops_per_iter(int op) {
  switch (op) {
    case PCPD_PIPE_PHILOX: return 3.0;   // Philox blocks
    case PCPD_PIPE_MIX_LO_LOP3:
    case PCPD_PIPE_MIX_LIGHT: return 2.0 * kChains * kUnroll;   // both kinds counted
    case PCPD_PIPE_MIX_WIDE_LOP3: return 3.0 * kChains * kUnroll;   // products and both logic ops
    default: return (double)kChains * kUnroll;
  }
}

}  // namespace

extern "C" int pcpd_pipe_rate(int op, uint32_t iters, uint32_t threads, double *lanes_per_sm_clock,
                              double *ms_out) {
  const PipeKernel k = kernel_of(op);
  if (!k || !lanes_per_sm_clock || threads == 0 || threads > 1024 || threads % 32 || iters == 0) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 6;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  unsigned long long *d_cyc = nullptr;
  uint32_t *d_sink = nullptr;
  if (cudaMalloc(&d_cyc, sms * sizeof(unsigned long long)) != cudaSuccess) return 2;
  if (cudaMalloc(&d_sink, (size_t)sms * threads * sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(d_cyc);
    return 2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k<<<sms, threads>>>(iters < 4 ? iters : 4u, 7u, d_cyc, d_sink);   // warm-up
  cudaEventRecord(e0);
  k<<<sms, threads>>>(iters, 7u, d_cyc, d_sink);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  std::vector<unsigned long long> cyc(sms);
  if (err == cudaSuccess)
    err = cudaMemcpy(cyc.data(), d_cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_cyc);
  cudaFree(d_sink);
  if (err != cudaSuccess) return 3;
  double mean_cyc = 0.0;
  for (int i = 0; i < sms; ++i) mean_cyc += (double)cyc[i];
  mean_cyc /= sms;
  *lanes_per_sm_clock = (double)threads * iters * ops_per_iter(op) / mean_cyc;
  if (ms_out) *ms_out = ms;
  return 0;
}

extern "C" int pcpd_pipe_count(void) { return PCPD_PIPE_COUNT; }
