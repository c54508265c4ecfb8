/*
 * pcpd_pipes.h -- C ABI of libpcpd_pipes.so: measured lane rates of the SM's integer pipes,
 * the denominators of the PCPD sweep's roofline.
 *
 * The sweep of arXiv 1301.6082 (bit-sliced PCPD, Sec. 4, Alg. 2; random bits from
 * Philox4x32-10) is integer work bound by the SM's integer pipes, not by memory and not by
 * tensor cores.  Its per-item work is counted in 32x32->64-bit products (Philox's
 * multiplies) and in three-input logic operations (Philox's XORs, the threshold compares of
 * Sec. 4.2-4.3 and the window logic).  This library measures how many such lane-operations
 * one SM completes per clock on the current device, so that the roofline fraction rests on
 * a measurement taken on the same GPU rather than on a datasheet figure.
 *
 * Method: one CTA per SM; every thread advances 8 independent dependency chains of one
 * operation written as inline PTX; thread 0 reads clock64 around the timed loop (after a
 * CTA barrier on both sides).  Rate = threads x iterations x operations per iteration /
 * mean elapsed SM cycles over the CTAs -- lane-operations per SM per clock, independent of
 * the clock frequency.
 */
#ifndef PCPD_PIPES_H
#define PCPD_PIPES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PCPD_PIPE_LOP3 = 0,          /* lop3.b32 (three-input XOR): the logic pipe */
    PCPD_PIPE_IMAD_LO = 1,       /* mad.lo.u32: low half of a 32x32 product plus an addend */
    PCPD_PIPE_IMAD_HI = 2,       /* mad.hi.u32: high half of a 32x32 product plus an addend */
    PCPD_PIPE_IMAD_WIDE = 3,     /* mad.wide.u32: the whole 64-bit product plus a 64-bit addend */
    PCPD_PIPE_IADD = 4,          /* two dependent add.u32 (a three-input add) */
    PCPD_PIPE_MIX_LO_LOP3 = 5,   /* mad.lo and lop3 chains side by side (both counted) */
    PCPD_PIPE_MIX_WIDE_LOP3 = 6, /* mad.wide and lop3 chains side by side (both counted) */
    PCPD_PIPE_PHILOX_SPLIT = 7,  /* Philox4x32-10 blocks, products as high and low multiplies
                                    (result in blocks, 3 independent blocks per iteration) */
    PCPD_PIPE_PHILOX_WIDE = 8,   /* the same with one widening multiply per product */
    PCPD_PIPE_COUNT = 9
};

/* Run operation `op` for `iters` loop iterations on one CTA of `threads` threads (a multiple
 * of 32, <= 1024) per SM of the current device, after a short warm-up launch.  On success
 * (0) *lanes_per_sm_clock = lane-operations (Philox: blocks) completed per SM per clock and
 * *ms_out (nullable) = the timed launch's CUDA-event duration in milliseconds.  Returns 1 for
 * a bad argument, 2 if a device allocation failed, 3 for another CUDA error, 6 without a
 * device.  Allocates and frees two small device buffers per call; waits for completion. */
int pcpd_pipe_rate(int op, uint32_t iters, uint32_t threads, double *lanes_per_sm_clock, double *ms_out);

/* Number of operations (PCPD_PIPE_COUNT). */
int pcpd_pipe_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PCPD_PIPES_H */
