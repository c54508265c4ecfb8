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
    PCPD_PIPE_LOP3 = 0,          /* lop3.b32 (three-input XOR), three register sources */
    PCPD_PIPE_LOP3_2R = 1,       /* lop3.b32 with two register sources and an immediate */
    PCPD_PIPE_IMAD_LO = 2,       /* mad.lo.u32: low half of a 32x32 product plus an addend
                                    (two register sources) */
    PCPD_PIPE_IMAD_LO_1R = 3,    /* mad.lo.u32 with one register source (constant factor and
                                    addend) */
    PCPD_PIPE_IMAD_HI = 4,       /* mul.hi.u32 by a constant: the high half of a product */
    PCPD_PIPE_IMAD_WIDE = 5,     /* mul.wide.u32 by a constant, the form every Philox multiply
                                    takes, its two halves XORed into the next factor (result in
                                    products; the XORs run on the logic pipe beside them) */
    PCPD_PIPE_IADD = 6,          /* two dependent add.u32 (a three-input add) */
    PCPD_PIPE_MIX_LO_LOP3 = 7,   /* IMAD_LO and LOP3 chains side by side (both counted) */
    PCPD_PIPE_MIX_LIGHT = 8,     /* IMAD_LO_1R and LOP3_2R chains side by side (both counted) */
    PCPD_PIPE_MIX_WIDE_LOP3 = 9, /* IMAD_WIDE chains beside LOP3_2R chains (products and all
                                    logic operations counted) */
    PCPD_PIPE_PHILOX = 10,       /* Philox4x32-10 blocks on counters that all change every
                                    iteration (result in blocks; 3 independent blocks per
                                    iteration and thread) */
    PCPD_PIPE_COUNT = 11
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
