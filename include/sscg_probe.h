/*
 * sscg_probe - arithmetic throughput probes of the GPU the library runs on.
 *
 * The s-step solver's kernels in FP64 arithmetic are bound by the FP64 units
 * of a GB300, not by its memory: its FP64 rate is about 1/64 of its FP32 rate.
 * These probes measure the roofs those kernels are held to.  Each launches one
 * kernel over a full-device grid (the SM count times as many 256-thread CTAs
 * as fit on an SM), whose threads run independent dependency chains of one
 * kind of instruction, and times it with CUDA events on the context's stream.
 * The paper has no counterpart: this is measurement support, not the method.
 *
 * Plain C ABI, part of libsscg.
 */
#ifndef SSCG_PROBE_H
#define SSCG_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Probe kinds.  Operation counts: one FP64 fused multiply-add, add or
 * multiply per thread and instruction is one operation; one warp-wide
 * mma.sync.m8n8k4.f64 is 256 multiply-adds (8 x 8 x 4); one FP32 FMA, one
 * 32-bit integer instruction, one wide multiply-add or one conversion per
 * thread is one operation. */
typedef enum {
    SSCG_PROBE_DFMA = 0,      /* fma(a, m, c), FP64 */
    SSCG_PROBE_DADD = 1,      /* a + c, FP64 */
    SSCG_PROBE_DMUL = 2,      /* a * m, FP64 */
    SSCG_PROBE_DMMA = 3,      /* mma.sync.aligned.m8n8k4.row.col.f64 (FP64 tensor instruction) */
    SSCG_PROBE_DFMA_DMMA = 4, /* even warps DFMA (iters_a), odd warps DMMA (iters_b), one launch */
    SSCG_PROBE_FFMA = 5,      /* fmaf, FP32 */
    SSCG_PROBE_IALU = 6,      /* (x ^ x' ^ y) + z on 32-bit integers (x' another chain): one LOP3 and one add */
    SSCG_PROBE_IMAD = 7,      /* x * m + x' on 32-bit integers (x' another chain) */
    SSCG_PROBE_IMAD_WIDE = 8, /* mad.wide.s32: a * m + c, 32 x 32 bits into a 64-bit sum (c another chain) */
    SSCG_PROBE_I2F64 = 9,     /* cvt.rn.f64.s64: a 64-bit integer to FP64 */
    SSCG_PROBE_F2I64 = 10     /* cvt.rzi.s64.f64: FP64 to a 64-bit integer, truncated */
} sscg_probe_kind;

typedef struct sscg_ctx sscg_ctx;

/* Launch probe `kind` with iters_a steps per chain (iters_b: the DMMA warps'
 * steps of SSCG_PROBE_DFMA_DMMA; ignored otherwise) and report the operations
 * per second over the whole device (*ops_per_s, the sum of both halves for
 * SSCG_PROBE_DFMA_DMMA) and the kernel's device time (*ms).  Synchronises the
 * context's stream.  Errors: SSCG_ERR_INVALID (kind, iteration counts <= 0
 * or above 2^40, null outputs), SSCG_ERR_CUDA. */
int sscg_probe_rate(sscg_ctx* ctx, int kind, int64_t iters_a, int64_t iters_b, double* ops_per_s, double* ms);

/* Latency of the on-chip s x s solves of Algorithm 6 (the serial tail of
 * each outer step, run by one warp of the last CTA): one warp times, with the
 * SM's cycle counter, the library's own routines on an s x s SPD matrix and
 * on the moments of a positive 16-point measure, each `reps` times, and
 * reports mean cycles in cycles[0..3]: the Cholesky factorisation, the
 * triangular solves with 1 and with s right-hand sides, and the monomial
 * step's first-step form (factorisation and one solve of the moment matrix).
 * Uses the library's static device storage, no caller memory; synchronises
 * the context's stream.  Errors: SSCG_ERR_INVALID (s outside 1..8, reps
 * outside 1..100000, null output), SSCG_BREAKDOWN (a factorisation
 * failed, which the fixed inputs do not cause), SSCG_ERR_CUDA. */
int sscg_probe_small_solve(sscg_ctx* ctx, int s, int reps, double* cycles);

#ifdef __cplusplus
}
#endif
#endif /* SSCG_PROBE_H */
