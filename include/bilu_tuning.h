/*
 * bilu_tuning.h -- tuning knobs and test hooks of libbilu.  They change how
 * the kernels of bilu.h are scheduled, never what they compute (the paper has
 * no counterpart: these are implementation parameters).  Process-wide,
 * host-side settings; not thread safe against concurrent calls.
 */
#ifndef BILU_TUNING_H
#define BILU_TUNING_H

#include <stdint.h>

#include "bilu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Target of consecutive block rows one CTA owns in the sync-free triangular
 * solves.  Dependencies inside a chunk resolve through shared memory,
 * dependencies across chunks through global memory.  0 (the default) picks
 * per pattern: n / (10 * SMs) rows, clamped to [32, 256], so that small
 * systems still spread over the GPU; where that hits 256 and the pattern
 * shows a line length L of 16..192 rows (the most common distance between
 * rows that do not depend on their predecessor: grid-line starts in a
 * natural ordering), 2 L instead -- two grid lines per chunk; 1 <= rows <=
 * 1024 fixes the target;
 * other values: BILU_ERR_ARG.  Takes effect for a pattern at its next
 * bilu_pattern_upload or bilu_pattern_schedule (the set-up calls that build
 * schedules); apply, factor and solve never rebuild one. */
int bilu_set_trisolve_chunk(int32_t rows);
int32_t bilu_get_trisolve_chunk(void);

/* The target the solves use for pattern p when none is set (bilu_set_trisolve_chunk(0)),
 * for inspection: host pattern, no device work.  Returns -1 for a NULL p. */
int32_t bilu_auto_trisolve_chunk(const bilu_pattern* p);

/* Target of consecutive block rows one CTA owns in the sync-free
 * factorization: 0 (the default) picks n / (2 * SMs) clamped to [64, 256],
 * or 3 L (three grid lines) where that hits 256 and a line length L of
 * 16..128 rows is detected (see bilu_set_trisolve_chunk);
 * 1 <= rows <= 1024 fixes it; other values: BILU_ERR_ARG.  Its schedule is
 * separate from the solves'; like theirs it is built by bilu_pattern_upload
 * and bilu_pattern_schedule only. */
int bilu_set_factor_chunk(int32_t rows);
int32_t bilu_get_factor_chunk(void);

/* The target the factorization uses for pattern p when none is set, for
 * inspection (as bilu_auto_trisolve_chunk).  Returns -1 for a NULL p. */
int32_t bilu_auto_factor_chunk(const bilu_pattern* p);

/* Warps per CTA in the triangular solves: 4 (default), 8 or 16, else
 * BILU_ERR_ARG.  More warps per chunk give each row more time to fetch its
 * operands ahead of its dependencies.  Applies to the next launch. */
int bilu_set_trisolve_warps(int32_t warps);

/* Resident CTAs per SM of the triangular solves' persistent grid: 0 (the
 * default) for as many as fit, else 1..32 (capped at what fits).  Fewer CTAs
 * keep fewer chunks in flight and fewer warps polling.  Applies to the next
 * launch; BILU_ERR_ARG outside 0..32. */
int bilu_set_trisolve_ctas_per_sm(int32_t ctas);

/* Host copy of the schedule the sync-free solves use for a target of `rows`
 * rows per chunk (the same one bilu_pattern_upload / bilu_pattern_schedule
 * build; the factorization builds one the same way for its own target).  Rows are cut into *nchunks chunks
 * of consecutive rows, chunk c = rows [bounds[c], bounds[c+1]).  A cut falls
 * before the row farthest from its nearest dependency (the largest gap
 * r - max{j < r in L(r)}, and likewise for U') among the rows with a gap > 1
 * in [rows/2, 3*rows/2] (at most 1024) rows from the chunk's start, the one
 * nearest the target among equal gaps; else at the target.
 *   bounds (n + 1 entries capacity): the cut rows, bounds[0] = 0,
 *     bounds[*nchunks] = n.
 *   ord_lower / ord_upper (n entries): the rows of each chunk, at the
 *     positions of the chunk's rows, listed by dependency level within the
 *     chunk (ascending rows break ties for L, descending rows for U').
 *   tick_lower / tick_upper (n entries capacity): the chunk each claim ticket
 *     hands out, a topological order of the chunk dependency graph.  The
 *     lower solve numbers chunks c = 0.. in ascending rows, the upper solve in
 *     descending rows (its chunk c is chunk nchunks - 1 - c above).
 * nchunks is required; any other output may be NULL.  Caller-allocated.  Host
 * only, except for a pattern bilu_symbolic_gpu left on the device, whose
 * schedule is built on the current device as bilu_pattern_upload builds it
 * (the same schedule; synchronises). */
int bilu_schedule_export(const bilu_pattern* p, int32_t rows, int32_t* nchunks, int32_t* bounds,
                         int32_t* ord_lower, int32_t* ord_upper, int32_t* tick_lower, int32_t* tick_upper);

/* Time limit of every bounded dependency wait in the factorization and the
 * triangular solves, in nanoseconds (default 2e9).  >= 1000, else
 * BILU_ERR_ARG.  A wait that runs out records BILU_ERR_TIMEOUT and the kernel
 * returns; it never traps. */
int bilu_set_spin_limit_ns(int64_t ns);

/* BiCGSTAB iterations enqueued between two host reads of the device state
 * (default 4).  1 <= iters <= 1000, else BILU_ERR_ARG. */
int bilu_set_check_every(int32_t iters);

/* Test hook: the lower triangular solve computes block row `row` but never
 * publishes it, so every row that depends on it waits until the spin limit
 * and the call reports BILU_ERR_TIMEOUT.  -1 (the default) disables it. */
int bilu_test_withhold_row(int32_t row);

/* Kernel classes for bilu_profile_read. */
enum bilu_prof_kernel {
  BILU_PROF_SPMV = 0,         /* bsr_spmv kernel */
  BILU_PROF_APPLY_PREP = 1,   /* apply: reset of the pending markers */
  BILU_PROF_LOWER = 2,        /* apply: sync-free L y = r */
  BILU_PROF_UPPER = 3,        /* apply: sync-free U' x = z (z = D^{-1} y) */
  BILU_PROF_BACKFILL = 4,     /* factor: A -> A' gather */
  BILU_PROF_FACTOR = 5,       /* factor: Algorithm 4 + D^{-1} */
  BILU_PROF_SCALE_UPPER = 6,  /* factor: U' = D^{-1} U */
  BILU_PROF_KRYLOV = 7,       /* BiCGSTAB vector updates and reductions */
  BILU_PROF_FACTOR_INIT = 8,  /* factor: reset of the ready flags */
  BILU_PROF_ADJOINT = 9,      /* adjoint: block gather-transposes and -lambda x^T */
  BILU_PROF_SYMBOLIC = 10,    /* device symbolic phase (bilu_symbolic_gpu) */
  BILU_PROF_DIAG = 11,        /* apply: z = D^{-1} y between the two sweeps */
  BILU_PROF_NKERNELS = 12
};

/* Per-kernel timing: when on, every launch of the library is bracketed by
 * CUDA events on its stream.  Enabling (or disabling) clears the counters. */
int bilu_profile_enable(int32_t on);

/* Waits for the recorded events and returns, for one kernel class, the
 * number of timed launches and their summed device time in milliseconds. */
int bilu_profile_read(int32_t kernel, int64_t* launches, double* total_ms);

/* Number of kernels the library has launched in this process (all classes,
 * whether or not profiling is on). */
int64_t bilu_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
