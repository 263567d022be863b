/* libegt_cpu: a multi-core CPU solver of the same EGT hot path in FP64, the
 * comparator the GPU library is measured against on the host's cores.
 *
 * It solves the game an egt_game_desc describes (include/egt.h) with the same
 * method and readings as the GPU library: EGT/as (Algorithms 3 + 4 of Kroer,
 * Farina, Sandholm, arXiv 1810.03063, with Step = Algorithm 2), the dilated
 * entropy smoothed best response (Sec. 5 recursion), the practically tuned
 * initial mu (Sec. 6; alpha times ||A|| sqrt(M_X M_Y), doubled while the
 * excessive gap is negative at the initial point), mu balancing, and the
 * saddle-point residual of Sec. 3 as the stopping test.  The products A y and
 * A^T x are taken per terminal from the hand-vs-hand structure (card-removal
 * inclusion-exclusion for folds, strength-sorted prefix sums with per-card
 * corrections for showdowns; O(T H) work per product instead of the
 * O(T H^2) of the sequence-form matrix), in FP64 with plain sums.  OpenMP
 * spreads the terminals of a product and the hands of a best response over
 * the threads.
 *
 * It shares the betting-tree compiler with the GPU library (the same
 * canonical numbering) and none of its kernels.  It is a measurement baseline:
 * the GPU library never calls it.
 *
 * All pointers are host pointers; the caller owns what it passes.  Calls
 * return an egt_status and never abort; egt_cpu_last_error() gives the
 * thread-local message of the last failure. */
#ifndef EGT_CPU_H
#define EGT_CPU_H

#include "egt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct egt_cpu_game egt_cpu_game;

typedef struct {
  double alpha;       /* initial mu = alpha ||A|| sqrt(M_X M_Y), doubled while EGV < 0 (> 0) */
  double eps_mbb;     /* stop when the residual is <= eps_mbb (0: run max_iters iterations) */
  int32_t max_iters;  /* iterations (accepted Decr calls) at most, >= 0 */
  int32_t gap_every;  /* residual after every gap_every-th iteration and at the last one (>= 1) */
  int32_t threads;    /* OpenMP threads (0: one per processor) */
} egt_cpu_opts;

typedef struct {
  int32_t iters;      /* iterations done */
  int32_t backoffs;   /* tau halvings of Algorithm 4 */
  int32_t products;   /* gradient products taken (3 per Step attempt, 2 per initial point) */
  int32_t threads;    /* OpenMP threads used */
  double gap_mbb;     /* last residual, mbb per hand */
  double mu[2];       /* final mu_x, mu_y */
  double tau;         /* final tau */
  double seconds;     /* wall time of the iterations (the initial point included) */
} egt_cpu_report;

/* Compile the game (same validation as egt_create_game, host only). */
EGT_API egt_status egt_cpu_create(const egt_game_desc* desc, egt_cpu_game** out);

/* Free the game.  NULL is a no-op. */
EGT_API egt_status egt_cpu_destroy(egt_cpu_game* game);

/* Solve from the initial point.  x_out, y_out (may be NULL): the final
 * iterates, [S_p][H] with hands in the description's input order.  Returns
 * EGT_OK, EGT_ERR_NOT_CONVERGED if eps_mbb > 0 was not reached within
 * max_iters, or an error. */
EGT_API egt_status egt_cpu_solve(egt_cpu_game* game, const egt_cpu_opts* opts, double* x_out, double* y_out,
                                 egt_cpu_report* report);

/* Sequences per player (S[2]) and hands (H). */
EGT_API egt_status egt_cpu_dims(const egt_cpu_game* game, int32_t* S, int32_t* H);

EGT_API const char* egt_cpu_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EGT_CPU_H */
