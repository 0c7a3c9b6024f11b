/*
 * nlh_bilevel.h -- reductions of the bilevel learning of alpha (Sec. 2,
 * Eq. Optimality_System_Regularization; Sec. 5.5, Eq. BilevelProblem).
 *
 * For a training pair (u_c clean, f noisy) and the lower-level solution
 * (alpha I + L) u = alpha f, the objective term is ||u - u_c||^2 and the
 * adjoint state solves (alpha I + L) p = u - u_c (with nlh_solve); the
 * derivative of ||u - u_c||^2 with respect to alpha is 2 <p, f - u>.
 *
 * Vectors are DEVICE FP64 arrays of N values owned by the caller; results
 * are written to HOST doubles and the call synchronises `stream`.  Sums use
 * fixed-order block partials (deterministic for a given N).
 */
#ifndef NLH_BILEVEL_H
#define NLH_BILEVEL_H

#include "nlh.h"

#ifdef __cplusplus
extern "C" {
#endif

/* r = u - uc (r may be NULL) and *sq = ||u - uc||^2.  Errors: NLH_ERR_ARG
 * (NULL u, uc or sq, N < 1), NLH_ERR_CUDA. */
nlh_status nlh_bilevel_misfit(int64_t N, const double *u, const double *uc, double *r,
                              double *sq, void *stream);

/* *dot = <p, f - u>.  Errors: NLH_ERR_ARG, NLH_ERR_CUDA. */
nlh_status nlh_bilevel_gradient_term(int64_t N, const double *p, const double *f,
                                     const double *u, double *dot, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NLH_BILEVEL_H */
