/*
 * nlh_selftest.h -- test hooks for the failure path of the library's bounded
 * device waits, and for the solver's stopping rules.
 *
 * Every wait inside the library's kernels (bulk copies, tensor-core
 * commits) is bounded: a wait that gives up records NLH_ERR_TIMEOUT in the
 * owning plan's or network's device error word, the kernel skips its
 * stores and returns, and the next synchronising call on that object
 * reports the status (and clears the word).  These hooks make such a wait
 * run out on purpose, without any fault: one CTA polls an mbarrier that
 * nothing ever completes (the non-blocking mbarrier.test_wait, 2^20
 * polls), then records NLH_ERR_TIMEOUT in the object's word exactly as a
 * library kernel would.  No result of the library depends on them.
 *
 * Conventions as in nlh.h.  Stream-ordered; no synchronisation.
 */
#ifndef NLH_SELFTEST_H
#define NLH_SELFTEST_H

#include "nlh.h"
#include "nlh_net.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Time out a wait into the plan's error word: the next nlh_solve (or
 * nlh_solve_batched) on the plan returns NLH_ERR_TIMEOUT; later calls work.
 * Errors: NLH_ERR_ARG (NULL plan), NLH_ERR_CUDA. */
nlh_status nlh_selftest_plan_timeout(nlh_plan plan, void *stream);

/* The same into the network's error word: nlh_net_check (and the other
 * synchronising network calls) then return NLH_ERR_TIMEOUT once.
 * Errors: NLH_ERR_ARG (NULL net), NLH_ERR_CUDA. */
nlh_status nlh_selftest_net_timeout(nlh_net net, void *stream);

/* The mixed solve's inner tolerance for a refinement step (nlh_solve_opts
 * .inner_tol = inner, outer tolerance tol, current FP64-accurate relative
 * residual rel), as the solver computes it.  Host only, no GPU needed. */
double nlh_selftest_inner_tolerance(double inner, double tol, double rel);

/* Replays the Krylov stopping rule on a host array of relative residuals
 * rel[0..n) (iteration k has rel[k]) with tolerance tol, maxit and the
 * stagnation window stag (0: off; the automatic inner tolerance uses 3).
 * Returns the iteration at which the solve stops, -1 if it runs through
 * all n, -2 for a NULL array or n < 0.  Host only, no GPU needed. */
int nlh_selftest_convergence(const double *rel, int n, double tol, int maxit, int stag);

#ifdef __cplusplus
}
#endif

#endif /* NLH_SELFTEST_H */
