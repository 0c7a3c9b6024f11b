/*
 * nlh_mis.h -- feature windows ranked by mutual information (Sec. 5).
 *
 * Sec. 5 scores every patch dimension by its mutual information (MIS) with
 * the noisy pixel values f (the target standing in for the clean image),
 * ranks the dimensions and groups them into L = ceil(D / 3) windows of at
 * most three dimensions.  The paper leaves the estimator open; this library
 * uses the plug-in mutual information, in nats, of the equal-width
 * bins x bins joint histogram of (feature d, f):
 *   lo, hi   the minimum and maximum of the variable over the N pixels;
 *   bin(x)   = min(bins - 1, floor((x - lo) * (bins / (hi - lo)))) in FP64
 *              (the difference and the product rounded separately; every
 *              value in bin 0 when hi = lo);
 *   MIS_d    = sum over c_ab > 0 of (c_ab / N) log(c_ab N / (c_a c_b)),
 *              with (c_ab N) / (c_a c_b) evaluated in that order.
 * Ranking: MIS descending, ties to the lower dimension; window l holds the
 * ranks 3l, 3l + 1, 3l + 2, the last window completed with -1 (a
 * zero-valued dimension), the layout nlh_plan_desc.windows takes.
 *
 * Conventions as in nlh.h: DEVICE arrays owned by the caller, `stream` a
 * cudaStream_t as void*, status codes with a message from nlh_last_error().
 */
#ifndef NLH_MIS_H
#define NLH_MIS_H

#include "nlh.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Scores and windows of an image's patch features.
 *   image    DEVICE n1 x n2 FP64, row-major; the features are those of
 *            nlh_patch_features(image, n1, n2, radius, pad) (computed on
 *            the fly, not stored), D = (2 radius + 1)^2
 *   bins     histogram bins per variable, 2..128
 *   mis      DEVICE D doubles: MIS of every patch dimension
 *   windows  DEVICE ceil(D / 3) x 3 int32 (may be NULL)
 *   counts   DEVICE D x bins x bins int32 joint counts c[d][a][b], a the
 *            feature bin, b the target bin (may be NULL: internal scratch)
 * Stream-ordered; no synchronisation.  Integer work (bins, counts, ranks)
 * is exact; the scores are deterministic for a given input.
 * Errors: NLH_ERR_ARG (NULL image or mis, n1, n2 < 1, radius outside 0..6,
 * pad not 0 or 1, bins outside 2..128), NLH_ERR_OOM, NLH_ERR_CUDA. */
nlh_status nlh_mis_windows(const double *image, int n1, int n2, int radius, int pad, int bins,
                           double *mis, int32_t *windows, int32_t *counts, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NLH_MIS_H */
