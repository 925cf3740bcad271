/* C ABI of the device Matérn random-field sampler.
 *
 * Section 2.1 draws the nodal modulus and thickness of every realisation from a
 * Gaussian Markov random field: the SPDE (kappa^2 - Laplacian)^(alpha/2) x = W with
 * nu = 1 (alpha = 2 on the 2-D wall surface) discretised with piecewise linear basis
 * functions, G_ij = <grad psi_i, grad psi_j>, C~ the lumped mass, and precision
 * Q_2 = (kappa^2 C~ + G)^T C~^-1 (kappa^2 C~ + G). The paper factors Q_2 (Cholesky) and
 * solves with the transposed factor. This library draws the same distribution as
 * x = K^-1 C~^(1/2) z with K = kappa^2 C~ + G (covariance K^-1 C~ K^-1 = Q_2^-1), which
 * needs only products with the sparse K: all S right-hand sides are solved together by
 * preconditioned conjugate gradients on the device, sample index innermost.
 *
 * Conventions: every call returns GMRF_OK (0) or a negative GMRF_ERR_*; gmrf_last_error
 * gives the message. Host inputs are copied; device arrays belong to the caller. Work
 * runs on the stream given at create; gmrf_sample returns after it has finished.   */
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GMRF_OK 0
#define GMRF_ERR_INVALID_ARG (-1) /* bad argument (message says which)                */
#define GMRF_ERR_ALLOC (-2)       /* device allocation failed                        */
#define GMRF_ERR_CUDA (-3)        /* a CUDA runtime call failed                      */
#define GMRF_ERR_NOT_CONVERGED (-9) /* some sample missed rtol within max_iter       */

typedef struct gmrf_ctx gmrf_ctx;

/* Assemble K = kappa^2 C~ + G of the triangulated surface on the host, in binary64, and
 * copy it to the device as CSR together with the Jacobi preconditioner and C~^(1/2).
 * xyz host [n_nodes][3], tri host [n_elems][3] (node ids in [0, n_nodes), every node in
 * some element, no element of zero area). corr_length > 0: the correlation length rho
 * of Section 2.1 (the distance at which the correlation is near 0.1); the library takes
 * kappa = sqrt(8 nu) / rho with nu = 1 and reports it in gmrf_info_t. stream:
 * cudaStream_t (NULL = legacy default stream).                                      */
int gmrf_create(int32_t n_nodes, int32_t n_elems, const double *xyz, const int32_t *tri,
                double corr_length, void *stream, gmrf_ctx **out);

/* Draw S fields. z: device [n_nodes][S] binary64 standard normals (sample index
 * innermost), read only. out: device [n_nodes][S] binary64, written with
 *     out = mean * exp(c * x)   (lognormal = 1)   or   out = mean + c * x   (0),
 * x = K^-1 C~^(1/2) z, where c = sigma sqrt(4 pi) kappa gives the Gaussian field c x the
 * marginal standard deviation sigma of the continuous Matern field (variance
 * 1 / (4 pi kappa^2) for nu = 1 on a 2-D surface, Section 2.1); sigma <= 0 means c = 1
 * (x itself). The solve is iterative refinement from x = 0: the
 * residual b - K x (b = C~^(1/2) z) is formed in binary64, a Jacobi-preconditioned
 * conjugate-gradient solve in binary32 reduces it by a quarter of the factor still needed
 * to reach rtol, clamped to [1e-4, 0.1], and x takes the
 * correction in binary64, until every sample has ||K x - b|| <= rtol ||b|| in binary64,
 * or max_iter binary32 iterations in all (then GMRF_ERR_NOT_CONVERGED, with out still
 * written). Each sample stops updating once it converges, so the result is
 * deterministic.
 * rtol in (0, 1), max_iter >= 1, S >= 1.                                            */
int gmrf_sample(gmrf_ctx *g, int32_t S, const double *z, double *out, double sigma, double mean,
                int32_t lognormal, double rtol, int32_t max_iter);

typedef struct {
    int32_t n_nodes;
    int64_t nnz;            /* stored entries of K                                  */
    int32_t iterations;     /* binary32 CG iterations of the last gmrf_sample       */
    double max_relres;      /* largest binary64 ||b - K x|| / ||b|| over samples     */
    double bytes_per_iter;  /* algorithmic HBM bytes of one CG iteration at that S  */
    int32_t last_S;
    int32_t refinements;    /* binary64 residual / correction steps it took         */
    double bytes_per_refinement; /* algorithmic HBM bytes of one of those steps    */
    double kappa;           /* sqrt(8) / corr_length                                */
} gmrf_info_t;

int gmrf_info(const gmrf_ctx *g, gmrf_info_t *info);

/* Message of the last failed call on g (or of the last failed gmrf_create when g is
 * NULL, per thread). */
const char *gmrf_last_error(const gmrf_ctx *g);

void gmrf_destroy(gmrf_ctx *g);

#ifdef __cplusplus
}
#endif
