/*
 * Plain FP64 CPU oracle for CoR-UTV and ALM-CoRUTV.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library. The product
 * path (the CUDA library and its Python binding) never calls it, and the two
 * implementations share no code, header, table or helper.
 *
 * Storage: every matrix is row-major float64; `ld` arguments are row strides
 * in elements. Status: 0 = ok, 1 = invalid argument, 2 = allocation failure.
 *
 * Citations are to Kaloorazi & de Lamare, "Study of Compressed Randomized UTV
 * Decompositions for Low-Rank Matrix Approximations in Data Science":
 * Sec. 3.1 (eqs. 4-9), Algorithm 1 (power method), Sec. 3.2 (costs),
 * Sec. 4 (eq. 13, Algorithm 2, the operators C_delta and S_delta), Sec. 5.3.
 */
#ifndef CORUTV_ORACLE_H
#define CORUTV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11). out = bijection of
 * ctr under key. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Standard Gaussian for entry (i, j) of random stream `stream` under `seed`:
 * ctr = (i, j, stream, 0), key = (seed_lo, seed_hi); the four 32-bit words
 * give two 53-bit uniforms u1 in (0,1], u2 in [0,1); z = sqrt(-2 ln u1) cos(2 pi u2)
 * (Box & Muller 1958, cosine branch). */
double or_gauss_entry(uint64_t seed, uint32_t stream, uint32_t i, uint32_t j);

/* psi[i*ell + j] = or_gauss_entry(seed, stream, i, j) for an n x ell matrix. */
void or_gauss_matrix(uint64_t seed, uint32_t stream, int64_t n, int64_t ell, double* psi);

/* Plain products of eqs. 4-5: C (m x l) = A X with A m x n (row stride lda)
 * and X n x l; C (n x l) = A^T Y with Y m x l. Ascending summation order. */
void or_gemm_ax(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda, const double* x,
               double* c);
void or_gemm_aty(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda, const double* y,
                 double* c);

/* Thin Householder QR of the m x l matrix C (m >= l): C = Q R, Q m x l with
 * orthonormal columns, R l x l upper triangular with diag(R) >= 0. */
int or_qr(int64_t m, int64_t l, const double* c, int64_t ldc, double* q, double* r);

/* Column-pivoted QR (Businger & Golub 1965) of the l x l matrix D (eq. 8):
 * D P = Qt Rt, perm[j] = index of the column of D moved to position j.
 * Step j picks the trailing column of largest recomputed residual 2-norm,
 * lowest index on ties. diag(Rt) >= 0. */
int or_qrcp(int64_t l, const double* d, double* qt, double* rt, int32_t* perm);

/* CoR-UTV with power method (Algorithm 1; eqs. 4-9). ell = k + p.
 * psi: optional n x ell Gaussian test matrix; NULL -> or_gauss_matrix(seed, stream).
 * literal = 0: the power loop re-orthonormalises after each product
 *              (C1 = A X, Q1 = qr(C1), C2 = A^T Q1, X = qr(C2));
 * literal = 1: Algorithm 1 as printed (C1 = A C2, C2 = A^T C1, no QR inside).
 * Outputs (each optional, NULL to skip): U m x ell, T ell x ell, V n x ell,
 * perm[ell], Q1 m x ell, Q2 n x ell, D ell x ell. */
int or_corutv(const double* a, int64_t m, int64_t n, int64_t lda,
              int64_t k, int64_t p, int64_t q,
              const double* psi, uint64_t seed, uint32_t stream, int literal,
              double* u, double* t, double* v, int32_t* perm,
              double* q1, double* q2, double* d);

/* Shrinkage operator S_delta(x) = sgn(x) max(|x| - delta, 0), elementwise (Sec. 4). */
void or_shrink(int64_t count, const double* x, double delta, double* out);

/* Spectral norm ||M||_2 by power iteration on M^T M (start vector of ones,
 * stop when the Rayleigh quotient changes by <= 1e-15 relative, <= 2000 its). */
double or_norm2(const double* mat, int64_t m, int64_t n, int64_t ldm);

/* ALM-CoRUTV (Algorithm 2). M m x n. The low-rank step is CoR-UTV with
 * ell = 2k and q = 1 (Sec. 5.3), a fresh Gaussian test matrix per iteration
 * (stream j + 1 under `seed`), and the CoR-UTV thresholding operator
 * C_delta(B) = U(:,1:r) T(1:r,:) V^T with r = #{i : T_ii > delta}.
 * mu update: mu_{j+1} = min(rho mu_j, mu_bar). Stops after an iteration with
 * zeta = ||M - L - S||_F / ||M||_F < tol, or after max_iter iterations.
 * Histories (optional, length max_iter): zeta_j, r_j, mu_j used in iteration j.
 * L and S are m x n outputs. */
int or_rpca(const double* mat, int64_t m, int64_t n, int64_t ldm, int64_t k,
            double lambda, double mu0, double mu_bar, double rho, double tol,
            int max_iter, uint64_t seed,
            double* l_out, double* s_out, int* iters, double* zeta, int* rank,
            double* zeta_hist, int* rank_hist, double* mu_hist);

#ifdef __cplusplus
}
#endif

#endif
