/*
 * Plain FP64 CPU oracle for CoR-UTV (Algorithm 1, eqs. 4-9) and ALM-CoRUTV
 * (Algorithm 2) of Kaloorazi & de Lamare.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path. Shares nothing with
 * the CUDA implementation.
 *
 * Every routine is the textbook definition written out with plain loops:
 * triple-loop products, Householder reflections, recomputed column norms.
 * OpenMP only splits independent output rows or columns across threads; the
 * summation order of each output element is the plain ascending loop, so
 * results do not depend on the thread count.
 */
#include "corutv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box      */
/* built from two 32x32->64 multiplications, with a Weyl-sequence key       */
/* schedule between rounds.                                                 */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_gauss_entry(uint64_t seed, uint32_t stream, uint32_t i, uint32_t j) {
    const uint32_t ctr[4] = {i, j, stream, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    const uint64_t a = (((uint64_t)w[0] << 32) | w[1]) >> 11; /* 53 random bits */
    const uint64_t b = (((uint64_t)w[2] << 32) | w[3]) >> 11;
    const double two_m53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    const double u1 = ((double)a + 1.0) * two_m53;   /* (0, 1] */
    const double u2 = (double)b * two_m53;           /* [0, 1) */
    const double two_pi = 6.283185307179586476925286766559;
    return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

void or_gauss_matrix(uint64_t seed, uint32_t stream, int64_t n, int64_t ell, double* psi) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < ell; ++j)
            psi[i * ell + j] = or_gauss_entry(seed, stream, (uint32_t)i, (uint32_t)j);
}

/* ------------------------------------------------------------------------ */
/* Plain products.                                                          */
/* ------------------------------------------------------------------------ */

/* C (m x l) = A (m x n, row stride lda) * X (n x l, row stride l). */
static void mm_ax(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda,
                  const double* x, double* c) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double* ci = c + i * l;
        for (int64_t j = 0; j < l; ++j) ci[j] = 0.0;
        const double* ai = a + i * lda;
        for (int64_t t = 0; t < n; ++t) {
            const double av = ai[t];
            const double* xt = x + t * l;
            for (int64_t j = 0; j < l; ++j) ci[j] += av * xt[j];
        }
    }
}

/* C (n x l) = A^T (n x m) * Y (m x l); A is m x n with row stride lda. Each
 * C[t][j] is summed over i = 0..m-1 in ascending order. */
static void mm_aty(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda,
                   const double* y, double* c) {
    const int64_t blk = 32;
#pragma omp parallel for schedule(static)
    for (int64_t c0 = 0; c0 < n; c0 += blk) {
        const int64_t c1 = imin(n, c0 + blk);
        for (int64_t t = c0; t < c1; ++t)
            for (int64_t j = 0; j < l; ++j) c[t * l + j] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double* ai = a + i * lda;
            const double* yi = y + i * l;
            for (int64_t t = c0; t < c1; ++t) {
                const double av = ai[t];
                double* ct = c + t * l;
                for (int64_t j = 0; j < l; ++j) ct[j] += av * yi[j];
            }
        }
    }
}

/* C (p x l) = X^T (p x m) * Y (m x l); X m x p, Y m x l, both row-major. */
static void mm_xty(int64_t m, int64_t p, int64_t l, const double* x, const double* y, double* c) {
    for (int64_t s = 0; s < p * l; ++s) c[s] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t s = 0; s < p; ++s) {
            const double xv = x[i * p + s];
            for (int64_t j = 0; j < l; ++j) c[s * l + j] += xv * y[i * l + j];
        }
}

/* C (m x l) = X (m x p) * Y (p x l). */
static void mm_xy(int64_t m, int64_t p, int64_t l, const double* x, const double* y, double* c) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < l; ++j) c[i * l + j] = 0.0;
        for (int64_t s = 0; s < p; ++s) {
            const double xv = x[i * p + s];
            for (int64_t j = 0; j < l; ++j) c[i * l + j] += xv * y[s * l + j];
        }
    }
}

void or_gemm_ax(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda, const double* x,
               double* c) {
    mm_ax(m, n, l, a, lda, x, c);
}

void or_gemm_aty(int64_t m, int64_t n, int64_t l, const double* a, int64_t lda, const double* y,
                 double* c) {
    mm_aty(m, n, l, a, lda, y, c);
}

/* ------------------------------------------------------------------------ */
/* Householder reflections (Golub & Van Loan, Sec. 5.1).                    */
/* For the column x = w[r0.., col] of the row-major work array w (stride    */
/* ldw), build H = I - tau v v^T with v[0] = 1 such that H x = beta e1;     */
/* v[1..] overwrites x[1..], beta overwrites x[0].                          */
/* ------------------------------------------------------------------------ */
static double house(int64_t len, double* w, int64_t ldw, int64_t r0, int64_t col) {
    double alpha = w[r0 * ldw + col];
    double xnorm2 = 0.0;
    for (int64_t i = 1; i < len; ++i) {
        const double e = w[(r0 + i) * ldw + col];
        xnorm2 += e * e;
    }
    if (xnorm2 == 0.0) return 0.0; /* H = I, beta = alpha */
    const double norm = sqrt(alpha * alpha + xnorm2);
    const double beta = alpha >= 0.0 ? -norm : norm;
    const double tau = (beta - alpha) / beta;
    const double scale = 1.0 / (alpha - beta);
    for (int64_t i = 1; i < len; ++i) w[(r0 + i) * ldw + col] *= scale;
    w[r0 * ldw + col] = beta;
    return tau;
}

/* Apply H (reflector stored in column `vcol` of w, rows r0..r0+len-1, with
 * implicit v[0] = 1) to columns [c0, c1) of the array z (row stride ldz),
 * rows r0..r0+len-1. */
static void apply_house(int64_t len, const double* w, int64_t ldw, int64_t vcol, double tau,
                        double* z, int64_t ldz, int64_t r0, int64_t c0, int64_t c1) {
    if (tau == 0.0) return;
    for (int64_t c = c0; c < c1; ++c) {
        double dot = z[r0 * ldz + c];
        for (int64_t i = 1; i < len; ++i) dot += w[(r0 + i) * ldw + vcol] * z[(r0 + i) * ldz + c];
        const double f = tau * dot;
        z[r0 * ldz + c] -= f;
        for (int64_t i = 1; i < len; ++i) z[(r0 + i) * ldz + c] -= f * w[(r0 + i) * ldw + vcol];
    }
}

/* Form the first l columns of Q = H_0 H_1 ... H_{l-1} (m x l) from the
 * reflectors stored below the diagonal of w (m x l, stride l). */
static void form_q(int64_t m, int64_t l, const double* w, const double* tau, double* q) {
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < l; ++j) q[i * l + j] = (i == j) ? 1.0 : 0.0;
    for (int64_t j = l - 1; j >= 0; --j)
        apply_house(m - j, w, l, j, tau[j], q, l, j, j, l);
}

/* Make diag(R) >= 0: C = Q R = (Q S)(S R) with S = diag(+-1). */
static void fix_signs(int64_t rows_q, int64_t l, double* q, double* r) {
    for (int64_t j = 0; j < l; ++j) {
        if (r[j * l + j] < 0.0) {
            for (int64_t c = 0; c < l; ++c) r[j * l + c] = -r[j * l + c];
            for (int64_t i = 0; i < rows_q; ++i) q[i * l + j] = -q[i * l + j];
        }
    }
}

int or_qr(int64_t m, int64_t l, const double* c, int64_t ldc, double* q, double* r) {
    if (m < l || l < 1 || ldc < l) return OR_EINVAL;
    double* w = (double*)malloc(sizeof(double) * (size_t)(m * l));
    double* tau = (double*)malloc(sizeof(double) * (size_t)l);
    if (!w || !tau) { free(w); free(tau); return OR_ENOMEM; }
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < l; ++j) w[i * l + j] = c[i * ldc + j];
    for (int64_t j = 0; j < l; ++j) {
        tau[j] = house(m - j, w, l, j, j);
        apply_house(m - j, w, l, j, tau[j], w, l, j, j + 1, l);
    }
    for (int64_t i = 0; i < l; ++i)
        for (int64_t j = 0; j < l; ++j) r[i * l + j] = (j >= i) ? w[i * l + j] : 0.0;
    form_q(m, l, w, tau, q);
    fix_signs(m, l, q, r);
    free(w);
    free(tau);
    return OR_OK;
}

int or_qrcp(int64_t l, const double* d, double* qt, double* rt, int32_t* perm) {
    if (l < 1) return OR_EINVAL;
    double* w = (double*)malloc(sizeof(double) * (size_t)(l * l));
    double* tau = (double*)malloc(sizeof(double) * (size_t)l);
    if (!w || !tau) { free(w); free(tau); return OR_ENOMEM; }
    memcpy(w, d, sizeof(double) * (size_t)(l * l));
    for (int64_t j = 0; j < l; ++j) perm[j] = (int32_t)j;
    for (int64_t j = 0; j < l; ++j) {
        /* recomputed residual norms of the trailing columns (no downdating) */
        int64_t piv = j;
        double best = -1.0;
        for (int64_t c = j; c < l; ++c) {
            double s = 0.0;
            for (int64_t i = j; i < l; ++i) s += w[i * l + c] * w[i * l + c];
            const double nrm = sqrt(s);
            if (nrm > best) { best = nrm; piv = c; }
        }
        if (piv != j) {
            for (int64_t i = 0; i < l; ++i) {
                const double tmp = w[i * l + j];
                w[i * l + j] = w[i * l + piv];
                w[i * l + piv] = tmp;
            }
            const int32_t tp = perm[j];
            perm[j] = perm[piv];
            perm[piv] = tp;
        }
        tau[j] = house(l - j, w, l, j, j);
        apply_house(l - j, w, l, j, tau[j], w, l, j, j + 1, l);
    }
    for (int64_t i = 0; i < l; ++i)
        for (int64_t j = 0; j < l; ++j) rt[i * l + j] = (j >= i) ? w[i * l + j] : 0.0;
    form_q(l, l, w, tau, qt);
    fix_signs(l, l, qt, rt);
    free(w);
    free(tau);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* CoR-UTV (Sec. 3.1, Algorithm 1).                                         */
/* ------------------------------------------------------------------------ */
int or_corutv(const double* a, int64_t m, int64_t n, int64_t lda,
              int64_t k, int64_t p, int64_t q,
              const double* psi, uint64_t seed, uint32_t stream, int literal,
              double* u, double* t, double* v, int32_t* perm_out,
              double* q1_out, double* q2_out, double* d_out) {
    const int64_t l = k + p;
    /* k <= ell < min(m, n) (Sec. 3.1) */
    if (k < 1 || p < 0 || q < 0 || l >= imin(m, n) || lda < n) return OR_EINVAL;
    const size_t ml = (size_t)(m * l), nl = (size_t)(n * l), ll = (size_t)(l * l);
    double* x = (double*)malloc(sizeof(double) * nl);
    double* c1 = (double*)malloc(sizeof(double) * ml);
    double* c2 = (double*)malloc(sizeof(double) * nl);
    double* q1 = (double*)malloc(sizeof(double) * ml);
    double* q2 = (double*)malloc(sizeof(double) * nl);
    double* r = (double*)malloc(sizeof(double) * ll);
    double* w = (double*)malloc(sizeof(double) * ml);
    double* d = (double*)malloc(sizeof(double) * ll);
    double* qt = (double*)malloc(sizeof(double) * ll);
    double* rt = (double*)malloc(sizeof(double) * ll);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)l);
    int status = OR_OK;
    if (!x || !c1 || !c2 || !q1 || !q2 || !r || !w || !d || !qt || !rt || !perm) {
        status = OR_ENOMEM;
        goto done;
    }
    /* Step 1: Gaussian test matrix (eq. 4's Psi; Algorithm 1 draws it as C2). */
    if (psi) memcpy(x, psi, sizeof(double) * nl);
    else or_gauss_matrix(seed, stream, n, l, x);

    if (literal) {
        /* Algorithm 1 as printed: i = 1..q+1 of C1 = A C2, C2 = A^T C1. */
        for (int64_t it = 0; it <= q; ++it) {
            mm_ax(m, n, l, a, lda, x, c1);      /* eq. 4 */
            mm_aty(m, n, l, a, lda, c1, c2);    /* eq. 5 */
            memcpy(x, c2, sizeof(double) * nl);
        }
        if ((status = or_qr(m, l, c1, l, q1, r))) goto done;
        if ((status = or_qr(n, l, c2, l, q2, r))) goto done;
    } else {
        /* Same loop with each sketch re-orthonormalised before it is used;
         * in exact arithmetic Q1 and Q2 are unchanged (QR with diag(R) > 0
         * is invariant under right-multiplication by such an R). */
        for (int64_t it = 0; it <= q; ++it) {
            mm_ax(m, n, l, a, lda, x, c1);      /* eq. 4 */
            if ((status = or_qr(m, l, c1, l, q1, r))) goto done;
            mm_aty(m, n, l, a, lda, q1, c2);    /* eq. 5 with C1 -> Q1 */
            if (it < q && (status = or_qr(n, l, c2, l, x, r))) goto done;
        }
        if ((status = or_qr(n, l, c2, l, q2, r))) goto done;
    }
    /* eq. 7: D = Q1^T A Q2 */
    mm_ax(m, n, l, a, lda, q2, w);
    mm_xty(m, l, l, q1, w, d);
    /* eq. 8: D P = Qt Rt */
    if ((status = or_qrcp(l, d, qt, rt, perm))) goto done;
    /* eq. 9: U = Q1 Qt, T = Rt, V = Q2 P */
    if (u) mm_xy(m, l, l, q1, qt, u);
    if (t) memcpy(t, rt, sizeof(double) * ll);
    if (v)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < l; ++j) v[i * l + j] = q2[i * l + perm[j]];
    if (perm_out) memcpy(perm_out, perm, sizeof(int32_t) * (size_t)l);
    if (q1_out) memcpy(q1_out, q1, sizeof(double) * ml);
    if (q2_out) memcpy(q2_out, q2, sizeof(double) * nl);
    if (d_out) memcpy(d_out, d, sizeof(double) * ll);
done:
    free(x); free(c1); free(c2); free(q1); free(q2); free(r); free(w);
    free(d); free(qt); free(rt); free(perm);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Robust PCA (Sec. 4, Algorithm 2).                                        */
/* ------------------------------------------------------------------------ */
void or_shrink(int64_t count, const double* x, double delta, double* out) {
    for (int64_t i = 0; i < count; ++i) {
        const double mag = fabs(x[i]) - delta;
        const double sgn = (x[i] > 0.0) ? 1.0 : ((x[i] < 0.0) ? -1.0 : 0.0);
        out[i] = mag > 0.0 ? sgn * mag : 0.0;
    }
}

double or_norm2(const double* mat, int64_t m, int64_t n, int64_t ldm) {
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    double* mv = (double*)malloc(sizeof(double) * (size_t)m);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    if (!v || !mv || !w) { free(v); free(mv); free(w); return -1.0; }
    for (int64_t j = 0; j < n; ++j) v[j] = 1.0 / sqrt((double)n);
    double lam = 0.0;
    for (int it = 0; it < 2000; ++it) {
        mm_ax(m, n, 1, mat, ldm, v, mv);
        mm_aty(m, n, 1, mat, ldm, mv, w);
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += w[j] * w[j];
        const double nw = sqrt(s); /* = lambda_max estimate of M^T M */
        if (nw == 0.0) { lam = 0.0; break; }
        for (int64_t j = 0; j < n; ++j) v[j] = w[j] / nw;
        const double done = fabs(nw - lam) <= 1e-15 * nw;
        lam = nw;
        if (done) break;
    }
    free(v); free(mv); free(w);
    return sqrt(lam);
}

int or_rpca(const double* mat, int64_t m, int64_t n, int64_t ldm, int64_t k,
            double lambda, double mu0, double mu_bar, double rho, double tol,
            int max_iter, uint64_t seed,
            double* l_out, double* s_out, int* iters, double* zeta, int* rank,
            double* zeta_hist, int* rank_hist, double* mu_hist) {
    const int64_t l = 2 * k; /* ell = 2k (Sec. 5.3) */
    if (k < 1 || l >= imin(m, n) || ldm < n || max_iter < 1 || !l_out || !s_out) return OR_EINVAL;
    const size_t mn = (size_t)(m * n);
    double* y = (double*)calloc(mn, sizeof(double));
    double* b = (double*)malloc(sizeof(double) * mn);
    double* u = (double*)malloc(sizeof(double) * (size_t)(m * l));
    double* t = (double*)malloc(sizeof(double) * (size_t)(l * l));
    double* v = (double*)malloc(sizeof(double) * (size_t)(n * l));
    double* tv = (double*)malloc(sizeof(double) * (size_t)(l * n)); /* T(1:r,:) V^T */
    int status = OR_OK;
    if (!y || !b || !u || !t || !v || !tv) { status = OR_ENOMEM; goto done; }
    double mnorm2 = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) mnorm2 += mat[i * ldm + j] * mat[i * ldm + j];
    const double mnorm = sqrt(mnorm2);
    double mu = mu0;
    for (int64_t e = 0; e < (int64_t)mn; ++e) s_out[e] = 0.0; /* S_0 = 0, Y_0 = 0 */
    int j = 0;
    double zj = 0.0;
    int rj = 0;
    for (j = 0; j < max_iter; ++j) {
        const double inv_mu = 1.0 / mu;
        /* B = M - S_j + Y_j / mu_j */
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < n; ++c)
                b[i * n + c] = mat[i * ldm + c] - s_out[i * n + c] + y[i * n + c] * inv_mu;
        /* L_{j+1} = C_{1/mu_j}(B) */
        status = or_corutv(b, m, n, n, k, l - k, 1, NULL, seed, (uint32_t)(j + 1), 0,
                           u, t, v, NULL, NULL, NULL, NULL);
        if (status) goto done;
        rj = 0;
        for (int64_t i = 0; i < l; ++i)
            if (t[i * l + i] > inv_mu) ++rj;
        /* tv (r x n) = T(1:r, :) V^T */
        for (int64_t s = 0; s < rj; ++s)
            for (int64_t c = 0; c < n; ++c) {
                double acc = 0.0;
                for (int64_t h = 0; h < l; ++h) acc += t[s * l + h] * v[c * l + h];
                tv[s * n + c] = acc;
            }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < n; ++c) {
                double acc = 0.0;
                for (int64_t s = 0; s < rj; ++s) acc += u[i * l + s] * tv[s * n + c];
                l_out[i * n + c] = acc;
            }
        /* S_{j+1} = S_{lambda/mu_j}(M - L_{j+1} + Y_j / mu_j) */
        const double delta = lambda * inv_mu;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < n; ++c) {
                const double xv = mat[i * ldm + c] - l_out[i * n + c] + y[i * n + c] * inv_mu;
                double sv;
                or_shrink(1, &xv, delta, &sv);
                s_out[i * n + c] = sv;
            }
        /* Y_{j+1} = Y_j + mu_j (M - L_{j+1} - S_{j+1}); zeta from the same residual */
        double res2 = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t c = 0; c < n; ++c) {
                const double rres = mat[i * ldm + c] - l_out[i * n + c] - s_out[i * n + c];
                y[i * n + c] += mu * rres;
                res2 += rres * rres;
            }
        zj = sqrt(res2) / mnorm;
        if (zeta_hist) zeta_hist[j] = zj;
        if (rank_hist) rank_hist[j] = rj;
        if (mu_hist) mu_hist[j] = mu;
        /* continuation, capped at mu_bar */
        mu = fmin(rho * mu, mu_bar);
        if (zj < tol) { ++j; break; }
    }
    if (iters) *iters = j;
    if (zeta) *zeta = zj;
    if (rank) *rank = rj;
done:
    free(y); free(b); free(u); free(t); free(v); free(tv);
    return status;
}
