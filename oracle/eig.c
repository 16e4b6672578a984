/*
 * Oracle: dense symmetric eigensolver. TEST INFRASTRUCTURE ONLY; see oracle.h.
 *
 * Method (Golub & Van Loan, Matrix Computations, Section 8.3):
 *  1. Householder tridiagonalisation T = Q0^T A Q0, each reflector applied
 *     to the trailing block as the symmetric rank-2 update A - v w^T - w v^T.
 *  2. Symmetric QR iteration on T: deflate negligible subdiagonal entries,
 *     then apply an implicit QR step with the Wilkinson shift to the lowest
 *     unreduced block, chasing the bulge with plane rotations. Rotations
 *     are applied to whole rows/columns of the dense T and accumulated in Q.
 * Eigenvalues are returned ascending with matching eigenvector columns.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define AT(M, i, j) (M)[(size_t)(i) * n + (j)]

/* Rotate rows r, r+1 of M (n x n): [row_r; row_r1] <- [c s; -s c][row_r; row_r1]. */
static void rot_rows(int n, double *M, int r, double c, double s) {
    for (int j = 0; j < n; ++j) {
        double a = AT(M, r, j), b = AT(M, r + 1, j);
        AT(M, r, j) = c * a + s * b;
        AT(M, r + 1, j) = -s * a + c * b;
    }
}

/* Rotate columns r, r+1 of M: [col_r, col_r1] <- [col_r, col_r1][c -s; s c]. */
static void rot_cols(int n, double *M, int r, double c, double s) {
    for (int i = 0; i < n; ++i) {
        double a = AT(M, i, r), b = AT(M, i, r + 1);
        AT(M, i, r) = c * a + s * b;
        AT(M, i, r + 1) = -s * a + c * b;
    }
}

static void tridiagonalise(int n, double *T, double *Q) {
    double *v = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    for (int j = 0; j + 2 < n; ++j) {
        int m = n - j - 1; /* length of the column below the diagonal */
        double xnorm2 = 0.0;
        for (int i = 0; i < m; ++i) xnorm2 += AT(T, j + 1 + i, j) * AT(T, j + 1 + i, j);
        double tail2 = xnorm2 - AT(T, j + 1, j) * AT(T, j + 1, j);
        if (tail2 == 0.0) continue; /* already in tridiagonal form here */
        double x0 = AT(T, j + 1, j);
        double alpha = (x0 >= 0.0) ? -sqrt(xnorm2) : sqrt(xnorm2);
        /* v = x - alpha e1 (sign chosen to avoid cancellation), beta = 2/(v.v). */
        for (int i = 0; i < m; ++i) v[i] = AT(T, j + 1 + i, j);
        v[0] -= alpha;
        double vv = 0.0;
        for (int i = 0; i < m; ++i) vv += v[i] * v[i];
        double beta = 2.0 / vv;
        /* p = beta A22 v; w = p - (beta p.v / 2) v; A22 -= v w^T + w v^T. */
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s += AT(T, j + 1 + i, j + 1 + l) * v[l];
            p[i] = beta * s;
        }
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += p[i] * v[i];
        for (int i = 0; i < m; ++i) w[i] = p[i] - 0.5 * beta * pv * v[i];
        for (int i = 0; i < m; ++i)
            for (int l = 0; l < m; ++l)
                AT(T, j + 1 + i, j + 1 + l) -= v[i] * w[l] + w[i] * v[l];
        /* The reflector maps column j below the diagonal to alpha e1. */
        AT(T, j + 1, j) = alpha;
        AT(T, j, j + 1) = alpha;
        for (int i = 1; i < m; ++i) {
            AT(T, j + 1 + i, j) = 0.0;
            AT(T, j, j + 1 + i) = 0.0;
        }
        /* Q <- Q (I - beta v v^T) on columns j+1 .. n-1. */
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += AT(Q, r, j + 1 + i) * v[i];
            for (int i = 0; i < m; ++i) AT(Q, r, j + 1 + i) -= beta * s * v[i];
        }
    }
    free(v);
    free(p);
    free(w);
}

/* One implicit symmetric QR step with Wilkinson shift on block lo..hi. */
static void qr_step(int n, double *T, double *Q, int lo, int hi) {
    double a = AT(T, hi - 1, hi - 1), b = AT(T, hi, hi - 1), c = AT(T, hi, hi);
    double dd = 0.5 * (a - c);
    double sgn = (dd >= 0.0) ? 1.0 : -1.0;
    double mu = c - b * b / (dd + sgn * hypot(dd, b));
    double x = AT(T, lo, lo) - mu;
    double z = AT(T, lo + 1, lo);
    for (int r = lo; r < hi; ++r) {
        double h = hypot(x, z);
        double cs = (h == 0.0) ? 1.0 : x / h;
        double sn = (h == 0.0) ? 0.0 : z / h;
        rot_rows(n, T, r, cs, sn);
        rot_cols(n, T, r, cs, sn);
        rot_cols(n, Q, r, cs, sn);
        if (r > lo) {
            /* The rotation annihilated the bulge at (r+1, r-1). */
            AT(T, r + 1, r - 1) = 0.0;
            AT(T, r - 1, r + 1) = 0.0;
        }
        if (r + 1 < hi) {
            x = AT(T, r + 1, r);
            z = AT(T, r + 2, r);
        }
    }
}

int orc_sym_eig(int n, const double *A, double *lam, double *Q) {
    double *T = (double *)malloc(sizeof(double) * n * n);
    memcpy(T, A, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) AT(Q, i, j) = (i == j) ? 1.0 : 0.0;
    tridiagonalise(n, T, Q);
    int status = 0, steps = 0, max_steps = 30 * n + 30;
    for (;;) {
        for (int i = 0; i + 1 < n; ++i) {
            double off = fabs(AT(T, i + 1, i));
            if (off <= DBL_EPSILON * (fabs(AT(T, i, i)) + fabs(AT(T, i + 1, i + 1)))) {
                AT(T, i + 1, i) = 0.0;
                AT(T, i, i + 1) = 0.0;
            }
        }
        int hi = n - 1;
        while (hi > 0 && AT(T, hi, hi - 1) == 0.0) --hi;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && AT(T, lo, lo - 1) != 0.0) --lo;
        if (++steps > max_steps) {
            status = 1;
            break;
        }
        qr_step(n, T, Q, lo, hi);
    }
    for (int i = 0; i < n; ++i) lam[i] = AT(T, i, i);
    /* Sort ascending (selection sort), permuting eigenvector columns alike. */
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int j = i + 1; j < n; ++j)
            if (lam[j] < lam[best]) best = j;
        if (best != i) {
            double t = lam[i];
            lam[i] = lam[best];
            lam[best] = t;
            for (int r = 0; r < n; ++r) {
                double q = AT(Q, r, i);
                AT(Q, r, i) = AT(Q, r, best);
                AT(Q, r, best) = q;
            }
        }
    }
    free(T);
    return status;
}
