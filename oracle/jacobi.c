/*
 * FP64 CPU oracle: Jacobi eigensolver and one-sided Jacobi SVD.
 *
 * Test infrastructure only.  Nothing on the product path links or calls this
 * file; it is built into a stand-alone shared object that the oracle's Python
 * module loads with ctypes.  It shares no code with the CUDA path.
 *
 * oracle_eigh_jacobi: cyclic two-sided Jacobi for a symmetric matrix, used for
 *   the EVD step H = V Sigma V^T of Algorithm 1 (step "Compute EVD of H").
 *   Rotations follow the classical symmetric Schur decomposition (Golub & Van
 *   Loan, Sec. 8.5): for a pivot (p,q), tau = (a_qq - a_pp) / (2 a_pq),
 *   t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c.
 *
 * oracle_svd_onesided: Hestenes one-sided Jacobi SVD of an m x n matrix
 *   (m >= n), an SVD route that does not pass through the polar factor; the
 *   tests use it to cross-check the polar route (W = U V^T, Definition 2.1).
 *
 * Both return results unsorted; ordering and sign conventions are applied in
 * the Python layer.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double offdiag_norm2(int n, const double *a) {
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    return s;
}

/* a: n x n row-major symmetric (overwritten; its diagonal holds eigenvalues on
 * return), v: n x n row-major eigenvectors as columns.  Returns the number of
 * sweeps used, or -1 if max_sweeps was reached without convergence. */
int oracle_eigh_jacobi(int n, double *a, double *v, double rel_tol, int max_sweeps) {
    memset(v, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    double fro2 = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) fro2 += a[k] * a[k];
    if (fro2 == 0.0) return 0;
    const double thr2 = rel_tol * rel_tol * fro2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (offdiag_norm2(n, a) <= thr2) return sweep;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J = identity except J_pp = J_qq = c, J_pq = s, J_qp = -s */
                for (int k = 0; k < n; ++k) {           /* columns p, q */
                    double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {           /* rows p, q */
                    double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                a[(size_t)p * n + q] = 0.0;
                a[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {           /* V <- V J */
                    double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    return offdiag_norm2(n, a) <= thr2 ? max_sweeps : -1;
}

/* One-sided Jacobi.  at: n x m row-major holding A^T (row j = column j of A),
 * overwritten with (U Sigma)^T; vt: n x n row-major holding V^T on return.
 * Returns sweeps used or -1. */
int oracle_svd_onesided(int m, int n, double *at, double *vt, double tol, int max_sweeps) {
    memset(vt, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) vt[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *cp = at + (size_t)p * m, *cq = at + (size_t)q * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int k = 0; k < m; ++k) {
                    alpha += cp[k] * cp[k];
                    beta += cq[k] * cq[k];
                    gamma += cp[k] * cq[k];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < m; ++k) {
                    double x = cp[k], y = cq[k];
                    cp[k] = c * x - s * y;
                    cq[k] = s * x + c * y;
                }
                double *vp = vt + (size_t)p * n, *vq = vt + (size_t)q * n;
                for (int k = 0; k < n; ++k) {
                    double x = vp[k], y = vq[k];
                    vp[k] = c * x - s * y;
                    vq[k] = s * x + c * y;
                }
            }
        }
        if (!rotated) return sweep;
    }
    return -1;
}
