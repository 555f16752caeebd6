// Blocked Householder QR of batched tall matrices (m >= n) with diag(R) >= 0: the QR
// fallback of Algorithm 1 (Appendix A.2) and the QR preprocessing of rectangular inputs
// (Section 4.1, rectangular matrices).
#pragma once
#include "ops.cuh"

namespace psvd {

// Panel shape for m rows: panel width nb (64 or 32) and cluster size cl (8 or 16 CTAs per
// matrix) such that each CTA's slab of ceil(m / cl) rows x nb columns fits in shared memory.
// Returns false when no shape fits (m too large for the cluster panel).
bool qr_shape(int m, int *nb, int *cl);

struct QrWS {
    int B = 0, m = 0, n = 0, nb = 0, cl = 0, npan = 0, ks = 1;
    long long ldm = 0, ldn = 0;
    float *UThi = nullptr, *UTlo = nullptr;   // [B][n][ldm] the matrix transposed, being factored
    float *YThi = nullptr, *YTlo = nullptr;   // [B][n][ldm] reflector j as row j (1 at j, 0 above)
    float *Yhi = nullptr, *Ylo = nullptr;     // [B][m][ldn] the same reflectors as columns
    float *QThi = nullptr, *QTlo = nullptr;   // [B][n][ldm] Q^T being accumulated
    float *tau = nullptr, *beta = nullptr;    // [B][n]
    float *Tm = nullptr;                      // [B][npan][nb][nb] compact-WY T of every panel
    float *Gpart = nullptr;                   // [B][cl][nb][nb] per-CTA partial Y^T Y of a panel
    float *Wp = nullptr;                      // [ks][B][nb][n] partial Y^T X of a panel (K split)
    float *W2hi = nullptr, *W2lo = nullptr;   // [B][n][nb] (op(T) Y^T X)^T
    int *skip = nullptr;                      // [B] 1 = matrix not factored (flag[b] == 0)
    unsigned *err = nullptr;

    template <class C>
    void carve(C &cv, int B_, int m_, int n_) {
        B = B_; m = m_; n = n_;
        if (!qr_shape(m, &nb, &cl)) { nb = 64; cl = 8; }
        npan = (n + nb - 1) / nb;
        ldm = pad_ld(m); ldn = pad_ld(n);
        ks = 8;
        const long long B64 = B, nm = (long long)n * ldm;
        UThi = cv.template take<float>(B64 * nm); UTlo = cv.template take<float>(B64 * nm);
        YThi = cv.template take<float>(B64 * nm); YTlo = cv.template take<float>(B64 * nm);
        Yhi = cv.template take<float>(B64 * m * ldn); Ylo = cv.template take<float>(B64 * m * ldn);
        QThi = cv.template take<float>(B64 * nm); QTlo = cv.template take<float>(B64 * nm);
        tau = cv.template take<float>(B64 * n); beta = cv.template take<float>(B64 * n);
        Tm = cv.template take<float>(B64 * npan * nb * nb);
        Gpart = cv.template take<float>(B64 * cl * nb * nb);
        Wp = cv.template take<float>((long long)ks * B64 * nb * n);
        W2hi = cv.template take<float>(B64 * n * nb); W2lo = cv.template take<float>(B64 * n * nb);
        skip = cv.template take<int>(B64);
        err = cv.template take<unsigned>(4);
    }
};

// Q R = A for the matrices with flag[b] != 0 (flag may be null: all), diag(R) >= 0.
// A: batch x m x n (user layout, read), Q: batch x m x n out (may alias A; written only for
// flagged matrices), R: batch x n x n out (upper triangular; may be null).  Asynchronous.
int qr_factor(const float *A, float *Q, float *R, const int *flag, QrWS &w, cudaStream_t st);

}  // namespace psvd
