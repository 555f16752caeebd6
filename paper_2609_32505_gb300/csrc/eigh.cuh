// Symmetric eigensolver for H = V Sigma V^T (the EVD of Algorithm 1).
#pragma once
#include <algorithm>

#include "ops.cuh"

namespace psvd {

constexpr int kWY = 128;   // reflectors per compact-WY block in the back-transform
constexpr int kBtSplit = 8; // largest K split of the back-transform's V^T Y products

struct EighWS {
    int B = 0, n = 0, nblk = 0, chunk = 0, nrp = 0;   // nrp: rows of Vh, padded to kWY
    long long ldn = 0;
    float *Aw = nullptr;          // working copy of H (n x n per matrix)
    float *Vh = nullptr;          // Householder vectors as rows (n x ldn), v_k[k+1] = 1
    float *tau = nullptr;         // [B][n]
    double *d = nullptr, *e = nullptr, *lam = nullptr;   // tridiagonal and eigenvalues [B][n]
    float *pbuf = nullptr;        // [groups][2][n]
    unsigned *bar = nullptr;      // [groups] barrier counters
    float *Vhi = nullptr, *Vlo = nullptr;      // Householder rows split (n x ldn)
    float *Yhi = nullptr, *Ylo = nullptr;      // Householder vectors as columns (n x ldn)
    float *VThi = nullptr, *VTlo = nullptr;    // current V^T split (n x ldn)
    float *S = nullptr;                        // V^T Y for a pair of blocks (n x 2 kWY), K-split slices
    float *S2hi = nullptr, *S2lo = nullptr;    // the pair's S2 split (n x 2 kWY)
    float *Tm = nullptr;                       // [B][nblk][kWY][kWY]
    float *Gm = nullptr;                       // [B][nblk][kWY][kWY]  Y^T Y per block
    float *Gab = nullptr;                      // [B][nblk/2][kWY][kWY]  Y_a^T Y_b per pair of blocks
    double *xs = nullptr;                      // inverse-iteration vectors, interleaved [n][chunk]
    float *xf = nullptr;                       // the normalized eigenvectors of T, interleaved [n][chunk]
    double *u0 = nullptr, *u1 = nullptr, *u2 = nullptr, *lm = nullptr;
    unsigned *piv = nullptr;            // pivot bits, [ceil(n/32)][chunk]
    unsigned *err = nullptr;
    int groups = 0;

    template <class C>
    void carve(C &cv, int B_, int n_, int groups_) {
        B = B_; n = n_; groups = groups_;
        ldn = pad_ld(n);
        nblk = n > 2 ? (n - 2 + kWY - 1) / kWY : 0;
        nrp = (int)round_up(n < 1 ? 1 : n, kWY);
        const long long B64 = B, nn = (long long)n * ldn, np = (long long)nrp * ldn;
        // inverse-iteration scratch holds whole matrices: n vectors x n entries each
        chunk = n * (int)std::max<long long>(1, std::min<long long>(B64, (1LL << 24) / ((long long)n * n)));
        Aw = cv.template take<float>(B64 * n * ldn);
        Vh = cv.template take<float>(B64 * np);
        tau = cv.template take<float>(B64 * n);
        d = cv.template take<double>(B64 * n);
        e = cv.template take<double>(B64 * n);
        lam = cv.template take<double>(B64 * n);
        pbuf = cv.template take<float>((long long)groups * 2 * ldn);
        bar = cv.template take<unsigned>((long long)groups * (2 * 160 + 1) + 1);   // release + arrival flags per group
        Vhi = cv.template take<float>(B64 * np);
        Vlo = cv.template take<float>(B64 * np);
        Yhi = cv.template take<float>(B64 * nn);
        Ylo = cv.template take<float>(B64 * nn);
        VThi = cv.template take<float>(B64 * nn);
        VTlo = cv.template take<float>(B64 * nn);
        S = cv.template take<float>(kBtSplit * B64 * n * 2 * kWY);
        S2hi = cv.template take<float>(B64 * n * 2 * kWY);
        S2lo = cv.template take<float>(B64 * n * 2 * kWY);
        Tm = cv.template take<float>(B64 * (nblk > 0 ? nblk : 1) * kWY * kWY);
        Gm = cv.template take<float>(B64 * (nblk > 0 ? nblk : 1) * kWY * kWY);
        Gab = cv.template take<float>(B64 * (nblk > 1 ? nblk / 2 : 1) * kWY * kWY);
        xs = cv.template take<double>((long long)n * chunk);
        xf = cv.template take<float>((long long)n * chunk);
        u0 = cv.template take<double>((long long)n * chunk);
        u1 = cv.template take<double>((long long)n * chunk);
        u2 = cv.template take<double>((long long)n * chunk);
        lm = cv.template take<double>((long long)n * chunk);
        piv = cv.template take<unsigned>((long long)((n + 31) / 32) * chunk);
        err = cv.template take<unsigned>(4);
    }
};

int eigh_groups(int B, int n);

// Eigendecomposition of the symmetric matrices Hs (B x n x n, FP32, full storage).
// Writes eigenvalues descending to S (B x n, may be null) and V^T split into
// ws.VThi / ws.VTlo (rows = eigenvectors, largest-|.| entry positive), and V^T to
// VT (B x n x n, may be null).
int eigh_forward(const float *Hs, float *S, float *VT, EighWS &ws, cudaStream_t st);

}  // namespace psvd
