// Thin SVD by Algorithm 1: polar factor W, H = (W^T M)_sym, EVD H = V Sigma V^T,
// U = W V, and the QR fallback of Appendix A.2 when a column norm of U is off 1.
//
// Mixed precision: BF16/TF32 polynomial steps leave W rotated inside low-sigma
// subspaces by angles the orthogonality residual cannot see.  The FP32-accurate
// product Hhat = W^T M keeps that rotation in its skew part; in the eigenbasis of
// sym(Hhat) = V Sigma V^T it reads V^T Hhat V = Sigma + K with K skew, and the
// first-order SVD of Sigma + K is U_e = I + X, V_e = I - X with
// X_ij = K_ij / (sigma_i + sigma_j) -- the same eigenbasis Lyapunov solve the
// paper's backward uses (Proposition D.3), with no spectral-gap denominators.
// The factors become U = W V E, V^T <- E V^T with E = I + X + X^2/2.
#include <cmath>
#include <cstring>

#include <vector>

#include "eigh.cuh"
#include "polar.cuh"
#include "qr.cuh"

namespace psvd {

// U = W V: stores U (user layout) and accumulates column sums of squares.
struct EpiColNorm {
    int m, n;
    float *U;
    float *colss;   // [B][n]
    struct Acc {};
    PSVD_DEV void begin(Acc &) const {}
    PSVD_DEV void chunk(Acc &, int b, int r, int c0, int, int, float (&v)[16]) const {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            const float x = (r < m && c < n) ? v[i] : 0.f;
            if (r < m && c < n) U[(long long)b * m * n + (long long)r * n + c] = x;
            const float s = warp_sum(x * x);
            if ((threadIdx.x & 31) == 0 && c < n && s != 0.f) atomicAdd(&colss[(long long)b * n + c], s);
        }
    }
    PSVD_DEV void finish(Acc &, int, int, int) const {}
};

// skip: matrices the caller recomputes anyway (a learned schedule that fell back), whose
// not-converged U must not start the QR fallback
__global__ void qr_flag_kernel(const float *colss, int n, double eps_qr, const int *skip, int *flag, int *any) {
    const int b = blockIdx.x;
    if (skip && skip[b]) {
        if (threadIdx.x == 0) flag[b] = 0;
        return;
    }
    int bad = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double nr = sqrt((double)colss[(long long)b * n + j]);
        bad |= !(fabs(nr - 1.0) <= eps_qr);
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        flag[b] = bad;
        if (bad) atomicAdd(any, 1);
    }
}

// ------------------------------------------------------------ QR fallback
// Householder QR of U (m x n) kept transposed (row j of UT = column j of U), one
// group barrier per column, then Q = H_0 ... H_{n-1} [I; 0] column by column and the
// sign of column j set so that R_jj >= 0.  Only matrices with flag[b] run.
struct QrParams {
    float *U;          // user layout, overwritten with Q for flagged matrices
    float *UT;         // [B][n][m]
    float *tau, *beta; // [B][n]
    const int *flag;
    unsigned *bar, *err;
    int B, m, n, g;
    uint32_t spin;     // poll bound of the grid barrier
};

__global__ void __launch_bounds__(256) qr_householder_kernel(QrParams P) {
    __shared__ double red[32];
    const int m = P.m, n = P.n;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * nw + warp, GW = P.g * nw;
    unsigned nbar = 0;
    for (int b = 0; b < P.B; ++b) {
        if (!P.flag[b]) continue;                 // uniform across the grid
        float *UT = P.UT + (long long)b * n * m;
        const float *U = P.U + (long long)b * m * n;
        for (int c = gw; c < n; c += GW)
            for (int r = lane; r < m; r += 32) UT[(long long)c * m + r] = U[(long long)r * n + c];
        group_barrier(P.bar, (++nbar) * P.g, P.err, P.spin);
        for (int j = 0; j < n; ++j) {
            float *x = UT + (long long)j * m;
            // v_j from column j (rows j..m-1), computed redundantly by every CTA
            double s2 = 0.0;
            for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) s2 += (double)x[r] * x[r];
            s2 = block_sum(s2, red);
            const double alpha = x[j];
            double beta, tau, scal;
            if (s2 == 0.0) { beta = alpha; tau = 0.0; scal = 0.0; }
            else {
                beta = -copysign(sqrt(alpha * alpha + s2), alpha);
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            // apply H_j = I - tau v v^T to owned columns c > j
            for (int c = gw; c < n; c += GW) {
                if (c <= j) continue;
                float *y = UT + (long long)c * m;
                double dot = lane == 0 ? (double)y[j] : 0.0;
                for (int r = j + 1 + lane; r < m; r += 32) dot += (double)x[r] * scal * y[r];
                dot = warp_sum(dot);
                const float f = (float)(tau * dot);
                if (lane == 0) y[j] -= f;
                for (int r = j + 1 + lane; r < m; r += 32) y[r] -= f * (float)(x[r] * scal);
            }
            group_barrier(P.bar, (++nbar) * P.g, P.err, P.spin);
            if (blockIdx.x == 0) {
                // store v_j in place (v_j[j] = 1 implicit) once every CTA has used x
                for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) x[r] = (float)(x[r] * scal);
                if (threadIdx.x == 0) {
                    P.tau[(long long)b * n + j] = (float)tau;
                    P.beta[(long long)b * n + j] = (float)beta;
                }
            }
            group_barrier(P.bar, (++nbar) * P.g, P.err, P.spin);
        }
    }
}

// Q column c = H_0 ... H_{n-1} e_c, sign-fixed; one warp per column.
__global__ void qr_form_q_kernel(QrParams P, float *qbuf) {
    const int m = P.m, n = P.n;
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long gwarp = (long long)blockIdx.x * nw + warp;
    const int b = blockIdx.y;
    if (!P.flag[b] || gwarp >= n) return;
    const int c = (int)gwarp;
    const float *UT = P.UT + (long long)b * n * m;
    float *q = qbuf + ((long long)b * n + c) * m;
    for (int r = lane; r < m; r += 32) q[r] = r == c ? 1.f : 0.f;
    __syncwarp();
    for (int j = (c < n - 1 ? c : n - 1); j >= 0; --j) {
        const float tau = P.tau[(long long)b * n + j];
        if (tau == 0.f) continue;
        const float *v = UT + (long long)j * m;
        float dot = lane == 0 ? q[j] : 0.f;
        for (int r = j + 1 + lane; r < m; r += 32) dot += v[r] * q[r];
        dot = warp_sum(dot);
        const float f = tau * dot;
        if (lane == 0) q[j] -= f;
        for (int r = j + 1 + lane; r < m; r += 32) q[r] -= f * v[r];
        __syncwarp();
    }
    const float sg = P.beta[(long long)b * n + c] < 0.f ? -1.f : 1.f;
    float *U = P.U + (long long)b * m * n;
    for (int r = lane; r < m; r += 32) U[(long long)r * n + c] = sg * q[r];
}

// ------------------------------------------------------------ mixed-precision correction
__global__ void skewT_kernel(const float *Hraw, int n, float *hi, float *lo, long long ld, unsigned *kmax) {
    // K^T = -skew(Hraw) stored as the B operand of V^T K (B[j][k] = K[k][j]); the largest
    // |K_ij| of each matrix goes to kmax (float bits, one atomic per block)
    __shared__ unsigned wmax[8];
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    unsigned bits = 0;
    if (i < n && j < n) {
        const float *h = Hraw + (long long)b * n * n;
        const float kt = 0.5f * (h[(long long)j * n + i] - h[(long long)i * n + j]);
        float hh, ll;
        split_tf32(kt, hh, ll);
        hi[(long long)b * n * ld + (long long)i * ld + j] = hh;
        lo[(long long)b * n * ld + (long long)i * ld + j] = ll;
        bits = __float_as_uint(fabsf(kt));
    }
    const int t = threadIdx.y * 16 + threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    if ((t & 31) == 0) wmax[t >> 5] = bits;
    __syncthreads();
    if (t == 0) {
        unsigned m = wmax[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) m = max(m, wmax[w]);
        if (m) atomicMax(&kmax[b], m);
    }
}

// Precision of the correction's products, per matrix.  TF32 rounds each operand to 2^-11
// relative, so a product whose result is a small correction can drop the split when its
// absolute error stays below FP32 resolution:
//  which = 0 (V^T K and (V^T K) V, then X = Ktilde / (s_i + s_j)): TF32 when
//    2^-11 max|K| / (2 s_min) <= 2^-21, the bound of the error this puts into X;
//  which = 1 (X V^T, added to V^T): TF32 when 2^-11 max|X| <= 2^-23.
// Otherwise (or for a non-finite bound) the split-TF32 products are kept.
__global__ void corr_prec_kernel(const unsigned *vmax, const float *S, int n, int B, int which, int *prec) {
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float v = __uint_as_float(vmax[b]);
        bool tf32;
        if (which == 0) {
            const float smin = S[(long long)b * n + n - 1];
            tf32 = smin > 0.f && v * 0x1p-11f <= 0x1p-21f * 2.f * smin;
        } else {
            tf32 = v * 0x1p-11f <= 0x1p-23f;
        }
        prec[b] = tf32 ? PREC_TF32 : PREC_TF32X3;
    }
}

// X = Ktilde / (s_i + s_j) (skew); writes X split into TF32 hi/lo (the first-order
// product X V^T is taken in split-TF32) and -X_hi (B operand of X^2).
// Also records max |X_ij| per matrix in xmax (float bits; the values are >= 0, and a NaN
// compares above every finite value, so it forces the fallback).
// One block per 32 x 32 tile (32 x 8 threads): the tile of Ktilde and its mirror tile are
// staged in shared memory, so both reads are coalesced; the tile's largest |X| is reduced in
// the block and recorded with one atomic.
__global__ void __launch_bounds__(256) corr_x_kernel(const float *Kt, const float *S, int n, float *X, float *Xlo,
                                                     float *Xneg, long long ld, unsigned *xmax) {
    __shared__ float tk[32][33], tm[32][33];
    __shared__ unsigned wmax[8];
    const int b = blockIdx.z, i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float *K = Kt + (long long)b * n * n;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        tk[r][tx] = (i0 + r < n && j0 + tx < n) ? K[(long long)(i0 + r) * n + j0 + tx] : 0.f;
        tm[r][tx] = (j0 + r < n && i0 + tx < n) ? K[(long long)(j0 + r) * n + i0 + tx] : 0.f;
    }
    __syncthreads();
    unsigned bits = 0;
    const int j = j0 + tx;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r;
        if (i < n && j < n) {
            const float si = S[(long long)b * n + i], sj = S[(long long)b * n + j];
            const float den = si + sj;
            const float k = 0.5f * (tk[r][tx] - tm[tx][r]);        // exact skew part
            const float x = den > 0.f ? k / den : 0.f;
            float xh, xl;
            split_tf32(x, xh, xl);
            const long long o = (long long)b * n * ld + (long long)i * ld + j;
            X[o] = xh;
            Xlo[o] = xl;
            Xneg[o] = -xh;
            bits = max(bits, __float_as_uint(fabsf(x)));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, o));
    if (tx == 0) wmax[ty] = bits;
    __syncthreads();
    if (ty == 0 && tx == 0) {
        unsigned m = wmax[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) m = max(m, wmax[w]);
        if (m) atomicMax(&xmax[b], m);
    }
}

// ------------------------------------------------------------ reconstruction check
// ||A - U Sigma V^T||_F^2 = E_z ||(A - U Sigma V^T) z||^2 for Rademacher z (Hutchinson's
// estimator); kProbes probes give an estimate whose relative spread is about
// sqrt(2 / (kProbes * r_eff)), r_eff the effective rank of the error (high for the dense
// second-order error the mixed path leaves).  Sums are float-float, so the difference
// A z - U (Sigma V^T z) keeps ~1e-14 relative accuracy where the error is ~1e-6.
constexpr int kProbes = 8;

// Signs of the kProbes probes at column j: bits of a 32-bit integer hash of j.
PSVD_DEV unsigned probe_hash(int j) {
    unsigned h = (unsigned)j * 0x9E3779B1u + 0x632BE5ABu;
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h;
}
PSVD_DEV float probe_sign(unsigned h, int p) { return (h >> p) & 1u ? -1.f : 1.f; }

// Y[b][p][i] = sigma_i (V^T z_p)_i: one warp per row i of V^T.
__global__ void probe_vt_kernel(const float *VT, const float *S, int n, float *Y) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const float *v = VT + ((long long)b * n + i) * n;
    ff acc[kProbes];
#pragma unroll
    for (int p = 0; p < kProbes; ++p) acc[p] = ff_zero();
    for (int j = lane; j < n; j += 32) {
        const float x = v[j];
        const unsigned h = probe_hash(j);
#pragma unroll
        for (int p = 0; p < kProbes; ++p) acc[p] = ff_add(acc[p], ff{probe_sign(h, p) * x, 0.f});
    }
#pragma unroll
    for (int p = 0; p < kProbes; ++p) acc[p] = warp_sum(acc[p]);
    if (lane == 0) {
        const float sg = S[(long long)b * n + i];
#pragma unroll
        for (int p = 0; p < kProbes; ++p) Y[((long long)b * kProbes + p) * n + i] = sg * __fadd_rn(acc[p].hi, acc[p].lo);
    }
}

// Per row r: res_p = A[r, :] z_p - U[r, :] Y[p, :]; sums[b] += (||A[r, :]||^2, sum_p res_p^2),
// one warp per row, reduced over the block before one atomic pair.
__global__ void __launch_bounds__(256) probe_resid_kernel(const float *A, const float *U, const float *Y, int m,
                                                          int n, double *sums) {
    __shared__ double red[2][8];
    const int b = blockIdx.y, wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + wp;
    double a2 = 0.0, rs = 0.0;
    if (r < m) {
        const float *a = A + ((long long)b * m + r) * n, *u = U + ((long long)b * m + r) * n;
        const float *y = Y + (long long)b * kProbes * n;
        ff acc[kProbes];
#pragma unroll
        for (int p = 0; p < kProbes; ++p) acc[p] = ff_zero();
        ff an = ff_zero();
        for (int j = lane; j < n; j += 32) {
            const float x = a[j], uu = u[j];
            const unsigned h = probe_hash(j);
            an = ff_fma(an, x, x);
#pragma unroll
            for (int p = 0; p < kProbes; ++p) {
                acc[p] = ff_add(acc[p], ff{probe_sign(h, p) * x, 0.f});
                acc[p] = ff_fma(acc[p], -uu, y[(long long)p * n + j]);
            }
        }
        an = warp_sum(an);
        a2 = (double)an.hi + (double)an.lo;
#pragma unroll
        for (int p = 0; p < kProbes; ++p) {
            const ff t = warp_sum(acc[p]);
            const double d = (double)t.hi + (double)t.lo;
            rs += d * d;
        }
    }
    if (lane == 0) { red[0][wp] = a2; red[1][wp] = rs; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sr = 0.0;
        for (int w = 0; w < 8; ++w) { sa += red[0][w]; sr += red[1][w]; }
        if (sa != 0.0) atomicAdd(&sums[2 * b], sa);
        if (sr != 0.0) atomicAdd(&sums[2 * b + 1], sr);
    }
}

// Matrices to recompute on the plain FP32-accurate path, with the reason as bits: 1 = the
// mixed result's correction rotation or estimated reconstruction error is too large to
// trust (mixed precision: xmax and sums given; both recorded in info), 2 = the learned
// schedule missed tol within its budget (sched_fb given).
__global__ void rerun_flag_kernel(const unsigned *xmax, const double *sums, const int *sched_fb, int B,
                                  float corr_limit, float recon_limit, int *mflag, int *count, psvd_info *info) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    int f = 0;
    if (xmax) {
        const float x = __uint_as_float(xmax[b]);
        const float est = sums[2 * b] > 0.0 ? (float)sqrt(sums[2 * b + 1] / (kProbes * sums[2 * b])) : 0.f;
        if (!(x <= corr_limit) || !(est <= recon_limit)) f |= 1;
        if (info) { info[b].corr_max = x; info[b].recon_est = est; }
    }
    if (sched_fb && sched_fb[b]) f |= 2;
    mflag[b] = f;
    if (f) atomicAdd(count, 1);
}

// Results of the FP32-accurate rerun replace the flagged matrices' records.
__global__ void info_scatter_kernel(psvd_info *info, const psvd_info *infoc, const int *idx, const int *whys,
                                    int F) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= F) return;
    psvd_info r = infoc[j];
    const int why = whys[j];
    r.prec_fallback = why & 1;
    r.sched_fallback = (why >> 1) & 1;
    r.corr_max = info[idx[j]].corr_max;
    r.recon_est = info[idx[j]].recon_est;
    info[idx[j]] = r;
}

// Second-order singular values of Sigma + K: diag(e^-X (Sigma + K) e^-X)_i =
// sigma_i + sum_j (sigma_i + sigma_j) X_ij^2 (one warp per row).
__global__ void sigma_refresh_kernel(const float *X, const float *S, int n, long long ld, float *Sout, float *Sout2) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const float *x = X + (long long)b * n * ld + (long long)i * ld;
    const float *s = S + (long long)b * n;
    const float si = s[i];
    float acc = 0.f;
    for (int j = lane; j < n; j += 32) acc += (si + s[j]) * x[j] * x[j];
    acc = warp_sum(acc);
    if (lane == 0) {
        Sout[(long long)b * n + i] = si + acc;
        if (Sout2) Sout2[(long long)b * n + i] = si + acc;
    }
}

// Second-order part of the update, h = X^2/2 - X^4/8 (TF32 operand): with it,
// I + X + h and I - X + h satisfy (I + F)(I + F)^T = I + O(X^8), the -X^4/8 term being
// one Newton-Schulz step on I + X + X^2/2 (whose Gram is I + X^4/4).
__global__ void corr_h_kernel(const float *X2, const float *X4, int n, long long ld, float *Hh) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long p = (long long)b * n * n + (long long)i * n + j;
    Hh[(long long)b * n * ld + (long long)i * ld + j] = tf32_round(0.5f * X2[p] - 0.125f * X4[p]);
}

// X^2 split for the X^2 X^2 product (symmetric operand)
__global__ void x2_split_kernel(const float *X2, int n, long long ld, float *hi) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    hi[(long long)b * n * ld + (long long)i * ld + j] = tf32_round(X2[(long long)b * n * n + (long long)i * n + j]);
}

// (V E)^T = V^T - X V^T + h V^T and V^T <- V^T + X V^T + h V^T, in FP32, re-split;
// XV = X V^T (split-TF32 product), HV = h V^T (TF32 product), both n x n.
__global__ void add_split_kernel(const float *vthi, const float *vtlo, const float *XV, const float *HV, int n,
                                 long long ld, float *VEt_hi, float *VEt_lo, float *VThi, float *VTlo, float *VT) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    const long long p = (long long)b * n * n + (long long)i * n + j;
    const float v = vthi[o] + vtlo[o];
    const float xv = XV[p], hv = HV[p];
    const float ve = v + (hv - xv);
    const float vn = v + (hv + xv);
    float h, l;
    split_tf32(ve, h, l);
    VEt_hi[o] = h;
    VEt_lo[o] = l;
    split_tf32(vn, h, l);
    VThi[o] = h;
    VTlo[o] = l;
    if (VT) VT[p] = vn;
}

__global__ void hilo_store_kernel(const float *hi, const float *lo, int n, long long ld, float *out) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    out[(long long)b * n * n + (long long)i * n + j] = hi[o] + lo[o];
}

// A bounded device-side wait that expired anywhere in the call (product-kernel pipeline,
// grid barriers of the eigensolver or the QR) turns every record's status into
// PSVD_ERR_TIMEOUT: the outputs are not to be trusted.
__global__ void err_status_kernel(const unsigned *e0, const unsigned *e1, const unsigned *e2, psvd_info *info,
                                  int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const unsigned e = (e0 ? *e0 : 0u) | (e1 ? *e1 : 0u) | (e2 ? *e2 : 0u);
    if (e & DEV_ERR_TIMEOUT) info[b].status = PSVD_ERR_TIMEOUT;
}

__global__ void info_qr_kernel(psvd_info *info, const int *flag, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) info[b].qr_fallback = flag[b];
}

// ------------------------------------------------------------ driver
struct SvdWS {
    PolarWS pw;
    EighWS ew;
    float *S = nullptr;         // eigenvalues as FP32 [B][n]
    float *colss = nullptr;     // [B][n]
    int *flag = nullptr, *any = nullptr;
    float *UT = nullptr, *qtau = nullptr, *qbeta = nullptr, *qbuf = nullptr;   // unblocked QR (large m)
    unsigned *qbar = nullptr;
    QrWS qw;                    // blocked QR (m within the cluster panel)
    bool blocked_qr = false;
    float *Vhi = nullptr, *Vlo = nullptr;            // V = (V^T)^T split
    float *Khi = nullptr, *Klo = nullptr, *T1 = nullptr, *T1hi = nullptr, *T1lo = nullptr, *Kt = nullptr;
    float *X = nullptr, *Xneg = nullptr, *X2 = nullptr, *F = nullptr, *Ft = nullptr, *VEt = nullptr;
    unsigned *xmax = nullptr, *kmax = nullptr;
    int *cprec = nullptr;        // [2][B] precision of the correction products (corr_prec_kernel)
    int *mflag = nullptr;
    double *rsums = nullptr;     // [B][2] reconstruction-check sums
    float *Yp = nullptr;         // [B][kProbes][n] sigma (V^T z) for the check
    bool mixed = false, learned = false;

    template <class C>
    void carve(C &cv, int B, int m, int n, const psvd_opts &o) {
        mixed = o.precision != PSVD_PREC_FP32;
        learned = o.schedule == PSVD_SCHED_LEARNED;
        pw.carve(cv, B, m, n, polar_kcap(o), o.precision);
        ew.carve(cv, B, n, eigh_groups(B, n));
        const long long B64 = B, ld = pad_ld(n), nn = (long long)n * ld;
        S = cv.template take<float>(B64 * n);
        colss = cv.template take<float>(B64 * n);
        flag = cv.template take<int>(B64);
        any = cv.template take<int>(4);
        int qnb = 0, qcl = 0;
        blocked_qr = qr_shape(m, &qnb, &qcl);
        if (blocked_qr) {
            qw.carve(cv, B, m, n);
        } else {
            UT = cv.template take<float>(B64 * n * m);
            qtau = cv.template take<float>(B64 * n);
            qbeta = cv.template take<float>(B64 * n);
            qbuf = cv.template take<float>(B64 * n * m);
            qbar = cv.template take<unsigned>(4);
        }
        mflag = cv.template take<int>(B64);
        if (mixed) {
            Vhi = cv.template take<float>(B64 * nn);
            Vlo = cv.template take<float>(B64 * nn);
            Khi = cv.template take<float>(B64 * nn);
            Klo = cv.template take<float>(B64 * nn);
            T1 = cv.template take<float>(B64 * n * n);
            T1hi = cv.template take<float>(B64 * nn);
            T1lo = cv.template take<float>(B64 * nn);
            Kt = cv.template take<float>(B64 * n * n);
            X = cv.template take<float>(B64 * nn);
            Xneg = cv.template take<float>(B64 * nn);
            X2 = cv.template take<float>(B64 * n * n);
            F = cv.template take<float>(B64 * nn);
            Ft = cv.template take<float>(B64 * nn);
            VEt = cv.template take<float>(B64 * nn * 2);
            xmax = cv.template take<unsigned>(B64);
            kmax = cv.template take<unsigned>(B64);
            cprec = cv.template take<int>(B64 * 2);
            rsums = cv.template take<double>(B64 * 2);
            Yp = cv.template take<float>(B64 * kProbes * n);
        }
    }
};

static int num_sms_svd() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <class Epi>
static int gemm3(const float *ahi, const float *alo, int M, int K, long long lda, long long bsa, const float *bhi,
                 const float *blo, int N, long long ldb, long long bsb, int B, int prec, const Epi &e, unsigned *err,
                 cudaStream_t st) {
    MatView vah = view_of(ahi, M, K, lda, bsa, B), val = view_of(alo ? alo : ahi, M, K, lda, bsa, B);
    MatView vbh = view_of(bhi, N, K, ldb, bsb, B), vbl = view_of(blo ? blo : bhi, N, K, ldb, bsb, B);
    GemmShape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = K; s.prec_uniform = prec; s.err = err;
    cudaError_t r = prec == PREC_TF32X3 ? launch_gemm(nullptr, nullptr, &vah, &val, &vbh, &vbl, s, B, e, st)
                                        : launch_gemm(nullptr, nullptr, &vah, nullptr, &vbh, nullptr, s, B, e, st);
    return r == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

// As gemm3, with the precision of each matrix read on the device from prec[B] (TF32 or
// split-TF32; both operand splits supplied).
template <class Epi>
static int gemm3p(const float *ahi, const float *alo, int M, int K, long long lda, long long bsa, const float *bhi,
                  const float *blo, int N, long long ldb, long long bsb, int B, const int *prec, const Epi &e,
                  unsigned *err, cudaStream_t st) {
    MatView vah = view_of(ahi, M, K, lda, bsa, B), val = view_of(alo, M, K, lda, bsa, B);
    MatView vbh = view_of(bhi, N, K, ldb, bsb, B), vbl = view_of(blo, N, K, ldb, bsb, B);
    GemmShape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = K; s.prec_uniform = PREC_TF32X3; s.prec = prec; s.err = err;
    s.prof_as = PREC_TF32X3 + 1;   // timed with the split-TF32 products (the per-matrix class is the polar chain)
    return launch_gemm(nullptr, nullptr, &vah, &val, &vbh, &vbl, s, B, e, st) == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

int svd_forward(const float *A, float *U, float *Sout, float *VT, SvdWS &w, const psvd_opts &o, psvd_info *info,
                cudaStream_t st) {
    PolarWS &p = w.pw;
    const int B = p.B, m = p.m, n = p.n;
    const long long ld = pad_ld(n), nn = (long long)n * ld;
    if (cudaMemsetAsync(w.any, 0, sizeof(int) * 4, st)) return PSVD_ERR_CUDA;
    // a learned schedule's misses are recomputed with the rest of the rerun (below), not here
    if (int rc = polar_forward(A, nullptr, nullptr, true, p, o, info, st, false)) return rc;
    if (int rc = eigh_forward(p.Hsym, Sout, nullptr, w.ew, st)) return rc;
    if (cudaMemcpyAsync(w.S, Sout, sizeof(float) * (size_t)B * n, cudaMemcpyDeviceToDevice, st)) return PSVD_ERR_CUDA;
    const float *vthi = w.ew.VThi, *vtlo = w.ew.VTlo;
    const float *bu_hi = vthi, *bu_lo = vtlo;        // B operand of U = W V: rows of V^T
    dim3 g16((n + 15) / 16, (n + 15) / 16, B), b16(16, 16);
    if (w.mixed) {
        // V = (V^T)^T split (TF32 operand of the update products)
        SplitOut vo;
        vo.hi = w.Vhi; vo.lo = w.Vlo; vo.ld = ld; vo.bstride = nn;
        if (prepare_operand(vthi, ld, nn, B, n, n, true, 1.f, nullptr, vo, st)) return PSVD_ERR_CUDA;
        if (cudaMemsetAsync(w.kmax, 0, sizeof(unsigned) * (size_t)B, st)) return PSVD_ERR_CUDA;
        skewT_kernel<<<g16, b16, 0, st>>>(p.Hraw, n, w.Khi, w.Klo, ld, w.kmax);     // K^T, K = skew(Hhat)
        corr_prec_kernel<<<1, 32, 0, st>>>(w.kmax, w.S, n, B, 0, w.cprec);
        count_launch(2);
        // T1 = V^T K   (B operand B[j][k] = K[k][j] = K^T[j][k])
        EpiStore e1 = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3p(vthi, vtlo, n, n, ld, nn, w.Khi, w.Klo, n, ld, nn, B, w.cprec, e1, p.err, st)) return rc;
        SplitOut to;
        to.hi = w.T1hi; to.lo = w.T1lo; to.ld = ld; to.bstride = nn;
        if (prepare_operand(w.T1, n, (long long)n * n, B, n, n, false, 1.f, nullptr, to, st)) return PSVD_ERR_CUDA;
        // Ktilde = T1 V   (B operand B[j][k] = V[k][j] = V^T[j][k])
        EpiStore e2 = epi_store_plain(w.Kt, n, (long long)n * n, n, n);
        if (int rc = gemm3p(w.T1hi, w.T1lo, n, n, ld, nn, vthi, vtlo, n, ld, nn, B, w.cprec, e2, p.err, st)) return rc;
        if (cudaMemsetAsync(w.xmax, 0, sizeof(unsigned) * (size_t)B, st)) return PSVD_ERR_CUDA;
        corr_x_kernel<<<dim3((n + 31) / 32, (n + 31) / 32, B), dim3(32, 8), 0, st>>>(w.Kt, w.S, n, w.X, w.Ft, w.Xneg,
                                                                                    ld, w.xmax);   // X_lo in Ft
        sigma_refresh_kernel<<<dim3((n + 7) / 8, B), 256, 0, st>>>(w.X, w.S, n, ld, Sout, nullptr);
        corr_prec_kernel<<<1, 32, 0, st>>>(w.xmax, w.S, n, B, 1, w.cprec + B);
        count_launch(3);
        // X^2 = X X   (B operand B[j][k] = X[k][j] = -X[j][k])
        EpiStore e3 = epi_store_plain(w.X2, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.X, nullptr, n, n, ld, nn, w.Xneg, nullptr, n, ld, nn, B, PREC_TF32, e3, p.err, st)) return rc;
        // X^4 = X^2 X^2 (X^2 symmetric), kept in T1
        x2_split_kernel<<<g16, b16, 0, st>>>(w.X2, n, ld, w.T1hi);
        count_launch(1);
        EpiStore e3b = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.T1hi, nullptr, n, n, ld, nn, w.T1hi, nullptr, n, ld, nn, B, PREC_TF32, e3b, p.err, st)) return rc;
        corr_h_kernel<<<g16, b16, 0, st>>>(w.X2, w.T1, n, ld, w.F);                 // h in F
        count_launch(1);
        // X V^T (split-TF32, into T1) and h V^T (TF32, into Kt); B operand B[j][k] = V^T[k][j] = V[j][k]
        float *VEt_hi = w.VEt, *VEt_lo = w.VEt + (long long)B * nn;
        EpiStore e4 = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3p(w.X, w.Ft, n, n, ld, nn, w.Vhi, w.Vlo, n, ld, nn, B, w.cprec + B, e4, p.err, st)) return rc;
        EpiStore e5 = epi_store_plain(w.Kt, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.F, nullptr, n, n, ld, nn, w.Vhi, nullptr, n, ld, nn, B, PREC_TF32, e5, p.err, st)) return rc;
        add_split_kernel<<<g16, b16, 0, st>>>(vthi, vtlo, w.T1, w.Kt, n, ld, VEt_hi, VEt_lo, w.ew.VThi, w.ew.VTlo,
                                              VT);
        count_launch(1);
        bu_hi = VEt_hi;
        bu_lo = VEt_lo;
    }
    // U = W (V E), with the column-norm check of Algorithm 1
    if (cudaMemsetAsync(w.colss, 0, sizeof(float) * (size_t)B * n, st)) return PSVD_ERR_CUDA;
    {
        EpiColNorm e;
        e.m = m; e.n = n; e.U = U; e.colss = w.colss;
        if (int rc = gemm3(p.Xhi[0], p.Xlo[0], m, n, p.ldn, (long long)m * p.ldn, bu_hi, bu_lo, n, ld, nn, B,
                           PREC_TF32X3, e, p.err, st))
            return rc;
    }
    if (!w.mixed) {
        hilo_store_kernel<<<g16, b16, 0, st>>>(vthi, vtlo, n, ld, VT);
        count_launch(1);
    }
    qr_flag_kernel<<<B, 256, 0, st>>>(w.colss, n, o.eps_qr, w.learned ? p.fallback : nullptr, w.flag, w.any);
    count_launch(1);
    if (w.mixed) {
        // the mixed result's reconstruction error, estimated from kProbes probes of the final
        // factors, and the decision to keep it or recompute the matrix on the FP32 path
        PSVD_TRY(cudaMemsetAsync(w.rsums, 0, sizeof(double) * 2 * (size_t)B, st));
        probe_vt_kernel<<<dim3((n + 7) / 8, B), 256, 0, st>>>(VT, Sout, n, w.Yp);
        probe_resid_kernel<<<dim3((m + 7) / 8, B), 256, 0, st>>>(A, U, w.Yp, m, n, w.rsums);
        count_launch(2);
    }
    if (info) {
        err_status_kernel<<<(B + 127) / 128, 128, 0, st>>>(p.err, w.ew.err, nullptr, info, B);
        count_launch(1);
    }
    if (w.mixed || w.learned) {
        rerun_flag_kernel<<<(B + 127) / 128, 128, 0, st>>>(
            w.mixed ? w.xmax : nullptr, w.rsums, w.learned ? p.fallback : nullptr, B, (float)PSVD_MIXED_CORR_MAX,
            (float)PSVD_MIXED_RECON_MAX, w.mflag, w.any + 1, info);
        count_launch(1);
    }
    return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

// QR fallback (Appendix A.2) of the matrices with flag[b] != 0 (a device array): U is
// replaced by the Q of its QR with diag(R) >= 0, in place.
static int qr_fallback(float *U, SvdWS &w, const int *flag, psvd_info *info, cudaStream_t st) {
    PolarWS &p = w.pw;
    const int B = p.B, m = p.m, n = p.n;
    if (w.blocked_qr) {
        PSVD_TRY(cudaMemsetAsync(w.qw.err, 0, sizeof(unsigned) * 4, st));
        PSVD_TRY_RC(qr_factor(U, U, nullptr, flag, w.qw, st));
    } else {
        QrParams q;
        q.U = U; q.UT = w.UT; q.tau = w.qtau; q.beta = w.qbeta; q.flag = flag; q.bar = w.qbar; q.err = p.err;
        q.B = B; q.m = m; q.n = n; q.spin = barrier_spin();
        q.g = std::max(1, std::min(num_sms_svd(), n / 8));
        PSVD_TRY(cudaMemsetAsync(w.qbar, 0, sizeof(unsigned) * 4, st));
        int occ = 0;
        PSVD_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qr_householder_kernel, 256, 0));
        if (occ * num_sms_svd() < q.g) return cuda_fail(cudaErrorCooperativeLaunchTooLarge, __FILE__, __LINE__);
        void *args[] = {&q};
        PSVD_TRY(cudaLaunchCooperativeKernel((void *)qr_householder_kernel, dim3(q.g), dim3(256), args, 0, st));
        qr_form_q_kernel<<<dim3((n + 7) / 8, B), 256, 0, st>>>(q, w.qbuf);
        count_launch(2);
    }
    if (info) {
        info_qr_kernel<<<(B + 127) / 128, 128, 0, st>>>(info, flag, B);
        err_status_kernel<<<(B + 127) / 128, 128, 0, st>>>(w.blocked_qr ? w.qw.err : nullptr, nullptr, nullptr, info,
                                                           B);
        count_launch(2);
    }
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

}  // namespace psvd

using namespace psvd;

static psvd_opts svd_resolve(const psvd_opts *p) {
    psvd_opts o;
    psvd_default_opts(&o);
    if (p) o = *p;
    return o;
}

// The FP32-accurate rerun of the matrices the first pass flagged (a mixed result that failed
// its checks, or a learned schedule that missed tol): options of the plain conservative path, and the workspace layout (gathered inputs, outputs, records,
// index list, then the plain pipeline's own workspace), carved from the start of the
// same workspace once the mixed pass has finished with it.
static psvd_opts plain_opts(const psvd_opts &o) {
    psvd_opts p = o;
    p.precision = PSVD_PREC_FP32;
    p.schedule = PSVD_SCHED_CANS;
    p.lower_bound = nullptr;
    p.budget = 0;
    return p;
}
struct RerunWS {
    float *A = nullptr, *U = nullptr, *S = nullptr, *VT = nullptr;
    psvd_info *info = nullptr;
    int *idx = nullptr, *why = nullptr;   // rerun matrix j is batch entry idx[j], for reasons why[j]
    size_t head = 0;                      // bytes of the above; the plain pipeline's region follows
    template <class C>
    void carve(C &cv, int F, int m, int n) {
        const long long F64 = F;
        A = cv.template take<float>(F64 * m * n);
        U = cv.template take<float>(F64 * m * n);
        S = cv.template take<float>(F64 * n);
        VT = cv.template take<float>(F64 * n * n);
        info = cv.template take<psvd_info>(F64);
        idx = cv.template take<int>(F64);
        why = cv.template take<int>(F64);
        head = (size_t)round_up((long long)cv.used, 256);
    }
};

static int svd_direct(const float *A, float *U, float *S, float *VT, int B, int m, int n, const psvd_opts &o,
                      void *ws, size_t ws_bytes, psvd_info *info, cudaStream_t st);

// Recompute the matrices with flags[b] != 0 (host copy of the first pass's reasons) on the
// plain FP32-accurate path and scatter the results back.
static int rerun_flagged(const float *A, float *U, float *S, float *VT, int B, int m, int n,
                         const std::vector<int> &flags, const psvd_opts &o, void *ws, size_t ws_bytes,
                         psvd_info *info, cudaStream_t st) {
    std::vector<int> idx, why;
    for (int b = 0; b < B; ++b)
        if (flags[b]) { idx.push_back(b); why.push_back(flags[b]); }
    const int F = (int)idx.size();
    if (F == 0) return PSVD_OK;
    const psvd_opts po = plain_opts(o);
    Carver cv(ws, ws_bytes);
    RerunWS r;
    r.carve(cv, F, m, n);
    if (cv.overflow || r.head >= ws_bytes) return PSVD_ERR_WORKSPACE;
    const size_t mn = (size_t)m * n, nn = (size_t)n * n;
    PSVD_TRY(cudaMemcpyAsync(r.idx, idx.data(), sizeof(int) * (size_t)F, cudaMemcpyHostToDevice, st));
    PSVD_TRY(cudaMemcpyAsync(r.why, why.data(), sizeof(int) * (size_t)F, cudaMemcpyHostToDevice, st));
    for (int j = 0; j < F; ++j)
        PSVD_TRY(cudaMemcpyAsync(r.A + j * mn, A + idx[j] * mn, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
    PSVD_TRY_RC(svd_direct(r.A, r.U, r.S, r.VT, F, m, n, po, static_cast<char *>(ws) + r.head, ws_bytes - r.head,
                           info ? r.info : nullptr, st));
    for (int j = 0; j < F; ++j) {
        const size_t b = (size_t)idx[j];
        PSVD_TRY(cudaMemcpyAsync(U + b * mn, r.U + j * mn, sizeof(float) * mn, cudaMemcpyDeviceToDevice, st));
        PSVD_TRY(cudaMemcpyAsync(S + b * n, r.S + (size_t)j * n, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        PSVD_TRY(cudaMemcpyAsync(VT + b * nn, r.VT + j * nn, sizeof(float) * nn, cudaMemcpyDeviceToDevice, st));
    }
    if (info) {
        info_scatter_kernel<<<(F + 127) / 128, 128, 0, st>>>(info, r.info, r.idx, r.why, F);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    return PSVD_OK;
}

// Workspace of the method on M itself (first pass + room for the rerun of flagged matrices).
static size_t svd_direct_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts &o) {
    Sizer s;
    SvdWS w;
    w.carve(s, (int)batch, (int)m, (int)n, o);
    size_t need = s.used;
    if (o.precision != PSVD_PREC_FP32 || o.schedule == PSVD_SCHED_LEARNED) {
        // room for rerunning every matrix on the FP32-accurate path: the gathered copies, then
        // the plain pipeline's own workspace
        Sizer s2;
        RerunWS r;
        r.carve(s2, (int)batch, (int)m, (int)n);
        need = std::max(need, r.head + svd_direct_bytes(batch, m, n, plain_opts(o)));
    }
    return need + 256;
}

// The method on M itself: first pass, then (mixed precision or learned schedule) the rerun of
// the flagged matrices, with its one host synchronization.
// The one host synchronization of the call: the first pass's per-matrix flags (QR fallback,
// and for mixed precision or the learned schedule, the rerun reasons) are read back; the
// matrices that need it then get the QR fallback, the others the rerun on the plain path.
static int svd_direct(const float *A, float *U, float *S, float *VT, int B, int m, int n, const psvd_opts &o,
                      void *ws, size_t ws_bytes, psvd_info *info, cudaStream_t st) {
    Carver cv(ws, ws_bytes);
    SvdWS w;
    w.carve(cv, B, m, n, o);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    PSVD_TRY_RC(svd_forward(A, U, S, VT, w, o, info, st));
    const bool rerun = w.mixed || w.learned;
    std::vector<int> qflag(B), mflag(B, 0);
    PSVD_TRY(cudaMemcpyAsync(qflag.data(), w.flag, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, st));
    if (rerun) PSVD_TRY(cudaMemcpyAsync(mflag.data(), w.mflag, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, st));
    PSVD_TRY(cudaStreamSynchronize(st));
    std::vector<int> qr_only(B, 0);
    bool any_qr = false, any_rerun = false;
    for (int b = 0; b < B; ++b) {
        qr_only[b] = qflag[b] && !mflag[b];     // a rerun matrix gets its own QR decision in the rerun
        any_qr |= qr_only[b] != 0;
        any_rerun |= mflag[b] != 0;
    }
    if (any_qr) {
        PSVD_TRY(cudaMemcpyAsync(w.flag, qr_only.data(), sizeof(int) * (size_t)B, cudaMemcpyHostToDevice, st));
        PSVD_TRY_RC(qr_fallback(U, w, w.flag, info, st));
    }
    if (any_rerun) return rerun_flagged(A, U, S, VT, B, m, n, mflag, o, ws, ws_bytes, info, st);
    return PSVD_OK;
}

// QR preprocessing (Section 4.1, rectangular matrices): M = Q R, SVD of R, U = Q U_R.
// Layout: Q, R, U_R, then one region shared in turn by the QR, the square pipeline on R and
// the operands of the final product.
struct PreqrLayout {
    float *Q = nullptr, *R = nullptr, *UR = nullptr;
    char *rest = nullptr;
    size_t rest_bytes = 0, need = 0;
    void plan(void *ws, size_t ws_bytes, int64_t B, int64_t m, int64_t n, const psvd_opts &sq) {
        Carver cv(ws, ws_bytes);
        Q = cv.take<float>(B * m * n);
        R = cv.take<float>(B * n * n);
        UR = cv.take<float>(B * n * n);
        const size_t head = (size_t)round_up((long long)cv.used, 256);
        Sizer q;
        QrWS qw;
        qw.carve(q, (int)B, (int)m, (int)n);
        const long long ld = pad_ld(n);
        const size_t ops = (size_t)(2 * B * m * ld + 2 * B * n * ld) * sizeof(float) + 1024;
        const size_t region = std::max(std::max(q.used + 256, svd_direct_bytes(B, n, n, sq)), ops);
        need = head + region;
        rest = ws ? static_cast<char *>(ws) + head : nullptr;
        rest_bytes = ws_bytes > head ? ws_bytes - head : 0;
    }
};

static psvd_opts square_opts(const psvd_opts &o) {
    psvd_opts p = o;
    p.preqr = 0;
    return p;
}

static bool use_preqr(const psvd_opts &o, int64_t m, int64_t n) {
    int nb = 0, cl = 0;
    return o.preqr && m > n && qr_shape((int)m, &nb, &cl);
}

extern "C" size_t psvd_svd_workspace_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts *opts) {
    psvd_opts o = svd_resolve(opts);
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    if (use_preqr(o, m, n)) {
        PreqrLayout l;
        l.plan(nullptr, 0, batch, m, n, square_opts(o));
        return l.need + 256;
    }
    return svd_direct_bytes(batch, m, n, o);
}

extern "C" int psvd_svd_fwd(const float *A, float *U, float *S, float *VT, int64_t batch, int64_t m, int64_t n,
                            const psvd_opts *opts, void *ws, size_t ws_bytes, psvd_info *info, void *stream) {
    psvd_opts o = svd_resolve(opts);
    if (!A || !U || !S || !VT || batch <= 0 || n <= 0 || m < n || batch > 65535 || n > 16384 ||
        (long long)m * n > (1LL << 31))
        return PSVD_ERR_ARG;
    if (o.precision != PSVD_PREC_FP32 && o.precision != PSVD_PREC_MIXED && o.precision != PSVD_PREC_MIXED_BF16)
        return PSVD_ERR_ARG;
    if (o.schedule < PSVD_SCHED_CANS || o.schedule > PSVD_SCHED_PE) return PSVD_ERR_ARG;
    if ((o.schedule == PSVD_SCHED_LEARNED || o.schedule == PSVD_SCHED_PE) && !o.lower_bound) return PSVD_ERR_ARG;
    if (o.preqr != 0 && o.preqr != 1) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_svd_workspace_bytes(batch, m, n, &o)) return PSVD_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = (int)batch, M = (int)m, N = (int)n;
    if (!use_preqr(o, m, n)) return svd_direct(A, U, S, VT, B, M, N, o, ws, ws_bytes, info, st);
    const psvd_opts sq = square_opts(o);
    PreqrLayout l;
    l.plan(ws, ws_bytes, batch, m, n, sq);
    {
        Carver cv(l.rest, l.rest_bytes);
        QrWS qw;
        qw.carve(cv, B, M, N);
        if (cv.overflow) return PSVD_ERR_WORKSPACE;
        PSVD_TRY_RC(qr_factor(A, l.Q, l.R, nullptr, qw, st));
    }
    PSVD_TRY_RC(svd_direct(l.R, l.UR, S, VT, B, N, N, sq, l.rest, l.rest_bytes, info, st));
    // U = Q U_R: B operand B[k][j] = U_R[j][k] (U_R transposed)
    Carver cv(l.rest, l.rest_bytes);
    const long long ld = pad_ld(N);
    float *qhi = cv.take<float>((size_t)B * M * ld), *qlo = cv.take<float>((size_t)B * M * ld);
    float *uhi = cv.take<float>((size_t)B * N * ld), *ulo = cv.take<float>((size_t)B * N * ld);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    SplitOut a, bt;
    a.hi = qhi; a.lo = qlo; a.ld = ld; a.bstride = (long long)M * ld;
    bt.hi = uhi; bt.lo = ulo; bt.ld = ld; bt.bstride = (long long)N * ld;
    PSVD_TRY(prepare_operand(l.Q, N, (long long)M * N, B, M, N, false, 1.f, nullptr, a, st));
    PSVD_TRY(prepare_operand(l.UR, N, (long long)N * N, B, N, N, true, 1.f, nullptr, bt, st));
    unsigned *err = reinterpret_cast<unsigned *>(cv.take<unsigned>(4));
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    EpiStore e = epi_store_plain(U, N, (long long)M * N, M, N);
    return gemm3(qhi, qlo, M, N, ld, (long long)M * ld, uhi, ulo, N, ld, (long long)N * ld, B, PREC_TF32X3, e, err,
                 st);
}
