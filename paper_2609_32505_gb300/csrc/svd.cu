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

#include "eigh.cuh"
#include "polar.cuh"

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

__global__ void qr_flag_kernel(const float *colss, int n, double eps_qr, int *flag, int *any) {
    const int b = blockIdx.x;
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
        group_barrier(P.bar, (++nbar) * P.g, P.err);
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
            group_barrier(P.bar, (++nbar) * P.g, P.err);
            if (blockIdx.x == 0) {
                // store v_j in place (v_j[j] = 1 implicit) once every CTA has used x
                for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) x[r] = (float)(x[r] * scal);
                if (threadIdx.x == 0) {
                    P.tau[(long long)b * n + j] = (float)tau;
                    P.beta[(long long)b * n + j] = (float)beta;
                }
            }
            group_barrier(P.bar, (++nbar) * P.g, P.err);
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
__global__ void skewT_kernel(const float *Hraw, int n, float *hi, float *lo, long long ld) {
    // K^T = -skew(Hraw) stored as the B operand of V^T K (B[j][k] = K[k][j])
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const float *h = Hraw + (long long)b * n * n;
    const float kt = 0.5f * (h[(long long)j * n + i] - h[(long long)i * n + j]);
    float hh, ll;
    split_tf32(kt, hh, ll);
    hi[(long long)b * n * ld + (long long)i * ld + j] = hh;
    lo[(long long)b * n * ld + (long long)i * ld + j] = ll;
}

// X = Ktilde / (s_i + s_j) (skew); writes X (tf32) and -X (for B operands), and
// the two update factors F = X + X^2/2 and Ft = -X + X^2/2 once X^2 is known.
__global__ void corr_x_kernel(const float *Kt, const float *S, int n, float *X, float *Xneg, long long ld) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const float si = S[(long long)b * n + i], sj = S[(long long)b * n + j];
    const float den = si + sj;
    float k = Kt[(long long)b * n * n + (long long)i * n + j];
    k = 0.5f * (k - Kt[(long long)b * n * n + (long long)j * n + i]);   // exact skew part
    const float x = den > 0.f ? k / den : 0.f;
    X[(long long)b * n * ld + (long long)i * ld + j] = tf32_round(x);
    Xneg[(long long)b * n * ld + (long long)i * ld + j] = tf32_round(-x);
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

// F = X + X^2/2 - X^4/8 and Ft = -X + X^2/2 - X^4/8: (I + F)(I + F)^T = I + O(X^8), the
// -X^4/8 term being one Newton-Schulz step on I + X + X^2/2 (whose Gram is I + X^4/4).
__global__ void corr_f_kernel(const float *X2, const float *X4, const float *X, int n, long long ld, float *F,
                              float *Ft) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    const long long p = (long long)b * n * n + (long long)i * n + j;
    const float x = X[o];
    const float h = 0.5f * X2[p] - 0.125f * X4[p];
    F[o] = tf32_round(x + h);
    Ft[o] = tf32_round(-x + h);
}

// X^2 split for the X^2 X^2 product (symmetric operand)
__global__ void x2_split_kernel(const float *X2, int n, long long ld, float *hi) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    hi[(long long)b * n * ld + (long long)i * ld + j] = tf32_round(X2[(long long)b * n * n + (long long)i * n + j]);
}

__global__ void add_split_kernel(const float *vthi, const float *vtlo, const float *FV, const float *FtV, int n,
                                 long long ld, float *VEt_hi, float *VEt_lo, float *VThi, float *VTlo, float *VT) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    const float v = vthi[o] + vtlo[o];
    const float ve = v + (FtV[o] + VEt_lo[o]);                       // (V E)^T = V^T + Ft V^T
    const float vn = v + FV[(long long)b * n * n + (long long)i * n + j];   // V^T <- V^T + F V^T
    float h, l;
    split_tf32(ve, h, l);
    VEt_hi[o] = h;
    VEt_lo[o] = l;
    split_tf32(vn, h, l);
    VThi[o] = h;
    VTlo[o] = l;
    if (VT) VT[(long long)b * n * n + (long long)i * n + j] = vn;
}



__global__ void hilo_store_kernel(const float *hi, const float *lo, int n, long long ld, float *out) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    out[(long long)b * n * n + (long long)i * n + j] = hi[o] + lo[o];
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
    float *UT = nullptr, *qtau = nullptr, *qbeta = nullptr, *qbuf = nullptr;
    unsigned *qbar = nullptr;
    float *Vhi = nullptr, *Vlo = nullptr;            // V = (V^T)^T split
    float *Khi = nullptr, *Klo = nullptr, *T1 = nullptr, *T1hi = nullptr, *T1lo = nullptr, *Kt = nullptr;
    float *X = nullptr, *Xneg = nullptr, *X2 = nullptr, *F = nullptr, *Ft = nullptr, *VEt = nullptr;
    bool mixed = false;

    template <class C>
    void carve(C &cv, int B, int m, int n, const psvd_opts &o) {
        mixed = o.precision == PSVD_PREC_MIXED;
        pw.carve(cv, B, m, n, polar_kcap(o), mixed);
        ew.carve(cv, B, n, eigh_groups(B, n));
        const long long B64 = B, ld = pad_ld(n), nn = (long long)n * ld;
        S = cv.template take<float>(B64 * n);
        colss = cv.template take<float>(B64 * n);
        flag = cv.template take<int>(B64);
        any = cv.template take<int>(4);
        UT = cv.template take<float>(B64 * n * m);
        qtau = cv.template take<float>(B64 * n);
        qbeta = cv.template take<float>(B64 * n);
        qbuf = cv.template take<float>(B64 * n * m);
        qbar = cv.template take<unsigned>(4);
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

int svd_forward(const float *A, float *U, float *Sout, float *VT, SvdWS &w, const psvd_opts &o, psvd_info *info,
                cudaStream_t st) {
    PolarWS &p = w.pw;
    const int B = p.B, m = p.m, n = p.n;
    const long long ld = pad_ld(n), nn = (long long)n * ld;
    if (int rc = polar_forward(A, nullptr, nullptr, true, p, o, info, st)) return rc;
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
        skewT_kernel<<<g16, b16, 0, st>>>(p.Hraw, n, w.Khi, w.Klo, ld);     // K^T, K = skew(Hhat)
        count_launch(1);
        // T1 = V^T K   (B operand B[j][k] = K[k][j] = K^T[j][k])
        EpiStore e1 = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3(vthi, vtlo, n, n, ld, nn, w.Khi, w.Klo, n, ld, nn, B, PREC_TF32X3, e1, p.err, st)) return rc;
        SplitOut to;
        to.hi = w.T1hi; to.lo = w.T1lo; to.ld = ld; to.bstride = nn;
        if (prepare_operand(w.T1, n, (long long)n * n, B, n, n, false, 1.f, nullptr, to, st)) return PSVD_ERR_CUDA;
        // Ktilde = T1 V   (B operand B[j][k] = V[k][j] = V^T[j][k])
        EpiStore e2 = epi_store_plain(w.Kt, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.T1hi, w.T1lo, n, n, ld, nn, vthi, vtlo, n, ld, nn, B, PREC_TF32X3, e2, p.err, st)) return rc;
        corr_x_kernel<<<g16, b16, 0, st>>>(w.Kt, w.S, n, w.X, w.Xneg, ld);
        sigma_refresh_kernel<<<dim3((n + 7) / 8, B), 256, 0, st>>>(w.X, w.S, n, ld, Sout, nullptr);
        count_launch(2);
        // X^2 = X X   (B operand B[j][k] = X[k][j] = -X[j][k])
        EpiStore e3 = epi_store_plain(w.X2, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.X, nullptr, n, n, ld, nn, w.Xneg, nullptr, n, ld, nn, B, PREC_TF32, e3, p.err, st)) return rc;
        // X^4 = X^2 X^2 (X^2 symmetric), kept in T1
        x2_split_kernel<<<g16, b16, 0, st>>>(w.X2, n, ld, w.T1hi);
        count_launch(1);
        EpiStore e3b = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.T1hi, nullptr, n, n, ld, nn, w.T1hi, nullptr, n, ld, nn, B, PREC_TF32, e3b, p.err, st)) return rc;
        corr_f_kernel<<<g16, b16, 0, st>>>(w.X2, w.T1, w.X, n, ld, w.F, w.Ft);
        count_launch(1);
        // Ft V^T (kept split in VEt) and F V^T (in T1); B operand B[j][k] = V^T[k][j] = V[j][k]
        float *VEt_hi = w.VEt, *VEt_lo = w.VEt + (long long)B * nn;
        EpiStore e4;
        memset(&e4, 0, sizeof(e4));
        e4.rows = n; e4.cols = n; e4.alpha = 1.f;
        e4.hi = VEt_hi; e4.lo = VEt_lo; e4.ldh = ld; e4.bsh = nn;
        if (int rc = gemm3(w.Ft, nullptr, n, n, ld, nn, w.Vhi, nullptr, n, ld, nn, B, PREC_TF32, e4, p.err, st)) return rc;
        EpiStore e5 = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = gemm3(w.F, nullptr, n, n, ld, nn, w.Vhi, nullptr, n, ld, nn, B, PREC_TF32, e5, p.err, st)) return rc;
        // (V E)^T = V^T + Ft V^T and V^T <- V^T + F V^T, in FP32, re-split
        add_split_kernel<<<g16, b16, 0, st>>>(vthi, vtlo, w.T1, VEt_hi, n, ld, VEt_hi, VEt_lo, w.ew.VThi, w.ew.VTlo,
                                              VT);
        count_launch(1);
        bu_hi = VEt_hi;
        bu_lo = VEt_lo;
    }
    // U = W (V E), with the column norms of Algorithm 1 step 7
    if (cudaMemsetAsync(w.colss, 0, sizeof(float) * (size_t)B * n, st) ||
        cudaMemsetAsync(w.any, 0, sizeof(int) * 4, st))
        return PSVD_ERR_CUDA;
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
    qr_flag_kernel<<<B, 256, 0, st>>>(w.colss, n, o.eps_qr, w.flag, w.any);
    count_launch(1);
    int nflag = 0;
    if (cudaMemcpyAsync(&nflag, w.any, sizeof(int), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
        return PSVD_ERR_CUDA;
    if (nflag > 0) {
        QrParams q;
        q.U = U; q.UT = w.UT; q.tau = w.qtau; q.beta = w.qbeta; q.flag = w.flag; q.bar = w.qbar; q.err = p.err;
        q.B = B; q.m = m; q.n = n;
        q.g = std::max(1, std::min(num_sms_svd(), n / 8));
        if (cudaMemsetAsync(w.qbar, 0, sizeof(unsigned) * 4, st)) return PSVD_ERR_CUDA;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qr_householder_kernel, 256, 0) != cudaSuccess ||
            occ * num_sms_svd() < q.g)
            return PSVD_ERR_CUDA;
        void *args[] = {&q};
        if (cudaLaunchCooperativeKernel((void *)qr_householder_kernel, dim3(q.g), dim3(256), args, 0, st) != cudaSuccess)
            return PSVD_ERR_CUDA;
        qr_form_q_kernel<<<dim3((n + 7) / 8, B), 256, 0, st>>>(q, w.qbuf);
        count_launch(2);
        if (info) {
            info_qr_kernel<<<(B + 127) / 128, 128, 0, st>>>(info, w.flag, B);
            count_launch(1);
        }
    }
    return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

}  // namespace psvd

using namespace psvd;

static psvd_opts svd_resolve(const psvd_opts *p) {
    psvd_opts o;
    psvd_default_opts(&o);
    if (p) o = *p;
    return o;
}

extern "C" size_t psvd_svd_workspace_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts *opts) {
    psvd_opts o = svd_resolve(opts);
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    Sizer s;
    SvdWS w;
    w.carve(s, (int)batch, (int)m, (int)n, o);
    return s.used + 256;
}

extern "C" int psvd_svd_fwd(const float *A, float *U, float *S, float *VT, int64_t batch, int64_t m, int64_t n,
                            const psvd_opts *opts, void *ws, size_t ws_bytes, psvd_info *info, void *stream) {
    psvd_opts o = svd_resolve(opts);
    if (!A || !U || !S || !VT || batch <= 0 || n <= 0 || m < n || batch > 65535 || n > 16384 ||
        (long long)m * n > (1LL << 31))
        return PSVD_ERR_ARG;
    if (o.precision != PSVD_PREC_FP32 && o.precision != PSVD_PREC_MIXED) return PSVD_ERR_ARG;
    if (o.schedule == PSVD_SCHED_LEARNED && !o.lower_bound) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_svd_workspace_bytes(batch, m, n, &o)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    SvdWS w;
    w.carve(cv, (int)batch, (int)m, (int)n, o);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return svd_forward(A, U, S, VT, w, o, info, static_cast<cudaStream_t>(stream));
}
