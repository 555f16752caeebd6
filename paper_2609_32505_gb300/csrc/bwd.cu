// Regularized SVD / polar backward (Algorithm 4, Algorithm 3) from cached factors.
//
// Algorithm 4 evaluated in the eigenbasis of H = V Sigma V^T (V^T V = I):
//   A_U = U^T Ubar, B_V = V^T Vbar, Y = M V, Z = Y^T Ubar      (= V^T M^T Wbar V, as Wbar V = Ubar)
//   B   = skew(B_V + A_U)                                       (= (V^T Vbar_tot - Vbar_tot^T V)/2)
//   V^T Hbar V = diag(Sbar) + K_eps^T o B
//   V^T C V    = sym(V^T Hbar V - D_R Z D_R),  D_R = Sigma (Sigma^2 + eps^(1/2))^-1
//   V^T X V    = T_eps o V^T C V
//   Mbar       = (Ubar D_R + 2 Y (V^T X V)) V^T                 (= Wbar R_eps + 2 M X)
// Algorithm 3 (polar) is the same chain with V^T Hbar V computed from Hbar and
// G = Wbar V in place of Ubar.  Six products on the split-TF32 tcgen05 kernel plus
// one elementwise kernel that holds every mask (K_eps, T_eps, D_R).
#include <cmath>
#include <cstring>

#include "eigh.cuh"

namespace psvd {

struct BwdWS {
    int B = 0, m = 0, n = 0;
    long long ldn = 0, ldm = 0;
    float *UThi = nullptr, *UTlo = nullptr;      // U^T (n x m)
    float *GThi = nullptr, *GTlo = nullptr;      // Ubar^T or (Wbar V)^T (n x m)
    float *G = nullptr;                          // Ubar or Wbar V row-major FP32 (m x n) for the epilogue
    float *Mhi = nullptr, *Mlo = nullptr;        // M (m x n)
    float *VThi = nullptr, *VTlo = nullptr;      // V^T (n x n)
    float *Vhi = nullptr, *Vlo = nullptr;        // V (n x n)
    float *dVThi = nullptr, *dVTlo = nullptr;    // Vbar^T (n x n) or sym(Hbar) (polar)
    float *Yhi = nullptr, *Ylo = nullptr;        // Y = M V (m x n)
    float *YThi = nullptr, *YTlo = nullptr;      // Y^T (n x m)
    float *AU = nullptr, *BV = nullptr, *Z = nullptr;   // n x n FP32
    float *Xhi = nullptr, *Xlo = nullptr;        // V^T X V (n x n)
    float *Qhi = nullptr, *Qlo = nullptr;        // (m x n)
    float *Wbhi = nullptr, *Wblo = nullptr;      // Wbar (m x n), polar only
    float *S = nullptr;                          // sigma FP32 (polar: eigenvalues of H)
    float *T1 = nullptr, *T1hi = nullptr, *T1lo = nullptr;  // polar: V^T Hbar
    unsigned *err = nullptr;
    EighWS ew;
    bool polar = false;

    template <class C>
    void carve(C &cv, int B_, int m_, int n_, bool polar_) {
        B = B_; m = m_; n = n_; polar = polar_;
        ldn = pad_ld(n); ldm = pad_ld(m);
        const long long B64 = B, mn = (long long)m * ldn, nm = (long long)n * ldm, nn = (long long)n * ldn;
        UThi = cv.template take<float>(B64 * nm); UTlo = cv.template take<float>(B64 * nm);
        GThi = cv.template take<float>(B64 * nm); GTlo = cv.template take<float>(B64 * nm);
        G = cv.template take<float>(B64 * m * n);
        Mhi = cv.template take<float>(B64 * mn); Mlo = cv.template take<float>(B64 * mn);
        VThi = cv.template take<float>(B64 * nn); VTlo = cv.template take<float>(B64 * nn);
        Vhi = cv.template take<float>(B64 * nn); Vlo = cv.template take<float>(B64 * nn);
        dVThi = cv.template take<float>(B64 * nn); dVTlo = cv.template take<float>(B64 * nn);
        Yhi = cv.template take<float>(B64 * mn); Ylo = cv.template take<float>(B64 * mn);
        YThi = cv.template take<float>(B64 * nm); YTlo = cv.template take<float>(B64 * nm);
        AU = cv.template take<float>(B64 * n * n); BV = cv.template take<float>(B64 * n * n);
        Z = cv.template take<float>(B64 * n * n);
        Xhi = cv.template take<float>(B64 * nn); Xlo = cv.template take<float>(B64 * nn);
        Qhi = cv.template take<float>(B64 * mn); Qlo = cv.template take<float>(B64 * mn);
        S = cv.template take<float>(B64 * n);
        err = cv.template take<unsigned>(4);
        if (polar) {
            Wbhi = cv.template take<float>(B64 * mn); Wblo = cv.template take<float>(B64 * mn);
            T1 = cv.template take<float>(B64 * n * n);
            T1hi = cv.template take<float>(B64 * nn); T1lo = cv.template take<float>(B64 * nn);
            ew.carve(cv, B, n, eigh_groups(B, n));
        }
    }
};

// D_R entry: sigma / (sigma^2 + eps^(1/2)), or the pseudo-inverse 1/sigma (eps = 0)
PSVD_DEV float dr_of(float s, float sqrt_eps, int exact) {
    if (exact) return s > 0.f ? 1.f / s : 0.f;
    return s / (s * s + sqrt_eps);
}

// V^T X V = T o sym(E_H - D_R Z D_R) with E_H = diag(Sbar) + K^T o skew(B_V + A_U)
// (svd) or E_H = the given V^T Hbar V (polar, `EH`).
__global__ void bwd_core_kernel(const float *AU, const float *BV, const float *Z, const float *EH, const float *S,
                                const float *dS, int n, float eps, int kreg_mode, float tie_tol, float *Xhi,
                                float *Xlo, long long ldx) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long bo = (long long)b * n * n, ij = bo + (long long)i * n + j, ji = bo + (long long)j * n + i;
    const float *s = S + (long long)b * n;
    const float si = s[i], sj = s[j];
    const int exact = kreg_mode == 2;
    const float sq = sqrtf(eps), q4 = sqrtf(sq);
    // E_H(i, j) and E_H(j, i)
    float eh_ij, eh_ji;
    if (EH) {
        eh_ij = EH[ij];
        eh_ji = EH[ji];
    } else {
        const float tij = (BV ? BV[ij] : 0.f) + (AU ? AU[ij] : 0.f);
        const float tji = (BV ? BV[ji] : 0.f) + (AU ? AU[ji] : 0.f);
        const float bij = 0.5f * (tij - tji);       // B = skew part
        // K_ij = (s_i - s_j) / ((s_i - s_j)^2 + reg); (K^T)_ij = K_ji = -K_ij
        float kij;
        const float d = si - sj;
        if (kreg_mode == 0) kij = d / (d * d + sq);
        else if (kreg_mode == 1) kij = d / (d * d + eps * eps);
        else {
            const float smax = fmaxf(fabsf(s[0]), fabsf(s[n - 1]));
            kij = fabsf(d) <= tie_tol * smax ? 0.f : 1.f / d;
        }
        // (K^T o B)_ij = K_ji B_ij = -K_ij B_ij; symmetric, since K and B are both skew
        eh_ij = -kij * bij;
        if (i == j && dS) eh_ij += dS[(long long)b * n + i];
        eh_ji = eh_ij;
    }
    const float di = dr_of(si, sq, exact), dj = dr_of(sj, sq, exact);
    const float zij = Z ? Z[ij] : 0.f, zji = Z ? Z[ji] : 0.f;
    const float c = 0.5f * ((eh_ij - di * zij * dj) + (eh_ji - dj * zji * di));
    const float ssum = si + sj;
    float t;
    if (exact) t = ssum > 0.f ? 1.f / ssum : 0.f;
    else t = ssum / (ssum * ssum + q4);
    float h, l;
    split_tf32(t * c, h, l);
    Xhi[(long long)b * n * ldx + (long long)i * ldx + j] = h;
    Xlo[(long long)b * n * ldx + (long long)i * ldx + j] = l;
}

// Q = G D_R + 2 acc (acc = Y (V^T X V)), split row-major
struct EpiQ {
    int m, n;
    const float *G;      // m x n FP32 (nullable = zero)
    const float *S;
    float sqrt_eps;
    int exact;
    float *hi, *lo;
    long long ld;
    struct Acc {};
    // element path through the product kernel's shared-memory transpose, so that a warp
    // reads G and writes hi/lo in 64-byte row segments
    static constexpr bool kElem = true;
    PSVD_DEV bool staged() const { return true; }
    PSVD_DEV void elem(Acc &, int b, int r, int c, float v) const {
        if (r >= m || c >= n) return;
        float x = 2.f * v;
        if (G) x += G[(long long)b * m * n + (long long)r * n + c] * dr_of(S[(long long)b * n + c], sqrt_eps, exact);
        float h, l;
        split_tf32(x, h, l);
        const long long o = (long long)b * m * ld + (long long)r * ld + c;
        hi[o] = h;
        lo[o] = l;
    }
    PSVD_DEV void begin(Acc &) const {}
    PSVD_DEV void chunk(Acc &a, int b, int r, int c0, int, int, float (&v)[16]) const {
#pragma unroll
        for (int i = 0; i < 16; ++i) elem(a, b, r, c0 + i, v[i]);
    }
    PSVD_DEV void finish(Acc &, int, int, int) const {}
};

__global__ void sym_split_kernel(const float *H, int n, float *hi, float *lo, long long ld) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const float *h = H + (long long)b * n * n;
    float x = 0.5f * (h[(long long)i * n + j] + h[(long long)j * n + i]), a, c;
    split_tf32(x, a, c);
    hi[(long long)b * n * ld + (long long)i * ld + j] = a;
    lo[(long long)b * n * ld + (long long)i * ld + j] = c;
}

template <class Epi>
static int g3(const float *ahi, const float *alo, int M, int K, long long lda, long long bsa, const float *bhi,
              const float *blo, int N, long long ldb, long long bsb, int B, const Epi &e, unsigned *err,
              cudaStream_t st) {
    MatView vah = view_of(ahi, M, K, lda, bsa, B), val = view_of(alo, M, K, lda, bsa, B);
    MatView vbh = view_of(bhi, N, K, ldb, bsb, B), vbl = view_of(blo, N, K, ldb, bsb, B);
    GemmShape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = K; s.prec_uniform = PREC_TF32X3; s.err = err;
    return launch_gemm(nullptr, nullptr, &vah, &val, &vbh, &vbl, s, B, e, st) == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

static SplitOut so(float *hi, float *lo, long long ld, long long bs) {
    SplitOut s;
    s.hi = hi; s.lo = lo; s.ld = ld; s.bstride = bs;
    return s;
}

// Shared tail: Y = M V (row-major + transposed), Z = Y^T G, core, Q, dA = Q V^T.
static int bwd_tail(BwdWS &w, bool have_g, const float *EH, const float *AU, const float *BV, const float *dS,
                    float eps, int kreg, float *dA, cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n;
    const long long ldn = w.ldn, ldm = w.ldm, mn = (long long)m * ldn, nm = (long long)n * ldm, nn = (long long)n * ldn;
    {   // Y = M V : B operand B[j][k] = V[k][j] = V^T[j][k]
        EpiStore e;
        memset(&e, 0, sizeof(e));
        e.rows = m; e.cols = n; e.alpha = 1.f;
        e.hi = w.Yhi; e.lo = w.Ylo; e.ldh = ldn; e.bsh = mn;
        e.hi_t = w.YThi; e.lo_t = w.YTlo; e.ldht = ldm; e.bsht = nm;
        if (int rc = g3(w.Mhi, w.Mlo, m, n, ldn, mn, w.VThi, w.VTlo, n, ldn, nn, B, e, w.err, st)) return rc;
    }
    if (have_g) {   // Z = Y^T G
        EpiStore e = epi_store_plain(w.Z, n, (long long)n * n, n, n);
        if (int rc = g3(w.YThi, w.YTlo, n, m, ldm, nm, w.GThi, w.GTlo, n, ldm, nm, B, e, w.err, st)) return rc;
    }
    dim3 g16((n + 15) / 16, (n + 15) / 16, B), b16(16, 16);
    bwd_core_kernel<<<g16, b16, 0, st>>>(AU, BV, have_g ? w.Z : nullptr, EH, w.S, dS, n, eps, kreg, 1e-6f, w.Xhi,
                                         w.Xlo, ldn);
    count_launch(1);
    {   // Q = G D_R + 2 Y (V^T X V)  (B operand = V^T X V, symmetric)
        EpiQ e;
        e.m = m; e.n = n; e.G = have_g ? w.G : nullptr; e.S = w.S; e.sqrt_eps = sqrtf(eps); e.exact = kreg == 2;
        e.hi = w.Qhi; e.lo = w.Qlo; e.ld = ldn;
        if (int rc = g3(w.Yhi, w.Ylo, m, n, ldn, mn, w.Xhi, w.Xlo, n, ldn, nn, B, e, w.err, st)) return rc;
    }
    {   // dA = Q V^T : B operand B[j][k] = V^T[k][j] = V[j][k]
        EpiStore e = epi_store_plain(dA, n, (long long)m * n, m, n);
        if (int rc = g3(w.Qhi, w.Qlo, m, n, ldn, mn, w.Vhi, w.Vlo, n, ldn, nn, B, e, w.err, st)) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

int svd_backward(const float *A, const float *U, const float *S, const float *VT, const float *dU, const float *dS,
                 const float *dVT, float *dA, BwdWS &w, double eps, int kreg, cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n;
    const long long ldn = w.ldn, ldm = w.ldm, mn = (long long)m * ldn, nm = (long long)n * ldm, nn = (long long)n * ldn;
    const float feps = kreg == 2 ? 0.f : (float)eps;
    if (cudaMemcpyAsync(w.S, S, sizeof(float) * (size_t)B * n, cudaMemcpyDeviceToDevice, st)) return PSVD_ERR_CUDA;
    if (prepare_operand(A, n, (long long)m * n, B, m, n, false, 1.f, nullptr, so(w.Mhi, w.Mlo, ldn, mn), st) ||
        prepare_operand(VT, n, (long long)n * n, B, n, n, false, 1.f, nullptr, so(w.VThi, w.VTlo, ldn, nn), st) ||
        prepare_operand(VT, n, (long long)n * n, B, n, n, true, 1.f, nullptr, so(w.Vhi, w.Vlo, ldn, nn), st))
        return PSVD_ERR_CUDA;
    if (dU) {
        if (prepare_operand(U, n, (long long)m * n, B, m, n, true, 1.f, nullptr, so(w.UThi, w.UTlo, ldm, nm), st) ||
            prepare_operand(dU, n, (long long)m * n, B, m, n, true, 1.f, nullptr, so(w.GThi, w.GTlo, ldm, nm), st))
            return PSVD_ERR_CUDA;
        if (cudaMemcpyAsync(w.G, dU, sizeof(float) * (size_t)B * m * n, cudaMemcpyDeviceToDevice, st))
            return PSVD_ERR_CUDA;
        EpiStore e = epi_store_plain(w.AU, n, (long long)n * n, n, n);       // A_U = U^T Ubar
        if (int rc = g3(w.UThi, w.UTlo, n, m, ldm, nm, w.GThi, w.GTlo, n, ldm, nm, B, e, w.err, st)) return rc;
    }
    if (dVT) {
        if (prepare_operand(dVT, n, (long long)n * n, B, n, n, false, 1.f, nullptr, so(w.dVThi, w.dVTlo, ldn, nn), st))
            return PSVD_ERR_CUDA;
        EpiStore e = epi_store_plain(w.BV, n, (long long)n * n, n, n);       // B_V = V^T Vbar
        if (int rc = g3(w.VThi, w.VTlo, n, n, ldn, nn, w.dVThi, w.dVTlo, n, ldn, nn, B, e, w.err, st)) return rc;
    }
    return bwd_tail(w, dU != nullptr, nullptr, dU ? w.AU : nullptr, dVT ? w.BV : nullptr, dS, feps, kreg, dA, st);
}

__global__ void hilo_to_f32_kernel(const float *hi, const float *lo, int n, long long ld, float *out) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long o = (long long)b * n * ld + (long long)i * ld + j;
    out[(long long)b * n * n + (long long)i * n + j] = hi[o] + lo[o];
}

int polar_backward(const float *A, const float *H, const float *dW, const float *dH, float *dA, BwdWS &w, double eps,
                   cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n;
    const long long ldn = w.ldn, ldm = w.ldm, mn = (long long)m * ldn, nm = (long long)n * ldm, nn = (long long)n * ldn;
    // EVD of H (symmetrized by the eigensolver's reads of the full matrix)
    if (int rc = eigh_forward(H, w.S, nullptr, w.ew, st)) return rc;
    if (cudaMemcpyAsync(w.VThi, w.ew.VThi, sizeof(float) * (size_t)B * nn, cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(w.VTlo, w.ew.VTlo, sizeof(float) * (size_t)B * nn, cudaMemcpyDeviceToDevice, st))
        return PSVD_ERR_CUDA;
    if (prepare_operand(A, n, (long long)m * n, B, m, n, false, 1.f, nullptr, so(w.Mhi, w.Mlo, ldn, mn), st))
        return PSVD_ERR_CUDA;
    float *VTf = w.T1;   // V^T as plain FP32 (n x n)
    {
        dim3 g16((n + 15) / 16, (n + 15) / 16, B), b16(16, 16);
        hilo_to_f32_kernel<<<g16, b16, 0, st>>>(w.VThi, w.VTlo, n, ldn, VTf);
        count_launch(1);
    }
    if (prepare_operand(VTf, n, (long long)n * n, B, n, n, true, 1.f, nullptr, so(w.Vhi, w.Vlo, ldn, nn), st))
        return PSVD_ERR_CUDA;
    const float *EH = nullptr;
    if (dH) {
        dim3 g16((n + 15) / 16, (n + 15) / 16, B), b16(16, 16);
        sym_split_kernel<<<g16, b16, 0, st>>>(dH, n, w.dVThi, w.dVTlo, ldn);    // sym(Hbar)
        count_launch(1);
        // T1 = V^T sym(Hbar)  (B operand B[j][k] = Hs[k][j] = Hs[j][k])
        EpiStore e = epi_store_plain(w.T1, n, (long long)n * n, n, n);
        if (int rc = g3(w.VThi, w.VTlo, n, n, ldn, nn, w.dVThi, w.dVTlo, n, ldn, nn, B, e, w.err, st)) return rc;
        if (prepare_operand(w.T1, n, (long long)n * n, B, n, n, false, 1.f, nullptr, so(w.T1hi, w.T1lo, ldn, nn), st))
            return PSVD_ERR_CUDA;
        // E_H = T1 V  (B operand B[j][k] = V[k][j] = V^T[j][k])
        EpiStore e2 = epi_store_plain(w.BV, n, (long long)n * n, n, n);
        if (int rc = g3(w.T1hi, w.T1lo, n, n, ldn, nn, w.VThi, w.VTlo, n, ldn, nn, B, e2, w.err, st)) return rc;
        EH = w.BV;
    } else {
        if (cudaMemsetAsync(w.BV, 0, sizeof(float) * (size_t)B * n * n, st)) return PSVD_ERR_CUDA;
        EH = w.BV;
    }
    if (dW) {
        // G = Wbar V (row-major FP32 for the epilogue, and transposed split for Z)
        if (prepare_operand(dW, n, (long long)m * n, B, m, n, false, 1.f, nullptr, so(w.Wbhi, w.Wblo, ldn, mn), st))
            return PSVD_ERR_CUDA;
        EpiStore e;
        memset(&e, 0, sizeof(e));
        e.rows = m; e.cols = n; e.alpha = 1.f;
        e.out = w.G; e.ld = n; e.bs = (long long)m * n;
        e.hi_t = w.GThi; e.lo_t = w.GTlo; e.ldht = ldm; e.bsht = nm;
        if (int rc = g3(w.Wbhi, w.Wblo, m, n, ldn, mn, w.VThi, w.VTlo, n, ldn, nn, B, e, w.err, st)) return rc;
    }
    return bwd_tail(w, dW != nullptr, EH, nullptr, nullptr, nullptr, (float)eps, eps == 0.0 ? 2 : 0, dA, st);
}


// ------------------------------------------------------------ EVD backward (Theorem 4.3)
// Hbar = V (diag(Sbar) + 1/2 K^T o (P - P^T)) V^T with P = V^T Vbar, K replaced by its
// Tikhonov regularization K_eps (Section 5.2) in modes 0 and 1.  The middle factor E is
// symmetric (K^T and P - P^T are both skew), so V E and (V E) V^T are both TN products
// with V row-major as an operand.
struct EvdBwdWS {
    int B = 0, n = 0;
    long long ldn = 0;
    float *VThi = nullptr, *VTlo = nullptr, *Vhi = nullptr, *Vlo = nullptr;
    float *dVThi = nullptr, *dVTlo = nullptr, *P = nullptr;
    float *Ehi = nullptr, *Elo = nullptr, *Zhi = nullptr, *Zlo = nullptr;
    unsigned *err = nullptr;
    template <class C>
    void carve(C &cv, int B_, int n_) {
        B = B_; n = n_; ldn = pad_ld(n);
        const long long B64 = B, nn = (long long)n * ldn;
        VThi = cv.template take<float>(B64 * nn); VTlo = cv.template take<float>(B64 * nn);
        Vhi = cv.template take<float>(B64 * nn); Vlo = cv.template take<float>(B64 * nn);
        dVThi = cv.template take<float>(B64 * nn); dVTlo = cv.template take<float>(B64 * nn);
        P = cv.template take<float>(B64 * n * n);
        Ehi = cv.template take<float>(B64 * nn); Elo = cv.template take<float>(B64 * nn);
        Zhi = cv.template take<float>(B64 * nn); Zlo = cv.template take<float>(B64 * nn);
        err = cv.template take<unsigned>(4);
    }
};

// E_ij = delta_ij Sbar_i - 1/2 K_ij (P_ij - P_ji)   ((K^T)_ij = K_ji = -K_ij), split TF32.
__global__ void evd_core_kernel(const float *P, const float *S, const float *dS, int n, float eps, int kreg_mode,
                                float tie_tol, float *Ehi, float *Elo, long long ld) {
    const int b = blockIdx.z;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= n || j >= n) return;
    const long long bo = (long long)b * n * n;
    const float *s = S + (long long)b * n;
    const float d = s[i] - s[j];
    float kij;
    if (kreg_mode == 0) kij = d / (d * d + sqrtf(eps));
    else if (kreg_mode == 1) kij = d / (d * d + eps * eps);
    else {
        const float smax = fmaxf(fabsf(s[0]), fabsf(s[n - 1]));
        kij = fabsf(d) <= tie_tol * smax ? 0.f : 1.f / d;
    }
    const float pij = P ? P[bo + (long long)i * n + j] : 0.f, pji = P ? P[bo + (long long)j * n + i] : 0.f;
    float e = -0.5f * kij * (pij - pji);
    if (i == j) e = dS ? dS[(long long)b * n + i] : 0.f;
    float h, l;
    split_tf32(e, h, l);
    Ehi[(long long)b * n * ld + (long long)i * ld + j] = h;
    Elo[(long long)b * n * ld + (long long)i * ld + j] = l;
}

int eigh_backward(const float *S, const float *VT, const float *dS, const float *dVT, float *dH, EvdBwdWS &w,
                  double eps, int kreg, cudaStream_t st) {
    const int B = w.B, n = w.n;
    const long long ldn = w.ldn, nn = (long long)n * ldn;
    PSVD_TRY(prepare_operand(VT, n, (long long)n * n, B, n, n, false, 1.f, nullptr, so(w.VThi, w.VTlo, ldn, nn), st));
    PSVD_TRY(prepare_operand(VT, n, (long long)n * n, B, n, n, true, 1.f, nullptr, so(w.Vhi, w.Vlo, ldn, nn), st));
    if (dVT) {
        PSVD_TRY(prepare_operand(dVT, n, (long long)n * n, B, n, n, false, 1.f, nullptr, so(w.dVThi, w.dVTlo, ldn, nn),
                                 st));
        // P = V^T Vbar: P[i][k] = sum_j VT[i][j] dVT[k][j]
        EpiStore e = epi_store_plain(w.P, n, (long long)n * n, n, n);
        PSVD_TRY_RC(g3(w.VThi, w.VTlo, n, n, ldn, nn, w.dVThi, w.dVTlo, n, ldn, nn, B, e, w.err, st));
    }
    dim3 g16((n + 15) / 16, (n + 15) / 16, B), b16(16, 16);
    evd_core_kernel<<<g16, b16, 0, st>>>(dVT ? w.P : nullptr, S, dS, n, kreg == 2 ? 0.f : (float)eps, kreg, 1e-6f,
                                         w.Ehi, w.Elo, ldn);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    {   // Z = V E (E symmetric, so the B operand B[k][j] = E[j][k] is E itself)
        EpiStore e;
        memset(&e, 0, sizeof(e));
        e.rows = n; e.cols = n; e.alpha = 1.f;
        e.hi = w.Zhi; e.lo = w.Zlo; e.ldh = ldn; e.bsh = nn;
        PSVD_TRY_RC(g3(w.Vhi, w.Vlo, n, n, ldn, nn, w.Ehi, w.Elo, n, ldn, nn, B, e, w.err, st));
    }
    {   // Hbar = Z V^T: B operand B[k][j] = V^T[j][k] = V[k][j], V row-major
        EpiStore e = epi_store_plain(dH, n, (long long)n * n, n, n);
        PSVD_TRY_RC(g3(w.Zhi, w.Zlo, n, n, ldn, nn, w.Vhi, w.Vlo, n, ldn, nn, B, e, w.err, st));
    }
    return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

}  // namespace psvd

using namespace psvd;

extern "C" size_t psvd_eigh_bwd_workspace_bytes(int64_t batch, int64_t n) {
    if (batch <= 0 || n <= 0) return 0;
    Sizer s;
    EvdBwdWS w;
    w.carve(s, (int)batch, (int)n);
    return s.used + 256;
}

extern "C" int psvd_eigh_bwd(const float *S, const float *VT, const float *dS, const float *dVT, float *dH,
                             int64_t batch, int64_t n, double eps, int kreg_mode, void *ws, size_t ws_bytes,
                             void *stream) {
    if (!S || !VT || !dH || batch <= 0 || n <= 0 || batch > 65535 || n > 16384 || kreg_mode < 0 || kreg_mode > 2 ||
        !(eps >= 0.0) || (eps == 0.0 && kreg_mode != 2))
        return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_eigh_bwd_workspace_bytes(batch, n)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    EvdBwdWS w;
    w.carve(cv, (int)batch, (int)n);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return eigh_backward(S, VT, dS, dVT, dH, w, eps, kreg_mode, static_cast<cudaStream_t>(stream));
}

extern "C" size_t psvd_svd_bwd_workspace_bytes(int64_t batch, int64_t m, int64_t n) {
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    Sizer s;
    BwdWS w;
    w.carve(s, (int)batch, (int)m, (int)n, false);
    return s.used + 256;
}

extern "C" size_t psvd_polar_bwd_workspace_bytes(int64_t batch, int64_t m, int64_t n) {
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    Sizer s;
    BwdWS w;
    w.carve(s, (int)batch, (int)m, (int)n, true);
    return s.used + 256;
}

extern "C" int psvd_svd_bwd(const float *A, const float *U, const float *S, const float *VT, const float *dU,
                            const float *dS, const float *dVT, float *dA, int64_t batch, int64_t m, int64_t n,
                            double eps, int kreg_mode, void *ws, size_t ws_bytes, void *stream) {
    if (!A || !U || !S || !VT || !dA || batch <= 0 || n <= 0 || m < n || batch > 65535 || n > 16384 ||
        kreg_mode < 0 || kreg_mode > 2 || !(eps >= 0.0) || (eps == 0.0 && kreg_mode != 2))
        return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_svd_bwd_workspace_bytes(batch, m, n)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    BwdWS w;
    w.carve(cv, (int)batch, (int)m, (int)n, false);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return svd_backward(A, U, S, VT, dU, dS, dVT, dA, w, eps, kreg_mode, static_cast<cudaStream_t>(stream));
}

extern "C" int psvd_polar_bwd(const float *A, const float *W, const float *H, const float *dW, const float *dH,
                              float *dA, int64_t batch, int64_t m, int64_t n, double eps, void *ws, size_t ws_bytes,
                              void *stream) {
    (void)W;
    if (!A || !H || !dA || batch <= 0 || n <= 0 || m < n || batch > 65535 || n > 16384 || !(eps >= 0.0))
        return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_polar_bwd_workspace_bytes(batch, m, n)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    BwdWS w;
    w.carve(cv, (int)batch, (int)m, (int)n, true);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return polar_backward(A, H, dW, dH, dA, w, eps, static_cast<cudaStream_t>(stream));
}
