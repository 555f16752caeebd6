// Matmul-only symmetric eigensolver by spectral divide and conquer on the polar
// decomposition: the EVD of Algorithm 1 computed from the same polynomial iteration that
// gives the polar factor, so that, apart from small leaf problems, all of its work is
// products on the tensor cores.
//
// For symmetric H and a split point mu, X = H - mu I has the polar factor W = sign(X)
// (Definition 2.1: X = W |X| with W = Q sign(Lambda - mu) Q^T), computed by the CANS
// iteration of Algorithm 1.  P = (I + W) / 2 is the orthogonal projector onto the
// eigenvectors with eigenvalues above mu, and k = trace(P) of them lie there.  Orthonormal
// bases of range(P) and range(I - P) are the polar factors of P Omega_1 (n x k) and
// (I - P) Omega_2 (n x (n - k)) for a fixed Gaussian Omega, each refined once more through
// the projector (the polar factor of P V_1 spans range(P) to working accuracy).  Then
// H_1 = V_1^T H V_1 and H_2 = V_2^T H V_2 are split again, down to leaves of at most kLeaf
// rows that the tridiagonal eigensolver takes, and V = [V_1 Z_1, V_2 Z_2].  The eigenvalues
// of H_1 all exceed those of H_2, so the descending order needs no merge.
// mu is the midpoint of the two middle entries of diag(H) (it lies between the extreme
// eigenvalues).  A block whose diagonal spread and off-diagonal entries are within 1e-5 of
// its largest diagonal entry (a near multiple of I, whose H - mu I has no defined sign) goes
// to the leaf solver whole.  The host reads diag(H), its spread and k at every split (two
// synchronizations each).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "eigh.cuh"
#include "polar.cuh"

namespace psvd {

constexpr int kLeaf = 512;       // blocks up to this size go to the tridiagonal eigensolver
constexpr int kMaxDepth = 6;     // deeper blocks (unbalanced splits) go there whatever their size

// Stack allocator over a workspace region: each level takes its buffers and gives them back.
struct Stack {
    char *base;
    size_t cap, top = 0;
    bool sizing;
    template <class T>
    T *take(size_t count) {
        top = (size_t)round_up((long long)top, 256);
        T *p = sizing ? nullptr : reinterpret_cast<T *>(base + top);
        top += count * sizeof(T);
        if (!sizing && top > cap) return nullptr;
        return p;
    }
    size_t peak = 0;
    void note() { peak = std::max(peak, top); }
};

// ---------------------------------------------------------------- kernels
__global__ void dc_diag_kernel(const float *H, int n, float *d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = H[(long long)i * n + i];
}

// *offmax = max |H_ij| over i != j, as the bits of a non-negative float (which order as
// unsigned integers); *offmax must hold 0 on entry
__global__ void dc_offmax_kernel(const float *H, int n, unsigned *offmax) {
    __shared__ float red[32];
    float m = 0.f;
    const long long nn = (long long)n * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x)
        if (t / n != t % n) m = fmaxf(m, fabsf(H[t]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        m = warp_max(m);
        if (threadIdx.x == 0) atomicMax(offmax, __float_as_uint(m));
    }
}

// X = H - mu I
__global__ void dc_shift_kernel(const float *H, int n, float mu, float *X) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    X[t] = H[t] - (i == j ? mu : 0.f);
}

// P = (I + (W + W^T)/2) / 2 and trace(P) (one block reduces the diagonal into *tr)
__global__ void dc_projector_kernel(const float *W, int n, float *P) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    const float s = 0.5f * (W[t] + W[(long long)j * n + i]);
    P[t] = 0.5f * ((i == j ? 1.f : 0.f) + s);
}

__global__ void dc_trace_kernel(const float *P, int n, double *tr) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)P[(long long)i * n + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *tr = s;
}

// Omega^T (n x n, row j = column j of Omega): N(0, 1) entries from a counter hash (Box-Muller)
__global__ void dc_gauss_kernel(int n, unsigned seed, float *OT) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    unsigned h1 = (unsigned)t * 0x9E3779B1u ^ seed, h2 = (unsigned)(t >> 32) * 0x85EBCA77u ^ (seed * 0xC2B2AE3Du);
    h1 ^= h1 >> 16; h1 *= 0x7FEB352Du; h1 ^= h1 >> 15; h1 *= 0x846CA68Bu; h1 ^= h1 >> 16;
    h2 ^= h1 + 0x632BE5ABu; h2 ^= h2 >> 16; h2 *= 0x7FEB352Du; h2 ^= h2 >> 15; h2 *= 0x846CA68Bu; h2 ^= h2 >> 16;
    const float u1 = ((h1 >> 8) + 1u) * (1.f / 16777217.f), u2 = (h2 >> 8) * (1.f / 16777216.f);
    OT[t] = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// C = alpha A + beta B (elementwise, n_elem)
__global__ void dc_axpby_kernel(const float *A, float alpha, const float *B, float beta, long long n_elem, float *C) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_elem) C[t] = alpha * A[t] + (B ? beta * B[t] : 0.f);
}

// V (n x n, column j = eigenvector j) -> VT rows with the largest-|.| entry positive, and S
__global__ void dc_finalize_kernel(const float *V, const float *lam, int n, float *S, float *VT) {
    const int j = blockIdx.x;
    __shared__ float sv[32];
    __shared__ int si[32];
    float best = -1.f;
    int bi = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float a = fabsf(V[(long long)i * n + j]);
        if (!(a == a)) a = -1.f;
        if (a > best || (a == best && i < bi)) { best = a; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && si[w] < bi)) { best = sv[w]; bi = si[w]; }
        si[0] = bi;
    }
    __syncthreads();
    bi = si[0];
    const float sg = V[(long long)bi * n + j] < 0.f ? -1.f : 1.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) VT[(long long)j * n + i] = sg * V[(long long)i * n + j];
    if (threadIdx.x == 0 && S) S[j] = lam[j];
}

// column block: D[:, c0 : c0 + N] (ld) <- E (M x N, contiguous)
__global__ void dc_place_kernel(const float *E, int M, int N, float *D, int ld, int c0) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)M * N) return;
    const int i = (int)(t / N), j = (int)(t % N);
    D[(long long)i * ld + c0 + j] = E[t];
}

// ---------------------------------------------------------------- products
// D (M x N, row-major, ld N) = A (M x K, ld lda) B (K x N, ld ldb), FP32-accurate split-TF32
static int dc_mm(const float *A, int lda, const float *Bm, int ldb, float *D, int M, int N, int K, Stack &stk,
                 unsigned *err, cudaStream_t st) {
    const size_t mark = stk.top;
    const long long ldk = pad_ld(K);
    float *ahi = stk.take<float>((size_t)M * ldk), *alo = stk.take<float>((size_t)M * ldk);
    float *bhi = stk.take<float>((size_t)N * ldk), *blo = stk.take<float>((size_t)N * ldk);
    stk.note();
    if (stk.sizing) { stk.top = mark; return PSVD_OK; }
    if (!blo) return PSVD_ERR_WORKSPACE;
    SplitOut a, b;
    a.hi = ahi; a.lo = alo; a.ld = ldk; a.bstride = (long long)M * ldk;
    b.hi = bhi; b.lo = blo; b.ld = ldk; b.bstride = (long long)N * ldk;
    PSVD_TRY(prepare_operand(A, lda, (long long)M * lda, 1, M, K, false, 1.f, nullptr, a, st));
    PSVD_TRY(prepare_operand(Bm, ldb, (long long)K * ldb, 1, K, N, true, 1.f, nullptr, b, st));
    MatView vah = view_of(ahi, M, K, ldk, (long long)M * ldk, 1), val = view_of(alo, M, K, ldk, (long long)M * ldk, 1);
    MatView vbh = view_of(bhi, N, K, ldk, (long long)N * ldk, 1), vbl = view_of(blo, N, K, ldk, (long long)N * ldk, 1);
    GemmShape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = K; s.prec_uniform = PREC_TF32X3; s.err = err;
    EpiStore e = epi_store_plain(D, N, (long long)M * N, M, N);
    PSVD_TRY(launch_gemm(nullptr, nullptr, &vah, &val, &vbh, &vbl, s, 1, e, st));
    stk.top = mark;
    return PSVD_OK;
}

// W (m x k) = polar factor of G (m x k), FP32-accurate conservative CANS
static int dc_polar(const float *G, int m, int k, float *W, Stack &stk, cudaStream_t st) {
    const size_t mark = stk.top;
    psvd_opts o;
    psvd_default_opts(&o);
    PolarWS w;
    Sizer sz;
    w.carve(sz, 1, m, k, polar_kcap(o), o.precision);
    char *mem = stk.take<char>(sz.used + 256);
    stk.note();
    if (stk.sizing) { stk.top = mark; return PSVD_OK; }
    if (!mem) return PSVD_ERR_WORKSPACE;
    Carver cv(mem, sz.used + 256);
    w.carve(cv, 1, m, k, polar_kcap(o), o.precision);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    PSVD_TRY_RC(polar_forward(G, W, nullptr, false, w, o, nullptr, st));
    stk.top = mark;
    return PSVD_OK;
}

static int dc_leaf(const float *H, int n, float *lam, float *V, Stack &stk, cudaStream_t st) {
    const size_t mark = stk.top;
    Sizer sz;
    EighWS probe;
    probe.carve(sz, 1, n, 1);
    char *mem = stk.take<char>(sz.used + 256);
    float *VT = stk.take<float>((size_t)n * n);
    stk.note();
    if (stk.sizing) { stk.top = mark; return PSVD_OK; }
    if (!mem || !VT) return PSVD_ERR_WORKSPACE;
    Carver cv(mem, sz.used + 256);
    EighWS ew;
    ew.carve(cv, 1, n, 1);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    PSVD_TRY_RC(eigh_forward(H, lam, VT, ew, st));
    // V = VT^T (columns = eigenvectors)
    SplitOut t;
    t.hi = V; t.lo = nullptr; t.ld = n; t.bstride = (long long)n * n;
    PSVD_TRY(prepare_operand(VT, n, (long long)n * n, 1, n, n, true, 1.f, nullptr, t, st));
    stk.top = mark;
    return PSVD_OK;
}

// Eigenvalues (descending) and eigenvectors (columns of V, n x n) of symmetric H (n x n).
static int dc_solve(const float *H, int n, float *lam, float *V, int depth, unsigned *err, Stack &stk,
                    cudaStream_t st) {
    if (n <= kLeaf || depth >= kMaxDepth) return dc_leaf(H, n, lam, V, stk, st);
    const size_t mark = stk.top;
    const long long nn = (long long)n * n;
    float *X = stk.take<float>(nn), *W = stk.take<float>(nn), *P = stk.take<float>(nn), *OT = stk.take<float>(nn);
    float *G = stk.take<float>(nn), *V12 = stk.take<float>(nn), *T = stk.take<float>(nn);
    float *dg = stk.take<float>(n);
    double *tr = stk.take<double>(1);
    unsigned *om = stk.take<unsigned>(1);
    stk.note();
    int k = n / 2;
    if (!stk.sizing) {
        if (!tr || !om) return PSVD_ERR_WORKSPACE;
        std::vector<float> d(n);
        unsigned omb = 0;
        PSVD_TRY(cudaMemsetAsync(om, 0, sizeof(unsigned), st));
        dc_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(H, n, dg);
        dc_offmax_kernel<<<(unsigned)std::min((long long)4 * num_sms(), (nn + 255) / 256), 256, 0, st>>>(H, n, om);
        count_launch(2);
        PSVD_TRY(cudaMemcpyAsync(d.data(), dg, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
        PSVD_TRY(cudaMemcpyAsync(&omb, om, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        PSVD_TRY(cudaStreamSynchronize(st));
        std::sort(d.begin(), d.end());
        float offmax;
        memcpy(&offmax, &omb, sizeof(float));
        // a (near) multiple of I has no usable split: H - mu I is at the level of the
        // rounding of H and its sign is undefined, so the leaf solver takes it whole
        const float dscale = std::max(std::fabs(d.front()), std::fabs(d.back()));
        if (!(std::max(d.back() - d.front(), 2.f * offmax) > 1e-5f * dscale)) {
            stk.top = mark;
            return dc_leaf(H, n, lam, V, stk, st);
        }
        // split point: the midpoint of the two middle diagonal entries, so that a diagonal
        // input with distinct entries is never split at one of its eigenvalues
        const float mu = 0.5f * (d[n / 2 - 1] + d[n / 2]);
        const unsigned blocks = (unsigned)((nn + 255) / 256);
        dc_shift_kernel<<<blocks, 256, 0, st>>>(H, n, mu, X);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    PSVD_TRY_RC(dc_polar(X, n, n, W, stk, st));                      // W = sign(H - mu I)
    if (!stk.sizing) {
        const unsigned blocks = (unsigned)((nn + 255) / 256);
        dc_projector_kernel<<<blocks, 256, 0, st>>>(W, n, P);
        dc_trace_kernel<<<1, 256, 0, st>>>(P, n, tr);
        dc_gauss_kernel<<<blocks, 256, 0, st>>>(n, 0x5EEDu + (unsigned)depth * 7919u, OT);
        count_launch(3);
        double trace = 0.0;
        PSVD_TRY(cudaMemcpyAsync(&trace, tr, sizeof(double), cudaMemcpyDeviceToHost, st));
        PSVD_TRY(cudaStreamSynchronize(st));
        k = (int)std::lround(trace);
        if (k <= 0 || k >= n) {                  // every eigenvalue on one side (H = c I): no split
            stk.top = mark;
            return dc_leaf(H, n, lam, V, stk, st);
        }
    }
    const int k2 = n - k;
    // V1 = polar(P Omega_1), refined as polar(P V1); V2 likewise with I - P.  G holds P Omega,
    // with Omega^T rows 0..k-1 for the first block and k..n-1 for the second.
    float *V1 = V12, *V2 = V12 + (long long)n * k;              // n x k and n x k2, contiguous
    float *G1 = G, *G2 = G + (long long)n * k;
    // Omega itself (n x n row-major) from its transpose, for the products with column blocks
    if (!stk.sizing) {
        SplitOut t;
        t.hi = T; t.lo = nullptr; t.ld = n; t.bstride = nn;       // T = OT^T = Omega (n x n)
        PSVD_TRY(prepare_operand(OT, n, nn, 1, n, n, true, 1.f, nullptr, t, st));
    }
    // G1 = P Omega[:, 0:k], G2 = (I - P) Omega[:, k:n] = Omega[:, k:n] - P Omega[:, k:n]
    PSVD_TRY_RC(dc_mm(P, n, T, n, G1, n, k, n, stk, err, st));
    PSVD_TRY_RC(dc_mm(P, n, T + k, n, G2, n, k2, n, stk, err, st));
    if (!stk.sizing) {
        // Omega[:, k:n] as a contiguous n x k2 block into X (free now), then G2 = X - G2
        const long long e2 = (long long)n * k2;
        SplitOut t;
        t.hi = X; t.lo = nullptr; t.ld = k2; t.bstride = e2;
        PSVD_TRY(prepare_operand(OT + (long long)k * n, n, (long long)k2 * n, 1, k2, n, true, 1.f, nullptr, t, st));
        dc_axpby_kernel<<<(unsigned)((e2 + 255) / 256), 256, 0, st>>>(X, 1.f, G2, -1.f, e2, G2);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    PSVD_TRY_RC(dc_polar(G1, n, k, V1, stk, st));
    PSVD_TRY_RC(dc_polar(G2, n, k2, V2, stk, st));
    // refinement through the projector
    PSVD_TRY_RC(dc_mm(P, n, V1, k, G1, n, k, n, stk, err, st));
    PSVD_TRY_RC(dc_mm(P, n, V2, k2, G2, n, k2, n, stk, err, st));
    if (!stk.sizing) {
        const long long e2 = (long long)n * k2;
        dc_axpby_kernel<<<(unsigned)((e2 + 255) / 256), 256, 0, st>>>(V2, 1.f, G2, -1.f, e2, G2);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    PSVD_TRY_RC(dc_polar(G1, n, k, V1, stk, st));
    PSVD_TRY_RC(dc_polar(G2, n, k2, V2, stk, st));
    // H1 = V1^T (H V1), H2 = V2^T (H V2); V1^T, V2^T by transposed copies into P (free now)
    float *H1 = X, *H2 = X + (long long)k * k;                       // k^2 + k2^2 <= n^2
    float *V1T = P, *V2T = P + (long long)n * k;
    if (!stk.sizing) {
        SplitOut t1, t2;
        t1.hi = V1T; t1.lo = nullptr; t1.ld = n; t1.bstride = (long long)k * n;
        t2.hi = V2T; t2.lo = nullptr; t2.ld = n; t2.bstride = (long long)k2 * n;
        PSVD_TRY(prepare_operand(V1, k, (long long)n * k, 1, n, k, true, 1.f, nullptr, t1, st));
        PSVD_TRY(prepare_operand(V2, k2, (long long)n * k2, 1, n, k2, true, 1.f, nullptr, t2, st));
    }
    PSVD_TRY_RC(dc_mm(H, n, V1, k, T, n, k, n, stk, err, st));                 // T = H V1 (n x k)
    PSVD_TRY_RC(dc_mm(V1T, n, T, k, H1, k, k, n, stk, err, st));               // H1 = V1^T T
    PSVD_TRY_RC(dc_mm(H, n, V2, k2, T, n, k2, n, stk, err, st));
    PSVD_TRY_RC(dc_mm(V2T, n, T, k2, H2, k2, k2, n, stk, err, st));
    // the two halves
    float *Z1 = G, *Z2 = G + (long long)k * k;                                  // k^2 + k2^2 <= n^2
    PSVD_TRY_RC(dc_solve(H1, k, lam, Z1, depth + 1, err, stk, st));
    PSVD_TRY_RC(dc_solve(H2, k2, lam + k, Z2, depth + 1, err, stk, st));
    // V = [V1 Z1, V2 Z2]
    PSVD_TRY_RC(dc_mm(V1, k, Z1, k, T, n, k, k, stk, err, st));
    if (!stk.sizing) {
        dc_place_kernel<<<(unsigned)(((long long)n * k + 255) / 256), 256, 0, st>>>(T, n, k, V, n, 0);
        count_launch(1);
    }
    PSVD_TRY_RC(dc_mm(V2, k2, Z2, k2, T, n, k2, k2, stk, err, st));
    if (!stk.sizing) {
        dc_place_kernel<<<(unsigned)(((long long)n * k2 + 255) / 256), 256, 0, st>>>(T, n, k2, V, n, k);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    stk.top = mark;
    return PSVD_OK;
}

}  // namespace psvd

using namespace psvd;

static size_t dc_bytes(int64_t n) {
    // the split sizes are data-dependent: size every level for the full n (an upper bound),
    // and the leaf for n (an unbalanced split may hand a large block to the leaf solver)
    Stack stk{nullptr, 0, 0, true};
    const long long nn = n * n;
    size_t level = 0;
    {
        Stack s{nullptr, 0, 0, true};
        s.take<float>(7 * nn);
        s.take<float>(n);
        s.take<double>(1);
        const size_t fixed = s.top;
        Stack q{nullptr, 0, 0, true};
        dc_polar(nullptr, (int)n, (int)n, nullptr, q, nullptr);
        Stack g{nullptr, 0, 0, true};
        dc_mm(nullptr, 0, nullptr, 0, nullptr, (int)n, (int)n, (int)n, g, nullptr, nullptr);
        level = fixed + std::max(q.peak, g.peak) + 1024;
    }
    Stack lf{nullptr, 0, 0, true};
    dc_leaf(nullptr, (int)n, nullptr, nullptr, lf, nullptr);
    (void)stk;
    return (size_t)kMaxDepth * level + lf.peak + (size_t)(nn + n) * sizeof(float) + 4096;
}

extern "C" size_t psvd_eigh_dc_workspace_bytes(int64_t n) {
    if (n <= 0) return 0;
    return dc_bytes(n);
}

extern "C" int psvd_eigh_dc(const float *Hs, float *S, float *VT, int64_t batch, int64_t n, void *ws, size_t ws_bytes,
                            void *stream) {
    if (!Hs || !S || !VT || batch <= 0 || n <= 0 || n > 16384 || batch > 65535) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (!ws || ws_bytes < psvd_eigh_dc_workspace_bytes(n)) return PSVD_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    const long long nn = n * n;
    float *V = reinterpret_cast<float *>(base);
    float *lam = V + nn;
    unsigned *err = reinterpret_cast<unsigned *>(lam + n);
    const size_t head = (size_t)round_up((long long)((nn + n) * sizeof(float) + 64), 256);
    for (int64_t b = 0; b < batch; ++b) {
        Stack stk{base + head, ws_bytes - head, 0, false};
        PSVD_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
        PSVD_TRY_RC(dc_solve(Hs + b * nn, (int)n, lam, V, 0, err, stk, st));
        dc_finalize_kernel<<<(unsigned)n, 128, 0, st>>>(V, lam, (int)n, S + b * n, VT + b * nn);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    return PSVD_OK;
}
