// Symmetric eigendecomposition H = V Sigma V^T (Algorithm 1 step 5), in four stages:
//  1. Householder tridiagonalization Q^T H Q = T (FP32, persistent cooperative kernel,
//     one group barrier per reflector; the row that the next reflector is built from
//     is left un-updated and corrected on the fly, so the rank-2 update of step k and
//     the matrix-vector product of step k+1 touch only rows owned by the same warp).
//  2. Eigenvalues of T by Sturm-count bisection (FP32, on T scaled to unit norm).
//  3. Eigenvectors of T by inverse iteration (FP64, one thread per eigenvalue,
//     partially pivoted tridiagonal LU), Rayleigh-quotient refinement of the shift,
//     modified Gram-Schmidt inside clusters of close eigenvalues.
//  4. Back-transform V^T = Z^T Q^T with compact-WY blocks of kWY reflectors on the
//     tcgen05 split-TF32 product kernel, then the sign convention (largest-|.| entry
//     of each eigenvector positive).
#include <cfloat>
#include <cmath>
#include <cstring>

#include "eigh.cuh"

namespace psvd {

constexpr int kTrdThreads = 256;
struct TrdParams {
    const float *H;
    float *Aw, *Vh, *tau;
    double *d, *e;
    float *pbuf;
    unsigned *bar, *err;
    int B, n, groups, g;
    long long ldn;
};

__global__ void __launch_bounds__(kTrdThreads) sytrd_kernel(TrdParams P) {
    extern __shared__ float sm[];
    __shared__ double red[32];
    const int n = P.n;
    float *bx = sm, *bv = sm + n, *bw = sm + 2 * n;
    const int grp = blockIdx.x / P.g, cig = blockIdx.x % P.g;
    if (grp >= P.groups) return;
    const int nwarp = kTrdThreads / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = cig * nwarp + warp, GW = P.g * nwarp;
    unsigned *ctr = P.bar + grp;
    unsigned nbar = 0;
    for (int b = grp; b < P.B; b += P.groups) {
        const float *Hb = P.H + (long long)b * n * n;
        float *A = P.Aw + (long long)b * n * n;
        float *Vh = P.Vh + (long long)b * n * P.ldn;
        for (int i = gw; i < n; i += GW)
            for (int j = lane; j < n; j += 32) A[(long long)i * n + j] = Hb[(long long)i * n + j];
        for (int j = threadIdx.x; j < n; j += blockDim.x) { bv[j] = 0.f; bw[j] = 0.f; }
        group_barrier(ctr, (++nbar) * P.g, P.err);
        for (int k = 0; k + 2 < n; ++k) {
            // x = row k (columns k+1..n-1), corrected by the deferred update of step k-1
            const float vk = bv[k], wk = bw[k];
            const float *Ak = A + (long long)k * n;
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) bx[j] = Ak[j] - (vk * bw[j] + wk * bv[j]);
            __syncthreads();
            double s2 = 0.0;
            for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) s2 += (double)bx[j] * bx[j];
            s2 = block_sum(s2, red);
            const double alpha = bx[k + 1];
            double beta, tau, scal;
            if (s2 == 0.0) { beta = alpha; tau = 0.0; scal = 0.0; }
            else {
                beta = -copysign(sqrt(alpha * alpha + s2), alpha);
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            __syncthreads();
            for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) bx[j] = (float)(bx[j] * scal);
            if (threadIdx.x == 0) bx[k + 1] = 1.f;
            __syncthreads();
            const float ftau = (float)tau;
            if (cig == 0) {
                if (threadIdx.x == 0) {
                    P.d[(long long)b * n + k] = (double)Ak[k] - 2.0 * (double)vk * (double)wk;
                    P.e[(long long)b * n + k] = beta;
                    P.tau[(long long)b * n + k] = ftau;
                }
                for (int j = threadIdx.x; j < n; j += blockDim.x)
                    Vh[(long long)k * P.ldn + j] = j > k ? bx[j] : 0.f;
            }
            // p_i = tau * (A v)_i for owned trailing rows
            float *pb = P.pbuf + ((long long)grp * 2 + (k & 1)) * n;
            for (int i = gw; i < n; i += GW) {
                if (i <= k) continue;
                const float *Ai = A + (long long)i * n;
                float acc = 0.f;
                for (int j = k + 1 + lane; j < n; j += 32) acc += Ai[j] * bx[j];
                acc = warp_sum(acc);
                if (lane == 0) pb[i] = ftau * acc;
            }
            group_barrier(ctr, (++nbar) * P.g, P.err);
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) bw[j] = pb[j];
            __syncthreads();
            double pv = 0.0;
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) pv += (double)bw[j] * bx[j];
            pv = block_sum(pv, red);
            const float K = (float)(0.5 * tau * pv);
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) bw[j] -= K * bx[j];
            __syncthreads();
            // rank-2 update of owned rows i >= k+2 (row k+1 is corrected by the next step)
            for (int i = gw; i < n; i += GW) {
                if (i < k + 2) continue;
                float *Ai = A + (long long)i * n;
                const float vi = bx[i], wi = bw[i];
                for (int j = k + 2 + lane; j < n; j += 32) Ai[j] -= vi * bw[j] + wi * bx[j];
            }
            float *t = bv; bv = bx; bx = t;     // v_k becomes the correction vector of step k+1
            __syncthreads();
        }
        group_barrier(ctr, (++nbar) * P.g, P.err);
        if (cig == 0) {
            if (threadIdx.x == 0) {
                double *d = P.d + (long long)b * n, *e = P.e + (long long)b * n;
                if (n == 1) {
                    d[0] = A[0];
                } else {
                    const int k = n - 2;
                    d[k] = (double)A[(long long)k * n + k] - 2.0 * (double)bv[k] * (double)bw[k];
                    e[k] = (double)A[(long long)k * n + k + 1] - ((double)bv[k] * bw[k + 1] + (double)bw[k] * bv[k + 1]);
                    d[k + 1] = A[(long long)(k + 1) * n + k + 1];
                    P.tau[(long long)b * n + k] = 0.f;
                }
                P.tau[(long long)b * n + n - 1] = 0.f;
                e[n - 1] = 0.0;
            }
            for (int r = n - 2 < 0 ? 0 : n - 2; r < n; ++r)
                for (int j = threadIdx.x; j < n; j += blockDim.x) Vh[(long long)r * P.ldn + j] = 0.f;
        }
        group_barrier(ctr, (++nbar) * P.g, P.err);
    }
}

// ------------------------------------------------------------ bisection (FP32)
// ascending index j: the largest x with at most j eigenvalues below it.
PSVD_DEV int sturm_count(const float *d, const float *e2, int n, float x, float pivmin) {
    int c = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
    for (int t = 1; t < n; ++t) {
        q = d[t] - x - e2[t - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.f;
    }
    return c;
}

__global__ void tri_bisect_kernel(const double *D, const double *E, int n, double *lam, double *tnorm_out) {
    extern __shared__ float s[];
    float *d = s, *e2 = s + n;
    __shared__ float sh_lo[32], sh_hi[32];
    const int b = blockIdx.y;
    const double *Db = D + (long long)b * n, *Eb = E + (long long)b * n;
    // Gershgorin interval and scale
    float glo = FLT_MAX, ghi = -FLT_MAX;
    double tn = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double r = (j > 0 ? fabs(Eb[j - 1]) : 0.0) + (j < n - 1 ? fabs(Eb[j]) : 0.0);
        tn = fmax(tn, fabs(Db[j]) + r);
    }
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    __shared__ double sh_tn[32];
    if ((threadIdx.x & 31) == 0) sh_tn[threadIdx.x >> 5] = tn;
    __syncthreads();
    tn = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tn = fmax(tn, sh_tn[i]);
    const double inv = tn > 0.0 ? 1.0 / tn : 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        d[j] = (float)(Db[j] * inv);
        const double ej = j < n - 1 ? Eb[j] * inv : 0.0;
        e2[j] = (float)(ej * ej);
        const float r = (float)((j > 0 ? fabs(Eb[j - 1]) : 0.0) + (j < n - 1 ? fabs(Eb[j]) : 0.0)) * (float)inv;
        glo = fminf(glo, d[j] - r);
        ghi = fmaxf(ghi, d[j] + r);
    }
    glo = -warp_max(-glo);
    ghi = warp_max(ghi);
    if ((threadIdx.x & 31) == 0) { sh_lo[threadIdx.x >> 5] = glo; sh_hi[threadIdx.x >> 5] = ghi; }
    __syncthreads();
    glo = FLT_MAX; ghi = -FLT_MAX;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { glo = fminf(glo, sh_lo[i]); ghi = fmaxf(ghi, sh_hi[i]); }
    if (blockIdx.x == 0 && threadIdx.x == 0 && tnorm_out) tnorm_out[b] = tn;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // descending index
    if (i >= n) return;
    if (tn == 0.0) { lam[(long long)b * n + i] = 0.0; return; }
    const int j = n - 1 - i;
    const float pivmin = 1e-30f;
    const float pad = 4.f * FLT_EPSILON * n + 1e-30f;
    float lo = glo - pad, hi = ghi + pad;
    for (int it = 0; it < 80; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (hi - lo <= 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + 2e-30f) break;
        if (sturm_count(d, e2, n, mid, pivmin) <= j) lo = mid;
        else hi = mid;
    }
    lam[(long long)b * n + i] = 0.5 * ((double)lo + (double)hi) * tn;
}

// ------------------------------------------------------------ inverse iteration (FP64)
PSVD_DEV double hash_unit(unsigned a, unsigned b) {
    unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    return (double)h * (2.0 / 4294967296.0) - 1.0;
}

struct InvitParams {
    const double *D, *E, *tn;
    double *lam;
    double *xs, *u0, *u1, *u2, *lm;
    signed char *piv;
    int n, first, count;     // vectors [first, first + count) of the flattened (b, i) index
    long long stride;        // = chunk
};

// factor T - mu I = P L U (U with two superdiagonals)
PSVD_DEV void tri_factor(const InvitParams &P, const double *D, const double *E, int n, double mu, double tiny,
                         int t) {
    const long long s = P.stride;
    double a = D[0] - mu;
    double bsup = n > 1 ? E[0] : 0.0;
    for (int j = 0; j < n - 1; ++j) {
        const double c = E[j];
        const double dn = D[j + 1] - mu;
        const double en = j + 1 < n - 1 ? E[j + 1] : 0.0;
        if (fabs(a) >= fabs(c)) {
            if (a == 0.0) a = tiny;
            const double m = c / a;
            P.u0[j * s + t] = a; P.u1[j * s + t] = bsup; P.u2[j * s + t] = 0.0; P.lm[j * s + t] = m;
            P.piv[j * s + t] = 0;
            a = dn - m * bsup;
            bsup = en;
        } else {
            const double m = a / c;
            P.u0[j * s + t] = c; P.u1[j * s + t] = dn; P.u2[j * s + t] = en; P.lm[j * s + t] = m;
            P.piv[j * s + t] = 1;
            a = bsup - m * dn;
            bsup = -m * en;
        }
    }
    if (fabs(a) < tiny) a = a < 0 ? -tiny : tiny;
    P.u0[(long long)(n - 1) * s + t] = a;
}

PSVD_DEV void tri_solve_normalize(const InvitParams &P, int n, int t) {
    const long long s = P.stride;
    double *x = P.xs;
    for (int j = 0; j < n - 1; ++j) {
        double xj = x[j * s + t], xn = x[(j + 1) * s + t];
        if (P.piv[j * s + t]) { const double tmp = xj; xj = xn; xn = tmp; x[j * s + t] = xj; }
        x[(j + 1) * s + t] = xn - P.lm[j * s + t] * xj;
    }
    double x1 = x[(long long)(n - 1) * s + t] / P.u0[(long long)(n - 1) * s + t];
    x[(long long)(n - 1) * s + t] = x1;
    double x2 = 0.0;
    double nrm = x1 * x1;
    for (int j = n - 2; j >= 0; --j) {
        const double v = (x[j * s + t] - P.u1[j * s + t] * x1 - P.u2[j * s + t] * x2) / P.u0[j * s + t];
        x[j * s + t] = v;
        x2 = x1; x1 = v;
        nrm += v * v;
    }
    const double inv = nrm > 0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int j = 0; j < n; ++j) x[j * s + t] *= inv;
}

PSVD_DEV double tri_rayleigh(const InvitParams &P, const double *D, const double *E, int n, int t) {
    const long long s = P.stride;
    double r = 0.0, prev = 0.0;
    for (int j = 0; j < n; ++j) {
        const double xj = P.xs[j * s + t];
        r += D[j] * xj * xj;
        if (j > 0) r += 2.0 * E[j - 1] * prev * xj;
        prev = xj;
    }
    return r;
}

__global__ void tri_invit_kernel(InvitParams P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.count) return;
    const int n = P.n;
    const long long gi = (long long)P.first + t;
    const int b = (int)(gi / n), i = (int)(gi % n);
    const double *D = P.D + (long long)b * n, *E = P.E + (long long)b * n;
    const double tn = P.tn[b];
    double mu = P.lam[gi];
    const long long s = P.stride;
    if (n == 1) { P.xs[t] = 1.0; return; }
    if (!(tn > 0.0)) {
        // T = 0: every vector is an eigenvector; take the unit vectors
        for (int j = 0; j < n; ++j) P.xs[j * s + t] = j == i ? 1.0 : 0.0;
        P.lam[gi] = 0.0;
        return;
    }
    const double tiny = fmax(tn * 2.2e-16, 1e-280);
    for (int j = 0; j < n; ++j) P.xs[j * s + t] = hash_unit((unsigned)i, (unsigned)j) + 0.0625;
    tri_factor(P, D, E, n, mu, tiny, t);
    tri_solve_normalize(P, n, t);
    tri_solve_normalize(P, n, t);
    // refine the shift with the Rayleigh quotient and iterate once more
    const double rq = tri_rayleigh(P, D, E, n, t);
    if (fabs(rq - mu) < 1e-4 * fmax(tn, 1e-300)) mu = rq;
    tri_factor(P, D, E, n, mu, tiny, t);
    tri_solve_normalize(P, n, t);
    P.lam[gi] = tri_rayleigh(P, D, E, n, t);
}

// Modified Gram-Schmidt inside clusters of eigenvalues closer than ctol * ||T||,
// then Rayleigh quotients again, then enforce descending order.  One block per matrix.
__global__ void tri_cluster_kernel(InvitParams P, const double *bisect_lam, double ctol) {
    __shared__ double red[32];
    const int n = P.n;
    const int b_first = P.first / n;
    const int b = b_first + blockIdx.x;
    if ((long long)b * n >= (long long)P.first + P.count) return;
    const long long s = P.stride;
    const int base = (int)((long long)b * n - P.first);
    const double *D = P.D + (long long)b * n, *E = P.E + (long long)b * n;
    const double tol = ctol * P.tn[b];
    const double *bl = bisect_lam + (long long)b * n;
    int i0 = 0;
    while (i0 < n) {
        int i1 = i0 + 1;
        while (i1 < n && bl[i1 - 1] - bl[i1] <= tol) ++i1;
        if (i1 - i0 >= 2) {
            for (int i = i0; i < i1; ++i) {
                const int ti = base + i;
                for (int l = i0; l < i; ++l) {
                    const int tl = base + l;
                    double dot = 0.0;
                    for (int j = threadIdx.x; j < n; j += blockDim.x) dot += P.xs[j * s + ti] * P.xs[j * s + tl];
                    dot = block_sum(dot, red);
                    for (int j = threadIdx.x; j < n; j += blockDim.x) P.xs[j * s + ti] -= dot * P.xs[j * s + tl];
                    __syncthreads();
                }
                double nr = 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) nr += P.xs[j * s + ti] * P.xs[j * s + ti];
                nr = block_sum(nr, red);
                const double inv = nr > 0 ? 1.0 / sqrt(nr) : 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) P.xs[j * s + ti] *= inv;
                __syncthreads();
                double r = 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const double xj = P.xs[j * s + ti];
                    r += D[j] * xj * xj;
                    if (j + 1 < n) r += 2.0 * E[j] * xj * P.xs[(j + 1) * s + ti];
                }
                r = block_sum(r, red);
                if (threadIdx.x == 0) P.lam[(long long)b * n + i] = r;
                __syncthreads();
            }
        }
        i0 = i1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double *l = P.lam + (long long)b * n;
        for (int i = 1; i < n; ++i) if (l[i] > l[i - 1]) l[i] = l[i - 1];
    }
}

// Z^T rows (eigenvectors of T) from the interleaved FP64 vectors -> V^T split (n x ldn)
__global__ void zt_store_kernel(const double *xs, long long stride, int n, int first_b, int first, float *VThi,
                                float *VTlo, long long ldn) {
    __shared__ double tile[32][33];
    const int bb = blockIdx.z;
    const int b = first_b + bb;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;   // i: eigen index, j: component
    const long long tb = (long long)b * n - first;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (j < n && i < n) ? xs[(long long)j * stride + tb + i] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < n && j < n) {
            float h, l;
            split_tf32((float)tile[threadIdx.x][r], h, l);
            const long long o = (long long)b * n * ldn + (long long)i * ldn + j;
            VThi[o] = h;
            VTlo[o] = l;
        }
    }
}

// ------------------------------------------------------------ back-transform
// Upper-triangular T of the forward compact-WY form H_k0 ... H_k1-1 = I - Y T Y^T,
// one block per (WY block, matrix): G = Y^T Y, then T[:c, c] = -tau_c T[:c, :c] G[:c, c].
__global__ void larft_kernel(const float *Vh, const float *tau, int n, long long ldn, int nblk, float *Tm) {
    extern __shared__ float sm2[];
    float *G = sm2, *T = sm2 + kWY * kWY;
    const int blk = blockIdx.x, b = blockIdx.y;
    const int k0 = blk * kWY;
    const int nb = min(kWY, n - 2 - k0);
    const float *V = Vh + (long long)b * n * ldn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int p = warp; p < nb * nb; p += nw) {
        const int a = p / nb, c = p % nb;
        if (a > c) continue;
        const float *va = V + (long long)(k0 + a) * ldn, *vc = V + (long long)(k0 + c) * ldn;
        float acc = 0.f;
        for (int r = k0 + c + 1 + lane; r < n; r += 32) acc += va[r] * vc[r];
        acc = warp_sum(acc);
        if (lane == 0) G[a * kWY + c] = acc;
    }
    for (int p = threadIdx.x; p < kWY * kWY; p += blockDim.x) T[p] = 0.f;
    __syncthreads();
    const float *tb = tau + (long long)b * n + k0;
    if (threadIdx.x == 0) T[0] = tb[0];
    __syncthreads();
    for (int c = 1; c < nb; ++c) {
        const float tc = tb[c];
        float v = 0.f;
        if (threadIdx.x < c) {
            const int a = threadIdx.x;
            for (int l = a; l < c; ++l) v += T[a * kWY + l] * G[l * kWY + c];
        }
        __syncthreads();
        if (threadIdx.x < c) T[threadIdx.x * kWY + c] = -tc * v;
        if (threadIdx.x == 0) T[c * kWY + c] = tc;
        __syncthreads();
    }
    float *out = Tm + ((long long)b * nblk + blk) * kWY * kWY;
    for (int p = threadIdx.x; p < kWY * kWY; p += blockDim.x) out[p] = T[p];
}

// S2 = S T^T (n x nb), split into TF32 hi/lo.
__global__ void s_times_tt_kernel(const float *S, const float *Tm, int n, int nblk, int blk, int nb, float *S2hi,
                                  float *S2lo) {
    const int b = blockIdx.y;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // over n * kWY
    if (idx >= (long long)n * kWY) return;
    const int i = (int)(idx / kWY), j = (int)(idx % kWY);
    const float *Tb = Tm + ((long long)b * nblk + blk) * kWY * kWY;
    const float *Si = S + (long long)b * n * kWY + (long long)i * kWY;
    float acc = 0.f;
    if (j < nb)
        for (int l = j; l < nb; ++l) acc += Si[l] * Tb[j * kWY + l];
    float h, lo;
    split_tf32(acc, h, lo);
    S2hi[(long long)b * n * kWY + idx] = h;
    S2lo[(long long)b * n * kWY + idx] = lo;
}

// V^T[:, r0 + c] -= acc, kept split in hi/lo.
struct EpiSubSplit {
    int rows, cols;
    float *hi, *lo;
    long long ld, bs;
    struct Acc {};
    PSVD_DEV void begin(Acc &) const {}
    PSVD_DEV void chunk(Acc &, int b, int r, int c0, int, int, float (&v)[16]) const {
        if (r >= rows) return;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c >= cols) break;
            const long long o = b * bs + (long long)r * ld + c;
            const float x = (hi[o] + lo[o]) - v[i];
            float h, l;
            split_tf32(x, h, l);
            hi[o] = h;
            lo[o] = l;
        }
    }
    PSVD_DEV void finish(Acc &, int, int, int) const {}
};

// sign convention + outputs: each row of V^T flipped so its largest-|.| entry is positive
__global__ void eig_finalize_kernel(float *VThi, float *VTlo, long long ldn, int n, const double *lam, float *S,
                                    float *VT) {
    const int b = blockIdx.y, i = blockIdx.x;
    float *h = VThi + (long long)b * n * ldn + (long long)i * ldn;
    float *l = VTlo + (long long)b * n * ldn + (long long)i * ldn;
    __shared__ float sv[32];
    __shared__ int si[32];
    // argmax of |.| with the lowest index on ties; NaN entries never win and the
    // index always stays inside the row
    float best = -1.f;
    int bi = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float a = fabsf(h[j] + l[j]);
        if (!(a == a)) a = -1.f;
        if (a > best || (a == best && j < bi)) { best = a; bi = j; }
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
    if (bi < 0 || bi >= n) bi = 0;
    const float sg = (h[bi] + l[bi]) < 0.f ? -1.f : 1.f;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float hh = sg * h[j], ll = sg * l[j];
        h[j] = hh;
        l[j] = ll;
        if (VT) VT[(long long)b * n * n + (long long)i * n + j] = hh + ll;
    }
    if (threadIdx.x == 0 && S) S[(long long)b * n + i] = (float)lam[(long long)b * n + i];
}

// ------------------------------------------------------------ host
static int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

static int trd_ctas_per_group(int n) { return std::max(1, std::min(num_sms(), n / 32)); }

int eigh_groups(int B, int n) {
    const int g = trd_ctas_per_group(n);
    return std::max(1, std::min(B, num_sms() / g));
}

int eigh_forward(const float *Hs, float *S, float *VT, EighWS &w, cudaStream_t st) {
    const int B = w.B, n = w.n;
    const long long ldn = w.ldn;
    PSVD_TRY(cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * (w.groups + 1), st));
    PSVD_TRY(cudaMemsetAsync(w.err, 0, sizeof(unsigned) * 4, st));
    PSVD_TRY(cudaMemsetAsync(w.e, 0, sizeof(double) * (size_t)B * n, st));
    // 1. tridiagonalization
    {
        TrdParams P;
        P.H = Hs; P.Aw = w.Aw; P.Vh = w.Vh; P.tau = w.tau; P.d = w.d; P.e = w.e; P.pbuf = w.pbuf;
        P.bar = w.bar; P.err = w.err; P.B = B; P.n = n; P.groups = w.groups; P.g = trd_ctas_per_group(n);
        P.ldn = ldn;
        const size_t smem = sizeof(float) * 3 * (size_t)n;
        PSVD_TRY(cudaFuncSetAttribute(sytrd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        PSVD_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sytrd_kernel, kTrdThreads, smem));
        if (occ * num_sms() < w.groups * P.g) return cuda_fail(cudaErrorCooperativeLaunchTooLarge, __FILE__, __LINE__);
        void *args[] = {&P};
        PSVD_TRY(cudaLaunchCooperativeKernel((void *)sytrd_kernel, dim3(w.groups * P.g), dim3(kTrdThreads), args,
                                             smem, st));
        count_launch(1);
    }
    // 2. eigenvalues
    double *tn = reinterpret_cast<double *>(w.S2hi);   // B doubles of scratch (S2 is free until stage 4)
    {
        dim3 g((n + 255) / 256, B);
        const size_t smem = sizeof(float) * 2 * (size_t)n;
        PSVD_TRY(cudaFuncSetAttribute(tri_bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tri_bisect_kernel<<<g, 256, smem, st>>>(w.d, w.e, n, w.lam, tn);
        PSVD_TRY(cudaGetLastError());
        count_launch(1);
    }
    // keep the bisection values for cluster detection
    double *bis = reinterpret_cast<double *>(w.S);   // B*n doubles (S holds B*n*kWY floats)
    PSVD_TRY(cudaMemcpyAsync(bis, w.lam, sizeof(double) * (size_t)B * n, cudaMemcpyDeviceToDevice, st));
    // 3. eigenvectors of T, chunk by chunk (chunks hold whole matrices)
    const int per = std::max(1, w.chunk / n);
    for (int b0 = 0; b0 < B; b0 += per) {
        const int nb = std::min(per, B - b0);
        InvitParams P;
        P.D = w.d; P.E = w.e; P.tn = tn; P.lam = w.lam;
        P.xs = w.xs; P.u0 = w.u0; P.u1 = w.u1; P.u2 = w.u2; P.lm = w.lm; P.piv = w.piv;
        P.n = n; P.first = b0 * n; P.count = nb * n; P.stride = w.chunk;
        tri_invit_kernel<<<(P.count + 127) / 128, 128, 0, st>>>(P);
        tri_cluster_kernel<<<nb, 256, 0, st>>>(P, bis, 1e-5);
        dim3 g((n + 31) / 32, (n + 31) / 32, nb), blk(32, 8);
        zt_store_kernel<<<g, blk, 0, st>>>(w.xs, w.chunk, n, b0, b0 * n, w.VThi, w.VTlo, ldn);
        PSVD_TRY(cudaGetLastError());
        count_launch(3);
    }
    // 4. back-transform V^T = Z^T H_{n-3} ... H_0, compact-WY blocks in descending order
    if (w.nblk > 0) {
        SplitOut vo, yo;
        vo.hi = w.Vhi; vo.lo = w.Vlo; vo.ld = ldn; vo.bstride = (long long)n * ldn;
        yo.hi = w.Yhi; yo.lo = w.Ylo; yo.ld = ldn; yo.bstride = (long long)n * ldn;
        PSVD_TRY(prepare_operand(w.Vh, ldn, (long long)n * ldn, B, n, n, false, 1.f, nullptr, vo, st));
        PSVD_TRY(prepare_operand(w.Vh, ldn, (long long)n * ldn, B, n, n, true, 1.f, nullptr, yo, st));
        const size_t smem = sizeof(float) * 2 * kWY * kWY;
        PSVD_TRY(cudaFuncSetAttribute(larft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        larft_kernel<<<dim3(w.nblk, B), 256, smem, st>>>(w.Vh, w.tau, n, ldn, w.nblk, w.Tm);
        PSVD_TRY(cudaGetLastError());
        count_launch(1);
        for (int blk = w.nblk - 1; blk >= 0; --blk) {
            const int k0 = blk * kWY;
            const int nb = std::min(kWY, n - 2 - k0);
            const int r0 = ((k0 + 1) / 32) * 32;
            const int Lr = n - r0;
            // S = V^T[:, r0:] Y[r0:, blk]   (n x nb)
            {
                MatView ahi = view_of(w.VThi + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView alo = view_of(w.VTlo + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView bhi = view_of(w.Vhi + (long long)k0 * ldn + r0, nb, Lr, ldn, (long long)n * ldn, B);
                MatView blo = view_of(w.Vlo + (long long)k0 * ldn + r0, nb, Lr, ldn, (long long)n * ldn, B);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = n; s.N = nb; s.K = Lr; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                EpiStore e = epi_store_plain(w.S, kWY, (long long)n * kWY, n, nb);
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st));
            }
            {
                dim3 g((unsigned)(((long long)n * kWY + 255) / 256), B);
                s_times_tt_kernel<<<g, 256, 0, st>>>(w.S, w.Tm, n, w.nblk, blk, nb, w.S2hi, w.S2lo);
                PSVD_TRY(cudaGetLastError());
                count_launch(1);
            }
            // V^T[:, r0:] -= S2 Y[r0:, blk]^T
            {
                MatView ahi = view_of(w.S2hi, n, nb, kWY, (long long)n * kWY, B);
                MatView alo = view_of(w.S2lo, n, nb, kWY, (long long)n * kWY, B);
                MatView bhi = view_of(w.Yhi + (long long)r0 * ldn + k0, Lr, nb, ldn, (long long)n * ldn, B);
                MatView blo = view_of(w.Ylo + (long long)r0 * ldn + k0, Lr, nb, ldn, (long long)n * ldn, B);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = n; s.N = Lr; s.K = nb; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                EpiSubSplit e;
                e.rows = n; e.cols = Lr; e.hi = w.VThi + r0; e.lo = w.VTlo + r0; e.ld = ldn;
                e.bs = (long long)n * ldn;
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st));
            }
        }
    }
    eig_finalize_kernel<<<dim3(n, B), 128, 0, st>>>(w.VThi, w.VTlo, ldn, n, w.lam, S, VT);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

}  // namespace psvd

using namespace psvd;

extern "C" size_t psvd_eigh_workspace_bytes(int64_t batch, int64_t n) {
    if (batch <= 0 || n <= 0) return 0;
    Sizer s;
    EighWS w;
    w.carve(s, (int)batch, (int)n, (int)batch);
    return s.used + 256;
}

extern "C" int psvd_eigh(const float *Hs, float *S, float *VT, int64_t batch, int64_t n, void *ws, size_t ws_bytes,
                         void *stream) {
    if (!Hs || (!S && !VT) || batch <= 0 || n <= 0 || n > 16384 || batch > 65535) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_eigh_workspace_bytes(batch, n)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    EighWS w;
    w.carve(cv, (int)batch, (int)n, eigh_groups((int)batch, (int)n));
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return eigh_forward(Hs, S, VT, w, static_cast<cudaStream_t>(stream));
}
