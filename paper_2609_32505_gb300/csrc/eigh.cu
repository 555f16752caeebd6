// Symmetric eigendecomposition H = V Sigma V^T (the EVD of Algorithm 1), in four stages:
//  1. Householder tridiagonalization Q^T H Q = T (FP32, persistent cooperative kernel,
//     one group barrier per reflector; the row that the next reflector is built from
//     is left un-updated and corrected on the fly, so the rank-2 update of step k and
//     the matrix-vector product of step k+1 touch only rows owned by the same warp).
//  2. Eigenvalues of T by Sturm-count multisection (FP32, on T scaled to unit norm);
//     eigenvalues with close neighbours refined by multisection with float-float counts.
//  3. Eigenvectors of T by inverse iteration (one thread per eigenvalue, partially
//     pivoted tridiagonal LU, operands streamed through shared memory; float-float
//     recurrences where a warp's eigenvalues are well separated, FP64 otherwise),
//     Rayleigh quotients, modified Gram-Schmidt inside clusters of close eigenvalues.
//  4. Back-transform V^T = Z^T Q^T with compact-WY blocks of kWY reflectors on the
//     tcgen05 split-TF32 product kernel, then the sign convention (largest-|.| entry
//     of each eigenvector positive).
#include <cfloat>
#include <cmath>
#include <cstring>

#include "eigh.cuh"

namespace psvd {

// Launch shape of the tridiagonalization (compile-time; measured on GB300 at n = 4096):
// 512 threads and one CTA per SM beat 256 x 2; the grid barrier is an arrival counter
// every CTA polls (release add, acquire loads): eigh 66.4 ms, against 67.3 with fenced
// atomics, 76.5 with a release flag that one CTA sets after polling every arrival flag,
// and 30% more when every CTA polls every flag.  The per-step row pass moves the trailing
// matrix through L2 twice, so it is bound by SM-L2 bandwidth: use every SM once the
// matrix has enough rows (one CTA per 24 rows).
#ifndef PSVD_TRD_THREADS
#define PSVD_TRD_THREADS 512
#endif
#ifndef PSVD_TRD_MINB
#define PSVD_TRD_MINB 1
#endif
#ifndef PSVD_TRD_ROWDIV
#define PSVD_TRD_ROWDIV 24
#endif
#ifndef PSVD_TRD_BARRIER
#define PSVD_TRD_BARRIER 3      // 0: release flag, 1: every CTA polls every flag, 2: arrival counter,
#endif                          // 3: arrival counter with release/acquire operations
#ifndef PSVD_TRD_SLEEP
#define PSVD_TRD_SLEEP 40
#endif
constexpr int kTrdThreads = PSVD_TRD_THREADS;
constexpr double kFFEps = 3.5527136788005009e-15;   // 2^-48, the float-float unit roundoff
struct TrdParams {
    const float *H;
    float *Aw, *Vh, *tau;
    double *d, *e;
    float *pbuf;
    unsigned *bar, *err;
    int B, n, groups, g, nrp;
    long long ldn;
    uint32_t spin;           // poll bound of the grid barrier
};

// Householder step data: x (row k, columns > k, corrected) -> v (v[k+1] = 1), tau, beta.
// Every CTA computes it redundantly from the same inputs, so no broadcast is needed.
// The squared norm is a compensated FP32 sum (relative error ~ u, independent of n);
// beta, tau and the scaling follow in FP32 as in single-precision LAPACK.
PSVD_DEV void householder_from_row(float *bx, int k, int n, float *red, float &ftau, double &beta_out) {
    ff s2p = ff_zero();
    for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) s2p = ff_fma(s2p, bx[j], bx[j]);
    const float s2 = block_sum_ff(s2p, red);
    const float alpha = bx[k + 1];
    float beta, tau, scal;
    if (s2 == 0.f) { beta = alpha; tau = 0.f; scal = 0.f; }
    else {
        beta = -copysignf(sqrtf(__fmaf_rn(alpha, alpha, s2)), alpha);
        tau = (beta - alpha) / beta;
        scal = 1.f / (alpha - beta);
    }
    __syncthreads();
    for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) bx[j] = bx[j] * scal;
    if (threadIdx.x == 0) bx[k + 1] = 1.f;
    __syncthreads();
    ftau = tau;
    beta_out = beta;
}

// Two vectors at once: d1 = s1 and d2 = s2 on the 16-byte chunks covering [jstart, n),
// with every global load issued before the first shared-memory store; the entries
// from n up to the end of the last chunk are zeroed.
PSVD_DEV void load2_vec4(float *d1, const float *s1, float *d2, const float *s2, int jstart, int n) {
    const int c0 = jstart >> 2, c1 = (n + 3) >> 2;
    const float4 *a4 = reinterpret_cast<const float4 *>(s1), *b4 = reinterpret_cast<const float4 *>(s2);
    float4 *x4 = reinterpret_cast<float4 *>(d1), *y4 = reinterpret_cast<float4 *>(d2);
    float4 ra[4], rb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + threadIdx.x + u * blockDim.x;
        if (c < c1) { ra[u] = a4[c]; rb[u] = b4[c]; }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + threadIdx.x + u * blockDim.x;
        if (c < c1) { x4[c] = ra[u]; y4[c] = rb[u]; }
    }
    for (int c = c0 + threadIdx.x + 4 * blockDim.x; c < c1; c += blockDim.x) { x4[c] = a4[c]; y4[c] = b4[c]; }
    if (n & 3) {                                   // uniform: a partial last chunk
        __syncthreads();
        for (int j = n + threadIdx.x; j < 4 * c1; j += blockDim.x) { d1[j] = 0.f; d2[j] = 0.f; }
    }
}

// One pass over an owned row i: optional rank-2 update with (u_v, u_w) on columns
// >= jstart, and optional dot product of the updated row with s_v (same columns).
// Rows are padded to 16-byte multiples; columns < jstart are rewritten unchanged.
template <bool kUpd, bool kDot>
PSVD_DEV float row_pass(float *Ai, int jstart, int n, const float *uv, const float *uw, float uvi, float uwi,
                        const float *sv) {
    constexpr int U = 4;      // float4 loads in flight per lane
    const int lane = threadIdx.x & 31;
    const int cs = jstart >> 2, c1 = (n + 3) >> 2;
    float4 *A4 = reinterpret_cast<float4 *>(Ai);
    const float4 *V4 = reinterpret_cast<const float4 *>(uv);
    const float4 *W4 = reinterpret_cast<const float4 *>(uw);
    const float4 *S4 = reinterpret_cast<const float4 *>(sv);
    float acc = 0.f;
    // the chunk holding jstart: columns below jstart are left as they are
    if (lane == 0 && cs < c1) {
        float4 a = A4[cs];
        float x[4] = {a.x, a.y, a.z, a.w};
        const float4 vv = kUpd ? V4[cs] : make_float4(0, 0, 0, 0), ww = kUpd ? W4[cs] : make_float4(0, 0, 0, 0);
        const float4 ss = kDot ? S4[cs] : make_float4(0, 0, 0, 0);
        const float vq[4] = {vv.x, vv.y, vv.z, vv.w}, wq[4] = {ww.x, ww.y, ww.z, ww.w};
        const float sq[4] = {ss.x, ss.y, ss.z, ss.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (4 * cs + e < jstart) continue;
            if (kUpd) x[e] -= uvi * wq[e] + uwi * vq[e];
            if (kDot) acc += x[e] * sq[e];
        }
        if (kUpd) A4[cs] = make_float4(x[0], x[1], x[2], x[3]);
    }
    // full chunks: entries past n are zero in the row and in every vector
    for (int c = cs + 1 + lane; c < c1; c += 32 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c + 32 * u < c1) a[u] = A4[c + 32 * u];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int cc = c + 32 * u;
            if (cc < c1) {
                float4 x = a[u];
                if (kUpd) {
                    const float4 vv = V4[cc], ww = W4[cc];
                    x.x -= uvi * ww.x + uwi * vv.x;
                    x.y -= uvi * ww.y + uwi * vv.y;
                    x.z -= uvi * ww.z + uwi * vv.z;
                    x.w -= uvi * ww.w + uwi * vv.w;
                    A4[cc] = x;
                }
                if (kDot) {
                    const float4 ss = S4[cc];
                    acc += x.x * ss.x + x.y * ss.y + x.z * ss.z + x.w * ss.w;
                }
            }
        }
    }
    return kDot ? warp_sum(acc) : 0.f;
}

// Tridiagonalization Q^T H Q = T.  Step k builds the reflector from row k (columns
// > k) of the current matrix; row k is never updated in place (the row a reflector is
// built from is corrected on the fly with the previous step's v, w).  After the group
// barrier of step k every CTA holds v_k and w_k, builds v_{k+1} from row k+1, and then
// makes one pass over its owned rows that applies the rank-2 update of step k and
// accumulates the matrix-vector product of step k+1.
__global__ void __launch_bounds__(kTrdThreads, PSVD_TRD_MINB) sytrd_kernel(TrdParams P) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float red[64];
    __shared__ float s_alpha;
    const int n = P.n;
    const int ln = (int)P.ldn;
    float *bufs[3] = {sm, sm + ln, sm + 2 * ln};
    const int grp = blockIdx.x / P.g, cig = blockIdx.x % P.g;
    if (grp >= P.groups) return;
    const int nwarp = kTrdThreads / 32, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // rows go to warps warp-major across the CTAs (row i -> CTA i % g), so every CTA owns
    // about n / g rows spread over the whole matrix and loses them at the same rate
    const int gw = warp * P.g + cig, GW = P.g * nwarp;
    unsigned *rel = P.bar + (long long)grp * (P.g + 1);
    unsigned *arr = rel + 1;
    unsigned nbar = 0;
#if PSVD_TRD_BARRIER == 1
#define TRD_BARRIER() flag_barrier_all(arr, cig, P.g, ++nbar, P.err)
#elif PSVD_TRD_BARRIER == 2
#define TRD_BARRIER() group_barrier(rel, (unsigned)P.g * (++nbar), P.err, P.spin)
#elif PSVD_TRD_BARRIER == 3
#define TRD_BARRIER() counter_barrier<PSVD_TRD_SLEEP>(rel, (unsigned)P.g * (++nbar), P.err, P.spin)
#else
#define TRD_BARRIER() flag_barrier(arr, rel, cig, P.g, ++nbar, P.err)
#endif
    for (int b = grp; b < P.B; b += P.groups) {
        const float *Hb = P.H + (long long)b * n * n;
        float *A = P.Aw + (long long)b * n * ln;
        float *Vh = P.Vh + (long long)b * P.nrp * P.ldn;
        double *D = P.d + (long long)b * n, *E = P.e + (long long)b * n;
        for (int i = gw; i < n; i += GW)
            for (int j = lane; j < ln; j += 32) A[(long long)i * ln + j] = j < n ? Hb[(long long)i * n + j] : 0.f;
        for (int j = threadIdx.x; j < 3 * ln; j += blockDim.x) sm[j] = 0.f;
        TRD_BARRIER();
        float *bv = bufs[0], *bw = bufs[1], *bn = bufs[2];   // v_k, w_k, next v
        float tau_k = 0.f;
        if (n >= 3) {
            // reflector 0 from row 0, then the plain matrix-vector product of step 0
            for (int j = 1 + threadIdx.x; j < n; j += blockDim.x) bv[j] = A[j];
            __syncthreads();
            double beta;
            householder_from_row(bv, 0, n, red, tau_k, beta);
            if (cig == 0) {
                if (threadIdx.x == 0) { D[0] = A[0]; E[0] = beta; P.tau[(long long)b * n] = tau_k; }
                for (int j = threadIdx.x; j < n; j += blockDim.x) Vh[j] = j > 0 ? bv[j] : 0.f;
            }
            float *pb = P.pbuf + ((long long)grp * 2 + 0) * ln;
            for (int i = gw; i < n; i += GW) {
                if (i < 1) continue;
                const float acc = row_pass<false, true>(A + (long long)i * ln, 1, n, nullptr, nullptr, 0.f, 0.f, bv);
                if (lane == 0) pb[i] = tau_k * acc;
            }
            TRD_BARRIER();
        }
        for (int k = 0; k + 2 < n; ++k) {
            // w_k = p_k - (tau_k/2)(p_k . v_k) v_k
            const float *pb = P.pbuf + ((long long)grp * 2 + (k & 1)) * ln;
            const bool more = k + 3 < n;          // a reflector k+1 exists
            const float *Ar = A + (long long)(k + 1) * ln;
            // p_k and the stored row k+1 travel together (row k+1 is final up to the
            // pending update of step k, applied below)
            load2_vec4(bw, pb, bn, Ar, k + 1, n);
            __syncthreads();
            const float akk = bn[k + 1];
            ff pvp = ff_zero();
            for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) pvp = ff_fma(pvp, bw[j], bv[j]);
            const float K = 0.5f * tau_k * block_sum_ff(pvp, red);
            const float vk = bv[k + 1];
            const float wk = __fmaf_rn(-K, vk, bw[k + 1]);     // w_k[k+1], as the loops below form it
            float tau_n = 0.f;
            if (more) {
                // one pass: w_k = p_k - K v_k; row k+1 corrected by (v_k, w_k) (its entry k+2 is
                // alpha, the rest enter the norm of reflector k+1), then the norm's reduction,
                // whose barriers also publish w_k, the corrected row and alpha
                ff s2p = ff_zero();
                for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
                    const float wj = __fmaf_rn(-K, bv[j], bw[j]);
                    bw[j] = wj;
                    if (j >= k + 2) {
                        const float xj = bn[j] - (vk * wj + wk * bv[j]);
                        bn[j] = xj;
                        if (j == k + 2) s_alpha = xj;
                        else s2p = ff_fma(s2p, xj, xj);
                    }
                }
                const float s2 = block_sum_ff(s2p, red);
                const float alpha = s_alpha;
                float beta_f, scal;
                if (s2 == 0.f) { beta_f = alpha; tau_n = 0.f; scal = 0.f; }
                else {
                    beta_f = -copysignf(sqrtf(__fmaf_rn(alpha, alpha, s2)), alpha);
                    tau_n = (beta_f - alpha) / beta_f;
                    scal = 1.f / (alpha - beta_f);
                }
                for (int j = k + 3 + threadIdx.x; j < n; j += blockDim.x) bn[j] *= scal;
                if (threadIdx.x == 0) bn[k + 2] = 1.f;
                __syncthreads();
                const double beta = beta_f;
                if (cig == (k + 1) % P.g) {     // the CTAs take turns storing the reflector
                    if (threadIdx.x == 0) {
                        D[k + 1] = (double)akk - 2.0 * (double)vk * (double)wk;
                        E[k + 1] = beta;
                        P.tau[(long long)b * n + k + 1] = tau_n;
                    }
                    for (int j = threadIdx.x; j < n; j += blockDim.x)
                        Vh[(long long)(k + 1) * P.ldn + j] = j > k + 1 ? bn[j] : 0.f;
                }
            } else {
                for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) bw[j] = __fmaf_rn(-K, bv[j], bw[j]);
                __syncthreads();
            }
            // fused pass: rank-2 update of step k and matrix-vector product of step k+1
            float *pn = P.pbuf + ((long long)grp * 2 + ((k + 1) & 1)) * ln;
            for (int i = gw; i < n; i += GW) {
                if (i < k + 2) continue;
                float *Ai = A + (long long)i * ln;
                if (more) {
                    const float acc = row_pass<true, true>(Ai, k + 2, n, bv, bw, bv[i], bw[i], bn);
                    if (lane == 0) pn[i] = tau_n * acc;
                } else {
                    row_pass<true, false>(Ai, k + 2, n, bv, bw, bv[i], bw[i], nullptr);
                }
            }
            if (more) {
                TRD_BARRIER();                      // ends with a CTA barrier
                float *t = bv; bv = bn; bn = t;     // v_{k+1} becomes current
                tau_k = tau_n;
            }
        }
        TRD_BARRIER();
        if (cig == 0 && threadIdx.x == 0) {
            if (n == 1) {
                D[0] = A[0];
            } else {
                // last 2 x 2 block: row n-2 still carries the pending update of the last step
                const int k = n - 2;
                const float vk = n >= 3 ? bv[k] : 0.f, wk = n >= 3 ? bw[k] : 0.f;
                const float vl = n >= 3 ? bv[k + 1] : 0.f, wl = n >= 3 ? bw[k + 1] : 0.f;
                D[k] = (double)A[(long long)k * ln + k] - 2.0 * (double)vk * (double)wk;
                E[k] = (double)A[(long long)k * ln + k + 1] - ((double)vk * wl + (double)wk * vl);
                D[k + 1] = A[(long long)(k + 1) * ln + k + 1];
                P.tau[(long long)b * n + k] = 0.f;
            }
            P.tau[(long long)b * n + n - 1] = 0.f;
            E[n - 1] = 0.0;
        }
        if (cig == 0)
            for (int r = n - 2 < 0 ? 0 : n - 2; r < n; ++r)
                for (int j = threadIdx.x; j < n; j += blockDim.x) Vh[(long long)r * P.ldn + j] = 0.f;
        TRD_BARRIER();
    }
}

#undef TRD_BARRIER

// ------------------------------------------------------------ bisection (FP32)
// ascending index j: the largest x with at most j eigenvalues below it.
PSVD_DEV int sturm_count(const float *d, const float *e2, int n, float x, float pivmin) {
    int c = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
    for (int t = 1; t < n; ++t) {
        q = d[t] - x - __fdividef(e2[t - 1], q);
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
    // 9-way multisection: the 8 lanes of a group evaluate the Sturm count at the 8
    // interior points of [lo, hi]; the counts are non-decreasing in x, so the lanes whose
    // count is <= j form a prefix and its length selects the next interval.
    const int grp = threadIdx.x >> 3, l = threadIdx.x & 7;
    const int i = blockIdx.x * (blockDim.x >> 3) + grp;   // descending index
    const bool valid = i < n;
    const int j = n - 1 - i;
    const float pivmin = 1e-30f;
    const float pad = 4.f * FLT_EPSILON * n + 1e-30f;
    float lo = glo - pad, hi = ghi + pad;
    const unsigned gshift = (threadIdx.x & 31) & ~7u;
    bool stalled = false;
    for (int round = 0; round < 24; ++round) {
        const bool active = valid && tn > 0.0 && !stalled &&
                            hi - lo > 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + 2e-30f;
        if (!__any_sync(0xffffffffu, active)) break;
        const float w = hi - lo;
        const float x = lo + w * ((float)(l + 1) * (1.f / 9.f));
        const bool le = active && sturm_count(d, e2, n, x, pivmin) <= j;
        const unsigned bits = (__ballot_sync(0xffffffffu, le) >> gshift) & 0xFFu;
        if (active) {
            const int k = __popc(bits);
            const float nlo = k > 0 ? lo + w * ((float)k * (1.f / 9.f)) : lo;
            const float nhi = k < 8 ? lo + w * ((float)(k + 1) * (1.f / 9.f)) : hi;
            if (nlo <= lo && nhi >= hi) stalled = true;   // no progress at float resolution
            else { lo = nlo; hi = nhi; }
        }
    }
    if (!valid || l != 0) return;
    if (tn == 0.0) { lam[(long long)b * n + i] = 0.0; return; }
    lam[(long long)b * n + i] = 0.5 * ((double)lo + (double)hi) * tn;
}

// ------------------------------------------------------------ refinement (float-float)
// Float-float quotient a / b (a, b two-float values, b.hi != 0): the FP32 quotient of the
// leading words, then one correction from the exact residual a - r b, so that the result
// carries ~2^-44 relative accuracy on the FP32 pipe.
PSVD_DEV ff ff_div(ff a, ff b) {
    const float r = __fdividef(a.hi, b.hi);
    const float p = __fmul_rn(r, b.hi);
    const float pe = __fmaf_rn(r, b.hi, -p);                  // r b.hi = p + pe exactly
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), __fsub_rn(a.lo, __fmul_rn(r, b.lo)));
    const float r2 = __fdividef(res, b.hi);
    const float h = __fadd_rn(r, r2);
    return ff{h, __fsub_rn(r2, __fsub_rn(h, r))};
}

// Sturm count of T/tn - x I in float-float arithmetic (~2^-44 relative, on the FP32 pipe, which
// GB300 has 64 times as wide as its FP64 pipe).  dd[t] = {d_t / tn, e_{t-1}^2 / tn^2} as
// float-float pairs (e_{-1} = 0); pivots floored at pivmin (the scaled entries are <= 1, so
// e^2 / pivmin stays finite).  The count is that of a matrix perturbed by a few units of 2^-44
// of its norm.
PSVD_DEV int sturm_count_ff(const float4 *__restrict__ dd, int n, ff x, float pivmin) {
    int c = 0;
    float4 v = dd[0];
    ff q = ff_add(ff{v.x, v.y}, ff{-x.hi, -x.lo});
    if (fabsf(q.hi) < pivmin) q = ff{-pivmin, 0.f};
    c += q.hi < 0.f;
    for (int t = 1; t < n; ++t) {
        v = dd[t];
        const ff a = ff_add(ff{v.x, v.y}, ff{-x.hi, -x.lo});
        const ff r = ff_div(ff{v.z, v.w}, q);
        q = ff_add(a, ff{-r.hi, -r.lo});
        if (fabsf(q.hi) < pivmin) q = ff{-pivmin, 0.f};
        c += q.hi < 0.f;
    }
    return c;
}

// dd[b][t] = {split(d_t / tn), split(e_{t-1}^2 / tn^2)} for the float-float Sturm counts, and
// de[b][t] = {split(d_t / tn), split(e_t / tn)} (e_{n-1} = 0) for float-float inverse iteration.
__global__ void sturm_prep_kernel(const double *D, const double *E, const double *tnorm, int n, float4 *dd,
                                  float4 *de) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (t >= n) return;
    const double tn = tnorm[b], inv = tn > 0.0 ? 1.0 / tn : 0.0;
    const double dv = D[(long long)b * n + t] * inv;
    const double ev = t > 0 ? E[(long long)b * n + t - 1] * inv : 0.0;
    const double e2 = ev * ev;
    const float dh = (float)dv, eh = (float)e2;
    dd[(long long)b * n + t] = make_float4(dh, (float)(dv - (double)dh), eh, (float)(e2 - (double)eh));
    const double en = t + 1 < n ? E[(long long)b * n + t] * inv : 0.0;
    const float enh = (float)en;
    de[(long long)b * n + t] = make_float4(dh, (float)(dv - (double)dh), enh, (float)(en - (double)enh));
}

// 1/a by the hardware's approximate reciprocal refined with two Newton-Raphson steps
// (y <- y + y (1 - a y), each doubling the correct bits); |a| is kept >= tiny > 0 by the
// pivot floor, far from the denormal and overflow ranges.
PSVD_DEV double recip64(double a) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    double e = fma(-a, y, 1.0);
    y = fma(y, e, y);
    e = fma(-a, y, 1.0);
    return fma(y, e, y);
}

// Eigenvalues whose FP32 neighbours are closer than `near` * ||T|| are refined by 9-way
// multisection (8 lanes per eigenvalue) from a bracket around the FP32 value, with
// float-float Sturm counts, down to 16 * 2^-48 ||T|| (~6e-14 ||T||; the FP64 counts that
// reached 4 u_64 ||T|| kept the narrow FP64 pipe busy for ~30 ms on graded spectra at n = 4096).
// With such shifts three inverse-iteration solves separate gaps down to ~1e-11 ||T|| by
// themselves; closer groups get the Gram-Schmidt of tri_cluster_kernel.
__global__ void tri_refine_kernel(const float4 *DD, int n, const double *tnorm, double near, double *lam) {
    const int b = blockIdx.y;
    const int grp = threadIdx.x >> 3, l = threadIdx.x & 7;
    const int i = blockIdx.x * (blockDim.x >> 3) + grp;     // descending index
    const float4 *dd = DD + (long long)b * n;
    double *lb = lam + (long long)b * n;
    const double tn = tnorm[b];
    bool active = i < n && n > 1 && tn > 0.0;
    double mid = 0.0;
    if (active) {
        mid = lb[i];
        double g = 1e300;
        if (i > 0) g = fmin(g, lb[i - 1] - mid);
        if (i + 1 < n) g = fmin(g, mid - lb[i + 1]);
        active = g < near * tn;
    }
    const bool refined = active;
    const int j = n - 1 - i;                                 // ascending index
    const float pivmin = 1e-30f;                             // on T / tn
    const double inv = tn > 0.0 ? 1.0 / tn : 0.0;
    const double stop = 16.0 * kFFEps * tn;
    auto count = [&](double x) {
        const double xs = x * inv;
        const float xh = (float)xs;
        return sturm_count_ff(dd, n, ff{xh, (float)(xs - (double)xh)}, pivmin);
    };
    double w = 64.0 * FLT_EPSILON * tn;
    double lo = mid - w, hi = mid + w;
    const unsigned gshift = (threadIdx.x & 31) & ~7u;
    // a bracket with count(lo) <= j < count(hi), widened if the FP32 value was off
    for (int tries = 0; tries < 6; ++tries) {
        bool need = false;
        if (active) {
            const double x = l == 0 ? lo : hi;
            const int c = l < 2 ? count(x) : 0;
            const bool ok = l == 0 ? c <= j : (l == 1 ? c > j : true);
            const unsigned bad = (__ballot_sync(0xffffffffu, !ok) >> gshift) & 0x3u;
            need = bad != 0;
        } else {
            __ballot_sync(0xffffffffu, false);
        }
        if (!__any_sync(0xffffffffu, need)) break;
        if (need) { w *= 16.0; lo = mid - w; hi = mid + w; }
    }
    for (int round = 0; round < 24; ++round) {
        const bool go = active && hi - lo > stop;
        if (!__any_sync(0xffffffffu, go)) break;
        const double width = hi - lo;
        const double x = lo + width * ((double)(l + 1) / 9.0);
        const bool le = go && count(x) <= j;
        const unsigned bits = (__ballot_sync(0xffffffffu, le) >> gshift) & 0xFFu;
        if (go) {
            const int k = __popc(bits);
            const double nlo = k > 0 ? lo + width * ((double)k / 9.0) : lo;
            const double nhi = k < 8 ? lo + width * ((double)(k + 1) / 9.0) : hi;
            if (nlo <= lo && nhi >= hi) active = false;
            else { lo = nlo; hi = nhi; }
        }
    }
    if (refined && l == 0) lb[i] = 0.5 * (lo + hi);
}

// ------------------------------------------------------------ inverse iteration (FP64)
PSVD_DEV double hash_unit(unsigned a, unsigned b) {
    unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    return (double)h * (2.0 / 4294967296.0) - 1.0;
}

// Eigenvalues closer than kRefineNear ||T|| (by their FP32 values) are refined in FP64;
// Gram-Schmidt then runs only inside groups closer than kClusterTol ||T||.
constexpr double kRefineNear = 1e-5;
constexpr double kClusterTol = 1e-11;

struct InvitParams {
    const double *D, *E, *tn;
    const float4 *de;        // [b][j] = {d_j / tn, e_j / tn} as float-float pairs (e_{n-1} = 0)
    const double *lam0;      // the eigenvalues before inverse iteration (for the gaps)
    double *lam;
    double *xs, *u0, *u1, *u2, *lm;
    float *xf;               // the normalized eigenvectors, interleaved [n][stride] like xs
    unsigned *piv;           // pivot flags, bit (j % 32) of word [j / 32][t]
    int n, first, count;     // vectors [first, first + count) of the flattened (b, i) index
    long long stride;        // = chunk
};

// Each thread owns one eigenvector and walks its length-n recurrences in order.  The
// operands of every pass are streamed through a per-warp shared-memory ring with
// cp.async (kIvR stages of kIvJ rows, up to kIvNA arrays), so a warp keeps about
// (kIvR - 1) kIvJ rows of loads in flight instead of waiting on each one.  (Measured at
// n = 4096: 8 or 16 vectors per warp instead of 32 leave the time unchanged, each vector's
// chain of dependent operations sets it; plain loads prefetched 2, 4 or 8 steps ahead into
// registers instead of the ring make eigh ~11 ms slower.)
constexpr int kIvJ = 16, kIvR = 4, kIvNA = 4, kIvW = 32;
constexpr int kIvStage = kIvNA * kIvJ * kIvW;                     // doubles per stage
constexpr size_t kIvSmem = sizeof(double) * kIvR * kIvStage;      // 64 KB per warp

PSVD_DEV void cp_async8(double *sdst, const double *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
PSVD_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
PSVD_DEV void cp_async_wait_ring() { asm volatile("cp.async.wait_group %0;" ::"n"(kIvR - 2) : "memory"); }

// One streamed operand: row k lives at p + k * stride (p already at row 0; stride may be
// negative), rows k in [kmin, kmax) exist, the others are not fetched (their slots are
// left as they are and the body does not read them).
struct IvArr {
    const double *p;
    long long stride;
    int kmin, kmax;
};

// Streams `nsteps` rows of NA operands through the ring; body(k, ring slot pointer) consumes
// them in order, slot(a) = p + a*kIvJ*32.  The issuing walks one pointer per operand, so a
// row costs an add, a copy and a shared address per operand.
template <int NA, class Body>
PSVD_DEV void iv_stream(double *ring, int nsteps, const IvArr (&arr)[NA], Body body) {
    const int lane = threadIdx.x & 31;
    const int nst = (nsteps + kIvJ - 1) / kIvJ;
    const double *next[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) next[a] = arr[a].p;
    int kn = 0;                                    // row the pointers stand at
    auto issue = [&](int st) {
        if (st < nst) {
            double *buf = ring + (st % kIvR) * kIvStage + lane;
            for (int jj = 0; jj < kIvJ && kn < nsteps; ++jj, ++kn) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (kn >= arr[a].kmin && kn < arr[a].kmax) cp_async8(buf + (a * kIvJ + jj) * kIvW, next[a]);
                    next[a] += arr[a].stride;
                }
            }
        }
        cp_async_commit();
    };
    for (int st = 0; st < kIvR - 1; ++st) issue(st);
    for (int st = 0; st < nst; ++st) {
        cp_async_wait_ring();
        const double *buf = ring + (st % kIvR) * kIvStage + lane;
#pragma unroll 4
        for (int jj = 0; jj < kIvJ; ++jj) {
            const int k = st * kIvJ + jj;
            if (k >= nsteps) break;
            body(k, buf + jj * kIvW);
        }
        issue(st + kIvR - 1);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __threadfence_block();   // this pass's stores before the next pass's async reads
}
#define IV_SLOT(p, a) (p)[(a) * kIvJ * kIvW]

PSVD_DEV double iv_start(int i, int j) { return hash_unit((unsigned)i, (unsigned)j) + 0.0625; }

// Factor T - mu I = P L U (U with two superdiagonals, reciprocal pivots in u0).
PSVD_DEV void iv_factor(const InvitParams &P, double *ring, const double *D, const double *E, int n, double mu,
                        double tiny, int t) {
    const long long s = P.stride;
    double a = D[0] - mu;
    double bsup = E[0];
    unsigned word = 0;
    const IvArr arr[3] = {{D + 1, 1, 0, n - 1}, {E, 1, 0, n - 1}, {E + 1, 1, 0, n - 2}};
    iv_stream(ring, n - 1, arr,
              [&](int j, const double *p) {
                  const double c = IV_SLOT(p, 1);
                  const double dn = IV_SLOT(p, 0) - mu;
                  const double en = j + 1 < n - 1 ? IV_SLOT(p, 2) : 0.0;
                  const long long o = (long long)j * s + t;
                  if (fabs(a) >= fabs(c)) {
                      if (fabs(a) < tiny) a = a < 0 ? -tiny : tiny;
                      const double ra = recip64(a);
                      const double m = c * ra;
                      P.u0[o] = ra; P.u1[o] = bsup; P.u2[o] = 0.0; P.lm[o] = m;
                      a = dn - m * bsup;
                      bsup = en;
                  } else {
                      const double rc = recip64(c);
                      const double m = a * rc;
                      P.u0[o] = rc; P.u1[o] = dn; P.u2[o] = en; P.lm[o] = m;
                      word |= 1u << (j & 31);
                      a = bsup - m * dn;
                      bsup = -m * en;
                  }
                  if ((j & 31) == 31 || j == n - 2) { P.piv[(long long)(j >> 5) * s + t] = word; word = 0; }
              });
    if (fabs(a) < tiny) a = a < 0 ? -tiny : tiny;
    P.u0[(long long)(n - 1) * s + t] = recip64(a);
}

// Forward part of one solve: x <- P-and-L applied to b, where b = scale * x, or the
// start vector when `first`.
PSVD_DEV void iv_forward(const InvitParams &P, double *ring, int n, int t, int i, bool first, double scale) {
    const long long s = P.stride;
    double *x = P.xs;
    double carry = first ? iv_start(i, 0) : x[t] * scale;
    unsigned pword = 0;
    unsigned pnext = P.piv[t];
    const IvArr arr[2] = {{x + s + t, s, 0, first ? 0 : n - 1}, {P.lm + t, s, 0, n - 1}};
    iv_stream(ring, n - 1, arr,
              [&](int j, const double *p) {
                  if ((j & 31) == 0) {
                      pword = pnext;
                      const long long nw = (long long)((j >> 5) + 1);
                      if ((nw << 5) < n - 1) pnext = P.piv[nw * s + t];
                  }
                  double a = carry;
                  double b = first ? iv_start(i, j + 1) : IV_SLOT(p, 0) * scale;
                  if ((pword >> (j & 31)) & 1u) { const double tmp = a; a = b; b = tmp; }
                  x[(long long)j * s + t] = a;
                  carry = b - IV_SLOT(p, 1) * a;
              });
    x[(long long)(n - 1) * s + t] = carry;
}

// Backward part: U x = y in place; returns ||x||^2.
PSVD_DEV double iv_backward(const InvitParams &P, double *ring, int n, int t) {
    const long long s = P.stride;
    double *x = P.xs;
    const long long last = (long long)(n - 1) * s + t;
    double x1 = x[last] * P.u0[last], x2 = 0.0;
    x[last] = x1;
    double nrm = x1 * x1;
    const long long o0 = (long long)(n - 2) * s + t;     // row n - 2 - k at step k
    const IvArr arr[4] = {{x + o0, -s, 0, n - 1}, {P.u0 + o0, -s, 0, n - 1}, {P.u1 + o0, -s, 0, n - 1},
                          {P.u2 + o0, -s, 0, n - 1}};
    iv_stream(ring, n - 1, arr,
              [&](int k, const double *p) {
                  const double v = (IV_SLOT(p, 0) - IV_SLOT(p, 2) * x1 - IV_SLOT(p, 3) * x2) * IV_SLOT(p, 1);
                  x[(long long)(n - 2 - k) * s + t] = v;
                  x2 = x1;
                  x1 = v;
                  nrm += v * v;
              });
    return nrm;
}

// xf <- scale * x (rounded to FP32) and the Rayleigh quotient x^T T x of the scaled vector.
PSVD_DEV double iv_finish(const InvitParams &P, double *ring, const double *D, const double *E, int n, int t,
                          double scale) {
    const long long s = P.stride;
    double *x = P.xs;
    double r = 0.0, prev = 0.0;
    const IvArr arr[3] = {{x + t, s, 0, n}, {D, 1, 0, n}, {E - 1, 1, 1, n}};   // E[j - 1] from j = 1 on
    iv_stream(ring, n, arr,
              [&](int j, const double *p) {
                  const double xj = IV_SLOT(p, 0) * scale;
                  P.xf[(long long)j * s + t] = (float)xj;
                  r += IV_SLOT(p, 1) * xj * xj;
                  if (j > 0) r += 2.0 * IV_SLOT(p, 2) * prev * xj;
                  prev = xj;
              });
    return r;
}

// ------------------------------------------------ inverse iteration in float-float
// The same factorization and solves on T / tn with two-float values on the FP32 pipe, for
// vectors whose eigenvalue is at least kIvFFGap ||T|| from its neighbours.  The factors
// and the vectors between passes are stored as (hi, lo) pairs in the 8-byte slots of the
// FP64 arrays.  A factorization in ~2^-46 arithmetic is exact for a matrix within a few
// 2^-46 ||T|| of T, so these vectors are off by ~1e-13 ||T|| / gap <= 1e-7; closer
// eigenvalues keep the FP64 recurrences above.  Rounding the right-hand sides (the stored
// vectors) perturbs nothing but the start of each solve.
constexpr double kIvFFGap = 1e-6;
constexpr float kIvFFTiny = 0x1p-44f;          // pivot floor on T / tn

PSVD_DEV ff ff_sel(bool c, ff a, ff b) { return ff{c ? a.hi : b.hi, c ? a.lo : b.lo}; }
PSVD_DEV ff ff_ld(const double *slot) {
    const float2 v = *reinterpret_cast<const float2 *>(slot);
    return ff{v.x, v.y};
}
PSVD_DEV void ff_st(double *slot, ff v) { *reinterpret_cast<float2 *>(slot) = make_float2(v.hi, v.lo); }
PSVD_DEV float iv_start_f(int i, int j) {
    unsigned h = (unsigned)i * 0x9E3779B1u ^ ((unsigned)j + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    return __fmaf_rn((float)(h >> 8), 0x1p-23f, -0.9375f);          // in [-0.9375, 1.0625)
}

// Factor T/tn - mu I = P L U as iv_factor does; stored per row: u0 = 1 / pivot, u1 u0 and
// u2 u0 (the superdiagonals pre-scaled, so that each back-substitution step is one
// dependent multiply-add), and the multiplier.  The pivot choice and both row orders are
// evaluated with selects (no divergence inside the warp).
PSVD_DEV void ivf_factor(const InvitParams &P, double *ring, const float4 *de, int n, ff mu, int t) {
    const long long s = P.stride;
    const float4 r0 = de[0];
    ff a = ff_add(ff{r0.x, r0.y}, ff_neg(mu));
    ff bs = ff{r0.z, r0.w};
    unsigned word = 0;
    const double *dd = reinterpret_cast<const double *>(de);     // (d, e) pairs: 2 slots per row
    const IvArr arr[3] = {{dd + 2, 2, 0, n - 1}, {dd + 1, 2, 0, n - 1}, {dd + 3, 2, 0, n - 1}};
    iv_stream(ring, n - 1, arr,
              [&](int j, const double *p) {
                  const ff dn = ff_add(ff_ld(&IV_SLOT(p, 0)), ff_neg(mu));
                  const ff c = ff_ld(&IV_SLOT(p, 1));
                  const ff en = ff_ld(&IV_SLOT(p, 2));
                  const bool pv = fabsf(a.hi) < fabsf(c.hi);
                  ff den = ff_sel(pv, c, a);
                  if (fabsf(den.hi) < kIvFFTiny) den = ff{den.hi < 0.f ? -kIvFFTiny : kIvFFTiny, 0.f};
                  const ff m = ff_div(ff_sel(pv, a, c), den);
                  const ff rp = ff_div(ff{1.f, 0.f}, den);
                  const ff y = ff_sel(pv, dn, bs);
                  a = ff_add(ff_sel(pv, bs, dn), ff_neg(ff_mul(m, y)));
                  const ff me = ff_mul(m, en);
                  const ff u2 = pv ? en : ff{0.f, 0.f};
                  bs = ff_sel(pv, ff_neg(me), en);
                  const long long o = (long long)j * s + t;
                  ff_st(P.u0 + o, rp);
                  ff_st(P.u1 + o, ff_mul(y, rp));
                  ff_st(P.u2 + o, ff_mul(u2, rp));
                  ff_st(P.lm + o, m);
                  word |= (unsigned)pv << (j & 31);
                  if ((j & 31) == 31 || j == n - 2) { P.piv[(long long)(j >> 5) * s + t] = word; word = 0; }
              });
    if (fabsf(a.hi) < kIvFFTiny) a = ff{a.hi < 0.f ? -kIvFFTiny : kIvFFTiny, 0.f};
    ff_st(P.u0 + (long long)(n - 1) * s + t, ff_div(ff{1.f, 0.f}, a));
}

// Forward part of one solve (the pivots and L), right-hand side scale * x or the start vector.
PSVD_DEV void ivf_forward(const InvitParams &P, double *ring, int n, int t, int i, bool first, float scale) {
    const long long s = P.stride;
    double *x = P.xs;
    ff carry = first ? ff{iv_start_f(i, 0), 0.f} : ff_mulf(ff_ld(x + t), scale);
    unsigned pword = 0;
    unsigned pnext = P.piv[t];
    const IvArr arr[2] = {{x + s + t, s, 0, first ? 0 : n - 1}, {P.lm + t, s, 0, n - 1}};
    iv_stream(ring, n - 1, arr,
              [&](int j, const double *p) {
                  if ((j & 31) == 0) {
                      pword = pnext;
                      const long long nw = (long long)((j >> 5) + 1);
                      if ((nw << 5) < n - 1) pnext = P.piv[nw * s + t];
                  }
                  const ff bn = first ? ff{iv_start_f(i, j + 1), 0.f} : ff_mulf(ff_ld(&IV_SLOT(p, 0)), scale);
                  const bool sw = (pword >> (j & 31)) & 1u;
                  const ff a = ff_sel(sw, bn, carry);
                  const ff b = ff_sel(sw, carry, bn);
                  ff_st(x + (long long)j * s + t, a);
                  carry = ff_add(b, ff_neg(ff_mul(ff_ld(&IV_SLOT(p, 1)), a)));
              });
    ff_st(x + (long long)(n - 1) * s + t, carry);
}

// Backward part: U x = y in place; returns ||x||^2 (float-float).
PSVD_DEV ff ivf_backward(const InvitParams &P, double *ring, int n, int t) {
    const long long s = P.stride;
    double *x = P.xs;
    const long long last = (long long)(n - 1) * s + t;
    ff x1 = ff_mul(ff_ld(x + last), ff_ld(P.u0 + last)), x2 = ff{0.f, 0.f};
    ff_st(x + last, x1);
    ff nrm = ff_fma(ff_zero(), x1.hi, x1.hi);
    const long long o0 = (long long)(n - 2) * s + t;     // row n - 2 - k at step k
    const IvArr arr[4] = {{x + o0, -s, 0, n - 1}, {P.u0 + o0, -s, 0, n - 1}, {P.u1 + o0, -s, 0, n - 1},
                          {P.u2 + o0, -s, 0, n - 1}};
    iv_stream(ring, n - 1, arr,
              [&](int k, const double *p) {
                  ff r = ff_mul(ff_ld(&IV_SLOT(p, 0)), ff_ld(&IV_SLOT(p, 1)));
                  r = ff_add(r, ff_neg(ff_mul(ff_ld(&IV_SLOT(p, 3)), x2)));
                  const ff v = ff_add(r, ff_neg(ff_mul(ff_ld(&IV_SLOT(p, 2)), x1)));
                  ff_st(x + (long long)(n - 2 - k) * s + t, v);
                  x2 = x1;
                  x1 = v;
                  nrm = ff_fma(nrm, v.hi, v.hi);
              });
    return nrm;
}

// xf <- scale * x (FP32) and the Rayleigh quotient x^T (T/tn) x / x^T x of that vector.
PSVD_DEV double ivf_finish(const InvitParams &P, double *ring, const float4 *de, int n, int t, float scale) {
    const long long s = P.stride;
    const double *x = P.xs;
    const double *dd = reinterpret_cast<const double *>(de);
    ff num = ff_zero(), den = ff_zero();
    float prev = 0.f;
    const IvArr arr[3] = {{x + t, s, 0, n}, {dd, 2, 0, n}, {dd - 1, 2, 1, n}};   // e_{j-1} from j = 1 on
    iv_stream(ring, n, arr,
              [&](int j, const double *p) {
                  const float xj = __fmul_rn(__fadd_rn(ff_ld(&IV_SLOT(p, 0)).hi, ff_ld(&IV_SLOT(p, 0)).lo), scale);
                  P.xf[(long long)j * s + t] = xj;
                  // x_j (d_j x_j + 2 e_{j-1} x_{j-1})
                  ff q = ff_mulf(ff_ld(&IV_SLOT(p, 1)), xj);
                  if (j > 0) q = ff_add(q, ff_mulf(ff_ld(&IV_SLOT(p, 2)), __fmul_rn(2.f, prev)));
                  num = ff_add(num, ff_mulf(q, xj));
                  den = ff_fma(den, xj, xj);
                  prev = xj;
              });
    return ((double)num.hi + (double)num.lo) / ((double)den.hi + (double)den.lo);
}

// One warp per block: 32 eigenvectors, each by inverse iteration from a fixed
// pseudo-random start.  The bisection shift is accurate to ~1e-7 ||T||: three solves
// reduce the other components by (shift error / gap)^3.  A warp whose 32 eigenvalues are
// all at least kIvFFGap ||T|| from their neighbours runs the float-float recurrences, the
// others the FP64 ones (the choice is per warp, so no warp runs both).
__global__ void __launch_bounds__(kIvW) tri_invit_kernel(InvitParams P) {
    extern __shared__ __align__(16) double ivring[];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = P.n;
    const long long gi = (long long)P.first + t;
    const int b = (int)(gi / n), i = (int)(gi % n);
    bool ffok = true;
    double tn = 0.0;
    if (t < P.count) {
        tn = P.tn[b];
        const double *lb = P.lam0 + (long long)b * n;
        double g = 1e300;
        if (i > 0) g = fmin(g, lb[i - 1] - lb[i]);
        if (i + 1 < n) g = fmin(g, lb[i] - lb[i + 1]);
        ffok = n > 1 && tn > 0.0 && g >= kIvFFGap * tn;
    }
    const bool use_ff = __all_sync(0xffffffffu, ffok);
    if (t >= P.count) return;
    const long long s = P.stride;
    const double mu = P.lam[gi];
    if (use_ff) {
        const float4 *de = P.de + (long long)b * n;
        const double ms = mu / tn;
        const float mh = (float)ms;
        ivf_factor(P, ivring, de, n, ff{mh, (float)(ms - (double)mh)}, t);
        float scale = 1.f;
        for (int it = 0; it < 3; ++it) {
            ivf_forward(P, ivring, n, t, i, it == 0, scale);
            const ff nrm = ivf_backward(P, ivring, n, t);
            const double nv = (double)nrm.hi + (double)nrm.lo;
            scale = nv > 0.0 ? (float)(1.0 / sqrt(nv)) : 0.f;
        }
        P.lam[gi] = ivf_finish(P, ivring, de, n, t, scale) * tn;
        return;
    }
    const double *D = P.D + (long long)b * n, *E = P.E + (long long)b * n;
    if (n == 1) { P.xf[t] = 1.f; return; }
    if (!(tn > 0.0)) {
        // T = 0: every vector is an eigenvector; take the unit vectors
        for (int j = 0; j < n; ++j) P.xf[j * s + t] = j == i ? 1.f : 0.f;
        P.lam[gi] = 0.0;
        return;
    }
    const double tiny = fmax(tn * 2.2e-16, 1e-280);
    iv_factor(P, ivring, D, E, n, mu, tiny, t);
    double scale = 1.0;
    for (int it = 0; it < 3; ++it) {
        iv_forward(P, ivring, n, t, i, it == 0, scale);
        const double nrm = iv_backward(P, ivring, n, t);
        scale = nrm > 0 ? 1.0 / sqrt(nrm) : 0.0;
    }
    P.lam[gi] = iv_finish(P, ivring, D, E, n, t, scale);
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
    // links: bit i set when eigenvalues i - 1 and i are closer than tol; found in parallel,
    // so that the walk below only visits clusters (most spectra have none)
    constexpr int kLinkWords = 2048;
    __shared__ unsigned link[kLinkWords];
    const bool fits = n <= 32 * kLinkWords;
    int any = 1;
    if (fits) {
        for (int q = threadIdx.x; q < (n + 31) / 32; q += blockDim.x) link[q] = 0u;
        __syncthreads();
        int mine = 0;
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x)
            if (bl[i - 1] - bl[i] <= tol) { atomicOr(&link[i >> 5], 1u << (i & 31)); mine = 1; }
        any = __syncthreads_or(mine);
    }
    int i0 = 0;
    while (any && i0 < n) {
        if (fits) {                  // skip to the first link after i0 (bits are read-only now)
            int i = i0 + 1;
            while (i < n) {
                const unsigned wd = link[i >> 5] >> (i & 31);
                if (wd) { i += __ffs(wd) - 1; break; }
                i = (i | 31) + 1;
            }
            if (i >= n) break;
            i0 = i - 1;
        }
        int i1 = i0 + 1;
        if (fits) { while (i1 < n && ((link[i1 >> 5] >> (i1 & 31)) & 1u)) ++i1; }
        else { while (i1 < n && bl[i1 - 1] - bl[i1] <= tol) ++i1; }
        if (i1 - i0 >= 2) {
            for (int i = i0; i < i1; ++i) {
                const int ti = base + i;
                float *xf = P.xf;
                for (int l = i0; l < i; ++l) {
                    const int tl = base + l;
                    double dot = 0.0;
                    for (int j = threadIdx.x; j < n; j += blockDim.x)
                        dot += (double)xf[j * s + ti] * (double)xf[j * s + tl];
                    dot = block_sum(dot, red);
                    for (int j = threadIdx.x; j < n; j += blockDim.x)
                        xf[j * s + ti] = (float)((double)xf[j * s + ti] - dot * (double)xf[j * s + tl]);
                    __syncthreads();
                }
                double nr = 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) nr += (double)xf[j * s + ti] * (double)xf[j * s + ti];
                nr = block_sum(nr, red);
                const double inv = nr > 0 ? 1.0 / sqrt(nr) : 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) xf[j * s + ti] = (float)((double)xf[j * s + ti] * inv);
                __syncthreads();
                double r = 0.0;
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const double xj = xf[j * s + ti];
                    r += D[j] * xj * xj;
                    if (j + 1 < n) r += 2.0 * E[j] * xj * (double)xf[(j + 1) * s + ti];
                }
                r = block_sum(r, red);
                if (threadIdx.x == 0) P.lam[(long long)b * n + i] = r;
                __syncthreads();
            }
        }
        i0 = i1;
    }
    __syncthreads();
    // descending order: l[i] <- min(l[0..i]) (a running minimum), as a block scan: each thread
    // takes a contiguous segment, the segment minima are scanned in shared memory, then every
    // thread applies its prefix
    __shared__ double segmin[1024];
    double *l = P.lam + (long long)b * n;
    const int T = blockDim.x, seg = (n + T - 1) / T;
    const int s0 = min(n, (int)threadIdx.x * seg), s1 = min(n, s0 + seg);
    double mn = INFINITY;
    for (int i = s0; i < s1; ++i) mn = fmin(mn, l[i]);
    segmin[threadIdx.x] = mn;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 1; t < T; ++t) segmin[t] = fmin(segmin[t], segmin[t - 1]);
    __syncthreads();
    double run = threadIdx.x > 0 ? segmin[threadIdx.x - 1] : INFINITY;
    for (int i = s0; i < s1; ++i) {
        const double v = fmin(run, l[i]);
        if (v != l[i]) l[i] = v;
        run = v;
    }
}

// Z^T rows (eigenvectors of T) from the interleaved FP32 vectors -> V^T split (n x ldn)
__global__ void zt_store_kernel(const float *xs, long long stride, int n, int first_b, int first, float *VThi,
                                float *VTlo, long long ldn) {
    __shared__ float tile[32][33];
    const int bb = blockIdx.z;
    const int b = first_b + bb;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;   // i: eigen index, j: component
    const long long tb = (long long)b * n - first;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (j < n && i < n) ? xs[(long long)j * stride + tb + i] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < n && j < n) {
            float h, l;
            split_tf32(tile[threadIdx.x][r], h, l);
            const long long o = (long long)b * n * ldn + (long long)i * ldn + j;
            VThi[o] = h;
            VTlo[o] = l;
        }
    }
}

// ------------------------------------------------------------ back-transform
// Upper-triangular T of the forward compact-WY form H_k0 ... H_k1-1 = I - Y T Y^T, one
// block per (WY block, matrix), from G = Y^T Y (computed on the tensor cores, symmetric).
// Splitting the block's reflectors into halves a, b gives T = [T_aa, -T_aa G_ab T_bb; 0, T_bb],
// so T is built by recursive halving: the four 32 x 32 diagonal blocks column by column
// (T[i][c] = -tau_c sum_{i <= k < c} T[i][k] G[k][c], one warp per block, lane i holding row
// i in registers), then the off-diagonal blocks of the 64- and 128-wide levels as two small
// products each.  The serial depth is 32 columns instead of 128.
static_assert(kWY % 32 == 0 && (kWY & (kWY - 1)) == 0 && kWY / 32 <= 8, "larft halving assumes 32 x 2^j reflectors");
constexpr int kLtLd = kWY + 1;                  // padded row stride of G and T in shared memory
constexpr size_t kLtSmem = sizeof(float) * ((size_t)2 * kWY * kLtLd + (kWY / 2) * (kWY / 2) + kWY);
__global__ void __launch_bounds__(256) larft_kernel(const float *Gm, const float *tau, int n, int nblk, float *Tm) {
    extern __shared__ float sm2[];
    float *G = sm2, *T = G + kWY * kLtLd, *W = T + kWY * kLtLd, *ts = W + (kWY / 2) * (kWY / 2);
    const int blk = blockIdx.x, b = blockIdx.y;
    const int k0 = blk * kWY;
    const int nb = min(kWY, n - 2 - k0);
    const float *Gb = Gm + ((long long)b * nblk + blk) * kWY * kWY;
    for (int p = threadIdx.x; p < kWY * kWY; p += blockDim.x) {
        const int r = p / kWY, c = p % kWY;
        G[r * kLtLd + c] = Gb[p];
        T[r * kLtLd + c] = 0.f;
    }
    for (int c = threadIdx.x; c < kWY; c += blockDim.x) ts[c] = c < nb ? tau[(long long)b * n + k0 + c] : 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < kWY / 32) {
        const int o = 32 * warp, i = lane;
        float tr[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < c; ++k)
                if (k >= i) s = fmaf(tr[k], G[(o + k) * kLtLd + o + c], s);
            tr[c] = c < i ? 0.f : (c == i ? ts[o + c] : -ts[o + c] * s);
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) T[(o + i) * kLtLd + o + c] = tr[c];
    }
    __syncthreads();
    for (int h = 32; h < kWY; h *= 2) {
        const int np = kWY / (2 * h), hh = h * h;
        // W_p = G[a:a+h, b:b+h] T[b:b+h, b:b+h]   (a = 2 h p, b = a + h; T_bb upper triangular)
        for (int e = threadIdx.x; e < np * hh; e += blockDim.x) {
            const int p = e / hh, r = (e / h) % h, j = e % h;
            const int a = 2 * h * p, bb = a + h;
            float s = 0.f;
            for (int k = 0; k <= j; ++k) s = fmaf(G[(a + r) * kLtLd + bb + k], T[(bb + k) * kLtLd + bb + j], s);
            W[e] = s;
        }
        __syncthreads();
        // T[a:a+h, b:b+h] = -T[a:a+h, a:a+h] W_p   (T_aa upper triangular)
        for (int e = threadIdx.x; e < np * hh; e += blockDim.x) {
            const int p = e / hh, r = (e / h) % h, j = e % h;
            const int a = 2 * h * p, bb = a + h;
            const float *wp = W + p * hh;
            float s = 0.f;
            for (int k = r; k < h; ++k) s = fmaf(T[(a + r) * kLtLd + a + k], wp[k * h + j], s);
            T[(a + r) * kLtLd + bb + j] = -s;
        }
        __syncthreads();
    }
    float *out = Tm + ((long long)b * nblk + blk) * kWY * kWY;
    for (int p = threadIdx.x; p < kWY * kWY; p += blockDim.x) out[p] = T[(p / kWY) * kLtLd + p % kWY];
}

// S2 = S T^T (n x nb), split into TF32 hi/lo; S is the sum of `ks` K-split slices of
// B x n x kWY each, added in slice order.  One block of kWY threads per kStRows rows of S:
// T is staged once per block in shared memory with rows padded to kWY + 1 floats (thread j
// reads row j, so the lanes of a warp hit distinct banks), and each thread forms output
// column j of all kStRows rows.
constexpr int kStRows = 16;
constexpr size_t kStSmem = sizeof(float) * ((size_t)kWY * (kWY + 1) + (size_t)kStRows * kWY);
__global__ void __launch_bounds__(kWY) s_times_tt_kernel(const float *S, int ks, int B, const float *Tm, int n,
                                                         int nblk, int blk, int nb, float *S2hi, float *S2lo) {
    extern __shared__ float stsm[];
    float *Ts = stsm, *sr = stsm + kWY * (kWY + 1);
    const int i0 = blockIdx.x * kStRows, b = blockIdx.y, j = threadIdx.x;
    const float *Tb = Tm + ((long long)b * nblk + blk) * kWY * kWY;
    // T (kWY x kWY, 16-byte aligned rows) as float4 loads, eight in flight per thread
    const float4 *T4 = reinterpret_cast<const float4 *>(Tb);
    for (int q0 = j; q0 < kWY * kWY / 4; q0 += 8 * kWY) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = q0 + u * kWY < kWY * kWY / 4 ? T4[q0 + u * kWY] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * kWY;
            if (q >= kWY * kWY / 4) break;
            float *d = Ts + (4 * q / kWY) * (kWY + 1) + (4 * q) % kWY;
            d[0] = v[u].x; d[1] = v[u].y; d[2] = v[u].z; d[3] = v[u].w;
        }
    }
    // the kStRows rows of S, every slice's load issued before the sums
    const long long slice = (long long)B * n * kWY;
#pragma unroll
    for (int r = 0; r < kStRows; ++r) {
        const int i = i0 + r;
        float sv = 0.f;
        if (i < n) {
            const long long o = (long long)b * n * kWY + (long long)i * kWY + j;
            float x[kBtSplit];
#pragma unroll
            for (int c = 0; c < kBtSplit; ++c) x[c] = c < ks ? S[c * slice + o] : 0.f;
            sv = x[0];
#pragma unroll
            for (int c = 1; c < kBtSplit; ++c) if (c < ks) sv += x[c];
        }
        sr[r * kWY + j] = sv;
    }
    __syncthreads();
    float acc[kStRows];
#pragma unroll
    for (int r = 0; r < kStRows; ++r) acc[r] = 0.f;
    if (j < nb)
        for (int l = j; l < nb; ++l) {
            const float t = Ts[j * (kWY + 1) + l];
#pragma unroll
            for (int r = 0; r < kStRows; ++r) acc[r] += sr[r * kWY + l] * t;
        }
#pragma unroll
    for (int r = 0; r < kStRows; ++r) {
        const int i = i0 + r;
        if (i >= n) break;
        const long long o = (long long)b * n * kWY + (long long)i * kWY + j;
        float h, lo;
        split_tf32(acc[r], h, lo);
        S2hi[o] = h;
        S2lo[o] = lo;
    }
}

// Two compact-WY blocks in one update (b = a block, a = the block above it, applied first):
//   M (I - Y_a T_a^T Y_a^T)(I - Y_b T_b^T Y_b^T) = M - S2_a Y_a^T - S2_b Y_b^T,
//   S2_a = S_a T_a^T,  S2_b = (S_b' - S2_a G_ab) T_b^T,
// with S_a = M Y_a and S_b' = M Y_b from one product (S: columns [0, kWY) block b, [kWY, 2 kWY)
// block a, the sum of ks K-split slices) and G_ab = Y_a^T Y_b.  S2 gets the same column order.
// One block of 2 kWY threads per kPrRows rows (each thread one column of half the rows):
// T_a and G_ab^T staged in shared memory with rows padded to kPrLd floats, so that a thread
// reads 4 consecutive entries of its row as one float4 and the rows of S as float4
// broadcasts; T_b replaces T_a once the first phase is done.  With two matrices resident,
// 28 rows per block fit, so n = 4096 takes 147 blocks: one wave on the SMs.  T is upper
// triangular and zero past its block's width, and S is zeroed past the pair's width, so
// the sums run over whole float4s.
constexpr int kPrRows = 28, kPrLd = kWY + 4;
static_assert(kPrRows % 2 == 0, "two halves of the rows");
constexpr size_t kPrSmem =
    sizeof(float) * (2 * (size_t)kWY * kPrLd + (size_t)kPrRows * 2 * kWY + (size_t)kPrRows * kWY);
__global__ void __launch_bounds__(2 * kWY) s_pair_kernel(const float *S, int ks, int B, const float *Tm,
                                                          const float *Gab, int n, int nblk, int npair, int blk_b,
                                                          int q, int nb_a, float *S2hi, float *S2lo) {
    extern __shared__ __align__(16) float psm[];
    float *Ta = psm, *Gt = Ta + kWY * kPrLd, *Tb = Ta;  // T_b is loaded over T_a after phase one
    float *sr = Gt + kWY * kPrLd;                     // [kPrRows][2 kWY]: S rows, then S_b in place
    float *s2a = sr + kPrRows * 2 * kWY;              // [kPrRows][kWY]
    const int i0 = blockIdx.x * kPrRows, b = blockIdx.y, t = threadIdx.x;
    const int W = kWY + nb_a;
    // a kWY x kWY matrix (16-byte aligned rows) as float4 loads, eight in flight, into rows
    // padded to kPrLd; G_ab is stored transposed (row j of Gt = column j of G_ab)
    auto stage = [&](const float *src, float *dst, bool transposed) {
        const float4 *g4 = reinterpret_cast<const float4 *>(src);
        for (int q0 = t; q0 < kWY * kWY / 4; q0 += 8 * 2 * kWY) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = q0 + u * 2 * kWY < kWY * kWY / 4 ? g4[q0 + u * 2 * kWY] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = 4 * (q0 + u * 2 * kWY);
                if (e >= kWY * kWY) break;
                const int r = e / kWY, c = e % kWY;
                const float x[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                if (!transposed) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) dst[r * kPrLd + c + h] = x[h];
                } else {
#pragma unroll
                    for (int h = 0; h < 4; ++h) dst[(c + h) * kPrLd + r] = x[h];
                }
            }
        }
    };
    stage(Tm + ((long long)b * nblk + blk_b + 1) * kWY * kWY, Ta, false);
    stage(Gab + ((long long)b * npair + q) * kWY * kWY, Gt, true);
    const long long slice = (long long)B * n * 2 * kWY;
#pragma unroll
    for (int r = 0; r < kPrRows; ++r) {
        const int i = i0 + r;
        float sv = 0.f;
        if (i < n && t < W) {
            const long long o = ((long long)b * n + i) * 2 * kWY + t;
            float x[kBtSplit];
#pragma unroll
            for (int c = 0; c < kBtSplit; ++c) x[c] = c < ks ? S[c * slice + o] : 0.f;
            sv = x[0];
#pragma unroll
            for (int c = 1; c < kBtSplit; ++c) if (c < ks) sv += x[c];
        }
        sr[r * 2 * kWY + t] = sv;
    }
    __syncthreads();
    // every phase: thread t takes column j = t % kWY of the kPrRows / 2 rows of half t / kWY
    constexpr int kH = kPrRows / 2;
    const int j = t % kWY, rh = (t / kWY) * kH;
    const int na4 = (nb_a + 3) & ~3;
    auto dot4 = [](float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; };
    float acc[kH];
#pragma unroll
    for (int r = 0; r < kH; ++r) acc[r] = 0.f;
    for (int l = j & ~3; l < na4; l += 4) {          // S2_a = S_a T_a^T
        const float4 tv = *reinterpret_cast<const float4 *>(Ta + j * kPrLd + l);
#pragma unroll
        for (int r = 0; r < kH; ++r)
            acc[r] += dot4(*reinterpret_cast<const float4 *>(sr + (rh + r) * 2 * kWY + kWY + l), tv);
    }
#pragma unroll
    for (int r = 0; r < kH; ++r) s2a[(rh + r) * kWY + j] = acc[r];
    __syncthreads();                                 // T_a is no longer read: T_b takes its place
    stage(Tm + ((long long)b * nblk + blk_b) * kWY * kWY, Tb, false);
#pragma unroll
    for (int r = 0; r < kH; ++r) acc[r] = sr[(rh + r) * 2 * kWY + j];
    for (int l = 0; l < na4; l += 4) {               // S_b = S_b' - S2_a G_ab
        const float4 gv = *reinterpret_cast<const float4 *>(Gt + j * kPrLd + l);
#pragma unroll
        for (int r = 0; r < kH; ++r) acc[r] -= dot4(*reinterpret_cast<const float4 *>(s2a + (rh + r) * kWY + l), gv);
    }
    __syncthreads();                                 // every thread has read S_b' before it is replaced
#pragma unroll
    for (int r = 0; r < kH; ++r) sr[(rh + r) * 2 * kWY + j] = acc[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kH; ++r) acc[r] = 0.f;
    for (int l = j & ~3; l < kWY; l += 4) {          // S2_b = S_b T_b^T (block b is full)
        const float4 tv = *reinterpret_cast<const float4 *>(Tb + j * kPrLd + l);
#pragma unroll
        for (int r = 0; r < kH; ++r) acc[r] += dot4(*reinterpret_cast<const float4 *>(sr + (rh + r) * 2 * kWY + l), tv);
    }
#pragma unroll
    for (int r = 0; r < kH; ++r) {
        const int i = i0 + rh + r;
        if (i >= n) break;
        const long long o = ((long long)b * n + i) * 2 * kWY;
        float h, lo;
        split_tf32(acc[r], h, lo);
        S2hi[o + j] = h;
        S2lo[o + j] = lo;
        split_tf32(s2a[(rh + r) * kWY + j], h, lo);
        S2hi[o + kWY + j] = h;
        S2lo[o + kWY + j] = lo;
    }
}

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
// CTAs per matrix for the tridiagonalization and matrices in flight.
static int trd_ctas_per_group(int n) {
    return std::max(1, std::min(std::min(PSVD_TRD_MINB * num_sms(), 320), n / PSVD_TRD_ROWDIV));
}

int eigh_groups(int B, int n) {
    const int g = trd_ctas_per_group(n);
    return std::max(1, std::min(B, (PSVD_TRD_MINB * num_sms()) / g));
}

int eigh_forward(const float *Hs, float *S, float *VT, EighWS &w, cudaStream_t st) {
    const int B = w.B, n = w.n;
    const long long ldn = w.ldn;
    PSVD_TRY(cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * (size_t)w.groups * (trd_ctas_per_group(n) + 1), st));
    PSVD_TRY(cudaMemsetAsync(w.err, 0, sizeof(unsigned) * 4, st));
    PSVD_TRY(cudaMemsetAsync(w.e, 0, sizeof(double) * (size_t)B * n, st));
    PSVD_TRY(cudaMemsetAsync(w.Vh, 0, sizeof(float) * (size_t)B * w.nrp * ldn, st));
    // 1. tridiagonalization
    {
        TrdParams P;
        P.H = Hs; P.Aw = w.Aw; P.Vh = w.Vh; P.tau = w.tau; P.d = w.d; P.e = w.e; P.pbuf = w.pbuf;
        P.bar = w.bar; P.err = w.err; P.B = B; P.n = n; P.groups = w.groups; P.g = trd_ctas_per_group(n); P.nrp = w.nrp;
        P.ldn = ldn;
        P.spin = barrier_spin();
        const size_t smem = sizeof(float) * 3 * (size_t)ldn;
        PSVD_TRY(cudaFuncSetAttribute(sytrd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int occ = 0;
        PSVD_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sytrd_kernel, kTrdThreads, smem));
        if (occ * num_sms() < w.groups * P.g) return cuda_fail(cudaErrorCooperativeLaunchTooLarge, __FILE__, __LINE__);
        void *args[] = {&P};
        const bool prof = prof_on();
        if (prof) prof_begin(st);
        PSVD_TRY(cudaLaunchCooperativeKernel((void *)sytrd_kernel, dim3(w.groups * P.g), dim3(kTrdThreads), args,
                                             smem, st));
        count_launch(1);
        if (prof) {
            const double j = (double)std::max(0, n - 2);   // sum_{t=1}^{n-2} 8 t^2
            prof_end(st, 8.0 * j * (j + 1) * (2 * j + 1) / 6.0 * B, PSVD_PROF_TRD);
        }
    }
    // 2. eigenvalues
    double *tn = reinterpret_cast<double *>(w.S2hi);   // B doubles of scratch (S2 is free until stage 4)
    {
        dim3 g((n + 31) / 32, B);       // 32 eigenvalues x 8 lanes per block
        const size_t smem = sizeof(float) * 2 * (size_t)n;
        PSVD_TRY(cudaFuncSetAttribute(tri_bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tri_bisect_kernel<<<g, 256, smem, st>>>(w.d, w.e, n, w.lam, tn);
        PSVD_TRY(cudaGetLastError());
        count_launch(1);
    }
    {
        float4 *dd = reinterpret_cast<float4 *>(w.S2lo);   // 2 x B x n float4 (S2 is free until stage 4)
        sturm_prep_kernel<<<dim3((n + 255) / 256, B), 256, 0, st>>>(w.d, w.e, tn, n, dd, dd + (size_t)B * n);
        dim3 g((n + 31) / 32, B);       // 32 eigenvalues x 8 lanes per block
        tri_refine_kernel<<<g, 256, 0, st>>>(dd, n, tn, kRefineNear, w.lam);
        PSVD_TRY(cudaGetLastError());
        count_launch(2);
    }
    // keep the eigenvalues for cluster detection
    double *bis = reinterpret_cast<double *>(w.S);   // B*n doubles (S holds B*n*kWY floats)
    PSVD_TRY(cudaMemcpyAsync(bis, w.lam, sizeof(double) * (size_t)B * n, cudaMemcpyDeviceToDevice, st));
    // 3. eigenvectors of T, chunk by chunk (chunks hold whole matrices)
    PSVD_TRY(cudaFuncSetAttribute(tri_invit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIvSmem));
    const int per = std::max(1, w.chunk / n);
    for (int b0 = 0; b0 < B; b0 += per) {
        const int nb = std::min(per, B - b0);
        InvitParams P;
        P.D = w.d; P.E = w.e; P.tn = tn; P.lam = w.lam; P.lam0 = bis;
        P.de = reinterpret_cast<const float4 *>(w.S2lo) + (size_t)B * n;
        P.xs = w.xs; P.xf = w.xf; P.u0 = w.u0; P.u1 = w.u1; P.u2 = w.u2; P.lm = w.lm; P.piv = w.piv;
        P.n = n; P.first = b0 * n; P.count = nb * n; P.stride = w.chunk;
        tri_invit_kernel<<<(P.count + kIvW - 1) / kIvW, kIvW, kIvSmem, st>>>(P);
        tri_cluster_kernel<<<nb, 256, 0, st>>>(P, bis, kClusterTol);
        dim3 g((n + 31) / 32, (n + 31) / 32, nb), blk(32, 8);
        zt_store_kernel<<<g, blk, 0, st>>>(w.xf, w.chunk, n, b0, b0 * n, w.VThi, w.VTlo, ldn);
        PSVD_TRY(cudaGetLastError());
        count_launch(3);
    }
    // 4. back-transform V^T = Z^T H_{n-3} ... H_0, compact-WY blocks in descending order
    if (w.nblk > 0) {
        SplitOut vo, yo;
        const long long np = (long long)w.nrp * ldn;
        vo.hi = w.Vhi; vo.lo = w.Vlo; vo.ld = ldn; vo.bstride = np;
        yo.hi = w.Yhi; yo.lo = w.Ylo; yo.ld = ldn; yo.bstride = (long long)n * ldn;
        PSVD_TRY(prepare_operand(w.Vh, ldn, np, B, w.nrp, n, false, 1.f, nullptr, vo, st));
        PSVD_TRY(prepare_operand(w.Vh, ldn, np, B, n, n, true, 1.f, nullptr, yo, st));
        // G = Y^T Y of every WY block: blocks of kWY Householder rows as a batch
        for (int b = 0; b < B; ++b) {
            MatView vh = view_of(w.Vhi + b * np, kWY, n, ldn, (long long)kWY * ldn, w.nblk);
            MatView vl = view_of(w.Vlo + b * np, kWY, n, ldn, (long long)kWY * ldn, w.nblk);
            GemmShape s;
            memset(&s, 0, sizeof(s));
            s.M = kWY; s.N = kWY; s.K = n; s.prec_uniform = PREC_TF32X3; s.err = w.err;
            EpiStore e = epi_store_plain(w.Gm + (long long)b * w.nblk * kWY * kWY, kWY, (long long)kWY * kWY, kWY, kWY);
            PSVD_TRY(launch_gemm(nullptr, nullptr, &vh, &vl, &vh, &vl, s, w.nblk, e, st));
        }
        PSVD_TRY(cudaFuncSetAttribute(larft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLtSmem));
        larft_kernel<<<dim3(w.nblk, B), 256, kLtSmem, st>>>(w.Gm, w.tau, n, w.nblk, w.Tm);
        PSVD_TRY(cudaFuncSetAttribute(s_times_tt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStSmem));
        PSVD_TRY(cudaGetLastError());
        count_launch(1);
        // The blocks are applied in pairs (s_pair_kernel): one V^T Y product of width 2 kWY and
        // one update with K = 2 kWY per pair halve the read-modify-write passes over V^T.
        // With an odd count the lowest block (blk 0) goes last on its own.
        const int first = w.nblk & 1, npair = w.nblk / 2;
        auto single = [&](int blk) -> int {
            const int k0 = blk * kWY;
            const int nb = std::min(kWY, n - 2 - k0);
            const int r0 = ((k0 + 1) / 32) * 32;
            const int Lr = n - r0;
            int ks = 1;
            // S = V^T[:, r0:] Y[r0:, blk]   (n x nb), as ks partial sums over K
            {
                MatView ahi = view_of(w.VThi + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView alo = view_of(w.VTlo + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView bhi = view_of(w.Vhi + (long long)k0 * ldn + r0, nb, Lr, ldn, (long long)w.nrp * ldn, B);
                MatView blo = view_of(w.Vlo + (long long)k0 * ldn + r0, nb, Lr, ldn, (long long)w.nrp * ldn, B);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = n; s.N = nb; s.K = Lr; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                // N = nb <= 128 leaves ceil(n / 128) tiles per matrix: split K so that about
                // one wave of CTAs runs, at least 4 k-blocks per range
                const int tiles = ((n + kBM - 1) / kBM) * B;
                s.ksplit = std::max(1, std::min(std::min(kBtSplit, (num_sms() + tiles - 1) / tiles), Lr / 128));
                ks = s.ksplit;
                EpiStore e = epi_store_plain(w.S, kWY, (long long)n * kWY, n, nb);
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st));
            }
            {
                s_times_tt_kernel<<<dim3((n + kStRows - 1) / kStRows, B), kWY, kStSmem, st>>>(w.S, ks, B, w.Tm, n,
                                                                                            w.nblk, blk, nb, w.S2hi,
                                                                                            w.S2lo);
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
            return PSVD_OK;
        };
        if (npair > 0) {
            // G_ab = Y_a^T Y_b of every pair (a = b + 1): Householder rows of the two blocks
            for (int b = 0; b < B; ++b) {
                const float *hb = w.Vhi + b * np, *lb = w.Vlo + b * np;
                const long long ps = (long long)2 * kWY * ldn;
                MatView ah = view_of(hb + (long long)(first + 1) * kWY * ldn, kWY, n, ldn, ps, npair);
                MatView al = view_of(lb + (long long)(first + 1) * kWY * ldn, kWY, n, ldn, ps, npair);
                MatView bh = view_of(hb + (long long)first * kWY * ldn, kWY, n, ldn, ps, npair);
                MatView bl = view_of(lb + (long long)first * kWY * ldn, kWY, n, ldn, ps, npair);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = kWY; s.N = kWY; s.K = n; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                EpiStore e = epi_store_plain(w.Gab + (long long)b * npair * kWY * kWY, kWY, (long long)kWY * kWY,
                                             kWY, kWY);
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ah, &al, &bh, &bl, s, npair, e, st));
            }
            PSVD_TRY(cudaFuncSetAttribute(s_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrSmem));
        }
        for (int q = npair - 1; q >= 0; --q) {
            const int blk_b = first + 2 * q;
            const int k0 = blk_b * kWY;
            const int nb_a = std::min(kWY, n - 2 - (k0 + kWY));
            const int W = kWY + nb_a;
            const int r0 = ((k0 + 1) / 32) * 32;
            const int Lr = n - r0;
            int ks = 1;
            // S = V^T[:, r0:] [Y_b Y_a][r0:, :]   (n x W), as ks partial sums over K
            {
                MatView ahi = view_of(w.VThi + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView alo = view_of(w.VTlo + r0, n, Lr, ldn, (long long)n * ldn, B);
                MatView bhi = view_of(w.Vhi + (long long)k0 * ldn + r0, W, Lr, ldn, (long long)w.nrp * ldn, B);
                MatView blo = view_of(w.Vlo + (long long)k0 * ldn + r0, W, Lr, ldn, (long long)w.nrp * ldn, B);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = n; s.N = W; s.K = Lr; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                const int tiles = ((n + kBM - 1) / kBM) * B;
                s.ksplit = std::max(1, std::min(std::min(kBtSplit, (num_sms() + tiles - 1) / tiles), Lr / 128));
                ks = s.ksplit;
                EpiStore e = epi_store_plain(w.S, 2 * kWY, (long long)n * 2 * kWY, n, W);
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st));
            }
            s_pair_kernel<<<dim3((n + kPrRows - 1) / kPrRows, B), 2 * kWY, kPrSmem, st>>>(
                w.S, ks, B, w.Tm, w.Gab, n, w.nblk, npair, blk_b, q, nb_a, w.S2hi, w.S2lo);
            PSVD_TRY(cudaGetLastError());
            count_launch(1);
            // V^T[:, r0:] -= S2 [Y_b Y_a][r0:, :]^T
            {
                MatView ahi = view_of(w.S2hi, n, W, 2 * kWY, (long long)n * 2 * kWY, B);
                MatView alo = view_of(w.S2lo, n, W, 2 * kWY, (long long)n * 2 * kWY, B);
                MatView bhi = view_of(w.Yhi + (long long)r0 * ldn + k0, Lr, W, ldn, (long long)n * ldn, B);
                MatView blo = view_of(w.Ylo + (long long)r0 * ldn + k0, Lr, W, ldn, (long long)n * ldn, B);
                GemmShape s;
                memset(&s, 0, sizeof(s));
                s.M = n; s.N = Lr; s.K = W; s.prec_uniform = PREC_TF32X3; s.err = w.err;
                EpiSubSplit e;
                e.rows = n; e.cols = Lr; e.hi = w.VThi + r0; e.lo = w.VTlo + r0; e.ld = ldn;
                e.bs = (long long)n * ldn;
                PSVD_TRY(launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st));
            }
        }
        if (first) PSVD_TRY_RC(single(0));
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
