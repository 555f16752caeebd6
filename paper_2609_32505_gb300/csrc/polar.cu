// Polar factor W of M (Definition 2.1) by the matmul-only polynomial iteration of
// Algorithm 1 (steps 1-4):
//   X0 = M / sqrt(||M||_1 ||M||_inf)                          (Algorithm 2)
//   step k:  G_k = X_k^T X_k,  r_k = ||G_k - I||_F / sqrt(n)   (stop if r_k <= tol)
//            P_k = c1_k I + c3_k G_k,  X_{k+1} = X_k P_k         (degree-3 CANS / NS step)
//   H = (W^T M)_sym with W = X_final                           (FP64 averaging)
// Each step is three launches: the Gram product (upper-triangle tiles, with the
// polynomial and the residual fused in its epilogue), a per-matrix decision
// kernel (stop / precision of the next step), and the apply product X_k P_k
// whose epilogue writes X_{k+1} both row-major and transposed in the precision
// the next step uses.  Matrices that finished are skipped by every later CTA.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "polar.cuh"
#include "qr.cuh"
#include "schedule.h"

namespace psvd {

// ------------------------------------------------------------ Algorithm 2
// Row and column l1 norms in a fixed summation order (no atomics), so that the scale
// and every result downstream of it are reproducible run to run.
// rows: one warp per row; columns: one thread per column, rows in order.
__global__ void row_l1_kernel(const float *__restrict__ A, int m, int n, float *rowsum, int *nonfinite) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.y;
    if (warp >= m) return;
    const float *a = A + (long long)b * m * n + (long long)warp * n;
    float s = 0.f;
    bool bad = false;
    for (int j = lane; j < n; j += 32) {
        const float x = a[j];
        bad |= !isfinite(x);
        s += fabsf(x);
    }
    s = warp_sum(s);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        rowsum[(long long)b * m + warp] = s;
        if (bad) nonfinite[b] = 1;
    }
}

// Column sums of |A| in row slabs of kL1Rows rows: colpart[b][s][c] = sum over the rows of
// slab s of |A[i][c]|.  A block of 32 lanes x 8 row lanes; each lane covers 4 columns (one
// float4 with kVec: n % 4 == 0 and A 16-byte aligned) and sums every 8th row of the slab with
// 8 loads in flight, then the 8 row lanes are added in a fixed order, so the result does not
// depend on scheduling.
template <bool kVec>
__global__ void __launch_bounds__(256) col_l1_kernel(const float *__restrict__ A, int m, int n, float *colpart) {
    __shared__ float4 part[8][32];
    const int lane = threadIdx.x & 31, rl = threadIdx.x >> 5;
    const int c0 = blockIdx.x * 128 + 4 * lane;
    const int b = blockIdx.z, S = l1_slabs(m);
    const float *a = A + (long long)b * m * n;
    for (int sl = blockIdx.y; sl < S; sl += gridDim.y) {
        const long long r0 = (long long)sl * kL1Rows;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 < n) {
            for (int t0 = 0; t0 < kL1Rows / 8; t0 += 8) {
                float4 x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const long long i = r0 + rl + 8 * (t0 + t);
                    x[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (i < m) {
                        const float *q = a + i * n + c0;
                        if (kVec) x[t] = *reinterpret_cast<const float4 *>(q);
                        else {
                            x[t].x = q[0];
                            if (c0 + 1 < n) x[t].y = q[1];
                            if (c0 + 2 < n) x[t].z = q[2];
                            if (c0 + 3 < n) x[t].w = q[3];
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    acc.x += fabsf(x[t].x); acc.y += fabsf(x[t].y); acc.z += fabsf(x[t].z); acc.w += fabsf(x[t].w);
                }
            }
        }
        __syncthreads();                      // the previous slab's sums have been read
        part[rl][lane] = acc;
        __syncthreads();
        if (rl == 0 && c0 < n) {
            float4 s4 = part[0][lane];
#pragma unroll
            for (int r = 1; r < 8; ++r) {
                const float4 q = part[r][lane];
                s4.x += q.x; s4.y += q.y; s4.z += q.z; s4.w += q.w;
            }
            float *o = colpart + ((long long)b * S + sl) * n + c0;
            o[0] = s4.x;
            if (c0 + 1 < n) o[1] = s4.y;
            if (c0 + 2 < n) o[2] = s4.z;
            if (c0 + 3 < n) o[3] = s4.w;
        }
    }
}

// Launches both passes on `st`; colpart holds B x l1_slabs(m) x n floats.
cudaError_t l1_norms(const float *A, int B, int m, int n, float *rowsum, float *colpart, int *nonfinite,
                     cudaStream_t st) {
    row_l1_kernel<<<dim3((unsigned)(((long long)m * 32 + 255) / 256), B), 256, 0, st>>>(A, m, n, rowsum, nonfinite);
    const dim3 gc((n + 127) / 128, std::min(l1_slabs(m), 65535), B);
    if (((uintptr_t)A & 15) == 0 && (n & 3) == 0) col_l1_kernel<true><<<gc, 256, 0, st>>>(A, m, n, colpart);
    else col_l1_kernel<false><<<gc, 256, 0, st>>>(A, m, n, colpart);
    count_launch(2);
    return cudaGetLastError();
}

// One block per matrix: s = sqrt(max col l1 * max row l1); special cases set the
// matrix done (zero matrix: W = 0 and the QR step supplies U; non-finite input).
// (launched with kNormThreads threads; the slab sums of a column are loaded eight at a time)
__global__ void __launch_bounds__(kNormThreads) norm_finalize_kernel(const float *rowsum, const float *colsum,
                                                                      const int *nonfinite, int m, int n,
                                                                      float *scale, int *done, int *status,
                                                                      int *fin) {
    __shared__ float sm[2][32];
    const int b = blockIdx.x;
    float r = 0.f, c = 0.f;
    for (int i = threadIdx.x; i < m; i += blockDim.x) r = fmaxf(r, rowsum[(long long)b * m + i]);
    const int S = l1_slabs(m);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float cs = 0.f;                              // slab partial sums, added in slab order
        for (int q0 = 0; q0 < S; q0 += 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = q0 + u < S ? colsum[((long long)b * S + q0 + u) * n + j] : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) cs += x[u];
        }
        c = fmaxf(c, cs);
    }
    r = warp_max(r);
    c = warp_max(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) { sm[0][w] = r; sm[1][w] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) { r = fmaxf(r, sm[0][i]); c = fmaxf(c, sm[1][i]); }
        r = fmaxf(r, sm[0][0]);
        c = fmaxf(c, sm[1][0]);
        const double s = sqrt((double)r * (double)c);
        scale[b] = (float)s;
        if (nonfinite[b]) { done[b] = 1; status[b] = PSVD_ERR_NONFINITE; fin[b] = 0; }
        else if (s == 0.0) { done[b] = 1; status[b] = PSVD_OK; fin[b] = 0; }
    }
}

__global__ void polar_init_kernel(int B, int prec0, int *done, int *fin, int *status, int *prec, int *steps,
                                  int *fallback) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    done[b] = 0; fin[b] = 0; status[b] = PSVD_OK; fallback[b] = 0;
    prec[b] = prec0;
    steps[b] = steps[B + b] = steps[2 * B + b] = 0;
}

// ------------------------------------------------------------ schedules
struct CoefTable {
    int len;
    float c1[72], c3[72];
};

// coef[(k * B + b) * 2 + {0,1}] for k < K.  Learned: greedy optimal cubics from [l_b, 1] per
// matrix (FP64), each applied to x / kPeDamp while the tracked interval is wider than
// kPeWidth (undamped greedy cubics from a small bound lose accuracy: relative
// reconstruction ~2e-4 at kappa = 1e6 in FP32 against ~3e-6 damped, for the same number of
// steps), and the step budget before the conservative rerun; with gate_x3, a matrix whose
// bound is below PSVD_MIXED_LB_MIN starts on the split-TF32 rung.
// Damped (schedule PSVD_SCHED_PE, the Polar-Express-style comparison): the same damped cubics
// from [l_b, 1] until a damped step stops shrinking the interval (width below 0.1 and less
// than 10% gained: the damped fixed point near 1 - 1.5e-4, the plateau the ablation
// describes), then undamped from there; no budget and no rerun.
constexpr double kPeDamp = 1.01, kPeWidth = 1e-2;
__global__ void schedule_fill_kernel(int B, int K, CoefTable tab, const float *lower, int learned, double tol,
                                     int budget_opt, const int *active, float *coef, int *budget, int gate_x3,
                                     int *prec, int pe = 0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (active && !active[b]) return;
    if (learned || pe) {
        double l = (double)lower[b];
        if (learned && gate_x3 && !(l >= PSVD_MIXED_LB_MIN)) prec[b] = PREC_TF32X3;
        if (!(l > 1e-12)) l = 1e-12;
        if (l > 0.999) l = 0.999;
        double lo = l, hi = 1.0;
        bool damping = true;
        for (int k = 0; k < K; ++k) {
            const double width = fmax(1.0 - lo, hi - 1.0);
            double nlo, nhi;
            Cubic c;
            if (damping) {
                c = damped_cubic(lo, hi, kPeDamp, &nlo, &nhi);
                const double nw = fmax(1.0 - nlo, nhi - 1.0);
                if (learned ? width <= kPeWidth : (width < 0.1 && nw > 0.9 * width)) damping = false;
            }
            if (!damping) { c = cans_cubic(lo, hi); nlo = 1.0 - c.e; nhi = 1.0 + c.e; }
            coef[((long long)k * B + b) * 2 + 0] = (float)c.c1;
            coef[((long long)k * B + b) * 2 + 1] = (float)c.c3;
            lo = nlo;
            hi = nhi;
            if (!damping && hi - 1.0 < 1e-9 && 1.0 - lo < 1e-9) {
                // converged interval: c1 = 3/2 + O(e^2), c3 = -1/2 + O(e^2) round to the same
                // floats for every later half-width e < 1e-9, so the rest of the table is
                // the next cubic repeated (the FP64 pipe is narrow: this saves ~40 steps)
                const Cubic f = cans_cubic(lo, hi);
                for (int r = k + 1; r < K; ++r) {
                    coef[((long long)r * B + b) * 2 + 0] = (float)f.c1;
                    coef[((long long)r * B + b) * 2 + 1] = (float)f.c3;
                }
                break;
            }
        }
        budget[b] = learned ? (budget_opt > 0 ? budget_opt : greedy_steps_to(l, 0.5 * tol, K) + 5) : K;
        return;
    }
    if (!learned) {
        for (int k = 0; k < K; ++k) {
            const int i = k < tab.len ? k : tab.len - 1;
            coef[((long long)k * B + b) * 2 + 0] = tab.c1[i];
            coef[((long long)k * B + b) * 2 + 1] = tab.c3[i];
        }
        budget[b] = K;
        return;
    }
}

// ------------------------------------------------------------ step epilogues
PSVD_DEV void store_prec(int p, long long o, float x, __nv_bfloat16 *p16, float *phi, float *plo) {
    if (p == PREC_BF16) p16[o] = __float2bfloat16_rn(x);
    else if (p == PREC_TF32) phi[o] = tf32_round(x);
    else { float h, l; split_tf32(x, h, l); phi[o] = h; plo[o] = l; }
}

// Per-matrix decision after the Gram of step k.
// mixed: 0 every step split-TF32; 1 TF32 until the residual drops below kTauTF32; 2 BF16
// above kTauBF16 first.  The precision never decreases from one step to the next.
struct DecideArgs {
    int k, B, n, mixed, learned, kcap;
    double tol;
    int *done, *fin, *status, *prec, *steps, *fallback, *notdone;
    const double *res;
    const int *budget;
    float *fres;
};

PSVD_DEV void decide_matrix(const DecideArgs &d, int b) {
    if (d.done[b]) return;
    const int k = d.k, B = d.B;
    const double r = sqrt(d.res[(long long)k * B + b] / (double)d.n);
    const int pk = d.prec[(long long)k * B + b];
    if (!(r <= 1e30)) {                              // NaN / overflow in the iteration
        d.done[b] = 1; d.fin[b] = k; d.status[b] = PSVD_NOT_CONVERGED; d.fres[b] = (float)r;
        return;
    }
    if (r <= d.tol) { d.done[b] = 1; d.fin[b] = k; d.status[b] = PSVD_OK; d.fres[b] = (float)r; return; }
    if (k >= d.kcap) { d.done[b] = 1; d.fin[b] = k; d.status[b] = PSVD_NOT_CONVERGED; d.fres[b] = (float)r; return; }
    if (d.learned && k >= d.budget[b]) {
        d.done[b] = 1; d.fin[b] = k; d.status[b] = PSVD_NOT_CONVERGED; d.fres[b] = (float)r; d.fallback[b] = 1;
        return;
    }
    int pn = PREC_TF32X3;
    if (d.mixed) {
        const int want = (d.mixed == 2 && r > kTauBF16) ? PREC_BF16 : (r > kTauTF32 ? PREC_TF32 : PREC_TF32X3);
        pn = want > pk ? want : pk;
    }
    d.prec[(long long)(k + 1) * B + b] = pn;
    d.steps[pk * B + b] += 1;
    atomicAdd(&d.notdone[k], 1);
}

// Gram tile G = X^T X (tiles reaching the upper triangle): every entry with col >= row
// adds to ||G - I||_F^2 (off-diagonal entries twice) and stores P = c1 I + c3 G and its
// mirror in the precision of this step's apply; entries below the diagonal are left to
// the tile that holds their mirror.  The row-major entries go through the staged
// (coalesced) element pass, the mirrors through trans() on the thread's own row.
struct EpiGram {
    int n, B;
    DecideArgs dec;      // this step's per-matrix decision, run by the launch's last CTA
    const float *coef;   // coef + k*B*2
    const int *prec;     // prec + k*B
    double *res;         // res + k*B
    __nv_bfloat16 *P16;
    float *Phi, *Plo;
    long long ldp;
    struct Acc { ff r; int p; float c1, c3; };     // ||G - I||^2 partial, float-float (FP32 pipe)
    static constexpr bool kElem = true, kTrans = true, kTail = true;
    PSVD_DEV bool staged() const { return true; }
    PSVD_DEV void tail() const {
        for (int b = threadIdx.x; b < dec.B; b += blockDim.x) decide_matrix(dec, b);
    }
    PSVD_DEV void begin(Acc &a) const { a.r = ff_zero(); a.p = -1; }
    PSVD_DEV void load(Acc &a, int b) const {
        if (a.p < 0) { a.p = prec[b]; a.c1 = coef[2 * b]; a.c3 = coef[2 * b + 1]; }
    }
    PSVD_DEV void elem(Acc &a, int b, int r, int c, float g) const {
        if (r >= n || c >= n || c < r) return;
        load(a, b);
        const float d = g - (r == c ? 1.f : 0.f);
        a.r = ff_fma(a.r, r == c ? d : 2.f * d, d);
        const float pv = a.c3 * g + (r == c ? a.c1 : 0.f);
        store_prec(a.p, (long long)b * n * ldp + (long long)r * ldp + c, pv, P16, Phi, Plo);
    }
    PSVD_DEV void trans(Acc &a, int b, int r, int c0, float (&v)[16]) const {
        if (r >= n) return;
        load(a, b);
        const long long base = (long long)b * n * ldp + r;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c >= n) break;
            if (c <= r) continue;
            store_prec(a.p, base + (long long)c * ldp, a.c3 * v[i], P16, Phi, Plo);
        }
    }
    PSVD_DEV void chunk(Acc &a, int b, int r, int c0, int, int, float (&v)[16]) const {
#pragma unroll
        for (int i = 0; i < 16; ++i) elem(a, b, r, c0 + i, v[i]);
        trans(a, b, r, c0, v);
    }
    PSVD_DEV void finish(Acc &a, int b, int, int) const {
        const double s = warp_sum((double)a.r.hi + (double)a.r.lo);
        if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&res[b], s);
    }
};

// X_{k+1} = X_k P_k: stored row-major (staged, coalesced) and transposed (trans(), lanes
// on consecutive rows) in the next step's precision.
struct EpiApply {
    int m, n, B;
    const int *prec_next;   // prec + (k+1)*B
    __nv_bfloat16 *X16, *XT16;
    float *Xhi, *Xlo, *XThi, *XTlo;
    long long ldn, ldm;
    struct Acc { int p; };
    static constexpr bool kElem = true, kTrans = true;
    PSVD_DEV bool staged() const { return true; }
    PSVD_DEV void begin(Acc &a) const { a.p = -1; }
    PSVD_DEV void elem(Acc &a, int b, int r, int c, float x) const {
        if (r >= m || c >= n) return;
        if (a.p < 0) a.p = prec_next[b];
        store_prec(a.p, (long long)b * m * ldn + (long long)r * ldn + c, x, X16, Xhi, Xlo);
    }
    PSVD_DEV void trans(Acc &a, int b, int r, int c0, float (&v)[16]) const {
        if (r >= m) return;
        if (a.p < 0) a.p = prec_next[b];
        const long long tb = (long long)b * n * ldm + r;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c >= n) break;
            store_prec(a.p, tb + (long long)c * ldm, v[i], XT16, XThi, XTlo);
        }
    }
    PSVD_DEV void chunk(Acc &a, int b, int r, int c0, int, int, float (&v)[16]) const {
#pragma unroll
        for (int i = 0; i < 16; ++i) elem(a, b, r, c0 + i, v[i]);
        trans(a, b, r, c0, v);
    }
    PSVD_DEV void finish(Acc &, int, int, int) const {}
};

// W (user layout) from X_fin; leaves W split row-major in Xhi[0]/Xlo[0] and
// transposed in XThi[0]/XTlo[0] for the products that follow (H, U).
__global__ void polar_finalize_kernel(int m, int n, int B, const int *fin, const int *prec, const int *status,
                                      PolarWS ws, float *W) {
    __shared__ float tile[32][33];
    const int b = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int f = fin[b];
    const int par = f & 1;
    const int p = prec[(long long)f * B + b];
    const bool nan_out = status[b] == PSVD_ERR_NONFINITE;
    const bool copy = par != 0 || p != PREC_TF32X3 || nan_out;
    const long long rbase = (long long)b * m * ws.ldn;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        float x = 0.f;
        if (r < m && c < n) {
            const long long o = rbase + (long long)r * ws.ldn + c;
            if (nan_out) x = __int_as_float(0x7fc00000);
            else if (p == PREC_BF16) x = __bfloat162float(ws.X16[par][o]);
            else if (p == PREC_TF32) x = ws.Xhi[par][o];
            else x = ws.Xhi[par][o] + ws.Xlo[par][o];
            if (W) W[(long long)b * m * n + (long long)r * n + c] = x;
            if (copy) { float h, l; split_tf32(x, h, l); ws.Xhi[0][o] = h; ws.Xlo[0][o] = l; }
        }
        tile[i][threadIdx.x] = x;
    }
    if (!copy) return;                     // uniform per block
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < n && r < m) {
            float h, l;
            split_tf32(tile[threadIdx.x][i], h, l);
            const long long o = (long long)b * n * ws.ldm + (long long)c * ws.ldm + r;
            ws.XThi[0][o] = h;
            ws.XTlo[0][o] = l;
        }
    }
}

// H = (Hraw + Hraw^T) / 2, stored FP32 (Hsym, and H_out when given).
__global__ void __launch_bounds__(256) symmetrize_kernel(const float *Hraw, int n, float *Hsym, float *Hout) {
    // One 32 x 32 tile per block (32 x 8 threads), its mirror tile staged in shared memory so
    // that both reads are coalesced.  (h_ij + h_ji) / 2 is formed as the FP32 sum scaled by
    // 1/2: the scaling is exact, so the result equals the FP64 average rounded to FP32 (the
    // FP64 symmetrization) except where the average is subnormal.
    __shared__ float tm[32][33];
    const int b = blockIdx.z, i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float *h = Hraw + (long long)b * n * n;
#pragma unroll
    for (int r = ty; r < 32; r += 8)
        tm[r][tx] = (j0 + r < n && i0 + tx < n) ? h[(long long)(j0 + r) * n + i0 + tx] : 0.f;
    __syncthreads();
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + tx;
        if (i < n && j < n) {
            const long long o = (long long)b * n * n + (long long)i * n + j;
            const float v = __fmul_rn(__fadd_rn(h[(long long)i * n + j], tm[tx][r]), 0.5f);
            Hsym[o] = v;
            if (Hout) Hout[o] = v;
        }
    }
}

// hist[k * B + b] = ||G_k - I||_F / sqrt(n) at the Gram of step k (0 where the matrix had
// already finished, or the step was never reached), for the matrices with only[b] != 0
// (all when only is null).
__global__ void res_history_kernel(const double *res, int K, int B, int n, const int *only, double *hist) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= K * B) return;
    if (only && !only[t % B]) return;
    hist[t] = sqrt(res[t] / (double)n);
}

__global__ void polar_info_kernel(int B, const int *status, const int *fin, const int *steps, const int *fallback,
                                  const float *fres, const float *scale, psvd_info *info) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    psvd_info r;
    r.status = status[b];
    r.iters = steps[b] + steps[B + b] + steps[2 * B + b];
    r.qr_fallback = 0;
    r.sched_fallback = fallback[b];
    r.prec_fallback = 0;
    r.corr_max = 0.f;
    r.recon_est = 0.f;
    r.steps_bf16 = steps[b];
    r.steps_tf32 = steps[B + b];
    r.steps_3xtf32 = steps[2 * B + b];
    r.ortho_resid = fres[b];
    r.scale = scale[b];
    info[b] = r;
}

// ------------------------------------------------------------ host driver
// Step k: Gram (with the polynomial and residual epilogue, and the per-matrix decision run
// by its last CTA), then apply.  The Gram launch is gated on `gram_gate` (the count of
// matrices still iterating; nullptr = always run) and the apply launch on this step's own
// count, so once every matrix has finished the remaining launches of the budget return at
// once.
static int launch_step(PolarWS &w, int k, bool apply, double tol, bool learned, float *fres, const int *gram_gate,
                       cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n;
    const int par = k & 1, npar = (k + 1) & 1;
    // Gram: A = B = X^T (n x m, K = m), upper-triangle tiles
    {
        MatView v16 = w.bf16 ? view_of16(w.XT16[par], n, m, w.ldm, (long long)n * w.ldm, B) : MatView();
        MatView vhi = view_of(w.XThi[par], n, m, w.ldm, (long long)n * w.ldm, B);
        MatView vlo = view_of(w.XTlo[par], n, m, w.ldm, (long long)n * w.ldm, B);
        GemmShape s;
        memset(&s, 0, sizeof(s));
        s.M = n; s.N = n; s.K = m; s.sym = 1;
        s.prec = w.prec + (long long)k * B;
        s.skip = w.done;
        s.gate = gram_gate;
        s.ticket = w.ticket + k;
        s.err = w.err;
        EpiGram e;
        e.n = n; e.B = B;
        e.dec = DecideArgs{k, B, n, w.bf16 ? 2 : (w.mixed ? 1 : 0), learned ? 1 : 0, w.kcap, tol, w.done, w.fin,
                           w.status, w.prec, w.steps, w.fallback, w.notdone, w.res, w.budget, fres};
        e.coef = w.coef + (long long)k * B * 2;
        e.prec = w.prec + (long long)k * B;
        e.res = w.res + (long long)k * B;
        e.P16 = w.P16; e.Phi = w.Phi; e.Plo = w.Plo; e.ldp = w.ldn;
        cudaError_t er = launch_gemm(w.bf16 ? &v16 : nullptr, w.bf16 ? &v16 : nullptr, &vhi, &vlo, &vhi, &vlo, s,
                                     B, e, st);
        if (er != cudaSuccess) return PSVD_ERR_CUDA;
    }
    if (!apply) return PSVD_OK;
    // Apply: A = X (m x n, K = n), B = P (n x n, symmetric)
    {
        MatView a16 = w.bf16 ? view_of16(w.X16[par], m, n, w.ldn, (long long)m * w.ldn, B) : MatView();
        MatView ahi = view_of(w.Xhi[par], m, n, w.ldn, (long long)m * w.ldn, B);
        MatView alo = view_of(w.Xlo[par], m, n, w.ldn, (long long)m * w.ldn, B);
        MatView b16 = w.bf16 ? view_of16(w.P16, n, n, w.ldn, (long long)n * w.ldn, B) : MatView();
        MatView bhi = view_of(w.Phi, n, n, w.ldn, (long long)n * w.ldn, B);
        MatView blo = view_of(w.Plo, n, n, w.ldn, (long long)n * w.ldn, B);
        GemmShape s;
        memset(&s, 0, sizeof(s));
        s.M = m; s.N = n; s.K = n;
        s.prec = w.prec + (long long)k * B;
        s.skip = w.done;
        s.gate = w.notdone + k;          // matrices still iterating after this step's decision
        s.err = w.err;
        EpiApply e;
        e.m = m; e.n = n; e.B = B;
        e.prec_next = w.prec + (long long)(k + 1) * B;
        e.X16 = w.X16[npar]; e.XT16 = w.XT16[npar];
        e.Xhi = w.Xhi[npar]; e.Xlo = w.Xlo[npar]; e.XThi = w.XThi[npar]; e.XTlo = w.XTlo[npar];
        e.ldn = w.ldn; e.ldm = w.ldm;
        cudaError_t er = launch_gemm(w.bf16 ? &a16 : nullptr, w.bf16 ? &b16 : nullptr, &ahi, &alo, &bhi, &blo, s,
                                     B, e, st);
        if (er != cudaSuccess) return PSVD_ERR_CUDA;
    }
    return PSVD_OK;
}

// Launches steps 0..kmax (kmax <= kcap) with no host synchronization: the decision kernel
// of step k counts the matrices still iterating in notdone[k], and the launches after the
// last matrix has finished find their gate at 0 and return at once.  `first_gate` gates
// the Gram launch of step 0 (nullptr: always run).
static int run_iteration(PolarWS &w, int kmax, double tol, bool learned, float *fres, const int *first_gate,
                         cudaStream_t st) {
    for (int k = 0; k <= kmax; ++k) {
        const int *gate = k == 0 ? first_gate : w.notdone + (k - 1);
        if (int rc = launch_step(w, k, k < w.kcap, tol, learned, fres, gate, st)) return rc;
    }
    return PSVD_OK;
}

__global__ void fallback_reset_kernel(int B, int prec0, const int *fallback, int *done, int *prec, int *count) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (fallback[b]) { done[b] = 0; prec[b] = prec0; atomicAdd(count, 1); }
    else done[b] = 1;
}

// restores done[] = 1 for every matrix after a rerun pass (all are final now)
__global__ void set_all_done_kernel(int B, int *done) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) done[b] = 1;
}

static int prepare_x0(const float *A, PolarWS &w, cudaStream_t st, const int *skip) {
    const int B = w.B, m = w.m, n = w.n;
    SplitOut r, t;
    r.ld = w.ldn; r.bstride = (long long)m * w.ldn;
    t.ld = w.ldm; t.bstride = (long long)n * w.ldm;
    if (w.bf16) { r.h16 = w.X16[0]; t.h16 = w.XT16[0]; }
    else { r.hi = w.Xhi[0]; r.lo = w.Xlo[0]; t.hi = w.XThi[0]; t.lo = w.XTlo[0]; }
    if (prepare_operand(A, n, (long long)m * n, B, m, n, false, 1.f, w.scale, r, st, skip) ||
        prepare_operand(A, n, (long long)m * n, B, m, n, true, 1.f, w.scale, t, st, skip))
        return PSVD_ERR_CUDA;
    return PSVD_OK;
}

int polar_forward(const float *A, float *W, float *H_out, bool want_h, PolarWS &w, const psvd_opts &o,
                  psvd_info *info, cudaStream_t st, bool rerun_learned) {
    const int B = w.B, m = w.m, n = w.n;
    const bool learned = o.schedule == PSVD_SCHED_LEARNED;
    if (cudaMemsetAsync(w.rowsum, 0, sizeof(float) * (size_t)B * m, st) ||
        cudaMemsetAsync(w.nonfinite, 0, sizeof(int) * (size_t)B, st) ||
        cudaMemsetAsync(w.res, 0, sizeof(double) * (size_t)(w.kcap + 2) * B, st) ||
        cudaMemsetAsync(w.notdone, 0, sizeof(int) * (size_t)(w.kcap + 2), st) ||
        cudaMemsetAsync(w.ticket, 0, sizeof(unsigned) * (size_t)(w.kcap + 2), st) ||
        cudaMemsetAsync(w.fres, 0, sizeof(float) * (size_t)B, st) ||
        cudaMemsetAsync(w.misc, 0, sizeof(int) * 8, st) ||
        cudaMemsetAsync(w.err, 0, sizeof(unsigned) * 4, st))
        return PSVD_ERR_CUDA;
    const int prec0 = w.bf16 ? PREC_BF16 : (w.mixed ? PREC_TF32 : PREC_TF32X3);
    polar_init_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, prec0, w.done, w.fin, w.status, w.prec, w.steps,
                                                        w.fallback);
    if (l1_norms(A, B, m, n, w.rowsum, w.colsum, w.nonfinite, st) != cudaSuccess) return PSVD_ERR_CUDA;
    norm_finalize_kernel<<<B, kNormThreads, 0, st>>>(w.rowsum, w.colsum, w.nonfinite, m, n, w.scale, w.done, w.status,
                                            w.fin);
    count_launch(2);
    // coefficient tables: conservative CANS (Appendix B.8), classical NS, or learned bounds
    CoefTable tab;
    memset(&tab, 0, sizeof(tab));
    std::vector<Cubic> cons = cans_schedule(o.delta, o.pre_iters, std::min(w.kcap + 1, 72));
    std::vector<Cubic> sched = o.schedule == PSVD_SCHED_NS ? std::vector<Cubic>(1, Cubic{1.5, -0.5, 0.0}) : cons;
    tab.len = (int)sched.size();
    for (int i = 0; i < tab.len; ++i) { tab.c1[i] = (float)sched[i].c1; tab.c3[i] = (float)sched[i].c3; }
    const int gate_x3 = learned && w.mixed && !w.bf16 ? 1 : 0;
    schedule_fill_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, w.kcap + 1, tab, o.lower_bound, learned ? 1 : 0,
                                                          o.tol, o.budget, nullptr, w.coef, w.budget, gate_x3,
                                                          w.prec, o.schedule == PSVD_SCHED_PE ? 1 : 0);
    count_launch(1);
    if (int rc = prepare_x0(A, w, st, nullptr)) return rc;   // zero matrices get X0 = 0
    if (want_h) {
        SplitOut at;
        at.hi = w.AThi; at.lo = w.ATlo; at.ld = w.ldm; at.bstride = (long long)n * w.ldm;
        if (prepare_operand(A, n, (long long)m * n, B, m, n, true, 1.f, nullptr, at, st)) return PSVD_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return PSVD_ERR_CUDA;
    // Host-side bound on the steps any matrix can take: the cap for the conservative and
    // Newton-Schulz schedules; for the learned one, the largest budget a lower bound can
    // produce (the bound is clamped to >= 1e-12 on the device) or the caller's budget.
    int kmax = w.kcap;
    if (learned) kmax = std::min(w.kcap, o.budget > 0 ? o.budget : greedy_steps_to(1e-12, 0.5 * o.tol, w.kcap + 1) + 5);
    if (int rc = run_iteration(w, kmax, o.tol, learned, w.fres, nullptr, st)) return rc;
    if (learned && rerun_learned) {
        if (o.res_history) {        // the learned pass's history; the rerun overwrites its own matrices'
            const int K = w.kcap + 1;
            res_history_kernel<<<(K * B + 127) / 128, 128, 0, st>>>(w.res, K, B, n, nullptr, o.res_history);
            count_launch(1);
        }
        // Matrices whose learned schedule missed tol within budget are rerun from X0 with the
        // conservative schedule.  Nothing is read back: the rerun's steps are launched for the
        // whole budget, gated on the number of rerun matrices (misc[0]) and then on the
        // per-step counts, so without a fallback every one of them returns at once.
        fallback_reset_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, prec0, w.fallback, w.done, w.prec, w.misc);
        count_launch(1);
        CoefTable ct;
        memset(&ct, 0, sizeof(ct));
        ct.len = (int)cons.size();
        for (int i = 0; i < ct.len; ++i) { ct.c1[i] = (float)cons[i].c1; ct.c3[i] = (float)cons[i].c3; }
        schedule_fill_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, w.kcap + 1, ct, nullptr, 0, o.tol, 0,
                                                              w.fallback, w.coef, w.budget, 0, w.prec);
        count_launch(1);
        if (cudaMemsetAsync(w.res, 0, sizeof(double) * (size_t)(w.kcap + 2) * B, st) ||
            cudaMemsetAsync(w.notdone, 0, sizeof(int) * (size_t)(w.kcap + 2), st) ||
            cudaMemsetAsync(w.ticket, 0, sizeof(unsigned) * (size_t)(w.kcap + 2), st))
            return PSVD_ERR_CUDA;
        if (int rc = prepare_x0(A, w, st, w.done)) return rc;
        if (int rc = run_iteration(w, w.kcap, o.tol, false, w.fres, w.misc, st)) return rc;
        if (o.res_history) {
            const int K = w.kcap + 1;
            res_history_kernel<<<(K * B + 127) / 128, 128, 0, st>>>(w.res, K, B, n, w.fallback, o.res_history);
            count_launch(1);
        }
        set_all_done_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, w.done);
        count_launch(1);
    }
    // W out + final split layouts
    {
        dim3 g((n + 31) / 32, (m + 31) / 32, B), blk(32, 8);
        polar_finalize_kernel<<<g, blk, 0, st>>>(m, n, B, w.fin, w.prec, w.status, w, W);
        count_launch(1);
    }
    if (want_h) {
        MatView ahi = view_of(w.XThi[0], n, m, w.ldm, (long long)n * w.ldm, B);
        MatView alo = view_of(w.XTlo[0], n, m, w.ldm, (long long)n * w.ldm, B);
        MatView bhi = view_of(w.AThi, n, m, w.ldm, (long long)n * w.ldm, B);
        MatView blo = view_of(w.ATlo, n, m, w.ldm, (long long)n * w.ldm, B);
        GemmShape s;
        memset(&s, 0, sizeof(s));
        s.M = n; s.N = n; s.K = m; s.prec_uniform = PREC_TF32X3; s.err = w.err;
        EpiStore e = epi_store_plain(w.Hraw, n, (long long)n * n, n, n);
        if (launch_gemm(nullptr, nullptr, &ahi, &alo, &bhi, &blo, s, B, e, st) != cudaSuccess) return PSVD_ERR_CUDA;
        symmetrize_kernel<<<dim3((n + 31) / 32, (n + 31) / 32, B), dim3(32, 8), 0, st>>>(w.Hraw, n, w.Hsym, H_out);
        count_launch(1);
    }
    if (info) {
        polar_info_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, w.status, w.fin, w.steps, w.fallback, w.fres, w.scale,
                                                           info);
        count_launch(1);
    }
    if (o.res_history && !(learned && rerun_learned)) {
        const int K = w.kcap + 1;
        res_history_kernel<<<(K * B + 127) / 128, 128, 0, st>>>(w.res, K, B, n, nullptr, o.res_history);
        count_launch(1);
    }
    return cudaGetLastError() == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA;
}

}  // namespace psvd

// ------------------------------------------------------------ C ABI
using namespace psvd;

static bool opts_ok(const psvd_opts &o) {
    return (o.precision == PSVD_PREC_FP32 || o.precision == PSVD_PREC_MIXED || o.precision == PSVD_PREC_MIXED_BF16) &&
           (o.schedule >= PSVD_SCHED_CANS && o.schedule <= PSVD_SCHED_PE) && o.delta > 0 && o.delta < 1 &&
           o.pre_iters >= 0 && o.pre_iters <= 8 && o.max_iter >= 1 && o.max_iter <= 64 && o.tol > 0 &&
           o.eps_qr > 0 && (o.preqr == 0 || o.preqr == 1) &&
           ((o.schedule != PSVD_SCHED_LEARNED && o.schedule != PSVD_SCHED_PE) || o.lower_bound != nullptr);
}

static psvd_opts resolve_opts(const psvd_opts *p) {
    psvd_opts o;
    psvd_default_opts(&o);
    if (p) o = *p;
    return o;
}

static size_t polar_direct_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts &o) {
    Sizer s;
    PolarWS w;
    w.carve(s, (int)batch, (int)m, (int)n, polar_kcap(o), o.precision);
    return s.used + 256;
}

// QR preprocessing (Section 4.1, rectangular matrices): M = Q R, polar decomposition of R,
// W = Q W_R, H = H_R.  Layout: Q, R, W_R, then one region shared in turn by the QR, the
// iteration on R and the operands of the final product.
struct PolarPreqr {
    float *Q = nullptr, *R = nullptr, *WR = nullptr;
    char *rest = nullptr;
    size_t rest_bytes = 0, need = 0;
    void plan(void *ws, size_t ws_bytes, int64_t B, int64_t m, int64_t n, const psvd_opts &o) {
        Carver cv(ws, ws_bytes);
        Q = cv.take<float>(B * m * n);
        R = cv.take<float>(B * n * n);
        WR = cv.take<float>(B * n * n);
        const size_t head = (size_t)round_up((long long)cv.used, 256);
        Sizer q;
        QrWS qw;
        qw.carve(q, (int)B, (int)m, (int)n);
        const long long ld = pad_ld(n);
        const size_t ops = (size_t)(2 * B * m * ld + 2 * B * n * ld) * sizeof(float) + 1024;
        need = head + std::max(std::max(q.used + 256, polar_direct_bytes(B, n, n, o)), ops);
        rest = ws ? static_cast<char *>(ws) + head : nullptr;
        rest_bytes = ws_bytes > head ? ws_bytes - head : 0;
    }
};

static bool polar_use_preqr(const psvd_opts &o, int64_t m, int64_t n) {
    int nb = 0, cl = 0;
    return o.preqr == 1 && m > n && qr_shape((int)m, &nb, &cl);
}

extern "C" size_t psvd_polar_workspace_bytes(int64_t batch, int64_t m, int64_t n, const psvd_opts *opts) {
    psvd_opts o = resolve_opts(opts);
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    if (polar_use_preqr(o, m, n)) {
        PolarPreqr l;
        l.plan(nullptr, 0, batch, m, n, o);
        return l.need + 256;
    }
    return polar_direct_bytes(batch, m, n, o);
}

extern "C" int psvd_polar_fwd(const float *A, float *W, float *H, int64_t batch, int64_t m, int64_t n,
                              const psvd_opts *opts, void *ws, size_t ws_bytes, psvd_info *info, void *stream) {
    psvd_opts o = resolve_opts(opts);
    if (!A || !W || batch <= 0 || n <= 0 || m < n || batch > 65535 || m > (1 << 28) / 1 || !opts_ok(o))
        return PSVD_ERR_ARG;
    if ((long long)m * n > (1LL << 31)) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_polar_workspace_bytes(batch, m, n, &o)) return PSVD_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = (int)batch, M = (int)m, N = (int)n;
    if (!polar_use_preqr(o, m, n)) {
        Carver cv(ws, ws_bytes);
        PolarWS w;
        w.carve(cv, B, M, N, polar_kcap(o), o.precision);
        if (cv.overflow) return PSVD_ERR_WORKSPACE;
        return polar_forward(A, W, H, H != nullptr, w, o, info, st);
    }
    PolarPreqr l;
    l.plan(ws, ws_bytes, batch, m, n, o);
    {
        Carver cv(l.rest, l.rest_bytes);
        QrWS qw;
        qw.carve(cv, B, M, N);
        if (cv.overflow) return PSVD_ERR_WORKSPACE;
        PSVD_TRY_RC(qr_factor(A, l.Q, l.R, nullptr, qw, st));
    }
    {
        Carver cv(l.rest, l.rest_bytes);
        PolarWS w;
        w.carve(cv, B, N, N, polar_kcap(o), o.precision);
        if (cv.overflow) return PSVD_ERR_WORKSPACE;
        PSVD_TRY_RC(polar_forward(l.R, l.WR, H, H != nullptr, w, o, info, st));
    }
    // W = Q W_R: B operand B[k][j] = W_R[j][k] (W_R transposed)
    Carver cv(l.rest, l.rest_bytes);
    const long long ld = pad_ld(N);
    float *qhi = cv.take<float>((size_t)B * M * ld), *qlo = cv.take<float>((size_t)B * M * ld);
    float *whi = cv.take<float>((size_t)B * N * ld), *wlo = cv.take<float>((size_t)B * N * ld);
    unsigned *err = cv.take<unsigned>(4);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    SplitOut a, bt;
    a.hi = qhi; a.lo = qlo; a.ld = ld; a.bstride = (long long)M * ld;
    bt.hi = whi; bt.lo = wlo; bt.ld = ld; bt.bstride = (long long)N * ld;
    PSVD_TRY(prepare_operand(l.Q, N, (long long)M * N, B, M, N, false, 1.f, nullptr, a, st));
    PSVD_TRY(prepare_operand(l.WR, N, (long long)N * N, B, N, N, true, 1.f, nullptr, bt, st));
    MatView ah = view_of(qhi, M, N, ld, (long long)M * ld, B), al = view_of(qlo, M, N, ld, (long long)M * ld, B);
    MatView bh = view_of(whi, N, N, ld, (long long)N * ld, B), bl = view_of(wlo, N, N, ld, (long long)N * ld, B);
    GemmShape s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = N; s.prec_uniform = PREC_TF32X3; s.err = err;
    EpiStore e = epi_store_plain(W, N, (long long)M * N, M, N);
    PSVD_TRY(launch_gemm(nullptr, nullptr, &ah, &al, &bh, &bl, s, B, e, st));
    return PSVD_OK;
}

// ------------------------------------------------------------ allocation-free variant
// Scratch for psvd_polar_fwd_noalloc: a fixed device array in this file, present on every
// GPU that loads the library until the process exits.  Host code must not pass the
// symbol itself to a kernel (on the host it names a stand-in object); its device address
// is looked up with cudaGetSymbolAddress once per device, with that device current, and
// again after the device's context has changed (cudaDeviceReset reloads the module).
static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

#include <mutex>

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};
}  // namespace

extern "C" size_t psvd_polar_noalloc_capacity(void) { return kNoAllocScratchBytes; }

extern "C" int psvd_polar_fwd_noalloc(const float *A, float *W, float *H, int64_t batch, int64_t m, int64_t n,
                                      const psvd_opts *opts, psvd_info *info, void *stream) {
    psvd_opts o = resolve_opts(opts);
    // the same argument checks as psvd_polar_fwd; the QR preprocessing needs a workspace
    if (!A || !W || batch <= 0 || n <= 0 || m < n || batch > 65535 || m > (1 << 28) / 1 || !opts_ok(o) ||
        o.preqr != 0)
        return PSVD_ERR_ARG;
    if ((long long)m * n > (1LL << 31)) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    const size_t need = psvd_polar_workspace_bytes(batch, m, n, &o);
    if (need > kNoAllocScratchBytes)
        return fail_msg(PSVD_ERR_WORKSPACE,
                        "psvd_polar_fwd_noalloc: a %lld x %lld x %lld problem needs %zu bytes of scratch, "
                        "the static array holds %zu", (long long)batch, (long long)m, (long long)n, need,
                        kNoAllocScratchBytes);
    int dev = 0;
    PSVD_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return PSVD_ERR_ARG;
    const unsigned long long ctx = current_context_id();
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
            void *p = nullptr;
            PSVD_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_noalloc_ptr[dev] = p;
            g_noalloc_ctx[dev] = ctx;
        }
        scratch = g_noalloc_ptr[dev];
    }
    Carver cv(scratch, kNoAllocScratchBytes);
    PolarWS w;
    w.carve(cv, (int)batch, (int)m, (int)n, polar_kcap(o), o.precision);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return polar_forward(A, W, H, H != nullptr, w, o, info, static_cast<cudaStream_t>(stream));
}
