// Blocked Householder QR (m >= n, diag(R) >= 0) for the QR fallback of Algorithm 1
// (Appendix A.2) and the QR preprocessing of rectangular inputs (Section 4.1).
//
// The matrix is kept transposed and split into TF32 hi/lo halves (UT: row j = column j).
// Panels of nb columns are factored by one thread-block cluster per matrix: each of the
// cl CTAs holds a slab of the panel's rows in shared memory, and the per-column dot
// products (the norm below the diagonal and the projections of the later panel columns)
// are summed across the cluster through distributed shared memory -- one cluster barrier
// per column, where the unblocked kernel needed three grid barriers.  The panel's
// reflectors H_j = I - tau_j v_j v_j^T then act on the trailing columns in compact-WY form
// H_j0 ... H_j0+nb-1 = I - Y T Y^T as two split-TF32 tcgen05 products:
//   W = Y^T X (K split over CTAs),  X -= Y (T^T W)
// and Q = H_0 ... H_{n-1} [I; 0] is accumulated backwards the same way with T in place of T^T.
// Finally Q and R get the signs that make diag(R) >= 0.
#include <cooperative_groups.h>

#include <cmath>
#include <cstring>

#include "qr.cuh"

namespace psvd {

namespace cg = cooperative_groups;

constexpr int kQrThreads = 512;
constexpr size_t kQrSlabMax = 180 * 1024;   // shared memory for one CTA's slab of the panel

// Slab column stride: odd, so that the lanes of a warp (consecutive columns, same row) fall
// in distinct shared-memory banks.
__host__ __device__ inline int qr_slab_stride(int S) { return (S & 1) ? S : S + 1; }

static size_t qr_panel_smem(int m, int nb, int cl) {
    const int S = qr_slab_stride((m + cl - 1) / cl);
    const size_t slab = std::max<size_t>((size_t)S * nb, (size_t)2 * nb * (nb + 1)) * sizeof(float);
    const size_t red = sizeof(float) * (size_t)kQrThreads;
    return sizeof(double) * ((size_t)2 * cl * 2 * nb + 5 * nb) + red + slab;
}

bool qr_shape(int m, int *nb, int *cl) {
    const int nbs[2] = {64, 32}, cls[2] = {8, 16};
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            const int S = qr_slab_stride((m + cls[c] - 1) / cls[c]);
            if ((size_t)S * nbs[a] * sizeof(float) <= kQrSlabMax) { *nb = nbs[a]; *cl = cls[c]; return true; }
        }
    return false;
}

struct PanelArgs {
    float *UThi, *UTlo, *YThi, *YTlo, *Yhi, *Ylo, *tau, *beta, *Tm, *Gpart;
    const int *skip;
    int m, n, j0, pw, panel, npan, nb, cl;
    long long ldm, ldn;
};

// One cluster per matrix factors columns j0 .. j0 + pw - 1 (rows j0 .. m - 1).  CTA q of the
// cluster owns rows [j0 + q S, j0 + (q + 1) S), S = ceil((m - j0) / cl), column-major in
// shared memory.  For column j every CTA contributes, over its rows r > j, the partial sums
// P_c' = sum x_r y_c',r (c' = j: the squared norm below the diagonal) and, from the owner of
// row j, the row-j values; each CTA writes its vector into a slot of every CTA of the cluster,
// and after the barrier every CTA adds the slots in rank order (so all get the same totals,
// bit for bit) and builds the reflector redundantly: beta = -sign(alpha) sqrt(alpha^2 + s2),
// tau = (beta - alpha) / beta, v = [1; x / (alpha - beta)].  Slots are double-buffered by
// column parity, which makes one barrier per column enough.  The slots and their sums are
// FP32, like the partial sums they hold (FP64 sums of the cluster's 8 or 16 partials took
// ~40% of a column's time on the narrow FP64 pipe, measured, and added no accuracy that
// the FP32 partial sums had).
__global__ void __launch_bounds__(kQrThreads, 1) qr_panel_kernel(PanelArgs P) {
    cg::cluster_group cluster = cg::this_cluster();
    const int CL = P.cl, rank = (int)cluster.block_rank();
    const int b = blockIdx.x / CL;
    if (P.skip[b]) return;                       // uniform across the cluster
    extern __shared__ __align__(16) double qsm[];
    const int nb = P.nb, pw = P.pw, j0 = P.j0, m = P.m, n = P.n;
    float *xch = reinterpret_cast<float *>(qsm); // [2][CL][2 nb] slots, double-buffered by column parity
    double *part = qsm + 2 * CL * 2 * nb;        // [2 nb] doubles of room
    float *vec = reinterpret_cast<float *>(part); // [2 nb] this CTA's vector of the column
    float *coef = reinterpret_cast<float *>(part + 4 * nb);   // [nb] f_c' of this column, then [2] scal, beta
    float *scal_s = coef + nb;
    float *red = reinterpret_cast<float *>(part + 5 * nb);    // [kQrThreads] row-block partial sums
    float *slab = red + kQrThreads;                           // [pw][Sp] column-major, Sp odd
    const int S = (m - j0 + CL - 1) / CL;
    const int Sp = qr_slab_stride(S);
    const int r0 = j0 + rank * S;
    const int nr = max(0, min(m, r0 + S) - r0);
    const int tid = threadIdx.x;
    const long long ubase = (long long)b * n * P.ldm;
    // thread -> (column cc, row block rb): the lanes of a warp share rb and hold consecutive columns
    const int nrb = kQrThreads / nb, cc = tid % nb, rb = tid / nb;
    const int rbs = (nr + nrb - 1) / nrb;
    const int rlo = rb * rbs, rhi = min(nr, rlo + rbs);

    for (int c = 0; c < pw; ++c) {
        const float *hi = P.UThi + ubase + (long long)(j0 + c) * P.ldm + r0;
        const float *lo = P.UTlo + ubase + (long long)(j0 + c) * P.ldm + r0;
        for (int rr = tid; rr < nr; rr += blockDim.x) slab[c * Sp + rr] = hi[rr] + lo[rr];
    }
    __syncthreads();

    for (int c = 0; c < pw; ++c) {
        const int j = j0 + c, par = c & 1;
        const int jl = j - r0;
        const bool own = jl >= 0 && jl < nr;
        const int start = max(0, jl + 1);
        const int live = pw - c;                 // entries c .. pw-1 of the vectors are needed
        const float *x = slab + c * Sp;
        // partial dot products of column c with columns cc >= c over rows r > j of this block
        if (cc >= c && cc < pw) {
            const float *y = slab + cc * Sp;
            float a0 = 0.f, a1 = 0.f;
            int rr = max(rlo, start);
            for (; rr + 1 < rhi; rr += 2) {
                a0 = fmaf(x[rr], y[rr], a0);
                a1 = fmaf(x[rr + 1], y[rr + 1], a1);
            }
            if (rr < rhi) a0 = fmaf(x[rr], y[rr], a0);
            red[rb * nb + cc] = a0 + a1;
        }
        // the previous column becomes its reflector (v below the diagonal, beta on it); no
        // thread reads it in this phase (the dot products above start at column c)
        if (c > 0) {
            const int jlp = j - 1 - r0;
            float *xp = slab + (c - 1) * Sp;
            const float fsp = scal_s[0];
            for (int rr = max(0, jlp + 1) + tid; rr < nr; rr += blockDim.x) xp[rr] *= fsp;
            if (jlp >= 0 && jlp < nr && tid == 0) xp[jlp] = scal_s[1];
        }
        __syncthreads();
        // this CTA's vector (sum over the row blocks; the row-j values from its owner), formed
        // once in shared memory, then copied into a slot of every CTA of the cluster
        for (int k = tid; k < 2 * live; k += blockDim.x) {
            if (k < live) {
                const int e = c + k;
                float sum = 0.f;
                for (int q = 0; q < nrb; ++q) sum += red[q * nb + e];
                vec[e] = sum;
            } else {
                const int e = nb + c + (k - live);
                vec[e] = own ? slab[(e - nb) * Sp + jl] : 0.f;
            }
        }
        __syncthreads();
        // the row-j values are nonzero only in the CTA that owns row j: only it sends them,
        // and the readers take them from its slot
        const int nsend = own ? 2 * live : live;
        for (int t = tid; t < CL * nsend; t += blockDim.x) {
            const int peer = t / nsend, k = t - peer * nsend;
            const int e = k < live ? c + k : nb + c + (k - live);
            float *dst = cluster.map_shared_rank(xch + ((long long)par * CL + rank) * 2 * nb, peer);
            dst[e] = vec[e];
        }
        cluster.sync();
        // warp 0: the cluster totals, the reflector (FP32, as single-precision Householder QR
        // computes it) and the coefficient f_c' = tau (v^T y_c') = tau (y_c',j + scal P_c')
        if (tid < 32) {
            const int lane = tid;
            const float *slots = xch + (long long)par * CL * 2 * nb;
            const float *oslot = slots + (long long)((j - j0) / S) * 2 * nb;   // the owner of row j
            float s2 = 0.f;
            for (int q = 0; q < CL; ++q) s2 += slots[q * 2 * nb + c];
            const float alpha = oslot[nb + c];
            const float fa = alpha, f2 = s2;
            float beta, tau, scal;
            if (f2 == 0.f) { beta = fa; tau = 0.f; scal = 0.f; }
            else {
                beta = -copysignf(sqrtf(fmaf(fa, fa, f2)), fa);
                tau = (beta - fa) / beta;
                scal = 1.f / (fa - beta);
            }
            for (int k = c + 1 + lane; k < pw; k += 32) {
                float pc = 0.f;
                for (int q = 0; q < CL; ++q) pc += slots[q * 2 * nb + k];
                coef[k] = tau * (oslot[nb + k] + pc * scal);
            }
            if (lane == 0) {
                scal_s[0] = scal;
                scal_s[1] = beta;
                if (rank == 0) {
                    P.tau[(long long)b * n + j] = tau;
                    P.beta[(long long)b * n + j] = beta;
                }
            }
        }
        __syncthreads();
        // y -= f_c' v for the later panel columns, v = [1; x * scal]
        if (cc > c && cc < pw) {
            float *y = slab + cc * Sp;
            const float f = coef[cc] * scal_s[0];
            for (int rr = max(rlo, start); rr < rhi; ++rr) y[rr] = fmaf(-f, x[rr], y[rr]);
            if (own && jl >= rlo && jl < rhi) y[jl] -= coef[cc];
        }
        __syncthreads();
    }
    if (pw > 0) {                                // the last column's reflector
        const int jlp = j0 + pw - 1 - r0;
        float *xp = slab + (pw - 1) * Sp;
        const float fsp = scal_s[0];
        for (int rr = max(0, jlp + 1) + tid; rr < nr; rr += blockDim.x) xp[rr] *= fsp;
        if (jlp >= 0 && jlp < nr && tid == 0) xp[jlp] = scal_s[1];
        __syncthreads();
    }

    // the factored panel back to UT (R entries above the diagonal, beta on it, v below);
    // the reflectors also as clean rows (YT: 0 above, 1 on the diagonal) and columns (Y)
    for (int c = 0; c < pw; ++c) {
        const int j = j0 + c;
        const long long o = ubase + (long long)j * P.ldm + r0;
        for (int rr = tid; rr < nr; rr += blockDim.x) {
            const int r = r0 + rr;
            const float v = slab[c * Sp + rr];
            float h, l;
            split_tf32(v, h, l);
            P.UThi[o + rr] = h;
            P.UTlo[o + rr] = l;
            split_tf32(r < j ? 0.f : (r == j ? 1.f : v), h, l);
            P.YThi[o + rr] = h;
            P.YTlo[o + rr] = l;
        }
    }
    const long long ybase = (long long)b * m * P.ldn;
    for (int t = tid; t < nr * pw; t += blockDim.x) {
        const int rr = t / pw, c = t - rr * pw;
        const int r = r0 + rr, j = j0 + c;
        const float v = slab[c * Sp + rr];
        float h, l;
        split_tf32(r < j ? 0.f : (r == j ? 1.f : v), h, l);
        P.Yhi[ybase + (long long)r * P.ldn + j] = h;
        P.Ylo[ybase + (long long)r * P.ldn + j] = l;
    }
    // partial G = Y^T Y over this CTA's rows (upper triangle), summed by CTA 0 into T
    float *gp = P.Gpart + ((long long)b * CL + rank) * nb * nb;
    for (int t = tid; t < pw * pw; t += blockDim.x) {
        const int i = t / pw, k = t - i * pw;
        if (k < i) continue;
        const int ji = j0 + i, jk = j0 + k;
        float acc = 0.f;
        for (int rr = max(0, jk - r0); rr < nr; ++rr) {      // Y_r,k = 0 above its diagonal (jk >= ji)
            const int r = r0 + rr;
            const float yi = r == ji ? 1.f : slab[i * Sp + rr];
            const float yk = r == jk ? 1.f : slab[k * Sp + rr];
            acc = fmaf(yi, yk, acc);
        }
        gp[i * nb + k] = acc;
    }
    __threadfence();
    cluster.sync();
    if (rank != 0) return;
    const int ldt = nb + 1;                          // padded rows: conflict-free column access
    float *G = slab, *T = slab + nb * ldt;           // the slab is no longer needed
    __syncthreads();
    for (int t = tid; t < pw * pw; t += blockDim.x) {
        const int i = t / pw, k = t - i * pw;
        float s = 0.f;
        if (k >= i)
            for (int q = 0; q < CL; ++q) s += P.Gpart[((long long)b * CL + q) * nb * nb + i * nb + k];
        G[i * ldt + k] = s;
        T[i * ldt + k] = 0.f;
    }
    __syncthreads();
    // T[c][c] = tau_c, T[:c, c] = -tau_c T[:c, :c] G[:c, c]  (G upper triangle)
    const float *tb = P.tau + (long long)b * n + j0;
    if (tid == 0) T[0] = tb[0];
    __syncthreads();
    for (int c = 1; c < pw; ++c) {
        float v = 0.f;
        if (tid < c)
            for (int l = tid; l < c; ++l) v += T[tid * ldt + l] * G[l * ldt + c];
        __syncthreads();
        if (tid < c) T[tid * ldt + c] = -tb[c] * v;
        if (tid == 0) T[c * ldt + c] = tb[c];
        __syncthreads();
    }
    float *out = P.Tm + ((long long)b * P.npan + P.panel) * nb * nb;
    for (int t = tid; t < nb * nb; t += blockDim.x) out[t] = t / nb < pw && t % nb < pw ? T[(t / nb) * ldt + t % nb] : 0.f;
}

// W2^T[c][i] = sum_l op(T)[i][l] W[l][c], W = sum of the ks K-split slices of Y^T X; op = T^T
// (factorization, X <- (I - Y T Y^T)^T X) or T (accumulation of Q, X <- (I - Y T Y^T) X).
// Tm holds the nb x nb T of every (matrix, panel).  One block of 8 warps per kTaCols columns:
// the block's columns of W (slices summed) are staged in shared memory with coalesced loads,
// warp g forms outputs i = g, g + 8, ... of every column (lane = column), and the block's
// rows of W2^T (kTaCols x nb, contiguous) are written back as float4.
constexpr int kTaCols = 32, kTaWarps = 8;
__global__ void __launch_bounds__(32 * kTaWarps) qr_tapply_kernel(const float *Wp, int ks, int B, int nb, int pw,
                                                                  int n, int ncol, const float *Tm, int npan,
                                                                  int panel, int trans, const int *skip,
                                                                  float *W2hi, float *W2lo) {
    __shared__ float Ts[64 * 65];                   // op(T), rows padded
    __shared__ float ws[64][kTaCols + 1];           // W[l][c] for the block's columns
    __shared__ __align__(16) float oh[kTaCols * 64], ol[kTaCols * 64];   // W2^T rows, hi and lo
    const int b = blockIdx.y;
    if (skip[b]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = blockIdx.x * kTaCols;
    const float *T = Tm + ((long long)b * npan + panel) * nb * nb;
    for (int t = threadIdx.x; t < pw * pw; t += blockDim.x) {
        const int i = t / pw, l = t - i * pw;
        Ts[i * 65 + l] = trans ? T[l * nb + i] : T[i * nb + l];
    }
    for (int l = warp; l < pw; l += kTaWarps) {
        const int c = c0 + lane;
        float sum = 0.f;
        if (c < ncol)
            for (int kc = 0; kc < ks; ++kc) sum += Wp[(((long long)kc * B + b) * nb + l) * n + c];
        ws[l][lane] = sum;
    }
    __syncthreads();
    for (int i = warp; i < nb; i += kTaWarps) {
        float sum = 0.f;
        if (i < pw)
            for (int l = 0; l < pw; ++l) sum += Ts[i * 65 + l] * ws[l][lane];
        float h, lo;
        split_tf32(sum, h, lo);
        oh[lane * 64 + i] = h;
        ol[lane * 64 + i] = lo;
    }
    __syncthreads();
    // rows c0 .. c0 + kTaCols - 1 of W2^T are contiguous (row length nb <= 64)
    const int ncols = min(kTaCols, ncol - c0);
    float *dh = W2hi + ((long long)b * n + c0) * nb, *dl = W2lo + ((long long)b * n + c0) * nb;
    if (nb == 64) {
        float4 *dh4 = reinterpret_cast<float4 *>(dh), *dl4 = reinterpret_cast<float4 *>(dl);
        const float4 *oh4 = reinterpret_cast<const float4 *>(oh), *ol4 = reinterpret_cast<const float4 *>(ol);
        for (int e = threadIdx.x; e < ncols * 16; e += blockDim.x) { dh4[e] = oh4[e]; dl4[e] = ol4[e]; }
    } else {
        for (int e = threadIdx.x; e < ncols * nb; e += blockDim.x) {
            const int c = e / nb, i = e - c * nb;
            dh[e] = oh[c * 64 + i];
            dl[e] = ol[c * 64 + i];
        }
    }
}

__global__ void qr_skip_kernel(const int *flag, int B, int *skip) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) skip[b] = flag ? (flag[b] ? 0 : 1) : 0;
}

// Q^T = [I 0] (split: hi = identity, lo = 0) for the factored matrices
__global__ void qr_qinit_kernel(int n, int m, long long ldm, const int *skip, float *QThi, float *QTlo) {
    const int b = blockIdx.z;
    if (skip[b]) return;
    const int c = blockIdx.y, r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const long long o = ((long long)b * n + c) * ldm + r;
    QThi[o] = r == c ? 1.f : 0.f;
    QTlo[o] = 0.f;
}

// Q[r][c] = sign(beta_c) Q^T[c][r] (transposed through a shared tile) and, if R is given,
// R[r][c] = sign(beta_r) (r < c ? UT[c][r] : r == c ? beta_c : 0).
__global__ void qr_store_kernel(const float *QThi, const float *QTlo, const float *UThi, const float *UTlo,
                                const float *beta, int m, int n, long long ldm, const int *skip, float *Q,
                                float *R) {
    __shared__ float tile[32][33];
    const int b = blockIdx.z;
    if (skip[b]) return;
    const int c0 = blockIdx.y * 32, r0 = blockIdx.x * 32;   // c: column of Q (row of Q^T)
    const float *bb = beta + (long long)b * n;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        float v = 0.f;
        if (c < n && r < m) {
            const long long o = ((long long)b * n + c) * ldm + r;
            v = (bb[c] < 0.f ? -1.f : 1.f) * (QThi[o] + QTlo[o]);
        }
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < m && c < n) Q[((long long)b * m + r) * n + c] = tile[threadIdx.x][i];
    }
    if (!R) return;
    // R rows r < n: reads UT[c][r] (row c of UT, coalesced over r = threadIdx.x), same tile shape
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        float v = 0.f;
        if (c < n && r < n) {
            const long long o = ((long long)b * n + c) * ldm + r;
            v = r < c ? UThi[o] + UTlo[o] : (r == c ? fabsf(bb[c]) : 0.f);
            if (r < c && bb[r] < 0.f) v = -v;
        }
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < n && c < n) R[((long long)b * n + r) * n + c] = tile[threadIdx.x][i];
    }
}

// One compact-WY application to rows [c0, c0 + ncol) of X^T (hi/lo, leading dim ldm), entries
// from j0 on: X^T[c][j0 + r] -= sum_i W2^T[c][i] Y[j0 + r][j0 + i] with W2 = op(T) Y^T X.
static int qr_apply_block(QrWS &w, int j0, int pw, int panel, int c0, int ncol, float *Xhi, float *Xlo, int trans,
                          cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n, nb = w.nb;
    const int K = m - j0;
    const long long nm = (long long)n * w.ldm;
    // W = Y^T X: A = Y^T rows of the panel (pw x K), B = X^T rows (ncol x K), split over K
    int ks = 1;
    {
        MatView ah = view_of(w.YThi + (long long)j0 * w.ldm + j0, pw, K, w.ldm, nm, B);
        MatView al = view_of(w.YTlo + (long long)j0 * w.ldm + j0, pw, K, w.ldm, nm, B);
        MatView bh = view_of(Xhi + (long long)c0 * w.ldm + j0, ncol, K, w.ldm, nm, B);
        MatView bl = view_of(Xlo + (long long)c0 * w.ldm + j0, ncol, K, w.ldm, nm, B);
        GemmShape s;
        memset(&s, 0, sizeof(s));
        s.M = pw; s.N = ncol; s.K = K; s.prec_uniform = PREC_TF32X3; s.skip = w.skip; s.err = w.err;
        const int tiles = ((ncol + 255) / 256) * B;
        s.ksplit = std::max(1, std::min(std::min(w.ks, (num_sms() + tiles - 1) / tiles), (K + 127) / 128));
        ks = s.ksplit;
        EpiStore e = epi_store_plain(w.Wp, n, (long long)nb * n, pw, ncol);
        PSVD_TRY(launch_gemm(nullptr, nullptr, &ah, &al, &bh, &bl, s, B, e, st));
    }
    {
        dim3 g((ncol + kTaCols - 1) / kTaCols, B);
        qr_tapply_kernel<<<g, 32 * kTaWarps, 0, st>>>(w.Wp, ks, B, nb, pw, n, ncol, w.Tm, w.npan, panel, trans,
                                                      w.skip, w.W2hi, w.W2lo);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    {
        MatView ah = view_of(w.W2hi, ncol, pw, nb, (long long)n * nb, B);
        MatView al = view_of(w.W2lo, ncol, pw, nb, (long long)n * nb, B);
        MatView bh = view_of(w.Yhi + (long long)j0 * w.ldn + j0, K, pw, w.ldn, (long long)m * w.ldn, B);
        MatView bl = view_of(w.Ylo + (long long)j0 * w.ldn + j0, K, pw, w.ldn, (long long)m * w.ldn, B);
        GemmShape s;
        memset(&s, 0, sizeof(s));
        s.M = ncol; s.N = K; s.K = pw; s.prec_uniform = PREC_TF32X3; s.skip = w.skip; s.err = w.err;
        EpiSubSplit e;
        e.rows = ncol; e.cols = K; e.hi = Xhi + (long long)c0 * w.ldm + j0; e.lo = Xlo + (long long)c0 * w.ldm + j0;
        e.ld = w.ldm; e.bs = nm;
        PSVD_TRY(launch_gemm(nullptr, nullptr, &ah, &al, &bh, &bl, s, B, e, st));
    }
    return PSVD_OK;
}

int qr_factor(const float *A, float *Q, float *R, const int *flag, QrWS &w, cudaStream_t st) {
    const int B = w.B, m = w.m, n = w.n, nb = w.nb, CL = w.cl;
    const long long nm = (long long)n * w.ldm;
    qr_skip_kernel<<<(B + 127) / 128, 128, 0, st>>>(flag, B, w.skip);
    count_launch(1);
    {
        SplitOut t;
        t.hi = w.UThi; t.lo = w.UTlo; t.ld = w.ldm; t.bstride = nm;
        PSVD_TRY(prepare_operand(A, n, (long long)m * n, B, m, n, true, 1.f, nullptr, t, st, w.skip));
    }
    const size_t smem = qr_panel_smem(m, nb, CL);
    PSVD_TRY(cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CL > 8) PSVD_TRY(cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(B * CL));
    cfg.blockDim = dim3(kQrThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int p = 0; p < w.npan; ++p) {
        const int j0 = p * nb, pw = std::min(nb, n - j0);
        PanelArgs a;
        a.UThi = w.UThi; a.UTlo = w.UTlo; a.YThi = w.YThi; a.YTlo = w.YTlo; a.Yhi = w.Yhi; a.Ylo = w.Ylo;
        a.tau = w.tau; a.beta = w.beta; a.Tm = w.Tm; a.Gpart = w.Gpart; a.skip = w.skip;
        a.m = m; a.n = n; a.j0 = j0; a.pw = pw; a.panel = p; a.npan = w.npan; a.nb = nb; a.cl = CL;
        a.ldm = w.ldm; a.ldn = w.ldn;
        PSVD_TRY(cudaLaunchKernelEx(&cfg, qr_panel_kernel, a));
        count_launch(1);
        const int c0 = j0 + pw, ncol = n - c0;
        if (ncol > 0) PSVD_TRY_RC(qr_apply_block(w, j0, pw, p, c0, ncol, w.UThi, w.UTlo, 1, st));
    }
    {
        dim3 g((m + 127) / 128, n, B);
        qr_qinit_kernel<<<g, 128, 0, st>>>(n, m, w.ldm, w.skip, w.QThi, w.QTlo);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    for (int p = w.npan - 1; p >= 0; --p) {
        const int j0 = p * nb, pw = std::min(nb, n - j0);
        PSVD_TRY_RC(qr_apply_block(w, j0, pw, p, j0, n - j0, w.QThi, w.QTlo, 0, st));
    }
    {
        dim3 g((m + 31) / 32, (n + 31) / 32, B), blk(32, 8);
        qr_store_kernel<<<g, blk, 0, st>>>(w.QThi, w.QTlo, w.UThi, w.UTlo, w.beta, m, n, w.ldm, w.skip, Q, R);
        count_launch(1);
        PSVD_TRY(cudaGetLastError());
    }
    return PSVD_OK;
}

}  // namespace psvd

using namespace psvd;

extern "C" size_t psvd_qr_workspace_bytes(int64_t batch, int64_t m, int64_t n) {
    if (batch <= 0 || m <= 0 || n <= 0) return 0;
    Sizer s;
    QrWS w;
    w.carve(s, (int)batch, (int)m, (int)n);
    return s.used + 256;
}

extern "C" int psvd_qr(const float *A, float *Q, float *R, int64_t batch, int64_t m, int64_t n, void *ws,
                       size_t ws_bytes, void *stream) {
    int nb = 0, cl = 0;
    if (!A || !Q || batch <= 0 || n <= 0 || m < n || batch > 65535 || n > 16384 || (long long)m * n > (1LL << 31))
        return PSVD_ERR_ARG;
    if (!qr_shape((int)m, &nb, &cl))
        return fail_msg(PSVD_ERR_ARG, "psvd_qr: m = %lld rows exceed the cluster panel", (long long)m);
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_qr_workspace_bytes(batch, m, n)) return PSVD_ERR_WORKSPACE;
    Carver cv(ws, ws_bytes);
    QrWS w;
    w.carve(cv, (int)batch, (int)m, (int)n);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    return qr_factor(A, Q, R, nullptr, w, static_cast<cudaStream_t>(stream));
}
