// Learned lower bound for the polynomial schedule: sketch features of the
// normalized matrix and a small MLP (8 -> 64 -> 64 -> 1, ReLU) trained with Adam on
// spectra the method itself produces.  The predicted value is log of a lower bound on
// sigma_min(X0); the schedule then starts from [l, 1] (greedy optimal cubics) and a
// matrix whose residual misses the tolerance within budget is rerun with the
// conservative CANS schedule.
#include <cmath>
#include <cstring>

#include "ops.cuh"

namespace psvd {

cudaError_t l1_norms(const float *A, int B, int m, int n, float *rowsum, float *colsum, int *nonfinite,
                     cudaStream_t st);
__global__ void norm_finalize_kernel(const float *rowsum, const float *colsum, const int *nonfinite, int m, int n,
                                     float *scale, int *done, int *status, int *fin);

constexpr int kH = 64, kF = 8;
constexpr int kP_W1 = 0, kP_b1 = kH * kF, kP_W2 = kP_b1 + kH, kP_b2 = kP_W2 + kH * kH, kP_W3 = kP_b2 + kH,
              kP_b3 = kP_W3 + kH, kNP = kP_b3 + 1;
static_assert(kNP == PSVD_MLP_NPARAMS, "parameter layout");

constexpr int kXtyChunks = 32;     // row chunks of X0^T T (partial sums, reduced in order)
constexpr int kFroBlocks = 64;     // blocks per matrix of ||X0||_F^2 (partial sums, reduced in order)

struct SketchWS {
    float *rowsum, *colsum, *scale, *T, *Y, *Ypart, *acc, *fro, *fropart;
    int *nonfinite, *done, *status, *fin;
    template <class C>
    void carve(C &cv, long long B, long long m, long long n, long long s) {
        rowsum = cv.template take<float>(B * m);
        colsum = cv.template take<float>(B * n);
        scale = cv.template take<float>(B);
        T = cv.template take<float>(B * m * s);
        Y = cv.template take<float>(B * n * s);
        Ypart = cv.template take<float>(B * kXtyChunks * n * s);
        fropart = cv.template take<float>(B * kFroBlocks * 2);
        acc = cv.template take<float>(B * 4);
        fro = cv.template take<float>(B);
        nonfinite = cv.template take<int>(B);
        done = cv.template take<int>(B);
        status = cv.template take<int>(B);
        fin = cv.template take<int>(B);
    }
};

// out[b][i][p] = (1/scale_b) sum_k A[b][i][k] Y[b][k][p]     (X0 Y, one warp per (b, i))
__global__ void xy_kernel(const float *A, const float *scale, const float *Y, int m, int n, int s, float *out) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.y;
    if (warp >= m) return;
    const float *a = A + (long long)b * m * n + (long long)warp * n;
    const float *y = Y + (long long)b * n * s;
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    float acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
    for (int k = lane; k < n; k += 32) {
        const float x = a[k] * sc;
#pragma unroll
        for (int p = 0; p < 8; ++p) if (p < s) acc[p] += x * y[(long long)k * s + p];
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const float v = warp_sum(acc[p]);
        if (lane == 0 && p < s) out[(long long)b * m * s + (long long)warp * s + p] = v;
    }
}

// part[b][r][k][p] = (1/scale_b) sum over rows i of chunk r of A[b][i][k] T[b][i][p]
// (X0^T T split over kXtyChunks row chunks; one thread per (b, r, k), coalesced over k)
__global__ void xty_part_kernel(const float *A, const float *scale, const float *T, int m, int n, int s,
                                float *part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y, r = blockIdx.z;
    if (k >= n) return;
    const int rows = (m + kXtyChunks - 1) / kXtyChunks;
    const int i0 = r * rows, i1 = min(m, i0 + rows);
    const float *a = A + (long long)b * m * n;
    const float *t = T + (long long)b * m * s;
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    float acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
    for (int i = i0; i < i1; ++i) {
        const float x = a[(long long)i * n + k] * sc;
#pragma unroll
        for (int p = 0; p < 8; ++p) if (p < s) acc[p] += x * t[(long long)i * s + p];
    }
    float *o = part + (((long long)b * kXtyChunks + r) * n + k) * s;
#pragma unroll
    for (int p = 0; p < 8; ++p) if (p < s) o[p] = acc[p];
}

// out[b][k][p] = sum_r part[b][r][k][p], in chunk order
__global__ void xty_reduce_kernel(const float *part, int n, int s, float *out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (idx >= (long long)n * s) return;
    float v = 0.f;
    for (int r = 0; r < kXtyChunks; ++r) v += part[((long long)b * kXtyChunks + r) * n * s + idx];
    out[(long long)b * n * s + idx] = v;
}

// acc[b][j] += sum z .* y  (Hutchinson term for power j)
__global__ void zdot_kernel(const float *Z, const float *Y, int n, int s, int j, float *acc) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    float v = 0.f;
    for (long long i = threadIdx.x; i < (long long)n * s; i += blockDim.x)
        v += Z[(long long)b * n * s + i] * Y[(long long)b * n * s + i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        acc[b * 4 + j] = t;
    }
}

// ||X0||_F^2 per matrix: kFroBlocks compensated partial sums (hi, lo), reduced in order
__global__ void fro_part_kernel(const float *A, const float *scale, long long mn, float *part) {
    __shared__ float red[64];
    const int b = blockIdx.y, blk = blockIdx.x;
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    ff v = ff_zero();
    for (long long i = (long long)blk * blockDim.x + threadIdx.x; i < mn; i += (long long)kFroBlocks * blockDim.x) {
        const float x = A[(long long)b * mn + i] * sc;
        v = ff_fma(v, x, x);
    }
    const float t = block_sum_ff(v, red);
    if (threadIdx.x == 0) { part[((long long)b * kFroBlocks + blk) * 2] = t; part[((long long)b * kFroBlocks + blk) * 2 + 1] = 0.f; }
}

__global__ void fro_reduce_kernel(const float *part, int B, float *fro) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    ff v = ff_zero();
    for (int k = 0; k < kFroBlocks; ++k) v = ff_add(v, ff{part[((long long)b * kFroBlocks + k) * 2], 0.f});
    fro[b] = __fadd_rn(v.hi, v.lo);
}

__global__ void features_kernel(const float *acc, const float *fro, int B, int m, int n, int s, float *F) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float inv = 1.f / ((float)n * (float)s);
    const float tiny = 1e-30f;
    float t[4];
    for (int j = 0; j < 4; ++j) t[j] = acc[b * 4 + j] * inv;
    float *f = F + (long long)b * kF;
    for (int j = 0; j < 4; ++j) f[j] = logf(fmaxf(t[j], tiny));
    f[4] = logf(fmaxf(fro[b] / (float)n, tiny));
    f[5] = logf(fmaxf(t[3], tiny) / fmaxf(t[2], tiny));
    f[6] = logf((float)n) / 10.f;
    f[7] = logf((float)m / (float)n);
}

// ------------------------------------------------------------ MLP
// One thread per sample; parameters staged in shared memory.
__global__ void mlp_fwd_kernel(const float *params, const float *F, int nb, float *Y) {
    __shared__ float P[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    float f[kF], h1[kH];
#pragma unroll
    for (int i = 0; i < kF; ++i) f[i] = F[(long long)t * kF + i];
    for (int o = 0; o < kH; ++o) {
        float z = P[kP_b1 + o];
#pragma unroll
        for (int i = 0; i < kF; ++i) z += P[kP_W1 + o * kF + i] * f[i];
        h1[o] = fmaxf(z, 0.f);
    }
    float y = P[kP_b3];
    for (int o = 0; o < kH; ++o) {
        float z = P[kP_b2 + o];
        for (int i = 0; i < kH; ++i) z += P[kP_W2 + o * kH + i] * h1[i];
        y += P[kP_W3 + o] * fmaxf(z, 0.f);
    }
    Y[t] = y;
}

// Gradients of 0.5 mean (y - target)^2; block-level accumulation in shared memory.
__global__ void mlp_grad_kernel(const float *params, const float *F, const float *target, int nb, float *grads,
                                float *loss) {
    __shared__ float P[kNP];
    __shared__ float G[kNP];
    __shared__ float lsum;
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) { P[i] = params[i]; G[i] = 0.f; }
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nb) {
        float f[kF], z1[kH], h1[kH], z2[kH];
#pragma unroll
        for (int i = 0; i < kF; ++i) f[i] = F[(long long)t * kF + i];
        for (int o = 0; o < kH; ++o) {
            float z = P[kP_b1 + o];
#pragma unroll
            for (int i = 0; i < kF; ++i) z += P[kP_W1 + o * kF + i] * f[i];
            z1[o] = z;
            h1[o] = fmaxf(z, 0.f);
        }
        float y = P[kP_b3];
        for (int o = 0; o < kH; ++o) {
            float z = P[kP_b2 + o];
            for (int i = 0; i < kH; ++i) z += P[kP_W2 + o * kH + i] * h1[i];
            z2[o] = z;
            y += P[kP_W3 + o] * fmaxf(z, 0.f);
        }
        const float r = y - target[t];
        atomicAdd(&lsum, 0.5f * r * r / nb);
        const float dy = r / nb;
        atomicAdd(&G[kP_b3], dy);
        float dh1[kH];
        for (int i = 0; i < kH; ++i) dh1[i] = 0.f;
        for (int o = 0; o < kH; ++o) {
            const float h2 = fmaxf(z2[o], 0.f);
            atomicAdd(&G[kP_W3 + o], dy * h2);
            const float dz2 = z2[o] > 0.f ? dy * P[kP_W3 + o] : 0.f;
            if (dz2 != 0.f) {
                atomicAdd(&G[kP_b2 + o], dz2);
                for (int i = 0; i < kH; ++i) {
                    atomicAdd(&G[kP_W2 + o * kH + i], dz2 * h1[i]);
                    dh1[i] += dz2 * P[kP_W2 + o * kH + i];
                }
            }
        }
        for (int o = 0; o < kH; ++o) {
            const float dz1 = z1[o] > 0.f ? dh1[o] : 0.f;
            if (dz1 != 0.f) {
                atomicAdd(&G[kP_b1 + o], dz1);
#pragma unroll
                for (int i = 0; i < kF; ++i) atomicAdd(&G[kP_W1 + o * kF + i], dz1 * f[i]);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kNP; i += blockDim.x)
        if (G[i] != 0.f) atomicAdd(&grads[i], G[i]);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, lsum);
}

__global__ void adam_kernel(float *params, const float *grads, float *m1, float *m2, float lr, float b1t, float b2t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float g = grads[i];
    const float a = 0.9f * m1[i] + 0.1f * g;
    const float b = 0.999f * m2[i] + 0.001f * g * g;
    m1[i] = a;
    m2[i] = b;
    const float mh = a / (1.f - b1t), vh = b / (1.f - b2t);
    params[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

}  // namespace psvd

using namespace psvd;

extern "C" size_t psvd_sketch_workspace_bytes(int64_t batch, int64_t m, int64_t n, int64_t s) {
    if (batch <= 0 || m <= 0 || n <= 0 || s <= 0) return 0;
    Sizer z;
    SketchWS w;
    w.carve(z, batch, m, n, s);
    return z.used + 256;
}

extern "C" int psvd_sketch_features(const float *A, const float *Z, int64_t s, float *F, int64_t batch, int64_t m,
                                    int64_t n, void *ws, size_t ws_bytes, void *stream) {
    if (!A || !Z || !F || batch <= 0 || n <= 0 || m < n || s < 1 || s > 8 || batch > 65535) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_sketch_workspace_bytes(batch, m, n, s)) return PSVD_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carver cv(ws, ws_bytes);
    SketchWS w;
    w.carve(cv, batch, m, n, s);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    const int B = (int)batch, M = (int)m, Nn = (int)n, S = (int)s;
    PSVD_TRY(cudaMemsetAsync(w.rowsum, 0, sizeof(float) * batch * m, st));
    PSVD_TRY(cudaMemsetAsync(w.colsum, 0, sizeof(float) * batch * n, st));
    PSVD_TRY(cudaMemsetAsync(w.nonfinite, 0, sizeof(int) * batch, st));
    PSVD_TRY(l1_norms(A, B, M, Nn, w.rowsum, w.colsum, w.nonfinite, st));
    norm_finalize_kernel<<<B, 256, 0, st>>>(w.rowsum, w.colsum, w.nonfinite, M, Nn, w.scale, w.done, w.status, w.fin);
    fro_part_kernel<<<dim3(kFroBlocks, B), 256, 0, st>>>(A, w.scale, (long long)m * n, w.fropart);
    fro_reduce_kernel<<<(B + 127) / 128, 128, 0, st>>>(w.fropart, B, w.fro);
    count_launch(3);
    // Y_{j+1} = X0^T (X0 Y_j), Y_0 = Z; f_j = <Z, Y_{j+1}> / (n s)
    const float *Y = Z;
    for (int j = 0; j < 4; ++j) {
        xy_kernel<<<dim3((M * 32 + 255) / 256, B), 256, 0, st>>>(A, w.scale, Y, M, Nn, S, w.T);
        xty_part_kernel<<<dim3((Nn + 127) / 128, B, kXtyChunks), 128, 0, st>>>(A, w.scale, w.T, M, Nn, S, w.Ypart);
        xty_reduce_kernel<<<dim3((unsigned)(((long long)Nn * S + 255) / 256), B), 256, 0, st>>>(w.Ypart, Nn, S, w.Y);
        zdot_kernel<<<B, 256, 0, st>>>(Z, w.Y, Nn, S, j, w.acc);
        count_launch(4);
        Y = w.Y;
    }
    features_kernel<<<(B + 127) / 128, 128, 0, st>>>(w.acc, w.fro, B, M, Nn, S, F);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_fwd(const float *params, const float *F, float *Y, int64_t nb, void *stream) {
    if (!params || !F || !Y || nb <= 0) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    mlp_fwd_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(params, F, (int)nb, Y);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

// Lower bound of sigma_min(X0) from the network's log prediction: margin * exp(y), kept
// inside [1e-12, 0.999] (the schedule needs 0 < l < 1).
__global__ void lower_bound_kernel(float *Y, int nb, float margin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) Y[i] = fminf(fmaxf(margin * expf(Y[i]), 1e-12f), 0.999f);
}

extern "C" int psvd_mlp_lower_bound(const float *params, const float *F, float *LB, int64_t nb, float margin,
                                    void *stream) {
    if (!params || !F || !LB || nb <= 0 || !(margin > 0.f)) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_fwd_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(params, F, (int)nb, LB);
    lower_bound_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(LB, (int)nb, margin);
    count_launch(2);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_grad(const float *params, const float *F, const float *target, int64_t nb, float *grads,
                             float *loss, void *stream) {
    if (!params || !F || !target || !grads || nb <= 0) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PSVD_TRY(cudaMemsetAsync(grads, 0, sizeof(float) * kNP, st));
    if (loss) PSVD_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    mlp_grad_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(params, F, target, (int)nb, grads, loss);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_train_step(float *params, float *grads, float *m1, float *m2, const float *F,
                                   const float *target, int64_t nb, float lr, int step, float *loss, void *stream) {
    if (!m1 || !m2 || step < 1) return PSVD_ERR_ARG;
    if (int rc = psvd_mlp_grad(params, F, target, nb, grads, loss, stream)) return rc;
    const float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    adam_kernel<<<(kNP + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grads, m1, m2, lr, b1t, b2t);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

namespace psvd {

// ------------------------------------------------------------ training helpers
// Per-feature mean and sample standard deviation over nb rows (one block per feature, FP64
// sums in a fixed order), floored at 1e-6, and the standardized copy Fs = (F - mean) / std.
__global__ void feat_stats_kernel(const float *F, int nb, float *stats) {
    __shared__ double red[32];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += (double)F[(long long)i * kF + f];
    s = block_sum(s, red);
    const double mean = s / nb;
    double q = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double d = (double)F[(long long)i * kF + f] - mean;
        q += d * d;
    }
    q = block_sum(q, red);
    if (threadIdx.x == 0) {
        stats[f] = (float)mean;
        stats[kF + f] = (float)fmax(sqrt(nb > 1 ? q / (nb - 1) : 0.0), 1e-6);
    }
}

__global__ void feat_standardize_kernel(const float *F, const float *stats, long long total, float *Fs) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int f = (int)(t % kF);
    Fs[t] = (F[t] - stats[f]) / stats[kF + f];
}

// A network trained on standardized features, made to act on raw ones:
// W1 <- W1 / std (column-wise), b1 <- b1 - W1_new mean.  One block of kH threads (one per row).
__global__ void mlp_fold_kernel(float *params, const float *stats) {
    const int r = threadIdx.x;
    if (r >= kH) return;
    float *w = params + kP_W1 + r * kF;
    float acc = 0.f;
    for (int f = 0; f < kF; ++f) {
        w[f] = w[f] / stats[kF + f];
        acc += w[f] * stats[f];
    }
    params[kP_b1 + r] -= acc;
}

// Minibatch rows: Fb[i] = F[idx[i]], tb[i] = t[idx[i]].
__global__ void mlp_gather_kernel(const float *F, const float *t, const int *idx, int nbo, float *Fb, float *tb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbo) return;
    const int j = idx[i];
#pragma unroll
    for (int f = 0; f < kF; ++f) Fb[(long long)i * kF + f] = F[(long long)j * kF + f];
    tb[i] = t[j];
}

// margin = exp(-max(q, 0)) with q the `quantile` of the over-prediction d = y - target
// (linear interpolation between the order statistics d_(k) and d_(k+1), k = floor((nb-1) q),
// the usual definition).  Each order statistic is found exactly, in one block, by bisection
// over the 32-bit keys that order the floats (sign bit flipped for positive values, all bits
// for negative ones): the smallest key K with #{d : key(d) <= K} > k is the key of d_(k).
PSVD_DEV unsigned order_key(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
PSVD_DEV float key_value(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void mlp_margin_kernel(const float *Y, const float *target, int nb, float quantile, float *margin) {
    __shared__ int cnt[32];
    const double h = (double)(nb - 1) * quantile;
    const int k = (int)floor(h);
    const int nw = (int)(blockDim.x >> 5);
    float os[2];
    for (int which = 0; which < 2; ++which) {
        const int kk = min(k + which, nb - 1);
        unsigned long long lo = 0, hi = 0xffffffffull;      // answer in [lo, hi]
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) >> 1;
            int c = 0;
            for (int i = threadIdx.x; i < nb; i += blockDim.x) c += order_key(Y[i] - target[i]) <= (unsigned)mid;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = c;
            __syncthreads();
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += cnt[w];
            if (tot > kk) hi = mid; else lo = mid + 1;
        }
        os[which] = key_value((unsigned)lo);
    }
    if (threadIdx.x == 0) {
        const double q = (double)os[0] + (h - k) * ((double)os[1] - (double)os[0]);
        margin[0] = (float)exp(-fmax(q, 0.0));
    }
}

}  // namespace psvd

using namespace psvd;

extern "C" int psvd_mlp_standardize(const float *F, int64_t nb, float *Fs, float *stats, void *stream) {
    if (!F || !stats || nb <= 0 || nb > (1LL << 30)) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    feat_stats_kernel<<<kF, 256, 0, st>>>(F, (int)nb, stats);
    count_launch(1);
    if (Fs) {
        const long long total = nb * kF;
        feat_standardize_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(F, stats, total, Fs);
        count_launch(1);
    }
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_fold(float *params, const float *stats, void *stream) {
    if (!params || !stats) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    mlp_fold_kernel<<<1, kH, 0, static_cast<cudaStream_t>(stream)>>>(params, stats);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_gather(const float *F, const float *target, const int *idx, int64_t nb, float *Fb,
                               float *tb, void *stream) {
    if (!F || !target || !idx || !Fb || !tb || nb <= 0 || nb > (1LL << 30)) return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    mlp_gather_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(F, target, idx,
                                                                                                   (int)nb, Fb, tb);
    count_launch(1);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}

extern "C" int psvd_mlp_calibrate(const float *params, const float *F, const float *target, int64_t nb,
                                  float quantile, float *Y, float *margin, void *stream) {
    if (!params || !F || !target || !Y || !margin || nb <= 0 || nb > (1LL << 30) || !(quantile >= 0.f) ||
        !(quantile <= 1.f))
        return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_fwd_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(params, F, (int)nb, Y);
    mlp_margin_kernel<<<1, 1024, 0, st>>>(Y, target, (int)nb, quantile, margin);
    count_launch(2);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}
