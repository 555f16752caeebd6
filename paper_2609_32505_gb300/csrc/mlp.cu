// Learned lower bound for the polynomial schedule: sketch features of the
// normalized matrix and a small MLP (8 -> 64 -> 64 -> 1, ReLU) trained with Adam on
// spectra the method itself produces.  The predicted value is log of a lower bound on
// sigma_min(X0); the schedule then starts from [l, 1] (greedy optimal cubics) and a
// matrix whose residual misses the tolerance within budget is rerun with the
// conservative CANS schedule.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ops.cuh"

namespace psvd {

cudaError_t l1_norms(const float *A, int B, int m, int n, float *rowsum, float *colsum, int *nonfinite,
                     cudaStream_t st);
__global__ void __launch_bounds__(kNormThreads) norm_finalize_kernel(const float *rowsum, const float *colsum,
                                                                      const int *nonfinite, int m, int n,
                                     float *scale, int *done, int *status, int *fin);

constexpr int kH = 64, kF = 8;
constexpr int kP_W1 = 0, kP_b1 = kH * kF, kP_W2 = kP_b1 + kH, kP_b2 = kP_W2 + kH * kH, kP_W3 = kP_b2 + kH,
              kP_b3 = kP_W3 + kH, kNP = kP_b3 + 1;
static_assert(kNP == PSVD_MLP_NPARAMS, "parameter layout");

constexpr int kXtyChunks = 32;     // row chunks of X0^T T (partial sums, reduced in order)
constexpr int kFroBlocks = 256;    // blocks per matrix of ||X0||_F^2 (partial sums, reduced in order)
constexpr int kZdotBlocks = 16;    // slices per matrix of the Hutchinson dot products
constexpr int kTs = 8;             // row stride of T = X0 Y (two float4 per row)

struct SketchWS {
    float *rowsum, *colsum, *scale, *T, *Y, *ZT, *Ypart, *acc, *fro, *fropart;
    int *nonfinite, *done, *status, *fin;
    template <class C>
    void carve(C &cv, long long B, long long m, long long n, long long s) {
        rowsum = cv.template take<float>(B * m);
        colsum = cv.template take<float>(B * l1_slabs((int)m) * n);
        scale = cv.template take<float>(B);
        T = cv.template take<float>(B * m * kTs);
        Y = cv.template take<float>(B * n * s);
        ZT = cv.template take<float>(B * n * s);
        Ypart = cv.template take<float>(B * kXtyChunks * n * s);
        fropart = cv.template take<float>(B * kFroBlocks);
        acc = cv.template take<float>(B * 4 * kZdotBlocks);
        fro = cv.template take<float>(B);
        nonfinite = cv.template take<int>(B);
        done = cv.template take<int>(B);
        status = cv.template take<int>(B);
        fin = cv.template take<int>(B);
    }
};

// The probes are kept probe-major inside the sketch: YT[b][p][k] (k contiguous), so a warp's
// reads of a probe row are coalesced; T = X0 Y is stored with rows of kTs = 8 floats.

// ZT[b][p][k] = Z[b][k][p]
__global__ void probe_transpose_kernel(const float *Z, int n, int s, float *ZT) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (t >= (long long)n * s) return;
    const int p = (int)(t / n), k = (int)(t % n);
    ZT[(b * s + p) * n + k] = Z[(b * n + k) * s + p];
}

// T[b][i][p] = (1/scale_b) sum_k A[b][i][k] YT[b][p][k]     (X0 Y).
// Vector form (n % 4 == 0 and A 16-byte aligned): a block of 8 warps takes kXyRows rows,
// two per warp; the probe columns of each K chunk are staged once per block in shared memory
// and every staged float4 serves both rows of a warp, so the probes are read from L2 once per
// kXyRows rows instead of once per row.
constexpr int kXyRows = 16, kXyKc = 512;
__global__ void __launch_bounds__(256) xy_vec_kernel(const float *A, const float *scale, const float *YT, int m,
                                                     int n, int s, float *T) {
    __shared__ float4 yt[8][kXyKc / 4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, b = blockIdx.y;
    const int r0 = blockIdx.x * kXyRows + 2 * warp;
    const int c4 = n >> 2;
    const float4 *a4[2];
#pragma unroll
    for (int q = 0; q < 2; ++q)
        a4[q] = reinterpret_cast<const float4 *>(A + (long long)b * m * n + (long long)min(r0 + q, m - 1) * n);
    const float4 *y4 = reinterpret_cast<const float4 *>(YT + (long long)b * s * n);
    float acc[2][8];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[q][p] = 0.f;
    for (int k0 = 0; k0 < c4; k0 += kXyKc / 4) {
        const int kc = min(kXyKc / 4, c4 - k0);
        __syncthreads();                                  // the previous chunk has been used
        for (int e = threadIdx.x; e < s * (kXyKc / 4); e += blockDim.x) {
            const int p = e / (kXyKc / 4), c = e % (kXyKc / 4);
            if (c < kc) yt[p][c] = y4[(long long)p * c4 + k0 + c];
        }
        __syncthreads();
        for (int c = lane; c < kc; c += 32) {
            const float4 x0 = a4[0][k0 + c], x1 = a4[1][k0 + c];
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                if (p < s) {
                    const float4 v = yt[p][c];
                    acc[0][p] += x0.x * v.x + x0.y * v.y + x0.z * v.z + x0.w * v.w;
                    acc[1][p] += x1.x * v.x + x1.y * v.y + x1.z * v.z + x1.w * v.w;
                }
            }
        }
    }
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const float v = warp_sum(acc[q][p]) * sc;
            if (lane == 0 && r0 + q < m) T[((long long)b * m + r0 + q) * kTs + p] = p < s ? v : 0.f;
        }
}

// Scalar form of the same product (any n or alignment): one warp per row.
__global__ void __launch_bounds__(256) xy_kernel(const float *A, const float *scale, const float *YT, int m, int n,
                                                 int s, float *T) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.y;
    if (warp >= m) return;
    const float *a = A + (long long)b * m * n + (long long)warp * n;
    const float *y = YT + (long long)b * s * n;
    float acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
    for (int k = lane; k < n; k += 32) {
        const float x = a[k];
#pragma unroll
        for (int p = 0; p < 8; ++p) if (p < s) acc[p] += x * y[(long long)p * n + k];
    }
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const float v = warp_sum(acc[p]) * sc;
        if (lane == 0) T[((long long)b * m + warp) * kTs + p] = p < s ? v : 0.f;
    }
}

// part[b][r][p][k] = (1/scale_b) sum over rows i of chunk r of A[b][i][k] T[b][i][p]
// (X0^T T split over kXtyChunks row chunks).  Vector form: one thread per (b, r, 4 columns),
// float4 loads of eight rows in flight; the chunk's rows of T are staged in shared memory.
constexpr int kXtyMaxRows = 512;       // rows of a chunk staged at once
__global__ void __launch_bounds__(128) xty_vec_kernel(const float *A, const float *scale, const float *T, int m,
                                                      int n, int s, float *part) {
    __shared__ float4 ts[kXtyMaxRows][2];
    const int k = 4 * (blockIdx.x * blockDim.x + threadIdx.x), b = blockIdx.y, r = blockIdx.z;
    const int rows = (m + kXtyChunks - 1) / kXtyChunks;
    const int i0 = r * rows, i1 = min(m, i0 + rows);
    const float4 *t4 = reinterpret_cast<const float4 *>(T + (long long)b * m * kTs);
    float acc[4][8];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[e][p] = 0.f;
    for (int j0 = i0; j0 < i1; j0 += kXtyMaxRows) {
        const int j1 = min(i1, j0 + kXtyMaxRows);
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * (j1 - j0); e += blockDim.x) ts[e >> 1][e & 1] = t4[(long long)(j0 + (e >> 1)) * 2 + (e & 1)];
        __syncthreads();
        if (k < n) {
            const float *a = A + (long long)b * m * n + k;
            for (int i = j0; i < j1; i += 8) {
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    x[u] = i + u < j1 ? *reinterpret_cast<const float4 *>(a + (long long)(i + u) * n)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (i + u >= j1) break;
                    const float4 t0 = ts[i + u - j0][0], t1 = ts[i + u - j0][1];
                    const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                    const float xv[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
#pragma unroll
                        for (int p = 0; p < 8; ++p) acc[e][p] += xv[e] * tv[p];
                }
            }
        }
    }
    if (k >= n) return;
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    float *o = part + (((long long)b * kXtyChunks + r) * s) * n + k;
#pragma unroll
    for (int p = 0; p < 8; ++p)
        if (p < s) *reinterpret_cast<float4 *>(o + (long long)p * n) =
            make_float4(acc[0][p] * sc, acc[1][p] * sc, acc[2][p] * sc, acc[3][p] * sc);
}

// Scalar form: one thread per (b, r, k), coalesced over k, sixteen rows of loads in flight.
__global__ void __launch_bounds__(128) xty_part_kernel(const float *A, const float *scale, const float *T, int m,
                                                       int n, int s, float *part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y, r = blockIdx.z;
    if (k >= n) return;
    const int rows = (m + kXtyChunks - 1) / kXtyChunks;
    const int i0 = r * rows, i1 = min(m, i0 + rows);
    const float *a = A + (long long)b * m * n + k;
    const float4 *t4 = reinterpret_cast<const float4 *>(T + (long long)b * m * kTs);
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    float acc[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) acc[p] = 0.f;
    for (int i = i0; i < i1; i += 16) {
        float x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = i + u < i1 ? a[(long long)(i + u) * n] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (i + u < i1) {
                const float4 t0 = t4[(long long)(i + u) * 2], t1 = t4[(long long)(i + u) * 2 + 1];
                acc[0] += x[u] * t0.x; acc[1] += x[u] * t0.y; acc[2] += x[u] * t0.z; acc[3] += x[u] * t0.w;
                acc[4] += x[u] * t1.x; acc[5] += x[u] * t1.y; acc[6] += x[u] * t1.z; acc[7] += x[u] * t1.w;
            }
        }
    }
    float *o = part + (((long long)b * kXtyChunks + r) * s) * n + k;
#pragma unroll
    for (int p = 0; p < 8; ++p) if (p < s) o[(long long)p * n] = acc[p] * sc;
}

// YT[b][p][k] = sum_r part[b][r][p][k], in chunk order
__global__ void xty_reduce_kernel(const float *part, int n, int s, float *YT) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (idx >= (long long)n * s) return;
    float v = 0.f;
    for (int r = 0; r < kXtyChunks; ++r) v += part[((long long)b * kXtyChunks + r) * n * s + idx];
    YT[(long long)b * n * s + idx] = v;
}

// accpart[b][j][blk] = sum over slice blk of z .* y  (Hutchinson term for power j, in
// kZdotBlocks slices added in order by features_kernel; both probe-major)
__global__ void zdot_kernel(const float *Z, const float *Y, int n, int s, int j, float *accpart) {
    __shared__ float red[32];
    const int b = blockIdx.y, blk = blockIdx.x;
    const long long len = (long long)n * s, per = (len + kZdotBlocks - 1) / kZdotBlocks;
    const long long e0 = blk * per, e1 = min(len, e0 + per);
    float v = 0.f;
    for (long long i = e0 + threadIdx.x; i < e1; i += blockDim.x)
        v += Z[(long long)b * len + i] * Y[(long long)b * len + i];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        accpart[((long long)b * 4 + j) * kZdotBlocks + blk] = t;
    }
}

// ||X0||_F^2 per matrix: kFroBlocks compensated partial sums, reduced in order.  With vec
// (m n % 4 == 0 and A 16-byte aligned) float4 loads, four in flight per thread.
template <bool kVec>
__global__ void __launch_bounds__(256) fro_part_kernel(const float *A, const float *scale, long long mn, float *part) {
    __shared__ float red[64];
    const int b = blockIdx.y, blk = blockIdx.x;
    const float sc = scale[b] > 0.f ? 1.f / scale[b] : 0.f;
    const float *a = A + (long long)b * mn;
    ff v = ff_zero();
    const long long stride = (long long)kFroBlocks * blockDim.x;
    if (kVec) {
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const long long n4 = mn >> 2;
        for (long long i = (long long)blk * blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                x[u] = i + u * stride < n4 ? a4[i + u * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float e0 = x[u].x * sc, e1 = x[u].y * sc, e2 = x[u].z * sc, e3 = x[u].w * sc;
                v = ff_fma(v, e0, e0); v = ff_fma(v, e1, e1); v = ff_fma(v, e2, e2); v = ff_fma(v, e3, e3);
            }
        }
    } else {
        for (long long i = (long long)blk * blockDim.x + threadIdx.x; i < mn; i += stride) {
            const float x = a[i] * sc;
            v = ff_fma(v, x, x);
        }
    }
    const float t = block_sum_ff(v, red);
    if (threadIdx.x == 0) part[(long long)b * kFroBlocks + blk] = t;
}

// One warp per matrix: the kFroBlocks partial sums in a fixed order (lane-strided float-float
// sums, then the warp tree), so the result does not depend on scheduling.
__global__ void fro_reduce_kernel(const float *part, int B, float *fro) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= B) return;
    ff v = ff_zero();
    for (int k = lane; k < kFroBlocks; k += 32) v = ff_add(v, ff{part[(long long)b * kFroBlocks + k], 0.f});
    v = warp_sum(v);
    if (lane == 0) fro[b] = __fadd_rn(v.hi, v.lo);
}

__global__ void features_kernel(const float *acc, const float *fro, int B, int m, int n, int s, float *F) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float inv = 1.f / ((float)n * (float)s);
    const float tiny = 1e-30f;
    float t[4];
    for (int j = 0; j < 4; ++j) {
        float sum = 0.f;
        for (int q = 0; q < kZdotBlocks; ++q) sum += acc[((long long)b * 4 + j) * kZdotBlocks + q];
        t[j] = sum * inv;
    }
    float *f = F + (long long)b * kF;
    for (int j = 0; j < 4; ++j) f[j] = logf(fmaxf(t[j], tiny));
    f[4] = logf(fmaxf(fro[b] / (float)n, tiny));
    f[5] = logf(fmaxf(t[3], tiny) / fmaxf(t[2], tiny));
    f[6] = logf((float)n) / 10.f;
    f[7] = logf((float)m / (float)n);
}

// ------------------------------------------------------------ MLP
// One warp per sample; parameters staged in shared memory (W2 with rows padded to kH + 1
// floats, so that the lanes' reads of one column fall in distinct banks).  Lane l computes
// hidden units l and l + 32 of both layers.
constexpr int kFwdWarps = 4;
__global__ void __launch_bounds__(32 * kFwdWarps) mlp_fwd_kernel(const float *params, const float *F, int nb,
                                                                  float *Y) {
    __shared__ float P[kNP];
    __shared__ float W2s[kH * (kH + 1)];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) P[i] = params[i];
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) W2s[(i / kH) * (kH + 1) + i % kH] = params[kP_W2 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x * kFwdWarps + (threadIdx.x >> 5); t < nb; t += gridDim.x * kFwdWarps) {
        float f[kF];
#pragma unroll
        for (int i = 0; i < kF; ++i) f[i] = F[(long long)t * kF + i];
        float h[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int o = lane + 32 * q;
            float z = P[kP_b1 + o];
#pragma unroll
            for (int i = 0; i < kF; ++i) z += P[kP_W1 + o * kF + i] * f[i];
            h[q] = fmaxf(z, 0.f);
        }
        float z2[2] = {P[kP_b2 + lane], P[kP_b2 + lane + 32]};
#pragma unroll 8
        for (int i = 0; i < kH; ++i) {
            const float hi = __shfl_sync(0xffffffffu, h[i >> 5], i & 31);
            z2[0] += W2s[lane * (kH + 1) + i] * hi;
            z2[1] += W2s[(lane + 32) * (kH + 1) + i] * hi;
        }
        float y = P[kP_W3 + lane] * fmaxf(z2[0], 0.f) + P[kP_W3 + lane + 32] * fmaxf(z2[1], 0.f);
        y = warp_sum(y);
        if (lane == 0) Y[t] = y + P[kP_b3];
    }
}

static unsigned mlp_fwd_blocks(long long nb) {
    return (unsigned)std::min<long long>((nb + kFwdWarps - 1) / kFwdWarps, 65535);
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
    PSVD_TRY(cudaMemsetAsync(w.nonfinite, 0, sizeof(int) * batch, st));
    PSVD_TRY(l1_norms(A, B, M, Nn, w.rowsum, w.colsum, w.nonfinite, st));
    norm_finalize_kernel<<<B, kNormThreads, 0, st>>>(w.rowsum, w.colsum, w.nonfinite, M, Nn, w.scale, w.done, w.status,
                                                     w.fin);
    const bool vec_mn = ((uintptr_t)A & 15) == 0 && ((m * n) & 3) == 0;
    const bool vec_n = ((uintptr_t)A & 15) == 0 && (n & 3) == 0;
    if (vec_mn) fro_part_kernel<true><<<dim3(kFroBlocks, B), 256, 0, st>>>(A, w.scale, (long long)m * n, w.fropart);
    else fro_part_kernel<false><<<dim3(kFroBlocks, B), 256, 0, st>>>(A, w.scale, (long long)m * n, w.fropart);
    fro_reduce_kernel<<<(B + 3) / 4, 128, 0, st>>>(w.fropart, B, w.fro);
    count_launch(3);
    // Y_{j+1} = X0^T (X0 Y_j), Y_0 = Z; f_j = <Z, Y_{j+1}> / (n s)
    probe_transpose_kernel<<<dim3((unsigned)(((long long)Nn * S + 255) / 256), B), 256, 0, st>>>(Z, Nn, S, w.ZT);
    count_launch(1);
    const float *Y = w.ZT;
    for (int j = 0; j < 4; ++j) {
        if (vec_n) {
            xy_vec_kernel<<<dim3((M + kXyRows - 1) / kXyRows, B), 256, 0, st>>>(A, w.scale, Y, M, Nn, S, w.T);
            xty_vec_kernel<<<dim3((Nn / 4 + 127) / 128, B, kXtyChunks), 128, 0, st>>>(A, w.scale, w.T, M, Nn, S,
                                                                                      w.Ypart);
        } else {
            xy_kernel<<<dim3((unsigned)(((long long)M * 32 + 255) / 256), B), 256, 0, st>>>(A, w.scale, Y, M, Nn, S, w.T);
            xty_part_kernel<<<dim3((Nn + 127) / 128, B, kXtyChunks), 128, 0, st>>>(A, w.scale, w.T, M, Nn, S, w.Ypart);
        }
        xty_reduce_kernel<<<dim3((unsigned)(((long long)Nn * S + 255) / 256), B), 256, 0, st>>>(w.Ypart, Nn, S, w.Y);
        zdot_kernel<<<dim3(kZdotBlocks, B), 256, 0, st>>>(w.ZT, w.Y, Nn, S, j, w.acc);
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
    mlp_fwd_kernel<<<mlp_fwd_blocks(nb), 32 * kFwdWarps, 0, static_cast<cudaStream_t>(stream)>>>(params, F, (int)nb, Y);
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
    mlp_fwd_kernel<<<mlp_fwd_blocks(nb), 32 * kFwdWarps, 0, st>>>(params, F, (int)nb, LB);
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
    mlp_fwd_kernel<<<mlp_fwd_blocks(nb), 32 * kFwdWarps, 0, st>>>(params, F, (int)nb, Y);
    mlp_margin_kernel<<<1, 1024, 0, st>>>(Y, target, (int)nb, quantile, margin);
    count_launch(2);
    PSVD_TRY(cudaGetLastError());
    return PSVD_OK;
}
