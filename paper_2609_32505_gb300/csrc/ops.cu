// Operand preparation (scale, transpose, TF32 hi/lo split, BF16 cast) and the
// generic batched TN product entry point.
#include <cstring>

#include "ops.cuh"

namespace psvd {

__global__ void prepare_kernel(const float *__restrict__ src, long long lds, long long bss, int rows, int cols,
                               int trans, float scale, const float *__restrict__ scale_ptr, SplitOut dst,
                               const int *__restrict__ skip) {
    __shared__ float tile[32][33];
    const int b = blockIdx.z;
    if (skip && skip[b]) return;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    float sc = scale;
    if (scale_ptr) {
        const float s = scale_ptr[b];
        sc = s > 0.f ? 1.f / s : 0.f;
    }
    const float *S = src + b * bss;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? S[(long long)r * lds + c] * sc : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int r, c;
        float x;
        if (trans) { r = c0 + i; c = r0 + threadIdx.x; x = tile[threadIdx.x][i]; if (r >= cols || c >= rows) continue; }
        else { r = r0 + i; c = c0 + threadIdx.x; x = tile[i][threadIdx.x]; if (r >= rows || c >= cols) continue; }
        const long long o = b * dst.bstride + (long long)r * dst.ld + c;
        if (dst.hi) {
            if (dst.lo) { float h, l; split_tf32(x, h, l); dst.hi[o] = h; dst.lo[o] = l; }
            else dst.hi[o] = x;
        }
        if (dst.h16) dst.h16[o] = __float2bfloat16_rn(x);
    }
}

cudaError_t prepare_operand(const float *src, long long lds, long long bss, int batch, int rows, int cols,
                            bool trans, float scale, const float *scale_ptr, const SplitOut &dst,
                            cudaStream_t st, const int *skip) {
    if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch), block(32, 8);
    prepare_kernel<<<grid, block, 0, st>>>(src, lds, bss, rows, cols, trans ? 1 : 0, scale, scale_ptr, dst, skip);
    count_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) cuda_fail(e, __FILE__, __LINE__);
    return e;
}

}  // namespace psvd

using namespace psvd;

extern "C" {

size_t psvd_gemm_workspace_bytes(int64_t batch, int64_t M, int64_t N, int64_t K) {
    const long long ld = pad_ld(K);
    return (size_t)(batch * (M + N) * ld) * (2 * sizeof(float) + sizeof(__nv_bfloat16)) + 4096;
}

int psvd_gemm_tn(const float *A, const float *B, float *D, int64_t batch, int64_t M, int64_t N, int64_t K,
                 int precision, void *ws, size_t ws_bytes, void *stream) {
    if (!A || !B || !D || batch <= 0 || M <= 0 || N <= 0 || K <= 0 || precision < 0 || precision > 2)
        return PSVD_ERR_ARG;
    if (int e = check_device()) return e;
    if (ws_bytes < psvd_gemm_workspace_bytes(batch, M, N, K)) return PSVD_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long ld = pad_ld(K);
    Carver cv(ws, ws_bytes);
    float *ahi = cv.take<float>(batch * M * ld), *alo = cv.take<float>(batch * M * ld);
    float *bhi = cv.take<float>(batch * N * ld), *blo = cv.take<float>(batch * N * ld);
    __nv_bfloat16 *a16 = cv.take<__nv_bfloat16>(batch * M * ld), *b16 = cv.take<__nv_bfloat16>(batch * N * ld);
    if (cv.overflow) return PSVD_ERR_WORKSPACE;
    SplitOut da, db;
    da.ld = db.ld = ld;
    da.bstride = M * ld; db.bstride = N * ld;
    if (precision == PREC_BF16) { da.h16 = a16; db.h16 = b16; }
    else { da.hi = ahi; db.hi = bhi; if (precision == PREC_TF32X3) { da.lo = alo; db.lo = blo; } }
    if (prepare_operand(A, K, M * K, (int)batch, (int)M, (int)K, false, 1.f, nullptr, da, st) != cudaSuccess ||
        prepare_operand(B, K, N * K, (int)batch, (int)N, (int)K, false, 1.f, nullptr, db, st) != cudaSuccess)
        return PSVD_ERR_CUDA;
    MatView va16 = view_of16(a16, (int)M, (int)K, ld, M * ld, (int)batch);
    MatView vb16 = view_of16(b16, (int)N, (int)K, ld, N * ld, (int)batch);
    MatView vah = view_of(ahi, (int)M, (int)K, ld, M * ld, (int)batch), val = view_of(alo, (int)M, (int)K, ld, M * ld, (int)batch);
    MatView vbh = view_of(bhi, (int)N, (int)K, ld, N * ld, (int)batch), vbl = view_of(blo, (int)N, (int)K, ld, N * ld, (int)batch);
    GemmShape shp;
    memset(&shp, 0, sizeof(shp));
    shp.M = (int)M; shp.N = (int)N; shp.K = (int)K; shp.prec_uniform = precision;
    EpiStore epi = epi_store_plain(D, N, M * N, (int)M, (int)N);
    cudaError_t e;
    if (precision == PREC_BF16) e = launch_gemm(&va16, &vb16, nullptr, nullptr, nullptr, nullptr, shp, (int)batch, epi, st);
    else if (precision == PREC_TF32) e = launch_gemm(nullptr, nullptr, &vah, nullptr, &vbh, nullptr, shp, (int)batch, epi, st);
    else e = launch_gemm(nullptr, nullptr, &vah, &val, &vbh, &vbl, shp, (int)batch, epi, st);
    return cuda_status(e);
}

}  // extern "C"
