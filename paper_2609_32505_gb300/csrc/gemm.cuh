// tcgen05 "TN" GEMM for sm_103a:  D[b][i][j] = sum_k A[b][i][k] * B[b][j][k]
// with both operands K-major (row-major with K contiguous) in global memory.
//
// Every product of the method is put in this form by keeping transposed copies
// where needed (X and X^T for the polynomial steps, U^T, V, ... in the backward),
// so one well-tested kernel serves the Gram matrix, the polynomial apply, H, U and
// the backward chain.
//
// Tile 128 x 128 (UMMA M = 128, N = 128, cta_group::1), accumulator in 128 TMEM
// columns.  Each pipeline stage holds four 16 KB sub-tiles of 128 rows x 128 B,
// each in the canonical 128-byte-swizzled K-major layout written by TMA:
//   PREC_TF32X3 : A_hi, A_lo, B_hi, B_lo over 32 fp32 of K;   3 MMAs per k-step
//                 (hi*hi + hi*lo + lo*hi: split-TF32, FP32-accurate products)
//   PREC_TF32   : A[k0:32], A[k32:64], B[k0:32], B[k32:64];   1 MMA per k-step
//   PREC_BF16   : A[k0:64], A[k64:128], B[k0:64], B[k64:128]; 1 MMA per k-step
// Warp roles: warps 0-3 epilogue (TMEM lanes 32w..32w+31), warp 4 TMA producer,
// warp 5 MMA issuer.  The precision is chosen per CTA at run time (per batch
// entry), which lets the polar iteration switch precision matrix by matrix.
#pragma once
#include "common.cuh"

namespace psvd {

enum Prec : int { PREC_BF16 = 0, PREC_TF32 = 1, PREC_TF32X3 = 2 };

constexpr int kBM = 128, kBN = 128;
constexpr int kSub = 16384;             // one 128 x 128 B sub-tile
constexpr int kStageBytes = 4 * kSub;   // 64 KB
constexpr int kStages = 3;
constexpr int kGemmThreads = 192;
constexpr int kGemmSmem = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kFlushKB = 2;           // split-TF32: flush the accumulator every 2 k-blocks (K = 64)
constexpr uint32_t kTmemCols = 512;    // 2 x 128 double-buffered accumulator + 128 cross terms

struct GemmMaps {
    CUtensorMap a_bf16, b_bf16;  // used when a CTA runs in PREC_BF16
    CUtensorMap a_hi, a_lo;      // fp32 (TF32 uses a_hi only)
    CUtensorMap b_hi, b_lo;
};

struct GemmShape {
    int M, N, K;            // logical sizes
    int tiles_m, tiles_n;   // ceil(M/128), ceil(N/128)
    int sym;                // 1: upper-triangle tiles only (i <= j); requires A == B
    int prec_uniform;       // used when prec == nullptr
    const int *prec;        // [batch] per-matrix precision, or nullptr
    const int *skip;        // [batch] nonzero = matrix finished, CTA returns at once (or nullptr)
    unsigned *err;          // device error word
};

PSVD_DEV void sym_tile(int t, int T, int &i, int &j) {
    // enumerate (i, j) with i <= j row by row
    int row = 0, base = 0;
    while (row < T && t >= base + (T - row)) { base += T - row; ++row; }
    i = row;
    j = row + (t - base);
}

template <class Epi>
__global__ void __launch_bounds__(kGemmThreads, 1)
gemm_tn_kernel(const __grid_constant__ GemmMaps maps, const GemmShape shp, Epi epi) {
    const int b = blockIdx.z;
    if (shp.skip && shp.skip[b]) return;           // uniform across the CTA
    int ti, tj;
    if (shp.sym) sym_tile(blockIdx.x, shp.tiles_m, ti, tj);
    else { ti = blockIdx.y; tj = blockIdx.x; }
    const int prec = shp.prec ? shp.prec[b] : shp.prec_uniform;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;      // [2] accumulator chunk complete (tcgen05.commit)
    uint64_t *acc_empty = acc_full + 2;        // [2] accumulator chunk drained by the epilogue (4 warps)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 4); }
        fence_barrier_init();
        s_abort = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    if (warp == 4 && lane == 0) {
        tma_prefetch(prec == PREC_BF16 ? &maps.a_bf16 : &maps.a_hi);
        tma_prefetch(prec == PREC_BF16 ? &maps.b_bf16 : &maps.b_hi);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int kstep = prec == PREC_BF16 ? 128 : (prec == PREC_TF32 ? 64 : 32);
    const int nkb = (shp.K + kstep - 1) / kstep;
    // Split-TF32 flushes the (truncating) tensor-core accumulator into FP32
    // registers every kFlushKB k-blocks; single-pass precisions use one chunk.
    const int F = prec == PREC_TF32X3 ? kFlushKB : (nkb > 0 ? nkb : 1);
    const int nq = (nkb + F - 1) / F;
    const int row_a = ti * kBM, row_b = tj * kBN;

    if (warp == 4) {
        if (lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % kStages;
                if (!mbar_wait(&empty[s], ((kb / kStages) & 1) ^ 1, shp.err)) { s_abort = 1; break; }
                uint8_t *st = smem + s * kStageBytes;
                mbar_arrive_expect_tx(&full[s], kStageBytes);
                const int k0 = kb * kstep;
                if (prec == PREC_TF32X3) {
                    tma_load_3d(st + 0 * kSub, &maps.a_hi, &full[s], k0, row_a, b);
                    tma_load_3d(st + 1 * kSub, &maps.a_lo, &full[s], k0, row_a, b);
                    tma_load_3d(st + 2 * kSub, &maps.b_hi, &full[s], k0, row_b, b);
                    tma_load_3d(st + 3 * kSub, &maps.b_lo, &full[s], k0, row_b, b);
                } else if (prec == PREC_TF32) {
                    tma_load_3d(st + 0 * kSub, &maps.a_hi, &full[s], k0, row_a, b);
                    tma_load_3d(st + 1 * kSub, &maps.a_hi, &full[s], k0 + 32, row_a, b);
                    tma_load_3d(st + 2 * kSub, &maps.b_hi, &full[s], k0, row_b, b);
                    tma_load_3d(st + 3 * kSub, &maps.b_hi, &full[s], k0 + 32, row_b, b);
                } else {
                    tma_load_3d(st + 0 * kSub, &maps.a_bf16, &full[s], k0, row_a, b);
                    tma_load_3d(st + 1 * kSub, &maps.a_bf16, &full[s], k0 + 64, row_a, b);
                    tma_load_3d(st + 2 * kSub, &maps.b_bf16, &full[s], k0, row_b, b);
                    tma_load_3d(st + 3 * kSub, &maps.b_bf16, &full[s], k0 + 64, row_b, b);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t id_tf32 = idesc_f32acc(kFmtTF32, kBM, kBN);
            const uint32_t id_bf16 = idesc_f32acc(kFmtBF16, kBM, kBN);
            const uint32_t t_small = tmem + 2 * kBN;     // split-TF32 cross terms
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                const int q = kb / F, buf = q & 1;
                const bool chunk_start = (kb % F) == 0;
                if (chunk_start && q >= 2 && !mbar_wait(&acc_empty[buf], ((q >> 1) - 1) & 1, shp.err)) {
                    ok = false; s_abort = 1; break;
                }
                const uint32_t t_big = tmem + buf * kBN;
                const int s = kb % kStages;
                if (!mbar_wait(&full[s], (kb / kStages) & 1, shp.err)) { ok = false; s_abort = 1; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * kStageBytes);
                if (prec == PREC_TF32X3) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t ahi = sdesc_k128(sa + 0 * kSub + 32 * k);
                        const uint64_t alo = sdesc_k128(sa + 1 * kSub + 32 * k);
                        const uint64_t bhi = sdesc_k128(sa + 2 * kSub + 32 * k);
                        const uint64_t blo = sdesc_k128(sa + 3 * kSub + 32 * k);
                        umma_tf32(t_small, alo, bhi, id_tf32, (kb | k) != 0);
                        umma_tf32(t_small, ahi, blo, id_tf32, 1);
                        umma_tf32(t_big, ahi, bhi, id_tf32, (!chunk_start) || k != 0);
                    }
                } else {
                    const uint32_t id = prec == PREC_TF32 ? id_tf32 : id_bf16;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint64_t ad = sdesc_k128(sa + h * kSub + 32 * k);
                            const uint64_t bd = sdesc_k128(sa + (2 + h) * kSub + 32 * k);
                            const uint32_t en = (!chunk_start) || h != 0 || k != 0;
                            if (prec == PREC_TF32) umma_tf32(t_big, ad, bd, id, en);
                            else umma_f16(t_big, ad, bd, id, en);
                        }
                    }
                }
                umma_commit(&empty[s]);                    // frees the stage once these MMAs complete
                if ((kb % F) == F - 1 || kb == nkb - 1) umma_commit(&acc_full[buf]);
            }
            if (!ok) { mbar_arrive(&acc_full[0]); mbar_arrive(&acc_full[1]); }   // release the epilogue
        }
    } else {
        // epilogue: warps 0-3; thread owns output row ti*128 + threadIdx.x and keeps the
        // 128-column accumulator in FP32 registers (round-to-nearest adds)
        float acc[kBN];
#pragma unroll
        for (int c = 0; c < kBN; ++c) acc[c] = 0.f;
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
        bool ok = true;
        for (int q = 0; q < nq && ok; ++q) {
            const int buf = q & 1;
            ok = mbar_wait(&acc_full[buf], (q >> 1) & 1, shp.err) && !s_abort;
            tc_fence_after();
            if (ok) {
#pragma unroll
                for (int c = 0; c < kBN; c += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + uint32_t(buf * kBN + c), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c + i] += v[i];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        if (ok && prec == PREC_TF32X3 && nkb > 0) {
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < kBN; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + uint32_t(2 * kBN + c), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c + i] += v[i];
            }
        }
        if (ok) {
            const int r = row_a + threadIdx.x;
            typename Epi::Acc ea;
            epi.begin(ea);
#pragma unroll
            for (int c = 0; c < kBN; c += 16) {
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = acc[c + i];
                epi.chunk(ea, b, r, row_b + c, ti, tj, v);
            }
            epi.finish(ea, b, ti, tj);
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------- host side
// A 3-D view of a batch of row-major matrices with a padded leading dimension.
struct MatView {
    const void *ptr = nullptr;
    int rows = 0, cols = 0;     // logical
    long long ld = 0;           // elements between rows
    long long bstride = 0;      // elements between batch entries
    int batch = 1;
    bool bf16 = false;
};

// Encodes a TMA descriptor: box = 128 rows x 128 B (32 fp32 / 64 bf16), 128-byte
// swizzle, zero fill outside [cols] x [rows].  Returns false if the driver rejects it.
bool make_tmap(CUtensorMap *out, const MatView &v);

void count_launch(int n = 1);
int cuda_fail(cudaError_t e, const char *file, int line);

// Optional per-launch timing of the product kernel (CUDA events on the launching
// stream); `flops` is the algorithmic count of the launch, `prec` its class.
void prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st, double flops, int prec);
bool prof_on();


template <class Epi>
cudaError_t launch_gemm(const MatView *a16, const MatView *b16, const MatView *ahi, const MatView *alo,
                        const MatView *bhi, const MatView *blo, GemmShape shp, int batch, const Epi &epi,
                        cudaStream_t st) {
    // Set on every launch, through the same kernel handle the launch below uses: each
    // .cu file that instantiates this template registers its own copy of the kernel, so
    // a process-wide "already configured" flag would leave other copies unconfigured.
    {
        cudaError_t e = cudaFuncSetAttribute(gemm_tn_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kGemmSmem);
        if (e != cudaSuccess) { cuda_fail(e, __FILE__, __LINE__); return e; }
    }
    GemmMaps maps;
    memset(&maps, 0, sizeof(maps));
    // Any map that is not supplied aliases a supplied one of the same role; the
    // kernel only dereferences the maps of the precision it runs.
    const MatView *A32 = ahi ? ahi : alo, *B32 = bhi ? bhi : blo;
    if ((a16 && !make_tmap(&maps.a_bf16, *a16)) || (b16 && !make_tmap(&maps.b_bf16, *b16)) ||
        (A32 && !make_tmap(&maps.a_hi, *A32)) || (alo && !make_tmap(&maps.a_lo, *alo)) ||
        (B32 && !make_tmap(&maps.b_hi, *B32)) || (blo && !make_tmap(&maps.b_lo, *blo))) {
        cuda_fail(cudaErrorInvalidValue, "tensor map encode", __LINE__);
        return cudaErrorInvalidValue;
    }
    shp.tiles_m = (shp.M + kBM - 1) / kBM;
    shp.tiles_n = (shp.N + kBN - 1) / kBN;
    dim3 grid;
    if (shp.sym) grid = dim3(shp.tiles_m * (shp.tiles_m + 1) / 2, 1, batch);
    else grid = dim3(shp.tiles_n, shp.tiles_m, batch);
    if (grid.x == 0 || grid.y == 0 || batch == 0) return cudaSuccess;
    const bool prof = prof_on();
    if (prof) prof_begin(st);
    gemm_tn_kernel<Epi><<<grid, kGemmThreads, kGemmSmem, st>>>(maps, shp, epi);
    count_launch();
    if (prof) {
        // algorithmic flops: 2 M N K per matrix (M (M + 1) K for the symmetric Gram)
        const double f = shp.sym ? (double)shp.M * (shp.M + 1) * shp.K : 2.0 * shp.M * shp.N * (double)shp.K;
        prof_end(st, f * batch, shp.prec ? -1 : shp.prec_uniform);
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) cuda_fail(le, __FILE__, __LINE__);
    return le;
}

}  // namespace psvd
