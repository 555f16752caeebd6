// tcgen05 "TN" GEMM for sm_103a:  D[b][i][j] = sum_k A[b][i][k] * B[b][j][k]
// with both operands K-major (row-major with K contiguous) in global memory.
//
// Every product of the method is put in this form by keeping transposed copies
// where needed (X and X^T for the polynomial steps, U^T, V, ... in the backward),
// so one well-tested kernel serves the Gram matrix, the polynomial apply, H, U and
// the backward chain.
//
// Persistent kernel: one CTA per SM walks a static list of output tiles of
// 128 x BN (BN = 256, or 128 when N <= 128), UMMA M = 128, N = BN, cta_group::1.
// 128-wide tiles cost about twice as much per flop as 256-wide ones on GB300 (a fixed
// cost per MMA instruction; measured with one mainloop version, BF16 at 8192^3: 559
// against 1049 TFLOP/s), so they are used only where N <= 128.
// Shared memory holds a 192 KB ring of units (4 x 48 KB at BN = 256, 6 x 32 KB at
// BN = 128), each one TMA'd k-block: an A sub-tile (128 rows x 128 B) and a B sub-tile
// (BN rows x 128 B), both in the canonical 128-byte-swizzled K-major layout:
//   PREC_BF16   : 64 bf16 of K per unit, one unit per k-block
//   PREC_TF32   : 32 fp32 of K per unit, one unit per k-block
//   PREC_TF32X3 : 32 fp32 of K, two units per k-block (hi parts, lo parts);
//                 hi*hi + hi*lo + lo*hi (split-TF32, FP32-accurate products)
// Two accumulators of 128 x 256 FP32 in TMEM (all 512 columns) let the MMA warp
// run the next tile (or the next split-TF32 chunk) while the epilogue drains the
// previous one.  The tensor core accumulates with truncation; split-TF32 tiles are
// therefore flushed into round-to-nearest FP32 registers after every k-block.
// Warp roles: warps 0-7 epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31 and
// the column half w / 4), warp 8 TMA producer, warp 9 MMA issuer.  The precision is
// chosen per tile at run time from the tile's batch entry, which lets the polar
// iteration switch precision matrix by matrix.
#pragma once
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace psvd {

enum Prec : int { PREC_BF16 = 0, PREC_TF32 = 1, PREC_TF32X3 = 2 };

constexpr int kBM = 128;
constexpr int kUnitA = 16384;                  // 128 rows x 128 B
constexpr int kUnitB = 32768;                  // up to 256 rows x 128 B
constexpr int kUnitBytes = kUnitA + kUnitB;    // 48 KB
constexpr int kStages = 4;                     // ring units at BN = 256
constexpr int kRingBytes = kStages * kUnitBytes;
constexpr int kMaxStages = kRingBytes / (kUnitA + 128 * 128);   // ring units at BN = 128 (6)
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = (kEpiWarps + 2) * 32;
constexpr int kStageRow = 17;                  // staging row stride (floats): conflict-free
constexpr int kStageBytes = kEpiWarps * 32 * kStageRow * 4;
constexpr int kGemmSmem = kRingBytes + 1024 /*align*/ + 256 /*barriers*/ + kStageBytes;
static_assert((2 * kMaxStages + 4) * 8 + 4 <= 256, "barrier area");
constexpr int kAccCols = 256;                  // TMEM columns per accumulator
constexpr uint32_t kTmemCols = 512;

struct GemmMaps {
    CUtensorMap a_bf16, b_bf16;  // used by PREC_BF16 tiles
    CUtensorMap a_hi, a_lo;      // fp32 (TF32 uses a_hi only)
    CUtensorMap b_hi, b_lo;
};

struct GemmShape {
    int M, N, K;            // logical sizes
    int tiles_m, tiles_n;   // ceil(M/128), ceil(N/BN)
    int bn;                 // 128 or 256
    int batch;
    int sym;                // 1: only tiles that reach the upper triangle (col >= row); requires A == B
    int ksplit;             // > 1: every tile repeated over ksplit disjoint k-block ranges; the
                            // epilogue of range kc gets batch index b + kc * batch (partial sums)
    int prec_uniform;       // used when prec == nullptr
    const int *prec;        // [batch] per-matrix precision, or nullptr
    const int *skip;        // [batch] nonzero = matrix finished, its tiles are skipped (or nullptr)
    const int *gate;        // nullptr, or a device counter: 0 = nothing left to do, the whole launch
                            // returns at once (written by an earlier kernel on the same stream)
    unsigned *ticket;       // nullptr, or a zeroed counter: the last CTA to finish runs epi.tail()
    unsigned *err;          // device error word
    int prof_as;            // profiling class + 1 for the launch timing (0: by precision)
};

// First tile column of row ti that reaches the upper triangle.
PSVD_DEV int sym_first_col(int ti, int bn) { return (kBM * ti) / bn; }

// Tile t of one matrix -> (ti, tj).
PSVD_DEV void tile_coords(const GemmShape &s, int t, int &ti, int &tj) {
    if (!s.sym) { ti = t / s.tiles_n; tj = t % s.tiles_n; return; }
    int row = 0;
    for (;;) {
        const int cnt = s.tiles_n - sym_first_col(row, s.bn);
        if (t < cnt || row == s.tiles_m - 1) break;
        t -= cnt;
        ++row;
    }
    ti = row;
    tj = sym_first_col(row, s.bn) + t;
}

PSVD_DEV int tiles_per_matrix(const GemmShape &s) {
    if (!s.sym) return s.tiles_m * s.tiles_n;
    int c = 0;
    for (int r = 0; r < s.tiles_m; ++r) c += s.tiles_n - sym_first_col(r, s.bn);
    return c;
}

// k-blocks of a tile and accumulation phases (flush points) per tile.
PSVD_DEV int kblocks(const GemmShape &s, int prec) {
    const int kstep = prec == PREC_BF16 ? 64 : 32;
    return (s.K + kstep - 1) / kstep;
}

// One work item of the persistent tile list: matrix b, k range kc (of ksplit), tile (ti, tj),
// k-blocks [kb0, kb0 + nkb).
struct TileJob { int b, kc, ti, tj, kb0, nkb, prec; };
PSVD_DEV TileJob tile_job(const GemmShape &s, int t, int tpm) {
    TileJob j;
    const int ks = s.ksplit > 1 ? s.ksplit : 1;
    const int per = tpm * ks;
    j.b = t / per;
    const int rem = t % per;
    j.kc = rem / tpm;
    tile_coords(s, rem % tpm, j.ti, j.tj);
    j.prec = s.prec ? s.prec[j.b] : s.prec_uniform;
    const int all = kblocks(s, j.prec);
    const int each = (all + ks - 1) / ks;
    j.kb0 = j.kc * each;
    j.nkb = max(0, min(all, j.kb0 + each) - j.kb0);
    return j;
}

// Epilogues that define a per-element elem(acc, b, r, c, v) and a runtime staged() get
// their values through a per-warp shared-memory transpose, so that each store instruction
// of a warp covers two rows x 16 consecutive columns instead of 32 rows x 1 column.
template <class E, class = void> struct EpiHasElem : std::false_type {};
template <class E> struct EpiHasElem<E, std::void_t<decltype(E::kElem)>> : std::integral_constant<bool, E::kElem> {};
// Staged epilogues that also write a transposed copy define trans(acc, b, r, c0, v[16]):
// it runs on the thread's own row (lanes = consecutive rows, so the transposed stores of a
// warp are coalesced) next to the staged row-major element pass.
template <class E, class = void> struct EpiHasTrans : std::false_type {};
template <class E> struct EpiHasTrans<E, std::void_t<decltype(E::kTrans)>> : std::integral_constant<bool, E::kTrans> {};
// Read-modify-write epilogues define pre(b, r, c) (the value read at (r, c)) and
// elem_pre(acc, b, r, c, v, p): the staged pass issues the 16 reads of a chunk before its
// first store, since stores to the array being read would otherwise order every read
// after the previous element's store (one read in flight per thread).
template <class E, class = void> struct EpiHasPre : std::false_type {};
template <class E> struct EpiHasPre<E, std::void_t<decltype(E::kPre)>> : std::integral_constant<bool, E::kPre> {};
// Epilogues with a tail() run it once per launch, in the last CTA to finish (shp.ticket set),
// after every CTA's epilogue writes and atomics are visible: a per-launch reduction step
// (the polar iteration's per-matrix decision) without a launch of its own.
template <class E, class = void> struct EpiHasTail : std::false_type {};
template <class E> struct EpiHasTail<E, std::void_t<decltype(E::kTail)>> : std::integral_constant<bool, E::kTail> {};

// Consumer side of the operand ring, as seen by the MMA issuer: shared-memory address of
// unit 0, unit size, unit count, barriers, and the position of the next unit with the
// parity of its current fill.
struct MmaRing {
    uint32_t base, unit_bytes, nst;
    uint64_t *full, *empty;
    unsigned *err;
    uint32_t stage, phase;
    PSVD_DEV uint32_t take() {                 // returns the stage, advances the position
        const uint32_t s = stage;
        if (++stage == nst) { stage = 0; phase ^= 1; }
        return s;
    }
};

// Descriptor of the k-th 32-byte K step inside a 128-byte swizzled row: the start address
// field (bits 0-13, in 16-byte units) advances by 2; a unit ends below 228 KB, so the
// field never carries.
PSVD_DEV uint64_t sdesc_step(uint64_t d, int k) { return d + (uint64_t)(2 * k); }

// One BF16 or TF32 tile: all its k-blocks accumulate into `tacc` (one phase).
template <bool kTF32>
PSVD_DEV bool mma_tile(MmaRing &r, int nkb, uint32_t tacc, uint32_t id) {
    for (int kb = 0; kb < nkb; ++kb) {
        const uint32_t par = r.phase;
        const uint32_t s = r.take();
        if (!mbar_wait(&r.full[s], par, r.err)) return false;
        tc_fence_after();
        const uint32_t a0 = r.base + s * r.unit_bytes;
        const uint64_t ad = sdesc_k128(a0), bd = sdesc_k128(a0 + kUnitA);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t en = (kb > 0 || k > 0) ? 1u : 0u;
            if constexpr (kTF32) umma_tf32(tacc, sdesc_step(ad, k), sdesc_step(bd, k), id, en);
            else umma_f16(tacc, sdesc_step(ad, k), sdesc_step(bd, k), id, en);
        }
        umma_commit(&r.empty[s]);
    }
    return true;
}

// One split-TF32 tile: every k-block (hi unit, lo unit) is its own phase in the next
// accumulator, flushed by the epilogue into round-to-nearest FP32 registers.
PSVD_DEV bool mma_tile_x3(MmaRing &r, int nkb, uint32_t tmem, uint64_t *acc_full, uint64_t *acc_empty, uint32_t &q,
                          uint32_t id) {
    for (int kb = 0; kb < nkb; ++kb) {
        const uint32_t buf = q & 1;
        if (q >= 2 && !mbar_wait(&acc_empty[buf], ((q >> 1) - 1) & 1, r.err)) return false;
        const uint32_t tacc = tmem + buf * kAccCols;
        const uint32_t p0 = r.phase;
        const uint32_t s0 = r.take();
        const uint32_t p1 = r.phase;
        const uint32_t s1 = r.take();
        if (!mbar_wait(&r.full[s0], p0, r.err) || !mbar_wait(&r.full[s1], p1, r.err)) return false;
        tc_fence_after();
        const uint32_t a0 = r.base + s0 * r.unit_bytes, a1 = r.base + s1 * r.unit_bytes;
        const uint64_t ahi = sdesc_k128(a0), bhi = sdesc_k128(a0 + kUnitA);
        const uint64_t alo = sdesc_k128(a1), blo = sdesc_k128(a1 + kUnitA);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            umma_tf32(tacc, sdesc_step(alo, k), sdesc_step(bhi, k), id, k != 0);
            umma_tf32(tacc, sdesc_step(ahi, k), sdesc_step(blo, k), id, 1);
            umma_tf32(tacc, sdesc_step(ahi, k), sdesc_step(bhi, k), id, 1);
        }
        umma_commit(&r.empty[s0]);
        umma_commit(&r.empty[s1]);
        umma_commit(&acc_full[buf]);
        ++q;
    }
    return true;
}

template <class Epi>
__global__ void __launch_bounds__(kGemmThreads, 1)
gemm_tn_kernel(const __grid_constant__ GemmMaps maps, const GemmShape shp, Epi epi) {
    // A gated launch with nothing left to do returns before any allocation (uniform: every
    // thread reads the same word, final since the kernel that wrote it has completed).
    if (shp.gate && *shp.gate == 0) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kRingBytes);
    uint64_t *empty = full + kMaxStages;
    uint64_t *acc_full = empty + kMaxStages;   // [2] accumulator phase complete (tcgen05.commit)
    uint64_t *acc_empty = acc_full + 2;        // [2] accumulator drained by the epilogue (8 warps)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    float *stage = reinterpret_cast<float *>(smem + kRingBytes + 256);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bn = shp.bn;
    const uint32_t unit_bytes = (uint32_t)(kUnitA + bn * 128);   // also the ring stride (1024-aligned)
    const uint32_t nst = kRingBytes / unit_bytes;                // 4 or 6
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], kEpiWarps); }
        fence_barrier_init();
        s_abort = 0;
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    if (warp == kEpiWarps && lane == 0) {
        tma_prefetch(&maps.a_hi); tma_prefetch(&maps.b_hi);
        tma_prefetch(&maps.a_bf16); tma_prefetch(&maps.b_bf16);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int tpm = tiles_per_matrix(shp);
    const int total = tpm * (shp.ksplit > 1 ? shp.ksplit : 1) * shp.batch;

    if (warp == kEpiWarps) {
        // ------------------------------------------------------------ TMA producer
        // The ring position (stage) and its parity advance by counting: this thread and the
        // MMA issuer sit on the tensor pipe's critical path, where even an integer division
        // per k-block shows up in the MMA rate.
        if (lane == 0) {
            uint32_t ps = 0, pphase = 0;
            for (int t = blockIdx.x; t < total && !s_abort; t += gridDim.x) {
                const TileJob jb = tile_job(shp, t, tpm);
                const int b = jb.b, prec = jb.prec, nkb = jb.nkb;
                if (shp.skip && shp.skip[b]) continue;
                const int row_a = jb.ti * kBM, row_b = jb.tj * bn;
                const CUtensorMap *ma0 = &maps.a_hi, *mb0 = &maps.b_hi, *ma1 = &maps.a_lo, *mb1 = &maps.b_lo;
                if (prec == PREC_BF16) { ma0 = &maps.a_bf16; mb0 = &maps.b_bf16; }
                const int kstep = prec == PREC_BF16 ? 64 : 32;
                const int nu = prec == PREC_TF32X3 ? 2 : 1;
                for (int kb = 0; kb < nkb; ++kb) {
                    const int k0 = (jb.kb0 + kb) * kstep;
                    for (int h = 0; h < nu; ++h) {
                        if (!mbar_wait(&empty[ps], pphase ^ 1, shp.err)) { s_abort = 1; break; }
                        uint8_t *st = smem + ps * unit_bytes;
                        mbar_arrive_expect_tx(&full[ps], unit_bytes);
                        tma_load_3d(st, h ? ma1 : ma0, &full[ps], k0, row_a, b);
                        tma_load_3d(st + kUnitA, h ? mb1 : mb0, &full[ps], k0, row_b, b);
                        if (++ps == nst) { ps = 0; pphase ^= 1; }
                    }
                    if (s_abort) break;
                }
            }
        }
    } else if (warp == kEpiWarps + 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_tf32 = idesc_f32acc(kFmtTF32, kBM, bn);
            const uint32_t id_bf16 = idesc_f32acc(kFmtBF16, kBM, bn);
            MmaRing ring{smem_u32(smem), unit_bytes, nst, full, empty, shp.err, 0u, 0u};
            uint32_t q = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const TileJob jb = tile_job(shp, t, tpm);
                if ((shp.skip && shp.skip[jb.b]) || jb.nkb <= 0) continue;
                if (jb.prec == PREC_TF32X3) {
                    ok = mma_tile_x3(ring, jb.nkb, tmem, acc_full, acc_empty, q, id_tf32);
                } else {
                    const uint32_t buf = q & 1;
                    if (q >= 2 && !mbar_wait(&acc_empty[buf], ((q >> 1) - 1) & 1, shp.err)) { ok = false; break; }
                    const uint32_t tacc = tmem + buf * kAccCols;
                    ok = jb.prec == PREC_TF32 ? mma_tile<true>(ring, jb.nkb, tacc, id_tf32)
                                              : mma_tile<false>(ring, jb.nkb, tacc, id_bf16);
                    if (!ok) break;
                    umma_commit(&acc_full[buf]);
                    ++q;
                }
            }
            if (!ok) {
                s_abort = 1;
                mbar_arrive(&acc_full[0]);          // release the epilogue
                mbar_arrive(&acc_full[1]);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // thread owns output row ti*128 + 32 (warp % 4) + lane and BN/2 columns
        // starting at (warp / 4) * BN/2, kept in round-to-nearest FP32 registers
        const int quad = warp & 3, half = warp >> 2;
        const int ncols = bn >> 1;
        const uint32_t lane_base = uint32_t(quad * 32) << 16;
        uint32_t q = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
            const TileJob jb = tile_job(shp, t, tpm);
            const int b = jb.b, prec = jb.prec, nkb = jb.nkb, ti = jb.ti, tj = jb.tj;
            if (shp.skip && shp.skip[b]) continue;
            const int be = b + jb.kc * shp.batch;     // epilogue's batch index (partial-sum slice)
            const int nph = nkb == 0 ? 0 : (prec == PREC_TF32X3 ? nkb : 1);
            float acc[128];
#pragma unroll
            for (int c = 0; c < 128; ++c) acc[c] = 0.f;
            bool ok = true;
            for (int ph = 0; ph < nph; ++ph, ++q) {
                const uint32_t buf = q & 1;
                ok = mbar_wait(&acc_full[buf], (q >> 1) & 1, shp.err) && !s_abort;
                tc_fence_after();
                if (ok) {
                    const uint32_t tb = tmem + lane_base + buf * kAccCols + half * ncols;
#pragma unroll
                    for (int c = 0; c < 128; c += 16) {
                        if (c < ncols) {
                            float v[16];
                            tmem_ld16(tb + c, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) acc[c + i] += v[i];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
                if (!ok) break;
            }
            if (!ok) break;
            const int r = ti * kBM + quad * 32 + lane;
            const int cbase = tj * bn + half * ncols;
            typename Epi::Acc ea;
            epi.begin(ea);
            bool staged = false;
            if constexpr (EpiHasElem<Epi>::value) staged = epi.staged();
            if (staged) {
                if constexpr (EpiHasElem<Epi>::value) {
                    float *sw = stage + warp * 32 * kStageRow;
                    const int r0 = ti * kBM + quad * 32, rr0 = lane >> 4, cc = lane & 15;
#pragma unroll
                    for (int c = 0; c < 128; c += 16) {
                        if (c < ncols) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) sw[lane * kStageRow + i] = acc[c + i];
                            __syncwarp();
                            if constexpr (EpiHasPre<Epi>::value) {
                                float pv[16];
#pragma unroll
                                for (int k = 0; k < 16; ++k) pv[k] = epi.pre(be, r0 + 2 * k + rr0, cbase + c + cc);
#pragma unroll
                                for (int k = 0; k < 16; ++k) {
                                    const int rr = 2 * k + rr0;
                                    epi.elem_pre(ea, be, r0 + rr, cbase + c + cc, sw[rr * kStageRow + cc], pv[k]);
                                }
                            } else {
#pragma unroll 4
                                for (int k = 0; k < 16; ++k) {
                                    const int rr = 2 * k + rr0;
                                    epi.elem(ea, be, r0 + rr, cbase + c + cc, sw[rr * kStageRow + cc]);
                                }
                            }
                            __syncwarp();
                            if constexpr (EpiHasTrans<Epi>::value) {
                                float v[16];
#pragma unroll
                                for (int i = 0; i < 16; ++i) v[i] = acc[c + i];
                                epi.trans(ea, be, r, cbase + c, v);
                            }
                        }
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 128; c += 16) {
                    if (c < ncols) {
                        float v[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = acc[c + i];
                        epi.chunk(ea, be, r, cbase + c, ti, tj, v);
                    }
                }
            }
            epi.finish(ea, be, ti, tj);
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if constexpr (EpiHasTail<Epi>::value) {
        if (shp.ticket) {
            __shared__ int s_last;
            if (threadIdx.x == 0) {
                __threadfence();                                  // this CTA's writes before its ticket
                s_last = atomicAdd(shp.ticket, 1u) == gridDim.x - 1;
                if (s_last) __threadfence();                      // every other CTA's, before the tail
            }
            __syncthreads();
            if (s_last) epi.tail();
        }
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

// Encodes a TMA descriptor: box = box_rows rows x 128 B (32 fp32 / 64 bf16), 128-byte
// swizzle, zero fill outside [cols] x [rows].  Returns false if the driver rejects it.
bool make_tmap(CUtensorMap *out, const MatView &v, int box_rows = 128);

void count_launch(int n = 1);
int cuda_fail(cudaError_t e, const char *file, int line);
int num_sms();

// Optional per-launch timing of the product kernel (CUDA events on the launching
// stream); `flops` is the algorithmic count of the launch, `prec` its class.
void prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st, double flops, int prec);
bool prof_on();

// Host copy of the tile count (same enumeration as the device).
inline int host_tiles_per_matrix(const GemmShape &s) {
    if (!s.sym) return s.tiles_m * s.tiles_n;
    int c = 0;
    for (int r = 0; r < s.tiles_m; ++r) c += s.tiles_n - (kBM * r) / s.bn;
    return c;
}

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
    shp.bn = shp.N > 128 ? 256 : 128;
    if (shp.bn == 256) {
        // A launch with fewer 256-wide tiles than half the SMs is bound by one tile's serial
        // k-loop (and, for split-TF32, its per-k-block flushes): 128-wide tiles put twice
        // as many CTAs to work on it.
        GemmShape t = shp;
        t.tiles_m = (t.M + kBM - 1) / kBM;
        t.tiles_n = (t.N + 255) / 256;
        const long long tiles = (long long)host_tiles_per_matrix(t) * (shp.ksplit > 1 ? shp.ksplit : 1) * batch;
        if (2 * tiles <= num_sms()) shp.bn = 128;
    }
    GemmMaps maps;
    memset(&maps, 0, sizeof(maps));
    // Any map that is not supplied aliases a supplied one of the same role; the
    // kernel only dereferences the maps of the precision a tile runs.
    const MatView *Ap = ahi ? ahi : (alo ? alo : a16), *Bp = bhi ? bhi : (blo ? blo : b16);
    if (!Ap || !Bp) {
        cuda_fail(cudaErrorInvalidValue, "launch_gemm: missing operand", __LINE__);
        return cudaErrorInvalidValue;
    }
    if (!make_tmap(&maps.a_hi, ahi ? *ahi : *Ap) || !make_tmap(&maps.a_lo, alo ? *alo : *Ap) ||
        !make_tmap(&maps.a_bf16, a16 ? *a16 : *Ap) || !make_tmap(&maps.b_hi, bhi ? *bhi : *Bp, shp.bn) ||
        !make_tmap(&maps.b_lo, blo ? *blo : *Bp, shp.bn) || !make_tmap(&maps.b_bf16, b16 ? *b16 : *Bp, shp.bn)) {
        cuda_fail(cudaErrorInvalidValue, "tensor map encode", __LINE__);
        return cudaErrorInvalidValue;
    }
    shp.tiles_m = (shp.M + kBM - 1) / kBM;
    shp.tiles_n = (shp.N + shp.bn - 1) / shp.bn;
    shp.batch = batch;
    if (shp.tiles_m == 0 || shp.tiles_n == 0 || batch == 0) return cudaSuccess;
    const long long total = (long long)host_tiles_per_matrix(shp) * (shp.ksplit > 1 ? shp.ksplit : 1) * batch;
    const int grid = (int)std::min<long long>(total, num_sms());
    const bool prof = prof_on();
    if (prof) prof_begin(st);
    gemm_tn_kernel<Epi><<<grid, kGemmThreads, kGemmSmem, st>>>(maps, shp, epi);
    count_launch();
    if (prof) {
        // algorithmic flops: 2 M N K per matrix (M (M + 1) K for the symmetric Gram)
        const double f = shp.sym ? (double)shp.M * (shp.M + 1) * shp.K : 2.0 * shp.M * shp.N * (double)shp.K;
        prof_end(st, f * batch, shp.prof_as > 0 ? shp.prof_as - 1 : (shp.prec ? -1 : shp.prec_uniform));
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) cuda_fail(le, __FILE__, __LINE__);
    return le;
}

}  // namespace psvd
