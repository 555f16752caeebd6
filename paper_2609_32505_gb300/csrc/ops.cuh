// Operand preparation kernels and the generic store epilogue, shared by the
// polar, SVD and backward drivers.
#pragma once
#include "gemm.cuh"
#include "runtime.h"

namespace psvd {

// Internal buffers keep rows padded to a multiple of 32 elements (128 B of fp32)
// so that every TMA row stride is 16-byte aligned.
inline long long pad_ld(long long cols) { return round_up(cols < 1 ? 1 : cols, 32); }

// The column L1 norms of the normalization (Algorithm 2) are summed in slabs of kL1Rows
// rows; the buffer of column sums holds batch x l1_slabs(m) x n partial sums.
constexpr int kL1Rows = 256;
constexpr int kNormThreads = 1024;   // threads of the block that finishes the norms of one matrix
__host__ __device__ inline int l1_slabs(int m) { return m < 1 ? 1 : (m + kL1Rows - 1) / kL1Rows; }

// Output format of an operand-preparation pass.
struct SplitOut {
    float *hi = nullptr, *lo = nullptr;   // fp32 split (lo may be null: TF32 rounding only)
    __nv_bfloat16 *h16 = nullptr;         // bf16 copy
    long long ld = 0, bstride = 0;
};

// src (batch x rows x cols, leading dim lds, batch stride bss) scaled by `scale`
// (or by 1/scale_ptr[b] when scale_ptr != nullptr) -> dst in its padded layout,
// transposed when `trans` (dst is then cols x rows).
cudaError_t prepare_operand(const float *src, long long lds, long long bss, int batch, int rows, int cols,
                            bool trans, float scale, const float *scale_ptr, const SplitOut &dst,
                            cudaStream_t st, const int *skip = nullptr);

// MatViews of a SplitOut for TMA.
inline MatView view_of(const float *p, int rows, int cols, long long ld, long long bs, int batch) {
    MatView v; v.ptr = p; v.rows = rows; v.cols = cols; v.ld = ld; v.bstride = bs; v.batch = batch; v.bf16 = false;
    return v;
}
inline MatView view_of16(const __nv_bfloat16 *p, int rows, int cols, long long ld, long long bs, int batch) {
    MatView v; v.ptr = p; v.rows = rows; v.cols = cols; v.ld = ld; v.bstride = bs; v.batch = batch; v.bf16 = true;
    return v;
}

// Generic epilogue: D = alpha * acc (+ beta * C) stored row-major, transposed,
// and/or split into TF32 hi/lo halves (row-major or transposed).
struct EpiStore {
    int rows, cols;
    float alpha;
    const float *cin; long long ldc, bsc; float beta;      // optional addend
    float *out; long long ld, bs;                          // optional plain store
    float *out_t; long long ldt, bst;                      // optional transposed store
    float *hi, *lo; long long ldh, bsh;                    // optional split store
    float *hi_t, *lo_t; long long ldht, bsht;              // optional split transposed store
    struct Acc {};
    static constexpr bool kElem = true;
    // staged (coalesced) element path when nothing is stored transposed
    PSVD_DEV bool staged() const { return !out_t && !hi_t; }
    PSVD_DEV void elem(Acc &, int b, int r, int c, float v) const {
        if (r >= rows || c >= cols) return;
        float x = alpha * v;
        if (cin) x += beta * cin[b * bsc + (long long)r * ldc + c];
        if (out) out[b * bs + (long long)r * ld + c] = x;
        if (hi) {
            float h, l;
            split_tf32(x, h, l);
            hi[b * bsh + (long long)r * ldh + c] = h;
            if (lo) lo[b * bsh + (long long)r * ldh + c] = l;
        }
    }
    PSVD_DEV void begin(Acc &) const {}
    PSVD_DEV void chunk(Acc &, int b, int r, int c0, int, int, float (&v)[16]) const {
        if (r >= rows) return;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = c0 + i;
            if (c >= cols) break;
            float x = alpha * v[i];
            if (cin) x += beta * cin[b * bsc + (long long)r * ldc + c];
            if (out) out[b * bs + (long long)r * ld + c] = x;
            if (out_t) out_t[b * bst + (long long)c * ldt + r] = x;
            if (hi || hi_t) {
                float h, l;
                split_tf32(x, h, l);
                if (hi) { hi[b * bsh + (long long)r * ldh + c] = h; if (lo) lo[b * bsh + (long long)r * ldh + c] = l; }
                if (hi_t) { hi_t[b * bsht + (long long)c * ldht + r] = h; if (lo_t) lo_t[b * bsht + (long long)c * ldht + r] = l; }
            }
        }
    }
    PSVD_DEV void finish(Acc &, int, int, int) const {}
};

// In place: X[r][c] -= acc for a matrix kept split in TF32 hi/lo halves (the eigensolver's
// back-transform, the QR's trailing updates); the reads of a chunk are issued before its
// stores (pre / elem_pre).
struct EpiSubSplit {
    int rows, cols;
    float *hi, *lo;
    long long ld, bs;
    struct Acc {};
    static constexpr bool kElem = true, kPre = true;
    PSVD_DEV bool staged() const { return true; }
    // Read through the read-only path: every element is read once, before this thread
    // writes it, and no other thread touches it, so a stale cached copy can only be of an
    // element already read; the reads of the next chunk may then be issued ahead of this
    // chunk's stores.
    PSVD_DEV float pre(int b, int r, int c) const {
        if (r >= rows || c >= cols) return 0.f;
        const long long o = b * bs + (long long)r * ld + c;
        return __ldg(hi + o) + __ldg(lo + o);
    }
    PSVD_DEV void elem_pre(Acc &, int b, int r, int c, float v, float p) const {
        if (r >= rows || c >= cols) return;
        const long long o = b * bs + (long long)r * ld + c;
        float h, l;
        split_tf32(p - v, h, l);
        hi[o] = h;
        lo[o] = l;
    }
    PSVD_DEV void elem(Acc &a, int b, int r, int c, float v) const { elem_pre(a, b, r, c, v, pre(b, r, c)); }
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

inline EpiStore epi_store_plain(float *out, long long ld, long long bs, int rows, int cols) {
    EpiStore e;
    memset(&e, 0, sizeof(e));
    e.rows = rows; e.cols = cols; e.alpha = 1.f;
    e.out = out; e.ld = ld; e.bs = bs;
    return e;
}

}  // namespace psvd
