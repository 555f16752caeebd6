// Polar factor by polynomial iteration (the polar-factor part of Algorithm 1), shared by
// psvd_polar_fwd and psvd_svd_fwd.
#pragma once
#include "ops.cuh"

namespace psvd {

#ifndef PSVD_TAU_BF16
#define PSVD_TAU_BF16 5e-2
#endif
#ifndef PSVD_TAU_TF32
#define PSVD_TAU_TF32 2e-3
#endif
constexpr double kTauBF16 = PSVD_TAU_BF16;   // mixed path: leave BF16 once the residual is below this
constexpr double kTauTF32 = PSVD_TAU_TF32;   // ... and TF32 once below this (3xTF32 polish afterwards)

struct PolarWS {
    int B = 0, m = 0, n = 0, kcap = 0;
    bool mixed = false;     // precision switched per matrix and step (PSVD_PREC_MIXED*)
    bool bf16 = false;      // BF16 early steps and their operand copies (PSVD_PREC_MIXED_BF16)
    long long ldn = 0, ldm = 0;
    // iterate buffers, double-buffered by step parity
    __nv_bfloat16 *X16[2] = {}, *XT16[2] = {};
    float *Xhi[2] = {}, *Xlo[2] = {}, *XThi[2] = {}, *XTlo[2] = {};
    __nv_bfloat16 *P16 = nullptr;
    float *Phi = nullptr, *Plo = nullptr;
    float *AThi = nullptr, *ATlo = nullptr;     // M^T split (for H = W^T M)
    float *Hraw = nullptr;                      // W^T M before symmetrization
    float *Hsym = nullptr;                      // (W^T M)_sym, FP32 copy
    float *rowsum = nullptr, *colsum = nullptr, *scale = nullptr;
    // per-matrix state
    int *done = nullptr, *fin = nullptr, *status = nullptr, *prec = nullptr, *steps = nullptr;
    int *budget = nullptr, *fallback = nullptr, *notdone = nullptr, *nonfinite = nullptr;
    double *res = nullptr;
    float *coef = nullptr, *fres = nullptr;
    int *misc = nullptr;
    unsigned *ticket = nullptr;   // [kcap + 2] per-step CTA tickets of the Gram launches
    unsigned *err = nullptr;

    template <class C>
    void carve(C &cv, int B_, int m_, int n_, int kcap_, int precision) {
        B = B_; m = m_; n = n_; kcap = kcap_;
        mixed = precision != PSVD_PREC_FP32;
        bf16 = precision == PSVD_PREC_MIXED_BF16;
        ldn = pad_ld(n); ldm = pad_ld(m);
        const long long B64 = B;
        for (int p = 0; p < 2; ++p) {
            if (bf16) {
                X16[p] = cv.template take<__nv_bfloat16>(B64 * m * ldn);
                XT16[p] = cv.template take<__nv_bfloat16>(B64 * n * ldm);
            }
            Xhi[p] = cv.template take<float>(B64 * m * ldn);
            Xlo[p] = cv.template take<float>(B64 * m * ldn);
            XThi[p] = cv.template take<float>(B64 * n * ldm);
            XTlo[p] = cv.template take<float>(B64 * n * ldm);
        }
        if (bf16) P16 = cv.template take<__nv_bfloat16>(B64 * n * ldn);
        Phi = cv.template take<float>(B64 * n * ldn);
        Plo = cv.template take<float>(B64 * n * ldn);
        AThi = cv.template take<float>(B64 * n * ldm);
        ATlo = cv.template take<float>(B64 * n * ldm);
        Hraw = cv.template take<float>(B64 * n * n);
        Hsym = cv.template take<float>(B64 * n * n);
        rowsum = cv.template take<float>(B64 * m);
        colsum = cv.template take<float>(B64 * l1_slabs(m) * n);
        scale = cv.template take<float>(B64);
        done = cv.template take<int>(B64);
        fin = cv.template take<int>(B64);
        status = cv.template take<int>(B64);
        prec = cv.template take<int>((long long)(kcap + 2) * B64);
        steps = cv.template take<int>(3 * B64);
        budget = cv.template take<int>(B64);
        fallback = cv.template take<int>(B64);
        notdone = cv.template take<int>(kcap + 2);
        nonfinite = cv.template take<int>(B64);
        res = cv.template take<double>((long long)(kcap + 2) * B64);
        coef = cv.template take<float>((long long)(kcap + 1) * B64 * 2);
        fres = cv.template take<float>(B64);
        misc = cv.template take<int>(8);
        ticket = cv.template take<unsigned>(kcap + 2);
        err = cv.template take<unsigned>(4);
    }
};

inline int polar_kcap(const psvd_opts &o) { return o.max_iter + (o.schedule == PSVD_SCHED_CANS ? o.pre_iters : 0); }

// Runs the iteration of Algorithm 1 (normalize, schedule, iterate) for all matrices, then
// writes W (user layout, may be null) and leaves W^T split in XThi[0]/XTlo[0] and W
// split in Xhi[0]/Xlo[0].  If `want_h`, also computes Hsym = (W^T M)_sym (FP64
// averaging) and copies it to H_out (may be null).  Never synchronizes: the step budget is
// launched whole and finished matrices are skipped on the device.  Fills info (device,
// may be null).  With the learned schedule, matrices that miss tol within their budget
// (ws.fallback) are rerun from X0 with the conservative schedule when `rerun_learned`;
// otherwise they are left to the caller (svd_fwd recomputes them on its plain path).
int polar_forward(const float *A, float *W, float *H_out, bool want_h, PolarWS &ws, const psvd_opts &o,
                  psvd_info *info, cudaStream_t st, bool rerun_learned = true);

}  // namespace psvd
