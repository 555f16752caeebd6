// Shared device helpers for the sm_103a kernels: mbarriers, TMA tile loads,
// tcgen05 (UMMA) descriptors/issue/TMEM access, TF32 rounding, bounded waits.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/psvd.h"

#define PSVD_DEV __device__ __forceinline__

namespace psvd {

// Device-side error word (bit flags); read back by the host in debug checks.
enum : unsigned { DEV_ERR_TIMEOUT = 1u, DEV_ERR_BOUNDS = 2u };

// Upper bound on polls of any spin-wait.  try_wait itself suspends for a
// hardware-defined interval, so this is well above any legitimate wait.
constexpr uint32_t kSpinLimit = 1u << 22;

PSVD_DEV uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
PSVD_DEV void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
PSVD_DEV void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
PSVD_DEV void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
PSVD_DEV void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
PSVD_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: returns false (and raises the error word) if the phase never completes.
PSVD_DEV bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, DEV_ERR_TIMEOUT);
    return false;
}

// ---------------------------------------------------------------- TMA
PSVD_DEV void tma_prefetch(const CUtensorMap *m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}
// 3-D tiled load (x = innermost element index, y = row, z = batch) completing on `bar`.
PSVD_DEV void tma_load_3d(void *smem_dst, const CUtensorMap *m, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// ---------------------------------------------------------------- tcgen05
PSVD_DEV void tmem_alloc(uint32_t *slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
PSVD_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
PSVD_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
PSVD_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 B, 8-row (1024 B) swizzle atoms stacked along M/N.
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused
// for swizzled K-major), stride byte offset >> 4 (32-45) = 1024 B between 8-row
// groups, descriptor version 1 (bit 46), swizzle mode 2 = 128 B (bits 61-63).
PSVD_DEV uint64_t sdesc_k128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor for kind::f16 / kind::tf32 with FP32 accumulation, both
// operands K-major: D format F32 (bits 4-5 = 1), A/B format (bits 7-9 / 10-12:
// 1 = BF16, 2 = TF32), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_f32acc(uint32_t ab_fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
constexpr uint32_t kFmtBF16 = 1, kFmtTF32 = 2;

PSVD_DEV void umma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
PSVD_DEV void umma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
// Arrive on `bar` once all previously issued MMAs of this thread have completed.
PSVD_DEV void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns: thread t of the warp receives
// row (lane_base + t), columns [col, col + 16).
PSVD_DEV void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- numerics
// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest, ties away.
PSVD_DEV float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// x = hi + lo with hi, lo both TF32-representable and |x - hi - lo| <= 2^-22 |x|.
PSVD_DEV void split_tf32(float x, float &hi, float &lo) {
    hi = tf32_round(x);
    lo = tf32_round(x - hi);
}

PSVD_DEV float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
PSVD_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
PSVD_DEV float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

constexpr uint32_t kBarrierSpin = 1u << 24;

// Group barrier over `g` co-resident CTAs (cooperative launch): monotonic counter,
// bounded spin; on expiry (or an error raised elsewhere) it records the error and
// lets the CTA run on so that every CTA terminates.
// `spin` bounds the polls (kBarrierSpin unless a test lowered it through
// psvd_debug_set_barrier_spin).
PSVD_DEV void group_barrier(unsigned *ctr, unsigned target, unsigned *err, uint32_t spin = kBarrierSpin) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        for (uint32_t i = 0;; ++i) {
            if (*(volatile unsigned *)ctr >= target) break;
            if (*(volatile unsigned *)err) break;
            if (i > spin) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
            __nanosleep(40);
        }
        __threadfence();
    }
    __syncthreads();
}

// Counter barrier over co-resident CTAs with release/acquire operations instead of full
// fences: thread 0 of each CTA adds 1 with release semantics (its CTA's writes, ordered
// before it by the CTA barrier, become visible with it) and polls the counter with
// acquire loads until it reaches `target`; bounded, stops early on a raised error word.
template <int kSleepNs>
PSVD_DEV void counter_barrier(unsigned *ctr, unsigned target, unsigned *err, uint32_t spin = kBarrierSpin) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
        for (uint32_t i = 0;; ++i) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (i > spin) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
            if ((i & 63) == 63 && *(volatile unsigned *)err) break;
            if (kSleepNs > 0) __nanosleep(kSleepNs);
        }
    }
    __syncthreads();
}

// Flag barrier over `g` co-resident CTAs: CTA c publishes arrive[c] = gen; CTA 0 polls all
// arrival flags in parallel and publishes release = gen, which every other CTA polls.
// Every wait is bounded and stops at once when the error word is raised elsewhere.
PSVD_DEV void flag_barrier(unsigned *arrive, unsigned *release, int cig, int g, unsigned gen, unsigned *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *(volatile unsigned *)&arrive[cig] = gen;
    }
    if (cig == 0) {
        for (int c = threadIdx.x; c < g; c += blockDim.x) {
            for (uint32_t i = 0;; ++i) {
                if (*(volatile unsigned *)&arrive[c] >= gen) break;
                if (*(volatile unsigned *)err) break;
                if (i > kBarrierSpin) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
                __nanosleep(20);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            *(volatile unsigned *)release = gen;
        }
    } else if (threadIdx.x == 0) {
        for (uint32_t i = 0;; ++i) {
            if (*(volatile unsigned *)release >= gen) break;
            if (*(volatile unsigned *)err) break;
            if (i > kBarrierSpin) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
            __nanosleep(20);
        }
    }
    __threadfence();
    __syncthreads();
}

// ---------------------------------------------------------------- float-float sums
// Compensated FP32 accumulation (Knuth's TwoSum and the FMA-based exact product,
// written with the _rn intrinsics so that no add is contracted into an FMA): the
// pair (hi, lo) carries about twice the FP32 precision.  On GB300 the FP64 pipe is
// narrow, and these sums keep long reductions on the FP32 pipe.
struct ff { float hi, lo; };
PSVD_DEV ff ff_zero() { return ff{0.f, 0.f}; }
PSVD_DEV ff ff_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return ff{h, __fsub_rn(t, __fsub_rn(h, s))};
}
// a + x * y
PSVD_DEV ff ff_fma(ff a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const float s = __fadd_rn(a.hi, p);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float t = __fadd_rn(e, __fadd_rn(a.lo, pe));
    const float h = __fadd_rn(s, t);
    return ff{h, __fsub_rn(t, __fsub_rn(h, s))};
}
// a * b and a * (float) b: the exact product of the leading words plus the cross terms
PSVD_DEV ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return ff{h, __fsub_rn(e, __fsub_rn(h, p))};
}
PSVD_DEV ff ff_mulf(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    const float h = __fadd_rn(p, e);
    return ff{h, __fsub_rn(e, __fsub_rn(h, p))};
}
PSVD_DEV ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
PSVD_DEV ff warp_sum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}
// Block-wide sum, returned to every thread as the nearest FP32 value; `red` holds
// 2 x 32 floats of shared memory.  Contains two __syncthreads.
PSVD_DEV float block_sum_ff(ff v, float *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { red[w] = v.hi; red[32 + w] = v.lo; }
    __syncthreads();
    // every warp reduces the per-warp partials the same way (same result everywhere)
    const int nw = (int)(blockDim.x >> 5);
    ff t = l < nw ? ff{red[l], red[32 + l]} : ff_zero();
    t = warp_sum(t);
    return __fadd_rn(t.hi, t.lo);
}

// Flag barrier over `g` co-resident CTAs in which every CTA polls every arrival
// flag (no release hop): CTA c publishes arrive[c] = gen, then its threads wait
// until all g flags have reached gen.  Bounded like flag_barrier.
PSVD_DEV void flag_barrier_all(unsigned *arrive, int cig, int g, unsigned gen, unsigned *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *(volatile unsigned *)&arrive[cig] = gen;
    }
    for (int c = threadIdx.x; c < g; c += blockDim.x) {
        for (uint32_t i = 0;; ++i) {
            if (*(volatile unsigned *)&arrive[c] >= gen) break;
            if (*(volatile unsigned *)err) break;
            if (i > kBarrierSpin) { atomicOr(err, DEV_ERR_TIMEOUT); break; }
            __nanosleep(20);
        }
    }
    __threadfence();
    __syncthreads();
}

PSVD_DEV double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

}  // namespace psvd
