// Host runtime pieces shared by every entry point: TMA descriptor encoding through
// the driver entry point (no libcuda link dependency), launch accounting, status
// strings, workspace carving.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "gemm.cuh"
#include "runtime.h"

namespace psvd {

static char g_err[512] = "";
static std::atomic<uint32_t> g_barrier_spin{0};
uint32_t barrier_spin() {
    const uint32_t v = g_barrier_spin.load(std::memory_order_relaxed);
    return v ? v : kBarrierSpin;
}
static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// ---- product-kernel profiling (off by default) ----
namespace {
constexpr int kProfCap = 8192;
struct Prof {
    bool on = false;
    int n = 0;
    cudaEvent_t ev[2 * kProfCap];
    double flops[kProfCap];
    int prec[kProfCap];
    bool created = false;
} g_prof;
std::mutex g_prof_mu;
}  // namespace

bool prof_on() { return g_prof.on; }

int cuda_fail(cudaError_t e, const char *file, int line) {
    const char *f = strrchr(file, '/');
    snprintf(g_err, sizeof(g_err), "%s (%s) at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), f ? f + 1 : file,
             line);
    return PSVD_ERR_CUDA;
}
int fail_msg(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

unsigned long long current_context_id() {
    typedef CUresult (*GetCur)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

void prof_begin(cudaStream_t st) {
    if (g_prof.n < kProfCap) cudaEventRecord(g_prof.ev[2 * g_prof.n], st);
}
void prof_end(cudaStream_t st, double flops, int prec) {
    if (g_prof.n < kProfCap) {
        cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], st);
        g_prof.flops[g_prof.n] = flops;
        g_prof.prec[g_prof.n] = prec;
        ++g_prof.n;
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool make_tmap(CUtensorMap *out, const MatView &v, int box_rows) {
    auto fn = encode_fn();
    if (!fn || !v.ptr) return false;
    const int esz = v.bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)v.cols, (cuuint64_t)v.rows, (cuuint64_t)v.batch};
    cuuint64_t strides[2] = {(cuuint64_t)v.ld * esz, (cuuint64_t)v.bstride * esz};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    if ((strides[0] % 16) || (strides[1] % 16) || (reinterpret_cast<uintptr_t>(v.ptr) % 16)) {
        snprintf(g_err, sizeof(g_err), "tensor map alignment: strides=(%llu,%llu) ptr=%p",
                 (unsigned long long)strides[0], (unsigned long long)strides[1], v.ptr);
        return false;
    }
    CUresult r = fn(out, v.bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void *>(v.ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        snprintf(g_err, sizeof(g_err), "cuTensorMapEncodeTiled=%d dims=(%llu,%llu,%llu) strides=(%llu,%llu) ptr=%p",
                 (int)r, (unsigned long long)dims[0], (unsigned long long)dims[1], (unsigned long long)dims[2],
                 (unsigned long long)strides[0], (unsigned long long)strides[1], v.ptr);
    return r == CUDA_SUCCESS;
}

int num_sms() {
    static int sms = 0, sms_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (sms <= 0 || sms_dev != dev) {
        sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        sms_dev = dev;
    }
    return sms;
}

int check_device() {
    static int cached = -100;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSVD_ERR_CUDA;
    static int cached_dev = -1;
    if (cached != -100 && cached_dev == dev) return cached;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return PSVD_ERR_CUDA;
    cached = (p.major == 10 && (p.minor == 3 || p.minor == 0)) ? PSVD_OK : PSVD_ERR_UNSUPPORTED;
    cached_dev = dev;
    return cached;
}

}  // namespace psvd

extern "C" {

uint64_t psvd_kernel_launch_count(void) { return psvd::g_launches.load(); }

int psvd_debug_set_barrier_spin(uint32_t polls) {
    psvd::g_barrier_spin.store(polls, std::memory_order_relaxed);
    return PSVD_OK;
}

const char *psvd_last_error(void) { return psvd::g_err; }

int psvd_profile_enable(int on) {
    using namespace psvd;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (on && !g_prof.created) {
        for (int i = 0; i < 2 * kProfCap; ++i)
            if (cudaEventCreate(&g_prof.ev[i]) != cudaSuccess) return PSVD_ERR_CUDA;
        g_prof.created = true;
    }
    g_prof.on = on != 0;
    g_prof.n = 0;
    return PSVD_OK;
}

// out[4 * c + {0,1,2,3}] for class c (PSVD_PROF_*): launches, total ms, total algorithmic
// work (flops for the product kernel, bytes for the tridiagonalization), max single-launch ms.
int psvd_profile_read(double *out) {
    using namespace psvd;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < 4 * PSVD_PROF_CLASSES; ++i) out[i] = 0.0;
    for (int i = 0; i < g_prof.n; ++i) {
        if (cudaEventSynchronize(g_prof.ev[2 * i + 1]) != cudaSuccess) return PSVD_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) != cudaSuccess) return PSVD_ERR_CUDA;
        const int c = g_prof.prec[i] < 0 ? PSVD_PROF_MIXED : g_prof.prec[i];
        if (c >= PSVD_PROF_CLASSES) continue;
        out[4 * c] += 1.0;
        out[4 * c + 1] += ms;
        out[4 * c + 2] += g_prof.flops[i];
        if (ms > out[4 * c + 3]) out[4 * c + 3] = ms;
    }
    g_prof.n = 0;
    return PSVD_OK;
}

const char *psvd_status_string(int s) {
    switch (s) {
        case PSVD_OK: return "ok";
        case PSVD_NOT_CONVERGED: return "polar iteration reached its step cap before the tolerance";
        case PSVD_ERR_ARG: return "invalid argument (sizes, m < n, or a required null pointer)";
        case PSVD_ERR_WORKSPACE: return "workspace smaller than the size query requires";
        case PSVD_ERR_NONFINITE: return "input contains NaN or Inf";
        case PSVD_ERR_CUDA: return "CUDA launch or runtime error";
        case PSVD_ERR_TIMEOUT: return "bounded device wait expired";
        case PSVD_ERR_UNSUPPORTED: return "device is not a compute capability 10.x (Blackwell) GPU";
        default: return "unknown status";
    }
}

void psvd_default_opts(psvd_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PSVD_PREC_FP32;
    o->schedule = PSVD_SCHED_CANS;
    o->delta = 0.99;
    o->pre_iters = 2;
    o->max_iter = 50;
    o->tol = 1e-5;
    o->eps_qr = 1e-5;
    o->lower_bound = nullptr;
    o->budget = 0;
}

}  // extern "C"
