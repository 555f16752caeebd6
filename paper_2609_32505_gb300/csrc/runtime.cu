// Host runtime pieces shared by every entry point: TMA descriptor encoding through
// the driver entry point (no libcuda link dependency), launch accounting, status
// strings, workspace carving.
#include <atomic>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "gemm.cuh"
#include "runtime.h"

namespace psvd {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

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

bool make_tmap(CUtensorMap *out, const MatView &v) {
    auto fn = encode_fn();
    if (!fn || !v.ptr) return false;
    const int esz = v.bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)v.cols, (cuuint64_t)v.rows, (cuuint64_t)v.batch};
    cuuint64_t strides[2] = {(cuuint64_t)v.ld * esz, (cuuint64_t)v.bstride * esz};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), 128u, 1u};
    cuuint32_t estr[3] = {1, 1, 1};
    if ((strides[0] % 16) || (strides[1] % 16) || (reinterpret_cast<uintptr_t>(v.ptr) % 16)) return false;
    CUresult r = fn(out, v.bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void *>(v.ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
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
