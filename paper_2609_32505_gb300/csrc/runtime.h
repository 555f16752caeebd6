// Host-side helpers shared by the entry points.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/psvd.h"

namespace psvd {

int check_device();
// Poll bound of the grid barriers of the cooperative kernels (see psvd_debug_set_barrier_spin).
uint32_t barrier_spin();
void count_launch(int n);

inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace; every block is 256-byte aligned.
struct Carver {
    char *base;
    size_t cap, used = 0;
    bool overflow = false;
    Carver(void *p, size_t c) : base(static_cast<char *>(p)), cap(c) {}
    template <class T>
    T *take(size_t count) {
        size_t off = (size_t)round_up((long long)used, 256);
        size_t bytes = count * sizeof(T);
        used = off + bytes;
        if (!base || used > cap) { overflow = true; return nullptr; }
        return reinterpret_cast<T *>(base + off);
    }
};

// Sizing pass: same carving sequence with a null base.
struct Sizer {
    size_t used = 0;
    template <class T>
    T *take(size_t count) {
        used = (size_t)round_up((long long)used, 256) + count * sizeof(T);
        return nullptr;
    }
};

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? PSVD_OK : PSVD_ERR_CUDA; }

// Records where a CUDA call failed (readable through psvd_last_error) and returns
// PSVD_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *file, int line);
// Records a free-form message for psvd_last_error (printf-style) and returns `status`.
int fail_msg(int status, const char *fmt, ...);
// Unique ID of the calling thread's current CUDA context (cuCtxGetId through the driver
// entry point; distinct for a context created after cudaDeviceReset), 0 if unavailable.
unsigned long long current_context_id();
#define PSVD_TRY(expr)                                                        \
    do {                                                                      \
        cudaError_t _psvd_e = (expr);                                         \
        if (_psvd_e != cudaSuccess) return psvd::cuda_fail(_psvd_e, __FILE__, __LINE__); \
    } while (0)
#define PSVD_TRY_RC(expr)                                                     \
    do {                                                                      \
        int _psvd_rc = (expr);                                                \
        if (_psvd_rc) return _psvd_rc;                                        \
    } while (0)

}  // namespace psvd
