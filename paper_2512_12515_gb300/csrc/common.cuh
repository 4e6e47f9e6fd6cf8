// Shared helpers of the ppRPA GB300 library (host + device).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/pprpa.h"

namespace pprpa {

// Records a message for pprpa_last_error() and returns `code`.
int set_error(int code, const std::string& msg);

// Counts a kernel launch (for pprpa_kernel_launches()).
void count_launch(long long n = 1);

#define PP_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return ::pprpa::set_error(e_ == cudaErrorMemoryAllocation ? PPRPA_ERR_OOM \
                                                                      : PPRPA_ERR_CUDA, \
                                      std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define PP_CHECK_LAUNCH()                                                           \
    do {                                                                            \
        ::pprpa::count_launch();                                                    \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            return ::pprpa::set_error(PPRPA_ERR_CUDA,                               \
                                      std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define PP_TRY(expr)               \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != PPRPA_OK) return rc_; \
    } while (0)

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Status words a kernel can raise (bit flags in a device int).
enum DeviceStatus : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,   // a bounded spin-wait expired
    DEV_NOTPD = 2,     // Cholesky found a non-positive pivot
    DEV_FEWROOTS = 4,  // fewer positive-norm Ritz values than requested
};

}  // namespace pprpa
