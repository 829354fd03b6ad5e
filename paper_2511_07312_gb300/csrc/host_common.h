// host_common.h -- host-side helpers shared by the library's translation units:
// thread-local error text, CUDA error checks, argument checks, launch sizing.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <string>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "stratego.h"

namespace stg {

// An NVTX range named after the C entry point, open for the duration of the
// call (visible in Nsight Systems and Nsight Compute range filters; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define ST_NVTX(name) ::stg::NvtxRange st_nvtx_range_(name)

void set_error(const char* fmt, ...);

#define ST_CHECK_ARG(cond, ...)                  \
    do {                                         \
        if (!(cond)) {                           \
            ::stg::set_error(__VA_ARGS__);       \
            return ST_ERR_INVALID;               \
        }                                        \
    } while (0)

#define ST_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::stg::set_error("%s failed: %s", #call, cudaGetErrorString(e_));      \
            return ST_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

// rollout: the call runs rollouts, so the rollout-policy bit is allowed.
inline bool rules_ok(const st_rules* r, bool rollout = false)
{
    const uint32_t allowed = ST_RULE_TWO_SQUARE | ST_RULE_CHASE | (rollout ? ST_ROLLOUT_MAGNET : 0u);
    return r && r->battleless_limit >= 1 && r->battleless_limit <= ST_MAX_BATTLELESS && r->max_plies >= 1 &&
           (r->flags & ~allowed) == 0;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Number of SMs of the current device.
int sm_count();

}  // namespace stg
