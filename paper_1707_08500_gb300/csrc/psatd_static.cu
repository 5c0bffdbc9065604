// psatd_push_static: the push on a library-owned static device workspace, for
// callers that cannot allocate device memory (see include/psatd.h).
#include <cuda_runtime.h>

#include <mutex>

#include "psatd.h"
#include "psatd_internal.h"

namespace psatd {
int push_into(psatd_plan_s* p, char* base, size_t cap, double c_dt, const double dx[3], const psatd_fields* f,
              double* gauss_dev, cudaStream_t s);
int set_error(psatd_plan_s* p, int code, const char* msg);
}  // namespace psatd

// The workspace of psatd_push_static.  In host code this name is only a
// stand-in for the device symbol: its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_ws[PSATD_STATIC_WORKSPACE_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

extern "C" int psatd_push_static(psatd_plan_t plan, double c_dt, const double dx[3], const psatd_fields* fields,
                                 double* gauss_dev, void* stream) {
    if (!plan) return PSATD_E_ARG;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return psatd::set_error(plan, PSATD_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return psatd::set_error(plan, PSATD_E_ARG, "device ordinal out of range");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_ws);
            if (e != cudaSuccess || !ptr)
                return psatd::set_error(plan, PSATD_E_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
            g_addr[dev] = ptr;
        }
        base = g_addr[dev];
    }
    return psatd::push_into(plan, static_cast<char*>(base), PSATD_STATIC_WORKSPACE_BYTES, c_dt, dx, fields, gauss_dev,
                            static_cast<cudaStream_t>(stream));
}
