// An entry point for callers that may not allocate device memory.
//
// Some host applications own every byte of device memory through their own
// pool and forbid allocations once their time loop runs (an allocation
// there can synchronise the device, fragment the pool, or is simply not
// allowed by the host's memory policy).  sunb_integrate_robertson_noalloc
// lets such a caller integrate a batch of Robertson cells without a
// context: it takes the inputs and outputs from the caller and keeps its
// own scratch -- the work-queue counter and the per-cell counters -- in a
// file-scope static device array of fixed size, so that it calls no
// cudaMalloc, cudaFree or other allocating routine.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "sunb.h"
#include "kernels_thread.cuh"

using namespace sunb;

void sunb_internal_set_error(const std::string &msg);   // sunb_api.cu

namespace {

constexpr long long NOALLOC_MAX_CELLS = 65536;
constexpr size_t NOALLOC_SCRATCH_BYTES = 256 + 32 * (size_t)NOALLOC_MAX_CELLS;   // 2 MiB + 256 B

// [0, 8): work-queue counter; [256, ...): per-cell counters, 8 int32 each.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).  In host code the array's name is
// only a host-side stand-in, never a usable device address.
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= MAX_DEVICES) {
        sunb_internal_set_error("noalloc: device index out of range");
        return SUNB_ILL_INPUT;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            sunb_internal_set_error(std::string("noalloc: cudaGetSymbolAddress failed: ") +
                                    cudaGetErrorString(e));
            return SUNB_CUDA_ERROR;
        }
        // the step-size choice evaluates this unit's exp and log tables
        const cudaError_t t = fill_math_tables();
        if (t != cudaSuccess) {
            sunb_internal_set_error(std::string("noalloc: math table copy failed: ") + cudaGetErrorString(t));
            return SUNB_CUDA_ERROR;
        }
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return SUNB_SUCCESS;
}

}  // namespace

extern "C" int sunb_integrate_robertson_noalloc(const double *dev_k, double *dev_y, int64_t n_cells,
                                                double t0, double tout, double rtol,
                                                const double *host_atol, int32_t max_steps,
                                                int32_t *dev_status, void *stream)
{
    if (!dev_k || !dev_y || !host_atol) {
        sunb_internal_set_error("noalloc: k, y and atol must not be NULL");
        return SUNB_ILL_INPUT;
    }
    if (n_cells < 0 || n_cells > NOALLOC_MAX_CELLS) {
        sunb_internal_set_error("noalloc: n_cells must lie in 0..65536 (the size of the static scratch)");
        return SUNB_ILL_INPUT;
    }
    if (!(rtol > 0.0) || !(rtol < 1.0) || !(host_atol[0] > 0.0) || !(host_atol[1] > 0.0) ||
        !(host_atol[2] > 0.0) || !std::isfinite(t0) || !std::isfinite(tout) || tout < t0) {
        sunb_internal_set_error("noalloc: need 0 < rtol < 1, positive atol and finite t0 <= tout");
        return SUNB_ILL_INPUT;
    }
    if (n_cells == 0) return SUNB_SUCCESS;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        sunb_internal_set_error("noalloc: no CUDA device");
        return SUNB_CUDA_ERROR;
    }
    void *scratch = nullptr;
    const int rc = scratch_address(device, &scratch);
    if (rc != SUNB_SUCCESS) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the queue counter keeps the previous call's value: clear it first
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        sunb_internal_set_error(std::string("noalloc: cudaMemsetAsync: ") + cudaGetErrorString(e));
        return SUNB_CUDA_ERROR;
    }
    Controls ctl;
    ctl.rtol = rtol;
    ctl.t0 = t0;
    ctl.tout = tout;
    ctl.max_steps = max_steps > 0 ? max_steps : 100000;
    ctl.max_order = 5;
    // the context path's thread-per-cell kernel, with the queue counter and
    // the per-cell counters in the static scratch: the same cell arithmetic
    ThreadArgs a{};
    a.n = n_cells;
    a.y = dev_y;
    a.params = dev_k;
    a.stats = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(scratch) + 256);
    a.status = dev_status;
    a.queue = static_cast<unsigned long long *>(scratch);
    a.ctl = ctl;
    for (int i = 0; i < 3; ++i) a.atol[i] = host_atol[i];
    a.spread_lanes = 0;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const long long want = (n_cells + 255) / 256;
    const int grid = (int)(want < 4LL * sms ? want : 4LL * sms);
    thread_kernel<RobertsonProblem><<<grid, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        sunb_internal_set_error(std::string("noalloc: launch: ") + cudaGetErrorString(e));
        return SUNB_CUDA_ERROR;
    }
    return SUNB_SUCCESS;
}
