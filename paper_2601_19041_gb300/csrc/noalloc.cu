// Decode entry point for callers that must not allocate device memory.
//
// Some programs cannot call cudaMalloc when they want a tour: a host
// application whose caching allocator (or fixed memory budget) already owns
// the free device memory, or a latency-critical serving loop where an
// allocation could synchronise the device or fail under memory pressure.
// hac_solve_noalloc serves them with a fixed scratch area compiled into the
// library: a file-scope __device__ array that every GPU loading the library
// holds until the process exits.  Everything else (inputs, outputs) stays
// with the caller.
#include <mutex>

#include "hac_internal.cuh"

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)HAC_NOALLOC_MAX_BYTES;
constexpr int MAX_DEVICES = 64;

// The scratch itself.  In host code this name is only a host-side stand-in for
// the symbol, never a device address: the device address is obtained below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES];   // device address of the array, per device ordinal

// Set-up, once per device with that device current: look up the array's
// device address.  Runs inside the first call on a device.
int scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return HAC_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return HAC_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return HAC_ECUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HAC_OK;
}

}  // namespace

extern "C" int hac_solve_noalloc(const hac_instance *in, const hac_params *p,
                                 int32_t inputs_on_device, int32_t *best_tour, double *best_len,
                                 void *stream)
{
    size_t need = 0;
    int st = hac_batch_workspace_size(in, p, 1, inputs_on_device, &need);
    if (st) return st;
    if (need > NOALLOC_BYTES) return HAC_ENOMEM;   // instance too large for the fixed scratch
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;
    // no CUDA graph and no profiling events: nothing in this call allocates
    hac_exec ex;
    hac_exec_default(&ex);
    ex.use_graph = 0;
    ex.profile = 0;
    int32_t *tours[1] = {best_tour};
    return hac_solve_batch(in, p, 1, inputs_on_device, scratch, NOALLOC_BYTES, &ex, tours,
                           best_len, nullptr, nullptr, stream);
}
