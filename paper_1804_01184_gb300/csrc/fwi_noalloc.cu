// fwi_noalloc.cu -- forward modelling for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they
// need a forward model: a service whose device memory is fixed at start-up and must not
// grow afterwards, a plugin inside a framework that owns all device memory, or code running
// where an allocation may block on other work.  fwi_model_noalloc serves them: it runs
// fwi_model on a scratch buffer that is part of the library image itself, a file-scope
// __device__ array of FWI_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library
// holds until the process exits.  The caller still passes its inputs and outputs.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/fwi.h"

namespace {

// The scratch array.  In host code this name is only a host-side stand-in for the device
// symbol, not a device address: the address a kernel may use comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[FWI_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};     // device address of g_scratch on each device, once resolved

}  // namespace

namespace fwi_internal {
void set_error(const char *msg);    // fwi_api.cu: the message fwi_last_error() returns
}

extern "C" int fwi_model_noalloc(const fwi_grid *g, fwi_param pz, const float *xi_a, const float *xi_b,
                                 const fwi_sources *src, const fwi_receivers *rec, float *traces, void *stream)
{
    char msg[256];
    if (!g || !src || !rec) {
        fwi_internal::set_error("fwi_model_noalloc: null grid, sources or receivers");
        return FWI_EINVAL;
    }
    const size_t need = fwi_workspace_bytes(g, src->ns, rec->nr, FWI_OP_MODEL, 0);
    if (need == 0) {
        fwi_internal::set_error("fwi_model_noalloc: invalid grid or sizes");
        return FWI_EINVAL;
    }
    if (need > (size_t)FWI_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof msg,
                 "fwi_model_noalloc: this grid needs %zu bytes of scratch even one shot at a time; the "
                 "built-in scratch holds %zu (use fwi_model with a caller workspace)",
                 need, (size_t)FWI_NOALLOC_SCRATCH_BYTES);
        fwi_internal::set_error(msg);
        return FWI_ENOMEM;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        snprintf(msg, sizeof msg, "fwi_model_noalloc: no usable current device (%s)", cudaGetErrorString(e));
        fwi_internal::set_error(msg);
        return FWI_ECUDA;
    }
    void *scratch;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof msg, "fwi_model_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                fwi_internal::set_error(msg);
                return FWI_ECUDA;
            }
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    // fwi_model clears everything it needs zeroed (wavefield state, status word) itself, so
    // whatever the previous call left in the scratch does not matter.
    return fwi_model(g, pz, xi_a, xi_b, src, rec, traces, scratch, (size_t)FWI_NOALLOC_SCRATCH_BYTES, stream);
}

// The status word fwi_model_noalloc's kernels record lives at the start of the built-in
// scratch of the current device; fwi_status reads and clears it there.  Before any call on
// this device there is nothing to report.
extern "C" int fwi_status_noalloc(void *stream)
{
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        char msg[160];
        snprintf(msg, sizeof msg, "fwi_status_noalloc: no usable current device (%s)", cudaGetErrorString(e));
        fwi_internal::set_error(msg);
        return FWI_ECUDA;
    }
    void *scratch;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        scratch = g_addr[dev];
    }
    return scratch ? fwi_status(scratch, stream) : FWI_OK;
}
