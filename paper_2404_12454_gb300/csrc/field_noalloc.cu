// gbd_field_noalloc: the field computation of gbd_field for callers that may not allocate
// device memory -- for example a plugin inside a host application that owns every device
// allocation, or a real-time loop whose memory is fixed at start-up -- and so can neither
// call cudaMalloc nor hand the library a workspace.  Its scratch (the projected beamlet
// records and the per-split partial fields) lives in one fixed array in this file, which
// every GPU that loads the library keeps for the life of the process.
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "gbd.h"
#include "gbd_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GBD_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_addr;  // device ordinal -> device address of the array

// Device address of the scratch array on the current device.  In host code the array's
// name only stands in for the symbol and is not a device address, so the address is
// looked up once per device, with that device current, and cached.
gbd_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gbd_set_error(GBD_ECUDA, cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return GBD_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return gbd_set_error(GBD_ECUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                         : "scratch array has no device address");
    g_noalloc_addr[dev] = p;
    *out = p;
    return GBD_OK;
}

}  // namespace

extern "C" gbd_status gbd_field_noalloc(const gbd_beamlet* beamlets, int32_t n_beamlets,
                                        double wavelength, const gbd_detector* detector,
                                        int32_t precision, void* field_out, void* stream) {
    void* scratch = nullptr;
    gbd_status st = scratch_address(&scratch);
    if (st != GBD_OK) return st;
    return gbd_field_fixed_scratch(beamlets, n_beamlets, wavelength, detector, precision, scratch,
                                   GBD_NOALLOC_SCRATCH_BYTES, field_out,
                                   static_cast<cudaStream_t>(stream));
}
