// Potential evaluation that performs no device allocation.
//
// ibem_potential allocates a temporary source table (and, on first use, the
// handle's work vectors) on every call.  Some callers cannot allocate at the
// moment they need a potential: code recording a CUDA graph (cudaMalloc is not
// allowed during stream capture), real-time or embedded loops that must not
// touch the allocator, processes whose memory is reserved up front by a pool
// they do not own.  ibem_potential_noalloc serves them: its scratch lives in
// one file-scope device array of IBEM_NOALLOC_SCRATCH_BYTES, so the call only
// launches kernels and clears the caller's output.  The array is part of the
// library image; every GPU that loads libibem holds it until the process exits.
#include <mutex>

#include "ibem_internal.cuh"


// The scratch: lifted density w* (nb doubles per element), then the source table
// (one double4 per Gauss point).  Shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IBEM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so the
// kernels must be given this address instead.
cudaError_t scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[device]);
    return cudaSuccess;
}

}  // namespace

extern "C" ibem_status ibem_potential_noalloc(ibem_handle* h, const double* w_dev, int nrhs,
                                              const double* pts_dev, int64_t npts, double* u_dev) {
    using namespace ibem;
    if (!h) return IBEM_ERR_ARG;
    if (nrhs < 0 || npts < 0 || (nrhs > 0 && npts > 0 && (!w_dev || !pts_dev || !u_dev))) {
        h->err = "ibem_potential_noalloc: bad arguments";
        return IBEM_ERR_ARG;
    }
    if (h->helm) {
        h->err = "ibem_potential_noalloc: Laplace handles only; use ibem_potential for Helmholtz";
        return IBEM_ERR_ARG;
    }
    if (nrhs == 0 || npts == 0) return IBEM_OK;
    const Plan& P = h->P;
    const int QQ = P.Q * P.Q;
    const int64_t nsrc = P.E * QQ;
    const size_t ws_bytes = (((size_t)P.Nstar * sizeof(double) + 255) / 256) * 256;
    const size_t need = ws_bytes + (size_t)nsrc * sizeof(double4_32a);
    if (need > (size_t)IBEM_NOALLOC_SCRATCH_BYTES) {
        h->err = "ibem_potential_noalloc: this discretisation needs " + std::to_string(need) +
                 " bytes of scratch, more than the fixed " + std::to_string((size_t)IBEM_NOALLOC_SCRATCH_BYTES) +
                 "; use ibem_potential";
        return IBEM_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(h->device);
    unsigned char* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(h->device, &scratch);
    if (e != cudaSuccess) {
        h->err = std::string("ibem_potential_noalloc: ") + cudaGetErrorString(e);
        return IBEM_ERR_CUDA;
    }
    double* ws = reinterpret_cast<double*>(scratch);
    double4_32a* srcs = reinterpret_cast<double4_32a*>(scratch + ws_bytes);
    // the scratch is fully overwritten by every call and needs no clearing; the
    // output is cleared by the shared launch sequence
    e = launch_potential_ws(h, w_dev, nrhs, pts_dev, npts, u_dev, ws, srcs);
    if (e != cudaSuccess) {
        h->err = std::string("ibem_potential_noalloc: ") + cudaGetErrorString(e);
        return IBEM_ERR_CUDA;
    }
    return IBEM_OK;
}
