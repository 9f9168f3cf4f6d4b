// noalloc.cu -- nh_diagnostics_noalloc: the global diagnostics reduction for
// callers that cannot allocate device memory.
//
// The ordinary path (nh_diagnostics) keeps its per-block partial sums in the
// context workspace that the caller allocated beforehand.  Some callers have
// no such workspace and may not allocate one at the point of the call: a host
// application that hands the library only its own input and output buffers
// and forbids any further device allocation (a fixed memory budget, or a
// custom allocator that every allocation must go through), or a time-critical
// loop that cannot afford the implicit device synchronisation of cudaMalloc.
// This entry point serves them: its only scratch is the file-scope array
// below, which the CUDA runtime places in device memory when it loads this
// library's module.  The function itself calls no cudaMalloc, cudaFree or any
// other allocating routine.
#include <mutex>
#include <string>

#include "nh_internal.cuh"

namespace {

constexpr int kNoallocMaxBlocks = NH_NOALLOC_MAX_ITEMS / 256;  // at most 1024 reduction blocks
constexpr int kNoallocValues = 6;                               // mass, energy, max|u|, min|n|, max|n|, nonfinite

// Per-block partial results of the reduction (value-major: value k of block b
// at k * blocks + b).  Every GPU that loads the library holds this array
// (48 KiB) until the process exits.  Each block overwrites its own entries,
// so nothing needs clearing between calls.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * kNoallocValues];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_partials_dev[kMaxDevices] = {};

// Errors are reported like the other context-free failures: through
// nh_last_error(NULL).
int noalloc_fail(int code, const std::string& msg)
{
    nh::set_global_error(msg);
    return code;
}

// Device address of g_noalloc_partials on the current device.  In host code
// the symbol is only a host-side stand-in, so the address is obtained once per
// device, with that device current, and cached.
int partials_address(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(NH_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(NH_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_dev[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess)
            return noalloc_fail(NH_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_partials_dev[dev] = static_cast<double*>(ptr);
    }
    *out = g_partials_dev[dev];
    return NH_OK;
}

}  // namespace

extern "C" int nh_diagnostics_noalloc(const nh_params* p, const void* f, const void* n, const void* u,
                                      const void* rho, double* out, void* stream)
{
    if (!p || !f || !n || !u || !rho || !out) return noalloc_fail(NH_EINVAL, "NULL argument");
    std::string err;
    if (nh::validate_params(p, err) != NH_OK) return noalloc_fail(NH_EINVAL, err);  // the checks of nh_create
    const bool fp64 = p->precision == NH_FP64 && p->storage == NH_STORE_F64;
    const bool fp32 = p->precision == NH_FP32 && p->storage == NH_STORE_F32;
    if (!fp64 && !fp32)
        return noalloc_fail(NH_EINVAL, "nh_diagnostics_noalloc supports FP64/F64 and FP32/F32 populations only");
    // A bound on the work of one call, not on the scratch: the reduction runs at
    // most 1024 blocks (the scratch holds their partials) that stride over the
    // domain, so larger domains would reduce correctly but are kept to at most
    // 256 column chunks per block.
    const long long items = (long long)p->nx * p->ny * ((p->nz + 15) / 16);
    if (items > NH_NOALLOC_MAX_ITEMS)
        return noalloc_fail(NH_EINVAL, "domain larger than this entry point accepts: nx*ny*ceil(nz/16) = " +
                                           std::to_string(items) + " > " + std::to_string(NH_NOALLOC_MAX_ITEMS));
    double* partials = nullptr;
    int r = partials_address(&partials);
    if (r) return r;

    nh::DiagArgs a;
    a.f = f;
    a.storage = p->storage;
    a.shifted = p->shifted;
    a.n = n;
    a.u = u;
    a.rho = rho;
    a.precision = p->precision;
    a.scale = nullptr;  // read only by the 16-bit stores, which are rejected above
    a.g = nh::Geom{p->nx, p->ny, p->nz, p->walls_z, p->anchoring, p->nx * p->ny * p->nz};
    a.K = p->K;
    a.q0 = p->q0;
    a.W0 = p->W0;
    a.frank3 = p->frank3 == 1;
    a.solid = nullptr;  // no obstacles
    a.kd1 = a.frank3 ? p->K11 - p->K : 0.0;
    a.kd2 = a.frank3 ? p->K22 - p->K : 0.0;
    a.kd3 = a.frank3 ? p->K33 - p->K : 0.0;
    a.n_tubes = 0;      // no tube tracking: the trig tables are not read
    a.trig = nullptr;
    a.partials = partials;
    a.result = out;
    a.blocks = kNoallocMaxBlocks;
    cudaError_t e = nh::launch_diagnostics(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return noalloc_fail(NH_ECUDA, std::string("diagnostics launch: ") + cudaGetErrorString(e));
    return NH_OK;
}
