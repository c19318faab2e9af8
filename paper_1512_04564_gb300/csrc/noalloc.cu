// Allocation-free variant of ct_sqs_diag.
//
// Some callers cannot allocate device memory once they are running: a
// process whose device memory is reserved up front by its own pool (a
// serving process, or a framework that owns every byte of the device), or a
// latency-critical reconstruction loop that must not enter cudaMalloc /
// cudaFree, which can block and synchronise the whole device.  For them,
// ct_sqs_diag_noalloc computes D_L = A'(w (A 1)) with its intermediate
// sinogram w (A 1) in a file-scope device array of this compile unit's
// module, instead of in the geometry's workspace.  It calls no cudaMalloc,
// cudaFree or allocating library routine.  When the geometry already keeps
// its ray sums A 1 (from an earlier ct_sqs_diag or ct_geom_precompute), the
// weights are one elementwise product; otherwise one forward projection of
// the weights over all views writes them.
//
// The array's device address is looked up once per device, with that device
// current, by the first call made on that device; make that first call
// before any stream capture.  Under CUDA's lazy module loading that lookup
// is also what loads the module on the device, so the first call on each
// device needs 4 MiB of device memory outside any pool the caller reserved;
// from then on the device holds the array until the process exits.  The
// cached address is valid for the life of the device's primary context (a
// cudaDeviceReset invalidates it).  All calls share the array: calls that
// overlap on the GPU (different streams, or host threads racing on one
// device) race on it.  Every element the back-projection reads is written
// by the same call, so nothing needs clearing between calls.
#include <mutex>

#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr long long kNoAllocMaxCells = 1ll << 20;  // na * ns limit: 4 MiB of float32
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_sqs_scratch[kNoAllocMaxCells];

std::mutex g_scratch_mu;
float *g_scratch_ptr[kMaxDevices] = {};

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_sqs_diag_noalloc(const ct_geom *g, const float *w, float *d_l, void *stream)
{
    if (!g || !w || !d_l) { set_error("ct_sqs_diag_noalloc: null argument"); return CT_EINVAL; }
    if (g->helical) { set_error("ct_sqs_diag_noalloc: 2-D fan-beam geometries only"); return CT_ENOTSUP; }
    const long long cells = (long long)g->fan.na * g->fan.ns;
    if (cells > kNoAllocMaxCells) {
        set_error("ct_sqs_diag_noalloc: the sinogram has %lld cells (na * ns); the allocation-free scratch holds "
                  "at most %lld (4 MiB)", cells, kNoAllocMaxCells);
        return CT_EINVAL;
    }
    int dev = -1;
    CT_CUDA_TRY(cudaGetDevice(&dev), "ct_sqs_diag_noalloc: current device");
    if (dev != g->device) {
        set_error("ct_sqs_diag_noalloc: current device %d, geometry created on device %d", dev, g->device);
        return CT_EINVAL;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("ct_sqs_diag_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
        return CT_EINVAL;
    }
    float *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            CT_CUDA_TRY(cudaGetSymbolAddress(&p, g_sqs_scratch), "ct_sqs_diag_noalloc: scratch address");
            g_scratch_ptr[dev] = (float *)p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // q = w (A 1) over all views into the static scratch (from the kept ray sums if the geometry has
    // them; computing and keeping them would allocate), then D_L = A' q
    if (g->d_a1)
        CT_CUDA_TRY(launch_weighted_ray_sums(g, w, scratch, s), "ct_sqs_diag_noalloc weights");
    else
        CT_CUDA_TRY(launch_fp(g->fan, FP_ONES_W, nullptr, g->d_views_all, g->fan.na, scratch, nullptr, w, s),
                    "ct_sqs_diag_noalloc forward");
    CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, scratch, g->d_views_all, g->fan.na, d_l, 1.0f, 0, nullptr, s),
                "ct_sqs_diag_noalloc back");
    return CT_OK;
}
