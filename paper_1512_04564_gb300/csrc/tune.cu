// Projector autotuner: for one geometry, time every available forward and
// back-projector decomposition on a representative subset and keep the
// fastest (stored in the geometry; launch_fp / launch_bp follow it).
//   forward: resident-matrix rows (warp per ray) | 32-cell bundles (footprint
//            once per pixel, shared-memory routing) | 8 lanes per ray
//   back:    stored footprints | footprints on the fly
#include <vector>

#include "ct_internal.cuh"

namespace ct {
namespace {

__global__ void fill_kernel(float *p, size_t n, float v)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_geom_autotune(ct_geom *g, int views_per_launch, int *fp_choice, int *bp_choice, void *stream)
{
    if (!g) { set_error("ct_geom_autotune: null geometry"); return CT_EINVAL; }
    if (g->helical) { set_error("ct_geom_autotune: 2-D fan-beam geometries only"); return CT_ENOTSUP; }
    const int na = g->fan.na, ns = g->fan.ns;
    int nv = views_per_launch > 0 ? views_per_launch : (na < 24 ? na : 24);
    if (nv > na) nv = na;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t npix = (size_t)g->fan.nx * g->fan.ny;
    float *x = nullptr, *y = nullptr;
    CT_CUDA_TRY(cudaMalloc(&x, sizeof(float) * npix), "autotune buffers");
    if (cudaMalloc(&y, sizeof(float) * (size_t)nv * ns) != cudaSuccess) {
        cudaFree(x);
        set_error("autotune buffers: out of memory");
        return CT_ENOMEM;
    }
    struct Bufs {
        float *a, *b;
        ~Bufs() { cudaFree(a); cudaFree(b); }
    } bufs{x, y};
    fill_kernel<<<256, 256, 0, st>>>(x, npix, 1.0f);
    fill_kernel<<<256, 256, 0, st>>>(y, (size_t)nv * ns, 1.0f);
    // evenly spread views, as one ordered subset
    std::vector<int> hv(nv);
    for (int k = 0; k < nv; k++) hv[k] = (int)((long)k * na / nv);
    const int *dv = nullptr;
    ct_status s0 = stage_views(g, hv.data(), nv, &dv, st);
    if (s0 != CT_OK) return s0;
    cudaEvent_t e0, e1;
    CT_CUDA_TRY(cudaEventCreate(&e0), "event");
    CT_CUDA_TRY(cudaEventCreate(&e1), "event");
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    auto time_it = [&](auto launch, float *ms) -> cudaError_t {
        cudaError_t e = launch();  // warm-up
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
        for (int r = 0; r < 5; r++)
            if ((e = launch()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        return cudaEventElapsedTime(ms, e0, e1);
    };
    FanDev G = g->fan;
    const bool bundle_ok = G.max_span <= 12 && G.nx <= 2048 && G.ny <= 2048;
    int best_fp = FP_VAR_RAY, best_bp = BP_VAR_FLY;
    float best = 1e30f;
    const int fps[3] = {FP_VAR_CSR, FP_VAR_BUNDLE, FP_VAR_RAY};
    for (int c : fps) {
        if (c == FP_VAR_CSR && !G.row_ptr) continue;
        if (c == FP_VAR_BUNDLE && !bundle_ok) continue;
        FanDev T = G;
        T.fp_variant = c;
        float ms = 0.0f;
        CT_CUDA_TRY(time_it([&] { return launch_fp(T, FP_PLAIN, x, dv, nv, y, nullptr, nullptr, st); }, &ms),
                    "autotune forward");
        if (ms < best) { best = ms; best_fp = c; }
    }
    best = 1e30f;
    const int bps[2] = {BP_VAR_STORED, BP_VAR_FLY};
    float* xo = x;
    for (int c : bps) {
        if (c == BP_VAR_STORED && !G.rec_data) continue;
        FanDev T = G;
        T.bp_variant = c;
        float ms = 0.0f;
        CT_CUDA_TRY(time_it([&] { return launch_bp(T, BP_PLAIN, y, dv, nv, xo, 1.0f, 0, nullptr, st); }, &ms),
                    "autotune back");
        if (ms < best) { best = ms; best_bp = c; }
    }
    g->fan.fp_variant = best_fp;
    g->fan.bp_variant = best_bp;
    drop_ray_sums(g);  // recomputed with the chosen forward projector when next needed
    if (fp_choice) *fp_choice = best_fp;
    if (bp_choice) *bp_choice = best_bp;
    return CT_OK;
}
