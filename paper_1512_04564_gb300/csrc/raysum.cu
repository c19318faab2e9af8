// Ray sums A 1 of a geometry's system matrix, kept with the geometry.
//
// The SQS majorizer of the data term is D_L = diag(A' W A 1) (Sec. III-A).  A 1
// depends on the scan geometry only, so it is computed once per geometry (by
// ct_geom_precompute with the resident matrix, or by the first call that
// needs it) and every later D_L is one elementwise product w (A 1) and one
// back-projection over all views.
#include "ct_internal.cuh"

namespace ct {
namespace {

__global__ void __launch_bounds__(256) fill_ones_kernel(float *__restrict__ p, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 1.0f;
}

__global__ void __launch_bounds__(256) mul_kernel(const float *__restrict__ a, const float *__restrict__ b,
                                                  float *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __ldg(&a[i]) * __ldg(&b[i]);
}

long long sino_cells(const ct_geom *g)
{
    return (long long)g->fan.na * g->fan.ns * (g->helical ? g->hx.nt : 1);
}

}  // namespace

void drop_ray_sums(ct_geom *g)
{
    cudaFree(g->d_a1);
    g->d_a1 = nullptr;
}

cudaError_t ensure_ray_sums(ct_geom *g, cudaStream_t st)
{
    if (g->d_a1) return cudaSuccess;
    const long long n = sino_cells(g);
    float *a1 = nullptr;
    cudaError_t e = cudaMalloc(&a1, sizeof(float) * (size_t)n);
    if (e != cudaSuccess) return e;
    // w = 1 in the sinogram workspace, then the forward projector's "w (A 1)" mode over all views
    fill_ones_kernel<<<4 * 152, 256, 0, st>>>(g->d_sino_ws, n);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = g->helical ? launch_fp_helix(g, FP_ONES_W, nullptr, g->d_views_all, g->fan.na, a1, nullptr, g->d_sino_ws, st)
                       : launch_fp(g->fan, FP_ONES_W, nullptr, g->d_views_all, g->fan.na, a1, nullptr, g->d_sino_ws, st);
    if (e != cudaSuccess) {
        cudaFree(a1);
        return e;
    }
    g->d_a1 = a1;
    return cudaSuccess;
}

cudaError_t launch_weighted_ray_sums(const ct_geom *g, const float *w, float *out, cudaStream_t st)
{
    mul_kernel<<<4 * 152, 256, 0, st>>>(w, g->d_a1, out, sino_cells(g));
    return cudaGetLastError();
}

}  // namespace ct
