// Filtered back-projection for a full-scan equiangular fan beam: the initial
// image of Algorithm 1 ("an initial (FBP) image", Sec. III-A).  Textbook
// fan-beam FBP with equiangular rays (Kak & Slaney, Ch. 3):
//   p'(beta, gamma) = D cos(gamma) p(beta, gamma);
//   q = dgamma * (p' conv g), g(0) = 1/(8 dgamma^2), g(n dgamma) = 0 (even n),
//       -1 / (2 pi^2 sin^2(n dgamma)) (odd n), optionally Hann-apodised by the
//       3-tap [1/4, 1/2, 1/4] smoothing of g;
//   f(x, y) = dbeta sum_views q(beta, gamma'(x, y)) / L^2, linear interpolation in gamma.
#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr int kFiltThreads = 256;

// One CTA per view: pre-weighted row and the filter taps in shared memory.
__global__ void __launch_bounds__(kFiltThreads) fbp_filter_kernel(FanDev G, const float *__restrict__ y,
                                                                 float *__restrict__ q, int window)
{
    extern __shared__ float sm[];
    float *row = sm;                // [ns]
    float *taps = sm + G.ns;        // [2 ns + 1]: g(n) for n = -ns .. ns
    const int v = blockIdx.x;
    const int ns = G.ns;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const float gam = fmaf((float)s, G.dgamma, G.gamma0);
        row[s] = G.dso * cosf(gam) * y[(size_t)v * ns + s];
    }
    const float inv8 = 1.0f / (8.0f * G.dgamma * G.dgamma);
    const float c = -1.0f / (2.0f * 9.8696044010893586f);  // -1 / (2 pi^2)
    for (int i = threadIdx.x; i < 2 * ns + 1; i += blockDim.x) {
        const int n = i - ns;
        float gv;
        if (window == 1) {  // Hann: 1/4 g(n-1) + 1/2 g(n) + 1/4 g(n+1)
            gv = 0.0f;
#pragma unroll
            for (int d = -1; d <= 1; d++) {
                const int m = n + d;
                float gm;
                if (m == 0) gm = inv8;
                else if (m & 1) { const float sn = sinf((float)m * G.dgamma); gm = c / (sn * sn); }
                else gm = 0.0f;
                gv = fmaf(d == 0 ? 0.5f : 0.25f, gm, gv);
            }
        } else {
            if (n == 0) gv = inv8;
            else if (n & 1) { const float sn = sinf((float)n * G.dgamma); gv = c / (sn * sn); }
            else gv = 0.0f;
        }
        taps[i] = gv;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        float acc = 0.0f;
        for (int k = 0; k < ns; k++) acc = fmaf(row[k], taps[s - k + ns], acc);
        q[(size_t)v * ns + s] = G.dgamma * acc;
    }
}

// Pixel-driven distance-weighted back-projection with linear interpolation.  The
// detector coordinate of the pixel centre is its anchor's FP64-derived one plus
// the offset point_u gives (the footprint code's), instead of a full atan2 per
// (pixel, view).
__global__ void __launch_bounds__(256) fbp_backproject_kernel(FanDev G, const float *__restrict__ q,
                                                              float *__restrict__ x, float dbeta)
{
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31), iy = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (ix >= G.nx || iy >= G.ny) return;
    float acc = 0.0f;
    for (int v = 0; v < G.na; v++) {
        const float2 cs = __ldg(&G.view_cs[v]);
        float px, py;
        const Anchor A = pixel_anchor(G, v, ix, iy, px, py);
        float S, L;
        point_u(G, A, px, py, S, L);
        const float ox = px * G.dx, oy = py * G.dy;
        const float cpar = G.dso + (A.ax + fmaf(ox, cs.x, oy * cs.y)), cperp = A.ay + fmaf(oy, cs.x, -ox * cs.y);
        const float fl = floorf(S + L);
        const int i0 = A.n + (int)fl;
        const float f = (S - fl) + L;
        const float *row = q + (size_t)v * G.ns;
        const float v0 = ((unsigned)i0 < (unsigned)G.ns) ? __ldg(&row[i0]) : 0.0f;
        const float v1 = ((unsigned)(i0 + 1) < (unsigned)G.ns) ? __ldg(&row[i0 + 1]) : 0.0f;
        acc = fmaf(fmaf(f, v1 - v0, v0), __frcp_rn(fmaf(cpar, cpar, cperp * cperp)), acc);
    }
    x[(size_t)iy * G.nx + ix] = dbeta * acc;
}

}  // namespace

cudaError_t launch_fbp(const ct_geom *g, const float *y, float *x, int window, cudaStream_t st)
{
    const FanDev &G = g->fan;
    const size_t smem = sizeof(float) * (3 * (size_t)G.ns + 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fbp_filter_kernel<<<G.na, kFiltThreads, smem, st>>>(G, y, g->d_sino_ws, window);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float dbeta = (float)(g->desc.orbit_deg * M_PI / 180.0 / g->desc.na);
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    fbp_backproject_kernel<<<grid, 256, 0, st>>>(G, g->d_sino_ws, x, dbeta);
    return cudaGetLastError();
}

ct_status validate_fbp(const ct_geom *g, int window)
{
    if (window != CT_FBP_RAMP && window != CT_FBP_HANN) {
        set_error("unknown FBP window %d", window);
        return CT_EINVAL;
    }
    if (g->helical) {
        set_error("FBP is implemented for 2-D fan-beam scans only");
        return CT_ENOTSUP;
    }
    if (std::fabs(g->desc.orbit_deg - 360.0) > 1e-9) {
        set_error("FBP needs a full 360-degree scan (orbit %g)", g->desc.orbit_deg);
        return CT_ENOTSUP;
    }
    if (3 * (size_t)g->fan.ns + 1 > 227 * 1024 / sizeof(float)) {
        set_error("FBP filter row of %d cells exceeds shared memory", g->fan.ns);
        return CT_ENOTSUP;
    }
    return CT_OK;
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_fbp(const ct_geom *g, const float *y, float *x, int window, void *stream)
{
    if (!g || !y || !x) { set_error("ct_fbp: null argument"); return CT_EINVAL; }
    ct_status st = validate_fbp(g, window);
    if (st != CT_OK) return st;
    CT_CUDA_TRY(launch_fbp(g, y, x, window, (cudaStream_t)stream), "ct_fbp launch");
    return CT_OK;
}
