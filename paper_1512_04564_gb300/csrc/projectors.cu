// Separable-footprint fan-beam projector pair for sm_103a.
//
// A is the SF system matrix of the PWLS problem (Sec. III, Eq. (ct_problem));
// each a_ij comes from one device function (sf_footprint) used by both the
// ray-driven forward projector and the voxel-driven back-projector, so the
// pair is matched.  Both are FP32-ALU bound gathers (no tensor-core
// contraction exists in them).
//
// Forward projector: each detector cell (ray) is owned by 8 lanes of one
// warp, each lane marching 1/8 of the image columns (or rows, for steep
// rays) through the cell's fan wedge; the 8 partial sums are combined with
// warp shuffles.  No atomics.  Fused epilogues: plain y = A x, the weighted
// residual r = w (A x - y) of the subset gradient (Eq. (ct_substitution)), and
// w * (A 1) for the SQS diagonal.
//
// Back-projector: one CTA per 16x16 pixel tile (one anchor per view), one
// pixel per thread, gathering from the cells its footprint covers.  Fused
// epilogues: plain x = scale A'r (+x), and the relaxed OS-LALM g/h updates of
// Algorithm 1/2 (Sec. III-A).
#include <cstdio>

#include "ct_internal.cuh"

namespace ct {

namespace {

constexpr int kFpThreads = 256;
constexpr int kFpSeg = 8;  // lanes per ray
constexpr float kRangePad = 0.02f;  // pixels of padding on the wedge's row/column range

__device__ __forceinline__ float cell_weight(const Footprint &F, int s)
{
    const float j = (float)(s - F.n);
    return F.amp * (trap_cdf(F, j + 0.5f) - trap_cdf(F, j - 0.5f));
}

template <int MODE>
__global__ void __launch_bounds__(kFpThreads) fp_fan2d_kernel(FanDev G, const float *__restrict__ x,
                                                              const int *__restrict__ views, int nviews,
                                                              float *__restrict__ out, const float *__restrict__ y,
                                                              const float *__restrict__ w)
{
    const int lane = threadIdx.x & 31;
    const long gwarp = ((long)blockIdx.x * kFpThreads + threadIdx.x) >> 5;
    const long ray = gwarp * (32 / kFpSeg) + lane / kFpSeg;
    const int seg = lane % kFpSeg;
    const long nrays = (long)nviews * G.ns;
    const bool valid = ray < nrays;
    float acc = 0.0f;
    int k = 0, s = 0, v = 0;
    if (valid) {
        k = (int)(ray / G.ns);
        s = (int)(ray - (long)k * G.ns);
        v = __ldg(&views[k]);
        const float2 cs = __ldg(&G.view_cs[v]);
        const float beta = __ldg(&G.view_beta[v]);
        const float phi = beta + fmaf((float)s, G.dgamma, G.gamma0);
        float sp, cp;
        sincosf(phi, &sp, &cp);
        const float Sx = -G.dso * cs.x, Sy = -G.dso * cs.y;
        const float phl = phi - 0.5f * G.dgamma, phh = phi + 0.5f * G.dgamma;
        if (fabsf(cp) >= fabsf(sp)) {
            // shallow ray: march columns; the wedge's edges are y = Sy + (x - Sx) tan(phi -+ dgamma/2)
            const float tl = tanf(phl), th = tanf(phh);
            const int c0 = seg * G.nx / kFpSeg, c1 = (seg + 1) * G.nx / kFpSeg;
            for (int ix = c0; ix < c1; ix++) {
                const float xl = fmaf((float)ix, G.dx, G.x_edge0) - Sx, xr = xl + G.dx;
                const float y1 = fmaf(xl, tl, Sy), y2 = fmaf(xr, tl, Sy);
                const float y3 = fmaf(xl, th, Sy), y4 = fmaf(xr, th, Sy);
                const float ylo = (fminf(fminf(y1, y2), fminf(y3, y4)) - G.y_edge0) * G.inv_dy - kRangePad;
                const float yhi = (fmaxf(fmaxf(y1, y2), fmaxf(y3, y4)) - G.y_edge0) * G.inv_dy + kRangePad;
                const int iy0 = max(0, (int)floorf(fmaxf(ylo, -1.0f)));
                const int iy1 = min(G.ny - 1, (int)floorf(fminf(yhi, (float)G.ny)));
                for (int iy = iy0; iy <= iy1; iy++) {
                    const float xv = (MODE == FP_ONES_W) ? 1.0f : __ldg(&x[(size_t)iy * G.nx + ix]);
                    if (xv == 0.0f) continue;
                    const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
                    acc = fmaf(cell_weight(F, s), xv, acc);
                }
            }
        } else {
            // steep ray: march rows; x = Sx + (y - Sy) cot(phi -+ dgamma/2)
            const float tl = cosf(phl) / sinf(phl), th = cosf(phh) / sinf(phh);
            const int r0 = seg * G.ny / kFpSeg, r1 = (seg + 1) * G.ny / kFpSeg;
            for (int iy = r0; iy < r1; iy++) {
                const float yb = fmaf((float)iy, G.dy, G.y_edge0) - Sy, yt = yb + G.dy;
                const float x1 = fmaf(yb, tl, Sx), x2 = fmaf(yt, tl, Sx);
                const float x3 = fmaf(yb, th, Sx), x4 = fmaf(yt, th, Sx);
                const float xlo = (fminf(fminf(x1, x2), fminf(x3, x4)) - G.x_edge0) * G.inv_dx - kRangePad;
                const float xhi = (fmaxf(fmaxf(x1, x2), fmaxf(x3, x4)) - G.x_edge0) * G.inv_dx + kRangePad;
                const int ix0 = max(0, (int)floorf(fmaxf(xlo, -1.0f)));
                const int ix1 = min(G.nx - 1, (int)floorf(fminf(xhi, (float)G.nx)));
                for (int ix = ix0; ix <= ix1; ix++) {
                    const float xv = (MODE == FP_ONES_W) ? 1.0f : __ldg(&x[(size_t)iy * G.nx + ix]);
                    if (xv == 0.0f) continue;
                    const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
                    acc = fmaf(cell_weight(F, s), xv, acc);
                }
            }
        }
    }
#pragma unroll
    for (int o = kFpSeg / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (!valid || seg != 0) return;
    const size_t oi = (size_t)k * G.ns + s;
    if (MODE == FP_PLAIN) {
        out[oi] = acc;
    } else if (MODE == FP_RESID) {
        const size_t yi = (size_t)v * G.ns + s;
        out[oi] = __ldg(&w[yi]) * (acc - __ldg(&y[yi]));
    } else {  // FP_ONES_W: out is [na][ns] in natural view order
        const size_t yi = (size_t)v * G.ns + s;
        out[yi] = __ldg(&w[yi]) * acc;
    }
}

template <int MODE>
__global__ void __launch_bounds__(256) bp_fan2d_kernel(FanDev G, const float *__restrict__ sino,
                                                       const int *__restrict__ views, int nviews,
                                                       float *__restrict__ xo, float scale, int accumulate,
                                                       SolveDev S)
{
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int ix = blockIdx.x * kTile + lx, iy = blockIdx.y * kTile + ly;
    const int tile = blockIdx.y * G.ntx + blockIdx.x;
    const int ntiles = G.ntx * G.nty;
    const float ox = ((float)lx - kTileHalf) * G.dx;
    const float oy = ((float)ly - kTileHalf) * G.dy;
    float rho = 1.0f;
    if (MODE == BP_SOLVE_UPDATE) rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float acc = 0.0f;
    for (int k = 0; k < nviews; k++) {
        const int v = __ldg(&views[k]);
        const float2 cs = __ldg(&G.view_cs[v]);
        const float4 A = __ldg(&G.anchor[(size_t)v * ntiles + tile]);
        const Footprint F = sf_footprint(G, cs.x, cs.y, A, ox, oy);
        const int slo = max(F.n + (int)floorf(F.t0 - 0.5f) + 1, 0);
        const int shi = min(F.n + (int)ceilf(F.t3 + 0.5f) - 1, G.ns - 1);
        const float *row = sino + (size_t)k * G.ns;
        float Fp = trap_cdf(F, (float)(slo - F.n) - 0.5f);
        float vacc = 0.0f;
        for (int s = slo; s <= shi; s++) {
            const float Fn = trap_cdf(F, (float)(s - F.n) + 0.5f);
            vacc = fmaf(Fn - Fp, __ldg(&row[s]), vacc);
            Fp = Fn;
        }
        acc = fmaf(F.amp, vacc, acc);
    }
    const bool inside = ix < G.nx && iy < G.ny;
    const size_t j = (size_t)iy * G.nx + ix;
    if (MODE == BP_PLAIN) {
        if (inside) xo[j] = accumulate ? fmaf(scale, acc, xo[j]) : scale * acc;
        return;
    }
    if (inside) {
        const float zeta = S.M_scale * acc;  // M grad L_m
        if (MODE == BP_SOLVE_INIT) {
            // zeta = g = M grad L_M(x); h = D_L x - zeta (Algorithm 2 keeps zeta in h)
            S.g[j] = zeta;
            S.h[j] = (S.algorithm == CT_ALG_PROPOSED) ? fmaf(S.d_l[j], S.x[j], -zeta) : zeta;
        } else {
            const float g = S.g[j];
            const float xp = S.x_new[j];
            const float a = S.alpha;
            const float ir = 1.0f / (rho + 1.0f);
            S.g[j] = fmaf(rho * ir, fmaf(a, zeta, (1.0f - a) * g), g * ir);
            if (S.algorithm == CT_ALG_PROPOSED)
                S.h[j] = fmaf(a, fmaf(S.d_l[j], xp, -zeta), (1.0f - a) * S.h[j]);
            else
                S.h[j] = zeta;
            S.x[j] = xp;
        }
    }
    if (MODE == BP_SOLVE_UPDATE) {
        // the last block to finish advances the subiteration counter (rho for the next one)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int done = atomicAdd(&S.counter[1], 1);
            if (done == (int)(gridDim.x * gridDim.y) - 1) {
                S.counter[1] = 0;
                S.counter[0] += 1;
                __threadfence();
            }
        }
    }
}

}  // namespace

cudaError_t launch_fp(const FanDev &G, int mode, const float *x, const int *views, int nviews, float *out,
                      const float *y, const float *w, cudaStream_t st)
{
    const long nrays = (long)nviews * G.ns;
    const long rays_per_block = kFpThreads / kFpSeg;
    const unsigned blocks = (unsigned)((nrays + rays_per_block - 1) / rays_per_block);
    if (blocks == 0) return cudaSuccess;
    switch (mode) {
    case FP_PLAIN: fp_fan2d_kernel<FP_PLAIN><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    case FP_RESID: fp_fan2d_kernel<FP_RESID><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    default: fp_fan2d_kernel<FP_ONES_W><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_bp(const FanDev &G, int mode, const float *sino, const int *views, int nviews, float *x,
                      float scale, int accumulate, const SolveDev *S, cudaStream_t st)
{
    dim3 grid(G.ntx, G.nty);
    SolveDev s0{};
    const SolveDev &SS = S ? *S : s0;
    switch (mode) {
    case BP_PLAIN: bp_fan2d_kernel<BP_PLAIN><<<grid, 256, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
    case BP_SOLVE_INIT: bp_fan2d_kernel<BP_SOLVE_INIT><<<grid, 256, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
    default: bp_fan2d_kernel<BP_SOLVE_UPDATE><<<grid, 256, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
    }
    return cudaGetLastError();
}

}  // namespace ct

// ---------------------------------------------------------------- C ABI

using namespace ct;

extern "C" ct_status ct_forward(const ct_geom *g, const float *x, float *y, const int *views, int nviews,
                                void *stream)
{
    if (!g || !x || !y) { set_error("ct_forward: null argument"); return CT_EINVAL; }
    ct_status st = validate_views(g, views, nviews);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int *dv = nullptr;
    if ((st = stage_views(g, views, nviews, &dv, s)) != CT_OK) return st;
    CT_CUDA_TRY(launch_fp(g->fan, FP_PLAIN, x, dv, nviews, y, nullptr, nullptr, s), "ct_forward launch");
    return CT_OK;
}

extern "C" ct_status ct_back(const ct_geom *g, const float *y, float *x, const int *views, int nviews, float scale,
                             int accumulate, void *stream)
{
    if (!g || !x || !y) { set_error("ct_back: null argument"); return CT_EINVAL; }
    ct_status st = validate_views(g, views, nviews);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int *dv = nullptr;
    if ((st = stage_views(g, views, nviews, &dv, s)) != CT_OK) return st;
    CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, y, dv, nviews, x, scale, accumulate, nullptr, s), "ct_back launch");
    return CT_OK;
}

extern "C" ct_status ct_sqs_diag(const ct_geom *g, const float *w, float *d_l, void *stream)
{
    if (!g || !w || !d_l) { set_error("ct_sqs_diag: null argument"); return CT_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    // q = w (A 1) over all views, then D_L = A' q
    CT_CUDA_TRY(launch_fp(g->fan, FP_ONES_W, nullptr, g->d_views_all, g->fan.na, g->d_sino_ws, nullptr, w, s),
                "ct_sqs_diag forward");
    CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, g->d_sino_ws, g->d_views_all, g->fan.na, d_l, 1.0f, 0, nullptr, s),
                "ct_sqs_diag back");
    return CT_OK;
}
