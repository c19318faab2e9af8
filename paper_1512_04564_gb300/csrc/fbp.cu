// Filtered back-projection for a full-scan equiangular fan beam: the initial
// image of Algorithm 1 ("an initial (FBP) image", Sec. III-A).  Textbook
// fan-beam FBP with equiangular rays (Kak & Slaney, Ch. 3):
//   p'(beta, gamma) = D cos(gamma) p(beta, gamma);
//   q = dgamma * (p' conv g), g(0) = 1/(8 dgamma^2), g(n dgamma) = 0 (even n),
//       -1 / (2 pi^2 sin^2(n dgamma)) (odd n), optionally Hann-apodised by the
//       3-tap [1/4, 1/2, 1/4] smoothing of g;
//   f(x, y) = dbeta sum_views q(beta, gamma'(x, y)) / L^2, linear interpolation in gamma.
// A helical scan (no helical FBP is given in the paper) is reconstructed slice by slice from its
// single-slice rebinning: for each slice the turn of views whose source heights are centred on it, from
// each view the detector row where the slice's height at the isocentre projects, then the fan-beam FBP.
#include <algorithm>
#include <cmath>

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
                                                              float *__restrict__ x, float dbeta, int v_first, int nv)
{
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31), iy = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (ix >= G.nx || iy >= G.ny) return;
    float acc = 0.0f;
    for (int v = v_first; v < v_first + nv; v++) {
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
        const float *row = q + (size_t)(v - v_first) * G.ns;
        const float v0 = ((unsigned)i0 < (unsigned)G.ns) ? __ldg(&row[i0]) : 0.0f;
        const float v1 = ((unsigned)(i0 + 1) < (unsigned)G.ns) ? __ldg(&row[i0 + 1]) : 0.0f;
        acc = fmaf(fmaf(f, v1 - v0, v0), __frcp_rn(fmaf(cpar, cpar, cperp * cperp)), acc);
    }
    x[(size_t)iy * G.nx + ix] = dbeta * acc;
}

// Single-slice rebinning of a helical scan for the slice at height zk (mm): row i of p is view v0 + i's
// detector row at the height where the slice's point at the isocentre projects, h = (zk - z_src) dsd /
// dso, interpolated linearly between the two nearest rows (clamped to the detector), times
// dsd / sqrt(dsd^2 + h_c^2) (the cosine of that row height's cone angle), which turns the oblique line
// integral into a transaxial one.  One CTA per view; its row parameters in FP64.
__global__ void __launch_bounds__(256) ssrb_kernel(int ns, int nt, int na, const float *__restrict__ y,
                                                   float *__restrict__ p, int v0, double zk, double beta0,
                                                   double dbeta, double beta_mid, double feed, double dsd, double dso,
                                                   double dt, double c_row)
{
    __shared__ int s_t0;
    __shared__ float s_f, s_c;
    const int i = blockIdx.x, v = v0 + i;
    if (threadIdx.x == 0) {
        const double zsrc = feed * (beta0 + v * dbeta - beta_mid) / (2.0 * 3.14159265358979323846);
        const double h = (zk - zsrc) * dsd / dso;
        const double tc = fmin(fmax(h / dt + c_row, 0.0), nt - 1.0);
        const int t0 = min((int)floor(tc), max(nt - 2, 0));
        const double hc = (tc - c_row) * dt;
        s_t0 = t0;
        s_f = (float)(tc - t0);
        s_c = (float)(dsd / sqrt(dsd * dsd + hc * hc));
    }
    __syncthreads();
    const float *r0 = y + ((size_t)v * nt + s_t0) * ns;
    const float f = s_f, c = s_c;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const float a = __ldg(&r0[s]);
        const float b = nt > 1 ? __ldg(&r0[s + ns]) : a;
        p[(size_t)i * ns + s] = c * fmaf(f, b - a, a);
    }
}

}  // namespace

// Views per turn of a helical scan, 0 unless it spans at least one turn with a whole number of views per turn.
static int views_per_turn(const ct_geom *g)
{
    const double turns = g->desc.orbit_deg / 360.0;
    const int na_turn = (int)std::lround(g->desc.na / turns);
    if (turns < 1.0 || std::fabs(na_turn * turns - g->desc.na) > 1e-9 * g->desc.na) return 0;
    return na_turn;
}

cudaError_t launch_fbp(const ct_geom *g, const float *y, float *x, int window, cudaStream_t st)
{
    const FanDev &G = g->fan;
    const size_t smem = sizeof(float) * (3 * (size_t)G.ns + 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fbp_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    const float dbeta = (float)(g->desc.orbit_deg * M_PI / 180.0 / g->desc.na);
    if (!g->helical) {
        fbp_filter_kernel<<<G.na, kFiltThreads, smem, st>>>(G, y, g->d_sino_ws, window);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        fbp_backproject_kernel<<<grid, 256, 0, st>>>(G, g->d_sino_ws, x, dbeta, 0, G.na);
        return cudaGetLastError();
    }
    // helical: per slice, single-slice rebinning of the turn of views whose source heights are centred on
    // it, then the fan-beam FBP of that turn into the slice ([nz][ny][nx] volume)
    const ct_geom_desc &d = g->desc;
    const int na_turn = views_per_turn(g), nz = g->hx.nz, nt = g->hx.nt;
    const double deg = M_PI / 180.0;
    const double beta0 = d.orbit_start_deg * deg, dbeta_d = d.orbit_deg * deg / d.na;
    const double beta_mid = (d.orbit_start_deg + 0.5 * d.orbit_deg) * deg;
    const double feed = d.pitch * d.nt * d.dt * d.dso / d.dsd;  // table feed per turn
    const double c_row = (d.nt - 1) / 2.0 - d.offset_t;
    float *pbuf = g->d_sino_ws, *qbuf = g->d_sino_ws + (size_t)na_turn * G.ns;
    for (int k = 0; k < nz; k++) {
        const double zk = (k - (nz - 1) / 2.0 + d.offset_z) * d.dz;
        int vc = 0;
        double best = INFINITY;
        for (int v = 0; v < d.na; v++) {  // the view whose source is nearest the slice (first of equals)
            const double dz = std::fabs(feed * (beta0 + v * dbeta_d - beta_mid) / (2.0 * M_PI) - zk);
            if (dz < best) { best = dz; vc = v; }
        }
        const int v0 = std::min(std::max(vc - na_turn / 2, 0), d.na - na_turn);
        ssrb_kernel<<<na_turn, 256, 0, st>>>(G.ns, nt, d.na, y, pbuf, v0, zk, beta0, dbeta_d, beta_mid, feed, d.dsd,
                                              d.dso, d.dt, c_row);
        fbp_filter_kernel<<<na_turn, kFiltThreads, smem, st>>>(G, pbuf, qbuf, window);
        fbp_backproject_kernel<<<grid, 256, 0, st>>>(G, qbuf, x + (size_t)k * G.nx * G.ny, dbeta, v0, na_turn);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

ct_status validate_fbp(const ct_geom *g, int window)
{
    if (window != CT_FBP_RAMP && window != CT_FBP_HANN) {
        set_error("unknown FBP window %d", window);
        return CT_EINVAL;
    }
    if (g->helical) {
        const int na_turn = views_per_turn(g);
        if (!na_turn) {
            set_error("helical FBP needs at least one turn with a whole number of views per turn");
            return CT_ENOTSUP;
        }
        if (2 * (size_t)na_turn > (size_t)g->desc.na * g->hx.nt) {  // the rebinned turn and its filtered copy
            set_error("helical FBP: the geometry's sinogram workspace cannot hold two rebinned turns");
            return CT_ENOTSUP;
        }
    } else if (std::fabs(g->desc.orbit_deg - 360.0) > 1e-9) {
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
