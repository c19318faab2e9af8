// Internal declarations of the CT library: geometry object, device footprint
// arithmetic shared by the forward and back projectors, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "../../include/ct.h"

namespace ct {

constexpr int kTile = 16;            // pixels per side of a back-projector tile (CTA) and record block
constexpr int kAnchor = 8;           // pixels per side of an anchor tile (FP64-derived reference point)
constexpr float kAnchorHalf = 3.5f;  // offset of an anchor tile's centre from its first pixel, in pixels

// Fan-beam geometry as the kernels see it (passed by value).
struct FanDev {
    int nx, ny, ns, na;
    int ntx, nty;             // 16x16 back-projector tiles along x and y
    int nax, nay;             // 8x8 anchor tiles along x and y
    float dx, dy, hx, hy;     // pixel size and half size (mm)
    float inv_dx, inv_dy;
    float inv_dg;             // detector cells per radian (dsd / ds)
    float dgamma;             // cell width in radians
    float gamma0;             // fan angle of cell 0's centre (rad)
    float dso;
    float x_edge0, y_edge0;   // x of the left edge of column 0, y of the lower edge of row 0 (mm)
    float cxo, cyo;           // (nx-1)/2 - offset_x, (ny-1)/2 - offset_y (pixel index of the origin)
    int max_span;             // upper bound on the detector cells one pixel footprint overlaps
    const float4 *anchor;     // [na][nay*nax][3]: the Anchor of each (view, 8x8 tile), FP64-derived: view-frame
                              // position of the tile centre relative to the source (t_par - dso, t_perp), its
                              // detector coordinate u = gamma/dgamma + (ns-1)/2 - offset_s as n + af + alo,
                              // and the derivatives of u and of e per pixel step (see point_u)
    const float2 *view_cs;    // [na]: (cos beta, sin beta)
    const float *view_beta;   // [na]: beta in [0, 2 pi)
    // resident system matrix (ct_geom_precompute); null when footprints are computed on the fly
    // Back-projector records in chunks of 32 pixel slots (see the layout at kRecGroup); null when
    // footprints are computed on the fly
    const unsigned char *rec_data;
    const unsigned int *rec_grp;  // [na][ntiles][8]: the chunk's start in 32-byte units (bits 0-27) and K (28-31)
    int bp_vs;                    // warps per record chunk of the back-projector, each on every bp_vs-th view
    const long long *row_ptr; // [na*ns + 1]: start of each ray's entry pairs (ray-major; the entries in march
                              // order, two per pair, a ray with an odd count padded by a zero entry)
    const float2 *row_w;      // [pairs]: a_ij of the pair's two entries
    const int *row_d;         // [pairs]: the two pixel indices as 16-bit offsets (low, high) from the first
                              // index of the pair's chunk (the ray's pairs in runs of 32 from its first)
    const int *row_first;     // [na*ns + 1]: first chunk of each ray in row_base
    const int *row_base;      // [chunks]: pixel index of each chunk's first entry
                              // Pixel indices of the rows address the packed image [x | x^T] (2 nx ny
                              // floats): a shallow ray's entries (marched column by column) index x,
                              // iy nx + ix; a steep ray's (marched row by row) index x^T, nx ny + ix ny + iy,
                              // so that consecutive entries of either kind are near each other in memory.
    float *xpack;             // [2 nx ny]: packing scratch of the forward projector (with the matrix)
    const int *ray_order;     // [ceil(ns/8)]: blocks of 8 adjacent cells, most entries first
    int fp_variant;           // forward projector chosen by ct_geom_autotune (FP_AUTO: default order)
    int bp_variant;           // back-projector chosen by ct_geom_autotune (BP_AUTO)
};

// Solver state shared by the kernels of one subiteration (device pointers).
struct SolveDev {
    float *x;        // canonical image x (caller's x_inout)
    float *x_new;    // x+ written by the update kernel
    float *g, *h;    // split-variable and dual recursions (Algorithm 2 keeps zeta in h)
    const float *d_l;
    float *resid;    // subset residual slab [views of subset][ns]
    const float *rho_tab;  // rho for subiteration t (0-based)
    int *counter;    // [0]: subiterations done; [1]: block-completion counter of the back-projector
    float alpha, M_scale;
    int algorithm;   // CT_ALG_*
    int nonneg;
    const float *kappa;  // regularizer voxel weights kappa_n (same layout as x), or nullptr for kappa = 1
};

// Axial part of a helical cone-beam geometry (the transaxial part is a FanDev
// whose views run over all turns).  Volumes inside the library are stored
// column-major, [iy][ix][iz] (z fastest); the C ABI's [iz][iy][ix] is
// transposed on entry and exit.
struct HelixDev {
    int nz, nt;
    float ct0;               // row coordinate of detector height 0: (nt-1)/2 - offset_t = ct0i - ofr
    float ct0i;              // (nt-1)/2 - round(offset_t): an integer or half-integer, exact in FP32
    float ofr;               // offset_t - round(offset_t), in [-1/2, 1/2]
    float kA, inv_kA;        // dz * dsd / dt (rows spanned by one voxel times its source distance), 1 / kA
    const float2 *view_zb;   // [na]: (z of the volume's lower face - z_src(view)) / dz = zbi + zbf, zbi integer
    const float *row_c;      // [nt]: 1 / cos(cone angle of row t) = sqrt(1 + (v_t / dsd)^2)
    const float4 *tile_ax;   // [na][nay*nax]: at each anchor tile's centre, voxels per row 1/a = L/kA and
                             // rows per voxel a = kA/L, each as hi + lo floats (FP64-derived)
    int trap;                // axial footprint: 0 rectangle (SF-TR), 1 trapezoid (SF-TT)
    float dso;               // source-to-isocentre distance (the FanDev's)
};

}  // namespace ct

// The opaque handle of the C ABI.
struct ct_geom {
    ct_geom_desc desc;
    ct::FanDev fan;
    int helical = 0;               // desc.kind == CT_HELICAL_CONE_ARC
    ct::HelixDev hx{};
    float2 *d_view_zb = nullptr;   // helical tables
    float *d_row_c = nullptr;
    float4 *d_tile_ax = nullptr;
    float *d_vol_ws = nullptr;     // helical: one column-major volume for the ABI's layout changes
    int hx_zc = 0;                 // helical: voxels per back-projector thread (chunk along z)
    float4 *d_anchor = nullptr;
    float2 *d_view_cs = nullptr;
    float *d_view_beta = nullptr;
    int *d_views_all = nullptr;   // identity list [0, na)
    int *d_views_stage = nullptr; // caller view lists are staged here [na]
    int *d_ray_order = nullptr;   // FanDev::ray_order
    float *d_a1 = nullptr;        // ray sums A 1 over all views [na][nt][ns] (raysum.cu), or null
    float *d_sino_ws = nullptr;   // [na][nt][ns] sinogram workspace (D_L; nt = 1 in 2-D)
    // solver workspace (allocated at the first solve)
    size_t solve_bytes = 0;
    void *d_solve = nullptr;
    double fov_radius = 0.0;
    // resident system matrix (ct_geom_precompute)
    long long *d_row_ptr = nullptr;
    float2 *d_row_w = nullptr;
    int *d_row_d = nullptr;
    int *d_row_first = nullptr;
    int *d_row_base = nullptr;
    unsigned char *d_rec_data = nullptr;
    unsigned int *d_rec_grp = nullptr;
    unsigned long long rec_bytes = 0;  // the records' share of matrix_bytes
    float *d_xpack = nullptr;     // FanDev::xpack
    unsigned long long matrix_bytes = 0;
    int device = 0;
};

namespace ct {

void set_error(const char *fmt, ...);
ct_status cuda_fail(cudaError_t e, const char *what);

#define CT_CUDA_TRY(expr, what)                                  \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return ::ct::cuda_fail(_e, what); \
    } while (0)

// ---------------------------------------------------------------- device arithmetic

// FP64-derived reference point of one (view, 8x8 pixel tile): the tile centre's view-frame position
// and detector coordinate, and the first-order change of the detector coordinate per pixel step.
struct Anchor {
    float ax, ay;              // (t_par - dso, t_perp) of the tile centre relative to the source (mm)
    float af, alo;             // its detector coordinate u_A = n + af + alo (af on the exact grid, see point_u)
    float kxh, kxl, kyh, kyl;  // du / d(pixel step along x), du / d(pixel step along y) at u_A: hi + lo
    float mx, my;              // (a . d) / |a|^2 per pixel step along x and y (a: the centre, d: the step)
    int n;
};

__device__ __forceinline__ Anchor load_anchor(const FanDev &G, int v, int atile)
{
    const float4 *p = G.anchor + 3 * ((size_t)v * (G.nax * G.nay) + atile);
    const float4 q0 = __ldg(p), q1 = __ldg(p + 1), q2 = __ldg(p + 2);
    Anchor A;
    A.ax = q0.x; A.ay = q0.y; A.af = q0.z; A.alo = q0.w;
    A.kxh = q1.x; A.kxl = q1.y; A.kyh = q1.z; A.kyl = q1.w;
    A.mx = q2.x; A.my = q2.y; A.n = __float_as_int(q2.z);
    return A;
}

// Detector coordinate of the point (px, py) pixel steps from the anchor tile's centre (px, py multiples
// of 1/2, |px|, |py| <= kAnchor / 2), returned as A.n + S + L.  The exact value is
//     u = u_A + atan(N / (1 + e)) / dgamma,
// N / dgamma = lin = kx px + ky py (the linear term, in cells), e = mx px + my py, so
//     u - u_A = lin - [lin e / (1 + e) + (z - atan z) / dgamma],   z = lin dgamma / (1 + e),
// with z - atan z = z^3/3 - z^5/5 + z^7/7 - ... (|z| <= ~0.1: the next term is below 3e-10 rad).
// The host rounds af and kxh, kyh onto a grid of 2^-p cells chosen so that S = af + kxh px + kyh py is
// exact in FP32 for every such point (and so are sums and differences of S values of one tile); the
// remainders kxl, kyl, alo and the nonlinear correction, all small, form L.  A footprint vertex is then
// (S - base) + L relative to an integer base cell: one FP32 rounding at the vertex's distance from it.
__device__ __forceinline__ void point_u(const FanDev &G, const Anchor &A, float px, float py, float &S, float &L)
{
    S = fmaf(A.kxh, px, fmaf(A.kyh, py, A.af));
    const float lo = fmaf(A.kxl, px, A.kyl * py);
    const float lin = (S - A.af) + lo;
    const float e = fmaf(A.mx, px, A.my * py);
    const float lr = lin * __fdividef(1.0f, 1.0f + e);
    const float z = lr * G.dgamma;
    const float z2 = z * z;
    const float c3 = lr * z2 * fmaf(z2, fmaf(z2, 1.0f / 7.0f, -0.2f), 1.0f / 3.0f);
    L = (A.alo + lo) - fmaf(lr, e, c3);
}

// Separable footprint of one pixel in one view: a unit-height trapezoid with
// sorted vertices t0..t3 in detector-cell units relative to cell n (cell n + j
// covers [j - 1/2, j + 1/2]), times the amplitude amp (chord through the
// pixel along the ray through its centre).
struct Footprint {
    float t0, t1, t2, t3;
    float amp;
    float w1, w3;      // t1 - t0, t3 - t2
    float i2w1, i2w3;  // 1/(2 w1) and 1/(2 w3), 0 for a vertical edge
    float m;           // (t1 + t2) / 2: integrals left of it are taken from t0, right of it from t3
    float area;        // w1/2 + (t2 - t1) + w3/2
    int n;
};

// Footprint from its four corner coordinates (S_k, L_k) (corners (-,-), (+,-), (-,+), (+,+) of the pixel),
// amplitude and the anchor's base cell.
__device__ __forceinline__ Footprint footprint_from_corners(const float (&S)[4], const float (&L)[4], float amp, int n_a)
{
    const float fl = floorf(0.5f * (S[0] + S[3]));
    float t[4];
#pragma unroll
    for (int k = 0; k < 4; k++) t[k] = (S[k] - fl) + L[k];
    const float a0 = fminf(t[0], t[1]), a1 = fmaxf(t[0], t[1]);
    const float b0 = fminf(t[2], t[3]), b1 = fmaxf(t[2], t[3]);
    Footprint F;
    F.t0 = fminf(a0, b0);
    F.t3 = fmaxf(a1, b1);
    const float m0 = fmaxf(a0, b0), m1 = fminf(a1, b1);
    F.t1 = fminf(m0, m1);
    F.t2 = fmaxf(m0, m1);
    F.w1 = F.t1 - F.t0;
    F.w3 = F.t3 - F.t2;
    F.i2w1 = F.w1 > 0.0f ? __fdividef(0.5f, F.w1) : 0.0f;
    F.i2w3 = F.w3 > 0.0f ? __fdividef(0.5f, F.w3) : 0.0f;
    F.m = 0.5f * (F.t1 + F.t2);
    F.area = fmaf(0.5f, F.w1 + F.w3, F.t2 - F.t1);
    F.amp = amp;
    F.n = n_a + (int)fl;
    return F;
}

// Chord through a pixel along the ray through its centre, |c| / max(|c_x| / dx, |c_y| / dy), c the
// centre relative to the source (view frame: cpar, cperp).
__device__ __forceinline__ float pixel_amplitude(const FanDev &G, float cb, float sb, float cpar, float cperp)
{
    const float r2 = fmaf(cpar, cpar, cperp * cperp);
    const float imx = fabsf(fmaf(cpar, cb, -cperp * sb)) * G.inv_dx;
    const float imy = fabsf(fmaf(cpar, sb, cperp * cb)) * G.inv_dy;
    return __fdividef(r2 * rsqrtf(r2), fmaxf(imx, imy));
}

// Footprint of the pixel whose centre is (px, py) pixel steps from the anchor tile's centre, in the view
// with direction (cb, sb).
__device__ __forceinline__ Footprint sf_footprint(const FanDev &G, float cb, float sb, const Anchor &A, float px, float py)
{
    float S[4], L[4];
#pragma unroll
    for (int k = 0; k < 4; k++) point_u(G, A, px + ((k & 1) ? 0.5f : -0.5f), py + ((k & 2) ? 0.5f : -0.5f), S[k], L[k]);
    const float ox = px * G.dx, oy = py * G.dy;
    const float cpar = G.dso + (A.ax + fmaf(ox, cb, oy * sb)), cperp = A.ay + fmaf(oy, cb, -ox * sb);
    return footprint_from_corners(S, L, pixel_amplitude(G, cb, sb, cpar, cperp), A.n);
}

// Signed tail of the unit trapezoid at u: left of the plateau's midpoint m, its integral over (-inf, u]
// (rising ramp a^2/(2 w1), a = clamp(u - t0, 0, w1), plus the plateau part); right of m, minus its
// integral over [u, inf) (the mirror image, from t3).  Both are small near the ends of the footprint,
// so a cell's weight (a difference of tails, plus the area for the cell holding m) keeps its relative
// precision however thin the sliver of footprint it takes.
__device__ __forceinline__ float trap_tail(const Footprint &F, float u)
{
    const bool left = u <= F.m;
    const float x = left ? u - F.t0 : F.t3 - u;
    const float y = left ? u - F.t1 : F.t2 - u;
    const float w = left ? F.w1 : F.w3;
    const float iw = left ? F.i2w1 : F.i2w3;
    const float a = fminf(fmaxf(x, 0.0f), w);
    const float h = fmaf(a * a, iw, fmaxf(y, 0.0f));
    return left ? h : -h;
}

// First and last cell (relative to n) the footprint overlaps, and the cell holding m.
__device__ __forceinline__ int foot_first(const Footprint &F) { return (int)floorf(F.t0 - 0.5f) + 1; }
__device__ __forceinline__ int foot_last(const Footprint &F) { return (int)ceilf(F.t3 + 0.5f) - 1; }
__device__ __forceinline__ int foot_mid(const Footprint &F) { return (int)floorf(F.m + 0.5f); }

// Unit-amplitude integral of the footprint over relative cell j, given the tails at its lower and upper
// edges: hi - lo, plus the area for the cell holding m.
__device__ __forceinline__ float cell_integral(const Footprint &F, int j, float h_lo, float h_hi)
{
    return (h_hi - h_lo) + (j == foot_mid(F) ? F.area : 0.0f);
}

// Unit-amplitude integrals of the footprint over its cells j0 = foot_first(F), j0 + 1, ... (at most maxc):
// emit(i, value) for cell j0 + i.  Returns the number of cells.
template <class Emit>
__device__ __forceinline__ int foot_cells(const Footprint &F, int maxc, Emit &&emit)
{
    const int j0 = foot_first(F);
    const int cnt = max(min(foot_last(F) + 1 - j0, maxc), 0);
    const int jm = foot_mid(F);
    float hp = 0.0f;  // the tail is 0 at the first cell's lower edge
    for (int i = 0; i < cnt; i++) {
        const float hn = trap_tail(F, (float)(j0 + i) + 0.5f);
        emit(i, (hn - hp) + (j0 + i == jm ? F.area : 0.0f));
        hp = hn;
    }
    return cnt;
}

// sum_s a_s r_s over the cells of one footprint (row = detector row of one view), by summation by parts
// over the cell edges: the tail is 0 at the first cell's lower edge and the last cell's upper edge, so
// only interior edges are evaluated, plus the area times the residual of the cell holding m.  Cells
// outside [0, ns) read as 0.  COHERENT loads bypass L1 (rows rewritten by other CTAs of a persistent
// kernel).
template <bool COHERENT>
__device__ __forceinline__ float footprint_dot_t(const Footprint &F, const float *row, int ns)
{
    const int j0 = foot_first(F), jl = foot_last(F);
    int s = F.n + j0;
    auto ld = [&](int c) { return ((unsigned)c < (unsigned)ns) ? (COHERENT ? __ldcg(&row[c]) : __ldg(&row[c])) : 0.0f; };
    float rp = ld(s);
    float acc = 0.0f;
    for (int j = j0; j < jl; j++) {
        s++;
        const float rn = ld(s);
        acc = fmaf(trap_tail(F, (float)j + 0.5f), rp - rn, acc);
        rp = rn;
    }
    return F.amp * fmaf(F.area, ld(F.n + foot_mid(F)), acc);
}

__device__ __forceinline__ float footprint_dot(const Footprint &F, const float *__restrict__ row, int ns)
{
    return footprint_dot_t<false>(F, row, ns);
}

// Anchor of pixel (ix, iy) in view v, and the pixel centre's offset from the anchor tile's centre in
// pixel steps (px, py: half-integers).  Small anchor tiles keep the offsets, and with them the FP32
// corrections of the footprint's position, small.
__device__ __forceinline__ Anchor pixel_anchor(const FanDev &G, int v, int ix, int iy, float &px, float &py)
{
    const int ax = ix / kAnchor, ay = iy / kAnchor;
    px = (float)(ix - ax * kAnchor) - kAnchorHalf;
    py = (float)(iy - ay * kAnchor) - kAnchorHalf;
    return load_anchor(G, v, ay * G.nax + ax);
}

// Footprint of pixel (ix, iy) in view v (loads its anchor).
__device__ __forceinline__ Footprint pixel_footprint(const FanDev &G, int v, float cb, float sb, int ix, int iy)
{
    float px, py;
    const Anchor A = pixel_anchor(G, v, ix, iy, px, py);
    return sf_footprint(G, cb, sb, A, px, py);
}

// Weight a_ij of pixel footprint F in detector cell s.
__device__ __forceinline__ float cell_weight(const Footprint &F, int s)
{
    const int j = s - F.n;
    return F.amp * cell_integral(F, j, trap_tail(F, (float)j - 0.5f), trap_tail(F, (float)j + 0.5f));
}

constexpr float kRangePad = 0.02f;  // pixels of padding on a wedge's row/column range

// Whether ray (v, s) is steep (|sin phi| > |cos phi|): ray_visit then marches it row by row, else
// column by column.  The same arithmetic as ray_visit's test.
__device__ __forceinline__ bool ray_steep(const FanDev &G, int v, int s)
{
    const float phi = __ldg(&G.view_beta[v]) + fmaf((float)s, G.dgamma, G.gamma0);
    float sp, cp;
    sincosf(phi, &sp, &cp);
    return !(fabsf(cp) >= fabsf(sp));
}

// Visit the pixels whose squares can meet the fan wedge of cell s in view v:
// shallow rays march the columns (steep rays the rows) in [seg/nseg, (seg+1)/nseg)
// of the image and visit, in each, the rows (columns) between the wedge's two
// edge lines (padded by kRangePad pixels).  visit(ix, iy) is called in march order.
template <class Visit>
__device__ __forceinline__ void ray_visit(const FanDev &G, int v, int s, int seg, int nseg, Visit &&visit)
{
    const float2 cs = __ldg(&G.view_cs[v]);
    const float beta = __ldg(&G.view_beta[v]);
    const float phi = beta + fmaf((float)s, G.dgamma, G.gamma0);
    float sp, cp;
    sincosf(phi, &sp, &cp);
    const float Sx = -G.dso * cs.x, Sy = -G.dso * cs.y;
    const float phl = phi - 0.5f * G.dgamma, phh = phi + 0.5f * G.dgamma;
    if (fabsf(cp) >= fabsf(sp)) {
        // shallow ray: the wedge's edges are y = Sy + (x - Sx) tan(phi -+ dgamma/2)
        const float tl = tanf(phl), th = tanf(phh);
        const int c0 = seg * G.nx / nseg, c1 = (seg + 1) * G.nx / nseg;
        for (int ix = c0; ix < c1; ix++) {
            const float xl = fmaf((float)ix, G.dx, G.x_edge0) - Sx, xr = xl + G.dx;
            const float y1 = fmaf(xl, tl, Sy), y2 = fmaf(xr, tl, Sy);
            const float y3 = fmaf(xl, th, Sy), y4 = fmaf(xr, th, Sy);
            const float ylo = (fminf(fminf(y1, y2), fminf(y3, y4)) - G.y_edge0) * G.inv_dy - kRangePad;
            const float yhi = (fmaxf(fmaxf(y1, y2), fmaxf(y3, y4)) - G.y_edge0) * G.inv_dy + kRangePad;
            const int iy0 = max(0, (int)floorf(fmaxf(ylo, -1.0f)));
            const int iy1 = min(G.ny - 1, (int)floorf(fminf(yhi, (float)G.ny)));
            for (int iy = iy0; iy <= iy1; iy++) visit(ix, iy);
        }
    } else {
        // steep ray: x = Sx + (y - Sy) cot(phi -+ dgamma/2)
        const float tl = cosf(phl) / sinf(phl), th = cosf(phh) / sinf(phh);
        const int r0 = seg * G.ny / nseg, r1 = (seg + 1) * G.ny / nseg;
        for (int iy = r0; iy < r1; iy++) {
            const float yb = fmaf((float)iy, G.dy, G.y_edge0) - Sy, yt = yb + G.dy;
            const float x1 = fmaf(yb, tl, Sx), x2 = fmaf(yt, tl, Sx);
            const float x3 = fmaf(yb, th, Sx), x4 = fmaf(yt, th, Sx);
            const float xlo = (fminf(fminf(x1, x2), fminf(x3, x4)) - G.x_edge0) * G.inv_dx - kRangePad;
            const float xhi = (fmaxf(fmaxf(x1, x2), fmaxf(x3, x4)) - G.x_edge0) * G.inv_dx + kRangePad;
            const int ix0 = max(0, (int)floorf(fmaxf(xlo, -1.0f)));
            const int ix1 = min(G.nx - 1, (int)floorf(fminf(xhi, (float)G.nx)));
            for (int ix = ix0; ix <= ix1; ix++) visit(ix, iy);
        }
    }
}

// One ray of the resident matrix, warp-cooperative (all 32 lanes call it with the same range):
// sum of a_ij x_j over the entry pairs [b, e).  Lane l takes pairs b + l + 32 c, so each warp load
// covers one chunk of the ray: one 8-byte load of two weights, one 4-byte load of two 16-bit offsets,
// and the chunk's base pixel index (a broadcast load); two pairs are in flight per lane.  chunk0: the
// ray's first chunk in row_base.  x: the packed image [x | x^T] the row indices address.  ONES: sum of
// a_ij (x = 1).  COHERENT: x read with L1-bypassing loads.
template <bool ONES, bool COHERENT>
__device__ __forceinline__ float csr_ray_dot(const FanDev &G, long long b, long long e, int chunk0,
                                             const float *__restrict__ x, int lane)
{
    constexpr int U = 2;  // pairs in flight per lane (four: 40 registers, fewer warps, slower)
    float acc[2 * U];
#pragma unroll
    for (int q = 0; q < 2 * U; q++) acc[q] = 0.0f;
    int c = chunk0;
    for (long long c0 = b; c0 < e; c0 += 32 * U, c += U) {
        float2 w[U];
        int p[2 * U];
        bool ok[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
            const long long i = c0 + 32 * q + lane;
            ok[q] = i < e;
            w[q] = ok[q] ? __ldcs(&G.row_w[i]) : make_float2(0.0f, 0.0f);
            if (!ONES) {
                const int d = ok[q] ? __ldcs(&G.row_d[i]) : 0;
                const int base = ok[q] ? __ldg(&G.row_base[c + q]) : 0;
                p[2 * q] = base + (int)(short)(d & 0xffff);
                p[2 * q + 1] = base + (d >> 16);
            }
        }
        if (ONES) {
#pragma unroll
            for (int q = 0; q < U; q++) {
                acc[2 * q] += w[q].x;
                acc[2 * q + 1] += w[q].y;
            }
            continue;
        }
        float xv[2 * U];  // all gathers issued before the multiply-adds
#pragma unroll
        for (int q = 0; q < 2 * U; q++) xv[q] = ok[q >> 1] ? (COHERENT ? __ldcg(&x[p[q]]) : __ldg(&x[p[q]])) : 0.0f;
#pragma unroll
        for (int q = 0; q < U; q++) {
            acc[2 * q] = fmaf(w[q].x, xv[2 * q], acc[2 * q]);
            acc[2 * q + 1] = fmaf(w[q].y, xv[2 * q + 1], acc[2 * q + 1]);
        }
    }
    float t = 0.0f;
#pragma unroll
    for (int q = 0; q < 2 * U; q++) t += acc[q];
    return t;
}

// Second half of the packed image [x | x^T] for one block of 32 columns x 8 rows (block (blockIdx.x,
// blockIdx.y), 256 threads), whose values the block has staged in t[row][column]: thread i writes column
// 32 bx + i / 8, rows 8 by .. 8 by + 7 of the block going to consecutive addresses of x^T.  With rows of
// 36 floats both the staging and this read are free of shared-memory bank conflicts.
__device__ __forceinline__ void write_transposed_block(const FanDev &G, const float (*t)[36], float *xp)
{
    const int c = threadIdx.x >> 3, r = threadIdx.x & 7;
    const int ix = blockIdx.x * 32 + c, iy = blockIdx.y * 8 + r;
    if (ix < G.nx && iy < G.ny) xp[(size_t)G.nx * G.ny + (size_t)ix * G.ny + iy] = t[r][c];
}

// ---------------------------------------------------------------- launchers (projectors.cu)

enum FpMode { FP_PLAIN = 0, FP_RESID = 1, FP_ONES_W = 2 };
enum FpVariant { FP_AUTO = 0, FP_VAR_CSR = 1, FP_VAR_BUNDLE = 2, FP_VAR_RAY = 3 };
enum BpVariant { BP_AUTO = 0, BP_VAR_STORED = 1, BP_VAR_FLY = 2 };
enum BpMode { BP_PLAIN = 0, BP_SOLVE_INIT = 1, BP_SOLVE_UPDATE = 2 };

// out rows follow `views` (device list of nviews view indices).  With the resident rows the forward
// projector reads the packed image [x | x^T]: xpack, if the caller has it (e.g. written by the update
// kernel), else x is packed into G.xpack first.
cudaError_t launch_fp(const FanDev &G, int mode, const float *x, const int *views, int nviews, float *out,
                      const float *y, const float *w, cudaStream_t st, const float *xpack = nullptr);
// [x | x^T] of an nx x ny image into xp (2 nx ny floats).
cudaError_t launch_pack(const FanDev &G, const float *x, float *xp, cudaStream_t st);
cudaError_t launch_bp(const FanDev &G, int mode, const float *sino, const int *views, int nviews, float *x,
                      float scale, int accumulate, const SolveDev *S, cudaStream_t st);
cudaError_t launch_reg_gradient(const FanDev &G, const float *x, const float *kappa, float beta, float delta,
                                int potential, float *grad, float *curv, cudaStream_t st);
cudaError_t launch_reg_update(const FanDev &G, const SolveDev &S, float beta, float delta, int potential,
                              int maxcurv, cudaStream_t st);

cudaError_t build_matrix(ct_geom *g, unsigned long long max_bytes, cudaStream_t st, bool *too_big);
// Ray sums A 1 of the geometry (raysum.cu): computed once and kept in g->d_a1; dropped when the
// projector path changes (ct_geom_precompute, ct_geom_autotune).
cudaError_t ensure_ray_sums(ct_geom *g, cudaStream_t st);
void drop_ray_sums(ct_geom *g);
cudaError_t launch_weighted_ray_sums(const ct_geom *g, const float *w, float *out, cudaStream_t st);  // w (A 1)
cudaError_t launch_fbp(const ct_geom *g, const float *y, float *x, int window, cudaStream_t st);
ct_status validate_fbp(const ct_geom *g, int window);

ct_status validate_views(const ct_geom *g, const int *views, int nviews);

// helical cone-beam (helical.cu); volumes column-major [iy][ix][iz]
cudaError_t launch_fp_helix(const ct_geom *g, int mode, const float *x, const int *views, int nviews, float *out,
                            const float *y, const float *w, cudaStream_t st);
cudaError_t launch_bp_helix(const ct_geom *g, int mode, const float *sino, const int *views, int nviews, float *x,
                            float scale, int accumulate, const SolveDev *S, cudaStream_t st);
cudaError_t launch_reg_gradient_helix(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                                      int potential, float *grad, float *curv, cudaStream_t st);
cudaError_t launch_reg_update_helix(const ct_geom *g, const SolveDev &S, float beta, float delta, int potential,
                                    int maxcurv, cudaStream_t st);
cudaError_t launch_rmsd_helix(const ct_geom *g, const float *x, const float *xr, float r2max, double *partial,
                              int *counter, float *trace, int M, float hu, cudaStream_t st);
// largest chunk whose magnified extent (plus extra_rows) fits the row buffer, 0 if none
int helix_chunk_voxels(double a_max, double extra_rows);
int helix_max_rows();
int helix_max_span();
int helix_max_march();
// [iz][iy][ix] -> column-major, and back (dst = scale * src (+ dst if accumulate))
cudaError_t launch_to_columns(const ct_geom *g, const float *src, float *dst, cudaStream_t st);
cudaError_t launch_to_slices(const ct_geom *g, const float *src, float *dst, float scale, int accumulate,
                             cudaStream_t st);
ct_status helix_forward(const ct_geom *g, const float *x, float *y, const int *views, int nviews, cudaStream_t st);
ct_status helix_back(const ct_geom *g, const float *y, float *x, const int *views, int nviews, float scale,
                     int accumulate, cudaStream_t st);
ct_status helix_sqs_diag(const ct_geom *g, const float *w, float *d_l, cudaStream_t st);
ct_status helix_reg_gradient(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                             int potential, float *grad, float *curv, cudaStream_t st);
ct_status stage_views(const ct_geom *g, const int *views, int nviews, const int **dev_views, cudaStream_t st);

// ---------------------------------------------------------------- stored cell-weight records (resident matrix)

// A record is the weights a_ij of one (view, pixel) footprint's cells, clipped to the detector: n0 the
// first cell, cnt <= 15 cells.  The records of 32 consecutive pixel slots of a 16x16 tile (one warp of the
// back-projectors; slots in tile order, 8 groups a tile) and one view form a chunk of 64 + 128 K bytes,
// K the group's largest cnt:
//   bytes 0 - 63   each slot's n0 (bits 0-11) and cnt (bits 12-15), u16
//   bytes 64 -     weight i of slot l at float 32 i + l (i < K; zero for i >= the slot's cnt)
// so that the warp reads weight i of all 32 slots with one coalesced 128-byte load, and every address
// follows from the group's word (chunk start and K) alone.
constexpr int kRecGroup = 32;
constexpr int kRecMaxCells = 15;
constexpr int kRecInline = 5;  // weights a lane holds in registers (a footprint covers 2 - 5 cells, rarely more)

// One slot's record of one view, its first kRecInline weights loaded.
struct RecSlot {
    unsigned nc;  // first cell (bits 0-11) and count (12-15)
    float w[kRecInline];
};

__device__ __forceinline__ const float *rec_weights(const FanDev &G, unsigned word)
{
    return reinterpret_cast<const float *>(G.rec_data + 32 * (size_t)(word & 0x0fffffffu) + 64) + (threadIdx.x & 31);
}

// The record of this lane's slot in the chunk of group word `word` (every lane of the warp calls it: the
// loads of weights i < K are warp-uniform).
__device__ __forceinline__ RecSlot rec_fetch(const FanDev &G, unsigned word)
{
    const int K = (int)(word >> 28), lane = threadIdx.x & 31;
    const unsigned char *c = G.rec_data + 32 * (size_t)(word & 0x0fffffffu);
    const float *wp = reinterpret_cast<const float *>(c + 64) + lane;
    RecSlot r;
    r.nc = __ldcs(reinterpret_cast<const unsigned short *>(c) + lane);
#pragma unroll
    for (int i = 0; i < kRecInline; i++) r.w[i] = i < K ? __ldcs(wp + 32 * i) : 0.0f;
    return r;
}

// sum_k a_k row[n0 + k] over one record; word() gives the chunk's word again for the rare records wider
// than kRecInline cells.  COHERENT loads of the row bypass L1 (rows rewritten by other CTAs of a
// persistent kernel).
template <bool COHERENT = false, class Word>
__device__ __forceinline__ float rec_dot(const FanDev &G, const RecSlot &r, const float *rows, Word word)
{
    const int cnt = (int)(r.nc >> 12);
    const float *row = rows + (r.nc & 0xfffu);
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < kRecInline; i++)
        if (i < cnt) acc = fmaf(r.w[i], COHERENT ? __ldcg(&row[i]) : __ldg(&row[i]), acc);
    if (cnt > kRecInline) {
        const float *wp = rec_weights(G, word());
#pragma unroll 1
        for (int i = kRecInline; i < cnt; i++)
            acc = fmaf(__ldcs(wp + 32 * i), COHERENT ? __ldcg(&row[i]) : __ldg(&row[i]), acc);
    }
    return acc;
}

// Word of group `group` (tile * 8 + warp of the tile) of view v.
__device__ __forceinline__ unsigned rec_word(const FanDev &G, int v, unsigned group)
{
    return __ldg(&G.rec_grp[(size_t)v * ((size_t)G.ntx * G.nty * 8) + group]);
}

// ---------------------------------------------------------------- regularizer (Eq. (def_reg))

struct Pot {
    int kind;
    float inv_delta;
    int maxcurv;  // 1: the SQS curvature is the potential's maximum curvature (1) instead of Huber's omega(t)
    // phi'(t) and omega(t) = phi'(t)/t
    __device__ __forceinline__ void eval(float t, float &dphi, float &omega) const
    {
        if (kind == CT_POT_HYPERBOLA) {
            const float q = t * inv_delta;
            omega = rsqrtf(fmaf(q, q, 1.0f));
        } else if (kind == CT_POT_FAIR) {
            omega = 1.0f / fmaf(fabsf(t), inv_delta, 1.0f);
        } else {
            omega = 1.0f;
        }
        dphi = t * omega;
    }
};

// COHERENT loads bypass L1 and the read-only path: needed when x is rewritten
// by other CTAs of the same (persistent) kernel.
template <bool COHERENT = false>
__device__ __forceinline__ float ld_img(const float *p)
{
    return COHERENT ? __ldcg(p) : __ldg(p);
}

// grad R_j and the SQS diagonal D_R,j of Eq. (def_reg) at pixel (ix, iy):
//   grad R_j = kappa_j sum_i beta_i [kappa_{j+s_i} phi'(x_j - x_{j+s_i}) - kappa_{j-s_i} phi'(x_{j-s_i} - x_j)]
//   D_R,j    = kappa_j sum_i 2 beta_i [kappa_{j+s_i} omega(.) + kappa_{j-s_i} omega(.)]
// (KAPPA = false: kappa = 1, and the kappa pointer is not read).
template <bool COHERENT = false, bool KAPPA = false>
__device__ __forceinline__ void reg_terms(const FanDev &G, const float *__restrict__ x, int ix, int iy, float beta,
                                          Pot P, float &grad, float &curv, const float *__restrict__ kappa = nullptr)
{
    const size_t j = (size_t)iy * G.nx + ix;
    const float xj = ld_img<COHERENT>(&x[j]);
    const int ddx[4] = {1, 0, 1, 1};
    const int ddy[4] = {0, 1, 1, -1};
    const float bd = beta * 0.70710678118654752f;
    grad = 0.0f;
    curv = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float bi = (i < 2) ? beta : bd;
        const int fx = ix + ddx[i], fy = iy + ddy[i];
        if (fx >= 0 && fx < G.nx && fy >= 0 && fy < G.ny) {
            const size_t f = (size_t)fy * G.nx + fx;
            const float bk = KAPPA ? bi * ld_img<COHERENT>(&kappa[f]) : bi;
            float d, o;
            P.eval(xj - ld_img<COHERENT>(&x[f]), d, o);
            grad = fmaf(bk, d, grad);
            curv = fmaf(2.0f * bk, P.maxcurv ? 1.0f : o, curv);
        }
        const int bx = ix - ddx[i], by = iy - ddy[i];
        if (bx >= 0 && bx < G.nx && by >= 0 && by < G.ny) {
            const size_t b = (size_t)by * G.nx + bx;
            const float bk = KAPPA ? bi * ld_img<COHERENT>(&kappa[b]) : bi;
            float d, o;
            P.eval(ld_img<COHERENT>(&x[b]) - xj, d, o);
            grad = fmaf(-bk, d, grad);
            curv = fmaf(2.0f * bk, P.maxcurv ? 1.0f : o, curv);
        }
    }
    if (KAPPA) {
        const float kj = ld_img<COHERENT>(&kappa[j]);
        grad *= kj;
        curv *= kj;
    }
}

// footprint_dot with L1-bypassing loads of the detector row (rows rewritten by
// other CTAs of a persistent kernel); same arithmetic.
__device__ __forceinline__ float footprint_dot_coherent(const Footprint &F, const float *row, int ns)
{
    return footprint_dot_t<true>(F, row, ns);
}

}  // namespace ct
