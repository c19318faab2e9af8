// Geometry object of the C ABI: validation, FP64-derived device tables, error state.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ct_internal.cuh"

namespace ct {

// f(lo, hi, worker) over [0, n) split into contiguous ranges, one per host thread (up to 16); every
// element is computed as in a single-threaded loop, so the tables do not depend on the thread count.
template <class F>
static void host_parallel_for(int n, F f)
{
    const unsigned hc = std::thread::hardware_concurrency();
    const int nw = std::max(1, std::min({(int)(hc ? hc : 1), 16, (n + 7) / 8}));
    if (nw == 1) {
        f(0, n, 0);
        return;
    }
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; w++) {
        const int lo = (int)((long long)n * w / nw), hi = (int)((long long)n * (w + 1) / nw);
        pool.emplace_back([=] { f(lo, hi, w); });
    }
    for (auto &t : pool) t.join();
}

namespace {

// Anchor tables in FP64 on the device, one thread per (view, 8x8 anchor tile): u at the tile centre and its
// derivatives per pixel step.  For a tile centre a (relative to the source, view frame) and a step
// d = R(beta) (px dx, py dy), the fan angle changes by atan(N / (1 + e)), N = cross(a, d) / |a|^2,
// e = a.d / |a|^2, both linear in (px, py).  The views' cos and sin come from the host.
struct AnchorParams {
    int na, nax, nay;
    double cxo, cyo, dx, dy, dso, inv_dg, c0;
    float dso_f;  // the kernels' FP32 dso
};

struct TileGeo {
    double tpar, tperp, u, kx, ky, mx, my;
};

__device__ TileGeo tile_geo(const AnchorParams &P, double cb, double sb, int tx, int ty)
{
    const double X = (tx * kAnchor + (double)kAnchorHalf - P.cxo) * P.dx;
    const double Y = (ty * kAnchor + (double)kAnchorHalf - P.cyo) * P.dy;
    TileGeo t;
    t.tpar = P.dso + X * cb + Y * sb;
    t.tperp = -X * sb + Y * cb;
    const double a2 = t.tpar * t.tpar + t.tperp * t.tperp;
    t.u = atan2(t.tperp, t.tpar) * P.inv_dg + P.c0;
    // a step along x: d = dx (cb, -sb) in the view frame; along y: d = dy (sb, cb)
    t.kx = (t.tpar * (-P.dx * sb) - t.tperp * (P.dx * cb)) / a2 * P.inv_dg;
    t.ky = (t.tpar * (P.dy * cb) - t.tperp * (P.dy * sb)) / a2 * P.inv_dg;
    t.mx = (t.tpar * (P.dx * cb) + t.tperp * (-P.dx * sb)) / a2;
    t.my = (t.tpar * (P.dy * sb) + t.tperp * (P.dy * cb)) / a2;
    return t;
}

// max over (view, tile) of |kx| + |ky| (non-negative doubles order as their bit patterns)
__global__ void __launch_bounds__(256) anchor_kmax_kernel(AnchorParams P, const double2 *__restrict__ vcs,
                                                          unsigned long long *kmax)
{
    const long long n = (long long)P.na * P.nax * P.nay;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double km = 0.0;
    if (i < n) {
        const int nt = P.nax * P.nay, v = (int)(i / nt), tile = (int)(i - (long long)v * nt);
        const double2 c = vcs[v];
        const TileGeo t = tile_geo(P, c.x, c.y, tile % P.nax, tile / P.nax);
        km = fabs(t.kx) + fabs(t.ky);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) km = fmax(km, __shfl_xor_sync(0xffffffffu, km, o));
    if ((threadIdx.x & 31) == 0) atomicMax(kmax, (unsigned long long)__double_as_longlong(km));
}

// the anchors, with af and kxh, kyh rounded onto the grid of 1/qa and 1/qk cells
__global__ void __launch_bounds__(256) anchor_fill_kernel(AnchorParams P, const double2 *__restrict__ vcs, double qk,
                                                          double qa, float4 *__restrict__ anc)
{
    const long long n = (long long)P.na * P.nax * P.nay;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nt = P.nax * P.nay, v = (int)(i / nt), tile = (int)(i - (long long)v * nt);
    const double2 c = vcs[v];
    const TileGeo t = tile_geo(P, c.x, c.y, tile % P.nax, tile / P.nax);
    const double kxh = rint(t.kx * qk) / qk, kyh = rint(t.ky * qk) / qk;
    const double nn = floor(t.u), fr = t.u - nn;
    const double af = rint(fr * qa) / qa;
    float4 *q = anc + 3 * i;
    // t_par as dso (the kernels' float) + a small float
    q[0] = make_float4((float)(t.tpar - (double)P.dso_f), (float)t.tperp, (float)af, (float)(fr - af));
    q[1] = make_float4((float)kxh, (float)(t.kx - kxh), (float)kyh, (float)(t.ky - kyh));
    q[2] = make_float4((float)t.mx, (float)t.my, __int_as_float((int)nn), 0.0f);  // the base cell, as int bits
}

}  // namespace

namespace {
thread_local std::string g_last_error;
}

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

ct_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CT_ENOMEM : CT_ECUDA;
}

ct_status validate_views(const ct_geom *g, const int *views, int nviews)
{
    if (nviews < 1 || nviews > g->fan.na) {
        set_error("nviews=%d must be in [1, na=%d]", nviews, g->fan.na);
        return CT_EINVAL;
    }
    if (!views) {
        if (nviews != g->fan.na) {
            set_error("views == NULL selects all %d views, but nviews=%d", g->fan.na, nviews);
            return CT_EINVAL;
        }
        return CT_OK;
    }
    for (int k = 0; k < nviews; k++) {
        if (views[k] < 0 || views[k] >= g->fan.na) {
            set_error("views[%d]=%d outside [0, %d)", k, views[k], g->fan.na);
            return CT_EINVAL;
        }
    }
    return CT_OK;
}

ct_status stage_views(const ct_geom *g, const int *views, int nviews, const int **dev_views, cudaStream_t st)
{
    if (!views) {
        *dev_views = g->d_views_all;
        return CT_OK;
    }
    CT_CUDA_TRY(cudaMemcpyAsync(g->d_views_stage, views, sizeof(int) * nviews, cudaMemcpyHostToDevice, st),
                "staging view list");
    *dev_views = g->d_views_stage;
    return CT_OK;
}

}  // namespace ct

using namespace ct;

static void free_geom(ct_geom *g)
{
    if (!g) return;
    cudaFree(g->d_anchor);
    cudaFree(g->d_view_cs);
    cudaFree(g->d_view_beta);
    cudaFree(g->d_views_all);
    cudaFree(g->d_views_stage);
    cudaFree(g->d_sino_ws);
    cudaFree(g->d_solve);
    cudaFree(g->d_row_ptr);
    cudaFree(g->d_row_w);
    cudaFree(g->d_row_d);
    cudaFree(g->d_row_first);
    cudaFree(g->d_row_base);
    cudaFree(g->d_rec_data);
    cudaFree(g->d_rec_grp);
    cudaFree(g->d_xpack);
    cudaFree(g->d_view_zb);
    cudaFree(g->d_row_c);
    cudaFree(g->d_tile_ax);
    cudaFree(g->d_vol_ws);
    cudaFree(g->d_a1);
    cudaFree(g->d_ray_order);
    delete g;
}

extern "C" ct_status ct_geom_create(const ct_geom_desc *d, ct_geom **out)
{
    if (!d || !out) { set_error("ct_geom_create: null argument"); return CT_EINVAL; }
    *out = nullptr;
    const bool helical = d->kind == CT_HELICAL_CONE_ARC;
    if (d->kind != CT_FAN_ARC_2D && !helical) {
        set_error("geometry kind %d is not supported (CT_FAN_ARC_2D=%d, CT_HELICAL_CONE_ARC=%d)", d->kind,
                  CT_FAN_ARC_2D, CT_HELICAL_CONE_ARC);
        return CT_ENOTSUP;
    }
    if (helical) {
        if (d->nz < 1 || d->nt < 1 || d->nz > 4096 || !(d->dz > 0) || !(d->dt > 0) || !std::isfinite(d->pitch) ||
            !std::isfinite(d->offset_z) || !std::isfinite(d->offset_t)) {
            set_error("bad helical sizes nz=%d nt=%d or lengths", d->nz, d->nt);
            return CT_EINVAL;
        }
        if (d->nt > helix_max_rows() || d->nx > helix_max_march() || d->ny > helix_max_march()) {
            set_error("helical scans support up to %d detector rows and %d pixels per side", helix_max_rows(),
                      helix_max_march());
            return CT_ENOTSUP;
        }
    }
    if (d->nx < 1 || d->ny < 1 || d->ns < 1 || d->na < 1 || d->nx > 65536 || d->ny > 65536 || d->ns > (1 << 20) ||
        d->na > (1 << 20)) {
        set_error("bad sizes nx=%d ny=%d ns=%d na=%d", d->nx, d->ny, d->ns, d->na);
        return CT_EINVAL;
    }
    if (!(d->dx > 0) || !(d->dy > 0) || !(d->ds > 0) || !(d->dso > 0) || !(d->dsd > 0) || !std::isfinite(d->orbit_deg) ||
        !std::isfinite(d->orbit_start_deg) || !std::isfinite(d->offset_x) || !std::isfinite(d->offset_y) ||
        !std::isfinite(d->offset_s)) {
        set_error("bad geometry lengths/angles");
        return CT_EINVAL;
    }
    // image extent: farthest pixel corner from the isocentre
    const double cxo = (d->nx - 1) / 2.0 - d->offset_x, cyo = (d->ny - 1) / 2.0 - d->offset_y;
    double r_img = 0.0;
    for (int cx = 0; cx < 2; cx++)
        for (int cy = 0; cy < 2; cy++) {
            const double X = ((cx ? d->nx - 0.5 : -0.5) - cxo) * d->dx;
            const double Y = ((cy ? d->ny - 0.5 : -0.5) - cyo) * d->dy;
            r_img = std::fmax(r_img, std::hypot(X, Y));
        }
    const double pmax = std::fmax(d->dx, d->dy);
    // The footprint arithmetic expands small angles in series; it needs every pixel
    // at least 50 pixel widths in front of the source.
    if (d->dso - r_img < 50.0 * pmax) {
        set_error("image reaches within %.3g mm of the source (needs >= 50 pixels = %.3g mm)", d->dso - r_img,
                  50.0 * pmax);
        return CT_EINVAL;
    }
    const double dg = d->ds / d->dsd;
    const double half_fan = (d->ns / 2.0 + std::fabs(d->offset_s)) * dg;
    if (half_fan >= 1.4) {
        set_error("fan half-angle %.3g rad is too wide", half_fan);
        return CT_EINVAL;
    }

    // helical: widest axial shadow of one voxel, in rows (closest column to the source)
    int zc = 0;
    if (helical) {
        const int span = (int)std::ceil(std::sqrt(d->dx * d->dx + d->dy * d->dy) / ((d->dso - r_img) * dg)) + 2;
        if (span > helix_max_span()) {
            set_error("detector cells too fine for the voxels: a column's footprint spans %d cells (max %d)", span,
                      helix_max_span());
            return CT_ENOTSUP;
        }
        if (d->axial != CT_AXIAL_RECT && d->axial != CT_AXIAL_TRAP) {
            set_error("unknown axial footprint %d", d->axial);
            return CT_EINVAL;
        }
        const double a_max = d->dz * d->dsd / d->dt / (d->dso - r_img);
        double extra_rows = 0.0;
        if (d->axial == CT_AXIAL_TRAP) {
            // ramp half-width h = eps |z - z_src| / dz voxels, eps = (L_max - L_min) / (L_max + L_min)
            // <= diagonal / (2 (dso - r_img)); the kernels need h < 1/2 (a voxel's two ramps apart)
            const double eps_max = std::hypot(d->dx, d->dy) / (2.0 * (d->dso - r_img));
            const double face0 = (-d->nz / 2.0 + d->offset_z) * d->dz, face1 = face0 + d->nz * d->dz;
            const double cover = d->nt * d->dt * d->dso / d->dsd;
            const double zs = std::fabs(d->pitch) * cover * std::fabs(d->orbit_deg) / 720.0;  // |z_src| at the ends
            const double zmax = std::fmax(std::fabs(face0), std::fabs(face1)) + zs;
            const double h_max = eps_max * zmax / d->dz;
            if (!(h_max < 0.5)) {
                set_error("trapezoid axial footprints too wide for the voxels (ramp half-width up to %.3g voxels; "
                          "needs < 0.5)", h_max);
                return CT_ENOTSUP;
            }
            extra_rows = 2.0 * h_max * a_max;
        }
        zc = helix_chunk_voxels(a_max, extra_rows);
        if (zc == 0) {
            set_error("voxels too tall for the detector rows: one voxel's shadow exceeds the row buffer");
            return CT_ENOTSUP;
        }
    }

    ct_geom *g = new ct_geom();
    g->desc = *d;
    g->helical = helical ? 1 : 0;
    g->hx_zc = zc;
    cudaGetDevice(&g->device);
    FanDev &F = g->fan;
    F.nx = d->nx; F.ny = d->ny; F.ns = d->ns; F.na = d->na;
    F.ntx = (d->nx + kTile - 1) / kTile;
    F.nty = (d->ny + kTile - 1) / kTile;
    F.nax = (d->nx + kAnchor - 1) / kAnchor;
    F.nay = (d->ny + kAnchor - 1) / kAnchor;
    F.dx = (float)d->dx; F.dy = (float)d->dy;
    F.hx = (float)(0.5 * d->dx); F.hy = (float)(0.5 * d->dy);
    F.inv_dx = (float)(1.0 / d->dx); F.inv_dy = (float)(1.0 / d->dy);
    F.inv_dg = (float)(1.0 / dg);
    F.dgamma = (float)dg;
    F.gamma0 = (float)((-(d->ns - 1) / 2.0 + d->offset_s) * dg);
    F.dso = (float)d->dso;
    F.x_edge0 = (float)((-0.5 - cxo) * d->dx);
    F.y_edge0 = (float)((-0.5 - cyo) * d->dy);
    F.cxo = (float)cxo; F.cyo = (float)cyo;
    // widest footprint: a pixel diagonal at the smallest source distance, plus partial cells at both ends
    F.max_span = (int)std::ceil(std::sqrt(d->dx * d->dx + d->dy * d->dy) / ((d->dso - r_img) * dg)) + 2;

    const int na = d->na, ntiles = F.nax * F.nay;  // anchor tiles
    std::vector<float2> cs(na);
    std::vector<float> bet(na);
    std::vector<double2> vcs(na);  // cos, sin of each view angle (FP64) for the anchor kernels
    for (int v = 0; v < na; v++) {
        double deg = std::fmod(d->orbit_start_deg + (double)v * d->orbit_deg / na, 360.0);
        if (deg < 0) deg += 360.0;
        const double b = deg * M_PI / 180.0, cb = std::cos(b), sb = std::sin(b);
        vcs[v] = make_double2(cb, sb);
        cs[v] = make_float2((float)cb, (float)sb);
        bet[v] = (float)b;
    }
    std::vector<int> ident(na);
    for (int v = 0; v < na; v++) ident[v] = v;
    AnchorParams AP;
    AP.na = na;
    AP.nax = F.nax;
    AP.nay = F.nay;
    AP.cxo = cxo;
    AP.cyo = cyo;
    AP.dx = d->dx;
    AP.dy = d->dy;
    AP.dso = d->dso;
    AP.inv_dg = 1.0 / dg;
    AP.c0 = (d->ns - 1) / 2.0 - d->offset_s;
    AP.dso_f = F.dso;
    const long long n_anchor = (long long)na * ntiles;
    const unsigned anchor_blocks = (unsigned)((n_anchor + 255) / 256);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&g->d_anchor, sizeof(float4) * 3 * (size_t)n_anchor);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_view_cs, sizeof(float2) * na);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_view_beta, sizeof(float) * na);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_views_all, sizeof(int) * na);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_views_stage, sizeof(int) * na);
    const size_t rows = helical ? (size_t)d->nt : 1;
    if (e == cudaSuccess) e = cudaMalloc(&g->d_sino_ws, sizeof(float) * (size_t)na * d->ns * rows);
    // the anchor tables: the largest |du/dpx| + |du/dpy| fixes the grid of the exact FP32 linear term (S =
    // af + kxh px + kyh py over all tiles and points |px|, |py| <= kAnchor / 2 stays below 2^(24 - p) in
    // magnitude, so FP32 holds every such S, a multiple of 2^-p, exactly), then the tables themselves
    double2 *d_vcs = nullptr;
    unsigned long long *d_kmax = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_vcs, sizeof(double2) * na + 256);
    if (e == cudaSuccess) {
        d_kmax = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(d_vcs) + ((sizeof(double2) * na + 15) & ~(size_t)15));
        e = cudaMemcpy(d_vcs, vcs.data(), sizeof(double2) * na, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(d_kmax, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        anchor_kmax_kernel<<<anchor_blocks, 256>>>(AP, d_vcs, d_kmax);
        e = cudaGetLastError();
    }
    unsigned long long kbits = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&kbits, d_kmax, sizeof(kbits), cudaMemcpyDeviceToHost);
    int p = 0;
    double s_bound = 0.0;
    if (e == cudaSuccess) {
        double kmax;
        std::memcpy(&kmax, &kbits, sizeof kmax);
        s_bound = 2.0 + kAnchor * kmax;  // af <= 1, plus twice the largest |kx px + ky py|
        p = 23 - (int)std::ceil(std::log2(s_bound));
        if (p < 8) {
            cudaFree(d_vcs);
            set_error("detector cells too fine for the pixels: a tile's footprint spans %.0f cells", s_bound);
            free_geom(g);
            return CT_ENOTSUP;
        }
        anchor_fill_kernel<<<anchor_blocks, 256>>>(AP, d_vcs, std::ldexp(1.0, p - 1), std::ldexp(1.0, p), g->d_anchor);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(d_vcs);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_view_cs, cs.data(), sizeof(float2) * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_view_beta, bet.data(), sizeof(float) * na, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_views_all, ident.data(), sizeof(int) * na, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        ct_status st = cuda_fail(e, "ct_geom_create");
        free_geom(g);
        return st;
    }
    if (e == cudaSuccess && helical) {
        // axial tables (FP64 on the host): per view, the volume's lower face relative to the source
        // height in voxel units (hi + lo floats); per row, 1/cos of its cone angle
        std::vector<float2> zbv(na);
        std::vector<float> rc(d->nt);
        std::vector<float4> tax((size_t)na * ntiles);
        const double face0 = (-d->nz / 2.0 + d->offset_z) * d->dz;
        const double mid = (d->orbit_start_deg + 0.5 * d->orbit_deg) * M_PI / 180.0;
        const double cover = d->nt * d->dt * d->dso / d->dsd;
        const double kA = d->dz * d->dsd / d->dt;
        host_parallel_for(na, [&](int v0, int v1, int) {
        for (int v = v0; v < v1; v++) {
            const double b = (d->orbit_start_deg + (double)v * d->orbit_deg / na) * M_PI / 180.0;
            const double zsrc = d->pitch * cover * (b - mid) / (2.0 * M_PI);
            const double zb = (face0 - zsrc) / d->dz;
            const double zbi = std::nearbyint(zb);
            zbv[v] = make_float2((float)zbi, (float)(zb - zbi));
            const double cb = std::cos(b), sb = std::sin(b);
            for (int ty = 0; ty < F.nay; ty++)
                for (int tx = 0; tx < F.nax; tx++) {
                    const double X = (tx * kAnchor + (double)kAnchorHalf - cxo) * d->dx;
                    const double Y = (ty * kAnchor + (double)kAnchorHalf - cyo) * d->dy;
                    const double tpar = d->dso + X * cb + Y * sb, tperp = -X * sb + Y * cb;
                    const double L = std::sqrt(tpar * tpar + tperp * tperp);
                    const double ia = L / kA, a = kA / L;
                    const float iah = (float)ia, ah = (float)a;
                    tax[(size_t)v * ntiles + ty * F.nax + tx] =
                        make_float4(iah, (float)(ia - (double)iah), ah, (float)(a - (double)ah));
                }
        }
        });
        for (int t = 0; t < d->nt; t++) {
            const double vt = (t - (d->nt - 1) / 2.0 + d->offset_t) * d->dt;
            rc[t] = (float)std::sqrt(1.0 + (vt / d->dsd) * (vt / d->dsd));
        }
        e = cudaMalloc(&g->d_view_zb, sizeof(float2) * na);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_row_c, sizeof(float) * d->nt);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_vol_ws, sizeof(float) * (size_t)d->nx * d->ny * d->nz);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_tile_ax, sizeof(float4) * tax.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_tile_ax, tax.data(), sizeof(float4) * tax.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_view_zb, zbv.data(), sizeof(float2) * na, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_row_c, rc.data(), sizeof(float) * d->nt, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            ct_status st = cuda_fail(e, "ct_geom_create (helical tables)");
            free_geom(g);
            return st;
        }
        g->hx.nz = d->nz;
        g->hx.nt = d->nt;
        const double ofr = d->offset_t - std::nearbyint(d->offset_t);
        g->hx.ct0 = (float)((d->nt - 1) / 2.0 - d->offset_t);
        g->hx.ct0i = (float)((d->nt - 1) / 2.0 - std::nearbyint(d->offset_t));
        g->hx.ofr = (float)ofr;
        g->hx.kA = (float)kA;
        g->hx.inv_kA = (float)(1.0 / kA);
        g->hx.view_zb = g->d_view_zb;
        g->hx.row_c = g->d_row_c;
        g->hx.tile_ax = g->d_tile_ax;
        g->hx.trap = d->axial == CT_AXIAL_TRAP ? 1 : 0;
        g->hx.dso = F.dso;
    }
    F.anchor = g->d_anchor;
    F.view_cs = g->d_view_cs;
    F.view_beta = g->d_view_beta;
    const double r_fan = d->dso * std::sin(std::fmin(half_fan, M_PI / 2));
    g->fov_radius = std::fmin(r_fan, 0.5 * std::fmin(d->nx * d->dx, d->ny * d->dy));
    *out = g;
    return CT_OK;
}

extern "C" void ct_geom_destroy(ct_geom *g) { free_geom(g); }

extern "C" const char *ct_last_error(void) { return ct::g_last_error.c_str(); }

extern "C" int ct_version(void) { return 100; }
