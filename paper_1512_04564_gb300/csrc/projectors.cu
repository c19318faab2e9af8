// Separable-footprint fan-beam projector pair for sm_103a.
//
// A is the SF system matrix of the PWLS problem (Sec. III, Eq. (ct_problem));
// each a_ij comes from one device function (sf_footprint) used by both the
// ray-driven forward projector and the voxel-driven back-projector, so the
// pair is matched.  Both are FP32-ALU bound gathers (no tensor-core
// contraction exists in them).
//
// Forward projector (ray-driven, cell-owned outputs, no atomics):
// * bundle kernel: one CTA per (view, 32 adjacent detector cells); its 8 warps
//   split the image columns (rows, for steep bundles) that the bundle's fan
//   wedge crosses.  In each round a warp packs the next 32 wedge pixels
//   (across columns, by a warp prefix scan) one per lane, evaluates each
//   pixel's footprint once and stages its cell weights in shared memory;
//   then every lane, as the owner of one cell, gathers the weights of the
//   pixels its own wedge crosses.  The 8 warps' partial sums are added in a
//   fixed order, so results are deterministic.
// * ray kernel (fallback for detectors so fine that one footprint covers more
//   than kMaxSpan cells): 8 lanes per cell march 1/8 of the columns each,
//   evaluating every wedge pixel's footprint, combined by warp shuffles.
// Fused epilogues: plain y = A x, the weighted residual r = w (A x - y) of
// the subset gradient (Eq. (ct_substitution)), and w (A 1) for the SQS
// diagonal.
//
// * resident-matrix kernel (after ct_geom_precompute): one warp per ray
//   streams the ray's stored (pixel, a_ij) entries and gathers x.
//
// Back-projector: one CTA per 16x16 pixel tile (or half tile), gathering from
// the cells its footprint covers: footprints evaluated on the fly (corners
// shared by neighbouring pixels, staged per view in shared memory), or the
// resident matrix's per-(view, pixel) records of cell weights.  Fused epilogues: plain
// x = scale A'r (+x), and the relaxed OS-LALM g/h updates of Algorithm 1/2
// (Sec. III-A).
#include <cstdio>

#include "ct_internal.cuh"

namespace ct {

namespace {

constexpr int kFpThreads = 256;
constexpr int kFpSeg = 8;  // lanes per ray (ray kernel)
constexpr int kBundleWarps = 8;     // warps per bundle CTA
constexpr int kMaxSpan = 12;        // cells per staged footprint (bundle kernel)
constexpr int kMaxMarch = 2048;     // longest march axis the bundle kernel stages
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBpThreads = 128;     // back-projector CTA: one 16x16 tile, two pixels per thread

// Marching frame of a bundle: "march" is the axis the wedge is walked along
// (x for shallow bundles, y for steep ones), "cross" the other axis.
struct March {
    float m_edge0, m_d;     // march axis: edge of index 0, pixel size
    float c_edge0, c_invd;  // cross axis: edge of index 0, 1/pixel size
    float Sm, Sc;           // source position (march, cross)
    int n_march, n_cross;
    bool col;
};

// Cross-axis pixel range [lo, hi] of the wedge between the lines of slopes T1, T2
// (cross = Sc + (march - Sm) T) inside the march slab of index a.
__device__ __forceinline__ void wedge_range(const March &M, int a, float T1, float T2, int &lo, int &hi)
{
    const float ml = fmaf((float)a, M.m_d, M.m_edge0) - M.Sm, mr = ml + M.m_d;
    const float c1 = fmaf(ml, T1, M.Sc), c2 = fmaf(mr, T1, M.Sc);
    const float c3 = fmaf(ml, T2, M.Sc), c4 = fmaf(mr, T2, M.Sc);
    const float clo = (fminf(fminf(c1, c2), fminf(c3, c4)) - M.c_edge0) * M.c_invd - kRangePad;
    const float chi = (fmaxf(fmaxf(c1, c2), fmaxf(c3, c4)) - M.c_edge0) * M.c_invd + kRangePad;
    lo = max(0, (int)floorf(fmaxf(clo, -1.0f)));
    hi = min(M.n_cross - 1, (int)floorf(fminf(chi, (float)M.n_cross)));
}

__device__ __forceinline__ float march_slope(const March &M, float ang)
{
    float sn, cn;
    sincosf(ang, &sn, &cn);
    return M.col ? sn / cn : cn / sn;
}

// Number of entries of the warp-wide nondecreasing array `incl` that are <= key (< 32 if incl[31] > key).
__device__ __forceinline__ int count_le(int incl, int key)
{
    int pos = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(kFull, incl, pos + step - 1);
        if (v <= key) pos += step;
    }
    return pos;
}

template <int MODE>
__global__ void __launch_bounds__(kBundleWarps * 32, 5) fp_bundle_kernel(FanDev G, const float *__restrict__ x,
                                                                       const int *__restrict__ views, int nviews,
                                                                       float *__restrict__ out,
                                                                       const float *__restrict__ y,
                                                                       const float *__restrict__ w)
{
    __shared__ int s_pre[kMaxMarch + 1];  // pixels of the bundle's wedge before march index a
    __shared__ int s_lo[kMaxMarch];       // first wedge pixel (cross index) at march index a
    __shared__ float s_w[kBundleWarps][32][kMaxSpan + 1];
    __shared__ int s_c[kBundleWarps][32];  // first cell (relative to s0) of each staged pixel
    __shared__ int s_n[kBundleWarps][32];  // number of staged cells of each pixel
    __shared__ int s_part[kBundleWarps];
    __shared__ float s_acc[kBundleWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = (G.ns + 31) >> 5;
    const int k = blockIdx.x / nb;
    const int s0 = (blockIdx.x - k * nb) * 32;
    const int v = __ldg(&views[k]);
    const float2 cs = __ldg(&G.view_cs[v]);
    const float beta = __ldg(&G.view_beta[v]);
    const int s_last = min(s0 + 31, G.ns - 1);
    const float a_lo = beta + fmaf((float)s0 - 0.5f, G.dgamma, G.gamma0);
    const float a_hi = beta + fmaf((float)s_last + 0.5f, G.dgamma, G.gamma0);
    float sn, cn;
    sincosf(0.5f * (a_lo + a_hi), &sn, &cn);
    March M;
    M.col = fabsf(cn) >= fabsf(sn);
    const float Sx = -G.dso * cs.x, Sy = -G.dso * cs.y;
    if (M.col) {
        M.m_edge0 = G.x_edge0; M.m_d = G.dx; M.c_edge0 = G.y_edge0; M.c_invd = G.inv_dy;
        M.Sm = Sx; M.Sc = Sy; M.n_march = G.nx; M.n_cross = G.ny;
    } else {
        M.m_edge0 = G.y_edge0; M.m_d = G.dy; M.c_edge0 = G.x_edge0; M.c_invd = G.inv_dx;
        M.Sm = Sy; M.Sc = Sx; M.n_march = G.ny; M.n_cross = G.nx;
    }
    const int nm = M.n_march;
    {   // wedge pixel counts per march index, then an exclusive scan over the CTA
        const float TB1 = march_slope(M, a_lo), TB2 = march_slope(M, a_hi);
        const int per = (nm + kBundleWarps * 32 - 1) / (kBundleWarps * 32);
        const int a0 = threadIdx.x * per;
        int run = 0;
        for (int i = 0; i < per; i++) {
            const int a = a0 + i;
            if (a < nm) {
                int lo, hi;
                wedge_range(M, a, TB1, TB2, lo, hi);
                s_lo[a] = lo;
                const int c = max(hi - lo + 1, 0);
                s_pre[a] = c;
                run += c;
            }
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        int base = 0;
        for (int q = 0; q < warp; q++) base += s_part[q];
        int pos = base + incl - run;
        for (int i = 0; i < per; i++) {
            const int a = a0 + i;
            if (a < nm) {
                const int c = s_pre[a];
                s_pre[a] = pos;
                pos += c;
            }
        }
        if (threadIdx.x == kBundleWarps * 32 - 1) s_pre[nm] = pos;
        __syncthreads();
    }
    const int T = s_pre[nm];
    const int s_mine = s0 + lane;
    const float my_a = beta + fmaf((float)s_mine, G.dgamma, G.gamma0);
    const float t1 = march_slope(M, my_a - 0.5f * G.dgamma), t2 = march_slope(M, my_a + 0.5f * G.dgamma);
    float(*sw)[kMaxSpan + 1] = s_w[warp];
    int *scf = s_c[warp];
    int *sns = s_n[warp];
    float acc = 0.0f;
    // this warp's equal share of the wedge pixels
    const int t_end = (int)(((long)(warp + 1) * T) / kBundleWarps);
    int t0 = (int)(((long)warp * T) / kBundleWarps);
    int col = 0;
    while (t0 < t_end) {
        while (s_pre[col + 1] <= t0) col++;  // march index holding task t0 (uniform)
        // lane l: end (exclusive) task index of march index col + l
        const int e = s_pre[min(col + lane + 1, nm)];
        const int n = min(min(32, t_end - t0), __shfl_sync(kFull, e, 31) - t0);
        const int t = t0 + lane;
        const int ls = min(count_le(e, t), 31);
        const int c = col + ls;
        int cf = 1 << 20, cnt = 0;
        if (lane < n) {  // pixel role
            const int bc = s_lo[c] + (t - s_pre[c]);
            const int ix = M.col ? c : bc, iy = M.col ? bc : c;
            const float xv = (MODE == FP_ONES_W) ? 1.0f : __ldg(&x[(size_t)iy * G.nx + ix]);
            if (xv != 0.0f) {
                const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
                const float xa = xv * F.amp;
                cnt = foot_cells(F, kMaxSpan, [&](int i, float a) { sw[lane][i] = a * xa; });
                cf = F.n + foot_first(F) - s0;
            }
        }
        scf[lane] = cf;
        sns[lane] = cnt;
        __syncwarp();
        // cell role: gather the staged weights of the pixels this lane's wedge crosses
        const int lmax = __shfl_sync(kFull, ls, n - 1);
        for (int l = 0; l <= lmax; l++) {
            const int cc = col + l;
            const int pre_c = s_pre[cc];
            const int task_lo = max(pre_c, t0), task_hi = min(__shfl_sync(kFull, e, l), t0 + n);  // [lo, hi)
            const int row0 = s_lo[cc] - pre_c;  // cross index of task t is row0 + t
            int q_lo, q_hi;
            wedge_range(M, cc, t1, t2, q_lo, q_hi);
            q_lo = max(q_lo, row0 + task_lo);
            q_hi = min(q_hi, row0 + task_hi - 1);
            for (int q = q_lo; q <= q_hi; q++) {
                const int slot = q - row0 - t0;
                const int i = lane - scf[slot];
                if ((unsigned)i < (unsigned)sns[slot]) acc += sw[slot][i];
            }
        }
        __syncwarp();
        t0 += n;
    }
    s_acc[warp][lane] = acc;
    __syncthreads();
    if (warp != 0 || s_mine >= G.ns) return;
    float sum = 0.0f;
#pragma unroll
    for (int q = 0; q < kBundleWarps; q++) sum += s_acc[q][lane];
    const size_t yi = (size_t)v * G.ns + s_mine;
    if (MODE == FP_PLAIN) out[(size_t)k * G.ns + s_mine] = sum;
    else if (MODE == FP_RESID) out[(size_t)k * G.ns + s_mine] = __ldg(&w[yi]) * (sum - __ldg(&y[yi]));
    else out[yi] = __ldg(&w[yi]) * sum;
}

template <int MODE>
__global__ void __launch_bounds__(kFpThreads) fp_ray_kernel(FanDev G, const float *__restrict__ x,
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
        ray_visit(G, v, s, seg, kFpSeg, [&](int ix, int iy) {
            const float xv = (MODE == FP_ONES_W) ? 1.0f : __ldg(&x[(size_t)iy * G.nx + ix]);
            if (xv == 0.0f) return;
            const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
            acc = fmaf(cell_weight(F, s), xv, acc);
        });
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

// Resident-matrix forward projection: one warp per ray streams the ray's
// entry pairs (two a_ij and two 16-bit pixel-index offsets each, two pairs in
// flight per lane), gathers from the packed image [x | x^T] (x itself for a
// shallow ray, the transposed copy for a steep one) through L1/L2 and reduces
// by shuffles.  The 8 warps of a CTA take 8 adjacent cells of one view,
// whose wedges cover nearly the same pixels.  CTAs run the cell blocks in the
// geometry's ray_order (most entries first, every view of the list for each
// block), so that the end of the launch is made of short rays.
template <int MODE>
__global__ void __launch_bounds__(256) fp_csr_kernel(FanDev G, const float *__restrict__ x,
                                                     const int *__restrict__ views, int nviews,
                                                     float *__restrict__ out, const float *__restrict__ y,
                                                     const float *__restrict__ w)
{
    const int lane = threadIdx.x & 31;
    const int rank = (int)(blockIdx.x / (unsigned)nviews), k = (int)(blockIdx.x - (unsigned)rank * nviews);
    const int s = 8 * __ldg(&G.ray_order[rank]) + (threadIdx.x >> 5);
    if (s >= G.ns) return;  // whole warp
    const int v = __ldg(&views[k]);
    const size_t r = (size_t)v * G.ns + s;
    const long long b = __ldg(&G.row_ptr[r]), e = __ldg(&G.row_ptr[r + 1]);
    float acc = csr_ray_dot<MODE == FP_ONES_W, false>(G, b, e, __ldg(&G.row_first[r]), x, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane != 0) return;
    if (MODE == FP_PLAIN) out[(size_t)k * G.ns + s] = acc;
    else if (MODE == FP_RESID) out[(size_t)k * G.ns + s] = __ldg(&w[r]) * (acc - __ldg(&y[r]));
    else out[r] = __ldg(&w[r]) * acc;
}

template <int MODE>
__device__ __forceinline__ void bp_epilogue(const FanDev &G, const SolveDev &S, float *__restrict__ xo, int ix,
                                            int iy, float acc, float rho, float scale, int accumulate)
{
    if (ix >= G.nx || iy >= G.ny) return;
    const size_t j = (size_t)iy * G.nx + ix;
    if (MODE == BP_PLAIN) {
        xo[j] = accumulate ? fmaf(scale, acc, xo[j]) : scale * acc;
        return;
    }
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

// Resident-matrix back-projection, one CTA per half tile (16 x 8 pixels, the first or last 128 slots of a
// tile), one pixel per thread: twice the CTAs and warps of a full-tile CTA, which with 1024 tiles at
// 512 x 512 left the SMs 60% empty.  Warp w reads chunk w of the half tile per view: its word (start and
// K) two views ahead of use, its record (first cell and count, K weights in coalesced 128-byte loads)
// one view ahead.
template <int MODE>
__global__ void __launch_bounds__(kBpThreads, 16) bp_records_kernel(FanDev G, const float *__restrict__ sino,
                                                                  const int *__restrict__ views, int nviews,
                                                                  float *__restrict__ xo, float scale,
                                                                  int accumulate, SolveDev S)
{
    const int half = blockIdx.y & 1, ty = blockIdx.y >> 1;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile + half * (kTile / 2);
    const int ix = blockIdx.x * kTile + lx, iy = ty * kTile + ly;
    const unsigned group = (unsigned)(ty * G.ntx + blockIdx.x) * (kTile * kTile / kRecGroup) +
                           (half * kBpThreads + threadIdx.x) / kRecGroup;
    float rho = 1.0f;
    if (MODE == BP_SOLVE_UPDATE) rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float acc = 0.0f;
    unsigned word = 0;
    RecSlot r{};
    if (nviews > 0) r = rec_fetch(G, rec_word(G, __ldg(&views[0]), group));
    if (nviews > 1) word = rec_word(G, __ldg(&views[1]), group);
    for (int k = 0; k < nviews; k++) {
        const RecSlot cur = r;
        if (k + 1 < nviews) r = rec_fetch(G, word);
        if (k + 2 < nviews) word = rec_word(G, __ldg(&views[k + 2]), group);
        acc += rec_dot(G, cur, sino + (size_t)k * G.ns, [&] { return rec_word(G, __ldg(&views[k]), group); });
    }
    bp_epilogue<MODE>(G, S, xo, ix, iy, acc, rho, scale, accumulate);
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

// The same with the views split (images too small for bp_records_kernel to fill the SMs: a warp walking all
// of a launch's views one after another is bound by their latency, not the bytes): VS = 2 or 4 warps share a
// record chunk, warp q taking views q, q + VS, ...; their sums are added in a fixed order (q = 0, 1, ...)
// through shared memory.  A CTA of 4 warps covers 4 / VS chunks.  (Grids under one wave: more registers.)
template <int MODE, int VS>
__global__ void __launch_bounds__(kBpThreads, 8) bp_records_split_kernel(FanDev G, const float *__restrict__ sino,
                                                                  const int *__restrict__ views, int nviews,
                                                                  float *__restrict__ xo, float scale,
                                                                  int accumulate, SolveDev S)
{
    constexpr int kCpc = (kBpThreads / kRecGroup) / VS;           // chunks per CTA
    constexpr int kSubs = (kTile * kTile / kRecGroup) / kCpc;      // CTAs per tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.y % kSubs, ty = blockIdx.y / kSubs;
    const int chunk = sub * kCpc + warp / VS, q = warp % VS;       // chunk of the tile, view phase
    const int slot = chunk * kRecGroup + lane;
    const int ix = blockIdx.x * kTile + (slot & (kTile - 1)), iy = ty * kTile + slot / kTile;
    const unsigned group = (unsigned)(ty * G.ntx + blockIdx.x) * (kTile * kTile / kRecGroup) + chunk;
    float rho = 1.0f;
    if (MODE == BP_SOLVE_UPDATE) rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float acc = 0.0f;
    unsigned word = 0;
    RecSlot r{};
    if (q < nviews) r = rec_fetch(G, rec_word(G, __ldg(&views[q]), group));
    if (q + VS < nviews) word = rec_word(G, __ldg(&views[q + VS]), group);
    for (int k = q; k < nviews; k += VS) {
        const RecSlot cur = r;
        if (k + VS < nviews) r = rec_fetch(G, word);
        if (k + 2 * VS < nviews) word = rec_word(G, __ldg(&views[k + 2 * VS]), group);
        acc += rec_dot(G, cur, sino + (size_t)k * G.ns, [&] { return rec_word(G, __ldg(&views[k]), group); });
    }
    {
        __shared__ float s_part[kBpThreads];
        s_part[threadIdx.x] = acc;
        __syncthreads();
        if (q == 0)
#pragma unroll
            for (int p = 1; p < VS; p++) acc += s_part[threadIdx.x + 32 * p];
    }
    if (q == 0) bp_epilogue<MODE>(G, S, xo, ix, iy, acc, rho, scale, accumulate);
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

// Back-projection with the footprints evaluated on the fly: one CTA per 16x16 tile (four 8x8 anchor
// tiles), one pixel per thread.  A pixel corner is shared by up to four pixels, so per view the CTA
// first computes the detector coordinates (S, L) of the 4 x 9 x 9 corners of its anchor tiles into
// shared memory (double-buffered: the next view's corners are computed while this view's are used, one
// barrier per view); each pixel then builds its footprint from its four corners, its amplitude from its
// centre ray, and takes the dot product with the view's detector row.
constexpr int kBpFlyThreads = kTile * kTile;
constexpr int kCornerSide = kAnchor + 1;                  // corners per side of an anchor tile
constexpr int kTileCorners = 4 * kCornerSide * kCornerSide;  // 324 per CTA

template <int MODE>
__global__ void __launch_bounds__(kBpFlyThreads, 4) bp_fan2d_kernel(FanDev G, const float *__restrict__ sino,
                                                                 const int *__restrict__ views, int nviews,
                                                                 float *__restrict__ xo, float scale, int accumulate,
                                                                 SolveDev S)
{
    __shared__ float2 s_c[2][kTileCorners];  // (S, L) of corner (quadrant, cy, cx)
    __shared__ int s_n[2][4];                // base cell of each quadrant's anchor
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int ix = blockIdx.x * kTile + lx, iy = blockIdx.y * kTile + ly;
    const bool inside = ix < G.nx && iy < G.ny;
    const int q = (ly >= kAnchor ? 2 : 0) + (lx >= kAnchor ? 1 : 0);
    const int c0 = q * (kCornerSide * kCornerSide) + (ly & (kAnchor - 1)) * kCornerSide + (lx & (kAnchor - 1));
    // pixel centre in the image frame (mm)
    const float xc = ((float)ix - G.cxo) * G.dx, yc = ((float)iy - G.cyo) * G.dy;
    float rho = 1.0f;
    if (MODE == BP_SOLVE_UPDATE) rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    // corner staging: corner c (and c + 256 for the first 68 threads) of view k into buffer b
    auto stage = [&](int k, int b) {
        const int v = __ldg(&views[k]);
#pragma unroll
        for (int rep = 0; rep < 2; rep++) {
            const int c = threadIdx.x + rep * kBpFlyThreads;
            if (c < kTileCorners) {
                const int cq = c / (kCornerSide * kCornerSide), r = c - cq * (kCornerSide * kCornerSide);
                const int cy = r / kCornerSide, cx = r - cy * kCornerSide;
                const int atx = 2 * blockIdx.x + (cq & 1), aty = 2 * blockIdx.y + (cq >> 1);
                if (atx < G.nax && aty < G.nay) {
                    const Anchor A = load_anchor(G, v, aty * G.nax + atx);
                    float Sv, Lv;
                    point_u(G, A, (float)(cx - kAnchor / 2), (float)(cy - kAnchor / 2), Sv, Lv);
                    s_c[b][c] = make_float2(Sv, Lv);
                    if (r == 0) s_n[b][cq] = A.n;
                }
            }
        }
    };
    float acc = 0.0f;
    if (nviews > 0) stage(0, 0);
    __syncthreads();
    for (int k = 0; k < nviews; k++) {
        const int b = k & 1;
        if (k + 1 < nviews) stage(k + 1, b ^ 1);
        if (inside) {
            const int v = __ldg(&views[k]);
            const float2 cs = __ldg(&G.view_cs[v]);
            const float2 p0 = s_c[b][c0], p1 = s_c[b][c0 + 1];
            const float2 p2 = s_c[b][c0 + kCornerSide], p3 = s_c[b][c0 + kCornerSide + 1];
            const float Sk[4] = {p0.x, p1.x, p2.x, p3.x}, Lk[4] = {p0.y, p1.y, p2.y, p3.y};
            // centre ray relative to the source (image frame): chord |c| / max(|c_x| / dx, |c_y| / dy)
            const float cxv = fmaf(G.dso, cs.x, xc), cyv = fmaf(G.dso, cs.y, yc);
            const float r2 = fmaf(cxv, cxv, cyv * cyv);
            const float amp = __fdividef(r2 * rsqrtf(r2), fmaxf(fabsf(cxv) * G.inv_dx, fabsf(cyv) * G.inv_dy));
            const Footprint F = footprint_from_corners(Sk, Lk, amp, s_n[b][q]);
            acc += footprint_dot(F, sino + (size_t)k * G.ns, G.ns);
        }
        __syncthreads();
    }
    if (inside) bp_epilogue<MODE>(G, S, xo, ix, iy, acc, rho, scale, accumulate);
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

// The packed image [x | x^T] the resident rows index: xp[j] = x[j] and xp[nx ny + ix ny + iy] = x[iy nx + ix].
// 32 x 8 pixel blocks, transposed through shared memory so that both halves are written in whole sectors.
__global__ void __launch_bounds__(256) pack_kernel(FanDev G, const float *__restrict__ x, float *__restrict__ xp)
{
    __shared__ float t[8][36];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int ix = blockIdx.x * 32 + lx, iy = blockIdx.y * 8 + ly;
    if (ix < G.nx && iy < G.ny) {
        const float v = __ldg(&x[(size_t)iy * G.nx + ix]);
        xp[(size_t)iy * G.nx + ix] = v;
        t[ly][lx] = v;
    }
    __syncthreads();
    write_transposed_block(G, t, xp);
}

}  // namespace

cudaError_t launch_pack(const FanDev &G, const float *x, float *xp, cudaStream_t st)
{
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    pack_kernel<<<grid, 256, 0, st>>>(G, x, xp);
    return cudaGetLastError();
}

cudaError_t launch_fp(const FanDev &G, int mode, const float *x, const int *views, int nviews, float *out,
                      const float *y, const float *w, cudaStream_t st, const float *xpack)
{
    if (nviews <= 0) return cudaSuccess;
    const bool bundle_ok = G.max_span <= kMaxSpan && G.nx <= kMaxMarch && G.ny <= kMaxMarch;
    int var = G.fp_variant;
    if (var == FP_VAR_CSR && !G.row_ptr) var = FP_AUTO;
    if (var == FP_VAR_BUNDLE && !bundle_ok) var = FP_AUTO;
    if (var == FP_AUTO) var = G.row_ptr ? FP_VAR_CSR : (bundle_ok ? FP_VAR_BUNDLE : FP_VAR_RAY);
    if (var == FP_VAR_CSR) {
        const unsigned blocks = (unsigned)nviews * (unsigned)((G.ns + 7) / 8);
        if (mode != FP_ONES_W) {  // the rows index the packed image
            if (!xpack) {
                const cudaError_t e = launch_pack(G, x, G.xpack, st);
                if (e != cudaSuccess) return e;
                xpack = G.xpack;
            }
            x = xpack;
        }
        switch (mode) {
        case FP_PLAIN: fp_csr_kernel<FP_PLAIN><<<blocks, 256, 0, st>>>(G, x, views, nviews, out, y, w); break;
        case FP_RESID: fp_csr_kernel<FP_RESID><<<blocks, 256, 0, st>>>(G, x, views, nviews, out, y, w); break;
        default: fp_csr_kernel<FP_ONES_W><<<blocks, 256, 0, st>>>(G, x, views, nviews, out, y, w); break;
        }
        return cudaGetLastError();
    }
    if (var == FP_VAR_BUNDLE) {
        const unsigned blocks = (unsigned)nviews * (unsigned)((G.ns + 31) / 32);
        switch (mode) {
        case FP_PLAIN: fp_bundle_kernel<FP_PLAIN><<<blocks, kBundleWarps * 32, 0, st>>>(G, x, views, nviews, out, y, w); break;
        case FP_RESID: fp_bundle_kernel<FP_RESID><<<blocks, kBundleWarps * 32, 0, st>>>(G, x, views, nviews, out, y, w); break;
        default: fp_bundle_kernel<FP_ONES_W><<<blocks, kBundleWarps * 32, 0, st>>>(G, x, views, nviews, out, y, w); break;
        }
        return cudaGetLastError();
    }
    const long nrays = (long)nviews * G.ns;
    const long rays_per_block = kFpThreads / kFpSeg;
    const unsigned blocks = (unsigned)((nrays + rays_per_block - 1) / rays_per_block);
    switch (mode) {
    case FP_PLAIN: fp_ray_kernel<FP_PLAIN><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    case FP_RESID: fp_ray_kernel<FP_RESID><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    default: fp_ray_kernel<FP_ONES_W><<<blocks, kFpThreads, 0, st>>>(G, x, views, nviews, out, y, w); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_bp(const FanDev &G, int mode, const float *sino, const int *views, int nviews, float *x,
                      float scale, int accumulate, const SolveDev *S, cudaStream_t st)
{
    dim3 grid(G.ntx, G.nty);
    SolveDev s0{};
    const SolveDev &SS = S ? *S : s0;
    const bool stored = G.rec_data && G.bp_variant != BP_VAR_FLY;
    if (stored) {
        const int vs = G.bp_vs == 4 ? 4 : (G.bp_vs == 2 ? 2 : 1);
        const dim3 hgrid(G.ntx, 2 * vs * G.nty);  // 2 vs CTAs per tile
#define CT_BP_REC(VS)                                                                                                     \
        switch (mode) {                                                                                                   \
        case BP_PLAIN: bp_records_split_kernel<BP_PLAIN, VS><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break; \
        case BP_SOLVE_INIT: bp_records_split_kernel<BP_SOLVE_INIT, VS><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break; \
        default: bp_records_split_kernel<BP_SOLVE_UPDATE, VS><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break; \
        }
        if (vs == 1) {
            switch (mode) {
            case BP_PLAIN: bp_records_kernel<BP_PLAIN><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
            case BP_SOLVE_INIT: bp_records_kernel<BP_SOLVE_INIT><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
            default: bp_records_kernel<BP_SOLVE_UPDATE><<<hgrid, kBpThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
            }
        } else if (vs == 2) {
            CT_BP_REC(2)
        } else {
            CT_BP_REC(4)
        }
#undef CT_BP_REC
        return cudaGetLastError();
    }
    switch (mode) {
    case BP_PLAIN: bp_fan2d_kernel<BP_PLAIN><<<grid, kBpFlyThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
    case BP_SOLVE_INIT: bp_fan2d_kernel<BP_SOLVE_INIT><<<grid, kBpFlyThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
    default: bp_fan2d_kernel<BP_SOLVE_UPDATE><<<grid, kBpFlyThreads, 0, st>>>(G, sino, views, nviews, x, scale, accumulate, SS); break;
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
    if (g->helical) return helix_forward(g, x, y, views, nviews, s);
    const int *dv = nullptr;
    if ((st = stage_views(g, views, nviews, &dv, s)) != CT_OK) return st;
    CT_CUDA_TRY(launch_fp(g->fan, FP_PLAIN, x, dv, nviews, y, nullptr, nullptr, s), "ct_forward launch");
    return CT_OK;
}

extern "C" ct_status ct_pack_image(const ct_geom *g, const float *x, float *xpack, void *stream)
{
    if (!g || !x || !xpack) { set_error("ct_pack_image: null argument"); return CT_EINVAL; }
    if (g->helical) { set_error("ct_pack_image: 2-D geometries only"); return CT_EINVAL; }
    CT_CUDA_TRY(launch_pack(g->fan, x, xpack, (cudaStream_t)stream), "ct_pack_image launch");
    return CT_OK;
}

extern "C" ct_status ct_forward_packed(const ct_geom *g, const float *xpack, float *y, const int *views, int nviews,
                                       void *stream)
{
    if (!g || !xpack || !y) { set_error("ct_forward_packed: null argument"); return CT_EINVAL; }
    if (g->helical) { set_error("ct_forward_packed: 2-D geometries only"); return CT_EINVAL; }
    ct_status st = validate_views(g, views, nviews);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int *dv = nullptr;
    if ((st = stage_views(g, views, nviews, &dv, s)) != CT_OK) return st;
    // the first half is x itself, for the projectors that do not index the packed image
    CT_CUDA_TRY(launch_fp(g->fan, FP_PLAIN, xpack, dv, nviews, y, nullptr, nullptr, s, xpack),
                "ct_forward_packed launch");
    return CT_OK;
}

extern "C" ct_status ct_back(const ct_geom *g, const float *y, float *x, const int *views, int nviews, float scale,
                             int accumulate, void *stream)
{
    if (!g || !x || !y) { set_error("ct_back: null argument"); return CT_EINVAL; }
    ct_status st = validate_views(g, views, nviews);
    if (st != CT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (g->helical) return helix_back(g, y, x, views, nviews, scale, accumulate, s);
    const int *dv = nullptr;
    if ((st = stage_views(g, views, nviews, &dv, s)) != CT_OK) return st;
    CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, y, dv, nviews, x, scale, accumulate, nullptr, s), "ct_back launch");
    return CT_OK;
}

extern "C" ct_status ct_sqs_diag(const ct_geom *g, const float *w, float *d_l, void *stream)
{
    if (!g || !w || !d_l) { set_error("ct_sqs_diag: null argument"); return CT_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    if (g->helical) return helix_sqs_diag(g, w, d_l, s);
    // q = w (A 1) over all views (A 1 kept with the geometry), then D_L = A' q
    CT_CUDA_TRY(ensure_ray_sums(const_cast<ct_geom *>(g), s), "ct_sqs_diag ray sums");
    CT_CUDA_TRY(launch_weighted_ray_sums(g, w, g->d_sino_ws, s), "ct_sqs_diag weights");
    CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, g->d_sino_ws, g->d_views_all, g->fan.na, d_l, 1.0f, 0, nullptr, s),
                "ct_sqs_diag back");
    return CT_OK;
}
