// Helical cone-beam CT (3-D) on sm_103a: the separable-footprint projector
// pair with a trapezoid transaxial and a rectangle axial footprint (SF-TR),
// the 26-neighbour regularizer (Eq. (def_reg), 13 directions) with the fused
// x-update of Algorithm 1/2, the RMSD reduction, and the changes between the
// C ABI's [iz][iy][ix] volumes and the column-major [iy][ix][iz] volumes the
// kernels use (a voxel column is contiguous, so the forward projector reads a
// column's z-range as one run and the back-projector writes its chunk as one).
//
//   a_{(v,t,s),j} = l_xy(j) * c_t * T_j(s) * R_j(t)
//
//   T_j(s): cell integral of the column's transaxial trapezoid (sf_footprint,
//           with the per-(view, 16x16 tile) FP64-derived anchors of the 2-D path);
//   l_xy:   the column's transaxial chord (the footprint amplitude);
//   R_j(t): overlap, in rows, of row t with the voxel's z-extent magnified by
//           dsd / L (L: transaxial source-to-column distance); voxel boundary k
//           falls at row coordinate u_k = a (k + zb_v) + ct0, a = dz dsd / (dt L);
//   c_t:    1 / cos(cone angle of row t).
//
// With the trapezoid axial footprint (SF-TT) the voxel's z-faces project at
// every magnification between those of the column's farthest and nearest
// corners (L_max, L_min), so each face's shadow edge becomes a linear ramp.
// Summed over a column, the voxels' trapezoids are the rectangle model at the
// ramps' centre (L = the harmonic mean of L_min and L_max) with each jump from
// x_{k-1} to x_k replaced by a ramp of half-width h_k = eps |z_k - z_src| / dz
// voxels, eps = (L_max - L_min) / (L_max + L_min).  So both kernels run the
// rectangle arithmetic at that L and add, at every row boundary that a ramp
// straddles at distance d (voxels) from its centre, (x_k - x_{k-1}) a
// (h_k - d)^2 / (4 h_k) to the row below and subtract it from the row above
// (ramps of one column never overlap: the geometry keeps h_k < 1/2).
//
// Forward projector (ray-driven, cell-owned outputs, no atomics): one CTA per
// (view, 32 adjacent cells); its warps split the image columns of the
// bundle's transaxial fan wedge.  Per round a warp stages 32 columns, one per
// lane: the lane evaluates the column's footprint once (cell weights) and its
// axial profile p_t = sum_k x_k R_k(t) over all rows; then each lane, as the
// owner of one cell, adds weight x profile for every staged column its own
// wedge crosses, for all rows at once.  Partial sums of the warps are added in
// a fixed order.
//
// Back-projector (voxel-driven, no atomics): one thread per (column, chunk of
// ZC voxels); per view it evaluates the column's footprint, forms the row
// sums q_t = c_t sum_s w_s y[t][s] over the rows its chunk reaches, and
// integrates them over each voxel's magnified extent through their running
// sum.  Fused epilogues as in 2-D (plain, and the g/h updates of Algorithm 1/2).
#include <cmath>

#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHxWarps = 4;         // warps per forward-projector CTA
constexpr int kHxMaxSpan = 12;      // cells per staged transaxial footprint
constexpr int kHxMaxMarch = 2048;   // longest march axis of a wedge
constexpr int kHxBpCols = 128;      // back-projector CTA: 16 x 8 columns
constexpr int kHxQMax = 64;         // rows one back-projector chunk may reach
constexpr int kHxMaxRows = 64;      // detector rows supported

// Marching frame of a bundle wedge: "march" is the axis walked along (x for
// shallow bundles, y for steep ones), "cross" the other.
struct March {
    float m_edge0, m_d;
    float c_edge0, c_invd;
    float Sm, Sc;
    int n_march, n_cross;
    bool col;
};

// Cross-axis column range [lo, hi] of the wedge between the lines of slopes T1,
// T2 (cross = Sc + (march - Sm) T) inside the march slab of index a.
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

// Number of entries of the warp-wide nondecreasing array `incl` that are <= key.
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

// Axial scale of column (ix, iy) in one view: voxels per row ia = L/kA and rows
// per voxel a = kA/L, L the transaxial source-to-column distance, each as hi +
// lo floats.  L = L_A + (L - L_A) with L_A the tile centre's FP64-derived
// distance and L - L_A = (2 A.d + |d|^2) / (L + L_A) (A: anchor vector, d:
// column offset), which is small and so accurate in FP32; the rounding of A
// cancels between |A + d| and |A| to first order.
struct ColumnAxial {
    float ia_hi, ia_lo, a_hi, a_lo;
};

//
// TT (trapezoid axial footprint): the scale is taken at the harmonic mean H of
// the column's nearest and farthest corner distances, L_min,max^2 = L^2 + q -+ P
// (P = |C_x| dx + |C_y| dy with C the column centre relative to the source in
// the world frame, q = (dx^2 + dy^2) / 4), again as a small correction
// H - L = (L (d+ + d-) + 2 d+ d-) / (2L + d+ + d-), d+- = L_max,min - L; eps
// receives (L_max - L_min) / (L_max + L_min).
template <bool TT>
__device__ __forceinline__ ColumnAxial column_axial(const HelixDev &H, const Anchor &A, float4 X, float cb, float sb,
                                                    float ox, float oy, float pdx, float pdy, float &eps)
{
    const float dpar = fmaf(ox, cb, oy * sb), dperp = fmaf(oy, cb, -ox * sb);
    const float cpar = H.dso + (A.ax + dpar), cperp = A.ay + dperp;  // A.ax: the anchor's t_par - dso
    const float L = sqrtf(fmaf(cpar, cpar, cperp * cperp));
    const float LA = X.x * H.kA;
    const float num = fmaf(2.0f, fmaf(H.dso, dpar, fmaf(A.ax, dpar, A.ay * dperp)), fmaf(dpar, dpar, dperp * dperp));
    float dL = __fdividef(num, L + LA);
    float Lc = L;
    eps = 0.0f;
    if (TT) {
        const float Cx = fmaf(cpar, cb, -cperp * sb), Cy = fmaf(cpar, sb, cperp * cb);
        const float P = fmaf(fabsf(Cx), pdx, fabsf(Cy) * pdy);
        const float q = 0.25f * fmaf(pdx, pdx, pdy * pdy);
        const float dp = __fdividef(P + q, sqrtf(fmaf(L, L, P + q)) + L);
        const float dm = __fdividef(q - P, sqrtf(fmaf(L, L, q - P)) + L);
        const float den = 2.0f * L + dp + dm;
        const float dH = __fdividef(fmaf(L, dp + dm, 2.0f * dp * dm), den);
        eps = __fdividef(dp - dm, den);
        dL += dH;
        Lc = L + dH;
    }
    ColumnAxial C;
    C.ia_hi = X.x;
    C.ia_lo = fmaf(dL, H.inv_kA, X.y);
    C.a_hi = X.z;
    C.a_lo = fmaf(-X.z, __fdividef(dL, Lc), X.w);
    return C;
}

// Ramp correction at a row boundary that lies at voxel coordinate z = K + f
// (0 <= f < 1) of a column: sum over the ramps of boundaries K and K+1 that
// straddle it of (x_k - x_{k-1}) (h_k - d)^2 / (4 h_k), d its distance from
// the ramp's centre, h_k = eps |k + zb|.  xv(k) returns x_k (0 outside).
template <class XV>
__device__ __forceinline__ float ramp_correction(int K, float f, float eps, float zb, XV xv)
{
    float c = 0.0f;
    const float h0 = eps * fabsf((float)K + zb);
    if (f < h0) {
        const float d = h0 - f;
        c = (xv(K) - xv(K - 1)) * __fdividef(d * d, 4.0f * h0);
    }
    const float h1 = eps * fabsf((float)(K + 1) + zb);
    const float g = 1.0f - f;
    if (g < h1) {
        const float d = h1 - g;
        c = fmaf(xv(K + 1) - xv(K), __fdividef(d * d, 4.0f * h1), c);
    }
    return c;
}

// ramp_correction with the voxel values around the boundary given: xm = x_{K-1}, x0 = x_K, xp = x_{K+1}.
__device__ __forceinline__ float ramp_correction_w(int K, float f, float eps, float zb, float xm, float x0, float xp)
{
    float c = 0.0f;
    const float h0 = eps * fabsf((float)K + zb);
    if (f < h0) {
        const float d = h0 - f;
        c = (x0 - xm) * __fdividef(d * d, 4.0f * h0);
    }
    const float h1 = eps * fabsf((float)(K + 1) + zb);
    const float g = 1.0f - f;
    if (g < h1) {
        const float d = h1 - g;
        c = fmaf(xp - x0, __fdividef(d * d, 4.0f * h1), c);
    }
    return c;
}

// Detector-row boundary b (row coordinate b - 1/2) of a column, in voxel
// coordinates z = K + f (voxel K spans [K, K+1], 0 <= f < 1):
//   z = (b - 1/2 - ct0i + ofr) ia - zbi - zbf.
// The integer parts are exact, so f is formed by one fma at magnitude ~1 and
// resolves the boundary to ~1e-7 voxel (a thin sliver of a voxel keeps its
// relative accuracy).  cz = ofr * ia - zbf.
__device__ __forceinline__ void row_boundary(float b_minus_c, float ia_hi, float ia_lo, float zbi, float cz, int nz,
                                             int &K, float &f)
{
    const float sm = fmaf(b_minus_c, ia_lo, cz);
    const float approx = fmaf(b_minus_c, ia_hi, sm - zbi);
    K = (int)floorf(fminf(fmaxf(approx, -2.0f), (float)nz + 1.0f));
    f = fmaf(b_minus_c, ia_hi, -(zbi + (float)K)) + sm;
    if (f < 0.0f) { K -= 1; f += 1.0f; }
    else if (f >= 1.0f) { K += 1; f -= 1.0f; }
}

template <int MODE, int NT, bool TT>
__global__ void __launch_bounds__(kHxWarps * 32, 5) fp_helix_kernel(FanDev G, HelixDev H, const float *__restrict__ x,
                                                                const int *__restrict__ views, int nviews,
                                                                float *__restrict__ out, const float *__restrict__ y,
                                                                const float *__restrict__ w)
{
    constexpr int PS = NT + 4;  // stride of a staged axial profile (floats; float4-aligned)
    __shared__ float s_w[kHxWarps][32][kHxMaxSpan + 1];
    __shared__ int s_c[kHxWarps][32];
    __shared__ int s_n[kHxWarps][32];
    __shared__ int s_part[kHxWarps];
    __shared__ float s_rc[NT];
    extern __shared__ float4 s_dyn4[];
    float *s_p = reinterpret_cast<float *>(s_dyn4);  // [warp][32][PS] profiles; later [warp][NT][32] partial sums
    int *s_pre = reinterpret_cast<int *>(s_p + kHxWarps * 32 * PS);  // [nmax + 1] wedge columns before march index a
    int *s_lo = s_pre + max(G.nx, G.ny) + 1;                          // [nmax] first wedge column at march index a
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = (G.ns + 31) >> 5;
    const int k = blockIdx.x / nb;
    const int s0 = (blockIdx.x - k * nb) * 32;
    const int v = __ldg(&views[k]);
    const float2 cs = __ldg(&G.view_cs[v]);
    const float beta = __ldg(&G.view_beta[v]);
    const float2 zb = __ldg(&H.view_zb[v]);
    if (threadIdx.x < NT) s_rc[threadIdx.x] = threadIdx.x < H.nt ? __ldg(&H.row_c[threadIdx.x]) : 0.0f;
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
    {   // wedge columns per march index, then an exclusive scan over the CTA
        const float TB1 = march_slope(M, a_lo), TB2 = march_slope(M, a_hi);
        const int per = (nm + kHxWarps * 32 - 1) / (kHxWarps * 32);
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
        if (threadIdx.x == kHxWarps * 32 - 1) s_pre[nm] = pos;
        __syncthreads();
    }
    const int T = s_pre[nm];
    const int s_mine = s0 + lane;
    const float my_a = beta + fmaf((float)s_mine, G.dgamma, G.gamma0);
    const float t1 = march_slope(M, my_a - 0.5f * G.dgamma), t2 = march_slope(M, my_a + 0.5f * G.dgamma);
    float(*sw)[kHxMaxSpan + 1] = s_w[warp];
    int *scf = s_c[warp];
    int *sns = s_n[warp];
    float *sp = s_p + (size_t)warp * 32 * PS;
    const int nt = H.nt, nz = H.nz;
    float acc[NT];
#pragma unroll
    for (int t = 0; t < NT; t++) acc[t] = 0.0f;
    const int t_end = (int)(((long)(warp + 1) * T) / kHxWarps);
    int t0 = (int)(((long)warp * T) / kHxWarps);
    int col = 0;
    while (t0 < t_end) {
        while (s_pre[col + 1] <= t0) col++;
        const int e = s_pre[min(col + lane + 1, nm)];
        const int n = min(min(32, t_end - t0), __shfl_sync(kFull, e, 31) - t0);
        const int t = t0 + lane;
        const int ls = min(count_le(e, t), 31);
        const int c = col + ls;
        int cf = 1 << 20, cnt = 0;
        if (lane < n) {  // column role: footprint weights and axial parameters of one column
            const int bc = s_lo[c] + (t - s_pre[c]);
            const int ix = M.col ? c : bc, iy = M.col ? bc : c;
            float px, py;
            const Anchor A = pixel_anchor(G, v, ix, iy, px, py);
            const float ox = px * G.dx, oy = py * G.dy;
            const size_t ai = (size_t)v * (G.nax * G.nay) + (iy / kAnchor) * G.nax + ix / kAnchor;
            const Footprint F = sf_footprint(G, cs.x, cs.y, A, px, py);
            cnt = foot_cells(F, kHxMaxSpan, [&](int i, float a) { sw[lane][i] = a * F.amp; });
            cf = F.n + foot_first(F) - s0;
            // axial parameters; the lowest and highest row boundaries give the voxel range
            const float4 X = __ldg(&H.tile_ax[ai]);
            float eps;
            const ColumnAxial C = column_axial<TT>(H, A, X, cs.x, cs.y, ox, oy, G.dx, G.dy, eps);
            const float cz = fmaf(H.ofr, C.ia_hi + C.ia_lo, -zb.y);
            int K0, K1;
            float f0, f1;
            row_boundary(-0.5f - H.ct0i, C.ia_hi, C.ia_lo, zb.x, cz, nz, K0, f0);
            row_boundary((float)nt - 0.5f - H.ct0i, C.ia_hi, C.ia_lo, zb.x, cz, nz, K1, f1);
            // the widest ramp the column's row boundaries can meet (|z - z_src| is convex in K)
            const float zbf = zb.x + zb.y;
            const float hcol = TT ? eps * fmaxf(fabsf((float)K0 + zbf), fabsf((float)(K1 + 1) + zbf)) : 0.0f;
            // the column's axial profile, its rows in order:
            // p_r = a * sum_k x_k |[k, k+1] ∩ [z(r - 1/2), z(r + 1/2)]|, each row boundary placed exactly
            // (row_boundary), the voxels read from the column's contiguous z-run (L1); TT adds at every
            // row boundary the ramp corrections, + to the row below, - to the row above
            const float4 P = make_float4(C.ia_hi, C.ia_lo, C.a_hi + C.a_lo, cz);
            const float *xg = x + ((size_t)iy * G.nx + ix) * nz;
            auto xv = [&](int kk) -> float {
                if (kk < 0 || kk >= nz) return 0.0f;
                return (MODE == FP_ONES_W) ? 1.0f : __ldg(&xg[kk]);
            };
            const float eps_l = eps;
            int Kl = K0;
            float fl = f0;
            // voxels Kl - 1 .. Kl + 2 of the column in registers (0 outside the volume): the rows walk up
            // the column, so a row's voxels and the ramp corrections at its upper boundary come from the
            // window, and the one new voxel a shift by one needs is loaded a row before it is used
            float w0 = xv(Kl - 1), w1 = xv(Kl), w2 = xv(Kl + 1), w3 = xv(Kl + 2);
            float cl = TT ? ramp_correction_w(Kl, fl, eps_l, zbf, w0, w1, w2) : 0.0f;
            float *pl = sp + lane * PS;
            for (int r = 0; r < nt; r++) {
                int Kh;
                float fh;
                row_boundary((float)r + 0.5f - H.ct0i, P.x, P.y, zb.x, P.w, nz, Kh, fh);
                // this row: voxels Kl .. Kh, the first from fl, the last to fh
                const int d = Kh - Kl;
                const float c1 = d == 0 ? fh - fl : 1.0f - fl;
                const float c2 = d == 1 ? fh : (d >= 2 ? 1.0f : 0.0f);
                const float c3 = d == 2 ? fh : (d >= 3 ? 1.0f : 0.0f);
                float rs = fmaf(w1, c1, fmaf(w2, c2, w3 * c3));
                if (d >= 3) {  // a row spanning more than three voxels
                    for (int kk = Kl + 3; kk < Kh; kk++) rs += xv(kk);
                    rs = fmaf(xv(Kh), fh, rs);
                }
                // shift the window to Kh - 1 .. Kh + 2
                if (d == 1) {
                    w0 = w1; w1 = w2; w2 = w3; w3 = xv(Kh + 2);
                } else if (d == 2) {
                    w0 = w2; w1 = w3; w2 = xv(Kh + 1); w3 = xv(Kh + 2);
                } else if (d != 0) {
                    w0 = xv(Kh - 1); w1 = xv(Kh); w2 = xv(Kh + 1); w3 = xv(Kh + 2);
                }
                float sacc = rs;
                if (TT) {
                    const float ch = (fminf(fh, 1.0f - fh) < hcol) ? ramp_correction_w(Kh, fh, eps_l, zbf, w0, w1, w2) : 0.0f;
                    sacc += ch - cl;
                    cl = ch;
                }
                pl[r] = P.z * sacc;
                Kl = Kh;
                fl = fh;
            }
            for (int r = nt; r < NT; r++) pl[r] = 0.0f;  // rows the float4 reads below cover
        }
        scf[lane] = cf;
        sns[lane] = cnt;
        __syncwarp();
        // cell role: add weight x profile of every staged column this lane's wedge crosses
        const int lmax = __shfl_sync(kFull, ls, n - 1);
        for (int l = 0; l <= lmax; l++) {
            const int cc = col + l;
            const int pre_c = s_pre[cc];
            const int task_lo = max(pre_c, t0), task_hi = min(__shfl_sync(kFull, e, l), t0 + n);
            const int row0 = s_lo[cc] - pre_c;
            int q_lo, q_hi;
            wedge_range(M, cc, t1, t2, q_lo, q_hi);
            q_lo = max(q_lo, row0 + task_lo);
            q_hi = min(q_hi, row0 + task_hi - 1);
            for (int q = q_lo; q <= q_hi; q++) {
                const int slot = q - row0 - t0;
                const int i = lane - scf[slot];
                if ((unsigned)i < (unsigned)sns[slot]) {
                    const float wt = sw[slot][i];
                    const float4 *p4 = reinterpret_cast<const float4 *>(sp + slot * PS);
#pragma unroll
                    for (int r4 = 0; r4 < NT / 4; r4++) {
                        const float4 p = p4[r4];
                        acc[4 * r4 + 0] = fmaf(wt, p.x, acc[4 * r4 + 0]);
                        acc[4 * r4 + 1] = fmaf(wt, p.y, acc[4 * r4 + 1]);
                        acc[4 * r4 + 2] = fmaf(wt, p.z, acc[4 * r4 + 2]);
                        acc[4 * r4 + 3] = fmaf(wt, p.w, acc[4 * r4 + 3]);
                    }
                }
            }
        }
        __syncwarp();
        t0 += n;
    }
    // warps' partial sums, added in a fixed order
    __syncthreads();
    float *red = s_p;  // [warp][NT][32]
#pragma unroll
    for (int r = 0; r < NT; r++) red[(warp * NT + r) * 32 + lane] = acc[r];
    __syncthreads();
    for (int q = threadIdx.x; q < NT * 32; q += kHxWarps * 32) {
        const int r = q >> 5, l = q & 31, s = s0 + l;
        if (r >= nt || s >= G.ns) continue;
        float sum = 0.0f;
#pragma unroll
        for (int wq = 0; wq < kHxWarps; wq++) sum += red[(wq * NT + r) * 32 + l];
        sum *= s_rc[r];
        const size_t ri = ((size_t)v * nt + r) * G.ns + s;
        const size_t oi = ((size_t)k * nt + r) * G.ns + s;
        if (MODE == FP_PLAIN) out[oi] = sum;
        else if (MODE == FP_RESID) out[oi] = __ldg(&w[ri]) * (sum - __ldg(&y[ri]));
        else out[ri] = __ldg(&w[ri]) * sum;
    }
}

template <int MODE>
__device__ __forceinline__ void bp_helix_epilogue(const SolveDev &S, float *__restrict__ xo, size_t j, float acc,
                                                  float rho, float scale, int accumulate)
{
    if (MODE == BP_PLAIN) {
        xo[j] = accumulate ? fmaf(scale, acc, xo[j]) : scale * acc;
        return;
    }
    const float zeta = S.M_scale * acc;  // M grad L_m
    if (MODE == BP_SOLVE_INIT) {
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

// Row position of voxel boundary k of a column: its row coordinate is
// u + 1/2 = (k + zbi)(a_hi + a_lo) + zbf a + ct0i + 1/2 - ofr = r + fr (row r,
// 0 <= fr < 1); with k + zbi and ct0i + 1/2 - r exact, fr comes from one fma
// at magnitude ~1.  cb0 = zbf a - ofr.
struct RowPos {
    int r;
    float fr;
};

__device__ __forceinline__ RowPos row_pos(int k, float zbi, float a_hi, float a_lo, float cb0, float c_half, int nt)
{
    const float Z = (float)k + zbi;
    const float sm = fmaf(Z, a_lo, cb0);
    const float approx = fmaf(Z, a_hi, sm + c_half);
    RowPos p;
    p.r = (int)floorf(fminf(fmaxf(approx, -2.0f), (float)nt + 1.0f));
    p.fr = fmaf(Z, a_hi, c_half - (float)p.r) + sm;
    if (p.fr < 0.0f) { p.r -= 1; p.fr += 1.0f; }
    else if (p.fr >= 1.0f) { p.r += 1; p.fr -= 1.0f; }
    return p;
}

// Running sum of the row sums at a voxel boundary, over rows [t_lo, t_lo + nr):
// qb[i] = sum of q over the first i rows, linear inside a row.
__device__ __forceinline__ float row_cdf(const float *qb, RowPos p, int t_lo, int nr)
{
    const int rel = p.r - t_lo;
    if (rel < 0) return 0.0f;
    if (rel >= nr) return qb[nr * kHxBpCols];
    const float lo = qb[rel * kHxBpCols], hi = qb[(rel + 1) * kHxBpCols];
    return fmaf(p.fr, hi - lo, lo);
}

// TT: adjoint of the ramp correction of voxel boundary k (at row position p,
// ramp half-width hw rows): sum over the row boundaries the ramp straddles of
// (hw - d)^2 / (4 hw) (q below - q above); voxel k receives +, voxel k-1 -.
__device__ __forceinline__ float ramp_adjoint(const float *qb, RowPos p, float hw, int t_lo, int nr)
{
    auto q = [&](int t) -> float {
        const int i = t - t_lo;
        return (i >= 0 && i < nr) ? qb[(i + 1) * kHxBpCols] - qb[i * kHxBpCols] : 0.0f;
    };
    float D = 0.0f;
    if (p.fr < hw) {
        const float d = hw - p.fr;
        D = __fdividef(d * d, 4.0f * hw) * (q(p.r - 1) - q(p.r));
    }
    const float g = 1.0f - p.fr;
    if (g < hw) {
        const float d = hw - g;
        D = fmaf(__fdividef(d * d, 4.0f * hw), q(p.r) - q(p.r + 1), D);
    }
    return D;
}

template <int MODE, int ZC, bool TT>
__global__ void __launch_bounds__(kHxBpCols) bp_helix_kernel(FanDev G, HelixDev H, const float *__restrict__ sino,
                                                             const int *__restrict__ views, int nviews,
                                                             float *__restrict__ xo, float scale, int accumulate,
                                                             SolveDev S)
{
    __shared__ float s_qb[(kHxQMax + 1) * kHxBpCols];
    __shared__ float s_w[kHxMaxSpan * kHxBpCols];
    __shared__ float s_rc[kHxMaxRows];
    const int tid = threadIdx.x;
    const int ix = blockIdx.x * 16 + (tid & 15), iy = blockIdx.y * 8 + (tid >> 4);
    const int z0 = blockIdx.z * ZC;
    if (tid < kHxMaxRows) s_rc[tid] = tid < H.nt ? __ldg(&H.row_c[tid]) : 0.0f;
    __syncthreads();
    const bool inside = ix < G.nx && iy < G.ny;
    const int ixc = min(ix, G.nx - 1), iyc = min(iy, G.ny - 1);
    const int atile = (iyc / kAnchor) * G.nax + ixc / kAnchor;
    const int ntiles = G.nax * G.nay;
    const float px = (float)(ixc - (ixc / kAnchor) * kAnchor) - kAnchorHalf;
    const float py = (float)(iyc - (iyc / kAnchor) * kAnchor) - kAnchorHalf;
    const float ox = px * G.dx, oy = py * G.dy;
    float *qb = s_qb + tid;
    float *wq = s_w + tid;
    float rho = 1.0f;
    if (MODE == BP_SOLVE_UPDATE) rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float acc[ZC];
#pragma unroll
    for (int i = 0; i < ZC; i++) acc[i] = 0.0f;
    const int nt = H.nt;
    if (inside) {
        for (int k = 0; k < nviews; k++) {
            const int v = __ldg(&views[k]);
            const float2 cs = __ldg(&G.view_cs[v]);
            const Anchor A = load_anchor(G, v, atile);
            const float2 zb = __ldg(&H.view_zb[v]);
            float eps;
            const ColumnAxial Cx = column_axial<TT>(H, A, __ldg(&H.tile_ax[(size_t)v * ntiles + atile]), cs.x, cs.y,
                                                    ox, oy, G.dx, G.dy, eps);
            const float a = Cx.a_hi + Cx.a_lo;
            const float zbf = zb.x + zb.y;
            // rows the chunk's shadow reaches (approximate ends, widened by 1e-3 row and, with
            // trapezoids, by the end faces' ramp half-widths)
            const float ea = eps * a;
            const float hwA = TT ? ea * fabsf((float)z0 + zbf) : 0.0f;
            const float hwB = TT ? ea * fabsf((float)(z0 + ZC) + zbf) : 0.0f;
            const float uA = fmaf(a, (float)z0 + zbf, H.ct0);
            const float uB = fmaf(a, (float)ZC, uA);
            const int t_lo = (int)fmaxf(floorf(uA - hwA + 0.499f), 0.0f);
            const int t_hi = (int)fminf(floorf(uB + hwB + 0.501f), (float)(nt - 1));
            if (t_lo > t_hi) continue;  // the chunk's shadow misses the detector in this view
            const Footprint F = sf_footprint(G, cs.x, cs.y, A, px, py);
            const int sfirst = F.n + foot_first(F);
            const int cnt = foot_cells(F, kHxMaxSpan, [&](int i, float a) {
                const int s = sfirst + i;
                wq[i * kHxBpCols] = ((unsigned)s < (unsigned)G.ns) ? a * F.amp : 0.0f;
            });
            const int i0 = max(-sfirst, 0);
            const int i1 = min(cnt, G.ns - sfirst);
            // running sums of q_t = c_t sum_s w_s y[t][s] over rows t_lo..t_hi
            float Q = 0.0f;
            qb[0] = 0.0f;
            for (int t = t_lo; t <= t_hi; t++) {
                const float *row = sino + ((size_t)k * nt + t) * G.ns;
                float d = 0.0f;
                for (int i = i0; i < i1; i++) d = fmaf(wq[i * kHxBpCols], __ldg(&row[sfirst + i]), d);
                Q = fmaf(s_rc[t], d, Q);
                qb[(t - t_lo + 1) * kHxBpCols] = Q;
            }
            const int nr = t_hi - t_lo + 1;
            const float cb0 = fmaf(zb.y, a, -H.ofr);
            const float c_half = H.ct0i + 0.5f;
            RowPos pp = row_pos(z0, zb.x, Cx.a_hi, Cx.a_lo, cb0, c_half, nt);
            float Cp = row_cdf(qb, pp, t_lo, nr);
            const float hw_max = fmaxf(hwA, hwB);  // the widest ramp of the chunk (rows)
            float Dp = (TT && fminf(pp.fr, 1.0f - pp.fr) < hw_max) ? ramp_adjoint(qb, pp, hwA, t_lo, nr) : 0.0f;
#pragma unroll
            for (int i = 0; i < ZC; i++) {
                const RowPos p = row_pos(z0 + i + 1, zb.x, Cx.a_hi, Cx.a_lo, cb0, c_half, nt);
                const float C = row_cdf(qb, p, t_lo, nr);
                acc[i] += C - Cp;
                Cp = C;
                if (TT) {
                    const float D = fminf(p.fr, 1.0f - p.fr) < hw_max
                                        ? ramp_adjoint(qb, p, ea * fabsf((float)(z0 + i + 1) + zbf), t_lo, nr)
                                        : 0.0f;
                    acc[i] += Dp - D;
                    Dp = D;
                }
            }
        }
        const size_t jc = ((size_t)iy * G.nx + ix) * H.nz;
#pragma unroll
        for (int i = 0; i < ZC; i++)
            if (z0 + i < H.nz) bp_helix_epilogue<MODE>(S, xo, jc + z0 + i, acc[i], rho, scale, accumulate);
    }
    if (MODE == BP_SOLVE_UPDATE) {
        // the last block to finish advances the subiteration counter (rho for the next one)
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const int done = atomicAdd(&S.counter[1], 1);
            if (done == (int)(gridDim.x * gridDim.y * gridDim.z) - 1) {
                S.counter[1] = 0;
                S.counter[0] += 1;
                __threadfence();
            }
        }
    }
}

// ---------------------------------------------------------------- regularizer (13 directions, 26 neighbours)

struct VolDims {
    int nx, ny, nz;
    long long sx, sy, sz;  // element strides along x, y, z
};

// grad R_j = kappa_j sum over the 26 neighbours n of beta/||s|| kappa_n phi'(x_j - x_n);
// D_R,j = kappa_j sum 2 beta/||s|| kappa_n omega(x_j - x_n) (pairs outside the volume absent;
// KAPPA = false: kappa = 1 and the pointer is not read).
template <bool KAPPA>
__device__ __forceinline__ void reg_terms3(const float *__restrict__ x, const float *__restrict__ kappa,
                                           const VolDims &D, int ix, int iy, int iz, long long j, float beta, Pot P,
                                           float &grad, float &curv)
{
    const float xj = __ldg(&x[j]);
    const float b1 = beta, b2 = beta * 0.70710678118654752f, b3 = beta * 0.57735026918962576f;
    grad = 0.0f;
    curv = 0.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; dz++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) {
                const int n2 = dx * dx + dy * dy + dz * dz;
                if (n2 == 0) continue;
                const int fx = ix + dx, fy = iy + dy, fz = iz + dz;
                if (fx < 0 || fx >= D.nx || fy < 0 || fy >= D.ny || fz < 0 || fz >= D.nz) continue;
                const long long n = j + dx * D.sx + dy * D.sy + dz * D.sz;
                const float b0 = n2 == 1 ? b1 : (n2 == 2 ? b2 : b3);
                const float bi = KAPPA ? b0 * __ldg(&kappa[n]) : b0;
                float d, o;
                P.eval(xj - __ldg(&x[n]), d, o);
                grad = fmaf(bi, d, grad);
                curv = fmaf(2.0f * bi, P.maxcurv ? 1.0f : o, curv);
            }
    if (KAPPA) {
        const float kj = __ldg(&kappa[j]);
        grad *= kj;
        curv *= kj;
    }
}

// One thread per voxel in memory order of a volume with strides D.
template <bool KAPPA>
__global__ void __launch_bounds__(256) reg_gradient3_kernel(VolDims D, int zfast, const float *__restrict__ x,
                                                           const float *__restrict__ kappa, float beta, Pot P,
                                                           float *__restrict__ grad, float *__restrict__ curv)
{
    const long long n = (long long)D.nx * D.ny * D.nz;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int ix, iy, iz;
    if (zfast) {
        iz = (int)(j % D.nz);
        const long long c = j / D.nz;
        ix = (int)(c % D.nx);
        iy = (int)(c / D.nx);
    } else {
        ix = (int)(j % D.nx);
        const long long c = j / D.nx;
        iy = (int)(c % D.ny);
        iz = (int)(c / D.ny);
    }
    float gr, cv;
    reg_terms3<KAPPA>(x, kappa, D, ix, iy, iz, j, beta, P, gr, cv);
    grad[j] = gr;
    if (curv) curv[j] = cv;
}

// Fused x-update of Algorithm 1/2 on a column-major volume.
template <bool KAPPA>
__global__ void __launch_bounds__(256) reg_update3_kernel(VolDims D, SolveDev S, float beta, Pot P)
{
    const long long n = (long long)D.nx * D.ny * D.nz;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int iz = (int)(j % D.nz);
    const long long c = j / D.nz;
    const int ix = (int)(c % D.nx), iy = (int)(c / D.nx);
    const float rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float gr, cv;
    reg_terms3<KAPPA>(S.x, S.kappa, D, ix, iy, iz, j, beta, P, gr, cv);
    const float xj = S.x[j], dl = S.d_l[j], g = S.g[j], h = S.h[j];
    const float s = (S.algorithm == CT_ALG_PROPOSED) ? fmaf(rho, fmaf(dl, xj, -h), (1.0f - rho) * g)
                                                     : fmaf(rho, h, (1.0f - rho) * g);
    const float den = fmaf(rho, dl, cv);
    float xn = den > 0.0f ? xj - (s + gr) / den : xj;
    if (S.nonneg) xn = fmaxf(xn, 0.0f);
    S.x_new[j] = xn;
}

// RMSD over the field-of-view cylinder of a column-major volume (see the 2-D
// rmsd kernel: per-block partial sums, the last block writes the trace entry).
__global__ void __launch_bounds__(256) rmsd3_kernel(FanDev G, int nz, const float *__restrict__ x,
                                                    const float *__restrict__ xr, float r2max,
                                                    double *__restrict__ partial, int *__restrict__ counter,
                                                    float *__restrict__ trace, int M, float hu)
{
    __shared__ double ss[256];
    __shared__ double sc[256];
    double s = 0.0, c = 0.0;
    const long long n = (long long)G.nx * G.ny * nz;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const long long col = j / nz;
        const int ix = (int)(col % G.nx), iy = (int)(col / G.nx);
        const float X = ((float)ix - G.cxo) * G.dx, Y = ((float)iy - G.cyo) * G.dy;
        if (fmaf(X, X, Y * Y) <= r2max) {
            const double d = (double)x[j] - (double)xr[j];
            s += d * d;
            c += 1.0;
        }
    }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = ss[0];
        partial[2 * blockIdx.x + 1] = sc[0];
        __threadfence();
        const int done = atomicAdd(&counter[2], 1);
        if (done == (int)gridDim.x - 1) {
            __threadfence();
            double S = 0.0, C = 0.0;
            for (int b = 0; b < (int)gridDim.x; b++) {
                S += __ldcg(&partial[2 * b]);
                C += __ldcg(&partial[2 * b + 1]);
            }
            const int it = __ldcg(&counter[0]) / M - 1;
            trace[it] = C > 0 ? (float)(sqrt(S / C) * hu) : 0.0f;
            counter[2] = 0;
        }
    }
}

// ---------------------------------------------------------------- layout changes

// dst[c][r] = src[r][c] for an R x C matrix (tiles of 32 x 32 through shared memory).
__global__ void __launch_bounds__(256) transpose_kernel(const float *__restrict__ src, float *__restrict__ dst,
                                                        long long R, long long C, float scale, int accumulate)
{
    __shared__ float tile[32][33];
    const long long tiles_c = (C + 31) / 32;
    const long long c0 = ((long long)blockIdx.x % tiles_c) * 32, r0 = ((long long)blockIdx.x / tiles_c) * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const long long r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = __ldg(&src[r * C + c]);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const long long c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) {
            const float v = scale * tile[threadIdx.x][i];
            dst[c * R + r] = accumulate ? dst[c * R + r] + v : v;
        }
    }
}

cudaError_t transpose(const float *src, float *dst, long long R, long long C, float scale, int accumulate,
                      cudaStream_t st)
{
    const long long tiles = ((C + 31) / 32) * ((R + 31) / 32);
    transpose_kernel<<<(unsigned)tiles, dim3(32, 8), 0, st>>>(src, dst, R, C, scale, accumulate);
    return cudaGetLastError();
}

Pot make_pot(int potential, float delta, int maxcurv = 0)
{
    return Pot{potential, potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / delta, maxcurv};
}

template <int MODE, bool TT>
cudaError_t fp_helix_dispatch(const ct_geom *g, const float *x, const int *views, int nviews, float *out,
                              const float *y, const float *w, cudaStream_t st)
{
    const FanDev &G = g->fan;
    const HelixDev &H = g->hx;
    const unsigned blocks = (unsigned)nviews * (unsigned)((G.ns + 31) / 32);
    const int nt = H.nt;
    const int nmax = G.nx > G.ny ? G.nx : G.ny;
#define CT_FP_HX(NTV)                                                                                       \
    fp_helix_kernel<MODE, NTV, TT><<<blocks, kHxWarps * 32,                                                 \
                                     sizeof(float) * kHxWarps * 32 * (NTV + 4) + sizeof(int) * (2 * nmax + 1), \
                                     st>>>(G, H, x, views, nviews, out, y, w)
    if (nt <= 8) CT_FP_HX(8);
    else if (nt <= 16) CT_FP_HX(16);
    else if (nt <= 32) CT_FP_HX(32);
    else {
        const size_t dyn = sizeof(float) * kHxWarps * 32 * (64 + 4) + sizeof(int) * (2 * nmax + 1);
        cudaError_t e = cudaFuncSetAttribute(fp_helix_kernel<MODE, 64, TT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        CT_FP_HX(64);
    }
#undef CT_FP_HX
    return cudaGetLastError();
}

template <int MODE, bool TT>
cudaError_t bp_helix_dispatch(const ct_geom *g, const float *sino, const int *views, int nviews, float *x,
                              float scale, int accumulate, const SolveDev &S, cudaStream_t st)
{
    const FanDev &G = g->fan;
    const HelixDev &H = g->hx;
    const int zc = g->hx_zc;
    dim3 grid((G.nx + 15) / 16, (G.ny + 7) / 8, (H.nz + zc - 1) / zc);
#define CT_BP_HX(Z) bp_helix_kernel<MODE, Z, TT><<<grid, kHxBpCols, 0, st>>>(G, H, sino, views, nviews, x, scale, accumulate, S)
    switch (zc) {
    case 16: CT_BP_HX(16); break;
    case 8: CT_BP_HX(8); break;
    case 4: CT_BP_HX(4); break;
    case 2: CT_BP_HX(2); break;
    default: CT_BP_HX(1); break;
    }
#undef CT_BP_HX
    return cudaGetLastError();
}

}  // namespace

int helix_chunk_voxels(double a_max, double extra_rows)
{
    for (int zc = 16; zc >= 1; zc >>= 1)
        if (std::ceil(zc * a_max + extra_rows) + 2.0 <= (double)kHxQMax) return zc;
    return 0;
}

int helix_max_rows() { return kHxMaxRows; }
int helix_max_span() { return kHxMaxSpan; }
int helix_max_march() { return kHxMaxMarch; }

cudaError_t launch_fp_helix(const ct_geom *g, int mode, const float *x, const int *views, int nviews, float *out,
                            const float *y, const float *w, cudaStream_t st)
{
    const bool tt = g->hx.trap != 0;
    switch (mode) {
    case FP_PLAIN:
        return tt ? fp_helix_dispatch<FP_PLAIN, true>(g, x, views, nviews, out, y, w, st)
                  : fp_helix_dispatch<FP_PLAIN, false>(g, x, views, nviews, out, y, w, st);
    case FP_RESID:
        return tt ? fp_helix_dispatch<FP_RESID, true>(g, x, views, nviews, out, y, w, st)
                  : fp_helix_dispatch<FP_RESID, false>(g, x, views, nviews, out, y, w, st);
    default:
        return tt ? fp_helix_dispatch<FP_ONES_W, true>(g, x, views, nviews, out, y, w, st)
                  : fp_helix_dispatch<FP_ONES_W, false>(g, x, views, nviews, out, y, w, st);
    }
}

cudaError_t launch_bp_helix(const ct_geom *g, int mode, const float *sino, const int *views, int nviews, float *x,
                            float scale, int accumulate, const SolveDev *S, cudaStream_t st)
{
    SolveDev s0{};
    const SolveDev &SS = S ? *S : s0;
    const bool tt = g->hx.trap != 0;
    switch (mode) {
    case BP_PLAIN:
        return tt ? bp_helix_dispatch<BP_PLAIN, true>(g, sino, views, nviews, x, scale, accumulate, SS, st)
                  : bp_helix_dispatch<BP_PLAIN, false>(g, sino, views, nviews, x, scale, accumulate, SS, st);
    case BP_SOLVE_INIT:
        return tt ? bp_helix_dispatch<BP_SOLVE_INIT, true>(g, sino, views, nviews, x, scale, accumulate, SS, st)
                  : bp_helix_dispatch<BP_SOLVE_INIT, false>(g, sino, views, nviews, x, scale, accumulate, SS, st);
    default:
        return tt ? bp_helix_dispatch<BP_SOLVE_UPDATE, true>(g, sino, views, nviews, x, scale, accumulate, SS, st)
                  : bp_helix_dispatch<BP_SOLVE_UPDATE, false>(g, sino, views, nviews, x, scale, accumulate, SS, st);
    }
}

static VolDims column_dims(const ct_geom *g)
{
    const int nx = g->fan.nx, ny = g->fan.ny, nz = g->hx.nz;
    return VolDims{nx, ny, nz, (long long)nz, (long long)nx * nz, 1};
}

cudaError_t launch_reg_gradient_helix(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                                      int potential, float *grad, float *curv, cudaStream_t st)
{
    // the C ABI's layout, [iz][iy][ix]
    const int nx = g->fan.nx, ny = g->fan.ny, nz = g->hx.nz;
    const VolDims D{nx, ny, nz, 1, (long long)nx, (long long)nx * ny};
    const long long n = (long long)nx * ny * nz;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (kappa)
        reg_gradient3_kernel<true><<<blocks, 256, 0, st>>>(D, 0, x, kappa, beta, make_pot(potential, delta), grad, curv);
    else
        reg_gradient3_kernel<false><<<blocks, 256, 0, st>>>(D, 0, x, kappa, beta, make_pot(potential, delta), grad, curv);
    return cudaGetLastError();
}

cudaError_t launch_reg_update_helix(const ct_geom *g, const SolveDev &S, float beta, float delta, int potential,
                                    int maxcurv, cudaStream_t st)
{
    const VolDims D = column_dims(g);
    const long long n = (long long)D.nx * D.ny * D.nz;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (S.kappa)
        reg_update3_kernel<true><<<blocks, 256, 0, st>>>(D, S, beta, make_pot(potential, delta, maxcurv));
    else
        reg_update3_kernel<false><<<blocks, 256, 0, st>>>(D, S, beta, make_pot(potential, delta, maxcurv));
    return cudaGetLastError();
}

cudaError_t launch_rmsd_helix(const ct_geom *g, const float *x, const float *xr, float r2max, double *partial,
                              int *counter, float *trace, int M, float hu, cudaStream_t st)
{
    rmsd3_kernel<<<152, 256, 0, st>>>(g->fan, g->hx.nz, x, xr, r2max, partial, counter, trace, M, hu);
    return cudaGetLastError();
}

cudaError_t launch_to_columns(const ct_geom *g, const float *src, float *dst, cudaStream_t st)
{
    return transpose(src, dst, g->hx.nz, (long long)g->fan.nx * g->fan.ny, 1.0f, 0, st);
}

cudaError_t launch_to_slices(const ct_geom *g, const float *src, float *dst, float scale, int accumulate,
                             cudaStream_t st)
{
    return transpose(src, dst, (long long)g->fan.nx * g->fan.ny, g->hx.nz, scale, accumulate, st);
}

ct_status helix_forward(const ct_geom *g, const float *x, float *y, const int *views, int nviews, cudaStream_t st)
{
    const int *dv = nullptr;
    ct_status s = stage_views(g, views, nviews, &dv, st);
    if (s != CT_OK) return s;
    CT_CUDA_TRY(launch_to_columns(g, x, g->d_vol_ws, st), "ct_forward layout");
    CT_CUDA_TRY(launch_fp_helix(g, FP_PLAIN, g->d_vol_ws, dv, nviews, y, nullptr, nullptr, st), "ct_forward launch");
    return CT_OK;
}

ct_status helix_back(const ct_geom *g, const float *y, float *x, const int *views, int nviews, float scale,
                     int accumulate, cudaStream_t st)
{
    const int *dv = nullptr;
    ct_status s = stage_views(g, views, nviews, &dv, st);
    if (s != CT_OK) return s;
    CT_CUDA_TRY(launch_bp_helix(g, BP_PLAIN, y, dv, nviews, g->d_vol_ws, 1.0f, 0, nullptr, st), "ct_back launch");
    CT_CUDA_TRY(launch_to_slices(g, g->d_vol_ws, x, scale, accumulate, st), "ct_back layout");
    return CT_OK;
}

ct_status helix_sqs_diag(const ct_geom *g, const float *w, float *d_l, cudaStream_t st)
{
    const int na = g->fan.na;
    CT_CUDA_TRY(ensure_ray_sums(const_cast<ct_geom *>(g), st), "ct_sqs_diag ray sums");
    CT_CUDA_TRY(launch_weighted_ray_sums(g, w, g->d_sino_ws, st), "ct_sqs_diag weights");
    CT_CUDA_TRY(launch_bp_helix(g, BP_PLAIN, g->d_sino_ws, g->d_views_all, na, g->d_vol_ws, 1.0f, 0, nullptr, st),
                "ct_sqs_diag back");
    CT_CUDA_TRY(launch_to_slices(g, g->d_vol_ws, d_l, 1.0f, 0, st), "ct_sqs_diag layout");
    return CT_OK;
}

ct_status helix_reg_gradient(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                             int potential, float *grad, float *curv, cudaStream_t st)
{
    CT_CUDA_TRY(launch_reg_gradient_helix(g, x, kappa, beta, delta, potential, grad, curv, st),
                "ct_reg_gradient launch");
    return CT_OK;
}

}  // namespace ct
