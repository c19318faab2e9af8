/*
 * ORACLE -- test infrastructure only.  Plain FP64 separable-footprint
 * projector (trapezoid x rectangle, "SF-TR") for 3-D helical cone-beam CT
 * with a cylindrical (arc) detector.  Loaded only by the tests, the smoke
 * check and the benchmark's CPU-baseline leg; shares no code with the CUDA
 * library.
 *
 * System matrix of the PWLS problem (Sec. III, Eq. (ct_problem)) for the 3-D
 * helical scans of Sec. IV (separable-footprint projector):
 *
 *   a_{(v,t,s),j} = l_xy(j) * c_t * T_j(s) * R_j(t)
 *
 *   T_j(s) = (1/dgamma) * integral over cell s of the transaxial unit
 *            trapezoid whose vertices are the fan angles of the four (x, y)
 *            corners of voxel j's column (the 2-D fan-beam footprint);
 *   l_xy   = chord through the column's (x, y) square along the transaxial
 *            ray through its centre, min(dx/|cos theta|, dy/|sin theta|);
 *   R_j(t) = (1/dt) * length of the overlap of detector row t with the
 *            voxel's z-extent magnified onto the detector: a voxel at
 *            transaxial distance L from the source spans heights
 *            (z - z_src) * dsd / L for z in [z_j - dz/2, z_j + dz/2];
 *   c_t    = sqrt(1 + (v_t / dsd)^2) = 1 / cos(cone angle of row t): the
 *            ray through row t (height v_t on the cylinder at dsd) crosses
 *            the voxel over l_xy / cos(cone angle).
 *
 * With axial = 1 the axial factor is a trapezoid instead (SF-TT, the other
 * axial model of the cited separable-footprint method):
 *
 *   R_j(t) = (1/dt) * integral over row t of the unit trapezoid whose
 *            vertices are the detector heights of the voxel's two z-faces
 *            seen from the nearest and the farthest of its column's four
 *            (x, y) corners (transaxial distances L_min, L_max): the shadow's
 *            edges smeared over the range of magnifications the voxel spans.
 *
 * Geometry: voxel (ix, iy, iz) centred at ((ix-(nx-1)/2+ox) dx,
 * (iy-(ny-1)/2+oy) dy, (iz-(nz-1)/2+oz) dz); view v at angle
 * beta_v = orbit_start + v * orbit / na (orbit may span several turns);
 * source at (-dso cos b, -dso sin b, z_src) with
 * z_src = pitch * (nt dt dso / dsd) * (beta_v - beta_mid) / (2 pi), beta_mid
 * the mid-scan angle (pitch = table feed per turn over the detector's axial
 * coverage at the isocentre); cell s at fan angle (s-(ns-1)/2+offset_s) ds/dsd;
 * row t at height v_t = (t-(nt-1)/2+offset_t) dt on the detector.  Volumes
 * are [iz][iy][ix] (x fastest); sinograms [view][row][cell] (cell fastest).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, offset_x, offset_y, offset_z;
    int ns, nt, na;
    double ds, dt, offset_s, offset_t;
    double dso, dsd, orbit_deg, orbit_start_deg, pitch;
    int axial; /* 0: rectangle axial footprint (SF-TR); 1: trapezoid (SF-TT) */
} orc_helix_geom;

static double hx_beta(const orc_helix_geom *g, int v)
{
    return (g->orbit_start_deg + (double)v * g->orbit_deg / (double)g->na) * M_PI / 180.0;
}

static double hx_source_z(const orc_helix_geom *g, double beta)
{
    const double mid = (g->orbit_start_deg + 0.5 * g->orbit_deg) * M_PI / 180.0;
    const double cover = g->nt * g->dt * g->dso / g->dsd;
    return g->pitch * cover * (beta - mid) / (2.0 * M_PI);
}

/* row coordinate (in rows, row t centred at t) of detector height h */
static double hx_row_of(const orc_helix_geom *g, double h)
{
    return h / g->dt + ((g->nt - 1) / 2.0 - g->offset_t);
}

static double hx_cone_factor(const orc_helix_geom *g, int t)
{
    const double vt = ((double)t - (g->nt - 1) / 2.0 + g->offset_t) * g->dt;
    return sqrt(1.0 + (vt / g->dsd) * (vt / g->dsd));
}

/* integral of the unit trapezoid with sorted vertices t[0..3] over (-inf, u] */
static double hx_trap_cdf(const double t[4], double u)
{
    double area = 0.0;
    if (u <= t[0]) return 0.0;
    if (u < t[1]) { double d = u - t[0]; return d * d / (2.0 * (t[1] - t[0])); }
    area = 0.5 * (t[1] - t[0]);
    if (u < t[2]) return area + (u - t[1]);
    area += t[2] - t[1];
    if (u < t[3]) {
        double d = t[3] - u;
        return area + 0.5 * (t[3] - t[2]) - d * d / (2.0 * (t[3] - t[2]));
    }
    return area + 0.5 * (t[3] - t[2]);
}

/* Column (ix, iy) in the view with direction (cb, sb): trapezoid vertices in
 * cell units (cell s centred at s), chord l_xy, transaxial distance L of the
 * column's centre and the smallest and largest of its corners' (lmm[0..1]). */
static void hx_column(const orc_helix_geom *g, double cb, double sb, int ix, int iy, double tau[4], double *lxy,
                      double *L, double lmm[2])
{
    const double xc = ((double)ix - (g->nx - 1) / 2.0 + g->offset_x) * g->dx;
    const double yc = ((double)iy - (g->ny - 1) / 2.0 + g->offset_y) * g->dy;
    const double cells_per_rad = g->dsd / g->ds;
    const double c0 = (g->ns - 1) / 2.0 - g->offset_s;
    int k = 0;
    for (int sy = -1; sy <= 1; sy += 2)
        for (int sx = -1; sx <= 1; sx += 2) {
            /* corner relative to the source, in the view frame (along the central ray, across it) */
            const double px = xc + 0.5 * sx * g->dx + g->dso * cb, py = yc + 0.5 * sy * g->dy + g->dso * sb;
            const double along = px * cb + py * sb, across = -px * sb + py * cb;
            tau[k++] = atan2(across, along) * cells_per_rad + c0;
            const double lc = sqrt(px * px + py * py);
            if (k == 1 || lc < lmm[0]) lmm[0] = lc;
            if (k == 1 || lc > lmm[1]) lmm[1] = lc;
        }
    for (int i = 1; i < 4; i++) { /* insertion sort */
        double v = tau[i];
        int m = i - 1;
        while (m >= 0 && tau[m] > v) { tau[m + 1] = tau[m]; m--; }
        tau[m + 1] = v;
    }
    const double rx = xc + g->dso * cb, ry = yc + g->dso * sb;
    *L = sqrt(rx * rx + ry * ry);
    const double ac = fabs(rx) / *L, as = fabs(ry) / *L;
    const double lx = ac > 0.0 ? g->dx / ac : INFINITY, ly = as > 0.0 ? g->dy / as : INFINITY;
    *lxy = lx < ly ? lx : ly;
}

/* Visit every nonzero a_{(v,t,s),j} of view v with j in column (ix, iy);
 * iz_only >= 0 restricts j to that slice, s_only >= 0 the cells to that one. */
typedef void (*hx_visit)(void *ctx, int t, int s, size_t j, double a);

static void hx_view_column(const orc_helix_geom *g, int v, int ix, int iy, int iz_only, int s_only, hx_visit visit,
                           void *ctx)
{
    const double b = hx_beta(g, v), cb = cos(b), sb = sin(b), zsrc = hx_source_z(g, b);
    double tau[4], lxy, L, lmm[2];
    hx_column(g, cb, sb, ix, iy, tau, &lxy, &L, lmm);
    int s_lo = (int)floor(tau[0] - 0.5) + 1, s_hi = (int)ceil(tau[3] + 0.5) - 1;
    if (s_lo < 0) s_lo = 0;
    if (s_hi > g->ns - 1) s_hi = g->ns - 1;
    if (s_only >= 0) {
        if (s_only < s_lo || s_only > s_hi) return;
        s_lo = s_hi = s_only;
    }
    if (s_lo > s_hi) return;
    const double mag = g->dsd / L;
    const int iz_first = iz_only >= 0 ? iz_only : 0, iz_last = iz_only >= 0 ? iz_only : g->nz - 1;
    for (int iz = iz_first; iz <= iz_last; iz++) {
        const double zc = ((double)iz - (g->nz - 1) / 2.0 + g->offset_z) * g->dz;
        double u0, u1, ua[4];
        if (g->axial == 1) { /* trapezoid: each face at the near and the far magnification */
            const double zf[2] = {zc - 0.5 * g->dz - zsrc, zc + 0.5 * g->dz - zsrc};
            for (int f = 0; f < 2; f++)
                for (int m = 0; m < 2; m++) ua[2 * f + m] = hx_row_of(g, zf[f] * g->dsd / lmm[m]);
            for (int i = 1; i < 4; i++) { /* insertion sort */
                double v = ua[i];
                int q = i - 1;
                while (q >= 0 && ua[q] > v) { ua[q + 1] = ua[q]; q--; }
                ua[q + 1] = v;
            }
            u0 = ua[0];
            u1 = ua[3];
        } else {
            u0 = hx_row_of(g, (zc - 0.5 * g->dz - zsrc) * mag);
            u1 = hx_row_of(g, (zc + 0.5 * g->dz - zsrc) * mag);
        }
        int t_lo = (int)floor(u0 - 0.5) + 1, t_hi = (int)ceil(u1 + 0.5) - 1;
        if (t_lo < 0) t_lo = 0;
        if (t_hi > g->nt - 1) t_hi = g->nt - 1;
        const size_t j = ((size_t)iz * g->ny + iy) * g->nx + ix;
        for (int t = t_lo; t <= t_hi; t++) {
            double rt;
            if (g->axial == 1) {
                rt = hx_trap_cdf(ua, t + 0.5) - hx_trap_cdf(ua, t - 0.5);
                if (!(rt > 0.0)) continue;
            } else {
                const double lo = u0 > t - 0.5 ? u0 : t - 0.5, hi = u1 < t + 0.5 ? u1 : t + 0.5;
                if (hi <= lo) continue;
                rt = hi - lo;
            }
            const double ct = hx_cone_factor(g, t);
            for (int s = s_lo; s <= s_hi; s++) {
                const double ts = hx_trap_cdf(tau, s + 0.5) - hx_trap_cdf(tau, s - 0.5);
                if (ts > 0.0) visit(ctx, t, s, j, lxy * ct * ts * rt);
            }
        }
    }
}

static int hx_check(const orc_helix_geom *g)
{
    if (!g || g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->ns <= 0 || g->nt <= 0 || g->na <= 0) return 1;
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0) || !(g->ds > 0) || !(g->dt > 0) || !(g->dso > 0) ||
        !(g->dsd > 0))
        return 1;
    if (g->axial != 0 && g->axial != 1) return 1;
    return 0;
}

static int hx_check_views(const orc_helix_geom *g, const int *views, int nviews)
{
    for (int k = 0; k < nviews; k++)
        if (views[k] < 0 || views[k] >= g->na) return 1;
    return 0;
}

typedef struct {
    int ns;
    const double *x;
    double *yview; /* [nt][ns] */
} hx_fp_ctx;

static void hx_fp_visit(void *c, int t, int s, size_t j, double a)
{
    hx_fp_ctx *p = (hx_fp_ctx *)c;
    p->yview[(size_t)t * p->ns + s] += a * p->x[j];
}

typedef struct {
    int ns;
    const double *yview;
    double *x;
} hx_bp_ctx;

static void hx_bp_visit(void *c, int t, int s, size_t j, double a)
{
    hx_bp_ctx *p = (hx_bp_ctx *)c;
    p->x[j] += a * p->yview[(size_t)t * p->ns + s];
}

/* y[k][t][s] = sum_j a_{(views[k],t,s),j} x_j; parallel over views (each owns its rows). */
int orc_helix_forward(const orc_helix_geom *g, const double *x, const int *views, int nviews, double *y)
{
    if (hx_check(g) || hx_check_views(g, views, nviews)) return 1;
    const size_t per = (size_t)g->nt * g->ns;
    memset(y, 0, sizeof(double) * per * nviews);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nviews; k++) {
        hx_fp_ctx c = {g->ns, x, y + per * k};
        for (int iy = 0; iy < g->ny; iy++)
            for (int ix = 0; ix < g->nx; ix++) hx_view_column(g, views[k], ix, iy, -1, -1, hx_fp_visit, &c);
    }
    return 0;
}

/* x_j = sum_k sum_{t,s} a_{(views[k],t,s),j} y[k][t][s]; parallel over columns
 * (each owns its voxels), views summed in list order. */
int orc_helix_back(const orc_helix_geom *g, const double *y, const int *views, int nviews, double *x)
{
    if (hx_check(g) || hx_check_views(g, views, nviews)) return 1;
    const size_t nvox = (size_t)g->nx * g->ny * g->nz, per = (size_t)g->nt * g->ns;
    memset(x, 0, sizeof(double) * nvox);
#pragma omp parallel for schedule(dynamic)
    for (int col = 0; col < g->nx * g->ny; col++) {
        const int ix = col % g->nx, iy = col / g->nx;
        for (int k = 0; k < nviews; k++) {
            hx_bp_ctx c = {g->ns, y + per * k, x};
            hx_view_column(g, views[k], ix, iy, -1, -1, hx_bp_visit, &c);
        }
    }
    return 0;
}

typedef struct {
    size_t nvox;
    int ns;
    double *A; /* [(k, t, s)][j] of the views in the list */
} hx_mat_ctx;

static void hx_mat_visit(void *c, int t, int s, size_t j, double a)
{
    hx_mat_ctx *p = (hx_mat_ctx *)c;
    p->A[((size_t)t * p->ns + s) * p->nvox + j] += a;
}

/* dense A_views: [(nviews * nt * ns)][nvox] (small geometries only) */
int orc_helix_matrix(const orc_helix_geom *g, const int *views, int nviews, double *A)
{
    if (hx_check(g) || hx_check_views(g, views, nviews)) return 1;
    const size_t nvox = (size_t)g->nx * g->ny * g->nz, rows = (size_t)g->nt * g->ns;
    memset(A, 0, sizeof(double) * rows * nviews * nvox);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nviews; k++) {
        hx_mat_ctx c = {nvox, g->ns, A + rows * nvox * k};
        for (int iy = 0; iy < g->ny; iy++)
            for (int ix = 0; ix < g->nx; ix++) hx_view_column(g, views[k], ix, iy, -1, -1, hx_mat_visit, &c);
    }
    return 0;
}

typedef struct {
    int t, s;
    const double *x;
    double acc;
} hx_ray_ctx;

static void hx_ray_visit(void *c, int t, int s, size_t j, double a)
{
    hx_ray_ctx *p = (hx_ray_ctx *)c;
    if (t == p->t && s == p->s) p->acc += a * p->x[j];
}

/* out[r] = [A x] of ray (view rv[r], row rt[r], cell rs[r]) (sampled rays of large volumes) */
int orc_helix_forward_rays(const orc_helix_geom *g, const double *x, const int *rv, const int *rt, const int *rs,
                           int nrays, double *out)
{
    if (hx_check(g) || hx_check_views(g, rv, nrays)) return 1;
    for (int r = 0; r < nrays; r++)
        if (rt[r] < 0 || rt[r] >= g->nt || rs[r] < 0 || rs[r] >= g->ns) return 1;
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < nrays; r++) {
        hx_ray_ctx c = {rt[r], rs[r], x, 0.0};
        for (int iy = 0; iy < g->ny; iy++)
            for (int ix = 0; ix < g->nx; ix++) hx_view_column(g, rv[r], ix, iy, -1, rs[r], hx_ray_visit, &c);
        out[r] = c.acc;
    }
    return 0;
}

typedef struct {
    size_t j;
    int ns;
    const double *yview;
    double acc;
} hx_vox_ctx;

static void hx_vox_visit(void *c, int t, int s, size_t j, double a)
{
    hx_vox_ctx *p = (hx_vox_ctx *)c;
    if (j == p->j) p->acc += a * p->yview[(size_t)t * p->ns + s];
}

/* out[i] = [A_views' y] at voxel vox[i] (flat index into [nz][ny][nx]) */
int orc_helix_back_voxels(const orc_helix_geom *g, const double *y, const int *views, int nviews, const long long *vox,
                          int nvoxq, double *out)
{
    if (hx_check(g) || hx_check_views(g, views, nviews)) return 1;
    const long long nvox = (long long)g->nx * g->ny * g->nz;
    const size_t per = (size_t)g->nt * g->ns;
    for (int i = 0; i < nvoxq; i++)
        if (vox[i] < 0 || vox[i] >= nvox) return 1;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < nvoxq; i++) {
        const long long col = vox[i] % ((long long)g->nx * g->ny);
        const int ix = (int)(col % g->nx), iy = (int)(col / g->nx);
        const int iz = (int)(vox[i] / ((long long)g->nx * g->ny));
        double acc = 0.0;
        for (int k = 0; k < nviews; k++) {
            hx_vox_ctx c = {(size_t)vox[i], g->ns, y + per * k, 0.0};
            hx_view_column(g, views[k], ix, iy, iz, -1, hx_vox_visit, &c);
            acc += c.acc;
        }
        out[i] = acc;
    }
    return 0;
}

/* source height of view v (mm) */
double orc_helix_source_z(const orc_helix_geom *g, int v) { return hx_source_z(g, hx_beta(g, v)); }
