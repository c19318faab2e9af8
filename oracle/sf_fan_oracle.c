/*
 * ORACLE -- test infrastructure only.  Plain FP64 separable-footprint (SF)
 * projector for 2-D fan-beam CT with an equiangular (arc) detector.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file; the product path never does.  It shares no code with the CUDA
 * library.
 *
 * What it computes (the system matrix A of the PWLS problem, Sec. III,
 * Eq. (ct_problem); the paper takes A from the separable-footprint method of
 * Long, Fessler and Balter, cited there):
 *
 *   For pixel j and view beta, the four pixel corners are projected from the
 *   source onto the detector; their fan angles, sorted, are the vertices
 *   tau0 <= tau1 <= tau2 <= tau3 of a unit-height trapezoid T_j(gamma)
 *   (0 outside [tau0, tau3], 1 on [tau1, tau2], linear in between).
 *   The amplitude l_j is the chord length through the pixel along the ray
 *   through its centre, l = min(dx/|cos theta|, dy/|sin theta|).
 *   The detector cell s has rectangular response over
 *   [gamma_s - dgamma/2, gamma_s + dgamma/2], so
 *
 *     a_{(beta,s), j} = l_j * (1/dgamma) * integral_{cell s} T_j(gamma) dgamma.
 *
 *   Forward projection is y_i = sum_j a_ij x_j and back-projection is
 *   x_j = sum_i a_ij y_i, both from the same a_ij.
 *
 * Geometry: pixel (ix, iy) centre ((ix-(nx-1)/2+offset_x) dx, (iy-(ny-1)/2+offset_y) dy);
 * view angle beta_v = orbit_start + v*orbit/na; source at -dso*(cos b, sin b);
 * fan angle of a point P is atan2((P-S).e_perp, (P-S).e) with e=(cos b, sin b),
 * e_perp=(-sin b, cos b); bin s is centred at gamma_s=(s-(ns-1)/2+offset_s) dgamma,
 * dgamma = ds/dsd.  Images are [iy][ix]; sinograms are [view][bin].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int nx, ny;
    double dx, dy, offset_x, offset_y;
    int ns, na;
    double ds, offset_s, dso, dsd, orbit_deg, orbit_start_deg;
} orc_fan_geom;

static double orc_view_angle(const orc_fan_geom *g, int v)
{
    return (g->orbit_start_deg + (double)v * g->orbit_deg / (double)g->na) * M_PI / 180.0;
}

/* integral of the unit trapezoid with sorted vertices t[0..3] over (-inf, u] */
static double orc_trap_cdf(const double t[4], double u)
{
    if (u <= t[0]) return 0.0;
    if (u <= t[1]) { double d = u - t[0]; return d * d / (2.0 * (t[1] - t[0])); }
    double a = 0.5 * (t[1] - t[0]);
    if (u <= t[2]) return a + (u - t[1]);
    double b = a + (t[2] - t[1]);
    if (u < t[3]) { double d = t[3] - u; return b + 0.5 * (t[3] - t[2]) - d * d / (2.0 * (t[3] - t[2])); }
    return b + 0.5 * (t[3] - t[2]);
}

/* Trapezoid vertices (in detector-bin units, u = gamma/dgamma + (ns-1)/2 - offset_s,
 * so that bin s covers [s-1/2, s+1/2]) and amplitude of pixel (ix,iy) in the view
 * with direction (cb, sb). */
static void orc_pixel_footprint(const orc_fan_geom *g, double cb, double sb, int ix, int iy,
                                double tau[4], double *amp)
{
    const double xc = ((double)ix - (g->nx - 1) / 2.0 + g->offset_x) * g->dx;
    const double yc = ((double)iy - (g->ny - 1) / 2.0 + g->offset_y) * g->dy;
    const double inv_dg = g->dsd / g->ds;
    const double c0 = (g->ns - 1) / 2.0 - g->offset_s;
    int k = 0;
    for (int sy = -1; sy <= 1; sy += 2) {
        for (int sx = -1; sx <= 1; sx += 2) {
            double px = xc + 0.5 * sx * g->dx, py = yc + 0.5 * sy * g->dy;
            double tpar = g->dso + px * cb + py * sb;
            double tperp = -px * sb + py * cb;
            tau[k++] = atan2(tperp, tpar) * inv_dg + c0;
        }
    }
    /* insertion sort of four values */
    for (int i = 1; i < 4; i++) {
        double v = tau[i];
        int m = i - 1;
        while (m >= 0 && tau[m] > v) { tau[m + 1] = tau[m]; m--; }
        tau[m + 1] = v;
    }
    /* chord through the pixel along the ray from the source through its centre */
    double rx = xc + g->dso * cb, ry = yc + g->dso * sb;
    double r = sqrt(rx * rx + ry * ry);
    double ac = fabs(rx) / r, as = fabs(ry) / r;
    double lx = ac > 0.0 ? g->dx / ac : INFINITY;
    double ly = as > 0.0 ? g->dy / as : INFINITY;
    *amp = lx < ly ? lx : ly;
}

/* bins [s_lo, s_hi] that the footprint can touch, clipped to the detector */
static void orc_bin_range(const orc_fan_geom *g, const double tau[4], int *s_lo, int *s_hi)
{
    int lo = (int)floor(tau[0] - 0.5) + 1;
    int hi = (int)ceil(tau[3] + 0.5) - 1;
    if (lo < 0) lo = 0;
    if (hi > g->ns - 1) hi = g->ns - 1;
    *s_lo = lo;
    *s_hi = hi;
}

static double orc_weight(const double tau[4], double amp, int s)
{
    return amp * (orc_trap_cdf(tau, s + 0.5) - orc_trap_cdf(tau, s - 0.5));
}

static int orc_check(const orc_fan_geom *g)
{
    if (!g || g->nx <= 0 || g->ny <= 0 || g->ns <= 0 || g->na <= 0) return 1;
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->ds > 0) || !(g->dso > 0) || !(g->dsd > 0)) return 1;
    return 0;
}

/* y[k][s] = sum_j a_{(views[k], s), j} x_j */
int orc_fan_forward(const orc_fan_geom *g, const double *x, const int *views, int nviews, double *y)
{
    if (orc_check(g)) return 1;
    memset(y, 0, sizeof(double) * (size_t)nviews * g->ns);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nviews; k++) {
        double b = orc_view_angle(g, views[k]);
        double cb = cos(b), sb = sin(b);
        double *yk = y + (size_t)k * g->ns;
        for (int iy = 0; iy < g->ny; iy++) {
            for (int ix = 0; ix < g->nx; ix++) {
                double xj = x[(size_t)iy * g->nx + ix];
                if (xj == 0.0) continue;
                double tau[4], amp;
                int lo, hi;
                orc_pixel_footprint(g, cb, sb, ix, iy, tau, &amp);
                orc_bin_range(g, tau, &lo, &hi);
                for (int s = lo; s <= hi; s++) yk[s] += orc_weight(tau, amp, s) * xj;
            }
        }
    }
    return 0;
}

/* x_j = sum_k sum_s a_{(views[k], s), j} y[k][s] */
int orc_fan_back(const orc_fan_geom *g, const double *y, const int *views, int nviews, double *x)
{
    if (orc_check(g)) return 1;
    double *cbs = (double *)malloc(sizeof(double) * 2 * (size_t)(nviews > 0 ? nviews : 1));
    if (!cbs) return 2;
    for (int k = 0; k < nviews; k++) {
        double b = orc_view_angle(g, views[k]);
        cbs[2 * k] = cos(b);
        cbs[2 * k + 1] = sin(b);
    }
#pragma omp parallel for schedule(dynamic)
    for (int iy = 0; iy < g->ny; iy++) {
        for (int ix = 0; ix < g->nx; ix++) {
            double acc = 0.0;
            for (int k = 0; k < nviews; k++) {
                double tau[4], amp;
                int lo, hi;
                orc_pixel_footprint(g, cbs[2 * k], cbs[2 * k + 1], ix, iy, tau, &amp);
                orc_bin_range(g, tau, &lo, &hi);
                const double *yk = y + (size_t)k * g->ns;
                for (int s = lo; s <= hi; s++) acc += orc_weight(tau, amp, s) * yk[s];
            }
            x[(size_t)iy * g->nx + ix] = acc;
        }
    }
    free(cbs);
    return 0;
}

/* Dense A for the listed views: A[(k*ns + s)*(nx*ny) + j].  Small problems only. */
int orc_fan_matrix(const orc_fan_geom *g, const int *views, int nviews, double *A)
{
    if (orc_check(g)) return 1;
    const size_t npix = (size_t)g->nx * g->ny;
    memset(A, 0, sizeof(double) * npix * (size_t)nviews * g->ns);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nviews; k++) {
        double b = orc_view_angle(g, views[k]);
        double cb = cos(b), sb = sin(b);
        for (int iy = 0; iy < g->ny; iy++) {
            for (int ix = 0; ix < g->nx; ix++) {
                double tau[4], amp;
                int lo, hi;
                orc_pixel_footprint(g, cb, sb, ix, iy, tau, &amp);
                orc_bin_range(g, tau, &lo, &hi);
                for (int s = lo; s <= hi; s++)
                    A[((size_t)k * g->ns + s) * npix + (size_t)iy * g->nx + ix] = orc_weight(tau, amp, s);
            }
        }
    }
    return 0;
}

/* Forward projection of single rays (view, bin): out[r] = sum_j a_{r j} x_j.
 * Brute force over every pixel, for spot checks at sizes the full oracle is slow on. */
int orc_fan_forward_rays(const orc_fan_geom *g, const double *x, const int *ray_view, const int *ray_bin,
                         int nrays, double *out)
{
    if (orc_check(g)) return 1;
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < nrays; r++) {
        double b = orc_view_angle(g, ray_view[r]);
        double cb = cos(b), sb = sin(b);
        int s = ray_bin[r];
        double acc = 0.0;
        for (int iy = 0; iy < g->ny; iy++) {
            for (int ix = 0; ix < g->nx; ix++) {
                double xj = x[(size_t)iy * g->nx + ix];
                if (xj == 0.0) continue;
                double tau[4], amp;
                int lo, hi;
                orc_pixel_footprint(g, cb, sb, ix, iy, tau, &amp);
                orc_bin_range(g, tau, &lo, &hi);
                if (s >= lo && s <= hi) acc += orc_weight(tau, amp, s) * xj;
            }
        }
        out[r] = acc;
    }
    return 0;
}

/* Back-projection at single pixels: out[p] = sum_k sum_s a_{(views[k],s), pix[p]} y[k][s]. */
int orc_fan_back_pixels(const orc_fan_geom *g, const double *y, const int *views, int nviews, const int *pix,
                        int npix_sel, double *out)
{
    if (orc_check(g)) return 1;
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < npix_sel; p++) {
        int ix = pix[p] % g->nx, iy = pix[p] / g->nx;
        double acc = 0.0;
        for (int k = 0; k < nviews; k++) {
            double b = orc_view_angle(g, views[k]);
            double tau[4], amp;
            int lo, hi;
            orc_pixel_footprint(g, cos(b), sin(b), ix, iy, tau, &amp);
            orc_bin_range(g, tau, &lo, &hi);
            const double *yk = y + (size_t)k * g->ns;
            for (int s = lo; s <= hi; s++) acc += orc_weight(tau, amp, s) * yk[s];
        }
        out[p] = acc;
    }
    return 0;
}

/* Number of OpenMP threads a parallel region uses (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
