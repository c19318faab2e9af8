/*
 * ct.h -- C ABI of the GB300 (sm_103a) relaxed OS-LALM CT reconstruction library.
 *
 * The library solves the penalized weighted least-squares CT problem of
 * Nien & Fessler, "Relaxed Linearized Algorithms for Faster X-Ray CT Image
 * Reconstruction" (Sec. III, Eq. (ct_problem)):
 *
 *     x_hat = argmin_{x in Omega} 1/2 ||y - A x||_W^2 + R(x)
 *
 * with A a separable-footprint (SF) fan-beam projector, W = diag(w) the
 * statistical weights, R the edge-preserving regularizer of Eq. (def_reg)
 * and Omega = {x >= 0}, using the proposed relaxed OS-LALM of Algorithm 1
 * (or the simple relaxation of Algorithm 2) with the continuation sequence
 * of Eq. (dec_rho).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are float32 [ny][nx] (x fastest); sinograms are float32
 *   [view][bin] (bin fastest), view-major.  Pixel (ix, iy) is centred at
 *   ((ix - (nx-1)/2 + offset_x) dx, (iy - (ny-1)/2 + offset_y) dy) mm.
 *   View v has angle beta_v = orbit_start + v * orbit / na; the source sits
 *   at -dso (cos beta, sin beta); bin s is centred at fan angle
 *   (s - (ns-1)/2 + offset_s) ds / dsd (equiangular arc detector, ds is the
 *   cell's arc length at dsd).
 * - Array arguments named x, y, w, d_l, x_inout, x_ref are DEVICE pointers to
 *   caller-owned memory; they must be 4-byte aligned and must not alias
 *   each other unless stated.  `views` lists are HOST arrays.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  ct_forward, ct_back, ct_sqs_diag and ct_reg_gradient are
 *   asynchronous on it; ct_relaxed_oslalm_solve synchronises it before
 *   filling the report.
 * - Every entry point validates its arguments on the host and returns a
 *   status without launching anything when they are invalid;
 *   ct_last_error() then returns a message (thread-local, valid until the
 *   next call on the same thread).
 * - The library allocates device memory only for the workspace owned by a
 *   ct_geom (geometry tables at creation, the ray sums A 1 at the first call
 *   that needs them, solver state at the first solve); ct_geom_destroy frees
 *   it.  Calls that use one ct_geom must not run
 *   concurrently on different streams.
 */
#ifndef CT_H
#define CT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CT_OK = 0,
    CT_EINVAL = 1,   /* invalid argument (sizes, pointers, parameters) */
    CT_ENOMEM = 2,   /* device allocation failed */
    CT_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    CT_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    CT_ENOTSUP = 5   /* geometry kind or option not supported */
} ct_status;

enum { CT_FAN_ARC_2D = 1, CT_HELICAL_CONE_ARC = 2 };

/* Axial footprint of the helical projector (the 3-D separable-footprint
 * method the paper cites for A, Sec. III, has two axial models):
 * CT_AXIAL_RECT (SF-TR): the voxel's z-extent magnified at its column
 * centre's distance from the source, a rectangle in the detector row
 * coordinate; CT_AXIAL_TRAP (SF-TT): a trapezoid whose edges ramp between the
 * magnifications of the column's nearest and farthest (x, y) corners. */
enum { CT_AXIAL_RECT = 0, CT_AXIAL_TRAP = 1 };

typedef struct ct_geom ct_geom; /* opaque; owns device geometry tables and workspace */

/* Scan geometry (plain data, copied by ct_geom_create).  Lengths in mm,
 * angles in degrees.  For CT_FAN_ARC_2D the fields nz, dz, offset_z, nt, dt,
 * offset_t, pitch and axial are ignored.
 *
 * CT_HELICAL_CONE_ARC (3-D helical cone-beam, cylindrical detector): volumes
 * are float32 [nz][ny][nx], voxel (ix, iy, iz) centred at the pixel's (x, y)
 * and z = (iz - (nz-1)/2 + offset_z) dz; sinograms are float32
 * [view][row][cell]; row t lies at height (t - (nt-1)/2 + offset_t) dt on the
 * cylinder of radius dsd.  The views span orbit_deg (several turns allowed);
 * the source rises z_src = pitch * (nt dt dso / dsd) * (beta - beta_mid) / 2 pi
 * (table feed per turn = pitch times the detector's axial coverage at the
 * isocentre, centred on the volume at mid-scan).  The system matrix is
 * a = l_xy * c_t * T(s) * R(t): T the transaxial trapezoid footprint (as in
 * 2-D), l_xy its chord, c_t = 1 / cos(cone angle of row t), R the axial
 * footprint selected by `axial`. */
typedef struct {
    int kind;
    int nx, ny, nz;
    double dx, dy, dz;
    double offset_x, offset_y, offset_z; /* in pixels */
    int ns, nt, na;
    double ds, dt;
    double offset_s, offset_t; /* in detector cells */
    double dso, dsd;           /* source-to-isocentre, source-to-detector */
    double orbit_deg, orbit_start_deg;
    double pitch;
    int axial; /* CT_AXIAL_RECT or CT_AXIAL_TRAP (helical only; 0 for 2-D) */
} ct_geom_desc;

/* Create the device-side description of a scan geometry (Sec. III: A is the
 * forward projection matrix of the scan).  Checks that every pixel lies at
 * least 50 pixel widths in front of the source and that the fan half-angle is
 * below 1.4 rad, and precomputes per-view and per-(view, 16x16 pixel tile)
 * FP64-derived tables in device memory.  On success *out owns that memory; release it with
 * ct_geom_destroy.  Errors: CT_EINVAL (bad sizes), CT_ENOTSUP (kind),
 * CT_ENOMEM, CT_ECUDA. */
ct_status ct_geom_create(const ct_geom_desc *desc, ct_geom **out);

/* Free a geometry and all device memory it owns (NULL is a no-op).  Call it
 * only once no work using it is pending on any stream. */
void ct_geom_destroy(ct_geom *g);

/* Build the resident system matrix of a 2-D geometry: the same SF weights
 * a_ij that the projectors otherwise evaluate on the fly (Sec. III: A is the
 * forward projection matrix of the scan), stored once in device memory
 * owned by g as (1) ray-major compressed rows (a_ij in pairs, and the pixel
 * indices as 16-bit offsets from a 32-bit base per run of 32 pairs) for the
 * ray-driven forward projector, whose steep rays index a transposed copy of
 * the image (the projector packs [x | x^T] into a 2 nx ny scratch that g
 * also owns, or the solver's update kernel writes it) and (2) per-(view,
 * pixel) records of the pixel's cell weights (first cell and count in 16
 * bits, then the weights, interleaved across chunks of 32 pixels) for the
 * voxel-driven back-projector.  Afterwards ct_forward,
 * ct_back, ct_sqs_diag and ct_relaxed_oslalm_solve stream it instead of
 * recomputing footprints; results stay within FP32 rounding of the
 * on-the-fly path.  Also computes the ray sums A 1 from it (see ct_sqs_diag).  max_bytes: refuse with CT_ENOMEM (nothing kept) when the
 * matrix needs more; 0 means "whatever device memory allows".  bytes_out
 * (optional host pointer) receives the matrix size.  Runs on `stream` and
 * synchronises it.  Calling it again is a no-op.  Errors: CT_EINVAL,
 * CT_ENOMEM, CT_ENOTSUP (an image too wide for the 16-bit offsets),
 * CT_ECUDA. */
ct_status ct_geom_precompute(ct_geom *g, unsigned long long max_bytes, unsigned long long *bytes_out, void *stream);

/* Sizes of the resident matrix of g (an implementation detail; the paper has
 * no counterpart): matrix_bytes the whole (as ct_geom_precompute reports),
 * record_bytes the back-projector's records within it (0 when it keeps
 * none: footprints wider than 15 cells, or more than 4096 cells).  Both 0
 * before ct_geom_precompute.  Either pointer may be NULL.  Errors: CT_EINVAL
 * (null geometry). */
ct_status ct_geom_matrix_info(const ct_geom *g, unsigned long long *matrix_bytes, unsigned long long *record_bytes);

/* Projector autotuner (an implementation choice; the paper has no
 * counterpart).  Times, on a subset of views_per_launch evenly spread views
 * (<= 0: 24), every forward-projector decomposition available for g
 * (1 = resident-matrix rows, 2 = 32-cell bundles, 3 = 8 lanes per ray) and
 * every back-projector (1 = stored footprints, 2 = footprints on the fly),
 * and keeps the fastest for all later calls on g.  Run it after
 * ct_geom_precompute if the matrix is wanted among the candidates.
 * fp_choice, bp_choice: optional host outputs.  Allocates two temporary
 * buffers; synchronises the stream.  Errors: CT_EINVAL, CT_ENOMEM, CT_ECUDA. */
ct_status ct_geom_autotune(ct_geom *g, int views_per_launch, int *fp_choice, int *bp_choice, void *stream);

/* Forward projection y = A_V x (Sec. III, Eq. (ct_problem); SF footprints,
 * ray-driven).  x: device [ny][nx]; y: device [nviews][ns], row k is view
 * views[k].  views: host array of nviews indices in [0, na), or NULL for all
 * na views in order (then nviews must be na).  1 <= nviews <= na.  Output
 * rows are overwritten.  With the resident matrix (ct_geom_precompute) x is
 * first packed as [x | x^T] into a scratch image g owns (one extra small
 * launch; see ct_pack_image).  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_forward(const ct_geom *g, const float *x, float *y, const int *views, int nviews, void *stream);

/* The packed image [x | x^T] of a 2-D geometry: xpack[j] = x[j] and
 * xpack[nx ny + ix ny + iy] = x[iy nx + ix] (device, 2 nx ny floats, caller-
 * owned).  It is what the resident matrix's rows index (steep rays read the
 * transposed copy, where their consecutive pixels are adjacent);
 * ct_forward packs its x this way itself.  Errors: CT_EINVAL (null
 * argument, helical geometry), CT_ECUDA. */
ct_status ct_pack_image(const ct_geom *g, const float *x, float *xpack, void *stream);

/* ct_forward of an image already packed by ct_pack_image (2-D geometries):
 * the same y, without the packing pass, for callers that project one image
 * many times.  Errors: as ct_forward, and CT_EINVAL for a helical geometry. */
ct_status ct_forward_packed(const ct_geom *g, const float *xpack, float *y, const int *views, int nviews,
                            void *stream);

/* Back-projection x = scale * A_V' y (+ x if accumulate != 0), with the same
 * a_ij as ct_forward (voxel-driven, no atomics).  y: device [nviews][ns];
 * x: device [ny][nx]; views as for ct_forward.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_back(const ct_geom *g, const float *y, float *x, const int *views, int nviews, float scale,
                  int accumulate, void *stream);

/* SQS majorizer of the data term, D_L = diag(A' W A 1) over all views
 * (Sec. III-A: the diagonal majorizing matrix of A'WA).  w: device [na][ns]
 * weights; d_l: device [ny][nx] output.  A 1 depends on the geometry only: it
 * is computed at the first call (or by ct_geom_precompute) and kept with the
 * geometry, so a call costs one elementwise product and one back-projection.
 * Uses the geometry's sinogram workspace.  Errors: CT_EINVAL, CT_ENOMEM,
 * CT_ECUDA. */
ct_status ct_sqs_diag(const ct_geom *g, const float *w, float *d_l, void *stream);

/* Same result as ct_sqs_diag, without allocating any device memory (nor
 * using the geometry's workspace): for callers that cannot allocate once running (a
 * process whose device memory is reserved up front by its own pool, or a
 * latency-critical loop that must not enter cudaMalloc/cudaFree, which can
 * block and synchronise the device).  The paper has no counterpart; it is an
 * operational variant.  The intermediate sinogram w (A 1) lives in a 4 MiB
 * device array inside the library (held by every GPU that loads it until the
 * process exits), so na * ns must be <= 1,048,576 (CT_EINVAL otherwise).  The
 * first call on a device looks up that array's address with the device
 * current; make it before any stream capture.  Under CUDA's lazy module
 * loading that first call also loads the array onto the device, so it needs
 * 4 MiB of device memory outside any pool the caller reserved.  The address
 * is cached for the life of the device's primary context (a cudaDeviceReset
 * invalidates it).  Uses the geometry's kept ray sums A 1 when it has them,
 * else one forward projection of w over all views.  All calls share the
 * array: calls that overlap on the GPU race.  The geometry's device must be
 * current.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_sqs_diag_noalloc(const ct_geom *g, const float *w, float *d_l, void *stream);

enum { CT_FBP_RAMP = 0, CT_FBP_HANN = 1 };

/* Filtered back-projection of a full 360-degree equiangular fan-beam scan,
 * the initial image of Algorithm 1 ("an initial (FBP) image", Sec. III-A;
 * the paper does not specify it).  Textbook equiangular fan-beam FBP:
 * D cos(gamma) pre-weighting, band-limited ramp filter in the fan angle
 * (window CT_FBP_RAMP, or CT_FBP_HANN for its Hann-apodised version),
 * distance-weighted back-projection with linear interpolation.  y: device
 * [na][ns] line integrals; x: device [ny][nx] output (same units per mm).
 * A helical geometry (no helical FBP is given in the paper; a reading):
 * y is [na][nt][ns], x the [nz][ny][nx] volume, and each slice is the
 * fan-beam FBP of its single-slice rebinning: the turn of views whose
 * source heights are centred on the slice, from each view the detector row
 * where the slice's height at the isocentre projects (linear between rows,
 * times the cosine of that row's cone angle); the scan must span at least
 * one turn with a whole number of views per turn.  Uses the geometry's
 * sinogram workspace.  Errors: CT_EINVAL, CT_ENOTSUP (a 2-D orbit other than
 * 360 degrees, a helical scan without whole turns, or ns > 19,000),
 * CT_ECUDA. */
ct_status ct_fbp(const ct_geom *g, const float *y, float *x, int window, void *stream);

enum { CT_POT_HYPERBOLA = 0, CT_POT_FAIR = 1, CT_POT_QUADRATIC = 2 };
enum { CT_ALG_PROPOSED = 0, CT_ALG_SIMPLE = 1 };
enum { CT_CURV_HUBER = 0, CT_CURV_MAX = 1 };

/* Gradient and Huber-curvature SQS diagonal of the regularizer
 * R(x) = sum_i beta_i sum_n kappa_n kappa_{n+s_i} phi([C_i x]_n)
 * (Eq. (def_reg)) over the 8 neighbours in 2-D (26 in 3-D),
 * beta_i = beta / ||s_i||.  kappa: optional device image of the voxel
 * weights kappa_n (same layout as x), NULL for kappa = 1.  potential:
 * CT_POT_*, delta > 0 its scale (same units as x).  grad, curv: device
 * outputs shaped as x (curv may be NULL).  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_reg_gradient(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                          int potential, float *grad, float *curv, void *stream);

/* Voxel weights for resolution uniformity, kappa_n of Eq. (def_reg) (Sec. III
 * cites Fessler and Rogers for them; the paper gives no formula):
 * kappa_j = sqrt( [A' w]_j / [A' 1]_j ), the square root of the a_ij-weighted
 * mean of the statistical weights of the rays through voxel j over all views
 * (the cited work weights by a_ij^2; the first power needs only A'), and 0
 * where no ray meets voxel j.  w: device sinogram of weights (>= 0), shaped
 * as for ct_sqs_diag; kappa: device output shaped as the image.  Uses the
 * geometry's sinogram workspace and allocates one image of stream-ordered
 * device scratch for the call.  Errors: CT_EINVAL, CT_ENOMEM, CT_ECUDA. */
ct_status ct_kappa(const ct_geom *g, const float *w, float *kappa, void *stream);

/* Parameters of ct_relaxed_oslalm_solve. */
typedef struct {
    int M;              /* number of ordered subsets, 1 <= M <= na (interleaved: v mod M) */
    int n_iter;         /* outer iterations (each visits all M subsets) */
    float alpha;        /* relaxation, 1 <= alpha < 2 (Algorithm 1: 1.999 in the paper) */
    float beta;         /* regularization parameter (>= 0) */
    float delta;        /* potential scale (> 0 unless potential is quadratic) */
    int potential;      /* CT_POT_* */
    int algorithm;      /* CT_ALG_PROPOSED (Algorithm 1) or CT_ALG_SIMPLE (Algorithm 2) */
    int nonneg;         /* 1: Omega = {x >= 0}; 0: unconstrained */
    int continuation;   /* 1: rho_k(alpha) of Eq. (dec_rho), k = subiterations; 0: rho = rho_fixed */
    float rho_fixed;    /* used when continuation == 0 (> 0) */
    const float *x_ref; /* optional device [ny][nx] reference (x*) for the RMSD trace, or NULL */
    float hu_per_unit;  /* HU per unit of x, for RMSD reporting */
    float fov_radius;   /* RMSD mask radius in mm; <= 0 selects the scan's full field of view */
    float stop_rmsd_hu; /* > 0: stop after the first iteration with RMSD <= this (needs x_ref) */
    int init_fbp;       /* 1: overwrite x_inout with the Hann-windowed FBP of y first (timed with the solve) */
    int curvature;      /* D_R majorizer (Sec. II-B): CT_CURV_HUBER (Huber's optimal curvature, the default)
                           or CT_CURV_MAX (the potential's maximum curvature, phi''(0) = 1) */
    float dl_scale;     /* D_L <- dl_scale * diag(A'WA1) (supplement's majorizer study); 0 reads as 1 */
    const float *kappa; /* optional device image of the regularizer's voxel weights kappa_n (Eq. (def_reg),
                           e.g. from ct_kappa; same layout as x_inout), NULL for kappa = 1 */
    /* Checkpoint and resume.  The solver state after outer iteration k is (x, g, h, k): D_L is recomputed
       from w, rho depends only on the subiteration count k M (Eq. (dec_rho)), and the next subset is 0.
       g_state, h_state: optional device images (layout of x_inout); when given, the solve writes its final
       g and h (Algorithm 2: h holds zeta) into them.  start_iter > 0 resumes after that many outer
       iterations: g and h are read from g_state and h_state (both required; init_fbp must be 0) instead
       of the initial gradient step, x_inout holds the iterate, and rho continues at subiteration
       start_iter M.  A run split this way gives the same x, g and h, bit for bit, as one uninterrupted
       run on the same GPU. */
    int start_iter;
    float *g_state;
    float *h_state;
} ct_solve_params;

/* Report filled by ct_relaxed_oslalm_solve.  The two array pointers are
 * optional caller-owned HOST arrays of at least n_iter entries. */
typedef struct {
    int iters_done;
    double seconds;         /* device time of the whole solve (D_L, initialisation, iterations) */
    double seconds_to_tol;  /* device time until the first iteration with RMSD <= stop tolerance
                               (or <= 1 HU when stop_rmsd_hu <= 0); negative if never reached */
    float rmsd_hu_last;     /* RMSD of the last iterate, or -1 without x_ref */
    float *rmsd_trace_hu;   /* optional out: RMSD after each iteration */
    double *iter_seconds;   /* optional out: device time from the solve's start to the end of each iteration */
} ct_solve_report;

/* Relaxed OS-LALM (Algorithm 1, or Algorithm 2 when algorithm ==
 * CT_ALG_SIMPLE) for Eq. (ct_problem) with W = diag(w):
 *   D_L = diag(A'WA1); rho = 1; zeta = g = M grad L_M(x); h = D_L x - zeta;
 *   per subiteration (subset m): s = rho (D_L x - h) + (1 - rho) g;
 *   x+ = [x - (rho D_L + D_R)^{-1}(s + grad R(x))]_Omega (D_R: Huber curvature);
 *   zeta = M grad L_m(x+); g+ = rho/(rho+1)(alpha zeta + (1-alpha) g) + g/(rho+1);
 *   h+ = alpha (D_L x+ - zeta) + (1-alpha) h; rho <- rho_{k}(alpha).
 * y, w: device [na][ns] sinogram and weights (w >= 0).  x_inout: device
 * [ny][nx], the initial image on entry (or the FBP of y when init_fbp = 1,
 * which needs a 360-degree scan; for a helical geometry the rebinned
 * slice-by-slice FBP of ct_fbp, which needs whole turns) and the result on
 * return.  The solve
 * runs on `stream` as CUDA-graph replays of one outer iteration and
 * synchronises the stream before returning.  Errors: CT_EINVAL, CT_ENOMEM,
 * CT_ECUDA. */
ct_status ct_relaxed_oslalm_solve(const ct_geom *g, const float *y, const float *w, const ct_solve_params *p,
                                  float *x_inout, ct_solve_report *report, void *stream);

/* Batched relaxed OS-LALM: nslices independent problems (Algorithm 1 or 2
 * each, with its own geometry, sinogram, weights and parameters).  Slices
 * of two or more geometries are all solved by ct_relaxed_oslalm_solve, on up
 * to four concurrent host threads with a stream each (the slices of one
 * geometry, which owns the solver workspace, one after another).  Slices of
 * one geometry: those of at least 384 x 384 pixels, whose own subsets fill
 * the GPU, one after another by ct_relaxed_oslalm_solve; the smaller ones
 * together in one persistent cooperative launch, after per-slice setup
 * launches (D_L, initial gradient, optional FBP).  There, slice i runs
 * n_iter_i * M_i subiterations; all slices advance in lockstep super-steps,
 * and each super-step's regularizer, forward-projection and back-projection
 * work of every active slice is spread over all SMs.  Report times count from
 * the start of the call's device work (an event on `stream`); `seconds` is the
 * same total in every report.  geoms, y, w, x_inout: host
 * arrays of nslices pointers (device data as in ct_relaxed_oslalm_solve;
 * slices may share a geometry); params: host array of nslices parameter
 * sets (a slice with x_ref and stop_rmsd_hu > 0 stops at the end of the
 * first outer iteration whose RMSD is at or below it, as in
 * ct_relaxed_oslalm_solve; the others run n_iter iterations);
 * reports: optional host array of nslices reports, whose per-iteration times
 * come from the device clock at each slice's iteration ends.  Allocates one
 * device arena per call for the batched slices; a large slice's solve
 * allocates its geometry's solver workspace as ct_relaxed_oslalm_solve
 * does.  1 <= nslices <= 1024.  Synchronises the stream.  Errors: CT_EINVAL, CT_ENOTSUP, CT_ENOMEM, CT_ECUDA,
 * CT_ETIMEOUT (a bounded grid-barrier wait gave up; the results are then
 * undefined). */
ct_status ct_relaxed_oslalm_solve_batched(const ct_geom *const *geoms, const float *const *y, const float *const *w,
                                          const ct_solve_params *params, float *const *x_inout, int nslices,
                                          ct_solve_report *reports, void *stream);

/* Failure-detection hook of the batched solve's persistent launch (no
 * counterpart in the paper; the batched solver's grid barrier is this
 * library's).  Every grid-barrier wait of later batched launches polls at
 * most max_polls times (about 100 ns apart; 0 restores the built-in limit
 * of 2^24 polls), and with missing > 0 the barrier waits for that many
 * participants beyond the grid, which never arrive: every wait then runs out,
 * each CTA records the failure and returns, and the call returns CT_ETIMEOUT
 * with the GPU context intact.  Process-wide; set it only while no batched
 * solve runs.  (0, 0) is normal operation.  Errors: CT_EINVAL (max_polls < 0,
 * missing outside [0, 1024]). */
ct_status ct_debug_barrier(long long max_polls, int missing);

/* Message describing the last failure on this thread ("" if none). */
const char *ct_last_error(void);

/* Library version (major * 100 + minor). */
int ct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CT_H */
