// Relaxed OS-LALM driver (Algorithm 1 / Algorithm 2, Sec. III-A) on one GPU.
//
// Setup (once per solve): D_L = diag(A'WA1) over all views; zeta = g =
// M grad L_M(x) from the last subset; h = D_L x - zeta.  One outer iteration
// (M subiterations of: regularizer + x-update, subset forward projection
// with the weighted residual, subset back-projection with the g/h update)
// plus the RMSD-to-reference reduction is captured once as a CUDA graph and
// replayed n_iter times.  rho for subiteration t is read on the device from
// a table of the continuation sequence (Eq. (dec_rho)) indexed by a device
// counter that the back-projector's last block advances, so every replay
// sees the right rho without host involvement.
//
// Subsets are interleaved (S_m = {v : v mod M = m}) and visited m = 0..M-1.
#include <cmath>
#include <cstring>
#include <vector>

#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr int kRmsdBlocks = 152;

__global__ void __launch_bounds__(256) rmsd_kernel(FanDev G, const float *__restrict__ x, const float *__restrict__ xr,
                                                   float r2max, double *__restrict__ partial, int *__restrict__ counter,
                                                   float *__restrict__ trace, int M, float hu)
{
    __shared__ double ss[8];
    __shared__ double sc[8];
    double s = 0.0, c = 0.0;
    // rows by block, columns by thread: the pixel's position without integer division
    for (int iy = blockIdx.x; iy < G.ny; iy += gridDim.x) {
        const float Y = ((float)iy - G.cyo) * G.dy;
        const size_t row = (size_t)iy * G.nx;
        for (int ix = threadIdx.x; ix < G.nx; ix += blockDim.x) {
            const float X = ((float)ix - G.cxo) * G.dx;
            if (fmaf(X, X, Y * Y) <= r2max) {
                const double d = (double)x[row + ix] - (double)xr[row + ix];
                s += d * d;
                c += 1.0;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S0 = 0.0, C0 = 0.0;
        for (int q = 0; q < 8; q++) {
            S0 += ss[q];
            C0 += sc[q];
        }
        partial[2 * blockIdx.x] = S0;
        partial[2 * blockIdx.x + 1] = C0;
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

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

struct Workspace {
    float *x_new, *g, *h, *d_l, *resid, *rho_tab, *trace;
    int *perm, *counter;
    double *partial;
    float *x_col, *xref_col;  // helical: column-major copies of x and x_ref
    float *kappa_col;         // helical with kappa: column-major copy of kappa
};

ct_status ensure_workspace(ct_geom *g, int max_sub, int T, int n_iter, bool kappa, Workspace &W)
{
    const size_t npix = (size_t)g->fan.nx * g->fan.ny * (g->helical ? g->hx.nz : 1);
    const size_t view_len = (size_t)g->fan.ns * (g->helical ? g->hx.nt : 1);
    const size_t vol_h = g->helical ? npix * 4 : 0;
    size_t off[13], sz = 0;
    // x_new holds the packed image [x+ | x+^T] in 2-D (the resident rows index it)
    const size_t sizes[13] = {npix * (g->helical ? 4 : 8), npix * 4, npix * 4, npix * 4, (size_t)max_sub * view_len * 4,
                              (size_t)T * 4, (size_t)(n_iter > 0 ? n_iter : 1) * 4, (size_t)g->fan.na * 4, 16 * 4,
                              (size_t)kRmsdBlocks * 2 * 8, vol_h, vol_h, kappa ? vol_h : 0};
    for (int i = 0; i < 13; i++) {
        off[i] = sz;
        sz += align_up(sizes[i]);
    }
    if (sz > g->solve_bytes) {
        cudaFree(g->d_solve);
        g->d_solve = nullptr;
        g->solve_bytes = 0;
        CT_CUDA_TRY(cudaMalloc(&g->d_solve, sz), "allocating solver workspace");
        g->solve_bytes = sz;
    }
    char *b = (char *)g->d_solve;
    W.x_new = (float *)(b + off[0]);
    W.g = (float *)(b + off[1]);
    W.h = (float *)(b + off[2]);
    W.d_l = (float *)(b + off[3]);
    W.resid = (float *)(b + off[4]);
    W.rho_tab = (float *)(b + off[5]);
    W.trace = (float *)(b + off[6]);
    W.perm = (int *)(b + off[7]);
    W.counter = (int *)(b + off[8]);
    W.partial = (double *)(b + off[9]);
    W.x_col = g->helical ? (float *)(b + off[10]) : nullptr;
    W.xref_col = g->helical ? (float *)(b + off[11]) : nullptr;
    W.kappa_col = g->helical && kappa ? (float *)(b + off[12]) : nullptr;
    return CT_OK;
}

double rho_continuation(long k, double alpha)
{
    if (k == 0) return 1.0;
    const double q = M_PI / (alpha * (double)(k + 1));
    return q * std::sqrt(1.0 - 0.25 * q * q);
}

// The launches of one subiteration step, for either geometry kind.
cudaError_t step_update(const ct_geom *g, const SolveDev &S, const ct_solve_params *p, cudaStream_t st)
{
    return g->helical ? launch_reg_update_helix(g, S, p->beta, p->delta, p->potential, p->curvature, st)
                      : launch_reg_update(g->fan, S, p->beta, p->delta, p->potential, p->curvature, st);
}

cudaError_t step_fp(const ct_geom *g, int mode, const float *x, const int *views, int nviews, float *out,
                    const float *y, const float *w, cudaStream_t st, const float *xpack = nullptr)
{
    return g->helical ? launch_fp_helix(g, mode, x, views, nviews, out, y, w, st)
                      : launch_fp(g->fan, mode, x, views, nviews, out, y, w, st, xpack);
}

cudaError_t step_bp(const ct_geom *g, int mode, const float *sino, const int *views, int nviews, float *x,
                    const SolveDev *S, cudaStream_t st, float scale = 1.0f)
{
    return g->helical ? launch_bp_helix(g, mode, sino, views, nviews, x, scale, 0, S, st)
                      : launch_bp(g->fan, mode, sino, views, nviews, x, scale, 0, S, st);
}

struct Events {
    std::vector<cudaEvent_t> ev;
    ~Events()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_relaxed_oslalm_solve(const ct_geom *gc, const float *y, const float *w,
                                             const ct_solve_params *p, float *x, ct_solve_report *rep, void *stream)
{
    ct_geom *g = const_cast<ct_geom *>(gc);
    if (!g || !y || !w || !p || !x) { set_error("ct_relaxed_oslalm_solve: null argument"); return CT_EINVAL; }
    const int na = g->fan.na;
    if (p->M < 1 || p->M > na) { set_error("M=%d must be in [1, na=%d]", p->M, na); return CT_EINVAL; }
    if (p->n_iter < 0 || p->n_iter > 1000000) { set_error("n_iter=%d out of range", p->n_iter); return CT_EINVAL; }
    if (!(p->alpha >= 1.0f && p->alpha < 2.0f)) { set_error("alpha=%g must be in [1, 2)", p->alpha); return CT_EINVAL; }
    if (!(p->beta >= 0.0f)) { set_error("beta must be >= 0"); return CT_EINVAL; }
    if (p->potential < CT_POT_HYPERBOLA || p->potential > CT_POT_QUADRATIC) {
        set_error("unknown potential %d", p->potential);
        return CT_EINVAL;
    }
    if (p->potential != CT_POT_QUADRATIC && !(p->delta > 0.0f)) { set_error("delta must be > 0"); return CT_EINVAL; }
    if (p->algorithm != CT_ALG_PROPOSED && p->algorithm != CT_ALG_SIMPLE) {
        set_error("unknown algorithm %d", p->algorithm);
        return CT_EINVAL;
    }
    if (!p->continuation && !(p->rho_fixed > 0.0f)) { set_error("rho_fixed must be > 0"); return CT_EINVAL; }
    if (p->stop_rmsd_hu > 0.0f && !p->x_ref) { set_error("stop_rmsd_hu needs x_ref"); return CT_EINVAL; }
    if ((long)p->n_iter * p->M > 200000000L) { set_error("n_iter * M too large"); return CT_EINVAL; }
    if (p->init_fbp != 0 && p->init_fbp != 1) { set_error("init_fbp must be 0 or 1"); return CT_EINVAL; }
    if (p->curvature != CT_CURV_HUBER && p->curvature != CT_CURV_MAX) {
        set_error("unknown curvature %d", p->curvature);
        return CT_EINVAL;
    }
    if (!(p->dl_scale >= 0.0f) || !std::isfinite(p->dl_scale)) { set_error("dl_scale must be >= 0"); return CT_EINVAL; }
    if (p->init_fbp) {
        ct_status sf = validate_fbp(g, CT_FBP_HANN);
        if (sf != CT_OK) return sf;
    }
    if (p->start_iter < 0 || (long)p->start_iter * p->M > 200000000L) {
        set_error("start_iter=%d out of range", p->start_iter);
        return CT_EINVAL;
    }
    if (p->start_iter > 0 && (!p->g_state || !p->h_state || p->init_fbp)) {
        set_error("resuming (start_iter > 0) needs g_state and h_state and init_fbp = 0");
        return CT_EINVAL;
    }

    const int M = p->M;
    // interleaved subsets, stored contiguously: perm = [S_0 | S_1 | ... | S_{M-1}]
    std::vector<int> perm;
    std::vector<int> off(M + 1, 0), cnt(M, 0);
    perm.reserve(na);
    for (int m = 0; m < M; m++) {
        off[m] = (int)perm.size();
        for (int v = m; v < na; v += M) perm.push_back(v);
        cnt[m] = (int)perm.size() - off[m];
    }
    off[M] = na;
    int max_sub = 0;
    for (int m = 0; m < M; m++) max_sub = cnt[m] > max_sub ? cnt[m] : max_sub;
    const long T = (long)p->n_iter * M;
    std::vector<float> rho((size_t)(T > 0 ? T : 1));
    // rho of the subiterations this call runs: a resumed solve continues the sequence after start_iter * M
    const long t0 = (long)p->start_iter * M;
    for (long t = 0; t < T; t++)
        rho[t] = (float)(p->continuation ? rho_continuation(t0 + t, p->alpha) : (double)p->rho_fixed);

    Workspace W;
    ct_status st = ensure_workspace(g, max_sub, (int)(T > 0 ? T : 1), p->n_iter, p->kappa != nullptr, W);
    if (st != CT_OK) return st;

    cudaStream_t user = (cudaStream_t)stream, ws = nullptr;
    CT_CUDA_TRY(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking), "creating solver stream");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sguard{ws};
    Events E;
    const int nev = 3 + p->n_iter;
    E.ev.resize(nev, nullptr);
    for (int i = 0; i < nev; i++) CT_CUDA_TRY(cudaEventCreate(&E.ev[i]), "creating events");
    cudaEvent_t ev_in = E.ev[0], ev_start = E.ev[1], ev_end = E.ev[2];

    CT_CUDA_TRY(cudaEventRecord(ev_in, user), "ordering after caller's stream");
    CT_CUDA_TRY(cudaStreamWaitEvent(ws, ev_in, 0), "ordering after caller's stream");
    CT_CUDA_TRY(cudaMemcpyAsync(W.perm, perm.data(), sizeof(int) * na, cudaMemcpyHostToDevice, ws), "upload subsets");
    CT_CUDA_TRY(cudaMemcpyAsync(W.rho_tab, rho.data(), sizeof(float) * rho.size(), cudaMemcpyHostToDevice, ws),
                "upload rho");
    CT_CUDA_TRY(cudaMemsetAsync(W.counter, 0, 16 * sizeof(int), ws), "reset counters");

    SolveDev S;
    S.x = g->helical ? W.x_col : x;
    S.x_new = W.x_new;
    S.g = W.g;
    S.h = W.h;
    S.d_l = W.d_l;
    S.resid = W.resid;
    S.rho_tab = W.rho_tab;
    S.counter = W.counter;
    S.alpha = p->alpha;
    S.M_scale = (float)M;
    S.algorithm = p->algorithm;
    S.nonneg = p->nonneg;
    S.kappa = g->helical ? W.kappa_col : p->kappa;
    const FanDev &G = g->fan;
    const double R = p->fov_radius > 0.0f ? (double)p->fov_radius : g->fov_radius;
    const float r2max = (float)(R * R);

    // capture one outer iteration
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (p->n_iter > 0) {
        CT_CUDA_TRY(cudaStreamBeginCapture(ws, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = cudaSuccess;
        for (int m = 0; m < M && e == cudaSuccess; m++) {
            e = step_update(g, S, p, ws);
            if (e == cudaSuccess)  // the update kernel wrote x+ packed
                e = step_fp(g, FP_RESID, W.x_new, W.perm + off[m], cnt[m], W.resid, y, w, ws, W.x_new);
            if (e == cudaSuccess) e = step_bp(g, BP_SOLVE_UPDATE, W.resid, W.perm + off[m], cnt[m], nullptr, &S, ws);
        }
        if (e == cudaSuccess && p->x_ref) {
            if (g->helical) {
                e = launch_rmsd_helix(g, S.x, W.xref_col, r2max, W.partial, W.counter, W.trace, M, p->hu_per_unit, ws);
            } else {
                rmsd_kernel<<<kRmsdBlocks, 256, 0, ws>>>(G, x, p->x_ref, r2max, W.partial, W.counter, W.trace, M,
                                                         p->hu_per_unit);
                e = cudaGetLastError();
            }
        }
        cudaError_t e2 = cudaStreamEndCapture(ws, &graph);
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "capturing iteration"); }
        if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiating iteration graph");
        e = cudaGraphUpload(exec, ws);
        if (e != cudaSuccess) { cudaGraphExecDestroy(exec); return cuda_fail(e, "uploading graph"); }
    }
    struct ExecGuard {
        cudaGraphExec_t e;
        ~ExecGuard() { if (e) cudaGraphExecDestroy(e); }
    } eguard{exec};

    // the geometry's ray sums A 1 (computed once per geometry, like the resident matrix)
    CT_CUDA_TRY(ensure_ray_sums(g, ws), "ray sums A 1");
    CT_CUDA_TRY(cudaEventRecord(ev_start, ws), "event");
    if (p->init_fbp) CT_CUDA_TRY(launch_fbp(g, y, x, CT_FBP_HANN, ws), "initial FBP image");
    if (g->helical) {  // the kernels work on column-major volumes
        CT_CUDA_TRY(launch_to_columns(g, x, W.x_col, ws), "x layout");
        if (p->x_ref) CT_CUDA_TRY(launch_to_columns(g, p->x_ref, W.xref_col, ws), "x_ref layout");
        if (p->kappa) CT_CUDA_TRY(launch_to_columns(g, p->kappa, W.kappa_col, ws), "kappa layout");
    }
    // D_L = diag(A' W A 1) over all views: w (A 1), then one back-projection
    CT_CUDA_TRY(launch_weighted_ray_sums(g, w, g->d_sino_ws, ws), "D_L weights");
    CT_CUDA_TRY(step_bp(g, BP_PLAIN, g->d_sino_ws, g->d_views_all, na, W.d_l, nullptr, ws,
                        p->dl_scale > 0.0f ? p->dl_scale : 1.0f), "D_L back");
    if (p->start_iter > 0) {
        // resume: g and h from the checkpoint
        const size_t nvox = (size_t)G.nx * G.ny * (g->helical ? g->hx.nz : 1);
        if (g->helical) {
            CT_CUDA_TRY(launch_to_columns(g, p->g_state, W.g, ws), "g layout");
            CT_CUDA_TRY(launch_to_columns(g, p->h_state, W.h, ws), "h layout");
        } else {
            CT_CUDA_TRY(cudaMemcpyAsync(W.g, p->g_state, sizeof(float) * nvox, cudaMemcpyDeviceToDevice, ws), "g");
            CT_CUDA_TRY(cudaMemcpyAsync(W.h, p->h_state, sizeof(float) * nvox, cudaMemcpyDeviceToDevice, ws), "h");
        }
    } else {
        // rho = 1, zeta = g = M grad L_M(x), h = D_L x - zeta  (last subset)
        CT_CUDA_TRY(step_fp(g, FP_RESID, S.x, W.perm + off[M - 1], cnt[M - 1], W.resid, y, w, ws), "init forward");
        CT_CUDA_TRY(step_bp(g, BP_SOLVE_INIT, W.resid, W.perm + off[M - 1], cnt[M - 1], nullptr, &S, ws),
                    "init back");
    }

    const float tol = p->stop_rmsd_hu > 0.0f ? p->stop_rmsd_hu : 1.0f;
    int done = 0;
    for (int it = 0; it < p->n_iter; it++) {
        CT_CUDA_TRY(cudaGraphLaunch(exec, ws), "graph launch");
        CT_CUDA_TRY(cudaEventRecord(E.ev[3 + it], ws), "event");
        done = it + 1;
        if (p->stop_rmsd_hu > 0.0f) {
            float r = 0.0f;
            CT_CUDA_TRY(cudaMemcpyAsync(&r, W.trace + it, sizeof(float), cudaMemcpyDeviceToHost, ws), "read rmsd");
            CT_CUDA_TRY(cudaStreamSynchronize(ws), "sync");
            if (r <= tol) break;
        }
    }
    if (g->helical) CT_CUDA_TRY(launch_to_slices(g, W.x_col, x, 1.0f, 0, ws), "x layout");
    // checkpoint: the final g and h (x is the caller's x_inout)
    for (int q = 0; q < 2; q++) {
        float *dst = q == 0 ? p->g_state : p->h_state;
        const float *src = q == 0 ? W.g : W.h;
        if (!dst) continue;
        if (g->helical)
            CT_CUDA_TRY(launch_to_slices(g, src, dst, 1.0f, 0, ws), "state layout");
        else
            CT_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)G.nx * G.ny, cudaMemcpyDeviceToDevice, ws),
                        "state");
    }
    CT_CUDA_TRY(cudaEventRecord(ev_end, ws), "event");
    CT_CUDA_TRY(cudaEventRecord(ev_in, ws), "event");
    CT_CUDA_TRY(cudaStreamWaitEvent(user, ev_in, 0), "ordering caller's stream");
    CT_CUDA_TRY(cudaStreamSynchronize(ws), "solve");

    std::vector<float> trace(done > 0 ? done : 1, -1.0f);
    if (p->x_ref && done > 0)
        CT_CUDA_TRY(cudaMemcpy(trace.data(), W.trace, sizeof(float) * done, cudaMemcpyDeviceToHost), "read trace");
    if (rep) {
        rep->iters_done = done;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev_start, ev_end);
        rep->seconds = ms * 1e-3;
        rep->seconds_to_tol = -1.0;
        rep->rmsd_hu_last = (p->x_ref && done > 0) ? trace[done - 1] : -1.0f;
        for (int it = 0; it < done; it++) {
            float mi = 0.0f;
            cudaEventElapsedTime(&mi, ev_start, E.ev[3 + it]);
            if (rep->iter_seconds) rep->iter_seconds[it] = mi * 1e-3;
            if (p->x_ref) {
                if (rep->rmsd_trace_hu) rep->rmsd_trace_hu[it] = trace[it];
                if (rep->seconds_to_tol < 0.0 && trace[it] <= tol) rep->seconds_to_tol = mi * 1e-3;
            }
        }
    }
    return CT_OK;
}
