// Batched relaxed OS-LALM: many 2-D slices of uneven size, view count and
// subset count (Algorithm 1 per slice, Sec. III-A).  Slices of several
// geometries run the single-slice solver concurrently (solve_lanes); slices of
// one geometry that are large enough to fill the GPU alone go through the
// single-slice solver one after another, and the rest are solved together in
// ONE persistent cooperative launch.
//
// All slices advance in lockstep super-steps t = 0, 1, ...: slice i runs its
// subiteration t while t < n_iter * M_i, or until an outer iteration ends with
// its RMSD to x_ref at or below its stopping tolerance (the slice then leaves
// the launch; the launch ends when every slice has).  Each super-step has three phases,
// separated by a grid barrier, and the work units of every active slice are
// spread over all CTAs:
//   A. regularizer + x-update (256-pixel chunks); also, for slices that just
//      finished an outer iteration, the RMSD to x_ref and a %globaltimer stamp;
//   B. subset forward projection + weighted residual (units of 8 rays, one
//      warp per ray: resident-matrix rows, or the footprints on the fly);
//   C. subset back-projection + g/h update (16x16 tiles, one pixel per thread).
// The grid barrier is a generation counter with a bounded spin: if a wait
// gives up, the kernel records an error status and every CTA returns.
// Setup (D_L, initial gradient, optional FBP) uses the single-slice kernels.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ct_internal.cuh"

namespace ct {
namespace {

constexpr int kMaxSlices = 1024;
constexpr int kThreads = 256;
constexpr long long kMaxSpins = 1ll << 24;  // x ~100 ns sleep: ~2 s per barrier at most

// Failure-detection hook (ct_debug_barrier): the poll limit of every barrier wait, and a number of
// participants the barrier waits for beyond the grid, which never arrive (0 in normal use).
std::atomic<long long> g_barrier_polls{kMaxSpins};
std::atomic<int> g_barrier_missing{0};

struct BatchSlice {
    FanDev G;
    float *x, *x_new, *g, *h, *d_l, *resid;  // x_new: packed [x+ | x+^T] (2 nx ny floats)
    const float *y, *w, *x_ref;
    const float *kappa;  // regularizer voxel weights, or nullptr for kappa = 1
    const int *perm;     // views in subset order
    const int *sub_off;  // [M+1] offsets into perm
    const float *rho;    // [T]
    double *rmsd_acc;    // [n_iter][2]: sum of squares, count (FOV)
    unsigned long long *stamp;  // [n_iter] %globaltimer at the end of each outer iteration
    int *done_at;        // 0 while running; t + 1 once the slice stopped at super-step t (RMSD <= stop_hu)
    float stop_hu, hu;   // stopping tolerance (HU; 0: run all iterations) and HU per unit of x
    Pot P;
    float alpha, beta, r2max;
    int M, T, n_iter, nonneg, algorithm;
};

struct BatchCtl {
    unsigned int count;
    unsigned int gen;
    int error;
    int missing;             // participants beyond the grid that the barrier waits for (failure tests)
    unsigned long long t_start;
    long long max_polls;     // poll limit of one barrier wait
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait; returns false (for every thread of
// the CTA) once any CTA has given up.
__device__ bool grid_barrier(BatchCtl *ctl)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &ctl->gen;
        volatile int *verr = &ctl->error;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&ctl->count, 1u) + 1u;
        const long long max_polls = ctl->max_polls;
        int ok = 1;
        if (arrived == gridDim.x + (unsigned int)ctl->missing) {
            atomicExch(&ctl->count, 0u);
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g0) {
                if (*verr) { ok = 0; break; }
                if (++spins > max_polls) {
                    atomicExch(&ctl->error, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok && (*verr == 0);
    }
    __syncthreads();
    __threadfence();  // every thread: order its later loads after the barrier
    return s_ok != 0;
}

// Exclusive prefix over slices of their work units in this phase (shared memory).
template <class Units>
__device__ int build_prefix(int *s_pre, int nsl, Units units)
{
    __shared__ int s_part[kThreads / 32];
    // each thread sums a contiguous block of slices
    const int per = (nsl + kThreads - 1) / kThreads;
    const int a0 = threadIdx.x * per;
    int run = 0;
    for (int i = 0; i < per; i++) {
        const int s = a0 + i;
        if (s < nsl) {
            const int u = units(s);
            s_pre[s] = u;
            run += u;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_part[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int q = 0; q < warp; q++) base += s_part[q];
    int pos = base + incl - run;
    for (int i = 0; i < per; i++) {
        const int s = a0 + i;
        if (s < nsl) {
            const int u = s_pre[s];
            s_pre[s] = pos;
            pos += u;
        }
    }
    if (threadIdx.x == kThreads - 1) s_pre[nsl] = pos;
    __syncthreads();
    return s_pre[nsl];
}

// slice owning unit u: largest s with s_pre[s] <= u
__device__ __forceinline__ int find_slice(const int *s_pre, int nsl, int u)
{
    int lo = 0, hi = nsl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ void rmsd_units(const BatchSlice &B, int iter, int chunk)
{
    const int j = chunk * kThreads + threadIdx.x;
    const int npix = B.G.nx * B.G.ny;
    double s = 0.0, c = 0.0;
    if (j < npix) {
        const int ix = j % B.G.nx, iy = j / B.G.nx;
        const float X = ((float)ix - B.G.cxo) * B.G.dx, Y = ((float)iy - B.G.cyo) * B.G.dy;
        if (fmaf(X, X, Y * Y) <= B.r2max) {
            const double d = (double)__ldcg(&B.x[j]) - (double)B.x_ref[j];
            s = d * d;
            c = 1.0;
        }
    }
    // warp sums, then one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c > 0.0) {
        atomicAdd(&B.rmsd_acc[2 * iter], s);
        atomicAdd(&B.rmsd_acc[2 * iter + 1], c);
    }
}

// The on-the-fly projector paths of a slice without a resident matrix, out of line: inlined, their
// footprint arithmetic would cost the resident-matrix paths of the same phases their registers.
// Lane `lane` of a warp's share of ray (v, sc): sum over the wedge pixels it visits of a_ij x_j.
__device__ __noinline__ float fly_ray_part(const BatchSlice &B, int v, int sc, int lane)
{
    const float2 cs = __ldg(&B.G.view_cs[v]);
    float acc = 0.0f;
    ray_visit(B.G, v, sc, lane, 32, [&](int ix, int iy) {
        const float xv = __ldcg(&B.x_new[(size_t)iy * B.G.nx + ix]);
        if (xv == 0.0f) return;
        const Footprint F = pixel_footprint(B.G, v, cs.x, cs.y, ix, iy);
        acc = fmaf(cell_weight(F, sc), xv, acc);
    });
    return acc;
}

// sum over the subset's views v0 .. v0 + nv - 1 of pixel (ix, iy)'s footprint against the residual rows.
__device__ __noinline__ float fly_pixel_back(const BatchSlice &B, int v0, int nv, int ix, int iy)
{
    float acc = 0.0f;
    for (int k = 0; k < nv; k++) {
        const int v = B.perm[v0 + k];
        const float2 cs = __ldg(&B.G.view_cs[v]);
        const Footprint F = pixel_footprint(B.G, v, cs.x, cs.y, ix, iy);
        acc += footprint_dot_coherent(F, B.resid + (size_t)k * B.G.ns, B.G.ns);
    }
    return acc;
}

// Whether the RMSD of slice B to x_ref at the end of the outer iteration that subiteration t - 1 closed
// is at or below the slice's stopping tolerance (its sums are complete: the atomics of phase A precede a
// grid barrier).
__device__ __forceinline__ bool at_tol(const BatchSlice &B, int t)
{
    if (!(B.stop_hu > 0.0f) || t <= 0 || t > B.T || (t % B.M) != 0) return false;
    const int it = t / B.M - 1;
    const double c = __ldcg(&B.rmsd_acc[2 * it + 1]);
    return c > 0.0 && sqrt(__ldcg(&B.rmsd_acc[2 * it]) / c) * (double)B.hu <= (double)B.stop_hu;
}

// Whether slice B stopped before or at super-step t (done_at is written in phase B of the stopping
// super-step and read after later barriers).
__device__ __forceinline__ bool stopped(const BatchSlice &B, int t)
{
    const int d = __ldcg(B.done_at);
    return d != 0 && d - 1 <= t;
}

__global__ void __launch_bounds__(kThreads, 5) batched_kernel(const BatchSlice *__restrict__ SL, int nsl, int Tmax,
                                                             BatchCtl *ctl)
{
    __shared__ int s_pre[kMaxSlices + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->t_start = global_ns();
    for (int t = 0; t <= Tmax; t++) {
        // ---- phase A: iteration-end bookkeeping (RMSD, stamps) and K1 (regularizer + x-update)
        {
            // slices whose outer iteration ended with subiteration t-1
            auto ended = [&](int s) {
                const BatchSlice &B = SL[s];
                return t > 0 && t <= B.T && (t % B.M) == 0 && !stopped(B, t - 1);
            };
            if (blockIdx.x == 0 && threadIdx.x < 32) {
                for (int s = lane; s < nsl; s += 32)
                    if (ended(s)) SL[s].stamp[t / SL[s].M - 1] = global_ns();
            }
            const int total = build_prefix(s_pre, nsl, [&](int s) {
                const BatchSlice &B = SL[s];
                const int chunks = (B.G.nx * B.G.ny + kThreads - 1) / kThreads;
                const int rm = (ended(s) && B.x_ref) ? chunks : 0;
                const int k1 = (t < B.T && !stopped(B, t)) ? chunks : 0;
                return rm + k1;
            });
            if (total == 0) break;  // every slice has stopped (all CTAs see the same state)
            for (int u = blockIdx.x; u < total; u += gridDim.x) {
                const int s = find_slice(s_pre, nsl, u);
                const BatchSlice &B = SL[s];
                const int chunks = (B.G.nx * B.G.ny + kThreads - 1) / kThreads;
                int local = u - s_pre[s];
                const bool do_rmsd = ended(s) && B.x_ref;
                if (do_rmsd && local < chunks) {
                    rmsd_units(B, t / B.M - 1, local);
                    continue;
                }
                if (do_rmsd) local -= chunks;
                const int j = local * kThreads + threadIdx.x;
                if (j >= B.G.nx * B.G.ny) continue;
                const int ix = j % B.G.nx, iy = j / B.G.nx;
                const float rho = B.rho[t];
                float gr, cv;
                if (B.kappa)
                    reg_terms<true, true>(B.G, B.x, ix, iy, B.beta, B.P, gr, cv, B.kappa);
                else
                    reg_terms<true, false>(B.G, B.x, ix, iy, B.beta, B.P, gr, cv);
                const float xj = __ldcg(&B.x[j]), dl = __ldcg(&B.d_l[j]), g = __ldcg(&B.g[j]), h = __ldcg(&B.h[j]);
                const float sv = (B.algorithm == CT_ALG_PROPOSED) ? fmaf(rho, fmaf(dl, xj, -h), (1.0f - rho) * g)
                                                                  : fmaf(rho, h, (1.0f - rho) * g);
                const float den = fmaf(rho, dl, cv);
                float xn = den > 0.0f ? xj - (sv + gr) / den : xj;
                if (B.nonneg) xn = fmaxf(xn, 0.0f);
                B.x_new[j] = xn;
                if (B.G.row_ptr)  // the transposed half of the packed image the resident rows index
                    B.x_new[(size_t)B.G.nx * B.G.ny + (size_t)ix * B.G.ny + iy] = xn;
            }
        }
        if (t == Tmax) break;
        if (!grid_barrier(ctl)) return;
        // ---- phase B: subset forward projection with the weighted residual (one warp per ray)
        {
            // slices whose iteration that just ended met their tolerance stop here
            if (blockIdx.x == 0)
                for (int s = threadIdx.x; s < nsl; s += kThreads)
                    if (!stopped(SL[s], t) && at_tol(SL[s], t)) *SL[s].done_at = t + 1;
            const int total = build_prefix(s_pre, nsl, [&](int s) {
                const BatchSlice &B = SL[s];
                if (t >= B.T || stopped(B, t) || at_tol(B, t)) return 0;
                const int m = t % B.M;
                const int rays = (B.sub_off[m + 1] - B.sub_off[m]) * B.G.ns;
                return (rays + 7) / 8;
            });
            for (int u = blockIdx.x; u < total; u += gridDim.x) {
                const int s = find_slice(s_pre, nsl, u);
                const BatchSlice &B = SL[s];
                const int m = t % B.M;
                const int nv = B.sub_off[m + 1] - B.sub_off[m];
                const int r = (u - s_pre[s]) * 8 + warp;
                if (r >= nv * B.G.ns) continue;  // whole warp
                const int k = r / B.G.ns, sc = r - k * B.G.ns;
                const int v = B.perm[B.sub_off[m] + k];
                const size_t ri = (size_t)v * B.G.ns + sc;
                float acc = 0.0f;
                if (B.G.row_ptr) {
                    acc = csr_ray_dot<false, true>(B.G, B.G.row_ptr[ri], B.G.row_ptr[ri + 1], B.G.row_first[ri],
                                                   B.x_new, lane);
                } else {
                    acc = fly_ray_part(B, v, sc, lane);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) B.resid[(size_t)k * B.G.ns + sc] = __ldg(&B.w[ri]) * (acc - __ldg(&B.y[ri]));
            }
        }
        if (!grid_barrier(ctl)) return;
        // ---- phase C: subset back-projection + g/h update (16x16 tiles, one pixel per thread)
        {
            const int total = build_prefix(s_pre, nsl, [&](int s) {
                const BatchSlice &B = SL[s];
                return (t < B.T && !stopped(B, t) && !at_tol(B, t)) ? B.G.ntx * B.G.nty : 0;
            });
            for (int u = blockIdx.x; u < total; u += gridDim.x) {
                const int s = find_slice(s_pre, nsl, u);
                const BatchSlice &B = SL[s];
                const int tile = u - s_pre[s];
                const int ty = tile / B.G.ntx, tx = tile - ty * B.G.ntx;
                const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
                const int ix = tx * kTile + lx, iy = ty * kTile + ly;
                const int m = t % B.M;
                const int v0 = B.sub_off[m], nv = B.sub_off[m + 1] - v0;
                const int ixc = min(ix, B.G.nx - 1), iyc = min(iy, B.G.ny - 1);  // anchor of an in-image pixel
                float acc = 0.0f;
                if (B.G.rec_data) {  // stored records (warp w: chunk w of the tile), the next view's prefetched
                    const unsigned group = (unsigned)tile * (kTile * kTile / kRecGroup) + (threadIdx.x >> 5);
                    RecSlot r{};
                    if (nv > 0) r = rec_fetch(B.G, rec_word(B.G, B.perm[v0], group));
                    for (int k = 0; k < nv; k++) {
                        const RecSlot cur = r;
                        if (k + 1 < nv) r = rec_fetch(B.G, rec_word(B.G, B.perm[v0 + k + 1], group));
                        acc += rec_dot<true>(B.G, cur, B.resid + (size_t)k * B.G.ns,
                                             [&] { return rec_word(B.G, B.perm[v0 + k], group); });
                    }
                } else {
                    acc = fly_pixel_back(B, v0, nv, ixc, iyc);
                }
                if (ix >= B.G.nx || iy >= B.G.ny) continue;
                const size_t j = (size_t)iy * B.G.nx + ix;
                const float rho = B.rho[t];
                const float zeta = (float)B.M * acc;
                const float g = __ldcg(&B.g[j]), xp = __ldcg(&B.x_new[j]), a = B.alpha;
                const float ir = 1.0f / (rho + 1.0f);
                B.g[j] = fmaf(rho * ir, fmaf(a, zeta, (1.0f - a) * g), g * ir);
                if (B.algorithm == CT_ALG_PROPOSED)
                    B.h[j] = fmaf(a, fmaf(__ldcg(&B.d_l[j]), xp, -zeta), (1.0f - a) * __ldcg(&B.h[j]));
                else
                    B.h[j] = zeta;
                B.x[j] = xp;
            }
        }
        if (!grid_barrier(ctl)) return;
    }
}

double rho_cont(long k, double alpha)
{
    if (k == 0) return 1.0;
    const double q = M_PI / (alpha * (double)(k + 1));
    return q * std::sqrt(1.0 - 0.25 * q * q);
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace ct

using namespace ct;

namespace {

// Argument checks of one slice (index i, for the message).
ct_status validate_slice(int i, const ct_geom *g, const float *y, const float *w, const float *x,
                         const ct_solve_params *p, int dev)
{
    if (!g || !y || !w || !x) { set_error("slice %d: null argument", i); return CT_EINVAL; }
    if (g->device != dev) { set_error("slice %d: geometry on device %d, current %d", i, g->device, dev); return CT_EINVAL; }
    if (g->helical) { set_error("slice %d: batched solves take 2-D fan-beam slices", i); return CT_ENOTSUP; }
    if (p->M < 1 || p->M > g->fan.na || p->n_iter < 1 || p->n_iter > 100000 || !(p->alpha >= 1.0f && p->alpha < 2.0f) ||
        !(p->beta >= 0.0f) || p->potential < CT_POT_HYPERBOLA || p->potential > CT_POT_QUADRATIC ||
        (p->potential != CT_POT_QUADRATIC && !(p->delta > 0.0f)) ||
        (p->algorithm != CT_ALG_PROPOSED && p->algorithm != CT_ALG_SIMPLE) ||
        (!p->continuation && !(p->rho_fixed > 0.0f)) ||
        (p->curvature != CT_CURV_HUBER && p->curvature != CT_CURV_MAX) || !(p->dl_scale >= 0.0f)) {
        set_error("slice %d: invalid solver parameters", i);
        return CT_EINVAL;
    }
    if (p->init_fbp) {
        ct_status sf = validate_fbp(g, CT_FBP_HANN);
        if (sf != CT_OK) return sf;
    }
    if ((long)p->n_iter * p->M > 50000000L) { set_error("slice %d: n_iter * M too large", i); return CT_EINVAL; }
    if (p->start_iter != 0) { set_error("slice %d: batched solves do not resume (start_iter)", i); return CT_ENOTSUP; }
    return CT_OK;
}

// The persistent cooperative launch over nslices (already validated) slices.
ct_status persistent_batch(const ct_geom *const *geoms, const float *const *y, const float *const *w,
                           const ct_solve_params *params, float *const *x_inout, int nslices,
                           ct_solve_report *reports, void *stream)
{
    int dev = 0;
    CT_CUDA_TRY(cudaGetDevice(&dev), "current device");
    // size the arena
    std::vector<size_t> off(nslices);
    size_t total = 0;
    int Tmax = 0;
    for (int i = 0; i < nslices; i++) {
        const ct_geom *g = geoms[i];
        const ct_solve_params *p = &params[i];
        const int T = p->n_iter * p->M;
        Tmax = std::max(Tmax, T);
        int max_sub = (g->fan.na + p->M - 1) / p->M;
        const size_t npix = (size_t)g->fan.nx * g->fan.ny;
        off[i] = total;
        total += al256(npix * 8) + al256(npix * 4) * 3 + al256((size_t)max_sub * g->fan.ns * 4) + al256((size_t)g->fan.na * 4) +
                 al256((size_t)(p->M + 1) * 4) + al256((size_t)T * 4) + al256((size_t)p->n_iter * 16) +
                 al256((size_t)p->n_iter * 8) + al256(4);
    }
    const size_t desc_off = total;
    total += al256(sizeof(BatchSlice) * nslices) + al256(sizeof(BatchCtl));
    char *arena = nullptr;
    CT_CUDA_TRY(cudaMalloc(&arena, total), "allocating the batch arena");
    struct ArenaGuard {
        char *p;
        ~ArenaGuard() { cudaFree(p); }
    } aguard{arena};

    cudaStream_t user = (cudaStream_t)stream, ws = nullptr;
    CT_CUDA_TRY(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking), "creating batch stream");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sguard{ws};
    cudaEvent_t ev_in, ev0, ev1, ev2;
    CT_CUDA_TRY(cudaEventCreate(&ev_in), "event");
    CT_CUDA_TRY(cudaEventCreate(&ev0), "event");
    CT_CUDA_TRY(cudaEventCreate(&ev1), "event");
    CT_CUDA_TRY(cudaEventCreate(&ev2), "event");
    struct EvGuard {
        cudaEvent_t a, b, c, d;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c); cudaEventDestroy(d); }
    } eguard{ev_in, ev0, ev1, ev2};
    CT_CUDA_TRY(cudaEventRecord(ev_in, user), "event");
    CT_CUDA_TRY(cudaStreamWaitEvent(ws, ev_in, 0), "ordering after caller's stream");

    std::vector<BatchSlice> hs(nslices);
    CT_CUDA_TRY(cudaMemsetAsync(arena, 0, total, ws), "clearing the batch arena");
    for (int i = 0; i < nslices; i++) {
        const ct_geom *g = geoms[i];
        const ct_solve_params *p = &params[i];
        const int M = p->M, T = p->n_iter * M;
        const int max_sub = (g->fan.na + M - 1) / M;
        const size_t npix = (size_t)g->fan.nx * g->fan.ny;
        char *b = arena + off[i];
        BatchSlice &B = hs[i];
        B.G = g->fan;
        B.x = x_inout[i];
        B.x_new = (float *)b; b += al256(npix * 8);  // packed [x+ | x+^T]
        B.g = (float *)b; b += al256(npix * 4);
        B.h = (float *)b; b += al256(npix * 4);
        B.d_l = (float *)b; b += al256(npix * 4);
        B.resid = (float *)b; b += al256((size_t)max_sub * g->fan.ns * 4);
        int *perm = (int *)b; b += al256((size_t)g->fan.na * 4);
        int *sub = (int *)b; b += al256((size_t)(M + 1) * 4);
        float *rho = (float *)b; b += al256((size_t)T * 4);
        B.rmsd_acc = (double *)b; b += al256((size_t)p->n_iter * 16);
        B.stamp = (unsigned long long *)b; b += al256((size_t)p->n_iter * 8);
        B.done_at = (int *)b;
        B.stop_hu = p->x_ref ? p->stop_rmsd_hu : 0.0f;
        B.hu = p->hu_per_unit;
        B.y = y[i];
        B.w = w[i];
        B.x_ref = p->x_ref;
        B.kappa = p->kappa;
        B.perm = perm;
        B.sub_off = sub;
        B.rho = rho;
        B.P = Pot{p->potential, p->potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / p->delta, p->curvature};
        B.alpha = p->alpha;
        B.beta = p->beta;
        const double R = p->fov_radius > 0.0f ? (double)p->fov_radius : g->fov_radius;
        B.r2max = (float)(R * R);
        B.M = M;
        B.T = T;
        B.n_iter = p->n_iter;
        B.nonneg = p->nonneg;
        B.algorithm = p->algorithm;
        std::vector<int> hp;
        std::vector<int> ho(M + 1);
        for (int m = 0; m < M; m++) {
            ho[m] = (int)hp.size();
            for (int v = m; v < g->fan.na; v += M) hp.push_back(v);
        }
        ho[M] = g->fan.na;
        std::vector<float> hr(T);
        for (int k = 0; k < T; k++) hr[k] = (float)(p->continuation ? rho_cont(k, p->alpha) : (double)p->rho_fixed);
        CT_CUDA_TRY(cudaMemcpyAsync(perm, hp.data(), sizeof(int) * hp.size(), cudaMemcpyHostToDevice, ws), "upload");
        CT_CUDA_TRY(cudaMemcpyAsync(sub, ho.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice, ws), "upload");
        CT_CUDA_TRY(cudaMemcpyAsync(rho, hr.data(), sizeof(float) * T, cudaMemcpyHostToDevice, ws), "upload");
        CT_CUDA_TRY(cudaStreamSynchronize(ws), "upload");  // host vectors go out of scope
    }
    BatchSlice *dsl = (BatchSlice *)(arena + desc_off);
    BatchCtl *ctl = (BatchCtl *)(arena + desc_off + al256(sizeof(BatchSlice) * nslices));
    CT_CUDA_TRY(cudaMemcpyAsync(dsl, hs.data(), sizeof(BatchSlice) * nslices, cudaMemcpyHostToDevice, ws), "upload");
    BatchCtl hc0{};
    hc0.max_polls = g_barrier_polls.load();
    hc0.missing = g_barrier_missing.load();
    CT_CUDA_TRY(cudaMemcpyAsync(ctl, &hc0, sizeof(hc0), cudaMemcpyHostToDevice, ws), "upload");

    // persistent grid: every CTA co-resident (cooperative launch)
    int nsm = 0, per_sm = 0;
    CT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
    CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel, kThreads, 0), "occupancy");
    if (per_sm < 1) { set_error("batched kernel cannot be resident"); return CT_ECUDA; }
    const int grid = nsm * per_sm;

    // the geometries' ray sums A 1 (computed once per geometry, like the resident matrix)
    for (int i = 0; i < nslices; i++) CT_CUDA_TRY(ensure_ray_sums(const_cast<ct_geom *>(geoms[i]), ws), "ray sums A 1");
    CT_CUDA_TRY(cudaEventRecord(ev0, ws), "event");
    for (int i = 0; i < nslices; i++) {
        const ct_geom *g = geoms[i];
        const ct_solve_params *p = &params[i];
        BatchSlice &B = hs[i];
        if (p->init_fbp) CT_CUDA_TRY(launch_fbp(g, y[i], x_inout[i], CT_FBP_HANN, ws), "initial FBP");
        CT_CUDA_TRY(launch_weighted_ray_sums(g, w[i], g->d_sino_ws, ws), "D_L weights");
        CT_CUDA_TRY(launch_bp(g->fan, BP_PLAIN, g->d_sino_ws, g->d_views_all, g->fan.na, B.d_l,
                              p->dl_scale > 0.0f ? p->dl_scale : 1.0f, 0, nullptr, ws),
                    "D_L back");
        // rho = 1, zeta = g = M grad L_M(x), h = D_L x - zeta (last subset)
        const int M = p->M;
        const int vlast = (g->fan.na - (M - 1) + M - 1) / M;  // views in subset M-1
        const int off_last = g->fan.na - vlast;
        SolveDev S{};
        S.x = x_inout[i];
        S.g = B.g;
        S.h = B.h;
        S.d_l = B.d_l;
        S.M_scale = (float)M;
        S.algorithm = p->algorithm;
        CT_CUDA_TRY(launch_fp(g->fan, FP_RESID, x_inout[i], B.perm + off_last, vlast, B.resid, y[i], w[i], ws),
                    "init forward");
        CT_CUDA_TRY(launch_bp(g->fan, BP_SOLVE_INIT, B.resid, B.perm + off_last, vlast, nullptr, 1.0f, 0, &S, ws),
                    "init back");
    }
    CT_CUDA_TRY(cudaEventRecord(ev1, ws), "event");
    int nsl = nslices;
    void *args[] = {(void *)&dsl, (void *)&nsl, (void *)&Tmax, (void *)&ctl};
    CT_CUDA_TRY(cudaLaunchCooperativeKernel((void *)batched_kernel, dim3(grid), dim3(kThreads), args, 0, ws),
                "persistent batched launch");
    CT_CUDA_TRY(cudaEventRecord(ev2, ws), "event");
    CT_CUDA_TRY(cudaEventRecord(ev_in, ws), "event");
    CT_CUDA_TRY(cudaStreamWaitEvent(user, ev_in, 0), "ordering caller's stream");
    CT_CUDA_TRY(cudaStreamSynchronize(ws), "batched solve");

    BatchCtl hctl;
    CT_CUDA_TRY(cudaMemcpy(&hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost), "read status");
    if (hctl.error) {
        set_error("batched solve: a grid barrier wait gave up");
        return CT_ETIMEOUT;
    }
    float ms_setup = 0.0f, ms_all = 0.0f;
    cudaEventElapsedTime(&ms_setup, ev0, ev1);
    cudaEventElapsedTime(&ms_all, ev0, ev2);
    if (reports) {
        for (int i = 0; i < nslices; i++) {
            const ct_solve_params *p = &params[i];
            const int n = p->n_iter;
            std::vector<double> acc(2 * (size_t)n);
            std::vector<unsigned long long> st(n);
            CT_CUDA_TRY(cudaMemcpy(acc.data(), hs[i].rmsd_acc, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost), "read");
            CT_CUDA_TRY(cudaMemcpy(st.data(), hs[i].stamp, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost),
                        "read");
            int done_at = 0;
            CT_CUDA_TRY(cudaMemcpy(&done_at, hs[i].done_at, sizeof(int), cudaMemcpyDeviceToHost), "read");
            ct_solve_report *r = &reports[i];
            r->iters_done = done_at ? (done_at - 1) / p->M : n;
            r->seconds = ms_all * 1e-3;
            r->seconds_to_tol = -1.0;
            r->rmsd_hu_last = -1.0f;
            const float tol = p->stop_rmsd_hu > 0.0f ? p->stop_rmsd_hu : 1.0f;
            for (int k = 0; k < r->iters_done; k++) {
                const double tk = ms_setup * 1e-3 + (double)(st[k] - hctl.t_start) * 1e-9;
                if (r->iter_seconds) r->iter_seconds[k] = tk;
                if (p->x_ref) {
                    const float v = acc[2 * k + 1] > 0 ? (float)(std::sqrt(acc[2 * k] / acc[2 * k + 1]) * p->hu_per_unit)
                                                       : 0.0f;
                    if (r->rmsd_trace_hu) r->rmsd_trace_hu[k] = v;
                    r->rmsd_hu_last = v;
                    if (r->seconds_to_tol < 0.0 && v <= tol) r->seconds_to_tol = tk;
                }
            }
        }
    }
    return CT_OK;
}

// A slice of at least this many pixels keeps every SM busy with its own
// subsets (a 384 x 384 slice has 576 back-projection tiles and, at 984 views
// in 20 subsets, over 20,000 rays per subset), so the graph-replayed
// single-slice solver, whose projector kernels run at full occupancy, is
// faster for it than a share of the persistent launch's super-steps; only
// smaller slices are batched.
constexpr long kSoloPixels = 384L * 384L;

// Report of a slice solved alone: its RMSD trace and iteration times, shifted
// by the device time of the slices solved before it.
void fill_solo_report(ct_solve_report *r, const ct_solve_params *p, const ct_solve_report &got,
                      const std::vector<float> &trace, const std::vector<double> &times, double t0)
{
    const int n = got.iters_done;
    const float tol = p->stop_rmsd_hu > 0.0f ? p->stop_rmsd_hu : 1.0f;
    r->iters_done = n;
    r->seconds_to_tol = -1.0;
    r->rmsd_hu_last = got.rmsd_hu_last;
    for (int k = 0; k < n; k++) {
        const double tk = t0 + times[k];
        if (r->iter_seconds) r->iter_seconds[k] = tk;
        if (p->x_ref) {
            if (r->rmsd_trace_hu) r->rmsd_trace_hu[k] = trace[k];
            if (r->seconds_to_tol < 0.0 && trace[k] <= tol) r->seconds_to_tol = tk;
        }
    }
}

// Slices solved concurrently: the slices of one geometry (which owns its solver workspace) form a group;
// up to kSoloLanes lanes, each a host thread running the single-slice graph solver on a stream of its own,
// take the groups one after another from a queue ordered by work (pixels x views x iterations, largest
// first) and solve a group's slices in turn.  Slices then share the GPU: a 384 x 384 slice's projector
// launches fill about half of it, a 256 x 256 slice's less, and one lane's per-iteration host step (the
// stopping test) leaves the GPU to the others; taking groups from a queue keeps the lanes busy although
// slices stop after different iteration counts.  Each report counts from `ev0` (recorded on the caller's
// stream); *t_end receives the device time from ev0 to the last lane's end.
constexpr int kSoloLanes = 4;

ct_status solve_lanes(const ct_geom *const *geoms, const float *const *y, const float *const *w,
                      const ct_solve_params *params, float *const *x_inout, const std::vector<int> &solo,
                      ct_solve_report *reports, cudaStream_t caller, int dev, double *t_end)
{
    // geometries in order of first appearance, with their slices and work
    std::vector<const ct_geom *> gkey;
    std::vector<std::vector<int>> gsl;
    std::vector<double> gwork;
    for (int i : solo) {
        size_t k = 0;
        while (k < gkey.size() && gkey[k] != geoms[i]) k++;
        if (k == gkey.size()) {
            gkey.push_back(geoms[i]);
            gsl.emplace_back();
            gwork.push_back(0.0);
        }
        gsl[k].push_back(i);
        gwork[k] += (double)geoms[i]->fan.nx * geoms[i]->fan.ny * geoms[i]->fan.na * std::max(params[i].n_iter, 1);
    }
    const int nl = std::min<int>(kSoloLanes, (int)gkey.size());
    std::vector<int> queue(gkey.size());
    for (size_t k = 0; k < queue.size(); k++) queue[k] = (int)k;
    std::stable_sort(queue.begin(), queue.end(), [&](int a, int b) { return gwork[a] > gwork[b]; });
    std::atomic<int> next{0};
    cudaEvent_t ev0 = nullptr;
    CT_CUDA_TRY(cudaEventCreate(&ev0), "event");
    struct EvGuard {
        cudaEvent_t e;
        ~EvGuard() { cudaEventDestroy(e); }
    } g0{ev0};
    CT_CUDA_TRY(cudaEventRecord(ev0, caller), "event");
    std::vector<ct_status> status(nl, CT_OK);
    std::vector<std::string> message(nl);
    std::vector<double> lane_end(nl, 0.0);
    auto run = [&](int l) {
        cudaStream_t ls = nullptr;
        cudaEvent_t ev = nullptr;
        auto fail = [&](ct_status st) {
            status[l] = st;
            message[l] = ct_last_error();
        };
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&ev) != cudaSuccess || cudaStreamWaitEvent(ls, ev0, 0) != cudaSuccess) {
            set_error("batched solve: setting up a lane stream failed");
            fail(CT_ECUDA);
        }
        while (status[l] == CT_OK) {
            const int gq = next.fetch_add(1);
            if (gq >= (int)queue.size()) break;
            for (const int i : gsl[queue[gq]]) {
                ct_solve_params pi = params[i];
                std::vector<float> trace(std::max(pi.n_iter, 1));
                std::vector<double> times(std::max(pi.n_iter, 1));
                ct_solve_report got{};
                got.rmsd_trace_hu = trace.data();
                got.iter_seconds = times.data();
                float ms = 0.0f;
                if (cudaEventRecord(ev, ls) != cudaSuccess) {
                    set_error("batched solve: event record failed");
                    fail(CT_ECUDA);
                    break;
                }
                const ct_status st = ct_relaxed_oslalm_solve(geoms[i], y[i], w[i], &pi, x_inout[i], &got, ls);
                if (st != CT_OK) {
                    fail(st);
                    break;
                }
                cudaEventElapsedTime(&ms, ev0, ev);  // both complete: the solve synchronised its stream
                if (reports) fill_solo_report(&reports[i], &params[i], got, trace, times, ms * 1e-3);
                lane_end[l] = ms * 1e-3 + got.seconds;
            }
        }
        if (ev) cudaEventDestroy(ev);
        if (ls) {
            cudaStreamSynchronize(ls);
            cudaStreamDestroy(ls);
        }
    };
    if (nl == 1) {
        run(0);
    } else {
        std::vector<std::thread> pool;
        for (int l = 0; l < nl; l++) pool.emplace_back(run, l);
        for (auto &t : pool) t.join();
    }
    for (int l = 0; l < nl; l++)
        if (status[l] != CT_OK) {
            set_error("%s", message[l].c_str());
            return status[l];
        }
    *t_end = *std::max_element(lane_end.begin(), lane_end.end());
    return CT_OK;
}

}  // namespace

extern "C" ct_status ct_debug_barrier(long long max_polls, int missing)
{
    if (max_polls < 0 || missing < 0 || missing > 1024) {
        set_error("ct_debug_barrier: need max_polls >= 0 and 0 <= missing <= 1024");
        return CT_EINVAL;
    }
    g_barrier_polls.store(max_polls > 0 ? max_polls : kMaxSpins);
    g_barrier_missing.store(missing);
    return CT_OK;
}

extern "C" ct_status ct_relaxed_oslalm_solve_batched(const ct_geom *const *geoms, const float *const *y,
                                                     const float *const *w, const ct_solve_params *params,
                                                     float *const *x_inout, int nslices, ct_solve_report *reports,
                                                     void *stream)
{
    if (!geoms || !y || !w || !params || !x_inout || nslices < 1 || nslices > kMaxSlices) {
        set_error("ct_relaxed_oslalm_solve_batched: null argument or nslices outside [1, %d]", kMaxSlices);
        return CT_EINVAL;
    }
    int dev = 0;
    CT_CUDA_TRY(cudaGetDevice(&dev), "current device");
    for (int i = 0; i < nslices; i++) {
        const ct_status st = validate_slice(i, geoms[i], y[i], w[i], x_inout[i], &params[i], dev);
        if (st != CT_OK) return st;
    }
    // slices of two or more geometries: every slice by the single-slice solver, concurrently over the
    // geometries (lanes); slices of one geometry (they share its workspace, so run one at a time): the large
    // ones alone, the rest in one persistent launch after them
    bool several = false;
    for (int i = 1; i < nslices; i++) several = several || geoms[i] != geoms[0];
    std::vector<int> solo, shared;
    for (int i = 0; i < nslices; i++)
        ((several || (long)geoms[i]->fan.nx * geoms[i]->fan.ny >= kSoloPixels) ? solo : shared).push_back(i);

    double t_total = 0.0;  // device time of the slices solved so far
    if (!solo.empty()) {
        const ct_status st = solve_lanes(geoms, y, w, params, x_inout, solo, reports, (cudaStream_t)stream, dev,
                                         &t_total);
        if (st != CT_OK) return st;
    }
    if (!shared.empty()) {
        const size_t n = shared.size();
        std::vector<const ct_geom *> gs(n);
        std::vector<const float *> ys(n), wsl(n);
        std::vector<float *> xs(n);
        std::vector<ct_solve_params> ps(n);
        std::vector<ct_solve_report> rs(n);
        for (size_t k = 0; k < n; k++) {
            const int i = shared[k];
            gs[k] = geoms[i];
            ys[k] = y[i];
            wsl[k] = w[i];
            xs[k] = x_inout[i];
            ps[k] = params[i];
            if (reports) rs[k] = reports[i];
        }
        const ct_status st = persistent_batch(gs.data(), ys.data(), wsl.data(), ps.data(), xs.data(), (int)n,
                                              reports ? rs.data() : nullptr, stream);
        if (st != CT_OK) return st;
        if (reports) {
            for (size_t k = 0; k < n; k++) {
                ct_solve_report *r = &reports[shared[k]];
                *r = rs[k];
                if (r->iter_seconds)
                    for (int it = 0; it < r->iters_done; it++) r->iter_seconds[it] += t_total;
                if (r->seconds_to_tol >= 0.0) r->seconds_to_tol += t_total;
            }
        }
        t_total += rs.empty() || !reports ? 0.0 : rs[0].seconds;
    }
    if (reports)
        for (int i = 0; i < nslices; i++) reports[i].seconds = t_total;
    return CT_OK;
}
