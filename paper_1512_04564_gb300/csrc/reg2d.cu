// Edge-preserving regularizer (Sec. III, Eq. (def_reg)) over the 8 neighbours of
// a 2-D image, its Huber-curvature SQS diagonal, and the fused x-update of
// Algorithm 1/2 (kappa: the optional voxel weights kappa_n, 1 when absent):
//
//   grad R_j = kappa_j sum_i beta_i [kappa_{j+s_i} phi'(x_j - x_{j+s_i}) - kappa_{j-s_i} phi'(x_{j-s_i} - x_j)]
//   D_R,j    = kappa_j sum_i 2 beta_i [kappa_{j+s_i} omega(x_j - x_{j+s_i}) + kappa_{j-s_i} omega(x_{j-s_i} - x_j)],
//              omega = phi'(t)/t
//   s        = rho (D_L x - h) + (1 - rho) g         (Algorithm 1)
//            = rho zeta + (1 - rho) g                (Algorithm 2; zeta is kept in h)
//   x+       = [x - (rho D_L + D_R)^{-1} (s + grad R)]_Omega
//
// Directions (1,0), (0,1), (1,1), (1,-1) with beta_i = beta/||s_i||; pairs
// reaching outside the image are absent.  The 2-D image of a fan-beam slice
// stays in L2, so neighbours are read through the read-only cache.
#include "ct_internal.cuh"

namespace ct {

namespace {

template <bool KAPPA>
__global__ void __launch_bounds__(256) reg_gradient_kernel(FanDev G, const float *__restrict__ x,
                                                           const float *__restrict__ kappa, float beta, Pot P,
                                                           float *__restrict__ grad, float *__restrict__ curv)
{
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31), iy = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (ix >= G.nx || iy >= G.ny) return;
    float gr, cv;
    reg_terms<false, KAPPA>(G, x, ix, iy, beta, P, gr, cv, kappa);
    const size_t j = (size_t)iy * G.nx + ix;
    grad[j] = gr;
    if (curv) curv[j] = cv;
}

// x+ into S.x_new; with the resident matrix also its transposed half of the packed image [x+ | x+^T]
// that the forward projector's rows index (S.x_new then holds 2 nx ny floats).
template <bool KAPPA>
__global__ void __launch_bounds__(256) reg_update_kernel(FanDev G, SolveDev S, float beta, Pot P)
{
    __shared__ float t[8][36];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int ix = blockIdx.x * 32 + lx, iy = blockIdx.y * 8 + ly;
    if (ix < G.nx && iy < G.ny) {
        const float rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
        float gr, cv;
        reg_terms<false, KAPPA>(G, S.x, ix, iy, beta, P, gr, cv, S.kappa);
        const size_t j = (size_t)iy * G.nx + ix;
        const float xj = S.x[j], dl = S.d_l[j], g = S.g[j], h = S.h[j];
        const float s = (S.algorithm == CT_ALG_PROPOSED) ? fmaf(rho, fmaf(dl, xj, -h), (1.0f - rho) * g)
                                                         : fmaf(rho, h, (1.0f - rho) * g);
        const float den = fmaf(rho, dl, cv);
        float xn = den > 0.0f ? xj - (s + gr) / den : xj;
        if (S.nonneg) xn = fmaxf(xn, 0.0f);
        S.x_new[j] = xn;
        t[ly][lx] = xn;
    }
    if (!G.row_ptr) return;  // the same for the whole grid
    __syncthreads();
    write_transposed_block(G, t, S.x_new);
}

__global__ void __launch_bounds__(256) fill_kernel(float *__restrict__ p, long long n, float v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// kappa_j = sqrt(num_j / den_j) with num = A'w, den = A'1; 0 where den_j = 0.
__global__ void __launch_bounds__(256) kappa_finish_kernel(float *__restrict__ kappa, const float *__restrict__ den,
                                                           long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = den[i];
        kappa[i] = d > 0.0f ? sqrtf(fmaxf(kappa[i], 0.0f) / d) : 0.0f;
    }
}

}  // namespace

cudaError_t launch_reg_gradient(const FanDev &G, const float *x, const float *kappa, float beta, float delta,
                                int potential, float *grad, float *curv, cudaStream_t st)
{
    Pot P{potential, potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / delta};
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    if (kappa)
        reg_gradient_kernel<true><<<grid, 256, 0, st>>>(G, x, kappa, beta, P, grad, curv);
    else
        reg_gradient_kernel<false><<<grid, 256, 0, st>>>(G, x, kappa, beta, P, grad, curv);
    return cudaGetLastError();
}

cudaError_t launch_reg_update(const FanDev &G, const SolveDev &S, float beta, float delta, int potential,
                              int maxcurv, cudaStream_t st)
{
    Pot P{potential, potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / delta, maxcurv};
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    if (S.kappa)
        reg_update_kernel<true><<<grid, 256, 0, st>>>(G, S, beta, P);
    else
        reg_update_kernel<false><<<grid, 256, 0, st>>>(G, S, beta, P);
    return cudaGetLastError();
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_reg_gradient(const ct_geom *g, const float *x, const float *kappa, float beta, float delta,
                                     int potential, float *grad, float *curv, void *stream)
{
    if (!g || !x || !grad) { set_error("ct_reg_gradient: null argument"); return CT_EINVAL; }
    if (potential < CT_POT_HYPERBOLA || potential > CT_POT_QUADRATIC) {
        set_error("unknown potential %d", potential);
        return CT_EINVAL;
    }
    if (!(beta >= 0.0f) || (potential != CT_POT_QUADRATIC && !(delta > 0.0f))) {
        set_error("need beta >= 0 and delta > 0");
        return CT_EINVAL;
    }
    if (g->helical) return helix_reg_gradient(g, x, kappa, beta, delta, potential, grad, curv, (cudaStream_t)stream);
    CT_CUDA_TRY(launch_reg_gradient(g->fan, x, kappa, beta, delta, potential, grad, curv, (cudaStream_t)stream),
                "ct_reg_gradient launch");
    return CT_OK;
}

extern "C" ct_status ct_kappa(const ct_geom *g, const float *w, float *kappa, void *stream)
{
    if (!g || !w || !kappa) { set_error("ct_kappa: null argument"); return CT_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int na = g->fan.na;
    const long long nvox = (long long)g->fan.nx * g->fan.ny * (g->helical ? g->hx.nz : 1);
    const long long nsino = (long long)na * g->fan.ns * (g->helical ? g->hx.nt : 1);
    float *den = nullptr;
    CT_CUDA_TRY(cudaMallocAsync(&den, sizeof(float) * (size_t)nvox, s), "ct_kappa scratch");
    struct Free {
        float *p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } guard{den, s};
    fill_kernel<<<4 * 152, 256, 0, s>>>(g->d_sino_ws, nsino, 1.0f);
    CT_CUDA_TRY(cudaGetLastError(), "ct_kappa fill");
    ct_status st = ct_back(g, g->d_sino_ws, den, nullptr, na, 1.0f, 0, stream);  // A'1
    if (st != CT_OK) return st;
    st = ct_back(g, w, kappa, nullptr, na, 1.0f, 0, stream);  // A'w
    if (st != CT_OK) return st;
    kappa_finish_kernel<<<4 * 152, 256, 0, s>>>(kappa, den, nvox);
    CT_CUDA_TRY(cudaGetLastError(), "ct_kappa finish");
    return CT_OK;
}
