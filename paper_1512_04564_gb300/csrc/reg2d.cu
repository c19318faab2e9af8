// Edge-preserving regularizer (Sec. III, Eq. (def_reg)) over the 8 neighbours of
// a 2-D image, its Huber-curvature SQS diagonal, and the fused x-update of
// Algorithm 1/2:
//
//   grad R_j = sum_i beta_i [phi'(x_j - x_{j+s_i}) - phi'(x_{j-s_i} - x_j)]
//   D_R,j    = sum_i 2 beta_i [omega(x_j - x_{j+s_i}) + omega(x_{j-s_i} - x_j)],  omega = phi'(t)/t
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

__global__ void __launch_bounds__(256) reg_gradient_kernel(FanDev G, const float *__restrict__ x, float beta, Pot P,
                                                           float *__restrict__ grad, float *__restrict__ curv)
{
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31), iy = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (ix >= G.nx || iy >= G.ny) return;
    float gr, cv;
    reg_terms(G, x, ix, iy, beta, P, gr, cv);
    const size_t j = (size_t)iy * G.nx + ix;
    grad[j] = gr;
    if (curv) curv[j] = cv;
}

__global__ void __launch_bounds__(256) reg_update_kernel(FanDev G, SolveDev S, float beta, Pot P)
{
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31), iy = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (ix >= G.nx || iy >= G.ny) return;
    const float rho = __ldcg(&S.rho_tab[__ldcg(&S.counter[0])]);
    float gr, cv;
    reg_terms(G, S.x, ix, iy, beta, P, gr, cv);
    const size_t j = (size_t)iy * G.nx + ix;
    const float xj = S.x[j], dl = S.d_l[j], g = S.g[j], h = S.h[j];
    const float s = (S.algorithm == CT_ALG_PROPOSED) ? fmaf(rho, fmaf(dl, xj, -h), (1.0f - rho) * g)
                                                     : fmaf(rho, h, (1.0f - rho) * g);
    const float den = fmaf(rho, dl, cv);
    float xn = den > 0.0f ? xj - (s + gr) / den : xj;
    if (S.nonneg) xn = fmaxf(xn, 0.0f);
    S.x_new[j] = xn;
}

}  // namespace

cudaError_t launch_reg_gradient(const FanDev &G, const float *x, float beta, float delta, int potential, float *grad,
                                float *curv, cudaStream_t st)
{
    Pot P{potential, potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / delta};
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    reg_gradient_kernel<<<grid, 256, 0, st>>>(G, x, beta, P, grad, curv);
    return cudaGetLastError();
}

cudaError_t launch_reg_update(const FanDev &G, const SolveDev &S, float beta, float delta, int potential,
                              int maxcurv, cudaStream_t st)
{
    Pot P{potential, potential == CT_POT_QUADRATIC ? 0.0f : 1.0f / delta, maxcurv};
    dim3 grid((G.nx + 31) / 32, (G.ny + 7) / 8);
    reg_update_kernel<<<grid, 256, 0, st>>>(G, S, beta, P);
    return cudaGetLastError();
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_reg_gradient(const ct_geom *g, const float *x, float beta, float delta, int potential,
                                     float *grad, float *curv, void *stream)
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
    if (g->helical) return helix_reg_gradient(g, x, beta, delta, potential, grad, curv, (cudaStream_t)stream);
    CT_CUDA_TRY(launch_reg_gradient(g->fan, x, beta, delta, potential, grad, curv, (cudaStream_t)stream),
                "ct_reg_gradient launch");
    return CT_OK;
}
