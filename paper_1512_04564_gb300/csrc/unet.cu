// Learned warm start: a U-Net mapping an FBP image to an estimate of the PWLS
// solution x*, built on BF16 3x3 convolutions with FP32 accumulation on the
// tensor cores (tcgen05.mma in inline PTX), forward and backward, plus the
// small kernels around them.  The paper has no counterpart; the C ABI is in
// include/ct_unet.h.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ct_unet.h"
#include "ct_internal.cuh"
#include "tc_conv_tma.cuh"
#include "tc_gemm.cuh"

namespace ct {
namespace {

using bf16 = __nv_bfloat16;

// Plain GEMM C[M][N] = A[M][K] * B[N][K]^T (BF16 in, FP32 out).
template <int NT>
struct PlainGemm {
    const bf16 *A, *B;
    float *C;
    int M, N, K;
    struct Ctx {
        int m0, n0;
    };
    __device__ Ctx init(int m0, int n0, int) const { return Ctx{m0, n0}; }
    __device__ void load(int s, uint32_t sa, uint32_t sb, const Ctx &x, int tid) const
    {
        const int k0 = s * tc::kStageK, m0 = x.m0, n0 = x.n0;
        // a warp stages 16 rows x 2 adjacent 16-byte chunks: 32-byte sectors from global memory,
        // and the 8 row residues mod 8 (the shared-memory bank groups of the core-matrix layout)
        const int jr = 2 * (tid >> 5) + (tid & 1), rr = (tid >> 1) & 15;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int r = rr + 16 * i, j = jr;
            const int m = m0 + r, k = k0 + 8 * j;
            const bool ok = m < M && k < K;
            tc::cp_async16(sa + tc::tile_offset(r, 8 * j), ok ? A + (size_t)m * K + k : A, ok);
        }
#pragma unroll
        for (int i = 0; i < NT / 16; i++) {
            const int r = rr + 16 * i, j = jr;
            const int n = n0 + r, k = k0 + 8 * j;
            const bool ok = n < N && k < K;
            tc::cp_async16(sb + tc::tile_offset(r, 8 * j), ok ? B + (size_t)n * K + k : B, ok);
        }
    }
    __device__ void store(int m, int n, const float (&v)[16], const Ctx &) const
    {
        if (m >= M) return;
#pragma unroll
        for (int i = 0; i < 16; i++)
            if (n + i < N) C[(size_t)m * N + n + i] = v[i];
    }
};

// Input of a 3x3 convolution as the GEMM sees it: the channel concatenation of
// tensor 1 (c1 channels, optionally stored at half resolution and read through
// a nearest-neighbour 2x upsampling) and tensor 2 (c2 channels, full
// resolution), all BF16 NHWC.  Channel counts are multiples of 8.
struct ConvIn {
    const bf16 *t1;
    int c1, up1;
    const bf16 *t2;
    int c2;
    __device__ __forceinline__ const bf16 *at(int n, int y, int x, int c, int H, int W) const
    {
        if (c < c1) {
            if (up1) return t1 + (((size_t)n * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1)) * c1 + c;
            return t1 + (((size_t)n * H + y) * W + x) * c1 + c;
        }
        return t2 + (((size_t)n * H + y) * W + x) * c2 + (c - c1);
    }
};

enum ConvEpi { EPI_RELU = 0, EPI_DGRAD = 1 };

// Implicit-GEMM 3x3 convolution (padding 1): rows = output pixels, K = (tap,
// input channel), B = weights [N][9][Ci] (K contiguous).
//   EPI_RELU : out[p][n] = bf16(relu(acc + bias[n]))                    (forward)
//   EPI_DGRAD: the weights are the flipped transpose, the input is dOut, and
//              acc is dL/d(input of the forward conv); it is masked by the
//              forward input's ReLU support and split into the gradients of
//              tensor 1 (full resolution) and tensor 2.
template <int NT, int EPI>
struct ConvGemm {
    ConvIn in;
    const bf16 *w;
    const float *bias;
    bf16 *out;        // EPI_RELU: [P][N];  EPI_DGRAD: gradient of tensor 1 [P][m1]
    ConvIn mask;      // EPI_DGRAD: the forward input (ReLU support); mask.c1 + mask.c2 = N
    bf16 *out2;       // EPI_DGRAD: gradient of tensor 2 [P][mask.c2]
    int B, H, W, Ci, N;
    struct Ctx {
        int n[8], y[8], x[8];
        int m0, n0;
    };
    __device__ Ctx init(int m0, int n0, int tid) const
    {
        Ctx c;
        c.m0 = m0;
        c.n0 = n0;
        const int P = B * H * W;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int p = m0 + ((tid >> 1) & 15) + 16 * i;  // the rows load() stages (see there)
            if (p < P) {
                c.x[i] = p % W;
                const int q = p / W;
                c.y[i] = q % H;
                c.n[i] = q / H;
            } else {
                c.n[i] = -1;
                c.y[i] = c.x[i] = 0;
            }
        }
        return c;
    }
    __device__ void load(int s, uint32_t sa, uint32_t sb, const Ctx &c, int tid) const
    {
        // a warp stages 16 rows x 2 adjacent 16-byte chunks (32-byte global sectors; the 8 row
        // residues mod 8 spread the shared-memory stores over all bank groups)
        const int j = 2 * (tid >> 5) + (tid & 1), rr = (tid >> 1) & 15, Kt = 9 * Ci;
        const int k = s * tc::kStageK + 8 * j;
        const int tap = k / Ci, ci = k - tap * Ci;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int r = rr + 16 * i;
            const int yy = c.y[i] + dy, xx = c.x[i] + dx;
            const bool ok = k < Kt && c.n[i] >= 0 && yy >= 0 && yy < H && xx >= 0 && xx < W;
            tc::cp_async16(sa + tc::tile_offset(r, 8 * j), ok ? in.at(c.n[i], yy, xx, ci, H, W) : in.t1, ok);
        }
#pragma unroll
        for (int i = 0; i < NT / 16; i++) {
            const int r = rr + 16 * i, jj = j;
            const int n = c.n0 + r, kk = s * tc::kStageK + 8 * jj;
            const bool ok = n < N && kk < Kt;
            tc::cp_async16(sb + tc::tile_offset(r, 8 * jj), ok ? w + (size_t)n * Kt + kk : w, ok);
        }
    }
    __device__ void store(int p, int n, const float (&v)[16], const Ctx &c) const
    {
        if (p >= B * H * W || n >= N) return;
        __align__(16) bf16 o[16];
        if (EPI == EPI_RELU) {
#pragma unroll
            for (int i = 0; i < 16; i++) o[i] = __float2bfloat16_rn(fmaxf(v[i] + __ldg(&bias[n + i]), 0.0f));
            uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)p * N + n);
            dst[0] = reinterpret_cast<const uint4 *>(o)[0];
            dst[1] = reinterpret_cast<const uint4 *>(o)[1];
        } else {
            const int x = p % W, q = p / W, y = q % H, im = q / H;
            const bf16 *mk = mask.at(im, y, x, n, H, W);
            __align__(16) bf16 mv[16];
            reinterpret_cast<uint4 *>(mv)[0] = __ldg(reinterpret_cast<const uint4 *>(mk));
            reinterpret_cast<uint4 *>(mv)[1] = __ldg(reinterpret_cast<const uint4 *>(mk) + 1);
#pragma unroll
            for (int i = 0; i < 16; i++) o[i] = __float2bfloat16_rn(__bfloat162float(mv[i]) > 0.0f ? v[i] : 0.0f);
            bf16 *dst = n < mask.c1 ? out + (size_t)p * mask.c1 + n : out2 + (size_t)p * mask.c2 + (n - mask.c1);
            reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
            reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
        }
    }
};

// Weight gradient of a 3x3 convolution as a GEMM: rows m = (tap, ci) plus one
// row of ones (m = 9 Ci: the bias gradient), columns = output channels, K =
// output pixels (split over blockIdx.z).  Tiles are staged transposed (pixels
// along K) with plain loads and 2-byte shared stores.  Partial sums go to
// part[split][m][n] (FP32); a reduction kernel adds the splits.
template <int NT>
struct WgradGemm {
    ConvIn in;
    const bf16 *gout;  // [P][N]
    float *part;
    int B, H, W, Ci, N, Mrows, Mpad, steps_per_split, k_steps_total;
    struct Ctx {
        int m0, n0, s0;
    };
    __device__ Ctx init(int m0, int n0, int) const { return Ctx{m0, n0, (int)blockIdx.z * steps_per_split}; }
    __device__ void load(int s, uint32_t sa, uint32_t sb, const Ctx &c, int tid) const
    {
        const int P = B * H * W;
        const int gs = c.s0 + s;
        const int p0 = gs * tc::kStageK;
        const bool stage_ok = gs < k_steps_total;
        // A: 16 groups of 8 rows x 64 pixels
#pragma unroll 2
        for (int i = 0; i < 8; i++) {
            const int t = tid + 128 * i, kk = t & 63, g = t >> 6;
            const int m = c.m0 + 8 * g;
            const int p = p0 + kk;
            __align__(16) bf16 v[8];
            reinterpret_cast<uint4 *>(v)[0] = make_uint4(0u, 0u, 0u, 0u);
            if (stage_ok && p < P) {
                if (m < 9 * Ci) {
                    const int tap = m / Ci, ci = m - tap * Ci;
                    const int x = p % W, q = p / W, y = q % H, im = q / H;
                    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
                    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                        reinterpret_cast<uint4 *>(v)[0] = __ldg(reinterpret_cast<const uint4 *>(in.at(im, yy, xx, ci, H, W)));
                } else if (m == 9 * Ci) {
                    v[0] = __float2bfloat16_rn(1.0f);
                }
            }
            const uint32_t base = sa + tc::tile_offset(8 * g, kk);
            const unsigned short *u = reinterpret_cast<const unsigned short *>(v);
#pragma unroll
            for (int e = 0; e < 8; e++)
                asm volatile("st.shared.u16 [%0], %1;" ::"r"(base + 16 * e), "h"(u[e]) : "memory");
        }
        // B: NT/8 groups of 8 output channels x 64 pixels
#pragma unroll 2
        for (int i = 0; i < NT / 16; i++) {
            const int t = tid + 128 * i, kk = t & 63, g = t >> 6;
            const int n = c.n0 + 8 * g, p = p0 + kk;
            __align__(16) bf16 v[8];
            reinterpret_cast<uint4 *>(v)[0] = make_uint4(0u, 0u, 0u, 0u);
            if (stage_ok && p < P && n < N)
                reinterpret_cast<uint4 *>(v)[0] = __ldg(reinterpret_cast<const uint4 *>(gout + (size_t)p * N + n));
            const uint32_t base = sb + tc::tile_offset(8 * g, kk);
            const unsigned short *u = reinterpret_cast<const unsigned short *>(v);
#pragma unroll
            for (int e = 0; e < 8; e++)
                asm volatile("st.shared.u16 [%0], %1;" ::"r"(base + 16 * e), "h"(u[e]) : "memory");
        }
    }
    __device__ void store(int m, int n, const float (&v)[16], const Ctx &) const
    {
        if (m >= Mpad || n >= N) return;
        float *dst = part + ((size_t)blockIdx.z * Mpad + m) * N + n;
#pragma unroll
        for (int i = 0; i < 16; i += 4)
            reinterpret_cast<float4 *>(dst)[i / 4] = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
};

template <int NT, class Ld>
cudaError_t launch_gemm(const Ld &L, int mtiles, int ntiles, int k_steps, int *err, cudaStream_t st)
{
    const int bytes = tc::GemmSmem<NT, tc::gemm_stages(NT)>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(tc::gemm_kernel<NT, Ld>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    tc::gemm_kernel<NT, Ld><<<dim3(mtiles, ntiles), 128, bytes, st>>>(L, k_steps, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small kernels (CUDA cores)

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// dW[n][m] (m = tap * Ci + ci, the [Co][9][Ci] layout) and db[n] from the split partials.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int splits, int Mpad, int N, int Ci,
                                    float *__restrict__ dw, float *__restrict__ db)
{
    const int Mrows = 9 * Ci + 1;
    const long long total = (long long)Mrows * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(t / N), n = (int)(t % N);
        float acc = 0.0f;
        for (int z = 0; z < splits; z++) acc += part[((size_t)z * Mpad + m) * N + n];
        if (m < 9 * Ci) dw[(size_t)n * 9 * Ci + m] = acc;
        else db[n] = acc;
    }
}

// First layer (one input channel): out[p][c] = bf16(relu(b[c] + sum_tap bf16(w[c][tap]) bf16(s x[p + tap]))).
__global__ void __launch_bounds__(256) first_conv_fwd_kernel(const float *__restrict__ x, const float *__restrict__ w,
                                                             const float *__restrict__ b, float scale,
                                                             bf16 *__restrict__ out, int B, int H, int W, int C)
{
    const int P = B * H * W;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int xx = p % W, q = p / W, y = q % H, n = q / H;
    float in[9];
#pragma unroll
    for (int t = 0; t < 9; t++) {
        const int yy = y + t / 3 - 1, xs = xx + t % 3 - 1;
        in[t] = (yy >= 0 && yy < H && xs >= 0 && xs < W) ? bfr(scale * x[((size_t)n * H + yy) * W + xs]) : 0.0f;
    }
    for (int c0 = 0; c0 < C; c0 += 8) {
        __align__(16) bf16 o[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int c = c0 + e;
            float acc = __ldg(&b[c]);
#pragma unroll
            for (int t = 0; t < 9; t++) acc = fmaf(bfr(__ldg(&w[c * 9 + t])), in[t], acc);
            o[e] = __float2bfloat16_rn(fmaxf(acc, 0.0f));
        }
        *reinterpret_cast<uint4 *>(out + (size_t)p * C + c0) = *reinterpret_cast<const uint4 *>(o);
    }
}

// First-layer weight gradient: per block, partial sums over its pixels of
// g[p][c] * bf16(s x[p + tap]) (tap 9: 1, the bias) -> part[block][c][10].
__global__ void __launch_bounds__(960) first_conv_wgrad_kernel(const float *__restrict__ x, float scale,
                                                               const bf16 *__restrict__ g, int B, int H, int W, int C,
                                                               int pix_per_block, float *__restrict__ part)
{
    const int P = B * H * W;
    const int c = threadIdx.x / 10, tap = threadIdx.x % 10;
    float acc = 0.0f;
    if (c < C) {
        const int p_end = min(P, (blockIdx.x + 1) * pix_per_block);
        for (int p = blockIdx.x * pix_per_block; p < p_end; p++) {
            float v = 1.0f;
            if (tap < 9) {
                const int xx = p % W, q = p / W, y = q % H, n = q / H;
                const int yy = y + tap / 3 - 1, xs = xx + tap % 3 - 1;
                v = (yy >= 0 && yy < H && xs >= 0 && xs < W) ? bfr(scale * __ldg(&x[((size_t)n * H + yy) * W + xs])) : 0.0f;
            }
            acc = fmaf(__bfloat162float(g[(size_t)p * C + c]), v, acc);
        }
        part[(size_t)blockIdx.x * C * 10 + threadIdx.x] = acc;
    }
}

// Sum of `rows` partial vectors of length len.
__global__ void sum_rows_kernel(const float *__restrict__ part, int rows, int len, float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float acc = 0.0f;
    for (int r = 0; r < rows; r++) acc += part[(size_t)r * len + i];
    out[i] = acc;
}

// First-layer gradient [c][tap] (tap 9: bias) -> W [c][9] and b [c].
__global__ void first_layer_scatter_kernel(const float *__restrict__ g, int C, float *__restrict__ dw,
                                           float *__restrict__ db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C * 10) return;
    const int c = i / 10, tap = i % 10;
    if (tap < 9) dw[c * 9 + tap] = g[i];
    else db[c] = g[i];
}

// Output layer (1x1 conv to one channel, residual): y[p] = x[p] + (b + sum_c bf16(w[c]) f[p][c]) / s.
__global__ void __launch_bounds__(256) final_conv_fwd_kernel(const bf16 *__restrict__ f, const float *__restrict__ w,
                                                             const float *__restrict__ b, const float *__restrict__ x,
                                                             float inv_scale, float *__restrict__ y, int P, int C)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float acc = __ldg(&b[0]);
    for (int c0 = 0; c0 < C; c0 += 8) {
        __align__(16) bf16 v[8];
        *reinterpret_cast<uint4 *>(v) = __ldg(reinterpret_cast<const uint4 *>(f + (size_t)p * C + c0));
#pragma unroll
        for (int e = 0; e < 8; e++) acc = fmaf(bfr(__ldg(&w[c0 + e])), __bfloat162float(v[e]), acc);
    }
    y[p] = fmaf(acc, inv_scale, x[p]);
}

// Output layer backward: gz = gy / s; gf[p][c] = bf16(gz bf16(w[c]) [f > 0]); per-block partial sums of
// gz f[p][c] (weight gradient) and gz (bias gradient) -> part[block][C + 1].
__global__ void __launch_bounds__(256) final_conv_bwd_kernel(const float *__restrict__ gy, const bf16 *__restrict__ f,
                                                             const float *__restrict__ w, float inv_scale,
                                                             bf16 *__restrict__ gf, float *__restrict__ part, int P,
                                                             int C)
{
    extern __shared__ float red[];  // [C + 1]
    for (int i = threadIdx.x; i <= C; i += blockDim.x) red[i] = 0.0f;
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        const float gz = gy[p] * inv_scale;
        for (int c0 = 0; c0 < C; c0 += 8) {
            __align__(16) bf16 v[8];
            __align__(16) bf16 o[8];
            *reinterpret_cast<uint4 *>(v) = __ldg(reinterpret_cast<const uint4 *>(f + (size_t)p * C + c0));
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const float fv = __bfloat162float(v[e]);
                o[e] = __float2bfloat16_rn(fv > 0.0f ? gz * bfr(__ldg(&w[c0 + e])) : 0.0f);
                atomicAdd(&red[c0 + e], gz * fv);
            }
            *reinterpret_cast<uint4 *>(gf + (size_t)p * C + c0) = *reinterpret_cast<const uint4 *>(o);
        }
        atomicAdd(&red[C], gz);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= C; i += blockDim.x) part[(size_t)blockIdx.x * (C + 1) + i] = red[i];
}

// 2x2 max pooling, one thread per (output pixel, 8 channels).
__global__ void maxpool_fwd_kernel(const bf16 *__restrict__ in, bf16 *__restrict__ out, int B, int H, int W, int C)
{
    const int Ho = H >> 1, Wo = W >> 1, G = C >> 3;
    const long long total = (long long)B * Ho * Wo * G;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int g = (int)(t % G);
    const long long q = t / G;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), n = (int)(q / ((long long)Wo * Ho));
    __align__(16) bf16 m[8];
    for (int k = 0; k < 4; k++) {
        __align__(16) bf16 v[8];
        const size_t src = (((size_t)n * H + 2 * yo + (k >> 1)) * W + 2 * xo + (k & 1)) * C + 8 * g;
        *reinterpret_cast<uint4 *>(v) = __ldg(reinterpret_cast<const uint4 *>(in + src));
#pragma unroll
        for (int e = 0; e < 8; e++) m[e] = (k == 0 || __bfloat162float(v[e]) > __bfloat162float(m[e])) ? v[e] : m[e];
    }
    *reinterpret_cast<uint4 *>(out + (size_t)q * C + 8 * g) = *reinterpret_cast<const uint4 *>(m);
}

// Max-pool backward, added into gin: the first maximal input of each 2x2 window (in the order
// (0,0), (0,1), (1,0), (1,1)) receives the pooled gradient; sums in FP32, rounded once.
__global__ void maxpool_bwd_add_kernel(const bf16 *__restrict__ gpool, const bf16 *__restrict__ in,
                                       bf16 *__restrict__ gin, int B, int H, int W, int C)
{
    const int Ho = H >> 1, Wo = W >> 1, G = C >> 3;
    const long long total = (long long)B * Ho * Wo * G;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int g = (int)(t % G);
    const long long q = t / G;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), n = (int)(q / ((long long)Wo * Ho));
    __align__(16) bf16 v[4][8];
    size_t src[4];
    for (int k = 0; k < 4; k++) {
        src[k] = (((size_t)n * H + 2 * yo + (k >> 1)) * W + 2 * xo + (k & 1)) * C + 8 * g;
        *reinterpret_cast<uint4 *>(v[k]) = __ldg(reinterpret_cast<const uint4 *>(in + src[k]));
    }
    __align__(16) bf16 gp[8];
    *reinterpret_cast<uint4 *>(gp) = __ldg(reinterpret_cast<const uint4 *>(gpool + (size_t)q * C + 8 * g));
    int arg[8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        int a = 0;
        float best = __bfloat162float(v[0][e]);
        for (int k = 1; k < 4; k++)
            if (__bfloat162float(v[k][e]) > best) { best = __bfloat162float(v[k][e]); a = k; }
        arg[e] = a;
    }
    for (int k = 0; k < 4; k++) {
        __align__(16) bf16 o[8];
        *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(gin + src[k]);
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (arg[e] == k) o[e] = __float2bfloat16_rn(__bfloat162float(o[e]) + __bfloat162float(gp[e]));
        *reinterpret_cast<uint4 *>(gin + src[k]) = *reinterpret_cast<const uint4 *>(o);
    }
}

// Backward of the nearest 2x upsampling: gT[q][c] = sum of the four children's gradients (FP32, rounded once).
__global__ void upsample_bwd_kernel(const bf16 *__restrict__ gup, bf16 *__restrict__ gT, int B, int H, int W, int C)
{
    const int Ho = H >> 1, Wo = W >> 1, G = C >> 3;
    const long long total = (long long)B * Ho * Wo * G;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int g = (int)(t % G);
    const long long q = t / G;
    const int xo = (int)(q % Wo), yo = (int)((q / Wo) % Ho), n = (int)(q / ((long long)Wo * Ho));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 4; k++) {
        __align__(16) bf16 v[8];
        const size_t src = (((size_t)n * H + 2 * yo + (k >> 1)) * W + 2 * xo + (k & 1)) * C + 8 * g;
        *reinterpret_cast<uint4 *>(v) = __ldg(reinterpret_cast<const uint4 *>(gup + src));
#pragma unroll
        for (int e = 0; e < 8; e++) acc[e] += __bfloat162float(v[e]);
    }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int e = 0; e < 8; e++) o[e] = __float2bfloat16_rn(acc[e]);
    *reinterpret_cast<uint4 *>(gT + (size_t)q * C + 8 * g) = *reinterpret_cast<const uint4 *>(o);
}

// BF16 copies of a 3x3 layer's FP32 weights [Co][9][Ci]: as is (forward) and as the flipped transpose
// wt[ci][8 - tap][co] (input gradient).
__global__ void prep_weights_kernel(const float *__restrict__ w, bf16 *__restrict__ wf, bf16 *__restrict__ wt, int Co,
                                    int Ci)
{
    const int total = Co * 9 * Ci;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int ci = i % Ci, tap = (i / Ci) % 9, co = i / (9 * Ci);
    const bf16 v = __float2bfloat16_rn(w[i]);
    wf[i] = v;
    wt[((size_t)ci * 9 + (8 - tap)) * Co + co] = v;
}

// Adam (Kingma & Ba) on the FP32 master parameters, with decoupled weight decay.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2, float wd)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p[i]);
    }
}

// ---------------------------------------------------------------- convolution launchers

// The driver's tensor-map encoder, through the runtime (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// Tensor maps of the TMA convolution (tc_conv_tma.cuh), when it takes this layer: a single full-resolution
// input of a multiple of 32 channels, a multiple of 32 output channels, 128-pixel tiles that are one
// part of a row (W a multiple of 128) or whole rows of one image (128 a multiple of W, H W of 128), and
// 16-byte aligned tensors.  A: the input [B][H][W][Ci], box 32 channels x the tile's pixels; B: the
// weights [N][9 Ci], box 32 K-elements x nt channels; both with the 64-byte swizzle, zeros outside.
bool conv_tma_maps(const ConvIn &in, const bf16 *w, int B, int H, int W, int N, int nt, CUtensorMap &ma,
                   CUtensorMap &mb)
{
    if (in.c2 != 0 || in.up1 || in.c1 % 32 != 0 || N % 32 != 0) return false;
    if (!((W % 128 == 0) || (W < 128 && 128 % W == 0 && (H * W) % 128 == 0))) return false;
    if (((uintptr_t)in.t1 & 15) || ((uintptr_t)w & 15)) return false;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t Ci = (cuuint64_t)in.c1, Kt = 9 * Ci;
    const cuuint64_t dimA[4] = {Ci, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strA[3] = {Ci * 2, (cuuint64_t)W * Ci * 2, (cuuint64_t)H * W * Ci * 2};
    const cuuint32_t boxA[4] = {32, (cuuint32_t)std::min(W, 128), (cuuint32_t)(W >= 128 ? 1 : 128 / W), 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(in.t1), dimA, strA, boxA, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t dimB[2] = {Kt, (cuuint64_t)N};
    const cuuint64_t strB[1] = {Kt * 2};
    const cuuint32_t boxB[2] = {32, (cuuint32_t)nt};
    return enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(w), dimB, strB, boxB, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, int ST, class L>
cudaError_t launch_conv_tma_st(const CUtensorMap &ma, const CUtensorMap &mb, const L &epi, tc::ConvTmaGeo geo,
                               int mtiles, int ntiles, int *err, cudaStream_t st)
{
    const int bytes = tc::ConvTmaSmem<NT, ST>::kBytes;
    cudaError_t e =
        cudaFuncSetAttribute(tc::conv_tma_kernel<NT, ST, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    tc::conv_tma_kernel<NT, ST, L><<<dim3(mtiles, ntiles), 128, bytes, st>>>(ma, mb, epi, geo, err);
    return cudaGetLastError();
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

// Two stages when the grid covers the SMs twice or more (several CTAs per SM overlap one another's
// copies), four when it does not.
template <int NT, class L>
cudaError_t launch_conv_tma(const CUtensorMap &ma, const CUtensorMap &mb, const L &epi, tc::ConvTmaGeo geo, int mtiles,
                            int ntiles, int *err, cudaStream_t st)
{
    if ((long)mtiles * ntiles >= 2L * sm_count()) return launch_conv_tma_st<NT, 2>(ma, mb, epi, geo, mtiles, ntiles, err, st);
    return launch_conv_tma_st<NT, 4>(ma, mb, epi, geo, mtiles, ntiles, err, st);
}

template <int EPI>
cudaError_t conv3x3_tc(const ConvIn &in, const bf16 *w, const float *bias, bf16 *out, const ConvIn &mask, bf16 *out2,
                       int B, int H, int W, int N, int *err, cudaStream_t st)
{
    const int Ci = in.c1 + in.c2, P = B * H * W;
    const int mt = (P + 127) / 128, ks = (9 * Ci + tc::kStageK - 1) / tc::kStageK;
    // the largest power-of-two tile in [32, 256] that divides N
    int nt = 256;
    while (nt > 32 && N % nt != 0) nt >>= 1;
    const int ntiles = (N + nt - 1) / nt;
    CUtensorMap ma, mb;
    if (conv_tma_maps(in, w, B, H, W, N, nt, ma, mb)) {
        const tc::ConvTmaGeo geo{H, W, Ci, 9 * Ci / 32};
        switch (nt) {
        case 256: return launch_conv_tma<256>(ma, mb, ConvGemm<256, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, geo, mt, ntiles, err, st);
        case 128: return launch_conv_tma<128>(ma, mb, ConvGemm<128, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, geo, mt, ntiles, err, st);
        case 64: return launch_conv_tma<64>(ma, mb, ConvGemm<64, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, geo, mt, ntiles, err, st);
        default: return launch_conv_tma<32>(ma, mb, ConvGemm<32, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, geo, mt, ntiles, err, st);
        }
    }
    switch (nt) {
    case 256: return launch_gemm<256>(ConvGemm<256, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, mt, ntiles, ks, err, st);
    case 128: return launch_gemm<128>(ConvGemm<128, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, mt, ntiles, ks, err, st);
    case 64: return launch_gemm<64>(ConvGemm<64, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, mt, ntiles, ks, err, st);
    default: return launch_gemm<32>(ConvGemm<32, EPI>{in, w, bias, out, mask, out2, B, H, W, Ci, N}, mt, ntiles, ks, err, st);
    }
}

struct WgradPlan {
    int Mpad, mtiles, splits, steps_per_split, k_steps_total, nt, ntiles;
    size_t part_floats;
};

WgradPlan wgrad_plan(int B, int H, int W, int Ci, int N)
{
    WgradPlan w;
    const int Mrows = 9 * Ci + 1;
    w.mtiles = (Mrows + 127) / 128;
    w.Mpad = w.mtiles * 128;
    w.nt = 256;
    while (w.nt > 32 && N % w.nt != 0) w.nt >>= 1;
    w.ntiles = (N + w.nt - 1) / w.nt;
    const long long P = (long long)B * H * W;
    w.k_steps_total = (int)((P + tc::kStageK - 1) / tc::kStageK);
    // about four CTAs per SM in total, at least 8 K-slices each
    int splits = (int)std::max(1LL, std::min<long long>(w.k_steps_total / 8, 608 / (w.mtiles * w.ntiles)));
    splits = std::min(splits, 256);
    w.steps_per_split = (w.k_steps_total + splits - 1) / splits;
    w.splits = (w.k_steps_total + w.steps_per_split - 1) / w.steps_per_split;
    w.part_floats = (size_t)w.splits * w.Mpad * N;
    return w;
}

cudaError_t conv3x3_wgrad_tc(const ConvIn &in, const bf16 *gout, float *dw, float *db, float *part, int B, int H, int W,
                             int N, int *err, cudaStream_t st)
{
    const int Ci = in.c1 + in.c2;
    const WgradPlan pl = wgrad_plan(B, H, W, Ci, N);
    cudaError_t e;
    const dim3 grid(pl.mtiles, pl.ntiles, pl.splits);
#define CT_WG(NTV)                                                                                                     \
    {                                                                                                                  \
        using L = WgradGemm<NTV>;                                                                                      \
        const int bytes = tc::GemmSmem<NTV, tc::gemm_stages(NTV)>::kBytes;                                             \
        e = cudaFuncSetAttribute(tc::gemm_kernel<NTV, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);         \
        if (e != cudaSuccess) return e;                                                                                \
        tc::gemm_kernel<NTV, L><<<grid, 128, bytes, st>>>(                                                             \
            L{in, gout, part, B, H, W, Ci, N, 9 * Ci + 1, pl.Mpad, pl.steps_per_split, pl.k_steps_total},              \
            pl.steps_per_split, err);                                                                                  \
    }
    switch (pl.nt) {
    case 256: CT_WG(256) break;
    case 128: CT_WG(128) break;
    case 64: CT_WG(64) break;
    default: CT_WG(32) break;
    }
#undef CT_WG
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long total = (long long)(9 * Ci + 1) * N;
    wgrad_reduce_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, st>>>(part, pl.splits,
                                                                                                pl.Mpad, N, Ci, dw, db);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ct

using namespace ct;

extern "C" ct_status ct_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int *err, void *stream)
{
    if (!A || !B || !C || !err) { set_error("ct_gemm_bf16: null argument"); return CT_EINVAL; }
    if (M < 1 || N < 1 || K < 8 || K % 8 != 0) {
        set_error("ct_gemm_bf16: need M, N >= 1 and K a positive multiple of 8 (M=%d N=%d K=%d)", M, N, K);
        return CT_EINVAL;
    }
    if (((uintptr_t)A | (uintptr_t)B) & 15) { set_error("ct_gemm_bf16: A and B must be 16-byte aligned"); return CT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int mt = (M + 127) / 128, ks = (K + tc::kStageK - 1) / tc::kStageK;
    const bf16 *a = (const bf16 *)A, *b = (const bf16 *)B;
    cudaError_t e;
    if (N <= 32) e = launch_gemm<32>(PlainGemm<32>{a, b, C, M, N, K}, mt, 1, ks, err, st);
    else if (N <= 64) e = launch_gemm<64>(PlainGemm<64>{a, b, C, M, N, K}, mt, 1, ks, err, st);
    else if (N <= 128) e = launch_gemm<128>(PlainGemm<128>{a, b, C, M, N, K}, mt, 1, ks, err, st);
    else e = launch_gemm<256>(PlainGemm<256>{a, b, C, M, N, K}, mt, (N + 255) / 256, ks, err, st);
    CT_CUDA_TRY(e, "ct_gemm_bf16 launch");
    return CT_OK;
}

// ---------------------------------------------------------------- the network object

struct ct_unet {
    ct_unet_desc d{};
    int L = 0, C0 = 0, H = 0, W = 0, Bmax = 0;
    struct Conv {
        int c1, up1, c2, co;   // input: tensor 1 (c1 ch, up1: half resolution), tensor 2 (c2 ch); output co ch
        size_t w_off, b_off;   // offsets of W [co][9][c1+c2] and b [co] in the parameter vector
        bf16 *wf = nullptr, *wt = nullptr;
    };
    std::vector<Conv> conv;  // encoder a/b per level 0..L-1, then decoder a/b for levels L-2..0
    size_t out_w_off = 0, out_b_off = 0, nparams = 0;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    bf16 *wbf = nullptr;
    std::vector<bf16 *> a, s, p, e, f, gs;
    bf16 *G[3] = {nullptr, nullptr, nullptr};
    float *x = nullptr, *part = nullptr;
    size_t part_floats = 0;
    int *err = nullptr;
    int last_B = 0, step = 0;
    std::vector<void *> allocs;
    int ch(int l) const { return C0 << l; }
    int enc(int l, int b) const { return 2 * l + b; }
    int dec(int l, int b) const { return 2 * L + 2 * (L - 2 - l) + b; }
};

namespace {

struct Rng {  // SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) with Box-Muller normals
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

cudaError_t prep_all(ct_unet *n, cudaStream_t st)
{
    for (size_t i = 1; i < n->conv.size(); i++) {
        const auto &c = n->conv[i];
        const int ci = c.c1 + c.c2, tot = c.co * 9 * ci;
        prep_weights_kernel<<<(tot + 255) / 256, 256, 0, st>>>(n->params + c.w_off, c.wf, c.wt, c.co, ci);
    }
    return cudaGetLastError();
}

template <class T>
T *take(ct_unet *n, size_t count, cudaError_t &e)
{
    if (e != cudaSuccess) return nullptr;
    void *ptr = nullptr;
    e = cudaMalloc(&ptr, std::max<size_t>(count * sizeof(T), 16));
    if (e == cudaSuccess) n->allocs.push_back(ptr);
    return (T *)ptr;
}

void free_unet(ct_unet *n)
{
    if (!n) return;
    for (void *p : n->allocs) cudaFree(p);
    delete n;
}

ConvIn single(const bf16 *t, int c) { return ConvIn{t, c, 0, nullptr, 0}; }

}  // namespace

extern "C" ct_status ct_unet_create(const ct_unet_desc *d, ct_unet **out)
{
    if (!d || !out) { set_error("ct_unet_create: null argument"); return CT_EINVAL; }
    *out = nullptr;
    const int L = d->levels, C0 = d->base_channels;
    if (L < 2 || L > 5 || C0 < 16 || C0 % 16 != 0 || C0 > 96) {
        set_error("ct_unet_create: need 2 <= levels <= 5 and base_channels a multiple of 16 in [16, 96]");
        return CT_EINVAL;
    }
    if (d->height < (1 << (L - 1)) || d->width < (1 << (L - 1)) || d->height % (1 << (L - 1)) ||
        d->width % (1 << (L - 1)) || d->max_batch < 1 || (long long)d->max_batch * d->height * d->width > (1LL << 30) ||
        !(d->in_scale > 0.0f)) {
        set_error("ct_unet_create: height and width must be multiples of 2^(levels-1); max_batch >= 1; in_scale > 0");
        return CT_EINVAL;
    }
    ct_unet *n = new ct_unet();
    n->d = *d;
    n->L = L;
    n->C0 = C0;
    n->H = d->height;
    n->W = d->width;
    n->Bmax = d->max_batch;
    // layers and parameter offsets
    size_t off = 0;
    auto add = [&](int c1, int up1, int c2, int co) {
        ct_unet::Conv c;
        c.c1 = c1; c.up1 = up1; c.c2 = c2; c.co = co;
        c.w_off = off;
        off += (size_t)co * 9 * (c1 + c2);
        c.b_off = off;
        off += co;
        n->conv.push_back(c);
    };
    for (int l = 0; l < L; l++) {
        add(l == 0 ? 1 : n->ch(l - 1), 0, 0, n->ch(l));
        add(n->ch(l), 0, 0, n->ch(l));
    }
    for (int l = L - 2; l >= 0; l--) {
        add(n->ch(l + 1), 1, n->ch(l), n->ch(l));
        add(n->ch(l), 0, 0, n->ch(l));
    }
    n->out_w_off = off;
    off += C0;
    n->out_b_off = off;
    off += 1;
    n->nparams = off;
    cudaError_t e = cudaSuccess;
    n->params = take<float>(n, off, e);
    n->grads = take<float>(n, off, e);
    n->adam_m = take<float>(n, off, e);
    n->adam_v = take<float>(n, off, e);
    size_t nbf = 0;
    for (size_t i = 1; i < n->conv.size(); i++) nbf += 2 * (size_t)n->conv[i].co * 9 * (n->conv[i].c1 + n->conv[i].c2);
    n->wbf = take<bf16>(n, nbf, e);
    if (e == cudaSuccess) {
        size_t o = 0;
        for (size_t i = 1; i < n->conv.size(); i++) {
            const size_t sz = (size_t)n->conv[i].co * 9 * (n->conv[i].c1 + n->conv[i].c2);
            n->conv[i].wf = n->wbf + o;
            n->conv[i].wt = n->wbf + o + sz;
            o += 2 * sz;
        }
    }
    const size_t B = d->max_batch;
    n->a.resize(L); n->s.resize(L); n->p.resize(L); n->e.resize(L); n->f.resize(L); n->gs.resize(L);
    for (int l = 0; l < L; l++) {
        const size_t px = B * (size_t)(n->H >> l) * (n->W >> l);
        n->a[l] = take<bf16>(n, px * n->ch(l), e);
        n->s[l] = take<bf16>(n, px * n->ch(l), e);
        if (l + 1 < L) {
            n->p[l] = take<bf16>(n, px / 4 * n->ch(l), e);
            n->e[l] = take<bf16>(n, px * n->ch(l), e);
            n->f[l] = take<bf16>(n, px * n->ch(l), e);
            n->gs[l] = take<bf16>(n, px * n->ch(l), e);
        }
    }
    const size_t gsz = 2 * B * n->H * n->W * (size_t)C0;
    for (int i = 0; i < 3; i++) n->G[i] = take<bf16>(n, gsz, e);
    n->x = take<float>(n, B * n->H * n->W, e);
    // wgrad partials: the largest split plan over the layers
    size_t pf = 0;
    for (size_t i = 1; i < n->conv.size(); i++) {
        const auto &c = n->conv[i];
        // layer i runs at the resolution of its output level
        int lev = 0;
        if (i < (size_t)2 * L) lev = (int)i / 2;
        else lev = L - 2 - (int)(i - 2 * L) / 2;
        const WgradPlan pl = wgrad_plan(d->max_batch, n->H >> lev, n->W >> lev, c.c1 + c.c2, c.co);
        pf = std::max(pf, pl.part_floats);
    }
    const int P0 = d->max_batch * n->H * n->W;
    pf = std::max(pf, (size_t)((P0 + 255) / 256) * (size_t)(C0 * 10 + C0 + 1));
    n->part_floats = pf;
    n->part = take<float>(n, pf, e);
    n->err = take<int>(n, 1, e);
    if (e != cudaSuccess) {
        ct_status st = cuda_fail(e, "ct_unet_create");
        free_unet(n);
        return st;
    }
    // He-normal weights, zero biases, a small output layer (the network starts near the identity)
    std::vector<float> h(off, 0.0f);
    Rng rng{d->seed ^ 0x5DEECE66Dull};
    for (size_t i = 0; i < n->conv.size(); i++) {
        const auto &c = n->conv[i];
        const int ci = c.c1 + c.c2;
        const double sd = std::sqrt(2.0 / (9.0 * ci));
        for (size_t k = 0; k < (size_t)c.co * 9 * ci; k++) h[c.w_off + k] = (float)(sd * rng.normal());
    }
    for (int k = 0; k < C0; k++) h[n->out_w_off + k] = (float)(1e-2 * std::sqrt(1.0 / C0) * rng.normal());
    e = cudaMemcpy(n->params, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(n->grads, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int));
    if (e == cudaSuccess) e = prep_all(n, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ct_status st = cuda_fail(e, "ct_unet_create (init)");
        free_unet(n);
        return st;
    }
    *out = n;
    return CT_OK;
}

extern "C" void ct_unet_destroy(ct_unet *n) { free_unet(n); }

extern "C" long long ct_unet_num_params(const ct_unet *n) { return n ? (long long)n->nparams : -1; }

extern "C" ct_status ct_unet_get_params(const ct_unet *n, float *host, int which)
{
    if (!n || !host || which < 0 || which > 1) { set_error("ct_unet_get_params: bad argument"); return CT_EINVAL; }
    CT_CUDA_TRY(cudaMemcpy(host, which == 0 ? n->params : n->grads, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost),
                "ct_unet_get_params");
    return CT_OK;
}

extern "C" ct_status ct_unet_set_params(ct_unet *n, const float *host)
{
    if (!n || !host) { set_error("ct_unet_set_params: null argument"); return CT_EINVAL; }
    CT_CUDA_TRY(cudaMemcpy(n->params, host, sizeof(float) * n->nparams, cudaMemcpyHostToDevice), "ct_unet_set_params");
    CT_CUDA_TRY(prep_all(n, nullptr), "ct_unet_set_params (bf16 copies)");
    CT_CUDA_TRY(cudaDeviceSynchronize(), "ct_unet_set_params");
    return CT_OK;
}

extern "C" ct_status ct_unet_forward(ct_unet *n, const float *x, float *y, int B, void *stream)
{
    if (!n || !x || !y) { set_error("ct_unet_forward: null argument"); return CT_EINVAL; }
    if (B < 1 || B > n->Bmax) { set_error("ct_unet_forward: batch %d outside [1, %d]", B, n->Bmax); return CT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int L = n->L, H = n->H, W = n->W, C0 = n->C0;
    const int P0 = B * H * W;
    CT_CUDA_TRY(cudaMemcpyAsync(n->x, x, sizeof(float) * P0, cudaMemcpyDeviceToDevice, st), "ct_unet_forward input");
    const ConvIn none{nullptr, 0, 0, nullptr, 0};
    {
        const auto &c = n->conv[n->enc(0, 0)];
        first_conv_fwd_kernel<<<(P0 + 255) / 256, 256, 0, st>>>(n->x, n->params + c.w_off, n->params + c.b_off,
                                                               n->d.in_scale, n->a[0], B, H, W, C0);
        CT_CUDA_TRY(cudaGetLastError(), "first layer");
    }
    for (int l = 0; l < L; l++) {
        const int Hl = H >> l, Wl = W >> l;
        if (l > 0) {
            const int cp = n->ch(l - 1);
            const long long tot = (long long)B * Hl * Wl * (cp / 8);
            maxpool_fwd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n->s[l - 1], n->p[l - 1], B, 2 * Hl,
                                                                              2 * Wl, cp);
            const auto &c = n->conv[n->enc(l, 0)];
            CT_CUDA_TRY(conv3x3_tc<EPI_RELU>(single(n->p[l - 1], cp), c.wf, n->params + c.b_off, n->a[l], none,
                                             nullptr, B, Hl, Wl, c.co, n->err, st), "encoder conv a");
        }
        const auto &c = n->conv[n->enc(l, 1)];
        CT_CUDA_TRY(conv3x3_tc<EPI_RELU>(single(n->a[l], n->ch(l)), c.wf, n->params + c.b_off, n->s[l], none,
                                         nullptr, B, Hl, Wl, c.co, n->err, st), "encoder conv b");
    }
    const bf16 *T = n->s[L - 1];
    for (int l = L - 2; l >= 0; l--) {
        const int Hl = H >> l, Wl = W >> l;
        const auto &ca = n->conv[n->dec(l, 0)];
        CT_CUDA_TRY(conv3x3_tc<EPI_RELU>(ConvIn{T, n->ch(l + 1), 1, n->s[l], n->ch(l)}, ca.wf, n->params + ca.b_off,
                                         n->e[l], none, nullptr, B, Hl, Wl, ca.co, n->err, st), "decoder conv a");
        const auto &cb = n->conv[n->dec(l, 1)];
        CT_CUDA_TRY(conv3x3_tc<EPI_RELU>(single(n->e[l], n->ch(l)), cb.wf, n->params + cb.b_off, n->f[l], none,
                                         nullptr, B, Hl, Wl, cb.co, n->err, st), "decoder conv b");
        T = n->f[l];
    }
    final_conv_fwd_kernel<<<(P0 + 255) / 256, 256, 0, st>>>(T, n->params + n->out_w_off, n->params + n->out_b_off,
                                                            n->x, 1.0f / n->d.in_scale, y, P0, C0);
    CT_CUDA_TRY(cudaGetLastError(), "output layer");
    n->last_B = B;
    return CT_OK;
}

extern "C" ct_status ct_unet_backward(ct_unet *n, const float *gy, int B, void *stream)
{
    if (!n || !gy) { set_error("ct_unet_backward: null argument"); return CT_EINVAL; }
    if (B != n->last_B) { set_error("ct_unet_backward: batch %d differs from the last forward's %d", B, n->last_B); return CT_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int L = n->L, H = n->H, W = n->W, C0 = n->C0;
    const int P0 = B * H * W;
    const ConvIn none{nullptr, 0, 0, nullptr, 0};
    float *gr = n->grads;
    // output layer
    {
        const int blocks = (P0 + 255) / 256;
        final_conv_bwd_kernel<<<blocks, 256, sizeof(float) * (C0 + 1), st>>>(gy, n->f[0],
                                                                            n->params + n->out_w_off,
                                                                            1.0f / n->d.in_scale, n->G[0], n->part, P0, C0);
        sum_rows_kernel<<<(C0 + 1 + 255) / 256, 256, 0, st>>>(n->part, blocks, C0 + 1, gr + n->out_w_off);
        CT_CUDA_TRY(cudaGetLastError(), "output layer backward");
    }
    int cur = 0;  // index of the buffer holding the gradient being propagated
    for (int l = 0; l <= L - 2; l++) {
        const int Hl = H >> l, Wl = W >> l;
        const int X = cur, Y = cur ^ 1;
        const auto &cb = n->conv[n->dec(l, 1)];
        CT_CUDA_TRY(conv3x3_wgrad_tc(single(n->e[l], n->ch(l)), n->G[X], gr + cb.w_off, gr + cb.b_off, n->part, B, Hl,
                                     Wl, cb.co, n->err, st), "decoder b wgrad");
        CT_CUDA_TRY(conv3x3_tc<EPI_DGRAD>(single(n->G[X], cb.co), cb.wt, nullptr, n->G[Y], single(n->e[l], n->ch(l)),
                                          nullptr, B, Hl, Wl, n->ch(l), n->err, st), "decoder b dgrad");
        const auto &ca = n->conv[n->dec(l, 0)];
        const bf16 *T = (l + 1 == L - 1) ? n->s[L - 1] : n->f[l + 1];
        const ConvIn cat{T, n->ch(l + 1), 1, n->s[l], n->ch(l)};
        CT_CUDA_TRY(conv3x3_wgrad_tc(cat, n->G[Y], gr + ca.w_off, gr + ca.b_off, n->part, B, Hl, Wl, ca.co, n->err, st),
                    "decoder a wgrad");
        CT_CUDA_TRY(conv3x3_tc<EPI_DGRAD>(single(n->G[Y], ca.co), ca.wt, nullptr, n->G[X], cat, n->gs[l], B, Hl, Wl,
                                          n->ch(l + 1) + n->ch(l), n->err, st), "decoder a dgrad");
        const long long tot = (long long)B * (Hl / 2) * (Wl / 2) * (n->ch(l + 1) / 8);
        upsample_bwd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n->G[X], n->G[Y], B, Hl, Wl, n->ch(l + 1));
        CT_CUDA_TRY(cudaGetLastError(), "upsample backward");
        cur = Y;
    }
    for (int l = L - 1; l >= 0; l--) {
        const int Hl = H >> l, Wl = W >> l;
        bf16 *gsl = (l == L - 1) ? n->G[cur] : n->gs[l];
        bf16 *ga = n->G[2];
        bf16 *gp = n->G[(l == L - 1) ? (cur ^ 1) : 0];
        const auto &cb = n->conv[n->enc(l, 1)];
        CT_CUDA_TRY(conv3x3_wgrad_tc(single(n->a[l], n->ch(l)), gsl, gr + cb.w_off, gr + cb.b_off, n->part, B, Hl, Wl,
                                     cb.co, n->err, st), "encoder b wgrad");
        CT_CUDA_TRY(conv3x3_tc<EPI_DGRAD>(single(gsl, cb.co), cb.wt, nullptr, ga, single(n->a[l], n->ch(l)), nullptr,
                                          B, Hl, Wl, n->ch(l), n->err, st), "encoder b dgrad");
        const auto &ca = n->conv[n->enc(l, 0)];
        if (l == 0) {
            const int ppb = 1024, blocks = (P0 + ppb - 1) / ppb;
            first_conv_wgrad_kernel<<<blocks, C0 * 10, 0, st>>>(n->x, n->d.in_scale, ga, B, H, W, C0, ppb, n->part);
            // part[block][c * 10 + tap] -> W (c * 9 + tap) and b (9 C0 + c), which are contiguous
            CT_CUDA_TRY(cudaGetLastError(), "first layer wgrad");
            sum_rows_kernel<<<(C0 * 10 + 255) / 256, 256, 0, st>>>(n->part, blocks, C0 * 10, n->part + (size_t)blocks * C0 * 10);
            first_layer_scatter_kernel<<<(C0 * 10 + 255) / 256, 256, 0, st>>>(n->part + (size_t)blocks * C0 * 10, C0,
                                                                             gr + ca.w_off, gr + ca.b_off);
            CT_CUDA_TRY(cudaGetLastError(), "first layer wgrad reduce");
        } else {
            const int cp = n->ch(l - 1);
            CT_CUDA_TRY(conv3x3_wgrad_tc(single(n->p[l - 1], cp), ga, gr + ca.w_off, gr + ca.b_off, n->part, B, Hl, Wl,
                                         ca.co, n->err, st), "encoder a wgrad");
            CT_CUDA_TRY(conv3x3_tc<EPI_DGRAD>(single(ga, ca.co), ca.wt, nullptr, gp, single(n->p[l - 1], cp), nullptr,
                                              B, Hl, Wl, cp, n->err, st), "encoder a dgrad");
            const long long tot = (long long)B * Hl * Wl * (cp / 8);
            maxpool_bwd_add_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(gp, n->s[l - 1], n->gs[l - 1], B,
                                                                                  2 * Hl, 2 * Wl, cp);
            CT_CUDA_TRY(cudaGetLastError(), "max-pool backward");
        }
    }
    (void)none;
    return CT_OK;
}

extern "C" ct_status ct_unet_adam(ct_unet *n, float lr, float beta1, float beta2, float eps, float weight_decay,
                                  void *stream)
{
    if (!n) { set_error("ct_unet_adam: null network"); return CT_EINVAL; }
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) ||
        !(weight_decay >= 0.0f)) {
        set_error("ct_unet_adam: bad hyper-parameters");
        return CT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    n->step++;
    const float bc1 = (float)(1.0 - std::pow((double)beta1, n->step));
    const float bc2 = (float)(1.0 - std::pow((double)beta2, n->step));
    adam_kernel<<<(unsigned)std::min<long long>(((long long)n->nparams + 255) / 256, 2048), 256, 0, st>>>(
        n->params, n->grads, n->adam_m, n->adam_v, (long long)n->nparams, lr, beta1, beta2, eps, bc1, bc2, weight_decay);
    CT_CUDA_TRY(cudaGetLastError(), "adam");
    CT_CUDA_TRY(prep_all(n, st), "bf16 weight copies");
    return CT_OK;
}

extern "C" ct_status ct_unet_status(ct_unet *n)
{
    if (!n) { set_error("ct_unet_status: null network"); return CT_EINVAL; }
    int h = 0;
    CT_CUDA_TRY(cudaMemcpy(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost), "ct_unet_status");
    if (h) {
        cudaMemset(n->err, 0, sizeof(int));
        set_error("a bounded tensor-core pipeline wait gave up");
        return CT_ETIMEOUT;
    }
    return CT_OK;
}

// ---------------------------------------------------------------- single-layer entries (for testing)

namespace {
ct_status check_conv_args(int c1, int up1, int c2, int co, int B, int H, int W)
{
    if (c1 < 8 || c1 % 16 != 0 || (c2 != 0 && (c2 < 8 || c2 % 8 != 0)) || co < 16 || co % 16 != 0 || B < 1 || H < 1 ||
        W < 1 || (up1 && (H % 2 || W % 2)) || (long long)B * H * W > (1LL << 30)) {
        set_error("conv3x3: need c1 a multiple of 16, c2 0 or a multiple of 8, co a multiple of 16, even H and W "
                  "with an upsampled input");
        return CT_EINVAL;
    }
    return CT_OK;
}
bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }
}  // namespace

extern "C" ct_status ct_conv3x3_bf16(const void *in1, int c1, int up1, const void *in2, int c2, const void *w,
                                     const float *bias, void *out, int B, int H, int W, int co, int *err, void *stream)
{
    if (!in1 || !w || !bias || !out || !err || (c2 && !in2)) { set_error("ct_conv3x3_bf16: null argument"); return CT_EINVAL; }
    ct_status s = check_conv_args(c1, up1, c2, co, B, H, W);
    if (s != CT_OK) return s;
    if (!aligned16(in1) || (in2 && !aligned16(in2)) || !aligned16(w) || !aligned16(out)) {
        set_error("ct_conv3x3_bf16: tensors must be 16-byte aligned");
        return CT_EINVAL;
    }
    const ConvIn in{(const bf16 *)in1, c1, up1 ? 1 : 0, (const bf16 *)in2, c2};
    CT_CUDA_TRY(conv3x3_tc<EPI_RELU>(in, (const bf16 *)w, bias, (bf16 *)out, ConvIn{nullptr, 0, 0, nullptr, 0},
                                     nullptr, B, H, W, co, err, (cudaStream_t)stream), "ct_conv3x3_bf16");
    return CT_OK;
}

extern "C" ct_status ct_conv3x3_bf16_dgrad(const void *gout, int co, const void *wt, const void *m1, int c1, int up1,
                                           const void *m2, int c2, void *g1, void *g2, int B, int H, int W, int *err,
                                           void *stream)
{
    if (!gout || !wt || !m1 || !g1 || !err || (c2 && (!m2 || !g2))) {
        set_error("ct_conv3x3_bf16_dgrad: null argument");
        return CT_EINVAL;
    }
    ct_status s = check_conv_args(c1, up1, c2, co, B, H, W);
    if (s != CT_OK) return s;
    if ((c1 + c2) % 16 != 0) { set_error("ct_conv3x3_bf16_dgrad: c1 + c2 must be a multiple of 16"); return CT_EINVAL; }
    const ConvIn mask{(const bf16 *)m1, c1, up1 ? 1 : 0, (const bf16 *)m2, c2};
    CT_CUDA_TRY(conv3x3_tc<EPI_DGRAD>(ConvIn{(const bf16 *)gout, co, 0, nullptr, 0}, (const bf16 *)wt, nullptr,
                                      (bf16 *)g1, mask, (bf16 *)g2, B, H, W, c1 + c2, err, (cudaStream_t)stream),
                "ct_conv3x3_bf16_dgrad");
    return CT_OK;
}

extern "C" long long ct_conv3x3_wgrad_workspace(int B, int H, int W, int ci, int co)
{
    if (B < 1 || H < 1 || W < 1 || ci < 1 || co < 1) return -1;
    return (long long)wgrad_plan(B, H, W, ci, co).part_floats;
}

extern "C" ct_status ct_conv3x3_bf16_wgrad(const void *in1, int c1, int up1, const void *in2, int c2, const void *gout,
                                           int co, float *dw, float *db, float *work, long long work_floats, int B,
                                           int H, int W, int *err, void *stream)
{
    if (!in1 || !gout || !dw || !db || !work || !err || (c2 && !in2)) {
        set_error("ct_conv3x3_bf16_wgrad: null argument");
        return CT_EINVAL;
    }
    ct_status s = check_conv_args(c1, up1, c2, co, B, H, W);
    if (s != CT_OK) return s;
    if (work_floats < ct_conv3x3_wgrad_workspace(B, H, W, c1 + c2, co)) {
        set_error("ct_conv3x3_bf16_wgrad: workspace too small (need %lld floats)",
                  ct_conv3x3_wgrad_workspace(B, H, W, c1 + c2, co));
        return CT_EINVAL;
    }
    const ConvIn in{(const bf16 *)in1, c1, up1 ? 1 : 0, (const bf16 *)in2, c2};
    CT_CUDA_TRY(conv3x3_wgrad_tc(in, (const bf16 *)gout, dw, db, work, B, H, W, co, err, (cudaStream_t)stream),
                "ct_conv3x3_bf16_wgrad");
    return CT_OK;
}
