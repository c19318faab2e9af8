// Implicit-GEMM 3x3 convolution on sm_103a with TMA operand staging (one CTA: a 128 x NT output tile).
//
// Rows are 128 consecutive output pixels of one image, K = (tap, input channel) with the channel
// fastest, in planes of 32 channels: the A plane of K-offset k (tap k / Ci, channels k mod Ci .. +31) is
// the input tensor [B][H][W][Ci] (BF16 NHWC) shifted by the tap, read by ONE tiled TMA copy of a box of
// 32 channels x the tile's pixels (128 pixels of one row, or 128 / W whole rows); coordinates outside the
// image read as zeros, which is the convolution's zero padding.  The B plane is the box of 32 K-elements
// x NT output channels of the weights [N][9 Ci].  Both land 64-byte swizzled (planes of rows 64 bytes
// apart) and the MMAs read them through swizzled descriptors.
//
// Roles: thread 0 is the producer (waits until the MMAs of the stage a buffer last held are complete,
// then issues the stage's copies against its mbarrier); thread 32 issues the MMAs (waits for the stage's
// copies, issues 128 x NT x 16 tcgen05.mma per 16 K-elements into one tensor-memory accumulator, commits
// them to the buffer's "empty" barrier).  ST stages are in flight: two when the grid fills the SMs several
// times over (more CTAs per SM hide the copies' latency), four for the deep layers' small grids.  After the last stage one
// more commit marks the accumulator complete; all four warps then read it (warp w: rows 32w .. 32w+31)
// and hand 16 columns at a time to the epilogue object's store().
//
// Every wait is bounded: a wait that gives up sets the error flag and the CTA's abort flag, the producer
// stops issuing, and the CTA frees its tensor memory only after the final commit shows the MMAs it issued
// complete and the copies it issued have landed (those waits bounded too).
#pragma once

#include <cuda.h>

#include "tc.cuh"

namespace ct {
namespace tc {

template <int NT, int ST>
struct ConvTmaSmem {
    static constexpr int kPlaneA = 128 * 64;  // bytes: 128 rows x 32 BF16
    static constexpr int kPlaneB = NT * 64;
    static constexpr int kStage = 2 * kPlaneA + 2 * kPlaneB;  // two 32-element K planes of A and of B
    static constexpr int kBytes = ST * kStage + 256 + 1024;  // + barriers, flags, alignment slack
};

// Geometry of one convolution as the producer sees it.
struct ConvTmaGeo {
    int H, W, Ci;
    int k_planes;  // 9 Ci / 32
};

__device__ __forceinline__ int vload(const int *p) { return *(volatile const int *)p; }

template <int NT, int ST, class Epi>
__global__ void __launch_bounds__(128) conv_tma_kernel(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB, Epi E,
                                                       ConvTmaGeo geo, int *err)
{
    using S = ConvTmaSmem<NT, ST>;
    extern __shared__ unsigned char tc_dyn_smem[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)tc_dyn_smem + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + ST * S::kStage);
    uint64_t *empty = full + ST;
    uint64_t *done = empty + ST;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *sabort = reinterpret_cast<int *>(tslot + 1);
    int *sissued = sabort + 1;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const int k_steps = (geo.k_planes + 1) / 2;
    const uint32_t sbase = smem_u32(base);
    if (warp == 0) tmem_alloc(tslot, NT);
    if (tid == 0) {
        for (int b = 0; b < ST; b++) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        mbar_init(done, 1);
        *sabort = 0;
        *sissued = 0;
        fence_mbar_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        // producer: the stage's A and B planes by TMA, counted in bytes on its "full" barrier
        const int HW = geo.H * geo.W;
        const int img = m0 / HW, rem = m0 - img * HW;
        const int y0 = rem / geo.W, x0 = rem - y0 * geo.W;
        int issued = 0;
        for (int s = 0; s < k_steps; s++) {
            const int b = s % ST;
            if (vload(sabort)) break;
            // the buffer's previous stage (s - ST) must have been consumed by its MMAs
            if (s >= ST && !mbar_wait(&empty[b], ((s / ST) - 1) & 1, err)) {
                *(volatile int *)sabort = 1;
                break;
            }
            const int np = min(2, geo.k_planes - 2 * s);
            mbar_arrive_expect_tx(&full[b], (uint32_t)np * (S::kPlaneA + S::kPlaneB));
            const uint32_t st = sbase + b * S::kStage;
            for (int h = 0; h < np; h++) {
                const int k = 64 * s + 32 * h, tap = k / geo.Ci, c = k - tap * geo.Ci;
                tma_load_4d(st + h * S::kPlaneA, &mapA, c, x0 + tap % 3 - 1, y0 + tap / 3 - 1, img, &full[b]);
                tma_load_2d(st + 2 * S::kPlaneA + h * S::kPlaneB, &mapB, k, n0, &full[b]);
            }
            issued = s + 1;
        }
        *(volatile int *)sissued = issued;
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(NT);
        for (int s = 0; s < k_steps; s++) {
            const int b = s % ST;
            if (!mbar_wait(&full[b], (s / ST) & 1, err)) {
                *(volatile int *)sabort = 1;
                break;
            }
            fence_after_sync();
            const int np = min(2, geo.k_planes - 2 * s);
            const uint32_t st = sbase + b * S::kStage;
            for (int h = 0; h < np; h++) {
#pragma unroll
                for (int q = 0; q < 2; q++)
                    mma_bf16(tmem, smem_desc_sw64(st + h * S::kPlaneA + 32 * q),
                             smem_desc_sw64(st + 2 * S::kPlaneA + h * S::kPlaneB + 32 * q), idesc,
                             (s > 0 || h > 0 || q > 0) ? 1u : 0u);
            }
            mma_commit(&empty[b]);
        }
        mma_commit(done);  // fires once every MMA issued above has completed (also after an abort)
    }
    // the accumulator: complete when `done` fires
    if (!mbar_wait(done, 0, err)) *(volatile int *)sabort = 1;
    __syncthreads();
    const bool ok = vload(sabort) == 0;
    if (ok) {
        fence_after_sync();
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        const int m = m0 + 32 * warp + (tid & 31);
        const typename Epi::Ctx ctx{};
#pragma unroll 1
        for (int c = 0; c < NT; c += 16) {
            float v[16];
            tmem_ld16(trow + c, v);
            E.store(m, n0 + c, v, ctx);
        }
    } else if (tid == 0) {
        // give-up path: wait (bounded) until the copies still in flight have landed
        const int issued = vload(sissued);
        for (int s = max(0, issued - ST); s < issued; s++) mbar_wait(&full[s % ST], (s / ST) & 1, nullptr);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NT);
}

}  // namespace tc
}  // namespace ct
