// Tensor-core GEMM core for sm_103a: D (128 x NT, FP32, in tensor memory) =
// sum over K of A (128 x K) * B (NT x K)^T with BF16 operands, both K-major.
// One CTA of 128 threads computes one 128 x NT tile:
//   * all threads stage K-slices of 64 elements of A and B into shared memory
//     (a loader object decides where the elements come from: plain matrices,
//     implicit im2col of a 3x3 convolution, or transposed gradient tiles),
//     ST stages deep so staging of slices s+1 .. s+ST-1 overlaps the MMAs of slice s
//     (init() returns the thread's per-tile context, load() stages a slice,
//     store() consumes 16 accumulator columns of one row);
//   * thread 0 issues four 128 x NT x 16 tcgen05.mma per slice into one
//     tensor-memory accumulator and commits them to the slice's mbarrier;
//   * the epilogue reads the accumulator rows (warp w owns rows 32w..32w+31)
//     16 columns at a time and hands them to the loader's store().
// Every mbarrier wait is bounded (error flag, no hang); after a wait gives up no
// more MMAs are issued, and the tensor memory is freed only once a final commit
// shows the MMAs already issued complete (that wait bounded too).
#pragma once

#include "tc.cuh"

namespace ct {
namespace tc {

template <int NT, int ST>
struct GemmSmem {
    static constexpr int kA = 128 * kStageK * 2;
    static constexpr int kB = NT * kStageK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kBytes = ST * kStage + 64 + 1024;  // + barriers, TMEM slot, abort flag, drain barrier,
                                                            // alignment slack
};

// Pipeline depth: two stages, so that four CTAs (16 warps) share an SM; three or four stages (two CTAs
// per SM) measured slower on the U-Net layers (forward 3.08 ms vs 2.72 ms at batch 16).
__host__ __device__ constexpr int gemm_stages(int) { return 2; }

template <int NT, class Ld, int ST = gemm_stages(NT)>
__global__ void __launch_bounds__(128) gemm_kernel(Ld L, int k_steps, int *err)
{
    static_assert(NT == 32 || NT == 64 || NT == 128 || NT == 256, "NT must be a power of two in [32, 256]");
    static_assert(ST >= 2 && ST <= 4, "2 to 4 stages");
    using S = GemmSmem<NT, ST>;
    extern __shared__ unsigned char tc_dyn_smem[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)tc_dyn_smem + 1023) & ~(uintptr_t)1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + ST * S::kStage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + ST);
    int *sabort = reinterpret_cast<int *>(bar + ST + 1);
    uint64_t *drain = bar + ST + 2;  // completion of every MMA issued (the give-up path)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * NT;
    const uint32_t sbase = smem_u32(base);
    if (warp == 0) tmem_alloc(tslot, NT);
    if (tid == 0) {
        for (int b = 0; b < ST; b++) mbar_init(&bar[b], 1);
        mbar_init(drain, 1);
        *sabort = 0;
        fence_mbar_init();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_bf16(NT);

    const typename Ld::Ctx ctx = L.init(m0, n0, tid);
    // prologue: slices 0 .. ST-2 (one commit group each, possibly empty)
#pragma unroll
    for (int p = 0; p < ST - 1; p++) {
        if (p < k_steps) L.load(p, sbase + p * S::kStage, sbase + p * S::kStage + S::kA, ctx, tid);
        cp_async_commit();
    }
    for (int s = 0; s < k_steps; s++) {
        const int b = s % ST;
        const uint32_t sa = sbase + b * S::kStage, sb = sa + S::kA;
        const int sn = s + ST - 1;  // the slice staged now, into the buffer of slice s-1
        if (sn < k_steps) {
            const int bn = sn % ST;
            // that buffer was read by the MMAs of slice s-1: wait for them before refilling it
            if (s >= 1 && !mbar_wait(&bar[bn], ((s - 1) / ST) & 1, err)) *sabort = 1;
            const uint32_t na = sbase + bn * S::kStage;
            if (!*sabort) L.load(sn, na, na + S::kA, ctx, tid);
        }
        cp_async_commit();
        cp_async_wait<ST - 1>();  // the group of slice s is complete
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && !*sabort) {
            fence_after_sync();
#pragma unroll
            for (int q = 0; q < kStageK / 16; q++)
                mma_bf16(tmem, smem_desc(sa + 256 * q), smem_desc(sb + 256 * q), idesc, (s > 0 || q > 0) ? 1u : 0u);
            mma_commit(&bar[b]);
        }
    }
    // the last slice's MMAs complete the accumulator (tcgen05 MMAs complete in order)
    const int last = k_steps - 1;
    if (!*sabort && !mbar_wait(&bar[last % ST], (last / ST) & 1, err)) *sabort = 1;
    __syncthreads();
    const bool ok = !*sabort;
    if (!ok) {
        // a wait gave up: before the tensor memory is freed, wait (bounded again) for every MMA thread 0
        // issued, tracked by one more commit; the accumulator is not read
        if (tid == 0) mma_commit(drain);
        mbar_wait(drain, 0, err);
    }
    fence_after_sync();
    if (ok) {
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        const int m = m0 + 32 * warp + (tid & 31);
#pragma unroll 1
        for (int c = 0; c < NT; c += 16) {
            float v[16];
            tmem_ld16(trow + c, v);
            L.store(m, n0 + c, v, ctx);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NT);
}

}  // namespace tc
}  // namespace ct
