// Resident system matrix of a 2-D fan-beam geometry (ct_geom_precompute).
//
// The SF weights a_ij (Sec. III, Eq. (ct_problem): A is the projection
// matrix) depend on the geometry only.  For a 2-D scan the whole matrix fits
// in HBM (about 8.4 GB for 512x512 pixels, 984 views x 888 cells), so it is
// evaluated once with the same device functions the on-the-fly projectors
// use and then streamed:
//   * ray-major rows: for every ray, its a_ij in the order the ray kernel
//     visits the pixels (march order), two per 12-byte pair (two weights, two
//     16-bit pixel-index offsets from the first index of the pair's run of 32
//     pairs) plus one 32-bit base index per run, for the ray-driven
//     projector.  The indices address the packed image [x | x^T]: a steep
//     ray, marched row by row, indexes the transposed copy, so that the 64
//     entries a warp gathers at once lie on a few columns of x^T instead of
//     some twenty rows of x;
//   * per-(view, pixel) records for the voxel-driven back-projector, in
//     chunks of 32 pixels of a 16x16 tile: each footprint's first cell and
//     cell count in 16 bits, then K weights per pixel interleaved across the
//     32 (K the chunk's widest footprint), about 18 bytes per record at
//     512x512 against 24 for five padded weights and a base cell.
//     Geometries with footprints wider than 15 cells keep no records and
//     back-project on the fly.
// Building it: count each ray's nonzero weights, exclusive-scan the counts
// into row pointers, fill the rows; size each record chunk, exclusive-scan
// the sizes into chunk starts, fill the chunks.
#include <algorithm>
#include <vector>

#include "ct_internal.cuh"

namespace ct {
namespace {

__global__ void __launch_bounds__(256) matrix_count_kernel(FanDev G, long long *__restrict__ counts)
{
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long)G.na * G.ns) return;
    const int v = (int)(ray / G.ns), s = (int)(ray - (long)v * G.ns);
    const float2 cs = __ldg(&G.view_cs[v]);
    long long c = 0;
    ray_visit(G, v, s, 0, 1, [&](int ix, int iy) {
        const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
        if (cell_weight(F, s) != 0.0f) c++;
    });
    counts[ray] = (c + 1) / 2;  // entry pairs
}

// Entries of one ray in march order, two per pair: a_ij, and the pixel index as a 16-bit offset from
// the first index of its chunk (the ray's pairs in runs of 32), chunk bases in base[chunk0[ray] ..];
// an odd count ends with a zero entry; *too_far is set if an offset does not fit.
__global__ void __launch_bounds__(256) matrix_fill_kernel(FanDev G, const long long *__restrict__ row_ptr,
                                                          const int *__restrict__ chunk0, float *__restrict__ wts,
                                                          short *__restrict__ offs, int *__restrict__ base,
                                                          int *__restrict__ too_far)
{
    const long ray = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= (long)G.na * G.ns) return;
    const int v = (int)(ray / G.ns), s = (int)(ray - (long)v * G.ns);
    const float2 cs = __ldg(&G.view_cs[v]);
    const long long b = 2 * row_ptr[ray], end = 2 * row_ptr[ray + 1];  // entry slots
    long long p = b;
    int cur = 0, c = chunk0[ray];
    const bool steep = ray_steep(G, v, s);
    ray_visit(G, v, s, 0, 1, [&](int ix, int iy) {
        const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
        const float wv = cell_weight(F, s);
        if (wv != 0.0f && p < end) {
            const int j = steep ? G.nx * G.ny + ix * G.ny + iy : iy * G.nx + ix;
            if ((p - b) % 64 == 0) {
                cur = j;
                base[c++] = j;
            }
            const int dj = j - cur;
            if (dj > 32767 || dj < -32768) atomicExch(too_far, 1);
            wts[p] = wv;
            offs[p] = (short)dj;
            p++;
        }
    });
    if (p < end) {  // pad the last pair
        wts[p] = 0.0f;
        offs[p] = 0;
    }
}

// Back-projector records (layout at kRecGroup), one CTA per (view, tile): thread t = slot t, warp w the
// chunk of group w.  A record holds the footprint's cells with a nonzero a_ij (as cell_weight evaluates
// them: the same a_ij as the ray-major rows), clipped to the detector.  COUNT: each chunk's size
// (32-byte units) to units[]; a footprint of more than kRecMaxCells cells sets *wide (the build then
// keeps no records).  Otherwise units[] holds each chunk's start (exclusive scan of the sizes): write
// the chunks and the groups' words.
template <bool COUNT>
__global__ void __launch_bounds__(256) matrix_rec_kernel(FanDev G, long long *__restrict__ units,
                                                         unsigned char *__restrict__ data,
                                                         unsigned int *__restrict__ grp, int *wide)
{
    const int ntiles = G.ntx * G.nty;
    const int v = blockIdx.x / ntiles, tile = blockIdx.x - v * ntiles;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile, lane = threadIdx.x & 31;
    const int ty = tile / G.ntx, tx = tile - ty * G.ntx;
    // pixels of a partial tile beyond the image get the edge pixel's (unused) record
    const int ix = min(tx * kTile + lx, G.nx - 1), iy = min(ty * kTile + ly, G.ny - 1);
    const float2 cs = __ldg(&G.view_cs[v]);
    const Footprint F = pixel_footprint(G, v, cs.x, cs.y, ix, iy);
    const int c0 = max(F.n + foot_first(F), 0), c1 = min(F.n + foot_last(F), G.ns - 1);
    int cnt = max(c1 - c0 + 1, 0);
    if (cnt > kRecMaxCells) {
        if (COUNT) atomicExch(wide, 1);
        cnt = kRecMaxCells;  // (only reached when the count pass has already rejected the build)
    }
    const int K = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
    const size_t g = (size_t)blockIdx.x * (kTile * kTile / kRecGroup) + (threadIdx.x >> 5);
    if (COUNT) {
        if (lane == 0) units[g] = 2 + 4 * K;
        return;
    }
    const long long u = units[g];
    unsigned char *c = data + 32 * (size_t)u;
    reinterpret_cast<unsigned short *>(c)[lane] = (unsigned short)((cnt > 0 ? c0 : 0) | (cnt << 12));
    float *w = reinterpret_cast<float *>(c + 64) + lane;
    for (int i = 0; i < K; i++) w[32 * i] = i < cnt ? cell_weight(F, c0 + i) : 0.0f;
    if (lane == 0) grp[g] = (unsigned int)u | ((unsigned int)K << 28);
}

// in-place exclusive scan of blocks of 1024 values; block totals to sums
__global__ void __launch_bounds__(1024) scan_block_kernel(long long *__restrict__ a, long long n,
                                                          long long *__restrict__ sums)
{
    __shared__ long long sm[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long v = i < n ? a[i] : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long t = sm[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        sm[lane] = t;
    }
    __syncthreads();
    const long long incl = x + (warp > 0 ? sm[warp - 1] : 0);
    if (i < n) a[i] = incl - v;
    if (threadIdx.x == 1023) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) scan_add_kernel(long long *__restrict__ a, long long n,
                                                        const long long *__restrict__ sums)
{
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) a[i] += sums[blockIdx.x];
}

cudaError_t exclusive_scan(long long *a, long long n, cudaStream_t st)
{
    const long long nb = (n + 1023) / 1024;
    long long *sums = nullptr;
    cudaError_t e = cudaMalloc(&sums, sizeof(long long) * nb);
    if (e != cudaSuccess) return e;
    scan_block_kernel<<<(unsigned)nb, 1024, 0, st>>>(a, n, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess && nb > 1) {
        e = exclusive_scan(sums, nb, st);
        if (e == cudaSuccess) {
            scan_add_kernel<<<(unsigned)nb, 1024, 0, st>>>(a, n, sums);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(sums);
    return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t build_matrix(ct_geom *g, unsigned long long max_bytes, cudaStream_t st, bool *too_big)
{
    *too_big = false;
    FanDev G = g->fan;
    const long long R = (long long)G.na * G.ns;
    const size_t ntile_px = (size_t)G.ntx * G.nty * kTile * kTile;
    long long *rp = nullptr;
    float2 *wts = nullptr;
    int *steps = nullptr;
    int *first = nullptr;
    int *base = nullptr;
    unsigned char *rdata = nullptr;
    unsigned int *rgrp = nullptr;
    long long *ulen = nullptr;
    float *xp = nullptr;
    if (2LL * G.nx * G.ny >= (1LL << 31)) return cudaErrorNotSupported;  // packed-image indices are 32-bit
    cudaError_t e = cudaMalloc(&rp, sizeof(long long) * (R + 1));
    if (e != cudaSuccess) return e;
    auto fail = [&](cudaError_t err) {
        cudaFree(rdata);
        cudaFree(ulen);
        cudaFree(xp);
        cudaFree(rp);
        cudaFree(wts);
        cudaFree(steps);
        cudaFree(first);
        cudaFree(base);
        cudaFree(rgrp);
        return err;
    };
    if ((e = cudaMemsetAsync(rp + R, 0, sizeof(long long), st)) != cudaSuccess) return fail(e);
    matrix_count_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(G, rp);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    if ((e = exclusive_scan(rp, R + 1, st)) != cudaSuccess) return fail(e);
    long long nnz = 0;  // entry pairs
    if ((e = cudaMemcpy(&nnz, rp + R, sizeof(long long), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e);
    // rows: pointers, chunk pointers, 12 bytes per pair, a base index per 32 pairs (bounded by nnz/32 + R)
    const unsigned long long bytes = (unsigned long long)(R + 1) * 8ull + (unsigned long long)R * 4ull +
                                     (unsigned long long)nnz * 12ull + ((unsigned long long)nnz / 32 + R) * 4ull +
                                     (unsigned long long)G.na * ntile_px * 8ull;  // records: an estimate, known below
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if ((max_bytes && bytes > max_bytes) || bytes > (unsigned long long)(0.9 * (double)free_b)) {
        *too_big = true;
        g->matrix_bytes = bytes;
        return fail(cudaSuccess);
    }
    if ((e = cudaMalloc(&wts, sizeof(float2) * (size_t)(nnz > 0 ? nnz : 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&steps, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1))) != cudaSuccess) return fail(e);
    // chunk pointers (runs of 32 pairs of each ray), on the host from the row pointers
    std::vector<long long> hp((size_t)R + 1);
    if ((e = cudaMemcpy(hp.data(), rp, sizeof(long long) * (R + 1), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(e);
    std::vector<int> hc((size_t)R + 2);
    long long nchunks = 0;
    for (long long r = 0; r < R; r++) {
        hc[r] = (int)nchunks;
        nchunks += (hp[r + 1] - hp[r] + 31) / 32;
    }
    hc[R] = (int)nchunks;
    hc[R + 1] = 0;  // the too-far flag
    if (nchunks >= (1LL << 31) - 4) return fail(cudaErrorNotSupported);
    // (R + 2 entries and a spare int for the records' wide flag)
    if ((e = cudaMalloc(&first, sizeof(int) * (size_t)(R + 3))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&base, sizeof(int) * (size_t)(nchunks + 4))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(first, hc.data(), sizeof(int) * (R + 2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMalloc(&xp, sizeof(float) * 2 * (size_t)G.nx * G.ny)) != cudaSuccess) return fail(e);
    matrix_fill_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(G, rp, first, reinterpret_cast<float *>(wts),
                                                                    reinterpret_cast<short *>(steps), base, first + R + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    // records: each chunk's size, their exclusive scan (the chunks' starts), then the chunks
    int *wide = first + R + 2;
    const unsigned nfoot = (unsigned)((size_t)G.ntx * G.nty * G.na);
    const long long ng = (long long)nfoot * (kTile * kTile / kRecGroup);
    long long units = 0;
    int hw = 0;
    bool keep_rec = G.ns <= 4096;  // first cells are 12-bit
    if ((e = cudaMemsetAsync(wide, 0, sizeof(int), st)) != cudaSuccess) return fail(e);
    if (keep_rec) {
        if ((e = cudaMalloc(&ulen, sizeof(long long) * (size_t)(ng + 1))) != cudaSuccess) return fail(e);
        if ((e = cudaMemsetAsync(ulen + ng, 0, sizeof(long long), st)) != cudaSuccess) return fail(e);
        matrix_rec_kernel<true><<<nfoot, 256, 0, st>>>(G, ulen, nullptr, nullptr, wide);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
        if ((e = exclusive_scan(ulen, ng + 1, st)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(&hw, wide, sizeof(hw), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(&units, ulen + ng, sizeof(units), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e);
        // footprints wider than a record can hold, or chunk starts beyond 28 bits: back-project on the fly
        keep_rec = !hw && units < (1LL << 28);
    }
    if (keep_rec) {
        if ((e = cudaMalloc(&rdata, 32 * (size_t)(units > 0 ? units : 1))) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&rgrp, sizeof(unsigned int) * (size_t)ng)) != cudaSuccess) return fail(e);
        matrix_rec_kernel<false><<<nfoot, 256, 0, st>>>(G, ulen, rdata, rgrp, wide);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    cudaFree(ulen);
    ulen = nullptr;
    const unsigned long long rec_bytes =
        rdata ? 32ull * (unsigned long long)units + 4ull * (unsigned long long)ng : 0ull;
    int far = 0;
    if ((e = cudaMemcpy(&far, first + R + 1, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return fail(e);
    if (far) {  // pixel-index steps beyond 16 bits (an image too wide for them): no resident matrix
        g->matrix_bytes = 0;
        return fail(cudaErrorNotSupported);
    }
    // blocks of 8 adjacent cells by their entries over all views, most first: the forward projector
    // launches them in that order, so that the short rays fill the end of the launch
    const int nblk = (G.ns + 7) / 8;
    {
        std::vector<long long> tot(nblk, 0);
        for (int v = 0; v < G.na; v++)
            for (int b = 0; b < nblk; b++) {
                const long long r0 = (long long)v * G.ns + 8 * b, r1 = std::min(r0 + 8, (long long)(v + 1) * G.ns);
                tot[b] += hp[r1] - hp[r0];
            }
        std::vector<int> order(nblk);
        for (int b = 0; b < nblk; b++) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tot[a] > tot[b]; });
        if (!g->d_ray_order && (e = cudaMalloc(&g->d_ray_order, sizeof(int) * nblk)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(g->d_ray_order, order.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
    }
    // the exact size: row pointers, chunk pointers (+ flags), entries, chunk bases, records
    g->matrix_bytes = (unsigned long long)(R + 1) * 8ull + (unsigned long long)(R + 3) * 4ull +
                      (unsigned long long)nnz * 12ull + (unsigned long long)(nchunks + 4) * 4ull + rec_bytes;
    g->rec_bytes = rec_bytes;
    g->d_row_ptr = rp;
    g->d_row_w = wts;
    g->d_row_d = steps;
    g->d_row_first = first;
    g->d_row_base = base;
    g->d_rec_data = rdata;
    g->d_rec_grp = rgrp;
    g->d_xpack = xp;
    g->fan.xpack = xp;
    g->fan.row_ptr = rp;
    g->fan.row_w = wts;
    g->fan.row_d = steps;
    g->fan.row_first = first;
    g->fan.row_base = base;
    g->fan.ray_order = g->d_ray_order;
    g->fan.rec_data = rdata;
    g->fan.rec_grp = rgrp;
    {   // view split of the back-projector: 1, 2 or 4 warps per chunk, the most that keep its CTAs of 4 warps
        // (16 per SM) within one wave; small images then still fill the GPU (a fixed rule of the geometry and
        // the device, so that a solve and its resumption run the same arithmetic)
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long half_tiles = 2L * G.ntx * G.nty, slots = 16L * (nsm > 0 ? nsm : 1);
        int vs = 1;
        while (vs < 4 && half_tiles * vs * 2 <= slots) vs *= 2;
        g->fan.bp_vs = vs;
    }
    return cudaSuccess;
}

}  // namespace ct

using namespace ct;

extern "C" ct_status ct_geom_precompute(ct_geom *g, unsigned long long max_bytes, unsigned long long *bytes_out,
                                        void *stream)
{
    if (!g) { set_error("ct_geom_precompute: null geometry"); return CT_EINVAL; }
    if (g->helical) {
        set_error("ct_geom_precompute: the resident matrix is built for 2-D fan-beam geometries only");
        return CT_ENOTSUP;
    }
    const bool built_now = !g->d_row_ptr;
    if (!g->d_row_ptr) {
        bool too_big = false;
        cudaError_t e = build_matrix(g, max_bytes, (cudaStream_t)stream, &too_big);
        if (e == cudaErrorNotSupported) {
            set_error("ct_geom_precompute: the image is too wide for the matrix's 16-bit pixel steps");
            return CT_ENOTSUP;
        }
        if (e != cudaSuccess) return cuda_fail(e, "building the system matrix");
        if (too_big) {
            if (bytes_out) *bytes_out = g->matrix_bytes;
            set_error("system matrix needs %llu bytes (limit %llu, or 90%% of free device memory)", g->matrix_bytes,
                      max_bytes);
            return CT_ENOMEM;
        }
    }
    if (built_now) {  // the ray sums A 1 from the resident matrix (the path every later D_L uses)
        drop_ray_sums(g);
        CT_CUDA_TRY(ensure_ray_sums(g, (cudaStream_t)stream), "ray sums A 1");
        CT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "ray sums A 1");
    }
    if (bytes_out) *bytes_out = g->matrix_bytes;
    return CT_OK;
}

extern "C" ct_status ct_geom_matrix_info(const ct_geom *g, unsigned long long *matrix_bytes,
                                         unsigned long long *record_bytes)
{
    if (!g) { set_error("ct_geom_matrix_info: null geometry"); return CT_EINVAL; }
    const bool built = g->d_row_ptr != nullptr;
    if (matrix_bytes) *matrix_bytes = built ? g->matrix_bytes : 0ull;
    if (record_bytes) *record_bytes = built ? g->rec_bytes : 0ull;
    return CT_OK;
}
