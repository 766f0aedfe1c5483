// a1 - Neighbour blocks (paper Sec. 2.3, "Neighbor list").
//
// Atoms are sorted into a cell grid whose numbering follows one dimension contiguously
// (Sec. 2.3.1, box partitioning), then cut into groups of exactly 32 consecutive atoms
// (B_size = warp size). Interacting group pairs are those whose bounding boxes are
// within cutoff + buffer; they form the "adjacency" of Sec. 2.3.1, compacted into a
// list sorted by the first group. Bonded pairs whose scale differs from 1 are not
// stored per atom (Sec. 1.2.1 moves them out of the pair loop); here each group pair
// that holds any gets a 32 x 32-bit mask instead.
//
// GB300 choices (differences from the paper): cells are 1/4 of a 32-atom cube along x
// and the cell order snakes through x and y, so every run of 32 atoms stays compact
// without the paper's iterative refinement; the block-pair test is a brute-force
// bounding-box sweep over block pairs (n_blocks^2 / 2 tests, a few ms even at 10^6
// atoms), which needs no bit matrix at all.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

struct CellGrid {
    int nx, ny, nz;
    double lx, ly, lz;
};

__device__ __forceinline__ double wrap1(double x, double L) {
    double w = x - L * floor(x / L);
    return (w >= L) ? 0.0 : w;
}

__global__ void k_cell_key(const double *__restrict__ xyz, int n, CellGrid g, int *__restrict__ key) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = wrap1(xyz[3 * i + 0], g.lx), y = wrap1(xyz[3 * i + 1], g.ly), z = wrap1(xyz[3 * i + 2], g.lz);
    // clamp: a non-finite coordinate must not index outside the cell arrays
    int cx = isfinite(x) ? max(0, min(g.nx - 1, (int)(x / g.lx * g.nx))) : 0;
    int cy = isfinite(y) ? max(0, min(g.ny - 1, (int)(y / g.ly * g.ny))) : 0;
    int cz = isfinite(z) ? max(0, min(g.nz - 1, (int)(z / g.lz * g.nz))) : 0;
    // serpentine numbering: y reverses on odd z-planes, x reverses on odd rows
    int cyy = (cz & 1) ? (g.ny - 1 - cy) : cy;
    int row = cz * g.ny + cyy;
    int cxx = (row & 1) ? (g.nx - 1 - cx) : cx;
    key[i] = row * g.nx + cxx;
}

__global__ void k_histogram(const int *__restrict__ key, int n, int *__restrict__ count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&count[key[i]], 1);
}

// exclusive scan of m ints with one block of 1024 threads (build-time only)
__global__ void k_scan_single(const int *__restrict__ in, int *__restrict__ out, int m, int *__restrict__ total) {
    __shared__ int sums[1024];
    int t = threadIdx.x;
    int chunk = (m + 1023) / 1024;
    int b = t * chunk, e = min(m, b + chunk);
    int s = 0;
    for (int k = b; k < e; ++k) s += in[k];
    sums[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = (t >= off) ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int run = sums[t] - s;
    for (int k = b; k < e; ++k) {
        int v = in[k];
        out[k] = run;
        run += v;
    }
    if (t == 1023 && total) *total = sums[1023];
}

__global__ void k_scatter(const int *__restrict__ key, int n, const int *__restrict__ start,
                          int *__restrict__ cursor, int *__restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = key[i];
    perm[start[k] + atomicAdd(&cursor[k], 1)] = i;
}

// deterministic order inside each cell: ascending atom index (insertion sort; cells hold ~8)
__global__ void k_sort_cells(const int *__restrict__ start, const int *__restrict__ count, int ncell,
                             int *__restrict__ perm) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], m = count[c];
    for (int a = 1; a < m; ++a) {
        int v = perm[b + a];
        int k = a - 1;
        while (k >= 0 && perm[b + k] > v) { perm[b + k + 1] = perm[b + k]; --k; }
        perm[b + k + 1] = v;
    }
}

__global__ void k_finish_perm(int *__restrict__ perm, int n, int n_pad, int *__restrict__ iperm) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    if (s >= n) { perm[s] = -1; return; }
    iperm[perm[s]] = s;
}

// one warp per block: bounding box of its atoms (wrapped coordinates)
__global__ void k_block_bbox(const double *__restrict__ xyz, const int *__restrict__ perm, int nb,
                             double lx, double ly, double lz, float4 *__restrict__ center,
                             float4 *__restrict__ half, unsigned *__restrict__ hmax_bits) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= nb) return;
    int a = perm[w * 32 + lane];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    if (a >= 0) {
        double p[3] = {wrap1(xyz[3 * a], lx), wrap1(xyz[3 * a + 1], ly), wrap1(xyz[3 * a + 2], lz)};
        for (int d = 0; d < 3; ++d) lo[d] = hi[d] = p[d];
    }
    for (int off = 16; off; off >>= 1)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    if (lane == 0) {
        center[w] = make_float4((float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                                (float)(0.5 * (lo[2] + hi[2])), 0.f);
        float h[3];
        for (int d = 0; d < 3; ++d) h[d] = (float)(0.5 * (hi[d] - lo[d])) + 1e-4f;
        half[w] = make_float4(h[0], h[1], h[2], 0.f);
        for (int d = 0; d < 3; ++d) atomicMax(&hmax_bits[d], __float_as_uint(h[d]));
    }
}

__device__ __forceinline__ bool blocks_near(float4 ci, float4 hi, float4 cj, float4 hj, float3 L, float r2) {
    float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
    dx -= L.x * rintf(dx / L.x);
    dy -= L.y * rintf(dy / L.y);
    dz -= L.z * rintf(dz / L.z);
    float gx = fmaxf(0.f, fabsf(dx) - hi.x - hj.x);
    float gy = fmaxf(0.f, fabsf(dy) - hi.y - hj.y);
    float gz = fmaxf(0.f, fabsf(dz) - hi.z - hj.z);
    return gx * gx + gy * gy + gz * gz < r2;
}

// one warp per block I: count (fill == nullptr) or write its partners J >= I
__global__ void k_tiles(const float4 *__restrict__ center, const float4 *__restrict__ half, int nb,
                        float3 L, float r2, int *__restrict__ count, const int *__restrict__ off,
                        int2 *__restrict__ tiles, float4 *__restrict__ tshift, float4 *__restrict__ tshift_lo,
                        double3 Ld) {
    int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (I >= nb) return;
    float4 ci = center[I], hi = half[I];
    int pos = tiles ? off[I] : 0;
    int cnt = 0;
    for (int base = I; base < nb; base += 32) {
        int J = base + lane;
        bool hit = false;
        if (J < nb) hit = blocks_near(ci, hi, center[J], half[J], L, r2);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (tiles && hit) {
            int k = pos + __popc(m & ((1u << lane) - 1u));
            tiles[k] = make_int2(I, J);
            float4 cj = center[J];
            // origin of J's image next to I, relative to I's origin: c_J - c_I + L k in FP64,
            // split into float hi + lo (the centres are the blocks' position origins)
            const double ox = (double)cj.x - (double)ci.x + Ld.x * rintf((ci.x - cj.x) / L.x);
            const double oy = (double)cj.y - (double)ci.y + Ld.y * rintf((ci.y - cj.y) / L.y);
            const double oz = (double)cj.z - (double)ci.z + Ld.z * rintf((ci.z - cj.z) / L.z);
            const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
            tshift[k] = make_float4(hx, hy, hz, 0.f);
            tshift_lo[k] = make_float4((float)(ox - hx), (float)(oy - hy), (float)(oz - hz), 0.f);
        }
        pos += __popc(m);
        cnt += __popc(m);
    }
    if (!tiles && lane == 0) count[I] = cnt;
}

__device__ int find_tile(const int2 *__restrict__ tiles, int b, int e, int J) {
    while (b < e) {
        int m = (b + e) >> 1;
        int v = tiles[m].y;
        if (v == J) return m;
        if (v < J) b = m + 1; else e = m;
    }
    return -1;
}

// pass 0: flag tiles holding excluded pairs; pass 1: set the mask bits
__global__ void k_excl(const int *__restrict__ off, const int *__restrict__ atoms, int n,
                       const int *__restrict__ iperm, const int2 *__restrict__ tiles,
                       const int *__restrict__ tile_off, int *__restrict__ tile_flag,
                       const int *__restrict__ tile_excl, unsigned *__restrict__ masks,
                       int pass, int *__restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = off[i]; k < off[i + 1]; ++k) {
        int j = atoms[k];
        if (j == i || j < 0 || j >= n) continue;
        int si = iperm[i], sj = iperm[j];
        int bI = si >> 5, li = si & 31, bJ = sj >> 5, lj = sj & 31;
        if (bI > bJ) { int t = bI; bI = bJ; bJ = t; t = li; li = lj; lj = t; }
        int t = find_tile(tiles, tile_off[bI], tile_off[bI + 1], bJ);
        if (t < 0) { atomicExch(err, 1); continue; }
        if (pass == 0) {
            tile_flag[t] = 1;
        } else {
            unsigned *m = masks + (size_t)tile_excl[t] * 32;
            atomicOr(&m[li], 1u << lj);
            if (bI == bJ) atomicOr(&m[lj], 1u << li);
        }
    }
}

__global__ void k_assign_slots(const int *__restrict__ flag, const int *__restrict__ scan, int m,
                               int *__restrict__ tile_excl) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) tile_excl[t] = flag[t] ? scan[t] : -1;
}

template <class P>
int grow(ap_ctx *ctx, P **ptr, int *cap, long need, size_t elem) {
    if (need <= *cap) return AP_OK;
    long c = std::max<long>(need + need / 4 + 64, 1024);
    if (*ptr) AP_CUDA(cudaFree(*ptr));
    *ptr = nullptr;
    AP_CUDA(cudaMalloc((void **)ptr, (size_t)c * elem));
    *cap = (int)c;
    return AP_OK;
}

}  // namespace

int nb_build(ap_ctx *ctx, const double *d_xyz, const int *d_off, const int *d_atoms, int n_excl) {
    const ap_params &P = ctx->prm;
    cudaStream_t s = ctx->s0;
    const int n = ctx->n, n_pad = ctx->n_pad, nb = ctx->n_blocks;
    double vol = P.box[0] * P.box[1] * P.box[2];
    double rho = n / vol;
    double c = std::cbrt(32.0 / rho);
    CellGrid g;
    g.ny = std::max(1, (int)std::floor(P.box[1] / c));
    g.nz = std::max(1, (int)std::floor(P.box[2] / c));
    g.nx = std::max(1, (int)std::floor(4.0 * P.box[0] / c));
    g.lx = P.box[0]; g.ly = P.box[1]; g.lz = P.box[2];
    long ncell = (long)g.nx * g.ny * g.nz;
    if (ncell > (1L << 26)) return ap_fail(ctx, AP_ERR_ARG, "cell grid too large");

    int r;
    if ((r = grow(ctx, &ctx->cell_count, &ctx->cap_cells, 3 * ncell + 3, sizeof(int)))) return r;
    if ((r = grow(ctx, &ctx->tmp_int, &ctx->cap_tmp, std::max<long>(n, 4L * nb + 8), sizeof(int)))) return r;
    int *count = ctx->cell_count, *start = count + ncell, *cursor = start + ncell;
    int *key = ctx->tmp_int;
    const int T = 256;

    AP_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * ncell, s));
    AP_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, s));
    k_cell_key<<<ap_grid_for(n, T), T, 0, s>>>(d_xyz, n, g, key);
    k_histogram<<<ap_grid_for(n, T), T, 0, s>>>(key, n, count);
    k_scan_single<<<1, 1024, 0, s>>>(count, start, (int)ncell, nullptr);
    k_scatter<<<ap_grid_for(n, T), T, 0, s>>>(key, n, start, cursor, ctx->perm);
    k_sort_cells<<<ap_grid_for(ncell, T), T, 0, s>>>(start, count, (int)ncell, ctx->perm);
    k_finish_perm<<<ap_grid_for(n_pad, T), T, 0, s>>>(ctx->perm, n, n_pad, ctx->iperm);
    AP_CUDA(cudaGetLastError());

    // block boxes
    float4 *half = nullptr;
    unsigned *hmax = nullptr;
    AP_CUDA(cudaMallocAsync((void **)&half, sizeof(float4) * nb + 16, s));
    AP_CUDA(cudaMallocAsync((void **)&hmax, sizeof(unsigned) * 4, s));
    AP_CUDA(cudaMemsetAsync(hmax, 0, sizeof(unsigned) * 4, s));
    k_block_bbox<<<ap_grid_for((long)nb * 32, T), T, 0, s>>>(d_xyz, ctx->perm, nb, P.box[0], P.box[1], P.box[2],
                                                           ctx->bcenter, half, hmax);
    float3 L = make_float3((float)P.box[0], (float)P.box[1], (float)P.box[2]);
    float rl = (float)(P.cutoff + P.buffer);
    int *bcount = key;                 // reuse: key no longer needed
    int *boff = key + nb + 1;
    k_tiles<<<ap_grid_for((long)nb * 32, T), T, 0, s>>>(ctx->bcenter, half, nb, L, rl * rl, bcount, nullptr,
                                                      nullptr, nullptr, nullptr, make_double3(P.box[0], P.box[1], P.box[2]));
    int *d_total = boff + nb + 1;
    k_scan_single<<<1, 1024, 0, s>>>(bcount, boff, nb, d_total);
    int ntiles = 0;
    unsigned hm[3];
    AP_CUDA(cudaMemcpyAsync(&ntiles, d_total, sizeof(int), cudaMemcpyDeviceToHost, s));
    AP_CUDA(cudaMemcpyAsync(hm, hmax, sizeof(unsigned) * 3, cudaMemcpyDeviceToHost, s));
    AP_CUDA(cudaStreamSynchronize(s));
    AP_CUDA(cudaMemcpyAsync(boff + nb, &ntiles, sizeof(int), cudaMemcpyHostToDevice, s));
    if (ntiles <= 0) return ap_fail(ctx, AP_ERR_ARG, "no interacting blocks");

    if ((r = grow(ctx, &ctx->tiles, &ctx->cap_tiles, ntiles, sizeof(int2)))) return r;
    if (ctx->tshift) cudaFree(ctx->tshift);
    if (ctx->tshift_lo) cudaFree(ctx->tshift_lo);
    if (ctx->tile_excl) cudaFree(ctx->tile_excl);
    AP_CUDA(cudaMalloc((void **)&ctx->tshift, sizeof(float4) * ctx->cap_tiles));
    AP_CUDA(cudaMalloc((void **)&ctx->tshift_lo, sizeof(float4) * ctx->cap_tiles));
    AP_CUDA(cudaMalloc((void **)&ctx->tile_excl, sizeof(int) * ctx->cap_tiles));
    k_tiles<<<ap_grid_for((long)nb * 32, T), T, 0, s>>>(ctx->bcenter, half, nb, L, rl * rl, nullptr, boff,
                                                      ctx->tiles, ctx->tshift, ctx->tshift_lo,
                                                      make_double3(P.box[0], P.box[1], P.box[2]));
    ctx->n_tiles = ntiles;
    // keep the per-block tile offsets at the head of tmp_int for the exclusion pass
    int *tile_off = boff;

    // per-tile shift is exact when every dimension satisfies L > 2 r_c + 4 (h_max + buffer/2)
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
        float h;
        memcpy(&h, &hm[d], sizeof(float));
        if (!(P.box[d] > 2.0 * P.cutoff + 4.0 * (h + 0.5 * P.buffer))) ok = false;
    }
    ctx->minimg = ok ? 0 : 1;

    // exclusion masks
    ctx->n_excl_tiles = 0;
    AP_CUDA(cudaMemsetAsync(ctx->tile_excl, 0xff, sizeof(int) * ntiles, s));
    if (n_excl > 0) {
        int *flag = nullptr, *scan = nullptr, *err = nullptr;
        AP_CUDA(cudaMallocAsync((void **)&flag, sizeof(int) * (2L * ntiles + 4), s));
        scan = flag + ntiles + 1;
        AP_CUDA(cudaMallocAsync((void **)&err, sizeof(int) * 2, s));
        AP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * ntiles, s));
        AP_CUDA(cudaMemsetAsync(err, 0, sizeof(int) * 2, s));
        k_excl<<<ap_grid_for(n, T), T, 0, s>>>(d_off, d_atoms, n, ctx->iperm, ctx->tiles, tile_off, flag,
                                              nullptr, nullptr, 0, err);
        k_scan_single<<<1, 1024, 0, s>>>(flag, scan, ntiles, err + 1);
        int hv[2];
        AP_CUDA(cudaMemcpyAsync(hv, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
        AP_CUDA(cudaStreamSynchronize(s));
        if (hv[0]) {
            cudaFreeAsync(flag, s); cudaFreeAsync(err, s); cudaFreeAsync(half, s); cudaFreeAsync(hmax, s);
            return ap_fail(ctx, AP_ERR_ARG, "an excluded pair is farther apart than cutoff+buffer");
        }
        int nex = hv[1];
        if ((r = grow(ctx, &ctx->excl_mask, &ctx->cap_excl, (long)nex * 32, sizeof(unsigned)))) return r;
        k_assign_slots<<<ap_grid_for(ntiles, T), T, 0, s>>>(flag, scan, ntiles, ctx->tile_excl);
        AP_CUDA(cudaMemsetAsync(ctx->excl_mask, 0, sizeof(unsigned) * 32 * (size_t)std::max(nex, 1), s));
        k_excl<<<ap_grid_for(n, T), T, 0, s>>>(d_off, d_atoms, n, ctx->iperm, ctx->tiles, tile_off, flag,
                                              ctx->tile_excl, ctx->excl_mask, 1, err);
        ctx->n_excl_tiles = nex;
        AP_CUDA(cudaFreeAsync(flag, s));
        AP_CUDA(cudaFreeAsync(err, s));
    }
    AP_CUDA(cudaMemcpyAsync(ctx->tile_off, tile_off, sizeof(int) * (nb + 1), cudaMemcpyDeviceToDevice, s));
    AP_CUDA(cudaFreeAsync(half, s));
    AP_CUDA(cudaFreeAsync(hmax, s));
    AP_CUDA(cudaStreamSynchronize(s));
    AP_CUDA(cudaGetLastError());
    if ((r = filter_alloc(ctx))) return r;
    ctx->lists_valid = 1;
    ctx->config_valid = 0;
    ctx->graph_ok = 0;             // pointers may have moved: rebuild the solve graph
    ctx->graph_tried = 0;
    if (ctx->solve_exec) { cudaGraphExecDestroy(ctx->solve_exec); ctx->solve_exec = nullptr; }
    return AP_OK;
}
