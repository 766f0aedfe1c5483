// Per-configuration list filtering (paper Sec. 2.3.2, "List filtering": an atom belongs to a
// group's neighbourhood when it is within range of some atom of the group; neighbour lists
// are padded with phantom atoms to a multiple of B_size).
//
// The block-pair lists are built with cutoff + buffer and reused for many steps; once the
// positions of a step are known they stay fixed for the field, every PCG matrix-vector
// product and the forces. So at each configuration, for every block I, the atoms of its
// partner blocks J > I that lie within r_c of some atom of I (preselected by I's bounding
// box) are packed into 32-wide
// chunks (positions relative to block I's origin, in the periodic image next to I, padding
// with NaN phantoms) with their exclusion bits carried over. The real-space kernels then
// run over
//   work = [(I, diagonal block), (I, chunk 0), (I, chunk 1), ...] for every I,
// which keeps only a fraction of the candidate pairs of the block-pair tiles while
// preserving the 32 x 32 warp tile. The in-range pair bits of every item (and their transposes) are found
// here too, once per configuration.
#include "common.cuh"
#include "pair_math.cuh"

#include <algorithm>

namespace {

template <class T, bool MINIMG>
__global__ void __launch_bounds__(256) k_filter(
    const int2 *__restrict__ tiles, const int *__restrict__ tile_off, const float4 *__restrict__ tshift,
    const int *__restrict__ tile_excl, const unsigned *__restrict__ excl_mask,
    const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd, int nb,
    T rc2, T Lx, T Ly, T Lz, const float4 *__restrict__ tshift_lo, int *__restrict__ chunk_j,
    typename V4<T>::type *__restrict__ chunk_pos,
    int *__restrict__ chunk_src, unsigned *__restrict__ chunk_mask, int *__restrict__ chunk_flag,
    int *__restrict__ nchunk) {
    typedef typename V4<T>::type T4;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= nb) return;
    // bounding box of block I at the current positions (padding slots hold NaN)
    T4 pi = posq[I * 32 + lane];
    const bool vi = isfinite((float)pi.x);
    T lo[3] = {vi ? pi.x : T(1e30), vi ? pi.y : T(1e30), vi ? pi.z : T(1e30)};
    T hi[3] = {vi ? pi.x : T(-1e30), vi ? pi.y : T(-1e30), vi ? pi.z : T(-1e30)};
    for (int off = 16; off; off >>= 1)
        for (int d = 0; d < 3; ++d) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    const T cx = T(0.5) * (lo[0] + hi[0]), cy = T(0.5) * (lo[1] + hi[1]), cz = T(0.5) * (lo[2] + hi[2]);
    const int base = tile_off[I];
    const int t_end = tile_off[I + 1];
    int count = 0;
    // four tiles per round: their loads are issued together (one warp walks all of block I's
    // tiles, so latency, not bandwidth, bounds this loop), then the selections are packed in
    // tile order
    constexpr int U = 4;
    for (int t0 = base; t0 < t_end; t0 += U) {
        int Jv[U], ev[U];
        T4 qv[U];
        float4 ohv[U], olv[U];
        T wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u;
            Jv[u] = -1;
            qv[u].x = qv[u].y = qv[u].z = qv[u].w = T(0);
            ohv[u] = olv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            wv[u] = T(0);
            ev[u] = -1;
            if (t < t_end) {
                Jv[u] = tiles[t].y;
                const int sj = Jv[u] * 32 + lane;
                qv[u] = posq[sj];
                wv[u] = dipd[sj].w;
                ohv[u] = tshift[t];
                olv[u] = tshift_lo[t];
                ev[u] = tile_excl[t];
            }
        }
        // each candidate moved to block I's origin and periodic image, and its box test
        T xv[U], yv[U], zv[U];
        bool sv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int J = Jv[u];
            const T4 q = qv[u];
            // positions are relative to their block's origin: move j's to block I's origin and
            // periodic image with the tile's offset, kept as a float pair (hi + lo) so that the
            // result (a few A) has full FP32 precision at any box size
            const float4 oh = ohv[u], ol = olv[u];
            T x = (q.x + (T)ol.x) + (T)oh.x, y = (q.y + (T)ol.y) + (T)oh.y, z = (q.z + (T)ol.z) + (T)oh.z;
            if (MINIMG) {
                x -= Lx * rint((x - cx) / Lx);
                y -= Ly * rint((y - cy) / Ly);
                z -= Lz * rint((z - cz) / Lz);
            }
            const T gx = max(T(0), max(lo[0] - x, x - hi[0]));
            const T gy = max(T(0), max(lo[1] - y, y - hi[1]));
            const T gz = max(T(0), max(lo[2] - z, z - hi[2]));
            xv[u] = x;
            yv[u] = y;
            zv[u] = z;
            sv[u] = J >= 0 && J != I && isfinite((float)x) && (gx * gx + gy * gy + gz * gz < rc2);
        }
        // The box test only preselects; the paper's criterion is r_c of some atom of the group
        // (about half the box's candidates in water): the U candidates of each lane against
        // block I's 32 atoms (each shuffled once per round; padding slots hold NaN and never
        // pass). rc2 carries a 1e-5 margin over the pair masks' r_c^2, so no pair within r_c is
        // dropped by rounding.
        bool any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) any |= sv[u];
        if (__any_sync(0xffffffffu, any)) {
            bool nv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) nv[u] = false;
#pragma unroll 4
            for (int il = 0; il < 32; ++il) {
                const T xi = __shfl_sync(0xffffffffu, pi.x, il), yi = __shfl_sync(0xffffffffu, pi.y, il),
                        zi = __shfl_sync(0xffffffffu, pi.z, il);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    T dx = xv[u] - xi, dy = yv[u] - yi, dz = zv[u] - zi;
                    if (MINIMG) {
                        dx -= Lx * rint(dx / Lx);
                        dy -= Ly * rint(dy / Ly);
                        dz -= Lz * rint(dz / Lz);
                    }
                    nv[u] |= dx * dx + dy * dy + dz * dz < rc2;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) sv[u] = sv[u] && nv[u];
        }
        // pack the selections in tile order
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int J = Jv[u];
            if (J < 0 || J == I) continue;   // uniform over the warp
            const bool sel = sv[u];
            const unsigned m = __ballot_sync(0xffffffffu, sel);
            if (sel) {
                const int k = count + __popc(m & ((1u << lane) - 1u));
                const int e = ev[u];
                const size_t slot = (size_t)(base + (k >> 5)) * 32 + (k & 31);
                chunk_j[slot] = J * 32 + lane;
                T4 v;
                v.x = xv[u]; v.y = yv[u]; v.z = zv[u]; v.w = wv[u];
                chunk_pos[slot] = v;
                chunk_src[slot] = e >= 0 ? (e << 5) | lane : -1;
            }
            count += __popc(m);
        }
    }
    const int nc = (count + 31) >> 5;
    // phantom padding of the last chunk
    if (nc > 0) {
        const int k = count + lane;
        if (k < nc * 32) {
            const size_t slot = (size_t)(base + (k >> 5)) * 32 + (k & 31);
            chunk_j[slot] = -1;
            T4 v;
            v.x = v.y = v.z = (T)NAN; v.w = T(0);
            chunk_pos[slot] = v;
            chunk_src[slot] = -1;
        }
    }
    __syncwarp();
    // exclusion masks of the chunks: word i-lane -> bit chunk position
    for (int c = 0; c < nc; ++c) {
        const size_t cs = (size_t)(base + c) * 32;
        const int src = chunk_src[cs + lane];
        const unsigned any = __ballot_sync(0xffffffffu, src >= 0);
        if (lane == 0) chunk_flag[base + c] = any ? 1 : 0;
        if (!any) continue;
        unsigned mine = 0u;
        for (int il = 0; il < 32; ++il) {
            const bool b = src >= 0 && ((excl_mask[(size_t)(src >> 5) * 32 + il] >> (src & 31)) & 1u);
            const unsigned w = __ballot_sync(0xffffffffu, b);
            if (lane == il) mine = w;
        }
        chunk_mask[cs + lane] = mine;
    }
    if (lane == 0) nchunk[I] = nc;
}

// flat work list (I, -1) then (I, chunk) for every block, in block order: first the
// offsets (exclusive scan of 1 + nchunk, one CTA), then one warp per block writes its items
__global__ void k_work_offsets(const int *__restrict__ nchunk, int nb, int *__restrict__ off,
                               int *__restrict__ n_work) {
    __shared__ int sums[1024];
    const int t = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b = min(nb, t * per), e = min(nb, b + per);
    int s = 0;
    for (int k = b; k < e; ++k) s += 1 + nchunk[k];
    sums[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int v = t >= d ? sums[t - d] : 0;
        __syncthreads();
        sums[t] += v;
        __syncthreads();
    }
    int pos = sums[t] - s;
    for (int k = b; k < e; ++k) {
        off[k] = pos;
        pos += 1 + nchunk[k];
    }
    if (t == 1023) *n_work = sums[1023];
}

__global__ void k_work_fill(const int *__restrict__ nchunk, const int *__restrict__ tile_off,
                            const int *__restrict__ off, int nb, int2 *__restrict__ work) {
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= nb) return;
    const int o = off[I], nc = nchunk[I], t0 = tile_off[I];
    if (lane == 0) work[o] = make_int2(I, -1);
    for (int c = lane; c < nc; c += 32) work[o + 1 + c] = make_int2(I, t0 + c);
}

// transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane r -> bit r of lane
// c): five butterfly stages, each swapping the off-diagonal blocks of lanes l and l ^ j
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
    const unsigned lo_masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0, j = 16; st < 5; ++st, j >>= 1) {
        const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
        const unsigned lo = lo_masks[st];
        x = (lane & j) ? ((x & ~lo) | ((y >> j) & lo)) : ((x & lo) | ((y & lo) << j));
    }
    return x;
}

// cost of staging one work item in the pair kernels, in in-range pairs: the work partition
// weighs every item as its pair count plus this (measured best of 0..256 on GB300 at 96,000
// atoms for the matvec, permanent field and force kernels together)
constexpr int ITEM_WEIGHT = 128;

// per-item in-range pair masks at the current configuration: word (item, i-lane) has bit
// j-lane set when the pair is within r_c (diagonal items: j-lane > i-lane, each pair once);
// also each item's weight for the work partition (pairs + ITEM_WEIGHT)
template <class T, bool MINIMG>
__global__ void __launch_bounds__(256) k_pairmask(const int2 *__restrict__ work, const int *__restrict__ n_work,
                                                  const typename V4<T>::type *__restrict__ posq,
                                                  const typename V4<T>::type *__restrict__ chunk_pos, T rc2, T Lx,
                                                  T Ly, T Lz, unsigned *__restrict__ pmask,
                                                  unsigned *__restrict__ pmask_t, T rs2, unsigned *__restrict__ smask,
                                                  unsigned *__restrict__ smask_t, unsigned *__restrict__ pstart,
                                                  unsigned *__restrict__ sstart, int *__restrict__ pcount,
                                                  int *__restrict__ item_cnt, int item_weight) {
    typedef typename V4<T>::type T4;
    const int lane = threadIdx.x & 31;
    const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long nitems = *n_work;
    for (long t = w; t < nitems; t += nw) {
        const int2 it = work[t];
        const T4 a = posq[it.x * 32 + lane];
        const T4 b = it.y < 0 ? posq[it.x * 32 + lane] : chunk_pos[(size_t)it.y * 32 + lane];
        T xj = b.x, yj = b.y, zj = b.z;
        unsigned m = 0u, ms = 0u;
        for (int s = 0; s < 32; ++s) {
            const int jl = (lane + s) & 31;
            T dx = a.x - xj, dy = a.y - yj, dz = a.z - zj;
            if (MINIMG) {
                dx -= Lx * rint(dx / Lx);
                dy -= Ly * rint(dy / Ly);
                dz -= Lz * rint(dz / Lz);
            }
            const T r2 = dx * dx + dy * dy + dz * dz;
            const bool in = (r2 < rc2) && (it.y >= 0 || jl > lane);
            m |= in ? (1u << jl) : 0u;
            ms |= (in && r2 < rs2) ? (1u << jl) : 0u;
            const int src = (lane + 1) & 31;
            xj = __shfl_sync(0xffffffffu, xj, src);
            yj = __shfl_sync(0xffffffffu, yj, src);
            zj = __shfl_sync(0xffffffffu, zj, src);
        }
        pmask[(size_t)t * 32 + lane] = m;
        // transposes: word of j-lane c has bit i-lane set for every pair (i, c)
        const unsigned mt = warp_transpose32(m, lane), mst = warp_transpose32(ms, lane);
        pmask_t[(size_t)t * 32 + lane] = mt;
        smask[(size_t)t * 32 + lane] = ms;
        smask_t[(size_t)t * 32 + lane] = mst;
        // where each lane's share of the sides starts, for every pair kernel of this configuration
        pstart[(size_t)t * 32 + lane] = side_start(m, mt, lane);
        sstart[(size_t)t * 32 + lane] = side_start(ms, mst, lane);
        int c = __popc(m);
        for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (lane == 0) {
            atomicAdd(pcount, c);
            item_cnt[t] = c + item_weight;
        }
    }
}

// per-item weights -> exclusive prefix in place, total at [n_work]: chunk sums, a one-block
// scan of the chunk sums, then each chunk's own scan plus its offset (all coalesced)
constexpr int SCAN_T = 256, SCAN_PER = 8, SCAN_CHUNK = SCAN_T * SCAN_PER;

__device__ __forceinline__ int block_excl_scan(int x, int &total) {
    __shared__ int wsum[SCAN_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = x;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    int base = 0;
    total = 0;
    for (int q = 0; q < SCAN_T / 32; ++q) {
        if (q < w) base += wsum[q];
        total += wsum[q];
    }
    __syncthreads();
    return base + v - x;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_chunks(const int *__restrict__ a, const int *__restrict__ n_work,
                                                        int *__restrict__ csum) {
    const int n = *n_work;
    const int c0 = blockIdx.x * SCAN_CHUNK;
    if (c0 >= n) return;   // whole block: uniform
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        const int k = c0 + r * SCAN_T + threadIdx.x;
        s += k < n ? a[k] : 0;
    }
    int total;
    block_excl_scan(s, total);
    if (threadIdx.x == 0) csum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int *__restrict__ csum, const int *__restrict__ n_work) {
    __shared__ int wsum[32];
    const int n = *n_work;
    const int nc = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int carry = 0;
    for (int c0 = 0; c0 < nc; c0 += 1024) {
        const int k = c0 + threadIdx.x;
        const int x = k < nc ? csum[k] : 0;
        int v = x;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        int base = 0, total = 0;
        for (int q = 0; q < 32; ++q) {
            if (q < w) base += wsum[q];
            total += wsum[q];
        }
        if (k < nc) csum[k] = carry + base + v - x;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) csum[nc] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(int *__restrict__ a, const int *__restrict__ n_work,
                                                       const int *__restrict__ csum) {
    const int n = *n_work;
    const int c0 = blockIdx.x * SCAN_CHUNK;
    if (blockIdx.x == 0 && threadIdx.x == 0) a[n] = csum[(n + SCAN_CHUNK - 1) / SCAN_CHUNK];
    if (c0 >= n) return;
    // thread t owns SCAN_PER consecutive items; loads are staged through shared memory so
    // that global accesses stay coalesced
    __shared__ int tile[SCAN_CHUNK];
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        const int k = c0 + r * SCAN_T + threadIdx.x;
        tile[r * SCAN_T + threadIdx.x] = k < n ? a[k] : 0;
    }
    __syncthreads();
    int v[SCAN_PER], s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        v[r] = tile[threadIdx.x * SCAN_PER + r];
        s += v[r];
    }
    int total;
    int e = block_excl_scan(s, total) + csum[blockIdx.x];
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        tile[threadIdx.x * SCAN_PER + r] = e;
        e += v[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        const int k = c0 + r * SCAN_T + threadIdx.x;
        if (k < n) a[k] = tile[r * SCAN_T + threadIdx.x];
    }
}

template <class T>
int filter_t(ap_ctx *ctx, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    const ap_params &P = ctx->prm;
    const T rc2 = (T)(P.cutoff * P.cutoff * (1.0 + 1e-5));
    const int nb = ctx->n_blocks;
    auto kern = ctx->minimg ? k_filter<T, true> : k_filter<T, false>;
    kern<<<ap_grid_for((long)nb * 32, 256), 256, 0, s>>>(
        ctx->tiles, ctx->tile_off, ctx->tshift, ctx->tile_excl, ctx->excl_mask, (const T4 *)ctx->posq,
        (const T4 *)ctx->dipd, nb, rc2, (T)P.box[0], (T)P.box[1], (T)P.box[2], ctx->tshift_lo, ctx->chunk_j,
        (T4 *)ctx->chunk_pos,
        ctx->chunk_src, ctx->chunk_mask, ctx->chunk_flag, ctx->nchunk);
    k_work_offsets<<<1, 1024, 0, s>>>(ctx->nchunk, nb, ctx->work_off, ctx->n_work);
    k_work_fill<<<ap_grid_for((long)nb * 32, 256), 256, 0, s>>>(ctx->nchunk, ctx->tile_off, ctx->work_off, nb, ctx->work);
    AP_CUDA(cudaMemsetAsync(ctx->n_work + 1, 0, sizeof(int), s));
    const T rcm = (T)(P.cutoff * P.cutoff);
    auto km = ctx->minimg ? k_pairmask<T, true> : k_pairmask<T, false>;
    km<<<ctx->sm_count * 8, 256, 0, s>>>(ctx->work, ctx->n_work, (const T4 *)ctx->posq, (const T4 *)ctx->chunk_pos, rcm,
                                         (T)P.box[0], (T)P.box[1], (T)P.box[2], ctx->pmask, ctx->pmask_t,
                                         (T)(AP_SHORT_RANGE * AP_SHORT_RANGE), ctx->smask, ctx->smask_t, ctx->pstart,
                                         ctx->sstart, ctx->n_work + 1,
                                         ctx->item_start, ITEM_WEIGHT);
    const int nchunks = (int)((ctx->cap_chunks + (long)nb + SCAN_CHUNK - 1) / SCAN_CHUNK);
    k_scan_chunks<<<nchunks, SCAN_T, 0, s>>>(ctx->item_start, ctx->n_work, ctx->scan_tmp);
    k_scan_top<<<1, 1024, 0, s>>>(ctx->scan_tmp, ctx->n_work);
    k_scan_apply<<<nchunks, SCAN_T, 0, s>>>(ctx->item_start, ctx->n_work, ctx->scan_tmp);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // namespace

int filter_launch(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? filter_t<double>(ctx, s) : filter_t<float>(ctx, s);
}

// (re)allocate the chunk arrays after a list build: capacity = block-pair tiles
int filter_alloc(ap_ctx *ctx) {
    const long cap = ctx->cap_tiles;
    if (cap <= ctx->cap_chunks) return AP_OK;
    void *ptrs[] = {ctx->chunk_j, ctx->chunk_pos, ctx->chunk_src, ctx->chunk_mask, ctx->chunk_flag, ctx->work,
                    ctx->pmask, ctx->pmask_t, ctx->smask, ctx->smask_t, ctx->pstart, ctx->sstart, ctx->item_start,
                    ctx->scan_tmp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    const size_t es = ctx->prec == AP_FP64 ? 8 : 4;
    AP_CUDA(cudaMalloc((void **)&ctx->chunk_j, sizeof(int) * 32 * cap));
    AP_CUDA(cudaMalloc((void **)&ctx->chunk_pos, 4 * es * 32 * cap));
    AP_CUDA(cudaMalloc((void **)&ctx->chunk_src, sizeof(int) * 32 * cap));
    AP_CUDA(cudaMalloc((void **)&ctx->chunk_mask, sizeof(unsigned) * 32 * cap));
    AP_CUDA(cudaMalloc((void **)&ctx->chunk_flag, sizeof(int) * cap));
    AP_CUDA(cudaMalloc((void **)&ctx->work, sizeof(int2) * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->item_start, sizeof(int) * (cap + ctx->n_blocks + 1)));
    AP_CUDA(cudaMalloc((void **)&ctx->scan_tmp, sizeof(int) * ((cap + ctx->n_blocks) / SCAN_CHUNK + 2)));
    if (!ctx->work_off) AP_CUDA(cudaMalloc((void **)&ctx->work_off, sizeof(int) * (ctx->n_blocks + 1)));
    AP_CUDA(cudaMalloc((void **)&ctx->pmask, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->pmask_t, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->smask, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->smask_t, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->pstart, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    AP_CUDA(cudaMalloc((void **)&ctx->sstart, sizeof(unsigned) * 32 * (cap + ctx->n_blocks)));
    ctx->cap_chunks = (int)cap;
    return AP_OK;
}
