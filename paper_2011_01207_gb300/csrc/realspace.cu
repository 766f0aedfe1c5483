// a2 / a5 - Real-space pair kernels over 32 x 32 atom tiles (paper Sec. 2.3, Fig. groups_inte:
// a group of B_size atoms against another, B_size^2 interactions with the j data read
// from neighbouring lanes by warp intrinsics instead of global memory).
//
// One warp owns a contiguous run of tiles (block pairs I <= J, sorted by I). Lane l holds
// atom l of block I in registers; the 32 atoms of block J start one per lane and rotate
// one lane per step (__shfl_sync), so after 32 steps every (i, j) pair has met once and
// the j-side partial sums are back in their own lanes. Diagonal tiles (I == J) visit each
// ordered pair and add only to i. Pair arithmetic is in T (FP32 in the mixed mode); a
// tile row's 32 terms are summed in T, then added in FP64 - across a warp's tiles of the
// same I in registers, and into the global FP64 accumulators with atomics.
#include "common.cuh"
#include "pair_math.cuh"

#include <algorithm>
#include <cmath>

namespace {

template <class T, bool MINIMG>
__device__ __forceinline__ void pair_vector(const PairConsts<T> &pc, T xi, T yi, T zi, T xj, T yj, T zj,
                                            T sx, T sy, T sz, T &dx, T &dy, T &dz) {
    dx = xi - xj;
    dy = yi - yj;
    dz = zi - zj;
    if (MINIMG) {
        dx -= pc.L[0] * ap_rint(dx * pc.iL[0]);
        dy -= pc.L[1] * ap_rint(dy * pc.iL[1]);
        dz -= pc.L[2] * ap_rint(dz * pc.iL[2]);
    } else {
        dx += sx;
        dy += sy;
        dz += sz;
    }
}

__device__ __forceinline__ void flush3(double *acc, int n_pad, int slot, double a, double b, double c) {
    atomicAdd(acc + slot, a);
    atomicAdd(acc + n_pad + slot, b);
    atomicAdd(acc + 2 * n_pad + slot, c);
}

template <class T>
__device__ __forceinline__ T shfl1(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Work items come from the per-configuration filter: (I, -1) is block I against itself,
// (I, c) is block I against filtered chunk c (32 atoms of partner blocks, positions already
// in the periodic image next to I, padding = NaN phantoms). Items are sorted by I, so a
// warp keeps block I's i-side sums in FP64 registers across consecutive items.

// ---------------------------------------------------------------------------------------
// a2: permanent multipole field, E_i += E(R; q_j, d_j, Q_j) and E_j += E(-R; q_i, d_i, Q_i)
template <class T, bool MINIMG>
__global__ void __launch_bounds__(256) k_perm_field(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ quad0, const typename V4<T>::type *__restrict__ quad1,
    double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    const int lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long nitems = *wa.n_work;
    const long t0 = nitems * gw / nw, t1 = nitems * (gw + 1) / nw;
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    int curI = -1;
    double ax = 0, ay = 0, az = 0;
    T xi = 0, yi = 0, zi = 0, qi = 0, dix = 0, diy = 0, diz = 0, ti = 0;
    T qxx = 0, qxy = 0, qxz = 0, qyy = 0, qyz = 0, qzz = 0;
    for (long t = t0; t < t1; ++t) {
        const int2 it = wa.work[t];
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
            ax = ay = az = 0;
            curI = it.x;
            const int si = curI * 32 + lane;
            T4 a = posq[si], b = dipd[si], c = quad0[si], d = quad1[si];
            xi = a.x; yi = a.y; zi = a.z; qi = a.w;
            dix = b.x; diy = b.y; diz = b.z; ti = b.w;
            qxx = c.x; qxy = c.y; qxz = c.z; qyy = c.w; qyz = d.x; qzz = d.y;
        }
        const bool diag = it.y < 0;
        int sj;
        T xj, yj, zj, tj;
        unsigned mask;
        if (diag) {
            sj = curI * 32 + lane;
            const T4 a = posq[sj];
            xj = a.x; yj = a.y; zj = a.z; tj = ti;
            const int e = wa.tile_excl[wa.tile_off[curI]];
            mask = e >= 0 ? wa.excl_mask[(size_t)e * 32 + lane] : 0u;
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            const T4 a = cpos[cs];
            xj = a.x; yj = a.y; zj = a.z; tj = a.w;
            mask = wa.chunk_flag[it.y] ? wa.chunk_mask[cs] : 0u;
        }
        T qj = 0, djx = 0, djy = 0, djz = 0, pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
        if (sj >= 0) {
            const T4 a = posq[sj], b = dipd[sj], c = quad0[sj], d = quad1[sj];
            qj = a.w; djx = b.x; djy = b.y; djz = b.z;
            pxx = c.x; pxy = c.y; pxz = c.z; pyy = c.w; pyz = d.x; pzz = d.y;
        }
        T fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll 2
        for (int s = 0; s < 32; ++s) {
            const int jl = (lane + s) & 31;
            if (!(diag && s == 0)) {
                T dx, dy, dz;
                pair_vector<T, MINIMG>(pc, xi, yi, zi, xj, yj, zj, T(0), T(0), T(0), dx, dy, dz);
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < pc.rc2) {
                    const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
                    T B[3], U[3], oml[3];
                    screened<T, 3>(pc, r, rinv, rinv2, B, U);
                    thole_oml<T, 3>(pc.thole_a * r2 * r * ti * tj, oml);
                    const bool ex = (mask >> jl) & 1u;
                    const T R1 = B[0] - (ex ? U[0] : oml[0] * U[0]);
                    const T R2 = B[1] - (ex ? U[1] : oml[1] * U[1]);
                    const T R3 = B[2] - (ex ? U[2] : oml[2] * U[2]);
                    // field at i from site j
                    T dR = djx * dx + djy * dy + djz * dz;
                    T Qx = pxx * dx + pxy * dy + pxz * dz;
                    T Qy = pxy * dx + pyy * dy + pyz * dz;
                    T Qz = pxz * dx + pyz * dy + pzz * dz;
                    T RQR = Qx * dx + Qy * dy + Qz * dz;
                    T fac = qj * R1 + dR * R2 + RQR * R3 * T(1.0 / 3.0);
                    const T q2 = T(2.0 / 3.0) * R2;
                    fx += fac * dx - R1 * djx - q2 * Qx;
                    fy += fac * dy - R1 * djy - q2 * Qy;
                    fz += fac * dz - R1 * djz - q2 * Qz;
                    if (!diag) {
                        // field at j from site i (R -> -R)
                        dR = dix * dx + diy * dy + diz * dz;
                        Qx = qxx * dx + qxy * dy + qxz * dz;
                        Qy = qxy * dx + qyy * dy + qyz * dz;
                        Qz = qxz * dx + qyz * dy + qzz * dz;
                        RQR = Qx * dx + Qy * dy + Qz * dz;
                        fac = qi * R1 - dR * R2 + RQR * R3 * T(1.0 / 3.0);
                        gx += -fac * dx - R1 * dix + q2 * Qx;
                        gy += -fac * dy - R1 * diy + q2 * Qy;
                        gz += -fac * dz - R1 * diz + q2 * Qz;
                    }
                }
            }
            const int src = (lane + 1) & 31;
            xj = shfl1(xj, src); yj = shfl1(yj, src); zj = shfl1(zj, src); qj = shfl1(qj, src);
            djx = shfl1(djx, src); djy = shfl1(djy, src); djz = shfl1(djz, src); tj = shfl1(tj, src);
            pxx = shfl1(pxx, src); pxy = shfl1(pxy, src); pxz = shfl1(pxz, src);
            pyy = shfl1(pyy, src); pyz = shfl1(pyz, src); pzz = shfl1(pzz, src);
            gx = shfl1(gx, src); gy = shfl1(gy, src); gz = shfl1(gz, src);
        }
        ax += (double)fx; ay += (double)fy; az += (double)fz;
        if (!diag && sj >= 0) flush3(acc, n_pad, sj, (double)gx, (double)gy, (double)gz);
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
}

// ---------------------------------------------------------------------------------------
// a5: dipole-field matrix-vector product, E_i += -R1 p_j + R2 (p_j.R) R (and i <-> j).
// Positions are fixed during a solve, so the in-range pairs of every work item and their
// transposed bit matrix were found once per configuration. Per item, a warp stages the
// 32 i-atoms and 32 j-atoms in shared memory and writes a queue of "pair sides"
// (target atom, source atom): the row bits give the field at each i-atom, the column bits
// the field at each j-atom. The queue is sorted by target, and each lane takes an equal
// contiguous slice of it, accumulating in registers while the target stays the same and
// adding to a shared per-target sum only when it changes (a few times per lane per item).
// So every lane evaluates one in-range pair side per step, whatever the pair distribution;
// the field expression is even in R, so one code path serves both sides.
template <class T>
struct MvSmem {
    typename V4<T>::type pos[64];    // x, y, z, Thole factor: [0,32) block I, [32,64) the item's j atoms
    typename V4<T>::type p[64];      // dipoles of the same atoms
    T acc[3][64];                    // per-target sums of the item
    unsigned short queue[2048];      // (target << 5) | source-lane, sorted by target
};

template <class T, bool MINIMG, bool SHORT = false>
__global__ void __launch_bounds__(128) k_matvec(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ pv, double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    __shared__ MvSmem<T> smem[4];
    MvSmem<T> &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long nitems = *wa.n_work;
    const long t0 = nitems * gw / nw, t1 = nitems * (gw + 1) / nw;
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    int curI = -1;
    double ax = 0, ay = 0, az = 0;
    for (long t = t0; t < t1; ++t) {
        const int2 it = wa.work[t];
        __syncwarp();   // every lane is done with the previous item's staging
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
            ax = ay = az = 0;
            curI = it.x;
            const int si = curI * 32 + lane;
            T4 a = posq[si];
            a.w = dipd[si].w;
            S.pos[lane] = a;
            S.p[lane] = pv[si];
        }
        const bool diag = it.y < 0;
        int sj = -1;
        if (diag) {
            S.pos[32 + lane] = S.pos[lane];
            S.p[32 + lane] = S.p[lane];
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            S.pos[32 + lane] = cpos[cs];
            T4 z;
            z.x = z.y = z.z = z.w = T(0);
            S.p[32 + lane] = sj >= 0 ? pv[sj] : z;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.acc[c][lane] = T(0);
            S.acc[c][32 + lane] = T(0);
        }
        // queue: row sides (target i-lane, source j-lane), then column sides (target 32 + j-lane)
        unsigned row = SHORT ? wa.smask[(size_t)t * 32 + lane] : wa.pmask[(size_t)t * 32 + lane];
        unsigned col = SHORT ? wa.smask_t[(size_t)t * 32 + lane] : wa.pmask_t[(size_t)t * 32 + lane];
        const int nr = __popc(row), nc = __popc(col);
        int ir = nr, ic = nc;
        for (int off = 1; off < 32; off <<= 1) {
            const int vr = __shfl_up_sync(0xffffffffu, ir, off);
            const int vc = __shfl_up_sync(0xffffffffu, ic, off);
            if (lane >= off) { ir += vr; ic += vc; }
        }
        const int prow = __shfl_sync(0xffffffffu, ir, 31);
        const int total = prow + __shfl_sync(0xffffffffu, ic, 31);
        int pos = ir - nr;
        while (row) {
            const int b = __ffs(row) - 1;
            row &= row - 1u;
            S.queue[pos++] = (unsigned short)((lane << 5) | b);
        }
        pos = prow + ic - nc;
        while (col) {
            const int b = __ffs(col) - 1;
            col &= col - 1u;
            S.queue[pos++] = (unsigned short)(((32 + lane) << 5) | b);
        }
        __syncwarp();
        const int per = (total + 31) >> 5;
        const int e0 = lane * per, e1 = min(total, e0 + per);
        int cur = -1;
        T4 self;
        self.x = self.y = self.z = self.w = T(0);
        T f0 = 0, f1 = 0, f2 = 0;
        for (int e = e0; e < e1; ++e) {
            const int q = S.queue[e];
            const int tg = q >> 5;
            if (tg != cur) {
                if (cur >= 0) {
                    atomicAdd(&S.acc[0][cur], f0);
                    atomicAdd(&S.acc[1][cur], f1);
                    atomicAdd(&S.acc[2][cur], f2);
                }
                f0 = f1 = f2 = T(0);
                cur = tg;
                self = S.pos[tg];
            }
            const int src = (q & 31) + (tg < 32 ? 32 : 0);   // a row side's source is a j atom
            const T4 other = S.pos[src], po = S.p[src];
            T dx, dy, dz;
            pair_vector<T, MINIMG>(pc, self.x, self.y, self.z, other.x, other.y, other.z, T(0), T(0), T(0), dx, dy, dz);
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
            T B[2], U[2], oml[2];
            screened<T, 2>(pc, r, rinv, rinv2, B, U);
            thole_oml<T, 2>(pc.thole_a * r2 * r * self.w * other.w, oml);
            const T R1 = B[0] - oml[0] * U[0];
            const T R2 = B[1] - oml[1] * U[1];
            const T pr = (po.x * dx + po.y * dy + po.z * dz) * R2;
            f0 += pr * dx - R1 * po.x;
            f1 += pr * dy - R1 * po.y;
            f2 += pr * dz - R1 * po.z;
        }
        if (cur >= 0) {
            atomicAdd(&S.acc[0][cur], f0);
            atomicAdd(&S.acc[1][cur], f1);
            atomicAdd(&S.acc[2][cur], f2);
        }
        __syncwarp();
        ax += (double)S.acc[0][lane];
        ay += (double)S.acc[1][lane];
        az += (double)S.acc[2][lane];
        if (diag) {
            ax += (double)S.acc[0][32 + lane];
            ay += (double)S.acc[1][32 + lane];
            az += (double)S.acc[2][32 + lane];
        } else if (sj >= 0) {
            flush3(acc, n_pad, sj, (double)S.acc[0][32 + lane], (double)S.acc[1][32 + lane],
                   (double)S.acc[2][32 + lane]);
        }
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
}

template <class T>
PairConsts<T> make_consts(const ap_ctx *ctx) {
    PairConsts<T> pc;
    const ap_params &P = ctx->prm;
    double b = P.ewald_beta;
    pc.beta = (T)b;
    pc.c[0] = 0;
    for (int k = 1; k <= 4; ++k) pc.c[k] = (T)(std::pow(2.0 * b * b, k) / (b * AP_SQRT_PI));
    pc.thole_a = (T)P.thole_a;
    pc.rc2 = (T)(P.cutoff * P.cutoff);
    for (int d = 0; d < 3; ++d) {
        pc.L[d] = (T)P.box[d];
        pc.iL[d] = (T)(1.0 / P.box[d]);
    }
    pc.n = ctx->n;
    return pc;
}


template <class K>
int resident_grid(ap_ctx *ctx, K kernel, int threads) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return std::max(1, per_sm) * ctx->sm_count;
}

template <class T>
int perm_field_t(ap_ctx *ctx, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->minimg ? k_perm_field<T, true> : k_perm_field<T, false>;
    static int grids[2] = {0, 0};
    int &grid = grids[ctx->minimg];
    if (!grid) grid = resident_grid(ctx, kern, 256);
    kern<<<grid, 256, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)ctx->quad0,
                              (const T4 *)ctx->quad1, ctx->acc, ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int matvec_t(ap_ctx *ctx, const void *p, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->minimg ? k_matvec<T, true> : k_matvec<T, false>;
    static int grids[2] = {0, 0};
    int &g0 = grids[ctx->minimg];
    if (!g0) g0 = resident_grid(ctx, kern, 128);
    const int grid = std::max(ctx->sm_count, g0 / std::max(1, ctx->tune_mv_div));
    kern<<<grid, 128, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)p, ctx->acc,
                              ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int short_t(ap_ctx *ctx, const void *p, double *out, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->minimg ? k_matvec<T, true, true> : k_matvec<T, false, true>;
    static int grids[2] = {0, 0};
    int &grid = grids[ctx->minimg];
    if (!grid) grid = resident_grid(ctx, kern, 128);
    kern<<<grid, 128, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)p, out,
                              ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // namespace

int short_matvec_launch(ap_ctx *ctx, const void *p, double *out, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? short_t<double>(ctx, p, out, s) : short_t<float>(ctx, p, out, s);
}

int real_field_launch(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? perm_field_t<double>(ctx, s) : perm_field_t<float>(ctx, s);
}

int real_matvec_launch(ap_ctx *ctx, const void *p, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? matvec_t<double>(ctx, p, s) : matvec_t<float>(ctx, p, s);
}
