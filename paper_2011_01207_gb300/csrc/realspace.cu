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

// ---------------------------------------------------------------------------------------
// a2: permanent multipole field, E_i += E(R; q_j, d_j, Q_j) and E_j += E(-R; q_i, d_i, Q_i)
template <class T, bool MINIMG>
__global__ void __launch_bounds__(256) k_perm_field(
    const int2 *__restrict__ tiles, const float4 *__restrict__ tshift, const int *__restrict__ tile_excl,
    const unsigned *__restrict__ masks, int ntiles, const typename V4<T>::type *__restrict__ posq,
    const typename V4<T>::type *__restrict__ dipd, const typename V4<T>::type *__restrict__ quad0,
    const typename V4<T>::type *__restrict__ quad1, double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    const int lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long t0 = ntiles * gw / nw, t1 = ntiles * (gw + 1) / nw;
    int curI = -1;
    double ax = 0, ay = 0, az = 0;
    T xi = 0, yi = 0, zi = 0, qi = 0, dix = 0, diy = 0, diz = 0, ti = 0;
    T qxx = 0, qxy = 0, qxz = 0, qyy = 0, qyz = 0, qzz = 0;
    for (long t = t0; t < t1; ++t) {
        const int2 IJ = tiles[t];
        if (IJ.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
            ax = ay = az = 0;
            curI = IJ.x;
            const int si = curI * 32 + lane;
            T4 a = posq[si], b = dipd[si], c = quad0[si], d = quad1[si];
            xi = a.x; yi = a.y; zi = a.z; qi = a.w;
            dix = b.x; diy = b.y; diz = b.z; ti = b.w;
            qxx = c.x; qxy = c.y; qxz = c.z; qyy = c.w; qyz = d.x; qzz = d.y;
        }
        const int sj = IJ.y * 32 + lane;
        T4 a = posq[sj], b = dipd[sj], c = quad0[sj], d = quad1[sj];
        T xj = a.x, yj = a.y, zj = a.z, qj = a.w, djx = b.x, djy = b.y, djz = b.z, tj = b.w;
        T pxx = c.x, pxy = c.y, pxz = c.z, pyy = c.w, pyz = d.x, pzz = d.y;
        T sx = 0, sy = 0, sz = 0;
        if (!MINIMG) {
            float4 sh = tshift[t];
            sx = sh.x; sy = sh.y; sz = sh.z;
        }
        const int slot = tile_excl[t];
        const unsigned mask = slot >= 0 ? masks[slot * 32 + lane] : 0u;
        const bool diag = IJ.x == IJ.y;
        T fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll 2
        for (int s = 0; s < 32; ++s) {
            const int jl = (lane + s) & 31;
            if (!(diag && s == 0)) {
                T dx, dy, dz;
                pair_vector<T, MINIMG>(pc, xi, yi, zi, xj, yj, zj, sx, sy, sz, dx, dy, dz);
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
                    T q2 = T(2.0 / 3.0) * R2;
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
        if (!diag && sj < pc.n) flush3(acc, n_pad, sj, (double)gx, (double)gy, (double)gz);
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
}

// ---------------------------------------------------------------------------------------
// a5: dipole-field matrix-vector product, E_i += -R1 p_j + R2 (p_j.R) R (and i <-> j)
template <class T, bool MINIMG>
__global__ void __launch_bounds__(256) k_matvec(
    const int2 *__restrict__ tiles, const float4 *__restrict__ tshift, int ntiles,
    const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ pv, double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    const int lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long t0 = ntiles * gw / nw, t1 = ntiles * (gw + 1) / nw;
    int curI = -1;
    double ax = 0, ay = 0, az = 0;
    T xi = 0, yi = 0, zi = 0, ti = 0, pix = 0, piy = 0, piz = 0;
    for (long t = t0; t < t1; ++t) {
        const int2 IJ = tiles[t];
        if (IJ.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3(acc, n_pad, curI * 32 + lane, ax, ay, az);
            ax = ay = az = 0;
            curI = IJ.x;
            const int si = curI * 32 + lane;
            T4 a = posq[si], b = pv[si];
            xi = a.x; yi = a.y; zi = a.z; ti = dipd[si].w;
            pix = b.x; piy = b.y; piz = b.z;
        }
        const int sj = IJ.y * 32 + lane;
        T4 a = posq[sj], b = pv[sj];
        T xj = a.x, yj = a.y, zj = a.z, tj = dipd[sj].w, pjx = b.x, pjy = b.y, pjz = b.z;
        T sx = 0, sy = 0, sz = 0;
        if (!MINIMG) {
            float4 sh = tshift[t];
            sx = sh.x; sy = sh.y; sz = sh.z;
        }
        const bool diag = IJ.x == IJ.y;
        T fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll 4
        for (int s = 0; s < 32; ++s) {
            if (!(diag && s == 0)) {
                T dx, dy, dz;
                pair_vector<T, MINIMG>(pc, xi, yi, zi, xj, yj, zj, sx, sy, sz, dx, dy, dz);
                const T r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < pc.rc2) {
                    const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
                    T B[2], U[2], oml[2];
                    screened<T, 2>(pc, r, rinv, rinv2, B, U);
                    thole_oml<T, 2>(pc.thole_a * r2 * r * ti * tj, oml);
                    const T R1 = B[0] - oml[0] * U[0];
                    const T R2 = B[1] - oml[1] * U[1];
                    T pr = (pjx * dx + pjy * dy + pjz * dz) * R2;
                    fx += pr * dx - R1 * pjx;
                    fy += pr * dy - R1 * pjy;
                    fz += pr * dz - R1 * pjz;
                    pr = (pix * dx + piy * dy + piz * dz) * R2;
                    gx += pr * dx - R1 * pix;
                    gy += pr * dy - R1 * piy;
                    gz += pr * dz - R1 * piz;
                }
            }
            const int src = (lane + 1) & 31;
            xj = shfl1(xj, src); yj = shfl1(yj, src); zj = shfl1(zj, src); tj = shfl1(tj, src);
            pjx = shfl1(pjx, src); pjy = shfl1(pjy, src); pjz = shfl1(pjz, src);
            gx = shfl1(gx, src); gy = shfl1(gy, src); gz = shfl1(gz, src);
        }
        ax += (double)fx; ay += (double)fy; az += (double)fz;
        if (!diag && sj < pc.n) flush3(acc, n_pad, sj, (double)gx, (double)gy, (double)gz);
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
    kern<<<grid, 256, 0, s>>>(ctx->tiles, ctx->tshift, ctx->tile_excl, ctx->excl_mask, ctx->n_tiles,
                              (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)ctx->quad0,
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
    int &grid = grids[ctx->minimg];
    if (!grid) grid = resident_grid(ctx, kern, 256);
    kern<<<grid, 256, 0, s>>>(ctx->tiles, ctx->tshift, ctx->n_tiles, (const T4 *)ctx->posq,
                              (const T4 *)ctx->dipd, (const T4 *)p, ctx->acc, ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // namespace

int real_field_launch(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? perm_field_t<double>(ctx, s) : perm_field_t<float>(ctx, s);
}

int real_matvec_launch(ap_ctx *ctx, const void *p, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? matvec_t<double>(ctx, p, s) : matvec_t<float>(ctx, p, s);
}
