// a3 / a6 - Smooth particle-mesh Ewald (paper Sec. 1.2.2, "Reciprocal space scheme": spread
// the multipolar density with order-5 B-splines, forward FFT, product with the reciprocal
// kernel, backward FFT, gather with B-spline derivatives; Fig. reci_scheme: atomics on
// the grid). FFTs are cuFFT; spread, convolution and gather are the kernels below.
//
// Conventions (shared with the oracle by definition, not by code):
//   u_a = K_a x_a / L_a, b = floor(u_a), w = u_a - b; stencil points k = (b - t) mod K_a,
//   t = 0..4, weight M_5(w + t); a site spreads (q + d.grad + (1/3) Q:grad grad) of its
//   weights, each Cartesian derivative being (K_a / L_a) d/du_a;
//   phi_grid = C2R[ B(m) C(m) R2C[Q] ] (cuFFT's unnormalised inverse);
//   C(m) = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), C(0) = 0, m aliased to [-K/2, K/2);
//   B(m) = prod_a |b_a(m_a)|^2, |b(m)|^2 = 1/|sum_{k=0}^{3} M_5(k+1) e^{2 pi i m k / K}|^2,
//   replaced by the mean of its neighbours where the sum vanishes (m = K/2).
// Grid layout: [z][y][x], x contiguous; complex half grid [z][y][x/2+1].
#include "common.cuh"

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstdint>
#include <cmath>
#include <type_traits>
#include <vector>

namespace {

template <class T>
struct Stencil {
    int k[3][5];        // grid indices per dimension
    T th[3][5];         // M_5(w + t)
    T d1[3][5];         // first u-derivative
    T d2[3][5];         // second
    T d3[3][5];         // third
};

// B-spline values of orders 2..5 at w + t, t = 0..4, by the two-term recursion
// M_n(x) = [x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)] / (n - 1), starting from M_1 = 1 on [0,1).
template <class T, int NDER>
__device__ __forceinline__ void bspline5(T w, T *th, T *d1, T *d2, T *d3) {
    T m[4][6];           // m[n-2][t+1] = M_n(w + t), with m[.][0] = M_n(w - 1) = 0
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int t = 0; t < 6; ++t) m[a][t] = T(0);
    // M_2(w + t): t = 0 -> w, t = 1 -> 1 - w
    m[0][1] = w;
    m[0][2] = T(1) - w;
#pragma unroll
    for (int n = 3; n <= 5; ++n) {
        const T inv = T(1) / T(n - 1);
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const T x = w + T(t);
            m[n - 2][t + 1] = (x * m[n - 3][t + 1] + (T(n) - x) * m[n - 3][t]) * inv;
        }
    }
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        th[t] = m[3][t + 1];
        if (NDER >= 1) d1[t] = m[2][t + 1] - m[2][t];
        if (NDER >= 2) d2[t] = m[1][t + 1] - T(2) * m[1][t] + (t >= 1 ? m[1][t - 1] : T(0));
        if (NDER >= 3)
            d3[t] = m[0][t + 1] - T(3) * m[0][t] + (t >= 1 ? T(3) * m[0][t - 1] : T(0)) -
                    (t >= 2 ? m[0][t - 2] : T(0));
    }
}

template <class T>
struct PmeConsts {
    int K[3];
    T s[3];           // K_a / L_a
    int n;
};

// stencil of one atom from its origin floor(u) mod K and fraction u - floor(u), u = K x / L
// (formed in FP64 when the configuration is loaded)
template <class T, int NDER>
__device__ __forceinline__ void make_stencil(const PmeConsts<T> &pc, int4 ib, typename V4<T>::type w,
                                             Stencil<T> &st) {
    const int ibs[3] = {ib.x, ib.y, ib.z};
    const T ws[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int K = pc.K[d];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const int k = ibs[d] - t;
            st.k[d][t] = k < 0 ? k + K : k;
        }
        bspline5<T, NDER>(ws[d], st.th[d], st.d1[d], st.d2[d], st.d3[d]);
    }
}

// adds v[t] to row[k[t]], t = 0..4, where k[t] = k[0] - t (mod K): the stencil's five points
// along x. Unless the row wraps they are contiguous, and in FP32 they take two vector atomics
// (float4 and float2 are native on sm_90 and later) for three of the four alignments of the
// first point to a 16-byte boundary and three for the fourth, instead of five scalar ones; a
// float4 may also cover the point after the stencil (adding zero) when that point is still
// inside the row of Kx points.
template <class T>
__device__ __forceinline__ void add_row5(T *row, const int *k, const T *v, int) {
#pragma unroll
    for (int t = 0; t < 5; ++t) atomicAdd(row + k[t], v[t]);
}
__device__ __forceinline__ void add_row5(float *row, const int *k, const float *v, int Kx) {
    if (k[0] >= 4) {
        float *p0 = row + (k[0] - 4);   // point t = 4; p0[j] takes v[4 - j]
        const unsigned mis = (unsigned)(reinterpret_cast<uintptr_t>(p0) & 15u) >> 2;
        if (mis == 0) {
            atomicAdd(reinterpret_cast<float4 *>(p0), make_float4(v[4], v[3], v[2], v[1]));
            atomicAdd(p0 + 4, v[0]);
        } else if (mis == 3) {
            atomicAdd(p0, v[4]);
            atomicAdd(reinterpret_cast<float4 *>(p0 + 1), make_float4(v[3], v[2], v[1], v[0]));
        } else if (mis == 2) {
            atomicAdd(reinterpret_cast<float2 *>(p0), make_float2(v[4], v[3]));
            if (k[0] + 1 < Kx) {
                atomicAdd(reinterpret_cast<float4 *>(p0 + 2), make_float4(v[2], v[1], v[0], 0.0f));
            } else {
                atomicAdd(reinterpret_cast<float2 *>(p0 + 2), make_float2(v[2], v[1]));
                atomicAdd(p0 + 4, v[0]);
            }
        } else {
            atomicAdd(p0, v[4]);
            atomicAdd(reinterpret_cast<float2 *>(p0 + 1), make_float2(v[3], v[2]));
            atomicAdd(reinterpret_cast<float2 *>(p0 + 3), make_float2(v[1], v[0]));
        }
    } else {
#pragma unroll
        for (int t = 0; t < 5; ++t) atomicAdd(row + k[t], v[t]);
    }
}

// spreads (the dipoles p, the permanent multipoles q, d, Q) ------------------------------
// adds the stencil row v[0..4] to the grid (FX: the fixed-point grid, one 64-bit atomic per point)
template <class T, bool FX>
__device__ __forceinline__ void grid_row5(void *grid, size_t row, const int *k, const T *v, int Kx) {
    if constexpr (FX) {
        unsigned long long *g = reinterpret_cast<unsigned long long *>(grid) + row;
#pragma unroll
        for (int t = 0; t < 5; ++t) atomicAdd(g + k[t], (unsigned long long)ap_to_fx(v[t]));
    } else {
        add_row5(reinterpret_cast<T *>(grid) + row, k, v, Kx);
    }
}

// fixed-point grid -> T grid for the FFT; clears the fixed-point grid for its next use
template <class T>
__global__ void k_grid_from_fx(long long *__restrict__ gfx, T *__restrict__ grid, size_t m) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    grid[i] = (T)ap_from_fx(gfx[i]);
    gfx[i] = 0;
}

// k-space product with B(m) C(m) ----------------------------------------------------------
template <class T>
__global__ void k_convolve(typename FftTypes<T>::cplx *__restrict__ c, const T *__restrict__ green, size_t m) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    T g = green[i];
    c[i].x *= g;
    c[i].y *= g;
}

// gather the field -grad(phi) at every atom ---------------------------------------------
template <class T>
__global__ void k_gather_field(const int4 *__restrict__ stb, const typename V4<T>::type *__restrict__ stw,
                               const T *__restrict__ phi, T *__restrict__ out, int n_pad, PmeConsts<T> pc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pc.n) return;
    Stencil<T> st;
    make_stencil<T, 1>(pc, stb[i], stw[i], st);
    const int Kx = pc.K[0], Ky = pc.K[1];
    T gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int t3 = 0; t3 < 5; ++t3) {
        const T z0 = st.th[2][t3], z1 = st.d1[2][t3];
#pragma unroll
        for (int t2 = 0; t2 < 5; ++t2) {
            const T y0 = st.th[1][t2], y1 = st.d1[1][t2];
            const T *row = phi + ((size_t)st.k[2][t3] * Ky + st.k[1][t2]) * Kx;
            T s0 = 0, s1 = 0;
#pragma unroll
            for (int t1 = 0; t1 < 5; ++t1) {
                const T v = row[st.k[0][t1]];
                s0 += st.th[0][t1] * v;
                s1 += st.d1[0][t1] * v;
            }
            gx += s1 * y0 * z0;
            gy += s0 * y1 * z0;
            gz += s0 * y0 * z1;
        }
    }
    out[i] = -gx * pc.s[0];
    out[n_pad + i] = -gy * pc.s[1];
    out[2 * n_pad + i] = -gz * pc.s[2];
}

// One thread per atom (the spreads of large systems, whose atoms alone fill the GPU's thread
// slots): the whole 5 x 5 x 5 stencil, 25 rows of five points.
template <class T, bool FX>
__global__ void k_spread_multipoles(const typename V4<T>::type *__restrict__ posq,
                                    const typename V4<T>::type *__restrict__ dipd,
                                    const typename V4<T>::type *__restrict__ quad0,
                                    const typename V4<T>::type *__restrict__ quad1, void *__restrict__ grid,
                                    PmeConsts<T> pc, const int4 *__restrict__ stb,
                                    const typename V4<T>::type *__restrict__ stw) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pc.n) return;
    typename V4<T>::type a = posq[i], b = dipd[i], c = quad0[i], d = quad1[i];
    Stencil<T> st;
    make_stencil<T, 2>(pc, stb[i], stw[i], st);
    const T sx = pc.s[0], sy = pc.s[1], sz = pc.s[2];
    const T q = a.w, dx = b.x * sx, dy = b.y * sy, dz = b.z * sz;
    const T third = T(1.0 / 3.0);
    const T Qxx = c.x * sx * sx * third, Qyy = c.w * sy * sy * third, Qzz = d.y * sz * sz * third;
    const T Qxy = c.y * sx * sy * T(2.0 / 3.0), Qxz = c.z * sx * sz * T(2.0 / 3.0), Qyz = d.x * sy * sz * T(2.0 / 3.0);
    const int Kx = pc.K[0], Ky = pc.K[1];
#pragma unroll
    for (int t3 = 0; t3 < 5; ++t3) {
        const T z0 = st.th[2][t3], z1 = st.d1[2][t3], z2 = st.d2[2][t3];
#pragma unroll
        for (int t2 = 0; t2 < 5; ++t2) {
            const T y0 = st.th[1][t2], y1 = st.d1[1][t2], y2 = st.d2[1][t2];
            const T A = q * y0 * z0 + dy * y1 * z0 + dz * y0 * z1 + Qyy * y2 * z0 + Qzz * y0 * z2 + Qyz * y1 * z1;
            const T Bc = dx * y0 * z0 + Qxy * y1 * z0 + Qxz * y0 * z1;
            const T Cc = Qxx * y0 * z0;
            const size_t row = ((size_t)st.k[2][t3] * Ky + st.k[1][t2]) * Kx;
            T v[5];
#pragma unroll
            for (int t1 = 0; t1 < 5; ++t1) v[t1] = st.th[0][t1] * A + st.d1[0][t1] * Bc + st.d2[0][t1] * Cc;
            grid_row5<T, FX>(grid, row, st.k[0], v, Kx);
        }
    }
}

// spread induced dipoles p --------------------------------------------------------------
template <class T, bool FX>
__global__ void k_spread_dipoles(const int4 *__restrict__ stb, const typename V4<T>::type *__restrict__ stw,
                                 const typename V4<T>::type *__restrict__ pv, void *__restrict__ grid,
                                 PmeConsts<T> pc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pc.n) return;
    typename V4<T>::type b = pv[i];
    Stencil<T> st;
    make_stencil<T, 1>(pc, stb[i], stw[i], st);
    const T px = b.x * pc.s[0], py = b.y * pc.s[1], pz = b.z * pc.s[2];
    const int Kx = pc.K[0], Ky = pc.K[1];
#pragma unroll
    for (int t3 = 0; t3 < 5; ++t3) {
        const T z0 = st.th[2][t3], z1 = st.d1[2][t3];
#pragma unroll
        for (int t2 = 0; t2 < 5; ++t2) {
            const T y0 = st.th[1][t2], y1 = st.d1[1][t2];
            const T A = py * y1 * z0 + pz * y0 * z1;
            const T Bc = px * y0 * z0;
            const size_t row = ((size_t)st.k[2][t3] * Ky + st.k[1][t2]) * Kx;
            T v[5];
#pragma unroll
            for (int t1 = 0; t1 < 5; ++t1) v[t1] = st.th[0][t1] * A + st.d1[0][t1] * Bc;
            grid_row5<T, FX>(grid, row, st.k[0], v, Kx);
        }
    }
}

// Systems of up to two waves of five threads per atom spread with five threads per atom (one
// per z-plane t3 of its stencil), a warp holding six atoms in lanes 0-29, lanes 30 and 31
// idle. One thread per atom left most of the GPU's thread slots empty (96,000 threads for
// 311,296 slots) and kept too few reductions in flight for the L2 (dipole spread 42.8 ->
// 38.4 us per launch at 96,000 atoms); at 1,065,000 atoms the slots are full either way and
// the five threads' repeated x and y stencils cost more (277 against 295 us). Each thread
// forms the x and y stencils and its own plane's z weights, and covers that plane's 25
// points.
struct Lane5 {
    int t3;        // this thread's z-plane of the stencil
    long i;        // the atom
    bool ok;       // a real atom (lanes 30, 31 and atoms past the end are not)
};
__device__ __forceinline__ Lane5 lane5(int n) {
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int a = lane / 5;
    Lane5 l;
    l.t3 = lane - 5 * a;
    l.i = warp * 6 + a;
    l.ok = lane < 30 && l.i < n;
    return l;
}

// the x and y stencils of an atom and the z weights (value and derivatives up to NDER = 1 or
// 2) and index of plane t3
template <class T, int NDER = 1>
__device__ __forceinline__ void make_stencil_plane(const PmeConsts<T> &pc, int4 ib, typename V4<T>::type w, int t3,
                                                   Stencil<T> &st, int &kz, T &z0, T &z1, T *z2 = nullptr) {
    const int ibs[2] = {ib.x, ib.y};
    const T ws[2] = {w.x, w.y};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const int K = pc.K[d];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const int k = ibs[d] - t;
            st.k[d][t] = k < 0 ? k + K : k;
        }
        bspline5<T, NDER>(ws[d], st.th[d], st.d1[d], st.d2[d], st.d3[d]);
    }
    bspline5<T, NDER>(w.z, st.th[2], st.d1[2], st.d2[2], st.d3[2]);
    z0 = st.th[2][0];
    z1 = st.d1[2][0];
    T zz = NDER >= 2 ? st.d2[2][0] : T(0);
#pragma unroll
    for (int t = 1; t < 5; ++t)
        if (t3 == t) {
            z0 = st.th[2][t];
            z1 = st.d1[2][t];
            if (NDER >= 2) zz = st.d2[2][t];
        }
    if (NDER >= 2) *z2 = zz;
    const int k = ib.z - t3;
    kz = k < 0 ? k + pc.K[2] : k;
}

template <class T, bool FX>
__global__ void k_spread_dipoles5(const int4 *__restrict__ stb, const typename V4<T>::type *__restrict__ stw,
                                  const typename V4<T>::type *__restrict__ pv, void *__restrict__ grid,
                                  PmeConsts<T> pc) {
    const Lane5 l = lane5(pc.n);
    if (!l.ok) return;
    const typename V4<T>::type b = pv[l.i];
    Stencil<T> st;
    int kz;
    T z0, z1;
    make_stencil_plane<T>(pc, stb[l.i], stw[l.i], l.t3, st, kz, z0, z1);
    const T px = b.x * pc.s[0], py = b.y * pc.s[1], pz = b.z * pc.s[2];
    const int Kx = pc.K[0], Ky = pc.K[1];
#pragma unroll
    for (int t2 = 0; t2 < 5; ++t2) {
        const T y0 = st.th[1][t2], y1 = st.d1[1][t2];
        const T A = py * y1 * z0 + pz * y0 * z1;
        const T Bc = px * y0 * z0;
        const size_t row = ((size_t)kz * Ky + st.k[1][t2]) * Kx;
        T v[5];
#pragma unroll
        for (int t1 = 0; t1 < 5; ++t1) v[t1] = st.th[0][t1] * A + st.d1[0][t1] * Bc;
        grid_row5<T, FX>(grid, row, st.k[0], v, Kx);
    }
}

template <class T, bool FX>
__global__ void k_spread_multipoles5(const typename V4<T>::type *__restrict__ posq,
                                     const typename V4<T>::type *__restrict__ dipd,
                                     const typename V4<T>::type *__restrict__ quad0,
                                     const typename V4<T>::type *__restrict__ quad1, void *__restrict__ grid,
                                     PmeConsts<T> pc, const int4 *__restrict__ stb,
                                     const typename V4<T>::type *__restrict__ stw) {
    const Lane5 l = lane5(pc.n);
    if (!l.ok) return;
    const typename V4<T>::type a = posq[l.i], b = dipd[l.i], c = quad0[l.i], d = quad1[l.i];
    Stencil<T> st;
    int kz;
    T z0, z1, z2;
    make_stencil_plane<T, 2>(pc, stb[l.i], stw[l.i], l.t3, st, kz, z0, z1, &z2);
    const T sx = pc.s[0], sy = pc.s[1], sz = pc.s[2];
    const T q = a.w, dx = b.x * sx, dy = b.y * sy, dz = b.z * sz;
    const T third = T(1.0 / 3.0);
    const T Qxx = c.x * sx * sx * third, Qyy = c.w * sy * sy * third, Qzz = d.y * sz * sz * third;
    const T Qxy = c.y * sx * sy * T(2.0 / 3.0), Qxz = c.z * sx * sz * T(2.0 / 3.0), Qyz = d.x * sy * sz * T(2.0 / 3.0);
    const int Kx = pc.K[0], Ky = pc.K[1];
#pragma unroll
    for (int t2 = 0; t2 < 5; ++t2) {
        const T y0 = st.th[1][t2], y1 = st.d1[1][t2], y2 = st.d2[1][t2];
        const T A = q * y0 * z0 + dy * y1 * z0 + dz * y0 * z1 + Qyy * y2 * z0 + Qzz * y0 * z2 + Qyz * y1 * z1;
        const T Bc = dx * y0 * z0 + Qxy * y1 * z0 + Qxz * y0 * z1;
        const T Cc = Qxx * y0 * z0;
        const size_t row = ((size_t)kz * Ky + st.k[1][t2]) * Kx;
        T v[5];
#pragma unroll
        for (int t1 = 0; t1 < 5; ++t1) v[t1] = st.th[0][t1] * A + st.d1[0][t1] * Bc + st.d2[0][t1] * Cc;
        grid_row5<T, FX>(grid, row, st.k[0], v, Kx);
    }
}

// derivatives of phi up to third order (20 components) for the forces -------------------
// component order: [0] phi; [1..3] x y z; [4..9] xx yy zz xy xz yz;
// [10..19] xxx yyy zzz xxy xxz xyy yyz xzz yzz xyz
template <class T>
__global__ void k_gather_derivs(const int4 *__restrict__ stb, const typename V4<T>::type *__restrict__ stw,
                                const T *__restrict__ phi, double *__restrict__ out, int n_pad, int ncomp,
                                PmeConsts<T> pc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pc.n) return;
    Stencil<T> st;
    make_stencil<T, 3>(pc, stb[i], stw[i], st);
    const int Kx = pc.K[0], Ky = pc.K[1];
    T D[20];
#pragma unroll
    for (int c = 0; c < 20; ++c) D[c] = 0;
#pragma unroll
    for (int t3 = 0; t3 < 5; ++t3) {
        const T z[4] = {st.th[2][t3], st.d1[2][t3], st.d2[2][t3], st.d3[2][t3]};
#pragma unroll
        for (int t2 = 0; t2 < 5; ++t2) {
            const T y[4] = {st.th[1][t2], st.d1[1][t2], st.d2[1][t2], st.d3[1][t2]};
            const T *row = phi + ((size_t)st.k[2][t3] * Ky + st.k[1][t2]) * Kx;
            T S[4] = {0, 0, 0, 0};
#pragma unroll
            for (int t1 = 0; t1 < 5; ++t1) {
                const T v = row[st.k[0][t1]];
                S[0] += st.th[0][t1] * v;
                S[1] += st.d1[0][t1] * v;
                S[2] += st.d2[0][t1] * v;
                S[3] += st.d3[0][t1] * v;
            }
            D[0] += S[0] * y[0] * z[0];
            D[1] += S[1] * y[0] * z[0];
            D[2] += S[0] * y[1] * z[0];
            D[3] += S[0] * y[0] * z[1];
            D[4] += S[2] * y[0] * z[0];
            D[5] += S[0] * y[2] * z[0];
            D[6] += S[0] * y[0] * z[2];
            D[7] += S[1] * y[1] * z[0];
            D[8] += S[1] * y[0] * z[1];
            D[9] += S[0] * y[1] * z[1];
            D[10] += S[3] * y[0] * z[0];
            D[11] += S[0] * y[3] * z[0];
            D[12] += S[0] * y[0] * z[3];
            D[13] += S[2] * y[1] * z[0];
            D[14] += S[2] * y[0] * z[1];
            D[15] += S[1] * y[2] * z[0];
            D[16] += S[0] * y[2] * z[1];
            D[17] += S[1] * y[0] * z[2];
            D[18] += S[0] * y[1] * z[2];
            D[19] += S[1] * y[1] * z[1];
        }
    }
    const T sx = pc.s[0], sy = pc.s[1], sz = pc.s[2];
    const T f[20] = {1, sx, sy, sz, sx * sx, sy * sy, sz * sz, sx * sy, sx * sz, sy * sz,
                     sx * sx * sx, sy * sy * sy, sz * sz * sz, sx * sx * sy, sx * sx * sz, sx * sy * sy,
                     sy * sy * sz, sx * sz * sz, sy * sz * sz, sx * sy * sz};
    for (int c = 0; c < ncomp; ++c) out[(size_t)c * n_pad + i] = (double)(D[c] * f[c]);
}

template <class T>
PmeConsts<T> pme_consts(const ap_ctx *ctx) {
    PmeConsts<T> pc;
    for (int d = 0; d < 3; ++d) {
        pc.K[d] = ctx->K[d];
        pc.s[d] = (T)(ctx->K[d] / ctx->prm.box[d]);
    }
    pc.n = ctx->n;
    return pc;
}

// cardinal B-spline M_n(x) on the host (for the moduli), by the same recursion
double bspline_host(int n, double x) {
    if (n == 1) return (x >= 0.0 && x < 1.0) ? 1.0 : 0.0;
    return (x * bspline_host(n - 1, x) + (n - x) * bspline_host(n - 1, x - 1.0)) / (n - 1);
}

std::vector<double> moduli(int K, int order) {
    std::vector<double> b(K);
    std::vector<char> bad(K, 0);
    for (int m = 0; m < K; ++m) {
        double re = 0, im = 0;
        for (int k = 0; k <= order - 2; ++k) {
            double v = bspline_host(order, k + 1.0);
            double arg = 2.0 * M_PI * m * k / K;
            re += v * std::cos(arg);
            im += v * std::sin(arg);
        }
        double den = re * re + im * im;
        if (den < 1e-10) bad[m] = 1; else b[m] = 1.0 / den;
    }
    for (int m = 0; m < K; ++m)
        if (bad[m]) b[m] = 0.5 * (b[(m + K - 1) % K] + b[(m + 1) % K]);
    return b;
}

template <class T>
int init_t(ap_ctx *ctx) {
    const int Kx = ctx->K[0], Ky = ctx->K[1], Kz = ctx->K[2];
    const int hx = Kx / 2 + 1;
    const ap_params &P = ctx->prm;
    std::vector<double> bx = moduli(Kx, P.pme_order), by = moduli(Ky, P.pme_order), bz = moduli(Kz, P.pme_order);
    std::vector<T> g((size_t)Kz * Ky * hx);
    const double vol = P.box[0] * P.box[1] * P.box[2];
    const double b2 = P.ewald_beta * P.ewald_beta;
    for (int iz = 0; iz < Kz; ++iz) {
        double mz = (iz <= Kz / 2 ? iz : iz - Kz) / P.box[2];
        if (2 * iz == Kz) mz = -mz;   // K/2 aliases to -K/2 (same |m|)
        for (int iy = 0; iy < Ky; ++iy) {
            double my = (iy <= Ky / 2 ? iy : iy - Ky) / P.box[1];
            for (int ix = 0; ix < hx; ++ix) {
                double mx = ix / P.box[0];
                double m2 = mx * mx + my * my + mz * mz;
                double v = 0.0;
                if (ix || iy || iz)
                    v = std::exp(-M_PI * M_PI * m2 / b2) / (M_PI * vol * m2) * bx[ix] * by[iy] * bz[iz];
                g[((size_t)iz * Ky + iy) * hx + ix] = (T)v;
            }
        }
    }
    AP_CUDA(cudaMemcpy(ctx->green, g.data(), sizeof(T) * g.size(), cudaMemcpyHostToDevice));
    bool dbl = sizeof(T) == 8;
    AP_CUFFT(cufftPlan3d(&ctx->plan_r2c, Kz, Ky, Kx, dbl ? CUFFT_D2Z : CUFFT_R2C));
    AP_CUFFT(cufftPlan3d(&ctx->plan_c2r, Kz, Ky, Kx, dbl ? CUFFT_Z2D : CUFFT_C2R));
    if (ctx->fixed) {
        AP_CUDA(cudaMalloc((void **)&ctx->grid_fx, sizeof(long long) * ctx->ngrid));
        AP_CUDA(cudaMemset(ctx->grid_fx, 0, sizeof(long long) * ctx->ngrid));
    }
    return AP_OK;
}

// the context's own grids and plans as a PmeBufs view
PmeBufs own_bufs(ap_ctx *ctx) {
    PmeBufs b;
    b.grid = ctx->grid;
    b.cgrid = ctx->cgrid;
    b.grid_fx = ctx->grid_fx;
    b.r2c = ctx->plan_r2c;
    b.c2r = ctx->plan_c2r;
    return b;
}

// launch shape of the five-threads-per-atom kernels: ceil(n / 6) warps in blocks of
// `threads` (a multiple of 32)
inline int lane5_blocks(int n, int threads) {
    const long warps = (n + 5) / 6;
    return (int)((warps * 32 + threads - 1) / threads);
}

// the field -grad(phi) of the grid phi at every atom, into out[3][n_pad]
template <class T>
int gather_launch(ap_ctx *ctx, const T *phi, T *out, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PmeConsts<T> pc = pme_consts<T>(ctx);
    const int th = ctx->tune_pme_threads;
    k_gather_field<T><<<ap_grid_for(ctx->n, th), th, 0, s>>>(ctx->stb, (const T4 *)ctx->stw, phi, out, ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int fft_roundtrip(ap_ctx *ctx, const PmeBufs &b, T *in, T *out, cudaStream_t s) {
    typedef typename FftTypes<T>::cplx C;
    AP_CUFFT(cufftSetStream(b.r2c, s));
    AP_CUFFT(cufftSetStream(b.c2r, s));
    if (sizeof(T) == 8) {
        AP_CUFFT(cufftExecD2Z(b.r2c, (cufftDoubleReal *)in, (cufftDoubleComplex *)b.cgrid));
    } else {
        AP_CUFFT(cufftExecR2C(b.r2c, (cufftReal *)in, (cufftComplex *)b.cgrid));
    }
    k_convolve<T><<<ap_grid_for((long)ctx->ncgrid, 256), 256, 0, s>>>((C *)b.cgrid, (const T *)ctx->green,
                                                                     ctx->ncgrid);
    AP_CUDA(cudaGetLastError());
    if (sizeof(T) == 8) {
        AP_CUFFT(cufftExecZ2D(b.c2r, (cufftDoubleComplex *)b.cgrid, (cufftDoubleReal *)out));
    } else {
        AP_CUFFT(cufftExecC2R(b.c2r, (cufftComplex *)b.cgrid, (cufftReal *)out));
    }
    return AP_OK;
}

// spread into ctx->grid: the induced dipoles `src` (multi = false) or the permanent
// multipoles (multi = true). Mixed/FP64 modes: FP32/T atomics on a cleared grid. AP_FIXED:
// 64-bit fixed-point atomics on ctx->grid_fx (kept cleared), then converted into the grid.
template <class T>
int spread_t(ap_ctx *ctx, const PmeBufs &bf, const void *src, bool multi, cudaStream_t s, bool cleared = false) {
    typedef typename V4<T>::type T4;
    PmeConsts<T> pc = pme_consts<T>(ctx);
    const bool fx = ctx->fixed != 0;
    void *g = fx ? (void *)bf.grid_fx : bf.grid;
    // five threads per atom while they make at most two waves of the GPU's thread slots
    const bool five = 5L * ctx->n <= 2L * 2048 * ctx->sm_count;
    if (!fx && !cleared) AP_CUDA(cudaMemsetAsync(bf.grid, 0, sizeof(T) * ctx->ngrid, s));
    if (multi) {
        if (five) {
            auto kern = fx ? k_spread_multipoles5<T, true> : k_spread_multipoles5<T, false>;
            kern<<<lane5_blocks(ctx->n, 128), 128, 0, s>>>((const T4 *)ctx->posq, (const T4 *)ctx->dipd,
                                                            (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, g, pc,
                                                            ctx->stb, (const T4 *)ctx->stw);
        } else {
            auto kern = fx ? k_spread_multipoles<T, true> : k_spread_multipoles<T, false>;
            kern<<<ap_grid_for(ctx->n, 128), 128, 0, s>>>((const T4 *)ctx->posq, (const T4 *)ctx->dipd,
                                                           (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, g, pc,
                                                           ctx->stb, (const T4 *)ctx->stw);
        }
    } else {
        const int th = ctx->tune_pme_threads;
        if (five) {
            auto kern = fx ? k_spread_dipoles5<T, true> : k_spread_dipoles5<T, false>;
            kern<<<lane5_blocks(ctx->n, th), th, 0, s>>>(ctx->stb, (const T4 *)ctx->stw, (const T4 *)src, g, pc);
        } else {
            auto kern = fx ? k_spread_dipoles<T, true> : k_spread_dipoles<T, false>;
            kern<<<ap_grid_for(ctx->n, th), th, 0, s>>>(ctx->stb, (const T4 *)ctx->stw, (const T4 *)src, g, pc);
        }
    }
    AP_CUDA(cudaGetLastError());
    if (fx) {
        k_grid_from_fx<T><<<ap_grid_for((long)ctx->ngrid, 256), 256, 0, s>>>(bf.grid_fx, (T *)bf.grid, ctx->ngrid);
        AP_CUDA(cudaGetLastError());
    }
    return AP_OK;
}

template <class T>
int multipole_field_t(ap_ctx *ctx, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PmeConsts<T> pc = pme_consts<T>(ctx);
    const PmeBufs bf = own_bufs(ctx);
    int r = spread_t<T>(ctx, bf, nullptr, true, s);
    if (r) return r;
    r = fft_roundtrip<T>(ctx, bf, (T *)ctx->grid, (T *)ctx->grid2, s);
    if (r) return r;
    return gather_launch<T>(ctx, (const T *)ctx->grid2, (T *)ctx->rec, s);
}

template <class T>
int dipole_field_t(ap_ctx *ctx, const void *p, void *rec_out, const PmeBufs &bf, cudaStream_t s, bool cleared) {
    int r = spread_t<T>(ctx, bf, p, false, s, cleared);
    if (r) return r;
    r = fft_roundtrip<T>(ctx, bf, (T *)bf.grid, (T *)bf.grid, s);
    if (r) return r;
    return gather_launch<T>(ctx, (const T *)bf.grid, (T *)rec_out, s);
}

// Structure-factor share of the virial. A homogeneous strain leaves the B-spline moduli and
// the fractional coordinates unchanged and moves only the volume and the Cartesian m of C(m),
// so the reciprocal energy's strain derivative at fixed global multipoles holds
//   f sum_m B(m) C(m) Re[S_mu conj S_M + |S_mu|^2 / 2] K(m),
//   K(m)_ab = -delta_ab + 2 (1/|m|^2 + pi^2/beta^2) m_a m_b,
// with S_X the transform of X's spread grid (the potential-derivative terms are per atom, in
// the force kernel). The permanent part is read off the permanent potential:
// R2C[phi_M] = K^3 B C S_M (unnormalised inverse). The sum runs over the half spectrum:
// points with kx = 0 or kx = Kx/2 (Kx even) stand for themselves, the others for their
// conjugate partner too, weight 2; where exactly one of the two components of an
// off-diagonal m_a m_b sits at a Nyquist index (y or z), the aliased m of the partner keeps
// that component and flips the other, so the pair's products cancel (weight 0).
// One block of 256 threads per 256 points, FP64 sums, nine atomics per block (fixed point in
// AP_FIXED: per-block sums converted and added as integers; the launch shape depends on the
// grid only, so the result is reproducible).
template <class T>
__global__ void k_virial_sf(const typename FftTypes<T>::cplx *__restrict__ Fmu,
                            const typename FftTypes<T>::cplx *__restrict__ Phi, const T *__restrict__ green,
                            int Kx, int Ky, int Kz, double iLx, double iLy, double iLz, double pib2,
                            double inv_k3, double f, size_t m, double *__restrict__ acc, int fixed) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (idx < m) {
        const int hx = Kx / 2 + 1;
        const int ix = (int)(idx % hx);
        const int iy = (int)((idx / hx) % Ky);
        const int iz = (int)(idx / ((size_t)hx * Ky));
        const int kx = ix < (Kx + 1) / 2 ? ix : ix - Kx;
        const int ky = iy < (Ky + 1) / 2 ? iy : iy - Ky;
        const int kz = iz < (Kz + 1) / 2 ? iz : iz - Kz;
        const double mv[3] = {kx * iLx, ky * iLy, kz * iLz};
        const double m2 = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
        if (m2 > 0.0) {
            const double fr = (double)Fmu[idx].x, fi = (double)Fmu[idx].y;
            double w = 0.5 * (double)green[idx] * (fr * fr + fi * fi);
            if (Phi) w += (fr * (double)Phi[idx].x + fi * (double)Phi[idx].y) * inv_k3;
            const bool edge = ix == 0 || (Kx % 2 == 0 && ix == Kx / 2);
            const double wt = edge ? 1.0 : 2.0;
            const bool nyq[3] = {Kx % 2 == 0 && ix == Kx / 2, Ky % 2 == 0 && iy == Ky / 2,
                                 Kz % 2 == 0 && iz == Kz / 2};
            const double c = 2.0 * (1.0 / m2 + pib2);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    double wab = wt;
                    if (a != b && !edge && (nyq[a] != nyq[b])) wab = 0.0;
                    v[3 * a + b] = f * wab * w * ((a == b ? -1.0 : 0.0) + c * mv[a] * mv[b]);
                }
        }
    }
    // block reduction: warps, then nine atomics
    __shared__ double sm[8][9];
    const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double x = v[k];
        for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (l == 0) sm[wp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += sm[k][threadIdx.x];
        if (fixed)
            atomicAdd(reinterpret_cast<unsigned long long *>(acc) + threadIdx.x, (unsigned long long)ap_to_fx(t));
        else
            atomicAdd(acc + threadIdx.x, t);
    }
}

// forces: phi_mu derivatives (20 comps, into gbuf[0..19]) and phi_M second derivatives
// (components 4..9, into gbuf[20..25]); the spread of mu uses ctx->p as scratch. With vir
// given, the structure-factor share of the virial is added to it between the forward
// transform and the convolution (with_M: the permanent-induced and induced-induced terms;
// otherwise the induced-induced term alone).
template <class T>
int forces_t(ap_ctx *ctx, const void *mu4, double *gbuf, int with_M, cudaStream_t s, double *vir) {
    typedef typename V4<T>::type T4;
    typedef typename FftTypes<T>::cplx C;
    PmeConsts<T> pc = pme_consts<T>(ctx);
    const PmeBufs bf = own_bufs(ctx);
    int r = spread_t<T>(ctx, bf, mu4, false, s);
    if (r) return r;
    if (!vir) {
        r = fft_roundtrip<T>(ctx, bf, (T *)ctx->grid, (T *)ctx->grid, s);
        if (r) return r;
    } else {
        const bool dbl = sizeof(T) == 8;
        AP_CUFFT(cufftSetStream(bf.r2c, s));
        AP_CUFFT(cufftSetStream(bf.c2r, s));
        if (dbl) AP_CUFFT(cufftExecD2Z(bf.r2c, (cufftDoubleReal *)ctx->grid, (cufftDoubleComplex *)ctx->cgrid));
        else AP_CUFFT(cufftExecR2C(bf.r2c, (cufftReal *)ctx->grid, (cufftComplex *)ctx->cgrid));
        if (with_M) {
            // the permanent potential, copied so that its grid stays untouched for later calls
            AP_CUDA(cudaMemcpyAsync(ctx->grid, ctx->grid2, sizeof(T) * ctx->ngrid, cudaMemcpyDeviceToDevice, s));
            if (dbl) AP_CUFFT(cufftExecD2Z(bf.r2c, (cufftDoubleReal *)ctx->grid, (cufftDoubleComplex *)ctx->cgrid_v));
            else AP_CUFFT(cufftExecR2C(bf.r2c, (cufftReal *)ctx->grid, (cufftComplex *)ctx->cgrid_v));
        }
        const ap_params &P = ctx->prm;
        const double k3 = (double)ctx->K[0] * ctx->K[1] * ctx->K[2];
        k_virial_sf<T><<<ap_grid_for((long)ctx->ncgrid, 256), 256, 0, s>>>(
            (const C *)ctx->cgrid, with_M ? (const C *)ctx->cgrid_v : nullptr, (const T *)ctx->green, ctx->K[0],
            ctx->K[1], ctx->K[2], 1.0 / P.box[0], 1.0 / P.box[1], 1.0 / P.box[2],
            M_PI * M_PI / (P.ewald_beta * P.ewald_beta), 1.0 / k3, AP_COULOMB, ctx->ncgrid, vir, ctx->fixed);
        k_convolve<T><<<ap_grid_for((long)ctx->ncgrid, 256), 256, 0, s>>>((C *)ctx->cgrid, (const T *)ctx->green,
                                                                         ctx->ncgrid);
        AP_CUDA(cudaGetLastError());
        if (dbl) AP_CUFFT(cufftExecZ2D(bf.c2r, (cufftDoubleComplex *)ctx->cgrid, (cufftDoubleReal *)ctx->grid));
        else AP_CUFFT(cufftExecC2R(bf.c2r, (cufftComplex *)ctx->cgrid, (cufftReal *)ctx->grid));
    }
    k_gather_derivs<T><<<ap_grid_for(ctx->n, 128), 128, 0, s>>>(ctx->stb, (const T4 *)ctx->stw, (const T *)ctx->grid,
                                                               gbuf, ctx->n_pad, 20, pc);
    if (with_M)
        k_gather_derivs<T><<<ap_grid_for(ctx->n, 128), 128, 0, s>>>(ctx->stb, (const T4 *)ctx->stw,
                                                                   (const T *)ctx->grid2,
                                                                   gbuf + (size_t)20 * ctx->n_pad, ctx->n_pad, 10, pc);
    else
        AP_CUDA(cudaMemsetAsync(gbuf + (size_t)20 * ctx->n_pad, 0, sizeof(double) * 10 * ctx->n_pad, s));
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// one stage alone, for timing (the spreads include the fixed-point conversion in AP_FIXED)
template <class T>
int stage_t(ap_ctx *ctx, int stage, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    typedef typename FftTypes<T>::cplx C;
    PmeConsts<T> pc = pme_consts<T>(ctx);
    switch (stage) {
    case 0:
        return spread_t<T>(ctx, own_bufs(ctx), ctx->p, false, s);
    case 1:
        k_convolve<T><<<ap_grid_for((long)ctx->ncgrid, 256), 256, 0, s>>>((C *)ctx->cgrid, (const T *)ctx->green,
                                                                         ctx->ncgrid);
        break;
    case 2:
        return gather_launch<T>(ctx, (const T *)ctx->grid, (T *)ctx->rec, s);
    case 3:
        return spread_t<T>(ctx, own_bufs(ctx), nullptr, true, s);
    case 4:
        return fft_roundtrip<T>(ctx, own_bufs(ctx), (T *)ctx->grid, (T *)ctx->grid, s);
    default:
        return ap_fail(ctx, AP_ERR_ARG, "unknown PME stage");
    }
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // namespace

int pme_stage_launch(ap_ctx *ctx, int stage, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? stage_t<double>(ctx, stage, s) : stage_t<float>(ctx, stage, s);
}

int pme_init(ap_ctx *ctx) { return ctx->prec == AP_FP64 ? init_t<double>(ctx) : init_t<float>(ctx); }

int pme_multipole_field(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? multipole_field_t<double>(ctx, s) : multipole_field_t<float>(ctx, s);
}

int pme_dipole_field(ap_ctx *ctx, const void *p, cudaStream_t s, bool grid_cleared) {
    const PmeBufs bf = own_bufs(ctx);
    return ctx->prec == AP_FP64 ? dipole_field_t<double>(ctx, p, ctx->rec, bf, s, grid_cleared)
                                : dipole_field_t<float>(ctx, p, ctx->rec, bf, s, grid_cleared);
}

int pme_dipole_field_into(ap_ctx *ctx, const void *p, void *rec_out, const PmeBufs *bufs, cudaStream_t s) {
    const PmeBufs bf = bufs ? *bufs : own_bufs(ctx);
    return ctx->prec == AP_FP64 ? dipole_field_t<double>(ctx, p, rec_out, bf, s, false)
                                : dipole_field_t<float>(ctx, p, rec_out, bf, s, false);
}

// a second set of grids and cuFFT plans of the context's sizes (for concurrent passes)
int pme_bufs_create(ap_ctx *ctx, PmeBufs *b) {
    const bool dbl = ctx->prec == AP_FP64;
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    AP_CUDA(cudaMalloc(&b->grid, es * ctx->ngrid));
    AP_CUDA(cudaMalloc(&b->cgrid, 2 * es * ctx->ncgrid));
    if (ctx->fixed) {
        AP_CUDA(cudaMalloc((void **)&b->grid_fx, sizeof(long long) * ctx->ngrid));
        AP_CUDA(cudaMemset(b->grid_fx, 0, sizeof(long long) * ctx->ngrid));
    }
    AP_CUFFT(cufftPlan3d(&b->r2c, ctx->K[2], ctx->K[1], ctx->K[0], dbl ? CUFFT_D2Z : CUFFT_R2C));
    AP_CUFFT(cufftPlan3d(&b->c2r, ctx->K[2], ctx->K[1], ctx->K[0], dbl ? CUFFT_Z2D : CUFFT_C2R));
    return AP_OK;
}

void pme_bufs_destroy(PmeBufs *b) {
    if (b->grid) cudaFree(b->grid);
    if (b->cgrid) cudaFree(b->cgrid);
    if (b->grid_fx) cudaFree(b->grid_fx);
    if (b->r2c) cufftDestroy(b->r2c);
    if (b->c2r) cufftDestroy(b->c2r);
    *b = PmeBufs();
}

int pme_forces_derivs(ap_ctx *ctx, const void *mu4, double *gbuf, cudaStream_t s, double *vir) {
    return ctx->prec == AP_FP64 ? forces_t<double>(ctx, mu4, gbuf, 1, s, vir)
                                : forces_t<float>(ctx, mu4, gbuf, 1, s, vir);
}

// the dipoles' potential derivatives only (the permanent multipoles' part left zero)
int pme_forces_derivs_mu(ap_ctx *ctx, const void *mu4, double *gbuf, cudaStream_t s, double *vir) {
    return ctx->prec == AP_FP64 ? forces_t<double>(ctx, mu4, gbuf, 0, s, vir)
                                : forces_t<float>(ctx, mu4, gbuf, 0, s, vir);
}
