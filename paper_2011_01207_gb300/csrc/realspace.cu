// a2 / a5 - Real-space pair kernels over 32-atom groups (paper Sec. 2.3: a group of B_size
// atoms against another, B_size^2 interactions, with the paper's group-to-atom list
// filtering).
//
// A work item is block I against one filtered 32-atom chunk of its partner blocks (or
// against itself). The in-range pairs of every item are known as 32-bit masks (row and
// transposed) from the per-configuration filter. A warp stages the item's 64 atoms in
// shared memory; the masks' bits are its pair sides (target, source), which in word order
// are sorted by target; each lane walks an equal contiguous share of them in place, so no
// lane evaluates an out-of-range pair and the work per lane is even whatever the pair
// distribution. Pair
// arithmetic is in T (FP32 in the mixed mode); sums per target are kept in T within an
// item (registers, then a shared per-target slot), and in FP64 across items: block I's in
// registers while consecutive items share I, the chunk atoms' with FP64 atomics.
#include "common.cuh"
#include "pair_math.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace {

// running sums of block I's atom `slot` (three components) to the global accumulators
template <class PA>
__device__ __forceinline__ void flush3(double *acc, int n_pad, int slot, const typename PA::run_t &a,
                                       const typename PA::run_t &b, const typename PA::run_t &c) {
    PA::run_flush(acc + slot, a);
    PA::run_flush(acc + n_pad + slot, b);
    PA::run_flush(acc + 2 * n_pad + slot, c);
}
// one item's sums of a chunk atom: components c0, c0 + 1, c0 + 2 of the item's target 32 + lane
template <class PA, class S>
__device__ __forceinline__ void flush3_item(double *acc, int n_pad, int slot, const S &sm, int c0, int lane) {
    PA::item_flush(acc + slot, sm.acc[c0][32 + lane]);
    PA::item_flush(acc + n_pad + slot, sm.acc[c0 + 1][32 + lane]);
    PA::item_flush(acc + 2 * n_pad + slot, sm.acc[c0 + 2][32 + lane]);
}

// Work items come from the per-configuration filter: (I, -1) is block I against itself,
// (I, c) is block I against filtered chunk c (32 atoms of partner blocks, positions already
// in the periodic image next to I, padding = NaN phantoms). Items are sorted by I, so a
// warp keeps block I's i-side sums in FP64 registers across consecutive items.

// ---------------------------------------------------------------------------------------
// a2: permanent multipole field, E_i += E(R; q_j, d_j, Q_j) and E_j += E(-R; q_i, d_i, Q_i).
// Same pair sides as the matvec below: every in-range pair gives the side "field at
// the target from the source's multipole" for both atoms, and with R = x_target - x_source
// one expression serves both sides. The exclusion bit of the pair (sigma = 0 in R_n) is
// looked up in the item's 32-word mask.
template <class T, class A>
struct PfSmem {
    typename V4<T>::type pos[64];   // x, y, z, Thole factor: [0,32) block I, [32,64) the item's j atoms
    typename V4<T>::type qd[64];    // charge, dipole
    typename V4<T>::type qa[64];    // Qxx, Qxy, Qxz, Qyy
    T qb[2][64];                    // Qyz, Qzz
    A acc[3][64];                   // per-target sums of the item
    unsigned ex[32];                // exclusion words: lane i, bit j
    unsigned words[64];             // pair bits: rows of the i atoms, then columns of the j atoms
};

// One side of the permanent field: the field at the target of the source's (q, d, Q), with
// R = x_target - x_source and the pair's exclusion bit (sigma = 0 in R_n)
template <class T>
__device__ __forceinline__ void pf_contract(T R1, T R2, T R3, T dx, T dy, T dz, const typename V4<T>::type &m,
                                            const typename V4<T>::type &qa, T qyz, T qzz, T &g0, T &g1, T &g2) {
    const T dR = m.y * dx + m.z * dy + m.w * dz;
    const T Qx = qa.x * dx + qa.y * dy + qa.z * dz;
    const T Qy = qa.y * dx + qa.w * dy + qyz * dz;
    const T Qz = qa.z * dx + qyz * dy + qzz * dz;
    const T RQR = Qx * dx + Qy * dy + Qz * dz;
    const T fac = m.x * R1 + dR * R2 + RQR * R3 * T(1.0 / 3.0);
    const T q2 = T(2.0 / 3.0) * R2;
    g0 = fac * dx - R1 * m.y - q2 * Qx;
    g1 = fac * dy - R1 * m.z - q2 * Qy;
    g2 = fac * dz - R1 * m.w - q2 * Qz;
}

template <class T, bool MINIMG, class SM>
__device__ __forceinline__ void pf_side(SM &S, const PairConsts<T> &pc, const typename V4<T>::type &self, int tg,
                                        int src, T &g0, T &g1, T &g2) {
    typedef typename V4<T>::type T4;
    const int sl = src & 31;   // the source's lane within its half
    const bool exb = tg < 32 ? (S.ex[tg] >> sl) & 1u : (S.ex[sl] >> (tg - 32)) & 1u;
    const T4 o = S.pos[src], m = S.qd[src], qa = S.qa[src];
    const T qyz = S.qb[0][src], qzz = S.qb[1][src];
    T dx, dy, dz;
    pair_vector<T, MINIMG>(pc, self.x, self.y, self.z, o.x, o.y, o.z, T(0), T(0), T(0), dx, dy, dz);
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
    T B[3], U[3], oml[3];
    screened<T, 3>(pc, r, rinv, rinv2, B, U);
    thole_oml<T, 3>(pc.thole_a * r2 * r * self.w * o.w, oml);
    const T R1 = B[0] - (exb ? U[0] : oml[0] * U[0]);
    const T R2 = B[1] - (exb ? U[1] : oml[1] * U[1]);
    const T R3 = B[2] - (exb ? U[2] : oml[2] * U[2]);
    pf_contract<T>(R1, R2, R3, dx, dy, dz, m, qa, qyz, qzz, g0, g1, g2);
}

// the walk over a lane's share of the item's sides, as matvec_walk (plain stores on leaving a
// target, atomics for the last one)
template <class T, bool MINIMG, class PA, class SM>
__device__ __forceinline__ void pf_walk(SM &S, SideSlice &slice, const PairConsts<T> &pc) {
    typedef typename V4<T>::type T4;
    int cur = -1;
    T4 self;
    self.x = self.y = self.z = self.w = T(0);
    T f0 = 0, f1 = 0, f2 = 0;
    while (slice.left > 0) {
        int tg, src;
        slice.next(S.words, tg, src);
        if (tg != cur) {
            if (cur >= 0) {
                PA::shared_put(&S.acc[0][cur], f0);
                PA::shared_put(&S.acc[1][cur], f1);
                PA::shared_put(&S.acc[2][cur], f2);
            }
            f0 = f1 = f2 = T(0);
            cur = tg;
            self = S.pos[tg];
        }
        T g0, g1, g2;
        pf_side<T, MINIMG>(S, pc, self, tg, src, g0, g1, g2);
        f0 += g0;
        f1 += g1;
        f2 += g2;
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
        PA::shared_add(&S.acc[0][cur], f0);
        PA::shared_add(&S.acc[1][cur], f1);
        PA::shared_add(&S.acc[2][cur], f2);
    }
}

// FP32: two consecutive sides per step, their R_1..R_3 in packed f32x2 arithmetic
// (radial123_x2), the multipole contractions per side; an odd last side takes the scalar path
template <bool MINIMG, class PA, class SM>
__device__ __forceinline__ void pf_walk_x2(SM &S, SideSlice &slice, const PairConsts<float> &pc,
                                           const PairConsts2 &k) {
    int cur = -1;
    float4 self = make_float4(0.f, 0.f, 0.f, 0.f);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    auto leave = [&](int next, const float4 &nself) {
        if (cur >= 0) {
            PA::shared_put(&S.acc[0][cur], f0);
            PA::shared_put(&S.acc[1][cur], f1);
            PA::shared_put(&S.acc[2][cur], f2);
        }
        cur = next;
        self = nself;
    };
    while (slice.left > 1) {
        int ta, sa, tb, sb;
        slice.next(S.words, ta, sa);
        slice.next(S.words, tb, sb);
        if (ta != cur) {
            leave(ta, S.pos[ta]);
            f0 = f1 = f2 = 0.f;
        }
        const float4 selfb = tb == ta ? self : S.pos[tb];
        const int la = sa & 31, lb = sb & 31;
        const bool exa = ta < 32 ? (S.ex[ta] >> la) & 1u : (S.ex[la] >> (ta - 32)) & 1u;
        const bool exb = tb < 32 ? (S.ex[tb] >> lb) & 1u : (S.ex[lb] >> (tb - 32)) & 1u;
        const float4 oa = S.pos[sa], ob = S.pos[sb];
        float dxa, dya, dza, dxb, dyb, dzb;
        pair_vector<float, MINIMG>(pc, self.x, self.y, self.z, oa.x, oa.y, oa.z, 0.f, 0.f, 0.f, dxa, dya, dza);
        pair_vector<float, MINIMG>(pc, selfb.x, selfb.y, selfb.z, ob.x, ob.y, ob.z, 0.f, 0.f, 0.f, dxb, dyb, dzb);
        const float2 dx = make_float2(dxa, dxb), dy = make_float2(dya, dyb), dz = make_float2(dza, dzb);
        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float2 R1, R2, R3;
        radial123_x2(k, r2, make_float2(self.w * oa.w, selfb.w * ob.w), exa, exb, R1, R2, R3);
        float g0, g1, g2;
        pf_contract<float>(R1.x, R2.x, R3.x, dxa, dya, dza, S.qd[sa], S.qa[sa], S.qb[0][sa], S.qb[1][sa], g0, g1,
                           g2);
        f0 += g0;
        f1 += g1;
        f2 += g2;
        pf_contract<float>(R1.y, R2.y, R3.y, dxb, dyb, dzb, S.qd[sb], S.qa[sb], S.qb[0][sb], S.qb[1][sb], g0, g1,
                           g2);
        if (tb == cur) {
            f0 += g0;
            f1 += g1;
            f2 += g2;
        } else {
            leave(tb, selfb);
            f0 = g0;
            f1 = g1;
            f2 = g2;
        }
    }
    if (slice.left > 0) {
        int tg, src;
        slice.next(S.words, tg, src);
        if (tg != cur) {
            leave(tg, S.pos[tg]);
            f0 = f1 = f2 = 0.f;
        }
        float g0, g1, g2;
        pf_side<float, MINIMG>(S, pc, self, tg, src, g0, g1, g2);
        f0 += g0;
        f1 += g1;
        f2 += g2;
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
        PA::shared_add(&S.acc[0][cur], f0);
        PA::shared_add(&S.acc[1][cur], f1);
        PA::shared_add(&S.acc[2][cur], f2);
    }
}

template <class T>
__host__ __device__ constexpr int pf_warps() { return sizeof(T) == 4 ? 4 : 2; }

template <class T, bool MINIMG, bool FX>
__global__ void __launch_bounds__(128, 8) k_perm_field(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ quad0, const typename V4<T>::type *__restrict__ quad1,
    double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    typedef PairAcc<T, FX> PA;
    __shared__ PfSmem<T, typename PA::shared_t> smem[pf_warps<T>()];
    PfSmem<T, typename PA::shared_t> &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    PairConsts2 k2;
    if constexpr (std::is_same<T, float>::value) k2 = make_consts2(pc);
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    long t0, t1;
    work_range(wa, gw, nw, t0, t1);
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    int curI = -1;
    typename PA::run_t ax, ay, az;
    PA::run_zero(ax);
    PA::run_zero(ay);
    PA::run_zero(az);
    for (long t = t0; t < t1; ++t) {
        const int2 it = wa.work[t];
        __syncwarp();
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3<PA>(acc, n_pad, curI * 32 + lane, ax, ay, az);
            PA::run_zero(ax);
            PA::run_zero(ay);
            PA::run_zero(az);
            curI = it.x;
            const int si = curI * 32 + lane;
            const T4 a = posq[si], b = dipd[si], c = quad0[si], d = quad1[si];
            T4 p, m;
            p.x = a.x; p.y = a.y; p.z = a.z; p.w = b.w;
            m.x = a.w; m.y = b.x; m.z = b.y; m.w = b.z;
            S.pos[lane] = p;
            S.qd[lane] = m;
            S.qa[lane] = c;
            S.qb[0][lane] = d.x;
            S.qb[1][lane] = d.y;
        }
        const bool diag = it.y < 0;
        int sj = -1;
        unsigned ex;
        if (diag) {
            S.pos[32 + lane] = S.pos[lane];
            S.qd[32 + lane] = S.qd[lane];
            S.qa[32 + lane] = S.qa[lane];
            S.qb[0][32 + lane] = S.qb[0][lane];
            S.qb[1][32 + lane] = S.qb[1][lane];
            const int e = wa.tile_excl[wa.tile_off[curI]];
            ex = e >= 0 ? wa.excl_mask[(size_t)e * 32 + lane] : 0u;
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            S.pos[32 + lane] = cpos[cs];
            T4 m, c, d;
            m.x = m.y = m.z = m.w = T(0);
            c = m;
            d = m;
            if (sj >= 0) {
                const T4 a = posq[sj], b = dipd[sj];
                c = quad0[sj];
                d = quad1[sj];
                m.x = a.w; m.y = b.x; m.z = b.y; m.w = b.z;
            }
            S.qd[32 + lane] = m;
            S.qa[32 + lane] = c;
            S.qb[0][32 + lane] = d.x;
            S.qb[1][32 + lane] = d.y;
            ex = wa.chunk_flag[it.y] ? wa.chunk_mask[cs] : 0u;
        }
        S.ex[lane] = ex;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.acc[c][lane] = 0;
            S.acc[c][32 + lane] = 0;
        }
        SideSlice slice;
        slice.load(wa.pmask[(size_t)t * 32 + lane], wa.pmask_t[(size_t)t * 32 + lane], wa.pstart[(size_t)t * 32 + lane],
                 lane, S.words);
        if constexpr (std::is_same<T, float>::value) pf_walk_x2<MINIMG, PA>(S, slice, pc, k2);
        else pf_walk<T, MINIMG, PA>(S, slice, pc);
        __syncwarp();
        PA::run_add(ax, S.acc[0][lane]);
        PA::run_add(ay, S.acc[1][lane]);
        PA::run_add(az, S.acc[2][lane]);
        if (diag) {
            PA::run_add(ax, S.acc[0][32 + lane]);
            PA::run_add(ay, S.acc[1][32 + lane]);
            PA::run_add(az, S.acc[2][32 + lane]);
        } else if (sj >= 0) {
            flush3_item<PA>(acc, n_pad, sj, S, 0, lane);
        }
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush3<PA>(acc, n_pad, curI * 32 + lane, ax, ay, az);
}

// ---------------------------------------------------------------------------------------
// a5: dipole-field matrix-vector product, E_i += -R1 p_j + R2 (p_j.R) R (and i <-> j).
// Positions are fixed during a solve, so the in-range pairs of every work item and their
// transposed bit matrix were found once per configuration. Per item, a warp stages the
// 32 i-atoms and 32 j-atoms in shared memory; the "pair sides" (target atom, source atom)
// are the row bits (field at each i-atom) and the column bits (field at each j-atom). In
// word order they are sorted by target, and each lane walks an equal contiguous share of
// them in place (SideSlice), accumulating in registers while the target stays the same and
// adding to a shared per-target sum only when it changes (a few times per lane per item).
// So every lane evaluates one in-range pair side per step, whatever the pair distribution;
// the field expression is even in R, so one code path serves both sides. In FP32 a lane takes
// two consecutive sides per step and evaluates their radial terms in the packed f32x2
// arithmetic of sm_100+ (matvec_walk_x2): the kernel is issue-bound, and the packed form
// takes about half the issue slots for that part (84.5 -> 69.8 us per launch at 96,000
// atoms, at 64 registers and 8 CTAs per SM instead of 40 and 12).
template <class T, class A>
struct MvSmem {
    typename V4<T>::type pos[64];    // x, y, z, Thole factor: [0,32) block I, [32,64) the item's j atoms
    typename V4<T>::type p[64];      // dipoles of the same atoms
    A acc[3][64];                    // per-target sums of the item
    unsigned words[64];              // pair bits: rows of the i atoms, then columns of the j atoms
};

// One pair side's contribution to the field at its target: -R1 p_src + R2 (p_src.R) R, with
// R = x_target - x_source (the expression is even in R, so it serves both sides of a pair).
template <class T, bool MINIMG>
__device__ __forceinline__ void mv_side(const PairConsts<T> &pc, const typename V4<T>::type &self,
                                        const typename V4<T>::type &other, const typename V4<T>::type &po, T &g0,
                                        T &g1, T &g2) {
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
    g0 = pr * dx - R1 * po.x;
    g1 = pr * dy - R1 * po.y;
    g2 = pr * dz - R1 * po.z;
}

// The walk over a lane's share of an item's pair sides (SideSlice), summing per target.
// A lane's share is a contiguous run of the target-sorted sides, so a lane that moves on
// from a target is the only lane that ever leaves it: any other lane with sides of that
// target holds it as its last one. Leaving takes a plain store; the last target of every
// lane is added atomically after the walk.
template <class T, bool MINIMG, class PA, class SM>
__device__ __forceinline__ void matvec_walk(SM &S, SideSlice &sl, const PairConsts<T> &pc) {
    typedef typename V4<T>::type T4;
    int cur = -1;
    T4 self;
    self.x = self.y = self.z = self.w = T(0);
    T f0 = 0, f1 = 0, f2 = 0;
    while (sl.left > 0) {
        int tg, src;
        sl.next(S.words, tg, src);
        if (tg != cur) {
            if (cur >= 0) {
                PA::shared_put(&S.acc[0][cur], f0);
                PA::shared_put(&S.acc[1][cur], f1);
                PA::shared_put(&S.acc[2][cur], f2);
            }
            f0 = f1 = f2 = T(0);
            cur = tg;
            self = S.pos[tg];
        }
        T g0, g1, g2;
        mv_side<T, MINIMG>(pc, self, S.pos[src], S.p[src], g0, g1, g2);
        f0 += g0;
        f1 += g1;
        f2 += g2;
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
        PA::shared_add(&S.acc[0][cur], f0);
        PA::shared_add(&S.acc[1][cur], f1);
        PA::shared_add(&S.acc[2][cur], f2);
    }
}

// The same walk in FP32 with two consecutive sides (a, then b) per step, their radial terms
// in packed f32x2 arithmetic (radial12_x2); an odd last side takes the scalar path. Side b
// either continues a's target or starts the next one, so the ownership rule above holds
// unchanged.
template <bool MINIMG, class PA, class SM>
__device__ __forceinline__ void matvec_walk_x2(SM &S, SideSlice &sl, const PairConsts<float> &pc,
                                               const PairConsts2 &k) {
    int cur = -1;
    float4 self = make_float4(0.f, 0.f, 0.f, 0.f);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    while (sl.left > 1) {
        int ta, sa, tb, sb;
        sl.next(S.words, ta, sa);
        sl.next(S.words, tb, sb);
        if (ta != cur) {
            if (cur >= 0) {
                PA::shared_put(&S.acc[0][cur], f0);
                PA::shared_put(&S.acc[1][cur], f1);
                PA::shared_put(&S.acc[2][cur], f2);
            }
            f0 = f1 = f2 = 0.f;
            cur = ta;
            self = S.pos[ta];
        }
        const float4 selfb = tb == ta ? self : S.pos[tb];
        const float4 oa = S.pos[sa], ob = S.pos[sb], pa = S.p[sa], pb = S.p[sb];
        float dxa, dya, dza, dxb, dyb, dzb;
        pair_vector<float, MINIMG>(pc, self.x, self.y, self.z, oa.x, oa.y, oa.z, 0.f, 0.f, 0.f, dxa, dya, dza);
        pair_vector<float, MINIMG>(pc, selfb.x, selfb.y, selfb.z, ob.x, ob.y, ob.z, 0.f, 0.f, 0.f, dxb, dyb, dzb);
        const float2 dx = make_float2(dxa, dxb), dy = make_float2(dya, dyb), dz = make_float2(dza, dzb);
        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float2 R1, R2;
        radial12_x2(k, r2, make_float2(self.w * oa.w, selfb.w * ob.w), R1, R2);
        const float pra = (pa.x * dxa + pa.y * dya + pa.z * dza) * R2.x;
        const float prb = (pb.x * dxb + pb.y * dyb + pb.z * dzb) * R2.y;
        f0 += pra * dxa - R1.x * pa.x;
        f1 += pra * dya - R1.x * pa.y;
        f2 += pra * dza - R1.x * pa.z;
        const float g0 = prb * dxb - R1.y * pb.x, g1 = prb * dyb - R1.y * pb.y, g2 = prb * dzb - R1.y * pb.z;
        if (tb == cur) {
            f0 += g0;
            f1 += g1;
            f2 += g2;
        } else {
            PA::shared_put(&S.acc[0][cur], f0);
            PA::shared_put(&S.acc[1][cur], f1);
            PA::shared_put(&S.acc[2][cur], f2);
            f0 = g0;
            f1 = g1;
            f2 = g2;
            cur = tb;
            self = selfb;
        }
    }
    if (sl.left > 0) {
        int tg, src;
        sl.next(S.words, tg, src);
        if (tg != cur) {
            if (cur >= 0) {
                PA::shared_put(&S.acc[0][cur], f0);
                PA::shared_put(&S.acc[1][cur], f1);
                PA::shared_put(&S.acc[2][cur], f2);
            }
            f0 = f1 = f2 = 0.f;
            cur = tg;
            self = S.pos[tg];
        }
        float g0, g1, g2;
        mv_side<float, MINIMG>(pc, self, S.pos[src], S.p[src], g0, g1, g2);
        f0 += g0;
        f1 += g1;
        f2 += g2;
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
        PA::shared_add(&S.acc[0][cur], f0);
        PA::shared_add(&S.acc[1][cur], f1);
        PA::shared_add(&S.acc[2][cur], f2);
    }
}

template <class T>
__host__ __device__ constexpr int mv_blocks_per_sm() { return sizeof(T) == 4 ? 8 : 12; }

template <class T, bool MINIMG, bool SHORT, bool FX>
__global__ void __launch_bounds__(128, mv_blocks_per_sm<T>()) k_matvec(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ pv, double *__restrict__ acc, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    typedef PairAcc<T, FX> PA;
    __shared__ MvSmem<T, typename PA::shared_t> smem[4];
    MvSmem<T, typename PA::shared_t> &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    constexpr bool PK = std::is_same<T, float>::value;   // FP32: two sides per step, packed
    PairConsts2 k2;
    if constexpr (PK) k2 = make_consts2(pc);
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    long t0, t1;
    work_range(wa, gw, nw, t0, t1);
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    int curI = -1;
    typename PA::run_t ax, ay, az;
    PA::run_zero(ax);
    PA::run_zero(ay);
    PA::run_zero(az);
    for (long t = t0; t < t1; ++t) {
        // the short-range field skips, before staging anything, the items whose atoms are all
        // farther apart than the short radius; block I's sums carry over
        if (SHORT && !__any_sync(0xffffffffu, (wa.sstart[(size_t)t * 32 + lane] >> 11) != 0u)) continue;
        const int2 it = wa.work[t];
        __syncwarp();   // every lane is done with the previous item's staging
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush3<PA>(acc, n_pad, curI * 32 + lane, ax, ay, az);
            PA::run_zero(ax);
            PA::run_zero(ay);
            PA::run_zero(az);
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
            S.acc[c][lane] = 0;
            S.acc[c][32 + lane] = 0;
        }
        const size_t wl = (size_t)t * 32 + lane;
        SideSlice sl;
        if (SHORT) sl.load(wa.smask[wl], wa.smask_t[wl], wa.sstart[wl], lane, S.words);
        else sl.load(wa.pmask[wl], wa.pmask_t[wl], wa.pstart[wl], lane, S.words);
        if constexpr (PK) matvec_walk_x2<MINIMG, PA>(S, sl, pc, k2);
        else matvec_walk<T, MINIMG, PA>(S, sl, pc);
        __syncwarp();
        PA::run_add(ax, S.acc[0][lane]);
        PA::run_add(ay, S.acc[1][lane]);
        PA::run_add(az, S.acc[2][lane]);
        if (diag) {
            PA::run_add(ax, S.acc[0][32 + lane]);
            PA::run_add(ay, S.acc[1][32 + lane]);
            PA::run_add(az, S.acc[2][32 + lane]);
        } else if (sj >= 0) {
            flush3_item<PA>(acc, n_pad, sj, S, 0, lane);
        }
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush3<PA>(acc, n_pad, curI * 32 + lane, ax, ay, az);
}

// f1: the same product for two dipole sets at once (AMOEBA's d and p dipoles share the
// operator): the pair tensor (R1, R2) of every pair side is evaluated once and applied to
// both sources, so the radial work - most of the kernel - is paid once for two vectors.
template <class T, class A>
struct Mv2Smem {
    typename V4<T>::type pos[64];
    typename V4<T>::type p[2][64];   // the two dipole sets of the item's atoms
    A acc[6][64];                    // per-target sums: set 0 x y z, set 1 x y z
    unsigned words[64];
};

// one side's contribution to both sets' fields at its target, given R and (R1, R2)
template <class T>
__device__ __forceinline__ void mv2_terms(T dx, T dy, T dz, T R1, T R2, const typename V4<T>::type &po,
                                          const typename V4<T>::type &pq, T *g) {
    const T pr0 = (po.x * dx + po.y * dy + po.z * dz) * R2;
    const T pr1 = (pq.x * dx + pq.y * dy + pq.z * dz) * R2;
    g[0] = pr0 * dx - R1 * po.x;
    g[1] = pr0 * dy - R1 * po.y;
    g[2] = pr0 * dz - R1 * po.z;
    g[3] = pr1 * dx - R1 * pq.x;
    g[4] = pr1 * dy - R1 * pq.y;
    g[5] = pr1 * dz - R1 * pq.z;
}

// the two-set walk (ownership as in matvec_walk)
template <class T, bool MINIMG, class PA, class SM>
__device__ __forceinline__ void matvec2_walk(SM &S, SideSlice &sl, const PairConsts<T> &pc) {
    typedef typename V4<T>::type T4;
    int cur = -1;
    T4 self;
    self.x = self.y = self.z = self.w = T(0);
    T f[6] = {0, 0, 0, 0, 0, 0};
    while (sl.left > 0) {
        int tg, src;
        sl.next(S.words, tg, src);
        if (tg != cur) {
            if (cur >= 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) PA::shared_put(&S.acc[c][cur], f[c]);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] = T(0);
            cur = tg;
            self = S.pos[tg];
        }
        const T4 other = S.pos[src];
        T dx, dy, dz;
        pair_vector<T, MINIMG>(pc, self.x, self.y, self.z, other.x, other.y, other.z, T(0), T(0), T(0), dx, dy, dz);
        const T r2 = dx * dx + dy * dy + dz * dz;
        const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
        T B[2], U[2], oml[2];
        screened<T, 2>(pc, r, rinv, rinv2, B, U);
        thole_oml<T, 2>(pc.thole_a * r2 * r * self.w * other.w, oml);
        T g[6];
        mv2_terms<T>(dx, dy, dz, B[0] - oml[0] * U[0], B[1] - oml[1] * U[1], S.p[0][src], S.p[1][src], g);
#pragma unroll
        for (int c = 0; c < 6; ++c) f[c] += g[c];
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) PA::shared_add(&S.acc[c][cur], f[c]);
    }
}

// FP32: two consecutive sides per step, (R1, R2) of both in packed f32x2 arithmetic
template <bool MINIMG, class PA, class SM>
__device__ __forceinline__ void matvec2_walk_x2(SM &S, SideSlice &sl, const PairConsts<float> &pc,
                                                const PairConsts2 &k) {
    int cur = -1;
    float4 self = make_float4(0.f, 0.f, 0.f, 0.f);
    float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto leave = [&](int next, const float4 &nself) {
        if (cur >= 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) PA::shared_put(&S.acc[c][cur], f[c]);
        }
        cur = next;
        self = nself;
    };
    while (sl.left > 1) {
        int ta, sa, tb, sb;
        sl.next(S.words, ta, sa);
        sl.next(S.words, tb, sb);
        if (ta != cur) {
            leave(ta, S.pos[ta]);
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] = 0.f;
        }
        const float4 selfb = tb == ta ? self : S.pos[tb];
        const float4 oa = S.pos[sa], ob = S.pos[sb];
        float dxa, dya, dza, dxb, dyb, dzb;
        pair_vector<float, MINIMG>(pc, self.x, self.y, self.z, oa.x, oa.y, oa.z, 0.f, 0.f, 0.f, dxa, dya, dza);
        pair_vector<float, MINIMG>(pc, selfb.x, selfb.y, selfb.z, ob.x, ob.y, ob.z, 0.f, 0.f, 0.f, dxb, dyb, dzb);
        const float2 dx = make_float2(dxa, dxb), dy = make_float2(dya, dyb), dz = make_float2(dza, dzb);
        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float2 R1, R2;
        radial12_x2(k, r2, make_float2(self.w * oa.w, selfb.w * ob.w), R1, R2);
        float g[6];
        mv2_terms<float>(dxa, dya, dza, R1.x, R2.x, S.p[0][sa], S.p[1][sa], g);
#pragma unroll
        for (int c = 0; c < 6; ++c) f[c] += g[c];
        mv2_terms<float>(dxb, dyb, dzb, R1.y, R2.y, S.p[0][sb], S.p[1][sb], g);
        if (tb == cur) {
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] += g[c];
        } else {
            leave(tb, selfb);
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] = g[c];
        }
    }
    if (sl.left > 0) {
        int tg, src;
        sl.next(S.words, tg, src);
        if (tg != cur) {
            leave(tg, S.pos[tg]);
#pragma unroll
            for (int c = 0; c < 6; ++c) f[c] = 0.f;
        }
        const float4 other = S.pos[src];
        float dx, dy, dz;
        pair_vector<float, MINIMG>(pc, self.x, self.y, self.z, other.x, other.y, other.z, 0.f, 0.f, 0.f, dx, dy, dz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
        float B[2], U[2], oml[2];
        screened<float, 2>(pc, r, rinv, rinv2, B, U);
        thole_oml<float, 2>(pc.thole_a * r2 * r * self.w * other.w, oml);
        float g[6];
        mv2_terms<float>(dx, dy, dz, B[0] - oml[0] * U[0], B[1] - oml[1] * U[1], S.p[0][src], S.p[1][src], g);
#pragma unroll
        for (int c = 0; c < 6; ++c) f[c] += g[c];
    }
    __syncwarp();   // the plain stores land before the last targets are added
    if (cur >= 0) {
#pragma unroll
        for (int c = 0; c < 6; ++c) PA::shared_add(&S.acc[c][cur], f[c]);
    }
}

template <class T, bool MINIMG, bool FX>
__global__ void __launch_bounds__(128) k_matvec2(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ pv0, const typename V4<T>::type *__restrict__ pv1,
    double *__restrict__ acc0, double *__restrict__ acc1, int n_pad, PairConsts<T> pc) {
    typedef typename V4<T>::type T4;
    typedef PairAcc<T, FX> PA;
    __shared__ Mv2Smem<T, typename PA::shared_t> smem[4];
    Mv2Smem<T, typename PA::shared_t> &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    PairConsts2 k2;
    if constexpr (std::is_same<T, float>::value) k2 = make_consts2(pc);
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    long t0, t1;
    work_range(wa, gw, nw, t0, t1);
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    int curI = -1;
    typename PA::run_t a[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) PA::run_zero(a[c]);
    for (long t = t0; t < t1; ++t) {
        const int2 it = wa.work[t];
        __syncwarp();
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) {
                flush3<PA>(acc0, n_pad, curI * 32 + lane, a[0], a[1], a[2]);
                flush3<PA>(acc1, n_pad, curI * 32 + lane, a[3], a[4], a[5]);
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) PA::run_zero(a[c]);
            curI = it.x;
            const int si = curI * 32 + lane;
            T4 q = posq[si];
            q.w = dipd[si].w;
            S.pos[lane] = q;
            S.p[0][lane] = pv0[si];
            S.p[1][lane] = pv1[si];
        }
        const bool diag = it.y < 0;
        int sj = -1;
        if (diag) {
            S.pos[32 + lane] = S.pos[lane];
            S.p[0][32 + lane] = S.p[0][lane];
            S.p[1][32 + lane] = S.p[1][lane];
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            S.pos[32 + lane] = cpos[cs];
            T4 z;
            z.x = z.y = z.z = z.w = T(0);
            S.p[0][32 + lane] = sj >= 0 ? pv0[sj] : z;
            S.p[1][32 + lane] = sj >= 0 ? pv1[sj] : z;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            S.acc[c][lane] = 0;
            S.acc[c][32 + lane] = 0;
        }
        SideSlice sl;
        sl.load(wa.pmask[(size_t)t * 32 + lane], wa.pmask_t[(size_t)t * 32 + lane], wa.pstart[(size_t)t * 32 + lane],
                 lane, S.words);
        if constexpr (std::is_same<T, float>::value) matvec2_walk_x2<MINIMG, PA>(S, sl, pc, k2);
        else matvec2_walk<T, MINIMG, PA>(S, sl, pc);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 6; ++c) PA::run_add(a[c], S.acc[c][lane]);
        if (diag) {
#pragma unroll
            for (int c = 0; c < 6; ++c) PA::run_add(a[c], S.acc[c][32 + lane]);
        } else if (sj >= 0) {
            flush3_item<PA>(acc0, n_pad, sj, S, 0, lane);
            flush3_item<PA>(acc1, n_pad, sj, S, 3, lane);
        }
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) {
        flush3<PA>(acc0, n_pad, curI * 32 + lane, a[0], a[1], a[2]);
        flush3<PA>(acc1, n_pad, curI * 32 + lane, a[3], a[4], a[5]);
    }
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
    auto kern = ctx->fixed ? (ctx->minimg ? k_perm_field<T, true, true> : k_perm_field<T, false, true>)
                           : (ctx->minimg ? k_perm_field<T, true, false> : k_perm_field<T, false, false>);
    static int grids[4] = {0, 0, 0, 0};
    int &grid = grids[ctx->minimg + 2 * ctx->fixed];
    if (!grid) grid = resident_grid(ctx, kern, 32 * pf_warps<T>());
    kern<<<grid, 32 * pf_warps<T>(), 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd,
                                             (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, ctx->acc, ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int matvec_t(ap_ctx *ctx, const void *p, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->fixed ? (ctx->minimg ? k_matvec<T, true, false, true> : k_matvec<T, false, false, true>)
                           : (ctx->minimg ? k_matvec<T, true, false, false> : k_matvec<T, false, false, false>);
    static int grids[4] = {0, 0, 0, 0};
    int &g0 = grids[ctx->minimg + 2 * ctx->fixed];
    if (!g0) g0 = resident_grid(ctx, kern, 128);
    const int grid = ctx->tune_mv_per_sm > 0 ? std::min(g0, ctx->tune_mv_per_sm * ctx->sm_count) : g0;
    kern<<<grid, 128, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)p, ctx->acc,
                              ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int matvec2_t(ap_ctx *ctx, const void *p0, const void *p1, double *acc0, double *acc1, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->fixed ? (ctx->minimg ? k_matvec2<T, true, true> : k_matvec2<T, false, true>)
                           : (ctx->minimg ? k_matvec2<T, true, false> : k_matvec2<T, false, false>);
    static int grids[4] = {0, 0, 0, 0};
    int &grid = grids[ctx->minimg + 2 * ctx->fixed];
    if (!grid) grid = resident_grid(ctx, kern, 128);
    kern<<<grid, 128, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, (const T4 *)ctx->dipd, (const T4 *)p0,
                              (const T4 *)p1, acc0, acc1, ctx->n_pad, pc);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int short_t(ap_ctx *ctx, const void *p, double *out, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc = make_consts<T>(ctx);
    auto kern = ctx->fixed ? (ctx->minimg ? k_matvec<T, true, true, true> : k_matvec<T, false, true, true>)
                           : (ctx->minimg ? k_matvec<T, true, true, false> : k_matvec<T, false, true, false>);
    static int grids[4] = {0, 0, 0, 0};
    int &grid = grids[ctx->minimg + 2 * ctx->fixed];
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

// CTAs of the real-space matvec that fit on one SM at once (the autotuner's upper bound)
int real_matvec_resident_per_sm(ap_ctx *ctx) {
    int per_sm = 0;
    if (ctx->prec == AP_FP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_matvec<double, false, false, false>, 128, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_matvec<float, false, false, false>, 128, 0);
    return std::max(1, per_sm);
}

int real_matvec_launch(ap_ctx *ctx, const void *p, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? matvec_t<double>(ctx, p, s) : matvec_t<float>(ctx, p, s);
}

int real_matvec2_launch(ap_ctx *ctx, const void *p0, const void *p1, double *acc0, double *acc1, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? matvec2_t<double>(ctx, p0, p1, acc0, acc1, s)
                                : matvec2_t<float>(ctx, p0, p1, acc0, acc1, s);
}
