// a9 - Polarization energy and forces at fixed induced dipoles ("final force evaluation",
// paper Sec. 1.2).
//
// E_pol = -(f/2) sum_i mu_i . E_i. At the solution of A mu = E, dE_pol/dx at fixed mu is the
// gradient of  -f sum_{i<j} mu_i T_ij mu_j - f sum_i mu_i . E_i  (variational property):
//   real space: each unordered pair carries
//       U_ij = -f [mu_i . E(R; M_j) + mu_j . E(-R; M_i) + mu_i . T(R) mu_j],  R = x_i - x_j;
//   reciprocal: f <dQ_mu/dx, phi_M + phi_mu> + f <dQ_M/dx, phi_mu>, from the smooth-PME
//               potentials' derivatives up to third order at the atoms;
//   frames:     global multipoles rotate with their frame atoms: dU/d(global dipole) and
//               dU/d(global quadrupole) are chained through the frame construction.
// Pair arithmetic in T, accumulation in FP64 as in the other real-space kernels.
//
// Virial (on request): V_ab = dE_pol/de_ab under x -> (I + e) x of positions and box, which
// the paper's real-space loop updates with the energy and the forces (Sec. 1.2.1) and sums in
// double precision (Sec. 2.2). At fixed mu it is
//   pairs:      sum over pairs of (dU/dR)_a R_b (R the image vector);
//   frames:     sum over frame vectors v of (dU/dv)_a v_b;
//   reciprocal: -f sum_j [grad phi_{M+mu} mu_j^T + grad phi_mu d_j^T + (2/3) H(phi_mu) Q_j]
//               plus the structure-factor sum of pme.cu (volume and |m| of C(m));
// accumulated per block in FP64 (fixed point in AP_FIXED) into nine device slots.
#include "common.cuh"
#include "pair_math.cuh"

#include <cmath>
#include <type_traits>

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s);

namespace {

// the twelve running sums of block I's atom s (force, dU/dd, dU/dQ) to the accumulators
template <class PA>
__device__ __forceinline__ void flush12(double *frc, double *gdip, double *gquad, int n_pad, int s,
                                        const typename PA::run_t *a) {
    for (int c = 0; c < 3; ++c) PA::run_flush(frc + c * n_pad + s, a[c]);
    for (int c = 0; c < 3; ++c) PA::run_flush(gdip + c * n_pad + s, a[3 + c]);
    for (int c = 0; c < 6; ++c) PA::run_flush(gquad + c * n_pad + s, a[6 + c]);
}
// one item's twelve sums of a chunk atom s (already scaled)
template <class PA>
__device__ __forceinline__ void flush12_item(double *frc, double *gdip, double *gquad, int n_pad, int s,
                                             const typename PA::shared_t *a) {
    for (int c = 0; c < 3; ++c) PA::item_flush(frc + c * n_pad + s, a[c]);
    for (int c = 0; c < 3; ++c) PA::item_flush(gdip + c * n_pad + s, a[3 + c]);
    for (int c = 0; c < 6; ++c) PA::item_flush(gquad + c * n_pad + s, a[6 + c]);
}
// FP64 value v added to slot k of an array of FP64 numbers or (fixed) fixed-point integers,
// by the only thread that updates that slot
__device__ __forceinline__ void add_plain(double *arr, size_t k, double v, int fixed) {
    if (fixed)
        reinterpret_cast<long long *>(arr)[k] += ap_to_fx(v);
    else
        arr[k] += v;
}

// adds the nine values v of every thread of a block of NT threads to acc[0..8]: FP64 sums
// and FP64 atomics, or (FX) values already in fixed point, integer sums and integer atomics
// (order-independent, so bitwise reproducible)
template <int NT, class V>
__device__ __forceinline__ void block_add9(V *v, double *acc) {
    __shared__ V sm[NT / 32][9];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        V x = v[k];
        for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (l == 0) sm[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        V t = 0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) t += sm[k][threadIdx.x];
        if constexpr (std::is_integral<V>::value)
            atomicAdd(reinterpret_cast<unsigned long long *>(acc) + threadIdx.x, (unsigned long long)t);
        else
            atomicAdd(acc + threadIdx.x, t);
    }
}

// out_a = sum_b mu_b dE_b/dR_a for the field E(R) of a multipole (q, d, Q) at the origin
template <class T>
__device__ __forceinline__ void mu_dot_field_grad(T q, const T *d, const T *Q /*xx xy xz yy yz zz*/, const T *mu,
                                                  T dx, T dy, T dz, T R1, T R2, T R3, T R4, T *out) {
    const T R[3] = {dx, dy, dz};
    const T QR[3] = {Q[0] * dx + Q[1] * dy + Q[2] * dz, Q[1] * dx + Q[3] * dy + Q[4] * dz,
                     Q[2] * dx + Q[4] * dy + Q[5] * dz};
    const T Qm[3] = {Q[0] * mu[0] + Q[1] * mu[1] + Q[2] * mu[2], Q[1] * mu[0] + Q[3] * mu[1] + Q[4] * mu[2],
                     Q[2] * mu[0] + Q[4] * mu[1] + Q[5] * mu[2]};
    const T muR = mu[0] * dx + mu[1] * dy + mu[2] * dz;
    const T dR = d[0] * dx + d[1] * dy + d[2] * dz;
    const T dmu = d[0] * mu[0] + d[1] * mu[1] + d[2] * mu[2];
    const T RQR = QR[0] * dx + QR[1] * dy + QR[2] * dz;
    const T muQR = mu[0] * QR[0] + mu[1] * QR[1] + mu[2] * QR[2];
    const T cR = -q * muR * R2 + dmu * R2 - dR * muR * R3 + T(2.0 / 3.0) * muQR * R3 - RQR * muR * R4 * T(1.0 / 3.0);
    const T cmu = q * R1 + dR * R2 + RQR * R3 * T(1.0 / 3.0);
    const T cd = muR * R2;
    const T cQm = -T(2.0 / 3.0) * R2;
    const T cQR = T(2.0 / 3.0) * muR * R3;
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = cR * R[a] + cmu * mu[a] + cd * d[a] + cQm * Qm[a] + cQR * QR[a];
}

// One warp per work item, pair sides walked in place as in the real-space field kernels: every
// in-range pair gives the side (target t, source s) for both atoms, and with
// R = x_t - x_s the same expressions give t's force and t's dU/dd, dU/dQ. Per side the
// kernel accumulates, without the constant factors,
//   F_t / f         += mu_t.G(R; M_s) - mu_s.G(R; q_t, -d_t, Q_t) + d(mu_t T mu_s)/dR
//   dU/dd_t / (-f)  += -R_1 mu_s + R_2 (mu_s.R) R
//   dU/dQ_t / (-f/3) += R_2 sym(mu_s R) - R_3 (mu_s.R) R R
// so the pair's force is evaluated once per side (twice per pair) in exchange for lanes
// that only ever see in-range pairs. In FP32 a lane takes two sides per step with their
// radial terms in packed f32x2 arithmetic (fo_walk_x2): 255.9 -> 229.9 us at 96,000 atoms,
// at 96 registers and 5 CTAs per SM (the same walk at 80 registers, 6 per SM, spilled more
// and took 243.7 us).
template <class T, class A>
struct FoSmem {
    typename V4<T>::type pos[64];   // x, y, z, Thole factor: [0,32) block I, [32,64) the item's j atoms
    typename V4<T>::type qd[64];    // charge, dipole
    typename V4<T>::type qa[64];    // Qxx, Qxy, Qxz, Qyy
    typename V4<T>::type mu[64];    // induced dipole
    T qb[2][64];                    // Qyz, Qzz
    A acc[12][64];                  // per-target sums of the item
    unsigned ex[32];                // exclusion words: lane i, bit j
    unsigned words[64];             // pair bits: rows of the i atoms, then columns of the j atoms
};

template <class T>
constexpr int fo_warps() { return sizeof(T) == 4 ? 4 : 2; }

// the target atom of a pair side: position and Thole factor, charge and dipole, quadrupole
template <class T>
struct FoTarget {
    typename V4<T>::type pos, qd, qa, mu;
    T qyz, qzz;
};
template <class T, class SM>
__device__ __forceinline__ void fo_target(const SM &S, int t, FoTarget<T> &g) {
    g.pos = S.pos[t];
    g.qd = S.qd[t];
    g.qa = S.qa[t];
    g.mu = S.mu[t];
    g.qyz = S.qb[0][t];
    g.qzz = S.qb[1][t];
}

// one side's terms, given its R = x_target - x_source and its radial functions Rd (with the
// pair's scale), Ru (unscaled): the force, dU/dd and dU/dQ of the target (unscaled sums), and
// with VS the side's F R^T
template <class T, bool VS, class SM>
__device__ __forceinline__ void fo_side_terms(const SM &S, const FoTarget<T> &g, int src, T dx, T dy, T dz,
                                              const T *Rd, const T *Ru, T *f, T *vs) {
    typedef typename V4<T>::type T4;
    const T4 om = S.qd[src], oa = S.qa[src], ou = S.mu[src];
    const T oyz = S.qb[0][src], ozz = S.qb[1][src];
    const T mt[3] = {g.mu.x, g.mu.y, g.mu.z}, ms[3] = {ou.x, ou.y, ou.z};
    const T ds[3] = {om.y, om.z, om.w}, ndt[3] = {-g.qd.y, -g.qd.z, -g.qd.w};
    const T Qs[6] = {oa.x, oa.y, oa.z, oa.w, oyz, ozz};
    const T Qt[6] = {g.qa.x, g.qa.y, g.qa.z, g.qa.w, g.qyz, g.qzz};
    T A[3], Bv[3];
    mu_dot_field_grad<T>(om.x, ds, Qs, mt, dx, dy, dz, Rd[0], Rd[1], Rd[2], Rd[3], A);
    mu_dot_field_grad<T>(g.qd.x, ndt, Qt, ms, dx, dy, dz, Rd[0], Rd[1], Rd[2], Rd[3], Bv);
    const T mts = mt[0] * ms[0] + mt[1] * ms[1] + mt[2] * ms[2];
    const T mtr = mt[0] * dx + mt[1] * dy + mt[2] * dz;
    const T msr = ms[0] * dx + ms[1] * dy + ms[2] * dz;
    const T cR = Ru[1] * mts - Ru[2] * mtr * msr;
    const T R[3] = {dx, dy, dz};
    T fs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fs[k] = A[k] - Bv[k] + cR * R[k] + Ru[1] * (mt[k] * msr + ms[k] * mtr);
        f[k] += fs[k];
        f[3 + k] += -Rd[0] * ms[k] + Rd[1] * msr * R[k];
    }
    if constexpr (VS) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) vs[3 * a + b] += fs[a] * R[b];
    }
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
        f[6 + k] += Rd[1] * (ms[ia[k]] * R[ib[k]] + R[ia[k]] * ms[ib[k]]) - Rd[2] * msr * R[ia[k]] * R[ib[k]];
}

// one side in full (scalar radial terms)
template <class T, bool MINIMG, bool VS, class SM>
__device__ __forceinline__ void fo_side(const SM &S, const PairConsts<T> &pc, const FoTarget<T> &g, int tg, int src,
                                        T *f, T *vs) {
    typedef typename V4<T>::type T4;
    const int sl = src & 31;   // the source's lane within its half
    const bool exb = tg < 32 ? (S.ex[tg] >> sl) & 1u : (S.ex[sl] >> (tg - 32)) & 1u;
    const T4 o = S.pos[src];
    T dx, dy, dz;
    pair_vector<T, MINIMG>(pc, g.pos.x, g.pos.y, g.pos.z, o.x, o.y, o.z, T(0), T(0), T(0), dx, dy, dz);
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T rinv = ap_rsqrt(r2), r = r2 * rinv, rinv2 = rinv * rinv;
    T B[4], U[4], oml[4];
    screened<T, 4>(pc, r, rinv, rinv2, B, U);
    thole_oml<T, 4>(pc.thole_a * r2 * r * g.pos.w * o.w, oml);
    T Rd[4], Ru[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) Rd[k] = B[k] - (exb ? U[k] : oml[k] * U[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) Ru[k] = B[k] - oml[k] * U[k];
    fo_side_terms<T, VS>(S, g, src, dx, dy, dz, Rd, Ru, f, vs);
}

// The walk over a lane's share of the item's sides (plain stores on leaving a target, the last
// target left in `cur` for the caller's atomic add)
template <class T, bool MINIMG, bool VS, class PA, class SM>
__device__ __forceinline__ void fo_walk(SM &S, SideSlice &slice, const PairConsts<T> &pc, const T *scf, int &cur,
                                        T *f, T *vs) {
    FoTarget<T> g;
    while (slice.left > 0) {
        int tg, src;
        slice.next(S.words, tg, src);
        if (tg != cur) {
            if (cur >= 0) {   // the only lane that leaves this target: a plain store
#pragma unroll
                for (int k = 0; k < 12; ++k) PA::shared_put(&S.acc[k][cur], f[k] * scf[k]);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) f[k] = T(0);
            cur = tg;
            fo_target<T>(S, tg, g);
        }
        fo_side<T, MINIMG, VS>(S, pc, g, tg, src, f, vs);
    }
}

// FP32: two consecutive sides per step, their radial terms in packed f32x2 arithmetic
// (radial_forces_x2), the multipole terms per side; an odd last side takes the scalar path
template <bool MINIMG, bool VS, class PA, class SM>
__device__ __forceinline__ void fo_walk_x2(SM &S, SideSlice &slice, const PairConsts<float> &pc,
                                           const PairConsts2 &k, const float *scf, int &cur, float *f, float *vs) {
    FoTarget<float> g;
    auto enter = [&](int t) {
        if (cur >= 0) {   // the only lane that leaves this target: a plain store
#pragma unroll
            for (int q = 0; q < 12; ++q) PA::shared_put(&S.acc[q][cur], f[q] * scf[q]);
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) f[q] = 0.f;
        cur = t;
        fo_target<float>(S, t, g);
    };
    while (slice.left > 1) {
        int ta, sa, tb, sb;
        slice.next(S.words, ta, sa);
        slice.next(S.words, tb, sb);
        if (ta != cur) enter(ta);
        const float4 pb = tb == ta ? g.pos : S.pos[tb];
        const int la = sa & 31, lb = sb & 31;
        const bool exa = ta < 32 ? (S.ex[ta] >> la) & 1u : (S.ex[la] >> (ta - 32)) & 1u;
        const bool exb = tb < 32 ? (S.ex[tb] >> lb) & 1u : (S.ex[lb] >> (tb - 32)) & 1u;
        const float4 oa = S.pos[sa], ob = S.pos[sb];
        float dxa, dya, dza, dxb, dyb, dzb;
        pair_vector<float, MINIMG>(pc, g.pos.x, g.pos.y, g.pos.z, oa.x, oa.y, oa.z, 0.f, 0.f, 0.f, dxa, dya, dza);
        pair_vector<float, MINIMG>(pc, pb.x, pb.y, pb.z, ob.x, ob.y, ob.z, 0.f, 0.f, 0.f, dxb, dyb, dzb);
        const float2 dx = make_float2(dxa, dxb), dy = make_float2(dya, dyb), dz = make_float2(dza, dzb);
        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
        float2 Rd2[4], Ru2[3];
        radial_forces_x2(k, r2, make_float2(g.pos.w * oa.w, pb.w * ob.w), exa, exb, Rd2, Ru2);
        {
            const float Rd[4] = {Rd2[0].x, Rd2[1].x, Rd2[2].x, Rd2[3].x}, Ru[3] = {Ru2[0].x, Ru2[1].x, Ru2[2].x};
            fo_side_terms<float, VS>(S, g, sa, dxa, dya, dza, Rd, Ru, f, vs);
        }
        if (tb != cur) enter(tb);
        {
            const float Rd[4] = {Rd2[0].y, Rd2[1].y, Rd2[2].y, Rd2[3].y}, Ru[3] = {Ru2[0].y, Ru2[1].y, Ru2[2].y};
            fo_side_terms<float, VS>(S, g, sb, dxb, dyb, dzb, Rd, Ru, f, vs);
        }
    }
    if (slice.left > 0) {
        int tg, src;
        slice.next(S.words, tg, src);
        if (tg != cur) enter(tg);
        fo_side<float, MINIMG, VS>(S, pc, g, tg, src, f, vs);
    }
}

// VIR: also the pairs' virial. Without per-pair minimum image every position of an item is
// relative to block I's origin, and the item holds both sides of each of its pairs, whose
// forces are opposite; so the item's sum over pairs of (dU/dR) R^T = -sum over sides of
// F_t R^T / 2 equals -sum over its 64 targets of F_t x_t^T, formed once per item from the
// per-target sums the kernel keeps anyway. With per-pair minimum image (small boxes) the
// sides' F R^T are summed as they come.
template <class T, bool MINIMG, bool FX, bool VIR>
__global__ void __launch_bounds__(128, VIR ? 4 : 5) k_pair_forces(
    WorkArgs wa, const typename V4<T>::type *__restrict__ posq,
    const typename V4<T>::type *__restrict__ dipd, const typename V4<T>::type *__restrict__ quad0,
    const typename V4<T>::type *__restrict__ quad1, const typename V4<T>::type *__restrict__ muv,
    double *__restrict__ frc, double *__restrict__ gdip, double *__restrict__ gquad, int n_pad, PairConsts<T> pc,
    double fconst, double *__restrict__ vir) {
    typedef typename V4<T>::type T4;
    typedef PairAcc<T, FX> PA;
    __shared__ FoSmem<T, typename PA::shared_t> smem[fo_warps<T>()];
    FoSmem<T, typename PA::shared_t> &S = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    PairConsts2 k2;
    if constexpr (std::is_same<T, float>::value) k2 = make_consts2(pc);
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    long t0, t1;
    work_range(wa, gw, nw, t0, t1);
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    const double sc[12] = {fconst, fconst, fconst, -fconst, -fconst, -fconst, -fconst / 3, -fconst / 3,
                           -fconst / 3, -fconst / 3, -fconst / 3, -fconst / 3};
    // FP64 mode: per-item sums are unscaled and scaled in FP64; mixed and fixed point: scaled
    // in T as they enter the item's sums (so that no FP64 multiply runs per item, and the
    // fixed-point integers hold the final quantities)
    constexpr bool PRESCALE = FX || sizeof(T) == 4;
    T scf[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) scf[k] = PRESCALE ? (T)sc[k] : T(1);
    int curI = -1;
    typename PA::run_t ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) PA::run_zero(ai[k]);
    typedef typename std::conditional<FX, long long, double>::type vacc_t;
    vacc_t vacc[9];                 // this lane's share of the virial (VIR)
#pragma unroll
    for (int k = 0; k < 9; ++k) vacc[k] = 0;
    for (long t = t0; t < t1; ++t) {
        const int2 it = wa.work[t];
        __syncwarp();
        if (it.x != curI) {
            if (curI >= 0 && curI * 32 + lane < pc.n) flush12<PA>(frc, gdip, gquad, n_pad, curI * 32 + lane, ai);
#pragma unroll
            for (int k = 0; k < 12; ++k) PA::run_zero(ai[k]);
            curI = it.x;
            const int si = curI * 32 + lane;
            const T4 a = posq[si], b = dipd[si], c = quad0[si], d = quad1[si];
            T4 p, m;
            p.x = a.x; p.y = a.y; p.z = a.z; p.w = b.w;
            m.x = a.w; m.y = b.x; m.z = b.y; m.w = b.z;
            S.pos[lane] = p;
            S.qd[lane] = m;
            S.qa[lane] = c;
            S.mu[lane] = muv[si];
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
            S.mu[32 + lane] = S.mu[lane];
            S.qb[0][32 + lane] = S.qb[0][lane];
            S.qb[1][32 + lane] = S.qb[1][lane];
            const int e = wa.tile_excl[wa.tile_off[curI]];
            ex = e >= 0 ? wa.excl_mask[(size_t)e * 32 + lane] : 0u;
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            S.pos[32 + lane] = cpos[cs];
            T4 m, c, d, u;
            m.x = m.y = m.z = m.w = T(0);
            c = m;
            d = m;
            u = m;
            if (sj >= 0) {
                const T4 a = posq[sj], b = dipd[sj];
                c = quad0[sj];
                d = quad1[sj];
                u = muv[sj];
                m.x = a.w; m.y = b.x; m.z = b.y; m.w = b.z;
            }
            S.qd[32 + lane] = m;
            S.qa[32 + lane] = c;
            S.mu[32 + lane] = u;
            S.qb[0][32 + lane] = d.x;
            S.qb[1][32 + lane] = d.y;
            ex = wa.chunk_flag[it.y] ? wa.chunk_mask[cs] : 0u;
        }
        S.ex[lane] = ex;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            S.acc[k][lane] = 0;
            S.acc[k][32 + lane] = 0;
        }
        SideSlice slice;
        slice.load(wa.pmask[(size_t)t * 32 + lane], wa.pmask_t[(size_t)t * 32 + lane], wa.pstart[(size_t)t * 32 + lane],
                 lane, S.words);
        int cur = -1;
        T f[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) f[k] = T(0);
        T vs[9];                    // sum of F_side R^T over this lane's sides (VIR, MINIMG)
#pragma unroll
        for (int k = 0; k < 9; ++k) vs[k] = T(0);
        if constexpr (std::is_same<T, float>::value)
            fo_walk_x2<MINIMG, VIR && MINIMG, PA>(S, slice, pc, k2, scf, cur, f, vs);
        else
            fo_walk<T, MINIMG, VIR && MINIMG, PA>(S, slice, pc, scf, cur, f, vs);
        __syncwarp();   // the plain stores land before the last targets are added
        if (cur >= 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) PA::shared_add(&S.acc[k][cur], f[k] * scf[k]);
        }
        __syncwarp();
        if constexpr (VIR) {
            // in kcal/mol: each side's force is f times the kernel's sums, the pair's virial half
            // the sum over its two sides
            double v[9];
            if constexpr (MINIMG) {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = -0.5 * fconst * (double)vs[k];
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = 0.0;
                const bool oki = curI * 32 + lane < pc.n;          // padding slots hold NaN positions
                const bool okj = diag ? oki : sj >= 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int tt = h ? 32 + lane : lane;
                    if (!(h ? okj : oki)) continue;
                    const T4 ps = S.pos[tt];
                    const double x[3] = {(double)ps.x, (double)ps.y, (double)ps.z};
                    double F[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        F[a] = FX ? ap_from_fx((long long)S.acc[a][tt])
                                  : (PRESCALE ? 1.0 : sc[a]) * (double)S.acc[a][tt];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) v[3 * a + b] -= F[a] * x[b];
                }
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if constexpr (FX) vacc[k] += ap_to_fx(v[k]);
                else vacc[k] += v[k];
            }
        }
        typename PA::shared_t ti[12], tj[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ti[k] = S.acc[k][lane];
            tj[k] = S.acc[k][32 + lane];
            if constexpr (!PRESCALE) {
                ti[k] *= sc[k];
                tj[k] *= sc[k];
            }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) PA::run_add(ai[k], ti[k]);
        if (diag) {
#pragma unroll
            for (int k = 0; k < 12; ++k) PA::run_add(ai[k], tj[k]);
        } else if (sj >= 0) {
            flush12_item<PA>(frc, gdip, gquad, n_pad, sj, tj);
        }
    }
    if (curI >= 0 && curI * 32 + lane < pc.n) flush12<PA>(frc, gdip, gquad, n_pad, curI * 32 + lane, ai);
    if constexpr (VIR) block_add9<32 * fo_warps<T>()>(vacc, vir);
}

// reciprocal-space gradient and source terms per atom
// D: phi_mu derivatives [20][n_pad] then phi_M derivatives [10][n_pad] (component order of pme.cu)
// one atom's share of the reciprocal virial from its potential derivatives (layout of D as in
// k_recip_forces), its induced dipole and its global multipoles
template <class T>
__device__ __forceinline__ void recip_atom_virial(const double *__restrict__ D, const double *__restrict__ mu,
                                                  const typename V4<T>::type *__restrict__ dipd,
                                                  const typename V4<T>::type *__restrict__ quad0,
                                                  const typename V4<T>::type *__restrict__ quad1, int s, int n_pad,
                                                  double f, double *v) {
    typedef T C;
    auto Du = [&](int c) { return (C)D[(size_t)c * n_pad + s]; };
    auto DM = [&](int c) { return (C)D[(size_t)(20 + c) * n_pad + s]; };
    const C m[3] = {(C)mu[s], (C)mu[n_pad + s], (C)mu[2 * n_pad + s]};
    const typename V4<T>::type b = dipd[s], c = quad0[s], d = quad1[s];
    const C dd[3] = {b.x, b.y, b.z};
    const C Q[3][3] = {{c.x, c.y, c.z}, {c.y, c.w, d.x}, {c.z, d.x, d.y}};
    const C Hu[3][3] = {{Du(4), Du(7), Du(8)}, {Du(7), Du(5), Du(9)}, {Du(8), Du(9), Du(6)}};
    const C gu[3] = {Du(1), Du(2), Du(3)}, gM[3] = {DM(1), DM(2), DM(3)};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const C hq = Hu[a][0] * Q[0][e] + Hu[a][1] * Q[1][e] + Hu[a][2] * Q[2][e];
            v[3 * a + e] = -f * (double)((gM[a] + gu[a]) * m[e] + gu[a] * dd[e] + C(2.0 / 3.0) * hq);
        }
}

// VIR (blocks of 128 threads): also the atoms' share of the reciprocal virial,
// -f [grad phi_{M+mu} mu^T + grad phi_mu d^T + (2/3) H(phi_mu) Q]
template <class T, bool VIR>
__global__ void k_recip_forces(const double *__restrict__ D, const double *__restrict__ mu,
                               const typename V4<T>::type *__restrict__ posq,
                               const typename V4<T>::type *__restrict__ dipd,
                               const typename V4<T>::type *__restrict__ quad0,
                               const typename V4<T>::type *__restrict__ quad1, int n, int n_pad, double f,
                               double self_coef, double *__restrict__ frc, double *__restrict__ gdip,
                               double *__restrict__ gquad, int fixed, double *__restrict__ vir) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (VIR) {
        double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (s < n) recip_atom_virial<T>(D, mu, dipd, quad0, quad1, s, n_pad, f, v);
        if (fixed) {
            long long vf[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) vf[k] = ap_to_fx(v[k]);
            block_add9<128>(vf, vir);
        } else {
            block_add9<128>(v, vir);
        }
    }
    if (s >= n) return;
    typedef T C;   // FP32 in the mixed and fixed modes (FP64 is slow on this part), FP64 in AP_FP64
    auto Du = [&](int c) { return (C)D[(size_t)c * n_pad + s]; };
    auto DM = [&](int c) { return (C)D[(size_t)(20 + c) * n_pad + s]; };
    const C m[3] = {(C)mu[s], (C)mu[n_pad + s], (C)mu[2 * n_pad + s]};
    typename V4<T>::type a = posq[s], b = dipd[s], c = quad0[s], d = quad1[s];
    const C q = a.w, dd[3] = {b.x, b.y, b.z};
    const C Qxx = c.x, Qxy = c.y, Qxz = c.z, Qyy = c.w, Qyz = d.x, Qzz = d.y;
    // symmetric Hessians: index (xx yy zz xy xz yz) -> 4..9
    C Hu[3][3] = {{Du(4), Du(7), Du(8)}, {Du(7), Du(5), Du(9)}, {Du(8), Du(9), Du(6)}};
    C HM[3][3] = {{DM(4), DM(7), DM(8)}, {DM(7), DM(5), DM(9)}, {DM(8), DM(9), DM(6)}};
    const C gu[3] = {Du(1), Du(2), Du(3)};
    // sum_bc Q_bc T_abc with T the third derivatives of phi_mu
    const C Txxx = Du(10), Tyyy = Du(11), Tzzz = Du(12), Txxy = Du(13), Txxz = Du(14), Txyy = Du(15),
                 Tyyz = Du(16), Txzz = Du(17), Tyzz = Du(18), Txyz = Du(19);
    const C QT[3] = {
        Qxx * Txxx + Qyy * Txyy + Qzz * Txzz + 2 * (Qxy * Txxy + Qxz * Txxz + Qyz * Txyz),
        Qxx * Txxy + Qyy * Tyyy + Qzz * Tyzz + 2 * (Qxy * Txyy + Qxz * Txyz + Qyz * Tyyz),
        Qxx * Txxz + Qyy * Tyyz + Qzz * Tzzz + 2 * (Qxy * Txyz + Qxz * Txzz + Qyz * Tyzz)};
    for (int k = 0; k < 3; ++k) {
        C g = 0;
        for (int l = 0; l < 3; ++l) g += m[l] * (Hu[k][l] + HM[k][l]) + dd[l] * Hu[k][l];
        g += q * gu[k] + QT[k] * C(1.0 / 3.0);
        add_plain(frc, (size_t)k * n_pad + s, -f * (double)g, fixed);
        add_plain(gdip, (size_t)k * n_pad + s, f * (double)gu[k] - f * self_coef * (double)m[k], fixed);
    }
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) add_plain(gquad, (size_t)k * n_pad + s, f * (1.0 / 3.0) * (double)Hu[ia[k]][ib[k]], fixed);
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
template <class C>
__device__ __forceinline__ C dot3(const C *a, const C *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class C>
__device__ __forceinline__ void cross3(const C *a, const C *b, C *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// frame chain rule: dU/dR = G_d d_l^T + 2 G_Q R Q_l, then through the axis construction
// the chain rule of one atom's frame: forces on the atom and its z- and x-atoms; with v
// given, also its frame vectors' virial (dU/dv) v^T into v[0..8]
template <class C>
__device__ __forceinline__ void frame_chain(const double *__restrict__ gdip, const double *__restrict__ gquad,
                                            const double *__restrict__ rot, const double *__restrict__ mpl,
                                            const double *__restrict__ fvec, const int *__restrict__ frame_s, int n,
                                            int n_pad, double *__restrict__ frc, int fixed, int s, double *vout) {
    if (s >= n) return;
    const int type = frame_s[3 * s];
    if (type != AP_FRAME_Z_THEN_X && type != AP_FRAME_BISECTOR) return;
    const int zs = frame_s[3 * s + 1], xs = frame_s[3 * s + 2];
    C R[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a][b] = rot[9 * s + 3 * a + b];
    const double *m = mpl + 10 * s;
    const C dl[3] = {(C)m[1], (C)m[2], (C)m[3]};
    const C Ql[3][3] = {{(C)m[4], (C)m[5], (C)m[6]}, {(C)m[5], (C)m[7], (C)m[8]}, {(C)m[6], (C)m[8], (C)m[9]}};
    const C Gd[3] = {(C)acc_value(gdip, s, fixed), (C)acc_value(gdip, (size_t)n_pad + s, fixed),
                     (C)acc_value(gdip, (size_t)2 * n_pad + s, fixed)};
    C g6[6];
    for (int k = 0; k < 6; ++k) g6[k] = (C)acc_value(gquad, (size_t)k * n_pad + s, fixed);
    const C GQ[3][3] = {{g6[0], g6[1], g6[2]}, {g6[1], g6[3], g6[4]}, {g6[2], g6[4], g6[5]}};
    C RQ[3][3], dR[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) RQ[a][b] = R[a][0] * Ql[0][b] + R[a][1] * Ql[1][b] + R[a][2] * Ql[2][b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            dR[a][b] = Gd[a] * dl[b] + C(2) * (GQ[a][0] * RQ[0][b] + GQ[a][1] * RQ[1][b] + GQ[a][2] * RQ[2][b]);
    C gx[3], gy[3], gz[3], xa[3], za[3];
    for (int a = 0; a < 3; ++a) {
        gx[a] = dR[a][0]; gy[a] = dR[a][1]; gz[a] = dR[a][2];
        xa[a] = R[a][0]; za[a] = R[a][2];
    }
    C t[3];
    cross3(gy, za, t);
    for (int a = 0; a < 3; ++a) gx[a] += t[a];
    cross3(xa, gy, t);
    for (int a = 0; a < 3; ++a) gz[a] += t[a];
    const C vz[3] = {(C)fvec[6 * s], (C)fvec[6 * s + 1], (C)fvec[6 * s + 2]};
    const C vx[3] = {(C)fvec[6 * s + 3], (C)fvec[6 * s + 4], (C)fvec[6 * s + 5]};
    C g_vz[3], g_vx[3];
    if (type == AP_FRAME_Z_THEN_X) {
        const C vxz = dot3(vx, za);
        C w[3];
        for (int a = 0; a < 3; ++a) w[a] = vx[a] - vxz * za[a];
        // reciprocal norms with rsqrt: FP64 division and sqrt are slow on this part
        const C inw = rsq(dot3(w, w)), inz = rsq(dot3(vz, vz));
        const C gxx = dot3(gx, xa);
        C gw[3];
        for (int a = 0; a < 3; ++a) gw[a] = (gx[a] - gxx * xa[a]) * inw;
        const C gwz = dot3(gw, za);
        for (int a = 0; a < 3; ++a) {
            g_vx[a] = gw[a] - gwz * za[a];
            gz[a] = gz[a] - gwz * vx[a] - vxz * gw[a];
        }
        const C gzz = dot3(gz, za);
        for (int a = 0; a < 3; ++a) g_vz[a] = (gz[a] - gzz * za[a]) * inz;
    } else {
        const C in1 = rsq(dot3(vz, vz)), in2 = rsq(dot3(vx, vx));
        C u1[3], u2[3], sv[3], w[3];
        for (int a = 0; a < 3; ++a) { u1[a] = vz[a] * in1; u2[a] = vx[a] * in2; sv[a] = u1[a] + u2[a]; }
        const C u2z = dot3(u2, za);
        for (int a = 0; a < 3; ++a) w[a] = u2[a] - u2z * za[a];
        const C inw = rsq(dot3(w, w)), ins = rsq(dot3(sv, sv));
        const C gxx = dot3(gx, xa);
        C gw[3], gu2[3], gs[3];
        for (int a = 0; a < 3; ++a) gw[a] = (gx[a] - gxx * xa[a]) * inw;
        const C gwz = dot3(gw, za);
        for (int a = 0; a < 3; ++a) {
            gu2[a] = gw[a] - gwz * za[a];
            gz[a] = gz[a] - gwz * u2[a] - u2z * gw[a];
        }
        const C gzz = dot3(gz, za);
        for (int a = 0; a < 3; ++a) gs[a] = (gz[a] - gzz * za[a]) * ins;
        for (int a = 0; a < 3; ++a) gu2[a] += gs[a];
        const C a1 = dot3(gs, u1), a2 = dot3(gu2, u2);
        for (int a = 0; a < 3; ++a) {
            g_vz[a] = (gs[a] - a1 * u1[a]) * in1;
            g_vx[a] = (gu2[a] - a2 * u2[a]) * in2;
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (fixed) {
            unsigned long long *fx = reinterpret_cast<unsigned long long *>(frc);
            atomicAdd(fx + a * n_pad + zs, (unsigned long long)ap_to_fx(-(double)g_vz[a]));
            atomicAdd(fx + a * n_pad + xs, (unsigned long long)ap_to_fx(-(double)g_vx[a]));
            atomicAdd(fx + a * n_pad + s, (unsigned long long)ap_to_fx((double)g_vz[a] + (double)g_vx[a]));
        } else {
            atomicAdd(frc + a * n_pad + zs, -(double)g_vz[a]);
            atomicAdd(frc + a * n_pad + xs, -(double)g_vx[a]);
            atomicAdd(frc + a * n_pad + s, (double)g_vz[a] + (double)g_vx[a]);
        }
    }
    if (vout) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                vout[3 * a + b] = (double)g_vz[a] * (double)vz[b] + (double)g_vx[a] * (double)vx[b];
    }
}

// VIR (blocks of 128 threads): also the frames' share of the virial, sum over the frame
// vectors v of (dU/dv) v^T
template <class C, bool VIR>
__global__ void k_frame_forces(const double *__restrict__ gdip, const double *__restrict__ gquad,
                               const double *__restrict__ rot, const double *__restrict__ mpl,
                               const double *__restrict__ fvec, const int *__restrict__ frame_s, int n, int n_pad,
                               double *__restrict__ frc, int fixed, double *__restrict__ vir) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    frame_chain<C>(gdip, gquad, rot, mpl, fvec, frame_s, n, n_pad, frc, fixed, s, VIR ? v : nullptr);
    if constexpr (VIR) {
        if (fixed) {
            long long vf[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) vf[k] = ap_to_fx(v[k]);
            block_add9<128>(vf, vir);
        } else {
            block_add9<128>(v, vir);
        }
    }
}

template <class T>
__global__ void k_mu_load(const double *__restrict__ mu_in, const int *__restrict__ perm, int n, int n_pad,
                          double *__restrict__ mu_s, typename V4<T>::type *__restrict__ p) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    double m[3] = {0, 0, 0};
    if (s < n) {
        int i = perm[s];
        for (int c = 0; c < 3; ++c) m[c] = mu_in[3 * i + c];
    }
    for (int c = 0; c < 3; ++c) mu_s[c * n_pad + s] = m[c];
    typename V4<T>::type v;
    v.x = (T)m[0]; v.y = (T)m[1]; v.z = (T)m[2]; v.w = (T)0;
    p[s] = v;
}

__global__ void k_energy(const double *__restrict__ mu, const double *__restrict__ E, int n_pad, double scale,
                         double *__restrict__ out, int fixed) {
    __shared__ double sm[8];
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (s < n_pad)
        for (int c = 0; c < 3; ++c) v += mu[c * n_pad + s] * E[c * n_pad + s];
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        if (fixed)   // energy in fixed point with 30 fractional bits: order-independent sum
            atomicAdd(reinterpret_cast<unsigned long long *>(out), (unsigned long long)llrint(scale * t * 1073741824.0));
        else
            atomicAdd(out, scale * t);
    }
}

// fixed-point energy (30 fractional bits) -> FP64
__global__ void k_energy_out(const double *__restrict__ e, double *__restrict__ out) {
    *out = (double)*reinterpret_cast<const long long *>(e) * (1.0 / 1073741824.0);
}

// force accumulators in fixed point, sorted slots -> FP64, caller order
__global__ void k_unsort3_fx(const double *__restrict__ src, int n_pad, const int *__restrict__ iperm, int n,
                             double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = iperm[i];
    for (int c = 0; c < 3; ++c) out[3 * i + c] = acc_value(src, (size_t)c * n_pad + s, 1);
}

// the real-space force kernel over the current work items with the dipoles in ctx->p and
// the multipoles (posq q, dipd, quad0, quad1) given, accumulating into frc, gdip and gquad;
// with vir given, also the pairs' virial into vir[0..8]
template <class T>
int pair_forces_t(ap_ctx *ctx, cudaStream_t s, const void *posq, const void *dipd, const void *quad0,
                  const void *quad1, double *frc, double *gdip, double *gquad, double *vir = nullptr) {
    typedef typename V4<T>::type T4;
    PairConsts<T> pc;
    const ap_params &P = ctx->prm;
    const double b = P.ewald_beta;
    pc.beta = (T)b;
    pc.c[0] = 0;
    for (int k = 1; k <= 4; ++k) pc.c[k] = (T)(std::pow(2.0 * b * b, k) / (b * AP_SQRT_PI));
    pc.thole_a = (T)P.thole_a;
    pc.rc2 = (T)(P.cutoff * P.cutoff);
    for (int dd = 0; dd < 3; ++dd) { pc.L[dd] = (T)P.box[dd]; pc.iL[dd] = (T)(1.0 / P.box[dd]); }
    pc.n = ctx->n;
    typedef void (*Kern)(WorkArgs, const T4 *, const T4 *, const T4 *, const T4 *, const T4 *, double *, double *,
                         double *, int, PairConsts<T>, double, double *);
    static const Kern kerns[8] = {k_pair_forces<T, false, false, false>, k_pair_forces<T, true, false, false>,
                                  k_pair_forces<T, false, true, false>,  k_pair_forces<T, true, true, false>,
                                  k_pair_forces<T, false, false, true>,  k_pair_forces<T, true, false, true>,
                                  k_pair_forces<T, false, true, true>,   k_pair_forces<T, true, true, true>};
    const int which = ctx->minimg + 2 * ctx->fixed + 4 * (vir ? 1 : 0);
    const Kern kern = kerns[which];
    static int grids[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int &grid = grids[which];
    if (!grid) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * fo_warps<T>(), 0);
        grid = std::max(1, per_sm) * ctx->sm_count;
    }
    kern<<<grid, 32 * fo_warps<T>(), 0, s>>>(work_args(ctx), (const T4 *)posq, (const T4 *)dipd,
                                            (const T4 *)quad0, (const T4 *)quad1, (const T4 *)ctx->p,
                                            frc, gdip, gquad, ctx->n_pad, pc, AP_COULOMB, vir);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// `extra`, if given, runs on the force stream after the pair and reciprocal terms and before
// the frame chain rule: it may add to ctx->frc, ctx->gdip and ctx->gquad (and, while
// ctx->vir_active is set, to that virial accumulator). vir: nine device slots (FP64, or fixed
// point in AP_FIXED) cleared here and accumulating the virial, or NULL.
template <class T>
int forces_t(ap_ctx *ctx, const double *d_mu, double *d_energy, double *d_forces,
             int (*extra)(ap_ctx *, cudaStream_t), double *vir) {
    typedef typename V4<T>::type T4;
    cudaStream_t s = ctx->s0;
    const int n = ctx->n, n_pad = ctx->n_pad;
    const double f = AP_COULOMB;
    const double self_coef = 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI);
    if (vir) AP_CUDA(cudaMemsetAsync(vir, 0, sizeof(double) * 9, s));
    k_mu_load<T><<<ap_grid_for(n_pad, 256), 256, 0, s>>>(d_mu, ctx->perm, n, n_pad, ctx->mu_s, (T4 *)ctx->p);
    // reciprocal-space potential derivatives on the second stream, concurrent with the
    // energy and the real-space pair forces (they write only gbuf and the grid); joined
    // before the kernels that update the force arrays per atom
    AP_CUDA(cudaEventRecord(ctx->ev_fork, s));
    AP_CUDA(cudaStreamWaitEvent(ctx->s1, ctx->ev_fork, 0));
    int rc = pme_forces_derivs(ctx, ctx->p, ctx->gbuf, ctx->s1, vir);
    if (rc) return rc;
    AP_CUDA(cudaMemsetAsync(ctx->frc, 0, sizeof(double) * 3 * n_pad, s));
    AP_CUDA(cudaMemsetAsync(ctx->gdip, 0, sizeof(double) * 3 * n_pad, s));
    AP_CUDA(cudaMemsetAsync(ctx->gquad, 0, sizeof(double) * 6 * n_pad, s));
    AP_CUDA(cudaMemsetAsync(ctx->red + 8, 0, sizeof(double), s));
    // energy
    k_energy<<<ap_grid_for(n_pad, 256), 256, 0, s>>>(ctx->mu_s, ctx->E, n_pad, -0.5 * f, ctx->red + 8, ctx->fixed);
    rc = pair_forces_t<T>(ctx, s, ctx->posq, ctx->dipd, ctx->quad0, ctx->quad1, ctx->frc, ctx->gdip, ctx->gquad, vir);
    if (rc) return rc;
    AP_CUDA(cudaEventRecord(ctx->ev_join, ctx->s1));
    AP_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    auto krec = vir ? k_recip_forces<T, true> : k_recip_forces<T, false>;
    krec<<<ap_grid_for(n, 128), 128, 0, s>>>(ctx->gbuf, ctx->mu_s, (const T4 *)ctx->posq, (const T4 *)ctx->dipd,
                                            (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, n, n_pad, f, self_coef,
                                            ctx->frc, ctx->gdip, ctx->gquad, ctx->fixed, vir);
    AP_CUDA(cudaGetLastError());
    ctx->vir_active = vir;
    rc = extra ? extra(ctx, s) : AP_OK;
    ctx->vir_active = nullptr;
    if (rc) return rc;
    auto kfr = vir ? k_frame_forces<T, true> : k_frame_forces<T, false>;
    kfr<<<ap_grid_for(n, 128), 128, 0, s>>>(ctx->gdip, ctx->gquad, ctx->rot, ctx->mpl, ctx->fvec, ctx->frame_s, n,
                                           n_pad, ctx->frc, ctx->fixed, vir);
    AP_CUDA(cudaGetLastError());
    if (ctx->fixed) {
        k_unsort3_fx<<<ap_grid_for(n, 256), 256, 0, s>>>(ctx->frc, n_pad, ctx->iperm, n, d_forces);
        k_energy_out<<<1, 1, 0, s>>>(ctx->red + 8, d_energy);
    } else {
        unsort3(ctx, ctx->frc, d_forces, s);
        AP_CUDA(cudaMemcpyAsync(d_energy, ctx->red + 8, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// forces of the mutual term alone, -(f/2) mu . T mu, for caller-order dipoles d_mu: the
// single-set force path with the permanent multipoles replaced by zeros (mz: posq, dipd,
// quad0, quad1 with q, d and Q zero, positions and Thole factors kept) and without the
// permanent potential's reciprocal part or the frame chain rule. gd, gq: scratch for the
// dipole and quadrupole derivatives the kernels also write (not used). vir: as in forces_t.
template <class T>
int mutual_forces_t(ap_ctx *ctx, const double *d_mu, void *const *mz, double *gd, double *gq, double *d_forces,
                    double *vir) {
    typedef typename V4<T>::type T4;
    cudaStream_t s = ctx->s0;
    const int n = ctx->n, n_pad = ctx->n_pad;
    const double f = AP_COULOMB;
    const double self_coef = 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI);
    if (vir) AP_CUDA(cudaMemsetAsync(vir, 0, sizeof(double) * 9, s));
    k_mu_load<T><<<ap_grid_for(n_pad, 256), 256, 0, s>>>(d_mu, ctx->perm, n, n_pad, ctx->mu_s, (T4 *)ctx->p);
    AP_CUDA(cudaMemsetAsync(ctx->frc, 0, sizeof(double) * 3 * n_pad, s));
    AP_CUDA(cudaMemsetAsync(gd, 0, sizeof(double) * 3 * n_pad, s));
    AP_CUDA(cudaMemsetAsync(gq, 0, sizeof(double) * 6 * n_pad, s));
    AP_CUDA(cudaEventRecord(ctx->ev_fork, s));
    AP_CUDA(cudaStreamWaitEvent(ctx->s1, ctx->ev_fork, 0));
    int rc = pme_forces_derivs_mu(ctx, ctx->p, ctx->gbuf, ctx->s1, vir);
    if (rc) return rc;
    rc = pair_forces_t<T>(ctx, s, mz[0], mz[1], mz[2], mz[3], ctx->frc, gd, gq, vir);
    if (rc) return rc;
    AP_CUDA(cudaEventRecord(ctx->ev_join, ctx->s1));
    AP_CUDA(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    auto krec = vir ? k_recip_forces<T, true> : k_recip_forces<T, false>;
    krec<<<ap_grid_for(n, 128), 128, 0, s>>>(ctx->gbuf, ctx->mu_s, (const T4 *)mz[0], (const T4 *)mz[1],
                                            (const T4 *)mz[2], (const T4 *)mz[3], n, n_pad, f, self_coef, ctx->frc,
                                            gd, gq, ctx->fixed, vir);
    AP_CUDA(cudaGetLastError());
    if (ctx->fixed)
        k_unsort3_fx<<<ap_grid_for(n, 256), 256, 0, s>>>(ctx->frc, n_pad, ctx->iperm, n, d_forces);
    else
        unsort3(ctx, ctx->frc, d_forces, s);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// d_out[0..8] = value(a) - value(b) (b optional) of two virial accumulators in FP64 or (fixed)
// fixed point
__global__ void k_virial_out(const double *__restrict__ a, const double *__restrict__ b, int fixed,
                             double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 9) return;
    double v = acc_value(a, k, fixed);
    if (b) v -= acc_value(b, k, fixed);
    out[k] = v;
}

}  // namespace

int pair_forces_launch(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64
               ? pair_forces_t<double>(ctx, s, ctx->posq, ctx->dipd, ctx->quad0, ctx->quad1, ctx->frc, ctx->gdip,
                                       ctx->gquad)
               : pair_forces_t<float>(ctx, s, ctx->posq, ctx->dipd, ctx->quad0, ctx->quad1, ctx->frc, ctx->gdip,
                                      ctx->gquad);
}

int mutual_forces_run(ap_ctx *ctx, const double *d_mu, void *const *mz, double *gd, double *gq, double *d_forces,
                      double *vir) {
    return ctx->prec == AP_FP64 ? mutual_forces_t<double>(ctx, d_mu, mz, gd, gq, d_forces, vir)
                                : mutual_forces_t<float>(ctx, d_mu, mz, gd, gq, d_forces, vir);
}

// the virial accumulators: slots 16..24 of the context's reduction scratch for a force call,
// 32..40 for the mutual pass of the two-set forces
double *virial_acc(ap_ctx *ctx, int which) { return ctx->red + (which ? 32 : 16); }

int virial_out(ap_ctx *ctx, const double *a, const double *b, double *d_virial) {
    k_virial_out<<<1, 32, 0, ctx->s0>>>(a, b, ctx->fixed, d_virial);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int forces_run(ap_ctx *ctx, const double *d_mu, double *d_energy, double *d_forces, double *d_virial) {
    double *vir = d_virial ? virial_acc(ctx, 0) : nullptr;
    const int rc = ctx->prec == AP_FP64 ? forces_t<double>(ctx, d_mu, d_energy, d_forces, nullptr, vir)
                                        : forces_t<float>(ctx, d_mu, d_energy, d_forces, nullptr, vir);
    if (rc || !d_virial) return rc;
    return virial_out(ctx, vir, nullptr, d_virial);
}

int forces_run_ex(ap_ctx *ctx, const double *d_mu, double *d_energy, double *d_forces,
                  int (*extra)(ap_ctx *, cudaStream_t), double *vir) {
    return ctx->prec == AP_FP64 ? forces_t<double>(ctx, d_mu, d_energy, d_forces, extra, vir)
                                : forces_t<float>(ctx, d_mu, d_energy, d_forces, extra, vir);
}
