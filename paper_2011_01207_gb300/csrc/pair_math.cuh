// Radial functions of one atom pair, shared by the real-space tile kernels.
//
// Screened:  B_0 = erfc(beta r)/r,  B_n = [(2n-1) B_{n-1} + (2 beta^2)^n e^{-beta^2 r^2}/(beta sqrt(pi))] / r^2
// Coulomb:   U_n = (2n-1)!! / r^(2n+1)
// Thole:     s = a r^3 / sqrt(alpha_i alpha_j),  1 - lambda_3 = e^-s, 1 - lambda_5 = (1+s) e^-s,
//            1 - lambda_7 = (1 + s + 3/5 s^2) e^-s, 1 - lambda_9 = (1 + s + 18/35 s^2 + 9/35 s^3) e^-s
// Kernel:    R_n = B_n - (1 - sigma lambda_{2n+1}) U_n  (sigma = 1, or 0 for excluded pairs)
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

__device__ __forceinline__ float ap_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double ap_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float ap_exp(float x) { return expf(x); }
__device__ __forceinline__ double ap_exp(double x) { return exp(x); }
__device__ __forceinline__ float ap_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double ap_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float ap_rint(float x) { return rintf(x); }
__device__ __forceinline__ double ap_rint(double x) { return rint(x); }

template <class T>
struct PairConsts {
    T beta;            // Ewald beta
    T c[5];            // c[n] = (2 beta^2)^n / (beta sqrt(pi)), n = 1..4 (c[0] unused)
    T thole_a;
    T rc2;             // cutoff^2
    T L[3], iL[3];     // box and its inverse
    int n;             // real atoms; slots >= n are padding
};

// pair vector R = x_i - x_j: minimum image per pair (MINIMG), or plus a fixed image shift
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

// erfc(x) given e2 = exp(-x^2), x >= 0. FP32: the rational approximation of Abramowitz &
// Stegun, Handbook of Mathematical Functions (1964), formula 7.1.26,
//   erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},  t = 1 / (1 + p x),
// absolute error <= 1.5e-7, which reuses the e^{-x^2} the recursion needs anyway.
// FP64: the library erfc.
__device__ __forceinline__ float erfc_e2(float x, float e2) {
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f),
                                         -0.284496736f), 0.254829592f);
    return poly * e2;
}
__device__ __forceinline__ double erfc_e2(double x, double) { return erfc(x); }
__device__ __forceinline__ float ap_fexp(float x) { return __expf(x); }
__device__ __forceinline__ double ap_fexp(double x) { return exp(x); }

// Packed FP32 pairs: the f32x2 add/sub/mul/fma instructions of sm_100 and later do two FP32
// operations in one issue slot. The pair kernels are issue-bound, so two pair sides
// evaluated side by side in the two halves of each register pair take about half the
// issue slots of their radial arithmetic. The special-function unit has no packed form:
// 2^x and 1/x are the PTX approximations applied to each half.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 ex2_2(float2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

// Constants of the packed radial terms, from PairConsts<float>: the exponents are taken to
// base 2 (e^-y = 2^(-y log2 e)), so each exponential is one multiply and one 2^x.
struct PairConsts2 {
    float2 ce;        // -beta^2 log2(e): e^{-beta^2 r^2} = 2^{ce r^2}
    float2 pb;        // A&S 7.1.26's p times beta: t = 1 / (1 + pb r)
    float2 c1, c2, c3, c4;   // (2 beta^2)^n / (beta sqrt(pi)), n = 1..4
    float2 ta;        // Thole a
    float2 nl2e;      // -log2(e)
};
__host__ __device__ inline PairConsts2 make_consts2(const PairConsts<float> &pc) {
    const float l2e = 1.4426950408889634f;
    PairConsts2 k;
    k.ce = make_float2(-pc.beta * pc.beta * l2e, -pc.beta * pc.beta * l2e);
    k.pb = make_float2(0.3275911f * pc.beta, 0.3275911f * pc.beta);
    k.c1 = make_float2(pc.c[1], pc.c[1]);
    k.c2 = make_float2(pc.c[2], pc.c[2]);
    k.c3 = make_float2(pc.c[3], pc.c[3]);
    k.c4 = make_float2(pc.c[4], pc.c[4]);
    k.ta = make_float2(pc.thole_a, pc.thole_a);
    k.nl2e = make_float2(-l2e, -l2e);
    return k;
}

// R_1, R_2 of the dipole operator (sigma = 1) for two pair sides at once, from r^2 and the
// sides' Thole factor products ww = w_target w_source: the same terms as screened<float, 2>
// and thole_oml<float, 2>, with erfc from A&S 7.1.26.
__device__ __forceinline__ void radial12_x2(const PairConsts2 &k, float2 r2, float2 ww, float2 &R1, float2 &R2) {
    const float2 rinv = rsqrt2(r2);
    const float2 r = mul2(r2, rinv), rinv2 = mul2(rinv, rinv);
    const float2 e2 = ex2_2(mul2(r2, k.ce));
    const float2 t = rcp2(fma2(k.pb, r, splat2(1.0f)));
    const float2 poly = mul2(t, fma2(t, fma2(t, fma2(t, fma2(t, splat2(1.061405429f), splat2(-1.453152027f)),
                                                      splat2(1.421413741f)),
                                             splat2(-0.284496736f)),
                                     splat2(0.254829592f)));
    const float2 b0 = mul2(mul2(poly, e2), rinv);
    const float2 b1 = mul2(fma2(k.c1, e2, b0), rinv2);
    const float2 u1 = mul2(rinv, rinv2);
    const float2 r3 = mul2(splat2(3.0f), rinv2);
    const float2 b2 = mul2(fma2(splat2(3.0f), b1, mul2(k.c2, e2)), rinv2);
    const float2 u2 = mul2(u1, r3);
    const float2 s = mul2(mul2(r2, r), mul2(ww, k.ta));
    const float2 e = ex2_2(mul2(s, k.nl2e));
    const float2 oml1 = fma2(s, e, e);
    R1 = sub2(b1, mul2(e, u1));
    R2 = sub2(b2, mul2(oml1, u2));
}

// Screened B_1..B_nmax and Coulomb U_1..U_nmax at r (rinv = 1/r, rinv2 = 1/r^2).
template <class T, int NMAX>
__device__ __forceinline__ void screened(const PairConsts<T> &pc, T r, T rinv, T rinv2, T *B, T *U) {
    T x = pc.beta * r;
    T e2 = ap_fexp(-x * x);
    T b = erfc_e2(x, e2) * rinv;
    T u = rinv;
#pragma unroll
    for (int k = 1; k <= NMAX; ++k) {
        b = (T(2 * k - 1) * b + pc.c[k] * e2) * rinv2;
        u = T(2 * k - 1) * u * rinv2;
        B[k - 1] = b;
        U[k - 1] = u;
    }
}

// 1 - lambda_{2k+1} for k = 1..NMAX from the Thole argument s
template <class T, int NMAX>
__device__ __forceinline__ void thole_oml(T s, T *oml) {
    T e = ap_fexp(-s);
    oml[0] = e;
    if (NMAX > 1) oml[1] = (T(1) + s) * e;
    if (NMAX > 2) oml[2] = (T(1) + s + T(0.6) * s * s) * e;
    if (NMAX > 3) oml[3] = (T(1) + s + s * s * (T(18.0 / 35.0) + T(9.0 / 35.0) * s)) * e;
}

// R_1, R_2, R_3 with the scale sigma of each side (exa, exb: excluded pairs, sigma = 0, whose
// R_n = B_n - U_n), for two pair sides at once: the terms of screened<float, 3> and
// thole_oml<float, 3>
__device__ __forceinline__ void radial123_x2(const PairConsts2 &k, float2 r2, float2 ww, bool exa, bool exb,
                                             float2 &R1, float2 &R2, float2 &R3) {
    const float2 rinv = rsqrt2(r2);
    const float2 r = mul2(r2, rinv), rinv2 = mul2(rinv, rinv);
    const float2 e2 = ex2_2(mul2(r2, k.ce));
    const float2 t = rcp2(fma2(k.pb, r, splat2(1.0f)));
    const float2 poly = mul2(t, fma2(t, fma2(t, fma2(t, fma2(t, splat2(1.061405429f), splat2(-1.453152027f)),
                                                      splat2(1.421413741f)),
                                             splat2(-0.284496736f)),
                                     splat2(0.254829592f)));
    const float2 b0 = mul2(mul2(poly, e2), rinv);
    const float2 b1 = mul2(fma2(k.c1, e2, b0), rinv2);
    const float2 u1 = mul2(rinv, rinv2);
    const float2 b2 = mul2(fma2(splat2(3.0f), b1, mul2(k.c2, e2)), rinv2);
    const float2 u2 = mul2(mul2(splat2(3.0f), u1), rinv2);
    const float2 b3 = mul2(fma2(splat2(5.0f), b2, mul2(k.c3, e2)), rinv2);
    const float2 u3 = mul2(mul2(splat2(5.0f), u2), rinv2);
    const float2 s = mul2(mul2(r2, r), mul2(ww, k.ta));
    const float2 e = ex2_2(mul2(s, k.nl2e));
    const float2 s1 = add2(splat2(1.0f), s);
    float2 o1 = e, o2 = mul2(s1, e), o3 = mul2(fma2(splat2(0.6f), mul2(s, s), s1), e);
    if (exa) o1.x = o2.x = o3.x = 1.0f;
    if (exb) o1.y = o2.y = o3.y = 1.0f;
    R1 = sub2(b1, mul2(o1, u1));
    R2 = sub2(b2, mul2(o2, u2));
    R3 = sub2(b3, mul2(o3, u3));
}

// The force kernel's radial terms for two pair sides at once: Rd_n = B_n - (1 - sigma
// lambda_(2n+1)) U_n for n = 1..4 with each side's exclusion scale (exa, exb: sigma = 0),
// and Ru_n = B_n - (1 - lambda_(2n+1)) U_n for n = 1..3 (sigma = 1); the terms of
// screened<float, 4> and thole_oml<float, 4>
__device__ __forceinline__ void radial_forces_x2(const PairConsts2 &k, float2 r2, float2 ww, bool exa, bool exb,
                                                 float2 *Rd, float2 *Ru) {
    const float2 rinv = rsqrt2(r2);
    const float2 r = mul2(r2, rinv), rinv2 = mul2(rinv, rinv);
    const float2 e2 = ex2_2(mul2(r2, k.ce));
    const float2 t = rcp2(fma2(k.pb, r, splat2(1.0f)));
    const float2 poly = mul2(t, fma2(t, fma2(t, fma2(t, fma2(t, splat2(1.061405429f), splat2(-1.453152027f)),
                                                      splat2(1.421413741f)),
                                             splat2(-0.284496736f)),
                                     splat2(0.254829592f)));
    const float2 b0 = mul2(mul2(poly, e2), rinv);
    float2 b[4], u[4];
    b[0] = mul2(fma2(k.c1, e2, b0), rinv2);
    u[0] = mul2(rinv, rinv2);
    b[1] = mul2(fma2(splat2(3.0f), b[0], mul2(k.c2, e2)), rinv2);
    u[1] = mul2(mul2(splat2(3.0f), u[0]), rinv2);
    b[2] = mul2(fma2(splat2(5.0f), b[1], mul2(k.c3, e2)), rinv2);
    u[2] = mul2(mul2(splat2(5.0f), u[1]), rinv2);
    b[3] = mul2(fma2(splat2(7.0f), b[2], mul2(k.c4, e2)), rinv2);
    u[3] = mul2(mul2(splat2(7.0f), u[2]), rinv2);
    const float2 s = mul2(mul2(r2, r), mul2(ww, k.ta));
    const float2 e = ex2_2(mul2(s, k.nl2e));
    const float2 s1 = add2(splat2(1.0f), s), ss = mul2(s, s);
    float2 o[4];
    o[0] = e;
    o[1] = mul2(s1, e);
    o[2] = mul2(fma2(splat2(0.6f), ss, s1), e);
    o[3] = mul2(fma2(ss, fma2(splat2(9.0f / 35.0f), s, splat2(18.0f / 35.0f)), s1), e);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const float2 ru = sub2(b[n], mul2(o[n], u[n])), rx = sub2(b[n], u[n]);
        if (n < 3) Ru[n] = ru;
        Rd[n] = make_float2(exa ? rx.x : ru.x, exb ? rx.y : ru.y);
    }
}

// First index i in [lo, hi] with start[i] >= a, for a nondecreasing start[] with
// start[hi] >= a and start[i] < a for every i < lo; the 32 lanes of a warp search together,
// each round testing 32 evenly spaced entries of the interval (one load per lane) and
// keeping the 1/32 of it where the answer lies, so the dependent loads number
// log32(hi - lo) + 1 instead of log2(hi - lo).
__device__ __forceinline__ long warp_lower_bound(const int *__restrict__ start, long lo, long hi, long a, int lane) {
    while (hi - lo > 32) {
        const long step = (hi - lo + 31) >> 5;                       // sample j at lo + (j + 1) step
        const long idx = min(lo + (long)(lane + 1) * step, hi);      // lane 31's sample is hi itself
        const unsigned ge = __ballot_sync(0xffffffffu, start[idx] >= a);
        const int k = __ffs(ge) - 1;                                 // first sample at or above a
        const long nhi = min(lo + (long)(k + 1) * step, hi);
        if (k > 0) lo += (long)k * step + 1;                         // sample k - 1 was below a
        hi = nhi;
    }
    const long idx = lo + lane;
    const unsigned ge = __ballot_sync(0xffffffffu, idx < hi && start[idx] >= a);
    return ge ? lo + __ffs(ge) - 1 : hi;
}

// Items [t0, t1) of warp gw of nw: consecutive items holding an equal share of the total
// item weight (in-range pairs plus a fixed staging cost per item, as exclusive prefix sums),
// so that warps get equal work whatever the pair density of their items; item order
// (grouped by block I) is kept. Called by all 32 lanes of the warp together; the end is
// looked for first among the 32 items from t0, where it nearly always is.
__device__ __forceinline__ void work_range(const WorkArgs &wa, long gw, long nw, long &t0, long &t1) {
    const int lane = threadIdx.x & 31;
    const long nitems = *wa.n_work;
    const long total = wa.item_start[nitems];
    const long a = total * gw / nw, b = total * (gw + 1) / nw;
    t0 = warp_lower_bound(wa.item_start, 0, nitems, a, lane);
    if (gw == nw - 1) {
        t1 = nitems;
        return;
    }
    const long idx = t0 + lane;
    const unsigned ge = __ballot_sync(0xffffffffu, idx < nitems && wa.item_start[idx] >= b);
    if (ge) t1 = t0 + __ffs(ge) - 1;
    else t1 = t0 + 32 >= nitems ? nitems : warp_lower_bound(wa.item_start, t0 + 32, nitems, b, lane);
}

// Pair sides of one 32 x 32 work item, walked in place (one warp). Word w < 32 is row i = w
// (bits: the item's j atoms in range of i), word 32 + j the column of j (bits: the i atoms);
// the target of a side in word w is atom w of the item's 64 (i atoms first) and its source
// atom b + 32 or b for bit b of a row or column word. In word order the sides are sorted by
// target, and lane l owns the l-th of 32 equal contiguous shares of them.
//
// side_start() (run once per configuration, with the masks) finds where lane `lane`'s share
// starts and packs it: the word (bits 0-5), the position of its first bit in that word
// (bits 6-10) and the number of sides in the share (bits 11-31; at most 64). All 32 lanes
// call it together, each with its row word `row` and column word `col`.
__device__ __forceinline__ unsigned side_start(unsigned row, unsigned col, int lane) {
    // inclusive prefix counts of the row words (low half) and of the column words (high
    // half) in one scan: each count is at most 32 * 32, so the halves never carry
    int v = __popc(row) | (__popc(col) << 16);
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    const int last = __shfl_sync(0xffffffffu, v, 31);
    const int nrow = last & 0xffff, total = nrow + (last >> 16);
    const int per = (total + 31) >> 5;
    const int e0 = min(total, lane * per);
    const int left = min(total, e0 + per) - e0;
    // inclusive prefix of word w: lane w's low half, or the rows' total plus lane (w - 32)'s
    // high half
    auto prefix = [&](int w) {
        const int u = __shfl_sync(0xffffffffu, v, w & 31);
        return w < 32 ? (u & 0xffff) : nrow + (u >> 16);
    };
    // first word whose inclusive prefix exceeds e0
    int lo = 0, hi = 63;
    for (int r = 0; r < 6; ++r) {   // 64 words: six halvings (lo == hi after the last)
        const int mid = (lo + hi) >> 1;
        const int pm = prefix(mid);
        if (lo < hi) {
            if (pm > e0) hi = mid; else lo = mid + 1;
        }
    }
    const int pb = prefix(max(lo - 1, 0));   // every lane shuffles (warp-collective)
    const int before = lo > 0 ? pb : 0;
    const int pick = lo & 31;
    const unsigned wr = __shfl_sync(0xffffffffu, row, pick), wc = __shfl_sync(0xffffffffu, col, pick);
    unsigned m = lo < 32 ? wr : wc;
    for (int k = e0 - before; k > 0; --k) m &= m - 1u;   // skip the sides before e0
    const int pos = left > 0 ? __ffs(m) - 1 : 0;
    const int w = left > 0 ? lo : 0;
    return (unsigned)w | ((unsigned)pos << 6) | ((unsigned)left << 11);
}

struct SideSlice {
    int w;         // current word
    unsigned m;    // its bits not yet taken
    int left;      // sides left in this lane's share

    // stages the item's 64 words (row, col: this lane's) in shared memory and places the
    // lane at its share's start (`start` from side_start)
    __device__ __forceinline__ void load(unsigned row, unsigned col, unsigned start, int lane, unsigned *words) {
        words[lane] = row;
        words[32 + lane] = col;
        __syncwarp();
        w = start & 63;
        left = (int)(start >> 11);
        m = left > 0 ? words[w] & (~0u << ((start >> 6) & 31)) : 0u;
    }
    // next side: target word, source bit; advances over empty words
    __device__ __forceinline__ void next(const unsigned *words, int &target, int &source) {
        while (m == 0u) m = words[++w];
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        --left;
        target = w;
        source = w < 32 ? b + 32 : b;
    }
};

// Exact FP32 -> FP64 conversion with integer operations only (FP64 instructions issue at a
// small fraction of the FP32 rate on this part): the sign, the exponent rebased from 127 to
// 1023 and the 23 mantissa bits moved to the top of the 52. Zero and subnormal inputs
// (below 1.2e-38) give a signed zero; infinities and NaNs keep their class.
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu, s = u & 0x80000000u, m = u & 0x7fffffu;
    unsigned hi = s | ((e + 896u) << 20) | (m >> 3);
    hi = e == 0u ? s : hi;
    hi = e == 0xffu ? (s | 0x7ff00000u | (m >> 3)) : hi;
    const unsigned lo = e == 0u ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// Compensated FP32 sum hi + lo: each addition is Knuth's TwoSum (the rounding error of
// hi + x, recovered exactly in FP32, is added to lo), so the pair carries ~48 bits.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ void f2_add(F2 &a, float x) {
    const float t = a.hi + x;
    const float z = t - a.hi;
    a.lo += (a.hi - (t - z)) + (x - z);
    a.hi = t;
}

// Accumulation of the pair kernels' partial sums. Per-target sums of an item are kept in
// shared memory (shared_t; plain stores by a target's only leaving lane, atomics for the
// last targets), running sums across items in registers (run_t), and both are added to the
// global FP64 accumulators with FP64 atomics:
//   FP64 mode: everything in FP64;
//   mixed mode: items in FP32, running sums in a compensated FP32 pair, converted to FP64
//     exactly once per flush, so the per-item path issues no FP64 instruction;
//   FX = true (AP_FIXED): 64-bit fixed point throughout (integer additions, so the totals do
//     not depend on their order); the global accumulators then hold fixed-point integers
//     in the same 8-byte slots.
template <class T, bool FX>
struct PairAcc;
template <>
struct PairAcc<double, false> {
    typedef double shared_t;
    typedef double run_t;
    static __device__ __forceinline__ void shared_add(shared_t *p, double v) { atomicAdd(p, v); }
    static __device__ __forceinline__ void shared_put(shared_t *p, double v) { *p = v; }
    static __device__ __forceinline__ void run_zero(run_t &r) { r = 0.0; }
    static __device__ __forceinline__ void run_add(run_t &r, shared_t v) { r += v; }
    static __device__ __forceinline__ void run_flush(double *p, const run_t &r) { atomicAdd(p, r); }
    static __device__ __forceinline__ void item_flush(double *p, shared_t v) { atomicAdd(p, v); }
};
template <>
struct PairAcc<float, false> {
    typedef float shared_t;
    typedef F2 run_t;
    static __device__ __forceinline__ void shared_add(shared_t *p, float v) { atomicAdd(p, v); }
    static __device__ __forceinline__ void shared_put(shared_t *p, float v) { *p = v; }
    static __device__ __forceinline__ void run_zero(run_t &r) { r.hi = r.lo = 0.f; }
    static __device__ __forceinline__ void run_add(run_t &r, shared_t v) { f2_add(r, v); }
    static __device__ __forceinline__ void run_flush(double *p, const run_t &r) {
        atomicAdd(p, f2d_exact(r.hi) + f2d_exact(r.lo));
    }
    static __device__ __forceinline__ void item_flush(double *p, shared_t v) { atomicAdd(p, f2d_exact(v)); }
};
template <class T>
struct PairAcc<T, true> {
    typedef unsigned long long shared_t;
    typedef long long run_t;
    static __device__ __forceinline__ void shared_add(shared_t *p, T v) {
        atomicAdd(p, (unsigned long long)ap_to_fx(v));
    }
    static __device__ __forceinline__ void shared_put(shared_t *p, T v) { *p = (unsigned long long)ap_to_fx(v); }
    static __device__ __forceinline__ void run_zero(run_t &r) { r = 0; }
    static __device__ __forceinline__ void run_add(run_t &r, shared_t v) { r += (long long)v; }
    static __device__ __forceinline__ void run_flush(double *p, const run_t &r) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)r);
    }
    static __device__ __forceinline__ void item_flush(double *p, shared_t v) {
        atomicAdd(reinterpret_cast<unsigned long long *>(p), v);
    }
};
