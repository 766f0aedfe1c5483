// f1 - AMOEBA's two induced-dipole sets. The polarization interactions carry three scale
// factors (paper Sec. 2.3): the direct field that induces the d dipoles is scaled between
// atoms of one polarization group, the field that induces the p dipoles between bonded
// neighbours, and the mutual field not at all. So there are two right-hand sides and two
// solutions of the same system A = alpha^-1 - T:
//
//   E_d = E_c + sum_listed sigma_d F_lambda,   E_p = E_c + sum_listed sigma_p F_lambda
//   mu_d = A^-1 E_d,  mu_p = A^-1 E_p,  E_pol = -(f/2) sum_i mu_d,i . E_p,i
//
// E_c is the field with every listed (scaled) pair left out of real space (the exclusion
// masks of the pair kernels); F_lambda is a listed pair's Thole-damped Coulomb field
// (radial functions lambda_{2n+1} U_n), added back with each set's scale by a small kernel
// over the listed pairs - the paper's separate scaling-correction kernel.
//
// Both systems are solved together by two PCG recurrences in lockstep: one iteration
// applies T to both search directions with the two-set pair kernel (each pair tensor
// evaluated once) and two PME passes, and the loop stops when the larger convergence
// measure is <= tol.
//
// Forces (-dE_pol/dx with mu_d's response folded in through mu_p, A symmetric):
//   F = F_1(mu_s) - F_T(delta) + F_listed,
// with mu_s = (mu_d + mu_p)/2, delta = (mu_d - mu_p)/2, F_1(mu) the single-set force of
// -f mu . E_c - (f/2) mu . T mu, F_T(delta) the force of the mutual term -(f/2) delta . T delta
// alone (the single-set path with the permanent multipoles zeroed), and F_listed the
// gradient of -(f/2) sum_listed (sigma_d mu_p,I + sigma_p mu_d,I) . F_lambda including its
// multipole-orientation (frame) terms.
#include "common.cuh"
#include "vec_f32.cuh"

#include <type_traits>

#include <cmath>
#include <cstdlib>

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s);
void dp_release_impl(ap_ctx *ctx);

struct DpState {
    double rz[2], pq[2], gamma[2], beta[2], eps[2], eps0[2];
    double tol;
    int iter, max_iter, done, status, nonfinite, guard;
    unsigned int blocks_done, blocks_done2;
};

struct DpBuffers {
    int n_pairs = 0, cap_pairs = 0;
    int2 *pairs = nullptr;        // listed pairs, caller atom indices
    double2 *scales = nullptr;    // (sigma_d, sigma_p)
    double *E2 = nullptr;         // [2][3][n_pad] E_d, E_p (slot order)
    double *corr = nullptr;       // [2][3][n_pad] listed-pair field terms (FP64 or fixed point)
    double *mu2 = nullptr, *r2 = nullptr, *q2 = nullptr;   // [2][3][n_pad] (FP64 mode)
    float4 *mu2f = nullptr, *r2f = nullptr, *q2f = nullptr;  // [2][n_pad] (mixed and fixed modes)
    void *p2 = nullptr;           // T4 [2][n_pad] search directions
    double *acc2 = nullptr;       // [3][n_pad] real-space accumulator of the second set
    void *rec2 = nullptr;         // T [3][n_pad] reciprocal field of the second set
    double *part = nullptr;       // [4][blocks] partial sums
    DpState *st = nullptr, *st_host = nullptr;
    double *mus = nullptr;        // [2][3][n_pad] mu_d, mu_p in slot order (force terms)
    double *cbuf = nullptr;       // [3][n][3] caller order: mu_s, delta, mutual forces of delta
    void *mz = nullptr;           // T4 [4][n_pad]: posq, dipd, quad0, quad1 with the multipoles zeroed
    double *gsc = nullptr;        // [9][n_pad] scratch multipole derivatives of the mutual pass
    double *e_scr = nullptr;      // [2] energy scratch
    int *flag = nullptr;          // [1] validation flag
    PmeBufs pme2;                 // grids and plans of the second set's PME pass
    cudaStream_t s_rec2 = nullptr;  // its stream, concurrent with the first set's PME pass
    cudaEvent_t ev_join2 = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_tried = 0;
    int field_valid = 0;
};

namespace {

constexpr int NT = 256;

DpBuffers *dpb(ap_ctx *ctx) { return (DpBuffers *)ctx->dp; }

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// block-wide sums of K values; thread 0 returns them
template <int K>
__device__ __forceinline__ void block_sumk(double *v) {
    __shared__ double sm[NT / 32][K];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double s = warp_sum(v[k]);
        if (l == 0) sm[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int q = 0; q < NT / 32; ++q) t += sm[q][k];
            v[k] = t;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(counter, 1u);
        last = ticket == gridDim.x - 1;
        if (last) *counter = 0u;
    }
    __syncthreads();
    return last;
}

// fixed-order sums of K partial arrays of `nb` entries (one block of NT threads)
template <int K>
__device__ __forceinline__ void sum_parts(const double *part, int nb, double *out) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        v[k] = 0.0;
        for (int b = threadIdx.x; b < nb; b += NT) v[k] += __ldcg(part + k * nb + b);
    }
    block_sumk<K>(v);
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = v[k];
}

__device__ __forceinline__ void add_acc(double *arr, size_t k, double v, int fixed) {
    if (fixed)
        atomicAdd(reinterpret_cast<unsigned long long *>(arr) + k, (unsigned long long)ap_to_fx(v));
    else
        atomicAdd(arr + k, v);
}

// ---- listed pairs ----------------------------------------------------------------------
__global__ void k_pairs_check(const int *__restrict__ pairs, const double *__restrict__ scales, int m, int n,
                              int2 *__restrict__ out, double2 *__restrict__ sout, int *__restrict__ bad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int i = pairs[2 * k], j = pairs[2 * k + 1];
    const double sd = scales[2 * k], sp = scales[2 * k + 1];
    const bool ok = i >= 0 && i < n && j >= 0 && j < n && i != j && isfinite(sd) && isfinite(sp);
    if (!ok) atomicExch(bad, 1);
    out[k] = ok ? make_int2(i, j) : make_int2(0, 0);
    sout[k] = ok ? make_double2(sd, sp) : make_double2(1.0, 1.0);   // a no-op entry
}

// minimum-image vector x_a - x_b of two slots from the block origins and block-relative
// positions, in FP64
template <class T>
__device__ __forceinline__ void slot_vector(const typename V4<T>::type *posq, const float4 *bcenter, int a, int b,
                                            double3 L, double3 iL, double *R) {
    const typename V4<T>::type pa = posq[a], pb = posq[b];
    const float4 ca = bcenter[a >> 5], cb = bcenter[b >> 5];
    R[0] = ((double)ca.x - (double)cb.x) + ((double)pa.x - (double)pb.x);
    R[1] = ((double)ca.y - (double)cb.y) + ((double)pa.y - (double)pb.y);
    R[2] = ((double)ca.z - (double)cb.z) + ((double)pa.z - (double)pb.z);
    R[0] -= L.x * rint(R[0] * iL.x);
    R[1] -= L.y * rint(R[1] * iL.y);
    R[2] -= L.z * rint(R[2] * iL.z);
}

// Thole-damped Coulomb radial functions lambda_{2n+1} U_n, n = 1..4 (U_n = (2n-1)!!/r^{2n+1}),
// in FP64 for the few listed pairs
__device__ __forceinline__ void damped_coulomb(double r2, double u_thole, double *Rn) {
    const double rinv = rsqrt(r2), rinv2 = rinv * rinv;
    const double r = r2 * rinv;
    const double s = u_thole * r2 * r;
    const double e = exp(-s);
    const double U1 = rinv * rinv2, U2 = 3.0 * U1 * rinv2, U3 = 5.0 * U2 * rinv2, U4 = 7.0 * U3 * rinv2;
    Rn[0] = (1.0 - e) * U1;
    Rn[1] = (1.0 - (1.0 + s) * e) * U2;
    Rn[2] = (1.0 - (1.0 + s + 0.6 * s * s) * e) * U3;
    Rn[3] = (1.0 - (1.0 + s + (18.0 / 35.0) * s * s + (9.0 / 35.0) * s * s * s) * e) * U4;
}

template <class T>
struct Multipole {
    double q, d[3], Q[6];   // Q: xx xy xz yy yz zz
    __device__ __forceinline__ void load(const typename V4<T>::type *posq, const typename V4<T>::type *dipd,
                                         const typename V4<T>::type *quad0, const typename V4<T>::type *quad1,
                                         int s) {
        const typename V4<T>::type a = posq[s], b = dipd[s], c = quad0[s], e = quad1[s];
        q = a.w;
        d[0] = b.x; d[1] = b.y; d[2] = b.z;
        Q[0] = c.x; Q[1] = c.y; Q[2] = c.z; Q[3] = c.w; Q[4] = e.x; Q[5] = e.y;
    }
    __device__ __forceinline__ void QR(const double *R, double *o) const {
        o[0] = Q[0] * R[0] + Q[1] * R[1] + Q[2] * R[2];
        o[1] = Q[1] * R[0] + Q[3] * R[1] + Q[4] * R[2];
        o[2] = Q[2] * R[0] + Q[4] * R[1] + Q[5] * R[2];
    }
};

// field at R (target - source) of a multipole with radial functions Rn = (R1, R2, R3):
// E = (q R1 + (d.R) R2 + (R.Q.R) R3/3) R - R1 d - (2/3) R2 Q R
template <class T>
__device__ __forceinline__ void multipole_field(const Multipole<T> &M, const double *R, const double *Rn, double *E) {
    double qr[3];
    M.QR(R, qr);
    const double dR = M.d[0] * R[0] + M.d[1] * R[1] + M.d[2] * R[2];
    const double RQR = qr[0] * R[0] + qr[1] * R[1] + qr[2] * R[2];
    const double c = M.q * Rn[0] + dR * Rn[1] + RQR * Rn[2] * (1.0 / 3.0);
    for (int a = 0; a < 3; ++a) E[a] = c * R[a] - Rn[0] * M.d[a] - (2.0 / 3.0) * Rn[1] * qr[a];
}

// listed-pair terms of E_d and E_p: sigma_x F_lambda at both atoms of every listed pair
// inside the cutoff (one thread per pair)
template <class T>
__global__ void k_listed_field(const int2 *__restrict__ pairs, const double2 *__restrict__ scales, int m,
                               const int *__restrict__ iperm, const typename V4<T>::type *__restrict__ posq,
                               const typename V4<T>::type *__restrict__ dipd,
                               const typename V4<T>::type *__restrict__ quad0,
                               const typename V4<T>::type *__restrict__ quad1, const float4 *__restrict__ bcenter,
                               double3 L, double3 iL, double rc2, double thole_a, int n_pad, double *__restrict__ corr,
                               int fixed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int2 pr = pairs[k];
    const double2 sc = scales[k];
    if (sc.x == 1.0 && sc.y == 1.0) return;
    const int a = iperm[pr.x], b = iperm[pr.y];
    double R[3];
    slot_vector<T>(posq, bcenter, a, b, L, iL, R);
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    if (!(r2 < rc2)) return;
    double Rn[4];
    damped_coulomb(r2, thole_a * (double)dipd[a].w * (double)dipd[b].w, Rn);
    Multipole<T> Ma, Mb;
    Ma.load(posq, dipd, quad0, quad1, a);
    Mb.load(posq, dipd, quad0, quad1, b);
    double Ea[3], Eb[3], Rm[3] = {-R[0], -R[1], -R[2]};
    multipole_field<T>(Mb, R, Rn, Ea);    // at a from b
    multipole_field<T>(Ma, Rm, Rn, Eb);   // at b from a
    const size_t set = (size_t)3 * n_pad;
    for (int c = 0; c < 3; ++c) {
        if (sc.x != 0.0) {
            add_acc(corr, (size_t)c * n_pad + a, sc.x * Ea[c], fixed);
            add_acc(corr, (size_t)c * n_pad + b, sc.x * Eb[c], fixed);
        }
        if (sc.y != 0.0) {
            add_acc(corr, set + (size_t)c * n_pad + a, sc.y * Ea[c], fixed);
            add_acc(corr, set + (size_t)c * n_pad + b, sc.y * Eb[c], fixed);
        }
    }
}

// E_d, E_p = E_c + listed terms; clears the listed-term accumulator
__global__ void k_dp_fields(const double *__restrict__ E, double *__restrict__ corr, int n_pad,
                            double *__restrict__ E2, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    for (int k = 0; k < 2; ++k)
        for (int c = 0; c < 3; ++c) {
            const size_t i = (size_t)k * 3 * n_pad + (size_t)c * n_pad + s;
            E2[i] = E[(size_t)c * n_pad + s] + acc_value(corr, i, fixed);
            corr[i] = 0.0;
        }
}

// ---- lockstep PCG on the two systems -----------------------------------------------------
// the initial state from the totals r.z and z.z of both systems (thread 0 of the last block)
__device__ void dp_init_state(DpState *st, const double *tot, int n, double tol, int max_iter) {
    st->tol = tol;
    st->iter = 0;
    st->max_iter = max_iter;
    st->guard = 0;
    st->status = AP_OK;
    st->nonfinite = 0;
    for (int k = 0; k < 2; ++k) {
        st->rz[k] = tot[2 * k];
        st->eps[k] = st->eps0[k] = AP_DEBYE * sqrt(tot[2 * k + 1] / n);
        st->beta[k] = st->gamma[k] = st->pq[k] = 0.0;
        if (!isfinite(st->eps[k])) st->nonfinite = 1;
    }
    st->done = (fmax(st->eps[0], st->eps[1]) <= tol) || st->nonfinite;
    if (st->nonfinite) st->status = AP_ERR_NONFINITE;
}

// gamma_k from the totals p_k.q_k
__device__ void dp_set_gamma(DpState *st, const double *tot) {
    for (int k = 0; k < 2; ++k) {
        st->pq[k] = tot[k];
        // a recurrence that has converged exactly (r.z = 0) stays where it is
        st->gamma[k] = (st->rz[k] != 0.0) ? st->rz[k] / tot[k] : 0.0;
    }
}

// closes an iteration from the totals r.z and z.z: eps_k, the stop decision on the larger
// one, beta_k, and the WHILE condition (never beyond max_iter iterations)
__device__ void dp_close_iteration(DpState *st, const double *tot, int n, cudaGraphConditionalHandle h,
                                   int use_cond) {
    st->iter += 1;
    st->guard += 1;
    bool bad = false;
    for (int k = 0; k < 2; ++k) {
        st->eps[k] = AP_DEBYE * sqrt(tot[2 * k + 1] / n);
        bad = bad || !isfinite(st->eps[k]) || !isfinite(st->gamma[k]);
        st->beta[k] = (st->rz[k] != 0.0) ? tot[2 * k] / st->rz[k] : 0.0;
        st->rz[k] = tot[2 * k];
    }
    if (bad) st->nonfinite = 1;
    if (fmax(st->eps[0], st->eps[1]) <= st->tol || bad) {
        st->done = 1;
        st->status = bad ? AP_ERR_NONFINITE : AP_OK;
    } else if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = AP_NOT_CONVERGED;
    }
    if (use_cond) cudaGraphSetConditional(h, (!st->done && st->guard < st->max_iter) ? 1u : 0u);
}


template <class T>
__global__ void k_dp_guess(const double *__restrict__ gd, const double *__restrict__ gp,
                           const double *__restrict__ E2, const double *__restrict__ alpha,
                           const int *__restrict__ perm, int n, int n_pad, double *__restrict__ mu2,
                           typename V4<T>::type *__restrict__ p2, double self_coef, double *__restrict__ dg) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double al = alpha[s];
    dg[s] = al > 0.0 ? 1.0 / al - self_coef : 0.0;
    for (int k = 0; k < 2; ++k) {
        const double *g = k ? gp : gd;
        double m[3] = {0.0, 0.0, 0.0};
        if (s < n) {
            if (g) {
                const int i = perm[s];
                for (int c = 0; c < 3; ++c) m[c] = g[3 * i + c];
            } else {
                for (int c = 0; c < 3; ++c) m[c] = al * E2[(size_t)k * 3 * n_pad + (size_t)c * n_pad + s];
            }
        }
        for (int c = 0; c < 3; ++c) mu2[(size_t)k * 3 * n_pad + (size_t)c * n_pad + s] = m[c];
        typename V4<T>::type v;
        v.x = (T)m[0]; v.y = (T)m[1]; v.z = (T)m[2]; v.w = (T)0;
        p2[(size_t)k * n_pad + s] = v;
    }
}

struct DpVecs {
    double *acc[2];
    const void *rec[2];
};

// r_k = E_k - A mu_k; clears the accumulators and the directions; partial r.z and z.z of
// both systems. The last block sets the initial state.
template <class T>
__global__ void k_dp_init_residual(const double *__restrict__ E2, const double *__restrict__ alpha,
                                   const double *__restrict__ mu2, DpVecs v, const double *__restrict__ dg, int n_pad,
                                   int n, double *__restrict__ r2, typename V4<T>::type *__restrict__ p2,
                                   double *__restrict__ part, DpState *st, double tol, int max_iter, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    if (s < n_pad) {
        const double a = alpha[s], d = dg[s];
        for (int k = 0; k < 2; ++k) {
            const T *rec = (const T *)v.rec[k];
            for (int c = 0; c < 3; ++c) {
                const size_t i = (size_t)k * 3 * n_pad + (size_t)c * n_pad + s, j = (size_t)c * n_pad + s;
                const double Amu = a > 0.0 ? mu2[i] * d - acc_value(v.acc[k], j, fixed) - (double)rec[j] : 0.0;
                const double rr = a > 0.0 ? E2[i] - Amu : 0.0;
                r2[i] = rr;
                v.acc[k][j] = 0.0;
                red[2 * k] += rr * a * rr;
                red[2 * k + 1] += a * rr * a * rr;
            }
            typename V4<T>::type z;
            z.x = z.y = z.z = z.w = (T)0;
            p2[(size_t)k * n_pad + s] = z;
        }
    }
    block_sumk<4>(red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[k * gridDim.x + blockIdx.x] = red[k];
    if (!last_block(&st->blocks_done)) return;
    double tot[4];
    sum_parts<4>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_init_state(st, tot, n, tol, max_iter);
}

__global__ void k_dp_set_cond(cudaGraphConditionalHandle h, const DpState *st) {
    cudaGraphSetConditional(h, (st->done || st->max_iter < 1) ? 0u : 1u);
}

// p_k = alpha r_k + beta_k p_k
template <class T>
__global__ void k_dp_direction(const double *__restrict__ r2, const double *__restrict__ alpha, int n_pad,
                               typename V4<T>::type *__restrict__ p2, const DpState *__restrict__ st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double a = alpha[s];
    for (int k = 0; k < 2; ++k) {
        const double b = st->beta[k];
        const double *r = r2 + (size_t)k * 3 * n_pad;
        typename V4<T>::type v = p2[(size_t)k * n_pad + s];
        v.x = (T)(a * r[s] + b * (double)v.x);
        v.y = (T)(a * r[n_pad + s] + b * (double)v.y);
        v.z = (T)(a * r[2 * n_pad + s] + b * (double)v.z);
        p2[(size_t)k * n_pad + s] = v;
    }
}

// q_k = A p_k; partial p_k.q_k; clears the accumulators. The last block sets gamma_k.
template <class T>
__global__ void k_dp_apply(const typename V4<T>::type *__restrict__ p2, const double *__restrict__ dg, DpVecs v,
                           int n_pad, double *__restrict__ q2, double *__restrict__ part, DpState *st, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double red[2] = {0.0, 0.0};
    if (s < n_pad) {
        const double d = dg[s];
        for (int k = 0; k < 2; ++k) {
            const T *rec = (const T *)v.rec[k];
            const typename V4<T>::type pv = p2[(size_t)k * n_pad + s];
            const double pp[3] = {(double)pv.x, (double)pv.y, (double)pv.z};
            for (int c = 0; c < 3; ++c) {
                const size_t j = (size_t)c * n_pad + s;
                const double qq = pp[c] * d - acc_value(v.acc[k], j, fixed) - (double)rec[j];
                q2[(size_t)k * 3 * n_pad + j] = qq;
                v.acc[k][j] = 0.0;
                red[k] += pp[c] * qq;
            }
        }
    }
    block_sumk<2>(red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = red[0];
        part[gridDim.x + blockIdx.x] = red[1];
    }
    if (!last_block(&st->blocks_done)) return;
    double tot[2];
    sum_parts<2>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_set_gamma(st, tot);
}

// mu_k += gamma_k p_k; r_k -= gamma_k q_k; partial r.z and z.z; the last block closes the
// iteration: eps_k, the stop decision on the larger one, beta_k, and the WHILE condition
// (never beyond max_iter iterations)
template <class T>
__global__ void k_dp_update(const typename V4<T>::type *__restrict__ p2, const double *__restrict__ q2,
                            const double *__restrict__ alpha, int n_pad, double *__restrict__ mu2,
                            double *__restrict__ r2, DpState *st, double *__restrict__ part, int n,
                            cudaGraphConditionalHandle h, int use_cond) {
    const double g[2] = {st->gamma[0], st->gamma[1]};
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    if (s < n_pad) {
        const double a = alpha[s];
        for (int k = 0; k < 2; ++k) {
            const typename V4<T>::type pv = p2[(size_t)k * n_pad + s];
            const double pp[3] = {(double)pv.x, (double)pv.y, (double)pv.z};
            for (int c = 0; c < 3; ++c) {
                const size_t i = (size_t)k * 3 * n_pad + (size_t)c * n_pad + s;
                mu2[i] += g[k] * pp[c];
                const double rr = r2[i] - g[k] * q2[i];
                r2[i] = rr;
                const double z = a * rr;
                red[2 * k] += rr * z;
                red[2 * k + 1] += z * z;
            }
        }
    }
    block_sumk<4>(red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[k * gridDim.x + blockIdx.x] = red[k];
    if (!last_block(&st->blocks_done2)) return;
    double tot[4];
    sum_parts<4>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_close_iteration(st, tot, n, h, use_cond);
}

// ---- the same lockstep iteration with FP32 vectors (mixed and fixed-point modes): mu, r, q
// and p of both systems as float4 per slot, the diagonal and alpha as a float2; dot products
// and norms as compensated FP32 sums finished in FP64 (vec_f32.cuh), as the single-set PCG

__global__ void k_dp_guess_f(const double *__restrict__ gd, const double *__restrict__ gp,
                             const double *__restrict__ E2, const double *__restrict__ alpha,
                             const int *__restrict__ perm, int n, int n_pad, float4 *__restrict__ mu2,
                             float4 *__restrict__ p2, double self_coef, float2 *__restrict__ dga) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double al = alpha[s];
    dga[s] = make_float2(al > 0.0 ? (float)(1.0 / al - self_coef) : 0.f, (float)al);
    for (int k = 0; k < 2; ++k) {
        const double *g = k ? gp : gd;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s < n) {
            if (g) {
                const int i = perm[s];
                m = make_float4((float)g[3 * i], (float)g[3 * i + 1], (float)g[3 * i + 2], 0.f);
            } else {
                const double *e = E2 + (size_t)k * 3 * n_pad;
                m = make_float4((float)(al * e[s]), (float)(al * e[n_pad + s]), (float)(al * e[2 * (size_t)n_pad + s]),
                                0.f);
            }
        }
        mu2[(size_t)k * n_pad + s] = m;
        p2[(size_t)k * n_pad + s] = m;
    }
}

// the compensated sums a[0..3] of the block, partials part[k][block]
__device__ __forceinline__ void dp_block_parts4(const F2 *a, double *part) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    block_sum2_f2<NT>(a[0], a[1], t[0], t[1]);
    __syncthreads();
    block_sum2_f2<NT>(a[2], a[3], t[2], t[3]);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[k * gridDim.x + blockIdx.x] = t[k];
}

// r_k = E_k - A mu_k (formed in FP64 once per solve, stored in FP32); clears the accumulators
// and the directions; partial r.z and z.z of both systems. The last block sets the state.
__global__ void k_dp_init_residual_f(const double *__restrict__ E2, const float2 *__restrict__ dga,
                                     const float4 *__restrict__ mu2, DpVecs v, int n_pad, int n,
                                     float4 *__restrict__ r2, float4 *__restrict__ p2, double *__restrict__ part,
                                     DpState *st, double tol, int max_iter, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 red[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (s < n_pad) {
        const float2 d = dga[s];
        for (int k = 0; k < 2; ++k) {
            const float *rec = (const float *)v.rec[k];
            const float4 m = mu2[(size_t)k * n_pad + s];
            const float mv[3] = {m.x, m.y, m.z};
            float rv[3];
            for (int c = 0; c < 3; ++c) {
                const size_t i = (size_t)k * 3 * n_pad + (size_t)c * n_pad + s, j = (size_t)c * n_pad + s;
                const double Amu = d.y > 0.f ? (double)mv[c] * d.x - acc_value(v.acc[k], j, fixed) - (double)rec[j] : 0.0;
                rv[c] = d.y > 0.f ? (float)(E2[i] - Amu) : 0.f;
                v.acc[k][j] = 0.0;
                const float z = d.y * rv[c];
                f2_add_prod(red[2 * k], rv[c], z);
                f2_add_prod(red[2 * k + 1], z, z);
            }
            r2[(size_t)k * n_pad + s] = make_float4(rv[0], rv[1], rv[2], 0.f);
            p2[(size_t)k * n_pad + s] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    dp_block_parts4(red, part);
    if (!last_block(&st->blocks_done)) return;
    double tot[4];
    sum_parts<4>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_init_state(st, tot, n, tol, max_iter);
}

// p_k = alpha r_k + beta_k p_k
__global__ void k_dp_direction_f(const float4 *__restrict__ r2, const float2 *__restrict__ dga, int n_pad,
                                 float4 *__restrict__ p2, const DpState *__restrict__ st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const float a = dga[s].y;
    for (int k = 0; k < 2; ++k) {
        const float b = (float)st->beta[k];
        const float4 r = r2[(size_t)k * n_pad + s];
        float4 p = p2[(size_t)k * n_pad + s];
        p.x = fmaf(a, r.x, b * p.x);
        p.y = fmaf(a, r.y, b * p.y);
        p.z = fmaf(a, r.z, b * p.z);
        p2[(size_t)k * n_pad + s] = p;
    }
}

// q_k = A p_k; partial p_k.q_k; clears the accumulators. The last block sets gamma_k.
__global__ void k_dp_apply_f(const float4 *__restrict__ p2, const float2 *__restrict__ dga, DpVecs v, int n_pad,
                             float4 *__restrict__ q2, double *__restrict__ part, DpState *st, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 red[2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (s < n_pad) {
        const float d = dga[s].x;
        for (int k = 0; k < 2; ++k) {
            const float *rec = (const float *)v.rec[k];
            const float4 pv = p2[(size_t)k * n_pad + s];
            const float pp[3] = {pv.x, pv.y, pv.z};
            float qq[3];
            for (int c = 0; c < 3; ++c) {
                const size_t j = (size_t)c * n_pad + s;
                qq[c] = fmaf(pp[c], d, -acc_f32(v.acc[k], j, fixed)) - rec[j];
                v.acc[k][j] = 0.0;
                f2_add_prod(red[k], pp[c], qq[c]);
            }
            q2[(size_t)k * n_pad + s] = make_float4(qq[0], qq[1], qq[2], 0.f);
        }
    }
    double t0 = 0.0, t1 = 0.0;
    block_sum2_f2<NT>(red[0], red[1], t0, t1);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t0;
        part[gridDim.x + blockIdx.x] = t1;
    }
    if (!last_block(&st->blocks_done)) return;
    double tot[2];
    sum_parts<2>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_set_gamma(st, tot);
}

// mu_k += gamma_k p_k; r_k -= gamma_k q_k; partial r.z and z.z; the last block closes the
// iteration
__global__ void k_dp_update_f(const float4 *__restrict__ p2, const float4 *__restrict__ q2,
                              const float2 *__restrict__ dga, int n_pad, float4 *__restrict__ mu2,
                              float4 *__restrict__ r2, DpState *st, double *__restrict__ part, int n,
                              cudaGraphConditionalHandle h, int use_cond) {
    const float g[2] = {(float)st->gamma[0], (float)st->gamma[1]};
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 red[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (s < n_pad) {
        const float a = dga[s].y;
        for (int k = 0; k < 2; ++k) {
            const size_t i = (size_t)k * n_pad + s;
            const float4 pv = p2[i], qv = q2[i];
            float4 m = mu2[i], rv = r2[i];
            m.x = fmaf(g[k], pv.x, m.x);
            m.y = fmaf(g[k], pv.y, m.y);
            m.z = fmaf(g[k], pv.z, m.z);
            rv.x = fmaf(-g[k], qv.x, rv.x);
            rv.y = fmaf(-g[k], qv.y, rv.y);
            rv.z = fmaf(-g[k], qv.z, rv.z);
            mu2[i] = m;
            r2[i] = rv;
            const float rr[3] = {rv.x, rv.y, rv.z};
            for (int c = 0; c < 3; ++c) {
                const float z = a * rr[c];
                f2_add_prod(red[2 * k], rr[c], z);
                f2_add_prod(red[2 * k + 1], z, z);
            }
        }
    }
    dp_block_parts4(red, part);
    if (!last_block(&st->blocks_done2)) return;
    double tot[4];
    sum_parts<4>(part, gridDim.x, tot);
    if (threadIdx.x == 0) dp_close_iteration(st, tot, n, h, use_cond);
}

// FP32 dipoles of one system to the caller's order in FP64
__global__ void k_dp_unsort_f4(const float4 *__restrict__ src, const int *__restrict__ iperm, int n,
                               double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = src[iperm[i]];
    out[3 * i] = v.x;
    out[3 * i + 1] = v.y;
    out[3 * i + 2] = v.z;
}

double self_coef_of(const ap_ctx *ctx) { return 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI); }

DpVecs vecs_of(ap_ctx *ctx) {
    DpBuffers *B = dpb(ctx);
    DpVecs v;
    v.acc[0] = ctx->acc;
    v.acc[1] = B->acc2;
    v.rec[0] = ctx->rec;
    v.rec[1] = B->rec2;
    return v;
}

// T applied to both directions: real space (two-set kernel) on `main`, the two PME passes
// on `aux` and on the second set's own stream with its own grids, all joined into `main`
template <class T>
int matvec2(ap_ctx *ctx, cudaStream_t main, cudaStream_t aux) {
    typedef typename V4<T>::type T4;
    DpBuffers *B = dpb(ctx);
    const T4 *p0 = (const T4 *)B->p2, *p1 = p0 + ctx->n_pad;
    AP_CUDA(cudaEventRecord(ctx->ev_fork, main));
    AP_CUDA(cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
    AP_CUDA(cudaStreamWaitEvent(B->s_rec2, ctx->ev_fork, 0));
    int rc = pme_dipole_field_into(ctx, p0, ctx->rec, nullptr, aux);
    if (rc) return rc;
    rc = pme_dipole_field_into(ctx, p1, B->rec2, &B->pme2, B->s_rec2);
    if (rc) return rc;
    rc = real_matvec2_launch(ctx, p0, p1, ctx->acc, B->acc2, main);
    if (rc) return rc;
    AP_CUDA(cudaEventRecord(ctx->ev_join, aux));
    AP_CUDA(cudaEventRecord(B->ev_join2, B->s_rec2));
    AP_CUDA(cudaStreamWaitEvent(main, ctx->ev_join, 0));
    AP_CUDA(cudaStreamWaitEvent(main, B->ev_join2, 0));
    return AP_OK;
}

template <class T>
int enqueue_iteration(ap_ctx *ctx, cudaGraphConditionalHandle h, int use_cond, cudaStream_t main, cudaStream_t aux) {
    typedef typename V4<T>::type T4;
    DpBuffers *B = dpb(ctx);
    const int nb = ap_grid_for(ctx->n_pad, NT);
    if constexpr (std::is_same<T, float>::value) {
        k_dp_direction_f<<<nb, NT, 0, main>>>(B->r2f, ctx->dga_f, ctx->n_pad, (float4 *)B->p2, B->st);
        AP_CUDA(cudaGetLastError());
        int rc = matvec2<T>(ctx, main, aux);
        if (rc) return rc;
        k_dp_apply_f<<<nb, NT, 0, main>>>((const float4 *)B->p2, ctx->dga_f, vecs_of(ctx), ctx->n_pad, B->q2f,
                                          B->part, B->st, ctx->fixed);
        k_dp_update_f<<<nb, NT, 0, main>>>((const float4 *)B->p2, B->q2f, ctx->dga_f, ctx->n_pad, B->mu2f, B->r2f,
                                           B->st, B->part, ctx->n, h, use_cond);
    } else {
        k_dp_direction<T><<<nb, NT, 0, main>>>(B->r2, ctx->alpha, ctx->n_pad, (T4 *)B->p2, B->st);
        AP_CUDA(cudaGetLastError());
        int rc = matvec2<T>(ctx, main, aux);
        if (rc) return rc;
        k_dp_apply<T><<<nb, NT, 0, main>>>((const T4 *)B->p2, ctx->dg, vecs_of(ctx), ctx->n_pad, B->q2, B->part,
                                            B->st, ctx->fixed);
        k_dp_update<T><<<nb, NT, 0, main>>>((const T4 *)B->p2, B->q2, ctx->alpha, ctx->n_pad, B->mu2, B->r2, B->st,
                                             B->part, ctx->n, h, use_cond);
    }
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int build_graph(ap_ctx *ctx) {
    DpBuffers *B = dpb(ctx);
    B->exec_tried = 1;
    const char *env = getenv("AP_SOLVE_GRAPH");
    if (env && env[0] == '0') return AP_OK;
    cudaGraph_t g = nullptr;
    AP_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return AP_OK;
    }
    cudaKernelNodeParams kp = {};
    const DpState *stp = B->st;
    void *args[2] = {(void *)&h, (void *)&stp};
    kp.func = (void *)k_dp_set_cond;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    cudaGraphNode_t n_set, n_while;
    AP_CUDA(cudaGraphAddKernelNode(&n_set, g, nullptr, 0, &kp));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    AP_CUDA(cudaGraphAddNode(&n_while, g, &n_set, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = nullptr;
    AP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    AP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration<T>(ctx, h, 1, cs, ctx->s1);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (rc || ec != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        ctx->err.clear();
        return AP_OK;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return AP_OK;
    }
    cudaGraphDestroy(g);
    B->exec = ex;
    return AP_OK;
}

template <class T>
int solve_t(ap_ctx *ctx, const double *gd, const double *gp, double tol, int max_iter, double *d_mu_d,
            double *d_mu_p, ap_solve_info *info) {
    typedef typename V4<T>::type T4;
    DpBuffers *B = dpb(ctx);
    cudaStream_t s = ctx->s0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    AP_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return ap_fail(ctx, AP_ERR_ARG, "induced_dipoles_pcg_dp cannot be captured into a graph");
    const int nb = ap_grid_for(ctx->n_pad, NT);
    AP_CUDA(cudaMemsetAsync(B->st, 0, sizeof(DpState), s));
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, s));
    AP_CUDA(cudaMemsetAsync(B->acc2, 0, sizeof(double) * 3 * ctx->n_pad, s));
    constexpr bool F32 = std::is_same<T, float>::value;   // FP32 vectors (mixed and fixed modes)
    if (F32)
        k_dp_guess_f<<<nb, NT, 0, s>>>(gd, gp, B->E2, ctx->alpha, ctx->perm, ctx->n, ctx->n_pad, B->mu2f,
                                       (float4 *)B->p2, self_coef_of(ctx), ctx->dga_f);
    else
        k_dp_guess<T><<<nb, NT, 0, s>>>(gd, gp, B->E2, ctx->alpha, ctx->perm, ctx->n, ctx->n_pad, B->mu2, (T4 *)B->p2,
                                         self_coef_of(ctx), ctx->dg);
    AP_CUDA(cudaGetLastError());
    int rc = matvec2<T>(ctx, s, ctx->s1);
    if (rc) return rc;
    if (F32)
        k_dp_init_residual_f<<<nb, NT, 0, s>>>(B->E2, ctx->dga_f, B->mu2f, vecs_of(ctx), ctx->n_pad, ctx->n, B->r2f,
                                               (float4 *)B->p2, B->part, B->st, tol, max_iter, ctx->fixed);
    else
        k_dp_init_residual<T><<<nb, NT, 0, s>>>(B->E2, ctx->alpha, B->mu2, vecs_of(ctx), ctx->dg, ctx->n_pad, ctx->n,
                                                 B->r2, (T4 *)B->p2, B->part, B->st, tol, max_iter, ctx->fixed);
    AP_CUDA(cudaGetLastError());
    if (!B->exec_tried) {
        rc = build_graph<T>(ctx);
        if (rc) return rc;
    }
    if (B->exec) {
        AP_CUDA(cudaGraphLaunch(B->exec, s));
    } else {
        for (int it = 0; it < max_iter; ++it) {
            AP_CUDA(cudaMemcpyAsync(B->st_host, B->st, sizeof(DpState), cudaMemcpyDeviceToHost, s));
            AP_CUDA(cudaStreamSynchronize(s));
            if (B->st_host->done) break;
            rc = enqueue_iteration<T>(ctx, 0, 0, ctx->s0, ctx->s1);
            if (rc) return rc;
        }
    }
    if (F32) {
        k_dp_unsort_f4<<<ap_grid_for(ctx->n, 256), 256, 0, s>>>(B->mu2f, ctx->iperm, ctx->n, d_mu_d);
        k_dp_unsort_f4<<<ap_grid_for(ctx->n, 256), 256, 0, s>>>(B->mu2f + ctx->n_pad, ctx->iperm, ctx->n, d_mu_p);
    } else {
        unsort3(ctx, B->mu2, d_mu_d, s);
        unsort3(ctx, B->mu2 + (size_t)3 * ctx->n_pad, d_mu_p, s);
    }
    AP_CUDA(cudaGetLastError());
    if (info) {
        AP_CUDA(cudaMemcpyAsync(B->st_host, B->st, sizeof(DpState), cudaMemcpyDeviceToHost, s));
        AP_CUDA(cudaStreamSynchronize(s));
        const DpState *h = B->st_host;
        info->iterations = h->iter;
        info->eps_debye = fmax(h->eps[0], h->eps[1]);
        info->eps_initial = fmax(h->eps0[0], h->eps0[1]);
        info->status = h->status;
        if (h->nonfinite) return ap_fail(ctx, AP_ERR_NONFINITE, "non-finite value in the PCG reductions");
        return h->status;
    }
    return AP_OK;
}

// ---- energy and forces -------------------------------------------------------------------
__global__ void k_dp_split(const double *__restrict__ md, const double *__restrict__ mp, int n3,
                           double *__restrict__ cbuf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const double a = md[k], b = mp[k];
    cbuf[k] = 0.5 * (a + b);
    cbuf[n3 + k] = 0.5 * (a - b);
}

// copies of the configuration arrays with the permanent multipoles zeroed: positions, Thole
// factors and polarizabilities kept
template <class T>
__global__ void k_zero_multipoles(const typename V4<T>::type *__restrict__ posq,
                                  const typename V4<T>::type *__restrict__ dipd,
                                  const typename V4<T>::type *__restrict__ quad1, int n_pad,
                                  typename V4<T>::type *__restrict__ mz) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    typename V4<T>::type a = posq[s], b = dipd[s], d = quad1[s], z;
    a.w = T(0);
    b.x = b.y = b.z = T(0);
    z.x = z.y = z.z = z.w = T(0);
    d.x = d.y = d.w = T(0);
    mz[s] = a;
    mz[(size_t)n_pad + s] = b;
    mz[(size_t)2 * n_pad + s] = z;
    mz[(size_t)3 * n_pad + s] = d;
}

// both sets into slot order (the listed-pair force kernel reads them by slot)
__global__ void k_dp_slots(const double *__restrict__ md, const double *__restrict__ mp,
                           const int *__restrict__ perm, int n, int n_pad, double *__restrict__ mus) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const int i = s < n ? perm[s] : -1;
    for (int c = 0; c < 3; ++c) {
        mus[(size_t)c * n_pad + s] = i >= 0 ? md[3 * i + c] : 0.0;
        mus[(size_t)3 * n_pad + (size_t)c * n_pad + s] = i >= 0 ? mp[3 * i + c] : 0.0;
    }
}

// E_pol = -(f/2) sum mu_d . E_p over slots; deterministic (fixed-order block partials)
__global__ void k_dp_energy(const double *__restrict__ mus, const double *__restrict__ E2, int n_pad, double scale,
                            double *__restrict__ part, unsigned int *counter, double *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (s < n_pad)
        for (int c = 0; c < 3; ++c)
            v[0] += mus[(size_t)c * n_pad + s] * E2[(size_t)3 * n_pad + (size_t)c * n_pad + s];
    block_sumk<1>(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
    if (!last_block(counter)) return;
    double tot[1];
    sum_parts<1>(part, gridDim.x, tot);
    if (threadIdx.x == 0) *out = scale * tot[0];
}

// F = F_1(mu_s) - F_T(delta), in caller order
__global__ void k_dp_force_combine(const double *__restrict__ ft, int n3, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    out[k] -= ft[k];
}

// adds v[0..8] of every thread of a block of NT threads to acc[0..8] (FP64 atomics, or
// integer atomics for values already in fixed point)
template <int NT, class V>
__device__ __forceinline__ void block_add9_dp(V *v, double *acc) {
    __shared__ V sm[NT / 32][9];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int e = 0; e < 9; ++e) {
        V x = v[e];
        for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (l == 0) sm[w][e] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        V t = 0;
        for (int e = 0; e < NT / 32; ++e) t += sm[e][threadIdx.x];
        if constexpr (std::is_integral<V>::value)
            atomicAdd(reinterpret_cast<unsigned long long *>(acc) + threadIdx.x, (unsigned long long)t);
        else
            atomicAdd(acc + threadIdx.x, t);
    }
}

// one listed pair k of k_listed_forces; v (optional) receives its virial
template <class T>
__device__ __forceinline__ void listed_pair_forces(
    const int2 *__restrict__ pairs, const double2 *__restrict__ scales, int m, const int *__restrict__ iperm,
    const typename V4<T>::type *__restrict__ posq, const typename V4<T>::type *__restrict__ dipd,
    const typename V4<T>::type *__restrict__ quad0, const typename V4<T>::type *__restrict__ quad1,
    const float4 *__restrict__ bcenter, double3 L, double3 iL, double rc2, double thole_a,
    const double *__restrict__ mus, int n_pad, double f, double *__restrict__ frc, double *__restrict__ gdip,
    double *__restrict__ gquad, int fixed, int k, double *v) {
    if (k >= m) return;
    const int2 pr = pairs[k];
    const double2 sc = scales[k];
    if (sc.x == 1.0 && sc.y == 1.0) return;
    const int a = iperm[pr.x], b = iperm[pr.y];
    double R0[3];
    slot_vector<T>(posq, bcenter, a, b, L, iL, R0);
    const double r2 = R0[0] * R0[0] + R0[1] * R0[1] + R0[2] * R0[2];
    if (!(r2 < rc2)) return;
    double Rn[4];
    damped_coulomb(r2, thole_a * (double)dipd[a].w * (double)dipd[b].w, Rn);
    const double h = 0.5 * f;
    for (int dir = 0; dir < 2; ++dir) {
        const int I = dir ? b : a, J = dir ? a : b;
        const double sg = dir ? -1.0 : 1.0;
        const double R[3] = {sg * R0[0], sg * R0[1], sg * R0[2]};
        Multipole<T> M;
        M.load(posq, dipd, quad0, quad1, J);
        double w[3];
        for (int c = 0; c < 3; ++c)
            w[c] = sc.x * mus[(size_t)3 * n_pad + (size_t)c * n_pad + I] + sc.y * mus[(size_t)c * n_pad + I];
        double qr[3], qw[3];
        M.QR(R, qr);
        M.QR(w, qw);
        const double dR = M.d[0] * R[0] + M.d[1] * R[1] + M.d[2] * R[2];
        const double RQR = qr[0] * R[0] + qr[1] * R[1] + qr[2] * R[2];
        const double wR = w[0] * R[0] + w[1] * R[1] + w[2] * R[2];
        const double dw = M.d[0] * w[0] + M.d[1] * w[1] + M.d[2] * w[2];
        const double QRw = qr[0] * w[0] + qr[1] * w[1] + qr[2] * w[2];
        // sum_b dE_b/dR_a w_b for the field of multipole J
        double g[3];
        for (int c = 0; c < 3; ++c)
            g[c] = M.q * Rn[0] * w[c] - M.q * Rn[1] * R[c] * wR + Rn[1] * (R[c] * dw + M.d[c] * wR)
                 + dR * Rn[1] * w[c] - dR * Rn[2] * R[c] * wR - (2.0 / 3.0) * Rn[1] * qw[c]
                 + (2.0 / 3.0) * Rn[2] * (R[c] * QRw + qr[c] * wR) + (RQR / 3.0) * Rn[2] * w[c]
                 - (RQR / 3.0) * Rn[3] * R[c] * wR;
        // dU/dR = -h g: force +h g on I, -h g on J
        if (v)
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) v[3 * a + c] += -h * g[a] * R[c];
        for (int c = 0; c < 3; ++c) {
            add_acc(frc, (size_t)c * n_pad + I, h * g[c], fixed);
            add_acc(frc, (size_t)c * n_pad + J, -h * g[c], fixed);
            add_acc(gdip, (size_t)c * n_pad + J, -h * (-Rn[0] * w[c] + Rn[1] * wR * R[c]), fixed);
        }
        const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
        for (int e = 0; e < 6; ++e) {
            const int x = ia[e], y = ib[e];
            const double sym = w[x] * R[y] + R[x] * w[y];
            add_acc(gquad, (size_t)e * n_pad + J, -h * (-(Rn[1] / 3.0) * sym + (Rn[2] / 3.0) * wR * R[x] * R[y]), fixed);
        }
    }
}

// gradient of -(f/2) sum over listed ordered pairs (I, J) of w . F_lambda(R; M_J) with
// w = sigma_d mu_p,I + sigma_p mu_d,I: force on I and J, dU/d(global dipole) and
// dU/d(global quadrupole) of J (one thread per unordered pair, both orders); with vir
// non-NULL (blocks of 128 threads) also the pairs' virial, sum of (dU/dR) R^T
template <class T>
__global__ void k_listed_forces(const int2 *__restrict__ pairs, const double2 *__restrict__ scales, int m,
                                const int *__restrict__ iperm, const typename V4<T>::type *__restrict__ posq,
                                const typename V4<T>::type *__restrict__ dipd,
                                const typename V4<T>::type *__restrict__ quad0,
                                const typename V4<T>::type *__restrict__ quad1, const float4 *__restrict__ bcenter,
                                double3 L, double3 iL, double rc2, double thole_a, const double *__restrict__ mus,
                                int n_pad, double f, double *__restrict__ frc, double *__restrict__ gdip,
                                double *__restrict__ gquad, int fixed, double *__restrict__ vir) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    listed_pair_forces<T>(pairs, scales, m, iperm, posq, dipd, quad0, quad1, bcenter, L, iL, rc2, thole_a, mus, n_pad,
                          f, frc, gdip, gquad, fixed, k, vir ? v : nullptr);
    if (vir) {   // uniform over the launch
        if (fixed) {
            long long vf[9];
            for (int e = 0; e < 9; ++e) vf[e] = ap_to_fx(v[e]);
            block_add9_dp<128>(vf, vir);
        } else {
            block_add9_dp<128>(v, vir);
        }
    }
}


template <class T>
int listed_forces_t(ap_ctx *ctx, cudaStream_t s) {
    typedef typename V4<T>::type T4;
    DpBuffers *B = dpb(ctx);
    if (B->n_pairs == 0) return AP_OK;
    const ap_params &P = ctx->prm;
    k_listed_forces<T><<<ap_grid_for(B->n_pairs, 128), 128, 0, s>>>(
        B->pairs, B->scales, B->n_pairs, ctx->iperm, (const T4 *)ctx->posq, (const T4 *)ctx->dipd,
        (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, ctx->bcenter, make_double3(P.box[0], P.box[1], P.box[2]),
        make_double3(1.0 / P.box[0], 1.0 / P.box[1], 1.0 / P.box[2]), P.cutoff * P.cutoff, P.thole_a, B->mus,
        ctx->n_pad, AP_COULOMB, ctx->frc, ctx->gdip, ctx->gquad, ctx->fixed, ctx->vir_active);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int listed_forces(ap_ctx *ctx, cudaStream_t s) {
    return ctx->prec == AP_FP64 ? listed_forces_t<double>(ctx, s) : listed_forces_t<float>(ctx, s);
}

template <class T>
int fields_t(ap_ctx *ctx, double *d_field_d, double *d_field_p) {
    typedef typename V4<T>::type T4;
    DpBuffers *B = dpb(ctx);
    cudaStream_t s = ctx->s0;
    const ap_params &P = ctx->prm;
    if (B->n_pairs > 0) {
        k_listed_field<T><<<ap_grid_for(B->n_pairs, 128), 128, 0, s>>>(
            B->pairs, B->scales, B->n_pairs, ctx->iperm, (const T4 *)ctx->posq, (const T4 *)ctx->dipd,
            (const T4 *)ctx->quad0, (const T4 *)ctx->quad1, ctx->bcenter, make_double3(P.box[0], P.box[1], P.box[2]),
            make_double3(1.0 / P.box[0], 1.0 / P.box[1], 1.0 / P.box[2]), P.cutoff * P.cutoff, P.thole_a,
            ctx->n_pad, B->corr, ctx->fixed);
    }
    k_dp_fields<<<ap_grid_for(ctx->n_pad, 256), 256, 0, s>>>(ctx->E, B->corr, ctx->n_pad, B->E2, ctx->fixed);
    AP_CUDA(cudaGetLastError());
    if (d_field_d) unsort3(ctx, B->E2, d_field_d, s);
    if (d_field_p) unsort3(ctx, B->E2 + (size_t)3 * ctx->n_pad, d_field_p, s);
    AP_CUDA(cudaGetLastError());
    B->field_valid = 1;
    return AP_OK;
}

template <class P>
int dmalloc(ap_ctx *ctx, P **p, size_t bytes) {
    AP_CUDA(cudaMalloc((void **)p, bytes));
    AP_CUDA(cudaMemset(*p, 0, bytes));
    return AP_OK;
}

int reserve_all(ap_ctx *ctx);

// all two-set buffers, or none (a failed allocation releases what was taken)
int reserve(ap_ctx *ctx) {
    if (ctx->dp) return AP_OK;
    const int r = reserve_all(ctx);
    if (r) dp_release_impl(ctx);
    return r;
}

int reserve_all(ap_ctx *ctx) {
    DpBuffers *B = new DpBuffers();
    ctx->dp = B;
    const size_t np = ctx->n_pad, n = ctx->n;
    const size_t tsz = ctx->prec == AP_FP64 ? sizeof(double) : sizeof(float);
    const int nb = ap_grid_for(ctx->n_pad, NT);
    int r;
    if ((r = dmalloc(ctx, &B->E2, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->corr, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->mu2, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->r2, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->q2, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->mu2f, sizeof(float4) * 2 * np))) return r;
    if ((r = dmalloc(ctx, &B->r2f, sizeof(float4) * 2 * np))) return r;
    if ((r = dmalloc(ctx, &B->q2f, sizeof(float4) * 2 * np))) return r;
    if ((r = dmalloc(ctx, (char **)&B->p2, 4 * tsz * 2 * np))) return r;
    if ((r = dmalloc(ctx, &B->acc2, sizeof(double) * 3 * np))) return r;
    if ((r = dmalloc(ctx, (char **)&B->rec2, tsz * 3 * np))) return r;
    if ((r = dmalloc(ctx, &B->part, sizeof(double) * 4 * (nb + 1)))) return r;
    if ((r = dmalloc(ctx, &B->st, sizeof(DpState)))) return r;
    AP_CUDA(cudaMallocHost((void **)&B->st_host, sizeof(DpState)));
    if ((r = dmalloc(ctx, &B->mus, sizeof(double) * 6 * np))) return r;
    if ((r = dmalloc(ctx, &B->cbuf, sizeof(double) * 9 * n))) return r;
    if ((r = dmalloc(ctx, (char **)&B->mz, 4 * tsz * 4 * np))) return r;
    if ((r = dmalloc(ctx, &B->gsc, sizeof(double) * 9 * np))) return r;
    if ((r = dmalloc(ctx, &B->e_scr, sizeof(double) * 2 + sizeof(unsigned int)))) return r;
    if ((r = dmalloc(ctx, &B->flag, sizeof(int)))) return r;
    if ((r = pme_bufs_create(ctx, &B->pme2))) return r;
    int lo = 0, hi = 0;
    AP_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    AP_CUDA(cudaStreamCreateWithPriority(&B->s_rec2, cudaStreamNonBlocking, hi));
    AP_CUDA(cudaEventCreateWithFlags(&B->ev_join2, cudaEventDisableTiming));
    return AP_OK;
}

}  // namespace

int dp_set_pairs(ap_ctx *ctx, int n_pairs, const int *d_pairs, const double *d_scales) {
    int r = reserve(ctx);
    if (r) return r;
    DpBuffers *B = dpb(ctx);
    B->n_pairs = 0;   // no table until this one is copied and checked
    B->field_valid = 0;
    if (n_pairs > B->cap_pairs) {
        if (B->pairs) cudaFree(B->pairs);
        if (B->scales) cudaFree(B->scales);
        B->pairs = nullptr;
        B->scales = nullptr;
        B->cap_pairs = 0;
        AP_CUDA(cudaMalloc((void **)&B->pairs, sizeof(int2) * n_pairs));
        AP_CUDA(cudaMalloc((void **)&B->scales, sizeof(double2) * n_pairs));
        B->cap_pairs = n_pairs;
    }
    if (n_pairs == 0) return AP_OK;
    AP_CUDA(cudaMemsetAsync(B->flag, 0, sizeof(int), ctx->s0));
    k_pairs_check<<<ap_grid_for(n_pairs, 256), 256, 0, ctx->s0>>>(d_pairs, d_scales, n_pairs, ctx->n, B->pairs,
                                                                 B->scales, B->flag);
    AP_CUDA(cudaGetLastError());
    int bad = 0;
    AP_CUDA(cudaMemcpyAsync(&bad, B->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->s0));
    AP_CUDA(cudaStreamSynchronize(ctx->s0));
    if (bad) return ap_fail(ctx, AP_ERR_ARG, "a listed pair has an atom index out of range, i == j, or a non-finite scale");
    B->n_pairs = n_pairs;
    return AP_OK;
}

int dp_fields(ap_ctx *ctx, double *d_field_d, double *d_field_p) {
    if (!ctx->dp) return ap_fail(ctx, AP_ERR_STATE, "set_scaled_pairs() must come first");
    return ctx->prec == AP_FP64 ? fields_t<double>(ctx, d_field_d, d_field_p)
                                : fields_t<float>(ctx, d_field_d, d_field_p);
}

int dp_solve(ap_ctx *ctx, const double *gd, const double *gp, double tol, int max_iter, double *d_mu_d,
             double *d_mu_p, ap_solve_info *info) {
    if (!ctx->dp || !dpb(ctx)->field_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field_dp() must come first");
    ctx->last_solver = 2;
    return ctx->prec == AP_FP64 ? solve_t<double>(ctx, gd, gp, tol, max_iter, d_mu_d, d_mu_p, info)
                                : solve_t<float>(ctx, gd, gp, tol, max_iter, d_mu_d, d_mu_p, info);
}

int dp_forces(ap_ctx *ctx, const double *d_mu_d, const double *d_mu_p, double *d_energy, double *d_forces,
              double *d_virial) {
    if (!ctx->dp || !dpb(ctx)->field_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field_dp() must come first");
    DpBuffers *B = dpb(ctx);
    cudaStream_t s = ctx->s0;
    const int n3 = 3 * ctx->n;
    double *mu_s = B->cbuf, *dl = B->cbuf + n3, *ft = B->cbuf + 2 * n3;
    k_dp_split<<<ap_grid_for(n3, 256), 256, 0, s>>>(d_mu_d, d_mu_p, n3, B->cbuf);
    k_dp_slots<<<ap_grid_for(ctx->n_pad, 256), 256, 0, s>>>(d_mu_d, d_mu_p, ctx->perm, ctx->n, ctx->n_pad, B->mus);
    const int nb = ap_grid_for(ctx->n_pad, NT);
    k_dp_energy<<<nb, NT, 0, s>>>(B->mus, B->E2, ctx->n_pad, -0.5 * AP_COULOMB, B->part,
                                  (unsigned int *)(B->e_scr + 2), d_energy);
    AP_CUDA(cudaGetLastError());
    const size_t t4 = (ctx->prec == AP_FP64 ? sizeof(double) : sizeof(float)) * 4;
    void *mz[4];
    for (int k = 0; k < 4; ++k) mz[k] = (char *)B->mz + t4 * ctx->n_pad * k;
    if (ctx->prec == AP_FP64)
        k_zero_multipoles<double><<<ap_grid_for(ctx->n_pad, 256), 256, 0, s>>>(
            (const V4<double>::type *)ctx->posq, (const V4<double>::type *)ctx->dipd,
            (const V4<double>::type *)ctx->quad1, ctx->n_pad, (V4<double>::type *)B->mz);
    else
        k_zero_multipoles<float><<<ap_grid_for(ctx->n_pad, 256), 256, 0, s>>>(
            (const V4<float>::type *)ctx->posq, (const V4<float>::type *)ctx->dipd,
            (const V4<float>::type *)ctx->quad1, ctx->n_pad, (V4<float>::type *)B->mz);
    AP_CUDA(cudaGetLastError());
    int r;
    // the virial splits as the forces do: single-set terms at mu_s (with the listed pairs) minus
    // the mutual term of delta
    double *v1 = d_virial ? virial_acc(ctx, 0) : nullptr, *v2 = d_virial ? virial_acc(ctx, 1) : nullptr;
    if ((r = mutual_forces_run(ctx, dl, mz, B->gsc, B->gsc + (size_t)3 * ctx->n_pad, ft, v2))) return r;
    if ((r = forces_run_ex(ctx, mu_s, B->e_scr, d_forces, listed_forces, v1))) return r;
    k_dp_force_combine<<<ap_grid_for(n3, 256), 256, 0, s>>>(ft, n3, d_forces);
    AP_CUDA(cudaGetLastError());
    if (d_virial && (r = virial_out(ctx, v1, v2, d_virial))) return r;
    return AP_OK;
}

// the two-set real-space product on the current directions alone (timing), or (clear) a
// reset of the second accumulator afterwards
int dp_matvec2_launch(ap_ctx *ctx, cudaStream_t s, int clear) {
    if (!ctx->dp) return ap_fail(ctx, AP_ERR_STATE, "set_scaled_pairs() must come first");
    DpBuffers *B = dpb(ctx);
    if (clear) {
        AP_CUDA(cudaMemsetAsync(B->acc2, 0, sizeof(double) * 3 * ctx->n_pad, s));
        return AP_OK;
    }
    const size_t t4 = (ctx->prec == AP_FP64 ? sizeof(double) : sizeof(float)) * 4;
    const char *p0 = (const char *)B->p2;
    return real_matvec2_launch(ctx, p0, p0 + t4 * ctx->n_pad, ctx->acc, B->acc2, s);
}

int dp_info(ap_ctx *ctx, ap_solve_info *info) {
    if (!ctx->dp) return ap_fail(ctx, AP_ERR_STATE, "no two-set solve on this context");
    DpBuffers *B = dpb(ctx);
    AP_CUDA(cudaMemcpyAsync(B->st_host, B->st, sizeof(DpState), cudaMemcpyDeviceToHost, ctx->s0));
    AP_CUDA(cudaStreamSynchronize(ctx->s0));
    const DpState *h = B->st_host;
    info->iterations = h->iter;
    info->eps_debye = fmax(h->eps[0], h->eps[1]);
    info->eps_initial = fmax(h->eps0[0], h->eps0[1]);
    info->status = h->status;
    if (h->nonfinite) return ap_fail(ctx, AP_ERR_NONFINITE, "non-finite value in the PCG reductions");
    return AP_OK;
}

void dp_forget_graph(ap_ctx *ctx) {
    DpBuffers *B = dpb(ctx);
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
    B->exec_tried = 0;
}

void dp_release(ap_ctx *ctx) { dp_release_impl(ctx); }

void dp_release_impl(ap_ctx *ctx) {
    DpBuffers *B = dpb(ctx);
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    void *ptrs[] = {B->pairs, B->scales, B->E2, B->corr, B->mu2, B->r2, B->q2, B->p2, B->acc2, B->rec2, B->part,
                    B->st, B->mus, B->cbuf, B->e_scr, B->flag, B->mz, B->gsc, B->mu2f, B->r2f, B->q2f};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (B->st_host) cudaFreeHost(B->st_host);
    pme_bufs_destroy(&B->pme2);
    if (B->s_rec2) cudaStreamDestroy(B->s_rec2);
    if (B->ev_join2) cudaEventDestroy(B->ev_join2);
    delete B;
    ctx->dp = nullptr;
}
