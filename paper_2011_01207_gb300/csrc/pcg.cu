// a4 + a7 - Initial guess and the preconditioned conjugate gradient (paper Sec. 1.3: PCG with
// one polarization matrix-vector product per iteration; Sec. 3: diagonal preconditioner,
// threshold 1e-5).
//
//   mu_0 = guess (default alpha E);  r_0 = E - A mu_0;  z_0 = alpha r_0;  p_0 = z_0
//   loop:  q = A p;  gamma = (r.z)/(p.q);  mu += gamma p;  r -= gamma q;  z = alpha r
//          eps = 4.80321 sqrt(sum |z|^2 / n);  stop if eps <= tol
//          beta = (r.z)_new/(r.z)_old;  p = z + beta p
// with A = alpha^-1 - T and T p = T_real p (blocked pair kernel) + T_rec p (PME) + self p.
//
// FP64 mode: vectors mu, r, q in FP64, the search direction p in T for the pair and PME
// kernels, dot products and norms as FP64 block sums. Mixed and fixed modes: every vector in
// FP32 with FP64-grade sums of the dot products and norms (the kernels with the _f suffix).
// The convergence test runs on the device: the update kernel's last block decides, and
// inside a CUDA graph it drives a conditional WHILE node, so a whole solve is one graph
// launch with no host round trip per iteration (the paper's host-synchronous loop is what
// made DHFR drop to 12 ns/day, Sec. 3).
#include "common.cuh"
#include "vec_f32.cuh"

#include <cmath>
#include <cstdlib>
#include <type_traits>

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s);

namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// block-wide sum of two values, lane 0 of warp 0 returns them
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sa[NT / 32], sb[NT / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < NT / 32 ? sa[l] : 0.0;
        b = l < NT / 32 ? sb[l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

constexpr int NT = 256;

// mu_0 and the matvec input p := mu_0 (caller-order guess gathered into slots)
// also the diagonal of A, 1/alpha - self coefficient, so the iterations need no division
template <class T>
__global__ void k_init_guess(const double *__restrict__ guess, const double *__restrict__ E,
                             const double *__restrict__ alpha, const int *__restrict__ perm, int n, int n_pad,
                             double *__restrict__ mu, typename V4<T>::type *__restrict__ p, double self_coef,
                             double *__restrict__ dg) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double al = alpha[s];
    dg[s] = al > 0.0 ? 1.0 / al - self_coef : 0.0;
    double m[3] = {0.0, 0.0, 0.0};
    if (s < n) {
        if (guess) {
            int i = perm[s];
            for (int c = 0; c < 3; ++c) m[c] = guess[3 * i + c];
        } else {
            for (int c = 0; c < 3; ++c) m[c] = alpha[s] * E[c * n_pad + s];
        }
    }
    for (int c = 0; c < 3; ++c) mu[c * n_pad + s] = m[c];
    typename V4<T>::type v;
    v.x = (T)m[0]; v.y = (T)m[1]; v.z = (T)m[2]; v.w = (T)0;
    p[s] = v;
}

// sum of nparts partials (one block of NT threads, fixed order: deterministic)
__device__ __forceinline__ void sum_partials2(const double *part, int nparts, double &a, double &b) {
    a = 0.0;
    b = 0.0;
    for (int k = threadIdx.x; k < nparts; k += NT) {
        a += __ldcg(part + k);
        b += __ldcg(part + nparts + k);
    }
    block_sum2<NT>(a, b);
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, const PcgState *st) {
    cudaGraphSetConditional(h, (st->done || st->max_iter < 1) ? 0u : 1u);
}

// closes an iteration (thread 0 of the update kernel's last block, after the partials are
// summed in a fixed order): sets the convergence measure, beta and the stop decision; inside
// the graph it also drives the WHILE node - never beyond max_iter iterations, so the loop
// cannot spin forever
__device__ void finish_iteration(PcgState *st, double rzn, double zzt, int n, cudaGraphConditionalHandle h,
                                 int use_cond) {
    const double eps = AP_DEBYE * sqrt(zzt / n);
    st->iter += 1;
    st->guard += 1;
    st->eps = eps;
    const bool bad = !isfinite(eps) || !isfinite(st->gamma);
    if (bad) st->nonfinite = 1;
    if (eps <= st->tol || bad) {
        st->done = 1;
        st->status = bad ? AP_ERR_NONFINITE : AP_OK;
    } else if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = AP_NOT_CONVERGED;
    }
    st->beta = rzn / st->rz;
    st->rz = rzn;
    if (use_cond) {
        const bool more = !st->done && st->guard < st->max_iter;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// true in exactly one block per launch, the last to finish, once every block's partial sums
// are globally visible; the counter is reset for the next launch
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

// r_0 = E - A mu_0, partial sums of r.z and z.z; clears acc and p. The last block sums the
// partials in a fixed order and sets the initial state (eps_0, the stop decision).
template <class T>
__global__ void k_init_residual(const double *__restrict__ E, const double *__restrict__ alpha,
                                const double *__restrict__ mu, double *__restrict__ acc,
                                const T *__restrict__ rec, const double *__restrict__ dg, int n_pad,
                                double *__restrict__ r, typename V4<T>::type *__restrict__ p,
                                double *__restrict__ part, int fixed, PcgState *st, int n, double tol,
                                int max_iter) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0, zz = 0.0;
    if (s < n_pad) {
        const double a = alpha[s], d = dg[s];
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            double Amu = a > 0.0 ? mu[k] * d - acc_value(acc, k, fixed) - (double)rec[k] : 0.0;
            double rr = a > 0.0 ? E[k] - Amu : 0.0;
            r[k] = rr;
            acc[k] = 0.0;
            rz += rr * a * rr;
            zz += a * rr * a * rr;
        }
        typename V4<T>::type v;
        v.x = v.y = v.z = v.w = (T)0;
        p[s] = v;
    }
    block_sum2<NT>(rz, zz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rz;
        part[gridDim.x + blockIdx.x] = zz;
    }
    if (!last_block(&st->blocks_done)) return;
    double rzt, zzt;
    sum_partials2(part, gridDim.x, rzt, zzt);
    if (threadIdx.x != 0) return;
    const double eps = AP_DEBYE * sqrt(zzt / n);
    st->rz = rzt;
    st->eps = eps;
    st->eps0 = eps;
    st->tol = tol;
    st->iter = 0;
    st->max_iter = max_iter;
    st->beta = 0.0;
    st->gamma = 0.0;
    st->nonfinite = !isfinite(eps);
    st->done = (eps <= tol) || st->nonfinite;
    st->status = st->nonfinite ? AP_ERR_NONFINITE : AP_OK;
    st->pq = st->rz_new = st->zz = 0.0;
    st->guard = 0;
}

// p = alpha r + beta p
template <class T>
__global__ void k_direction(const double *__restrict__ r, const double *__restrict__ alpha, int n_pad,
                            typename V4<T>::type *__restrict__ p, const PcgState *__restrict__ st) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double b = st->beta, a = alpha[s];
    typename V4<T>::type v = p[s];
    v.x = (T)(a * r[s] + b * (double)v.x);
    v.y = (T)(a * r[n_pad + s] + b * (double)v.y);
    v.z = (T)(a * r[2 * n_pad + s] + b * (double)v.z);
    p[s] = v;
}

// q = A p = (1/alpha - self) p - T_real p - T_rec p; partial p.q; clears acc. The last
// block sums the partials and sets gamma = (r.z) / (p.q).
template <class T>
__global__ void k_apply(const typename V4<T>::type *__restrict__ p, const double *__restrict__ dg,
                        double *__restrict__ acc, const T *__restrict__ rec, int n_pad, double *__restrict__ q,
                        double *__restrict__ part, PcgState *st, int fixed) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double pq = 0.0, dummy = 0.0;
    if (s < n_pad) {
        const double d = dg[s];
        typename V4<T>::type v = p[s];
        const double pv[3] = {(double)v.x, (double)v.y, (double)v.z};
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            const double qq = pv[c] * d - acc_value(acc, k, fixed) - (double)rec[k];
            q[k] = qq;
            acc[k] = 0.0;
            pq += pv[c] * qq;
        }
    }
    block_sum2<NT>(pq, dummy);
    if (threadIdx.x == 0) part[blockIdx.x] = pq;
    if (!last_block(&st->blocks_done)) return;
    double tot = 0.0, dummy2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += NT) tot += __ldcg(part + k);
    block_sum2<NT>(tot, dummy2);
    if (threadIdx.x == 0) {
        st->pq = tot;
        st->gamma = st->rz / tot;
    }
}

// mu += gamma p; r -= gamma q; partial r.z and z.z per block; the last block sums them and
// closes the iteration
template <class T>
__global__ void k_update(const typename V4<T>::type *__restrict__ p, const double *__restrict__ q,
                         const double *__restrict__ alpha, int n_pad, double *__restrict__ mu,
                         double *__restrict__ r, PcgState *st, double *__restrict__ part, int n,
                         cudaGraphConditionalHandle h, int use_cond) {
    const double gamma = st->gamma;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0, zz = 0.0;
    if (s < n_pad) {
        const double a = alpha[s];
        typename V4<T>::type v = p[s];
        const double pv[3] = {(double)v.x, (double)v.y, (double)v.z};
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            mu[k] += gamma * pv[c];
            const double rr = r[k] - gamma * q[k];
            r[k] = rr;
            const double z = a * rr;
            rz += rr * z;
            zz += z * z;
        }
    }
    block_sum2<NT>(rz, zz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rz;
        part[gridDim.x + blockIdx.x] = zz;
    }
    if (!last_block(&st->blocks_done2)) return;
    double rzn, zzt;
    sum_partials2(part, gridDim.x, rzn, zzt);
    if (threadIdx.x == 0) finish_iteration(st, rzn, zzt, n, h, use_cond);
}

// ---------------------------------------------------------------------------------------
// The same iteration with the vectors in FP32 (mixed and fixed-point modes): mu, r, q and p
// stored as float4 per slot, the diagonal and alpha as a float2, every vector operation in
// FP32. The dot products and norms keep FP64-grade sums without FP64 arithmetic per slot:
// each product is split exactly into its rounded value and error (fma), both summed in a
// compensated FP32 pair (TwoSum, ~48 bits) per thread, warp and block; the block's pair is
// converted exactly to FP64 and the last block adds the partials in FP64 in a fixed order.
// (GB300 issues FP64 at a small fraction of its FP32 rate; the FP64 kernels above spent a
// few microseconds per iteration on it.)

// mu_0 (FP32) and the matvec input p := mu_0; the diagonal 1/alpha - self and alpha as FP32
__global__ void k_init_guess_f(const double *__restrict__ guess, const double *__restrict__ E,
                               const double *__restrict__ alpha, const int *__restrict__ perm, int n, int n_pad,
                               float4 *__restrict__ mu, float4 *__restrict__ p, double self_coef,
                               float2 *__restrict__ dga) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const double al = alpha[s];
    dga[s] = make_float2(al > 0.0 ? (float)(1.0 / al - self_coef) : 0.f, (float)al);
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < n) {
        if (guess) {
            const int i = perm[s];
            m = make_float4((float)guess[3 * i], (float)guess[3 * i + 1], (float)guess[3 * i + 2], 0.f);
        } else {
            m = make_float4((float)(al * E[s]), (float)(al * E[n_pad + s]), (float)(al * E[2 * n_pad + s]), 0.f);
        }
    }
    mu[s] = m;
    p[s] = m;
}

// r_0 = E - A mu_0 (formed in FP64 once per solve, stored in FP32), partial r.z and z.z of the
// stored r; clears acc and p. The last block sets the initial state.
__global__ void k_init_residual_f(const double *__restrict__ E, const float2 *__restrict__ dga,
                                  const float4 *__restrict__ mu, double *__restrict__ acc,
                                  const float *__restrict__ rec, int n_pad, float4 *__restrict__ r,
                                  float4 *__restrict__ p, double *__restrict__ part, int fixed, PcgState *st, int n,
                                  double tol, int max_iter) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 rz = {0.f, 0.f}, zz = {0.f, 0.f};
    if (s < n_pad) {
        const float2 d = dga[s];
        const float4 m = mu[s];
        const float mv[3] = {m.x, m.y, m.z};
        float rv[3];
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            const double Amu = d.y > 0.f ? (double)mv[c] * d.x - acc_value(acc, k, fixed) - (double)rec[k] : 0.0;
            rv[c] = d.y > 0.f ? (float)(E[k] - Amu) : 0.f;
            acc[k] = 0.0;
            const float z = d.y * rv[c];
            f2_add_prod(rz, rv[c], z);
            f2_add_prod(zz, z, z);
        }
        r[s] = make_float4(rv[0], rv[1], rv[2], 0.f);
        p[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    double brz = 0.0, bzz = 0.0;
    block_sum2_f2<NT>(rz, zz, brz, bzz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = brz;
        part[gridDim.x + blockIdx.x] = bzz;
    }
    if (!last_block(&st->blocks_done)) return;
    double rzt, zzt;
    sum_partials2(part, gridDim.x, rzt, zzt);
    if (threadIdx.x != 0) return;
    const double eps = AP_DEBYE * sqrt(zzt / n);
    st->rz = rzt;
    st->eps = eps;
    st->eps0 = eps;
    st->tol = tol;
    st->iter = 0;
    st->max_iter = max_iter;
    st->beta = 0.0;
    st->gamma = 0.0;
    st->nonfinite = !isfinite(eps);
    st->done = (eps <= tol) || st->nonfinite;
    st->status = st->nonfinite ? AP_ERR_NONFINITE : AP_OK;
    st->pq = st->rz_new = st->zz = 0.0;
    st->guard = 0;
}

// p = alpha r + beta p; clears the real-space accumulator and the PME grid for the next product
// (here rather than in k_apply_f, whose last-block fence would wait for these stores, or as a
// separate clearing step at the head of the reciprocal branch, which is the longer branch of
// the product)
__global__ void k_direction_f(const float4 *__restrict__ r, const float2 *__restrict__ dga, int n_pad,
                              float4 *__restrict__ p, const PcgState *__restrict__ st, double *__restrict__ acc,
                              float *__restrict__ grid, size_t ngrid) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    float4 *g4 = reinterpret_cast<float4 *>(grid);   // cudaMalloc'd: 16-byte aligned
    for (size_t i = s; i < ngrid / 4; i += stride) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < (int)(ngrid & 3)) grid[(ngrid & ~(size_t)3) + s] = 0.f;
    if (s >= n_pad) return;
    acc[s] = 0.0;
    acc[n_pad + s] = 0.0;
    acc[2 * (size_t)n_pad + s] = 0.0;
    const float b = (float)st->beta, a = dga[s].y;
    const float4 rv = r[s];
    float4 v = p[s];
    v.x = fmaf(a, rv.x, b * v.x);
    v.y = fmaf(a, rv.y, b * v.y);
    v.z = fmaf(a, rv.z, b * v.z);
    p[s] = v;
}

// q = (1/alpha - self) p - T_real p - T_rec p; partial p.q. The last block sets
// gamma = (r.z) / (p.q).
__global__ void k_apply_f(const float4 *__restrict__ p, const float2 *__restrict__ dga, const double *__restrict__ acc,
                          const float *__restrict__ rec, int n_pad, float4 *__restrict__ q, double *__restrict__ part,
                          PcgState *st, int fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 pq = {0.f, 0.f}, none = {0.f, 0.f};
    if (s < n_pad) {
        const float d = dga[s].x;
        const float4 v = p[s];
        const float pv[3] = {v.x, v.y, v.z};
        float qv[3];
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            qv[c] = fmaf(pv[c], d, -acc_f32(acc, k, fixed)) - rec[k];
            f2_add_prod(pq, pv[c], qv[c]);
        }
        q[s] = make_float4(qv[0], qv[1], qv[2], 0.f);
    }
    double bpq = 0.0, unused = 0.0;
    block_sum2_f2<NT>(pq, none, bpq, unused);
    if (threadIdx.x == 0) part[blockIdx.x] = bpq;
    if (!last_block(&st->blocks_done)) return;
    double tot = 0.0, dummy2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += NT) tot += __ldcg(part + k);
    block_sum2<NT>(tot, dummy2);
    if (threadIdx.x == 0) {
        st->pq = tot;
        st->gamma = st->rz / tot;
    }
}

// mu += gamma p; r -= gamma q; partial r.z and z.z; the last block closes the iteration
__global__ void k_update_f(const float4 *__restrict__ p, const float4 *__restrict__ q,
                           const float2 *__restrict__ dga, int n_pad, float4 *__restrict__ mu,
                           float4 *__restrict__ r, PcgState *st, double *__restrict__ part, int n,
                           cudaGraphConditionalHandle h, int use_cond) {
    const float g = (float)st->gamma;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    F2 rz = {0.f, 0.f}, zz = {0.f, 0.f};
    if (s < n_pad) {
        const float a = dga[s].y;
        const float4 pv = p[s], qv = q[s];
        float4 m = mu[s], rv = r[s];
        m.x = fmaf(g, pv.x, m.x);
        m.y = fmaf(g, pv.y, m.y);
        m.z = fmaf(g, pv.z, m.z);
        rv.x = fmaf(-g, qv.x, rv.x);
        rv.y = fmaf(-g, qv.y, rv.y);
        rv.z = fmaf(-g, qv.z, rv.z);
        mu[s] = m;
        r[s] = rv;
        const float rr[3] = {rv.x, rv.y, rv.z};
        for (int c = 0; c < 3; ++c) {
            const float z = a * rr[c];
            f2_add_prod(rz, rr[c], z);
            f2_add_prod(zz, z, z);
        }
    }
    double brz = 0.0, bzz = 0.0;
    block_sum2_f2<NT>(rz, zz, brz, bzz);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = brz;
        part[gridDim.x + blockIdx.x] = bzz;
    }
    if (!last_block(&st->blocks_done2)) return;
    double rzn, zzt;
    sum_partials2(part, gridDim.x, rzn, zzt);
    if (threadIdx.x == 0) finish_iteration(st, rzn, zzt, n, h, use_cond);
}

// the FP32 dipoles to the caller's order in FP64
__global__ void k_unsort_f4(const float4 *__restrict__ src, const int *__restrict__ iperm, int n,
                            double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = src[iperm[i]];
    out[3 * i] = v.x;
    out[3 * i + 1] = v.y;
    out[3 * i + 2] = v.z;
}

// T p: reciprocal branch on `aux`, real space on `main`, joined back into `main`
template <class T>
int matvec_into(ap_ctx *ctx, const void *p, cudaStream_t main, cudaStream_t aux, bool grid_cleared = false) {
    AP_CUDA(cudaEventRecord(ctx->ev_fork, main));
    AP_CUDA(cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
    int rc = pme_dipole_field(ctx, p, aux, grid_cleared);
    if (rc) return rc;
    rc = real_matvec_launch(ctx, p, main);
    if (rc) return rc;
    AP_CUDA(cudaEventRecord(ctx->ev_join, aux));
    AP_CUDA(cudaStreamWaitEvent(main, ctx->ev_join, 0));
    return AP_OK;
}

template <class T>
int matvec_into(ap_ctx *ctx, const void *p) { return matvec_into<T>(ctx, p, ctx->s0, ctx->s1); }

double self_coef(const ap_ctx *ctx) { return 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI); }

template <class T>
int enqueue_iteration(ap_ctx *ctx, cudaGraphConditionalHandle h, int use_cond, cudaStream_t main,
                      cudaStream_t aux) {
    typedef typename V4<T>::type T4;
    const int nb = ap_grid_for(ctx->n_pad, NT);
    double *part_pq = ctx->red_part, *part_rz = ctx->red_part + nb;
    if constexpr (std::is_same<T, float>::value) {
        k_direction_f<<<nb, NT, 0, main>>>(ctx->r_f, ctx->dga_f, ctx->n_pad, (float4 *)ctx->p, ctx->st, ctx->acc,
                                           (float *)ctx->grid, ctx->ngrid);
        AP_CUDA(cudaGetLastError());
        int rc = matvec_into<T>(ctx, ctx->p, main, aux, true);   // the grid was cleared above
        if (rc) return rc;
        k_apply_f<<<nb, NT, 0, main>>>((const float4 *)ctx->p, ctx->dga_f, ctx->acc, (const float *)ctx->rec,
                                       ctx->n_pad, ctx->q_f, part_pq, ctx->st, ctx->fixed);
        k_update_f<<<nb, NT, 0, main>>>((const float4 *)ctx->p, ctx->q_f, ctx->dga_f, ctx->n_pad, ctx->mu_f, ctx->r_f,
                                        ctx->st, part_rz, ctx->n, h, use_cond);
    } else {
        k_direction<T><<<nb, NT, 0, main>>>(ctx->r, ctx->alpha, ctx->n_pad, (T4 *)ctx->p, ctx->st);
        AP_CUDA(cudaGetLastError());
        int rc = matvec_into<T>(ctx, ctx->p, main, aux);
        if (rc) return rc;
        k_apply<T><<<nb, NT, 0, main>>>((const T4 *)ctx->p, ctx->dg, ctx->acc, (const T *)ctx->rec, ctx->n_pad,
                                         ctx->qv, part_pq, ctx->st, ctx->fixed);
        k_update<T><<<nb, NT, 0, main>>>((const T4 *)ctx->p, ctx->qv, ctx->alpha, ctx->n_pad, ctx->mu, ctx->r,
                                          ctx->st, part_rz, ctx->n, h, use_cond);
    }
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// the solve loop as one graph: [set condition] -> WHILE { one iteration }
template <class T>
int build_graph(ap_ctx *ctx) {
    ctx->graph_tried = 1;
    // AP_SOLVE_GRAPH=0 keeps the host-driven loop (the same kernels, launched one by one):
    // profilers cannot attribute kernels inside graphs that hold conditional nodes
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
    const PcgState *stp = ctx->st;
    void *args[2] = {(void *)&h, (void *)&stp};
    kp.func = (void *)k_set_cond;
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
    // capture on a library-owned stream: the caller's may be the legacy default stream,
    // which cannot be captured; the instantiated graph is launched on the caller's stream
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
        return AP_OK;      // fall back to the host loop
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return AP_OK;
    }
    cudaGraphDestroy(g);
    ctx->solve_exec = ex;
    ctx->graph_ok = 1;
    return AP_OK;
}

template <class T>
int solve_t(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, double *d_mu, ap_solve_info *info) {
    typedef typename V4<T>::type T4;
    const int nb = ap_grid_for(ctx->n_pad, NT);
    cudaStream_t s = ctx->s0;
    AP_CUDA(cudaMemsetAsync(ctx->st, 0, sizeof(PcgState), s));
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, s));
    constexpr bool F32 = std::is_same<T, float>::value;   // FP32 vectors (mixed and fixed modes)
    if (F32)
        k_init_guess_f<<<nb, NT, 0, s>>>(d_guess, ctx->E, ctx->alpha, ctx->perm, ctx->n, ctx->n_pad, ctx->mu_f,
                                         (float4 *)ctx->p, self_coef(ctx), ctx->dga_f);
    else
        k_init_guess<T><<<nb, NT, 0, s>>>(d_guess, ctx->E, ctx->alpha, ctx->perm, ctx->n, ctx->n_pad, ctx->mu,
                                           (T4 *)ctx->p, self_coef(ctx), ctx->dg);
    AP_CUDA(cudaGetLastError());
    int rc = matvec_into<T>(ctx, ctx->p);
    if (rc) return rc;
    if (F32)
        k_init_residual_f<<<nb, NT, 0, s>>>(ctx->E, ctx->dga_f, ctx->mu_f, ctx->acc, (const float *)ctx->rec,
                                            ctx->n_pad, ctx->r_f, (float4 *)ctx->p, ctx->red_part, ctx->fixed,
                                            ctx->st, ctx->n, tol, max_iter);
    else
        k_init_residual<T><<<nb, NT, 0, s>>>(ctx->E, ctx->alpha, ctx->mu, ctx->acc, (const T *)ctx->rec, ctx->dg,
                                              ctx->n_pad, ctx->r, (T4 *)ctx->p, ctx->red_part, ctx->fixed, ctx->st,
                                              ctx->n, tol, max_iter);
    AP_CUDA(cudaGetLastError());
    // the solution to the caller's order, in FP64
    auto unsort_mu = [&](cudaStream_t st) {
        if (F32) k_unsort_f4<<<ap_grid_for(ctx->n, 256), 256, 0, st>>>(ctx->mu_f, ctx->iperm, ctx->n, d_mu);
        else unsort3(ctx, ctx->mu, d_mu, st);
    };
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    AP_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusActive) {
        // the caller is capturing a larger graph: add the WHILE node to it directly
        if (info) return ap_fail(ctx, AP_ERR_ARG, "h_info must be NULL while the stream is being captured");
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        AP_CUDA(cudaStreamGetCaptureInfo(s, &cap, nullptr, &g, &deps, nullptr, &ndeps));
        cudaGraphConditionalHandle h;
        AP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        k_set_cond<<<1, 1, 0, s>>>(h, ctx->st);
        AP_CUDA(cudaGetLastError());
        AP_CUDA(cudaStreamGetCaptureInfo(s, &cap, nullptr, &g, &deps, nullptr, &ndeps));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        AP_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
        AP_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        AP_CUDA(cudaStreamBeginCaptureToGraph(ctx->s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        rc = enqueue_iteration<T>(ctx, h, 1, ctx->s2, ctx->s3);
        cudaGraph_t captured = nullptr;
        cudaError_t ec = cudaStreamEndCapture(ctx->s2, &captured);
        if (rc) return rc;
        if (ec != cudaSuccess) return ap_fail(ctx, AP_ERR_CUDA, std::string("body capture: ") + cudaGetErrorString(ec));
        unsort_mu(s);
        AP_CUDA(cudaGetLastError());
        return AP_OK;
    }
    if (!ctx->graph_tried) {
        if (build_graph<T>(ctx) != AP_OK) {   // no graph: the host-driven loop below
            cudaGetLastError();
            ctx->err.clear();
            ctx->graph_ok = 0;
        }
    }
    if (ctx->graph_ok) {
        AP_CUDA(cudaGraphLaunch(ctx->solve_exec, s));
    } else {
        // host-driven loop: one status read per iteration
        for (int it = 0; it < max_iter; ++it) {
            AP_CUDA(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
            AP_CUDA(cudaStreamSynchronize(s));
            if (ctx->st_host->done) break;
            rc = enqueue_iteration<T>(ctx, 0, 0, ctx->s0, ctx->s1);
            if (rc) return rc;
        }
    }
    unsort_mu(s);
    AP_CUDA(cudaGetLastError());
    if (info) {
        AP_CUDA(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        AP_CUDA(cudaStreamSynchronize(s));
        info->iterations = ctx->st_host->iter;
        info->eps_debye = ctx->st_host->eps;
        info->eps_initial = ctx->st_host->eps0;
        info->status = ctx->st_host->status;
        if (ctx->st_host->nonfinite) return ap_fail(ctx, AP_ERR_NONFINITE, "non-finite value in the PCG reductions");
        return ctx->st_host->status;
    }
    return AP_OK;
}

}  // namespace

// T applied to ctx->p (real space on `main`, reciprocal on `aux`, joined into `main`), into
// ctx->acc and ctx->rec; for other solvers of the same system
int dipole_operator_into(ap_ctx *ctx, cudaStream_t main, cudaStream_t aux) {
    return ctx->prec == AP_FP64 ? matvec_into<double>(ctx, ctx->p, main, aux)
                                : matvec_into<float>(ctx, ctx->p, main, aux);
}

// one iteration's vector work (direction, q = A p with its p.q reduction, update with its
// r.z / z.z reduction) on `s`, for timing; it advances the last solve's state
int pcg_vectors_launch(ap_ctx *ctx, cudaStream_t s) {
    const int nb = ap_grid_for(ctx->n_pad, NT);
    double *part_pq = ctx->red_part, *part_rz = ctx->red_part + nb;
    if (ctx->prec == AP_FP64) {
        typedef V4<double>::type T4;
        k_direction<double><<<nb, NT, 0, s>>>(ctx->r, ctx->alpha, ctx->n_pad, (T4 *)ctx->p, ctx->st);
        k_apply<double><<<nb, NT, 0, s>>>((const T4 *)ctx->p, ctx->dg, ctx->acc, (const double *)ctx->rec, ctx->n_pad,
                                          ctx->qv, part_pq, ctx->st, ctx->fixed);
        k_update<double><<<nb, NT, 0, s>>>((const T4 *)ctx->p, ctx->qv, ctx->alpha, ctx->n_pad, ctx->mu, ctx->r, ctx->st,
                                           part_rz, ctx->n, 0, 0);
    } else {
        k_direction_f<<<nb, NT, 0, s>>>(ctx->r_f, ctx->dga_f, ctx->n_pad, (float4 *)ctx->p, ctx->st, ctx->acc,
                                        (float *)ctx->grid, ctx->ngrid);
        k_apply_f<<<nb, NT, 0, s>>>((const float4 *)ctx->p, ctx->dga_f, ctx->acc, (const float *)ctx->rec, ctx->n_pad,
                                    ctx->q_f, part_pq, ctx->st, ctx->fixed);
        k_update_f<<<nb, NT, 0, s>>>((const float4 *)ctx->p, ctx->q_f, ctx->dga_f, ctx->n_pad, ctx->mu_f, ctx->r_f,
                                     ctx->st, part_rz, ctx->n, 0, 0);
    }
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int pcg_solve(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, double *d_mu, ap_solve_info *info) {
    return ctx->prec == AP_FP64 ? solve_t<double>(ctx, d_guess, tol, max_iter, d_mu, info)
                                : solve_t<float>(ctx, d_guess, tol, max_iter, d_mu, info);
}

// a plain T p for tests: out[n][3] (caller order) = (T_real + T_rec + self) applied to v
template <class T>
__global__ void k_load_vec(const double *__restrict__ v, const int *__restrict__ perm, int n, int n_pad,
                           typename V4<T>::type *__restrict__ p) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    typename V4<T>::type w;
    w.x = w.y = w.z = w.w = (T)0;
    if (s < n) {
        int i = perm[s];
        w.x = (T)v[3 * i]; w.y = (T)v[3 * i + 1]; w.z = (T)v[3 * i + 2];
    }
    p[s] = w;
}

template <class T>
__global__ void k_tp_out(const typename V4<T>::type *__restrict__ p, const double *__restrict__ acc,
                         const T *__restrict__ rec, double self_coef, int n_pad, double *__restrict__ out, int fixed) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    typename V4<T>::type v = p[s];
    const double pv[3] = {(double)v.x, (double)v.y, (double)v.z};
    for (int c = 0; c < 3; ++c)
        out[c * n_pad + s] = acc_value(acc, (size_t)c * n_pad + s, fixed) + (double)rec[c * n_pad + s] + self_coef * pv[c];
}

template <class T>
int apply_t(ap_ctx *ctx, const double *d_v, double *d_out) {
    typedef typename V4<T>::type T4;
    const int nb = ap_grid_for(ctx->n_pad, NT);
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, ctx->s0));
    k_load_vec<T><<<nb, NT, 0, ctx->s0>>>(d_v, ctx->perm, ctx->n, ctx->n_pad, (T4 *)ctx->p);
    int rc = matvec_into<T>(ctx, ctx->p);
    if (rc) return rc;
    k_tp_out<T><<<nb, NT, 0, ctx->s0>>>((const T4 *)ctx->p, ctx->acc, (const T *)ctx->rec, self_coef(ctx),
                                         ctx->n_pad, ctx->qv, ctx->fixed);
    unsort3(ctx, ctx->qv, d_out, ctx->s0);
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, ctx->s0));
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int dipole_field_apply(ap_ctx *ctx, const double *d_v, double *d_out) {
    return ctx->prec == AP_FP64 ? apply_t<double>(ctx, d_v, d_out) : apply_t<float>(ctx, d_v, d_out);
}
