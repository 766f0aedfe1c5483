// a8 - Learned initial guess: a per-atom perceptron 16 -> 128 -> 128 -> 3 (ReLU) whose output
// corrects the direct-field guess, mu0_i = alpha_i E_i + s_out R_i y_i (R_i the atom's frame).
// Features are rotation-invariant (fields expressed in the atom's local frame), so the
// guess rotates with the system. BF16 weights and activations, FP32 accumulation on the
// tcgen05 tensor cores with TMEM accumulators; one CTA of 128 threads handles 128 atoms at a
// time (M = 128), one thread per atom row for the epilogues.
//
// The paper has no learned component; this is the guess of the solver's PCG (any guess is
// allowed: PCG still converges to the same tolerance, it only changes the iteration count).
#include "common.cuh"
#include "tc.cuh"

#include <cmath>

#define MLP_IN 16
#define MLP_H 128
#define MLP_OUT 3
#define MLP_OUTP 16
// packed parameter block (bytes)
#define MLP_W1T_OFF 0                      // bf16 W1^T [128][16], core-matrix layout
#define MLP_W2T_OFF 4096                   // bf16 W2^T [128][128]
#define MLP_W3T_OFF (4096 + 32768)         // bf16 W3^T [16][128] (rows >= 3 zero)
#define MLP_B1_OFF (MLP_W3T_OFF + 4096)    // fp32 b1[128]
#define MLP_B2_OFF (MLP_B1_OFF + 512)      // fp32 b2[128]
#define MLP_B3_OFF (MLP_B2_OFF + 512)      // fp32 b3[16]
#define MLP_PACKED_BYTES (MLP_B3_OFF + 64)
// master parameters (fp32): W1 [16][128], b1, W2 [128][128], b2, W3 [128][3], b3
#define MLP_P_W1 0
#define MLP_P_B1 (MLP_P_W1 + MLP_IN * MLP_H)
#define MLP_P_W2 (MLP_P_B1 + MLP_H)
#define MLP_P_B2 (MLP_P_W2 + MLP_H * MLP_H)
#define MLP_P_W3 (MLP_P_B2 + MLP_H)
#define MLP_P_B3 (MLP_P_W3 + MLP_H * MLP_OUT)
#define MLP_NPARAM (MLP_P_B3 + MLP_OUT)

#define MLP_E_SCALE 0.05
#define MLP_OUT_SCALE 0.02

static __device__ int g_mlp_error;   // set when a bounded tensor-core wait gave up

namespace {

__global__ void k_mlp_pack(const float *__restrict__ p, unsigned char *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    __nv_bfloat16 *w1 = (__nv_bfloat16 *)(out + MLP_W1T_OFF);
    __nv_bfloat16 *w2 = (__nv_bfloat16 *)(out + MLP_W2T_OFF);
    __nv_bfloat16 *w3 = (__nv_bfloat16 *)(out + MLP_W3T_OFF);
    if (t < MLP_H * MLP_IN) {   // W1t[n][k] = W1[k][n]
        const int n = t / MLP_IN, k = t % MLP_IN;
        w1[tc::cm_offset(n, k, MLP_IN) / 2] = __float2bfloat16(p[MLP_P_W1 + k * MLP_H + n]);
    }
    if (t < MLP_H * MLP_H) {    // W2t[n][k] = W2[k][n]
        const int n = t / MLP_H, k = t % MLP_H;
        w2[tc::cm_offset(n, k, MLP_H) / 2] = __float2bfloat16(p[MLP_P_W2 + k * MLP_H + n]);
    }
    if (t < MLP_OUTP * MLP_H) { // W3t[o][h] = W3[h][o], zero rows o >= 3
        const int o = t / MLP_H, h = t % MLP_H;
        w3[tc::cm_offset(o, h, MLP_H) / 2] = __float2bfloat16(o < MLP_OUT ? p[MLP_P_W3 + h * MLP_OUT + o] : 0.f);
    }
    float *b1 = (float *)(out + MLP_B1_OFF), *b2 = (float *)(out + MLP_B2_OFF), *b3 = (float *)(out + MLP_B3_OFF);
    if (t < MLP_H) {
        b1[t] = p[MLP_P_B1 + t];
        b2[t] = p[MLP_P_B2 + t];
    }
    if (t < MLP_OUTP) b3[t] = t < MLP_OUT ? p[MLP_P_B3 + t] : 0.f;
}

struct __align__(16) FwdSmem {
    unsigned char w1[4096];
    unsigned char w2[32768];
    unsigned char w3[4096];
    unsigned char a[32768];      // activations: X [128][16] or H [128][128], core-matrix layout
    float b1[MLP_H], b2[MLP_H], b3[MLP_OUTP];
    uint64_t mbar;
    uint32_t taddr;
};

// bias + ReLU of this thread's TMEM row (128 columns) -> bf16 row of the next A operand
__device__ __forceinline__ void epilogue_relu(uint32_t trow, const float *bias, unsigned char *a, int row) {
#pragma unroll 1
    for (int c = 0; c < MLP_H; c += 32) {
        float v[32];
        tc::tmem_ld32(trow + c, v);
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
            __align__(16) __nv_bfloat16 h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16(fmaxf(v[g + e] + bias[c + g + e], 0.f));
            *(uint4 *)(a + tc::cm_offset(row, c + g, MLP_H)) = *(const uint4 *)h;
        }
    }
}

__global__ void __launch_bounds__(128) k_mlp_forward(const unsigned char *__restrict__ packed,
                                                     const float *__restrict__ feat, int n, float *__restrict__ y) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    FwdSmem &S = *reinterpret_cast<FwdSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights and biases into shared memory (the packed block mirrors the layout)
    {
        const uint4 *src = (const uint4 *)packed;
        uint4 *dw = (uint4 *)S.w1;
        for (int k = tid; k < (4096 + 32768 + 4096) / 16; k += 128) dw[k] = src[k];
        const float *bsrc = (const float *)(packed + MLP_B1_OFF);
        for (int k = tid; k < MLP_H; k += 128) {
            S.b1[k] = bsrc[k];
            S.b2[k] = bsrc[MLP_H + k];
        }
        if (tid < MLP_OUTP) S.b3[tid] = bsrc[2 * MLP_H + tid];
    }
    if (warp == 0) tc::tmem_alloc(&S.taddr, 128);
    if (tid == 0) tc::mbar_init(&S.mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = S.taddr;
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    const uint32_t sa = tc::smem_u32(S.a), sw1 = tc::smem_u32(S.w1), sw2 = tc::smem_u32(S.w2),
                   sw3 = tc::smem_u32(S.w3);
    constexpr uint32_t ID1 = tc::idesc_bf16(128, MLP_H, 0, 0);
    constexpr uint32_t ID3 = tc::idesc_bf16(128, MLP_OUTP, 0, 0);
    uint32_t phase = 0;
    bool ok = true;
    const int ntiles = (n + 127) / 128;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int atom = tile * 128 + tid;
        // features -> bf16 A operand [128][16]
        {
            __align__(16) __nv_bfloat16 h[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) h[k] = __float2bfloat16(atom < n ? feat[(size_t)atom * 16 + k] : 0.f);
            *(uint4 *)(S.a + tc::cm_offset(tid, 0, MLP_IN)) = *(const uint4 *)&h[0];
            *(uint4 *)(S.a + tc::cm_offset(tid, 8, MLP_IN)) = *(const uint4 *)&h[8];
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            tc::mma_bf16(tbase, tc::smem_desc(sa, 128, 256), tc::smem_desc(sw1, 128, 256), ID1, 0);
            tc::commit(&S.mbar);
        }
        ok = tc::mbar_wait(&S.mbar, phase);
        phase ^= 1;
        tc::fence_after();
        if (ok) epilogue_relu(trow, S.b1, S.a, tid);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < MLP_H / 16; ++kk)
                tc::mma_bf16(tbase, tc::smem_desc(sa + kk * 256, 128, 2048), tc::smem_desc(sw2 + kk * 256, 128, 2048),
                             ID1, kk > 0);
            tc::commit(&S.mbar);
        }
        if (ok) {
            ok = tc::mbar_wait(&S.mbar, phase);
            phase ^= 1;
        }
        tc::fence_after();
        if (ok) epilogue_relu(trow, S.b2, S.a, tid);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < MLP_H / 16; ++kk)
                tc::mma_bf16(tbase, tc::smem_desc(sa + kk * 256, 128, 2048), tc::smem_desc(sw3 + kk * 256, 128, 2048),
                             ID3, kk > 0);
            tc::commit(&S.mbar);
        }
        if (ok) {
            ok = tc::mbar_wait(&S.mbar, phase);
            phase ^= 1;
        }
        tc::fence_after();
        if (ok) {
            float v[32];
            tc::tmem_ld32(trow, v);
            if (atom < n)
                for (int o = 0; o < MLP_OUT; ++o) y[(size_t)atom * MLP_OUT + o] = v[o] + S.b3[o];
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (!ok && tid == 0) atomicExch(&g_mlp_error, 1);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
}

// features in slot order (e = field / E_SCALE): e_i in the atom's frame (3), the short-range
// first-order induced field e1_i in the same frame (3), e at the z- and x-atoms in i's frame
// (3 + 3), |e_i|, |e1_i|, alpha_i, frame kind (0 global, 0.5 Z-then-X, 1 bisector)
// C: the arithmetic type (FP32 in the mixed and fixed modes - the features are FP32 inputs
// of a BF16 network, and FP64 is slow on this part - FP64 in AP_FP64)
template <class C>
__global__ void k_features(const double *__restrict__ E, const double *__restrict__ E1, const double *__restrict__ rot,
                           const double *__restrict__ alpha, const int *__restrict__ frame_s, int n, int n_pad,
                           float *__restrict__ feat, int e1_fixed) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    C R[9];
    for (int k = 0; k < 9; ++k) R[k] = (C)rot[9 * s + k];
    auto loc = [&](const double *F, int slot, C *o, int fx) {
        const C e[3] = {(C)(acc_value(F, slot, fx) * (1.0 / MLP_E_SCALE)),
                        (C)(acc_value(F, (size_t)n_pad + slot, fx) * (1.0 / MLP_E_SCALE)),
                        (C)(acc_value(F, (size_t)2 * n_pad + slot, fx) * (1.0 / MLP_E_SCALE))};
        for (int b = 0; b < 3; ++b) o[b] = R[0 * 3 + b] * e[0] + R[1 * 3 + b] * e[1] + R[2 * 3 + b] * e[2];
    };
    C f[16];
    loc(E, s, f, 0);
    loc(E1, s, f + 3, e1_fixed);
    const int type = frame_s[3 * s];
    if (type != AP_FRAME_NONE) {
        loc(E, frame_s[3 * s + 1], f + 6, 0);
        loc(E, frame_s[3 * s + 2], f + 9, 0);
    } else {
        for (int k = 6; k < 12; ++k) f[k] = C(0);
    }
    f[12] = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    f[13] = sqrt(f[3] * f[3] + f[4] * f[4] + f[5] * f[5]);
    f[14] = (C)alpha[s];
    f[15] = type == AP_FRAME_BISECTOR ? C(1) : (type == AP_FRAME_Z_THEN_X ? C(0.5) : C(0));
    for (int k = 0; k < 16; ++k) feat[(size_t)s * 16 + k] = (float)f[k];
}

// p = alpha E (input of the short-range feature field)
template <class T>
__global__ void k_alpha_field(const double *__restrict__ E, const double *__restrict__ alpha, int n_pad,
                              typename V4<T>::type *__restrict__ p) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    typename V4<T>::type v;
    v.x = (T)(alpha[s] * E[s]);
    v.y = (T)(alpha[s] * E[n_pad + s]);
    v.z = (T)(alpha[s] * E[2 * n_pad + s]);
    v.w = (T)0;
    p[s] = v;
}

// mu0 = alpha E + s_out R y (slot order in, caller order out)
__global__ void k_guess_assemble(const double *__restrict__ E, const double *__restrict__ rot,
                                 const double *__restrict__ alpha, const float *__restrict__ y,
                                 const int *__restrict__ perm, int n, int n_pad, double *__restrict__ mu0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double *R = rot + 9 * s;
    const double yy[3] = {y[3 * s], y[3 * s + 1], y[3 * s + 2]};
    const int i = perm[s];
    for (int a = 0; a < 3; ++a)
        mu0[3 * i + a] = alpha[s] * E[a * n_pad + s] +
                         MLP_OUT_SCALE * (R[3 * a] * yy[0] + R[3 * a + 1] * yy[1] + R[3 * a + 2] * yy[2]);
}

// caller-order features and targets t = R^T (mu - alpha E) / s_out
__global__ void k_features_out(const float *__restrict__ fs, const double *__restrict__ E,
                               const double *__restrict__ rot, const double *__restrict__ alpha,
                               const int *__restrict__ perm, const double *__restrict__ mu, int n, int n_pad,
                               float *__restrict__ feat, float *__restrict__ target) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm[s];
    for (int k = 0; k < 16; ++k) feat[(size_t)i * 16 + k] = fs[(size_t)s * 16 + k];
    if (target && mu) {
        const double *R = rot + 9 * s;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = mu[3 * i + a] - alpha[s] * E[a * n_pad + s];
        for (int b = 0; b < 3; ++b)
            target[3 * i + b] = (float)((R[b] * d[0] + R[3 + b] * d[1] + R[6 + b] * d[2]) / MLP_OUT_SCALE);
    }
}

// ---------------------------------------------------------------------------------------
// Training: forward, loss L = (1/2B) sum |y - t|^2 and the backward pass on the tensor cores.
// Per tile of 128 atoms (M = 128, one thread per atom row for the epilogues):
//   Z1 = X W1 + b1, H1 = relu; Z2 = H1 W2 + b2, H2 = relu; Y = H2 W3 + b3; dY = (Y - T)/B
//   dW3 += H2^T dY      (A = H2 read MN-major, B = dY MN-major)
//   dH2 = dY W3^T       (B = W3^T bytes read MN-major)      dZ2 = dH2 (H2 > 0)
//   dW2 += H1^T dZ2, db2 += dZ2^T 1, dH1 = dZ2 W2^T          dZ1 = dH1 (H1 > 0)
//   dW1^T += dZ1^T X, db1 += dZ1^T 1
// The gradient accumulators stay in tensor memory across the CTA's tiles and are added to
// the global FP32 gradient once per CTA. A 32 KB guard follows the operand buffers.
struct __align__(16) TrainSmem {
    unsigned char w1[4096], w2[32768], w3[4096];
    unsigned char x[4096], h1[32768], h2[32768], dy[4096], dz2[32768], dz1[32768], ones[4096];
    float b1[MLP_H], b2[MLP_H], b3[MLP_OUTP];
    uint64_t mbar;
    uint32_t taddr;
    float red[8];
    unsigned char guard[32768];
};

// TMEM columns
#define TM_H 0        // [0,128): hidden pre-activations / dH
#define TM_Y 128      // output (16)
#define TM_DW3 160    // dW3 [h][o] (16)
#define TM_DB2 192    // db2 in column 0 (16)
#define TM_DW1 224    // dW1^T [a][f] (16)
#define TM_DB1 256    // db1 in column 0 (16)
#define TM_DW2 384    // dW2 [a][h] (128)

__device__ __forceinline__ void relu_mask_bf16(uint32_t trow, const unsigned char *hsrc, unsigned char *dst, int row) {
    // dst = bf16( tmem_row * (h > 0) ), h read from hsrc (same layout, bf16)
#pragma unroll 1
    for (int c = 0; c < MLP_H; c += 32) {
        float v[32];
        tc::tmem_ld32(trow + c, v);
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
            const uint32_t off = tc::cm_offset(row, c + g, MLP_H);
            __align__(16) __nv_bfloat16 hv[8], o[8];
            *(uint4 *)hv = *(const uint4 *)(hsrc + off);
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16(__bfloat162float(hv[e]) > 0.f ? v[g + e] : 0.f);
            *(uint4 *)(dst + off) = *(const uint4 *)o;
        }
    }
}

__global__ void __launch_bounds__(128) k_mlp_grad(const unsigned char *__restrict__ packed,
                                                  const float *__restrict__ feat, const float *__restrict__ target,
                                                  int n, float inv_b, float *__restrict__ grad, double *__restrict__ loss) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const uint4 *src = (const uint4 *)packed;
        uint4 *dw = (uint4 *)S.w1;
        for (int k = tid; k < (4096 + 32768 + 4096) / 16; k += 128) dw[k] = src[k];
        const float *bsrc = (const float *)(packed + MLP_B1_OFF);
        for (int k = tid; k < MLP_H; k += 128) {
            S.b1[k] = bsrc[k];
            S.b2[k] = bsrc[MLP_H + k];
        }
        if (tid < MLP_OUTP) S.b3[tid] = bsrc[2 * MLP_H + tid];
        // ones column (B operand [atom][16], column 0 = 1)
        __align__(16) __nv_bfloat16 o[8];
        for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16(e == 0 ? 1.f : 0.f);
        *(uint4 *)(S.ones + tc::cm_offset(tid, 0, 16)) = *(const uint4 *)o;
        for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16(0.f);
        *(uint4 *)(S.ones + tc::cm_offset(tid, 8, 16)) = *(const uint4 *)o;
    }
    if (warp == 0) tc::tmem_alloc(&S.taddr, 512);
    if (tid == 0) tc::mbar_init(&S.mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tb = S.taddr;
    const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
    const uint32_t sx = tc::smem_u32(S.x), sh1 = tc::smem_u32(S.h1), sh2 = tc::smem_u32(S.h2),
                   sdy = tc::smem_u32(S.dy), sdz2 = tc::smem_u32(S.dz2), sdz1 = tc::smem_u32(S.dz1),
                   sones = tc::smem_u32(S.ones), sw1 = tc::smem_u32(S.w1), sw2 = tc::smem_u32(S.w2),
                   sw3 = tc::smem_u32(S.w3);
    constexpr uint32_t I_KK_128 = tc::idesc_bf16(128, 128, 0, 0);
    constexpr uint32_t I_KK_16 = tc::idesc_bf16(128, 16, 0, 0);
    constexpr uint32_t I_MM_16 = tc::idesc_bf16(128, 16, 1, 1);
    constexpr uint32_t I_MM_128 = tc::idesc_bf16(128, 128, 1, 1);
    constexpr uint32_t I_KM_128 = tc::idesc_bf16(128, 128, 0, 1);
    uint32_t phase = 0;
    bool ok = true;
    int first = 1;
    double my_loss = 0.0, db3[3] = {0.0, 0.0, 0.0};
    auto sync_mma = [&]() {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    };
    auto wait = [&]() {
        if (ok) ok = tc::mbar_wait(&S.mbar, phase);
        phase ^= 1;
        tc::fence_after();
    };
    const int ntiles = (n + 127) / 128;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int atom = tile * 128 + tid;
        const bool valid = atom < n;
        {
            __align__(16) __nv_bfloat16 h[16];
            for (int k = 0; k < 16; ++k) h[k] = __float2bfloat16(valid ? feat[(size_t)atom * 16 + k] : 0.f);
            *(uint4 *)(S.x + tc::cm_offset(tid, 0, 16)) = *(const uint4 *)&h[0];
            *(uint4 *)(S.x + tc::cm_offset(tid, 8, 16)) = *(const uint4 *)&h[8];
        }
        sync_mma();
        if (tid == 0) {
            tc::mma_bf16(tb + TM_H, tc::smem_desc(sx, 128, 256), tc::smem_desc(sw1, 128, 256), I_KK_128, 0);
            tc::commit(&S.mbar);
        }
        wait();
        if (ok) epilogue_relu(tb + lanebase + TM_H, S.b1, S.h1, tid);
        sync_mma();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < 8; ++kk)
                tc::mma_bf16(tb + TM_H, tc::smem_desc(sh1 + kk * 256, 128, 2048), tc::smem_desc(sw2 + kk * 256, 128, 2048),
                             I_KK_128, kk > 0);
            tc::commit(&S.mbar);
        }
        wait();
        if (ok) epilogue_relu(tb + lanebase + TM_H, S.b2, S.h2, tid);
        sync_mma();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < 8; ++kk)
                tc::mma_bf16(tb + TM_Y, tc::smem_desc(sh2 + kk * 256, 128, 2048), tc::smem_desc(sw3 + kk * 256, 128, 2048),
                             I_KK_16, kk > 0);
            tc::commit(&S.mbar);
        }
        wait();
        // loss and dY
        {
            float v[32];
            if (ok) tc::tmem_ld32(tb + lanebase + TM_Y, v);
            __align__(16) __nv_bfloat16 d[16];
            for (int k = 0; k < 16; ++k) d[k] = __float2bfloat16(0.f);
            if (valid && ok) {
                for (int o = 0; o < MLP_OUT; ++o) {
                    const float e = v[o] + S.b3[o] - target[(size_t)atom * MLP_OUT + o];
                    my_loss += 0.5 * (double)e * e * inv_b;
                    const float g = e * inv_b;
                    db3[o] += g;
                    d[o] = __float2bfloat16(g);
                }
            }
            *(uint4 *)(S.dy + tc::cm_offset(tid, 0, 16)) = *(const uint4 *)&d[0];
            *(uint4 *)(S.dy + tc::cm_offset(tid, 8, 16)) = *(const uint4 *)&d[8];
        }
        sync_mma();
        if (tid == 0 && ok) {
            // dW3 += H2^T dY
            for (int kk = 0; kk < 8; ++kk)
                tc::mma_bf16(tb + TM_DW3, tc::smem_desc(sh2 + kk * 4096, 2048, 128), tc::smem_desc(sdy + kk * 512, 256, 128),
                             I_MM_16, (kk > 0) || !first);
            // dH2 = dY W3^T
            tc::mma_bf16(tb + TM_H, tc::smem_desc(sdy, 128, 256), tc::smem_desc(sw3, 2048, 128), I_KM_128, 0);
            tc::commit(&S.mbar);
        }
        wait();
        if (ok) relu_mask_bf16(tb + lanebase + TM_H, S.h2, S.dz2, tid);
        sync_mma();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < 8; ++kk) {
                // dW2 += H1^T dZ2 ; db2 += dZ2^T 1
                tc::mma_bf16(tb + TM_DW2, tc::smem_desc(sh1 + kk * 4096, 2048, 128),
                             tc::smem_desc(sdz2 + kk * 4096, 2048, 128), I_MM_128, (kk > 0) || !first);
                tc::mma_bf16(tb + TM_DB2, tc::smem_desc(sdz2 + kk * 4096, 2048, 128), tc::smem_desc(sones + kk * 512, 256, 128),
                             I_MM_16, (kk > 0) || !first);
            }
            // dH1 = dZ2 W2^T (W2^T bytes read MN-major)
            for (int kk = 0; kk < 8; ++kk)
                tc::mma_bf16(tb + TM_H, tc::smem_desc(sdz2 + kk * 256, 128, 2048), tc::smem_desc(sw2 + kk * 4096, 2048, 128),
                             I_KM_128, kk > 0);
            tc::commit(&S.mbar);
        }
        wait();
        if (ok) relu_mask_bf16(tb + lanebase + TM_H, S.h1, S.dz1, tid);
        sync_mma();
        if (tid == 0 && ok) {
            for (int kk = 0; kk < 8; ++kk) {
                // dW1^T += dZ1^T X ; db1 += dZ1^T 1
                tc::mma_bf16(tb + TM_DW1, tc::smem_desc(sdz1 + kk * 4096, 2048, 128), tc::smem_desc(sx + kk * 512, 256, 128),
                             I_MM_16, (kk > 0) || !first);
                tc::mma_bf16(tb + TM_DB1, tc::smem_desc(sdz1 + kk * 4096, 2048, 128), tc::smem_desc(sones + kk * 512, 256, 128),
                             I_MM_16, (kk > 0) || !first);
            }
            tc::commit(&S.mbar);
        }
        wait();
        first = 0;
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    // accumulated gradients of this CTA -> global (thread = TMEM lane = row)
    if (ok && !first) {
        const int r = tid;
        float v[32];
        for (int c = 0; c < MLP_H; c += 32) {   // dW2[a = r][h]
            tc::tmem_ld32(tb + lanebase + TM_DW2 + c, v);
            for (int k = 0; k < 32; ++k) atomicAdd(&grad[MLP_P_W2 + r * MLP_H + c + k], v[k]);
        }
        tc::tmem_ld32(tb + lanebase + TM_DW3, v);   // dW3[h = r][o]
        for (int o = 0; o < MLP_OUT; ++o) atomicAdd(&grad[MLP_P_W3 + r * MLP_OUT + o], v[o]);
        tc::tmem_ld32(tb + lanebase + TM_DW1, v);   // dW1^T[a = r][f] -> W1[f][a]
        for (int f = 0; f < MLP_IN; ++f) atomicAdd(&grad[MLP_P_W1 + f * MLP_H + r], v[f]);
        tc::tmem_ld32(tb + lanebase + TM_DB2, v);
        atomicAdd(&grad[MLP_P_B2 + r], v[0]);
        tc::tmem_ld32(tb + lanebase + TM_DB1, v);
        atomicAdd(&grad[MLP_P_B1 + r], v[0]);
    }
    // loss and db3: block reduction
    for (int off = 16; off; off >>= 1) {
        my_loss += __shfl_xor_sync(0xffffffffu, my_loss, off);
        for (int o = 0; o < 3; ++o) db3[o] += __shfl_xor_sync(0xffffffffu, db3[o], off);
    }
    if (lane == 0) {
        atomicAdd(loss, my_loss);
        for (int o = 0; o < 3; ++o) atomicAdd(&grad[MLP_P_B3 + o], (float)db3[o]);
    }
    if (!ok && tid == 0) atomicExch(&g_mlp_error, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; clears the gradient
__global__ void k_adam(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int np, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    g[k] = 0.f;
}

int features_slots(ap_ctx *ctx) {
    const int n = ctx->n;
    cudaStream_t st = ctx->s0;
    if (ctx->prec == AP_FP64)
        k_alpha_field<double><<<ap_grid_for(ctx->n_pad, 256), 256, 0, st>>>(ctx->E, ctx->alpha, ctx->n_pad, (dvec4 *)ctx->p);
    else
        k_alpha_field<float><<<ap_grid_for(ctx->n_pad, 256), 256, 0, st>>>(ctx->E, ctx->alpha, ctx->n_pad, (float4 *)ctx->p);
    AP_CUDA(cudaMemsetAsync(ctx->e1s, 0, sizeof(double) * 3 * ctx->n_pad, st));
    int r = short_matvec_launch(ctx, ctx->p, ctx->e1s, st);
    if (r) return r;
    if (ctx->prec == AP_FP64)
        k_features<double><<<ap_grid_for(n, 128), 128, 0, st>>>(ctx->E, ctx->e1s, ctx->rot, ctx->alpha, ctx->frame_s, n,
                                                                ctx->n_pad, ctx->mlp_feat, ctx->fixed);
    else
        k_features<float><<<ap_grid_for(n, 128), 128, 0, st>>>(ctx->E, ctx->e1s, ctx->rot, ctx->alpha, ctx->frame_s, n,
                                                               ctx->n_pad, ctx->mlp_feat, ctx->fixed);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int forward_launch(const void *packed, const float *feat, int n, float *y, cudaStream_t s) {
    static bool attr = false;
    const size_t bytes = sizeof(FwdSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp smem: ") + cudaGetErrorString(e));
        attr = true;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (n + 127) / 128;
    const int grid = std::max(1, std::min(ntiles, 2 * sms));
    k_mlp_forward<<<grid, 128, bytes, s>>>((const unsigned char *)packed, feat, n, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp forward: ") + cudaGetErrorString(e));
    return AP_OK;
}

}  // namespace

extern "C" {

int ap_mlp_param_count(void) { return MLP_NPARAM; }
int ap_mlp_packed_bytes(void) { return MLP_PACKED_BYTES; }

int ap_mlp_pack(const float *d_params, void *d_packed, void *stream) {
    if (!d_params || !d_packed) return ap_fail(nullptr, AP_ERR_ARG, "null pointer");
    k_mlp_pack<<<(MLP_H * MLP_H + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, (unsigned char *)d_packed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp pack: ") + cudaGetErrorString(e));
    return AP_OK;
}

int ap_mlp_forward(const void *d_packed, const float *d_feat, int n, float *d_y, void *stream) {
    if (!d_packed || !d_feat || !d_y || n <= 0) return ap_fail(nullptr, AP_ERR_ARG, "bad arguments");
    return forward_launch(d_packed, d_feat, n, d_y, (cudaStream_t)stream);
}

int ap_mlp_train_step(float *d_params, float *d_grad, float *d_m, float *d_v, int step, float lr,
                      const float *d_feat, const float *d_target, int n, double *d_loss, void *d_packed, void *stream) {
    if (!d_params || !d_grad || !d_m || !d_v || !d_feat || !d_target || !d_loss || !d_packed || n <= 0 || step < 1)
        return ap_fail(nullptr, AP_ERR_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    static bool attr = false;
    const size_t bytes = sizeof(TrainSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp train smem: ") + cudaGetErrorString(e));
        attr = true;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // gradient of the current parameters (d_packed must hold them, see ap_mlp_pack)
    const int ntiles = (n + 127) / 128;
    k_mlp_grad<<<std::max(1, std::min(ntiles, sms)), 128, bytes, s>>>((const unsigned char *)d_packed, d_feat, d_target,
                                                                     n, 1.0f / n, d_grad, d_loss);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(d_params, d_grad, d_m, d_v, MLP_NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    k_mlp_pack<<<(MLP_H * MLP_H + 255) / 256, 256, 0, s>>>(d_params, (unsigned char *)d_packed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp train: ") + cudaGetErrorString(e));
    return AP_OK;
}

int ap_mlp_gradient(const void *d_packed, const float *d_feat, const float *d_target, int n, float *d_grad,
                    double *d_loss, void *stream) {
    if (!d_packed || !d_feat || !d_target || !d_grad || !d_loss || n <= 0) return ap_fail(nullptr, AP_ERR_ARG, "bad arguments");
    static bool attr = false;
    const size_t bytes = sizeof(TrainSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp train smem: ") + cudaGetErrorString(e));
        attr = true;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (n + 127) / 128;
    k_mlp_grad<<<std::max(1, std::min(ntiles, sms)), 128, bytes, (cudaStream_t)stream>>>(
        (const unsigned char *)d_packed, d_feat, d_target, n, 1.0f / n, d_grad, d_loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("mlp gradient: ") + cudaGetErrorString(e));
    return AP_OK;
}

int ap_mlp_status(void) {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_mlp_error, sizeof(int)) != cudaSuccess) return AP_ERR_CUDA;
    if (v) {
        int z = 0;
        cudaMemcpyToSymbol(g_mlp_error, &z, sizeof(int));
        return AP_ERR_TIMEOUT;
    }
    return AP_OK;
}

int ap_mlp_features(ap_ctx *ctx, const double *d_mu, float *d_feat, float *d_target) {
    if (!ctx || !d_feat) return AP_ERR_ARG;
    ctx->err.clear();
    if (!ctx->config_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field() must come first");
    if (d_target && !d_mu) return ap_fail(ctx, AP_ERR_ARG, "targets need the dipoles");
    const int n = ctx->n;
    int r = features_slots(ctx);
    if (r) return r;
    k_features_out<<<ap_grid_for(n, 128), 128, 0, ctx->s0>>>(ctx->mlp_feat, ctx->E, ctx->rot, ctx->alpha, ctx->perm,
                                                            d_mu, n, ctx->n_pad, d_feat, d_target);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

int ap_learned_guess(ap_ctx *ctx, const void *d_packed, double *d_mu0) {
    if (!ctx || !d_packed || !d_mu0) return AP_ERR_ARG;
    ctx->err.clear();
    if (!ctx->config_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field() must come first");
    const int n = ctx->n;
    int r = features_slots(ctx);
    if (r) return r;
    r = forward_launch(d_packed, ctx->mlp_feat, n, ctx->mlp_y, ctx->s0);
    if (r) return ap_fail(ctx, r, ap_last_error(nullptr));
    k_guess_assemble<<<ap_grid_for(n, 128), 128, 0, ctx->s0>>>(ctx->E, ctx->rot, ctx->alpha, ctx->mlp_y, ctx->perm, n,
                                                              ctx->n_pad, d_mu0);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // extern "C"
