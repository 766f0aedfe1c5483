// FP32 vector kernels of the mixed and fixed-point solvers: dot products and norms with
// FP64-grade sums and no FP64 arithmetic per element. Each product is split exactly into its
// rounded value and its error (an fma), both summed in a compensated FP32 pair (F2, TwoSum)
// per thread and across the warp and block; the block's pair is converted exactly to FP64.
#pragma once
#include "pair_math.cuh"

// a += x y, the product carried exactly as its rounded value and rounding error
__device__ __forceinline__ void f2_add_prod(F2 &a, float x, float y) {
    const float p = x * y;
    f2_add(a, p);
    a.lo += fmaf(x, y, -p);
}

// block-wide sums of two compensated pairs; thread 0 gets them in FP64
// (every thread of the block calls it; its shared scratch is reused by the next call, so
// two calls in a row need a __syncthreads() between them)
template <int NT_>
__device__ __forceinline__ void block_sum2_f2(F2 a, F2 b, double &da, double &db) {
    __shared__ float sh[4][NT_ / 32];
    for (int off = 16; off; off >>= 1) {
        const float ah = __shfl_xor_sync(0xffffffffu, a.hi, off), al = __shfl_xor_sync(0xffffffffu, a.lo, off);
        const float bh = __shfl_xor_sync(0xffffffffu, b.hi, off), bl = __shfl_xor_sync(0xffffffffu, b.lo, off);
        f2_add(a, ah);
        a.lo += al;
        f2_add(b, bh);
        b.lo += bl;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[0][w] = a.hi;
        sh[1][w] = a.lo;
        sh[2][w] = b.hi;
        sh[3][w] = b.lo;
    }
    __syncthreads();
    if (w == 0) {
        F2 x, y;
        x.hi = l < NT_ / 32 ? sh[0][l] : 0.f;
        x.lo = l < NT_ / 32 ? sh[1][l] : 0.f;
        y.hi = l < NT_ / 32 ? sh[2][l] : 0.f;
        y.lo = l < NT_ / 32 ? sh[3][l] : 0.f;
        for (int off = 16; off; off >>= 1) {
            const float xh = __shfl_xor_sync(0xffffffffu, x.hi, off), xl = __shfl_xor_sync(0xffffffffu, x.lo, off);
            const float yh = __shfl_xor_sync(0xffffffffu, y.hi, off), yl = __shfl_xor_sync(0xffffffffu, y.lo, off);
            f2_add(x, xh);
            x.lo += xl;
            f2_add(y, yh);
            y.lo += yl;
        }
        da = f2d_exact(x.hi) + f2d_exact(x.lo);
        db = f2d_exact(y.hi) + f2d_exact(y.lo);
    }
}

// an accumulator slot of the real-space product in FP32 (FP64 or, fixed, 2^-34 fixed point:
// the integer's conversion and an exact power-of-two scale round once, as the FP64 path)
__device__ __forceinline__ float acc_f32(const double *acc, size_t k, int fixed) {
    return fixed ? (float)reinterpret_cast<const long long *>(acc)[k] * (1.0f / 17179869184.0f) : (float)acc[k];
}

