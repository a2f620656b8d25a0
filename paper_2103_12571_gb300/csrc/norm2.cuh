// Sums of squares of FP64 values, accurate to about 2^-44 relative, without
// FP64 arithmetic: each value x is split into two floats hi + lo with integer
// bit operations (|x - hi - lo| <= 2^-48 |x|), scaled by a two-float weight,
// squared with the exact product error (fmaf), and accumulated as an
// unevaluated float pair (s, c) with Knuth's two-sum.  The FP64 pipe of this
// GPU is narrow and busy in the residual kernel; these steps run on the FP32
// and integer pipes.  Block results are combined in FP64.
#pragma once
#ifdef __CUDACC__
#include "common.cuh"
#endif

namespace ac {

// Residual entries are scaled by this power of two before squaring, so that
// relative residuals between about 1e-25 and 1e13 (times ||w||_inf) stay in
// the normal float range for their squares.
constexpr double kNormPrescale = 1048576.0;   // 2^20

struct F2Acc {
    float s, c;   // value s + c
};

__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &x, 8);
    return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, 4);
    return f;
#endif
}

// x = hi + lo + O(2^-48 |x|): hi = x rounded to nearest float (normal range;
// zero below it, infinity above it), lo = the rounded remainder.  Values
// below 2^-74 in magnitude get lo = 0.
__host__ __device__ __forceinline__ void split_d2f(double x, float& hi, float& lo) {
    const unsigned long long b = bits_of(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sign = hw & 0x80000000u;
    const int E = (int)((hw >> 20) & 0x7FFu);          // biased FP64 exponent
    const int e = E - 896;                             // biased FP32 exponent
    const unsigned mant = ((hw & 0xFFFFFu) << 3) | (lw >> 29);   // top 23 mantissa bits
    const unsigned rest = lw & 0x1FFFFFFFu;            // low 29 mantissa bits
    const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (mant & 1u));
    unsigned f = ((unsigned)e << 23) + mant + up;
    f = e <= 0 ? 0u : f;
    f = (e >= 255 || f >= 0x7F800000u) ? 0x7F800000u : f;
    hi = float_of(sign | f);
    // x - hi = (rest - up * 2^29) * 2^(E - 1075)
    const int rem = (int)rest - (int)(up << 29);
    const int pe = E - 948;                            // biased FP32 exponent of 2^(E - 1075)
    const float pw = float_of(pe >= 1 && pe <= 254 ? ((unsigned)pe << 23) : 0u);
    const float l = (float)rem * pw;
    lo = sign ? -l : l;
}

// Two-float weight w = wh + wl of a double (host side).
inline void split_weight(double w, float& wh, float& wl) {
    wh = (float)w;
    wl = (float)(w - (double)wh);
}

// acc += ((hi + lo) (wh + wl))^2
__host__ __device__ __forceinline__ void f2_add_sq(F2Acc& acc, float hi, float lo, float wh, float wl) {
    const float p = hi * wh;
    const float pe = fmaf(hi, wh, -p);                 // exact error of hi * wh
    const float q = fmaf(hi, wl, fmaf(lo, wh, pe));    // y = p + q
    const float s = p * p;
    const float se = fmaf(p, p, -s);                   // exact error of p * p
    const float t = fmaf(2.0f * p, q, se);             // y^2 = s + t (+ q^2, below 2^-46 of s)
    const float S = acc.s + s;                         // two-sum of acc.s and s
    const float bb = S - acc.s;
    const float err = (acc.s - (S - bb)) + (s - bb);
    const float c = acc.c + (err + t);
    acc.s = S + c;                                     // renormalise: |acc.c| <= ulp(acc.s)
    acc.c = c - (acc.s - S);
}

// a += b for float pairs
__host__ __device__ __forceinline__ void f2_add(F2Acc& a, F2Acc b) {
    const float S = a.s + b.s;
    const float bb = S - a.s;
    const float err = (a.s - (S - bb)) + (b.s - bb);
    const float c = a.c + (b.c + err);
    a.s = S + c;
    a.c = c - (a.s - S);
}

#ifdef __CUDACC__
// Block-wide sum of float pairs, returned as a double in thread 0 (red: 32
// doubles of shared memory).
__device__ __forceinline__ double block_sum_f2(F2Acc v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        F2Acc w;
        w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
        f2_add(v, w);
    }
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[wp] = (double)v.s + (double)v.c;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) tot += red[i];
    }
    return tot;
}

// Block-wide maximum of non-negative doubles given as bit patterns (for
// x >= 0 the IEEE order is the unsigned integer order; NaN sorts above
// infinity and so propagates).  Result valid in thread 0.
__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[wp] = v;
    __syncthreads();
    unsigned long long m = 0ull;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) m = red[i] > m ? red[i] : m;
    }
    return m;
}
#endif

}  // namespace ac
