// Device helpers shared by the solver kernels: complex arithmetic on
// float2/double2 and batched radix-2 FFTs in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ac {

template <typename R> struct Cx;
template <> struct Cx<float> { typedef float2 T; };
template <> struct Cx<double> { typedef double2 T; };

__device__ __forceinline__ float2 cmake(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
// acc += a * b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
template <typename C> __device__ __forceinline__ C cdiv(C a, C b) {
    // a / b with scaling by the larger component of b
    typedef decltype(a.x) R;
    R s = fabs(b.x) > fabs(b.y) ? fabs(b.x) : fabs(b.y);
    R bx = b.x / s, by = b.y / s;
    R den = bx * bx + by * by;
    C r;
    r.x = (a.x * bx + a.y * by) / (den * s);
    r.y = (a.y * bx - a.x * by) / (den * s);
    return r;
}

__device__ __forceinline__ int bitrev(int i, int logn) {
    return logn == 0 ? 0 : (int)(__brev((unsigned)i) >> (32 - logn));
}

// Batched radix-2 decimation-in-frequency FFT in shared memory, forward sign
// (X_k = sum_j x_j exp(-2 pi i j k / n)): natural order in, bit-reversed order
// out.  Element (j, b) of batch b lives at data[j * js + b * bs].  tw[k] =
// exp(-2 pi i k / n), k < n/2.  All threads of the block call this; it ends
// with __syncthreads().  BFAST: consecutive threads take consecutive batches
// (use when bs == 1), else consecutive butterflies of one batch.
template <typename C, bool BFAST>
__device__ void fft_dif(C* data, int logn, int nbatch, int logbatch_or_neg, int js, int bs,
                        const C* __restrict__ tw) {
    const int n = 1 << logn;
    const int half = n >> 1;
    const long total = (long)nbatch * half;
    for (int s = 0; s < logn; ++s) {
        const int logh = logn - 1 - s;
        const int h = 1 << logh;
        for (long t = threadIdx.x; t < total; t += blockDim.x) {
            int b, i;
            if (BFAST) {
                if (logbatch_or_neg >= 0) { b = (int)(t & (nbatch - 1)); i = (int)(t >> logbatch_or_neg); }
                else { i = (int)(t / nbatch); b = (int)(t - (long)i * nbatch); }
            } else {
                b = (int)(t >> (logn - 1));
                i = (int)(t & (half - 1));
            }
            const int k = i & (h - 1);
            const int j0 = ((i >> logh) << (logh + 1)) + k;
            C* p0 = data + (long)j0 * js + (long)b * bs;
            C* p1 = p0 + (long)h * js;
            C x0 = *p0, x1 = *p1;
            *p0 = cadd(x0, x1);
            *p1 = cmul(csub(x0, x1), tw[k << s]);
        }
        __syncthreads();
    }
}

// Inverse companion: radix-2 decimation-in-time FFT with the conjugate
// twiddles (backward sign, unnormalised), bit-reversed order in, natural
// order out.
template <typename C, bool BFAST>
__device__ void fft_dit_inv(C* data, int logn, int nbatch, int logbatch_or_neg, int js, int bs,
                            const C* __restrict__ tw) {
    const int n = 1 << logn;
    const int half = n >> 1;
    const long total = (long)nbatch * half;
    for (int s = 0; s < logn; ++s) {
        const int logh = s;
        const int h = 1 << logh;
        for (long t = threadIdx.x; t < total; t += blockDim.x) {
            int b, i;
            if (BFAST) {
                if (logbatch_or_neg >= 0) { b = (int)(t & (nbatch - 1)); i = (int)(t >> logbatch_or_neg); }
                else { i = (int)(t / nbatch); b = (int)(t - (long)i * nbatch); }
            } else {
                b = (int)(t >> (logn - 1));
                i = (int)(t & (half - 1));
            }
            const int k = i & (h - 1);
            const int j0 = ((i >> logh) << (logh + 1)) + k;
            C* p0 = data + (long)j0 * js + (long)b * bs;
            C* p1 = p0 + (long)h * js;
            C x0 = *p0;
            C x1 = cmulc(*p1, tw[k << (logn - 1 - s)]);
            *p0 = cadd(x0, x1);
            *p1 = csub(x0, x1);
        }
        __syncthreads();
    }
}

// Block-wide sum of a float (result valid in thread 0).
__device__ __forceinline__ float block_sum(float v, float* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    v = 0.f;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? scratch[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}
__device__ __forceinline__ float block_max(float v, float* scratch) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    v = 0.f;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? scratch[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}
__device__ __forceinline__ double block_sum_d(double v, double* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? scratch[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

}  // namespace ac
