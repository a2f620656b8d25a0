// Mixed-radix (8, 4, 2) in-place FFTs over batches of columns held in shared
// memory, for power-of-two lengths, plus FP64 <-> FP32 conversions on the
// integer pipe.
//
// Forward transforms are decimation in frequency: natural order in,
// "digit-reversed" order out; inverse transforms are decimation in time from
// that order back to natural order.  The solver only needs to know which slot
// holds which frequency (digitrev), so no reordering pass is ever made.
//
// A DIF stage of radix R on blocks of size ns (m = ns / R) maps, for every
// j < m, the R inputs x_q = data[j + q m] to
//     y_r = w_ns^{j r} sum_q x_q w_R^{q r},   w_n = exp(-2 pi i / n),
// stored at data[j + r m]; the inverse stage undoes it (up to a factor R).
#pragma once
#include "common.cuh"

namespace ac {

// Stage plan of a length-2^logn transform with radices up to 2^MAXB: full
// stages of MAXB bits while at least MAXB bits remain, then one stage with
// the rest.  The time transforms use MAXB = 3 (radix 8), the spatial ones
// MAXB = 4 (radix 16).  Forward and inverse of one length must use the same plan.
template <int MAXB>
__host__ __device__ __forceinline__ int fft_nstages(int logn) { return (logn + MAXB - 1) / MAXB; }
template <int MAXB>
__host__ __device__ __forceinline__ int fft_stage_bits(int logn, int s) {
    const int full = logn / MAXB;
    return s < full ? MAXB : logn - MAXB * full;
}

// slot of frequency k after the forward transform (and input slot of the inverse)
template <int MAXB>
__host__ __device__ __forceinline__ int digitrev(int k, int logn) {
    int p = 0, used = 0;
    const int ns = fft_nstages<MAXB>(logn);
    for (int s = 0; s < ns; ++s) {
        const int b = fft_stage_bits<MAXB>(logn, s);
        used += b;
        p |= (k & ((1 << b) - 1)) << (logn - used);
        k >>= b;
    }
    return p;
}

// frequency held by slot p (inverse of digitrev)
template <int MAXB>
__host__ __device__ __forceinline__ int slot_freq(int p, int logn) {
    int k = 0, used = 0, shift = 0;
    const int ns = fft_nstages<MAXB>(logn);
    for (int s = 0; s < ns; ++s) {
        const int b = fft_stage_bits<MAXB>(logn, s);
        used += b;
        k |= ((p >> (logn - used)) & ((1 << b) - 1)) << shift;
        shift += b;
    }
    return k;
}

// cos(2 pi k / 16) for k < 16, as a literal of the working precision, used
// by the register DFTs (k is a compile-time constant after unrolling)
template <typename R>
__device__ __forceinline__ R cos16(int k) {
    switch (k & 15) {
        case 0: return (R)1.0;
        case 1: case 15: return (R)0.92387953251128675613;
        case 2: case 14: return (R)0.70710678118654752440;
        case 3: case 13: return (R)0.38268343236508977173;
        case 4: case 12: return (R)0.0;
        case 5: case 11: return (R)-0.38268343236508977173;
        case 6: case 10: return (R)-0.70710678118654752440;
        case 7: case 9: return (R)-0.92387953251128675613;
        default: return (R)-1.0;
    }
}

template <typename C, bool INV>
__device__ __forceinline__ C rot(C a, int k, int n) {
    // a * exp(-+2 pi i k / n), n in {2, 4, 8, 16}.  Rotations by -1 and -+i
    // are exact swaps and negations: without fast-math the compiler keeps
    // multiplications by 0.0 and 1.0, which would cost real FMAs.
    typedef decltype(a.x) R;
    const int kk = (k * (16 / n)) & 15;
    if (kk == 0) return a;
    if (kk == 8) return cmake(-a.x, -a.y);
    if (kk == 4 || kk == 12) {
        // exp(-i pi/2) = -i (forward, kk = 4); the other three cases by symmetry
        const bool minus_i = (kk == 4) != INV;
        return minus_i ? cmake(a.y, -a.x) : cmake(-a.y, a.x);
    }
    const R c = cos16<R>(kk);
    const R s = INV ? cos16<R>(kk + 12) : -cos16<R>(kk + 12);   // -+ sin(2 pi kk / 16)
    C r;
    r.x = a.x * c - a.y * s;
    r.y = a.x * s + a.y * c;
    return r;
}

// Complex add, subtract and multiply for the transforms.  In FP64 they are
// written as FMAs whose operands are all registers (one = 1.0, zero = 0.0
// loaded at run time): on this GPU such DFMAs issue about 16% faster than
// DADD and DMUL, and a * 1 + b, a * b + 0 round exactly like a + b, a * b.
// In FP32 the plain operations run at full rate.
template <typename C, typename R>
__device__ __forceinline__ C xadd(C a, C b, R one) {
    if constexpr (sizeof(R) == 8) return cmake(fma(a.x, one, b.x), fma(a.y, one, b.y));
    else return cadd(a, b);
}
template <typename C, typename R>
__device__ __forceinline__ C xsub(C a, C b, R one) {
    if constexpr (sizeof(R) == 8) return cmake(fma(-b.x, one, a.x), fma(-b.y, one, a.y));
    else return csub(a, b);
}
// a * b, or a * conj(b) (CONJ)
template <bool CONJ, typename C, typename R>
__device__ __forceinline__ C xmul(C a, C b, R zero) {
    if constexpr (sizeof(R) == 8) {
        const R by = CONJ ? -b.y : b.y;
        C r;
        r.x = fma(a.x, b.x, fma(-a.y, by, zero));
        r.y = fma(a.x, by, fma(a.y, b.x, zero));
        return r;
    } else {
        return CONJ ? cmulc(a, b) : cmul(a, b);
    }
}

// In-register R-point DFT (forward: y_r = sum_q x_q w_R^{qr}; INV: conjugate),
// natural order in and out.  one: a register holding 1.0 (see xadd).
template <int R, bool INV, typename C, typename RR>
__device__ __forceinline__ void small_dft(C* v, RR one) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int j0 = 0; j0 < R; j0 += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                C a = v[j0 + k], b = v[j0 + k + h];
                v[j0 + k] = xadd(a, b, one);
                v[j0 + k + h] = rot<C, INV>(xsub(a, b, one), k, 2 * h);
            }
        }
    }
    // undo the bit reversal of the radix-2 cascade
    C t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 1, x = i; b < R; b <<= 1, x >>= 1) r = (r << 1) | (x & 1);
        t[i] = v[r];
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// One stage over all batches.  Element (j, b, mm) lives at
// data[j * js + b * bs + mm * ms]; b < 2^logb; mm < MI is looped per thread.
// BFAST: consecutive threads take consecutive b (else consecutive j).
template <typename C, int R, int MI, bool INV, bool BFAST, bool UNIT>
__device__ __forceinline__ void fft_stage(C* data, int logn, int logns, int logb, int js, int bs, int ms,
                                          const C* __restrict__ tw) {
    constexpr int logR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    const int logm = logns - logR;
    const int m = 1 << logm;
    const int logitems_b = logn - logR;  // items per batch
    const int total = 1 << (logitems_b + logb);
    const int twshift = logn - logns;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int b, i;
        if (BFAST) {
            b = t & ((1 << logb) - 1);
            i = t >> logb;
        } else {
            i = t & ((1 << logitems_b) - 1);
            b = t >> logitems_b;
        }
        const int j = i & (m - 1);
        const int base = ((i >> logm) << logns) + j;
        C w[R];
        if (!UNIT) {
#pragma unroll
            for (int r = 1; r < R; ++r) w[r] = tw[(j * r) << twshift];
        }
        // tw[0] = 1 - 0i: register copies of 1 and 0 for the FP64 FMA forms
        const C w0 = tw[0];
        const auto one = w0.x;
        const auto zero = w0.y;
        // shared-memory offsets fit in 32 bits
        C* p = data + (base * js + b * bs);
        const int mjs = m * js;
#pragma unroll
        for (int mm = 0; mm < MI; ++mm) {
            C v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = p[r * mjs + mm * ms];
            if (!INV) {
                small_dft<R, false>(v, one);
                if (!UNIT) {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[r] = xmul<false>(v[r], w[r], zero);
                }
            } else {
                if (!UNIT) {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[r] = xmul<true>(v[r], w[r], zero);
                }
                small_dft<R, true>(v, one);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) p[r * mjs + mm * ms] = v[r];
        }
    }
    __syncthreads();
}

// radix dispatch; only radices up to 2^MAXB are instantiated (a radix-16
// stage that is never taken would still raise the kernel's register count)
template <typename C, int MI, bool INV, bool BFAST, bool UNIT, int MAXB>
__device__ __forceinline__ void fft_stage_r(int bits, C* data, int logn, int logns, int logb, int js, int bs, int ms,
                                            const C* __restrict__ tw) {
    if (MAXB >= 4 && bits == 4)
        fft_stage<C, (MAXB >= 4 ? 16 : 8), MI, INV, BFAST, UNIT>(data, logn, logns, logb, js, bs, ms, tw);
    else if (bits == 3) fft_stage<C, 8, MI, INV, BFAST, UNIT>(data, logn, logns, logb, js, bs, ms, tw);
    else if (bits == 2) fft_stage<C, 4, MI, INV, BFAST, UNIT>(data, logn, logns, logb, js, bs, ms, tw);
    else fft_stage<C, 2, MI, INV, BFAST, UNIT>(data, logn, logns, logb, js, bs, ms, tw);
}

// Forward transform of length 2^logn (tw: 2^logn entries w_n^k), radices up
// to 2^MAXB.  Ends with __syncthreads(); callers must synchronise before it.
// The last stage has unit twiddles (its blocks have one column).
template <typename C, int MI, bool BFAST, int MAXB = 3>
__device__ void fft_fwd(C* data, int logn, int logb, int js, int bs, int ms, const C* __restrict__ tw) {
    const int ns = fft_nstages<MAXB>(logn);
    int logns = logn;
    for (int s = 0; s < ns; ++s) {
        const int bits = fft_stage_bits<MAXB>(logn, s);
        if (s == ns - 1) fft_stage_r<C, MI, false, BFAST, true, MAXB>(bits, data, logn, logns, logb, js, bs, ms, tw);
        else fft_stage_r<C, MI, false, BFAST, false, MAXB>(bits, data, logn, logns, logb, js, bs, ms, tw);
        logns -= bits;
    }
}

// Inverse (unnormalised) transform: digit-reversed order in, natural out.
template <typename C, int MI, bool BFAST, int MAXB = 3>
__device__ void fft_inv(C* data, int logn, int logb, int js, int bs, int ms, const C* __restrict__ tw) {
    const int ns = fft_nstages<MAXB>(logn);
    for (int s = ns - 1; s >= 0; --s) {
        const int bits = fft_stage_bits<MAXB>(logn, s);
        const int logns = logn - MAXB * s;   // block size entering DIF stage s (all earlier stages are full)
        if (s == ns - 1) fft_stage_r<C, MI, true, BFAST, true, MAXB>(bits, data, logn, logns, logb, js, bs, ms, tw);
        else fft_stage_r<C, MI, true, BFAST, false, MAXB>(bits, data, logn, logns, logb, js, bs, ms, tw);
    }
}

// The last forward stage, a per-slot operation and the first inverse stage
// in one pass: both stages work on blocks of 2^bits consecutive slots with
// unit twiddles, so each thread transforms its block, replaces every output
// v (slot `slot` of batch b) by op(v, slot, b) and transforms the block back.
template <typename C, int R, bool BFAST, typename Op>
__device__ __forceinline__ void fft_last_op_first(C* data, int logn, int logb, int js, int bs,
                                                  const C* __restrict__ tw, Op op) {
    constexpr int logR = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
    const int logitems_b = logn - logR;
    const int total = 1 << (logitems_b + logb);
    const auto one = tw[0].x;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int b, i;
        if (BFAST) {
            b = t & ((1 << logb) - 1);
            i = t >> logb;
        } else {
            i = t & ((1 << logitems_b) - 1);
            b = t >> logitems_b;
        }
        const int base = i << logR;
        C* p = data + (base * js + b * bs);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * js];
        small_dft<R, false>(v, one);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = op(v[r], base + r, b);
        small_dft<R, true>(v, one);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * js] = v[r];
    }
    __syncthreads();
}

// Forward transform, op on every slot of the spectrum (digit-reversed order,
// see digitrev), inverse transform (not normalised): fft_fwd, a pass of op
// and fft_inv with the two middle stages fused.  Ends with __syncthreads();
// callers must synchronise before it.
template <typename C, bool BFAST, int MAXB, typename Op>
__device__ void fft_fwd_op_inv(C* data, int logn, int logb, int js, int bs, const C* __restrict__ tw, Op op) {
    const int ns = fft_nstages<MAXB>(logn);
    int logns = logn;
    for (int s = 0; s < ns - 1; ++s) {
        const int bits = fft_stage_bits<MAXB>(logn, s);
        fft_stage_r<C, 1, false, BFAST, false, MAXB>(bits, data, logn, logns, logb, js, bs, 0, tw);
        logns -= bits;
    }
    const int lb = fft_stage_bits<MAXB>(logn, ns - 1);
    if (MAXB >= 4 && lb == 4) fft_last_op_first<C, (MAXB >= 4 ? 16 : 8), BFAST>(data, logn, logb, js, bs, tw, op);
    else if (lb == 3) fft_last_op_first<C, 8, BFAST>(data, logn, logb, js, bs, tw, op);
    else if (lb == 2) fft_last_op_first<C, 4, BFAST>(data, logn, logb, js, bs, tw, op);
    else fft_last_op_first<C, 2, BFAST>(data, logn, logb, js, bs, tw, op);
    for (int s = ns - 2; s >= 0; --s) {
        const int bits = fft_stage_bits<MAXB>(logn, s);
        fft_stage_r<C, 1, true, BFAST, false, MAXB>(bits, data, logn, logn - MAXB * s, logb, js, bs, 0, tw);
    }
}

// ---- FP64 <-> FP32 on the integer pipe (the FP64 pipe of this GPU is narrow)

// Round-to-nearest-even double -> float for the normal float range; values
// below it become signed zero, values above it infinity (NaN too).
__device__ __forceinline__ float d2f_int(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;
    const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned f = ((unsigned)e << 23) + mant;
    f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (mant & 1u));
    f = e <= 0 ? 0u : f;
    f = (e >= 255 || f >= 0x7F800000u) ? 0x7F800000u : f;
    return __uint_as_float(sign | f);
}

// Exact float -> double for normal floats (subnormal floats become zero).
__device__ __forceinline__ double f2d_int(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned sign = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned mant = b & 0x7FFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | (mant >> 3);
    unsigned lo = mant << 29;
    hi = e == 0 ? sign : hi;
    lo = e == 0 ? 0u : lo;
    hi = e == 255 ? (sign | 0x7FF00000u | (mant >> 3)) : hi;
    return __hiloint2double((int)hi, (int)lo);
}

template <typename R> __device__ __forceinline__ R to_real(double x);
template <> __device__ __forceinline__ float to_real<float>(double x) { return d2f_int(x); }
template <> __device__ __forceinline__ double to_real<double>(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_int(x); }
__device__ __forceinline__ double to_double(double x) { return x; }

// ---- shifted division of the spatial solves

// Reciprocal of a positive double: a float seed (FP32 reciprocal, converted
// on the integer pipe) and two Newton-Raphson steps y <- y + y (1 - x y),
// each of which doubles the number of correct bits (24 -> 48 -> full FP64).
// Valid for x in the normal float range, which the shifted symbols
// |1 - mu sigma|^2 of the solver stay in.
__device__ __forceinline__ double rcp_newton(double x, double one) {
    double y = f2d_int(__frcp_rn(d2f_int(x)));
    y = fma(y, fma(-x, y, one), y);
    y = fma(y, fma(-x, y, one), y);
    return y;
}
__device__ __forceinline__ float rcp_newton(float x, float) { return __frcp_rn(x); }

// v / den: multiply by conj(den) / |den|^2 (den = 1 - mu sigma, with
// |den| >= 1 whenever Re(mu sigma) <= 0; in any case far from 0 here).  In
// FP64 every product and sum is an FMA with register operands (zero: a
// register holding 0.0), as in the transforms.
template <typename C, typename R>
__device__ __forceinline__ C div_by(C v, C den, R one, R zero) {
    if constexpr (sizeof(R) == 8) {
        const R inv = rcp_newton(fma(den.x, den.x, fma(den.y, den.y, zero)), one);
        const R px = fma(v.x, den.x, fma(v.y, den.y, zero));    // v * conj(den)
        const R py = fma(v.y, den.x, fma(-v.x, den.y, zero));
        return cmake(fma(px, inv, zero), fma(py, inv, zero));
    } else {
        const R inv = rcp_newton(fma(den.x, den.x, den.y * den.y), one);
        return cscale(cmulc(v, den), inv);
    }
}
template <typename C, typename R>
__device__ __forceinline__ C div_one_minus(C v, C m, R one, R zero) {
    return div_by(v, xsub(cmake(one, zero), m, one), one, zero);
}

}  // namespace ac
