#pragma once
// Time-direction kernels of one Richardson iteration (templates; the
// explicit instantiations live in k_fwd_f32.cu, k_fwd_f64.cu and k_upd.cu,
// compiled in parallel).
//
// k_fwd: step (i) FP64 residual r = w - C u of eq. (globalsys), step (ii) the
//   alpha-scaling J^{-1} and the length-L FFT along time of eq. (s1)
//   (Algorithm 1, the steps computing r~ and x), and the node mixing
//   x^1 = S_l^{-1} x of eq. (d1).  One CTA owns P grid points and all L*M
//   values at each of them; the residual is written into shared memory in
//   the transform precision, the FFT runs there (mixed radix 8/4/2, DIF,
//   digit-reversed output, which the per-frequency work does not care
//   about), and only the
//   F = L/2 + 1 non-redundant frequencies of the real data are stored.
//   Two real columns are transformed as one complex column.
// k_upd: eq. (d3) and (Gsubstitution) as one mix y = P_l x^2 with
//   P_l = G_l^{-1} S_l, the inverse FFT along time of eq. (s3) (DIT from
//   digit-reversed order), the un-scaling by J, and the FP64 update
//   u += e of the correction form of eq. (Riteration).
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "norm2.cuh"
#include "tma.cuh"

namespace ac {



// Register copies of the stencil taps and a zero: on this GPU an FP64 FMA
// whose operands all come from registers issues at the full FP64 rate, while
// DMUL, DADD and FMAs with a constant-bank or immediate operand run about 16%
// slower, so every multiply below is an FMA on registers.
struct RegCoef {
    double tx[7], ty[7], c0, zero;
};

// Right-hand-side-only rows (no stencil): the scaled w_l = s_l (u0 in block 1
// plus b_l) when no iterate is given, or, for the recompute form of
// eq. (Riteration), w + (C_alpha - C) u, where (C_alpha - C) u = -alpha (H u_L)
// in block 1 (H^T u_L for the adjoint).  This is its own kernel variant
// (RAD = 0): a runtime branch here would be predicated into the stencil
// variants, and predicated-off FP64 instructions still occupy the FP64 pipe.
template <int MM>
__device__ __forceinline__ void source_point(const FwdArgs& a, const RegCoef& k, int l, long n, double r[MM]) {
    const long N = a.g.N;
    const double s = a.s[l];
    const int lb = a.b_reversed ? (a.L - 1 - l) : l;
#pragma unroll
    for (int m = 0; m < MM; ++m) {
        double w = (l == 0 && a.u0) ? a.u0[n] : 0.0;
        if (a.b) w += a.b[((long)lb * MM + m) * N + n];
        r[m] = w;
    }
    if (a.recompute && a.u && l == 0) {
        const double* uL = a.u + (long)(a.L - 1) * MM * N + n;
        if (!a.transposed) {
            const double c = -a.alpha * uL[(long)(MM - 1) * N];
#pragma unroll
            for (int m = 0; m < MM; ++m) r[m] += c;
        } else {
            double c = 0.0;
#pragma unroll
            for (int j = 0; j < MM; ++j) c += uL[(long)j * N];
            r[MM - 1] += -a.alpha * c;
        }
    }
#pragma unroll
    for (int m = 0; m < MM; ++m) r[m] = fma(s, r[m], k.zero);
}

// Full residual rows r_l = w_l - (C u)_l.  RAD (stencil radius) and DIM are
// compile-time: FP64 instructions that a runtime test predicates off still
// occupy the FP64 pipe of this GPU.  For the same reason GEN = false is the
// plain forward operator without a forcing term b (no runtime tests of
// a.transposed or a.b); GEN = true reads both at run time (adjoint, forcing).
template <int MM, int RAD, int DIM, bool GEN>
__device__ __forceinline__ void residual_point(const FwdArgs& a, const RegCoef& k, int l, long n, const int* dxo,
                                               const int* dyo, double r[MM]) {
    if (RAD == 0) {
        source_point<MM>(a, k, l, n, r);
        return;
    }
    const Grid& g = a.g;
    const long N = g.N;
    const double s = a.s[l];
    const int lb = a.b_reversed ? (a.L - 1 - l) : l;
    const double* ub = a.u + (long)l * MM * N + n;
    double uc[MM], Au[MM];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
        const double* uj = ub + (long)j * N;
        uc[j] = uj[0];
        double acc = fma(k.c0, uc[j], k.zero);   // combined centre tap of both axes
#pragma unroll
        for (int o = 0; o < 2 * RAD; ++o) {   // offsets -1, +1, -2, +2, -3, +3
            acc = fma(k.tx[stencil_tap(o)], uj[dxo[o]], acc);
            if (DIM == 2) acc = fma(k.ty[stencil_tap(o)], uj[dyo[o]], acc);
        }
        Au[j] = acc;
    }
    const double* qs = a.qs + l * MM * MM;
    double sp[MM];
    if (!GEN || !a.transposed) {
        double c = 0.0;
        if (l > 0) c = ub[-(long)N];                     // u_{l-1, M} (block l-1, last node)
        if (l == 0 && a.u0) c += a.u0[n];
        const double sc = fma(s, c, k.zero);
#pragma unroll
        for (int m = 0; m < MM; ++m) sp[m] = sc;
    } else {
#pragma unroll
        for (int m = 0; m < MM; ++m) sp[m] = k.zero;
        if (l > 0) {
            double c = 0.0;
            const double* up = ub - (long)MM * N;
#pragma unroll
            for (int j = 0; j < MM; ++j) c += up[(long)j * N];  // (H^T u_{l-1})_M = sum_j u_{l-1,j}
            sp[MM - 1] = fma(s, c, k.zero);
        }
        if (l == 0 && a.u0) {
#pragma unroll
            for (int m = 0; m < MM; ++m) sp[m] += a.u0[n];
        }
    }
    if (GEN && a.b) {
#pragma unroll
        for (int m = 0; m < MM; ++m) sp[m] = fma(s, a.b[((long)lb * MM + m) * N + n], sp[m]);
    }
    const double ms = -s;
#pragma unroll
    for (int m = 0; m < MM; ++m) {
        double t = fma(ms, uc[m], sp[m]);
#pragma unroll
        for (int j = 0; j < MM; ++j) t = fma(qs[m * MM + j], Au[j], t);
        r[m] = t;
    }
}

template <typename R, int MM, int RAD, int DIM, bool GEN>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 3 : 0) k_fwd(FwdArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    R* Zr = reinterpret_cast<R*>(smem_raw);
    C* Z = reinterpret_cast<C*>(smem_raw);
    const int P = a.P, HP = P >> 1;
    const int logP = 31 - __clz(P);
    const int L = a.L;
    const long N = a.g.N;
    const long n0 = (long)(blockIdx.x + a.tile0) * P;

    __shared__ double coef_s[16];
    if (threadIdx.x < 16) {
        const int i = threadIdx.x;
        coef_s[i] = i < 7 ? a.g.tx[i] : (i < 14 ? a.g.ty[i - 7] : (i == 14 ? a.g.c0 : 0.0));
    }
    __syncthreads();
    RegCoef kc;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        kc.tx[i] = coef_s[i];
        kc.ty[i] = coef_s[7 + i];
    }
    kc.c0 = coef_s[14];
    kc.zero = coef_s[15];

    // this thread's grid point is fixed (blockDim is a multiple of P)
    const int p = threadIdx.x & (P - 1);
    const long n = n0 + p;
    int dxo[6] = {0, 0, 0, 0, 0, 0}, dyo[6] = {0, 0, 0, 0, 0, 0};
    if (n < N) {
        const int nx = a.g.nx;
        const long iy = n / nx;
        const int ix = (int)(n - iy * nx);
#pragma unroll
        for (int o = 0; o < 2 * (RAD > 0 ? RAD : 1); ++o) {
            int jx = ix + stencil_offset(o);
            jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
            dxo[o] = jx - ix;
            if (a.g.dim == 2) {
                long jy = iy + stencil_offset(o);
                const int ny = a.g.ny;
                jy = jy < 0 ? jy + ny : (jy >= ny ? jy - ny : jy);
                dyo[o] = (int)((jy - iy) * nx);
            }
        }
    }
    // sum of (r / w_scale)^2 * 2^40 as a float pair (FP32 and integer pipes)
    F2Acc sq{0.f, 0.f};
#ifndef AC_FWD_LUNROLL
#define AC_FWD_LUNROLL 1
#endif
    // AC_FWD_LUNROLL time steps per pass (independent FP64 dependency chains)
    const int lstep = blockDim.x >> logP;
    for (int l0 = threadIdx.x >> logP; l0 < L; l0 += AC_FWD_LUNROLL * lstep) {
        double r[AC_FWD_LUNROLL][MM];
#pragma unroll
        for (int u = 0; u < AC_FWD_LUNROLL; ++u) {
            const int l = l0 + u * lstep;
            if (n < N && l < L) residual_point<MM, RAD, DIM, GEN>(a, kc, l, n, dxo, dyo, r[u]);
        }
#pragma unroll
        for (int u = 0; u < AC_FWD_LUNROLL; ++u) {
            const int l = l0 + u * lstep;
            if (l >= L) break;
            const float2 wv = a.wnorm[l];
#pragma unroll
            for (int m = 0; m < MM; ++m) {
                R v = (R)0;
                if (n < N) {
                    float hi, lo;
                    split_d2f(r[u][m], hi, lo);
                    if constexpr (sizeof(R) == 4) v = hi;   // hi is r rounded to nearest float
                    else v = r[u][m];
                    f2_add_sq(sq, hi, lo, wv.x, wv.y);
                }
                Zr[((long)l * MM + m) * P + p] = v;
            }
        }
    }
    __syncthreads();

    const int logHP = logP - 1;
    fft_fwd<C, MM, true>(Z, a.logL, logHP, MM * HP, 1, HP, reinterpret_cast<const C*>(a.tw));

    const C* Sinv = reinterpret_cast<const C*>(a.Sinv);
    C* X = reinterpret_cast<C*>(a.X);
    // in FP64, register copies of 0.5 and 0.0 (from the first twiddle,
    // 1 - 0i): h (a + b) = h a + h b exactly, written as two FMAs with
    // register operands instead of an add and a multiply by a constant.
    // In FP32 literals.
    const C w0 = reinterpret_cast<const C*>(a.tw)[0];
    const R half = sizeof(R) == 8 ? w0.x * (R)0.5 : (R)0.5, zero = sizeof(R) == 8 ? w0.y : (R)0;
    for (int idx = threadIdx.x; idx < a.F * HP; idx += blockDim.x) {
        const int k = idx >> logHP, q = idx & (HP - 1);
        const int pk = digitrev<3>(k, a.logL), pn = digitrev<3>((L - k) & (L - 1), a.logL);
        const bool realbin = (k == 0) || (2 * k == L);
        C A[MM], B[MM];
#pragma unroll
        for (int m = 0; m < MM; ++m) {
            const C zk = Z[((long)pk * MM + m) * HP + q];
            const C zn = Z[((long)pn * MM + m) * HP + q];
            if constexpr (sizeof(R) == 8) {
                A[m] = cmake(fma(zk.x, half, fma(zn.x, half, zero)),
                             realbin ? zero : fma(zk.y, half, fma(-zn.y, half, zero)));
                B[m] = cmake(fma(zk.y, half, fma(zn.y, half, zero)),
                             realbin ? zero : fma(zn.x, half, fma(-zk.x, half, zero)));
            } else {
                A[m] = cmake(half * (zk.x + zn.x), realbin ? (R)0 : half * (zk.y - zn.y));
                B[m] = cmake(half * (zk.y + zn.y), realbin ? (R)0 : half * (zn.x - zk.x));
            }
        }
        const C* S = Sinv + (long)k * MM * MM;
        const long nn = n0 + 2 * q;
#pragma unroll
        for (int m = 0; m < MM; ++m) {
            C xa = cmake(zero, zero), xb = xa;
#pragma unroll
            for (int j = 0; j < MM; ++j) {
                const C sm = S[m * MM + j];
                xa = cfma(sm, A[j], xa);
                xb = cfma(sm, B[j], xb);
            }
            C* dst = X + ((long)k * MM + m) * N + nn;
            if (nn + 1 < N) { dst[0] = xa; dst[1] = xb; }
            else if (nn < N) dst[0] = xa;
        }
    }
    const double tot = block_sum_f2(sq, red);
    if (threadIdx.x == 0) a.part[blockIdx.x + a.tile0] = tot;
}

template <typename R, int MM>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 3 : 0) k_upd(UpdArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    C* Z = reinterpret_cast<C*>(smem_raw);
    const int P = a.P, HP = P >> 1;
    const int logP = 31 - __clz(P), logHP = logP - 1;
    const int L = a.L;
    const long N = a.N;
    const long n0 = (long)(blockIdx.x + a.tile0) * P;
    const C* X = reinterpret_cast<const C*>(a.X);
    const C* Pm = reinterpret_cast<const C*>(a.Pm);

    // in FP64, register copies of 1.0 and 0.0 (first twiddle): the sums and
    // the first products below are then FMAs with register operands only.
    // In FP32 literals (registers would only raise the register count).
    const C w0 = reinterpret_cast<const C*>(a.tw)[0];
    const R one = sizeof(R) == 8 ? w0.x : (R)1, zero = sizeof(R) == 8 ? w0.y : (R)0;
    for (int idx = threadIdx.x; idx < a.F * HP; idx += blockDim.x) {
        const int k = idx >> logHP, q = idx & (HP - 1);
        const long nn = n0 + 2 * q;
        C xa[MM], xb[MM];
#pragma unroll
        for (int j = 0; j < MM; ++j) {
            const C* src = X + ((long)k * MM + j) * N + nn;
            xa[j] = nn < N ? src[0] : cmake((R)0, (R)0);
            xb[j] = nn + 1 < N ? src[1] : cmake((R)0, (R)0);
        }
        const C* Pk = Pm + (long)k * MM * MM;
        const bool realbin = (k == 0) || (2 * k == L);
        const int pk = digitrev<3>(k, a.logL), pn = digitrev<3>((L - k) & (L - 1), a.logL);
#pragma unroll
        for (int m = 0; m < MM; ++m) {
            C ya = cmake(zero, zero), yb = ya;
#pragma unroll
            for (int j = 0; j < MM; ++j) {
                const C pm = Pk[m * MM + j];
                ya = cfma(pm, xa[j], ya);
                yb = cfma(pm, xb[j], yb);
            }
            if (realbin) { ya.y = zero; yb.y = zero; }
            // Z_k = Y_a + i Y_b; Z_{L-k} = conj(Y_a) + i conj(Y_b)
            Z[((long)pk * MM + m) * HP + q] = cmake(fma(-yb.y, one, ya.x), fma(ya.y, one, yb.x));
            if (!realbin) Z[((long)pn * MM + m) * HP + q] = cmake(fma(ya.x, one, yb.y), fma(-ya.y, one, yb.x));
        }
    }
    __syncthreads();

    fft_inv<C, MM, true>(Z, a.logL, logHP, MM * HP, 1, HP, reinterpret_cast<const C*>(a.tw));

    // max over the last time block, in FP64 as bit patterns (integer pipe):
    // of |z| (correction form: |e| = sv |z| with one sv for the whole block),
    // or of |u_new - u_old| (overwrite form)
    const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long emax = 0ull;
    const bool pairs = (N & 1) == 0 && a.out_aligned16;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < L * MM * HP; idx += blockDim.x) {
        const int q = idx & (HP - 1);
        const int lm = idx >> logHP;
        const int l = lm / MM, m = lm - l * MM;
        const C z = Z[idx];
        const long nn = n0 + 2 * q;
        const double sv = a.sinv[l];
        double* o = a.out + ((long)l * MM + m) * N + nn;
        const double za = to_double(z.x), zb = to_double(z.y);
        if (l == L - 1 && !a.diff_last) {
            const unsigned long long ba = bits_of(za) & kAbs, bb = bits_of(zb) & kAbs;
            emax = ba > emax ? ba : emax;
            emax = bb > emax ? bb : emax;
        }
        double prev0 = 0.0, prev1 = 0.0;
        if (a.diff_last && l == L - 1) {
            if (nn < N) prev0 = o[0];
            if (nn + 1 < N) prev1 = o[1];
        }
        if (nn + 1 < N && pairs) {
            double2 v = a.accumulate ? *reinterpret_cast<double2*>(o) : make_double2(0.0, 0.0);
            v.x = fma(sv, za, v.x);
            v.y = fma(sv, zb, v.y);
            *reinterpret_cast<double2*>(o) = v;
        } else {
            if (nn < N) o[0] = fma(sv, za, a.accumulate ? o[0] : 0.0);
            if (nn + 1 < N) o[1] = fma(sv, zb, a.accumulate ? o[1] : 0.0);
        }
        if (a.diff_last && l == L - 1) {   // overwrite mode: |u_L^{k+1} - u_L^k| (old values read above)
            const unsigned long long ba = nn < N ? bits_of(prev0 - fma(sv, za, 0.0)) & kAbs : 0ull;
            const unsigned long long bb = nn + 1 < N ? bits_of(prev1 - fma(sv, zb, 0.0)) & kAbs : 0ull;
            emax = ba > emax ? ba : emax;
            emax = bb > emax ? bb : emax;
        }
    }
    const unsigned long long mx = block_max_bits(emax, red);
    if (threadIdx.x == 0) {
        const double v = __longlong_as_double((long long)mx);
        a.part[blockIdx.x + a.tile0] = a.diff_last ? v : v * a.sinv[L - 1];
    }
}

// TMA-staged update kernel (complex64 plans, correction form u += e): the
// same mix, inverse FFT and update as k_upd, in a persistent CTA that walks
// over tiles of P grid points.  The copy engine brings the next tile's rows
// of X (F*M rows of P complex values) and of u (L*M rows of P doubles) into
// the second of two shared-memory buffers, as 2D tensor tiles, while the CTA
// mixes, transforms and updates the current tile; so neither the mix nor the
// read-modify-write of u waits on a global load.  Full tiles only (N a
// multiple of P), u and X 16-byte aligned.
template <int MM>
__global__ void __launch_bounds__(256) k_upd_tma(const __grid_constant__ CUtensorMap mapX,
                                                 const __grid_constant__ CUtensorMap mapU, UpdArgs a,
                                                 UpdTmaGeom t) {
    typedef float2 C;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    __shared__ __align__(8) uint64_t full[2];
    C* Xs[2] = {reinterpret_cast<C*>(smem_raw), reinterpret_cast<C*>(smem_raw + t.xbuf)};
    double* Us[2] = {reinterpret_cast<double*>(smem_raw + 2 * t.xbuf),
                     reinterpret_cast<double*>(smem_raw + 2 * t.xbuf + t.ubuf)};
    C* Z = reinterpret_cast<C*>(smem_raw + 2 * (t.xbuf + t.ubuf));
    const int P = a.P, HP = P >> 1;
    const int logP = 31 - __clz(P), logHP = logP - 1;
    const int L = a.L;
    const long N = a.N;
    const C* Pm = reinterpret_cast<const C*>(a.Pm);
    const int count = blockIdx.x < t.ntiles ? (t.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    // thread 0: the boxes of local tile i into buffer b
    auto issue = [&](int i, int b) {
        const int n0 = ((int)blockIdx.x + i * (int)gridDim.x) * P;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[b], t.tile_bytes);
        for (int k = 0; k < t.xboxes; ++k)
            tma_load_2d(Xs[b] + (size_t)k * t.xrows * P, &mapX, 2 * n0, k * t.xrows, &full[b]);
        for (int k = 0; k < t.uboxes; ++k)
            tma_load_2d(Us[b] + (size_t)k * t.urows * P, &mapU, n0, k * t.urows, &full[b]);
    };
    if (count > 0 && threadIdx.x == 0) issue(0, 0);

    const unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long emax = 0ull;
    for (int i = 0; i < count; ++i) {
        const int b = i & 1;
        const long n0 = (long)((int)blockIdx.x + i * (int)gridDim.x) * P;
        // buffer b ^ 1 was last read in iteration i - 1, which ended with a block barrier
        if (i + 1 < count && threadIdx.x == 0) issue(i + 1, b ^ 1);
        const bool ok = mbar_wait_bounded(&full[b], (unsigned)((i >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            // the copy engine did not deliver within the limit: report it, give
            // the copies in flight another bounded wait, and leave
            if (threadIdx.x == 0) atomicExch(t.err, 1);
            mbar_wait_bounded(&full[b], (unsigned)((i >> 1) & 1));
            if (i + 1 < count) mbar_wait_bounded(&full[b ^ 1], (unsigned)(((i + 1) >> 1) & 1));
            return;
        }
        // y = P_k x per stored frequency, from the staged rows of X (as k_upd)
        const C* Xb = Xs[b];
        for (int idx = threadIdx.x; idx < a.F * HP; idx += blockDim.x) {
            const int k = idx >> logHP, q = idx & (HP - 1);
            C xa[MM], xb[MM];
#pragma unroll
            for (int j = 0; j < MM; ++j) {
                const C* src = Xb + ((long)k * MM + j) * P + 2 * q;
                xa[j] = src[0];
                xb[j] = src[1];
            }
            const C* Pk = Pm + (long)k * MM * MM;
            const bool realbin = (k == 0) || (2 * k == L);
            const int pk = digitrev<3>(k, a.logL), pn = digitrev<3>((L - k) & (L - 1), a.logL);
#pragma unroll
            for (int m = 0; m < MM; ++m) {
                C ya = cmake(0.f, 0.f), yb = ya;
#pragma unroll
                for (int j = 0; j < MM; ++j) {
                    const C pm = Pk[m * MM + j];
                    ya = cfma(pm, xa[j], ya);
                    yb = cfma(pm, xb[j], yb);
                }
                if (realbin) {
                    ya.y = 0.f;
                    yb.y = 0.f;
                }
                Z[((long)pk * MM + m) * HP + q] = cmake(ya.x - yb.y, ya.y + yb.x);
                if (!realbin) Z[((long)pn * MM + m) * HP + q] = cmake(ya.x + yb.y, yb.x - ya.y);
            }
        }
        __syncthreads();
        fft_inv<C, MM, true>(Z, a.logL, logHP, MM * HP, 1, HP, reinterpret_cast<const C*>(a.tw));
        // u += sinv_l * z from the staged rows of u
        const double* Ub = Us[b];
#pragma unroll 4
        for (int idx = threadIdx.x; idx < L * MM * HP; idx += blockDim.x) {
            const int q = idx & (HP - 1);
            const int lm = idx >> logHP;
            const int l = lm / MM, m = lm - l * MM;
            const C z = Z[idx];
            const double sv = a.sinv[l];
            const double za = to_double(z.x), zb = to_double(z.y);
            if (l == L - 1) {
                const unsigned long long ba = bits_of(za) & kAbs, bb = bits_of(zb) & kAbs;
                emax = ba > emax ? ba : emax;
                emax = bb > emax ? bb : emax;
            }
            double2 v = *reinterpret_cast<const double2*>(Ub + (long)lm * P + 2 * q);
            v.x = fma(sv, za, v.x);
            v.y = fma(sv, zb, v.y);
            *reinterpret_cast<double2*>(a.out + ((long)l * MM + m) * N + n0 + 2 * q) = v;
        }
        __syncthreads();
    }
    const unsigned long long mx = block_max_bits(emax, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = __longlong_as_double((long long)mx) * a.sinv[L - 1];
}

template <typename R, int MM, int RAD, int DIM, bool GEN>
static cudaError_t launch_fwd_t(const FwdArgs& a, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_fwd<R, MM, RAD, DIM, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_fwd<R, MM, RAD, DIM, GEN><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R, int MM, bool GEN>
static cudaError_t launch_fwd_g(const FwdArgs& a, int grid, size_t smem, cudaStream_t st) {
    const bool d2 = a.g.dim == 2;
    switch (a.g.rad) {
        case 1:
            return d2 ? launch_fwd_t<R, MM, 1, 2, GEN>(a, grid, smem, st)
                      : launch_fwd_t<R, MM, 1, 1, GEN>(a, grid, smem, st);
        case 2:
            return d2 ? launch_fwd_t<R, MM, 2, 2, GEN>(a, grid, smem, st)
                      : launch_fwd_t<R, MM, 2, 1, GEN>(a, grid, smem, st);
        case 3:
            return d2 ? launch_fwd_t<R, MM, 3, 2, GEN>(a, grid, smem, st)
                      : launch_fwd_t<R, MM, 3, 1, GEN>(a, grid, smem, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R, int MM>
static cudaError_t launch_fwd_m(const FwdArgs& a, int grid, size_t smem, cudaStream_t st) {
    if (!a.u || a.recompute) return launch_fwd_t<R, MM, 0, 1, true>(a, grid, smem, st);
    if (a.b || a.transposed) return launch_fwd_g<R, MM, true>(a, grid, smem, st);
    return launch_fwd_g<R, MM, false>(a, grid, smem, st);
}

template <typename R>
cudaError_t launch_fwd(const FwdArgs& a, int grid, size_t smem, cudaStream_t st) {
    switch (a.M) {
        case 1: return launch_fwd_m<R, 1>(a, grid, smem, st);
        case 2: return launch_fwd_m<R, 2>(a, grid, smem, st);
        case 3: return launch_fwd_m<R, 3>(a, grid, smem, st);
        case 4: return launch_fwd_m<R, 4>(a, grid, smem, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ac
