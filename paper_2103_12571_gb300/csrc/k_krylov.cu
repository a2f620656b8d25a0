// Inexact inner solves of eq. (d2), (I - mu_{l,m} dT A) x^2 = x^1, by Krylov
// iterations on the periodic stencil of A.  The paper's implementation uses
// unpreconditioned GMRES with relative tolerance tau at this step (Sec. 4.1);
// the error analysis of Lemma 3 / Theorem 2 covers any inner solver that
// meets tau.  Two batched solvers, one CTA per (frequency, node) system, with
// the vectors in shared memory when they fit, else in a global scratch slice:
//
// k_bicgstab: BiCGStab.  Per iteration two stencil products and three fused
//   block reductions (<r0, v>; <t, s>, <t, t>; <r0, r>, <r, r>).  In
//   complex64 the recursively updated residual drifts away from the true one
//   once it falls below about kappa * eps_32, and the iteration stalls there;
//   with FP64 reliable updates (mu64 and x64 given) the solution is kept in an
//   FP64 accumulator, and whenever the recursive residual has dropped tenfold
//   since the last update (or meets tau) the update so far is added to it and
//   the residual is replaced by b - (I - mu A) x computed in FP64.  The
//   iteration continues with that residual, and convergence is decided on
//   it, so complex64 solves reach tolerances below the FP32 floor; a
//   stagnated system restarts from its true residual (at most 8 times).  The loop is
//   bounded by max_iter and stops early when the residual has not dropped
//   below 0.99 of its best value for 256 iterations (stagnation at the
//   precision floor).  A near-breakdown of the bi-orthogonality (|<r0, v>|
//   tiny relative to |r0| |v|, or <r0, r> = 0 or omega = 0) restarts the
//   iteration with r0 = r; after 64 restarts, or on a NaN, the system is
//   reported as broken down (negative iteration count).
// k_gmres: restarted GMRES(m), x0 = 0, as in the paper.  Arnoldi with
//   classical Gram-Schmidt and one reorthogonalisation pass (all projections
//   of a pass in one fused block reduction), complex Givens rotations on the
//   Hessenberg matrix, and the true residual b - A x recomputed at every
//   restart; it stops when the rotated residual estimate, or the true
//   residual at a restart, is at most tau |b|, after max_iter Arnoldi steps,
//   or after 8 restarts without a 1% gain (stagnation).
//
// Iteration counts per system: converged it; stagnated it + 2000000;
// iteration cap it + 1000000; breakdown or NaN -it.
#include "common.cuh"
#include "kernels.h"

namespace ac {

template <typename C>
struct BicgVecs {
    C *x, *r, *r0, *p, *v, *t;
};

// y = (I - mu A) x  with mu = dT * mu_{l,m}
template <typename R, typename C>
__device__ __forceinline__ void apply_shifted(const Grid& g, C mu, const C* __restrict__ x, C* __restrict__ y) {
    const int N = g.N, nx = g.nx;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int iy = i / nx, ix = i - iy * nx;
        C acc = cscale(x[i], (R)g.c0);
#pragma unroll
        for (int o = 0; o < 6; ++o) {   // offsets -1, +1, -2, +2, -3, +3
            if (o < 2 * g.rad) {
                const int tap = stencil_tap(o);
                int jx = ix + stencil_offset(o);
                jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
                const C xv = x[iy * nx + jx];
                acc.x += (R)g.tx[tap] * xv.x;
                acc.y += (R)g.tx[tap] * xv.y;
                if (g.dim == 2) {
                    int jy = iy + stencil_offset(o);
                    jy = jy < 0 ? jy + g.ny : (jy >= g.ny ? jy - g.ny : jy);
                    const C yv = x[jy * nx + ix];
                    acc.x += (R)g.ty[tap] * yv.x;
                    acc.y += (R)g.ty[tap] * yv.y;
                }
            }
        }
        y[i] = csub(x[i], cmul(mu, acc));
    }
}

// (A x)_i in FP64 for the reliable updates
__device__ __forceinline__ double2 stencil_fp64(const Grid& g, const double2* __restrict__ x, int i) {
    const int nx = g.nx;
    const int iy = i / nx, ix = i - iy * nx;
    const double2 c = x[i];
    double ax = g.c0 * c.x, ay = g.c0 * c.y;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        if (o < 2 * g.rad) {
            const int tap = stencil_tap(o);
            int jx = ix + stencil_offset(o);
            jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
            const double2 xv = x[iy * nx + jx];
            ax = fma(g.tx[tap], xv.x, ax);
            ay = fma(g.tx[tap], xv.y, ay);
            if (g.dim == 2) {
                int jy = iy + stencil_offset(o);
                jy = jy < 0 ? jy + g.ny : (jy >= g.ny ? jy - g.ny : jy);
                const double2 yv = x[jy * nx + ix];
                ax = fma(g.ty[tap], yv.x, ax);
                ay = fma(g.ty[tap], yv.y, ay);
            }
        }
    }
    return make_double2(ax, ay);
}

// block-wide sums of NV real values (results broadcast to every thread)
template <typename R, int NV>
__device__ __forceinline__ void block_sums(R (&v)[NV], R* scratch) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[k * 32 + w] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        R s = lane < nw ? scratch[k * 32 + lane] : (R)0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        v[k] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(512) k_bicgstab(BicgArgs a, void* scratch, int use_smem) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ R red[6 * 32];
    __shared__ double redd[32];
    const int N = a.g.N;
    C* base = use_smem ? reinterpret_cast<C*>(smem_raw)
                       : reinterpret_cast<C*>(scratch) + (long)blockIdx.x * 6 * N;
    BicgVecs<C> V{base, base + N, base + 2 * N, base + 3 * N, base + 4 * N, base + 5 * N};
    C* bx = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * N;   // right-hand side in, solution out
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C zero = cmake((R)0, (R)0);
    // FP64 reliable updates (complex64 solves with an FP64 accumulator)
    const bool rel = sizeof(R) == 4 && a.x64 != nullptr && a.mu64 != nullptr;
    double2* x64 = rel ? a.x64 + (long)blockIdx.x * N : nullptr;
    const double2 mu64 = rel ? a.mu64[blockIdx.x] : make_double2(0.0, 0.0);

    // x0 = 0, r = r0 = b, p = v = 0
    R nb[1] = {(R)0};
    double nb64[1] = {0.0};
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const C b = bx[i];
        V.x[i] = zero;
        V.r[i] = b;
        V.r0[i] = b;
        V.p[i] = zero;
        V.v[i] = zero;
        nb[0] += b.x * b.x + b.y * b.y;
        if (rel) {
            x64[i] = make_double2(0.0, 0.0);
            nb64[0] += (double)b.x * (double)b.x + (double)b.y * (double)b.y;
        }
    }
    block_sums<R, 1>(nb, red);
    if (rel) block_sums<double, 1>(nb64, redd);
    const R bnorm2 = nb[0];
    const R tol2 = (R)(a.tau * a.tau) * bnorm2;
    const double tol2_64 = a.tau * a.tau * nb64[0];
    R rmax2 = bnorm2;   // largest recursive |r|^2 since the last reliable update
    // Reliable update: x64 += x, x = 0, r = b - (I - mu A) x64 in FP64 (kept
    // in the working precision).  Returns |r|^2 in FP64; rn2 and rho_out get
    // |r|^2 and <r0, r> in the working precision.
    auto refresh = [&](R& rn2, C& rho_out) -> double {
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const C xi = V.x[i];
            double2 xd = x64[i];
            xd.x += (double)xi.x;
            xd.y += (double)xi.y;
            x64[i] = xd;
            V.x[i] = zero;
        }
        __syncthreads();
        double d[1] = {0.0};
        R f[3] = {(R)0, (R)0, (R)0};
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const double2 Ax = stencil_fp64(a.g, x64, i);
            const double2 xd = x64[i];
            const C b = bx[i];
            // r = b - x + mu A x
            const double rx = (double)b.x - xd.x + (mu64.x * Ax.x - mu64.y * Ax.y);
            const double ry = (double)b.y - xd.y + (mu64.x * Ax.y + mu64.y * Ax.x);
            d[0] += rx * rx + ry * ry;
            const C rf = cmake((R)rx, (R)ry);
            V.r[i] = rf;
            const C c = cmulc(rf, V.r0[i]);
            f[0] += c.x;
            f[1] += c.y;
            f[2] += rf.x * rf.x + rf.y * rf.y;
        }
        block_sums<double, 1>(d, redd);
        block_sums<R, 3>(f, red);
        rn2 = f[2];
        rho_out = cmake(f[0], f[1]);
        return d[0];
    };
    // |<r0, w>| below this fraction of |r0| |w| counts as a breakdown of the
    // bi-orthogonality and restarts the iteration with r0 = r
    const R brk = sizeof(R) == 8 ? (R)1e-12 : (R)1e-6;
    C rho = cmake(bnorm2, (R)0);           // <r0, r> with r = r0
    R r0n2 = bnorm2;                       // |r0|^2
    C alpha = cmake((R)1, (R)0), omega = cmake((R)1, (R)0);
    C beta = cmake((R)0, (R)0);
    int it = 0, status = 0, since_best = 0, restarts = 0, stag_restarts = 0;
    R best = bnorm2;
    if (bnorm2 == (R)0) status = 1;
    if (!(bnorm2 >= (R)0) || bnorm2 > (R)3e38) status = -1;   // non-finite right-hand side: reported, x = 0
    while (status == 0 && it < a.max_iter) {
        ++it;
        // p = r + beta (p - omega v)   (beta = 0 right after a (re)start)
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            V.p[i] = cadd(V.r[i], cmul(beta, csub(V.p[i], cmul(omega, V.v[i]))));
        __syncthreads();
        apply_shifted<R, C>(a.g, mu, V.p, V.v);
        R d1[3] = {(R)0, (R)0, (R)0};   // <r0, v> = sum conj(r0) v, |v|^2
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const C vv = V.v[i];
            const C c = cmulc(vv, V.r0[i]);
            d1[0] += c.x;
            d1[1] += c.y;
            d1[2] += vv.x * vv.x + vv.y * vv.y;
        }
        block_sums<R, 3>(d1, red);
        const C r0v = cmake(d1[0], d1[1]);
        const R r0v_abs = sqrt(r0v.x * r0v.x + r0v.y * r0v.y);
        if (!(r0v_abs > brk * sqrt(r0n2 * d1[2]))) {
            // restart from the current residual
            if (++restarts > 64) { status = -1; break; }
            R d0[1] = {(R)0};
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const C rr = V.r[i];
                V.r0[i] = rr;
                d0[0] += rr.x * rr.x + rr.y * rr.y;
            }
            block_sums<R, 1>(d0, red);
            r0n2 = d0[0];
            rho = cmake(d0[0], (R)0);
            beta = cmake((R)0, (R)0);
            if (r0n2 == (R)0) { status = 1; break; }
            if (!(r0n2 > (R)0)) { status = -1; break; }   // NaN
            continue;
        }
        alpha = cdiv(rho, r0v);
        // s = r - alpha v (stored in r)
        for (int i = threadIdx.x; i < N; i += blockDim.x) V.r[i] = csub(V.r[i], cmul(alpha, V.v[i]));
        __syncthreads();
        apply_shifted<R, C>(a.g, mu, V.r, V.t);
        R d2[4] = {(R)0, (R)0, (R)0, (R)0};   // <t, s>, <t, t>, <s, s>
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const C t = V.t[i], s = V.r[i];
            const C ts = cmulc(s, t);
            d2[0] += ts.x;
            d2[1] += ts.y;
            d2[2] += t.x * t.x + t.y * t.y;
            d2[3] += s.x * s.x + s.y * s.y;
        }
        block_sums<R, 4>(d2, red);
        if (d2[3] <= tol2 || !(d2[2] > (R)0)) {   // converged on s (or t = 0): x += alpha p
            for (int i = threadIdx.x; i < N; i += blockDim.x) V.x[i] = cadd(V.x[i], cmul(alpha, V.p[i]));
            if (!rel) {
                status = d2[3] <= tol2 ? 1 : -1;
                break;
            }
            // decide on the true residual; if it is above tau, restart from it
            R rn2;
            C rh;
            const double t2 = refresh(rn2, rh);
            if (t2 <= tol2_64) { status = 1; break; }
            if (!(t2 == t2) || !(rn2 > (R)0)) { status = -1; break; }
            if (++restarts > 64) { status = -1; break; }
            for (int i = threadIdx.x; i < N; i += blockDim.x) V.r0[i] = V.r[i];
            r0n2 = rn2;
            rho = cmake(rn2, (R)0);
            beta = cmake((R)0, (R)0);
            rmax2 = rn2;
            __syncthreads();
            continue;
        }
        omega = cscale(cmake(d2[0], d2[1]), (R)1 / d2[2]);
        // x += alpha p + omega s;  r = s - omega t
        R d3[3] = {(R)0, (R)0, (R)0};
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            V.x[i] = cadd(V.x[i], cadd(cmul(alpha, V.p[i]), cmul(omega, V.r[i])));
            const C rn = csub(V.r[i], cmul(omega, V.t[i]));
            V.r[i] = rn;
            const C c = cmulc(rn, V.r0[i]);
            d3[0] += c.x;
            d3[1] += c.y;
            d3[2] += rn.x * rn.x + rn.y * rn.y;
        }
        block_sums<R, 3>(d3, red);
        if (rel) {
            rmax2 = d3[2] > rmax2 ? d3[2] : rmax2;
            if (d3[2] <= tol2 || d3[2] < (R)0.01 * rmax2) {
                R rn2;
                C rh;
                const double t2 = refresh(rn2, rh);
                if (t2 <= tol2_64) { status = 1; break; }
                if (!(t2 == t2)) { status = -1; break; }
                d3[0] = rh.x;
                d3[1] = rh.y;
                d3[2] = rn2;
                rmax2 = rn2;
                // progress is measured on true residuals from here on (the
                // recursive one may have drifted below what is attainable)
                best = rn2;
                since_best = 0;
            }
        } else if (d3[2] <= tol2) {
            status = 1;
            break;
        }
        if (!(d3[2] == d3[2])) { status = -1; break; }   // NaN
        if (d3[2] < (R)0.99 * best) {
            best = d3[2];
            since_best = 0;
        } else if (++since_best >= 256) {
            if (rel && stag_restarts < 8) {
                // restart from the FP64 true residual with a fresh shadow vector
                ++stag_restarts;
                R rn2;
                C rh;
                const double t2 = refresh(rn2, rh);
                if (t2 <= tol2_64) { status = 1; break; }
                if (!(t2 == t2) || !(rn2 > (R)0)) { status = -1; break; }
                for (int i = threadIdx.x; i < N; i += blockDim.x) V.r0[i] = V.r[i];
                r0n2 = rn2;
                rho = cmake(rn2, (R)0);
                beta = cmake((R)0, (R)0);
                rmax2 = rn2;
                best = rn2;
                since_best = 0;
                __syncthreads();
                continue;
            }
            status = 2;   // stagnated
            break;
        }
        const C rho_new = cmake(d3[0], d3[1]);
        const R om_abs = sqrt(omega.x * omega.x + omega.y * omega.y);
        // <r0, r> shrinks naturally as the iteration converges; only an exact
        // zero (or a zero omega) is a breakdown here
        if (!(fabs(rho_new.x) + fabs(rho_new.y) > (R)0) || om_abs == (R)0) {
            if (++restarts > 64) { status = -1; break; }
            R d0[1] = {(R)0};
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const C rr = V.r[i];
                V.r0[i] = rr;
                d0[0] += rr.x * rr.x + rr.y * rr.y;
            }
            block_sums<R, 1>(d0, red);
            r0n2 = d0[0];
            rho = cmake(d0[0], (R)0);
            beta = cmake((R)0, (R)0);
            continue;
        }
        beta = cmul(cdiv(rho_new, rho), cdiv(alpha, omega));
        rho = rho_new;
    }
    __syncthreads();
    if (rel) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const C xi = V.x[i];
            const double2 xd = x64[i];
            bx[i] = cmake((R)(xd.x + (double)xi.x), (R)(xd.y + (double)xi.y));
        }
    } else {
        for (int i = threadIdx.x; i < N; i += blockDim.x) bx[i] = V.x[i];
    }
    // converged: it; stagnated: it + 2000000; iteration cap: it + 1000000; breakdown: -it
    if (threadIdx.x == 0)
        a.iters[blockIdx.x] = status < 0 ? -it : (status == 1 ? it : (status == 2 ? it + 2000000 : it + 1000000));
}

template <typename R>
cudaError_t launch_bicgstab(const BicgArgs& a, void* scratch, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const size_t need = sizeof(C) * 6 * (size_t)a.g.N;
    const int use_smem = need <= 200 * 1024;
    const size_t smem = use_smem ? need : 0;
    if (use_smem) {
        cudaError_t e = cudaFuncSetAttribute(k_bicgstab<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    } else if (!scratch) {
        return cudaErrorInvalidValue;
    }
    k_bicgstab<R><<<a.planes, 512, smem, st>>>(a, scratch, use_smem);
    return cudaGetLastError();
}

template cudaError_t launch_bicgstab<float>(const BicgArgs&, void*, cudaStream_t);
template cudaError_t launch_bicgstab<double>(const BicgArgs&, void*, cudaStream_t);

// ------------------------------------------------------------------ GMRES
constexpr int kGmresMaxM = 32;

// Projections h_k = <V_k, w> = sum_i conj(V_k[i]) w[i], k < nk, into h[]
// (shared memory, visible to all threads on return).
template <typename R, typename C>
__device__ void multi_dot(const C* V, long N, const C* w, int nk, C* red, C* h) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < nk; ++k) {
        const C* vk = V + (long)k * N;
        C s = cmake((R)0, (R)0);
        for (long i = threadIdx.x; i < N; i += blockDim.x) s = cadd(s, cmulc(w[i], vk[i]));
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) red[k * 32 + wp] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        C s = cmake((R)0, (R)0);
        for (int q = 0; q < nw; ++q) s = cadd(s, red[k * 32 + q]);
        h[k] = s;
    }
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(512) k_gmres(GmresArgs a, void* scratch, int use_smem) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ C H[(kGmresMaxM + 1) * kGmresMaxM];   // Hessenberg, column-major: H[j * (m+1) + i]
    __shared__ C red[(kGmresMaxM + 1) * 32];
    __shared__ C hv[kGmresMaxM + 1];
    __shared__ C gs[kGmresMaxM + 1];                  // rotated right-hand side beta e_1
    __shared__ C sn[kGmresMaxM], yv[kGmresMaxM];
    __shared__ R cs[kGmresMaxM];
    __shared__ R rsum[6 * 32];
    __shared__ int flag;                              // 1: leave the Arnoldi loop
    const int m = a.restart < 1 ? 1 : (a.restart > kGmresMaxM ? kGmresMaxM : a.restart);
    const long N = a.g.N;
    C* V = use_smem ? reinterpret_cast<C*>(smem_raw)
                    : reinterpret_cast<C*>(scratch) + (long)blockIdx.x * (m + 2) * N;
    C* x = V + (long)(m + 1) * N;
    C* bx = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * N;   // right-hand side in, solution out
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C zero = cmake((R)0, (R)0);

    // x = 0, r = b in V_0
    R nb[1] = {(R)0};
    for (long i = threadIdx.x; i < N; i += blockDim.x) {
        const C b = bx[i];
        x[i] = zero;
        V[i] = b;
        nb[0] += b.x * b.x + b.y * b.y;
    }
    block_sums<R, 1>(nb, rsum);
    const R bnorm = sqrt(nb[0]);
    const R tol = (R)a.tau * bnorm;
    int it = 0, status = 0, since_best = 0;
    R best = bnorm, beta = bnorm;
    if (bnorm == (R)0) status = 1;
    if (!(bnorm >= (R)0) || bnorm > (R)1.8e19) status = -1;   // non-finite right-hand side: reported, x = 0
    bool first = true;
    while (status == 0) {
        if (!first) {
            // r = b - A x into V_0 (A x through V_1)
            __syncthreads();
            apply_shifted<R, C>(a.g, mu, x, V + N);
            __syncthreads();
            R d[1] = {(R)0};
            for (long i = threadIdx.x; i < N; i += blockDim.x) {
                const C r = csub(bx[i], V[N + i]);
                V[i] = r;
                d[0] += r.x * r.x + r.y * r.y;
            }
            block_sums<R, 1>(d, rsum);
            beta = sqrt(d[0]);
            if (!(beta == beta)) { status = -1; break; }
            if (beta <= tol) { status = 1; break; }
            if (beta < (R)0.99 * best) {
                best = beta;
                since_best = 0;
            } else if (++since_best >= 8) {
                status = 2;
                break;
            }
            if (it >= a.max_iter) { status = 3; break; }
        }
        first = false;
        // V_0 = r / beta
        const R ib = (R)1 / beta;
        for (long i = threadIdx.x; i < N; i += blockDim.x) V[i] = cscale(V[i], ib);
        if (threadIdx.x == 0) {
            gs[0] = cmake(beta, (R)0);
            flag = 0;
        }
        int j = 0;
        for (; j < m; ++j) {
            C* w = V + (long)(j + 1) * N;
            __syncthreads();
            apply_shifted<R, C>(a.g, mu, V + (long)j * N, w);
            __syncthreads();
            for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[j * (m + 1) + i] = zero;
            // two passes of classical Gram-Schmidt against V_0..V_j
            for (int pass = 0; pass < 2; ++pass) {
                multi_dot<R, C>(V, N, w, j + 1, red, hv);
                for (long i = threadIdx.x; i < N; i += blockDim.x) {
                    C acc = w[i];
                    for (int k = 0; k <= j; ++k) acc = csub(acc, cmul(hv[k], V[(long)k * N + i]));
                    w[i] = acc;
                }
                if (threadIdx.x == 0)
                    for (int k = 0; k <= j; ++k) H[j * (m + 1) + k] = cadd(H[j * (m + 1) + k], hv[k]);
                __syncthreads();
            }
            R d[1] = {(R)0};
            for (long i = threadIdx.x; i < N; i += blockDim.x) d[0] += w[i].x * w[i].x + w[i].y * w[i].y;
            block_sums<R, 1>(d, rsum);
            const R hn = sqrt(d[0]);
            if (hn > (R)0) {
                const R ih = (R)1 / hn;
                for (long i = threadIdx.x; i < N; i += blockDim.x) w[i] = cscale(w[i], ih);
            }
            ++it;
            if (threadIdx.x == 0) {
                C* hc = H + j * (m + 1);
                hc[j + 1] = cmake(hn, (R)0);
                for (int k = 0; k < j; ++k) {   // earlier rotations
                    const C h0 = hc[k], h1 = hc[k + 1];
                    hc[k] = cadd(cscale(h0, cs[k]), cmul(sn[k], h1));
                    hc[k + 1] = csub(cscale(h1, cs[k]), cmul(cconj(sn[k]), h0));
                }
                // new rotation zeroing hc[j + 1] (real, >= 0)
                const C av = hc[j];
                const R aa = sqrt(av.x * av.x + av.y * av.y);
                const R rho = sqrt(aa * aa + hn * hn);
                R c;
                C sv;
                if (aa == (R)0) {
                    c = (R)0;
                    sv = cmake((R)1, (R)0);
                    hc[j] = cmake(hn, (R)0);
                } else {
                    c = aa / rho;
                    sv = cscale(av, hn / (aa * rho));          // a conj(b) / (|a| rho), b = hn real
                    hc[j] = cscale(av, rho / aa);
                }
                hc[j + 1] = zero;
                cs[j] = c;
                sn[j] = sv;
                const C gj = gs[j];
                gs[j] = cscale(gj, c);
                gs[j + 1] = cscale(cmul(cconj(sv), gj), (R)-1);
                const R est = sqrt(gs[j + 1].x * gs[j + 1].x + gs[j + 1].y * gs[j + 1].y);
                if (!(est == est) || !(rho > (R)0)) flag = 2;        // NaN or singular
                else if (est <= tol || hn == (R)0 || it >= a.max_iter) flag = 1;
            }
            __syncthreads();
            if (flag) break;
        }
        const int nk = j < m ? j + 1 : m;   // columns built in this cycle
        if (flag == 2) {
            status = -1;
            break;
        }
        // y = R^{-1} g (upper triangular), x += V y
        if (threadIdx.x == 0) {
            for (int k = nk - 1; k >= 0; --k) {
                C acc = gs[k];
                for (int q = k + 1; q < nk; ++q) acc = csub(acc, cmul(H[q * (m + 1) + k], yv[q]));
                yv[k] = cdiv(acc, H[k * (m + 1) + k]);
            }
        }
        __syncthreads();
        for (long i = threadIdx.x; i < N; i += blockDim.x) {
            C acc = x[i];
            for (int k = 0; k < nk; ++k) acc = cfma(yv[k], V[(long)k * N + i], acc);
            x[i] = acc;
        }
        // the restart recomputes the true residual and decides
    }
    __syncthreads();
    for (long i = threadIdx.x; i < N; i += blockDim.x) bx[i] = x[i];
    if (threadIdx.x == 0)
        a.iters[blockIdx.x] = status < 0 ? -it : (status == 1 ? it : (status == 2 ? it + 2000000 : it + 1000000));
}

size_t gmres_vector_bytes(int restart, long long N, size_t csize) {
    const int m = restart < 1 ? 1 : (restart > kGmresMaxM ? kGmresMaxM : restart);
    return (size_t)(m + 2) * (size_t)N * csize;
}

template <typename R>
cudaError_t launch_gmres(const GmresArgs& a, void* scratch, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const size_t need = gmres_vector_bytes(a.restart, a.g.N, sizeof(C));
    const int use_smem = need <= 160 * 1024;
    const size_t smem = use_smem ? need : 0;
    if (use_smem) {
        cudaError_t e = cudaFuncSetAttribute(k_gmres<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    } else if (!scratch) {
        return cudaErrorInvalidValue;
    }
    k_gmres<R><<<a.planes, 512, smem, st>>>(a, scratch, use_smem);
    return cudaGetLastError();
}

template cudaError_t launch_gmres<float>(const GmresArgs&, void*, cudaStream_t);
template cudaError_t launch_gmres<double>(const GmresArgs&, void*, cudaStream_t);

}  // namespace ac
