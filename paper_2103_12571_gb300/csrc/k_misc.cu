// FP64 operator and reduction kernels around the Richardson iteration:
// C u and C^T u (eq. (globalsys)), the gradient contractions of the adjoint,
// norms of the right-hand side w, and small helpers.
#include "common.cuh"
#include "kernels.h"

namespace ac {

struct Nbr {
    int dx[6], dy[6];  // offsets -1, +1, -2, +2, -3, +3 as deltas of the flat index
};

__device__ __forceinline__ Nbr neighbours(const Grid& g, long n) {
    Nbr b;
    const int nx = g.nx;
    const long iy = n / nx;
    const int ix = (int)(n - iy * nx);
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        int jx = ix + stencil_offset(o);
        jx = jx < 0 ? jx + nx : (jx >= nx ? jx - nx : jx);
        b.dx[o] = jx - ix;
        b.dy[o] = 0;
        if (g.dim == 2) {
            long jy = iy + stencil_offset(o);
            jy = jy < 0 ? jy + g.ny : (jy >= g.ny ? jy - g.ny : jy);
            b.dy[o] = (int)((jy - iy) * nx);
        }
    }
    return b;
}

// sum_o tx[o] v(x+o) + ty[o] v(y+o) with the centre tap c (taps on offsets -3..3)
__device__ __forceinline__ double stencil(const double* v, const Nbr& b, int rad, int dim,
                                          const double* tx, const double* ty, double c) {
    double acc = c * v[0];
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        if (o < 2 * rad) {
            acc = fma(tx[stencil_tap(o)], v[b.dx[o]], acc);
            if (dim == 2) acc = fma(ty[stencil_tap(o)], v[b.dy[o]], acc);
        }
    }
    return acc;
}

// out = C u (transposed = 0) or C^T u (transposed = 1; then dtQ holds dT Q^T
// and the taps those of A^T), natural time order.
__global__ void k_apply(ApplyArgs a) {
    const long N = a.g.N;
    const int M = a.M;
    const long total = (long)a.L * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int l = (int)(t / N);
        const long n = t - (long)l * N;
        const Nbr b = neighbours(a.g, n);
        double Au[8];
        const double* ub = a.u + (long)l * M * N + n;
        for (int j = 0; j < M; ++j)
            Au[j] = stencil(ub + (long)j * N, b, a.g.rad, a.g.dim, a.g.tx, a.g.ty, a.g.c0);
        double coup_all = 0.0, coup_last = 0.0;
        if (!a.transposed) {
            if (l > 0) coup_all = ub[-(long)N];                       // u_{l-1,M}
        } else {
            if (l + 1 < a.L)
                for (int j = 0; j < M; ++j) coup_last += ub[(long)(M + j) * N];  // sum_j u_{l+1,j}
        }
        for (int m = 0; m < M; ++m) {
            double v = ub[(long)m * N] - coup_all - (m == M - 1 ? coup_last : 0.0);
            for (int j = 0; j < M; ++j) v = fma(-a.dtQ[m * M + j], Au[j], v);
            a.out[((long)l * M + m) * N + n] = v;
        }
    }
}

// Partial sums of lam . (dT Q (x) D) u for D = Lap, D_x, D_y.
__global__ void __launch_bounds__(256) k_grad(GradArgs a) {
    __shared__ double red[32];
    const long N = a.g.N;
    const int M = a.M;
    const long total = (long)a.L * N;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int l = (int)(t / N);
        const long n = t - (long)l * N;
        const Nbr b = neighbours(a.g, n);
        double Lu[8], Dx[8], Dy[8];
        const double* ub = a.u + (long)l * M * N + n;
        for (int j = 0; j < M; ++j) {
            const double* v = ub + (long)j * N;
            Lu[j] = stencil(v, b, a.g.rad, a.g.dim, a.d2x, a.d2y, a.d2x[3] + (a.g.dim == 2 ? a.d2y[3] : 0.0));
            Dx[j] = stencil(v, b, a.g.rad, 1, a.d1x, a.d1x, a.d1x[3]);
            Dy[j] = 0.0;
            if (a.g.dim == 2) {
                // y-derivative only: use the y offsets with the d1y taps
                double acc = a.d1y[3] * v[0];
                for (int o = 0; o < 2 * a.g.rad; ++o) acc = fma(a.d1y[stencil_tap(o)], v[b.dy[o]], acc);
                Dy[j] = acc;
            }
        }
        const double* lb = a.lam + (long)l * M * N + n;
        for (int m = 0; m < M; ++m) {
            double ql = 0.0, qx = 0.0, qy = 0.0;
            for (int j = 0; j < M; ++j) {
                const double q = a.dtQ[m * M + j];
                ql = fma(q, Lu[j], ql);
                qx = fma(q, Dx[j], qx);
                qy = fma(q, Dy[j], qy);
            }
            const double lv = lb[(long)m * N];
            s0 = fma(lv, ql, s0);
            s1 = fma(lv, qx, s1);
            s2 = fma(lv, qy, s2);
        }
    }
    s0 = block_sum_d(s0, red);
    if (threadIdx.x == 0) a.part[blockIdx.x * 3 + 0] = s0;
    s1 = block_sum_d(s1, red);
    if (threadIdx.x == 0) a.part[blockIdx.x * 3 + 1] = s1;
    s2 = block_sum_d(s2, red);
    if (threadIdx.x == 0) a.part[blockIdx.x * 3 + 2] = s2;
}

__global__ void k_sum_blocks(const double* lam, int M, long N, double* du0) {
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += lam[(long)m * N + n];
        du0[n] = s;
    }
}

__global__ void k_reverse_time(double* v, int L, long blk) {
    const long total = (long)(L / 2) * blk;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int l = (int)(t / blk);
        const long i = t - (long)l * blk;
        double* a = v + (long)l * blk + i;
        double* b = v + (long)(L - 1 - l) * blk + i;
        const double x = *a;
        *a = *b;
        *b = x;
    }
}

// per-block sum of squares (part[2b]) and max |v| (part[2b+1]) in FP64
__global__ void __launch_bounds__(256) k_norms(const double* v, long n, double* part) {
    __shared__ double red[32];
    double s = 0.0, mx = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double x = v[i];
        s = fma(x, x, s);
        mx = fmax(mx, fabs(x));
    }
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = s;
    // max via the same reduction tree
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r = fmax(r, red[w]);
        part[2 * blockIdx.x + 1] = r;
    }
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t st) {
    long total = (long)a.L * a.g.N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_apply<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_grad(const GradArgs& a, int grid, cudaStream_t st) {
    k_grad<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sum_blocks(const double* lam, int M, int N, double* du0, cudaStream_t st) {
    int grid = (N + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_sum_blocks<<<grid, 256, 0, st>>>(lam, M, N, du0);
    return cudaGetLastError();
}

cudaError_t launch_reverse_time(double* v, int L, long long blk, cudaStream_t st) {
    long total = (long)(L / 2) * blk;
    if (total == 0) return cudaSuccess;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_reverse_time<<<grid, 256, 0, st>>>(v, L, blk);
    return cudaGetLastError();
}

cudaError_t launch_norms(const double* v, long long n, double* part, int grid, cudaStream_t st) {
    k_norms<<<grid, 256, 0, st>>>(v, n, part);
    return cudaGetLastError();
}

}  // namespace ac

namespace ac {

// sum of squares and max |w| of w = (u0 stacked over the M nodes of block 0) + b
__global__ void __launch_bounds__(256) k_wnorms(const double* u0, const double* b, int L, int M, long N,
                                                double* part) {
    __shared__ double red[32];
    const long total = b ? (long)L * M * N : (long)M * N;
    double s = 0.0, mx = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long blk = (long)M * N;
        const long l = i / blk;
        const long n = (i - l * blk) % N;
        double w = b ? b[i] : 0.0;
        if (l == 0 && u0) w += u0[n];
        s = fma(w, w, s);
        mx = fmax(mx, fabs(w));
    }
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = s;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r = fmax(r, red[w]);
        part[2 * blockIdx.x + 1] = r;
    }
}

// u[l][m][n] = u0[n] (0 if u0 is null): the initial iterate of Sec. 5
__global__ void k_fill_stack(const double* u0, double* u, long total, long N) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
        u[i] = u0 ? u0[i % N] : 0.0;
}

cudaError_t launch_wnorms(const double* u0, const double* b, int L, int M, long long N, double* part, int grid,
                          cudaStream_t st) {
    k_wnorms<<<grid, 256, 0, st>>>(u0, b, L, M, N, part);
    return cudaGetLastError();
}

// per-block max |A u0|
__global__ void __launch_bounds__(256) k_a_inf(Grid g, const double* u0, double* part) {
    __shared__ double red[32];
    double mx = 0.0;
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < g.N; n += (long)gridDim.x * blockDim.x) {
        const Nbr b = neighbours(g, n);
        mx = fmax(mx, fabs(stencil(u0 + n, b, g.rad, g.dim, g.tx, g.ty, g.c0)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r = fmax(r, red[w]);
        part[blockIdx.x] = r;
    }
}

cudaError_t launch_a_inf(const Grid& g, const double* u0, double* part, int grid, cudaStream_t st) {
    k_a_inf<<<grid, 256, 0, st>>>(g, u0, part);
    return cudaGetLastError();
}

// v[l][m][n] = sum_j dtQ[m][j] b[l][j][n]
__global__ void k_colloc_rhs(const double* b, const double* dtQ, double* v, int L, int M, long N) {
    const long total = (long)L * N;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int l = (int)(t / N);
        const long n = t - (long)l * N;
        const double* bl = b + (long)l * M * N + n;
        double bj[8];
        for (int j = 0; j < M; ++j) bj[j] = bl[(long)j * N];
        for (int m = 0; m < M; ++m) {
            double acc = 0.0;
            for (int j = 0; j < M; ++j) acc = fma(dtQ[m * M + j], bj[j], acc);
            v[((long)l * M + m) * N + n] = acc;
        }
    }
}

cudaError_t launch_colloc_rhs(const double* b, const double* dtQ, double* v, int L, int M, long long N,
                              cudaStream_t st) {
    const long total = (long)L * N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_colloc_rhs<<<grid, 256, 0, st>>>(b, dtQ, v, L, M, N);
    return cudaGetLastError();
}

cudaError_t launch_fill_stack(const double* u0, double* u, int L, int M, long long N, cudaStream_t st) {
    const long total = (long)L * M * N;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_fill_stack<<<grid, 256, 0, st>>>(u0, u, total, N);
    return cudaGetLastError();
}

// Sequential collocation stepping by diagonalisation of Q (the baseline the
// paper calls T_Mpar, Sec. 4.2): with Q = S diag(lambda) S^{-1}, one step
//   (I - dT Q (x) A) u_l = 1 (x) u_{l-1,M} + v_l
// is z = (S^{-1} (x) I) rhs, M shifted solves (I - dT lambda_m A) z_m, and
// u_l = (S (x) I) z.  k_seq_in forms z (transform precision), k_seq_out
// forms u_l (real part, FP64).
template <typename R>
__global__ void __launch_bounds__(256) k_seq_in(int M, long N, const double* __restrict__ uprev,
                                                const double* __restrict__ v, const double* __restrict__ Sinv,
                                                typename Cx<R>::T* __restrict__ X) {
    typedef typename Cx<R>::T C;
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
        const double up = uprev[n];
        double w[4];
        for (int j = 0; j < M; ++j) w[j] = up + (v ? v[(long)j * N + n] : 0.0);
        for (int m = 0; m < M; ++m) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < M; ++j) {
                re = fma(Sinv[2 * (m * M + j)], w[j], re);
                im = fma(Sinv[2 * (m * M + j) + 1], w[j], im);
            }
            C z;
            z.x = (R)re;
            z.y = (R)im;
            X[(long)m * N + n] = z;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_seq_out(int M, long N, const typename Cx<R>::T* __restrict__ X,
                                                 const double* __restrict__ S, double* __restrict__ out) {
    typedef typename Cx<R>::T C;
    for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < N; n += (long)gridDim.x * blockDim.x) {
        double zr[4], zi[4];
        for (int j = 0; j < M; ++j) {
            const C z = X[(long)j * N + n];
            zr[j] = (double)z.x;
            zi[j] = (double)z.y;
        }
        for (int m = 0; m < M; ++m) {
            double acc = 0.0;
            for (int j = 0; j < M; ++j) {
                acc = fma(S[2 * (m * M + j)], zr[j], acc);
                acc = fma(-S[2 * (m * M + j) + 1], zi[j], acc);
            }
            out[(long)m * N + n] = acc;
        }
    }
}

static int seq_grid(long long N) {
    long g = (long)((N + 255) / 256);
    return (int)(g > 152 * 8 ? 152 * 8 : g);
}

template <typename R>
cudaError_t launch_seq_in(int M, long long N, const double* uprev, const double* v, const double* Sinv, void* X,
                          cudaStream_t st) {
    if (M < 1 || M > 4) return cudaErrorInvalidValue;
    k_seq_in<R><<<seq_grid(N), 256, 0, st>>>(M, N, uprev, v, Sinv, reinterpret_cast<typename Cx<R>::T*>(X));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_seq_out(int M, long long N, const void* X, const double* S, double* out, cudaStream_t st) {
    if (M < 1 || M > 4) return cudaErrorInvalidValue;
    k_seq_out<R><<<seq_grid(N), 256, 0, st>>>(M, N, reinterpret_cast<const typename Cx<R>::T*>(X), S, out);
    return cudaGetLastError();
}

template cudaError_t launch_seq_in<float>(int, long long, const double*, const double*, const double*, void*,
                                          cudaStream_t);
template cudaError_t launch_seq_in<double>(int, long long, const double*, const double*, const double*, void*,
                                           cudaStream_t);
template cudaError_t launch_seq_out<float>(int, long long, const void*, const double*, double*, cudaStream_t);
template cudaError_t launch_seq_out<double>(int, long long, const void*, const double*, double*, cudaStream_t);

// ---------------------------------------------- outer Krylov vector kernels
// Space-time vectors of n FP64 values.  k_mdot: partial sums of <V_j, w>,
// j < k <= 8 per launch (one pass over w), per block into part[j * grid + b].
// k_maxpy: y = beta y + sum_j c_j V_j, j < k <= 8.
__global__ void __launch_bounds__(256) k_mdot(VecList V, int k, const double* __restrict__ w, long n,
                                              double* __restrict__ part) {
    __shared__ double red[8 * 8];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < k) acc[j] = fma(V.v[j][i], wi, acc[j]);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        double s = acc[j];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[j * 8 + wp] = s;
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x * 8 + q];
        part[(long)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_maxpy(VecList V, Coefs c, int k, double beta, double* __restrict__ y,
                                               long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double acc = beta == 0.0 ? 0.0 : beta * y[i];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < k) acc = fma(c.c[j], V.v[j][i], acc);
        y[i] = acc;
    }
}

int krylov_grid() { return 152 * 8; }

cudaError_t launch_mdot(const VecList& V, int k, const double* w, long long n, double* part, cudaStream_t st) {
    if (k < 1 || k > 8) return cudaErrorInvalidValue;
    k_mdot<<<krylov_grid(), 256, 0, st>>>(V, k, w, n, part);
    return cudaGetLastError();
}

cudaError_t launch_maxpy(const VecList& V, const Coefs& c, int k, double beta, double* y, long long n,
                         cudaStream_t st) {
    if (k < 0 || k > 8) return cudaErrorInvalidValue;
    k_maxpy<<<krylov_grid(), 256, 0, st>>>(V, c, k, beta, y, n);
    return cudaGetLastError();
}

// r = w - Cu with w = (u0 stacked in block 0) + b, natural time order
__global__ void __launch_bounds__(256) k_w_minus(const double* __restrict__ u0, const double* __restrict__ b,
                                                 const double* __restrict__ Cu, double* __restrict__ r, long MN,
                                                 long N, long total) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        double w = (i < MN && u0) ? u0[i % N] : 0.0;
        if (b) w += b[i];
        r[i] = w - Cu[i];
    }
}

cudaError_t launch_w_minus(const double* u0, const double* b, const double* Cu, double* r, int L, int M,
                           long long N, cudaStream_t st) {
    k_w_minus<<<krylov_grid(), 256, 0, st>>>(u0, b, Cu, r, (long)M * N, N, (long)L * M * N);
    return cudaGetLastError();
}

}  // namespace ac

namespace ac {

// FP64 FMA throughput probe: 8 independent chains of FMAs per thread whose
// operands are all registers (a and b are loaded from memory, not taken
// from the constant bank, which would slow the FMAs).
__global__ void __launch_bounds__(256) k_dfma_rate(const double* __restrict__ ab, int rounds,
                                                    double* __restrict__ sink) {
    const double a = ab[0], b = ab[1];
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == ab[2]) sink[blockIdx.x] = s;   // ab[2] is never reached: keeps the chains live
}

cudaError_t launch_dfma_rate(const double* ab, int rounds, double* sink, int grid, cudaStream_t st) {
    k_dfma_rate<<<grid, 256, 0, st>>>(ab, rounds, sink);
    return cudaGetLastError();
}

}  // namespace ac
