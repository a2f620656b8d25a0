// Argument blocks and launchers of the solver kernels (internal to the
// library).  All pointers are device pointers.
#pragma once
#include <cuda_runtime.h>

#include "radices.h"

namespace ac {

// Off-centre stencil offsets in the order the kernels visit them (radius 1,
// then 2, then 3) and the matching tap index offset + 3.
__host__ __device__ constexpr int stencil_offset(int o) { return (o & 1) ? (o >> 1) + 1 : -((o >> 1) + 1); }
__host__ __device__ constexpr int stencil_tap(int o) { return stencil_offset(o) + 3; }

// Geometry of the periodic grid and the per-axis stencil of A.
struct Grid {
    int dim, nx, ny, N;      // N = nx * ny (ny = 1 in 1D)
    int rad;                 // stencil radius (1..3)
    double tx[7], ty[7];     // per-axis taps on offsets -3..3 (A = x part + y part)
    double c0;               // tx[3] + ty[3], the combined centre tap
};

// Residual + alpha-scaling + forward time FFT + node mixing (steps i-ii and
// eq. (d1)):  X[f][m][n] = sum_j Sinv_f[m][j] * FFT_l( s_l * (w - C u)_{l,j,n} ).
struct FwdArgs {
    Grid g;
    int M, L, logL, F, P;        // P grid points per block
    int tile0;                   // first tile (block b works on tile tile0 + b; partial at part[tile0 + b])
    const double* u;             // L*M*N or null (then r = b)
    const double* u0;            // N or null: block-1 right-hand side
    const double* b;             // L*M*N or null: full right-hand side
    int b_reversed;              // read b[L-1-l] instead of b[l]
    int transposed;              // coupling H^T (adjoint) instead of H
    int recompute;               // paper's form: r = w + (C_alpha - C) u, i.e. w - alpha H u_L in block 1 only
    double alpha;                // alpha of the recompute form
    const double* qs;            // [L][M][M] s_l * dT * Q (Q^T if transposed)
    const double* s;             // [L] s_l = alpha^{l/L}
    const float2* wnorm;         // [L] 2^20 / (s_l * w_scale) as a float pair (hi, lo), for the residual norm
    const void* tw;              // L/2 twiddles exp(-2 pi i k / L), complex of the kernel type
    const void* Sinv;            // [F][M][M] complex of the kernel type
    void* X;                     // [F][M][N] complex of the kernel type
    double* part;                // [gridDim.x] partial sums of (2^20 r / w_scale)^2
};

// Node back-mixing + inverse time FFT + un-scaling + update (eqs. (d3),
// (Gsubstitution), (s3)):  out_l (+)= sinv_l * IFFT_k( P_f X[f] )_l.
struct UpdArgs {
    int N, M, L, logL, F, P;
    int tile0;                   // first tile, as in FwdArgs (k_upd; k_upd_tma ignores it)
    const void* X;               // [F][M][N]
    const void* Pm;              // [F][M][M]
    const void* tw;              // L/2 twiddles
    const double* sinv;          // [L] alpha^{-l/L} / L
    double* out;                 // L*M*N
    int accumulate;              // 1: out += e, 0: out = e
    int out_aligned16;           // out is 16-byte aligned (set by launch_upd): double2 access allowed
    int diff_last;               // with accumulate = 0: part = max |out_new - out_old| over the last time block
    double* part;                // [gridDim.x] max |e| (or |u_new - u_old|) over the last time block
};

// Geometry of the TMA-staged update kernel (k_upd_tma): per tile, X rows in
// xboxes boxes of xrows rows, u rows in uboxes boxes of urows rows; two X
// and two u buffers and the transform buffer Z in dynamic shared memory.
struct UpdTmaGeom {
    int ntiles;                  // N / P
    int xboxes, xrows, uboxes, urows;
    unsigned tile_bytes;         // bytes the copy engine delivers per tile (whole boxes)
    unsigned xbuf, ubuf, zbuf;   // bytes of one X buffer, one u buffer and of Z (multiples of 128)
    int* err;                    // set to 1 if a wait on the copy engine timed out
};

// Spatial solves of eq. (d2) on the F*M planes X[f][m][:].
struct SpaceArgs {
    int nx, ny, lognx, logny, planes, M;
    void* X;
    const void* mu_dT;           // [F*M] complex dT * mu_{f,m}
    const void* sig_x;           // [nx] complex symbol of the x part of A
    const void* sig_y;           // [ny] complex symbol of the y part (2D)
    const void* tw_x;            // [nx] twiddles exp(-2 pi i k / nx), k < nx
    const void* tw_y;            // [ny] twiddles
    int rows_per_block, cols_per_block;
    FftRadices rx, ry;           // radix plans of the mixed-radix (non-power-of-two) solves
    int cluster;                 // CTAs per cluster of the single-pass 2D solve (4, 8, 16)
};

// BiCGStab on (I - dT mu A) x = X-plane with the stencil, tolerance tau.
struct BicgArgs {
    Grid g;
    int planes, M, max_iter;
    double tau;
    void* X;                     // in: right-hand sides, out: solutions
    const void* mu_dT;
    int* iters;                  // [planes] iterations used (negative on breakdown)
    // complex64 solves with FP64 reliable updates (both null otherwise)
    const double2* mu64;         // [planes] dT mu in FP64
    double2* x64;                // [planes][N] FP64 solution accumulators
};

struct GmresArgs {
    Grid g;
    int planes, M, max_iter, restart;
    double tau;
    void* X;                     // in: right-hand sides, out: solutions
    const void* mu_dT;
    int* iters;                  // [planes] Arnoldi steps used (encoding as BicgArgs)
};

struct ApplyArgs {
    Grid g;
    int M, L, transposed;
    const double* u;
    double* out;
    const double* dtQ;           // [M][M] dT * Q (Q^T if transposed)
};

struct GradArgs {
    Grid g;
    int M, L;
    const double* u;
    const double* lam;
    const double* dtQ;           // [M][M] dT * Q
    double d2x[7], d1x[7], d2y[7], d1y[7];  // second/first derivative taps per axis, offsets -3..3
    double* part;                // [gridDim.x][3]
};

template <typename R> cudaError_t launch_fwd(const FwdArgs& a, int grid, size_t smem, cudaStream_t st);
// sequential stepping by diagonalisation of Q: z = (S^{-1} (x) I)(1 (x) uprev + v)
// (v: M*N or null; Sinv, S: M*M complex as interleaved doubles; X: M*N complex
// of precision R), and out = Re (S (x) I) z
template <typename R>
cudaError_t launch_seq_in(int M, long long N, const double* uprev, const double* v, const double* Sinv, void* X,
                          cudaStream_t st);
template <typename R>
cudaError_t launch_seq_out(int M, long long N, const void* X, const double* S, double* out, cudaStream_t st);
// outer Krylov vector kernels (at most 8 vectors per launch)
struct VecList {
    const double* v[8];
};
struct Coefs {
    double c[8];
};
int krylov_grid();
// part[j * krylov_grid() + b] = block b's partial sum of <V_j, w>, j < k
cudaError_t launch_mdot(const VecList& V, int k, const double* w, long long n, double* part, cudaStream_t st);
// y = beta y + sum_{j<k} c_j V_j  (beta = 0: y is not read)
cudaError_t launch_maxpy(const VecList& V, const Coefs& c, int k, double beta, double* y, long long n,
                         cudaStream_t st);
// r = (u0 stacked in block 0) + b - Cu  (u0, b may be null)
cudaError_t launch_w_minus(const double* u0, const double* b, const double* Cu, double* r, int L, int M,
                           long long N, cudaStream_t st);
template <typename R> cudaError_t launch_gmres(const GmresArgs& a, void* scratch, cudaStream_t st);
// bytes of Krylov vectors per system (basis of restart + 1 vectors and x)
size_t gmres_vector_bytes(int restart, long long N, size_t csize);
template <typename R> cudaError_t launch_upd(const UpdArgs& a, int grid, size_t smem, cudaStream_t st);
// TMA-staged update (complex64, correction form); maps: X as [F*M rows][2N floats],
// u as [L*M rows][N doubles] (CUtensorMap, passed by address)
cudaError_t launch_upd_tma(const void* mapX, const void* mapU, const UpdArgs& a, const UpdTmaGeom& g, int grid,
                           cudaStream_t st);
size_t upd_tma_smem(const UpdTmaGeom& g);
int upd_tma_ctas_per_sm(int M, const UpdTmaGeom& g);
// shared memory the update kernel needs for these arguments (rsize = bytes per real of the transform)
size_t upd_smem(const UpdArgs& a, size_t rsize);
template <typename R> cudaError_t launch_space_1d(const SpaceArgs& a, cudaStream_t st);
template <typename R> cudaError_t launch_space_2d_small(const SpaceArgs& a, cudaStream_t st);
template <typename R> cudaError_t launch_space_rows(const SpaceArgs& a, int inverse, cudaStream_t st);
template <typename R> cudaError_t launch_space_cols(const SpaceArgs& a, cudaStream_t st);
// Single-pass 2D solve, one plane per cluster of a.cluster CTAs.  With fits
// non-null nothing is launched: *fits receives the number of clusters the
// device can hold at once (0: the launch would fail).
template <typename R> cudaError_t launch_space_cluster(const SpaceArgs& a, cudaStream_t st, int* fits);
// shared memory per CTA of the single-pass 2D solve
size_t space_cluster_smem(int nx, int ny, int cs, size_t csize);
// Mixed-radix solves (grid sizes with prime factors 2, 3, 5, 7 only): one CTA
// per 1D plane, and the row / column passes of the three-pass 2D solve.
template <typename R> cudaError_t launch_space_mr_1d(const SpaceArgs& a, cudaStream_t st);
template <typename R> cudaError_t launch_space_mr_rows(const SpaceArgs& a, int inverse, cudaStream_t st);
template <typename R> cudaError_t launch_space_mr_cols(const SpaceArgs& a, cudaStream_t st);
// Shared memory of a mixed-radix pass (0: 1D plane of n, 1: batch rows of n,
// 2: batch columns of ny) for complex values of csize bytes.
size_t space_mr_smem(int pass, int n, int batch, int ny, size_t csize);
template <typename R> cudaError_t launch_bicgstab(const BicgArgs& a, void* scratch, cudaStream_t st);
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t st);
cudaError_t launch_grad(const GradArgs& a, int grid, cudaStream_t st);
cudaError_t launch_sum_blocks(const double* lam, int M, int N, double* du0, cudaStream_t st);
cudaError_t launch_reverse_time(double* v, int L, long long blk, cudaStream_t st);
cudaError_t launch_norms(const double* v, long long n, double* part, int grid, cudaStream_t st);

}  // namespace ac
