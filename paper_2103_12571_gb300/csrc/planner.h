// Host-side planner of the alpha-circulant solver: collocation data, the
// per-frequency eigen-tables, stencil coefficients and symbols.  Plain C++,
// double precision, no CUDA.
#pragma once
#include <complex>
#include <vector>

#include "alphacirc.h"
#include "radices.h"

namespace ac {

typedef std::complex<double> cd;

// Radau IIA nodes in (0, 1], t[M-1] = 1.  Returns false for M outside 1..8.
bool radau_nodes(int M, double* t);
// q_{mi} = int_0^{t_m} c_i, row-major M x M.
bool collocation_matrix(int M, const double* t, double* Q);

// Eigen-decomposition B = S diag(mu) S^{-1} of a small complex matrix
// (row-major n x n, n <= 8).  Columns of S have unit 2-norm.  Returns the
// 1-norm condition number of S, or a negative value if the Schur iteration
// failed to converge.
double eig_small(int n, const cd* B, cd* mu, cd* S, cd* Sinv);

// Per-frequency tables for alpha (see ac_freq_tables in alphacirc.h).
// mu: F*M, Sinv, P: F*M*M.  Returns the largest cond(S_f), negative on failure.
double freq_tables(int M, int L, double alpha, bool transposed, const double* Q,
                   const double* t, cd* mu, cd* Sinv, cd* P, double* cond);

// Finite-difference weights on offsets -3..3 (index o + 3) of the scheme
// (order, upwind) for a velocity component c: d1 = first derivative times h
// (upwind-biased against the sign of c when upwind), d2 = centred second
// derivative times h^2.  False if the scheme is not supported.
bool derivative_weights(int order, int upwind, double c, double d1[7], double d2[7]);

// The stencil of a problem on offsets -3..3: per-axis taps of
// A = nu Lap - c . grad, the scaled derivative weights d1/h and d2/h^2 per
// axis, and the radius (largest offset used by either derivative).
struct Stencil {
    double tx[7], ty[7];
    double d1x[7], d2x[7], d1y[7], d2y[7];
    int rad;
};
bool problem_stencil(const ac_problem& prob, Stencil* st);

// Symbol sigma(k) = sum_o taps[o + 3] exp(2 pi i k o / n), k = 0..n-1.
void axis_symbol(int n, const double taps[7], cd* sigma);

// w_n^k = exp(-2 pi i k / n), k < n (the full circle: the mixed-radix FFT
// stages index it with j * r).
void twiddles(int n, std::vector<cd>& tw);

// Launch shape of the solver for a problem: which spatial solve runs and
// the tiles of the time and spatial kernels.  ac_setup and the
// allocation-free preconditioner both take it from here, so that they run
// the same launches.
struct PlanShape {
    int spatial_path;               // 0: 1D FFT, one CTA per plane; 1: 2D FFT, one CTA per plane;
                                    // 2: 2D FFT in three passes; 3: BiCGStab; 4: GMRES;
                                    // 5: 1D mixed-radix FFT, one CTA per plane; 6: 2D mixed-radix
                                    // FFT in three passes (5, 6: sizes that are not powers of two);
                                    // 7: 2D FFT in one pass over a thread-block cluster
    int rows_per_block, cols_per_block;   // three-pass tiles (also set for path 7, whose
                                          // plans fall back to path 2 where the clusters do not fit)
    int cluster;                    // path 7: CTAs per cluster
    FftRadices rx, ry;              // radix plans of paths 5 and 6
    int P, grid;                    // residual kernel: grid points per CTA, CTAs
    int P_upd, grid_upd;            // update kernel: grid points per CTA, CTAs
};
// Radix plan of a mixed-radix FFT of length n (radices 8, 7, 5, 4, 3, 2, in
// that order of preference).  False if n has a prime factor above 7.
bool fft_radices(int n, FftRadices* out);

// Null on success, else a message naming the unsupported size.  rad: the
// stencil radius (Krylov paths need 2 rad + 1 points per axis).  cluster_req
// (2D power-of-two FFT solves of planes above 160 KB): 4, 8 or 16 ask for the
// single-pass solve over a cluster of that many CTAs (at most 200 KB of
// shared memory each); 0 or -1 keep the three-pass solve, which measured
// faster on every workload tried.
const char* plan_shape(const ac_problem& prob, int M, int L, int precision, int inner, int rad,
                       int cluster_req, PlanShape* out);

// The alpha-dependent tables of one preconditioner (Lemma 1, eq. (QGL)):
// per step l: s_l = alpha^{l/L}, qs_l = s_l dT Q (Q^T if transposed),
// sinv_l = alpha^{-l/L} / L times space_scale (1/N after the unnormalised
// spatial FFT solves, 1 after Krylov solves), the residual-norm weight 2^20 / (s_l w_scale)
// as a float pair; per stored frequency f: dT mu_{f,m}, S_f^{-1} and
// P_f = G_f^{-1} S_f.  Returns false (with worst_cond set) if some S_f is
// ill-conditioned (cond > 1e10) or the eigen-decomposition failed.
struct AlphaTables {
    std::vector<double> qs, s, sinv;
    std::vector<float> wnorm;       // 2 L floats: (hi, lo) per step
    std::vector<cd> mu_dT, Sinv, P;
    double worst_cond;
};
bool alpha_tables(int M, int L, double dT, const double* Q, const double* t, double alpha, bool transposed,
                  double wscale, double space_scale, AlphaTables* out);

}  // namespace ac
