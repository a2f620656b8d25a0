// Host-side planner of the alpha-circulant solver: collocation data, the
// per-frequency eigen-tables, stencil coefficients and symbols.  Plain C++,
// double precision, no CUDA.
#pragma once
#include <complex>
#include <vector>

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

// Central-difference coefficients on offsets -2..2 (index o + 2):
// d1: first derivative times h, d2: second derivative times h^2.
void central_coeffs(int order, double d1[5], double d2[5]);

// Per-axis taps of A = nu Lap - c d/dx on offsets -2..2 (index o + 2).
void axis_taps(int order, int n, double length, double nu, double c, double taps[5]);

// Symbol sigma(k) = sum_o taps[o] exp(2 pi i k o / n), k = 0..n-1.
void axis_symbol(int n, const double taps[5], cd* sigma);

}  // namespace ac
