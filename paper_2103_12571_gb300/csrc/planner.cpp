// Host-side planner: Radau IIA data (Sec. 2.1, 2.3), the eigen-decomposition
// of Q G_l^{-1} per time frequency (Lemma 1, eq. (QGL), Algorithm 1), the
// alpha sequence of Algorithm 2 and stencil symbols.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "alphacirc.h"

namespace ac {

// ---------------------------------------------------------------- nodes, Q
// P_{M-1}(x) + P_M(x) and its derivative by the three-term recurrence.
static void radau_poly(int M, double x, double* p, double* dp) {
    double pk = 1.0, pkm1 = 0.0, dpk = 0.0, dpkm1 = 0.0;  // P_0, P_{-1}
    double prev = 0.0, dprev = 0.0;
    for (int k = 0; k < M; ++k) {
        // P_{k+1} = ((2k+1) x P_k - k P_{k-1}) / (k+1)
        double pn = ((2 * k + 1) * x * pk - k * pkm1) / (k + 1);
        double dpn = ((2 * k + 1) * (pk + x * dpk) - k * dpkm1) / (k + 1);
        prev = pk;
        dprev = dpk;
        pkm1 = pk;
        dpkm1 = dpk;
        pk = pn;
        dpk = dpn;
    }
    *p = pk + prev;      // P_M + P_{M-1}
    *dp = dpk + dprev;
}

bool radau_nodes(int M, double* t) {
    if (M < 1 || M > 8) return false;
    double x[8];
    for (int j = 0; j < M; ++j) x[j] = -std::cos(2.0 * M_PI * j / (2.0 * M - 1.0));
    x[0] = -1.0;
    // Newton with deflation of the roots already found
    for (int j = 1; j < M; ++j) {
        double xj = x[j];
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            radau_poly(M, xj, &p, &dp);
            double s = 0.0;
            for (int i = 0; i < j; ++i) s += 1.0 / (xj - x[i]);
            double step = p / (dp - p * s);
            xj -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        x[j] = xj;
    }
    for (int j = 0; j < M; ++j) t[j] = 0.5 * (1.0 - x[j]);
    std::sort(t, t + M);
    t[M - 1] = 1.0;
    return true;
}

// Dense real solve A X = B (n x n, nrhs columns) by Gaussian elimination with
// partial pivoting; A, B row-major, overwritten.
static bool solve_real(int n, double* A, int nrhs, double* B) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            for (int k = 0; k < nrhs; ++k) std::swap(B[c * nrhs + k], B[piv * nrhs + k]);
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            for (int k = 0; k < nrhs; ++k) B[r * nrhs + k] -= f * B[c * nrhs + k];
        }
    }
    for (int c = n - 1; c >= 0; --c)
        for (int k = 0; k < nrhs; ++k) {
            double s = B[c * nrhs + k];
            for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * B[j * nrhs + k];
            B[c * nrhs + k] = s / A[c * n + c];
        }
    return true;
}

// Q maps the monomials t^k to t^{k+1}/(k+1) on the nodes (the Vandermonde
// relation Q W = D_M W of Lemma 2's proof), so Q = W' W^{-1}; solved here as
// W^T Q^T = W'^T.
bool collocation_matrix(int M, const double* t, double* Q) {
    if (M < 1 || M > 8) return false;
    double WT[64], WpT[64];
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < M; ++k) {
            WT[k * M + m] = std::pow(t[m], k);
            WpT[k * M + m] = std::pow(t[m], k + 1) / (k + 1);
        }
    if (!solve_real(M, WT, M, WpT)) return false;  // WpT now holds Q^T
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < M; ++i) Q[m * M + i] = WpT[i * M + m];
    return true;
}

// ------------------------------------------------------- small complex eig
// Complex Schur form by Householder reduction to Hessenberg form and shifted
// QR steps with Givens rotations; eigenvectors by back substitution.
static bool schur_small(int n, cd* A, cd* Z) {
    for (int i = 0; i < n * n; ++i) Z[i] = 0.0;
    for (int i = 0; i < n; ++i) Z[i * n + i] = 1.0;
    // Hessenberg reduction
    for (int k = 0; k + 2 < n; ++k) {
        int len = n - k - 1;
        cd v[8];
        double xn = 0.0;
        for (int i = 0; i < len; ++i) {
            v[i] = A[(k + 1 + i) * n + k];
            xn += std::norm(v[i]);
        }
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        cd ph = std::abs(v[0]) > 0 ? v[0] / std::abs(v[0]) : cd(1.0);
        v[0] += ph * xn;
        double vn = 0.0;
        for (int i = 0; i < len; ++i) vn += std::norm(v[i]);
        vn = std::sqrt(vn);
        for (int i = 0; i < len; ++i) v[i] /= vn;
        // A <- (I - 2 v v^H) A (rows k+1..)
        for (int j = 0; j < n; ++j) {
            cd s = 0.0;
            for (int i = 0; i < len; ++i) s += std::conj(v[i]) * A[(k + 1 + i) * n + j];
            for (int i = 0; i < len; ++i) A[(k + 1 + i) * n + j] -= 2.0 * v[i] * s;
        }
        // A <- A (I - 2 v v^H) (cols k+1..), Z likewise
        for (int r = 0; r < n; ++r) {
            cd s = 0.0, sz = 0.0;
            for (int i = 0; i < len; ++i) {
                s += A[r * n + k + 1 + i] * v[i];
                sz += Z[r * n + k + 1 + i] * v[i];
            }
            for (int i = 0; i < len; ++i) {
                A[r * n + k + 1 + i] -= 2.0 * s * std::conj(v[i]);
                Z[r * n + k + 1 + i] -= 2.0 * sz * std::conj(v[i]);
            }
        }
        for (int i = k + 2; i < n; ++i) A[i * n + k] = 0.0;
    }
    // shifted QR iterations
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        if (++total > 1000) return false;
        int l = hi;
        while (l > 0) {
            double s = std::abs(A[l * n + l]) + std::abs(A[(l - 1) * n + l - 1]);
            if (std::abs(A[l * n + l - 1]) <= eps * (s > 0 ? s : 1.0)) break;
            --l;
        }
        if (l > 0) A[l * n + l - 1] = 0.0;
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        ++iter;
        // Wilkinson shift from the trailing 2x2 block
        cd a = A[(hi - 1) * n + hi - 1], b = A[(hi - 1) * n + hi];
        cd c = A[hi * n + hi - 1], d = A[hi * n + hi];
        cd tr2 = 0.5 * (a + d);
        cd disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
        cd mu1 = tr2 + disc, mu2 = tr2 - disc;
        cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
        if (iter % 11 == 10) mu = d + cd(std::abs(c), 0.0);  // exceptional shift
        for (int k = l; k <= hi; ++k) A[k * n + k] -= mu;
        cd gc[8], gs[8];
        for (int k = l; k < hi; ++k) {
            cd x = A[k * n + k], y = A[(k + 1) * n + k];
            double r = std::sqrt(std::norm(x) + std::norm(y));
            cd cc = r > 0 ? x / r : cd(1.0), ss = r > 0 ? y / r : cd(0.0);
            gc[k] = cc;
            gs[k] = ss;
            for (int j = k; j < n; ++j) {  // rows k, k+1 <- G [row k; row k+1]
                cd p = A[k * n + j], q = A[(k + 1) * n + j];
                A[k * n + j] = std::conj(cc) * p + std::conj(ss) * q;
                A[(k + 1) * n + j] = -ss * p + cc * q;
            }
        }
        for (int k = l; k < hi; ++k) {  // columns k, k+1 <- [col k, col k+1] G^H
            cd cc = gc[k], ss = gs[k];
            int rmax = std::min(k + 2, n - 1);
            for (int r = 0; r <= rmax; ++r) {
                cd p = A[r * n + k], q = A[r * n + k + 1];
                A[r * n + k] = p * cc + q * ss;
                A[r * n + k + 1] = -p * std::conj(ss) + q * std::conj(cc);
            }
            for (int r = 0; r < n; ++r) {
                cd p = Z[r * n + k], q = Z[r * n + k + 1];
                Z[r * n + k] = p * cc + q * ss;
                Z[r * n + k + 1] = -p * std::conj(ss) + q * std::conj(cc);
            }
        }
        for (int k = l; k <= hi; ++k) A[k * n + k] += mu;
    }
    return true;
}

// Inverse by Gauss-Jordan with partial pivoting; returns false if singular.
static bool invert_small(int n, const cd* S, cd* X) {
    cd a[64];
    std::memcpy(a, S, sizeof(cd) * n * n);
    for (int i = 0; i < n * n; ++i) X[i] = 0.0;
    for (int i = 0; i < n; ++i) X[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(a[r * n + c]) > std::abs(a[piv * n + c])) piv = r;
        if (std::abs(a[piv * n + c]) == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(a[c * n + k], a[piv * n + k]);
                std::swap(X[c * n + k], X[piv * n + k]);
            }
        cd inv = 1.0 / a[c * n + c];
        for (int k = 0; k < n; ++k) {
            a[c * n + k] *= inv;
            X[c * n + k] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            cd f = a[r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[r * n + k] -= f * a[c * n + k];
                X[r * n + k] -= f * X[c * n + k];
            }
        }
    }
    return true;
}

static double norm1(int n, const cd* A) {
    double best = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += std::abs(A[i * n + j]);
        best = std::max(best, s);
    }
    return best;
}

double eig_small(int n, const cd* B, cd* mu, cd* S, cd* Sinv) {
    cd T[64], Z[64];
    std::memcpy(T, B, sizeof(cd) * n * n);
    if (!schur_small(n, T, Z)) return -1.0;
    double scale = norm1(n, B);
    if (scale == 0.0) scale = 1.0;
    for (int k = 0; k < n; ++k) {
        mu[k] = T[k * n + k];
        cd y[8];
        for (int i = 0; i < n; ++i) y[i] = 0.0;
        y[k] = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            cd s = 0.0;
            for (int j = i + 1; j <= k; ++j) s += T[i * n + j] * y[j];
            cd den = T[i * n + i] - T[k * n + k];
            if (std::abs(den) < 1e-14 * scale) den = cd(1e-14 * scale, 0.0);  // defective: cond(S) will expose it
            y[i] = -s / den;
        }
        double nrm = 0.0;
        cd v[8];
        for (int r = 0; r < n; ++r) {
            v[r] = 0.0;
            for (int j = 0; j <= k; ++j) v[r] += Z[r * n + j] * y[j];
            nrm += std::norm(v[r]);
        }
        nrm = std::sqrt(nrm);
        for (int r = 0; r < n; ++r) S[r * n + k] = v[r] / nrm;
    }
    if (!invert_small(n, S, Sinv)) return 1e300;
    return norm1(n, S) * norm1(n, Sinv);
}

double freq_tables(int M, int L, double alpha, bool transposed, const double* Q,
                   const double* t, cd* mu, cd* Sinv, cd* P, double* cond) {
    (void)t;
    const int F = L / 2 + 1;
    double worst = 0.0;
    for (int f = 0; f < F; ++f) {
        // d_f of Lemma 1 (0-based f), r_f = d_f / (1 + d_f)
        cd d = -std::pow(alpha, 1.0 / L) * std::exp(cd(0.0, -2.0 * M_PI * f / L));
        cd r = d / (1.0 + d);
        // G_f^{-1} = I - r H_M  (H_M^T for the transposed system)
        cd Ginv[64], B[64], S[64];
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                double h = transposed ? (i == M - 1 ? 1.0 : 0.0) : (j == M - 1 ? 1.0 : 0.0);
                Ginv[i * M + j] = (i == j ? 1.0 : 0.0) - r * h;
            }
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                cd s = 0.0;
                for (int k = 0; k < M; ++k)
                    s += (transposed ? Q[k * M + i] : Q[i * M + k]) * Ginv[k * M + j];
                B[i * M + j] = s;
            }
        double c = eig_small(M, B, mu + f * M, S, Sinv + f * M * M);
        if (c < 0) return -1.0;
        if (cond) cond[f] = c;
        worst = std::max(worst, c);
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) {
                cd s = 0.0;
                for (int k = 0; k < M; ++k) s += Ginv[i * M + k] * S[k * M + j];
                P[(f * M + i) * M + j] = s;
            }
    }
    return worst;
}

// ---------------------------------------------------------------- stencils
// Standard finite-difference weights (exact on polynomials up to the degree
// the number of points allows), as integer numerators over a denominator,
// on consecutive offsets starting at lo.
namespace {
struct FdRow {
    int lo, den, n;
    int num[7];
};
// centred first derivative, order 2, 4, 6
const FdRow kCentralD1[3] = {{-1, 2, 3, {-1, 0, 1}},
                             {-2, 12, 5, {1, -8, 0, 8, -1}},
                             {-3, 60, 7, {-1, 9, -45, 0, 45, -9, 1}}};
// centred second derivative, order 2, 4, 6
const FdRow kCentralD2[3] = {{-1, 1, 3, {1, -2, 1}},
                             {-2, 12, 5, {-1, 16, -30, 16, -1}},
                             {-3, 180, 7, {2, -27, 270, -490, 270, -27, 2}}};
// upwind-biased first derivative for a positive velocity, order 1..5
const FdRow kUpwindD1[5] = {{-1, 1, 2, {-1, 1}},
                            {-2, 2, 3, {1, -4, 3}},
                            {-2, 6, 4, {1, -6, 3, 2}},
                            {-3, 12, 5, {-1, 6, -18, 10, 3}},
                            {-3, 60, 6, {-2, 15, -60, 20, 30, -3}}};

void put_row(const FdRow& r, double w[7], bool mirror) {
    for (int i = 0; i < 7; ++i) w[i] = 0.0;
    for (int j = 0; j < r.n; ++j) {
        const int o = r.lo + j;
        const double v = (double)r.num[j] / r.den;
        if (mirror) w[3 - o] = -v;   // w'(o) = -w(-o)
        else w[3 + o] = v;
    }
}

int support(const double w[7]) {
    int r = 0;
    for (int o = -3; o <= 3; ++o)
        if (w[o + 3] != 0.0) r = std::max(r, std::abs(o));
    return r;
}
}  // namespace

bool derivative_weights(int order, int upwind, double c, double d1[7], double d2[7]) {
    if (upwind) {
        if (order < 1 || order > 5) return false;
        put_row(kUpwindD1[order - 1], d1, c < 0.0);
        const int lap = order + (order & 1);
        put_row(kCentralD2[lap / 2 - 1], d2, false);
    } else {
        if (order != 2 && order != 4 && order != 6) return false;
        put_row(kCentralD1[order / 2 - 1], d1, false);
        put_row(kCentralD2[order / 2 - 1], d2, false);
    }
    return true;
}

bool problem_stencil(const ac_problem& prob, Stencil* st) {
    const int dim = prob.dim;
    double d1[7], d2[7];
    int rad = 1;
    for (int i = 0; i < 7; ++i) st->tx[i] = st->ty[i] = st->d1x[i] = st->d2x[i] = st->d1y[i] = st->d2y[i] = 0.0;
    const double hx = prob.lx / prob.nx;
    if (!derivative_weights(prob.order, prob.upwind, prob.cx, d1, d2)) return false;
    rad = std::max(rad, std::max(support(d1), support(d2)));
    for (int i = 0; i < 7; ++i) {
        st->d1x[i] = d1[i] / hx;
        st->d2x[i] = d2[i] / (hx * hx);
        st->tx[i] = prob.nu * st->d2x[i] - prob.cx * st->d1x[i];
    }
    if (dim == 2) {
        const double hy = prob.ly / prob.ny;
        if (!derivative_weights(prob.order, prob.upwind, prob.cy, d1, d2)) return false;
        rad = std::max(rad, std::max(support(d1), support(d2)));
        for (int i = 0; i < 7; ++i) {
            st->d1y[i] = d1[i] / hy;
            st->d2y[i] = d2[i] / (hy * hy);
            st->ty[i] = prob.nu * st->d2y[i] - prob.cy * st->d1y[i];
        }
    }
    st->rad = rad;
    return true;
}

void axis_symbol(int n, const double taps[7], cd* sigma) {
    for (int k = 0; k < n; ++k) {
        cd s = 0.0;
        for (int o = -3; o <= 3; ++o) {
            if (taps[o + 3] == 0.0) continue;
            long long ko = (((long long)k * o) % n + n) % n;  // k*o mod n, nonnegative
            double th = 2.0 * M_PI * (double)ko / n;
            s += taps[o + 3] * cd(std::cos(th), std::sin(th));
        }
        sigma[k] = s;
    }
}

void twiddles(int n, std::vector<cd>& tw) {
    tw.resize(n);
    for (int k = 0; k < n; ++k) tw[k] = std::exp(cd(0.0, -2.0 * M_PI * k / n));
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool fft_radices(int n, FftRadices* o) {
    static const int pref[6] = {8, 7, 5, 4, 3, 2};
    o->ns = 0;
    if (n < 1) return false;
    for (int i = 0; i < 6; ++i) {
        while (n % pref[i] == 0) {
            if (o->ns == 15) return false;
            o->r[o->ns++] = pref[i];
            n /= pref[i];
        }
    }
    return n == 1;
}

// shared memory per CTA of the single-pass cluster solve (rows, x and y
// tables, column twiddles), 0 if cs CTAs cannot hold a plane
static size_t cluster_bytes(int nx, int ny, int cs, size_t csz) {
    if (ny % cs || ny / cs < cs) return 0;
    const size_t m = (size_t)ny / cs;
    return csz * (m * nx + nx + 2 * m);
}

const char* plan_shape(const ac_problem& prob, int M, int L, int precision, int inner, int rad, int cluster_req,
                       PlanShape* o) {
    if (cluster_req != 0 && cluster_req != -1 && cluster_req != 4 && cluster_req != 8 && cluster_req != 16)
        return "cluster size must be 0 or -1 (three passes), 4, 8 or 16";
    const int nx = prob.nx, ny = prob.dim == 2 ? prob.ny : 1;
    const long long N = (long long)nx * ny;
    const size_t cs = precision == AC_C128 ? 16 : 8;   // bytes per complex of the transform
    *o = PlanShape{};
    o->rows_per_block = 1;
    o->cols_per_block = 1;
    if (inner == AC_INNER_FFT && (!is_pow2(nx) || !is_pow2(ny))) {
        // Mixed-radix Stockham transforms between two shared-memory buffers.
        if (!fft_radices(nx, &o->rx) || !fft_radices(ny, &o->ry))
            return "the FFT inner solver needs grid sizes whose prime factors are 2, 3, 5 and 7";
        const size_t limit = 200 * 1024;
        if (prob.dim == 1) {
            if (2 * (size_t)nx * cs > limit) return "1D grid too large for the one-CTA mixed-radix FFT solve";
            o->spatial_path = 5;
        } else {
            o->spatial_path = 6;
            // rows: about 64 KB per CTA (three CTAs per SM); columns: 8 (complex64)
            // or 4 (complex128) per CTA, fewer if a tile would not fit
            int rpb = (int)(65536 / (2 * (size_t)nx * cs));
            if (rpb < 1) rpb = 1;
            if (rpb > ny) rpb = ny;
            o->rows_per_block = rpb;
            int W = cs == 16 ? 4 : 8;
            if (W > nx) W = nx;
            while (W > 1 && (2 * (size_t)ny * W + W + ny) * cs > limit) W >>= 1;
            o->cols_per_block = W;
            if (2 * (size_t)nx * cs > limit || (2 * (size_t)ny * W + W + ny) * cs > limit)
                return "2D grid too large for the three-pass mixed-radix FFT solve";
        }
    } else if (inner == AC_INNER_FFT) {
        if (prob.dim == 1) {
            if ((size_t)nx * cs > 160 * 1024) return "1D grid too large for the one-CTA FFT solve";
            o->spatial_path = 0;
        } else if ((size_t)nx * ny * cs <= 160 * 1024) {
            o->spatial_path = 1;
        } else {
            o->spatial_path = 2;
            int rpb = (int)(32768 / ((size_t)nx * cs));
            if (rpb < 1) rpb = 1;
            while (rpb & (rpb - 1)) rpb &= rpb - 1;
            o->rows_per_block = rpb < ny ? rpb : ny;
            int W = (int)(128 / cs);
            if (W > nx) W = nx;
            o->cols_per_block = W;
            if ((size_t)nx * cs > 160 * 1024 || (size_t)ny * W * cs > 160 * 1024)
                return "2D grid too large for the three-pass FFT solve";
            if (cluster_req == 4 || cluster_req == 8 || cluster_req == 16) {
                const size_t b = cluster_bytes(nx, ny, cluster_req, cs);
                if (b == 0 || b > 200 * 1024) return "the requested cluster cannot hold a plane";
                o->spatial_path = 7;
                o->cluster = cluster_req;
            }
        }
    } else {
        o->spatial_path = inner == AC_INNER_GMRES ? 4 : 3;
        if (nx < 2 * rad + 1 || (prob.dim == 2 && ny < 2 * rad + 1)) return "grid smaller than the stencil";
    }
    // tile of the time kernels: P points, L*M*P reals of shared memory
    const size_t rsz = cs / 2;
    int P = 256;
    while (P > 2 && (size_t)L * M * P * rsz > 50 * 1024) P >>= 1;
    while (P > 16 && (N + P - 1) / P < 2 * 152) P >>= 1;
    if ((size_t)L * M * P * rsz > 200 * 1024) return "L*M too large for the shared-memory time transform";
    // The update kernel is latency-bound: smaller tiles while its grid has
    // fewer than three CTAs per SM (1D advection, 4096 points: 16 -> 8 points,
    // 18% faster); on larger grids halving the tile measured slower.
    int Pu = P;
    while (Pu > 8 && (N + Pu - 1) / Pu < 3 * 152) Pu >>= 1;
    // The residual kernel is FP64-bound.  In complex64 plans smaller tiles
    // (more CTAs) let its FP64 phase overlap better with the transform phases
    // of other CTAs: a quarter of tiles of 64 points and more (2D heat 256^2:
    // 64 -> 16 points, 6% faster than 64), half of tiles of 16 to 32 points
    // (1D advection: 16 -> 8, 3%); tiles under 8 points and complex128 plans
    // measured slower.
    o->P = precision != AC_C64 ? P : (P >= 64 ? P / 4 : (P >= 16 ? P / 2 : P));
    o->grid = (int)((N + o->P - 1) / o->P);
    o->P_upd = Pu;
    o->grid_upd = (int)((N + Pu - 1) / Pu);
    return nullptr;
}

bool alpha_tables(int M, int L, double dT, const double* Q, const double* t, double alpha, bool transposed,
                  double wscale, double space_scale, AlphaTables* o) {
    const int F = L / 2 + 1;
    o->qs.assign((size_t)L * M * M, 0.0);
    o->s.assign(L, 0.0);
    o->sinv.assign(L, 0.0);
    o->wnorm.assign(2 * (size_t)L, 0.f);
    for (int l = 0; l < L; ++l) {
        o->s[l] = (l == 0) ? 1.0 : std::pow(alpha, (double)l / L);
        o->sinv[l] = ((l == 0) ? 1.0 : std::pow(alpha, -(double)l / L)) / L * space_scale;
        const double w = 1048576.0 / (o->s[l] * wscale);   // 2^20: the kernels' norm prescale
        const float wh = (float)w;
        o->wnorm[2 * l] = wh;
        o->wnorm[2 * l + 1] = (float)(w - (double)wh);
        for (int m = 0; m < M; ++m)
            for (int j = 0; j < M; ++j)
                o->qs[((size_t)l * M + m) * M + j] = o->s[l] * dT * (transposed ? Q[j * M + m] : Q[m * M + j]);
    }
    o->mu_dT.assign((size_t)F * M, cd(0.0));
    o->Sinv.assign((size_t)F * M * M, cd(0.0));
    o->P.assign((size_t)F * M * M, cd(0.0));
    o->worst_cond = freq_tables(M, L, alpha, transposed, Q, t, o->mu_dT.data(), o->Sinv.data(), o->P.data(), nullptr);
    if (o->worst_cond < 0 || o->worst_cond > 1e10) return false;
    for (auto& v : o->mu_dT) v *= dT;
    return true;
}

}  // namespace ac

// ------------------------------------------------------------- C ABI (host)
extern "C" int ac_stencil_taps(const ac_problem* prob, double* tx, double* ty, int* rad) {
    if (!prob || !tx || !ty) return AC_ERR_INVALID_ARG;
    if ((prob->dim != 1 && prob->dim != 2) || prob->nx < 1 || (prob->dim == 2 && prob->ny < 1) ||
        !(prob->lx > 0) || (prob->dim == 2 && !(prob->ly > 0)))
        return AC_ERR_INVALID_ARG;
    ac::Stencil st;
    if (!ac::problem_stencil(*prob, &st)) return AC_ERR_INVALID_ARG;
    for (int i = 0; i < 7; ++i) {
        tx[i] = st.tx[i];
        ty[i] = st.ty[i];
    }
    if (rad) *rad = st.rad;
    return AC_OK;
}

extern "C" int ac_plan_shape(const ac_problem* prob, int M, int L, int precision, int inner,
                             const ac_alpha_schedule* sched, ac_plan_info* out) {
    if (!prob || !out) return AC_ERR_INVALID_ARG;
    if ((prob->dim != 1 && prob->dim != 2) || prob->nx < 2 || (prob->dim == 2 && prob->ny < 2) ||
        !(prob->lx > 0) || (prob->dim == 2 && !(prob->ly > 0)))
        return AC_ERR_INVALID_ARG;
    if (M < 1 || M > 4 || L < 2 || L > 1024 || (L & (L - 1))) return AC_ERR_INVALID_ARG;
    if (precision != AC_C128 && precision != AC_C64) return AC_ERR_INVALID_ARG;
    if (inner != AC_INNER_FFT && inner != AC_INNER_BICGSTAB && inner != AC_INNER_GMRES) return AC_ERR_INVALID_ARG;
    ac::Stencil st;
    if (!ac::problem_stencil(*prob, &st)) return AC_ERR_INVALID_ARG;
    ac::PlanShape sh;
    if (ac::plan_shape(*prob, M, L, precision, inner, st.rad, sched ? sched->space_cluster : 0, &sh))
        return AC_ERR_INVALID_ARG;
    *out = ac_plan_info{};
    out->N = prob->nx * (prob->dim == 2 ? prob->ny : 1);
    out->M = M;
    out->L = L;
    out->F = L / 2 + 1;
    out->tile_fwd = sh.P;
    out->tile_upd = sh.P_upd;
    out->spatial_path = sh.spatial_path;
    out->space_cluster = sh.spatial_path == 7 ? sh.cluster : 0;
    return AC_OK;
}

extern "C" int ac_radau_nodes(int M, double* t) {
    if (!t) return AC_ERR_INVALID_ARG;
    return ac::radau_nodes(M, t) ? AC_OK : AC_ERR_INVALID_ARG;
}

extern "C" int ac_collocation_matrix(int M, double* Q) {
    double t[8];
    if (!Q || !ac::radau_nodes(M, t)) return AC_ERR_INVALID_ARG;
    return ac::collocation_matrix(M, t, Q) ? AC_OK : AC_ERR_INVALID_ARG;
}

extern "C" int ac_freq_tables(int M, int L, double alpha, int transposed, double* mu,
                              double* Sinv, double* P, double* cond) {
    if (M < 1 || M > 8 || L < 1 || !(alpha > 0.0) || !(alpha < 1.0) || !mu || !Sinv || !P)
        return AC_ERR_INVALID_ARG;
    double t[8], Q[64];
    ac::radau_nodes(M, t);
    ac::collocation_matrix(M, t, Q);
    const int F = L / 2 + 1;
    std::vector<ac::cd> vmu(F * M), vS(F * M * M), vP(F * M * M);
    double worst = ac::freq_tables(M, L, alpha, transposed != 0, Q, t, vmu.data(), vS.data(),
                                   vP.data(), cond);
    std::memcpy(mu, vmu.data(), sizeof(double) * 2 * F * M);
    std::memcpy(Sinv, vS.data(), sizeof(double) * 2 * F * M * M);
    std::memcpy(P, vP.data(), sizeof(double) * 2 * F * M * M);
    if (worst < 0 || worst > 1e10) return AC_ERR_NOT_DIAGONALIZABLE;
    return AC_OK;
}

extern "C" int ac_alpha_sequence(double m0, double gamma, int n, double* alphas, double* ms) {
    if (!(m0 > 0) || !(gamma > 0) || n < 0 || !alphas || !ms) return AC_ERR_INVALID_ARG;
    double m = m0;
    ms[0] = m0;
    for (int k = 0; k < n; ++k) {
        alphas[k] = std::sqrt(gamma / m);   // alpha_{k+1} = sqrt(gamma / m_k)
        m = 2.0 * std::sqrt(m * gamma);     // m_{k+1} = 2 sqrt(m_k gamma)
        ms[k + 1] = m;
    }
    return AC_OK;
}
