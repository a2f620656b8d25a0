// A preconditioner solve that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a solve:
// for example code whose whole device memory has been handed to another
// framework's caching allocator (so cudaMalloc would fail or fragment that
// pool), or a latency-critical loop in which the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  Such callers
// cannot build an ac_plan, because ac_setup allocates its workspace.
// ac_precond_solve_noalloc gives them e = C_alpha^{-1} r with every piece of
// working memory -- the complex F*M*N transform buffer, the twiddle, symbol
// and eigenbasis tables and the block partial sums -- carved out of one
// file-scope device array of fixed size.  It runs the same kernels as
// ac_precond_solve.
//
// The array lives in every GPU that loads the library until the process
// exits.  All calls on a device share it: two calls whose GPU work overlaps
// (different streams, or different host threads) race on it, so callers must
// order them.  Nothing in it has to start at zero: every call rewrites all of
// the regions it reads.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "alphacirc.h"
#include "kernels.h"
#include "planner.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
    std::once_flag once;
    void* ptr = nullptr;
    cudaError_t err = cudaSuccess;
};
DeviceScratch g_dev[kMaxDevices];

}  // namespace

// message for ac_last_error(), kept by the C ABI layer
void ac_internal_set_error(const char* msg);

namespace {

int nfail(int code, const char* msg) {
    std::string m = std::string("ac_precond_solve_noalloc: ") + msg;
    ac_internal_set_error(m.c_str());
    return code;
}

// Device address of the scratch array on the current device.  Host code must
// not pass g_scratch itself to a kernel: on the host that name is only a
// stand-in.  The address is looked up once per device, with that device
// current.
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nfail(AC_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return nfail(AC_ERR_INVALID_ARG, "device ordinal out of range");
    DeviceScratch& d = g_dev[dev];
    std::call_once(d.once, [&d]() { d.err = cudaGetSymbolAddress(&d.ptr, g_scratch); });
    if (d.err != cudaSuccess || !d.ptr) return nfail(AC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    *out = static_cast<unsigned char*>(d.ptr);
    return AC_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// host complex table -> device, in the transform precision
cudaError_t put_c(void* dst, const std::vector<ac::cd>& v, bool dbl, cudaStream_t st) {
    if (dbl) return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(ac::cd), cudaMemcpyHostToDevice, st);
    std::vector<float> f(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        f[2 * i] = (float)v[i].real();
        f[2 * i + 1] = (float)v[i].imag();
    }
    return cudaMemcpyAsync(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, st);
}

template <typename R>
int run(const ac_problem* prob, int M, int L, double dT, double alpha, const double* r, double* e,
        cudaStream_t st) {
    const bool dbl = sizeof(R) == 8;
    const int precision = dbl ? AC_C128 : AC_C64;
    const size_t cs = 2 * sizeof(R);
    const int nx = prob->nx, ny = prob->dim == 2 ? prob->ny : 1;
    const long long N = (long long)nx * ny;
    const int F = L / 2 + 1;

    ac::Stencil sten;
    if (!ac::problem_stencil(*prob, &sten)) return nfail(AC_ERR_INVALID_ARG, "unsupported stencil");
    // spatial path and kernel tiles: the ones ac_setup chooses for this problem
    ac::PlanShape sh;
    if (const char* why = ac::plan_shape(*prob, M, L, precision, AC_INNER_FFT, sten.rad, 0, &sh))
        return nfail(AC_ERR_INVALID_ARG, why);

    // carve the scratch array
    size_t off = 0;
    auto take = [&off](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t oX = take((size_t)F * M * N * cs);
    const size_t otwL = take((size_t)L * cs), otwx = take((size_t)nx * cs), otwy = take((size_t)ny * cs);
    const size_t osx = take((size_t)nx * cs), osy = take((size_t)ny * cs);
    const size_t oqs = take(sizeof(double) * (size_t)L * M * M), os = take(sizeof(double) * L);
    const size_t own = take(2 * sizeof(float) * L), osinv = take(sizeof(double) * L);
    const size_t oSinv = take((size_t)F * M * M * cs), oP = take((size_t)F * M * M * cs);
    const size_t omu = take((size_t)F * M * cs);
    const size_t opf = take(sizeof(double) * sh.grid), opu = take(sizeof(double) * sh.grid_upd);
    if (off > kScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "problem needs %.1f MiB of scratch; the fixed no-allocation scratch holds %zu MiB "
                      "(use ac_setup + ac_precond_solve instead)",
                      off / 1048576.0, kScratchBytes >> 20);
        return nfail(AC_ERR_INVALID_ARG, msg);
    }
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;

    // host tables: Radau IIA data, twiddles, stencil symbols and the
    // alpha-dependent tables, from the same routines as ac_setup
    double t[8], Q[64];
    ac::radau_nodes(M, t);
    ac::collocation_matrix(M, t, Q);
    std::vector<ac::cd> twL, twx, twy, sx(nx), sy(ny, ac::cd(0.0));
    ac::twiddles(L, twL);
    ac::twiddles(nx, twx);
    ac::twiddles(ny, twy);
    ac::axis_symbol(nx, sten.tx, sx.data());
    if (prob->dim == 2) ac::axis_symbol(ny, sten.ty, sy.data());
    ac::AlphaTables T;
    if (!ac::alpha_tables(M, L, dT, Q, t, alpha, false, 1.0, 1.0 / (double)N, &T))
        return nfail(AC_ERR_NOT_DIAGONALIZABLE, "Q G_l^{-1} not diagonalisable");

    cudaError_t ce = cudaSuccess;
    auto chk = [&ce](cudaError_t x) {
        if (ce == cudaSuccess) ce = x;
    };
    chk(put_c(base + otwL, twL, dbl, st));
    chk(put_c(base + otwx, twx, dbl, st));
    chk(put_c(base + otwy, twy, dbl, st));
    chk(put_c(base + osx, sx, dbl, st));
    chk(put_c(base + osy, sy, dbl, st));
    chk(cudaMemcpyAsync(base + oqs, T.qs.data(), T.qs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(base + os, T.s.data(), T.s.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(base + own, T.wnorm.data(), T.wnorm.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    chk(cudaMemcpyAsync(base + osinv, T.sinv.data(), T.sinv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    chk(put_c(base + oSinv, T.Sinv, dbl, st));
    chk(put_c(base + oP, T.P, dbl, st));
    chk(put_c(base + omu, T.mu_dT, dbl, st));
    if (ce != cudaSuccess) return nfail(AC_ERR_CUDA, cudaGetErrorString(ce));

    ac::Grid g;
    g.dim = prob->dim;
    g.nx = nx;
    g.ny = ny;
    g.N = (int)N;
    g.rad = sten.rad;
    for (int i = 0; i < 7; ++i) {
        g.tx[i] = sten.tx[i];
        g.ty[i] = sten.ty[i];
    }
    g.c0 = sten.tx[3] + sten.ty[3];

    ac::FwdArgs fa{};
    fa.g = g;
    fa.M = M;
    fa.L = L;
    fa.logL = log2i(L);
    fa.F = F;
    fa.P = sh.P;
    fa.u = nullptr;
    fa.u0 = nullptr;
    fa.b = r;
    fa.b_reversed = 0;
    fa.transposed = 0;
    fa.qs = reinterpret_cast<const double*>(base + oqs);
    fa.s = reinterpret_cast<const double*>(base + os);
    fa.wnorm = reinterpret_cast<const float2*>(base + own);
    fa.tw = base + otwL;
    fa.Sinv = base + oSinv;
    fa.X = base + oX;
    fa.part = reinterpret_cast<double*>(base + opf);
    chk(ac::launch_fwd<R>(fa, sh.grid, (size_t)L * M * sh.P * sizeof(R), st));

    ac::SpaceArgs sa{};
    sa.nx = nx;
    sa.ny = ny;
    sa.lognx = log2i(nx);
    sa.logny = log2i(ny);
    sa.planes = F * M;
    sa.M = M;
    sa.X = base + oX;
    sa.mu_dT = base + omu;
    sa.sig_x = base + osx;
    sa.sig_y = base + osy;
    sa.tw_x = base + otwx;
    sa.tw_y = base + otwy;
    sa.rows_per_block = sh.rows_per_block;
    sa.cols_per_block = sh.cols_per_block;
    sa.rx = sh.rx;
    sa.ry = sh.ry;
    sa.cluster = sh.cluster;
    if (sh.spatial_path == 7) {
        // as ac_setup: the three passes where the device cannot hold the clusters
        int fits = 0;
        if (ac::launch_space_cluster<R>(sa, st, &fits) != cudaSuccess || fits < 1) {
            (void)cudaGetLastError();
            sh.spatial_path = 2;
        }
    }
    if (sh.spatial_path == 0) chk(ac::launch_space_1d<R>(sa, st));
    else if (sh.spatial_path == 1) chk(ac::launch_space_2d_small<R>(sa, st));
    else if (sh.spatial_path == 2) {
        chk(ac::launch_space_rows<R>(sa, 0, st));
        chk(ac::launch_space_cols<R>(sa, st));
        chk(ac::launch_space_rows<R>(sa, 1, st));
    } else if (sh.spatial_path == 7) {
        chk(ac::launch_space_cluster<R>(sa, st, nullptr));
    } else if (sh.spatial_path == 5) {
        chk(ac::launch_space_mr_1d<R>(sa, st));
    } else {
        chk(ac::launch_space_mr_rows<R>(sa, 0, st));
        chk(ac::launch_space_mr_cols<R>(sa, st));
        chk(ac::launch_space_mr_rows<R>(sa, 1, st));
    }

    ac::UpdArgs ua{};
    ua.N = (int)N;
    ua.M = M;
    ua.L = L;
    ua.logL = log2i(L);
    ua.F = F;
    ua.P = sh.P_upd;
    ua.X = base + oX;
    ua.Pm = base + oP;
    ua.tw = base + otwL;
    ua.sinv = reinterpret_cast<const double*>(base + osinv);
    ua.out = e;
    ua.accumulate = 0;
    ua.part = reinterpret_cast<double*>(base + opu);
    chk(ac::launch_upd<R>(ua, sh.grid_upd, (size_t)L * M * sh.P * sizeof(R), st));
    if (ce != cudaSuccess) return nfail(AC_ERR_CUDA, cudaGetErrorString(ce));
    return AC_OK;
}

}  // namespace

extern "C" int ac_precond_solve_noalloc(const ac_problem* prob, int M, int L, double dT, double alpha,
                                        int precision, const double* r, double* e, void* stream) {
    if (!prob || !r || !e) return nfail(AC_ERR_INVALID_ARG, "null argument");
    if (prob->dim != 1 && prob->dim != 2) return nfail(AC_ERR_INVALID_ARG, "dim must be 1 or 2");
    if (prob->upwind ? (prob->order < 1 || prob->order > 5) : (prob->order != 2 && prob->order != 4 && prob->order != 6))
        return nfail(AC_ERR_INVALID_ARG, "order must be 2, 4 or 6 (centred) or 1..5 (upwind)");
    const int ny = prob->dim == 2 ? prob->ny : 1;
    if (prob->nx < 2 || (prob->dim == 2 && ny < 2))
        return nfail(AC_ERR_INVALID_ARG, "grid sizes must be >= 2");
    if (M < 1 || M > 4) return nfail(AC_ERR_INVALID_ARG, "M must be 1..4");
    if (!pow2(L) || L < 2 || L > 1024) return nfail(AC_ERR_INVALID_ARG, "L must be a power of two in 2..1024");
    if (!(dT > 0)) return nfail(AC_ERR_INVALID_ARG, "dT must be positive");
    if (!(alpha > 0.0) || !(alpha < 1.0)) return nfail(AC_ERR_INVALID_ARG, "alpha must be in (0,1)");
    if (!(prob->lx > 0) || (prob->dim == 2 && !(prob->ly > 0))) return nfail(AC_ERR_INVALID_ARG, "bad box length");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == AC_C128) return run<double>(prob, M, L, dT, alpha, r, e, st);
    if (precision == AC_C64) return run<float>(prob, M, L, dT, alpha, r, e, st);
    return nfail(AC_ERR_INVALID_ARG, "bad precision");
}
