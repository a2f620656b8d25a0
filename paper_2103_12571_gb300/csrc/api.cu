// C ABI of the alpha-circulant Richardson solver: plan set-up, table
// management and the launch sequences of Algorithm 1 (one iteration), the
// Richardson loop with the alpha rules of Sec. 3.3 / Algorithm 2, the adjoint
// solve and the gradient contractions.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "alphacirc.h"
#include "kernels.h"
#include "norm2.cuh"
#include "planner.h"

namespace ac {
cudaError_t launch_wnorms(const double* u0, const double* b, int L, int M, long long N, double* part,
                          int grid, cudaStream_t st);
cudaError_t launch_fill_stack(const double* u0, double* u, int L, int M, long long N, cudaStream_t st);
cudaError_t launch_a_inf(const Grid& g, const double* u0, double* part, int grid, cudaStream_t st);
cudaError_t launch_colloc_rhs(const double* b, const double* dtQ, double* v, int L, int M, long long N,
                              cudaStream_t st);
cudaError_t launch_dfma_rate(const double* ab, int rounds, double* sink, int grid, cudaStream_t st);
}

using ac::cd;

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// lets the allocation-free entry point (noalloc.cu) report through ac_last_error
void ac_internal_set_error(const char* msg) { g_err = msg; }

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(AC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                                  \
    } while (0)

// Profiler kinds.  KK_SPACE_ROWS / KK_SPACE_COLS time the launches of the
// three-pass 2D spatial solve one by one (inside the KK_SPACE group).
enum KernelKind { KK_FWD = 0, KK_SPACE, KK_UPD, KK_APPLY, KK_GRAD, KK_AUX, KK_SPACE_ROWS, KK_SPACE_COLS, KK_COUNT };
static const char* kKindNames[KK_COUNT] = {"resid_tfft_mix", "spatial_solve", "mix_tifft_update",
                                           "apply_C", "grad_contract", "aux", "space_rows", "space_cols"};

struct EventPair {
    int kind;
    cudaEvent_t a, b;
};

// most chunks of ac_richardson_step_host's copy/compute pipeline
static const int kHostChunks = 32;

struct ac_plan {
    ac_problem prob;
    int M, L, logL, F, N, P, grid;
    int P_upd, grid_upd;   // tile of the update kernel
    double dT;
    ac_alpha_schedule sched;
    int precision, inner, device;
    int spatial_path;
    int rows_per_block, cols_per_block;
    ac::FftRadices rx, ry;   // radix plans of the mixed-radix FFT paths (5, 6)
    int cluster;             // path 7: CTAs per cluster
    size_t csize;  // bytes per complex of the transform type
    // host data
    double t[8], Q[64];
    ac::Grid grid_fwd, grid_adj;  // A and A^T
    double d1x[7], d2x[7], d1y[7], d2y[7];   // derivative weights / h, / h^2 on offsets -3..3
    // device buffers
    void* X = nullptr;
    void* tw_L = nullptr;
    void* tw_x = nullptr;
    void* tw_y = nullptr;
    void* sig_x = nullptr;   // A
    void* sig_y = nullptr;
    void* sigT_x = nullptr;  // A^T
    void* sigT_y = nullptr;
    double* d_qs = nullptr;
    double* d_s = nullptr;
    float2* d_wnorm = nullptr;   // [L] 2^20 / (s_l w_scale) as float pairs (residual norm)
    double* d_sinv = nullptr;
    void* d_Sinv = nullptr;
    void* d_P = nullptr;
    void* d_mu = nullptr;
    double* d_part_fwd = nullptr;
    double* d_part_upd = nullptr;
    double* d_part_d = nullptr;  // FP64 reductions
    double* d_dtQ = nullptr;     // dT Q
    double* d_dtQT = nullptr;    // dT Q^T
    void* d_bicg = nullptr;      // Krylov vectors when they do not fit in shared memory
    double2* d_mu64 = nullptr;   // complex64 BiCGStab: dT mu in FP64 (reliable updates)
    double2* d_x64 = nullptr;    // complex64 BiCGStab: FP64 solution accumulators, F*M*N
    // TMA-staged update kernel (complex64 plans, correction form)
    bool tma_ok = false;
    int tma_P = 0, tma_grid = 0;
    ac::UpdTmaGeom tgeo{};
    CUtensorMap mapX{};                  // X as [F*M rows][2N floats]
    CUtensorMap mapU{};                  // the last u as [L*M rows][N doubles]
    const void* mapU_ptr = nullptr;
    int* d_err = nullptr;                // set by a kernel whose bounded wait timed out
    int upd_grid_used = 0;               // partial results written by the last update launch
    int* d_iters = nullptr;      // Krylov iterations per system
    int* h_iters = nullptr;      // pinned copy
    double* h_part_fwd = nullptr;  // pinned
    double* h_part_upd = nullptr;
    double* h_part_d = nullptr;
    int part_d_len = 0;
    // table cache key
    double cur_alpha = -1.0;
    int cur_transposed = -1;
    double cur_wscale = -1.0;
    long long workspace = 0;
    long long launches = 0;
    cudaEvent_t ev_res = nullptr;
    // ac_richardson_step_host: device copies of the host arrays, copy streams
    // and the events that order copies and kernels (created on first use)
    double* d_hu = nullptr;
    double* d_hu0 = nullptr;
    double* d_hb = nullptr;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kHostChunks] = {};
    cudaEvent_t ev_out[kHostChunks + 4] = {};
    cudaEvent_t ev_start = nullptr, ev_u0 = nullptr, ev_done = nullptr;
    // sequential stepping by diagonalisation of Q (ac_sequential_solve)
    double* d_seq_S = nullptr;      // [M][M] complex S, Q = S diag(lambda) S^{-1}
    double* d_seq_Sinv = nullptr;   // [M][M] complex S^{-1}
    void* d_seq_mu = nullptr;       // [M] complex dT * lambda_m, transform precision
    cudaStream_t seq_capture = nullptr;
    cudaGraphExec_t seq_exec = nullptr;
    const void* seq_key[3] = {nullptr, nullptr, nullptr};
    long long seq_launches = 0;     // kernels per replay of the graph
    // outer flexible GMRES (ac_krylov_solve)
    double* d_kry = nullptr;        // 2m + 2 space-time vectors
    int kry_m = 0;
    double* d_kpart = nullptr;      // [8][krylov_grid] partial dot products
    double* h_kpart = nullptr;      // pinned copy
    // profiling
    bool prof = false;
    std::vector<EventPair> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[KK_COUNT] = {0};
    long long prof_count[KK_COUNT] = {0};
};

// ----------------------------------------------------------------- helpers
static cudaEvent_t get_event(ac_plan* p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    ac_plan* p;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(ac_plan* p_, int k, cudaStream_t s) : p(p_), kind(k), st(s) {
        if (p->prof && kind >= 0) {
            a = get_event(p);
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (p->prof && a) {
            cudaEvent_t b = get_event(p);
            cudaEventRecord(b, st);
            p->pending.push_back({kind, a, b});
        }
    }
};

static void drain_profile(ac_plan* p) {
    for (auto& e : p->pending) {
        cudaEventSynchronize(e.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.a, e.b);
        p->prof_ms[e.kind] += ms;
        p->prof_count[e.kind] += 1;
        p->pool.push_back(e.a);
        p->pool.push_back(e.b);
    }
    p->pending.clear();
}

template <typename T>
static cudaError_t dalloc(ac_plan* p, T** ptr, size_t bytes) {
    p->workspace += (long long)bytes;
    return cudaMalloc((void**)ptr, bytes);
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Upload a complex table in the transform precision.
static cudaError_t upload_c(const ac_plan* p, void* dst, const cd* src, size_t n, cudaStream_t st) {
    if (p->precision == AC_C128) {
        return cudaMemcpyAsync(dst, src, n * sizeof(cd), cudaMemcpyHostToDevice, st);
    }
    std::vector<float> tmp(2 * n);
    for (size_t i = 0; i < n; ++i) {
        tmp[2 * i] = (float)src[i].real();
        tmp[2 * i + 1] = (float)src[i].imag();
    }
    return cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice, st);
}

// The spatial FFT solves return N times the solution (unnormalised inverse
// transforms); the back transforms after them absorb 1/N.
static bool krylov_path(const ac_plan* p) { return p->spatial_path == 3 || p->spatial_path == 4; }
static double space_scale(const ac_plan* p) { return krylov_path(p) ? 1.0 : 1.0 / (double)p->N; }

// Alpha-dependent tables (ac::alpha_tables): qs, s, the residual-norm
// weights, sinv (FP64 / float pairs) and the per-frequency Sinv, P, dT mu
// (transform precision).
static int ensure_tables(ac_plan* p, double alpha, int transposed, double wscale, cudaStream_t st) {
    if (alpha == p->cur_alpha && transposed == p->cur_transposed && wscale == p->cur_wscale) return AC_OK;
    if (!(alpha > 0.0) || !(alpha < 1.0)) return fail(AC_ERR_INVALID_ARG, "alpha must be in (0,1), got %g", alpha);
    ac::AlphaTables T;
    if (!ac::alpha_tables(p->M, p->L, p->dT, p->Q, p->t, alpha, transposed != 0, wscale, space_scale(p), &T))
        return fail(AC_ERR_NOT_DIAGONALIZABLE, "Q G_l^{-1} not diagonalisable for alpha=%g (cond %g)", alpha,
                    T.worst_cond);
    CK(cudaMemcpyAsync(p->d_qs, T.qs.data(), T.qs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->d_s, T.s.data(), T.s.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->d_sinv, T.sinv.data(), T.sinv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->d_wnorm, T.wnorm.data(), T.wnorm.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(upload_c(p, p->d_Sinv, T.Sinv.data(), T.Sinv.size(), st));
    CK(upload_c(p, p->d_P, T.P.data(), T.P.size(), st));
    CK(upload_c(p, p->d_mu, T.mu_dT.data(), T.mu_dT.size(), st));
    if (p->d_mu64)
        CK(cudaMemcpyAsync(p->d_mu64, T.mu_dT.data(), T.mu_dT.size() * sizeof(cd), cudaMemcpyHostToDevice, st));
    p->cur_alpha = alpha;
    p->cur_transposed = transposed;
    p->cur_wscale = wscale;
    return AC_OK;
}

// Relative tolerance of the BiCGStab inner solves: the schedule's tau (1e-8
// if unset), floored at 2^-20 in the complex64 form, where FP32 arithmetic
// cannot certify a smaller relative residual.
static int gmres_restart(const ac_plan* p) {
    const int m = p->sched.inner_restart > 0 ? p->sched.inner_restart : 30;
    return std::min(m, 32);
}

static double inner_tau(const ac_plan* p, bool reliable = false) {
    double tau = p->sched.tau > 0 ? p->sched.tau : 1e-8;
    if (p->precision == AC_C64 && !reliable) tau = std::max(tau, std::ldexp(1.0, -20));
    return tau;
}

// complex64 BiCGStab inside the preconditioner runs with FP64 reliable
// updates and honours tau below the FP32 floor
static bool bicg_reliable(const ac_plan* p) { return p->spatial_path == 3 && p->d_mu64 && p->d_x64; }

// The shifted spatial solves of eq. (d2), (I - mu dT A) x = X_plane, in place
// on `planes` planes of N complex values with per-plane shifts mu_dT, by the
// plan's inner solver.  fetch_iters: copy the Krylov iteration counts to the
// host (a stream-ordered copy; off inside graph capture).
static ac::SpaceArgs space_args(const ac_plan* p, void* X, const void* mu_dT, int planes, int transposed) {
    ac::SpaceArgs sa{};
    sa.nx = p->prob.nx;
    sa.ny = p->prob.dim == 2 ? p->prob.ny : 1;
    sa.lognx = ilog2(sa.nx);
    sa.logny = ilog2(sa.ny);
    sa.planes = planes;
    sa.M = p->M;
    sa.X = X;
    sa.mu_dT = mu_dT;
    sa.sig_x = transposed ? p->sigT_x : p->sig_x;
    sa.sig_y = transposed ? p->sigT_y : p->sig_y;
    sa.tw_x = p->tw_x;
    sa.tw_y = p->tw_y;
    sa.rows_per_block = p->rows_per_block;
    sa.cols_per_block = p->cols_per_block;
    sa.rx = p->rx;
    sa.ry = p->ry;
    sa.cluster = p->cluster;
    return sa;
}

template <typename R>
static int run_spatial(ac_plan* p, void* X, const void* mu_dT, int planes, int transposed, bool fetch_iters,
                       cudaStream_t st, bool prof_passes = false) {
    const ac::SpaceArgs sa = space_args(p, X, mu_dT, planes, transposed);
    if (p->spatial_path == 0) {
        CK(ac::launch_space_1d<R>(sa, st));
        p->launches++;
    } else if (p->spatial_path == 1) {
        CK(ac::launch_space_2d_small<R>(sa, st));
        p->launches++;
    } else if (p->spatial_path == 2) {
        const bool pp = prof_passes && p->prof;
        {
            ProfScope ps(p, pp ? KK_SPACE_ROWS : -1, st);
            CK(ac::launch_space_rows<R>(sa, 0, st));
        }
        {
            ProfScope ps(p, pp ? KK_SPACE_COLS : -1, st);
            CK(ac::launch_space_cols<R>(sa, st));
        }
        {
            ProfScope ps(p, pp ? KK_SPACE_ROWS : -1, st);
            CK(ac::launch_space_rows<R>(sa, 1, st));
        }
        p->launches += 3;
    } else if (p->spatial_path == 7) {
        CK(ac::launch_space_cluster<R>(sa, st, nullptr));
        p->launches++;
    } else if (p->spatial_path == 5) {
        CK(ac::launch_space_mr_1d<R>(sa, st));
        p->launches++;
    } else if (p->spatial_path == 6) {
        const bool pp = prof_passes && p->prof;
        {
            ProfScope ps(p, pp ? KK_SPACE_ROWS : -1, st);
            CK(ac::launch_space_mr_rows<R>(sa, 0, st));
        }
        {
            ProfScope ps(p, pp ? KK_SPACE_COLS : -1, st);
            CK(ac::launch_space_mr_cols<R>(sa, st));
        }
        {
            ProfScope ps(p, pp ? KK_SPACE_ROWS : -1, st);
            CK(ac::launch_space_mr_rows<R>(sa, 1, st));
        }
        p->launches += 3;
    } else if (p->spatial_path == 3) {
        ac::BicgArgs ba{};
        ba.g = transposed ? p->grid_adj : p->grid_fwd;
        ba.planes = planes;
        ba.M = p->M;
        ba.max_iter = p->sched.inner_max_iter > 0 ? p->sched.inner_max_iter : 4000;
        const bool rel = bicg_reliable(p) && mu_dT == p->d_mu;
        ba.tau = inner_tau(p, rel);
        ba.X = X;
        ba.mu_dT = mu_dT;
        ba.iters = p->d_iters;
        ba.mu64 = rel ? p->d_mu64 : nullptr;
        ba.x64 = rel ? p->d_x64 : nullptr;
        CK(ac::launch_bicgstab<R>(ba, p->d_bicg, st));
        p->launches++;
        if (fetch_iters)
            CK(cudaMemcpyAsync(p->h_iters, p->d_iters, sizeof(int) * planes, cudaMemcpyDeviceToHost, st));
    } else if (p->spatial_path == 4) {
        ac::GmresArgs ga{};
        ga.g = transposed ? p->grid_adj : p->grid_fwd;
        ga.planes = planes;
        ga.M = p->M;
        ga.max_iter = p->sched.inner_max_iter > 0 ? p->sched.inner_max_iter : 4000;
        ga.restart = gmres_restart(p);
        ga.tau = inner_tau(p);
        ga.X = X;
        ga.mu_dT = mu_dT;
        ga.iters = p->d_iters;
        CK(ac::launch_gmres<R>(ga, p->d_bicg, st));
        p->launches++;
        if (fetch_iters)
            CK(cudaMemcpyAsync(p->h_iters, p->d_iters, sizeof(int) * planes, cudaMemcpyDeviceToHost, st));
    } else {
        return fail(AC_ERR_INVALID_ARG, "inner solver path %d not available", p->spatial_path);
    }
    return AC_OK;
}

// ----------------------------------------------------- TMA tensor maps
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// 2D tensor map over rows x inner elements (row stride inner * esize bytes)
// with boxes of box_rows x box_inner elements, no swizzle, zero fill.
static bool encode_2d(CUtensorMap* m, CUtensorMapDataType dt, size_t esize, const void* base, uint64_t inner,
                      uint64_t rows, uint32_t box_inner, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * esize};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t round128(size_t v) { return (v + 127) & ~size_t(127); }

// Tile geometry of the TMA-staged update kernel for tiles of P points: the
// X rows (F*M) and u rows (L*M) of a tile in boxes of at most 256 rows, two
// buffers of each and the transform buffer within 113 KB (two CTAs per SM).
static bool tma_geometry(const ac_plan* p, int P, ac::UpdTmaGeom* g) {
    const int FM = p->F * p->M, LM = p->L * p->M;
    if (P < 8 || P > 128 || p->N % P != 0 || (p->N & 1)) return false;
    g->ntiles = p->N / P;
    g->xboxes = (FM + 255) / 256;
    g->xrows = (FM + g->xboxes - 1) / g->xboxes;
    g->uboxes = (LM + 255) / 256;
    g->urows = (LM + g->uboxes - 1) / g->uboxes;
    const size_t xb = (size_t)g->xboxes * g->xrows * P * sizeof(float2);
    const size_t ub = (size_t)g->uboxes * g->urows * P * sizeof(double);
    g->tile_bytes = (unsigned)(xb + ub);
    g->xbuf = (unsigned)round128(xb);
    g->ubuf = (unsigned)round128(ub);
    g->zbuf = (unsigned)round128((size_t)LM * (P / 2) * sizeof(float2));
    return 2 * ((size_t)g->xbuf + g->ubuf) + g->zbuf <= 113 * 1024;
}

// On request (AC_UPDATE_TMA), chooses the TMA tile (the largest that fits)
// and encodes the map of X; leaves tma_ok false when the kernel does not
// apply.  Not the default: on the 2D heat workloads it measured slower than
// the plain update kernel (256^2, L = 64: 87-118 us against 74-76 us; 128^2,
// L = 32: 18-27 us against 16.3 us), whose four CTAs per SM hide the global
// latency as well as the staged double buffers of two.
static void setup_tma(ac_plan* p) {
    p->tma_ok = false;
    if (p->precision != AC_C64 || p->sched.update_kernel != AC_UPDATE_TMA) return;
    for (int P = 64; P >= 8; P >>= 1) {
        ac::UpdTmaGeom g{};
        if (!tma_geometry(p, P, &g)) continue;
        g.err = p->d_err;
        const int per_sm = ac::upd_tma_ctas_per_sm(p->M, g);
        int dev = 0, sms = 0;
        if (per_sm < 1 || cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return;
        if (!encode_2d(&p->mapX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), p->X, 2 * (uint64_t)p->N,
                       (uint64_t)p->F * p->M, (uint32_t)(2 * P), (uint32_t)g.xrows))
            return;
        p->tgeo = g;
        p->tma_P = P;
        p->tma_grid = std::min(g.ntiles, per_sm * sms);
        p->tma_ok = true;
        return;
    }
}

// ------------------------------------------------------ one preconditioner
// out (+)= C_alpha^{-1} (w - C u)   [u may be null: out (+)= C_alpha^{-1} w]
static ac::FwdArgs fwd_args(const ac_plan* p, const double* u, const double* u0, const double* b, int b_rev,
                           int transposed, int recompute) {
    ac::FwdArgs fa{};
    fa.g = transposed ? p->grid_adj : p->grid_fwd;
    fa.M = p->M;
    fa.L = p->L;
    fa.logL = p->logL;
    fa.F = p->F;
    fa.P = p->P;
    fa.u = u;
    fa.u0 = u0;
    fa.b = b;
    fa.b_reversed = b_rev;
    fa.transposed = transposed;
    fa.recompute = recompute;
    fa.alpha = p->cur_alpha;
    fa.qs = p->d_qs;
    fa.s = p->d_s;
    fa.wnorm = p->d_wnorm;
    fa.tw = p->tw_L;
    fa.Sinv = p->d_Sinv;
    fa.X = p->X;
    fa.part = p->d_part_fwd;
    return fa;
}

template <typename R>
static int stage_a(ac_plan* p, const double* u, const double* u0, const double* b, int b_rev, int transposed,
                   cudaStream_t st, bool record_res, int recompute = 0, bool fwd_only = false) {
    const ac::FwdArgs fa = fwd_args(p, u, u0, b, b_rev, transposed, recompute);
    const size_t smem = (size_t)p->L * p->M * p->P * sizeof(R);
    {
        ProfScope ps(p, KK_FWD, st);
        CK(ac::launch_fwd<R>(fa, p->grid, smem, st));
        p->launches++;
    }
    if (record_res) {
        CK(cudaMemcpyAsync(p->h_part_fwd, p->d_part_fwd, sizeof(double) * p->grid, cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(p->ev_res, st));
    }
    if (fwd_only) return AC_OK;
    {
        ProfScope ps(p, KK_SPACE, st);
        int rc = run_spatial<R>(p, p->X, p->d_mu, p->F * p->M, transposed, true, st, true);
        if (rc) return rc;
    }
    return AC_OK;
}

static ac::UpdArgs upd_args(const ac_plan* p, double* out, int accumulate, int diff_last) {
    ac::UpdArgs ua{};
    ua.N = p->N;
    ua.M = p->M;
    ua.L = p->L;
    ua.logL = p->logL;
    ua.F = p->F;
    ua.P = p->P_upd;
    ua.X = p->X;
    ua.Pm = p->d_P;
    ua.tw = p->tw_L;
    ua.sinv = p->d_sinv;
    ua.out = out;
    ua.accumulate = accumulate;
    ua.diff_last = diff_last;
    ua.part = p->d_part_upd;
    return ua;
}

template <typename R>
static int stage_b(ac_plan* p, double* out, int accumulate, cudaStream_t st, int diff_last = 0) {
    const size_t smem = (size_t)p->L * p->M * p->P * sizeof(R);
    ac::UpdArgs ua = upd_args(p, out, accumulate, diff_last);
    // the TMA-staged kernel for u += e on an aligned u (the map of u is
    // encoded once per u buffer)
    const bool tma = p->tma_ok && sizeof(R) == 4 && accumulate && !diff_last && ((uintptr_t)out & 15) == 0;
    if (tma && p->mapU_ptr != out) {
        if (!encode_2d(&p->mapU, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, sizeof(double), out, (uint64_t)p->N,
                       (uint64_t)p->L * p->M, (uint32_t)p->tma_P, (uint32_t)p->tgeo.urows))
            return fail(AC_ERR_CUDA, "cuTensorMapEncodeTiled failed for u");
        p->mapU_ptr = out;
    }
    {
        ProfScope ps(p, KK_UPD, st);
        if (tma) {
            ua.P = p->tma_P;
            CK(ac::launch_upd_tma(&p->mapX, &p->mapU, ua, p->tgeo, p->tma_grid, st));
            p->upd_grid_used = p->tma_grid;
        } else {
            CK(ac::launch_upd<R>(ua, p->grid_upd, smem, st));
            p->upd_grid_used = p->grid_upd;
        }
        p->launches++;
    }
    return AC_OK;
}

static int precond_a(ac_plan* p, const double* u, const double* u0, const double* b, int b_rev, int transposed,
                     cudaStream_t st, bool record_res, int recompute = 0, bool fwd_only = false) {
    if (p->precision == AC_C128)
        return stage_a<double>(p, u, u0, b, b_rev, transposed, st, record_res, recompute, fwd_only);
    return stage_a<float>(p, u, u0, b, b_rev, transposed, st, record_res, recompute, fwd_only);
}

// the spatial solves alone (after a precond_a with fwd_only)
static int precond_space(ac_plan* p, int transposed, cudaStream_t st) {
    ProfScope ps(p, KK_SPACE, st);
    if (p->precision == AC_C128)
        return run_spatial<double>(p, p->X, p->d_mu, p->F * p->M, transposed, true, st, true);
    return run_spatial<float>(p, p->X, p->d_mu, p->F * p->M, transposed, true, st, true);
}

static int precond_b(ac_plan* p, double* out, int accumulate, cudaStream_t st, int diff_last = 0) {
    if (p->precision == AC_C128) return stage_b<double>(p, out, accumulate, st, diff_last);
    return stage_b<float>(p, out, accumulate, st, diff_last);
}

// ||w - C u||_2 with the residual kernel alone (its transform output is unused)
static int residual_only(ac_plan* p, const double* u, const double* u0, const double* b, int b_rev, int transposed,
                         double wscale, double wn2, double* res, cudaStream_t st) {
    int rc = precond_a(p, u, u0, b, b_rev, transposed, st, true, 0, true);
    if (rc) return rc;
    CK(cudaEventSynchronize(p->ev_res));
    double s = 0.0;
    for (int i = 0; i < p->grid; ++i) s += p->h_part_fwd[i];
    *res = std::sqrt(s) * (wscale / ac::kNormPrescale) / wn2;
    return AC_OK;
}

static int precond(ac_plan* p, const double* u, const double* u0, const double* b, int b_rev, int transposed,
                   double* out, int accumulate, cudaStream_t st, bool record_res) {
    int rc = precond_a(p, u, u0, b, b_rev, transposed, st, record_res);
    if (rc) return rc;
    return precond_b(p, out, accumulate, st);
}

// ||w||_2 and ||w||_inf with w = (u0 stacked in block 0) + b
static int w_norms(ac_plan* p, const double* u0, const double* b, double* n2, double* ninf, cudaStream_t st) {
    const int grid = 152 * 2;
    {
        ProfScope ps(p, KK_AUX, st);
        CK(ac::launch_wnorms(u0, b, p->L, p->M, p->N, p->d_part_d, grid, st));
        p->launches++;
    }
    CK(cudaMemcpyAsync(p->h_part_d, p->d_part_d, sizeof(double) * 2 * grid, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double s = 0.0, mx = 0.0;
    for (int i = 0; i < grid; ++i) {
        s += p->h_part_d[2 * i];
        mx = std::max(mx, p->h_part_d[2 * i + 1]);
    }
    *n2 = std::sqrt(s);
    *ninf = mx;
    return AC_OK;
}

// ||A u0||_inf (A^T for the transposed system) by a stencil kernel
static int a_u0_inf(ac_plan* p, const double* u0, int transposed, double* out, cudaStream_t st) {
    const int grid = 152 * 2;
    {
        ProfScope ps(p, KK_AUX, st);
        CK(ac::launch_a_inf(transposed ? p->grid_adj : p->grid_fwd, u0, p->d_part_d, grid, st));
        p->launches++;
    }
    CK(cudaMemcpyAsync(p->h_part_d, p->d_part_d, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (int i = 0; i < grid; ++i) mx = std::max(mx, p->h_part_d[i]);
    *out = mx;
    return AC_OK;
}

static double a_inf_norm(const ac_plan* p) {
    double s = 0.0;
    for (int i = 0; i < 7; ++i) {
        if (i == 3) continue;
        s += std::fabs(p->grid_fwd.tx[i]) + (p->prob.dim == 2 ? std::fabs(p->grid_fwd.ty[i]) : 0.0);
    }
    return s + std::fabs(p->grid_fwd.c0);
}

static double pow2_scale(double v) {
    if (!(v > 0.0) || !std::isfinite(v)) return 1.0;
    int e;
    std::frexp(v, &e);
    return std::ldexp(1.0, e);
}

// Largest BiCGStab iteration count over the systems of the last inner solve,
// and the number of systems that stopped above tau (cap, stagnation, breakdown).
static int inner_summary(const ac_plan* p, int* failed) {
    int worst = 0, bad = 0;
    for (int i = 0; i < p->F * p->M; ++i) {
        int v = p->h_iters[i];
        if (v < 0) {
            v = -v;
            ++bad;
        } else if (v >= 1000000) {
            v %= 1000000;
            ++bad;
        }
        worst = std::max(worst, v);
    }
    *failed = bad;
    return worst;
}

// Reads (and clears) the kernels' error flag; the stream must be synchronised.
static int kernel_flag(ac_plan* p) {
    int h = 0;
    CK(cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CK(cudaMemset(p->d_err, 0, sizeof(int)));
        return fail(AC_ERR_CUDA, "a wait on the copy engine in the update kernel timed out");
    }
    return AC_OK;
}

// The Richardson loop shared by the forward and the adjoint solve.
static int richardson_loop(ac_plan* p, const double* u0, const double* b, int b_rev, int transposed, double* u,
                           double tol, ac_stats* stats, cudaStream_t st) {
    ac_stats local;
    ac_stats* S = stats ? stats : &local;
    std::memset(S, 0, sizeof(ac_stats));
    double wn2 = 0, winf = 0;
    int rc = w_norms(p, u0, b, &wn2, &winf, st);
    if (rc) return rc;
    S->w_norm2 = wn2;
    S->w_inf = winf;
    if (!std::isfinite(wn2)) return fail(AC_ERR_NOT_FINITE, "right-hand side is not finite");
    if (wn2 == 0.0) {
        CK(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)p->L * p->M * p->N, st));
        S->converged = 1;
        return AC_OK;
    }
    const double wscale = pow2_scale(winf);
    const ac_alpha_schedule& sc = p->sched;
    const int max_iter = std::min(std::max(sc.max_iter, 1), AC_MAX_STATS - 1);
    const double eps = p->precision == AC_C128 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    const double tau = p->inner != AC_INNER_FFT ? inner_tau(p, bicg_reliable(p)) : 0.0;
    const double gam = p->L * (3.0 * eps + tau) * winf;
    // m0 ~ ||u^(0) - u*||_inf: T max|u_t(0)| = T ||A u0 + b||_inf (Sec. 3.3, the
    // Lipschitz estimate) when the caller gives none; for a zero initial
    // iterate (adjoint) the bound L ||w||_inf
    double m = sc.m0;
    if (sc.mode == AC_ALPHA_PAPER && !(m > 0)) {
        if (u0) {
            double au0 = 0.0;
            rc = a_u0_inf(p, u0, transposed, &au0, st);
            if (rc) return rc;
            m = p->L * p->dT * (au0 + (b ? winf : 0.0));
        }
        if (!(m > 0)) m = p->L * winf;
    }
    // in the correction form the per-iteration error factor is about
    // alpha + L (3 eps + tau) / alpha, minimal at this alpha; Algorithm 2's
    // alpha_k (which tend to 1/2) are capped there
    const double alpha_mixed = std::min(0.25, std::max(1e-8, std::sqrt(p->L * (3.0 * eps + tau))));
    if (sc.form == AC_FORM_PAPER) {
        // eq. (Riteration) as printed, with Algorithm 2's loop and stop test
        if (sc.stop_rule != AC_STOP_PAPER)
            return fail(AC_ERR_INVALID_ARG, "AC_FORM_PAPER needs AC_STOP_PAPER (the form has no residual)");
        for (int k = 0; k < max_iter; ++k) {
            if (sc.mode == AC_ALPHA_PAPER && m <= tol) {
                S->converged = 1;
                break;
            }
            double alpha = sc.mode == AC_ALPHA_FIXED ? sc.alpha0 : alpha_mixed;
            double m_next = 0.0;
            if (sc.mode == AC_ALPHA_PAPER) {
                alpha = std::min(0.5, std::max(std::sqrt(gam / m), 1e-12));   // alpha_{k+1} = sqrt(gamma / m_k)
                m_next = 2.0 * std::sqrt(m * gam);                             // m_{k+1} = 2 sqrt(m_k gamma)
            }
            rc = ensure_tables(p, alpha, transposed, wscale, st);
            if (rc) return rc;
            rc = precond_a(p, u, u0, b, b_rev, transposed, st, false, 1);
            if (rc) return rc;
            rc = precond_b(p, u, 0, st, 1);
            if (rc) return rc;
            CK(cudaMemcpyAsync(p->h_part_upd, p->d_part_upd, sizeof(double) * p->upd_grid_used, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double mx = 0.0;
            for (int i = 0; i < p->upd_grid_used; ++i) mx = std::max(mx, p->h_part_upd[i]);
            for (int i = 0; i < p->upd_grid_used; ++i)
                if (std::isnan(p->h_part_upd[i])) mx = p->h_part_upd[i];
            S->alpha[k] = alpha;
            S->m[k] = sc.mode == AC_ALPHA_PAPER ? m : 0.0;
            S->diff_last[k] = mx;
            S->iters = k + 1;
            if (sc.mode == AC_ALPHA_PAPER) m = m_next;
            if (!std::isfinite(mx)) return fail(AC_ERR_NOT_FINITE, "iterate not finite at iteration %d", k);
            if (mx <= tol) {
                S->converged = 1;
                break;
            }
        }
        double res = 0.0;
        rc = residual_only(p, u, u0, b, b_rev, transposed, wscale, wn2, &res, st);
        if (rc) return rc;
        S->res_rel[S->iters] = res;
        CK(cudaStreamSynchronize(st));
        return S->converged ? AC_OK
                            : fail(AC_ERR_NO_CONVERGENCE, "Algorithm 2 not converged after %d iterations", S->iters);
    }
    int grew = 0;
    double prev_res = 1e300;
    // Safeguard of the adaptive rules: the correction-form alpha assumes inner
    // solves that meet tau.  When the residual grows, they evidently did not
    // (Krylov inner solves stall where the shifted systems are badly
    // conditioned, and their condition number grows with alpha), so alpha is
    // cut to a quarter from that iteration on (growth by more than a factor 2,
    // so that fluctuations at the attainable floor do not shrink alpha).
    double alpha_scale = 1.0;
    for (int k = 0;; ++k) {
        double alpha;
        double m_next = 0.0;
        const double cap = alpha_mixed * alpha_scale;
        if (sc.mode == AC_ALPHA_FIXED) alpha = sc.alpha0;
        else if (sc.mode == AC_ALPHA_MIXED) alpha = cap;
        else {
            alpha = std::sqrt(gam / m);          // alpha_{k+1} = sqrt(gamma / m_k)
            m_next = 2.0 * std::sqrt(m * gam);   // m_{k+1} = 2 sqrt(m_k gamma)
            alpha = std::min(cap, std::max(alpha, 1e-12));
        }
        rc = ensure_tables(p, alpha, transposed, wscale, st);
        if (rc) return rc;
        // residual of u^(k), transform and spatial solve; the host reads the
        // residual norm while the spatial solve runs and only then queues the
        // update, so a converged u^(k) is returned unchanged.  The spatial
        // solve is queued before the norm is known, except when the residual
        // is predicted to meet tol (the last two residuals extrapolated
        // geometrically): then it would be wasted, and it is queued only if the
        // prediction fails.
        bool speculate = true;
        if (sc.stop_rule == AC_STOP_RESIDUAL && k >= 2 && S->res_rel[k - 2] > 0.0) {
            const double pred = S->res_rel[k - 1] * (S->res_rel[k - 1] / S->res_rel[k - 2]);
            speculate = !(pred <= tol);
        }
        rc = precond_a(p, u, u0, b, b_rev, transposed, st, true, 0, !speculate);
        if (rc) return rc;
        CK(cudaEventSynchronize(p->ev_res));
        if (k > 0 && krylov_path(p)) S->inner_iters[k - 1] = inner_summary(p, &S->inner_failed[k - 1]);
        double s = 0.0;
        for (int i = 0; i < p->grid; ++i) s += p->h_part_fwd[i];
        const double res = std::sqrt(s) * (wscale / ac::kNormPrescale) / wn2;
        S->res_rel[k] = res;
        S->m[k] = sc.mode == AC_ALPHA_PAPER ? m : 0.0;
        S->iters = k;
        if (!std::isfinite(res)) {
            CK(cudaStreamSynchronize(st));
            return fail(AC_ERR_NOT_FINITE, "residual norm not finite at iteration %d", k);
        }
        bool done = false;
        if (sc.stop_rule == AC_STOP_RESIDUAL && res <= tol) done = true;
        if (sc.stop_rule == AC_STOP_PAPER && k > 0 && (S->diff_last[k - 1] <= tol || m <= tol)) done = true;
        if (done) {
            S->converged = 1;
            break;
        }
        if (k >= max_iter) break;
        if (res > prev_res) {
            if (++grew >= 3) {
                CK(cudaStreamSynchronize(st));
                return fail(AC_ERR_NO_CONVERGENCE, "residual grew three times in a row (iteration %d)", k);
            }
            if (sc.mode != AC_ALPHA_FIXED && res > 2.0 * prev_res) {
                // a real blow-up (not noise at the attainable floor): redo this
                // iteration's transform and spatial solve with a quarter of alpha
                alpha_scale *= 0.25;
                alpha = sc.mode == AC_ALPHA_MIXED ? alpha_mixed * alpha_scale
                                                  : std::min(alpha_mixed * alpha_scale, alpha);
                rc = ensure_tables(p, alpha, transposed, wscale, st);
                if (rc) return rc;
                rc = precond_a(p, u, u0, b, b_rev, transposed, st, false, 0, false);
                if (rc) return rc;
                speculate = true;   // the spatial solve is queued
            }
        } else grew = 0;
        prev_res = res;
        S->alpha[k] = alpha;
        if (!speculate) {
            rc = precond_space(p, transposed, st);
            if (rc) return rc;
        }
        rc = precond_b(p, u, 1, st);
        if (rc) return rc;
        if (sc.mode == AC_ALPHA_PAPER) m = m_next;
        if (sc.stop_rule == AC_STOP_PAPER) {
            CK(cudaMemcpyAsync(p->h_part_upd, p->d_part_upd, sizeof(double) * p->upd_grid_used, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            double mx = 0.0;
            for (int i = 0; i < p->upd_grid_used; ++i) mx = std::max(mx, p->h_part_upd[i]);
            for (int i = 0; i < p->upd_grid_used; ++i)
                if (std::isnan(p->h_part_upd[i])) mx = p->h_part_upd[i];
            S->diff_last[k] = mx;
        }
    }
    CK(cudaStreamSynchronize(st));
    rc = kernel_flag(p);
    if (rc) return rc;
    return S->converged ? AC_OK : fail(AC_ERR_NO_CONVERGENCE, "stop rule not met after %d iterations", S->iters);
}

// --------------------------------------------------------------- C ABI
// ------------------------------------------- sequential stepping (baseline)
static int ensure_seq_tables(ac_plan* p, cudaStream_t st) {
    if (p->d_seq_S) return AC_OK;
    const int M = p->M;
    std::vector<cd> B((size_t)M * M), lam(M), S((size_t)M * M), Sinv((size_t)M * M);
    for (int i = 0; i < M * M; ++i) B[i] = p->Q[i];
    const double c = ac::eig_small(M, B.data(), lam.data(), S.data(), Sinv.data());
    if (c < 0 || c > 1e10) return fail(AC_ERR_NOT_DIAGONALIZABLE, "Q is not diagonalisable (cond %g)", c);
    for (auto& v : lam) v *= p->dT;
    for (auto& v : S) v *= space_scale(p);   // the back-mix absorbs the FFT solves' factor N
    cudaError_t e = cudaMalloc((void**)&p->d_seq_S, sizeof(cd) * M * M);
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_seq_Sinv, sizeof(cd) * M * M);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_seq_mu, (size_t)M * p->csize);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_seq_S, S.data(), sizeof(cd) * M * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_seq_Sinv, Sinv.data(), sizeof(cd) * M * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = upload_c(p, p->d_seq_mu, lam.data(), lam.size(), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        // leave no partial state behind: the next call starts over
        for (void** b : {(void**)&p->d_seq_S, (void**)&p->d_seq_Sinv, &p->d_seq_mu}) {
            if (*b) cudaFree(*b);
            *b = nullptr;
        }
        return fail(AC_ERR_CUDA, "sequential tables: %s", cudaGetErrorString(e));
    }
    return AC_OK;
}

// the L steps, launched on st (used inside the graph capture)
template <typename R>
static int seq_steps(ac_plan* p, const double* u0, const double* b, double* u, cudaStream_t st) {
    const long long N = p->N;
    const int M = p->M;
    for (int l = 0; l < p->L; ++l) {
        const double* uprev = l == 0 ? u0 : u + ((size_t)(l - 1) * M + (M - 1)) * N;
        const double* v = b ? b + (size_t)l * M * N : nullptr;
        CK(ac::launch_seq_in<R>(M, N, uprev, v, p->d_seq_Sinv, p->X, st));
        int rc = run_spatial<R>(p, p->X, p->d_seq_mu, M, 0, false, st);
        if (rc) return rc;
        CK(ac::launch_seq_out<R>(M, N, p->X, p->d_seq_S, u + (size_t)l * M * N, st));
        p->launches += 2;
    }
    return AC_OK;
}

// ------------------------------------------------ outer Krylov (FGMRES)
// dot products out[j] = <V_j, w>, j < k (8 per pass over w; host sums the
// per-block partials)
static int kry_dots(ac_plan* p, double* const* V, int k, const double* w, double* out, cudaStream_t st) {
    const int G = ac::krylov_grid();
    const long long n = (long long)p->L * p->M * p->N;
    for (int j0 = 0; j0 < k; j0 += 8) {
        const int kk = std::min(8, k - j0);
        ac::VecList vl{};
        for (int j = 0; j < kk; ++j) vl.v[j] = V[j0 + j];
        CK(ac::launch_mdot(vl, kk, w, n, p->d_kpart, st));
        p->launches++;
        CK(cudaMemcpyAsync(p->h_kpart, p->d_kpart, sizeof(double) * kk * G, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int j = 0; j < kk; ++j) {
            double sum = 0.0;
            for (int b = 0; b < G; ++b) sum += p->h_kpart[(size_t)j * G + b];
            out[j0 + j] = sum;
        }
    }
    return AC_OK;
}

// y = beta y + sum_{j<k} c_j V_j
static int kry_axpy(ac_plan* p, double* const* V, const double* c, int k, double beta, double* y, cudaStream_t st) {
    const long long n = (long long)p->L * p->M * p->N;
    int j0 = 0;
    do {
        const int kk = std::min(8, k - j0);
        ac::VecList vl{};
        ac::Coefs cf{};
        for (int j = 0; j < kk; ++j) {
            vl.v[j] = V[j0 + j];
            cf.c[j] = c[j0 + j];
        }
        CK(ac::launch_maxpy(vl, cf, kk, j0 == 0 ? beta : 1.0, y, n, st));
        p->launches++;
        j0 += 8;
    } while (j0 < k);
    return AC_OK;
}

static int kry_alloc(ac_plan* p, int m) {
    const size_t D = (size_t)p->L * p->M * p->N;
    if (p->d_kry && p->kry_m >= m) return AC_OK;
    if (p->d_kry) cudaFree(p->d_kry);
    p->d_kry = nullptr;
    p->kry_m = 0;
    cudaError_t e = cudaMalloc((void**)&p->d_kry, sizeof(double) * D * (2 * (size_t)m + 2));
    if (e == cudaSuccess && !p->d_kpart) e = cudaMalloc((void**)&p->d_kpart, sizeof(double) * 8 * ac::krylov_grid());
    if (e == cudaSuccess && !p->h_kpart) e = cudaMallocHost((void**)&p->h_kpart, sizeof(double) * 8 * ac::krylov_grid());
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "Krylov workspace: %s", cudaGetErrorString(e));
    p->kry_m = m;
    return AC_OK;
}

// ------------------------------------------ one step on host buffers
//
// The iterate moves in and out in chunks of grid points (whole tiles of the
// time kernels), each chunk a strided copy of L*M rows.  The copies in go in
// the order: the stencil halo at the end of the grid (needed by chunk 0,
// periodic), then each chunk followed by the halo at the start of the next
// one, so that the residual kernel of chunk c can run as soon as chunk c and
// that halo have landed.  Each chunk of the updated iterate goes back to the
// host while the update kernel works on the next; the last update chunk is
// split in four so that little is left to copy after the last kernel.  The
// kernels and their tiles are the device step's, so the result is the same
// bit for bit.

static int host_step_resources(ac_plan* p, bool with_b) {
    cudaError_t e = cudaSuccess;
    const size_t vec = sizeof(double) * (size_t)p->L * p->M * p->N;
    if (!p->d_hu) {
        e = dalloc(p, &p->d_hu, vec);
        if (e != cudaSuccess) p->d_hu = nullptr;
    }
    if (e == cudaSuccess && !p->d_hu0) {
        e = dalloc(p, &p->d_hu0, sizeof(double) * p->N);
        if (e != cudaSuccess) p->d_hu0 = nullptr;
    }
    if (e == cudaSuccess && with_b && !p->d_hb) {
        e = dalloc(p, &p->d_hb, vec);
        if (e != cudaSuccess) p->d_hb = nullptr;
    }
    if (e == cudaSuccess && !p->s_in) e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->s_out) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
    for (int c = 0; c < kHostChunks && e == cudaSuccess; ++c)
        if (!p->ev_in[c]) e = cudaEventCreateWithFlags(&p->ev_in[c], cudaEventDisableTiming);
    for (int c = 0; c < kHostChunks + 4 && e == cudaSuccess; ++c)
        if (!p->ev_out[c]) e = cudaEventCreateWithFlags(&p->ev_out[c], cudaEventDisableTiming);
    for (cudaEvent_t* ev : {&p->ev_start, &p->ev_u0, &p->ev_done})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "host-step buffers: %s", cudaGetErrorString(e));
    return AC_OK;
}

// Split `tiles` tiles of P points (N points in all) into at most `want`
// chunks of whole tiles, boundaries t[0..K]; every chunk holds at least
// `halo` points, else fewer chunks are used (K = 1 at worst).
static int chunk_tiles(int tiles, int P, long N, long halo, int want, int* t) {
    int K = std::max(1, std::min(std::min(want, kHostChunks), tiles));
    const int T = (tiles + K - 1) / K;
    K = (tiles + T - 1) / T;
    if ((long)T * P < halo) K = 1;
    for (int c = 0; c < K; ++c) t[c] = c * T;
    t[K] = tiles;
    while (K > 1 && std::min((long)t[K] * P, N) - (long)t[K - 1] * P < halo) t[--K] = tiles;
    return K;
}

template <typename R>
static int host_step(ac_plan* p, double alpha, const double* u0h, const double* bh, double* uh, double* res,
                     int chunks, cudaStream_t st) {
    const long N = p->N;
    const size_t rows = (size_t)p->L * p->M, pitch = sizeof(double) * (size_t)N;
    const long halo = (long)p->grid_fwd.rad * (p->prob.dim == 2 ? p->prob.nx : 1);
    int tf[kHostChunks + 1], tu[kHostChunks + 4];
    const int want = chunks > 0 ? chunks : 8;
    const int Kf = chunk_tiles(p->grid, p->P, N, 2 * halo, want, tf);
    int Ku = chunk_tiles(p->grid_upd, p->P_upd, N, 0, want, tu);
    if (Ku > 1 && tu[Ku] - tu[Ku - 1] >= 4) {   // the last update chunk in four
        const int a0 = tu[Ku - 1], n = tu[Ku] - a0;
        for (int i = 1; i <= 4; ++i) tu[Ku - 1 + i] = a0 + (int)((long)n * i / 4);
        Ku += 3;
    }
    const double* d_u0 = u0h ? p->d_hu0 : nullptr;
    const double* d_b = bh ? p->d_hb : nullptr;

    // copies in, after the work already queued on the caller's stream
    CK(cudaEventRecord(p->ev_start, st));
    CK(cudaStreamWaitEvent(p->s_in, p->ev_start, 0));
    if (u0h) CK(cudaMemcpyAsync(p->d_hu0, u0h, sizeof(double) * N, cudaMemcpyHostToDevice, p->s_in));
    CK(cudaEventRecord(p->ev_u0, p->s_in));
    auto copy_in = [&](long a, long e) -> cudaError_t {
        if (e <= a) return cudaSuccess;
        cudaError_t ce = cudaMemcpy2DAsync(p->d_hu + a, pitch, uh + a, pitch, sizeof(double) * (e - a), rows,
                                           cudaMemcpyHostToDevice, p->s_in);
        if (ce == cudaSuccess && bh)
            ce = cudaMemcpy2DAsync(p->d_hb + a, pitch, bh + a, pitch, sizeof(double) * (e - a), rows,
                                   cudaMemcpyHostToDevice, p->s_in);
        return ce;
    };
    // point ranges [beg, end) of the chunks; chunks hold at least 2 halo points
    auto beg = [&](int c) { return (long)tf[c] * p->P; };
    auto end = [&](int c) { return std::min((long)tf[c + 1] * p->P, N); };
    const long h = Kf > 1 ? halo : 0;
    CK(copy_in(N - h, N));                                   // halo of chunk 0 across the periodic seam
    for (int c = 0; c < Kf; ++c) {
        const long a = c == 0 ? beg(c) : beg(c) + h;         // chunk c's first h points came earlier
        const long e = c == Kf - 1 ? end(c) - h : end(c);    // the last h points came first
        CK(copy_in(a, e));
        if (c + 1 < Kf) CK(copy_in(beg(c + 1), beg(c + 1) + h));   // the halo at the start of the next chunk
        CK(cudaEventRecord(p->ev_in[c], p->s_in));
    }

    // ||w|| (for the reported residual) needs u0 and all of b before the first residual kernel
    double wn2 = 1.0, winf = 1.0;
    if (res) {
        CK(cudaStreamWaitEvent(st, bh ? p->ev_in[Kf - 1] : p->ev_u0, 0));
        int rc = w_norms(p, d_u0, d_b, &wn2, &winf, st);
        if (rc) return rc;
    }
    const double wscale = res ? pow2_scale(winf) : (p->cur_wscale > 0 ? p->cur_wscale : 1.0);
    int rc = ensure_tables(p, alpha, 0, wscale, st);
    if (rc) return rc;

    // residual + time FFT + node mix, chunk by chunk: ev_in[c] marks chunk c,
    // the halo after it and (copied first) the halo before chunk 0 as landed;
    // chunk c's halo before it lies in chunk c - 1 (or is that first copy)
    ac::FwdArgs fa = fwd_args(p, p->d_hu, d_u0, d_b, 0, 0, 0);
    const size_t smem_f = (size_t)p->L * p->M * p->P * sizeof(R);
    CK(cudaStreamWaitEvent(st, p->ev_u0, 0));
    for (int c = 0; c < Kf; ++c) {
        CK(cudaStreamWaitEvent(st, p->ev_in[c], 0));
        fa.tile0 = tf[c];
        CK(ac::launch_fwd<R>(fa, tf[c + 1] - tf[c], smem_f, st));
        p->launches++;
    }
    if (res) {
        CK(cudaMemcpyAsync(p->h_part_fwd, p->d_part_fwd, sizeof(double) * p->grid, cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(p->ev_res, st));
    }

    rc = run_spatial<R>(p, p->X, p->d_mu, p->F * p->M, 0, true, st);
    if (rc) return rc;

    // update chunk by chunk; each chunk returns to the host while the next is updated
    ac::UpdArgs ua = upd_args(p, p->d_hu, 1, 0);
    const size_t smem_u = (size_t)p->L * p->M * p->P * sizeof(R);
    for (int c = 0; c < Ku; ++c) {
        ua.tile0 = tu[c];
        CK(ac::launch_upd<R>(ua, tu[c + 1] - tu[c], smem_u, st));
        p->launches++;
        CK(cudaEventRecord(p->ev_out[c], st));
        CK(cudaStreamWaitEvent(p->s_out, p->ev_out[c], 0));
        const long a = (long)tu[c] * p->P_upd, e = std::min((long)tu[c + 1] * p->P_upd, N);
        CK(cudaMemcpy2DAsync(uh + a, pitch, p->d_hu + a, pitch, sizeof(double) * (e - a), rows,
                             cudaMemcpyDeviceToHost, p->s_out));
    }
    p->upd_grid_used = p->grid_upd;
    // the caller's stream resumes after the last copy out
    CK(cudaEventRecord(p->ev_done, p->s_out));
    CK(cudaStreamWaitEvent(st, p->ev_done, 0));
    if (res) {
        CK(cudaEventSynchronize(p->ev_res));
        double s = 0.0;
        for (int i = 0; i < p->grid; ++i) s += p->h_part_fwd[i];
        *res = wn2 > 0 ? std::sqrt(s) * (wscale / ac::kNormPrescale) / wn2 : std::sqrt(s) * (wscale / ac::kNormPrescale);
    }
    return AC_OK;
}

extern "C" {

const char* ac_status_string(int s) {
    switch (s) {
        case AC_OK: return "ok";
        case AC_ERR_INVALID_ARG: return "invalid argument";
        case AC_ERR_NOT_DIAGONALIZABLE: return "Q G_l^{-1} not diagonalisable";
        case AC_ERR_NO_CONVERGENCE: return "no convergence";
        case AC_ERR_INNER_BREAKDOWN: return "inner solver breakdown";
        case AC_ERR_CUDA: return "CUDA error";
        case AC_ERR_NOT_FINITE: return "non-finite value";
    }
    return "unknown status";
}

const char* ac_last_error(void) { return g_err.c_str(); }

void ac_destroy(ac_plan* p) {
    if (!p) return;
    drain_profile(p);
    for (auto e : p->pool) cudaEventDestroy(e);
    void* bufs[] = {p->X, p->tw_L, p->tw_x, p->tw_y, p->sig_x, p->sig_y, p->sigT_x, p->sigT_y,
                    p->d_qs, p->d_s, p->d_wnorm, p->d_sinv, p->d_Sinv, p->d_P, p->d_mu,
                    p->d_part_fwd, p->d_part_upd, p->d_part_d, p->d_dtQ, p->d_dtQT, p->d_bicg,
                    p->d_iters, p->d_mu64, p->d_x64, p->d_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->h_part_fwd) cudaFreeHost(p->h_part_fwd);
    if (p->h_part_upd) cudaFreeHost(p->h_part_upd);
    if (p->h_part_d) cudaFreeHost(p->h_part_d);
    if (p->h_iters) cudaFreeHost(p->h_iters);
    if (p->ev_res) cudaEventDestroy(p->ev_res);
    if (p->seq_exec) cudaGraphExecDestroy(p->seq_exec);
    if (p->seq_capture) cudaStreamDestroy(p->seq_capture);
    for (void* b : {(void*)p->d_seq_S, (void*)p->d_seq_Sinv, p->d_seq_mu, (void*)p->d_kry, (void*)p->d_kpart})
        if (b) cudaFree(b);
    if (p->h_kpart) cudaFreeHost(p->h_kpart);
    for (void* b : {(void*)p->d_hu, (void*)p->d_hu0, (void*)p->d_hb})
        if (b) cudaFree(b);
    for (int c = 0; c < kHostChunks; ++c)
        if (p->ev_in[c]) cudaEventDestroy(p->ev_in[c]);
    for (int c = 0; c < kHostChunks + 4; ++c)
        if (p->ev_out[c]) cudaEventDestroy(p->ev_out[c]);
    for (cudaEvent_t e : {p->ev_start, p->ev_u0, p->ev_done})
        if (e) cudaEventDestroy(e);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    delete p;
}

int ac_setup(const ac_problem* prob, int M, int L, double dT, const ac_alpha_schedule* sched, int precision,
             int inner, ac_plan** out) {
    if (!prob || !sched || !out) return fail(AC_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (prob->dim != 1 && prob->dim != 2) return fail(AC_ERR_INVALID_ARG, "dim must be 1 or 2");
    if (prob->upwind ? (prob->order < 1 || prob->order > 5) : (prob->order != 2 && prob->order != 4 && prob->order != 6))
        return fail(AC_ERR_INVALID_ARG, "order must be 2, 4 or 6 (centred) or 1..5 (upwind)");
    const int ny = prob->dim == 2 ? prob->ny : 1;
    if (prob->nx < 2 || ny < 1 || (prob->dim == 2 && ny < 2))
        return fail(AC_ERR_INVALID_ARG, "grid too small");
    if (M < 1 || M > 4) return fail(AC_ERR_INVALID_ARG, "M must be 1..4");
    if (!is_pow2(L) || L < 2 || L > 1024) return fail(AC_ERR_INVALID_ARG, "L must be a power of two in 2..1024");
    if (!(dT > 0)) return fail(AC_ERR_INVALID_ARG, "dT must be positive");
    if (precision != AC_C128 && precision != AC_C64) return fail(AC_ERR_INVALID_ARG, "bad precision");
    if (inner != AC_INNER_FFT && inner != AC_INNER_BICGSTAB && inner != AC_INNER_GMRES)
        return fail(AC_ERR_INVALID_ARG, "bad inner solver");
    if (!(prob->lx > 0) || (prob->dim == 2 && !(prob->ly > 0))) return fail(AC_ERR_INVALID_ARG, "bad box length");
    const long long Nll = (long long)prob->nx * ny;
    if (Nll > (1LL << 30)) return fail(AC_ERR_INVALID_ARG, "grid too large");

    ac_plan* p = new ac_plan();
    p->prob = *prob;
    p->prob.ny = ny;
    p->M = M;
    p->L = L;
    p->logL = ilog2(L);
    p->F = L / 2 + 1;
    p->N = (int)Nll;
    p->dT = dT;
    p->sched = *sched;
    p->precision = precision;
    p->inner = inner;
    p->csize = precision == AC_C128 ? 16 : 8;
    cudaGetDevice(&p->device);
    ac::radau_nodes(M, p->t);
    ac::collocation_matrix(M, p->t, p->Q);

    // stencil taps of A and A^T (A^T: the taps mirrored, o -> -o)
    ac::Stencil sten;
    if (!ac::problem_stencil(p->prob, &sten)) {
        ac_destroy(p);
        return fail(AC_ERR_INVALID_ARG, "unsupported stencil");
    }
    ac::Grid g;
    g.dim = prob->dim;
    g.nx = prob->nx;
    g.ny = ny;
    g.N = p->N;
    g.rad = sten.rad;
    for (int i = 0; i < 7; ++i) {
        g.tx[i] = sten.tx[i];
        g.ty[i] = sten.ty[i];
    }
    g.c0 = sten.tx[3] + sten.ty[3];
    p->grid_fwd = g;
    for (int i = 0; i < 7; ++i) {
        g.tx[i] = sten.tx[6 - i];
        g.ty[i] = sten.ty[6 - i];
    }
    p->grid_adj = g;
    for (int i = 0; i < 7; ++i) {
        p->d1x[i] = sten.d1x[i];
        p->d2x[i] = sten.d2x[i];
        p->d1y[i] = sten.d1y[i];
        p->d2y[i] = sten.d2y[i];
    }

    // spatial solve path and kernel tiles
    const size_t cs = p->csize;
    ac::PlanShape shape;
    if (const char* why = ac::plan_shape(p->prob, M, L, precision, inner, sten.rad, sched->space_cluster, &shape)) {
        ac_destroy(p);
        return fail(AC_ERR_INVALID_ARG, "%s", why);
    }
    p->spatial_path = shape.spatial_path;
    p->rows_per_block = shape.rows_per_block;
    p->cols_per_block = shape.cols_per_block;
    p->rx = shape.rx;
    p->ry = shape.ry;
    p->cluster = shape.cluster;
    if (p->spatial_path == 7) {
        // a cluster that the device cannot hold falls back to the three passes
        int fits = 0;
        const ac::SpaceArgs sa = space_args(p, nullptr, nullptr, 1, 0);
        cudaError_t ce = precision == AC_C128 ? ac::launch_space_cluster<double>(sa, 0, &fits)
                                              : ac::launch_space_cluster<float>(sa, 0, &fits);
        if (ce != cudaSuccess || fits < 1) {
            (void)cudaGetLastError();
            if (sched->space_cluster > 0) {
                ac_destroy(p);
                return fail(AC_ERR_INVALID_ARG, "the requested cluster of %d CTAs does not fit on this device",
                            sched->space_cluster);
            }
            p->spatial_path = 2;
            p->cluster = 0;
        }
    }
    p->P = shape.P;
    p->grid = shape.grid;
    p->P_upd = shape.P_upd;
    p->grid_upd = shape.grid_upd;

    // device buffers
    cudaError_t e = cudaSuccess;
#define AL(ptr, bytes)                                                  \
    do {                                                                \
        if (e == cudaSuccess) e = dalloc(p, &(ptr), (bytes));           \
    } while (0)
    const int F = p->F;
    AL(p->X, (size_t)F * M * p->N * cs);
    AL(p->tw_L, (size_t)L * cs);
    AL(p->tw_x, (size_t)prob->nx * cs);
    AL(p->tw_y, (size_t)ny * cs);
    AL(p->sig_x, (size_t)prob->nx * cs);
    AL(p->sig_y, (size_t)ny * cs);
    AL(p->sigT_x, (size_t)prob->nx * cs);
    AL(p->sigT_y, (size_t)ny * cs);
    AL(p->d_qs, sizeof(double) * (size_t)L * M * M);
    AL(p->d_s, sizeof(double) * L);
    AL(p->d_wnorm, sizeof(float2) * L);
    AL(p->d_sinv, sizeof(double) * L);
    AL(p->d_Sinv, (size_t)F * M * M * cs);
    AL(p->d_P, (size_t)F * M * M * cs);
    AL(p->d_mu, (size_t)F * M * cs);
    AL(p->d_part_fwd, sizeof(double) * p->grid);
    AL(p->d_part_upd, sizeof(double) * std::max(p->grid_upd, 8 * 152));
    p->part_d_len = std::max(2 * 152 * 2, 3 * 152 * 4);
    AL(p->d_part_d, sizeof(double) * p->part_d_len);
    AL(p->d_dtQ, sizeof(double) * M * M);
    AL(p->d_dtQT, sizeof(double) * M * M);
    AL(p->d_err, sizeof(int));
    if (p->spatial_path == 3) {
        AL(p->d_iters, sizeof(int) * F * M);
        if (6 * cs * (size_t)p->N > 200 * 1024) AL(p->d_bicg, 6 * cs * (size_t)p->N * F * M);
        if (precision == AC_C64) {
            AL(p->d_mu64, sizeof(double2) * F * M);
            AL(p->d_x64, sizeof(double2) * (size_t)p->N * F * M);
        }
    } else if (p->spatial_path == 4) {
        AL(p->d_iters, sizeof(int) * F * M);
        const size_t per = ac::gmres_vector_bytes(gmres_restart(p), p->N, cs);
        if (per > 160 * 1024) AL(p->d_bicg, per * F * M);
    }
#undef AL
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_part_fwd, sizeof(double) * p->grid);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_part_upd, sizeof(double) * std::max(p->grid_upd, 8 * 152));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_part_d, sizeof(double) * p->part_d_len);
    if (e == cudaSuccess && krylov_path(p)) e = cudaMallocHost((void**)&p->h_iters, sizeof(int) * F * M);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_res, cudaEventDisableTiming);  // spin: low latency
    if (e != cudaSuccess) {
        int rc = fail(AC_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(e));
        ac_destroy(p);
        return rc;
    }
    // constant tables
    std::vector<cd> tw, sx(prob->nx), sy(ny), sxT(prob->nx), syT(ny);
    int rc = AC_OK;
    auto up = [&](void* dst, const std::vector<cd>& v) {
        if (rc == AC_OK && upload_c(p, dst, v.data(), v.size(), 0) != cudaSuccess)
            rc = fail(AC_ERR_CUDA, "table upload failed");
    };
    ac::twiddles(L, tw);
    up(p->tw_L, tw);
    ac::twiddles(prob->nx, tw);
    up(p->tw_x, tw);
    ac::twiddles(ny, tw);
    up(p->tw_y, tw);
    ac::axis_symbol(prob->nx, p->grid_fwd.tx, sx.data());
    ac::axis_symbol(prob->nx, p->grid_adj.tx, sxT.data());
    if (prob->dim == 2) {
        ac::axis_symbol(ny, p->grid_fwd.ty, sy.data());
        ac::axis_symbol(ny, p->grid_adj.ty, syT.data());
    } else {
        sy.assign(ny, cd(0.0));
        syT.assign(ny, cd(0.0));
    }
    up(p->sig_x, sx);
    up(p->sig_y, sy);
    up(p->sigT_x, sxT);
    up(p->sigT_y, syT);
    double dtQ[64], dtQT[64];
    for (int m = 0; m < M; ++m)
        for (int j = 0; j < M; ++j) {
            dtQ[m * M + j] = dT * p->Q[m * M + j];
            dtQT[m * M + j] = dT * p->Q[j * M + m];
        }
    if (rc == AC_OK && (cudaMemcpy(p->d_dtQ, dtQ, sizeof(double) * M * M, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(p->d_dtQT, dtQT, sizeof(double) * M * M, cudaMemcpyHostToDevice) != cudaSuccess))
        rc = fail(AC_ERR_CUDA, "table upload failed");
    if (rc == AC_OK && cudaMemset(p->d_err, 0, sizeof(int)) != cudaSuccess) rc = fail(AC_ERR_CUDA, "set-up failed");
    if (rc == AC_OK && cudaDeviceSynchronize() != cudaSuccess) rc = fail(AC_ERR_CUDA, "set-up sync failed");
    if (rc != AC_OK) {
        ac_destroy(p);
        return rc;
    }
    p->upd_grid_used = p->grid_upd;
    setup_tma(p);
    *out = p;
    return AC_OK;
}

int ac_plan_get_info(const ac_plan* p, ac_plan_info* info) {
    if (!p || !info) return fail(AC_ERR_INVALID_ARG, "null argument");
    info->N = p->N;
    info->M = p->M;
    info->L = p->L;
    info->F = p->F;
    info->tile_fwd = p->P;
    info->tile_upd = p->P_upd;
    info->spatial_path = p->spatial_path;
    info->workspace_bytes = p->workspace;
    info->launches = p->launches;
    info->update_kernel = p->tma_ok ? AC_UPDATE_TMA : AC_UPDATE_PLAIN;
    info->update_tile_tma = p->tma_ok ? p->tma_P : 0;
    info->space_cluster = p->spatial_path == 7 ? p->cluster : 0;
    return AC_OK;
}

static int apply_impl(ac_plan* p, const double* u, double* out, int transposed, void* stream) {
    if (!p || !u || !out) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    ac::ApplyArgs a{};
    a.g = transposed ? p->grid_adj : p->grid_fwd;
    a.M = p->M;
    a.L = p->L;
    a.transposed = transposed;
    a.u = u;
    a.out = out;
    a.dtQ = transposed ? p->d_dtQT : p->d_dtQ;
    ProfScope ps(p, KK_APPLY, st);
    CK(ac::launch_apply(a, st));
    p->launches++;
    return AC_OK;
}

int ac_apply_C(ac_plan* p, const double* u, double* Cu, void* stream) { return apply_impl(p, u, Cu, 0, stream); }

int ac_collocation_rhs(ac_plan* p, const double* bnodes, double* v, void* stream) {
    if (!p || !bnodes || !v || bnodes == v) return fail(AC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    ProfScope ps(p, KK_AUX, st);
    CK(ac::launch_colloc_rhs(bnodes, p->d_dtQ, v, p->L, p->M, p->N, st));
    p->launches++;
    return AC_OK;
}
int ac_apply_CT(ac_plan* p, const double* lam, double* out, void* stream) {
    return apply_impl(p, lam, out, 1, stream);
}

int ac_precond_solve(ac_plan* p, double alpha, const double* r, double* e, void* stream) {
    if (!p || !r || !e) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_tables(p, alpha, 0, p->cur_wscale > 0 ? p->cur_wscale : 1.0, st);
    if (rc) return rc;
    return precond(p, nullptr, nullptr, r, 0, 0, e, 0, st, false);
}

int ac_richardson_step(ac_plan* p, double alpha, const double* u0, const double* b, double* u,
                       double* res_rel_out, void* stream) {
    if (!p || !u) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    double wn2 = 1.0, winf = 1.0;
    if (res_rel_out) {
        int rc = w_norms(p, u0, b, &wn2, &winf, st);
        if (rc) return rc;
    }
    const double wscale = res_rel_out ? pow2_scale(winf) : (p->cur_wscale > 0 ? p->cur_wscale : 1.0);
    int rc = ensure_tables(p, alpha, 0, wscale, st);
    if (rc) return rc;
    rc = precond(p, u, u0, b, 0, 0, u, 1, st, res_rel_out != nullptr);
    if (rc) return rc;
    if (res_rel_out) {
        CK(cudaEventSynchronize(p->ev_res));
        double s = 0.0;
        for (int i = 0; i < p->grid; ++i) s += p->h_part_fwd[i];
        *res_rel_out = wn2 > 0 ? std::sqrt(s) * (wscale / ac::kNormPrescale) / wn2 : std::sqrt(s) * (wscale / ac::kNormPrescale);
    }
    return AC_OK;
}

int ac_richardson_step_host(ac_plan* p, double alpha, const double* u0, const double* b, double* u, int chunks,
                            double* res_rel_out, void* stream) {
    if (!p || !u) return fail(AC_ERR_INVALID_ARG, "null argument");
    if (chunks < 0) return fail(AC_ERR_INVALID_ARG, "chunks must be >= 0");
    int rc = host_step_resources(p, b != nullptr);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->precision == AC_C128) return host_step<double>(p, alpha, u0, b, u, res_rel_out, chunks, st);
    return host_step<float>(p, alpha, u0, b, u, res_rel_out, chunks, st);
}

int ac_richardson_solve(ac_plan* p, const double* u0, const double* b, double* u, int init_u, double tol,
                        ac_stats* stats, void* stream) {
    if (!p || !u) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (!init_u) {
        ProfScope ps(p, KK_AUX, st);
        CK(ac::launch_fill_stack(u0, u, p->L, p->M, p->N, st));
        p->launches++;
    }
    return richardson_loop(p, u0, b, 0, 0, u, tol, stats, st);
}

int ac_window_solve(ac_plan* p, const double* u0, int n_windows, double* u_end, double* work, double tol,
                    ac_stats* stats, int* iters_total, void* stream) {
    if (!p || !u0 || !u_end || !work || n_windows < 1 || u_end == u0) return fail(AC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t blk = (size_t)p->N * sizeof(double);
    const double* start = u0;
    int total = 0;
    for (int w = 0; w < n_windows; ++w) {
        int rc = ac_richardson_solve(p, start, nullptr, work, 0, tol, stats, stream);
        if (stats) total += stats->iters;
        if (rc) {
            if (iters_total) *iters_total = total;
            return rc;
        }
        // last node of the last step: u[L-1][M-1][:]
        CK(cudaMemcpyAsync(u_end, work + ((size_t)(p->L - 1) * p->M + (p->M - 1)) * p->N, blk,
                           cudaMemcpyDeviceToDevice, st));
        start = u_end;
    }
    if (iters_total) *iters_total = total;
    return AC_OK;
}

int ac_sequential_solve(ac_plan* p, const double* u0, const double* b, double* u, void* stream) {
    if (!p || !u0 || !u || u == u0) return fail(AC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_seq_tables(p, st);
    if (rc) return rc;
    if (!p->seq_exec || p->seq_key[0] != u0 || p->seq_key[1] != b || p->seq_key[2] != u) {
        if (p->seq_exec) {
            cudaGraphExecDestroy(p->seq_exec);
            p->seq_exec = nullptr;
        }
        if (!p->seq_capture) CK(cudaStreamCreateWithFlags(&p->seq_capture, cudaStreamNonBlocking));
        const long long before = p->launches;
        CK(cudaStreamBeginCapture(p->seq_capture, cudaStreamCaptureModeThreadLocal));
        rc = p->precision == AC_C128 ? seq_steps<double>(p, u0, b, u, p->seq_capture)
                                     : seq_steps<float>(p, u0, b, u, p->seq_capture);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->seq_capture, &graph);   // always end the capture
        p->seq_launches = p->launches - before;
        p->launches = before;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->seq_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->seq_exec = nullptr;
            return fail(AC_ERR_CUDA, "sequential graph: %s", cudaGetErrorString(e));
        }
        p->seq_key[0] = u0;
        p->seq_key[1] = b;
        p->seq_key[2] = u;
    }
    CK(cudaGraphLaunch(p->seq_exec, st));
    p->launches += p->seq_launches;
    return AC_OK;
}

int ac_krylov_solve(ac_plan* p, const double* u0, const double* b, double* u, int init_u, double tol, int restart,
                    ac_stats* stats, void* stream) {
    if (!p || !u || (!u0 && !b) || (!init_u && !u0)) return fail(AC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int m = restart > 0 ? std::min(restart, 32) : 10;
    int rc = kry_alloc(p, m);
    if (rc) return rc;
    ac_stats local;
    ac_stats* S = stats ? stats : &local;
    std::memset(S, 0, sizeof(ac_stats));
    double wn2 = 0, winf = 0;
    rc = w_norms(p, u0, b, &wn2, &winf, st);
    if (rc) return rc;
    S->w_norm2 = wn2;
    S->w_inf = winf;
    if (!std::isfinite(wn2)) return fail(AC_ERR_NOT_FINITE, "right-hand side is not finite");
    const size_t D = (size_t)p->L * p->M * p->N;
    if (wn2 == 0.0) {
        CK(cudaMemsetAsync(u, 0, sizeof(double) * D, st));
        S->converged = 1;
        return AC_OK;
    }
    // the preconditioner's alpha: the fixed one, else the correction-form rule
    const double eps = p->precision == AC_C128 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    const double tau = p->inner != AC_INNER_FFT ? inner_tau(p, bicg_reliable(p)) : 0.0;
    const double alpha = p->sched.mode == AC_ALPHA_FIXED
                             ? p->sched.alpha0
                             : std::min(0.25, std::max(1e-8, std::sqrt(p->L * (3.0 * eps + tau))));
    rc = ensure_tables(p, alpha, 0, pow2_scale(winf), st);
    if (rc) return rc;
    if (!init_u) {
        CK(ac::launch_fill_stack(u0, u, p->L, p->M, p->N, st));
        p->launches++;
    }
    std::vector<double*> V(m + 1), Z(m);
    for (int i = 0; i <= m; ++i) V[i] = p->d_kry + (size_t)i * D;
    for (int i = 0; i < m; ++i) Z[i] = p->d_kry + (size_t)(m + 1 + i) * D;
    double* T = p->d_kry + (size_t)(2 * m + 1) * D;
    const int max_steps = std::min(std::max(p->sched.max_iter, 1), AC_MAX_STATS - 1);
    std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), h(m + 1), h2(m + 1), y(m);
    int steps = 0;
    bool converged = false;
    for (;;) {
        // true residual r = w - C u into V_0
        rc = apply_impl(p, u, T, 0, st);
        if (rc) return rc;
        CK(ac::launch_w_minus(u0, b, T, V[0], p->L, p->M, p->N, st));
        p->launches++;
        double beta2 = 0.0;
        rc = kry_dots(p, &V[0], 1, V[0], &beta2, st);
        if (rc) return rc;
        const double beta = std::sqrt(beta2);
        S->res_rel[steps] = beta / wn2;
        if (!std::isfinite(beta)) return fail(AC_ERR_NOT_FINITE, "residual is not finite");
        if (beta <= tol * wn2) {
            converged = true;
            break;
        }
        if (steps >= max_steps) break;
        const double ib = 1.0 / beta;
        rc = kry_axpy(p, V.data(), nullptr, 0, ib, V[0], st);
        if (rc) return rc;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m; ++j) {
            // z_j = C_alpha^{-1} v_j, w = C z_j (flexible: z_j kept)
            rc = precond(p, nullptr, nullptr, V[j], 0, 0, Z[j], 0, st, false);
            if (rc) return rc;
            rc = apply_impl(p, Z[j], V[j + 1], 0, st);
            if (rc) return rc;
            // classical Gram-Schmidt, two passes
            for (int i = 0; i <= j; ++i) H[(size_t)j * (m + 1) + i] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                rc = kry_dots(p, V.data(), j + 1, V[j + 1], h.data(), st);
                if (rc) return rc;
                for (int i = 0; i <= j; ++i) {
                    H[(size_t)j * (m + 1) + i] += h[i];
                    h2[i] = -h[i];
                }
                rc = kry_axpy(p, V.data(), h2.data(), j + 1, 1.0, V[j + 1], st);
                if (rc) return rc;
            }
            double hn2 = 0.0;
            rc = kry_dots(p, &V[j + 1], 1, V[j + 1], &hn2, st);
            if (rc) return rc;
            const double hn = std::sqrt(hn2);
            if (hn > 0.0) {
                rc = kry_axpy(p, V.data(), nullptr, 0, 1.0 / hn, V[j + 1], st);
                if (rc) return rc;
            }
            // Givens rotations on column j
            double* hc = &H[(size_t)j * (m + 1)];
            for (int i = 0; i < j; ++i) {
                const double a0 = hc[i], a1 = hc[i + 1];
                hc[i] = cs[i] * a0 + sn[i] * a1;
                hc[i + 1] = -sn[i] * a0 + cs[i] * a1;
            }
            const double rho = std::hypot(hc[j], hn);
            if (!(rho > 0.0)) return fail(AC_ERR_INNER_BREAKDOWN, "GMRES breakdown (singular Hessenberg)");
            cs[j] = hc[j] / rho;
            sn[j] = hn / rho;
            hc[j] = rho;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            S->alpha[steps] = alpha;
            ++steps;
            S->res_rel[steps] = std::fabs(g[j + 1]) / wn2;
            if (std::fabs(g[j + 1]) <= tol * wn2 || hn == 0.0 || steps >= max_steps) {
                ++j;
                break;
            }
        }
        const int k = std::min(j, m);
        for (int i = k - 1; i >= 0; --i) {   // y = R^{-1} g
            double acc = g[i];
            for (int q = i + 1; q < k; ++q) acc -= H[(size_t)q * (m + 1) + i] * y[q];
            y[i] = acc / H[(size_t)i * (m + 1) + i];
        }
        rc = kry_axpy(p, Z.data(), y.data(), k, 1.0, u, st);
        if (rc) return rc;
    }
    S->iters = steps;
    S->converged = converged ? 1 : 0;
    return converged ? AC_OK : fail(AC_ERR_NO_CONVERGENCE, "outer GMRES: %d steps, residual %.3e", steps,
                                    S->res_rel[steps]);
}

int ac_adjoint_solve(ac_plan* p, const double* g, double* lam, double tol, ac_stats* stats, void* stream) {
    if (!p || !g || !lam || g == lam) return fail(AC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    // solve in reversed time: lam'[l] = lam[L-1-l], rhs g'[l] = g[L-1-l]
    CK(cudaMemsetAsync(lam, 0, sizeof(double) * (size_t)p->L * p->M * p->N, st));
    int rc = richardson_loop(p, nullptr, g, 1, 1, lam, tol, stats, st);
    if (rc != AC_OK && rc != AC_ERR_NO_CONVERGENCE) return rc;
    {
        ProfScope ps(p, KK_AUX, st);
        cudaError_t e = ac::launch_reverse_time(lam, p->L, (long long)p->M * p->N, st);
        if (e != cudaSuccess) return fail(AC_ERR_CUDA, "reverse failed: %s", cudaGetErrorString(e));
        p->launches++;
    }
    return rc;
}

int ac_grad_params(ac_plan* p, const double* u, const double* lam, double* du0, double* dparams, void* stream) {
    if (!p || !u || !lam || !dparams) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    ac::GradArgs a{};
    a.g = p->grid_fwd;
    a.M = p->M;
    a.L = p->L;
    a.u = u;
    a.lam = lam;
    a.dtQ = p->d_dtQ;
    for (int i = 0; i < 7; ++i) {
        a.d2x[i] = p->d2x[i];
        a.d1x[i] = p->d1x[i];
        a.d2y[i] = p->d2y[i];
        a.d1y[i] = p->d1y[i];
    }
    a.part = p->d_part_d;
    const int grid = std::min(p->part_d_len / 3, 152 * 4);
    {
        ProfScope ps(p, KK_GRAD, st);
        CK(ac::launch_grad(a, grid, st));
        p->launches++;
    }
    if (du0) {
        ProfScope ps(p, KK_GRAD, st);
        CK(ac::launch_sum_blocks(lam, p->M, p->N, du0, st));
        p->launches++;
    }
    CK(cudaMemcpyAsync(p->h_part_d, p->d_part_d, sizeof(double) * 3 * grid, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double s[3] = {0, 0, 0};
    for (int i = 0; i < grid; ++i)
        for (int c = 0; c < 3; ++c) s[c] += p->h_part_d[3 * i + c];
    dparams[0] = s[0];
    dparams[1] = -s[1];
    dparams[2] = p->prob.dim == 2 ? -s[2] : 0.0;
    return AC_OK;
}

int ac_measure_fp64_fma_rate(double* fma_per_s, void* stream) {
    if (!fma_per_s) return fail(AC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = 8 * sms, rounds = 8192;
    double* buf = nullptr;
    CK(cudaMalloc((void**)&buf, sizeof(double) * (4 + grid)));
    const double ab[3] = {0.999999, 1e-6, 1234.5678};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(buf, ab, sizeof(ab), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = ac::launch_dfma_rate(buf, rounds, buf + 4, grid, st);   // warm-up
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = ac::launch_dfma_rate(buf, rounds, buf + 4, grid, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "FP64 rate probe: %s", cudaGetErrorString(e));
    *fma_per_s = (double)grid * 256.0 * 8.0 * rounds / (best * 1e-3);
    return AC_OK;
}

int ac_profile_enable(ac_plan* p, int on) {
    if (!p) return fail(AC_ERR_INVALID_ARG, "null plan");
    drain_profile(p);
    p->prof = on != 0;
    for (int k = 0; k < KK_COUNT; ++k) {
        p->prof_ms[k] = 0;
        p->prof_count[k] = 0;
    }
    return AC_OK;
}

int ac_profile_read(ac_plan* p, int cap, const char** names, double* ms, long long* count) {
    if (!p) return fail(AC_ERR_INVALID_ARG, "null plan");
    drain_profile(p);
    const int n = std::min(cap, (int)KK_COUNT);
    for (int k = 0; k < n; ++k) {
        if (names) names[k] = kKindNames[k];
        if (ms) ms[k] = p->prof_ms[k];
        if (count) count[k] = p->prof_count[k];
    }
    return KK_COUNT;
}

}  // extern "C"
