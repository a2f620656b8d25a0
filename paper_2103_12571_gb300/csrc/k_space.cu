// Spatial solves of eq. (d2), (I - mu_{l,m} dT A) x^2 = x^1, for every stored
// time frequency l and node m (Algorithm 1, inner loop).  For the periodic
// constant-coefficient A the solve is exact in the discrete Fourier basis:
// x^2 = IFFT( FFT(x^1) / (1 - dT mu sigma(k)) ), sigma the stencil symbol.
// Forward FFTs leave the spectrum in digit-reversed order and the inverse
// FFTs take it back from there, so no reordering pass is needed: the
// division only needs the true wavenumber of each slot (digitrev).  The
// inverse transforms are not normalised: the planes come back multiplied by
// N = nx ny, and the back transform that follows (the update kernel's
// unscaling table, the sequential stepping's back-mix) absorbs 1/N.
//
// Radix plans (template SB: stages of up to 2^SB points).  Complex64
// transforms use radix 8 (register pressure).  Complex128 transforms run on
// the FP64 pipe, where the instruction count per point is what counts: per
// point and stage a radix-16 stage costs 14.25 FP64 instructions with
// twiddles (10.5 without), radix 8 10.5 (7), radix 4 7 (4), radix 2 4 (2),
// so lengths 2^6 and 2^9 take radix 8 (8*8*8: 28 per point for 512 points,
// against 30.5 for 16*16*2) and the others radix 16.
#include <cooperative_groups.h>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace ac {

// One CTA per 1D plane held in shared memory.
template <typename R, int SB>
__global__ void __launch_bounds__(512) k_space_1d(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int n = a.nx, logn = a.lognx;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    const R one = tw[0].x, zero = tw[0].y;
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sig = reinterpret_cast<const C*>(a.sig_x);
    fft_fwd_op_inv<C, false, SB>(d, logn, 0, 1, 0, tw, [&](C v, int slot, int) {
        return div_one_minus(v, cmul(mu, sig[slot_freq<SB>(slot, logn)]), one, zero);
    });
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = d[i];   // times n (not normalised)
}

// One CTA per 2D plane held in shared memory (row FFTs, column FFTs, divide,
// inverse column and row FFTs).
template <typename R, int SBX, int SBY>
__global__ void __launch_bounds__(512) k_space_2d_small(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int nx = a.nx, ny = a.ny, lx = a.lognx, ly = a.logny;
    const long N = (long)nx * ny;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * N;
    for (long i = threadIdx.x; i < N; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* twx = reinterpret_cast<const C*>(a.tw_x);
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    const R one = twx[0].x, zero = twx[0].y;
    fft_fwd<C, 1, false, SBX>(d, lx, ly, 1, nx, 0, twx);   // rows (x index fastest across threads)
    // columns (column index fastest): forward, divide, inverse
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    fft_fwd_op_inv<C, true, SBY>(d, ly, lx, nx, 1, twy, [&](C v, int ys, int xs) {
        return div_one_minus(v, cmul(mu, cadd(sx[slot_freq<SBX>(xs, lx)], sy[slot_freq<SBY>(ys, ly)])), one, zero);
    });
    fft_inv<C, 1, false, SBX>(d, lx, ly, 1, nx, 0, twx);
    for (long i = threadIdx.x; i < N; i += blockDim.x) x[i] = d[i];   // times N (not normalised)
}

// Row pass of the three-pass 2D path: rows_per_block contiguous rows of length
// nx; forward FFT, or inverse FFT (not normalised).
template <typename R, int SBX>
__global__ void __launch_bounds__(256) k_space_rows(SpaceArgs a, int inverse) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int nx = a.nx, rpb = a.rows_per_block;
    const int logr = 31 - __clz(rpb);
    const int ld = rpb + 1;                   // padded stride of the transposed layout d[x][row]
    const long r0 = (long)blockIdx.x * rpb;   // rows_per_block divides planes * ny
    C* x = reinterpret_cast<C*>(a.X) + r0 * nx;
    const long cnt = (long)rpb * nx;
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int row = (int)(i >> a.lognx), ix = (int)(i & (nx - 1));
        d[ix * ld + row] = x[i];
    }
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    if (!inverse) {
        fft_fwd<C, 1, true, SBX>(d, a.lognx, logr, ld, 1, 0, tw);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int row = (int)(i >> a.lognx), ix = (int)(i & (nx - 1));
            x[i] = d[ix * ld + row];
        }
    } else {
        fft_inv<C, 1, true, SBX>(d, a.lognx, logr, ld, 1, 0, tw);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int row = (int)(i >> a.lognx), ix = (int)(i & (nx - 1));
            x[i] = d[ix * ld + row];
        }
    }
}

// Column pass: a tile of W consecutive x slots (digit-reversed order of the
// row pass's plan SBX) times all ny rows of one plane; forward FFT along y,
// divide, inverse FFT along y.  1 - mu sigma_x of the tile's x slots and
// mu sigma_y of every y slot are formed once per CTA, so the denominator of a
// point is one complex subtraction.
template <typename R, int SBX, int SBY>
__global__ void __launch_bounds__(256) k_space_cols(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int nx = a.nx, ny = a.ny, W = a.cols_per_block;
    const int tiles = nx / W;
    const int plane = blockIdx.x / tiles;
    const int c0 = (blockIdx.x - plane * tiles) * W;
    const int logW = 31 - __clz(W);
    C* x = reinterpret_cast<C*>(a.X) + (long)plane * nx * ny + c0;
    const long cnt = (long)ny * W;
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = (int)(i >> logW), w = (int)(i & (W - 1));
        d[i] = x[(long)iy * nx + w];
    }
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[plane];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    const R one = twy[0].x, zero = twy[0].y;
    C* mx = d + cnt;                  // W entries: 1 - mu sigma_x of this tile's x slots
    C* my = mx + W;                   // ny entries: mu sigma_y per y slot
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const C m = cmul(mu, sx[slot_freq<SBX>(c0 + i, a.lognx)]);
        mx[i] = cmake(one - m.x, -m.y);
    }
    for (int i = threadIdx.x; i < ny; i += blockDim.x) my[i] = cmul(mu, sy[slot_freq<SBY>(i, a.logny)]);
    __syncthreads();
    fft_fwd_op_inv<C, true, SBY>(d, a.logny, logW, W, 1, twy,
                                 [&](C v, int ys, int w) { return div_by(v, xsub(mx[w], my[ys], one), one, zero); });
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = (int)(i >> logW), w = (int)(i & (W - 1));
        x[(long)iy * nx + w] = d[i];
    }
}

// ---- single-pass 2D solve over a thread-block cluster
//
// One plane per cluster of CS CTAs; CTA c holds rows [c m, c m + m) of the
// plane (m = ny / CS) in its shared memory, so X is read and written once.
// Rows are transformed locally.  The column transform of length ny = CS m is
// a DIF stage of radix CS whose butterflies combine rows j, j + m, ...,
// j + (CS - 1) m, one from each CTA, followed by local DIF transforms of
// length m.  The butterflies of rows j are done by one CTA (CTA c takes
// j in [c m / CS, (c + 1) m / CS)), which reads the CS inputs from the
// other CTAs' shared memory and writes the CS outputs back to the same
// places, so the exchange is in place and every value crosses the cluster
// once each way.  After the forward column transform, CTA c holds the
// frequencies ky = c + CS k' (k' at local slot digitrev(k')).  The inverse
// runs the steps backwards.

namespace cg = cooperative_groups;

// Radix-CS stage across the cluster on rows j of every CTA (see above).
template <typename C, int CS, bool INV>
__device__ __forceinline__ void cluster_stage(cg::cluster_group& cl, C* d, int rank, int m, int nx, int lx,
                                              const C* __restrict__ tw) {
    const int per = m / CS;
    const int items = per << lx;
    const C w0 = tw[0];
    const auto one = w0.x;
    const auto zero = w0.y;
    C* rem[CS];
#pragma unroll
    for (int q = 0; q < CS; ++q) rem[q] = cl.map_shared_rank(d, q);
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int j = rank * per + (t >> lx);
        const int off = (j << lx) + (t & (nx - 1));
        C v[CS];
#pragma unroll
        for (int q = 0; q < CS; ++q) v[q] = rem[q][off];
        if (!INV) {
            small_dft<CS, false>(v, one);
#pragma unroll
            for (int r = 1; r < CS; ++r) v[r] = xmul<false>(v[r], tw[j * r], zero);   // w_ny^{j r}
        } else {
#pragma unroll
            for (int r = 1; r < CS; ++r) v[r] = xmul<true>(v[r], tw[j * r], zero);
            small_dft<CS, true>(v, one);
        }
#pragma unroll
        for (int r = 0; r < CS; ++r) rem[r][off] = v[r];
    }
}

// Global -> shared: 16-byte asynchronous copies (no register staging), one
// commit group; cp_async_wait() waits for this thread's copies.
__device__ __forceinline__ void load_async16(void* sdst, const void* gsrc, int n16) {
    const unsigned s = smem_addr(sdst);
    const char* g = reinterpret_cast<const char*>(gsrc);
    for (int k = threadIdx.x; k < n16; k += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + 16u * k), "l"(g + 16 * (size_t)k)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared -> global: one bulk copy by thread 0 after all threads' writes
// (16-byte aligned addresses, bytes a multiple of 16).  Thread 0 waits until
// the copy has read shared memory, so the CTA may exit afterwards.
__device__ __forceinline__ void store_bulk(void* gdst, const void* ssrc, unsigned bytes) {
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                     "r"(smem_addr(ssrc)), "r"(bytes)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
}

template <typename R, int CS, int SBX, int SBY>
__global__ void __launch_bounds__(256) k_space_cluster(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int plane = blockIdx.x / CS;
    const int nx = a.nx, lx = a.lognx;
    const int lm = a.logny - (CS == 16 ? 4 : (CS == 8 ? 3 : 2));
    const int m = 1 << lm;
    const int cnt = m << lx;
    C* d = reinterpret_cast<C*>(smem_raw);   // m rows x nx
    C* mx = d + cnt;                         // nx: 1 - mu sigma_x per x slot
    C* my = mx + nx;                         // m: mu sigma_y per local y slot
    C* twm = my + m;                         // m: w_m^k
    C* x = reinterpret_cast<C*>(a.X) + ((long)plane * CS + rank) * cnt;
    load_async16(d, x, (int)(cnt * sizeof(C) / 16));   // lands while the tables are formed
    const C* twx = reinterpret_cast<const C*>(a.tw_x);
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    const R one = twx[0].x, zero = twx[0].y;
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[plane];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const C t = cmul(mu, sx[slot_freq<SBX>(i, lx)]);
        mx[i] = cmake(one - t.x, -t.y);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        my[i] = cmul(mu, sy[rank + CS * slot_freq<SBY>(i, lm)]);
        twm[i] = twy[i * CS];
    }
    cp_async_wait();
    __syncthreads();
    fft_fwd<C, 1, false, SBX>(d, lx, lm, 1, nx, 0, twx);   // rows
    cl.sync();
    cluster_stage<C, CS, false>(cl, d, rank, m, nx, lx, twy);
    cl.sync();
    // columns, local stages: forward, divide, inverse
    fft_fwd_op_inv<C, true, SBY>(d, lm, lx, nx, 1, twm,
                                 [&](C v, int p, int xs) { return div_by(v, xsub(mx[xs], my[p], one), one, zero); });
    cl.sync();
    cluster_stage<C, CS, true>(cl, d, rank, m, nx, lx, twy);
    cl.sync();   // no CTA reads another's shared memory after this point
    fft_inv<C, 1, false, SBX>(d, lx, lm, 1, nx, 0, twx);
    store_bulk(x, d, (unsigned)(cnt * sizeof(C)));         // times N (not normalised)
}

// The radix plan of a length-2^logn transform in the precision R (see the
// file comment).
template <typename R>
static int plan_bits(int logn) {
    if (sizeof(R) == 4) return 3;
    return (logn == 6 || logn == 9) ? 3 : 4;
}

template <typename K>
static cudaError_t set_smem(K kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R, int SB>
static cudaError_t launch_1d_sb(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx;
    cudaError_t e = set_smem(k_space_1d<R, SB>, smem);
    if (e != cudaSuccess) return e;
    k_space_1d<R, SB><<<a.planes, 512, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_1d(const SpaceArgs& a, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) return launch_1d_sb<R, 3>(a, st);
    else return plan_bits<R>(a.lognx) == 3 ? launch_1d_sb<R, 3>(a, st) : launch_1d_sb<R, 4>(a, st);
}

template <typename R, int SBX, int SBY>
static cudaError_t launch_2d_small_sb(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx * a.ny;
    cudaError_t e = set_smem(k_space_2d_small<R, SBX, SBY>, smem);
    if (e != cudaSuccess) return e;
    k_space_2d_small<R, SBX, SBY><<<a.planes, 512, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_2d_small(const SpaceArgs& a, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        return launch_2d_small_sb<R, 3, 3>(a, st);
    } else {
        const int bx = plan_bits<R>(a.lognx), by = plan_bits<R>(a.logny);
        if (bx == 3) return by == 3 ? launch_2d_small_sb<R, 3, 3>(a, st) : launch_2d_small_sb<R, 3, 4>(a, st);
        return by == 3 ? launch_2d_small_sb<R, 4, 3>(a, st) : launch_2d_small_sb<R, 4, 4>(a, st);
    }
}

template <typename R, int SBX>
static cudaError_t launch_rows_sb(const SpaceArgs& a, int inverse, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx * (a.rows_per_block + 1);
    cudaError_t e = set_smem(k_space_rows<R, SBX>, smem);
    if (e != cudaSuccess) return e;
    long rows = (long)a.planes * a.ny;
    int grid = (int)(rows / a.rows_per_block);
    k_space_rows<R, SBX><<<grid, 256, smem, st>>>(a, inverse);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_rows(const SpaceArgs& a, int inverse, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) return launch_rows_sb<R, 3>(a, inverse, st);
    else return plan_bits<R>(a.lognx) == 3 ? launch_rows_sb<R, 3>(a, inverse, st) : launch_rows_sb<R, 4>(a, inverse, st);
}

template <typename R, int SBX, int SBY>
static cudaError_t launch_cols_sb(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * ((size_t)a.ny * a.cols_per_block + a.cols_per_block + a.ny);
    cudaError_t e = set_smem(k_space_cols<R, SBX, SBY>, smem);
    if (e != cudaSuccess) return e;
    int grid = a.planes * (a.nx / a.cols_per_block);
    k_space_cols<R, SBX, SBY><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_cols(const SpaceArgs& a, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        return launch_cols_sb<R, 3, 3>(a, st);
    } else {
        const int bx = plan_bits<R>(a.lognx), by = plan_bits<R>(a.logny);
        if (bx == 3) return by == 3 ? launch_cols_sb<R, 3, 3>(a, st) : launch_cols_sb<R, 3, 4>(a, st);
        return by == 3 ? launch_cols_sb<R, 4, 3>(a, st) : launch_cols_sb<R, 4, 4>(a, st);
    }
}

size_t space_cluster_smem(int nx, int ny, int cs, size_t csize) {
    const size_t m = (size_t)ny / cs;
    return csize * (m * nx + nx + 2 * m);
}

template <typename R, int CS, int SBX, int SBY>
static cudaError_t cluster_config(const SpaceArgs& a, cudaStream_t st, cudaLaunchConfig_t* cfg,
                                  cudaLaunchAttribute* at) {
    typedef typename Cx<R>::T C;
    const size_t smem = space_cluster_smem(a.nx, a.ny, CS, sizeof(C));
    auto kern = k_space_cluster<R, CS, SBX, SBY>;
    cudaError_t e = set_smem(kern, smem);
    if (e == cudaSuccess && CS > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3((unsigned)(a.planes * CS));
    cfg->blockDim = dim3(256);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
    return cudaSuccess;
}

// launch (fits == nullptr) or count the clusters that fit on the device at once
template <typename R, int CS, int SBX, int SBY>
static cudaError_t cluster_go(const SpaceArgs& a, cudaStream_t st, int* fits) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cudaError_t e = cluster_config<R, CS, SBX, SBY>(a, st, &cfg, at);
    if (e != cudaSuccess) return e;
    if (fits) return cudaOccupancyMaxActiveClusters(fits, k_space_cluster<R, CS, SBX, SBY>, &cfg);
    e = cudaLaunchKernelEx(&cfg, k_space_cluster<R, CS, SBX, SBY>, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename R, int CS>
static cudaError_t cluster_cs(const SpaceArgs& a, cudaStream_t st, int* fits) {
    const int lm = a.logny - (CS == 16 ? 4 : (CS == 8 ? 3 : 2));
    if constexpr (sizeof(R) == 4) {
        return cluster_go<R, CS, 3, 3>(a, st, fits);
    } else {
        const int bx = plan_bits<R>(a.lognx), by = plan_bits<R>(lm);
        if (bx == 3) return by == 3 ? cluster_go<R, CS, 3, 3>(a, st, fits) : cluster_go<R, CS, 3, 4>(a, st, fits);
        return by == 3 ? cluster_go<R, CS, 4, 3>(a, st, fits) : cluster_go<R, CS, 4, 4>(a, st, fits);
    }
}

template <typename R>
cudaError_t launch_space_cluster(const SpaceArgs& a, cudaStream_t st, int* fits) {
    if (a.cluster == 4) return cluster_cs<R, 4>(a, st, fits);
    if (a.cluster == 8) return cluster_cs<R, 8>(a, st, fits);
    if (a.cluster == 16) return cluster_cs<R, 16>(a, st, fits);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_space_cluster<float>(const SpaceArgs&, cudaStream_t, int*);
template cudaError_t launch_space_cluster<double>(const SpaceArgs&, cudaStream_t, int*);
template cudaError_t launch_space_1d<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_1d<double>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_2d_small<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_2d_small<double>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_rows<float>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_rows<double>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_cols<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_cols<double>(const SpaceArgs&, cudaStream_t);

}  // namespace ac
