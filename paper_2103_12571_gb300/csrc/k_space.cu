// Spatial solves of eq. (d2), (I - mu_{l,m} dT A) x^2 = x^1, for every stored
// time frequency l and node m (Algorithm 1, inner loop).  For the periodic
// constant-coefficient A the solve is exact in the discrete Fourier basis:
// x^2 = IFFT( FFT(x^1) / (1 - dT mu sigma(k)) ), sigma the stencil symbol.
// Forward FFTs leave the spectrum in digit-reversed order and the inverse
// FFTs take it back from there, so no reordering pass is needed: the
// division only needs the true wavenumber of each slot (digitrev).
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace ac {

// v / (1 - mu * sig): multiply by conj(den) / |den|^2 with one reciprocal
// (|den| >= 1 here whenever Re(mu sig) <= 0, so no scaling is needed)
__device__ __forceinline__ float rcp_c64(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_c64(double x) { return 1.0 / x; }

template <typename C>
__device__ __forceinline__ C shift_div(C v, C mu, C sig) {
    C den = cmul(mu, sig);
    den.x = (decltype(den.x))1 - den.x;
    den.y = -den.y;
    const auto inv = rcp_c64(den.x * den.x + den.y * den.y);
    return cscale(cmulc(v, den), inv);
}

// One CTA per 1D plane held in shared memory.
template <typename R>
__global__ void __launch_bounds__(512) k_space_1d(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    constexpr int SB = sizeof(R) == 8 ? 4 : 3;   // radix 16 in FP64, radix 8 in FP32 (register pressure)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int n = a.nx, logn = a.lognx;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    fft_fwd<C, 1, false, SB>(d, logn, 0, 1, 0, 0, tw);
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sig = reinterpret_cast<const C*>(a.sig_x);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[digitrev<SB>(i, logn)] = shift_div(d[digitrev<SB>(i, logn)], mu, sig[i]);
    __syncthreads();
    fft_inv<C, 1, false, SB>(d, logn, 0, 1, 0, 0, tw);
    const R sc = (R)1 / (R)n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = cscale(d[i], sc);
}

// One CTA per 2D plane held in shared memory (row FFTs, column FFTs, divide,
// inverse column and row FFTs).
template <typename R>
__global__ void __launch_bounds__(512) k_space_2d_small(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    constexpr int SB = sizeof(R) == 8 ? 4 : 3;   // radix 16 in FP64, radix 8 in FP32 (register pressure)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int nx = a.nx, ny = a.ny, lx = a.lognx, ly = a.logny;
    const long N = (long)nx * ny;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * N;
    for (long i = threadIdx.x; i < N; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* twx = reinterpret_cast<const C*>(a.tw_x);
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    fft_fwd<C, 1, false, SB>(d, lx, ly, 1, nx, 0, twx);   // rows (x index fastest across threads)
    fft_fwd<C, 1, true, SB>(d, ly, lx, nx, 1, 0, twy);    // columns (column index fastest)
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    for (long i = threadIdx.x; i < N; i += blockDim.x) {
        const int ky = (int)(i >> lx), kx = (int)(i & (nx - 1));
        const long slot = ((long)digitrev<SB>(ky, ly) << lx) + digitrev<SB>(kx, lx);
        d[slot] = shift_div(d[slot], mu, cadd(sx[kx], sy[ky]));
    }
    __syncthreads();
    fft_inv<C, 1, true, SB>(d, ly, lx, nx, 1, 0, twy);
    fft_inv<C, 1, false, SB>(d, lx, ly, 1, nx, 0, twx);
    const R sc = (R)1 / (R)N;
    for (long i = threadIdx.x; i < N; i += blockDim.x) x[i] = cscale(d[i], sc);
}

// Row pass of the three-pass 2D path: rows_per_block contiguous rows of length
// nx; forward FFT, or inverse FFT with the 1/(nx ny) normalisation.
template <typename R>
__global__ void __launch_bounds__(256) k_space_rows(SpaceArgs a, int inverse) {
    typedef typename Cx<R>::T C;
    constexpr int SB = sizeof(R) == 8 ? 4 : 3;   // radix 16 in FP64, radix 8 in FP32 (register pressure)
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
        fft_fwd<C, 1, true, SB>(d, a.lognx, logr, ld, 1, 0, tw);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int row = (int)(i >> a.lognx), ix = (int)(i & (nx - 1));
            x[i] = d[ix * ld + row];
        }
    } else {
        fft_inv<C, 1, true, SB>(d, a.lognx, logr, ld, 1, 0, tw);
        const R sc = (R)1 / ((R)nx * (R)a.ny);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int row = (int)(i >> a.lognx), ix = (int)(i & (nx - 1));
            x[i] = cscale(d[ix * ld + row], sc);
        }
    }
}

// Column pass: a tile of W consecutive x slots (digit-reversed order) times
// all ny rows of one plane; forward FFT along y, divide, inverse FFT along y.
template <typename R>
__global__ void __launch_bounds__(256) k_space_cols(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    constexpr int SB = sizeof(R) == 8 ? 4 : 3;   // radix 16 in FP64, radix 8 in FP32 (register pressure)
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
    __syncthreads();
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    fft_fwd<C, 1, true, SB>(d, a.logny, logW, W, 1, 0, twy);
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[plane];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    // symbol of the x slots of this tile and of every y slot
    C* sxs = d + cnt;                 // W entries
    C* sys = sxs + W;                 // ny entries, indexed by y slot
    for (int i = threadIdx.x; i < W; i += blockDim.x) sxs[i] = sx[slot_freq<SB>(c0 + i, a.lognx)];
    for (int i = threadIdx.x; i < ny; i += blockDim.x) sys[i] = sy[slot_freq<SB>(i, a.logny)];
    __syncthreads();
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int ys = (int)(i >> logW), w = (int)(i & (W - 1));
        d[i] = shift_div(d[i], mu, cadd(sxs[w], sys[ys]));
    }
    __syncthreads();
    fft_inv<C, 1, true, SB>(d, a.logny, logW, W, 1, 0, twy);
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = (int)(i >> logW), w = (int)(i & (W - 1));
        x[(long)iy * nx + w] = d[i];
    }
}

template <typename K>
static cudaError_t set_smem(K kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R>
cudaError_t launch_space_1d(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx;
    cudaError_t e = set_smem(k_space_1d<R>, smem);
    if (e != cudaSuccess) return e;
    k_space_1d<R><<<a.planes, 512, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_2d_small(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx * a.ny;
    cudaError_t e = set_smem(k_space_2d_small<R>, smem);
    if (e != cudaSuccess) return e;
    k_space_2d_small<R><<<a.planes, 512, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_rows(const SpaceArgs& a, int inverse, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.nx * (a.rows_per_block + 1);
    cudaError_t e = set_smem(k_space_rows<R>, smem);
    if (e != cudaSuccess) return e;
    long rows = (long)a.planes * a.ny;
    int grid = (int)(rows / a.rows_per_block);
    k_space_rows<R><<<grid, 256, smem, st>>>(a, inverse);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_cols(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * ((size_t)a.ny * a.cols_per_block + a.cols_per_block + a.ny);
    cudaError_t e = set_smem(k_space_cols<R>, smem);
    if (e != cudaSuccess) return e;
    int grid = a.planes * (a.nx / a.cols_per_block);
    k_space_cols<R><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_space_1d<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_1d<double>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_2d_small<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_2d_small<double>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_rows<float>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_rows<double>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_cols<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_cols<double>(const SpaceArgs&, cudaStream_t);

}  // namespace ac
