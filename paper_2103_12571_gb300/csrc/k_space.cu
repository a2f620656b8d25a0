// Spatial solves of eq. (d2), (I - mu_{l,m} dT A) x^2 = x^1, for every stored
// time frequency l and node m (Algorithm 1, inner loop).  For the periodic
// constant-coefficient A the solve is exact in the discrete Fourier basis:
// x^2 = IFFT( FFT(x^1) / (1 - dT mu sigma(k)) ), sigma the stencil symbol.
// The forward FFT is decimation-in-frequency (bit-reversed output) and the
// inverse decimation-in-time (bit-reversed input), so no reordering pass is
// needed: the division only needs the true wavenumber of each slot.
#include "common.cuh"
#include "kernels.h"

namespace ac {

template <typename C>
__device__ __forceinline__ C shift_div(C v, C mu, C sig) {
    // v / (1 - mu * sig)
    C den = cmul(mu, sig);
    den.x = (decltype(den.x))1 - den.x;
    den.y = -den.y;
    return cdiv(v, den);
}

// One CTA per 1D plane held in shared memory.
template <typename R>
__global__ void __launch_bounds__(512) k_space_1d(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int n = a.nx, logn = a.lognx;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    fft_dif<C, false>(d, logn, 1, 0, 1, 0, tw);
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sig = reinterpret_cast<const C*>(a.sig_x);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = shift_div(d[i], mu, sig[bitrev(i, logn)]);
    __syncthreads();
    fft_dit_inv<C, false>(d, logn, 1, 0, 1, 0, tw);
    const R sc = (R)1 / (R)n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = cscale(d[i], sc);
}

// One CTA per 2D plane held in shared memory (row FFTs, column FFTs, divide,
// inverse column and row FFTs).
template <typename R>
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
    fft_dif<C, false>(d, lx, ny, -1, 1, nx, twx);            // rows
    fft_dif<C, true>(d, ly, nx, lx, nx, 1, twy);             // columns
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    for (long i = threadIdx.x; i < N; i += blockDim.x) {
        const int iy = (int)(i >> lx), ix = (int)(i & (nx - 1));
        const C s = cadd(sx[bitrev(ix, lx)], sy[bitrev(iy, ly)]);
        d[i] = shift_div(d[i], mu, s);
    }
    __syncthreads();
    fft_dit_inv<C, true>(d, ly, nx, lx, nx, 1, twy);
    fft_dit_inv<C, false>(d, lx, ny, -1, 1, nx, twx);
    const R sc = (R)1 / (R)N;
    for (long i = threadIdx.x; i < N; i += blockDim.x) x[i] = cscale(d[i], sc);
}

// Row pass of the three-pass 2D path: rows_per_block contiguous rows of length
// nx; forward DIF, or inverse DIT with the 1/(nx ny) normalisation.
template <typename R>
__global__ void __launch_bounds__(256) k_space_rows(SpaceArgs a, int inverse) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* d = reinterpret_cast<C*>(smem_raw);
    const int nx = a.nx, rpb = a.rows_per_block;
    const long total_rows = (long)a.planes * a.ny;
    const long r0 = (long)blockIdx.x * rpb;
    const int nr = (int)((total_rows - r0) < rpb ? (total_rows - r0) : rpb);
    C* x = reinterpret_cast<C*>(a.X) + r0 * nx;
    const long cnt = (long)nr * nx;
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) d[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    if (!inverse) {
        fft_dif<C, false>(d, a.lognx, nr, -1, 1, nx, tw);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) x[i] = d[i];
    } else {
        fft_dit_inv<C, false>(d, a.lognx, nr, -1, 1, nx, tw);
        const R sc = (R)1 / ((R)nx * (R)a.ny);
        for (long i = threadIdx.x; i < cnt; i += blockDim.x) x[i] = cscale(d[i], sc);
    }
}

// Column pass: a tile of W consecutive (bit-reversed) x slots times all ny
// rows of one plane; forward DIF along y, divide, inverse DIT along y.
template <typename R>
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
    __syncthreads();
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    fft_dif<C, true>(d, a.logny, W, logW, W, 1, twy);
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[plane];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    for (long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = (int)(i >> logW), w = (int)(i & (W - 1));
        const C s = cadd(sx[bitrev(c0 + w, a.lognx)], sy[bitrev(iy, a.logny)]);
        d[i] = shift_div(d[i], mu, s);
    }
    __syncthreads();
    fft_dit_inv<C, true>(d, a.logny, W, logW, W, 1, twy);
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
    size_t smem = sizeof(C) * (size_t)a.nx * a.rows_per_block;
    cudaError_t e = set_smem(k_space_rows<R>, smem);
    if (e != cudaSuccess) return e;
    long rows = (long)a.planes * a.ny;
    int grid = (int)((rows + a.rows_per_block - 1) / a.rows_per_block);
    k_space_rows<R><<<grid, 256, smem, st>>>(a, inverse);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_cols(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    size_t smem = sizeof(C) * (size_t)a.ny * a.cols_per_block;
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
