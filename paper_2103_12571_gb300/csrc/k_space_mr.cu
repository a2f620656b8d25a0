// Spatial solves of eq. (d2), (I - mu_{l,m} dT A) x^2 = x^1, on periodic
// grids whose sizes are not powers of two but have no prime factor above 7
// (the 700 x 700 grid of the paper's advection test, the 350 and 600 points
// per axis of its heat ladder).  As on power-of-two grids the solve is exact
// in the discrete Fourier basis, x^2 = IFFT( FFT(x^1) / (1 - dT mu sigma(k)) ),
// and the inverse transforms are not normalised (the planes come back times
// N = nx ny; the back transform that follows absorbs 1/N).
//
// Transforms: Stockham autosort FFTs with radices 8, 7, 5, 4, 3, 2, out of
// place between two shared-memory buffers, natural order in and out (so the
// division indexes the true wavenumber).  Stage s of radix R, after stages
// whose radices multiply to Ns, maps for every j < n/R (k = j mod Ns) the R
// inputs a[j + r n/R], each times w^{r k n/(Ns R)} (w = exp(-2 pi i / n),
// conjugated in the inverse), through an R-point DFT to
// b[(j - k) R + k + r Ns].  The roots of the odd DFTs are read from the same
// full-circle table as the twiddles (w^{q n/R}).
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace ac {

// In-register DFT of odd length R in {3, 5, 7} (forward: y_r = sum_q x_q
// w_R^{qr}; INV: conjugate roots), natural order in and out.  With
// a_q = x_q + x_{R-q} and b_q = x_q - x_{R-q} (q = 1..(R-1)/2),
//     y_0 = x_0 + sum_q a_q,
//     y_r, y_{R-r} = x_0 + sum_q a_q cos(2 pi q r / R) -+ i sum_q b_q sin(2 pi q r / R)
// (upper sign forward).  c[q], s[q]: cos and sin of 2 pi q / R.
template <int R, bool INV, typename C, typename RR>
__device__ __forceinline__ void odd_dft(C* v, const RR* c, const RR* s, RR one, RR zero) {
    constexpr int h = (R - 1) / 2;
    C a[h + 1], b[h + 1];
#pragma unroll
    for (int q = 1; q <= h; ++q) {
        a[q] = xadd(v[q], v[R - q], one);
        b[q] = xsub(v[q], v[R - q], one);
    }
    C y[R];
    y[0] = v[0];
#pragma unroll
    for (int q = 1; q <= h; ++q) y[0] = xadd(y[0], a[q], one);
#pragma unroll
    for (int r = 1; r <= h; ++r) {
        C A = v[0], B = cmake(zero, zero);
#pragma unroll
        for (int q = 1; q <= h; ++q) {
            const int m = (q * r) % R;            // angle 2 pi m / R; sin changes sign past R/2
            const bool neg = m > h;
            const RR cq = c[neg ? R - m : m], sq = s[neg ? R - m : m];
            A.x = fma(a[q].x, cq, A.x);
            A.y = fma(a[q].y, cq, A.y);
            B.x = fma(neg ? -b[q].x : b[q].x, sq, B.x);
            B.y = fma(neg ? -b[q].y : b[q].y, sq, B.y);
        }
        const C minus_iB = cmake(B.y, -B.x);     // -i B
        const C yp = xadd(A, minus_iB, one);      // A - i B
        const C ym = xsub(A, minus_iB, one);      // A + i B
        y[r] = INV ? ym : yp;
        y[R - r] = INV ? yp : ym;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = y[i];
}

// One Stockham stage of radix R over nb transforms of length n: element
// (j, b) of a transform at src/dst[j * js + b * bs].  bfast: consecutive
// threads take consecutive b (else consecutive j).  Ends with __syncthreads().
template <typename C, int R, bool INV>
__device__ __forceinline__ void mr_stage(const C* __restrict__ src, C* __restrict__ dst, int n, int Ns, int nb,
                                         int js, int bs, bool bfast, const C* __restrict__ tw) {
    typedef decltype(C().x) RR;
    const int m = n / R;                 // butterflies per transform
    const int items = m * nb;
    const int stride = n / (Ns * R);     // twiddle-table step per r k
    const C w0 = tw[0];                  // 1 - 0i: register 1.0 and 0.0 for the FP64 FMA forms
    const RR one = w0.x, zero = w0.y;
    RR cr[R / 2 + 1], sr[R / 2 + 1];
    if constexpr (R == 3 || R == 5 || R == 7) {
#pragma unroll
        for (int q = 1; q <= R / 2; ++q) {
            const C w = tw[q * m];       // exp(-2 pi i q / R)
            cr[q] = w.x;
            sr[q] = -w.y;
        }
    }
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
        int j, b;
        if (bfast) {
            j = t / nb;
            b = t - j * nb;
        } else {
            b = t / m;
            j = t - b * m;
        }
        const int k = j % Ns;
        const C* p = src + (j * js + b * bs);
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * m * js];
        if (Ns > 1) {
            const int tk = k * stride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = xmul<INV>(v[r], tw[r * tk], zero);
        }
        if constexpr (R == 3 || R == 5 || R == 7) odd_dft<R, INV>(v, cr, sr, one, zero);
        else small_dft<R, INV>(v, one);
        C* q = dst + (((j - k) * R + k) * js + b * bs);
#pragma unroll
        for (int r = 0; r < R; ++r) q[r * Ns * js] = v[r];
    }
    __syncthreads();
}

// Whole transform of length n (plan rd), reading buffer a and using b as the
// other buffer; returns the buffer that holds the result (a or b).
// The caller synchronises before it; it ends with __syncthreads().
template <typename C, bool INV>
__device__ C* mr_fft(C* a, C* b, const FftRadices& rd, int n, int nb, int js, int bs, bool bfast,
                     const C* __restrict__ tw) {
    int Ns = 1;
    for (int s = 0; s < rd.ns; ++s) {
        const int R = rd.r[s];
        switch (R) {
            case 8: mr_stage<C, 8, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
            case 7: mr_stage<C, 7, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
            case 5: mr_stage<C, 5, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
            case 4: mr_stage<C, 4, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
            case 3: mr_stage<C, 3, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
            default: mr_stage<C, 2, INV>(a, b, n, Ns, nb, js, bs, bfast, tw); break;
        }
        C* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// One CTA per 1D plane: two buffers of nx values in shared memory.
template <typename R>
__global__ void __launch_bounds__(256) k_space_mr_1d(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.nx;
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + n;
    C* x = reinterpret_cast<C*>(a.X) + (long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) b0[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    const R one = tw[0].x;
    C* d = mr_fft<C, false>(b0, b1, a.rx, n, 1, 1, 0, false, tw);
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[blockIdx.x];
    const C* sig = reinterpret_cast<const C*>(a.sig_x);
    const R zero = tw[0].y;
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = div_one_minus(d[i], cmul(mu, sig[i]), one, zero);
    __syncthreads();
    d = mr_fft<C, true>(d, d == b0 ? b1 : b0, a.rx, n, 1, 1, 0, false, tw);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = d[i];   // times n (not normalised)
}

// Row pass of the three-pass 2D solve: rows_per_block rows of nx (the last
// CTA may hold fewer), row-major in shared memory; forward FFT, or inverse
// FFT (not normalised).
template <typename R>
__global__ void __launch_bounds__(256) k_space_mr_rows(SpaceArgs a, int inverse) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, rpb = a.rows_per_block;
    const long rows = (long)a.planes * a.ny;
    const long r0 = (long)blockIdx.x * rpb;
    const int nr = (int)(rows - r0 < rpb ? rows - r0 : rpb);
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + (long)rpb * nx;
    C* x = reinterpret_cast<C*>(a.X) + r0 * nx;
    const int cnt = nr * nx;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) b0[i] = x[i];
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(a.tw_x);
    C* d = inverse ? mr_fft<C, true>(b0, b1, a.rx, nx, nr, 1, nx, false, tw)
                   : mr_fft<C, false>(b0, b1, a.rx, nx, nr, 1, nx, false, tw);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) x[i] = d[i];
}

// Column pass: a tile of W consecutive x wavenumbers (the last tile of a
// plane may be narrower) times all ny rows of one plane; forward FFT along y,
// divide, inverse FFT along y.  1 - mu sigma_x of the tile's wavenumbers and
// mu sigma_y of every y wavenumber are formed once per CTA.
template <typename R>
__global__ void __launch_bounds__(256) k_space_mr_cols(SpaceArgs a) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = a.nx, ny = a.ny, W = a.cols_per_block;
    const int tiles = (nx + W - 1) / W;
    const int plane = blockIdx.x / tiles;
    const int c0 = (blockIdx.x - plane * tiles) * W;
    const int wn = nx - c0 < W ? nx - c0 : W;   // columns of this tile
    const int cnt = ny * wn;
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + ny * W;
    C* mx = b1 + ny * W;                        // W entries: 1 - mu sigma_x
    C* my = mx + W;                             // ny entries: mu sigma_y
    C* x = reinterpret_cast<C*>(a.X) + (long)plane * nx * ny + c0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = i / wn, w = i - iy * wn;
        b0[i] = x[(long)iy * nx + w];
    }
    const C mu = reinterpret_cast<const C*>(a.mu_dT)[plane];
    const C* sx = reinterpret_cast<const C*>(a.sig_x);
    const C* sy = reinterpret_cast<const C*>(a.sig_y);
    const C* twy = reinterpret_cast<const C*>(a.tw_y);
    const R one = twy[0].x, zero = twy[0].y;
    for (int i = threadIdx.x; i < wn; i += blockDim.x) {
        const C m = cmul(mu, sx[c0 + i]);
        mx[i] = cmake(one - m.x, -m.y);
    }
    for (int i = threadIdx.x; i < ny; i += blockDim.x) my[i] = cmul(mu, sy[i]);
    __syncthreads();
    C* d = mr_fft<C, false>(b0, b1, a.ry, ny, wn, wn, 1, true, twy);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int ky = i / wn, w = i - ky * wn;
        d[i] = div_by(d[i], xsub(mx[w], my[ky], one), one, zero);
    }
    __syncthreads();
    d = mr_fft<C, true>(d, d == b0 ? b1 : b0, a.ry, ny, wn, wn, 1, true, twy);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int iy = i / wn, w = i - iy * wn;
        x[(long)iy * nx + w] = d[i];
    }
}

template <typename K>
static cudaError_t set_smem_mr(K kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

size_t space_mr_smem(int pass, int n, int batch, int ny, size_t csize) {
    if (pass == 0) return 2 * csize * (size_t)n;                     // 1D: two planes
    if (pass == 1) return 2 * csize * (size_t)n * batch;             // rows: two tiles of batch rows
    return csize * (2 * (size_t)ny * batch + batch + ny);            // cols: two tiles + tables
}

template <typename R>
cudaError_t launch_space_mr_1d(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const size_t smem = space_mr_smem(0, a.nx, 1, 1, sizeof(C));
    cudaError_t e = set_smem_mr(k_space_mr_1d<R>, smem);
    if (e != cudaSuccess) return e;
    k_space_mr_1d<R><<<a.planes, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_mr_rows(const SpaceArgs& a, int inverse, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const size_t smem = space_mr_smem(1, a.nx, a.rows_per_block, a.ny, sizeof(C));
    cudaError_t e = set_smem_mr(k_space_mr_rows<R>, smem);
    if (e != cudaSuccess) return e;
    const long rows = (long)a.planes * a.ny;
    const int grid = (int)((rows + a.rows_per_block - 1) / a.rows_per_block);
    k_space_mr_rows<R><<<grid, 256, smem, st>>>(a, inverse);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_space_mr_cols(const SpaceArgs& a, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const size_t smem = space_mr_smem(2, a.nx, a.cols_per_block, a.ny, sizeof(C));
    cudaError_t e = set_smem_mr(k_space_mr_cols<R>, smem);
    if (e != cudaSuccess) return e;
    const int grid = a.planes * ((a.nx + a.cols_per_block - 1) / a.cols_per_block);
    k_space_mr_cols<R><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_space_mr_1d<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_mr_1d<double>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_mr_rows<float>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_mr_rows<double>(const SpaceArgs&, int, cudaStream_t);
template cudaError_t launch_space_mr_cols<float>(const SpaceArgs&, cudaStream_t);
template cudaError_t launch_space_mr_cols<double>(const SpaceArgs&, cudaStream_t);

}  // namespace ac
