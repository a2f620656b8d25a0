// Explicit instantiations of the update kernel k_upd (eqs. (d3), (Gsubstitution),
// (s3) and the FP64 update of eq. (Riteration)).
#include "k_time.cuh"

namespace ac {

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

size_t upd_smem(const UpdArgs& a, size_t rsize) { return (size_t)a.L * a.M * a.P * rsize; }

template <typename R>
cudaError_t launch_upd(const UpdArgs& a_in, int grid, size_t smem_unused, cudaStream_t st) {
    (void)smem_unused;
    UpdArgs a = a_in;
    a.out_aligned16 = aligned16(a.out);   // double2 accesses only on 16-byte aligned buffers
    const size_t smem = upd_smem(a, sizeof(R));
    switch (a.M) {
#define AC_CASE(MMV)                                                                          \
    case MMV: {                                                                               \
        cudaError_t e = cudaFuncSetAttribute(k_upd<R, MMV>,                                   \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                             (int)smem);                                      \
        if (e != cudaSuccess) return e;                                                       \
        k_upd<R, MMV><<<grid, 256, smem, st>>>(a);                                            \
        return cudaGetLastError();                                                            \
    }
        AC_CASE(1) AC_CASE(2) AC_CASE(3) AC_CASE(4)
#undef AC_CASE
    }
    return cudaErrorInvalidValue;
}

size_t upd_tma_smem(const UpdTmaGeom& g) { return 2 * (size_t)(g.xbuf + g.ubuf) + g.zbuf; }

cudaError_t launch_upd_tma(const void* mapX, const void* mapU, const UpdArgs& a, const UpdTmaGeom& g, int grid,
                           cudaStream_t st) {
    const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(mapX);
    const CUtensorMap& mu = *reinterpret_cast<const CUtensorMap*>(mapU);
    const size_t smem = upd_tma_smem(g);
    switch (a.M) {
#define AC_CASE(MMV)                                                                                      \
    case MMV: {                                                                                           \
        cudaError_t e = cudaFuncSetAttribute(k_upd_tma<MMV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                                  \
        if (e != cudaSuccess) return e;                                                                   \
        k_upd_tma<MMV><<<grid, 256, smem, st>>>(mx, mu, a, g);                                           \
        return cudaGetLastError();                                                                        \
    }
        AC_CASE(1) AC_CASE(2) AC_CASE(3) AC_CASE(4)
#undef AC_CASE
    }
    return cudaErrorInvalidValue;
}

// CTAs of the TMA-staged update kernel that fit on one SM with this geometry
int upd_tma_ctas_per_sm(int M, const UpdTmaGeom& g) {
    const size_t smem = upd_tma_smem(g);
    int n = 0;
    cudaError_t e = cudaSuccess;
    switch (M) {
        case 1: e = cudaFuncSetAttribute(k_upd_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_upd_tma<1>, 256, smem); break;
        case 2: e = cudaFuncSetAttribute(k_upd_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_upd_tma<2>, 256, smem); break;
        case 3: e = cudaFuncSetAttribute(k_upd_tma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_upd_tma<3>, 256, smem); break;
        case 4: e = cudaFuncSetAttribute(k_upd_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_upd_tma<4>, 256, smem); break;
    }
    return e == cudaSuccess ? n : 0;
}

template cudaError_t launch_upd<float>(const UpdArgs&, int, size_t, cudaStream_t);
template cudaError_t launch_upd<double>(const UpdArgs&, int, size_t, cudaStream_t);

}  // namespace ac
