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

template cudaError_t launch_upd<float>(const UpdArgs&, int, size_t, cudaStream_t);
template cudaError_t launch_upd<double>(const UpdArgs&, int, size_t, cudaStream_t);

}  // namespace ac
