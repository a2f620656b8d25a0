// Explicit instantiations of the residual / time-FFT kernel k_fwd (eq. (globalsys),
// eq. (s1), eq. (d1)) with a complex64 transform.
#include "k_time.cuh"

namespace ac {

template cudaError_t launch_fwd<float>(const FwdArgs&, int, size_t, cudaStream_t);

}  // namespace ac
