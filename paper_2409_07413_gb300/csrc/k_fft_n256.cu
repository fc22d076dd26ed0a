// k_fft_n256.cu -- the transform kernels of side 256 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<256>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
