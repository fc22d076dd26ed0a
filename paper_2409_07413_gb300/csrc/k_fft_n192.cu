// k_fft_n192.cu -- the transform kernels of side 192 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<192>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
