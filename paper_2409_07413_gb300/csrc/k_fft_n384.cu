// k_fft_n384.cu -- the transform kernels of side 384 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<384>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
