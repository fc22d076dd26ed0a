// k_fft_n768.cu -- the transform kernels of side 768 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<768>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
