// k_fft_n1024.cu -- the transform kernels of side 1024 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<1024>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
