// k_fft_n128.cu -- the transform kernels of side 128 (instantiation only; see k_fft.cuh).
#include "k_fft.cuh"

namespace spring {
template spring_status run_fft_op<128>(const FftOp&, cudaStream_t, bool);
}  // namespace spring
