// Complex FP64 instantiation of the fused FFT kinetic step (kernels in qf_fft_impl.cuh).
#include <math.h>

#include "qf_fft_impl.cuh"

namespace qf {

template cudaError_t launch_fft_pass<double>(int, int, FftPassArgs<double>, cpx<double>*, cudaStream_t, int*, bool);
template int fft_final_blocks<double>(int);
template int fft_final_blocks_max<double>(int);

}  // namespace qf
