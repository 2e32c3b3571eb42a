// FFT launchers instantiated for float (the FP32 translation unit of fft_launch.cuh).
#include "fft_launch.cuh"

namespace nlp {
template cudaError_t launch_fft_contig<float>(cpx<float> *, int64_t, const FftLen<float> &, int, float, cudaStream_t);
template cudaError_t launch_fwd_r2c<float>(const float *, const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_inv_c2r<float>(float *, const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_fft_strided<float>(cpx<float> *, const StridedDesc &, const FftLen<float> &, int, cudaStream_t);
template cudaError_t launch_fft_four<float>(const cpx<float> *, cpx<float> *, const StridedDesc &, const DevPlan<float> &, int, cudaStream_t);
template bool cols_on_reg_engine<float>(const FftLen<float> &);
}  // namespace nlp
