// FFT launchers instantiated for double (the FP64 translation unit of fft_launch.cuh).
#include "fft_launch.cuh"

namespace nlp {
template cudaError_t launch_fft_contig<double>(cpx<double> *, int64_t, const FftLen<double> &, int, double, cudaStream_t);
template cudaError_t launch_fwd_r2c<double>(const double *, const DevPlan<double> &, cudaStream_t);
template cudaError_t launch_inv_c2r<double>(double *, const DevPlan<double> &, cudaStream_t);
template cudaError_t launch_fft_strided<double>(cpx<double> *, const StridedDesc &, const FftLen<double> &, int, cudaStream_t);
template cudaError_t launch_fft_four<double>(const cpx<double> *, cpx<double> *, const StridedDesc &, const DevPlan<double> &, int, cudaStream_t);
template bool cols_on_reg_engine<double>(const FftLen<double> &);
}  // namespace nlp
