// Fused type-2 interpolation -> node scaling -> type-1 spreading (the O(M) part of the
// NUFFT evaluation of Eq. (ifft), Sec. 2.1).
//
// Nodes are the k -> -k half of the spherical/polar quadrature set, binned at plan time by
// the fine-grid tile holding their first tap.  One CTA takes one chunk of one tile:
//   1. stage the forward spectrum on the tile window (tile + w - 1 cells per axis) in shared
//      memory, reading the half spectrum and mirroring (conjugate at -l) where the window
//      reaches negative / beyond-Nyquist positions of the last axis;
//   2. per node (one warp per node): w kernel values per axis, interpolation as a sum over
//      the w^d taps (lanes over the last two axes, loop over the first), warp reduction,
//      scaling by the node weight, and spreading of the scaled value into a shared-memory
//      window with shared atomics;
//   3. add the window to the global half spectrum G with the Hermitian fold: a tap at
//      position l contributes v at l and conj(v) at -l, and only positions whose last
//      index lies in [0, nf/2] are stored.
// No global atomics are needed inside a tile; tiles meet only in step 3.
#include "common.cuh"
#include "launch.h"
#include "spread_common.cuh"
#include "spread_dev.cuh"

namespace nlp {

template <typename T>
__global__ void __launch_bounds__(256) k_interp_spread(DevPlan<T> P) {
    extern __shared__ unsigned char smraw[];
    spread_generic_block<T>(P, blockIdx.x, smraw);
}

template <typename T> size_t interp_spread_smem(const DevPlan<T> &P) {
    const int w0 = P.dim == 3 ? P.w : 1;
    const size_t WW = (size_t)(P.T_tile[0] + w0 - 1) * (P.T_tile[1] + P.w - 1) * (P.T_tile[2] + P.w - 1);
    const size_t rows = (size_t)(P.T_tile[0] + w0 - 1) * (P.T_tile[1] + P.w - 1);
    return generic_win_table_offset<T>(WW) + 2 * rows * sizeof(int64_t);
}

template <typename T> cudaError_t launch_interp_spread(const DevPlan<T> &P, cudaStream_t st) {
    if (P.nchunks == 0) return cudaSuccess;
    const size_t sm = interp_spread_smem(P);
    cudaError_t e = allow_smem<k_interp_spread<T>>();
    if (e != cudaSuccess) return e;
    k_interp_spread<T><<<(unsigned)P.nchunks, 256, sm, st>>>(P);
    return cudaGetLastError();
}

template size_t interp_spread_smem<float>(const DevPlan<float> &);
template size_t interp_spread_smem<double>(const DevPlan<double> &);
template cudaError_t launch_interp_spread<float>(const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_interp_spread<double>(const DevPlan<double> &, cudaStream_t);

}  // namespace nlp
