// Fused type-2 interpolation -> node scaling -> type-1 spreading (the O(M) part of the
// NUFFT evaluation of Eq. (ifft), Sec. 2.1), generic kernel for 2D plans and for the 3D
// widths the register kernels do not cover.
//
// Nodes are the k -> -k half of the spherical/polar quadrature set, binned at plan time by
// the fine-grid tile holding their first tap.  One CTA takes one chunk of one tile:
//   1. stage the forward spectrum on the tile window (tile + w - 1 cells per axis) in shared
//      memory, reading the half spectrum and mirroring (conjugate at -l) where the window
//      reaches negative / beyond-Nyquist positions of the last axis;
//   2. per node (one warp per node): w kernel values per axis, interpolation as a sum over
//      the w^d taps (lanes over the last two axes, loop over the first), warp reduction,
//      scaling by the node weight, and spreading of the scaled value into the warp's own
//      copy of the window;
//   3. write the sum of the warps' copies (in warp order) to the chunk's scratch slot; the
//      combine pass (spread_common.cuh) folds the slots into G.
#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "spread_common.cuh"
#include "spread_dev.cuh"

namespace nlp {

template <typename T>
__global__ void __launch_bounds__(256) k_interp_spread(DevPlan<T> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    spread_generic_block<T>(P, blockIdx.x, smraw);
}

// warps (= window copies) per CTA: as many as fit in the shared memory, at most 8
template <typename T> int generic_warps(const DevPlan<T> &P, size_t limit) {
    const size_t WW = (size_t)P.win_n[0] * P.win_n[1] * P.win_n[2];
    const size_t rows = (size_t)P.win_n[0] * P.win_n[1];
    for (int nw = 8; nw >= 1; --nw)
        if (generic_smem_bytes<T>(WW, rows, nw) <= limit) return nw;
    return 0;
}

template <typename T> size_t interp_spread_smem(const DevPlan<T> &P, int nwarps) {
    const size_t WW = (size_t)P.win_n[0] * P.win_n[1] * P.win_n[2];
    const size_t rows = (size_t)P.win_n[0] * P.win_n[1];
    return generic_smem_bytes<T>(WW, rows, nwarps);
}

template <typename T> cudaError_t launch_interp_spread(const DevPlan<T> &P, cudaStream_t st) {
    if (P.nchunks == 0) return cudaSuccess;
    const int nw = generic_warps(P, (size_t)max_dyn_smem());
    if (nw < 1) return cudaErrorInvalidValue;
    const size_t sm = interp_spread_smem(P, nw);
    cudaError_t e = allow_smem<k_interp_spread<T>>();
    if (e != cudaSuccess) return e;
    k_interp_spread<T><<<(unsigned)P.nchunks, 32 * nw, sm, st>>>(P);
    return cudaGetLastError();
}

template int generic_warps<float>(const DevPlan<float> &, size_t);
template int generic_warps<double>(const DevPlan<double> &, size_t);
template size_t interp_spread_smem<float>(const DevPlan<float> &, int);
template size_t interp_spread_smem<double>(const DevPlan<double> &, int);
template cudaError_t launch_interp_spread<float>(const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_interp_spread<double>(const DevPlan<double> &, cudaStream_t);

}  // namespace nlp
