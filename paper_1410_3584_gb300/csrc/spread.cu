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

namespace nlp {

template <typename T>
__global__ void __launch_bounds__(256) k_interp_spread(DevPlan<T> P) {
    extern __shared__ unsigned char smraw[];
    const int w = P.w;
    const int w0 = P.dim == 3 ? w : 1;
    const int W0 = P.T_tile[0] + w0 - 1, W1 = P.T_tile[1] + w - 1, W2 = P.T_tile[2] + w - 1;
    const int WW = W0 * W1 * W2;
    cpx<T> *sF = (cpx<T> *)smraw;
    cpx<T> *sG = sF + WW;
    T *spsi = (T *)(sG + WW);
    const Chunk ch = P.chunks[blockIdx.x];

    for (int q = threadIdx.x; q < WW; q += blockDim.x) {
        const int c = q % W2, t = q / W2, b = t % W1, a = t / W1;
        sF[q] = load_herm(P, ch.bx + a, ch.by + b, ch.bz + c);
        sG[q] = mk<T>(0, 0);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *ps = spsi + warp * 3 * kMaxWidth;
    const T two_w = (T)2 / (T)w;
    const int sa = W1 * W2;
    for (int j = ch.j0 + warp; j < ch.j1; j += nw) {
        const T d0 = P.nd[4 * (int64_t)j + 0], d1 = P.nd[4 * (int64_t)j + 1];
        const T d2 = P.nd[4 * (int64_t)j + 2], om = P.nd[4 * (int64_t)j + 3];
        const uint32_t o = P.no[j];
        const int o0 = o & 0xff, o1 = (o >> 8) & 0xff, o2 = (o >> 16) & 0xff;
        for (int t = lane; t < 3 * kMaxWidth; t += 32) {
            const int ax = t / kMaxWidth, tt = t % kMaxWidth;
            T v = (T)0;
            if (ax == 0) v = (w0 == 1) ? (tt == 0 ? (T)1 : (T)0) : (tt < w ? es_kernel<T>(((T)tt - d0) * two_w, P.beta) : (T)0);
            else if (tt < w) v = es_kernel<T>(((T)tt - (ax == 1 ? d1 : d2)) * two_w, P.beta);
            ps[t] = v;
        }
        __syncwarp();
        // interpolation
        cpx<T> acc = mk<T>(0, 0);
        for (int p = lane; p < w * w; p += 32) {
            const int b = p / w, c = p % w;
            const T wbc = ps[kMaxWidth + b] * ps[2 * kMaxWidth + c];
            const cpx<T> *col = sF + (o0 * W1 + (o1 + b)) * W2 + (o2 + c);
            T sx = 0, sy = 0;
            for (int a = 0; a < w0; ++a) {
                const T wa = ps[a];
                const cpx<T> f = col[a * sa];
                sx += wa * f.x;
                sy += wa * f.y;
            }
            acc.x += wbc * sx;
            acc.y += wbc * sy;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        cpx<T> cj;
        if (P.pois == nullptr) {
            cj = scale(acc, om);
        } else {
            // Algorithm 1: W(k) = (rho-hat(k) - (C0 - i k.M1) e^{-sigma^2 |k|^2/2}) / |k| in FP64
            // (om already holds (2pi)^-2 w_r w_phi / |k|)
            const double kx = P.pois[3 * (int64_t)j], ky = P.pois[3 * (int64_t)j + 1], kr = P.pois[3 * (int64_t)j + 2];
            const double g = exp(-0.5 * P.sigma * P.sigma * kr * kr);
            const double re = P.hvol * (double)acc.x - P.mom[0] * g;
            const double im = P.hvol * (double)acc.y + (kx * P.mom[1] + ky * P.mom[2]) * g;
            cj = mk<T>((T)((double)om * re), (T)((double)om * im));
        }
        // spreading
        for (int p = lane; p < w * w; p += 32) {
            const int b = p / w, c = p % w;
            const T wbc = ps[kMaxWidth + b] * ps[2 * kMaxWidth + c];
            const cpx<T> v = scale(cj, wbc);
            cpx<T> *col = sG + (o0 * W1 + (o1 + b)) * W2 + (o2 + c);
            for (int a = 0; a < w0; ++a) {
                const T wa = ps[a];
                red_add(col + a * sa, scale(v, wa));
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int q = threadIdx.x; q < WW; q += blockDim.x) {
        const cpx<T> v = sG[q];
        if (v.x == (T)0 && v.y == (T)0) continue;
        const int c = q % W2, t = q / W2, b = t % W1, a = t / W1;
        store_fold(P, ch.bx + a, ch.by + b, ch.bz + c, v);
    }
}

template <typename T> size_t interp_spread_smem(const DevPlan<T> &P) {
    const int w0 = P.dim == 3 ? P.w : 1;
    const size_t WW = (size_t)(P.T_tile[0] + w0 - 1) * (P.T_tile[1] + P.w - 1) * (P.T_tile[2] + P.w - 1);
    return 2 * WW * sizeof(cpx<T>) + 8 * 3 * kMaxWidth * sizeof(T);
}

template <typename T> cudaError_t launch_interp_spread(const DevPlan<T> &P, cudaStream_t st) {
    if (P.nchunks == 0) return cudaSuccess;
    const size_t sm = interp_spread_smem(P);
    cudaError_t e = cudaFuncSetAttribute(k_interp_spread<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_interp_spread<T><<<(unsigned)P.nchunks, 256, sm, st>>>(P);
    return cudaGetLastError();
}

template size_t interp_spread_smem<float>(const DevPlan<float> &);
template size_t interp_spread_smem<double>(const DevPlan<double> &);
template cudaError_t launch_interp_spread<float>(const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_interp_spread<double>(const DevPlan<double> &, cudaStream_t);

}  // namespace nlp
