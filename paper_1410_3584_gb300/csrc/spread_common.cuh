// Device helpers shared by the interpolation/spreading kernels (spread.cu, spread_reg.cu).
#pragma once
#include "common.cuh"

namespace nlp {

// exponential-of-semicircle spreading function at x = 2 (tap - node) / w, |x| < 1
template <typename T>
__device__ __forceinline__ T es_kernel(T x, T beta) {
    const T s = (T)1 - x * x;
    return s > (T)0 ? exp(beta * (sqrt(s) - (T)1)) : (T)0;
}

__device__ __forceinline__ int wrapn(int l, int N) {
    int r = l % N;
    return r < 0 ? r + N : r;
}

template <typename T>
__device__ __forceinline__ cpx<T> load_herm(const DevPlan<T> &P, int g0, int g1, int g2) {
    const int l0 = wrapn(g0, P.nf[0]), l1 = wrapn(g1, P.nf[1]), l2 = wrapn(g2, P.nf[2]);
    if (2 * l2 <= P.nf[2]) return P.F[((int64_t)l0 * P.nf[1] + l1) * P.nh + l2];
    const int m0 = l0 ? P.nf[0] - l0 : 0, m1 = l1 ? P.nf[1] - l1 : 0, m2 = P.nf[2] - l2;
    return conj(P.F[((int64_t)m0 * P.nf[1] + m1) * P.nh + m2]);
}

template <typename T>
__device__ __forceinline__ void red_add(cpx<T> *p, cpx<T> v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

template <typename T>
__device__ __forceinline__ void store_fold(const DevPlan<T> &P, int g0, int g1, int g2, cpx<T> v) {
    const int l0 = wrapn(g0, P.nf[0]), l1 = wrapn(g1, P.nf[1]), l2 = wrapn(g2, P.nf[2]);
    const int N2 = P.nf[2];
    const int m0 = l0 ? P.nf[0] - l0 : 0, m1 = l1 ? P.nf[1] - l1 : 0;
    if (2 * l2 <= N2) red_add(P.G + ((int64_t)l0 * P.nf[1] + l1) * P.nh + l2, v);
    if (l2 == 0 || 2 * l2 >= N2) {
        const int m2 = l2 ? N2 - l2 : 0;
        red_add(P.G + ((int64_t)m0 * P.nf[1] + m1) * P.nh + m2, conj(v));
    }
}

__host__ __device__ __forceinline__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Window rows of a tile chunk in the half spectrum.  Row r = a Wt1 + b of the tile window is
// the fine-grid line (l0, l1) = (bx + a, by + b) mod (nf0, nf1); its Hermitian mirror is the
// line (-l0, -l1).  The half-spectrum offsets of both lines are tabulated once per chunk, so
// that filling and folding the window costs one table read and one add per cell.
template <typename T>
__device__ __forceinline__ void window_row_table(const DevPlan<T> &P, const Chunk &ch, int Wt0, int Wt1,
                                                 int64_t *rowoff, int64_t *rowmir) {
    for (int r = threadIdx.x; r < Wt0 * Wt1; r += blockDim.x) {
        const int a = r / Wt1, b = r - a * Wt1;
        const int l0 = wrapn(ch.bx + a, P.nf[0]), l1 = wrapn(ch.by + b, P.nf[1]);
        const int m0 = l0 ? P.nf[0] - l0 : 0, m1 = l1 ? P.nf[1] - l1 : 0;
        rowoff[r] = ((int64_t)l0 * P.nf[1] + l1) * P.nh;
        rowmir[r] = ((int64_t)m0 * P.nf[1] + m1) * P.nh;
    }
}

// The window column along the last axis that a thread fills and folds for every row it
// visits (thread t: column t mod Wt2, rows t / Wt2 + k (blockDim / Wt2)), with the last-axis
// wrap and the Hermitian decisions of load_herm / store_fold taken once per chunk.
struct WinCol {
    int c, r0, rstep;
    int l2;      // wrapped last-axis index
    bool herm;   // fill: F read from the mirror line at nf2 - l2, conjugated
    bool prim;   // fold: add at (l0, l1, l2)
    bool mir;    // fold: add the conjugate at (m0, m1, mz)
    int mz;
};

template <typename T>
__device__ __forceinline__ WinCol window_col(const DevPlan<T> &P, const Chunk &ch, int Wt2, int rows) {
    WinCol k;
    k.c = threadIdx.x % Wt2;
    k.rstep = blockDim.x / Wt2;
    k.r0 = threadIdx.x / Wt2;
    if (k.r0 >= k.rstep) k.r0 = rows;   // threads beyond rstep * Wt2 idle
    const int N2 = P.nf[2];
    k.l2 = wrapn(ch.bz + k.c, N2);
    k.herm = 2 * k.l2 > N2;
    k.prim = 2 * k.l2 <= N2;
    k.mir = k.l2 == 0 || 2 * k.l2 >= N2;
    k.mz = k.l2 ? N2 - k.l2 : 0;
    return k;
}

// sF := F on the window (cells r * pitch + c), sG := 0
template <typename T>
__device__ __forceinline__ void window_fill(const DevPlan<T> &P, const WinCol &k, const int64_t *rowoff,
                                            const int64_t *rowmir, int rows, int pitch, cpx<T> *sF, cpx<T> *sG) {
    const int N2 = P.nf[2];
    for (int r = k.r0; r < rows; r += k.rstep) {
        const cpx<T> v = k.herm ? conj(P.F[rowmir[r] + (N2 - k.l2)]) : P.F[rowoff[r] + k.l2];
        sF[r * pitch + k.c] = v;
        sG[r * pitch + k.c] = mk<T>(0, 0);
    }
}

// G += the window sG, folded onto the half spectrum
template <typename T>
__device__ __forceinline__ void window_fold(const DevPlan<T> &P, const WinCol &k, const int64_t *rowoff,
                                            const int64_t *rowmir, int rows, int pitch, const cpx<T> *sG) {
    for (int r = k.r0; r < rows; r += k.rstep) {
        const cpx<T> v = sG[r * pitch + k.c];
        if (v.x == (T)0 && v.y == (T)0) continue;
        if (k.prim) red_add(P.G + rowoff[r] + k.l2, v);
        if (k.mir) red_add(P.G + rowmir[r] + k.mz, conj(v));
    }
}

}  // namespace nlp
