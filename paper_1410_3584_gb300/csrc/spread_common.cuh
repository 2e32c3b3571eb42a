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

}  // namespace nlp
