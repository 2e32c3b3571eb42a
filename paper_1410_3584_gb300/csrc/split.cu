// Improved algorithm (plan option method = 2; Sec. 2.1, Eq. (3.9), Fig. 3.1).
//
// With a partition of unity p(k),
//     phi = (2pi)^{-d} int (1 - p) U-hat rho-hat e^{ik.x} dk + (2pi)^{-d} int p U-hat rho-hat e^{ik.x} dk
//         = I_1 + I_2.
// w = (1 - p) U-hat is smooth: p = exp(-|k|^2/a) for the 3D Coulomb and dipolar symbols and for
// the 2D Laplace symbol 1/|k|^2 ((1 - e^{-s/a})/s is entire in s = |k|^2), p = erfc(|k|/l) for the
// 2D Coulomb symbol 1/|k| (w = erf(|k|/l)/|k| is entire in |k|^2).  I_1 is taken by the rectangle
// rule on the frequencies of the doubled grid (spacing 2 pi / (2 n h) per axis) with the
// trapezoid rho-hat: I_1(x_i) = (2n)^{-d} sum_m w(k_m) rho~(k_m) e^{i k_m . x_i}, an aperiodic FFT
// convolution with an analytic multiplier.  Its x-space kernel (3D Coulomb
// erfc(sqrt(a)|x|/2)/(4 pi |x|), 2D Coulomb erfc(l|x|/2)/(2 pi |x|), 2D Laplace E_1(a|x|^2/4)/(4 pi))
// is short-ranged, so the doubled grid's periodic images do not reach the box once the scale is
// chosen at plan time.  I_2 is the NUFFT of the plan itself on the small ball where p is not
// negligible (node weights carry p(k_j); for the 2D Laplace kernel that NUFFT is Algorithm 1,
// whose u_1 the plan takes at the widened width).  The evaluation runs I_2 into phi and then
// I_1 accumulating into phi, I_1 reusing the forward spectrum buffer of I_2.
#include <cmath>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace nlp {

// w(k_m) / (nf0 nf1 nf2) on the R2C half spectrum [nf0][nf1][nh] of the doubled grid
// form: 0 = (1 - e^{-|k|^2/a}) / |k|^2, 1 = (1 - e^{-|k|^2/a}) (3 (n.k)^2/|k|^2 - 1), 2 = erf(|k|/a) / |k|
template <typename T>
__global__ void k_split_multiplier(cpx<T> *K, int nf0, int nf1, int nf2, int nh, double dk0, double dk1, double dk2,
                                   double a, int form, double ax0, double ax1, double ax2, double scale) {
    const int64_t M = (int64_t)nf0 * nf1 * nh;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < M; q += (int64_t)gridDim.x * blockDim.x) {
        const int l2 = (int)(q % nh);
        const int64_t t = q / nh;
        const int l1 = (int)(t % nf1), l0 = (int)(t / nf1);
        const int m0 = 2 * l0 < nf0 ? l0 : l0 - nf0, m1 = 2 * l1 < nf1 ? l1 : l1 - nf1;
        const double k0 = m0 * dk0, k1 = m1 * dk1, k2v = l2 * dk2;
        const double kk = k0 * k0 + k1 * k1 + k2v * k2v;
        double w;
        if (form == 2) {
            const double kr = sqrt(kk);
            w = kk > 0.0 ? erf(kr / a) / kr : 2.0 / (a * sqrt(M_PI));   // limit at k = 0
        } else if (kk > 0.0) {
            const double one_m_p = -expm1(-kk / a);
            if (form == 1) {
                const double nk = ax0 * k0 + ax1 * k1 + ax2 * k2v;
                w = one_m_p * (3.0 * nk * nk / kk - 1.0);
            } else {
                w = one_m_p / kk;
            }
        } else {
            w = form == 1 ? 0.0 : 1.0 / a;   // limits at k = 0
        }
        K[q] = mk<T>((T)(w * scale), (T)0);
    }
}

template <typename T> static DevPlan<T> &main_of(nlp_plan_s *p);
template <> DevPlan<float> &main_of<float>(nlp_plan_s *p) { return p->pf; }
template <> DevPlan<double> &main_of<double>(nlp_plan_s *p) { return p->pd; }
template <typename T> static DevPlan<T> &part1_of(nlp_plan_s *p);
template <> DevPlan<float> &part1_of<float>(nlp_plan_s *p) { return p->pf1; }
template <> DevPlan<double> &part1_of<double>(nlp_plan_s *p) { return p->pd1; }

template <typename T> static nlp_status build_split_t(nlp_plan_s *p) {
    DevPlan<T> &D = main_of<T>(p);
    DevPlan<T> &E = part1_of<T>(p);
    E = D;   // lengths, twiddles, grid sizes
    nlp_status s;
    void *d;
    for (int a = 0; a < 3; ++a) {   // unit deconvolution: I_1 transforms rho itself
        std::vector<T> ones((size_t)D.n[a], (T)1);
        if ((s = alloc_dev(p, &d, sizeof(T) * ones.size()))) return s;
        if (cudaMemcpy(d, ones.data(), sizeof(T) * ones.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return NLP_ERR_CUDA;
        E.deconv[a] = (const T *)d;
    }
    const int64_t M = (int64_t)D.nf[0] * D.nf[1] * D.nh;
    if ((s = alloc_dev(p, &d, sizeof(cpx<T>) * (size_t)M))) return s;
    double ax[3] = {0, 0, 1};
    const double *da = p->opts.dipole_axis;
    const double nn = std::sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
    if (nn > 0)
        for (int a = 0; a < 3; ++a) ax[a] = da[a] / nn;
    const double dk[3] = {2.0 * M_PI / (D.nf[0] * p->h[0]), 2.0 * M_PI / (D.nf[1] * p->h[1]),
                          2.0 * M_PI / (D.nf[2] * p->h[2])};
    const double scale = 1.0 / ((double)D.nf[0] * D.nf[1] * D.nf[2]);
    const int blocks = (int)std::min<int64_t>((M + 255) / 256, 152 * 16);
    const int form = p->kernel == NLP_DIPOLE_3D ? 1 : (p->split_erfc ? 2 : 0);
    k_split_multiplier<T><<<blocks, 256, 0, p->stream>>>((cpx<T> *)d, D.nf[0], D.nf[1], D.nf[2], D.nh, dk[0], dk[1],
                                                         dk[2], p->split_a, form, ax[0], ax[1], ax[2], scale);
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    E.Khat = (const cpx<T> *)d;
    E.F = E.G = D.F;   // the forward spectrum of I_2 is free once I_2 has run
    E.accumulate = 1;
    E.pois = nullptr;
    E.mom = nullptr;
    return NLP_OK;
}

nlp_status build_split(nlp_plan_s *p) {
    if (p->grid.dim == 1 || p->kernel == NLP_CONFINED_2D) return NLP_ERR_UNSUPPORTED;
    return p->prec == NLP_FP64 ? build_split_t<double>(p) : build_split_t<float>(p);
}

}  // namespace nlp
