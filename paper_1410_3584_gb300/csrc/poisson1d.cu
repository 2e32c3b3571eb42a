// 1D Poisson potential (Sec. 2.2, the 1D case): phi = U * rho with U(x) = -|x|/2.
//
// The Gaussian G_1 = rho-hat(0) G - (x rho)-hat(0) G' (G of width sigma, unit mass) carries
// the mass and the first moment of rho; its potential u_1 = rho-hat(0) u_{1,1} - (x rho)-hat(0)
// u_{1,2} solves Eq. (1DPois) in closed form.  The rest, u_2 = U * (rho - G_1), has the
// Fourier integrand W(k) = (rho-hat(k) - G_1-hat(k)) / k^2, smooth at k = 0 with
// W(0) = -(x^2 rho)-hat(0)/2 + sigma^2 rho-hat(0)/2, so u_2 is a regular FFT quadrature:
//   rho-hat(k_l) = h e^{i k_l L} sum_m rho_m e^{-2 pi i l m / 2n}      (trapezoid, zero padded)
//   u_2(x_m)     = (dk / 2 pi) sum_l W(k_l) e^{-i k_l L} e^{+2 pi i l m / 2n}
// with k_l = l dk, dk = pi / (n h), l = -n..n-1 (e^{i k_l L} = i^l on this grid), terms with
// |k_l| > P dropped, sigma = 6 sqrt(2) / P.  FP64 throughout (the grids have at most 1024
// points).  One evaluation: moments + zero padding (one CTA), forward FFT, W(k) with the
// phases, inverse FFT, crop + u_1 -- five launches; the elementwise FP64 steps (exp, erf) run
// over many SMs.  (A single fused CTA was measured slower: 0.115 vs 0.093 ms at n = 1024, the
// FP64 exp/erf and FFT work of one SM outweighing four launch latencies.)
#include <cmath>

#include "launch.h"
#include "plan.h"

namespace nlp {

constexpr int kMomThreads = 256;

// C0 = h sum rho, M1 = h sum x rho, M2 = h sum x^2 rho (block reduction in a fixed order);
// work = rho zero-padded to 2n (complex)
__global__ void __launch_bounds__(kMomThreads) k_p1d_moments(const double *rho, int n, double L, double h,
                                                             cpx<double> *work, double *mom) {
    __shared__ double s[3][kMomThreads];
    double c0 = 0, m1 = 0, m2 = 0;
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const double r = rho[m], x = -L + m * h;
        c0 += r;
        m1 += x * r;
        m2 += x * x * r;
        work[m] = mk<double>(r, 0.0);
        work[m + n] = mk<double>(0.0, 0.0);
    }
    s[0][threadIdx.x] = c0;
    s[1][threadIdx.x] = m1;
    s[2][threadIdx.x] = m2;
    __syncthreads();
    for (int off = kMomThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mom[0] = h * s[0][0];
        mom[1] = h * s[1][0];
        mom[2] = h * s[2][0];
    }
}

// i^q for integer q
__device__ __forceinline__ cpx<double> ipow(int q) {
    switch (q & 3) {
        case 0: return mk<double>(1, 0);
        case 1: return mk<double>(0, 1);
        case 2: return mk<double>(-1, 0);
        default: return mk<double>(0, -1);
    }
}

// work[idx] (forward DFT of the padded rho at l = idx or idx - 2n) -> (dk/2pi) W(k_l) e^{-i k_l L}
__global__ void k_p1d_w(cpx<double> *work, const double *mom, int n, double h, double P, double sigma) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * n) return;
    const int l = idx < n ? idx : idx - 2 * n;
    const double dk = M_PI / (n * h);
    const double k = l * dk;
    const double C0 = mom[0], M1 = mom[1], M2 = mom[2];
    cpx<double> W;
    if (l == 0) {
        W = mk<double>(-0.5 * M2 + 0.5 * sigma * sigma * C0, 0.0);
    } else if (fabs(k) > P) {
        W = mk<double>(0.0, 0.0);
    } else {
        const cpx<double> rh = scale(work[idx] * ipow(l), h);         // rho-hat(k_l), e^{i k_l L} = i^l
        const double g = exp(-0.5 * k * k * sigma * sigma);
        const cpx<double> g1 = mk<double>(C0 * g, -k * M1 * g);         // (C0 - i k M1) e^{-k^2 sigma^2/2}
        W = scale(rh - g1, 1.0 / (k * k));
    }
    work[idx] = scale(W * ipow(-l), dk / (2.0 * M_PI));                // e^{-i k_l L} = i^{-l}
}

// phi_m = Re u_2(x_m) + C0 u_{1,1}(x_m) - M1 u_{1,2}(x_m)
__global__ void k_p1d_u1(double *phi, const cpx<double> *work, const double *mom, int n, double L, double h,
                         double sigma) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double x = -L + m * h;
    const double e = erf(x / (M_SQRT2 * sigma));
    const double u11 = -sigma / sqrt(2.0 * M_PI) * exp(-x * x / (2.0 * sigma * sigma)) - 0.5 * x * e;
    const double u12 = -0.5 * e;
    phi[m] = work[m].x + mom[0] * u11 - mom[1] * u12;
}

nlp_status plan_build_1d(nlp_plan_s *p) {
    if (p->prec != NLP_FP64) return NLP_ERR_UNSUPPORTED;
    const int n = p->grid.n[0];
    const double L = p->grid.L[0];
    const double h = 2.0 * L / n;
    double P = M_PI / h;
    if (p->opts.kmax > 0) P = std::min(P, p->opts.kmax);
    p->p1d_n = n;
    p->p1d_P = P;
    p->sigma = 6.0 * std::sqrt(2.0) / P;
    p->n3[0] = p->n3[1] = 1;
    p->n3[2] = n;
    p->L3[2] = L;
    p->h[2] = h;
    nlp_status s;
    if ((s = make_fft_len<double>(p, 2 * n, &p->p1d_len))) return s;
    void *d;
    if ((s = alloc_dev(p, &d, sizeof(cpx<double>) * 2 * (size_t)n))) return s;
    p->p1d_work = d;
    if ((s = alloc_dev(p, &d, sizeof(double) * 4))) return s;
    p->p1d_mom = (double *)d;
    p->info.dim = 1;
    p->info.kernel = p->kernel;
    p->info.precision = p->prec;
    p->info.n[0] = p->info.n[1] = 1;
    p->info.n[2] = n;
    p->info.nf[0] = p->info.nf[1] = 1;
    p->info.nf[2] = 2 * n;
    p->info.kmax = P;
    p->info.sigma_poisson = p->sigma;
    p->info.workspace_bytes = p->bytes;
    return NLP_OK;
}

nlp_status eval_1d(nlp_plan_s *p, const double *rho, double *phi) {
    const int n = p->p1d_n;
    const double L = p->grid.L[0], h = p->h[2];
    cpx<double> *work = (cpx<double> *)p->p1d_work;
    cudaStream_t st = p->stream;
    k_p1d_moments<<<1, kMomThreads, 0, st>>>(rho, n, L, h, work, p->p1d_mom);
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    if (launch_fft_contig<double>(work, 1, p->p1d_len, -1, 1.0, st) != cudaSuccess) return NLP_ERR_CUDA;
    k_p1d_w<<<(2 * n + 255) / 256, 256, 0, st>>>(work, p->p1d_mom, n, h, p->p1d_P, p->sigma);
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    if (launch_fft_contig<double>(work, 1, p->p1d_len, +1, 1.0, st) != cudaSuccess) return NLP_ERR_CUDA;
    k_p1d_u1<<<(n + 255) / 256, 256, 0, st>>>(phi, work, p->p1d_mom, n, L, h, p->sigma);
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    return NLP_OK;
}

}  // namespace nlp
