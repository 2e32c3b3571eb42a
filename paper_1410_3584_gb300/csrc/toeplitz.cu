// Precomputed-kernel evaluation (plan option method = 1).
//
// The quadrature sum of Eq. (ifft) on the grid is a discrete convolution: expanding
// rho-hat_j = h^d sum_i' rho_i' e^{-i k_j . x_i'} and exchanging the finite sums gives
//     phi_i = sum_i' K(i - i') rho_i',   K(m) = sum_j omega_j cos(k_j . m h),
// with omega_j = h^d (2 pi)^{-d} w_j |k_j|^{d-1} U-hat(k_j) the node weights of the plan (the
// node set is symmetric, so the sum over e^{+} is real).  K is needed for m in (-n, n)^d.
// Plan time: K on the doubled grid by a type-1 NUFFT of the weights alone (spreading with
// rho-hat := 1 on an auxiliary plan of 2n points per axis, same h, same nodes), then its
// spectrum K-hat on the 2n grid.  Evaluation: zero-pad rho to 2n, forward FFT, multiply by
// K-hat, inverse FFT, crop -- the aperiodic convolution, exact because |i - i'| < n.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace nlp {

nlp_status plan_build(nlp_plan_s *p);

template <typename T> __global__ void k_mul_spec(cpx<T> *F, const cpx<T> *K, int64_t M) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < M; q += (int64_t)gridDim.x * blockDim.x)
        F[q] = F[q] * K[q];
}

template <typename T> cudaError_t launch_mul_spec(cpx<T> *F, const cpx<T> *K, int64_t M, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((M + 255) / 256, 152 * 16);
    k_mul_spec<T><<<blocks, 256, 0, st>>>(F, K, M);
    return cudaGetLastError();
}
template cudaError_t launch_mul_spec<float>(cpx<float> *, const cpx<float> *, int64_t, cudaStream_t);
template cudaError_t launch_mul_spec<double>(cpx<double> *, const cpx<double> *, int64_t, cudaStream_t);

template <typename T> __global__ void k_scale_spec(cpx<T> *F, int64_t M, double s) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < M; q += (int64_t)gridDim.x * blockDim.x)
        F[q] = scale(F[q], (T)s);
}

template <typename T> static nlp_status ones_table(nlp_plan_s *p, int n, const T **out) {
    std::vector<T> v(n, (T)1);
    void *d;
    nlp_status s = alloc_dev(p, &d, sizeof(T) * n);
    if (s) return s;
    cudaMemcpy(d, v.data(), sizeof(T) * n, cudaMemcpyHostToDevice);
    *out = (const T *)d;
    return NLP_OK;
}

template <typename T> static DevPlan<T> &dev_of(nlp_plan_s *p);
template <> DevPlan<float> &dev_of<float>(nlp_plan_s *p) { return p->pf; }
template <> DevPlan<double> &dev_of<double>(nlp_plan_s *p) { return p->pd; }

template <typename T> static nlp_status build_kernel(nlp_plan_s *p) {
    DevPlan<T> &D = dev_of<T>(p);
    cudaStream_t st = p->stream;
    // ---- auxiliary plan: 2n points per axis, same spacing, same nodes and weights
    nlp_plan_s *aux = new (std::nothrow) nlp_plan_s();
    if (!aux) return NLP_ERR_OOM;
    aux->grid = p->grid;
    for (int a = 0; a < p->grid.dim; ++a) {
        aux->grid.n[a] = 2 * p->grid.n[a];
        aux->grid.L[a] = 2.0 * p->grid.L[a];
    }
    aux->kernel = p->kernel;
    aux->prec = p->prec;
    aux->opts = p->opts;
    aux->opts.kmax = p->info.kmax;
    aux->opts.n_r = p->info.n_r;
    aux->opts.n_theta = p->grid.dim == 3 ? p->info.n_theta : 0;
    aux->opts.n_phi = p->info.n_phi;
    aux->opts.spread_variant = 1;
    aux->opts.method = 0;
    aux->opts.tile = 0;
    aux->stream = st;
    nlp_status s = plan_build(aux);
    auto free_aux = [&]() {
        cudaStreamSynchronize(st);
        for (void *a : aux->allocs) cudaFree(a);
        delete aux;
    };
    if (s) { free_aux(); return s; }
    DevPlan<T> &A = dev_of<T>(aux);
    // K on the aux grid: type-1 of the weights (rho-hat := 1): spread, inverse FFT, deconvolve
    void *dK;
    const size_t NK = (size_t)A.n[0] * A.n[1] * A.n[2];
    if ((s = alloc_dev(aux, &dK, sizeof(T) * NK))) { free_aux(); return s; }
    A.ones_mode = 1;
    const int64_t nhA = A.nh;
    if (launch_interp_spread<T>(A, st) != cudaSuccess || launch_window_sum<T>(A, st) != cudaSuccess ||
        launch_combine<T>(A, st) != cudaSuccess) {
        free_aux();
        return NLP_ERR_CUDA;
    }
    const bool three = p->grid.dim == 3;
    StridedDesc b1{};
    b1.n_in = A.nf[1]; b1.n_out = A.n[1]; b1.es = nhA; b1.ncol = (int)nhA;
    b1.nouter = three ? A.n[0] : 1; b1.os = (int64_t)A.nf[1] * nhA;
    b1.outer_map_n = three ? A.n[0] : 0; b1.outer_map_N = A.nf[0];
    if (three) {
        StridedDesc b0{};
        b0.n_in = A.nf[0]; b0.n_out = A.n[0]; b0.es = (int64_t)A.nf[1] * nhA; b0.ncol = (int)nhA;
        b0.nouter = A.nf[1]; b0.os = nhA;
        if (launch_fft_strided<T>(A.G, b0, A.len[0], +1, st) != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }
    }
    if (launch_fft_strided<T>(A.G, b1, A.len[1], +1, st) != cudaSuccess ||
        launch_inv_c2r<T>((T *)dK, A, st) != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }

    // ---- K-hat on the main fine grid (2n): R2C of K placed with m at position m mod 2n.
    // The aux grid index i holds m = i - n; the R2C kernel puts index i of an N-point line at
    // (i - N/2) mod N, which for N = 2n is exactly m mod 2n.
    DevPlan<T> K = D;
    for (int a = 0; a < 3; ++a) {
        K.n[a] = D.nf[a];
        if ((s = ones_table<T>(p, D.nf[a], &K.deconv[a]))) { free_aux(); return s; }
    }
    void *dKh;
    const size_t spec = (size_t)D.nf[0] * D.nf[1] * D.nh;
    if ((s = alloc_dev(p, &dKh, sizeof(cpx<T>) * spec))) { free_aux(); return s; }
    K.F = K.G = (cpx<T> *)dKh;
    if (launch_fwd_r2c<T>((const T *)dK, K, st) != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }
    StridedDesc f1{};
    f1.n_in = D.nf[1]; f1.n_out = D.nf[1]; f1.es = D.nh; f1.ncol = D.nh;
    f1.nouter = D.nf[0]; f1.os = (int64_t)D.nf[1] * D.nh;
    if (D.nf[1] > 1 && launch_fft_strided<T>(K.F, f1, D.len[1], -1, st) != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }
    if (three) {
        StridedDesc f0{};
        f0.n_in = D.nf[0]; f0.n_out = D.nf[0]; f0.es = (int64_t)D.nf[1] * D.nh; f0.ncol = D.nh;
        f0.nouter = D.nf[1]; f0.os = D.nh;
        if (launch_fft_strided<T>(K.F, f0, D.len[0], -1, st) != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }
    }
    // the unnormalised inverse transform of the evaluation carries a factor prod(2n)
    double nfp = 1.0;
    for (int a = 0; a < 3; ++a) nfp *= D.nf[a];
    k_scale_spec<T><<<152 * 8, 256, 0, st>>>(K.F, (int64_t)spec, 1.0 / nfp);
    if (cudaGetLastError() != cudaSuccess) { free_aux(); return NLP_ERR_CUDA; }
    free_aux();
    // ---- evaluation descriptor: unit deconvolution, in-place spectrum, K-hat
    DevPlan<T> &E = dev_of<T>(p);
    for (int a = 0; a < 3; ++a)
        if ((s = ones_table<T>(p, D.n[a], &E.deconv[a]))) return s;
    E.G = E.F;
    E.Khat = (const cpx<T> *)dKh;
    return cudaDeviceSynchronize() == cudaSuccess ? NLP_OK : NLP_ERR_CUDA;
}

nlp_status build_toeplitz(nlp_plan_s *p) {
    if (p->kernel == NLP_POISSON_2D) return NLP_ERR_UNSUPPORTED;
    return p->prec == NLP_FP64 ? build_kernel<double>(p) : build_kernel<float>(p);
}

}  // namespace nlp
