// Plan object behind the opaque nlp_plan handle.
#pragma once
#include <vector>
#include <string>

#include "common.cuh"

struct nlp_plan_s {
    nlp_grid grid{};          // as given (dim 1, 2 or 3)
    nlp_kernel kernel{};
    nlp_precision prec{};
    nlp_opts opts{};
    cudaStream_t stream = nullptr;
    nlp_plan_info info{};
    double h[3] = {1, 1, 1};  // collapsed 3D view (2D: axis 0 is a dummy of size 1)
    int n3[3] = {1, 1, 1};
    double L3[3] = {1, 1, 1};
    nlp::DevPlan<float> pf{};
    nlp::DevPlan<double> pd{};
    std::vector<void *> allocs;         // every device allocation of the plan
    size_t bytes = 0;
    // 2D Poisson (Algorithm 1) extras
    double sigma = 0;
    double sigma_u1 = 0;   // width of u_1's Gaussian (sigma, or widened by the method-2 partition)
    double *d_pois = nullptr;           // per-node FP64 data: kx, ky, r (hemisphere order)
    double *d_red = nullptr;            // FP64 reduction scratch
    int red_blocks = 0;
    // gradient flow / time splitting workspace (plain grid FFTs), allocated on first use
    void *d_work = nullptr;             // host struct describing the work buffers
    void (*work_free)(void *) = nullptr;
    size_t work_bytes = 0;
    void *d_host_io = nullptr;          // device buffers for nlp_eval_potential_host
    // FFT lengths of the plain (non-oversampled) grid for GF / TS
    nlp::FftLen<float> plain_f[3]{};
    nlp::FftLen<double> plain_d[3]{};
    bool plain_ready = false;
    // stage timers (CUDA events on the plan stream), off unless enabled
    int timing = 0;
    int nev = 0;
    cudaEvent_t ev[32] = {};
    int ev_stage[32] = {};
    // improved algorithm (method 2): I_2 is the NUFFT of pf / pd (small ball), I_1 the FFT
    // convolution described by pf1 / pd1 (analytic multiplier, accumulating into phi)
    int split = 0;
    double split_a = 0, split_k2 = 0;   // partition scale (a, or l for the erfc partition), ball radius
    int split_erfc = 0;                 // 1: p = erfc(|k|/l) (2D Coulomb), 0: p = exp(-|k|^2/a)
    nlp::DevPlan<float> pf1{};
    nlp::DevPlan<double> pd1{};
    // 1D Poisson (NLP_POISSON_1D): FFT length 2n, zero-padded complex work array, FP64 moments
    int p1d_n = 0;
    double p1d_P = 0;
    nlp::FftLen<double> p1d_len{};
    void *p1d_work = nullptr;
    double *p1d_mom = nullptr;
};

namespace nlp {
// host utilities shared by the plan and the tests' debug exports
void gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w);
void es_params(double tol, int *w, double *beta);
double es_fourier(double xi, int w, double beta);
nlp_status alloc_dev(nlp_plan_s *p, void **ptr, size_t bytes);
template <typename T> nlp_status make_fft_len(nlp_plan_s *p, int N, FftLen<T> *out);
// radix sequences of an FFT length: shared-memory Stockham engine (4, 2, 3, 5) and register
// engine (16s, one 8/4/2, 3s, 5s); false if N has another prime factor
bool factor_radices(int N, int *rad, int *nrad);
bool factor_radices_reg(int N, int *rad, int *nrad);
}  // namespace nlp
