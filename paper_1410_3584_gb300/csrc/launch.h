// Host-side launchers of the device kernels (one per kernel family).
#pragma once
#include "common.cuh"

namespace nlp {

// Dynamic shared-memory opt-in limit of the current device.  Every kernel that may take more
// than the default 48 KB is given, once, the whole opt-in limit minus its static shared
// memory (not the size of the launch at hand), so launches of different sizes from several
// host threads never change a limit that another thread's launch relies on.  The setup runs
// on the device current at the first call.
int max_dyn_smem();
template <auto Kernel> inline cudaError_t allow_smem() {
    static const cudaError_t status = [] {
        cudaFuncAttributes a{};
        cudaError_t e = cudaFuncGetAttributes(&a, Kernel);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    max_dyn_smem() - (int)a.sharedSizeBytes);
    }();
    return status;
}

// One strided C2C FFT pass (see k_fft_strided).
struct StridedDesc {
    int n_in, n_out;      // input / output windows (>= N means the whole line)
    int64_t es;           // element stride along the transformed axis (complex units)
    int ncol;             // contiguous columns per outer line
    int nouter;           // outer lines
    int64_t os;           // stride between outer lines
    int outer_map_n;      // > 0: outer index o addresses line (o - outer_map_n/2) mod outer_map_N
    int outer_map_N;
    void *out;            // null: in place; else the output array (same layout as the input)
};

template <typename T> cudaError_t launch_fwd_r2c(const T *rho, const DevPlan<T> &P, cudaStream_t st);
template <typename T> cudaError_t launch_inv_c2r(T *phi, const DevPlan<T> &P, cudaStream_t st);
template <typename T>
cudaError_t launch_fft_strided(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int sign, cudaStream_t st);
template <typename T>
cudaError_t launch_fft_four(const cpx<T> *in, cpx<T> *out, const StridedDesc &d, const DevPlan<T> &D, int sign,
                            cudaStream_t st);
template <typename T> bool cols_on_reg_engine(const FftLen<T> &L);

template <typename T>
cudaError_t launch_fft_contig(cpx<T> *data, int64_t nlines, const FftLen<T> &L, int sign, T post, cudaStream_t st);

// Fused interpolate -> scale -> spread over all node chunks (see spread.cu): each chunk's
// tile window goes to its slot of P.win; launch_combine then writes every cell of G.
template <typename T> cudaError_t launch_interp_spread(const DevPlan<T> &P, cudaStream_t st);
template <typename T> int generic_warps(const DevPlan<T> &P, size_t smem_limit);
template <typename T> size_t interp_spread_smem(const DevPlan<T> &P, int nwarps);
// Register-column variants for 3D (see spread_reg.cu); W = sub-tile edge + w - 1.
template <typename T> bool reg_kernel_supported(int W);
template <typename T> bool warp_kernel_used(int W);   // FP32 one-warp-per-piece kernel
template <typename T> size_t interp_spread_reg_smem(const DevPlan<T> &P, int nwarps_warp_kernel);
template <typename T> cudaError_t launch_interp_spread_reg(const DevPlan<T> &P, cudaStream_t st);
// FP32 plans of the one-warp-per-piece kernels (P.cnode set): interpolation half, before
// launch_interp_spread_reg (which then runs the spreading half)
template <typename T> cudaError_t launch_interp_warp(const DevPlan<T> &P, cudaStream_t st);
template <typename T> cudaError_t launch_window_sum(const DevPlan<T> &P, cudaStream_t st);   // tiles of several chunks
template <typename T> cudaError_t launch_combine(const DevPlan<T> &P, cudaStream_t st);

// 2D Poisson (Algorithm 1) FP64 parts (see poisson2d.cu).  L, h: collapsed 3D view.
template <typename T>
cudaError_t launch_poisson_moments(const T *rho, const DevPlan<T> &P, const double *L, const double *h,
                                   double *part, int nblocks, double *mom, cudaStream_t st);
template <typename T> cudaError_t launch_poisson_origin(const DevPlan<T> &P, double *mom, cudaStream_t st);
template <typename T>
cudaError_t launch_poisson_u1(T *phi, const DevPlan<T> &P, const double *L, const double *h, cudaStream_t st);
// plan time: the u_{1,1}, u_{1,2} table of the grid (3 doubles per point)
cudaError_t launch_u1_table(double *tab, int nx, int ny, const double *L, const double *h, double sigma,
                            cudaStream_t st);

// precomputed-kernel method: F *= K-hat (toeplitz.cu)
template <typename T> cudaError_t launch_mul_spec(cpx<T> *F, const cpx<T> *K, int64_t M, cudaStream_t st);

// plan-time per-node kernel-value table of the register kernels (plan.cu)
template <typename T>
cudaError_t launch_psi_table(T *tab, const T *nd, const uint32_t *no, int64_t M, int w, int Wsub, int Ts, double beta,
                             cudaStream_t st);

}  // namespace nlp
