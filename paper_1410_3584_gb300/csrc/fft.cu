// Hand-written FFT passes for the oversampled grids of the NUFFT (and the plain grids of
// the gradient flow / time splitting).  Mixed radix 2/3/4/5 Stockham autosort in shared
// memory; one CTA transforms a batch of lines.  Twiddles are FP64-built tables rounded
// to the plan precision.
//
// Layout convention: a 3D array [n0][n1][n2] with the last axis contiguous; the real-to-
// complex half spectrum along the last axis has nh = N2/2 + 1 entries.  2D arrays are
// handled as 3D with n0 = 1.
#include "common.cuh"
#include "launch.h"
#include "fft_dev.cuh"

namespace nlp {
// ------------------------------------------------------------------ launchers
template <typename T> static int lines_per_block(int N) {
    // keep 2 * N * (nb+1) complex + twiddles within 160 KB
    const int budget = 160 * 1024 / (int)sizeof(cpx<T>);
    int nb = 16;
    while (nb > 1 && 2 * N * (nb + 1) + N > budget) nb >>= 1;
    return nb;
}

template <typename T> static size_t fft_smem_bytes(int N, int nb) {
    return sizeof(cpx<T>) * ((size_t)N + 2 * (size_t)N * (nb + 1));
}

// line pairs per block of the register-engine R2C / C2R kernels
template <typename T> constexpr int pairs_per_block() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T>
cudaError_t launch_fwd_r2c(const T *rho, const DevPlan<T> &P, cudaStream_t st) {
    if (P.len[2].nrad_reg > 0) {
        constexpr int NBC = pairs_per_block<T>();
        const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
        const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * 2;
        allow_smem<k_fwd_r2c_reg<T, NBC>>();
        k_fwd_r2c_reg<T, NBC><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * 16, sm, st>>>(rho, P);
        return cudaGetLastError();
    }
    const int N = P.len[2].N;
    const int nb = lines_per_block<T>(N);
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = fft_smem_bytes<T>(N, nb);
    allow_smem<k_fwd_r2c<T>>();
    k_fwd_r2c<T><<<(unsigned)((npairs + nb - 1) / nb), 256, sm, st>>>(rho, P, nb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inv_c2r(T *phi, const DevPlan<T> &P, cudaStream_t st) {
    if (P.len[2].nrad_reg > 0) {
        constexpr int NBC = pairs_per_block<T>();
        const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
        const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * (P.len[2].nrad_reg > 2 ? 2 : 1);
        allow_smem<k_inv_c2r_reg<T, NBC>>();
        k_inv_c2r_reg<T, NBC><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * 16, sm, st>>>(phi, P);
        return cudaGetLastError();
    }
    const int N = P.len[2].N;
    const int nb = lines_per_block<T>(N);
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = fft_smem_bytes<T>(N, nb);
    allow_smem<k_inv_c2r<T>>();
    k_inv_c2r<T><<<(unsigned)((npairs + nb - 1) / nb), 256, sm, st>>>(phi, P, nb);
    return cudaGetLastError();
}

// columns per block of the register engine: 16 x 8 B (FP32) or 8 x 16 B (FP64) = 128 B rows
template <typename T> constexpr int cols_per_block() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T>
cudaError_t launch_fft_strided(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int sign,
                               cudaStream_t st) {
    if (L.nrad_reg > 0) {
        constexpr int NBC = cols_per_block<T>();
        const size_t sm = sizeof(cpx<T>) * (size_t)L.N * NBC * (L.nrad_reg > 2 ? 2 : 1);
        const int ctiles = (d.ncol + NBC - 1) / NBC;
        const unsigned grid = (unsigned)((int64_t)d.nouter * ctiles);
        if (sign < 0) {
            allow_smem<k_fft_cols<T, -1, NBC>>();
            k_fft_cols<T, -1, NBC><<<grid, NBC * 16, sm, st>>>(data, d, L);
        } else {
            allow_smem<k_fft_cols<T, +1, NBC>>();
            k_fft_cols<T, +1, NBC><<<grid, NBC * 16, sm, st>>>(data, d, L);
        }
        return cudaGetLastError();
    }
    const int nb = d.ncol >= 16 ? lines_per_block<T>(L.N) : d.ncol;
    const size_t sm = fft_smem_bytes<T>(L.N, nb);
    const int ctiles = (d.ncol + nb - 1) / nb;
    const unsigned grid = (unsigned)((int64_t)d.nouter * ctiles);
    if (sign < 0) {
        allow_smem<k_fft_strided<T, -1>>();
        k_fft_strided<T, -1><<<grid, 256, sm, st>>>(data, d, L, nb);
    } else {
        allow_smem<k_fft_strided<T, +1>>();
        k_fft_strided<T, +1><<<grid, 256, sm, st>>>(data, d, L, nb);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_contig(cpx<T> *data, int64_t nlines, const FftLen<T> &L, int sign, T post, cudaStream_t st) {
    const int nb = lines_per_block<T>(L.N);
    const size_t sm = fft_smem_bytes<T>(L.N, nb);
    const unsigned grid = (unsigned)((nlines + nb - 1) / nb);
    if (sign < 0) {
        allow_smem<k_fft_contig<T, -1>>();
        k_fft_contig<T, -1><<<grid, 256, sm, st>>>(data, nlines, L, nb, post);
    } else {
        allow_smem<k_fft_contig<T, +1>>();
        k_fft_contig<T, +1><<<grid, 256, sm, st>>>(data, nlines, L, nb, post);
    }
    return cudaGetLastError();
}
template cudaError_t launch_fft_contig<float>(cpx<float> *, int64_t, const FftLen<float> &, int, float, cudaStream_t);
template cudaError_t launch_fft_contig<double>(cpx<double> *, int64_t, const FftLen<double> &, int, double, cudaStream_t);

template cudaError_t launch_fwd_r2c<float>(const float *, const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_fwd_r2c<double>(const double *, const DevPlan<double> &, cudaStream_t);
template cudaError_t launch_inv_c2r<float>(float *, const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_inv_c2r<double>(double *, const DevPlan<double> &, cudaStream_t);
template cudaError_t launch_fft_strided<float>(cpx<float> *, const StridedDesc &, const FftLen<float> &, int, cudaStream_t);
template cudaError_t launch_fft_strided<double>(cpx<double> *, const StridedDesc &, const FftLen<double> &, int, cudaStream_t);

}  // namespace nlp
