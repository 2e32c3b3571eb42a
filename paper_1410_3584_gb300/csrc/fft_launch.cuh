// Launchers of the hand-written FFT passes (included once per precision by fft_f32.cu and
// fft_f64.cu, which instantiate them).
//
// Hand-written FFT passes for the oversampled grids of the NUFFT (and the plain grids of
// the gradient flow / time splitting).  Lengths with a register-engine factorisation run on
// the register radix engine (k_fft_cols, k_fwd_r2c_reg, k_inv_c2r_reg); the mixed radix
// 2/3/4/5 shared-memory Stockham kernels remain for descriptors built without it.  One CTA
// transforms a batch of lines.  Twiddles are FP64-built tables rounded to the plan precision.
//
// Layout convention: a 3D array [n0][n1][n2] with the last axis contiguous; the real-to-
// complex half spectrum along the last axis has nh = N2/2 + 1 entries.  2D arrays are
// handled as 3D with n0 = 1.
#pragma once
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

// Lines per block of the register-engine kernels: 16 (FP32) / 8 (FP64) so that one position of
// a block's lines is a 128-byte row, halved while the shared memory of a block would exceed
// kRegSmemBudget (long lines, e.g. N = 2048).  Below kRegMinLines lines per block (16
// threads each) a block is too small to hide its latencies and the pass runs on the 256-thread
// shared-memory Stockham kernels instead (measured on 2D 2048-point lines: 2x faster in FP32
// C2R, 2.5x in every FP64 pass).
constexpr size_t kRegSmemBudget = 100 * 1024;
constexpr int kRegMinLines = 4;
template <typename T> constexpr int lines_max() { return sizeof(T) == 4 ? 16 : 8; }
static int pick_lines(int nmax, size_t bytes_per_line) {
    int nb = nmax;
    while (nb > 1 && bytes_per_line * nb > kRegSmemBudget) nb >>= 1;
    return nb;
}

// Last-axis lines too long for 16 threads a line pair (N >= 1024): 128 threads a pair (one
// radix-16 butterfly each per pass), one (FP64) or two (FP32) pairs per block, two shared
// buffers of a padded line each.
template <typename T> static bool long_lines_reg(const FftLen<T> &L) { return L.N >= 1024 && L.N <= 4096; }
template <typename T> constexpr int long_pairs() { return sizeof(T) == 4 ? 2 : 1; }
template <typename T> static cudaError_t r2c_reg_long(const T *rho, const DevPlan<T> &P, cudaStream_t st) {
    constexpr int NBC = long_pairs<T>(), TPC = 128;
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * 2;
    if (FixedLen<Rad2048>::match(P.len[2])) {   // radix sequence fixed at compile time
        allow_smem<k_fwd_r2c_reg<T, NBC, TPC, Rad2048>>();
        k_fwd_r2c_reg<T, NBC, TPC, Rad2048><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * TPC, sm, st>>>(rho, P);
        return cudaGetLastError();
    }
    allow_smem<k_fwd_r2c_reg<T, NBC, TPC>>();
    k_fwd_r2c_reg<T, NBC, TPC><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * TPC, sm, st>>>(rho, P);
    return cudaGetLastError();
}
template <typename T> static cudaError_t c2r_reg_long(T *phi, const DevPlan<T> &P, cudaStream_t st) {
    constexpr int NBC = long_pairs<T>(), TPC = 128;
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * 2;
    if (FixedLen<Rad2048>::match(P.len[2])) {
        allow_smem<k_inv_c2r_reg<T, NBC, TPC, Rad2048>>();
        k_inv_c2r_reg<T, NBC, TPC, Rad2048><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * TPC, sm, st>>>(phi, P);
        return cudaGetLastError();
    }
    allow_smem<k_inv_c2r_reg<T, NBC, TPC>>();
    k_inv_c2r_reg<T, NBC, TPC><<<(unsigned)((npairs + NBC - 1) / NBC), NBC * TPC, sm, st>>>(phi, P);
    return cudaGetLastError();
}

// Calls fn(FL{}) with the radix sequence of L when it has compile-time kernels (FP32: the
// upsampled lengths 128, 192, 256, 320, 384 of 64^3 ... 192^3 grids; FP64: 256) and returns
// true; false otherwise.
template <typename T, class Fn> static bool with_fixed_len(const FftLen<T> &L, Fn &&fn) {
    if (FixedLen<Rad256>::match(L)) { fn(Rad256{}); return true; }
    if constexpr (sizeof(T) == 4) {
        if (FixedLen<Rad128>::match(L)) { fn(Rad128{}); return true; }
        if (FixedLen<Rad192>::match(L)) { fn(Rad192{}); return true; }
        if (FixedLen<Rad320>::match(L)) { fn(Rad320{}); return true; }
        if (FixedLen<Rad384>::match(L)) { fn(Rad384{}); return true; }
    }
    return false;
}

template <typename T, int NBC> static cudaError_t r2c_reg(const T *rho, const DevPlan<T> &P, cudaStream_t st) {
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * (r2c_inplace(P.len[2]) ? 1 : 2);
    const unsigned grid = (unsigned)((npairs + NBC - 1) / NBC);
    if constexpr (NBC == lines_max<T>()) {   // sizes fixed at compile time
        cudaError_t e = cudaSuccess;
        if (with_fixed_len(P.len[2], [&](auto fl) {
                using FL = decltype(fl);
                allow_smem<k_fwd_r2c_reg<T, NBC, 16, FL>>();
                k_fwd_r2c_reg<T, NBC, 16, FL><<<grid, NBC * 16, sm, st>>>(rho, P);
                e = cudaGetLastError();
            }))
            return e;
    }
    allow_smem<k_fwd_r2c_reg<T, NBC>>();
    k_fwd_r2c_reg<T, NBC><<<grid, NBC * 16, sm, st>>>(rho, P);
    return cudaGetLastError();
}
template <typename T, int NBC> static cudaError_t c2r_reg(T *phi, const DevPlan<T> &P, cudaStream_t st) {
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = sizeof(cpx<T>) * (size_t)NBC * line_ld(P.len[2].N) * (P.len[2].nrad_reg > 2 ? 2 : 1);
    const unsigned grid = (unsigned)((npairs + NBC - 1) / NBC);
    if constexpr (NBC == lines_max<T>()) {
        cudaError_t e = cudaSuccess;
        if (with_fixed_len(P.len[2], [&](auto fl) {
                using FL = decltype(fl);
                allow_smem<k_inv_c2r_reg<T, NBC, 16, FL>>();
                k_inv_c2r_reg<T, NBC, 16, FL><<<grid, NBC * 16, sm, st>>>(phi, P);
                e = cudaGetLastError();
            }))
            return e;
    }
    allow_smem<k_inv_c2r_reg<T, NBC>>();
    k_inv_c2r_reg<T, NBC><<<grid, NBC * 16, sm, st>>>(phi, P);
    return cudaGetLastError();
}
template <typename T, int NBC>
static cudaError_t cols_reg(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int sign, cudaStream_t st) {
    const size_t sm = sizeof(cpx<T>) * (size_t)L.N * NBC * (L.nrad_reg > 2 ? 2 : 1);
    const unsigned grid = (unsigned)cols_blocks<T, NBC>(d);
    if constexpr (NBC == lines_max<T>()) {
        cudaError_t e = cudaSuccess;
        if (with_fixed_len(L, [&](auto fl) {
                using FL = decltype(fl);
                if (sign < 0) {
                    allow_smem<k_fft_cols<T, -1, NBC, FL>>();
                    k_fft_cols<T, -1, NBC, FL><<<grid, NBC * 16, sm, st>>>(data, d, L);
                } else {
                    allow_smem<k_fft_cols<T, +1, NBC, FL>>();
                    k_fft_cols<T, +1, NBC, FL><<<grid, NBC * 16, sm, st>>>(data, d, L);
                }
                e = cudaGetLastError();
            }))
            return e;
    }
    if (sign < 0) {
        allow_smem<k_fft_cols<T, -1, NBC>>();
        k_fft_cols<T, -1, NBC><<<grid, NBC * 16, sm, st>>>(data, d, L);
    } else {
        allow_smem<k_fft_cols<T, +1, NBC>>();
        k_fft_cols<T, +1, NBC><<<grid, NBC * 16, sm, st>>>(data, d, L);
    }
    return cudaGetLastError();
}

// calls F<NBC>() for the chosen power of two NBC <= lines_max<T>()
#define NLP_LINES_SWITCH(T, nb, CALL)                          \
    switch (nb) {                                              \
        case 16: if constexpr (lines_max<T>() >= 16) return CALL(16); [[fallthrough]]; \
        case 8: return CALL(8);                                \
        case 4: return CALL(4);                                \
        case 2: return CALL(2);                                \
        default: return CALL(1);                               \
    }

template <typename T>
cudaError_t launch_fwd_r2c(const T *rho, const DevPlan<T> &P, cudaStream_t st) {
    if (P.len[2].nrad_reg > 0) {
        const int nb = pick_lines(lines_max<T>(), sizeof(cpx<T>) * (size_t)line_ld(P.len[2].N) *
                                                      (r2c_inplace(P.len[2]) ? 1 : 2));
        if (nb >= kRegMinLines) {
#define NLP_CALL(K) r2c_reg<T, K>(rho, P, st)
            NLP_LINES_SWITCH(T, nb, NLP_CALL)
#undef NLP_CALL
        }
        if (long_lines_reg(P.len[2])) return r2c_reg_long<T>(rho, P, st);
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
        const int nb = pick_lines(lines_max<T>(), sizeof(cpx<T>) * (size_t)line_ld(P.len[2].N) *
                                                      (P.len[2].nrad_reg > 2 ? 2 : 1));
        if (nb >= kRegMinLines) {
#define NLP_CALL(K) c2r_reg<T, K>(phi, P, st)
            NLP_LINES_SWITCH(T, nb, NLP_CALL)
#undef NLP_CALL
        }
        if (long_lines_reg(P.len[2])) return c2r_reg_long<T>(phi, P, st);
    }
    const int N = P.len[2].N;
    const int nb = lines_per_block<T>(N);
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const size_t sm = fft_smem_bytes<T>(N, nb);
    allow_smem<k_inv_c2r<T>>();
    k_inv_c2r<T><<<(unsigned)((npairs + nb - 1) / nb), 256, sm, st>>>(phi, P, nb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_strided(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int sign,
                               cudaStream_t st) {
    if (L.nrad_reg > 0) {
        const int nb = pick_lines(lines_max<T>(), sizeof(cpx<T>) * (size_t)L.N * (L.nrad_reg > 2 ? 2 : 1));
        if (nb >= kRegMinLines) {
#define NLP_CALL(K) cols_reg<T, K>(data, d, L, sign, st)
            NLP_LINES_SWITCH(T, nb, NLP_CALL)
#undef NLP_CALL
        }
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

// The register engine takes a column pass when a block of at least kRegMinLines columns fits.
template <typename T> bool cols_on_reg_engine(const FftLen<T> &L) {
    return L.nrad_reg > 0 &&
           pick_lines(lines_max<T>(), sizeof(cpx<T>) * (size_t)L.N * (L.nrad_reg > 2 ? 2 : 1)) >= kRegMinLines;
}

template <typename T, int SGN, int STEP, int TPC>
static cudaError_t four_step_tpc(const cpx<T> *in, cpx<T> *out, const StridedDesc &d, const DevPlan<T> &D,
                                 cudaStream_t st) {
    constexpr int NBC = 256 / TPC;
    const FftLen<T> &Ls = D.len4[STEP - 1];
    const int N1 = D.len4[0].N, N2 = D.len4[1].N;
    const int64_t cols = (int64_t)(STEP == 1 ? N2 : N1) * d.ncol;
    const size_t sm = cols_smem_bytes<T>(Ls, NBC);
    const unsigned grid = (unsigned)((cols + NBC - 1) / NBC);
    // sub-lines with a compile-time radix sequence: 64 points (step 1) and 32 points (either step)
    if constexpr (TPC == 4 && STEP == 1)
        if (FixedLen<Rad64>::match(Ls)) {
            allow_smem<k_fft_four<T, SGN, NBC, TPC, STEP, Rad64>>();
            k_fft_four<T, SGN, NBC, TPC, STEP, Rad64><<<grid, 256, sm, st>>>(in, out, d, D.len[1], Ls, N1, N2);
            return cudaGetLastError();
        }
    if constexpr (TPC == 2)
        if (FixedLen<Rad32>::match(Ls)) {
            allow_smem<k_fft_four<T, SGN, NBC, TPC, STEP, Rad32>>();
            k_fft_four<T, SGN, NBC, TPC, STEP, Rad32><<<grid, 256, sm, st>>>(in, out, d, D.len[1], Ls, N1, N2);
            return cudaGetLastError();
        }
    allow_smem<k_fft_four<T, SGN, NBC, TPC, STEP>>();
    k_fft_four<T, SGN, NBC, TPC, STEP><<<(unsigned)((cols + NBC - 1) / NBC), 256, sm, st>>>(in, out, d, D.len[1], Ls,
                                                                                          N1, N2);
    return cudaGetLastError();
}

// threads per sub-line: the power of two nearest below N_sub / 16, 1..8
template <typename T, int SGN, int STEP>
static cudaError_t four_step(const cpx<T> *in, cpx<T> *out, const StridedDesc &d, const DevPlan<T> &D,
                             cudaStream_t st) {
    const int n = D.len4[STEP - 1].N / 16;
    if (n >= 8) return four_step_tpc<T, SGN, STEP, 8>(in, out, d, D, st);
    if (n >= 4) return four_step_tpc<T, SGN, STEP, 4>(in, out, d, D, st);
    if (n >= 2) return four_step_tpc<T, SGN, STEP, 2>(in, out, d, D, st);
    return four_step_tpc<T, SGN, STEP, 1>(in, out, d, D, st);
}

// the 2D axis-1 pass as the four-step decomposition: in -> S4 (step 1) -> out (step 2)
template <typename T>
cudaError_t launch_fft_four(const cpx<T> *in, cpx<T> *out, const StridedDesc &d, const DevPlan<T> &D, int sign,
                            cudaStream_t st) {
    if (!D.four || !D.S4 || d.nouter != 1) return cudaErrorInvalidValue;
    cudaError_t e = sign < 0 ? four_step<T, -1, 1>(in, D.S4, d, D, st) : four_step<T, +1, 1>(in, D.S4, d, D, st);
    if (e != cudaSuccess) return e;
    return sign < 0 ? four_step<T, -1, 2>(D.S4, out, d, D, st) : four_step<T, +1, 2>(D.S4, out, d, D, st);
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
}  // namespace nlp
