// FFT device code shared by the single-plan kernels (fft_launch.cuh) and the batched persistent
// kernel (batch.cu): small DFTs, the shared-memory Stockham engine and the per-block bodies
// of the R2C / C2R / strided passes (block index passed explicitly).
#pragma once
#include <type_traits>
#include "common.cuh"
#include "launch.h"

namespace nlp {

// ------------------------------------------------------------------ small DFTs
template <typename T, int SGN>
__device__ __forceinline__ void dft2(cpx<T> *v) {
    cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}
template <typename T, int SGN>
__device__ __forceinline__ void dft4(cpx<T> *v) {
    cpx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = mul_i(v[1] - v[3], SGN);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
}
template <typename T, int SGN>
__device__ __forceinline__ void dft3(cpx<T> *v) {
    const T s = (T)(SGN * 0.86602540378443864676);   // sign * sin(2 pi / 3)
    cpx<T> t = v[1] + v[2], u = v[1] - v[2];
    cpx<T> m = v[0] - scale(t, (T)0.5);
    cpx<T> iu = mul_i(scale(u, s), 1);
    v[0] = v[0] + t;
    v[1] = m + iu;
    v[2] = m - iu;
}
template <typename T, int SGN>
__device__ __forceinline__ void dft5(cpx<T> *v) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)(SGN * 0.95105651629515357212), s2 = (T)(SGN * 0.58778525229247312917);
    cpx<T> a = v[1] + v[4], b = v[2] + v[3], c = v[1] - v[4], d = v[2] - v[3];
    cpx<T> p1 = v[0] + scale(a, c1) + scale(b, c2);
    cpx<T> p2 = v[0] + scale(a, c2) + scale(b, c1);
    cpx<T> q1 = mul_i(scale(c, s1) + scale(d, s2), 1);
    cpx<T> q2 = mul_i(scale(c, s2) - scale(d, s1), 1);
    v[0] = v[0] + a + b;
    v[1] = p1 + q1;
    v[4] = p1 - q1;
    v[2] = p2 + q2;
    v[3] = p2 - q2;
}

// Batched Stockham FFT of nb lines of length N held as src[i * ldb + b]; ping-pong with
// dst.  Returns the buffer holding the result.  All threads of the block participate.
template <typename T, int SGN>
__device__ cpx<T> *fft_smem(cpx<T> *src, cpx<T> *dst, const FftLen<T> &L, const cpx<T> *tw, int nb,
                            int ldb) {
    const int N = L.N;
    int Ns = 1;
    for (int s = 0; s < L.nrad; ++s) {
        const int R = L.rad[s];
        const int nbf = N / R;
        const int tws = N / (Ns * R);
        for (int q = threadIdx.x; q < nbf * nb; q += blockDim.x) {
            const int b = q % nb;
            const int j = q / nb;
            const int k = j % Ns;
            cpx<T> v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) v[r] = src[(j + r * nbf) * ldb + b];
            if (k) {
#pragma unroll
                for (int r = 1; r < 5; ++r)
                    if (r < R) {
                        cpx<T> t = tw[k * r * tws];
                        if (SGN > 0) t = conj(t);
                        v[r] = v[r] * t;
                    }
            }
            if (R == 4) dft4<T, SGN>(v);
            else if (R == 2) dft2<T, SGN>(v);
            else if (R == 3) dft3<T, SGN>(v);
            else dft5<T, SGN>(v);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) dst[(base + r * Ns) * ldb + b] = v[r];
        }
        __syncthreads();
        cpx<T> *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T> *s_tw, const FftLen<T> &L) {
    for (int i = threadIdx.x; i < L.N; i += blockDim.x) s_tw[i] = L.tw[i];
}

__device__ __forceinline__ int wrapi(int l, int N) {
    int r = l % N;
    return r < 0 ? r + N : r;
}

// ------------------------------------------------------------------ forward R2C lines
// Real grid lines along the last axis (grid index order, n2 points) are multiplied by the
// deconvolution factors, zero-padded to N2 = nf2 (point i goes to (i - n2/2) mod N2),
// transformed (e^{-}), and written as half spectra into F[l0][l1][0..nh), where
// (l0, l1) are the wrapped fine positions of the line.  Two real lines travel as one
// complex line (x1 + i x2) and are separated after the transform.
template <typename T>
__device__ __forceinline__ void fwd_r2c_block(const T *__restrict__ rho, const DevPlan<T> &P, int nb, int bid, unsigned char *smraw) {
    const FftLen<T> &L = P.len[2];
    const int N = L.N, n2 = P.n[2], ldb = nb + 1;
    cpx<T> *s_tw = (cpx<T> *)smraw;
    cpx<T> *A = s_tw + N;
    cpx<T> *B = A + N * ldb;
    load_twiddles(s_tw, L);
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const int64_t p0 = (int64_t)bid * nb;
    // zero padded positions, load window
    for (int q = threadIdx.x; q < N * nb; q += blockDim.x) {
        const int b = q / N, l = q % N;
        // l is the fine position; window point i with (i - n2/2) mod N == l
        int i = l < n2 / 2 ? l + n2 / 2 : l - N + n2 / 2;
        cpx<T> v = mk<T>(0, 0);
        const int64_t p = p0 + b;
        if (p < npairs && i >= 0 && i < n2) {
            const int64_t line0 = 2 * p, line1 = 2 * p + 1;
            const int i0a = (int)(line0 / P.n[1]), i1a = (int)(line0 % P.n[1]);
            const int i0b = (int)(line1 / P.n[1]), i1b = (int)(line1 % P.n[1]);
            const T d2 = P.deconv[2][i];
            v.x = rho[line0 * n2 + i] * (P.deconv[0][i0a] * P.deconv[1][i1a] * d2);
            v.y = rho[line1 * n2 + i] * (P.deconv[0][i0b] * P.deconv[1][i1b] * d2);
        }
        A[l * ldb + b] = v;
    }
    __syncthreads();
    cpx<T> *R = fft_smem<T, -1>(A, B, L, s_tw, nb, ldb);
    const int nh = P.nh;
    for (int q = threadIdx.x; q < nh * nb * 2; q += blockDim.x) {
        const int k = q % nh;
        const int t = q / nh;
        const int b = t >> 1, which = t & 1;
        const int64_t p = p0 + b;
        if (p >= npairs) continue;
        cpx<T> z = R[k * ldb + b];
        cpx<T> zc = conj(R[((N - k) % N) * ldb + b]);
        cpx<T> x = which == 0 ? scale(z + zc, (T)0.5) : mul_i(scale(z - zc, (T)0.5), -1);
        const int64_t line = 2 * p + which;
        const int i0 = (int)(line / P.n[1]), i1 = (int)(line % P.n[1]);
        const int l0 = wrapi(i0 - P.n[0] / 2, P.nf[0]), l1 = wrapi(i1 - P.n[1] / 2, P.nf[1]);
        P.F[((int64_t)l0 * P.nf[1] + l1) * nh + k] = x;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fwd_r2c(const T *__restrict__ rho, DevPlan<T> P, int nb) {
    extern __shared__ unsigned char smraw[];
    fwd_r2c_block<T>(rho, P, nb, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ inverse C2R lines
// Half spectra G[l0][l1][0..nh) of the wrapped fine positions of each output grid line
// are transformed back (e^{+}); the output window point i of the line is fine position
// (i - n2/2) mod N2 and is multiplied by the deconvolution factors.
template <typename T>
__device__ __forceinline__ void inv_c2r_block(T *__restrict__ phi, const DevPlan<T> &P, int nb, int bid, unsigned char *smraw) {
    const FftLen<T> &L = P.len[2];
    const int N = L.N, n2 = P.n[2], ldb = nb + 1, nh = P.nh;
    cpx<T> *s_tw = (cpx<T> *)smraw;
    cpx<T> *A = s_tw + N;
    cpx<T> *B = A + N * ldb;
    load_twiddles(s_tw, L);
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const int64_t p0 = (int64_t)bid * nb;
    for (int q = threadIdx.x; q < nh * nb; q += blockDim.x) {
        const int k = q % nh, b = q / nh;
        const int64_t p = p0 + b;
        cpx<T> x1 = mk<T>(0, 0), x2 = mk<T>(0, 0);
        if (p < npairs) {
            const int64_t la = 2 * p, lb = 2 * p + 1;
            const int l0a = wrapi((int)(la / P.n[1]) - P.n[0] / 2, P.nf[0]);
            const int l1a = wrapi((int)(la % P.n[1]) - P.n[1] / 2, P.nf[1]);
            const int l0b = wrapi((int)(lb / P.n[1]) - P.n[0] / 2, P.nf[0]);
            const int l1b = wrapi((int)(lb % P.n[1]) - P.n[1] / 2, P.nf[1]);
            x1 = P.G[((int64_t)l0a * P.nf[1] + l1a) * nh + k];
            x2 = P.G[((int64_t)l0b * P.nf[1] + l1b) * nh + k];
            if (k == 0 || 2 * k == N) {   // half-spectrum ends of a real line are real
                x1.y = 0;
                x2.y = 0;
            }
        }
        // Z[k] = X1[k] + i X2[k];  Z[N-k] = conj(X1[k]) + i conj(X2[k])
        A[k * ldb + b] = x1 + mul_i(x2, 1);
        if (k != 0 && 2 * k != N) A[(N - k) * ldb + b] = conj(x1) + mul_i(conj(x2), 1);
    }
    __syncthreads();
    cpx<T> *R = fft_smem<T, +1>(A, B, L, s_tw, nb, ldb);
    for (int q = threadIdx.x; q < n2 * nb * 2; q += blockDim.x) {
        const int i = q % n2;
        const int t = q / n2;
        const int b = t >> 1, which = t & 1;
        const int64_t p = p0 + b;
        if (p >= npairs) continue;
        const int l = wrapi(i - n2 / 2, N);
        const cpx<T> z = R[l * ldb + b];
        const int64_t line = 2 * p + which;
        const int i0 = (int)(line / P.n[1]), i1 = (int)(line % P.n[1]);
        const T v = (which == 0 ? z.x : z.y) * (P.deconv[0][i0] * P.deconv[1][i1] * P.deconv[2][i]);
        if (P.accumulate) phi[line * n2 + i] += v;
        else phi[line * n2 + i] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_inv_c2r(T *__restrict__ phi, DevPlan<T> P, int nb) {
    extern __shared__ unsigned char smraw[];
    inv_c2r_block<T>(phi, P, nb, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ strided C2C pass
// Transforms lines along one non-contiguous axis.  Block = (outer line, tile of nb
// contiguous columns).  Input window: n_in points (fine positions (i - n_in/2) mod N, the
// rest treated as zero) or the whole line; output window likewise.
template <typename T, int SGN>
__device__ __forceinline__ void fft_strided_block(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int nb, int bid, unsigned char *smraw) {
    const int N = L.N, ldb = nb + 1;
    cpx<T> *s_tw = (cpx<T> *)smraw;
    cpx<T> *A = s_tw + N;
    cpx<T> *B = A + N * ldb;
    load_twiddles(s_tw, L);
    const int ctiles = (d.ncol + nb - 1) / nb;
    const int o = bid / ctiles;
    const int c0 = (bid % ctiles) * nb;
    const int oo = d.outer_map_n > 0 ? wrapi(o - d.outer_map_n / 2, d.outer_map_N) : o;
    cpx<T> *base = data + (int64_t)oo * d.os + c0;
    cpx<T> *obase = (d.out ? (cpx<T> *)d.out : data) + (int64_t)oo * d.os + c0;
    const int ncl = min(nb, d.ncol - c0);
    if (d.n_in < N) {
        for (int q = threadIdx.x; q < N * nb; q += blockDim.x) A[(q / nb) * ldb + (q % nb)] = mk<T>(0, 0);
        __syncthreads();
    }
    const int nin = d.n_in < N ? d.n_in : N;
    for (int q = threadIdx.x; q < nin * nb; q += blockDim.x) {
        const int b = q % nb, i = q / nb;
        const int l = d.n_in < N ? wrapi(i - d.n_in / 2, N) : i;
        A[l * ldb + b] = b < ncl ? base[(int64_t)l * d.es + b] : mk<T>(0, 0);
    }
    __syncthreads();
    cpx<T> *R = fft_smem<T, SGN>(A, B, L, s_tw, nb, ldb);
    const int nout = d.n_out < N ? d.n_out : N;
    for (int q = threadIdx.x; q < nout * nb; q += blockDim.x) {
        const int b = q % nb, i = q / nb;
        if (b >= ncl) continue;
        const int l = d.n_out < N ? wrapi(i - d.n_out / 2, N) : i;
        obase[(int64_t)l * d.es + b] = R[l * ldb + b];
    }
}

template <typename T, int SGN>
__global__ void __launch_bounds__(256) k_fft_strided(cpx<T> *data, StridedDesc d, FftLen<T> L, int nb) {
    extern __shared__ unsigned char smraw[];
    fft_strided_block<T, SGN>(data, d, L, nb, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ register radix engine
// e^{SGN 2 pi i m / 16} for a compile-time m (after unrolling)
template <typename T, int SGN> __device__ __forceinline__ cpx<T> w16(int m) {
    constexpr double C[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                              0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                              -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                              0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
    const int q = m & 15;
    // sin(2 pi q / 16) = cos(2 pi (q - 4) / 16)
    return mk<T>((T)C[q], (T)(SGN * C[(q + 12) & 15]));
}

template <typename T, int SGN, int R> struct Dft;
template <typename T, int SGN> struct Dft<T, SGN, 2> {
    static __device__ __forceinline__ void run(cpx<T> *v) { dft2<T, SGN>(v); }
};
template <typename T, int SGN> struct Dft<T, SGN, 3> {
    static __device__ __forceinline__ void run(cpx<T> *v) { dft3<T, SGN>(v); }
};
template <typename T, int SGN> struct Dft<T, SGN, 4> {
    static __device__ __forceinline__ void run(cpx<T> *v) { dft4<T, SGN>(v); }
};
template <typename T, int SGN> struct Dft<T, SGN, 5> {
    static __device__ __forceinline__ void run(cpx<T> *v) { dft5<T, SGN>(v); }
};
// DFT of size R1 R2 in registers by one Cooley-Tukey split: n = n1 + R1 n2, k = k2 + R2 k1
template <typename T, int SGN, int R1, int R2> struct DftSplit {
    static __device__ __forceinline__ void run(cpx<T> *v) {
        constexpr int N = R1 * R2;
        cpx<T> y[N];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            cpx<T> s[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) s[n2] = v[n1 + R1 * n2];
            Dft<T, SGN, R2>::run(s);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2)
                y[n1 * R2 + k2] = (n1 * k2 == 0) ? s[k2] : s[k2] * w16<T, SGN>(n1 * k2 * (16 / N));
        }
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            cpx<T> s[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) s[n1] = y[n1 * R2 + k2];
            Dft<T, SGN, R1>::run(s);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[k2 + R2 * k1] = s[k1];
        }
    }
};
template <typename T, int SGN> struct Dft<T, SGN, 8> {
    static __device__ __forceinline__ void run(cpx<T> *v) { DftSplit<T, SGN, 2, 4>::run(v); }
};
template <typename T, int SGN> struct Dft<T, SGN, 16> {
    static __device__ __forceinline__ void run(cpx<T> *v) { DftSplit<T, SGN, 4, 4>::run(v); }
};

// One Stockham pass of radix R over the butterflies j = t, t + tpc, ... of one line:
// inputs src(j + r N/R), twiddles e^{SGN 2 pi i k r / (Ns R)} with k = j mod Ns, outputs
// dst((j / Ns) Ns R + k + r Ns).  src / dst address the line by position.
template <typename T, int SGN, int R, class Src, class Dst>
__device__ __forceinline__ void reg_pass(Src &src, Dst &dst, int N, int Ns, const cpx<T> *__restrict__ tw, int t,
                                         int tpc) {
    const int nbf = N / R, tws = N / (Ns * R);
    const uint32_t mag = Ns > 1 ? 0xFFFFFFFFu / (uint32_t)Ns + 1u : 0u;   // j / Ns = umulhi(j, mag), j Ns < 2^32
    for (int j = t; j < nbf; j += tpc) {
        cpx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src(j + r * nbf);
        int jq = j, k = 0;
        if (Ns > 1) {
            jq = (int)__umulhi((uint32_t)j, mag);
            k = j - jq * Ns;
        }
        if (k) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                cpx<T> w = tw[k * r * tws];
                if (SGN > 0) w = conj(w);
                v[r] = v[r] * w;
            }
        }
        Dft<T, SGN, R>::run(v);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst(base + r * Ns, v[r]);
    }
}

template <typename T, int SGN, class Src, class Dst>
__device__ __forceinline__ void reg_pass_any(int R, Src &src, Dst &dst, int N, int Ns, const cpx<T> *tw, int t,
                                             int tpc) {
    switch (R) {
        case 16: reg_pass<T, SGN, 16>(src, dst, N, Ns, tw, t, tpc); break;
        case 8: reg_pass<T, SGN, 8>(src, dst, N, Ns, tw, t, tpc); break;
        case 4: reg_pass<T, SGN, 4>(src, dst, N, Ns, tw, t, tpc); break;
        case 2: reg_pass<T, SGN, 2>(src, dst, N, Ns, tw, t, tpc); break;
        case 3: reg_pass<T, SGN, 3>(src, dst, N, Ns, tw, t, tpc); break;
        default: reg_pass<T, SGN, 5>(src, dst, N, Ns, tw, t, tpc); break;
    }
}

// One Stockham pass of radix R done in place on shared memory, for lines where every thread
// owns exactly one butterfly (N / R == tpc, all threads of the block taking part): all inputs
// are read into registers, the block synchronises, then the outputs overwrite the buffer.
template <typename T, int SGN, int R, class Src, class Dst>
__device__ __forceinline__ void reg_pass_inplace(Src &src, Dst &dst, int N, int Ns, const cpx<T> *__restrict__ tw,
                                                 int t) {
    const int nbf = N / R, tws = N / (Ns * R);
    const int j = t;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src(j + r * nbf);
    const int jq = j / Ns, k = j - jq * Ns;
    if (k) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            cpx<T> w = tw[k * r * tws];
            if (SGN > 0) w = conj(w);
            v[r] = v[r] * w;
        }
    }
    Dft<T, SGN, R>::run(v);
    __syncthreads();
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst(base + r * Ns, v[r]);
}

// the R2C kernels transform in one shared buffer when the length is two register passes whose
// last has one butterfly per thread (16 threads per line)
template <typename T> __host__ __device__ inline bool r2c_inplace(const FftLen<T> &L) {
    return L.nrad_reg == 2 && L.rad_reg[1] == 16 && L.N == 16 * 16;
}

// FFT of the lines of a block, line (column) b of the block handled by the tpc threads with
// the same b.  The first pass reads the line through gsrc(position), the last pass writes it
// through gdst(position, value); intermediate results live in shared memory (position p of
// line b at s[idx(p, b)]), ping-ponging between sA (after passes 0, 2, ...) and sB (after
// passes 1, 3, ...).  All threads of the block must call it.
template <typename T, int SGN, class GSrc, class GDst, class Idx>
__device__ __forceinline__ void fft_reg_lines(const FftLen<T> &L, cpx<T> *sA, cpx<T> *sB, const Idx &idx, int b, int t,
                                              int tpc, GSrc &gsrc, GDst &gdst) {
    const int N = L.N;
    int Ns = 1;
    for (int s = 0; s < L.nrad_reg; ++s) {
        const int R = L.rad_reg[s];
        const bool first = s == 0, last = s == L.nrad_reg - 1;
        cpx<T> *in = (s & 1) ? sA : sB;
        cpx<T> *out = (s & 1) ? sB : sA;
        auto ssrc = [&](int l) { return in[idx(l, b)]; };
        auto sdst = [&](int l, cpx<T> v) { out[idx(l, b)] = v; };
        if (first && last) reg_pass_any<T, SGN>(R, gsrc, gdst, N, Ns, L.tw, t, tpc);
        else if (first) reg_pass_any<T, SGN>(R, gsrc, sdst, N, Ns, L.tw, t, tpc);
        else if (last) reg_pass_any<T, SGN>(R, ssrc, gdst, N, Ns, L.tw, t, tpc);
        else reg_pass_any<T, SGN>(R, ssrc, sdst, N, Ns, L.tw, t, tpc);
        __syncthreads();
        Ns *= R;
    }
}

// Lines whose register-engine factorisation is fixed at compile time (the upsampled lengths
// of the common grids): the same passes as fft_reg_lines for that radix sequence (pass s
// writes (s odd ? sB : sA), the last pass writes through gdst), without the run-time radix
// dispatch, so the sizes, strides and twiddle steps are constants.  Radices<> is the run-time
// engine.
template <int... R> struct Radices {};

template <typename T, int SGN, int TPC, int N, int Ns, int S, int R, int... Rest> struct FixedPasses {
    template <class Src, class GDst, class Idx>
    static __device__ __forceinline__ void run(const cpx<T> *tw, cpx<T> *sA, cpx<T> *sB, const Idx &idx, int b,
                                               int t, Src &src, GDst &gdst) {
        if constexpr (sizeof...(Rest) == 0) {
            reg_pass<T, SGN, R>(src, gdst, N, Ns, tw, t, TPC);
            __syncthreads();
        } else {
            cpx<T> *out = (S & 1) ? sB : sA;
            auto sdst = [&](int l, cpx<T> v) { out[idx(l, b)] = v; };
            reg_pass<T, SGN, R>(src, sdst, N, Ns, tw, t, TPC);
            __syncthreads();
            auto ssrc = [&](int l) { return out[idx(l, b)]; };
            FixedPasses<T, SGN, TPC, N, Ns * R, S + 1, Rest...>::run(tw, sA, sB, idx, b, t, ssrc, gdst);
        }
    }
};

template <class FL> struct FixedLen;
template <int... R> struct FixedLen<Radices<R...>> {
    static constexpr int npass = (int)sizeof...(R);
    static constexpr bool on = npass > 0;
    static constexpr int N = (1 * ... * R);
    template <typename T> static __host__ __device__ bool match(const FftLen<T> &L) {
        if constexpr (npass == 0) {
            return false;
        } else {
            constexpr int r[] = {R...};
            if (L.N != N || L.nrad_reg != npass) return false;
            for (int i = 0; i < npass; ++i)
                if (L.rad_reg[i] != r[i]) return false;
            return true;
        }
    }
    // TPC threads a line (the thread index t < TPC)
    template <typename T, int SGN, int TPC, class Src, class GDst, class Idx>
    static __device__ __forceinline__ void lines(const FftLen<T> &L, cpx<T> *sA, cpx<T> *sB, const Idx &idx, int b,
                                                 int t, Src &src, GDst &gdst) {
        if constexpr (on) FixedPasses<T, SGN, TPC, N, 1, 0, R...>::run(L.tw, sA, sB, idx, b, t, src, gdst);
    }
};
using Rad256 = Radices<16, 16>;
using Rad128 = Radices<16, 8>;
using Rad192 = Radices<16, 4, 3>;
using Rad320 = Radices<16, 4, 5>;
using Rad384 = Radices<16, 8, 3>;
using Rad2048 = Radices<16, 16, 8>;   // 2D 1024^2: last axis (128 threads a line pair)
using Rad64 = Radices<16, 4>;         // 2D four-step sub-lines
using Rad32 = Radices<16, 2>;

// Strided C2C pass on the register engine: the same operation as k_fft_strided, NBC
// columns per block, 16 threads per column.  The columns of all outer indices are numbered
// q = o ncol + c and block bid takes q = bid NBC .. bid NBC + NBC - 1 (a block may span two
// outer indices), so no block is left mostly idle when ncol is not a multiple of NBC (the
// half-spectrum width n/2 + 1).  Pruned input / output windows are predicated loads / stores
// (positions outside the input window read as zero).
template <typename T, int NBC>
__host__ __device__ inline int64_t cols_blocks(const StridedDesc &d) {
    return ((int64_t)d.nouter * d.ncol + NBC - 1) / NBC;
}

template <typename T, int SGN, int NBC, class FL = Radices<>>
__device__ __forceinline__ void fft_cols_block(cpx<T> *data, const StridedDesc &d, const FftLen<T> &L, int bid,
                                               unsigned char *smraw) {
    const int N = L.N;
    cpx<T> *sA = (cpx<T> *)smraw;
    cpx<T> *sB = sA + (size_t)N * NBC;
    const int b = threadIdx.x % NBC, t = threadIdx.x / NBC;
    const int64_t q = (int64_t)bid * NBC + b;
    const bool colok = q < (int64_t)d.nouter * d.ncol;
    const int o = colok ? (int)(q / d.ncol) : 0, c = colok ? (int)(q - (int64_t)o * d.ncol) : 0;
    const int oo = d.outer_map_n > 0 ? wrapi(o - d.outer_map_n / 2, d.outer_map_N) : o;
    cpx<T> *base = data + (int64_t)oo * d.os + c;
    cpx<T> *obase = (d.out ? (cpx<T> *)d.out : data) + (int64_t)oo * d.os + c;
    // window of n points: positions [0, n - n/2) and [N - n/2, N)
    const int ilo = d.n_in < N ? d.n_in - d.n_in / 2 : N, ihi = d.n_in < N ? N - d.n_in / 2 : N;
    const int olo = d.n_out < N ? d.n_out - d.n_out / 2 : N, ohi = d.n_out < N ? N - d.n_out / 2 : N;
    auto gsrc = [&](int l) -> cpx<T> {
        return (colok && (l < ilo || l >= ihi)) ? base[(int64_t)l * d.es] : mk<T>(0, 0);
    };
    auto gdst = [&](int l, cpx<T> v) {
        if (colok && (l < olo || l >= ohi)) obase[(int64_t)l * d.es] = v;
    };
    auto idx = [](int l, int c) { return l * NBC + c; };
    if constexpr (FixedLen<FL>::on) FixedLen<FL>::template lines<T, SGN, 16>(L, sA, sB, idx, b, t, gsrc, gdst);
    else fft_reg_lines<T, SGN>(L, sA, sB, idx, b, t, 16, gsrc, gdst);
}

template <typename T, int SGN, int NBC, class FL = Radices<>>
__global__ void __launch_bounds__(NBC * 16, 4) k_fft_cols(cpx<T> *data, StridedDesc d, FftLen<T> L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_cols_block<T, SGN, NBC, FL>(data, d, L, blockIdx.x, smraw);
}

// Long column passes (2D: fine axis 1 with N = N1 N2 points, too long for a register-engine
// block of enough columns to coalesce): the four-step decomposition, two passes of short
// transforms over the same columns.
//   step 1: for every column and j2 < N2, the N1-point transform of positions j1 N2 + j2
//           (input window applied), output k1 multiplied by w_N^{j2 k1} (w = e^{SGN 2 pi i / N})
//           and written to position k1 N2 + j2 of out;
//   step 2: for every column and k1 < N1, the N2-point transform of positions k1 N2 + j2 of
//           in, output k2 written to position k1 + N1 k2 of out (output window applied);
// so that X[k1 + N1 k2] = sum_j2 w_N2^{j2 k2} w_N^{j2 k1} sum_j1 x[j1 N2 + j2] w_N1^{j1 k1}.
// Block: NBC of the (sub-line, column) pairs q = s ncol + c, TPC threads each (the sub-lines
// are short: TPC ~ N_sub / 16 keeps the threads of a radix-16 pass busy and a block's
// columns one long coalesced row); 2D descriptors only (one outer line).
template <typename T, int SGN, int NBC, int TPC, int STEP, class FL = Radices<>>
__device__ __forceinline__ void fft_four_block(const cpx<T> *in, cpx<T> *out, const StridedDesc &d,
                                               const FftLen<T> &L, const FftLen<T> &Ls, int N1, int N2, int bid,
                                               unsigned char *smraw) {
    const int N = L.N;
    cpx<T> *sA = (cpx<T> *)smraw;
    cpx<T> *sB = sA + (size_t)Ls.N * NBC;
    const int b = threadIdx.x % NBC, t = threadIdx.x / NBC;
    const int nsub = STEP == 1 ? N2 : N1;
    const int64_t q = (int64_t)bid * NBC + b;
    const bool ok = q < (int64_t)nsub * d.ncol;
    const int sl = ok ? (int)(q / d.ncol) : 0, c = ok ? (int)(q - (int64_t)sl * d.ncol) : 0;
    const cpx<T> *ib = in + c;
    cpx<T> *ob = out + c;
    const int ilo = d.n_in < N ? d.n_in - d.n_in / 2 : N, ihi = d.n_in < N ? N - d.n_in / 2 : N;
    const int olo = d.n_out < N ? d.n_out - d.n_out / 2 : N, ohi = d.n_out < N ? N - d.n_out / 2 : N;
    auto gsrc = [&](int l) -> cpx<T> {
        const int pos = STEP == 1 ? l * N2 + sl : sl * N2 + l;
        const bool inw = STEP == 2 || pos < ilo || pos >= ihi;
        return (ok && inw) ? ib[(int64_t)pos * d.es] : mk<T>(0, 0);
    };
    auto gdst = [&](int k, cpx<T> v) {
        if (!ok) return;
        if (STEP == 1) {
            cpx<T> w = L.tw[(int)(((int64_t)sl * k) % N)];
            if (SGN > 0) w = conj(w);
            ob[(int64_t)(k * N2 + sl) * d.es] = v * w;
        } else {
            const int pos = sl + N1 * k;
            if (pos < olo || pos >= ohi) ob[(int64_t)pos * d.es] = v;
        }
    };
    auto idx = [](int l, int cc) { return l * NBC + cc; };
    if constexpr (FixedLen<FL>::on) FixedLen<FL>::template lines<T, SGN, TPC>(Ls, sA, sB, idx, b, t, gsrc, gdst);
    else fft_reg_lines<T, SGN>(Ls, sA, sB, idx, b, t, TPC, gsrc, gdst);
}

template <typename T, int SGN, int NBC, int TPC, int STEP, class FL = Radices<>>
__global__ void __launch_bounds__(NBC * TPC, FixedLen<FL>::on ? 4 : 2) k_fft_four(const cpx<T> *in, cpx<T> *out,
                                                                                 StridedDesc d, FftLen<T> L,
                                                                                 FftLen<T> Ls, int N1, int N2) {
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_four_block<T, SGN, NBC, TPC, STEP, FL>(in, out, d, L, Ls, N1, N2, blockIdx.x, smraw);
}

// shared-memory bytes of the register-engine passes for line length N
template <typename T> __host__ __device__ inline size_t cols_smem_bytes(const FftLen<T> &L, int nbc) {
    return sizeof(cpx<T>) * (size_t)L.N * nbc * (L.nrad_reg > 2 ? 2 : 1);
}

// Padded line-major shared layout for the contiguous-axis kernels: position l of line b at
// b * LDL + l + l / 16, so that unit-stride and stride-16 position accesses of 16 threads of
// one line fall on distinct banks.
__host__ __device__ __forceinline__ int line_ld(int N) { return N + N / 16 + 1; }

// Forward R2C along the last axis on the register engine: the same operation as
// k_fwd_r2c.  NBC line pairs per block, 16 threads per pair (consecutive threads walk one
// line, so the global loads and stores are contiguous).  The first pass reads rho,
// deconvolved and zero-padded, straight from HBM; the last pass lands in shared memory,
// where the spectra of the two real lines are separated and written as half spectra.
template <typename T, int NBC, bool kInplace = true, int TPC = 16, class FL = Radices<>>
__device__ __forceinline__ void fwd_r2c_reg_block(const T *__restrict__ rho, const DevPlan<T> &P, int bid,
                                                  unsigned char *smraw) {
    constexpr bool kFixed = FixedLen<FL>::on;
    static_assert(!kFixed || kInplace, "fixed radix sequences: single-plan kernels");
    const FftLen<T> &L = P.len[2];
    const int N = L.N, n2 = P.n[2], nh = P.nh, LDL = line_ld(N);
    cpx<T> *sA = (cpx<T> *)smraw;
    cpx<T> *sB = sA + (size_t)NBC * LDL;
    const int t = threadIdx.x % TPC, b = threadIdx.x / TPC;
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const int64_t p = (int64_t)bid * NBC + b;
    const bool ok = p < npairs;
    const int64_t line0 = 2 * p, line1 = 2 * p + 1;
    const int i0a = ok ? (int)(line0 / P.n[1]) : 0, i1a = ok ? (int)(line0 % P.n[1]) : 0;
    const int i0b = ok ? (int)(line1 / P.n[1]) : 0, i1b = ok ? (int)(line1 % P.n[1]) : 0;
    const T fa = P.deconv[0][i0a] * P.deconv[1][i1a], fb = P.deconv[0][i0b] * P.deconv[1][i1b];
    auto gsrc = [&](int l) -> cpx<T> {
        const int i = l < n2 / 2 ? l + n2 / 2 : l - N + n2 / 2;   // window point at fine position l
        if (!ok || i < 0 || i >= n2) return mk<T>(0, 0);
        const T d2 = P.deconv[2][i];
        return mk<T>(rho[line0 * n2 + i] * (fa * d2), rho[line1 * n2 + i] * (fb * d2));
    };
    auto idx = [LDL](int l, int c) { return c * LDL + l + (l >> 4); };
    cpx<T> *res;
    // 256 = 16 x 16: the first pass lands in sA, the second transforms sA in place
    auto inplace256 = [&](int Nn) {
        auto sdst = [&](int l, cpx<T> v) { sA[idx(l, b)] = v; };
        auto ssrc = [&](int l) { return sA[idx(l, b)]; };
        reg_pass<T, -1, 16>(gsrc, sdst, Nn, 1, L.tw, t, 16);
        __syncthreads();
        reg_pass_inplace<T, -1, 16>(ssrc, sdst, Nn, 16, L.tw, t);
        __syncthreads();
    };
    if constexpr (std::is_same<FL, Rad256>::value && TPC == 16) {
        res = sA;
        inplace256(256);
    } else if constexpr (kFixed) {
        res = ((FixedLen<FL>::npass - 1) & 1) ? sB : sA;
        auto gdst = [&](int l, cpx<T> v) { res[idx(l, b)] = v; };
        FixedLen<FL>::template lines<T, -1, TPC>(L, sA, sB, idx, b, t, gsrc, gdst);
    } else if (kInplace && TPC == 16 && r2c_inplace(L)) {
        res = sA;
        inplace256(N);
    } else {
        res = ((L.nrad_reg - 1) & 1) ? sB : sA;
        auto gdst = [&](int l, cpx<T> v) { res[idx(l, b)] = v; };
        fft_reg_lines<T, -1>(L, sA, sB, idx, b, t, TPC, gsrc, gdst);
    }
    if (!ok) return;
    const int l0a = wrapi(i0a - P.n[0] / 2, P.nf[0]), l1a = wrapi(i1a - P.n[1] / 2, P.nf[1]);
    const int l0b = wrapi(i0b - P.n[0] / 2, P.nf[0]), l1b = wrapi(i1b - P.n[1] / 2, P.nf[1]);
    cpx<T> *Fa = P.F + ((int64_t)l0a * P.nf[1] + l1a) * nh, *Fb = P.F + ((int64_t)l0b * P.nf[1] + l1b) * nh;
    for (int k = t; k < nh; k += TPC) {
        const cpx<T> z = res[idx(k, b)];
        const int kc = k == 0 ? 0 : N - k;
        const cpx<T> zc = conj(res[idx(kc, b)]);
        Fa[k] = scale(z + zc, (T)0.5);
        Fb[k] = mul_i(scale(z - zc, (T)0.5), -1);
    }
}

template <typename T, int NBC, int TPC = 16, class FL = Radices<>>
__global__ void __launch_bounds__(NBC * TPC, TPC == 16 ? 4 : 2) k_fwd_r2c_reg(const T *__restrict__ rho, DevPlan<T> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    fwd_r2c_reg_block<T, NBC, true, TPC, FL>(rho, P, blockIdx.x, smraw);
}

// Inverse C2R along the last axis on the register engine: the same operation as
// k_inv_c2r.  The first pass reads the half spectra of a line pair from HBM and forms
// Z = X1 + i X2 on the fly (Z[N - k] = conj(X1[k]) + i conj(X2[k])); the last pass writes
// the output window, deconvolved, straight to HBM.
template <typename T, int NBC, int TPC = 16, class FL = Radices<>>
__device__ __forceinline__ void inv_c2r_reg_block(T *__restrict__ phi, const DevPlan<T> &P, int bid,
                                                  unsigned char *smraw) {

    const FftLen<T> &L = P.len[2];
    const int N = L.N, n2 = P.n[2], nh = P.nh, LDL = line_ld(N);
    cpx<T> *sA = (cpx<T> *)smraw;
    cpx<T> *sB = sA + (size_t)NBC * LDL;
    const int t = threadIdx.x % TPC, b = threadIdx.x / TPC;
    const int64_t npairs = (int64_t)P.n[0] * P.n[1] / 2;
    const int64_t p = (int64_t)bid * NBC + b;
    const bool ok = p < npairs;
    const int64_t line0 = 2 * p, line1 = 2 * p + 1;
    const int i0a = ok ? (int)(line0 / P.n[1]) : 0, i1a = ok ? (int)(line0 % P.n[1]) : 0;
    const int i0b = ok ? (int)(line1 / P.n[1]) : 0, i1b = ok ? (int)(line1 % P.n[1]) : 0;
    const int l0a = wrapi(i0a - P.n[0] / 2, P.nf[0]), l1a = wrapi(i1a - P.n[1] / 2, P.nf[1]);
    const int l0b = wrapi(i0b - P.n[0] / 2, P.nf[0]), l1b = wrapi(i1b - P.n[1] / 2, P.nf[1]);
    const cpx<T> *Ga = P.G + ((int64_t)l0a * P.nf[1] + l1a) * nh, *Gb = P.G + ((int64_t)l0b * P.nf[1] + l1b) * nh;
    auto gsrc = [&](int l) -> cpx<T> {
        if (!ok) return mk<T>(0, 0);
        const bool lo = 2 * l <= N;
        const int k = lo ? l : N - l;
        cpx<T> x1 = Ga[k], x2 = Gb[k];
        if (k == 0 || 2 * k == N) {   // half-spectrum ends of a real line are real
            x1.y = 0;
            x2.y = 0;
        }
        return lo ? x1 + mul_i(x2, 1) : conj(x1) + mul_i(conj(x2), 1);
    };
    const T fa = P.deconv[0][i0a] * P.deconv[1][i1a], fb = P.deconv[0][i0b] * P.deconv[1][i1b];
    const int hi0 = n2 - n2 / 2, lo1 = N - n2 / 2;
    auto gdst = [&](int l, cpx<T> z) {
        if (!ok) return;
        int i;
        if (l < hi0) i = l + n2 / 2;
        else if (l >= lo1) i = l - lo1;
        else return;
        const T d2 = P.deconv[2][i];
        const T va = z.x * (fa * d2), vb = z.y * (fb * d2);
        if (P.accumulate) {
            phi[line0 * n2 + i] += va;
            phi[line1 * n2 + i] += vb;
        } else {
            phi[line0 * n2 + i] = va;
            phi[line1 * n2 + i] = vb;
        }
    };
    auto idx = [LDL](int l, int c) { return c * LDL + l + (l >> 4); };
    if constexpr (FixedLen<FL>::on) FixedLen<FL>::template lines<T, +1, TPC>(L, sA, sB, idx, b, t, gsrc, gdst);
    else fft_reg_lines<T, +1>(L, sA, sB, idx, b, t, TPC, gsrc, gdst);
}

template <typename T, int NBC, int TPC = 16, class FL = Radices<>>
__global__ void __launch_bounds__(NBC * TPC, TPC == 16 ? 4 : 2) k_inv_c2r_reg(T *__restrict__ phi, DevPlan<T> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    inv_c2r_reg_block<T, NBC, TPC, FL>(phi, P, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ contiguous C2C pass
// In-place transform of nlines contiguous complex lines of length N, scaled by post.
template <typename T, int SGN>
__global__ void __launch_bounds__(256) k_fft_contig(cpx<T> *data, int64_t nlines, FftLen<T> L, int nb, T post) {
    extern __shared__ unsigned char smraw[];
    const int N = L.N, ldb = nb + 1;
    cpx<T> *s_tw = (cpx<T> *)smraw;
    cpx<T> *A = s_tw + N;
    cpx<T> *B = A + N * ldb;
    load_twiddles(s_tw, L);
    const int64_t l0 = (int64_t)blockIdx.x * nb;
    for (int q = threadIdx.x; q < N * nb; q += blockDim.x) {
        const int b = q / N, i = q % N;
        A[i * ldb + b] = (l0 + b < nlines) ? data[(l0 + b) * N + i] : mk<T>(0, 0);
    }
    __syncthreads();
    cpx<T> *R = fft_smem<T, SGN>(A, B, L, s_tw, nb, ldb);
    for (int q = threadIdx.x; q < N * nb; q += blockDim.x) {
        const int b = q / N, i = q % N;
        if (l0 + b < nlines) data[(l0 + b) * N + i] = scale(R[i * ldb + b], post);
    }
}


}  // namespace nlp
