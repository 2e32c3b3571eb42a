// Ground state and dynamics steps on the plain grid (Sec. 3.1 and Sec. 4.1):
//   - backward-Euler normalized gradient flow with the stabilised Fourier fixed point
//     (the linear solve the paper omits; reading stated in nlpot.h),
//   - energies of Sec. 3.2,
//   - time splitting (Strang / Yoshida) with the kinetic flow solved exactly in Fourier space.
// The nonlocal potential of each step comes from the NUFFT evaluator of the same plan.
// Sums, minima/maxima and norms are reduced in FP64 for both plan precisions.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace nlp {

nlp_status eval_any(nlp_plan_s *p, const void *rho, void *phi);
size_t grid_points(const nlp_plan_s *p);

constexpr int kRedBlocks = 608;   // 152 SMs x 4
enum { S_MIN = 0, S_MAX, S_DIFF, S_NORM, S_CHANGE, S_EPOT, S_EINT, S_EKIN,
       S_CHEB_Q, S_CHEB_R0, S_CHEB_R1, S_COUNT = 16 };

template <typename T> struct Work {
    T *rho, *pot, *b, *x, *xn, *r, *xf;   // xf: inner iterate captured at convergence
    T *d;                                 // last inner update (Chebyshev recurrence)
    T *dtab;                              // Fourier diagonal of the inner solve (per step)
    int *iflag;                           // [0] first converged inner iteration, [1] first non-finite one
    cpx<T> *spec;       // plain-grid spectrum (R2C half for GF)
    double *part;       // kRedBlocks x 2 partials
    double *scal;       // S_COUNT scalars
    DevPlan<T> PD;      // plain-grid FFT descriptor (nf = n, unit deconvolution, F = G = spec)
};

template <typename T> static nlp_status ensure_work(nlp_plan_s *p, Work<T> *&W) {
    if (p->d_work) {
        W = (Work<T> *)p->d_work;
        return NLP_OK;
    }
    // owned here until the whole set is allocated: a failure part-way frees the host struct
    // (its device buffers are already in p->allocs and go with the plan)
    std::unique_ptr<Work<T>> own(new Work<T>());
    W = own.get();
    const size_t N = grid_points(p);
    const int n0 = p->n3[0], n1 = p->n3[1], n2 = p->n3[2];
    const size_t nh = (size_t)n2 / 2 + 1;
    void *d;
    nlp_status s;
    T *bufs[8];
    for (int i = 0; i < 8; ++i) {
        if ((s = alloc_dev(p, &d, sizeof(T) * N))) return s;
        bufs[i] = (T *)d;
    }
    W->rho = bufs[0]; W->pot = bufs[1]; W->b = bufs[2]; W->x = bufs[3]; W->xn = bufs[4]; W->r = bufs[5];
    W->xf = bufs[6];
    W->d = bufs[7];
    if ((s = alloc_dev(p, &d, sizeof(int) * 2))) return s;
    W->iflag = (int *)d;
    if ((s = alloc_dev(p, &d, sizeof(cpx<T>) * (size_t)n0 * n1 * nh))) return s;
    W->spec = (cpx<T> *)d;
    if ((s = alloc_dev(p, &d, sizeof(T) * (size_t)n0 * n1 * nh))) return s;
    W->dtab = (T *)d;
    if ((s = alloc_dev(p, &d, sizeof(double) * 2 * kRedBlocks))) return s;
    W->part = (double *)d;
    if ((s = alloc_dev(p, &d, sizeof(double) * S_COUNT))) return s;
    W->scal = (double *)d;
    DevPlan<T> &D = W->PD;
    memset(&D, 0, sizeof(D));
    D.dim = p->grid.dim;
    const int nn[3] = {n0, n1, n2};
    for (int a = 0; a < 3; ++a) {
        D.n[a] = nn[a];
        D.nf[a] = nn[a];
        if ((s = make_fft_len<T>(p, nn[a], &D.len[a]))) return s;
        std::vector<T> ones(nn[a], (T)1);
        if ((s = alloc_dev(p, &d, sizeof(T) * nn[a]))) return s;
        cudaMemcpy(d, ones.data(), sizeof(T) * nn[a], cudaMemcpyHostToDevice);
        D.deconv[a] = (const T *)d;
    }
    D.nh = (int)nh;
    D.F = D.G = W->spec;
    p->d_work = own.release();
    p->work_free = [](void *w) { delete (Work<T> *)w; };
    p->info.workspace_bytes = p->bytes;
    return NLP_OK;
}

// ------------------------------------------------------------------ reductions (FP64)
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// op 0 sum, 1 max, 2 min
__device__ double block_reduce(double v, int op) {
    __shared__ double sh[32];
    v = op == 0 ? warp_sum(v) : (op == 1 ? warp_max(v) : warp_min(v));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const double id = op == 0 ? 0.0 : (op == 1 ? -INFINITY : INFINITY);
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[lane] : id;
    if (wid == 0) v = op == 0 ? warp_sum(v) : (op == 1 ? warp_max(v) : warp_min(v));
    return v;
}

// final pass: one block folds kRedBlocks partials (fixed order) into scal[slot] (* mul)
__global__ void k_red_final(const double *part, int nparts, int stride, int off, int op, double mul, double *out) {
    const double id = op == 0 ? 0.0 : (op == 1 ? -INFINITY : INFINITY);
    double v = id;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const double t = part[stride * i + off];
        v = op == 0 ? v + t : (op == 1 ? fmax(v, t) : fmin(v, t));
    }
    v = block_reduce(v, op);
    if (threadIdx.x == 0) *out = op == 0 ? v * mul : v;
}

#define GRID_STRIDE(q, N) for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (N); q += (int64_t)gridDim.x * blockDim.x)

// rho = x^2
template <typename T> __global__ void k_square(const T *x, T *rho, int64_t N) {
    GRID_STRIDE(q, N) { const T v = x[q]; rho[q] = v * v; }
}

// b = V + g rho + beta pot; partial min (slot 0) and max (slot 1)
template <typename T>
__global__ void k_make_b(const T *V, const T *rho, const T *pot, T g, T beta, T *b, int64_t N, double *part) {
    double mn = INFINITY, mx = -INFINITY;
    GRID_STRIDE(q, N) {
        const T v = V[q] + g * rho[q] + beta * pot[q];
        b[q] = v;
        mn = fmin(mn, (double)v);
        mx = fmax(mx, (double)v);
    }
    mn = block_reduce(mn, 2);
    mx = block_reduce(mx, 1);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = mn; part[2 * blockIdx.x + 1] = mx; }
}

// r = phi / tau + (alpha - b) x,  alpha = (min b + max b)/2 from device scalars
template <typename T>
__global__ void k_rhs(const T *phi, const T *b, const T *x, T inv_tau, const double *scal, T *r, int64_t N) {
    const T alpha = (T)(0.5 * (scal[S_MIN] + scal[S_MAX]));
    GRID_STRIDE(q, N) r[q] = phi[q] * inv_tau + (alpha - b[q]) * x[q];
}

__device__ __forceinline__ double wave2(int l, int n, double L) {
    const int p = (2 * l < n) ? l : l - n;     // FFT frequency index
    const double mu = M_PI * p / L;
    return mu * mu;
}

// dtab = 1 / ((1/tau + alpha + |mu|^2/2) N) on the R2C half spectrum [n0][n1][nh]: the Fourier
// diagonal of the inner solve, fixed for one gradient-flow step (alpha from device scalars)
template <typename T>
__global__ void k_diag_table(T *dtab, int n0, int n1, int n2, int nh, double L0, double L1, double L2,
                             double inv_tau, const double *scal, double invN) {
    const double alpha = 0.5 * (scal[S_MIN] + scal[S_MAX]);
    const int64_t M = (int64_t)n0 * n1 * nh;
    GRID_STRIDE(q, M) {
        const int l2 = (int)(q % nh);
        const int64_t t = q / nh;
        const int l1 = (int)(t % n1), l0 = (int)(t / n1);
        double m2 = (n2 > 1 ? wave2(l2, n2, L2) : 0.0) + (n1 > 1 ? wave2(l1, n1, L1) : 0.0) +
                    (n0 > 1 ? wave2(l0, n0, L0) : 0.0);
        dtab[q] = (T)(invN / (inv_tau + alpha + 0.5 * m2));
    }
}

// spec *= dtab (one inner iteration's Fourier-diagonal solve)
template <typename T> __global__ void k_diag_apply(cpx<T> *spec, const T *__restrict__ dtab, int64_t M) {
    GRID_STRIDE(q, M) spec[q] = scale(spec[q], dtab[q]);
}


// Chebyshev acceleration of the inner fixed point.  With G(x) = M^{-1}(phi^n/tau + (alpha - b) x),
// M = 1/tau + alpha - Delta/2 and A = 1/tau - Delta/2 + b = M + (b - alpha), the preconditioned
// residual is G(x) - x and the eigenvalues of M^{-1} A lie in [1 - q, 1 + q],
// q = (max b - min b) / (2/tau + max b + min b).  The semi-iteration on that interval
// (centre 1, half-width q; Chebyshev acceleration as in Saad, Iterative Methods for Sparse
// Linear Systems, Alg. 12.1) takes x_1 = G(x_0) and then
//   d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / q) (G(x_k) - x_k),  x_{k+1} = x_k + d_k,
//   rho_0 = q,  rho_k = 1 / (2/q - rho_{k-1}),
// with the same fixed point (the backward-Euler solution).  q outside (0, 1) falls back to
// the plain iteration x_{k+1} = G(x_k).
__global__ void k_cheb_init(double *scal, double inv_tau) {
    const double bmin = scal[S_MIN], bmax = scal[S_MAX];
    const double q = 0.5 * (bmax - bmin) / (inv_tau + 0.5 * (bmax + bmin));
    scal[S_CHEB_Q] = q;
    scal[S_CHEB_R0] = 0.0;
    scal[S_CHEB_R1] = q;   // rho_0
}

__device__ __forceinline__ bool cheb_ok(double q) { return q > 1e-300 && q < 1.0; }

// iteration it: d = c1 d + c2 (xn - x), x += d; partial max |d|
template <typename T>
__global__ void k_cheb_update(T *x, const T *xn, T *d, const double *scal, int it, int64_t N, double *part) {
    const double q = scal[S_CHEB_Q];
    double c1 = 0.0, c2 = 1.0;
    if (it > 1 && cheb_ok(q)) {
        c1 = scal[S_CHEB_R1] * scal[S_CHEB_R0];
        c2 = 2.0 * scal[S_CHEB_R1] / q;
    }
    double m = 0.0;
    const bool first = c1 == 0.0;   // d holds no previous update yet (it may be uninitialised)
    GRID_STRIDE(k, N) {
        const double r = (double)xn[k] - (double)x[k];
        const T dn = (T)(first ? c2 * r : c1 * (double)d[k] + c2 * r);
        d[k] = dn;
        x[k] = x[k] + dn;
        m = fmax(m, fabs((double)dn));
    }
    m = block_reduce(m, 1);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = m;
}

// inner-iteration bookkeeping on the device: records the first iteration whose update
// max|x^(m+1) - x^(m)| is <= tol (flag[0]) or non-finite (flag[1]); advances the
// Chebyshev coefficients (rho_{k-1}, rho_k) for the next iteration
__global__ void k_inner_check(double *scal, double tol, int it, int *flag) {
    const double q = scal[S_CHEB_Q];
    if (it > 1 && cheb_ok(q)) {
        const double r1 = scal[S_CHEB_R1];
        scal[S_CHEB_R0] = r1;
        scal[S_CHEB_R1] = 1.0 / (2.0 / q - r1);
    } else if (it == 1 && cheb_ok(q)) {
        scal[S_CHEB_R0] = q;                       // rho_0
        scal[S_CHEB_R1] = 1.0 / (2.0 / q - q);     // rho_1
    }
    if (flag[0] || flag[1]) return;
    const double d = scal[S_DIFF];
    if (!isfinite(d)) flag[1] = it;
    else if (d <= tol) flag[0] = it;
}

// dst = src on the iteration that converged (later iterations leave dst alone)
template <typename T> __global__ void k_capture(const int *flag, int it, const T *src, T *dst, int64_t N) {
    if (flag[0] != it) return;
    GRID_STRIDE(q, N) dst[q] = src[q];
}

// partial sum x^2
template <typename T> __global__ void k_sumsq(const T *x, int64_t N, double *part) {
    double s = 0.0;
    GRID_STRIDE(q, N) { const double v = (double)x[q]; s += v * v; }
    s = block_reduce(s, 0);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = s;
}

// phi_new = x / sqrt(norm); partial max |phi_new - phi_old|; phi overwritten
template <typename T> __global__ void k_finish(const T *x, T *phi, const double *scal, int64_t N, double *part) {
    const double s = 1.0 / sqrt(scal[S_NORM]);
    double m = 0.0;
    GRID_STRIDE(q, N) {
        const T nv = (T)((double)x[q] * s);
        m = fmax(m, fabs((double)nv - (double)phi[q]));
        phi[q] = nv;
    }
    m = block_reduce(m, 1);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = m;
}

// partial sums: V x^2 (slot 0) and (g x^2 + beta pot) x^2 (slot 1)
template <typename T>
__global__ void k_epot_eint(const T *x, const T *V, const T *pot, double g, double beta, int64_t N, double *part) {
    double a = 0.0, c = 0.0;
    GRID_STRIDE(q, N) {
        const double r = (double)x[q] * (double)x[q];
        a += (double)V[q] * r;
        c += (g * r + beta * (double)pot[q]) * r;
    }
    a = block_reduce(a, 0);
    c = block_reduce(c, 0);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = c; }
}

// partial sum of |mu|^2 |spec|^2 over the full spectrum represented by the half spectrum
template <typename T>
__global__ void k_ekin(const cpx<T> *spec, int n0, int n1, int n2, int nh, double L0, double L1, double L2,
                       double *part) {
    const int64_t M = (int64_t)n0 * n1 * nh;
    double s = 0.0;
    GRID_STRIDE(q, M) {
        const int l2 = (int)(q % nh);
        const int64_t t = q / nh;
        const int l1 = (int)(t % n1), l0 = (int)(t / n1);
        const double m2 = wave2(l2, n2, L2) + (n1 > 1 ? wave2(l1, n1, L1) : 0.0) + (n0 > 1 ? wave2(l0, n0, L0) : 0.0);
        const double wgt = (l2 == 0 || 2 * l2 == n2) ? 1.0 : 2.0;
        const cpx<T> v = spec[q];
        s += wgt * m2 * ((double)v.x * v.x + (double)v.y * v.y);
    }
    s = block_reduce(s, 0);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = s;
}

// ------------------------------------------------------------------ plain-grid FFTs
template <typename T> static StridedDesc plain_axis(const DevPlan<T> &D, int axis, int ncol, int64_t es_last) {
    StridedDesc d{};
    const int n0 = D.n[0], n1 = D.n[1];
    d.n_in = D.len[axis].N;
    d.n_out = D.len[axis].N;
    d.ncol = ncol;
    if (axis == 1) {
        d.es = es_last;
        d.nouter = n0;
        d.os = (int64_t)n1 * es_last;
    } else {
        d.es = (int64_t)n1 * es_last;
        d.nouter = n1;
        d.os = es_last;
    }
    return d;
}

// real x -> half spectrum (shift-consistent placement, see fft_dev.cuh)
template <typename T> static cudaError_t r2c_plain(const T *x, DevPlan<T> &D, cudaStream_t st) {
    cudaError_t e = launch_fwd_r2c<T>(x, D, st);
    if (e) return e;
    if (D.n[1] > 1 && (e = launch_fft_strided<T>(D.F, plain_axis(D, 1, D.nh, D.nh), D.len[1], -1, st))) return e;
    if (D.n[0] > 1 && (e = launch_fft_strided<T>(D.F, plain_axis(D, 0, D.nh, D.nh), D.len[0], -1, st))) return e;
    return cudaSuccess;
}
template <typename T> static cudaError_t c2r_plain(T *x, DevPlan<T> &D, cudaStream_t st) {
    cudaError_t e;
    if (D.n[0] > 1 && (e = launch_fft_strided<T>(D.G, plain_axis(D, 0, D.nh, D.nh), D.len[0], +1, st))) return e;
    if (D.n[1] > 1 && (e = launch_fft_strided<T>(D.G, plain_axis(D, 1, D.nh, D.nh), D.len[1], +1, st))) return e;
    return launch_inv_c2r<T>(x, D, st);
}

static dim3 eg() { return dim3(kRedBlocks); }

template <typename T>
static nlp_status reduce_to(nlp_plan_s *p, Work<T> *W, int off, int op, double mul, int slot) {
    k_red_final<<<1, 256, 0, p->stream>>>(W->part, kRedBlocks, 2, off, op, mul, W->scal + slot);
    return cudaGetLastError() ? NLP_ERR_CUDA : NLP_OK;
}

template <typename T> static nlp_status read_scal(nlp_plan_s *p, Work<T> *W, double *host) {
    if (cudaMemcpyAsync(host, W->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, p->stream)) return NLP_ERR_CUDA;
    if (cudaStreamSynchronize(p->stream)) return NLP_ERR_CUDA;
    return NLP_OK;
}

static double hvol_of(const nlp_plan_s *p) {
    double v = 1.0;
    for (int a = 0; a < 3; ++a) if (p->n3[a] > 1) v *= p->h[a];
    return v;
}

template <typename T>
static nlp_status energies_t(nlp_plan_s *p, Work<T> *W, const T *x, const T *V, double beta, double g, double *E) {
    cudaStream_t st = p->stream;
    const int64_t N = (int64_t)grid_points(p);
    k_square<T><<<eg(), 256, 0, st>>>(x, W->rho, N);
    nlp_status s = eval_any(p, W->rho, W->pot);
    if (s) return s;
    k_epot_eint<T><<<eg(), 256, 0, st>>>(x, V, W->pot, g, beta, N, W->part);
    const double hv = hvol_of(p);
    if ((s = reduce_to(p, W, 0, 0, hv, S_EPOT)) || (s = reduce_to(p, W, 1, 0, 0.5 * hv, S_EINT))) return s;
    DevPlan<T> &D = W->PD;
    if (r2c_plain<T>(x, D, st)) return NLP_ERR_CUDA;
    k_ekin<T><<<eg(), 256, 0, st>>>(D.F, D.n[0], D.n[1], D.n[2], D.nh, p->L3[0], p->L3[1], p->L3[2], W->part);
    if ((s = reduce_to(p, W, 0, 0, 0.5 * hv / (double)N, S_EKIN))) return s;
    double h[S_COUNT];
    if ((s = read_scal(p, W, h))) return s;
    const double Ek = h[S_EKIN], Ep = h[S_EPOT], Ei = h[S_EINT];
    E[0] = Ek + Ep + Ei;
    E[1] = Ek;
    E[2] = Ep;
    E[3] = Ei;
    E[4] = E[0] + Ei;
    for (int i = 0; i < 5; ++i)
        if (!std::isfinite(E[i])) return NLP_ERR_DIVERGED;
    return NLP_OK;
}

template <typename T>
static nlp_status gf_step_t(nlp_plan_s *p, T *phi, const T *V, double beta, double g, double tau, double inner_tol,
                            int max_inner, double *max_change, int *inner_iters, double *energies) {
    Work<T> *W;
    nlp_status s = ensure_work<T>(p, W);
    if (s) return s;
    cudaStream_t st = p->stream;
    const int64_t N = (int64_t)grid_points(p);
    DevPlan<T> &D = W->PD;
    // rho = |phi^n|^2, Phi = U * rho, b = V + g rho + beta Phi, alpha from min/max b
    k_square<T><<<eg(), 256, 0, st>>>(phi, W->rho, N);
    if ((s = eval_any(p, W->rho, W->pot))) return s;
    k_make_b<T><<<eg(), 256, 0, st>>>(V, W->rho, W->pot, (T)g, (T)beta, W->b, N, W->part);
    if ((s = reduce_to(p, W, 0, 2, 1.0, S_MIN)) || (s = reduce_to(p, W, 1, 1, 1.0, S_MAX))) return s;
    if (cudaMemcpyAsync(W->x, phi, sizeof(T) * N, cudaMemcpyDeviceToDevice, st)) return NLP_ERR_CUDA;
    // Inner solve: the Chebyshev-accelerated fixed point (k_cheb_init).  The convergence test
    // runs on the device every iteration; the host reads its decision every kCheckEvery
    // iterations, so up to kCheckEvery - 1 iterations may run past convergence.  Their results
    // are not used: the iterate of the first converged iteration is captured in xf, so the
    // step equals one that stopped exactly there.
    constexpr int kCheckEvery = 4;
    if (cudaMemsetAsync(W->iflag, 0, sizeof(int) * 2, st)) return NLP_ERR_CUDA;
    k_cheb_init<<<1, 1, 0, st>>>(W->scal, 1.0 / tau);
    const int64_t Mspec = (int64_t)D.n[0] * D.n[1] * D.nh;
    k_diag_table<T><<<eg(), 256, 0, st>>>(W->dtab, D.n[0], D.n[1], D.n[2], D.nh, p->L3[0], p->L3[1], p->L3[2],
                                          1.0 / tau, W->scal, 1.0 / (double)N);
    int flags[2] = {0, 0};
    for (int it = 1; it <= max_inner; ++it) {
        k_rhs<T><<<eg(), 256, 0, st>>>(phi, W->b, W->x, (T)(1.0 / tau), W->scal, W->r, N);
        if (r2c_plain<T>(W->r, D, st)) return NLP_ERR_CUDA;
        k_diag_apply<T><<<eg(), 256, 0, st>>>(D.F, W->dtab, Mspec);
        if (c2r_plain<T>(W->xn, D, st)) return NLP_ERR_CUDA;
        k_cheb_update<T><<<eg(), 256, 0, st>>>(W->x, W->xn, W->d, W->scal, it, N, W->part);
        if ((s = reduce_to(p, W, 0, 1, 1.0, S_DIFF))) return s;
        k_inner_check<<<1, 1, 0, st>>>(W->scal, inner_tol, it, W->iflag);
        k_capture<T><<<eg(), 256, 0, st>>>(W->iflag, it, W->x, W->xf, N);
        if (it % kCheckEvery == 0 || it == max_inner) {
            if (cudaMemcpyAsync(flags, W->iflag, sizeof(flags), cudaMemcpyDeviceToHost, st) ||
                cudaStreamSynchronize(st))
                return NLP_ERR_CUDA;
            if (flags[0] || flags[1]) break;
        }
    }
    if (flags[1] && (!flags[0] || flags[1] < flags[0])) return NLP_ERR_DIVERGED;
    const bool conv = flags[0] != 0;
    if (inner_iters) *inner_iters = conv ? flags[0] : max_inner;
    const T *res = conv ? W->xf : W->x;
    double hs[S_COUNT];
    // normalise, change
    k_sumsq<T><<<eg(), 256, 0, st>>>(res, N, W->part);
    if ((s = reduce_to(p, W, 0, 0, hvol_of(p), S_NORM))) return s;
    k_finish<T><<<eg(), 256, 0, st>>>(res, phi, W->scal, N, W->part);
    if ((s = reduce_to(p, W, 0, 1, 1.0, S_CHANGE))) return s;
    if ((s = read_scal(p, W, hs))) return s;
    if (!std::isfinite(hs[S_CHANGE]) || !std::isfinite(hs[S_NORM])) return NLP_ERR_DIVERGED;
    if (max_change) *max_change = hs[S_CHANGE] / tau;
    if (energies && (s = energies_t<T>(p, W, phi, V, beta, g, energies))) return s;
    return conv ? NLP_OK : NLP_ERR_NOT_CONVERGED;
}

nlp_status gf_step_impl(nlp_plan_s *p, void *phi, const void *V, double beta, double g, double tau, double inner_tol,
                        int max_inner, double *max_change, int *inner_iters, double *energies) {
    if (p->prec == NLP_FP64)
        return gf_step_t<double>(p, (double *)phi, (const double *)V, beta, g, tau, inner_tol, max_inner, max_change,
                                 inner_iters, energies);
    return gf_step_t<float>(p, (float *)phi, (const float *)V, beta, g, tau, inner_tol, max_inner, max_change,
                            inner_iters, energies);
}

nlp_status energies_impl(nlp_plan_s *p, const void *phi, const void *V, double beta, double g, double *E) {
    if (p->prec == NLP_FP64) {
        Work<double> *W;
        nlp_status s = ensure_work<double>(p, W);
        return s ? s : energies_t<double>(p, W, (const double *)phi, (const double *)V, beta, g, E);
    }
    Work<float> *W;
    nlp_status s = ensure_work<float>(p, W);
    return s ? s : energies_t<float>(p, W, (const float *)phi, (const float *)V, beta, g, E);
}

// ------------------------------------------------------------------ time splitting
// psi *= exp(-i s |mu|^2 / 2) / N on the full complex spectrum [n0][n1][n2]
template <typename T>
__global__ void k_kin_phase(cpx<T> *psi, int n0, int n1, int n2, double L0, double L1, double L2, double s,
                            double invN) {
    const int64_t M = (int64_t)n0 * n1 * n2;
    GRID_STRIDE(q, M) {
        const int l2 = (int)(q % n2);
        const int64_t t = q / n2;
        const int l1 = (int)(t % n1), l0 = (int)(t / n1);
        const double m2 = wave2(l2, n2, L2) + (n1 > 1 ? wave2(l1, n1, L1) : 0.0) + (n0 > 1 ? wave2(l0, n0, L0) : 0.0);
        double sn, cs;
        sincos(-0.5 * s * m2, &sn, &cs);
        psi[q] = psi[q] * mk<T>((T)(cs * invN), (T)(sn * invN));
    }
}

template <typename T> __global__ void k_abs2(const cpx<T> *psi, T *rho, int64_t N) {
    GRID_STRIDE(q, N) { const cpx<T> v = psi[q]; rho[q] = v.x * v.x + v.y * v.y; }
}

// psi *= exp(-i (V + g rho + beta pot) s)   (Eq. (sps-eq68))
template <typename T>
__global__ void k_pot_phase(cpx<T> *psi, const T *V, const T *rho, const T *pot, double g, double beta, double s,
                            int64_t N) {
    GRID_STRIDE(q, N) {
        const double th = -s * ((double)V[q] + g * (double)rho[q] + beta * (double)pot[q]);
        double sn, cs;
        sincos(th, &sn, &cs);
        psi[q] = psi[q] * mk<T>((T)cs, (T)sn);
    }
}

template <typename T> static nlp_status kinetic(nlp_plan_s *p, Work<T> *W, cpx<T> *psi, double s) {
    cudaStream_t st = p->stream;
    DevPlan<T> &D = W->PD;
    const int n0 = D.n[0], n1 = D.n[1], n2 = D.n[2];
    const int64_t N = (int64_t)n0 * n1 * n2;
    if (launch_fft_contig<T>(psi, (int64_t)n0 * n1, D.len[2], -1, (T)1, st)) return NLP_ERR_CUDA;
    if (n1 > 1 && launch_fft_strided<T>(psi, plain_axis(D, 1, n2, n2), D.len[1], -1, st)) return NLP_ERR_CUDA;
    if (n0 > 1 && launch_fft_strided<T>(psi, plain_axis(D, 0, n2, n2), D.len[0], -1, st)) return NLP_ERR_CUDA;
    k_kin_phase<T><<<eg(), 256, 0, st>>>(psi, n0, n1, n2, p->L3[0], p->L3[1], p->L3[2], s, 1.0 / (double)N);
    if (n0 > 1 && launch_fft_strided<T>(psi, plain_axis(D, 0, n2, n2), D.len[0], +1, st)) return NLP_ERR_CUDA;
    if (n1 > 1 && launch_fft_strided<T>(psi, plain_axis(D, 1, n2, n2), D.len[1], +1, st)) return NLP_ERR_CUDA;
    if (launch_fft_contig<T>(psi, (int64_t)n0 * n1, D.len[2], +1, (T)1, st)) return NLP_ERR_CUDA;
    return cudaGetLastError() ? NLP_ERR_CUDA : NLP_OK;
}

template <typename T>
static nlp_status strang(nlp_plan_s *p, Work<T> *W, cpx<T> *psi, const T *V, double beta, double g, double tau) {
    const int64_t N = (int64_t)grid_points(p);
    nlp_status s;
    if ((s = kinetic<T>(p, W, psi, 0.5 * tau))) return s;
    k_abs2<T><<<eg(), 256, 0, p->stream>>>(psi, W->rho, N);
    if ((s = eval_any(p, W->rho, W->pot))) return s;
    k_pot_phase<T><<<eg(), 256, 0, p->stream>>>(psi, V, W->rho, W->pot, g, beta, tau, N);
    return kinetic<T>(p, W, psi, 0.5 * tau);
}

template <typename T>
static nlp_status ts_t(nlp_plan_s *p, cpx<T> *psi, const T *V, double beta, double g, double tau, int order) {
    Work<T> *W;
    nlp_status s = ensure_work<T>(p, W);
    if (s) return s;
    if (order == 2) return strang<T>(p, W, psi, V, beta, g, tau);
    const double w1 = 1.0 / (2.0 - std::cbrt(2.0)), w0 = 1.0 - 2.0 * w1;   // Yoshida
    if ((s = strang<T>(p, W, psi, V, beta, g, w1 * tau))) return s;
    if ((s = strang<T>(p, W, psi, V, beta, g, w0 * tau))) return s;
    return strang<T>(p, W, psi, V, beta, g, w1 * tau);
}

nlp_status ts_step_impl(nlp_plan_s *p, void *psi, const void *V, double beta, double g, double tau, int order) {
    if (p->prec == NLP_FP64) return ts_t<double>(p, (cpx<double> *)psi, (const double *)V, beta, g, tau, order);
    return ts_t<float>(p, (cpx<float> *)psi, (const float *)V, beta, g, tau, order);
}

// ------------------------------------------------------------------ energies without allocation
// nlp_energies allocates the plan's gradient-flow workspace on its first call.  Some callers
// cannot let a library call cudaMalloc at that point: a process whose device memory is
// already reserved by another allocator (a framework's caching pool, an arena sized at
// start-up), where a new cudaMalloc fails or fragments that pool, and latency-bound loops
// where the device-wide synchronisation that cudaMalloc / cudaFree may imply is not
// acceptable.  nlp_energies_noalloc computes the same energies with every buffer carved from
// one file-scope static device array.  The potential evaluation inside uses the plan's
// spectra, which nlp_plan_create already allocated.
constexpr int64_t kNoAllocMaxPoints = 32768;          // grid points (e.g. 32^3 or 128 x 256)
constexpr size_t kNoAllocBytes = 1u << 20;            // 1 MiB per device, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[128] = {};

// Device address of the static array on the current device (set up once per device).
static nlp_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NLP_ERR_CUDA;
    if (dev < 0 || dev >= 128) return NLP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return NLP_ERR_CUDA;
        g_noalloc_ptr[dev] = ptr;
    }
    *out = g_noalloc_ptr[dev];
    return NLP_OK;
}

template <typename T> __global__ void k_fill_twiddles(cpx<T> *tw, int N) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)k / (double)N, &sn, &cs);
        tw[k] = mk<T>((T)cs, (T)(-sn));
    }
}

template <typename T> __global__ void k_fill_value(T *a, int n, T v) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) a[k] = v;
}

template <typename T>
static nlp_status energies_noalloc_t(nlp_plan_s *p, const T *x, const T *V, double beta, double g, double *E) {
    const int64_t N = (int64_t)grid_points(p);
    if (N > kNoAllocMaxPoints) return NLP_ERR_INVALID_ARG;
    const int n[3] = {p->n3[0], p->n3[1], p->n3[2]};
    const size_t nh = (size_t)n[2] / 2 + 1;
    // layout of the static array, checked before any launch
    size_t sizes[11] = {sizeof(T) * N, sizeof(T) * N, sizeof(cpx<T>) * n[0] * n[1] * nh,
                        sizeof(double) * 2 * kRedBlocks, sizeof(double) * S_COUNT};
    for (int a = 0; a < 3; ++a) {
        sizes[5 + a] = n[a] > 1 ? sizeof(cpx<T>) * n[a] : 0;
        sizes[8 + a] = sizeof(T) * n[a];
    }
    size_t off[11], total = 0;
    for (int i = 0; i < 11; ++i) {
        off[i] = total;
        total += (sizes[i] + 255) & ~(size_t)255;
    }
    if (total > kNoAllocBytes) return NLP_ERR_INVALID_ARG;
    void *base = nullptr;
    nlp_status s = noalloc_scratch(&base);
    if (s) return s;
    char *b = (char *)base;
    Work<T> W;
    memset(&W, 0, sizeof(W));
    W.rho = (T *)(b + off[0]);
    W.pot = (T *)(b + off[1]);
    W.spec = (cpx<T> *)(b + off[2]);
    W.part = (double *)(b + off[3]);
    W.scal = (double *)(b + off[4]);
    DevPlan<T> &D = W.PD;
    D.dim = p->grid.dim;
    for (int a = 0; a < 3; ++a) {
        D.n[a] = n[a];
        D.nf[a] = n[a];
        D.len[a].N = n[a];
        if (n[a] > 1) {
            // both radix lists, as make_fft_len fills them: the passes run on the same engines
            // as in nlp_energies
            if (!factor_radices(n[a], D.len[a].rad, &D.len[a].nrad) ||
                !factor_radices_reg(n[a], D.len[a].rad_reg, &D.len[a].nrad_reg))
                return NLP_ERR_UNSUPPORTED;
            cpx<T> *tw = (cpx<T> *)(b + off[5 + a]);
            k_fill_twiddles<T><<<(n[a] + 255) / 256, 256, 0, p->stream>>>(tw, n[a]);
            D.len[a].tw = tw;
        }
        T *ones = (T *)(b + off[8 + a]);
        k_fill_value<T><<<(n[a] + 255) / 256, 256, 0, p->stream>>>(ones, n[a], (T)1);
        D.deconv[a] = ones;
    }
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    D.nh = (int)nh;
    D.F = D.G = W.spec;
    return energies_t<T>(p, &W, x, V, beta, g, E);
}

nlp_status energies_noalloc_impl(nlp_plan_s *p, const void *phi, const void *V, double beta, double g, double *E) {
    if (p->prec == NLP_FP64) return energies_noalloc_t<double>(p, (const double *)phi, (const double *)V, beta, g, E);
    return energies_noalloc_t<float>(p, (const float *)phi, (const float *)V, beta, g, E);
}

}  // namespace nlp
