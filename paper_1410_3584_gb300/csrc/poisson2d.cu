// 2D Poisson potential, Algorithm 1 (Sec. 2.2): the FP64 parts.
//   step 1: (x rho)-hat(0) = M1 by an FP64 trapezoid reduction; rho-hat(0) = C0 taken from
//           the same type-2 transform that gives rho-hat at the nodes (interpolation at k = 0),
//           so that the transform error cancels in W(k) near the origin;
//   step 2: u_1 = C0 u_{1,1} - M1 . u_{1,2} (Eqs. (phi1_exct), (phi12_ext)) in FP64, added to
//           u_2 on the grid (step 4);
//   step 3 (u_2) runs through the shared NUFFT kernels with the W(k) scaling of spread.cu.
#include "common.cuh"
#include "launch.h"
#include <algorithm>

namespace nlp {

// E_1(z), z > 0: series for z <= 1 (Abramowitz & Stegun 5.1.11),
//   E_1(z) = -gamma - ln z - sum_{k>=1} (-z)^k / (k k!),
// continued fraction for z > 1 (A&S 5.1.22), evaluated by the modified Lentz method:
//   E_1(z) = e^{-z} / (z + 1 - 1^2/(z + 3 - 2^2/(z + 5 - ...))).
__device__ double expint_e1(double z) {
    const double euler = 0.57721566490153286061;
    if (z <= 1.0) {
        double term = 1.0, sum = 0.0;
        for (int k = 1; k < 60; ++k) {
            term *= -z / k;                 // (-z)^k / k!
            const double add = term / k;
            sum += add;
            if (fabs(add) < 1e-17 * fabs(sum)) break;
        }
        return -euler - log(z) - sum;
    }
    if (z > 740.0) return 0.0;
    const double tiny = 1e-300;
    double b = z + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 500; ++i) {
        const double an = -(double)i * i;
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-16) break;
    }
    return h * exp(-z);
}

// Per-block FP64 partial sums of rho, x rho, y rho (grid index order, x_m = -L + m h).
template <typename T>
__global__ void k_moments_partial(const T *__restrict__ rho, int nx, int ny, double Lx, double Ly, double hx,
                                  double hy, double *part) {
    double s0 = 0, s1 = 0, s2 = 0;
    const int64_t N = (int64_t)nx * ny;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / ny), j = (int)(q % ny);
        const double v = (double)rho[q];
        s0 += v;
        s1 += (-Lx + i * hx) * v;
        s2 += (-Ly + j * hy) * v;
    }
    __shared__ double sh[3][32];
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = s0; sh[1][warp] = s1; sh[2][warp] = s2; }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        s0 = lane < nw ? sh[0][lane] : 0.0;
        s1 = lane < nw ? sh[1][lane] : 0.0;
        s2 = lane < nw ? sh[2][lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        }
        if (lane == 0) {
            part[3 * blockIdx.x] = s0;
            part[3 * blockIdx.x + 1] = s1;
            part[3 * blockIdx.x + 2] = s2;
        }
    }
}

__global__ void k_moments_final(const double *part, int nblocks, double hvol, double *mom) {
    // one warp, fixed order: deterministic
    double s[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += 32)
        for (int c = 0; c < 3; ++c) s[c] += part[3 * b + c];
    for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], off);
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) mom[c] = hvol * s[c];
}

// rho-hat(0) from the forward spectrum: the type-2 interpolation at k = 0 (one block).
template <typename T>
__global__ void k_interp_origin(DevPlan<T> P, double *mom) {
    const int w = P.w;
    const int s0 = (int)ceil(-0.5 * w);   // first tap of a node at z = 0
    const double two_w = 2.0 / w;
    double acc = 0.0;
    for (int p = threadIdx.x; p < w * w; p += blockDim.x) {
        const int b = p / w, c = p % w;
        const int l1 = s0 + b, l2 = s0 + c;
        const double x1 = (double)(l1) * two_w, x2 = (double)(l2) * two_w;
        const double s1 = 1.0 - x1 * x1, s2 = 1.0 - x2 * x2;
        const double k1 = s1 > 0 ? exp((double)P.beta * (sqrt(s1) - 1.0)) : 0.0;
        const double k2 = s2 > 0 ? exp((double)P.beta * (sqrt(s2) - 1.0)) : 0.0;
        const int m1 = ((l1 % P.nf[1]) + P.nf[1]) % P.nf[1];
        const int m2 = ((l2 % P.nf[2]) + P.nf[2]) % P.nf[2];
        cpx<T> f;
        if (2 * m2 <= P.nf[2]) f = P.F[(int64_t)m1 * P.nh + m2];
        else f = conj(P.F[(int64_t)(m1 ? P.nf[1] - m1 : 0) * P.nh + (P.nf[2] - m2)]);
        acc += (double)f.x * k1 * k2;   // imaginary part cancels by symmetry of the taps
    }
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        mom[0] = P.hvol * t;
    }
}

// u_{1,1}(x) and u_{1,2}(x) of the auxiliary Gaussian at every grid point (FP64; Eqs.
// (phi1_exct), (phi12_ext)): they depend only on the grid and sigma, so the plan tabulates
// them once and every evaluation adds C0 u_{1,1} - M1 . u_{1,2}.
__global__ void k_u1_table(double *tab, int nx, int ny, double Lx, double Ly, double hx, double hy, double sigma) {
    const int64_t N = (int64_t)nx * ny;
    const double inv4pi = 0.25 / 3.14159265358979323846, inv2pi = 0.5 / 3.14159265358979323846;
    const double euler = 0.57721566490153286061;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / ny), j = (int)(q % ny);
        const double x = -Lx + i * hx, y = -Ly + j * hy;
        const double r2 = x * x + y * y;
        double u11, u12x = 0, u12y = 0;
        if (r2 > 0) {
            const double z = r2 / (2.0 * sigma * sigma);
            u11 = -(expint_e1(z) + log(r2)) * inv4pi;
            const double f = -(1.0 - exp(-z)) * inv2pi / r2;
            u12x = f * x;
            u12y = f * y;
        } else {
            u11 = (euler - log(2.0 * sigma * sigma)) * inv4pi;
        }
        tab[3 * q] = u11;
        tab[3 * q + 1] = u12x;
        tab[3 * q + 2] = u12y;
    }
}

// phi += C0 u_{1,1}(x) - M1 . u_{1,2}(x) from the plan's table (FP64 arithmetic)
template <typename T> __global__ void k_u1_add(T *phi, int64_t N, const double *__restrict__ tab, const double *mom) {
    const double C0 = mom[0], M1x = mom[1], M1y = mom[2];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        phi[q] = (T)((double)phi[q] + C0 * tab[3 * q] - (M1x * tab[3 * q + 1] + M1y * tab[3 * q + 2]));
}

cudaError_t launch_u1_table(double *tab, int nx, int ny, const double *L, const double *h, double sigma,
                            cudaStream_t st) {
    const int64_t N = (int64_t)nx * ny;
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 8);
    k_u1_table<<<blocks, 256, 0, st>>>(tab, nx, ny, L[1], L[2], h[1], h[2], sigma);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poisson_moments(const T *rho, const DevPlan<T> &P, const double *L, const double *h,
                                   double *part, int nblocks, double *mom, cudaStream_t st) {
    k_moments_partial<T><<<nblocks, 256, 0, st>>>(rho, P.n[1], P.n[2], L[1], L[2], h[1], h[2], part);
    k_moments_final<<<1, 32, 0, st>>>(part, nblocks, P.hvol, mom);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poisson_origin(const DevPlan<T> &P, double *mom, cudaStream_t st) {
    k_interp_origin<T><<<1, 256, 0, st>>>(P, mom);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poisson_u1(T *phi, const DevPlan<T> &P, const double *L, const double *h, cudaStream_t st) {
    const int64_t N = (int64_t)P.n[1] * P.n[2];
    const int blocks = (int)std::min<int64_t>((N + 255) / 256, 152 * 8);
    (void)L;
    (void)h;
    k_u1_add<T><<<blocks, 256, 0, st>>>(phi, N, P.u1tab, P.mom);
    return cudaGetLastError();
}

#define INST(T)                                                                                              \
    template cudaError_t launch_poisson_moments<T>(const T *, const DevPlan<T> &, const double *, const double *, \
                                                   double *, int, double *, cudaStream_t);                   \
    template cudaError_t launch_poisson_origin<T>(const DevPlan<T> &, double *, cudaStream_t);              \
    template cudaError_t launch_poisson_u1<T>(T *, const DevPlan<T> &, const double *, const double *, cudaStream_t);
INST(float)
INST(double)

}  // namespace nlp
