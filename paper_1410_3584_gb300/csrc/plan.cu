// Plan construction (host): quadrature of Eq. (ifft) (Sec. 2.1), spreading-function
// tables, node binning by fine-grid tile, FFT tables and workspace.
#include <atomic>
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "plan.h"

namespace nlp {

int max_dyn_smem() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    int v = cache[dev & 63].load();
    if (v) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
        return 48 * 1024;
    cache[dev & 63].store(v);
    return v;
}

// ------------------------------------------------------------------ Gauss-Legendre
// Nodes are the roots of the Legendre polynomial P_n, found by Newton's method from the
// asymptotic guess cos(pi (i + 3/4)/(n + 1/2)); P_n and P_n' come from the three-term
// recurrence (j P_j = (2j-1) x P_{j-1} - (j-1) P_{j-2}).  Weights 2 / ((1-x^2) P_n'(x)^2).
static void legendre_pd(int n, double z, double *pn, double *dp) {
    double pc = z, pm = 1.0;
    for (int j = 2; j <= n; ++j) {
        const double pj = ((2.0 * j - 1.0) * z * pc - (j - 1.0) * pm) / j;
        pm = pc;
        pc = pj;
    }
    *pn = (n == 0) ? 1.0 : pc;
    *dp = n * (z * pc - pm) / (z * z - 1.0);
}

void gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pd(n, z, &pn, &dp);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-16) break;
        }
        legendre_pd(n, z, &pn, &dp);
        const double wt = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = mid - half * z;      // roots come in +- pairs; ascending order
        x[n - 1 - i] = mid + half * z;
        w[i] = w[n - 1 - i] = half * wt;
    }
}

// ------------------------------------------------------------------ spreading function
// "Exponential of semicircle" (Barnett, Magland & af Klinteberg 2019), upsampling 2:
// phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), w = ceil(log10(1/tol)) + 1, beta = 2.30 w.
void es_params(double tol, int *w, double *beta) {
    int ww = (int)std::ceil(std::log10(1.0 / tol)) + 1;
    ww = std::max(2, std::min(ww, kMaxWidth));
    *w = ww;
    *beta = 2.30 * ww;
}

// psi-hat(xi) = int phi(z) cos(xi z) dz over |z| < w/2; with z = (w/2) sin(theta) the
// integrand exp(beta (cos theta - 1)) cos(xi w/2 sin theta) cos theta is smooth on
// [0, pi/2] and a 100-point Gauss-Legendre rule resolves it.
double es_fourier(double xi, int w, double beta) {
    static thread_local std::vector<double> gx, gw;
    if (gx.empty()) gauss_legendre(100, 0.0, 0.5 * M_PI, gx, gw);
    double s = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
        const double th = gx[i];
        s += gw[i] * std::exp(beta * (std::cos(th) - 1.0)) * std::cos(xi * 0.5 * w * std::sin(th)) * std::cos(th);
    }
    return w * s;
}

nlp_status alloc_dev(nlp_plan_s *p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return NLP_OK;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return NLP_ERR_OOM;
    }
    p->allocs.push_back(*ptr);
    p->bytes += bytes;
    return NLP_OK;
}

bool factor_radices(int N, int *rad, int *nrad) {
    int k = 0;
    while (N % 4 == 0 && k < kMaxRadices) { rad[k++] = 4; N /= 4; }
    while (N % 2 == 0 && k < kMaxRadices) { rad[k++] = 2; N /= 2; }
    while (N % 3 == 0 && k < kMaxRadices) { rad[k++] = 3; N /= 3; }
    while (N % 5 == 0 && k < kMaxRadices) { rad[k++] = 5; N /= 5; }
    *nrad = k;
    return N == 1;
}

// radices of the register engine: as many 16s as the power of two allows, the rest of it as
// one 8, 4 or 2, then 3s and 5s
bool factor_radices_reg(int N, int *rad, int *nrad) {
    int k = 0, p2 = 0;
    while (N % 2 == 0) { N /= 2; ++p2; }
    while (p2 >= 4 && k < 8) { rad[k++] = 16; p2 -= 4; }
    if (p2 > 0 && k < 8) rad[k++] = 1 << p2;
    while (N % 3 == 0 && k < 8) { rad[k++] = 3; N /= 3; }
    while (N % 5 == 0 && k < 8) { rad[k++] = 5; N /= 5; }
    *nrad = k;
    return N == 1;
}

template <typename T> nlp_status make_fft_len(nlp_plan_s *p, int N, FftLen<T> *out) {
    memset(out, 0, sizeof(*out));
    out->N = N;
    if (N == 1) return NLP_OK;
    if (!factor_radices(N, out->rad, &out->nrad)) return NLP_ERR_UNSUPPORTED;
    if (!factor_radices_reg(N, out->rad_reg, &out->nrad_reg)) return NLP_ERR_UNSUPPORTED;
    std::vector<cpx<T>> tw(N);
    for (int k = 0; k < N; ++k) {
        const double a = 2.0 * M_PI * (double)k / (double)N;
        tw[k].x = (T)std::cos(a);
        tw[k].y = (T)(-std::sin(a));
    }
    void *d = nullptr;
    nlp_status s = alloc_dev(p, &d, sizeof(cpx<T>) * N);
    if (s) return s;
    if (cudaMemcpy(d, tw.data(), sizeof(cpx<T>) * N, cudaMemcpyHostToDevice) != cudaSuccess) return NLP_ERR_CUDA;
    out->tw = (const cpx<T> *)d;
    return NLP_OK;
}
template nlp_status make_fft_len<float>(nlp_plan_s *, int, FftLen<float> *);
template nlp_status make_fft_len<double>(nlp_plan_s *, int, FftLen<double> *);

// W_1 of the 2D confined Coulomb kernel at eps |k| = t: (2/pi) int_0^inf exp(-t^2 s^2 / 2) / (1 + s^2) ds
// = exp(a) erfc(sqrt a) with a = t^2 / 2 (a classical integral); for large arguments the
// asymptotic series of exp(x^2) erfc(x), x = t / sqrt 2, avoids overflow
static double confined_w1(double t) {
    const double x = t / std::sqrt(2.0);
    if (x < 20.0) return std::exp(x * x) * std::erfc(x);
    const double y = 1.0 / (2.0 * x * x);
    return (1.0 - y * (1.0 - 3.0 * y * (1.0 - 5.0 * y * (1.0 - 7.0 * y)))) / (x * std::sqrt(M_PI));
}

static bool good_len(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    return n == 1;
}

// psi[j][a][i] = phi(2 (i - r_a - delta_a) / w), r_a = (tile offset of node j) mod Ts, zero
// outside the w taps: the kernel values of node j on the sub-window of its segment (FP64).
template <typename T>
__global__ void k_psi_table(T *tab, const T *nd, const uint32_t *no, int64_t M, int w, int Wsub, int Ts, double beta) {
    const int64_t total = M * 3 * Wsub;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / (3 * Wsub);
        const int r3 = (int)(e - j * 3 * Wsub), a = r3 / Wsub, i = r3 - a * Wsub;
        // Ts < 0: offsets are already taken from the sub-window origin
        const int r = Ts < 0 ? 0 : (int)((no[j] >> (8 * a)) & 0xff) % Ts;
        const int t = i - r;
        double v = 0.0;
        if (Ts < 0 || (t >= 0 && t < w)) {
            const double x = 2.0 * ((double)t - (double)nd[4 * j + a]) / w;
            const double sv = 1.0 - x * x;
            v = sv > 0 ? exp(beta * (sqrt(sv) - 1.0)) : 0.0;
        }
        tab[e] = (T)v;
    }
}

template <typename T>
cudaError_t launch_psi_table(T *tab, const T *nd, const uint32_t *no, int64_t M, int w, int Wsub, int Ts, double beta,
                             cudaStream_t st) {
    k_psi_table<T><<<152 * 16, 256, 0, st>>>(tab, nd, no, M, w, Wsub, Ts, beta);
    return cudaGetLastError();
}

static int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Node record before conversion to the plan precision.
struct HostNode {
    double z[3];     // fine-grid coordinates (cells); axis 0 = 0 in 2D
    double omega;    // h^d (2pi)^-d * quadrature weight * |k|^{d-1} U-hat
    double k[2], r;  // 2D Poisson: k and |k|
};

// Combine entries (see spread_common.cuh): for every chunk window, the output tiles of G its
// cells reach directly and through the Hermitian mirror, with the index offsets that map an
// output cell back to the window cell.  Per axis the window cells give a set of (tile, offset)
// pairs; the entries are the products of the three sets (direct: last-axis cells in [0, nf/2],
// mirror: last-axis cells at 0 or >= nf/2), sorted by tile, then by chunk.
template <typename T>
static nlp_status build_combine(nlp_plan_s *p, DevPlan<T> &D, const std::vector<Chunk> &act) {
    const int N[3] = {D.nf[0], D.nf[1], D.nf[2]};
    const int Nout[3] = {D.nf[0], D.nf[1], D.nh};
    const bool two = p->grid.dim == 2;
    // tile edges: a (y, z) face of at most 128 cells (one thread each in blocks of 128)
    D.cmb_t[0] = two ? 1 : 8;
    D.cmb_t[1] = 8;
    D.cmb_t[2] = two ? 16 : 8;
    for (int a = 0; a < 3; ++a) D.cmb_n[a] = (Nout[a] + D.cmb_t[a] - 1) / D.cmb_t[a];
    D.cmb_tiles = (int64_t)D.cmb_n[0] * D.cmb_n[1] * D.cmb_n[2];
    // chunks of one tile share its origin: group their slots (ascending); the first slot of
    // each group receives the group's sum before the combine, which then reads only it
    std::vector<std::pair<std::array<int, 3>, int>> byorg(act.size());
    for (size_t c = 0; c < act.size(); ++c) byorg[c] = {{act[c].bx, act[c].by, act[c].bz}, (int)c};
    std::sort(byorg.begin(), byorg.end());
    std::vector<int> grp, grp_list, reps;
    for (size_t i = 0; i < byorg.size();) {
        size_t k = i;
        while (k < byorg.size() && byorg[k].first == byorg[i].first) ++k;
        reps.push_back(byorg[i].second);
        if (k - i > 1) {
            grp.push_back((int)grp_list.size());
            grp.push_back((int)(k - i));
            for (size_t u = i; u < k; ++u) grp_list.push_back(byorg[u].second);
        }
        i = k;
    }
    D.ngroups = (int64_t)grp.size() / 2;
    D.grp_parts = (int)((D.win_cells + wsum_cells<T>() - 1) / wsum_cells<T>());
    D.grp = nullptr;
    D.grp_list = nullptr;
    if (D.ngroups > 0) {
        void *dg = nullptr, *dl = nullptr;
        nlp_status s;
        if ((s = alloc_dev(p, &dg, sizeof(int) * grp.size()))) return s;
        if ((s = alloc_dev(p, &dl, sizeof(int) * grp_list.size()))) return s;
        cudaMemcpy(dg, grp.data(), sizeof(int) * grp.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dl, grp_list.data(), sizeof(int) * grp_list.size(), cudaMemcpyHostToDevice);
        D.grp = (const int *)dg;
        D.grp_list = (const int *)dl;
    }
    struct Key { int64_t tile; CombEntry e; };
    std::vector<Key> keys;
    keys.reserve(reps.size() * 12);
    auto wrap = [](int64_t x, int n) { int64_t r = x % n; return (int)(r < 0 ? r + n : r); };
    for (int c : reps) {
        const int b[3] = {act[c].bx, act[c].by, act[c].bz};
        std::vector<std::pair<int, int>> dir[3], mir[3];
        for (int a = 0; a < 3; ++a) {
            for (int u = 0; u < D.win_n[a]; ++u) {
                const int l = wrap((int64_t)b[a] + u, N[a]);
                const bool last = a == 2;
                if (!last || 2 * l <= N[2]) dir[a].push_back({l / D.cmb_t[a], u - l});
                if (!last || l == 0 || 2 * l >= N[2]) {
                    const int m = (N[a] - l) % N[a];
                    mir[a].push_back({m / D.cmb_t[a], u + m});
                }
            }
            for (auto *v : {&dir[a], &mir[a]}) {
                std::sort(v->begin(), v->end());
                v->erase(std::unique(v->begin(), v->end()), v->end());
            }
        }
        for (int mr = 0; mr < 2; ++mr) {
            const auto *S = mr ? mir : dir;
            for (const auto &x : S[0])
                for (const auto &y : S[1])
                    for (const auto &z : S[2]) {
                        Key k;
                        k.tile = ((int64_t)x.first * D.cmb_n[1] + y.first) * D.cmb_n[2] + z.first;
                        k.e.chunk = (int)c;
                        k.e.mirror = mr;
                        k.e.o[0] = x.second;
                        k.e.o[1] = y.second;
                        k.e.o[2] = z.second;
                        keys.push_back(k);
                    }
        }
    }
    std::sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) {
        if (a.tile != b.tile) return a.tile < b.tile;
        if (a.e.chunk != b.e.chunk) return a.e.chunk < b.e.chunk;
        if (a.e.mirror != b.e.mirror) return a.e.mirror < b.e.mirror;
        for (int d = 0; d < 3; ++d)
            if (a.e.o[d] != b.e.o[d]) return a.e.o[d] < b.e.o[d];
        return false;
    });
    std::vector<int> off(D.cmb_tiles + 1, 0);
    std::vector<CombEntry> ent(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
        off[keys[i].tile + 1]++;
        ent[i] = keys[i].e;
    }
    std::vector<int> live;
    for (int64_t t = 0; t < D.cmb_tiles; ++t) {
        if (off[t + 1] > 0) live.push_back((int)t);
        off[t + 1] += off[t];
    }
    void *doff = nullptr, *dent = nullptr, *dact = nullptr;
    nlp_status s;
    if ((s = alloc_dev(p, &dact, sizeof(int) * std::max<size_t>(1, live.size())))) return s;
    if (!live.empty()) cudaMemcpy(dact, live.data(), sizeof(int) * live.size(), cudaMemcpyHostToDevice);
    D.cmb_act = (const int *)dact;
    D.cmb_nact = (int64_t)live.size();
    if ((s = alloc_dev(p, &doff, sizeof(int) * off.size()))) return s;
    if ((s = alloc_dev(p, &dent, sizeof(CombEntry) * std::max<size_t>(1, ent.size())))) return s;
    cudaMemcpy(doff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice);
    if (!ent.empty()) cudaMemcpy(dent, ent.data(), sizeof(CombEntry) * ent.size(), cudaMemcpyHostToDevice);
    D.cmb_off = (const int *)doff;
    D.cmb = (const CombEntry *)dent;
    p->info.combine_entries = (int64_t)ent.size();
    return NLP_OK;
}

template <typename T>
static nlp_status build_device(nlp_plan_s *p, const std::vector<HostNode> &nodes, DevPlan<T> &D) {
    D.dim = p->grid.dim;
    for (int a = 0; a < 3; ++a) {
        D.n[a] = p->n3[a];
        D.nf[a] = p->n3[a] == 1 ? 1 : 2 * p->n3[a];
    }
    D.nh = D.nf[2] / 2 + 1;
    D.w = p->info.width;
    D.beta = (T)p->info.beta_es;
    // register kernel (3D): sub-tile edge Ts with column length W = Ts + w - 1 (see spread_reg.cu)
    D.sub_T = 0;
    int Tt = p->opts.tile;
    if (p->grid.dim == 3 && p->opts.spread_variant != 1) {
        const int Ts = 2;
        if (reg_kernel_supported<T>(Ts + D.w - 1)) {
            D.sub_T = Ts;
            if (Tt == 0) Tt = sizeof(T) == 8 ? 4 : 8;
            if (Tt % Ts) Tt = (Tt / Ts + 1) * Ts;
        }
    }
    if (Tt == 0) Tt = (p->grid.dim == 2) ? 16 : (sizeof(T) == 8 ? 4 : 8);
    D.T_tile[0] = p->grid.dim == 3 ? Tt : 1;
    D.T_tile[1] = Tt;
    D.T_tile[2] = Tt;
    p->info.tile = Tt;
    p->info.sub_tile = D.sub_T;
    D.win_n[0] = D.T_tile[0] + (p->grid.dim == 3 ? D.w : 1) - 1;
    D.win_n[1] = D.T_tile[1] + D.w - 1;
    D.win_n[2] = D.T_tile[2] + D.w - 1;
    D.win_cells = (int64_t)D.win_n[0] * D.win_n[1] * D.win_n[2];
    const bool warp_k = D.sub_T > 0 && warp_kernel_used<T>(D.sub_T + D.w - 1);
    if (D.sub_T == 0 && generic_warps(D, (size_t)max_dyn_smem()) < 1) return NLP_ERR_UNSUPPORTED;
    if (D.sub_T > 0 && interp_spread_reg_smem(D, 4) > (size_t)max_dyn_smem()) return NLP_ERR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a) {
        nlp_status s = make_fft_len<T>(p, D.nf[a], &D.len[a]);
        if (s) return s;
    }
    // 2D: a fine axis 1 too long for the register engine's column blocks runs as two passes of
    // short transforms (four-step, N = N1 N2 with N2 in {32, 16, 8, 4}) through a scratch spectrum
    D.four = 0;
    D.S4 = nullptr;
    if (p->grid.dim == 2 && !cols_on_reg_engine<T>(D.len[1])) {
        const int N = D.len[1].N;
        for (int n2 : {32, 16, 8, 4}) {
            if (N % n2 || N / n2 < 2) continue;
            FftLen<T> a, b;
            if (make_fft_len<T>(p, N / n2, &a) || make_fft_len<T>(p, n2, &b)) return NLP_ERR_OOM;
            if (a.nrad_reg == 0 || b.nrad_reg == 0 || N / n2 > 128) continue;   // sub-lines of <= 128 points
            void *d4 = nullptr;
            nlp_status s = alloc_dev(p, &d4, sizeof(cpx<T>) * (size_t)D.nf[0] * D.nf[1] * D.nh);
            if (s) return s;
            D.len4[0] = a;
            D.len4[1] = b;
            D.S4 = (cpx<T> *)d4;
            D.four = 1;
            break;
        }
    }
    // deconvolution tables 1/psi-hat(2 pi (i - n/2)/nf)
    for (int a = 0; a < 3; ++a) {
        std::vector<T> dc(D.n[a]);
        for (int i = 0; i < D.n[a]; ++i) {
            if (D.n[a] == 1) { dc[i] = (T)1; continue; }
            const double xi = 2.0 * M_PI * (double)(i - D.n[a] / 2) / (double)D.nf[a];
            dc[i] = (T)(1.0 / es_fourier(xi, D.w, p->info.beta_es));
        }
        void *d;
        nlp_status s = alloc_dev(p, &d, sizeof(T) * dc.size());
        if (s) return s;
        cudaMemcpy(d, dc.data(), sizeof(T) * dc.size(), cudaMemcpyHostToDevice);
        D.deconv[a] = (const T *)d;
    }
    const size_t spec = (size_t)D.nf[0] * D.nf[1] * D.nh;
    void *dF, *dG;
    nlp_status s = alloc_dev(p, &dF, sizeof(cpx<T>) * spec);
    if (s) return s;
    s = alloc_dev(p, &dG, sizeof(cpx<T>) * spec);
    if (s) return s;
    D.F = (cpx<T> *)dF;
    D.G = (cpx<T> *)dG;
    // G: zeros outside the tiles the combine pass writes, kept so by every evaluation
    if (cudaMemset(dG, 0, sizeof(cpx<T>) * spec) != cudaSuccess) return NLP_ERR_CUDA;

    // ---- bin nodes by tile of their first tap, then by sub-tile inside the tile
    const int64_t M = (int64_t)nodes.size();
    const int wa[3] = {p->grid.dim == 3 ? D.w : 1, D.w, D.w};
    const int Ts = D.sub_T;
    const int nsub = (Ts > 0) ? D.T_tile[2] / Ts : 1;            // sub-tiles per tile edge (3D)
    const int64_t nsub3 = (int64_t)nsub * nsub * nsub;
    std::vector<int64_t> s0(M * 3), tb(M * 3);
    int64_t tmin[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, tmax[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; ++j)
        for (int a = 0; a < 3; ++a) {
            const int64_t sj = (int64_t)std::ceil(nodes[j].z[a] - 0.5 * wa[a]);
            s0[3 * j + a] = sj;
            tb[3 * j + a] = floordiv(sj, D.T_tile[a]);
        }
    for (int64_t j = 0; j < M; ++j)
        for (int a = 0; a < 3; ++a) {
            tmin[a] = std::min(tmin[a], tb[3 * j + a]);
            tmax[a] = std::max(tmax[a], tb[3 * j + a]);
        }
    int64_t K[3] = {1, 1, 1};
    if (M > 0)
        for (int a = 0; a < 3; ++a) K[a] = tmax[a] - tmin[a] + 1;
    const int64_t ntile = K[0] * K[1] * K[2];
    const int64_t nkey = ntile * nsub3;
    std::vector<int64_t> cnt(M > 0 ? nkey + 1 : 1, 0);
    std::vector<int64_t> key(M);
    for (int64_t j = 0; j < M; ++j) {
        const int64_t tk = ((tb[3 * j] - tmin[0]) * K[1] + (tb[3 * j + 1] - tmin[1])) * K[2] + (tb[3 * j + 2] - tmin[2]);
        int64_t sk = 0;
        if (Ts > 0)
            for (int a = 0; a < 3; ++a) sk = sk * nsub + (s0[3 * j + a] - tb[3 * j + a] * D.T_tile[a]) / Ts;
        key[j] = tk * nsub3 + sk;
        cnt[key[j] + 1]++;
    }
    for (int64_t t = 0; t < (M > 0 ? nkey : 0); ++t) cnt[t + 1] += cnt[t];
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - (M > 0 ? 1 : 0));
    std::vector<int64_t> order(M);
    for (int64_t j = 0; j < M; ++j) order[pos[key[j]]++] = j;
    // chunks (generic kernel: node ranges of one tile) and segments (register kernel:
    // runs of one sub-tile, chunked at segment boundaries)
    // generic chunks: 3D windows are large (fill and fold amortised over many nodes); the 2D
    // windows are small and the polar nodes crowd the tiles near k = 0, so short chunks spread
    // those tiles over many CTAs (measured at 1024^2: spread 0.27 -> 0.05 ms FP32)
#ifndef NLP_CHUNK3_F32
#define NLP_CHUNK3_F32 2048
#endif
    const int CH = p->grid.dim == 3 ? (sizeof(T) == 8 ? 256 : NLP_CHUNK3_F32) : (sizeof(T) == 8 ? 32 : 64);
    std::vector<Chunk> chunks, rchunks;
    std::vector<int> seg_node;
    std::vector<uint32_t> seg_sub;
    int64_t ntiles_used = 0;
    for (int64_t t = 0; t < (M > 0 ? ntile : 0); ++t) {
        const int64_t c0 = cnt[t * nsub3], c1 = cnt[(t + 1) * nsub3];
        if (c1 == c0) continue;
        ++ntiles_used;
        const int64_t k2 = t % K[2], k1 = (t / K[2]) % K[1], k0 = t / (K[1] * K[2]);
        Chunk ch;
        ch.bx = (int)((k0 + tmin[0]) * D.T_tile[0]);
        ch.by = (int)((k1 + tmin[1]) * D.T_tile[1]);
        ch.bz = (int)((k2 + tmin[2]) * D.T_tile[2]);
        const int64_t nch = (c1 - c0 + CH - 1) / CH;
        for (int64_t c = 0; c < nch; ++c) {
            ch.j0 = (int)(c0 + (c1 - c0) * c / nch);
            ch.j1 = (int)(c0 + (c1 - c0) * (c + 1) / nch);
            chunks.push_back(ch);
        }
        if (Ts > 0) {
            // pieces of at most SEGMAX nodes of one sub-tile (dense sub-tiles spread over all
            // warps of a CTA); a chunk closes at a piece boundary once it holds CH nodes
            const int SEGMAX = sizeof(T) == 8 ? 32 : 64;
            int64_t acc = 0;
            Chunk rc = ch;
            rc.j0 = (int)seg_sub.size();
            auto close = [&]() {
                rc.j1 = (int)seg_sub.size();
                if (rc.j1 > rc.j0) {
                    // heaviest pieces first inside the chunk (dynamic assignment to warps)
                    std::vector<int> idx(rc.j1 - rc.j0);
                    std::iota(idx.begin(), idx.end(), rc.j0);
                    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
                        return seg_node[2 * a + 1] - seg_node[2 * a] > seg_node[2 * b + 1] - seg_node[2 * b];
                    });
                    std::vector<int> sn(2 * idx.size());
                    std::vector<uint32_t> ss(idx.size());
                    for (size_t i = 0; i < idx.size(); ++i) {
                        sn[2 * i] = seg_node[2 * idx[i]];
                        sn[2 * i + 1] = seg_node[2 * idx[i] + 1];
                        ss[i] = seg_sub[idx[i]];
                    }
                    std::copy(sn.begin(), sn.end(), seg_node.begin() + 2 * rc.j0);
                    std::copy(ss.begin(), ss.end(), seg_sub.begin() + rc.j0);
                    rchunks.push_back(rc);
                }
                rc.j0 = (int)seg_sub.size();
                acc = 0;
            };
            for (int64_t u = 0; u < nsub3; ++u) {
                int64_t a0 = cnt[t * nsub3 + u];
                const int64_t a1 = cnt[t * nsub3 + u + 1];
                const uint32_t so = (uint32_t)((u / (nsub * nsub)) * Ts) | (uint32_t)(((u / nsub) % nsub) * Ts) << 8 |
                                    (uint32_t)((u % nsub) * Ts) << 16;
                while (a0 < a1) {
                    const int64_t take = std::min<int64_t>(a1 - a0, SEGMAX);
                    if (acc > 0 && acc + take > CH) close();
                    seg_node.push_back((int)a0);
                    seg_node.push_back((int)(a0 + take));
                    seg_sub.push_back(so);
                    acc += take;
                    a0 += take;
                }
            }
            close();
        }
    }
    auto by_size = [](const Chunk &a, const Chunk &b) { return (a.j1 - a.j0) > (b.j1 - b.j0); };
    std::stable_sort(chunks.begin(), chunks.end(), by_size);
    if (Ts > 0) {   // heaviest chunks (most nodes) first
        auto nodes_of = [&](const Chunk &c) {
            int64_t n = 0;
            for (int i = c.j0; i < c.j1; ++i) n += seg_node[2 * i + 1] - seg_node[2 * i];
            return n;
        };
        std::vector<std::pair<int64_t, int>> w(rchunks.size());
        for (size_t i = 0; i < rchunks.size(); ++i) w[i] = {nodes_of(rchunks[i]), (int)i};
        std::stable_sort(w.begin(), w.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
        std::vector<Chunk> sorted(rchunks.size());
        for (size_t i = 0; i < w.size(); ++i) sorted[i] = rchunks[w[i].second];
        rchunks.swap(sorted);
    }
    // node records, padded by 16 zero records: batch loads of the FP32 warp kernel may reach
    // past a piece's last node (those nodes get weight zero)
    std::vector<T> nd(4 * (size_t)(M + 16), (T)0);
    std::vector<uint32_t> no(M);
    const int Wsub = Ts + D.w - 1;
    // per-chunk sums of |omega_j| (they bound each chunk's window, see spread_dev.cuh)
    {
        std::vector<double> aom(M + 1, 0.0);
        for (int64_t q = 0; q < M; ++q) aom[q + 1] = aom[q] + std::fabs(nodes[order[q]].omega);
        auto up = [](double v) { return (float)(v * (1.0 + 1e-6)); };
        for (Chunk &c : chunks) c.wsum = up(aom[c.j1] - aom[c.j0]);
        for (Chunk &c : rchunks) {
            double sum = 0.0;
            for (int i = c.j0; i < c.j1; ++i) sum += aom[seg_node[2 * i + 1]] - aom[seg_node[2 * i]];
            c.wsum = up(sum);
        }
    }
    std::vector<double> pois;
    if (p->kernel == NLP_POISSON_2D) pois.resize(3 * (size_t)M);
    for (int64_t q = 0; q < M; ++q) {
        const int64_t j = order[q];
        uint32_t packed = 0;
        for (int a = 0; a < 3; ++a) {
            const int64_t sj = s0[3 * j + a];
            const int64_t o = sj - tb[3 * j + a] * D.T_tile[a];
            // offset of the node from its first tap; for the FP32 warp kernel, from the origin
            // of its sub-window (first tap + tile offset mod Ts), which that kernel evaluates
            // the kernel values against
            const double base = warp_k ? (double)(sj - o % Ts) : (double)sj;
            nd[4 * q + a] = (T)(nodes[j].z[a] - base);
            packed |= (uint32_t)o << (8 * a);
        }
        nd[4 * q + 3] = (T)nodes[j].omega;
        no[q] = packed;

        if (!pois.empty()) {
            pois[3 * q] = nodes[j].k[0];
            pois[3 * q + 1] = nodes[j].k[1];
            pois[3 * q + 2] = nodes[j].r;
        }
    }
    void *dnd = nullptr, *dno = nullptr, *dch = nullptr;
    if ((s = alloc_dev(p, &dnd, sizeof(T) * nd.size()))) return s;
    if ((s = alloc_dev(p, &dno, sizeof(uint32_t) * no.size()))) return s;
    if ((s = alloc_dev(p, &dch, sizeof(Chunk) * chunks.size()))) return s;
    if (M) {
        cudaMemcpy(dnd, nd.data(), sizeof(T) * nd.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dno, no.data(), sizeof(uint32_t) * no.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dch, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice);
    }
    D.rchunks = nullptr;
    D.nrchunks = 0;
    D.psi_tab = nullptr;
    if (Ts > 0 && M) {
        // team kernel: kernel values of every node (the nodes are fixed per plan), placed in
        // the sub-window of its segment; computed on the device from (delta, offsets).  The
        // FP32 warp kernel evaluates them per evaluation instead.
#ifdef NLP_WARP_TABLE
        const bool tab = true;
#else
        const bool tab = !warp_k;
#endif
        if (tab) {
            void *dpt;
            if ((s = alloc_dev(p, &dpt, sizeof(T) * (size_t)(M + 16) * 3 * Wsub))) return s;
            cudaMemsetAsync(dpt, 0, sizeof(T) * (size_t)(M + 16) * 3 * Wsub, p->stream);   // padding records
            if (launch_psi_table<T>((T *)dpt, (const T *)dnd, (const uint32_t *)dno, M, D.w, Wsub,
                                    warp_k ? -1 : Ts, p->info.beta_es, p->stream) != cudaSuccess)
                return NLP_ERR_CUDA;
            D.psi_tab = (const T *)dpt;
        }
        void *dsn, *dss, *drc;
        if ((s = alloc_dev(p, &dsn, sizeof(int) * seg_node.size()))) return s;
        if ((s = alloc_dev(p, &dss, sizeof(uint32_t) * seg_sub.size()))) return s;
        if ((s = alloc_dev(p, &drc, sizeof(Chunk) * rchunks.size()))) return s;
        cudaMemcpy(dsn, seg_node.data(), sizeof(int) * seg_node.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dss, seg_sub.data(), sizeof(uint32_t) * seg_sub.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(drc, rchunks.data(), sizeof(Chunk) * rchunks.size(), cudaMemcpyHostToDevice);
        D.seg_node = (const int *)dsn;
        D.seg_sub = (const uint32_t *)dss;
        D.rchunks = (const Chunk *)drc;
        D.nrchunks = (int64_t)rchunks.size();
        p->info.segments = (int64_t)seg_sub.size();
    }
    D.psi_gen = nullptr;
    if (p->grid.dim == 2 && M) {
        // 2D (generic kernel): the kernel values of every node on its own w taps, evaluated
        // once per plan in FP64 instead of per evaluation in the plan precision
        void *dpg;
        if ((s = alloc_dev(p, &dpg, sizeof(T) * (size_t)M * 3 * D.w))) return s;
        if (launch_psi_table<T>((T *)dpg, (const T *)dnd, (const uint32_t *)dno, M, D.w, D.w, 1, p->info.beta_es,
                                p->stream) != cudaSuccess)
            return NLP_ERR_CUDA;
        D.psi_gen = (const T *)dpg;
    }
    D.pois = nullptr;
    D.mom = nullptr;
    D.u1tab = nullptr;
    D.hvol = p->h[1] * p->h[2] * (p->grid.dim == 3 ? p->h[0] : 1.0);
    D.sigma = p->sigma;
    if (!pois.empty()) {
        void *dp, *dm, *dr;
        if ((s = alloc_dev(p, &dp, sizeof(double) * pois.size()))) return s;
        cudaMemcpy(dp, pois.data(), sizeof(double) * pois.size(), cudaMemcpyHostToDevice);
        p->d_pois = (double *)dp;
        p->red_blocks = 256;
        if ((s = alloc_dev(p, &dr, sizeof(double) * 3 * (p->red_blocks + 1)))) return s;
        p->d_red = (double *)dr;
        if ((s = alloc_dev(p, &dm, sizeof(double) * 4))) return s;
        cudaMemset(dm, 0, sizeof(double) * 4);
        D.pois = p->d_pois;
        D.mom = (const double *)dm;
        void *du;
        const int64_t Ng = (int64_t)p->n3[1] * p->n3[2];
        if ((s = alloc_dev(p, &du, sizeof(double) * 3 * (size_t)Ng))) return s;
        if (launch_u1_table((double *)du, p->n3[1], p->n3[2], p->L3, p->h, p->sigma_u1, p->stream) != cudaSuccess)
            return NLP_ERR_CUDA;
        D.u1tab = (const double *)du;
    }
    D.nd = (const T *)dnd;
    D.no = (const uint32_t *)dno;
    D.chunks = (const Chunk *)dch;
    D.nchunks = (int64_t)chunks.size();
    p->info.tiles = ntiles_used;
    p->info.chunks = D.nchunks;
    // FP32 warp kernels: per-node c_j (padded like the node records) and per-chunk bounds
    D.cnode = nullptr;
    D.csum = nullptr;
    if (warp_k && D.nrchunks > 0) {
        void *dc = nullptr, *ds = nullptr;
        if ((s = alloc_dev(p, &dc, sizeof(cpx<T>) * (size_t)(M + 16)))) return s;
        if ((s = alloc_dev(p, &ds, sizeof(T) * (size_t)D.nrchunks))) return s;
        cudaMemset(dc, 0, sizeof(cpx<T>) * (size_t)(M + 16));
        D.cnode = (cpx<T> *)dc;
        D.csum = (T *)ds;
    }
    // window scratch (one slot per chunk of the kernel that runs) and the combine entries
    {
        const std::vector<Chunk> &act = Ts > 0 ? rchunks : chunks;
        void *dw = nullptr;
        if ((s = alloc_dev(p, &dw, sizeof(cpx<T>) * (size_t)D.win_cells * std::max<size_t>(1, act.size())))) return s;
        D.win = (cpx<T> *)dw;
        if ((s = build_combine<T>(p, D, act))) return s;
    }
    if (cudaGetLastError() != cudaSuccess) return NLP_ERR_CUDA;
    return NLP_OK;
}

nlp_status build_split(nlp_plan_s *p);
nlp_status build_toeplitz(nlp_plan_s *p);

static int roundup16(double x) { return (int)(16.0 * std::ceil(x / 16.0)); }

// x with erfc(x) = y, 0 < y < 1: bisection on [0, 30] to the last bit (erfc is decreasing)
static double erfc_inverse(double y) {
    double lo = 0.0, hi = 30.0;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        (std::erfc(mid) > y ? lo : hi) = mid;
    }
    return 0.5 * (lo + hi);
}

nlp_status plan_build_1d(nlp_plan_s *p);

nlp_status plan_build(nlp_plan_s *p) {
    const nlp_grid &g = p->grid;
    const int d = g.dim;
    if (d == 1) return plan_build_1d(p);
    // collapsed 3D view
    if (d == 3) {
        for (int a = 0; a < 3; ++a) { p->n3[a] = g.n[a]; p->L3[a] = g.L[a]; }
    } else {
        p->n3[0] = 1; p->L3[0] = 1.0;
        p->n3[1] = g.n[0]; p->L3[1] = g.L[0];
        p->n3[2] = g.n[1]; p->L3[2] = g.L[1];
    }
    double hmax = 0, R2 = 0, Rp2 = 0;
    for (int a = 0; a < 3; ++a) {
        p->h[a] = (p->n3[a] == 1) ? 1.0 : 2.0 * p->L3[a] / p->n3[a];
        if (p->n3[a] > 1) hmax = std::max(hmax, p->h[a]);
    }
    for (int a = 0; a < d; ++a) R2 += g.L[a] * g.L[a];
    Rp2 = g.L[0] * g.L[0] + g.L[1] * g.L[1];
    const double Ptrunc = p->opts.kmax > 0 ? p->opts.kmax : M_PI / hmax;
    // improved algorithm (method 2): the NUFFT part I_2 only needs the ball where the
    // partition p(k) is above eps (Eq. (3.9)); I_1 is built after the nodes.  p = exp(-|k|^2/a)
    // for the 3D kernels and the 2D Laplace kernel, p = erfc(|k|/l) for 2D Coulomb (the only
    // choice of the two for which (1 - p)/|k| is smooth at k = 0); the scale puts the decay of
    // I_1's x-space kernel at the doubled grid's nearest image (distance 2 min L) near eps.
    double P = Ptrunc;
    if (p->opts.method == 2) {
        const bool f64 = p->prec == NLP_FP64;
        const double kappa = f64 ? 5.5 : 3.8, eps = f64 ? 1e-16 : 1e-8;
        double Lmin = g.L[0];
        for (int a = 1; a < d; ++a) Lmin = std::min(Lmin, g.L[a]);
        p->split = 1;
        if (p->kernel == NLP_COULOMB_2D) {
            p->split_erfc = 1;
            p->split_a = kappa / Lmin;
            p->split_k2 = std::min(Ptrunc, p->split_a * erfc_inverse(eps));
        } else {
            p->split_a = (kappa / Lmin) * (kappa / Lmin);
            p->split_k2 = std::min(Ptrunc, std::sqrt(p->split_a * std::log(1.0 / eps)));
        }
        P = p->split_k2;
        p->info.split_a = p->split_a;
        p->info.split_radius = p->split_k2;
    }
    int nr = p->opts.n_r, nth = p->opts.n_theta, nph = p->opts.n_phi;
    if (nr <= 0) nr = roundup16(P * std::sqrt(R2) / 2.0 + 16.0);
    if (d == 3 && nth <= 0) nth = nr;
    if (nph <= 0) nph = roundup16(P * (d == 3 ? std::sqrt(Rp2) : std::sqrt(R2)) + 32.0);
    if (d == 2) nth = 1;
    if ((d == 3 && (nth % 2)) || (nph % 2)) return NLP_ERR_INVALID_ARG;
    double tol = p->opts.nufft_tol > 0 ? p->opts.nufft_tol : (p->prec == NLP_FP64 ? 1e-12 : 1e-6);
    p->opts.nufft_tol = tol;
    int w;
    double beta;
    es_params(tol, &w, &beta);
    p->info.dim = d;
    p->info.kernel = p->kernel;
    p->info.precision = p->prec;
    for (int a = 0; a < 3; ++a) {
        p->info.n[a] = p->n3[a];
        p->info.nf[a] = p->n3[a] == 1 ? 1 : 2 * p->n3[a];
    }
    p->info.width = w;
    p->info.beta_es = beta;
    p->info.kmax = Ptrunc;
    p->info.n_r = nr;
    p->info.n_theta = nth;
    p->info.n_phi = nph;

    // ---- quadrature nodes of the k -> -k half (Eq. (ifft)); weights carry h^d (2pi)^-d and
    //      the Jacobian-weighted symbol |k|^{d-1} U-hat (Eq. (Kernal)); see nlpot.h
    std::vector<double> r, wr, u, wu;
    gauss_legendre(nr, 0.0, P, r, wr);
    std::vector<HostNode> nodes;
    const double twopi = 2.0 * M_PI;
    const double wph = twopi / nph;
    double hvol = 1.0;
    for (int a = 0; a < 3; ++a) if (p->n3[a] > 1) hvol *= p->h[a];
    const double pref = hvol / std::pow(twopi, d);
    double nax[3] = {0, 0, 1};
    if (p->kernel == NLP_DIPOLE_3D) {
        const double *da = p->opts.dipole_axis;
        const double nn = std::sqrt(da[0] * da[0] + da[1] * da[1] + da[2] * da[2]);
        if (nn > 0) for (int a = 0; a < 3; ++a) nax[a] = da[a] / nn;
    }
    std::vector<double> cph(nph), sph(nph);
    for (int c = 0; c < nph; ++c) {
        cph[c] = std::cos(twopi * c / nph);
        sph[c] = std::sin(twopi * c / nph);
    }
    if (d == 3) {
        gauss_legendre(nth, -1.0, 1.0, u, wu);
        nodes.resize((size_t)nr * (nth / 2) * nph);
#pragma omp parallel for collapse(2) schedule(static)
        for (int ia = 0; ia < nr; ++ia)
            for (int ib = nth / 2; ib < nth; ++ib) {   // u > 0 half (ascending GL nodes)
                const double st = std::sqrt(std::max(0.0, 1.0 - u[ib] * u[ib]));
                for (int ic = 0; ic < nph; ++ic) {
                    HostNode &hn = nodes[((size_t)ia * (nth / 2) + (ib - nth / 2)) * nph + ic];
                    hn = HostNode{};
                    const double k[3] = {r[ia] * st * cph[ic], r[ia] * st * sph[ic], r[ia] * u[ib]};
                    double J = 1.0;
                    if (p->kernel == NLP_DIPOLE_3D) {
                        const double nk = nax[0] * k[0] + nax[1] * k[1] + nax[2] * k[2];
                        J = 3.0 * nk * nk - r[ia] * r[ia];
                    }
                    hn.omega = pref * wr[ia] * wu[ib] * wph * J;
                    if (p->split) hn.omega *= std::exp(-r[ia] * r[ia] / p->split_a);   // p(k) of Eq. (3.9)
                    for (int a = 0; a < 3; ++a) hn.z[a] = k[a] * p->h[a] * (2.0 * p->n3[a]) / twopi;
                }
            }
        p->info.nodes_total = (int64_t)nr * nth * nph;
    } else {
        nodes.reserve((size_t)nr * (nph / 2));
        for (int ia = 0; ia < nr; ++ia)
            for (int ic = 0; ic < nph / 2; ++ic) {     // phi in [0, pi): k_y >= 0 half
                HostNode hn{};
                const double k[2] = {r[ia] * cph[ic], r[ia] * sph[ic]};
                if (p->kernel == NLP_POISSON_2D)       // W(k) form of Algorithm 1; h^2 applied in-kernel
                    hn.omega = wr[ia] * wph / (twopi * twopi * r[ia]);
                else if (p->kernel == NLP_CONFINED_2D) // |k| U-hat = W_1(|k|), Eq. (2Dw1)
                    hn.omega = pref * wr[ia] * wph * confined_w1(p->opts.confine_eps * r[ia]);
                else
                    hn.omega = pref * wr[ia] * wph;    // Coulomb 2D: |k| U-hat = 1
                if (p->split)                          // p(k) of Eq. (3.9)
                    hn.omega *= p->split_erfc ? std::erfc(r[ia] / p->split_a) : std::exp(-r[ia] * r[ia] / p->split_a);
                hn.z[0] = 0.0;
                hn.z[1] = k[0] * p->h[1] * (2.0 * p->n3[1]) / twopi;
                hn.z[2] = k[1] * p->h[2] * (2.0 * p->n3[2]) / twopi;
                hn.k[0] = k[0];
                hn.k[1] = k[1];
                hn.r = r[ia];
                nodes.push_back(hn);
            }
        p->info.nodes_total = (int64_t)nr * nph;
    }
    p->info.nodes_half = (int64_t)nodes.size();
    if (p->kernel == NLP_POISSON_2D) p->sigma = 6.0 * std::sqrt(2.0) / P;
    p->info.sigma_poisson = p->sigma;
    // u_1 of Algorithm 1; with the partition, p G_1-hat is G_1-hat of the Gaussian widened by
    // exp(-|k|^2/a) = exp(-(2/a)|k|^2/2), whose potential u_1 has sigma^2 + 2/a
    p->sigma_u1 = p->split ? std::sqrt(p->sigma * p->sigma + 2.0 / p->split_a) : p->sigma;

    nlp_status s = (p->prec == NLP_FP64) ? build_device<double>(p, nodes, p->pd) : build_device<float>(p, nodes, p->pf);
    if (s) return s;
    if (p->opts.method == 1) {
        std::vector<HostNode>().swap(nodes);
        if ((s = build_toeplitz(p))) return s;
    }
    if (p->opts.method == 2 && (s = build_split(p))) return s;
    p->info.workspace_bytes = p->bytes;
    return NLP_OK;
}

nlp_status validate(const nlp_grid *g, nlp_kernel kernel, nlp_precision prec, const nlp_opts *o) {
    if (!g) return NLP_ERR_INVALID_ARG;
    if (g->dim < 1 || g->dim > 3) return NLP_ERR_INVALID_ARG;
    if ((kernel == NLP_COULOMB_3D || kernel == NLP_DIPOLE_3D) && g->dim != 3) return NLP_ERR_INVALID_ARG;
    if ((kernel == NLP_COULOMB_2D || kernel == NLP_POISSON_2D || kernel == NLP_CONFINED_2D) && g->dim != 2)
        return NLP_ERR_INVALID_ARG;
    if ((kernel == NLP_POISSON_1D) != (g->dim == 1)) return NLP_ERR_INVALID_ARG;
    if ((int)kernel < 0 || (int)kernel > 5) return NLP_ERR_INVALID_ARG;
    if (kernel == NLP_POISSON_1D && prec == NLP_FP32) return NLP_ERR_UNSUPPORTED;
    if (kernel == NLP_POISSON_1D && o && o->method != 0) return NLP_ERR_UNSUPPORTED;
    if (kernel == NLP_CONFINED_2D && o && !(o->confine_eps >= 0.0 && std::isfinite(o->confine_eps)))
        return NLP_ERR_INVALID_ARG;
    if (prec != NLP_FP64 && prec != NLP_FP32) return NLP_ERR_INVALID_ARG;
    for (int a = 0; a < g->dim; ++a) {
        const int n = g->n[a];
        if (n < 8 || n % 2 || !good_len(n) || n > (g->dim == 3 ? 256 : 1024)) return NLP_ERR_INVALID_ARG;
        if (!(g->L[a] > 0.0) || !std::isfinite(g->L[a])) return NLP_ERR_INVALID_ARG;
    }
    if (o) {
        if (o->nufft_tol != 0.0 && !(o->nufft_tol >= 1e-14 && o->nufft_tol <= 1e-2)) return NLP_ERR_INVALID_ARG;
        if (o->kmax < 0.0 || !std::isfinite(o->kmax)) return NLP_ERR_INVALID_ARG;
        if (o->n_r < 0 || o->n_theta < 0 || o->n_phi < 0) return NLP_ERR_INVALID_ARG;
        if (o->n_r > 4096 || o->n_theta > 4096 || o->n_phi > 8192) return NLP_ERR_INVALID_ARG;
        if ((o->n_theta % 2) || (o->n_phi % 2)) return NLP_ERR_INVALID_ARG;
        if (o->tile != 0 && (o->tile < 2 || o->tile > 32)) return NLP_ERR_INVALID_ARG;
        if (o->spread_variant < 0 || o->spread_variant > 1) return NLP_ERR_INVALID_ARG;
        if (o->method < 0 || o->method > 2) return NLP_ERR_INVALID_ARG;
        if (o->method == 1 && kernel == NLP_POISSON_2D) return NLP_ERR_UNSUPPORTED;
        if (o->method == 2 && !(g->dim == 3 || kernel == NLP_COULOMB_2D || kernel == NLP_POISSON_2D))
            return NLP_ERR_UNSUPPORTED;
        if (o->method == 1)   // the kernel is built on a 4n-point fine grid
            for (int a = 0; a < g->dim; ++a)
                if (4 * g->n[a] > kMaxFftLen) return NLP_ERR_UNSUPPORTED;
        for (int i = 0; i < 5; ++i)
            if (o->reserved[i]) return NLP_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(o->dipole_axis[a])) return NLP_ERR_INVALID_ARG;
    }
    return NLP_OK;
}

}  // namespace nlp
