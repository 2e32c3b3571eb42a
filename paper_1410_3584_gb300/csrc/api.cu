// C-ABI entry points of libnlpot (declared in include/nlpot.h).
#include <cmath>
#include <cstring>
#include <new>

#include "launch.h"
#include "plan.h"

namespace nlp {
nlp_status validate(const nlp_grid *g, nlp_kernel kernel, nlp_precision prec, const nlp_opts *o);
nlp_status plan_build(nlp_plan_s *p);
nlp_status gf_step_impl(nlp_plan_s *p, void *phi, const void *V, double beta, double g, double tau,
                        double inner_tol, int max_inner, double *max_change, int *inner_iters, double *energies);
nlp_status energies_impl(nlp_plan_s *p, const void *phi, const void *V, double beta, double g, double *energies);
nlp_status ts_step_impl(nlp_plan_s *p, void *psi, const void *V, double beta, double g, double tau, int order);
nlp_status energies_noalloc_impl(nlp_plan_s *p, const void *phi, const void *V, double beta, double g, double *E);

// Stage markers for the optional event timers (ids are part of the ABI: nlpot.h).
static inline void mark(nlp_plan_s *p, int stage) {
    if (!p->timing || p->nev >= 32) return;
    cudaEventRecord(p->ev[p->nev], p->stream);
    p->ev_stage[p->nev++] = stage;
}

// phi = U * rho on the plan's stream (see nlp_eval_potential).
template <typename T>
nlp_status eval_impl(nlp_plan_s *p, DevPlan<T> &D, const T *rho, T *phi) {
    cudaStream_t st = p->stream;
    const bool three = p->grid.dim == 3;
    const bool pois = p->kernel == NLP_POISSON_2D && D.mom != nullptr;   // not the I_1 part of method 2
    const int64_t nh = D.nh;
    if (pois) {
        NLP_CUDA_TRY(launch_poisson_moments<T>(rho, D, p->L3, p->h, p->d_red, p->red_blocks, (double *)D.mom, st));
        mark(p, NLP_STAGE_POISSON);
    }
    // type 2: deconvolve, zero-pad, forward FFT (last axis, then axis 1, then axis 0)
    NLP_CUDA_TRY(launch_fwd_r2c<T>(rho, D, st));
    mark(p, NLP_STAGE_FWD_LAST);
    StridedDesc a1{};
    a1.n_in = D.n[1];
    a1.n_out = D.nf[1];
    a1.es = nh;
    a1.ncol = (int)nh;
    a1.nouter = three ? D.n[0] : 1;
    a1.os = (int64_t)D.nf[1] * nh;
    a1.outer_map_n = three ? D.n[0] : 0;
    a1.outer_map_N = D.nf[0];
    if (!three && D.four) NLP_CUDA_TRY(launch_fft_four<T>(D.F, D.F, a1, D, -1, st));
    else NLP_CUDA_TRY(launch_fft_strided<T>(D.F, a1, D.len[1], -1, st));
    mark(p, NLP_STAGE_FWD_MID);
    StridedDesc a0{};
    if (three) {
        a0.n_in = D.n[0];
        a0.n_out = D.nf[0];
        a0.es = (int64_t)D.nf[1] * nh;
        a0.ncol = (int)nh;
        a0.nouter = D.nf[1];
        a0.os = nh;
        NLP_CUDA_TRY(launch_fft_strided<T>(D.F, a0, D.len[0], -1, st));
        mark(p, NLP_STAGE_FWD_FIRST);
    }
    if (pois) {
        NLP_CUDA_TRY(launch_poisson_origin<T>(D, (double *)D.mom, st));
        mark(p, NLP_STAGE_POISSON);
    }
    if (D.Khat) {
        // precomputed discrete kernel: pointwise product with its spectrum (in place)
        NLP_CUDA_TRY(launch_mul_spec<T>(D.F, D.Khat, (int64_t)D.nf[0] * D.nf[1] * nh, st));
        mark(p, NLP_STAGE_SPREAD);
    } else {
        // interpolate, scale, spread (each chunk's window to its scratch slot), then combine
        // the windows into G (every cell of G written once, in a fixed order)
        if (D.cnode) {
            NLP_CUDA_TRY(launch_interp_warp<T>(D, st));
            mark(p, NLP_STAGE_INTERP);
        }
        if (D.sub_T > 0) NLP_CUDA_TRY(launch_interp_spread_reg<T>(D, st));
        else NLP_CUDA_TRY(launch_interp_spread<T>(D, st));
        mark(p, NLP_STAGE_SPREAD);
        if (D.ngroups > 0) {
            NLP_CUDA_TRY(launch_window_sum<T>(D, st));
            mark(p, NLP_STAGE_WINDOW_SUM);
        }
        NLP_CUDA_TRY(launch_combine<T>(D, st));
        mark(p, NLP_STAGE_COMBINE);
    }
    // type 1: inverse FFT (axis 0, axis 1, last axis), deconvolve, crop.  After a spread, the
    // first inverse pass reads G and writes F (free once the spread has read it), so G keeps
    // the zeros the combine pass does not rewrite; the other passes work on F.
    const bool oop = D.Khat == nullptr && D.G != D.F;
    cpx<T> *R = oop ? D.F : D.G;
    if (three) {
        StridedDesc b0 = a0;
        b0.n_in = D.nf[0];
        b0.n_out = D.n[0];
        b0.out = R;
        NLP_CUDA_TRY(launch_fft_strided<T>(D.G, b0, D.len[0], +1, st));
        mark(p, NLP_STAGE_INV_FIRST);
    }
    StridedDesc b1 = a1;
    b1.n_in = D.nf[1];
    b1.n_out = D.n[1];
    b1.out = R;
    if (!three && D.four) NLP_CUDA_TRY(launch_fft_four<T>(D.G, R, b1, D, +1, st));
    else NLP_CUDA_TRY(launch_fft_strided<T>(three ? R : D.G, b1, D.len[1], +1, st));
    mark(p, NLP_STAGE_INV_MID);
    DevPlan<T> Dr = D;
    Dr.G = R;
    NLP_CUDA_TRY(launch_inv_c2r<T>(phi, Dr, st));
    mark(p, NLP_STAGE_INV_LAST);
    if (pois) {
        NLP_CUDA_TRY(launch_poisson_u1<T>(phi, D, p->L3, p->h, st));
        mark(p, NLP_STAGE_POISSON);
    }
    return NLP_OK;
}

nlp_status eval_1d(nlp_plan_s *p, const double *rho, double *phi);

nlp_status eval_any(nlp_plan_s *p, const void *rho, void *phi) {
    if (p->grid.dim == 1) return eval_1d(p, (const double *)rho, (double *)phi);
    p->nev = 0;
    mark(p, -1);
    nlp_status s;
    if (p->prec == NLP_FP64) {
        s = eval_impl<double>(p, p->pd, (const double *)rho, (double *)phi);
        // improved algorithm: I_2 (above, small-ball NUFFT) + I_1 (FFT convolution, accumulated)
        if (!s && p->split) s = eval_impl<double>(p, p->pd1, (const double *)rho, (double *)phi);
        return s;
    }
    s = eval_impl<float>(p, p->pf, (const float *)rho, (float *)phi);
    if (!s && p->split) s = eval_impl<float>(p, p->pf1, (const float *)rho, (float *)phi);
    return s;
}

size_t grid_points(const nlp_plan_s *p) {
    size_t N = 1;
    for (int a = 0; a < p->grid.dim; ++a) N *= (size_t)p->grid.n[a];
    return N;
}

size_t real_size(const nlp_plan_s *p) { return p->prec == NLP_FP64 ? 8 : 4; }

}  // namespace nlp

using namespace nlp;

extern "C" {

const char *nlp_version(void) { return "nlpot 0.1 (sm_103a)"; }

const char *nlp_status_string(nlp_status s) {
    switch (s) {
        case NLP_OK: return "ok";
        case NLP_ERR_INVALID_ARG: return "invalid argument";
        case NLP_ERR_UNSUPPORTED: return "unsupported configuration";
        case NLP_ERR_OOM: return "out of device memory";
        case NLP_ERR_CUDA: return "CUDA error";
        case NLP_ERR_TIMEOUT: return "device wait timed out";
        case NLP_ERR_DIVERGED: return "iteration diverged (non-finite values)";
        case NLP_ERR_NOT_CONVERGED: return "inner iteration did not converge";
    }
    return "unknown status";
}

void nlp_plan_destroy(nlp_plan p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    for (void *a : p->allocs) cudaFree(a);
    if (p->d_work && p->work_free) p->work_free(p->d_work);
    for (int i = 0; i < 32; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    delete p;
}

nlp_status nlp_plan_create(const nlp_grid *grid, nlp_kernel kernel, nlp_precision prec, const nlp_opts *opts,
                           void *stream, nlp_plan *out) {
    if (!out) return NLP_ERR_INVALID_ARG;
    *out = nullptr;
    nlp_status s = validate(grid, kernel, prec, opts);
    if (s) return s;
    nlp_plan_s *p = new (std::nothrow) nlp_plan_s();
    if (!p) return NLP_ERR_OOM;
    p->grid = *grid;
    p->kernel = kernel;
    p->prec = prec;
    if (opts) p->opts = *opts;
    else memset(&p->opts, 0, sizeof(p->opts));
    p->stream = (cudaStream_t)stream;
    try {
        s = plan_build(p);
    } catch (const std::bad_alloc &) {
        s = NLP_ERR_OOM;
    } catch (...) {
        s = NLP_ERR_CUDA;
    }
    if (s == NLP_OK && cudaDeviceSynchronize() != cudaSuccess) s = NLP_ERR_CUDA;
    if (s) {
        nlp_plan_destroy(p);
        return s;
    }
    *out = p;
    return NLP_OK;
}

nlp_status nlp_plan_get_info(nlp_plan p, nlp_plan_info *out) {
    if (!p || !out) return NLP_ERR_INVALID_ARG;
    *out = p->info;
    return NLP_OK;
}

nlp_status nlp_eval_potential(nlp_plan p, const void *rho_dev, void *phi_dev) {
    if (!p || !rho_dev || !phi_dev || rho_dev == phi_dev) return NLP_ERR_INVALID_ARG;
    return eval_any(p, rho_dev, phi_dev);
}

nlp_status nlp_eval_potential_host(nlp_plan p, const void *rho_host, void *phi_host) {
    if (!p || !rho_host || !phi_host) return NLP_ERR_INVALID_ARG;
    const size_t bytes = grid_points(p) * real_size(p);
    if (!p->d_host_io) {
        nlp_status s = alloc_dev(p, &p->d_host_io, 2 * bytes);
        if (s) return s;
        p->info.workspace_bytes = p->bytes;
    }
    char *drho = (char *)p->d_host_io, *dphi = drho + bytes;
    NLP_CUDA_TRY(cudaMemcpyAsync(drho, rho_host, bytes, cudaMemcpyHostToDevice, p->stream));
    nlp_status s = eval_any(p, drho, dphi);
    if (s) return s;
    NLP_CUDA_TRY(cudaMemcpyAsync(phi_host, dphi, bytes, cudaMemcpyDeviceToHost, p->stream));
    NLP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    return NLP_OK;
}

nlp_status nlp_gf_step(nlp_plan p, void *phi_dev, const void *V_dev, double beta, double g, double tau,
                       double inner_tol, int max_inner, double *max_change, int *inner_iters, double *energies) {
    if (!p || !phi_dev || !V_dev || !(tau > 0) || !(inner_tol > 0) || max_inner < 1) return NLP_ERR_INVALID_ARG;
    if (p->grid.dim == 1) return NLP_ERR_UNSUPPORTED;
    return gf_step_impl(p, phi_dev, V_dev, beta, g, tau, inner_tol, max_inner, max_change, inner_iters, energies);
}

nlp_status nlp_gf_solve(nlp_plan p, void *phi_dev, const void *V_dev, double beta, double g, double tau,
                        double stop_tol, int max_steps, double inner_tol, int max_inner, int *steps,
                        double *max_change, double *energies) {
    if (!p || !phi_dev || !V_dev || !(tau > 0) || !(stop_tol > 0) || max_steps < 1 || !(inner_tol > 0) ||
        max_inner < 1)
        return NLP_ERR_INVALID_ARG;
    if (p->grid.dim == 1) return NLP_ERR_UNSUPPORTED;
    double ch = INFINITY;
    int n = 0;
    nlp_status s = NLP_OK;
    while (n < max_steps) {
        s = gf_step_impl(p, phi_dev, V_dev, beta, g, tau, inner_tol, max_inner, &ch, nullptr, nullptr);
        ++n;
        // an inner solve that hit its cap still leaves a normalised iterate; keep going
        if (s != NLP_OK && s != NLP_ERR_NOT_CONVERGED) break;
        s = NLP_OK;
        if (ch <= stop_tol) break;
    }
    if (steps) *steps = n;
    if (max_change) *max_change = ch;
    if (s) return s;
    if (energies && (s = energies_impl(p, phi_dev, V_dev, beta, g, energies))) return s;
    return ch <= stop_tol ? NLP_OK : NLP_ERR_NOT_CONVERGED;
}

nlp_status nlp_energies(nlp_plan p, const void *phi_dev, const void *V_dev, double beta, double g, double *energies) {
    if (!p || !phi_dev || !V_dev || !energies) return NLP_ERR_INVALID_ARG;
    if (p->grid.dim == 1) return NLP_ERR_UNSUPPORTED;
    return energies_impl(p, phi_dev, V_dev, beta, g, energies);
}

nlp_status nlp_energies_noalloc(nlp_plan p, const void *phi_dev, const void *V_dev, double beta, double g,
                                double *energies) {
    if (!p || !phi_dev || !V_dev || !energies) return NLP_ERR_INVALID_ARG;
    if (p->kernel == NLP_POISSON_2D || p->grid.dim == 1) return NLP_ERR_UNSUPPORTED;
    return energies_noalloc_impl(p, phi_dev, V_dev, beta, g, energies);
}

nlp_status nlp_ts_step(nlp_plan p, void *psi_dev, const void *V_dev, double beta, double g, double tau, int order) {
    if (!p || !psi_dev || !V_dev || !(tau > 0) || (order != 2 && order != 4)) return NLP_ERR_INVALID_ARG;
    if (p->grid.dim == 1) return NLP_ERR_UNSUPPORTED;
    return ts_step_impl(p, psi_dev, V_dev, beta, g, tau, order);
}

nlp_status nlp_set_stage_timing(nlp_plan p, int on) {
    if (!p) return NLP_ERR_INVALID_ARG;
    if (on && !p->ev[0])
        for (int i = 0; i < 32; ++i)
            if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return NLP_ERR_CUDA;
    p->timing = on ? 1 : 0;
    p->nev = 0;
    return NLP_OK;
}

nlp_status nlp_get_stage_times(nlp_plan p, int *stage_ids, double *ms, int max, int *count) {
    if (!p || !count) return NLP_ERR_INVALID_ARG;
    *count = 0;
    if (!p->timing || p->nev < 2) return NLP_OK;
    if (cudaEventSynchronize(p->ev[p->nev - 1]) != cudaSuccess) return NLP_ERR_CUDA;
    int c = 0;
    for (int i = 1; i < p->nev && c < max; ++i, ++c) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev[i - 1], p->ev[i]) != cudaSuccess) return NLP_ERR_CUDA;
        if (ms) ms[c] = (double)t;
        if (stage_ids) stage_ids[c] = p->ev_stage[i];
    }
    *count = c;
    return NLP_OK;
}

}  // extern "C"
