// Fused interpolate -> scale -> spread for 3D with register-resident columns, and the combine
// pass that folds the chunks' windows into the spreading target.
//
// Same operation as k_interp_spread (spread.cu); different work decomposition.  Nodes of a
// tile are sorted at plan time by 2^3 sub-tile; a run of at most 64 (FP32) / 32 (FP64) nodes
// of one sub-tile is a piece, and all nodes of a piece reach the same sub-window of
// W = 2 + w - 1 cells per axis.  Two kernels:
//   - k_interp_warp then k_spread_warp (FP32, W <= 8): one warp per piece, see spread_dev.cuh.
//   - k_interp_spread_reg (FP64, and FP32 with W > 8): a team of warps owns one piece: lane
//     (cx, cy) holds the z-column of the sub-window (F in registers for FP32, read from the
//     shared window per node for FP64) and a G accumulator column in registers.  Nodes are
//     processed in batches of NB with their kernel values from the plan-time table; the
//     partial sums of the NB nodes are reduced across the team with one multi-value transpose
//     reduction (log2(32) shuffle steps for all 2 NB values together) and a short cross-warp
//     pass; scaled values come back through shared memory and spreading is W more
//     multiply-adds into the register accumulators.  Each team adds its pieces to its own
//     copy of the tile window (plain read-modify-write, pieces in sequence), and the copies
//     are summed in team order when the chunk's window is written to its scratch slot.
#include "common.cuh"
#include "launch.h"
#include "spread_common.cuh"
#include "spread_dev.cuh"

namespace nlp {

constexpr int kWarpBlock = 128;   // threads per CTA of the one-warp-per-piece kernel


template <int W> struct RegCfg {
    static constexpr int TT = ((W * W + 31) / 32) * 32;       // threads per team
    static constexpr int NT = (512 / TT) > 0 ? (512 / TT) : 1; // most teams per CTA (share the F window)
    static constexpr int TW = TT / 32;                         // warps per team
};

__device__ __forceinline__ void team_sync(int team, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(nthreads) : "memory");
}

// Shared memory of the team kernel for nt teams: F window and nt G windows (dense, as the
// scratch slot), per-team kernel values, partial sums and scaled values, then the two row
// tables of the window.
template <typename T, int W, int NB> __host__ __device__ constexpr size_t reg_win_table_offset(size_t WW, int nt) {
    return align16((size_t)(1 + nt) * WW * sizeof(cpx<T>) +
                   (size_t)nt * (NB * 3 * W + RegCfg<W>::TW * 2 * NB + 2 * NB) * sizeof(T));
}

template <typename T, int W, int NB>
__global__ void __launch_bounds__(RegCfg<W>::TT *RegCfg<W>::NT) k_interp_spread_reg(DevPlan<T> P) {
    constexpr int TT = RegCfg<W>::TT, TW = RegCfg<W>::TW;
    constexpr int V = 2 * NB;
    constexpr int SH = 5 - Log2<V>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Wt0 = P.win_n[0], Wt1 = P.win_n[1], Wt2 = P.win_n[2];
    const int WW = Wt0 * Wt1 * Wt2;
    const int nt = blockDim.x / TT;
    cpx<T> *sF = (cpx<T> *)smraw;
    const int team = threadIdx.x / TT, tl = threadIdx.x % TT;
    cpx<T> *sG = sF + (size_t)(1 + team) * WW;
    T *psi = (T *)(sF + (size_t)(1 + nt) * WW) + team * (NB * 3 * W + TW * V + V);
    T *red = psi + NB * 3 * W;
    T *cbuf = red + TW * V;
    const Chunk ch = P.rchunks[blockIdx.x];
    const int rows = Wt0 * Wt1;
    int64_t *rowoff = (int64_t *)(smraw + reg_win_table_offset<T, W, NB>(WW, nt)), *rowmir = rowoff + rows;

    window_row_table(P, ch, Wt0, Wt1, rowoff, rowmir);
    const WinCol wc = window_col(P, ch, Wt2, rows);
    __syncthreads();
    window_fill(P, wc, rowoff, rowmir, rows, Wt2, sF);
    for (int q = threadIdx.x; q < nt * WW; q += blockDim.x) sF[WW + q] = mk<T>(0, 0);
    __syncthreads();

    const bool active = tl < W * W;
    const int cx = active ? tl / W : 0, cy = active ? tl % W : 0;
    const int lane = threadIdx.x & 31, wt = tl >> 5;
    for (int sg = ch.j0 + team; sg < ch.j1; sg += nt) {
        const uint32_t so = P.seg_sub[sg];
        const int so0 = so & 0xff, so1 = (so >> 8) & 0xff, so2 = (so >> 16) & 0xff;
        const int j0 = P.seg_node[2 * sg], j1 = P.seg_node[2 * sg + 1];
        const int colbase = ((so0 + cx) * Wt1 + (so1 + cy)) * Wt2 + so2;
        // FP32 keeps the F column in registers; FP64 reads it from shared memory per node,
        // which halves the column registers so that more than one team fits on an SM
        constexpr bool kFRegs = sizeof(T) == 4;
        constexpr int WF = kFRegs ? W : 1;
        T fx[WF], fy[WF], gx[W], gy[W];
#pragma unroll
        for (int z = 0; z < W; ++z) {
            if constexpr (kFRegs) {
                const cpx<T> f = active ? sF[colbase + z] : mk<T>(0, 0);
                fx[z] = f.x;
                fy[z] = f.y;
            }
            gx[z] = (T)0;
            gy[z] = (T)0;
        }
        const cpx<T> *fcol = sF + (active ? colbase : 0);
        for (int jb = j0; jb < j1; jb += NB) {
            const int nb = min(NB, j1 - jb);
            // kernel values of the batch: a contiguous block of the plan-time table
            {
                const T *src = P.psi_tab + (int64_t)jb * 3 * W;
                for (int q = tl; q < nb * 3 * W; q += TT) psi[q] = src[q];
            }
            team_sync(team, TT);
            // interpolation partials of the NB nodes
            T v[V];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                v[2 * k] = (T)0;
                v[2 * k + 1] = (T)0;
                if (k < nb) {   // uniform across the team: empty batch slots cost nothing
                    const T *pk = psi + k * 3 * W;
                    const T wxy = pk[cx] * pk[W + cy];
                    T sx = (T)0, sy = (T)0;
                    T pzv[W];
                    load_row<T, W>(pk + 2 * W, pzv);
                    // the node's w z taps are z = 0..W-2 or 1..W-1 of the sub-window (the other
                    // cell holds an exact zero kernel value): skip it, uniformly across the team
                    auto tap = [&](int z) {
                        if constexpr (kFRegs) {
                            sx += fx[z] * pzv[z];
                            sy += fy[z] * pzv[z];
                        } else {
                            const cpx<T> f = fcol[z];
                            sx += f.x * pzv[z];
                            sy += f.y * pzv[z];
                        }
                    };
                    if (pzv[0] == (T)0) {
#pragma unroll
                        for (int z = 1; z < W; ++z) tap(z);
                    } else {
#pragma unroll
                        for (int z = 0; z < W - 1; ++z) tap(z);
                    }
                    if (active) {
                        v[2 * k] = wxy * sx;
                        v[2 * k + 1] = wxy * sy;
                    }
                }
            }
            warp_reduce_multi<T, V>(v, lane);
            if ((lane & ((1 << SH) - 1)) == 0) red[wt * V + ((lane >> SH) & (V - 1))] = v[0];
            team_sync(team, TT);
            if (tl < V) {
                T s = (T)0;
#pragma unroll
                for (int u = 0; u < TW; ++u) s += red[u * V + tl];
                const int k = tl >> 1;
                cbuf[tl] = (k < nb) ? s * P.nd[4 * ((int64_t)jb + k) + 3] : (T)0;
            }
            team_sync(team, TT);
            // spreading into the register columns
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (k < nb) {
                    const T *pk = psi + k * 3 * W;
                    const T wxy = active ? pk[cx] * pk[W + cy] : (T)0;
                    const T cr = cbuf[2 * k] * wxy, ci = cbuf[2 * k + 1] * wxy;
                    T pzv[W];
                    load_row<T, W>(pk + 2 * W, pzv);
                    if (pzv[0] == (T)0) {
#pragma unroll
                        for (int z = 1; z < W; ++z) {
                            gx[z] += cr * pzv[z];
                            gy[z] += ci * pzv[z];
                        }
                    } else {
#pragma unroll
                        for (int z = 0; z < W - 1; ++z) {
                            gx[z] += cr * pzv[z];
                            gy[z] += ci * pzv[z];
                        }
                    }
                }
            }
            team_sync(team, TT);
        }
        // this team's window: each lane owns its column; the team's pieces follow each other
        // (every batch ends with a team barrier), so plain read-modify-write is race free
        if (active) {
#pragma unroll
            for (int z = 0; z < W; ++z) {
                cpx<T> g = sG[colbase + z];
                g.x += gx[z];
                g.y += gy[z];
                sG[colbase + z] = g;
            }
        }
    }
    __syncthreads();
    cpx<T> *out = P.win + (int64_t)blockIdx.x * P.win_cells;
    for (int q = threadIdx.x; q < WW; q += blockDim.x) {
        cpx<T> s = sF[WW + q];
        for (int k = 1; k < nt; ++k) s = s + sF[(size_t)(1 + k) * WW + q];
        out[q] = s;
    }
}

#ifndef NLP_WARP_MINB
#define NLP_WARP_MINB 5
#endif
template <int W>
__global__ void __launch_bounds__(kWarpBlock, NLP_WARP_MINB) k_interp_warp(DevPlan<float> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    interp_warp_block<W, kWarpNB>(P, blockIdx.x, smraw);
}

template <int W>
__global__ void __launch_bounds__(kWarpBlock, NLP_WARP_MINB) k_spread_warp(DevPlan<float> P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    spread_warp_block<W, kWarpNB>(P, blockIdx.x, smraw);
}

template <typename T> __global__ void __launch_bounds__(256) k_window_sum(DevPlan<T> P) {
    __shared__ __align__(16) long long sb[window_sum_smem<T>() / sizeof(long long)];
    window_sum_block<T>(P, blockIdx.x, sb);
}

// 128 threads: a 3D tile (8 x 8 x 8) is 4 cells per thread, a 2D tile (1 x 8 x 16) one
template <typename T, int CPT> __global__ void __launch_bounds__(128) k_combine(DevPlan<T> P) {
    __shared__ CombStage st[kCombStage];
    combine_block<T, CPT>(P, P.cmb_act[blockIdx.x], st);
}

// supported column lengths: FP32 W = 5..11 (w = 4..10 with Ts = 2), FP64 W = 9..16 (w = 8..15)
template <typename T> bool reg_kernel_supported(int W) {
    return sizeof(T) == 8 ? (W >= 9 && W <= 16) : (W >= 5 && W <= 11);
}
template <typename T> bool warp_kernel_used(int W) { return sizeof(T) == 4 && W >= 5 && W <= 8; }

template <typename T> static constexpr int nb_of() { return sizeof(T) == 8 ? 8 : 4; }   // nodes per batch (register budget)

// teams per CTA of the team kernel: as many as fit (at most NT), each with its own window
template <typename T, int W> static int reg_teams(const DevPlan<T> &P) {
    const size_t WW = (size_t)P.win_n[0] * P.win_n[1] * P.win_n[2];
    const size_t rows = (size_t)P.win_n[0] * P.win_n[1];
    for (int nt = RegCfg<W>::NT; nt >= 1; --nt)
        if (reg_win_table_offset<T, W, nb_of<T>()>(WW, nt) + 2 * rows * sizeof(int64_t) <= (size_t)max_dyn_smem()) return nt;
    return 0;
}

template <typename T, int W> static size_t reg_smem(const DevPlan<T> &P, int nwarps_warpkernel) {
    if constexpr (sizeof(T) == 4 && W <= 8) {
        return std::max(warp_layout<W, kWarpNB>(P.win_n[0], P.win_n[1], P.win_n[2], nwarps_warpkernel, false).bytes,
                        warp_layout<W, kWarpNB>(P.win_n[0], P.win_n[1], P.win_n[2], nwarps_warpkernel, true).bytes);
    } else {
        const size_t WW = (size_t)P.win_n[0] * P.win_n[1] * P.win_n[2];
        const size_t rows = (size_t)P.win_n[0] * P.win_n[1];
        const int nt = std::max(1, reg_teams<T, W>(P));
        return reg_win_table_offset<T, W, nb_of<T>()>(WW, nt) + 2 * rows * sizeof(int64_t);
    }
}

template <typename T, int W> static cudaError_t launch_w(const DevPlan<T> &P, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && W <= 8) {
        // spreading half (the interpolation half runs first, launch_interp_warp)
        const size_t sm = warp_layout<W, kWarpNB>(P.win_n[0], P.win_n[1], P.win_n[2], kWarpBlock / 32, true).bytes;
        cudaError_t e = allow_smem<k_spread_warp<W>>();
        if (e == cudaSuccess)   // several small blocks per SM, each with its own tile window
            e = cudaFuncSetAttribute(k_spread_warp<W>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        k_spread_warp<W><<<(unsigned)P.nrchunks, kWarpBlock, sm, st>>>(P);
        return cudaGetLastError();
    } else {
        constexpr int NB = nb_of<T>();
        const int nt = reg_teams<T, W>(P);
        if (nt < 1) return cudaErrorInvalidValue;
        const size_t sm = reg_smem<T, W>(P, 0);
        cudaError_t e = allow_smem<k_interp_spread_reg<T, W, NB>>();
        if (e != cudaSuccess) return e;
        k_interp_spread_reg<T, W, NB><<<(unsigned)P.nrchunks, RegCfg<W>::TT * nt, sm, st>>>(P);
        return cudaGetLastError();
    }
}

#define NLP_REG_SWITCH(T, W, CALL)                       \
    switch (W) {                                         \
        case 5: CALL(T, 5); case 6: CALL(T, 6);          \
        case 7: CALL(T, 7); case 8: CALL(T, 8);          \
        case 9: CALL(T, 9); case 10: CALL(T, 10);        \
        case 11: CALL(T, 11); case 12: CALL(T, 12);      \
        case 13: CALL(T, 13); case 14: CALL(T, 14);      \
        case 15: CALL(T, 15); case 16: CALL(T, 16);      \
        default: break;                                  \
    }

template <> size_t interp_spread_reg_smem<float>(const DevPlan<float> &P, int nwarps) {
    const int W = P.sub_T + P.w - 1;
#define SM_F(T, X) if constexpr (X >= 5 && X <= 11) return reg_smem<T, X>(P, nwarps); break;
    NLP_REG_SWITCH(float, W, SM_F)
#undef SM_F
    return 0;
}
template <> size_t interp_spread_reg_smem<double>(const DevPlan<double> &P, int nwarps) {
    const int W = P.sub_T + P.w - 1;
#define SM_D(T, X) if constexpr (X >= 9 && X <= 16) return reg_smem<T, X>(P, nwarps); break;
    NLP_REG_SWITCH(double, W, SM_D)
#undef SM_D
    return 0;
}

template <> cudaError_t launch_interp_spread_reg<float>(const DevPlan<float> &P, cudaStream_t st) {
    if (P.nrchunks == 0) return cudaSuccess;
    const int W = P.sub_T + P.w - 1;
#define L_F(T, X) if constexpr (X >= 5 && X <= 11) return launch_w<T, X>(P, st); break;
    NLP_REG_SWITCH(float, W, L_F)
#undef L_F
    return cudaErrorInvalidValue;
}
template <> cudaError_t launch_interp_spread_reg<double>(const DevPlan<double> &P, cudaStream_t st) {
    if (P.nrchunks == 0) return cudaSuccess;
    const int W = P.sub_T + P.w - 1;
#define L_D(T, X) if constexpr (X >= 9 && X <= 16) return launch_w<T, X>(P, st); break;
    NLP_REG_SWITCH(double, W, L_D)
#undef L_D
    return cudaErrorInvalidValue;
}

template <int W> static cudaError_t launch_interp_w(const DevPlan<float> &P, cudaStream_t st) {
    const size_t sm = warp_layout<W, kWarpNB>(P.win_n[0], P.win_n[1], P.win_n[2], kWarpBlock / 32, false).bytes;
    cudaError_t e = allow_smem<k_interp_warp<W>>();
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_interp_warp<W>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    k_interp_warp<W><<<(unsigned)P.nrchunks, kWarpBlock, sm, st>>>(P);
    return cudaGetLastError();
}

template <> cudaError_t launch_interp_warp<float>(const DevPlan<float> &P, cudaStream_t st) {
    if (P.nrchunks == 0) return cudaSuccess;
    switch (P.sub_T + P.w - 1) {
        case 5: return launch_interp_w<5>(P, st);
        case 6: return launch_interp_w<6>(P, st);
        case 7: return launch_interp_w<7>(P, st);
        case 8: return launch_interp_w<8>(P, st);
        default: return cudaErrorInvalidValue;
    }
}
template <> cudaError_t launch_interp_warp<double>(const DevPlan<double> &, cudaStream_t) { return cudaErrorInvalidValue; }

template <typename T> cudaError_t launch_window_sum(const DevPlan<T> &P, cudaStream_t st) {
    if (P.ngroups == 0) return cudaSuccess;
    k_window_sum<T><<<(unsigned)(P.ngroups * P.grp_parts), 256, 0, st>>>(P);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_combine(const DevPlan<T> &P, cudaStream_t st) {
    if (P.cmb_nact == 0) return cudaSuccess;
    if (P.cmb_t[0] == 1) k_combine<T, 1><<<(unsigned)P.cmb_nact, 128, 0, st>>>(P);
    else k_combine<T, 4><<<(unsigned)P.cmb_nact, 128, 0, st>>>(P);
    return cudaGetLastError();
}

template bool reg_kernel_supported<float>(int);
template bool reg_kernel_supported<double>(int);
template bool warp_kernel_used<float>(int);
template bool warp_kernel_used<double>(int);
template cudaError_t launch_window_sum<float>(const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_window_sum<double>(const DevPlan<double> &, cudaStream_t);
template cudaError_t launch_combine<float>(const DevPlan<float> &, cudaStream_t);
template cudaError_t launch_combine<double>(const DevPlan<double> &, cudaStream_t);

}  // namespace nlp
