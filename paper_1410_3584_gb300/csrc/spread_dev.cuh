// Interpolation/spreading device code shared by the single-plan kernels (spread.cu,
// spread_reg.cu) and the batched persistent kernel (batch.cu): per-block bodies with the
// block index passed explicitly.  Each body processes one chunk and writes the chunk's tile
// window to its scratch slot (the combine pass of spread_common.cuh folds the slots into G).
#pragma once
#include "common.cuh"
#include "spread_common.cuh"

namespace nlp {

// Reduce V values across the 32 lanes of a warp (V a power of two <= 32).  Recursive
// halving: at the step with offset s each lane keeps the half of its values selected by
// its lane bit s and adds the other half received from lane ^ s.  On return v[0] of lane
// L is the warp sum of value index (L >> (5 - log2 V)) & (V - 1).
template <typename T, int V>
__device__ __forceinline__ void warp_reduce_multi(T (&v)[V], int lane) {
    int off = 16;
#pragma unroll
    for (int half = V / 2; half >= 1; half /= 2) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const T send = up ? v[i] : v[i + half];
            const T keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
        off >>= 1;
    }
    for (; off >= 1; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
}

// the W kernel values of one axis of a node, from shared memory, in 16- or 8-byte loads where
// the row is aligned for them (rows start at multiples of W elements of 16-byte aligned buffers)
template <typename T, int W> __device__ __forceinline__ void load_row(const T *p, T (&out)[W]) {
    if constexpr (sizeof(T) == 4 && W % 4 == 0) {
#pragma unroll
        for (int i = 0; i < W / 4; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(p)[i];
            out[4 * i] = v.x;
            out[4 * i + 1] = v.y;
            out[4 * i + 2] = v.z;
            out[4 * i + 3] = v.w;
        }
    } else if constexpr (sizeof(T) == 4 && W % 2 == 0) {
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const float2 v = reinterpret_cast<const float2 *>(p)[i];
            out[2 * i] = v.x;
            out[2 * i + 1] = v.y;
        }
    } else if constexpr (sizeof(T) == 8 && W % 2 == 0) {
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const double2 v = reinterpret_cast<const double2 *>(p)[i];
            out[2 * i] = v.x;
            out[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) out[i] = p[i];
    }
}

template <bool B> struct BoolC { static constexpr bool value = B; };
template <int V> struct Log2 { static constexpr int value = 1 + Log2<V / 2>::value; };
template <> struct Log2<1> { static constexpr int value = 0; };

// ======================================================================= generic kernel
// One warp per node (lanes over the taps of the last two axes, a loop over the first), for
// 2D plans and for 3D widths the register kernels do not cover.  Each warp spreads into its
// own copy of the tile window (plain read-modify-write: within a node the lanes own distinct
// cells, and a warp's nodes follow each other), and the copies are summed in warp order
// when the chunk's window is written out.
//
// Shared memory: F window, nwin warp windows, kernel values of nwin warps, row tables.
template <typename T> __host__ __device__ constexpr size_t generic_win_table_offset(size_t WW, int nwin) {
    return align16((size_t)(1 + nwin) * WW * sizeof(cpx<T>) + (size_t)nwin * 3 * kMaxWidth * sizeof(T));
}
template <typename T> __host__ __device__ constexpr size_t generic_smem_bytes(size_t WW, size_t rows, int nwin) {
    return generic_win_table_offset<T>(WW, nwin) + 2 * rows * sizeof(int64_t);
}

template <typename T>
__device__ __forceinline__ void spread_generic_block(const DevPlan<T> &P, int bid, unsigned char *smraw) {
    const int w = P.w;
    const int w0 = P.dim == 3 ? w : 1;
    const int W0 = P.win_n[0], W1 = P.win_n[1], W2 = P.win_n[2];
    const int WW = W0 * W1 * W2;
    const int nw = blockDim.x >> 5;
    cpx<T> *sF = (cpx<T> *)smraw;
    cpx<T> *sGall = sF + WW;
    T *spsi = (T *)(sGall + (size_t)nw * WW);
    const int rows = W0 * W1;
    int64_t *rowoff = (int64_t *)(smraw + generic_win_table_offset<T>(WW, nw)), *rowmir = rowoff + rows;
    const Chunk ch = P.chunks[bid];

    window_row_table(P, ch, W0, W1, rowoff, rowmir);
    const WinCol wc = window_col(P, ch, W2, rows);
    __syncthreads();
    if (!P.ones_mode) window_fill(P, wc, rowoff, rowmir, rows, W2, sF);
    for (int q = threadIdx.x; q < nw * WW; q += blockDim.x) sGall[q] = mk<T>(0, 0);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *ps = spsi + warp * 3 * kMaxWidth;
    cpx<T> *sG = sGall + (size_t)warp * WW;
    const T two_w = (T)2 / (T)w;
    const int sa = W1 * W2;
    for (int j = ch.j0 + warp; j < ch.j1; j += nw) {
        const T d0 = P.nd[4 * (int64_t)j + 0], d1 = P.nd[4 * (int64_t)j + 1];
        const T d2 = P.nd[4 * (int64_t)j + 2], om = P.nd[4 * (int64_t)j + 3];
        const uint32_t o = P.no[j];
        const int o0 = o & 0xff, o1 = (o >> 8) & 0xff, o2 = (o >> 16) & 0xff;
        for (int t = lane; t < 3 * kMaxWidth; t += 32) {
            const int ax = t / kMaxWidth, tt = t % kMaxWidth;
            T v = (T)0;
            if (ax == 0) v = (w0 == 1) ? (tt == 0 ? (T)1 : (T)0) : (tt < w ? es_kernel<T>(((T)tt - d0) * two_w, P.beta) : (T)0);
            else if (tt < w) v = P.psi_gen ? P.psi_gen[((int64_t)j * 3 + ax) * w + tt]
                                           : es_kernel<T>(((T)tt - (ax == 1 ? d1 : d2)) * two_w, P.beta);
            ps[t] = v;
        }
        __syncwarp();
        // interpolation
        cpx<T> acc = mk<T>(0, 0);
        if (!P.ones_mode)
            for (int p = lane; p < w * w; p += 32) {
                const int b = p / w, c = p % w;
                const T wbc = ps[kMaxWidth + b] * ps[2 * kMaxWidth + c];
                const cpx<T> *col = sF + (o0 * W1 + (o1 + b)) * W2 + (o2 + c);
                T sx = 0, sy = 0;
                for (int a = 0; a < w0; ++a) {
                    const T wa = ps[a];
                    const cpx<T> f = col[a * sa];
                    sx += wa * f.x;
                    sy += wa * f.y;
                }
                acc.x += wbc * sx;
                acc.y += wbc * sy;
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        cpx<T> cj;
        if (P.ones_mode) {
            cj = mk<T>(om, (T)0);
        } else if (P.pois == nullptr) {
            cj = scale(acc, om);
        } else {
            // Algorithm 1: W(k) = (rho-hat(k) - (C0 - i k.M1) e^{-sigma^2 |k|^2/2}) / |k| in FP64
            // (om already holds (2pi)^-2 w_r w_phi / |k|)
            const double kx = P.pois[3 * (int64_t)j], ky = P.pois[3 * (int64_t)j + 1], kr = P.pois[3 * (int64_t)j + 2];
            const double g = exp(-0.5 * P.sigma * P.sigma * kr * kr);
            const double re = P.hvol * (double)acc.x - P.mom[0] * g;
            const double im = P.hvol * (double)acc.y + (kx * P.mom[1] + ky * P.mom[2]) * g;
            cj = mk<T>((T)((double)om * re), (T)((double)om * im));
        }
        // spreading into this warp's window
        for (int p = lane; p < w * w; p += 32) {
            const int b = p / w, c = p % w;
            const T wbc = ps[kMaxWidth + b] * ps[2 * kMaxWidth + c];
            const cpx<T> v = scale(cj, wbc);
            cpx<T> *col = sG + (o0 * W1 + (o1 + b)) * W2 + (o2 + c);
            for (int a = 0; a < w0; ++a) {
                const T wa = ps[a];
                cpx<T> g = col[a * sa];
                g.x += v.x * wa;
                g.y += v.y * wa;
                col[a * sa] = g;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    cpx<T> *out = P.win + (int64_t)bid * P.win_cells;
    for (int q = threadIdx.x; q < WW; q += blockDim.x) {
        cpx<T> s = sGall[q];
        for (int k = 1; k < nw; ++k) s = s + sGall[(size_t)k * WW + q];
        out[q] = s;
    }
}

// ======================================================================= FP32 warp kernel
// One warp per piece (a run of at most 64 nodes of one 2^3 sub-tile, whose nodes all reach
// the same sub-window of W^3 cells, W = w + 1): lane L owns the sub-window z-columns
// a = (L mod W', L div W') and b (32 further columns), where W' = W for W^2 <= 64.  Per piece
// the lane holds both F columns and both G accumulator columns in registers; per batch of
// NB nodes it
//   1. evaluates the 3 W kernel values of each node from its position (lanes (axis, tap)),
//   2. interpolates: per column a complex z-contraction with packed FP32x2 FMAs, weighted by
//      the column's x/y kernel values, reduced over the warp for all NB nodes at once,
//   3. scales by the node weight and spreads: per column a complex x z outer product with
//      packed FMAs into the G registers.
// At the end of a piece the G columns are added to the chunk's shared window as 32-bit
// fixed-point integers: integer addition is associative, so the warps' order does not change
// the sums.  The quantum q of a chunk is a power of two chosen before any spreading from a
// bound on every cell of its window: |G| <= sum_j |c_j| (the kernel is at most 1) and
// |c_j| = |omega_j| |rho-hat_j| <= |omega_j| sqrt(2) max|F| (max_delta sum_t psi)^3, so with
// S = sum_j |omega_j| (plan time, per chunk) every partial sum of a cell stays below
// B = sqrt(2) max|F| C^3 S <= 2^30 q.
template <int W, int NB> struct WarpGeo {
    static constexpr int V = 2 * NB;
    static constexpr int SS = 32;               // floats of one node's kernel values: x[8] y[8] z pairs[16]
    static constexpr int STAGE = NB * SS + V;   // floats per warp
};

struct WarpLayout {
    int Wt0, Wt1, Wt2;
    int RP, SP;       // F window: cell (a, b, c) at a SP + b RP + c (RP even, SP / 2 odd: 16-byte column
                      // loads of the 8 lanes of a quarter warp fall in distinct bank groups)
    int RG, SG;       // G window: cell (a, b, c) at a SG + b RG + c (RG odd)
    size_t offG, offStage, offRows, bytes;
};

template <int W, int NB>
__host__ __device__ inline WarpLayout warp_layout(int Wt0, int Wt1, int Wt2, int nwarps) {
    WarpLayout L;
    L.Wt0 = Wt0;
    L.Wt1 = Wt1;
    L.Wt2 = Wt2;
    L.RP = (Wt2 + 1) & ~1;
    L.SP = Wt1 * L.RP;
    if ((L.SP / 2) % 2 == 0) L.SP += 2;
    L.RG = Wt2 | 1;
    L.SG = Wt1 * L.RG;
    L.offG = align16((size_t)Wt0 * L.SP * sizeof(float2));
    L.offStage = align16(L.offG + (size_t)Wt0 * L.SG * sizeof(int2));
    L.offRows = align16(L.offStage + (size_t)nwarps * WarpGeo<W, NB>::STAGE * sizeof(float));
    L.bytes = L.offRows + 2 * (size_t)Wt0 * Wt1 * sizeof(int64_t);
    return L;
}

// exp(beta (sqrt(1 - x^2) - 1)) for x = (i - d) 2/w with the exponent written as
// -beta x^2 / (1 + sqrt(1 - x^2)) (no cancellation near x = 0); 0 outside |x| < 1.
// nbl2 = -beta log2(e).  rsqrt / rcp / ex2 are the hardware approximations.
__device__ __forceinline__ float es_fast(float i_f, float d, float c2w, float nbl2) {
    const float x = (i_f - d) * c2w;
    const float x2 = x * x;
    const float s = 1.0f - x2;
    float rs, rd, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));
    const float den = fmaf(s, rs, 1.0f);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(den));
    const float arg = (x * (x * nbl2)) * rd;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(arg));
    return s > 0.0f ? e : 0.0f;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int W, int NB>
__device__ __forceinline__ void spread_warp_block(const DevPlan<float> &P, int bid, unsigned char *smraw) {
    static_assert(W * W <= 64 && W >= 4 && W <= 8, "two columns per lane, at most 8 z taps");
    using G = WarpGeo<W, NB>;
    constexpr int V = G::V;
    constexpr int SH = 5 - Log2<V>::value;
    const int w = P.w;
    const int nwarps = blockDim.x >> 5;
    const WarpLayout L = warp_layout<W, NB>(P.win_n[0], P.win_n[1], P.win_n[2], nwarps);
    cpx<float> *sF = (cpx<float> *)smraw;
    int2 *sG = (int2 *)(smraw + L.offG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *stage = (float *)(smraw + L.offStage) + warp * G::STAGE;
    float *cb = stage + NB * G::SS;
    const int rows = L.Wt0 * L.Wt1;
    int64_t *rowoff = (int64_t *)(smraw + L.offRows), *rowmir = rowoff + rows;
    const Chunk ch = P.rchunks[bid];
    __shared__ int s_next, s_max;
    if (threadIdx.x == 0) {
        s_next = ch.j0 + nwarps;
        s_max = 0;
    }
    window_row_table(P, ch, L.Wt0, L.Wt1, rowoff, rowmir);
    const WinCol wc = window_col(P, ch, L.Wt2, rows);
    __syncthreads();
    float mx = 0.0f;
    if (!P.ones_mode) mx = window_fill(P, wc, rowoff, rowmir, rows, L.RP, sF, L.Wt1, L.SP);
    for (int q = threadIdx.x; q < L.Wt0 * L.SG; q += blockDim.x) sG[q] = make_int2(0, 0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) atomicMax(&s_max, __float_as_int(mx));   // non-negative floats order as integers
    __syncthreads();
    // fixed-point quantum of this chunk (a power of two, so that int * q is exact)
    float B = P.ones_mode ? ch.wsum : 1.41421356f * __int_as_float(s_max) * P.psi_sum3 * ch.wsum;
    B *= 1.01f;
    int ex = 0;
    if (B > 0.0f && B <= 3.0e38f) frexpf(B, &ex);   // B < 2^ex
    ex = max(ex, -96);
    const float qinv = ldexpf(1.0f, 30 - ex);
    const float qf = (B == B) ? ldexpf(1.0f, ex - 30) : B;   // a NaN input stays NaN in the window

    const int ca = lane, cbc = lane + 32;
    const bool act_a = (W * W >= 32) || ca < W * W;
    const bool act_b = (W * W == 64) || cbc < W * W;
    const int xa = act_a ? ca % W : 0, ya = act_a ? ca / W : 0;
    const int xb = act_b ? cbc % W : 0, yb = act_b ? cbc / W : 0;
    // kernel-value lanes: lane = axis * 8 + tap for lanes < 24
    const int kv_ax = lane >> 3, kv_i = lane & 7;
    const bool kv_on = lane < 24 && kv_i < W;
    const float kv_if = (float)kv_i;
    const float c2w = 2.0f / (float)w, nbl2 = -(float)P.beta * 1.44269504f;
    const int kv_st = kv_ax == 2 ? 16 + 2 * kv_i : kv_ax * 8 + kv_i;
    // G flush order: lanes of the upper half of each y quartet add the imaginary word first,
    // so that the 32 lanes of one atomic instruction hit 32 banks (W = 8 geometry)
    const int sw = (ya >> 1) & 1;
    // node records of a batch: per kernel-value lane, the node's offset from its sub-window
    // origin along the lane's axis (for plans of this kernel the node records hold that
    // offset, see plan.cu) for each node; per lane k < NB the node weight
    float pd[NB], wf;
    auto fetch = [&](int jbn, int nbn) {
#pragma unroll
        for (int k = 0; k < NB; ++k)
            pd[k] = (kv_on && k < nbn) ? __ldg(P.nd + 4 * ((int64_t)jbn + k) + kv_ax) : 0.0f;
        wf = (lane < nbn) ? __ldg(P.nd + 4 * ((int64_t)jbn + lane) + 3) : 0.0f;
    };
    int sg = ch.j0 + warp;
    uint32_t so = 0;
    int j0 = 0, j1 = 0;
    if (sg < ch.j1) {
        so = P.seg_sub[sg];
        j0 = P.seg_node[2 * sg];
        j1 = P.seg_node[2 * sg + 1];
        fetch(j0, min(NB, j1 - j0));
    }
    while (sg < ch.j1) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&s_next, 1);
        const int sg_n = __shfl_sync(0xffffffffu, nxt, 0);
        uint32_t so_n = 0;
        int j0_n = 0, j1_n = 0;
        if (sg_n < ch.j1) {
            so_n = P.seg_sub[sg_n];
            j0_n = P.seg_node[2 * sg_n];
            j1_n = P.seg_node[2 * sg_n + 1];
        }
        const int so0 = so & 0xff, so1 = (so >> 8) & 0xff, so2 = (so >> 16) & 0xff;
        const int fa0 = (so0 + xa) * L.SP + (so1 + ya) * L.RP + so2;
        const int fb0 = (so0 + xb) * L.SP + (so1 + yb) * L.RP + so2;
        const int ga0 = (so0 + xa) * L.SG + (so1 + ya) * L.RG + so2;
        const int gb0 = (so0 + xb) * L.SG + (so1 + yb) * L.RG + so2;
        float2 fa[W], fb[W], ga[W], gb[W];
        // F columns of the piece (16-byte loads: column starts are even cells of an even pitch)
#pragma unroll
        for (int z = 0; z + 1 < W; z += 2) {
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
            if (!P.ones_mode) {
                if (act_a) u = *reinterpret_cast<const float4 *>(sF + fa0 + z);
                if (act_b) v = *reinterpret_cast<const float4 *>(sF + fb0 + z);
            }
            fa[z] = f2(u.x, u.y);
            fa[z + 1] = f2(u.z, u.w);
            fb[z] = f2(v.x, v.y);
            fb[z + 1] = f2(v.z, v.w);
        }
        if constexpr (W % 2) {
            const cpx<float> u = (!P.ones_mode && act_a) ? sF[fa0 + W - 1] : mk<float>(0.f, 0.f);
            const cpx<float> v = (!P.ones_mode && act_b) ? sF[fb0 + W - 1] : mk<float>(0.f, 0.f);
            fa[W - 1] = f2(u.x, u.y);
            fb[W - 1] = f2(v.x, v.y);
        }
#pragma unroll
        for (int z = 0; z < W; ++z) ga[z] = gb[z] = f2(0.f, 0.f);

        auto batch = [&](auto full_tag, int nb, float wcur) {
            constexpr bool FULL = decltype(full_tag)::value;
            float v[V], wa[NB], wb[NB];
            // interpolation partials
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                v[2 * k] = v[2 * k + 1] = 0.f;
                wa[k] = wb[k] = 0.f;
                if (FULL || k < nb) {
                    const float *pk = stage + k * G::SS;
                    const float px = pk[xa];
                    wa[k] = act_a ? px * pk[8 + ya] : 0.f;
                    wb[k] = act_b ? (W == 8 ? px : pk[xb]) * pk[8 + yb] : 0.f;
                    if (!P.ones_mode) {
                        float2 sa = f2(0.f, 0.f), sb = f2(0.f, 0.f);
#pragma unroll
                        for (int z = 0; z + 1 < W; z += 2) {
                            const float4 pz = *reinterpret_cast<const float4 *>(pk + 16 + 2 * z);
                            sa = __ffma2_rn(fa[z], f2(pz.x, pz.y), sa);
                            sb = __ffma2_rn(fb[z], f2(pz.x, pz.y), sb);
                            sa = __ffma2_rn(fa[z + 1], f2(pz.z, pz.w), sa);
                            sb = __ffma2_rn(fb[z + 1], f2(pz.z, pz.w), sb);
                        }
                        if constexpr (W % 2) {
                            const float2 pz = *reinterpret_cast<const float2 *>(pk + 16 + 2 * (W - 1));
                            sa = __ffma2_rn(fa[W - 1], pz, sa);
                            sb = __ffma2_rn(fb[W - 1], pz, sb);
                        }
                        v[2 * k] = wa[k] * sa.x + wb[k] * sb.x;
                        v[2 * k + 1] = wa[k] * sa.y + wb[k] * sb.y;
                    }
                }
            }
            if (!P.ones_mode) warp_reduce_multi<float, V>(v, lane);
            {
                const int idx = (lane >> SH) & (V - 1);
                const int k = idx >> 1;
                const float wk = __shfl_sync(0xffffffffu, wcur, k);   // weight of node k of the batch
                if ((lane & ((1 << SH) - 1)) == 0) {
                    float c = P.ones_mode ? ((idx & 1) ? 0.f : wk) : v[0] * wk;
                    cb[idx] = (FULL || k < nb) ? c : 0.f;
                }
            }
            __syncwarp();
            // spreading into the register columns
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (FULL || k < nb) {
                    const float *pk = stage + k * G::SS;
                    const float2 c = *reinterpret_cast<const float2 *>(cb + 2 * k);
                    const float2 ca2 = f2(c.x * wa[k], c.y * wa[k]), cb2 = f2(c.x * wb[k], c.y * wb[k]);
#pragma unroll
                    for (int z = 0; z + 1 < W; z += 2) {
                        const float4 pz = *reinterpret_cast<const float4 *>(pk + 16 + 2 * z);
                        ga[z] = __ffma2_rn(ca2, f2(pz.x, pz.y), ga[z]);
                        gb[z] = __ffma2_rn(cb2, f2(pz.x, pz.y), gb[z]);
                        ga[z + 1] = __ffma2_rn(ca2, f2(pz.z, pz.w), ga[z + 1]);
                        gb[z + 1] = __ffma2_rn(cb2, f2(pz.z, pz.w), gb[z + 1]);
                    }
                    if constexpr (W % 2) {
                        const float2 pz = *reinterpret_cast<const float2 *>(pk + 16 + 2 * (W - 1));
                        ga[W - 1] = __ffma2_rn(ca2, pz, ga[W - 1]);
                        gb[W - 1] = __ffma2_rn(cb2, pz, gb[W - 1]);
                    }
                }
            }
        };
        for (int jb = j0; jb < j1; jb += NB) {
            const int nb = min(NB, j1 - jb);
            // kernel values of the batch from the fetched node offsets
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (kv_on) {
                    const float e = (k < nb) ? es_fast(kv_if, pd[k], c2w, nbl2) : 0.f;
                    if (kv_ax == 2) *reinterpret_cast<float2 *>(stage + k * G::SS + kv_st) = f2(e, e);
                    else stage[k * G::SS + kv_st] = e;
                }
            }
            const float wcur = wf;
            __syncwarp();
            if (jb + NB < j1)
                fetch(jb + NB, min(NB, j1 - jb - NB));
            else if (sg_n < ch.j1)
                fetch(j0_n, min(NB, j1_n - j0_n));
            if (nb == NB)
                batch(BoolC<true>{}, nb, wcur);
            else
                batch(BoolC<false>{}, nb, wcur);
            __syncwarp();
        }
        // add the piece's columns to the window in fixed point
#pragma unroll
        for (int z = 0; z < W; ++z) {
            if (act_a) {
                int *c = &sG[ga0 + z].x;
                const int re = __float2int_rn(ga[z].x * qinv), im = __float2int_rn(ga[z].y * qinv);
                atomicAdd(c + sw, sw ? im : re);
                atomicAdd(c + (sw ^ 1), sw ? re : im);
            }
            if (act_b) {
                int *c = &sG[gb0 + z].x;
                const int re = __float2int_rn(gb[z].x * qinv), im = __float2int_rn(gb[z].y * qinv);
                atomicAdd(c + sw, sw ? im : re);
                atomicAdd(c + (sw ^ 1), sw ? re : im);
            }
        }
        sg = sg_n;
        so = so_n;
        j0 = j0_n;
        j1 = j1_n;
    }
    __syncthreads();
    // the chunk's window, dense, to its scratch slot
    cpx<float> *out = P.win + (int64_t)bid * P.win_cells;
    const int WW = L.Wt0 * L.Wt1 * L.Wt2;
    for (int q = threadIdx.x; q < WW; q += blockDim.x) {
        const int c = q % L.Wt2, r = q / L.Wt2;
        const int b = r % L.Wt1, a = r / L.Wt1;
        const int2 g = sG[a * L.SG + b * L.RG + c];
        out[q] = mk<float>((float)g.x * qf, (float)g.y * qf);
    }
}

}  // namespace nlp
