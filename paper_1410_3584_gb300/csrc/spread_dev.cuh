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

// ======================================================================= FP32 warp kernels
// Interpolation and spreading run as two kernels over the same chunks and pieces (a piece: a
// run of at most 64 nodes of one 2^3 sub-tile, whose nodes all reach the same sub-window of
// W^3 cells, W = w + 1), one warp per piece; lane L owns the sub-window z-columns
// a = (L mod W, L div W) and b = a + 32 (in column order).  Holding only F (interpolation) or
// only G (spreading) in registers keeps each kernel's register and shared-memory footprint
// at half of a fused one, for more resident warps.  Per batch of NB nodes a warp
//   1. evaluates the 3 W kernel values of each node from its position (the 3 W NB values
//      spread evenly over the lanes) into a per-warp stage, each value stored twice so that
//      (v, v) pairs load as packed operands,
//   2. (interpolation) per column a complex z-contraction with packed FP32x2 FMAs, the
//      batch's nodes interleaved, weighted by the column's x/y kernel values; the 32 lane
//      partials of the batch's 2 NB sums are reduced together by a shuffle tree in a fixed
//      order, one batch behind (the shuffles of batch i run while batch i + 1 computes);
//      c_j = rho-hat_j omega_j goes to the node array and |c_j| into the chunk's bound,
//   2'. (spreading) per column a complex x z outer product of c_j with packed FMAs into the G
//      registers; at the end of a piece the columns are added to the chunk's shared window
//      in fixed point, and the window goes to the chunk's scratch slot.
// A piece's last batch is padded with the records that follow it, given weight zero, so every
// batch runs the same code.
//
// Fixed point (spreading).  The warps of a CTA add their pieces' columns into the chunk's
// shared window concurrently; integer addition is associative, so the window does not depend
// on their order.  The quantum is a power of two (int * q is exact) chosen from a bound known
// before the sums: every cell obeys |re G|, |im G| <= sum_j (|re c_j| + |im c_j|) =: B2 (the
// kernel is at most 1), summed by the interpolation kernel in a fixed order, and
// q2 = 2^(ceil log2 1.01 B2 - 30), so all partial sums stay below 2^31 in magnitude.
#ifndef NLP_WARP_NB
#define NLP_WARP_NB 4
#endif
constexpr int kWarpNB = NLP_WARP_NB;   // nodes per batch of the FP32 warp kernels

template <int W, int NB> struct WarpGeo {
    static constexpr int SS = 48;               // floats per node: x, y, z kernel values, each as (v, v)
    static constexpr int STAGE = NB * SS;       // floats per warp
    static constexpr int KV = 3 * 8 * NB;       // kernel values per batch (8 taps per axis)
    static constexpr int KR = (KV + 31) / 32;   // evaluation rounds per lane
};

// Shared memory of the two kernels.  F window cell (a, b, c) at a SP + b RP + c (RP even,
// SP / 2 odd: 16-byte column loads of the 8 lanes of a quarter warp fall in distinct bank
// groups); G window cell (a, b, c) at a SG + b RG + c (RG odd).
struct WarpLayout {
    int Wt0, Wt1, Wt2;
    int RP, SP, RG, SG;
    size_t offStage, offRec, offRows, offRowW, bytes;
};
// per warp: node records (and, spreading, c_j) of two pieces, staged one piece ahead
constexpr int kRecNodes = 64 + 8;   // a piece (<= 64 nodes) and the padding its last batch reads

template <int W, int NB>
__host__ __device__ inline WarpLayout warp_layout(int Wt0, int Wt1, int Wt2, int nwarps, bool spreading) {
    WarpLayout L;
    L.Wt0 = Wt0;
    L.Wt1 = Wt1;
    L.Wt2 = Wt2;
    L.RP = (Wt2 + 1) & ~1;
    L.SP = Wt1 * L.RP;
    if ((L.SP / 2) % 2 == 0) L.SP += 2;
    L.RG = Wt2 | 1;
    L.SG = Wt1 * L.RG;
    const size_t rows = (size_t)Wt0 * Wt1;
    const size_t win = spreading ? (size_t)Wt0 * L.SG * sizeof(int2) : (size_t)Wt0 * L.SP * sizeof(float2);
    L.offStage = align16(win);
    L.offRec = align16(L.offStage + (size_t)nwarps * WarpGeo<W, NB>::STAGE * sizeof(float));
    const size_t rec = (size_t)kRecNodes * (spreading ? sizeof(float4) + sizeof(float2) : sizeof(float4));
    L.offRows = align16(L.offRec + (size_t)nwarps * 2 * rec);
    L.offRowW = L.offRows + (spreading ? 0 : 2 * rows * sizeof(int64_t));
    L.bytes = L.offRowW + rows * sizeof(int) + 32 * sizeof(float);
    return L;
}

// exp(beta (sqrt(1 - x^2) - 1)) for x = (i - d) 2/w with the exponent written as
// -beta x^2 / (1 + sqrt(1 - x^2)) (no cancellation near x = 0); 0 outside |x| < 1.
// nbl2 = -beta log2(e).  rsqrt / rcp / ex2 are the hardware approximations.
__device__ __forceinline__ float es_fast(float i_f, float d, float c2w, float nbl2) {
    const float x = (i_f - d) * c2w;
    const float s = fmaf(-x, x, 1.0f);
    float rs, rd, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(s));
    const float den = fmaf(s, rs, 1.0f);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(den));
    const float arg = (x * (x * nbl2)) * rd;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(arg));
    return s > 0.0f ? e : 0.0f;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// es_fast for two values at once: the same operations, the FP32 ones as packed FP32x2 (each
// lane of a packed operation rounds as the scalar one), the approximations per value.
__device__ __forceinline__ float2 es_fast2(float2 i_f, float2 d, float c2w, float nbl2) {
    const float2 x = __fmul2_rn(__fadd2_rn(i_f, f2(-d.x, -d.y)), f2(c2w, c2w));
    const float2 s = __ffma2_rn(f2(-x.x, -x.y), x, f2(1.0f, 1.0f));
    float2 rs, rd, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.x) : "f"(s.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.y) : "f"(s.y));
    const float2 den = __ffma2_rn(s, rs, f2(1.0f, 1.0f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd.y) : "f"(den.y));
    const float2 arg = __fmul2_rn(__fmul2_rn(x, __fmul2_rn(x, f2(nbl2, nbl2))), rd);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(arg.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(arg.y));
    return f2(s.x > 0.0f ? e.x : 0.0f, s.y > 0.0f ? e.y : 0.0f);
}

// power-of-two quantum q = 2^(e - 30) for a bound B (1.01 B < 2^e); 2^-126 floor; NaN bound -> NaN
__device__ __forceinline__ void fixed_quantum(float B, float &q, float &qinv) {
    B *= 1.01f;
    int ex = 0;
    if (B > 0.0f && B <= 3.0e38f) frexpf(B, &ex);
    ex = max(ex, -96);
    qinv = ldexpf(1.0f, 30 - ex);
    q = (B == B) ? ldexpf(1.0f, ex - 30) : B;
}

__device__ __forceinline__ void cp_async(void *dst, const void *src, int bytes16or8) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes16or8 == 16) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage the records (and c_j) of the nodes [j0, j0 + n + NB) of a piece into a warp's buffer.
template <int NB>
__device__ __forceinline__ void stage_piece(const DevPlan<float> &P, int j0, int n, float4 *rec, float2 *cbuf,
                                            int lane) {
    const int m = min(n + NB, kRecNodes);
    for (int i = lane; i < m; i += 32) {
        cp_async(rec + i, P.nd + 4 * ((int64_t)j0 + i), 16);
        if (cbuf) cp_async(cbuf + i, P.cnode + j0 + i, 8);
    }
    cp_async_commit();
}

// Per-lane set-up shared by both warp kernels: column ownership and the kernel-value rounds.
template <int W, int NB> struct WarpLane {
    static constexpr int KR = WarpGeo<W, NB>::KR;
    bool act_a, act_b;
    int xa, ya, xb, yb;
    int kv_fo[KR], kv_st[KR];   // per round: record offset (4 node + axis) and stage offset
    float kv_t[KR];             // per round: tap index
    float c2w, nbl2;
    __device__ __forceinline__ WarpLane(int lane, int w, float beta) {
        const int ca = lane, cbc = lane + 32;
        act_a = (W * W >= 32) || ca < W * W;
        act_b = (W * W == 64) || cbc < W * W;
        xa = act_a ? ca % W : 0;
        ya = act_a ? ca / W : 0;
        xb = act_b ? cbc % W : 0;
        yb = act_b ? cbc / W : 0;
        // round u evaluates value q = lane + 32 u of the batch (node q / 24, axis (q mod 24) / 8,
        // tap q mod 8); rounds past the batch's values repeat the last one
#pragma unroll
        for (int u = 0; u < KR; ++u) {
            const int q = min(lane + 32 * u, WarpGeo<W, NB>::KV - 1);
            const int k = q / 24, v = q - 24 * (q / 24);
            kv_fo[u] = 4 * k + (v >> 3);
            kv_st[u] = k * WarpGeo<W, NB>::SS + 2 * v;
            kv_t[u] = (float)(v & 7);
        }
        c2w = 2.0f / (float)w;
        nbl2 = -beta * 1.44269504f;
    }
    // node offsets of the batch starting at staged record b (the records hold each node's
    // offset from its sub-window origin)
    __device__ __forceinline__ void fetch(const float *rec, int b, float (&pd)[KR]) const {
        const float *base = rec + 4 * b;
#pragma unroll
        for (int u = 0; u < KR; ++u) pd[u] = base[kv_fo[u]];
    }
    __device__ __forceinline__ void evaluate(const float (&pd)[KR], float *stage) const {
        // rounds in pairs (packed arithmetic), an odd last round alone
#pragma unroll
        for (int u = 0; u + 1 < KR; u += 2) {
            const float2 e = es_fast2(f2(kv_t[u], kv_t[u + 1]), f2(pd[u], pd[u + 1]), c2w, nbl2);
            *reinterpret_cast<float2 *>(stage + kv_st[u]) = f2(e.x, e.x);
            *reinterpret_cast<float2 *>(stage + kv_st[u + 1]) = f2(e.y, e.y);
        }
        if constexpr (KR % 2) {
            const float e = es_fast(kv_t[KR - 1], pd[KR - 1], c2w, nbl2);
            *reinterpret_cast<float2 *>(stage + kv_st[KR - 1]) = f2(e, e);
        }
    }
    // x/y weights (w, w) of the lane's two columns for node k of the stage
    __device__ __forceinline__ void weights(const float *pk, float2 &wa2, float2 &wb2) const {
        const float2 px = *reinterpret_cast<const float2 *>(pk + 2 * xa);
        wa2 = __fmul2_rn(px, *reinterpret_cast<const float2 *>(pk + 16 + 2 * ya));
        wb2 = __fmul2_rn(W == 8 ? px : *reinterpret_cast<const float2 *>(pk + 2 * xb),
                         *reinterpret_cast<const float2 *>(pk + 16 + 2 * yb));
        if (!act_a) wa2 = f2(0.f, 0.f);
        if (!act_b) wb2 = f2(0.f, 0.f);
    }
};

// the chunk window's rows: offsets in the half spectrum (line and mirror) and in the window
template <typename T>
__device__ __forceinline__ void warp_window_rows(const DevPlan<T> &P, const Chunk &ch, const WarpLayout &L,
                                                 bool spreading, int64_t *rowoff, int *rowW) {
    const int rows = L.Wt0 * L.Wt1;
    if (!spreading) window_row_table(P, ch, L.Wt0, L.Wt1, rowoff, rowoff + rows);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int a = r / L.Wt1, b = r - a * L.Wt1;
        rowW[r] = spreading ? a * L.SG + b * L.RG : a * L.SP + b * L.RP;
    }
}

// The lane partials of one batch's 2 NB sums (node k: real part v[2k], imaginary v[2k + 1]),
// waiting for their reduction; jb < 0: none.
template <int NB> struct PendingSums {
    static constexpr int V = 2 * NB;
    static_assert(V == 8, "lane layout of the batch sums");
    float v[V];
    int jb = -1, nb = 0;
    float w = 0.0f;   // lane k < NB: omega of node k (zero past the piece)
    __device__ __forceinline__ PendingSums() {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = 0.0f;
    }
    // all 2 NB sums reduced together (recursive halving, fixed shuffle order): the real part of
    // node k lands in lanes 8k .. 8k+3, its imaginary part in 8k+4 .. 8k+7; lane 8k stores
    // c_k = rho-hat_k omega_k and adds |c_k| to the bound.  Every lane must call it.
    __device__ __forceinline__ void emit(const DevPlan<float> &P, int lane, float &bsum) {
        float r[V];
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = v[i];
        warp_reduce_multi<float, V>(r, lane);
        const float im = __shfl_down_sync(0xffffffffu, r[0], 4);
        const int k = lane >> 3;
        const float wk = __shfl_sync(0xffffffffu, w, k);
        if ((lane & 7) == 0 && jb >= 0) {
            const float2 c = f2(r[0] * wk, im * wk);
            if (k < nb) P.cnode[jb + k] = mk<float>(c.x, c.y);
            bsum += fabsf(c.x) + fabsf(c.y);
        }
        jb = -1;
    }
};

template <int W, int NB>
__device__ __forceinline__ void interp_warp_block(const DevPlan<float> &P, int bid, unsigned char *smraw) {
    static_assert(W * W <= 64 && W >= 4 && W <= 8, "two columns per lane, at most 8 z taps");
    using G = WarpGeo<W, NB>;
    constexpr int SS = G::SS, KR = G::KR;
    const int nwarps = blockDim.x >> 5;
    const WarpLayout L = warp_layout<W, NB>(P.win_n[0], P.win_n[1], P.win_n[2], nwarps, false);
    cpx<float> *sF = (cpx<float> *)smraw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *stage = (float *)(smraw + L.offStage) + warp * G::STAGE;
    const int rows = L.Wt0 * L.Wt1;
    int64_t *rowoff = (int64_t *)(smraw + L.offRows), *rowmir = rowoff + rows;
    int *rowF = (int *)(smraw + L.offRowW);
    float *wsum = (float *)(rowF + rows);
    const Chunk ch = P.rchunks[bid];
    warp_window_rows(P, ch, L, false, rowoff, rowF);
    const WinCol wc = window_col(P, ch, L.Wt2, rows);
    __syncthreads();
    {
        // four loads in flight per thread before their stores
        const int N2 = P.nf[2];
        const int64_t *rt = wc.herm ? rowmir : rowoff;
        const int col = wc.herm ? N2 - wc.l2 : wc.l2;
        for (int r = wc.r0; r < rows; r += 4 * wc.rstep) {
            cpx<float> v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ru = r + u * wc.rstep;
                v[u] = ru < rows ? P.F[rt[ru] + col] : mk<float>(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int ru = r + u * wc.rstep;
                if (ru < rows) sF[rowF[ru] + wc.c] = wc.herm ? conj(v[u]) : v[u];
            }
        }
    }
    __syncthreads();

    const WarpLane<W, NB> ln(lane, P.w, (float)P.beta);
    float4 *recb = (float4 *)(smraw + L.offRec) + warp * 2 * kRecNodes;   // two piece buffers
    float pd[KR];
    float bsum = 0.0f;   // lanes 8k: sum of |re c| + |im c| of the warp's k-th batch nodes
    PendingSums<NB> pend;
    int sg = ch.j0 + warp, buf = 0;
    uint32_t so = 0;
    int j0 = 0, j1 = 0;
    if (sg < ch.j1) {
        so = P.seg_sub[sg];
        j0 = P.seg_node[2 * sg];
        j1 = P.seg_node[2 * sg + 1];
        stage_piece<NB>(P, j0, j1 - j0, recb, nullptr, lane);
    }
    while (sg < ch.j1) {
        // pieces are sorted heaviest first: warps take them round-robin; the next piece's
        // records are staged while this one computes
        const int sg_n = sg + nwarps;
        uint32_t so_n = 0;
        int j0_n = 0, j1_n = 0;
        if (sg_n < ch.j1) {
            so_n = P.seg_sub[sg_n];
            j0_n = P.seg_node[2 * sg_n];
            j1_n = P.seg_node[2 * sg_n + 1];
            stage_piece<NB>(P, j0_n, j1_n - j0_n, recb + (buf ^ 1) * kRecNodes, nullptr, lane);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        __syncwarp();
        const float *rec = (const float *)(recb + buf * kRecNodes);
        const int so0 = so & 0xff, so1 = (so >> 8) & 0xff, so2 = (so >> 16) & 0xff;
        const int fa0 = (so0 + ln.xa) * L.SP + (so1 + ln.ya) * L.RP + so2;
        const int fb0 = (so0 + ln.xb) * L.SP + (so1 + ln.yb) * L.RP + so2;
        float2 fa[W], fb[W];
        // F columns of the piece (16-byte loads: column starts are even cells of an even pitch)
#pragma unroll
        for (int z = 0; z + 1 < W; z += 2) {
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
            if (ln.act_a) u = *reinterpret_cast<const float4 *>(sF + fa0 + z);
            if (ln.act_b) v = *reinterpret_cast<const float4 *>(sF + fb0 + z);
            fa[z] = f2(u.x, u.y);
            fa[z + 1] = f2(u.z, u.w);
            fb[z] = f2(v.x, v.y);
            fb[z + 1] = f2(v.z, v.w);
        }
        if constexpr (W % 2) {
            const cpx<float> u = ln.act_a ? sF[fa0 + W - 1] : mk<float>(0.f, 0.f);
            const cpx<float> v = ln.act_b ? sF[fb0 + W - 1] : mk<float>(0.f, 0.f);
            fa[W - 1] = f2(u.x, u.y);
            fb[W - 1] = f2(v.x, v.y);
        }
        for (int jb = j0; jb < j1; jb += NB) {
            const int nb = min(NB, j1 - jb), b = jb - j0;
            ln.fetch(rec, b, pd);
            const float wcur = lane < nb ? rec[4 * (b + lane) + 3] : 0.0f;   // omega, zero past the piece
            ln.evaluate(pd, stage);
            __syncwarp();
            // the previous batch's sums: their shuffle tree is independent of this batch's
            // arithmetic below, so the two interleave
            pend.emit(P, lane, bsum);
            // the z sums of the batch's nodes interleaved (z pairs outer, nodes inner)
            float2 sa[NB], sb[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) sa[k] = sb[k] = f2(0.f, 0.f);
#pragma unroll
            for (int z = 0; z + 1 < W; z += 2) {
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const float4 pz = *reinterpret_cast<const float4 *>(stage + k * SS + 32 + 2 * z);
                    sa[k] = __ffma2_rn(fa[z], f2(pz.x, pz.y), sa[k]);
                    sb[k] = __ffma2_rn(fb[z], f2(pz.x, pz.y), sb[k]);
                    sa[k] = __ffma2_rn(fa[z + 1], f2(pz.z, pz.w), sa[k]);
                    sb[k] = __ffma2_rn(fb[z + 1], f2(pz.z, pz.w), sb[k]);
                }
            }
            if constexpr (W % 2) {
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const float2 pz = *reinterpret_cast<const float2 *>(stage + k * SS + 32 + 2 * (W - 1));
                    sa[k] = __ffma2_rn(fa[W - 1], pz, sa[k]);
                    sb[k] = __ffma2_rn(fb[W - 1], pz, sb[k]);
                }
            }
            // weighted by the columns' x/y kernel values: this batch becomes the pending one
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                float2 wa2, wb2;
                ln.weights(stage + k * SS, wa2, wb2);
                const float2 vk = __ffma2_rn(sb[k], wb2, __fmul2_rn(sa[k], wa2));
                pend.v[2 * k] = vk.x;
                pend.v[2 * k + 1] = vk.y;
            }
            pend.jb = jb;
            pend.nb = nb;
            pend.w = wcur;
            __syncwarp();
        }
        buf ^= 1;
        sg = sg_n;
        so = so_n;
        j0 = j0_n;
        j1 = j1_n;
    }
    cp_async_wait<0>();
    pend.emit(P, lane, bsum);
    // the chunk's bound for the spreading kernel: lane sums, then warps, in fixed order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, off);
    if (lane == 0) wsum[warp] = bsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int u = 0; u < nwarps; ++u) t += wsum[u];
        P.csum[bid] = t;
    }
}

template <int W, int NB>
__device__ __forceinline__ void spread_warp_block(const DevPlan<float> &P, int bid, unsigned char *smraw) {
    static_assert(W * W <= 64 && W >= 4 && W <= 8, "two columns per lane, at most 8 z taps");
    using G = WarpGeo<W, NB>;
    constexpr int SS = G::SS, KR = G::KR;
    const int nwarps = blockDim.x >> 5;
    const WarpLayout L = warp_layout<W, NB>(P.win_n[0], P.win_n[1], P.win_n[2], nwarps, true);
    int2 *sG = (int2 *)smraw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *stage = (float *)(smraw + L.offStage) + warp * G::STAGE;
    const int rows = L.Wt0 * L.Wt1;
    int *rowG = (int *)(smraw + L.offRowW);
    const Chunk ch = P.rchunks[bid];
    warp_window_rows(P, ch, L, true, nullptr, rowG);
    for (int q = threadIdx.x; q < L.Wt0 * L.SG; q += blockDim.x) sG[q] = make_int2(0, 0);
    const WinCol wc = window_col(P, ch, L.Wt2, rows);
    __syncthreads();
    float q2, q2inv;
    fixed_quantum(P.ones_mode ? ch.wsum : P.csum[bid], q2, q2inv);

    const WarpLane<W, NB> ln(lane, P.w, (float)P.beta);
    // G flush order: lanes of the upper half of each y quartet add the imaginary word first,
    // so that the 32 lanes of one atomic instruction hit 32 banks (W = 8 geometry)
    const int sw = (ln.ya >> 1) & 1;
    // this warp's region: two piece buffers of records, then their c_j
    float4 *recb = (float4 *)(smraw + L.offRec + (size_t)warp * 2 * kRecNodes * (sizeof(float4) + sizeof(float2)));
    float2 *cbb = (float2 *)(recb + 2 * kRecNodes);
    float pd[KR];
    int sg = ch.j0 + warp, buf = 0;
    uint32_t so = 0;
    int j0 = 0, j1 = 0;
    if (sg < ch.j1) {
        so = P.seg_sub[sg];
        j0 = P.seg_node[2 * sg];
        j1 = P.seg_node[2 * sg + 1];
        stage_piece<NB>(P, j0, j1 - j0, recb, P.ones_mode ? nullptr : cbb, lane);
    }
    while (sg < ch.j1) {
        const int sg_n = sg + nwarps;
        uint32_t so_n = 0;
        int j0_n = 0, j1_n = 0;
        if (sg_n < ch.j1) {
            so_n = P.seg_sub[sg_n];
            j0_n = P.seg_node[2 * sg_n];
            j1_n = P.seg_node[2 * sg_n + 1];
            stage_piece<NB>(P, j0_n, j1_n - j0_n, recb + (buf ^ 1) * kRecNodes,
                            P.ones_mode ? nullptr : cbb + (buf ^ 1) * kRecNodes, lane);
        } else {
            cp_async_commit();
        }
        cp_async_wait<1>();
        __syncwarp();
        const float *rec = (const float *)(recb + buf * kRecNodes);
        const float2 *cpc = cbb + buf * kRecNodes;
        const int so0 = so & 0xff, so1 = (so >> 8) & 0xff, so2 = (so >> 16) & 0xff;
        float2 ga[W], gb[W];
#pragma unroll
        for (int z = 0; z < W; ++z) ga[z] = gb[z] = f2(0.f, 0.f);
        for (int jb = j0; jb < j1; jb += NB) {
            const int nb = min(NB, j1 - jb), b = jb - j0;
            ln.fetch(rec, b, pd);
            // the batch's c_j, zero past the piece; ones mode: (omega_j, 0)
            float2 cv[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k)
                cv[k] = k >= nb ? f2(0.f, 0.f) : (P.ones_mode ? f2(rec[4 * (b + k) + 3], 0.f) : cpc[b + k]);
            ln.evaluate(pd, stage);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const float *pk = stage + k * SS;
                float2 wa2, wb2;
                ln.weights(pk, wa2, wb2);
                const float2 ca2 = __fmul2_rn(cv[k], wa2), cb2 = __fmul2_rn(cv[k], wb2);
#pragma unroll
                for (int z = 0; z + 1 < W; z += 2) {
                    const float4 pz = *reinterpret_cast<const float4 *>(pk + 32 + 2 * z);
                    ga[z] = __ffma2_rn(ca2, f2(pz.x, pz.y), ga[z]);
                    gb[z] = __ffma2_rn(cb2, f2(pz.x, pz.y), gb[z]);
                    ga[z + 1] = __ffma2_rn(ca2, f2(pz.z, pz.w), ga[z + 1]);
                    gb[z + 1] = __ffma2_rn(cb2, f2(pz.z, pz.w), gb[z + 1]);
                }
                if constexpr (W % 2) {
                    const float2 pz = *reinterpret_cast<const float2 *>(pk + 32 + 2 * (W - 1));
                    ga[W - 1] = __ffma2_rn(ca2, pz, ga[W - 1]);
                    gb[W - 1] = __ffma2_rn(cb2, pz, gb[W - 1]);
                }
            }
            __syncwarp();
        }
        // add the piece's columns to the window in fixed point
        const int ga0 = (so0 + ln.xa) * L.SG + (so1 + ln.ya) * L.RG + so2;
        const int gb0 = (so0 + ln.xb) * L.SG + (so1 + ln.yb) * L.RG + so2;
        int *pa = &sG[ga0].x + sw, *pb = &sG[gb0].x + sw;
        const float2 qi2 = f2(q2inv, q2inv);
#pragma unroll
        for (int z = 0; z < W; ++z) {
            if (ln.act_a) {
                const float2 u = __fmul2_rn(ga[z], qi2);
                const int re = __float2int_rn(u.x), im = __float2int_rn(u.y);
                atomicAdd(pa + 2 * z, sw ? im : re);
                atomicAdd(pa + 2 * z + 1 - 2 * sw, sw ? re : im);
            }
            if (ln.act_b) {
                const float2 u = __fmul2_rn(gb[z], qi2);
                const int re = __float2int_rn(u.x), im = __float2int_rn(u.y);
                atomicAdd(pb + 2 * z, sw ? im : re);
                atomicAdd(pb + 2 * z + 1 - 2 * sw, sw ? re : im);
            }
        }
        buf ^= 1;
        sg = sg_n;
        so = so_n;
        j0 = j0_n;
        j1 = j1_n;
    }
    cp_async_wait<0>();
    __syncthreads();
    // the chunk's window, dense, to its scratch slot (thread: column wc.c of rows r0 + k rstep)
    cpx<float> *out = P.win + (int64_t)bid * P.win_cells + wc.c;
    for (int r = wc.r0; r < rows; r += wc.rstep) {
        const int2 g = sG[rowG[r] + wc.c];
        out[r * L.Wt2] = mk<float>((float)g.x * q2, (float)g.y * q2);
    }
}

}  // namespace nlp
