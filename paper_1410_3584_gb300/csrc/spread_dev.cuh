// Interpolation/spreading device code shared by the single-plan kernels (spread.cu,
// spread_reg.cu) and the batched persistent kernel (batch.cu): per-block bodies with the
// block index passed explicitly.
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

// Shared memory of the generic kernel: F and G windows, kernel values of up to kGenericSlots
// warps, then the two row tables of the window.
constexpr int kGenericSlots = 8;
template <typename T> __host__ __device__ constexpr size_t generic_win_table_offset(size_t WW) {
    return align16(2 * WW * sizeof(cpx<T>) + (size_t)kGenericSlots * 3 * kMaxWidth * sizeof(T));
}

template <typename T>
__device__ __forceinline__ void spread_generic_block(const DevPlan<T> &P, int bid, unsigned char *smraw) {
    const int w = P.w;
    const int w0 = P.dim == 3 ? w : 1;
    const int W0 = P.T_tile[0] + w0 - 1, W1 = P.T_tile[1] + w - 1, W2 = P.T_tile[2] + w - 1;
    const int WW = W0 * W1 * W2;
    cpx<T> *sF = (cpx<T> *)smraw;
    cpx<T> *sG = sF + WW;
    T *spsi = (T *)(sG + WW);
    const int rows = W0 * W1;
    int64_t *rowoff = (int64_t *)(smraw + generic_win_table_offset<T>(WW)), *rowmir = rowoff + rows;
    const Chunk ch = P.chunks[bid];

    window_row_table(P, ch, W0, W1, rowoff, rowmir);
    const WinCol wc = window_col(P, ch, W2, rows);
    __syncthreads();
    if (P.ones_mode) {
        for (int q = threadIdx.x; q < WW; q += blockDim.x) sF[q] = sG[q] = mk<T>(0, 0);
    } else {
        window_fill(P, wc, rowoff, rowmir, rows, W2, sF, sG);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *ps = spsi + warp * 3 * kMaxWidth;
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
        // spreading
        for (int p = lane; p < w * w; p += 32) {
            const int b = p / w, c = p % w;
            const T wbc = ps[kMaxWidth + b] * ps[2 * kMaxWidth + c];
            const cpx<T> v = scale(cj, wbc);
            cpx<T> *col = sG + (o0 * W1 + (o1 + b)) * W2 + (o2 + c);
            for (int a = 0; a < w0; ++a) {
                const T wa = ps[a];
                red_add(col + a * sa, scale(v, wa));
            }
        }
        __syncwarp();
    }
    __syncthreads();
    window_fold(P, wc, rowoff, rowmir, rows, W2, sG);
}

// Shared memory of the warp kernel: F and G windows (z pitch Wt2 + 1), kernel values and
// reduced values of up to kWarpSlots warps, then the two row tables of the window.
constexpr int kWarpSlots = 8;
template <typename T, int W, int NB> __host__ __device__ constexpr size_t warp_win_table_offset(size_t WWp) {
    return align16(2 * WWp * sizeof(cpx<T>) + (size_t)kWarpSlots * (NB * 3 * W + 2 * NB) * sizeof(T));
}

// One warp per segment (W*W <= 64): lane L owns the z-columns L and L + 32 of the sub-window
// (their G accumulators in registers, their F values read from the shared window per node),
// so interpolation sums reduce inside the warp and the node loop needs no block barrier.
template <typename T, int W, int NB>
__device__ __forceinline__ void spread_warp_block(const DevPlan<T> &P, int bid, unsigned char *smraw) {
    static_assert(W * W <= 64, "two columns per lane");
    constexpr int V = 2 * NB;
    constexpr int SH = 5 - Log2<V>::value;
    const int w = P.w;
    const int Wt0 = P.T_tile[0] + w - 1, Wt1 = P.T_tile[1] + w - 1, Wt2 = P.T_tile[2] + w - 1;
    // window cells (a, b, c) at (a Wt1 + b) P2 + c with the z pitch padded by one cell: with
    // x fastest across the lanes, the 8-byte column accesses of a warp (tile 8, w 7: pitches
    // 210 and 15 cells) hit every bank pair exactly twice
    const int P2 = Wt2 + 1, WWp = Wt0 * Wt1 * P2;
    cpx<T> *sF = (cpx<T> *)smraw;
    cpx<T> *sG = sF + WWp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *psi = (T *)(sG + WWp) + warp * (NB * 3 * W + V);
    T *cb = psi + NB * 3 * W;
    const int rows = Wt0 * Wt1;
    int64_t *rowoff = (int64_t *)(smraw + warp_win_table_offset<T, W, NB>(WWp)), *rowmir = rowoff + rows;
    const Chunk ch = P.rchunks[bid];
    __shared__ int next_seg;
    if (threadIdx.x == 0) next_seg = ch.j0 + nwarps;

    window_row_table(P, ch, Wt0, Wt1, rowoff, rowmir);
    const WinCol wc = window_col(P, ch, Wt2, rows);
    __syncthreads();
    window_fill(P, wc, rowoff, rowmir, rows, P2, sF, sG);
    __syncthreads();

    const int ca = lane, cbc = lane + 32;
    // W*W > 32 for W >= 6: column a always active; W = 8: both columns of every lane
    const bool act_a = (W * W >= 32) || ca < W * W;
    const bool act_b = (W * W == 64) || cbc < W * W;
    const int xa = ca % W, ya = ca / W;
    const int xb = act_b ? cbc % W : 0, yb = act_b ? cbc / W : 0;
    constexpr bool kSameX = 32 % W == 0;   // then column b has the x of column a
    // the batch's kernel values are a contiguous block of the plan-time table; the next
    // block (of this piece or of the warp's next piece) is fetched into registers while the
    // current batch computes
    constexpr int PQ = (NB * 3 * W + 31) / 32;
    T pf[PQ], wf;
    auto fetch = [&](int jbn, int nbn) {
        const T *src = P.psi_tab + (int64_t)jbn * 3 * W;
#pragma unroll
        for (int u = 0; u < PQ; ++u) {
            const int q = lane + 32 * u;
            pf[u] = (q < nbn * 3 * W) ? __ldg(src + q) : (T)0;
        }
        wf = (lane < nbn) ? __ldg(P.nd + 4 * ((int64_t)jbn + lane) + 3) : (T)0;
    };
    // pieces are sorted heaviest first; each warp takes the next free one, claiming it (and
    // loading its descriptor) while the current piece computes
    int sg = ch.j0 + warp;
    uint32_t so = 0;
    int j0 = 0, j1 = 0;
    if (sg < ch.j1) {
        so = P.seg_sub[sg];
        j0 = P.seg_node[2 * sg];
        j1 = P.seg_node[2 * sg + 1];
        fetch(j0, min(NB, j1 - j0));
    }
    // lanes of odd x add the imaginary word of a cell first: with x fastest across the lanes
    // the two lanes that share a bank have x of opposite parity, so each add is conflict-free
    const int sw = xa & 1;
    while (sg < ch.j1) {
        int nxt = 0;
        if (lane == 0) nxt = atomicAdd(&next_seg, 1);
        const int sg_n = __shfl_sync(0xffffffffu, nxt, 0);
        uint32_t so_n = 0;
        int j0_n = 0, j1_n = 0;
        if (sg_n < ch.j1) {
            so_n = P.seg_sub[sg_n];
            j0_n = P.seg_node[2 * sg_n];
            j1_n = P.seg_node[2 * sg_n + 1];
        }
        const int so0 = so & 0xff, so1 = (so >> 8) & 0xff, so2 = (so >> 16) & 0xff;
        const int basea = ((so0 + (act_a ? xa : 0)) * Wt1 + (so1 + (act_a ? ya : 0))) * P2 + so2;
        const int baseb = ((so0 + xb) * Wt1 + (so1 + yb)) * P2 + so2;
        // G columns in registers; the F columns are read from the shared window per node, which
        // frees their registers for more warps per SM
        T gax[W], gay[W], gbx[W], gby[W];
#pragma unroll
        for (int z = 0; z < W; ++z) gax[z] = gay[z] = gbx[z] = gby[z] = (T)0;
        const cpx<T> *fca = sF + (act_a ? basea : 0), *fcb = sF + (act_b ? baseb : 0);
        // one batch of nodes; FULL (nb == NB) runs without per-node guards so that the
        // independent FMA chains of the batch's nodes interleave
        auto batch = [&](auto full_tag, int nb, T wcur) {
            constexpr bool FULL = decltype(full_tag)::value;
            T v[V], wa[NB], wb[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                v[2 * k] = v[2 * k + 1] = (T)0;
                wa[k] = wb[k] = (T)0;
                if (FULL || k < nb) {
                    const T *pk = psi + k * 3 * W;
                    const T pxa = pk[xa];
                    wa[k] = act_a ? pxa * pk[W + ya] : (T)0;
                    wb[k] = act_b ? (kSameX ? pxa : pk[xb]) * pk[W + yb] : (T)0;
                    T sax = 0, say = 0, sbx = 0, sby = 0;
                    T pzv[W];
                    load_row<T, W>(pk + 2 * W, pzv);
#pragma unroll
                    for (int z = 0; z < W; ++z) {
                        const T pz = pzv[z];
                        const cpx<T> fa = fca[z], fb = fcb[z];
                        sax += fa.x * pz;
                        say += fa.y * pz;
                        sbx += fb.x * pz;
                        sby += fb.y * pz;
                    }
                    v[2 * k] = wa[k] * sax + wb[k] * sbx;
                    v[2 * k + 1] = wa[k] * say + wb[k] * sby;
                }
            }
            warp_reduce_multi<T, V>(v, lane);
            {
                const int idx = (lane >> SH) & (V - 1);
                const int k = idx >> 1;
                const T wk = __shfl_sync(0xffffffffu, wcur, k);   // weight of node k of the batch
                if ((lane & ((1 << SH) - 1)) == 0) cb[idx] = (FULL || k < nb) ? v[0] * wk : (T)0;
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (FULL || k < nb) {
                    const T *pk = psi + k * 3 * W;
                    const T cr = cb[2 * k], ci = cb[2 * k + 1];
                    const T ar = cr * wa[k], ai = ci * wa[k], br = cr * wb[k], bi = ci * wb[k];
                    T pzv[W];
                    load_row<T, W>(pk + 2 * W, pzv);
#pragma unroll
                    for (int z = 0; z < W; ++z) {
                        const T pz = pzv[z];
                        gax[z] += ar * pz;
                        gay[z] += ai * pz;
                        gbx[z] += br * pz;
                        gby[z] += bi * pz;
                    }
                }
            }
        };
        for (int jb = j0; jb < j1; jb += NB) {
            const int nb = min(NB, j1 - jb);
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int q = lane + 32 * u;
                if (q < NB * 3 * W) psi[q] = pf[u];
            }
            const T wcur = wf;
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
        // overlapping windows of the block's warps: shared-memory atomics (zeros included: a
        // zero test per cell costs more than the add it would skip)
#pragma unroll
        for (int z = 0; z < W; ++z) {
            if (act_a) {
                T *c = &sG[basea + z].x;
                atomicAdd(c + sw, sw ? gay[z] : gax[z]);
                atomicAdd(c + (sw ^ 1), sw ? gax[z] : gay[z]);
            }
            if (act_b) {
                T *c = &sG[baseb + z].x;
                atomicAdd(c + sw, sw ? gby[z] : gbx[z]);
                atomicAdd(c + (sw ^ 1), sw ? gbx[z] : gby[z]);
            }
        }
        sg = sg_n;
        so = so_n;
        j0 = j0_n;
        j1 = j1_n;
    }
    __syncthreads();
    window_fold(P, wc, rowoff, rowmir, rows, P2, sG);
}

}  // namespace nlp
