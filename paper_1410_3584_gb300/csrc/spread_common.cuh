// Device helpers shared by the interpolation/spreading kernels (spread.cu, spread_reg.cu,
// batch.cu): the spreading function, the tile window of the forward spectrum, and the
// combine pass that turns the chunks' windows into the spreading target G.
//
// Spreading without global atomics.  Every chunk (a run of the nodes of one fine-grid tile)
// accumulates the spread of its nodes over its tile window on chip, in an order fixed by
// the kernel, and writes that window once to its own slot of a scratch array.  The combine
// pass then owns each tile of G: for every output cell it adds, in a fixed order, the window
// cells of all slots that reach it, including the Hermitian mirror (a tap at position l of
// the k -> -k half contributes v at l and conj(v) at -l; only last-axis positions in
// [0, nf/2] are stored).  No value is ever added to global memory by two threads, so two
// evaluations of the same input give bit-identical results.
#pragma once
#include "common.cuh"

namespace nlp {

// exponential-of-semicircle spreading function at x = 2 (tap - node) / w, |x| < 1
template <typename T>
__device__ __forceinline__ T es_kernel(T x, T beta) {
    const T s = (T)1 - x * x;
    return s > (T)0 ? exp(beta * (sqrt(s) - (T)1)) : (T)0;
}

__device__ __forceinline__ int wrapn(int l, int N) {
    int r = l % N;
    return r < 0 ? r + N : r;
}

__host__ __device__ __forceinline__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Window rows of a tile chunk in the half spectrum.  Row r = a Wt1 + b of the tile window is
// the fine-grid line (l0, l1) = (bx + a, by + b) mod (nf0, nf1); its Hermitian mirror is the
// line (-l0, -l1).  The half-spectrum offsets of both lines are tabulated once per chunk, so
// that filling the window costs one table read and one add per cell.
template <typename T>
__device__ __forceinline__ void window_row_table(const DevPlan<T> &P, const Chunk &ch, int Wt0, int Wt1,
                                                 int64_t *rowoff, int64_t *rowmir) {
    for (int r = threadIdx.x; r < Wt0 * Wt1; r += blockDim.x) {
        const int a = r / Wt1, b = r - a * Wt1;
        const int l0 = wrapn(ch.bx + a, P.nf[0]), l1 = wrapn(ch.by + b, P.nf[1]);
        const int m0 = l0 ? P.nf[0] - l0 : 0, m1 = l1 ? P.nf[1] - l1 : 0;
        rowoff[r] = ((int64_t)l0 * P.nf[1] + l1) * P.nh;
        rowmir[r] = ((int64_t)m0 * P.nf[1] + m1) * P.nh;
    }
}

// The window column along the last axis that a thread fills for every row it visits
// (thread t: column t mod Wt2, rows t / Wt2 + k (blockDim / Wt2)), with the last-axis wrap
// and the Hermitian decision taken once per chunk.
struct WinCol {
    int c, r0, rstep;
    int l2;      // wrapped last-axis index
    bool herm;   // F read from the mirror line at nf2 - l2, conjugated
};

template <typename T>
__device__ __forceinline__ WinCol window_col(const DevPlan<T> &P, const Chunk &ch, int Wt2, int rows) {
    WinCol k;
    k.c = threadIdx.x % Wt2;
    k.rstep = blockDim.x / Wt2;
    k.r0 = threadIdx.x / Wt2;
    if (k.r0 >= k.rstep) k.r0 = rows;   // threads beyond rstep * Wt2 idle
    const int N2 = P.nf[2];
    k.l2 = wrapn(ch.bz + k.c, N2);
    k.herm = 2 * k.l2 > N2;
    return k;
}

// sF := F on the window (cell (r, c) at r * pitch + c for rows r < rows, or at
// (r / Wt1) * plane + (r % Wt1) * pitch + c when plane > 0); returns the largest |re| or |im|
// of the cells this thread filled.
template <typename T>
__device__ __forceinline__ T window_fill(const DevPlan<T> &P, const WinCol &k, const int64_t *rowoff,
                                         const int64_t *rowmir, int rows, int pitch, cpx<T> *sF, int Wt1 = 1,
                                         int plane = 0) {
    const int N2 = P.nf[2];
    T mx = (T)0;
    for (int r = k.r0; r < rows; r += k.rstep) {
        const cpx<T> v = k.herm ? conj(P.F[rowmir[r] + (N2 - k.l2)]) : P.F[rowoff[r] + k.l2];
        const int q = plane > 0 ? (r / Wt1) * plane + (r % Wt1) * pitch + k.c : r * pitch + k.c;
        sF[q] = v;
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
    return mx;
}

// ------------------------------------------------------------------ combine
// Tiles with many nodes are split into several chunks, whose windows share the tile's origin.
// First pass (window_sum_block): per such tile, the windows of its chunks are added cell by
// cell into its first slot.  Part p of group g covers window cells [C p, C p + C),
// C = wsum_cells<T>(); of the 256 threads of a block, thread (s, c) takes cell C p + c and the
// members of subset s (members s, s + S, s + 2S, ... in order, S = 256 / C), so that a heavy
// group (the FP32 tile at k = 0 holds up to ~150 chunks) is read with S times the loads in
// flight; the S partial sums of a cell are then added in subset order (S = 1: one sum in
// member order).  Shared memory: 256 member offsets, then (S - 1) C partial sums.
template <typename T> constexpr size_t window_sum_smem() {
    return 256 * sizeof(long long) + (size_t)(256 / wsum_cells<T>() - 1) * wsum_cells<T>() * sizeof(cpx<T>);
}

template <typename T>
__device__ __forceinline__ void window_sum_block(const DevPlan<T> &P, int64_t task, long long *sb) {
    constexpr int C = wsum_cells<T>(), S = 256 / C;
    const int64_t g = task / P.grp_parts;
    const int c = threadIdx.x % C, sub = threadIdx.x / C;
    const int64_t q = (task % P.grp_parts) * C + c;
    const bool act = q < P.win_cells && threadIdx.x < 256;
    const int first = P.grp[2 * g], count = P.grp[2 * g + 1];
    T sx = (T)0, sy = (T)0;
    // the members' slot offsets, staged 256 at a time (a multiple of S: subsets stay aligned)
    for (int m0 = 0; m0 < count; m0 += 256) {
        const int mc = min(256, count - m0);
        __syncthreads();
        for (int i = threadIdx.x; i < mc; i += blockDim.x) sb[i] = (long long)P.grp_list[first + m0 + i] * P.win_cells;
        __syncthreads();
        if (!act) continue;
        for (int i = sub; i < mc; i += 16 * S) {
            cpx<T> v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = (i + S * u < mc) ? P.win[sb[i + S * u] + q] : mk<T>(0, 0);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                sx += v[u].x;
                sy += v[u].y;
            }
        }
    }
    if constexpr (S > 1) {
        cpx<T> *red = reinterpret_cast<cpx<T> *>(sb + 256);
        __syncthreads();
        if (act && sub > 0) red[(sub - 1) * C + c] = mk<T>(sx, sy);
        __syncthreads();
        if (act && sub == 0) {
#pragma unroll
            for (int k = 0; k < S - 1; ++k) {
                const cpx<T> r = red[k * C + c];
                sx += r.x;
                sy += r.y;
            }
        }
    }
    if (act && sub == 0) P.win[(long long)P.grp_list[first] * P.win_cells + q] = mk<T>(sx, sy);
}

// Second pass: output tile t = (t0, t1, t2) covers cells [t_d T_d, min((t_d + 1) T_d, N_d)) of G
// with N = (nf0, nf1, nh).  The pass visits the tiles that some window reaches and writes each
// of their cells exactly once; the other tiles of G hold zeros from plan time (no pass writes
// G otherwise: the first inverse FFT pass reads G and writes its result elsewhere).  The
// tile's entries are staged in shared memory, 64 at a time.  A thread owns the cells of one
// (y, z) position of the tile along x and adds their window values in entry order; the loads
// of four entries and all its cells are issued together.
struct CombStage {
    long long base;    // slot * window cells
    int o0, o1, o2, s; // offsets and sign (+1 direct, -1 mirror)
};
constexpr int kCombStage = 64;

template <typename T, int CPT>
__device__ __forceinline__ void combine_block(const DevPlan<T> &P, int64_t tile, CombStage *st) {
    const int T0 = P.cmb_t[0], T1 = P.cmb_t[1], T2 = P.cmb_t[2];
    const int t2 = (int)(tile % P.cmb_n[2]);
    const int t1 = (int)((tile / P.cmb_n[2]) % P.cmb_n[1]);
    const int t0 = (int)(tile / ((int64_t)P.cmb_n[2] * P.cmb_n[1]));
    const int e0 = P.cmb_off[tile], e1 = P.cmb_off[tile + 1];
    const int W0 = P.win_n[0], W1 = P.win_n[1], W2 = P.win_n[2];
    const int64_t W12 = (int64_t)W1 * W2;
    const int N0 = P.nf[0], N1 = P.nf[1], N2 = P.nh;
    // thread: the (y, z) cell (c1, c2) of the tile for x = c0, c0 + S, ... (S = blockDim / (T1 T2),
    // CPT = ceil(T0 / S) cells)
    const int yz = T1 * T2;
    const int S = max(1, (int)blockDim.x / yz);
    const int c2 = threadIdx.x % T2, c1 = (threadIdx.x / T2) % T1, c0 = threadIdx.x / yz;
    const int l1 = t1 * T1 + c1, l2 = t2 * T2 + c2, lx = t0 * T0 + c0;
    const bool okyz = threadIdx.x < S * yz && l1 < N1 && l2 < N2;
    bool okx[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) okx[u] = okyz && c0 + u * S < T0 && lx + u * S < N0;
    T sx[CPT], sy[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) sx[u] = sy[u] = (T)0;
    constexpr int EB = CPT >= 4 ? 4 : 8;   // entries per batch of loads
    for (int eb = e0; eb < e1; eb += kCombStage) {
        const int ne = min(kCombStage, e1 - eb);
        __syncthreads();
        for (int i = threadIdx.x; i < ne; i += blockDim.x) {
            const CombEntry E = P.cmb[eb + i];
            st[i].base = (long long)E.chunk * P.win_cells;
            st[i].o0 = E.o[0];
            st[i].o1 = E.o[1];
            st[i].o2 = E.o[2];
            st[i].s = E.mirror ? -1 : 1;
        }
        __syncthreads();
        if (!okyz) continue;
        for (int e = 0; e < ne; e += EB) {
            cpx<T> v[EB][CPT];
#pragma unroll
            for (int k = 0; k < EB; ++k) {
                const CombStage E = st[min(e + k, ne - 1)];
                const int a1 = E.s * l1 + E.o1, a2 = E.s * l2 + E.o2;
                const bool inyz = e + k < ne && (unsigned)a1 < (unsigned)W1 && (unsigned)a2 < (unsigned)W2;
                const cpx<T> *row = P.win + E.base + (int64_t)a1 * W2 + a2;
                const int a00 = E.s * lx + E.o0, da = E.s * S;
#pragma unroll
                for (int u = 0; u < CPT; ++u) {
                    const int a0 = a00 + u * da;
                    v[k][u] = (inyz && okx[u] && (unsigned)a0 < (unsigned)W0) ? row[a0 * W12] : mk<T>(0, 0);
                    if (E.s < 0) v[k][u].y = -v[k][u].y;
                }
            }
#pragma unroll
            for (int k = 0; k < EB; ++k)
#pragma unroll
                for (int u = 0; u < CPT; ++u) {
                    sx[u] += v[k][u].x;
                    sy[u] += v[k][u].y;
                }
        }
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u)
        if (okx[u]) P.G[((int64_t)(lx + u * S) * P.nf[1] + l1) * P.nh + l2] = mk<T>(sx[u], sy[u]);
}

}  // namespace nlp
