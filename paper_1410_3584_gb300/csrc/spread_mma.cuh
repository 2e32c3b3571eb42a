// Fused interpolate -> scale -> spread on the tensor cores (FP32 plans, sub-window W = 8).
//
// Same operation and data as spread_warp_block (one warp per piece: a run of at most 64 nodes
// of one 2^3 sub-tile, all sharing the 8^3 sub-window of the tile window).  With the 64
// columns c = (x, y) of the sub-window and a batch of 8 nodes, the two z contractions are
// dense 64 x 8 x 8 products:
//   interpolation  S[c][n] = sum_z F[c][z] psi_z,n[z]                       (F . Psi_z)
//   spreading      G[c][z] += sum_n A[c][n] psi_z,n[z],  A[c][n] = c_n psi_x,n[x] psi_y,n[y]
// and run as mma.sync m16n8k8 TF32 (four 16-row tiles of columns each), every product split
// into hi + lo TF32 parts with the three cross terms hi.hi + hi.lo + lo.hi (relative error
// ~1e-7, FP32 level; the fourth term lo.lo is below FP32 rounding).  The x/y weights and the
// reduction over the columns stay on the FP32 pipes: with row r = 16 t + g (g = lane / 4) of
// column tile t holding column (x, y) = (g, 2t + r / 8), lane g owns column x = g for all y,
// so v_n = psi_x,n[g] sum_y psi_y,n[y] S[(g, y)][n] is 8 multiply-adds per node and lane and a
// reduction over the 8 lanes of equal lane % 4.  The interpolation's node order is permuted
// (B column j = node (j even ? j/2 : j/2 + 4)) so that the lane that ends with v_n for nodes
// q = lane % 4 and q + 4 is the lane whose spreading A fragment needs exactly those nodes:
// the scaled values never leave the registers.
#pragma once
#include "spread_common.cuh"
#include "spread_dev.cuh"

namespace nlp {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// hi = x rounded to TF32, lo = x - hi (its low mantissa bits are dropped by the MMA)
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_rna(x);
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// d += a . b for one m16n8k8 tile (A row-major 16 x 8, B column-major 8 x 8, FP32 accumulators)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += a . b with a and b given as TF32 hi/lo pairs: hi.hi + hi.lo + lo.hi
__device__ __forceinline__ void mma_3xtf32_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                                 const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bl);
    mma_tf32(d, ah, bh);
}

// the same with a in FP32 (split here)
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const float (&a)[4], const uint32_t (&bh)[2],
                                           const uint32_t (&bl)[2]) {
    uint32_t ah[4], al[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tf32_split(a[i], ah[i], al[i]);
    mma_3xtf32_split(d, ah, al, bh, bl);
}

constexpr int kMmaNB = 8;   // nodes per batch (the n extent of one MMA)

template <typename T>
__device__ __forceinline__ void spread_mma_block(const DevPlan<T> &P, int bid, unsigned char *smraw) {
    static_assert(sizeof(T) == 4, "FP32 plans");
    constexpr int W = 8, NB = kMmaNB;
    const int w = P.w;
    const int Wt0 = P.T_tile[0] + w - 1, Wt1 = P.T_tile[1] + w - 1, Wt2 = P.T_tile[2] + w - 1;
    const int P2 = Wt2 + 1, WWp = Wt0 * Wt1 * P2;   // z pitch padded by one cell
    cpx<T> *sF = (cpx<T> *)smraw;
    cpx<T> *sG = sF + WWp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    T *psi = (T *)(sG + WWp) + warp * (NB * 3 * W + 2 * NB);
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

    const int g = lane >> 2, q = lane & 3;           // MMA group (column x) and thread in group
    const int nodeB = (g & 1) ? (g >> 1) + 4 : (g >> 1);   // interpolation B column g -> node

    // kernel values of the batch (8 nodes x [x|y|z] x 8) and node weights, fetched into registers
    // one batch ahead (of this piece or of the warp's next piece)
    constexpr int PQ = NB * 3 * W / 32;
    T pf[PQ], wf;
    auto fetch = [&](int jbn, int nbn) {
        const T *src = P.psi_tab + (int64_t)jbn * 3 * W;
#pragma unroll
        for (int u = 0; u < PQ; ++u) {
            const int e = lane + 32 * u;
            pf[u] = (e < nbn * 3 * W) ? __ldg(src + e) : (T)0;
        }
        wf = (lane < nbn) ? __ldg(P.nd + 4 * ((int64_t)jbn + lane) + 3) : (T)0;
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
        // window cell of column (g, y), z: ((so0 + g) Wt1 + so1 + y) P2 + so2 + z
        const int cbase = ((so0 + g) * Wt1 + so1) * P2 + so2;
        // F as interpolation A fragments: tile t, element i -> column (g, 2t + (i & 1)),
        // z = q + 4 (i >> 1); split into TF32 hi/lo per batch (keeping the split for the whole
        // piece needs 168 registers, 3 CTAs per SM, and was measured slower)
        float Fr[4][4], Fi[4][4], Gr[4][4], Gi[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const cpx<T> f = sF[cbase + (2 * t + (i & 1)) * P2 + q + 4 * (i >> 1)];
                Fr[t][i] = f.x;
                Fi[t][i] = f.y;
                Gr[t][i] = Gi[t][i] = 0.f;
            }
        for (int jb = j0; jb < j1; jb += NB) {
#pragma unroll
            for (int u = 0; u < PQ; ++u) psi[lane + 32 * u] = pf[u];
            const T wcur = wf;
            __syncwarp();
            if (jb + NB < j1)
                fetch(jb + NB, min(NB, j1 - jb - NB));
            else if (sg_n < ch.j1)
                fetch(j0_n, min(NB, j1_n - j0_n));
            // psi row of node k: [x 0..7 | y 0..7 | z 0..7] at psi + 24 k (zeros for absent nodes)
            const T *pq = psi + q * 3 * W, *pq4 = psi + (q + 4) * 3 * W;
            // ---- interpolation: S = F . Psi_z (B column g = node nodeB), then the x/y weights
            uint32_t bh[2], bl[2];
            tf32_split(psi[nodeB * 3 * W + 2 * W + q], bh[0], bl[0]);
            tf32_split(psi[nodeB * 3 * W + 2 * W + q + 4], bh[1], bl[1]);
            float vr0 = 0.f, vi0 = 0.f, vr4 = 0.f, vi4 = 0.f;   // nodes q and q + 4
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float Sr[4] = {0.f, 0.f, 0.f, 0.f}, Si[4] = {0.f, 0.f, 0.f, 0.f};
                mma_3xtf32(Sr, Fr[t], bh, bl);
                mma_3xtf32(Si, Fi[t], bh, bl);
                // S element i: column (g, 2t + (i >> 1)), node q (i even) or q + 4 (i odd)
                const T y0q = pq[W + 2 * t], y1q = pq[W + 2 * t + 1];
                const T y0q4 = pq4[W + 2 * t], y1q4 = pq4[W + 2 * t + 1];
                vr0 += Sr[0] * y0q + Sr[2] * y1q;
                vi0 += Si[0] * y0q + Si[2] * y1q;
                vr4 += Sr[1] * y0q4 + Sr[3] * y1q4;
                vi4 += Si[1] * y0q4 + Si[3] * y1q4;
            }
            const T xq = pq[g], xq4 = pq4[g];
            vr0 *= xq;
            vi0 *= xq;
            vr4 *= xq4;
            vi4 *= xq4;
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                vr0 += __shfl_xor_sync(0xffffffffu, vr0, off);
                vi0 += __shfl_xor_sync(0xffffffffu, vi0, off);
                vr4 += __shfl_xor_sync(0xffffffffu, vr4, off);
                vi4 += __shfl_xor_sync(0xffffffffu, vi4, off);
            }
            // scale by the node weights: c_n = omega_n rho-hat-sum_n (lane n holds omega_n)
            const T om0 = __shfl_sync(0xffffffffu, wcur, q), om4 = __shfl_sync(0xffffffffu, wcur, q + 4);
            // ---- spreading: A[c][n] = c_n psi_x,n[g] psi_y,n[y], k = q (node q) and q + 4
            const T ar0 = vr0 * om0 * xq, ai0 = vi0 * om0 * xq, ar4 = vr4 * om4 * xq4, ai4 = vi4 * om4 * xq4;
            tf32_split(pq[2 * W + g], bh[0], bl[0]);      // B[k = q][z = g]
            tf32_split(pq4[2 * W + g], bh[1], bl[1]);     // B[k = q + 4][z = g]
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                // A element i: column (g, 2t + (i & 1)), node q (i < 2) or q + 4 (i >= 2)
                const T y0q = pq[W + 2 * t], y1q = pq[W + 2 * t + 1];
                const T y0q4 = pq4[W + 2 * t], y1q4 = pq4[W + 2 * t + 1];
                const float Ar[4] = {ar0 * y0q, ar0 * y1q, ar4 * y0q4, ar4 * y1q4};
                const float Ai[4] = {ai0 * y0q, ai0 * y1q, ai4 * y0q4, ai4 * y1q4};
                mma_3xtf32(Gr[t], Ar, bh, bl);
                mma_3xtf32(Gi[t], Ai, bh, bl);
            }
            __syncwarp();
        }
        // G element i of tile t: column (g, 2t + (i >> 1)), z = 2q + (i & 1); shared adds
        // (windows of the block's warps overlap).  Per column the lane adds four words v[zp][ri]
        // (z parity, real/imaginary part); in step s it adds the word (zp, ri) = bits of s ^ q,
        // so the 32 lanes of one add sit at word offsets 4 (g + q) + q (mod 32) -- with the
        // window's x stride of 4 (mod 32) words, distinct banks.  The lane-dependent order is
        // two predicated swaps per group of four.
        const bool swz = (q & 2) != 0, swr = (q & 1) != 0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int yp = 0; yp < 2; ++yp) {
                T v00 = Gr[t][2 * yp], v01 = Gi[t][2 * yp], v10 = Gr[t][2 * yp + 1], v11 = Gi[t][2 * yp + 1];
                if (swz) {
                    const T a = v00, b = v01;
                    v00 = v10; v01 = v11; v10 = a; v11 = b;
                }
                if (swr) {
                    const T a = v00, b = v10;
                    v00 = v01; v10 = v11; v01 = a; v11 = b;
                }
                T *cell = &sG[cbase + (2 * t + yp) * P2 + 2 * q].x;
                const int zx = q >> 1, rx = q & 1;
                atomicAdd(cell + 2 * (0 ^ zx) + (0 ^ rx), v00);
                atomicAdd(cell + 2 * (0 ^ zx) + (1 ^ rx), v01);
                atomicAdd(cell + 2 * (1 ^ zx) + (0 ^ rx), v10);
                atomicAdd(cell + 2 * (1 ^ zx) + (1 ^ rx), v11);
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
