// Shared definitions of the nlpot CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/nlpot.h"

namespace nlp {

// window cells per 256-thread block of the window-sum pass (spread_common.cuh): FP32 64 cells
// with the members in 4 subsets (chunks of 2048 nodes: few, long member lists), FP64 256 cells
// read in member order (chunks of 256 nodes: many short lists)
template <typename T> constexpr int wsum_cells() { return sizeof(T) == 4 ? 64 : 256; }

// ---------------------------------------------------------------- complex arithmetic
template <typename T> struct cpx;
template <> struct __align__(8) cpx<float> { float x, y; };
template <> struct __align__(16) cpx<double> { double x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk<T>(a.x, -a.y); }
// multiply by +i (s = +1) or -i (s = -1)
template <typename T> __host__ __device__ __forceinline__ cpx<T> mul_i(cpx<T> a, int s) {
    return s > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ---------------------------------------------------------------- limits
constexpr int kMaxRadices = 16;     // FFT stages per length (N <= 2048 = 4^5 * 2)
constexpr int kMaxFftLen = 2048;
constexpr int kMaxWidth = 16;       // spreading-function width

// One FFT length: its radix sequence and a twiddle table exp(-2 pi i k / N), k < N.
template <typename T> struct FftLen {
    int N;
    int nrad;
    int rad[kMaxRadices];     // radices 4, 2, 3, 5 (shared-memory Stockham engine)
    int nrad_reg;
    int rad_reg[8];           // radices 16, 8, 4, 2, 3, 5 (register engine of the column passes)
    const cpx<T> *tw;         // device: e^{-2 pi i m / N}, m = 0..N-1
};

// Interp/spread work item: one chunk of the nodes of one tile.  Each chunk accumulates its
// tile window (tile + w - 1 cells per axis) on chip and writes it, once, to its own slot of
// the window scratch; the combine pass sums the slots into the spreading target.
struct Chunk {
    int bx, by, bz;     // unwrapped fine-grid cell of the tile origin
    int j0, j1;         // node range in the sorted node arrays
    float wsum;         // sum of |omega_j| over the chunk's nodes (bounds its window, see spread_dev.cuh)
};

// One window slot feeding one combine tile of the spreading target G (the k -> -k half
// spectrum).  For an output cell l of the tile, the slot's window cell is a_d = l_d + o_d
// (direct) or a_d = -l_d + o_d (mirror: the conjugate of the window value at -l goes to l),
// taken only when 0 <= a_d < window extent on every axis.
struct CombEntry {
    int chunk;          // window slot
    int mirror;         // 0 direct, 1 Hermitian mirror
    int o[3];
};

// Device pointers and sizes of one plan, in the plan precision T.
template <typename T> struct DevPlan {
    int dim;
    int n[3];           // grid (dim 2: n[2] = 1, last axis is axis 1)
    int nf[3];          // fine grid
    int nh;             // half spectrum length along the last axis (nf_last/2 + 1)
    int w;              // spreading width
    T beta;             // ES shape
    int T_tile[3];      // tile edge per axis (2D: T_tile[2] = 1)
    FftLen<T> len[3];   // FFT lengths of the fine axes
    // 2D, fine axis 1 too long for a register-engine block of enough columns: the four-step
    // decomposition N = N1 N2 (len4[0]: N1, len4[1]: N2) through the scratch spectrum S4
    int four;
    FftLen<T> len4[2];
    cpx<T> *S4;
    const T *deconv[3]; // 1/psi-hat(i 2pi/nf) per axis, i = 0..n-1 (grid index order)
    cpx<T> *F;          // forward spectrum, [nf0][nf1][nh] (3D) or [nf0][nh] (2D)
    cpx<T> *G;          // spread target, same layout
    // nodes, sorted by chunk: (delta_x, delta_y, delta_z, omega) and packed tile offsets
    const T *nd;        // 4 per node
    const uint32_t *no; // o_x | o_y << 8 | o_z << 16
    const Chunk *chunks;
    int64_t nchunks;
    // 2D Poisson (Algorithm 1): per-node FP64 (kx, ky, |k|) in node order, device FP64
    // moments {C0, M1x, M1y}, cell area and the auxiliary Gaussian width
    const double *pois;
    const double *mom;
    const double *u1tab;   // per grid point {u_{1,1}, u_{1,2} x, u_{1,2} y} (built at plan time)
    double hvol;
    double sigma;
    // register kernel (3D): sub-tile edge (0 = generic kernel only), segments = pieces of
    // runs of nodes of one sub-tile ([start, end) node pairs, packed sub-tile origin),
    // chunks = ranges of segments of one tile
    int sub_T;
    const int *seg_node;
    const uint32_t *seg_sub;
    const Chunk *rchunks;
    int64_t nrchunks;
    const T *psi_tab;   // per node: kernel values [3][W] in sub-window coordinates (register kernels)
    const T *psi_gen;   // 2D generic kernel: per node kernel values [3][w] on its own taps (axis 0 unused)
    int ones_mode;      // spreading of the weights alone (rho-hat := 1): builds the discrete kernel
    const cpx<T> *Khat; // precomputed-kernel method: spectrum of K on the 2n grid (else null)
    int accumulate;     // 1: the final pass adds into phi instead of overwriting it
    // window scratch and its combine into G (see spread_common.cuh)
    cpx<T> *win;        // one slot of win_n[0] x win_n[1] x win_n[2] cells per chunk of the active kernel
    int win_n[3];       // window extent (tile + w - 1 per axis; axis 0 of 2D plans: 1)
    int64_t win_cells;
    const int *grp;         // tiles split into several chunks: {first, count} into grp_list, per group
    const int *grp_list;    // slots of each such tile, ascending; the first one receives their sum
    int64_t ngroups;
    int grp_parts;          // window-sum tasks per group (wsum_cells<T>() cells of the window each)
    const int *cmb_off;     // per combine tile: its entries are cmb[cmb_off[t] .. cmb_off[t+1])
    const CombEntry *cmb;
    int cmb_t[3];       // combine tile edge per axis
    int cmb_n[3];       // combine tiles per axis (over nf0 x nf1 x nh)
    int64_t cmb_tiles;
    const int *cmb_act; // the tiles that windows reach (the others of G stay zero from plan time)
    int64_t cmb_nact;
    cpx<T> *cnode;      // FP32 warp kernels: c_j = rho-hat_j omega_j per node (interpolation -> spreading)
    T *csum;            // FP32 warp kernels: per chunk sum of |re c_j| + |im c_j| (bounds the window)
};

}  // namespace nlp

#define NLP_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return NLP_ERR_CUDA;        \
    } while (0)
