// Internal declarations shared by the gbnfft CUDA translation units.
//
// Notation follows Section 2 of the paper: d dimensions, bandwidths N_t, grid sizes n_t,
// window cutoff m, M nodes x_j. A node's grid position is n_t x_t = base_t + frac_t with
// base_t = floor(n_t x_t) and frac_t in [0, 1]; its taps on axis t are the grid points
// l_t = base_t - m + i, i = 0..2m, of which i = 0 is inside the closed support |n x - l| <= m
// (eq. Inm) only when frac_t == 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbnfft.h"

namespace gbnfft {

constexpr int kMaxDim = 3;
constexpr int kMaxM = 8;           // window cutoffs 1..8 are instantiated
constexpr int kMaxSub = 1024;      // largest spreading subproblem (nodes of one bin per work item)

// Per-axis constants of the normalised window psibar(t) = psi(t) / psi(0), in grid units
// (Kaiser-Bessel, Gaussian, B-spline or sinc; the pairs are written out on the host at plan
// creation). psi(0) is folded into the deconvolution factors, which keeps FP32 values in range
// at any m. The kernels see the window only through the per-tap polynomials below and these
// two edge constants.
struct AxisWin {
    double prm;     // shape parameter: KB b, Gaussian b, sinc a (B-spline: unused)
    double edge_w;  // psibar(+-m) (the extra tap of a node on a grid point)
    double edge_dw; // d psibar / dt at t = m (from inside the support)
};

// Window values are evaluated from per-tap polynomials: for a node with offset frac in [0, 1]
// and tap i in 1..2m, psibar(frac + m - i) = P_i(z), z = 2 frac - 1, a polynomial of degree
// poly_degree(fp64, m) fitted at plan creation (Chebyshev interpolation in FP64, converted to
// monomials). The degree keeps the absolute error below ~1e-7 (FP32) / ~4e-15 (FP64) of
// psibar(0) = 1 for every oversampling factor sigma in (1, 16].
// Table layout per axis: coefficient k of tap i at [k * kPolyTaps + (i - 1)].
constexpr int kPolyTaps = 16;  // 2 * kMaxM
__host__ __device__ constexpr int poly_degree(bool fp64, int m)
{
    return fp64 ? (m <= 2 ? 18 : m <= 4 ? 16 : m == 5 ? 15 : 14)
                : (m <= 1 ? 11 : m == 2 ? 10 : m == 3 ? 9 : 8);
}
__host__ __device__ constexpr int poly_axis_stride(bool fp64, int m)
{
    return (poly_degree(fp64, m) + 1) * kPolyTaps;
}

// A spreading subproblem: up to kMaxSub consecutive sorted nodes of one bin.
struct SubProb {
    int bin;
    int start;
    int count;
    int pad;
};

// Stripe form of B^H (d = 2, see spread_impl.cuh): a super-bin is kStripeS stripes side by side
// along the last axis, a stripe being stripe_width(m) >= 2m cells (a whole number of sort bins)
// wide and one sort bin high. Stripes j and j + 2 of a super-bin never share a tile cell, so the
// kStripeHalves half-warps of a CTA spread the even stripes together, then the odd ones, into
// one tile.
constexpr int kStripeWarps = 4;
constexpr int kStripeHalves = 2 * kStripeWarps;
constexpr int kStripeS = 2 * kStripeHalves;
constexpr int kStripeItemDefault = 64;  // nodes per stripe per work item (super-bins are cut into
                                        // parts so that no stripe's part exceeds it)
__host__ __device__ constexpr int stripe_width(int m)
{
    return 2 * m <= 2 ? 2 : 2 * m <= 4 ? 4 : 2 * m <= 8 ? 8 : 16;
}

// Work of the stripe form, built by set_nodes from the sort bins.
struct StripeWork {
    const int *bin_start;   // per sort bin: position of its first node in sorted order
    const int *bin_count;   // per sort bin: number of nodes
    const SubProb *items;   // work items {bin = super-bin, start = part p, count = parts P}
    int *work;              // [0] items, [1] next unclaimed item, [2] CTAs finished
    int max_items;          // bound on the number of items
    int R;                  // sort bins per stripe along the last axis (0: no stripe work)
    int nsb1;               // super-bins along the last axis
};

// Spreading methods (see spread_impl.cuh); kSpreadAuto picks by tile size.
constexpr int kSpreadAuto = 0;
constexpr int kSpreadThread = 1;
constexpr int kSpreadWarpAtomic = 2;
constexpr int kSpreadWarpPrivate = 3;
constexpr int kSpreadOctet = 4;
constexpr int kSpreadHalf = 5;
constexpr int kSpreadPlane = 6;
constexpr int kSpreadStripe = 7;
constexpr int kSpreadRows = 8;

// Interpolation methods (see interp_impl.cuh).
constexpr int kInterpAuto = 0;
constexpr int kInterpThread = 1;
constexpr int kInterpWarp = 2;
constexpr int kInterpTile = 3;
constexpr int kInterpOctet = 4;

// Geometry passed by value to every kernel.
struct Geom {
    int d;
    int m;
    int spread_method;
    int interp_method;
    int n[kMaxDim];        // grid size per axis (even)
    int cbits[kMaxDim];    // bits of the axis' cell index in a packed cell, ceil(log2 n)
    int cmask[kMaxDim];    // (1 << cbits) - 1
    int N[kMaxDim];        // bandwidth per axis
    int bs[kMaxDim];       // bin (tile) size per axis, power of two
    int bslog[kMaxDim];
    int nb[kMaxDim];       // bins per axis
    AxisWin win[kMaxDim];
    const void *poly;      // device table of window polynomials (plan precision), d axes
    const void *poly_host; // host copy of the same table (source of WinCoef kernel arguments)
    const void *lin;       // lookup tables of the window (PRE_LIN_PSI), d axes, or null
    int lin_k;             // samples per unit of t of those tables; 0 = polynomial window
    StripeWork sw;         // stripe-form spreading work (set before each spreading launch)
};

// The window polynomial table as a kernel argument (same layout as the device table). Kernels
// that evaluate the window for every node take it by value with __grid_constant__: the
// coefficients are then read through the constant cache (as FMA operands where the tap index is
// known at compile time) rather than from shared memory, which the grid gathers need.
template <typename T, int MM> struct WinCoef {
    T c[kMaxDim * poly_axis_stride(sizeof(T) == 8, MM)];
};

template <typename T, int MM> inline WinCoef<T, MM> make_wincoef(const Geom &g)
{
    WinCoef<T, MM> w;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    const T *h = static_cast<const T *>(g.poly_host);
    for (int e = 0; e < kMaxDim * AS; e++) w.c[e] = (h && e < g.d * AS) ? h[e] : (T)0;
    return w;
}

// x mod n for x in [-n, 2n). Grid indices of taps and of tile cells never leave that range:
// taps lie within m < n/2 cells of a grid point, and bins are at most n/2 wide unless a single
// bin covers the axis (see setup_bins), so a tile ends before origin + n/2 + m <= 2n.
__host__ __device__ __forceinline__ int wrapn(int x, int n)
{
    x = x < 0 ? x + n : x;
    return x >= n ? x - n : x;
}

// x mod n for any x (tile cells of a partial last bin can lie beyond 2n).
__host__ __device__ __forceinline__ int modn(int x, int n)
{
    x %= n;
    return x < 0 ? x + n : x;
}

// Node record in sorted order. FP32: {cell bits, frac0, frac1, frac2}; FP64: cell in the
// first 8 bytes, then frac0..2. cell is the row-major index of (base_t mod n_t).
struct alignas(16) RecF {
    int cell;
    float fr[3];
};
struct alignas(16) RecD {
    int cell;
    int pad;
    double fr[3];
};
template <typename T> struct RecOf;
template <> struct RecOf<float> { using type = RecF; };
template <> struct RecOf<double> { using type = RecD; };

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Device status word values (a subset of nfft_status_code).
constexpr int kStatusOk = 0;

// ------------------------------------------------------------------------------------------
// Launchers (each enqueues on `stream`, returns cudaError_t of the launch)
// ------------------------------------------------------------------------------------------

// set_nodes: cell / row sub-bin / rank per node (a sub-bin is one grid row of a bin: the cell
// along axis 0 in 1-D and 2-D, the (axis 0, axis 1) pair in 3-D; index bin * S0 + row with
// S0 = bs0, or bs0 * bs1 in 3-D), then the bin totals, the scan over bins, the sub-bin starts,
// the counting sort (scatter), then subproblems.
template <typename T>
cudaError_t launch_node_bin(const Geom &g, const T *x, int64_t M, int *sub_count, int2 *sub_rank,
                            int *status, cudaStream_t stream);
cudaError_t launch_bin_totals(const int *sub_count, int S0, int nbins, int *bin_count,
                              cudaStream_t stream);
cudaError_t launch_sub_starts(const int *sub_count, const int *bin_start, int S0, int nbins,
                              int *sub_start, cudaStream_t stream);
cudaError_t launch_bin_scan(const int *bin_count, int *bin_start, int *sub_start, int *nsub_total,
                            int nbins, int sub_max, cudaStream_t stream, int nb0 = 0,
                            int nb1 = 0);
template <typename T>
cudaError_t launch_node_scatter(const Geom &g, const T *x, int64_t M, const int2 *sub_rank,
                                const int *sub_start, typename RecOf<T>::type *rec, int *perm,
                                cudaStream_t stream);
cudaError_t launch_fill_subprobs(const int *bin_count, const int *bin_start, const int *sub_start,
                                 SubProb *subs, int nbins, int sub_max, cudaStream_t stream);

// Work items of the stripe form (d = 2): per super-bin (kStripeS stripes of R sort bins in one
// sort-bin row) the node count of its heaviest stripe, the exclusive scan of the part counts
// P = ceil(count / item), and the item list {super-bin, part p, parts P}; sb_count, sb_start
// and sb_sub hold nsb values, work the item count (then zeroed work counters).
cudaError_t launch_stripe_items(const int *bin_count, int nb0, int nb1, int R, int nsb1,
                                int *sb_count, int *sb_start, int *sb_sub, int *work,
                                SubProb *items, int item, cudaStream_t stream);

// One axis pass of the pruned d-variate FFT.
//   in  : [outer][Lin][inner]   out : [outer][Lout][inner]
//   deconv: the per-axis factors, computed in FP64 and stored in the plan's precision.
//   pad  (forward, D fused): Lin = N_t, Lout = L = n_t; input index i (k = i - N_t/2) lands at
//        FFT position k mod n_t after multiplication by deconv[i]; other positions are zero.
//   crop (adjoint, D^H fused): Lin = L = n_t, Lout = N_t; output i takes FFT position
//        (i - N_t/2) mod n_t times deconv[i].
//   sign: -1 forward e^{-2 pi i kl/L}, +1 inverse.
template <typename T>
cudaError_t launch_fft_axis(const typename Cplx<T>::type *in, typename Cplx<T>::type *out,
                            int64_t outer, int64_t inner, int L, int Nt, int pad_mode, int sign,
                            const typename Cplx<T>::type *twiddle, const T *deconv,
                            cudaStream_t stream);

// Tables and scratch of one axis whose FFT length is not a power of two (Bluestein, see
// fft_impl.cuh): M = the power-of-two convolution length (>= 2L - 1), chirp[j] = e^(-pi i j^2/L)
// (L values), filt_fwd / filt_inv the length-M transforms of the wrapped conj(chirp) / chirp
// divided by M, twM the length-M twiddles, and two scratch buffers of lines x M values.
template <typename T> struct BluesteinAxis {
    int M;
    const void *chirp, *filt_fwd, *filt_inv, *twM;
    void *buf0, *buf1;
};
template <typename T>
cudaError_t launch_fft_axis_bluestein(const typename Cplx<T>::type *in,
                                      typename Cplx<T>::type *out, int64_t outer, int64_t inner,
                                      int L, int Nt, int pad_mode, int sign, const T *deconv,
                                      const BluesteinAxis<T> &ax, cudaStream_t stream);

// B: f[perm[s]] = sum over taps of grid * prod psibar. The tiled form walks the subproblem list
// built by set_nodes (subs, nsub_total, at most max_subs entries).
template <typename T>
cudaError_t launch_interp(const Geom &g, const typename Cplx<T>::type *grid,
                          const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                          const SubProb *subs, const int *nsub_total, int max_subs,
                          typename Cplx<T>::type *f, cudaStream_t stream);

// B^H: grid += spread of f over subproblems (grid must be zeroed first).
template <typename T>
cudaError_t launch_spread(const Geom &g, const typename Cplx<T>::type *f,
                          const typename RecOf<T>::type *rec, const int *perm,
                          const SubProb *subs, int *nsub_total, int max_subs,
                          typename Cplx<T>::type *grid, cudaStream_t stream);

// Node gradient: gx[perm[s]*d + t] = Re(conj(w[perm[s]]) * n_t * sum grid * dpsibar_t * ...).
template <typename T>
cudaError_t launch_grad(const Geom &g, const typename Cplx<T>::type *grid,
                        const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                        const typename Cplx<T>::type *w, T *gx, cudaStream_t stream);

// ------------------------------------------------------------------------------------------
// Fused batches: one launch per stage over every plan of a batch (see batch_fused.cu)
// ------------------------------------------------------------------------------------------
constexpr int kFusedMax = 128;          // plans of a fused batch (per-plan kernel arguments)
constexpr int kFusedFftThreads = 512;   // threads of a fused FFT CTA: P = 4096 / L lines of L

// Pointers that change from call to call, one per plan, passed to the kernels by value.
struct FusedPtrs {
    const void *in[kFusedMax];
    void *out[kFusedMax];
};

// First CTA of every plan in the per-node stages (128 sorted nodes per CTA) and in the zeroing
// of the grids, [kFusedMax + 1] entries each (the last one is the total), passed by value.
struct FusedOffsets {
    int node_block0[kFusedMax + 1];
    int zero_block0[kFusedMax + 1];
};

// A work item: CTA-sized piece `block` of plan `plan`'s work in one stage.
struct FusedItem {
    int plan;
    int block;
};

// One pruned-FFT pass of one plan (the arguments of launch_fft_axis, with P and LS fixed so that
// a block is P lines of L = 2^logl points on kFusedFftThreads threads).
struct FusedFftPass {
    const void *in;      // input lines; null: the call's input pointer of the plan
    void *out;           // output lines; null: the call's output pointer of the plan
    long long outer, inner;
    int logl, Nt, P, LS, pad_mode;
    const void *tw;      // twiddles of the pass' length (plan precision)
    const void *deconv;  // deconvolution factors of the pass' axis (plan precision)
};

// The per-node stages of one plan (interpolation, node gradient, spreading) in a fused launch.
struct FusedNodePlan {
    Geom g;
    void *grid;          // the plan's spreading grid (gA)
    void *fgrid;         // the plan's forward grid (gC), read by B and the node gradient
    const void *rec;     // sorted node records
    const int *perm;     // sorted position -> caller's node index
    const SubProb *subs; // spreading subproblems of the plan
    const int *nsub;     // [0]: number of subproblems
    int M;
    long long G;         // |I_n|
};

template <typename T>
cudaError_t launch_fft_fused(const FusedFftPass *passes, const FusedItem *items, int nitems,
                             int sign, size_t smem, const FusedPtrs &ptrs, cudaStream_t stream);
// FP32, d = 2 (batch_fused.cu): zeroing of the plans' grids, interpolation (grad = false: out[p]
// = f_p) or node gradient (grad = true: in[p] = w_p, out[p] = gx_p), and half-warp spreading
// (in[p] = f_p) with its item prefix. g0 is any plan's geometry (m is shared); shared_window:
// every plan has g0's window polynomials.
int zero_fused_blocks(long long G, size_t csize);
cudaError_t launch_zero_fused(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                              size_t csize, cudaStream_t stream);
cudaError_t launch_interp_fused(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                                const Geom &g0, const FusedPtrs &ptrs, bool grad,
                                bool shared_window, cudaStream_t stream);
cudaError_t launch_spread_fused(const FusedNodePlan *plans, int nplans, int *item_start,
                                int *work, int max_items, int tile_cells, const Geom &g0,
                                const FusedPtrs &ptrs, bool shared_window, int rows_bs0,
                                int rows_g, cudaStream_t stream);
int half_tile_cells_f32(int m, int bs0, int bs1);  // cells of one half-warp tile (FP32)
size_t half_smem_bytes_f32(int m, int tile_cells);  // shared memory of the half-warp form

// Dispatch on the window cutoff m (kernels are instantiated for m = 1..kMaxM).
#define GBNFFT_DISPATCH_M(FN, T, D, ...)                                                          \
    switch (g.m) {                                                                               \
    case 1: return FN<T, D, 1>(__VA_ARGS__);                                                     \
    case 2: return FN<T, D, 2>(__VA_ARGS__);                                                     \
    case 3: return FN<T, D, 3>(__VA_ARGS__);                                                     \
    case 4: return FN<T, D, 4>(__VA_ARGS__);                                                     \
    case 5: return FN<T, D, 5>(__VA_ARGS__);                                                     \
    case 6: return FN<T, D, 6>(__VA_ARGS__);                                                     \
    case 7: return FN<T, D, 7>(__VA_ARGS__);                                                     \
    case 8: return FN<T, D, 8>(__VA_ARGS__);                                                     \
    default: return cudaErrorInvalidValue;                                                       \
    }

// Opt a kernel in to `bytes` of dynamic shared memory (needed whenever static + dynamic shared
// memory exceeds 48 KB). The setting is per kernel and device; it is made once and raised when
// a larger size is requested (the cache is keyed by kernel address and device).
cudaError_t ensure_dynamic_smem_ptr(const void *kernel, size_t bytes);
template <typename K> cudaError_t ensure_dynamic_smem(K kernel, size_t bytes)
{
    return ensure_dynamic_smem_ptr(reinterpret_cast<const void *>(kernel), bytes);
}

namespace detail {
// Per-dimension launchers, each instantiated (for float and double) in its own translation
// unit k_<kernel>_<dtype>_d<D>.cu so that the library compiles in parallel.
template <typename T, int D>
cudaError_t interp_d(const Geom &g, const typename Cplx<T>::type *grid,
                     const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                     const SubProb *subs, const int *nsub_total, int max_subs,
                     typename Cplx<T>::type *f, cudaStream_t stream);
template <typename T, int D>
cudaError_t grad_d(const Geom &g, const typename Cplx<T>::type *grid,
                   const typename RecOf<T>::type *rec, const int *perm, int64_t M,
                   const typename Cplx<T>::type *w, T *gx, cudaStream_t stream);
template <typename T, int D>
cudaError_t spread_d(const Geom &g, const typename Cplx<T>::type *f,
                     const typename RecOf<T>::type *rec, const int *perm, const SubProb *subs,
                     int *nsub_total, int max_subs, typename Cplx<T>::type *grid,
                     cudaStream_t stream);
}  // namespace detail

int num_sms();

}  // namespace gbnfft
