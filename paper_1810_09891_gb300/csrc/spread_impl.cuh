// Step B^H of Algorithm "adjoint NFFT" (Section 2): g_l = sum_{j in I^T_{n,m}(l)} f_j psi~(x_j - l/n).
//
// GPU form of the paper's blockwise adjoint (Section 3.1, Table tab:nfftflags,
// NFFT_OMP_BLOCKWISE_ADJOINT): the grid is cut into bins, and each CTA takes one subproblem
// (at most kMaxSub sorted nodes of one bin). It accumulates their contributions into a
// shared-memory tile covering the bin plus a halo of m cells on each side, then adds the tile
// into the global grid with one vector atomic per complex cell. The kernels are persistent: a
// grid of a few CTAs per SM walks the subproblem list, whose length is read from device memory
// (it is only known on the device after the sort).
//
// Three ways to fill the tile (Geom::spread_method):
//   kSpreadThread  one thread per node, shared-memory atomics (interleaved re/im tile);
//   kSpreadWarpAtomic  one warp per node, the lanes cover the node's taps (so a warp never
//                  writes one cell twice), shared-memory atomics into one tile (re and im planes);
//   kSpreadWarpPrivate one warp per node as above, but every warp owns a private tile and adds
//                  with plain loads and stores (no atomics); the tiles are summed at the flush;
//   kSpreadOctet / kSpreadHalf (d = 2) eight or sixteen lanes per node, a private tile per
//                  group of lanes (see below);
//   kSpreadPlane   (d = 3) one tile per CTA whose planes are owned by the warps (see below).
// Coincident and clustered nodes (a radial trajectory puts every spoke through the origin) make
// the atomics of the first form collide; the warp forms do not.
#pragma once

#include "gbnfft_internal.cuh"
#include "window.cuh"

namespace gbnfft {
namespace detail {

// Dynamic scheduling of the subproblem list: work[0] holds the list length, work[1] the next
// unclaimed entry and work[2] the number of CTAs that have finished. A CTA claims one entry at a
// time with an atomic fetch (heavy and light bins of a nonuniform node set then even out across
// the SMs); the last CTA to finish puts both counters back to zero for the next launch. Nothing
// waits on another CTA.
__device__ __forceinline__ int next_subproblem(int *work, int *s_slot)
{
    __syncthreads();  // every thread has read the previous entry
    if (threadIdx.x == 0) *s_slot = atomicAdd(work + 1, 1);
    __syncthreads();
    return *s_slot;
}

__device__ __forceinline__ void finish_subproblems(int *work)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 2, 1) == (int)gridDim.x - 1) {
            work[1] = 0;
            work[2] = 0;
        }
    }
}



static __device__ __forceinline__ void global_add(float2 *p, float re, float im)
{
    atomicAdd(p, make_float2(re, im));  // vector reduction (sm_90 and later)
}
static __device__ __forceinline__ void global_add(double2 *p, double re, double im)
{
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

template <typename T, int D, int MM, int START>
__device__ __forceinline__ void spread_node(const Geom &g, const T *__restrict__ tab, T *tile,
                                            const int *tdim, const int *loc, const T *frac, T vr,
                                            T vi)
{
    constexpr int NT = 2 * MM + 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    if (D == 1) {
        T w0[NT];
        eval_taps<T, MM, START>(g, tab, 0, frac[0], w0);
#pragma unroll
        for (int i = START; i < NT; i++) {
            T *c = tile + 2 * (loc[0] + i);
            atomicAdd(c, vr * w0[i]);
            atomicAdd(c + 1, vi * w0[i]);
        }
    } else if (D == 2) {
        T w1[NT];
        eval_taps<T, MM, START>(g, tab + AS, 1, frac[1], w1);
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = eval_tap<T, MM>(g, tab, 0, i0, frac[0]);
            const T ar = vr * w0, ai = vi * w0;
            T *row = tile + 2 * ((loc[0] + i0) * tdim[1] + loc[1]);
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                atomicAdd(row + 2 * i1, ar * w1[i1]);
                atomicAdd(row + 2 * i1 + 1, ai * w1[i1]);
            }
        }
    } else {
        T w1[NT], w2[NT];
        eval_taps<T, MM, START>(g, tab + AS, 1, frac[1], w1);
        eval_taps<T, MM, START>(g, tab + 2 * AS, 2, frac[2], w2);
        for (int i0 = START; i0 < NT; i0++) {
            const T w0 = eval_tap<T, MM>(g, tab, 0, i0, frac[0]);
            const T ar = vr * w0, ai = vi * w0;
            T *plane = tile + 2 * ((loc[0] + i0) * tdim[1] * tdim[2]);
#pragma unroll
            for (int i1 = START; i1 < NT; i1++) {
                const T br = ar * w1[i1], bi = ai * w1[i1];
                T *row = plane + 2 * ((loc[1] + i1) * tdim[2] + loc[2]);
#pragma unroll
                for (int i2 = START; i2 < NT; i2++) {
                    atomicAdd(row + 2 * i2, br * w2[i2]);
                    atomicAdd(row + 2 * i2 + 1, bi * w2[i2]);
                }
            }
        }
    }
}

template <typename T, int D, int MM>
__global__ void __launch_bounds__(256)
    spread_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                  const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
                  const SubProb *__restrict__ subs, int *__restrict__ nsub_total,
                  typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) T tab[kMaxDim * poly_axis_stride(sizeof(T) == 8, MM)];
    load_window_tables<T, MM>(tab, g.poly, D);
    T *tile = reinterpret_cast<T *>(smem_raw);
    int tdim[D];
    int cells = 1;
#pragma unroll
    for (int t = 0; t < D; t++) {
        tdim[t] = g.bs[t] + 2 * MM;
        cells *= tdim[t];
    }
    const int nsub = nsub_total[0];
    __shared__ int s_sp;
    for (int sp = next_subproblem(nsub_total, &s_sp); sp < nsub;
         sp = next_subproblem(nsub_total, &s_sp)) {
        const SubProb P = subs[sp];
        int origin[D];
        {
            int b = P.bin;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                origin[t] = (b % g.nb[t]) * g.bs[t];
                b /= g.nb[t];
            }
        }
        for (int e = threadIdx.x; e < 2 * cells; e += blockDim.x) tile[e] = (T)0;
        __syncthreads();

        for (int k = threadIdx.x; k < P.count; k += blockDim.x) {
            const int s = P.start + k;
            const typename RecOf<T>::type r = rec[s];
            const C v = f[perm[s]];
            int cell = r.cell;
            int loc[D];
            T frac[D];
            bool edge = false;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                loc[t] = (cell & g.cmask[t]) - origin[t];  // in [0, bs_t)
                cell >>= g.cbits[t];
                frac[t] = r.fr[t];
                edge |= (frac[t] == (T)0);
            }
            if (!edge)
                spread_node<T, D, MM, 1>(g, tab, tile, tdim, loc, frac, v.x, v.y);
            else
                spread_node<T, D, MM, 0>(g, tab, tile, tdim, loc, frac, v.x, v.y);
        }
        __syncthreads();

        // flush: tile cell (a_0..a_{d-1}) is grid point (origin_t - m + a_t) mod n_t
        for (int e = threadIdx.x; e < cells; e += blockDim.x) {
            const T re = tile[2 * e], im = tile[2 * e + 1];
            if (re == (T)0 && im == (T)0) continue;
            int rem = e;
            size_t gi = 0;
            int a[D];
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                a[t] = rem % tdim[t];
                rem /= tdim[t];
            }
#pragma unroll
            for (int t = 0; t < D; t++)
                gi = gi * g.n[t] + (size_t)wrapn(origin[t] - MM + a[t], g.n[t]);
            global_add(grid + gi, re, im);
        }
        __syncthreads();
    }
    finish_subproblems(nsub_total);
}

// ----------------------------------------------------------------------------- warp forms

constexpr int kSpreadWarps = 8;  // warps per CTA of the warp forms

// Shared memory of the warp forms: the tile(s), then a staging area for one chunk of
// kSpreadChunk sorted nodes (their records and values, loaded with coalesced reads while the
// previous chunk is being spread).
constexpr int kSpreadChunk = 32 * kSpreadWarps;

template <typename T>
__host__ __device__ constexpr size_t spread_stage_bytes()
{
    return kSpreadChunk * (sizeof(typename RecOf<T>::type) + sizeof(typename Cplx<T>::type));
}

// The taps of one node, 32 at a time across the lanes of a warp. Tap q enumerates the
// (2m + 1 - START)^d box row-major (last axis fastest, so neighbouring lanes hit neighbouring
// cells); its weight is the product of the per-axis window values held by lanes t*NT + i.
// `off` is the tile index of the box corner (loc_t + START on every axis); `st` the tile strides.
template <typename T, int D, int MM, int START>
__device__ __forceinline__ void tap_of_lane(int q, const int *st, T wa, T wb, T &w, int &rel)
{
    constexpr int NT = 2 * MM + 1;
    constexpr int NW = D * NT;
    constexpr int PER = NT - START;
    int rem = q;
    w = (T)1;
    rel = 0;
#pragma unroll
    for (int t = D - 1; t >= 0; t--) {
        const int a = rem % PER;
        rem /= PER;
        const int src = t * NT + a + START;
        const T wa_s = __shfl_sync(0xffffffffu, wa, src & 31);
        T wt = wa_s;
        if (NW > 32) {
            const T wb_s = __shfl_sync(0xffffffffu, wb, src & 31);
            wt = src < 32 ? wa_s : wb_s;
        }
        w *= wt;
        rel += a * st[t];
    }
}

// Private tile of complex values: plain read-modify-write, one 8- or 16-byte access per tap.
template <typename T, int D, int MM, int START>
__device__ __forceinline__ void spread_warp_taps_private(typename Cplx<T>::type *tile,
                                                         const int *st, int off, T wa, T wb,
                                                         typename Cplx<T>::type v, int lane)
{
    using C = typename Cplx<T>::type;
    constexpr int PER = 2 * MM + 1 - START;
    constexpr int TAPS = D == 1 ? PER : (D == 2 ? PER * PER : PER * PER * PER);
    constexpr int ITER = (TAPS + 31) / 32;
    if (ITER <= 8) {
#pragma unroll
        for (int k = 0; k < ITER; k++) {
            const int q = 32 * k + lane;
            T w;
            int rel;
            tap_of_lane<T, D, MM, START>(q < TAPS ? q : 0, st, wa, wb, w, rel);
            if (q < TAPS) {
                C c = tile[off + rel];
                c.x += w * v.x;
                c.y += w * v.y;
                tile[off + rel] = c;
            }
        }
    } else {
#pragma unroll 1
        for (int k = 0; k < ITER; k++) {
            const int q = 32 * k + lane;
            T w;
            int rel;
            tap_of_lane<T, D, MM, START>(q < TAPS ? q : 0, st, wa, wb, w, rel);
            if (q < TAPS) {
                C c = tile[off + rel];
                c.x += w * v.x;
                c.y += w * v.y;
                tile[off + rel] = c;
            }
        }
    }
}

// One tile for the CTA, real and imaginary planes, shared-memory atomics.
template <typename T, int D, int MM, int START>
__device__ __forceinline__ void spread_warp_taps_atomic(T *re, T *im, const int *st, int off,
                                                        T wa, T wb, typename Cplx<T>::type v,
                                                        int lane)
{
    constexpr int PER = 2 * MM + 1 - START;
    constexpr int TAPS = D == 1 ? PER : (D == 2 ? PER * PER : PER * PER * PER);
    constexpr int ITER = (TAPS + 31) / 32;
#pragma unroll 4
    for (int k = 0; k < ITER; k++) {
        const int q = 32 * k + lane;
        T w;
        int rel;
        tap_of_lane<T, D, MM, START>(q < TAPS ? q : 0, st, wa, wb, w, rel);
        if (q < TAPS) {
            atomicAdd(re + off + rel, w * v.x);
            atomicAdd(im + off + rel, w * v.y);
        }
    }
}

template <typename T, int D, int MM, bool PRIVATE>
__global__ void __launch_bounds__(32 * kSpreadWarps)
    spread_warp_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                       const typename RecOf<T>::type *__restrict__ rec,
                       const int *__restrict__ perm, const SubProb *__restrict__ subs,
                       int *__restrict__ nsub_total, typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    constexpr int NT = 2 * MM + 1;        // tap slots per axis (slot 0 only on a grid point)
    constexpr int NW = D * NT;            // window values per node
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) T tab[kMaxDim * AS];
    load_window_tables<T, MM>(tab, g.poly, D);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    // Lane (t * NT + i) evaluates the window of tap i on axis t for every node (lanes + 32 for
    // the second set when NW > 32): its polynomial coefficients stay in registers.
    constexpr int DEG = PolyDeg<T, MM>::value;
    T ca[DEG + 1], cb[DEG + 1];
    int ta = 0, ia = 0, tb = 0, ib = 0;
    T ea = (T)0, eb = (T)0;
    {
        const int qa = lane < NW ? lane : 0;
        ta = qa / NT;
        ia = qa - ta * NT;
        const int qb = (NW > 32 && lane + 32 < NW) ? lane + 32 : 0;
        tb = qb / NT;
        ib = qb - tb * NT;
#pragma unroll
        for (int k = 0; k <= DEG; k++) {
            ca[k] = ia > 0 ? tab[ta * AS + k * kPolyTaps + ia - 1] : (T)0;
            cb[k] = (NW > 32 && ib > 0) ? tab[tb * AS + k * kPolyTaps + ib - 1] : (T)0;
        }
        ea = (T)g.win[ta].edge_w;
        eb = (T)g.win[tb].edge_w;
    }
    int tdim[D];
    int cells = 1;
#pragma unroll
    for (int t = 0; t < D; t++) {
        tdim[t] = g.bs[t] + 2 * MM;
        cells *= tdim[t];
    }
    T *sm = reinterpret_cast<T *>(smem_raw);
    const size_t tile_reals = (size_t)2 * cells * (PRIVATE ? kSpreadWarps : 1);
    Rec *st_rec = reinterpret_cast<Rec *>(smem_raw + ((tile_reals * sizeof(T) + 15) / 16) * 16);
    C *st_val = reinterpret_cast<C *>(st_rec + kSpreadChunk);
    // private: one complex tile per warp; atomic: one re plane and one im plane per CTA
    C *ptile = reinterpret_cast<C *>(sm) + (size_t)warp * cells;
    T *re = sm;
    T *im = sm + cells;
    int st[D];  // tile strides
    st[D - 1] = 1;
#pragma unroll
    for (int t = D - 2; t >= 0; t--) st[t] = st[t + 1] * tdim[t + 1];
    const int nsub = nsub_total[0];
    __shared__ int s_sp;
    for (int sp = next_subproblem(nsub_total, &s_sp); sp < nsub;
         sp = next_subproblem(nsub_total, &s_sp)) {
        const SubProb P = subs[sp];
        int origin[D];
        {
            int b = P.bin;
#pragma unroll
            for (int t = D - 1; t >= 0; t--) {
                origin[t] = (b % g.nb[t]) * g.bs[t];
                b /= g.nb[t];
            }
        }
        // first chunk of node data in flight while the tile is cleared
        Rec r_next;
        C v_next;
        if (tid < P.count) {
            r_next = rec[P.start + tid];
            v_next = f[perm[P.start + tid]];
        }
        if (PRIVATE) {
            T *pz = reinterpret_cast<T *>(ptile);
            for (int e = lane; e < 2 * cells; e += 32) pz[e] = (T)0;
        } else {
            for (int e = tid; e < 2 * cells; e += blockDim.x) sm[e] = (T)0;
        }

        for (int c0 = 0; c0 < P.count; c0 += kSpreadChunk) {
            const int cnt = min(kSpreadChunk, P.count - c0);
            if (tid < cnt) {
                st_rec[tid] = r_next;
                st_val[tid] = v_next;
            }
            __syncthreads();
            {
                const int nx = c0 + kSpreadChunk + tid;  // prefetch the next chunk
                if (nx < P.count) {
                    r_next = rec[P.start + nx];
                    v_next = f[perm[P.start + nx]];
                }
            }
            for (int k = warp; k < cnt; k += kSpreadWarps) {
                const Rec r = st_rec[k];
                const C v = st_val[k];
                int cell = r.cell;
                int loc[D];
                T frac[D];
                bool edge = false;
#pragma unroll
                for (int t = D - 1; t >= 0; t--) {
                    loc[t] = (cell & g.cmask[t]) - origin[t];
                    cell >>= g.cbits[t];
                    frac[t] = r.fr[t];
                    edge |= (frac[t] == (T)0);
                }
                // lane (t * NT + i) holds psibar of tap i on axis t (two rounds when NW > 32)
                T wa = (T)0, wb = (T)0;
                {
                    T fa = frac[0], fb = frac[0];
#pragma unroll
                    for (int t = 1; t < D; t++) {
                        if (ta == t) fa = frac[t];
                        if (tb == t) fb = frac[t];
                    }
                    if (g.lin_k) {  // lookup-table window
                        if (lane < NW)
                            wa = lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, ta), g.lin_k, ia,
                                                fa, ea);
                        if (NW > 32 && lane + 32 < NW)
                            wb = lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, tb), g.lin_k, ib,
                                                fb, eb);
                    } else {
                        if (lane < NW) wa = ia > 0 ? poly_horner<T, DEG>(ca, (T)2 * fa - (T)1)
                                                   : (fa == (T)0 ? ea : (T)0);
                        if (NW > 32 && lane + 32 < NW)
                            wb = ib > 0 ? poly_horner<T, DEG>(cb, (T)2 * fb - (T)1)
                                        : (fb == (T)0 ? eb : (T)0);
                    }
                }
                int off = 0;
#pragma unroll
                for (int t = 0; t < D; t++) off += loc[t] * st[t];
                if (edge) {  // warp-uniform (one node per warp)
                    if (PRIVATE)
                        spread_warp_taps_private<T, D, MM, 0>(ptile, st, off, wa, wb, v, lane);
                    else
                        spread_warp_taps_atomic<T, D, MM, 0>(re, im, st, off, wa, wb, v, lane);
                } else {
                    int off1 = off;
#pragma unroll
                    for (int t = 0; t < D; t++) off1 += st[t];  // first tap slot is 1
                    if (PRIVATE)
                        spread_warp_taps_private<T, D, MM, 1>(ptile, st, off1, wa, wb, v, lane);
                    else
                        spread_warp_taps_atomic<T, D, MM, 1>(re, im, st, off1, wa, wb, v, lane);
                }
                if (PRIVATE) __syncwarp();
            }
            __syncthreads();
        }
        if (P.count == 0) __syncthreads();

        // flush: tile cell (a_0..a_{d-1}) is grid point (origin_t - m + a_t) mod n_t; one warp
        // per tile row, lanes along the contiguous last axis
        const int rows = cells / tdim[D - 1];
        for (int row = warp; row < rows; row += kSpreadWarps) {
            size_t gbase = 0;
            {
                int rem = row;
                int a[D];
                a[D - 1] = 0;
#pragma unroll
                for (int t = D - 2; t >= 0; t--) {
                    a[t] = rem % tdim[t];
                    rem /= tdim[t];
                }
#pragma unroll
                for (int t = 0; t < D - 1; t++)
                    gbase = gbase * g.n[t] + (size_t)wrapn(origin[t] - MM + a[t], g.n[t]);
                gbase *= g.n[D - 1];
            }
            for (int a = lane; a < tdim[D - 1]; a += 32) {
                const int e = row * tdim[D - 1] + a;
                T vr, vi;
                if (PRIVATE) {
                    vr = (T)0;
                    vi = (T)0;
                    const C *all = reinterpret_cast<const C *>(sm);
#pragma unroll
                    for (int w = 0; w < kSpreadWarps; w++) {
                        const C c = all[(size_t)w * cells + e];
                        vr += c.x;
                        vi += c.y;
                    }
                } else {
                    vr = sm[e];
                    vi = sm[cells + e];
                }
                if (vr == (T)0 && vi == (T)0) continue;
                const size_t gi =
                    gbase + (size_t)wrapn(origin[D - 1] - MM + a, g.n[D - 1]);
                global_add(grid + gi, vr, vi);
            }
        }
        __syncthreads();
    }
    finish_subproblems(nsub_total);
}

// ----------------------------------------------------------------------------- octet form (d = 2)
// Eight lanes per node, four nodes per warp, 32 private complex tiles per CTA. Lane l of a group
// owns the tap rows a0 = l, l + 8, ... of its node (each a run of 2m (+1) contiguous tile cells)
// and adds them with plain read-modify-write; the column weights are evaluated once per lane
// (taps l and l + 8) and shared inside the group with shuffles. Per node this costs about a
// quarter of the warp form's instructions.
constexpr int kOctets = 4 * kSpreadWarps;  // groups (and private tiles) per CTA

// Cells between consecutive private tiles: for FP32 an odd multiple of 8 cells (half the 32
// banks), so that the four groups of a warp, each touching 8 contiguous cells of its own tile,
// fall in alternating bank halves; FP64 groups already fill all banks.
template <typename T> __host__ __device__ inline int octet_tile_stride(int cells)
{
    if (sizeof(T) == 8) return cells;
    return cells + ((8 - cells % 16) + 16) % 16;
}

template <typename T, int MM, int START>
__device__ __forceinline__ void spread_octet_node(typename Cplx<T>::type *tile, int st0, int off,
                                                  T frac0, T frac1, const T *ca, T ea,
                                                  const T *cb, T eb,
                                                  typename Cplx<T>::type v, int l,
                                                  unsigned mask, const T *la, const T *lb, int K)
{
    using C = typename Cplx<T>::type;
    constexpr int DEG = PolyDeg<T, MM>::value;
    constexpr int NT = 2 * MM + 1;
    constexpr int PER = NT - START;
    const T z0 = (T)2 * frac0 - (T)1, z1 = (T)2 * frac1 - (T)1;
    if (START == 1 && K == 0) {
        // Mirrored taps (see window_taps): pair p < m holds column taps p + 1 and 2m - p, pair
        // m + q holds row taps q + 1 and 2m - q, each as (E + zO, E - zO) from one even/odd
        // Horner evaluation; lane l evaluates pairs l and l + 8.
        constexpr int KE = DEG - (DEG & 1), KO = DEG - 1 + (DEG & 1), NP = 2 * MM;
        T pa = (T)0, ma = (T)0, pb = (T)0, mb = (T)0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int pp = l + 8 * h;
            if ((h == 0 || NP > 8) && pp < NP) {
                const bool colp = pp < MM;
                const T *cc = colp ? cb : ca;
                const T z = colp ? z1 : z0;
                const int i = (colp ? pp : pp - MM) + 1;
                const T u = z * z;
                T e = cc[KE * kPolyTaps + i - 1], o = cc[KO * kPolyTaps + i - 1];
#pragma unroll
                for (int k = KE - 2; k >= 0; k -= 2) e = fma(e, u, cc[k * kPolyTaps + i - 1]);
#pragma unroll
                for (int k = KO - 2; k >= 1; k -= 2) o = fma(o, u, cc[k * kPolyTaps + i - 1]);
                if (h == 0) {
                    pa = fma(z, o, e);
                    ma = fma(-z, o, e);
                } else {
                    pb = fma(z, o, e);
                    mb = fma(-z, o, e);
                }
            }
        }
        // column weights of this lane: columns a = l and l + 8 hold taps a + 1
        T w1[2] = {(T)0, (T)0};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (h == 1 && PER <= 8) break;
            const int t = l + 8 * h + 1;
            const int pp = t <= MM ? t - 1 : 2 * MM - t;  // column pair of tap t (or its mirror)
            const int src = pp & 7;
            const T vpa = __shfl_sync(mask, pa, src, 8), vma = __shfl_sync(mask, ma, src, 8);
            const T vpb = NP > 8 ? __shfl_sync(mask, pb, src, 8) : (T)0;
            const T vmb = NP > 8 ? __shfl_sync(mask, mb, src, 8) : (T)0;
            const T plus = pp < 8 ? vpa : vpb, minus = pp < 8 ? vma : vmb;
            w1[h] = t <= PER ? (t <= MM ? plus : minus) : (T)0;
        }
        const T ar = w1[0] * v.x, ai = w1[0] * v.y, br = w1[1] * v.x, bi = w1[1] * v.y;
        C *col = tile + off + l;
#pragma unroll
        for (int a0 = 0; a0 < PER; a0++) {
            const int t = a0 + 1;                                  // row tap
            const int pp = t <= MM ? MM + t - 1 : 3 * MM - t;      // its row pair
            const T var = pp < 8 ? (t <= MM ? pa : ma) : (t <= MM ? pb : mb);
            const T w0 = __shfl_sync(mask, var, pp & 7, 8);
            C *row = col + a0 * st0;
            if (l < PER) {
                C c = row[0];
                c.x += w0 * ar;
                c.y += w0 * ai;
                row[0] = c;
            }
            if (PER > 8 && l + 8 < PER) {
                C c = row[8];
                c.x += w0 * br;
                c.y += w0 * bi;
                row[8] = c;
            }
        }
        return;
    }
    // this lane's columns a1 = l and l + 8, and the row weights a0 = l, l + 8 it broadcasts
    T w1a = (T)0, w1b = (T)0, w0a = (T)0, w0b = (T)0;
    if (l < PER) {
        const int i = START + l;
        if (K) {  // lookup-table window (la, lb: the axes' tables)
            w1a = lin_tap<T, MM>(lb, K, i, frac1, eb);
            w0a = lin_tap<T, MM>(la, K, i, frac0, ea);
        } else {
            w1a = i == 0 ? (frac1 == (T)0 ? eb : (T)0) : poly_horner_tap<T, DEG>(cb, i, z1);
            w0a = i == 0 ? (frac0 == (T)0 ? ea : (T)0) : poly_horner_tap<T, DEG>(ca, i, z0);
        }
    }
    if (PER > 8 && l + 8 < PER) {
        const int i = START + l + 8;
        w1b = K ? lin_tap<T, MM>(lb, K, i, frac1, eb) : poly_horner_tap<T, DEG>(cb, i, z1);
        w0b = K ? lin_tap<T, MM>(la, K, i, frac0, ea) : poly_horner_tap<T, DEG>(ca, i, z0);
    }
    const T ar = w1a * v.x, ai = w1a * v.y, br = w1b * v.x, bi = w1b * v.y;
    C *col = tile + off + l;
#pragma unroll
    for (int a0 = 0; a0 < PER; a0++) {
        const T w0 = __shfl_sync(mask, a0 < 8 ? w0a : w0b, a0 & 7, 8);
        C *row = col + a0 * st0;
        if (l < PER) {
            C c = row[0];
            c.x += w0 * ar;
            c.y += w0 * ai;
            row[0] = c;
        }
        if (PER > 8 && l + 8 < PER) {
            C c = row[8];
            c.x += w0 * br;
            c.y += w0 * bi;
            row[8] = c;
        }
    }
}

template <typename T, int MM>
__global__ void __launch_bounds__(32 * kSpreadWarps)
    spread_octet_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                        const typename RecOf<T>::type *__restrict__ rec,
                        const int *__restrict__ perm, const SubProb *__restrict__ subs,
                        int *__restrict__ nsub_total, typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    __shared__ __align__(16) T tab[kMaxDim * AS];
    load_window_tables<T, MM>(tab, g.poly, 2);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int l = lane & 7, oct = tid >> 3;
    const unsigned mask = 0xffu << (lane & 24);
    const int td0 = g.bs[0] + 2 * MM, td1 = g.bs[1] + 2 * MM;
    const int cells = td0 * td1;
    const int tstride = octet_tile_stride<T>(cells);  // staggers the tiles over the banks
    C *tiles = reinterpret_cast<C *>(smem_raw);
    C *mine = tiles + (size_t)oct * tstride;
    Rec *st_rec = reinterpret_cast<Rec *>(smem_raw + (size_t)kOctets * tstride * sizeof(C));
    C *st_val = reinterpret_cast<C *>(st_rec + kSpreadChunk);
    const T *ca = tab, *cb = tab + AS;
    const T ea = (T)g.win[0].edge_w, eb = (T)g.win[1].edge_w;
    const T *la = g.lin_k ? lin_axis<T, MM>(g.lin, g.lin_k, 0) : nullptr;
    const T *lb = g.lin_k ? lin_axis<T, MM>(g.lin, g.lin_k, 1) : nullptr;
    const int nsub = nsub_total[0];
    __shared__ int s_sp;
    for (int sp = next_subproblem(nsub_total, &s_sp); sp < nsub;
         sp = next_subproblem(nsub_total, &s_sp)) {
        const SubProb P = subs[sp];
        const int org1 = (P.bin % g.nb[1]) * g.bs[1];
        const int org0 = (P.bin / g.nb[1]) * g.bs[0];
        Rec r_next;
        C v_next;
        if (tid < P.count) {
            r_next = rec[P.start + tid];
            v_next = f[perm[P.start + tid]];
        }
        {
            T *pz = reinterpret_cast<T *>(mine);
            for (int e = l; e < 2 * cells; e += 8) pz[e] = (T)0;
        }
        for (int c0 = 0; c0 < P.count; c0 += kSpreadChunk) {
            const int cnt = min(kSpreadChunk, P.count - c0);
            if (tid < cnt) {
                st_rec[tid] = r_next;
                st_val[tid] = v_next;
            }
            __syncthreads();
            {
                const int nx = c0 + kSpreadChunk + tid;
                if (nx < P.count) {
                    r_next = rec[P.start + nx];
                    v_next = f[perm[P.start + nx]];
                }
            }
            for (int k = oct; k < cnt; k += kOctets) {
                const Rec r = st_rec[k];
                const C v = st_val[k];
                const int loc1 = (r.cell & g.cmask[1]) - org1;
                const int loc0 = ((r.cell >> g.cbits[1]) & g.cmask[0]) - org0;
                const T fr0 = r.fr[0], fr1 = r.fr[1];
                if (fr0 == (T)0 || fr1 == (T)0)  // uniform inside the group (one node)
                    spread_octet_node<T, MM, 0>(mine, td1, loc0 * td1 + loc1, fr0, fr1, ca, ea,
                                                cb, eb, v, l, mask, la, lb, g.lin_k);
                else
                    spread_octet_node<T, MM, 1>(mine, td1, (loc0 + 1) * td1 + loc1 + 1, fr0,
                                                fr1, ca, ea, cb, eb, v, l, mask, la, lb, g.lin_k);
                __syncwarp(mask);
            }
            __syncthreads();
        }

        // flush: cell (a0, a1) of the tile is grid point ((org0 - m + a0) mod n0,
        // (org1 - m + a1) mod n1); one warp per tile row, lanes along the row
        for (int a0 = warp; a0 < td0; a0 += kSpreadWarps) {
            const size_t gbase = (size_t)wrapn(org0 - MM + a0, g.n[0]) * g.n[1];
            for (int a1 = lane; a1 < td1; a1 += 32) {
                const int e = a0 * td1 + a1;
                T vr = (T)0, vi = (T)0;
#pragma unroll 8
                for (int o = 0; o < kOctets; o++) {
                    const C c = tiles[(size_t)o * tstride + e];
                    vr += c.x;
                    vi += c.y;
                }
                if (vr == (T)0 && vi == (T)0) continue;
                global_add(grid + (gbase + (size_t)wrapn(org1 - MM + a1, g.n[1])), vr, vi);
            }
        }
        __syncthreads();
    }
    finish_subproblems(nsub_total);
}

// ------------------------------------------------------------------------ half-warp form (d = 2)
// Sixteen lanes per node, two nodes per warp, one private complex tile per half-warp. The lanes
// of a half form RG row groups x CW columns (CW = the 2m taps per axis rounded up to a power of
// two); lane (rg, c) owns tap column c and tap rows rg, rg + RG, ... of its node. The window
// weights are evaluated once per node, by the thread that stages the node (all taps of an axis
// at once, mirrored pairs sharing one polynomial evaluation): the row weights are staged in the
// order the row groups read them (one vector load per lane), the column weights already times
// the node value. A node on a grid point of an axis has 2m + 1 taps on that axis: taps 1 .. 2m
// as for any node, and tap 0 (weight edge_w) one cell before them; the window stays a product
// over the axes, so the extra row and column of taps take one more read-modify-write per lane.
// The tile row pitch is padded so that the row groups of one half fall on distinct banks.
//
// The CTAs are small (kHalfWarps warps): the flush reads every private tile of the CTA at every
// cell, so its shared-memory traffic per subproblem grows with the number of tiles per CTA,
// while small CTAs keep the same number of warps per SM. The flush zeroes the tiles as it reads
// them, so a tile is cleared once at kernel start and then stays clean between subproblems.
#ifndef GBNFFT_HALF_WARPS
#define GBNFFT_HALF_WARPS 2
#endif
constexpr int kHalfWarps = GBNFFT_HALF_WARPS;
constexpr int kHalfTiles = 2 * kHalfWarps;     // half-warps (and private tiles) per CTA
constexpr int kHalfChunk = 32 * kHalfWarps;    // nodes staged per round (one per thread)

template <int MM> struct HalfShape {
    static constexpr int PER = 2 * MM;
    static constexpr int CW = PER <= 2 ? 2 : PER <= 4 ? 4 : PER <= 8 ? 8 : 16;
    static constexpr int RG = 16 / CW;
    static constexpr int ROWS = (PER + RG - 1) / RG;
    static constexpr int RP = ROWS == 1 ? 1 : ((ROWS + 3) & ~3);  // staged row weights per group
    static constexpr int RW = RG * RP;                             // staged row weights per node
};

// Row pitch (in cells) of a half-warp tile whose rows hold td1 cells: one half touches RG rows
// of CW contiguous cells per access; a pitch of CW cells modulo one 128-byte bank cycle puts
// those RG runs side by side in the banks. Runs that fill a bank cycle need no padding.
template <typename T, int MM> __host__ __device__ inline int half_pitch(int td1)
{
    constexpr int cw = HalfShape<MM>::CW;
    constexpr int cplx = 2 * (int)sizeof(T);
    constexpr int mod = 128 / cplx;  // cells per bank cycle
    if (HalfShape<MM>::RG == 1 || cw * cplx >= 128) return td1;
    return td1 + ((cw - td1 % mod) + mod) % mod;
}

// One staged chunk of the half-warp form, per node k < kHalfChunk:
//   info[k]  tile offset of the node's tap (1, 1) | grid-point flags << 28 (bit t: frac_t = 0,
//            so tap 0 of axis t is live)
//   val[k]   the node value
//   row[k * RW + g * RP + j]   the weight of tap row g + j * RG + 1 (row group g reads RP in a row)
//   col[k * CW + (c ^ swz(k))] the weight of tap column c + 1 times the node value; the index is
//            swizzled (swz(k) = (k / 2) mod CW) so that the stores of one thread per node and
//            the loads of two nodes per warp both spread over the banks
template <typename T, int MM> struct HalfStageLayout {
    using Sh = HalfShape<MM>;
    static constexpr size_t info = 0;
    static constexpr size_t val = ((size_t)kHalfChunk * sizeof(int) + 15) / 16 * 16;
    static constexpr size_t row = val + (size_t)kHalfChunk * 2 * sizeof(T);
    static constexpr size_t col = row + ((size_t)kHalfChunk * Sh::RW * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t bytes = col + (size_t)kHalfChunk * Sh::CW * 2 * sizeof(T);
};

template <typename T, int MM>
__host__ __device__ constexpr size_t half_stage_bytes()
{
    return HalfStageLayout<T, MM>::bytes;
}

// Shared memory of the half-warp form: the staged chunk of nodes first, then the kHalfTiles
// private tiles (td0 rows of `pitch` cells each).
template <typename T, int MM>
__device__ __forceinline__ typename Cplx<T>::type *half_tiles(unsigned char *smem)
{
    return reinterpret_cast<typename Cplx<T>::type *>(smem + half_stage_bytes<T, MM>());
}

// One subproblem of the half-warp form: the CTA stages its nodes a chunk at a time, every
// half-warp adds one node after another into its private tile, and the flush adds the CTA's
// tiles into the grid and zeroes them. `coef` is the polynomial window table of axis 0 (axis 1
// follows it; unused with the lookup-table window).
template <typename T, int MM, bool LIN>
__device__ __forceinline__ void half_subproblem(
    const Geom &g, const SubProb &P, const typename Cplx<T>::type *__restrict__ f,
    const typename RecOf<T>::type *__restrict__ rec, const int *__restrict__ perm,
    typename Cplx<T>::type *__restrict__ grid, unsigned char *smem, const T *__restrict__ coef)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    using Sh = HalfShape<MM>;
    using Lay = HalfStageLayout<T, MM>;
    constexpr int PER = Sh::PER, CW = Sh::CW, RG = Sh::RG, ROWS = Sh::ROWS;
    constexpr int RP = Sh::RP, RW = Sh::RW;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    const int tid = threadIdx.x, lane = tid & 31;
    const int h = lane & 15, half = tid >> 4;
    const unsigned mask = 0xffffu << (lane & 16);
    const int c = h & (CW - 1), rg = h / CW;
    const int td0 = g.bs[0] + 2 * MM, td1 = g.bs[1] + 2 * MM;
    const int pitch = half_pitch<T, MM>(td1);
    const int tcells = td0 * pitch;
    int *st_info = reinterpret_cast<int *>(smem + Lay::info);
    C *st_val = reinterpret_cast<C *>(smem + Lay::val);
    T *st_row = reinterpret_cast<T *>(smem + Lay::row);
    C *st_col = reinterpret_cast<C *>(smem + Lay::col);
    C *tiles = half_tiles<T, MM>(smem);
    C *mine = tiles + (size_t)half * tcells;
    C *const lane_col = mine + rg * pitch + c;
    const T e0 = (T)g.win[0].edge_w, e1 = (T)g.win[1].edge_w;
    const int org1 = (P.bin % g.nb[1]) * g.bs[1];
    const int org0 = (P.bin / g.nb[1]) * g.bs[0];
    Rec r_next;
    C v_next;
    if (tid < P.count) {
        r_next = rec[P.start + tid];
        v_next = f[perm[P.start + tid]];
    }
    for (int c0 = 0; c0 < P.count; c0 += kHalfChunk) {
        const int cnt = min(kHalfChunk, P.count - c0);
        if (tid < cnt) {  // stage this thread's node: tile offset, weights, value
            const int loc1 = (r_next.cell & g.cmask[1]) - org1;
            const int loc0 = ((r_next.cell >> g.cbits[1]) & g.cmask[0]) - org0;
            const T fr0 = r_next.fr[0], fr1 = r_next.fr[1];
            T w0[2 * MM + 1], w1[2 * MM + 1];  // taps 1 .. 2m of each axis
            if constexpr (LIN) {
                lin_taps<T, MM, 1>(lin_axis<T, MM>(g.lin, g.lin_k, 0), g.lin_k, fr0, e0, w0);
                lin_taps<T, MM, 1>(lin_axis<T, MM>(g.lin, g.lin_k, 1), g.lin_k, fr1, e1, w1);
            } else {
                window_taps<T, MM, 1>(coef, fr0, e0, w0);
                window_taps<T, MM, 1>(coef + AS, fr1, e1, w1);
            }
            const int gp = (fr0 == (T)0 ? 1 : 0) | (fr1 == (T)0 ? 2 : 0);
            st_info[tid] = ((loc0 + 1) * pitch + loc1 + 1) | (gp << 28);
            st_val[tid] = v_next;
            T *rw = st_row + tid * RW;
#pragma unroll
            for (int q = 0; q < RW; q++) {
                const int rr = q / RP + (q % RP) * RG;
                rw[q] = rr < PER ? w0[rr + 1] : (T)0;
            }
            C *cw = st_col + tid * CW;
            const int sw = (tid >> 1) & (CW - 1);
#pragma unroll
            for (int q = 0; q < PER; q++) {
                C a;
                a.x = w1[q + 1] * v_next.x;
                a.y = w1[q + 1] * v_next.y;
                cw[q ^ sw] = a;
            }
        }
        __syncthreads();  // (also orders the previous flush's zeroing before these adds)
        {
            const int nx = c0 + kHalfChunk + tid;
            if (nx < P.count) {
                r_next = rec[P.start + nx];
                v_next = f[perm[P.start + nx]];
            }
        }
        for (int k = half; k < cnt; k += kHalfTiles) {
            const int info = st_info[k];
            const C cv = st_col[k * CW + (c ^ ((k >> 1) & (CW - 1)))];
            T w0r[RP];
#pragma unroll
            for (int j = 0; j < RP; j++) w0r[j] = st_row[k * RW + rg * RP + j];
            const int off = info & 0x0fffffff;
            C *col = lane_col + off;
#pragma unroll
            for (int j = 0; j < ROWS; j++) {
                const int rr = rg + j * RG;
                if (c < PER && rr < PER) {
                    C a = col[j * RG * pitch];
                    a.x += w0r[j] * cv.x;
                    a.y += w0r[j] * cv.y;
                    col[j * RG * pitch] = a;
                }
            }
            const int gp = info >> 28;
            if (gp != 0 && h < PER) {  // uniform inside the half: a node on a grid point
                C *base = mine + off;
                if (gp & 1) {  // row tap 0 of axis 0 over the column taps 1 .. 2m (c == h)
                    C *p = base - pitch + h;
                    C a = *p;
                    a.x += e0 * cv.x;
                    a.y += e0 * cv.y;
                    *p = a;
                }
                if (gp & 2) {  // column tap 0 of axis 1 over the row taps 1 .. 2m
                    const C v = st_val[k];
                    const T w = st_row[k * RW + (h % RG) * RP + h / RG] * e1;
                    C *p = base + h * pitch - 1;
                    C a = *p;
                    a.x += w * v.x;
                    a.y += w * v.y;
                    *p = a;
                }
                if (gp == 3 && h == 0) {  // the corner: tap 0 of both axes
                    const C v = st_val[k];
                    const T w = e0 * e1;
                    C *p = base - pitch - 1;
                    C a = *p;
                    a.x += w * v.x;
                    a.y += w * v.y;
                    *p = a;
                }
            }
            __syncwarp(mask);
        }
        __syncthreads();
    }

    // flush: cell (a0, a1) of the tile is grid point ((org0 - m + a0) mod n0,
    // (org1 - m + a1) mod n1); consecutive threads take consecutive cells; each cell is read
    // from every tile and zeroed there
    C z;
    z.x = (T)0;
    z.y = (T)0;
    constexpr int kStep = 32 * kHalfWarps;
    const int dq = kStep / td1, dr = kStep - dq * td1;
    int a0 = tid / td1, a1 = tid - a0 * td1;
    for (int idx = tid; idx < td0 * td1; idx += kStep) {
        const int e = a0 * pitch + a1;
        T vr = (T)0, vi = (T)0;
#pragma unroll
        for (int o = 0; o < kHalfTiles; o++) {
            const C cv = tiles[(size_t)o * tcells + e];
            tiles[(size_t)o * tcells + e] = z;
            vr += cv.x;
            vi += cv.y;
        }
        if (vr != (T)0 || vi != (T)0) {
            const size_t gi = (size_t)wrapn(org0 - MM + a0, g.n[0]) * g.n[1] +
                              (size_t)wrapn(org1 - MM + a1, g.n[1]);
            global_add(grid + gi, vr, vi);
        }
        a0 += dq;  // (a0, a1) = the cell of idx + kStep
        a1 += dr;
        if (a1 >= td1) {
            a1 -= td1;
            a0++;
        }
    }
}

template <typename T, int MM, bool LIN>
__global__ void __launch_bounds__(32 * kHalfWarps)
    spread_half_kernel(Geom g, const __grid_constant__ WinCoef<T, MM> wc,
                       const typename Cplx<T>::type *__restrict__ f,
                       const typename RecOf<T>::type *__restrict__ rec,
                       const int *__restrict__ perm, const SubProb *__restrict__ subs,
                       int *__restrict__ nsub_total, typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    {
        const int tcells = (g.bs[0] + 2 * MM) * half_pitch<T, MM>(g.bs[1] + 2 * MM);
        C *tiles = half_tiles<T, MM>(smem_raw);
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int e = threadIdx.x; e < kHalfTiles * tcells; e += 32 * kHalfWarps) tiles[e] = z;
    }
    const int nsub = nsub_total[0];
    __shared__ int s_sp;
    for (int sp = next_subproblem(nsub_total, &s_sp); sp < nsub;
         sp = next_subproblem(nsub_total, &s_sp))
        half_subproblem<T, MM, LIN>(g, subs[sp], f, rec, perm, grid, smem_raw, wc.c);
    finish_subproblems(nsub_total);
}

// ------------------------------------------------------------------------------ rows form (d = 2)
// No shared-memory tile at all: a group of G lanes (a half-warp when the tile is at most 16
// cells wide, else the whole warp) keeps one subproblem's whole tile in registers. Lane c of
// the group owns column c of the tile (bin + 2m halo along the last axis) and all td0 = b0 + 2m
// tile rows of that column. Each node's window values are computed once, by the lane that
// stages it: the column weights times the node value, and the row weights already placed at
// the node's tile rows in a zero-filled column of td0 values. A node then costs every lane of
// the group one multiply-add per tile row, with no branch on the node's position, and a few
// shared-memory loads (instead of a read-modify-write per tap, which bounds the tile forms on
// the shared-memory pipe). Tap 0 of an axis is nonzero only on a grid point. The two
// half-warps of a warp take consecutive subproblems; at the end of a subproblem every nonzero
// cell is added into the grid once (one vector atomic). The warps are independent: each claims
// its own subproblems from the plan's work counter.
constexpr int kRowsWarps = 4;

template <typename T, int MM, int BS0, int G> struct RowsShape {
    static constexpr int NT = 2 * MM + 1;                          // taps per axis
    static constexpr int TD0 = BS0 + 2 * MM;                       // tile rows (registers)
    static constexpr int TDP = (TD0 * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
    static constexpr int GROUPS = 32 / G;                          // subproblems per warp
    // per group: G nodes staged, each TDP row values, NT column values, one column offset;
    // a group stride that is not a multiple of 128 bytes keeps the two groups' loads of one
    // instruction on different banks
    static constexpr size_t raw = (size_t)G * (TDP * sizeof(T) +
                                              NT * sizeof(typename Cplx<T>::type) + sizeof(int));
    static constexpr size_t raw16 = (raw + 15) / 16 * 16;
    static constexpr size_t group = raw16 + (raw16 % 128 == 0 ? 16 : 0);
    static constexpr size_t per_warp = group * GROUPS;
};

// n values from 16-byte aligned shared memory (n a multiple of 16 / sizeof(T))
template <typename T, int N>
__device__ __forceinline__ void load_aligned16(const T *p, T *w)
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + i);
            w[i] = v.x;
            w[i + 1] = v.y;
            w[i + 2] = v.z;
            w[i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const double2 v = *reinterpret_cast<const double2 *>(p + i);
            w[i] = v.x;
            w[i + 1] = v.y;
        }
    }
}

// Staging area of one group of the rows form (G nodes).
template <typename T, int MM, int BS0, int G> struct RowsStage {
    using C = typename Cplx<T>::type;
    using Sh = RowsShape<T, MM, BS0, G>;
    T *w0;   // [G][TDP] row weights at the node's tile rows
    C *cv;   // [G][NT] column weights times the node value
    int *at; // [G] the node's first tile column
    __device__ __forceinline__ RowsStage(unsigned char *base)
        : w0(reinterpret_cast<T *>(base)),
          cv(reinterpret_cast<C *>(base + G * Sh::TDP * sizeof(T))),
          at(reinterpret_cast<int *>(base + G * (Sh::TDP * sizeof(T) + Sh::NT * sizeof(C))))
    {
    }
};

// One subproblem P of one group (gl = the lane's index in its group): `most` is the larger
// node count of the warp's two subproblems (the warp runs that many rounds; the group with
// fewer nodes idles at the end). Every lane of the warp calls it. `coef` is the polynomial
// window table of axis 0 (axis 1 follows it).
template <typename T, int MM, int MODE, int BS0, int G>
__device__ __forceinline__ void rows_subproblem(
    const Geom &g, const T *__restrict__ coef, const SubProb &P, int most,
    const typename Cplx<T>::type *__restrict__ f, const typename RecOf<T>::type *__restrict__ rec,
    const int *__restrict__ perm, typename Cplx<T>::type *__restrict__ grid,
    const RowsStage<T, MM, BS0, G> &st, int gl)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    using Sh = RowsShape<T, MM, BS0, G>;
    constexpr int NT = Sh::NT, TD0 = Sh::TD0, TDP = Sh::TDP;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    const int org1 = (P.bin % g.nb[1]) * g.bs[1];
    const int org0 = (P.bin / g.nb[1]) * g.bs[0];
    C acc[TD0];
#pragma unroll
    for (int j = 0; j < TD0; j++) {
        acc[j].x = (T)0;
        acc[j].y = (T)0;
    }
    Rec nr;  // this lane's node of the next round, loaded one round ahead
    C nv;
    if (gl < P.count) {
        nr = rec[P.start + gl];
        nv = f[perm[P.start + gl]];
    }
    for (int k0 = 0; k0 < most; k0 += G) {
        const int cnt = min(G, P.count - k0);  // this group's nodes in this round (may be <= 0)
        if (gl < cnt) {  // stage this lane's node
            const Rec r = nr;
            const C v = nv;
            if (k0 + G + gl < P.count) {
                const int s = P.start + k0 + G + gl;
                nr = rec[s];
                nv = f[perm[s]];
            }
            const int loc1 = (r.cell & g.cmask[1]) - org1;
            const int loc0 = ((r.cell >> g.cbits[1]) & g.cmask[0]) - org0;
            T w0[NT], w1[NT];
            eval_taps<T, MM, 0, MODE>(g, coef, 0, r.fr[0], w0);
            eval_taps<T, MM, 0, MODE>(g, coef + AS, 1, r.fr[1], w1);
            T *wr = st.w0 + gl * TDP;  // tile rows loc0 .. loc0 + 2m, zeros elsewhere
#pragma unroll
            for (int j = 0; j < TDP; j++) wr[j] = (T)0;
#pragma unroll
            for (int t = 0; t < NT; t++) wr[loc0 + t] = w0[t];
#pragma unroll
            for (int t = 0; t < NT; t++) {
                C q;
                q.x = w1[t] * v.x;
                q.y = w1[t] * v.y;
                st.cv[gl * NT + t] = q;
            }
            st.at[gl] = loc1;
        }
        __syncwarp();
        const int cm = min(G, most - k0);
        // one node of the round (the two groups differ only at the end of the smaller one)
        auto add_node = [&](int k) {
            if (k < cnt) {
                const int t = gl - st.at[k];  // this column's tap of the node
                const bool in = (unsigned)t < (unsigned)NT;
                const C cv = st.cv[k * NT + (in ? t : 0)];
                const T cr = in ? cv.x : (T)0, ci = in ? cv.y : (T)0;
                T w[TDP];
                load_aligned16<T, TDP>(st.w0 + k * TDP, w);
#pragma unroll
                for (int j = 0; j < TD0; j++) {
                    acc[j].x = fma(w[j], cr, acc[j].x);
                    acc[j].y = fma(w[j], ci, acc[j].y);
                }
            }
        };
        int k = 0;
        for (; k + 2 <= cm; k += 2) {
            add_node(k);
            add_node(k + 1);
        }
        if (k < cm) add_node(k);
        __syncwarp();
    }
    // tile cell (j, gl) is grid point ((org0 - m + j) mod n0, (org1 - m + gl) mod n1)
    if (P.count > 0 && gl < g.bs[1] + 2 * MM) {
        const size_t gcol = (size_t)wrapn(org1 - MM + gl, g.n[1]);
#pragma unroll
        for (int j = 0; j < TD0; j++)
            if (acc[j].x != (T)0 || acc[j].y != (T)0)
                global_add(grid + (size_t)wrapn(org0 - MM + j, g.n[0]) * g.n[1] + gcol,
                           acc[j].x, acc[j].y);
    }
}

// Per-warp claims of the rows form: lane 0 takes GROUPS consecutive entries of the list at a
// time (work[1] the next unclaimed entry); the last warp to finish puts work[1] and work[2] back
// to zero for the next launch.
__device__ __forceinline__ int rows_claim(int *work, int groups)
{
    int sp0 = 0;
    if ((threadIdx.x & 31) == 0) sp0 = atomicAdd(work + 1, groups);
    return __shfl_sync(0xffffffffu, sp0, 0);
}

__device__ __forceinline__ void rows_finish(int *work)
{
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        if (atomicAdd(work + 2, 1) == (int)(gridDim.x * (blockDim.x >> 5)) - 1) {
            work[1] = 0;
            work[2] = 0;
        }
    }
}

template <typename T, int MM, bool LIN, int BS0, int G>
__global__ void __launch_bounds__(32 * kRowsWarps)
    spread_rows_kernel(Geom g, const __grid_constant__ WinCoef<T, MM> wc,
                       const typename Cplx<T>::type *__restrict__ f,
                       const typename RecOf<T>::type *__restrict__ rec,
                       const int *__restrict__ perm, const SubProb *__restrict__ subs,
                       int *__restrict__ work, typename Cplx<T>::type *__restrict__ grid)
{
    using Sh = RowsShape<T, MM, BS0, G>;
    constexpr int GROUPS = Sh::GROUPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const RowsStage<T, MM, BS0, G> st(smem_raw + (size_t)warp * Sh::per_warp +
                                      (size_t)grp * Sh::group);
    const int nsub = work[0];
    auto entry = [&](int sp0) {  // this group's entry of a claim (empty past the list)
        SubProb P;
        P.bin = 0;
        P.start = 0;
        P.count = 0;
        if (sp0 + grp < nsub) P = subs[sp0 + grp];
        return P;
    };
    int sp0 = rows_claim(work, GROUPS);
    SubProb P = entry(sp0);
    while (sp0 < nsub) {
        const int sp0n = rows_claim(work, GROUPS);  // the next claim, read while this one runs
        const SubProb Pn = entry(sp0n);
        int most = P.count;
        if constexpr (GROUPS == 2) most = max(most, __shfl_xor_sync(0xffffffffu, most, 16));
        rows_subproblem<T, MM, LIN ? 2 : 1, BS0, G>(g, wc.c, P, most, f, rec, perm, grid, st, gl);
        sp0 = sp0n;
        P = Pn;
    }
    rows_finish(work);
}

// ----------------------------------------------------------------------------- plane form (d = 3)
// One shared tile per CTA, no atomics and no private copies: the eight warps own the tile's
// planes along axis 0 by residue (warp w adds into the planes a0 with a0 mod 8 = w), and every
// warp walks every node of the subproblem, adding the taps of the node that fall into its own
// planes. A node's support spans 2m consecutive planes, so for m = 4 each warp takes exactly one
// plane (2m x 2m taps, two rounds of its lanes) of every node, and no two warps ever touch the
// same cell. The window values, which every warp would otherwise evaluate again, are computed
// once per node when a chunk of nodes is staged (three threads per node, one per axis): the
// axis-1 and axis-2 values, the axis-0 values times f_j, and the tile offset of the node's first
// tap. Lanes cover a plane row-major (last axis fastest); the row pitch puts the rows written in
// one round side by side in the banks.
constexpr int kPlaneWarps = 8;
constexpr int kPlaneChunk = 64;  // nodes staged at a time

// Row pitch (cells) of the plane tile: for FP32 with 2m = 8 an access of 16 lanes covers 2 rows
// of 8 cells, which share a 128-byte wavefront when the pitch is 8 mod 16 cells. FP64 rows of 8
// cells fill a wavefront by themselves.
template <typename T> __host__ __device__ inline int plane_pitch(int td2)
{
    if (sizeof(T) == 8) return td2;
    return td2 + ((8 - td2 % 16) + 16) % 16;
}

// Staged data per node: a packed offset word, NT complex axis-0 terms and 2 NT + 1 reals
// (axis-1 values, axis-2 values, one pad to an odd stride).
template <typename T, int MM>
__host__ __device__ constexpr size_t plane_stage_bytes()
{
    return kPlaneChunk * (sizeof(unsigned) + (2 * MM + 1) * sizeof(typename Cplx<T>::type) +
                          (4 * MM + 3) * sizeof(T)) +
           16;
}

// The taps of one node in the planes i0, i0 + 8, ... (< P) of one warp: P x P taps per plane,
// weight w_0(i0) f_j (staged in ak) times w_1(i1) w_2(i2) (staged in wk).
template <typename T, int MM, int START>
__device__ __forceinline__ void plane_taps(typename Cplx<T>::type *first, int i0, int pstride,
                                           int pitch, const T *wk,
                                           const typename Cplx<T>::type *ak, int lane)
{
    using C = typename Cplx<T>::type;
    constexpr int NT = 2 * MM + 1;
    constexpr int P = NT - START;
    constexpr int TAPS = P * P;
    constexpr int ITER = (TAPS + 31) / 32;
    for (; i0 < P; i0 += kPlaneWarps) {
        const C A = ak[i0 + START];
        C *row0 = first + i0 * pstride;
        if constexpr (32 % P == 0) {  // the lane's column is the same in every round
            const int i2 = lane % P;
            const T w2 = wk[NT + i2 + START];
            const T br = w2 * A.x, bi = w2 * A.y;
#pragma unroll
            for (int k = 0; k < ITER; k++) {
                const int i1 = lane / P + k * (32 / P);
                if (i1 < P) {
                    const T w1 = wk[i1 + START];
                    C *p = row0 + i1 * pitch + i2;
                    C a = *p;
                    a.x += w1 * br;
                    a.y += w1 * bi;
                    *p = a;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < ITER; k++) {
                const int q = lane + 32 * k;
                if (q < TAPS) {
                    const int i1 = q / P, i2 = q - (q / P) * P;
                    const T w = wk[i1 + START] * wk[NT + i2 + START];
                    C *p = row0 + i1 * pitch + i2;
                    C a = *p;
                    a.x += w * A.x;
                    a.y += w * A.y;
                    *p = a;
                }
            }
        }
    }
}

template <typename T, int MM, bool LIN>
__global__ void __launch_bounds__(32 * kPlaneWarps)
    spread_plane_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                        const typename RecOf<T>::type *__restrict__ rec,
                        const int *__restrict__ perm, const SubProb *__restrict__ subs,
                        int *__restrict__ nsub_total, typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    constexpr int NT = 2 * MM + 1;  // tap slots per axis (slot 0 only on a grid point)
    constexpr int SW = 2 * NT + 1;  // staged reals per node
    constexpr int MODE = LIN ? 2 : 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    static_assert(32 * kPlaneWarps >= 3 * kPlaneChunk, "three staging threads per node");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) T tab[kMaxDim * AS];
    load_window_tables<T, MM>(tab, g.poly, 3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int s_ax = tid / kPlaneChunk, s_nd = tid - s_ax * kPlaneChunk;  // staging role
    const int td0 = g.bs[0] + 2 * MM, td1 = g.bs[1] + 2 * MM, td2 = g.bs[2] + 2 * MM;
    const int pitch = plane_pitch<T>(td2);
    const int pstride = td1 * pitch;
    const int tcells = td0 * pstride;
    C *tile = reinterpret_cast<C *>(smem_raw);
    C *st_a = reinterpret_cast<C *>(smem_raw + ((size_t)tcells * sizeof(C) + 15) / 16 * 16);
    T *st_w = reinterpret_cast<T *>(st_a + kPlaneChunk * NT);
    unsigned *st_pk = reinterpret_cast<unsigned *>(st_w + kPlaneChunk * SW);
    {
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int e = tid; e < tcells; e += 32 * kPlaneWarps) tile[e] = z;
    }
    const int nsub = nsub_total[0];
    __shared__ int s_sp;
    for (int sp = next_subproblem(nsub_total, &s_sp); sp < nsub;
         sp = next_subproblem(nsub_total, &s_sp)) {
        const SubProb P = subs[sp];
        int org[3];
        {
            int b = P.bin;
#pragma unroll
            for (int t = 2; t >= 0; t--) {
                org[t] = (b % g.nb[t]) * g.bs[t];
                b /= g.nb[t];
            }
        }
        // staging: thread (axis s_ax < 3, node s_nd) evaluates one axis of one node
        Rec r_next;
        C v_next;
        if (s_ax < 3 && s_nd < P.count) {
            r_next = rec[P.start + s_nd];
            if (s_ax == 0) v_next = f[perm[P.start + s_nd]];
        }
        for (int c0 = 0; c0 < P.count; c0 += kPlaneChunk) {
            const int cnt = min(kPlaneChunk, P.count - c0);
            if (s_ax < 3 && s_nd < cnt) {
                int cell = r_next.cell;
                const int loc2 = (cell & g.cmask[2]) - org[2];
                cell >>= g.cbits[2];
                const int loc1 = (cell & g.cmask[1]) - org[1];
                cell >>= g.cbits[1];
                const int loc0 = (cell & g.cmask[0]) - org[0];
                const T fr0 = r_next.fr[0], fr1 = r_next.fr[1], fr2 = r_next.fr[2];
                const int start = (fr0 == (T)0 || fr1 == (T)0 || fr2 == (T)0) ? 0 : 1;
                const T frt = s_ax == 0 ? fr0 : (s_ax == 1 ? fr1 : fr2);
                T w[NT];
                if (start) {
                    eval_taps<T, MM, 1, MODE>(g, tab + s_ax * AS, s_ax, frt, w);
                    w[0] = (T)0;
                } else {
                    eval_taps<T, MM, 0, MODE>(g, tab + s_ax * AS, s_ax, frt, w);
                }
                if (s_ax > 0) {
                    T *dst = st_w + s_nd * SW + (s_ax - 1) * NT;
#pragma unroll
                    for (int i = 0; i < NT; i++) dst[i] = w[i];
                } else {
                    C *a = st_a + s_nd * NT;
#pragma unroll
                    for (int i = 0; i < NT; i++) {
                        C t;
                        t.x = w[i] * v_next.x;
                        t.y = w[i] * v_next.y;
                        a[i] = t;
                    }
                    const unsigned first =
                        (unsigned)(((loc0 + start) * td1 + loc1 + start) * pitch + loc2 + start);
                    st_pk[s_nd] = first | ((unsigned)((loc0 + start) & 7) << 28) |
                                  ((unsigned)start << 31);
                }
            }
            __syncthreads();  // (also orders the previous flush's zeroing before these adds)
            {
                const int nx = c0 + kPlaneChunk + s_nd;  // prefetch the next chunk
                if (s_ax < 3 && nx < P.count) {
                    r_next = rec[P.start + nx];
                    if (s_ax == 0) v_next = f[perm[P.start + nx]];
                }
            }
            for (int k = 0; k < cnt; k++) {
                const unsigned pk = st_pk[k];
                const int start = (int)(pk >> 31);
                // the planes of this warp: a0 = (first plane) + i0 with a0 mod 8 = warp
                const int i0 = (warp - (int)((pk >> 28) & 7u)) & (kPlaneWarps - 1);
                C *first = tile + (pk & 0x0fffffffu);
                if (start)
                    plane_taps<T, MM, 1>(first, i0, pstride, pitch, st_w + k * SW, st_a + k * NT,
                                         lane);
                else
                    plane_taps<T, MM, 0>(first, i0, pstride, pitch, st_w + k * SW, st_a + k * NT,
                                         lane);
                __syncwarp();
            }
            __syncthreads();
        }

        // flush: cell (a0, a1, a2) of the tile is grid point ((org_t - m + a_t) mod n_t);
        // consecutive lanes take consecutive cells of a row; each cell is zeroed after reading
        C z;
        z.x = (T)0;
        z.y = (T)0;
        const int rows = td0 * td1;
        for (int row = warp; row < rows; row += kPlaneWarps) {
            const int a0 = row / td1, a1 = row - a0 * td1;
            const size_t gbase = ((size_t)wrapn(org[0] - MM + a0, g.n[0]) * g.n[1] +
                                  (size_t)wrapn(org[1] - MM + a1, g.n[1])) *
                                 g.n[2];
            for (int a2 = lane; a2 < td2; a2 += 32) {
                C *p = tile + (size_t)row * pitch + a2;
                const C cv = *p;
                if (cv.x == (T)0 && cv.y == (T)0) continue;
                *p = z;
                global_add(grid + gbase + (size_t)wrapn(org[2] - MM + a2, g.n[2]), cv.x, cv.y);
            }
        }
    }
    finish_subproblems(nsub_total);
}

// ---------------------------------------------------------------------------- stripe form (d = 2)
// One shared tile per CTA and no private copies. The tile covers a super-bin: kStripeS stripes
// side by side along the last axis, each stripe_width(m) = W >= 2m cells wide (a whole number of
// sort bins) and one sort bin high, plus the halo of m cells. A node of stripe j adds into tile
// columns W j + 1 ... W j + W - 1 + 2m (W j ... on a grid point), so stripes j and j + 2 never
// touch a common cell: the CTA's kStripeHalves half-warps take the even stripes together, then,
// after a barrier, the odd ones. A half-warp walks the sorted nodes of its stripe sixteen at a
// time: lane h stages node h (its tile offset, z = 2 frac - 1 per axis, its value), then the
// sixteen lanes add every staged node with the lane layout of the half-warp form (lane (rg, c):
// tap column c, tap rows rg, rg + RG, ...; row weights by shuffles). A work item is
// (super-bin, part p of P): part p takes the p-th P-th of every stripe's node range, P sized so
// that no stripe's part exceeds the item size (a half-warp walks its part node after node, so the
// heaviest stripe sets an item's duration). The flush adds the tile into the grid (one vector
// atomic per nonzero cell) and zeroes it; the tile is cleared once at kernel start.
template <int MM> struct StripeShape {
    static constexpr int W = stripe_width(MM);
    static constexpr int TD1 = kStripeS * W + 2 * MM;
};

// Row pitch (cells) of the stripe tile: the half-warp's RG rows of CW cells fall side by side in
// the banks (as half_pitch).
template <typename T, int MM> __host__ __device__ constexpr int stripe_pitch()
{
    constexpr int td1 = StripeShape<MM>::TD1;
    constexpr int cw = HalfShape<MM>::CW;
    constexpr int mod = 128 / (2 * (int)sizeof(T));
    return (HalfShape<MM>::RG == 1 || cw * 2 * (int)sizeof(T) >= 128)
               ? td1
               : td1 + ((cw - td1 % mod) + mod) % mod;
}

// Staged per node: tile offset of the first tap (bit 31 set: the node is on a grid point; the
// low bits then give the offset of tap slot 0), its sorted index, and the window arguments
// (z = 2 frac - 1, or frac itself for the lookup-table window).
template <typename T> struct alignas(16) StripeStage {
    int off;
    int s;
    T u0, u1;
};

template <typename T, int MM>
__host__ __device__ constexpr size_t stripe_smem_bytes(int td0)
{
    return (size_t)td0 * stripe_pitch<T, MM>() * sizeof(typename Cplx<T>::type) +
           (size_t)kStripeHalves * 16 * (sizeof(StripeStage<T>) + sizeof(typename Cplx<T>::type));
}

// Window values of the stripe form: with 2 * 2m <= 16 (m <= 4) every lane of a half-warp holds
// the polynomial of one tap (lanes h < 2m: tap h + 1 of the last axis, the next 2m lanes: tap
// h - 2m + 1 of the first axis), evaluates it once per node and the lanes exchange the values by
// shuffles; for larger m each lane evaluates its column tap and one row tap.
template <int MM> struct StripeWin {
    static constexpr bool ONE = 4 * MM <= 16;
};

template <typename T, int MM, bool LIN>
__global__ void __launch_bounds__(32 * kStripeWarps, (StripeWin<MM>::ONE && MM > 1) ? 10 : 8)
    spread_stripe_kernel(Geom g, const typename Cplx<T>::type *__restrict__ f,
                         const typename RecOf<T>::type *__restrict__ rec,
                         const int *__restrict__ perm, typename Cplx<T>::type *__restrict__ grid)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    using Sh = HalfShape<MM>;
    constexpr int PER = Sh::PER, CW = Sh::CW, RG = Sh::RG, ROWS = Sh::ROWS;
    constexpr int NT = 2 * MM + 1;
    constexpr int AS = poly_axis_stride(sizeof(T) == 8, MM);
    constexpr int DEG = PolyDeg<T, MM>::value;
    constexpr int TD1 = StripeShape<MM>::TD1;
    constexpr int SW = StripeShape<MM>::W;
    constexpr int PITCH = stripe_pitch<T, MM>();
    constexpr bool ONE = StripeWin<MM>::ONE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int2 s_rng[kStripeS];
    __shared__ int s_sp;
    const T *tab = static_cast<const T *>(g.poly);
    const int tid = threadIdx.x, lane = tid & 31;
    const int h = lane & 15, half = tid >> 4;
    const unsigned mask = 0xffffu << (lane & 16);
    const int c = h & (CW - 1), rg = h / CW;
    const int td0 = g.bs[0] + 2 * MM;
    const int cells = td0 * TD1;
    C *tile = reinterpret_cast<C *>(smem_raw);
    StripeStage<T> *stage = reinterpret_cast<StripeStage<T> *>(
        smem_raw + (size_t)td0 * PITCH * sizeof(C)) + half * 16;
    C *sval = reinterpret_cast<C *>(smem_raw + (size_t)td0 * PITCH * sizeof(C) +
                                    (size_t)kStripeHalves * 16 * sizeof(StripeStage<T>)) +
              half * 16;
    // polynomial coefficients in registers (zeros for lanes without a tap)
    constexpr int NC = ONE ? 1 : 2;
    T cf[NC][DEG + 1];
#pragma unroll
    for (int k = 0; k <= DEG; k++) {
        if constexpr (ONE) {
            const bool col = h < PER, row = h >= PER && h < 2 * PER;
            cf[0][k] = col ? tab[AS + k * kPolyTaps + h]
                           : (row ? tab[k * kPolyTaps + h - PER] : (T)0);
        } else {
            cf[0][k] = c < PER ? tab[AS + k * kPolyTaps + c] : (T)0;
            cf[NC - 1][k] = h < PER ? tab[k * kPolyTaps + h] : (T)0;
        }
    }
    const bool lane_col_axis = h < PER;  // ONE: this lane's polynomial is a column tap
    const T e0 = (T)g.win[0].edge_w, e1 = (T)g.win[1].edge_w;
    {
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int e = tid; e < td0 * PITCH; e += 32 * kStripeWarps) tile[e] = z;
    }
    const StripeWork &sw = g.sw;
    const int nitems = sw.work[0];
    C *const lane_col = tile + rg * PITCH + c;
    for (int sp = next_subproblem(sw.work, &s_sp); sp < nitems;
         sp = next_subproblem(sw.work, &s_sp)) {
        const SubProb it = sw.items[sp];
        const int sb0 = it.bin / sw.nsb1, sb1 = it.bin - sb0 * sw.nsb1;
        const int org0 = sb0 * g.bs[0], org1 = sb1 * (kStripeS * SW);
        if (tid < kStripeS) {  // node range of this item's part of stripe tid
            const int fb1 = (sb1 * kStripeS + tid) * sw.R;
            int2 rg2 = make_int2(0, 0);
            if (fb1 < g.nb[1]) {
                const int fbrow = sb0 * g.nb[1];
                const int last = min(fb1 + sw.R, g.nb[1]) - 1;
                const int s0 = sw.bin_start[fbrow + fb1];
                const int s1 = sw.bin_start[fbrow + last] + sw.bin_count[fbrow + last];
                const long long len = s1 - s0;
                rg2.x = s0 + (int)(len * it.start / it.count);
                rg2.y = s0 + (int)(len * (it.start + 1) / it.count);
            }
            s_rng[tid] = rg2;
        }
        __syncthreads();
#pragma unroll 1
        for (int ph = 0; ph < 2; ph++) {
            const int2 ab = s_rng[ph + 2 * half];
            const int a = ab.x, b = ab.y;
            Rec r_next;
            C v_next;
            if (a + h < b) {
                r_next = rec[a + h];
                v_next = f[perm[a + h]];
            }
            for (int k0 = a; k0 < b; k0 += 16) {
                const int nk = min(16, b - k0);
                if (h < nk) {
                    const int loc1 = (r_next.cell & g.cmask[1]) - org1;
                    const int loc0 = ((r_next.cell >> g.cbits[1]) & g.cmask[0]) - org0;
                    const T fr0 = r_next.fr[0], fr1 = r_next.fr[1];
                    StripeStage<T> st;
                    st.off = (fr0 == (T)0 || fr1 == (T)0)
                                 ? (int)(0x80000000u | (unsigned)(loc0 * PITCH + loc1))
                                 : (loc0 + 1) * PITCH + loc1 + 1;
                    st.s = k0 + h;
                    st.u0 = LIN ? fr0 : (T)2 * fr0 - (T)1;
                    st.u1 = LIN ? fr1 : (T)2 * fr1 - (T)1;
                    stage[h] = st;
                    sval[h] = v_next;
                }
                __syncwarp(mask);
                if (k0 + 16 + h < b) {  // the next chunk is in flight while this one is added
                    r_next = rec[k0 + 16 + h];
                    v_next = f[perm[k0 + 16 + h]];
                }
                for (int k = 0; k < nk; k++) {
                    const StripeStage<T> st = stage[k];
                    const C v = sval[k];
                    if (st.off >= 0) {  // uniform inside the half (one node)
                        T w1, w0h;
                        if constexpr (LIN) {
                            w1 = c < PER ? lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, 1),
                                                          g.lin_k, c + 1, st.u1, e1)
                                         : (T)0;
                            w0h = h < PER ? lin_tap<T, MM>(lin_axis<T, MM>(g.lin, g.lin_k, 0),
                                                           g.lin_k, h + 1, st.u0, e0)
                                          : (T)0;
                        } else if constexpr (ONE) {
                            const T wl = poly_horner<T, DEG>(cf[0], lane_col_axis ? st.u1 : st.u0);
                            w1 = __shfl_sync(mask, wl, c, 16);
                            w0h = wl;  // row tap rr lives in lane PER + rr
                        } else {
                            w1 = poly_horner<T, DEG>(cf[0], st.u1);
                            w0h = poly_horner<T, DEG>(cf[NC - 1], st.u0);
                        }
                        const T ar = w1 * v.x, ai = w1 * v.y;
                        C *col = lane_col + st.off;
#pragma unroll
                        for (int j = 0; j < ROWS; j++) {
                            const int rr = rg + j * RG;
                            const T w0 = __shfl_sync(mask, w0h, (ONE && !LIN) ? PER + rr : rr, 16);
                            if (c < PER && rr < PER) {
                                C q = col[j * RG * PITCH];
                                q.x += w0 * ar;
                                q.y += w0 * ai;
                                col[j * RG * PITCH] = q;
                            }
                        }
                    } else {  // on a grid point: 2m + 1 taps on some axis
                        const Rec r = rec[st.s];
                        const T fr0 = r.fr[0], fr1 = r.fr[1];
                        C *base = tile + (st.off & 0x7fffffff);
                        for (int q = h; q < NT * NT; q += 16) {
                            const int a0 = q / NT, a1 = q - a0 * NT;
                            const T w = eval_tap<T, MM, LIN ? 2 : 1>(g, tab, 0, a0, fr0) *
                                        eval_tap<T, MM, LIN ? 2 : 1>(g, tab + AS, 1, a1, fr1);
                            C *pc = base + a0 * PITCH + a1;
                            C t = *pc;
                            t.x += w * v.x;
                            t.y += w * v.y;
                            *pc = t;
                        }
                    }
                    __syncwarp(mask);
                }
            }
            __syncthreads();  // the other colour class touches the same cells
        }
        // flush: cell (a0, a1) is grid point ((org0 - m + a0) mod n0, (org1 - m + a1) mod n1)
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int idx = tid; idx < cells; idx += 32 * kStripeWarps) {
            const int a0 = idx / TD1, a1 = idx - a0 * TD1;
            C *pc = tile + a0 * PITCH + a1;
            const C cv = *pc;
            if (cv.x == (T)0 && cv.y == (T)0) continue;
            *pc = z;
            const size_t gi = (size_t)wrapn(org0 - MM + a0, g.n[0]) * g.n[1] +
                              (size_t)wrapn(org1 - MM + a1, g.n[1]);
            global_add(grid + gi, cv.x, cv.y);
        }
    }
    finish_subproblems(sw.work);
}

// Shared memory left for the dynamic part once the static window tables are placed.
template <typename T, int MM> constexpr size_t spread_dyn_limit()
{
    return 227 * 1024 - kMaxDim * poly_axis_stride(sizeof(T) == 8, MM) * sizeof(T);
}

template <typename K>
static cudaError_t launch_persistent(K kernel, size_t smem, int threads, int max_subs, int &blocks)
{
    cudaError_t e0 = ensure_dynamic_smem(kernel, smem);
    if (e0 != cudaSuccess) return e0;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidValue;
    blocks = num_sms() * per_sm;
    if (blocks > max_subs) blocks = max_subs;
    if (blocks < 1) blocks = 1;
    return cudaSuccess;
}

template <typename T, int MM, int BS0, int G>
cudaError_t launch_rows(const Geom &g, const typename Cplx<T>::type *f,
                        const typename RecOf<T>::type *rec, const int *perm,
                        const SubProb *subs, int *work, typename Cplx<T>::type *grid,
                        int warps_cap, cudaStream_t stream)
{
    const size_t smem = RowsShape<T, MM, BS0, G>::per_warp * kRowsWarps;
    int blocks = 0;
    cudaError_t e;
    if (g.lin_k) {
        e = launch_persistent(spread_rows_kernel<T, MM, true, BS0, G>, smem, 32 * kRowsWarps,
                              warps_cap, blocks);
        if (e != cudaSuccess) return e;
        spread_rows_kernel<T, MM, true, BS0, G><<<blocks, 32 * kRowsWarps, smem, stream>>>(
            g, make_wincoef<T, MM>(g), f, rec, perm, subs, work, grid);
    } else {
        e = launch_persistent(spread_rows_kernel<T, MM, false, BS0, G>, smem, 32 * kRowsWarps,
                              warps_cap, blocks);
        if (e != cudaSuccess) return e;
        spread_rows_kernel<T, MM, false, BS0, G><<<blocks, 32 * kRowsWarps, smem, stream>>>(
            g, make_wincoef<T, MM>(g), f, rec, perm, subs, work, grid);
    }
    return cudaGetLastError();
}

template <typename T, int D, int MM>
cudaError_t launch_spread_m(const Geom &g, const typename Cplx<T>::type *f,
                            const typename RecOf<T>::type *rec, const int *perm,
                            const SubProb *subs, int *nsub_total, int max_subs,
                            typename Cplx<T>::type *grid, cudaStream_t stream)
{
    size_t cells = 1;
    for (int t = 0; t < D; t++) cells *= (size_t)(g.bs[t] + 2 * MM);
    const size_t tile = cells * 2 * sizeof(T);
    int method = g.spread_method;
    if (method == kSpreadAuto) {
        method = tile * kSpreadWarps <= 64 * 1024 ? kSpreadWarpPrivate : kSpreadWarpAtomic;
        // measured fastest for 2-D: register tiles in FP32, sixteen lanes per node with private
        // tiles in FP64 (where the window evaluation, once per node, dominates)
        if (D == 2) method = sizeof(T) == 8 ? kSpreadHalf : kSpreadRows;
        if (D == 3) method = kSpreadPlane;
    }
    // a form whose shared memory does not fit falls back to the one-tile form
    constexpr size_t limit = spread_dyn_limit<T, MM>();
    const size_t octet_tiles =
        (size_t)octet_tile_stride<T>((int)cells) * sizeof(typename Cplx<T>::type) * kOctets;
    const size_t half_tiles = (size_t)(g.bs[0] + 2 * MM) *
                              (size_t)half_pitch<T, MM>(g.bs[D - 1] + 2 * MM) *
                              sizeof(typename Cplx<T>::type) * kHalfTiles;
    constexpr size_t half_stage = half_stage_bytes<T, MM>();
    if (method == kSpreadOctet &&
        (D != 2 || 2 * MM + 1 > 16 || octet_tiles + spread_stage_bytes<T>() > limit))
        method = kSpreadWarpPrivate;
    if (method == kSpreadRows &&
        (D != 2 || g.bs[D - 1] + 2 * MM > 32 || (g.bs[0] != 4 && g.bs[0] != 8)))
        method = kSpreadHalf;
    const int rows_g = g.bs[D - 1] + 2 * MM <= 16 ? 16 : 32;  // lanes per tile of the rows form
    if (method == kSpreadStripe &&
        (D != 2 || g.sw.R <= 0 || stripe_smem_bytes<T, MM>(g.bs[0] + 2 * MM) > limit))
        method = kSpreadHalf;
    if (method == kSpreadHalf && (D != 2 || half_tiles + half_stage > 227 * 1024))
        method = kSpreadWarpPrivate;
    const size_t plane_tile = D == 3 ? ((size_t)(g.bs[0] + 2 * MM) * (size_t)(g.bs[1] + 2 * MM) *
                                           (size_t)plane_pitch<T>(g.bs[D - 1] + 2 * MM) *
                                           sizeof(typename Cplx<T>::type) + 15) / 16 * 16
                                     : 0;
    if (method == kSpreadPlane && (D != 3 || plane_tile + plane_stage_bytes<T, MM>() > limit))
        method = kSpreadWarpAtomic;
    if (method == kSpreadWarpPrivate && tile * kSpreadWarps + 16 + spread_stage_bytes<T>() > limit)
        method = kSpreadWarpAtomic;
    if (method == kSpreadWarpAtomic && tile + 16 + spread_stage_bytes<T>() > limit)
        method = kSpreadThread;
    if (tile > limit) return cudaErrorInvalidValue;
    int blocks = 0;
    cudaError_t e;
    if (method == kSpreadThread) {
        e = launch_persistent(spread_kernel<T, D, MM>, tile, 256, max_subs, blocks);
        if (e != cudaSuccess) return e;
        spread_kernel<T, D, MM><<<blocks, 256, tile, stream>>>(g, f, rec, perm, subs, nsub_total,
                                                               grid);
    } else if (method == kSpreadWarpAtomic) {
        const size_t smem = (tile + 15) / 16 * 16 + spread_stage_bytes<T>();
        e = launch_persistent(spread_warp_kernel<T, D, MM, false>, smem, 32 * kSpreadWarps,
                              max_subs, blocks);
        if (e != cudaSuccess) return e;
        spread_warp_kernel<T, D, MM, false><<<blocks, 32 * kSpreadWarps, smem, stream>>>(
            g, f, rec, perm, subs, nsub_total, grid);
    } else if (method == kSpreadOctet) {
        if constexpr (D == 2) {
            const size_t smem = octet_tiles + spread_stage_bytes<T>();
            e = launch_persistent(spread_octet_kernel<T, MM>, smem, 32 * kSpreadWarps, max_subs,
                                  blocks);
            if (e != cudaSuccess) return e;
            spread_octet_kernel<T, MM><<<blocks, 32 * kSpreadWarps, smem, stream>>>(
                g, f, rec, perm, subs, nsub_total, grid);
        }
    } else if (method == kSpreadHalf) {
        if constexpr (D == 2) {
            const size_t smem = half_tiles + half_stage;
            if (g.lin_k) {
                e = launch_persistent(spread_half_kernel<T, MM, true>, smem, 32 * kHalfWarps,
                                      max_subs, blocks);
                if (e != cudaSuccess) return e;
                spread_half_kernel<T, MM, true><<<blocks, 32 * kHalfWarps, smem, stream>>>(
                    g, make_wincoef<T, MM>(g), f, rec, perm, subs, nsub_total, grid);
            } else {
                e = launch_persistent(spread_half_kernel<T, MM, false>, smem, 32 * kHalfWarps,
                                      max_subs, blocks);
                if (e != cudaSuccess) return e;
                spread_half_kernel<T, MM, false><<<blocks, 32 * kHalfWarps, smem, stream>>>(
                    g, make_wincoef<T, MM>(g), f, rec, perm, subs, nsub_total, grid);
            }
        }
    } else if (method == kSpreadRows) {
        if constexpr (D == 2) {
            const int warps_cap = (max_subs + kRowsWarps - 1) / kRowsWarps;
            if (g.bs[0] == 4)
                e = rows_g == 16 ? launch_rows<T, MM, 4, 16>(g, f, rec, perm, subs, nsub_total,
                                                              grid, warps_cap, stream)
                                 : launch_rows<T, MM, 4, 32>(g, f, rec, perm, subs, nsub_total,
                                                              grid, warps_cap, stream);
            else
                e = rows_g == 16 ? launch_rows<T, MM, 8, 16>(g, f, rec, perm, subs, nsub_total,
                                                              grid, warps_cap, stream)
                                 : launch_rows<T, MM, 8, 32>(g, f, rec, perm, subs, nsub_total,
                                                              grid, warps_cap, stream);
            if (e != cudaSuccess) return e;
        }
    } else if (method == kSpreadStripe) {
        if constexpr (D == 2) {
            const size_t smem = stripe_smem_bytes<T, MM>(g.bs[0] + 2 * MM);
            if (g.lin_k) {
                e = launch_persistent(spread_stripe_kernel<T, MM, true>, smem, 32 * kStripeWarps,
                                      g.sw.max_items, blocks);
                if (e != cudaSuccess) return e;
                spread_stripe_kernel<T, MM, true><<<blocks, 32 * kStripeWarps, smem, stream>>>(
                    g, f, rec, perm, grid);
            } else {
                e = launch_persistent(spread_stripe_kernel<T, MM, false>, smem, 32 * kStripeWarps,
                                      g.sw.max_items, blocks);
                if (e != cudaSuccess) return e;
                spread_stripe_kernel<T, MM, false><<<blocks, 32 * kStripeWarps, smem, stream>>>(
                    g, f, rec, perm, grid);
            }
        }
    } else if (method == kSpreadPlane) {
        if constexpr (D == 3) {
            const size_t smem = plane_tile + plane_stage_bytes<T, MM>();
            if (g.lin_k) {
                e = launch_persistent(spread_plane_kernel<T, MM, true>, smem, 32 * kPlaneWarps,
                                      max_subs, blocks);
                if (e != cudaSuccess) return e;
                spread_plane_kernel<T, MM, true><<<blocks, 32 * kPlaneWarps, smem, stream>>>(
                    g, f, rec, perm, subs, nsub_total, grid);
            } else {
                e = launch_persistent(spread_plane_kernel<T, MM, false>, smem, 32 * kPlaneWarps,
                                      max_subs, blocks);
                if (e != cudaSuccess) return e;
                spread_plane_kernel<T, MM, false><<<blocks, 32 * kPlaneWarps, smem, stream>>>(
                    g, f, rec, perm, subs, nsub_total, grid);
            }
        }
    } else if (method == kSpreadWarpPrivate) {
        const size_t smem = (tile * kSpreadWarps + 15) / 16 * 16 + spread_stage_bytes<T>();
        e = launch_persistent(spread_warp_kernel<T, D, MM, true>, smem, 32 * kSpreadWarps,
                              max_subs, blocks);
        if (e != cudaSuccess) return e;
        spread_warp_kernel<T, D, MM, true><<<blocks, 32 * kSpreadWarps, smem, stream>>>(
            g, f, rec, perm, subs, nsub_total, grid);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}



template <typename T, int D>
cudaError_t spread_d(const Geom &g, const typename Cplx<T>::type *f,
                     const typename RecOf<T>::type *rec, const int *perm, const SubProb *subs,
                     int *nsub_total, int max_subs, typename Cplx<T>::type *grid,
                     cudaStream_t stream)
{
    GBNFFT_DISPATCH_M(launch_spread_m, T, D, g, f, rec, perm, subs, nsub_total, max_subs, grid,
                      stream)
}

}  // namespace detail
}  // namespace gbnfft
