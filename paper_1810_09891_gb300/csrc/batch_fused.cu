// Fused batches: every plan of a batch in one launch per stage (the batched form of the paper's
// plan, Section 3.1, run many times over). A stage's CTAs walk a work list that spans all plans:
//   - zeroing of the grids: (plan, chunk) blocks;
//   - B (interpolation) and the node gradient: (plan, 128 sorted nodes) blocks;
//   - B^H (spreading): the plans' subproblem lists concatenated, claimed one at a time through a
//     work counter (persistent CTAs, as in the single-plan half-warp form);
//   - the FFT passes: (plan, P lines) blocks (launch_fft_fused, fft_impl.cuh).
// The kernels here are the 2-D FP32 forms (rows or half-warp spreading, thread interpolation) for
// plans of one window cutoff m and one window; a CTA (a warp group in the rows form) looks its
// plan up in the per-plan table and reads that plan's geometry before working on it; the window
// polynomials come from the kernel argument when every plan has the same ones, else from each
// plan's table.
#include "interp_impl.cuh"
#include "spread_impl.cuh"

namespace gbnfft {
namespace detail {

namespace {

constexpr int kZeroThreads = 256;
constexpr int kZeroPerThread = 8;  // float4 stores per thread and block

// The plan whose blocks [first(p), first(p + 1)) contain block b (first is nondecreasing).
template <typename Get>
__device__ __forceinline__ int find_plan(int nplans, int b, Get first)
{
    int lo = 0, hi = nplans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first(mid) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Copy plan p's geometry into shared memory (every thread of the CTA calls it).
__device__ __forceinline__ void load_geom(const FusedNodePlan *__restrict__ plans, int p, Geom *sg)
{
    const int *src = reinterpret_cast<const int *>(&plans[p].g);
    int *dst = reinterpret_cast<int *>(sg);
    constexpr int words = (int)(sizeof(Geom) / sizeof(int));
    for (int e = threadIdx.x; e < words; e += blockDim.x) dst[e] = src[e];
}

__global__ void __launch_bounds__(kZeroThreads)
    zero_fused_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                      const __grid_constant__ FusedOffsets off, size_t csize)
{
    const int nblocks = off.zero_block0[nplans];
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int p = find_plan(nplans, b, [&](int q) { return off.zero_block0[q]; });
        const size_t n4 = (size_t)plans[p].G * csize / 16;  // grids are 256-byte aligned
        float4 *g4 = static_cast<float4 *>(plans[p].grid);
        const size_t base = (size_t)(b - off.zero_block0[p]) * kZeroThreads * kZeroPerThread;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < kZeroPerThread; k++) {
            const size_t e = base + (size_t)k * kZeroThreads + threadIdx.x;
            if (e < n4) g4[e] = z;
        }
    }
}

// The prefix of the plans' subproblem counts (read on the device after set_nodes): item_start[p]
// is plan p's first item in the batch's list; work[0] the item count, work[1..2] the counters.
__global__ void __launch_bounds__(kFusedMax)
    fused_items_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                       int *__restrict__ item_start, int *__restrict__ work)
{
    __shared__ int s[kFusedMax];
    const int p = threadIdx.x;
    const int c = (p < nplans && plans[p].M > 0) ? plans[p].nsub[0] : 0;
    s[p] = c;
    __syncthreads();
    for (int off = 1; off < kFusedMax; off <<= 1) {  // inclusive scan (Hillis-Steele)
        const int v = p >= off ? s[p - off] : 0;
        __syncthreads();
        s[p] += v;
        __syncthreads();
    }
    if (p < nplans) item_start[p] = s[p] - c;
    if (p == kFusedMax - 1) {
        item_start[nplans] = s[p];
        work[0] = s[p];
        work[1] = 0;
        work[2] = 0;
    }
}

// SHARED: every plan has the same window polynomials (the same oversampling factors), passed
// once as a kernel argument (constant-bank operands); otherwise each plan's own table is read
// from global memory.
// One CTA per block of 128 sorted nodes of one plan; the plan comes from the block offsets in
// the kernel argument and its geometry is read through L1.
template <typename T, int MM, bool SHARED>
__global__ void __launch_bounds__(kInterpThreads)
    interp_fused_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                        const __grid_constant__ FusedOffsets off,
                        const __grid_constant__ WinCoef<T, MM> wc,
                        const __grid_constant__ FusedPtrs ptrs)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    const int b = blockIdx.x;
    const int p = find_plan(nplans, b, [&](int q) { return off.node_block0[q]; });
    const Geom &sg = plans[p].g;
    {
        const int s = (b - off.node_block0[p]) * kInterpThreads + threadIdx.x;
        if (s < plans[p].M) {
            const Rec r = static_cast<const Rec *>(plans[p].rec)[s];
            int base[2];
            T frac[2];
            bool edge;
            decode_node<T, 2>(sg, r, base, frac, edge);
            const C *grid = static_cast<const C *>(plans[p].fgrid);
            const T *tab = SHARED ? wc.c : static_cast<const T *>(sg.poly);
            const C v = edge ? interp_node<T, 2, MM, 0, 1>(sg, tab, grid, base, frac)
                             : interp_node<T, 2, MM, 1, 1>(sg, tab, grid, base, frac);
            static_cast<C *>(ptrs.out[p])[plans[p].perm[s]] = v;
        }
    }
}

template <typename T, int MM, bool SHARED>
__global__ void __launch_bounds__(kInterpThreads)
    grad_fused_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                      const __grid_constant__ FusedOffsets off,
                      const __grid_constant__ WinCoef<T, MM> wc,
                      const __grid_constant__ FusedPtrs ptrs)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    const int b = blockIdx.x;
    const int p = find_plan(nplans, b, [&](int q) { return off.node_block0[q]; });
    const Geom &sg = plans[p].g;
    {
        const int s = (b - off.node_block0[p]) * kInterpThreads + threadIdx.x;
        if (s < plans[p].M) {
            const Rec r = static_cast<const Rec *>(plans[p].rec)[s];
            int base[2];
            T frac[2];
            bool edge;
            decode_node<T, 2>(sg, r, base, frac, edge);
            const C *grid = static_cast<const C *>(plans[p].fgrid);
            const T *tab = SHARED ? wc.c : static_cast<const T *>(sg.poly);
            C acc[2];
            if (!edge)
                grad_node<T, 2, MM, 1>(sg, tab, grid, base, frac, acc);
            else
                grad_node<T, 2, MM, 0>(sg, tab, grid, base, frac, acc);
            const int j = plans[p].perm[s];
            const C wj = static_cast<const C *>(ptrs.in[p])[j];
            T *gx = static_cast<T *>(ptrs.out[p]);
#pragma unroll
            for (int t = 0; t < 2; t++)  // Re(conj(w) * n_t * acc_t)
                gx[(size_t)j * 2 + t] = (T)sg.n[t] * (wj.x * acc[t].x + wj.y * acc[t].y);
        }
    }
}

// B^H of every plan: the CTAs claim subproblems of the concatenated lists through the batch's
// work counter; the private tiles start clean and every flush leaves the cells it covered clean
// again, so consecutive subproblems of different plans (different bin shapes) share them. With
// SHARED every plan has the window polynomials of `wc` (kernel parameter space); otherwise each
// plan's own table is read from global memory.
template <typename T, int MM, bool SHARED>
__global__ void __launch_bounds__(32 * kHalfWarps)
    spread_fused_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                        const int *__restrict__ item_start, int *__restrict__ work,
                        int tile_cells, const __grid_constant__ WinCoef<T, MM> wc,
                        const __grid_constant__ FusedPtrs ptrs)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Geom sg;
    __shared__ int s_sp;
    {
        C *tiles = half_tiles<T, MM>(smem_raw);
        C z;
        z.x = (T)0;
        z.y = (T)0;
        for (int e = threadIdx.x; e < kHalfTiles * tile_cells; e += 32 * kHalfWarps) tiles[e] = z;
    }
    __shared__ int s_start[kFusedMax + 1];
    for (int q = threadIdx.x; q <= nplans; q += blockDim.x) s_start[q] = item_start[q];
    const int nitems = work[0];
    int cur = -1;  // the plan whose geometry is loaded
    for (int sp = next_subproblem(work, &s_sp); sp < nitems; sp = next_subproblem(work, &s_sp)) {
        const int p = find_plan(nplans, sp, [&](int q) { return s_start[q]; });
        if (p != cur) {  // uniform in the CTA
            load_geom(plans, p, &sg);
            __syncthreads();
            cur = p;
        }
        const SubProb P = plans[p].subs[sp - s_start[p]];
        const T *coef = SHARED ? wc.c : static_cast<const T *>(plans[p].g.poly);
        half_subproblem<T, MM, false>(sg, P, static_cast<const C *>(ptrs.in[p]),
                                      static_cast<const Rec *>(plans[p].rec), plans[p].perm,
                                      static_cast<C *>(plans[p].grid), smem_raw, coef);
    }
    finish_subproblems(work);
}

// B^H of every plan in the rows form (register tiles, one subproblem per half-warp or warp):
// the warps claim entries of the concatenated subproblem lists through the batch's work
// counter; each group looks up its own entry's plan, so the two groups of a warp may work on
// different plans. Every plan has sort bins of BS0 rows and tiles at most G cells wide.
template <typename T, int MM, int BS0, int G, bool SHARED>
__global__ void __launch_bounds__(32 * kRowsWarps)
    spread_rows_fused_kernel(const FusedNodePlan *__restrict__ plans, int nplans,
                             const int *__restrict__ item_start, int *__restrict__ work,
                             const __grid_constant__ WinCoef<T, MM> wc,
                             const __grid_constant__ FusedPtrs ptrs)
{
    using C = typename Cplx<T>::type;
    using Rec = typename RecOf<T>::type;
    using Sh = RowsShape<T, MM, BS0, G>;
    constexpr int GROUPS = Sh::GROUPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_start[kFusedMax + 1];
    for (int q = threadIdx.x; q <= nplans; q += blockDim.x) s_start[q] = item_start[q];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const RowsStage<T, MM, BS0, G> st(smem_raw + (size_t)warp * Sh::per_warp +
                                      (size_t)grp * Sh::group);
    const int nitems = work[0];
    auto entry = [&](int sp0, int &p) {  // this group's entry of a claim and its plan
        SubProb P;
        P.bin = 0;
        P.start = 0;
        P.count = 0;
        p = 0;
        const int sp = sp0 + grp;
        if (sp < nitems) {
            p = find_plan(nplans, sp, [&](int q) { return s_start[q]; });
            P = plans[p].subs[sp - s_start[p]];
        }
        return P;
    };
    int p;
    int sp0 = rows_claim(work, GROUPS);
    SubProb P = entry(sp0, p);
    while (sp0 < nitems) {
        int pn;
        const int sp0n = rows_claim(work, GROUPS);  // the next claim, read while this one runs
        const SubProb Pn = entry(sp0n, pn);
        int most = P.count;
        if constexpr (GROUPS == 2) most = max(most, __shfl_xor_sync(0xffffffffu, most, 16));
        const Geom &g = plans[p].g;
        const T *coef = SHARED ? wc.c : static_cast<const T *>(g.poly);
        rows_subproblem<T, MM, 1, BS0, G>(g, coef, P, most, static_cast<const C *>(ptrs.in[p]),
                                          static_cast<const Rec *>(plans[p].rec), plans[p].perm,
                                          static_cast<C *>(plans[p].grid), st, gl);
        sp0 = sp0n;
        P = Pn;
        p = pn;
    }
    rows_finish(work);
}

template <typename K>
int persistent_blocks(K kernel, int threads, size_t smem, int cap)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    int blocks = per_sm * num_sms();
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

template <typename T, int MM, bool SHARED>
cudaError_t interp_fused_ms(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                            const WinCoef<T, MM> &wc, const FusedPtrs &ptrs, bool grad,
                            cudaStream_t stream)
{
    const int nblocks = off.node_block0[nplans];
    if (grad)
        grad_fused_kernel<T, MM, SHARED><<<nblocks, kInterpThreads, 0, stream>>>(
            plans, nplans, off, wc, ptrs);
    else
        interp_fused_kernel<T, MM, SHARED><<<nblocks, kInterpThreads, 0, stream>>>(
            plans, nplans, off, wc, ptrs);
    return cudaGetLastError();
}

template <typename T, int MM>
cudaError_t interp_fused_m(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                           const Geom &g0, const FusedPtrs &ptrs, bool grad, bool shared,
                           cudaStream_t stream)
{
    const WinCoef<T, MM> wc = make_wincoef<T, MM>(g0);
    return shared ? interp_fused_ms<T, MM, true>(plans, nplans, off, wc, ptrs, grad, stream)
                  : interp_fused_ms<T, MM, false>(plans, nplans, off, wc, ptrs, grad, stream);
}

template <typename T, int MM, bool SHARED>
cudaError_t spread_fused_ms(const FusedNodePlan *plans, int nplans, const int *item_start,
                            int *work, int max_items, int tile_cells, const WinCoef<T, MM> &wc,
                            const FusedPtrs &ptrs, cudaStream_t stream)
{
    const size_t smem = half_stage_bytes<T, MM>() +
                        (size_t)kHalfTiles * tile_cells * sizeof(typename Cplx<T>::type);
    cudaError_t e = ensure_dynamic_smem(spread_fused_kernel<T, MM, SHARED>, smem);
    if (e != cudaSuccess) return e;
    const int blocks =
        persistent_blocks(spread_fused_kernel<T, MM, SHARED>, 32 * kHalfWarps, smem, max_items);
    if (!blocks) return cudaErrorInvalidValue;
    spread_fused_kernel<T, MM, SHARED><<<blocks, 32 * kHalfWarps, smem, stream>>>(
        plans, nplans, item_start, work, tile_cells, wc, ptrs);
    return cudaGetLastError();
}

template <typename T, int MM, int BS0, int G, bool SHARED>
cudaError_t spread_rows_fused_ms(const FusedNodePlan *plans, int nplans, const int *item_start,
                                 int *work, int max_items, const WinCoef<T, MM> &wc,
                                 const FusedPtrs &ptrs, cudaStream_t stream)
{
    using Sh = RowsShape<T, MM, BS0, G>;
    const size_t smem = Sh::per_warp * kRowsWarps;
    cudaError_t e = ensure_dynamic_smem(spread_rows_fused_kernel<T, MM, BS0, G, SHARED>, smem);
    if (e != cudaSuccess) return e;
    const int cap = (max_items + Sh::GROUPS * kRowsWarps - 1) / (Sh::GROUPS * kRowsWarps);
    const int blocks = persistent_blocks(spread_rows_fused_kernel<T, MM, BS0, G, SHARED>,
                                         32 * kRowsWarps, smem, cap);
    if (!blocks) return cudaErrorInvalidValue;
    spread_rows_fused_kernel<T, MM, BS0, G, SHARED><<<blocks, 32 * kRowsWarps, smem, stream>>>(
        plans, nplans, item_start, work, wc, ptrs);
    return cudaGetLastError();
}

template <typename T, int MM, int BS0, int G>
cudaError_t spread_rows_fused_m(const FusedNodePlan *plans, int nplans, const int *item_start,
                                int *work, int max_items, const WinCoef<T, MM> &wc,
                                const FusedPtrs &ptrs, bool shared, cudaStream_t stream)
{
    return shared ? spread_rows_fused_ms<T, MM, BS0, G, true>(plans, nplans, item_start, work,
                                                              max_items, wc, ptrs, stream)
                  : spread_rows_fused_ms<T, MM, BS0, G, false>(plans, nplans, item_start, work,
                                                               max_items, wc, ptrs, stream);
}

template <typename T, int MM>
cudaError_t spread_fused_m(const FusedNodePlan *plans, int nplans, const int *item_start,
                           int *work, int max_items, int tile_cells, const Geom &g0,
                           const FusedPtrs &ptrs, bool shared, int rows_bs0, int rows_g,
                           cudaStream_t stream)
{
    const WinCoef<T, MM> wc = make_wincoef<T, MM>(g0);
    if (rows_bs0 == 4 && rows_g == 16)
        return spread_rows_fused_m<T, MM, 4, 16>(plans, nplans, item_start, work, max_items, wc,
                                                 ptrs, shared, stream);
    if (rows_bs0 == 4 && rows_g == 32)
        return spread_rows_fused_m<T, MM, 4, 32>(plans, nplans, item_start, work, max_items, wc,
                                                 ptrs, shared, stream);
    if (rows_bs0 == 8 && rows_g == 16)
        return spread_rows_fused_m<T, MM, 8, 16>(plans, nplans, item_start, work, max_items, wc,
                                                 ptrs, shared, stream);
    if (rows_bs0 == 8 && rows_g == 32)
        return spread_rows_fused_m<T, MM, 8, 32>(plans, nplans, item_start, work, max_items, wc,
                                                 ptrs, shared, stream);
    return shared ? spread_fused_ms<T, MM, true>(plans, nplans, item_start, work, max_items,
                                                 tile_cells, wc, ptrs, stream)
                  : spread_fused_ms<T, MM, false>(plans, nplans, item_start, work, max_items,
                                                  tile_cells, wc, ptrs, stream);
}

}  // namespace
}  // namespace detail

cudaError_t launch_zero_fused(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                              size_t csize, cudaStream_t stream)
{
    const int nblocks = off.zero_block0[nplans];
    if (nblocks <= 0) return cudaSuccess;
    const int blocks = detail::persistent_blocks(detail::zero_fused_kernel, detail::kZeroThreads,
                                                 0, nblocks);
    if (!blocks) return cudaErrorInvalidValue;
    detail::zero_fused_kernel<<<blocks, detail::kZeroThreads, 0, stream>>>(plans, nplans, off,
                                                                           csize);
    return cudaGetLastError();
}

int zero_fused_blocks(long long G, size_t csize)
{
    const long long per = (long long)detail::kZeroThreads * detail::kZeroPerThread * 16;
    return (int)((G * (long long)csize + per - 1) / per);
}

cudaError_t launch_interp_fused(const FusedNodePlan *plans, int nplans, const FusedOffsets &off,
                                const Geom &g0, const FusedPtrs &ptrs, bool grad,
                                bool shared_window, cudaStream_t stream)
{
    if (off.node_block0[nplans] <= 0) return cudaSuccess;
    switch (g0.m) {
#define GB_CASE(MM)                                                                               \
    case MM:                                                                                      \
        return detail::interp_fused_m<float, MM>(plans, nplans, off, g0, ptrs, grad,            \
                                                 shared_window, stream);
        GB_CASE(1) GB_CASE(2) GB_CASE(3) GB_CASE(4) GB_CASE(5) GB_CASE(6) GB_CASE(7) GB_CASE(8)
#undef GB_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spread_fused(const FusedNodePlan *plans, int nplans, int *item_start,
                                int *work, int max_items, int tile_cells, const Geom &g0,
                                const FusedPtrs &ptrs, bool shared_window, int rows_bs0,
                                int rows_g, cudaStream_t stream)
{
    detail::fused_items_kernel<<<1, kFusedMax, 0, stream>>>(plans, nplans, item_start, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (max_items <= 0) return cudaSuccess;
    switch (g0.m) {
#define GB_CASE(MM)                                                                               \
    case MM:                                                                                      \
        return detail::spread_fused_m<float, MM>(plans, nplans, item_start, work, max_items,      \
                                                 tile_cells, g0, ptrs, shared_window, rows_bs0, \
                                                 rows_g, stream);
        GB_CASE(1) GB_CASE(2) GB_CASE(3) GB_CASE(4) GB_CASE(5) GB_CASE(6) GB_CASE(7) GB_CASE(8)
#undef GB_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbnfft

namespace gbnfft {

// Cells of one private tile of the half-warp form for FP32 (td0 rows of the padded pitch).
int half_tile_cells_f32(int m, int bs0, int bs1)
{
    int pitch = 0;
    switch (m) {
#define GB_CASE(MM)                                                                               \
    case MM: pitch = detail::half_pitch<float, MM>(bs1 + 2 * MM); break;
        GB_CASE(1) GB_CASE(2) GB_CASE(3) GB_CASE(4) GB_CASE(5) GB_CASE(6) GB_CASE(7) GB_CASE(8)
#undef GB_CASE
    default: return 0;
    }
    return (bs0 + 2 * m) * pitch;
}

size_t half_smem_bytes_f32(int m, int tile_cells)
{
    size_t stage = 0;
    switch (m) {
#define GB_CASE(MM)                                                                               \
    case MM: stage = detail::half_stage_bytes<float, MM>(); break;
        GB_CASE(1) GB_CASE(2) GB_CASE(3) GB_CASE(4) GB_CASE(5) GB_CASE(6) GB_CASE(7) GB_CASE(8)
#undef GB_CASE
    default: return ~size_t(0);
    }
    return stage + (size_t)detail::kHalfTiles * tile_cells * sizeof(float2);
}

}  // namespace gbnfft
