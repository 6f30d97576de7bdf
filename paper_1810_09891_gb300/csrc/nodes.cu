// Node precomputation (set_nodes): grid cell and offset of every node, then a counting sort of
// the nodes into bins (tiles of the oversampled grid; inside a bin by grid row along axis 0),
// then the list of spreading subproblems.
// This is the GPU form of the paper's node sorting (Section 3.1, Table tab:nfftflags,
// NFFT_SORT_NODES): nodes that share a tile are processed together by the interpolation and
// spreading kernels.
#include <map>
#include <mutex>
#include <utility>

#include "gbnfft_internal.cuh"

namespace gbnfft {

cudaError_t ensure_dynamic_smem_ptr(const void *kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(kernel, dev);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    done[key] = bytes;
    return cudaSuccess;
}

// |n x| must stay below 2^52 for floor() and the offset to be exact in FP64.
static constexpr double kMaxAbsNx = 4503599627370496.0;

// Grid position of coordinate t of a node: base = floor(n x) (as an integer), frac = n x - base.
// frac is computed in FP64 for both precisions. Returns false for NaN, inf or |n x| >= 2^52.
template <typename T>
__device__ __forceinline__ bool node_pos(T xt, int n, long long &base, double &frac)
{
    const double tt = (double)n * (double)xt;
    if (!(fabs(tt) < kMaxAbsNx)) {
        base = 0;
        frac = 0.5;
        return false;
    }
    const double bf = floor(tt);
    base = (long long)bf;
    frac = tt - bf;  // in [0, 1]; equals 1 only when tt is a tiny negative number
    return true;
}

// Sort key of a node: its bin, and inside the bin its grid row (a sub-bin: the cell along axis 0
// in 1-D and 2-D, the (axis 0, axis 1) cell pair in 3-D): nodes of a bin end up ordered by row,
// so that neighbouring threads of the interpolation read the same grid rows.
__host__ __device__ inline int row_subbins(const Geom &g)
{
    return g.d == 3 ? g.bs[0] * g.bs[1] : g.bs[0];
}

template <typename T>
__global__ void node_bin_kernel(Geom g, const T *__restrict__ x, int M, int *__restrict__ sub_count,
                                int2 *__restrict__ sub_rank, int *__restrict__ status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int bin = 0, row = 0;
    bool ok = true;
    for (int t = 0; t < g.d; t++) {
        long long base;
        double frac;
        ok &= node_pos<T>(x[(long long)j * g.d + t], g.n[t], base, frac);
        long long b = base % g.n[t];  // base mod n
        if (b < 0) b += g.n[t];
        bin = bin * g.nb[t] + ((int)b >> g.bslog[t]);
        if (t == 0) row = (int)b & (g.bs[0] - 1);
        if (t == 1 && g.d == 3) row = row * g.bs[1] + ((int)b & (g.bs[1] - 1));
    }
    if (!ok) atomicCAS(status, kStatusOk, (int)NFFT_EBADNODE);
    const int sub = bin * row_subbins(g) + row;
    const int rank = atomicAdd(&sub_count[sub], 1);
    sub_rank[j] = make_int2(sub, rank);
}

template <typename T>
cudaError_t launch_node_bin(const Geom &g, const T *x, int64_t M, int *sub_count, int2 *sub_rank,
                            int *status, cudaStream_t stream)
{
    if (M == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((M + threads - 1) / threads);
    node_bin_kernel<T><<<blocks, threads, 0, stream>>>(g, x, (int)M, sub_count, sub_rank, status);
    return cudaGetLastError();
}

// Per bin: its node count, the sum over its S0 row sub-bins.
__global__ void bin_totals_kernel(const int *__restrict__ sub_count, int S0, int nbins,
                                  int *__restrict__ bin_count)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    int sum = 0;
    for (int r = 0; r < S0; r++) sum += sub_count[b * S0 + r];
    bin_count[b] = sum;
}

// Per row sub-bin: its first position in sorted order (the bin's start plus the rows before).
__global__ void sub_starts_kernel(const int *__restrict__ sub_count,
                                  const int *__restrict__ bin_start, int S0, int nbins,
                                  int *__restrict__ sub_start)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    int run = bin_start[b];
    for (int r = 0; r < S0; r++) {
        sub_start[b * S0 + r] = run;
        run += sub_count[b * S0 + r];
    }
}

cudaError_t launch_bin_totals(const int *sub_count, int S0, int nbins, int *bin_count,
                              cudaStream_t stream)
{
    const int threads = 256;
    bin_totals_kernel<<<(nbins + threads - 1) / threads, threads, 0, stream>>>(sub_count, S0,
                                                                              nbins, bin_count);
    return cudaGetLastError();
}

cudaError_t launch_sub_starts(const int *sub_count, const int *bin_start, int S0, int nbins,
                              int *sub_start, cudaStream_t stream)
{
    const int threads = 256;
    sub_starts_kernel<<<(nbins + threads - 1) / threads, threads, 0, stream>>>(
        sub_count, bin_start, S0, nbins, sub_start);
    return cudaGetLastError();
}

// Exclusive scans of the bin counts and of the subproblem counts ceil(count / sub_max), in one
// CTA of 1024 threads (each thread owns a contiguous chunk of slots). The scan visits the bins
// in slot order: the natural order, or with nb1 > 0 (2-D) blocks of 2 x 2 bins one after the
// other (block rows along axis 0, blocks along axis 1, inside a block the bins row-major), so
// that consecutive sorted nodes cover a compact region of twice the bin in each direction;
// slots of a partial block outside the bin grid are empty. With `staged` the counts are first
// copied into shared memory (padded by one word per 32, so that the threads' chunks of 32 fall
// on distinct banks) and the bin starts written back from there; a thread walking its chunk in
// global memory would wait for one load after another.
__host__ __device__ inline int scan_pad(int i) { return i + (i >> 5); }

// The bin in slot i (-1: a slot of a partial block outside the grid).
__host__ __device__ inline int scan_bin(int i, int nbins, int nb0, int nb1)
{
    if (nb1 <= 0) return i < nbins ? i : -1;
    const int blk = i >> 2, q = i & 3, nbb1 = (nb1 + 1) >> 1;
    const int b0 = 2 * (blk / nbb1) + (q >> 1), b1 = 2 * (blk % nbb1) + (q & 1);
    return (b0 < nb0 && b1 < nb1) ? b0 * nb1 + b1 : -1;
}

__host__ __device__ inline int scan_slots(int nbins, int nb0, int nb1)
{
    return nb1 <= 0 ? nbins : 4 * ((nb0 + 1) >> 1) * ((nb1 + 1) >> 1);
}

__global__ void __launch_bounds__(1024)
    bin_scan_kernel(const int *__restrict__ count, int *__restrict__ start,
                    int *__restrict__ sub_start, int *__restrict__ nsub_total, int nbins,
                    int nb0, int nb1, int sub_max, int staged)
{
    extern __shared__ int s_cnt[];  // scan_pad(slots) words when staged
    __shared__ int s_a[1024];
    __shared__ int s_b[1024];
    const int tid = threadIdx.x;
    const int slots = scan_slots(nbins, nb0, nb1);
    if (staged) {
        for (int i = tid; i < slots; i += 1024) {
            const int bin = scan_bin(i, nbins, nb0, nb1);
            s_cnt[scan_pad(i)] = bin >= 0 ? count[bin] : 0;
        }
        __syncthreads();
    }
    auto cnt_at = [&](int i) {
        if (staged) return s_cnt[scan_pad(i)];
        const int bin = scan_bin(i, nbins, nb0, nb1);
        return bin >= 0 ? count[bin] : 0;
    };
    const int chunk = (slots + 1023) / 1024;
    const int lo = min(slots, tid * chunk), hi = min(slots, lo + chunk);
    int a = 0, b = 0;
    for (int i = lo; i < hi; i++) {
        const int c = cnt_at(i);
        a += c;
        b += (c + sub_max - 1) / sub_max;
    }
    s_a[tid] = a;
    s_b[tid] = b;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partial sums
    for (int off = 1; off < 1024; off <<= 1) {
        const int va = tid >= off ? s_a[tid - off] : 0;
        const int vb = tid >= off ? s_b[tid - off] : 0;
        __syncthreads();
        s_a[tid] += va;
        s_b[tid] += vb;
        __syncthreads();
    }
    int ra = s_a[tid] - a, rb = s_b[tid] - b;  // exclusive prefix of this chunk
    for (int i = lo; i < hi; i++) {
        const int c = cnt_at(i);
        const int bin = scan_bin(i, nbins, nb0, nb1);
        if (bin >= 0) sub_start[bin] = rb;
        rb += (c + sub_max - 1) / sub_max;
        if (staged)
            s_cnt[scan_pad(i)] = ra;  // (only this thread reads its chunk)
        else if (bin >= 0)
            start[bin] = ra;
        ra += c;
    }
    if (staged) {
        __syncthreads();
        for (int i = tid; i < slots; i += 1024) {
            const int bin = scan_bin(i, nbins, nb0, nb1);
            if (bin >= 0) start[bin] = s_cnt[scan_pad(i)];
        }
    }
    if (tid == 1023) {
        nsub_total[0] = s_b[1023];
        nsub_total[1] = 0;  // work counters of the spreading kernels (next entry, CTAs done)
        nsub_total[2] = 0;
    }
}

cudaError_t launch_bin_scan(const int *bin_count, int *bin_start, int *sub_start, int *nsub_total,
                            int nbins, int sub_max, cudaStream_t stream, int nb0, int nb1)
{
    constexpr int kStagedMax = 49152;  // slots staged in shared memory (196 KB with padding)
    const int slots = scan_slots(nbins, nb0, nb1);
    const int staged = slots <= kStagedMax ? 1 : 0;
    const size_t smem = staged ? (size_t)(scan_pad(slots) + 1) * sizeof(int) : 0;
    if (staged) {
        const cudaError_t e = ensure_dynamic_smem(bin_scan_kernel, smem);
        if (e != cudaSuccess) return e;
    }
    bin_scan_kernel<<<1, 1024, smem, stream>>>(bin_count, bin_start, sub_start, nsub_total,
                                               nbins, nb0, nb1, sub_max, staged);
    return cudaGetLastError();
}

template <typename T>
__global__ void node_scatter_kernel(Geom g, const T *__restrict__ x, int M,
                                    const int2 *__restrict__ sub_rank,
                                    const int *__restrict__ sub_start,
                                    typename RecOf<T>::type *__restrict__ rec, int *__restrict__ perm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    typename RecOf<T>::type r;
    r.cell = 0;
    for (int t = 0; t < kMaxDim; t++) r.fr[t] = (T)0;
    for (int t = 0; t < g.d; t++) {
        long long base;
        double frac;
        node_pos<T>(x[(long long)j * g.d + t], g.n[t], base, frac);
        long long b = base % g.n[t];
        if (b < 0) b += g.n[t];
        r.cell = (r.cell << g.cbits[t]) | (int)b;
        r.fr[t] = (T)frac;
    }
    const int2 br = sub_rank[j];
    const int pos = sub_start[br.x] + br.y;
    rec[pos] = r;
    perm[pos] = j;
}

template <typename T>
cudaError_t launch_node_scatter(const Geom &g, const T *x, int64_t M, const int2 *sub_rank,
                                const int *sub_start, typename RecOf<T>::type *rec, int *perm,
                                cudaStream_t stream)
{
    if (M == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((M + threads - 1) / threads);
    node_scatter_kernel<T><<<blocks, threads, 0, stream>>>(g, x, (int)M, sub_rank, sub_start, rec,
                                                           perm);
    return cudaGetLastError();
}

__global__ void fill_subprobs_kernel(const int *__restrict__ count, const int *__restrict__ start,
                                     const int *__restrict__ sub_start, SubProb *__restrict__ subs,
                                     int nbins, int sub_max)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int c = count[b];
    const int s0 = sub_start[b];
    // ceil(c / sub_max) parts of equal size (within one node): the warps that take consecutive
    // parts then run equally long
    const int parts = (c + sub_max - 1) / sub_max;
    for (int k = 0; k < parts; k++) {
        const int lo = (int)((long long)c * k / parts), hi = (int)((long long)c * (k + 1) / parts);
        SubProb p;
        p.bin = b;
        p.start = start[b] + lo;
        p.count = hi - lo;
        p.pad = 0;
        subs[s0 + k] = p;
    }
}

cudaError_t launch_fill_subprobs(const int *bin_count, const int *bin_start, const int *sub_start,
                                 SubProb *subs, int nbins, int sub_max, cudaStream_t stream)
{
    const int threads = 256;
    fill_subprobs_kernel<<<(nbins + threads - 1) / threads, threads, 0, stream>>>(
        bin_count, bin_start, sub_start, subs, nbins, sub_max);
    return cudaGetLastError();
}

// Node count of the heaviest stripe of every super-bin (a stripe is R sort bins): a work item
// takes one part of every stripe, and a stripe's part is walked by one half-warp, so the parts
// are sized by the heaviest stripe.
__global__ void superbin_count_kernel(const int *__restrict__ count, int nb0, int nb1, int R,
                                      int nsb1, int *__restrict__ sb_count)
{
    const int sb = blockIdx.x * blockDim.x + threadIdx.x;
    if (sb >= nb0 * nsb1) return;
    const int b0 = sb / nsb1, c0 = (sb - b0 * nsb1) * kStripeS * R;
    const int c1 = min(c0 + kStripeS * R, nb1);
    int most = 0;
    for (int s = c0; s < c1; s += R) {
        int sum = 0;
        for (int c = s; c < min(s + R, c1); c++) sum += count[b0 * nb1 + c];
        most = max(most, sum);
    }
    sb_count[sb] = most;
}

__global__ void fill_stripe_items_kernel(const int *__restrict__ sb_count,
                                         const int *__restrict__ sb_sub, SubProb *__restrict__ items,
                                         int nsb, int item)
{
    const int sb = blockIdx.x * blockDim.x + threadIdx.x;
    if (sb >= nsb) return;
    const int c = sb_count[sb];
    const int parts = (c + item - 1) / item;
    for (int k = 0; k < parts; k++) {
        SubProb p;
        p.bin = sb;
        p.start = k;
        p.count = parts;
        p.pad = 0;
        items[sb_sub[sb] + k] = p;
    }
}

cudaError_t launch_stripe_items(const int *bin_count, int nb0, int nb1, int R, int nsb1,
                                int *sb_count, int *sb_start, int *sb_sub, int *work,
                                SubProb *items, int item, cudaStream_t stream)
{
    const int nsb = nb0 * nsb1;
    const int threads = 256;
    superbin_count_kernel<<<(nsb + threads - 1) / threads, threads, 0, stream>>>(
        bin_count, nb0, nb1, R, nsb1, sb_count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_bin_scan(sb_count, sb_start, sb_sub, work, nsb, item, stream);
    if (e != cudaSuccess) return e;
    fill_stripe_items_kernel<<<(nsb + threads - 1) / threads, threads, 0, stream>>>(
        sb_count, sb_sub, items, nsb, item);
    return cudaGetLastError();
}

template cudaError_t launch_node_bin<float>(const Geom &, const float *, int64_t, int *, int2 *,
                                            int *, cudaStream_t);
template cudaError_t launch_node_bin<double>(const Geom &, const double *, int64_t, int *, int2 *,
                                             int *, cudaStream_t);
template cudaError_t launch_node_scatter<float>(const Geom &, const float *, int64_t, const int2 *,
                                                const int *, RecF *, int *, cudaStream_t);
template cudaError_t launch_node_scatter<double>(const Geom &, const double *, int64_t,
                                                 const int2 *, const int *, RecD *, int *,
                                                 cudaStream_t);

int num_sms()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return v;
}

}  // namespace gbnfft
