/*
 * gbnfft.h - C ABI of a nonequispaced fast Fourier transform (NFFT) for one NVIDIA GB300 GPU.
 *
 * The library computes, for d = 1, 2 or 3, the NFFT of Schmischke, "NFFT Interface for Julia"
 * (arXiv 1810.09891), Section 2:
 *
 *   forward (Algorithm "NFFT"):          f_j   ~ sum_{k in I_N} fhat_k e^{-2 pi i k.x_j},
 *                                        computed as f = B F D fhat,
 *   adjoint (Algorithm "adjoint NFFT"):  hhat_k ~ sum_j f_j e^{+2 pi i k.x_j},
 *                                        computed as hhat = D^H F^H B^H f,
 *
 * with nodes x_j on the torus T^d = [-1/2, 1/2)^d, the index set
 * I_N = { k : -N_t/2 <= k_t <= N_t/2 - 1 } (Section 2, eq. index_set), an oversampled FFT grid
 * of size n = sigma N and a Kaiser-Bessel window truncated to |n_t x_t - l_t| <= m
 * (Section 2, eq. window_cutoff and eq. Inm). D divides by the window's Fourier coefficients and
 * zero-pads, F is the d-variate FFT of size n, B interpolates the grid at the nodes with the
 * window, and B^H spreads node values onto the grid (the transposed index set of Section 2).
 *
 * Every call that computes runs hand-written CUDA kernels (sm_103a) on the plan's stream and
 * returns without waiting for them. There is no CPU fallback: a call either enqueues GPU work
 * or returns an error code.
 *
 * Memory and layout (all device pointers unless the function name ends in _host):
 *   - Complex values are interleaved (re, im): float2 for NFFT_FP32, double2 for NFFT_FP64.
 *   - fhat / hhat: |I_N| complex values, row-major over (k_0, ..., k_{d-1}) with axis t at
 *     position k_t + N_t/2 (the centred order of the paper's Julia example, Section 4.2,
 *     extended row-major to d > 1).
 *   - x: M x d reals of the plan's precision, row-major (node j, coordinate t). Any finite real
 *     is accepted; it is taken modulo 1 (the torus).
 *   - f: M complex values in the caller's node order.
 *   - Pointers must be aligned to one complex value (8 bytes FP32, 16 bytes FP64); the caller
 *     owns all of them. No input array is modified.
 *
 * Errors: every function returns an nfft_status_code. Argument errors are detected on the host
 * before anything is enqueued. Errors found on the GPU (a node that is NaN or infinite) are
 * recorded in a device-side status word and reported by nfft_status() (which waits for the
 * stream). For tests of the out-of-memory paths, the environment variable GBNFFT_FAIL_ALLOC
 * makes the library refuse its own device allocations on the host, as if the device were out of
 * memory (NFFT_ENOMEM): it names the allocation sites to refuse, comma-separated ("tables" in
 * nfft_plan_create, "workspace" in nfft_set_nodes, "stage" in the _host calls, "lin" in
 * NFFT_OPT_WINDOW_TABLE, "batch" in the first fused batch call), or "all". It is read at every
 * allocation.
 *
 * Tracing: every stage of every call is wrapped in an NVTX range named "gbnfft <stage>" (see
 * enum nfft_stage), visible in any profiler that records NVTX.
 *
 * Threads: a plan is not thread-safe; distinct plans may be used from distinct threads.
 */
#ifndef GBNFFT_H
#define GBNFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbnfft_plan *nfft_plan;

/* Precision of x, fhat, f and the internal grid. */
enum nfft_dtype { NFFT_FP32 = 0, NFFT_FP64 = 1 };

enum nfft_status_code {
    NFFT_OK = 0,
    NFFT_EINVAL = 1,      /* bad argument: dimension, size, null or misaligned pointer */
    NFFT_ENOMEM = 2,      /* a device allocation failed, or the workspace given is too small */
    NFFT_ECUDA = 3,       /* a CUDA runtime call failed */
    NFFT_ENOTREADY = 4,   /* a transform was requested before nfft_set_nodes */
    NFFT_EBADNODE = 5,    /* a node coordinate was NaN, infinite or too large (|n x| >= 2^52) */
    NFFT_ETIMEOUT = 6,    /* reserved: a bounded device-side wait gave up */
    NFFT_EUNSUPPORTED = 7, /* valid for the paper's method but not built here (see below) */
    NFFT_ESCRATCH = 8      /* larger than the fixed scratch of nfft_trafo_1d_noalloc */
};

/* Plan creation: Section 3.1, Table tab:params (N, M, n, m) plus the precision.
 *   d      1, 2 or 3.
 *   N      d even bandwidths, N_t >= 2 (Section 2, eq. index_set: N in 2 N^d).
 *   M      number of nodes, M >= 0 and M < 2^31.
 *   n      d FFT lengths, or NULL for the paper's default n_t = 2^(ceil(log2 N_t) + 1)
 *          (Section 2, after eq. gl). Each n_t must be even and > N_t (Section 3.1). Powers of
 *          two up to 16384 (FP32) / 8192 (FP64) use the radix-8/4/2 FFT; other even lengths up
 *          to 4096 (FP32) / 2048 (FP64) use Bluestein's chirp transform (the workspace grows by
 *          two buffers of |I_n| / n_t x M values, M the power of two >= 2 n_t - 1). Larger
 *          lengths, |I_n| >= 2^31 or more than 31 bits of packed cell index (sum over the
 *          axes of ceil(log2 n_t)) give NFFT_EUNSUPPORTED.
 *   m      window cutoff, 1 <= m <= 8, with 2m + 2 <= n_t; m <= 0 selects the paper's default 8
 *          (Section 3.1).
 *   dtype  NFFT_FP32 or NFFT_FP64.
 * The plan binds the calling thread's current CUDA device and the legacy default stream; it
 * owns small device tables (window factors, twiddles, a status word), allocated here. */
int nfft_plan_create(nfft_plan *out, int d, const int64_t *N, int64_t M, const int64_t *n,
                     int m, int dtype);

/* Release the plan, its tables and any workspace it allocated itself. NULL is accepted. */
int nfft_destroy(nfft_plan plan);

/* Make every later call enqueue on this CUDA stream (a cudaStream_t; NULL = legacy default).
 * A plan keeps separate grids for the forward transform (and the node gradient) and for the
 * adjoint, so one forward (or node gradient) and one adjoint may run at the same time on two
 * streams. Any other two calls of a plan on different streams share workspace and must be
 * ordered by the caller (an event, or a synchronisation); nfft_set_nodes must be ordered
 * before and after every transform. */
int nfft_set_stream(nfft_plan plan, void *cuda_stream);

/* Device workspace the plan needs: oversampled grids (one set for the forward transform, one
 * for the adjoint), sorted node records, bin tables. */
int nfft_workspace_size(nfft_plan plan, size_t *bytes);

/* Hand the plan a caller-owned device workspace of at least nfft_workspace_size() bytes,
 * aligned to 256 bytes. It must stay valid until the plan is destroyed or given another one.
 * Without this call, nfft_set_nodes allocates the workspace itself (owned by the plan). */
int nfft_set_workspace(nfft_plan plan, void *dev_ptr, size_t bytes);

/* Precomputation for a node set (the paper's "precomputation" of Section 4.2, NFFT_SORT_NODES
 * of Table tab:nfftflags): for every node, the grid cell floor(n_t x_t) and the offset inside
 * it (computed in FP64 for both precisions), then a counting sort of the nodes into tiles of
 * the grid. x (M x d, device) may be freed once the stream has passed this call. */
int nfft_set_nodes(nfft_plan plan, const void *x);

/* Forward NFFT, Algorithm "NFFT": f = B F D fhat. fhat: |I_N| complex, f: M complex. */
int nfft_trafo(nfft_plan plan, const void *fhat, void *f);

/* Adjoint NFFT, Algorithm "adjoint NFFT": hhat = D^H F^H B^H f. f: M complex,
 * hhat: |I_N| complex. */
int nfft_adjoint(nfft_plan plan, const void *f, void *fhat);

/* Node gradient (derivative of the approximation s of Section 2, eq. s_approx, with respect
 * to the node coordinates): gx[j*d + t] = Re( conj(w_j) * d s_c / d x_t (x_j) ), where s_c is
 * the NFFT approximation built from the coefficients c (|I_N| complex) and w (M complex) is one
 * weight per node. For a real loss L of f = NFFT(fhat, x) (PyTorch's convention for complex
 * gradients), dL/dx = nfft_grad_x(c = fhat, w = dL/df); for hhat = NFFT^H(f, x),
 * dL/dx = nfft_grad_x(c = dL/dhhat, w = f). gx: M x d reals of the plan's precision. */
int nfft_grad_x(nfft_plan plan, const void *coef, const void *w, void *gx);

/* Host-buffer versions: copy the inputs from host memory to device buffers owned by the plan
 * (allocated on first use), run the transform, copy the result back, and wait for the stream.
 * Pinned host memory makes the copies asynchronous and faster; pageable memory also works. */
int nfft_set_nodes_host(nfft_plan plan, const void *x_host);
int nfft_trafo_host(nfft_plan plan, const void *fhat_host, void *f_host);
int nfft_adjoint_host(nfft_plan plan, const void *f_host, void *fhat_host);

/* Wait for the plan's stream and return the first error any kernel recorded since the last
 * call (NFFT_OK if none), then clear it. A CUDA error seen while waiting gives NFFT_ECUDA. */
int nfft_status(nfft_plan plan);

/* Batches: many independent transforms of uneven N and M run concurrently (the paper's plan
 * of Section 3.1, many times over). A batch borrows `count` plans created on one device (they
 * stay owned by the caller and must outlive the batch; their nodes are set with
 * nfft_set_nodes as usual). Every batch call enqueues on the batch's stream
 * (nfft_batch_set_stream; NULL = legacy default): it forks into `streams` side streams owned by
 * the batch (0 = 8, at most count and 64), runs plan i on side stream lane i (plans assigned
 * largest first to the least-loaded lane, work ~ M_i + |I_n,i|; the plan's own stream is
 * restored afterwards) and joins the side streams back into the batch's stream, so later work
 * on that stream sees every result. The calls record into a CUDA graph as parallel branches.
 * A plan may appear only once in a batch (a repeated plan gives NFFT_EINVAL: its two copies
 * would run at once over one workspace). Pointer arrays hold one device pointer per plan, with
 * the layouts of nfft_trafo, nfft_adjoint and nfft_grad_x. Every plan is checked (nodes set, pointers non-null and
 * aligned) before any work is enqueued; a failure returns NFFT_ENOTREADY or NFFT_EINVAL with
 * nothing enqueued. A CUDA error while enqueuing stops issuing the remaining plans, still joins
 * the side streams, and returns NFFT_ECUDA. The arrays are read during the call only. */
typedef struct gbnfft_batch *nfft_batch;
int nfft_batch_create(nfft_batch *out, const nfft_plan *plans, int count, int streams);
/* Wait for the batch's side streams and release them. NULL gives NFFT_EINVAL. */
int nfft_batch_destroy(nfft_batch batch);
int nfft_batch_set_stream(nfft_batch batch, void *cuda_stream);
/* Number of plans and of side streams (either pointer may be NULL). */
int nfft_batch_size(nfft_batch batch, int *count, int *streams);
/* Side stream lane of plan i, or -1 for an invalid batch or index. */
int nfft_batch_lane(nfft_batch batch, int i);
/* Forward NFFT of every plan: f[i] = NFFT_i(fhat[i]). */
int nfft_batch_trafo(nfft_batch batch, const void *const *fhat, void *const *f);
/* Adjoint NFFT of every plan: fhat[i] = NFFT_i^H(f[i]). */
int nfft_batch_adjoint(nfft_batch batch, const void *const *f, void *const *fhat);
/* Node gradient of every plan: gx[i] = nfft_grad_x(plan i, coef[i], w[i]). */
int nfft_batch_grad_x(nfft_batch batch, const void *const *coef, const void *const *w,
                      void *const *gx);

/* Fused execution of a batch. When the plans qualify - at most 128 plans, all d = 2 and
 * NFFT_FP32, one m and one window kind, power-of-two n_t in 16..4096, the polynomial window
 * (NFFT_OPT_WINDOW_TABLE 0), automatic or half-warp
 * spreading (NFFT_OPT_SPREAD_METHOD 0 or 5) and automatic or thread interpolation - every batch
 * call runs each stage for all plans in one launch on the batch's stream: the FFT passes over a
 * work list of (plan, lines) blocks, the interpolation and node gradient over (plan, 128 nodes)
 * blocks, and the spreading over the plans' subproblem lists concatenated and claimed by
 * persistent warps (the register-tile form 8, when every plan spreads automatically with sort
 * bins of one height, 4 or 8 rows) or CTAs (the half-warp form 5). The first fused call allocates the per-plan tables (device memory and pinned
 * host memory), uploads them on the batch's stream and waits for the upload; a call after a
 * plan's workspace or tuning changed rebuilds them the same way. Make such a call before
 * capturing the batch's calls into a CUDA graph (allocation and waiting are not allowed during
 * capture). A batch whose plans no longer qualify runs plan by plan on the side streams. Results equal
 * those of the plans' own calls up to the order of floating-point additions in the spreading.
 * nfft_batch_set_fused(batch, 0) turns fused execution off (plan by plan on side streams, the
 * default when the plans do not qualify); enable = 1 turns it on (the default) and returns
 * NFFT_EUNSUPPORTED if the plans do not qualify. nfft_batch_get_fused reports whether the next
 * call runs fused. */
int nfft_batch_set_fused(nfft_batch batch, int enable);
int nfft_batch_get_fused(nfft_batch batch, int *fused);

/* Plan parameters after defaults: d, N[3], n[3], M, m, dtype, the tile (bin) size used to
 * sort the nodes, the workspace size and the window (NFFT_OPT_WINDOW). Unused trailing entries
 * are 0. */
typedef struct nfft_info {
    int d;
    int m;
    int dtype;
    int64_t M;
    int64_t N[3];
    int64_t n[3];
    int64_t bin[3];
    size_t workspace_bytes;
    int window;
    int window_table; /* NFFT_OPT_WINDOW_TABLE (0 = polynomial window) */
} nfft_info;
int nfft_get_info(nfft_plan plan, nfft_info *info);

/* Per-stage timing with CUDA events recorded on the plan's stream. While enabled, every call
 * records one event pair around each stage it runs; nfft_profile_read waits for the stream,
 * adds up the elapsed milliseconds per stage into ms[stage] (and the number of timed calls into
 * count[stage] when count is not NULL) for stages < nstages, and forgets the recorded pairs.
 * nfft_profile(plan, 0) stops recording; enabling also forgets earlier pairs. */
enum nfft_stage {
    NFFT_STAGE_SET_NODES = 0,   /* node cell/offset + counting sort + subproblem list */
    NFFT_STAGE_FFT_FORWARD = 1, /* D and F: the pruned forward FFT passes */
    NFFT_STAGE_INTERP = 2,      /* B: window interpolation */
    NFFT_STAGE_ZERO_GRID = 3,   /* clearing the grid before spreading */
    NFFT_STAGE_SPREAD = 4,      /* B^H: tiled spreading */
    NFFT_STAGE_FFT_ADJOINT = 5, /* F^H and D^H: the pruned inverse FFT passes */
    NFFT_STAGE_GRAD = 6,        /* node-gradient interpolation */
    NFFT_NUM_STAGES = 7
};
int nfft_profile(nfft_plan plan, int enable);
int nfft_profile_read(nfft_plan plan, double *ms, int64_t *count, int nstages);

/* Plan options. NFFT_OPT_WINDOW selects the window function (Section 4.1 names the choices;
 * the default is Kaiser-Bessel); it changes the result (the approximation error, not the
 * exact transform the plan approximates). The others only tune speed and never change the
 * result beyond rounding.
 *   NFFT_OPT_WINDOW         0 Kaiser-Bessel psi(t) = sinh(b sqrt(m^2 - t^2)) / (pi sqrt(...)),
 *                           b = pi (2 - 1/sigma); 1 Gaussian psi(t) = exp(-t^2 / b),
 *                           b = 2 sigma m / ((2 sigma - 1) pi); 2 B-spline psi(t) = M_2m(t),
 *                           the centred cardinal B-spline of order 2m; 3 sinc
 *                           psi(t) = sinc^2m(pi a t), a = (2 sigma - 1) / (2 m sigma). t is in
 *                           grid units (t = n_t x_t), sigma = n_t / N_t per axis, and psi is cut
 *                           off to |t| <= m. The node precomputation stays valid. Waits for the
 *                           device to go idle, then rewrites the plan's tables in place; a CUDA graph
 *                           captured before the change keeps the old edge constants in its
 *                           kernel arguments and must be captured again.
 *   NFFT_OPT_SPREAD_METHOD  0 automatic, 1 one thread per node with shared-memory atomics,
 *                           2 one warp per node with shared-memory atomics,
 *                           3 one warp per node with a private tile per warp (no atomics),
 *                           4 (d = 2) eight lanes per node, a private tile per eight lanes,
 *                           5 (d = 2) sixteen lanes per node, a private tile per half-warp,
 *                           6 (d = 3) one tile per CTA, its planes along axis 0 owned by the
 *                           CTA's warps (no atomics, no private copies),
 *                           7 (d = 2) one tile per CTA over a super-bin of stripes of whole bins
 *                           along the last axis (each at least 2m cells wide); the CTA's
 *                           half-warps spread the even stripes together, then the odd ones (no
 *                           atomics, no private copies). Needs a last-axis bin of at most
 *                           2m rounded up to a power of two and n_(d-1) >= 16 such stripes + 2m,
 *                           8 (d = 2) no shared-memory tile: a group of lanes (a half-warp when
 *                           the last-axis bin + 2m <= 16, else a warp) holds a subproblem's whole
 *                           tile in registers, lane c all rows of tile column c; each node's
 *                           row weights are staged at its tile rows, so a node costs every lane
 *                           one multiply-add per tile row. Needs a last-axis bin + 2m <= 32 and
 *                           an axis-0 bin of 4 or 8.
 *                           Automatic: 8 for d = 2 in FP32, 5 for d = 2 in FP64, 6 for d = 3.
 *                           A form whose tile does not fit or whose d does not match runs as
 *                           the nearest form that fits (6 -> 2 -> 1, 7 -> 5, 8 -> 5,
 *                           4/5 -> 3 -> 2 -> 1).
 *   NFFT_OPT_INTERP_METHOD  0 automatic, 1 one thread per node (gathers from the grid),
 *                           2 one warp per node, 3 one thread per node gathering from a
 *                           shared-memory tile of the node's bin, 4 (d = 2, 3 and m <= 4;
 *                           else 1) eight lanes per node reading contiguous row segments.
 *   NFFT_OPT_BIN_0..2       bin (tile) size on axis 0..d-1: a power of two, 0 = default (1-D
 *                           1024; 2-D 4 x 8 in FP32 with m <= 4, else 8 x 16; 3-D 8 x 8 x 16);
 *                           clipped to n_t (power-of-two n_t) or to the largest power of two
 *                           <= n_t / 2 (other n_t, whose last bin is then partial).
 *                           Changing a bin size discards the node precomputation (call
 *                           nfft_set_nodes again) and may change nfft_workspace_size: a
 *                           caller-owned workspace that became too small makes nfft_set_nodes
 *                           return NFFT_ENOMEM.
 *   NFFT_OPT_WINDOW_TABLE   K = 0 (default): the window is evaluated from per-tap polynomials
 *                           fitted to FP32 / FP64 accuracy. K in 2..65536: PRE_LIN_PSI
 *                           (Section 3.1, Table tab:nfftflags) - the window is read from a
 *                           table of its values at K points per unit of t = n_t x and linearly
 *                           interpolated (error ~ K^-2 max|psi''| / 8, so it changes the result).
 *                           The node derivative at a table sample is the slope of the segment
 *                           above it (from inside the support at t = +m). The table (d x (K+1)
 *                           x 2m values, plan precision) is allocated here and rebuilt when the
 *                           window changes; waits for the device to go idle.
 *   NFFT_OPT_SUBPROBLEM     nodes per spreading work item (a power of two in 32..1024, 0 = the
 *                           default: for 2-D FP32 64 with bins of at most 32 cells, else 128;
 *                           otherwise 1024): the sorted nodes of a bin are
 *                           cut into items of at most this many nodes. Like a bin size, it
 *                           discards the node precomputation and may change nfft_workspace_size.
 *   NFFT_OPT_STRIPE_ITEM    nodes per stripe in one work item of spreading form 7 (a power of
 *                           two in 8..65536, 0 = the default 64): a super-bin whose heaviest
 *                           stripe holds more nodes is cut into parts, each taking a share of
 *                           every stripe. Discards the node precomputation like a bin size. */
enum nfft_option {
    NFFT_OPT_SPREAD_METHOD = 1,
    NFFT_OPT_BIN_0 = 2,
    NFFT_OPT_BIN_1 = 3,
    NFFT_OPT_BIN_2 = 4,
    NFFT_OPT_INTERP_METHOD = 5,
    NFFT_OPT_WINDOW = 6,
    NFFT_OPT_SUBPROBLEM = 7,
    NFFT_OPT_WINDOW_TABLE = 8,
    NFFT_OPT_STRIPE_ITEM = 9
};
int nfft_set_option(nfft_plan plan, int key, int64_t value);

/* Static description of an error code. */
const char *nfft_strerror(int code);

/* Make `device` the calling thread's current CUDA device for this library (the device that the
 * next nfft_plan_create binds). */
int nfft_use_device(int device);

/* Forward 1-D NFFT in FP64 that allocates no device memory. The paper has no counterpart: its
 * library always allocates through its plan.
 *
 * For callers that cannot call cudaMalloc where they transform: code whose device memory is
 * owned by another allocator (a framework's caching pool or a host application's memory budget
 * that forbids raw allocations), and latency-bound loops that cannot take the device
 * synchronisation that cudaMalloc / cudaFree imply. The planned path cannot serve them, because
 * nfft_plan_create and nfft_set_nodes allocate.
 *
 * Computes f_j ~ sum_{k=-N/2}^{N/2-1} fhat_k e^{-2 pi i k x_j}, the same transform as nfft_trafo
 * on a 1-D NFFT_FP64 plan with the same N, n, m (Kaiser-Bessel window), up to rounding.
 *   N       even bandwidth, 2 <= N <= 4096.
 *   M       number of nodes, 0 <= M < 2^31.
 *   n       pointer to the FFT length (power of two, N < n <= 8192, 2m + 2 <= n), or NULL for
 *           the default 2^(ceil(log2 N) + 1).
 *   m       window cutoff 1..8 (<= 0 selects 8).
 *   x       M node coordinates (device, FP64), taken mod 1; |x_j| must be below 2^52 / n, and
 *           a node that is not finite or not below that bound gives NaN in f_j.
 *   fhat    N complex128 coefficients, index k + N/2 (device, 16-byte aligned).
 *   f       M complex128 outputs (device, 16-byte aligned).
 *   stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 * Scratch: a fixed 288 KiB array in device memory inside the library, held by every GPU that
 * loads the library until the process exits. Sizes beyond it (n > 8192 or N > 4096) return
 * NFFT_ESCRATCH. Nothing in it has to start at zero: each call rewrites what it reads. All calls
 * share the array: calls that overlap on the GPU (other streams, other threads) race and give
 * wrong results, so serialise them.
 * Set-up: the first call on a device looks up the array's device address there
 * (cudaGetSymbolAddress) and keeps it for the life of the process. The kept address does not
 * survive cudaDeviceReset (or any other destruction of the device's primary context): do not
 * call this entry point after one.
 * Returns without waiting for the GPU. */
int nfft_trafo_1d_noalloc(int64_t N, int64_t M, const int64_t *n, int m, const double *x,
                          const void *fhat, void *f, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBNFFT_H */
