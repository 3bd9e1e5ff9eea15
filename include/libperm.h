/*
 * libperm.h -- C ABI of libperm: matrix permanents on one GB300 (sm_103a).
 *
 * The permanent of an n x n matrix A is per(A) = sum over all permutations s of
 * {0..n-1} of prod_i a[i][s(i)]  (Su & Zheng, arXiv:1802.02779, Section 3.1,
 * Eq. (1)).  It is the quantity a boson-sampling amplitude is proportional to
 * (Section 2).  libperm evaluates it with two GPU methods:
 *
 *  - Store-zechin (Section 4): per(A) is developed along a row without signs
 *    (Section 3.1, property 4); every sub-permanent
 *        T_k[S] = per(rows 0..k-1, columns S),  |S| = k,
 *    is computed once, as  T_k[S] = sum_{j in S, ascending} a[k-1][j] * T_{k-1}[S \ {j}],
 *    stored, and reused by every larger minor that contains it.  This is the
 *    primary method.
 *  - Ryser's inclusion-exclusion formula (Section 3.3, Eqs. (2)-(4)) walked in
 *    Gray-code order.  It needs no tables and is the fallback when the
 *    Store-zechin tables do not fit the memory budget (and for n > 35).
 *    For integer matrices it is also the default (PERM_METHOD_AUTO): on a
 *    GB300 its register-resident walk is faster than the integer tables at
 *    every order measured (n = 2..30), while for complex matrices Store-zechin
 *    is faster from n = 10 on.
 *
 * Element types
 *   PERM_C128  complex128 entries, row-major, interleaved (re, im) doubles --
 *              the layout of torch.complex128 / numpy.complex128.  Computed in
 *              IEEE binary64 (no reduced precision anywhere); the last sum of
 *              each method is compensated (double-double).
 *   PERM_U01   0/1 entries stored as int64.  Exact: computed modulo 2^64 or
 *              2^128 (or 2^192 with PERM_FLAG_WIDE), the width chosen per
 *              matrix from an upper bound on per(A) (min of the products of
 *              row sums and of column sums, and Bregman's bound), so the result
 *              is the exact permanent.
 *   PERM_I64   small nonnegative integer entries (each at most 2^40) stored as
 *              int64.  Exact as above (row/column-sum bound).
 *
 * Conventions
 *   - Matrices of one call are concatenated: matrix i starts at element
 *     offset_i = sum_{j<i} n_j^2 of `mats`.  Device buffers must be aligned to
 *     their element type (16 bytes for complex128 -- as torch and cudaMalloc
 *     give them).
 *   - n = 0 is allowed and gives per = 1 (empty product).  1 <= n <= 35 may use
 *     Store-zechin; Ryser accepts n <= 40 (complex) and n <= 40 (integers).
 *   - Results: PERM_C128 -> double2 out[count] (re, im).  Integer types ->
 *     uint64 out[2*count], (low, high) words of a 128-bit unsigned value; with
 *     PERM_FLAG_WIDE uint64 out[4*count], the four words of a 256-bit unsigned
 *     value, least significant first (the fourth is always zero).
 *   - `item_status` (optional, device int[count]) receives PERM_OK, or
 *     PERM_EOVERFLOW when the bound reaches 2^128 (2^192 with PERM_FLAG_WIDE
 *     and Ryser; the result is then per(A) modulo that power of two), or
 *     PERM_EINVAL for an entry that is negative, above 2^40, or not 0/1 for
 *     PERM_U01.
 *
 * Ownership: the caller owns every input and output buffer; the library owns
 * its workspace (Store-zechin tables, Ryser partial sums, item descriptors),
 * allocated in perm_plan_create and freed in perm_plan_destroy.  perm_batch
 * itself never allocates, except for the one-time graph set-up of
 * PERM_FLAG_GRAPH.
 *
 * Errors: argument errors are returned synchronously and nothing is launched.
 * CUDA failures map to PERM_ECUDA.  Per-matrix conditions go to item_status.
 * No function aborts the process.
 *
 * Thread safety: a plan may be used by one host thread at a time, and the work
 * of two calls on one plan must not overlap on the GPU (they share the plan's
 * workspace): use one stream per plan, or one plan per stream.  Different plans
 * are independent.
 */
#ifndef LIBPERM_H
#define LIBPERM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum perm_status {
    PERM_OK = 0,
    PERM_EINVAL = 1,      /* bad argument (size, pointer, dtype, method) */
    PERM_ENOMEM = 2,      /* workspace does not fit the budget or the device */
    PERM_EOVERFLOW = 3,   /* integer bound >= 2^128, or 2^192 with PERM_FLAG_WIDE (per-item status) */
    PERM_ECUDA = 4,       /* a CUDA runtime call failed */
    PERM_EAGAIN = 5,      /* try again: queue full (submit) or not done (poll) */
    PERM_ETIMEDOUT = 6,   /* a bounded wait gave up */
    PERM_ESHUTDOWN = 7,   /* the server is shutting down */
    PERM_ENOTFOUND = 8    /* unknown ticket */
} perm_status;

typedef enum perm_dtype {
    PERM_C128 = 1,
    PERM_U01 = 2,
    PERM_I64 = 3
} perm_dtype;

typedef enum perm_method {
    PERM_METHOD_AUTO = 0,   /* complex: Store-zechin when its tables fit, else Ryser;
                               integers: Ryser (the faster method on GB300) */
    PERM_METHOD_SZ = 1,     /* Store-zechin only (PERM_ENOMEM if it cannot fit) */
    PERM_METHOD_RYSER = 2   /* Ryser / Gray code only */
} perm_method;

/* perm_opts.flags */
#define PERM_FLAG_PLAIN 1u    /* one kernel launch per matrix (the unbatched baseline) */
#define PERM_FLAG_GRAPH 2u    /* capture each batch shape as a CUDA graph and replay it: the
                                 first perm_batch call with a given (sizes, mats, out,
                                 item_status) on a non-default stream allocates a small
                                 descriptor buffer, captures and instantiates a graph; later
                                 calls with the same signature only launch the graph (16 are
                                 cached per plan, least recently used evicted) */
#define PERM_FLAG_AUTOTUNE 4u /* at plan creation, time candidate launch shapes on synthetic
                                 batches and keep the fastest: the batched Store-zechin kernel's
                                 CTA size and chain width; for complex plans of n_max >= 21 also
                                 the largest order run one CTA per matrix (19..22) and the layer
                                 path's CTA size, chain width and CTAs per launch for orders up
                                 to 24.  Results are
                                 bit-identical for every choice; perm_plan_describe reports
                                 them; cached per (device, dtype, n_max) for the process and in
                                 the file LIBPERM_TUNE_CACHE names, if set */
#define PERM_FLAG_WIDE 8u     /* integer plans only (PERM_EINVAL for PERM_C128): results are
                                 256-bit slots (four uint64 per matrix), and Ryser computes
                                 modulo 2^192, so every permanent whose bound is below 2^192 is
                                 exact -- all 0/1 matrices up to n = 40 (40! < 2^160).
                                 Store-zechin (PERM_METHOD_SZ) stays at most 128 bits wide and
                                 reports PERM_EOVERFLOW above that */

typedef struct perm_opts {
    size_t mem_budget_bytes;  /* workspace cap; 0 = 45% of the free device memory */
    int max_batch;            /* matrices per perm_batch call; 0 = 65536 */
    int method;               /* perm_method */
    unsigned flags;           /* PERM_FLAG_* */
    int ctas_per_sm;          /* persistent CTAs per SM for batched launches; 0 = tuned */
    int low_cols;             /* Store-zechin low-column count m, 1..13 (shared-memory chain width), for every
                                 launch of the plan; 0 = the defaults: 12 for the batched kernel and for
                                 more than four matrices of an order <= 24 per launch, 13 above order 24,
                                 and for at most four matrices of an order n <= 24 (one dataflow launch)
                                 floor((n - 1 + floor(log2 count)) / 2) clamped to 9..12 */
} perm_opts;

typedef struct perm_plan_s *perm_plan_t;
typedef struct perm_server_s *perm_server_t;

/* Create a plan for matrices of order <= n_max and element type `dtype` on the
   current CUDA device.  `opts` may be NULL (all defaults).  Allocates the
   workspace.  Returns PERM_EINVAL for n_max outside [0, 40] or a bad dtype,
   PERM_ENOMEM if the workspace does not fit (with PERM_METHOD_SZ forced). */
perm_status perm_plan_create(int n_max, perm_dtype dtype, const perm_opts *opts,
                             perm_plan_t *out);

/* Free a plan and its workspace (synchronises the device first). NULL is a no-op. */
perm_status perm_plan_destroy(perm_plan_t plan);

/* Workspace bytes the plan holds on the device. */
size_t perm_plan_workspace_bytes(perm_plan_t plan);

/* A JSON description of the plan's choices (methods' order limits, chain widths,
   CTA size, grid, workspace, whether it was autotuned), written like snprintf
   into buf[len]; returns the length it needed, or -1 for a NULL plan. */
int perm_plan_describe(perm_plan_t plan, char *buf, size_t len);

/* Permanents of `count` matrices, asynchronously on `stream` (a cudaStream_t;
   NULL = the legacy default stream).
     mats        device pointer, concatenated row-major matrices (see above)
     sizes       HOST int[count], each in [0, n_max]
     out         device pointer, double2[count], uint64[2*count], or uint64[4*count]
                 with PERM_FLAG_WIDE
     item_status device int[count] or NULL
   The call returns once the work is enqueued.  Inputs must stay valid and
   unmodified until the stream reaches that point. */
perm_status perm_batch(perm_plan_t plan, const void *mats, const int *sizes, int count,
                       void *out, int *item_status, void *stream);

/* Like perm_batch with HOST buffers: copies the matrices in, computes, copies
   the results (and statuses, if item_status != NULL) back, and synchronises
   `stream` before returning.  mats/out/item_status are host pointers. */
perm_status perm_batch_host(perm_plan_t plan, const void *mats, const int *sizes, int count,
                            void *out, int *item_status, void *stream);

/* Continuous-batching server (one device; the server owns its streams, and
   `stream` is ignored).  Requests of any n and dtype are queued, batched with
   whatever else is waiting, and completed asynchronously; work of different
   requests overlaps on the device.
     perm_submit copies the host matrix (n*n elements of `dtype`) and returns a
       ticket; PERM_EAGAIN if the queue is full.
     perm_poll returns PERM_EAGAIN until the ticket is done, then writes the 16
       result bytes (double2, or (low, high) uint64) and the item status; a
       server created with PERM_FLAG_WIDE writes 32 bytes for integer requests
       (four uint64, as perm_batch with that flag).
     perm_server_destroy stops the server; PERM_ETIMEDOUT if in-flight work
       does not finish within timeout_ms (the server is then left to drain in
       the background and its memory is not freed; at process exit its worker
       thread is stopped and joined before the CUDA runtime shuts down).
   Three lanes, by cost, each on streams of its own priority:
     - complex n <= 20 and integer n <= 28: one batch of every pending request
       as soon as the previous batch is done (highest priority);
     - complex 21 <= n <= 35 whose Store-zechin tables fit mem_budget_bytes:
       up to four jobs at once (a job: requests of one order, up to 16),
       admitted first come, first served while a contiguous free range of the
       budget holds the job's tables; each job's range is freed when the job
       finishes;
     - every other request with Ryser, batches of up to 64 requests and about
       0.7 s of work (a larger request runs alone; lowest priority).
   Server options: mem_budget_bytes = Store-zechin table budget (0 = min(100 GB,
   40 % of the free memory), reserved at creation); max_batch = queue
   capacity (0 = 65536); flags: PERM_FLAG_WIDE as for plans; the other fields
   are ignored.  Every result is the bits perm_batch gives for that matrix
   (PERM_METHOD_AUTO; PERM_METHOD_RYSER for the Ryser lane). */
perm_status perm_server_create(const perm_opts *opts, void *stream, perm_server_t *out);
perm_status perm_submit(perm_server_t server, const void *host_mat, int n, perm_dtype dtype,
                        uint64_t *ticket);
perm_status perm_poll(perm_server_t server, uint64_t ticket, void *out, int *item_status);
perm_status perm_server_destroy(perm_server_t server, int timeout_ms);

/* Amplitudes of all collision-free output patterns of boson-sampling inputs in
   one Store-zechin pass (Section 2: an amplitude is the permanent of the
   submatrix of the input rows and the pattern's output columns; Section 4's
   stored sub-permanents of the rows x cols matrix at level `rows` are exactly
   those permanents).
     mats   device pointer, `count` complex128 matrices of rows x cols, row-major
            (the input rows of the unitary restricted to the output modes)
     out    device pointer, count * C(cols, rows) double2: for matrix i, entry r is
            the permanent of the rows x rows submatrix whose columns are the r-th
            rows-subset of {0..cols-1} in colex order (subsets ordered by their
            largest element, then the next largest, ...)
   1 <= rows <= cols <= 13.  Each value is bit-identical to perm_batch on that
   submatrix.  Asynchronous on `stream`; PERM_EINVAL for bad sizes/pointers. */
perm_status perm_patterns(const void *mats, int count, int rows, int cols, void *out, void *stream);

/* Amplitudes of ALL output patterns, collisions included, in one pass.  An
   output pattern of `rows` photons in `cols` modes is a multiset M (mode j
   occupied t_j times); its amplitude is the permanent of the rows x rows matrix
   of the input rows and the columns of M with repetition (probability
   |per|^2 / prod_j t_j!).  Developing along a row (Section 3.1, property 4)
   gives T_k[M] = sum_{j in M} t_j a[k-1][j] T_{k-1}[M - j], which is evaluated
   level by level.
     out   count * C(cols + rows - 1, rows) double2; entry r of matrix i is the
           multiset whose sorted modes m_0 <= ... <= m_{rows-1} map to the r-th
           rows-subset {m_p + p} of {0..cols+rows-2} in colex order
   1 <= rows, cols <= 13 and 2 * C(cols + rows - 1, rows) <= 12000 (two levels in
   shared memory), else PERM_EINVAL.  Complex128, FP64 (last level
   double-double); asynchronous on `stream`. */
perm_status perm_patterns_multiset(const void *mats, int count, int rows, int cols, void *out,
                                   void *stream);

/* Store-zechin permanent of ONE matrix without allocating any device memory.
   The paper has no counterpart to this entry point.  It exists for callers
   that cannot call cudaMalloc: code inside a framework whose memory pool owns
   every byte of device memory (an allocation behind the pool's back can fail or
   starve it), and loops that cannot afford the device-wide synchronisation an
   allocation may cause.
     mat          device pointer, n*n row-major elements of `dtype`
     out          device pointer: double2 (PERM_C128) or two uint64 (integers)
     item_status  device int or NULL (PERM_OK, PERM_EOVERFLOW, PERM_EINVAL)
   The chain tables live in a fixed 64 MiB scratch array inside the library's
   device image, held on every device that loads the library until the process
   exits.  That bounds n: at most 22 for PERM_C128 and 23 for the integer types;
   larger n (and n < 0, a bad dtype or a NULL pointer) return PERM_EINVAL and
   launch nothing.  n = 0 gives 1.
   The first call on a device does a one-time set-up with that device current
   (it looks up the scratch address with cudaGetSymbolAddress and, unless a plan
   already did, uploads a 16 KB index table with cudaMemcpyToSymbol), so make
   that first call before any stream capture.  The work is asynchronous on
   `stream`.  Every call shares the one scratch array, which keeps the last
   call's contents (nothing in it has to start at zero: every table entry is
   written before it is read); calls whose work overlaps on the GPU, from
   different streams or threads, race on it and must be serialised by the
   caller.  Results are bit-identical to perm_batch with PERM_METHOD_SZ. */
perm_status perm_sz_noalloc(const void *mat, int n, perm_dtype dtype, void *out, int *item_status,
                            void *stream);

/* ONE large matrix by Ryser's formula split over several GPUs (Section 3.3,
   Eq. (4); for complex and 0/1 input Glynn's half-size form).  The codes of an
   order-n matrix are cut into a fixed number of pieces (a function of n and
   dtype only), the pieces perm_batch itself uses.  Each GPU (rank) computes the
   partial sums of a contiguous range of pieces; the ranks' partial sums are
   gathered in piece order (any transport: an all-gather, host copies), and one
   finishing call sums all of them in perm_batch's fixed order.  The result is
   therefore bit-identical to perm_batch with PERM_METHOD_RYSER, whatever the
   number of ranks.
     perm_ryser_pieces   host only (no GPU call): the number of pieces of an
                         order-n matrix and the bytes of one piece's partial sum
                         (32 for PERM_C128: two double-doubles; 40 for integers:
                         a 256-bit modular sum and a word of width/status).
                         PERM_EINVAL for n outside [1, 40] or a bad dtype.
     perm_ryser_split    host only: rank's share [*begin, *end) of `pieces`
                         pieces among `world` ranks (contiguous, balanced: sizes
                         differ by at most one).  PERM_EINVAL for pieces < 1,
                         world < 1 or rank outside [0, world).
     perm_ryser_partials partial sums of pieces [begin, end) of the matrix `mat`
                         (device, n*n elements of the plan's dtype) into
                         `partials` (device, (end - begin) * piece bytes), async
                         on `stream`.  The plan supplies dtype and width (its
                         PERM_FLAG_WIDE) and 1 <= n <= its n_max, else
                         PERM_EINVAL; begin == end launches nothing.
     perm_ryser_finish   sums `partials` (device, ALL pieces of the matrix in
                         piece order) and writes the permanent to `out` (device,
                         as perm_batch writes one result) and `item_status`
                         (device int or NULL), async on `stream`.
   The calls of one plan must be ordered on the GPU (one stream), as for
   perm_batch.  The caller owns every buffer. */
perm_status perm_ryser_pieces(int n, perm_dtype dtype, long long *pieces, size_t *piece_bytes);
perm_status perm_ryser_split(long long pieces, int rank, int world, long long *begin, long long *end);
perm_status perm_ryser_partials(perm_plan_t plan, const void *mat, int n, long long begin, long long end,
                                void *partials, void *stream);
perm_status perm_ryser_finish(perm_plan_t plan, int n, const void *partials, void *out, int *item_status,
                              void *stream);

/* Short text for a status code (static storage). */
const char *perm_strerror(perm_status status);

/* Library version as "major.minor.patch" (static storage). */
const char *perm_version(void);

/* Measurement helper: sustained FP64 fused-multiply-add throughput of the
   current device in FLOP/s (2 per FMA), timed with CUDA events over `ms_target`
   milliseconds of independent FMA chains on every SM.  Used as the roofline
   denominator for the complex kernels.  Returns PERM_ECUDA on failure. */
perm_status perm_measure_fp64_peak(double ms_target, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* LIBPERM_H */
