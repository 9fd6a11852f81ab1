/*
 * pce.h -- C ABI of the convolution-product expansion library.
 *
 * The library applies the convolution-product expansion of order m
 *
 *     H_m u = sum_{k=0}^{m-1} h_k * (w_k . u)                 (Eq. 1.4)
 *
 * and its adjoint
 *
 *     H_m^* v = sum_{k=0}^{m-1} conj(w_k) . (h~_k * v),   h~_k[i] = conj(h_k[-i]),
 *
 * on a periodic 1D grid of N points or a periodic 2D grid of Ny x Nx points.
 * "*" is the periodic discrete convolution of Section 3.5,
 * v[i] = sum_j u[i - j] h[j] with indices taken modulo the grid size (per
 * axis), and "." the pointwise product.  The paper asks for products with
 * both H_m and H_m^* (Introduction; Corollaries 4.2 and 4.4); the adjoint
 * formula follows from the reality of h_k and w_k.  Every product is
 * evaluated with the FFT convolution identity of Section 3.5: one forward
 * FFT of w_k . u per term, a pointwise product with the precomputed spectrum
 * hhat_k, accumulation of the m products, one inverse FFT.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Arrays are float32, row-major, contiguous.  A 2D array is [Ny][Nx] with
 *   x fastest; a batch of right-hand sides is [batch][Ny][Nx] (or [batch][N]).
 * - h_k is given with its origin at index 0 (offset -d stored at index N-d).
 * - Spectra are R2C half spectra along x: [Ny][Nx/2+1] complex64 (interleaved
 *   re, im), forward DFT X[f] = sum_j x[j] exp(-2 i pi j f / N) (the sign of
 *   the Fourier atoms of Section 2), unnormalised; inverses carry 1/N.
 * - Sizes are powers of two: N in [16, 262144] in 1D, Ny and Nx in [16, 2048]
 *   in 2D.  m >= 1.  Other sizes return PCE_ERR_UNSUPPORTED.  1D sizes above
 *   8192 run a four-step FFT (column FFTs, twiddles, row FFTs over an
 *   NY x NX view of the sequence); on those plans PCE_FLAG_LOWP_STORAGE and
 *   pce_backward return PCE_ERR_UNSUPPORTED.
 * - Pointers named "device" must be CUDA device (or managed) memory of the
 *   current device; a host pointer returns PCE_ERR_INVALID.
 * - Calls are stream-ordered on `stream` (a cudaStream_t; NULL is the legacy
 *   default stream).  pce_apply and pce_apply_adjoint never synchronise the
 *   host and allocate nothing.
 * - Errors are returned as pce_status, never by aborting; the message of the
 *   last failure on the calling thread is available from
 *   pce_last_error_string().  A failed call leaves its outputs unspecified.
 * - A plan owns scratch buffers that every apply on it uses: two applies of
 *   the same plan must not run concurrently (e.g. on two streams).
 */
#ifndef PCE_H_
#define PCE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PCE_OK = 0,
    PCE_ERR_INVALID = 1,      /* bad argument: null/host pointer, in-place call, bad m or batch */
    PCE_ERR_UNSUPPORTED = 2,  /* size outside the supported set */
    PCE_ERR_OOM = 3,          /* a device allocation of the plan failed */
    PCE_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    PCE_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up */
} pce_status;

typedef struct pce_plan* pce_plan_t;

/* Plan flags. */
#define PCE_FLAG_NONE 0u
/*
 * PCE_FLAG_UNFUSED: applies on this plan run the plain unfused per-term
 * pipeline instead of the fused kernels (2D plans; 1D plans ignore it).  For
 * every term: a window kernel writes w_k . u to memory, a full 2D R2C (row
 * pass, column pass) writes its spectrum to memory, a kernel multiplies it by
 * hhat_k and accumulates; one inverse 2D FFT ends the forward apply (the
 * adjoint mirrors this).  It computes the same operator with the same FFT
 * core and exists as the baseline the fused path is measured against.
 */
#define PCE_FLAG_UNFUSED 1u
/*
 * PCE_FLAG_LOWP_STORAGE: the applies read the windows as bfloat16 and the
 * spectra as FP16 complex, each term's spectrum divided by a power of two
 * s_k = 2^ceil(log2 max |Re hhat_k|, |Im hhat_k|), which halves the bytes of
 * w and hhat an apply reads.  FFTs, products and accumulations stay FP32.
 * The plan's operator is the one with the rounded w_k and hhat_k
 * (pce_plan_hhat returns the rounded spectra).  Not combinable with
 * PCE_FLAG_UNFUSED; pce_backward returns PCE_ERR_UNSUPPORTED on such plans.
 */
#define PCE_FLAG_LOWP_STORAGE 2u
/*
 * PCE_FLAG_PRODUCT_CONVOLUTION: the plan's operator is the product-convolution
 * form P_m u = sum_k w_k . (h_k * u) (windows on the output side; Section 1)
 * instead of H_m u = sum_k h_k * (w_k . u).  pce_apply computes P_m u and
 * pce_apply_adjoint P_m^* v = sum_k h~_k * (w_k . v).  The plan stores the
 * spectra of h~_k = conj(hhat_k) and runs the other direction's kernels (one
 * forward FFT of u, per term a product and an inverse FFT, windowed
 * accumulation).  pce_plan_hhat still returns hhat_k; plans from spectra take
 * hhat_k.  Combines with the other flags; pce_backward and pce_apply_noalloc
 * return PCE_ERR_UNSUPPORTED on such plans.
 */
#define PCE_FLAG_PRODUCT_CONVOLUTION 4u
/*
 * PCE_FLAG_SECTIONED: applies convolve every term on sections (Lemma 3.2) of
 * 1024 rows x L columns and add the sections into the output (overlap-add;
 * atomic adds, so the rounding order varies from run to run).  Each term's
 * support box is cut into column tiles of L - (width of h_k's support) + 1
 * columns, one section per tile (h_k's exact nonzeros are found at plan
 * time); L, a power of two from 16 to 2048, is the width of least modelled
 * FFT work.  Pays when the
 * grid is much larger than box + support (e.g. 2048 x 2048 with boxes of 511
 * and 73-pixel PSFs: two 1024-point column FFTs per term instead of one
 * 2048-point one shared with the other terms).  2D plans from pce_plan_create
 * only, fused, convolution-product form; with PCE_FLAG_LOWP_STORAGE the
 * section spectra are stored as half2 with their own per-term power-of-two
 * scales and the windows as bfloat16.  Box rows + support rows - 1 <= 1024
 * and support columns <= 2048 for every term.
 * Otherwise PCE_ERR_UNSUPPORTED.  Gradients and pce_apply_noalloc use the
 * plan's whole-grid structures.
 */
#define PCE_FLAG_SECTIONED 8u

/*
 * pce_plan_create -- precompute everything an operator needs (Eq. 1.4).
 *
 *   out    : receives the plan handle (host pointer to a handle).
 *   ndims  : 1 or 2.
 *   shape  : host array [ndims]: {N} or {Ny, Nx}.
 *   m      : number of terms.
 *   w      : device, [m][shape] float32 windows w_k.
 *   h      : device, [m][shape] float32 impulse responses h_k, origin at index 0.
 *   flags  : PCE_FLAG_NONE or a combination of PCE_FLAG_UNFUSED,
 *            PCE_FLAG_LOWP_STORAGE (not with PCE_FLAG_UNFUSED),
 *            PCE_FLAG_PRODUCT_CONVOLUTION and PCE_FLAG_SECTIONED (see each
 *            flag for the combinations); other bits return PCE_ERR_INVALID.
 *   stream : cudaStream_t used for the set-up work.
 *
 * The plan finds the support box of every w_k (the smallest periodic
 * rectangle holding its nonzeros: rows and columns outside it are skipped by
 * the forward row pass and the adjoint row pass, Lemma 3.2), keeps a copy of
 * w_k restricted to that box, computes hhat_k = R2C(h_k) with the library's
 * own FFT and FP32 twiddles generated in FP64, and allocates its scratch.
 * w and h are only read during the call and may be freed afterwards.  The
 * call synchronises `stream` before it returns.
 */
pce_status pce_plan_create(pce_plan_t* out, int ndims, const int64_t* shape, int m,
                           const float* w, const float* h, uint32_t flags, void* stream);

/*
 * pce_plan_create_from_spectra -- as pce_plan_create, with the impulse
 * responses given by their half spectra.
 *
 *   hhat : device, [m][Ny][Nx/2+1] (2D) or [m][N/2+1] (1D) complex64,
 *          interleaved float pairs.
 *
 * The operator is y = C2R( sum_k hhat_k . R2C(w_k . u) ) with the standard
 * C2R: the imaginary parts of the DC and Nyquist bins of the last axis are
 * discarded (in 2D: the DC and Nyquist columns are replaced by their
 * Hermitian parts along y).  With hhat_k = R2C(h_k) this is the same operator
 * as pce_plan_create.
 */
pce_status pce_plan_create_from_spectra(pce_plan_t* out, int ndims, const int64_t* shape, int m,
                                        const float* w, const float* hhat, uint32_t flags,
                                        void* stream);

/*
 * pce_plan_create_separable -- a 2D plan whose windows are tensor products,
 * w_k[r][c] = wy[k][r] * wx[k][c] (the tensor-product B-spline windows of the
 * paper's 2D examples, e.g. bilinear hats on a node grid).
 *
 *   shape : [2] = (Ny, Nx).
 *   wy    : device, [m][Ny] float32 row factors.
 *   wx    : device, [m][Nx] float32 column factors.
 *   h, flags, stream : as for pce_plan_create (hhat for the _from_spectra form).
 *
 * The operator is exactly that of pce_plan_create with w_k = wy_k (x) wx_k
 * (the plan also builds everything the general path needs).  For Ny = 1024
 * or 512 with FP32 storage and the fused kernels, applies take a faster path: terms
 * whose column factors are bitwise equal share one set of row transforms,
 * since R2C_x(wy_k(y) wx_j(x) u) = wy_k(y) R2C_x(wx_j u): the forward row
 * pass transforms one row set per distinct column factor instead of one per
 * term, the column pass applies wy_k on load, and the adjoint column pass
 * sums wy_k . Q_k per column factor before the single row pass over those
 * sums.  Results agree with the general path up to rounding order.
 * pce_plan_slots returns the number of distinct column factors when the fast
 * path is on, 0 otherwise.  The inputs may be freed after the call returns.
 */
pce_status pce_plan_create_separable(pce_plan_t* out, const int64_t* shape, int m, const float* wy,
                                     const float* wx, const float* h, uint32_t flags, void* stream);
pce_status pce_plan_create_separable_from_spectra(pce_plan_t* out, const int64_t* shape, int m,
                                                  const float* wy, const float* wx, const float* hhat,
                                                  uint32_t flags, void* stream);
int pce_plan_slots(pce_plan_t plan);

/*
 * pce_apply -- y = H_m u for `batch` right-hand sides (Eq. 1.4).
 *
 *   u : device, [batch][shape] float32 input.
 *   y : device, [batch][shape] float32 output; must not overlap u
 *       (PCE_ERR_INVALID if y == u).
 *   batch >= 0 (0 is a no-op).
 */
pce_status pce_apply(pce_plan_t plan, const float* u, float* y, int64_t batch, void* stream);

/*
 * pce_apply_adjoint -- x = H_m^* v for `batch` right-hand sides.
 *
 *   v : device, [batch][shape] float32 input.
 *   x : device, [batch][shape] float32 output; must not overlap v.
 */
pce_status pce_apply_adjoint(pce_plan_t plan, const float* v, float* x, int64_t batch,
                             void* stream);

/*
 * pce_plan_info -- read back plan facts (host pointers, may be NULL):
 *   m_out, box_out[4*m] = (r0, nr, c0, nc) support box of each w_k
 *   (1D: r0 = 0, nr = 1), scratch_bytes_out = device scratch the plan holds.
 */
pce_status pce_plan_info(pce_plan_t plan, int* m_out, int* box_out, int64_t* scratch_bytes_out);

/*
 * pce_plan_hhat -- copy the plan's spectra to `hhat` (device,
 * [m][Ny][Nx/2+1] or [m][N/2+1] complex64), stream-ordered on `stream`.
 * DC and Nyquist bins come back in the form the plan uses (see
 * pce_plan_create_from_spectra).
 */
pce_status pce_plan_hhat(pce_plan_t plan, float* hhat, void* stream);

/* pce_plan_destroy -- free the plan and all its device memory (synchronises the device). */
pce_status pce_plan_destroy(pce_plan_t plan);

/* Message of the last failing call on this thread ("" if none). */
const char* pce_last_error_string(void);

/* Number of kernel launches one pce_apply / pce_apply_adjoint of `batch` issues. */
int64_t pce_launch_count(pce_plan_t plan, int adjoint, int64_t batch);

/*
 * Per-kernel timing (measurement support; no counterpart in the paper).
 *
 * pce_plan_set_timing(plan, 1) makes every later apply on the plan bracket
 * each kernel it launches with a pair of CUDA events recorded on the apply's
 * stream; pce_plan_set_timing(plan, 0) stops recording and discards the
 * events.  pce_plan_timing() waits for the recorded events and returns, for
 * kernel kind `kind` (PCE_KERNEL_*), the summed device time in milliseconds
 * and the number of launches since timing was enabled.  Up to 65536 launches
 * are recorded; later launches run untimed.
 */
enum {
    PCE_KERNEL_ROWS_R2C_WINDOW = 0,  /* forward row pass: window, R2C (2D) */
    PCE_KERNEL_COLS_FWD = 1,         /* forward column FFT, spectral MAC, inverse column FFT (2D) */
    PCE_KERNEL_ROWS_C2R = 2,         /* forward row C2R (2D) */
    PCE_KERNEL_ROWS_R2C = 3,         /* adjoint row R2C of v (2D) */
    PCE_KERNEL_COLS_ADJ = 4,         /* adjoint column FFT, conj spectra, per-term inverse (2D) */
    PCE_KERNEL_ROWS_ADJ = 5,         /* adjoint row C2R, window, accumulate (2D) */
    PCE_KERNEL_FWD_1D = 6,           /* 1D forward, one CTA per right-hand side */
    PCE_KERNEL_ADJ_1D = 7,           /* 1D adjoint, one CTA per right-hand side */
    PCE_KERNEL_PLAIN = 8,            /* any kernel of the unfused pipeline (PCE_FLAG_UNFUSED) */
    PCE_KERNEL_KINDS = 9
};
pce_status pce_plan_set_timing(pce_plan_t plan, int enable);
pce_status pce_plan_timing(pce_plan_t plan, int kind, double* total_ms, int64_t* launches);

/*
 * Failure detection.  Kernels that wait for an asynchronous copy (an
 * mbarrier wait) give up after a bounded time (about a second) instead of
 * hanging, skip the work that needed the copy and record the timeout in the
 * plan's device status word.
 *
 * pce_plan_status: synchronise `stream`, return PCE_ERR_TIMEOUT if a kernel
 *   recorded a timeout since the last call (and clear it), else PCE_OK.
 * pce_plan_inject_wait_timeout (test support): with wait_cycles > 0, later
 *   applies arm their barriers without starting the copies, so each wait runs
 *   out after wait_cycles clock cycles and the results are wrong; 0 restores
 *   normal operation.  No copy is left in flight either way.
 */
pce_status pce_plan_status(pce_plan_t plan, void* stream);
pce_status pce_plan_inject_wait_timeout(pce_plan_t plan, int64_t wait_cycles);

/*
 * Gradients (autograd support).
 *
 * For a scalar loss L(y) with y = H_m u, given r = dL/dy, pce_backward
 * computes
 *   du    = dL/du = H_m^* r                                  [batch][shape]
 *   dw    = dL/dw_k = sum_b u_b . (h~_k * r_b)              [m][shape]
 *   dhhat = dL/dRe hhat_k + i dL/dIm hhat_k                  [m][Ny][Nx/2+1] (2D)
 *         = sum_b (c_f / P) R2C(r_b) . conj(R2C(w_k . u_b))  or [m][N/2+1] (1D)
 * where hhat_k are the spectra of the operator as pce_plan_create_from_spectra
 * defines it (c_f = 2 on the interior bins of the half spectrum, 1 on DC and
 * Nyquist).  The per-term spectra R2C(w_k . u_b) are recomputed, not kept by
 * the forward apply.  dw is dense: the gradient is nonzero also outside the
 * support of w_k.
 *
 *   u, r            : device, [batch][shape] float32 (forward input, dL/dy).
 *   du, dw, dhhat   : device outputs; any may be NULL to skip it.
 *   workspace       : device scratch of at least
 *                     pce_backward_workspace_bytes(plan, batch) bytes; the
 *                     call allocates nothing itself.
 *   batch >= 0 (batch = 0 writes zero gradients).
 * Stream-ordered on `stream`; uses the plan's scratch too (not concurrent
 * with applies of the same plan).
 */
int64_t pce_backward_workspace_bytes(pce_plan_t plan, int64_t batch);
pce_status pce_backward(pce_plan_t plan, const float* u, const float* r, float* du, float* dw,
                        float* dhhat, int64_t batch, void* workspace, int64_t workspace_bytes,
                        void* stream);

/*
 * pce_apply_noalloc -- y = H_m u like pce_apply, for callers that cannot
 * allocate device memory (no counterpart in the paper).
 *
 * Some callers cannot call cudaMalloc when they apply the operator: code
 * whose device memory is owned by another allocator (a framework's caching
 * pool, where a raw cudaMalloc can fail although the pool has room), code
 * that must not risk the implicit device synchronisation of cudaMalloc, or
 * code working under a fixed device-memory budget.  pce_apply itself does not
 * allocate, but it needs the plan's scratch, which is sized for a whole batch
 * chunk (about 1 GB for a 1024 x 1024, m = 16 plan).  This entry point runs
 * the same 2D forward kernels with their intermediates in a static block of
 * 64 MiB of device memory that the library reserves on every device it is
 * loaded on and keeps until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 *   plan   : a 2D plan (a 1D plan returns PCE_ERR_UNSUPPORTED: the 1D apply
 *            needs no scratch).
 *   u, y, batch, stream : as for pce_apply.
 *
 * A right-hand side needs (m * nr_max + Ny) * (Nx/2) * 8 bytes of scratch
 * (nr_max = most rows of a window's support box); a plan that needs more
 * than 64 MiB per right-hand side returns PCE_ERR_UNSUPPORTED with the
 * required size in pce_last_error_string().  Larger batches are processed in
 * chunks that fit.
 *
 * Every call looks up the device address of the static block on the
 * current device (cudaGetSymbolAddress, which allocates nothing), so a
 * device reset between calls is handled.  The first lookup on a device may
 * load the library's device code there: make the first call on a device
 * before any stream capture.  Every call on a device shares the same
 * block, which keeps the previous call's contents (nothing needs to start at
 * zero: every element a kernel reads is written earlier in the same call).
 * Calls whose work overlaps on the GPU (other streams, other threads, other
 * plans) race on the block and give wrong results: serialise them.
 * Separable and sectioned plans run here on their whole-grid structures
 * (the general kernels), with the same result up to rounding.
 */
pce_status pce_apply_noalloc(pce_plan_t plan, const float* u, float* y, int64_t batch, void* stream);

/* ------------------------------------------------------------------------
 * Batches of applies, CUDA-graph replay and the autotuner.
 *
 * The paper applies one operator at a time; serving many small or uneven
 * operators (other sizes, other m, both directions) at once is this
 * library's addition.  A task is one pce_apply or pce_apply_adjoint call.
 * ---------------------------------------------------------------------- */
typedef struct pce_task {
    pce_plan_t plan;     /* plan of the operator (not PCE_FLAG_UNFUSED)          */
    const float* in;     /* device, [batch][shape] float32                       */
    float* out;          /* device, [batch][shape] float32                       */
    int64_t batch;       /* right-hand sides, >= 0                               */
    int adjoint;         /* 0: out = H_m in;  1: out = H_m^* in                  */
    int reserved;        /* set to 0                                             */
} pce_task;

typedef struct pce_batch* pce_batch_t;

/*
 * pce_apply_batch -- run n independent tasks, stream-ordered after the work
 * already queued on `stream`; work queued on `stream` afterwards runs after
 * all of them.  Tasks on one plan share its scratch and run in order on one
 * lane (an internal stream); tasks on different plans run concurrently on up
 * to 16 lanes, plans assigned longest-first to the least loaded lane (cost =
 * the autotuned time, else the flop model).  Allocates nothing; the lane
 * streams are created at the first call on a device (make it outside any
 * stream capture).  Capturable into a CUDA graph (ThreadLocal or Relaxed
 * mode).  Errors: PCE_ERR_INVALID for a bad task (NULL plan, host or
 * overlapping in/out, plans of another device, a task writing memory another
 * task reads or writes), PCE_ERR_UNSUPPORTED for PCE_FLAG_UNFUSED plans.
 * Concurrent calls from several host threads are serialised internally.
 */
pce_status pce_apply_batch(const pce_task* tasks, int n, void* stream);

/*
 * pce_batch_create -- a reusable batch of n tasks (copied; the pointers they
 * hold are bound until pce_batch_destroy).  The tasks are spread over
 * `lanes` (1..64) streams by the same longest-first rule, task by task, and
 * every lane owns scratch for its largest task, so tasks of one plan also
 * run concurrently.  Allocates the lane scratch (pce_batch_info reports it).
 *   pce_batch_run    -- issue the batch on `stream` (fork onto the lanes,
 *                       join back), like pce_apply_batch.
 *   pce_batch_launch -- the same work as one CUDA graph launch on `stream`;
 *                       the first call captures and instantiates the graph
 *                       (on an internal stream; it must not be made while
 *                       `stream` is capturing in global mode).
 * Results are bitwise those of pce_apply / pce_apply_adjoint run with the
 * same right-hand sides per launch.  Runs of one batch must not overlap.
 */
pce_status pce_batch_create(pce_batch_t* out, const pce_task* tasks, int n, int lanes);
pce_status pce_batch_run(pce_batch_t batch, void* stream);
pce_status pce_batch_launch(pce_batch_t batch, void* stream);
/* lanes, scratch bytes, kernel launches per run, modelled makespan (ms) and,
 * if lane_of is not NULL, the lane of every task ([n] ints).  Any pointer may
 * be NULL. */
pce_status pce_batch_info(pce_batch_t batch, int* lanes, int64_t* scratch_bytes, int64_t* launches,
                          double* model_makespan_ms, int* lane_of);
pce_status pce_batch_destroy(pce_batch_t batch);

/*
 * pce_batch_autotune -- choose, for the whole batch, the column-variant and
 * row-variant policy (each: -1 = every plan's own choice, 0, 1 or 2 = that
 * variant for every task that has it, the others keeping their own; see
 * pce_plan_autotune) by timing the batch's graph launch under all sixteen
 * policies (L2 flushed, best of three) and keeping the fastest.  Variants chosen per plan in isolation can lose inside a
 * concurrent batch, which is why the batch is timed as a whole.  Runs the
 * batch (outputs are overwritten), allocates and frees temporary buffers,
 * synchronises `stream`, and drops the captured graph (the next
 * pce_batch_launch captures again).  pce_batch_tuning reads the policies
 * back; pce_batch_tuning_log lists every timed policy (col, row, ms per run)
 * and returns their number.
 */
pce_status pce_batch_autotune(pce_batch_t batch, void* stream);
pce_status pce_batch_tuning(pce_batch_t batch, int* col_policy, int* row_policy);
/* pce_batch_set_tuning -- set the policies pce_batch_autotune would choose, by
 * hand (column policy -1..4, row policy -1..2; a variant a task's plan does
 * not have falls back to that plan's kernels as under autotuning), e.g. to
 * give a second batch over the same plans the first one's choice.  Drops the
 * captured graph.  Host only. */
pce_status pce_batch_set_tuning(pce_batch_t batch, int col_policy, int row_policy);
int pce_batch_tuning_log(pce_batch_t batch, int max_entries, int* col_policy, int* row_policy,
                         double* ms_per_run);

/*
 * pce_schedule_lpt -- the lane rule, exposed for tests: tasks by decreasing
 * cost (ties by index), each to the lane with the least load so far (ties:
 * lowest lane).  Host only.  lane_of: [n] output; makespan may be NULL.
 */
pce_status pce_schedule_lpt(const double* cost, int n, int lanes, int* lane_of, double* makespan);

/*
 * pce_plan_autotune -- time the plan's applies (forward + adjoint of `batch`
 * right-hand sides of a fixed pattern, L2 flushed between repetitions, best
 * of three) for every candidate and keep the fastest:
 *   - column FFT variant for Ny = 512, 1024 and 2048: 0 = one-warp four-step
 *     (1024 points: 32 x 32; 512 points: 16 x 32 with the last radix-2 split
 *     over lane pairs; 2048 points: two such 1024-point warps per column),
 *     1 = block Stockham (radix 8); for Ny = 1024 and 512 also 2 (separable plans) = the
 *     one-warp four-step with each warp's held column and accumulator in
 *     tensor memory (more warps per SM), 3 (Ny = 1024) = variant 2 with pruned column
 *     transforms (separable plans whose row factors each lie in 512 rows
 *     starting on a multiple of 32: the forward FFT skips the zero half of
 *     its input, the adjoint computes the needed half of its output), 4 (Ny =
 *     1024) = variant 2 run slot by slot (separable plans with two or more
 *     column-factor slots: the row pass and the column pass of one slot at a
 *     time, so that one slot's intermediate and the accumulator fit in L2);
 *   - row-pass variant (2D): 0 = block Stockham rows, the adjoint with the
 *     next term's data prefetched into registers (2 CTAs per SM), 1 = block
 *     Stockham rows without prefetch (3 CTAs per SM), 2 = variant 1 with the
 *     forward's windowed R2C run by row pairs (each pair's rows loaded once
 *     for all the terms or slots whose box holds them) and, for rows of 1024
 *     or 512 points, the plain row transforms (the adjoint's input R2C and the
 *     forward's output C2R) by one warp per row pair;
 *   - right-hand sides per launch: powers of two up to the plan's scratch
 *     chunk (2D plans and 1D plans above 8192 points).
 * 1D plans up to 8192 points have nothing to choose and are only timed.  The
 * choice changes no value an apply computes beyond rounding order (the
 * column variants' FFTs round differently).  cache_path (may be NULL): a
 * JSON-lines file; a line whose key (device, shape, m, flags, support boxes,
 * batch) matches is used without timing, otherwise the measured choice is
 * appended.  Allocates and frees temporary buffers and synchronises the
 * stream.  pce_plan_tuning reads the choice back (ms_per_apply: measured
 * milliseconds per right-hand side per direction; 0 if never tuned).
 */
pce_status pce_plan_autotune(pce_plan_t plan, int64_t batch, const char* cache_path, void* stream);
pce_status pce_plan_tuning(pce_plan_t plan, int* chunk, int* col_variant, int* row_variant,
                           double* ms_per_apply);
/* pce_plan_set_tuning -- set the choices pce_plan_autotune would make, by
 * hand: chunk = right-hand sides per launch (0 = the plan's scratch chunk;
 * larger values are clamped to it), col_variant and row_variant as above.
 * A column variant the plan has no kernels for is PCE_ERR_UNSUPPORTED
 * (1 needs a 2D plan with 512, 1024 or 2048 rows, 2 a separable plan with 1024
 * or 512 rows, 3 a separable plan with 1024 rows whose row factors allow pruning, 4 such a plan with
 * two or more slots); row variants 1 and 2 need a 2D plan.  Changes no value an
 * apply computes beyond rounding order.  Host only, no synchronisation. */
pce_status pce_plan_set_tuning(pce_plan_t plan, int chunk, int col_variant, int row_variant);
/* Every candidate the last timed pce_plan_autotune measured: writes up to
 * max_entries (chunk, column variant, row variant, ms per apply) entries into
 * the arrays (any may be NULL) and returns how many there were (0 after a
 * cache hit or for NULL). */
int pce_plan_tuning_log(pce_plan_t plan, int max_entries, int* chunk, int* col_variant,
                        int* row_variant, double* ms_per_apply);

/* ------------------------------------------------------------------------
 * Construction of (h_k, w_k) (plan-time, not part of the apply).
 * ---------------------------------------------------------------------- */

/*
 * pce_construct_projection_1d -- the L2 projection of a sampled time-varying
 * impulse response onto m periodic hats (Corollary 4.3; hats of Definition
 * 2.2 with alpha = 1 at the nodes k/m).
 *
 *   T     : device, [n][n] float32, T[d][j] = T(x_d, y_j): the impulse
 *           response at shift d (origin at index 0, periodic) for the input
 *           position j; the kernel is K(x_i, y_j) = T[(i - j) mod n][j].
 *   n     : samples per axis, in [16, 262144]; m in [3, min(n, 512)].
 *   h_out : device, [m][n] float32: h_k[d], the projection coefficients of
 *           the rows of T (computed with FP64 sums and an FP64 Gram inverse).
 *   w_out : device, [m][n] float32: w_k[j] = B_{1,m}(j/n - k/m), periodic.
 *
 * T(x_d, y_j) ~ sum_k h_k[d] w_k[j] with the residual of every row orthogonal
 * to the hats, so that pce_plan_create(1, {n}, m, w_out, h_out, ...) applies
 * the projected operator.  Allocates and frees temporary device memory and
 * synchronises `stream`.  PCE_ERR_INVALID for bad sizes or host pointers.
 */
pce_status pce_construct_projection_1d(const float* T, int n, int m, float* h_out, float* w_out,
                                       void* stream);

/*
 * pce_construct_projection_bspline_1d -- the same L2 projection onto the
 * periodic cardinal B-splines of order alpha (Definition 2.2: B_{0,m} the
 * indicator of [-1/(2m), 1/(2m)], B_{alpha,m} = m B_{0,m} * B_{alpha-1,m}) at the
 * nodes k/m (Corollary 4.3: for T of class T^s the error falls like m^-s
 * when alpha >= s; smooth T give m^-(alpha+1)).
 *
 *   alpha : 1 (hats, the same result as pce_construct_projection_1d), 2 or 3.
 *   m     : in [alpha + 2, min(n, 512)].
 *   w_out : device, [m][n] float32: w_k[j] = B_{alpha,m}(j/n - k/m), periodic;
 *           support (alpha + 1) n / m samples.
 *   T, n, h_out, stream: as for pce_construct_projection_1d.
 *
 * PCE_ERR_INVALID for bad sizes, orders or host pointers.
 */
pce_status pce_construct_projection_bspline_1d(const float* T, int n, int m, int alpha, float* h_out,
                                               float* w_out, void* stream);

/*
 * pce_construct_projection_2d -- the L2 projection of a sampled 2D
 * time-varying impulse response onto the tensor-product hats of a gy x gx
 * node grid (Corollary 4.3 with the 2D windows of the workloads:
 * B_k(y) = B_{1,gy}(y1 - i/gy) B_{1,gx}(y2 - l/gx), k = i gx + l, Definition
 * 2.2 per axis).
 *
 *   T      : device, [ny][nx][sy][sx] float32: T[j][a][b] is the impulse
 *            response at input position j = (r, c) at the shift
 *            d = (a - sy/2, b - sx/2) (integer halves), i.e. the kernel is
 *            K(x_i, y_j) = T[j][(i - j) + (sy/2, sx/2)] inside the window and
 *            0 outside it (periodic indices).
 *   ny, nx : grid, each in [4, 4096]; sy, sx: the shift window, in
 *            [1, ny] x [1, nx]; gy, gx: node grid, each in [2, min(n, 64)].
 *   h_out  : device, [gy gx][ny][nx] float32: h_k on the shift grid (origin at
 *            index 0, periodic), the projection coefficients, zero outside
 *            the window (FP64 sums and an FP64 Gram inverse).
 *   wy_out : device, [gy gx][ny] float32: the row factor of window k.
 *   wx_out : device, [gy gx][nx] float32: its column factor.
 *
 * The windows are w_k = wy_k (x) wx_k, so pce_plan_create_separable({ny, nx},
 * gy gx, wy_out, wx_out, h_out, ...) applies the projected operator; the
 * Gram matrix of product windows is the Kronecker product of the two 1D
 * Gram matrices, so its inverse costs two small inversions.  Allocates and
 * frees temporary device memory and synchronises `stream`.
 * PCE_ERR_INVALID for bad sizes or host pointers.
 */
pce_status pce_construct_projection_2d(const float* T, int ny, int nx, int sy, int sx, int gy, int gx,
                                       float* h_out, float* wy_out, float* wx_out, void* stream);

/*
 * pce_construct_svd_1d -- the truncated singular value decomposition of a
 * sampled time-varying impulse response (Section 5.1): T(x, y) ~ sum_k
 * sigma_k f_k(x) e_k(y) with h_k = sigma_k f_k and w_k = e_k, the best rank-m
 * approximation of T (and of the operator, in the Hilbert-Schmidt norm).
 *
 *   T          : device, [n][n] float32, T[d][j] as for
 *                pce_construct_projection_1d; n in [16, 8192].
 *   m          : terms, in [1, min(n, 256)].
 *   oversample : extra directions of the randomised range finder (Halko,
 *                Martinsson and Tropp, 2011), in [0, 256]; the subspace has
 *                l = min(n, m + oversample) columns.  10 is typical.
 *   power_iters: power iterations of the range finder, in [0, 16]; each
 *                sharpens the subspace by the ratio sigma_{l+1} / sigma_k
 *                squared.  2 is typical.
 *   seed       : seed of the Gaussian test matrix (SplitMix64 counters,
 *                Box-Muller).
 *   h_out      : device, [m][n] float32: h_k = sigma_k f_k.
 *   w_out      : device, [m][n] float32: w_k = e_k, orthonormal, signed so
 *                that sum_j w_k[j] >= 0.
 *   sigma_out  : device, [m] float32, or NULL: sigma_1 >= ... >= sigma_m.
 *
 * Products with T run on the device with FP64 sums; the factorisations of
 * the n x l iterates (Householder QRs) and the one-sided Jacobi SVD of the
 * l x l triangular factor run on the host in FP64.  Terms beyond the numerical
 * rank of T (sigma_k <= 1e-12 sigma_1) are returned as zeros.  Cost: 2 q + 2
 * products of T with n x l matrices, n^2 l (2 q + 2) FP64 multiply-adds on the
 * device (GB300's FP64 rate is low: seconds for n = 4096), plus host QRs of
 * O(n l^2) each.  Allocates and frees temporary memory and synchronises
 * `stream`.  PCE_ERR_INVALID for bad sizes or host pointers.
 */
pce_status pce_construct_svd_1d(const float* T, int n, int m, int oversample, int power_iters,
                                unsigned long long seed, float* h_out, float* w_out, float* sigma_out,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCE_H_ */
