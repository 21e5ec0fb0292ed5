/*
 * phiks.h - C ABI of the GB300 (sm_103a) library for actions of phi-functions
 * of Kronecker sums (Caliari, Cassini, Zivcovich, "A mu-mode approach for
 * exponential integrators: actions of phi-functions of Kronecker sums",
 * arXiv 2210.07667).
 *
 * Problem (Sec. 1, eq. kronsum, eq. diffphi, eq. lincomb): for
 * K = A_d (+) ... (+) A_1 = sum_mu I_d x ... x A_mu x ... x I_1 (never formed),
 * compute either the same-vector set
 *     { phi_0(tau K) v, phi_1(tau K) v, ..., phi_p(tau K) v }
 * or the linear combination
 *     exp(tau K) v_0 + phi_1(tau K) v_1 + ... + phi_p(tau K) v_p,
 * optionally also at the time scales tau / 2^(j-1), j = 1..nscales
 * (eq. scaldiffphi, eq. scallincomb).
 *
 * Layout (Lemma 1 of Sec. 2): a vector of length N = n_1 * ... * n_d is the
 * column-major vec of an n_1 x ... x n_d tensor (mode 1 fastest).  Matrices
 * A_mu are n_mu x n_mu, column-major, real (complex for PHIKS_C128 plans:
 * interleaved real and imaginary parts, as are those plans' vectors).
 *
 * Conventions for every entry point:
 *   - pointers named "host" are CPU memory, all other buffers are device
 *     memory on the device that was current when the plan was made;
 *   - the caller owns every buffer it passes; the plan owns its device copies
 *     of A_mu (with powers 2..15 of a scaled A_mu - sigma_mu I, or 2..4 when
 *     those would pass 256 MiB), the cached small exponentials and its
 *     default workspace;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     apply calls are asynchronous on that stream except where stated;
 *   - nothing throws: each call returns a phiks_status and records a message
 *     that phiks_last_error() returns (thread-local);
 *   - everything an apply writes besides its outputs lives in its workspace
 *     or in the plan's cached small exponentials, so applies on one plan may
 *     overlap on the GPU (different streams) when each passes its own
 *     workspace and its norms (phiks_options).  The cached exponentials are
 *     ordered across streams by events: a call waits (on the device, not the
 *     host) for a cache entry another stream is still building, and a
 *     rebuild (no_cache) or an eviction waits for every earlier use on other
 *     streams.  The plan's host-side state (parameter and exponential
 *     caches) is not thread-safe, so issue the calls from one host thread;
 *   - an apply never synchronises with the host except where stated (the
 *     device norms, below); its allocations (the plan's own workspace, new
 *     cache entries, freed ones) are stream-ordered (cudaMallocAsync /
 *     cudaFreeAsync on the call's stream).
 */
#ifndef PHIKS_H
#define PHIKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PHIKS_MAX_D 8   /* largest tensor order d */
#define PHIKS_MAX_P 8   /* largest phi order p */

typedef struct phiks_plan_s* phiks_plan_t;
typedef struct phiks_batch_s* phiks_batch_t;

typedef enum {
  PHIKS_OK = 0,
  PHIKS_ERR_INVALID = 1,      /* bad argument (null pointer, size, p, nv ...) */
  PHIKS_ERR_OOM = 2,          /* device or host allocation failed */
  PHIKS_ERR_UNSUPPORTED = 3,  /* valid request this build does not implement */
  PHIKS_ERR_NO_PARAMS = 4,    /* no (s, q) meets the tolerance (Sec. 3.3) */
  PHIKS_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  PHIKS_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
} phiks_status;

/* Arithmetic of the mu-mode products.  FP64: vectors are double, products on
 * the FP64 pipe.  The split types keep vectors in float and run the products
 * on the tensor cores: TF32 (one product), TF32X3 and BF16X3 (three-term
 * compensated products, hi*hi + hi*lo + lo*hi, FP32 accumulation).
 * FP64_EMU: vectors double, products on the tensor cores as exact sums of
 * bf16 digit products (seven base-256 digits per operand, FP32 accumulation
 * that stays exact for n_mu <= 128); a Tucker operator's intermediate products
 * pass their exact sums to the next mode, which rounds them once to its fixed
 * point, and the last is rounded once to FP64; needs every n_mu a multiple of 8
 * and at most 128.  C128: complex A_mu and vectors (the
 * validation operator of Sec. 4.1), complex FP64 products on the FP64 pipe;
 * vectors are N complex numbers stored as 2 N doubles (real, imaginary).
 * Small exponentials, their squaring and the doubling-formula combination
 * stay FP64 in every type (complex plans hold each small matrix as its real
 * representation [[Re, -Im], [Im, Re]]). */
typedef enum {
  PHIKS_FP64 = 0, PHIKS_TF32 = 1, PHIKS_TF32X3 = 2, PHIKS_BF16X3 = 3, PHIKS_FP64_EMU = 4,
  PHIKS_C128 = 5
} phiks_dtype;

/* Quadrature rule for the phi integral (Sec. 3.3): Gauss-Lobatto-Legendre
 * (default; theta_1 = 0 and theta_q = 1 save one Tucker operator each) or
 * Gauss-Legendre. */
typedef enum { PHIKS_RULE_GLL = 0, PHIKS_RULE_GL = 1 } phiks_rule;

typedef struct {
  double tol;            /* delta of Sec. 3.3: ||R_q|| ||v|| <= delta (absolute,
                            2-norm).  Default 2^-53. */
  int nscales;           /* s-hat >= 1: outputs at tau, tau/2, ... tau/2^(nscales-1) */
  int rule;              /* phiks_rule */
  int qmin, qmax;        /* node-count range, default [3, 12] */
  int skip_phi0;         /* same-vector task: omit the phi_0 = exp(tau K) v blocks */
  int force_s, force_q;  /* >= 0: use this scaling / node count instead of the
                            selection of Sec. 3.3 (both or neither) */
  const double* vnorms;  /* host, nv entries ||v_l||_2 (0 for NULL vectors), or
                            NULL: the norms are computed on the device and the
                            call waits once for them to reach the host (see
                            phiks_apply_ex) */
  void* workspace;       /* device workspace of >= phiks_workspace_size bytes,
                            or NULL for the plan's own */
  size_t workspace_bytes;
  int no_cache;          /* recompute the small exponentials on every call */
  int graph;             /* nonzero: the kernels of a call (everything after the
                            norms and the (s, q) selection) are captured once
                            into a CUDA graph per (tau, p, vectors, output,
                            workspace, s, q, options, small-exponential storage)
                            and later identical calls replay it with one
                            launch.  Ignored while profiling, on the legacy
                            default stream and when `stream` is already
                            capturing. */
  int reserved[6];
} phiks_options;

/* Fill `opt` with the defaults above. */
void phiks_options_init(phiks_options* opt);

/* Build a plan for K = A_d (+) ... (+) A_1 (Sec. 1, eq. kronsum).
 *   d        tensor order, 1 <= d <= PHIKS_MAX_D
 *   n        host, d entries, n_mu >= 1
 *   A        host, d pointers to column-major n_mu x n_mu doubles (copied);
 *            PHIKS_C128: 2 n_mu^2 doubles, entry (i, j) at 2 (i + n_mu j)
 *            (real part) and 2 (i + n_mu j) + 1 (imaginary part)
 *   dtype    arithmetic of the mu-mode products (phiks_dtype)
 *   out      receives the plan; NULL on failure
 * Computes on the host the shifts sigma_mu = tr(A_mu)/n_mu (Remark of Sec. 3.1;
 * the real part for complex A_mu) and the numerical-range rectangles Xi_mu
 * (Sec. 3.3), and uploads A_mu. */
phiks_status phiks_plan(int d, const int64_t* n, const double* const* A, int dtype,
                        phiks_plan_t* out);

/* phiks_apply_ex with default options (one scale, tolerance 2^-53). */
phiks_status phiks_apply(phiks_plan_t plan, double tau, int p, const void* const* v, int nv,
                         void* out, void* stream);

/* Actions of phi-functions of tau K (Sec. 3.1 for nv == 1, Sec. 3.2 for
 * nv == p + 1).
 *   tau      time step (any nonzero real)
 *   p        highest phi order, 0 <= p <= PHIKS_MAX_P
 *   v        host array of nv device pointers to N elements each (double for
 *            PHIKS_FP64 and PHIKS_FP64_EMU, float otherwise); in the linear combination any v[l]
 *            may be NULL (a zero vector; v[0] == NULL skips the exp Tuckers)
 *   nv       1: same vector;  p + 1: linear combination
 *   out      device, written (not accumulated):
 *            same vector: nscales blocks, block j (j = 0..nscales-1) holds
 *              phi_0..phi_p (tau K / 2^j) v, each N elements, phi_0 first
 *              (phi_1..phi_p only when skip_phi0);
 *            linear combination: nscales blocks of N elements, block j =
 *              exp(c tau K) v_0 + sum_l c^l phi_l(c tau K) v_l, c = 2^-j
 *              (the c^l convention of eq. scallincomb).
 * The first call for a given (tau, s, q) builds the small exponentials
 * exp((1 - theta_i) tau A_mu / 2^s) on the device and caches them in the plan
 * (at most 8 entries; the least recently used is evicted).  Inside a stream
 * capture of the caller's the entry must exist already (PHIKS_ERR_INVALID
 * otherwise), as must a plan-owned workspace of the needed size; with
 * no_cache a captured call rebuilds the entry inside the graph, on `stream`,
 * without waiting for other streams' uses.
 * Without opt->vnorms the call waits once for the device norms of v to reach
 * the host.  When an earlier call with the same tau, p, nv, NULL pattern of v
 * and selection options selected (s, q), the call first enqueues its work with
 * that (s, q) and waits for the norms while the device runs it; if the norms
 * select another (s, q), it enqueues the work again with those (the results
 * in `out` are the latter's once the stream has run). */
phiks_status phiks_apply_ex(phiks_plan_t plan, double tau, int p, const void* const* v, int nv,
                            const phiks_options* opt, void* out, void* stream);

/* Device workspace bytes an apply with these arguments needs (for
 * phiks_options.workspace).  Host only. */
phiks_status phiks_workspace_size(phiks_plan_t plan, int p, int nv, int nscales, size_t* bytes);

/* The (s, q) the selection of Sec. 3.3 picks, and T# of eq. (Tpsv) / eq. (Tlcp),
 * for the given norms (host, nv entries).  Host only, no GPU work. */
phiks_status phiks_select_params(phiks_plan_t plan, double tau, int p, int nv,
                                 const double* vnorms, const phiks_options* opt,
                                 int* s, int* q, int* tcount);

/* Same selection without a plan and without any GPU work: the operators are
 * passed as in phiks_plan (host, column-major, not retained).  Useful to
 * inspect the cost T# of a problem before planning it. */
phiks_status phiks_choose_params(int d, const int64_t* n, const double* const* A, double tau,
                                 int p, int nv, const double* vnorms, const phiks_options* opt,
                                 int* s, int* q, int* tcount);

/* (s, q, T#, Tucker operators launched) of the last successful apply. */
phiks_status phiks_last_params(phiks_plan_t plan, int* s, int* q, int* tcount, int* tuckers);

/* Tucker operator W = V x_1 L_1 x_2 ... x_d L_d (Sec. 2) in the plan's dtype.
 *   V, W     device, N elements each (may not alias)
 *   L        host array of d device pointers to column-major n_mu x n_mu
 *            doubles (converted on the fly for the split dtypes); PHIKS_C128
 *            plans: the 2 n_mu x 2 n_mu real representation
 *            [[Re L, -Im L], [Im L, Re L]] of the complex L_mu */
phiks_status phiks_tucker(phiks_plan_t plan, const void* V, void* W, const double* const* L,
                          void* stream);

/* Batched FP64 matrix exponential E_b = exp(X_b) (the small exponentials of
 * Sec. 3.1 / Sec. 4 intro), by truncated Taylor series with scaling and
 * squaring.  X and E: device, `batch` column-major n x n matrices stored
 * back to back; X is not modified; X and E may not alias. */
phiks_status phiks_expm(int batch, int n, const double* X, double* E, void* stream);

/* Kernel timing for measurement tools.  While enabled, every mu-mode product
 * the plan launches is bracketed by two CUDA events on its stream: the FP64
 * mode-product kernel (the fused small-slab kernel: one bracket for all d
 * modes), or the tensor-core GEMM pass of FP64_EMU and of the split dtypes
 * (their operand split excluded).  phiks_profile_read synchronises the plan's
 * device, returns the summed milliseconds of those brackets, their count and
 * their algorithmic flops (2 N n_mu per mode), and resets the sums. */
phiks_status phiks_profile_enable(phiks_plan_t plan, int enable);
phiks_status phiks_profile_read(phiks_plan_t plan, double* ms, int64_t* launches, double* flops);

/* Synchronises `stream` and reports whether any tensor-core kernel of the plan
 * gave up a bounded device-side wait (then PHIKS_ERR_TIMEOUT, and the results
 * of the calls since the last check are not valid).  The status is cleared by
 * the read.  Every wait inside those kernels is limited to about a second. */
phiks_status phiks_device_status(phiks_plan_t plan, void* stream);

/* Number of kernels this library has launched in this process (all plans). */
uint64_t phiks_kernel_launches(void);

/* Tucker operator W = V x_1 L_1 x_2 ... x_d L_d in FP64 that allocates no
 * memory, for callers that cannot call cudaMalloc: applications that give all
 * device memory to their own pool up front, or latency-bound loops where
 * cudaMalloc / cudaFree (driver locks, device-wide synchronisation) are not
 * acceptable.  The paper has no counterpart; it is an addition of this
 * library.
 *   d        1 <= d <= PHIKS_MAX_D
 *   n        host, d sizes; N = n_1 ... n_d must not exceed 1,048,576
 *            (larger N returns PHIKS_ERR_INVALID)
 *   V, W     device, N doubles each, column-major tensors; the two ranges
 *            may not overlap (PHIKS_ERR_INVALID, checked before any device call)
 *   L        host array of d device pointers to column-major n_mu x n_mu doubles
 * No plan is needed.  The intermediate tensors live in a fixed 16 MiB
 * __device__ array inside the library (two halves of 1,048,576 doubles) that
 * every GPU loading the library keeps until the process exits.  All calls
 * share that array, so calls whose kernels overlap on the GPU (different
 * streams, or other host threads) race and give wrong results; serialise them
 * on one stream.  Every intermediate is fully overwritten, so nothing is
 * cleared between calls.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture begins.  Asynchronous on `stream`. */
phiks_status phiks_tucker_noalloc(int d, const int64_t* n, const double* V, double* W,
                                  const double* const* L, void* stream);

/* Batches of independent applies (the batched form: many instances of
 * different sizes, each with its own plan).  A batch object owns `nstreams`
 * worker streams on the current device. */
phiks_status phiks_batch_create(int nstreams, phiks_batch_t* out);
void phiks_batch_destroy(phiks_batch_t batch);

/* Apply every instance k (plans[k], taus[k], ps[k], nvs[k] vectors starting at
 * v[nvs[0] + ... + nvs[k-1]], options opts[k] or defaults when opts is NULL,
 * output outs[k]) exactly as phiks_apply_ex would.  The instances are spread
 * over the batch's worker streams, largest first, after waiting for `stream`;
 * `stream` waits for all of them before later work.  Plans must be distinct
 * (each owns the workspace its instance uses). */
phiks_status phiks_batch_apply(phiks_batch_t batch, int count, const phiks_plan_t* plans,
                               const double* taus, const int* ps, const void* const* v,
                               const int* nvs, const phiks_options* opts, void* const* outs,
                               void* stream);

/* Record the same work as phiks_batch_apply into one CUDA graph (stream
 * capture of `stream`, which must not be the legacy default stream) and
 * instantiate it; launch it with phiks_graph_launch.  Every instance must pass
 * its norms in opts[k].vnorms, and every plan must have run this apply once
 * (so that no allocation happens inside the capture).  The graph reads and
 * writes the same buffers on every launch. */
phiks_status phiks_batch_capture(phiks_batch_t batch, int count, const phiks_plan_t* plans,
                                 const double* taus, const int* ps, const void* const* v,
                                 const int* nvs, const phiks_options* opts, void* const* outs,
                                 void* stream, void** graph_exec);
phiks_status phiks_graph_launch(void* graph_exec, void* stream);
void phiks_graph_destroy(void* graph_exec);

/* Served form: a trace of requests arriving over time (continuous batching).
 * A request is one or two applies run in order (e.g. the two species of a
 * Brusselator stage), each described as for phiks_apply_ex with its norms. */
#define PHIKS_SERVE_MAX_APPLY 2
typedef struct {
  phiks_plan_t plan;
  double tau;
  int p, nv;              /* as in phiks_apply_ex */
  const void* const* v;   /* host array of nv device pointers */
  void* out;              /* device output */
  int nscales, skip_phi0;
  double tol;             /* 0: default 2^-53 */
  const double* vnorms;   /* host, nv norms (required: serving never synchronises) */
} phiks_apply_args;

typedef struct {
  int napply;
  phiks_apply_args apply[PHIKS_SERVE_MAX_APPLY];
} phiks_request;

typedef struct {
  int slots;              /* requests on the device at once (one stream each) */
  size_t hbm_budget;      /* workspace bytes in flight at most; 0 = no limit */
  int poll_us;            /* dispatcher pause when idle (0 = yield) */
  int graphs;             /* nonzero: every slot owns a workspace and staging
                             buffers (allocated once, sized for the largest
                             request); a request's inputs are copied in, its
                             applies replay CUDA graphs captured once per
                             (plan, tau, p, slot), its outputs are copied out.
                             0: a workspace per request from the pool and
                             direct kernel launches */
} phiks_serve_config;

/* Run the trace in real time on the current device: request k becomes
 * eligible arrival_s[k] seconds after the call starts (ascending), waits in a
 * FIFO queue, and is dispatched to a free slot when its workspace fits in the
 * budget; requests on different slots overlap on the GPU.  Workspaces come
 * from a memory pool owned by the call.  Outputs: latency_ms[k] from arrival
 * to completion of its kernels, queue_ms[k] (optional) from arrival to
 * dispatch, *makespan_s (optional) from start to the last completion.  A
 * request whose (tau, s, q) has no cached exponentials yet builds them on its
 * slot (requests of the same entry on other slots wait for it on the
 * device); warming the plans first keeps the parameter search and those
 * builds out of the latencies.  Returns after every request has finished. */
phiks_status phiks_serve_trace(const phiks_serve_config* cfg, int count, const phiks_request* reqs,
                               const double* arrival_s, double* latency_ms, double* queue_ms,
                               double* makespan_s);

/* Exponential integrators driving phiks: the linear-combination form of the
 * exponential Runge--Kutta methods of Sec. 2 (eq. RK) with the tableaux the
 * paper uses, every stage assembled from phiks calls whose scale outputs
 * (eq. comb, eq. scallincomb) give stages at halved times:
 *   PHIKS_EXP_EULER  eq. (expEullc), 1 call per step
 *   PHIKS_ETD2RK     eq. (ETD2RKlc), 2 calls
 *   PHIKS_EXPRK3     eq. (expRK3s3), c_2 = 1/4, c_3 = 1/2, gamma = -4/5, 3 calls
 *   PHIKS_EXPRK4S5   eq. (expRK4s5) assembled as in eq. (expRK4s5_smart), 5 calls
 *   PHIKS_EXPRK4S6   eq. (expRK4s6), c_2 = c_3 = 1/3, c_4 = 2/3, c_5 = 1/2,
 *                    c_6 = 1 (stages 3-4 and 5-6 from one call each), 4 calls
 * with the nonlinear term g evaluated on the device. */
typedef enum {
  PHIKS_EXP_EULER = 0, PHIKS_ETD2RK = 1, PHIKS_EXPRK3 = 2, PHIKS_EXPRK4S5 = 3, PHIKS_EXPRK4S6 = 4
} phiks_scheme;
typedef enum {
  PHIKS_NL_ADR_EXACT = 0,   /* Sec. 4.2: g = 1/(1+u^2) + Psi(t,x), exact solution e^t u_0 on the
                               Dirichlet grid x_i = i/(n+1) of [0,1]^3 (one block, d = 3) */
  PHIKS_NL_ALLEN_CAHN = 1,  /* Sec. 4.3: g = -u^3 / eps^2 (one block) */
  PHIKS_NL_BRUSSELATOR = 2  /* Sec. 4.4: w = [u; v] over two blocks of equal size,
                               g = [a + u^2 v; b u - u^2 v] */
} phiks_nonlinearity;
typedef struct {
  int kind;                 /* phiks_nonlinearity */
  double eps, alpha;        /* ADR: diffusion and advection coefficients; AC: eps */
  double a, b;              /* Brusselator: the reaction constants */
} phiks_nonlinear;

/* Grid of a plan: *d and n[0 .. d-1] (host; n has room for PHIKS_MAX_D). */
phiks_status phiks_plan_shape(phiks_plan_t plan, int* d, int64_t* n);

/* Advance w (device, FP64) from t0 to t0 + T in `steps` equal steps of
 * `scheme` for w' = K w + g(t, w) with K = diag(K_1, ..., K_nblocks)
 * block diagonal (eq. ODE2): block b is plans[b]'s Kronecker sum, acting on
 * the N_b entries of w after those of blocks 0..b-1 (column-major each).
 * plans: FP64 or FP64_EMU (real).  opt (may be NULL): tol and graph apply to every
 * phiks call; nscales, skip_phi0, vnorms and workspace are set internally.
 * Device scratch of about 24 N doubles comes from the stream-ordered
 * allocator.  Each phiks call synchronises `stream` once (the norms). */
phiks_status phiks_integrate_blocks(int nblocks, const phiks_plan_t* plans, int scheme,
                                    const phiks_nonlinear* g, double t0, double T, int steps,
                                    double* w, const phiks_options* opt, void* stream);

/* One block: phiks_integrate_blocks(1, &plan, ...); n and d must match the
 * plan's grid. */
phiks_status phiks_integrate(phiks_plan_t plan, const int64_t* n, int d, int scheme,
                             const phiks_nonlinear* g, double t0, double T, int steps, double* u,
                             void* stream);

/* Tuning of a plan's kernels: the tile shapes and mode orders the
 * autotuner chooses among (0 = the library's size-based default for each
 * knob).  Results of every setting agree to rounding: the modes of a Tucker
 * operator commute, and the tiles only regroup the same sums.
 *   fused         real FP64 plans: -1 by size (N <= 8192), 0 mode-by-mode
 *                 passes, 1 the fused small-slab kernel (all d modes of a
 *                 Tucker operator, and the batch's input combinations, in one
 *                 launch with the intermediates in shared memory; only when
 *                 16 N / n_d bytes and the matrices fit there)
 *   fused_rows    fused kernel: rows of the last mode per CTA (1, 2, 4, 8;
 *                 0 by batch size)
 *   fp64_tile     FP64 / C128 mode products: 1 16 x 16, 2 32 x 64 output tiles
 *   mode_order    FP64 / C128 mode-by-mode passes: a permutation of 0..d-1
 *                 (entries past d are ignored; phiks_get_tuning sets them -1)
 *   emu_cols      FP64_EMU GEMM pass: rows of L per tile, 16 or 32
 *   split_ntiles  split dtypes: GEMM column tiles per pass as a multiple of
 *                 ceil(n_pad / 256): 1, 2 or 4 (0: by size, narrower tiles
 *                 when a pass has fewer row tiles than SMs) */
typedef struct {
  int fused;
  int fused_rows;
  int fp64_tile;
  int mode_order[PHIKS_MAX_D];
  int emu_cols;
  int split_ntiles;
  int reserved[8];
} phiks_tuning;

/* The plan's current tuning (host only). */
phiks_status phiks_get_tuning(phiks_plan_t plan, phiks_tuning* tuning);
/* Set it (host only; checked, PHIKS_ERR_INVALID / PHIKS_ERR_UNSUPPORTED for a
 * knob the plan cannot take).  Drops the plan's captured call graphs. */
phiks_status phiks_set_tuning(phiks_plan_t plan, const phiks_tuning* tuning);

/* Autotuner: times every candidate tuning of the plan's dtype (tile shapes,
 * mode orders, fused or mode-by-mode) on `reps` applies of this call shape
 * (tau, p, nv and opt's nscales, skip_phi0, tolerance and graph; seeded
 * synthetic inputs in [-1, 1]) on `stream`, sets the fastest and returns it
 * with its milliseconds per apply.  Synchronises `stream` and allocates its
 * inputs and output (not for use inside a capture).  When the environment
 * variable PHIKS_TUNE_CACHE names a file, a line for the same (dtype, n_mu,
 * p, nv, nscales) found there is used instead of timing (its milliseconds
 * returned as recorded), and a new result is appended as one line
 * "<key> | <knobs> ms=<time>". */
phiks_status phiks_autotune(phiks_plan_t plan, double tau, int p, int nv, const phiks_options* opt,
                            int reps, void* stream, phiks_tuning* best, double* best_ms);

/* Fault injection for tests of the out-of-memory paths (not for production
 * use).  phiks_debug_fail_alloc(k): the library's device allocations (plans,
 * workspaces, cached exponentials, scratch; in every thread) let k more
 * succeed, then the next one fails as if the device were out of memory, and
 * later ones succeed again; k < 0 cancels a pending failure.  The failing
 * call returns PHIKS_ERR_OOM and releases what it had allocated.
 * phiks_debug_live_allocations(): device allocations the library holds now
 * (all plans together), to check that failed calls leak nothing. */
void phiks_debug_fail_alloc(int after);
int64_t phiks_debug_live_allocations(void);

/* A check of the bounded-wait failure path of the tensor-core kernels (not
 * for production use): launches on `stream` one CTA that allocates TMEM,
 * waits on an mbarrier nothing arrives at until limit_ms (0 < limit_ms <=
 * 2000) has passed, records the failure in the plan's device status word as
 * the plan's kernels do, frees the TMEM and returns.  Afterwards
 * phiks_device_status reports PHIKS_ERR_TIMEOUT (and clears it), the
 * plan's kernels queued before that read skip their work, and later calls
 * run normally.  Tensor-core plans only (PHIKS_ERR_UNSUPPORTED otherwise). */
phiks_status phiks_debug_wait_timeout(phiks_plan_t plan, double limit_ms, void* stream);

/* Release the plan and its device memory (synchronises its device). */
void phiks_destroy(phiks_plan_t plan);

/* Message for the last failing call on this thread ("" if none). */
const char* phiks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PHIKS_H */
