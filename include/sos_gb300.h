/*
 * sos_gb300.h -- C ABI of the GB300 engine for the over-parameterised
 * sum-of-squares objective of Keren, Osadchy and Poranne (arXiv 2410.19844).
 *
 * Problem (Sec. 1.1, Eq. 1 and Eq. 2).  A polynomial p of degree <= 2d in n
 * variables is a sum of squares iff p = m_d B m_d^T for a PSD matrix B, where
 * m_d lists the monomials of degree <= d.  Writing B = A A^T with A of size
 * N x r (N = C(n+d, d) monomials, r columns = r squares q_k), the engine
 * minimises
 *         loss(A) = 1/2 || c(A) - p ||^2 ,   c(A) = coefficients of sum_k q_k^2,
 * over the M = C(n+2d, 2d) coefficients of degree <= 2d, with first-order
 * steps (Adam, the paper's optimiser in Sec. 3, or plain gradient descent).
 * The factor 1/2 is this library's convention; the paper's error (Eq. 2) is
 * 2 * loss.  The gradient is grad = 2 H(c - p) A with H[a][b] = (c - p)[a+b].
 *
 * Monomial order (Sec. 1.1, the printed example (x1^2, x1x2, x2^2, x1, x2, 1)):
 * higher total degree first, then lexicographically larger exponent tuple
 * first (x1 compared first).  Rows of A, and entries of c and p, use it.
 *
 * Conventions for every entry point:
 *  - Every function returns a sos_status; no C++ exception crosses the ABI.
 *    On failure sos_last_error() returns a message (thread-local, valid until
 *    the next call on the same thread).
 *  - "dev" pointers are CUDA device pointers owned by the caller; "host"
 *    pointers are host memory owned by the caller.  The library owns only the
 *    plan (host tables and their device copies).
 *  - Matrices are dense and row-major.  A has N rows (monomials of degree
 *    <= d, in the order above) and r columns (squares).  p and c have M
 *    entries.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    entry points are asynchronous on that stream unless stated otherwise.
 *  - The first device call on a plan uploads its tables to the current
 *    device synchronously; make it before capturing a stream into a graph.
 *  - Element types follow `prec`: SOS_BF16 and SOS_FP32 take float A, p,
 *    grad; SOS_FP64 takes double.  SOS_BF16 rounds A to bfloat16 for the two
 *    contractions (tensor cores, FP32 accumulation); SOS_FP32 runs them on
 *    CUDA cores in FP32 (no TF32); SOS_FP64 in FP64.  Losses are double.
 */
#ifndef SOS_GB300_H
#define SOS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sos_plan_s* sos_plan_t;

typedef enum {
    SOS_OK = 0,
    SOS_E_INVALID = -1,      /* bad argument, size or pointer */
    SOS_E_CUDA = -2,         /* a CUDA runtime or driver call failed */
    SOS_E_NOMEM = -3,        /* an allocation failed or a table is too large */
    SOS_E_TIMEOUT = -4,      /* a bounded device wait gave up; the kernel returned */
    SOS_E_NONFINITE = -5,    /* a NaN or Inf appeared in c, p or the residual */
    SOS_E_UNSUPPORTED = -6   /* the request is valid but not implemented here */
} sos_status;

/* Precisions.  SOS_BF16: FP32 data, contractions on tensor cores from bf16
 * operands.  SOS_FP32, SOS_FP64: CUDA cores.  SOS_FP64_TC: FP64 data; the
 * forward c(A) is computed on tensor cores by the slicing method of
 * Ozaki et al. (error-free splitting of a matrix product): each row of A is
 * scaled by a power of two and cut into 5-bit integer slices, held exactly in
 * bf16; every product of two slices is exact in the tensor core's FP32
 * accumulator while r * 31^2 < 2^24 (r <= 17,458), and the products are
 * scaled and summed in FP64.  With s slices (sos_step_opts.slices, 8 by
 * default) each term A[a][k] A[b][k] is off by at most (s + 2) 2^(-5 s)
 * 2^(e_a + e_b), e_a the exponent of row a's largest entry: about 1e-11 of
 * the rows' scales for 8 slices.  Plans with 17,458 < r <= 74,565 use
 * slices of 4-bit digits held exactly in E4M3 bytes instead, s' =
 * ceil(5 s / 4) of them, exact while r * 15^2 < 2^24, each term off by at
 * most (s' + 2) 2^(-4 s') 2^(e_a + e_b); the environment variable
 * SOS_SLICE_FP8 (read once per process) forces E4M3 slices (1) or bf16
 * slices (0) for every plan.  The residual and loss are FP64; the adjoint
 * runs on tensor cores from bf16 H(r) and bf16 A (its error is proportional
 * to the residual, so iterations still converge to the exact fit); the update
 * subtracts an FP32 step from the FP64 iterate, and the optimiser's moments m
 * and v are FP32 arrays in this precision.  Supported by sos_coeffs,
 * sos_loss_grad (grad is double), sos_step and sos_solve; other calls reject
 * it with SOS_E_INVALID. */
typedef enum { SOS_BF16 = 0, SOS_FP32 = 1, SOS_FP64 = 2, SOS_FP64_TC = 3 } sos_prec;
typedef enum { SOS_ADAM = 0, SOS_GD = 1 } sos_opt;
typedef enum {
    SOS_VERDICT_ERROR = -1,
    SOS_VERDICT_NOT_CONVERGED = 0,   /* a gradient method never proves "not SOS" */
    SOS_VERDICT_SOS = 1              /* ||c(A) - p||_2 <= tol * ||p||_2 in FP64 */
} sos_verdict;

/* ---- plan (host only; no GPU needed) ---------------------------------- */

/* Builds the monomial tables for polynomials of degree <= two_d in n
 * variables with r squares (Sec. 1.1; the sizes follow from counting
 * monomials, Sec. 1.1).  Requires n >= 1, two_d even >= 2, r >= 1,
 * n + two_d <= 255.  The plan is host-side until its first device call.
 * Errors: SOS_E_INVALID for bad sizes, SOS_E_NOMEM when the tables do not
 * fit (M must stay below 2^31). */
int sos_plan_create(int n, int two_d, int64_t r, sos_plan_t* out);

/* The same call under its short name: sos_plan(n, 2d, r) builds the
 * monomial tables of Sec. 1.1 and the index table idx(a + b) of Eq. 1. */
int sos_plan(int n, int two_d, int64_t r, sos_plan_t* out);

/* Frees the plan, its host tables and (with its device current) its device
 * tables.  NULL is accepted. */
int sos_plan_destroy(sos_plan_t plan);

/* N = C(n+d, d) rows of A, M = C(n+2d, 2d) coefficients, r columns. */
int sos_plan_sizes(sos_plan_t plan, int64_t* N, int64_t* M, int64_t* r);

/* Writes the exponent table, one row of n bytes per monomial, in the
 * canonical order.  which = 0: the N monomials of degree <= d (host, N x n);
 * which = 1: the M monomials of degree <= 2d (host, M x n). */
int sos_plan_monomials(sos_plan_t plan, int which, uint8_t* exps);

/* Writes idx[a*N + b] = position of x^a x^b among the M coefficients, the
 * index table of the Gram identity (Eq. 1): c_g = sum_{a+b=g} (A A^T)_ab.
 * host N x N int32.  SOS_E_NOMEM if N*N exceeds 2^31 entries. */
int sos_plan_idx(sos_plan_t plan, int32_t* idx);

/* Test hook: copies rows [row0, row0 + rows) of the index table the kernels
 * read on the current device (the same idx(a, b) = position of x^a x^b as
 * sos_plan_idx, Eq. 1, but built on the device from the closed-form rank)
 * into host idx, N entries per row (host rows x N int32).  Uploads the plan
 * first when needed; synchronous.  SOS_E_INVALID for rows outside 0 .. N-1. */
int sos_plan_device_idx(sos_plan_t plan, int64_t row0, int64_t rows, int32_t* idx);

/* Bytes of device workspace that sos_coeffs / sos_loss_grad / sos_step need
 * for this plan and precision.  Callers allocate it (any 256-byte aligned
 * device buffer), initialise it once with sos_workspace_init, and pass it in. */
int sos_workspace_size(sos_plan_t plan, int prec, size_t* bytes);

/* Zeroes the workspace's status word and reduction counters (its first 256
 * bytes).  Call once after allocating a workspace, before its first use;
 * later calls keep it consistent themselves.  Asynchronous on `stream`. */
int sos_workspace_init(sos_plan_t plan, int prec, void* workspace, void* stream);

/* ---- one pass of the objective (device, asynchronous) ------------------ */

/* c(A) = coefficients of sum_k q_k^2 (Eq. 1 with B = A A^T).
 * A: dev N x r; c: dev M (float for BF16/FP32, double for FP64). */
int sos_coeffs(sos_plan_t plan, int prec, const void* A, void* c,
               void* workspace, void* stream);

/* loss = 1/2 ||c(A) - p||^2 (Eq. 2) and its gradient 2 H(c - p) A.
 * A: dev N x r; p: dev M; grad: dev N x r, or NULL for the loss only;
 * loss: dev double[2] = {loss, ||p||^2}.  A NaN or Inf in c or p is
 * reported through sos_read_status() after the stream completes. */
int sos_loss_grad(sos_plan_t plan, int prec, const void* A, const void* p,
                  void* grad, void* loss, void* workspace, void* stream);

/* The same pass for `batch` independent problems of one plan, FP32 or FP64
 * on CUDA cores (one launch per kernel for the whole batch).  A and grad:
 * dev batch x N x r; p: dev batch x M; loss: dev double[batch][2].  The
 * workspace comes from sos_workspace_size_batched. */
int sos_workspace_size_batched(sos_plan_t plan, int prec, int64_t batch, size_t* bytes);
int sos_loss_grad_batched(sos_plan_t plan, int prec, int64_t batch, const void* A,
                          const void* p, void* grad, void* loss, void* workspace,
                          void* stream);

/* The loss 1/2 ||c - p||^2 from coefficients the caller already has, for
 * callers that cannot allocate device memory when they call: a host framework
 * that only hands a library buffers it allocated itself, or a loop held to a
 * fixed memory budget, where an allocation inside the call could fail or
 * synchronise the device.  The paper has no counterpart to this entry point.
 * It runs the residual and loss reduction of sos_loss_grad with that
 * kernel's scratch (status word, ticket counters, per-block partial sums)
 * kept in a fixed 1 MiB array that the library holds on every GPU that loads
 * it, until the process exits.  It calls no allocator.
 *   prec: SOS_FP32 (float c, p, resid) or SOS_FP64 (double);
 *   c, p: dev batch x M; resid: dev batch x M (c - p) or NULL;
 *   loss: dev double[batch][2] = {1/2 ||c - p||^2, ||p||^2} per problem.
 * At most 1008 problems and 65,280 block partial sums per call (a problem
 * uses min(512, ceil(M / 1024)) blocks); larger calls return SOS_E_INVALID.
 * A NaN or Inf in c or p gives a non-finite loss (NaN or Inf); no status word
 * reports it, so check the loss.  The first call on a device looks up
 * the array's device address (synchronously); make it before any stream
 * capture.  Every call shares the array, so calls that overlap on the GPU
 * (other streams, other threads) race; each call clears what must start at
 * zero, stream-ordered, before it runs. */
int sos_loss_from_coeffs_static(int prec, int64_t batch, int64_t M, const void* c,
                                const void* p, void* resid, double* loss, void* stream);

/* Optimiser settings (Sec. 3: "basic ADAM"; the paper gives no constants,
 * these default to Kingma and Ba's: beta1 0.9, beta2 0.999, eps 1e-8). */
typedef struct {
    int optimizer;      /* sos_opt */
    double lr;
    double beta1, beta2, eps;
    int flags;          /* 0, or SOS_STEP_FP32_ADJOINT */
    int slices;         /* SOS_FP64_TC: 5-bit slices of A, 2..8 (0 = 8): each term of the
                           forward is off by at most (slices + 2) 2^(-5 slices) of its rows'
                           scales; it costs slices (slices + 1) / 2 tensor-core passes */
} sos_step_opts;

/* With SOS_FP64: contract the adjoint 2 H(r) A in FP32 from the FP64
 * residual and iterate (the forward, residual, loss and update stay FP64).
 * The gradient is then accurate to FP32 relative to its own size, which is
 * all a descent step needs, and the step costs a third of the FP64 work. */
#define SOS_STEP_FP32_ADJOINT 1

/* Optimiser state, all dev, caller-owned: A (N x r) updated in place; m and
 * v (N x r, zero before the first Adam step; unused by GD); t = number of
 * steps already taken (incremented by sos_step).  flags belongs to the
 * library: start it at 0, and set it back to 0 whenever A is changed outside
 * sos_step or the state is stepped with another workspace.  With SOS_BF16 the
 * workspace keeps a bf16 copy of A that sos_step refreshes from its fused
 * update; flags records that the copy is current and which of two buffers
 * holds it. */
typedef struct {
    void* A;
    void* m;
    void* v;
    int64_t t;
    int32_t flags;
    int32_t reserved;
} sos_state;

#define SOS_STATE_BF16_CURRENT 1
#define SOS_STATE_BF16_INDEX 2

/* One iteration: loss and gradient at A, then the update of A (and m, v).
 * loss: dev double[2] = {loss before the update, ||p||^2}, or NULL.
 * SOS_BF16 fuses the update into the adjoint kernel's epilogue (the gradient
 * is never stored); SOS_FP32 / SOS_FP64 store it in the workspace and update
 * in a separate kernel. */
int sos_step(sos_plan_t plan, int prec, sos_state* state, const void* p,
             const sos_step_opts* opts, void* loss, void* workspace, void* stream);

/* Returns the status word the last device pass left in the workspace
 * (SOS_OK, SOS_E_NONFINITE or SOS_E_TIMEOUT).  Synchronises `stream`. */
int sos_read_status(sos_plan_t plan, int prec, void* workspace, void* stream);

/* ---- the network's first layer (Sec. 2, Sec. 2.1) ------------------------- */

/* The paper's network produces the quartic form ||B Z A1 x||^2 in nf = n + 1
 * variables (Sec. 2, Eq. 4; the paper calls the first-layer matrix A, here
 * A1 to keep it apart from the coefficient matrix A):
 *   A1  dev m x nf, row-major: the linear first layer, v = A1 x;
 *   Z   the augmentation, (x_1 v, ..., x_nf v), index i*m + j;
 *   B   dev k x (nf*m), row-major: k outputs, one square each.
 * Output k is x^T M_k A1 x with M_k[i][j] = B[k][i*m + j] (B read as a stack
 * of nf x m blocks).  With P_k = M_k A1 the form is sum_k (x^T P_k x)^2, whose
 * coefficient matrix over the monomials x_i x_j (i <= j) is
 *   A_hat[(i,j)][k] = P_k[i][j] + P_k[j][i] (i < j),  P_k[i][i] (i = j).
 * The plan must have two_d = 4 and r = k; its degree-<=4 basis in n variables
 * is the form dehomogenised (x_nf = 1), so A_hat is the plan's N x k matrix
 * and c, the loss and its gradient are the core pass on A_hat.  The first
 * layer does not enlarge the set of forms; Sec. 2.1 and Sec. 3.3 use it to
 * speed up fits of targets with very unequal coefficients.
 * Element type: float for SOS_BF16 and SOS_FP32 (with SOS_BF16 only the core
 * contractions run on tensor cores), double for SOS_FP64.  m: 1 .. 65536.
 * Errors: SOS_E_INVALID for a plan with two_d != 4, a bad m or NULL pointers. */

/* Bytes of the workspace a first-layer call needs (it contains a plan
 * workspace of the same precision at offset 0, so sos_workspace_init applies). */
int sos_layer_workspace_size(sos_plan_t plan, int prec, int m, size_t* bytes);

/* A_hat (dev N x k) from B and A1. */
int sos_layer_expand(sos_plan_t plan, int prec, int m, const void* B, const void* A1,
                     void* A_hat, void* workspace, void* stream);

/* loss = 1/2 ||c(A_hat(B, A1)) - p||^2 (dev double[2] = {loss, ||p||^2}, or
 * NULL) and its gradients grad_B (dev k x nf*m) and grad_A1 (dev m x nf); a
 * NULL gradient pointer skips that gradient. */
int sos_layer_loss_grad(sos_plan_t plan, int prec, int m, const void* B, const void* A1,
                        const void* p, void* grad_B, void* grad_A1, void* loss,
                        void* workspace, void* stream);

/* Optimiser state of the network, all dev and caller-owned: B, A1 updated in
 * place; mB, vB (k x nf*m) and mA1, vA1 (m x nf) zero before the first Adam
 * step; t = steps already taken.  flags: SOS_LAYER_FIXED_A1 keeps A1 as it is
 * (the paper's A = I comparison; mA1, vA1 may then be NULL).
 * SOS_LAYER_BF16_CURRENT is set by a BF16 sos_layer_step whose layer GEMMs ran
 * on the tensor cores: its update also wrote the bf16 copy of the new B into
 * the workspace, and the next such step with the same workspace reuses it
 * instead of casting B.  The library clears it after any other step; clear it
 * yourself when B changes outside the library or the workspace changes. */
typedef struct {
    void* B;
    void* mB;
    void* vB;
    void* A1;
    void* mA1;
    void* vA1;
    int64_t t;
    int32_t flags;
    int32_t reserved;
} sos_layer_state;

#define SOS_LAYER_FIXED_A1 1
#define SOS_LAYER_BF16_CURRENT 2

/* One iteration: loss and gradients at (B, A1), then the update of B (and A1).
 * opts as for sos_step (SOS_STEP_FP32_ADJOINT applies to the core adjoint of
 * an SOS_FP64 step). */
int sos_layer_step(sos_plan_t plan, int prec, int m, sos_layer_state* state, const void* p,
                   const sos_step_opts* opts, void* loss, void* workspace, void* stream);

/* ---- certificate (synchronous) ------------------------------------------ */

/* FP64 certificate (Sec. 3: the error norm is about 1e-8 of the norm of the
 * coefficient vector for SOS inputs): evaluates c(A) in FP64 (A promoted),
 * rel = ||c(A) - p||_2 / ||p||_2, verdict = SOS if rel <= tol_rel.
 * A: dev N x r, float (a_is_double = 0) or double (1); p: dev M double.
 * rel_out, verdict_out: host.  `workspace` is unused (pass NULL): the call
 * allocates and frees its own FP64 scratch and synchronises `stream`. */
int sos_certify(sos_plan_t plan, const void* A, int a_is_double, const double* p,
                double tol_rel, double* rel_out, int* verdict_out,
                void* workspace, void* stream);

/* ---- solver (synchronous) ----------------------------------------------- */

typedef struct {
    int optimizer;            /* sos_opt, all stages */
    double lr_bf16, lr_fp32, lr_fp64;
    double beta1, beta2, eps;
    int64_t max_steps;        /* step budget of the BF16 + FP32 stages */
    int64_t check_every;      /* evaluate the loss every K steps */
    double switch_rel;        /* BF16 -> the next stage when ||c-p||/||p|| < switch_rel ... */
    int64_t stall_checks;     /* ... or after this many checks without a 1% gain;
                                 FP32 -> FP64 after as many */
    int64_t fp64_steps;       /* step budget of the FP64 stage (0: none) */
    int fp64_fp32_adjoint;    /* FP64 stage steps with SOS_STEP_FP32_ADJOINT */
    double cert_tol;          /* certificate threshold (Sec. 3: about 1e-8) */
    int start_prec;           /* SOS_BF16 (the ladder), SOS_FP32 (no BF16
                                 stage) or SOS_FP64 (FP64 steps only) */
    int tc_fp64;              /* 1 (default): after the BF16 stage, SOS_FP64_TC steps
                                 take the place of the FP32 and FP64 stages (up to
                                 fp64_steps, or until stall_checks checks without a
                                 1% gain), with slices chosen from the current
                                 residual so the forward stays about 2^-10 of it;
                                 the certificate is still the CUDA-core FP64
                                 evaluation.  Plans with r > 74,565 (r > 17,458
                                 with SOS_SLICE_FP8=0), or with the CTA-pair
                                 kernels switched off, take the CUDA-core
                                 stages.  0: always the CUDA-core stages */
} sos_solve_opts;

typedef struct {
    int verdict;              /* sos_verdict */
    int64_t steps, steps_bf16, steps_fp32, steps_fp64;
    double rel_start_fp64;    /* FP64 ||c-p||/||p|| at the start point */
    double rel_at_switch;     /* BF16-evaluated relative residual at the switch */
    double min_rel;           /* best relative residual checked in FP32 */
    double min_rel_fp64;      /* best relative residual checked in FP64 */
    double rel_resid_fp64;    /* certificate of the returned A */
} sos_result;

/* Defaults: Adam, lr 1e-2 in every stage, 20000 BF16+FP32 steps, checks
 * every 50, switch at 1e-3 or 4 stalled checks, 2000 FP64 steps with the
 * FP32 adjoint, tolerance 1e-8, start in BF16, the SOS_FP64_TC stage after
 * BF16 (tc_fp64 = 1). */
int sos_solve_opts_default(sos_solve_opts* opts);

/* Minimises 1/2 ||c(A) - p||^2 from the start point A by a precision ladder:
 * BF16 steps until the relative residual falls below switch_rel (or stalls),
 * then SOS_FP64_TC steps on an FP64 copy of the best BF16 point (tc_fp64 = 1)
 * -- or FP32 steps until they stall and FP64 steps on an FP64 copy of the
 * best FP32 point (tc_fp64 = 0) -- then the FP64 certificate of the best
 * checked point (Sec. 3: success is the minimum error over the iterations).
 * The Adam state carries over between stages.  A: dev N x r double, start
 * point in, best point out; p64: dev M double.  Allocates and frees its own
 * buffers and synchronises `stream`. */
int sos_solve(sos_plan_t plan, const double* p64, double* A, const sos_solve_opts* opts,
              sos_result* out, void* stream);

/* ---- groups: many small problems stepped together (serving) --------------- */

/* A group steps up to `capacity` independent problems, each with its own plan
 * (any n, 2d; r must equal N) and buffers, FP32 or FP64 on CUDA cores.  One
 * group step runs three kernels whose work lists cover every active problem
 * (64 x 64 tiles of every A A^T, coefficient chunks, tiles of every 2 H A with
 * the optimiser update fused), so large and small problems share the GPU.
 * No result depends on which other problems share the group: a problem's
 * iterates are bitwise the same alone or in a mix.  The optimiser (and beta1,
 * beta2, eps) is fixed per group; the step size per problem. */
typedef struct sos_group_s* sos_group_t;

/* flags: SOS_GROUP_FP32_ADJOINT (FP64 groups only) contracts the adjoint
 * 2 H(r) A in FP32 from the FP64 residual and iterate; the forward, the
 * residual, the loss and the update stay in FP64, so the certificate is
 * still an FP64 evaluation.  It takes two thirds of the FP64 work off the
 * step; the gradient it gives is accurate to FP32 relative to its own size. */
#define SOS_GROUP_FP32_ADJOINT 1

/* SOS_GROUP_FAST_FP64 (FP64 groups only) keeps FP64 arithmetic off the slow
 * FP64 pipe where it is not needed.  The forward accumulates in double-float
 * arithmetic on the FP32 pipes: products and sums are carried as two FP32
 * words, with error-free products and two-sums, about 2^-46 relative to the
 * sum of |products|.  The optimiser's update arithmetic runs in FP32, only when
 * the adjoint does too (with SOS_GROUP_FP32_ADJOINT), and is subtracted from
 * the FP64 iterate.  The residual, the loss and so the verdict stay FP64. */
#define SOS_GROUP_FAST_FP64 2

int sos_group_create(int prec, int capacity, int optimizer, double beta1, double beta2,
                     double eps, int flags, sos_group_t* out);
int sos_group_destroy(sos_group_t group);

/* Device scratch one problem of this plan needs in a group of precision prec
 * (the second buffer of its A, its Gram matrix, residual and partial sums). */
int sos_group_scratch_size(sos_plan_t plan, int prec, size_t* bytes);

/* Puts a problem into slot `slot` (0 <= slot < capacity), starting from its
 * current A: A, m, v dev N x r (zero m, v for a fresh Adam state), p dev M,
 * scratch dev sos_group_scratch_size bytes; all caller-owned and kept alive
 * until the slot is cleared.  t0 = optimiser steps already taken with this m,
 * v (0 for a fresh state), so that Adam's bias correction continues.  The
 * first call for a plan builds its device tables (allocates; do it before
 * capturing).  Takes effect at the next sos_group_sync. */
int sos_group_set(sos_group_t group, int slot, sos_plan_t plan, void* A, void* m, void* v,
                  const void* p, void* scratch, double lr, int64_t t0);
int sos_group_clear(sos_group_t group, int slot);

/* Changes the step size of an active slot (from the next sos_group_sync). */
int sos_group_set_lr(sos_group_t group, int slot, double lr);

/* Uploads the slot table and work lists after set/clear (stream-ordered;
 * waits for the group's earlier work first). */
int sos_group_sync(sos_group_t group, void* stream);

/* Runs `steps` steps of every active problem as one CUDA graph (captured on
 * first use for that step count, replayed after), ordered after the work
 * already queued on `stream` and before work queued on it later. */
int sos_group_run(sos_group_t group, int steps, void* stream);

/* Host double[2 * capacity]: {1/2 ||c - p||^2, ||p||^2} of each slot at the
 * last step (before its update); zeros for empty slots.  Synchronises. */
int sos_group_losses(sos_group_t group, double* losses, void* stream);

/* Where slot's iterates are: the update ping-pongs between A and the first
 * region of the scratch, so A_current holds the latest iterate and
 * A_previous the one before it -- the iterate whose loss the last step
 * computed and sos_group_losses reports.  steps_taken counts the steps run
 * in this group.  Any output may be NULL. */
int sos_group_state(sos_group_t group, int slot, void** A_current, void** A_previous,
                    int64_t* steps_taken);

/* Element-wise copy with conversion between FP32 and FP64 (prec codes
 * SOS_FP32 / SOS_FP64): y = x, count elements, dev, asynchronous. */
int sos_convert(const void* x, int x_prec, void* y, int y_prec, int64_t count, void* stream);

/* Diagnostic: a plain tcgen05 BF16 GEMM with FP32 output through the same
 * tile machinery as the two contractions.  D (dev m x n, row stride n) =
 * X (dev m x k bf16, row stride ldx) times Y^T (mode bit 0 clear: Y is n x k,
 * row stride ldy) or times Y (bit 0 set: Y is k x n, row stride ldy).  Mode
 * bit 1 runs it on CTA pairs (cta_group::2), as the contractions do unless
 * the environment variable SOS_CTA_PAIRS is 0.
 * Row strides must be multiples of 8 elements and the bases 16-byte
 * aligned.  status: dev int32, zero on entry; a timed-out wait sets it.
 * Synchronises `stream`. */
int sos_diag_gemm_bf16(int mode, const void* X, const void* Y, float* D,
                       int64_t m, int64_t n, int64_t k, int64_t ldx, int64_t ldy,
                       int32_t* status, void* stream);

/* Diagnostic for failure detection: one device thread waits, with the same
 * bounded mbarrier wait as the tensor-core kernels, on a barrier that nothing
 * arrives at.  After limit_ns (at most 5 s) it sets *status (dev int32, zero
 * on entry) to SOS_E_TIMEOUT and the kernel returns; the context stays usable.
 * Asynchronous on `stream`. */
int sos_diag_bounded_wait(uint64_t limit_ns, int32_t* status, void* stream);

/* ---- instrumentation ------------------------------------------------------ */

/* Number of kernels this library has launched since it was loaded. */
int64_t sos_launch_count(void);

/* on != 0: bracket every kernel launch with CUDA events on its stream
 * (device-side timing, stream-ordered; do not enable during graph capture). */
int sos_timing_enable(int on);

/* Drops the recorded events (waits for them first). */
int sos_timing_reset(void);

/* Writes one line per kernel, "name launches total_ms\n", for the launches
 * recorded since the last reset.  Waits for the recorded events. */
int sos_timing_report(char* buf, size_t cap);

const char* sos_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SOS_GB300_H */
