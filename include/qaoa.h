/*
 * qaoa.h -- C ABI of libqaoa: batched state-vector simulation of depth-p QAOA on sub-QUBOs and
 * the DQAOA decompose / merge steps around it, for NVIDIA GB300 (sm_103a).
 *
 * Method (arXiv 2506.10531, "GPU-Accelerated Distributed QAOA on Large-scale HPC Ecosystems"):
 *   - Section IV, Eq. 1-2: a QUBO min_x x^T Q x is mapped to the diagonal problem Hamiltonian
 *     H|z> = E(z)|z>, E(z) = z^T Q z, and the ansatz is
 *       |psi(gamma, beta)> = prod_{l=1..p} e^{-i beta_l B} e^{-i gamma_l H} |+>,
 *     layer 1 acting first, with the mixer generator B = sum_q X_q. (The paper prints
 *     H_X = -sum_q X_q; that convention is this library's with beta -> -beta.)
 *   - Section IV: the candidate sub-solution is read from the final state; this library returns
 *     the k most probable bitstrings (probability descending, ties to the smaller index).
 *   - Section V-A: random and impact-factor-directed (Algorithm 1) decomposition into
 *     sub-QUBOs; Section V step 3: aggregation that accepts only energy-lowering updates.
 *
 * Index convention: bit q of a basis index z is qubit q, which is sub-QUBO variable q (for a
 * decomposed sub-QUBO, global variable idx[q], the index set sorted ascending).
 *
 * Memory: every pointer marked "device" is caller-owned device memory; "host" is caller-owned
 * host memory. The library allocates only in qaoa_create, qaoa_reserve and the plan calls,
 * never inside a launch call. Calls marked "async" enqueue work on `stream` and return at once;
 * their outputs are valid once the stream has reached that point. Complex arrays are
 * interleaved (re, im): complex64 = two floats (8 bytes), complex128 = two doubles.
 *
 * Errors: every call returns a qaoa_status. Invalid arguments (n < 1 or n > 30, p < 1 or
 * p > 64, k < 0 or k > 16 or k > 2^n, a needed pointer NULL) give QAOA_E_INVALID before any
 * work is enqueued; a failing CUDA call gives QAOA_E_CUDA. qaoa_last_error() returns the
 * message of the last failure of the calling thread.
 */
#ifndef QAOA_H
#define QAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QAOA_OK = 0,
    QAOA_E_INVALID = 1,
    QAOA_E_NOMEM = 2,
    QAOA_E_CUDA = 3,
    QAOA_E_TIMEOUT = 4,
    QAOA_E_UNSUPPORTED = 5
} qaoa_status;

typedef struct qaoa_ctx qaoa_ctx;          /* opaque: device, workspace, launch plans */
typedef struct CUstream_st* qaoa_stream_t; /* a cudaStream_t; NULL is the legacy stream */

/* ---------------------------------------------------------------------------------------- */
/* Context                                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device` (makes it current on the calling thread). */
qaoa_status qaoa_create(qaoa_ctx** out, int device);
/* Free the context and its workspace (synchronises the device first). NULL is ignored. */
void qaoa_destroy(qaoa_ctx* ctx);
/* Message of the last failed call on this thread ("" if none). Valid until the next call. */
const char* qaoa_last_error(void);
/* Grow the context workspace to at least `bytes` (synchronous; allocates). Launch calls that
 * need scratch use this workspace and return QAOA_E_NOMEM if it is too small and cannot grow. */
qaoa_status qaoa_reserve(qaoa_ctx* ctx, size_t bytes);
/* Workspace bytes that qaoa_grad / qaoa_run_layers / qaoa_expect / qaoa_topk need for n qubits
 * (complex64 when dbl == 0, complex128 otherwise). */
size_t qaoa_workspace_bytes(int n, int dbl);

/* Kernel tier of the batched plans for complex64 instances of n qubits (plans created later).
 *   QAOA_TIER_AUTO: the autotuner's stored choice for (n, p), else the library's default
 *     (resident for n <= 14, cluster streaming for n = 15..17, streaming above);
 *   QAOA_TIER_CLUSTER: cluster tier with `param` local qubits per CTA (13 or 14; the cluster
 *     then has 2^(n - param) CTAs, at most 16); only 15 <= n <= 18;
 *   QAOA_TIER_STREAM: HBM streaming; n >= 15; `param` picks the forward passes: 0 TMA passes with
 *     two CTAs per SM (default), 1 TMA passes with one CTA per SM, 2 per-thread cp.async passes;
 *   QAOA_TIER_CSTREAM: cluster streaming (one thread-block cluster per instance runs all its
 *     passes through L2, tiles moved by TMA); 15 <= n <= 17, forward runs only (gradient
 *     instances use the streaming tier). QAOA_E_UNSUPPORTED if the device cannot run it.
 *   QAOA_TIER_RESIDENT: only n <= 14 (always resident); `param` is the widest register window of
 *     the forward sub-passes (5 qubits, or 4 for n <= 13; 0: the default, 4 for n <= 12 and 5
 *     above): a block has 2^(n - window) threads, so 4 doubles the threads per instance.
 * The resident tier is always used for n <= 14. */
enum { QAOA_TIER_AUTO = 0, QAOA_TIER_RESIDENT = 1, QAOA_TIER_CLUSTER = 2, QAOA_TIER_STREAM = 3,
       QAOA_TIER_CSTREAM = 4 };
qaoa_status qaoa_set_tier(qaoa_ctx* ctx, int n, int tier, int param);

/* Autotuner (no counterpart in the paper). Times every kernel configuration that can run a
 * complex64 batch of `count` instances of (n, p) with top-k length k -- for 15 <= n <= 30 the
 * three variants of the streaming tier (param 0, 1, 2 above), for 15 <= n <= 18 also the cluster
 * tier with 13 or 14 local qubits per CTA, for 15 <= n <= 17 the cluster-streaming tier; for
 * 6 <= n <= 14 the resident tier's register windows of 5 and (n <= 13) 4 qubits (the block sizes
 * they imply); for n <= 5 the single configuration -- on synthetic inputs (best of 5 timed plan
 * launches on `stream`, CUDA events) and stores the fastest (tier, param) for (n, p) in the
 * context; plans created later use it unless qaoa_set_tier overrides n. best_ms (may be NULL):
 * the winning batch time. Synchronous; allocates temporary buffers. */
qaoa_status qaoa_autotune(qaoa_ctx* ctx, int n, int p, int k, int count, qaoa_stream_t stream,
                          double* best_ms);
/* The stored choice for (n, p): tier 0 when none; param as in qaoa_set_tier. */
qaoa_status qaoa_tuning_get(qaoa_ctx* ctx, int n, int p, int* tier, int* param, double* ms);
/* Save / load the stored choices as JSON ({"format": "libqaoa-tuning-1", "entries": [...]}).
 * Loading adds the file's valid entries to the context. */
qaoa_status qaoa_tuning_save(qaoa_ctx* ctx, const char* path);
qaoa_status qaoa_tuning_load(qaoa_ctx* ctx, const char* path);

/* ---------------------------------------------------------------------------------------- */
/* Single instance, complex64 (FP32 energies). All pointers device, all calls async.         */
/* ---------------------------------------------------------------------------------------- */

/* E[z] = z^T Q z for z = 0..2^n-1 (Section IV, QUBO -> diagonal Hamiltonian).
 * Q: n*n floats, row-major; read as given (E uses Q_ij and Q_ji as separate terms).
 * E: 2^n floats. Built by Gray-code increments from direct FP32 evaluations. */
qaoa_status qaoa_build_energies(qaoa_ctx* ctx, int n, const float* Q, float* E,
                                qaoa_stream_t stream);

/* Apply p layers of Eq. 2 to psi in place: for l = 0..p-1, psi(z) *= e^{-i gamma[l] E(z)},
 * then e^{-i beta[l] X_q} on every qubit q. gamma, beta: p floats (device). E: 2^n floats.
 * psi: 2^n complex64 (in/out); with init_plus != 0 it is first set to |+> (not read). */
qaoa_status qaoa_run_layers(qaoa_ctx* ctx, int n, int p, const float* gamma, const float* beta,
                            const float* E, void* psi, int init_plus, qaoa_stream_t stream);

/* <C> = sum_z |psi(z)|^2 E(z) (Section IV, the cost C(theta) that the outer loop minimises).
 * psi: 2^n complex64, E: 2^n floats, out: one double (device). FP32 products summed in FP32
 * over at most 32 terms, FP64 above that, in a fixed order (deterministic). Uses workspace. */
qaoa_status qaoa_expect(qaoa_ctx* ctx, int n, const void* psi, const float* E, double* out,
                        qaoa_stream_t stream);

/* The k (1..16) most probable basis states of psi (Section IV, the measured candidate
 * sub-solution): idx[k] uint64 and prob[k] doubles (device; prob may be NULL), probability
 * descending, ties broken by the smaller index. prob = re*re + im*im of the stored complex64
 * amplitude, evaluated exactly in FP64 (one rounding). Uses workspace. */
qaoa_status qaoa_topk(qaoa_ctx* ctx, int n, const void* psi, int k, uint64_t* idx, double* prob,
                      qaoa_stream_t stream);

/* Measurement shots of a complex64 state (Section IV: the paper reads the sub-solution from
 * measured shots; qaoa_topk is this library's default). Shot s returns the smallest basis index z
 * whose cumulative probability exceeds u[s] times the total probability (inverse-CDF sampling
 * over |psi|^2 in FP64), with the caller's uniforms u[s] in [0, 1), so that a seeded generator
 * reproduces the shots. The cumulative sums are FP64 sums over parts of 2^(n-12) amplitudes
 * (n > 12), then a warp prefix scan inside a part: against a sequential sum, a uniform within a
 * few ulps of a boundary may select the neighbouring index. A target that no running sum exceeds
 * (rounding) returns the last nonzero amplitude of its part.
 *   n: 1..30; psi: 2^n complex64 (device), not all zero; shots: 0..2^26; u: shots doubles
 *   (device); out: shots uint64 (device). Uses workspace. Asynchronous on `stream`. */
qaoa_status qaoa_sample(qaoa_ctx* ctx, int n, const void* psi, int64_t shots, const double* u,
                        uint64_t* out, qaoa_stream_t stream);

/* Derivative-free minimisation for the gradient-free outer loop of Section IV (the paper tunes
 * each sub-QUBO's angles with COBYLA; this library's default is the adjoint gradient with Adam).
 * The method of Powell (1994), unconstrained case: a linear interpolation model on a simplex of
 * nvar + 1 points, trust-region steps of length rho against the model gradient, geometry steps
 * that keep the simplex well shaped, rho halved from rhobeg down to rhoend. Host code, no GPU.
 * Reverse communication: qaoa_cobyla_ask writes the next point to evaluate into x and returns 1
 * (the caller evaluates f there and calls qaoa_cobyla_tell), or writes the best point found and
 * returns 0 once rho has reached rhoend or maxfun values have been told. So many independent
 * minimisations can have their points evaluated together, e.g. one batched plan launch for every
 * sub-QUBO of a batch. nvar 1..256, 0 < rhoend <= rhobeg, maxfun >= nvar + 2, else create returns
 * QAOA_E_INVALID and allocates nothing. Non-finite values count as +inf. x: nvar host doubles
 * (the caller's). tell on a finished minimisation returns QAOA_E_INVALID; ask with a NULL state
 * or x returns 0. The state is owned by the caller and freed by qaoa_cobyla_destroy (NULL is a
 * no-op). Not thread-safe per state; independent states may be used from different threads. */
typedef struct qaoa_cobyla qaoa_cobyla;
qaoa_status qaoa_cobyla_create(int nvar, const double* x0, double rhobeg, double rhoend, int maxfun,
                               qaoa_cobyla** out);
int qaoa_cobyla_ask(qaoa_cobyla* s, double* x);
qaoa_status qaoa_cobyla_tell(qaoa_cobyla* s, double f);
/* Best point, its value and the number of values told so far (any pointer may be NULL). */
qaoa_status qaoa_cobyla_result(qaoa_cobyla* s, double* x, double* f, int* nfev);
void qaoa_cobyla_destroy(qaoa_cobyla* s);

/* <C> and top-k of a complex64 state, like qaoa_expect and qaoa_topk together, for callers that
 * cannot allocate device memory: code whose device memory is owned by another allocator or a
 * fixed budget (a host framework's memory pool, where an extra cudaMalloc fragments or exceeds
 * it), latency-critical loops that must not pay for cudaMalloc's implicit synchronisation, and
 * thin callers that hold no qaoa_ctx (and so no workspace). It needs no context and allocates
 * nothing: its scratch, the per-block partial sums and top-k lists (at most 1024 blocks x 16
 * entries, about 200 KB), is one fixed array inside the library, reserved on every GPU that
 * loads the library and held until the process exits. The paper has no counterpart.
 *   n: 1..30 (larger n is rejected with QAOA_E_INVALID); k: 0..16 and <= 2^n (0: no top-k);
 *   psi: 2^n complex64, E: 2^n floats (may be NULL when expect is NULL); expect: one double;
 *   idx: k uint64, prob: k doubles (may be NULL); all device pointers. Same results and order
 *   rules as qaoa_expect / qaoa_topk. Async on `stream`.
 * The first call on a device looks up the array's device address with that device current;
 * make that first call before any stream capture. The address is kept with the id of the
 * device's context, so the first call after that context is replaced (cudaDeviceReset) looks it
 * up again; that call too belongs outside a capture. Every call uses the same array, which keeps
 * the last call's contents (each call writes every slot before reading it, so nothing needs
 * clearing); calls whose work overlaps on the GPU (other streams, other host threads) race on it
 * and must be ordered by the caller. */
qaoa_status qaoa_expect_topk_static(int n, const void* psi, const float* E, int k, double* expect,
                                    uint64_t* idx, double* prob, qaoa_stream_t stream);

/* Adjoint gradient of <C> with respect to (gamma, beta) from |+> through p layers: the reverse
 * state-vector sweep of Jones & Gacon (2020, "Efficient calculation of gradients in classical
 * simulations of variational quantum algorithms"), the gradient source that stands in for the
 * paper's gradient-free COBYLA loop over the angles of Eq. 2 (Section IV).
 * expect (1 double, may be NULL), dgamma[p], dbeta[p] doubles (device). Uses workspace for the
 * forward and adjoint states when n exceeds the shared-memory tier. */
qaoa_status qaoa_grad(qaoa_ctx* ctx, int n, int p, const float* gamma, const float* beta,
                      const float* E, double* expect, double* dgamma, double* dbeta,
                      qaoa_stream_t stream);

/* ---- complex128 variants (FP64 energies, same semantics and layouts) ---- */
qaoa_status qaoa_build_energies_z(qaoa_ctx* ctx, int n, const double* Q, double* E,
                                  qaoa_stream_t stream);
qaoa_status qaoa_run_layers_z(qaoa_ctx* ctx, int n, int p, const double* gamma,
                              const double* beta, const double* E, void* psi, int init_plus,
                              qaoa_stream_t stream);
qaoa_status qaoa_expect_z(qaoa_ctx* ctx, int n, const void* psi, const double* E, double* out,
                          qaoa_stream_t stream);
qaoa_status qaoa_topk_z(qaoa_ctx* ctx, int n, const void* psi, int k, uint64_t* idx,
                        double* prob, qaoa_stream_t stream);
qaoa_status qaoa_grad_z(qaoa_ctx* ctx, int n, int p, const double* gamma, const double* beta,
                        const double* E, double* expect, double* dgamma, double* dbeta,
                        qaoa_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Batched sub-QUBO solves (Section V step 2: the sub-QUBOs of a cycle solved in parallel).  */
/* ---------------------------------------------------------------------------------------- */

enum { QAOA_INST_GRAD = 1 };

/* One instance. Offsets are element offsets into the pools of qaoa_batch_io. */
typedef struct {
    int32_t n;        /* qubits, 1..30 */
    int32_t p;        /* layers, 1..64 */
    int32_t k;        /* top-k length, 0..16 (0: no top-k) */
    int32_t flags;    /* QAOA_INST_GRAD: also d<C>/d(gamma, beta) */
    int64_t q_off;    /* n*n row-major Q at io->q + q_off */
    int64_t par_off;  /* gamma[p] then beta[p] at io->params + par_off; gradients at the same
                         offsets in io->grad */
    int64_t psi_off;  /* final state (2^n complex) at io->psi + psi_off, or -1: not returned */
    int64_t e_off;    /* energies (2^n) at io->e + e_off (8-byte aligned), or -1: not returned */
} qaoa_inst;

typedef struct {
    const void* q;       /* device: Q pool (float, or double for _z) */
    const void* params;  /* device: parameter pool (float, or double for _z) */
    void* psi;           /* device: state pool (complex64 / complex128) or NULL */
    void* e;             /* device: energy pool or NULL */
    double* expect;      /* device: count doubles, <C> of instance i at expect[i] */
    uint64_t* topk_idx;  /* device: count * k_stride, instance i at i * k_stride */
    double* topk_prob;   /* device: same layout, may be NULL */
    int32_t k_stride;
    double* grad;        /* device: gradient pool (same offsets as params) or NULL */
} qaoa_batch_io;

typedef struct qaoa_plan qaoa_plan;

/* Validate the descriptors (host array, `count` entries), choose a kernel tier per instance
 * (shared-memory resident, cluster, or HBM streaming) and upload the device descriptor
 * tables. Synchronous; allocates the plan's device memory. The io pointers are bound into the
 * plan: a later launch reads and writes the same buffers. */
qaoa_status qaoa_plan_create(qaoa_ctx* ctx, const qaoa_inst* desc, int count,
                             const qaoa_batch_io* io, int dbl, qaoa_plan** out);
/* Enqueue the whole batch on `stream` (kernel launches and memsets only, so the call can be
 * captured in a CUDA graph). Async. */
qaoa_status qaoa_plan_launch(qaoa_plan* plan, qaoa_stream_t stream);
/* Record the plan's launch sequence once into a CUDA graph (stream capture on `stream`, which
 * must not be capturing already); every later qaoa_plan_launch replays the graph with one
 * cudaGraphLaunch instead of issuing each kernel. The graph reads the same bound buffers, so
 * new inputs written there are picked up. Per-kernel timing is not available for a captured
 * plan. Synchronous. */
qaoa_status qaoa_plan_capture(qaoa_plan* plan, qaoa_stream_t stream);
/* Number of kernel launches one qaoa_plan_launch enqueues. */
int qaoa_plan_kernel_count(const qaoa_plan* plan);
/* Per-kernel timing: with on != 0 every later qaoa_plan_launch records a CUDA event before and
 * after each kernel on the launch stream. qaoa_plan_kernel_times then writes, for the last
 * launch, up to `max` entries: the duration in ms of kernel i (after synchronising on the last
 * event) and, in names (may be NULL), a pointer to a static string naming its kernel family. */
qaoa_status qaoa_plan_set_timing(qaoa_plan* plan, int on);
int qaoa_plan_kernel_times(qaoa_plan* plan, float* ms, const char** names, int max);
/* Algorithmic DRAM bytes of each kernel of one launch, in launch order (the bytes the
 * computation must move: states, energies and matrices read or written once, no re-reads);
 * returns the number of kernels written (at most max). */
int qaoa_plan_kernel_bytes(const qaoa_plan* plan, double* bytes, int max);
/* Device status of the plan's launches so far (synchronous: reads one word). Kernels with
 * device-side waits bound each wait; a wait that ran out sets the plan's status word, and this
 * call then returns QAOA_E_TIMEOUT (sticky for the plan). qaoa_batch_run and
 * dqaoa_session_cycle check it at their synchronisation point. */
qaoa_status qaoa_plan_check(qaoa_plan* plan);
/* Free the plan (synchronises the device first). NULL is ignored. */
void qaoa_plan_destroy(qaoa_plan* plan);

/* plan_create + plan_launch + (after a stream synchronisation) plan_destroy. Synchronous.
 * The plan (descriptors and streaming scratch) is placed in the context workspace when that is
 * at least as large as the plan (size it with qaoa_reserve): the call then allocates nothing.
 * Otherwise the plan is allocated for the call, so repeated calls belong on a set-up path;
 * the allocation-free hot path is a plan created once and launched with qaoa_plan_launch. */
qaoa_status qaoa_batch_run(qaoa_ctx* ctx, const qaoa_inst* desc, int count,
                           const qaoa_batch_io* io, qaoa_stream_t stream);
qaoa_status qaoa_batch_run_z(qaoa_ctx* ctx, const qaoa_inst* desc, int count,
                             const qaoa_batch_io* io, qaoa_stream_t stream);

/* One Adam step (Kingma & Ba 2015) on `count` parameters, the optimiser that replaces the
 * paper's COBYLA outer loop (Section IV): theta (floats, in/out), grad (doubles, e.g. the grad
 * pool of a batch with QAOA_INST_GRAD), m and v (floats, in/out, zero before step 1), all device;
 * step >= 1 is the 1-based step number used for bias correction. minimise != 0 descends <C>.
 * Async on `stream`. */
qaoa_status qaoa_adam_step(int count, float* theta, const double* grad, float* m, float* v,
                           int step, float lr, float beta1, float beta2, float eps, int minimise,
                           qaoa_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Reference "plain" GPU path: one instance per call, one kernel per gate (cost phase, one    */
/* kernel per qubit for the mixer) and a separate reduction. The comparison point of the     */
/* batched path; same arguments as qaoa_run_layers plus the reductions.                     */
/* ---------------------------------------------------------------------------------------- */
qaoa_status qaoa_plain_solve(qaoa_ctx* ctx, int n, int p, const float* Q, const float* gamma,
                             const float* beta, float* E, void* psi, int k, double* expect,
                             uint64_t* topk_idx, double* topk_prob, qaoa_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* DQAOA decomposition and aggregation (host, FP64)                                          */
/* ---------------------------------------------------------------------------------------- */

enum { DQAOA_RANDOM = 0, DQAOA_IFD = 1, DQAOA_BFS = 2, DQAOA_PFS = 3, DQAOA_SIGNED_IMPACT = 16,
       DQAOA_PAPER_MIXER = 32 };

/* Section V-A. Sub-QUBO index sets: idx[m*k] (host int32), each row sorted ascending.
 *   DQAOA_RANDOM: row j draws k distinct variables of 0..N-1 uniformly without replacement,
 *     SplitMix64 seeded with seed ^ (cycle * 0x9E3779B97F4A7C15) ^ j, partial Fisher-Yates
 *     (swap position i with i + draw(N - i)), draws by Lemire's multiply-shift with rejection.
 *   DQAOA_IFD (Algorithm 1): variables ranked by |impact| descending (ties: smaller index),
 *     impact_i = (1 - 2 x_i)(Q_ii + 2 sum_{j != i} Q_ij x_j), the energy change of flipping x_i;
 *     row j is the window ranking[j .. j+k-1] (needs m + k - 1 <= N; Q and x required).
 *   DQAOA_BFS, DQAOA_PFS (the graph traversals of Section V-A): j is a strong neighbour of i
 *     when j != i, Q_ij != 0 and |Q_ij| >= the d-th largest off-diagonal |Q_i.|, d = min(k - 1,
 *     nonzeros of row i off the diagonal), ties included. Row j starts at ranking[j] (the IFD
 *     ranking). BFS: FIFO queue, the front's strong neighbours join in ascending index order.
 *     PFS: the next variable is the best-ranked unselected strong neighbour of any selected one.
 *     A traversal that runs out restarts at the best-ranked unselected variable. Needs m <= N;
 *     Q and x required.
 *   DQAOA_SIGNED_IMPACT, or-ed with DQAOA_IFD, DQAOA_BFS or DQAOA_PFS: the ranking is impact_i
 *     ascending (the largest energy decrease first, ties: smaller index) instead of |impact_i|
 *     descending; Section V-A does not say which one "higher impact" means. Not valid with
 *     DQAOA_RANDOM; any other bit is invalid.
 * Q: N*N row-major symmetric doubles (host), x: N bytes 0/1 (host; RANDOM may pass NULL). */
qaoa_status dqaoa_draw_indices(const double* Q, int N, const uint8_t* x, int method, int m,
                               int k, uint64_t seed, uint64_t cycle, int32_t* idx);

/* Section V-A sub-QUBO matrices for given index sets: Qsub[j] = Q[S_j, S_j] (k*k full
 * symmetric, host doubles). With conditioned != 0 the couplings to the fixed variables
 * outside S_j are folded into the diagonal, Qsub[a][a] += 2 sum_{l not in S_j} Q[S_a][l] x_l,
 * so the sub-QUBO energy of y is E(x with x_S = y) minus a constant. The paper fixes the value
 * of that sum, not the order of its FP64 additions: here it is 32 interleaved partial sums
 * (l = r mod 32, each ascending) combined by the tree v_r <- v_r + v_{r xor d}, d = 16, 8, 4, 2,
 * 1 (result v_0), the order dqaoa_subqubo_build uses on the device (one warp per row), so host
 * and device matrices agree bit for bit; against any other order (a plain ascending sum) an
 * entry differs by FP64 rounding only. */
qaoa_status dqaoa_decompose(const double* Q, int N, const uint8_t* x, int method, int conditioned,
                            int m, int k, uint64_t seed, uint64_t cycle, int32_t* idx,
                            double* Qsub);

/* The same sub-QUBO matrices built on the device, as FP32 for the complex64 solver:
 * Q_dev N*N doubles, x_dev N bytes, idx_dev m*k int32, qsub_dev m*k*k floats (all device).
 * The conditioning sum is accumulated in FP64 in the order dqaoa_decompose states (32
 * interleaved partial sums combined by an xor tree) and rounded once to FP32. Async. */
qaoa_status dqaoa_subqubo_build(qaoa_ctx* ctx, const double* Q_dev, int N, const uint8_t* x_dev,
                                int m, int k, const int32_t* idx_dev, int conditioned,
                                float* qsub_dev, qaoa_stream_t stream);

/* Section V step 3, aggregation. Sequential over sub-QUBOs j = 0..m-1 and, within j, over the
 * K candidate bitstrings cand[j*K .. j*K+K-1] (host uint64; bit q sets variable idx[j*k+q]) in
 * the given order: a candidate replaces x on S_j when dE = E(x') - E(x) < -tau,
 * tau = 1e-12 sum |Q_ij|. dE = sum_{a: d_a != 0} d_a (2 (Qx)_a + sum_{b: d_b != 0} Q_ab d_b),
 * d = x' - x, with Qx kept up to date as variables flip. x: N bytes (host, in/out);
 * energy_out: E(x') = x'^T Q x' (host double, may be NULL); accepted_out: number of accepted
 * candidates (may be NULL). k <= 64. Synchronous. */
qaoa_status dqaoa_merge(const double* Q, int N, uint8_t* x, int m, int k, const int32_t* idx,
                        int K, const uint64_t* cand, double* energy_out, int* accepted_out);


/* ---------------------------------------------------------------------------------------- */
/* One DQAOA cycle in one call (Section V: decompose -> solve the sub-QUBOs in parallel ->    */
/* aggregate). A session owns the device copies of Q and x, the sub-QUBO pools, a batched    */
/* plan for m sub-QUBOs of k qubits at depth p, and pinned staging buffers.                  */
/* ---------------------------------------------------------------------------------------- */

typedef struct dqaoa_session dqaoa_session;

/* gamma, beta: p host doubles (the fixed parameters every sub-QUBO uses); K: top-k candidates
 * per sub-QUBO fed to the merge (1..16); method: one of DQAOA_RANDOM, DQAOA_IFD, DQAOA_BFS,
 * DQAOA_PFS, the last three optionally | DQAOA_SIGNED_IMPACT, and any of them optionally
 * | DQAOA_PAPER_MIXER: the mixer of Section IV's ansatz as printed, H_X = -sum_i X_i, i.e.
 * e^{+i beta_l sum X} per layer; without it the session applies e^{-i beta_l sum X} (the two are
 * the same circuit at beta -> -beta, which is how the flag is applied: the session stores -beta).
 * Allocates. */
qaoa_status dqaoa_session_create(qaoa_ctx* ctx, int N, int m, int k, int p, int K, int method,
                                 int conditioned, const double* gamma, const double* beta,
                                 dqaoa_session** out);
/* Run one cycle. Q: N*N host doubles (copied to the device when q_changed != 0, which the
 * first call needs); x: N host bytes, in/out (the global solution). seed/cycle select the
 * random index sets. energy_out: E(x') (may be NULL); accepted_out: accepted candidates (may
 * be NULL). Steps: index draw (host) -> sub-QUBO build, energies, p layers, <C> and top-K
 * (device, one stream) -> merge (host). Synchronous on `stream`. */
qaoa_status dqaoa_session_cycle(dqaoa_session* s, const double* Q, int q_changed, uint8_t* x,
                                uint64_t seed, uint64_t cycle, double* energy_out,
                                int* accepted_out, qaoa_stream_t stream);
/* Device work of the last cycle: per-sub-QUBO <C> (m doubles) and top-K indices (m*K uint64),
 * copied to host arrays (either may be NULL). A sampled cycle computes no top-K: after one,
 * expect is its <C> and topk is still the last dqaoa_session_cycle's. */
qaoa_status dqaoa_session_results(dqaoa_session* s, double* expect, uint64_t* topk);
/* A cycle whose sub-solutions are read from measured shots, as Section IV reads the candidate
 * bitstring from a measurement of the optimised state (dqaoa_session_cycle takes the top-K
 * bitstrings instead). Decomposition and solve as in dqaoa_session_cycle; then each sub-QUBO's
 * final state is sampled `shots` times by inverse CDF over |psi|^2 (qaoa_sample) with the
 * caller's uniforms u[j*shots + s] in [0, 1) (host doubles, m*shots), and the merge receives one
 * candidate per sub-QUBO: the shot of lowest sub-QUBO energy y^T Qsub_j y, evaluated in FP64 on
 * the sub-QUBO matrix of dqaoa_subqubo_build before its FP32 rounding (ties: the smaller
 * bitstring). This is the best measurement of the shots, the sub-solution the paper's QAOA
 * solver returns. shots: 1..2^20. The first call allocates the session's state pool
 * (m * 2^k complex64), its sampler scratch and a plan over all m sub-QUBOs; a call with more
 * shots than any before reallocates the shot buffers. Synchronous on `stream`; QAOA_E_TIMEOUT
 * when a device-side wait of the solve ran out (x is then left unchanged). */
qaoa_status dqaoa_session_cycle_sampled(dqaoa_session* s, const double* Q, int q_changed, uint8_t* x,
                                        uint64_t seed, uint64_t cycle, int shots, const double* u,
                                        double* energy_out, int* accepted_out, qaoa_stream_t stream);
/* Of the last sampled cycle, copied to host arrays (any may be NULL): the shots (m*shots
 * uint64, sub-QUBO j at j*shots), the candidate chosen per sub-QUBO (m uint64), and the final
 * states (m * 2^k complex64, standard frame, sub-QUBO j at j * 2^k). QAOA_E_INVALID before the
 * first sampled cycle. Synchronous. */
qaoa_status dqaoa_session_shots(dqaoa_session* s, uint64_t* shots_out, uint64_t* best_out, void* psi_out);
/* Times of the last cycle in ms, out[4]: the host's decompose-and-enqueue time (index draw,
 * copies and launches), the device time from the first copy to the last chunk's results, the
 * host merge time (the first chunk's merge overlaps the device), and the whole call. */
qaoa_status dqaoa_session_timing(dqaoa_session* s, double* out);
/* Device time of the last dqaoa_session_cycle's solve in ms: from the first chunk's launch to
 * the end of the last chunk's kernels (the chunks may overlap on the device). */
qaoa_status dqaoa_session_solve_ms(dqaoa_session* s, double* ms);
/* The batched plans the session launches, in order (for timing and kernel counts): the m
 * sub-QUBOs are solved in two chunks when m >= 128, else in one, the second on its own stream
 * (the two solves overlap on the device). The host merges the first chunk while the device
 * solves the second; the first holds floor(11 m / 16) sub-QUBOs (floor(9 m / 16) for N > 4096)
 * for the cluster-streaming tier,
 * else ceil(0.65 m) rounded up to a multiple of the instances whose tiles give each block of a
 * streaming launch one tile (at most m - 1). Returns NULL for i past the last plan. */
qaoa_plan* dqaoa_session_plan(dqaoa_session* s, int i);
void dqaoa_session_destroy(dqaoa_session* s);

/* ---------------------------------------------------------------------------------------- */
/* Serving: continuous batching of optimise-and-sample jobs. A job is one sub-QUBO (n, p, Q,  */
/* initial gamma/beta) that runs `steps` Adam steps on <C> (adjoint gradients; Adam replaces  */
/* the paper's COBYLA loop of Section IV) and then one forward pass returning <C> and the     */
/* top-k bitstrings at the final parameters (the sample step of Section V step 2). Jobs wait  */
/* in a FIFO queue and are admitted while a job slot and the job's scratch bytes (the HBM      */
/* footprint of its state buffers, qaoa_server_job_bytes) are free. Every tick runs one step   */
/* of every admitted job in a single batched launch; jobs join and leave between ticks. Q,    */
/* parameters, gradients and Adam moments stay on the device for the job's life. The kernels  */
/* are batch-invariant: a job's results do not depend on the other jobs of its ticks.         */
/* This has no counterpart in the paper (its sub-QUBOs run to completion one per core).       */
/* Single-threaded use. All memory is allocated by qaoa_server_create.                        */
/* ---------------------------------------------------------------------------------------- */

typedef struct qaoa_server qaoa_server;

typedef struct {
    int64_t job_id;
    int32_t n, p, steps, k;
    double expect;          /* <C> at the final parameters */
    uint64_t topk_idx[16];  /* k most probable bitstrings (probability desc, index asc) */
    double topk_prob[16];   /* their probabilities; unused entries -1 */
    float params[128];      /* final gamma[p] then beta[p] */
    double t_submit;        /* qaoa_server_clock() at submission */
    double t_done;          /* qaoa_server_clock() when poll saw the result */
} qaoa_job_result;

/* scratch_bytes: device bytes for the jobs' state buffers (admission budget); max_jobs: job
 * slots (1..65536); k: top-k length of the final pass (0..16). Allocates the job pools, the
 * scratch and pinned staging. Uses the current device. */
qaoa_status qaoa_server_create(qaoa_ctx* ctx, size_t scratch_bytes, int max_jobs, int k,
                               qaoa_server** out);
void qaoa_server_destroy(qaoa_server* s);
/* Scratch bytes a job of n qubits and p layers occupies while admitted. */
size_t qaoa_server_job_bytes(qaoa_server* s, int n, int p);
/* Queue a job. Q: n*n host floats (row-major); params: 2p host floats (gamma then beta);
 * steps >= 0 Adam steps at learning rate lr. Copies the inputs. QAOA_E_NOMEM if the job could
 * never fit the scratch budget. job_id may be NULL. */
qaoa_status qaoa_server_submit(qaoa_server* s, int n, int p, const float* Q, const float* params,
                               int steps, float lr, int64_t* job_id);
/* Admit queued jobs that fit, then enqueue one step of every admitted job on `stream` (async;
 * blocks only when three earlier ticks are still running). active/queued (may be NULL): jobs
 * admitted and waiting after admission. */
qaoa_status qaoa_server_tick(qaoa_server* s, qaoa_stream_t stream, int* active, int* queued);
/* Copy up to max finished jobs into out (in completion order) and return how many; with
 * wait != 0 first waits for every tick in flight. */
int qaoa_server_poll(qaoa_server* s, int wait, qaoa_job_result* out, int max);
/* Withdraw a job. A queued job leaves the queue; an admitted job leaves between ticks (its slot
 * and scratch are free for the next admission; the ticks already enqueued still run its step,
 * and no result of it is ever returned). QAOA_E_INVALID when the id is unknown, already
 * returned, or the job's final pass is already enqueued. */
qaoa_status qaoa_server_cancel(qaoa_server* s, int64_t job_id);
/* Fault injection on the host: the next `count` admission attempts fail as if the job's scratch
 * could not be allocated (the job keeps its place at the head of the queue, admission stops for
 * that tick and resumes at the next; the jobs already admitted run on). failures (may be NULL):
 * admission failures so far. count 0 clears a pending injection. */
qaoa_status qaoa_server_fail_admissions(qaoa_server* s, int count, long long* failures);
/* Queue and admission state, plus totals over the ticks so far: the algorithmic DRAM bytes of
 * every launched tick, the device time of the ticks already harvested and the kernel launches
 * enqueued (any may be NULL). */
qaoa_status qaoa_server_stats(qaoa_server* s, int* queued, int* active, size_t* scratch_used,
                              double* bytes_total, double* gpu_ms_total, long long* launches);
/* Monotonic host clock in seconds (the time base of t_submit / t_done). */
double qaoa_server_clock(void);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_H */
