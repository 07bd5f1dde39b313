/*
 * csfast — fast correlation for matching pursuit on GB300 (sm_103a).
 *
 * C ABI of libcsfast.so.  The library implements, for partial unitary sensing
 * matrices Phi = S_Omega A with A the unitary Walsh–Hadamard (Sylvester,
 * A(i,k) = (-1)^popcount(i&k)/sqrt(N)) or DFT (A(i,k) = exp(-2 pi i ik/N)/sqrt(N))
 * matrix (Sec. I of Kim et al., arXiv 1205.4139):
 *
 *   - the correlation kernel vector c = U^H S^T S U e_1      (Eq. kernelsum)
 *   - the conventional correlation h = Phi^H r              (Algorithm 1.1, step 2)
 *   - the fast correlation h = h_0 - sum x(t) P_{lambda_t} c (Eq. kernelsumOMP)
 *   - OMP (Algorithm 1.1) with either correlation, or the adaptive switch of
 *     Sec. IV, and an FP64 least-squares update whose Gram entries are read
 *     off c.
 *
 * Conventions for every entry point:
 *   - Indices are 0-based.  N is a power of two.  Omega is sorted ascending,
 *     duplicate-free, with entries in [0, N).
 *   - Element type F of r, y, h, h_0 and the correlation-side x follows the
 *     plan's (kind, prec):  WHT+FP64 double, WHT+FP32 float,
 *     DFT+FP64 double2 (re, im interleaved), DFT+FP32 float2.
 *     OMP coefficients (x_dev of cs_omp) are always FP64: double for WHT,
 *     interleaved complex double for DFT.
 *   - Pointers named *_dev are device pointers owned by the caller; they must
 *     stay valid until the work queued on `stream` has completed.  `stream`
 *     is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - Batched arrays are dense row-major: instance b of an F[n] array starts
 *     at element b*n.
 *   - A plan owns its device tables and a workspace that grows on demand.
 *     Calls that use the same plan must not overlap in time (queue them on
 *     one stream); different plans are independent.
 *   - Errors: argument problems are reported synchronously as CS_ERR_INVALID
 *     before anything is queued; sizes beyond the kernels' limits give
 *     CS_ERR_UNSUPPORTED; a failing CUDA call gives CS_ERR_CUDA (text via
 *     cs_last_error).  The library never aborts the process.
 */
#ifndef CSFAST_H
#define CSFAST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_plan_s* cs_plan_t;

typedef enum {
  CS_OK = 0,
  CS_ERR_INVALID = 1,
  CS_ERR_NOMEM = 2,
  CS_ERR_CUDA = 3,
  CS_ERR_UNSUPPORTED = 4
} cs_status;

typedef enum { CS_WHT = 0, CS_DFT = 1 } cs_kind;
typedef enum { CS_FP64 = 0, CS_FP32 = 1 } cs_prec;

/* Which correlation OMP uses at iteration t (t = 1 is always one transform,
 * Eq. kernelsumOMP):  FAST = kernel sums for every t > 1;  CONV = a transform
 * of the zero-filled residual at every t (Algorithm 1.1 step 2);  HYBRID =
 * kernel sums while t <= t_switch, transforms after (the adaptive strategy of
 * Sec. IV). */
typedef enum { CS_PATH_FAST = 0, CS_PATH_CONV = 1, CS_PATH_HYBRID = 2 } cs_path;

/* Halting rule of Algorithm 1.1 step 8 (the paper leaves it open): stop after
 * K iterations, or as soon as ||r_t|| < rel_tol * ||y|| (rel_tol = 0 disables
 * the tolerance).  A zero measurement halts before the first iteration; a
 * selected column whose Cholesky pivot is <= 1e-10 * M/N (numerically
 * dependent on the support) ends the run without being added.
 * t_switch < 0 selects the plan's switch point (cs_plan_switch): the one
 * cs_plan_tune measured, if it has run on this plan, else a crossover table
 * measured on GB300 by log2 N (the flop-model point of cs_plan_info is far
 * lower than the measured crossovers).
 * max_iter bounds the iterations of cs_sp / cs_cosamp (<= 0: K for SP, 50 for
 * CoSaMP); cs_omp ignores it (its bound is K). */
typedef struct {
  double rel_tol;
  int32_t path;
  int32_t t_switch;
  int32_t max_iter;
} cs_halt;

/* Build a plan for Phi = S_Omega A (Sec. I).  Computes on the device the
 * correlation kernel vector c = U^H S^T S U e_1 of Eq. (kernelsum) in FP64
 * (and rounded to FP32 for FP32 plans), the transform twiddles and the index
 * maps of Omega.  `omega_host` is a host array of M int32 (M may be 0).
 * Blocks until the plan's tables are built.  Limits: 1 <= N <= 2^24,
 * 0 <= M <= N.  Plans with N <= 8192 keep a whole instance on one SM (one
 * fused kernel per call); larger plans spread each instance over the GPU
 * with four-step transforms through global memory and queue a short
 * sequence of kernels per iteration (at most 65535 instances per call;
 * cs_omp_noalloc returns CS_ERR_UNSUPPORTED for them).  Plans with
 * 8192 < N <= 2^16 also keep the tables cs_omp_batched runs them with on one
 * SM (a DFT plan: its slot map in the one-CTA chains' order; the chains'
 * twiddles are built once per N and device and shared by all plans). */
cs_status cs_plan_create(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind,
                         int32_t prec, void* stream, cs_plan_t* out);

/* Storage of the correlation kernel vector (the paper's storage remarks,
 * Sec. III-B), chosen at plan creation; results are those of the full
 * vector up to FP rounding (CS_PLAN_C_INT: bit for bit):
 *   CS_PLAN_C_HALF  DFT: c is conjugate symmetric, c(N - d) = conj(c(d)), so
 *                   only d <= N/2 is stored (half the memory of c)
 *   CS_PLAN_C_INT   WHT: N c(d) = M - 2 #{i in Omega : popcount(i & d) odd}
 *                   is an integer, stored exactly as int32 (half the memory
 *                   of an FP64 c, no FP copy) */
enum { CS_PLAN_C_HALF = 1u, CS_PLAN_C_INT = 2u, CS_PLAN_TENSOR_CORES = 4u };

/* Tensor-core Hadamard transform (WHT FP32 plans).  cs_correlate computes
 * the fast Hadamard transform of Sec. III-B (Table I, 2N log2 N) with its
 * radix-16 stages on the tensor cores: each 16-point group is multiplied by
 * the +-1 matrix H_16 (tcgen05 MMAs, the FP32 data split exactly into three
 * BF16 parts, FP32 accumulation in tensor memory), the remaining radix-2, -4
 * or -8 stage on the CUDA cores; results agree with the FP32 transform to
 * FP32 accumulation error (bit-exact on a single nonzero).  This is the
 * default for 16 <= N <= 512, where it is faster on GB300 than the CUDA-core
 * butterflies; CS_PLAN_TENSOR_CORES extends it to N <= 4096, where the
 * butterflies are faster (the transform moves more bytes than it does
 * arithmetic, and splitting the operands costs more instructions than the
 * butterflies it replaces).  A device-detected timeout of the tensor-core
 * pipeline sets bit 1 of the plan's status word. */

/* cs_plan_create with storage flags (0 = full vector, as cs_plan_create).
 * CS_ERR_INVALID for unknown flags, CS_PLAN_C_HALF on a WHT plan,
 * CS_PLAN_C_INT on a DFT plan, both, or CS_PLAN_TENSOR_CORES on anything but
 * a WHT FP32 plan. */
cs_status cs_plan_create_ex(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                            uint32_t flags, void* stream, cs_plan_t* out);

/* Device bytes held by the plan's tables (slot maps, Omega grouped by
 * four-step row and by column for N > 8192, c in its storage format, twiddles, status
 * word), not counting the workspace or the chain twiddles shared by all
 * plans of one N. */
cs_status cs_plan_memory(cs_plan_t plan, int64_t* table_bytes);

/* Release the plan's device memory (synchronises the device first). */
cs_status cs_plan_destroy(cs_plan_t plan);

/* Report the plan's sizes and its flop-model hybrid switch point: the
 * largest t whose kernel-sum cost is no more than one transform's in the flop
 * model of Table I (Sec. IV's "excessive point").  Any output pointer may be
 * NULL. */
cs_status cs_plan_info(cs_plan_t plan, int64_t* N, int64_t* M, int32_t* kind, int32_t* prec,
                       int32_t* t_switch_default);

/* The switch point calls with t_switch < 0 use: cs_plan_tune's, if it has
 * run on this plan, else a GB300 default for the plan's N (64 for N <= 8192;
 * 128 to 160 for 2^14 <= N <= 2^19; 96 for larger N). */
cs_status cs_plan_switch(cs_plan_t plan, int32_t* t_switch);

/* Errors the kernels detected on the device since the last call (0 = none;
 * bit 0: an OMP launch stopped because its phase loop reached its bound,
 * which leaves that launch's outputs incomplete; bit 1: a tensor-core
 * transform's MMAs did not complete within its wait bound, which leaves that
 * call's outputs incomplete).  Synchronises `stream`,
 * then clears the word. */
cs_status cs_plan_status(cs_plan_t plan, int32_t* device_error, void* stream);

/* Copy the correlation kernel vector c (Eq. kernelsum) into c_dev:
 * `prec` CS_FP64 gives double / double2 [N], CS_FP32 float / float2 [N]. */
cs_status cs_plan_kernel(cs_plan_t plan, void* c_dev, int32_t prec, void* stream);

/* Conventional correlation (Algorithm 1.1 step 2): for each of `batch`
 * residuals r (F[M], entry m belongs to row Omega_m) computes
 * h = Phi^H r = A^H zf_Omega(r) (F[N]) with one transform.  h_dev may be NULL
 * when only the arg-max is wanted; argmax_dev (int32[batch], NULL allowed)
 * receives argmax_j |h(j)|^2, lowest j on ties (step 3). */
cs_status cs_correlate(cs_plan_t plan, const void* r_dev, int64_t batch, void* h_dev,
                       int32_t* argmax_dev, void* stream);

/* Fast correlation (Eq. kernelsum / kernelsumOMP):
 *   h(j) = h_0(j) - sum_{k<s} x(k) c(j (-) supp(k)),
 * (-) being (j - l) mod N for DFT and j XOR l for WHT.  Per instance:
 * h0 F[N], supp int32[s] (distinct, in [0, N)), x F[s].  h_dev may be NULL;
 * argmax_dev (NULL allowed) receives argmax over j not in supp of |h(j)|^2,
 * lowest j on ties (-1 if every j is in supp). s may be 0 (h = h_0). */
cs_status cs_correlate_fast(cs_plan_t plan, const void* h0_dev, const int32_t* supp_dev,
                            const void* x_dev, int32_t s, int64_t batch, void* h_dev,
                            int32_t* argmax_dev, void* stream);

/* OMP (Algorithm 1.1) on `batch` measurements y (F[M] each) sharing the
 * plan's Omega.  For N <= 8192 the whole batch is one fused persistent kernel:
 * one CTA per instance, or for batch <= 19 and K <= 256 eight CTAs of a
 * cluster per instance (same results bit for bit).  Larger plans run each
 * iteration as a few whole-GPU launches (four-step transform passes,
 * kernel-sum pass, least-squares phases).  Outputs per instance b:
 *   x_dev      FP64 coefficients [K] in selection order (double or
 *              interleaved complex double), zero past iters
 *   supp_dev   int32 [K] support in selection order, -1 past iters
 *   iters_dev  int32: number of selected columns
 *   resnorm_dev double: ||r|| / ||y|| at exit (0 for y = 0), from the FP64
 *              downdate ||r_t||^2 = ||y||^2 - sum |z_k|^2 of the Cholesky
 *              update, or in FP32 mode, once that downdate falls below
 *              1e-5 ||y||^2, from the explicit residual y - Phi x (one
 *              forward transform, FP64 accumulation), on which the
 *              tolerance test is then decided: the FP32 right-hand side
 *              leaves about 1e-7 ||y||^2 of rounding in the downdate, the
 *              explicit residual resolves ||r||/||y|| to a few 1e-7
 * Any output pointer except supp_dev may be NULL (supp_dev too when K = 0).  halt may be NULL
 * (rel_tol 1e-6, hybrid path, default switch).  Limits: 0 <= K <= min(M, 1024)
 * for N <= 8192, 0 <= K <= min(M, 4096) for larger plans. */
cs_status cs_omp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                 void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev,
                 void* stream);

/* OMP (Algorithm 1.1) on `count` independent instances that each have their
 * own plan (own Omega, N, M, kind and precision) and their own K: an uneven
 * batch.  The instances of one element type (kind, precision) and residence
 * (N <= 8192 in shared memory, larger N in global memory) run in one
 * persistent launch (two instances per CTA in shared memory, one per CTA and
 * several CTAs per SM in global memory), instances taken longest first.
 * With more than one launch, each runs on a stream the library owns, forked
 * from `stream` and joined back into it by events.  The call copies its
 * instance table from pageable host memory, so it cannot be captured into a
 * CUDA graph.  Instance b gets the
 * outputs cs_omp gives for (plans[b], y_dev[b], K[b]):
 *   plans      host array [count] of plans on the current device (a plan may
 *              appear more than once); plans with 8192 < N <= 2^16 need the
 *              full storage of c (no CS_PLAN_C_* flag)
 *   y_dev      host array [count] of device pointers, F[M_b] each
 *   K          host array [count], 0 <= K[b] <= M_b, and K[b] <= 1024 for
 *              N <= 2^16, K[b] <= 4096 for larger N
 *   x_dev      NULL, or host array [count] of device pointers, FP64 [K[b]]
 *   supp_dev   host array [count] of device pointers, int32 [K[b]] (an
 *              entry may be NULL where K[b] = 0)
 *   iters_dev, resnorm_dev  device arrays [count], indexed by b (each NULL
 *              allowed)
 * halt as in cs_omp; with t_switch < 0 an instance takes its plan's switch
 * point (cs_plan_switch) for N <= 8192, 32 for 8192 < N <= 2^16 (their
 * kernel sums stream c through L2), and its plan's switch point again (tuned,
 * else the GB300 table) for N > 2^16.
 * Instances with N <= 8192 give bit for bit the results of cs_omp on their
 * plan.  Those with 8192 < N <= 2^16 run the one-CTA radix-16 chains on
 * vectors in global memory, two passes per round trip through a
 * shared-memory tile, where cs_omp runs four-step transforms over the GPU,
 * and agree with it to rounding.  Those with N > 2^16 run cs_omp's
 * large-plan path (a few whole-GPU launches per iteration), one instance at a
 * time on a library stream beside the persistent launches, bit for bit as
 * cs_omp on their plan.  The workspace is allocated stream-ordered on `stream` and freed
 * after the launches.  The call may wait for `stream` while it copies the
 * instance table.  A device-detected error goes to plans[0]'s status word
 * (cs_plan_status).  Errors: CS_ERR_INVALID for bad arguments,
 * CS_ERR_UNSUPPORTED beyond the limits (message in cs_last_error). */
cs_status cs_omp_batched(const cs_plan_t* plans, int64_t count, const void* const* y_dev,
                         const int32_t* K, const cs_halt* halt, void* const* x_dev,
                         int32_t* const* supp_dev, int32_t* iters_dev, double* resnorm_dev,
                         void* stream);

/* The autotuner of cs_omp_batched (the paper has no counterpart): measures,
 * on the caller's uneven batch (same arguments as cs_omp_batched, hybrid
 * path, outputs discarded), the launch shape of each launch group present,
 * a group being the instances of one element type (kind, precision) and one
 * residence (N <= 8192 in shared memory, 8192 < N <= 2^16 in global memory;
 * instances with N > 2^16 are not tuned).  Per group it times the group's
 * persistent launch alone (one warm-up, best of two) first with as many
 * resident CTAs per SM as fit and with every smaller number (fewer CTAs keep
 * fewer instance vectors in flight, which L2 may then hold), then at the
 * best of those with the switch point of every instance at 16, 64 or 128
 * (global memory; default 32) or 32 or 128 (shared memory; default the
 * plan's), keeping a candidate only when it is 2 % faster.  The groups'
 * launches share the GPU inside one cs_omp_batched call, so the per-group
 * winners are then kept only if the whole call on the batch is 2 % faster
 * with them (or with their switch points alone) than with the shapes stored
 * before.  What is kept is stored per device and group for the process and
 * used by later cs_omp_batched calls (CTAs per SM always; the switch point
 * when their t_switch < 0).  If cap > 0, up to cap records (group = 4 DFT + 2 FP64 + 1
 * global memory, CTAs per SM with 0 = all that fit, switch point with -1 =
 * default, best time in ms) go to the output arrays (each NULL allowed) and
 * their number to *n_out.  count = 0 forgets the shapes stored for the
 * current device (later calls take the defaults again).  Allocates its
 * temporary outputs on `stream` and blocks until done.  Errors as
 * cs_omp_batched. */
cs_status cs_omp_batched_tune(const cs_plan_t* plans, int64_t count, const void* const* y_dev, const int32_t* K,
                              double rel_tol, int32_t* group_out, int32_t* ctas_out, int32_t* tswitch_out,
                              float* ms_out, int32_t cap, int32_t* n_out, void* stream);

/* Subspace pursuit and CoSaMP on `batch` measurements sharing the plan's
 * Omega, one CTA per instance for N <= 8192.  The paper applies its correlation to these
 * algorithms (Sec. I) and reports the cost of a fast CoSaMP (Sec. IV) without
 * defining them; they take their standard forms:
 *   SP:     T = top_K(Phi^H y), x = LS on T; each iteration T' = T + top_K of
 *           |Phi^H r| over j not in T, b = LS on T', T_new = K largest |b|,
 *           x_new = LS on T_new;
 *   CoSaMP: x = 0; each iteration T = top_2K(|Phi^H r|) + supp(x), b = LS on
 *           T, x_new = b kept on its K largest |b|;
 * both stop, keeping the previous iterate, when the residual norm does not
 * decrease, and stop when ||r|| < rel_tol ||y|| or after max_iter iterations.
 * top_k breaks ties toward the lower index.  halt->path selects the
 * correlation: CS_PATH_FAST = kernel sums over the estimate's support
 * (Eq. kernelsum), CS_PATH_CONV = transforms, CS_PATH_HYBRID = kernel sums
 * when K <= t_switch.  Least squares are FP64 (normal equations with the
 * Gram entries read off c): a Cholesky factor built column by column for
 * column sets of at most 96, conjugate gradients above (one CTA per instance
 * for N <= 8192, a cluster of 4 to 16 CTAs for larger N; see below).
 * Outputs per instance: x_dev FP64 [K] and supp_dev [K] on
 * the final support in ascending column order (-1 / 0 past its size),
 * iters_dev (iterations run), resnorm_dev (||r|| / ||y||).
 * Large plans (N > 8192) run the same steps with the correlation over the
 * whole GPU and the top-k over N in two stages (per tile, then per instance);
 * when a least-squares set can exceed 96 columns (SP: K > 48, CoSaMP:
 * K > 32) they solve the normal equations by FP64 conjugate gradients, one
 * thread-block cluster of 4 to 16 CTAs per instance, Gram products read off
 * the FP64 kernel vector, from the previous coefficients, to a relative
 * residual of 1e-12 (FP64 plans; 1e-10 for FP32 plans, whose data carry
 * FP32 rounding) in at most 2m iterations for m columns (64 to 4000); a
 * column set whose columns are dependent is then solved only as far as
 * the iterations reach, instead of dropping the dependent column.
 * On large plans the iterations after the first run in a device-side loop
 * (a CUDA graph with a conditional while node, built per call, that ends as
 * soon as every instance is finished) when at least 64 of them remain
 * allowed (max_iter - 1 >= 64) and the stream is not being captured;
 * otherwise the call queues max_iter iterations, those after an instance's
 * end returning at once.
 * Limits: 1 <= K, 2K <= M (SP), 3K <= M (CoSaMP), K <= 128 for N <= 8192,
 * K <= 1024 for larger N. */
cs_status cs_sp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev, void* stream);
cs_status cs_cosamp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                    void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev, void* stream);

/* cs_omp without any allocation by the library: the paper has no
 * counterpart; this exists for callers that must not allocate device memory
 * while they solve (cudaMalloc/cudaFree synchronise the device and may block,
 * which a latency-bound request loop cannot take, and some processes give
 * the library no device memory beyond their own buffers).  Same arguments,
 * outputs and results as cs_omp.  Instead of the plan's growable workspace it
 * uses one fixed 32 MiB device array that the library holds on every device
 * that loads it until the process exits.
 *   - The first call on a device looks up that array's device address with
 *     cudaGetSymbolAddress (with the device current) and caches it; make that
 *     first call before any stream capture.
 *   - One CTA runs two instances at a time; its share of the array is
 *     2N working elements (sizeof F each) plus 2 K(K+1)/2 factor entries (16
 *     bytes each for DFT, 8 for WHT), each part rounded up to 16 bytes, plus
 *     16 bytes.  If one CTA's share exceeds 32 MiB the call returns
 *     CS_ERR_UNSUPPORTED with a message in cs_last_error; otherwise it runs
 *     as many resident CTAs as fit.
 *   - t_switch < 0 takes the plan's switch point (cs_plan_switch), as cs_omp
 *     does.
 *   - Every call on a device shares the array and leaves its contents behind;
 *     the call clears what must start at zero.  Calls that overlap on the GPU
 *     (other streams, other threads, other plans) race on it: serialise them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine. */
cs_status cs_omp_noalloc(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K,
                         const cs_halt* halt, void* x_dev, int32_t* supp_dev, int32_t* iters_dev,
                         double* resnorm_dev, void* stream);

/* Measure the hybrid switch point (Sec. IV's adaptive strategy, with the
 * crossover measured instead of taken from the flop model of Table I).
 * Runs cs_omp with CS_PATH_HYBRID on the caller's batch (y_dev, batch, K,
 * rel_tol) at a ladder of switch points: 1 (transforms from t = 2 on), the
 * flop-model point, 8, 12, 16, 24, 36, ... and K (kernel sums throughout);
 * each is timed with CUDA events on `stream` (in rounds over the whole ladder: one warm-up round, then the best of five).
 * The fastest becomes the plan's switch point for calls that pass
 * t_switch < 0, and is written to *t_best.  If cap > 0, the first
 * min(cap, n) ladder entries and their times in ms go to cand_out (int32) and
 * ms_out (float), and n to *n_out (NULL allowed).  Allocates its temporary
 * outputs on `stream`, overwrites the plan's workspace and blocks until done.
 * Limits: those of cs_omp with 1 <= K, batch >= 1. */
cs_status cs_plan_tune(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, double rel_tol,
                       int32_t* t_best, int32_t* cand_out, float* ms_out, int32_t cap, int32_t* n_out,
                       void* stream);

/* ---------------------------------------------------------------- serving
 * A request runtime for recovery jobs of mixed N, M, K, kind, precision and
 * algorithm (the paper has no counterpart: this is the serving side of the
 * same path).  `workers` threads each own a CUDA stream on the device that
 * is current at cs_server_create.  A submitted job waits in a queue until a
 * worker is free and its device footprint (its plan's tables, workspace,
 * input and outputs) fits in what the memory budget has left; the worker
 * then builds the job's plan on its stream, runs the solve, copies the
 * results to the caller's host buffers and releases the job's memory, all
 * stream-ordered, so jobs of different workers overlap on the GPU and no
 * admission or release synchronises the device.  Admission is oldest first,
 * except that a later job that fits may start while the oldest does not fit;
 * once the oldest has been passed 8 times, nothing else starts before it.
 * Results are the same as a single cs_omp / cs_cosamp / cs_sp call on the
 * job alone. */
typedef enum { CS_ALGO_OMP = 0, CS_ALGO_COSAMP = 1, CS_ALGO_SP = 2 } cs_algo;

typedef struct {
  int32_t kind, prec, algo, K;
  int64_t N, M;
  const int32_t* omega_host;  /* [M], sorted; copied by cs_server_submit */
  const void* y_host;         /* [M] in the plan's element type; copied by cs_server_submit */
  cs_halt halt;
} cs_request;

typedef struct {
  int64_t ticket;
  int32_t status;        /* cs_status of the job's solve */
  int32_t iters;         /* as cs_omp's iters_dev (cs_sp / cs_cosamp: iterations) */
  int32_t device_error;  /* cs_plan_status of the job's plan after the solve */
  int32_t pad;
  double resnorm;        /* as cs_omp's resnorm_dev */
  double t_submit_us, t_admit_us, t_done_us;  /* host clock, microseconds since cs_server_create */
  int64_t footprint_bytes;
} cs_result;

typedef struct cs_server_s* cs_server_t;

/* Start `workers` (1..64) worker threads with a device-memory budget of
 * hbm_budget_bytes for the jobs in flight.  Raises the release threshold of
 * the device's default stream-ordered memory pool to the budget (if lower) so
 * that freed job memory stays pooled for the process. */
cs_status cs_server_create(int32_t workers, int64_t hbm_budget_bytes, cs_server_t* out);

/* Queue one job; returns at once with its ticket.  The request is checked
 * as cs_plan_create and the solve call would check it (CS_ERR_INVALID /
 * CS_ERR_UNSUPPORTED, synchronously); a job whose footprint exceeds the
 * whole budget is refused with CS_ERR_NOMEM.  omega and y are copied; x_host
 * (FP64 [K], complex interleaved for DFT) and supp_host (int32 [K]) receive
 * the results and must stay valid until the job's result has been polled. */
cs_status cs_server_submit(cs_server_t server, const cs_request* req, void* x_host, int32_t* supp_host,
                           int64_t* ticket);

/* Move up to `max` finished jobs' results to out (oldest finished first),
 * waiting up to wait_ms for the first one if none is ready; *n = count. */
cs_status cs_server_poll(cs_server_t server, cs_result* out, int32_t max, int32_t wait_ms, int32_t* n);

/* Jobs waiting, running and finished so far, and the budget in use. */
cs_status cs_server_stats(cs_server_t server, int64_t* pending, int64_t* running, int64_t* completed,
                          int64_t* bytes_in_use);

/* Finish every queued job, stop the workers and free the server (results
 * not polled yet are dropped). */
cs_status cs_server_destroy(cs_server_t server);

/* The admission rule on its own (host only, no device): given the pending
 * jobs' footprints oldest first and how often each has been passed, the
 * budget in use and the budget, the index of the job to start now, or -1. */
int32_t cs_admit_next(const int64_t* footprints, const int32_t* bypassed, int32_t n_pending, int64_t in_use,
                      int64_t budget, int32_t max_bypass);

/* Measurement helper (the paper has no counterpart): queues on `stream` a
 * kernel of independent FP32 fused multiply-adds over the whole GPU, iters
 * steps of eight chains per thread, and writes its flop count to *flops
 * (host).  Timing it with events on `stream` gives the FP32 non-tensor peak
 * that the kernel-sum correlation's roofline fraction is stated against.
 * sink_dev may be NULL (nothing is written).  CS_ERR_INVALID for iters < 1 or
 * flops NULL. */
cs_status cs_fma_probe(int32_t iters, float* sink_dev, double* flops, void* stream);

/* Short static description of a status code. */
const char* cs_status_string(cs_status s);

/* Thread-local text of the last CUDA error seen by this thread ("" if none). */
const char* cs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CSFAST_H */
