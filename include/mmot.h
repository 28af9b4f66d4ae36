/*
 * mmot.h -- C ABI of the GB300 library for multi-marginal optimal transport
 * with pairwise L1 cost (arXiv 2405.19246, "A numerical algorithm with linear
 * complexity for Multi-marginal Optimal Transport with L1 Cost").
 *
 * Problem (Sec. 2 for l = 3, Sec. 4.2 for general l):
 *   l discrete marginals; marginal k has N_k support points x_k (sorted,
 *   nondecreasing, any spacing) and weights mu_k >= 0 with sum mu_k = 1.
 *   Cost      c(y_1..y_l) = sum_{p<q} |y_p - y_q|.
 *   Kernel    K = exp(-c/eps).
 *   Plan      t = prod_k phi_k(i_k) K                     (Eq. k-marginal T value)
 *   Sinkhorn  phi_j <- mu_j / M_j, j = 1..l in order      (Sec. 4.2 update formulas)
 *   with the marginal product (tensor-vector product)
 *             M_j(i) = sum over the other marginals' points of
 *                      prod_{m != j} phi_m K               (Eq. Jk k margin)
 *   computed in O(sum_k N_k) work by the paper's separated summations
 *   (Sec. 3, Sec. 4.2) instead of the O(prod N_k) contraction.
 *
 * Potentials.  The library stores g_k = eps ln phi_k (FP64).  The paper's dual
 * variables are alpha_k = -g_k - eps/l (Sec. 2, definition of phi).  A zero
 * weight gives g = -inf.  Initial potentials are phi = 1/N_k (the
 * initialisation of Algorithm 1), i.e. g_k = -eps ln N_k.
 *
 * Conventions for every call:
 *   - Calls never throw and never abort; they return an mmot_status.  On an
 *     error mmot_last_error() gives a message (thread-local).
 *   - Pointers marked "host or device" may point to host memory or to device
 *     memory of the plan's GPU; the library detects which.
 *   - The plan copies every input into device memory it owns; caller buffers
 *     are never retained.  Output buffers are caller-owned.
 *   - Work is issued on the stream given to mmot_plan_create (borrowed, not
 *     owned; NULL = the legacy default stream).  Calls that return values to
 *     host memory synchronise that stream before returning.
 */
#ifndef MMOT_H
#define MMOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmot_plan_s *mmot_plan; /* opaque, owned by the library */

typedef enum {
    MMOT_OK = 0,
    MMOT_ERR_INVALID_ARG = 1,  /* bad size, eps, marginal index, weights      */
    MMOT_ERR_UNSORTED = 2,     /* a support x_k is not nondecreasing          */
    MMOT_ERR_OOM = 3,          /* device allocation failed                    */
    MMOT_ERR_CUDA = 4,         /* a CUDA runtime call failed                  */
    MMOT_ERR_TIMEOUT = 5,      /* a bounded inter-tile wait gave up           */
    MMOT_ERR_NOT_CONVERGED = 6,/* itr_max reached with residual > tol         */
    MMOT_ERR_NONFINITE = 7,    /* a product or potential became NaN or inf    */
    MMOT_ERR_RANGE = 8         /* input outside the supported range           */
} mmot_status;

typedef enum {
    MMOT_FP64 = 0,               /* all scan arithmetic in FP64                  */
    MMOT_FP32_SCAN_FP64_POT = 1  /* FP32 in-tile scans, FP64 log-domain carries,
                                    FP64 potentials, residual and objective     */
} mmot_precision;

typedef struct {
    int iters;        /* Sinkhorn iterations performed (one = l updates)        */
    double residual;  /* sum over marginals 1..l-1 of ||phi_k . M_k - mu_k||_1
                         after the last iteration (stopping test of Algorithm 1 / 4) */
    double W;         /* <C, T> of the regularised plan (Eq. k-mmot distance)    */
    double primal;    /* <C,T> + eps <T, ln T> = sum_k <g_k, marg_k>             */
    double dual;      /* sum_k <g_k, mu_k> + eps - eps Z                         */
    double mass;      /* Z = sum of all plan entries                             */
} mmot_result;

/* Create a plan (Sec. 4.2 problem statement; Algorithm 1 inputs).
 *   l      number of marginals, 2 <= l <= 8.
 *   N      host array of l sizes, N[k] >= 1, sum N[k] < 2^31.
 *   x      l pointers (host or device, see inputs_on_device) to N[k] FP64
 *          support points each, nondecreasing (else MMOT_ERR_UNSORTED).
 *   mu     l pointers to N[k] FP64 weights, >= 0, each summing to 1 within
 *          1e-12 (else MMOT_ERR_INVALID_ARG).  Zero weights are allowed.
 *   eps    entropic regularisation, > 0 and finite.
 *   prec   MMOT_FP64 or MMOT_FP32_SCAN_FP64_POT.
 *   inputs_on_device  0: x and mu are host pointers; 1: device pointers.
 *   cuda_stream       cudaStream_t to issue work on (borrowed).
 *   out    receives the plan; *out is NULL on failure.
 * Merges the supports into one order by (x, k, index) (the tie rule of the
 * order classes D_p, Eq. D_p), tiles it, and sets g_k = -eps ln N_k. */
mmot_status mmot_plan_create(int l, const int64_t *N, const double *const *x,
                             const double *const *mu, double eps, mmot_precision prec,
                             int inputs_on_device, void *cuda_stream, mmot_plan *out);

/* Marginal product of marginal k with the current potentials (Eq. Jk k margin,
 * computed as in Sec. 3.1 / Sec. 4.2):
 *   plan_marginal = 0: out[i] = M_k(i)
 *   plan_marginal = 1: out[i] = phi_k(i) M_k(i)   (the k-th marginal of the plan)
 *   plan_marginal = 2: out[i] = ln M_k(i)
 * out: N[k] FP64 values, host or device.  Potentials are not changed. */
mmot_status mmot_marginal(mmot_plan p, int k, int plan_marginal, double *out);

/* Run n_iters Gauss-Seidel Sinkhorn iterations (Sec. 4.2 update formulas;
 * Algorithm 4 loop body): for j = 1..l, g_j <- eps (ln mu_j - ln M_j).
 * If residual_out is not NULL it receives the residual of Algorithm 1's stopping test
 * (sum over marginals 1..l-1 of ||phi_k . M_k - mu_k||_1) after the last
 * iteration, which costs l-1 extra marginal products. */
mmot_status mmot_sinkhorn_step(mmot_plan p, int n_iters, double *residual_out);

/* Solve: iterate while t < itr_max and residual > tol (Algorithm 1 loop), the
 * residual being evaluated every `check_every` iterations (mmot_set_option),
 * then evaluate the objective terms (Eq. k-mmot distance).  tol <= 0 runs
 * exactly itr_max iterations.  Returns MMOT_ERR_NOT_CONVERGED (with out
 * filled) when itr_max is reached with residual > tol > 0. */
mmot_status mmot_solve(mmot_plan p, double tol, int itr_max, mmot_result *out);

/* Objective terms for the current potentials (residual over all l marginals,
 * W, primal, dual, mass); iters is left 0. */
mmot_status mmot_objective(mmot_plan p, mmot_result *out);

/* Copy potentials g_k = eps ln phi_k (N[k] FP64, host or device) out of or
 * into the plan: warm start and checkpoint/resume. */
mmot_status mmot_get_potentials(mmot_plan p, int k, double *g_out);
mmot_status mmot_set_potentials(mmot_plan p, int k, const double *g_in);

/* Reset every potential to the starting point phi_k = 1/N_k (the
 * initialisation of Algorithm 1), i.e. g_k = -eps ln N_k, on the device (no
 * host transfer). */
mmot_status mmot_reset_potentials(mmot_plan p);

/* Plan options (integers):
 *   MMOT_OPT_CHECK_EVERY   residual evaluation period in mmot_solve (default 10)
 *   MMOT_OPT_SPIN_LIMIT    inter-tile wait limit in polls (default ~1 s)
 *   MMOT_OPT_USE_GRAPH     capture the per-iteration launches in a CUDA graph (default 1)
 *   MMOT_OPT_PROFILE       1: bracket every kernel launch with CUDA events on the
 *                          plan's stream and accumulate per-kernel times (graphs
 *                          are not used while profiling); 0: off (default)
 *   MMOT_OPT_TEST_HOLD     test hook for the timeout path, 0 (default) or 1: the
 *                          first chunk of each carry scan never publishes its
 *                          flags, so the bounded waits of the later chunks run
 *                          out and calls return MMOT_ERR_TIMEOUT (results are
 *                          then undefined).  Needs more tiles than one chunk. */
enum { MMOT_OPT_CHECK_EVERY = 1, MMOT_OPT_SPIN_LIMIT = 2, MMOT_OPT_USE_GRAPH = 3, MMOT_OPT_PROFILE = 4,
       MMOT_OPT_TEST_HOLD = 5 };
mmot_status mmot_set_option(mmot_plan p, int option, int64_t value);

/* Per-kernel launch statistics collected while MMOT_OPT_PROFILE is on.
 *   kernel 0: backward look-back scan (k_bwd), 1: forward look-back scan +
 *   combine (k_fwd), 2: tile transfer operators (k_tops), 3: carry scan over
 *   tiles (k_carry), 4: tile products with known carries + combine (k_tile),
 *   5: per-level tile contributions (k_wpass), 6: per-level carry scan
 *   (k_lscan), 7: backward walk of the warp-tile products (k_wbwd).
 *   Marginal products use kernels 2-4 for l <= 5 and 4-7 for l >= 6;
 *   kernels 0-1 serve the objective sweeps of l >= 5.
 * Returns the number of launches and their summed device time in ms (CUDA
 * events on the plan's stream); synchronises the stream.  reset != 0 clears
 * the statistics after reading. */
mmot_status mmot_get_profile(mmot_plan p, int kernel, int64_t *launches, double *total_ms, int reset);

/* Plan information: number of tiles, points per tile, total points, kernel
 * launches per Sinkhorn iteration. */
typedef struct {
    int64_t total_points;
    int64_t tiles;
    int tile_points;
    int threads_per_block;
    int launches_per_iteration;
    int precision;
    int64_t kernel_launches;   /* library kernels launched on this plan so far */
    int64_t device_bytes;      /* device memory held by the plan */
    int uniform_grid;          /* 1: every marginal on one uniform grid, l <= 5 (Sec. 3's
                                  setting): the tile kernels form each point's position factor
                                  and marginal from its merged index instead of reading them */
} mmot_plan_info;
mmot_status mmot_get_info(mmot_plan p, mmot_plan_info *info);

/* Process-wide cap on the device memory that all plans (and the plans inside
 * batches) may hold together, in bytes; 0 (the default) means no cap.  It
 * lets a caller that shares the GPU with other work, such as a serving loop
 * admitting requests by a memory budget, bound the library's footprint: a
 * creation that would exceed the cap fails with MMOT_ERR_OOM before the
 * allocation that would cross it, and frees what it had taken.  Memory held
 * by existing plans is not affected.  bytes < 0: MMOT_ERR_INVALID_ARG. */
mmot_status mmot_set_memory_limit(int64_t bytes);

/* Device memory the library holds right now for all live plans and batches
 * (the quantity the cap above bounds), in bytes.  bytes == NULL:
 * MMOT_ERR_INVALID_ARG. */
mmot_status mmot_memory_in_use(int64_t *bytes);

/* ---- Shards of one instance -------------------------------------------------
 * One instance split into P shards: contiguous ranges of the merged order of
 * all support points (sorted by x, then marginal, then index), each held by
 * its own plan (one GPU each in a multi-GPU run; several plans on one GPU to
 * validate).  Every point of every marginal inside a range stays with its
 * shard, so the potentials never move; what crosses a cut is the vector of
 * the 2^(l-1) forward (or backward) subset states of Sec. 4.2 at the cut.
 * Those states are linear in the states entering a range, so each shard
 * reduces its range to a transfer operator (mmot_shard_operator); the
 * operators of all shards (at most 2 l 2^(l-1) numbers each) are exchanged,
 * composed in shard order with the decay exp(-w_s gap/eps) across each gap
 * between neighbouring shards (w_s = s(l - s)), and give every shard its
 * entering states (mmot_shard_set_inflow) before its products.  A Sinkhorn
 * update of marginal k (Gauss-Seidel, Algorithm 1) then runs shard-locally
 * (mmot_shard_update), and the stopping residual is the sum of the shards'
 * terms (mmot_shard_residual).  l <= 5 (tile operators).
 *
 * States are indexed by bit masks T over the marginals other than the
 * target k, bit b standing for marginal b if b < k and b + 1 otherwise; T = 0
 * is the empty state (always 1).
 *
 * mmot_shard_create: as mmot_plan_create for the shard's points (N[k] >= 1
 * points of every marginal, the shard's weights mu need not sum to 1), with
 * N_total the sizes of the whole instance (the initial potentials are
 * g_k = -eps ln N_total[k]).  l > 5: MMOT_ERR_RANGE.  mmot_sinkhorn_step,
 * mmot_solve and mmot_objective reject shard plans (MMOT_ERR_INVALID_ARG);
 * mmot_marginal works and uses the inflow when it was set for its target.
 *
 * mmot_shard_operator: for target k and the current potentials, writes
 * lnop[2][l][2^(l-1)] (host or device memory, natural logarithms, -inf for
 * 0).  lnop[0][s][U], U != 0: the factor with which a forward state S of
 * level |S| = s at the shard's left end x_L (before its first point) reaches
 * S + U at its right end x_R (after its last point) through the shard's
 * points of the marginals in U; it depends on s and U only (Sec. 4.2: the
 * rates of the levels passed and the injections).  lnop[0][s][0] = -w_s
 * (x_R - x_L)/eps, the decay of a state that picks up nothing.  lnop[1] is
 * the same for the backward states, from x_R to x_L.  Entries with
 * s + |U| > l - 1 are -inf.
 *
 * mmot_shard_set_inflow: the states entering the shard for target k, as
 * natural logarithms: lnF[T] the forward states at x_L, lnG[T] the backward
 * states at x_R, 2^(l-1) host values each (entry 0 ignored; NULL: nothing
 * enters from that side, the first or last shard).  NaN or +inf:
 * MMOT_ERR_INVALID_ARG.  Kept until the next call; products for other
 * targets see no inflow.
 *
 * mmot_shard_update: the potential update of marginal k on the shard's
 * points (Eq. of the update in Algorithm 1) with the inflow set for k
 * (else MMOT_ERR_INVALID_ARG).
 *
 * mmot_shard_residual: sum over the shard's points of marginal k of
 * |phi_k M_k - mu_k| with the inflow set for k, into *res (host). */
mmot_status mmot_shard_create(int l, const int64_t *N, const double *const *x, const double *const *mu,
                              const int64_t *N_total, double eps, mmot_precision prec, int inputs_on_device,
                              void *cuda_stream, mmot_plan *out);
mmot_status mmot_shard_operator(mmot_plan p, int k, double *lnop);
mmot_status mmot_shard_set_inflow(mmot_plan p, int k, const double *lnF, const double *lnG);
mmot_status mmot_shard_update(mmot_plan p, int k);
mmot_status mmot_shard_residual(mmot_plan p, int k, double *res);

/* ---- Two-dimensional product (Sec. 4.1, Algorithm 6, FTVP_2d) -------------
 * Three marginals on one uniform N x M grid with steps h1 (first index) and
 * h2 (second), L1 cost, kernel K = lambda1^{|i1-j1|+|i1-k1|+|j1-k1|}
 * lambda2^{|i2-j2|+|i2-k2|+|j2-k2|}, lambda_d = e^{-h_d/eps}:
 *     out(k1, k2) = sum_{i1,i2,j1,j2} K phi(i1, i2) psi(j1, j2),
 * the product that the two-dimensional Sinkhorn iteration needs for each
 * marginal (K is symmetric in the three marginals, so the product for the
 * first marginal is mmot_ftvp2d(psi, varphi) and so on).  O(N M) work: the
 * second index by the one-dimensional recurrences with vector states, each
 * step a one-dimensional product along the first index (6 M of them, in
 * parallel), all terms positive.
 * phi, psi, out: N * M doubles, column-major (element (i1, i2) at i1 + N i2),
 * host or device; FP64 in the linear domain, so inputs should be scaled to
 * moderate values.  1 <= N, M, N M <= 2^28, 0 <= lambda_d < 1, else
 * MMOT_ERR_INVALID_ARG.  Allocates device scratch (31 N M doubles) for the
 * call; work on cuda_stream (NULL: the legacy default stream), synchronised
 * before returning. */
mmot_status mmot_ftvp2d(int64_t N, int64_t M, const double *phi, const double *psi, double lambda1,
                        double lambda2, double *out, void *cuda_stream);

/* One marginal product without any device memory allocation.
 *
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: code running under a memory manager that owns the
 * whole device budget (a framework's caching pool), plug-ins that must not
 * change the process's allocation state, or latency-critical loops where the
 * implicit synchronisation of cudaMalloc is not acceptable.  It computes what
 * mmot_marginal computes on a plan (FP32 in-tile scans), for the potentials g
 * passed in, without creating a plan and without calling cudaMalloc, cudaFree
 * or any allocating library routine.
 *
 *   l, N, x, eps  as in mmot_plan_create (x host or device, sorted);
 *   g             l pointers to the potentials g_k = eps ln phi_k (host or
 *                 device; device when plan_marginal = 1);
 *   k, plan_marginal  as in mmot_marginal (0: M_k, 1: phi_k M_k, 2: ln M_k);
 *   out           N[k] FP64 values, device memory (caller-owned);
 *   cuda_stream   stream to use (borrowed).  The inputs are read in the
 *                 order of that stream (after work the caller queued on it),
 *                 and the call is synchronous: it synchronises the stream
 *                 before returning.  Do not issue it on a stream that is
 *                 being captured into a CUDA graph.
 * Limits: 2 <= l <= 5, sum N <= 2^19 points, at most 1024 tiles; larger
 * problems return MMOT_ERR_RANGE with a message.  Working storage is one
 * static 8 MiB device array per GPU, held by every GPU that loads the library
 * until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress).  All calls share the array: calls
 * that overlap on the same GPU (from several host threads or streams) race,
 * so callers must serialise them. */
mmot_status mmot_marginal_noalloc(int l, const int64_t *N, const double *const *x,
                                  const double *const *g, double eps, int k, int plan_marginal,
                                  double *out, void *cuda_stream);

/* Destroy a plan; NULL-safe. */
void mmot_destroy(mmot_plan p);

/* ---- Batches of independent instances -------------------------------------
 * The paper solves one instance at a time (Algorithm 1); a batch solves many
 * independent instances together.  Instances with the same l are laid out one
 * after another in one merged order whose tiles never straddle two instances
 * and across whose boundaries no state is carried, so every kernel launch of
 * a Sinkhorn iteration serves all instances of that l at once; each l forms a
 * group with its own launch sequence (split into consecutive parts above
 * 65536 tiles for l <= 5), all on the batch's stream.  Each
 * instance stops on its own: after every check its residual (marginals
 * 1..l-1, as in mmot_sinkhorn_step) is compared with tol and a converged
 * instance is frozen (no further updates; its potentials stay as they were
 * at the check that found it converged). */
typedef struct mmot_batch_s *mmot_batch;   /* opaque, owned by the library */

/* Create a batch of n >= 1 instances.
 *   l[i]         marginals of instance i (2..8).
 *   N, x, mu     the instances' arguments of mmot_plan_create concatenated:
 *                instance i owns entries o_i .. o_i + l[i] - 1 with
 *                o_i = l[0] + ... + l[i-1]; x and mu are host pointers.
 *   eps[i]       regularisation of instance i.
 *   prec         as in mmot_plan_create, for all instances.
 *   tile_points  upper bound on points per tile (0: the kernel's maximum);
 *                smaller tiles trade per-tile work for more parallelism and
 *                are chosen by an autotuner.
 *   cuda_stream  stream to use (borrowed), NULL: the batch creates one.
 * Potentials start at g = -eps ln N_k per instance. */
mmot_status mmot_batch_create(int n, const int *l, const int64_t *N, const double *const *x,
                              const double *const *mu, const double *eps, mmot_precision prec,
                              int tile_points, void *cuda_stream, mmot_batch *out);

/* Run n_iters Sinkhorn iterations on every instance not yet converged, then
 * check each of them (residual <= tol freezes it).  *active_out (may be
 * NULL) receives the number of instances still running. */
mmot_status mmot_batch_step(mmot_batch b, int n_iters, double tol, int *active_out);

/* Reset every instance to its initial potentials and unfreeze it. */
mmot_status mmot_batch_reset(mmot_batch b);

/* Solve every instance: reset, then steps of check_every iterations until
 * all are converged or itr_max iterations have run.  results (n entries,
 * may be NULL) receive per instance: iterations until convergence (or
 * itr_max), its last checked residual, and W, primal, dual, mass as in
 * mmot_objective.  Returns MMOT_ERR_NOT_CONVERGED (results filled) when some
 * instance did not converge. */
mmot_status mmot_batch_solve(mmot_batch b, double tol, int itr_max, int check_every, mmot_result *results);

/* Freeze instance i (no further updates), e.g. when a caller's iteration
 * budget for it is spent; its status keeps converged = 0. */
mmot_status mmot_batch_freeze(mmot_batch b, int i);

/* Iterations run, last checked residual and converged flag of instance i. */
mmot_status mmot_batch_status(mmot_batch b, int i, int *iters, double *residual, int *converged);

/* Potentials g_k of instance i (N_k FP64, host or device). */
mmot_status mmot_batch_get_potentials(mmot_batch b, int i, int k, double *g_out);

/* Replace the potentials g_k of instance i (N_k FP64, host or device; the
 * call is synchronous and orders a device input after all work queued on
 * the device).  A warm start: the Sinkhorn state of an instance is its l
 * potentials (Algorithm 1 updates one g_k at a time from the others), so
 * setting all l of them from another run continues that run at an iteration
 * boundary.  A frozen or converged instance becomes active again (status:
 * converged = 0, residual NaN until the next check).  Errors:
 * MMOT_ERR_INVALID_ARG for a NULL pointer, an index out of range or a NaN /
 * +inf value (the batch is unchanged); MMOT_ERR_CUDA for a failed copy. */
mmot_status mmot_batch_set_potentials(mmot_batch b, int i, int k, const double *g_in);

typedef struct {
    int instances;
    int groups;                /* launch groups: one per l, split into parts when
                                  one carry scan cannot take all its tiles     */
    int64_t total_points;
    int64_t tiles;
    int64_t kernel_launches;   /* library kernels launched on this batch so far */
} mmot_batch_info;
mmot_status mmot_batch_get_info(mmot_batch b, mmot_batch_info *info);

/* Destroy a batch; NULL-safe. */
void mmot_batch_destroy(mmot_batch b);

/* Message of the last error on this thread ("" if none). */
const char *mmot_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MMOT_H */
