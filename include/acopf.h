/*
 * acopf.h - C ABI of libacopf: GB300-native (sm_103a, FP64) evaluation of the
 * AC optimal power flow NLP callbacks and numeric assembly of the condensed
 * KKT matrix of a condensed-space interior-point method.
 *
 * Paper: S. Shin, F. Pacaud, M. Anitescu, "Accelerating Optimal Power Flow
 * with GPUs: SIMD Abstraction of Nonlinear Programs and Condensed-Space
 * Interior-Point Methods" (arXiv 2307.16830).
 *
 * Formulation (the paper lists the 15 computational patterns of the ACOPF
 * model in Sec. III.B but does not print the equations; the polar
 * branch-flow form below is the model its experiments use, Sec. V.A):
 *
 *   variables  x = [va (nb), vm (nb), pg (ng), qg (ng), p (2 nl), q (2 nl)]
 *              arc a < nl is the from end of branch a, arc nl + l the to end
 *              of branch l;
 *   constraints g = [ref (one per bus of type 3), pf, qf, pt, qt, ang, sf, st
 *              (one each per branch), Pbal, Qbal (one each per bus)] with
 *     ref  = va_i                         pf = p_l - P_f      qf = q_l - Q_f
 *     pt   = p_{nl+l} - P_t               qt = q_{nl+l} - Q_t
 *     ang  = va_f - va_t                  sf = p_l^2 + q_l^2  st = p_{nl+l}^2 + q_{nl+l}^2
 *     Pbal = Pd + Gs vm^2 - sum_{gens at i} pg + sum_{arcs at i} p_a
 *     Qbal = Qd - Bs vm^2 - sum_{gens at i} qg + sum_{arcs at i} q_a
 *   where (P_f, Q_f, P_t, Q_t) are the pi-model branch flows with series
 *   admittance 1/(r + jx), total charging b split half per end and a complex
 *   tap tau e^{j shift} on the from side (tau = 0 is read as 1);
 *   objective f = sum_g c2 pg^2 + c1 pg + c0.
 *
 * Sparse outputs, with the fixed orders that the *_structure calls return:
 *   Jacobian A = dg/dx in COO: ref rows; pf rows with entries [p_l, va_f,
 *     va_t, vm_f, vm_t]; qf [q_l, ...]; pt [p_{nl+l}, ...]; qt [q_{nl+l},
 *     ...]; ang [va_f, va_t]; sf [p_l, q_l]; st [p_{nl+l}, q_{nl+l}];
 *     balance vm terms (all Pbal rows, then all Qbal rows); generator terms
 *     (Pbal then Qbal, per generator); arc terms (Pbal then Qbal, per arc).
 *     Each branch pattern is stored entry-major: entry k of every branch,
 *     then entry k + 1 (slot = section + k * n_branch + l).
 *   Lagrangian Hessian W = sigma d2f + sum_r y_r d2g_r, lower triangle in COO
 *     with duplicates: the 10 entries of each branch's (va_f, va_t, vm_f,
 *     vm_t) block in the order (va_f,va_f) (va_t,va_f) (va_t,va_t)
 *     (vm_f,va_f) (vm_f,va_t) (vm_f,vm_f) (vm_t,va_f) (vm_t,va_t) (vm_t,vm_f)
 *     (vm_t,vm_t), each stored (max, min) of the global indices, entry-major;
 *     then the diagonals of p_l, q_l, p_{nl+l}, q_{nl+l}, entry-major; then
 *     (pg,pg) per generator; then (vm,vm) per bus.  The sign convention adds y_r g_r: the
 *     paper's L = f - y'g (Sec. II.A) is obtained by passing -y.
 *   Condensed KKT matrix M_cond = W + delta_w I + Sigma_x + A' D A with
 *     C = (delta_c Sigma_s + (1 + delta_c delta_w) I)^-1, D = (Sigma_s +
 *     delta_w I) C (Sec. IV.C), lower triangle in CSR: rows ascending,
 *     columns ascending within a row, every diagonal present, the pattern
 *     being the structural union of W, the diagonal and A'A.
 *
 * Conventions.  Indices are 0-based int32.  Host arrays passed to
 * acopf_model_create are copied; the caller keeps ownership of everything it
 * passes.  Every eval / assemble call takes DEVICE pointers to caller-owned
 * memory (for instance torch tensors) on the model's device, is asynchronous
 * on `stream` (NULL = the legacy default stream), never synchronises the
 * host and never allocates.  Outputs are fully overwritten.  Calls on one
 * model share the model's scratch (per-branch partial sums of the KKT
 * assembly): calls on the same model must not overlap on the GPU, so issue
 * them on one stream (or order them with events); different models are
 * independent.  To evaluate one model concurrently on several streams, give
 * each stream its own batch of that model (acopf_batch_create): every batch
 * instance has its own scratch.  No CPU fallback exists: without a usable
 * device every compute call returns ACOPF_E_CUDA or ACOPF_E_NO_DEVICE.
 * No call throws; errors are returned as acopf_status, with a message
 * readable through acopf_last_error() on the calling thread.
 */
#ifndef ACOPF_H_
#define ACOPF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* acopf_stream;

typedef int32_t acopf_status;
#define ACOPF_OK 0
#define ACOPF_E_INVALID_ARG (-1) /* null pointer, negative size, wrong model kind */
#define ACOPF_E_BAD_MODEL (-2)   /* network data rejected by validation */
#define ACOPF_E_CUDA (-3)        /* a CUDA runtime call or launch failed */
#define ACOPF_E_OOM (-4)         /* device or host allocation failed */
#define ACOPF_E_BUDGET (-5)      /* admission would exceed the memory budget */
#define ACOPF_E_TIMEOUT (-6)     /* a bounded wait ran out */
#define ACOPF_E_BUSY (-7)        /* resource in use (e.g. queue full) */
#define ACOPF_E_NO_DEVICE (-8)   /* model created host-only (device = -1) */

typedef struct acopf_model acopf_model;

/* Bus data, per unit.  type 3 marks a reference bus (one va = 0 row each). */
typedef struct {
  int32_t n;
  const int32_t* type;
  const double *Pd, *Qd, *Gs, *Bs, *Vmin, *Vmax;
} acopf_buses;

/* Branch data, per unit and radians.  f != t; r and x not both zero;
 * rate_a <= 0 means unrated (flow and thermal bounds infinite). */
typedef struct {
  int32_t n;
  const int32_t *f, *t;
  const double *r, *x, *b, *tap, *shift, *rate_a, *angmin, *angmax;
} acopf_branches;

/* Generator data; cost c2 pg^2 + c1 pg + c0. */
typedef struct {
  int32_t n;
  const int32_t* bus;
  const double *Pmin, *Pmax, *Qmin, *Qmax, *c2, *c1, *c0;
} acopf_gens;

/* Status name ("ACOPF_OK", ...).  Never NULL. */
const char* acopf_status_string(acopf_status s);

/* Message of the last failing call on this thread ("" if none). */
const char* acopf_last_error(void);

/* Build a model: validate the network, fix the variable and constraint
 * layout, the COO patterns of A and W and the CSR pattern of M_cond (the
 * host symbolic phase; parameterised per pattern and expanded over its data,
 * Sec. III.C), and upload the model to `device`.  device = -1 builds a
 * host-only model that answers the dims / bounds / structure queries but
 * returns ACOPF_E_NO_DEVICE from every compute call.  On success *out owns
 * the model; release it with acopf_model_destroy.  Errors:
 * ACOPF_E_INVALID_ARG, ACOPF_E_BAD_MODEL (the message names the first bad
 * entry), ACOPF_E_OOM, ACOPF_E_CUDA. */
acopf_status acopf_model_create(const acopf_buses* buses, const acopf_branches* branches,
                                const acopf_gens* gens, int device, acopf_model** out);

/* Free the model and its device memory.  NULL is accepted.  The caller must
 * make sure no call on the model is still running on the GPU. */
acopf_status acopf_model_destroy(acopf_model* model);

/* Sizes: n variables, m constraints, Jacobian / Hessian COO lengths, nnz of
 * the lower CSR of M_cond, and the device bytes the model holds (model data
 * plus its scratch).  Any output pointer may be NULL. */
acopf_status acopf_model_dims(const acopf_model* model, int64_t* n, int64_t* m, int64_t* nnz_jac,
                              int64_t* nnz_hess, int64_t* nnz_kkt, int64_t* device_bytes);

/* Counts of buses, branches, generators and reference buses (NULL allowed). */
acopf_status acopf_model_counts(const acopf_model* model, int32_t* n_bus, int32_t* n_branch,
                                int32_t* n_gen, int32_t* n_ref);

/* Host outputs: variable bounds xl, xu (length n), constraint bounds gl, gu
 * (length m); +-INFINITY where unbounded.  Any pointer may be NULL. */
acopf_status acopf_bounds(const acopf_model* model, double* xl, double* xu, double* gl, double* gu);

/* Host outputs: COO rows/cols of A (length nnz_jac), of the lower W
 * (length nnz_hess), and the lower CSR of M_cond (rowptr length n + 1,
 * colind length nnz_kkt). */
acopf_status acopf_jac_structure(const acopf_model* model, int32_t* rows, int32_t* cols);
acopf_status acopf_hess_structure(const acopf_model* model, int32_t* rows, int32_t* cols);
acopf_status acopf_kkt_structure(const acopf_model* model, int32_t* rowptr, int32_t* colind);

/* ---- device callbacks (Algorithm 1's f, grad f, g, grad g, Hessian of L) ----
 * x: device, length n.  y: device, length m.  Results are written to device
 * memory: f_dev one double; grad length n; cons length m; jvals nnz_jac;
 * hvals nnz_hess.  obj_weight is sigma in W = sigma d2f + sum_r y_r d2g_r. */
acopf_status acopf_eval_obj(const acopf_model* model, const double* x, double* f_dev,
                            acopf_stream stream);
acopf_status acopf_eval_grad(const acopf_model* model, const double* x, double* grad,
                             acopf_stream stream);
acopf_status acopf_eval_cons(const acopf_model* model, const double* x, double* cons,
                             acopf_stream stream);
acopf_status acopf_eval_jac_coo(const acopf_model* model, const double* x, double* jvals,
                                acopf_stream stream);
acopf_status acopf_eval_hess_coo(const acopf_model* model, const double* x, const double* y,
                                 double obj_weight, double* hvals, acopf_stream stream);

/* Numeric assembly of the lower CSR values of M_cond (Sec. IV.C) from given
 * Hessian and Jacobian values (device, in the COO orders above), Sigma_x
 * (device, length n, the diagonal of Z_lo (X - X_lo)^-1 + Z_hi (X_hi - X)^-1)
 * and Sigma_s (device, length m), with regularisation delta_w, delta_c >= 0
 * (Algorithm 1 uses 0, 0).  kvals: device, length nnz_kkt.  Uses the
 * model's scratch. */
acopf_status acopf_assemble_condensed_kkt_csr(const acopf_model* model, const double* hvals,
                                              const double* jvals, const double* sigma_x,
                                              const double* sigma_s, double delta_w,
                                              double delta_c, double* kvals, acopf_stream stream);

/* The fused unit of work of one IPM iteration: f, grad f, g, A, W and M_cond
 * at (x, y, Sigma_x, Sigma_s) in two kernel launches, the Jacobian and
 * Hessian values feeding the assembly straight from registers.  All
 * pointers device; every output must be non-NULL.  Results equal those of
 * the separate calls above up to floating-point rounding order. */
acopf_status acopf_eval_assemble(const acopf_model* model, const double* x, const double* y,
                                 double obj_weight, const double* sigma_x, const double* sigma_s,
                                 double delta_w, double delta_c, double* f_dev, double* grad,
                                 double* cons, double* jvals, double* hvals, double* kvals,
                                 acopf_stream stream);

/* Same unit of work with HOST buffers (pinned memory makes the copies
 * asynchronous DMA; pageable memory also works).  Copies x, y, Sigma_x,
 * Sigma_s to the model's device staging buffers, runs acopf_eval_assemble,
 * copies every output back and synchronises `stream` before returning.
 * Host outputs: f (1), grad (n), cons (m), jvals, hvals, kvals.  The
 * staging buffers are allocated on the first call and kept by the model. */
acopf_status acopf_eval_assemble_host(acopf_model* model, const double* x, const double* y,
                                      double obj_weight, const double* sigma_x,
                                      const double* sigma_s, double delta_w, double delta_c,
                                      double* f, double* grad, double* cons, double* jvals,
                                      double* hvals, double* kvals, acopf_stream stream);

/* ------------------------------------------------------------------------
 * Condensation around M_cond and step recovery (Sec. IV.C).
 *
 * The Newton system of the barrier problem (Sec. IV.B-C: unknowns dx, ds,
 * dy and the bound-dual steps dzl_x, dzu_x, dzl_s, dzu_s; right-hand sides
 * p_x, p_s, p_y, p_zl_x, p_zu_x, p_zl_s, p_zu_s) reduces to M_cond dx = rhs.
 * acopf_condense computes, at an interior iterate (x strictly inside
 * [xl, xu], slacks s strictly inside [sl, su]):
 *   Sigma_x = Zl_x (X - Xl)^-1 + Zu_x (Xu - X)^-1            (n)
 *   Sigma_s = Zl_s (S - Sl)^-1 + Zu_s (Su - S)^-1            (m)
 *   q_s     = p_s + (S - Sl)^-1 p_zl_s - (Su - S)^-1 p_zu_s  (m)
 *   rhs     = q_x + A' (C q_s + D q_y),  q_x = p_x + (X - Xl)^-1 p_zl_x - (Xu - X)^-1 p_zu_x,
 *             q_y = p_y, C = (delta_c Sigma_s + (1 + delta_c delta_w) I)^-1,
 *             D = (Sigma_s + delta_w I) C                    (n)
 * Sigma_x and Sigma_s are the diagonals acopf_eval_assemble takes.
 * acopf_recover_step computes, from a solution dx of M_cond dx = rhs,
 *   ds = C (A dx + delta_c q_s - q_y),  dy = (Sigma_s + delta_w I) ds - q_s,
 *   dzl_x = (X - Xl)^-1 (p_zl_x - Zl_x dx),  dzu_x = (Xu - X)^-1 (p_zu_x + Zu_x dx),
 *   dzl_s = (S - Sl)^-1 (p_zl_s - Zl_s ds),  dzu_s = (Su - S)^-1 (p_zu_s + Zu_s ds).
 * (Sec. IV.C prints ds = C (delta_c q_s - (q_y + A dx)); the sign of A dx
 * here is the one that solves the printed augmented system.)  A bound at
 * +-inf has no dual and no barrier term: its inverse gap is taken as zero
 * (pass zero duals and right-hand sides there).  A is the Jacobian at the
 * iterate, values in acopf_jac_structure's order.  All arrays are DEVICE
 * memory owned by the caller; calls are asynchronous on `stream` and
 * deterministic (fixed summation order).  The first call on a model
 * allocates the Jacobian's row and column lists and a row scratch (about
 * 16 bytes per Jacobian entry) and synchronises; make it before any stream
 * capture.  The row scratch is the model's, so these calls on one model must
 * not overlap on the GPU.  acopf_condense is two kernel launches,
 * acopf_recover_step one. */
typedef struct {
  const double *x, *s;           /* n, m */
  const double *xl, *xu;         /* n: variable bounds (+-inf allowed) */
  const double *sl, *su;         /* m: slack bounds (+-inf allowed) */
  const double *zl_x, *zu_x;     /* n: bound duals */
  const double *zl_s, *zu_s;     /* m */
  const double *p_x, *p_s, *p_y; /* n, m, m: right-hand sides */
  const double *p_zl_x, *p_zu_x; /* n */
  const double *p_zl_s, *p_zu_s; /* m */
} acopf_iterate;

acopf_status acopf_condense(acopf_model* model, const acopf_iterate* it, const double* jvals,
                            double delta_w, double delta_c, double* sigma_x, double* sigma_s,
                            double* q_s, double* rhs, acopf_stream stream);
acopf_status acopf_recover_step(acopf_model* model, const acopf_iterate* it, const double* jvals,
                                double delta_w, double delta_c, const double* sigma_s,
                                const double* q_s, const double* dx, double* ds, double* dy,
                                double* dzl_x, double* dzu_x, double* dzl_s, double* dzu_s,
                                acopf_stream stream);

/* Scaled residual of the first-order conditions (the termination test of
 * Algorithm 1, Sec. IV: "a scaled version of the residual" of Eq. first,
 * with the scaling of the interior-point reference the paper cites, s_max =
 * 100):
 *   r_d = [grad f - A'y - zl_x + zu_x ; y - zl_s + zu_s],  r_p = g(x) - s,
 *   r_c = [Zl_x (x - xl) - mu ; Zu_x (xu - x) - mu ; Zl_s (s - sl) - mu ;
 *          Zu_s (su - s) - mu] over finite bounds (n_z of them),
 *   s_d = max(100, (||y||_1 + ||z||_1) / (m + n_z)) / 100,
 *   s_c = max(100, ||z||_1 / n_z) / 100,
 *   E   = max(||r_d||_inf / s_d, ||r_p||_inf, ||r_c||_inf / s_c).
 * it: x, s, the bounds and the bound duals (the p_* fields are not read);
 * y (m), grad (n: acopf_eval_grad at x), cons (m: acopf_eval_cons at x),
 * jvals (acopf_eval_jac_coo at x): DEVICE arrays.  out: DEVICE array of 9
 * doubles receiving [E, ||r_d||_inf, ||r_p||_inf, ||r_c||_inf, ||y||_1,
 * ||z||_1, n_z, s_d, s_c].  Two kernel launches, asynchronous on `stream`;
 * sums in a fixed order.  Shares the model's condensation scratch (see
 * above): calls on one model must not overlap. */
acopf_status acopf_kkt_residual(acopf_model* model, const acopf_iterate* it, const double* y,
                                const double* grad, const double* cons, const double* jvals,
                                double mu, double* out, acopf_stream stream);

/* Sparse Cholesky factorization of M_cond and solves with it (the consumer
 * of the assembled matrix).  Sec. IV.C: M_aug has the inertia (n + m, 0, m)
 * exactly when M_cond is positive definite, so a factorization that meets a
 * non-positive pivot is the inertia test that raises (delta_w, delta_c);
 * Sec. V factorizes with a fill-reducing order fixed once per pattern and
 * refactors numerically every iteration.
 *
 * Symbolic phase (host, once per chol object): a minimum-degree order P of
 * M_cond's pattern (exact degrees on the elimination graph), the
 * elimination tree in postorder, fundamental supernodes (at most 64
 * columns), the row structure of each supernode and its place in its
 * parent's.  The numeric factorization (multifrontal: each supernode adds
 * its children's update matrices, factors its panel and forms its own
 * update matrix) and the solves are this library's kernels: one launch per
 * level of the supernodal elimination tree (leaves first), one thread block
 * per supernode, fixed summation order (bit-reproducible).
 *
 * acopf_chol_create: the symbolic phase and the device copies of its
 * arrays plus the factor's storage (acopf_chol_info's device_bytes);
 * synchronises.  ACOPF_E_NO_DEVICE for a host-only model; ACOPF_E_INVALID_ARG
 * when the elimination graph outgrows 2^28 entries (a pattern whose fill
 * is beyond a sparse factorization).  The object refers to the model,
 * which must outlive it.
 * acopf_chol_factor: kvals is the DEVICE lower-CSR value array of M_cond
 * (acopf_eval_assemble's kvals, acopf_kkt_structure's order).  Factorizes
 * P M_cond P' = L L' on `stream`; a pivot (the diagonal entry before its
 * square root) that is not above pivot_tol, or is NaN, fails; the
 * factorization continues past it with the pivot replaced by 1.
 * *first_bad_pivot (HOST) receives -1 when every pivot passes (M_cond
 * positive definite), else the smallest failing column in the order P.
 * Synchronises `stream` to return the test.  pivot_tol finite and >= 0,
 * else ACOPF_E_INVALID_ARG.
 * acopf_chol_solve: x = M_cond^-1 b with the last factorization (DEVICE b,
 * x of n doubles; they may alias); asynchronous on `stream`, and may be
 * captured into the caller's CUDA graph (the factorization, which returns
 * its test to the host, may not); ACOPF_E_INVALID_ARG unless the last
 * factorization passed the test.
 * Calls on one object use its scratch: they must not overlap on the GPU. */
typedef struct acopf_chol acopf_chol;
acopf_status acopf_chol_create(acopf_model* model, acopf_chol** out);
acopf_status acopf_chol_destroy(acopf_chol* chol);
acopf_status acopf_chol_factor(acopf_chol* chol, const double* kvals, double pivot_tol,
                               int32_t* first_bad_pivot, acopf_stream stream);
acopf_status acopf_chol_solve(acopf_chol* chol, const double* b, double* x, acopf_stream stream);
/* Counts of the symbolic phase: nnz_full, the entries of M_cond's full
 * symmetric pattern; nnz_factor, the entries of L (diagonal included);
 * max_col, the entries of L's largest column; factor_flops, the flops of
 * one numeric factorization (per column with c off-diagonal entries: 1
 * square root, c divisions and c (c + 1) / 2 multiply-adds); n_supernodes;
 * n_levels, the depth of the supernodal tree; storage, the doubles of the
 * supernodal blocks; update_storage, the doubles of the children's update
 * matrices and vectors the multifrontal factorization and solves pass up
 * the tree; factor_tasks, the tasks of the factorization's warp-task and
 * block-task graphs;
 * factor_launches and solve_launches, the kernel launches of one
 * factorization and of one solve. */
typedef struct {
  int64_t n, nnz_full, nnz_factor, max_col;
  double factor_flops;
  int64_t n_supernodes, n_levels;
  int64_t storage, update_storage;
  int64_t factor_tasks, factor_launches, solve_launches;
} acopf_chol_stats;
/* stats and device_bytes (all device memory of the object) may be NULL. */
acopf_status acopf_chol_info(const acopf_chol* chol, acopf_chol_stats* stats,
                             int64_t* device_bytes);
/* The symbolic phase alone, on the host (host-only models included): its
 * counts and, when perm is not NULL, the order (HOST, n entries: row i of
 * P M_cond P' is row perm[i] of M_cond). */
acopf_status acopf_chol_analyze(acopf_model* model, acopf_chol_stats* stats, int32_t* perm);
/* The order of a chol object, as acopf_chol_analyze's perm. */
acopf_status acopf_chol_permutation(const acopf_chol* chol, int32_t* perm);
/* Task trace (a profiling aid; the paper has no counterpart).  enable != 0
 * allocates a device trace buffer (ACOPF_E_OOM when that fails) and every
 * later factorization and solve records, per task of its task graph, six
 * int64 words: the task's kind word and first argument (supernode or
 * group), the GPU clock (ns) when a block took it, when its dependencies
 * were met, when it finished, and the SM that ran it; enable == 0 frees the
 * buffer.  acopf_chol_get_trace copies the last run of graph `which` (0 the
 * factorization's block tasks; the solves' block tasks: 1 forward,
 * 2 backward; their warp tasks: 3 forward, 4 backward; 5 the
 * factorization's warp tasks) into `out` (HOST,
 * 6 * capacity int64; NULL when capacity is 0) and sets *n_tasks to the
 * graph's task count; tasks
 * beyond `capacity` are not copied.  Synchronises the device. */
acopf_status acopf_chol_set_trace(acopf_chol* chol, int32_t enable);
acopf_status acopf_chol_get_trace(acopf_chol* chol, int32_t which, int64_t* out, int64_t capacity,
                                  int64_t* n_tasks);

/* The condensed-space interior-point method (Algorithm 1) on a model's
 * AC-OPF problem, driven from the host over this library's kernels: the
 * equality rows relaxed to [-tol, tol] and every finite constraint bound
 * widened by tol max(1, |bound|) (Eq. relax, Sec. IV.A); per iteration the
 * scaled residual of Eq. first (acopf_kkt_residual, the convergence test:
 * below tol), the monotone barrier update, the Newton right-hand side,
 * condensation, assembly and factorization of M_cond with the inertia
 * correction on delta_w (delta_c = 0), solve and step recovery (the printed
 * Delta y is minus the Newton step of y), the fraction-to-boundary step
 * bounds and the filter line search of the interior-point reference the
 * paper cites (its default constants), with its second-order correction:
 * when the first trial point is rejected without reducing the constraint
 * violation, the factored system is solved again with the constraint
 * residual replaced by alpha c(x) + c(x_trial) (up to 4 times while the
 * violation keeps falling by 1 %), and an accepted corrected point moves
 * the whole iterate along the corrected direction.  A step
 * below the line search's minimum enters a feasibility restoration: Gauss-
 * Newton steps on 1/2 ||g(x) - clip(g(x))||^2 (slacks following g, clipped
 * onto their box pushed inside) plus a log barrier on x's bounds and a
 * proximal term, factored on M_cond's pattern; it returns to the iteration
 * at the first point the filter accepts with at most 0.9 times the
 * violation (1e-3 times when the iteration came back to the restoration
 * without getting below the violation of its last exit), or ends the solve
 * with ACOPF_IPM_INFEASIBLE when the violation
 * stops decreasing (a point of local infeasibility).  (The status
 * ACOPF_IPM_LINE_SEARCH_FAILED is no longer produced.)  Initial point: voltage angles 0,
 * magnitudes 1, the rest at the middle of its bounds (0 when unbounded),
 * pushed into the interior; slacks at g(x0) pushed into their bounds;
 * y = 0; bound multipliers 1.
 * options: tol > 0, max_iter >= 0, mu_init > 0 (else ACOPF_E_INVALID_ARG).
 * x_out: HOST array of n doubles receiving the final x, or NULL.
 * history: HOST array of (max_iter + 1) x ACOPF_IPM_HISTORY_FIELDS doubles
 * (row k: f, residual, mu at iteration k's start, the constraint violation
 * sum |g - s|, then the step alpha, alpha_z and delta_w taken, alpha = 0
 * for an iteration that ran the restoration; NaN where not reached), or
 * NULL.  All work runs on `stream`; the call returns when
 * the solve ends.  It allocates its own device memory and a sparse Cholesky
 * object, and uses the model's scratch: no other call on the model may
 * overlap it.  ACOPF_E_NO_DEVICE for a host-only model. */
#define ACOPF_IPM_CONVERGED 0
#define ACOPF_IPM_MAX_ITER 1
#define ACOPF_IPM_LINE_SEARCH_FAILED 2
#define ACOPF_IPM_INERTIA_FAILED 3
#define ACOPF_IPM_INFEASIBLE 4
#define ACOPF_IPM_HISTORY_FIELDS 7
typedef struct {
  double tol;
  int32_t max_iter;
  double mu_init;
} acopf_ipm_options;
typedef struct {
  int32_t status, iterations;     /* status: ACOPF_IPM_*; iterations taken */
  int32_t factorizations;         /* of M_cond, inertia retries included */
  int32_t trial_points;           /* of the line searches */
  double objective, residual, mu; /* at the final point */
  double seconds;                 /* host wall time of the solve */
  double setup_seconds;           /* of which before the first iteration (symbolic phase of
                                     the factorization, allocation, initial point) */
} acopf_ipm_result;
acopf_status acopf_ipm_solve(acopf_model* model, const acopf_ipm_options* options, double* x_out,
                             double* history, acopf_ipm_result* result, acopf_stream stream);
/* The same solve with a sparse Cholesky object the caller created for this
 * model (acopf_chol_create) and keeps: the symbolic phase of the
 * factorization, most of the setup, is then paid once per network instead
 * of once per solve (repeated solves on one network: new loads, new set
 * points).  The object's factor is overwritten; it must not be used by
 * another call during the solve.  ACOPF_E_INVALID_ARG for a NULL object or
 * one created for another model; otherwise as acopf_ipm_solve, whose
 * results it reproduces bit for bit. */
acopf_status acopf_ipm_solve_chol(acopf_model* model, acopf_chol* chol,
                                  const acopf_ipm_options* options, double* x_out,
                                  double* history, acopf_ipm_result* result,
                                  acopf_stream stream);

/* Pipelined host-buffer evaluation: consecutive acopf_eval_assemble calls of
 * one model with HOST inputs and outputs, whose host-to-device copies,
 * kernels and device-to-host copies overlap (three streams, `depth` device
 * staging slots of one call each: inputs and outputs).  The paper has no
 * counterpart; it is the host-side form of the same unit of work.
 * acopf_pipeline_submit queues one call and returns without waiting (host
 * buffers as in acopf_eval_assemble_host; page-locked memory makes the
 * copies asynchronous); the caller keeps every buffer it passed valid and
 * unchanged, and reads no output, until acopf_pipeline_wait returns, and
 * gives calls in flight together distinct output buffers.  Calls
 * run in submission order and use the model's scratch, so no other call on
 * the model may overlap them.  depth in [2, 8]; the slots take depth x (the
 * bytes of one call's inputs and outputs) of device memory.  Destroy waits
 * for the submitted calls. */
typedef struct acopf_pipeline acopf_pipeline;
acopf_status acopf_pipeline_create(acopf_model* model, int32_t depth, acopf_pipeline** out);
acopf_status acopf_pipeline_destroy(acopf_pipeline* pipeline);
acopf_status acopf_pipeline_submit(acopf_pipeline* pipeline, const double* x, const double* y,
                                   double obj_weight, const double* sigma_x,
                                   const double* sigma_s, double delta_w, double delta_c,
                                   double* f, double* grad, double* cons, double* jvals,
                                   double* hvals, double* kvals);
acopf_status acopf_pipeline_wait(acopf_pipeline* pipeline);

/* Launch options of a model (not numerics: results are identical either way).
 * ACOPF_OPT_PDL (default 1): launch the second phase of a call with
 * programmatic dependent launch, so its independent work overlaps the first
 * phase; 0 launches it after the first phase completes. */
#define ACOPF_OPT_PDL 1
acopf_status acopf_model_set_option(acopf_model* model, int32_t option, int64_t value);

/* Number of kernel launches one call of each kind issues (for launch
 * accounting): kind 0 = eval_assemble, 1 = assemble_condensed_kkt_csr,
 * 2 = eval_obj, 3 = eval_grad, 4 = eval_cons, 5 = eval_jac_coo,
 * 6 = eval_hess_coo.  Returns -1 for an unknown kind. */
int32_t acopf_launches_per_call(int32_t kind);

/* Per-phase timing of acopf_eval_assemble, a measurement aid with no
 * counterpart in the paper.  After acopf_profile_begin(model, capacity) with
 * capacity > 0, the next `capacity` calls of acopf_eval_assemble on this
 * model record CUDA events on their stream before phase 1, between the two
 * phases and after phase 2 (profiled calls launch phase 2 without
 * programmatic dependent launch, since an event sits between the phases).
 * acopf_profile_end waits for the recorded events, returns the number of
 * profiled calls and the summed phase-1, phase-2 and whole-call durations in
 * milliseconds (NULL outputs allowed), and stops profiling.  Allocates and
 * frees CUDA events. */
acopf_status acopf_profile_begin(acopf_model* model, int32_t capacity);
acopf_status acopf_profile_end(acopf_model* model, int32_t* calls, double* phase1_ms,
                               double* phase2_ms, double* total_ms);

/* Measured FP64 fused-multiply-add throughput of `device` in GFLOP/s (2
 * flops per FMA): the best of five runs (after one warm-up) of a kernel of 8
 * blocks per SM x 256 threads, each thread running eight independent chains
 * of 16,384 dependent FMAs.  A measurement aid for rooflines: the paper has
 * no counterpart.  Allocates and frees a small device buffer. */
acopf_status acopf_measure_fp64_gflops(int device, double* gflops);

/* The same probe for each FP64 operation: G instructions per second of
 * FMA, add and multiply (per thread, i.e. lane operations).  Kernels whose
 * FP64 work mixes the three are bound by sum_op count_op / rate_op.  NULL
 * outputs are skipped. */
acopf_status acopf_measure_fp64_rates(int device, double* dfma, double* dadd, double* dmul);

/* Objective f = sum_g c2_g pg_g^2 + c1_g pg_g + c0_g, for callers that must
 * not allocate device memory.  The paper has no counterpart: it is a
 * variant of this library's objective reduction for code that may not call
 * cudaMalloc at all, such as a component running inside a host application
 * whose own allocator owns the device memory, or a solver loop under a
 * fixed memory budget.  It needs no model: pg, c2, c1, c0 are device arrays
 * of n_gen doubles (for instance pg = x + 2 n_bus of a model's point) and
 * f_dev one device double, all owned by the caller.
 * The call allocates nothing.  Its scratch, one partial sum per block plus
 * an arrival counter (about 8 KB), is a static device array that every GPU
 * loading this library holds until the process exits; n_gen is limited to
 * 16777216 (2^24) and larger values return ACOPF_E_INVALID_ARG.  The first
 * call on a device resolves the array's device address (with that device
 * current; a lookup that fails returns ACOPF_E_CUDA and is tried again by the
 * next call), so make that first call before any stream capture.  All calls
 * on a device share the array and it keeps the last call's contents: the
 * call clears the counter in stream order before its kernel, and calls that
 * overlap on the GPU (different streams without ordering) race.  The sum is
 * reduced in a fixed order, so equal inputs give bit-identical results. */
acopf_status acopf_objective_noalloc(int64_t n_gen, const double* pg, const double* c2,
                                     const double* c1, const double* c0, double* f_dev,
                                     acopf_stream stream);

/* ------------------------------------------------------------------------
 * Batched evaluation: many instances in one pair of launches.
 *
 * The paper evaluates one network per kernel launch (Sec. III.C: one GPU
 * thread per pattern instance); it mentions batched solvers only as related
 * work (Sec. I).  Here the same per-branch, per-bus and per-generator threads
 * of several instances, of uneven sizes, run together: phase 1 (objective,
 * gradient, constraints, Jacobian, Hessian and the branch-local part of
 * M_cond) over a flattened list of work items (instance, pattern group,
 * block) and phase 2 (the bus rows of M_cond) over a second list, each one
 * kernel launch, optionally replayed as a CUDA graph.
 *
 * An instance is (model, inputs, outputs): the same model may appear
 * several times (each instance has its own scratch), for instance as load
 * scenarios of one network that differ only in Pd and Qd.  Every instance's
 * outputs are bit-identical to those of acopf_eval_assemble on its model
 * (with the instance's Pd and Qd) at the same inputs: the same device code
 * runs on the same data in the same order.
 * ------------------------------------------------------------------------ */
typedef struct acopf_batch acopf_batch;

/* Inputs and outputs of one instance: DEVICE pointers, with the meaning,
 * sizes and ownership of acopf_eval_assemble's arguments.  Pd and Qd
 * (n_bus doubles each, device) replace the model's loads for this instance;
 * NULL keeps the model's.  The caller owns all of it and keeps it valid
 * while evaluations that use it are in flight. */
typedef struct {
  const double* x;
  const double* y;
  const double* sigma_x;
  const double* sigma_s;
  double obj_weight;
  double delta_w;
  double delta_c;
  const double* Pd;
  const double* Qd;
  double* f;
  double* grad;
  double* cons;
  double* jvals;
  double* hvals;
  double* kvals;
} acopf_batch_io;

/* Schedule of a batch: how its work items are ordered and launched (never
 * the numerics).  Bits 0-1 item order: 0 instances in the given order, 1
 * instances by decreasing size (largest first, so the long blocks start
 * early and small instances fill the tail), 2 pattern-group major (every
 * instance's branch blocks, then bus blocks, then generator blocks).  Bit 2
 * (ACOPF_SCHED_PDL): phase 2 with programmatic dependent launch.  Bit 3
 * (ACOPF_SCHED_GRAPH): the pair of launches replayed as a CUDA graph.  Bit 4
 * (ACOPF_SCHED_PERSISTENT): a grid of resident blocks (occupancy x SM
 * count) that strides over the item list instead of one block per item.
 * Schedules 0 .. ACOPF_BATCH_SCHEDULES - 1 with order < 3 are valid. */
#define ACOPF_SCHED_ORDER_GIVEN 0
#define ACOPF_SCHED_ORDER_SIZE 1
#define ACOPF_SCHED_ORDER_GROUP 2
#define ACOPF_SCHED_PDL 4
#define ACOPF_SCHED_GRAPH 8
#define ACOPF_SCHED_PERSISTENT 16
#define ACOPF_BATCH_SCHEDULES 32

/* Creates a batch of `count` >= 1 instances; instance i evaluates models[i]
 * (device models on one device; repeats allowed; the models must outlive
 * the batch).  Allocates the instances' scratch and the device tables.
 * Default schedule: ACOPF_SCHED_ORDER_SIZE | ACOPF_SCHED_PDL. */
acopf_status acopf_batch_create(acopf_model* const* models, int32_t count, acopf_batch** out);
acopf_status acopf_batch_destroy(acopf_batch* batch);

/* Sets the inputs and outputs of all `count` instances (io: HOST array of
 * count records holding device pointers; must equal the batch's count).
 * Validates them (non-NULL pointers, finite obj_weight, finite delta_w,
 * delta_c >= 0) and copies the per-instance tables to the device in order
 * on `stream`, so later evaluations on `stream` (or a graph replay) use
 * them.  Nothing is evaluated. */
acopf_status acopf_batch_set_io(acopf_batch* batch, const acopf_batch_io* io, int32_t count,
                                acopf_stream stream);

/* One fused evaluation (acopf_eval_assemble's unit of work) of every
 * instance, asynchronously on `stream`: two kernel launches, or one graph
 * launch.  ACOPF_E_INVALID_ARG before the first acopf_batch_set_io.
 * Evaluations of one batch must not overlap on the GPU (shared scratch). */
acopf_status acopf_batch_eval_assemble(acopf_batch* batch, acopf_stream stream);

/* Selects a schedule (see above); ACOPF_E_INVALID_ARG if not valid. */
acopf_status acopf_batch_set_schedule(acopf_batch* batch, int32_t schedule);

/* Autotuner: times every valid schedule (two warm-up evaluations, then
 * `reps` >= 1 timed with CUDA events on `stream`), selects the fastest and
 * returns it in *best.  times_ms (NULL or ACOPF_BATCH_SCHEDULES floats)
 * receives each schedule's mean milliseconds per evaluation, -1 for invalid
 * schedules.  Needs acopf_batch_set_io first; synchronises `stream`. */
acopf_status acopf_batch_autotune(acopf_batch* batch, acopf_stream stream, int32_t reps,
                                  int32_t* best, float* times_ms);

/* Current schedule, work items of each phase and device bytes the batch
 * holds (scratch and tables; not the models).  NULL outputs allowed. */
acopf_status acopf_batch_info(const acopf_batch* batch, int32_t* schedule, int64_t* items_phase1,
                              int64_t* items_phase2, int64_t* device_bytes);

/* ------------------------------------------------------------------------
 * Serving: a request loop over resident models.  The paper has no
 * counterpart (it runs one solve at a time); this is the serving form of
 * the evaluate-and-assemble unit of work (Sec. IV.C) for many IPM solves
 * that share one GPU.
 *
 * A request names a resident model (created by the caller with
 * acopf_model_create and kept for as long as requests use it) and asks for
 * n_calls fused evaluations (IPM iterations) at given points.  A server
 * thread admits queued requests in arrival order while the device bytes of
 * the admitted requests (inputs, outputs and scratch, allocated from the
 * server's stream-ordered pool) stay within the budget, and runs them:
 * An admitted request's device region is allocated and its inputs are
 * uploaded on the server's copy stream, apart from the compute stream that
 * runs the calls, so a large upload overlaps the calls of the requests
 * already running.
 *   ACOPF_SERVE_CONTINUOUS: continuous batching.  Each step ("tick") is one
 *     batched evaluation (the acopf_batch kernels) of admitted requests
 *     whose inputs are on the device and that have calls left, one call
 *     each, chosen within a work budget (ACOPF_SERVE_OPT_TICK_WORK: the
 *     longest-admitted one, then least remaining work first); requests join
 *     at the first tick after their upload completes and leave when their
 *     last call is done, so requests that arrive while others run share
 *     launches with them (a tick of one request runs that request's plain
 *     acopf_eval_assemble launches).  A bounded number of ticks is in flight
 *     (ACOPF_SERVE_OPT_INFLIGHT).
 *   ACOPF_SERVE_FIFO: plain launches.  Each admitted request's calls are
 *     queued as single-instance launches (acopf_eval_assemble's kernels) in
 *     arrival order on the compute stream, each request's after its upload.
 * Results do not depend on the mode or on co-scheduled requests: each
 * request has its own scratch and runs the code its single-instance call
 * runs, so its outputs are bit-identical to those of acopf_eval_assemble.
 * ------------------------------------------------------------------------ */
typedef struct acopf_server acopf_server;

/* A request.  All arrays are HOST memory owned by the caller, which keeps
 * them valid and unchanged until the request is done; page-locked memory
 * keeps the copies asynchronous (pageable memory works but makes the
 * server thread wait for the copies).  Inputs: n_points >= 1 point sets,
 * set k at x + k n, y + k m, sigma_x + k n, sigma_s + k m; call c uses set
 * c mod n_points.  Pd, Qd (n_bus each, or both NULL) replace the model's
 * loads.  Outputs (each may be NULL): f_calls receives the objective of
 * every call (n_calls doubles), grad, cons, jvals, hvals, kvals those of
 * the last call. */
typedef struct {
  const acopf_model* model;
  int32_t n_calls;
  int32_t n_points;
  const double* x;
  const double* y;
  const double* sigma_x;
  const double* sigma_s;
  double obj_weight;
  double delta_w;
  double delta_c;
  const double* Pd;
  const double* Qd;
  double* f_calls;
  double* grad;
  double* cons;
  double* jvals;
  double* hvals;
  double* kvals;
} acopf_request;

#define ACOPF_SERVE_CONTINUOUS 0
#define ACOPF_SERVE_FIFO 1

/* Server counters (totals since creation, and current / peak levels). */
typedef struct {
  int64_t submitted;
  int64_t completed;
  int64_t ticks;        /* batched evaluations (continuous mode) */
  int64_t launches;     /* kernel launches issued */
  int64_t bytes_in_use; /* device bytes of admitted requests */
  int64_t peak_bytes;
  int32_t active;       /* admitted, not yet done */
  int32_t queued;       /* waiting for admission */
  int32_t peak_active;
} acopf_server_stats;

/* Starts a server on `device` with its own two streams (compute, copy),
 * memory pool and thread.
 * budget_bytes > 0 caps the device bytes of admitted requests; max_active
 * >= 1 caps the number of admitted requests.  Returns ACOPF_E_NO_DEVICE for
 * device < 0. */
acopf_status acopf_server_create(int device, int64_t budget_bytes, int32_t mode,
                                 int32_t max_active, acopf_server** out);

/* Stops the server: requests still queued complete with ACOPF_E_BUSY,
 * admitted ones run to the end; then frees everything. */
acopf_status acopf_server_destroy(acopf_server* server);

/* Queues a request and returns its ticket.  ACOPF_E_BUDGET when the
 * request alone needs more device bytes than the budget; ACOPF_E_INVALID_ARG
 * for a bad request (NULL inputs, model on another device or host-only,
 * n_calls or n_points < 1, invalid scalars). */
acopf_status acopf_server_submit(acopf_server* server, const acopf_request* req,
                                 uint64_t* ticket);

/* Non-blocking state of a ticket: *done = 1 when finished, with the
 * request's status in *result (NULL allowed). */
acopf_status acopf_server_poll(acopf_server* server, uint64_t ticket, int32_t* done,
                               acopf_status* result);

/* Waits at most timeout_s seconds for a ticket; ACOPF_E_TIMEOUT if it is not
 * done by then (the request keeps running). */
acopf_status acopf_server_wait(acopf_server* server, uint64_t ticket, double timeout_s,
                               acopf_status* result);

/* Times of a finished ticket in seconds from submission: admission and
 * completion (host steady clock; completion is when the server saw the
 * request's last copy finish). */
acopf_status acopf_server_request_times(acopf_server* server, uint64_t ticket, double* admitted_s,
                                        double* done_s);

/* Forgets a finished ticket (its record is kept until then). */
acopf_status acopf_server_release(acopf_server* server, uint64_t ticket);

acopf_status acopf_server_get_stats(acopf_server* server, acopf_server_stats* out);

/* Server options (scheduling only; results never change).
 * ACOPF_SERVE_OPT_INFLIGHT (default 16, range 1..16): continuous-mode ticks
 * queued on the GPU ahead of completion.  More hides the host's per-tick
 * work behind the GPU's; fewer lets a new request join sooner.
 * ACOPF_SERVE_OPT_TICK_WORK (default 60,000, >= 1): the work budget of one
 * continuous-mode tick, counted as buses + branches + generators of one
 * call per request (an 80,000-bus call is about 200,000).  A tick takes the
 * longest-admitted runnable request, then others in order of least
 * remaining work (calls left x work per call) while the sum stays within
 * the budget. */
#define ACOPF_SERVE_OPT_INFLIGHT 1
#define ACOPF_SERVE_OPT_TICK_WORK 2
acopf_status acopf_server_set_option(acopf_server* server, int32_t option, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* ACOPF_H_ */
