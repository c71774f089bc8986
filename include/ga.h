/*
 * ga.h - C ABI of the GB300 library for GA-NGMRES-accelerated, regularisation-preconditioned
 * first-order optimisation of transport-constrained problems (He & Mang, arXiv 2510.08782).
 *
 * The library solves   minimise_v  obj(v) = 1/2 ||m(., 1) - m_1||^2 + alpha/2 <v, L v>
 * subject to a transport equation for m driven by a stationary velocity v on the periodic box
 * [0, 2 pi)^d (problem (1) of Sec. 1.1; the mass-preserving variant is problem (11) of Sec. 3.7;
 * the incompressible variant adds div v = 0, Sec. 3.6).
 *
 * Conventions shared by every call
 *   Layout     A scalar field is an array of prod(n) elements in C order (n[dim-1] is the
 *              contiguous axis). A vector field (v, g, s) holds `dim` such arrays back to back
 *              (component c first); component c points along axis c. Grid point l sits at
 *              x_l = 2 pi l / n (Sec. 2.2).
 *   Element    GA_PREC_FP64: double everywhere. GA_PREC_MIXED: fields (m0, m1, v, g, s) are
 *              float; the objective, inner products, Gram matrix and least squares are FP64.
 *   Memory     `mem` says where caller pointers live: GA_MEM_HOST (pageable or pinned host
 *              memory; the call copies in/out and synchronises) or GA_MEM_DEVICE (device memory
 *              of the context's GPU; the call is ordered on the context stream and returns after
 *              the result is complete on that stream).
 *   Ownership  ga_setup copies m0/m1 into context-owned device memory. Caller buffers are
 *              borrowed for the duration of a call only. ga_destroy frees everything.
 *   Errors     Every call returns ga_status and never aborts. After any status other than
 *              GA_OK and GA_ERR_NOT_CONVERGED, ga_last_error() holds a one-line reason. The context
 *              stays usable except after GA_ERR_CUDA. Null pointers, out-of-range sizes and
 *              options return GA_ERR_ARG. A NaN or Inf objective or gradient returns GA_ERR_NAN.
 *   Threads    A context is not thread-safe; distinct contexts are independent.
 */
#ifndef GA_H
#define GA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GA_OK = 0,
  GA_ERR_ARG = 1,            /* invalid argument, descriptor or option                   */
  GA_ERR_CUDA = 2,           /* a CUDA runtime error; the context must be destroyed      */
  GA_ERR_NOMEM = 3,          /* device allocation failed                                 */
  GA_ERR_NAN = 4,            /* NaN/Inf in the objective or the gradient                 */
  GA_ERR_LINESEARCH = 5,     /* Armijo search exhausted max_backtracks halvings          */
  GA_ERR_NOT_CONVERGED = 6,  /* informational: ga_solve hit max_iter; v and stats valid  */
  GA_ERR_TIMEOUT = 7         /* reserved: no call waits on the device, none returns it   */
} ga_status;

typedef enum {
  GA_MODEL_ADVECTION = 0,      /* d_t m + grad m . v = 0 (problem (1), Sec. 1.1)               */
  GA_MODEL_CONTINUITY = 1,     /* d_t pi + div(pi v) = 0 (problem (11), Sec. 3.7)             */
  GA_MODEL_INCOMPRESSIBLE = 2  /* advection with v kept divergence free (Sec. 3.6)            */
} ga_model;

typedef enum { GA_PREC_FP64 = 0, GA_PREC_MIXED = 1 } ga_precision;
typedef enum { GA_MEM_HOST = 0, GA_MEM_DEVICE = 1 } ga_mem;
/* GA_METHOD_GA_AA: Anderson acceleration AA(w) (Alg. 2) on the map q with the mixing schedule of
 * Alg. 3 (GA-AA; Sec. 2.3.2 and Sec. 3.3 compare it with GA-NGMRES). */
typedef enum { GA_METHOD_GA_NGMRES = 0, GA_METHOD_RPGD = 1, GA_METHOD_GA_AA = 2 } ga_method;

/* Problem description (Sec. 1.1 problem statement, Sec. 2.2 discretisation). */
typedef struct {
  int dim;          /* 2 or 3                                                               */
  int n[3];         /* grid n_1..n_dim; each 4..1024 and a product of 2, 3 and 5            */
  int nt;           /* time steps n_t >= 1 (h_t = 1/n_t)                                    */
  int model;        /* ga_model                                                             */
  int reg_order;    /* s in {1,2,3}: H^s seminorm, symbol |k|^{2s}                          */
  double alpha;     /* regularisation weight alpha > 0                                      */
  int prec;         /* ga_precision                                                         */
  int ckpt_every;   /* 0: store all n_t+1 states; K > 0: store every K-th, recompute the rest */
} ga_problem_desc;

/* Solver options (Alg. 3 inputs, line search of Sec. 2.3). */
typedef struct {
  int window;          /* w >= 0 (at most 62)                                               */
  int sigma;           /* NGMRES steps per period, >= 1                                     */
  int tau;             /* fixed-point steps per period, >= 0                                */
  int max_iter;        /* n_iter > 0                                                        */
  double rel_tol;      /* eps_rel: stop when ||g||_inf <= eps_rel ||g(v^(0))||_inf          */
  double armijo_c;     /* c in the Armijo condition (paper: 1e-4)                           */
  int max_backtracks;  /* halvings before GA_ERR_LINESEARCH (paper: unbounded; default 20)  */
  int variant;         /* 1: FP step when mod(k, sigma+tau) >= sigma (GA-NGMRES);
                          2: FP step when mod(k, sigma+tau) < tau (aNGMRES(w)[sigma]-FP[tau]) */
  int method;          /* ga_method                                                         */
  int graphs;          /* 0: launch kernel by kernel, the host taking the line-search and step
                          decisions (one synchronisation per evaluation).
                          1: as 0, but the evaluations the solver repeats (line-search objective,
                          gradients) are captured into CUDA graphs and replayed; costs 3 vector fields
                          of device memory.
                          2: device-driven: ga_solve is one CUDA graph launch (and ga_solve_batch one
                          launch for all problems when every context uses 2). Conditional graph
                          nodes loop over the iterations and the line-search trials and choose the
                          kind of step from control kernels that take the host's decisions on the
                          device; the host synchronises once per call. GA-NGMRES and RPGD only
                          (GA_ERR_ARG with GA-AA). ga_step runs one iteration of the same graph.
                          t_grad_ms then holds the device time of whole runs and t_obj_ms stays 0.
                          After a failed run the next ga_step starts afresh from its v_inout.
                          All three give the same iterates and counters, bit for bit.             */
} ga_solver_opts;

/* Per-context counters and last-iterate metrics (the columns of the paper's tables, Sec. 3.3). */
typedef struct {
  int iters;           /* iterations performed since setup/reset                            */
  int grad_evals;      /* reduced-gradient evaluations (1 state + 1 adjoint solve each)     */
  int obj_evals;       /* objective-only evaluations (1 state solve each)                   */
  int pde_solves;      /* state + adjoint transport solves                                  */
  int ls_trials;       /* line-search trials                                                */
  int last_branch;     /* 0: NGMRES step, 1: fixed-point step                               */
  int converged;       /* 1 once ||g||_inf <= rel_tol ||g0||_inf                             */
  double obj;          /* obj(v^(k))                                                        */
  double mismatch;     /* 1/2 ||m(1) - m_1||^2 at v^(k)                                     */
  double rel_grad_inf; /* ||g(v^(k))||_inf / ||g(v^(0))||_inf                                */
  double grad_inf0;    /* ||g(v^(0))||_inf                                                  */
  double rho_mem;      /* remembered line-search step                                       */
  double last_rho;     /* accepted step of the last line search                             */
  double t_grad_ms;    /* device time in gradient evaluations                               */
  double t_obj_ms;     /* device time in objective evaluations                              */
  double t_total_ms;   /* wall time inside ga_step/ga_solve                                 */
} ga_stats;

typedef struct ga_ctx ga_ctx; /* opaque; owns all device memory of one problem */

/* Create a context on the current CUDA device. m0, m1: template/reference (or densities pi0,
 * pi1) as scalar fields of the descriptor's element type. stream: a cudaStream_t (NULL = the
 * legacy default stream) on which all work of this context is ordered. (Inside a gradient the
 * body force's derivative passes run on a second stream the context owns, forked from this stream
 * by an event and joined back to it before the gradient's next step, so to the caller every call
 * is still ordered on `stream`; in a captured graph the fork and join are graph edges.) Before it allocates
 * anything, ga_setup compares the workspace (ga_workspace_bytes) with the device's free memory and
 * returns GA_ERR_NOMEM, with the two figures in the message, when it does not fit; a cudaMalloc that
 * still fails later (another allocator took the memory meanwhile) also returns GA_ERR_NOMEM. Either
 * way nothing stays allocated and *out is NULL. */
ga_status ga_setup(const ga_problem_desc* desc, const ga_solver_opts* opts, const void* m0,
                   const void* m1, int mem, void* stream, ga_ctx** out);

/* Device memory (bytes) that ga_setup allocates for this descriptor and these options: every field,
 * trajectory slot, spectral work area, window pool and FP64 scratch array of the context, summed as
 * requested (the allocator rounds each allocation up further). Host arithmetic only: no GPU is
 * needed. The discretise-then-optimise gradient adds one vector field on its first call.
 * GA_ERR_ARG for an invalid descriptor or options (the same checks as ga_setup). */
ga_status ga_workspace_bytes(const ga_problem_desc* desc, const ga_solver_opts* opts, size_t* bytes);

/* obj(v) (Eq. (1a)): one state solve (forward only). */
ga_status ga_objective(ga_ctx* ctx, const void* v, int mem, double* obj);

/* Reduced gradient g(v) = alpha L v + int_0^1 lambda grad m dt (Eq. (3); continuity model:
 * alpha L v - int pi grad lambda dt; incompressible: alpha L v + P int lambda grad m dt) with
 * the state and adjoint (Eq. (4)) solved by the semi-Lagrangian scheme of Sec. 2.2. Also
 * returns obj(v) when obj != NULL. g is a vector field (dim components). */
ga_status ga_gradient(ga_ctx* ctx, const void* v, void* g, int mem, double* obj);

/* Deformation diagnostics of a velocity v (the map y and det grad y shown with the results of
 * Sec. 3; for incompressible flows det grad y = 1). y maps a point at t = 1 to the origin of its
 * characteristic, so that the advected image is m(., 1) = m0(y). Outputs: u, a vector field (dim
 * components) in grid units with y_c(x) = x_c + h_c u_c(x), from the composition of the state
 * step's departure points, u_0 = 0, u_{j+1} = I[u_j](X-) + (X- - x); detj, a scalar field, from
 * the continuity state solve started from 1 (the Jacobian of the inverse flow map is the density
 * of the transported uniform measure). Uses the context's n_t and grid; 2 + dim state solves. */
ga_status ga_deformation(ga_ctx* ctx, const void* v, void* u, void* detj, int mem);

/* Gradient of the discrete objective (discretise-then-optimise; the solver and ga_gradient use the
 * paper's optimise-then-discretise gradient, Sec. 2.1): with m_{j+1} = A m_j the semi-Lagrangian step,
 * g = alpha L v + (1/h^d) dJ_data/dv, the data part from the transposed (scattered) interpolation, the
 * derivative of the cubic interpolant at the departure points and the chain rule through the RK2
 * departure points (incompressible model: P applied to it). Advection and incompressible models only
 * (GA_ERR_ARG for the continuity model). Agrees with finite differences of obj(v) to their truncation
 * error. FP32 results vary at the rounding level between runs (atomic scatter order). */
ga_status ga_gradient_dto(ga_ctx* ctx, const void* v, void* g, int mem, double* obj);

/* Preconditioned direction s = -(alpha L)^{-1} g with zero symbol entries of L set to one
 * (Sec. 2.2, Eq. (9)); incompressible model: s = -(alpha L)^{-1} P g. */
ga_status ga_precond(ga_ctx* ctx, const void* g, void* s, int mem);

/* One iteration of Alg. 3 (GA-NGMRES(w; sigma, tau)), of RPGD (Eq. (9)) or of GA-AA, including the
 * Armijo line search with step memory that defines q (Eq. (10)). The first call after setup or
 * ga_reset takes v^(0) from v_inout; every call writes v^(k+1) to v_inout. stats may be NULL. */
ga_status ga_step(ga_ctx* ctx, void* v_inout, int mem, ga_stats* stats);

/* Iterate ga_step until ||g||_inf <= rel_tol ||g0||_inf or max_iter iterations. Starts from
 * v_inout (Alg. 3 uses v^(0) = 0). Returns GA_ERR_NOT_CONVERGED (v_inout and stats valid) when
 * the cap is reached. */
ga_status ga_solve(ga_ctx* ctx, void* v_inout, int mem, ga_stats* stats);

/* Forget the iteration state (k = 0, empty window, rho memory = 1); data stay. */
ga_status ga_reset(ga_ctx* ctx);

/* Solve `count` independent problems, each with its own context (the batched form of the solver).
 * When every context was set up with graphs = 2, all the solves are chains of one CUDA graph,
 * launched once (on a library stream ordered after each context's stream and before its results are
 * read); the graph is kept for the next call with the same list of contexts and dropped when one of
 * them is destroyed. Otherwise the problems are driven concurrently by host workers, each on its own
 * context's stream, so their kernels overlap on the GPU; give every context its own stream for the
 * overlap to happen. Contexts must be distinct. v[i] is problem i's v_inout (all in memory `mem`); stats[i] (may be NULL)
 * receives its statistics. Returns the first non-OK status other than GA_ERR_NOT_CONVERGED in
 * problem order, else GA_ERR_NOT_CONVERGED if any problem hit its cap, else GA_OK. */
ga_status ga_solve_batch(int count, ga_ctx* const* ctxs, void* const* v, int mem, ga_stats* stats);

ga_status ga_get_stats(const ga_ctx* ctx, ga_stats* stats);
void ga_destroy(ga_ctx* ctx);
const char* ga_status_str(ga_status s);
const char* ga_last_error(const ga_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GA_H */
