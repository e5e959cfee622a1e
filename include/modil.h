/*
 * modil.h -- C ABI of the GB300 mODIL library (libmodil.so).
 *
 * mODIL (multiresolution Optimizing a DIscrete Loss) solves a PDE problem,
 * forward or inverse, by minimising a discrete loss with a gradient-based
 * optimiser.  The unknown field on the fine grid is the multigrid
 * decomposition u = M_L(u_1, ..., u_L) = u_1 + T_1 (u_2 + ... T_{L-1} u_L)
 * of per-level arrays u_i on grids N_i = N / 2^(i-1) (paper, Section 2.2,
 * the two displayed forms of M_L); T_i is cell-based linear interpolation
 * (Section 2.2, the 8x4 and 4x2 matrices).  The loss is the weighted sum of
 * squared discrete residuals plus squared data mismatches plus regularisers
 * (Section 2.1 displayed loss; Sections 3.2 and 3.4).  One optimiser step
 * composes the field, evaluates the residuals, reduces the loss, runs the
 * adjoint of the stencils and of the prolongations, and applies Adam
 * (Section 2.1) to every level.  Everything in a step runs in this library's
 * CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - Return value: MODIL_OK or a negative modil_status.  No call aborts the
 *    process.  modil_last_error() gives a message for the calling thread.
 *  - Grids are row-major with the LAST axis fastest.  Space-time problems use
 *    axes (t, x); 2-D problems (y, x); 3-D problems (z, y, x).
 *  - Every pointer passed in stays owned by the caller.  modil_create copies
 *    what it needs (measurements, coefficients, initial values) before
 *    returning.
 *  - The library's device memory is one arena.  The caller may supply it
 *    (arena != NULL, at least modil_arena_bytes() bytes, 256-byte aligned,
 *    e.g. a torch uint8 tensor) and then owns it; with arena == NULL the
 *    library allocates it with cudaMalloc and modil_destroy frees it.
 *  - Work is issued on the stream given to modil_create / modil_set_stream
 *    (a cudaStream_t; NULL is the legacy default stream).  Calls that return
 *    numbers to host memory synchronise that stream first; the others are
 *    asynchronous.
 *  - Device-side failures (non-finite loss) are latched in device memory and
 *    reported as MODIL_ERR_NONFINITE by the next call that returns numbers.
 */
#ifndef MODIL_H
#define MODIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct modil_problem modil_problem; /* opaque, library-owned */

typedef enum {
  MODIL_OK = 0,
  MODIL_ERR_ARG = -1,         /* invalid argument or descriptor            */
  MODIL_ERR_OOM = -2,         /* device or host allocation failed          */
  MODIL_ERR_CUDA = -3,        /* a CUDA runtime call failed                */
  MODIL_ERR_UNSUPPORTED = -4, /* valid request this build does not handle  */
  MODIL_ERR_NONFINITE = -5,   /* loss became NaN or Inf                     */
  MODIL_ERR_STATE = -6,       /* call not valid in the problem's state      */
  MODIL_ERR_TIMEOUT = -7      /* a bounded wait inside a kernel ran out: the
                                 pass skipped the affected tiles, so its
                                 results are incomplete; reported once       */
} modil_status;

/* PDE families (paper Section 3). */
enum {
  MODIL_PDE_BURGERS = 1, /* viscous Burgers u_t + (u^2/2)_x = nu u_xx, axes (t, x),
                            x in [-1, 1], t in [0, 1]; Section 3.2 with viscosity   */
  MODIL_PDE_HEAT = 2,    /* u_t = (k(u) u_x)_x with unknown k, axes (t, x) on [0,1]^2;
                            Section 3.4, the displayed implicit scheme              */
  MODIL_PDE_NS2D = 3,    /* steady incompressible Navier-Stokes, lid-driven cavity on
                            [0,1]^2 (square grid), fields 0 = u, 1 = v, 2 = p; collocated
                            finite volumes with Rhie-Chow continuity; Section 3.3   */
  MODIL_PDE_NS3D = 4,    /* steady Navier-Stokes past a body in 3-D with the body as
                            a penalisation field (Section 3.5, the penalised momentum
                            equation): axes (z, y, x) on [0,1] x [0,1] x [0,2], fields
                            0 = u, 1 = v, 2 = w (velocity along x, y, z), 3 = p,
                            4 = chihat with body fraction chi = 1/(1+exp(-(chihat-5)));
                            inlet x = 0 (u = (1,0,0)), outlet x = 2 (p = 0), free-slip
                            walls in y and z; ndim = 3                               */
  MODIL_PDE_POISSON = 5  /* Poisson equation lap(u) = f on [0,1]^d, d = ndim = 1, 2 or 3,
                            axes slowest first (Section 3.1).  Cell layout: finite
                            volumes at cell centres, zero Dirichlet walls by quadratic
                            extrapolation from the wall and the two nearest centres
                            (ghost = -2 u_0 + u_1 / 3), residual in every cell, every
                            axis >= 2 cells.  Node layout: finite differences at the
                            N + 1 nodes per axis, the Dirichlet value imposed on the
                            boundary nodes (the stencil reads 0 there, their
                            unknowns get no residual gradient), residual at interior
                            nodes.  f in aux, one
                            value per fine cell (node).  The 2-D cell layout runs in
                            the fused tile kernel, the others in a kernel per step of
                            the method (grids of a few tens of cells per axis)    */
};

enum { MODIL_F32 = 0, MODIL_F64 = 1 };
enum { MODIL_CELL = 0, MODIL_NODE = 1 };

#define MODIL_MAX_LEVELS 10
#define MODIL_MAX_FIELDS 5
#define MODIL_MAX_KNODES 64

/* Loss terms reported by the eval/step calls (doubles, in this order). */
enum { MODIL_TERM_TOTAL = 0, MODIL_TERM_RES = 1, MODIL_TERM_DATA = 2, MODIL_TERM_REG = 3,
       MODIL_NTERMS = 4 };

typedef struct {
  int pde;      /* MODIL_PDE_*                                                   */
  int dtype;    /* MODIL_F32 or MODIL_F64: storage and stencil arithmetic       */
  int ndim;     /* 2 for BURGERS, HEAT and NS2D; 3 for NS3D                     */
  int shape[3]; /* fine cells per axis, slowest first; unused entries 0         */
  int n_levels; /* L >= 1; every axis must be divisible by 2^(L-1); 1 = ODIL    */
  double coef[4]; /* BURGERS: coef[0] = nu.  HEAT: unused.  NS2D: coef[0] = Re,
                     coef[1] = Rhie-Chow factor (tau = coef[1] * h).  NS3D:
                     coef[0] = Re, coef[1] = D (viscosity D/Re), coef[2] = lambda
                     (penalisation), coef[3] = Rhie-Chow factor                   */
  double w_res;   /* residual weight: w_res * dV * sum r^2                       */
  double w_data;  /* data weight: w_data / n_meas * sum (u - y)^2                */
  double w_reg;   /* HEAT: w_reg * sum_j (q_{j+1} - 2 q_j + q_{j-1})^2           */
  int n_meas;     /* number of measurements (0 allowed)                          */
  const int32_t* meas_cell;  /* flat fine-grid cell index per measurement       */
  const int32_t* meas_field; /* field index per measurement, or NULL (field 0)  */
  const double* meas_value;  /* measured value                                  */
  int n_aux;                 /* HEAT: initial temperature, one per x cell;
                                POISSON: right-hand side f, one per fine cell
                                (row-major, n_aux = ny * nx)                   */
  const double* aux;
  int n_knodes;              /* HEAT: conductivity nodes q_0..q_{K}, K+1 <= 64  */
  const double* knodes;      /* initial q (copied)                              */
  double adam_lr, adam_beta1, adam_beta2, adam_eps;
  int n_points;               /* off-grid measurements (every family):            */
  const double* point_coord;  /* n_points x ndim physical coordinates, slowest
                                 axis first, in the problem's domain (by default
                                 Burgers t in [0,1], x in [-1,1]; heat, Poisson,
                                 cavity [0,1]^2; the body (z, y, x) in [0,1] x
                                 [0,1] x [0,2]; see domain_lo);
                                 the field there is interpolated linearly along
                                 each axis (bilinear, trilinear) between the
                                 two nearest cell centres
                                 (clamped between a wall and the outermost
                                 centre); cells and points share one data weight
                                 w_data / (n_meas + n_points)                   */
  const double* point_value;
  int tile[2];               /* fine tile (rows, cols); 0 = library default.
                                Burgers/heat/Poisson: 16x32 16x64 8x64 32x32 8x128;
                                Burgers without off-grid points also 32x60 (the
                                warp-streaming kernel, its default);
                                NS2D: 8x32 16x32.  NS3D: 0 only (4x8x16 cells)  */
  double domain_lo[3], domain_hi[3];
                             /* physical extent per axis, slowest first (2-D: entries
                                0 and 1), for Burgers, heat and Poisson: spacing
                                (hi - lo) / cells, the origin of off-grid points.
                                All zero: the family's own domain (Burgers t in
                                [0, 1], x in [-1, 1]; heat and Poisson [0, 1]^2).
                                The cavity and the body take only their own.    */
  const int32_t* point_field; /* field sampled at each off-grid point, or NULL
                                 (field 0): the cavity's u, v or p, the body's
                                 u, v, w, p or chihat                           */
  int layout;                 /* POISSON: MODIL_CELL (0, values at cell
                                 centres) or MODIL_NODE (1, values at the N + 1
                                 nodes per axis); the other families: 0       */
  int k_fixed;                /* HEAT: nonzero = the conductivity is known (the
                                 forward problem that makes a reference record,
                                 Section 3.4): the nodes stay at `knodes`, dL/dq
                                 reads as zero and no optimiser moves them;
                                 the other families: 0 (else MODIL_ERR_ARG)    */
  double k_scale;             /* HEAT: the unit in which the optimisers move the
                                 conductivity nodes (a diagonal preconditioner:
                                 Adam's node step is adam_lr * k_scale, L-BFGS
                                 works on q / k_scale); 0 = 1.  The nodes are
                                 ~0.02 where the temperatures are ~1, so an
                                 unscaled step overshoots them.  The other
                                 families: 0 (else MODIL_ERR_ARG)             */
} modil_desc;

/* Device bytes needed for a batch of n problems described by descs[0..n-1]. */
modil_status modil_arena_bytes(const modil_desc* descs, int n, size_t* bytes);

/* Create a batch of n >= 1 independent problems of one PDE family and dtype.
 * All levels start at zero, Adam moments at zero, step count 0.
 * arena: caller-owned device buffer of modil_arena_bytes() bytes or NULL.
 * stream: cudaStream_t for all work of this problem.  */
modil_status modil_create(const modil_desc* descs, int n, void* arena, size_t arena_bytes,
                          void* stream, modil_problem** out);

/* Wait for the problem's stream, then free the problem (and the arena if the
 * library allocated it).  NULL is a no-op. */
void modil_destroy(modil_problem* p);

modil_status modil_set_stream(modil_problem* p, void* stream);

/* Cells per axis of a level, slowest first: 2-D problems fill shape[0..1]
 * and set shape[2] = 0, 3-D problems fill all three. */
modil_status modil_level_shape(const modil_problem* p, int instance, int level, int shape[3]);

/* Copy one level (field, level 0 = finest) in or out; bytes must equal the
 * level size in the problem's dtype.  *_on_device selects device or host
 * memory for src/dst.  Writing a level also resets nothing else.  */
modil_status modil_write_level(modil_problem* p, int instance, int field, int level,
                               const void* src, size_t bytes, int src_on_device);
modil_status modil_read_level(modil_problem* p, int instance, int field, int level, void* dst,
                              size_t bytes, int dst_on_device);
/* Gradient dL/du_level from the last modil_eval_grad (or the last step). */
modil_status modil_read_grad(modil_problem* p, int instance, int field, int level, void* dst,
                             size_t bytes, int dst_on_device);
/* Composed fine field M_L(u_1..u_L), computed on the device. */
modil_status modil_read_field(modil_problem* p, int instance, int field, void* dst,
                              size_t bytes, int dst_on_device);
/* HEAT conductivity nodes q (doubles on the host) and their gradient. */
modil_status modil_write_knodes(modil_problem* p, int instance, const double* q, int n);
modil_status modil_read_knodes(modil_problem* p, int instance, double* q, int n);
modil_status modil_read_kgrad(modil_problem* p, int instance, double* gq, int n);

/* Loss of the current levels.  terms: n_instances * MODIL_NTERMS doubles on
 * the host (synchronises), or NULL.  */
modil_status modil_eval_loss(modil_problem* p, double* terms);
/* Loss and gradient for every level (read with modil_read_grad). */
modil_status modil_eval_grad(modil_problem* p, double* terms);
/* n_steps Adam steps of every instance.  terms (nullable) receives the loss
 * terms evaluated at the start of the last step.  Asynchronous when NULL. */
modil_status modil_step(modil_problem* p, int n_steps, double* terms);
/* Kernel launches one modil_step issues: the composition launches (one per
 * level, coarse to fine: the 3-D family and the warp-streaming Burgers
 * kernel), the fused fine kernel, one restriction+Adam kernel per coarser
 * level above the tail, one finalising (tail) kernel. */
modil_status modil_launches_per_step(const modil_problem* p, int* n);

/* One Adam step issued kernel by kernel with a CUDA event between launches;
 * ms[k] receives the device time of launch k (order as above).  Synchronises.
 * max_kernels: capacity of ms; *n_kernels: launches timed. */
modil_status modil_profile_step(modil_problem* p, float* ms, int max_kernels, int* n_kernels);
/* What each launch of modil_profile_step is: kind[k] 0 = composition of a
 * level, 1 = fused fine kernel, 2 = restriction+Adam of a level, 3 = tail;
 * level[k] its level (the tail: the first level it finishes). */
modil_status modil_profile_labels(const modil_problem* p, int* kind, int* level, int max_kernels,
                                  int* n_kernels);

/* ---- caller-owned parameters (e.g. a torch.autograd.Function) -------------
 * The layout of all levels of a batch in one buffer ("parameter vector"):
 * instance-major, then field, then level (finest first), each level
 * row-major; modil_param_count gives its length in elements of the dtype and
 * modil_level_offset the element offset of one level.  The evaluation is the
 * same as modil_eval_loss / modil_eval_grad (paper Section 2.1 loss, Section
 * 2.2 decomposition) but reads the levels from `levels` (device) instead of
 * the problem's own copy; the heat conductivity nodes come from the problem.
 *   modil_loss_fwd: loss terms (host, n_instances * MODIL_NTERMS, synchronises);
 *                   with terms == NULL it only launches the pass (asynchronous)
 *                   and the terms are read on the device (modil_terms_device).
 *   modil_loss_bwd: grads (device, parameter-vector layout) = grad_out * dL/dlevels;
 *                   asynchronous on the problem's stream.
 *   modil_terms_device: device address of instance 0's MODIL_NTERMS loss terms
 *                   (doubles, written by every pass) and the distance in doubles
 *                   between consecutive instances' terms; valid while the
 *                   problem lives. */
modil_status modil_param_count(const modil_problem* p, long long* n);
modil_status modil_level_offset(const modil_problem* p, int instance, int field, int level,
                                long long* offset);
modil_status modil_loss_fwd(modil_problem* p, const void* levels, double* terms);
modil_status modil_loss_bwd(modil_problem* p, const void* levels, double grad_out, void* grads);
modil_status modil_terms_device(const modil_problem* p, const double** terms, int* stride);

/* Persistent launch of the fine-tile kernel (Burgers, heat): on != 0 launches
 * as many blocks as fit on the GPU at once, each taking tiles of all
 * instances from an atomic queue until it is empty (useful for batches of
 * uneven instances); on == 0 launches one block per tile (default). */
modil_status modil_set_persistent(modil_problem* p, int on);

/* Steps taken so far (the Adam step counter t). */
modil_status modil_step_count(const modil_problem* p, long long* t);

/* Checkpoint and resume (the paper has no counterpart; its runs take up to
 * two hours).  modil_save synchronises the problem's stream and writes, to a
 * file at `path`, a header (format version, PDE, dtype, fields, instances,
 * parameter counts, a hash of every instance's level shapes, the step count)
 * followed by the current levels, the Adam moments m and v, the conductivity
 * nodes with their moments, and the per-instance step state.  modil_load
 * reads such a file into a problem created from the same descriptors (same
 * PDE, dtype and level shapes; otherwise MODIL_ERR_ARG and the problem is
 * unchanged) and continues from it: the steps that follow are bit for bit
 * those of the run that wrote it, since every reduction of a step has a
 * fixed order.  Measurements, weights and coefficients come from the
 * problem's own descriptors, not from the file.  Both return MODIL_ERR_ARG
 * when the file cannot be opened, written or read in full. */
modil_status modil_save(modil_problem* p, const char* path);
modil_status modil_load(modil_problem* p, const char* path);

/* Zero the Adam moments and the step counter of every instance. */
modil_status modil_reset_optimizer(modil_problem* p);

/* Loss and gradient of ONE problem with no device allocation at all.
 * The paper has no counterpart: this is an interface for callers that cannot
 * allocate device memory -- plug-ins whose host application owns every device
 * allocation through its own pool, loops that must not allocate once running
 * (cudaMalloc can synchronise the device), or code that only holds the
 * buffers it was given.  The working memory (per-tile partial sums, problem
 * tables, measurement runs) lives in one file-scope __device__ array of 8 MiB
 * that every GPU loading the library keeps until the process exits.
 *   desc:   one problem, as for modil_create (read on the host): Burgers,
 *           heat, Poisson or the cavity.
 *   levels: device, every field's levels back to back, field-major (field 0's
 *           levels, then field 1's, ...; within a field level 0 first, each
 *           row-major), dtype of desc; one field except the cavity (u, v, p).
 *           Conductivity nodes come from desc.  Must start on a 16-byte
 *           boundary (the kernels use 16-byte vector accesses).
 *   grads:  device output, dL/du of every level, same layout and alignment
 *           as levels.
 *   terms:  host output, MODIL_NTERMS doubles.  kgrad: host output of n_knodes
 *           doubles (heat) or NULL.
 *   stream: cudaStream_t; the call synchronises it before returning.
 * Returns MODIL_ERR_ARG if the problem needs more than the 8 MiB of working
 * memory or a pointer is misaligned, MODIL_ERR_UNSUPPORTED for the 3-D body
 * problem (it needs a composed-field buffer) and for off-grid points, before
 * anything runs on the GPU.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents (every
 * value a call reads is written by that call first), so calls that overlap on
 * the GPU -- on different streams or threads -- race and must be serialised
 * by the caller.  Calls no cudaMalloc, cudaFree or allocating routine. */
modil_status modil_eval_grad_noalloc(const modil_desc* desc, const void* levels, void* grads,
                                     double* terms, double* kgrad, void* stream);

/* Limited-memory BFGS on the levels of a problem: the optimiser the paper
 * uses for most of its results (SciPy's L-BFGS-B without bounds, Section 2.1;
 * a history of 50 pairs in Section 3.1).  The paper gives no algorithmic
 * detail; this is the textbook method: direction -H g over the newest
 * `history` pairs (s, y) with H0 = (s.y / y.y) I of the newest pair, H g
 * evaluated in the compact representation (Byrd, Nocedal and Schnabel 1994;
 * the same H g as the two-loop recursion) from batched dot products and one
 * pass over the stored vectors; the first direction -g with a first trial step of
 * 1 / ||g||; backtracking on the Armijo condition f(x + t d) <= f(x) +
 * 1e-4 t g.d, halving t, at most 40 trials (the run stops when none passes
 * or g.d >= 0); a pair is kept only when s.y > 1e-12 y.y.  Vectors live on
 * the device in the problem's dtype; dot products are reduced in FP64 in a
 * fixed order; the loss and gradient are the problem's own kernels.
 *   modil_lbfgs_create: single-instance problems (MODIL_ERR_UNSUPPORTED for
 *     a batch).  The unknowns are the levels of every field and, for the heat
 *     problem without k_fixed, its conductivity nodes after them (the pass
 *     reads the nodes from, and writes their gradient to, the problem's node
 *     arrays; Adam's node moments are untouched).  Allocates (2 history + 6)
 *     vectors of the unknowns in device memory.  The optimiser keeps a
 *     pointer to p, which must outlive it.
 *   modil_lbfgs_run: continues from the problem's current levels (and nodes;
 *     the pair history is kept across calls) for up to `iterations`
 *     iterations; writes the final levels (and nodes) and their gradient
 *     back into the problem (readable with modil_read_level / modil_read_grad
 *     / modil_read_knodes / modil_read_kgrad; Adam's state is untouched).
 *     loss: host output of iterations + 1 doubles or NULL: the loss at the
 *     start and after each completed iteration.  done: iterations completed.
 *     Synchronises the problem's stream (the line search reads the loss). */
typedef struct modil_lbfgs modil_lbfgs;
modil_status modil_lbfgs_create(modil_problem* p, int history, modil_lbfgs** out);
modil_status modil_lbfgs_run(modil_lbfgs* o, int iterations, double* loss, int* done);
void modil_lbfgs_destroy(modil_lbfgs* o);

/* Fault injection for tests (the paper has no counterpart): the number of
 * polls after which the 3-D body kernel's bounded wait for its tile copies
 * gives up (polls < 0 restores the default of 2^24; 0 gives up at once).  A
 * block whose wait runs out flags MODIL_ERR_TIMEOUT, waits (with the default
 * bound) for the copies still in flight, skips its tile and returns; the next
 * call that returns numbers reports the status once.  Affects every problem
 * on the current device; nothing hangs or faults. */
modil_status modil_test_set_spin_limit(long long polls);

/* Last error message of the calling thread ("" if none). */
const char* modil_last_error(void);

/* Library version string. */
const char* modil_version(void);

/* sizeof(modil_desc) as this library was compiled: a binding checks it
 * against its own copy of the struct before the first call. */
size_t modil_desc_size(void);

#ifdef __cplusplus
}
#endif
#endif /* MODIL_H */
