/*
 * dgnn.h - C ABI of libdgnn.so: nodal DGSEM for the 3D compressible Navier-Stokes
 * equations with a learned corrective forcing (arXiv 2207.11571), for NVIDIA GB300
 * (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: DG_OK (0) or a negative dg_status.  dg_last_error() returns a
 *   thread-local message describing the last failure of the calling thread.
 * - Unless a parameter says "host", array pointers are DEVICE pointers owned by the
 *   caller (for example torch CUDA tensors).  The library never frees them.  The
 *   library owns only what dg_create / nn_create allocate, released by
 *   dg_destroy / nn_destroy.
 * - Streams are cudaStream_t passed as void* (NULL = legacy default stream).  All
 *   work is enqueued on that stream; calls that return host values (diagnostics,
 *   stable dt, loss) synchronise that stream before returning.
 * - Conserved state q (Appendix A): five variables (rho, rho v1, rho v2, rho v3,
 *   rho e), FP64, layout [var][elem][node], node fastest.
 *   elem = ex + K (ey + K ez) on the periodic K^3 mesh of [-pi, pi]^3 (Sec. 3.1),
 *   node = i + n (j + n k), n = P + 1 Gauss-Lobatto points per direction, x fastest.
 *   N = K^3 n^3 nodes; q holds 5 N doubles.
 * - Nondimensionalisation: rho0 = V0 = L = 1, mu = 1/Re, p0 = 1/(gamma Mach^2),
 *   heat flux kappa grad T = mu gamma/((gamma-1) Pr) grad(p/rho).
 * - Errors: a NULL handle or pointer where one is required, or a size out of range,
 *   returns DG_ERR_INVALID_ARG without enqueuing work.  A CUDA failure returns
 *   DG_ERR_CUDA with the CUDA error string in dg_last_error().
 */
#ifndef DGNN_H
#define DGNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_INVALID_ARG = -1,
  DG_ERR_CUDA = -2,
  DG_ERR_NONFINITE = -3,   /* a diagnostic found NaN/Inf in the state */
  DG_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out (error flag set, kernel returned) */
  DG_ERR_IO = -5,          /* file missing, truncated or with a bad checksum */
  DG_ERR_UNSUPPORTED = -6, /* a parameter combination this build does not implement */
  DG_ERR_EXCHANGE = -7     /* a slab's exchange function reported a failure */
} dg_status;

typedef struct dg_ctx dg_ctx;
typedef struct nn_model nn_model;

/* Arithmetic of the spatial operator.  The state q is FP64 in both modes.
 * DG_PREC_FP64: every step in FP64, q updated in FP64 at every RK stage (parity path).
 * DG_PREC_FP32: fluxes, contractions and lifting in FP32 on the state relative to the
 *   reference (rho0 = 1, p0); within an RK3 step the stages accumulate the increment in
 *   FP32 and q is updated once per step in FP64. */
typedef enum {
  DG_PREC_FP64 = 0,
  DG_PREC_FP32 = 1
} dg_precision;

typedef struct {
  int precision;      /* dg_precision, default DG_PREC_FP64 */
  double gamma;       /* ratio of specific heats, default 1.4 */
  double Cs;          /* Smagorinsky constant, default 0.1 */
  double Prt;         /* turbulent Prandtl number, default 0.9 */
  double les_delta;   /* LES filter width; <= 0 selects h/(P+1) (default) */
  int elems_per_block;/* elements per CUDA block; <= 0 selects the tuned default for P */
  int block_shape;    /* 0: blocks of elems_per_block consecutive elements (default);
                         1: 2 x 2 x 2 cubes of elements (P <= 3 and even K only, else
                         DG_ERR_INVALID_ARG): a cube's twelve internal faces need no halo
                         and their interface fluxes are formed once for both sides */
  int volume_flux;    /* 0: standard strong-form volume term (default, the paper's);
                         1: kinetic-energy-preserving split form, 2 sum_m D_im F#(q_i, q_m)
                         with Pirozzoli's two-point flux for the Euler part (a robustness
                         variant for under-resolved turbulence, not in the paper; rows of
                         elements only: block_shape 1 returns DG_ERR_INVALID_ARG) */
} dg_opts;

/* Integral diagnostics (Sec. 2.4 Eq. 9 and kinetic-energy budget), FP64. */
typedef struct {
  double mass;          /* sum over nodes of w w w (h/2)^3 rho */
  double momentum[3];
  double energy;        /* integral of rho e */
  double ke;            /* (1/(2 pi)^3) integral rho |v|^2 / 2 */
  double dke_dt;        /* (1/(2 pi)^3) integral (v . R_m - |v|^2 R_rho / 2), R = p(q) (+ forcing) */
  double e_inf[3];      /* max |q - q_ref| for rho u, rho v, rho w (Eq. 9); 0 when q_ref is NULL */
  double max_wave;      /* max over nodes of |v| + c */
  int64_t nonfinite;    /* number of non-finite state values found */
} dg_diag;

/* Fills *opts with the defaults listed above.  Returns DG_ERR_INVALID_ARG on NULL. */
int dg_opts_default(dg_opts* opts);

/* Creates a solver for the periodic K^3 hex mesh of [-pi, pi]^3 (Sec. 3.1) at
 * polynomial order P (1 <= P <= 8) on Gauss-Lobatto nodes, for the flow (Re, Mach,
 * Pr) and closure (0: none; 1: Smagorinsky, Sec. 3.1 "LES").  Builds the basis on
 * the host in FP64, uploads it, and allocates the workspace (operator scratch and
 * the RK register).  opts may be NULL (defaults).  1 <= K <= 256.  DG_ERR_INVALID_ARG
 * (before any CUDA call) for arguments out of range: Re, Mach, Pr <= 0, gamma <= 1,
 * Cs < 0, Prt <= 0, a non-finite option, or the block_shape / volume_flux limits above. */
int dg_create(int K, int P, double Re, double Mach, double Pr, int closure,
              const dg_opts* opts, dg_ctx** out);
int dg_destroy(dg_ctx* ctx);

/* Host-only: the 1D Gauss-Lobatto basis of order P (1..8) that the solver uses
 * (Sec. 2.6: nodal Lagrange bases; nodes = endpoints and roots of L_P', weights
 * 2/(P(P+1) L_P(xi)^2), D[i*(P+1)+m] = l_m'(xi_i)).  Any output may be NULL. */
int dg_basis_1d(int P, double* xi, double* w, double* D);

/* Number of nodes N = K^3 (P+1)^3 and elements K^3 of the context. */
int dg_sizes(const dg_ctx* ctx, int64_t* nodes, int64_t* elems);

/* Taylor-Green vortex initial state (Sec. 3.1, Eq. 11) at the GL nodes:
 * rho = 1, v1 = sin x cos y cos z, v2 = -cos x sin y cos z, v3 = 0,
 * p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16, then q += perturbation.
 * q: device, 5 N doubles (written).  perturbation: device, 5 N doubles in the layout
 * of q, or NULL for none (the caller draws it). */
int dg_init_tgv(dg_ctx* ctx, double* q, const double* perturbation, void* stream);

/* dqdt = p(q) + s(q): the semi-discrete DGSEM operator (Sec. 2, Eq. 3/4): strong-form
 * volume term with sum-factorised derivative matrices, Roe advective and BR1 viscous
 * interface fluxes (Sec. 3.1), optional Smagorinsky viscosity, plus the network
 * forcing when forcing != NULL (Eq. 4).  q, dqdt: device, 5 N doubles. */
int dg_rhs(dg_ctx* ctx, const double* q, double* dqdt, const nn_model* forcing, void* stream);

/* dqdt = p(q) like dg_rhs, without any device allocation and without a context (the
 * paper has no counterpart: this is a service for callers that may not allocate device
 * memory, e.g. an in-situ hook inside another code's time loop whose device memory is
 * fixed at start-up, or a host thread that must not take the allocator's locks or
 * synchronise the device, as cudaMalloc and cudaFree may).  The mesh and flow are given
 * as in dg_create (default dg_opts apart from precision, no forcing).  q, dqdt: DEVICE,
 * 5 N doubles, N = K^3 (P+1)^3.
 * The two intermediate fields of the operator live in one scratch array inside the
 * library's device image (3.7 MB, kept by every GPU that loads the library until exit):
 * N may be at most 32768 nodes, larger meshes return DG_ERR_INVALID_ARG.  The first call
 * on a device (with that device current) does the set-up: it looks up the array's device
 * address and uploads the FP32 kernels' constant tables (synchronous copies, whatever the
 * precision asked for); make it before any stream capture.  Later calls only enqueue
 * kernels on stream.  The looked-up address belongs to the device's context: after
 * cudaDeviceReset no further call may be made.  All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU (other streams or host
 * threads) race and must be serialised by the caller. */
int dg_rhs_noalloc(int K, int P, double Re, double Mach, double Pr, int closure, int precision,
                   const double* q, double* dqdt, void* stream);

/* Advances q in place by nsteps low-storage RK3 steps of size dt (Sec. 2, Eq. 6 with
 * the third-order Runge-Kutta scheme of Sec. 3.1; Williamson 2N coefficients).  When
 * forcing != NULL the network forcing s(q_k) is evaluated on every stage state and
 * added to the operator (Eq. 4 integrated by RK3), or, after
 * dg_set_forcing_mode(ctx, DG_FORCING_POST), added once per step as in Algorithm 1.
 * q: device, 5 N doubles. */
int dg_rk3_step(dg_ctx* ctx, double* q, double dt, int nsteps, const nn_model* forcing,
                void* stream);

/* ---- Batches of independent solvers (no counterpart in the paper: a throughput service
 * for many small flows at once, e.g. a sweep over Re, mesh and order).  Every member
 * computes exactly what dg_rk3_step computes for it alone. ---- */
typedef struct dg_batch dg_batch;

/* One member: mesh, order and flow as the arguments of dg_create. */
typedef struct {
  int K;
  int P;
  double Re;
  double Mach;
  double Pr;
  int closure;
} dg_instance_desc;

#define DG_BATCH_MAX 16
#define DG_BATCH_NO_GRAPH 1 /* dg_batch_rk3_step flag: launch directly, no graph replay */
#define DG_BATCH_PERSISTENT 2 /* dg_batch_rk3_step flag: one persistent launch per RK stage for every
                                 member (FP32 operator, orders 1..6; else DG_ERR_UNSUPPORTED) */

/* Creates n (1..DG_BATCH_MAX) members from desc (host array of n), all with the same
 * opts (NULL = defaults; the precision and elements-per-block apply to every member).
 * Each member owns the workspace of a dg_create context.  Errors of a member's creation
 * return that member's status with its index in dg_last_error(). */
int dg_create_batch(const dg_instance_desc* desc, int n, const dg_opts* opts, dg_batch** out);
int dg_batch_destroy(dg_batch* batch);
int dg_batch_size(const dg_batch* batch, int* n);

/* Context of member i, borrowed: usable with every dg_* call that takes a context
 * (dg_init_tgv, dg_diagnostics, dg_stable_dt, dg_rk3_step, ...), released only by
 * dg_batch_destroy (dg_destroy on it returns DG_ERR_INVALID_ARG). */
int dg_batch_member(dg_batch* batch, int i, dg_ctx** out);

/* Advances every member i in place by nsteps RK3 steps of size dt[i], with the same
 * arithmetic as dg_rk3_step (no forcing).  q: HOST array of n DEVICE pointers, member i's
 * state (5 N_i doubles, distinct buffers); dt: HOST array of n step sizes.  Members of one
 * order share one launch per kernel phase and stage; members of different orders run as
 * parallel branches.  Unless flags has DG_BATCH_NO_GRAPH, one step is recorded as a CUDA
 * graph on the batch's private streams (the first call, and again whenever the q
 * pointers, dt values or elements-per-block change) and replayed nsteps times on stream;
 * the call must then not be made while that stream is being captured.  With
 * DG_BATCH_PERSISTENT each RK stage of every member, of every order, is one cooperative
 * launch whose blocks walk the gradient phase of all members, meet at a grid barrier
 * (a bounded wait: on expiry the first member's error flag is set, reported by its
 * dg_diagnostics as DG_ERR_TIMEOUT) and walk the flux phase; the per-element arithmetic
 * is that of dg_rk3_step. */
int dg_batch_rk3_step(dg_batch* batch, double* const* q, const double* dt, int nsteps, int flags,
                      void* stream);

/* Picks elements-per-block for each order present: dg_autotune on the largest member
 * of that order (q, dt: as in dg_batch_rk3_step), applied to all members of the order. */
int dg_batch_autotune(dg_batch* batch, double* const* q, const double* dt, void* stream);

/* Same as dg_rk3_step but q_host is a HOST array (pageable or pinned, 5 N doubles):
 * copies it to the device, advances, copies it back, and fills *diag (host, may be
 * NULL) for the final state.  Synchronises the stream.  DG_ERR_INVALID_ARG while
 * dg_advance_host_async calls of the context are pending. */
int dg_advance_host(dg_ctx* ctx, double* q_host, double dt, int nsteps,
                    const nn_model* forcing, dg_diag* diag, void* stream);

/* dg_advance_host in two calls, so that several contexts on several streams overlap
 * their copies with each other's kernels, and a context's next call is queued before
 * the previous one's results are read.  dg_advance_host_async enqueues on stream the
 * copy of q_host (HOST, 5 N doubles; pinned for the copies to run asynchronously) to
 * the context's device state, nsteps RK3 steps (as dg_rk3_step), the copy back into
 * q_host and, if want_diag != 0, the diagnostics of the final state into a pinned slot
 * of the context; it returns without waiting.  Up to two calls may be pending per
 * context, both on the same stream (the second one's copy in follows the first one's
 * copy back); a third call, or a second on another stream, returns DG_ERR_INVALID_ARG.
 * dg_advance_host_wait(ctx, diag, stream) waits for the OLDEST pending call only (an
 * event after its last copy; `stream` is used only when no call is pending, then it is
 * synchronised) and fills *diag (HOST, may be NULL; non-NULL requires want_diag in that
 * call, else DG_ERR_INVALID_ARG) from its slot.  A call's q_host must not be touched
 * until its wait has returned; collect every pending call before dg_destroy. */
int dg_advance_host_async(dg_ctx* ctx, double* q_host, double dt, int nsteps,
                          const nn_model* forcing, int want_diag, void* stream);
int dg_advance_host_wait(dg_ctx* ctx, dg_diag* diag, void* stream);

/* q_lo = G q_hi: the filter of Eq. 2, per element nodal(P_hi) -> Legendre modes ->
 * truncation to degree P_lo per direction -> nodal(P_lo) (Sec. 2.6), FP64.  Both
 * contexts must share K and P_lo <= P_hi.  q_hi, q_lo: device. */
int dg_project(const dg_ctx* hi, const dg_ctx* lo, const double* q_hi, double* q_lo,
               void* stream);

/* q_hi = I q_lo: each element's order-P_lo nodal polynomial evaluated at the order-P_hi
 * Gauss-Lobatto nodes (exact: Q_{P_lo} is contained in Q_{P_hi}), so dg_project(hi, lo)
 * returns q_lo.  Used to restart a high-order burst from a low-order state (retraining
 * the forcing of Algorithm 1 during a run).  Both contexts share K, P_lo <= P_hi; q_lo,
 * q_hi: device. */
int dg_prolong(const dg_ctx* lo, const dg_ctx* hi, const double* q_lo, double* q_hi, void* stream);

/* Diagnostics of q (FP64 reductions, deterministic order).  q_ref (device, same
 * layout) may be NULL; when given, e_inf = ||q - q_ref||_inf on the momenta (Eq. 9).
 * forcing (may be NULL) enters dke_dt.  out: HOST.  Returns DG_ERR_NONFINITE (after
 * filling *out) when the state holds NaN or Inf. */
int dg_diagnostics(dg_ctx* ctx, const double* q, const double* q_ref,
                   const nn_model* forcing, dg_diag* out, void* stream);

/* Stable time step dt = cfl h / ((P+1)^2 max(|v| + c)) (Sec. 2.3 gives the CFL
 * condition as a proportionality; this form is the library's reading).  dt_out: HOST. */
int dg_stable_dt(dg_ctx* ctx, const double* q, double cfl, double* dt_out, void* stream);

/* Training pairs of Algorithm 1 (Sec. 2.1):
 *   X[e] = element features of q_bar_n,
 *   Y[e] = element features of (q_bar_np1 - q_nn_np1) / dt   (difference in FP64),
 * for the n_vars variables starting at first_var (5 and 0: all; 3 and 1: momenta,
 * Sec. 2.2).  A feature index is v_slot * n^3 + node.  All three states use the
 * layout of q for context lo.  X, Y: device float arrays of K^3 * n_vars * n^3
 * values (row e = one element), written. */
int dg_make_pairs(const dg_ctx* lo, const double* q_bar_n, const double* q_nn_np1,
                  const double* q_bar_np1, double dt, int first_var, int n_vars,
                  float* X, float* Y, void* stream);

/* Measurement: advances q like dg_rk3_step (nsteps RK3 steps, no forcing) while
 * recording CUDA events on `stream` around every kernel launch.  Returns the summed
 * device time in milliseconds of the phase-A (BR1 gradient) and phase-B (flux, lift,
 * RK update) kernels, the number of launches of each, and the algorithmic bytes one
 * launch of each phase moves, averaged over the three RK stages (state, stage state,
 * stresses and RK increment: each value read or written once; neighbour reads not
 * counted).  All outputs are HOST pointers; any may be NULL.  Synchronises. */
int dg_profile_rk3(dg_ctx* ctx, double* q, double dt, int nsteps, double* ms_gradient,
                   double* ms_flux, int* launches_gradient, int* launches_flux,
                   double* flux_bytes_per_launch, double* gradient_bytes_per_launch,
                   void* stream);

/* Autotuner: times one RK3 step (on a scratch copy of the DEVICE state q; q is not
 * modified) for every elements-per-block value E = 1, 2, 4, ... that fits the block size
 * and shared memory of this P, and for 2 x 2 x 2 cube blocks where allowed (P <= 3, even
 * K, not a batch member), and keeps the fastest for the context.  best_E (HOST, may be
 * NULL) receives its elements per block (8 for cubes; dg_blocking tells the shape),
 * best_ms (HOST, may be NULL) its time per step.  Synchronises. */
int dg_autotune(dg_ctx* ctx, const double* q, double dt, int* best_E, double* best_ms, void* stream);

/* Where dg_rk3_step and dg_advance_host(_async) apply a network forcing (Sec. 2 Eq. 4,
 * Algorithm 1):
 *   DG_FORCING_STAGE (default): s(q_k) is added to the operator at every RK stage state
 *     q_k, i.e. Eq. 4 integrated by the RK3 scheme;
 *   DG_FORCING_POST: Algorithm 1's third loop read literally: s is evaluated once on q^n,
 *     the uncorrected RK3 step is taken, and q^{n+1} += dt s(q^n).
 * The two agree to O(dt^2).  dg_rhs always returns p(q) + s(q).  Returns
 * DG_ERR_INVALID_ARG on a NULL context or an unknown mode. */
enum { DG_FORCING_STAGE = 0, DG_FORCING_POST = 1 };
int dg_set_forcing_mode(dg_ctx* ctx, int mode);

/* The blocking the context's kernels use: elements per block and block shape (0: rows
 * of consecutive elements, 1: 2 x 2 x 2 cubes).  HOST pointers, either may be NULL. */
int dg_blocking(const dg_ctx* ctx, int* elems_per_block, int* block_shape);

/* Self-check of the integer-pipe FP64 <-> FP32 conversions the FP32 operator uses:
 * counts the n DEVICE inputs x where the round-to-nearest-even FP64 -> FP32 conversion
 * differs from the hardware conversion (mismatches[0]; inputs should be zero or within
 * the FP32 normal range, outside of which the library flushes to zero) and where the
 * widening FP32 -> FP64 is not exact (mismatches[1]).  mismatches: HOST, 2 values. */
int dg_check_conversions(const double* x, int64_t n, int64_t* mismatches, void* stream);

/* Self-check of the bounded device-side waits (failure detection without a fault): one
 * block waits on two mbarriers that nothing arrives on, with the operator's bulk-copy wait
 * and the tensor-core kernels' wait.  Both must give up after their limit (about one
 * second) and the kernel must return, leaving the context usable.  Returns DG_OK and the
 * elapsed time in *seconds (HOST, may be NULL); DG_ERR_CUDA if a wait reported success
 * without arrivals or on a CUDA error.  Synchronises the stream. */
int dg_check_bounded_waits(double* seconds, void* stream);

/* ---- Element-layer domain decomposition.  The paper runs its solver in parallel over
 * MPI ranks (Sec. 2.6, implementation details); here the periodic K^3 mesh is split into
 * slabs of whole element layers along z, one per GPU or rank, and each RK stage exchanges
 * the face traces of the slabs' boundary layers twice: the stage state before the BR1
 * gradient phase, the stage state and z-normal viscous fluxes before the flux phase (the
 * interface fluxes of Sec. 3.1 read both sides of a face).  Diagnostics reduce per slab
 * and are combined by dg_diag_combine (a fixed-order FP64 sum; the caller gathers the
 * slabs' dg_diag structs across ranks). ---- */

/* Exchange of one slab's traces, called by the library during dg_rhs, dg_rk3_step,
 * dg_diagnostics and dg_advance_host(_async) on a slab context, once per exchange point,
 * after the pack kernels are enqueued on stream.  send_lo holds the first owned layer's
 * lower-face traces (for the slab below), send_hi the last owned layer's upper-face traces
 * (for the slab above); the function must arrange, in the order of `stream`, that recv_lo
 * receives the lower neighbour's send_hi and recv_hi the upper neighbour's send_lo (the
 * mesh is periodic: slab 0's lower neighbour is the last slab), before the library's unpack
 * kernels that it enqueues on stream after the function returns.  bytes: the size of each
 * of the four DEVICE buffers' contents for this exchange (what: 0 FP64 state, 1 FP32 stage
 * state, 2 stage state and viscous fluxes).  Returns 0, or nonzero for a failure (the
 * library call then returns DG_ERR_EXCHANGE). */
typedef int (*dg_exchange_fn)(void* user, int what, const void* send_lo, const void* send_hi, void* recv_lo,
                              void* recv_hi, size_t bytes, void* stream);

/* Creates the slab of element layers [z_begin, z_begin + z_count) (0 <= z_begin,
 * 1 <= z_count, z_begin + z_count <= K) of the periodic K^3 mesh, with the arguments of
 * dg_create (rows of elements only: block_shape 1 returns DG_ERR_INVALID_ARG).  Its local
 * arrays hold z_count + 2 element layers: local layer 0 is global layer z_begin - 1 (mod K)
 * and local layer z_count + 1 is global layer z_begin + z_count (mod K), the ghost layers
 * whose face traces the exchange fills; local layers 1 .. z_count are the slab's own.
 * Layout of the local state as for q (dg_sizes returns the local counts), element
 * ex + K (ey + K lz).  dg_init_tgv fills every local layer from the global coordinates.
 * The network forcing is not offered on a slab (DG_ERR_UNSUPPORTED). */
int dg_create_part(int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts* opts,
                   int z_begin, int z_count, dg_ctx** out);

/* The slab's global layers and its owned nodes in the local arrays: the owned nodes are
 * [first_owned_node, first_owned_node + owned_nodes) of each variable's row (a whole-mesh
 * context reports 0, K, 0, N).  HOST pointers, any may be NULL. */
int dg_part_layout(const dg_ctx* ctx, int* z_begin, int* z_count, int64_t* first_owned_node,
                   int64_t* owned_nodes);

/* Sets the exchange function of a slab (fn NULL: none; a slab without one can evaluate
 * the operator only if it spans the whole mesh, z_count = K, when it is its own
 * neighbour).  user is passed through. */
int dg_part_set_exchange(dg_ctx* ctx, dg_exchange_fn fn, void* user);

/* Bytes of one side's traces for exchange `what` (0, 1, 2; see dg_exchange_fn).  HOST. */
int dg_part_trace_bytes(const dg_ctx* ctx, int what, size_t* bytes);

/* The slabs of one mesh on the current device, advanced together: parts[0..n) are the
 * slabs in layer order covering 0 .. K-1 (same mesh, order, flow and precision), q[i]
 * (HOST array of DEVICE pointers) slab i's local state.  The traces move between the
 * slabs' buffers by device copies on stream.  dg_group_rk3_step: nsteps RK3 steps as
 * dg_rk3_step; dg_group_rhs: dqdt[i] = p(q)[i] (owned layers written); dg_group_diagnostics:
 * the diagnostics of the whole mesh (HOST out) from the slabs' owned nodes. */
int dg_group_rk3_step(dg_ctx* const* parts, int n, double* const* q, double dt, int nsteps, void* stream);
int dg_group_rhs(dg_ctx* const* parts, int n, double* const* q, double* const* dqdt, void* stream);
int dg_group_diagnostics(dg_ctx* const* parts, int n, double* const* q, dg_diag* out, void* stream);

/* Combines the diagnostics of the n slabs of one mesh (HOST arrays): sums in slab order,
 * maxima of e_inf and max_wave.  On a slab, dg_diagnostics and dg_stable_dt see only its
 * own nodes: the mesh's diagnostics are the combination of all slabs', and its stable
 * step the minimum of the slabs' (dt from the combined max_wave). */
int dg_diag_combine(const dg_diag* parts, int n, dg_diag* out);

const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DGNN_H */
