/*
 * gbr.h -- C ABI of the B300 (sm_103a) library for the per-RK-stage right-hand
 * side of arXiv 2303.10785: MEG6 gradient-based reconstruction with the
 * improved MP limiter, curvilinear HLLC, alpha-damping viscous flux,
 * freestream-preserving conservative metrics and the geometric-conservation
 * term on moving meshes, advanced by SSP-RK3.
 *
 * Conventions (every entry point):
 *  - Plain pointers and sizes only.  Host pointers are borrowed for the call.
 *  - The caller owns the device workspace (any allocator, e.g. a torch tensor);
 *    the context keeps using it until gbr_destroy.  The library itself calls no
 *    device allocator.  gbr_workspace_bytes gives the exact size.
 *  - Work is enqueued on the caller's CUDA stream passed to gbr_create.
 *  - No exception or abort crosses the ABI: every call returns a gbr_status.
 *    Errors detected on the device (non-finite state, non-positive density) are
 *    sticky and surface at gbr_sync.
 *  - Not thread-safe per context; independent contexts are independent.
 *
 * Array layouts (doubles, C order, i fastest):
 *  nodes    [ndim][Nk][Nj][Ni] with N_d = n_d + 1 on a periodic axis (node n_d
 *           closes the period: node(n_d) = node(0) + constant period vector) and
 *           N_d = n_d + 1 + 2*ghost_nodes on a non-periodic axis (ghost node
 *           layers first).  2D: [2][Nj][Ni].
 *  state    [nv][nk][nj][ni], nv = ndim + 2, conserved (rho, rho u.., E).
 *  faces    direction d: [..][n with n_d -> n_d + 1]; face index f = 0..n_d is the
 *           interface i+1/2 with i = f - 1.
 */
#ifndef GBR_H
#define GBR_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBR_ABI_VERSION 4

typedef struct gbr_ctx gbr_ctx;

typedef enum {
  GBR_OK = 0,
  GBR_EINVAL = 1,      /* invalid argument (message in gbr_last_error / gbr_last_global_error) */
  GBR_ENOMEM = 2,      /* workspace smaller than gbr_workspace_bytes */
  GBR_ECUDA = 3,       /* a CUDA runtime call failed */
  GBR_ENONFINITE = 4,  /* the device saw a non-finite state or non-positive density */
  GBR_ETIMEOUT = 5,    /* gbr_sync deadline passed before the stream drained */
  GBR_ESTATE = 6       /* call out of order (e.g. stepping before metrics) */
} gbr_status;

/* Non-periodic sides: zero-gradient ghosts; Dirichlet inflow (x-low side only, gbr_set_inflow);
 * slip wall: ghost layer g mirrors cell g - 1, density and pressure as they are, the velocity
 * reflected about the unit normal of the wall interface (the paper's boundary-condition table
 * is an image missing from its text; this is the standard reflecting wall). */
enum { GBR_BC_ZEROGRAD = 1, GBR_BC_INFLOW = 2, GBR_BC_WALL = 3 };

/* Arithmetic of the right-hand side (gbr_params.precision):
 * GBR_PREC_FP64:  every step in FP64 (the paper's path).
 * GBR_PREC_MIXED: primitives, gradients, characteristic reconstruction, limiter,
 *                 HLLC and viscous fluxes computed and stored in FP32; the conserved
 *                 state, the metrics and 1/J, the GCL term, the flux divergence and
 *                 the RK accumulation in FP64.  Not in the paper (which compares FP32
 *                 and FP64 runs only as a whole).  The FP32 primitives hold p - p_ref,
 *                 p_ref the pressure of cell 0 of the state last given to gbr_set_state
 *                 (any constant gives the same scheme; one near the mean pressure keeps
 *                 the round-off independent of the Mach number). */
enum { GBR_PREC_FP64 = 0, GBR_PREC_MIXED = 1 };

/* Gradients of the primitives (gbr_params.gradient_scheme), Sec. 5.1 step 1:
 * GBR_GRAD_MEG6: explicit sixth-order E6 (Eq. E6_grads).
 * GBR_GRAD_MIG4: implicit fourth-order IG4 (Eq. IG4_grads, alpha = 5/14): one
 *                tridiagonal solve per grid line -- cyclic on periodic axes; on
 *                open axes over the padded line, whose three end points at each
 *                side take explicit rows (second-order one-sided, fourth-order
 *                biased, fourth-order central).  The metric derivative and
 *                interpolation of Sec. 7 use IG4 as well (step 2: the scheme's own
 *                gradients): one solve per geometry line with the same end rows, on
 *                periodic axes over the unwrapped line extended 64 cells beyond each
 *                side (IG4 on the unbounded line to round-off); wall-bounded axes
 *                without ghost nodes keep the App. C operators.
 *                Not available in gbr_rhs_static. */
enum { GBR_GRAD_MEG6 = 0, GBR_GRAD_MIG4 = 1 };

typedef struct {
  int ndim;            /* 2 or 3 */
  int n[3];            /* cells per axis, 1 .. 2^24 (n[2] = 1 in 2D) */
  int periodic[3];     /* 1 = periodic axis */
  int ghost_nodes;     /* node layers supplied beyond each non-periodic side (10 .. 1024), or 0: the
                          non-periodic axes end at the grid's last nodes and their metrics near
                          the ends take the one-sided formulas of App. C (>= 12 cells; static
                          meshes only) */
  int bc[3][2];        /* non-periodic sides: GBR_BC_ZEROGRAD, GBR_BC_WALL, or GBR_BC_INFLOW on
                          the x-low side */
  double gamma;        /* ratio of specific heats (Sec. 2: 1.4) */
  double prandtl;      /* Sec. 2: 0.71 */
  double reynolds;     /* <= 0: Euler, no viscous flux; mu_ref = 1/reynolds */
  double sutherland_s; /* S / T_ref of Sutherland's law; <= 0: constant viscosity */
  double t_ref;        /* Sutherland reference temperature in T = p/rho units */
  double alpha_damping;/* alpha^D of Eq. (AD-eqn1), paper value 4 */
  double mp_alpha, mp_beta, mp_eps; /* App. E limiter constants (4, 4, 1e-20) */
  int moving;          /* 1: reserve grid-velocity, time-metric and GCL storage */
  int precision;       /* GBR_PREC_FP64 or GBR_PREC_MIXED */
  int gradient_scheme; /* GBR_GRAD_MEG6 or GBR_GRAD_MIG4 */
} gbr_params;

/* Prescribed sinusoidal node motion (Sec. 8.2 families):
 * x_a(m, t) = origin_a + m_a h_a + amp_a sin(2 pi omega t) prod_b S_ab(m_b h_b),
 * S_ab(s) = sin(k_ab s) if k_ab != 0 else 1;  velocities are the analytic
 * time derivative.  m is the (unwrapped) node index. */
typedef struct {
  double origin[3], h[3], amp[3], omega, k[3][3];
} gbr_motion;

/* Field identifiers for gbr_get_field (read-back of intermediate results). */
enum {
  GBR_FIELD_CELL_METRICS = 0, /* [nd][nd][cells] hat metrics (Eq. GCL_metrics) */
  GBR_FIELD_CELL_DET = 1,     /* [cells] 1/J (Eq. Jac-matrix) */
  GBR_FIELD_CELL_TIME = 2,    /* [nd][cells] hat time metrics */
  GBR_FIELD_FACE_HAT = 3,     /* [nd][faces of dir] interface hat metrics (Eq. interp-formulae) */
  GBR_FIELD_FACE_UNHAT = 4,   /* [nd][nd][faces of dir] interface unhatted metrics (viscous) */
  GBR_FIELD_FACE_TIME = 5,    /* [faces of dir] interface hat time metric */
  GBR_FIELD_GCL = 6,          /* [cells] (1/J)_t (Eq. Jacb2) */
  GBR_FIELD_FACE_FLUX = 7     /* [nv][faces of dir] F^ - F^v of the last right-hand side */
};

/* Exact device workspace size for these parameters; 0 if they are invalid. */
size_t gbr_workspace_bytes(const gbr_params* p);

/* Create a context on `d_workspace` (>= gbr_workspace_bytes) and upload the
 * node coordinates (and, if given, node velocities) -- Sec. 3: the solution
 * lives at the centroid of each cell's vertices.  stream: a cudaStream_t or
 * NULL for the legacy default stream.  Errors: EINVAL (bad params or periodic
 * closure), ENOMEM (workspace too small), ECUDA. */
gbr_status gbr_create(const gbr_params* p, const double* nodes, const double* node_vel, void* d_workspace,
                      size_t ws_bytes, void* stream, gbr_ctx** out);

/* Sec. 4 + Sec. 7: conservative metrics with the MEG6 interface derivative,
 * the Jacobian, their interface interpolation, and for a moving mesh the time
 * metrics xi_t = -(x_t xi_x + ...) and (1/J)_t of Eq. (Jacb2). */
gbr_status gbr_compute_metrics(gbr_ctx* c);

/* Replace the node coordinates (and velocities) and recompute all metrics
 * (Sec. 4: recomputed after each change of a dynamic mesh).  Host arrays. */
gbr_status gbr_move_mesh(gbr_ctx* c, const double* nodes, const double* node_vel);

/* Prescribe an analytic motion evaluated on the device; gbr_rk_step then
 * recomputes the geometry at every stage time t, t+dt, t+dt/2.
 * Sets the solution time to t0 and computes the metrics at t0. */
gbr_status gbr_set_motion(gbr_ctx* c, const gbr_motion* m, double t0);

/* Conserved state in/out; on_device = 1: q is a device pointer.  On a
 * GBR_PREC_MIXED context gbr_set_state also sets the pressure offset p_ref of
 * the FP32 primitives from cell 0 (0 if that pressure is not finite). */
gbr_status gbr_set_state(gbr_ctx* c, const double* q, int on_device);
gbr_status gbr_get_state(gbr_ctx* c, double* q, int on_device);

/* Pipelined host transfers of the conserved state (no counterpart in the paper;
 * a calling convention for loops fed from host memory, e.g. one problem per
 * step).  Both return at once.  gbr_set_state_async uploads host_q into the
 * caller-owned device buffer d_stage on a copy stream of the context, and the
 * context's stream takes it as the state at this point of its order (work
 * enqueued before the call still sees the old state, work after it the new
 * one); gbr_get_state_async snapshots the state at this point of the stream
 * order into d_stage and downloads it to host_q on a second copy stream.  So
 * the upload of the next state and the download of the last one overlap the
 * steps in between.  On a GBR_PREC_MIXED context gbr_set_state_async sets
 * p_ref from cell 0 of host_q as gbr_set_state does.
 *  host_q: page-locked host memory (cudaHostAlloc / cudaHostRegister), [nv][cells]
 *          doubles; set: read up to the next gbr_sync (keep it unchanged until
 *          then), get: written by the time gbr_sync returns.
 *  d_stage: device buffer of nv*cells doubles owned by the caller, one for the
 *          uploads and another for the downloads, each reused across calls and
 *          not touched by the caller until gbr_sync.
 * Errors: EINVAL for a null argument or host memory that is not page-locked. */
gbr_status gbr_set_state_async(gbr_ctx* c, const double* host_q, double* d_stage);
gbr_status gbr_get_state_async(gbr_ctx* c, double* host_q, double* d_stage);

/* Jet-type boundary data: x-low inflow primitives [nv][nk][nj]
 * imposed in the x-low ghost cells of every following stage, and a sponge source
 * -sigma (Q - q_amb) with sigma per cell (host, NULL removes it).
 * gbr_set_inflow: on_device = 0: prim is host memory, copied before the call
 * returns; on_device = 1: prim is device memory, copied in stream order on the
 * context's stream (the caller keeps it alive until that copy has run), so a
 * time-dependent inflow can be changed between steps without a host round trip. */
gbr_status gbr_set_inflow(gbr_ctx* c, const double* prim, int on_device);
gbr_status gbr_set_sponge(gbr_ctx* c, const double* sigma, const double* q_amb);

/* dQ/dt = L(Q) = J (Res - (1/J)_t Q) [+ sponge] of the current state (Sec. 3,
 * Sec. 4 time split, Sec. 5).  dqdt: device array [nv][cells]. */
gbr_status gbr_rhs(gbr_ctx* c, double* dqdt);

/* App. B CFL time step of the current state; kept on the device.  dt_out:
 * host pointer (the call then waits for the result) or NULL. */
gbr_status gbr_compute_dt(gbr_ctx* c, double cfl, double* dt_out);

/* One SSP-RK3 step (App. B).  cfl_or_neg_dt > 0: CFL number (dt computed on
 * the device from the state at t^n); < 0: fixed dt = -cfl_or_neg_dt.  Moves
 * the mesh per stage when a motion is set.  Asynchronous. */
gbr_status gbr_rk_step(gbr_ctx* c, double cfl_or_neg_dt);

/* Wait for the stream and the copy streams of the pipelined transfers (polling,
 * up to timeout_s seconds; <= 0: no limit), then
 * report sticky device errors: ENONFINITE, or ETIMEOUT when a kernel's bounded
 * wait for a tile copy into shared memory ran out (the MIG4 line solves).
 * ETIMEOUT also when the stream did not drain before the deadline. */
gbr_status gbr_sync(gbr_ctx* c, double timeout_s);

/* Solution time and the last time step (waits for the stream). */
gbr_status gbr_get_time(gbr_ctx* c, double* t, double* dt);

/* Copy an intermediate field to a host array (see GBR_FIELD_*); dir selects the
 * face direction for face fields.  Waits for the stream. */
gbr_status gbr_get_field(gbr_ctx* c, int which, int dir, double* host_out);

/* Measurement hook (no counterpart in the paper): waits for the stream,
 * returns the summed CUDA-event time of the face-flux launches recorded since
 * the previous call (face_ms), their count, and the number of kernels the
 * context launched, then resets the tallies.  enable = 1 records events around
 * every face-flux launch from now on; 0 stops recording.  Out pointers may be NULL. */
gbr_status gbr_profile(gbr_ctx* c, int enable, double* face_ms, long long* face_launches, long long* launches);

/* Measurement hook (no counterpart in the paper): fused multiply-add throughput
 * of the current device in TFLOP/s (2 flops per FMA) -- FP64 for precision =
 * GBR_PREC_FP64, FP32 for GBR_PREC_MIXED -- the denominator of the arithmetic
 * roofline of the kernels, measured where they run.  One wave of resident
 * blocks, each thread running 8 independent FMA chains; the shortest of three
 * launches after a warm-up, timed with CUDA events on `stream` (a
 * cudaStream_t or NULL).  Synchronous.  tflops, ms (the timed launch's
 * duration): out pointers, may be NULL.  Errors: EINVAL (precision), ECUDA. */
gbr_status gbr_alu_peak(int precision, void* stream, double* tflops, double* ms);

/* Self-check of the FP64 reciprocal the kernels use in place of divisions (no
 * counterpart in the paper): Newton's method for 1/x from the hardware's
 * approximate reciprocal, meant to lie within one unit in the last place of the
 * correctly rounded 1/x for finite, nonzero, normal x whose reciprocal is normal.
 * Runs n such x on the device (SplitMix64 bit patterns of seed + index: random
 * sign and mantissa, biased exponent 23 .. 2023) and returns in *max_ulp the
 * largest distance, in units in the last place, between that reciprocal and the
 * FP64 division 1.0 / x.  Synchronous on `stream` (a cudaStream_t or NULL); no
 * allocation (one file-scope device counter, so concurrent calls share it).
 * Errors: EINVAL (n outside 1 .. 2^34, null max_ulp), ECUDA. */
gbr_status gbr_check_rcp(long long n, unsigned long long seed, void* stream, long long* max_ulp);

/* Self-check of the kernels' bounded waits (no counterpart in the paper).  The
 * MIG4 line solves wait for a TMA tile copy on an mbarrier with a bounded
 * number of polls; when they run out the block sets a sticky device flag and
 * leaves.  This call runs that timeout path on purpose: one block waits, for
 * `polls` polls (1 .. 65536, each suspending for at most about 1 us), on an
 * mbarrier that nothing completes.  Asynchronous; the next gbr_sync returns
 * GBR_ETIMEOUT, and the context stays usable (the flag stays set).
 * Errors: EINVAL for a null context or polls out of range. */
gbr_status gbr_check_bounded_wait(gbr_ctx* c, int polls);

/* Right-hand side with no device allocation anywhere (the paper has no
 * counterpart; this is a calling convention).  For callers that cannot call
 * cudaMalloc or own a workspace -- code running inside another framework's
 * memory pool or under a fixed device-memory budget, or code that must not
 * allocate after start-up.  Computes the metrics of `nodes` (and, with
 * node_vel and params.moving = 1, the time metrics and (1/J)_t) and writes
 * dqdt = L(q) exactly as gbr_create + gbr_compute_metrics + gbr_set_state +
 * gbr_rhs would.
 *  nodes, node_vel: host arrays as for gbr_create; q, dqdt: device arrays
 *  [nv][cells]; stream: cudaStream_t or NULL; msg/msg_len: optional
 *  caller buffer for an error message (no allocation).
 * All scratch lives in one file-scope device array of 64 MiB that every GPU
 * loading this library holds until the process exits; grids whose scratch
 * would exceed it are rejected with GBR_EINVAL before any device work.  Only
 * periodic and zero-gradient sides are accepted (no inflow data, no sponge),
 * and only params.precision = GBR_PREC_FP64.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Calls share the array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Asynchronous on `stream` after the host-to-device copy of the nodes.
 * Unlike gbr_sync, this call does not report a non-finite result or a
 * non-positive density (GBR_ENONFINITE): the device flag for them lives in the
 * shared array and is never read back, so a caller who needs that check must
 * test dqdt itself.  GBR_OK means that the work was enqueued. */
gbr_status gbr_rhs_static(const gbr_params* p, const double* nodes, const double* node_vel, const double* q,
                          double* dqdt, void* stream, char* msg, size_t msg_len);

/* ---------------------------------------------------------------------------
 * Batched stepping (not in the paper, whose solver runs one job per GPU).
 * A batch advances many contexts together: per kind of member (ndim, viscous,
 * precision, moving mesh, gradient scheme) every phase of an SSP-RK3 step is one
 * launch over a block -> (member, tile) work list, and the whole step (time steps
 * on the device, three stages, time advance) is captured as one CUDA graph,
 * replayed until the membership changes.  Members with a prescribed motion
 * (gbr_set_motion) recompute their geometry at every stage time with their own
 * launches, and MIG4 members solve their gradient lines with their own launches,
 * inside the same step.  Each member keeps its own state, metrics, time step and
 * error flag; its results are bitwise those of gbr_rk_step on it alone.  Members
 * must be contexts created on the batch's stream; while a member, a context is
 * advanced only through the batch (other calls on it stay in stream order).  Device tables live in a caller-owned workspace of
 * gbr_batch_workspace_bytes(max_members) bytes (256-byte aligned).
 * Not thread-safe per batch. */
typedef struct gbr_batch gbr_batch;

size_t gbr_batch_workspace_bytes(int max_members);
gbr_status gbr_batch_create(int max_members, void* d_workspace, size_t ws_bytes, void* stream, gbr_batch** out);
/* use_graph: capture and replay each step as a CUDA graph (default 1); autotune
 * (0: the phase kernels, 128 interfaces per tile; 2: the fused stage kernel for
 * every kind without per-member work, untimed; 1, the default:
 * per kind and size class (log2 of the kind's cells), time the candidates on the
 * live members' right-hand side and keep the fastest (default 1; the members'
 * states are not changed): the phase kernels with 64, 128 or 256 interfaces per
 * tile, and, for kinds without per-member work (static MEG6 members), the fused
 * stage kernel -- every phase of a stage in one persistent cooperative launch,
 * separated by grid-wide barriers (bounded waits: a barrier that does not
 * complete sets a sticky flag, and gbr_batch_sync returns GBR_ETIMEOUT from then
 * on); each with the
 * gradient sweep in two passes or one fused pass (FP64 kinds)).  EINVAL for
 * another autotune value. */
gbr_status gbr_batch_set_options(gbr_batch* b, int use_graph, int autotune);
/* cfl_or_neg_dt as for gbr_rk_step: > 0 CFL number, < 0 fixed step. */
gbr_status gbr_batch_add(gbr_batch* b, gbr_ctx* c, double cfl_or_neg_dt);
gbr_status gbr_batch_remove(gbr_batch* b, gbr_ctx* c);
/* Queue n_steps SSP-RK3 steps of every member (asynchronous; rebuilds the
 * tables, tuning and graph first when the membership changed). */
gbr_status gbr_batch_step(gbr_batch* b, int n_steps);
/* Drain the stream (GBR_ETIMEOUT after timeout_s > 0), check the fused stage
 * kernels' barrier flags (GBR_ETIMEOUT) and every member's error flag:
 * GBR_ENONFINITE names the first bad member (*bad_member, or -1). */
gbr_status gbr_batch_sync(gbr_batch* b, double timeout_s, int* bad_member);
/* Members, kinds, kernel launches per step and launches issued so far.  Without
 * graphs, a batch with moving-mesh or MIG4 members reports -1 launches per step
 * until its first step has been enqueued. */
gbr_status gbr_batch_info(gbr_batch* b, int* members, int* kinds, long long* launches_per_step, long long* launches);
/* The chosen tuning of kind `kind` (0 .. kinds-1): interfaces per tile, fused
 * gradient sweep (0/1), fused stage kernel (0/1). */
gbr_status gbr_batch_tuning(gbr_batch* b, int kind, int* nd, int* viscous, int* precision, int* face_block,
                            int* fused_grad, int* fused_stage);
/* Self-check of the fused stage kernel's bounded grid barrier (no counterpart in
 * the paper): one block waits, for `polls` polls (1 .. 2^22, each sleeping about
 * 200 ns), at a barrier that no arrival completes, then sets the sticky timeout
 * flag of the batch's first kind: the next gbr_batch_sync returns GBR_ETIMEOUT.
 * Asynchronous.  Errors: EINVAL (null batch, polls out of range), ESTATE (no
 * members). */
gbr_status gbr_batch_check_barrier(gbr_batch* b, int polls);
const char* gbr_batch_last_error(const gbr_batch* b);
void gbr_batch_destroy(gbr_batch* b);

/* Device-memory arena for admitting jobs by HBM footprint (not in the paper):
 * host bookkeeping of a caller-owned, 256-byte aligned device range; first fit
 * in address order, 256-byte granules, free neighbours merged.  No device
 * access.  gbr_arena_alloc returns GBR_ENOMEM when no free range is large
 * enough (the caller keeps the job queued).  Not thread-safe. */
typedef struct gbr_arena gbr_arena;
gbr_status gbr_arena_create(void* d_base, size_t bytes, gbr_arena** out);
gbr_status gbr_arena_alloc(gbr_arena* a, size_t bytes, void** ptr);
gbr_status gbr_arena_free(gbr_arena* a, void* ptr);
gbr_status gbr_arena_stats(const gbr_arena* a, size_t* used, size_t* free_total, size_t* largest_free, int* blocks);
void gbr_arena_destroy(gbr_arena* a);

const char* gbr_last_error(const gbr_ctx* c);
const char* gbr_last_global_error(void);
void gbr_destroy(gbr_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
