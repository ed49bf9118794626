/*
 * sbp.h - C ABI of the GB300 upwind-SBP elastic wave library.
 *
 * The library evaluates the semi-discrete velocity-stress elastic wave
 * equation on one boundary-conforming curvilinear block (Duru, Fung &
 * Williams, arXiv 2011.02600):
 *
 *   P~^-1 dQ/dt = sum_xi D-_xi F_xi(Q) + sum_xi B_xi(D+_xi Q) + sum SAT     (Sections 4.2, 5)
 *
 * with the upwind SBP pair (H, D-, D+) of interior order 2 to 7 along q, r
 * and s (Section 4.1, Table 1) or a traditional central SBP operator (Table 2),
 * metric terms e_xi = J grad(xi) (Section 2.2),
 * the free-surface penalty (Eq. SAT_free_surface) or the general penalty with
 * parameter gamma (Eq. SAT_General) on each face, fused with the stages of the
 * five-stage 2N-storage fourth-order Runge-Kutta scheme the paper uses
 * (Carpenter & Kennedy 1994, cited in Sections 1 and 7).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Nodes: nq x nr x ns (n_xi + 1 per axis), reference coordinates xi_i = i/(N-1).
 * Layout: a "field" is one scalar grid function stored [s][r][q] with q
 *   contiguous, row pitch ldq elements (ldq >= nq, rows start on 128-byte
 *   boundaries) and field stride fs elements (sbp_layout).  Element (i,j,k) of
 *   field f of a buffer is at  base + f*fs + k*ldq*nr + j*ldq + i.
 *   Padding elements are never read as data and may hold anything.
 * State Q: 9 fields (vx, vy, vz, sxx, syy, szz, sxy, sxz, syz) (Section 2.1).
 * Metrics (solver precision): 9 fields a[xi][eta] = J xi_eta, xi in (q,r,s),
 *   eta in (x,y,z), stored in the order a_qx a_qy a_qz a_rx ... a_sz.
 * Coefficients (solver precision): 3 fields 1/(rho J), lambda/J, mu/J.
 * Faces: 0..5 = (q=0, q=1, r=0, r=1, s=0, s=1).
 * Precision: 32 (float) or 64 (double) for the state, metrics and
 *   coefficients; setup inputs are always double.
 * Memory ownership: every buffer passed in is owned by the caller; the library
 *   never frees it.  Device buffers must stay valid while a grid uses them.
 *   The library allocates only small internal buffers (reduction partials,
 *   source weights, receiver indices, a status word), freed by sbp_destroy.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   are asynchronous unless stated; they return after enqueueing work.
 * Errors: every function returns SBP_OK (0) or a positive code; the message of
 *   the last failure on the calling thread is in sbp_last_error().  Invalid
 *   arguments are rejected on the host before any work is enqueued.  No kernel
 *   traps or asserts; device-side problems (non-finite state, non-positive
 *   Jacobian or moduli) are recorded in a status word read by sbp_status.
 */
#ifndef SBP_GB300_H
#define SBP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBP_OK 0
#define SBP_ERR_ARG 1          /* invalid argument (sizes, order, precision, pointers) */
#define SBP_ERR_UNSUPPORTED 2  /* valid request the library does not implement */
#define SBP_ERR_CUDA 3         /* a CUDA runtime call failed */
#define SBP_ERR_NONFINITE 4    /* the state or a reduction is NaN/Inf */
#define SBP_ERR_STATE 5        /* call out of sequence (e.g. stepping before sbp_bind) */
#define SBP_ERR_MESH 6         /* non-positive Jacobian or invalid moduli found on the device */

/* Operator codes (SbpGridDesc.order): 2..7 are the upwind dual pairs of Table 1
 * (Section 4.1, Eq. upw_SBP), even and odd orders; SBP_TRADITIONAL + 2, 4, 6 are
 * the traditional central SBP operators of Table 2, applied in place of both D-
 * and D+ (Section 6.2 compares them with the upwind pairs; Section 7.2 runs them
 * on topography).  The adjoint entry points accept the codes 2, 4 and 6. */
#define SBP_TRADITIONAL 100

#define SBP_BC_FREE 0  /* free surface, Eq. SAT_free_surface */
#define SBP_BC_CHAR 1  /* general condition with gamma, Eq. BC_General2 / Eq. SAT_General */
#define SBP_BC_INTERFACE 2  /* shared face with another block (sbp_set_interface) */

/* Status bits reported by sbp_status (device-side findings). */
#define SBP_STATUS_NONFINITE 1u
#define SBP_STATUS_BAD_MESH 2u
#define SBP_STATUS_BAD_MATERIAL 4u
#define SBP_STATUS_TIMEOUT 8u      /* an asynchronous tile copy did not complete in time */

typedef struct SbpGridDesc {
  int32_t nq, nr, ns;     /* nodes per axis; each >= sbp_min_nodes(order) */
  int32_t order;          /* operator code: upwind order 2..7, or SBP_TRADITIONAL + 2, 4, 6 */
  int32_t precision;      /* 32 or 64 */
  int32_t bc_kind[6];     /* SBP_BC_FREE, SBP_BC_CHAR or SBP_BC_INTERFACE per face */
  double bc_gamma[6];     /* gamma in [-1, 1] for SBP_BC_CHAR faces (Eq. BC_General2) */
} SbpGridDesc;

typedef struct SbpGrid SbpGrid;

/* Moment-tensor point source (Section 7.1, Eq. momententor_pointsource): the
 * stress rates receive -M g(t) delta_h, delta_h = phi_q phi_r phi_s /(J H)
 * with 1D weights on order+2 nodes satisfying the discrete moment conditions
 * up to degree order+1.  stf: 0 = Ricker (f0, t0), 1 = t/T^2 exp(-t/T) (T). */
typedef struct SbpSource {
  double ref[3];          /* reference coordinates (q, r, s) in [0,1] of the source */
  double moment[6];       /* Mxx, Myy, Mzz, Mxy, Mxz, Myz (N m) */
  int32_t stf;            /* 0 Ricker, 1 LOH1-type */
  double f0, t0, T;       /* Ricker peak frequency and delay; LOH1 time constant */
} SbpSource;

/* Smallest node count per axis for an operator code: 2b + max(r, q) (b closure
 * rows, interior stencil reach r and q), for a traditional operator at least that
 * of the upwind pair of the same order, whose D_c forms the metric terms.  ARG for
 * an unknown code. */
int sbp_min_nodes(int32_t order, int32_t* out);

/* Validate desc and create a grid handle (host memory only).  ARG on bad sizes,
 * order, precision, face kinds or gamma outside [-1, 1]. */
int sbp_create_grid(const SbpGridDesc* desc, SbpGrid** out);

/* Free the handle and the library's internal buffers (not the caller's). */
int sbp_destroy(SbpGrid* grid);

/* Layout of every field of this grid: row pitch ldq and field stride fs in
 * elements, and the element size in bytes of the solver precision. */
int sbp_layout(const SbpGrid* grid, int64_t* ldq, int64_t* fs, int64_t* elem_bytes);

/* Number of independent states B advanced together (the batched solver: many
 * sources on one mesh and medium).  All B states share the metrics and
 * coefficients; every stage kernel processes the B states in one launch.
 * Call before sbp_bind; default 1.  B in 1..1024. */
int sbp_set_batch(SbpGrid* grid, int32_t nb);

/* Make the grid one slab of a block decomposed along s (the multi-device layout:
 * each device owns a range of s-planes; prior art is the paper's MPI ghost-node
 * exchange, Section 7.2).  The grid's ns (SbpGridDesc, at least sbp_min_nodes
 * like every axis) counts its local planes:
 * ghost_lo ghost planes, the owned planes, ghost_hi ghost planes; local plane k
 * is plane k + k_offset of the block of ns_global planes.  A ghost count of 0
 * marks a face of the block (k_offset = 0 at the low face, k_offset + ns =
 * ns_global at the high face); otherwise it must be at least the interior
 * stencil's reach max(r, q).  The stages compute the owned planes only, with the
 * block's spacing and with closures and penalties at the block's faces alone, so
 * that, with the ghost planes of the state filled from the neighbours before
 * every stage (the caller's halo exchange), the owned planes evolve exactly as in
 * the undivided block.  sbp_energy sums the owned planes with the block's
 * weights, and sbp_metrics fills the owned planes of jmet with the block's
 * metrics (the block's spacing and closures, the coordinates of the ghost planes
 * as stencil taps); jmet given to sbp_set_material must hold the block's metrics
 * at every local plane, ghost planes included, e.g. from sbp_metrics on a slab
 * grid whose owned planes are these local planes.  Point sources, the adjoint and
 * the general kernel path return UNSUPPORTED on slab grids.  Call before
 * sbp_bind; ghost_lo = ghost_hi = 0 restores the whole block. */
int sbp_set_slab(SbpGrid* grid, int32_t ns_global, int32_t k_offset, int32_t ghost_lo, int32_t ghost_hi);

/* Bind the caller's device buffers (solver precision, layout of sbp_layout):
 * q0, q1: 9 B fields each (ping-pong state; state b occupies fields 9b..9b+8;
 * q0 holds the states after binding), dq: 9 B fields (Runge-Kutta register),
 * met: 9 fields, mat: 3 fields (shared by the B states).
 * Pointers must be 256-byte aligned and distinct.  Allocates the library's
 * internal buffers on the current device. */
int sbp_bind(SbpGrid* grid, void* q0, void* q1, void* dq, void* met, void* mat);

/* Section 2.2: from node coordinates xyz (3 FP64 fields x, y, z; device)
 * compute J and a[xi][eta] = J xi_eta (Cramer's rule, derivatives with
 * D_c = (D+ + D-)/2 of the upwind pair of the grid's order, also for the
 * traditional operators) into jmet (10 FP64 fields: J, then
 * the 9 metrics; device, caller-owned).  Flags SBP_STATUS_BAD_MESH where J <= 0.
 * On a slab grid every inner end needs at least the reach of that D_c in ghost
 * planes (for the traditional operators one more than sbp_set_slab asks):
 * SBP_ERR_ARG otherwise. */
int sbp_metrics(SbpGrid* grid, const double* xyz, double* jmet, void* stream);

/* Fill the bound met (a[xi][eta] cast to the solver precision) and mat
 * (1/(rho J), lambda/J, mu/J) from jmet (as produced by sbp_metrics) and rlm
 * (3 FP64 fields rho, lambda, mu; device).  Flags SBP_STATUS_BAD_MATERIAL where
 * rho <= 0, mu <= 0 or lambda + 2 mu <= 0.  Also finds whether the metrics are
 * those of a topography map x = L_x q, y = L_y r, z = z(q, r, s) (the configs'
 * layered and topographic grids): then a_q = (a_q,x, 0, 0) and a_r =
 * (0, c a_q,x, 0) with the constant c = L_x / L_y at every node, to 1e-11
 * relative (the vanishing components are rounding noise of D_c on the linear
 * x and y), and the tiled forward stage of the upwind orders 2, 4, 6 reads 4
 * metric fields (a_q,x, a_s) instead of 9 (sbp_map_path).  Synchronises the
 * stream.  Needs sbp_bind. */
int sbp_set_material(SbpGrid* grid, const double* jmet, const double* rlm, void* stream);

/* Metric path of the tiled forward stage (not part of the paper: its method is
 * the same on either path; the topography path only skips the metric components
 * that vanish).  SBP_MAP_AUTO (default): the topography path where
 * sbp_set_material found a topography map; SBP_MAP_GENERAL: always all nine
 * metric components.  May be called at any time; the next stage uses it. */
#define SBP_MAP_AUTO 0
#define SBP_MAP_GENERAL 1
#define SBP_MAP_TOPOGRAPHY 2
int sbp_set_map_path(SbpGrid* grid, int32_t path);

/* The metric path the tiled forward stage uses now: SBP_MAP_TOPOGRAPHY or
 * SBP_MAP_GENERAL (before sbp_set_material, on the general kernel path, for the
 * orders without a topography variant, or after SBP_MAP_GENERAL). */
int sbp_map_path(SbpGrid* grid, int32_t* path);

/* dQ/dt of the semi-discrete scheme with penalties (Eq.
 * gen_hyp_transformed_discrete_SAT multiplied by P~) for the state q (9 fields,
 * device) into out (9 fields, device); no time stepping, no source.  Needs
 * sbp_bind and sbp_set_material. */
int sbp_rhs(SbpGrid* grid, const void* q, void* out, void* stream);

/* One fused Runge-Kutta stage k in 0..4 on the bound buffers:
 * dq <- A_k dq + dt L(q_cur), q_next <- q_cur + B_k dq, then q_next becomes
 * current.  The source (if set) is evaluated at t + c_k dt.  Does not advance t. */
int sbp_rk_stage(SbpGrid* grid, int32_t stage, double dt, void* stream);

/* n full steps of size dt (five fused stages each), source at the stage times,
 * receivers recorded after each step; advances the grid time by n dt. */
int sbp_step_n(SbpGrid* grid, int32_t n, double dt, void* stream);

/* Kernel path for the stage: 0 (default) = the tiled kernel over every node
 * (shared-memory tiles by TMA; closure rows and face penalties included);
 * 1 = the general one-thread-per-node kernel over every node.  Both compute
 * the same scheme; path 1 exists to cross-check the tiled kernel. */
int sbp_set_kernel_path(SbpGrid* grid, int32_t path);

/* Per-kernel timing: when enabled, each stage-kernel launch is bracketed by
 * CUDA events recorded on the launching stream.  sbp_kernel_times waits for
 * the recorded events, returns the summed milliseconds and launch counts per
 * kernel kind (arrays of 3: index 0 the tiled stage kernel, 1 the general
 * stage kernel, 2 one adjoint stage, its two kernels together) since the
 * previous call, and clears them. */
int sbp_kernel_timing(SbpGrid* grid, int32_t enable);
int sbp_kernel_times(SbpGrid* grid, double* ms, int64_t* launches);

/* Which bound state buffer holds the current state: 0 (q0) or 1 (q1). */
int sbp_current(const SbpGrid* grid, int32_t* which);

/* Set / get the simulation time and the step counter (receivers record at
 * column step).  SBP_ERR_ARG for a negative step or a non-finite time. */
int sbp_set_time(SbpGrid* grid, double t, int64_t step);
int sbp_get_time(const SbpGrid* grid, double* t, int64_t* step);

/* Discrete energy E = 1/2 <Q, P~^-1 Q>_H (Eq. physical_energy_discrete with the
 * Jacobian weight) of the current state, accumulated in FP64.  Synchronises the
 * stream; NONFINITE if E is not finite. */
int sbp_energy(SbpGrid* grid, double* out, void* stream);

/* Place a point source in state 0 (replaces any previous sources).  jmet as
 * for sbp_set_material (J is read at the source's nodes). */
int sbp_set_source(SbpGrid* grid, const SbpSource* src, const double* jmet, void* stream);

/* One point source per state: srcs[b] acts on state b (n <= B).  The sources of
 * one batch share their time function (stf, f0, t0, T); UNSUPPORTED otherwise. */
int sbp_set_sources(SbpGrid* grid, int32_t n, const SbpSource* srcs, const double* jmet, void* stream);

/* Receivers (the stations of Section 7: particle velocity at surface nodes):
 * n nodes (at most 65535) given by host int32 (i, j, k) triples; traces is a
 * device buffer of B*n*3*n_t elements of the solver precision,
 * trace[b][r][c][step] (velocity component c of receiver r in state b after
 * step `step`); steps beyond n_t are not recorded.  traces = NULL makes the
 * library allocate and own the trace buffer (zeroed; freed by the next
 * sbp_set_receivers or by sbp_destroy); sbp_record_receivers copies it out.
 * n = 0 removes the receivers.  A rejected list leaves the current one in place. */
int sbp_set_receivers(SbpGrid* grid, int32_t n, const int32_t* ijk, void* traces, int32_t n_t);

/* Receivers by physical position: xyz holds n host FP64 (x, y, z) triples; each
 * receiver records at the node nearest to its point (Euclidean distance in the
 * node coordinates `coords`: 3 FP64 device fields x, y, z in the grid layout, as
 * given to sbp_metrics), searched among the nodes of face `face` (0..5, e.g. 5
 * for the free surface s = 1) or of the whole grid (face = -1); of nodes at
 * exactly the same distance the one first in [s][r][q] order is taken.  Then as
 * sbp_set_receivers(n, ijk, traces, n_t); ijk_out (host, 3 n int32, may be NULL)
 * receives the chosen nodes.  Synchronises the device.  ARG for non-finite
 * positions, a bad face or n outside 0..65535. */
int sbp_set_receivers_xyz(SbpGrid* grid, int32_t n, const double* xyz, const double* coords, int32_t face,
                          void* traces, int32_t n_t, int32_t* ijk_out);

/* Two blocks coupled at a shared face (Section 7.1 splits the LOH1 domain into
 * two blocks at its material interface and couples them weakly with penalties).
 * A face of kind SBP_BC_INTERFACE receives the penalty of Eq. penalty_terms with
 * the hat variables of a locked interface: velocity and traction (T = sigma n,
 * n = a_xi/|a_xi|) continuous, the outgoing characteristic of each side kept
 * (Appendix A's construction with the interface conditions in place of Eq.
 * BC_General2).  Block "-" has the shared face at xi = 1, block "+" at xi = 0 of
 * the same axis xi; the two faces must hold the same nodes in the same order
 * (same node counts on the face's two axes, same orientation) and the same
 * operator.
 * sbp_interface_trace writes, for face `face` of this grid and the state q (9 B
 * fields; NULL: the current state), the face trace the other block's penalty
 * needs: 8 B face arrays of the solver precision, member b's field c (v_x, v_y,
 * v_z, T_x, T_y, T_z, Z_p, Z_s) at trace[(8 b + c) n_face + idx], idx = k nr + j
 * on q faces, k nq + i on r faces, j nq + i on s faces.  sbp_set_interface tells
 * this grid where the other block's trace of the shared face lies (device
 * memory, read by every later stage or sbp_rhs; the caller refreshes it from the
 * other block's stage input before each stage, e.g. trace both blocks, then run
 * the stage on both).  A stage on a grid with an interface face lacking a trace
 * returns STATE; sbp_step_n returns UNSUPPORTED for such grids (their traces
 * must be refreshed between the stages), as do the adjoint calls. */
int sbp_interface_trace(SbpGrid* grid, int32_t face, const void* q, void* trace, void* stream);
int sbp_set_interface(SbpGrid* grid, int32_t face, const void* other_trace);

/* Memory and layout flags of the copy calls below. */
#define SBP_MEM_HOST 1      /* the caller's buffer is host memory (pageable or pinned); else device */
#define SBP_LAYOUT_DENSE 2  /* fields packed [field][s][r][q] without padding; else the grid layout */
#define SBP_MEM_ASYNC 4     /* sbp_get_state to host memory: enqueue only, do not wait for the copy */

/* Copy the recorded traces (B*n*3*n_t elements of the solver precision,
 * trace[b][r][c][step], steps not yet recorded hold zeros) to dst: host memory
 * with flags = SBP_MEM_HOST (the call then synchronises the stream), device
 * memory with flags = 0 (asynchronous).  STATE if no receivers are set. */
int sbp_record_receivers(SbpGrid* grid, void* dst, int32_t flags, void* stream);

/* Upload / download the current state (9 B fields of the solver precision):
 * src/dst in host (SBP_MEM_HOST) or device memory, in the grid layout (9 B
 * fields of fs elements, padding included) or packed [b*9 + field][s][r][q]
 * (SBP_LAYOUT_DENSE).  Both are enqueued on the stream; a download to host
 * memory synchronises the stream before returning unless flags include
 * SBP_MEM_ASYNC (then dst holds the state once the stream has passed the copy:
 * pinned dst, and the caller synchronises, e.g. to overlap the download with
 * another grid's work); an upload from pinned host memory is asynchronous, so
 * the buffer must stay unchanged until the stream has passed the copy.  The Runge-Kutta register needs no reset: a step's first
 * stage does not read it. */
int sbp_set_state(SbpGrid* grid, const void* src, int32_t flags, void* stream);
int sbp_get_state(SbpGrid* grid, void* dst, int32_t flags, void* stream);

/* Transposed operator: out = L^T w with L = P~ M the map Q -> dQ/dt of sbp_rhs
 * (penalties included, no source), transposed in the plain Euclidean inner
 * product of the 9-field vectors.  Built from the dual-pair relation of
 * Section 4.1 (Eq. upw_SBP): D-^T = B H^-1 - H D+ H^-1, D+^T = B H^-1 - H D- H^-1,
 * so it reuses the forward rows on H^-1 P~ w plus face terms.  w, out, scratch:
 * 9 B fields each (device, distinct; every member of a batch transformed).
 * UNSUPPORTED for operator codes other than 2, 4, 6. */
int sbp_rhs_adjoint(SbpGrid* grid, const void* w, void* out, void* scratch, void* stream);

/* Adjoint of fused Runge-Kutta stage k (the exact discrete adjoint of the
 * 2N-storage stage; run k = 4..0 after the adjoint of a step's later stages):
 *   wbar <- wbar + B_k ubar;  ubar <- ubar + dt L^T wbar;
 *   grad += dt (d(L u_stage)/d(rho, lambda, mu))^T wbar;  wbar <- A_k wbar.
 * ubar, wbar, scratch: 9 B fields (solver precision, device, updated in place;
 * member b at fields 9b..9b+8 as for the bound state); u_stage: the forward
 * stage inputs U_k of the B states (9 B fields); rlmj: FP64 rho, lambda, mu, J
 * (4 fields); grad: FP64 3 fields, shared by the B states, which all add into it
 * (the gradient of the summed misfit; may be NULL to skip the gradient, then
 * u_stage and rlmj may be NULL).  The impedances of the general penalty are
 * differentiated too.  UNSUPPORTED for operator codes other than 2, 4, 6. */
int sbp_adjoint_stage(SbpGrid* grid, int32_t stage, double dt, const void* u_stage, void* ubar, void* wbar,
                      void* scratch, const double* rlmj, double* grad, void* stream);

/* The adjoint of one whole step: sbp_adjoint_stage for k = 4, 3, 2, 1, 0 in one
 * call, with the same results.  u_stages: the five forward stage inputs U_0..U_4
 * back to back (group k, 9 B fields, at element offset k 9 B fs; device; may be
 * NULL with grad NULL); scratch: 18 B fields (two buffers of H^-1 P~ wbar used in
 * turn).  On the tiled kernel path the pointwise part of each stage k < 4 (wbar +
 * B_k ubar and H^-1 P~ of it) is formed in the epilogue of stage k + 1's L^T pass
 * instead of in a separate pass over the grid.  Between two calls the caller may
 * add the receivers' adjoint sources to ubar (sbp_misfit); wbar carries A_0 wbar
 * (zero for this scheme) into the next call.  Other arguments and errors as
 * sbp_adjoint_stage. */
int sbp_adjoint_step(SbpGrid* grid, double dt, const void* u_stages, void* ubar, void* wbar, void* scratch,
                     const double* rlmj, double* grad, void* stream);

/* Receiver misfit of the B states q (9 B fields): for member b, receiver r and
 * velocity component c, diff = v_c - data[(b n + r) 3 + c] (data: FP64 device,
 * 3 n per member); acc[(b n + r) 3 + c] += weight diff^2 / 2 (FP64 device, may
 * be NULL) and, if ubar (9 B fields) is not NULL, ubar_c of member b += weight
 * diff at the receiver node (the adjoint source; receivers that share a node add
 * their sources atomically, so the order of those additions is unspecified).
 * Needs sbp_set_receivers. */
int sbp_misfit(SbpGrid* grid, const void* q, const double* data, double weight, double* acc, void* ubar,
               void* stream);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * bounded wait on a shared-memory mbarrier that nothing completes, the wait
 * the tiled stage kernel uses for its tile copies.  After `polls` polls
 * (1..2^20, about 64 ns apart) it gives up and sets SBP_STATUS_TIMEOUT in the
 * status word; the context stays usable.  SBP_ERR_ARG for polls outside
 * that range. */
int sbp_selftest_wait_timeout(SbpGrid* grid, uint32_t polls, void* stream);

/* Measured FP64 arithmetic rate of the current device (no paper counterpart; the
 * denominator of the FP64 solver's roofline, which is bound by the FP64 pipe, not
 * by HBM): 8 independent fused multiply-add chains of `iters` steps (1000..1e8) in
 * each of 2048 threads per SM, timed with CUDA events on the stream after a
 * warm-up launch; *tflops = 2 x FMAs / time.  Changes no device setting; the
 * clocks are whatever the device runs at.  Synchronises the stream. */
int sbp_probe_fp64_rate(int32_t iters, double* tflops, void* stream);

/* Copy the device status word into *bits and clear it (synchronises). */
int sbp_status(SbpGrid* grid, uint32_t* bits, void* stream);

/* The 5-stage coefficients used by the kernels (A, B, and the derived stage
 * times c = row sums of the equivalent Butcher tableau). */
int sbp_rk_coefficients(double* A, double* B, double* C);

/* Energy of a state without allocating anything (no paper counterpart; an
 * addition for callers that manage all device memory themselves, such as code
 * whose framework owns a pooled allocator or that runs under a fixed memory
 * budget reserved up front, and for which a cudaMalloc inside the library is
 * not acceptable or may fail when device memory is nearly full).
 * Computes what sbp_energy computes, from plain pointers instead of a bound
 * grid: q (9 fields) and mat (3 fields: 1/(rho J), lambda/J, mu/J) in the
 * layout of sbp_layout (row pitch ldq, field stride fs), precision 32 or 64,
 * FP64 result in *out (host).  The partial sums live in a static device array
 * of 4096 doubles (plus the result and a status word, 32.8 KB), one per device,
 * kept until the process exits; nblocks (1..4096) partial sums are used, 0
 * selects 1184 (what sbp_energy uses, which gives the same result).  Sizes
 * outside these limits return SBP_ERR_ARG.  The first call on each device looks
 * up the array's device address, and so does the first call after a device
 * reset (cudaDeviceReset gives the device a new context, in which the array
 * may sit elsewhere); make that first call before any stream capture.  Every
 * call reuses the same array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Synchronises the stream; SBP_ERR_NONFINITE if the energy is not finite. */
int sbp_energy_noalloc(const void* q, const void* mat, int32_t nq, int32_t nr, int32_t ns, int64_t ldq,
                       int64_t fs, int32_t order, int32_t precision, int32_t nblocks, double* out,
                       void* stream);

/* ---- Learned surrogate (source parameters -> receiver traces) --------------
 * Kernels of a small network trained on the batched solver's seismograms.  All
 * pointers are device pointers owned by the caller; matrices are row-major;
 * "BF16" buffers hold __nv_bfloat16 values.  ARG on invalid sizes or null
 * pointers, CUDA on launch failures. */

/* C[M x N] = beta C + op(A) op(B) (+ bias[m]) (ReLU): op(A) = A (M x K, lda) or
 * A^T (A stored K x M) when transA; op(B) = B (K x N, ldb) or B^T (B stored
 * N x K) when transB.  A, B BF16; accumulation FP32 on tensor cores; C FP32
 * (c_bf16 = 0, beta 0 or 1) or BF16 (c_bf16 = 1, beta must be 0); bias FP32
 * per row or NULL.  Operands with leading dimensions that are multiples of 8
 * elements and 16-byte aligned bases run on the tcgen05 tensor cores (TMA
 * operand tiles, FP32 accumulator in tensor memory) when M, N >= 128 and
 * K >= 64; other products on the mma.sync kernels (sbp_nn_set_gemm_path). */
int sbp_nn_gemm(int32_t M, int32_t N, int32_t K, const void* A, int64_t lda, int32_t transA, const void* B,
                int64_t ldb, int32_t transB, void* C, int64_t ldc, int32_t c_bf16, const float* bias, int32_t relu,
                float beta, void* stream);
/* Which kernels sbp_nn_gemm uses, for the whole process: 0 = automatic (above),
 * 1 = the mma.sync kernels only, 2 = the tcgen05 kernel for every product whose
 * operands it can load.  ARG for other values. */
int sbp_nn_set_gemm_path(int32_t path);
/* Device-side findings of the surrogate kernels, read and cleared (synchronises
 * the device): bit 1 = a bounded wait of the tcgen05 GEMM gave up, so that
 * GEMM skipped its output. */
int sbp_nn_status(uint32_t* bits);
/* 1D convolution lowering, activations laid out [channel][batch * T]:
 * im2col: Xc[(c kw + k)][b T + t] = X[c][b T + t + k - pad] (zero outside the
 * sample); col2im sums the kw shifted copies back (FP32 in and out). */
int sbp_nn_im2col(const void* X, void* Xc, int32_t C, int32_t B, int32_t T, int32_t kw, int32_t pad, void* stream);
int sbp_nn_col2im(const float* dXc, void* dX, int32_t C, int32_t B, int32_t T, int32_t kw, int32_t pad,
                  void* stream);
/* Nearest x2 upsampling along time of `rows` rows of length T, BF16 (backward:
 * sum of pairs, FP32 in and out, X = gradient of the upsampled rows). */
int sbp_nn_upsample2(const void* X, void* Y, int64_t rows, int32_t T, int32_t backward, void* stream);
/* dZ = dA * (A > 0) (dA FP32, A and dZ BF16). */
int sbp_nn_relu_backward(const float* dA, const void* A, void* dZ, int64_t n, void* stream);
/* db[m] = sum_n dZ[m][n] (dZ BF16 M x N, db FP32). */
int sbp_nn_bias_grad(const void* dZ, float* db, int32_t M, int64_t N, void* stream);
/* Squared error: partial[b] = per-block FP64 sums of (Y - T)^2 over n values
 * (nblocks blocks); dY = 2 (Y - T)/n in BF16 (dY may be NULL). */
int sbp_nn_mse(const float* Y, const float* Tg, void* dY, int64_t n, double* partial, int32_t nblocks,
               void* stream);
/* Adam (bias-corrected, step >= 1) on FP32 weights w with gradient g and moments
 * m, v; also writes the BF16 copy w_bf16 (may be NULL). */
int sbp_nn_adam(float* w, const float* g, float* m, float* v, void* w_bf16, int64_t n, float lr, float b1, float b2,
                float eps, int32_t step, void* stream);
/* Reshape between the last MLP layer's output H [(c T0 + t)][b] and the
 * convolution layout X [c][b T0 + t] (backward: X -> H). */
int sbp_nn_mlp_to_conv(void* H, void* X, int32_t C, int32_t T0, int32_t B, int32_t backward, void* stream);
/* Traces are linear in the moment tensor: y[o][b T + t] = sum_{c<6} m[c][b]
 * G[(c n_out + o)][b T + t] with G the network's six Green's-function trace sets
 * (BF16, like the network's other activations) and m the Voigt moment components per
 * sample (FP32 [6][B]), y FP32; backward (backward = 1): dG[(c n_out + o)][b T + t] =
 * m[c][b] dy[o][b T + t] (dy, dG BF16). */
int sbp_nn_moment_combine(const void* G, const float* m, float* y, const void* dy, void* dG, int32_t n_out,
                          int32_t B, int32_t T, int32_t backward, void* stream);
/* y = BF16(x). */
int sbp_nn_cast_bf16(const float* x, void* y, int64_t n, void* stream);

/* Fourier features of the network's input (not part of the paper: the standard input
 * encoding of coordinate networks, for the surrogate's source-position input):
 * x FP32 [n_in][B] (normalised to [-1, 1]) -> y BF16 [n_in (1 + 2 L)][B]: rows
 * 0..n_in-1 are x, then for input i and k = 0..L-1 the rows n_in + 2 (i L + k) and
 * n_in + 2 (i L + k) + 1 hold sin(2^k pi x_i) and cos(2^k pi x_i).  L in 0..16
 * (L = 0: the cast alone).  Device buffers; SBP_ERR_ARG on bad sizes. */
int sbp_nn_fourier_features(const float* x, void* y, int32_t n_in, int64_t B, int32_t L, void* stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* sbp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SBP_GB300_H */
