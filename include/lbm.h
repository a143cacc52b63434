/*
 * lbm.h -- C ABI of the GB300 D3Q19 pseudopotential MRT lattice Boltzmann library.
 *
 * The library advances the method of Li, Du, Fei, Luo and Yu, "Three-dimensional
 * non-orthogonal multiple-relaxation-time lattice Boltzmann model for multiphase
 * flows" (arXiv 1805.08643) on one CUDA device:
 *
 *   rho = sum_a f_a, psi(rho)                              (Eq. 6; Sec. II B; Eq. 58)
 *   F   = -G psi(x) sum_a w_a psi(x + e_a) e_a             (Eq. 15, w = 1/6, 1/12)
 *   u   = (sum_a e_a f_a + F/2) / rho                      (Eq. 6)
 *   m   = M f,  m* = m - Lambda (m - m_eq) + (I - Lambda/2) S,  f* = M^-1 m*   (Eq. 4, 11-14, App. A)
 *   f_a(x + e_a, t + 1) = f*_a(x, t), periodic box         (Eq. 5)
 *
 * for the non-orthogonal transformation matrix of Eq. 12 or the usual orthogonal
 * D3Q19 matrix (d'Humieres et al., the paper's Ref. 11), and for the D3Q15
 * non-orthogonal variant the paper says follows the same construction
 * (Sec. II A; see LBM_OP_NONORTHOGONAL_D3Q15).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lattice units: dt = dx = c = 1, c_s^2 = 1/3.
 *  - Node index i = x + Nx*(y + Ny*z), x fastest; N = Nx*Ny*Nz.
 *  - Direction a = 0..Q-1, Q = 19 in the order of Eq. 2 (Q = 15 for the D3Q15
 *    operator: rest, +-x, +-y, +-z as in Eq. 2, then the corners (+,+,+)
 *    (-,-,-) (+,+,-) (-,-,+) (+,-,+) (-,+,-) (-,+,+) (+,-,-)).  Population
 *    arrays are structure-of-arrays: element (a, i) at offset a*N + i.
 *  - Every value crossing this boundary is a double, whatever the storage
 *    precision, except device buffers handed to lbm_bind.
 *  - "on_device" = 1: the pointer is CUDA device memory of the context's
 *    device; 0: host memory.  The caller owns every buffer it passes.
 *  - Work is queued on the stream given to lbm_create.  Calls that return host
 *    data (on_device = 0, lbm_diag, lbm_check) synchronise that stream.
 *  - No entry point aborts or prints.  Each returns an lbm_status; the text of
 *    the last error of a context is available from lbm_last_error.
 *  - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,        /* invalid argument (null pointer, bad size or enum)     */
  LBM_ERR_OOM = 2,        /* device allocation failed                             */
  LBM_ERR_CUDA = 3,       /* a CUDA runtime call failed (detail in lbm_last_error) */
  LBM_ERR_NONFINITE = 4,  /* a density or velocity became NaN or infinite         */
  LBM_ERR_EOS_DOMAIN = 5, /* rho <= 0, b rho/4 >= 1 or a negative sqrt radicand   */
  LBM_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up                   */
  LBM_ERR_STATE = 7,      /* call out of order (e.g. lbm_step before an init)     */
  LBM_ERR_BOUNDS = 8      /* debug build only: a kernel index fell outside its   */
                          /* buffer (the access went to element 0 instead)       */
} lbm_status;

/* Transformation matrix: the usual orthogonal one, or Eq. 12 (Sec. II B), both
 * on D3Q19; or the non-orthogonal construction on D3Q15 (Sec. II A says it
 * follows the same way; the paper prints none).  D3Q15 reading: the Eq. 7-10
 * monomials on the 15 velocities (1, e_x, e_y, e_z, |e|^2, 3e_x^2 - |e|^2,
 * e_y^2 - e_z^2, e_x e_y, e_x e_z, e_y e_z, e_x^2 e_y, e_x e_y^2, e_x^2 e_z,
 * e_x e_y e_z, e_x^2 e_y^2), equilibria and forcing moments of Eqs. 13-14 taken
 * from the D3Q19 rows each vector equals (their mean where several coincide;
 * zero for e_x e_y e_z), rates 1, s_e, s_nu x5, s_q x4, s_pi, and Eq. 15 weights
 * 1/3 (axes), 1/24 (corners).  A D3Q15 context runs the two-pass step (the
 * two-node kernels for the FP32-arithmetic forms with an even Nx, the one-node
 * kernels otherwise) or, for those forms, the work-list step (mode 5 of
 * lbm_set_tuning; the default with LBM_F32 storage); the other single-pass
 * variants, the no-alloc step (lbm_step_static) and batches are D3Q19 only. */
typedef enum {
  LBM_OP_ORTHOGONAL = 0,
  LBM_OP_NONORTHOGONAL = 1,
  LBM_OP_NONORTHOGONAL_D3Q15 = 2
} lbm_operator;

/* Pseudopotential (Sec. II B): square root of the Carnahan-Starling EOS
 * (Eq. 58), exponential psi0*exp(-rho0/rho), or none (no interaction force). */
typedef enum { LBM_EOS_CS = 0, LBM_EOS_EXP = 1, LBM_EOS_NONE = 2 } lbm_eos_kind;

/* Arithmetic and storage of the populations.  F64: FP64 arithmetic and storage.
 * F32: FP32 arithmetic, FP32 storage.  F32_STORE_F16: FP32 arithmetic, FP16
 * storage.  The reduced forms store deviations f_a - w_a rho_ref (the FP16 form
 * divides them by the lattice weight w_a) and keep the EOS and every global
 * reduction in FP64. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F32_STORE_F16 = 2 } lbm_precision;

typedef struct {
  int kind;            /* lbm_eos_kind                                           */
  double a, b, R, T;   /* Carnahan-Starling parameters (Eq. 58); T_c = 0.37733 a/(bR) */
  double psi0, rho0;   /* exponential form                                       */
} lbm_eos;

/* Relaxation rates s (not times).  Non-orthogonal operator (Eq. 11): s_e for
 * moment 4, s_nu for 5-9, s_q for 10-15, s_pi for 16-18.  Orthogonal operator:
 * s_e (energy e), s_eps (eps), s_q (q_x, q_y, q_z), s_nu (p_xx, p_ww, p_xy,
 * p_yz, p_xz), s_pi (pi_xx, pi_ww), s_m (m_x, m_y, m_z).  Conserved moments
 * relax with rate 1 (Sec. II B). */
typedef struct {
  double s_e, s_nu, s_q, s_pi, s_eps, s_m;
} lbm_rates;

/* Create a context for a periodic Nx x Ny x Nz box (grid = {Nx, Ny, Nz}, each
 * >= 3 so that the periodic neighbours are distinct).  G is the interaction
 * strength of Eq. 15; sigma the constant of Eq. 16 (0 disables that term).
 * cuda_stream is a cudaStream_t of the current device (NULL = legacy default
 * stream).  Allocates no device memory: call lbm_bind or let the first init
 * allocate.  Errors: LBM_ERR_ARG.  On success *out owns the context. */
lbm_status lbm_create(const int grid[3], const lbm_eos *eos, double G,
                      const lbm_rates *rates, int op, int precision, double sigma,
                      void *cuda_stream, lbm_ctx **out);

/* Bytes of the three device buffers a context needs: each of the two
 * population buffers (Q N stored values, and never less than 4N doubles: the
 * spare one stages rho and u for lbm_moments), the psi buffer (two time levels
 * of psi), and the scratch buffer (reductions and the error word). */
lbm_status lbm_buffer_bytes(const lbm_ctx *ctx, size_t *population_bytes,
                            size_t *psi_bytes, size_t *scratch_bytes);

/* Hand the context caller-owned device buffers of at least the sizes above,
 * 256-byte aligned (e.g. from a PyTorch allocation).  They must outlive the
 * context.  Without this call the first init allocates its own (LBM_ERR_OOM
 * when that fails).  Errors: LBM_ERR_ARG, LBM_ERR_STATE (already bound). */
lbm_status lbm_bind(lbm_ctx *ctx, void *f_a, void *f_b, void *psi, void *scratch);

/* Initial state at rest, f_a = w_a rho0(x) = M^-1 m_eq(rho0, u = 0), for:
 *  - one droplet, Eq. 59: rho0 = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 (r - R)/W),
 *    r the periodic minimum-image distance from centre (node coordinates 0..N-1);
 *  - n droplets (centres: n x 3 doubles, radii: n doubles, host memory): the
 *    pointwise maximum of their Eq. 59 profiles;
 *  - a liquid slab between planes lo < hi across axis (0 = x, 1 = y, 2 = z):
 *    rho0 = rho_v + (rho_l - rho_v)/2 [tanh(2 (c - lo)/W) - tanh(2 (c - hi)/W)];
 *  - an arbitrary density field rho (N doubles), with reference density rho_ref
 *    for the deviation storage of the reduced precisions.
 * The droplet and slab forms take rho_ref = rho_v.  Resets the step counter.
 * Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_init_droplet(lbm_ctx *ctx, const double centre[3], double R, double W,
                            double rho_l, double rho_v);
lbm_status lbm_init_droplets(lbm_ctx *ctx, int n, const double *centres, const double *radii,
                             double W, double rho_l, double rho_v);
lbm_status lbm_init_flat(lbm_ctx *ctx, int axis, double lo, double hi, double W,
                         double rho_l, double rho_v);
lbm_status lbm_init_field(lbm_ctx *ctx, const double *rho, int on_device, double rho_ref);

/* Advance n >= 1 time steps (asynchronous on the context's stream).  Each step
 * is the form's step kernels (lbm_set_tuning): by default, for FP32 storage
 * with an even Nx, one cooperative launch of the work-list single pass;
 * otherwise two kernels, the psi pass and the fused force + collision +
 * pull-streaming pass.  A work-list launch carries the context's launch count
 * (its completion and item-claim counters advance with every launch), so steps
 * must not be captured into a CUDA graph and replayed: a replayed launch finds
 * its counters out of step, stops early and reports LBM_ERR_TIMEOUT at the next
 * check.  Errors: LBM_ERR_ARG (n < 1), LBM_ERR_STATE (no init), LBM_ERR_CUDA;
 * LBM_ERR_EOS_DOMAIN / LBM_ERR_NONFINITE / LBM_ERR_TIMEOUT when a check
 * interval is set (below) and a check inside this call fails. */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* Density rho (N doubles) and velocity u (3N doubles, u_x block then u_y then
 * u_z) of the current state, Eq. 6 with the force of Eq. 15. */
lbm_status lbm_moments(lbm_ctx *ctx, double *rho, double *u, int on_device);

/* The post-streaming populations f_a(x, t) of the current time t (QN doubles,
 * SoA; Q = 19, or 15 for LBM_OP_NONORTHOGONAL_D3Q15), and the reverse: make
 * them the current state (keeps rho_ref). */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int on_device);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int on_device);

/* FP64 reductions over the box (synchronises): out[0] = total mass sum rho,
 * out[1..3] = total momentum sum rho u (Eq. 6), out[4] = max |u|. */
lbm_status lbm_diag(lbm_ctx *ctx, double out[5]);

/* Read and clear the device error word set by the kernels (synchronises):
 * LBM_OK, LBM_ERR_EOS_DOMAIN, LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT (a bounded
 * wait of a single-pass kernel gave up, or a work-list launch could not follow
 * its list) or, in the debug build of the library (compiled with
 * LBM_BOUNDS_CHECK), LBM_ERR_BOUNDS. */
lbm_status lbm_check(lbm_ctx *ctx);

/* Make lbm_step run lbm_check every k steps (0, the default, never). */
lbm_status lbm_set_check_interval(lbm_ctx *ctx, int k);

/* Per-kernel timing with CUDA events on the context's stream.  While enabled,
 * lbm_step records an event pair around every launch; lbm_kernel_times
 * (synchronises) returns the summed milliseconds and launch counts of the psi
 * pass and of the fused pass since the last reset, then resets them. */
lbm_status lbm_set_profiling(lbm_ctx *ctx, int enabled);
lbm_status lbm_kernel_times(lbm_ctx *ctx, double *ms_psi, long long *n_psi,
                            double *ms_fused, long long *n_fused);

/* Kernel choice for this context.  The default is 5 (below) for an LBM_F32
 * context with an even Nx (D3Q19 or D3Q15), the faster step there on GB300,
 * and 0 otherwise.  single_pass = 0 runs the psi pass and the fused pass.  1 (LBM_F32 and LBM_F32_STORE_F16 only) runs each
 * step as one kernel that also produces psi of the next step, recomputing
 * collisions on a one-node ring around each thread block's tile.  2 runs that
 * single pass with its data moved by bulk asynchronous copies (LBM_F32 only,
 * Nx a multiple of 4 and at least 40; 32x8 tiles).  3 (LBM_F32 and
 * LBM_F32_STORE_F16, Nx even) runs each step as one kernel that evaluates psi
 * of the step on chip from the pulled populations (producer warps, for the
 * thread block's 32x8 tile and a one-node ring) while consumer warps collide:
 * no psi array is read or written, and with FP32 storage the result is that
 * of the default two-pass step bit for bit; tile and z_planes do not apply.
 * 4 (same forms) runs each step as one cooperative launch in which the psi
 * pass of the next step trails the fused pass by one plane, reading the new
 * populations from L2; results equal the two-pass step bit for bit; the first
 * call in this mode allocates a small device array of progress flags (one int
 * per 64x4 tile and plane), freed by lbm_destroy.  5 (same forms; also
 * on D3Q15) runs each step as one cooperative launch over an ordered work list: each
 * item is the fused pass of one 64x4 tile of one plane plus the psi pass of
 * the next step for another tile, placed (and checked, on the host) at least
 * half a wave of the grid after the 27 fused tiles it reads; the FP64 EOS of the
 * psi work overlaps the fused work's HBM stream and the populations it pulls
 * come from L2 (Eqs. 3-6 in 2 x Q x s + 8 bytes per node); results equal the
 * two-pass step bit for bit; the first step in this mode allocates the item
 * table and counters (about 20 bytes per tile and plane), freed by
 * lbm_destroy.  tile picks the x-y tile of
 * the single-pass kernel (0: 32x4, 1: 32x8, 2: 64x4); z_planes the z planes
 * each thread block marches through (0 = automatic).  Results do not depend on
 * tile or z_planes.  Errors: LBM_ERR_ARG (bad value, a mode the context's
 * precision or Nx does not support, or a single-pass mode other than 5 on a D3Q15 context);
 * LBM_ERR_OOM / LBM_ERR_CUDA (mode 4's flag array or mode 5's item table
 * could not be allocated, at the first step in mode 5). */
lbm_status lbm_set_tuning(lbm_ctx *ctx, int single_pass, int tile, int z_planes);

/* Budget of the bounded device-side waits of the single-pass kernels (modes 2-5):
 * a wait polls at most spin_limit times (a few tens of nanoseconds apart) and
 * then gives up: it sets the context's error word (lbm_check returns
 * LBM_ERR_TIMEOUT) and the kernel goes on to its end, so no launch can hang.
 * spin_limit <= 0 restores the default, 2^22.  inject_unreachable != 0 is a
 * host-side fault injection for tests: every cross-block wait of modes 4 and 5
 * then waits for a count no block reaches, so each such wait runs out its
 * budget (the results of those steps are not meaningful; set it back to 0 and
 * re-initialise).  Takes effect at the next lbm_step.  Errors: LBM_ERR_ARG. */
lbm_status lbm_set_wait_budget(lbm_ctx *ctx, int spin_limit, int inject_unreachable);

/* Density-dependent shear viscosity (Sec. IV D: raising nu_V / nu_L lowers the
 * spurious currents; the paper gives no rule).  nu(rho) is linear in rho from
 * nu_v at rho_v to nu_l at rho_l and clamped between the two; each node relaxes
 * its shear moments with s_nu(rho) = 1 / (3 nu(rho) + 1/2) in place of s_nu.
 * nu_l <= 0 and nu_v <= 0 switch it off (the default).  Errors: LBM_ERR_ARG. */
lbm_status lbm_set_variable_viscosity(lbm_ctx *ctx, double rho_l, double rho_v, double nu_l, double nu_v);

/* Arithmetic of the EOS radicand in the psi pass of the FP32-arithmetic forms:
 * 0 (the default) FP64; 1 compensated FP32 pairs (error-free transformations,
 * about 44 significant bits, no FP64 instructions; GB300 has 2 FP64 lanes per
 * SM against 128 FP32).  The FP64 form always uses FP64.  Errors: LBM_ERR_ARG. */
lbm_status lbm_set_eos_arith(lbm_ctx *ctx, int mode);
lbm_status lbm_get_tuning(const lbm_ctx *ctx, int *single_pass, int *tile, int *z_planes);

/* Steps taken since the last init or lbm_set_populations. */
long long lbm_step_count(const lbm_ctx *ctx);

/* One FP64 time step that allocates no device memory (the paper has no
 * counterpart; this is a library service).  For callers that cannot call
 * cudaMalloc: code running while a CUDA graph is captured, hosts whose device
 * memory belongs to another allocator, loops that must never allocate.
 *  - f_in: the post-streaming populations f_a(x, t) of the box, device memory,
 *    19N doubles in the public SoA layout (as lbm_get_populations returns them);
 *    f_out (distinct, same layout) receives f_a(x, t + 1).  The caller owns both.
 *  - ctx supplies the box, physics and stream only; it must be LBM_F64.  Its own
 *    populations and buffers are neither read nor written, and it need not be
 *    initialised or bound.
 *  - The psi scratch is a static device array of 2^21 doubles (16 MiB, boxes of
 *    up to 2^21 nodes, e.g. 128^3) that every GPU loading the library holds until
 *    exit; larger boxes return LBM_ERR_ARG.  All calls share it: calls whose work
 *    overlaps on the GPU (different streams, or other processes' contexts in
 *    flight at once on one device) race and give wrong results.  Each call
 *    rewrites all psi it reads, so nothing needs clearing between calls.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 *    first call before any stream capture.  cudaDeviceReset invalidates the
 *    kept address: do not call this after resetting a device it has run on.
 *  - Asynchronous on the context's stream.  A density outside the EOS domain
 *    gives NaN populations in f_out (there is no error word on this path).
 * Errors: LBM_ERR_ARG (null or aliased pointers, precision, size, a D3Q15 context),
 * LBM_ERR_CUDA (the status of this call's own launches only: an error left
 * earlier on the calling thread is neither reported nor cleared). */
lbm_status lbm_step_static(const lbm_ctx *ctx, const double *f_in, double *f_out);

/* ------------------------------------------------------------------ batches
 * Many independent periodic boxes advanced together: every step runs
 * persistent launches over a table of work items (one x-y tile of one box and
 * a range of z planes each, largest boxes first): when every box has an even
 * Nx, the fused pass and then the psi pass of the new state on the two-node
 * kernels of lbm_step; otherwise one launch of the single-pass kernel.
 * lbm_batch_step replays the launches of two steps as a CUDA graph.  Boxes
 * may differ in size, operator, temperature, G, rates and sigma; they share the
 * precision (LBM_F32 or LBM_F32_STORE_F16) and the kind of EOS.  Boxes join
 * (lbm_batch_add) and leave (lbm_batch_remove) between calls: continuous
 * batching.  Each box's buffers come from the stream-ordered allocator of the
 * batch's stream and are charged to the batch's HBM budget (admission by
 * footprint).  A box's results do not depend on the other boxes of the batch.
 * Not in the paper: the paper steps one box at a time. */
typedef struct lbm_batch lbm_batch;

/* Device bytes one box of the given size holds in a batch (populations, two
 * psi levels, the previous velocity for lbm_batch_max_du); 0 for a bad grid. */
size_t lbm_batch_box_bytes(int precision, const int grid[3]);

/* precision: LBM_F32 or LBM_F32_STORE_F16; eos_kind: lbm_eos_kind shared by all
 * boxes; hbm_budget_bytes: the most device memory the boxes may hold;
 * cuda_stream: a cudaStream_t (NULL: the batch creates its own stream). */
lbm_status lbm_batch_create(int precision, int eos_kind, size_t hbm_budget_bytes, void *cuda_stream,
                            lbm_batch **out);

/* Add a box (parameters as in lbm_create; D3Q19 operators only); *id receives
 * its handle.  Errors: LBM_ERR_ARG, LBM_ERR_OOM when the budget or the device
 * has no room. */
lbm_status lbm_batch_add(lbm_batch *b, const int grid[3], const lbm_eos *eos, double G, const lbm_rates *rates,
                         int op, double sigma, int *id);
lbm_status lbm_batch_remove(lbm_batch *b, int id);

/* Initial states of one box, as lbm_init_droplet / lbm_init_flat.  A box takes
 * part in lbm_batch_step once it has been initialised. */
lbm_status lbm_batch_init_droplet(lbm_batch *b, int id, const double centre[3], double R, double W,
                                  double rho_l, double rho_v);
lbm_status lbm_batch_init_flat(lbm_batch *b, int id, int axis, double lo, double hi, double W, double rho_l,
                               double rho_v);

/* Step of the batch's boxes with an even Nx: 3 (the default) the work-list
 * single pass (one cooperative launch per step over tile jobs of all boxes:
 * fused jobs and the next step's psi jobs, each box's psi jobs half a wave of
 * the grid behind the fused jobs they read; its completion counters, 4 bytes
 * per tile and plane, are cleared by a memset in the step graph); 0, 1, 2 the
 * two-pass pair kernels with that tile shape (32x4, 32x8, 64x4): the fused pass
 * as a flat grid of one block per plane of a tile, one launch per operator (a
 * block-to-box table of 4 bytes per block), then the psi pass over work items
 * of a tile through z planes.  Boxes with an odd Nx run the one-node single
 * pass in the same step, tile shape as chosen (32x8 under 3).  For box id >= 0,
 * z_planes sets its planes per work item of the psi pass and the single pass
 * (0 = automatic).  Results do not depend on the choice (the work list and the
 * two-pass kernels are equal bit for bit). */
lbm_status lbm_batch_set_tuning(lbm_batch *b, int tile, int id, int z_planes);

/* Advance every initialised box n >= 1 steps (even n replays the two-step graph
 * only; an odd n also re-uploads the box table). */
lbm_status lbm_batch_step(lbm_batch *b, int n);

/* Per-box observables, as lbm_moments and lbm_diag. */
lbm_status lbm_batch_moments(lbm_batch *b, int id, double *rho, double *u, int on_device);
lbm_status lbm_batch_diag(lbm_batch *b, int id, double out[5]);

/* For the nid boxes in ids: out[k] = max over nodes of |u(t) - u(t_prev)|, where
 * t_prev is the previous call for that box (or its initialisation: u = 0),
 * FP64; host output, synchronises.  Used as the convergence test of a job. */
lbm_status lbm_batch_max_du(lbm_batch *b, int nid, const int *ids, double *out);

/* Read and clear the batch's device error word (as lbm_check). */
lbm_status lbm_batch_check(lbm_batch *b);

/* Live boxes, work items of the current table, device bytes charged. */
lbm_status lbm_batch_info(const lbm_batch *b, int *live_boxes, int *work_items, size_t *bytes_used);

/* Steps box id has taken since its initialisation (-1: no such box). */
long long lbm_batch_box_steps(const lbm_batch *b, int id);

/* How many times the batch has uploaded its descriptor and work-item tables and
 * captured its step graphs (after boxes join, leave, are initialised or retuned;
 * stepping alone, odd or even counts, never rebuilds).  -1 for a NULL batch. */
long long lbm_batch_graph_builds(const lbm_batch *b);

const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* Release the context and any device memory it allocated itself. */
void lbm_destroy(lbm_ctx *ctx);

/* Text of the last error of ctx ("" if none); ctx may be NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
