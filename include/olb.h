/*
 * olb.h -- C ABI of the GB300 semi-Lagrangian off-lattice Boltzmann library.
 *
 * The library advances the populations of one velocity set on a uniform,
 * periodic Cartesian grid by the semi-Lagrangian lattice Boltzmann step of
 * Wilde et al., "Cubature rules for weakly and fully compressible off-lattice
 * Boltzmann methods" (arXiv:2101.03982), Sec. 3:
 *
 *   1. pull: every population f_i is interpolated at the departure point
 *      x - xi_i dt (Sec. 3, Eq. sl_streaming) with a tensor product of
 *      equidistant Lagrange polynomials of degree p (one fixed stencil per
 *      velocity, because every node of a uniform grid has the same offset),
 *      or with the paper's cell-wise Lagrange elements on Gauss-Lobatto-
 *      Chebyshev points (olb_set_interpolation);
 *   2. moments rho = sum f_i, rho u = sum xi_i f_i (Sec. 3, Eqs. density and
 *      momentum); compressible runs add 2 rho C_v theta = sum |xi_i-u|^2 f_i/T0
 *      + sum g_i (Sec. 3, temperature relation);
 *   3. Hermite equilibrium of order N (Sec. 3 and Appendix A);
 *   4. BGK relaxation f <- f - (f - f^eq)/tau (Sec. 3, LBE), with
 *      tau = mu/(c_s^2 dt P) + 1/2, P = rho theta, per node when compressible;
 *      for Pr != 1 the heat flux relaxes at tau_2 through a quasi-equilibrium
 *      (olb_options.prandtl).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Layout: a scalar field is [nz][ny][nx], x fastest (2D: nz = 1).  A vector
 *   field u is structure-of-arrays [D][nz][ny][nx].  Populations are planes
 *   [plane][nz][ny][nx]; planes 0..Q-1 hold f_i in the order of the paper's
 *   tables, planes Q..2Q-1 hold g_i in compressible runs.
 * - "on_device": 1 means the pointer is CUDA device memory that the call uses
 *   on the handle's stream (for example a torch tensor's data_ptr()); 0 means
 *   host memory, copied synchronously inside the call.
 * - Ownership: the handle owns its population buffers, scratch and tables.
 *   Caller buffers are only read or written during the call that gets them.
 * - Errors: every int-returning call returns OLB_OK (0) or a negative code
 *   below; nothing aborts and nothing throws.  olb_last_error() describes the
 *   most recent failure of the calling thread.  A handle is used by one host
 *   thread at a time.
 * - Units: lengths in units of the domain (dx = grid spacing), times in the
 *   units of dt; the velocity set's abscissae are scaled by cs_scale.
 */
#ifndef OLB_H
#define OLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OLB_OK 0
#define OLB_EINVAL (-1)         /* invalid argument */
#define OLB_ENOMEM (-2)         /* device or host allocation failed */
#define OLB_ECUDA (-3)          /* a CUDA runtime call failed */
#define OLB_ENONFINITE (-4)     /* the state holds NaN or Inf */
#define OLB_ETIMEOUT (-5)       /* a bounded host wait ran out */
#define OLB_EBOUNDS (-6)        /* a size or index lies outside what the call supports */
#define OLB_EUNSUPPORTED (-7)   /* combination not built or not exact (e.g. N too high) */
#define OLB_ESTATE (-8)         /* call out of order (e.g. no step yet) */

/* Velocity sets (Sec. 2, Table 1; Tables 2-3; Appendices C-E). */
typedef enum {
  OLB_D2Q9 = 0,   /* Gauss-Hermite product of D1Q3, degree 5, c_s = 1 */
  OLB_D2Q19 = 1,  /* Haegemans-Piessens cubature, degree 9 (Appendix C) */
  OLB_D2Q25 = 2,  /* Gauss-Hermite product of D1Q5, degree 9 */
  OLB_D3Q13 = 3,  /* icosahedron, degree 5 (Table 2) */
  OLB_D3Q21 = 4,  /* dodecahedron, degree 5, c_s = sqrt(3/5) (Table 3) */
  OLB_D3Q27 = 5,  /* Gauss-Hermite product of D1Q3, degree 5 */
  OLB_D3V27 = 6,  /* Stroud-Secrest, degree 7 (Appendix D) */
  OLB_D3Q45 = 7   /* Konyaev cubature, degree 9 (Appendix E) */
} olb_velocity_set;

/* Storage of the populations.  Shifted storage keeps f_i - w_i rho0 (and
 * g_i - w_i (2C_v - D) rho0), rounded to nearest even; the arithmetic of the
 * step is then FP32.  OLB_FP64 stores f_i itself and computes in FP64. */
typedef enum {
  OLB_FP64 = 0,
  OLB_FP32_SHIFTED = 1,
  OLB_BF16_SHIFTED = 2,
  OLB_FP16_SHIFTED = 3
} olb_storage;

/* Periodic grid: dim in {2,3}; n[2] must be 1 when dim == 2; dx > 0. */
typedef struct {
  int dim;
  int n[3];
  double dx;
} olb_grid;

typedef struct {
  int interp_order;  /* p, Lagrange degree per axis; built: 1..6 (FP64), 2..4 (others) */
  int storage;       /* olb_storage */
  double cs_scale;   /* abscissae and c_s scaled by this factor (D2Q9 with c_s^2=1/3: 1/sqrt(3)) */
  int compressible;  /* 0: theta = 1, f only; 1: f and g, per-node tau(P) (requires c_s = 1) */
  double gamma;      /* heat capacity ratio (compressible), C_v = 1/(gamma-1) */
  double mu;         /* dynamic viscosity (compressible; the tau argument is then ignored) */
  double mu_exponent; /* compressible: mu(theta) = mu theta^mu_exponent (0: constant mu, as in Sec. 3) */
  double prandtl;    /* compressible: Prandtl number (default 1, plain BGK).  Sec. 3 varies Pr with a
                        quasi-equilibrium and gives no form; the form built here: f relaxes at tau to
                        f*, the equilibrium carrying the pulled f's central heat flux
                        sum_i f_i zeta_i |zeta_i|^2 (zeta = xi - u), and from f* to f^eq at
                        tau_2 = 1/2 + (tau - 1/2)/Pr; g likewise with its central first moment.
                        Pr != 1 needs N >= 3 and a set of degree >= 7 (OLB_EUNSUPPORTED otherwise) and
                        is refused for isothermal runs (OLB_EINVAL). */
  double rho0;       /* reference density of the shifted storage (default 1) */
  int allow_inexact; /* 1: accept a quadrature degree below 2N */
  int log_every;     /* the global sums are accumulated on steps whose count is a multiple of this (>= 1) */
  int kernel;        /* 0: automatic (the fastest step kernel built for the configuration), 1: the
                        single-role step kernel, 2: the two-phase kernel (staging slab), where built */
  void* stream;      /* cudaStream_t for every call of the handle; NULL = default stream */
} olb_options;

typedef struct olb_ctx* olb_handle;

/* Fill *opt with defaults: p = 3, FP64, cs_scale = 1, isothermal, gamma = 1.4,
 * mu = 0, mu_exponent = 0, prandtl = 1, rho0 = 1, allow_inexact = 0, log_every = 1, kernel = 0,
 * stream = NULL. */
void olb_default_options(olb_options* opt);

/* Abscissae count Q, dimension D, c_s, largest |xi_{i,alpha}| and degree of a
 * velocity set, unscaled.  Any pointer may be NULL.  No GPU needed. */
int olb_velocity_set_info(int velocity_set, int* Q, int* D, double* cs,
                          double* max_abs_xi, int* degree);

/* Copy the velocity set's abscissae (Q x D, row-major, unscaled) and weights. */
int olb_velocity_set_table(int velocity_set, double* xi, double* w);

/* Stencils of the cell-wise interpolation on Gauss-Lobatto-Chebyshev points
 * (Sec. 3, the paper's streaming): an axis of C cells of width H carries C p
 * nodes, node c p + k at H (c + (1 - cos(pi k / p)) / 2).  For a departure
 * point displaced by -shift cell widths, the node of residue k (k = 0..p-1)
 * reads the p + 1 nodes first[k] + m (m = 0..p, relative to the node) with
 * the Lagrange weights W[k (p + 1) + m] of the cell that contains the
 * departure point.  first: p ints, W: p (p + 1) doubles, caller-owned.  No
 * GPU needed.  OLB_EINVAL for p outside 1..OLB_GLC_MAX_P, a non-finite shift
 * or a null output.  olb_set_interpolation(h, 1) runs the step with these
 * stencils. */
#define OLB_GLC_MAX_P 8
int olb_glc_stencil(int p, double shift, int* first, double* W);

/* Create a simulation.  hermite_order N in {2,3,4} (Sec. 3); tau > 1/2 the
 * BGK relaxation time (ignored when compressible: tau(P) from opt->mu); dt > 0.
 * Allocates the two population buffers, the per-CTA scratch and the reduction
 * buffers on the current CUDA device.  Returns OLB_EUNSUPPORTED when the set's
 * degree is below 2N (the exactness rule d >= N + M of Sec. 2 with M = N)
 * unless allow_inexact is set. */
int olb_create(const olb_grid* grid, int velocity_set, int hermite_order, double tau,
               double dt, const olb_options* opt /* nullable */, olb_handle* out);

/* Release the handle and every device buffer it owns (no counterpart in the paper).
 * Synchronises the handle's stream first.  OLB_EINVAL for a null handle. */
int olb_destroy(olb_handle h);

/* Q, planes (Q or 2Q), nodes, dimension and the storage element size in bytes. */
int olb_shape(olb_handle h, int* Q, int* planes, size_t* nodes, int* dim, int* elem_bytes);

/* Per-velocity stencil table of the pull (Sec. 3, Eq. sl_streaming: the
 * population of velocity i is interpolated at the departure point x - xi_i dt,
 * i.e. at the offset delta = -xi_{i,a} dt / dx grid units along axis a):
 * m0[Q*3] (first support point per axis, grid units, row-major [i][a]) and
 * W[Q*3*(p+1)] the Lagrange weights of the p + 1 points m0 .. m0 + p at delta
 * (FP64, [i][a][j]).  Caller-owned host arrays of those sizes (either may be
 * NULL).  An axis with xi_{i,a} = 0 has m0 = 0 and the weights of delta = 0
 * (a Kronecker delta).  OLB_EINVAL for a null handle. */
int olb_stencil(olb_handle h, int* m0, double* W);

/* Initial state from macroscopic fields.  The paper does not state how the
 * populations start; this call implements the reading f_i = f_i^eq(rho, u,
 * theta), the Hermite equilibrium of order N of Sec. 3 and Appendix A (and
 * g_i = theta (2 C_v - D) f_i^eq, the compressible model's g equilibrium of
 * Sec. 3), with no non-equilibrium part.  rho [n], u [D][n], theta [n] or
 * NULL (= 1): FP64 fields in the layout above.  The result is rounded to the
 * storage type (shifted where the storage is).  OLB_EINVAL for a null handle,
 * rho or u; OLB_ENOMEM when a host-field staging buffer cannot be allocated. */
int olb_init_fields(olb_handle h, const double* rho, const double* u, const double* theta,
                    int on_device);

/* Advance n >= 0 steps of the semi-Lagrangian LBE (Sec. 3): each step pulls
 * every population from its departure point (Eq. sl_streaming), forms the
 * moments, the order-N Hermite equilibrium (Appendix A) and relaxes by BGK
 * (the LBE of Sec. 3; compressible: tau = mu/(c_s^2 dt P) + 1/2 per node).
 * The stored state is the post-collision one (one step = pull, then
 * collide).  Asynchronous on the handle's stream; OLB_EINVAL for n < 0,
 * OLB_ECUDA when a launch fails, OLB_ETIMEOUT when an earlier step gave up
 * waiting for a staging copy and no new state has been written since.  A step whose running count (since olb_create) is a multiple of
 * log_every also leaves per-CTA FP64 partial sums of the global reductions,
 * which olb_reductions() combines.  Device memory: the handle keeps each
 * plane with ghost layers of periodic copies around the interior, which the
 * step refreshes as it writes. */
int olb_step(olb_handle h, int n);

/* Moments of the stored post-collision state: rho = sum_i f_i and
 * rho u = sum_i xi_i f_i (Sec. 3, density and momentum moments), and for a
 * compressible state theta from 2 rho C_v theta = sum_i |xi_i - u|^2 f_i / T0
 * + sum_i g_i (Sec. 3, temperature relation; T0 = 1).  BGK conserves these, so
 * they equal the moments of the pulled populations of the last step.  Outputs
 * rho [n], u [D][n], theta [n] (nullable; 1 for isothermal states) in FP64,
 * host or device per on_device.  OLB_EINVAL for a null handle, rho or u. */
int olb_moments(olb_handle h, double* rho, double* u, double* theta, int on_device);

/* Global sums of the most recent step when that step accumulated them (else
 * of the stored state, with eps = NaN), in a fixed summation order:
 *   out[0] k     = mean |u|^2/2                       (Sec. 4.2, kinetic energy)
 *   out[1] k_rho = mean rho |u|^2/2
 *   out[2] eps   = mean 2 nu S:S, S = -Pi_neq/(2 P tau dt) (estimator; NaN without a step)
 *   out[3] mass  = sum rho
 *   out[4..6]    = sum rho u (x, y, z)
 *   out[7]       = number of nodes with non-finite rho, u or theta
 * Synchronises the stream.  Returns OLB_ENONFINITE (after filling out) when
 * out[7] > 0, and OLB_ETIMEOUT when a step kernel gave up waiting for one of
 * its staging copies (bounded wait; the step's output is then invalid). */
int olb_reductions(olb_handle h, double out[8]);

/* k and (nullable) the dissipation estimate; a view of olb_reductions(). */
int olb_kinetic_energy(olb_handle h, double* k, double* dissipation);

/* Enstrophy of the current state (Sec. 4.2): E = mean over the nodes of |curl u|^2, with u from
 * the moments of the stored populations and fourth-order central differences of spacing dx on
 * the periodic grid (2D: the z component only).  The scaled enstrophy is nu * E.  Off the
 * per-step path (three launches and a read-back); synchronises the handle's stream.
 * OLB_ENONFINITE if the result is not finite; OLB_EUNSUPPORTED while the inflow/outflow x
 * boundary is set (the differences are periodic). */
int olb_enstrophy(olb_handle h, double* enstrophy);

/* The populations f_i (planes Q..2Q-1: g_i) of the stored post-collision
 * state, the unknowns of the LBE of Sec. 3, as FP64 unshifted values in the
 * compact layout [planes][nz][ny][nx] (no ghost layers).  get converts from
 * the storage type exactly; set rounds to it (after removing the shift
 * w_i rho0) and refreshes the ghost layers.  OLB_EINVAL for a null handle or
 * array. */
int olb_get_populations(olb_handle h, double* f, int on_device);
int olb_set_populations(olb_handle h, const double* f, int on_device);

/* Non-periodic x for the standing shock of Sec. 4.1 (the paper does not state
 * its boundary treatment; this is a reading).  kind 1: after every writer of
 * the state (each step, init, set_populations, set_state) the ghost columns
 * left of x = 0 are set to the equilibrium of the inflow state (rho, u[D],
 * theta; theta is ignored for isothermal runs) and those right of x = nx - 1
 * to copies of the last column (zero-gradient outflow); y and z stay
 * periodic.  The current state's ghosts are refilled at once.  kind 0:
 * periodic again (every ghost copy rewritten from the interior).  OLB_EINVAL
 * for another kind, a null u, rho <= 0 or a non-finite value (theta <= 0 when
 * compressible).  The adjoint and the tape (olb_tape_*, olb_adjoint_step)
 * and olb_enstrophy (periodic differences) return OLB_EUNSUPPORTED while
 * kind 1 is set.  Switching back rewrites the ghosts in place (no allocation). */
int olb_set_x_boundary(olb_handle h, int kind, double rho, const double* u, double theta);

/* Raw stored state (checkpoint): exactly olb_state_bytes() bytes, the
 * storage values (shifted where the storage is) as [planes][nz][ny][nx]
 * without ghost layers.  olb_set_state also refreshes the ghost layers.
 * With on_device = 0, a buffer in page-locked host memory that is mapped into
 * the device's address space (cudaHostAlloc, cudaHostRegister, torch's
 * pin_memory) is read or written in place by the copy kernel over the
 * CPU-GPU link; other host memory goes through a temporary device buffer.
 * Both return once the host buffer is no longer used. */
size_t olb_state_bytes(olb_handle h);
int olb_get_state(olb_handle h, void* buf, size_t bytes, int on_device);
int olb_set_state(olb_handle h, const void* buf, size_t bytes, int on_device);

/* Wait for the handle's stream, polling with a bound of timeout_ms (<= 0: no bound),
 * then check the device error flag of the step kernels (no counterpart in the paper).
 * OLB_ETIMEOUT when the bound ran out or a step gave up waiting for a staging copy. */
int olb_synchronize(olb_handle h, int timeout_ms);

/* Interpolation of the pull (Sec. 3, Eq. sl_streaming).  scheme 0 (the
 * default): one equidistant Lagrange stencil of degree p per velocity and axis
 * on the uniform grid (every node has the same offset).  scheme 1: the
 * paper's own streaming, cell-wise Lagrange interpolation on Gauss-Lobatto-
 * Chebyshev points: every axis of n nodes is read as n / p cells of width
 * p dx, node c p + k at the GLC point k of cell c, and the departure point of
 * a node is interpolated with the Lagrange basis of the cell that contains it
 * (the stencils of olb_glc_stencil, per velocity, axis and residue k, with the
 * shift xi_a dt / (p dx)).  The moments, equilibrium and BGK are unchanged; a
 * step is then two launches (the pull into the second buffer, then the
 * collision), and the global sums stay plain node means.  OLB_EINVAL for
 * another scheme or an axis whose length is not a multiple of p;
 * OLB_EUNSUPPORTED for the inflow/outflow x boundary or departure points too
 * far for the staged box (a Courant number of several cells).  Every storage;
 * 16-bit values are interpolated in FP32.  While
 * scheme 1 is set the adjoint calls return OLB_EUNSUPPORTED. */
int olb_set_interpolation(olb_handle h, int scheme);

/* Bound of the step kernels' waits for their staging copies, in polls of the
 * copy's barrier (no counterpart in the paper; a diagnostic of the error path).
 * polls < 0 restores the default (2^24 polls, far beyond any copy's latency);
 * polls = 0 makes every step give up at its first wait, so that a test can
 * check the error path without a fault: the kernel raises the device error
 * flag, waits (with the default bound) for the copies it has in flight and
 * returns.  The next call that checks the flag returns OLB_ETIMEOUT; the
 * state is then invalid, and steps and reads return OLB_ETIMEOUT until a new
 * state is written (olb_init_fields, olb_set_populations, olb_set_state).
 * OLB_EINVAL for a null handle. */
int olb_set_wait_polls(olb_handle h, long long polls);

/* ---- Adjoint of the isothermal step (vector-Jacobian products) ----------------------------
 * The paper defines the forward step only (Sec. 3: pull by Eq. sl_streaming, BGK with the
 * Hermite equilibrium of Appendix A).  These calls give the exact transpose of its Jacobian
 * for the isothermal step (compressible = 0), FP64 or FP32 storage, p = 3 or 4, N = 2 or 3
 * (N = 2 for D3Q45), with the automatic kernel choice; other configurations return
 * OLB_EUNSUPPORTED.
 *
 * Adjoint arrays ("lambda") are compact [Q][nz][ny][nx], x fastest, in the adjoint type:
 * double for FP64 storage, float for FP32 storage; lambda_i(x) = dJ/df_i(x) of the
 * unshifted populations.  on_device = 1: device pointers on the handle's stream (the call is
 * asynchronous); 0: host pointers (the call completes and checks the device error flag).
 *
 * olb_tape_reserve  allocate nslots tape slots on the device (kept until destroy).  A slot holds
 *                   the moments (rho, rho u) of the pulled populations of one step (4 values per
 *                   node, adjoint type): the transposed collision depends on the state only
 *                   through them, and the transposed pull on nothing.
 * olb_tape_record   n forward steps of the handle's state (it advances by n steps), step s
 *                   keeping its pulled moments in slot s - 1.  Needs n <= nslots.
 * olb_tape_adjoint  lambda in: dJ/d(state after the last recorded step); lambda out:
 *                   dJ/d(state n steps earlier), 1 <= n <= recorded steps.  n + 1 launches of
 *                   the adjoint kernel plus one scatter and one gather.
 * olb_adjoint_step  one step: fwd_state is the state before the step in the olb_get_state
 *                   layout (olb_state_bytes bytes); lambda in: dJ/d(state after the step),
 *                   out: dJ/d(fwd_state).  Runs one recorded forward step from fwd_state into
 *                   tape slot 0 (clears a recorded trajectory); the handle's state is kept.
 * olb_moments_vjp   seed of a sweep from dJ/drho and dJ/du at the handle's current state:
 *                   lambda_i = dJ/drho + dJ/du . (xi_i - u) / rho.  grad_rho [n] and grad_u
 *                   [D][n] (FP64, either may be NULL = zero).
 * olb_equilibrium_vjp  gradients of sum_i lambda_i f_i^eq(rho, u) with respect to rho [n] and
 *                   u [D][n] (FP64), the last link from lambda of an initial state built by
 *                   olb_init_fields (theta = 1). */
int olb_tape_reserve(olb_handle h, int nslots);
int olb_tape_record(olb_handle h, int n);
int olb_tape_adjoint(olb_handle h, void* lambda, int n, int on_device);
int olb_adjoint_step(olb_handle h, const void* fwd_state, void* lambda, int on_device);
int olb_moments_vjp(olb_handle h, const double* grad_rho, const double* grad_u, void* lambda, int on_device);
int olb_equilibrium_vjp(olb_handle h, const double* rho, const double* u, const void* lambda, double* grad_rho,
                        double* grad_u, int on_device);

/* Global sums of a state held by the caller, computed without allocating.
 * No counterpart in the paper: this is for callers that cannot allocate device
 * memory at the point where they need the sums (a framework that owns all
 * device memory through its own pool, or a loop that must not pay for
 * cudaMalloc's implicit synchronisation).  The per-block partial sums live in a
 * fixed array inside the library image (OLB_NOALLOC_MAX_BLOCKS x 8 doubles =
 * 128 KiB on every GPU that loads the library, kept until the process exits),
 * so the call allocates nothing.
 *   populations: device pointer, [Q][nz][ny][nx] storage values (the layout of
 *                olb_get_state for an isothermal state: shifted by w_i rho0
 *                unless storage is OLB_FP64).  Only these Q planes of f are
 *                read: for a compressible state pass its first Q planes; its
 *                g planes and temperature are not used (k_rho is mean
 *                rho |u|^2 / 2, which needs neither);
 *   rho0:        the reference density the state was shifted with (the
 *                handle's rho0 option); ignored for OLB_FP64;
 *   out:         device pointer to 8 doubles, filled like olb_reductions()
 *                with out[2] = NaN (no dissipation estimate without a step);
 *   stream:      cudaStream_t or NULL; the call only enqueues work on it.
 * Grids of more than OLB_NOALLOC_MAX_BLOCKS * OLB_NOALLOC_NODES_PER_BLOCK nodes
 * are rejected with OLB_EBOUNDS.  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.  The address is cached per device together with
 * the identity of the device's context; after a cudaDeviceReset the next call
 * looks it up again.  All calls share the array and each overwrites the slots
 * it uses, so calls whose kernels overlap on the GPU race. */
#define OLB_NOALLOC_MAX_BLOCKS 2048
#define OLB_NOALLOC_NODES_PER_BLOCK 65536
int olb_state_sums_noalloc(int velocity_set, const olb_grid* grid, int storage, double cs_scale,
                           double rho0, const void* populations, double* out, void* stream);

/* Measured FP64 FMA throughput of the current device, in flop/s (an FMA is two
 * flops): the denominator of the FP64 step's roofline, which the narrow FP64
 * pipe bounds rather than HBM (Sec. 3's step in FP64 storage).  Runs a fixed
 * FMA loop (8 independent chains per thread, 4 blocks of 256 threads per SM)
 * on `stream` (cudaStream_t or NULL), synchronises it, and returns the best of
 * three timed launches after a warm-up (about 0.2 s in all).  OLB_ECUDA if a
 * launch or an event fails. */
int olb_fp64_fma_peak(void* stream, double* flops_per_s);

/* Message for an error code, and the calling thread's most recent failure. */
const char* olb_strerror(int code);
const char* olb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OLB_H */
