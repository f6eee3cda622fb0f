// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace olb {

constexpr int MAXQ = 45;       // largest velocity set (D3Q45)
constexpr int MAXPLANES = 90;  // f and g planes of D3Q45
constexpr int MAXP = 6;        // largest interpolation degree built
constexpr int NRED = 8;        // global reductions per step

struct VelocitySet {
  int Q, D, degree;
  double cs;
  double xi[MAXQ][3];
  double w[MAXQ];
};

// Fill *vs with the unscaled table of set `id` (olb_velocity_set); -1 if unknown.
int velocity_set(int id, VelocitySet* vs);

// Message returned by olb_last_error() for the calling thread.
void set_last_error(const std::string& msg);

// Device layout of one population plane: the interior n[0] x n[1] x n[2]
// nodes surrounded by ghost layers (gl on the low side, gr on the high side of
// each axis) that hold periodic copies, so that every staged box is a plain
// in-bounds tile.  np = gl + n + gr; np[0] keeps rows 16-byte aligned.
struct Padded {
  int n[3];
  int np[3];
  int gl[3];
  int gr[3];
  long long plane;  // np[0] * np[1] * np[2]
};

#if defined(__CUDACC__)
#define OLB_HD __host__ __device__ __forceinline__
#else
#define OLB_HD inline
#endif

OLB_HD long long pad_index(const Padded& P, int x, int y, int z) {
  return ((long long)(z + P.gl[2]) * P.np[1] + (y + P.gl[1])) * P.np[0] + (x + P.gl[0]);
}

// Per-velocity tables in the arithmetic type C of the step (kernel parameter).
template <typename C>
struct VelTab {
  C xi[MAXQ][3];   // abscissae (scaled)
  C xih[MAXQ][3];  // xi / c_s
  C w[MAXQ];
  C xi2[MAXQ];     // |xi|^2
  C rD[MAXQ];      // |xi/c_s|^2 - D
  C rpoly[MAXQ];   // r^2 - 2 (D+2) r + D (D+2), r = |xi/c_s|^2
  C xx[MAXQ][6];   // xi_a xi_b: xx, yy, zz, xy, xz, yz (2D: xx, yy, 0, xy, 0, 0)
  C wt[MAXQ];      // w / tau (isothermal)
};

// Fixed separable stencil of the pull: first support point and Lagrange
// weights per velocity and axis; bit a of active[i] set when xi_{i,a} != 0.
template <typename C, int P1>
struct StencilTab {
  int m0[MAXQ][3];
  int active[MAXQ];
  C W[MAXQ][3][P1];
};

// TMA descriptors of the two population buffers, one per staged box shape
// (bit 0: y extended by the stencil, bit 1: z extended).
struct TmaMaps {
  CUtensorMap m[2][4];
};

// Planes of each warpgroup of the two-phase step, balanced by the host.
struct WgSchedule {
  int n[4];
  unsigned char plane[4][MAXPLANES];
};

// Scalars of one step launch.
struct StepArgs {
  void* buf[2];         // population buffers (padded planes)
  int src;              // index of the current state in buf
  void* scratch;        // per-CTA staging of pulled populations
  void* slab;           // tape slab [tile][Q][tile nodes] of a recorded step: the forward step writes
                        // its pulled populations there, the adjoint reads them (null otherwise)
  double* partials;     // per-CTA reduction partials [grid][NRED]
  int* err;             // device error flag (1: a bounded wait ran out)
  long long wait_polls; // bound of the waits for staging copies (polls of the barrier)
  Padded pad;
  int nt[3];            // tiles per axis
  int ntiles;
  int Q, planes, N;
  int reduce;           // 1: accumulate the global sums this step
  int mode;             // adjoint kernel: 1 transposed collision, 2 transposed pull only
  int quad_ok;          // n[0] % 4 == 0: 4-node x groups never straddle the edge
  double rho_ref;       // rho0 for shifted storage, 0 for FP64
  double inv_tau;       // isothermal 1/tau
  double tau;           // isothermal tau
  double mu_dt;         // compressible: mu / (c_s^2 dt)
  double mu_exp;        // compressible: mu(theta) = mu theta^mu_exp
  int qe;               // compressible, Pr != 1: heat-flux quasi-equilibrium
  double inv_pr;        // 1 / Pr
  double two_cv;        // 2 C_v
  double gfac;          // 2 C_v - D
  double inv_cs;        // 1 / c_s
  double cs2;           // c_s^2
  double dt;
  // the same scalars rounded to FP32 for the FP32-arithmetic kernels (no
  // double-to-float conversions on the device)
  float f_rho_ref, f_inv_tau, f_tau, f_mu_dt, f_two_cv, f_gfac, f_inv_cs, f_cs2, f_dt, f_mu_exp, f_inv_pr;
  // FP32 equilibrium velocity u^_a = j_a fl(1/c_s) / rho (1 + g_a): the
  // rounding of the FP32 tables' first moment folded out (zero for FP64).
  // f_g for the isothermal BGK form (1 - 1/tau) f + (w/tau) e, f_gc for the
  // compressible form f - (f - w e) / tau.
  float f_g[3], f_gc[3];
};

// Launch of the fused step for storage `storage` (olb_storage); returns a
// cudaError_t value (0 on success) or -1 when the combination is not built.
struct StepLaunch {
  StepArgs a;
  int D, P, storage, compressible;
  const void* veltab;   // VelTab<C>
  const void* stentab;  // StencilTab<C, P+1>
  const void* stentab2; // adjoint kernel: stencil of the adjoint input (reflected or identity)
  const TmaMaps* maps;
  const WgSchedule* sched;
  int grid;             // CTAs
  int force_generic;    // 1: single-role kernel instead of the two-phase kernel
  void* stream;
};

// One pair of functions per storage and dimension (olb_step_<storage>_<D>d.cu).
int launch_step_f64_2d(const StepLaunch& L);
int launch_step_f64_3d(const StepLaunch& L);
int launch_step_f32_2d(const StepLaunch& L);
int launch_step_f32_3d(const StepLaunch& L);
int launch_step_bf16_2d(const StepLaunch& L);
int launch_step_bf16_3d(const StepLaunch& L);
int launch_step_f16_2d(const StepLaunch& L);
int launch_step_f16_3d(const StepLaunch& L);

// Shape and occupancy of the step kernel of a configuration: resident CTAs
// per SM, dynamic shared memory, staged box extents and nodes per tile.
struct StepInfo {
  int ctas_per_sm;
  size_t smem;
  int bxw, by, bz, tile, tx, ty, tz, vec;
  int wg;  // warpgroups of the two-phase kernel (0: the single-role kernel runs)
};
// Adjoint step of the isothermal two-phase kernel (FP64 and FP32 storage);
// -1 when the configuration is not built.
int launch_adj_f64_2d(const StepLaunch& L);
int launch_adj_f64_3d(const StepLaunch& L);
int launch_adj_f32_2d(const StepLaunch& L);
int launch_adj_f32_3d(const StepLaunch& L);

// mode: 0 the automatic choice (the two-phase kernel where it is built, else
// the single-role kernel), 1 the single-role kernel, 2 the two-phase kernel
// (the geometry of the adjoint).
int step_info_f64_2d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_f64_3d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_f32_2d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_f32_3d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_bf16_2d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_bf16_3d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_f16_2d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);
int step_info_f16_3d(int P, int comp, int Q, int N, int force_generic, StepInfo* out);

// Pull of the cell-wise interpolation on Gauss-Lobatto-Chebyshev points
// (olb_glc.cu): per velocity i, axis a and residue k = node mod p, the first
// support node relative to the node and the p + 1 Lagrange weights.
constexpr int GLC_PMAX = 8;
struct GlcArgs {
  Padded pad;
  long long nnodes;
  int planes, Q, D, p;
  int nt[3], ntiles;                // tiles per axis (glc_tile_shape) and their product
  int box_elems;                    // largest staged box (tile plus reach) over the velocities
  int b1_elems;                     // largest output of the x pass (tile width x box height x box depth)
  int vec16;                        // 1: stage with 16-byte copies (n[0] a multiple of 16 bytes' elements)
                                    // 16-bit storage: staged as stored, converted to FP32 in shared memory
  int active[MAXQ];                 // bit a: xi_{i,a} != 0
  int first[MAXQ * 3 * GLC_PMAX];   // [i][a][k]
  unsigned char lo[MAXQ * 3], hi[MAXQ * 3];  // [i][a] reach below and above the tile (0 when inactive)
  const void* W;                    // device [i][a][k][GLC_PMAX + 1], arithmetic type of the storage
};
// Tile of the GLC pull for dimension D and element size elem (8: FP64 arithmetic).
void glc_tile_shape(int D, int elem, int* tx, int* ty, int* tz);
// Dynamic shared memory of one CTA of the GLC pull (weights and two boxes).
// elem: arithmetic type; storage_elem: the stored type (16-bit storage adds its box).
size_t glc_smem_bytes(const GlcArgs& a, int elem, int storage_elem);
// storage 0 (FP64) or 1 (FP32); -1 for a storage not built.  Writes the pulled
// values of every plane of src into the interior of dst (padded layouts).
int launch_glc_pull(int storage, const GlcArgs& a, const void* src, void* dst, void* stream);

// Auxiliary kernels (olb_aux.cu).
struct AuxArgs {
  Padded pad;
  long long nnodes;         // interior nodes
  int Q, planes, D, N, storage, compressible;
  double rho_ref, gfac, two_cv, inv_cs, cs2;
  double rest_rho;          // init without fields: rho = rest_rho, u = 0, theta = 1
  double base[MAXPLANES];   // shift per plane (0 for FP64)
  double xi[MAXQ][3];
  double xih[MAXQ][3];
  double w[MAXQ];
};
int launch_init_fields(const AuxArgs& a, void* state, const double* rho, const double* u,
                       const double* theta, void* stream);
int launch_state_moments(const AuxArgs& a, const void* state, double* rho, double* u,
                         double* theta, double* partials, int grid, void* stream);
int launch_to_f64(const AuxArgs& a, const void* state, double* f, void* stream);
int launch_from_f64(const AuxArgs& a, void* state, const double* f, void* stream);
// Compact [plane][z][y][x] <-> padded state (raw storage values).
int launch_gather(const AuxArgs& a, const void* state, void* compact, void* stream);
int launch_scatter(const AuxArgs& a, void* state, const void* compact, void* stream);
int launch_reduce_final(const double* partials, int nslots, double* out, void* stream);
// Inflow state of the non-periodic x: rho, u (3 components, 0 beyond D), theta.
struct XInflow {
  double rho, u[3], theta;
};
// Inflow value of every plane in storage form (vals: planes elements).
int launch_xbc_values(const AuxArgs& a, const XInflow& in, void* vals, void* stream);
// Refill the x ghost columns: the inflow values on the left, copies of the
// last column on the right (every plane, every padded row).
int launch_xbc(const AuxArgs& a, void* state, const void* vals, void* stream);
// Every ghost copy of a state rewritten from its periodic image, in place.
int launch_periodic_ghosts(const AuxArgs& a, void* state, void* stream);
// Per-block partial sums of |curl u|^2 (slot 0 of NRED per block) of the
// velocity u [D][n] (FP64), fourth-order central differences of spacing dx.
int launch_enstrophy(const AuxArgs& a, const double* u, double dx, double* partials, int grid, void* stream);
// Adjoint seed and initial-state gradients (FP64 and FP32 storage; -1 otherwise).
// lam is compact [Q][z][y][x] in the adjoint type (double / float).
int launch_moments_vjp(const AuxArgs& a, const void* state, const double* grad_rho, const double* grad_u, void* lam,
                       void* stream);
int launch_equilibrium_vjp(const AuxArgs& a, const double* rho, const double* u, const void* lam, double* grad_rho,
                           double* grad_u, void* stream);

}  // namespace olb
