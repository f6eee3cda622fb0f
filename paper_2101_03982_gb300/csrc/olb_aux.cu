// Auxiliary kernels around the fused step: equilibrium initialisation from
// macroscopic fields (Sec. 3 equilibrium with Appendix A moments), moments of
// a stored state, FP64 <-> storage conversion, compact <-> padded copies, and
// the fixed-order final sum of the per-CTA reduction partials.  None of them
// is on the per-step path.  Every writer also fills the periodic copies in the
// ghost layers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "olb_internal.h"
#include "olb_step.cuh"

namespace olb {

namespace {

template <typename S>
__device__ __forceinline__ S from_double(double v);
template <>
__device__ __forceinline__ double from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <>
__device__ __forceinline__ __half from_double<__half>(double v) { return __double2half(v); }

template <typename S>
__device__ __forceinline__ double to_double(S v) { return (double)Store<S>::ld(v); }

constexpr int AUX_NT = 256;

__device__ __forceinline__ void node_xyz(const Padded& P, long long node, int& x, int& y, int& z) {
  x = (int)(node % P.n[0]);
  const long long r = node / P.n[0];
  y = (int)(r % P.n[1]);
  z = (int)(r / P.n[1]);
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) init_kernel(const __grid_constant__ AuxArgs a, S* state, const double* rho,
                                                   const double* u, const double* theta) {
  const long long n = a.nnodes;
  const bool comp = a.compressible != 0;
  for (long long node = blockIdx.x * (long long)AUX_NT + threadIdx.x; node < n;
       node += (long long)gridDim.x * AUX_NT) {
    int x, y, z;
    node_xyz(a.pad, node, x, y, z);
    const double r = rho ? rho[node] : a.rest_rho;
    const double ux = rho ? u[node] : 0.0, uy = rho ? u[n + node] : 0.0;
    const double uz = (rho && a.D == 3) ? u[2 * n + node] : 0.0;
    const double th = (comp && theta) ? theta[node] : 1.0;
    const double uhx = ux * a.inv_cs, uhy = uy * a.inv_cs, uhz = uz * a.inv_cs;
    const double q = uhx * uhx + uhy * uhy + uhz * uhz;
    const double t = th - 1.0;
    const double A = r - a.rho_ref;
    const double rth = r * th, gA = r * t + A;
    for (int i = 0; i < a.Q; ++i) {
      const double xr = a.xih[i][0] * a.xih[i][0] + a.xih[i][1] * a.xih[i][1] + a.xih[i][2] * a.xih[i][2];
      const double rD = xr - a.D, rp = xr * xr - 2.0 * (a.D + 2) * xr + a.D * (a.D + 2.0);
      const double s = a.xih[i][0] * uhx + a.xih[i][1] * uhy + a.xih[i][2] * uhz;
      const double ph = comp ? phi_m1<double, true>(s, q, t, rD, rp, a.N) : phi_m1<double, false>(s, q, t, rD, rp, a.N);
      store_all_images(state + (long long)i * a.pad.plane, a.pad, x, y, z, from_double<S>(a.w[i] * (A + r * ph)));
      if (comp)
        store_all_images(state + (long long)(a.Q + i) * a.pad.plane, a.pad, x, y, z,
                         from_double<S>(a.w[i] * a.gfac * (gA + rth * ph)));
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) moments_kernel(const __grid_constant__ AuxArgs a, const S* state, double* rho,
                                                      double* u, double* theta, double* partials) {
  const long long n = a.nnodes;
  const bool comp = a.compressible != 0;
  double red[NRED];
  for (int q = 0; q < NRED; ++q) red[q] = 0.0;
  for (long long node = blockIdx.x * (long long)AUX_NT + threadIdx.x; node < n;
       node += (long long)gridDim.x * AUX_NT) {
    int x, y, z;
    node_xyz(a.pad, node, x, y, z);
    const long long off = pad_index(a.pad, x, y, z);
    double A = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, B = 0.0, G = 0.0;
    for (int i = 0; i < a.Q; ++i) {
      const double v = to_double(state[(long long)i * a.pad.plane + off]);
      A += v;
      jx += a.xi[i][0] * v;
      jy += a.xi[i][1] * v;
      jz += a.xi[i][2] * v;
      B += (a.xi[i][0] * a.xi[i][0] + a.xi[i][1] * a.xi[i][1] + a.xi[i][2] * a.xi[i][2]) * v;
      if (comp) G += to_double(state[(long long)(a.Q + i) * a.pad.plane + off]);
    }
    const double r = a.rho_ref + A;
    const double ux = jx / r, uy = jy / r, uz = jz / r;
    const double u2 = ux * ux + uy * uy + uz * uz;
    double th = 1.0;
    if (comp) th = 1.0 + (B + G - r * u2 - a.two_cv * A) / (a.two_cv * r);
    if (rho) rho[node] = r;
    if (u) {
      u[node] = ux;
      u[n + node] = uy;
      if (a.D == 3) u[2 * n + node] = uz;
    }
    if (theta) theta[node] = th;
    red[0] += 0.5 * u2;
    red[1] += 0.5 * r * u2;
    red[3] += A;
    red[4] += jx;
    red[5] += jy;
    red[6] += jz;
    red[7] += (isfinite(r) && isfinite(ux) && isfinite(uy) && isfinite(uz) && isfinite(th)) ? 0.0 : 1.0;
  }
  if (!partials) return;
  __shared__ double sm[AUX_NT / 32][NRED];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < NRED; ++q) {
    double v = red[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double s = 0.0;
    for (int w = 0; w < AUX_NT / 32; ++w) s += sm[w][threadIdx.x];
    partials[(size_t)blockIdx.x * NRED + threadIdx.x] = s;
  }
}

// Row-wise walk over the compact layout [plane][z][y][x]: one warp per
// (plane, z, y) row with its lanes along x, so that the compact and the padded
// accesses are both coalesced and the row's coordinates are divided out once
// per row instead of once per element.
template <typename F>
__device__ __forceinline__ void for_each_row(const AuxArgs& a, F&& f) {
  const long long rows = (long long)a.planes * a.pad.n[2] * a.pad.n[1];
  const long long nw = (long long)gridDim.x * (AUX_NT / 32);
  for (long long r = blockIdx.x * (long long)(AUX_NT / 32) + (threadIdx.x >> 5); r < rows; r += nw) {
    const long long pz = r / a.pad.n[1];
    f(r, (int)(pz / a.pad.n[2]), (int)(r % a.pad.n[1]), (int)(pz % a.pad.n[2]), (int)(threadIdx.x & 31));
  }
}

// Write one row of values (v(x) for x = lane, lane + 32, ...) at its nodes and
// at every periodic copy in the ghost layers.  Four loads per lane are issued
// before their stores, so that a source across the CPU-GPU link has enough
// requests in flight.
template <typename S, typename V>
__device__ __forceinline__ void store_row_images(S* plane, const Padded& P, int y, int z, int lane, V&& v) {
  const int fz = first_image(z, P.n[2], P.gl[2]), fy = first_image(y, P.n[1], P.gl[1]);
  for (int x0 = lane; x0 < P.n[0]; x0 += 128) {
    S val[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (x0 + 32 * k < P.n[0]) val[k] = v(x0 + 32 * k);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int x = x0 + 32 * k;
      if (x >= P.n[0]) break;
      const int fx = first_image(x, P.n[0], P.gl[0]);
      for (int cz = fz; cz < P.n[2] + P.gr[2]; cz += P.n[2])
        for (int cy = fy; cy < P.n[1] + P.gr[1]; cy += P.n[1]) {
          S* row = plane + pad_index(P, 0, cy, cz);
          for (int cx = fx; cx < P.n[0] + P.gr[0]; cx += P.n[0]) row[cx] = val[k];
        }
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) to_f64_kernel(const __grid_constant__ AuxArgs a, const S* state, double* f) {
  for_each_row(a, [&](long long r, int p, int y, int z, int lane) {
    const S* src = state + (long long)p * a.pad.plane + pad_index(a.pad, 0, y, z);
    const double b = a.base[p];
    for (int x = lane; x < a.pad.n[0]; x += 32) f[r * a.pad.n[0] + x] = to_double(src[x]) + b;
  });
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) from_f64_kernel(const __grid_constant__ AuxArgs a, S* state, const double* f) {
  for_each_row(a, [&](long long r, int p, int y, int z, int lane) {
    const double* src = f + r * a.pad.n[0];
    const double b = a.base[p];
    store_row_images(state + (long long)p * a.pad.plane, a.pad, y, z, lane,
                     [&](int x) { return from_double<S>(src[x] - b); });
  });
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) gather_kernel(const __grid_constant__ AuxArgs a, const S* state, S* compact) {
  for_each_row(a, [&](long long r, int p, int y, int z, int lane) {
    const S* src = state + (long long)p * a.pad.plane + pad_index(a.pad, 0, y, z);
    S* dst = compact + r * a.pad.n[0];
    for (int x = lane; x < a.pad.n[0]; x += 32) dst[x] = src[x];
  });
}

template <typename S>
__global__ void __launch_bounds__(AUX_NT) scatter_kernel(const __grid_constant__ AuxArgs a, S* state, const S* compact) {
  for_each_row(a, [&](long long r, int p, int y, int z, int lane) {
    const S* src = compact + r * a.pad.n[0];
    store_row_images(state + (long long)p * a.pad.plane, a.pad, y, z, lane, [&](int x) { return src[x]; });
  });
}

// Non-periodic x (inflow and outflow, the standing-shock set-up of Sec. 4.1):
// the ghost columns left of x = 0 hold the equilibrium of the inflow state
// (its post-collision populations), those right of x = nx - 1 repeat the last
// column (zero-gradient outflow).
//
// The inflow value of every plane, in storage form, computed once when the
// boundary is set (one thread per plane; FP64 as the initialisation).
template <typename S>
__global__ void xbc_values_kernel(const __grid_constant__ AuxArgs a, XInflow in, S* vals) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.planes) return;
  const bool comp = a.compressible != 0;
  const double uhx = in.u[0] * a.inv_cs, uhy = in.u[1] * a.inv_cs, uhz = in.u[2] * a.inv_cs;
  const double q = uhx * uhx + uhy * uhy + uhz * uhz;
  const double r = in.rho, th = comp ? in.theta : 1.0, t = th - 1.0, A = r - a.rho_ref;
  const int i = p < a.Q ? p : p - a.Q;
  const double xr = a.xih[i][0] * a.xih[i][0] + a.xih[i][1] * a.xih[i][1] + a.xih[i][2] * a.xih[i][2];
  const double rD = xr - a.D, rp = xr * xr - 2.0 * (a.D + 2) * xr + a.D * (a.D + 2.0);
  const double s = a.xih[i][0] * uhx + a.xih[i][1] * uhy + a.xih[i][2] * uhz;
  const double ph = comp ? phi_m1<double, true>(s, q, t, rD, rp, a.N) : phi_m1<double, false>(s, q, t, rD, rp, a.N);
  vals[p] = from_double<S>(p < a.Q ? a.w[i] * (A + r * ph) : a.w[i] * a.gfac * (r * t + A + r * th * ph));
}

// The ghost fill, after every writer of the state: one warp per padded
// (plane, z, y) row, ghost rows included.
template <typename S>
__global__ void __launch_bounds__(AUX_NT) xbc_kernel(const __grid_constant__ AuxArgs a, S* state, const S* vals) {
  const Padded& P = a.pad;
  const long long rows_pp = (long long)P.np[1] * P.np[2];
  const long long rows = (long long)a.planes * rows_pp;
  const long long nw = (long long)gridDim.x * (AUX_NT / 32);
  const int lane = threadIdx.x & 31;
  for (long long row = blockIdx.x * (long long)(AUX_NT / 32) + (threadIdx.x >> 5); row < rows; row += nw) {
    const int p = (int)(row / rows_pp);
    S* line = state + (long long)p * P.plane + (row - (long long)p * rows_pp) * P.np[0];
    const S vin = vals[p];
    for (int k = lane; k < P.gl[0]; k += 32) line[k] = vin;
    const S last = line[P.gl[0] + P.n[0] - 1];
    for (int k = lane; k < P.gr[0]; k += 32) line[P.gl[0] + P.n[0] + k] = last;
  }
}

// Periodic ghost copies rewritten in place: one warp per padded (plane, z, y)
// row; every ghost cell takes the interior value of its periodic image.  Only
// interior cells are read and only ghost cells are written, so the rows can
// run in any order.
template <typename S>
__global__ void __launch_bounds__(AUX_NT) periodic_ghost_kernel(const __grid_constant__ AuxArgs a, S* state) {
  const Padded& P = a.pad;
  const long long rows_pp = (long long)P.np[1] * P.np[2];
  const long long rows = (long long)a.planes * rows_pp;
  const long long nw = (long long)gridDim.x * (AUX_NT / 32);
  const int lane = threadIdx.x & 31;
  auto image = [](int c, int n) { return ((c % n) + n) % n; };
  for (long long row = blockIdx.x * (long long)(AUX_NT / 32) + (threadIdx.x >> 5); row < rows; row += nw) {
    const int p = (int)(row / rows_pp);
    const long long r = row - (long long)p * rows_pp;
    const int yy = (int)(r % P.np[1]) - P.gl[1], zz = (int)(r / P.np[1]) - P.gl[2];
    const bool ghost_row = yy < 0 || yy >= P.n[1] || zz < 0 || zz >= P.n[2];
    S* plane = state + (long long)p * P.plane;
    S* line = plane + r * P.np[0];
    const S* src = plane + pad_index(P, 0, image(yy, P.n[1]), image(zz, P.n[2]));
    for (int k = lane; k < P.np[0]; k += 32) {
      const int xx = k - P.gl[0];
      if (ghost_row || xx < 0 || xx >= P.n[0]) line[k] = src[image(xx, P.n[0])];
    }
  }
}

// Seed of the adjoint sweep: lam_i = dJ/df_i for J(rho, u) given dJ/drho and
// dJ/du per node, with rho = sum f (Sec. 3) and d u/d f_i = (xi_i - u)/rho.
template <typename S, typename C>
__global__ void __launch_bounds__(AUX_NT) moments_vjp_kernel(const __grid_constant__ AuxArgs a, const S* state,
                                                          const double* grad_rho, const double* grad_u, C* lam) {
  const long long n = a.nnodes;
  for (long long node = blockIdx.x * (long long)AUX_NT + threadIdx.x; node < n;
       node += (long long)gridDim.x * AUX_NT) {
    int x, y, z;
    node_xyz(a.pad, node, x, y, z);
    const long long off = pad_index(a.pad, x, y, z);
    double A = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < a.Q; ++i) {
      const double v = to_double(state[(long long)i * a.pad.plane + off]);
      A += v;
      jx += a.xi[i][0] * v;
      jy += a.xi[i][1] * v;
      jz += a.xi[i][2] * v;
    }
    const double r = a.rho_ref + A;
    const double ux = jx / r, uy = jy / r, uz = jz / r;
    const double gr = grad_rho ? grad_rho[node] : 0.0;
    const double gx = grad_u ? grad_u[node] : 0.0, gy = grad_u ? grad_u[n + node] : 0.0;
    const double gz = (grad_u && a.D == 3) ? grad_u[2 * n + node] : 0.0;
    const double gu = gx * ux + gy * uy + gz * uz;
    for (int i = 0; i < a.Q; ++i) {
      const double gxi = gx * a.xi[i][0] + gy * a.xi[i][1] + gz * a.xi[i][2];
      lam[(long long)i * n + node] = (C)(gr + (gxi - gu) / r);
    }
  }
}

// Gradients of sum_i lam_i f_i^eq(rho, u) (isothermal, Appendix A closed form
// of order N) with respect to rho and u per node:
//   d/drho = sum_i lam_i w_i (1 + Phi_i),
//   d/du   = (rho / c_s) sum_i lam_i w_i (dPhi/ds xi^_i + 2 dPhi/dq u^).
template <typename C>
__global__ void __launch_bounds__(AUX_NT) equilibrium_vjp_kernel(const __grid_constant__ AuxArgs a, const double* rho,
                                                              const double* u, const C* lam, double* grad_rho,
                                                              double* grad_u) {
  const long long n = a.nnodes;
  for (long long node = blockIdx.x * (long long)AUX_NT + threadIdx.x; node < n;
       node += (long long)gridDim.x * AUX_NT) {
    const double r = rho[node];
    const double uhx = u[node] * a.inv_cs, uhy = u[n + node] * a.inv_cs;
    const double uhz = a.D == 3 ? u[2 * n + node] * a.inv_cs : 0.0;
    const double q = uhx * uhx + uhy * uhy + uhz * uhz;
    double gr = 0.0, bx = 0.0, by = 0.0, bz = 0.0, bq = 0.0;
    for (int i = 0; i < a.Q; ++i) {
      const double s = a.xih[i][0] * uhx + a.xih[i][1] * uhy + a.xih[i][2] * uhz;
      double ph = s + 0.5 * (s * s - q), ps = 1.0 + s, pq = -0.5;
      if (a.N >= 3) {
        ph += s * (s * s - 3.0 * q) / 6.0;
        ps += 0.5 * (s * s - q);
        pq -= 0.5 * s;
      }
      if (a.N >= 4) {
        ph += (s * s * s * s - 6.0 * s * s * q + 3.0 * q * q) / 24.0;
        ps += s * (s * s - 3.0 * q) / 6.0;
        pq += 0.25 * (q - s * s);
      }
      const double v = a.w[i] * (double)lam[(long long)i * n + node];
      gr += v * (1.0 + ph);
      bx += v * ps * a.xih[i][0];
      by += v * ps * a.xih[i][1];
      bz += v * ps * a.xih[i][2];
      bq += 2.0 * v * pq;
    }
    const double f = r * a.inv_cs;
    grad_rho[node] = gr;
    grad_u[node] = f * (bx + bq * uhx);
    grad_u[n + node] = f * (by + bq * uhy);
    if (a.D == 3) grad_u[2 * n + node] = f * (bz + bq * uhz);
  }
}

// Enstrophy of the velocity field u ([D][n], FP64), Sec. 4.2: the mean of
// |curl u|^2 with fourth-order central differences on the periodic grid,
//   d/dx g ~ (g(x-2) - 8 g(x-1) + 8 g(x+1) - g(x+2)) / (12 dx).
// Per-block FP64 partials in slot 0 of NRED (the other slots are zero).
__device__ __forceinline__ double d4(const double* g, const Padded& P, int x, int y, int z, int axis, double inv12dx) {
  int c[3] = {x, y, z};
  double v[4];
  const int sh[4] = {-2, -1, 1, 2};
  for (int k = 0; k < 4; ++k) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[axis] = (cc[axis] + sh[k] + 2 * P.n[axis]) % P.n[axis];
    v[k] = g[((long long)cc[2] * P.n[1] + cc[1]) * P.n[0] + cc[0]];
  }
  return (v[0] - 8.0 * v[1] + 8.0 * v[2] - v[3]) * inv12dx;
}

__global__ void __launch_bounds__(AUX_NT) enstrophy_kernel(const __grid_constant__ AuxArgs a, const double* u,
                                                        double inv12dx, double* partials) {
  const long long n = a.nnodes;
  const double* ux = u;
  const double* uy = u + n;
  const double* uz = a.D == 3 ? u + 2 * n : nullptr;
  double acc = 0.0;
  for (long long node = blockIdx.x * (long long)AUX_NT + threadIdx.x; node < n;
       node += (long long)gridDim.x * AUX_NT) {
    int x, y, z;
    node_xyz(a.pad, node, x, y, z);
    const double wz = d4(uy, a.pad, x, y, z, 0, inv12dx) - d4(ux, a.pad, x, y, z, 1, inv12dx);
    double w2 = wz * wz;
    if (a.D == 3) {
      const double wx = d4(uz, a.pad, x, y, z, 1, inv12dx) - d4(uy, a.pad, x, y, z, 2, inv12dx);
      const double wy = d4(ux, a.pad, x, y, z, 2, inv12dx) - d4(uz, a.pad, x, y, z, 0, inv12dx);
      w2 += wx * wx + wy * wy;
    }
    acc += w2;
  }
  __shared__ double sm[AUX_NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (threadIdx.x < NRED) {
    double s = 0.0;
    if (threadIdx.x == 0)
      for (int w = 0; w < AUX_NT / 32; ++w) s += sm[w];
    partials[(size_t)blockIdx.x * NRED + threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(256) reduce_final_kernel(const double* partials, int nslots, double* out) {
  __shared__ double sm[256];
  for (int q = 0; q < NRED; ++q) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nslots; k += 256) s += partials[(size_t)k * NRED + q];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sm[0];
    __syncthreads();
  }
}

int aux_grid(long long work) {
  long long g = (work + AUX_NT - 1) / AUX_NT;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

// One warp per (plane, z, y) row.
int row_grid(const AuxArgs& a) { return aux_grid((long long)a.planes * a.pad.n[2] * a.pad.n[1] * 32); }

template <typename F>
int by_storage(int storage, F&& f) {
  switch (storage) {
    case 0: return f((double*)nullptr);
    case 1: return f((float*)nullptr);
    case 2: return f((__nv_bfloat16*)nullptr);
    case 3: return f((__half*)nullptr);
    default: return -1;
  }
}

}  // namespace

int launch_init_fields(const AuxArgs& a, void* state, const double* rho, const double* u, const double* theta,
                       void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    init_kernel<S><<<aux_grid(a.nnodes), AUX_NT, 0, (cudaStream_t)stream>>>(a, (S*)state, rho, u, theta);
    return (int)cudaGetLastError();
  });
}

int launch_state_moments(const AuxArgs& a, const void* state, double* rho, double* u, double* theta,
                         double* partials, int grid, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    moments_kernel<S><<<grid, AUX_NT, 0, (cudaStream_t)stream>>>(a, (const S*)state, rho, u, theta, partials);
    return (int)cudaGetLastError();
  });
}

int launch_to_f64(const AuxArgs& a, const void* state, double* f, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    to_f64_kernel<S><<<row_grid(a), AUX_NT, 0, (cudaStream_t)stream>>>(a, (const S*)state, f);
    return (int)cudaGetLastError();
  });
}

int launch_from_f64(const AuxArgs& a, void* state, const double* f, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    from_f64_kernel<S><<<row_grid(a), AUX_NT, 0, (cudaStream_t)stream>>>(a, (S*)state, f);
    return (int)cudaGetLastError();
  });
}

int launch_gather(const AuxArgs& a, const void* state, void* compact, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    gather_kernel<S><<<row_grid(a), AUX_NT, 0, (cudaStream_t)stream>>>(a, (const S*)state,
                                                                                                    (S*)compact);
    return (int)cudaGetLastError();
  });
}

int launch_scatter(const AuxArgs& a, void* state, const void* compact, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    scatter_kernel<S><<<row_grid(a), AUX_NT, 0, (cudaStream_t)stream>>>(a, (S*)state,
                                                                                                     (const S*)compact);
    return (int)cudaGetLastError();
  });
}

int launch_xbc_values(const AuxArgs& a, const XInflow& in, void* vals, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    xbc_values_kernel<S><<<(a.planes + 127) / 128, 128, 0, (cudaStream_t)stream>>>(a, in, (S*)vals);
    return (int)cudaGetLastError();
  });
}

int launch_periodic_ghosts(const AuxArgs& a, void* state, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    const long long rows = (long long)a.planes * a.pad.np[1] * a.pad.np[2];
    periodic_ghost_kernel<S><<<aux_grid(rows * 32), AUX_NT, 0, (cudaStream_t)stream>>>(a, (S*)state);
    return (int)cudaGetLastError();
  });
}

int launch_xbc(const AuxArgs& a, void* state, const void* vals, void* stream) {
  return by_storage(a.storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    const long long rows = (long long)a.planes * a.pad.np[1] * a.pad.np[2];
    xbc_kernel<S><<<aux_grid(rows * 32), AUX_NT, 0, (cudaStream_t)stream>>>(a, (S*)state, (const S*)vals);
    return (int)cudaGetLastError();
  });
}

int launch_moments_vjp(const AuxArgs& a, const void* state, const double* grad_rho, const double* grad_u, void* lam,
                       void* stream) {
  const int g = aux_grid(a.nnodes);
  if (a.storage == 0) {
    moments_vjp_kernel<double, double><<<g, AUX_NT, 0, (cudaStream_t)stream>>>(a, (const double*)state, grad_rho,
                                                                             grad_u, (double*)lam);
  } else if (a.storage == 1) {
    moments_vjp_kernel<float, float><<<g, AUX_NT, 0, (cudaStream_t)stream>>>(a, (const float*)state, grad_rho, grad_u,
                                                                           (float*)lam);
  } else {
    return -1;
  }
  return (int)cudaGetLastError();
}

int launch_equilibrium_vjp(const AuxArgs& a, const double* rho, const double* u, const void* lam, double* grad_rho,
                           double* grad_u, void* stream) {
  const int g = aux_grid(a.nnodes);
  if (a.storage == 0) {
    equilibrium_vjp_kernel<double><<<g, AUX_NT, 0, (cudaStream_t)stream>>>(a, rho, u, (const double*)lam, grad_rho,
                                                                         grad_u);
  } else if (a.storage == 1) {
    equilibrium_vjp_kernel<float><<<g, AUX_NT, 0, (cudaStream_t)stream>>>(a, rho, u, (const float*)lam, grad_rho,
                                                                        grad_u);
  } else {
    return -1;
  }
  return (int)cudaGetLastError();
}

int launch_enstrophy(const AuxArgs& a, const double* u, double dx, double* partials, int grid, void* stream) {
  enstrophy_kernel<<<grid, AUX_NT, 0, (cudaStream_t)stream>>>(a, u, 1.0 / (12.0 * dx), partials);
  return (int)cudaGetLastError();
}

int launch_reduce_final(const double* partials, int nslots, double* out, void* stream) {
  reduce_final_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(partials, nslots, out);
  return (int)cudaGetLastError();
}

}  // namespace olb
