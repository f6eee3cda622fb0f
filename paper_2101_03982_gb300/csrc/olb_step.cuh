// Fused semi-Lagrangian pull + collide step (the hot path), sm_103a.
//
// One CTA owns a tile of nodes (3D: 32 x 8 x 8, 2D: 32 x 64) and walks the
// population planes one after another.  For plane i it stages the tile plus
// the stencil halo of velocity i in shared memory (16-byte cp.async copies,
// double buffered so that the next plane streams in while this one is
// interpolated), applies the separable 1D Lagrange passes z -> y -> x
// (skipping an axis with xi_{i,alpha} = 0, where the stencil is the identity),
// accumulates the moments of Sec. 3 in registers and parks the pulled value
// f~_i in a per-CTA staging slab that stays in L2.  After the last plane the
// same thread reads its own f~_i back, forms the Hermite equilibrium of
// Appendix A in closed form, relaxes with BGK (Sec. 3) and writes the next
// state with warp-coalesced stores.  Global sums (kinetic energy, dissipation
// estimate, mass, momentum, non-finite count) are reduced per CTA in FP64 in a
// fixed order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "olb_internal.h"

namespace olb {

template <typename S>
struct Store;
template <>
struct Store<double> {
  using C = double;
  __device__ static __forceinline__ double ld(double v) { return v; }
  __device__ static __forceinline__ double st(double v) { return v; }
};
template <>
struct Store<float> {
  using C = float;
  __device__ static __forceinline__ float ld(float v) { return v; }
  __device__ static __forceinline__ float st(float v) { return v; }
};
template <>
struct Store<__nv_bfloat16> {
  using C = float;
  __device__ static __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Store<__half> {
  using C = float;
  __device__ static __forceinline__ float ld(__half v) { return __half2float(v); }
  __device__ static __forceinline__ __half st(float v) { return __float2half_rn(v); }
};
template <typename C>
__device__ __forceinline__ C ldc(C v) {
  return v;
}

constexpr int NT = 512;  // threads per CTA
constexpr int NPT = 4;   // nodes per thread

template <int D>
struct TileShape;
template <>
struct TileShape<3> {
  static constexpr int X = 32, Y = 8, Z = 8;
};
template <>
struct TileShape<2> {
  static constexpr int X = 32, Y = 64, Z = 1;
};

template <int D, int P, typename S>
struct Layout {
  using C = typename Store<S>::C;
  static constexpr int TX = TileShape<D>::X, TY = TileShape<D>::Y, TZ = TileShape<D>::Z;
  static constexpr int TILE = TX * TY * TZ;
  static constexpr int VEC = 16 / (int)sizeof(S);
  static constexpr int BXW = ((TX + P + VEC - 1) + VEC - 1) / VEC * VEC;
  static constexpr int BY = TY + P;
  static constexpr int BZ = D == 3 ? TZ + P : 1;
  static constexpr int PL = BY * BXW;  // elements per z-plane of box and bufA
  static constexpr int BOX = BZ * PL;
  static constexpr int BUFA = D == 3 ? TZ * PL : 0;
  static constexpr int BUFB = TZ * TY * BXW;
  static constexpr size_t BYTES =
      2 * (size_t)BOX * sizeof(S) + (size_t)(BUFA + BUFB) * sizeof(C) + (NT / 32) * NRED * sizeof(double);
  static_assert(TILE == NT * NPT, "tile must be NT x NPT nodes");
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrap_mod(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// Local node k (0..NPT-1) of this thread inside the tile.
template <int D>
__device__ __forceinline__ void node_of(int k, int& lx, int& ly, int& lz) {
  const int local = threadIdx.x + NT * k;
  lx = local & 31;
  if (D == 3) {
    ly = (local >> 5) & 7;
    lz = local >> 8;
  } else {
    ly = local >> 5;
    lz = 0;
  }
}

// Hermite series of the equilibrium (Appendix A) contracted in closed form:
// f^eq_i / (w_i rho) - 1 for s = xi^_i . u^, q = |u^|^2, t = theta - 1,
// rD = |xi^_i|^2 - D, rpoly = r^2 - 2 (D+2) r + D (D+2).
template <typename C, bool COMP>
__device__ __forceinline__ C phi_m1(C s, C q, C t, C rD, C rpoly, int N) {
  const C s2 = s * s;
  C v = s;
  if (N >= 2) {
    C h = s2 - q;
    if (COMP) h = fma(t, rD, h);
    v = fma(C(0.5), h, v);
  }
  if (N >= 3) {
    C h = s * (s2 - C(3) * q);
    if (COMP) h = fma(C(3) * t * s, rD - C(2), h);
    v = fma(C(1.0 / 6.0), h, v);
  }
  if (N >= 4) {
    C h = s2 * s2 - C(6) * s2 * q + C(3) * q * q;
    if (COMP) h += C(6) * t * (s2 * (rD - C(4)) - q * (rD - C(2))) + C(3) * t * t * rpoly;
    v = fma(C(1.0 / 24.0), h, v);
  }
  return v;
}

// ---------------------------------------------------------------------------
// staging of one plane's box (tile + halo) into shared memory
// ---------------------------------------------------------------------------
template <int D, int P, typename S, int BYA, int BZA>
__device__ __forceinline__ void load_box(S* box, const S* plane, const StepArgs& a, int gx0, int gy0,
                                         int gz0) {
  using L = Layout<D, P, S>;
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  if (a.vec_ok) {
    constexpr int NV = L::BXW / L::VEC;
    constexpr int TOTAL = BZA * BYA * NV;
    for (int e = threadIdx.x; e < TOTAL; e += NT) {
      const int v = e % NV, r = e / NV, yy = r % BYA, zz = r / BYA;
      int gx = gx0 + v * L::VEC, gy = gy0 + yy, gz = gz0 + zz;
      if (a.tiny) {
        gx %= n0; gy %= n1; gz %= n2;
      } else {
        gx = gx >= n0 ? gx - n0 : gx;
        gy = gy >= n1 ? gy - n1 : gy;
        gz = gz >= n2 ? gz - n2 : gz;
      }
      cp_async16(box + (zz * L::BY + yy) * L::BXW + v * L::VEC,
                 plane + ((long long)gz * n1 + gy) * n0 + gx);
    }
  } else {
    constexpr int TOTAL = BZA * BYA * L::BXW;
    for (int e = threadIdx.x; e < TOTAL; e += NT) {
      const int x = e % L::BXW, r = e / L::BXW, yy = r % BYA, zz = r / BYA;
      const int gx = (gx0 + x) % n0, gy = (gy0 + yy) % n1, gz = (gz0 + zz) % n2;
      box[(zz * L::BY + yy) * L::BXW + x] = plane[((long long)gz * n1 + gy) * n0 + gx];
    }
  }
}

template <int D, int P, typename S, typename VT, typename STT>
__device__ __forceinline__ void stage_plane(S* box, const StepArgs& a, const STT& st, int plane, int tile) {
  using L = Layout<D, P, S>;
  const int i = plane < a.Q ? plane : plane - a.Q;
  const int tx = tile % a.nt[0], r = tile / a.nt[0];
  const int ty = r % a.nt[1], tz = r / a.nt[1];
  const int act = st.active[i];
  const int gxs = tx * L::TX + ((act & 1) ? st.m0[i][0] : 0);
  const int gys = ty * L::TY + ((act & 2) ? st.m0[i][1] : 0);
  const int gzs = tz * L::TZ + ((act & 4) ? st.m0[i][2] : 0);
  const int xa = gxs - wrap_mod(gxs, L::VEC);
  const int gx0 = wrap_mod(xa, a.n[0]), gy0 = wrap_mod(gys, a.n[1]), gz0 = D == 3 ? wrap_mod(gzs, a.n[2]) : 0;
  const S* src = static_cast<const S*>(a.src) + (long long)plane * a.nnodes;
  constexpr int BY1 = L::TY + P, BY0 = L::TY;
  constexpr int BZ1 = D == 3 ? L::TZ + P : 1, BZ0 = D == 3 ? L::TZ : 1;
  if (act & 2) {
    if (act & 4) load_box<D, P, S, BY1, BZ1>(box, src, a, gx0, gy0, gz0);
    else load_box<D, P, S, BY1, BZ0>(box, src, a, gx0, gy0, gz0);
  } else {
    if (act & 4) load_box<D, P, S, BY0, BZ1>(box, src, a, gx0, gy0, gz0);
    else load_box<D, P, S, BY0, BZ0>(box, src, a, gx0, gy0, gz0);
  }
}

// ---------------------------------------------------------------------------
// separable passes
// ---------------------------------------------------------------------------
template <int D, int P, typename S, int BYA>
__device__ __forceinline__ void zpass(const S* box, typename Store<S>::C* bufA, const typename Store<S>::C* Wz) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  constexpr int COLS = BYA * L::BXW;
  for (int col = threadIdx.x; col < COLS; col += NT) {
    C v[L::TZ + P];
#pragma unroll
    for (int k = 0; k < L::TZ + P; ++k) v[k] = Store<S>::ld(box[k * L::PL + col]);
#pragma unroll
    for (int z = 0; z < L::TZ; ++z) {
      C acc = Wz[0] * v[z];
#pragma unroll
      for (int k = 1; k <= P; ++k) acc = fma(Wz[k], v[z + k], acc);
      bufA[z * L::PL + col] = acc;
    }
  }
}

template <int D, int P, typename S, typename SRC, typename LD>
__device__ __forceinline__ void ypass(const SRC* src, typename Store<S>::C* bufB, const typename Store<S>::C* Wy,
                                      LD ld) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  constexpr int YCH = 8, NCH = L::TY / YCH;
  constexpr int ITEMS = L::TZ * NCH * L::BXW;
  for (int item = threadIdx.x; item < ITEMS; item += NT) {
    const int x = item % L::BXW, r = item / L::BXW, ch = r % NCH, z = r / NCH;
    const SRC* s = src + (z * L::BY + ch * YCH) * L::BXW + x;
    C v[YCH + P];
#pragma unroll
    for (int k = 0; k < YCH + P; ++k) v[k] = ld(s[k * L::BXW]);
    C* o = bufB + (z * L::TY + ch * YCH) * L::BXW + x;
#pragma unroll
    for (int y = 0; y < YCH; ++y) {
      C acc = Wy[0] * v[y];
#pragma unroll
      for (int k = 1; k <= P; ++k) acc = fma(Wy[k], v[y + k], acc);
      o[y * L::BXW] = acc;
    }
  }
}

template <int D, int P, typename S, int PY, typename SRC, typename LD>
__device__ __forceinline__ void xpass(const SRC* src, int xo, bool xact, const typename Store<S>::C* Wx,
                                      typename Store<S>::C out[NPT], LD ld) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    int lx, ly, lz;
    node_of<D>(k, lx, ly, lz);
    const SRC* s = src + (lz * PY + ly) * L::BXW + xo + lx;
    if (xact) {
      C acc = Wx[0] * ld(s[0]);
#pragma unroll
      for (int j = 1; j <= P; ++j) acc = fma(Wx[j], ld(s[j]), acc);
      out[k] = acc;
    } else {
      out[k] = ld(s[0]);
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool COMP>
__global__ void __launch_bounds__(NT, 1)
    sl_step_kernel(const StepArgs a, const __grid_constant__ VelTab<typename Store<S>::C> vt,
                   const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* boxes = reinterpret_cast<S*>(smem_raw);
  C* bufA = reinterpret_cast<C*>(smem_raw + 2 * (size_t)L::BOX * sizeof(S));
  C* bufB = bufA + L::BUFA;
  double* red_smem = reinterpret_cast<double*>(bufB + L::BUFB);

  const int Q = a.Q, planes = a.planes;
  C* scr = static_cast<C*>(a.scratch) + (size_t)blockIdx.x * planes * L::TILE;
  S* dst = static_cast<S*>(a.dst);
  const auto ldS = [](S v) { return Store<S>::ld(v); };
  const auto ldC = [](C v) { return v; };

  double red[NRED];
#pragma unroll
  for (int q = 0; q < NRED; ++q) red[q] = 0.0;

  int buf = 0;
  if ((int)blockIdx.x < a.ntiles) {
    stage_plane<D, P, S, VelTab<C>, StencilTab<C, P + 1>>(boxes, a, st, 0, blockIdx.x);
    cp_async_commit();
  }
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int tx = tile % a.nt[0], tr = tile / a.nt[0];
    const int ty = tr % a.nt[1], tz = tr / a.nt[1];
    const int x0 = tx * L::TX, y0 = ty * L::TY, z0 = tz * L::TZ;

    C Ad[NPT], jx[NPT], jy[NPT], jz[NPT];
    C Bp[NPT], Gp[NPT];          // compressible: per-group partial sums
    double Bd[NPT], Gd[NPT];     // compressible: FP64 totals
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      Ad[k] = jx[k] = jy[k] = jz[k] = C(0);
      Bp[k] = Gp[k] = C(0);
      Bd[k] = Gd[k] = 0.0;
    }

    for (int p = 0; p < planes; ++p) {
      S* box = boxes + buf * L::BOX;
      if (a.vec_ok) {
        cp_async_wait_all();
        __syncthreads();
        // stream the next plane (or the next tile's first plane) in behind this one
        if (p + 1 < planes) {
          stage_plane<D, P, S, VelTab<C>, StencilTab<C, P + 1>>(boxes + (buf ^ 1) * L::BOX, a, st, p + 1, tile);
        } else if (tile + (int)gridDim.x < a.ntiles) {
          stage_plane<D, P, S, VelTab<C>, StencilTab<C, P + 1>>(boxes + (buf ^ 1) * L::BOX, a, st, 0,
                                                                tile + gridDim.x);
        }
        cp_async_commit();
      } else {
        __syncthreads();
        if (p > 0 || tile != (int)blockIdx.x)
          stage_plane<D, P, S, VelTab<C>, StencilTab<C, P + 1>>(box, a, st, p, tile);
        __syncthreads();
      }

      const int i = p < Q ? p : p - Q;
      const int act = st.active[i];
      C Wx[P + 1], Wy[P + 1], Wz[P + 1];
#pragma unroll
      for (int j = 0; j <= P; ++j) {
        Wx[j] = st.W[i][0][j];
        Wy[j] = st.W[i][1][j];
        Wz[j] = D == 3 ? st.W[i][2][j] : C(0);
      }
      const int gxs = x0 + ((act & 1) ? st.m0[i][0] : 0);
      const int xo = wrap_mod(gxs, L::VEC);

      C out[NPT];
      if (D == 3 && (act & 4)) {
        if (act & 2) zpass<D, P, S, L::TY + P>(box, bufA, Wz);
        else zpass<D, P, S, L::TY>(box, bufA, Wz);
        __syncthreads();
        if (act & 2) {
          ypass<D, P, S>(bufA, bufB, Wy, ldC);
          __syncthreads();
          xpass<D, P, S, L::TY>(bufB, xo, act & 1, Wx, out, ldC);
        } else {
          xpass<D, P, S, L::BY>(bufA, xo, act & 1, Wx, out, ldC);
        }
      } else if (act & 2) {
        ypass<D, P, S>(box, bufB, Wy, ldS);
        __syncthreads();
        xpass<D, P, S, L::TY>(bufB, xo, act & 1, Wx, out, ldC);
      } else {
        xpass<D, P, S, L::BY>(box, xo, act & 1, Wx, out, ldS);
      }
      buf ^= 1;

      // moments (Sec. 3) and staging of f~_i for the collision
      if (p < Q) {
        const C cx = vt.xi[i][0], cy = vt.xi[i][1], cz = D == 3 ? vt.xi[i][2] : C(0);
        const C c2 = vt.xi2[i];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
          Ad[k] += out[k];
          jx[k] = fma(cx, out[k], jx[k]);
          jy[k] = fma(cy, out[k], jy[k]);
          if (D == 3) jz[k] = fma(cz, out[k], jz[k]);
          if (COMP) Bp[k] = fma(c2, out[k], Bp[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NPT; ++k) Gp[k] += out[k];
      }
      if (COMP && ((p & 7) == 7 || p == planes - 1)) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
          Bd[k] += (double)Bp[k];
          Gd[k] += (double)Gp[k];
          Bp[k] = Gp[k] = C(0);
        }
      }
#pragma unroll
      for (int k = 0; k < NPT; ++k) scr[p * L::TILE + threadIdx.x + NT * k] = out[k];
    }

    // ---- collision: equilibrium (Appendix A) and BGK (Sec. 3) -------------
    C rho[NPT], uhx[NPT], uhy[NPT], uhz[NPT], q[NPT], itau[NPT], tt[NPT], gA[NPT], rth[NPT];
    C Pi[NPT][6];
    bool inside[NPT];
    long long gidx[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      int lx, ly, lz;
      node_of<D>(k, lx, ly, lz);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      inside[k] = gx < a.n[0] && gy < a.n[1] && gz < a.n[2];
      gidx[k] = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
      rho[k] = C(a.rho_ref) + Ad[k];
      const C ir = C(1) / rho[k];
      const C ux = jx[k] * ir, uy = jy[k] * ir, uz = jz[k] * ir;
      const C ics = C(a.inv_cs);
      uhx[k] = ux * ics;
      uhy[k] = uy * ics;
      uhz[k] = uz * ics;
      q[k] = uhx[k] * uhx[k] + uhy[k] * uhy[k] + uhz[k] * uhz[k];
      double theta = 1.0, tau = a.tau;
      if (COMP) {
        const double r = (double)rho[k];
        const double u2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        const double thm1 = (Bd[k] + Gd[k] - r * u2 - a.two_cv * (double)Ad[k]) / (a.two_cv * r);
        theta = 1.0 + thm1;
        tau = a.mu_dt / (r * theta) + 0.5;
        itau[k] = C(1.0 / tau);
        tt[k] = C(thm1);
        gA[k] = C(r * thm1 + (double)Ad[k]);
        rth[k] = C(r * theta);
      } else {
        itau[k] = C(a.inv_tau);
        tt[k] = C(0);
        gA[k] = rth[k] = C(0);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) Pi[k][c] = C(0);
      if (inside[k]) {
        const double u2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        red[0] += 0.5 * u2;
        red[1] += 0.5 * (double)rho[k] * u2;
        red[3] += (double)rho[k];
        red[4] += (double)jx[k];
        red[5] += (double)jy[k];
        red[6] += (double)jz[k];
        const bool fin = isfinite((double)rho[k]) && isfinite((double)ux) && isfinite((double)uy) &&
                         isfinite((double)uz) && isfinite(theta);
        red[7] += fin ? 0.0 : 1.0;
        // tau and theta are needed again for the dissipation estimate below
        Bd[k] = theta;
        Gd[k] = tau;
      }
    }

    for (int i = 0; i < Q; ++i) {
      const C wi = vt.w[i], xhx = vt.xih[i][0], xhy = vt.xih[i][1], xhz = D == 3 ? vt.xih[i][2] : C(0);
      const C rD = vt.rD[i], rp = vt.rpoly[i];
      C xx[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) xx[c] = vt.xx[i][c];
      C v[NPT], vg[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        v[k] = scr[i * L::TILE + threadIdx.x + NT * k];
        if (COMP) vg[k] = scr[(Q + i) * L::TILE + threadIdx.x + NT * k];
      }
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const C s = fma(xhx, uhx[k], fma(xhy, uhy[k], xhz * uhz[k]));
        const C ph = phi_m1<C, COMP>(s, q[k], tt[k], rD, rp, a.N);
        const C feqd = wi * fma(rho[k], ph, Ad[k]);
        const C fneq = v[k] - feqd;
        const C post = fma(-fneq, itau[k], v[k]);
        if (inside[k]) dst[(long long)i * a.nnodes + gidx[k]] = Store<S>::st(post);
#pragma unroll
        for (int c = 0; c < 6; ++c) Pi[k][c] = fma(xx[c], fneq, Pi[k][c]);
        if (COMP) {
          const C geqd = wi * C(a.gfac) * fma(rth[k], ph, gA[k]);
          const C gpost = fma(-(vg[k] - geqd), itau[k], vg[k]);
          if (inside[k]) dst[(long long)(Q + i) * a.nnodes + gidx[k]] = Store<S>::st(gpost);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (!inside[k]) continue;
      const double theta = COMP ? Bd[k] : 1.0, tau = COMP ? Gd[k] : a.tau;
      const double pres = (double)rho[k] * theta * a.cs2;
      const double den = 2.0 * pres * tau * a.dt;
      const double ss = ((double)Pi[k][0] * Pi[k][0] + (double)Pi[k][1] * Pi[k][1] +
                         (double)Pi[k][2] * Pi[k][2] +
                         2.0 * ((double)Pi[k][3] * Pi[k][3] + (double)Pi[k][4] * Pi[k][4] +
                                (double)Pi[k][5] * Pi[k][5])) /
                        (den * den);
      const double nu = a.cs2 * theta * a.dt * (tau - 0.5);
      red[2] += 2.0 * nu * ss;
    }
  }

  // ---- per-CTA FP64 partials, fixed order -----------------------------------
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NRED; ++q) {
    double v = red[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red_smem[warp * NRED + q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red_smem[w * NRED + threadIdx.x];
    a.partials[(size_t)blockIdx.x * NRED + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers (instantiated per storage type)
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool COMP>
int launch_one(const StepLaunch& L) {
  using C = typename Store<S>::C;
  using Lay = Layout<D, P, S>;
  auto kern = sl_step_kernel<D, P, S, COMP>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
    if (e != cudaSuccess) return (int)e;
    attr_done = true;
  }
  const auto& vt = *static_cast<const VelTab<C>*>(L.veltab);
  const auto& st = *static_cast<const StencilTab<C, P + 1>*>(L.stentab);
  kern<<<L.grid, NT, Lay::BYTES, static_cast<cudaStream_t>(L.stream)>>>(L.a, vt, st);
  return (int)cudaGetLastError();
}

template <int D, int P, typename S, bool COMP>
int occupancy_one(size_t* smem) {
  using Lay = Layout<D, P, S>;
  auto kern = sl_step_kernel<D, P, S, COMP>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, Lay::BYTES) != cudaSuccess) return 0;
  *smem = Lay::BYTES;
  return n;
}

template <int D, int P, typename S>
void layout_of(int* bxw, int* by, int* bz, int* tile) {
  using Lay = Layout<D, P, S>;
  *bxw = Lay::BXW;
  *by = Lay::BY;
  *bz = Lay::BZ;
  *tile = Lay::TILE;
}

}  // namespace olb
