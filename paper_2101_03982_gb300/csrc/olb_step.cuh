// Fused semi-Lagrangian pull + collide step (the hot path), sm_103a.
//
// Each population plane lives in HBM with ghost layers that hold periodic
// copies of the opposite faces, so the stencil box of any tile is a plain
// in-bounds block.  One CTA owns a tile of nodes (3D: 32 x 8 x 8, 2D: 32 x 64)
// and walks the planes in order.  For plane i one thread issues a TMA tiled
// copy (cp.async.bulk.tensor, completion on an mbarrier) of the tile plus the
// stencil halo of velocity i into shared memory; the copy of plane i+1 is in
// flight while plane i is interpolated.  The separable 1D Lagrange passes
// z -> y -> x (Sec. 3, Eq. sl_streaming, uniform-grid form; an axis with
// xi_{i,alpha} = 0 is the identity and is skipped) run on 4-node x groups with
// 128-bit shared-memory accesses.  Each thread owns four consecutive x nodes:
// it accumulates the moments of Sec. 3 and parks the pulled values f~_i in a
// per-CTA staging slab that stays in L2.  After the last plane the thread
// reads its f~_i back, forms the Hermite equilibrium of Appendix A in closed
// form, relaxes with BGK (Sec. 3) and writes the new state with 128-bit stores
// (plus the periodic copies of boundary nodes).  Optional global sums (kinetic
// energy, dissipation estimate, mass, momentum, non-finite count) are reduced
// per warp and tile, then per CTA in FP64 in a fixed order.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

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

// ---- four consecutive elements (one x group) -------------------------------
__device__ __forceinline__ void ld4(const float* p, float o[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double o[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float o[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const __half* p, float o[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float v[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<unsigned*>(&a);
  u.y = *reinterpret_cast<unsigned*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void st4(__half* p, const float v[4]) {
  __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<unsigned*>(&a);
  u.y = *reinterpret_cast<unsigned*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

constexpr int NT = 512;  // threads per CTA; each owns 4 consecutive x nodes

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

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int roundup(int a, int m) { return (a + m - 1) / m * m; }

template <int D, int P, typename S>
struct Layout {
  using C = typename Store<S>::C;
  static constexpr int TX = TileShape<D>::X, TY = TileShape<D>::Y, TZ = TileShape<D>::Z;
  static constexpr int TILE = TX * TY * TZ;
  static constexpr int VEC = 16 / (int)sizeof(S);     // elements per 16-byte TMA granule
  static constexpr int ALIGN = cmax(VEC, 4);          // x alignment of rows and boxes
  static constexpr int BXW = roundup(TX + P + VEC - 1, ALIGN);
  static constexpr int NQX = BXW / 4;                 // 4-element groups per box row
  static constexpr int BY = TY + P;
  static constexpr int BZ = D == 3 ? TZ + P : 1;
  static constexpr size_t BOXB = (size_t)roundup(BZ * BY * BXW * (int)sizeof(S), 128);
  static constexpr int BUFA = D == 3 ? TZ * BY * BXW : 0;
  static constexpr int BUFB = TZ * TY * BXW;
  static constexpr size_t OFF_A = 2 * BOXB;
  static constexpr size_t OFF_B = OFF_A + roundup(BUFA * (int)sizeof(C), 16);
  static constexpr size_t OFF_R = OFF_B + roundup(BUFB * (int)sizeof(C), 16);
  static constexpr size_t OFF_M = OFF_R + (NT / 32) * NRED * sizeof(double);
  static constexpr size_t BYTES = OFF_M + 2 * sizeof(unsigned long long) + 128;  // +128: base alignment
  static_assert(TILE == NT * 4, "each thread owns one 4-node x group");
  static_assert(28 + 4 * ((VEC - 1 + 3 + P) / 4 + 1) <= BXW, "x pass reads inside the box row");
};

// ---------------------------------------------------------------------------
// Velocity of the FP32 equilibrium.  With the abscissae and weights rounded to
// FP32, the tables' first moment sum_i w_i xi_i (xi_i / c_s) differs from c_s I
// by their rounding (1e-8 to 6e-8 relative).  An equilibrium built on
// u^ = j / (rho c_s) would then carry the momentum j (1 + g) instead of j, and
// the collision would scale the momentum by that factor at every step.  The
// host computes the diagonal correction (the tables are symmetric under the
// reflection of every axis, so the first moment is diagonal) and the velocity
// is u^_a = j_a r (1 - g_a) with r = fl(1/c_s) / rho.  The correction is below
// half an FP32 ulp, so it enters before the single rounding of an FMA: it then
// acts on average instead of being rounded away.  FP64 runs use j r.
// ---------------------------------------------------------------------------
template <bool COMP, typename C>
__device__ __forceinline__ C uhat_of(const StepArgs& a, C j, C r, int axis) {
  if constexpr (std::is_same<C, float>::value) {
    const float g = COMP ? a.f_gc[axis] : a.f_g[axis];
    return fmaf(j, r, j * (r * g));
  } else {
    return j * r;
  }
}
__device__ __forceinline__ float2 uhat2_of(const StepArgs& a, float2 j, float2 r, int axis) {
  const float2 g = make_float2(a.f_g[axis], a.f_g[axis]);
  return __ffma2_rn(j, r, __fmul2_rn(j, __fmul2_rn(r, g)));
}

// ---------------------------------------------------------------------------
// mbarrier / TMA helpers (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the copy did not land within `limit` polls (the
// default bound, 2^24 polls, is far beyond any copy's latency).
constexpr long long WAIT_POLLS_DEFAULT = 1LL << 24;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  long long limit = WAIT_POLLS_DEFAULT) {
  for (long long spin = 0; spin < limit; ++spin)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];\n" ::"l"(
                   reinterpret_cast<unsigned long long>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
}

// L2 eviction policies: the staging slab is reused within a tile (keep), the
// new state is not read again by this launch (stream through).
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void stg16(void* p, uint4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void stg8(void* p, uint2 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;\n" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint4 ldg16(const void* p, unsigned long long pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}

// Four values of the arithmetic type to / from global memory with a policy.
__device__ __forceinline__ void gst4(float* p, const float v[4], unsigned long long pol) {
  stg16(p, make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3])),
        pol);
}
__device__ __forceinline__ void gst4(double* p, const double v[4], unsigned long long pol) {
  const unsigned long long a = __double_as_longlong(v[0]), b = __double_as_longlong(v[1]);
  const unsigned long long c = __double_as_longlong(v[2]), d = __double_as_longlong(v[3]);
  stg16(p, make_uint4((unsigned)a, (unsigned)(a >> 32), (unsigned)b, (unsigned)(b >> 32)), pol);
  stg16(p + 2, make_uint4((unsigned)c, (unsigned)(c >> 32), (unsigned)d, (unsigned)(d >> 32)), pol);
}
__device__ __forceinline__ void gst4(__nv_bfloat16* p, const float v[4], unsigned long long pol) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
  stg8(p, make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b)), pol);
}
__device__ __forceinline__ void gst4(__half* p, const float v[4], unsigned long long pol) {
  __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
  stg8(p, make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b)), pol);
}
__device__ __forceinline__ void gld4(const float* p, float o[4], unsigned long long pol) {
  const uint4 v = ldg16(p, pol);
  o[0] = __uint_as_float(v.x); o[1] = __uint_as_float(v.y); o[2] = __uint_as_float(v.z); o[3] = __uint_as_float(v.w);
}
__device__ __forceinline__ void gld4(const double* p, double o[4], unsigned long long pol) {
  const uint4 a = ldg16(p, pol), b = ldg16(p + 2, pol);
  o[0] = __longlong_as_double(((unsigned long long)a.y << 32) | a.x);
  o[1] = __longlong_as_double(((unsigned long long)a.w << 32) | a.z);
  o[2] = __longlong_as_double(((unsigned long long)b.y << 32) | b.x);
  o[3] = __longlong_as_double(((unsigned long long)b.w << 32) | b.z);
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
// staging: one TMA copy per plane and tile
// ---------------------------------------------------------------------------
// Origin (padded coordinates) and shape variant of the box of `plane` for `tile`.
template <int D, int P, typename S, typename STT>
__device__ __forceinline__ int box_origin(const StepArgs& a, const STT& st, int plane, int tile, int& X, int& Y,
                                          int& Z) {
  using L = Layout<D, P, S>;
  const int i = plane < a.Q ? plane : plane - a.Q;
  const int tx = tile % a.nt[0], r = tile / a.nt[0];
  const int ty = r % a.nt[1], tz = r / a.nt[1];
  const int act = st.active[i];
  X = tx * L::TX + a.pad.gl[0] + ((act & 1) ? st.m0[i][0] : 0);
  X -= X % L::VEC;
  Y = ty * L::TY + a.pad.gl[1] + ((act & 2) ? st.m0[i][1] : 0);
  Z = D == 3 ? tz * L::TZ + a.pad.gl[2] + ((act & 4) ? st.m0[i][2] : 0) : 0;
  return ((act & 2) ? 1 : 0) | ((D == 3 && (act & 4)) ? 2 : 0);
}

template <int D, int P, typename S, typename STT>
__device__ __forceinline__ void issue_box(S* dst, unsigned long long* bar, const CUtensorMap* maps4,
                                          const StepArgs& a, const STT& st, int plane, int tile) {
  using L = Layout<D, P, S>;
  int X, Y, Z;
  const int v = box_origin<D, P, S>(a, st, plane, tile, X, Y, Z);
  const unsigned bytes = (unsigned)(L::BXW * ((v & 1) ? L::BY : L::TY) * ((v & 2) ? L::BZ : L::TZ) * sizeof(S));
  mbar_expect_tx(bar, bytes);
  tma_load_4d(dst, &maps4[v], X, Y, Z, plane, bar);
}

// Warm L2 with the box of a plane staged PREFETCH planes later.
constexpr int PREFETCH = 8;
template <int D, int P, typename S, typename STT>
__device__ __forceinline__ void prefetch_box(const CUtensorMap* maps4, const StepArgs& a, const STT& st, int plane,
                                             int tile) {
  while (plane >= a.planes) {
    plane -= a.planes;
    tile += gridDim.x;
  }
  if (tile >= a.ntiles) return;
  int X, Y, Z;
  const int v = box_origin<D, P, S>(a, st, plane, tile, X, Y, Z);
  tma_prefetch_4d(&maps4[v], X, Y, Z, plane);
}

// ---------------------------------------------------------------------------
// separable passes on 4-element x groups
// ---------------------------------------------------------------------------
// z pass: box [TZ+P][BYA][BXW] (S) -> bufA [TZ][BYA][BXW] (C)
template <int D, int P, typename S, int BYA>
__device__ __forceinline__ void zpass(const S* box, typename Store<S>::C* bufA, const typename Store<S>::C* W) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  constexpr int ZCH = 2, NZC = L::TZ / ZCH;
  constexpr int ITEMS = L::NQX * BYA * NZC;
  constexpr int PL = BYA * L::BXW;
  for (int item = threadIdx.x; item < ITEMS; item += NT) {
    const int q = item % L::NQX, r = item / L::NQX, y = r % BYA, zc = r / BYA;
    const int off = (zc * ZCH * BYA + y) * L::BXW + 4 * q;
    C v[ZCH + P][4];
#pragma unroll
    for (int k = 0; k < ZCH + P; ++k) ld4(box + off + k * PL, v[k]);
#pragma unroll
    for (int z = 0; z < ZCH; ++z) {
      C o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        C acc = W[0] * v[z][e];
#pragma unroll
        for (int k = 1; k <= P; ++k) acc = fma(W[k], v[z + k][e], acc);
        o[e] = acc;
      }
      st4(bufA + off + z * PL, o);
    }
  }
}

// y pass: src [TZ][BY][BXW] (S box or C bufA) -> bufB [TZ][TY][BXW] (C)
template <int D, int P, typename S, typename SRC>
__device__ __forceinline__ void ypass(const SRC* src, typename Store<S>::C* bufB, const typename Store<S>::C* W) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  constexpr int YCH = 2, NYC = L::TY / YCH;
  constexpr int ITEMS = L::NQX * L::TZ * NYC;
  for (int item = threadIdx.x; item < ITEMS; item += NT) {
    const int q = item % L::NQX, r = item / L::NQX, yc = r % NYC, z = r / NYC;
    const SRC* s = src + (z * L::BY + yc * YCH) * L::BXW + 4 * q;
    C v[YCH + P][4];
#pragma unroll
    for (int k = 0; k < YCH + P; ++k) ld4(s + k * L::BXW, v[k]);
    C* o = bufB + (z * L::TY + yc * YCH) * L::BXW + 4 * q;
#pragma unroll
    for (int y = 0; y < YCH; ++y) {
      C w4[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        C acc = W[0] * v[y][e];
#pragma unroll
        for (int k = 1; k <= P; ++k) acc = fma(W[k], v[y + k][e], acc);
        w4[e] = acc;
      }
      st4(o + y * L::BXW, w4);
    }
  }
}

// x pass into the thread's four nodes: src [..][TY][BXW]; XO = first needed
// column of the group inside the 16-byte aligned box row.
template <int D, int P, typename S, int XO, bool XACT, typename SRC>
__device__ __forceinline__ void xpass(const SRC* src, int qx, int ly, int lz, const typename Store<S>::C* W,
                                      typename Store<S>::C out[4]) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  const SRC* s = src + (lz * L::TY + ly) * L::BXW + qx;
  if (!XACT) {
    ld4(s, out);
    return;
  }
  constexpr int NQ = (XO + 3 + P) / 4 + 1;
  C v[NQ * 4];
#pragma unroll
  for (int k = 0; k < NQ; ++k) ld4(s + 4 * k, &v[4 * k]);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    C acc = W[0] * v[XO + e];
#pragma unroll
    for (int j = 1; j <= P; ++j) acc = fma(W[j], v[XO + e + j], acc);
    out[e] = acc;
  }
}

template <int D, int P, typename S, typename SRC, int XO>
__device__ __forceinline__ void xpass_dispatch_rec(int xo, const SRC* src, int qx, int ly, int lz,
                                                   const typename Store<S>::C* W, typename Store<S>::C out[4]) {
  if constexpr (XO < Layout<D, P, S>::VEC) {
    if (xo == XO) {
      xpass<D, P, S, XO, true>(src, qx, ly, lz, W, out);
      return;
    }
    xpass_dispatch_rec<D, P, S, SRC, XO + 1>(xo, src, qx, ly, lz, W, out);
  }
}

template <int D, int P, typename S, typename SRC>
__device__ __forceinline__ void xpass_any(bool xact, int xo, const SRC* src, int qx, int ly, int lz,
                                          const typename Store<S>::C* W, typename Store<S>::C out[4]) {
  if (!xact) {
    xpass<D, P, S, 0, false>(src, qx, ly, lz, W, out);
    return;
  }
  xpass_dispatch_rec<D, P, S, SRC, 0>(xo, src, qx, ly, lz, W, out);
}

// mu(theta) / (c_s^2 dt) of the power law mu theta^omega; omega = 0, the
// constant viscosity of Sec. 3, skips the power.
__device__ __forceinline__ float mu_theta(float mu_dt, float theta, float omega) {
  if (omega == 0.f) return mu_dt;
  return mu_dt * powf(theta, omega);
}
__device__ __forceinline__ double mu_theta(double mu_dt, double theta, double omega) {
  if (omega == 0.0) return mu_dt;
  return mu_dt * pow(theta, omega);
}

// ---------------------------------------------------------------------------
// periodic copies of a node in the ghost layers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int first_image(int c, int n, int gl) {
  return c - n * ((c + gl) / n);  // smallest c + k n that is >= -gl
}

// Store one value at node (x, y, z) and at every periodic copy of it that
// falls in the ghost layers.
template <typename S>
__device__ void store_all_images(S* plane, const Padded& P, int x, int y, int z, S v) {
  for (int cz = first_image(z, P.n[2], P.gl[2]); cz < P.n[2] + P.gr[2]; cz += P.n[2])
    for (int cy = first_image(y, P.n[1], P.gl[1]); cy < P.n[1] + P.gr[1]; cy += P.n[1])
      for (int cx = first_image(x, P.n[0], P.gl[0]); cx < P.n[0] + P.gr[0]; cx += P.n[0])
        plane[pad_index(P, cx, cy, cz)] = v;
}

// Copies (excluding the node itself) of a 4-node x group whose x coordinate
// and every ghost width are multiples of 4 (n[0] % 4 == 0).
template <typename S, typename C>
__device__ void store_group_images(S* plane, const Padded& P, int x, int y, int z, const C v[4]) {
  for (int cz = first_image(z, P.n[2], P.gl[2]); cz < P.n[2] + P.gr[2]; cz += P.n[2])
    for (int cy = first_image(y, P.n[1], P.gl[1]); cy < P.n[1] + P.gr[1]; cy += P.n[1])
      for (int cx = first_image(x, P.n[0], P.gl[0]); cx < P.n[0] + P.gr[0]; cx += P.n[0])
        if (cx != x || cy != y || cz != z) st4(plane + pad_index(P, cx, cy, cz), v);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int D, int P, typename S, bool COMP>
__global__ void __launch_bounds__(NT, 1)
    sl_step_kernel(const StepArgs a, const __grid_constant__ VelTab<typename Store<S>::C> vt,
                   const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st,
                   const __grid_constant__ TmaMaps maps) {
  using L = Layout<D, P, S>;
  using C = typename Store<S>::C;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base, kept as arithmetic on the shared array so that the
  // compiler addresses it as shared memory (no generic loads and stores)
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  S* boxes[2] = {reinterpret_cast<S*>(base), reinterpret_cast<S*>(base + L::BOXB)};
  C* bufA = reinterpret_cast<C*>(base + L::OFF_A);
  C* bufB = reinterpret_cast<C*>(base + L::OFF_B);
  double* red_smem = reinterpret_cast<double*>(base + L::OFF_R);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(base + L::OFF_M);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = a.Q, planes = a.planes;
  const Padded& pd = a.pad;
  const CUtensorMap* maps4 = maps.m[a.src];
  S* dst = static_cast<S*>(a.buf[a.src ^ 1]);
  C* scr = static_cast<C*>(a.scratch) + (size_t)blockIdx.x * planes * L::TILE + 4 * tid;

  // this thread's nodes: x = qx..qx+3, row ly, layer lz of the tile
  const int qx = (tid & 7) * 4;
  const int ly = D == 3 ? ((tid >> 3) & 7) : (tid >> 3);
  const int lz = D == 3 ? (tid >> 6) : 0;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < (NT / 32) * NRED) red_smem[tid] = 0.0;  // per-warp FP64 totals
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < a.ntiles) {
    issue_box<D, P, S>(boxes[0], &bars[0], maps4, a, st, 0, blockIdx.x);
    for (int k = 1; k < PREFETCH; ++k) prefetch_box<D, P, S>(maps4, a, st, k, blockIdx.x);
  }
  const unsigned long long keep = policy_evict_last(), stream_out = policy_evict_first();

  int buf = 0;
  unsigned parity = 0;  // bit b: phase of bars[b]
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int tx = tile % a.nt[0], tr = tile / a.nt[0];
    const int ty = tr % a.nt[1], tz = tr / a.nt[1];
    const int x0 = tx * L::TX + qx, y = ty * L::TY + ly, z = tz * L::TZ + lz;

    C Ad[4], jx[4], jy[4], jz[4], Bp[4], Gp[4];
    double Bd[4], Gd[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Ad[e] = jx[e] = jy[e] = jz[e] = Bp[e] = Gp[e] = C(0);
      Bd[e] = Gd[e] = 0.0;
    }

    for (int p = 0; p < planes; ++p) {
      const bool ok = mbar_wait_bounded(&bars[buf], (parity >> buf) & 1u, a.wait_polls);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(a.err, 1);
        mbar_wait_bounded(&bars[buf], (parity >> buf) & 1u);
        return;
      }
      parity ^= 1u << buf;
      if (tid == 0) {
        int np_ = p + 1, nt_ = tile;
        if (np_ == planes) {
          np_ = 0;
          nt_ = tile + gridDim.x;
        }
        if (nt_ < a.ntiles) {
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          issue_box<D, P, S>(boxes[buf ^ 1], &bars[buf ^ 1], maps4, a, st, np_, nt_);
        }
        prefetch_box<D, P, S>(maps4, a, st, p + PREFETCH, tile);
      }
      const S* box = boxes[buf];
      const int i = p < Q ? p : p - Q;
      const int act = st.active[i];
      C Wx[P + 1], Wy[P + 1], Wz[P + 1];
#pragma unroll
      for (int j = 0; j <= P; ++j) {
        Wx[j] = st.W[i][0][j];
        Wy[j] = st.W[i][1][j];
        Wz[j] = D == 3 ? st.W[i][2][j] : C(0);
      }
      const bool xact = act & 1;
      const int xo = xact ? ((st.m0[i][0] % L::VEC) + L::VEC) % L::VEC : 0;

      C out[4];
      if (D == 3 && (act & 4)) {
        if (act & 2) {
          zpass<D, P, S, L::BY>(box, bufA, Wz);
          __syncthreads();
          ypass<D, P, S>(static_cast<const C*>(bufA), bufB, Wy);
          __syncthreads();
          xpass_any<D, P, S>(xact, xo, static_cast<const C*>(bufB), qx, ly, lz, Wx, out);
        } else {
          zpass<D, P, S, L::TY>(box, bufA, Wz);
          __syncthreads();
          xpass_any<D, P, S>(xact, xo, static_cast<const C*>(bufA), qx, ly, lz, Wx, out);
        }
      } else if (act & 2) {
        ypass<D, P, S>(box, bufB, Wy);
        __syncthreads();
        xpass_any<D, P, S>(xact, xo, static_cast<const C*>(bufB), qx, ly, lz, Wx, out);
      } else {
        xpass_any<D, P, S>(xact, xo, box, qx, ly, lz, Wx, out);
      }
      buf ^= 1;

      // moments (Sec. 3) and staging of f~_i for the collision
      if (p < Q) {
        const C cx = vt.xi[i][0], cy = vt.xi[i][1], cz = D == 3 ? vt.xi[i][2] : C(0);
        const C c2 = vt.xi2[i];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          Ad[e] += out[e];
          jx[e] = fma(cx, out[e], jx[e]);
          jy[e] = fma(cy, out[e], jy[e]);
          if (D == 3) jz[e] = fma(cz, out[e], jz[e]);
          if (COMP) Bp[e] = fma(c2, out[e], Bp[e]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) Gp[e] += out[e];
      }
      if (COMP && ((p & 7) == 7 || p == planes - 1)) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          Bd[e] += (double)Bp[e];
          Gd[e] += (double)Gp[e];
          Bp[e] = Gp[e] = C(0);
        }
      }
      gst4(scr + (size_t)p * L::TILE, out, keep);
    }

    // ---- collision: equilibrium (Appendix A) and BGK (Sec. 3) -------------
    const bool yz_in = y < pd.n[1] && z < pd.n[2];
    bool vin[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) vin[e] = yz_in && (x0 + e) < pd.n[0];
    const bool group = a.quad_ok && vin[0];
    const bool images = yz_in && (x0 < pd.gr[0] || x0 + 4 > pd.n[0] - pd.gl[0] || y < pd.gr[1] ||
                                  y >= pd.n[1] - pd.gl[1] || z < pd.gr[2] || z >= pd.n[2] - pd.gl[2]);
    const long long main_off = pad_index(pd, x0, y, z);

    C rho[4], uhx[4], uhy[4], uhz[4], q[4], itau[4], tt[4], gA[4], rth[4], Pi[4][6];
    C rtheta[4], rtau[4];
    const C ics = C(a.inv_cs);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      rho[e] = C(a.rho_ref) + Ad[e];
      const C ir = ics / rho[e];
      uhx[e] = uhat_of<COMP>(a, jx[e], ir, 0);
      uhy[e] = uhat_of<COMP>(a, jy[e], ir, 1);
      uhz[e] = uhat_of<COMP>(a, jz[e], ir, 2);
      q[e] = uhx[e] * uhx[e] + uhy[e] * uhy[e] + uhz[e] * uhz[e];
      if (COMP) {
        // temperature relation (Sec. 3) in FP64: energy minus kinetic part cancels
        const double r = (double)rho[e];
        const double jj = (double)jx[e] * jx[e] + (double)jy[e] * jy[e] + (double)jz[e] * jz[e];
        const double X = Bd[e] + Gd[e] - jj / r - a.two_cv * (double)Ad[e];
        const C thm1 = C(X) / (C(a.two_cv) * rho[e]);
        const C theta = C(1) + thm1;
        const C tau = mu_theta(C(a.mu_dt), theta, C(a.mu_exp)) / (rho[e] * theta) + C(0.5);
        itau[e] = C(1) / tau;
        tt[e] = thm1;
        gA[e] = fma(rho[e], thm1, Ad[e]);
        rth[e] = rho[e] * theta;
        rtheta[e] = theta;
        rtau[e] = tau;
      } else {
        itau[e] = C(a.inv_tau);
        tt[e] = gA[e] = rth[e] = C(0);
        rtheta[e] = C(1);
        rtau[e] = C(a.tau);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) Pi[e][c] = C(0);
    }

    // Pr != 1: the heat-flux quasi-equilibrium (Sec. 3 compressible model).
    // The pulled f's central heat flux H = sum_i f_i zeta^_i |zeta^_i|^2 and
    // g's central first moment Gh = sum_i g_i zeta^_i (zeta^ = xi^ - u^, the
    // equilibria contribute none: N >= 3, degree >= 7), with the shifted
    // storage's w rho0 parts added in closed form (sum_i w_i zeta^_i
    // |zeta^_i|^2 = -u^ (D + 2 + |u^|^2), sum_i w_i zeta^_i = -u^).  The
    // collision then adds (1/tau - 1/tau_2) times their Hermite projections,
    //   w_i (H . xi^_i)(|xi^_i|^2 - D - 2) / (2 (D + 2))  and  w_i (Gh . xi^_i).
    C Fk[4][3], Gk[4][3];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int c = 0; c < 3; ++c) Fk[e][c] = Gk[e][c] = C(0);
    const bool qe = COMP && a.qe != 0;
    if (qe) {
      C H[4][3], Gh[4][3], Gs[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        Gs[e] = C(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) H[e][c] = Gh[e][c] = C(0);
      }
      for (int i = 0; i < Q; ++i) {
        C v[4], vg[4];
        gld4(scr + (size_t)i * L::TILE, v, keep);
        gld4(scr + (size_t)(Q + i) * L::TILE, vg, keep);
        const C xhx = vt.xih[i][0], xhy = vt.xih[i][1], xhz = D == 3 ? vt.xih[i][2] : C(0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const C zx = xhx - uhx[e], zy = xhy - uhy[e], zz = xhz - uhz[e];
          const C fz = v[e] * fma(zx, zx, fma(zy, zy, zz * zz));
          H[e][0] = fma(fz, zx, H[e][0]);
          H[e][1] = fma(fz, zy, H[e][1]);
          H[e][2] = fma(fz, zz, H[e][2]);
          Gh[e][0] = fma(vg[e], xhx, Gh[e][0]);
          Gh[e][1] = fma(vg[e], xhy, Gh[e][1]);
          Gh[e][2] = fma(vg[e], xhz, Gh[e][2]);
          Gs[e] += vg[e];
        }
      }
      const C rr = C(a.rho_ref), ipr = std::is_same<C, float>::value ? C(a.f_inv_pr) : C(a.inv_pr);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const C kap = itau[e] - C(1) / fma(rtau[e] - C(0.5), ipr, C(0.5));  // 1/tau - 1/tau_2
        const C hr = rr * (C(D + 2) + q[e]), gr = fma(C(a.gfac), rr, Gs[e]);
        const C uh[3] = {uhx[e], uhy[e], uhz[e]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Fk[e][c] = kap * C(0.5 / (D + 2)) * fma(-hr, uh[c], H[e][c]);
          Gk[e][c] = kap * fma(-gr, uh[c], Gh[e][c]);
        }
      }
    }

    const bool red = a.reduce != 0;
    // velocities in batches: the staging loads of a batch are all in flight
    // before the first one is used
    constexpr int BATCH = COMP ? 4 : 8;
    for (int i0 = 0; i0 < Q; i0 += BATCH) {
      C v[BATCH][4], vg[BATCH][4];
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        if (i0 + b >= Q) break;
        gld4(scr + (size_t)(i0 + b) * L::TILE, v[b], keep);
        if (COMP) gld4(scr + (size_t)(Q + i0 + b) * L::TILE, vg[b], keep);
      }
#pragma unroll
      for (int b = 0; b < BATCH; ++b) {
        const int i = i0 + b;
        if (i >= Q) break;
        const C wi = vt.w[i], xhx = vt.xih[i][0], xhy = vt.xih[i][1], xhz = D == 3 ? vt.xih[i][2] : C(0);
        const C rD = vt.rD[i], rp = vt.rpoly[i];
        C o[4], og[4], fneq[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const C s = fma(xhx, uhx[e], fma(xhy, uhy[e], xhz * uhz[e]));
          const C ph = phi_m1<C, COMP>(s, q[e], tt[e], rD, rp, a.N);
          const C eqv = fma(rho[e], ph, Ad[e]);  // A + rho Phi
          const C feqd = wi * eqv;
          fneq[e] = v[b][e] - feqd;
          // isothermal FP32: (1 - 1/tau) f + (w/tau)(A + rho Phi), the form whose
          // first moment the host's correction f_g makes exact (see uhat_of)
          if (!COMP && std::is_same<C, float>::value)
            o[e] = fma(C(1) - C(a.f_inv_tau), v[b][e], C(vt.wt[i]) * eqv);
          else
            o[e] = fma(-fneq[e], itau[e], v[b][e]);
          if (COMP) {
            const C geqd = wi * C(a.gfac) * fma(rth[e], ph, gA[e]);
            og[e] = fma(-(vg[b][e] - geqd), itau[e], vg[b][e]);
            if (qe) {
              o[e] = fma(wi * (rD - C(2)), fma(Fk[e][0], xhx, fma(Fk[e][1], xhy, Fk[e][2] * xhz)), o[e]);
              og[e] = fma(wi, fma(Gk[e][0], xhx, fma(Gk[e][1], xhy, Gk[e][2] * xhz)), og[e]);
            }
          }
        }
        S* pf = dst + (long long)i * pd.plane;
        S* pg = dst + (long long)(Q + i) * pd.plane;
        if (group) {
          gst4(pf + main_off, o, stream_out);
          if (COMP) gst4(pg + main_off, og, stream_out);
          if (images) {
            store_group_images(pf, pd, x0, y, z, o);
            if (COMP) store_group_images(pg, pd, x0, y, z, og);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (!vin[e]) continue;
            store_all_images(pf, pd, x0 + e, y, z, Store<S>::st(o[e]));
            if (COMP) store_all_images(pg, pd, x0 + e, y, z, Store<S>::st(og[e]));
          }
        }
        if (red) {
          C xx[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) xx[c] = vt.xx[i][c];
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int c = 0; c < 6; ++c) Pi[e][c] = fma(xx[c], fneq[e], Pi[e][c]);
        }
      }
    }

    if (red) {
      // per-thread sums over its nodes, then per warp, then FP64 per warp and tile
      C t[NRED];
#pragma unroll
      for (int c = 0; c < NRED; ++c) t[c] = C(0);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (!vin[e]) continue;
        const C u2 = q[e] * C(a.cs2);
        t[0] += C(0.5) * u2;
        t[1] += C(0.5) * rho[e] * u2;
        t[3] += Ad[e];
        t[4] += jx[e];
        t[5] += jy[e];
        t[6] += jz[e];
        const bool fin = isfinite(rho[e]) && isfinite(uhx[e]) && isfinite(uhy[e]) && isfinite(uhz[e]) &&
                         isfinite(rtheta[e]);
        t[7] += fin ? C(0) : C(1);
        const C pres = rho[e] * rtheta[e] * C(a.cs2);
        const C den = C(2) * pres * rtau[e] * C(a.dt);
        const C ss = (Pi[e][0] * Pi[e][0] + Pi[e][1] * Pi[e][1] + Pi[e][2] * Pi[e][2] +
                      C(2) * (Pi[e][3] * Pi[e][3] + Pi[e][4] * Pi[e][4] + Pi[e][5] * Pi[e][5])) /
                     (den * den);
        const C nu = C(a.cs2) * rtheta[e] * C(a.dt) * (rtau[e] - C(0.5));
        t[2] += C(2) * nu * ss;
      }
#pragma unroll
      for (int c = 0; c < NRED; ++c) {
        C v = t[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red_smem[warp * NRED + c] += (double)v;
      }
    }
  }

  // ---- per-CTA FP64 partials, fixed order -----------------------------------
  if (a.reduce) {
    __syncthreads();
    if (tid < NRED) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red_smem[w * NRED + tid];
      a.partials[(size_t)blockIdx.x * NRED + tid] = s;
    }
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
  kern<<<L.grid, NT, Lay::BYTES, static_cast<cudaStream_t>(L.stream)>>>(L.a, vt, st, *L.maps);
  return (int)cudaGetLastError();
}

template <int D, int P, typename S, bool COMP>
int occupancy_one(size_t* smem) {
  using Lay = Layout<D, P, S>;
  auto kern = sl_step_kernel<D, P, S, COMP>;
  *smem = Lay::BYTES;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, Lay::BYTES) != cudaSuccess) return 0;
  return n;
}

template <int D, int P, typename S>
void layout_of(StepInfo* o) {
  using Lay = Layout<D, P, S>;
  o->bxw = Lay::BXW;
  o->by = Lay::BY;
  o->bz = Lay::BZ;
  o->tile = Lay::TILE;
  o->tx = Lay::TX;
  o->ty = Lay::TY;
  o->tz = Lay::TZ;
  o->vec = Lay::VEC;
}

}  // namespace olb
