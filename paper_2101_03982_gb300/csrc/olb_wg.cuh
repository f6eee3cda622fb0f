// Two-phase fused step (the hot path), sm_103a.
//
// Same method, data layout and results as sl_step_kernel (olb_step.cuh):
// ghost-padded planes, TMA-staged boxes, separable z/y/x Lagrange passes
// (Sec. 3, Eq. sl_streaming), moments, Hermite equilibrium (Appendix A) and
// BGK (Sec. 3).  Per tile of nodes:
//
//   Phase A (pull).  The CTA is NWG independent warpgroups of 128 threads.
//   Each warpgroup owns a host-balanced list of planes and streams them
//   through its own shared-memory box (one TMA copy per plane, completion on
//   the warpgroup's mbarrier; L2 prefetch of the plane after next), its own
//   z -> y -> x passes (warpgroup-local named barriers only; the z and y
//   passes use paired FP32 FMAs) and writes the pulled values f~_i of the
//   tile to the CTA's staging slab (kept in L2).  No per-node state is carried
//   from plane to plane, so the warpgroups never wait for each other here.
//
//   Phase B (collide).  One thread per node loads its Q pulled values (all
//   loads in flight together), forms rho, rho u (and the temperature), the
//   order-N equilibrium and the BGK update with the velocity loop unrolled
//   (per-velocity constants are constant-bank operands), and stores the new
//   state together with its periodic copies in the ghost layers (offsets
//   computed once per node).
//
// Two CTA barriers per tile separate the phases.  Every mbarrier wait is
// bounded: a wait that runs out raises the device error flag and the kernel
// returns after its copies in flight have landed.
#pragma once

#include <type_traits>

#include "olb_step.cuh"

// Unroll factor of the velocity loops of the shared-memory staged collision
// (their values are read from shared memory, so the loops need not be fully
// unrolled; a rolled loop keeps the code within the instruction cache).
#ifndef OLB_STAGED_UNROLL
#define OLB_STAGED_UNROLL 3
#endif

namespace olb {
namespace wg {

constexpr int STAGED_UNROLL = OLB_STAGED_UNROLL;

constexpr int WGT = 128;  // threads per warpgroup

constexpr size_t roundup_sz(size_t a, size_t m) { return (a + m - 1) / m * m; }

template <int D, int P, typename S>
struct GLayout {
  using C = typename Store<S>::C;
  using B = Layout<D, P, S>;
  // tile of the two-phase kernel: x and y as the single-role kernel, z depth WG_TZ
  static constexpr int WG_TZ = 8;
  static constexpr int TX = B::TX, TY = B::TY, TZ = D == 3 ? WG_TZ : 1, TILE = TX * TY * TZ, VEC = B::VEC;
  static constexpr int BXW = B::BXW, NQX = B::NQX, BY = B::BY, BZ = D == 3 ? TZ + P : 1;
  // outputs per thread of the z and y passes (a column of the box; the inputs
  // slide through a window of P + 1 rows, each loaded once)
  static constexpr int ZC = TZ, YC = TY < 8 ? TY : 8;
  static constexpr size_t BOXB = (size_t)roundup(BZ * BY * BXW * (int)sizeof(S), 128);
  static constexpr size_t ABYTES = (size_t)roundup((D == 3 ? TZ * BY * BXW : 4) * (int)sizeof(C), 128);
  static constexpr size_t BBYTES = (size_t)roundup(TZ * TY * BXW * (int)sizeof(C), 128);
  // 3D with storage of the arithmetic type: two boxes per warpgroup, the z
  // and y passes write in place (each column belongs to one thread), the copy
  // of the next plane but one lands while a plane is processed
  static constexpr bool INPL = D == 3 && sizeof(S) == sizeof(C);
  // 3D with 16-bit storage: two boxes of the storage type and one work buffer
  // of the arithmetic type; the first pass converts the box into the work
  // buffer (the later passes run in place there), so the box takes the copy
  // of the plane after next as soon as that pass is done
  static constexpr bool TWO16 = D == 3 && sizeof(S) == 2;
  static constexpr bool TWOBOX = INPL || TWO16;
  static constexpr size_t WGB = INPL ? 2 * BOXB : TWO16 ? 2 * BOXB + ABYTES : BOXB + ABYTES + BBYTES;
  static constexpr size_t BUDGET = 227 * 1024 - 2048;
  // warpgroups per CTA (at most NWG_MAX); CTAS resident CTAs per SM share the 16 warps
  static constexpr int NWG_MAX = 4;
  static constexpr int NWG = (int)(BUDGET / WGB) >= NWG_MAX ? NWG_MAX : (int)(BUDGET / WGB);
  static constexpr int CTAS = NWG_MAX == 4 ? 1 : 4 / NWG_MAX;
  static constexpr int NT = NWG * WGT;
  static constexpr size_t OFF_R = NWG * WGB;
  static constexpr size_t OFF_M = OFF_R + (NT / 32) * NRED * sizeof(double);
  // two mbarriers per warpgroup (its boxes) and two for the shared-memory staging of phase B
  static constexpr size_t BYTES = OFF_M + (2 * NWG + 2) * sizeof(unsigned long long) + 128;
  static_assert(NWG >= 1, "one warpgroup must fit");
};

// Shared-memory staging of phase B.  The compressible FP32 sets and the
// isothermal sets of more than 27 velocities read their pulled values from
// shared memory instead of registers: after phase A the staging slab is
// copied, one chunk of CHN nodes at a time, into shared memory.  3D in-place
// kernels use their (then idle) boxes, double-buffered when two chunks fit;
// the 2D compressible kernels keep issuing box copies through phase B and
// get one dedicated chunk buffer after the rest of their shared memory.
template <int D, int P, typename S, bool COMP, int QM, bool ADJ>
struct Staging {
  using L = GLayout<D, P, S>;
  using C = typename Store<S>::C;
  static constexpr int SPMAX = COMP ? 2 * QM : QM;  // planes of a chunk
  // isothermal sets of more than 27 velocities: node pairs on the paired FP32
  // pipe, possible because the values come from shared memory, not registers
  static constexpr bool SPAIR = !COMP && QM > 27;
  static constexpr int CHN = SPAIR ? 2 * L::NT : L::NT;  // nodes of a chunk
  static constexpr size_t SCHB = (size_t)SPMAX * CHN * sizeof(C);
  static constexpr bool FP32 = !ADJ && std::is_same<C, float>::value && L::TILE % CHN == 0;
  static constexpr bool IN_BOXES = FP32 && L::INPL && (COMP || SPAIR) && SCHB <= (size_t)L::NWG * L::WGB;
  static constexpr size_t OFF_S = roundup_sz(L::OFF_M + (2 * L::NWG + 2) * sizeof(unsigned long long), 128);
  static constexpr bool OWN = FP32 && D == 2 && COMP && OFF_S + SCHB + 128 <= L::BUDGET;
  static constexpr bool SMB = IN_BOXES || OWN;
  static constexpr int SNBUF = (IN_BOXES && 2 * SCHB <= (size_t)L::NWG * L::WGB) ? 2 : 1;
  // dynamic shared memory of the launch
  static constexpr size_t BYTES = OWN ? OFF_S + SCHB + 128 : L::BYTES;
};

// Scalars of the step in the arithmetic type.
template <typename C>
struct Scal;
template <>
struct Scal<float> {
  float rho_ref, inv_tau, tau, mu_dt, two_cv, gfac, inv_cs, cs2, dt, mu_exp, inv_pr;
  __device__ __forceinline__ explicit Scal(const StepArgs& a)
      : rho_ref(a.f_rho_ref), inv_tau(a.f_inv_tau), tau(a.f_tau), mu_dt(a.f_mu_dt), two_cv(a.f_two_cv),
        gfac(a.f_gfac), inv_cs(a.f_inv_cs), cs2(a.f_cs2), dt(a.f_dt), mu_exp(a.f_mu_exp), inv_pr(a.f_inv_pr) {}
};
template <>
struct Scal<double> {
  double rho_ref, inv_tau, tau, mu_dt, two_cv, gfac, inv_cs, cs2, dt, mu_exp, inv_pr;
  __device__ __forceinline__ explicit Scal(const StepArgs& a)
      : rho_ref(a.rho_ref), inv_tau(a.inv_tau), tau(a.tau), mu_dt(a.mu_dt), two_cv(a.two_cv), gfac(a.gfac),
        inv_cs(a.inv_cs), cs2(a.cs2), dt(a.dt), mu_exp(a.mu_exp), inv_pr(a.inv_pr) {}
};

// Pr != 1, the heat-flux quasi-equilibrium of the compressible model (Sec. 3
// varies Pr by a quasi-equilibrium): from the pulled values of one node,
// f_i = ldf(i) and g_i = ldg(i) (shifted storage: minus w_i rho0 and
// w_i (2 C_v - D) rho0), the central heat flux H = sum_i f_i zeta^_i
// |zeta^_i|^2 and g's central first moment Gh = sum_i g_i zeta^_i, zeta^ =
// xi^ - u^ (the equilibria carry none for N >= 3 on sets of degree >= 7; the
// shifts add -rho0 u^ (D + 2 + |u^|^2) and -(2 C_v - D) rho0 u^).  Returns
// Fk = kap H / (2 (D + 2)) and Gk = kap Gh, kap = 1/tau - 1/tau_2,
// tau_2 = 1/2 + (tau - 1/2)/Pr: the collision adds w_i (|xi^_i|^2 - D - 2)
// (Fk . xi^_i) to f_i and w_i (Gk . xi^_i) to g_i.
template <int D, typename C>
__device__ __forceinline__ C qe_dot(const VelTab<C>& vt, int i, const C k[3]) {
  C s = k[0] * vt.xih[i][0];
  s = fma(k[1], vt.xih[i][1], s);
  if (D == 3) s = fma(k[2], vt.xih[i][2], s);
  return s;
}

// FULL: unroll the velocity loop completely (ldf reads a register array).
template <int D, int QM, bool FULL, typename C, typename LF, typename LG>
__device__ __forceinline__ void qe_coeffs(const VelTab<C>& vt, int Q, const Scal<C>& sc, LF ldf, LG ldg, C uhx,
                                          C uhy, C uhz, C q, C itau, C tau, C Fk[3], C Gk[3]) {
  C H[3] = {C(0), C(0), C(0)}, Gh[3] = {C(0), C(0), C(0)}, Gs = C(0);
  auto add = [&](int i) {
    const C fi = ldf(i), gi = ldg(i);
    const C xhx = vt.xih[i][0], xhy = vt.xih[i][1], xhz = D == 3 ? vt.xih[i][2] : C(0);
    const C zx = xhx - uhx, zy = xhy - uhy, zz = xhz - uhz;
    const C fz = fi * fma(zx, zx, fma(zy, zy, zz * zz));
    H[0] = fma(fz, zx, H[0]);
    H[1] = fma(fz, zy, H[1]);
    H[2] = fma(fz, zz, H[2]);
    Gh[0] = fma(gi, xhx, Gh[0]);
    Gh[1] = fma(gi, xhy, Gh[1]);
    Gh[2] = fma(gi, xhz, Gh[2]);
    Gs += gi;
  };
  if constexpr (FULL) {
#pragma unroll
    for (int i = 0; i < QM; ++i)
      if (i < Q) add(i);
  } else {
#pragma unroll 3
    for (int i = 0; i < QM; ++i) {
      if (i >= Q) break;
      add(i);
    }
  }
  const C kap = itau - C(1) / fma(tau - C(0.5), sc.inv_pr, C(0.5));
  const C hr = sc.rho_ref * (C(D + 2) + q), gr = fma(sc.gfac, sc.rho_ref, Gs);
  const C uh[3] = {uhx, uhy, uhz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Fk[c] = kap * C(0.5 / (D + 2)) * fma(-hr, uh[c], H[c]);
    Gk[c] = kap * fma(-gr, uh[c], Gh[c]);
  }
}

// Two values of the arithmetic type; FP32 pairs use the paired FMA.
template <typename C>
struct Pr;
template <>
struct Pr<float> {
  using T = float2;
  static __device__ __forceinline__ T set(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ T mul(T a, T b) { return __fmul2_rn(a, b); }
};
template <>
struct Pr<double> {
  using T = double2;
  static __device__ __forceinline__ T set(double a) { return make_double2(a, a); }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
  static __device__ __forceinline__ T mul(T a, T b) { return make_double2(a.x * b.x, a.y * b.y); }
};

// Pairs of FP32 values (two neighbouring nodes) with the paired FP32 pipe.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Two neighbouring values of a plane of the state (8- or 4-byte aligned).
__device__ __forceinline__ void store_pair(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void store_pair(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void store_pair(double* p, float a, float b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void store_pair(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}

// A 4-node x group as two pairs.
template <typename SRC, typename T>
__device__ __forceinline__ void ld4p(const SRC* p, T& lo, T& hi) {
  typename Store<SRC>::C v[4];
  ld4(p, v);
  lo.x = v[0];
  lo.y = v[1];
  hi.x = v[2];
  hi.y = v[3];
}
template <typename C, typename T>
__device__ __forceinline__ void st4p(C* p, T lo, T hi) {
  const C v[4] = {lo.x, lo.y, hi.x, hi.y};
  st4(p, v);
}

// L2 prefetch of `bytes` (multiple of 16, 16-byte aligned address) of global memory.
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// x pass of one 4-node group from a row of C values (s: first node's column,
// rounded down to the 16-byte granule; XO: offset of the first needed value).
template <int P, int XO, bool XACT, typename SRC, typename C>
__device__ __forceinline__ void xrow(const SRC* s, const C* W, C out[4]) {
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

// 16-bit two-box staging: the x pass is the only pass of a plane at rest along y and z
__device__ __forceinline__ bool from_box_plane(bool zact, bool yact) { return !zact && !yact; }

__device__ __forceinline__ void wg_barrier(int wg) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + wg), "r"(WGT) : "memory");
}

// Barrier of one warpgroup that also returns whether any of its threads set c.
__device__ __forceinline__ bool wg_any(int wg, bool c) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred pin, pout;\n setp.ne.u32 pin, %1, 0;\n bar.red.or.pred pout, %2, %3, pin;\n"
      " selp.u32 %0, 1, 0, pout;\n}\n"
      : "=r"(r)
      : "r"((unsigned)c), "r"(1 + wg), "r"(WGT)
      : "memory");
  return r != 0;
}

// Offset of the single periodic copy of coordinate c in the ghost layers of an
// axis with n >= gl + gr nodes (0 when c has none); only copies the stencil
// reaches are written.
__device__ __forceinline__ int one_image(int c, int n, int reach_lo, int reach_hi) {
  if (c < reach_hi) return n;
  if (c >= n - reach_lo) return -n;
  return 0;
}


// d Phi/ds and d Phi/dq of the isothermal closed form of order N (theta = 1):
// Phi = s + (s^2 - q)/2 [+ s (s^2 - 3q)/6] [+ (s^4 - 6 s^2 q + 3 q^2)/24].
template <typename C, int N>
__device__ __forceinline__ void phi_grad(C s, C q, C& ph, C& ps, C& pq) {
  const C s2 = s * s;
  ph = fma(C(0.5), s2 - q, s);
  ps = C(1) + s;
  pq = C(-0.5);
  if (N >= 3) {
    ph = fma(C(1.0 / 6.0), s * (s2 - C(3) * q), ph);
    ps = fma(C(0.5), s2 - q, ps);
    pq = fma(C(-0.5), s, pq);
  }
  if (N >= 4) {
    ph = fma(C(1.0 / 24.0), s2 * s2 - C(6) * s2 * q + C(3) * q * q, ph);
    ps = fma(C(1.0 / 6.0), s * (s2 - C(3) * q), ps);
    pq = fma(C(0.25), q - s2, pq);
  }
}

// Periodic copies of one node in the ghost layers: 0, 1 (one axis), 3 (two
// axes) or 7 (three axes) plane offsets, the single-axis ones first.
struct Images {
  int n;
  int i0, i1, i2, i3, i4, i5, i6;
  bool many;  // an axis shorter than its two ghost widths: every copy is stored
  static __device__ __forceinline__ Images make(int sx, int sy, int sz, bool simple) {
    Images m;
    const int nax = (sx != 0) + (sy != 0) + (sz != 0);
    m.n = nax == 0 ? 0 : (nax == 1 ? 1 : (nax == 2 ? 3 : 7));
    const int a0 = sx ? sx : (sy ? sy : sz);
    const int a1 = sx ? (sy ? sy : sz) : (sy ? sz : 0);
    m.i0 = a0;
    m.i1 = a1;
    m.i2 = nax == 3 ? sz : a0 + a1;
    m.i3 = sx + sy;
    m.i4 = sx + sz;
    m.i5 = sy + sz;
    m.i6 = sx + sy + sz;
    m.many = !simple && m.n > 0;
    return m;
  }
  // store v at p (the node's address in its plane) and at its copies
  template <typename S>
  __device__ __forceinline__ void put(S* p, S v, const Padded& pd, long long off, int x, int y, int z) const {
    p[0] = v;
    if (!n) return;
    if (many) {
      store_all_images(p - off, pd, x, y, z, v);
      return;
    }
    p[i0] = v;
    if (n > 1) {
      p[i1] = v;
      p[i2] = v;
      if (n > 3) {
        p[i3] = v;
        p[i4] = v;
        p[i5] = v;
        p[i6] = v;
      }
    }
  }
};

// Body of the two-phase kernels.  ADJ = false: the forward step.  ADJ = true:
// one adjoint step (see sl_adj_kernel); planes q < Q are pulled from the
// forward state with the stencil st, planes Q + i from the adjoint input with
// the stencil st2, through the tensor maps maps.m[0] and maps.m[1].
template <int D, int P, typename S, bool COMP, int QM, int N, bool ADJ>
__device__ __forceinline__ void wg_body(const StepArgs& a, const VelTab<typename Store<S>::C>& vt,
                                        const StencilTab<typename Store<S>::C, P + 1>& st,
                                        const StencilTab<typename Store<S>::C, P + 1>& st2, const TmaMaps& maps,
                                        const WgSchedule& sched) {
  using L = GLayout<D, P, S>;
  using C = typename Store<S>::C;
  using PR = Pr<C>;
  // phase B on node pairs with the paired FP32 pipe (isothermal, FP32 arithmetic, up to 27 velocities)
  constexpr bool PAIRS = !ADJ && !COMP && std::is_same<C, float>::value && QM <= 27;
  constexpr bool APAIRS = ADJ && std::is_same<C, float>::value && QM <= 27 && N <= 3;
  // isothermal FP32 arithmetic relaxes as (1 - 1/tau) f + (w/tau)(A + rho Phi),
  // the form whose first moment the host's correction f_g makes exact (see uhat_of)
  constexpr bool ISO32 = !COMP && std::is_same<C, float>::value;
  // phase B from shared-memory chunks of the staging slab (see Staging)
  using SG = Staging<D, P, S, COMP, QM, ADJ>;
  constexpr int SPMAX = SG::SPMAX;
  constexpr bool SPAIR = SG::SPAIR;
  constexpr int CHN = SG::CHN;
  constexpr bool SMB = SG::SMB;
  constexpr int SNBUF = SG::SNBUF;
  using T2 = typename PR::T;
  constexpr int NT = L::NT;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base, kept as arithmetic on the shared array so that the
  // compiler addresses it as shared memory (no generic loads and stores)
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = tid / WGT, wt = tid % WGT;
  unsigned char* mine = base + wg * L::WGB;
  S* box = reinterpret_cast<S*>(mine);
  S* box1 = reinterpret_cast<S*>(mine + (L::TWOBOX ? L::BOXB : 0));
  C* bufA = reinterpret_cast<C*>(mine + (L::TWO16 ? 2 * L::BOXB : L::BOXB));
  C* bufB = reinterpret_cast<C*>(mine + L::BOXB + L::ABYTES);
  double* red_smem = reinterpret_cast<double*>(base + L::OFF_R);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + L::OFF_M) + 2 * wg;
  unsigned long long* sbar = reinterpret_cast<unsigned long long*>(base + L::OFF_M) + 2 * L::NWG;

  const int Q = a.Q, planes = a.planes;
  const Padded& pd = a.pad;
  const Scal<C> sc(a);
  const CUtensorMap* maps4 = maps.m[a.src];
  const int nplan = sched.n[wg];
  S* __restrict__ dst = static_cast<S*>(a.buf[a.src ^ 1]);
  C* __restrict__ scr = static_cast<C*>(a.scratch) + (size_t)blockIdx.x * planes * L::TILE;
  // The collision Jacobian of the isothermal step depends on the pulled
  // populations only through their moments: a recorded forward step keeps, per
  // tile t, A = sum of the stored pulled values and j = sum xi f~ of every node
  // in the tape slot [t][4][TILE], and the adjoint reads them there.
  C* const slab = static_cast<C*>(a.slab);
  const unsigned long long keep = policy_evict_last();

  // stencil table, tensor maps and tensor plane of a staged plane
  auto tab_of = [&](int plane) -> const StencilTab<C, P + 1>& { return (ADJ && plane >= Q) ? st2 : st; };
  auto maps_of = [&](int plane) -> const CUtensorMap* { return (ADJ && plane >= Q) ? maps.m[1] : maps4; };
  auto tplane_of = [&](int plane) { return (ADJ && plane >= Q) ? plane - Q : plane; };
  // padded-grid origin of a tile, cached (the divisions run once per tile)
  int org_tile = -1, org[3] = {0, 0, 0};
  auto box_coords = [&](int tile, int plane, int& X, int& Y, int& Z) {
    if (tile != org_tile) {
      const int tx = tile % a.nt[0], r = tile / a.nt[0];
      org[0] = tx * L::TX + pd.gl[0];
      org[1] = (r % a.nt[1]) * L::TY + pd.gl[1];
      org[2] = D == 3 ? (r / a.nt[1]) * L::TZ + pd.gl[2] : 0;
      org_tile = tile;
    }
    const int i = plane < Q ? plane : plane - Q;
    const auto& T = tab_of(plane);
    const int act = T.active[i];
    X = org[0] + ((act & 1) ? T.m0[i][0] : 0);
    X -= X % L::VEC;
    Y = org[1] + ((act & 2) ? T.m0[i][1] : 0);
    Z = D == 3 ? org[2] + ((act & 4) ? T.m0[i][2] : 0) : 0;
    return ((act & 2) ? 1 : 0) | ((D == 3 && (act & 4)) ? 2 : 0);
  };
  auto issue = [&](int tile, int plane, int b = 0) {
    int X, Y, Z;
    const int v = box_coords(tile, plane, X, Y, Z);
    const unsigned bytes = (unsigned)(L::BXW * ((v & 1) ? L::BY : L::TY) * ((v & 2) ? L::BZ : L::TZ) * sizeof(S));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar + b, bytes);
    tma_load_4d(b ? box1 : box, &maps_of(plane)[v], X, Y, Z, tplane_of(plane), bar + b);
  };
  // (tile, k) of the plane `steps` after (tile, k) in this warpgroup's stream
  auto advance = [&](int& t, int& k, int steps) {
    k += steps;
    while (k >= nplan) {
      k -= nplan;
      t += gridDim.x;
    }
  };
  auto prefetch = [&](int tile, int plane) {
    int X, Y, Z;
    const int v = box_coords(tile, plane, X, Y, Z);
    tma_prefetch_4d(&maps_of(plane)[v], X, Y, Z, tplane_of(plane));
  };

  if (wt == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  if (tid == 0) {
    mbar_init(sbar, 1);
    mbar_init(sbar + 1, 1);
  }
  unsigned spar = 0;                  // bit b: phase parity of staging barrier b
  unsigned spend = 0;                 // bit b: a staging copy into buffer b is in flight
  if (tid < (NT / 32) * NRED) red_smem[tid] = 0.0;
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  bool pending = false;   // a copy into box 0 is in flight
  bool pending1 = false;  // a copy into box 1 is in flight (two-box staging)
  if (nplan > 0 && (int)blockIdx.x < a.ntiles) {
    if (wt == 0) {
      issue(blockIdx.x, sched.plane[wg][0]);
      if (!L::TWOBOX && nplan > 1) prefetch(blockIdx.x, sched.plane[wg][1]);
    }
    pending = true;
    if (L::TWOBOX) {
      int t1 = blockIdx.x, k1 = 0;
      advance(t1, k1, 1);
      if (t1 < a.ntiles) {
        if (wt == 0) issue(t1, sched.plane[wg][k1], 1);
        pending1 = true;
      }
    }
  }
  unsigned parity = 0;  // bit b: phase parity of box b's barrier
  int cb = 0;           // box of the current plane (two-box staging)
  bool failed = false;

  // every axis holds at least one stencil reach on each side: a node has at
  // most one periodic copy per axis
  const bool simple = a.quad_ok && pd.n[0] >= pd.gl[0] + pd.gr[0] && pd.n[1] >= pd.gl[1] + pd.gr[1] &&
                      pd.n[2] >= pd.gl[2] + pd.gr[2];

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    C* const mom = slab ? slab + (size_t)tile * 4 * L::TILE : nullptr;  // this tile's moments on the tape
    // ---------------- phase A: pull every plane of the tile -----------------
    if constexpr (L::TWOBOX) {
      for (int k = 0; k < nplan && !failed; ++k) {
        const int plane = sched.plane[wg][k];
        if (wg_any(wg, !mbar_wait_bounded(bar + cb, (parity >> cb) & 1u, a.wait_polls))) {
          failed = true;
          break;
        }
        parity ^= 1u << cb;
        if (cb) pending1 = false;
        else pending = false;
        const int i = plane < Q ? plane : plane - Q;
        const auto& T = tab_of(plane);
        const int act = T.active[i];
        const bool zact = (act & 4) != 0, yact = (act & 2) != 0, xact = (act & 1) != 0;
        // bs: the staged plane; bx: where the passes run (the box itself when
        // the storage is the arithmetic type, else the work buffer)
        S* bs = cb ? box1 : box;
        C* bx = L::INPL ? reinterpret_cast<C*>(bs) : bufA;
        const int BYA = yact ? L::BY : L::TY;
        const int PLs = BYA * L::BXW;
        // 16-bit storage: the box is free once the first pass has read it
        auto release = [&]() {
          if constexpr (L::TWO16) {
            wg_barrier(wg);
            int t2 = tile, k2 = k;
            advance(t2, k2, 2);
            if (t2 < a.ntiles) {
              if (wt == 0) issue(t2, sched.plane[wg][k2], cb);
              if (cb) pending1 = true;
              else pending = true;
            }
          }
        };
        if (zact) {
          T2 W[P + 1];
#pragma unroll
          for (int j = 0; j <= P; ++j) W[j] = PR::set(T.W[i][2][j]);
          const int ncol = L::NQX * BYA;
          for (int col = wt; col < ncol; col += WGT) {
            const int q = col % L::NQX, y = col / L::NQX;
            const S* s0 = bs + y * L::BXW + 4 * q;
            C* c0 = bx + y * L::BXW + 4 * q;
            T2 win[P + 1][2];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) ld4p(s0 + kk * PLs, win[kk][0], win[kk][1]);
#pragma unroll
            for (int z = 0; z < L::TZ; ++z) {
              ld4p(s0 + (z + P) * PLs, win[(z + P) % (P + 1)][0], win[(z + P) % (P + 1)][1]);
              T2 o[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                T2 acc = PR::mul(W[0], win[z % (P + 1)][h]);
#pragma unroll
                for (int kk = 1; kk <= P; ++kk) acc = PR::fma(W[kk], win[(z + kk) % (P + 1)][h], acc);
                o[h] = acc;
              }
              st4p(c0 + z * PLs, o[0], o[1]);  // row z is no longer read by this column
            }
          }
          if constexpr (L::TWO16) release();
          else wg_barrier(wg);
        }
        if (yact) {
          T2 W[P + 1];
#pragma unroll
          for (int j = 0; j <= P; ++j) W[j] = PR::set(T.W[i][1][j]);
          constexpr int ncol = L::NQX * L::TZ;
          // in place in bx, or (16-bit storage, z at rest) from the box into bx
          auto ypass_from = [&](const auto* src) {
            for (int col = wt; col < ncol; col += WGT) {
              const int q = col % L::NQX, z = col / L::NQX;
              const auto* s0 = src + z * PLs + 4 * q;
              C* c0 = bx + z * PLs + 4 * q;
              T2 win[P + 1][2];
#pragma unroll
              for (int kk = 0; kk < P; ++kk) ld4p(s0 + kk * L::BXW, win[kk][0], win[kk][1]);
#pragma unroll
              for (int y = 0; y < L::TY; ++y) {
                ld4p(s0 + (y + P) * L::BXW, win[(y + P) % (P + 1)][0], win[(y + P) % (P + 1)][1]);
              T2 o[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                T2 acc = PR::mul(W[0], win[y % (P + 1)][h]);
#pragma unroll
                for (int kk = 1; kk <= P; ++kk) acc = PR::fma(W[kk], win[(y + kk) % (P + 1)][h], acc);
                o[h] = acc;
              }
                st4p(c0 + y * L::BXW, o[0], o[1]);
              }
            }
          };
          if (L::TWO16 && !zact) {
            ypass_from(static_cast<const S*>(bs));
            release();
          } else {
            ypass_from(static_cast<const C*>(bx));
            wg_barrier(wg);
          }
        }
        {
          C W[P + 1];
#pragma unroll
          for (int j = 0; j <= P; ++j) W[j] = T.W[i][0][j];
          const int xo = xact ? ((T.m0[i][0] % L::VEC) + L::VEC) % L::VEC : 0;
          // the x pass reads bx, or (16-bit storage, y and z at rest) the box
          const bool from_box = L::TWO16 && !zact && !yact;
          // one alignment variant per plane (dispatched once), rolled over the groups
          auto groups = [&](auto XOc, auto ACT) {
            constexpr int QPT = L::TILE / 4 / WGT;  // 4-node x groups per thread
            C* so = scr + (size_t)plane * L::TILE;
#pragma unroll 1
            for (int m = 0; m < QPT; ++m) {
              const int qi = wt + WGT * m;
              const int qx = (qi % (L::TX / 4)) * 4, ly = (qi / (L::TX / 4)) % L::TY,
                        lz = qi / (L::TX / 4 * L::TY);
              C out[4];
              const int off = (lz * BYA + ly) * L::BXW + qx;
              if (from_box)
                xrow<P, decltype(XOc)::value, decltype(ACT)::value>(bs + off, W, out);
              else
                xrow<P, decltype(XOc)::value, decltype(ACT)::value>(bx + off, W, out);
              gst4(so + 4 * qi, out, keep);
            }
          };
          if (!xact) {
            groups(std::integral_constant<int, 0>(), std::false_type());
          } else {
            switch (xo) {
              case 0: groups(std::integral_constant<int, 0>(), std::true_type()); break;
              case 1: groups(std::integral_constant<int, 1>(), std::true_type()); break;
              case 2: if constexpr (L::VEC > 2) groups(std::integral_constant<int, 2>(), std::true_type()); break;
              case 3: if constexpr (L::VEC > 3) groups(std::integral_constant<int, 3>(), std::true_type()); break;
              case 4: if constexpr (L::VEC > 4) groups(std::integral_constant<int, 4>(), std::true_type()); break;
              case 5: if constexpr (L::VEC > 5) groups(std::integral_constant<int, 5>(), std::true_type()); break;
              case 6: if constexpr (L::VEC > 6) groups(std::integral_constant<int, 6>(), std::true_type()); break;
              default: if constexpr (L::VEC > 7) groups(std::integral_constant<int, 7>(), std::true_type()); break;
            }
          }
        }
        if (L::TWO16 && from_box_plane(zact, yact)) {
          release();  // the x pass was the first to read the box; the work buffer was not used
        } else {
          wg_barrier(wg);  // box (work buffer) free
          if constexpr (!L::TWO16) {
            int t2 = tile, k2 = k;
            advance(t2, k2, 2);
            // with shared-memory staging the boxes serve phase B: the next tile's
            // copies start after it
            if (t2 < a.ntiles && (!SMB || t2 == tile)) {
              if (wt == 0) issue(t2, sched.plane[wg][k2], cb);
              if (cb) pending1 = true;
              else pending = true;
            }
          }
        }
        cb ^= 1;
      }
    } else
    for (int k = 0; k < nplan && !failed; ++k) {
      const int plane = sched.plane[wg][k];
      // every thread of the warpgroup takes the same decision
      if (wg_any(wg, !mbar_wait_bounded(bar, parity, a.wait_polls))) {
        failed = true;
        break;
      }
      parity ^= 1u;
      pending = false;
      const int i = plane < Q ? plane : plane - Q;
      const auto& T = tab_of(plane);
      const int act = T.active[i];
      const bool zact = D == 3 && (act & 4), yact = (act & 2) != 0, xact = (act & 1) != 0;
      if (wt == 0) {
        // warm L2 with the plane after next
        const int k2 = k + 2;
        if (k2 < nplan) prefetch(tile, sched.plane[wg][k2]);
        else if (tile + (int)gridDim.x < a.ntiles && k2 - nplan < nplan) prefetch(tile + gridDim.x, sched.plane[wg][k2 - nplan]);
      }
      // the next copy into the box starts as soon as the first pass has read it
      bool issued = false;
      auto issue_next = [&]() {
        issued = true;
        if (k + 1 < nplan) {
          if (wt == 0) issue(tile, sched.plane[wg][k + 1]);
          pending = true;
        } else if (tile + (int)gridDim.x < a.ntiles) {
          if (wt == 0) issue(tile + gridDim.x, sched.plane[wg][0]);
          pending = true;
        }
      };
      const C* xsrc_c = nullptr;
      if (zact) {
        T2 W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = PR::set(T.W[i][2][j]);
        const int BYA = yact ? L::BY : L::TY;
        const int PLs = BYA * L::BXW;
        const int ncol = L::NQX * BYA;
        for (int col = wt; col < ncol; col += WGT) {
          const int q = col % L::NQX, y = col / L::NQX;
          const S* src = box + y * L::BXW + 4 * q;
          C* out = bufA + y * L::BXW + 4 * q;
          T2 win[P + 1][2];
#pragma unroll
          for (int k = 0; k < P; ++k) ld4p(src + k * PLs, win[k][0], win[k][1]);
#pragma unroll
          for (int z = 0; z < L::ZC; ++z) {
            ld4p(src + (z + P) * PLs, win[(z + P) % (P + 1)][0], win[(z + P) % (P + 1)][1]);
            T2 o[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              T2 acc = PR::mul(W[0], win[z % (P + 1)][h]);
#pragma unroll
              for (int k = 1; k <= P; ++k) acc = PR::fma(W[k], win[(z + k) % (P + 1)][h], acc);
              o[h] = acc;
            }
            st4p(out + z * PLs, o[0], o[1]);
          }
        }
        wg_barrier(wg);
        issue_next();
        xsrc_c = bufA;
      }
      if (yact) {
        T2 W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = PR::set(T.W[i][1][j]);
        constexpr int NYC = L::TY / L::YC;
        constexpr int items = L::NQX * L::TZ * NYC;
        for (int item = wt; item < items; item += WGT) {
          const int q = item % L::NQX, r = item / L::NQX, yc = r % NYC, z = r / NYC;
          const int off = (z * L::BY + yc * L::YC) * L::BXW + 4 * q;
          C* out = bufB + (z * L::TY + yc * L::YC) * L::BXW + 4 * q;
          T2 win[P + 1][2];
          auto load = [&](int k, T2& lo, T2& hi) {
            if (zact) ld4p(bufA + off + k * L::BXW, lo, hi);
            else ld4p(box + off + k * L::BXW, lo, hi);
          };
#pragma unroll
          for (int k = 0; k < P; ++k) load(k, win[k][0], win[k][1]);
#pragma unroll
          for (int y = 0; y < L::YC; ++y) {
            load(y + P, win[(y + P) % (P + 1)][0], win[(y + P) % (P + 1)][1]);
            T2 o[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              T2 acc = PR::mul(W[0], win[y % (P + 1)][h]);
#pragma unroll
              for (int k = 1; k <= P; ++k) acc = PR::fma(W[k], win[(y + k) % (P + 1)][h], acc);
              o[h] = acc;
            }
            st4p(out + y * L::BXW, o[0], o[1]);
          }
        }
        wg_barrier(wg);
        if (!issued) issue_next();
        xsrc_c = bufB;
      }
      {
        C W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = T.W[i][0][j];
        const int xo = xact ? ((T.m0[i][0] % L::VEC) + L::VEC) % L::VEC : 0;
        constexpr int QPT = L::TILE / 4 / WGT;  // 4-node x groups per thread
#pragma unroll
        for (int m = 0; m < QPT; ++m) {
          const int qi = wt + WGT * m;
          const int qx = (qi % (L::TX / 4)) * 4, ly = (qi / (L::TX / 4)) % L::TY, lz = qi / (L::TX / 4 * L::TY);
          C out[4];
          if (xsrc_c)
            xpass_any<D, P, S>(xact, xo, xsrc_c, qx, ly, lz, W, out);
          else
            xpass_any<D, P, S>(xact, xo, static_cast<const S*>(box), qx, ly, lz, W, out);
          gst4(scr + (size_t)plane * L::TILE + 4 * qi, out, keep);
        }
      }
      wg_barrier(wg);  // buffers free
      if (!issued) issue_next();
    }
    // with shared-memory staging, phase B copies the slab this thread has just
    // written (generic proxy) with bulk copies (async proxy)
    if constexpr (SMB) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }

    // ---------------- phase B: collide every node of the tile ---------------
    const int tx = tile % a.nt[0], tr = tile / a.nt[0];
    const int ty = tr % a.nt[1], tz = tr / a.nt[1];
    const bool red = !ADJ && a.reduce != 0;
    C tsum[NRED];
#pragma unroll
    for (int c = 0; c < NRED; ++c) tsum[c] = C(0);

    // periodic copies of node (x, y, z) in the ghost layers (0, 1, 3 or 7)
    auto images_of = [&](int x, int y, int z) {
      const int dx = one_image(x, pd.n[0], pd.gl[0], pd.gr[0]);
      const int dy = one_image(y, pd.n[1], pd.gl[1], pd.gr[1]);
      const int dz = D == 3 ? one_image(z, pd.n[2], pd.gl[2], pd.gr[2]) : 0;
      return Images::make(dx, dy * pd.np[0], dz * pd.np[0] * pd.np[1], simple);
    };

    // The same collision reading the pulled value of plane q of node n from
    // src[q * stride] (a shared-memory chunk: stride = chunk size) where it is
    // used, instead of holding all values in registers (shared-memory staging).
    auto collide_from = [&](int n, const C* __restrict__ src, auto STc, auto RED) {
      constexpr int stride = decltype(STc)::value;
      constexpr bool R = decltype(RED)::value;
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      // moments (Sec. 3).  Compressible energy sums: FP32 groups of eight
      // merged by error-free additions into (hi, lo) pairs (the FP64 pipe of
      // this GPU is narrow; the cancellation below is done in FP64).
      auto merge = [](C& hi, C& lo, C v) {
        const C t = hi + v, e = t - hi;
        lo += (hi - (t - e)) + (v - e);
        hi = t;
      };
      C A = C(0), jx = C(0), jy = C(0), jz = C(0), Bp = C(0), Bh = C(0), Bl = C(0);
#pragma unroll STAGED_UNROLL
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        const C fi = src[i * stride];
        A += fi;
        jx = fma(vt.xi[i][0], fi, jx);
        jy = fma(vt.xi[i][1], fi, jy);
        if (D == 3) jz = fma(vt.xi[i][2], fi, jz);
        if (COMP) {
          Bp = fma(vt.xi2[i], fi, Bp);
          if ((i & 7) == 7) {
            merge(Bh, Bl, Bp);
            Bp = C(0);
          }
        }
      }
      const C rho = sc.rho_ref + A;
      if constexpr (!ADJ && !COMP) {
        if (mom) {  // a recorded step: the moments for the adjoint
          mom[n] = A;
          mom[L::TILE + n] = jx;
          mom[2 * L::TILE + n] = jy;
          mom[3 * L::TILE + n] = jz;
        }
      }
      const C ir = C(1) / rho;
      const C irc = sc.inv_cs / rho;
      const C uhx = uhat_of<COMP>(a, jx, irc, 0), uhy = uhat_of<COMP>(a, jy, irc, 1), uhz = uhat_of<COMP>(a, jz, irc, 2);
      const C q = uhx * uhx + uhy * uhy + uhz * uhz;
      C itau = sc.inv_tau, tt = C(0), gA = C(0), rth = C(0), theta = C(1), tau = sc.tau;
      if (COMP) {
        merge(Bh, Bl, Bp);
        // sum of the pulled g (Sec. 3 temperature relation), FP32 groups merged exactly
        C Gp = C(0), Gh = C(0), Gl = C(0);
#pragma unroll STAGED_UNROLL
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          Gp += src[(Q + i) * stride];
          if ((i & 7) == 7) {
            merge(Gh, Gl, Gp);
            Gp = C(0);
          }
        }
        merge(Gh, Gl, Gp);
        // 2 C_v (rho theta - rho) = B + G - |j|^2/rho - 2 C_v A, cancelling in FP64
        const C K = (jx * jx + jy * jy + jz * jz) * ir;
        const double X = fma(-a.two_cv, (double)A, (((double)Bh + (double)Bl) + ((double)Gh + (double)Gl)) - (double)K);
        tt = C(X) / (sc.two_cv * rho);
        theta = C(1) + tt;
        tau = mu_theta(sc.mu_dt, theta, sc.mu_exp) / (rho * theta) + C(0.5);
        itau = C(1) / tau;
        gA = fma(rho, tt, A);
        rth = rho * theta;
      }
      C Fk[3], Gk[3];
      const bool qe = COMP && a.qe != 0;
      if (qe)
        qe_coeffs<D, QM, false>(vt, Q, sc, [&](int i) { return src[i * stride]; },
                         [&](int i) { return src[(Q + i) * stride]; }, uhx, uhy, uhz, q, itau, tau, Fk, Gk);
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      // The closed form of order N (Appendix A) as a polynomial in s = xi^.u^,
      // Phi - 1 = c0 + s (c1 + s (c2 + s (c3 + s c4))), whose coefficients
      // depend on the velocity only through r_D = |xi^|^2 - D and
      // r_P = r^2 - 2 (D + 2) r + D (D + 2):
      //   c0 = a0 + a1 r_D + a2 r_P,  c1 = b0 + b1 r_D,  c2 = g0 + g1 r_D.
      C a0 = C(-0.5) * q, a1 = C(0), a2 = C(0), b0 = C(1), b1 = C(0), g0 = C(0.5), g1 = C(0), c3 = C(0),
        c4 = C(0);
      if (COMP) a1 = C(0.5) * tt;
      if (N >= 3) {
        b0 = b0 - C(0.5) * q - (COMP ? tt : C(0));
        if (COMP) b1 = C(0.5) * tt;
        c3 = C(1.0 / 6.0);
      }
      if (N >= 4) {
        a0 = fma(C(0.125) * q, q, a0);
        g0 = g0 - C(0.25) * q;
        c4 = C(1.0 / 24.0);
        if (COMP) {
          a0 = fma(C(0.5) * tt, q, a0);
          a1 = fma(C(-0.25) * tt, q, a1);
          a2 = C(0.125) * tt * tt;
          g0 = g0 - tt;
          g1 = C(0.25) * tt;
        }
      }
      auto phi = [&](int i) {
        C s = vt.xih[i][0] * uhx;
        s = fma(vt.xih[i][1], uhy, s);
        if (D == 3) s = fma(vt.xih[i][2], uhz, s);
        C c0 = a0, c1 = b0, c2 = g0;
        if (COMP) {
          c0 = fma(a1, vt.rD[i], c0);
          if (N >= 4) c0 = fma(a2, vt.rpoly[i], c0);
          if (N >= 3) c1 = fma(b1, vt.rD[i], c1);
          if (N >= 4) c2 = fma(g1, vt.rD[i], c2);
        }
        C hp = c2;
        if (N >= 4) hp = fma(fma(c4, s, c3), s, c2);
        else if (N >= 3) hp = fma(c3, s, c2);
        return fma(fma(hp, s, c1), s, c0);
      };
      // equilibrium (Appendix A), BGK (Sec. 3) and the stores: f_i, and in 2D
      // g_i from the same polynomial value (3D: g in a second loop, the
      // polynomial evaluated again, which keeps the loop body within the
      // instruction cache: measured 1% faster there, 3% slower in 2D)
      constexpr bool GMERGE = COMP && D == 2;
      S* pf = dst + off;
      const long long gofs = (long long)Q * pd.plane;
      C Pi[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
#pragma unroll STAGED_UNROLL
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        const C ph = phi(i);
        const C eqv = fma(rho, ph, A);  // A + rho Phi
        const C feqd = vt.w[i] * eqv;
        const C fi = src[i * stride];
        const C fneq = fi - feqd;
        C o = ISO32 ? fma(C(1) - sc.inv_tau, fi, vt.wt[i] * eqv) : fma(-fneq, itau, fi);
        if (qe) o = fma(vt.w[i] * (vt.rD[i] - C(2)), qe_dot<D>(vt, i, Fk), o);
        im.put(pf, Store<S>::st(o), pd, off, x, y, z);
        if constexpr (GMERGE) {
          const C geqd = vt.w[i] * sc.gfac * fma(rth, ph, gA);
          const C gi = src[(Q + i) * stride];
          C og = fma(-(gi - geqd), itau, gi);
          if (qe) og = fma(vt.w[i], qe_dot<D>(vt, i, Gk), og);
          im.put(pf + gofs, Store<S>::st(og), pd, off, x, y, z);
        }
        pf += pd.plane;
        if (R) {
#pragma unroll
          for (int c = 0; c < 6; ++c) Pi[c] = fma(vt.xx[i][c], fneq, Pi[c]);
        }
      }
      if constexpr (COMP && !GMERGE) {
#pragma unroll STAGED_UNROLL
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          const C geqd = vt.w[i] * sc.gfac * fma(rth, phi(i), gA);
          const C gi = src[(Q + i) * stride];
          C o = fma(-(gi - geqd), itau, gi);
          if (qe) o = fma(vt.w[i], qe_dot<D>(vt, i, Gk), o);
          im.put(pf, Store<S>::st(o), pd, off, x, y, z);
          pf += pd.plane;
        }
      }
      if (R) {
        const C u2 = q * sc.cs2;
        tsum[0] += C(0.5) * u2;
        tsum[1] += C(0.5) * rho * u2;
        tsum[3] += A;
        tsum[4] += jx;
        tsum[5] += jy;
        tsum[6] += jz;
        const bool fin = isfinite(rho) && isfinite(uhx) && isfinite(uhy) && isfinite(uhz) && isfinite(theta);
        tsum[7] += fin ? C(0) : C(1);
        const C pres = rho * theta * sc.cs2;
        const C den = C(2) * pres * tau * sc.dt;
        const C ss = (Pi[0] * Pi[0] + Pi[1] * Pi[1] + Pi[2] * Pi[2] +
                      C(2) * (Pi[3] * Pi[3] + Pi[4] * Pi[4] + Pi[5] * Pi[5])) /
                     (den * den);
        const C nu = sc.cs2 * theta * sc.dt * (tau - C(0.5));
        tsum[2] += C(2) * nu * ss;
      }
    };
    auto collide = [&](int n, auto RED) {
      constexpr bool R = decltype(RED)::value;
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      C f[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) f[i] = i < Q ? scr[(size_t)i * L::TILE + n] : C(0);
      // moments (Sec. 3).  Compressible energy sums: FP32 groups of eight
      // merged by error-free additions into (hi, lo) pairs (the FP64 pipe of
      // this GPU is narrow; the cancellation below is done in FP64).
      auto merge = [](C& hi, C& lo, C v) {
        const C t = hi + v, e = t - hi;
        lo += (hi - (t - e)) + (v - e);
        hi = t;
      };
      C A = C(0), jx = C(0), jy = C(0), jz = C(0), Bp = C(0), Bh = C(0), Bl = C(0);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        A += f[i];
        jx = fma(vt.xi[i][0], f[i], jx);
        jy = fma(vt.xi[i][1], f[i], jy);
        if (D == 3) jz = fma(vt.xi[i][2], f[i], jz);
        if (COMP) {
          Bp = fma(vt.xi2[i], f[i], Bp);
          if ((i & 7) == 7) {
            merge(Bh, Bl, Bp);
            Bp = C(0);
          }
        }
      }
      const C rho = sc.rho_ref + A;
      if constexpr (!ADJ && !COMP) {
        if (mom) {  // a recorded step: the moments for the adjoint
          mom[n] = A;
          mom[L::TILE + n] = jx;
          mom[2 * L::TILE + n] = jy;
          mom[3 * L::TILE + n] = jz;
        }
      }
      const C ir = C(1) / rho;
      const C irc = sc.inv_cs / rho;
      const C uhx = uhat_of<COMP>(a, jx, irc, 0), uhy = uhat_of<COMP>(a, jy, irc, 1), uhz = uhat_of<COMP>(a, jz, irc, 2);
      const C q = uhx * uhx + uhy * uhy + uhz * uhz;
      C itau = sc.inv_tau, tt = C(0), gA = C(0), rth = C(0), theta = C(1), tau = sc.tau;
      if (COMP) {
        merge(Bh, Bl, Bp);
        // sum of the pulled g (Sec. 3 temperature relation), FP32 groups merged exactly
        C Gp = C(0), Gh = C(0), Gl = C(0);
#pragma unroll
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          Gp += scr[(size_t)(Q + i) * L::TILE + n];
          if ((i & 7) == 7) {
            merge(Gh, Gl, Gp);
            Gp = C(0);
          }
        }
        merge(Gh, Gl, Gp);
        // 2 C_v (rho theta - rho) = B + G - |j|^2/rho - 2 C_v A, cancelling in FP64
        const C K = (jx * jx + jy * jy + jz * jz) * ir;
        const double X = fma(-a.two_cv, (double)A, (((double)Bh + (double)Bl) + ((double)Gh + (double)Gl)) - (double)K);
        tt = C(X) / (sc.two_cv * rho);
        theta = C(1) + tt;
        tau = mu_theta(sc.mu_dt, theta, sc.mu_exp) / (rho * theta) + C(0.5);
        itau = C(1) / tau;
        gA = fma(rho, tt, A);
        rth = rho * theta;
      }
      C Fk[3], Gk[3];
      const bool qe = COMP && a.qe != 0;
      if (qe)
        qe_coeffs<D, QM, true>(vt, Q, sc, [&](int i) { return f[i]; },
                         [&](int i) { return scr[(size_t)(Q + i) * L::TILE + n]; }, uhx, uhy, uhz, q, itau, tau, Fk,
                         Gk);
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      // The closed form of order N (Appendix A) as a polynomial in s = xi^.u^,
      // Phi - 1 = c0 + s (c1 + s (c2 + s (c3 + s c4))), whose coefficients
      // depend on the velocity only through r_D = |xi^|^2 - D and
      // r_P = r^2 - 2 (D + 2) r + D (D + 2):
      //   c0 = a0 + a1 r_D + a2 r_P,  c1 = b0 + b1 r_D,  c2 = g0 + g1 r_D.
      C a0 = C(-0.5) * q, a1 = C(0), a2 = C(0), b0 = C(1), b1 = C(0), g0 = C(0.5), g1 = C(0), c3 = C(0),
        c4 = C(0);
      if (COMP) a1 = C(0.5) * tt;
      if (N >= 3) {
        b0 = b0 - C(0.5) * q - (COMP ? tt : C(0));
        if (COMP) b1 = C(0.5) * tt;
        c3 = C(1.0 / 6.0);
      }
      if (N >= 4) {
        a0 = fma(C(0.125) * q, q, a0);
        g0 = g0 - C(0.25) * q;
        c4 = C(1.0 / 24.0);
        if (COMP) {
          a0 = fma(C(0.5) * tt, q, a0);
          a1 = fma(C(-0.25) * tt, q, a1);
          a2 = C(0.125) * tt * tt;
          g0 = g0 - tt;
          g1 = C(0.25) * tt;
        }
      }
      auto phi = [&](int i) {
        C s = vt.xih[i][0] * uhx;
        s = fma(vt.xih[i][1], uhy, s);
        if (D == 3) s = fma(vt.xih[i][2], uhz, s);
        C c0 = a0, c1 = b0, c2 = g0;
        if (COMP) {
          c0 = fma(a1, vt.rD[i], c0);
          if (N >= 4) c0 = fma(a2, vt.rpoly[i], c0);
          if (N >= 3) c1 = fma(b1, vt.rD[i], c1);
          if (N >= 4) c2 = fma(g1, vt.rD[i], c2);
        }
        C hp = c2;
        if (N >= 4) hp = fma(fma(c4, s, c3), s, c2);
        else if (N >= 3) hp = fma(c3, s, c2);
        return fma(fma(hp, s, c1), s, c0);
      };
      // equilibrium (Appendix A), BGK (Sec. 3) and the stores: f first
      S* pf = dst + off;
      C Pi[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        const C ph = phi(i);
        const C eqv = fma(rho, ph, A);  // A + rho Phi
        const C feqd = vt.w[i] * eqv;
        const C fneq = f[i] - feqd;
        C o = ISO32 ? fma(C(1) - sc.inv_tau, f[i], vt.wt[i] * eqv) : fma(-fneq, itau, f[i]);
        if (qe) o = fma(vt.w[i] * (vt.rD[i] - C(2)), qe_dot<D>(vt, i, Fk), o);
        im.put(pf, Store<S>::st(o), pd, off, x, y, z);
        pf += pd.plane;
        if (R) {
#pragma unroll
          for (int c = 0; c < 6; ++c) Pi[c] = fma(vt.xx[i][c], fneq, Pi[c]);
        }
      }
      if (COMP) {
        // then g: all staged g values loaded at once into the registers f held,
        // the polynomial evaluated again (cheaper than a load per velocity)
#pragma unroll
        for (int i = 0; i < QM; ++i) f[i] = i < Q ? scr[(size_t)(Q + i) * L::TILE + n] : C(0);
#pragma unroll
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          const C geqd = vt.w[i] * sc.gfac * fma(rth, phi(i), gA);
          C o = fma(-(f[i] - geqd), itau, f[i]);
          if (qe) o = fma(vt.w[i], qe_dot<D>(vt, i, Gk), o);
          im.put(pf, Store<S>::st(o), pd, off, x, y, z);
          pf += pd.plane;
        }
      }
      if (R) {
        const C u2 = q * sc.cs2;
        tsum[0] += C(0.5) * u2;
        tsum[1] += C(0.5) * rho * u2;
        tsum[3] += A;
        tsum[4] += jx;
        tsum[5] += jy;
        tsum[6] += jz;
        const bool fin = isfinite(rho) && isfinite(uhx) && isfinite(uhy) && isfinite(uhz) && isfinite(theta);
        tsum[7] += fin ? C(0) : C(1);
        const C pres = rho * theta * sc.cs2;
        const C den = C(2) * pres * tau * sc.dt;
        const C ss = (Pi[0] * Pi[0] + Pi[1] * Pi[1] + Pi[2] * Pi[2] +
                      C(2) * (Pi[3] * Pi[3] + Pi[4] * Pi[4] + Pi[5] * Pi[5])) /
                     (den * den);
        const C nu = sc.cs2 * theta * sc.dt * (tau - C(0.5));
        tsum[2] += C(2) * nu * ss;
      }
    };

    // Two neighbouring nodes (n, n + 1) of one x row per thread, FP32
    // isothermal sets up to 27 velocities: the paired FP32 pipe does both.
    // With c = A - rho q/2 [+ rho q^2/8], c1 = rho [- rho q/2], c2 = rho/2
    // [- rho q/4], c3 = [rho/6], c4 = [rho/24] (brackets: N >= 3, N >= 4),
    // A + rho Phi = c + s (c1 + s (c2 + s (c3 + s c4))), and the BGK update is
    // f_post = (1 - 1/tau) f + (w/tau)(A + rho Phi).
    auto collide2 = [&](int n) {
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      const bool in1 = x + 1 < pd.n[0];
      float2 f[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i)
        f[i] = i < Q ? *reinterpret_cast<const float2*>(scr + (size_t)i * L::TILE + n) : f2(0.f);
      float2 A = f2(0.f), jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        A = add2(A, f[i]);
        jx = fma2(f2(vt.xi[i][0]), f[i], jx);
        jy = fma2(f2(vt.xi[i][1]), f[i], jy);
        if (D == 3) jz = fma2(f2(vt.xi[i][2]), f[i], jz);
      }
      const float2 rho = add2(f2(sc.rho_ref), A);
      if (!ADJ && mom) {  // a recorded step: the moments for the adjoint
        float* mf = reinterpret_cast<float*>(mom) + n;
        *reinterpret_cast<float2*>(mf) = A;
        *reinterpret_cast<float2*>(mf + L::TILE) = jx;
        *reinterpret_cast<float2*>(mf + 2 * L::TILE) = jy;
        *reinterpret_cast<float2*>(mf + 3 * L::TILE) = jz;
      }
      const float2 irc = make_float2(sc.inv_cs / rho.x, sc.inv_cs / rho.y);
      const float2 uhx = uhat2_of(a, jx, irc, 0), uhy = uhat2_of(a, jy, irc, 1), uhz = uhat2_of(a, jz, irc, 2);
      const float2 q = fma2(uhz, uhz, fma2(uhy, uhy, mul2(uhx, uhx)));
      const float2 r2 = mul2(f2(0.5f), rho);
      float2 c = fma2(f2(-1.f), mul2(r2, q), A);
      float2 c1 = rho, c2 = r2, c3 = f2(0.f), c4 = f2(0.f);
      if (N >= 3) {
        c1 = fma2(f2(-1.f), mul2(r2, q), rho);
        c3 = mul2(f2(1.0f / 6.0f), rho);
      }
      if (N >= 4) {
        c = fma2(mul2(f2(0.125f), rho), mul2(q, q), c);
        c2 = fma2(f2(-0.5f), mul2(r2, q), r2);
        c4 = mul2(f2(1.0f / 24.0f), rho);
      }
      const float2 om = f2(1.f - sc.inv_tau);
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      S* pf = dst + off;
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        float2 s = mul2(f2(vt.xih[i][0]), uhx);
        s = fma2(f2(vt.xih[i][1]), uhy, s);
        if (D == 3) s = fma2(f2(vt.xih[i][2]), uhz, s);
        float2 t = c2;
        if (N >= 4) t = fma2(fma2(c4, s, c3), s, c2);
        else if (N >= 3) t = fma2(c3, s, c2);
        const float2 e = fma2(fma2(t, s, c1), s, c);  // A + rho Phi
        const float2 o = fma2(om, f[i], mul2(f2(vt.wt[i]), e));
        if (simple) {
          store_pair(pf, o.x, o.y);
          if (im.n) {
            store_pair(pf + im.i0, o.x, o.y);
            if (im.n > 1) {
              store_pair(pf + im.i1, o.x, o.y);
              store_pair(pf + im.i2, o.x, o.y);
              if (im.n > 3) {
                store_pair(pf + im.i3, o.x, o.y);
                store_pair(pf + im.i4, o.x, o.y);
                store_pair(pf + im.i5, o.x, o.y);
                store_pair(pf + im.i6, o.x, o.y);
              }
            }
          }
        } else {
          store_all_images(pf - off, pd, x, y, z, Store<S>::st(o.x));
          if (in1) store_all_images(pf - off, pd, x + 1, y, z, Store<S>::st(o.y));
        }
        pf += pd.plane;
      }
    };
    // collide2 reading each node pair's values where they are used from a
    // shared-memory chunk (src: the pair in plane 0, stride CH values)
    auto collide2_from = [&](int n, const float* __restrict__ src, auto CHc) {
      constexpr int CH = decltype(CHc)::value;
      auto fv = [&](int i) { return *reinterpret_cast<const float2*>(src + i * CH); };
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      const bool in1 = x + 1 < pd.n[0];
      float2 A = f2(0.f), jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        const float2 fi = fv(i);
        A = add2(A, fi);
        jx = fma2(f2(vt.xi[i][0]), fi, jx);
        jy = fma2(f2(vt.xi[i][1]), fi, jy);
        if (D == 3) jz = fma2(f2(vt.xi[i][2]), fi, jz);
      }
      const float2 rho = add2(f2(sc.rho_ref), A);
      if (!ADJ && mom) {  // a recorded step: the moments for the adjoint
        float* mf = reinterpret_cast<float*>(mom) + n;
        *reinterpret_cast<float2*>(mf) = A;
        *reinterpret_cast<float2*>(mf + L::TILE) = jx;
        *reinterpret_cast<float2*>(mf + 2 * L::TILE) = jy;
        *reinterpret_cast<float2*>(mf + 3 * L::TILE) = jz;
      }
      const float2 irc = make_float2(sc.inv_cs / rho.x, sc.inv_cs / rho.y);
      const float2 uhx = uhat2_of(a, jx, irc, 0), uhy = uhat2_of(a, jy, irc, 1), uhz = uhat2_of(a, jz, irc, 2);
      const float2 q = fma2(uhz, uhz, fma2(uhy, uhy, mul2(uhx, uhx)));
      const float2 r2 = mul2(f2(0.5f), rho);
      float2 c = fma2(f2(-1.f), mul2(r2, q), A);
      float2 c1 = rho, c2 = r2, c3 = f2(0.f), c4 = f2(0.f);
      if (N >= 3) {
        c1 = fma2(f2(-1.f), mul2(r2, q), rho);
        c3 = mul2(f2(1.0f / 6.0f), rho);
      }
      if (N >= 4) {
        c = fma2(mul2(f2(0.125f), rho), mul2(q, q), c);
        c2 = fma2(f2(-0.5f), mul2(r2, q), r2);
        c4 = mul2(f2(1.0f / 24.0f), rho);
      }
      const float2 om = f2(1.f - sc.inv_tau);
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      S* pf = dst + off;
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        float2 s = mul2(f2(vt.xih[i][0]), uhx);
        s = fma2(f2(vt.xih[i][1]), uhy, s);
        if (D == 3) s = fma2(f2(vt.xih[i][2]), uhz, s);
        float2 t = c2;
        if (N >= 4) t = fma2(fma2(c4, s, c3), s, c2);
        else if (N >= 3) t = fma2(c3, s, c2);
        const float2 e = fma2(fma2(t, s, c1), s, c);  // A + rho Phi
        const float2 o = fma2(om, fv(i), mul2(f2(vt.wt[i]), e));
        if (simple) {
          store_pair(pf, o.x, o.y);
          if (im.n) {
            store_pair(pf + im.i0, o.x, o.y);
            if (im.n > 1) {
              store_pair(pf + im.i1, o.x, o.y);
              store_pair(pf + im.i2, o.x, o.y);
              if (im.n > 3) {
                store_pair(pf + im.i3, o.x, o.y);
                store_pair(pf + im.i4, o.x, o.y);
                store_pair(pf + im.i5, o.x, o.y);
                store_pair(pf + im.i6, o.x, o.y);
              }
            }
          }
        } else {
          store_all_images(pf - off, pd, x, y, z, Store<S>::st(o.x));
          if (in1) store_all_images(pf - off, pd, x + 1, y, z, Store<S>::st(o.y));
        }
        pf += pd.plane;
      }
    };

    // The adjoint of the collision for two neighbouring nodes per thread on
    // the paired FP32 pipe (FP32, up to 27 velocities); same arithmetic as
    // `adjoint` below.
    auto adjoint2 = [&](int n) {
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      const bool in1 = x + 1 < pd.n[0];
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      S* pf = dst + off;
      const float* sg = reinterpret_cast<const float*>(scr) + (size_t)Q * L::TILE + n;
      auto put2 = [&](float2 o) {
        if (simple) {
          store_pair(pf, o.x, o.y);
          if (im.n) {
            store_pair(pf + im.i0, o.x, o.y);
            if (im.n > 1) {
              store_pair(pf + im.i1, o.x, o.y);
              store_pair(pf + im.i2, o.x, o.y);
              if (im.n > 3) {
                store_pair(pf + im.i3, o.x, o.y);
                store_pair(pf + im.i4, o.x, o.y);
                store_pair(pf + im.i5, o.x, o.y);
                store_pair(pf + im.i6, o.x, o.y);
              }
            }
          }
        } else {
          store_all_images(pf - off, pd, x, y, z, Store<S>::st(o.x));
          if (in1) store_all_images(pf - off, pd, x + 1, y, z, Store<S>::st(o.y));
        }
        pf += pd.plane;
      };
      if (a.mode == 2) {
#pragma unroll
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          put2(*reinterpret_cast<const float2*>(sg + (size_t)i * L::TILE));
        }
        return;
      }
      // moments of the pulled forward populations, recorded by the forward step
      const float* mf = reinterpret_cast<const float*>(mom) + n;
      const float2 A = *reinterpret_cast<const float2*>(mf);
      const float2 jx = *reinterpret_cast<const float2*>(mf + L::TILE);
      const float2 jy = *reinterpret_cast<const float2*>(mf + 2 * L::TILE);
      const float2 jz = *reinterpret_cast<const float2*>(mf + 3 * L::TILE);
      float2 sig[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) sig[i] = i < Q ? *reinterpret_cast<const float2*>(sg + (size_t)i * L::TILE) : f2(0.f);
      const float2 rho = add2(f2(sc.rho_ref), A);
      const float2 irc = make_float2(sc.inv_cs / rho.x, sc.inv_cs / rho.y);
      const float2 uhx = uhat2_of(a, jx, irc, 0), uhy = uhat2_of(a, jy, irc, 1), uhz = uhat2_of(a, jz, irc, 2);
      const float2 q = fma2(uhz, uhz, fma2(uhy, uhy, mul2(uhx, uhx)));
      float2 ca = f2(0.f), bx = f2(0.f), by = f2(0.f), bz = f2(0.f), bq = f2(0.f);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        float2 s = mul2(f2(vt.xih[i][0]), uhx);
        s = fma2(f2(vt.xih[i][1]), uhy, s);
        if (D == 3) s = fma2(f2(vt.xih[i][2]), uhz, s);
        // Phi, dPhi/ds, dPhi/dq of order N (isothermal)
        const float2 s2 = mul2(s, s);
        const float2 h = sub2(s2, q);
        float2 ph = fma2(f2(0.5f), h, s), ps = add2(f2(1.f), s), pq = f2(-0.5f);
        if (N >= 3) {
          ph = fma2(f2(1.0f / 6.0f), mul2(s, sub2(s2, mul2(f2(3.f), q))), ph);
          ps = fma2(f2(0.5f), h, ps);
          pq = fma2(f2(-0.5f), s, pq);
        }
        const float2 v = mul2(f2(vt.w[i]), sig[i]);
        // 1 + Phi - s dPhi/ds - 2 q dPhi/dq
        const float2 term = fma2(mul2(f2(-2.f), q), pq, fma2(mul2(f2(-1.f), s), ps, add2(f2(1.f), ph)));
        ca = fma2(v, term, ca);
        const float2 vs = mul2(v, ps);
        bx = fma2(vs, f2(vt.xih[i][0]), bx);
        by = fma2(vs, f2(vt.xih[i][1]), by);
        if (D == 3) bz = fma2(vs, f2(vt.xih[i][2]), bz);
        bq = fma2(mul2(f2(2.f), v), pq, bq);
      }
      bx = fma2(bq, uhx, bx);
      by = fma2(bq, uhy, by);
      bz = fma2(bq, uhz, bz);
      const float2 keep_s = f2(1.f - sc.inv_tau), itau = f2(sc.inv_tau);
#pragma unroll
      for (int k = 0; k < QM; ++k) {
        if (k >= Q) break;
        float2 g = fma2(bx, f2(vt.xih[k][0]), ca);
        g = fma2(by, f2(vt.xih[k][1]), g);
        if (D == 3) g = fma2(bz, f2(vt.xih[k][2]), g);
        put2(fma2(keep_s, sig[k], mul2(g, itau)));
      }
    };

    // adjoint of the collision of one node (isothermal): staged planes
    // q < Q hold the pulled forward populations f~, planes Q + i the pulled
    // adjoint sigma_i.  mu_k = (1 - 1/tau) sigma_k + (a + b . xi^_k) / tau with
    // a = sum_i w_i sigma_i (1 + Phi_i - s_i dPhi/ds - 2 q dPhi/dq) and
    // b = sum_i w_i sigma_i (dPhi/ds xi^_i + 2 dPhi/dq u^).  Mode 2 copies sigma.
    auto adjoint = [&](int n) {
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) return;
      const Images im = images_of(x, y, z);
      const long long off = pad_index(pd, x, y, z);
      S* pf = dst + off;
      const C* sg = scr + (size_t)Q * L::TILE + n;
      if (a.mode == 2) {
#pragma unroll
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          im.put(pf, Store<S>::st(sg[(size_t)i * L::TILE]), pd, off, x, y, z);
          pf += pd.plane;
        }
        return;
      }
      // moments of the pulled forward populations, recorded by the forward step
      const C A = mom[n], jx = mom[L::TILE + n], jy = mom[2 * L::TILE + n], jz = mom[3 * L::TILE + n];
      C sig[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) sig[i] = i < Q ? sg[(size_t)i * L::TILE] : C(0);
      const C irc = sc.inv_cs / (sc.rho_ref + A);
      const C uhx = uhat_of<COMP>(a, jx, irc, 0), uhy = uhat_of<COMP>(a, jy, irc, 1), uhz = uhat_of<COMP>(a, jz, irc, 2);
      const C q = uhx * uhx + uhy * uhy + uhz * uhz;
      C ca = C(0), bx = C(0), by = C(0), bz = C(0), bq = C(0);
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        C s = vt.xih[i][0] * uhx;
        s = fma(vt.xih[i][1], uhy, s);
        if (D == 3) s = fma(vt.xih[i][2], uhz, s);
        C ph, ps, pq;
        phi_grad<C, N>(s, q, ph, ps, pq);
        const C v = vt.w[i] * sig[i];
        ca = fma(v, C(1) + ph - s * ps - C(2) * q * pq, ca);
        const C vs = v * ps;
        bx = fma(vs, vt.xih[i][0], bx);
        by = fma(vs, vt.xih[i][1], by);
        if (D == 3) bz = fma(vs, vt.xih[i][2], bz);
        bq = fma(C(2) * v, pq, bq);
      }
      bx = fma(bq, uhx, bx);
      by = fma(bq, uhy, by);
      bz = fma(bq, uhz, bz);
      const C keep_s = C(1) - sc.inv_tau;
#pragma unroll
      for (int k = 0; k < QM; ++k) {
        if (k >= Q) break;
        C g = fma(bx, vt.xih[k][0], ca);
        g = fma(by, vt.xih[k][1], g);
        if (D == 3) g = fma(bz, vt.xih[k][2], g);
        im.put(pf, Store<S>::st(fma(keep_s, sig[k], g * sc.inv_tau)), pd, off, x, y, z);
        pf += pd.plane;
      }
    };

    if constexpr (SMB) {
      constexpr int NCH = L::TILE / CHN;
      C* sbuf = reinterpret_cast<C*>(base + (SG::OWN ? SG::OFF_S : 0));
      auto stage = [&](int c, int b) {
        if (tid == 0) {
          // the chunk buffer was last read through the generic proxy
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_expect_tx(sbar + b, (unsigned)(planes * CHN * sizeof(C)));
          C* d = sbuf + (size_t)b * SPMAX * CHN;
          for (int p = 0; p < planes; ++p)
            bulk_g2s(d + p * CHN, scr + (size_t)p * L::TILE + c * CHN, (unsigned)(CHN * sizeof(C)), sbar + b);
        }
        spend |= 1u << b;
      };
      stage(0, 0);
      if (SNBUF > 1 && NCH > 1) stage(1, 1);
      for (int c = 0; c < NCH; ++c) {
        const int b = SNBUF > 1 ? (c & 1) : 0;
        if (__syncthreads_or(!mbar_wait_bounded(sbar + b, (spar >> b) & 1u))) {
          failed = true;
          break;
        }
        spar ^= 1u << b;
        spend &= ~(1u << b);
        const C* chunk = sbuf + (size_t)b * SPMAX * CHN;
        if constexpr (SPAIR) {
          if (red) {  // logging steps: one node at a time (the sums fit in registers)
            for (int e = tid; e < CHN; e += L::NT)
              collide_from(c * CHN + e, chunk + e, std::integral_constant<int, CHN>(), std::true_type());
          } else {
            collide2_from(c * CHN + 2 * tid, reinterpret_cast<const float*>(chunk) + 2 * tid,
                          std::integral_constant<int, CHN>());
          }
        } else if (red) {
          collide_from(c * CHN + tid, chunk + tid, std::integral_constant<int, CHN>(), std::true_type());
        } else {
          collide_from(c * CHN + tid, chunk + tid, std::integral_constant<int, CHN>(), std::false_type());
        }
        __syncthreads();  // chunk buffer b read by every thread
        if (c + SNBUF < NCH) stage(c + SNBUF, b);
      }
      if (failed) break;
      // the boxes are free again: the next tile's first two copies of each
      // warpgroup (the one-box pull of the 2D kernels has issued its own)
      const int tn = tile + gridDim.x;
      if (SG::IN_BOXES && tn < a.ntiles && nplan > 0) {
        if (wt == 0) issue(tn, sched.plane[wg][0], cb);
        if (cb) pending1 = true;
        else pending = true;
        int t1 = tn, k1 = 0;
        advance(t1, k1, 1);
        if (t1 < a.ntiles) {
          if (wt == 0) issue(t1, sched.plane[wg][k1], cb ^ 1);
          if (cb ^ 1) pending1 = true;
          else pending = true;
        }
      }
    } else if constexpr (ADJ && APAIRS) {
      for (int n = 2 * tid; n < L::TILE; n += 2 * NT) adjoint2(n);
    } else if constexpr (ADJ) {
      for (int n = tid; n < L::TILE; n += NT) adjoint(n);
    } else if constexpr (PAIRS) {
      // the logging steps take the one-node path (its sums fit in registers)
      if (red) {
        for (int n = tid; n < L::TILE; n += NT) collide(n, std::integral_constant<bool, true>());
      } else {
        for (int n = 2 * tid; n < L::TILE; n += 2 * NT) collide2(n);
      }
    } else {
      if (red) {
        for (int n = tid; n < L::TILE; n += NT) collide(n, std::integral_constant<bool, true>());
      } else {
        for (int n = tid; n < L::TILE; n += NT) collide(n, std::integral_constant<bool, false>());
      }
    }
    if (red) {
#pragma unroll
      for (int c = 0; c < NRED; ++c) {
        C v = tsum[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red_smem[warp * NRED + c] += (double)v;
      }
    }
    __syncthreads();  // the staging slab is reused by the next tile
  }

  if (failed) {
    if (tid == 0) atomicExch(a.err, 1);
    // let the copies in flight land
    if (wt == 0 && pending) mbar_wait_bounded(bar, parity & 1u);
    if (wt == 0 && pending1) mbar_wait_bounded(bar + 1, (parity >> 1) & 1u);
    if (tid == 0 && (spend & 1u)) mbar_wait_bounded(sbar, spar & 1u);
    if (tid == 0 && (spend & 2u)) mbar_wait_bounded(sbar + 1, (spar >> 1) & 1u);
    return;
  }
  if (!ADJ && a.reduce) {
    __syncthreads();
    if (tid < NRED) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red_smem[w * NRED + tid];
      a.partials[(size_t)blockIdx.x * NRED + tid] = s;
    }
  }
}

// Forward step (Sec. 3): pull, moments, equilibrium, BGK, global sums.
template <int D, int P, typename S, bool COMP, int QM, int N>
__global__ void __launch_bounds__(GLayout<D, P, S>::NT, GLayout<D, P, S>::CTAS)
    sl_wg_kernel(const StepArgs a, const __grid_constant__ VelTab<typename Store<S>::C> vt,
                 const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st,
                 const __grid_constant__ TmaMaps maps, const __grid_constant__ WgSchedule sched) {
  wg_body<D, P, S, COMP, QM, N, false>(a, vt, st, st, maps, sched);
}

// One step of the adjoint sweep of the isothermal step, in terms of
// mu_t = dJ/d(pulled populations of step t):
//   mu_{t-1} = Jc(f~_{t-1})^T S^T mu_t,  f~_{t-1} = S f_{t-2},
// with S the pull (stencil st on the forward state, maps.m[0]) and S^T the
// pull with the reflected stencil st2 on mu_t (maps.m[1]).  With st2 the
// identity the kernel gives the first step of the sweep, Jc^T lambda; with
// mode 2 it only applies st2 (the last step, S^T mu_1).
template <int D, int P, typename S, int QM, int N>
__global__ void __launch_bounds__(GLayout<D, P, S>::NT, GLayout<D, P, S>::CTAS)
    sl_adj_kernel(const StepArgs a, const __grid_constant__ VelTab<typename Store<S>::C> vt,
                  const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st,
                  const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st2,
                  const __grid_constant__ TmaMaps maps, const __grid_constant__ WgSchedule sched) {
  wg_body<D, P, S, false, QM, N, true>(a, vt, st, st2, maps, sched);
}

template <int D, int P, typename S, int QM, int N>
int launch_adj(const StepLaunch& Lc) {
  using C = typename Store<S>::C;
  using Lay = GLayout<D, P, S>;
  auto kern = sl_adj_kernel<D, P, S, QM, N>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
    if (e != cudaSuccess) return (int)e;
    attr_done = true;
  }
  const auto& vt = *static_cast<const VelTab<C>*>(Lc.veltab);
  const auto& st = *static_cast<const StencilTab<C, P + 1>*>(Lc.stentab);
  const auto& st2 = *static_cast<const StencilTab<C, P + 1>*>(Lc.stentab2);
  kern<<<Lc.grid, Lay::NT, Lay::BYTES, static_cast<cudaStream_t>(Lc.stream)>>>(Lc.a, vt, st, st2, *Lc.maps,
                                                                               *Lc.sched);
  return (int)cudaGetLastError();
}

template <int D, int P, typename S, bool COMP, int QM, int N>
int launch_wg(const StepLaunch& Lc) {
  using C = typename Store<S>::C;
  using Lay = GLayout<D, P, S>;
  constexpr size_t bytes = Staging<D, P, S, COMP, QM, false>::BYTES;
  auto kern = sl_wg_kernel<D, P, S, COMP, QM, N>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    attr_done = true;
  }
  const auto& vt = *static_cast<const VelTab<C>*>(Lc.veltab);
  const auto& st = *static_cast<const StencilTab<C, P + 1>*>(Lc.stentab);
  kern<<<Lc.grid, Lay::NT, bytes, static_cast<cudaStream_t>(Lc.stream)>>>(Lc.a, vt, st, *Lc.maps, *Lc.sched);
  return (int)cudaGetLastError();
}

template <int D, int P, typename S, bool COMP, int QM, int N>
int occupancy_wg(StepInfo* o) {
  using Lay = GLayout<D, P, S>;
  constexpr size_t bytes = Staging<D, P, S, COMP, QM, false>::BYTES;
  auto kern = sl_wg_kernel<D, P, S, COMP, QM, N>;
  o->bxw = Lay::BXW;
  o->by = Lay::BY;
  o->bz = Lay::BZ;
  o->tile = Lay::TILE;
  o->tx = Lay::TX;
  o->ty = Lay::TY;
  o->tz = Lay::TZ;
  o->vec = Lay::VEC;
  o->smem = bytes;
  o->wg = Lay::NWG;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Lay::NT, bytes) != cudaSuccess) return 0;
  return n;
}

}  // namespace wg
}  // namespace olb
