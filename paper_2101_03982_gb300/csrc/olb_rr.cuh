// Register-resident fused step (the hot path of the isothermal sets with up to
// 28 populations in shifted FP32 storage), sm_103a.
//
// Same method, data layout and results as the two-phase kernel (olb_wg.cuh):
// ghost-padded planes, TMA-staged boxes, separable z/y/x Lagrange passes
// (Sec. 3, Eq. sl_streaming), moments, the order-N Hermite equilibrium in
// closed form (Appendix A) and BGK (Sec. 3).  What differs is where the
// pulled values live between the pull and the collision:
//
//   Tile 32 x 8 x 4 = 1024 nodes.  The CTA is four warpgroups; each streams
//   its host-balanced list of at most KMAX planes through two shared-memory
//   boxes (the TMA copy of a plane lands while the plane before it is
//   processed) and runs the z and y passes in place.  The x pass leaves each
//   thread the pulled values of its own 8 nodes (two 4-node x groups) in
//   registers, for every plane of its warpgroup: nothing is staged in global
//   memory and nothing is re-read.
//
//   Moments.  Each warpgroup sums rho and rho u over its planes for its nodes
//   and writes these partial moments to shared memory; after one CTA barrier
//   every thread finishes two nodes (rho, u / c_s) and after a second one
//   each warpgroup applies the equilibrium and BGK to its own planes with the
//   values still in registers, and stores them with 128-bit stores (ghost
//   copies included).
//
//   Logging steps also accumulate the non-equilibrium stress of each node
//   over the warpgroup's planes; the four partial stresses are added in a
//   fixed order through shared memory before the per-node sums, which are
//   reduced per warp and CTA in FP64 in a fixed order.
//
// Every mbarrier wait is bounded: a wait that runs out raises the device
// error flag and the kernel returns after its copies in flight have landed.
#pragma once

#include "olb_wg.cuh"

namespace olb {
namespace rr {

using wg::WGT;

// What a warpgroup needs of one of its planes, copied once per CTA from the
// kernel's parameter tables into shared memory: every per-plane lookup in the
// loops is then a broadcast shared-memory load instead of a constant-bank load
// with a run-time index (whose cache misses stalled the pull and the
// collision).
template <int P>
struct alignas(16) PlaneRec {
  int plane, act, m0[3], xo, pad0, pad1;  // index, active axes, stencil origin, x alignment of the box
  float xih[3], wt;                        // xi / c_s, w / tau
  float xi[3], w;                          // xi, w
  float xx[6], pad2[2];                    // xi_a xi_b
  float W[3][P + 1];                       // Lagrange weights per axis
};

template <int P, typename S>
struct RLayout {
  static constexpr int TX = 32, TY = 8, TZ = 4, TILE = TX * TY * TZ;
  static constexpr int VEC = 16 / (int)sizeof(S);
  static constexpr int ALIGN = cmax(VEC, 4);
  static constexpr int BXW = roundup(TX + P + VEC - 1, ALIGN);
  static constexpr int NQX = BXW / 4;
  static constexpr int BY = TY + P, BZ = TZ + P;
  static constexpr size_t BOXB = (size_t)roundup(BZ * BY * BXW * (int)sizeof(S), 128);
  static constexpr int NWG = 4, NT = NWG * WGT;
  static constexpr int KMAX = 7;                  // planes per warpgroup
  static constexpr int QPT = TILE / 4 / WGT;      // 4-node x groups per thread (2)
  // shared memory: two boxes per warpgroup, partial moments [NWG][4][TILE],
  // per-node coefficients [4][TILE] (A, u^x, u^y, u^z), logging partials,
  // mbarriers
  static constexpr size_t OFF_PART = NWG * 2 * BOXB;
  static constexpr size_t OFF_COEF = OFF_PART + (size_t)NWG * 4 * TILE * sizeof(float);
  static constexpr size_t OFF_R = OFF_COEF + (size_t)4 * TILE * sizeof(float);
  static constexpr size_t OFF_T = OFF_R + (NT / 32) * NRED * sizeof(double);
  static constexpr size_t OFF_M = OFF_T + (size_t)NWG * KMAX * sizeof(PlaneRec<P>);
  static constexpr size_t BYTES = OFF_M + 2 * NWG * sizeof(unsigned long long) + 128;
  static_assert(QPT == 2, "each thread owns two x groups");
  static_assert(BYTES <= 227 * 1024, "shared memory");
  static_assert(4 * ((3 + 3 + P) / 4 + 1) + TX - 4 <= BXW, "x pass reads inside the box row");
  // the non-equilibrium stress of the logging steps reuses the partial-moment area
  static_assert((size_t)NWG * 6 * (TILE / QPT) * sizeof(float) <= (size_t)NWG * 4 * TILE * sizeof(float),
                "stress buffer");
};

// 128-bit store of four FP32 values.
__device__ __forceinline__ void st4f(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int P, int N, bool RED>
__device__ __forceinline__ void rr_body(const StepArgs& a, const VelTab<float>& vt, const StencilTab<float, P + 1>& st,
                                        const TmaMaps& maps, const WgSchedule& sched) {
  using S = float;
  using L = RLayout<P, S>;
  using T2 = float2;
  constexpr int KMAX = L::KMAX;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base, kept as arithmetic on the shared array so that the
  // compiler addresses it as shared memory (no generic loads and stores)
  unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = tid / WGT, wt = tid % WGT;
  float* box0 = reinterpret_cast<float*>(base + (size_t)wg * 2 * L::BOXB);
  float* box1 = reinterpret_cast<float*>(base + (size_t)wg * 2 * L::BOXB + L::BOXB);
  float* part = reinterpret_cast<float*>(base + L::OFF_PART);
  float* coef = reinterpret_cast<float*>(base + L::OFF_COEF);
  double* red_smem = reinterpret_cast<double*>(base + L::OFF_R);
  PlaneRec<P>* ptab = reinterpret_cast<PlaneRec<P>*>(base + L::OFF_T);
  const PlaneRec<P>* mytab = ptab + wg * KMAX;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + L::OFF_M) + 2 * wg;

  const Padded& pd = a.pad;
  const CUtensorMap* maps4 = maps.m[a.src];
  const int nplan = sched.n[wg];
  float* __restrict__ dst = static_cast<float*>(a.buf[a.src ^ 1]);
  const float rho_ref = a.f_rho_ref, inv_cs = a.f_inv_cs, om = 1.f - a.f_inv_tau;

  // padded-grid coordinates of the box of a plane of a tile (one thread)
  auto box_coords = [&](int tile, const PlaneRec<P>& R, int& X, int& Y, int& Z) {
    const int tx = tile % a.nt[0], r = tile / a.nt[0];
    const int org[3] = {tx * L::TX + pd.gl[0], (r % a.nt[1]) * L::TY + pd.gl[1], (r / a.nt[1]) * L::TZ + pd.gl[2]};
    const int act = R.act;
    X = org[0] + ((act & 1) ? R.m0[0] : 0);
    X -= X % L::VEC;
    Y = org[1] + ((act & 2) ? R.m0[1] : 0);
    Z = org[2] + ((act & 4) ? R.m0[2] : 0);
    return ((act & 2) ? 1 : 0) | ((act & 4) ? 2 : 0);
  };
  // TMA copy of slot k's plane of `tile` into box b (one thread)
  auto issue = [&](int tile, int k, int b) {
    const PlaneRec<P>& R = mytab[k];
    int X, Y, Z;
    const int v = box_coords(tile, R, X, Y, Z);
    const unsigned bytes = (unsigned)(L::BXW * ((v & 1) ? L::BY : L::TY) * ((v & 2) ? L::BZ : L::TZ) * sizeof(S));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar + b, bytes);
    tma_load_4d(b ? box1 : box0, &maps4[v], X, Y, Z, R.plane, bar + b);
  };
  // (tile, k) of the plane `steps` after (tile, k) in this warpgroup's stream
  auto advance = [&](int& t, int& k, int steps) {
    k += steps;
    while (k >= nplan) {
      k -= nplan;
      t += gridDim.x;
    }
  };

  if (wt == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  if (tid < (L::NT / 32) * NRED) red_smem[tid] = 0.0;
  if (tid < L::NWG * KMAX) {
    const int w = tid / KMAX, k = tid % KMAX;
    if (k < sched.n[w]) {
      PlaneRec<P>& R = ptab[tid];
      const int i = sched.plane[w][k];
      R.plane = i;
      R.act = st.active[i];
      for (int c = 0; c < 3; ++c) {
        R.m0[c] = st.m0[i][c];
        R.xih[c] = vt.xih[i][c];
        R.xi[c] = vt.xi[i][c];
        for (int j = 0; j <= P; ++j) R.W[c][j] = st.W[i][c][j];
      }
      R.xo = (R.act & 1) ? ((st.m0[i][0] % L::VEC) + L::VEC) % L::VEC : 0;
      R.wt = vt.wt[i];
      R.w = vt.w[i];
      for (int c = 0; c < 6; ++c) R.xx[c] = vt.xx[i][c];
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  bool pending = false, pending1 = false;  // a copy into box 0 / box 1 is in flight
  if (nplan > 0 && (int)blockIdx.x < a.ntiles) {
    if (wt == 0) issue(blockIdx.x, 0, 0);
    pending = true;
    int t1 = blockIdx.x, k1 = 0;
    advance(t1, k1, 1);
    if (t1 < a.ntiles) {
      if (wt == 0) issue(t1, k1, 1);
      pending1 = true;
    }
  }
  unsigned parity = 0;  // bit b: phase parity of box b's barrier
  int cb = 0;           // box of the current plane
  bool failed = false;
  const bool simple = a.quad_ok && pd.n[0] >= pd.gl[0] + pd.gr[0] && pd.n[1] >= pd.gl[1] + pd.gr[1] &&
                      pd.n[2] >= pd.gl[2] + pd.gr[2];
  float tsum[NRED];
#pragma unroll
  for (int c = 0; c < NRED; ++c) tsum[c] = 0.f;
  // per-thread offsets in the box, computed once: the y column of the y pass
  // (z row yz, first x value yq2) and the first value of each x group's row
  // after the z and y passes (y extended by the stencil or not)
  constexpr int NPXc = L::BXW / 2;
  const int yz = wt / NPXc, yq2 = 2 * (wt % NPXc);
  // group m of this thread: row (lz, ly), first x qx; its offset in a box
  // whose y extent is TY (yact false) or BY
  const int xoffN0 = ((wt / (L::TX / 4 * L::TY)) * L::TY + (wt / (L::TX / 4)) % L::TY) * L::BXW + (wt % (L::TX / 4)) * 4;
  const int lz0 = wt / (L::TX / 4 * L::TY);
  static_assert(WGT == 2 * (L::TX / 4) * L::TY, "group m = 1 lies two z rows below group 0");
  auto xoff = [&](int m, bool yact) {
    const int lz = lz0 + 2 * m;
    return xoffN0 + 2 * m * L::TY * L::BXW + (yact ? lz * P * L::BXW : 0);
  };

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    // ------------- pull: the warpgroup's planes, values kept in registers -------------
    float v[KMAX][8];
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
#pragma unroll
      for (int e = 0; e < 8; ++e) v[k][e] = 0.f;
#pragma unroll 1
    for (int k = 0; k < nplan; ++k) {
      const PlaneRec<P>& R = mytab[k];
      if (wg::wg_any(wg, !mbar_wait_bounded(bar + cb, (parity >> cb) & 1u, a.wait_polls))) {
        failed = true;
        break;
      }
      parity ^= 1u << cb;
      if (cb) pending1 = false;
      else pending = false;
      const int act = R.act;
      const bool zact = (act & 4) != 0, yact = (act & 2) != 0, xact = (act & 1) != 0;
      float* bx = cb ? box1 : box0;
      const int BYA = yact ? L::BY : L::TY;
      const int PLs = BYA * L::BXW;
      static_assert(L::BXW == 2 * (L::BXW / 2), "pairs of x values per row");
      // z and y passes in place on pairs of x values (one column of pairs
      // per thread: its inputs slide through a window of P + 1 rows, each
      // output overwrites a row the column no longer reads)
      constexpr int NPX = L::BXW / 2;  // x pairs per box row
      if (zact) {
        T2 W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = wg::f2(R.W[2][j]);
        const int ncol = NPX * BYA;
        for (int col = wt; col < ncol; col += WGT) {
          float* c0 = bx + 2 * col;  // row col / NPX, pair col % NPX (BXW = 2 NPX)
          T2 win[P + 1];
#pragma unroll
          for (int kk = 0; kk < P; ++kk) win[kk] = *reinterpret_cast<const T2*>(c0 + kk * PLs);
#pragma unroll
          for (int z = 0; z < L::TZ; ++z) {
            win[(z + P) % (P + 1)] = *reinterpret_cast<const T2*>(c0 + (z + P) * PLs);
            T2 acc = wg::mul2(W[0], win[z % (P + 1)]);
#pragma unroll
            for (int kk = 1; kk <= P; ++kk) acc = wg::fma2(W[kk], win[(z + kk) % (P + 1)], acc);
            *reinterpret_cast<T2*>(c0 + z * PLs) = acc;
          }
        }
        wg::wg_barrier(wg);
      }
      if (yact) {
        T2 W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = wg::f2(R.W[1][j]);
        constexpr int ncol = NPX * L::TZ;
        static_assert(ncol <= WGT, "one y column per thread");
        if (wt < ncol) {
          float* c0 = bx + yz * PLs + yq2;
          T2 win[P + 1];
#pragma unroll
          for (int kk = 0; kk < P; ++kk) win[kk] = *reinterpret_cast<const T2*>(c0 + kk * L::BXW);
#pragma unroll
          for (int y = 0; y < L::TY; ++y) {
            win[(y + P) % (P + 1)] = *reinterpret_cast<const T2*>(c0 + (y + P) * L::BXW);
            T2 acc = wg::mul2(W[0], win[y % (P + 1)]);
#pragma unroll
            for (int kk = 1; kk <= P; ++kk) acc = wg::fma2(W[kk], win[(y + kk) % (P + 1)], acc);
            *reinterpret_cast<T2*>(c0 + y * L::BXW) = acc;
          }
        }
        wg::wg_barrier(wg);
      }
      // x pass: the two 4-node groups of this thread, one alignment variant per plane
      float out[8];
      {
        float W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = R.W[0][j];
        const int xo = R.xo;
        auto groups = [&](auto XOc, auto ACT) {
#pragma unroll
          for (int m = 0; m < L::QPT; ++m) {
            wg::xrow<P, decltype(XOc)::value, decltype(ACT)::value>(bx + xoff(m, yact), W, out + 4 * m);
          }
        };
        if (!xact) {
          groups(std::integral_constant<int, 0>(), std::false_type());
        } else {
          switch (xo) {
            case 0: groups(std::integral_constant<int, 0>(), std::true_type()); break;
            case 1: groups(std::integral_constant<int, 1>(), std::true_type()); break;
            case 2: groups(std::integral_constant<int, 2>(), std::true_type()); break;
            default: groups(std::integral_constant<int, 3>(), std::true_type()); break;
          }
        }
      }
      // into the register slot of this plane (k is uniform over the warpgroup)
      switch (k) {
#define OLB_RR_SLOT(K)                           \
  case K:                                        \
    _Pragma("unroll") for (int e = 0; e < 8; ++e) v[K][e] = out[e]; \
    break;
        OLB_RR_SLOT(0)
        OLB_RR_SLOT(1)
        OLB_RR_SLOT(2)
        OLB_RR_SLOT(3)
        OLB_RR_SLOT(4)
        OLB_RR_SLOT(5)
        default:
#pragma unroll
          for (int e = 0; e < 8; ++e) v[KMAX - 1][e] = out[e];
          break;
#undef OLB_RR_SLOT
      }
      wg::wg_barrier(wg);  // box free
      int t2 = tile, k2 = k;
      advance(t2, k2, 2);
      if (t2 < a.ntiles) {
        if (wt == 0) issue(t2, k2, cb);
        if (cb) pending1 = true;
        else pending = true;
      }
      cb ^= 1;
    }

    // ------------- partial moments of this warpgroup's planes -------------
    {
      float A[8], jx[8], jy[8], jz[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) A[e] = jx[e] = jy[e] = jz[e] = 0.f;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k >= nplan) break;
        const float cx = mytab[k].xi[0], cy = mytab[k].xi[1], cz = mytab[k].xi[2];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          A[e] += v[k][e];
          jx[e] = fmaf(cx, v[k][e], jx[e]);
          jy[e] = fmaf(cy, v[k][e], jy[e]);
          jz[e] = fmaf(cz, v[k][e], jz[e]);
        }
      }
#pragma unroll
      for (int m = 0; m < L::QPT; ++m) {
        const int n0 = 4 * (wt + WGT * m);
        float* pw = part + (size_t)wg * 4 * L::TILE + n0;
        st4f(pw, A[4 * m], A[4 * m + 1], A[4 * m + 2], A[4 * m + 3]);
        st4f(pw + L::TILE, jx[4 * m], jx[4 * m + 1], jx[4 * m + 2], jx[4 * m + 3]);
        st4f(pw + 2 * L::TILE, jy[4 * m], jy[4 * m + 1], jy[4 * m + 2], jy[4 * m + 3]);
        st4f(pw + 3 * L::TILE, jz[4 * m], jz[4 * m + 1], jz[4 * m + 2], jz[4 * m + 3]);
      }
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    const int tx = tile % a.nt[0], tr = tile / a.nt[0];
    const int ty = tr % a.nt[1], tz = tr / a.nt[1];

    // ------------- per-node moments: two nodes per thread, fixed order over the warpgroups -------------
    {
      const int n0 = 2 * tid;
      T2 s[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        s[c] = *reinterpret_cast<const T2*>(part + (size_t)c * L::TILE + n0);
#pragma unroll
        for (int w = 1; w < L::NWG; ++w)
          s[c] = wg::add2(s[c], *reinterpret_cast<const T2*>(part + (size_t)(w * 4 + c) * L::TILE + n0));
      }
      const T2 rho = wg::add2(wg::f2(rho_ref), s[0]);
      const T2 irc = make_float2(inv_cs / rho.x, inv_cs / rho.y);
      const T2 uhx = uhat2_of(a, s[1], irc, 0), uhy = uhat2_of(a, s[2], irc, 1), uhz = uhat2_of(a, s[3], irc, 2);
      if (RED) {
        // k, rho k, mass and momentum of the tile's interior nodes
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int n = n0 + h;
          const int x = tx * L::TX + n % L::TX, y = ty * L::TY + (n / L::TX) % L::TY,
                    z = tz * L::TZ + n / (L::TX * L::TY);
          if (x >= pd.n[0] || y >= pd.n[1] || z >= pd.n[2]) continue;
          const float r = h ? rho.y : rho.x, A = h ? s[0].y : s[0].x;
          const float ux = h ? uhx.y : uhx.x, uy = h ? uhy.y : uhy.x, uz = h ? uhz.y : uhz.x;
          const float u2 = (ux * ux + uy * uy + uz * uz) * a.f_cs2;
          tsum[0] += 0.5f * u2;
          tsum[1] += 0.5f * r * u2;
          tsum[3] += A;
          tsum[4] += h ? s[1].y : s[1].x;
          tsum[5] += h ? s[2].y : s[2].x;
          tsum[6] += h ? s[3].y : s[3].x;
          const bool fin = isfinite(r) && isfinite(ux) && isfinite(uy) && isfinite(uz);
          tsum[7] += fin ? 0.f : 1.f;
        }
      }
      *reinterpret_cast<T2*>(coef + n0) = s[0];
      *reinterpret_cast<T2*>(coef + L::TILE + n0) = uhx;
      *reinterpret_cast<T2*>(coef + 2 * L::TILE + n0) = uhy;
      *reinterpret_cast<T2*>(coef + 3 * L::TILE + n0) = uhz;
    }
    __syncthreads();

    // ------------- equilibrium and BGK of this warpgroup's planes -------------
    // With c = A - rho q/2, c1 = rho [- rho q/2], c2 = rho/2, c3 = [rho/6]
    // (brackets: N = 3), A + rho Phi = c + s (c1 + s (c2 + s c3)) and
    // f_post = (1 - 1/tau) f + (w/tau)(A + rho Phi).
#pragma unroll
    for (int m = 0; m < L::QPT; ++m) {
      const int qi = wt + WGT * m, n0 = 4 * qi;
      const int qx = (qi % (L::TX / 4)) * 4, ly = (qi / (L::TX / 4)) % L::TY, lz = qi / (L::TX / 4 * L::TY);
      const int x = tx * L::TX + qx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      const bool yzin = y < pd.n[1] && z < pd.n[2];
      const float4 cA = *reinterpret_cast<const float4*>(coef + n0);
      const float4 cx = *reinterpret_cast<const float4*>(coef + L::TILE + n0);
      const float4 cy = *reinterpret_cast<const float4*>(coef + 2 * L::TILE + n0);
      const float4 cz = *reinterpret_cast<const float4*>(coef + 3 * L::TILE + n0);
      T2 Ap[2] = {make_float2(cA.x, cA.y), make_float2(cA.z, cA.w)};
      T2 ux[2] = {make_float2(cx.x, cx.y), make_float2(cx.z, cx.w)};
      T2 uy[2] = {make_float2(cy.x, cy.y), make_float2(cy.z, cy.w)};
      T2 uz[2] = {make_float2(cz.x, cz.y), make_float2(cz.z, cz.w)};
      // N = 2: c2 = c1 / 2; N = 3 keeps c2 and c3 = c2 / 3
      T2 c0[2], c1[2], c2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const T2 rho = wg::add2(wg::f2(rho_ref), Ap[h]);
        const T2 q = wg::fma2(uz[h], uz[h], wg::fma2(uy[h], uy[h], wg::mul2(ux[h], ux[h])));
        const T2 r2 = wg::mul2(wg::f2(0.5f), rho);
        c0[h] = wg::fma2(wg::f2(-1.f), wg::mul2(r2, q), Ap[h]);
        c1[h] = rho;
        c2[h] = r2;
        if (N >= 3) c1[h] = wg::fma2(wg::f2(-1.f), wg::mul2(r2, q), rho);
      }
      // periodic copies.  With nx a multiple of 4 (and the x ghost widths,
      // which are), a 4-node group lies wholly inside or outside each ghost
      // reach, so its copies are whole aligned groups: one 128-bit store each.
      // Ragged groups and grids shorter than their ghost widths store node by
      // node.
      const int dy = wg::one_image(y, pd.n[1], pd.gl[1], pd.gr[1]) * pd.np[0];
      const int dz = wg::one_image(z, pd.n[2], pd.gl[2], pd.gr[2]) * pd.np[0] * pd.np[1];
      const int dxq = wg::one_image(x, pd.n[0], pd.gl[0], pd.gr[0]);
      const bool fast = simple && yzin && x + 3 < pd.n[0];
      const wg::Images imq = wg::Images::make(dxq, dy, dz, true);
      const long long off = pad_index(pd, x, y, z);
      float Pi[6][4];
      if (RED) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) Pi[c][e] = 0.f;
      }
      // equilibrium and BGK of plane `plane` for the group's 4 nodes (values f)
      auto relax = [&](const PlaneRec<P>& R, const float f4[4], float o[4]) {
        const T2 hx = wg::f2(R.xih[0]), hy = wg::f2(R.xih[1]), hz = wg::f2(R.xih[2]);
        const T2 wtau = wg::f2(R.wt);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          T2 s = wg::mul2(hx, ux[h]);
          s = wg::fma2(hy, uy[h], s);
          s = wg::fma2(hz, uz[h], s);
          T2 t = N >= 3 ? c2[h] : wg::mul2(wg::f2(0.5f), c1[h]);
          if (N >= 3) t = wg::fma2(wg::mul2(wg::f2(1.0f / 3.0f), c2[h]), s, c2[h]);
          const T2 eq = wg::fma2(wg::fma2(t, s, c1[h]), s, c0[h]);  // A + rho Phi
          const T2 f = make_float2(f4[2 * h], f4[2 * h + 1]);
          const T2 r = wg::fma2(wg::f2(om), f, wg::mul2(wtau, eq));
          o[2 * h] = r.x;
          o[2 * h + 1] = r.y;
          if (RED) {
            // f~ - f^eq (the shift w rho0 cancels): the node pair's stress
            const T2 fneq = wg::fma2(wg::f2(-R.w), eq, f);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              const float xx = R.xx[c];
              Pi[c][2 * h] = fmaf(xx, fneq.x, Pi[c][2 * h]);
              Pi[c][2 * h + 1] = fmaf(xx, fneq.y, Pi[c][2 * h + 1]);
            }
          }
        }
      };
      if (fast) {
        // aligned group: one 128-bit store per plane and per periodic copy
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
          if (k >= nplan) break;
          const PlaneRec<P>& R = mytab[k];
          float o[4];
          const float f4[4] = {v[k][4 * m], v[k][4 * m + 1], v[k][4 * m + 2], v[k][4 * m + 3]};
          relax(R, f4, o);
          float* pf = dst + (long long)R.plane * pd.plane + off;
          st4f(pf, o[0], o[1], o[2], o[3]);
          if (imq.n) {
            st4f(pf + imq.i0, o[0], o[1], o[2], o[3]);
            if (imq.n > 1) {
              st4f(pf + imq.i1, o[0], o[1], o[2], o[3]);
              st4f(pf + imq.i2, o[0], o[1], o[2], o[3]);
              if (imq.n > 3) {
                st4f(pf + imq.i3, o[0], o[1], o[2], o[3]);
                st4f(pf + imq.i4, o[0], o[1], o[2], o[3]);
                st4f(pf + imq.i5, o[0], o[1], o[2], o[3]);
                st4f(pf + imq.i6, o[0], o[1], o[2], o[3]);
              }
            }
          }
        }
      } else if (yzin) {
        // a ragged group or a tiny grid: node by node, in a rolled loop (kept
        // out of the unrolled path)
#pragma unroll 1
        for (int k = 0; k < nplan; ++k) {
          const PlaneRec<P>& R = mytab[k];
          float f4[4];
          switch (k) {
#define OLB_RR_READ(K)                                                        \
  case K:                                                                     \
    _Pragma("unroll") for (int e = 0; e < 4; ++e) f4[e] = v[K][4 * m + e]; \
    break;
            OLB_RR_READ(0)
            OLB_RR_READ(1)
            OLB_RR_READ(2)
            OLB_RR_READ(3)
            OLB_RR_READ(4)
            OLB_RR_READ(5)
            default:
#pragma unroll
              for (int e = 0; e < 4; ++e) f4[e] = v[KMAX - 1][4 * m + e];
              break;
#undef OLB_RR_READ
          }
          float o[4];
          relax(R, f4, o);
          float* pf = dst + (long long)R.plane * pd.plane + off;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (x + e >= pd.n[0]) break;
            const int dx = wg::one_image(x + e, pd.n[0], pd.gl[0], pd.gr[0]);
            const wg::Images im = wg::Images::make(dx, dy, dz, simple);
            im.put(pf + e, o[e], pd, off + e, x + e, y, z);
          }
        }
      }
      if (RED) {
        // The stress of the nodes of group m of every thread (512 nodes), per
        // warpgroup, through the partial-moment area (free after the barrier
        // that published the coefficients): [NWG][6][512]; then each thread
        // adds the four in a fixed order for one node and forms 2 nu S:S.
        float* pis = part;
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 6; ++c)
          st4f(pis + (size_t)(wg * 6 + c) * 512 + 4 * wt, Pi[c][0], Pi[c][1], Pi[c][2], Pi[c][3]);
        __syncthreads();
        {
          const int j = tid;                   // node j % 4 of group j / 4 (thread j / 4 of a warpgroup)
          const int gq = j / 4 + WGT * m;      // its 4-node group in the tile
          const int n = 4 * gq + (j % 4);
          const int nx = tx * L::TX + n % L::TX, ny = ty * L::TY + (n / L::TX) % L::TY,
                    nz = tz * L::TZ + n / (L::TX * L::TY);
          if (nx < pd.n[0] && ny < pd.n[1] && nz < pd.n[2]) {
            float pi[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              pi[c] = pis[(size_t)c * 512 + j];
#pragma unroll
              for (int w = 1; w < L::NWG; ++w) pi[c] += pis[(size_t)(w * 6 + c) * 512 + j];
            }
            const float rho = rho_ref + coef[n];
            const float pres = rho * a.f_cs2;
            const float den = 2.f * pres * a.f_tau * a.f_dt;
            const float ss = (pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] +
                              2.f * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5])) /
                             (den * den);
            const float nu = a.f_cs2 * a.f_dt * (a.f_tau - 0.5f);
            tsum[2] += 2.f * nu * ss;
          }
        }
      }
    }
    // the logging steps' stress area is the next tile's partial-moment area
    if (RED) __syncthreads();
  }

  if (failed) {
    if (tid == 0) atomicExch(a.err, 1);
    // let the copies in flight land
    if (wt == 0 && pending) mbar_wait_bounded(bar, parity & 1u);
    if (wt == 0 && pending1) mbar_wait_bounded(bar + 1, (parity >> 1) & 1u);
    return;
  }
  if (RED) {
#pragma unroll
    for (int c = 0; c < NRED; ++c) {
      float vv = tsum[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vv += __shfl_down_sync(0xffffffffu, vv, o);
      if (lane == 0) red_smem[warp * NRED + c] = (double)vv;
    }
    __syncthreads();
    if (tid < NRED) {
      double s = 0.0;
      for (int w = 0; w < L::NT / 32; ++w) s += red_smem[w * NRED + tid];
      a.partials[(size_t)blockIdx.x * NRED + tid] = s;
    }
  }
}

// Forward step (Sec. 3) of the isothermal sets of up to 4 KMAX velocities in
// shifted FP32 storage: pull, moments, equilibrium, BGK (and on logging steps
// the global sums).
template <int P, int N, bool RED>
__global__ void __launch_bounds__(RLayout<P, float>::NT, 1)
    sl_rr_kernel(const StepArgs a, const __grid_constant__ VelTab<float> vt,
                 const __grid_constant__ StencilTab<float, P + 1> st, const __grid_constant__ TmaMaps maps,
                 const __grid_constant__ WgSchedule sched) {
  rr_body<P, N, RED>(a, vt, st, maps, sched);
}

template <int P, int N>
int launch_rr(const StepLaunch& Lc) {
  using Lay = RLayout<P, float>;
  auto k0 = sl_rr_kernel<P, N, false>;
  auto k1 = sl_rr_kernel<P, N, true>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
    if (e != cudaSuccess) return (int)e;
    attr_done = true;
  }
  const auto& vt = *static_cast<const VelTab<float>*>(Lc.veltab);
  const auto& st = *static_cast<const StencilTab<float, P + 1>*>(Lc.stentab);
  auto kern = Lc.a.reduce ? k1 : k0;
  kern<<<Lc.grid, Lay::NT, Lay::BYTES, static_cast<cudaStream_t>(Lc.stream)>>>(Lc.a, vt, st, *Lc.maps, *Lc.sched);
  return (int)cudaGetLastError();
}

template <int P, int N>
int occupancy_rr(StepInfo* o) {
  using Lay = RLayout<P, float>;
  auto kern = sl_rr_kernel<P, N, true>;
  o->bxw = Lay::BXW;
  o->by = Lay::BY;
  o->bz = Lay::BZ;
  o->tile = Lay::TILE;
  o->tx = Lay::TX;
  o->ty = Lay::TY;
  o->tz = Lay::TZ;
  o->vec = Lay::VEC;
  o->smem = Lay::BYTES;
  o->wg = Lay::NWG;
  o->kmax = Lay::KMAX;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES) != cudaSuccess)
    return 0;
  if (cudaFuncSetAttribute(sl_rr_kernel<P, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Lay::BYTES) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Lay::NT, Lay::BYTES) != cudaSuccess) return 0;
  return n;
}

}  // namespace rr
}  // namespace olb
