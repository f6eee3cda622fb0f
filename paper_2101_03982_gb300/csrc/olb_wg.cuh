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
//   z -> y -> x passes (warpgroup-local named barriers only) and writes the
//   pulled values f~_i of the tile to the CTA's staging slab (kept in L2).
//   No per-node state is carried from plane to plane, so the warpgroups never
//   wait for each other inside the phase.
//
//   Phase B (collide).  One thread per node loads the Q pulled values of its
//   node (all loads in flight together), forms rho, rho u (and the
//   temperature), the equilibrium and the BGK update with the velocity loop
//   unrolled (QM >= Q slots, so the per-velocity constants are constant-bank
//   operands), and writes the new state and its periodic copies.
//
// Two CTA barriers per tile separate the phases.  Every mbarrier wait is
// bounded: a wait that runs out raises the device error flag and the kernel
// returns after its copies in flight have landed.
#pragma once

#include "olb_step.cuh"

namespace olb {
namespace wg {

constexpr int WGT = 128;  // threads per warpgroup

template <int D, int P, typename S>
struct GLayout {
  using C = typename Store<S>::C;
  using B = Layout<D, P, S>;
  static constexpr int TX = B::TX, TY = B::TY, TZ = B::TZ, TILE = B::TILE, VEC = B::VEC;
  static constexpr int BXW = B::BXW, NQX = B::NQX, BY = B::BY, BZ = B::BZ;
  static constexpr int ZCH = 2, YCH = 2;
  static constexpr size_t BOXB = B::BOXB;
  static constexpr size_t ABYTES = (size_t)roundup((D == 3 ? TZ * BY * BXW : 4) * (int)sizeof(C), 128);
  static constexpr size_t BBYTES = (size_t)roundup(TZ * TY * BXW * (int)sizeof(C), 128);
  static constexpr size_t WGB = BOXB + ABYTES + BBYTES;  // shared memory of one warpgroup
  static constexpr size_t BUDGET = 227 * 1024 - 2048;
  static constexpr int NWG = (int)(BUDGET / WGB) >= 4 ? 4 : (int)(BUDGET / WGB);
  static constexpr int NT = NWG * WGT;
  static constexpr size_t OFF_R = NWG * WGB;
  static constexpr size_t OFF_M = OFF_R + (NT / 32) * NRED * sizeof(double);
  static constexpr size_t BYTES = OFF_M + 4 * sizeof(unsigned long long) + 128;
  static_assert(NWG >= 1, "one warpgroup must fit");
};

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
// axis with n >= gl + gr nodes (0 when c has none).
__device__ __forceinline__ int one_image(int c, int n, int gl, int gr) {
  if (c < gr) return n;
  if (c >= n - gl) return -n;
  return 0;
}

template <int D, int P, typename S, bool COMP, int QM>
__global__ void __launch_bounds__(GLayout<D, P, S>::NT, 1)
    sl_wg_kernel(const StepArgs a, const __grid_constant__ VelTab<typename Store<S>::C> vt,
                 const __grid_constant__ StencilTab<typename Store<S>::C, P + 1> st,
                 const __grid_constant__ TmaMaps maps, const __grid_constant__ WgSchedule sched) {
  using L = GLayout<D, P, S>;
  using C = typename Store<S>::C;
  constexpr int NT = L::NT;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<size_t>(smem_raw) + 127) & ~size_t(127));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = tid / WGT, wt = tid % WGT;
  unsigned char* mine = base + wg * L::WGB;
  S* box = reinterpret_cast<S*>(mine);
  C* bufA = reinterpret_cast<C*>(mine + L::BOXB);
  C* bufB = reinterpret_cast<C*>(mine + L::BOXB + L::ABYTES);
  double* red_smem = reinterpret_cast<double*>(base + L::OFF_R);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(base + L::OFF_M) + wg;

  const int Q = a.Q, planes = a.planes;
  const Padded& pd = a.pad;
  const CUtensorMap* maps4 = maps.m[a.src];
  const int nplan = sched.n[wg];
  S* __restrict__ dst = static_cast<S*>(a.buf[a.src ^ 1]);
  C* __restrict__ scr = static_cast<C*>(a.scratch) + (size_t)blockIdx.x * planes * L::TILE;
  const unsigned long long keep = policy_evict_last(), stream_out = policy_evict_first();

  auto box_coords = [&](int tile, int plane, int& X, int& Y, int& Z) {
    const int tx = tile % a.nt[0], r = tile / a.nt[0];
    const int i = plane < Q ? plane : plane - Q;
    const int act = st.active[i];
    X = tx * L::TX + pd.gl[0] + ((act & 1) ? st.m0[i][0] : 0);
    X -= X % L::VEC;
    Y = (r % a.nt[1]) * L::TY + pd.gl[1] + ((act & 2) ? st.m0[i][1] : 0);
    Z = D == 3 ? (r / a.nt[1]) * L::TZ + pd.gl[2] + ((act & 4) ? st.m0[i][2] : 0) : 0;
    return ((act & 2) ? 1 : 0) | ((D == 3 && (act & 4)) ? 2 : 0);
  };
  auto issue = [&](int tile, int plane) {
    int X, Y, Z;
    const int v = box_coords(tile, plane, X, Y, Z);
    const unsigned bytes = (unsigned)(L::BXW * ((v & 1) ? L::BY : L::TY) * ((v & 2) ? L::BZ : L::TZ) * sizeof(S));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, bytes);
    tma_load_4d(box, &maps4[v], X, Y, Z, plane, bar);
  };
  auto prefetch = [&](int tile, int plane) {
    int X, Y, Z;
    const int v = box_coords(tile, plane, X, Y, Z);
    tma_prefetch_4d(&maps4[v], X, Y, Z, plane);
  };

  if (wt == 0) mbar_init(bar, 1);
  if (tid < (NT / 32) * NRED) red_smem[tid] = 0.0;
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  bool pending = false;  // a copy into this warpgroup's box is in flight
  if (nplan > 0 && (int)blockIdx.x < a.ntiles) {
    if (wt == 0) {
      issue(blockIdx.x, sched.plane[wg][0]);
      if (nplan > 1) prefetch(blockIdx.x, sched.plane[wg][1]);
    }
    pending = true;
  }
  unsigned parity = 0;
  bool failed = false;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    // ---------------- phase A: pull every plane of the tile -----------------
    for (int k = 0; k < nplan && !failed; ++k) {
      const int plane = sched.plane[wg][k];
      // every thread of the warpgroup takes the same decision
      if (wg_any(wg, !mbar_wait_bounded(bar, parity))) {
        failed = true;
        break;
      }
      parity ^= 1u;
      pending = false;
      const int i = plane < Q ? plane : plane - Q;
      const int act = st.active[i];
      const bool zact = D == 3 && (act & 4), yact = (act & 2) != 0, xact = (act & 1) != 0;
      if (wt == 0) {
        // warm L2 with the plane after next
        const int k2 = k + 2;
        if (k2 < nplan) prefetch(tile, sched.plane[wg][k2]);
        else if (tile + (int)gridDim.x < a.ntiles && k2 - nplan < nplan) prefetch(tile + gridDim.x, sched.plane[wg][k2 - nplan]);
      }
      const C* xsrc_c = nullptr;
      if (zact) {
        C W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = st.W[i][2][j];
        const int BYA = yact ? L::BY : L::TY;
        const int items = L::NQX * BYA * (L::TZ / L::ZCH);
        const int PLs = BYA * L::BXW;
        for (int item = wt; item < items; item += WGT) {
          const int q = item % L::NQX, r = item / L::NQX, y = r % BYA, zc = r / BYA;
          const int off = (zc * L::ZCH * BYA + y) * L::BXW + 4 * q;
          C v[L::ZCH + P][4];
#pragma unroll
          for (int kk = 0; kk < L::ZCH + P; ++kk) ld4(box + off + kk * PLs, v[kk]);
#pragma unroll
          for (int z = 0; z < L::ZCH; ++z) {
            C o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              C acc = W[0] * v[z][e];
#pragma unroll
              for (int kk = 1; kk <= P; ++kk) acc = fma(W[kk], v[z + kk][e], acc);
              o[e] = acc;
            }
            st4(bufA + off + z * PLs, o);
          }
        }
        wg_barrier(wg);
        xsrc_c = bufA;
      }
      if (yact) {
        C W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = st.W[i][1][j];
        constexpr int NYC = L::TY / L::YCH;
        constexpr int items = L::NQX * L::TZ * NYC;
        for (int item = wt; item < items; item += WGT) {
          const int q = item % L::NQX, r = item / L::NQX, yc = r % NYC, z = r / NYC;
          const int off = (z * L::BY + yc * L::YCH) * L::BXW + 4 * q;
          C v[L::YCH + P][4];
          if (zact) {
#pragma unroll
            for (int kk = 0; kk < L::YCH + P; ++kk) ld4(bufA + off + kk * L::BXW, v[kk]);
          } else {
#pragma unroll
            for (int kk = 0; kk < L::YCH + P; ++kk) ld4(box + off + kk * L::BXW, v[kk]);
          }
          C* o = bufB + (z * L::TY + yc * L::YCH) * L::BXW + 4 * q;
#pragma unroll
          for (int y = 0; y < L::YCH; ++y) {
            C w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              C acc = W[0] * v[y][e];
#pragma unroll
              for (int kk = 1; kk <= P; ++kk) acc = fma(W[kk], v[y + kk][e], acc);
              w4[e] = acc;
            }
            st4(o + y * L::BXW, w4);
          }
        }
        wg_barrier(wg);
        xsrc_c = bufB;
      }
      {
        C W[P + 1];
#pragma unroll
        for (int j = 0; j <= P; ++j) W[j] = st.W[i][0][j];
        const int xo = xact ? ((st.m0[i][0] % L::VEC) + L::VEC) % L::VEC : 0;
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
      wg_barrier(wg);  // box and buffers free
      if (k + 1 < nplan) {
        if (wt == 0) issue(tile, sched.plane[wg][k + 1]);
        pending = true;
      } else if (tile + (int)gridDim.x < a.ntiles) {
        if (wt == 0) issue(tile + gridDim.x, sched.plane[wg][0]);
        pending = true;
      }
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }

    // ---------------- phase B: collide every node of the tile ---------------
    const int tx = tile % a.nt[0], tr = tile / a.nt[0];
    const int ty = tr % a.nt[1], tz = tr / a.nt[1];
    const bool red = a.reduce != 0;
    const bool simple = a.quad_ok && pd.n[0] >= pd.gl[0] + pd.gr[0] && pd.n[1] >= pd.gl[1] + pd.gr[1] &&
                        pd.n[2] >= pd.gl[2] + pd.gr[2];
    C tsum[NRED];
#pragma unroll
    for (int c = 0; c < NRED; ++c) tsum[c] = C(0);
    for (int n = tid; n < L::TILE; n += NT) {
      const int lx = n % L::TX, ly = (n / L::TX) % L::TY, lz = n / (L::TX * L::TY);
      const int x = tx * L::TX + lx, y = ty * L::TY + ly, z = tz * L::TZ + lz;
      const bool inside = x < pd.n[0] && y < pd.n[1] && z < pd.n[2];
      C f[QM];
#pragma unroll
      for (int i = 0; i < QM; ++i) f[i] = i < Q ? scr[(size_t)i * L::TILE + n] : C(0);
      // moments (Sec. 3)
      C A = C(0), jx = C(0), jy = C(0), jz = C(0), Bp = C(0);
      double Bd = 0.0;
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
            Bd += (double)Bp;
            Bp = C(0);
          }
        }
      }
      const C rho = C(a.rho_ref) + A;
      const C ir = C(1) / rho;
      const C ics = C(a.inv_cs);
      const C uhx = jx * ir * ics, uhy = jy * ir * ics, uhz = jz * ir * ics;
      const C q = uhx * uhx + uhy * uhy + uhz * uhz;
      C itau = C(a.inv_tau), tt = C(0), gA = C(0), rth = C(0), theta = C(1), tau = C(a.tau);
      if (COMP) {
        Bd += (double)Bp;
        // sum of the pulled g (Sec. 3 temperature relation), FP32 groups into FP64
        double Gd = 0.0;
        C Gp = C(0);
#pragma unroll
        for (int i = 0; i < QM; ++i) {
          if (i >= Q) break;
          Gp += scr[(size_t)(Q + i) * L::TILE + n];
          if ((i & 7) == 7) {
            Gd += (double)Gp;
            Gp = C(0);
          }
        }
        Gd += (double)Gp;
        const double r = (double)rho;
        const double jj = (double)jx * jx + (double)jy * jy + (double)jz * jz;
        const double X = Bd + Gd - jj / r - a.two_cv * (double)A;
        tt = C(X) / (C(a.two_cv) * rho);
        theta = C(1) + tt;
        tau = C(a.mu_dt) / (rho * theta) + C(0.5);
        itau = C(1) / tau;
        gA = fma(rho, tt, A);
        rth = rho * theta;
      }
      // equilibrium (Appendix A), BGK (Sec. 3), stores with the periodic copies
      const long long off = pad_index(pd, x, y, z);
      const int dx = one_image(x, pd.n[0], pd.gl[0], pd.gr[0]);
      const int dy = one_image(y, pd.n[1], pd.gl[1], pd.gr[1]);
      const int dz = D == 3 ? one_image(z, pd.n[2], pd.gl[2], pd.gr[2]) : 0;
      const bool any_img = dx != 0 || dy != 0 || dz != 0;
      const long long sx = dx, sy = (long long)dy * pd.np[0], sz = (long long)dz * pd.np[0] * pd.np[1];
      C Pi[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
#pragma unroll
      for (int i = 0; i < QM; ++i) {
        if (i >= Q) break;
        const C s = fma(vt.xih[i][0], uhx, fma(vt.xih[i][1], uhy, D == 3 ? vt.xih[i][2] * uhz : C(0)));
        const C ph = phi_m1<C, COMP>(s, q, tt, vt.rD[i], vt.rpoly[i], a.N);
        const C feqd = vt.w[i] * fma(rho, ph, A);
        const C fneq = f[i] - feqd;
        const S o = Store<S>::st(fma(-fneq, itau, f[i]));
        S og{};
        if (COMP) {
          const C gv = scr[(size_t)(Q + i) * L::TILE + n];
          const C geqd = vt.w[i] * C(a.gfac) * fma(rth, ph, gA);
          og = Store<S>::st(fma(-(gv - geqd), itau, gv));
        }
        if (inside) {
          S* pf = dst + (long long)i * pd.plane;
          S* pg = dst + (long long)(Q + i) * pd.plane;
          pf[off] = o;
          if (COMP) pg[off] = og;
          if (any_img) {
            if (simple) {
#pragma unroll
              for (int c = 1; c < 8; ++c) {
                if (((c & 1) && !dx) || ((c & 2) && !dy) || ((c & 4) && !dz)) continue;
                const long long o2 = off + ((c & 1) ? sx : 0) + ((c & 2) ? sy : 0) + ((c & 4) ? sz : 0);
                pf[o2] = o;
                if (COMP) pg[o2] = og;
              }
            } else {
              store_all_images(pf, pd, x, y, z, o);
              if (COMP) store_all_images(pg, pd, x, y, z, og);
            }
          }
        }
        if (red) {
#pragma unroll
          for (int c = 0; c < 6; ++c) Pi[c] = fma(vt.xx[i][c], fneq, Pi[c]);
        }
      }
      if (red && inside) {
        const C u2 = q * C(a.cs2);
        tsum[0] += C(0.5) * u2;
        tsum[1] += C(0.5) * rho * u2;
        tsum[3] += A;
        tsum[4] += jx;
        tsum[5] += jy;
        tsum[6] += jz;
        const bool fin = isfinite(rho) && isfinite(uhx) && isfinite(uhy) && isfinite(uhz) && isfinite(theta);
        tsum[7] += fin ? C(0) : C(1);
        const C pres = rho * theta * C(a.cs2);
        const C den = C(2) * pres * tau * C(a.dt);
        const C ss = (Pi[0] * Pi[0] + Pi[1] * Pi[1] + Pi[2] * Pi[2] + C(2) * (Pi[3] * Pi[3] + Pi[4] * Pi[4] + Pi[5] * Pi[5])) /
                     (den * den);
        const C nu = C(a.cs2) * theta * C(a.dt) * (tau - C(0.5));
        tsum[2] += C(2) * nu * ss;
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
    if (wt == 0 && pending) mbar_wait_bounded(bar, parity);  // let the copy in flight land
    return;
  }
  if (a.reduce) {
    __syncthreads();
    if (tid < NRED) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += red_smem[w * NRED + tid];
      a.partials[(size_t)blockIdx.x * NRED + tid] = s;
    }
  }
}

template <int D, int P, typename S, bool COMP, int QM>
int launch_wg(const StepLaunch& Lc) {
  using C = typename Store<S>::C;
  using Lay = GLayout<D, P, S>;
  auto kern = sl_wg_kernel<D, P, S, COMP, QM>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES);
    if (e != cudaSuccess) return (int)e;
    attr_done = true;
  }
  const auto& vt = *static_cast<const VelTab<C>*>(Lc.veltab);
  const auto& st = *static_cast<const StencilTab<C, P + 1>*>(Lc.stentab);
  kern<<<Lc.grid, Lay::NT, Lay::BYTES, static_cast<cudaStream_t>(Lc.stream)>>>(Lc.a, vt, st, *Lc.maps, *Lc.sched);
  return (int)cudaGetLastError();
}

template <int D, int P, typename S, bool COMP, int QM>
int occupancy_wg(size_t* smem, int* nwg) {
  using Lay = GLayout<D, P, S>;
  auto kern = sl_wg_kernel<D, P, S, COMP, QM>;
  *smem = Lay::BYTES;
  *nwg = Lay::NWG;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::BYTES) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Lay::NT, Lay::BYTES) != cudaSuccess) return 0;
  return n;
}

}  // namespace wg
}  // namespace olb
