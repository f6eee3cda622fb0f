// Pull of the cell-wise interpolation on Gauss-Lobatto-Chebyshev points
// (Sec. 3, the paper's own streaming), sm_103a.
//
// An axis of C cells carries C p nodes; node c p + k sits at the k-th GLC
// point of cell c.  The departure point x - xi_i dt of a node lies in a cell
// found from the node's residue k = j mod p alone (the shift is the same at
// every node), and is interpolated with that cell's Lagrange basis on its
// p + 1 GLC points.  The host builds, per velocity, axis and residue, the
// first support node (relative to the node) and the p + 1 weights
// (olb_glc_stencil), and per velocity and axis the reach of those stencils.
//
// One CTA pulls one tile of one population plane.  It loads the tile and its
// reach into shared memory (rows along x, periodic wrap by index arithmetic:
// the ghost layers are not read), then applies the tensor product as
// separable passes, x, then y, then z, each reading the per-residue stencil
// of its output coordinate; an axis along which the velocity does not move is
// skipped.  The last pass writes the pulled values, coalesced along x, into
// the interior of a second padded state, which the fused step kernel then
// collides with an identity stencil.  The order of the passes is the nesting
// of the tensor-product sum sum_z w_z sum_y w_y sum_x w_x f.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "olb_internal.h"
#include "olb_step.cuh"

namespace olb {

namespace {

constexpr int GT = 512;  // threads per CTA (16 warps)
constexpr int GTX = 32;  // tile width along x: one output per lane

// 3D tiles: the reach of the stencils (up to p nodes on each side) is staged
// with the tile, so tall tiles keep the staged box a small multiple of it;
// 2D tiles are GTX x 32
template <typename C>
struct GlcTile {
  static constexpr int TY = 16;
  static constexpr int TZ = sizeof(C) == 8 ? 8 : 16;
};

// one element copied global -> shared without passing through registers
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(unsigned dst, const void* src) {
  if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}

// 16 bytes copied global -> shared (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ int wrap(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

template <typename S, int D, int P>
__global__ void __launch_bounds__(GT) glc_pull_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                     const GlcArgs a) {
  using C = typename Store<S>::C;
  constexpr int TY = D == 3 ? GlcTile<C>::TY : 32;
  constexpr int TZ = D == 3 ? GlcTile<C>::TZ : 1;
  constexpr int WS = GLC_PMAX + 1, P1 = P + 1, NW = GT / 32;
  extern __shared__ unsigned char smem_raw[];
  constexpr bool WIDE = std::is_same<S, C>::value;  // the storage is the arithmetic type
  C* wsm = reinterpret_cast<C*>(smem_raw);  // [3][GLC_PMAX][WS] weights of this velocity
  C* b0 = wsm + 3 * GLC_PMAX * WS;
  C* b1 = b0 + a.box_elems;  // a.b1_elems: the x pass's output
  // 16-bit storage: the box is staged as stored and converted into b0
  S* bs = WIDE ? reinterpret_cast<S*>(b0) : reinterpret_cast<S*>(b1 + a.b1_elems);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = (int)(blockIdx.x % (unsigned)a.ntiles);
  const int plane = (int)(blockIdx.x / (unsigned)a.ntiles);
  const int i = plane % a.Q;
  const int tx = tile % a.nt[0], tr = tile / a.nt[0];
  const int x0 = tx * GTX, y0 = (tr % a.nt[1]) * TY, z0 = (tr / a.nt[1]) * TZ;
  const int act = a.active[i];
  const int lox = a.lo[i * 3 + 0], loy = a.lo[i * 3 + 1], loz = D == 3 ? a.lo[i * 3 + 2] : 0;
  const int ex = GTX + lox + a.hi[i * 3 + 0];
  const int ey = TY + loy + a.hi[i * 3 + 1];
  const int ez = D == 3 ? TZ + loz + a.hi[i * 3 + 2] : 1;
  const int n0 = a.pad.n[0], n1 = a.pad.n[1], n2 = a.pad.n[2];

  const C* __restrict__ W = static_cast<const C*>(a.W);
  for (int t = threadIdx.x; t < 3 * P * P1; t += GT) {
    const int ax = t / (P * P1), r = t - ax * (P * P1), k = r / P1, m = r - k * P1;
    wsm[(ax * GLC_PMAX + k) * WS + m] = W[((size_t)(i * 3 + ax) * GLC_PMAX + k) * WS + m];
  }

  // the tile and its reach, rows along x: asynchronous copies (no register
  // round trip, so every copy of the CTA is in flight at once), 16 bytes at a
  // time where the grid allows it, else one element at a time; the row index
  // (yb, zb) advances without a division
  const S* __restrict__ sp = src + (size_t)plane * a.pad.plane;
  const unsigned b0s = smem_u32(bs);
  if (a.vec16) {
    // 16-byte copies: the box starts on a 16-byte column (the host rounds the
    // x reach), n0 is a multiple of VG, so a copy never straddles the wrap;
    // one warp takes 32 / cpr rows per iteration
    constexpr int VG = 16 / (int)sizeof(S);
    const int cpr = ex / VG, rpi = 32 / cpr;
    const int lr = lane / cpr, lc = lane - lr * cpr;
    if (lr < rpi) {
      const int gx = wrap(x0 - lox + lc * VG, n0);
      int row = warp * rpi + lr;
      int yb = row % ey, zb = row / ey;
      for (; row < ey * ez; row += NW * rpi) {
        cp_async16(b0s + (unsigned)((row * ex + lc * VG) * (int)sizeof(S)),
                   sp + pad_index(a.pad, gx, wrap(y0 - loy + yb, n1), D == 3 ? wrap(z0 - loz + zb, n2) : 0));
        yb += NW * rpi;
        while (yb >= ey) {
          yb -= ey;
          ++zb;
        }
      }
    }
  } else {
    const bool xin = x0 - lox >= 0 && x0 - lox + ex <= n0;  // no wrap along x
    int yb = warp, zb = 0;
    while (yb >= ey) {
      yb -= ey;
      ++zb;
    }
    for (int r = warp; r < ey * ez; r += NW) {
      const S* __restrict__ row = sp + pad_index(a.pad, 0, wrap(y0 - loy + yb, n1), D == 3 ? wrap(z0 - loz + zb, n2) : 0);
      const unsigned drow = b0s + (unsigned)(r * ex * (int)sizeof(S));
      if constexpr (sizeof(S) >= 4) {
        if (xin) {
          const S* __restrict__ rx = row + (x0 - lox);
          for (int xb = lane; xb < ex; xb += 32)
            cp_async_elem<sizeof(S)>(drow + (unsigned)(xb * (int)sizeof(S)), rx + xb);
        } else {
          for (int xb = lane; xb < ex; xb += 32)
            cp_async_elem<sizeof(S)>(drow + (unsigned)(xb * (int)sizeof(S)), row + wrap(x0 - lox + xb, n0));
        }
      } else {  // 2-byte elements: no asynchronous copy of that size, plain loads
        (void)drow;
        for (int xb = lane; xb < ex; xb += 32) bs[r * ex + xb] = row[wrap(x0 - lox + xb, n0)];
      }
      yb += NW;
      while (yb >= ey) {
        yb -= ey;
        ++zb;
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  if constexpr (!WIDE) {
    for (int e = threadIdx.x; e < ex * ey * ez; e += GT) b0[e] = Store<S>::ld(bs[e]);
    __syncthreads();
  }

  C* cur = b0;
  C* nxt = b1;
  int cy = ey;
  if (act & 1) {  // x pass: (ex, ey, ez) -> (GTX, ey, ez); the residue depends on the lane only
    const int k = (x0 + lane) % P;
    const C* s0 = cur + a.first[(i * 3 + 0) * GLC_PMAX + k] + lox + lane;
    C w[P1];
#pragma unroll
    for (int m = 0; m < P1; ++m) w[m] = wsm[(0 * GLC_PMAX + k) * WS + m];
#pragma unroll 4
    for (int r = warp; r < ey * ez; r += NW) {
      const C* s = s0 + r * ex;
      C acc = w[0] * s[0];
#pragma unroll
      for (int m = 1; m < P1; ++m) acc = fma(w[m], s[m], acc);
      nxt[r * GTX + lane] = acc;
    }
    C* t = cur;
    cur = nxt;
    nxt = t;
    __syncthreads();
  }
  // The y and z passes give each warp fixed output rows along the pass's axis
  // (NW is a multiple of TY and TZ's divisors below), so a warp's residue,
  // stencil weights and first support row are loaded once.
  static_assert(TY % NW == 0 || NW % TY == 0, "warps and tile rows");
  static_assert(NW % TZ == 0, "warps and tile depth");
  if (act & 2) {  // y pass: (GTX, ey, ez) -> (GTX, TY, ez)
    for (int oy = warp % TY; oy < TY; oy += NW) {
      const int k = (y0 + oy) % P;
      C w[P1];
#pragma unroll
      for (int m = 0; m < P1; ++m) w[m] = wsm[(1 * GLC_PMAX + k) * WS + m];
      const C* s = cur + (a.first[(i * 3 + 1) * GLC_PMAX + k] + loy + oy) * GTX + lane;
      C* o = nxt + oy * GTX + lane;
#pragma unroll 4
      for (int oz = warp / TY; oz < ez; oz += (NW > TY ? NW / TY : 1)) {
        const C* so = s + oz * cy * GTX;
        C acc = w[0] * so[0];
#pragma unroll
        for (int m = 1; m < P1; ++m) acc = fma(w[m], so[m * GTX], acc);
        o[oz * TY * GTX] = acc;
      }
    }
    C* t = cur;
    cur = nxt;
    nxt = t;
    cy = TY;
    __syncthreads();
  }
  // z pass (or the plain copy of the passes' result) into the padded interior
  S* __restrict__ dp = dst + (size_t)plane * a.pad.plane;
  const int gx = x0 + lane;
  const bool zpass = D == 3 && (act & 4);
  {
    const int oz = warp % TZ, gz = z0 + oz;
    const int k = gz % P;
    C w[P1];
#pragma unroll
    for (int m = 0; m < P1; ++m) w[m] = zpass ? wsm[(2 * GLC_PMAX + k) * WS + m] : C(0);
    const int zrow = zpass ? a.first[(i * 3 + 2) * GLC_PMAX + k] + loz + oz : oz;
    const C* s = cur + zrow * cy * GTX + lane;
    const bool on = gx < n0 && gz < n2;
    S* d = dp + pad_index(a.pad, gx, 0, gz);
#pragma unroll 4
    for (int oy = warp / TZ; oy < TY; oy += NW / TZ) {
      const C* so = s + oy * GTX;
      C v;
      if (zpass) {
        C acc = w[0] * so[0];
#pragma unroll
        for (int m = 1; m < P1; ++m) acc = fma(w[m], so[m * cy * GTX], acc);
        v = acc;
      } else {
        v = so[0];
      }
      if (on && y0 + oy < n1) d[(long long)(y0 + oy) * a.pad.np[0]] = Store<S>::st(v);
    }
  }
}

template <typename S>
int launch_typed(const GlcArgs& a, const void* src, void* dst, void* stream) {
  using C = typename Store<S>::C;
  const size_t bytes = glc_smem_bytes(a, sizeof(C), sizeof(S));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)a.planes * (unsigned)a.ntiles;
  void (*kern)(const S*, S*, const GlcArgs) = nullptr;
  switch (a.p) {
#define OLB_GLC_CASE(PP) \
  case PP: kern = a.D == 2 ? glc_pull_kernel<S, 2, PP> : glc_pull_kernel<S, 3, PP>; break;
    OLB_GLC_CASE(1)
    OLB_GLC_CASE(2)
    OLB_GLC_CASE(3)
    OLB_GLC_CASE(4)
    OLB_GLC_CASE(5)
    OLB_GLC_CASE(6)
#undef OLB_GLC_CASE
    default: return -1;  // orders above the step kernels' are not built
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return (int)e;
  kern<<<blocks, GT, bytes, s>>>(static_cast<const S*>(src), static_cast<S*>(dst), a);
  return (int)cudaGetLastError();
}

}  // namespace

void glc_tile_shape(int D, int elem, int* tx, int* ty, int* tz) {
  *tx = GTX;
  const bool f64 = elem == 8;
  *ty = D == 3 ? (f64 ? GlcTile<double>::TY : GlcTile<float>::TY) : 32;
  *tz = D == 3 ? (f64 ? GlcTile<double>::TZ : GlcTile<float>::TZ) : 1;
}

size_t glc_smem_bytes(const GlcArgs& a, int elem, int storage_elem) {
  size_t b = ((size_t)3 * GLC_PMAX * (GLC_PMAX + 1) + (size_t)a.box_elems + (size_t)a.b1_elems) * (size_t)elem;
  if (storage_elem != elem) b += ((size_t)a.box_elems * storage_elem + 15) / 16 * 16;  // the box as stored
  return b;
}

int launch_glc_pull(int storage, const GlcArgs& a, const void* src, void* dst, void* stream) {
  switch (storage) {
    case 0: return launch_typed<double>(a, src, dst, stream);
    case 1: return launch_typed<float>(a, src, dst, stream);
    case 2: return launch_typed<__nv_bfloat16>(a, src, dst, stream);
    case 3: return launch_typed<__half>(a, src, dst, stream);
    default: return -1;
  }
}

}  // namespace olb
