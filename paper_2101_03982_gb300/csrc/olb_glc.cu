// Pull of the cell-wise interpolation on Gauss-Lobatto-Chebyshev points
// (Sec. 3, the paper's own streaming), sm_103a.
//
// An axis of C cells carries C p nodes; node c p + k sits at the k-th GLC
// point of cell c.  The departure point x - xi_i dt of a node lies in a cell
// found from the node's residue k = j mod p alone (the shift is the same at
// every node), and is interpolated with that cell's Lagrange basis on its
// p + 1 GLC points.  The host builds, per velocity, axis and residue, the
// first support node (relative to the node) and the p + 1 weights
// (olb_glc_stencil); this kernel applies their tensor product to every node of
// every plane and writes the pulled values into the interior of a second
// padded state, which the fused step kernel then collides with an identity
// stencil.  Periodic wrap by index arithmetic (the ghost layers are not read).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "olb_internal.h"
#include "olb_step.cuh"

namespace olb {

namespace {

template <typename S, int D>
__global__ void __launch_bounds__(256) glc_pull_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                       const GlcArgs a) {
  using C = typename Store<S>::C;
  const C* __restrict__ W = static_cast<const C*>(a.W);
  const long long total = (long long)a.planes * a.nnodes;
  const int p = a.p, p1 = a.p + 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int plane = (int)(t / a.nnodes);
    const long long node = t - (long long)plane * a.nnodes;
    const int i = plane % a.Q;
    const int x = (int)(node % a.pad.n[0]);
    const long long r = node / a.pad.n[0];
    const int y = (int)(r % a.pad.n[1]), z = D == 3 ? (int)(r / a.pad.n[1]) : 0;
    const int c[3] = {x, y, z};
    // per axis: first support node (absolute, before the wrap), weights, count
    int f0[3], cnt[3];
    const C* w[3];
    for (int ax = 0; ax < 3; ++ax) {
      if (ax >= D || !((a.active[i] >> ax) & 1)) {
        f0[ax] = c[ax];
        cnt[ax] = 1;
        w[ax] = nullptr;  // identity
        continue;
      }
      const int k = c[ax] % p;
      const int idx = (i * 3 + ax) * GLC_PMAX + k;
      f0[ax] = c[ax] + a.first[idx];
      cnt[ax] = p1;
      w[ax] = W + (size_t)idx * (GLC_PMAX + 1);
    }
    const S* sp = src + (size_t)plane * a.pad.plane;
    C acc = C(0);
    for (int mz = 0; mz < cnt[2]; ++mz) {
      int zz = f0[2] + mz;
      zz = ((zz % a.pad.n[2]) + a.pad.n[2]) % a.pad.n[2];
      const C wz = w[2] ? w[2][mz] : C(1);
      C accy = C(0);
      for (int my = 0; my < cnt[1]; ++my) {
        int yy = f0[1] + my;
        yy = ((yy % a.pad.n[1]) + a.pad.n[1]) % a.pad.n[1];
        const C wy = w[1] ? w[1][my] : C(1);
        C accx = C(0);
        for (int mx = 0; mx < cnt[0]; ++mx) {
          int xx = f0[0] + mx;
          xx = ((xx % a.pad.n[0]) + a.pad.n[0]) % a.pad.n[0];
          const C wx = w[0] ? w[0][mx] : C(1);
          accx = fma(wx, Store<S>::ld(sp[pad_index(a.pad, xx, yy, zz)]), accx);
        }
        accy = fma(wy, accx, accy);
      }
      acc = fma(wz, accy, acc);
    }
    dst[(size_t)plane * a.pad.plane + pad_index(a.pad, x, y, z)] = Store<S>::st(acc);
  }
}

template <typename S>
int launch_typed(const GlcArgs& a, const void* src, void* dst, void* stream) {
  const long long total = (long long)a.planes * a.nnodes;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  if (blocks < 1) blocks = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (a.D == 2)
    glc_pull_kernel<S, 2><<<(int)blocks, 256, 0, s>>>(static_cast<const S*>(src), static_cast<S*>(dst), a);
  else
    glc_pull_kernel<S, 3><<<(int)blocks, 256, 0, s>>>(static_cast<const S*>(src), static_cast<S*>(dst), a);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_glc_pull(int storage, const GlcArgs& a, const void* src, void* dst, void* stream) {
  switch (storage) {
    case 0: return launch_typed<double>(a, src, dst, stream);
    case 1: return launch_typed<float>(a, src, dst, stream);
    default: return -1;  // the 16-bit storages are not built for this pull
  }
}

}  // namespace olb
