// Global sums of a population state without any device allocation.
//
// Some callers cannot allocate device memory when they want these sums: a
// coupling framework that owns every device byte through its own pool, or a
// loop that must never pay for cudaMalloc's implicit synchronisation.  This
// entry point takes the state and the output from the caller and keeps its
// per-block partial sums in a fixed array in device memory that is part of
// the library image: OLB_NOALLOC_MAX_BLOCKS blocks x 8 doubles (128 KiB), held
// by every GPU that loads the library until the process exits.
//
// The array is shared by all calls.  Each block overwrites its own slot before
// the final kernel reads it, so nothing has to start at zero, but calls whose
// kernels overlap on the GPU (different streams, no ordering between them)
// race on the array.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <string>

#include "olb.h"
#include "olb_internal.h"

namespace {

constexpr int NA_NT = 256;
constexpr int NA_MAX_BLOCKS = OLB_NOALLOC_MAX_BLOCKS;
constexpr int NA_RED = 8;

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS * NA_RED];

// Device address of g_noalloc_partials per device (the host-side name is only
// a stand-in), looked up with that device current, together with the identity
// of the context it belongs to: a device reset makes a new context (and loads
// the module again), so a changed identity means the address is looked up
// again.
std::mutex g_mu;
double* g_addr[64] = {};
unsigned long long g_ctx_id[64] = {};

// Identity of the calling thread's current context (0 when none or unknown).
unsigned long long current_ctx_id() {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  }
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

template <typename S>
__device__ __forceinline__ double val(S v);
template <>
__device__ __forceinline__ double val<double>(double v) { return v; }
template <>
__device__ __forceinline__ double val<float>(float v) { return (double)v; }
template <>
__device__ __forceinline__ double val<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <>
__device__ __forceinline__ double val<__half>(__half v) { return (double)__half2float(v); }

struct SumArgs {
  long long nodes, chunk;  // nodes, nodes per block
  int Q, D;
  double rho_ref;
  double xi[olb::MAXQ][3];
};

template <typename S>
__global__ void __launch_bounds__(NA_NT) noalloc_sums(const __grid_constant__ SumArgs a, const S* f, double* part) {
  double r[NA_RED] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long lo = blockIdx.x * a.chunk;
  const long long hi = lo + a.chunk < a.nodes ? lo + a.chunk : a.nodes;
  for (long long n = lo + threadIdx.x; n < hi; n += NA_NT) {
    double A = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < a.Q; ++i) {
      const double v = val(f[(long long)i * a.nodes + n]);
      A += v;
      jx += a.xi[i][0] * v;
      jy += a.xi[i][1] * v;
      jz += a.xi[i][2] * v;
    }
    const double rho = a.rho_ref + A;
    const double u2 = (jx * jx + jy * jy + jz * jz) / (rho * rho);
    r[0] += 0.5 * u2;
    r[1] += 0.5 * rho * u2;
    r[3] += A;
    r[4] += jx;
    r[5] += jy;
    r[6] += jz;
    r[7] += (isfinite(rho) && isfinite(u2)) ? 0.0 : 1.0;
  }
  __shared__ double sm[NA_NT / 32][NA_RED];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < NA_RED; ++q) {
    double v = r[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NA_RED) {
    double s = 0.0;
    for (int w = 0; w < NA_NT / 32; ++w) s += sm[w][threadIdx.x];
    part[(size_t)blockIdx.x * NA_RED + threadIdx.x] = s;  // every slot in use is written
  }
}

__global__ void __launch_bounds__(256) noalloc_final(const double* part, int blocks, long long nodes, double rho_ref,
                                                     double* out) {
  __shared__ double sm[256];
  for (int q = 0; q < NA_RED; ++q) {
    double s = 0.0;
    for (int k = threadIdx.x; k < blocks; k += 256) s += part[(size_t)k * NA_RED + q];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double v = sm[0];
      if (q == 0 || q == 1) v /= (double)nodes;
      if (q == 2) v = NAN;
      if (q == 3) v += rho_ref * (double)nodes;
      out[q] = v;
    }
    __syncthreads();
  }
}

int fail(int code, const std::string& m) {
  olb::set_last_error(m);
  return code;
}

}  // namespace

extern "C" int olb_state_sums_noalloc(int velocity_set, const olb_grid* grid, int storage, double cs_scale,
                                      double rho0, const void* populations, double* out, void* stream) {
  if (!grid || !populations || !out) return fail(OLB_EINVAL, "null grid, state or output");
  olb::VelocitySet vs;
  if (olb::velocity_set(velocity_set, &vs) != 0) return fail(OLB_EINVAL, "unknown velocity set");
  if (grid->dim != vs.D) return fail(OLB_EINVAL, "velocity set dimension differs from the grid's");
  if (grid->n[0] < 1 || grid->n[1] < 1 || grid->n[2] < 1) return fail(OLB_EINVAL, "grid sizes must be >= 1");
  if (!(cs_scale > 0.0)) return fail(OLB_EINVAL, "cs_scale must be positive");
  const long long nodes = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  const long long chunk = OLB_NOALLOC_NODES_PER_BLOCK;
  const long long blocks = (nodes + chunk - 1) / chunk;
  if (blocks > NA_MAX_BLOCKS)
    return fail(OLB_EBOUNDS, "state larger than the fixed scratch allows (at most " +
                                 std::to_string((long long)NA_MAX_BLOCKS * chunk) + " nodes)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(OLB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(OLB_EBOUNDS, "device index above 63");
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
      // first call on this device, or its context changed: (re)load the address
      e = cudaGetSymbolAddress((void**)&g_addr[dev], g_noalloc_partials);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return fail(OLB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_ctx_id[dev] = current_ctx_id();  // the lookup made the primary context current
    }
    part = g_addr[dev];
  }

  SumArgs a{};
  a.nodes = nodes;
  a.chunk = chunk;
  a.Q = vs.Q;
  a.D = vs.D;
  a.rho_ref = storage == OLB_FP64 ? 0.0 : rho0;
  for (int i = 0; i < vs.Q; ++i)
    for (int c = 0; c < 3; ++c) a.xi[i][c] = vs.xi[i][c] * cs_scale;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)blocks;
  switch (storage) {
    case OLB_FP64: noalloc_sums<double><<<nb, NA_NT, 0, s>>>(a, static_cast<const double*>(populations), part); break;
    case OLB_FP32_SHIFTED: noalloc_sums<float><<<nb, NA_NT, 0, s>>>(a, static_cast<const float*>(populations), part); break;
    case OLB_BF16_SHIFTED:
      noalloc_sums<__nv_bfloat16><<<nb, NA_NT, 0, s>>>(a, static_cast<const __nv_bfloat16*>(populations), part);
      break;
    case OLB_FP16_SHIFTED: noalloc_sums<__half><<<nb, NA_NT, 0, s>>>(a, static_cast<const __half*>(populations), part); break;
    default: return fail(OLB_EINVAL, "unknown storage");
  }
  noalloc_final<<<1, 256, 0, s>>>(part, nb, nodes, a.rho_ref, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OLB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return OLB_OK;
}
