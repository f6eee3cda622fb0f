// C ABI of the library (include/olb.h): handle lifetime, argument checks,
// stencil and table set-up on the host, and dispatch of the kernels.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "olb.h"
#include "olb_internal.h"

using namespace olb;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(OLB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

void olb::set_last_error(const std::string& msg) { g_last_error = msg; }

struct olb_ctx {
  olb_grid grid{};
  int vs_id = 0, N = 2, p = 3, storage = 0, comp = 0, allow_inexact = 0;
  double tau = 1.0, dt = 0.0, gamma = 1.4, mu = 0.0, mu_exp = 0.0, prandtl = 1.0, rho0 = 1.0, cs = 1.0,
         cs_scale = 1.0;
  VelocitySet set{};  // scaled abscissae
  int Q = 0, planes = 0, D = 0, elem = 8;
  long long nnodes = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  void* scratch = nullptr;
  double* partials = nullptr;
  double* red_dev = nullptr;
  int* err_dev = nullptr;
  int step_grid = 0, partial_slots = 0;
  int log_every = 1;
  int force_generic = 0;
  long long step_count = 0;
  int partials_valid = 0;  // 1: the partials hold the sums of the current state's step
  int state_bad = 0;       // 1: a step gave up waiting for a staging copy; no valid state since
  int glc = 0;             // 1: cell-wise Gauss-Lobatto-Chebyshev interpolation (olb_set_interpolation)
  GlcArgs glc_args{};
  void* glc_w = nullptr;                   // device weights of the GLC pull
  std::vector<unsigned char> st_glc_id;    // identity stencil: the collision of pulled values
  int xbc = 0;             // 1: non-periodic x (inflow / zero-gradient outflow ghost columns)
  XInflow inflow{};
  void* xbc_vals = nullptr;  // inflow value per plane, storage form
  Padded pad{};
  TmaMaps maps{};
  WgSchedule sched{};
  cudaStream_t stream = nullptr;
  int device = 0;
  StepInfo info{};
  StepArgs args{};
  std::vector<unsigned char> veltab, stentab;
  AuxArgs aux{};
  std::vector<int> m0;        // [Q][3], oracle convention on every axis
  std::vector<double> W;      // [Q][3][p+1]
  // adjoint: tape of forward states (padded, like buf) and the adjoint buffers
  std::vector<void*> tape;
  // slot s: the moments (A = sum of the stored pulled values, j) of recorded
  // step s + 1, per node in the two-phase kernel's tile order
  // [tile][4][tile nodes], arithmetic type
  int tape_len = 0;                // slots holding a recorded state
  void* adj[2] = {nullptr, nullptr};
  TmaMaps adj_maps{};              // m[k] of adj[k]
  StepInfo ainfo{};                // geometry of the adjoint kernel (the two-phase kernel's)
  int adj_grid = 0, adj_nt[3] = {0, 0, 0}, adj_ntiles = 0;
  void* adj_scratch = nullptr;
  std::vector<unsigned char> st_refl, st_id;  // reflected and identity stencils
  WgSchedule sched_adj{};          // the adjoint planes Q..2Q-1 of every launch
  int adj_ready = 0;
  // enstrophy diagnostic: velocity field and per-block partials
  double* ens_u = nullptr;
  double* ens_part = nullptr;
};

namespace {

int storage_bytes(int storage) {
  switch (storage) {
    case OLB_FP64: return 8;
    case OLB_FP32_SHIFTED: return 4;
    case OLB_BF16_SHIFTED:
    case OLB_FP16_SHIFTED: return 2;
    default: return 0;
  }
}

int step_info(int D, int P, int storage, int comp, int Q, int N, int force_generic, StepInfo* out) {
  const bool d2 = D == 2;
  switch (storage) {
    case OLB_FP64:
      return d2 ? step_info_f64_2d(P, comp, Q, N, force_generic, out) : step_info_f64_3d(P, comp, Q, N, force_generic, out);
    case OLB_FP32_SHIFTED:
      return d2 ? step_info_f32_2d(P, comp, Q, N, force_generic, out) : step_info_f32_3d(P, comp, Q, N, force_generic, out);
    case OLB_BF16_SHIFTED:
      return d2 ? step_info_bf16_2d(P, comp, Q, N, force_generic, out)
                : step_info_bf16_3d(P, comp, Q, N, force_generic, out);
    case OLB_FP16_SHIFTED:
      return d2 ? step_info_f16_2d(P, comp, Q, N, force_generic, out) : step_info_f16_3d(P, comp, Q, N, force_generic, out);
    default: return -1;
  }
}

int launch_step(int storage, int D, const StepLaunch& L) {
  const bool d2 = D == 2;
  switch (storage) {
    case OLB_FP64: return d2 ? launch_step_f64_2d(L) : launch_step_f64_3d(L);
    case OLB_FP32_SHIFTED: return d2 ? launch_step_f32_2d(L) : launch_step_f32_3d(L);
    case OLB_BF16_SHIFTED: return d2 ? launch_step_bf16_2d(L) : launch_step_bf16_3d(L);
    default: return d2 ? launch_step_f16_2d(L) : launch_step_f16_3d(L);
  }
}

// Lagrange stencil of degree p around offset delta (grid units): first point
// m0 and weights W[j] = prod_{k != j} (delta - m_k) / (m_j - m_k).
void lagrange_stencil(double delta, int p, int* m0, double* W) {
  int first = (p % 2 == 1) ? (int)std::floor(delta) - (p - 1) / 2 : (int)std::floor(delta + 0.5) - p / 2;
  *m0 = first;
  for (int j = 0; j <= p; ++j) {
    double prod = 1.0;
    for (int k = 0; k <= p; ++k)
      if (k != j) prod *= (delta - (first + k)) / (double)((first + j) - (first + k));
    W[j] = prod;
  }
}

template <typename C>
void fill_veltab(olb_ctx* h) {
  h->veltab.assign(sizeof(VelTab<C>), 0);
  auto* t = reinterpret_cast<VelTab<C>*>(h->veltab.data());
  const int D = h->D;
  for (int i = 0; i < h->Q; ++i) {
    double xh[3], x2 = 0.0, r = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double x = h->set.xi[i][a];
      xh[a] = x / h->cs;
      t->xi[i][a] = (C)x;
      t->xih[i][a] = (C)xh[a];
      x2 += x * x;
      r += xh[a] * xh[a];
    }
    t->w[i] = (C)h->set.w[i];
    t->wt[i] = (C)(h->set.w[i] / h->tau);
    t->xi2[i] = (C)x2;
    t->rD[i] = (C)(r - D);
    t->rpoly[i] = (C)(r * r - 2.0 * (D + 2) * r + D * (D + 2.0));
    const double* x = h->set.xi[i];
    t->xx[i][0] = (C)(x[0] * x[0]);
    t->xx[i][1] = (C)(x[1] * x[1]);
    t->xx[i][2] = (C)(x[2] * x[2]);
    t->xx[i][3] = (C)(x[0] * x[1]);
    t->xx[i][4] = (C)(x[0] * x[2]);
    t->xx[i][5] = (C)(x[1] * x[2]);
  }
}

// FP32 copy of the Lagrange weights of one stencil.  Rounded one by one to
// nearest, FP32 weights sum to 1 + O(1e-8): the pull would then scale every
// population, and the mass and momentum it carries, by that factor at every
// step (over 500 steps the kinetic energy of the 3D Taylor-Green vortex in
// FP32 drifted by up to 1e-4 from the FP64 run).  Here each weight is rounded
// up or down (staying within one ulp of its FP64 value), choosing among the
// 2^(p+1) combinations the one whose sum is closest to 1, then whose first and
// second moments about the departure point are closest to the exact ones; the
// sums are exact in FP64.
void nearest_sum_weights_f32(const double* W, const int* m, double delta, int n, float* out) {
  float lo[MAXP + 1], hi[MAXP + 1];
  double m1 = 0.0, m2 = 0.0;
  for (int j = 0; j < n; ++j) {
    const float f = (float)W[j];
    lo[j] = (double)f <= W[j] ? f : std::nextafter(f, -INFINITY);
    hi[j] = (double)f >= W[j] ? f : std::nextafter(f, INFINITY);
    m1 += W[j] * (m[j] - delta);
    m2 += W[j] * (m[j] - delta) * (m[j] - delta);
  }
  double best[3] = {INFINITY, INFINITY, INFINITY};
  for (int mask = 0; mask < (1 << n); ++mask) {
    double s = 0.0, e1 = 0.0, e2 = 0.0;
    for (int j = 0; j < n; ++j) {
      const double v = (mask >> j) & 1 ? hi[j] : lo[j];
      s += v;
      e1 += v * (m[j] - delta);
      e2 += v * (m[j] - delta) * (m[j] - delta);
    }
    const double c[3] = {std::fabs(s - 1.0), std::fabs(e1 - m1), std::fabs(e2 - m2)};
    if (c[0] < best[0] || (c[0] == best[0] && (c[1] < best[1] || (c[1] == best[1] && c[2] < best[2])))) {
      for (int k = 0; k < 3; ++k) best[k] = c[k];
      for (int j = 0; j < n; ++j) out[j] = (mask >> j) & 1 ? hi[j] : lo[j];
    }
  }
}

template <typename C, int P1>
void fill_stentab_p(olb_ctx* h) {
  h->stentab.assign(sizeof(StencilTab<C, P1>), 0);
  auto* t = reinterpret_cast<StencilTab<C, P1>*>(h->stentab.data());
  const int p = h->p;
  for (int i = 0; i < h->Q; ++i) {
    int act = 0;
    for (int a = 0; a < h->D; ++a) {
      if (h->set.xi[i][a] != 0.0) act |= 1 << a;
      t->m0[i][a] = h->m0[i * 3 + a];
      const double* Wd = &h->W[(i * 3 + a) * (p + 1)];
      if constexpr (std::is_same<C, float>::value) {
        int mm[MAXP + 1];
        for (int j = 0; j <= p; ++j) mm[j] = h->m0[i * 3 + a] + j;
        const double delta = -h->set.xi[i][a] * h->dt / h->grid.dx;
        nearest_sum_weights_f32(Wd, mm, delta, p + 1, t->W[i][a]);
      } else {
        for (int j = 0; j <= p; ++j) t->W[i][a][j] = (C)Wd[j];
      }
    }
    t->active[i] = act;
  }
}

// Inverse of the D x D block of M (the rest zero).
void inverse_block(const double M[3][3], int D, double inv[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) inv[a][b] = 0.0;
  if (D == 2) {
    const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    inv[0][0] = M[1][1] / det;
    inv[0][1] = -M[0][1] / det;
    inv[1][0] = -M[1][0] / det;
    inv[1][1] = M[0][0] / det;
    return;
  }
  const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                     M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                     M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      // adjugate: the cofactor of (b, a), signs from the cyclic index order
      const int a1 = (b + 1) % 3, a2 = (b + 2) % 3, b1 = (a + 1) % 3, b2 = (a + 2) % 3;
      inv[a][b] = (M[a1][b1] * M[a2][b2] - M[a1][b2] * M[a2][b1]) / det;
    }
}

// Correction g of the FP32 equilibrium velocity u^ = (I + diag(g)) u^0,
// u^0 = j fl(1/c_s) / rho (see uhat_of in olb_step.cuh).  The collision keeps the momentum j when the equilibrium's
// momentum, computed with the FP32 tables it is built from, is what the BGK
// form needs:
//  * isothermal, (1 - fl(1/tau)) f + fl(w/tau) e:  rho M_wt u^ = fl(1/tau) j
//    with M_wt = sum_i fl(w_i/tau) xi_i (xi_i/c_s), so
//    I + diag(g) = fl(1/tau) M_wt^-1 / fl(1/c_s);
//  * compressible, f - (f - w e)/tau:  rho M_w u^ = j with
//    M_w = sum_i fl(w_i) xi_i (xi_i/c_s), so I + diag(g) = M_w^-1 / fl(1/c_s).
// The products and sums of the FP32 table values are exact in FP64.
void fill_uhat_fix(olb_ctx* h) {
  const auto* t = reinterpret_cast<const VelTab<float>*>(h->veltab.data());
  const int D = h->D;
  double Mw[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Mt[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < h->Q; ++i)
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        const double xx = (double)t->xi[i][a] * (double)t->xih[i][b];
        Mw[a][b] += (double)t->w[i] * xx;
        Mt[a][b] += (double)t->wt[i] * xx;
      }
  double iw[3][3], it[3][3];
  inverse_block(Mw, D, iw);
  inverse_block(Mt, D, it);
  const double ics = (double)(float)(1.0 / h->cs);
  const double itau = (double)(float)(1.0 / h->tau);
  // the tables are symmetric under the reflection of every axis, so M is
  // diagonal (its off-diagonal sums cancel exactly): only the diagonal is kept
  for (int a = 0; a < 3; ++a) {
    h->args.f_g[a] = (!h->comp && a < D) ? (float)(itau * it[a][a] / ics - 1.0) : 0.f;
    h->args.f_gc[a] = a < D ? (float)(iw[a][a] / ics - 1.0) : 0.f;
  }
}

template <typename C>
void fill_stentab(olb_ctx* h) {
  switch (h->p) {
    case 1: fill_stentab_p<C, 2>(h); break;
    case 2: fill_stentab_p<C, 3>(h); break;
    case 3: fill_stentab_p<C, 4>(h); break;
    case 4: fill_stentab_p<C, 5>(h); break;
    case 5: fill_stentab_p<C, 6>(h); break;
    case 6: fill_stentab_p<C, 7>(h); break;
  }
}

void release(olb_ctx* h) {
  if (!h) return;
  for (int k = 0; k < 2; ++k)
    if (h->buf[k]) cudaFree(h->buf[k]);
  if (h->scratch) cudaFree(h->scratch);
  if (h->partials) cudaFree(h->partials);
  if (h->red_dev) cudaFree(h->red_dev);
  if (h->err_dev) cudaFree(h->err_dev);
  for (void* t : h->tape)
    if (t) cudaFree(t);
  for (int k = 0; k < 2; ++k)
    if (h->adj[k]) cudaFree(h->adj[k]);
  if (h->adj_scratch) cudaFree(h->adj_scratch);
  if (h->ens_u) cudaFree(h->ens_u);
  if (h->xbc_vals) cudaFree(h->xbc_vals);
  if (h->glc_w) cudaFree(h->glc_w);
  if (h->ens_part) cudaFree(h->ens_part);
  delete h;
}

// Ghost widths from the stencil reach: on each axis the pull reads offsets
// m0 .. m0 + p of every active velocity; x is widened to keep rows and staged
// boxes on 16-byte (and 4-node) boundaries.
void layout_padding(olb_ctx* h) {
  Padded& P = h->pad;
  const int align = std::max(16 / h->elem, 4);
  for (int a = 0; a < 3; ++a) {
    int lo = 0, hi = 0;
    if (a < h->D)
      for (int i = 0; i < h->Q; ++i) {
        if (h->set.xi[i][a] == 0.0) continue;
        lo = std::max(lo, -h->m0[i * 3 + a]);
        hi = std::max(hi, h->m0[i * 3 + a] + h->p);
      }
    P.n[a] = h->grid.n[a];
    if (a == 0) {
      P.gl[0] = (lo + align - 1) / align * align;
      const int np = (P.gl[0] + P.n[0] + hi + align - 1) / align * align;
      P.gr[0] = np - P.gl[0] - P.n[0];
    } else {
      P.gl[a] = lo;
      P.gr[a] = hi;
    }
    P.np[a] = P.gl[a] + P.n[a] + P.gr[a];
  }
  P.plane = (long long)P.np[0] * P.np[1] * P.np[2];
}

}  // namespace

// Planes of each warpgroup of the two-phase kernel: longest processing time
// first, with a plane's cost from the passes its stencil needs.
static void lpt_schedule(int nwg, std::vector<std::pair<double, int>> cost, WgSchedule* out) {
  WgSchedule& S = *out;
  std::memset(&S, 0, sizeof(S));
  if (nwg < 1) nwg = 1;
  std::stable_sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  double load[4] = {0, 0, 0, 0};
  std::vector<int> lists[4];
  for (const auto& cp : cost) {
    int best = 0;
    for (int w = 1; w < nwg; ++w)
      if (load[w] < load[best]) best = w;
    load[best] += cp.first;
    lists[best].push_back(cp.second);
  }
  for (int w = 0; w < nwg; ++w) {
    std::sort(lists[w].begin(), lists[w].end());
    S.n[w] = (int)lists[w].size();
    for (size_t k = 0; k < lists[w].size(); ++k) S.plane[w][k] = (unsigned char)lists[w][k];
  }
}

// Cost of pulling one plane of velocity i, relative to a plain copy: the
// fixed cost of staging a plane dominates; the x, y and z passes add the
// fractions measured on GB300 (clock64 per plane and warpgroup, D3Q27).
static double plane_cost(const olb_ctx* h, int i) {
  double c = 1.0;
  if (h->set.xi[i][0] != 0.0) c += 0.12;
  if (h->set.xi[i][1] != 0.0) c += 0.42;
  if (h->D == 3 && h->set.xi[i][2] != 0.0) c += 0.55;
  return c;
}

static void build_schedule(olb_ctx* h) {
  std::vector<std::pair<double, int>> cost;
  for (int p = 0; p < h->planes; ++p) cost.push_back({plane_cost(h, p % h->Q), p});
  lpt_schedule(h->info.wg, cost, &h->sched);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4D tiled descriptors (x, y, z, plane) of one padded buffer of `nplanes`
// planes, one per staged box shape.
int encode_maps(olb_ctx* h, void* buffer, int nplanes, CUtensorMap out[4], const StepInfo& g) {
  auto enc = encode_fn();
  if (!enc) return fail(OLB_ECUDA, "cuTensorMapEncodeTiled is not available");
  CUtensorMapDataType dt;
  switch (h->storage) {
    case OLB_FP64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case OLB_FP32_SHIFTED: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case OLB_BF16_SHIFTED: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
  }
  const Padded& P = h->pad;
  const cuuint64_t dims[4] = {(cuuint64_t)P.np[0], (cuuint64_t)P.np[1], (cuuint64_t)P.np[2], (cuuint64_t)nplanes};
  const cuuint64_t strides[3] = {(cuuint64_t)P.np[0] * h->elem, (cuuint64_t)P.np[0] * P.np[1] * h->elem,
                                 (cuuint64_t)P.plane * h->elem};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  for (int v = 0; v < 4; ++v) {
    const cuuint32_t box[4] = {(cuuint32_t)g.bxw, (cuuint32_t)((v & 1) ? g.by : g.ty),
                               (cuuint32_t)((v & 2) ? g.bz : g.tz), 1};
    CUresult r = enc(&out[v], dt, 4, buffer, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(OLB_ECUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
  }
  return OLB_OK;
}

int build_maps(olb_ctx* h) {
  for (int b = 0; b < 2; ++b) {
    const int rc = encode_maps(h, h->buf[b], h->planes, h->maps.m[b], h->info);
    if (rc) return rc;
  }
  return OLB_OK;
}

// Device error flag set by a step kernel whose bounded wait ran out.  The
// flag is moved to the handle (state_bad) and cleared on the device; the state
// stays invalid until a writer of a whole state (init, set_populations,
// set_state) runs.
int check_err(olb_ctx* h) {
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "error flag");
  if (v) {
    h->state_bad = 1;
    e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "error flag reset");
  }
  if (h->state_bad)
    return fail(OLB_ETIMEOUT, "a step kernel gave up waiting for a staging copy; the state is invalid "
                              "until a new one is written");
  return OLB_OK;
}

// A writer of a whole state starts a valid history: clear both error flags
// (stream-ordered after any step that ran before it).
int clear_err(olb_ctx* h) {
  h->state_bad = 0;
  cudaError_t e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
  return e == cudaSuccess ? OLB_OK : cuda_fail(e, "error flag reset");
}

int set_device(olb_ctx* h) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != h->device) {
    e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return OLB_OK;
}

int stream_sync(olb_ctx* h, int timeout_ms) {
  if (timeout_ms <= 0) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? OLB_OK : cuda_fail(e, "cudaStreamSynchronize");
  }
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(h->stream);
    if (e == cudaSuccess) return OLB_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
    auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) return fail(OLB_ETIMEOUT, "stream did not finish within the time limit");
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

// Copy `bytes` between a caller buffer and a device buffer on the stream;
// host copies are completed before returning.
int copy_in(olb_ctx* h, void* dev_dst, const void* src, size_t bytes, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dev_dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  return on_device ? OLB_OK : stream_sync(h, 0);
}

int copy_out(olb_ctx* h, void* dst, const void* dev_src, size_t bytes, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, dev_src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  return on_device ? OLB_OK : stream_sync(h, 0);
}

// Device address of host memory that the GPU can read and write in place:
// page-locked memory mapped into the device's address space (cudaHostAlloc or
// cudaHostRegister under unified addressing).  Kernels then move the bytes over
// the CPU-GPU link themselves, with no staging copy.  Null for any other
// memory (pageable host memory goes through a device buffer and a copy).
void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Device staging buffer for host-side FP64 arrays (freed by the caller).
int dev_alloc(olb_ctx* h, void** p, size_t bytes) {
  cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e != cudaSuccess) return fail(OLB_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  return OLB_OK;
}

int launch_rc(int rc, const char* what) {
  if (rc == 0) return OLB_OK;
  if (rc < 0) return fail(OLB_EUNSUPPORTED, std::string(what) + ": configuration not built");
  return cuda_fail((cudaError_t)rc, what);
}

// Refill the x ghost columns of buffer b when x is not periodic.
int apply_xbc(olb_ctx* h, void* b) {
  if (!h->xbc) return OLB_OK;
  return launch_rc(launch_xbc(h->aux, b, h->xbc_vals, h->stream), "x boundary");
}

// Launch description of the forward step on the handle's buffers.
StepLaunch base_launch(olb_ctx* h) {
  StepLaunch L{};
  L.a = h->args;
  L.D = h->D;
  L.P = h->p;
  L.storage = h->storage;
  L.compressible = h->comp;
  L.veltab = h->veltab.data();
  L.stentab = h->stentab.data();
  L.stentab2 = nullptr;
  L.maps = &h->maps;
  L.sched = &h->sched;
  L.grid = h->step_grid;
  L.force_generic = h->force_generic;
  L.stream = h->stream;
  return L;
}

// ---------------------------------------------------------------------------
// Adjoint of the isothermal step
// ---------------------------------------------------------------------------

size_t adj_elem(const olb_ctx* h) { return h->storage == OLB_FP64 ? sizeof(double) : sizeof(float); }

// Stencils of the adjoint input: the reflected stencil (transpose of the
// pull: first point -(m0 + p), weights in reverse order, same axes) and the
// identity (no axis active).
template <typename C, int P1>
void fill_adj_tabs_p(olb_ctx* h) {
  h->st_refl = h->stentab;
  h->st_id.assign(sizeof(StencilTab<C, P1>), 0);
  auto* r = reinterpret_cast<StencilTab<C, P1>*>(h->st_refl.data());
  auto* id = reinterpret_cast<StencilTab<C, P1>*>(h->st_id.data());
  const int p = h->p;
  const auto* f = reinterpret_cast<const StencilTab<C, P1>*>(h->stentab.data());
  for (int i = 0; i < h->Q; ++i) {
    for (int a = 0; a < 3; ++a) {
      r->m0[i][a] = -h->m0[i * 3 + a] - p;
      // the forward table's own weights reversed: the exact transpose of its pull
      for (int j = 0; j <= p; ++j) r->W[i][a][j] = f->W[i][a][p - j];
      id->m0[i][a] = 0;
      id->W[i][a][0] = (C)1;
    }
    id->active[i] = 0;
  }
}

template <typename C>
void fill_adj_tabs(olb_ctx* h) {
  if (h->p == 3) fill_adj_tabs_p<C, 4>(h);
  else fill_adj_tabs_p<C, 5>(h);
}

// Buffers, tables and schedules of the adjoint sweep (once per handle).
int adj_prepare(olb_ctx* h) {
  if (h->xbc) return fail(OLB_EUNSUPPORTED, "the adjoint is built for periodic grids only");
  if (h->glc) return fail(OLB_EUNSUPPORTED, "the adjoint is built for the uniform-grid interpolation only");
  if (h->adj_ready) return OLB_OK;
  if (h->comp) return fail(OLB_EUNSUPPORTED, "the adjoint is built for the isothermal step only");
  if (h->storage != OLB_FP64 && h->storage != OLB_FP32_SHIFTED)
    return fail(OLB_EUNSUPPORTED, "the adjoint is built for FP64 and FP32 storage");
  if (h->info.wg == 0 || (h->p != 3 && h->p != 4))
    return fail(OLB_EUNSUPPORTED, "the adjoint needs the two-phase kernel (p = 3 or 4, automatic kernel choice)");
  // geometry of the adjoint kernel: the two-phase kernel's tile, boxes and grid
  if (step_info(h->D, h->p, h->storage, h->comp, h->Q, h->N, 2, &h->ainfo) != 0 || h->ainfo.wg == 0 ||
      h->ainfo.ctas_per_sm < 1)
    return fail(OLB_EUNSUPPORTED, "the adjoint kernel is not built for this configuration");
  {
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    h->adj_nt[0] = (h->grid.n[0] + h->ainfo.tx - 1) / h->ainfo.tx;
    h->adj_nt[1] = (h->grid.n[1] + h->ainfo.ty - 1) / h->ainfo.ty;
    h->adj_nt[2] = (h->grid.n[2] + h->ainfo.tz - 1) / h->ainfo.tz;
    h->adj_ntiles = h->adj_nt[0] * h->adj_nt[1] * h->adj_nt[2];
    long long g = (long long)sms * h->ainfo.ctas_per_sm;
    h->adj_grid = (int)(g > h->adj_ntiles ? h->adj_ntiles : g);
  }
  // the reflected stencil must stay inside the ghost layers
  for (int i = 0; i < h->Q; ++i)
    for (int a = 0; a < h->D; ++a) {
      if (h->set.xi[i][a] == 0.0) continue;
      const int m0 = h->m0[i * 3 + a];
      if (m0 + h->p > h->pad.gl[a] || -m0 > h->pad.gr[a])
        return fail(OLB_EUNSUPPORTED, "reflected stencil reaches beyond the ghost layers (asymmetric set)");
    }
  if (h->storage == OLB_FP64) fill_adj_tabs<double>(h);
  else fill_adj_tabs<float>(h);
  const size_t bytes = (size_t)h->Q * h->pad.plane * h->elem;
  for (int k = 0; k < 2; ++k) {
    if (h->adj[k]) continue;
    cudaError_t e = cudaMalloc(&h->adj[k], bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->adj[k], 0, bytes, h->stream);
    if (e != cudaSuccess) return fail(OLB_ENOMEM, "adjoint buffers: " + std::string(cudaGetErrorString(e)));
    const int rc = encode_maps(h, h->adj[k], h->Q, h->adj_maps.m[k], h->ainfo);
    if (rc) return rc;
  }
  if (!h->adj_scratch) {
    const size_t sb = (size_t)h->adj_grid * 2 * h->Q * h->ainfo.tile * adj_elem(h);
    cudaError_t e = cudaMalloc(&h->adj_scratch, sb);
    if (e != cudaSuccess) return fail(OLB_ENOMEM, "adjoint staging: " + std::string(cudaGetErrorString(e)));
  }
  // every launch stages the adjoint planes only (the forward populations
  // come from the tape)
  std::vector<std::pair<double, int>> adj_planes;
  for (int i = 0; i < h->Q; ++i) adj_planes.push_back({plane_cost(h, i), h->Q + i});
  lpt_schedule(h->ainfo.wg, adj_planes, &h->sched_adj);
  h->adj_ready = 1;
  return OLB_OK;
}

// One launch of the adjoint kernel: adjoint input adj[in], output adj[out],
// moments of the pulled forward populations in tape slot `slot` (mode 1; -1
// in mode 2).  Only the adjoint planes are staged (sched_adj); phase B reads
// the moments from the slot.
int adj_launch(olb_ctx* h, int mode, const std::vector<unsigned char>& st2, int slot, int in, int out) {
  StepLaunch L = base_launch(h);
  L.a.buf[0] = h->adj[in];
  L.a.buf[1] = h->adj[out];
  L.a.slab = slot >= 0 ? h->tape[slot] : nullptr;
  L.a.src = 0;
  L.a.scratch = h->adj_scratch;
  L.a.planes = 2 * h->Q;
  L.a.reduce = 0;
  L.a.mode = mode;
  for (int k = 0; k < 3; ++k) L.a.nt[k] = h->adj_nt[k];
  L.a.ntiles = h->adj_ntiles;
  L.grid = h->adj_grid;
  TmaMaps M;
  std::memcpy(M.m[0], h->adj_maps.m[in], sizeof(M.m[0]));
  std::memcpy(M.m[1], h->adj_maps.m[in], sizeof(M.m[1]));
  L.stentab2 = st2.data();
  L.maps = &M;
  L.sched = &h->sched_adj;
  int r;
  if (h->storage == OLB_FP64) r = h->D == 2 ? launch_adj_f64_2d(L) : launch_adj_f64_3d(L);
  else r = h->D == 2 ? launch_adj_f32_2d(L) : launch_adj_f32_3d(L);
  return launch_rc(r, "sl_adjoint");
}

// Adjoint sweep over the forward states in `slots` (the input of the last
// step first).  lam_dev (compact [Q][n], adjoint type): on entry dJ/d(state
// after the last step), on return dJ/d(state before the first step).
int adjoint_sweep(olb_ctx* h, const std::vector<int>& slots, void* lam_dev) {
  int rc = launch_rc(launch_scatter(h->aux, h->adj[0], lam_dev, h->stream), "adjoint scatter");
  if (rc) return rc;
  int cur = 0;
  for (size_t k = 0; k < slots.size(); ++k) {
    const bool first = k == 0;
    rc = adj_launch(h, 1, first ? h->st_id : h->st_refl, slots[k], cur, cur ^ 1);
    if (rc) return rc;
    cur ^= 1;
  }
  rc = adj_launch(h, 2, h->st_refl, -1, cur, cur ^ 1);
  if (rc) return rc;
  cur ^= 1;
  return launch_rc(launch_gather(h->aux, h->adj[cur], lam_dev, h->stream), "adjoint gather");
}

// Tape slots (after adj_prepare): the moments of one step's pulled populations
// in the two-phase kernel's tile order.
int tape_grow(olb_ctx* h, int nslots) {
  const size_t bytes = (size_t)h->adj_ntiles * 4 * h->ainfo.tile * adj_elem(h);
  while ((int)h->tape.size() < nslots) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, h->stream);
    if (e != cudaSuccess) {
      if (p) cudaFree(p);
      return fail(OLB_ENOMEM, "tape slot: " + std::string(cudaGetErrorString(e)));
    }
    h->tape.push_back(p);
  }
  return OLB_OK;
}

// One forward step of the two-phase kernel from padded buffer `src` (maps
// `m`) into `dst` that also stores the moments of its pulled populations in
// tape slot `slot`.
int record_step(olb_ctx* h, void* src, const CUtensorMap* m, void* dst, int slot) {
  StepLaunch L = base_launch(h);
  L.force_generic = 2;
  L.a.reduce = 0;
  L.a.src = 0;
  L.a.buf[0] = src;
  L.a.buf[1] = dst;
  L.a.slab = h->tape[slot];
  for (int k = 0; k < 3; ++k) L.a.nt[k] = h->adj_nt[k];
  L.a.ntiles = h->adj_ntiles;
  L.grid = h->adj_grid;
  TmaMaps M;
  std::memcpy(M.m[0], m, sizeof(M.m[0]));
  std::memcpy(M.m[1], m, sizeof(M.m[1]));
  L.maps = &M;
  return launch_rc(launch_step(h->storage, h->D, L), "sl_step (recorded)");
}

}  // namespace

namespace {
// Identity stencil in the arithmetic type C: no axis active.
template <typename C, int P1>
void identity_stencil_p(olb_ctx* h, std::vector<unsigned char>& out) {
  out.assign(sizeof(StencilTab<C, P1>), 0);
  auto* t = reinterpret_cast<StencilTab<C, P1>*>(out.data());
  for (int i = 0; i < h->Q; ++i) {
    t->active[i] = 0;
    for (int a = 0; a < 3; ++a) t->W[i][a][0] = (C)1;
  }
}
template <typename C>
void identity_stencil(olb_ctx* h, std::vector<unsigned char>& out) {
  switch (h->p) {
    case 1: identity_stencil_p<C, 2>(h, out); break;
    case 2: identity_stencil_p<C, 3>(h, out); break;
    case 3: identity_stencil_p<C, 4>(h, out); break;
    case 4: identity_stencil_p<C, 5>(h, out); break;
    case 5: identity_stencil_p<C, 6>(h, out); break;
    default: identity_stencil_p<C, 7>(h, out); break;
  }
}

}  // namespace

extern "C" {

void olb_default_options(olb_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->interp_order = 3;
  opt->storage = OLB_FP64;
  opt->cs_scale = 1.0;
  opt->compressible = 0;
  opt->gamma = 1.4;
  opt->mu = 0.0;
  opt->mu_exponent = 0.0;
  opt->prandtl = 1.0;
  opt->rho0 = 1.0;
  opt->allow_inexact = 0;
  opt->log_every = 1;
  opt->kernel = 0;
  opt->stream = nullptr;
}

int olb_velocity_set_info(int velocity_set, int* Q, int* D, double* cs, double* max_abs_xi, int* degree) {
  VelocitySet vs;
  if (olb::velocity_set(velocity_set, &vs) != 0) return fail(OLB_EINVAL, "unknown velocity set");
  double m = 0.0;
  for (int i = 0; i < vs.Q; ++i)
    for (int a = 0; a < 3; ++a) m = std::fmax(m, std::fabs(vs.xi[i][a]));
  if (Q) *Q = vs.Q;
  if (D) *D = vs.D;
  if (cs) *cs = vs.cs;
  if (max_abs_xi) *max_abs_xi = m;
  if (degree) *degree = vs.degree;
  return OLB_OK;
}

int olb_velocity_set_table(int velocity_set, double* xi, double* w) {
  VelocitySet vs;
  if (olb::velocity_set(velocity_set, &vs) != 0) return fail(OLB_EINVAL, "unknown velocity set");
  for (int i = 0; i < vs.Q; ++i) {
    if (xi)
      for (int a = 0; a < vs.D; ++a) xi[i * vs.D + a] = vs.xi[i][a];
    if (w) w[i] = vs.w[i];
  }
  return OLB_OK;
}

int olb_glc_stencil(int p, double shift, int* first, double* W) {
  if (p < 1 || p > OLB_GLC_MAX_P) return fail(OLB_EINVAL, "GLC order p must be in 1..8");
  if (!std::isfinite(shift)) return fail(OLB_EINVAL, "shift must be finite");
  if (!first || !W) return fail(OLB_EINVAL, "null output");
  double z[OLB_GLC_MAX_P + 1];
  for (int m = 0; m <= p; ++m) z[m] = 0.5 * (1.0 - std::cos(M_PI * m / p));
  for (int k = 0; k < p; ++k) {
    // departure point of the node with local coordinate z[k], in cell widths
    const double xl = z[k] - shift;
    const double d = std::floor(xl), zeta = xl - d;
    first[k] = (int)d * p - k;
    for (int m = 0; m <= p; ++m) {
      double prod = 1.0;
      for (int l = 0; l <= p; ++l)
        if (l != m) prod *= (zeta - z[l]) / (z[m] - z[l]);
      W[k * (p + 1) + m] = prod;
    }
  }
  return OLB_OK;
}

int olb_create(const olb_grid* grid, int velocity_set, int hermite_order, double tau, double dt,
               const olb_options* opt_in, olb_handle* out) {
  if (!grid || !out) return fail(OLB_EINVAL, "null grid or output handle");
  *out = nullptr;
  olb_options opt;
  olb_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (grid->dim != 2 && grid->dim != 3) return fail(OLB_EINVAL, "grid dim must be 2 or 3");
  if (grid->n[0] < 1 || grid->n[1] < 1 || grid->n[2] < 1) return fail(OLB_EINVAL, "grid sizes must be >= 1");
  if (grid->dim == 2 && grid->n[2] != 1) return fail(OLB_EINVAL, "2D grid needs n[2] == 1");
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx)) return fail(OLB_EINVAL, "dx must be positive");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(OLB_EINVAL, "dt must be positive");
  if (hermite_order < 2 || hermite_order > 4) return fail(OLB_EINVAL, "hermite_order must be 2, 3 or 4");
  if (opt.interp_order < 1 || opt.interp_order > MAXP) return fail(OLB_EINVAL, "interp_order must be in 1..6");
  if (storage_bytes(opt.storage) == 0) return fail(OLB_EINVAL, "unknown storage");
  if (!(opt.cs_scale > 0.0) || !std::isfinite(opt.cs_scale)) return fail(OLB_EINVAL, "cs_scale must be positive");
  if (!(opt.rho0 > 0.0)) return fail(OLB_EINVAL, "rho0 must be positive");
  if (opt.log_every < 1) return fail(OLB_EINVAL, "log_every must be >= 1");
  if (opt.kernel < 0 || opt.kernel > 2)
    return fail(OLB_EINVAL, "kernel must be 0 (automatic), 1 (single-role) or 2 (two-phase)");

  VelocitySet vs;
  if (olb::velocity_set(velocity_set, &vs) != 0) return fail(OLB_EINVAL, "unknown velocity set");
  if (vs.D != grid->dim) return fail(OLB_EINVAL, "velocity set dimension differs from the grid's");
  if (vs.degree < 2 * hermite_order && !opt.allow_inexact)
    return fail(OLB_EUNSUPPORTED, "quadrature degree below 2N: the equilibrium moments are not exact (d >= N + M)");
  const double cs = vs.cs * opt.cs_scale;
  if (opt.compressible) {
    if (std::fabs(cs - 1.0) > 1e-12)
      return fail(OLB_EUNSUPPORTED, "compressible runs need c_s = 1 (T0 = 1)");
    if (!(opt.gamma > 1.0)) return fail(OLB_EINVAL, "gamma must exceed 1");
    if (!(opt.mu > 0.0)) return fail(OLB_EINVAL, "compressible runs need mu > 0");
    if (!std::isfinite(opt.mu_exponent)) return fail(OLB_EINVAL, "mu_exponent must be finite");
    if (!(opt.prandtl > 0.0) || !std::isfinite(opt.prandtl)) return fail(OLB_EINVAL, "prandtl must be positive");
    // the heat-flux projection is exact only where the set integrates sixth
    // moments, and f^eq has no central heat flux only for N >= 3
    if (opt.prandtl != 1.0 && (vs.degree < 7 || hermite_order < 3))
      return fail(OLB_EUNSUPPORTED, "prandtl != 1 needs N >= 3 and a velocity set of degree >= 7");
  } else if (!(tau > 0.5) || !std::isfinite(tau)) {
    return fail(OLB_EINVAL, "tau must exceed 1/2");
  } else if (opt.prandtl != 1.0) {
    return fail(OLB_EINVAL, "the Prandtl number is a parameter of the compressible model");
  }
  const long long nnodes = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  if (nnodes > (1LL << 31) - 1) return fail(OLB_EBOUNDS, "grid larger than 2^31 nodes");

  olb_ctx* h = new (std::nothrow) olb_ctx();
  if (!h) return fail(OLB_ENOMEM, "host allocation failed");
  h->grid = *grid;
  h->vs_id = velocity_set;
  h->N = hermite_order;
  h->p = opt.interp_order;
  h->storage = opt.storage;
  h->comp = opt.compressible ? 1 : 0;
  h->allow_inexact = opt.allow_inexact;
  h->log_every = opt.log_every;
  h->force_generic = opt.kernel;  // kernel mode: 0 automatic, 1 single-role, 2 two-phase
  h->tau = tau;
  h->dt = dt;
  h->gamma = opt.gamma;
  h->mu = opt.mu;
  h->mu_exp = opt.compressible ? opt.mu_exponent : 0.0;
  h->prandtl = opt.compressible ? opt.prandtl : 1.0;
  h->rho0 = opt.rho0;
  h->cs_scale = opt.cs_scale;
  h->cs = cs;
  h->set = vs;
  for (int i = 0; i < vs.Q; ++i)
    for (int a = 0; a < 3; ++a) h->set.xi[i][a] = vs.xi[i][a] * opt.cs_scale;
  h->set.cs = cs;
  h->Q = vs.Q;
  h->D = vs.D;
  h->planes = h->comp ? 2 * vs.Q : vs.Q;
  h->elem = storage_bytes(opt.storage);
  h->nnodes = nnodes;
  h->stream = static_cast<cudaStream_t>(opt.stream);

  if (step_info(h->D, h->p, h->storage, h->comp, h->Q, h->N, h->force_generic, &h->info) != 0) {
    release(h);
    return fail(OLB_EUNSUPPORTED, "interpolation order not built for this storage");
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    release(h);
    return cuda_fail(e, "cudaGetDevice");
  }
  if (h->info.ctas_per_sm < 1) {
    release(h);
    return fail(OLB_ECUDA, "step kernel cannot be resident on this device");
  }

  // stencil of the pull (Sec. 3, Eq. sl_streaming): delta = -xi dt / dx
  h->m0.assign(h->Q * 3, 0);
  h->W.assign(h->Q * 3 * (h->p + 1), 0.0);
  for (int i = 0; i < h->Q; ++i)
    for (int a = 0; a < 3; ++a) {
      const double delta = -h->set.xi[i][a] * dt / grid->dx;
      lagrange_stencil(delta, h->p, &h->m0[i * 3 + a], &h->W[(i * 3 + a) * (h->p + 1)]);
    }
  if (h->storage == OLB_FP64) {
    fill_veltab<double>(h);
    fill_stentab<double>(h);
  } else {
    fill_veltab<float>(h);
    fill_stentab<float>(h);
    fill_uhat_fix(h);
  }

  build_schedule(h);
  const double Cv = 1.0 / (h->gamma - 1.0);
  const double rho_ref = h->storage == OLB_FP64 ? 0.0 : h->rho0;
  layout_padding(h);
  StepArgs& a = h->args;
  a.pad = h->pad;
  a.nt[0] = (grid->n[0] + h->info.tx - 1) / h->info.tx;
  a.nt[1] = (grid->n[1] + h->info.ty - 1) / h->info.ty;
  a.nt[2] = (grid->n[2] + h->info.tz - 1) / h->info.tz;
  a.ntiles = a.nt[0] * a.nt[1] * a.nt[2];
  a.Q = h->Q;
  a.planes = h->planes;
  a.N = h->N;
  a.quad_ok = (grid->n[0] % 4) == 0;
  a.rho_ref = rho_ref;
  a.tau = tau;
  a.inv_tau = 1.0 / tau;
  a.mu_dt = h->mu / (cs * cs * dt);
  a.mu_exp = h->mu_exp;
  a.two_cv = 2.0 * Cv;
  a.gfac = 2.0 * Cv - h->D;
  a.inv_cs = 1.0 / cs;
  a.cs2 = cs * cs;
  a.dt = dt;
  a.f_rho_ref = (float)a.rho_ref;
  a.f_inv_tau = (float)a.inv_tau;
  a.f_tau = (float)a.tau;
  a.f_mu_dt = (float)a.mu_dt;
  a.f_two_cv = (float)a.two_cv;
  a.f_gfac = (float)a.gfac;
  a.f_inv_cs = (float)a.inv_cs;
  a.f_cs2 = (float)a.cs2;
  a.f_dt = (float)a.dt;
  a.f_mu_exp = (float)a.mu_exp;
  a.qe = h->prandtl != 1.0 ? 1 : 0;
  a.inv_pr = 1.0 / h->prandtl;
  a.f_inv_pr = (float)a.inv_pr;

  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    release(h);
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  long long g = (long long)sms * h->info.ctas_per_sm;
  if (g > a.ntiles) g = a.ntiles;
  h->step_grid = (int)g;
  const int aux_slots = 1024;
  h->partial_slots = h->step_grid > aux_slots ? h->step_grid : aux_slots;

  const size_t cbytes = h->storage == OLB_FP64 ? 8 : 4;
  const size_t state_bytes = (size_t)h->planes * h->pad.plane * h->elem;
  const size_t scratch_bytes = (size_t)h->step_grid * h->planes * h->info.tile * cbytes;
  for (int k = 0; k < 2; ++k) {
    e = cudaMalloc(&h->buf[k], state_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[k], 0, state_bytes, h->stream);
    if (e != cudaSuccess) {
      release(h);
      return fail(OLB_ENOMEM, "population buffers: " + std::string(cudaGetErrorString(e)));
    }
  }
  e = cudaMalloc(&h->scratch, scratch_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->partials, (size_t)h->partial_slots * NRED * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->red_dev, NRED * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->err_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) {
    release(h);
    return fail(OLB_ENOMEM, "scratch buffers: " + std::string(cudaGetErrorString(e)));
  }
  a.buf[0] = h->buf[0];
  a.buf[1] = h->buf[1];
  a.scratch = h->scratch;
  a.partials = h->partials;
  a.err = h->err_dev;
  a.wait_polls = 1LL << 24;
  {
    int rcm = build_maps(h);
    if (rcm != OLB_OK) {
      release(h);
      return rcm;
    }
  }

  AuxArgs& x = h->aux;
  x.pad = h->pad;
  x.nnodes = nnodes;
  x.Q = h->Q;
  x.planes = h->planes;
  x.D = h->D;
  x.N = h->N;
  x.storage = h->storage;
  x.compressible = h->comp;
  x.rho_ref = rho_ref;
  x.gfac = a.gfac;
  x.two_cv = a.two_cv;
  x.inv_cs = a.inv_cs;
  x.cs2 = a.cs2;
  for (int i = 0; i < h->Q; ++i) {
    for (int c = 0; c < 3; ++c) {
      x.xi[i][c] = h->set.xi[i][c];
      x.xih[i][c] = h->set.xi[i][c] / cs;
    }
    x.w[i] = h->set.w[i];
    x.base[i] = rho_ref * h->set.w[i];
    if (h->comp) x.base[h->Q + i] = rho_ref * h->set.w[i] * a.gfac;
  }
  x.rest_rho = h->rho0;
  // start from the uniform rest state rho = rho0, u = 0 (theta = 1)
  int rc0 = launch_rc(launch_init_fields(h->aux, h->buf[0], nullptr, nullptr, nullptr, h->stream), "init_rest");
  if (rc0 != OLB_OK) {
    release(h);
    return rc0;
  }
  *out = h;
  return OLB_OK;
}

int olb_destroy(olb_handle h) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  set_device(h);
  cudaStreamSynchronize(h->stream);
  release(h);
  return OLB_OK;
}

int olb_shape(olb_handle h, int* Q, int* planes, size_t* nodes, int* dim, int* elem_bytes) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (Q) *Q = h->Q;
  if (planes) *planes = h->planes;
  if (nodes) *nodes = (size_t)h->nnodes;
  if (dim) *dim = h->D;
  if (elem_bytes) *elem_bytes = h->elem;
  return OLB_OK;
}

int olb_stencil(olb_handle h, int* m0, double* W) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (m0) std::memcpy(m0, h->m0.data(), h->m0.size() * sizeof(int));
  if (W) std::memcpy(W, h->W.data(), h->W.size() * sizeof(double));
  return OLB_OK;
}

int olb_init_fields(olb_handle h, const double* rho, const double* u, const double* theta, int on_device) {
  if (!h || !rho || !u) return fail(OLB_EINVAL, "null handle or field");
  int rc = set_device(h);
  if (rc) return rc;
  rc = clear_err(h);
  if (rc) return rc;
  const size_t n = (size_t)h->nnodes;
  const double *dr = rho, *du = u, *dth = theta;
  void* tmp = nullptr;
  if (!on_device) {
    const size_t bytes = n * (size_t)(1 + h->D + (theta ? 1 : 0)) * sizeof(double);
    rc = dev_alloc(h, &tmp, bytes);
    if (rc) return rc;
    double* t = static_cast<double*>(tmp);
    cudaMemcpyAsync(t, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(t + n, u, n * h->D * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (theta) cudaMemcpyAsync(t + n * (1 + h->D), theta, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    dr = t;
    du = t + n;
    dth = theta ? t + n * (1 + h->D) : nullptr;
  }
  rc = launch_rc(launch_init_fields(h->aux, h->buf[h->cur], dr, du, dth, h->stream), "init_fields");
  if (rc == OLB_OK) rc = apply_xbc(h, h->buf[h->cur]);
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    if (rc == OLB_OK) rc = stream_sync(h, 0);
  }
  h->partials_valid = 0;
  return rc;
}

int olb_step(olb_handle h, int n) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (n < 0) return fail(OLB_EINVAL, "negative step count");
  if (h->state_bad)
    return fail(OLB_ETIMEOUT, "the state is invalid after a step gave up waiting for a staging copy; "
                              "write a new state first");
  int rc = set_device(h);
  if (rc) return rc;
  StepLaunch L = base_launch(h);
  if (h->glc) L.stentab = h->st_glc_id.data();
  for (int s = 0; s < n; ++s) {
    const long long count = h->step_count + 1;
    L.a.reduce = (count % h->log_every) == 0;
    if (h->glc) {
      // cell-wise GLC pull into the other buffer, then the collision of those
      // values (the step kernel with the identity stencil) back into this one
      rc = launch_rc(launch_glc_pull(h->storage, h->glc_args, h->buf[h->cur], h->buf[h->cur ^ 1], h->stream),
                     "GLC pull");
      if (rc) return rc;
      L.a.src = h->cur ^ 1;
      rc = launch_rc(launch_step(h->storage, h->D, L), "sl_step (collision)");
      if (rc) return rc;
      h->step_count = count;
      h->partials_valid = L.a.reduce;
      continue;
    }
    L.a.src = h->cur;
    const int r = launch_step(h->storage, h->D, L);
    rc = launch_rc(r, "sl_step");
    if (rc) return rc;
    h->cur ^= 1;
    rc = apply_xbc(h, h->buf[h->cur]);
    if (rc) return rc;
    h->step_count = count;
    h->partials_valid = L.a.reduce;
  }
  return OLB_OK;
}

int olb_moments(olb_handle h, double* rho, double* u, double* theta, int on_device) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  int rc = set_device(h);
  if (rc) return rc;
  const size_t n = (size_t)h->nnodes;
  double *dr = rho, *du = u, *dth = theta;
  void* tmp = nullptr;
  if (!on_device) {
    rc = dev_alloc(h, &tmp, n * (size_t)(2 + h->D) * sizeof(double));
    if (rc) return rc;
    double* t = static_cast<double*>(tmp);
    dr = rho ? t : nullptr;
    du = u ? t + n : nullptr;
    dth = theta ? t + n * (1 + h->D) : nullptr;
  }
  rc = check_err(h);
  if (rc == OLB_OK)
    rc = launch_rc(launch_state_moments(h->aux, h->buf[h->cur], dr, du, dth, nullptr, 1024, h->stream),
                   "state_moments");
  if (rc == OLB_OK && !on_device) {
    double* t = static_cast<double*>(tmp);
    if (rho) cudaMemcpyAsync(rho, t, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (u) cudaMemcpyAsync(u, t + n, n * h->D * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (theta) cudaMemcpyAsync(theta, t + n * (1 + h->D), n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    int r2 = stream_sync(h, 0);
    if (rc == OLB_OK) rc = r2;
  }
  return rc;
}

int olb_reductions(olb_handle h, double out[8]) {
  if (!h || !out) return fail(OLB_EINVAL, "null handle or output");
  int rc = set_device(h);
  if (rc) return rc;
  int slots;
  const bool from_step = h->partials_valid != 0;
  if (from_step) {
    slots = h->step_grid;
  } else {
    slots = 1024;
    rc = launch_rc(launch_state_moments(h->aux, h->buf[h->cur], nullptr, nullptr, nullptr, h->partials, slots,
                                        h->stream),
                   "state_moments");
    if (rc) return rc;
  }
  rc = launch_rc(launch_reduce_final(h->partials, slots, h->red_dev, h->stream), "reduce_final");
  if (rc) return rc;
  rc = copy_out(h, out, h->red_dev, NRED * sizeof(double), 0);
  if (rc) return rc;
  rc = check_err(h);
  if (rc) return rc;
  const double nn = (double)h->nnodes;
  out[0] /= nn;
  out[1] /= nn;
  out[2] = from_step ? out[2] / nn : NAN;
  out[3] += h->aux.rho_ref * nn;
  if (out[7] > 0.0) return fail(OLB_ENONFINITE, "state holds non-finite values");
  return OLB_OK;
}

int olb_enstrophy(olb_handle h, double* enstrophy) {
  if (!h || !enstrophy) return fail(OLB_EINVAL, "null handle or output");
  if (h->xbc) return fail(OLB_EUNSUPPORTED, "the enstrophy takes periodic differences: not defined with a non-periodic x");
  int rc = set_device(h);
  if (rc) return rc;
  const int slots = 1024;
  if (!h->ens_u) {
    cudaError_t e = cudaMalloc((void**)&h->ens_u, (size_t)h->nnodes * h->D * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->ens_part, (size_t)slots * NRED * sizeof(double));
    if (e != cudaSuccess) return fail(OLB_ENOMEM, "enstrophy buffers: " + std::string(cudaGetErrorString(e)));
  }
  rc = launch_rc(launch_state_moments(h->aux, h->buf[h->cur], nullptr, h->ens_u, nullptr, nullptr, slots, h->stream),
                 "state_moments");
  if (rc) return rc;
  rc = launch_rc(launch_enstrophy(h->aux, h->ens_u, h->grid.dx, h->ens_part, slots, h->stream), "enstrophy");
  if (rc) return rc;
  rc = launch_rc(launch_reduce_final(h->ens_part, slots, h->red_dev, h->stream), "reduce_final");
  if (rc) return rc;
  double out[NRED];
  rc = copy_out(h, out, h->red_dev, NRED * sizeof(double), 0);
  if (rc) return rc;
  rc = check_err(h);
  if (rc) return rc;
  *enstrophy = out[0] / (double)h->nnodes;
  if (!std::isfinite(*enstrophy)) return fail(OLB_ENONFINITE, "velocity field holds non-finite values");
  return OLB_OK;
}

int olb_kinetic_energy(olb_handle h, double* k, double* dissipation) {
  double r[NRED];
  int rc = olb_reductions(h, r);
  if (k) *k = r[0];
  if (dissipation) *dissipation = r[2];
  return rc;
}

int olb_get_populations(olb_handle h, double* f, int on_device) {
  if (!h || !f) return fail(OLB_EINVAL, "null handle or buffer");
  int rc = set_device(h);
  if (rc) return rc;
  rc = check_err(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->planes * h->nnodes * sizeof(double);
  double* d = f;
  void* tmp = nullptr;
  if (!on_device) {
    rc = dev_alloc(h, &tmp, bytes);
    if (rc) return rc;
    d = static_cast<double*>(tmp);
  }
  rc = launch_rc(launch_to_f64(h->aux, h->buf[h->cur], d, h->stream), "to_f64");
  if (rc == OLB_OK && !on_device) rc = copy_out(h, f, d, bytes, 0);
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    int r2 = stream_sync(h, 0);
    if (rc == OLB_OK) rc = r2;
  }
  return rc;
}

int olb_set_populations(olb_handle h, const double* f, int on_device) {
  if (!h || !f) return fail(OLB_EINVAL, "null handle or buffer");
  int rc = set_device(h);
  if (rc) return rc;
  rc = clear_err(h);
  if (rc) return rc;
  const size_t bytes = (size_t)h->planes * h->nnodes * sizeof(double);
  const double* d = f;
  void* tmp = nullptr;
  if (!on_device) {
    rc = dev_alloc(h, &tmp, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync");
    d = static_cast<const double*>(tmp);
  }
  if (rc == OLB_OK) rc = launch_rc(launch_from_f64(h->aux, h->buf[h->cur], d, h->stream), "from_f64");
  if (rc == OLB_OK) rc = apply_xbc(h, h->buf[h->cur]);
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    int r2 = stream_sync(h, 0);
    if (rc == OLB_OK) rc = r2;
  }
  h->partials_valid = 0;
  return rc;
}

size_t olb_state_bytes(olb_handle h) {
  if (!h) return 0;
  return (size_t)h->planes * h->nnodes * h->elem;
}

int olb_get_state(olb_handle h, void* buf, size_t bytes, int on_device) {
  if (!h || !buf) return fail(OLB_EINVAL, "null handle or buffer");
  if (bytes != olb_state_bytes(h)) return fail(OLB_EINVAL, "state size mismatch");
  int rc = set_device(h);
  if (rc) return rc;
  rc = check_err(h);
  if (rc) return rc;
  void* d = buf;
  void* tmp = nullptr;
  void* mapped = on_device ? nullptr : mapped_host(buf);
  if (mapped) {
    d = mapped;  // the gather writes the host buffer directly
  } else if (!on_device) {
    rc = dev_alloc(h, &tmp, bytes);
    if (rc) return rc;
    d = tmp;
  }
  rc = launch_rc(launch_gather(h->aux, h->buf[h->cur], d, h->stream), "gather");
  if (rc == OLB_OK && mapped) rc = stream_sync(h, 0);
  if (rc == OLB_OK && tmp) rc = copy_out(h, buf, d, bytes, 0);
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    int r2 = stream_sync(h, 0);
    if (rc == OLB_OK) rc = r2;
  }
  return rc;
}

int olb_set_state(olb_handle h, const void* buf, size_t bytes, int on_device) {
  if (!h || !buf) return fail(OLB_EINVAL, "null handle or buffer");
  if (bytes != olb_state_bytes(h)) return fail(OLB_EINVAL, "state size mismatch");
  int rc = set_device(h);
  if (rc) return rc;
  rc = clear_err(h);
  if (rc) return rc;
  const void* d = buf;
  void* tmp = nullptr;
  const void* mapped = on_device ? nullptr : mapped_host(buf);
  if (mapped) {
    d = mapped;  // the scatter reads the host buffer directly
  } else if (!on_device) {
    rc = dev_alloc(h, &tmp, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(tmp, buf, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync");
    d = tmp;
  }
  if (rc == OLB_OK) rc = launch_rc(launch_scatter(h->aux, h->buf[h->cur], d, h->stream), "scatter");
  if (rc == OLB_OK) rc = apply_xbc(h, h->buf[h->cur]);
  if (rc == OLB_OK && mapped) rc = stream_sync(h, 0);
  if (tmp) {
    cudaFreeAsync(tmp, h->stream);
    int r2 = stream_sync(h, 0);
    if (rc == OLB_OK) rc = r2;
  }
  h->partials_valid = 0;
  return rc;
}

int olb_set_x_boundary(olb_handle h, int kind, double rho, const double* u, double theta) {
  if (h && h->glc && kind != 0)
    return fail(OLB_EUNSUPPORTED, "the inflow/outflow x boundary is built for the uniform-grid interpolation only");
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (kind != 0 && kind != 1) return fail(OLB_EINVAL, "x boundary kind must be 0 (periodic) or 1 (inflow/outflow)");
  if (kind == 1) {
    if (!u) return fail(OLB_EINVAL, "null inflow velocity");
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(OLB_EINVAL, "inflow density must be positive");
    if (h->comp && (!(theta > 0.0) || !std::isfinite(theta)))
      return fail(OLB_EINVAL, "inflow temperature must be positive");
    for (int a = 0; a < h->D; ++a)
      if (!std::isfinite(u[a])) return fail(OLB_EINVAL, "inflow velocity must be finite");
  }
  int rc = set_device(h);
  if (rc) return rc;
  if (kind == 1) {
    if (!h->xbc_vals) {
      cudaError_t e = cudaMalloc(&h->xbc_vals, (size_t)h->planes * h->elem);
      if (e != cudaSuccess) {
        h->xbc_vals = nullptr;
        return fail(OLB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
      }
    }
    h->inflow.rho = rho;
    for (int a = 0; a < 3; ++a) h->inflow.u[a] = a < h->D ? u[a] : 0.0;
    h->inflow.theta = h->comp ? theta : 1.0;
    rc = launch_rc(launch_xbc_values(h->aux, h->inflow, h->xbc_vals, h->stream), "x boundary values");
    if (rc) return rc;
    h->xbc = 1;
    return apply_xbc(h, h->buf[h->cur]);
  }
  if (!h->xbc) return OLB_OK;
  // back to periodic: rewrite every ghost copy from the interior, in place
  // (the handle stays non-periodic if that fails)
  rc = launch_rc(launch_periodic_ghosts(h->aux, h->buf[h->cur], h->stream), "periodic ghosts");
  int r2 = stream_sync(h, 0);
  if (rc == OLB_OK) rc = r2;
  if (rc == OLB_OK) h->xbc = 0;
  return rc;
}

int olb_set_interpolation(olb_handle h, int scheme) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (scheme != 0 && scheme != 1) return fail(OLB_EINVAL, "scheme must be 0 (uniform Lagrange) or 1 (cell-wise GLC)");
  if (scheme == 0) {
    h->glc = 0;
    return OLB_OK;
  }
  if (h->xbc) return fail(OLB_EUNSUPPORTED, "the cell-wise GLC pull is built for periodic grids only");
  if (h->p > GLC_PMAX) return fail(OLB_EUNSUPPORTED, "GLC order above the built maximum");
  for (int a = 0; a < h->D; ++a)
    if (h->grid.n[a] % h->p != 0)
      return fail(OLB_EINVAL, "every axis must hold a whole number of cells (n multiple of p)");
  int rc = set_device(h);
  if (rc) return rc;
  GlcArgs& g = h->glc_args;
  g = GlcArgs{};
  g.pad = h->pad;
  g.nnodes = h->nnodes;
  g.planes = h->planes;
  g.Q = h->Q;
  g.D = h->D;
  g.p = h->p;
  const size_t nw = (size_t)MAXQ * 3 * GLC_PMAX * (GLC_PMAX + 1);
  std::vector<double> wd(nw, 0.0);
  const double H = h->p * h->grid.dx;  // cell width: p nodes per cell
  const bool f64 = h->storage == OLB_FP64;
  int T[3];
  glc_tile_shape(h->D, f64 ? 8 : 4, &T[0], &T[1], &T[2]);
  g.ntiles = 1;
  for (int a = 0; a < 3; ++a) {
    g.nt[a] = (h->grid.n[a] + T[a] - 1) / T[a];
    g.ntiles *= g.nt[a];
  }
  g.box_elems = 0;
  g.b1_elems = 0;
  // x reach rounded to whole 16-byte groups, so that every staged row starts
  // on a 16-byte boundary (the 16-byte staging path)
  const int VG = 16 / h->elem;  // stored elements per 16-byte copy
  int exmax = 0;
  for (int i = 0; i < h->Q; ++i) {
    int act = 0, ext[3] = {T[0], T[1], T[2]};
    for (int a = 0; a < h->D; ++a) {
      if (h->set.xi[i][a] == 0.0) continue;  // an axis the velocity does not move along: no pass
      act |= 1 << a;
      int first[GLC_PMAX];
      double W[GLC_PMAX * (GLC_PMAX + 1)];
      rc = olb_glc_stencil(h->p, h->set.xi[i][a] * h->dt / H, first, W);
      if (rc) return rc;
      int lo = 0, hi = 0;
      for (int k = 0; k < h->p; ++k) {
        const int idx = (i * 3 + a) * GLC_PMAX + k;
        g.first[idx] = first[k];
        for (int m = 0; m <= h->p; ++m) wd[(size_t)idx * (GLC_PMAX + 1) + m] = W[k * (h->p + 1) + m];
        lo = std::max(lo, -first[k]);
        hi = std::max(hi, first[k] + h->p);
      }
      if (a == 0) {
        lo = (lo + VG - 1) / VG * VG;
        hi = (T[0] + lo + hi + VG - 1) / VG * VG - T[0] - lo;
      }
      if (lo > 255 || hi > 255) return fail(OLB_EUNSUPPORTED, "GLC departure points too far for the staged box");
      g.lo[i * 3 + a] = (unsigned char)lo;
      g.hi[i * 3 + a] = (unsigned char)hi;
      ext[a] += lo + hi;
    }
    g.active[i] = act;
    g.box_elems = std::max(g.box_elems, ext[0] * ext[1] * ext[2]);
    g.b1_elems = std::max(g.b1_elems, T[0] * ext[1] * ext[2]);
    exmax = std::max(exmax, ext[0]);
  }
  g.vec16 = (h->grid.n[0] % VG == 0 && exmax % VG == 0 && exmax / VG <= 32) ? 1 : 0;
  if (glc_smem_bytes(g, f64 ? 8 : 4, h->elem) > 227 * 1024)
    return fail(OLB_EUNSUPPORTED, "GLC departure points too far for the staged box (Courant number too large)");
  const size_t bytes = nw * (f64 ? sizeof(double) : sizeof(float));
  if (!h->glc_w) {
    cudaError_t e = cudaMalloc(&h->glc_w, (size_t)nw * sizeof(double));
    if (e != cudaSuccess) return fail(OLB_ENOMEM, std::string("GLC weights: ") + cudaGetErrorString(e));
  }
  cudaError_t e;
  if (f64) {
    e = cudaMemcpyAsync(h->glc_w, wd.data(), bytes, cudaMemcpyHostToDevice, h->stream);
  } else {
    std::vector<float> wf(nw);
    for (size_t k = 0; k < nw; ++k) wf[k] = (float)wd[k];
    e = cudaMemcpyAsync(h->glc_w, wf.data(), bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "GLC weights upload");
  g.W = h->glc_w;
  if (f64) identity_stencil<double>(h, h->st_glc_id);
  else identity_stencil<float>(h, h->st_glc_id);
  h->glc = 1;
  return OLB_OK;
}

int olb_set_wait_polls(olb_handle h, long long polls) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  h->args.wait_polls = polls < 0 ? (1LL << 24) : polls;
  return OLB_OK;
}

int olb_synchronize(olb_handle h, int timeout_ms) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  int rc = set_device(h);
  if (rc) return rc;
  rc = stream_sync(h, timeout_ms);
  if (rc) return rc;
  return check_err(h);
}

int olb_tape_reserve(olb_handle h, int nslots) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (nslots < 1) return fail(OLB_EINVAL, "the tape needs at least one slot");
  int rc = set_device(h);
  if (rc) return rc;
  rc = adj_prepare(h);
  if (rc) return rc;
  return tape_grow(h, nslots);
}

int olb_tape_record(olb_handle h, int n) {
  if (!h) return fail(OLB_EINVAL, "null handle");
  if (h->xbc) return fail(OLB_EUNSUPPORTED, "the adjoint is built for periodic grids only");
  if (h->glc) return fail(OLB_EUNSUPPORTED, "the adjoint is built for the uniform-grid interpolation only");
  if (n < 0) return fail(OLB_EINVAL, "negative step count");
  if (n > (int)h->tape.size()) return fail(OLB_EBOUNDS, "tape has fewer than n slots");
  int rc = set_device(h);
  if (rc) return rc;
  rc = adj_prepare(h);
  if (rc) return rc;
  if (h->state_bad) return fail(OLB_ETIMEOUT, "the state is invalid after a wait ran out: set it again");
  // the state advances through the handle's buffers; step s also keeps its
  // pulled populations in slot s - 1
  for (int s = 1; s <= n; ++s) {
    rc = record_step(h, h->buf[h->cur], h->maps.m[h->cur], h->buf[h->cur ^ 1], s - 1);
    if (rc) return rc;
    h->cur ^= 1;
  }
  h->step_count += n;
  h->partials_valid = 0;
  h->tape_len = n + 1;
  return OLB_OK;
}

int olb_tape_adjoint(olb_handle h, void* lambda, int n, int on_device) {
  if (!h || !lambda) return fail(OLB_EINVAL, "null handle or adjoint buffer");
  const int L = h->tape_len - 1;
  if (n < 1 || n > L) return fail(OLB_EBOUNDS, "n must be between 1 and the number of recorded steps");
  int rc = set_device(h);
  if (rc) return rc;
  rc = adj_prepare(h);
  if (rc) return rc;
  std::vector<int> slots;
  for (int k = L; k > L - n; --k) slots.push_back(k - 1);
  const size_t bytes = (size_t)h->Q * h->nnodes * adj_elem(h);
  void* lam = lambda;
  if (!on_device) {
    rc = dev_alloc(h, &lam, bytes);
    if (rc) return rc;
    cudaMemcpyAsync(lam, lambda, bytes, cudaMemcpyHostToDevice, h->stream);
  }
  rc = adjoint_sweep(h, slots, lam);
  if (!on_device) {
    if (rc == OLB_OK) rc = copy_out(h, lambda, lam, bytes, 0);
    cudaFreeAsync(lam, h->stream);
    if (rc == OLB_OK) rc = check_err(h);
  }
  return rc;
}

int olb_adjoint_step(olb_handle h, const void* fwd_state, void* lambda, int on_device) {
  if (!h || !fwd_state || !lambda) return fail(OLB_EINVAL, "null handle, state or adjoint buffer");
  int rc = set_device(h);
  if (rc) return rc;
  rc = adj_prepare(h);
  if (rc) return rc;
  rc = tape_grow(h, 1);
  if (rc) return rc;
  const size_t sbytes = (size_t)h->planes * h->nnodes * h->elem;
  const size_t lbytes = (size_t)h->Q * h->nnodes * adj_elem(h);
  void* tmp = nullptr;
  if (!on_device) {
    rc = dev_alloc(h, &tmp, sbytes + lbytes);
    if (rc) return rc;
    cudaMemcpyAsync(tmp, fwd_state, sbytes, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(static_cast<char*>(tmp) + sbytes, lambda, lbytes, cudaMemcpyHostToDevice, h->stream);
  }
  const void* fs = on_device ? fwd_state : tmp;
  void* lam = on_device ? lambda : static_cast<char*>(tmp) + sbytes;
  // the forward step from fwd_state (in adj[1], ghosts filled by the scatter)
  // into adj[0] records its pulled populations in slot 0; the adjoint
  // buffers are free until the sweep starts
  rc = launch_rc(launch_scatter(h->aux, h->adj[1], fs, h->stream), "adjoint state scatter");
  h->tape_len = 0;  // slot 0 no longer holds a recorded trajectory
  if (rc == OLB_OK) rc = record_step(h, h->adj[1], h->adj_maps.m[1], h->adj[0], 0);
  if (rc == OLB_OK) rc = adjoint_sweep(h, std::vector<int>{0}, lam);
  if (!on_device) {
    if (rc == OLB_OK) rc = copy_out(h, lambda, lam, lbytes, 0);
    cudaFreeAsync(tmp, h->stream);
    if (rc == OLB_OK) rc = check_err(h);
  }
  return rc;
}

int olb_moments_vjp(olb_handle h, const double* grad_rho, const double* grad_u, void* lambda, int on_device) {
  if (!h || !lambda) return fail(OLB_EINVAL, "null handle or adjoint buffer");
  if (h->comp || (h->storage != OLB_FP64 && h->storage != OLB_FP32_SHIFTED))
    return fail(OLB_EUNSUPPORTED, "the adjoint is built for the isothermal step in FP64 and FP32 storage");
  int rc = set_device(h);
  if (rc) return rc;
  const size_t n = (size_t)h->nnodes;
  const size_t lbytes = (size_t)h->Q * n * adj_elem(h);
  const double *gr = grad_rho, *gu = grad_u;
  void* lam = lambda;
  void* tmp = nullptr;
  if (!on_device) {
    rc = dev_alloc(h, &tmp, lbytes + n * (1 + h->D) * sizeof(double));
    if (rc) return rc;
    double* t = reinterpret_cast<double*>(static_cast<char*>(tmp) + lbytes);
    lam = tmp;
    if (grad_rho) cudaMemcpyAsync(t, grad_rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (grad_u) cudaMemcpyAsync(t + n, grad_u, n * h->D * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    gr = grad_rho ? t : nullptr;
    gu = grad_u ? t + n : nullptr;
  }
  rc = launch_rc(launch_moments_vjp(h->aux, h->buf[h->cur], gr, gu, lam, h->stream), "moments_vjp");
  if (!on_device) {
    if (rc == OLB_OK) rc = copy_out(h, lambda, lam, lbytes, 0);
    cudaFreeAsync(tmp, h->stream);
  }
  return rc;
}

int olb_equilibrium_vjp(olb_handle h, const double* rho, const double* u, const void* lambda, double* grad_rho,
                        double* grad_u, int on_device) {
  if (!h || !rho || !u || !lambda || !grad_rho || !grad_u) return fail(OLB_EINVAL, "null argument");
  if (h->comp || (h->storage != OLB_FP64 && h->storage != OLB_FP32_SHIFTED))
    return fail(OLB_EUNSUPPORTED, "the adjoint is built for the isothermal step in FP64 and FP32 storage");
  int rc = set_device(h);
  if (rc) return rc;
  const size_t n = (size_t)h->nnodes;
  const size_t lbytes = (size_t)h->Q * n * adj_elem(h);
  const size_t fbytes = n * (1 + h->D) * sizeof(double);
  if (on_device)
    return launch_rc(launch_equilibrium_vjp(h->aux, rho, u, lambda, grad_rho, grad_u, h->stream), "equilibrium_vjp");
  void* tmp = nullptr;
  rc = dev_alloc(h, &tmp, lbytes + 2 * fbytes);
  if (rc) return rc;
  char* c = static_cast<char*>(tmp);
  double* din = reinterpret_cast<double*>(c + lbytes);
  double* dout = reinterpret_cast<double*>(c + lbytes + fbytes);
  cudaMemcpyAsync(c, lambda, lbytes, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(din, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(din + n, u, n * h->D * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  rc = launch_rc(launch_equilibrium_vjp(h->aux, din, din + n, c, dout, dout + n, h->stream), "equilibrium_vjp");
  if (rc == OLB_OK) {
    cudaMemcpyAsync(grad_rho, dout, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    rc = copy_out(h, grad_u, dout + n, n * h->D * sizeof(double), 0);
  }
  cudaFreeAsync(tmp, h->stream);
  if (rc == OLB_OK) rc = stream_sync(h, 0);
  return rc;
}

const char* olb_strerror(int code) {
  switch (code) {
    case OLB_OK: return "ok";
    case OLB_EINVAL: return "invalid argument";
    case OLB_ENOMEM: return "out of memory";
    case OLB_ECUDA: return "CUDA runtime error";
    case OLB_ENONFINITE: return "non-finite values in the state";
    case OLB_ETIMEOUT: return "timed out";
    case OLB_EBOUNDS: return "size out of bounds";
    case OLB_EUNSUPPORTED: return "unsupported configuration";
    case OLB_ESTATE: return "call out of order";
    default: return "unknown error";
  }
}

const char* olb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
