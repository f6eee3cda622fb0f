// Instantiations of the fused step, float storage, D = 3; written by gen_step_instances.py.
#include "olb_wg.cuh"

namespace olb {

namespace {
using S = float;

// Two-phase instance for (P, comp, Q, N): its launch and shape, or null.
using WgLaunch = int (*)(const StepLaunch&);
using WgOcc = int (*)(StepInfo*);
bool pick_wg(int P, int comp, int Q, int N, WgLaunch* l, WgOcc* o) {
  if (P == 3 && comp == 0 && N == 2 && Q <= 27) {
    *l = wg::launch_wg<3, 3, S, false, 27, 2>;
    *o = wg::occupancy_wg<3, 3, S, false, 27, 2>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 3 && Q <= 27) {
    *l = wg::launch_wg<3, 3, S, false, 27, 3>;
    *o = wg::occupancy_wg<3, 3, S, false, 27, 3>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 2 && true) {
    *l = wg::launch_wg<3, 3, S, false, 45, 2>;
    *o = wg::occupancy_wg<3, 3, S, false, 45, 2>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 3 && true) {
    *l = wg::launch_wg<3, 3, S, false, 45, 3>;
    *o = wg::occupancy_wg<3, 3, S, false, 45, 3>;
    return true;
  }
  if (P == 3 && comp == 1 && N == 4 && true) {
    *l = wg::launch_wg<3, 3, S, true, 45, 4>;
    *o = wg::occupancy_wg<3, 3, S, true, 45, 4>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 2 && Q <= 27) {
    *l = wg::launch_wg<3, 4, S, false, 27, 2>;
    *o = wg::occupancy_wg<3, 4, S, false, 27, 2>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 3 && Q <= 27) {
    *l = wg::launch_wg<3, 4, S, false, 27, 3>;
    *o = wg::occupancy_wg<3, 4, S, false, 27, 3>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 2 && true) {
    *l = wg::launch_wg<3, 4, S, false, 45, 2>;
    *o = wg::occupancy_wg<3, 4, S, false, 45, 2>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 3 && true) {
    *l = wg::launch_wg<3, 4, S, false, 45, 3>;
    *o = wg::occupancy_wg<3, 4, S, false, 45, 3>;
    return true;
  }
  if (P == 4 && comp == 1 && N == 4 && true) {
    *l = wg::launch_wg<3, 4, S, true, 45, 4>;
    *o = wg::occupancy_wg<3, 4, S, true, 45, 4>;
    return true;
  }
  return false;
}
}  // namespace

int launch_step_f32_3d(const StepLaunch& L) {
  WgLaunch l;
  WgOcc o;
  if (L.force_generic != 1 && pick_wg(L.P, L.compressible, L.a.Q, L.a.N, &l, &o)) return l(L);
  if (L.P == 2 && L.compressible == 0) return launch_one<3, 2, S, false>(L);
  if (L.P == 2 && L.compressible == 1) return launch_one<3, 2, S, true>(L);
  if (L.P == 3 && L.compressible == 0) return launch_one<3, 3, S, false>(L);
  if (L.P == 3 && L.compressible == 1) return launch_one<3, 3, S, true>(L);
  if (L.P == 4 && L.compressible == 0) return launch_one<3, 4, S, false>(L);
  if (L.P == 4 && L.compressible == 1) return launch_one<3, 4, S, true>(L);
  return -1;
}

int step_info_f32_3d(int P, int comp, int Q, int N, int force_generic, StepInfo* out) {
  WgLaunch l;
  WgOcc o;
  out->wg = 0;
  if (P == 2) {
    layout_of<3, 2, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 2, S, true>(&out->smem)
                            : occupancy_one<3, 2, S, false>(&out->smem);
    return 0;
  }
  if (P == 3) {
    layout_of<3, 3, S>(out);
    if (force_generic != 1 && pick_wg(P, comp, Q, N, &l, &o)) {
      out->ctas_per_sm = o(out);  // the two-phase kernel's own tile and shape
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<3, 3, S, true>(&out->smem)
                            : occupancy_one<3, 3, S, false>(&out->smem);
    return 0;
  }
  if (P == 4) {
    layout_of<3, 4, S>(out);
    if (force_generic != 1 && pick_wg(P, comp, Q, N, &l, &o)) {
      out->ctas_per_sm = o(out);  // the two-phase kernel's own tile and shape
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<3, 4, S, true>(&out->smem)
                            : occupancy_one<3, 4, S, false>(&out->smem);
    return 0;
  }
  return -1;
}

int launch_adj_f32_3d(const StepLaunch& L) {
  if (L.P == 3 && L.a.N == 2 && L.a.Q <= 27) return wg::launch_adj<3, 3, S, 27, 2>(L);
  if (L.P == 3 && L.a.N == 3 && L.a.Q <= 27) return wg::launch_adj<3, 3, S, 27, 3>(L);
  if (L.P == 3 && L.a.N == 2) return wg::launch_adj<3, 3, S, 45, 2>(L);
  if (L.P == 4 && L.a.N == 2 && L.a.Q <= 27) return wg::launch_adj<3, 4, S, 27, 2>(L);
  if (L.P == 4 && L.a.N == 3 && L.a.Q <= 27) return wg::launch_adj<3, 4, S, 27, 3>(L);
  if (L.P == 4 && L.a.N == 2) return wg::launch_adj<3, 4, S, 45, 2>(L);
  return -1;
}

}  // namespace olb
