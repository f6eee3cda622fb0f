// Instantiations of the fused step, double storage, D = 2; written by gen_step_instances.py.
#include "olb_wg.cuh"

namespace olb {

namespace {
using S = double;

// Two-phase instance for (P, comp, Q, N): its launch and shape, or null.
using WgLaunch = int (*)(const StepLaunch&);
using WgOcc = int (*)(StepInfo*);
bool pick_wg(int P, int comp, int Q, int N, WgLaunch* l, WgOcc* o) {
  if (P == 3 && comp == 0 && N == 2 && Q <= 9) {
    *l = wg::launch_wg<2, 3, S, false, 9, 2>;
    *o = wg::occupancy_wg<2, 3, S, false, 9, 2>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 3 && Q <= 9) {
    *l = wg::launch_wg<2, 3, S, false, 9, 3>;
    *o = wg::occupancy_wg<2, 3, S, false, 9, 3>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 2 && true) {
    *l = wg::launch_wg<2, 3, S, false, 27, 2>;
    *o = wg::occupancy_wg<2, 3, S, false, 27, 2>;
    return true;
  }
  if (P == 3 && comp == 0 && N == 3 && true) {
    *l = wg::launch_wg<2, 3, S, false, 27, 3>;
    *o = wg::occupancy_wg<2, 3, S, false, 27, 3>;
    return true;
  }
  if (P == 3 && comp == 1 && N == 4 && true) {
    *l = wg::launch_wg<2, 3, S, true, 27, 4>;
    *o = wg::occupancy_wg<2, 3, S, true, 27, 4>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 2 && Q <= 9) {
    *l = wg::launch_wg<2, 4, S, false, 9, 2>;
    *o = wg::occupancy_wg<2, 4, S, false, 9, 2>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 3 && Q <= 9) {
    *l = wg::launch_wg<2, 4, S, false, 9, 3>;
    *o = wg::occupancy_wg<2, 4, S, false, 9, 3>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 2 && true) {
    *l = wg::launch_wg<2, 4, S, false, 27, 2>;
    *o = wg::occupancy_wg<2, 4, S, false, 27, 2>;
    return true;
  }
  if (P == 4 && comp == 0 && N == 3 && true) {
    *l = wg::launch_wg<2, 4, S, false, 27, 3>;
    *o = wg::occupancy_wg<2, 4, S, false, 27, 3>;
    return true;
  }
  if (P == 4 && comp == 1 && N == 4 && true) {
    *l = wg::launch_wg<2, 4, S, true, 27, 4>;
    *o = wg::occupancy_wg<2, 4, S, true, 27, 4>;
    return true;
  }
  return false;
}
}  // namespace

int launch_step_f64_2d(const StepLaunch& L) {
  WgLaunch l;
  WgOcc o;
  if (L.force_generic != 1 && pick_wg(L.P, L.compressible, L.a.Q, L.a.N, &l, &o)) return l(L);
  if (L.P == 1 && L.compressible == 0) return launch_one<2, 1, S, false>(L);
  if (L.P == 1 && L.compressible == 1) return launch_one<2, 1, S, true>(L);
  if (L.P == 2 && L.compressible == 0) return launch_one<2, 2, S, false>(L);
  if (L.P == 2 && L.compressible == 1) return launch_one<2, 2, S, true>(L);
  if (L.P == 3 && L.compressible == 0) return launch_one<2, 3, S, false>(L);
  if (L.P == 3 && L.compressible == 1) return launch_one<2, 3, S, true>(L);
  if (L.P == 4 && L.compressible == 0) return launch_one<2, 4, S, false>(L);
  if (L.P == 4 && L.compressible == 1) return launch_one<2, 4, S, true>(L);
  if (L.P == 5 && L.compressible == 0) return launch_one<2, 5, S, false>(L);
  if (L.P == 5 && L.compressible == 1) return launch_one<2, 5, S, true>(L);
  if (L.P == 6 && L.compressible == 0) return launch_one<2, 6, S, false>(L);
  if (L.P == 6 && L.compressible == 1) return launch_one<2, 6, S, true>(L);
  return -1;
}

int step_info_f64_2d(int P, int comp, int Q, int N, int force_generic, StepInfo* out) {
  WgLaunch l;
  WgOcc o;
  out->wg = 0;
  if (P == 1) {
    layout_of<2, 1, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 1, S, true>(&out->smem)
                            : occupancy_one<2, 1, S, false>(&out->smem);
    return 0;
  }
  if (P == 2) {
    layout_of<2, 2, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 2, S, true>(&out->smem)
                            : occupancy_one<2, 2, S, false>(&out->smem);
    return 0;
  }
  if (P == 3) {
    layout_of<2, 3, S>(out);
    if (force_generic != 1 && pick_wg(P, comp, Q, N, &l, &o)) {
      out->ctas_per_sm = o(out);  // the two-phase kernel's own tile and shape
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<2, 3, S, true>(&out->smem)
                            : occupancy_one<2, 3, S, false>(&out->smem);
    return 0;
  }
  if (P == 4) {
    layout_of<2, 4, S>(out);
    if (force_generic != 1 && pick_wg(P, comp, Q, N, &l, &o)) {
      out->ctas_per_sm = o(out);  // the two-phase kernel's own tile and shape
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<2, 4, S, true>(&out->smem)
                            : occupancy_one<2, 4, S, false>(&out->smem);
    return 0;
  }
  if (P == 5) {
    layout_of<2, 5, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 5, S, true>(&out->smem)
                            : occupancy_one<2, 5, S, false>(&out->smem);
    return 0;
  }
  if (P == 6) {
    layout_of<2, 6, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 6, S, true>(&out->smem)
                            : occupancy_one<2, 6, S, false>(&out->smem);
    return 0;
  }
  return -1;
}

int launch_adj_f64_2d(const StepLaunch& L) {
  if (L.P == 3 && L.a.N == 2 && L.a.Q <= 9) return wg::launch_adj<2, 3, S, 9, 2>(L);
  if (L.P == 3 && L.a.N == 2) return wg::launch_adj<2, 3, S, 27, 2>(L);
  if (L.P == 3 && L.a.N == 3) return wg::launch_adj<2, 3, S, 27, 3>(L);
  if (L.P == 4 && L.a.N == 2 && L.a.Q <= 9) return wg::launch_adj<2, 4, S, 9, 2>(L);
  if (L.P == 4 && L.a.N == 2) return wg::launch_adj<2, 4, S, 27, 2>(L);
  if (L.P == 4 && L.a.N == 3) return wg::launch_adj<2, 4, S, 27, 3>(L);
  return -1;
}

}  // namespace olb
