// Instantiations of the fused step for double storage.  The two-phase kernel
// (olb_wg.cuh) is built for p = 3, 4 and runs unless the single-role kernel
// (olb_step.cuh, built for p = 1, 2, 3, 4, 5, 6) is asked for or is the only one built.
#include "olb_wg.cuh"

namespace olb {

int launch_step_f64_2d(const StepLaunch& L) {
  using S = double;
  if (!L.force_generic) {
    if (L.D == 2 && L.P == 3 && L.compressible == 0) {
      if (L.a.Q <= 9) return wg::launch_wg<2, 3, S, false, 9>(L);
      return wg::launch_wg<2, 3, S, false, 27>(L);
    }
    if (L.D == 2 && L.P == 3 && L.compressible == 1) {
      return wg::launch_wg<2, 3, S, true, 27>(L);
    }
    if (L.D == 2 && L.P == 4 && L.compressible == 0) {
      if (L.a.Q <= 9) return wg::launch_wg<2, 4, S, false, 9>(L);
      return wg::launch_wg<2, 4, S, false, 27>(L);
    }
    if (L.D == 2 && L.P == 4 && L.compressible == 1) {
      return wg::launch_wg<2, 4, S, true, 27>(L);
    }
  }
  if (L.D == 2 && L.P == 1 && L.compressible == 0) return launch_one<2, 1, S, false>(L);
  if (L.D == 2 && L.P == 1 && L.compressible == 1) return launch_one<2, 1, S, true>(L);
  if (L.D == 2 && L.P == 2 && L.compressible == 0) return launch_one<2, 2, S, false>(L);
  if (L.D == 2 && L.P == 2 && L.compressible == 1) return launch_one<2, 2, S, true>(L);
  if (L.D == 2 && L.P == 3 && L.compressible == 0) return launch_one<2, 3, S, false>(L);
  if (L.D == 2 && L.P == 3 && L.compressible == 1) return launch_one<2, 3, S, true>(L);
  if (L.D == 2 && L.P == 4 && L.compressible == 0) return launch_one<2, 4, S, false>(L);
  if (L.D == 2 && L.P == 4 && L.compressible == 1) return launch_one<2, 4, S, true>(L);
  if (L.D == 2 && L.P == 5 && L.compressible == 0) return launch_one<2, 5, S, false>(L);
  if (L.D == 2 && L.P == 5 && L.compressible == 1) return launch_one<2, 5, S, true>(L);
  if (L.D == 2 && L.P == 6 && L.compressible == 0) return launch_one<2, 6, S, false>(L);
  if (L.D == 2 && L.P == 6 && L.compressible == 1) return launch_one<2, 6, S, true>(L);
  return -1;
}

int step_info_f64_2d(int D, int P, int comp, int Q, int force_generic, StepInfo* out) {
  using S = double;
  if (D == 2 && P == 1) {
    layout_of<2, 1, S>(out);
    out->wg = 0;
    out->ctas_per_sm = comp ? occupancy_one<2, 1, S, true>(&out->smem) : occupancy_one<2, 1, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 2) {
    layout_of<2, 2, S>(out);
    out->wg = 0;
    out->ctas_per_sm = comp ? occupancy_one<2, 2, S, true>(&out->smem) : occupancy_one<2, 2, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 3) {
    layout_of<2, 3, S>(out);
    out->wg = 0;
    if (!force_generic) {
      int nwg = 0;
      out->ctas_per_sm = comp ? wg::occupancy_wg<2, 3, S, true, 27>(&out->smem, &nwg) : (Q <= 9 ? wg::occupancy_wg<2, 3, S, false, 9>(&out->smem, &nwg) : wg::occupancy_wg<2, 3, S, false, 27>(&out->smem, &nwg));
      out->wg = nwg;
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<2, 3, S, true>(&out->smem) : occupancy_one<2, 3, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 4) {
    layout_of<2, 4, S>(out);
    out->wg = 0;
    if (!force_generic) {
      int nwg = 0;
      out->ctas_per_sm = comp ? wg::occupancy_wg<2, 4, S, true, 27>(&out->smem, &nwg) : (Q <= 9 ? wg::occupancy_wg<2, 4, S, false, 9>(&out->smem, &nwg) : wg::occupancy_wg<2, 4, S, false, 27>(&out->smem, &nwg));
      out->wg = nwg;
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<2, 4, S, true>(&out->smem) : occupancy_one<2, 4, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 5) {
    layout_of<2, 5, S>(out);
    out->wg = 0;
    out->ctas_per_sm = comp ? occupancy_one<2, 5, S, true>(&out->smem) : occupancy_one<2, 5, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 6) {
    layout_of<2, 6, S>(out);
    out->wg = 0;
    out->ctas_per_sm = comp ? occupancy_one<2, 6, S, true>(&out->smem) : occupancy_one<2, 6, S, false>(&out->smem);
    return 0;
  }
  return -1;
}

}  // namespace olb
