// Instantiations of the fused step for __half storage.  The two-phase kernel
// (olb_wg.cuh) is built for p = 3, 4 and runs unless the single-role kernel
// (olb_step.cuh, built for p = 2, 3, 4) is asked for or is the only one built.
#include "olb_wg.cuh"

namespace olb {

int launch_step_f16(const StepLaunch& L) {
  using S = __half;
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
    if (L.D == 3 && L.P == 3 && L.compressible == 0) {
      if (L.a.Q <= 27) return wg::launch_wg<3, 3, S, false, 27>(L);
      return wg::launch_wg<3, 3, S, false, 45>(L);
    }
    if (L.D == 3 && L.P == 3 && L.compressible == 1) {
      return wg::launch_wg<3, 3, S, true, 45>(L);
    }
    if (L.D == 3 && L.P == 4 && L.compressible == 0) {
      if (L.a.Q <= 27) return wg::launch_wg<3, 4, S, false, 27>(L);
      return wg::launch_wg<3, 4, S, false, 45>(L);
    }
    if (L.D == 3 && L.P == 4 && L.compressible == 1) {
      return wg::launch_wg<3, 4, S, true, 45>(L);
    }
  }
  if (L.D == 2 && L.P == 2 && L.compressible == 0) return launch_one<2, 2, S, false>(L);
  if (L.D == 2 && L.P == 2 && L.compressible == 1) return launch_one<2, 2, S, true>(L);
  if (L.D == 2 && L.P == 3 && L.compressible == 0) return launch_one<2, 3, S, false>(L);
  if (L.D == 2 && L.P == 3 && L.compressible == 1) return launch_one<2, 3, S, true>(L);
  if (L.D == 2 && L.P == 4 && L.compressible == 0) return launch_one<2, 4, S, false>(L);
  if (L.D == 2 && L.P == 4 && L.compressible == 1) return launch_one<2, 4, S, true>(L);
  if (L.D == 3 && L.P == 2 && L.compressible == 0) return launch_one<3, 2, S, false>(L);
  if (L.D == 3 && L.P == 2 && L.compressible == 1) return launch_one<3, 2, S, true>(L);
  if (L.D == 3 && L.P == 3 && L.compressible == 0) return launch_one<3, 3, S, false>(L);
  if (L.D == 3 && L.P == 3 && L.compressible == 1) return launch_one<3, 3, S, true>(L);
  if (L.D == 3 && L.P == 4 && L.compressible == 0) return launch_one<3, 4, S, false>(L);
  if (L.D == 3 && L.P == 4 && L.compressible == 1) return launch_one<3, 4, S, true>(L);
  return -1;
}

int step_info_f16(int D, int P, int comp, int Q, int force_generic, StepInfo* out) {
  using S = __half;
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
  if (D == 3 && P == 2) {
    layout_of<3, 2, S>(out);
    out->wg = 0;
    out->ctas_per_sm = comp ? occupancy_one<3, 2, S, true>(&out->smem) : occupancy_one<3, 2, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 3) {
    layout_of<3, 3, S>(out);
    out->wg = 0;
    if (!force_generic) {
      int nwg = 0;
      out->ctas_per_sm = comp ? wg::occupancy_wg<3, 3, S, true, 45>(&out->smem, &nwg) : (Q <= 27 ? wg::occupancy_wg<3, 3, S, false, 27>(&out->smem, &nwg) : wg::occupancy_wg<3, 3, S, false, 45>(&out->smem, &nwg));
      out->wg = nwg;
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<3, 3, S, true>(&out->smem) : occupancy_one<3, 3, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 4) {
    layout_of<3, 4, S>(out);
    out->wg = 0;
    if (!force_generic) {
      int nwg = 0;
      out->ctas_per_sm = comp ? wg::occupancy_wg<3, 4, S, true, 45>(&out->smem, &nwg) : (Q <= 27 ? wg::occupancy_wg<3, 4, S, false, 27>(&out->smem, &nwg) : wg::occupancy_wg<3, 4, S, false, 45>(&out->smem, &nwg));
      out->wg = nwg;
      return 0;
    }
    out->ctas_per_sm = comp ? occupancy_one<3, 4, S, true>(&out->smem) : occupancy_one<3, 4, S, false>(&out->smem);
    return 0;
  }
  return -1;
}

}  // namespace olb
