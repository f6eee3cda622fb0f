// Instantiations of the fused step for double storage: the dimensions and
// interpolation degrees that are built.
#include "olb_step.cuh"

namespace olb {

int launch_step_f64(const StepLaunch& L) {
  using S = double;
  if (L.D == 2 && L.P == 1)
    return L.compressible ? launch_one<2, 1, S, true>(L) : launch_one<2, 1, S, false>(L);
  if (L.D == 2 && L.P == 2)
    return L.compressible ? launch_one<2, 2, S, true>(L) : launch_one<2, 2, S, false>(L);
  if (L.D == 2 && L.P == 3)
    return L.compressible ? launch_one<2, 3, S, true>(L) : launch_one<2, 3, S, false>(L);
  if (L.D == 2 && L.P == 4)
    return L.compressible ? launch_one<2, 4, S, true>(L) : launch_one<2, 4, S, false>(L);
  if (L.D == 2 && L.P == 5)
    return L.compressible ? launch_one<2, 5, S, true>(L) : launch_one<2, 5, S, false>(L);
  if (L.D == 2 && L.P == 6)
    return L.compressible ? launch_one<2, 6, S, true>(L) : launch_one<2, 6, S, false>(L);
  if (L.D == 3 && L.P == 1)
    return L.compressible ? launch_one<3, 1, S, true>(L) : launch_one<3, 1, S, false>(L);
  if (L.D == 3 && L.P == 2)
    return L.compressible ? launch_one<3, 2, S, true>(L) : launch_one<3, 2, S, false>(L);
  if (L.D == 3 && L.P == 3)
    return L.compressible ? launch_one<3, 3, S, true>(L) : launch_one<3, 3, S, false>(L);
  if (L.D == 3 && L.P == 4)
    return L.compressible ? launch_one<3, 4, S, true>(L) : launch_one<3, 4, S, false>(L);
  if (L.D == 3 && L.P == 5)
    return L.compressible ? launch_one<3, 5, S, true>(L) : launch_one<3, 5, S, false>(L);
  if (L.D == 3 && L.P == 6)
    return L.compressible ? launch_one<3, 6, S, true>(L) : launch_one<3, 6, S, false>(L);
  return -1;
}

int step_info_f64(int D, int P, int comp, StepInfo* out) {
  using S = double;
  if (D == 2 && P == 1) {
    layout_of<2, 1, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 1, S, true>(&out->smem) : occupancy_one<2, 1, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 2) {
    layout_of<2, 2, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 2, S, true>(&out->smem) : occupancy_one<2, 2, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 3) {
    layout_of<2, 3, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 3, S, true>(&out->smem) : occupancy_one<2, 3, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 4) {
    layout_of<2, 4, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 4, S, true>(&out->smem) : occupancy_one<2, 4, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 5) {
    layout_of<2, 5, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 5, S, true>(&out->smem) : occupancy_one<2, 5, S, false>(&out->smem);
    return 0;
  }
  if (D == 2 && P == 6) {
    layout_of<2, 6, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<2, 6, S, true>(&out->smem) : occupancy_one<2, 6, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 1) {
    layout_of<3, 1, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 1, S, true>(&out->smem) : occupancy_one<3, 1, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 2) {
    layout_of<3, 2, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 2, S, true>(&out->smem) : occupancy_one<3, 2, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 3) {
    layout_of<3, 3, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 3, S, true>(&out->smem) : occupancy_one<3, 3, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 4) {
    layout_of<3, 4, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 4, S, true>(&out->smem) : occupancy_one<3, 4, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 5) {
    layout_of<3, 5, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 5, S, true>(&out->smem) : occupancy_one<3, 5, S, false>(&out->smem);
    return 0;
  }
  if (D == 3 && P == 6) {
    layout_of<3, 6, S>(out);
    out->ctas_per_sm = comp ? occupancy_one<3, 6, S, true>(&out->smem) : occupancy_one<3, 6, S, false>(&out->smem);
    return 0;
  }
  return -1;
}

}  // namespace olb
