// Instantiations of the fused step for float storage: the dimensions and
// interpolation degrees that are built.
#include "olb_step.cuh"

namespace olb {

int launch_step_f32(const StepLaunch& L) {
  using S = float;
  if (L.D == 2 && L.P == 2)
    return L.compressible ? launch_one<2, 2, S, true>(L) : launch_one<2, 2, S, false>(L);
  if (L.D == 2 && L.P == 3)
    return L.compressible ? launch_one<2, 3, S, true>(L) : launch_one<2, 3, S, false>(L);
  if (L.D == 2 && L.P == 4)
    return L.compressible ? launch_one<2, 4, S, true>(L) : launch_one<2, 4, S, false>(L);
  if (L.D == 3 && L.P == 2)
    return L.compressible ? launch_one<3, 2, S, true>(L) : launch_one<3, 2, S, false>(L);
  if (L.D == 3 && L.P == 3)
    return L.compressible ? launch_one<3, 3, S, true>(L) : launch_one<3, 3, S, false>(L);
  if (L.D == 3 && L.P == 4)
    return L.compressible ? launch_one<3, 4, S, true>(L) : launch_one<3, 4, S, false>(L);
  return -1;
}

int step_info_f32(int D, int P, int comp, StepInfo* out) {
  using S = float;
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
  return -1;
}

}  // namespace olb
