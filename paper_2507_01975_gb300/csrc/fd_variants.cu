// fd_variants.cu -- further cluster shapes of the on-chip rollout kernel.
//
// fd_api.cu instantiates one configuration per (type, N): the one that keeps a
// batch's trajectories co-resident with the fewest CTAs each. The shapes here
// split a trajectory's rows over more CTAs (fewer rows per CTA), which puts
// more SMs to work on a small batch at the price of more cluster barriers and
// DSMEM traffic per step. fd_autotune times them against the default and
// keeps the fastest; fd_set_plan selects one by cluster size.
#include <vector>

#include "fd_launch.cuh"

using namespace ldfv;

void fd_extra_launchers(int dtype, int logn, int dord, std::vector<Launcher>& out) {
  if (dtype == FD_F32) {
    switch (logn) {
      case 5:
        out.push_back(make_launcher<float, 5, 2, 256>(dord));
        out.push_back(make_launcher<float, 5, 4, 256>(dord));
        break;
      case 6:
        out.push_back(make_launcher<float, 6, 2, 512>(dord));
        out.push_back(make_launcher<float, 6, 4, 512>(dord));
        break;
      case 7:
        out.push_back(make_launcher<float, 7, 4, 512>(dord));
        out.push_back(make_launcher<float, 7, 8, 512>(dord));
        break;
      default:
        break;
    }
  } else {
    switch (logn) {
      case 5:
        out.push_back(make_launcher<double, 5, 2, 256>(dord));
        out.push_back(make_launcher<double, 5, 4, 256>(dord));
        break;
      default:
        break;
    }
  }
}
