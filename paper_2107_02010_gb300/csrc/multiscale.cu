// Coarse-to-fine strategy of Section 2 (placeholder until the cluster-pair
// truncation lands): clustering, coarse solve, extrapolation, truncation.
#include "multiscale.cuh"
#include "prims.cuh"
#include "solver.cuh"

namespace otgb {

void Multiscale::cluster(Solver &, const otgb_params &, const float *, const float *, const float *, const float *,
                         const std::vector<float> &, const std::vector<float> &, const std::vector<float> &,
                         const std::vector<float> &, float *) {
    throw Error{OTGB_EINVAL, "multiscale solve not available in this build"};
}
int Multiscale::run_schedule(Solver &, const otgb_params &, const std::vector<double> &, int) { return OTGB_EINTERNAL; }
void Multiscale::before_fine_step(Solver &, double) {}

}  // namespace otgb
