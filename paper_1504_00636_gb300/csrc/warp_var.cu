// Team-kernel launches with the optional decision variants read at run time
// (normalised split axis, momentum-norm CV); see team.cuh.
#include "team.cuh"

namespace pma {

cudaError_t launch_team_variants(const Problem &P, const UnitSource &U, int mixed, int team,
                                 int cap, int grid, cudaStream_t st) {
  return launch_team_build<true>(P, U, mixed, team, cap, grid, st);
}

}  // namespace pma
