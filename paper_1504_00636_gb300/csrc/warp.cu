// Team-kernel launches with the paper's decision rule (Sec. 3, Steps 3-4 as
// printed), and the dispatch to the build with the optional variants.
#include "team.cuh"

namespace pma {

// shared memory of one CTA (one team, one unit of up to cap particles)
size_t team_smem(int mixed, int D, int cap) {
  return mixed ? team_smem_t<float>(D, cap) : team_smem_t<double>(D, cap);
}

// mode: 0 small-class cells, 1 large-class cells, 2 pieces of big cells
int team_blocks(int mixed, int D, int team, int cap, int smem_optin) {
  if (team == 12)
    return mixed ? team_blocks_d<float, 12>(D, cap, smem_optin)
                 : team_blocks_d<double, 12>(D, cap, smem_optin);
  if (team == 8)
    return mixed ? team_blocks_d<float, 8>(D, cap, smem_optin)
                 : team_blocks_d<double, 8>(D, cap, smem_optin);
  return 1;
}

cudaError_t launch_team(const Problem &P, int mixed, int mode, int team, int cap, int grid,
                        cudaStream_t st) {
  UnitSource U;
  U.mode = mode;
  if (mode == 0) {
    U.list = P.warp_list;
    U.count = P.warp_count;
    U.next = P.warp_next;
  } else if (mode == 3) {
    U.list = P.tiny_list;
    U.count = P.tiny_count;
    U.next = P.tiny_next;
  } else if (mode == 1) {
    U.list = P.block_list;
    U.count = P.block_count;
    U.next = P.unit_next;
  } else {
    U.list = nullptr;
    U.count = P.piece_count;
    U.next = P.unit_next + 1;
  }
  if (P.variant != 0) return launch_team_variants(P, U, mixed, team, cap, grid, st);
  return launch_team_build<false>(P, U, mixed, team, cap, grid, st);
}

}  // namespace pma
