// reach.h — pruned forward solve for a sparse right-hand side (internal).
#pragma once

#include <string>
#include <vector>

#include "plan.h"

namespace sym {

struct Reach {
  std::vector<int32_t> pbeta;   // nonzeros of b, permuted numbering, in the caller's order
  std::vector<int32_t> cols;    // Reach_L(beta), permuted numbering, increasing (topological)
  std::vector<int32_t> snodes;  // supernodes that hold reached columns, increasing
  std::vector<UpdTask> upd_tasks;     // pruned gather tasks (entries of reached descendants only)
  std::vector<UpdEntry> upd_entries;
  std::vector<Int4> tasks;      // S_FGATHER and S_FSTEP tasks of the pruned schedule
  std::vector<Launch> fwd;      // pruned forward launch schedule
};

// Reach set of beta (caller's numbering, nb distinct indices) and the pruned schedule.
int build_reach(const Plan &P, int64_t nb, const int32_t *beta, Reach &R, std::string &err);

}  // namespace sym
