// ordering.h — fill-reducing orderings from the pattern alone (internal to the library).
#pragma once

#include <cstdint>
#include <vector>

namespace sym {

// Adjacency (both directions, no diagonal) of the symmetric pattern given by its lower CSC.
void pattern_graph(int64_t n, const int64_t *Ap, const int32_t *Ai, std::vector<int64_t> &xadj,
                   std::vector<int32_t> &adj);

// perm[k] = the node placed at position k.
void order_min_degree(int64_t n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj,
                      std::vector<int32_t> &perm);
void order_nested_dissection(int64_t n, const std::vector<int64_t> &xadj, const std::vector<int32_t> &adj,
                             std::vector<int32_t> &perm);

}  // namespace sym
