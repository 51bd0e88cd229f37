// Fusion planner interface (host, FP64).
#pragma once

#include <vector>

#include "internal.h"

namespace qsim {

struct Block {
  std::vector<int> q;      // logical qubits; q[0] is the most significant matrix-index bit
  std::vector<cd> u;       // 2^|q| x 2^|q| row-major, composed in FP64
  std::vector<int> gates;  // indices of the gates it absorbed, ascending
};

// Matrix of gate g (targets and controls) on the index space of qubit list q.
void embed_gate(const Gate &g, const std::vector<int> &q, std::vector<cd> &out);
// Left-multiply block b by gate g, extending b's qubit list as needed.
void absorb(Block &b, const Gate &g, int gate_index);
// Greedy fusion into blocks of at most k qubits (a single gate wider than k stays alone).
std::vector<Block> plan_fusion(const std::vector<Gate> &gates, int k);
// Matrix over `from` re-indexed onto the superset `to` (identity on the extra qubits).
std::vector<cd> reindex(const std::vector<cd> &u, const std::vector<int> &from,
                        const std::vector<int> &to);

}  // namespace qsim
