// Fusion planner interface (host, FP64).
#pragma once

#include <vector>

#include "internal.h"

namespace qsim {

struct Block {
  std::vector<int> q;       // logical qubits; q[0] is the most significant matrix-index bit
  std::vector<cd> u;        // 2^|q| x 2^|q| row-major, composed in FP64 (compose_block)
  std::vector<int> gates;   // indices of the gates it holds, ascending
  std::vector<int> phases;  // diagonal gates on qubits outside q, applied as row phases
};

// A diagonal unitary gate on at most kMaxPhaseQubits qubits (targets and controls): it can
// run as a phase that depends only on those qubits' bits.
constexpr int kMaxPhaseQubits = 3;
bool is_phase_gate(const Gate &g);

// Matrix of gate g (targets and controls) on the index space of qubit list q.
void embed_gate(const Gate &g, const std::vector<int> &q, std::vector<cd> &out);
// b.u = product of b's gates (in list order) on the index space of b.q.
void compose_block(Block &b, const std::vector<Gate> &gates);
// compose_block for every block with wanted[i] set (all when wanted is empty), in parallel.
void compose_blocks(std::vector<Block> &blocks, const std::vector<Gate> &gates,
                    const std::vector<char> &wanted);
// Sequential grouping into blocks of at most k qubits (a gate wider than k stays alone).
std::vector<Block> plan_fusion(const std::vector<Gate> &gates, int k);
// Front-greedy grouping over k-qubit candidate sets of an n-qubit register; a block that
// brings in more than fresh_limit qubits the previous block did not hold is penalised.
// With max_phases > 0 a block also takes up to that many ready phase gates whose qubits
// are all outside its set (Block::phases).
std::vector<Block> plan_fusion_front(const std::vector<Gate> &gates, int k, int n, int fresh_limit,
                                     int max_phases);
// Matrix over `from` re-indexed onto the superset `to` (identity on the extra qubits).
std::vector<cd> reindex(const std::vector<cd> &u, const std::vector<int> &from,
                        const std::vector<int> &to);

}  // namespace qsim
