// Gate-fusion planner: groups gates into blocks of at most k qubits, then composes each
// block's 2^|q| x 2^|q| unitary in FP64.
//
// Two grouping strategies produce dependency-valid block lists (a block comes before any
// later block that shares a qubit with it, and a block's gates keep their relative order):
//
//  * plan_fusion - one pass over the gate list with several open blocks on disjoint qubit
//    sets. A gate whose qubits, together with every open block it touches, fit in k
//    qubits joins them (blocks on disjoint qubits commute, so merging them is exact);
//    otherwise the touched blocks are closed and the gate opens a new block.
//  * plan_fusion_front - repeatedly picks, among candidate k-qubit sets, the one that
//    absorbs the most gates from the front of the remaining list. Optionally a block also
//    takes ready diagonal gates that act only on qubits outside its set: they commute with
//    the block's unitary (disjoint qubits) and the fused kernel applies them as a phase
//    that depends on the row index alone.
//
// Grouping carries no matrices; compose_blocks builds them afterwards for the chosen plan
// only, in parallel over blocks.
#include <algorithm>
#include <thread>

#include "internal.h"
#include "planner.h"

namespace qsim {

namespace {

int index_of(const std::vector<int> &q, int x) {
  for (size_t i = 0; i < q.size(); ++i)
    if (q[i] == x) return (int)i;
  return -1;
}

unsigned long long qubit_mask(const Gate &g) {
  unsigned long long m = 0;
  for (int j = 0; j < g.nt; ++j) m |= 1ULL << g.t[j];
  for (int c : g.ctrl) m |= 1ULL << c;
  return m;
}

// Add gate gi to block b: its new qubits go to the end of b.q (less significant bits).
void add_to_group(Block &b, const Gate &g, int gi) {
  for (int j = 0; j < g.nt; ++j)
    if (index_of(b.q, g.t[j]) < 0) b.q.push_back(g.t[j]);
  for (int c : g.ctrl)
    if (index_of(b.q, c) < 0) b.q.push_back(c);
  b.gates.push_back(gi);
}

// Union of two groups on disjoint qubits; the gate list stays ascending.
Block merge_groups(const Block &a, const Block &b) {
  Block r;
  r.q = a.q;
  r.q.insert(r.q.end(), b.q.begin(), b.q.end());
  r.gates.resize(a.gates.size() + b.gates.size());
  std::merge(a.gates.begin(), a.gates.end(), b.gates.begin(), b.gates.end(), r.gates.begin());
  return r;
}

bool is_diagonal(const Gate &g) {
  const int gd = 1 << g.nt;
  for (int r = 0; r < gd; ++r)
    for (int c = 0; c < gd; ++c)
      if (r != c && g.m[(size_t)r * gd + c] != 0.0) return false;
  return true;
}

// u <- G u, G the embedding of gate g on the index space of qubit list q (q[0] = MSB):
// every column of u is a |q|-qubit vector that the gate updates in place.
void left_apply(std::vector<cd> &u, const std::vector<int> &q, const Gate &g) {
  const int kb = (int)q.size(), d = 1 << kb, gd = 1 << g.nt;
  int tpos[QSIM_MAX_FUSED];
  int tmask = 0, cmask = 0;
  for (int j = 0; j < g.nt; ++j) {
    tpos[j] = kb - 1 - index_of(q, g.t[j]);
    tmask |= 1 << tpos[j];
  }
  for (int c : g.ctrl) cmask |= 1 << (kb - 1 - index_of(q, c));
  auto gate_index = [&](int r) {  // target bits of row r as a gate-matrix index
    int a = 0;
    for (int j = 0; j < g.nt; ++j) a |= ((r >> tpos[j]) & 1) << (g.nt - 1 - j);
    return a;
  };
  if (is_diagonal(g)) {
    for (int r = 0; r < d; ++r) {
      if ((r & cmask) != cmask) continue;
      const int a = gate_index(r);
      const cd f = g.m[(size_t)a * gd + a];
      if (f == 1.0) continue;
      cd *row = &u[(size_t)r * d];
      for (int c = 0; c < d; ++c) row[c] *= f;
    }
    return;
  }
  int rows[1 << QSIM_MAX_FUSED];
  cd in[1 << QSIM_MAX_FUSED];
  for (int r0 = 0; r0 < d; ++r0) {
    if ((r0 & tmask) || (r0 & cmask) != cmask) continue;
    for (int a = 0; a < gd; ++a) {
      int r = r0;
      for (int j = 0; j < g.nt; ++j)
        if ((a >> (g.nt - 1 - j)) & 1) r |= 1 << tpos[j];
      rows[a] = r;
    }
    for (int c = 0; c < d; ++c) {
      for (int a = 0; a < gd; ++a) in[a] = u[(size_t)rows[a] * d + c];
      for (int a2 = 0; a2 < gd; ++a2) {
        cd acc = 0.0;
        for (int a = 0; a < gd; ++a) acc += g.m[(size_t)a2 * gd + a] * in[a];
        u[(size_t)rows[a2] * d + c] = acc;
      }
    }
  }
}

bool unit_modulus(cd v) { return std::abs(std::abs(v) - 1.0) <= 1e-12; }

constexpr size_t kScanLimit = 1 << 14;  // gates examined per candidate set and block
constexpr int kFreshPenalty = 4;        // price, in gates, of a set needing a stand-alone remap

}  // namespace

bool is_phase_gate(const Gate &g) {
  if (g.nt + (int)g.ctrl.size() > kMaxPhaseQubits || !is_diagonal(g)) return false;
  const int gd = 1 << g.nt;
  for (int a = 0; a < gd; ++a)
    if (!unit_modulus(g.m[(size_t)a * gd + a])) return false;
  return true;
}

void embed_gate(const Gate &g, const std::vector<int> &q, std::vector<cd> &out) {
  const int d = 1 << q.size();
  out.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) out[(size_t)i * d + i] = 1.0;
  left_apply(out, q, g);
}

void compose_block(Block &b, const std::vector<Gate> &gates) {
  const int d = 1 << b.q.size();
  b.u.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) b.u[(size_t)i * d + i] = 1.0;
  for (int gi : b.gates) left_apply(b.u, b.q, gates[gi]);
}

void compose_blocks(std::vector<Block> &blocks, const std::vector<Gate> &gates,
                    const std::vector<char> &wanted) {
  std::vector<size_t> todo;
  size_t work = 0;
  for (size_t i = 0; i < blocks.size(); ++i)
    if (wanted.empty() || wanted[i]) {
      todo.push_back(i);
      work += blocks[i].gates.size() << (2 * blocks[i].q.size());
    }
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  nt = std::min<unsigned>(nt, 16);
  // thread start-up costs tens of microseconds: stay serial for small plans
  if (work < (1u << 20)) nt = 1;
  nt = std::min<unsigned>(nt, (unsigned)std::max<size_t>(1, todo.size()));
  if (nt <= 1) {
    for (size_t i : todo) compose_block(blocks[i], gates);
    return;
  }
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; ++t)
    pool.emplace_back([&, t]() {
      for (size_t j = t; j < todo.size(); j += nt) compose_block(blocks[todo[j]], gates);
    });
  for (auto &th : pool) th.join();
}

std::vector<Block> plan_fusion(const std::vector<Gate> &gates, int k) {
  std::vector<Block> out;
  std::vector<Block> open;
  std::vector<int> owner(64, -1);
  auto rebuild_owner = [&]() {
    std::fill(owner.begin(), owner.end(), -1);
    for (size_t i = 0; i < open.size(); ++i)
      for (int x : open[i].q) owner[x] = (int)i;
  };
  for (size_t gi = 0; gi < gates.size(); ++gi) {
    const Gate &g = gates[gi];
    std::vector<int> gq(g.t, g.t + g.nt);
    gq.insert(gq.end(), g.ctrl.begin(), g.ctrl.end());
    std::vector<int> touched;
    for (int x : gq)
      if (owner[x] >= 0 && std::find(touched.begin(), touched.end(), owner[x]) == touched.end())
        touched.push_back(owner[x]);
    std::sort(touched.begin(), touched.end());
    std::vector<int> uni = gq;
    for (int b : touched)
      for (int x : open[b].q)
        if (std::find(uni.begin(), uni.end(), x) == uni.end()) uni.push_back(x);
    if ((int)uni.size() <= k) {
      Block merged;
      if (!touched.empty()) {
        merged = open[touched[0]];
        for (size_t j = 1; j < touched.size(); ++j) merged = merge_groups(merged, open[touched[j]]);
      }
      add_to_group(merged, g, (int)gi);
      for (int j = (int)touched.size() - 1; j >= 0; --j) open.erase(open.begin() + touched[j]);
      open.push_back(std::move(merged));
    } else {
      for (int b : touched) out.push_back(open[b]);
      for (int j = (int)touched.size() - 1; j >= 0; --j) open.erase(open.begin() + touched[j]);
      Block nb;
      add_to_group(nb, g, (int)gi);
      if ((int)nb.q.size() <= k) {
        open.push_back(std::move(nb));
      } else {
        out.push_back(std::move(nb));  // wider than k: emitted alone
      }
    }
    rebuild_owner();
  }
  for (auto &b : open) out.push_back(std::move(b));
  return out;
}

// Candidate sets S: every window of k consecutive qubits, the previous block's set and sets
// grown from the first few gates of the front. A gate is absorbed by S when all its qubits
// are in S and none of them is blocked; a remaining gate that touches S but is not absorbed
// blocks its qubits in S, so no later gate on them can move past it.
std::vector<Block> plan_fusion_front(const std::vector<Gate> &gates, int k, int n, int fresh_limit,
                                     int max_phases) {
  std::vector<Block> out;
  const size_t G = gates.size();
  std::vector<unsigned long long> gmask(G, 0);
  std::vector<char> phase(G, 0);
  for (size_t i = 0; i < G; ++i) {
    gmask[i] = qubit_mask(gates[i]);
    phase[i] = max_phases > 0 && is_phase_gate(gates[i]);
  }
  const unsigned long long all = n >= 64 ? ~0ULL : ((1ULL << n) - 1ULL);
  std::vector<size_t> ph, best_ph;
  std::vector<char> done(G, 0);
  size_t remaining = G, first = 0;
  std::vector<unsigned long long> windows;
  for (int q = 0; q + k <= n; ++q) windows.push_back(((1ULL << k) - 1ULL) << q);
  unsigned long long prev = 0;
  std::vector<size_t> take, best_take;
  std::vector<unsigned long long> cs;
  while (remaining > 0) {
    while (first < G && done[first]) ++first;
    const size_t end = std::min(G, first + kScanLimit);
    cs = windows;
    if (prev) cs.push_back(prev);
    int seeds = 0;
    for (size_t i0 = first; i0 < end && seeds < 8; ++i0) {
      if (done[i0] || __builtin_popcountll(gmask[i0]) > k) continue;
      ++seeds;
      unsigned long long S = gmask[i0], blocked = 0;
      for (size_t i = first; i < end; ++i) {
        if (done[i]) continue;
        const unsigned long long m = gmask[i];
        if (m & blocked) {
          blocked |= m;
          continue;
        }
        if (__builtin_popcountll(S | m) <= k && ((m & S) || i > i0)) {
          if (i >= i0) S |= m;
        } else {
          blocked |= m;
        }
      }
      // pad to k qubits with neighbours so the set is a full candidate
      for (int step = 0; step < n && __builtin_popcountll(S) < k; ++step) {
        const int lo = __builtin_ctzll(S) - 1, hi = 63 - __builtin_clzll(S) + 1;
        if (hi < n) S |= 1ULL << hi;
        if (lo >= 0 && __builtin_popcountll(S) < k) S |= 1ULL << lo;
      }
      cs.push_back(S);
    }
    int best = -1;
    unsigned long long best_s = 0;
    best_take.clear();
    best_ph.clear();
    for (unsigned long long S : cs) {
      take.clear();
      ph.clear();
      unsigned long long blocked = 0;
      for (size_t i = first; i < end; ++i) {
        if (done[i]) continue;
        const unsigned long long m = gmask[i];
        if (!(m & S)) {
          // outside the set: a ready phase gate is taken along, anything else blocks
          if (max_phases > 0) {
            if (phase[i] && !(m & blocked) && (int)ph.size() < max_phases) ph.push_back(i);
            else blocked |= m;
            if (blocked == all) break;
          }
          continue;
        }
        if ((m & ~S) == 0 && !(m & blocked)) take.push_back(i);
        else blocked |= max_phases > 0 ? m : (m & S);
        if (max_phases > 0 ? blocked == all : blocked == S) break;
      }
      const int fresh = prev ? __builtin_popcountll(S & ~prev) : 0;
      // phase gates do not enter the score: nearly every set could take them, and counting
      // them pulls the choice away from sets that keep the layout moving smoothly
      const int score = (int)take.size() * 64 + __builtin_popcountll(S & prev) -
                        (fresh > fresh_limit ? kFreshPenalty * 64 : 0);
      if (score > best && !take.empty()) {
        best = score;
        best_s = S;
        best_take = take;
        best_ph = ph;
      }
    }
    Block b;
    if (best_take.empty()) {
      // no candidate takes the first remaining gate (wider than k): it stands alone
      add_to_group(b, gates[first], (int)first);
      done[first] = 1;
      --remaining;
      out.push_back(std::move(b));
      prev = 0;
      continue;
    }
    for (size_t i : best_take) {
      add_to_group(b, gates[i], (int)i);
      done[i] = 1;
      --remaining;
    }
    for (size_t i : best_ph) {
      b.phases.push_back((int)i);
      done[i] = 1;
      --remaining;
    }
    out.push_back(std::move(b));
    prev = best_s;
  }
  return out;
}

// Re-index a matrix over qubit list `from` (from[0] = MSB) onto `to` (to[0] = MSB), which
// must contain `from`; qubits only in `to` get the identity.
std::vector<cd> reindex(const std::vector<cd> &u, const std::vector<int> &from,
                        const std::vector<int> &to) {
  const int kf = (int)from.size(), kt = (int)to.size();
  const int df = 1 << kf, dt = 1 << kt;
  std::vector<int> pos(kf);  // bit position in `to` index of from[j]
  int fmask = 0;
  for (int j = 0; j < kf; ++j) {
    pos[j] = kt - 1 - index_of(to, from[j]);
    fmask |= 1 << pos[j];
  }
  std::vector<cd> r((size_t)dt * dt, 0.0);
  for (int c = 0; c < dt; ++c) {
    int cf = 0;
    for (int j = 0; j < kf; ++j) cf |= ((c >> pos[j]) & 1) << (kf - 1 - j);
    for (int rf = 0; rf < df; ++rf) {
      const cd v = u[(size_t)rf * df + cf];
      if (v == 0.0) continue;
      int row = c & ~fmask;
      for (int j = 0; j < kf; ++j) row |= ((rf >> (kf - 1 - j)) & 1) << pos[j];
      r[(size_t)row * dt + c] = v;
    }
  }
  return r;
}

}  // namespace qsim
