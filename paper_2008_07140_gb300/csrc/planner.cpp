// Gate-fusion planner: merges consecutive gates into k-qubit unitaries composed in FP64.
//
// Greedy over the gate list with several open blocks on disjoint qubit sets. A gate whose
// qubits, together with every open block it touches, fit in k qubits joins them (the
// touched blocks are merged first; blocks on disjoint qubits commute, so their product is
// a Kronecker product). Otherwise the touched blocks are closed (emitted) and the gate
// starts a new block. A block is emitted before any later block that shares a qubit, so
// the emitted order respects every dependency of the original list.
#include <algorithm>

#include "internal.h"
#include "planner.h"

namespace qsim {

namespace {

int index_of(const std::vector<int> &q, int x) {
  for (size_t i = 0; i < q.size(); ++i)
    if (q[i] == x) return (int)i;
  return -1;
}

// U' = U (x) I on `extra` new qubits appended as less significant index bits.
void extend(Block &b, const std::vector<int> &extra) {
  if (extra.empty()) return;
  const int old_dim = 1 << b.q.size();
  const int e = (int)extra.size();
  const int dim = old_dim << e;
  std::vector<cd> u((size_t)dim * dim, 0.0);
  for (int r = 0; r < old_dim; ++r)
    for (int c = 0; c < old_dim; ++c) {
      const cd v = b.u[(size_t)r * old_dim + c];
      if (v == 0.0) continue;
      for (int t = 0; t < (1 << e); ++t) u[(size_t)((r << e) | t) * dim + ((c << e) | t)] = v;
    }
  b.q.insert(b.q.end(), extra.begin(), extra.end());
  b.u.swap(u);
}

// U = U_a (x) U_b with a's qubits first (more significant).
Block kron(const Block &a, const Block &b) {
  Block r;
  r.q = a.q;
  r.q.insert(r.q.end(), b.q.begin(), b.q.end());
  const int da = 1 << a.q.size(), db = 1 << b.q.size(), d = da * db;
  r.u.assign((size_t)d * d, 0.0);
  for (int ra = 0; ra < da; ++ra)
    for (int ca = 0; ca < da; ++ca) {
      const cd va = a.u[(size_t)ra * da + ca];
      if (va == 0.0) continue;
      for (int rb = 0; rb < db; ++rb)
        for (int cb = 0; cb < db; ++cb)
          r.u[(size_t)(ra * db + rb) * d + (ca * db + cb)] = va * b.u[(size_t)rb * db + cb];
    }
  r.gates = a.gates;
  r.gates.insert(r.gates.end(), b.gates.begin(), b.gates.end());
  std::sort(r.gates.begin(), r.gates.end());
  return r;
}

}  // namespace

void embed_gate(const Gate &g, const std::vector<int> &q, std::vector<cd> &out) {
  const int kb = (int)q.size();
  const int dim = 1 << kb;
  int tpos[QSIM_MAX_FUSED];
  for (int j = 0; j < g.nt; ++j) tpos[j] = kb - 1 - index_of(q, g.t[j]);
  int cmask = 0;
  for (int c : g.ctrl) cmask |= 1 << (kb - 1 - index_of(q, c));
  int tmask = 0;
  for (int j = 0; j < g.nt; ++j) tmask |= 1 << tpos[j];
  const int gd = 1 << g.nt;
  out.assign((size_t)dim * dim, 0.0);
  for (int c = 0; c < dim; ++c) {
    if ((c & cmask) != cmask) {
      out[(size_t)c * dim + c] = 1.0;
      continue;
    }
    int a = 0;
    for (int j = 0; j < g.nt; ++j) a |= ((c >> tpos[j]) & 1) << (g.nt - 1 - j);
    for (int a2 = 0; a2 < gd; ++a2) {
      const cd v = g.m[(size_t)a2 * gd + a];
      if (v == 0.0) continue;
      int r = c & ~tmask;
      for (int j = 0; j < g.nt; ++j) r |= ((a2 >> (g.nt - 1 - j)) & 1) << tpos[j];
      out[(size_t)r * dim + c] = v;
    }
  }
}

void absorb(Block &b, const Gate &g, int gate_index) {
  std::vector<int> extra;
  for (int j = 0; j < g.nt; ++j)
    if (index_of(b.q, g.t[j]) < 0) extra.push_back(g.t[j]);
  for (int c : g.ctrl)
    if (index_of(b.q, c) < 0) extra.push_back(c);
  if (b.q.empty()) {
    b.q = extra;
    const int d = 1 << b.q.size();
    b.u.assign((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i) b.u[(size_t)i * d + i] = 1.0;
  } else {
    extend(b, extra);
  }
  std::vector<cd> G;
  embed_gate(g, b.q, G);
  const int d = 1 << b.q.size();
  std::vector<cd> u((size_t)d * d, 0.0);
  for (int r = 0; r < d; ++r)
    for (int t = 0; t < d; ++t) {
      const cd v = G[(size_t)r * d + t];
      if (v == 0.0) continue;
      for (int c = 0; c < d; ++c) u[(size_t)r * d + c] += v * b.u[(size_t)t * d + c];
    }
  b.u.swap(u);
  b.gates.push_back(gate_index);
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
        for (size_t j = 1; j < touched.size(); ++j) merged = kron(merged, open[touched[j]]);
      }
      absorb(merged, g, (int)gi);
      for (int j = (int)touched.size() - 1; j >= 0; --j) open.erase(open.begin() + touched[j]);
      open.push_back(std::move(merged));
    } else {
      for (int b : touched) out.push_back(open[b]);
      for (int j = (int)touched.size() - 1; j >= 0; --j) open.erase(open.begin() + touched[j]);
      Block nb;
      absorb(nb, g, (int)gi);
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
