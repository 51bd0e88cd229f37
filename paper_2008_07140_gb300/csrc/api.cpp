// C ABI of libqsim: state lifetime, gate dispatch, the circuit executor and read-outs.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>

#include "internal.h"
#include "philox.cuh"
#include "planner.h"

namespace qsim {

const char *last_error();

int num_sms() {
  static int v = 0;
  if (v == 0) {
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
      v = c;
    else
      v = 152;
  }
  return v;
}

namespace {

StateDev dev_of(const qsim_state *s) {
  return StateDev{s->amps, s->n, s->dtype, s->stream, s->fmt, s->tc_lo_smem};
}

bool wants_split(const qsim_state *s) { return s->dtype == QSIM_C128 && !s->fp64_native && !s->auto_native; }

// The state holds exact values again (|0...0>, a host copy): a fresh split-sweep budget.
void exact_values(qsim_state *s) {
  s->split_sweeps = 0;
  s->auto_native = 0;
}

// Gate kernels on complex128 run on the split format unless the native FP64 kernels are
// selected; read-outs and host copies want plain doubles.
qsim_status ensure_split(qsim_state *s) {
  if (!wants_split(s) || s->fmt == 1) return QSIM_OK;
  QS_TRY(launch_to_split(dev_of(s)));
  s->fmt = 1;
  return QSIM_OK;
}

qsim_status ensure_plain(qsim_state *s) {
  if (s->fmt == 0) return QSIM_OK;
  QS_TRY(launch_to_plain(dev_of(s)));
  s->fmt = 0;
  return QSIM_OK;
}

// One split sweep of a single-gate call, or the switch to FP64 instructions when the
// budget is spent.
qsim_status spend_split_sweep(qsim_state *s) {
  if (!wants_split(s)) return QSIM_OK;
  if (s->split_sweeps + 1 > kSplitSweepLimit) {
    QS_TRY(ensure_plain(s));
    s->auto_native = 1;
    return QSIM_OK;
  }
  ++s->split_sweeps;
  return QSIM_OK;
}

size_t amp_bytes(int dtype) { return dtype == QSIM_C128 ? 16 : 8; }

qsim_status check_state(const qsim_state *s) {
  if (!s) {
    set_error("state is NULL");
    return QSIM_EINVAL;
  }
  return QSIM_OK;
}

qsim_status ensure_scratch(qsim_state *s) {
  const size_t need = reduce_scratch_bytes(s->n);
  if (s->scratch && s->scratch_bytes >= need) return QSIM_OK;
  if (s->scratch) {
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    cudaFree(s->scratch);
    s->scratch = nullptr;
  }
  QS_TRY_CUDA(cudaMalloc((void **)&s->scratch, need));
  s->scratch_bytes = need;
  return QSIM_OK;
}

// Device matrix arena: pinned host staging + device buffer, one upload at a time.
qsim_status arena_upload(qsim_state *s, const void *data, size_t bytes) {
  if (bytes == 0) return QSIM_OK;
  if (bytes > s->mat_bytes) {
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    if (s->mat_dev) cudaFree(s->mat_dev);
    if (s->mat_host) cudaFreeHost(s->mat_host);
    s->mat_dev = s->mat_host = nullptr;
    s->mat_bytes = 0;
    size_t cap = 1 << 16;
    while (cap < bytes) cap <<= 1;
    QS_TRY_CUDA(cudaMalloc(&s->mat_dev, cap));
    QS_TRY_CUDA(cudaHostAlloc(&s->mat_host, cap, cudaHostAllocDefault));
    s->mat_bytes = cap;
  }
  if (!s->mat_event) QS_TRY_CUDA(cudaEventCreateWithFlags(&s->mat_event, cudaEventDisableTiming));
  QS_TRY_CUDA(cudaEventSynchronize(s->mat_event));
  memcpy(s->mat_host, data, bytes);
  QS_TRY_CUDA(cudaMemcpyAsync(s->mat_dev, s->mat_host, bytes, cudaMemcpyHostToDevice, s->stream));
  QS_TRY_CUDA(cudaEventRecord(s->mat_event, s->stream));
  return QSIM_OK;
}

Ins make_ins(unsigned long long all_mask, unsigned long long set, int n) {
  Ins ins;
  ins.n = 0;
  ins.set = set;
  for (int q = 0; q < n; ++q)
    if (all_mask >> q & 1ULL) ins.pos[ins.n++] = q;
  return ins;
}

int classify2(const cd *m) {
  const bool diag = m[1] == 0.0 && m[2] == 0.0;
  if (diag) return 4;
  if (m[0] == 0.0 && m[3] == 0.0) return (m[1] == 1.0 && m[2] == 1.0) ? MC_SWAP : MC_ANTI;
  bool real = true;
  for (int i = 0; i < 4; ++i) real = real && m[i].imag() == 0.0;
  return real ? MC_REAL : MC_GENERIC;
}

void append_cast(std::vector<unsigned char> &buf, const cd *m, size_t count, int dtype) {
  const size_t off = buf.size();
  if (dtype == QSIM_C128) {
    buf.resize(off + count * 16);
    double *d = reinterpret_cast<double *>(buf.data() + off);
    for (size_t i = 0; i < count; ++i) {
      d[2 * i] = m[i].real();
      d[2 * i + 1] = m[i].imag();
    }
  } else {
    // hi floats, then the lo floats (FP64 rounding residues)
    buf.resize(off + count * 16);
    float *f = reinterpret_cast<float *>(buf.data() + off);
    for (size_t i = 0; i < count; ++i) {
      f[2 * i] = (float)m[i].real();
      f[2 * i + 1] = (float)m[i].imag();
      f[2 * count + 2 * i] = (float)(m[i].real() - (double)f[2 * i]);
      f[2 * count + 2 * i + 1] = (float)(m[i].imag() - (double)f[2 * i + 1]);
    }
  }
}

// One launch of the executor. Gates are in PHYSICAL qubits.
struct Action {
  enum Type { GATE, REMAP, FUSED_TC, FUSED_SIMT, ZERO_SLOTS, TO_SPLIT, DIAG } type;
  Gate g;            // GATE (nt <= 2), or FUSED_SIMT (targets = phys order, controls)
  size_t mat_off = 0;
  int k = 0;
  int L = 0;
  int m = 0;
  int hi[8] = {};
  int dst[16] = {};
  TcTilePlan tp{};  // FUSED_TC: tile rows and epilogue permutation
  DiagIdx di{};     // DIAG: the table's qubits (the table at mat_off; m = gates merged)
};

// Physical launch of a 1- or 2-target gate (matrix in g.m).
qsim_status launch_gate_phys(const StateDev &d, const Gate &g, int64_t *bytes) {
  unsigned long long cmask = 0;
  for (int c : g.ctrl) cmask |= 1ULL << c;
  const cd *m = g.m.data();
  if (g.nt == 1) {
    const unsigned long long bt = 1ULL << g.t[0];
    const int cls = classify2(m);
    if (cls == 4) {
      if (m[0] == 1.0 && m[3] == 1.0) return QSIM_OK;
      if (m[0] == 1.0)
        return d.split ? launch_phase_df(d, bt | cmask, m[3], bytes) : launch_phase(d, bt | cmask, m[3], bytes);
    }
    const Ins ins1 = make_ins(bt | cmask, cmask, d.n);
    return d.split ? launch_pair_df(d, ins1, 0, bt, m, cls, bytes) : launch_pair(d, ins1, 0, bt, m, cls, bytes);
  }
  const unsigned long long b0 = 1ULL << g.t[0], b1 = 1ULL << g.t[1];
  const Ins ins = make_ins(b0 | b1 | cmask, cmask, d.n);
  bool outer_identity = m[0] == 1.0 && m[15] == 1.0;
  for (int i = 1; i < 4 && outer_identity; ++i)
    outer_identity = m[i] == 0.0 && m[4 * i] == 0.0 && m[12 + i - 1] == 0.0 && m[4 * (i - 1) + 3] == 0.0;
  if (outer_identity) {
    const cd sub[4] = {m[5], m[6], m[9], m[10]};
    const int cls = classify2(sub);
    if (cls == 4 && sub[0] == 1.0 && sub[3] == 1.0) return QSIM_OK;
    // pair (index with only t1 set, index with only t0 set) = matrix rows 1 and 2
    return d.split ? launch_pair_df(d, ins, b1, b0, sub, cls, bytes) : launch_pair(d, ins, b1, b0, sub, cls, bytes);
  }
  bool diag = true;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c)
      if (r != c && m[4 * r + c] != 0.0) diag = false;
  if (diag && m[0] == 1.0 && m[5] == 1.0 && m[10] == 1.0)
    return d.split ? launch_phase_df(d, b0 | b1 | cmask, m[15], bytes) : launch_phase(d, b0 | b1 | cmask, m[15], bytes);
  const unsigned long long off[4] = {0, b1, b0, b0 | b1};
  return d.split ? launch_quad_df(d, ins, off, m, bytes) : launch_quad(d, ins, off, m, bytes);
}

qsim_status run_actions(qsim_state *s, const std::vector<Action> &acts, int64_t *bytes,
                        cudaStream_t stream) {
  StateDev d = dev_of(s);
  d.stream = stream;
  for (const Action &a : acts) {
    switch (a.type) {
      case Action::TO_SPLIT:
        QS_TRY(launch_to_split(d));
        d.split = 1;
        break;
      case Action::GATE: QS_TRY(launch_gate_phys(d, a.g, bytes)); break;
      case Action::ZERO_SLOTS:
        QS_TRY_CUDA(cudaMemsetAsync(s->norm_slots, 0, sizeof(double) * a.m, stream));
        break;
      case Action::REMAP: QS_TRY(launch_permute(d, a.L, a.hi, a.m, a.dst, bytes)); break;
      case Action::FUSED_TC:
        QS_TRY(launch_fused_tc(d, a.k, static_cast<const unsigned char *>(s->mat_dev) + a.mat_off, a.tp, bytes));
        break;
      case Action::DIAG: {
        const void *tab = static_cast<const unsigned char *>(s->mat_dev) + a.mat_off;
        QS_TRY(d.split ? launch_diag_df(d, a.di, tab, bytes) : launch_diag(d, a.di, tab, bytes));
        break;
      }
      case Action::FUSED_SIMT: {
        unsigned long long cmask = 0;
        for (int c : a.g.ctrl) cmask |= 1ULL << c;
        const void *mat = static_cast<const unsigned char *>(s->mat_dev) + a.mat_off;
        QS_TRY(d.split ? launch_fused_df(d, a.g.t, a.k, cmask, mat, bytes)
                       : launch_fused_simt_ctl(d, a.g.t, a.k, cmask, mat, bytes));
        break;
      }
    }
  }
  return QSIM_OK;
}

Gate to_phys(const qsim_state *s, const Gate &g) {
  Gate p = g;
  for (int j = 0; j < g.nt; ++j) p.t[j] = s->l2p[g.t[j]];
  for (auto &c : p.ctrl) c = s->l2p[c];
  return p;
}

void apply_permute_maps(qsim_state *s, int L, const int *hi, int m, const int *dst) {
  int pos[16];
  for (int b = 0; b < L; ++b) pos[b] = b;
  for (int j = 0; j < m; ++j) pos[L + j] = hi[j];
  int old_p2l[16];
  for (int b = 0; b < L + m; ++b) old_p2l[b] = s->p2l[pos[b]];
  for (int b = 0; b < L + m; ++b) {
    const int x = old_p2l[b];
    s->p2l[pos[dst[b]]] = x;
    s->l2p[x] = pos[dst[b]];
  }
}

// Plan one (physical) gate: per-gate kernels for 1-2 targets, the fused kernel otherwise.
void plan_gate(qsim_state *s, const Gate &lg, std::vector<Action> &acts, std::vector<unsigned char> &mats) {
  Action a;
  a.g = to_phys(s, lg);
  if (lg.nt <= 2) {
    a.type = Action::GATE;
  } else {
    a.type = Action::FUSED_SIMT;
    a.k = lg.nt;
    a.mat_off = mats.size();
    if (wants_split(s)) append_fused_df(mats, lg.m.data(), lg.nt, a.g.t);
    else append_cast(mats, lg.m.data(), lg.m.size(), s->dtype);
  }
  acts.push_back(std::move(a));
}

// Row-phase terms of a diagonal gate whose qubits all sit at physical positions >= k: the
// gate multiplies row x by exp(2 pi i f(x)), f(x) in turns from its diagonal on the bits of
// its qubits (targets and controls); by Moebius inversion f = sum over the subsets S of
// those bits of c_S [every bit of S set in x], c_S = sum_{U in S} (-1)^{|S \ U|} f(U). Each
// S with c_S != 0 (mod 1) is added to `terms` (mask of S's row-index bits, c_S in turns),
// adding up with a term of the same mask already there.
void row_phase_terms(const qsim_state *s, const Gate &g, int k, std::vector<unsigned long long> &masks,
                     std::vector<double> &coef) {
  std::vector<int> qs(g.t, g.t + g.nt);  // bit j of a pattern <-> qs[j]
  qs.insert(qs.end(), g.ctrl.begin(), g.ctrl.end());
  const int nq = (int)qs.size(), gd = 1 << g.nt, nc = (int)g.ctrl.size();
  std::vector<double> f((size_t)1 << nq, 0.0);
  for (int idx = 0; idx < (1 << nq); ++idx) {
    const int cbits = (idx >> g.nt) & ((1 << nc) - 1);
    if (cbits != (1 << nc) - 1) continue;  // a control is 0: identity
    int a = 0;  // gate-matrix index: t[0] is the most significant bit
    for (int j = 0; j < g.nt; ++j) a |= ((idx >> j) & 1) << (g.nt - 1 - j);
    const cd v = g.m[(size_t)a * gd + a];
    f[idx] = std::atan2(v.imag(), v.real()) / (2.0 * M_PI);
  }
  for (int S = 0; S < (1 << nq); ++S) {
    double c = 0.0;
    for (int U = S;; U = (U - 1) & S) {  // every subset U of S
      c += ((__builtin_popcount((unsigned)(S ^ U)) & 1) ? -1.0 : 1.0) * f[U];
      if (U == 0) break;
    }
    c -= std::floor(c);
    if (c == 0.0) continue;
    unsigned long long mask = 0;
    for (int j = 0; j < nq; ++j)
      if ((S >> j) & 1) mask |= 1ULL << (s->l2p[qs[j]] - k);
    size_t x = 0;
    while (x < masks.size() && masks[x] != mask) ++x;
    if (x == masks.size()) {
      masks.push_back(mask);
      coef.push_back(0.0);
    }
    coef[x] += c;
  }
}

// Re-label the output index of a 2^k x 2^k matrix: output bit t moves to bit colperm[t]
// (physical column bit t of the result lands on column bit colperm[t]).
void permute_output_bits(std::vector<cd> &u, int k, const int *colperm) {
  bool id = true;
  for (int t = 0; t < k; ++t) id = id && colperm[t] == t;
  if (id) return;
  const int d = 1 << k;
  std::vector<cd> r((size_t)d * d);
  for (int row = 0; row < d; ++row) {
    int row2 = 0;
    for (int t = 0; t < k; ++t)
      if ((row >> t) & 1) row2 |= 1 << colperm[t];
    for (int c = 0; c < d; ++c) r[(size_t)row2 * d + c] = u[(size_t)row * d + c];
  }
  u.swap(r);
}

// Qubit sets of the fused blocks after the current one (a view into the plan's list).
struct Upcoming {
  const std::vector<std::vector<int>> *sets = nullptr;
  size_t from = 0;
  // distance to the next block using logical qubit x (large if none does)
  int next_use(int x) const {
    if (!sets) return 1 << 30;
    for (size_t i = from; i < sets->size(); ++i)
      if (std::find((*sets)[i].begin(), (*sets)[i].end(), x) != (*sets)[i].end()) return (int)(i - from);
    return 1 << 30;
  }
};

// Plan the remap that brings the logical qubits `need` into physical positions [0, kk).
void plan_remap_low(qsim_state *s, const std::vector<int> &need, int kk, const Upcoming &future,
                    std::vector<Action> &acts) {
  std::vector<int> missing;
  for (int x : need)
    if (s->l2p[x] >= kk) missing.push_back(x);
  if (missing.empty()) return;
  std::vector<int> victims;  // physical positions < kk whose qubit is not needed
  for (int p = 0; p < kk; ++p)
    if (std::find(need.begin(), need.end(), s->p2l[p]) == need.end()) victims.push_back(p);
  auto next_use = [&](int x) { return future.next_use(x); };
  std::stable_sort(victims.begin(), victims.end(),
                   [&](int a, int b) { return next_use(s->p2l[a]) > next_use(s->p2l[b]); });
  // Missing qubits inside the low run of the remap tile (positions kk..L-1) swap within
  // the run; those above it become the tile's high qubits.
  const int L = remap_low_run(s->n, s->dtype, (int)missing.size());
  Action a;
  a.type = Action::REMAP;
  a.L = L;
  a.m = 0;
  for (int b = 0; b < 16; ++b) a.dst[b] = b;
  for (size_t j = 0; j < missing.size(); ++j)
    if (s->l2p[missing[j]] >= L) a.hi[a.m++] = s->l2p[missing[j]];
  int next_hi = 0;
  for (size_t j = 0; j < missing.size(); ++j) {
    const int px = s->l2p[missing[j]];
    const int lo = victims[j];
    const int tp = px < L ? px : L + next_hi++;  // tile position of the missing qubit
    a.dst[lo] = tp;
    a.dst[tp] = lo;
  }
  const int m = a.m;
  apply_permute_maps(s, L, a.hi, m, a.dst);
  acts.push_back(a);
}

// Plan the epilogue permutation of a fused tensor-core block so that the logical qubits
// `need` (the next fused block) end in physical positions [0, k). The block's tile row
// bits must contain every needed qubit above position k-1: a run of c >= 2 row bits just
// above the fused qubits plus at most 7 - c others. Returns false (identity plan) when the
// needed qubits do not fit; the next block then takes a separate remap sweep.
//
// The epilogue stores a thread's row values as float4 pairs into the 128-byte swizzled
// stage; a quarter warp (lane bits 0..2 = tile row bits 0..2) is free of bank conflicts
// when those three row bits land on three different 16-byte slot bits (slot = column bits
// 1..3 xor row bits 0..2 of the destination). So a missing qubit on tile row bit i < 3
// takes column i + 1 and a row content on bit i < 3 stays; the other row contents are
// placed by next use, soonest on the lowest rows, and the filler high rows of the tile are
// the rows whose qubits are needed soonest (the next transitions then find their qubits in
// low rows, where the tiles have long low runs).
bool plan_transition(qsim_state *s, const std::vector<int> &need, int k, const Upcoming &future,
                        TcTilePlan &tp, int *colperm) {
  tc_identity_plan(k, tp);
  for (int t = 0; t < k; ++t) colperm[t] = t;
  auto needed = [&](int x) { return std::find(need.begin(), need.end(), x) != need.end(); };
  std::vector<int> missing;
  for (int x : need)
    if (s->l2p[x] >= k) missing.push_back(x);
  if (missing.empty()) return true;
  std::vector<int> victims;
  for (int p = 0; p < k; ++p)
    if (!needed(s->p2l[p])) victims.push_back(p);
  const int m = (int)missing.size();
  if ((int)victims.size() < m) return false;
  auto next_use = [&](int x) { return future.next_use(x); };
  std::stable_sort(victims.begin(), victims.end(),
                   [&](int a, int b) { return next_use(s->p2l[a]) > next_use(s->p2l[b]); });
  victims.resize(m);  // the columns that leave: latest next use first
  const int rbits = s->n - k;
  if (rbits < 7) return false;
  int c = -1;
  for (int cc = 7; cc >= 2; --cc) {
    int outside = 0;
    for (int x : missing) outside += (s->l2p[x] - k >= cc);
    if (outside <= 7 - cc) {
      c = cc;
      break;
    }
  }
  if (c < 0) return false;
  std::vector<int> hb;
  for (int x : missing)
    if (s->l2p[x] - k >= c) hb.push_back(s->l2p[x] - k);
  {
    std::vector<int> cand;
    for (int r = c; r < rbits; ++r)
      if (std::find(hb.begin(), hb.end(), r) == hb.end() && next_use(s->p2l[k + r]) < (1 << 30)) cand.push_back(r);
    std::stable_sort(cand.begin(), cand.end(),
                     [&](int a, int b) { return next_use(s->p2l[k + a]) < next_use(s->p2l[k + b]); });
    for (size_t i = 0; i < cand.size() && (int)hb.size() < 7 - c; ++i) hb.push_back(cand[i]);
  }
  for (int r = c; (int)hb.size() < 7 - c && r < rbits; ++r)
    if (std::find(hb.begin(), hb.end(), r) == hb.end()) hb.push_back(r);
  if ((int)hb.size() != 7 - c) return false;
  std::sort(hb.begin(), hb.end());
  tp.c = c;
  tp.nh = 7 - c;
  for (int j = 0; j < tp.nh; ++j) tp.hbit[j] = hb[j];
  std::vector<int> ins;
  for (int r = 0; r < c; ++r) ins.push_back(r);
  ins.insert(ins.end(), hb.begin(), hb.end());
  std::sort(ins.begin(), ins.end());
  tp.ins_n = 7;
  for (int j = 0; j < 7; ++j) tp.ins[j] = ins[j];
  int P[12];
  for (int t = 0; t < k; ++t) P[t] = t;
  for (int b = 0; b < 7; ++b) P[k + b] = k + (b < c ? b : hb[b - c]);
  auto tile_bit = [&](int phys) {
    for (int t = 0; t < k + 7; ++t)
      if (P[t] == phys) return t;
    return -1;
  };
  // final tile bit of each content, by its tile bit now (columns in their current order)
  int dest[12];
  for (int t = 0; t < k + 7; ++t) dest[t] = -1;
  bool col_taken[QSIM_MAX_FUSED] = {};
  int mt[QSIM_MAX_FUSED];  // tile bit of each missing qubit
  for (int j = 0; j < m; ++j) {
    mt[j] = tile_bit(s->l2p[missing[j]]);
    if (mt[j] < k) return false;
  }
  const bool keep_col0 = m < k;  // some content stays in the columns: pair = 1
  int rho = -1;
  bool row_taken[7] = {};
  bool single = false;
  if (!keep_col0) {
    // Every column leaves. Preferred: single-complex stores (pair = 0), free of bank
    // conflicts when lane bits 0..3 land on four different 8-byte slot bits (column bit 0
    // and slot bits 0..2): a missing qubit on tile row bit 3 (else on bit 0..2) takes column
    // 0, and the other three lane bits take the slot bits 0..2, a missing qubit through
    // column s + 1, a row content through row s.
    auto mis_at = [&](int b) {
      for (int j = 0; j < m; ++j)
        if (mt[j] == k + b) return j;
      return -1;
    };
    int c0 = mis_at(3) >= 0 ? 3 : -1;
    for (int b : {0, 1, 2})
      if (c0 < 0 && mis_at(b) >= 0) c0 = b;
    if (c0 >= 0 && k >= 4) {
      single = true;
      dest[mt[mis_at(c0)]] = 0;
      col_taken[0] = true;
      int lane_of_slot[3] = {0, 1, 2};
      if (c0 != 3) lane_of_slot[c0] = 3;
      for (int sl = 0; sl < 3; ++sl) {
        const int i = lane_of_slot[sl], j = mis_at(i);
        if (j >= 0) {
          dest[mt[j]] = sl + 1;
          col_taken[sl + 1] = true;
        } else {
          dest[k + i] = k + sl;
          row_taken[sl] = true;
        }
      }
    }
  }
  if (!keep_col0 && !single) {
    // column 0 is fed from a lane row bit instead (pair = 2, lane pairs exchange values);
    // prefer bits 3, 4
    for (int pref : {3, 4, 0, 1, 2})
      for (int j = 0; j < m && rho < 0; ++j)
        if (mt[j] == k + pref) rho = pref;
    if (rho >= 0) {
      for (int j = 0; j < m; ++j)
        if (mt[j] == k + rho) dest[mt[j]] = 0;
      col_taken[0] = true;
    }
  } else if (keep_col0) {
    col_taken[0] = true;  // reserved for a content that stays
  }
  // missing qubits on tile row bits 0..2 take columns 1..3
  for (int j = 0; j < m; ++j) {
    const int i = mt[j] - k;
    if (dest[mt[j]] < 0 && i < 3 && i + 1 < k && !col_taken[i + 1]) {
      dest[mt[j]] = i + 1;
      col_taken[i + 1] = true;
    }
  }
  for (int j = 0; j < m; ++j)
    if (dest[mt[j]] < 0)
      for (int cc = k - 1; cc >= 1; --cc)
        if (!col_taken[cc]) {
          dest[mt[j]] = cc;
          col_taken[cc] = true;
          break;
        }
  for (int j = 0; j < m; ++j)
    if (dest[mt[j]] < 0) return false;
  // staying columns: column 0 first (pair = 1), then the free columns
  std::vector<int> stay;
  for (int p = 0; p < k; ++p)
    if (std::find(victims.begin(), victims.end(), p) == victims.end()) stay.push_back(p);
  if (keep_col0) {
    col_taken[0] = false;
    // the content already at column 0 stays there when it stays at all
    std::stable_sort(stay.begin(), stay.end(), [](int a, int b) { return (a == 0) > (b == 0); });
  }
  for (int p : stay) {
    if (!col_taken[p]) {
      dest[p] = p;
      col_taken[p] = true;
    }
  }
  for (int p : stay)
    if (dest[p] < 0)
      for (int cc = 0; cc < k; ++cc)
        if (!col_taken[cc]) {
          dest[p] = cc;
          col_taken[cc] = true;
          break;
        }
  // rows: the column-0 victim of pair = 2 goes to row bit rho; row contents on bits 0..2
  // stay; the rest by next use
  if (rho >= 0) {
    // the victim placed on column 0 (after the column permutation) is the first victim
    dest[victims[0]] = k + rho;
    row_taken[rho] = true;
  }
  std::vector<int> movers;  // contents still without a destination
  for (int b = 0; b < 7; ++b) {
    const int t = k + b;
    if (dest[t] >= 0) continue;  // a missing qubit, or a row content already placed
    if (b < 3 && !row_taken[b]) {
      dest[t] = t;
      row_taken[b] = true;
    } else {
      movers.push_back(t);
    }
  }
  for (int v : victims)
    if (dest[v] < 0) movers.push_back(v);
  std::stable_sort(movers.begin(), movers.end(),
                   [&](int a, int b) { return next_use(s->p2l[P[a]]) < next_use(s->p2l[P[b]]); });
  size_t mi = 0;
  for (int b = 0; b < 7; ++b)
    if (!row_taken[b]) {
      if (mi >= movers.size()) return false;
      dest[movers[mi++]] = k + b;
      row_taken[b] = true;
    }
  if (mi != movers.size()) return false;
  // columns: colperm puts the staying contents on their destination columns and the
  // victims on the columns the missing qubits take (the pair = 2 victim on column 0)
  bool post_used[QSIM_MAX_FUSED] = {};
  int post_dest[QSIM_MAX_FUSED];  // tile destination of the content on post-pi column j
  for (int p : stay) {
    colperm[p] = dest[p];
    post_used[dest[p]] = true;
    post_dest[dest[p]] = dest[p];
  }
  {
    std::vector<int> vic = victims;
    if (rho >= 0) {
      colperm[vic[0]] = 0;
      post_used[0] = true;
      post_dest[0] = dest[vic[0]];
      vic.erase(vic.begin());
    }
    for (int v : vic)
      for (int j = 0; j < k; ++j)
        if (!post_used[j]) {
          colperm[v] = j;
          post_used[j] = true;
          post_dest[j] = dest[v];
          break;
        }
  }
  tp.ident = 0;
  for (int cc = 0; cc < (1 << k); ++cc) {
    int d = 0;
    for (int t = 0; t < k; ++t)
      if ((cc >> t) & 1) d |= 1 << post_dest[t];
    tp.tcol[cc] = d;
  }
  for (int b = 0; b < 7; ++b) tp.wrow[b] = 1 << dest[k + b];
  tp.pair = tp.tcol[1] == 1 ? 1 : 0;
  tp.pair_row = 0;
  if (!tp.pair && rho >= 0 && tp.tcol[1] == (1 << (k + rho)) && tp.wrow[rho] == 1) {
    tp.pair = 2;
    tp.pair_row = rho;
  }
  if (!tc_plan_valid(s->n, k, tp)) {
    tc_identity_plan(k, tp);
    for (int t = 0; t < k; ++t) colperm[t] = t;
    return false;
  }
  int old_p2l[12];
  for (int t = 0; t < k + 7; ++t) old_p2l[t] = s->p2l[P[t]];
  for (int t = 0; t < k + 7; ++t) {
    const int x = old_p2l[t];
    s->p2l[P[dest[t]]] = x;
    s->l2p[x] = P[dest[t]];
  }
  return true;
}

// A block of one small gate (and no row phases) runs as that gate's own sweep.
bool per_gate_block(const Block &b, const std::vector<Gate> &gates) {
  return b.gates.size() == 1 && gates[b.gates[0]].nt <= 2 && b.phases.empty();
}

// Order the fused blocks for the remap-in-epilogue scheme: list scheduling that keeps
// every dependency (blocks sharing a qubit stay in their original order) and, among the
// ready blocks, takes single-gate blocks first (they do not care about the layout), then
// the block that shares the most qubits with the previous fused block (fewer qubits to
// bring down at the transition).
std::vector<Block> schedule_blocks(std::vector<Block> blocks, const std::vector<Gate> &gates, int k) {
  const size_t nb = blocks.size();
  std::vector<std::vector<size_t>> succ(nb);
  std::vector<int> npred(nb, 0);
  std::vector<int> last(64, -1);
  for (size_t i = 0; i < nb; ++i) {
    std::vector<int> preds;
    for (int x : blocks[i].q)
      if (last[x] >= 0 && std::find(preds.begin(), preds.end(), last[x]) == preds.end()) preds.push_back(last[x]);
    for (int p : preds) {
      succ[p].push_back(i);
      npred[i]++;
    }
    for (int x : blocks[i].q) last[x] = (int)i;
  }
  auto single = [&](size_t i) { return blocks[i].gates.size() == 1 && gates[blocks[i].gates[0]].nt <= 2; };
  std::vector<size_t> ready;
  for (size_t i = 0; i < nb; ++i)
    if (npred[i] == 0) ready.push_back(i);
  std::vector<Block> out;
  out.reserve(nb);
  std::vector<int> prev;  // qubits of the previous fused block
  while (!ready.empty()) {
    size_t pick = 0;
    int best = -1;
    for (size_t r = 0; r < ready.size(); ++r) {
      const size_t i = ready[r];
      int score;
      if (single(i) || (int)blocks[i].q.size() > k) {
        score = 1000;
      } else {
        score = 0;
        for (int x : blocks[i].q) score += std::find(prev.begin(), prev.end(), x) != prev.end();
      }
      if (score > best || (score == best && i < ready[pick])) {
        best = score;
        pick = r;
      }
    }
    const size_t i = ready[pick];
    ready.erase(ready.begin() + pick);
    if (!single(i) && (int)blocks[i].q.size() <= k) prev = blocks[i].q;
    for (size_t j : succ[i])
      if (--npred[j] == 0) ready.push_back(j);
    out.push_back(std::move(blocks[i]));
  }
  return out;
}

thread_local bool g_force_tc = false;  // dry-run planning without a device (this thread only)

// Segment boundaries of a plan (see plan_circuit): where each segment's actions start and
// the qubit layout the state has there.
struct SegMarks {
  std::vector<size_t> begin;  // [in] first gate of each segment, ascending, begin[0] = 0
  std::vector<size_t> act;    // [out] first action of each segment, plus acts.size()
  std::vector<std::array<int, 64>> l2p, p2l;  // [out] layout at each segment start, plus the end
  void mark(const qsim_state *s, size_t at) {
    act.push_back(at);
    std::array<int, 64> a, b;
    memcpy(a.data(), s->l2p, sizeof(int) * 64);
    memcpy(b.data(), s->p2l, sizeof(int) * 64);
    l2p.push_back(a);
    p2l.push_back(b);
  }
};

// Per-gate planning with merged diagonal gates. A diagonal gate joins an open group (at
// most kDiagBits qubits, targets and controls); a gate that is not diagonal first closes
// every group that shares a qubit with it, and commutes past the others, which stay open.
// The gates of a group therefore commute with every gate listed between them, and the
// group runs, when it closes, either as one table sweep or, when the per-gate sweeps would
// be cheaper (a few high-target phases), as those sweeps.
class DiagGroups {
 public:
  DiagGroups(qsim_state *s, std::vector<Action> &acts, std::vector<unsigned char> &mats)
      : s_(s), acts_(acts), mats_(mats) {}

  void add(const Gate &lg) {
    const Gate g = to_phys(s_, lg);
    unsigned long long qm = 0;
    for (int j = 0; j < g.nt; ++j) qm |= 1ULL << g.t[j];
    for (int c : g.ctrl) qm |= 1ULL << c;
    bool identity = g.nt <= 2;
    for (int r = 0; identity && r < (1 << g.nt); ++r)
      for (int c = 0; identity && c < (1 << g.nt); ++c) identity = g.m[r * (1 << g.nt) + c] == (r == c ? 1.0 : 0.0);
    if (identity) {  // launches nothing and commutes with everything
      plan_gate(s_, lg, acts_, mats_);
      return;
    }
    if (diag_gate(g) && __builtin_popcountll(qm) <= kDiagBits) {
      // the open group it overlaps most that has room, else a new group
      int best = -1, best_ov = -1;
      for (int k = 0; k < (int)open_.size(); ++k) {
        if (__builtin_popcountll(open_[k].q | qm) > kDiagBits) continue;
        const int ov = __builtin_popcountll(open_[k].q & qm);
        if (ov > best_ov) {
          best_ov = ov;
          best = k;
        }
      }
      if (best < 0) {
        if ((int)open_.size() == kMaxOpen) flush(0);
        open_.push_back(Group{});
        best = (int)open_.size() - 1;
      }
      open_[best].q |= qm;
      open_[best].gates.push_back(g);
      return;
    }
    for (int k = (int)open_.size() - 1; k >= 0; --k)
      if (open_[k].q & qm) flush(k);
    plan_gate(s_, lg, acts_, mats_);
  }

  void flush_all() {
    while (!open_.empty()) flush(0);
  }

 private:
  static constexpr int kMaxOpen = 8;
  struct Group {
    unsigned long long q = 0;
    std::vector<Gate> gates;  // physical qubits
  };

  void emit_gate(const Gate &g) {
    Action a;
    a.type = Action::GATE;
    a.g = g;
    acts_.push_back(std::move(a));
  }

  void flush(int k) {
    Group grp = std::move(open_[k]);
    open_.erase(open_.begin() + k);
    const int n = s_->n, B = s_->dtype == QSIM_C128 ? 16 : 8;
    // per-gate cost against one full sweep, in bytes, with a launch counted as the bytes
    // the sweep moves in that time
    const TuneTable *t = tune_table();
    const double gbs = t && t->gbs_pair_c64 > 0 ? t->gbs_pair_c64 : 6000.0;
    const double launch_b = (t && t->launch_us > 0 ? t->launch_us : 3.0) * 1e-6 * gbs * 1e9;
    double separate = 0.0;
    for (const Gate &g : grp.gates) separate += diag_gate_bytes(g, n, B) + launch_b;
    const double merged = 2.0 * B * std::ldexp(1.0, n) + launch_b;
    if (grp.gates.size() < 2 || separate <= merged) {
      for (const Gate &g : grp.gates) emit_gate(g);
      return;
    }
    Action a;
    a.type = Action::DIAG;
    a.di.nq = 0;
    for (int b = 0; b < n; ++b)
      if (grp.q >> b & 1ULL) a.di.pos[a.di.nq++] = b;
    std::vector<const Gate *> gp;
    for (const Gate &g : grp.gates) gp.push_back(&g);
    a.mat_off = append_diag_table(mats_, gp, a.di, s_->dtype, wants_split(s_));
    a.m = (int)grp.gates.size();
    acts_.push_back(std::move(a));
  }

  qsim_state *s_;
  std::vector<Action> &acts_;
  std::vector<unsigned char> &mats_;
  std::vector<Group> open_;
};

// With seg, the gate list is consecutive segments: fused blocks never mix two of them and
// keep their order, while qubit transitions still run in the epilogue of the block before
// (so a segment may end by moving the next segment's qubits). seg receives the action
// range and the layout at every segment boundary.
qsim_status plan_circuit(qsim_state *s, const std::vector<Gate> &gates, const qsim_run_opts &o,
                         std::vector<Action> &acts, std::vector<unsigned char> &mats, qsim_run_stats &st,
                         SegMarks *seg = nullptr) {
  st = qsim_run_stats{};
  st.gates = (int64_t)gates.size();
  if (seg) {
    seg->act.clear();
    seg->l2p.clear();
    seg->p2l.clear();
  }
  if (wants_split(s) && s->fmt == 0 && !gates.empty()) {
    Action c;
    c.type = Action::TO_SPLIT;
    acts.push_back(c);
    s->fmt = 1;
  }
  const size_t nseg = seg ? seg->begin.size() : 0;
  if (seg) seg->mark(s, 0);  // segment 0 also holds the format change
  if (o.fuse == 0 && !o.merge_diagonals) {
    for (size_t gi = 0; gi < gates.size(); ++gi) {
      while (seg && seg->act.size() < nseg && seg->begin[seg->act.size()] <= gi) seg->mark(s, acts.size());
      plan_gate(s, gates[gi], acts, mats);
    }
    while (seg && seg->act.size() <= nseg) seg->mark(s, acts.size());
    return QSIM_OK;
  }
  if (o.fuse == 0) {
    DiagGroups dg(s, acts, mats);
    for (size_t gi = 0; gi < gates.size(); ++gi) {
      if (seg && seg->act.size() < nseg && seg->begin[seg->act.size()] <= gi) {
        dg.flush_all();  // groups stay inside a segment
        while (seg->act.size() < nseg && seg->begin[seg->act.size()] <= gi) seg->mark(s, acts.size());
      }
      dg.add(gates[gi]);
    }
    dg.flush_all();
    while (seg && seg->act.size() <= nseg) seg->mark(s, acts.size());
    return QSIM_OK;
  }
  int k = o.fuse < 0 ? 5 : o.fuse;
  if (k < 2 || k > QSIM_MAX_FUSED) {
    set_error("fusion width %d not in 2..%d", k, QSIM_MAX_FUSED);
    return QSIM_EINVAL;
  }
  if (k > s->n) k = s->n;
  const StateDev d = dev_of(s);
  const bool tc = s->dtype == QSIM_C64 && o.remap && (g_force_tc ? (k == 4 || k == 5) && s->n >= k + 7
                                                                 : fused_tc_supported(d, k));
  // Two planners; the plan with fewer fused blocks wins. The front planner's blocks come
  // out in a layout-friendly order already, and on the tensor-core path they also take
  // diagonal gates outside their qubits as row phases. Sets that bring in all k = 5 qubits
  // at once are penalised: their transition needs tiles with a 4-row low run (slower).
  auto plan_blocks = [&](const std::vector<Gate> &gl) {
    std::vector<Block> bl = plan_fusion(gl, k);
    if (tc) bl = schedule_blocks(std::move(bl), gl, k);
    std::vector<Block> front = plan_fusion_front(gl, k, s->n, tc ? 4 : k, tc ? kTcMaxPhase : 0);
    if (front.size() < bl.size()) bl.swap(front);
    return bl;
  };
  std::vector<Block> blocks;
  std::vector<size_t> block_seg;  // segment of each block
  if (!seg) {
    blocks = plan_blocks(gates);
  } else {
    for (size_t sg = 0; sg < nseg; ++sg) {
      const size_t b0 = seg->begin[sg], b1 = sg + 1 < nseg ? seg->begin[sg + 1] : gates.size();
      if (b0 > b1 || b1 > gates.size()) {
        set_error("internal: segment bounds");
        return QSIM_EINVAL;
      }
      std::vector<Gate> sub(gates.begin() + b0, gates.begin() + b1);
      for (Block b : plan_blocks(sub)) {
        for (int &gi : b.gates) gi += (int)b0;
        for (int &gi : b.phases) gi += (int)b0;
        blocks.push_back(std::move(b));
        block_seg.push_back(sg);
      }
    }
  }
  // matrices only for the blocks that run fused (single small gates take per-gate sweeps)
  {
    std::vector<char> wanted(blocks.size(), 0);
    for (size_t i = 0; i < blocks.size(); ++i)
      wanted[i] = !per_gate_block(blocks[i], gates);
    compose_blocks(blocks, gates, wanted);
  }
  std::vector<std::vector<int>> future(blocks.size());
  for (size_t i = 0; i < blocks.size(); ++i) future[i] = blocks[i].q;
  for (size_t bi = 0; bi < blocks.size(); ++bi) {
    const Block &b = blocks[bi];
    while (seg && seg->act.size() <= block_seg[bi]) seg->mark(s, acts.size());
    if (per_gate_block(b, gates)) {
      plan_gate(s, gates[b.gates[0]], acts, mats);
      continue;
    }
    st.fused_blocks++;
    if (tc && (int)b.q.size() <= k) {
      plan_remap_low(s, b.q, k, Upcoming{&future, bi + 1}, acts);  // only if the previous block could not
      for (int x : b.q)
        if (s->l2p[x] >= k) {
          set_error("internal: remap left qubit %d at position %d", x, s->l2p[x]);
          return QSIM_EINVAL;
        }
      std::vector<int> to(k);
      for (int j = 0; j < k; ++j) to[j] = s->p2l[k - 1 - j];  // to[0] = MSB = phys k-1
      std::vector<cd> u = reindex(b.u, b.q, to);
      Action a;
      a.type = Action::FUSED_TC;
      a.k = k;
      // phase gates: on row bits only -> row phases; on the fused positions only -> into
      // the matrix; across both -> a sweep of their own after the block (they commute)
      std::vector<int> after;
      std::vector<unsigned long long> pmask;  // row-phase terms (masks, turns)
      std::vector<double> pcoef;
      int np = 0;
      {
        for (int gi : b.phases) {
          const Gate &g = gates[gi];
          std::vector<int> qs(g.t, g.t + g.nt);
          qs.insert(qs.end(), g.ctrl.begin(), g.ctrl.end());
          int low = 0;
          for (int x : qs) low += s->l2p[x] < k;
          if (low == (int)qs.size()) {
            Block pb;
            pb.q = to;
            pb.gates = {gi};
            compose_block(pb, gates);
            std::vector<cd> w((size_t)1 << (2 * k), 0.0);
            const int dk = 1 << k;
            for (int r = 0; r < dk; ++r)  // w = P u (P diagonal)
              for (int c = 0; c < dk; ++c) w[(size_t)r * dk + c] = pb.u[(size_t)r * dk + r] * u[(size_t)r * dk + c];
            u.swap(w);
          } else if (low == 0 && np < kTcMaxPhase) {
            std::vector<unsigned long long> m2 = pmask;
            std::vector<double> c2 = pcoef;
            row_phase_terms(s, g, k, m2, c2);
            if (m2.size() <= (size_t)kTcMaxTerms) {
              pmask.swap(m2);
              pcoef.swap(c2);
              ++np;
            } else {
              after.push_back(gi);
            }
          } else {
            after.push_back(gi);
          }
          st.phase_gates++;
        }
      }
      // bring the next fused block's qubits down in this block's epilogue; the output
      // columns may first be permuted (folded into the matrix below)
      tc_identity_plan(k, a.tp);
      int colperm[QSIM_MAX_FUSED];
      for (int t = 0; t < k; ++t) colperm[t] = t;
      for (size_t nj = bi + 1; nj < blocks.size(); ++nj) {
        const Block &nb = blocks[nj];
        if (per_gate_block(nb, gates)) continue;  // per-gate sweep
        if ((int)nb.q.size() <= k) {
          plan_transition(s, nb.q, k, Upcoming{&future, nj + 1}, a.tp, colperm);
        }
        break;
      }
      permute_output_bits(u, k, colperm);
      if (!a.tp.ident) st.epilogue_remaps++;
      a.tp.nterm = 0;
      for (size_t j = 0; j < pmask.size(); ++j) {
        const double c = pcoef[j] - std::floor(pcoef[j]);
        if (c == 0.0) continue;
        a.tp.term[a.tp.nterm].mask = pmask[j];
        a.tp.term[a.tp.nterm].c = (float)c;
        ++a.tp.nterm;
      }
      const size_t nf = tc_operand_floats(k);
      a.mat_off = (mats.size() + 1023) & ~(size_t)1023;  // TMA source rows stay aligned
      mats.resize(a.mat_off + nf * sizeof(float));
      float *dst = reinterpret_cast<float *>(mats.data() + a.mat_off);
      build_tc_operands(k, u.data(), dst, dst + nf / 2);
      acts.push_back(std::move(a));
      for (int gi : after) {
        plan_gate(s, gates[gi], acts, mats);
        st.phase_gates--;
      }
    } else {
      Action a;
      a.type = Action::FUSED_SIMT;
      a.k = (int)b.q.size();
      for (int j = 0; j < a.k; ++j) a.g.t[j] = s->l2p[b.q[j]];
      a.g.nt = a.k;
      a.mat_off = mats.size();
      if (wants_split(s)) append_fused_df(mats, b.u.data(), a.k, a.g.t);
      else append_cast(mats, b.u.data(), b.u.size(), s->dtype);
      acts.push_back(std::move(a));
    }
  }
  while (seg && seg->act.size() <= nseg) seg->mark(s, acts.size());
  return QSIM_OK;
}

// Give every fused tensor-core launch an input and an output norm slot; with renormalising
// on, launch i > 0 scales its input by sqrt(N_in(first) / N_out(i - 1)).
qsim_status assign_norm_slots(qsim_state *s, std::vector<Action> &acts, bool renorm) {
  size_t ntc = 0;
  for (const Action &a : acts) ntc += a.type == Action::FUSED_TC;
  if (ntc == 0 || !renorm) return QSIM_OK;
  const size_t need = 2 * ntc;
  if (s->norm_slots_n < need) {
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    if (s->norm_slots) cudaFree(s->norm_slots);
    s->norm_slots = nullptr;
    size_t cap = 256;
    while (cap < need) cap <<= 1;
    QS_TRY_CUDA(cudaMalloc((void **)&s->norm_slots, cap * sizeof(double)));
    s->norm_slots_n = cap;
  }
  int i = 0;
  for (Action &a : acts) {
    if (a.type != Action::FUSED_TC) continue;
    a.tp.slots = s->norm_slots;
    a.tp.in_slot = 2 * i;
    a.tp.out_slot = 2 * i + 1;
    a.tp.ref_slot = i > 0 ? 0 : -1;
    a.tp.prev_slot = i > 0 ? 2 * i - 1 : -1;
    ++i;
  }
  Action z;
  z.type = Action::ZERO_SLOTS;
  z.m = (int)need;
  acts.insert(acts.begin(), z);
  return QSIM_OK;
}

// Predicted time (ms) of an action list from the autotuner's bandwidth table.
double predict_ms(const qsim_state *s, const std::vector<Action> &acts, const std::vector<Gate> &) {
  const TuneTable *t = tune_table();
  if (!t) return 0.0;
  const double B = s->dtype == QSIM_C128 ? 16.0 : 8.0;
  const double full = 2.0 * B * (double)(1LL << s->n) / 1e9;  // GB of one full sweep
  const double pair = s->dtype == QSIM_C128 ? (s->fp64_native ? 0.3 * t->gbs_pair_df : t->gbs_pair_df)
                                            : t->gbs_pair_c64;
  double ms = 0.0;
  for (const Action &a : acts) {
    double gb = full, bw = pair;
    switch (a.type) {
      case Action::GATE: {
        const int nsel = (int)a.g.ctrl.size();
        const cd *m = a.g.m.data();
        bool phase = a.g.nt == 1 ? (m[1] == 0.0 && m[2] == 0.0 && m[0] == 1.0)
                                 : (m[0] == 1.0 && m[5] == 1.0 && m[10] == 1.0 && m[15] != 1.0);
        gb = full / (double)(1LL << nsel) / (phase ? (a.g.nt == 1 ? 2.0 : 4.0) : 1.0);
        break;
      }
      case Action::REMAP: bw = t->gbs_remap; break;
      case Action::FUSED_TC: bw = t->gbs_fused[a.k] > 0 ? t->gbs_fused[a.k] : pair; break;
      case Action::FUSED_SIMT:
        bw = s->fmt && a.k < 6 && t->gbs_fused_df[a.k] > 0 ? t->gbs_fused_df[a.k]
                                                          : pair / (double)(1 << (a.k > 3 ? a.k - 3 : 0));
        break;
      case Action::TO_SPLIT: bw = 0.4 * pair; break;
      case Action::DIAG: break;
      case Action::ZERO_SLOTS: gb = 0.0; break;
    }
    ms += gb / bw * 1e3 + t->launch_us * 1e-3;
  }
  return ms;
}

uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
  return h;
}

qsim_status validate_qubits(const qsim_state *s, const int *q, int nq, const int *c, int nc) {
  unsigned long long seen = 0;
  for (int j = 0; j < nq + nc; ++j) {
    const int x = j < nq ? q[j] : c[j - nq];
    if (x < 0 || x >= s->n) {
      set_error("qubit %d out of range [0, %d)", x, s->n);
      return QSIM_EINVAL;
    }
    if (seen >> x & 1ULL) {
      set_error("qubit %d listed twice", x);
      return QSIM_EINVAL;
    }
    seen |= 1ULL << x;
  }
  return QSIM_OK;
}

// Restore the identity layout with one remap sweep per transposition.
// Restore the identity layout with as few remap sweeps as possible: each sweep permutes the
// low run [0, L) together with up to 6 high positions gathered along the cycles of the
// current permutation, and every position of that tile whose logical qubit is also in the
// tile gets it back (a cycle of up to L + 6 positions closes in one sweep).
qsim_status canonicalize(qsim_state *s) {
  const StateDev d = dev_of(s);
  constexpr int kHi = 6;
  int L = remap_low_run(s->n, s->dtype, kHi);
  if (L < 1) L = 1;
  // every sweep returns at least one position's qubit and disturbs no correct position,
  // so n sweeps always suffice
  for (int guard = 0; guard <= s->n; ++guard) {
    bool misplaced = false;
    for (int p = 0; p < s->n; ++p) misplaced = misplaced || s->p2l[p] != p;
    if (!misplaced) return QSIM_OK;
    int hi[kHi], m = 0;
    auto in_tile = [&](int x) {
      if (x < L) return true;
      for (int j = 0; j < m; ++j)
        if (hi[j] == x) return true;
      return false;
    };
    // walk cycles from misplaced positions, taking their high positions into the tile
    for (int start = 0; start < s->n && m < kHi; ++start) {
      if (s->p2l[start] == start || (start >= L && in_tile(start))) continue;
      int y = start;
      for (int steps = 0; steps < s->n && m < kHi; ++steps) {
        if (y >= L && !in_tile(y)) hi[m++] = y;
        y = s->l2p[y];  // the position holding the logical qubit that belongs at y
        if (y == start) break;
      }
    }
    // tile index of a physical position in the tile
    auto tile_of = [&](int x) {
      if (x < L) return x;
      for (int j = 0; j < m; ++j)
        if (hi[j] == x) return L + j;
      return -1;
    };
    int dst[16], used = 0;
    for (int b = 0; b < L + m; ++b) dst[b] = -1;
    // contents whose home is in the tile go home
    for (int b = 0; b < L + m; ++b) {
      const int x = b < L ? b : hi[b - L];
      const int home = s->p2l[x];
      if (in_tile(home)) {
        dst[b] = tile_of(home);
        used |= 1 << dst[b];
      }
    }
    // the rest fill the tile positions whose own qubit is outside the tile
    int free_pos = 0;
    for (int b = 0; b < L + m; ++b) {
      if (dst[b] >= 0) continue;
      while (free_pos < L + m && ((used >> free_pos) & 1)) ++free_pos;
      dst[b] = free_pos;
      used |= 1 << free_pos;
    }
    int64_t bytes = 0;
    QS_TRY(launch_permute(d, L, hi, m, dst, &bytes));
    apply_permute_maps(s, L, hi, m, dst);
  }
  for (int p = 0; p < s->n; ++p)
    if (s->p2l[p] != p) {
      set_error("internal: layout not restored");
      return QSIM_EINVAL;
    }
  return QSIM_OK;
}

bool identity_layout(const qsim_state *s) {
  for (int p = 0; p < s->n; ++p)
    if (s->p2l[p] != p) return false;
  return true;
}

void reset_layout(qsim_state *s) {
  for (int q = 0; q < 64; ++q) s->l2p[q] = s->p2l[q] = q;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" {

const char *qsim_last_error(void) { return qsim::last_error(); }

const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

qsim_status qsim_gate_matrix(int kind, const double *params, int *k, double *out) {
  static const double zero[4] = {0, 0, 0, 0};
  if (!out || !k) {
    set_error("NULL output");
    return QSIM_EINVAL;
  }
  std::vector<cd> m;
  const int q = named_matrix(kind, params ? params : zero, m);
  if (q < 0) {
    set_error("unknown gate kind %d", kind);
    return QSIM_EINVAL;
  }
  *k = q;
  for (size_t i = 0; i < m.size(); ++i) {
    out[2 * i] = m[i].real();
    out[2 * i + 1] = m[i].imag();
  }
  return QSIM_OK;
}

static qsim_status make_state(int n, int dtype, void *stream, void *dev_ptr, qsim_state **out) {
  if (!out) {
    set_error("out is NULL");
    return QSIM_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > QSIM_MAX_QUBITS) {
    set_error("n = %d not in [1, %d]", n, QSIM_MAX_QUBITS);
    return QSIM_EINVAL;
  }
  if (dtype != QSIM_C64 && dtype != QSIM_C128) {
    set_error("unknown dtype %d", dtype);
    return QSIM_EINVAL;
  }
  if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) & 255u)) {
    set_error("device pointer must be 256-byte aligned");
    return QSIM_EINVAL;
  }
  std::unique_ptr<qsim_state> s(new qsim_state());
  s->n = n;
  s->dtype = dtype;
  s->stream = static_cast<cudaStream_t>(stream);
  reset_layout(s.get());
  {
    const cudaError_t ee = cudaEventCreateWithFlags(&s->mat_event, cudaEventDisableTiming);
    if (ee != cudaSuccess) return cuda_fail(ee, "cudaEventCreateWithFlags");
  }
  if (dev_ptr) {
    s->amps = dev_ptr;
    s->owned = false;
  } else {
    const size_t bytes = amp_bytes(dtype) << n;
    cudaError_t e = cudaMalloc(&s->amps, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cannot allocate %zu bytes for %d qubits: %s", bytes, n, cudaGetErrorString(e));
      return QSIM_ENOMEM;
    }
    s->owned = true;
    const qsim_status st = launch_fill_zero_state(dev_of(s.get()));
    if (st != QSIM_OK) {
      cudaFree(s->amps);
      return st;
    }
  }
  *out = s.release();
  return QSIM_OK;
}

qsim_status qsim_create(int n, int dtype, void *stream, qsim_state **out) {
  return make_state(n, dtype, stream, nullptr, out);
}

qsim_status qsim_wrap(void *dev_ptr, int n, int dtype, void *stream, qsim_state **out) {
  if (!dev_ptr) {
    set_error("dev_ptr is NULL");
    return QSIM_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(dev_ptr) & 255u) {
    set_error("dev_ptr must be 256-byte aligned (vector and tensor-map accesses)");
    return QSIM_EINVAL;
  }
  return make_state(n, dtype, stream, dev_ptr, out);
}

void qsim_destroy(qsim_state *s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  if (s->owned && s->amps) cudaFree(s->amps);
  if (s->scratch) cudaFree(s->scratch);
  if (s->mat_dev) cudaFree(s->mat_dev);
  if (s->mat_host) cudaFreeHost(s->mat_host);
  if (s->mat_event) cudaEventDestroy(s->mat_event);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->norm_slots) cudaFree(s->norm_slots);
  if (s->cap_stream) {
    cudaStreamSynchronize(s->cap_stream);
    cudaStreamDestroy(s->cap_stream);
  }
  delete s;
}

qsim_status qsim_reset(qsim_state *s) {
  QS_TRY(check_state(s));
  reset_layout(s);
  s->fmt = 0;
  exact_values(s);
  return launch_fill_zero_state(dev_of(s));
}

qsim_status qsim_set_stream(qsim_state *s, void *stream) {
  QS_TRY(check_state(s));
  QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
  s->stream = static_cast<cudaStream_t>(stream);
  return QSIM_OK;
}

qsim_status qsim_synchronize(qsim_state *s) {
  QS_TRY(check_state(s));
  QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
  QS_TRY_CUDA(cudaGetLastError());
  return tc_take_timeout();
}

qsim_status qsim_canonicalize(qsim_state *s) {
  QS_TRY(check_state(s));
  QS_TRY(ensure_plain(s));
  return canonicalize(s);
}

qsim_status qsim_selftest_bounded_wait(int ms, void *stream) {
  if (ms < 1 || ms > 10000) {
    set_error("selftest wait of %d ms not in [1, 10000]", ms);
    return QSIM_EINVAL;
  }
  return tc_wait_selftest(ms, static_cast<cudaStream_t>(stream));
}

qsim_status qsim_set_option(qsim_state *s, int option, int value) {
  QS_TRY(check_state(s));
  if (option == QSIM_OPT_FP64_NATIVE) {
    if (s->dtype != QSIM_C128) return QSIM_OK;
    QS_TRY(ensure_plain(s));
    s->fp64_native = value ? 1 : 0;
    return QSIM_OK;
  }
  if (option == QSIM_OPT_TC_LO_SMEM) {
    s->tc_lo_smem = value ? 1 : 0;
    return QSIM_OK;
  }
  set_error("unknown option %d", option);
  return QSIM_EINVAL;
}

qsim_status qsim_apply_gate(qsim_state *s, const int *targets, int nt, const int *controls, int nc,
                            const double *m) {
  QS_TRY(check_state(s));
  if (nt < 1 || nt > 2 || !targets || !m || nc < 0 || (nc > 0 && !controls)) {
    set_error("apply_gate needs 1 or 2 targets, a matrix and a valid control list");
    return QSIM_EINVAL;
  }
  QS_TRY(validate_qubits(s, targets, nt, controls, nc));
  Gate g;
  g.nt = nt;
  for (int j = 0; j < nt; ++j) g.t[j] = targets[j];
  for (int j = 0; j < nc; ++j) g.ctrl.push_back(controls[j]);
  const int dim = 1 << nt;
  g.m.resize((size_t)dim * dim);
  for (int i = 0; i < dim * dim; ++i) g.m[i] = cd(m[2 * i], m[2 * i + 1]);
  QS_TRY(spend_split_sweep(s));
  QS_TRY(ensure_split(s));
  int64_t bytes = 0;
  return launch_gate_phys(dev_of(s), to_phys(s, g), &bytes);
}

qsim_status qsim_apply_fused(qsim_state *s, const int *qubits, int k, const double *u) {
  QS_TRY(check_state(s));
  if (k < 1 || k > QSIM_MAX_FUSED || !qubits || !u) {
    set_error("apply_fused needs 1..%d qubits and a matrix", QSIM_MAX_FUSED);
    return QSIM_EINVAL;
  }
  QS_TRY(validate_qubits(s, qubits, k, nullptr, 0));
  Block b;
  b.q.assign(qubits, qubits + k);
  const int dim = 1 << k;
  b.u.resize((size_t)dim * dim);
  for (int i = 0; i < dim * dim; ++i) b.u[i] = cd(u[2 * i], u[2 * i + 1]);
  std::vector<Action> acts;
  std::vector<unsigned char> mats;
  const StateDev d = dev_of(s);
  if (s->dtype == QSIM_C64 && fused_tc_supported(d, k)) {
    plan_remap_low(s, b.q, k, Upcoming{}, acts);
    for (int x : b.q)
      if (s->l2p[x] >= k) {
        set_error("internal: remap left qubit %d at position %d", x, s->l2p[x]);
        return QSIM_EINVAL;
      }
    std::vector<int> to(k);
    for (int j = 0; j < k; ++j) to[j] = s->p2l[k - 1 - j];
    std::vector<cd> up = reindex(b.u, b.q, to);
    Action a;
    a.type = Action::FUSED_TC;
    a.k = k;
    tc_identity_plan(k, a.tp);
    const size_t nf = tc_operand_floats(k);
    mats.resize(nf * sizeof(float));
    float *dst = reinterpret_cast<float *>(mats.data());
    build_tc_operands(k, up.data(), dst, dst + nf / 2);
    acts.push_back(std::move(a));
  } else {
    QS_TRY(spend_split_sweep(s));
    QS_TRY(ensure_split(s));
    Action a;
    a.type = Action::FUSED_SIMT;
    a.k = k;
    a.g.nt = k;
    for (int j = 0; j < k; ++j) a.g.t[j] = s->l2p[qubits[j]];
    if (wants_split(s)) append_fused_df(mats, b.u.data(), k, a.g.t);
    else append_cast(mats, b.u.data(), b.u.size(), s->dtype);
    acts.push_back(std::move(a));
  }
  QS_TRY(arena_upload(s, mats.data(), mats.size()));
  int64_t bytes = 0;
  return run_actions(s, acts, &bytes, s->stream);
}

qsim_status qsim_run_circuit(qsim_state *s, const qsim_op *ops, size_t nops, const qsim_run_opts *opts) {
  QS_TRY(check_state(s));
  qsim_run_opts o{};
  if (opts) o = *opts;
  std::vector<Gate> gates;
  QS_TRY(expand_ops(ops, nops, s->n, gates));
  return run_gate_list(s, gates, o);
}

}  // extern "C"

namespace qsim {

struct PreparedPlan {
  int n = 0, dtype = 0, fmt_in = 0, fmt_out = 0;
  int l2p_in[64], l2p_out[64], p2l_out[64];
  std::vector<Action> acts;  // before norm slots are assigned
  std::vector<unsigned char> mats;
  qsim_run_stats st{};
  int fuse = 0;            // the width used (the autotuner's pick for fuse < 0)
  double predicted = 0.0;  // the autotuner's predicted time
  qsim_run_opts opts{};    // the options it was planned with
  std::vector<Gate> gates; // the gate list it was planned from (qsim_run_circuit's cache)
  SegMarks seg;            // segment boundaries (prepare_segments)
};

bool same_gates(const std::vector<Gate> &a, const std::vector<Gate> &b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i) {
    const Gate &x = a[i], &y = b[i];
    if (x.nt != y.nt || x.ctrl != y.ctrl || x.m != y.m) return false;
    for (int j = 0; j < x.nt; ++j)
      if (x.t[j] != y.t[j]) return false;
  }
  return true;
}

void PreparedPlanDeleter::operator()(PreparedPlan *p) const { delete p; }

qsim_status copy_state(qsim_state *dst, const qsim_state *src) {
  if (!dst || !src || dst->n != src->n || dst->dtype != src->dtype) {
    set_error("copy_state: states differ in size or type");
    return QSIM_EINVAL;
  }
  QS_TRY_CUDA(cudaMemcpyAsync(dst->amps, src->amps, amp_bytes(src->dtype) << src->n, cudaMemcpyDeviceToDevice,
                              dst->stream));
  memcpy(dst->l2p, src->l2p, sizeof(dst->l2p));
  memcpy(dst->p2l, src->p2l, sizeof(dst->p2l));
  dst->fmt = src->fmt;
  dst->split_sweeps = src->split_sweeps;
  dst->auto_native = src->auto_native;
  return QSIM_OK;
}

qsim_status run_gate_list(qsim_state *s, const std::vector<Gate> &gates, qsim_run_opts o) {
  const qsim_run_opts opts_in = o;
  // cache key: everything the launch sequence depends on
  uint64_t key = 1469598103934665603ULL;
  {
    key = fnv(key, &s->n, sizeof(int));
    key = fnv(key, &s->dtype, sizeof(int));
    key = fnv(key, &o, sizeof(o));
    key = fnv(key, s->l2p, sizeof(int) * s->n);
    key = fnv(key, &s->amps, sizeof(void *));
    key = fnv(key, &s->fmt, sizeof(int));
    key = fnv(key, &s->fp64_native, sizeof(int));
    key = fnv(key, &s->auto_native, sizeof(int));
    key = fnv(key, &s->tc_lo_smem, sizeof(int));
    for (const Gate &g : gates) {
      key = fnv(key, &g.nt, sizeof(int));
      key = fnv(key, g.t, sizeof(int) * g.nt);
      key = fnv(key, g.ctrl.data(), sizeof(int) * g.ctrl.size());
      key = fnv(key, g.m.data(), sizeof(cd) * g.m.size());
    }
  }
  std::vector<Action> acts;
  std::vector<unsigned char> mats;
  int saved_l2p[64], saved_p2l[64];
  memcpy(saved_l2p, s->l2p, sizeof(saved_l2p));
  memcpy(saved_p2l, s->p2l, sizeof(saved_p2l));
  const int saved_fmt = s->fmt;
  qsim_run_stats st;
  double predicted = 0.0;
  const bool reuse = s->last_plan && s->last_plan_key == key && plan_matches(*s->last_plan, s) &&
                     memcmp(&s->last_plan->opts, &o, sizeof(o)) == 0 && same_gates(s->last_plan->gates, gates);
  if (reuse) {
    // the same gate list from the same layout: take the last plan instead of planning
    const PreparedPlan &P = *s->last_plan;
    acts = P.acts;
    st = P.st;
    predicted = P.predicted;
    o.fuse = P.fuse;
    memcpy(s->l2p, P.l2p_out, sizeof(s->l2p));
    memcpy(s->p2l, P.p2l_out, sizeof(s->p2l));
    s->fmt = P.fmt_out;
  }
  if (!reuse && o.fuse < 0) {
    // autotuned width: plan every candidate on the host, keep the cheapest predicted plan
    QS_TRY(autotune(s->stream));
    int best_k = 0;
    double best_ms = 1e300;
    std::vector<int> cands = {0};
    if (s->dtype == QSIM_C64) {
      cands.push_back(4);
      cands.push_back(5);
    } else if (wants_split(s)) {
      for (int kk = 2; kk <= 5; ++kk) cands.push_back(kk);
    }
    for (int kk : cands) {
      qsim_run_opts oc = o;
      oc.fuse = kk;
      std::vector<Action> ta;
      std::vector<unsigned char> tm;
      qsim_run_stats ts;
      memcpy(s->l2p, saved_l2p, sizeof(saved_l2p));
      memcpy(s->p2l, saved_p2l, sizeof(saved_p2l));
      s->fmt = saved_fmt;
      if (plan_circuit(s, gates, oc, ta, tm, ts) != QSIM_OK) continue;
      const double ms = predict_ms(s, ta, gates);
      if (ms < best_ms) {
        best_ms = ms;
        best_k = kk;
      }
    }
    memcpy(s->l2p, saved_l2p, sizeof(saved_l2p));
    memcpy(s->p2l, saved_p2l, sizeof(saved_p2l));
    s->fmt = saved_fmt;
    o.fuse = best_k;
    predicted = best_ms;
  }
  qsim_status rc = QSIM_OK;
  if (!reuse) {
    rc = plan_circuit(s, gates, o, acts, mats, st);
    if (rc == QSIM_OK) {
      PlanPtr P(new PreparedPlan());
      P->n = s->n;
      P->dtype = s->dtype;
      P->fmt_in = saved_fmt;
      P->fmt_out = s->fmt;
      memcpy(P->l2p_in, saved_l2p, sizeof(saved_l2p));
      memcpy(P->l2p_out, s->l2p, sizeof(P->l2p_out));
      memcpy(P->p2l_out, s->p2l, sizeof(P->p2l_out));
      P->acts = acts;
      P->mats = std::move(mats);
      P->st = st;
      P->fuse = o.fuse;
      P->predicted = predicted;
      P->opts = opts_in;
      P->gates = gates;
      s->last_plan = std::move(P);
      s->last_plan_key = key;
    } else {
      s->last_plan.reset();
    }
  }
  if (rc == QSIM_OK && wants_split(s)) {
    int64_t sweeps = 0;
    for (const Action &a : acts) sweeps += a.type != Action::ZERO_SLOTS && a.type != Action::TO_SPLIT;
    if (s->split_sweeps + sweeps > kSplitSweepLimit) {
      // the split format's budget would run out: this run and the rest of the state's life
      // (until it holds exact values again) take FP64 instructions
      memcpy(s->l2p, saved_l2p, sizeof(saved_l2p));
      memcpy(s->p2l, saved_p2l, sizeof(saved_p2l));
      s->fmt = saved_fmt;
      s->last_plan.reset();
      QS_TRY(ensure_plain(s));
      s->auto_native = 1;
      return run_gate_list(s, gates, opts_in);
    }
    s->split_sweeps += sweeps;
  }
  const std::vector<unsigned char> &upload = s->last_plan ? s->last_plan->mats : mats;
  if (rc == QSIM_OK) rc = assign_norm_slots(s, acts, !o.no_renorm);
  if (rc == QSIM_OK) rc = arena_upload(s, upload.data(), upload.size());
  if (rc != QSIM_OK) {
    memcpy(s->l2p, saved_l2p, sizeof(saved_l2p));
    memcpy(s->p2l, saved_p2l, sizeof(saved_p2l));
    s->fmt = saved_fmt;
    return rc;
  }
  int64_t bytes = 0;
  if (!o.use_graph) {
    rc = run_actions(s, acts, &bytes, s->stream);
  } else {
    // The legacy default stream cannot be captured: use a private blocking stream, which
    // the legacy stream orders against implicitly.
    cudaStream_t cs = s->stream;
    if (cs == nullptr || cs == cudaStreamLegacy) {
      if (!s->cap_stream) QS_TRY_CUDA(cudaStreamCreate(&s->cap_stream));
      cs = s->cap_stream;
    }
    const bool cached = s->graph && s->graph_key == key && s->graph_mat_dev == s->mat_dev &&
                        s->graph_slots == s->norm_slots;
    if (!cached) {
      if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
      }
      if (cs != s->stream) {
        // the arena upload was queued on the state's stream: order the capture after it
        QS_TRY_CUDA(cudaEventRecord(s->mat_event, s->stream));
        QS_TRY_CUDA(cudaStreamWaitEvent(cs, s->mat_event, 0));
      }
      cudaGraph_t graph = nullptr;
      QS_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      rc = run_actions(s, acts, &bytes, cs);
      const cudaError_t e = cudaStreamEndCapture(cs, &graph);
      if (rc != QSIM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      const cudaError_t ie = cudaGraphInstantiate(&s->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        s->graph = nullptr;
        return cuda_fail(ie, "cudaGraphInstantiate");
      }
      s->graph_key = key;
      s->graph_mat_dev = s->mat_dev;
      s->graph_slots = s->norm_slots;
      s->graph_bytes = bytes;
    } else {
      bytes = s->graph_bytes;
      if (cs != s->stream) {
        QS_TRY_CUDA(cudaEventRecord(s->mat_event, s->stream));
        QS_TRY_CUDA(cudaStreamWaitEvent(cs, s->mat_event, 0));
      }
    }
    QS_TRY_CUDA(cudaGraphLaunch(s->graph, cs));
  }
  if (rc != QSIM_OK) return rc;
  for (const Action &a : acts) {
    if (a.type == Action::ZERO_SLOTS) continue;
    st.kernels++;
    st.sweeps++;
    if (a.type == Action::REMAP) st.remaps++;
    if (a.type == Action::DIAG) {
      st.diag_sweeps++;
      st.diag_gates += a.m;
    }
  }
  st.bytes = (double)bytes;
  st.fuse_width = o.fuse;
  st.predicted_ms = predicted;
  st.plan_reused = reuse ? 1 : 0;
  st.fp64_fallback = s->auto_native;
  st.upload_bytes = (int64_t)upload.size();
  s->stats = st;
  return QSIM_OK;
}

qsim_status prepare_gate_list(qsim_state *s, const std::vector<Gate> &gates, qsim_run_opts o, PlanPtr &out) {
  if (o.fuse < 0 || !o.no_renorm || o.use_graph) {
    set_error("prepare_gate_list: needs a fixed width, no renormalisation and no graph");
    return QSIM_EINVAL;
  }
  PlanPtr p(new PreparedPlan());
  p->n = s->n;
  p->dtype = s->dtype;
  p->fmt_in = s->fmt;
  memcpy(p->l2p_in, s->l2p, sizeof(p->l2p_in));
  int saved_p2l[64];
  memcpy(saved_p2l, s->p2l, sizeof(saved_p2l));
  qsim_status rc = plan_circuit(s, gates, o, p->acts, p->mats, p->st);
  p->fmt_out = s->fmt;
  memcpy(p->l2p_out, s->l2p, sizeof(p->l2p_out));
  memcpy(p->p2l_out, s->p2l, sizeof(p->p2l_out));
  // planning moved the state's layout ahead: put it back, nothing has run
  memcpy(s->l2p, p->l2p_in, sizeof(s->l2p));
  memcpy(s->p2l, saved_p2l, sizeof(s->p2l));
  s->fmt = p->fmt_in;
  if (rc != QSIM_OK) return rc;
  p->st.fuse_width = o.fuse;
  for (const Action &a : p->acts) {
    p->st.kernels++;
    p->st.sweeps++;
    if (a.type == Action::REMAP) p->st.remaps++;
    if (a.type == Action::DIAG) {
      p->st.diag_sweeps++;
      p->st.diag_gates += a.m;
    }
  }
  out = std::move(p);
  return QSIM_OK;
}

qsim_status prepare_segments(qsim_state *s, const std::vector<Gate> &gates, const std::vector<size_t> &seg_begin,
                             qsim_run_opts o, PlanPtr &out) {
  if (o.fuse < 0 || !o.no_renorm || o.use_graph || seg_begin.empty() || seg_begin[0] != 0) {
    set_error("prepare_segments: needs a fixed width, no renormalisation, no graph and segment 0 at gate 0");
    return QSIM_EINVAL;
  }
  PlanPtr p(new PreparedPlan());
  p->n = s->n;
  p->dtype = s->dtype;
  p->fmt_in = s->fmt;
  memcpy(p->l2p_in, s->l2p, sizeof(p->l2p_in));
  int saved_p2l[64];
  memcpy(saved_p2l, s->p2l, sizeof(saved_p2l));
  p->seg.begin = seg_begin;
  qsim_status rc = plan_circuit(s, gates, o, p->acts, p->mats, p->st, &p->seg);
  p->fmt_out = s->fmt;
  memcpy(p->l2p_out, s->l2p, sizeof(p->l2p_out));
  memcpy(p->p2l_out, s->p2l, sizeof(p->p2l_out));
  memcpy(s->l2p, p->l2p_in, sizeof(s->l2p));
  memcpy(s->p2l, saved_p2l, sizeof(s->p2l));
  s->fmt = p->fmt_in;
  if (rc != QSIM_OK) return rc;
  if (p->seg.act.size() != seg_begin.size() + 1) {
    set_error("internal: segment marks");
    return QSIM_EINVAL;
  }
  out = std::move(p);
  return QSIM_OK;
}

qsim_status run_prepared_segment(qsim_state *s, const PreparedPlan &p, int i, bool upload) {
  const SegMarks &m = p.seg;
  if (i < 0 || (size_t)i + 1 >= m.act.size() || p.n != s->n || p.dtype != s->dtype ||
      s->fmt != (i == 0 ? p.fmt_in : p.fmt_out) || memcmp(m.l2p[i].data(), s->l2p, sizeof(int) * s->n) != 0) {
    set_error("run_prepared_segment: the state is not where segment %d of the plan starts", i);
    return QSIM_EINVAL;
  }
  if (upload) QS_TRY(arena_upload(s, p.mats.data(), p.mats.size()));
  memcpy(s->l2p, m.l2p[i + 1].data(), sizeof(s->l2p));
  memcpy(s->p2l, m.p2l[i + 1].data(), sizeof(s->p2l));
  s->fmt = p.fmt_out;
  if (m.act[i + 1] == m.act[i]) return QSIM_OK;
  const std::vector<Action> part(p.acts.begin() + (ptrdiff_t)m.act[i], p.acts.begin() + (ptrdiff_t)m.act[i + 1]);
  int64_t bytes = 0;
  QS_TRY(run_actions(s, part, &bytes, s->stream));
  return QSIM_OK;
}

void segment_counts(const PreparedPlan &p, std::vector<int64_t> &sweeps, std::vector<int64_t> &remaps) {
  const SegMarks &m = p.seg;
  const size_t ns = m.act.empty() ? 0 : m.act.size() - 1;
  sweeps.assign(ns, 0);
  remaps.assign(ns, 0);
  for (size_t i = 0; i < ns; ++i)
    for (size_t a = m.act[i]; a < m.act[i + 1]; ++a) {
      if (p.acts[a].type == Action::ZERO_SLOTS) continue;
      sweeps[i]++;
      if (p.acts[a].type == Action::REMAP) remaps[i]++;
    }
}

qsim_status dry_plan_segments(int n, int dtype, const std::vector<Gate> &gates, const std::vector<size_t> &seg_begin,
                              qsim_run_opts o, std::vector<int64_t> &sweeps, std::vector<int64_t> &remaps) {
  qsim_state s;
  s.n = n;
  s.dtype = dtype;
  reset_layout(&s);
  PreparedPlan p;
  p.seg.begin = seg_begin;
  g_force_tc = true;
  const qsim_status rc = plan_circuit(&s, gates, o, p.acts, p.mats, p.st, &p.seg);
  g_force_tc = false;
  if (rc != QSIM_OK) return rc;
  segment_counts(p, sweeps, remaps);
  return QSIM_OK;
}

bool plan_matches(const PreparedPlan &p, const qsim_state *s) {
  return p.n == s->n && p.dtype == s->dtype && p.fmt_in == s->fmt &&
         memcmp(p.l2p_in, s->l2p, sizeof(int) * s->n) == 0;
}

qsim_status run_prepared(qsim_state *s, const PreparedPlan &p) {
  if (!plan_matches(p, s)) {
    set_error("run_prepared: the state's layout differs from the plan's");
    return QSIM_EINVAL;
  }
  QS_TRY(arena_upload(s, p.mats.data(), p.mats.size()));
  // as after planning in qsim_run_circuit: the state takes the exit layout and format,
  // then the actions (physical, a leading TO_SPLIT included) run
  memcpy(s->l2p, p.l2p_out, sizeof(s->l2p));
  memcpy(s->p2l, p.p2l_out, sizeof(s->p2l));
  s->fmt = p.fmt_out;
  int64_t bytes = 0;
  QS_TRY(run_actions(s, p.acts, &bytes, s->stream));
  s->stats = p.st;
  s->stats.bytes = (double)bytes;
  return QSIM_OK;
}

}  // namespace qsim

extern "C" {

qsim_status qsim_expand(int n, const qsim_op *ops, size_t nops, qsim_gate_rec *gates, size_t gate_cap,
                        int32_t *ctrls, size_t ctrl_cap, double *mats, size_t mat_cap, size_t sizes[3]) {
  if (!sizes || n < 1 || n > 64) {
    set_error("expand: bad n (%d) or NULL sizes", n);
    return QSIM_EINVAL;
  }
  std::vector<Gate> gl;
  QS_TRY(expand_ops(ops, nops, n, gl));
  size_t nc = 0, nm = 0;
  for (const Gate &g : gl) {
    nc += g.ctrl.size();
    nm += g.m.size();
  }
  sizes[0] = gl.size();
  sizes[1] = nc;
  sizes[2] = nm;
  if (!gates && !ctrls && !mats) return QSIM_OK;  // size query
  if (!gates || gate_cap < gl.size() || (nc && (!ctrls || ctrl_cap < nc)) || (nm && (!mats || mat_cap < nm))) {
    set_error("expand: output arrays too small (need %zu gates, %zu controls, %zu matrix entries)", gl.size(),
              nc, nm);
    return QSIM_EINVAL;
  }
  size_t co = 0, mo = 0;
  for (size_t i = 0; i < gl.size(); ++i) {
    const Gate &g = gl[i];
    qsim_gate_rec &r = gates[i];
    r.kind = g.kind;
    r.nt = g.nt;
    for (int j = 0; j < QSIM_MAX_FUSED; ++j) r.targets[j] = j < g.nt ? g.t[j] : -1;
    r.nc = (int32_t)g.ctrl.size();
    r.ctrl_off = (int32_t)co;
    r.mat_off = (int64_t)mo;
    for (int c : g.ctrl) ctrls[co++] = c;
    for (const cd &z : g.m) {
      mats[2 * mo] = z.real();
      mats[2 * mo + 1] = z.imag();
      ++mo;
    }
  }
  return QSIM_OK;
}

qsim_status qsim_plan_dry_run(int n, int dtype, const qsim_op *ops, size_t nops, const qsim_run_opts *opts,
                              qsim_run_stats *out) {
  if (!out || n < 1 || n > QSIM_MAX_QUBITS || (dtype != QSIM_C64 && dtype != QSIM_C128)) {
    set_error("plan_dry_run: bad arguments");
    return QSIM_EINVAL;
  }
  qsim_run_opts o{};
  if (opts) o = *opts;
  if (o.fuse < 0) o.fuse = 5;
  std::vector<Gate> gates;
  QS_TRY(expand_ops(ops, nops, n, gates));
  qsim_state s;
  s.n = n;
  s.dtype = dtype;
  reset_layout(&s);
  std::vector<Action> acts;
  std::vector<unsigned char> mats;
  qsim_run_stats st;
  g_force_tc = true;
  const qsim_status rc = plan_circuit(&s, gates, o, acts, mats, st);
  g_force_tc = false;
  if (rc != QSIM_OK) return rc;
  for (const Action &a : acts) {
    if (a.type == Action::ZERO_SLOTS) continue;
    st.kernels++;
    st.sweeps++;
    if (a.type == Action::REMAP) st.remaps++;
    if (a.type == Action::DIAG) {
      st.diag_sweeps++;
      st.diag_gates += a.m;
    }
  }
  st.fuse_width = o.fuse;
  *out = st;
  return QSIM_OK;
}

qsim_status qsim_last_run_stats(qsim_state *s, qsim_run_stats *out) {
  QS_TRY(check_state(s));
  if (!out) {
    set_error("out is NULL");
    return QSIM_EINVAL;
  }
  *out = s->stats;
  return QSIM_OK;
}

qsim_status qsim_amplitude(qsim_state *s, uint64_t index, double out[2]) {
  QS_TRY(check_state(s));
  if (!out || (s->n < 64 && index >> s->n)) {
    set_error("index out of range or NULL output");
    return QSIM_EINVAL;
  }
  uint64_t phys = 0;
  for (int q = 0; q < s->n; ++q)
    if (index >> q & 1ULL) phys |= 1ULL << s->l2p[q];
  if (s->dtype == QSIM_C128 && s->fmt == 1) {
    float v[4];  // split: (re_hi, im_hi, re_lo, im_lo)
    QS_TRY_CUDA(cudaMemcpyAsync(v, static_cast<double *>(s->amps) + 2 * phys, 16, cudaMemcpyDeviceToHost, s->stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = (double)v[0] + (double)v[2];
    out[1] = (double)v[1] + (double)v[3];
  } else if (s->dtype == QSIM_C128) {
    double v[2];
    QS_TRY_CUDA(cudaMemcpyAsync(v, static_cast<double *>(s->amps) + 2 * phys, 16, cudaMemcpyDeviceToHost, s->stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = v[0];
    out[1] = v[1];
  } else {
    float v[2];
    QS_TRY_CUDA(cudaMemcpyAsync(v, static_cast<float *>(s->amps) + 2 * phys, 8, cudaMemcpyDeviceToHost, s->stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = v[0];
    out[1] = v[1];
  }
  return QSIM_OK;
}

qsim_status qsim_probabilities(qsim_state *s, const int *qubits, int m, double *out) {
  QS_TRY(check_state(s));
  if (m < 1 || m > 24 || m > s->n || !qubits || !out) {
    set_error("probabilities needs 1..24 listed qubits and an output array");
    return QSIM_EINVAL;
  }
  QS_TRY(validate_qubits(s, qubits, m, nullptr, 0));
  QS_TRY(ensure_scratch(s));
  QS_TRY(ensure_plain(s));
  int phys[24];
  for (int j = 0; j < m; ++j) phys[j] = s->l2p[qubits[j]];
  return red_probs(dev_of(s), phys, m, s->scratch, out);
}

qsim_status qsim_measure(qsim_state *s, int qubit, double u, int *outcome, double *prob) {
  QS_TRY(check_state(s));
  if (!outcome || !(u >= 0.0 && u < 1.0)) {
    set_error("measure needs an outcome pointer and u in [0, 1)");
    return QSIM_EINVAL;
  }
  QS_TRY(validate_qubits(s, &qubit, 1, nullptr, 0));
  double p[2];
  QS_TRY(qsim_probabilities(s, &qubit, 1, p));
  const double tot = p[0] + p[1];
  if (!(tot > 0.0)) {
    set_error("measure: the state has zero norm");
    return QSIM_EINVAL;
  }
  const int r = u * tot < p[0] ? 0 : 1;
  // project onto the outcome and renormalise: diag(1/sqrt(p0), 0) or diag(0, 1/sqrt(p1))
  Gate g;
  g.nt = 1;
  g.t[0] = qubit;
  g.m = {cd(r == 0 ? 1.0 / std::sqrt(p[0]) : 0.0, 0.0), cd(0.0, 0.0), cd(0.0, 0.0),
         cd(r == 1 ? 1.0 / std::sqrt(p[1]) : 0.0, 0.0)};
  QS_TRY(ensure_split(s));
  int64_t bytes = 0;
  QS_TRY(launch_gate_phys(dev_of(s), to_phys(s, g), &bytes));
  *outcome = r;
  if (prob) *prob = p[r] / tot;
  return QSIM_OK;
}

qsim_status qsim_sample(qsim_state *s, const int *qubits, int m, uint64_t shots, uint64_t seed, uint64_t *out) {
  QS_TRY(check_state(s));
  if ((shots > 0 && !out) || m < 0 || m > s->n || (m > 0 && !qubits)) {
    set_error("bad sample arguments");
    return QSIM_EINVAL;
  }
  if (m > 0) QS_TRY(validate_qubits(s, qubits, m, nullptr, 0));
  if (shots == 0) return QSIM_OK;
  QS_TRY(ensure_scratch(s));
  QS_TRY(ensure_plain(s));
  if (!identity_layout(s)) QS_TRY(canonicalize(s));
  QS_TRY(red_sample_seeded(dev_of(s), seed, shots, s->scratch, out));
  if (m > 0) {
    for (uint64_t j = 0; j < shots; ++j) {
      uint64_t v = 0;
      for (int t = 0; t < m; ++t) v = (v << 1) | ((out[j] >> qubits[t]) & 1ULL);
      out[j] = v;
    }
  }
  return QSIM_OK;
}

qsim_status qsim_norm(qsim_state *s, double *out) {
  QS_TRY(check_state(s));
  if (!out) {
    set_error("out is NULL");
    return QSIM_EINVAL;
  }
  QS_TRY(ensure_scratch(s));
  QS_TRY(ensure_plain(s));
  return red_norm(dev_of(s), s->scratch, out);
}

qsim_status qsim_inner(qsim_state *a, qsim_state *b, double out[2]) {
  QS_TRY(check_state(a));
  QS_TRY(check_state(b));
  if (!out || a->n != b->n || a->dtype != b->dtype) {
    set_error("inner product needs two states of the same size and dtype");
    return QSIM_EINVAL;
  }
  if (b->stream != a->stream) QS_TRY_CUDA(cudaStreamSynchronize(b->stream));
  QS_TRY(ensure_plain(a));
  QS_TRY(ensure_plain(b));
  if (!identity_layout(a)) QS_TRY(canonicalize(a));
  if (!identity_layout(b)) {
    QS_TRY(canonicalize(b));
    if (b->stream != a->stream) QS_TRY_CUDA(cudaStreamSynchronize(b->stream));
  }
  QS_TRY(ensure_scratch(a));
  return red_inner(dev_of(a), b->amps, a->scratch, out);
}

qsim_status qsim_fidelity(qsim_state *a, qsim_state *b, double *out) {
  if (!out) {
    set_error("out is NULL");
    return QSIM_EINVAL;
  }
  double ab[2], na, nb;
  QS_TRY(qsim_inner(a, b, ab));
  QS_TRY(qsim_norm(a, &na));
  QS_TRY(qsim_norm(b, &nb));
  *out = (ab[0] * ab[0] + ab[1] * ab[1]) / (na * nb);
  return QSIM_OK;
}

qsim_status qsim_expect_z(qsim_state *s, double *out) {
  QS_TRY(check_state(s));
  if (!out) {
    set_error("out is NULL");
    return QSIM_EINVAL;
  }
  QS_TRY(ensure_scratch(s));
  QS_TRY(ensure_plain(s));
  double total = 0.0, p1[QSIM_MAX_QUBITS];
  QS_TRY(red_p1_all(dev_of(s), s->scratch, &total, p1));
  for (int q = 0; q < s->n; ++q) out[q] = (total - 2.0 * p1[s->l2p[q]]) / total;
  return QSIM_OK;
}

qsim_status qsim_copy_to_host(qsim_state *s, void *host) {
  QS_TRY(check_state(s));
  if (!host) {
    set_error("host is NULL");
    return QSIM_EINVAL;
  }
  QS_TRY(ensure_plain(s));
  if (!identity_layout(s)) QS_TRY(canonicalize(s));
  QS_TRY_CUDA(cudaMemcpyAsync(host, s->amps, amp_bytes(s->dtype) << s->n, cudaMemcpyDeviceToHost, s->stream));
  QS_TRY_CUDA(cudaStreamSynchronize(s->stream));
  return QSIM_OK;
}

qsim_status qsim_copy_to_host_async(qsim_state *s, void *host) {
  QS_TRY(check_state(s));
  if (!host) {
    set_error("host is NULL");
    return QSIM_EINVAL;
  }
  QS_TRY(ensure_plain(s));
  if (!identity_layout(s)) QS_TRY(canonicalize(s));
  QS_TRY_CUDA(cudaMemcpyAsync(host, s->amps, amp_bytes(s->dtype) << s->n, cudaMemcpyDeviceToHost, s->stream));
  return QSIM_OK;
}

qsim_status qsim_copy_from_host(qsim_state *s, const void *host) {
  QS_TRY(check_state(s));
  if (!host) {
    set_error("host is NULL");
    return QSIM_EINVAL;
  }
  reset_layout(s);
  s->fmt = 0;
  exact_values(s);
  QS_TRY_CUDA(cudaMemcpyAsync(s->amps, host, amp_bytes(s->dtype) << s->n, cudaMemcpyHostToDevice, s->stream));
  return QSIM_OK;
}

}  // extern "C"
