// Partial amplitude mode (Section 2.2, Eq. 4).
//
// The dividing line splits an n-qubit circuit into the upper block (qubits [0, cut)) and
// the lower block ([cut, n)). A gate across the line must be a controlled gate: its
// targets on one side, its controls C on the other split it by Eq. 4 (extended to several
// controls) into (I - P_C) (x) I + P_C (x) U, P_C the projector on C = 1...1. With c such
// gates the state is a sum of 2^c products, psi = sum_b upper_b (x) lower_b, and an
// amplitude is <x|psi> = sum_b upper_b[x mod 2^cut] lower_b[x >> cut].
//
// GPU organisation: the 2^(c+1) sub-circuits share prefixes. Between two decomposed gates
// a block's gates are a segment; branch b's sub-circuit is segment 0, the term of bit 0,
// segment 1, ... A depth-first walk over the branch bits keeps one state pair per level
// (c + 1 pairs): at level k the pair is copied (device to device), one copy takes term 1
// and the other term 0 (single-gate sweeps), and each continues with segment k + 1
// through the full-amplitude engine (fused sweeps; each block's segments are one plan).
// Segment s then runs 2^s times instead of 2^c. At each leaf one gather kernel adds
// upper[x_u] * lower[x_l] into an FP64 accumulator per requested index.
#include <algorithm>
#include <functional>
#include <vector>

#include "internal.h"

namespace qsim {

namespace {

struct Crossing {
  int far_side;                // block that holds the controls across the line
  std::vector<Gate> term0;     // far side, bit 0: I - P_C
  std::vector<Gate> term1;     // far side, bit 1: P_C
  Gate target;                 // target side, bit 1: the gate with its near-side controls
};

struct PartialPlan {
  int cut = 0, c = 0;
  std::vector<std::vector<Gate>> seg[2];  // seg[side][s]: gates after crossing s - 1
  std::vector<Crossing> cross;
};

// If g's matrix has the form P0 (x) I + P1 (x) U' in its first (most significant) target,
// turn that target into a control and keep U'.
bool peel_first_target(Gate &g) {
  if (g.nt < 2) return false;
  const int D = 1 << g.nt, d = D / 2;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const bool top = r < d, left = c < d;
      const cd v = g.m[(size_t)r * D + c];
      if (top && left) {
        if (std::abs(v - cd(r == c ? 1.0 : 0.0, 0.0)) > 1e-14) return false;
      } else if (top != left) {
        if (std::abs(v) > 1e-14) return false;
      }
    }
  std::vector<cd> u((size_t)d * d);
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) u[(size_t)r * d + c] = g.m[(size_t)(r + d) * D + (c + d)];
  g.ctrl.push_back(g.t[0]);
  for (int j = 1; j < g.nt; ++j) g.t[j - 1] = g.t[j];
  g.nt -= 1;
  g.m.swap(u);
  return true;
}

Gate diag1(int q, cd a, cd b, std::vector<int> ctrl) {
  Gate g;
  g.nt = 1;
  g.t[0] = q;
  g.ctrl = std::move(ctrl);
  g.m = {a, cd(0, 0), cd(0, 0), b};
  return g;
}

qsim_status make_plan(int n, const qsim_op *ops, size_t nops, int cut, PartialPlan &P) {
  if (n < 2 || n > 64) {
    set_error("partial mode: n = %d not in [2, 64]", n);
    return QSIM_EINVAL;
  }
  if (cut == 0) cut = n / 2;
  if (cut < 1 || cut >= n || cut > QSIM_MAX_QUBITS || n - cut > QSIM_MAX_QUBITS) {
    set_error("partial mode: cut %d leaves a block outside [1, %d] qubits", cut, QSIM_MAX_QUBITS);
    return QSIM_EINVAL;
  }
  std::vector<Gate> gates;
  QS_TRY(expand_ops(ops, nops, n, gates));
  P.cut = cut;
  P.c = 0;
  P.seg[0].assign(1, {});
  P.seg[1].assign(1, {});
  P.cross.clear();
  auto side = [cut](int q) { return q < cut ? 0 : 1; };
  auto local = [cut](int q) { return q < cut ? q : q - cut; };
  for (size_t gi = 0; gi < gates.size(); ++gi) {
    Gate g = gates[gi];
    int seen[2] = {0, 0};
    for (int j = 0; j < g.nt; ++j) seen[side(g.t[j])] = 1;
    for (int q : g.ctrl) seen[side(q)] = 1;
    if (!(seen[0] && seen[1])) {
      const int s = seen[0] ? 0 : 1;
      for (int j = 0; j < g.nt; ++j) g.t[j] = local(g.t[j]);
      for (int &q : g.ctrl) q = local(q);
      P.seg[s].back().push_back(std::move(g));
      continue;
    }
    // targets across the line: take them as controls, in listed order, while the matrix
    // has the controlled form
    for (;;) {
      int ts[2] = {0, 0};
      for (int j = 0; j < g.nt; ++j) ts[side(g.t[j])] = 1;
      if (!(ts[0] && ts[1])) break;
      if (!peel_first_target(g)) {
        set_error("gate %zu crosses the dividing line and is not a controlled gate", gi);
        return QSIM_EUNSUPPORTED;
      }
    }
    const int tside = side(g.t[0]);
    std::vector<int> far, near;
    for (int q : g.ctrl) (side(q) == tside ? near : far).push_back(local(q));
    Crossing X;
    X.far_side = 1 - tside;
    // I - P_C: diag(1, 0) on far[0], controlled by the other far qubits
    X.term0.push_back(diag1(far[0], cd(1, 0), cd(0, 0), std::vector<int>(far.begin() + 1, far.end())));
    for (int q : far) X.term1.push_back(diag1(q, cd(0, 0), cd(1, 0), {}));
    X.target = g;
    for (int j = 0; j < X.target.nt; ++j) X.target.t[j] = local(X.target.t[j]);
    X.target.ctrl = near;
    P.cross.push_back(std::move(X));
    P.seg[0].push_back({});
    P.seg[1].push_back({});
    P.c += 1;
  }
  if (P.c > 30) {
    set_error("partial mode: %d decomposed gates (2^%d sub-circuit pairs) is too many", P.c, P.c);
    return QSIM_EUNSUPPORTED;
  }
  return QSIM_OK;
}

// one block's segments as a gate list and the first gate of each segment
void block_gates(const PartialPlan &P, int side, std::vector<Gate> &all, std::vector<size_t> &begin) {
  all.clear();
  begin.clear();
  for (int sg = 0; sg <= P.c; ++sg) {
    begin.push_back(all.size());
    all.insert(all.end(), P.seg[side][sg].begin(), P.seg[side][sg].end());
  }
}

// segment s of each block runs 2^s times over the walk
int64_t walk_total(const std::vector<int64_t> &per_seg) {
  int64_t t = 0;
  for (size_t sg = 0; sg < per_seg.size(); ++sg) t += per_seg[sg] << sg;
  return t;
}

void fill_info(const PartialPlan &P, qsim_partial_info *info, int64_t runs, double gates_applied, int64_t sweeps,
               int64_t remaps) {
  if (!info) return;
  info->sweeps = sweeps;
  info->remaps = remaps;
  double branch = 0.0;  // gates of one branch pair: every segment plus the terms it takes
  for (int s = 0; s <= P.c; ++s) branch += (double)(P.seg[0][s].size() + P.seg[1][s].size());
  double terms = 0.0;  // summed over both values of each bit
  for (const Crossing &X : P.cross) terms += (double)(X.term0.size() + X.term1.size() + 1);
  info->gates_unshared = (double)(1LL << P.c) * branch + (double)(1LL << P.c) * terms / 2.0;
  info->cut = P.cut;
  info->decomposed = P.c;
  info->subcircuits = 2LL << P.c;
  info->segment_runs = runs;
  info->slots = P.c + 1;
  info->gates_applied = gates_applied;
}

struct GatherSide {
  const void *amps;
  int fmt;  // 0 complex64, 1 complex128, 2 complex128 split (re_hi, im_hi, re_lo, im_lo)
  int n;
  int l2p[QSIM_MAX_QUBITS];
};

__device__ __forceinline__ double2 load_amp(const GatherSide &S, unsigned long long x) {
  unsigned long long p = 0;
  for (int q = 0; q < S.n; ++q)
    if ((x >> q) & 1ULL) p |= 1ULL << S.l2p[q];
  if (S.fmt == 0) {
    const float2 v = static_cast<const float2 *>(S.amps)[p];
    return make_double2(v.x, v.y);
  }
  if (S.fmt == 1) return static_cast<const double2 *>(S.amps)[p];
  const float4 v = static_cast<const float4 *>(S.amps)[p];
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// acc[i] += upper[idx[i] mod 2^cut] * lower[idx[i] >> cut] in FP64
__global__ void k_partial_gather(const unsigned long long *idx, long long m, int cut, GatherSide U, GatherSide L,
                                 double2 *acc) {
  const unsigned long long mask = (1ULL << cut) - 1ULL;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long x = idx[i];
    const double2 a = load_amp(U, x & mask), b = load_amp(L, x >> cut);
    double2 s = acc[i];
    s.x += a.x * b.x - a.y * b.y;
    s.y += a.x * b.y + a.y * b.x;
    acc[i] = s;
  }
}

GatherSide side_of(const qsim_state *s) {
  GatherSide g;
  g.amps = s->amps;
  g.fmt = s->dtype == QSIM_C64 ? 0 : (s->fmt == 1 ? 2 : 1);
  g.n = s->n;
  for (int q = 0; q < QSIM_MAX_QUBITS; ++q) g.l2p[q] = q < s->n ? s->l2p[q] : 0;
  return g;
}

}  // namespace

}  // namespace qsim

using namespace qsim;

extern "C" qsim_status qsim_partial_plan(int n, const qsim_op *ops, size_t nops, int cut, qsim_partial_info *info) {
  PartialPlan P;
  QS_TRY(make_plan(n, ops, nops, cut, P));
  int64_t runs = 0;
  double gates = 0.0;
  for (int s = 0; s <= P.c; ++s) {
    runs += 2LL << s;  // both blocks
    gates += (double)(1LL << s) * (double)(P.seg[0][s].size() + P.seg[1][s].size());
    if (s > 0) {
      const Crossing &X = P.cross[s - 1];
      gates += (double)(1LL << (s - 1)) * (double)(X.term0.size() + X.term1.size() + 1);
    }
  }
  int64_t sweeps = 0, remaps = 0;
  qsim_run_opts ro{};
  ro.fuse = 5;
  ro.remap = 1;
  ro.no_renorm = 1;
  for (int side = 0; side < 2; ++side) {
    std::vector<Gate> all;
    std::vector<size_t> begin;
    block_gates(P, side, all, begin);
    if (all.empty()) continue;
    std::vector<int64_t> sw, rm;
    QS_TRY(dry_plan_segments(side == 0 ? P.cut : n - P.cut, QSIM_C64, all, begin, ro, sw, rm));
    sweeps += walk_total(sw);
    remaps += walk_total(rm);
  }
  fill_info(P, info, runs, gates, sweeps, remaps);
  return QSIM_OK;
}

extern "C" qsim_status qsim_partial_amplitudes(int n, const qsim_op *ops, size_t nops, const qsim_partial_opts *opts,
                                               const uint64_t *indices, size_t m, double *amps_out,
                                               qsim_partial_info *info, void *stream) {
  qsim_partial_opts o{};
  if (opts) o = *opts;
  if (o.dtype != QSIM_C64 && o.dtype != QSIM_C128) {
    set_error("partial mode: unknown dtype %d", o.dtype);
    return QSIM_EINVAL;
  }
  if (m > 0 && (!indices || !amps_out)) {
    set_error("partial mode: NULL indices or output");
    return QSIM_EINVAL;
  }
  PartialPlan P;
  QS_TRY(make_plan(n, ops, nops, o.cut, P));
  for (size_t i = 0; i < m; ++i)
    if (n < 64 && (indices[i] >> n)) {
      set_error("partial mode: index %zu out of range", i);
      return QSIM_EINVAL;
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  qsim_run_opts ro{};
  ro.fuse = o.fuse;
  ro.remap = o.remap;
  ro.no_renorm = 1;  // the projections change the norm
  const int w[2] = {P.cut, n - P.cut};

  unsigned long long *d_idx = nullptr;
  double2 *d_acc = nullptr;
  std::vector<qsim_state *> slot[2];
  slot[0].assign(P.c + 1, nullptr);
  slot[1].assign(P.c + 1, nullptr);
  auto cleanup = [&]() {
    for (int s = 0; s < 2; ++s)
      for (qsim_state *x : slot[s])
        if (x) qsim_destroy(x);
    if (d_idx) cudaFreeAsync(d_idx, st);
    if (d_acc) cudaFreeAsync(d_acc, st);
  };
  qsim_status rc = QSIM_OK;
  const size_t mm = m > 0 ? m : 1;
  {
    cudaError_t e = cudaMallocAsync((void **)&d_idx, sizeof(unsigned long long) * mm, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_acc, sizeof(double2) * mm, st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(d_idx, indices, sizeof(uint64_t) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, sizeof(double2) * mm, st);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "partial mode buffers");
    }
  }
  int64_t runs = 0, plan_sweeps = 0, plan_remaps = 0;
  double gates_applied = 0.0;
  // Each block's segments are planned once, as one plan (fused blocks never mix two
  // segments, and a segment's last epilogue already moves the next one's qubits). The terms
  // run between segments as single-gate sweeps, which keep the qubit layout, so every
  // branch enters segment s in the layout the plan has there, and all 2^s runs share it.
  qsim_run_opts ro_terms{};
  ro_terms.no_renorm = 1;
  PlanPtr splan[2];
  std::vector<char> uploaded[2];  // the slot's arena holds its block's plan matrices
  uploaded[0].assign(P.c + 1, 0);
  uploaded[1].assign(P.c + 1, 0);
  auto run_on = [&](int side, int segi, int sl, const std::vector<Gate> &pre) -> qsim_status {
    qsim_state *s = slot[side][sl];
    const std::vector<Gate> &seg = P.seg[side][segi];
    ++runs;
    gates_applied += (double)(pre.size() + seg.size());
    if (!pre.empty()) {
      QS_TRY(run_gate_list(s, pre, ro_terms));
      for (const Gate &g : pre)
        if (g.nt > 2) uploaded[side][sl] = 0;  // its matrix went through the arena
    }
    if (!splan[side]) return seg.empty() ? QSIM_OK : run_gate_list(s, seg, ro);
    QS_TRY(run_prepared_segment(s, *splan[side], segi, !uploaded[side][sl]));
    uploaded[side][sl] = 1;
    return QSIM_OK;
  };
  auto ensure = [&](int side, int k) -> qsim_status {
    if (!slot[side][k]) QS_TRY(qsim_create(w[side], o.dtype, stream, &slot[side][k]));
    return QSIM_OK;
  };
  auto gather = [&](int sl) -> qsim_status {
    if (m == 0) return QSIM_OK;
    const int grid = (int)std::min<long long>(((long long)m + 255) / 256, (long long)num_sms() * 8);
    k_partial_gather<<<grid, 256, 0, st>>>(d_idx, (long long)m, P.cut, side_of(slot[0][sl]), side_of(slot[1][sl]),
                                           d_acc);
    QS_TRY_CUDA(cudaGetLastError());
    return QSIM_OK;
  };
  // depth-first over the branch bits: the pair in slot `sl` holds both blocks after
  // segment k of the current prefix. The bit-1 branch continues in a copy one slot up,
  // the bit-0 branch in place, so slot sl <= k and c + 1 slots suffice.
  const std::vector<Gate> none;
  std::function<qsim_status(int, int)> walk = [&](int k, int sl) -> qsim_status {
    if (k == P.c) return gather(sl);
    const Crossing &X = P.cross[k];
    const std::vector<Gate> tgt(1, X.target);
    for (int side = 0; side < 2; ++side) {
      QS_TRY(ensure(side, sl + 1));
      QS_TRY(copy_state(slot[side][sl + 1], slot[side][sl]));
      // bit 1: P_C on the far block, the gate on the target block
      QS_TRY(run_on(side, k + 1, sl + 1, side == X.far_side ? X.term1 : tgt));
    }
    QS_TRY(walk(k + 1, sl + 1));
    // bit 0: I - P_C on the far block, nothing on the target block
    for (int side = 0; side < 2; ++side)
      QS_TRY(run_on(side, k + 1, sl, side == X.far_side ? X.term0 : none));
    return walk(k + 1, sl);
  };
  for (int side = 0; side < 2 && rc == QSIM_OK; ++side) {
    rc = ensure(side, 0);
    if (rc == QSIM_OK && ro.fuse >= 0) {
      std::vector<Gate> all;
      std::vector<size_t> begin;
      block_gates(P, side, all, begin);
      if (!all.empty()) rc = prepare_segments(slot[side][0], all, begin, ro, splan[side]);
      if (rc == QSIM_OK && splan[side]) {
        std::vector<int64_t> sw, rm;
        segment_counts(*splan[side], sw, rm);
        plan_sweeps += walk_total(sw);
        plan_remaps += walk_total(rm);
      }
    }
    if (rc == QSIM_OK) rc = run_on(side, 0, 0, {});
  }
  if (rc == QSIM_OK) rc = walk(0, 0);
  if (rc == QSIM_OK && m) {
    const cudaError_t e = cudaMemcpyAsync(amps_out, d_acc, sizeof(double2) * m, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "partial mode read-back");
  }
  if (rc == QSIM_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "partial mode");
  }
  cleanup();
  if (rc == QSIM_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "partial mode free");
  }
  fill_info(P, info, runs, gates_applied, plan_sweeps, plan_remaps);
  return rc;
}
