// Batched noisy Monte-Carlo trajectories (Section 2.4, the six Kraus sets of Eq. 5) in one
// persistent launch.
//
// Every trajectory evolves a complex64 state |0...0> through its program's gates. After
// each noisy gate, for each qubit the gate touches (ascending) and each enabled channel in
// channel order, a branch K_i is chosen with probability ||K_i psi||^2 / ||psi||^2 from
// the draw u = U01(Philox4x32-10(key = seed, counter = (trajectory, gate, qubit,
// channel))) (smallest i with u < p_1 + ... + p_i), and psi <- K_i psi / ||K_i psi||; or,
// for a two-qubit gate in Kronecker mode, one draw per channel over the products
// K_i (x) K_j. Every Eq. 5 operator has at most one non-zero entry per row and column, so
// K^dag K is diagonal: the branch weights follow from the populations of the gate's
// sectors. Depolarizing and the flips are multiples of unitaries with state-independent
// weights (the unitary is applied as it is); the two damping channels have K1 = diag(1,
// sqrt(1-p)), whose weight is at least 1 - p whatever the state.
//
// Device organisation: one 512-thread CTA per SM takes trajectories from an atomic work
// counter, widest first. A state of up to 14 qubits (128 KiB) lives in shared memory, a
// wider one in the CTA's slice of a global buffer (L2 / HBM). A gate whose damping draws
// could depend on the state (u >= 1 - p, rare) takes a read-only pass that sums
// |(U psi)_i|^2 over the sectors of the gate's qubits (FP32 Neumaier sums per thread,
// FP64 across threads). Thread 0 then draws the branches, tracks how each choice changes
// the sector sums, and folds the Paulis, the Kraus operators and the renormalisation into
// one small matrix M = c K ... P U, which one pass applies (entries carried as hi + lo
// floats). Other gates skip the sums and apply K1 unnormalised. No CTA ever waits on
// another.
// After the last gate the CTA writes <Z_q> for every qubit and, for the first `shots`
// trajectories, one sample drawn with counter (trajectory, gates, 0, 0x53414D50).
#include <algorithm>
#include <vector>

#include "internal.h"
#include "philox.cuh"
#include "planner.h"

namespace qsim {

namespace {

constexpr int kTT = 512;             // threads per CTA
constexpr int kSmemQubits = 14;      // states up to this width stay in shared memory
constexpr int kMaxW = QSIM_TRAJ_MAX_QUBITS;
constexpr int kUnroll = 2;           // items per thread per step of a pass

struct DGate {
  int ns;       // 1 or 2 qubits touched
  int s0, s1;   // touched qubits, s0 < s1; sector index bit j <-> s_j
  int noisy;    // the channels run after this gate
  double m[32]; // 2^ns x 2^ns complex (re, im) in sector order, row-major over 4 x 4
};

struct TrajArgs {
  const DGate *gates;
  const int *prog_off, *prog_len, *prog_w;
  const int *traj_prog, *order;
  int ntraj;
  const unsigned long long *seed;  // Philox key (host-mapped word, read at launch)
  unsigned channels;  // bit c: channel c runs
  int kron;           // joint draws for two-qubit gates
  double p[QSIM_NOISE_CHANNELS];
  int shots;
  float2 *scratch;
  int maxw;
  double *zexp;
  unsigned long long *samples;
  unsigned *events;
  int *nevents;
  int event_cap;
  int *counter;
  const long long *keep_off;  // [ntraj]: offset of the trajectory's kept final state, or -1
  float2 *keep;               // kept final states, normalised
};

__device__ __forceinline__ unsigned long long insert2(unsigned long long g, int ns, int s0, int s1) {
  unsigned long long low = g & ((1ULL << s0) - 1ULL);
  g = ((g ^ low) << 1) | low;
  if (ns == 2) {
    low = g & ((1ULL << s1) - 1ULL);
    g = ((g ^ low) << 1) | low;
  }
  return g;
}

// Neumaier (compensated) FP32 accumulation
struct KSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// complex double helpers for thread 0's operator algebra
struct Cd {
  double r, i;
};
__device__ __forceinline__ Cd cmul(Cd a, Cd b) { return Cd{a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cd cadd(Cd a, Cd b) { return Cd{a.r + b.r, a.i + b.i}; }

// M <- (A on sector bit j) M, A a 2x2 complex matrix, D = 2^ns
__device__ void left_apply(Cd *M, int D, int j, const Cd A[4]) {
  Cd out[16];
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const int rb = (r >> j) & 1;
      const int r0 = r & ~(1 << j), r1 = r | (1 << j);
      out[r * D + c] = cadd(cmul(A[rb * 2 + 0], M[r0 * D + c]), cmul(A[rb * 2 + 1], M[r1 * D + c]));
    }
  for (int x = 0; x < D * D; ++x) M[x] = out[x];
}

// Pass 1: per-thread compensated sums of |(U x)_r|^2 over the 2^NS sectors of the gate's
// qubits; kUnroll items per thread per step with all loads issued first.
template <int NS>
__device__ __forceinline__ void pass_sums(const float2 *st, long long items, int s0, int s1,
                                          const unsigned long long *off, const float *gm, KSum *ks, int tid) {
  constexpr int D = 1 << NS;
  for (long long it0 = tid; it0 < items; it0 += kUnroll * kTT) {
    float2 x[kUnroll][D];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long it = it0 + (long long)u * kTT;
      const unsigned long long base = insert2((unsigned long long)(it < items ? it : 0), NS, s0, s1);
#pragma unroll
      for (int c = 0; c < D; ++c) x[u][c] = it < items ? st[base + off[c]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        float yr = 0.f, yi = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float mr = gm[2 * (r * 4 + c)], mi = gm[2 * (r * 4 + c) + 1];
          yr = fmaf(mr, x[u][c].x, fmaf(-mi, x[u][c].y, yr));
          yi = fmaf(mr, x[u][c].y, fmaf(mi, x[u][c].x, yi));
        }
        ks[r].add(fmaf(yr, yr, yi * yi));  // padded items add exact zeros
      }
    }
  }
}

// Pass 2: x <- M x with M's entries as hi + lo floats (small terms first).
template <int NS>
__device__ __forceinline__ void pass_apply(float2 *st, long long items, int s0, int s1,
                                           const unsigned long long *off, const float *mhr, const float *mhi,
                                           const float *mlr, const float *mli, int tid) {
  constexpr int D = 1 << NS;
  for (long long it0 = tid; it0 < items; it0 += kUnroll * kTT) {
    float2 x[kUnroll][D];
    unsigned long long bases[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const long long it = it0 + (long long)u * kTT;
      bases[u] = insert2((unsigned long long)(it < items ? it : 0), NS, s0, s1);
#pragma unroll
      for (int c = 0; c < D; ++c) x[u][c] = it < items ? st[bases[u] + off[c]] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (it0 + (long long)u * kTT >= items) continue;
      float2 y[D];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        float lr = 0.f, li = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          lr += mlr[r * D + c] * x[u][c].x - mli[r * D + c] * x[u][c].y;
          li += mlr[r * D + c] * x[u][c].y + mli[r * D + c] * x[u][c].x;
        }
        float yr = lr, yi = li;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          yr = fmaf(mhr[r * D + c], x[u][c].x, fmaf(-mhi[r * D + c], x[u][c].y, yr));
          yi = fmaf(mhr[r * D + c], x[u][c].y, fmaf(mhi[r * D + c], x[u][c].x, yi));
        }
        y[r] = make_float2(yr, yi);
      }
#pragma unroll
      for (int r = 0; r < D; ++r) st[bases[u] + off[r]] = y[r];
    }
  }
}

constexpr unsigned kDamping = (1u << QSIM_NOISE_AMPLITUDE_DAMPING) | (1u << QSIM_NOISE_PHASE_DAMPING);

__device__ __forceinline__ int n_branches(int c) { return c == QSIM_NOISE_DEPOLARIZING ? 4 : 2; }

// 0 I, 1 X, 2 Y, 3 Z
__device__ void pauli(int which, Cd P[4]) {
  const Cd z{0, 0}, one{1, 0};
  switch (which) {
    case 1: P[0] = z; P[1] = one; P[2] = one; P[3] = z; break;
    case 2: P[0] = z; P[1] = Cd{0, -1}; P[2] = Cd{0, 1}; P[3] = z; break;
    case 3: P[0] = one; P[1] = z; P[2] = z; P[3] = Cd{-1, 0}; break;
    default: P[0] = one; P[1] = z; P[2] = z; P[3] = one; break;
  }
}

// Branch br of channel c (Eq. 5). For depolarizing and the flips, whose operators are
// sqrt(w) times a unitary, K receives that unitary and the weight w is returned; for the
// damping channels K receives the operator as printed and the result is -1 (the weight
// depends on the state).
__device__ double kraus_branch(int c, int br, double p, Cd K[4]) {
  switch (c) {
    case QSIM_NOISE_DEPOLARIZING: pauli(br, K); return br == 0 ? 1.0 - 3.0 * p / 4.0 : p / 4.0;
    case QSIM_NOISE_BIT_FLIP: pauli(br ? 1 : 0, K); return br ? 1.0 - p : p;
    case QSIM_NOISE_PHASE_FLIP: pauli(br ? 3 : 0, K); return br ? 1.0 - p : p;
    case QSIM_NOISE_BIT_PHASE_FLIP: pauli(br ? 2 : 0, K); return br ? 1.0 - p : p;
    case QSIM_NOISE_AMPLITUDE_DAMPING:
      K[0] = Cd{br ? 0.0 : 1.0, 0}; K[1] = Cd{br ? sqrt(p) : 0.0, 0};
      K[2] = Cd{0, 0}; K[3] = Cd{br ? 0.0 : sqrt(1.0 - p), 0};
      return -1.0;
    default:  // phase damping
      K[0] = Cd{br ? 0.0 : 1.0, 0}; K[1] = Cd{0, 0};
      K[2] = Cd{0, 0}; K[3] = Cd{br ? sqrt(p) : sqrt(1.0 - p), 0};
      return -1.0;
  }
}

__device__ __forceinline__ double abs2(Cd v) { return v.r * v.r + v.i * v.i; }

// Sector populations after K acts on sector bit j: with one non-zero per row and column,
// S'(b') = sum_b |K_b'b|^2 S(b).
__device__ void update_sums(double *S, int D, int j, const Cd K[4]) {
  for (int sct = 0; sct < D; ++sct)
    if (!((sct >> j) & 1)) {
      const double s0 = S[sct], s1 = S[sct | (1 << j)];
      S[sct] = abs2(K[0]) * s0 + abs2(K[1]) * s1;
      S[sct | (1 << j)] = abs2(K[2]) * s0 + abs2(K[3]) * s1;
    }
}

// sum over sectors of S * (K_i^dag K_i)_{bit j} [* (K_k^dag K_k)_{bit 0} for a joint branch]
__device__ double branch_weight(const double *S, int D, int j, const Cd Ki[4], const Cd *Kk) {
  double acc = 0.0;
  for (int sct = 0; sct < D; ++sct) {
    const int b = (sct >> j) & 1;
    double w = S[sct] * (abs2(Ki[b]) + abs2(Ki[2 + b]));
    if (Kk) {
      const int b0 = sct & 1;
      w *= abs2(Kk[b0]) + abs2(Kk[2 + b0]);
    }
    acc += w;
  }
  return acc;
}

// Smallest i with u < w_0 + ... + w_i; past the end (the sum rounded below u), the last i
// with w_i > 0.
__device__ int pick_branch(const double *w, int nw, double u) {
  double acc = 0.0;
  int last = 0;
  for (int i = 0; i < nw; ++i) {
    acc += w[i];
    if (w[i] > 0.0) last = i;
    if (u < acc) return i;
  }
  return last;
}

__device__ __forceinline__ double noise_draw(int t, int g, uint32_t site, int c, uint32_t k0, uint32_t k1) {
  const Philox4 x = philox4x32_10((uint32_t)t, (uint32_t)g, site, (uint32_t)c, k0, k1);
  return u01_from(x.v[0], x.v[1]);
}

__device__ __forceinline__ void record_event(const TrajArgs &a, int t, int g, int q, int c, int br, int &nev) {
  if (nev < a.event_cap)
    a.events[(size_t)t * a.event_cap + nev] = ((unsigned)g << 12) | ((unsigned)q << 6) | ((unsigned)c << 2) | (unsigned)br;
  ++nev;
}

// Whether gate g's branches could depend on the state: a damping draw at or above the
// weight that K1 (K1 (x) K1 for a joint draw) has for every state.
__device__ __noinline__ bool gate_uncertain(const DGate &G, int t, int g, const TrajArgs &a, uint32_t k0, uint32_t k1) {
  if (!G.noisy) return false;
  for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c) {
    if (!((a.channels >> c) & 1) || !((kDamping >> c) & 1)) continue;
    const double keep = 1.0 - a.p[c];
    if (a.kron && G.ns == 2) {
      if (!(noise_draw(t, g, QSIM_NOISE_KRON_SITE, c, k0, k1) < keep * keep)) return true;
    } else {
      for (int j = 0; j < G.ns; ++j)
        if (!(noise_draw(t, g, (uint32_t)(j == 0 ? G.s0 : G.s1), c, k0, k1) < keep)) return true;
    }
  }
  return false;
}

// Thread 0's operator algebra for gate g of trajectory t: draws the branches of every noise
// site of the gate and folds the chosen Paulis and Kraus operators into M = c K ... P U
// (2^ns x 2^ns, sector order). With the sector sums S of U psi known (sums_known) the
// damping branches follow Section 2.4 and M includes the renormalisation; without them
// every damping draw is below the weight K1 has whatever the state (the caller checked),
// so K1 is the branch and M leaves the state unnormalised. Events are appended to the
// trajectory's list.
__device__ __noinline__ void build_gate_op(const DGate &G, int t, int g, const TrajArgs &a, uint32_t k0, uint32_t k1,
                              bool sums_known, double *S, Cd *M, int &nev) {
  const int ns = G.ns, D = 1 << ns;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) M[r * D + c] = Cd{G.m[2 * (r * 4 + c)], G.m[2 * (r * 4 + c) + 1]};
  if (!G.noisy) return;
  Cd K[4], Kb[4];
  if (a.kron && ns == 2) {
    // one draw per channel over K_i (x) K_j, K_i on sector bit 1 (s1), K_j on bit 0 (s0)
    for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c) {
      if (!((a.channels >> c) & 1)) continue;
      const double p = a.p[c];
      const int nb = n_branches(c);
      const double u = noise_draw(t, g, QSIM_NOISE_KRON_SITE, c, k0, k1);
      const bool fixed = kraus_branch(c, 0, p, K) >= 0.0;
      if (!fixed && !sums_known) {  // K1 (x) K1 for certain, left unnormalised
        left_apply(M, D, 1, K);
        left_apply(M, D, 0, K);
        continue;
      }
      double w[16], tot = 0.0;
      for (int sct = 0; sct < D; ++sct) tot += S[sct];
      for (int x = 0; x < nb * nb; ++x) {
        const double wi = kraus_branch(c, x / nb, p, K), wj = kraus_branch(c, x % nb, p, Kb);
        w[x] = fixed ? wi * wj : branch_weight(S, D, 1, K, Kb) / tot;
      }
      const int x = pick_branch(w, nb * nb, u);
      const int bi = x / nb, bj = x % nb;
      if (fixed && x == 0) continue;  // the identity
      kraus_branch(c, bi, p, K);
      kraus_branch(c, bj, p, Kb);
      left_apply(M, D, 1, K);
      left_apply(M, D, 0, Kb);
      if (sums_known) {
        update_sums(S, D, 1, K);
        update_sums(S, D, 0, Kb);
      }
      if (!fixed) {  // renormalise: psi <- K psi / ||K psi||
        double nrm = 0.0;
        for (int sct = 0; sct < D; ++sct) nrm += S[sct];
        const double inv = 1.0 / sqrt(nrm);
        for (int xx = 0; xx < D * D; ++xx) M[xx] = Cd{M[xx].r * inv, M[xx].i * inv};
        for (int sct = 0; sct < D; ++sct) S[sct] /= nrm;
      }
      if (bj > 0) record_event(a, t, g, G.s0, c, bj, nev);
      if (bi > 0) record_event(a, t, g, G.s1, c, bi, nev);
    }
    return;
  }
  for (int j = 0; j < ns; ++j) {
    const int q = j == 0 ? G.s0 : G.s1;
    for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c) {
      if (!((a.channels >> c) & 1)) continue;
      const double p = a.p[c];
      const int nb = n_branches(c);
      const double u = noise_draw(t, g, (uint32_t)q, c, k0, k1);
      const bool fixed = kraus_branch(c, 0, p, K) >= 0.0;
      if (!fixed && !sums_known) {  // K1 for certain, left unnormalised
        left_apply(M, D, j, K);
        continue;
      }
      double w[4], tot = 0.0;
      for (int sct = 0; sct < D; ++sct) tot += S[sct];
      for (int x = 0; x < nb; ++x) {
        const double wx = kraus_branch(c, x, p, K);
        w[x] = fixed ? wx : branch_weight(S, D, j, K, nullptr) / tot;
      }
      const int br = pick_branch(w, nb, u);
      if (fixed && br == 0) continue;  // the identity
      kraus_branch(c, br, p, K);
      left_apply(M, D, j, K);
      if (sums_known) update_sums(S, D, j, K);
      if (!fixed) {  // renormalise: psi <- K psi / ||K psi||
        double nrm = 0.0;
        for (int sct = 0; sct < D; ++sct) nrm += S[sct];
        const double inv = 1.0 / sqrt(nrm);
        for (int xx = 0; xx < D * D; ++xx) M[xx] = Cd{M[xx].r * inv, M[xx].i * inv};
        for (int sct = 0; sct < D; ++sct) S[sct] /= nrm;
      }
      if (br > 0) record_event(a, t, g, q, c, br, nev);
    }
  }
}

// M (2^ns x 2^ns, row-major) as hi + lo floats: hr, hi, lr, li at m[0], m[16], m[32], m[48].
__device__ void store_split(const Cd *M, int D, float *m) {
  for (int xx = 0; xx < 16; ++xx) {
    const Cd v = xx < D * D ? M[xx] : Cd{0, 0};
    m[xx] = (float)v.r;
    m[16 + xx] = (float)v.i;
    m[32 + xx] = (float)(v.r - (double)m[xx]);
    m[48 + xx] = (float)(v.i - (double)m[16 + xx]);
  }
}

// A run of gates with state-independent branches on at most kRunQ qubits.
constexpr int kRunMax = 16;
constexpr int kLook = 256;    // gates of the program thread 0 looks ahead over
constexpr int kWinMinW = 17;  // from this width on, runs are chosen over qubit windows
enum { kStepDone = 0, kStepRun = 1, kStepSums = 2, kStepNorm = 3 };
constexpr int kRunQ = 4;  // 16 amplitudes per thread; 5 qubits (32) spill at 128 registers
struct RunGate {
  int ns, j0, j1;  // local bits (indices into the run's sorted qubit list)
};

// y = M x for the 2^NS amplitudes x[idx[0..]] (M's FP32 entries; a run's state is
// renormalised at every state-dependent draw and the read-outs divide by the final norm,
// so the ~2^-24 entry rounding only adds a relative error of ~1e-7 per gate)
template <int NS>
__device__ __forceinline__ void apply_small(float2 *x, const int *idx, const float *m) {
  constexpr int D = 1 << NS;
  float2 y[D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float yr = 0.f, yi = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const float2 v = x[idx[c]];
      yr = fmaf(m[r * D + c], v.x, fmaf(-m[16 + r * D + c], v.y, yr));
      yi = fmaf(m[r * D + c], v.y, fmaf(m[16 + r * D + c], v.x, yi));
    }
    y[r] = make_float2(yr, yi);
  }
#pragma unroll
  for (int r = 0; r < D; ++r) x[idx[r]] = y[r];
}

// One-qubit gate on local bit J of a group of 2^U amplitudes held in registers.
template <int U, int J>
__device__ __forceinline__ void run_gate1(float2 (&x)[1 << U], const float *m) {
#pragma unroll
  for (int i = 0; i < (1 << U); ++i) {
    if (i & (1 << J)) continue;
    const int idx[2] = {i, i | (1 << J)};
    apply_small<1>(x, idx, m);
  }
}

// Two-qubit gate on local bits J0 < J1 (sector index = bit J0 + 2 bit J1).
template <int U, int J0, int J1>
__device__ __forceinline__ void run_gate2(float2 (&x)[1 << U], const float *m) {
#pragma unroll
  for (int i = 0; i < (1 << U); ++i) {
    if ((i & (1 << J0)) || (i & (1 << J1))) continue;
    const int idx[4] = {i, i | (1 << J0), i | (1 << J1), i | (1 << J0) | (1 << J1)};
    apply_small<2>(x, idx, m);
  }
}

// Global offset of member i of a group: the sum of 2^pos[b] over the set bits b of i.
template <int U>
__device__ __forceinline__ unsigned long long group_off(int i, const unsigned long long *o) {
  unsigned long long v = 0;
#pragma unroll
  for (int b = 0; b < U; ++b)
    if ((i >> b) & 1) v += o[b];
  return v;
}

// One pass applying a run of gates: each thread loads groups of 2^U amplitudes (the run's
// qubits pos[0..U) sorted ascending), applies the gates in order in registers and stores.
template <int U>
__device__ void pass_run(float2 *st, long long N, const int *pos, int nrun, const RunGate *rg,
                         const float (*rm)[64], int tid) {
  constexpr int D = 1 << U;
  const long long items = N >> U;
  unsigned long long o[U];
#pragma unroll
  for (int b = 0; b < U; ++b) o[b] = 1ULL << pos[b];
  for (long long it = tid; it < items; it += kTT) {
    unsigned long long base = (unsigned long long)it;
#pragma unroll
    for (int b = 0; b < U; ++b) {
      const unsigned long long low = base & (o[b] - 1ULL);
      base = ((base ^ low) << 1) | low;
    }
    float2 x[D];
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = st[base + group_off<U>(i, o)];
    for (int q = 0; q < nrun; ++q) {
      const float *m = rm[q];
      const RunGate R = rg[q];
      if (R.ns == 1) {
        switch (R.j0) {
          case 0: run_gate1<U, 0>(x, m); break;
          case 1: if constexpr (U > 1) run_gate1<U, 1>(x, m); break;
          case 2: if constexpr (U > 2) run_gate1<U, 2>(x, m); break;
          case 3: if constexpr (U > 3) run_gate1<U, 3>(x, m); break;
          default: if constexpr (U > 4) run_gate1<U, 4>(x, m); break;
        }
      } else if constexpr (U >= 2) {
        switch (R.j0 * 8 + R.j1) {
          case 1: run_gate2<U, 0, 1>(x, m); break;
          case 2: if constexpr (U > 2) run_gate2<U, 0, 2>(x, m); break;
          case 10: if constexpr (U > 2) run_gate2<U, 1, 2>(x, m); break;
          case 3: if constexpr (U > 3) run_gate2<U, 0, 3>(x, m); break;
          case 11: if constexpr (U > 3) run_gate2<U, 1, 3>(x, m); break;
          case 19: if constexpr (U > 3) run_gate2<U, 2, 3>(x, m); break;
          case 4: if constexpr (U > 4) run_gate2<U, 0, 4>(x, m); break;
          case 12: if constexpr (U > 4) run_gate2<U, 1, 4>(x, m); break;
          case 20: if constexpr (U > 4) run_gate2<U, 2, 4>(x, m); break;
          default: if constexpr (U > 4) run_gate2<U, 3, 4>(x, m); break;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) st[base + group_off<U>(i, o)] = x[i];
  }
}

__global__ void __launch_bounds__(kTT, 1) k_traj(TrajArgs a) {
  extern __shared__ float2 sm_state[];
  __shared__ double red[32][4];
  __shared__ double sums[4];
  __shared__ float mhr[16], mhi[16], mlr[16], mli[16];
  __shared__ float gm[32];  // the gate's matrix (float) for the sector sums
  __shared__ int cur, step_kind, step_gate, run_n, run_u;
  __shared__ unsigned char punc[kLook], pdone[kLook];
  __shared__ unsigned pmask[kLook];
  __shared__ int run_pos[kRunQ];
  __shared__ RunGate rg[kRunMax];
  __shared__ float rmat[kRunMax][64];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned long long seed = *(volatile const unsigned long long *)a.seed;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

  for (;;) {
    if (tid == 0) cur = atomicAdd(a.counter, 1);
    __syncthreads();
    const int k = cur;
    if (k >= a.ntraj) break;
    const int t = a.order[k];
    const int prog = a.traj_prog[t];
    const int w = a.prog_w[prog];
    const long long N = 1LL << w;
    float2 *st = w <= kSmemQubits ? sm_state : a.scratch + (size_t)blockIdx.x * ((size_t)1 << a.maxw);
    for (long long i = tid; i < N; i += kTT) st[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
    int nev = 0;
    __syncthreads();

    const DGate *gl = a.gates + a.prog_off[prog];
    const int ng = a.prog_len[prog];
    // unnormalised K1 sites allowed in a row: each shrinks the squared norm by at most
    // prod (1 - p) over the damping channels, kept above 1e-6
    double shrink = 0.0;
    for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c)
      if (((a.channels & kDamping) >> c) & 1) shrink += log1p(-a.p[c]);
    const double keep = shrink < 0.0 ? fmin(1e9, log(1e-6) / shrink) : 1e9;
    // thread 0's view of the program: gates [first, filled) have their flags in the ring
    // punc / pdone (state-dependent draw, already applied); every gate before `first` is done
    int since = 0, first = 0, filled = 0;
    const bool windows = w >= kWinMinW;
    for (;;) {
      // ---- thread 0 plans the next step. A damping K1 is chosen when u < 1 - p P1 / N
      // and P1 / N <= 1, so a draw u < 1 - p ((1 - p)^2 for a joint draw) picks K1
      // whatever the state, and a gate whose draws are all like that has its branches
      // fixed in advance. Between two
      // gates with a state-dependent draw, the folded operators (U with its Paulis and K1,
      // left unnormalised) of gates on disjoint qubits commute, so those gates may run in
      // any order that keeps the order on each qubit: a run takes every gate of the
      // segment that lies in one set of at most kRunQ qubits and is not blocked by an
      // earlier gate, and one pass applies it. A gate with a state-dependent draw waits
      // until everything before it is done (and nothing after it is), then takes a
      // sector-sum pass and the branch of Section 2.4 with renormalisation.
      if (wid == 0) {
        // every lane of warp 0 keeps the same `first` and `filled`; lane 0 alone keeps
        // `since` and takes the ordered work (operators, events)
        while (first < filled && pdone[first % kLook]) ++first;
        const int lim = min(ng, first + kLook);
        for (int g = filled + lane; g < lim; g += 32) {
          const DGate &G = gl[g];
          punc[g % kLook] = gate_uncertain(G, t, g, a, k0, k1) ? 1 : 0;
          pdone[g % kLook] = 0;
          pmask[g % kLook] = (1u << G.s0) | (G.ns == 2 ? (1u << G.s1) : 0u);
        }
        filled = lim > filled ? lim : filled;
        __syncwarp();
        int kind = kStepRun, seg = first;
        if (first >= ng) {
          kind = kStepDone;
        } else if (lane == 0 && since > keep) {
          kind = kStepNorm;  // renormalise before the norm can get small
          since = 0;
        } else {
          while (seg < filled && !punc[seg % kLook]) ++seg;
          if (seg == first) kind = kStepSums;
        }
        kind = __shfl_sync(0xffffffffu, kind, 0);
        if (kind == kStepSums) {
          if (lane == 0) {
            step_gate = first;
            pdone[first % kLook] = 1;
            since = 0;
          }
        } else if (kind == kStepRun) {
          // candidate sets: the first gates of the segment grown in order, then (wide
          // states, where a pass costs far more than this search) every window of kRunQ
          // consecutive qubits; lane c scores candidate c
          unsigned grown = 0;
          for (int g = first; g < seg; ++g) {
            if (pdone[g % kLook]) continue;
            if (__popc(grown | pmask[g % kLook]) > kRunQ) break;
            grown |= pmask[g % kLook];
          }
          const int ncand = windows ? 1 + (w - kRunQ + 1) : 1;
          int n_here = -1;
          unsigned s_here = grown;
          if (lane < ncand) {
            const unsigned S = lane == 0 ? grown : (((1u << kRunQ) - 1u) << (lane - 1));
            s_here = S;
            unsigned blocked = 0;
            int n = 0;
            for (int g = first; g < seg && n < kRunMax; ++g) {
              if (pdone[g % kLook]) continue;
              const unsigned qm = pmask[g % kLook];
              if (!(qm & S)) continue;
              if (!(qm & ~S) && !(qm & blocked)) ++n;
              else blocked |= qm & S;
              if (blocked == S) break;
            }
            n_here = n;
          }
          // the candidate with the most gates (the lowest lane on ties)
          int best_n = n_here, best_lane = lane;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const int on = __shfl_xor_sync(0xffffffffu, best_n, o);
            const int ol = __shfl_xor_sync(0xffffffffu, best_lane, o);
            if (on > best_n || (on == best_n && ol < best_lane)) {
              best_n = on;
              best_lane = ol;
            }
          }
          const unsigned best_s = __shfl_sync(0xffffffffu, s_here, best_lane);
          if (lane == 0) {
            // take the chosen set's gates in program order and build their operators
            unsigned blocked = 0, umask = 0;
            int n = 0;
            for (int g = first; g < seg && n < kRunMax; ++g) {
              if (pdone[g % kLook]) continue;
              const unsigned qm = pmask[g % kLook];
              if (!(qm & best_s)) continue;
              if ((qm & ~best_s) || (qm & blocked)) {
                blocked |= qm & best_s;
                if (blocked == best_s) break;
                continue;
              }
              const DGate &G = gl[g];
              Cd M[16];
              double S[4] = {0.0, 0.0, 0.0, 0.0};
              build_gate_op(G, t, g, a, k0, k1, false, S, M, nev);
              store_split(M, 1 << G.ns, rmat[n]);
              rg[n].ns = G.ns;
              rg[n].j0 = G.s0;  // made local below
              rg[n].j1 = G.s1;
              pdone[g % kLook] = 1;
              umask |= qm;
              if (G.noisy) since += G.ns;
              ++n;
            }
            run_n = n;
            int u = 0;
            for (int q = 0; q < 32; ++q)
              if ((umask >> q) & 1) run_pos[u++] = q;
            run_u = u;
            for (int x = 0; x < n; ++x) {
              rg[x].j0 = __popc(umask & ((1u << rg[x].j0) - 1u));
              rg[x].j1 = rg[x].ns == 2 ? __popc(umask & ((1u << rg[x].j1) - 1u)) : 0;
            }
          }
        }
        if (lane == 0) step_kind = kind;
        __syncwarp();
      }
      __syncthreads();
      const int kind = step_kind;
      if (kind == kStepDone) break;
      if (kind == kStepRun) {
        switch (run_u) {
          case 1: pass_run<1>(st, N, run_pos, run_n, rg, rmat, tid); break;
          case 2: pass_run<2>(st, N, run_pos, run_n, rg, rmat, tid); break;
          case 3: pass_run<3>(st, N, run_pos, run_n, rg, rmat, tid); break;
          default: pass_run<4>(st, N, run_pos, run_n, rg, rmat, tid); break;
        }
        __syncthreads();
        continue;
      }
      if (kind == kStepNorm) {
        KSum tot;
        for (long long i = tid; i < N; i += kTT) {
          const float2 v = st[i];
          tot.add(fmaf(v.x, v.x, v.y * v.y));
        }
        const double v = warp_sum_d(tot.value());
        if (lane == 0) red[wid][0] = v;
        __syncthreads();
        if (tid == 0) {
          double sacc = 0.0;
          for (int x = 0; x < kTT / 32; ++x) sacc += red[x][0];
          sums[0] = sacc;
        }
        __syncthreads();
        const float sc = (float)(1.0 / sqrt(sums[0]));
        for (long long i = tid; i < N; i += kTT) {
          const float2 x = st[i];
          st[i] = make_float2(x.x * sc, x.y * sc);
        }
        __syncthreads();
        continue;
      }
      // ---- a gate with a state-dependent damping draw: sector sums of U psi, then the
      // branches of Section 2.4 with renormalisation, then one pass applying M
      const int g = step_gate;
      const DGate &G = gl[g];
      const int ns = G.ns, D = 1 << ns;
      const long long items = N >> ns;
      unsigned long long off[4];
      off[0] = 0;
      off[1] = 1ULL << G.s0;
      off[2] = ns == 2 ? (1ULL << G.s1) : 0;
      off[3] = off[1] | off[2];
      if (tid < 32) gm[tid] = (float)G.m[tid];
      __syncthreads();
      {
        KSum ks[4];
        if (ns == 1) pass_sums<1>(st, items, G.s0, G.s1, off, gm, ks, tid);
        else pass_sums<2>(st, items, G.s0, G.s1, off, gm, ks, tid);
        for (int r = 0; r < 4; ++r) {
          const double v = warp_sum_d(r < D ? ks[r].value() : 0.0);
          if (lane == 0) red[wid][r] = v;
        }
        __syncthreads();
        if (tid < 4) {
          double sacc = 0.0;
          for (int x = 0; x < kTT / 32; ++x) sacc += red[x][tid];
          sums[tid] = sacc;
        }
        __syncthreads();
      }
      if (tid == 0) {
        Cd M[16];
        double S[4] = {sums[0], sums[1], sums[2], sums[3]};
        build_gate_op(G, t, g, a, k0, k1, true, S, M, nev);
        for (int xx = 0; xx < 16; ++xx) {
          const Cd v = xx < D * D ? M[xx] : Cd{0, 0};
          mhr[xx] = (float)v.r;
          mhi[xx] = (float)v.i;
          mlr[xx] = (float)(v.r - (double)mhr[xx]);
          mli[xx] = (float)(v.i - (double)mhi[xx]);
        }
      }
      __syncthreads();
      if (ns == 1) pass_apply<1>(st, items, G.s0, G.s1, off, mhr, mhi, mlr, mli, tid);
      else pass_apply<2>(st, items, G.s0, G.s1, off, mhr, mhi, mlr, mli, tid);
      __syncthreads();
    }
    // events in gate order (runs may apply commuting gates out of order)
    if (tid == 0) {
      unsigned *ev = a.events + (size_t)t * a.event_cap;
      const int ne = nev < a.event_cap ? nev : a.event_cap;
      for (int i = 1; i < ne; ++i) {
        const unsigned v = ev[i];
        int j = i - 1;
        while (j >= 0 && (ev[j] >> 12) > (v >> 12)) {
          ev[j + 1] = ev[j];
          --j;
        }
        ev[j + 1] = v;
      }
    }

    // ---- read-out: <Z_q> = 1 - 2 P1(q) / N for every qubit. P1 sums run in FP32 over
    // chunks of kZChunk of the thread's amplitudes, then in FP64 across chunks.
    {
      constexpr int kZChunk = 32;
      float p1c[kMaxW];
      double p1[kMaxW];
      KSum tot;
      for (int q = 0; q < kMaxW; ++q) {
        p1c[q] = 0.f;
        p1[q] = 0.0;
      }
      int in_chunk = 0;
      for (long long i = tid; i < N; i += kTT) {
        const float2 v = st[i];
        const float pr = fmaf(v.x, v.x, v.y * v.y);
        tot.add(pr);
#pragma unroll
        for (int q = 0; q < kMaxW; ++q)
          if (q < w && ((i >> q) & 1)) p1c[q] += pr;
        if (++in_chunk == kZChunk) {
#pragma unroll
          for (int q = 0; q < kMaxW; ++q) {
            p1[q] += (double)p1c[q];
            p1c[q] = 0.f;
          }
          in_chunk = 0;
        }
      }
#pragma unroll
      for (int q = 0; q < kMaxW; ++q) p1[q] += (double)p1c[q];
      double totd = warp_sum_d(tot.value());
      if (lane == 0) red[wid][0] = totd;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int x = 0; x < kTT / 32; ++x) s += red[x][0];
        sums[0] = s;
      }
      __syncthreads();
      const double norm = sums[0];
      // the final state, normalised, for a trajectory whose state the caller keeps
      const long long ko = a.keep_off[t];
      if (ko >= 0) {
        const float sc = (float)(1.0 / sqrt(norm));
        for (long long i = tid; i < N; i += kTT) {
          const float2 v = st[i];
          a.keep[ko + i] = make_float2(v.x * sc, v.y * sc);
        }
      }
      for (int q = 0; q < w; ++q) {
        const double v = warp_sum_d(p1[q]);
        __syncthreads();
        if (lane == 0) red[wid][1] = v;
        __syncthreads();
        if (tid == 0) {
          double s = 0.0;
          for (int x = 0; x < kTT / 32; ++x) s += red[x][1];
          a.zexp[(size_t)t * kMaxW + q] = 1.0 - 2.0 * s / norm;
        }
      }
      if (tid == 0) a.nevents[t] = nev;
      // ---- one shot: smallest i with u * N < sum_{l <= i} |a_l|^2 (contiguous ranges)
      if (t < a.shots) {
        const long long R = (N + kTT - 1) / kTT;  // contiguous range per thread
        const long long lo = tid * R < N ? tid * R : N, hi = (tid + 1) * R < N ? (tid + 1) * R : N;
        KSum mine;
        for (long long i = lo; i < hi; ++i) {
          const float2 v = st[i];
          mine.add(fmaf(v.x, v.x, v.y * v.y));
        }
        __shared__ double pre[kTT];
        pre[tid] = mine.value();
        __syncthreads();
        __shared__ double target_s;
        __shared__ int owner;
        if (tid == 0) {
          double run = 0.0;
          for (int x = 0; x < kTT; ++x) {
            const double v = pre[x];
            pre[x] = run;
            run += v;
          }
          const Philox4 x = philox4x32_10((uint32_t)t, (uint32_t)ng, 0u, kSampleTag, k0, k1);
          target_s = u01_from(x.v[0], x.v[1]) * run;
          // the last thread whose range starts at or below the target and is not empty
          int o = 0;
          for (int y = 0; y < kTT; ++y)
            if (y * R < N && pre[y] <= target_s) o = y;
          owner = o;
        }
        __syncthreads();
        if (tid == owner) {
          KSum runk;
          long long pick = -1, last_nz = lo;
          for (long long i = lo; i < hi; ++i) {
            const float2 v = st[i];
            const float pr = fmaf(v.x, v.x, v.y * v.y);
            runk.add(pr);
            if (pr > 0.f) last_nz = i;
            if (pick < 0 && target_s < pre[tid] + runk.value()) pick = i;
          }
          a.samples[t] = (unsigned long long)(pick >= 0 ? pick : last_nz);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

}  // namespace qsim


// A prepared batch: its programs, outputs and scratch in one device block, and the seed
// in a word of mapped pinned host memory that every launch reads.
struct qsim_traj_plan {
  int device = 0;
  cudaStream_t home = nullptr;  // stream of qsim_traj_prepare; the block is freed on it
  unsigned char *dev = nullptr;
  unsigned long long *seed_host = nullptr;  // mapped pinned word
  qsim::TrajArgs args{};
  int grid = 0;
  int ntraj = 0, shots = 0, event_cap = 0;
  std::vector<int> keep_w;          // width of each kept trajectory
  std::vector<long long> keep_at;   // offset of each kept state in args.keep
};

using namespace qsim;

namespace {

std::atomic<unsigned long long> g_traj_attr{0};

qsim_status check_batch(const qsim_traj_batch *b) {
  if (!b || b->nprog < 1 || b->ntraj < 1 || !b->prog_qubits || !b->prog_ops || !b->prog_nops || !b->traj_prog) {
    set_error("run_trajectories: incomplete batch description");
    return QSIM_EINVAL;
  }
  if ((b->channels >> QSIM_NOISE_CHANNELS) != 0 || (b->kron != 0 && b->kron != 1)) {
    set_error("run_trajectories: unknown channel bits 0x%x or kron %d", b->channels, b->kron);
    return QSIM_EINVAL;
  }
  for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c)
    if (((b->channels >> c) & 1) && !(b->p[c] >= 0.0 && b->p[c] <= 1.0)) {
      set_error("run_trajectories: p of channel %d outside [0, 1]", c);
      return QSIM_EINVAL;
    }
  if (b->shots < 0 || b->shots > b->ntraj || b->event_cap < 0) {
    set_error("run_trajectories: bad shot count or event capacity");
    return QSIM_EINVAL;
  }
  return QSIM_OK;
}

void free_plan(qsim_traj_plan *p) {
  if (!p) return;
  if (p->dev) cudaFreeAsync(p->dev, p->home);
  if (p->seed_host) cudaFreeHost(p->seed_host);
  delete p;
}

}  // namespace

extern "C" qsim_status qsim_traj_prepare(const qsim_traj_batch *b, const int32_t *keep, int32_t nkeep,
                                         void *stream, qsim_traj_plan **out) {
  if (!out) {
    set_error("traj_prepare: out must be non-NULL");
    return QSIM_EINVAL;
  }
  *out = nullptr;
  QS_TRY(check_batch(b));
  if (nkeep < 0 || (nkeep > 0 && !keep)) {
    set_error("traj_prepare: bad list of kept trajectories");
    return QSIM_EINVAL;
  }
  std::vector<DGate> gates;
  std::vector<int> off(b->nprog), len(b->nprog), width(b->nprog);
  int maxw = 0;
  for (int p = 0; p < b->nprog; ++p) {
    const int w = b->prog_qubits[p];
    if (w < 2 || w > QSIM_TRAJ_MAX_QUBITS) {
      set_error("trajectory program %d: width %d not in [2, %d]", p, w, QSIM_TRAJ_MAX_QUBITS);
      return QSIM_EINVAL;
    }
    std::vector<Gate> gl;
    QS_TRY(expand_ops(b->prog_ops[p], b->prog_nops[p], w, gl));
    off[p] = (int)gates.size();
    len[p] = (int)gl.size();
    width[p] = w;
    maxw = std::max(maxw, w);
    for (const Gate &g : gl) {
      std::vector<int> sites(g.t, g.t + g.nt);
      sites.insert(sites.end(), g.ctrl.begin(), g.ctrl.end());
      std::sort(sites.begin(), sites.end());
      if (sites.size() > 2) {
        set_error("trajectory gates act on at most 2 qubits (program %d)", p);
        return QSIM_EUNSUPPORTED;
      }
      DGate d{};
      d.noisy = b->noisy_kinds == 0 || (g.kind >= 0 && g.kind < 32 && ((b->noisy_kinds >> g.kind) & 1u));
      d.ns = (int)sites.size();
      d.s0 = sites[0];
      d.s1 = d.ns == 2 ? sites[1] : 0;
      std::vector<int> msb_first(sites.rbegin(), sites.rend());  // sector bit j <-> sites[j]
      std::vector<cd> m;
      embed_gate(g, msb_first, m);
      const int D = 1 << d.ns;
      for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
          d.m[2 * (r * 4 + c)] = m[(size_t)r * D + c].real();
          d.m[2 * (r * 4 + c) + 1] = m[(size_t)r * D + c].imag();
        }
      gates.push_back(d);
    }
  }
  std::vector<int> tprog(b->ntraj), order(b->ntraj);
  for (int t = 0; t < b->ntraj; ++t) {
    const int p = b->traj_prog[t];
    if (p < 0 || p >= b->nprog) {
      set_error("trajectory %d: program %d out of range", t, p);
      return QSIM_EINVAL;
    }
    tprog[t] = p;
    order[t] = t;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return width[tprog[x]] > width[tprog[y]]; });
  std::vector<long long> keep_off(b->ntraj, -1LL);
  std::vector<int> keep_w(nkeep);
  std::vector<long long> keep_at(nkeep);
  long long keep_amps = 0;
  for (int i = 0; i < nkeep; ++i) {
    const int t = keep[i];
    if (t < 0 || t >= b->ntraj || keep_off[t] >= 0) {
      set_error("traj_prepare: kept trajectory %d out of range or repeated", t);
      return QSIM_EINVAL;
    }
    keep_w[i] = width[tprog[t]];
    keep_at[i] = keep_amps;
    keep_off[t] = keep_amps;
    keep_amps += 1LL << keep_w[i];
  }

  auto *plan = new qsim_traj_plan();
  plan->home = static_cast<cudaStream_t>(stream);
  plan->ntraj = b->ntraj;
  plan->shots = b->shots;
  plan->event_cap = b->event_cap;
  plan->keep_w = keep_w;
  plan->keep_at = keep_at;
  plan->grid = num_sms();
  cudaError_t e = cudaGetDevice(&plan->device);
  const size_t scratch_amps = maxw > kSmemQubits ? ((size_t)plan->grid << maxw) : 0;
  // one device allocation for everything
  size_t sz = 0;
  auto take = [&](size_t bytes) {
    const size_t at = (sz + 255) & ~(size_t)255;
    sz = at + bytes;
    return at;
  };
  const size_t o_gates = take(gates.size() * sizeof(DGate));
  const size_t o_off = take(sizeof(int) * b->nprog), o_len = take(sizeof(int) * b->nprog),
               o_w = take(sizeof(int) * b->nprog), o_tp = take(sizeof(int) * b->ntraj),
               o_ord = take(sizeof(int) * b->ntraj), o_cnt = take(sizeof(int)),
               o_z = take(sizeof(double) * kMaxW * b->ntraj), o_smp = take(sizeof(uint64_t) * b->ntraj),
               o_ev = take(sizeof(uint32_t) * (size_t)b->ntraj * (b->event_cap > 0 ? b->event_cap : 1)),
               o_nev = take(sizeof(int) * b->ntraj), o_ko = take(sizeof(long long) * b->ntraj),
               o_keep = take((size_t)keep_amps * sizeof(float2)), o_scr = take(scratch_amps * sizeof(float2));
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&plan->dev, sz, plan->home);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&plan->seed_host, sizeof(unsigned long long), cudaHostAllocMapped);
  unsigned long long *seed_dev = nullptr;
  if (e == cudaSuccess) {
    *plan->seed_host = b->seed;
    e = cudaHostGetDevicePointer((void **)&seed_dev, plan->seed_host, 0);
  }
  unsigned char *dev = plan->dev;
  auto h2d = [&](size_t at, const void *src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dev + at, src, bytes, cudaMemcpyHostToDevice, plan->home);
  };
  h2d(o_gates, gates.data(), gates.size() * sizeof(DGate));
  h2d(o_off, off.data(), sizeof(int) * b->nprog);
  h2d(o_len, len.data(), sizeof(int) * b->nprog);
  h2d(o_w, width.data(), sizeof(int) * b->nprog);
  h2d(o_tp, tprog.data(), sizeof(int) * b->ntraj);
  h2d(o_ord, order.data(), sizeof(int) * b->ntraj);
  h2d(o_ko, keep_off.data(), sizeof(long long) * b->ntraj);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(dev + o_smp, 0, sizeof(uint64_t) * b->ntraj, plan->home);  // shots never drawn read 0
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->home);  // the host arrays above go out of scope
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    free_plan(plan);
    return cuda_fail(e, "traj_prepare");
  }
  TrajArgs &a = plan->args;
  a.gates = reinterpret_cast<const DGate *>(dev + o_gates);
  a.prog_off = reinterpret_cast<const int *>(dev + o_off);
  a.prog_len = reinterpret_cast<const int *>(dev + o_len);
  a.prog_w = reinterpret_cast<const int *>(dev + o_w);
  a.traj_prog = reinterpret_cast<const int *>(dev + o_tp);
  a.order = reinterpret_cast<const int *>(dev + o_ord);
  a.ntraj = b->ntraj;
  a.seed = seed_dev;
  a.channels = b->channels;
  a.kron = b->kron;
  for (int c = 0; c < QSIM_NOISE_CHANNELS; ++c) a.p[c] = (b->channels >> c) & 1 ? b->p[c] : 0.0;
  a.shots = b->shots;
  a.scratch = reinterpret_cast<float2 *>(dev + o_scr);
  a.maxw = maxw;
  a.zexp = reinterpret_cast<double *>(dev + o_z);
  a.samples = reinterpret_cast<unsigned long long *>(dev + o_smp);
  a.events = reinterpret_cast<unsigned *>(dev + o_ev);
  a.nevents = reinterpret_cast<int *>(dev + o_nev);
  a.event_cap = b->event_cap;
  a.counter = reinterpret_cast<int *>(dev + o_cnt);
  a.keep_off = reinterpret_cast<const long long *>(dev + o_ko);
  a.keep = reinterpret_cast<float2 *>(dev + o_keep);
  *out = plan;
  return QSIM_OK;
}

extern "C" qsim_status qsim_traj_set_seed(qsim_traj_plan *p, uint64_t seed) {
  if (!p) {
    set_error("traj_set_seed: NULL plan");
    return QSIM_EINVAL;
  }
  *(volatile unsigned long long *)p->seed_host = seed;
  return QSIM_OK;
}

extern "C" qsim_status qsim_traj_launch(qsim_traj_plan *p, void *stream) {
  if (!p) {
    set_error("traj_launch: NULL plan");
    return QSIM_EINVAL;
  }
  int dev = 0;
  QS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) {
    set_error("traj_launch: plan prepared on device %d, current device %d", p->device, dev);
    return QSIM_EINVAL;
  }
  const size_t smem = sizeof(float2) << kSmemQubits;
  QS_TRY(smem_attr_once(k_traj, (int)smem, g_traj_attr));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TrajArgs &a = p->args;
  QS_TRY_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), st));
  QS_TRY_CUDA(cudaMemsetAsync(a.zexp, 0, sizeof(double) * kMaxW * p->ntraj, st));
  QS_TRY_CUDA(cudaMemsetAsync(a.nevents, 0, sizeof(int) * p->ntraj, st));
  k_traj<<<p->grid, kTT, smem, st>>>(a);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

extern "C" qsim_status qsim_traj_results(qsim_traj_plan *p, void *stream, double *zexp_out, uint64_t *samples_out,
                                         uint32_t *events_out, int32_t *nevents_out) {
  if (!p || !zexp_out || (p->shots > 0 && !samples_out) || (p->event_cap > 0 && !events_out)) {
    set_error("traj_results: NULL plan or output buffer");
    return QSIM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TrajArgs &a = p->args;
  QS_TRY_CUDA(cudaMemcpyAsync(zexp_out, a.zexp, sizeof(double) * kMaxW * p->ntraj, cudaMemcpyDeviceToHost, st));
  if (p->shots > 0)
    QS_TRY_CUDA(cudaMemcpyAsync(samples_out, a.samples, sizeof(uint64_t) * p->shots, cudaMemcpyDeviceToHost, st));
  if (p->event_cap > 0)
    QS_TRY_CUDA(cudaMemcpyAsync(events_out, a.events, sizeof(uint32_t) * (size_t)p->ntraj * p->event_cap,
                                cudaMemcpyDeviceToHost, st));
  if (nevents_out)
    QS_TRY_CUDA(cudaMemcpyAsync(nevents_out, a.nevents, sizeof(int) * p->ntraj, cudaMemcpyDeviceToHost, st));
  QS_TRY_CUDA(cudaStreamSynchronize(st));
  return QSIM_OK;
}

extern "C" qsim_status qsim_traj_state(qsim_traj_plan *p, int32_t i, void *stream, void *host_out) {
  if (!p || !host_out || i < 0 || i >= (int)p->keep_w.size()) {
    set_error("traj_state: NULL plan or buffer, or kept index %d out of range", i);
    return QSIM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  QS_TRY_CUDA(cudaMemcpyAsync(host_out, p->args.keep + p->keep_at[i], sizeof(float2) << p->keep_w[i],
                              cudaMemcpyDeviceToHost, st));
  QS_TRY_CUDA(cudaStreamSynchronize(st));
  return QSIM_OK;
}

extern "C" void qsim_traj_destroy(qsim_traj_plan *p) { free_plan(p); }

extern "C" qsim_status qsim_run_trajectories(const qsim_traj_batch *b, void *stream, double *zexp_out,
                                             uint64_t *samples_out, uint32_t *events_out, int32_t *nevents_out) {
  QS_TRY(check_batch(b));
  if (!zexp_out || (b->shots > 0 && !samples_out) || (b->event_cap > 0 && !events_out)) {
    set_error("run_trajectories: bad shot count or output buffers");
    return QSIM_EINVAL;
  }
  qsim_traj_plan *p = nullptr;
  QS_TRY(qsim_traj_prepare(b, nullptr, 0, stream, &p));
  qsim_status s = qsim_traj_launch(p, stream);
  if (s == QSIM_OK) s = qsim_traj_results(p, stream, zexp_out, samples_out, events_out, nevents_out);
  free_plan(p);
  return s;
}
