// Internal declarations shared by the host and device translation units of libqsim.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <complex>
#include <memory>
#include <functional>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

using cd = std::complex<double>;

// ------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
qsim_status cuda_fail(cudaError_t e, const char *what);

#define QS_TRY_CUDA(call)                                      \
  do {                                                         \
    cudaError_t qs_e_ = (call);                                \
    if (qs_e_ != cudaSuccess) return ::qsim::cuda_fail(qs_e_, #call); \
  } while (0)

#define QS_TRY(call)                       \
  do {                                     \
    qsim_status qs_s_ = (call);            \
    if (qs_s_ != QSIM_OK) return qs_s_;    \
  } while (0)

// Raises the dynamic shared-memory limit of kernel `func` to `bytes` on the current
// device, the first time a launch there needs it. `done` keeps one bit per device
// (0..63) and may be shared by threads: two threads that meet the first use together
// both set the attribute, which is harmless, and no device is ever skipped.
template <typename F>
qsim_status smem_attr_once(F *func, int bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  QS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QSIM_EINVAL;
  }
  const unsigned long long bit = 1ULL << dev;
  if (done.load(std::memory_order_acquire) & bit) return QSIM_OK;
  QS_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
  return QSIM_OK;
}

// ------------------------------------------------------------------------------------
// Gate IR after DAGGER / CONTROL expansion (logical qubits).
// ------------------------------------------------------------------------------------
struct Gate {
  int nt = 0;                 // number of target qubits; the matrix is 2^nt x 2^nt
  int t[QSIM_MAX_FUSED] = {}; // targets, t[0] = most significant matrix-index bit
  std::vector<int> ctrl;      // control qubits (gate acts where all are 1)
  std::vector<cd> m;          // row-major matrix
  int kind = -1;              // qsim_op kind of the instruction it was expanded from
};

// Gate library of the instruction set; returns the number of qubits or -1.
int named_matrix(int kind, const double *params, std::vector<cd> &m);

// Expand an op list (gates and block markers) into a flat gate list.
qsim_status expand_ops(const qsim_op *ops, size_t nops, int n, std::vector<Gate> &out);

// ------------------------------------------------------------------------------------
// Device-side launch descriptors
// ------------------------------------------------------------------------------------
constexpr int kMaxIns = 48;

// Positions (ascending) at which zero bits are inserted into a work-item index, and the
// bits that are then set (controls).
struct Ins {
  int n;
  int pos[kMaxIns];
  unsigned long long set;
};

// Matrix classes that get their own arithmetic.
enum MatClass : int {
  MC_GENERIC = 0,  // full complex 2x2 / 4x4
  MC_REAL = 1,     // real entries
  MC_ANTI = 2,     // [[0, b], [c, 0]]
  MC_SWAP = 3,     // [[0, 1], [1, 0]]
};

enum PhaseClass : int {
  PC_GENERAL = 0,  // multiply by a unit complex number
  PC_NEG = 1,      // multiply by -1
  PC_PLUS_I = 2,   // multiply by +i
  PC_MINUS_I = 3,  // multiply by -i
};

struct StateDev {
  void *amps;
  int n;
  int dtype;
  cudaStream_t stream;
  int split;  // complex128 held as split float pairs (gates run on the FP32 pipe)
  int tc_lo_smem = 0;  // fused tensor-core apply: low TF32 part in shared memory
};

// Per-gate sweeps (sweep.cu). Matrices are complex128, row-major.
qsim_status launch_pair(const StateDev &s, const Ins &ins, unsigned long long off0,
                        unsigned long long off1, const cd m[4], int cls, int64_t *bytes);
qsim_status launch_quad(const StateDev &s, const Ins &ins, const unsigned long long off[4],
                        const cd m[16], int64_t *bytes);
qsim_status launch_phase(const StateDev &s, unsigned long long mask, cd phase, int64_t *bytes);
qsim_status launch_fill_zero_state(const StateDev &s);

// FP64-accurate split-format sweeps for complex128 states (df.cu).
qsim_status launch_pair_df(const StateDev &s, const Ins &ins, unsigned long long off0, unsigned long long off1,
                           const cd m[4], int cls, int64_t *bytes);
qsim_status launch_quad_df(const StateDev &s, const Ins &ins, const unsigned long long off[4], const cd m[16],
                           int64_t *bytes);
qsim_status launch_phase_df(const StateDev &s, unsigned long long mask, cd ph, int64_t *bytes);
qsim_status launch_fused_df(const StateDev &s, const int *phys, int k, unsigned long long ctrl_mask,
                            const void *dev_mat, int64_t *bytes);
void append_fused_df(std::vector<unsigned char> &buf, const cd *u, int k, const int *phys);
qsim_status launch_to_split(const StateDev &s);
qsim_status launch_to_plain(const StateDev &s);

// Merged diagonal gates (sweep.cu, df.cu; tables from diag.cpp). Every amplitude x is
// multiplied by tab[idx(x)], where bit j of idx(x) is bit pos[j] of x (pos ascending,
// nq <= kDiagBits); the table holds the product of the group's diagonal entries for each
// combination of those bits. Table entries: complex64 (re, im, re_lo, im_lo) floats, lo the
// FP64 rounding residue; plain complex128 (re, im) doubles; split complex128 six floats
// (rh, rl, ih, il, r3, i3), the FP64 value exactly.
constexpr int kDiagBits = 10;
struct DiagIdx {
  int nq;
  int pos[kDiagBits];
};
qsim_status launch_diag(const StateDev &s, const DiagIdx &d, const void *dev_tab, int64_t *bytes);
qsim_status launch_diag_df(const StateDev &s, const DiagIdx &d, const void *dev_tab, int64_t *bytes);
// Gate with every off-diagonal entry zero, not the identity, on at most 2 targets.
bool diag_gate(const Gate &g);
// Table of a group of diagonal gates (physical qubits, all within pos[0..nq)) for a state of
// `dtype` (split: the split complex128 format), appended to buf at a 16-byte aligned offset,
// which it returns.
size_t append_diag_table(std::vector<unsigned char> &buf, const std::vector<const Gate *> &gs, const DiagIdx &d,
                       int dtype, bool split);
// Bytes one per-gate sweep of diagonal gate g moves, counted in 64-byte segments (amplitudes
// of B bytes each): the sweep touches the segments that hold an amplitude it changes.
double diag_gate_bytes(const Gate &g, int n, int B);

// Remap (remap.cu): permute the tile qubits {0..L-1} u hi[0..m) (m <= 6) in one sweep;
// the content of tile position b moves to tile position dst_of[b] (positions 0..L-1 are
// the low run, L + j is hi[j]). remap_low_run(n, dtype, m) is the default L (256-byte runs).
int remap_low_run(int n, int dtype, int m);
qsim_status launch_permute(const StateDev &s, int L, const int *hi, int m, const int *dst_of,
                           int64_t *bytes);

// Fused k-qubit unitary on CUDA cores (fused_simt.cu). phys[j] is the physical qubit of
// matrix-index bit (k-1-j); dev_mat holds the matrix (interleaved, state precision).
qsim_status launch_fused_simt_ctl(const StateDev &s, const int *phys, int k,
                                  unsigned long long ctrl_mask, const void *dev_mat,
                                  int64_t *bytes);

// Tensor-core 3xTF32 fused apply on physical qubits 0..k-1 (fused_tc.cu).
//
// A tile is 128 rows of 2^k amplitudes. Its 7 row bits, in the row-index space (physical
// index >> k), are a run 0..c-1 (c >= 2, one TMA box of 2^c rows) plus nh = 7 - c extra
// bits hbit[] (ascending, above the run), which select 2^nh boxes. Tiles enumerate the
// remaining bits (zeros inserted at ins[]). The epilogue writes the value at tile index
// (column cc, row r) to tile index tcol[cc] | OR_b(bit b of r ? wrow[b] : 0), a permutation
// of the k + 7 tile bits: with it a fused block also moves the qubits the next block
// needs into positions 0..k-1 in the same sweep.
//
// Norm tracking (FP64, in device slots): when `slots` is set, the kernel adds the squared
// norm of its input to slots[in_slot] and of its output to slots[out_slot]; when
// ref_slot >= 0 it first scales its input by sqrt(slots[ref_slot] / slots[prev_slot]).
// A circuit uses this to undo the small norm loss of each fused block (the tensor core's
// FP32 accumulation rounds toward zero) in the next block, relative to the first block's
// input norm, without an extra sweep.
constexpr int kTcMaxHbits = 5;  // row bits of a tile outside its low run of c >= 2
constexpr int kTcMaxPhase = 48;  // row-phase gates one fused launch can apply
constexpr int kTcMaxTerms = 96;  // their terms (below)
// A term of a launch's row phases: a row whose row-index bits at `mask` are all 1 is
// multiplied by exp(2 pi i c). A diagonal gate on row bits, exp(2 pi i f(x)) with f read
// from its diagonal, is the sum of its terms by Moebius inversion over the subsets S of its
// qubits' bits: f(x) = sum_S c_S [every bit of S set in x]; mask 0 is a phase of the whole
// state.
struct TcPhaseTerm {
  unsigned long long mask;
  float c;
};
struct TcTilePlan {
  int c, nh;
  int hbit[kTcMaxHbits];
  int ins_n;
  int ins[8];
  int ident;
  // 1: tile bit 0 maps to itself (columns 2g, 2g + 1 stay adjacent); 2: column bit 0 and
  // row bit pair_row (< 5, a lane bit of the epilogue warps) swap, and lane pairs exchange
  // values so that each still stores adjacent pairs; 0: single complex stores
  int pair, pair_row;
  int tcol[32];
  int wrow[7];
  // Filled by launch_fused_tc from tcol: byte offset and 16-byte swizzle bits that column
  // cc contributes to a single-complex destination (pair = 0 stores)
  int ubase[32];
  unsigned char xu[32];
  double *slots;
  int in_slot, out_slot, ref_slot, prev_slot;
  int nterm;   // row-phase terms applied to the tile's input rows (the layout before the epilogue)
  int nvary;   // set by launch_fused_tc: term[0 .. nvary) read a tile row bit, the rest do not
  TcPhaseTerm term[kTcMaxTerms];
};
bool fused_tc_supported(const StateDev &s, int k);
void tc_identity_plan(int k, TcTilePlan &p);
bool tc_plan_valid(int n, int k, const TcTilePlan &p);
qsim_status launch_fused_tc(const StateDev &s, int k, const void *dev_rmats, const TcTilePlan &plan,
                            int64_t *bytes);
// QSIM_ETIMEOUT (and clears the flag) if a bounded wait in the fused kernel ran out.
qsim_status tc_take_timeout();
qsim_status tc_wait_selftest(int ms, cudaStream_t st);
// Host-side preparation of the split R matrices (hi, lo) for one unitary.
void build_tc_operands(int k, const cd *u_phys, float *dst_hi, float *dst_lo);
size_t tc_operand_floats(int k);

// Reductions (reduce.cu). scratch holds at least reduce_scratch_bytes(n) bytes.
size_t reduce_scratch_bytes(int n);
qsim_status red_norm(const StateDev &s, double *scratch, double *host_out);
qsim_status red_inner(const StateDev &a, const void *b_amps, double *scratch, double host_out[2]);
qsim_status red_p1_all(const StateDev &s, double *scratch, double *host_total,
                       double *host_p1 /* n physical */);
qsim_status red_probs(const StateDev &s, const int *phys, int m, double *scratch,
                      double *host_out);
qsim_status red_sample_seeded(const StateDev &s, uint64_t seed, uint64_t shots, double *scratch,
                              uint64_t *host_idx);

int num_sms();

// Autotuner (tune.cpp): measured bandwidths (GB/s) of the sweep kinds on this device.
struct TuneTable {
  bool valid;
  double gbs_pair_c64, gbs_pair_df, gbs_remap, launch_us;
  double gbs_fused[6];     // tensor-core fused apply (complex64), by width
  double gbs_fused_df[6];  // CUDA-core fused apply, split complex128, by width
  int pair_grid_mult;
};
extern int g_pair_grid_mult;  // blocks per SM of the per-gate sweeps (default 8)
qsim_status autotune(cudaStream_t st);
const TuneTable *tune_table();

// A planned gate list (actions, matrices, entry and exit layout), defined in api.cpp.
struct PreparedPlan;
struct PreparedPlanDeleter {
  void operator()(PreparedPlan *p) const;
};
using PlanPtr = std::unique_ptr<PreparedPlan, PreparedPlanDeleter>;

}  // namespace qsim

// ------------------------------------------------------------------------------------
// The opaque state handle.
// ------------------------------------------------------------------------------------
struct qsim_state {
  int n = 0;
  int dtype = 0;
  int fmt = 0;          // complex128: 0 plain doubles, 1 split float pairs
  int fp64_native = 0;  // complex128: run gates with FP64 instructions on plain doubles
  // complex128 split format: sweeps applied since the state last held exact values (reset,
  // host copy); past kSplitSweepLimit the state switches to FP64 instructions (auto_native)
  int64_t split_sweeps = 0;
  int auto_native = 0;
  int tc_lo_smem = 0;   // complex64 fused tensor-core apply: low TF32 part in shared memory
  void *amps = nullptr;
  bool owned = false;
  cudaStream_t stream = nullptr;
  int l2p[64];  // logical -> physical qubit
  int p2l[64];  // physical -> logical qubit
  double *scratch = nullptr;
  size_t scratch_bytes = 0;
  // matrix arena for fused unitaries: pinned host staging + device copy
  void *mat_dev = nullptr;
  void *mat_host = nullptr;
  size_t mat_bytes = 0;
  cudaEvent_t mat_event = nullptr;
  // cached CUDA graph of the last captured circuit run
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_key = 0;
  void *graph_mat_dev = nullptr;  // arena the cached graph reads its matrices from
  double *graph_slots = nullptr;  // norm slots the cached graph uses
  double *norm_slots = nullptr;   // FP64 norm slots of fused blocks (2 per fused launch)
  size_t norm_slots_n = 0;
  int64_t graph_bytes = 0;
  cudaStream_t cap_stream = nullptr;  // private stream for capture when the state's is legacy
  qsim_run_stats stats{};
  // the last plan qsim_run_circuit made, reused when the same gate list runs again from
  // the same layout with the same options
  qsim::PlanPtr last_plan;
  uint64_t last_plan_key = 0;
};

namespace qsim {

// Split-format sweeps a complex128 state may take before it continues with FP64
// instructions. Each split update adds roundings of a few 2^-48 of the amplitudes it
// touches, with no preferred sign, so the error grows like the square root of the sweep
// count: measured 9.8e-13 after 9856 sweeps on a state whose largest amplitude is 1, which
// puts 4096 sweeps at about 6e-13, under the 1e-12 bar of the FP64 path.
constexpr int64_t kSplitSweepLimit = 4096;

// Run an expanded gate list on s: the body of qsim_run_circuit.
qsim_status run_gate_list(qsim_state *s, const std::vector<Gate> &gates, qsim_run_opts o);
// dst <- src: the amplitudes (device copy on dst's stream) and the qubit layout; the two
// states have the same width and dtype.
qsim_status copy_state(qsim_state *dst, const qsim_state *src);

// A gate list planned once from a given layout and run on any state of the same width and
// dtype that is in that layout (fixed fusion width, no renormalisation, no graph).
// Plans `gates` from s's current layout and format; s itself is left unchanged.
qsim_status prepare_gate_list(qsim_state *s, const std::vector<Gate> &gates, qsim_run_opts o, PlanPtr &out);
// Whether s has the plan's width, dtype, entry layout and format.
bool plan_matches(const PreparedPlan &p, const qsim_state *s);
// Uploads the plan's matrices into s's arena, launches it on s's stream and leaves s in
// the plan's exit layout (QSIM_EINVAL if plan_matches fails).
qsim_status run_prepared(qsim_state *s, const PreparedPlan &p);
// Plans a gate list made of consecutive segments (segment i starts at gate seg_begin[i],
// seg_begin[0] = 0) from s's current layout as one plan whose fused blocks never mix two
// segments; a segment may end by moving the next one's qubits in its last epilogue. s is
// left unchanged.
qsim_status prepare_segments(qsim_state *s, const std::vector<Gate> &gates, const std::vector<size_t> &seg_begin,
                             qsim_run_opts o, PlanPtr &out);
// Runs segment i of such a plan on s, which must be in the plan's layout and format at
// that segment's start (QSIM_EINVAL otherwise); upload first copies the plan's matrices
// into s's arena (once per state, and again after anything else wrote the arena).
qsim_status run_prepared_segment(qsim_state *s, const PreparedPlan &p, int i, bool upload);
// Sweeps and stand-alone remap sweeps of each segment of a segmented plan.
void segment_counts(const PreparedPlan &p, std::vector<int64_t> &sweeps, std::vector<int64_t> &remaps);
// Host-only: plans the segments for an n-qubit state of the given dtype from the identity
// layout (tensor-core path assumed where it applies) and counts as segment_counts does.
qsim_status dry_plan_segments(int n, int dtype, const std::vector<Gate> &gates, const std::vector<size_t> &seg_begin,
                              qsim_run_opts o, std::vector<int64_t> &sweeps, std::vector<int64_t> &remaps);

}  // namespace qsim
