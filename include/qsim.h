/*
 * qsim.h - C ABI of the GB300 full-amplitude state-vector library (libqsim.so).
 *
 * The method is the full-amplitude mode of Wang et al., "A quantum circuit simulator
 * and its applications on Sunway TaihuLight supercomputer" (Section 2.2): an n-qubit
 * state |phi> = sum_i a_i |i> is stored whole as 2^n complex amplitudes, with
 * i = sum_k i_k 2^k so that qubit k is bit k of the index (Eq. 1), and every gate
 * updates it in place (Eq. 2 for one qubit, Eq. 3 with a control qubit).
 *
 * Conventions used by every call:
 *  - Amplitudes are interleaved complex numbers (re, im): complex64 = two floats,
 *    complex128 = two doubles. A state of n qubits holds 2^n of them.
 *  - Qubit numbers are LOGICAL (the paper's numbering). The library may keep the
 *    amplitudes in a permuted physical order (a qubit remap); every read-out call
 *    translates back, so callers never see the physical order.
 *  - Matrices are complex128 in row-major order, interleaved (re, im), 2 doubles per
 *    entry. For a matrix on several qubits, the FIRST listed qubit is the MOST
 *    significant bit of the row/column index, as in the paper's CNOT, CZ, CR, SWAP,
 *    iSWAP and TOFFOLI matrices (Appendix A-1).
 *  - Host arrays passed in are owned by the caller and only read during the call.
 *  - Calls that change the state are asynchronous on the state's CUDA stream; calls
 *    that return numbers to the host synchronise that stream before returning.
 *  - Every call returns a qsim_status. On QSIM_EINVAL the state is unchanged. A CUDA
 *    error from an earlier asynchronous launch is reported as QSIM_ECUDA by the next
 *    call that synchronises. qsim_last_error() returns a message for the calling
 *    thread's most recent failure.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim_state qsim_state; /* opaque; created and freed by the library */

typedef enum {
  QSIM_C64 = 0,  /* complex64 amplitudes, FP32 arithmetic (FP64 in reductions)   */
  QSIM_C128 = 1  /* complex128 amplitudes, FP64-accurate arithmetic              */
} qsim_dtype;

typedef enum {
  QSIM_OK = 0,
  QSIM_EINVAL = 1,       /* bad argument: qubit out of range, duplicates, size ... */
  QSIM_ENOMEM = 2,       /* device allocation failed                              */
  QSIM_ECUDA = 3,        /* a CUDA call or kernel failed                           */
  QSIM_ETIMEOUT = 4,     /* a bounded device-side wait ran out                     */
  QSIM_EUNSUPPORTED = 5  /* valid request that the library does not implement      */
} qsim_status;

/* Largest qubit count a state may have (2^40 complex64 amplitudes = 8 TiB). */
#define QSIM_MAX_QUBITS 40
/* Largest fused-unitary width accepted by qsim_apply_fused. */
#define QSIM_MAX_FUSED 5

/*
 * Gate and block kinds of the instruction set (Appendix A-1). QSIM_OP_SX / QSIM_OP_SY
 * are the principal square roots of X and Y, used by random circuits; they are not in
 * the paper. QSIM_OP_MATRIX is an explicit matrix given by the caller.
 */
typedef enum {
  QSIM_OP_MATRIX = 0,
  QSIM_OP_H = 1, QSIM_OP_X = 2, QSIM_OP_Y = 3, QSIM_OP_Z = 4, QSIM_OP_S = 5, QSIM_OP_T = 6,
  QSIM_OP_SX = 7, QSIM_OP_SY = 8,
  QSIM_OP_RX = 9, QSIM_OP_RY = 10, QSIM_OP_RZ = 11, /* params[0] = theta (radians)     */
  QSIM_OP_U4 = 12,   /* params = (alpha, beta, gamma, delta), the angle form         */
  QSIM_OP_CNOT = 13, QSIM_OP_CZ = 14,
  QSIM_OP_CR = 15,   /* diag(1, 1, 1, e^{i theta}), params[0] = theta                */
  QSIM_OP_SWAP = 16, QSIM_OP_ISWAP = 17, QSIM_OP_TOFFOLI = 18,
  QSIM_OP_DAGGER = 32, QSIM_OP_ENDDAGGER = 33,   /* inverse of the enclosed block      */
  QSIM_OP_CONTROL = 34, QSIM_OP_ENDCONTROL = 35  /* qubits[0..nq) control the block    */
} qsim_op_kind;

/*
 * One instruction. For gates, qubits[0..nq) are listed as in the paper's syntax
 * (CNOT i,j: i = control, j = target; TOFFOLI i,j,k: i, j controls, k target).
 * controls[0..nc) are extra control qubits (the gate acts where all of them are 1).
 * For QSIM_OP_MATRIX, matrix points to a 2^nq x 2^nq complex128 matrix (nq <= 3).
 * Block markers use only kind (and qubits/nq for CONTROL).
 */
typedef struct {
  int32_t kind;
  int32_t nq;
  int32_t qubits[3];
  int32_t nc;
  const int32_t *controls;
  double params[4];
  const double *matrix;
} qsim_op;

/* Options of qsim_run_circuit. A zeroed struct (or NULL) means: per-gate, no remap. */
typedef struct {
  int32_t fuse;       /* 0: one sweep per gate; 2..5: fuse into k-qubit unitaries;
                         -1: pick k with the autotuner                              */
  int32_t remap;      /* nonzero: the planner may swap qubits to low positions     */
  int32_t use_graph;  /* nonzero: capture the launches in a CUDA graph, then launch */
  int32_t no_renorm;  /* nonzero: do not renormalise fused tensor-core blocks. By
                         default each fused block scales its input so that the state
                         keeps the norm it had before the first fused block (FP64
                         norms taken inside the fused kernels, no extra sweep): the
                         tensor cores' FP32 accumulation rounds toward zero and would
                         otherwise shrink the norm by a few 1e-7 per block            */
  int32_t merge_diagonals; /* nonzero, with fuse = 0: diagonal gates (every off-diagonal
                         entry zero; targets and controls on at most 10 qubits) that commute
                         past the gates listed between them run together as one sweep, which
                         multiplies each amplitude by the product of their diagonal entries
                         (a table of 2^q products over the q qubits they touch, formed in
                         double-double from the FP64 entries), whenever the separate sweeps
                         they replace would move more bytes (counted in 64-byte segments,
                         which a low-target phase touches whole) or cost more launches.
                         0: one sweep per gate, the plain method                      */
} qsim_run_opts;

/* Planner statistics of the last qsim_run_circuit on a state. */
typedef struct {
  int64_t gates;          /* listed gates after block expansion                     */
  int64_t sweeps;         /* state sweeps launched (gate, fused and remap sweeps)   */
  int64_t fused_blocks;   /* fused unitaries applied                                */
  int64_t remaps;         /* remap sweeps                                           */
  int64_t kernels;        /* kernel launches                                        */
  double bytes;           /* algorithmic HBM bytes of all sweeps                    */
  int64_t fuse_width;     /* fusion width used (0 = one sweep per gate)             */
  double predicted_ms;    /* autotuner's estimate for the chosen plan (fuse = -1)   */
  int64_t phase_gates;    /* diagonal gates on qubits outside a fused block's k, applied
                             by that block as per-row phases (tensor-core path)       */
  int64_t epilogue_remaps; /* fused launches whose epilogue also moved qubits (no sweep
                              of its own)                                             */
  int64_t plan_reused;    /* 1: the state's last plan was reused (the same gate list, options,
                             qubit layout and format as the run that made it), 0: planned */
  int64_t fp64_fallback;  /* complex128 in the split format: 1 when this run took FP64
                             instructions because the state had used up its budget of 4096
                             split sweeps since it last held exact values (qsim_reset,
                             qsim_copy_from_host, qsim_wrap); each split sweep adds roundings of
                             a few 2^-48, and past the budget their sum could exceed 1e-12. The
                             state stays on FP64 instructions until it holds exact values again */
  int64_t upload_bytes;   /* host-to-device bytes of the run: the plan's matrices, copied from
                             the state's pinned staging buffer */
  int64_t diag_sweeps;    /* merge_diagonals: merged diagonal sweeps of the run          */
  int64_t diag_gates;     /* merge_diagonals: gates those sweeps applied                  */
} qsim_run_stats;

/* ---- state lifetime -------------------------------------------------------------- */

/* QINIT n (Appendix A-1): allocate 2^n amplitudes on the current device, set |0...0>.
 * stream: a cudaStream_t (NULL = default stream). Fails with QSIM_ENOMEM if the
 * device has no room. */
qsim_status qsim_create(int n, int dtype, void *stream, qsim_state **out);

/* Like qsim_create, but on caller-owned device memory of 2^n amplitudes (e.g. a torch
 * tensor). The library never frees dev_ptr. The contents are taken as the state in
 * logical order; call qsim_reset for |0...0>. dev_ptr must be 256-byte aligned. While
 * the library works on the state the buffer may hold a permuted or (complex128) split
 * representation; qsim_canonicalize restores plain logical order. */
qsim_status qsim_wrap(void *dev_ptr, int n, int dtype, void *stream, qsim_state **out);

/* Free the handle (and the amplitudes if the library allocated them). */
void qsim_destroy(qsim_state *s);

/* Set |0...0> and the identity qubit layout. */
qsim_status qsim_reset(qsim_state *s);

/* Change the stream later calls are ordered on. */
qsim_status qsim_set_stream(qsim_state *s, void *stream);

/* Wait for all work queued on the state's stream; reports asynchronous errors. */
qsim_status qsim_synchronize(qsim_state *s);

/* Bring the amplitudes back to logical order (identity layout) and, for complex128, to
 * plain doubles (see qsim_set_option): afterwards the device buffer holds the state
 * exactly as the Eq. (1) index order defines it. */
qsim_status qsim_canonicalize(qsim_state *s);

/* State options. QSIM_OPT_FP64_NATIVE (complex128 only): 0 (default) runs gates in an
 * FP64-accurate split format - between calls each amplitude is held as
 * (re_hi, im_hi, re_lo, im_lo) floats with re = re_hi + re_lo, and the updates use
 * error-free FP32 transformations (about 2^-48 relative error per update) because GB300's
 * FP64 pipe is 64x slower than its FP32 pipe; 1 runs them with FP64 instructions on plain
 * doubles. Read-outs and host copies always see plain complex128 values. */
#define QSIM_OPT_FP64_NATIVE 1
/* QSIM_OPT_TC_LO_SMEM (complex64 fused tensor-core apply): 0 (default) keeps the low TF32
 * part of each state tile in tensor memory, which leaves shared memory for five (k = 5) or
 * eight (k = 4) loads in flight per SM; 1 keeps it in shared memory with three. Results
 * are identical; only the speed differs. */
#define QSIM_OPT_TC_LO_SMEM 2
qsim_status qsim_set_option(qsim_state *s, int option, int value);

/* ---- gates ------------------------------------------------------------------------ */

/* Apply a 1- or 2-qubit gate: Eq. (2) for nt = 1, nc = 0; Eq. (3) for nt = 1 with
 * controls; the 4x4 form (SWAP, iSWAP, any 2-qubit matrix) for nt = 2. m holds
 * 2^nt x 2^nt complex128 entries. Targets and controls must be distinct and < n. */
qsim_status qsim_apply_gate(qsim_state *s, const int *targets, int nt, const int *controls,
                            int nc, const double *m);

/* Apply a k-qubit unitary u (2^k x 2^k complex128, qubits[0] = most significant
 * index bit), 1 <= k <= QSIM_MAX_FUSED, in one state sweep. u is cast once to the
 * state's precision; on complex64 states with k >= 4 the product runs on the tensor
 * cores as a split-precision (3xTF32) complex GEMM with FP32 accumulation. */
qsim_status qsim_apply_fused(qsim_state *s, const int *qubits, int k, const double *u);

/* Run an instruction list (gates and DAGGER / CONTROL blocks, Appendix A-1) on the
 * state. Blocks are expanded on the host, matrices are composed in FP64, and the plan
 * (per-gate sweeps, or fused k-qubit unitaries with qubit remaps) follows opts. The
 * state keeps its last plan: the same expanded gate list (compared exactly) with the same
 * options, from the same qubit layout and format (as after qsim_reset or
 * qsim_copy_from_host), runs it again without planning (run_stats.plan_reused = 1). */
qsim_status qsim_run_circuit(qsim_state *s, const qsim_op *ops, size_t nops,
                             const qsim_run_opts *opts);

/* Measure the sweep kinds on the current device (pair sweep at several grid sizes, fused
 * tensor-core kernel for k = 4 and 5, remap sweep, split complex128 pair sweep and fused
 * apply for k = 2..5, launch cost) on a 128 MiB scratch state, once per device;
 * qsim_run_circuit with fuse = -1 then plans the circuit for each candidate width
 * (complex64: 0, 4, 5; split complex128: 0, 2..5) and runs the plan with the lowest
 * predicted time. Called implicitly by the first fuse = -1 run; call it before any stream
 * capture. out (may be NULL) receives up to nout values: GB/s of the complex64 pair
 * sweep, the split complex128 pair sweep, fused k = 4, fused k = 5, the remap sweep, then
 * the launch cost in microseconds, the chosen blocks per SM, and GB/s of the split
 * complex128 fused apply for k = 2, 3, 4, 5. */
qsim_status qsim_autotune(void *stream, double *out, int nout);

/* Plan an instruction list for an n-qubit state of `dtype` on the host only, as
 * qsim_run_circuit would from the identity layout (assuming the tensor-core kernel is
 * available), and report the plan's statistics; no device is touched. */
qsim_status qsim_plan_dry_run(int n, int dtype, const qsim_op *ops, size_t nops,
                              const qsim_run_opts *opts, qsim_run_stats *out);

/* One gate of an expanded instruction list: nt targets (targets[0] = the most significant
 * bit of the matrix index; unused entries -1), nc controls at ctrls[ctrl_off .. ctrl_off +
 * nc), the 2^nt x 2^nt complex128 matrix (row-major, interleaved) at mats[2 mat_off ..],
 * and the kind of the instruction it comes from. */
typedef struct {
  int32_t kind;
  int32_t nt;
  int32_t targets[QSIM_MAX_FUSED];
  int32_t nc;
  int32_t ctrl_off;
  int64_t mat_off;
} qsim_gate_rec;

/* Host only: the gate list that qsim_run_circuit applies for `ops` on n qubits (1..64):
 * DAGGER blocks reversed with adjoint matrices, CONTROL qubits appended to every gate of
 * their block (Appendix A-1), and CNOT, CZ, CR and TOFFOLI in controlled form (one target,
 * their first listed qubits as controls). sizes[0..2] receive the numbers of gates,
 * controls and complex matrix entries. With gates, ctrls and mats all NULL only the sizes
 * are written; otherwise the arrays (capacities gate_cap, ctrl_cap, mat_cap complex
 * entries) must hold them (QSIM_EINVAL and nothing written if not). Errors as
 * qsim_run_circuit (bad qubits, unbalanced blocks). */
qsim_status qsim_expand(int n, const qsim_op *ops, size_t nops, qsim_gate_rec *gates, size_t gate_cap,
                        int32_t *ctrls, size_t ctrl_cap, double *mats, size_t mat_cap, size_t sizes[3]);

/* Statistics of the state's last qsim_run_circuit. */
qsim_status qsim_last_run_stats(qsim_state *s, qsim_run_stats *out);

/* ---- read-outs (synchronise the stream) ----------------------------------------- */

/* Amplitude of logical basis index `index` as (re, im) doubles. */
qsim_status qsim_amplitude(qsim_state *s, uint64_t index, double out[2]);

/* PMEASURE (Appendix A-1): probabilities of the 2^m outcomes of the listed qubits,
 * state unchanged. out[j] for j = sum_t bit(qubits[t]) << (m-1-t): the first listed
 * qubit is the leftmost character of the printed outcome (Appendix A-2). FP64 sums.
 * 1 <= m <= 24, out holds 2^m doubles. */
qsim_status qsim_probabilities(qsim_state *s, const int *qubits, int m, double *out);

/* MEASURE (App. A-1): measure one qubit and keep evolving the post-measurement state. The
 * outcome is the smallest r in {0, 1} with u < P(0) + ... + P(r), P the FP64 marginal of
 * `qubit` (relative to the state's norm), u in [0, 1) supplied by the caller; the state is
 * then projected onto the outcome and renormalised to norm 1 (one sweep). *outcome gets r,
 * *prob (may be NULL) gets P(r). QSIM_EINVAL for a bad qubit, u outside [0, 1) or a state
 * of zero norm (no state change). Synchronises the state's stream. */
qsim_status qsim_measure(qsim_state *s, int qubit, double u, int *outcome, double *prob);

/* Draw `shots` outcomes of the listed qubits (m = 0 or qubits = NULL: all n qubits,
 * out = full logical basis index). Shot j uses u_j = U01(Philox4x32-10(key = seed,
 * counter = (j_lo, j_hi, 0, 0x53414D50))), U01(x0, x1) = ((x0 << 32 | x1) >> 11) 2^-53,
 * and picks the smallest logical index i with u_j * sum|a|^2 < sum_{l <= i} |a_l|^2,
 * then keeps the listed bits packed as in qsim_probabilities. The state is left in
 * logical order. */
qsim_status qsim_sample(qsim_state *s, const int *qubits, int m, uint64_t shots,
                        uint64_t seed, uint64_t *out);

/* Sum of |a_i|^2, accumulated in FP64. */
qsim_status qsim_norm(qsim_state *s, double *out);

/* <a|b> (FP64 accumulation) of two states of the same n and dtype. */
qsim_status qsim_inner(qsim_state *a, qsim_state *b, double out[2]);

/* |<a|b>|^2 / (<a|a><b|b>). */
qsim_status qsim_fidelity(qsim_state *a, qsim_state *b, double *out);

/* <Z_q> = sum_i (-1)^{i_q} |a_i|^2 / sum_i |a_i|^2 for every logical qubit q; out[n]. */
qsim_status qsim_expect_z(qsim_state *s, double *out);

/* Copy the whole state to / from host memory in logical order. host holds 2^n
 * amplitudes of the state's dtype. Pinned host memory gives the fastest copies. */
qsim_status qsim_copy_to_host(qsim_state *s, void *host);
qsim_status qsim_copy_from_host(qsim_state *s, const void *host);

/* Like qsim_copy_to_host, but asynchronous: the restore of logical order (if needed) and
 * the copy are queued on the state's stream and the call returns; host holds the state
 * once the stream has reached that point (qsim_synchronize). host should be pinned memory
 * (with pageable memory the copy is not asynchronous). Two states on two streams can then
 * overlap one state's copies with the other's gates. */
qsim_status qsim_copy_to_host_async(qsim_state *s, void *host);

/* PMEASURE without any allocation. The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory when they need the read-out - code that must
 * not synchronise the device (cudaFree does) and programs on a fixed memory budget.
 * amps: device pointer to 2^n plain amplitudes of `dtype` in their own index order (no
 * qubit remap is applied: qubits[] are bit positions of that array; for a library state,
 * call qsim_canonicalize first). out: DEVICE pointer to
 * 2^m doubles, written with out[j], j = sum_t bit(qubits[t]) << (m-1-t), like
 * qsim_probabilities. 1 <= m <= 10; larger m returns QSIM_EINVAL. Asynchronous on
 * `stream`; calls no allocating routine. Its scratch is a fixed 2 MiB device array inside
 * the library, held by every GPU that loads it until exit and shared by all calls: calls
 * that overlap on the GPU race on it, so order them on one stream. The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) and loads the
 * call's kernels on that device (cudaFuncGetAttributes), so later calls load no code. */
qsim_status qsim_probabilities_noalloc(const void *amps, int n, int dtype, const int *qubits,
                                       int m, double *out, void *stream);

/* ---- noisy trajectories (Section 2.4) --------------------------------------------- */

/* Widest trajectory state (complex64). */
#define QSIM_TRAJ_MAX_QUBITS 24

/* Noise channels of Eq. (5); at one noisy site they run in this order. */
#define QSIM_NOISE_DEPOLARIZING 0      /* I, X, Y, Z with weights 1 - 3p/4, p/4, p/4, p/4    */
#define QSIM_NOISE_AMPLITUDE_DAMPING 1 /* K1 = diag(1, sqrt(1-p)), K2 = sqrt(p) |0><1|        */
#define QSIM_NOISE_BIT_FLIP 2          /* K1 = sqrt(p) I, K2 = sqrt(1-p) X (p = 1: noiseless) */
#define QSIM_NOISE_PHASE_FLIP 3        /* K1 = sqrt(p) I, K2 = sqrt(1-p) Z (p = 1: noiseless) */
#define QSIM_NOISE_BIT_PHASE_FLIP 4    /* K1 = sqrt(p) I, K2 = sqrt(1-p) Y (p = 1: noiseless) */
#define QSIM_NOISE_PHASE_DAMPING 5     /* K1 = diag(1, sqrt(1-p)), K2 = sqrt(p) |1><1|        */
#define QSIM_NOISE_CHANNELS 6
/* Counter word 2 of the joint draw of a two-qubit gate (kron = 1). */
#define QSIM_NOISE_KRON_SITE 0x4B524F4Eu

/* A batch of Monte-Carlo trajectories of noisy circuits (Section 2.4). Program p is an
 * instruction list (gates on at most 2 qubits each, DAGGER/CONTROL blocks allowed) on
 * prog_qubits[p] qubits (2..24); trajectory t runs program traj_prog[t] from |0...0> in
 * complex64. A gate is noisy when noisy_kinds is 0 or has bit `kind` of the instruction it
 * comes from set (a gate inside DAGGER / CONTROL blocks keeps its own kind). After every
 * noisy gate, for every qubit it touches (ascending), each channel c with bit c of
 * `channels` set runs in channel order with its p[c] (a zeroed struct has no noise):
 * branch i is taken with probability ||K_i psi||^2 / ||psi||^2 when
 * u = U01(Philox4x32-10(key = seed, counter = (t, gate, qubit, c))) falls in its
 * cumulative interval (smallest i with u < p_1 + ... + p_i), then psi <- K_i psi /
 * ||K_i psi||. With kron = 1 a two-qubit gate on qubits a < b instead takes one draw per
 * channel, counter (t, gate, QSIM_NOISE_KRON_SITE, c), over the 2-qubit operators
 * K_i (x) K_j (K_i on b, K_j on a; joint index i * s + j for s branches). Gates are
 * counted from 0 in the expanded program. */
typedef struct {
  int32_t nprog;
  const int32_t *prog_qubits;      /* [nprog] */
  const qsim_op *const *prog_ops;  /* [nprog] instruction lists */
  const size_t *prog_nops;         /* [nprog] */
  int32_t ntraj;
  const int32_t *traj_prog;        /* [ntraj] program of each trajectory */
  uint64_t seed;
  uint32_t channels;               /* bit c set: channel c runs at every noisy site */
  uint32_t noisy_kinds;            /* bit k set: gates of kind k are noisy; 0: every gate */
  double p[QSIM_NOISE_CHANNELS];   /* Eq. (5)'s p of each channel, in [0, 1] */
  int32_t kron;                    /* 1: joint two-qubit draws; 0: one draw per qubit */
  int32_t shots;                   /* one shot from each trajectory t < shots */
  int32_t event_cap;               /* branch events kept per trajectory (0: none) */
} qsim_traj_batch;

/* Run every trajectory of the batch in one persistent kernel launch on `stream` and copy
 * the results to the host (this call synchronises the stream):
 *   zexp_out[t * QSIM_TRAJ_MAX_QUBITS + q] = <Z_q> of trajectory t's final state (q < its
 *     width; the rest 0);
 *   samples_out[t], t < shots: basis index drawn from trajectory t's final state with
 *     u = U01(Philox(seed, (t, gates, 0, 0x53414D50))), the smallest i with
 *     u * sum|a|^2 < sum_{l <= i} |a_l|^2;
 *   events_out[t * event_cap + e] (event_cap > 0) and nevents_out[t] (may be NULL): the
 *     number of the non-identity branches taken on one qubit and up to event_cap of them,
 *     in gate order, coded (gate << 12) | (qubit << 6) | (channel << 2) | branch, the
 *     branch numbered from 0 in Eq. (5)'s order (depolarizing 1 X, 2 Y, 3 Z; the other
 *     channels 1 = K2). A joint draw gives one event per qubit whose factor is not K1 (the
 *     lower qubit first). Gates on disjoint qubits may be applied out of list order (their
 *     operators commute), so when more than event_cap events occur the kept ones need not
 *     be the earliest.
 * Device memory: the programs, the outputs and, for widths above 14, 2^width complex64
 * amplitudes per SM are allocated on `stream` for the call and freed before it returns.
 * QSIM_EINVAL for a p outside [0, 1], an unknown channel bit or a bad buffer. */
qsim_status qsim_run_trajectories(const qsim_traj_batch *b, void *stream, double *zexp_out,
                                  uint64_t *samples_out, uint32_t *events_out, int32_t *nevents_out);

/* The same batch (Section 2.4) in three steps, so that the launch can be recorded into a
 * CUDA graph and replayed. qsim_run_trajectories is prepare + launch + results + destroy.
 *
 * qsim_traj_prepare: checks and expands the batch (errors as qsim_run_trajectories), then
 *   allocates one device block on `stream` for the programs, the outputs, the wide-state
 *   scratch and the kept states, uploads the programs and synchronises `stream`. keep[0..
 *   nkeep) (may be NULL when nkeep = 0) lists trajectories whose final state, normalised,
 *   is kept on the device for qsim_traj_state (2^width complex64 amplitudes each). The seed
 *   lives in one word of mapped pinned host memory that each launch reads when it starts.
 *   *out receives the plan (owned by the library until qsim_traj_destroy).
 * qsim_traj_set_seed: stores a new seed for the next launches (a host write; call it only
 *   while no launch of this plan is running, e.g. after qsim_traj_results returned).
 * qsim_traj_launch: three device memsets (work counter, <Z> sums, event counts) and one
 *   k_traj launch on `stream`, on the plan's device buffers only: no allocation, no host
 *   copy, no synchronisation, so a stream capture may record it. Launches of one plan
 *   share its buffers: order them (one stream) and read each one's results before the
 *   next. QSIM_EINVAL if the current device is not the plan's.
 * qsim_traj_results: copies the outputs of the last launch to the host exactly as
 *   qsim_run_trajectories documents them, and synchronises `stream`.
 * qsim_traj_state: copies kept state i (the i-th entry of keep) of the last launch to host
 *   memory (2^width complex64 values, logical order, sum |a|^2 = 1 up to FP32 rounding) and
 *   synchronises `stream`. QSIM_EINVAL for an index outside [0, nkeep).
 * qsim_traj_destroy: frees the plan; its device block is released in the order of the
 *   prepare stream, so every launch of the plan must be complete or ordered before it. */
typedef struct qsim_traj_plan qsim_traj_plan;
qsim_status qsim_traj_prepare(const qsim_traj_batch *b, const int32_t *keep, int32_t nkeep, void *stream,
                              qsim_traj_plan **out);
qsim_status qsim_traj_set_seed(qsim_traj_plan *p, uint64_t seed);
qsim_status qsim_traj_launch(qsim_traj_plan *p, void *stream);
qsim_status qsim_traj_results(qsim_traj_plan *p, void *stream, double *zexp_out, uint64_t *samples_out,
                              uint32_t *events_out, int32_t *nevents_out);
qsim_status qsim_traj_state(qsim_traj_plan *p, int32_t i, void *stream, void *host_out);
void qsim_traj_destroy(qsim_traj_plan *p);

/* ---- partial amplitude mode (Section 2.2, Eq. 4) ----------------------------------- */

/* The dividing line splits an n-qubit circuit (2 <= n <= 64) into the upper block, qubits
 * [0, cut), and the lower block, [cut, n) (each at most QSIM_MAX_QUBITS). A gate across the
 * line must be a controlled gate: its listed qubits are taken as controls, in order, while
 * its matrix has the form P0 (x) I + P1 (x) U' in them and the rest still crosses the line
 * (CNOT, CZ and CR across the line, TOFFOLI, gates inside CONTROL blocks); then its targets
 * lie on one side and its controls C on the other side split it by Eq. (4), extended to
 * several controls: (I - P_C) (x) I + P_C (x) U, P_C the projector on C = 1...1. SWAP and
 * ISWAP across the line have no such form (QSIM_EUNSUPPORTED). With c decomposed gates
 * (c <= 30) the 2^(c+1) sub-circuits give
 *     <x|psi> = sum_b upper_b[x mod 2^cut] * lower_b[x >> cut],
 * b over the 2^c choices of term. */
typedef struct {
  int32_t cut;    /* 0: n / 2 (the middle) */
  int32_t dtype;  /* QSIM_C64 or QSIM_C128: precision of the sub-circuit states */
  int32_t fuse;   /* qsim_run_opts.fuse of every sub-circuit segment (0, 2..5, -1) */
  int32_t remap;  /* qsim_run_opts.remap of every segment */
} qsim_partial_opts;

typedef struct {
  int32_t cut;           /* the dividing line used */
  int32_t decomposed;    /* c */
  int64_t subcircuits;   /* 2^(c+1) */
  int64_t segment_runs;  /* segment simulations: segment s of each block runs 2^s times */
  int32_t slots;         /* states of each block held at once: c + 1 */
  double gates_applied;  /* gate applications over all segment runs */
  double gates_unshared; /* gate applications of the 2^(c+1) sub-circuits run one by one */
  int64_t sweeps;        /* state sweeps of the segment runs over the whole walk (the
                            single-gate term sweeps not counted); qsim_partial_plan counts
                            them as planned for complex64, fuse 5, with remaps */
  int64_t remaps;        /* of those, stand-alone remap sweeps */
} qsim_partial_info;

/* Host-only: decompose the circuit and report the plan in *info (may be NULL); no device
 * work. QSIM_EUNSUPPORTED for a crossing gate without the controlled form. */
qsim_status qsim_partial_plan(int n, const qsim_op *ops, size_t nops, int cut, qsim_partial_info *info);

/* Amplitudes <indices[i]|psi> (i < m; host array, each index < 2^n) into amps_out[2 i],
 * amps_out[2 i + 1] (host, complex128) by the partial amplitude mode. The sub-circuits run
 * on the GPU through the full-amplitude engine on `stream`, prefix-shared: a depth-first
 * walk over the terms keeps c + 1 state pairs (2^cut + 2^(n - cut) amplitudes each, of the
 * chosen dtype) and runs segment s of each block 2^s times; every leaf adds
 * upper[x_u] * lower[x_l] into FP64 accumulators on the device. With fuse >= 0 each
 * block's segments are planned once, as one plan whose fused blocks stay within a segment;
 * the Eq. (4) terms run between segments as single-gate sweeps. Device memory is allocated
 * for the call and freed before it returns; the call synchronises `stream`. QSIM_EINVAL for
 * an index >= 2^n, an unknown dtype or NULL buffers (checked before any device work);
 * QSIM_EUNSUPPORTED as for qsim_partial_plan. */
qsim_status qsim_partial_amplitudes(int n, const qsim_op *ops, size_t nops, const qsim_partial_opts *opts,
                                    const uint64_t *indices, size_t m, double *amps_out, qsim_partial_info *info,
                                    void *stream);

/* ---- host gate library -------------------------------------------------------------- */

/* Matrix of a named gate of Appendix A-1 (kind < QSIM_OP_DAGGER, not MATRIX) into
 * out (2^k x 2^k complex128); *k receives the number of qubits it acts on. */
qsim_status qsim_gate_matrix(int kind, const double *params, int *k, double *out);

/* Self-test of the device-side failure path: launches a kernel whose waits use the same
 * bounded mbarrier wait as the fused kernel, on a barrier that nothing arrives at, with a
 * limit of `ms` milliseconds (1..10000). Returns QSIM_ETIMEOUT when the wait ran out and
 * was reported through the device flag (the expected outcome); the context stays usable.
 * No counterpart in the paper. */
qsim_status qsim_selftest_bounded_wait(int ms, void *stream);

/* Message of the calling thread's most recent failure ("" if none). */
const char *qsim_last_error(void);

/* Library version string. */
const char *qsim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */
