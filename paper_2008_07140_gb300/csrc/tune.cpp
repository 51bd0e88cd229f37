// Autotuner: device microbenchmarks, measured once per device, and the cost model that
// picks the fusion width of a circuit run (qsim_run_circuit with fuse = -1).
//
// The microbenchmarks run on a scratch state larger than L2 (2^24 complex64 amplitudes,
// 128 MiB): the generic pair sweep for several grid sizes (the fastest becomes the grid
// multiplier of the pair, phase and quad sweeps), the tensor-core fused kernel for k = 4
// and 5, the remap sweep, the split complex128 pair sweep and the launch overhead. The
// cost model prices a plan as sum over its launches of (algorithmic bytes / measured
// bandwidth of that launch's kind) + launch overhead.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace qsim {

namespace {

std::mutex g_tune_mu;
TuneTable g_tune[64];

double time_ms(cudaStream_t st, const std::function<qsim_status()> &f, int reps, qsim_status &rc) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  rc = f();  // warm-up
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps && rc == QSIM_OK; ++r) rc = f();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

}  // namespace

int g_pair_grid_mult = 8;

const TuneTable *tune_table() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  return g_tune[dev].valid ? &g_tune[dev] : nullptr;
}

qsim_status autotune(cudaStream_t st) {
  int dev = 0;
  QS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QSIM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune[dev].valid) return QSIM_OK;
  TuneTable t{};
  const int n = 24;
  void *buf = nullptr;
  QS_TRY_CUDA(cudaMalloc(&buf, (size_t)8 << n));
  void *mats = nullptr;
  cudaError_t ce = cudaMalloc(&mats, 1 << 16);
  if (ce != cudaSuccess) {
    cudaFree(buf);
    return cuda_fail(ce, "autotune buffers");
  }
  StateDev d{buf, n, QSIM_C64, st, 0};
  qsim_status rc = launch_fill_zero_state(d);
  const double bytes64 = 2.0 * 8 * (double)(1LL << n);
  // pair sweep, grid multipliers
  const cd u[4] = {cd(0.6, 0.0), cd(0.0, 0.8), cd(0.0, 0.8), cd(0.6, 0.0)};
  Ins ins;
  ins.n = 1;
  ins.pos[0] = 14;
  ins.set = 0;
  double best = 1e30;
  int best_mult = 8;
  for (int mult : {2, 4, 8, 16}) {
    if (rc != QSIM_OK) break;
    g_pair_grid_mult = mult;
    const double ms = time_ms(st, [&]() { return launch_pair(d, ins, 0, 1ULL << 14, u, MC_GENERIC, nullptr); }, 8, rc);
    if (ms < best) {
      best = ms;
      best_mult = mult;
    }
  }
  g_pair_grid_mult = best_mult;
  t.pair_grid_mult = best_mult;
  t.gbs_pair_c64 = bytes64 / (best * 1e-3) / 1e9;
  // launch overhead: a sweep of a tiny state
  {
    StateDev tiny{buf, 10, QSIM_C64, st, 0};
    Ins i2;
    i2.n = 1;
    i2.pos[0] = 3;
    i2.set = 0;
    if (rc == QSIM_OK)
      t.launch_us =
          1e3 * time_ms(st, [&]() { return launch_pair(tiny, i2, 0, 1ULL << 3, u, MC_GENERIC, nullptr); }, 32, rc);
  }
  // fused tensor-core kernel
  for (int k : {4, 5}) {
    if (rc != QSIM_OK || !fused_tc_supported(d, k)) continue;
    std::vector<float> ops(tc_operand_floats(k));
    std::vector<cd> eye((size_t)1 << (2 * k), 0.0);
    for (int i = 0; i < (1 << k); ++i) eye[(size_t)i * (1 << k) + i] = 1.0;
    build_tc_operands(k, eye.data(), ops.data(), ops.data() + ops.size() / 2);
    ce = cudaMemcpyAsync(mats, ops.data(), ops.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "autotune operands");
      break;
    }
    TcTilePlan tp;
    tc_identity_plan(k, tp);
    const double ms = time_ms(st, [&]() { return launch_fused_tc(d, k, mats, tp, nullptr); }, 8, rc);
    t.gbs_fused[k] = bytes64 / (ms * 1e-3) / 1e9;
  }
  // remap sweep (5 pairs)
  if (rc == QSIM_OK) {
    int hi[5] = {10, 12, 15, 18, 21}, dst[16];
    for (int b = 0; b < 10; ++b) dst[b] = b;
    for (int j = 0; j < 5; ++j) {
      dst[j] = 5 + j;
      dst[5 + j] = j;
    }
    const double ms = time_ms(st, [&]() { return launch_permute(d, 5, hi, 5, dst, nullptr); }, 8, rc);
    t.gbs_remap = bytes64 / (ms * 1e-3) / 1e9;
  }
  // split complex128 pair sweep on 2^23 amplitudes (the same 128 MiB)
  if (rc == QSIM_OK) {
    StateDev d2{buf, n - 1, QSIM_C128, st, 1};
    const double ms = time_ms(st, [&]() { return launch_pair_df(d2, ins, 0, 1ULL << 14, u, MC_GENERIC, nullptr); }, 8, rc);
    t.gbs_pair_df = 2.0 * 16 * (double)(1LL << (n - 1)) / (ms * 1e-3) / 1e9;
  }
  // split complex128 fused apply (CUDA cores, bound by FP32 issue), widths 2..5
  for (int k = 2; k <= 5 && rc == QSIM_OK; ++k) {
    StateDev d2{buf, n - 1, QSIM_C128, st, 1};
    std::vector<cd> eye((size_t)1 << (2 * k), 0.0);
    for (int i = 0; i < (1 << k); ++i) eye[(size_t)i * (1 << k) + i] = 1.0;
    int phys[QSIM_MAX_FUSED];
    for (int j = 0; j < k; ++j) phys[j] = 10 + 2 * j;
    std::vector<unsigned char> m;
    append_fused_df(m, eye.data(), k, phys);
    ce = cudaMemcpyAsync(mats, m.data(), m.size(), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "autotune operands");
      break;
    }
    const double ms = time_ms(st, [&]() { return launch_fused_df(d2, phys, k, 0ULL, mats, nullptr); }, 4, rc);
    t.gbs_fused_df[k] = 2.0 * 16 * (double)(1LL << (n - 1)) / (ms * 1e-3) / 1e9;
  }
  cudaStreamSynchronize(st);
  cudaFree(mats);
  cudaFree(buf);
  if (rc != QSIM_OK) return rc;
  t.valid = true;
  g_tune[dev] = t;
  return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

extern "C" qsim_status qsim_autotune(void *stream, double *out, int nout) {
  QS_TRY(autotune(static_cast<cudaStream_t>(stream)));
  const TuneTable *t = tune_table();
  if (out && t) {
    const double v[11] = {t->gbs_pair_c64, t->gbs_pair_df, t->gbs_fused[4], t->gbs_fused[5], t->gbs_remap,
                          t->launch_us, (double)t->pair_grid_mult, t->gbs_fused_df[2], t->gbs_fused_df[3],
                          t->gbs_fused_df[4], t->gbs_fused_df[5]};
    for (int i = 0; i < nout && i < 11; ++i) out[i] = v[i];
  }
  return QSIM_OK;
}
