// Allocation-free variant of the PMEASURE histogram (qsim_probabilities_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a read-out: code
// that must not synchronise the device (cudaFree does) and programs that run on a fixed,
// pre-planned memory budget. For them this entry point takes
// the amplitudes and the output buffer from the caller and keeps its scratch (one partial
// histogram per block) in a file-scope device array of fixed size, allocated once when the
// library is loaded and held by every GPU that loads it until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's contents. Every
// call writes each scratch entry before it reads it, so nothing has to start at zero.
// Calls whose kernels overlap on the GPU (two streams, or two threads) race on the array;
// order them on one stream or serialise them.
#include <mutex>

#include "internal.h"

namespace qsim {

namespace {

constexpr int kNaBlocks = 256;     // partial histograms (blocks of the histogram kernel)
constexpr int kNaMaxQubits = 10;   // at most 2^10 outcomes per call
constexpr int kNaThreads = 256;

// 256 blocks x 1024 bins x 8 bytes = 2 MiB per device.
static __device__ __align__(256) double g_na_scratch[kNaBlocks * (1 << kNaMaxQubits)];

struct NaBins {
  int m;
  int pos[kNaMaxQubits];
};

template <typename R>
__global__ void __launch_bounds__(kNaThreads)
    k_na_hist(const R *__restrict__ psi, long long amps, NaBins bn, double *__restrict__ partial) {
  __shared__ double hist[1 << kNaMaxQubits];
  const int nb = 1 << bn.m;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    const double re = (double)psi[2 * i], im = (double)psi[2 * i + 1];
    int s = 0;
#pragma unroll 1
    for (int t = 0; t < bn.m; ++t) s = (s << 1) | (int)(((unsigned long long)i >> bn.pos[t]) & 1ULL);
    atomicAdd(&hist[s], fma(re, re, im * im));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) partial[(long long)blockIdx.x * nb + b] = hist[b];
}

// out[c] = sum over the partial rows, in row order
__global__ void k_na_sum(const double *__restrict__ partial, int rows, int cols, double *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < rows; ++b) s += partial[(long long)b * cols + c];
    out[c] = s;
  }
}

// Device address of the scratch array, looked up once per device with that device
// current (a host-side name of a __device__ array is not a device address). The same
// first call also loads the three kernels on that device (cudaFuncGetAttributes), so that
// no later call needs to load code; with lazy module loading a first launch would
// otherwise load it then, and loading may allocate device memory.
std::mutex g_na_mu;
double *g_na_ptr[64] = {};

qsim_status na_scratch(double **out) {
  int dev = 0;
  QS_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device %d out of range for the static scratch table", dev);
    return QSIM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_na_mu);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_hist<float>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_hist<double>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_sum);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes(allocation-free kernels)");
    g_na_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_na_ptr[dev];
  return QSIM_OK;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" qsim_status qsim_probabilities_noalloc(const void *amps, int n, int dtype, const int *qubits,
                                                  int m, double *out, void *stream) {
  if (!amps || !out || !qubits) {
    set_error("probabilities_noalloc: amps, qubits and out must be non-NULL");
    return QSIM_EINVAL;
  }
  if (n < 1 || n > QSIM_MAX_QUBITS || (dtype != QSIM_C64 && dtype != QSIM_C128)) {
    set_error("probabilities_noalloc: bad n (%d) or dtype (%d)", n, dtype);
    return QSIM_EINVAL;
  }
  if (m < 1 || m > kNaMaxQubits || m > n) {
    set_error("probabilities_noalloc: %d listed qubits; the static scratch holds at most %d",
              m, kNaMaxQubits);
    return QSIM_EINVAL;
  }
  NaBins bn;
  bn.m = m;
  unsigned long long seen = 0;
  for (int t = 0; t < m; ++t) {
    const int q = qubits[t];
    if (q < 0 || q >= n || (seen >> q & 1ULL)) {
      set_error("probabilities_noalloc: qubit %d out of range or repeated", q);
      return QSIM_EINVAL;
    }
    seen |= 1ULL << q;
    bn.pos[t] = q;
  }
  double *scratch = nullptr;
  QS_TRY(na_scratch(&scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long total = 1LL << n;
  long long grid = (total + kNaThreads - 1) / kNaThreads;
  if (grid > kNaBlocks) grid = kNaBlocks;
  const int nb = 1 << m;
  if (dtype == QSIM_C128)
    k_na_hist<double><<<(int)grid, kNaThreads, 0, st>>>(static_cast<const double *>(amps), total, bn, scratch);
  else
    k_na_hist<float><<<(int)grid, kNaThreads, 0, st>>>(static_cast<const float *>(amps), total, bn, scratch);
  k_na_sum<<<(nb + 255) / 256, 256, 0, st>>>(scratch, (int)grid, nb, out);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}
