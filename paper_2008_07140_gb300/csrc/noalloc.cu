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

#include "fpair.cuh"
#include "internal.h"

namespace qsim {

namespace {

constexpr int kNaBlocks = 256;     // partial histograms (blocks of the histogram kernel)
constexpr int kNaMaxQubits = 10;   // at most 2^10 outcomes per call
constexpr int kNaThreads = 256;

// 256 blocks x 1024 bins x 8 bytes = 2 MiB per device.
static __device__ __align__(256) double g_na_scratch[kNaBlocks * (1 << kNaMaxQubits)];

// One bin per thread, as in the regular histogram: the thread number is spread over the
// five lowest index bits (a warp reads 32 consecutive amplitudes), every listed bit and
// further low bits up to 2^16 threads (at most kNaBlocks blocks); the thread walks the
// other bits, the lanes that share a bin add by shuffles, one lane per bin adds into the
// block's shared histogram, and the block writes its row of the scratch. Complex64 squares
// are summed in exact FP32 pairs per run of 8 (fpair.cuh), complex128 in FP64.
struct NaMap {
  int m;
  int lpos[kNaMaxQubits];  // listed positions; listed bit j is bin bit m - 1 - j
  int np;                  // thread bits
  int ppos[QSIM_MAX_QUBITS];
  unsigned long long qmask;  // the walked positions
  unsigned lane_free;        // lane bits (index bits 0..4) that are not listed
};

template <typename R>
__global__ void __launch_bounds__(kNaThreads)
    k_na_hist(const R *__restrict__ psi, NaMap mp, long long iters, double *__restrict__ partial) {
  __shared__ double hist[1 << kNaMaxQubits];
  const int nb = 1 << mp.m;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < (1ULL << mp.np);
  unsigned long long base = 0;
  for (int j = 0; j < mp.np; ++j)
    if ((t >> j) & 1ULL) base |= 1ULL << mp.ppos[j];
  int bin = 0;
  for (int j = 0; j < mp.m; ++j) bin |= (int)((base >> mp.lpos[j]) & 1ULL) << (mp.m - 1 - j);
  const unsigned long long Q = mp.qmask;
  double acc = 0.0;
  if (active) {
    unsigned long long k = 0;
    for (long long o = 0; o < iters; o += 8) {
      const int cnt = iters - o < 8 ? (int)(iters - o) : 8;
      R re[8], im[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (u < cnt) {
          const unsigned long long i = base | k;
          re[u] = psi[2 * i];
          im[u] = psi[2 * i + 1];
          k = ((k | ~Q) + 1ULL) & Q;
        } else {
          re[u] = im[u] = (R)0;
        }
      }
      if constexpr (sizeof(R) == 4) {
        FPair r{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          fpair_add_prod(r, re[u], re[u]);
          fpair_add_prod(r, im[u], im[u]);
        }
        acc += fpair_value(r);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(re[u], re[u], fma(im[u], im[u], acc));
      }
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < 5; ++b)
    if ((mp.lane_free >> b) & 1u) acc += __shfl_xor_sync(0xffffffffu, acc, 1 << b);
  if (active && (lane & mp.lane_free) == 0) atomicAdd(&hist[bin], acc);
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
  NaMap mp{};
  mp.m = m;
  unsigned long long seen = 0;
  for (int t = 0; t < m; ++t) {
    const int q = qubits[t];
    if (q < 0 || q >= n || (seen >> q & 1ULL)) {
      set_error("probabilities_noalloc: qubit %d out of range or repeated", q);
      return QSIM_EINVAL;
    }
    seen |= 1ULL << q;
    mp.lpos[t] = q;
  }
  unsigned long long pmask = seen;
  for (int b = 0; b < 5 && b < n; ++b) pmask |= 1ULL << b;
  const int target = n < 16 ? n : 16;  // 2^16 threads = kNaBlocks blocks of kNaThreads
  for (int b = 5; b < n && __builtin_popcountll(pmask) < target; ++b) pmask |= 1ULL << b;
  mp.np = 0;
  for (int b = 0; b < n; ++b)
    if (pmask >> b & 1ULL) mp.ppos[mp.np++] = b;
  mp.qmask = ((n >= 64 ? 0ULL : (1ULL << n)) - 1ULL) & ~pmask;
  mp.lane_free = 0;
  for (int b = 0; b < 5; ++b)
    if (!(seen >> b & 1ULL)) mp.lane_free |= 1u << b;
  double *scratch = nullptr;
  QS_TRY(na_scratch(&scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long iters = 1LL << (n - mp.np);
  const long long grid = ((1LL << mp.np) + kNaThreads - 1) / kNaThreads;  // <= kNaBlocks (np <= 16)
  const int nb = 1 << m;
  if (dtype == QSIM_C128)
    k_na_hist<double><<<(int)grid, kNaThreads, 0, st>>>(static_cast<const double *>(amps), mp, iters, scratch);
  else
    k_na_hist<float><<<(int)grid, kNaThreads, 0, st>>>(static_cast<const float *>(amps), mp, iters, scratch);
  k_na_sum<<<(nb + 255) / 256, 256, 0, st>>>(scratch, (int)grid, nb, out);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}
