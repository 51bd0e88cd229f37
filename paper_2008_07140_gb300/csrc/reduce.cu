// Read-only sweeps with FP64 accumulation: norm, inner product, per-qubit P(bit = 1),
// PMEASURE histograms (Appendix A-1) and inverse-CDF sampling.
//
// Sums are built in a fixed order for a given state size (per-thread running sums, a
// fixed warp tree, one partial per block, then one thread adding the block partials in
// block order), so norms and inner products are reproducible run to run. Histograms add
// into shared memory with atomics; their last bits may vary between runs.
#include <cuda_runtime.h>

#include <utility>

#include "internal.h"
#include "philox.cuh"

namespace qsim {

namespace {

constexpr int kRT = 256;  // threads per reduction block

inline int red_grid() { return 2 * num_sms(); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed tree; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}

template <typename R>
__device__ __forceinline__ void load_amp(const R *p, unsigned long long i, double &re, double &im) {
  re = (double)p[2 * i];
  im = (double)p[2 * i + 1];
}

template <typename R>
__global__ void __launch_bounds__(kRT) k_norm(const R *__restrict__ psi, long long amps,
                                               double *__restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    double re, im;
    load_amp(psi, i, re, im);
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  const double b = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

template <typename R>
__global__ void __launch_bounds__(kRT) k_inner(const R *__restrict__ a, const R *__restrict__ b,
                                                long long amps, double *__restrict__ partial) {
  __shared__ double sh[32];
  double sr = 0.0, si = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    double ar, ai, br, bi;
    load_amp(a, i, ar, ai);
    load_amp(b, i, br, bi);
    sr = fma(ar, br, fma(ai, bi, sr));
    si = fma(ar, bi, fma(-ai, br, si));
  }
  const double r0 = block_sum(sr, sh);
  const double r1 = block_sum(si, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = r0;
    partial[2 * blockIdx.x + 1] = r1;
  }
}

// Per block: total and, for every physical qubit q < n, the sum of |a_i|^2 with bit q set.
// Output layout: partial[block * (n + 1) + q], q = n holds the total.
template <typename R>
__global__ void __launch_bounds__(kRT) k_p1(const R *__restrict__ psi, int n, long long amps,
                                             double *__restrict__ partial) {
  __shared__ double sh[32];
  double acc[QSIM_MAX_QUBITS + 1];
#pragma unroll
  for (int q = 0; q <= QSIM_MAX_QUBITS; ++q) acc[q] = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    double re, im;
    load_amp(psi, i, re, im);
    const double p = fma(re, re, im * im);
    acc[QSIM_MAX_QUBITS] += p;
#pragma unroll
    for (int q = 0; q < QSIM_MAX_QUBITS; ++q)
      if (q < n && ((i >> q) & 1)) acc[q] += p;
  }
  for (int q = 0; q <= QSIM_MAX_QUBITS; ++q) {
    if (q < n || q == QSIM_MAX_QUBITS) {
      const double b = block_sum(acc[q], sh);
      if (threadIdx.x == 0) partial[(long long)blockIdx.x * (n + 1) + (q < n ? q : n)] = b;
    }
  }
}

// out[c] = sum over rows b of partial[b * cols + c], rows in order (one thread per column).
__global__ void k_column_sums(const double *__restrict__ partial, int rows, int cols,
                              double *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < rows; ++b) s += partial[(long long)b * cols + c];
    out[c] = s;
  }
}

struct Bins {
  int m;
  int pos[24];
};

__device__ __forceinline__ int bin_of(unsigned long long i, const Bins &bn) {
  int s = 0;
#pragma unroll 1
  for (int t = 0; t < bn.m; ++t) s = (s << 1) | (int)((i >> bn.pos[t]) & 1ULL);
  return s;
}

// Histogram with each thread's indices ordered so that its bin changes rarely. Thread t
// (0 <= t < 2^s) takes the indices t + 2^s k: the listed bits below s come from t and stay
// fixed, those at or above s come from k. The thread runs k with the high listed bits
// outermost, so it adds 2^(n - s - mh) probabilities in registers between two shared-memory
// atomics (exactly one atomic when every listed bit is below s). Consecutive lanes read
// consecutive indices. Blocks with the same t range split the k range (gridDim.y parts), so
// that enough warps keep loads in flight. k steps over the high listed bits with one add
// and two masks ((k | M) + 1) & ~M. For complex64 the FP64 pipe (2 FMAs per SM and clock)
// would bound the sweep at two FMAs per amplitude, so each run of 8 amplitudes is summed in
// FP32 as an unevaluated pair S + E: every square re^2 = p + e exactly (TwoProduct with
// FMA), the p are added by TwoSum and every error term goes into E, which stays below
// 2^-20 S; S + E equals the exact sum of the run to about 2^-44 relative, and the runs are
// added in FP64. Complex128 stays in FP64 throughout.
struct BinOrder {
  int s;                   // index bits given by the thread number
  int ml, mh;              // listed bits below s / at or above s
  int lpos[24], lbin[24];  // below s: index bit, bin bit
  int hpos[24], hbin[24];  // at or above s: index bit minus s (ascending), bin bit
};

template <typename R>
__global__ void __launch_bounds__(kRT) k_hist_ordered(const R *__restrict__ psi, int n, BinOrder bo,
                                                       double *__restrict__ partial) {
  extern __shared__ double hist[];
  const int nb = 1 << (bo.ml + bo.mh);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0.0;
  __syncthreads();
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (1ULL << bo.s)) {
    int lowbin = 0;
    for (int j = 0; j < bo.ml; ++j)
      if ((t >> bo.lpos[j]) & 1ULL) lowbin |= 1 << bo.lbin[j];
    unsigned long long M = 0;  // high listed positions in k
    for (int j = 0; j < bo.mh; ++j) M |= 1ULL << bo.hpos[j];
    const long long inner = 1LL << (n - bo.s - bo.mh);  // indices per pattern of the high bits
    const long long per = (inner + gridDim.y - 1) / gridDim.y;
    const long long o0 = (long long)blockIdx.y * per;
    const long long o1 = o0 + per < inner ? o0 + per : inner;
    for (int h = 0; h < (1 << bo.mh); ++h) {
      int bin = lowbin;
      unsigned long long hk = 0;
      for (int j = 0; j < bo.mh; ++j)
        if ((h >> j) & 1) {
          bin |= 1 << bo.hbin[j];
          hk |= 1ULL << bo.hpos[j];
        }
      unsigned long long k = (unsigned long long)o0;  // zeros inserted at the high listed bits
      for (int j = 0; j < bo.mh; ++j) {
        const unsigned long long low = k & ((1ULL << bo.hpos[j]) - 1ULL);
        k = ((k ^ low) << 1) | low;
      }
      double acc = 0.0;
      for (long long o = o0; o < o1; o += 8) {
        const int cnt = o1 - o < 8 ? (int)(o1 - o) : 8;
        R re[8], im[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (u < cnt) {
            const unsigned long long i = t | ((k | hk) << bo.s);
            re[u] = psi[2 * i];
            im[u] = psi[2 * i + 1];
            k = ((k | M) + 1ULL) & ~M;
          } else {
            re[u] = im[u] = (R)0;
          }
        }
        if constexpr (sizeof(R) == 4) {
          float S = 0.f, E = 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            // the _rn intrinsics are never contracted into an FMA, which would break TwoSum
            const float pr = __fmul_rn(re[u], re[u]), pi = __fmul_rn(im[u], im[u]);
            const float er = fmaf(re[u], re[u], -pr), ei = fmaf(im[u], im[u], -pi);
            const float s1 = __fadd_rn(S, pr);
            float bb = __fsub_rn(s1, S);
            const float t1 = __fadd_rn(__fsub_rn(S, __fsub_rn(s1, bb)), __fsub_rn(pr, bb));
            const float s2 = __fadd_rn(s1, pi);
            bb = __fsub_rn(s2, s1);
            const float t2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bb)), __fsub_rn(pi, bb));
            S = s2;
            E += (t1 + t2) + (er + ei);
          }
          acc += (double)S + (double)E;
        } else {
          R run = (R)0;
#pragma unroll
          for (int u = 0; u < 8; ++u) run = fma(re[u], re[u], fma(im[u], im[u], run));
          acc += (double)run;
        }
      }
      atomicAdd(&hist[bin], acc);
    }
  }
  __syncthreads();
  const long long row = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) partial[row * nb + b] = hist[b];
}

// Large histograms: global atomics straight into the output.
template <typename R>
__global__ void __launch_bounds__(kRT) k_hist_global(const R *__restrict__ psi, long long amps,
                                                      Bins bn, double *__restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    double re, im;
    load_amp(psi, i, re, im);
    const double p = fma(re, re, im * im);
    if (p != 0.0) atomicAdd(&out[bin_of((unsigned long long)i, bn)], p);
  }
}

// ---- sampling ------------------------------------------------------------------------
// The state is split into chunks of 2^clog amplitudes. One warp walks a chunk in steps
// of 32 consecutive amplitudes: an inclusive warp scan of |a|^2 plus a running offset.
// The chunk-sum kernel and the search kernel use the identical sequence of operations,
// so the search always finds the step that the chunk sums promise.

__device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename R>
__global__ void k_chunk_sums(const R *__restrict__ psi, int clog, long long nchunks,
                             double *__restrict__ csum) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long steps = (1LL << clog) >> 5;
  for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    double run = 0.0;
    const unsigned long long base = (unsigned long long)c << clog;
    for (long long st = 0; st < steps; ++st) {
      double re, im;
      load_amp(psi, base + (st << 5) + lane, re, im);
      const double incl = warp_incl_scan(fma(re, re, im * im), lane);
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) csum[c] = run;
  }
}

// Exclusive prefix of the chunk sums (one block, sequential per thread then across
// threads), total in prefix[nchunks].
__global__ void k_chunk_prefix(const double *__restrict__ csum, long long nchunks,
                               double *__restrict__ prefix) {
  __shared__ double tsum[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const long long per = (nchunks + T - 1) / T;
  const long long lo = t * per, hi = lo + per < nchunks ? lo + per : nchunks;
  double s = 0.0;
  for (long long c = lo; c < hi; ++c) s += csum[c];
  tsum[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int i = 0; i < T; ++i) {
      const double v = tsum[i];
      tsum[i] = run;
      run += v;
    }
    prefix[nchunks] = run;
  }
  __syncthreads();
  double run = tsum[t];
  for (long long c = lo; c < hi; ++c) {
    prefix[c] = run;
    run += csum[c];
  }
}

template <typename R>
__global__ void k_sample(const R *__restrict__ psi, int n, int clog, long long nchunks,
                         const double *__restrict__ prefix, const double *__restrict__ csum,
                         unsigned long long shots, uint32_t k0, uint32_t k1,
                         unsigned long long *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long steps = (1LL << clog) >> 5;
  for (long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < (long long)shots; s += warps) {
    const Philox4 x = philox4x32_10((uint32_t)s, (uint32_t)((unsigned long long)s >> 32), 0u,
                                    kSampleTag, k0, k1);
    const double target = u01_from(x.v[0], x.v[1]) * prefix[nchunks];
    // largest chunk c with prefix[c] <= target
    long long lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const long long mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= target) lo = mid;
      else hi = mid - 1;
    }
    const long long c = lo;
    // walk chunk c with the same operation sequence as k_chunk_sums, on a local offset
    const double tloc = target - prefix[c];
    const unsigned long long base = (unsigned long long)c << clog;
    unsigned long long pick = base, last_nz = base;
    bool found = false;
    double run = 0.0;
    for (long long st = 0; st < steps && !found; ++st) {
      double re, im;
      load_amp(psi, base + (st << 5) + lane, re, im);
      const double p = fma(re, re, im * im);
      const double incl = warp_incl_scan(p, lane);
      const unsigned nz = __ballot_sync(0xffffffffu, p > 0.0);
      if (nz) last_nz = base + (st << 5) + (unsigned long long)(31 - __clz(nz));
      const unsigned hit = __ballot_sync(0xffffffffu, tloc < run + incl);
      if (hit) {
        pick = base + (st << 5) + (unsigned long long)(__ffs(hit) - 1);
        found = true;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    // a target within rounding of the chunk's upper end: its last non-zero amplitude
    if (!found) pick = last_nz;
    if (lane == 0) out[s] = pick;
  }
}

template <typename R>
const R *amps_of(const StateDev &s) {
  return static_cast<const R *>(s.amps);
}

}  // namespace

size_t reduce_scratch_bytes(int n) {
  const size_t blocks = (size_t)2 * num_sms();
  size_t need = (blocks + 1) * 4096 * sizeof(double);           // histograms
  const size_t p1 = blocks * (size_t)(n + 1) * sizeof(double);  // per-qubit sums
  if (p1 > need) need = p1;
  const int clog = n - 18 > 12 ? n - 18 : (n < 12 ? n : 12);
  const size_t nch = (size_t)1 << (n - clog);
  const size_t samp = (2 * nch + 2) * sizeof(double);
  if (samp > need) need = samp;
  return need + 64 * sizeof(double);
}

qsim_status red_norm(const StateDev &s, double *scratch, double *host_out) {
  const int g = red_grid();
  const long long amps = 1LL << s.n;
  double *out = scratch + g;
  if (s.dtype == QSIM_C128) k_norm<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), amps, scratch);
  else k_norm<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), amps, scratch);
  k_column_sums<<<1, 32, 0, s.stream>>>(scratch, g, 1, out);
  QS_TRY_CUDA(cudaGetLastError());
  QS_TRY_CUDA(cudaMemcpyAsync(host_out, out, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  QS_TRY_CUDA(cudaStreamSynchronize(s.stream));
  return QSIM_OK;
}

qsim_status red_inner(const StateDev &a, const void *b_amps, double *scratch, double host_out[2]) {
  const int g = red_grid();
  const long long amps = 1LL << a.n;
  double *out = scratch + 2 * g;
  if (a.dtype == QSIM_C128)
    k_inner<double><<<g, kRT, 0, a.stream>>>(amps_of<double>(a), static_cast<const double *>(b_amps), amps, scratch);
  else
    k_inner<float><<<g, kRT, 0, a.stream>>>(amps_of<float>(a), static_cast<const float *>(b_amps), amps, scratch);
  k_column_sums<<<1, 32, 0, a.stream>>>(scratch, g, 2, out);
  QS_TRY_CUDA(cudaGetLastError());
  QS_TRY_CUDA(cudaMemcpyAsync(host_out, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, a.stream));
  QS_TRY_CUDA(cudaStreamSynchronize(a.stream));
  return QSIM_OK;
}

qsim_status red_p1_all(const StateDev &s, double *scratch, double *host_total, double *host_p1) {
  const int g = red_grid();
  const long long amps = 1LL << s.n;
  const int cols = s.n + 1;
  double *out = scratch + (size_t)g * cols;
  if (s.dtype == QSIM_C128) k_p1<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), s.n, amps, scratch);
  else k_p1<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), s.n, amps, scratch);
  k_column_sums<<<1, 64, 0, s.stream>>>(scratch, g, cols, out);
  QS_TRY_CUDA(cudaGetLastError());
  double tmp[QSIM_MAX_QUBITS + 1];
  QS_TRY_CUDA(cudaMemcpyAsync(tmp, out, cols * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  QS_TRY_CUDA(cudaStreamSynchronize(s.stream));
  for (int q = 0; q < s.n; ++q) host_p1[q] = tmp[q];
  *host_total = tmp[s.n];
  return QSIM_OK;
}

qsim_status red_probs(const StateDev &s, const int *phys, int m, double *scratch, double *host_out) {
  Bins bn;
  bn.m = m;
  for (int t = 0; t < m; ++t) bn.pos[t] = phys[t];
  const long long amps = 1LL << s.n;
  const int nb = 1 << m;
  if (m <= 12) {
    // 2^s threads with s <= 16: at most 256 blocks of kRT, within the scratch's rows
    BinOrder bo;
    bo.s = s.n < 16 ? s.n : 16;
    bo.ml = bo.mh = 0;
    int hp[24], hb[24];
    for (int t = 0; t < m; ++t) {
      const int pos = phys[t], bin = m - 1 - t;  // the first listed qubit is the most significant
      if (pos < bo.s) {
        bo.lpos[bo.ml] = pos;
        bo.lbin[bo.ml++] = bin;
      } else {
        hp[bo.mh] = pos - bo.s;
        hb[bo.mh++] = bin;
      }
    }
    for (int a = 0; a < bo.mh; ++a)  // ascending high positions (for the zero insertion)
      for (int b = a + 1; b < bo.mh; ++b)
        if (hp[b] < hp[a]) {
          std::swap(hp[a], hp[b]);
          std::swap(hb[a], hb[b]);
        }
    for (int j = 0; j < bo.mh; ++j) {
      bo.hpos[j] = hp[j];
      bo.hbin[j] = hb[j];
    }
    const long long threads = 1LL << bo.s;
    const int block = threads < kRT ? (int)threads : kRT;
    const int g = (int)((threads + block - 1) / block);
    // split the k range over gridDim.y: about 8 blocks per SM, within the scratch's rows
    // (one partial histogram per block) and at most one part per 64 indices of k
    const long long inner = 1LL << (s.n - bo.s - bo.mh);
    const long long rows_cap = (long long)(2 * num_sms() + 1) * 4096 / nb - 1;  // + the output row
    long long y = (8LL * num_sms() + g - 1) / g;
    if (y > rows_cap / g) y = rows_cap / g;
    if (y > inner / 64) y = inner / 64;
    if (y < 1) y = 1;
    const int rows = g * (int)y;
    double *out = scratch + (size_t)rows * nb;
    const size_t sh = (size_t)nb * sizeof(double);
    const dim3 grid((unsigned)g, (unsigned)y);
    if (s.dtype == QSIM_C128)
      k_hist_ordered<double><<<grid, block, sh, s.stream>>>(amps_of<double>(s), s.n, bo, scratch);
    else
      k_hist_ordered<float><<<grid, block, sh, s.stream>>>(amps_of<float>(s), s.n, bo, scratch);
    k_column_sums<<<(nb + 255) / 256, 256, 0, s.stream>>>(scratch, rows, nb, out);
    QS_TRY_CUDA(cudaGetLastError());
    QS_TRY_CUDA(cudaMemcpyAsync(host_out, out, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    QS_TRY_CUDA(cudaStreamSynchronize(s.stream));
    return QSIM_OK;
  }
  double *dout = nullptr;
  QS_TRY_CUDA(cudaMallocAsync((void **)&dout, (size_t)nb * sizeof(double), s.stream));
  cudaError_t e = cudaMemsetAsync(dout, 0, (size_t)nb * sizeof(double), s.stream);
  if (e == cudaSuccess) {
    if (s.dtype == QSIM_C128)
      k_hist_global<double><<<red_grid(), kRT, 0, s.stream>>>(amps_of<double>(s), amps, bn, dout);
    else
      k_hist_global<float><<<red_grid(), kRT, 0, s.stream>>>(amps_of<float>(s), amps, bn, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, dout, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s.stream);
  cudaFreeAsync(dout, s.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
  if (e != cudaSuccess) return cuda_fail(e, "probabilities (large histogram)");
  return QSIM_OK;
}

qsim_status red_sample_seeded(const StateDev &s, uint64_t seed, uint64_t shots, double *scratch,
                              uint64_t *host_idx) {
  const int clog = s.n - 18 > 12 ? s.n - 18 : (s.n < 12 ? s.n : 12);
  if (clog < 5) {
    set_error("sampling needs at least 5 qubits on the device path");
    return QSIM_EUNSUPPORTED;
  }
  const long long nch = 1LL << (s.n - clog);
  double *csum = scratch;
  double *prefix = scratch + nch;
  unsigned long long *dout = nullptr;
  QS_TRY_CUDA(cudaMallocAsync((void **)&dout, (size_t)shots * sizeof(uint64_t), s.stream));
  const int g = red_grid();
  if (s.dtype == QSIM_C128) k_chunk_sums<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), clog, nch, csum);
  else k_chunk_sums<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), clog, nch, csum);
  k_chunk_prefix<<<1, 1024, 0, s.stream>>>(csum, nch, prefix);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const long long sg = ((long long)shots * 32 + kRT - 1) / kRT;
  const int sgrid = (int)(sg < g ? (sg > 0 ? sg : 1) : g);
  if (s.dtype == QSIM_C128)
    k_sample<double><<<sgrid, kRT, 0, s.stream>>>(amps_of<double>(s), s.n, clog, nch, prefix, csum, shots, k0, k1, dout);
  else
    k_sample<float><<<sgrid, kRT, 0, s.stream>>>(amps_of<float>(s), s.n, clog, nch, prefix, csum, shots, k0, k1, dout);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_idx, dout, (size_t)shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s.stream);
  cudaFreeAsync(dout, s.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
  if (e != cudaSuccess) return cuda_fail(e, "sample");
  return QSIM_OK;
}

}  // namespace qsim
