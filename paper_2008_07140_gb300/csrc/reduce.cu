// Read-only sweeps with FP64 accumulation: norm, inner product, per-qubit P(bit = 1),
// PMEASURE histograms (Appendix A-1) and inverse-CDF sampling.
//
// Sums are built in a fixed order for a given state size (per-thread running sums, a
// fixed warp tree, one partial per block, then one warp per column adding the block
// partials in a fixed order), so norms, inner products and per-qubit sums are reproducible
// run to run. Histograms add per-bin sums into the output with FP64 atomics; their last
// bits may vary between runs.
#include <cuda_runtime.h>

#include "fpair.cuh"
#include "internal.h"
#include "philox.cuh"

namespace qsim {

namespace {

constexpr int kRT = 256;  // threads per reduction block

inline int red_grid() { return 2 * num_sms(); }
inline int stream_grid() { return 8 * num_sms(); }  // norm and inner product: more loads in flight

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
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    const float2 *p2 = reinterpret_cast<const float2 *>(psi);
    for (long long i0 = tid; i0 < amps; i0 += 8 * stride) {
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long i = i0 + u * stride;
        v[u] = i < amps ? p2[i] : make_float2(0.f, 0.f);
      }
      FPair r{0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        fpair_add_prod(r, v[u].x, v[u].x);
        fpair_add_prod(r, v[u].y, v[u].y);
      }
      acc += fpair_value(r);
    }
  } else {
    for (long long i = tid; i < amps; i += stride) {
      double re, im;
      load_amp(psi, i, re, im);
      acc = fma(re, re, acc);
      acc = fma(im, im, acc);
    }
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
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    // <a|b> = sum conj(a) b: re = ar br + ai bi, im = ar bi - ai br. A warp takes 256
    // consecutive amplitudes of each state per step in 16-byte loads (2 KiB runs: two read
    // streams at the same offsets keep their DRAM pages busy for longer than short pieces)
    const float4 *a4 = reinterpret_cast<const float4 *>(a), *b4 = reinterpret_cast<const float4 *>(b);
    const int lane = threadIdx.x & 31;
    const long long pairs = amps >> 1;           // amps >= 2: n >= 1
    const long long wstride = stride >> 5 << 7;  // amplitude pairs per step of all warps
    for (long long i0 = (tid >> 5 << 7) + lane; i0 < pairs; i0 += wstride) {
      float4 va[4], vb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long i = i0 + u * 32;
        va[u] = i < pairs ? a4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        vb[u] = i < pairs ? b4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      FPair r{0.f, 0.f}, m{0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        fpair_add_prod(r, va[u].x, vb[u].x);
        fpair_add_prod(r, va[u].y, vb[u].y);
        fpair_add_prod(m, va[u].x, vb[u].y);
        fpair_add_prod(m, -va[u].y, vb[u].x);
        fpair_add_prod(r, va[u].z, vb[u].z);
        fpair_add_prod(r, va[u].w, vb[u].w);
        fpair_add_prod(m, va[u].z, vb[u].w);
        fpair_add_prod(m, -va[u].w, vb[u].z);
      }
      sr += fpair_value(r);
      si += fpair_value(m);
    }
  } else {
    for (long long i = tid; i < amps; i += stride) {
      double ar, ai, br, bi;
      load_amp(a, i, ar, ai);
      load_amp(b, i, br, bi);
      sr = fma(ar, br, fma(ai, bi, sr));
      si = fma(ar, bi, fma(-ai, br, si));
    }
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

// Per-qubit sums for states of at least 12 qubits. A warp owns K = 2^lk consecutive
// segments of 4096 amplitudes (K = segments / warps, both powers of two); lane l reads index
// 4096 sg + 32 m + l for m = 0..127, so index bits 0..4 are the lane's, bits 5..11 are m's,
// bits 12..11+lk the segment's within the warp's range, and the bits above are the warp's.
// Per run of 8 values of m a lane forms the run total and the sums over m's bits 0..2
// (selected at compile time), per segment the sums over m's bits 3..6 from the run totals,
// and adds a segment's sums into FP64 accumulators; a bit that is fixed for the lane (lane
// bits, the warp's bits) takes the lane's total at the end. So an amplitude costs about
// two and a half additions instead of one per set bit. Complex64 sums in exact FP32 pairs;
// complex128 in FP64. Output layout as k_p1.
constexpr int kP1MaxLk = 12;  // with 2^14 warps: states of up to 38 qubits

__device__ __forceinline__ FPair square_pair(float2 v) {
  const float pr = __fmul_rn(v.x, v.x), pi = __fmul_rn(v.y, v.y);
  FPair p{pr, fmaf(v.x, v.x, -pr)};
  fpair_add(p, pi);
  p.e = __fadd_rn(p.e, fmaf(v.y, v.y, -pi));
  return p;
}

// Running sums of squares: FP32 pairs for complex64, doubles for complex128.
template <typename R>
struct SqSum;
template <>
struct SqSum<float> {
  FPair v{0.f, 0.f};
  using Amp = float2;
  __device__ __forceinline__ static SqSum square(float2 a) {
    SqSum r;
    r.v = square_pair(a);
    return r;
  }
  __device__ __forceinline__ void add(const SqSum &o) { fpair_add(v, o.v); }
  __device__ __forceinline__ double value() const { return fpair_value(v); }
};
template <>
struct SqSum<double> {
  double v = 0.0;
  using Amp = double2;
  __device__ __forceinline__ static SqSum square(double2 a) {
    SqSum r;
    r.v = fma(a.x, a.x, a.y * a.y);
    return r;
  }
  __device__ __forceinline__ void add(const SqSum &o) { v += o.v; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename R>
__global__ void __launch_bounds__(kRT, 3) k_p1_segments(const R *__restrict__ psi, int n, int lk,
                                                     long long warps_used, double *__restrict__ partial) {
  using S = SqSum<R>;
  using A = typename S::Amp;
  __shared__ double sh[32];
  __shared__ double bj[kP1MaxLk][kRT];  // sums over the segment-number bits, per thread
  const A *p2 = reinterpret_cast<const A *>(psi);
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double tot = 0.0, bm[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) bm[j] = 0.0;
  for (int j = 0; j < lk; ++j) bj[j][threadIdx.x] = 0.0;
  if (w < warps_used) {
    const long long K = 1LL << lk;
    for (long long j = 0; j < K; ++j) {
      const long long base = ((w << lk) + j) << 12;
      // runs of CW values of m (16 loads in flight per lane for complex64, 8 for complex128)
      constexpr int CW = sizeof(R) == 4 ? 16 : 8, LU = sizeof(R) == 4 ? 4 : 3;
      S T, B[7];
      for (int c = 0; c < 128 / CW; ++c) {
        A v[CW];
#pragma unroll
        for (int u = 0; u < CW; ++u) v[u] = p2[base + (long long)((c * CW + u) << 5) + lane];
        S ct, cb[LU];
#pragma unroll
        for (int u = 0; u < CW; ++u) {
          const S p = S::square(v[u]);
          ct.add(p);
#pragma unroll
          for (int b = 0; b < LU; ++b)
            if ((u >> b) & 1) cb[b].add(p);
        }
        T.add(ct);
#pragma unroll
        for (int b = 0; b < LU; ++b) B[b].add(cb[b]);
#pragma unroll
        for (int b = 0; b < 7 - LU; ++b)
          if ((c >> b) & 1) B[LU + b].add(ct);
      }
      const double td = T.value();
      tot += td;
#pragma unroll
      for (int b = 0; b < 7; ++b) bm[b] += B[b].value();
      for (int b = 0; b < lk; ++b)
        if ((j >> b) & 1) bj[b][threadIdx.x] += td;
    }
  }
  // qubit q's value for this thread, then a block sum per qubit (q = n: the total)
  for (int q = 0; q <= n; ++q) {
    double v = 0.0;  // selected with static indices, so bm stays in registers
    if (q == n) v = tot;
    else if (q < 5) v = ((lane >> q) & 1) ? tot : 0.0;
    else if (q >= 12 + lk) v = ((w >> (q - 12 - lk)) & 1) ? tot : 0.0;
#pragma unroll
    for (int b = 0; b < 7; ++b)
      if (q == 5 + b) v = bm[b];
    if (q >= 12 && q < 12 + lk) v = bj[q - 12][threadIdx.x];
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * (n + 1) + q] = b;
  }
}

// out[c] = sum over rows b of partial[b * cols + c]: one warp per column, lane l adding rows
// l, l + 32, ... in order, then a fixed shuffle tree (the same order every run).
__global__ void k_column_sums(const double *__restrict__ partial, int rows, int cols,
                              double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < cols; c += warps) {
    double s = 0.0;
    for (int b = lane; b < rows; b += 32) s += partial[(long long)b * cols + c];
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
}

// PMEASURE histogram with one bin per thread. The thread number t is spread over a set P of
// index bits: the five lowest (so that a warp reads 32 consecutive amplitudes), every
// listed bit, then the lowest other bits until 2^|P| threads keep the GPU busy; the
// thread walks the other bits Q (k -> ((k | ~Q) + 1) & Q steps to the next index with only
// Q bits set). Its bin is therefore fixed: it sums 2^(n - |P|) probabilities, the lanes of
// a warp that share a bin (those differing only in unlisted lane bits) add theirs by
// shuffles, and one lane per bin adds the sum to the output with an FP64 atomic. For
// complex64 each run of 8 squares is summed in FP32 as an exact pair (TwoProduct by FMA,
// TwoSum; about 2^-44 relative) with one FP64 addition per run: at 2 FP64 FMAs per SM and
// clock, FP64 arithmetic per amplitude would bound the sweep below HBM speed. Complex128
// stays in FP64. The atomics make the last bits of a bin depend on the order the warps
// finish in.
struct HistMap {
  int np;              // thread bits
  int ppos[QSIM_MAX_QUBITS];  // their index positions
  unsigned long long qmask;   // the walked positions
  int m;
  int lpos[24];        // listed positions; listed bit j is bin bit m - 1 - j
  unsigned lane_free;  // lane bits (index bits 0..4) that are not listed
};

template <typename R>
__global__ void __launch_bounds__(kRT) k_hist_threads(const R *__restrict__ psi, HistMap hm, long long iters,
                                                      double *__restrict__ out) {
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < (1ULL << hm.np);
  unsigned long long base = 0;
  for (int j = 0; j < hm.np; ++j)
    if ((t >> j) & 1ULL) base |= 1ULL << hm.ppos[j];
  int bin = 0;
  for (int j = 0; j < hm.m; ++j) bin |= (int)((base >> hm.lpos[j]) & 1ULL) << (hm.m - 1 - j);
  const unsigned long long Q = hm.qmask;
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
    if ((hm.lane_free >> b) & 1u) acc += __shfl_xor_sync(0xffffffffu, acc, 1 << b);
  if (active && (lane & hm.lane_free) == 0) atomicAdd(&out[bin], acc);
}

// ---- sampling ------------------------------------------------------------------------
// The state is split into chunks of 2^clog amplitudes. The chunk sums take the amplitudes
// in steps of 32 consecutive ones per warp, each lane summing its values (complex64 in
// exact FP32 pairs per run of 8, complex128 in FP64) and the warp adding the lanes at the
// end. The search for one shot walks its chunk in the same steps with an inclusive warp
// scan of |a|^2 plus a running offset (FP64). The two sums of a chunk agree to about
// 2^-44 relative; a target that lands in that sliver above the walk's total takes the
// chunk's last non-zero amplitude.

__device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename R>
__global__ void __launch_bounds__(kRT) k_chunk_sums(const R *__restrict__ psi, int clog, long long nchunks,
                                                    double *__restrict__ csum) {
  const int lane = threadIdx.x & 31;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long steps = (1LL << clog) >> 5;  // a multiple of 8 (clog >= 8)
  for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    double run = 0.0;
    const unsigned long long base = (unsigned long long)c << clog;
    for (long long st = 0; st < steps; st += 8) {
      R re[8], im[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const unsigned long long i = base + ((st + u) << 5) + lane;
        re[u] = psi[2 * i];
        im[u] = psi[2 * i + 1];
      }
      if constexpr (sizeof(R) == 4) {
        FPair r{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          fpair_add_prod(r, re[u], re[u]);
          fpair_add_prod(r, im[u], im[u]);
        }
        run += fpair_value(r);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) run = fma(re[u], re[u], fma(im[u], im[u], run));
      }
    }
    run = warp_sum(run);
    if (lane == 0) csum[c] = run;
  }
}

// Chunk sums for chunks of fewer than 256 amplitudes (states below 8 qubits): the walk's
// own operation sequence.
template <typename R>
__global__ void k_chunk_sums_scan(const R *__restrict__ psi, int clog, long long nchunks,
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

// Exclusive prefix of the chunk sums (one block of 1024 threads): each thread adds its
// contiguous range in order (loads eight at a time), the block scans the thread totals with
// a fixed shuffle tree, and each thread writes its range's prefixes. Total in
// prefix[nchunks].
__global__ void k_chunk_prefix(const double *__restrict__ csum, long long nchunks,
                               double *__restrict__ prefix) {
  __shared__ double wsum[32];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, wid = t >> 5;
  const long long per = (nchunks + T - 1) / T;
  const long long lo = t * per, hi = lo + per < nchunks ? lo + per : nchunks;
  double s = 0.0;
  for (long long c = lo; c < hi; c += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = c + u < hi ? csum[c + u] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  // inclusive scan of the thread totals: within the warp, then over the warp totals
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    double w = lane < (T >> 5) ? wsum[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double x = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += x;
    }
    wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  double excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0.0;
  double run = (wid > 0 ? wsum[wid - 1] : 0.0) + excl;  // exclusive start of this thread
  for (long long c = lo; c < hi; c += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = c + u < hi ? csum[c + u] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (c + u < hi) {
        prefix[c + u] = run;
        run += v[u];
      }
  }
  if (lo < nchunks && hi == nchunks) prefix[nchunks] = run;  // the owner of the last chunk
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
  const int g = stream_grid();
  const long long amps = 1LL << s.n;
  double *out = scratch + g;
  if (s.dtype == QSIM_C128) k_norm<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), amps, scratch);
  else k_norm<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), amps, scratch);
  k_column_sums<<<1, 32, 0, s.stream>>>(scratch, g, 1, out);  // one warp per column
  QS_TRY_CUDA(cudaGetLastError());
  QS_TRY_CUDA(cudaMemcpyAsync(host_out, out, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  QS_TRY_CUDA(cudaStreamSynchronize(s.stream));
  return QSIM_OK;
}

qsim_status red_inner(const StateDev &a, const void *b_amps, double *scratch, double host_out[2]) {
  const int g = stream_grid();
  const long long amps = 1LL << a.n;
  double *out = scratch + 2 * g;
  if (a.dtype == QSIM_C128)
    k_inner<double><<<g, kRT, 0, a.stream>>>(amps_of<double>(a), static_cast<const double *>(b_amps), amps, scratch);
  else
    k_inner<float><<<g, kRT, 0, a.stream>>>(amps_of<float>(a), static_cast<const float *>(b_amps), amps, scratch);
  k_column_sums<<<1, 64, 0, a.stream>>>(scratch, g, 2, out);
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
  int rows = g;
  if (s.n >= 12 && s.n - 12 - 14 <= kP1MaxLk) {
    // 2^lw warps (at most 2^14 = 2048 blocks of 8 warps, three resident per SM, so that the
    // last wave is short; rows x (n + 1) partial sums fit the scratch) over the 2^(n - 12)
    // segments, 2^lk consecutive segments each
    const int ls = s.n - 12;
    const int lw = ls < 14 ? ls : 14;
    const int lk = ls - lw;
    const long long warps = 1LL << lw;
    rows = (int)((warps * 32 + kRT - 1) / kRT);
    double *out2 = scratch + (size_t)rows * cols;
    if (s.dtype == QSIM_C128)
      k_p1_segments<double><<<rows, kRT, 0, s.stream>>>(amps_of<double>(s), s.n, lk, warps, scratch);
    else
      k_p1_segments<float><<<rows, kRT, 0, s.stream>>>(amps_of<float>(s), s.n, lk, warps, scratch);
    out = out2;
  } else if (s.dtype == QSIM_C128) {
    k_p1<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), s.n, amps, scratch);
  } else {
    k_p1<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), s.n, amps, scratch);
  }
  k_column_sums<<<(cols + 7) / 8, 256, 0, s.stream>>>(scratch, rows, cols, out);
  QS_TRY_CUDA(cudaGetLastError());
  double tmp[QSIM_MAX_QUBITS + 1];
  QS_TRY_CUDA(cudaMemcpyAsync(tmp, out, cols * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  QS_TRY_CUDA(cudaStreamSynchronize(s.stream));
  for (int q = 0; q < s.n; ++q) host_p1[q] = tmp[q];
  *host_total = tmp[s.n];
  return QSIM_OK;
}

qsim_status red_probs(const StateDev &s, const int *phys, int m, double *scratch, double *host_out) {
  if (m < 1 || m > 24) {
    set_error("probabilities: %d listed qubits (1..24)", m);
    return QSIM_EINVAL;
  }
  const size_t nb = (size_t)1 << m;
  HistMap hm{};
  hm.m = m;
  unsigned long long pmask = 0;
  for (int b = 0; b < 5 && b < s.n; ++b) pmask |= 1ULL << b;
  for (int t = 0; t < m; ++t) {
    hm.lpos[t] = phys[t];
    pmask |= 1ULL << phys[t];
  }
  const int target = s.n < 18 ? s.n : 18;  // 2^18 threads: about seven blocks per SM
  for (int b = 5; b < s.n && __builtin_popcountll(pmask) < target; ++b) pmask |= 1ULL << b;
  hm.np = 0;
  for (int b = 0; b < s.n; ++b)
    if (pmask >> b & 1ULL) hm.ppos[hm.np++] = b;
  hm.qmask = ((s.n >= 64 ? 0ULL : (1ULL << s.n)) - 1ULL) & ~pmask;
  hm.lane_free = 0;
  for (int b = 0; b < 5; ++b) {
    bool listed = false;
    for (int t = 0; t < m; ++t) listed = listed || phys[t] == b;
    if (!listed) hm.lane_free |= 1u << b;
  }
  const long long iters = 1LL << (s.n - hm.np);
  const long long threads = 1LL << hm.np;  // at most 2^29 (5 lane bits + 24 listed)
  const long long g = (threads + kRT - 1) / kRT;
  // the output in the scratch when it fits (up to 2^20 bins), else in a buffer of its own
  const bool own = nb * sizeof(double) > reduce_scratch_bytes(s.n);
  double *out = scratch;
  if (own) QS_TRY_CUDA(cudaMallocAsync((void **)&out, nb * sizeof(double), s.stream));
  cudaError_t e = cudaMemsetAsync(out, 0, nb * sizeof(double), s.stream);
  if (e == cudaSuccess) {
    if (s.dtype == QSIM_C128)
      k_hist_threads<double><<<(unsigned)g, kRT, 0, s.stream>>>(amps_of<double>(s), hm, iters, out);
    else
      k_hist_threads<float><<<(unsigned)g, kRT, 0, s.stream>>>(amps_of<float>(s), hm, iters, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out, nb * sizeof(double), cudaMemcpyDeviceToHost, s.stream);
  if (own) cudaFreeAsync(out, s.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
  if (e != cudaSuccess) return cuda_fail(e, "probabilities");
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
  // chunk sums with steps of 8 x 32 amplitudes need clog >= 8; smaller states keep the scan
  if (clog >= 8) {
    const int cg = stream_grid();
    if (s.dtype == QSIM_C128) k_chunk_sums<double><<<cg, kRT, 0, s.stream>>>(amps_of<double>(s), clog, nch, csum);
    else k_chunk_sums<float><<<cg, kRT, 0, s.stream>>>(amps_of<float>(s), clog, nch, csum);
  } else if (s.dtype == QSIM_C128) {
    k_chunk_sums_scan<double><<<g, kRT, 0, s.stream>>>(amps_of<double>(s), clog, nch, csum);
  } else {
    k_chunk_sums_scan<float><<<g, kRT, 0, s.stream>>>(amps_of<float>(s), clog, nch, csum);
  }
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
