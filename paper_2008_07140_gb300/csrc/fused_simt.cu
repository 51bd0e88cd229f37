// Fused k-qubit unitary (k <= 5) on CUDA cores for any physical qubit placement: each
// thread gathers the 2^k amplitudes of one base index, multiplies by the matrix held in
// shared memory, and scatters the result. This is the path for complex128 states and for
// placements the tensor-core kernel does not take; arithmetic is in the state precision.
#include "internal.h"

namespace qsim {

namespace {

constexpr int kThreads = 128;

struct Offs {
  unsigned long long o[32];
};

__device__ __forceinline__ unsigned long long insert_zeros_f(unsigned long long g, const Ins &ins) {
#pragma unroll 1
  for (int k = 0; k < ins.n; ++k) {
    const unsigned long long low = g & ((1ULL << ins.pos[k]) - 1ULL);
    g = ((g ^ low) << 1) | low;
  }
  return g | ins.set;
}

// For complex64 states the matrix buffer holds the hi floats (2 D^2) followed by the lo
// floats (the FP64 rounding residues), so the applied matrix is the FP64 one to ~2^-48.
template <typename R, int K>
__global__ void __launch_bounds__(kThreads)
    k_fused_simt(R *__restrict__ psi, long long items, Ins ins, Offs off, const R *__restrict__ mat) {
  constexpr int D = 1 << K;
  constexpr bool SPL = sizeof(R) == 4;
  constexpr int NM = (SPL ? 4 : 2) * D * D;
  __shared__ R sm[NM];
  for (int i = threadIdx.x; i < NM; i += blockDim.x) sm[i] = mat[i];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    const unsigned long long base = insert_zeros_f((unsigned long long)g, ins);
    R xr[D], xi[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const R *p = psi + 2 * (base + off.o[c]);
      xr[c] = p[0];
      xi[c] = p[1];
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      R yr = 0, yi = 0;
      if (SPL) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const R mr = sm[2 * D * D + 2 * (r * D + c)], mi = sm[2 * D * D + 2 * (r * D + c) + 1];
          yr += mr * xr[c] - mi * xi[c];
          yi += mr * xi[c] + mi * xr[c];
        }
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const R mr = sm[2 * (r * D + c)], mi = sm[2 * (r * D + c) + 1];
        yr = fma(mr, xr[c], fma(-mi, xi[c], yr));
        yi = fma(mr, xi[c], fma(mi, xr[c], yi));
      }
      R *p = psi + 2 * (base + off.o[r]);
      p[0] = yr;
      p[1] = yi;
    }
  }
}

template <typename R, int K>
void launch_k(const StateDev &s, long long items, const Ins &ins, const Offs &off, const void *mat) {
  long long grid = 8LL * num_sms();
  long long need = (items + kThreads - 1) / kThreads;
  if (need < grid) grid = need > 0 ? need : 1;
  k_fused_simt<R, K><<<(int)grid, kThreads, 0, s.stream>>>(static_cast<R *>(s.amps), items, ins, off,
                                                          static_cast<const R *>(mat));
}

}  // namespace

// phys[j] is the physical position of matrix-index bit (k-1-j); ctrl_mask holds physical
// control bits. dev_mat holds the 2^k x 2^k matrix, interleaved, in the state precision
// (complex64: hi floats then lo floats).
qsim_status launch_fused_simt_ctl(const StateDev &s, const int *phys, int k, unsigned long long ctrl_mask,
                                  const void *dev_mat, int64_t *bytes) {
  Ins ins;
  ins.n = 0;
  ins.set = ctrl_mask;
  unsigned long long all = ctrl_mask;
  for (int j = 0; j < k; ++j) all |= 1ULL << phys[j];
  for (int q = 0; q < s.n; ++q)
    if (all >> q & 1ULL) ins.pos[ins.n++] = q;
  Offs off;
  for (int r = 0; r < (1 << k); ++r) {
    unsigned long long o = 0;
    for (int j = 0; j < k; ++j)
      if ((r >> (k - 1 - j)) & 1) o |= 1ULL << phys[j];
    off.o[r] = o;
  }
  const long long items = 1LL << (s.n - ins.n);
  const int B = s.dtype == QSIM_C128 ? 16 : 8;
  if (bytes) *bytes += 2LL * B * (items << k);
  const bool dbl = s.dtype == QSIM_C128;
  switch (k) {
    case 1: dbl ? launch_k<double, 1>(s, items, ins, off, dev_mat) : launch_k<float, 1>(s, items, ins, off, dev_mat); break;
    case 2: dbl ? launch_k<double, 2>(s, items, ins, off, dev_mat) : launch_k<float, 2>(s, items, ins, off, dev_mat); break;
    case 3: dbl ? launch_k<double, 3>(s, items, ins, off, dev_mat) : launch_k<float, 3>(s, items, ins, off, dev_mat); break;
    case 4: dbl ? launch_k<double, 4>(s, items, ins, off, dev_mat) : launch_k<float, 4>(s, items, ins, off, dev_mat); break;
    case 5: dbl ? launch_k<double, 5>(s, items, ins, off, dev_mat) : launch_k<float, 5>(s, items, ins, off, dev_mat); break;
    default: set_error("fused width %d not in 1..5", k); return QSIM_EINVAL;
  }
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

}  // namespace qsim
