// Exact FP32 pair sums for complex64 read-outs (device helpers shared by the read-out
// kernels).
//
// Sums on the FP32 pipe (GB300 issues 2 FP64 FMAs per SM and clock, so FP64
// arithmetic per amplitude would bound these sweeps well below HBM speed): a value is kept
// as an unevaluated pair s + e. Products enter exactly (TwoProduct with FMA), leading parts
// are added by TwoSum and every error term goes into e; over a run of up to a few hundred
// terms s + e holds the exact sum to about 2^-40 relative, and the runs are added in FP64.
// The _rn intrinsics are never contracted into an FMA, which would break TwoSum.
#pragma once

#include <cuda_runtime.h>

namespace qsim {
namespace {

struct FPair {
  float s, e;
};

__device__ __forceinline__ void fpair_add(FPair &a, float p) {
  const float s = __fadd_rn(a.s, p);
  const float bb = __fsub_rn(s, a.s);
  a.e = __fadd_rn(a.e, __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb)));
  a.s = s;
}

__device__ __forceinline__ void fpair_add(FPair &a, const FPair &b) {
  fpair_add(a, b.s);
  a.e = __fadd_rn(a.e, b.e);
}

// a += x y exactly (up to the final rounding of e)
__device__ __forceinline__ void fpair_add_prod(FPair &a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float err = fmaf(x, y, -p);
  fpair_add(a, p);
  a.e = __fadd_rn(a.e, err);
}

__device__ __forceinline__ double fpair_value(const FPair &a) { return (double)a.s + (double)a.e; }

}  // namespace
}  // namespace qsim
