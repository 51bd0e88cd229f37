// FP64-accurate sweeps for complex128 states on the FP32 pipe ("split" format).
//
// GB300 issues 2 FP64 FMAs per SM per clock against 124 FP32 FMAs, so a complex128 2x2
// update (8 FP64 FMAs per amplitude) cannot keep up with HBM. Between calls a complex128
// state is therefore held as pairs of floats: each 16-byte amplitude is
// (re_hi, im_hi, re_lo, im_lo) with re = re_hi + re_lo exactly (a 48-bit significand), and
// the gate arithmetic uses error-free transformations in FP32:
//   TwoSum (Knuth):        s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a
//   Fast2Sum (Dekker):     s = a + b, e = b - (s - a)            for |a| >= |b|
//   TwoProduct with FMA:   p = a b,   e = fma(a, b, -p)
// Matrix entries are split into three floats, m = m_hi + m_lo + m_3 exactly for an FP64 m,
// so the kernels apply the FP64 matrix itself: with two floats (48 bits) every application
// of a gate would carry the same representation error, and that error adds up coherently
// over deep circuits. A real part of one output, sum_k m_k x_k over split values, is
// accumulated like the compensated dot product of Ogita, Rump and Oishi (2005): the leading
// products are summed with TwoSum, every error term (product errors, the cross terms
// m_hi x_lo, m_lo x_hi, m_lo x_lo, m_3 x_hi and the TwoSum errors) goes into one FP32
// compensation, and the result is renormalised with Fast2Sum. The error per update is a few
// units of 2^-48 of the terms' magnitudes, from roundings with no preferred sign.
#include "internal.h"

namespace qsim {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}

// Running sum of split products: S (leading) and E (compensation).
struct Acc {
  float s, e;
};

// first term m x, m = (mh, ml, m3), x = (xh, xl)
__device__ __forceinline__ Acc term0(float mh, float ml, float m3, float xh, float xl) {
  Acc a;
  a.s = mh * xh;
  float e = fmaf(mh, xh, -a.s);
  e = fmaf(mh, xl, e);
  e = fmaf(ml, xh, e);
  e = fmaf(ml, xl, e);
  a.e = fmaf(m3, xh, e);
  return a;
}

__device__ __forceinline__ void term(Acc &a, float mh, float ml, float m3, float xh, float xl) {
  const float p = mh * xh;
  float pe = fmaf(mh, xh, -p);
  pe = fmaf(mh, xl, pe);
  pe = fmaf(ml, xh, pe);
  pe = fmaf(ml, xl, pe);
  pe = fmaf(m3, xh, pe);
  float s, t;
  two_sum(a.s, p, s, t);
  a.s = s;
  a.e += t + pe;
}

__device__ __forceinline__ void finish(const Acc &a, float &hi, float &lo) { fast_two_sum(a.s, a.e, hi, lo); }

// A split complex amplitude in registers.
struct Z {
  float rh, ih, rl, il;
};

__device__ __forceinline__ Z load_z(const float *p) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  return Z{v.x, v.y, v.z, v.w};
}

__device__ __forceinline__ void store_z(float *p, const Z &z) {
  *reinterpret_cast<float4 *>(p) = make_float4(z.rh, z.ih, z.rl, z.il);
}

// Two consecutive split amplitudes with one 256-bit access (p 32-byte aligned).
// Used by the classes with little arithmetic (swap, anti-diagonal), which otherwise run into
// the load/store queue limit; the arithmetic-heavy classes keep two 16-byte accesses, which
// the compiler schedules more freely (measured: 1.36 against 1.45 ms per 28-qubit sweep).
__device__ __forceinline__ void load_z2(const float *p, Z &a, Z &b) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(a.rh), "=f"(a.ih), "=f"(a.rl), "=f"(a.il), "=f"(b.rh), "=f"(b.ih), "=f"(b.rl), "=f"(b.il)
               : "l"(p)
               : "memory");
}

__device__ __forceinline__ void store_z2(float *p, const Z &a, const Z &b) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.rh), "f"(a.ih),
               "f"(a.rl), "f"(a.il), "f"(b.rh), "f"(b.ih), "f"(b.rl), "f"(b.il)
               : "memory");
}

// Split complex matrix entry: re = rh + rl + r3, im = ih + il + i3.
struct Mz {
  float rh, rl, ih, il, r3, i3;
};

template <int N>
struct MzN {
  Mz m[N];
};

// y = sum_j m_j x_j over `n` complex terms (split arithmetic)
template <int N>
__device__ __forceinline__ Z cdot(const Mz *m, const Z *x) {
  // Re y = sum (m.r x.r - m.i x.i),  Im y = sum (m.r x.i + m.i x.r)
  Acc re = term0(m[0].rh, m[0].rl, m[0].r3, x[0].rh, x[0].rl);
  term(re, -m[0].ih, -m[0].il, -m[0].i3, x[0].ih, x[0].il);
  Acc im = term0(m[0].rh, m[0].rl, m[0].r3, x[0].ih, x[0].il);
  term(im, m[0].ih, m[0].il, m[0].i3, x[0].rh, x[0].rl);
#pragma unroll
  for (int j = 1; j < N; ++j) {
    term(re, m[j].rh, m[j].rl, m[j].r3, x[j].rh, x[j].rl);
    term(re, -m[j].ih, -m[j].il, -m[j].i3, x[j].ih, x[j].il);
    term(im, m[j].rh, m[j].rl, m[j].r3, x[j].ih, x[j].il);
    term(im, m[j].ih, m[j].il, m[j].i3, x[j].rh, x[j].rl);
  }
  Z y;
  finish(re, y.rh, y.rl);
  finish(im, y.ih, y.il);
  return y;
}

// y = m x for a real entry m (imaginary part zero)
__device__ __forceinline__ Z rdot2(const Mz &m0, const Z &x0, const Mz &m1, const Z &x1) {
  Acc re = term0(m0.rh, m0.rl, m0.r3, x0.rh, x0.rl);
  term(re, m1.rh, m1.rl, m1.r3, x1.rh, x1.rl);
  Acc im = term0(m0.rh, m0.rl, m0.r3, x0.ih, x0.il);
  term(im, m1.rh, m1.rl, m1.r3, x1.ih, x1.il);
  Z y;
  finish(re, y.rh, y.rl);
  finish(im, y.ih, y.il);
  return y;
}

__device__ __forceinline__ unsigned long long insert_zeros(unsigned long long g, const Ins &ins) {
#pragma unroll 1
  for (int k = 0; k < ins.n; ++k) {
    const unsigned long long low = g & ((1ULL << ins.pos[k]) - 1ULL);
    g = ((g ^ low) << 1) | low;
  }
  return g | ins.set;
}

template <int CLS>
__device__ __forceinline__ void apply2(Z &a, Z &b, const MzN<4> &m) {
  if (CLS == MC_SWAP) {
    const Z t = a;
    a = b;
    b = t;
  } else if (CLS == MC_ANTI) {
    const Z na = cdot<1>(&m.m[1], &b), nb = cdot<1>(&m.m[2], &a);
    a = na;
    b = nb;
  } else if (CLS == MC_REAL) {
    const Z na = rdot2(m.m[0], a, m.m[1], b), nb = rdot2(m.m[2], a, m.m[3], b);
    a = na;
    b = nb;
  } else if (CLS == 4) {
    a = cdot<1>(&m.m[0], &a);
    b = cdot<1>(&m.m[3], &b);
  } else {
    const Z x[2] = {a, b};
    const Z na = cdot<2>(&m.m[0], x), nb = cdot<2>(&m.m[2], x);
    a = na;
    b = nb;
  }
}

enum Mode { SPLIT = 0, INVEC = 1, SCALAR = 2 };

// Pair sweep. Chunks are 32 bytes = 2 amplitudes (aligned: the chunk index is even); SPLIT
// needs every inserted bit >= 1.
template <int CLS, int MODE>
__global__ void __launch_bounds__(kThreads)
    k_pair_df(float *__restrict__ psi, long long items, Ins ins, unsigned long long off0, unsigned long long off1,
              MzN<4> m) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    if (MODE == SPLIT) {
      const unsigned long long base = insert_zeros((unsigned long long)g * 2, ins);
      float *pa = psi + 4 * (base + off0), *pb = psi + 4 * (base + off1);
      Z a0, a1, b0, b1;
      if constexpr (CLS == MC_SWAP || CLS == MC_ANTI) {
        load_z2(pa, a0, a1);
        load_z2(pb, b0, b1);
      } else {
        a0 = load_z(pa);
        a1 = load_z(pa + 4);
        b0 = load_z(pb);
        b1 = load_z(pb + 4);
      }
      apply2<CLS>(a0, b0, m);
      apply2<CLS>(a1, b1, m);
      if constexpr (CLS == MC_SWAP || CLS == MC_ANTI) {
        store_z2(pa, a0, a1);
        store_z2(pb, b0, b1);
      } else {
        store_z(pa, a0);
        store_z(pa + 4, a1);
        store_z(pb, b0);
        store_z(pb + 4, b1);
      }
    } else if (MODE == INVEC) {  // target bit 0: the pair is the chunk
      const unsigned long long base = insert_zeros((unsigned long long)g * 2, ins);
      float *p = psi + 4 * base;
      Z a = load_z(p), b = load_z(p + 4);
      apply2<CLS>(a, b, m);
      store_z(p, a);
      store_z(p + 4, b);
    } else {
      const unsigned long long base = insert_zeros((unsigned long long)g, ins);
      float *pa = psi + 4 * (base + off0), *pb = psi + 4 * (base + off1);
      Z a = load_z(pa), b = load_z(pb);
      apply2<CLS>(a, b, m);
      store_z(pa, a);
      store_z(pb, b);
    }
  }
}

__global__ void __launch_bounds__(kThreads)
    k_quad_df(float *__restrict__ psi, long long items, Ins ins, ulonglong4 off, MzN<16> m) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const unsigned long long o[4] = {off.x, off.y, off.z, off.w};
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    const unsigned long long base = insert_zeros((unsigned long long)g, ins);
    Z x[4], y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) x[r] = load_z(psi + 4 * (base + o[r]));
#pragma unroll
    for (int r = 0; r < 4; ++r) y[r] = cdot<4>(&m.m[4 * r], x);
#pragma unroll
    for (int r = 0; r < 4; ++r) store_z(psi + 4 * (base + o[r]), y[r]);
  }
}

// Multiply every amplitude whose mask bits are all 1 by a unit complex phase.
template <int PC>
__global__ void __launch_bounds__(kThreads)
    k_phase_df(float *__restrict__ psi, long long items, Ins ins, Mz ph) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    const unsigned long long i = insert_zeros((unsigned long long)g, ins);
    float *p = psi + 4 * i;
    Z z = load_z(p);
    if (PC == PC_NEG) {
      z = Z{-z.rh, -z.ih, -z.rl, -z.il};
    } else if (PC == PC_PLUS_I) {
      z = Z{-z.ih, z.rh, -z.il, z.rl};
    } else if (PC == PC_MINUS_I) {
      z = Z{z.ih, -z.rh, z.il, -z.rl};
    } else {
      z = cdot<1>(&ph, &z);
    }
    store_z(p, z);
  }
}

// Merged diagonal gates on the split format: amplitude x times the exact FP64 table entry
// tab[idx(x)] (six floats), bit j of idx(x) = bit pos[j] of x; one compensated product per
// amplitude, as a single phase gate takes. A thread owns a 32-byte chunk of two amplitudes.
__global__ void __launch_bounds__(kThreads)
    k_diag_df(float *__restrict__ psi, long long items, DiagIdx d, const float *__restrict__ tab) {
  __shared__ Mz st[1 << kDiagBits];
  for (int i = threadIdx.x; i < (1 << d.nq); i += blockDim.x)
    st[i] = Mz{tab[6 * i], tab[6 * i + 1], tab[6 * i + 2], tab[6 * i + 3], tab[6 * i + 4], tab[6 * i + 5]};
  __syncthreads();
  unsigned odd = 0;  // index bit of position 0, set in the chunk's second amplitude
#pragma unroll
  for (int j = 0; j < kDiagBits; ++j)
    if (j < d.nq && d.pos[j] == 0) odd = 1u << j;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    const unsigned long long x0 = (unsigned long long)g * 2;
    unsigned hi = 0;
#pragma unroll
    for (int j = 0; j < kDiagBits; ++j)
      if (j < d.nq) hi |= (unsigned)((x0 >> d.pos[j]) & 1ULL) << j;
    float *p = psi + 4 * x0;
    const Z a = load_z(p), b = load_z(p + 4);
    store_z(p, cdot<1>(&st[hi], &a));
    store_z(p + 4, cdot<1>(&st[hi | odd], &b));
  }
}

template <int K>
__global__ void __launch_bounds__(128)
    k_fused_df(float *__restrict__ psi, long long items, Ins ins, const unsigned long long *__restrict__ offs,
               const float *__restrict__ mat) {
  constexpr int D = 1 << K;
  __shared__ Mz sm[D * D];
  __shared__ unsigned long long so[D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x)
    sm[i] = Mz{mat[6 * i], mat[6 * i + 1], mat[6 * i + 2], mat[6 * i + 3], mat[6 * i + 4], mat[6 * i + 5]};
  for (int i = threadIdx.x; i < D; i += blockDim.x) so[i] = offs[i];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
    const unsigned long long base = insert_zeros((unsigned long long)g, ins);
    Z x[D];
#pragma unroll
    for (int c = 0; c < D; ++c) x[c] = load_z(psi + 4 * (base + so[c]));
#pragma unroll 1
    for (int r = 0; r < D; ++r) store_z(psi + 4 * (base + so[r]), cdot<D>(&sm[r * D], x));
  }
}

// In-place format conversions: plain complex128 <-> split.
__global__ void k_to_split(double *__restrict__ psi, long long amps) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    const double2 v = reinterpret_cast<const double2 *>(psi)[i];
    const float rh = (float)v.x, ih = (float)v.y;
    const float rl = (float)(v.x - (double)rh), il = (float)(v.y - (double)ih);
    reinterpret_cast<float4 *>(psi)[i] = make_float4(rh, ih, rl, il);
  }
}

__global__ void k_to_plain(double *__restrict__ psi, long long amps) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < amps; i += stride) {
    const float4 v = reinterpret_cast<const float4 *>(psi)[i];
    reinterpret_cast<double2 *>(psi)[i] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
}

inline int grid_for(long long items, int threads) {
  long long per = 8LL * num_sms();
  long long need = (items + threads - 1) / threads;
  if (need < 1) need = 1;
  return (int)(need < per ? need : per);
}

// v = (rh + rl + r3) + i (ih + il + i3) exactly: each difference below is exact in FP64
Mz split_entry(const cd &v) {
  Mz z;
  const double dr = v.real() - (double)(z.rh = (float)v.real());
  const double di = v.imag() - (double)(z.ih = (float)v.imag());
  z.rl = (float)dr;
  z.il = (float)di;
  z.r3 = (float)(dr - (double)z.rl);
  z.i3 = (float)(di - (double)z.il);
  return z;
}

template <int CLS>
void pair_df_typed(const StateDev &s, const Ins &ins, unsigned long long off0, unsigned long long off1,
                   const MzN<4> &m) {
  float *psi = static_cast<float *>(s.amps);
  const long long bases = 1LL << (s.n - ins.n);
  const bool split_ok = ins.n == 0 || ins.pos[0] >= 1;
  if (split_ok && s.n - ins.n >= 1) {
    const long long items = bases / 2;
    k_pair_df<CLS, SPLIT><<<grid_for(items, kThreads), kThreads, 0, s.stream>>>(psi, items, ins, off0, off1, m);
    return;
  }
  // target at bit 0 with every control above it: the pair is one 32-byte chunk
  if (off0 == 0 && off1 == 1) {
    Ins ctl = ins;
    ctl.n = 0;
    bool ok = true;
    for (int k = 0; k < ins.n; ++k) {
      if (ins.pos[k] == 0) continue;
      ctl.pos[ctl.n++] = ins.pos[k];
    }
    for (int k = 0; k < ctl.n; ++k) ok = ok && ctl.pos[k] >= 1;
    if (ok) {
      const long long items = (1LL << (s.n - ctl.n)) / 2;
      k_pair_df<CLS, INVEC><<<grid_for(items, kThreads), kThreads, 0, s.stream>>>(psi, items, ctl, 0, 1, m);
      return;
    }
  }
  k_pair_df<CLS, SCALAR><<<grid_for(bases, kThreads), kThreads, 0, s.stream>>>(psi, bases, ins, off0, off1, m);
}

}  // namespace

qsim_status launch_pair_df(const StateDev &s, const Ins &ins, unsigned long long off0, unsigned long long off1,
                           const cd m[4], int cls, int64_t *bytes) {
  if (bytes) *bytes += 2LL * 16 * (2LL << (s.n - ins.n));
  MzN<4> mm;
  for (int i = 0; i < 4; ++i) mm.m[i] = split_entry(m[i]);
  switch (cls) {
    case MC_SWAP: pair_df_typed<MC_SWAP>(s, ins, off0, off1, mm); break;
    case MC_ANTI: pair_df_typed<MC_ANTI>(s, ins, off0, off1, mm); break;
    case MC_REAL: pair_df_typed<MC_REAL>(s, ins, off0, off1, mm); break;
    case 4: pair_df_typed<4>(s, ins, off0, off1, mm); break;
    default: pair_df_typed<MC_GENERIC>(s, ins, off0, off1, mm); break;
  }
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

qsim_status launch_quad_df(const StateDev &s, const Ins &ins, const unsigned long long off[4], const cd m[16],
                           int64_t *bytes) {
  if (bytes) *bytes += 2LL * 16 * (4LL << (s.n - ins.n));
  MzN<16> mm;
  for (int i = 0; i < 16; ++i) mm.m[i] = split_entry(m[i]);
  const long long items = 1LL << (s.n - ins.n);
  k_quad_df<<<grid_for(items, kThreads), kThreads, 0, s.stream>>>(static_cast<float *>(s.amps), items, ins,
                                                                  make_ulonglong4(off[0], off[1], off[2], off[3]),
                                                                  mm);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

qsim_status launch_phase_df(const StateDev &s, unsigned long long mask, cd ph, int64_t *bytes) {
  Ins ins;
  ins.n = 0;
  ins.set = mask;
  for (int q = 0; q < s.n; ++q)
    if (mask >> q & 1ULL) ins.pos[ins.n++] = q;
  const long long items = 1LL << (s.n - ins.n);
  if (bytes) *bytes += 2LL * 16 * items;
  float *psi = static_cast<float *>(s.amps);
  const Mz z = split_entry(ph);
  const int grid = grid_for(items, kThreads);
  if (ph == cd(-1.0, 0.0)) k_phase_df<PC_NEG><<<grid, kThreads, 0, s.stream>>>(psi, items, ins, z);
  else if (ph == cd(0.0, 1.0)) k_phase_df<PC_PLUS_I><<<grid, kThreads, 0, s.stream>>>(psi, items, ins, z);
  else if (ph == cd(0.0, -1.0)) k_phase_df<PC_MINUS_I><<<grid, kThreads, 0, s.stream>>>(psi, items, ins, z);
  else k_phase_df<PC_GENERAL><<<grid, kThreads, 0, s.stream>>>(psi, items, ins, z);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

qsim_status launch_diag_df(const StateDev &s, const DiagIdx &d, const void *dev_tab, int64_t *bytes) {
  if (d.nq < 1 || d.nq > kDiagBits || s.n < 1) {
    set_error("diagonal table over %d qubits (1..%d) on %d qubits", d.nq, kDiagBits, s.n);
    return QSIM_EINVAL;
  }
  const long long items = 1LL << (s.n - 1);
  if (bytes) *bytes += 2LL * 16 * (items * 2);
  k_diag_df<<<grid_for(items, kThreads), kThreads, 0, s.stream>>>(static_cast<float *>(s.amps), items, d,
                                                                  static_cast<const float *>(dev_tab));
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

// dev_mat: 2^k x 2^k split entries (rh, rl, ih, il, r3, i3) followed by 2^k offsets (u64).
qsim_status launch_fused_df(const StateDev &s, const int *phys, int k, unsigned long long ctrl_mask,
                            const void *dev_mat, int64_t *bytes) {
  unsigned long long all = ctrl_mask;
  for (int j = 0; j < k; ++j) all |= 1ULL << phys[j];
  Ins ins;
  ins.n = 0;
  ins.set = ctrl_mask;
  for (int q = 0; q < s.n; ++q)
    if (all >> q & 1ULL) ins.pos[ins.n++] = q;
  const long long items = 1LL << (s.n - ins.n);
  if (bytes) *bytes += 2LL * 16 * (items << k);
  const int D = 1 << k;
  const float *mat = static_cast<const float *>(dev_mat);
  const unsigned long long *offs = reinterpret_cast<const unsigned long long *>(mat + 6 * D * D);
  float *psi = static_cast<float *>(s.amps);
  const int grid = grid_for(items, 128);
  switch (k) {
    case 1: k_fused_df<1><<<grid, 128, 0, s.stream>>>(psi, items, ins, offs, mat); break;
    case 2: k_fused_df<2><<<grid, 128, 0, s.stream>>>(psi, items, ins, offs, mat); break;
    case 3: k_fused_df<3><<<grid, 128, 0, s.stream>>>(psi, items, ins, offs, mat); break;
    case 4: k_fused_df<4><<<grid, 128, 0, s.stream>>>(psi, items, ins, offs, mat); break;
    case 5: k_fused_df<5><<<grid, 128, 0, s.stream>>>(psi, items, ins, offs, mat); break;
    default: set_error("fused width %d not in 1..5", k); return QSIM_EINVAL;
  }
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

// Host layout of a split fused matrix for launch_fused_df (phys order as in the launch).
void append_fused_df(std::vector<unsigned char> &buf, const cd *u, int k, const int *phys) {
  const int D = 1 << k;
  const size_t off = buf.size();
  buf.resize(off + (size_t)D * D * 24 + (size_t)D * 8);
  float *f = reinterpret_cast<float *>(buf.data() + off);
  for (int i = 0; i < D * D; ++i) {
    const Mz z = split_entry(u[i]);
    f[6 * i] = z.rh;
    f[6 * i + 1] = z.rl;
    f[6 * i + 2] = z.ih;
    f[6 * i + 3] = z.il;
    f[6 * i + 4] = z.r3;
    f[6 * i + 5] = z.i3;
  }
  unsigned long long *o = reinterpret_cast<unsigned long long *>(f + 6 * D * D);
  for (int r = 0; r < D; ++r) {
    unsigned long long v = 0;
    for (int j = 0; j < k; ++j)
      if ((r >> (k - 1 - j)) & 1) v |= 1ULL << phys[j];
    o[r] = v;
  }
}

qsim_status launch_to_split(const StateDev &s) {
  const long long amps = 1LL << s.n;
  k_to_split<<<grid_for(amps, kThreads), kThreads, 0, s.stream>>>(static_cast<double *>(s.amps), amps);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

qsim_status launch_to_plain(const StateDev &s) {
  const long long amps = 1LL << s.n;
  k_to_plain<<<grid_for(amps, kThreads), kThreads, 0, s.stream>>>(static_cast<double *>(s.amps), amps);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

}  // namespace qsim
