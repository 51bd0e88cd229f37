// Fused k-qubit unitary (k = 4 or 5) on the tensor cores: a split-precision (3xTF32)
// complex GEMM with FP32 accumulation in tensor memory.
//
// With the k fused qubits at physical positions 0..k-1, a complex64 state is a row-major
// real matrix A[M][KR] with M = 2^(n-k) rows and KR = 2^(k+1) reals per row (2^k
// interleaved amplitudes). Applying U to every row is out = A R, where R (KR x KR) is the
// real form of U^T:  R[2l][2j] = Re U[j][l], R[2l+1][2j] = -Im U[j][l],
//                    R[2l][2j+1] = Im U[j][l], R[2l+1][2j+1] = Re U[j][l].
// Both operands are split into TF32 parts, A = Ahi + Alo and R = Rhi + Rlo, and
// out = Ahi Rhi + Alo Rhi + Ahi Rlo (the dropped Alo Rlo term is ~2^-22 relative).
//
// One CTA per SM walks its tiles of 128 rows. Thread 0 issues TMA loads (three stages of
// prefetch) and the tcgen05.mma instructions; all 128 threads split A into Ahi (in place)
// and Alo, and run the epilogue: tcgen05.ld of the 128 x KR FP32 accumulator, a write into
// a 128-byte-swizzled staging tile, and a TMA store back to the same rows (in place).
// Every mbarrier wait is bounded by a timer; on expiry the kernel records the fact in a
// device flag, drains its stores, frees its tensor memory and returns.
#include <cuda.h>

#include <cstring>

#include "internal.h"

namespace qsim {

namespace {

constexpr int kTcThreads = 128;
constexpr int kStages = 3;
constexpr unsigned long long kWaitLimitNs = 4000000000ULL;  // 4 s

__device__ int g_tc_timeout = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false if the time limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major with 128-byte swizzle: rows of 128 bytes, 8-row
// groups 1024 bytes apart (stride byte offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int K>
struct TcLayout {
  static constexpr int KR = 2 << K;               // reals per row
  static constexpr int NH = KR / 32;              // 128-byte column halves per row
  static constexpr int HALF = 128 * 128;          // one half of a 128-row tile
  static constexpr int TILE = 128 * KR * 4;       // A tile bytes
  static constexpr int RHALF = KR * 128;          // one half of an R operand (KR rows)
  static constexpr int RMAT = KR * KR * 4;        // one R operand
  static constexpr int OFF_A = 0;
  static constexpr int OFF_ALO = OFF_A + kStages * TILE;
  static constexpr int OFF_RHI = OFF_ALO + TILE;
  static constexpr int OFF_RLO = OFF_RHI + RMAT;
  static constexpr int OFF_OUT = OFF_RLO + RMAT;
  static constexpr int OFF_BAR = OFF_OUT + TILE;
  static constexpr int BYTES = OFF_BAR + 64;
  static constexpr int TMEM_COLS = KR < 32 ? 32 : KR;
  // instruction descriptor: D f32, A/B tf32, both K-major, N = KR, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KR >> 3) << 17) |
                                    ((uint32_t)(128 >> 4) << 24);
};

static_assert(TcLayout<5>::BYTES + 1024 <= 227 * 1024, "fused tensor-core tile does not fit");

template <int K>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_fused_tc(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_r,
               int ntiles) {
  using L = TcLayout<K>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);
  uint64_t *mma_bar = full + kStages;
  uint64_t *r_bar = mma_bar + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(r_bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    mbar_init(mma_bar, 1);
    mbar_init(r_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (tid == 0) {
    mbar_expect_tx(r_bar, 2 * L::RMAT);
    for (int h = 0; h < L::NH; ++h) {
      tma_load_2d(smem + L::OFF_RHI + h * L::RHALF, &tmap_r, 32 * h, 0, r_bar);
      tma_load_2d(smem + L::OFF_RLO + h * L::RHALF, &tmap_r, 32 * h, L::KR, r_bar);
    }
    for (int s = 0; s < kStages; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile >= ntiles) break;
      mbar_expect_tx(&full[s], L::TILE);
      for (int h = 0; h < L::NH; ++h)
        tma_load_2d(smem + L::OFF_A + s * L::TILE + h * L::HALF, &tmap_a, 32 * h, tile * 128, &full[s]);
    }
  }
  bool ok = mbar_wait(r_bar, 0);
  if (__syncthreads_or(!ok)) goto done;

  for (int it = 0;; ++it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= ntiles) break;
    const int s = it % kStages;
    unsigned char *a_s = smem + L::OFF_A + s * L::TILE;
    ok = mbar_wait(&full[s], (uint32_t)((it / kStages) & 1));
    if (__syncthreads_or(!ok)) goto done;

    // split A into TF32 parts: hi in place, lo into the Alo tile (same swizzled offsets)
    {
      float4 *ah = reinterpret_cast<float4 *>(a_s);
      float4 *al = reinterpret_cast<float4 *>(smem + L::OFF_ALO);
#pragma unroll 4
      for (int i = tid; i < L::TILE / 16; i += kTcThreads) {
        const float4 v = ah[i];
        float4 h, l;
        h.x = tf32_rna(v.x); l.x = v.x - h.x;
        h.y = tf32_rna(v.y); l.y = v.y - h.y;
        h.z = tf32_rna(v.z); l.z = v.z - h.z;
        h.w = tf32_rna(v.w); l.w = v.w - h.w;
        ah[i] = h;
        al[i] = l;
      }
    }
    fence_proxy_async();
    __syncthreads();

    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_u32(a_s), a_lo = smem_u32(smem + L::OFF_ALO);
      const uint32_t r_hi = smem_u32(smem + L::OFF_RHI), r_lo = smem_u32(smem + L::OFF_RLO);
#pragma unroll
      for (int ks = 0; ks < L::KR / 8; ++ks) {
        const uint32_t ao = (ks >> 2) * L::HALF + (ks & 3) * 32;
        const uint32_t ro = (ks >> 2) * L::RHALF + (ks & 3) * 32;
        mma_tf32(taddr, desc_sw128(a_hi + ao), desc_sw128(r_hi + ro), L::IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(taddr, desc_sw128(a_lo + ao), desc_sw128(r_hi + ro), L::IDESC, 1u);
        mma_tf32(taddr, desc_sw128(a_hi + ao), desc_sw128(r_lo + ro), L::IDESC, 1u);
      }
      mma_commit(mma_bar);
    }
    ok = mbar_wait(mma_bar, (uint32_t)(it & 1));
    tc_fence_after();
    if (tid == 0 && ok) {
      // the stage is free again: prefetch the tile kStages iterations ahead
      const int next = tile + kStages * gridDim.x;
      if (next < ntiles) {
        mbar_expect_tx(&full[s], L::TILE);
        for (int h = 0; h < L::NH; ++h)
          tma_load_2d(a_s + h * L::HALF, &tmap_a, 32 * h, next * 128, &full[s]);
      }
      bulk_wait_read0();  // the previous store has finished reading the staging tile
    }
    if (__syncthreads_or(!ok)) goto done;

    // epilogue: accumulator rows -> swizzled staging tile -> TMA store
    {
      const int r = warp * 32 + lane;
      unsigned char *out = smem + L::OFF_OUT;
#pragma unroll
      for (int h = 0; h < L::NH; ++h) {
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * h), v);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4 q = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
          *reinterpret_cast<float4 *>(out + h * L::HALF + r * 128 + ((c ^ (r & 7)) << 4)) = q;
        }
      }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      for (int h = 0; h < L::NH; ++h) tma_store_2d(&tmap_a, 32 * h, tile * 128, smem + L::OFF_OUT + h * L::HALF);
      bulk_commit();
    }
  }

done:
  if (!ok && tid == 0) atomicExch(&g_tc_timeout, 1);
  if (tid == 0) bulk_wait0();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"((uint32_t)L::TMEM_COLS)
                 : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D FP32 tensor map over rows of `row_floats` floats, boxes of 32 floats x box_rows rows,
// 128-byte swizzle.
qsim_status make_map(CUtensorMap *m, const void *base, int row_floats, unsigned long long rows, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return QSIM_EUNSUPPORTED;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)row_floats, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)row_floats * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QSIM_ECUDA;
  }
  return QSIM_OK;
}

float host_tf32_rna(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  if ((b & 0x7F800000u) != 0x7F800000u) b = (b + 0x1000u) & 0xFFFFE000u;
  float r;
  memcpy(&r, &b, 4);
  return r;
}

template <int K>
qsim_status launch_k(const StateDev &s, const void *rmats, int64_t *bytes) {
  using L = TcLayout<K>;
  static bool attr_set = false;
  if (!attr_set) {
    QS_TRY_CUDA(cudaFuncSetAttribute(k_fused_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES + 1024));
    attr_set = true;
  }
  CUtensorMap ma, mr;
  const unsigned long long rows = 1ULL << (s.n - K);
  QS_TRY(make_map(&ma, s.amps, L::KR, rows, 128));
  QS_TRY(make_map(&mr, rmats, L::KR, 2 * L::KR, L::KR));
  const int ntiles = (int)(rows / 128);
  int grid = num_sms();
  if (grid > ntiles) grid = ntiles;
  if (bytes) *bytes += 2LL * 8 * (1LL << s.n);
  k_fused_tc<K><<<grid, kTcThreads, L::BYTES + 1024, s.stream>>>(ma, mr, ntiles);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

}  // namespace

bool fused_tc_supported(const StateDev &s, int k) {
  // 128-row tiles, at most 2^31 tiles' worth of rows, and a driver with tensor maps
  return s.dtype == QSIM_C64 && (k == 4 || k == 5) && s.n >= k + 7 && s.n - k - 7 <= 30 &&
         encode_fn() != nullptr;
}

size_t tc_operand_floats(int k) { return (size_t)2 * (2 << k) * (2 << k); }

// Rt (the K-major copy of R: Rt[n][k] = R[k][n]) split into TF32 hi and lo parts.
void build_tc_operands(int k, const cd *u, float *dst_hi, float *dst_lo) {
  const int D = 1 << k, KR = 2 * D;
  for (int j = 0; j < D; ++j)
    for (int l = 0; l < D; ++l) {
      const cd v = u[(size_t)j * D + l];
      // R[2l][2j] = Re, R[2l+1][2j] = -Im, R[2l][2j+1] = Im, R[2l+1][2j+1] = Re
      const double e[2][2] = {{v.real(), v.imag()}, {-v.imag(), v.real()}};  // e[row parity][col parity]
      for (int rp = 0; rp < 2; ++rp)
        for (int cp = 0; cp < 2; ++cp) {
          const int kk = 2 * l + rp, nn = 2 * j + cp;
          const double x = e[rp][cp];
          const float hi = host_tf32_rna((float)x);
          const float lo = host_tf32_rna((float)(x - (double)hi));
          dst_hi[(size_t)nn * KR + kk] = hi;
          dst_lo[(size_t)nn * KR + kk] = lo;
        }
    }
}

qsim_status launch_fused_tc(const StateDev &s, int k, const void *dev_rmats, int, int, int64_t *bytes) {
  if (!fused_tc_supported(s, k)) {
    set_error("tensor-core fused apply needs complex64, k in {4, 5} and n >= k + 7");
    return QSIM_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(dev_rmats) & 127u) {
    set_error("fused operand buffer must be 128-byte aligned");
    return QSIM_EINVAL;
  }
  return k == 5 ? launch_k<5>(s, dev_rmats, bytes) : launch_k<4>(s, dev_rmats, bytes);
}

qsim_status tc_take_timeout() {
  int v = 0;
  QS_TRY_CUDA(cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int)));
  if (v) {
    const int zero = 0;
    QS_TRY_CUDA(cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)));
    set_error("a bounded wait in the tensor-core fused kernel ran out");
    return QSIM_ETIMEOUT;
  }
  return QSIM_OK;
}

}  // namespace qsim
