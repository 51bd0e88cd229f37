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
// Per k-step the MMA warp issues one N = 2 KR product of Ahi with [Rhi | Rlo] (main and
// first correction in separate accumulator columns) and one N = KR product of Alo with
// Rhi into the correction columns; the epilogue adds main + correction in FP32 with round
// to nearest. Keeping the corrections out of the main sum matters because the tensor
// core's FP32 accumulation rounds toward zero: fewer roundings on the large sum mean a
// smaller norm bias.
//
// A persistent, warp-specialised CTA (14 warps, one per SM) walks its 128-row tiles
// through a ring of shared-memory stages (six at k = 5, eight at k = 4, when the low TF32
// part of the tile lives in tensor memory; four and six when it lives in shared memory):
// warp 0 issues TMA loads, warp 1 issues tcgen05.mma into one of two tensor-memory
// accumulators, warps 2-9 split each landed tile into Ahi (in place) and Alo, and warps
// 10-13 read the accumulator out (tcgen05.ld), write the sum into the tile's own stage in
// the 128-byte swizzle (permuted when the epilogue also moves qubits) and TMA-store it back
// to the same rows. mbarriers hand each tile from role to role; every wait on them is
// bounded by a timer, and on expiry the kernel records the fact in a device flag, drains
// its stores, frees its tensor memory and returns.
#include <cuda.h>

#include <cstdlib>
#include <cstring>

#include "internal.h"

namespace qsim {

namespace {

constexpr int kMaxStages = 8;
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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

// Self-test of the bounded wait: every warp waits on a barrier that nothing arrives at.
__global__ void k_wait_selftest(unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0) atomicExch(&g_tc_timeout, 1);
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

// Rank 2 + md tensor-map copies (md = 1..3 size-2 dimensions for the tile's high row bits):
// coordinates (x, y, 0, ...), a whole box of 2^c rows x 2^md row groups per copy.
__device__ __forceinline__ void tma_load_md(int md, void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  const uint32_t d = smem_u32(dst), b = smem_u32(bar), z = 0;
  if (md == 1)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            d),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(b)
        : "memory");
  else if (md == 2)
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(d),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(z), "r"(b)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(d),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(z), "r"(z), "r"(b)
        : "memory");
}

__device__ __forceinline__ void tma_store_md(int md, const CUtensorMap *map, int x, int y, const void *src) {
  const uint32_t sa = smem_u32(src), z = 0;
  if (md == 1)
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map), "r"(x),
                 "r"(y), "r"(z), "r"(sa)
                 : "memory");
  else if (md == 2)
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(z), "r"(sa)
                 : "memory");
  else
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(z), "r"(z), "r"(sa)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
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

// Same, with the A operand read from tensor memory (row r in lane r, one TF32 element per
// column, K columns from a_tmem on).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
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

// Store NV consecutive 32-bit columns of this thread's lane (NV = 16 or 32).
template <int NV>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const float *v);
template <>
__device__ __forceinline__ void tmem_st<32>(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<16>(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Shared-memory plan of the fused kernel for k fused qubits (KR reals per row). With TLO
// the low TF32 part of A lives in tensor memory (two ping-pong buffers of KR columns next
// to the accumulators) and the shared memory it would take holds more TMA stages.
template <int K, bool TLO>
struct TcLayout {
  static constexpr int KR = 2 << K;               // reals per row: 32 (k = 4) or 64 (k = 5)
  static constexpr int NH = KR / 32;              // 128-byte column halves per row
  static constexpr int HALF = 128 * 128;          // one half of a 128-row tile (bytes)
  static constexpr int TILE = 128 * KR * 4;       // one 128-row tile (bytes)
  static constexpr int STAGES = TLO ? (K == 5 ? 6 : 8) : (K == 5 ? 4 : 6);
  static constexpr int BROWS = 2 * KR;            // B operand rows: Rhi^T then Rlo^T
  static constexpr int BHALF = BROWS * 128;       // one half of the B operand (bytes)
  // STAGES tiles: TMA destination, then Ahi, then the output tile for the TMA store
  static constexpr int OFF_A = 0;
  static constexpr int OFF_ALO = OFF_A + STAGES * TILE;   // two tiles of Alo (ping-pong)
  static constexpr int OFF_B = OFF_ALO + (TLO ? 0 : 2 * TILE);
  static constexpr int OFF_BAR = OFF_B + NH * BHALF;
  static constexpr int BAR_BYTES = 512;           // TcBars (static_assert below)
  static constexpr int BYTES = OFF_BAR + BAR_BYTES;
  static constexpr int ACC_COLS = 2 * KR;         // main columns then correction columns
  static constexpr int ALO_COL = 2 * ACC_COLS;    // Alo buffers (TLO) after two accumulators
  static constexpr int USED_COLS = ALO_COL + (TLO ? 2 * KR : 0);
  static constexpr int TMEM_COLS = USED_COLS <= 128 ? 128 : USED_COLS <= 256 ? 256 : 512;
  static constexpr int CTAS_PER_SM = 1;
  // instruction descriptors: D f32, A/B tf32, both K-major, M = 128, N = 2 KR or KR
  __host__ __device__ static constexpr uint32_t idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  }
};

static_assert(TcLayout<5, false>::BYTES + 1024 <= 227 * 1024, "fused tensor-core tiles do not fit");
static_assert(TcLayout<5, true>::BYTES + 1024 <= 227 * 1024, "fused tensor-core tiles do not fit");
static_assert(TcLayout<4, true>::BYTES + 1024 <= 227 * 1024, "fused tensor-core tiles do not fit");
static_assert(TcLayout<5, true>::STAGES <= kMaxStages && TcLayout<4, true>::STAGES <= kMaxStages, "stages");


// Warp roles: 0 TMA producer, 1 MMA issuer (and tensor-memory owner), 2-9 convert A into
// its TF32 parts, 10-13 epilogue (tensor memory -> staging tile -> TMA store).
constexpr int kConvWarps = 8;
constexpr int kEpiWarp0 = 2 + kConvWarps;
constexpr int kTcWarps = kEpiWarp0 + 4;

// Barriers (shared memory): full (TMA landed), conv (Ahi/Alo written), sfree (stage free:
// the TMA store of the tile written into it has read it out), lofree (Alo buffer free: its
// MMAs are done), mmad (accumulator ready), accfree (accumulator read out), stg (output
// tile written by all epilogue warps).
struct TcBars {
  uint64_t full[kMaxStages], conv[kMaxStages], sfree[kMaxStages], lofree[2], mmad[2], accfree[2], stg, rbar;
  uint32_t tmem;
};

static_assert(sizeof(TcBars) <= TcLayout<5, true>::BAR_BYTES, "barrier block overflows its shared-memory slot");
// kernel parameters: two tensor maps, two ints and the tile plan within the 4 KB limit
static_assert(2 * sizeof(CUtensorMap) + 16 + sizeof(TcTilePlan) <= 4096, "fused kernel parameters too large");

// Tile geometry and the epilogue permutation (see TcTilePlan in internal.h).
__device__ __forceinline__ unsigned long long tile_base_row(long long t, const TcTilePlan &p) {
  unsigned long long g = (unsigned long long)t;
#pragma unroll 1
  for (int k = 0; k < p.ins_n; ++k) {
    const unsigned long long low = g & ((1ULL << p.ins[k]) - 1ULL);
    g = ((g ^ low) << 1) | low;
  }
  return g;
}

__device__ __forceinline__ unsigned long long box_row(unsigned long long base, int box, const TcTilePlan &p) {
  unsigned long long r = base;
#pragma unroll
  for (int j = 0; j < kTcMaxHbits; ++j)
    if (j < p.nh && ((box >> j) & 1)) r |= 1ULL << p.hbit[j];
  return r;
}

// First row of copy g of a tile whose map covers hbit[0 .. md-1]: the bits of g select the
// leftover high bits hbit[md ..].
__device__ __forceinline__ unsigned long long group_row(unsigned long long base, int g, int md, const TcTilePlan &p) {
  unsigned long long r = base;
#pragma unroll
  for (int i = 0; i < kTcMaxHbits; ++i)
    if (md + i < p.nh && ((g >> i) & 1)) r |= 1ULL << p.hbit[md + i];
  return r;
}

// Global row index of local tile row r: the low run takes r's low c bits, the high row
// bits take the rest.
__device__ __forceinline__ unsigned long long tile_row(unsigned long long base, int r, const TcTilePlan &p) {
  unsigned long long g = base | (unsigned long long)(r & ((1 << p.c) - 1));
#pragma unroll
  for (int j = 0; j < kTcMaxHbits; ++j)
    if (j < p.nh && ((r >> (p.c + j)) & 1)) g |= 1ULL << p.hbit[j];
  return g;
}

// Turns of row-phase term e for global row `grow`: its coefficient when every bit of its
// mask is set in the row (the term's fields are read with uniform addresses).
__device__ __forceinline__ float term_turns(const TcPhaseTerm &e, unsigned long long grow) {
  return (grow & e.mask) == e.mask ? e.c : 0.0f;
}

// Turns of the plan's row-phase terms that are the same for every row of the tile with base
// row `base` (terms nvary .. nterm-1 read no tile row bit): the lanes of the warp take the
// terms in turn and add up by a butterfly, which leaves the same sum in every lane.
__device__ __forceinline__ float tile_turns(const TcTilePlan &p, unsigned long long base, int lane) {
  float t = 0.0f;
#pragma unroll 1
  for (int g = p.nvary + lane; g < p.nterm; g += 32) t += term_turns(p.term[g], base);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Product of the plan's row phases for global row `grow`, as a unit complex number, given
// the tile's common part t0 (tile_turns): the terms add up in turns (exact for dyadic
// angles such as those of T, S, CZ and the QFT's controlled phases) and the sum is reduced
// to [0, 1) before one sincospi.
__device__ __forceinline__ float2 row_phase(const TcTilePlan &p, float t0, unsigned long long grow) {
  float t = t0;
#pragma unroll 4
  for (int g = 0; g < p.nvary; ++g) t += term_turns(p.term[g], grow);
  t -= floorf(t);
  float sn, cs;
  sincospif(2.0f * t, &sn, &cs);
  return make_float2(cs, sn);
}

// v (two interleaved complex numbers) times the complex factor (fr, fi), with the
// rounding fixed (one product, one FMA per component) so that every code path that
// applies it gives the same bits.
__device__ __forceinline__ float4 cmul2(float4 v, float fr, float fi) {
  return make_float4(fmaf(v.x, fr, __fmul_rn(-v.y, fi)), fmaf(v.x, fi, __fmul_rn(v.y, fr)),
                     fmaf(v.z, fr, __fmul_rn(-v.w, fi)), fmaf(v.z, fi, __fmul_rn(v.w, fr)));
}

template <int K, bool TLO>
__global__ void __launch_bounds__(kTcWarps * 32, 1)
    k_fused_tc(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_r,
               int ntiles, int mdim, const __grid_constant__ TcTilePlan plan) {
  using L = TcLayout<K, TLO>;
  constexpr int kStages = L::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcBars *bars = reinterpret_cast<TcBars *>(smem + L::OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  bool ok = true;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->conv[s], kConvWarps);
      mbar_init(&bars->sfree[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bars->lofree[a], 1);
      mbar_init(&bars->mmad[a], 1);
      mbar_init(&bars->accfree[a], 4);
    }
    mbar_init(&bars->stg, 4);
    mbar_init(&bars->rbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem)),
                 "r"((uint32_t)L::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = bars->tmem;

  if (warp == 0) {
    // ---- producer: the B operand once, then A tiles as stages free up (whole warp loops,
    // lane 0 issues)
    if (lane == 0) {
      mbar_expect_tx(&bars->rbar, (uint32_t)(L::NH * L::BHALF));
      for (int h = 0; h < L::NH; ++h) tma_load_2d(smem + L::OFF_B + h * L::BHALF, &tmap_r, 32 * h, 0, &bars->rbar);
    }
    __syncwarp();
    for (int j = 0; j < my_tiles; ++j) {
      const int s = j % kStages, u = j / kStages;
      ok = __all_sync(0xffffffffu, mbar_wait(&bars->sfree[s], (uint32_t)((u & 1) ^ 1)));
      if (!ok) break;
      if (lane == 0) {
        mbar_expect_tx(&bars->full[s], L::TILE);
        const unsigned long long base = tile_base_row(blockIdx.x + (long long)j * gridDim.x, plan);
        const int brows = 1 << plan.c;
        unsigned char *dst = smem + L::OFF_A + s * L::TILE;
        if (mdim > 0) {
          // the map's size-2 dimensions cover hbit[0 .. mdim-1]; leftover high bits (nh = 4
          // or 5) split the tile into 2 or 4 copies of 2^(c + 3) rows
          for (int g = 0; g < (1 << (plan.nh - mdim)); ++g) {
            const int y = (int)group_row(base, g, mdim, plan);
            for (int h = 0; h < L::NH; ++h)
              tma_load_md(mdim, dst + h * L::HALF + (g << mdim) * brows * 128, &tmap_a, 32 * h, y, &bars->full[s]);
          }
        } else {
          for (int b = 0; b < (1 << plan.nh); ++b) {
            const int y = (int)box_row(base, b, plan);
            for (int h = 0; h < L::NH; ++h)
              tma_load_2d(dst + h * L::HALF + b * brows * 128, &tmap_a, 32 * h, y, &bars->full[s]);
          }
        }
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    // ---- MMA issuer: per k-step one N = 2 KR product of Ahi with [Rhi | Rlo] and one
    // N = KR product of Alo with Rhi into the correction columns (whole warp loops, lane 0
    // issues)
    ok = __all_sync(0xffffffffu, mbar_wait(&bars->rbar, 0));
    const uint32_t b0 = smem_u32(smem + L::OFF_B);
    for (int j = 0; j < my_tiles && ok; ++j) {
      const int s = j % kStages, u = j / kStages, a = j & 1, v = j >> 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&bars->conv[s], (uint32_t)(u & 1)) &&
                                       mbar_wait(&bars->accfree[a], (uint32_t)((v & 1) ^ 1)));
      if (!ok) break;
      tc_fence_after();
      if (lane == 0) {
        const uint32_t a_hi = smem_u32(smem + L::OFF_A + s * L::TILE);
        const uint32_t acc = taddr + (uint32_t)(a * L::ACC_COLS);
#pragma unroll
        for (int ks = 0; ks < L::KR / 8; ++ks) {
          const uint32_t ao = (ks >> 2) * L::HALF + (ks & 3) * 32;
          const uint32_t bo = (ks >> 2) * L::BHALF + (ks & 3) * 32;
          mma_tf32(acc, desc_sw128(a_hi + ao), desc_sw128(b0 + bo), L::idesc(2 * L::KR), ks > 0 ? 1u : 0u);
        }
        if constexpr (TLO) {
          const uint32_t a_lo = taddr + (uint32_t)(L::ALO_COL + (j & 1) * L::KR);
#pragma unroll
          for (int ks = 0; ks < L::KR / 8; ++ks) {
            const uint32_t bo = (ks >> 2) * L::BHALF + (ks & 3) * 32;
            mma_tf32_ts(acc + L::KR, a_lo + (uint32_t)(8 * ks), desc_sw128(b0 + bo), L::idesc(L::KR), 1u);
          }
        } else {
          const uint32_t a_lo = smem_u32(smem + L::OFF_ALO + (j & 1) * L::TILE);
#pragma unroll
          for (int ks = 0; ks < L::KR / 8; ++ks) {
            const uint32_t ao = (ks >> 2) * L::HALF + (ks & 3) * 32;
            const uint32_t bo = (ks >> 2) * L::BHALF + (ks & 3) * 32;
            mma_tf32(acc + L::KR, desc_sw128(a_lo + ao), desc_sw128(b0 + bo), L::idesc(L::KR), 1u);
          }
        }
        mma_commit(&bars->mmad[a]);
        mma_commit(&bars->lofree[j & 1]);
      }
      __syncwarp();
    }
  } else if (warp < kEpiWarp0) {
    // ---- converters: Ahi = tf32(A) in place, Alo = A - Ahi, for every element of the tile
    const int ct = tid - 64;  // 0 .. 32 kConvWarps - 1
    float scale = 1.0f;
    if (plan.slots && plan.ref_slot >= 0) {
      const double prev = plan.slots[plan.prev_slot], ref = plan.slots[plan.ref_slot];
      if (prev > 0.0 && ref > 0.0) scale = (float)sqrt(ref / prev);
    }
    double nin = 0.0;
    for (int j = 0; j < my_tiles && ok; ++j) {
      const int s = j % kStages, u = j / kStages;
      ok = __all_sync(0xffffffffu, mbar_wait(&bars->full[s], (uint32_t)(u & 1)) &&
                                       mbar_wait(&bars->lofree[j & 1], (uint32_t)(((j >> 1) & 1) ^ 1)));
      if (!ok) break;
      float sq = 0.0f;
      if constexpr (TLO) {
        // thread = one tile row (tensor-memory lane); the two converter warps of a lane
        // quarter split the row's columns. Ahi goes back in place, Alo to tensor memory.
        constexpr int NV = L::KR / 2;  // columns per thread: 32 (k = 5) or 16 (k = 4)
        const int q = warp & 3, r = q * 32 + lane, part = (warp - 2) >> 2;
        unsigned char *row = smem + L::OFF_A + s * L::TILE + (part * NV / 32) * L::HALF + r * 128;
        // row phases (diagonal gates on row qubits) and the renormalisation, one factor
        float fr = scale, fi = 0.0f;
        if (plan.nterm > 0) {
          const unsigned long long base = tile_base_row(blockIdx.x + (long long)j * gridDim.x, plan);
          const float2 f = row_phase(plan, tile_turns(plan, base, lane), tile_row(base, r, plan));
          fr = f.x * scale;
          fi = f.y * scale;
        }
        float lo[NV];
#pragma unroll
        for (int g = 0; g < NV / 4; ++g) {
          const int chunk = (part * NV % 32) / 4 + g;  // 16-byte chunk within the 128-byte row
          float4 *p = reinterpret_cast<float4 *>(row + ((chunk ^ (r & 7)) << 4));
          float4 v = *p;
          sq = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, sq))));
          v = cmul2(v, fr, fi);
          float4 h;
          h.x = tf32_rna(v.x); h.y = tf32_rna(v.y); h.z = tf32_rna(v.z); h.w = tf32_rna(v.w);
          *p = h;
          lo[4 * g] = v.x - h.x; lo[4 * g + 1] = v.y - h.y; lo[4 * g + 2] = v.z - h.z; lo[4 * g + 3] = v.w - h.w;
        }
        tmem_st<NV>(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(L::ALO_COL + (j & 1) * L::KR + part * NV), lo);
        tmem_wait_st();
        tc_fence_before();
      } else {
        float4 *ah = reinterpret_cast<float4 *>(smem + L::OFF_A + s * L::TILE);
        float4 *al = reinterpret_cast<float4 *>(smem + L::OFF_ALO + (j & 1) * L::TILE);
        const unsigned long long base =
            plan.nterm > 0 ? tile_base_row(blockIdx.x + (long long)j * gridDim.x, plan) : 0ULL;
        const float t0 = plan.nterm > 0 ? tile_turns(plan, base, lane) : 0.0f;
#pragma unroll 4
        for (int i = ct; i < L::TILE / 16; i += 32 * kConvWarps) {
          float4 v = ah[i];
          sq = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, sq))));
          float fr = scale, fi = 0.0f;
          if (plan.nterm > 0) {  // chunk i lies in row (i / 8) mod 128 of its half
            const float2 f = row_phase(plan, t0, tile_row(base, (i >> 3) & 127, plan));
            fr = f.x * scale;
            fi = f.y * scale;
          }
          v = cmul2(v, fr, fi);
          float4 h, l;
          // the high part is written back explicitly, rounded to nearest: handing the raw
          // FP32 tile to the tensor core also works (it drops the low bits) but that
          // truncation biases the norm (-4.5e-7 per fused block against -3.0e-7 measured)
          h.x = tf32_rna(v.x); h.y = tf32_rna(v.y); h.z = tf32_rna(v.z); h.w = tf32_rna(v.w);
          ah[i] = h;
          l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
          al[i] = l;
        }
      }
      nin += (double)sq;
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->conv[s]);
    }
    if (plan.slots) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nin += __shfl_xor_sync(0xffffffffu, nin, o);
      if (lane == 0) atomicAdd(&plan.slots[plan.in_slot], nin);
    }
  } else {
    // ---- epilogue: out = main + correction (FP32, round to nearest) into the stage tile
    const int q = warp & 3;           // tensor-memory lane quarter of this warp
    const int r = q * 32 + lane;      // tile row
    const bool issuer = warp == kEpiWarp0 && lane == 0;
    double nout = 0.0;
    int prev_s = -1;  // stage of the previous tile, freed once its TMA store has read it
    int trow = 0;     // destination tile-index bits contributed by this thread's row
#pragma unroll
    for (int b = 0; b < 7; ++b)
      if ((r >> b) & 1) trow |= plan.wrow[b];
    // Destination of each float4 this thread stores (byte offset in the stage), the same
    // for every tile of the launch: pair = 1 (the identity plan included) stores columns
    // 2g and 2g + 1 of its own row side by side; pair = 2 (column bit 0 swaps with lane row
    // bit rho) stores the column pair 2g + b of rows r0 and r0 | 2^rho, b = bit rho of the
    // lane. pair = 0 computes single-complex destinations per tile.
    const int rho = plan.pair_row, pb = plan.pair == 2 ? (lane >> rho) & 1 : 0;
    const int trow0 = pb ? (trow & ~plan.wrow[rho]) : trow;  // destination bits of r0
    int offs[L::NH * 8];
#pragma unroll
    for (int x = 0; x < L::NH * 8; ++x) {
      const int d = plan.tcol[2 * x + pb] | trow0;
      const int r2 = d >> K, c2 = d & ((1 << K) - 1);
      offs[x] = (c2 >> 4) * L::HALF + r2 * 128 + ((((c2 >> 1) & 7) ^ (r2 & 7)) << 4);
    }
    for (int j = 0; j < my_tiles && ok; ++j) {
      const int a = j & 1, v = j >> 1, s = j % kStages;
      float sq = 0.0f;
      ok = __all_sync(0xffffffffu, mbar_wait(&bars->mmad[a], (uint32_t)(v & 1)));
      if (!ok) break;
      tc_fence_after();
      // the MMAs are done with the tile's stage: the output goes back into it
      unsigned char *out = smem + L::OFF_A + s * L::TILE;
      const uint32_t acc = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * L::ACC_COLS);
#pragma unroll
      for (int h = 0; h < L::NH; ++h) {
        float m[32], c[32];
        tmem_ld32(acc + (uint32_t)(32 * h), m);
        tmem_ld32(acc + (uint32_t)(L::KR + 32 * h), c);
        tmem_wait_ld();
        if (plan.pair == 1) {
          // column bit 0 stays in place: columns 2g and 2g + 1 land side by side
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float4 o = make_float4(m[4 * g] + c[4 * g], m[4 * g + 1] + c[4 * g + 1],
                                         m[4 * g + 2] + c[4 * g + 2], m[4 * g + 3] + c[4 * g + 3]);
            sq = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, sq))));
            *reinterpret_cast<float4 *>(out + offs[8 * h + g]) = o;
          }
        } else if (plan.pair == 2) {
          // rows r and r ^ 2^rho (lanes of this warp) fill the two halves of each
          // destination pair. The thread with bit rho clear keeps its even columns and
          // sends its odd ones, its partner the reverse; each then stores (row r0 value,
          // row r1 value) for its columns.
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float2 o0 = make_float2(m[4 * g] + c[4 * g], m[4 * g + 1] + c[4 * g + 1]);
            const float2 o1 = make_float2(m[4 * g + 2] + c[4 * g + 2], m[4 * g + 3] + c[4 * g + 3]);
            sq = fmaf(o0.x, o0.x, fmaf(o0.y, o0.y, fmaf(o1.x, o1.x, fmaf(o1.y, o1.y, sq))));
            const float2 snd = pb ? o0 : o1, kp = pb ? o1 : o0;
            float2 rcv;
            rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, 1 << rho);
            rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, 1 << rho);
            *reinterpret_cast<float4 *>(out + offs[8 * h + g]) = pb ? make_float4(rcv.x, rcv.y, kp.x, kp.y)
                                                                    : make_float4(kp.x, kp.y, rcv.x, rcv.y);
          }
        } else {
          // the value of (row r, column cc) goes to tile index tcol[cc] | trow; the row's and
          // the column's bits are disjoint, so the byte offset splits into a part of the
          // thread (base_t, xt) and a part of the column (ubase, xu, from the host)
          const int rr = trow >> K, rc = trow & ((1 << K) - 1);
          const int base_t = (rc >> 4) * L::HALF + rr * 128 + (rc & 1) * 8;
          const int xt = ((rc >> 1) & 7) ^ (rr & 7);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int cc = 16 * h + e;
            const int off = base_t + plan.ubase[cc] + ((xt ^ (int)plan.xu[cc]) << 4);
            const float2 o = make_float2(m[2 * e] + c[2 * e], m[2 * e + 1] + c[2 * e + 1]);
            sq = fmaf(o.x, o.x, fmaf(o.y, o.y, sq));
            *reinterpret_cast<float2 *>(out + off) = o;
          }
        }
      }
      nout += (double)sq;
      tc_fence_before();
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->accfree[a]);
        mbar_arrive(&bars->stg);
      }
      // every epilogue warp waits for the whole output tile (a permuted tile mixes rows of
      // all four warps; the wait also keeps the four in step on the barrier's phases)
      ok = __all_sync(0xffffffffu, mbar_wait(&bars->stg, (uint32_t)(j & 1)));
      if (!ok) break;
      if (issuer) {
        const unsigned long long base = tile_base_row(blockIdx.x + (long long)j * gridDim.x, plan);
        const int brows = 1 << plan.c;
        if (mdim > 0) {
          for (int g = 0; g < (1 << (plan.nh - mdim)); ++g) {
            const int y = (int)group_row(base, g, mdim, plan);
            for (int h = 0; h < L::NH; ++h)
              tma_store_md(mdim, &tmap_a, 32 * h, y, out + h * L::HALF + (g << mdim) * brows * 128);
          }
        } else {
          for (int b = 0; b < (1 << plan.nh); ++b) {
            const int y = (int)box_row(base, b, plan);
            for (int h = 0; h < L::NH; ++h) tma_store_2d(&tmap_a, 32 * h, y, out + h * L::HALF + b * brows * 128);
          }
        }
        bulk_commit();
        // the previous tile's store has read its stage: hand that stage back to the producer
        bulk_wait_read1();
        if (prev_s >= 0) mbar_arrive(&bars->sfree[prev_s]);
      }
      prev_s = s;
      __syncwarp();
    }
    if (plan.slots) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nout += __shfl_xor_sync(0xffffffffu, nout, o);
      if (lane == 0) atomicAdd(&plan.slots[plan.out_slot], nout);
    }
    if (issuer) bulk_wait0();
  }

  __syncwarp();
  if (!ok && lane == 0) atomicExch(&g_tc_timeout, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
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

// Tensor map of rank 2 + md over the state rows: (row floats, rows, then one size-2
// dimension per high row bit hbit[0 .. md-1] with a stride of 2^hbit rows), boxes of
// 32 floats x box_rows rows x 2 x ... x 2, 128-byte swizzle. The copy of one box fills
// consecutive 128-byte rows in shared memory in the order of the 2-D box loop.
qsim_status make_map_md(CUtensorMap *m, const void *base, int row_floats, unsigned long long rows, int box_rows,
                        const int *hbit, int md) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return QSIM_EUNSUPPORTED;
  }
  cuuint64_t dims[5] = {(cuuint64_t)row_floats, (cuuint64_t)rows, 2, 2, 2};
  cuuint64_t strides[4] = {(cuuint64_t)row_floats * 4, 0, 0, 0};
  cuuint32_t box[5] = {32, (cuuint32_t)box_rows, 2, 2, 2};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  for (int j = 0; j < md; ++j) strides[1 + j] = ((cuuint64_t)1 << hbit[j]) * (cuuint64_t)row_floats * 4;
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)(2 + md), const_cast<void *>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (rank %d) failed (%d)", 2 + md, (int)r);
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

template <int K, bool TLO>
qsim_status launch_k(const StateDev &s, const void *rmats, const TcTilePlan &plan, int64_t *bytes) {
  using L = TcLayout<K, TLO>;
  // the shared-memory attribute is set once per device, on first use there
  static std::atomic<unsigned long long> attr_done{0};
  QS_TRY(smem_attr_once(k_fused_tc<K, TLO>, L::BYTES + 1024, attr_done));
  CUtensorMap ma, mr;
  const unsigned long long rows = 1ULL << (s.n - K);
  // tiles with high row bits: one copy per half covers up to three of them
  int mdim = plan.nh < 3 ? plan.nh : 3;
  if (mdim > 0 && make_map_md(&ma, s.amps, L::KR, rows, 1 << plan.c, plan.hbit, mdim) != QSIM_OK) mdim = 0;
  if (mdim == 0 && plan.c < 3) {
    // 2-D boxes of 4 rows would start copies 512 bytes apart; the 128-byte swizzle
    // wants 1024-byte aligned destinations
    set_error("fused tile plan with a low run of %d rows needs a rank-5 tensor map", 1 << plan.c);
    return QSIM_EUNSUPPORTED;
  }
  if (mdim == 0) QS_TRY(make_map(&ma, s.amps, L::KR, rows, 1 << plan.c));
  QS_TRY(make_map(&mr, rmats, L::KR, L::BROWS, L::BROWS));
  const int ntiles = (int)(rows / 128);
  int grid = num_sms() * L::CTAS_PER_SM;
  if (grid > ntiles) grid = ntiles;
  if (bytes) *bytes += 2LL * 8 * (1LL << s.n);
  k_fused_tc<K, TLO><<<grid, kTcWarps * 32, L::BYTES + 1024, s.stream>>>(ma, mr, ntiles, mdim, plan);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

}  // namespace

bool fused_tc_supported(const StateDev &s, int k) {
  // 128-row tiles, row indices that fit a signed 32-bit TMA coordinate, and a driver with
  // tensor maps
  return s.dtype == QSIM_C64 && (k == 4 || k == 5) && s.n >= k + 7 && s.n - k <= 31 &&
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

void tc_identity_plan(int k, TcTilePlan &p) {
  memset(&p, 0, sizeof(p));
  p.c = 7;
  p.nh = 0;
  p.ins_n = 7;
  for (int b = 0; b < 7; ++b) p.ins[b] = b;
  p.ident = 1;
  p.pair = 1;
  for (int c = 0; c < (1 << k); ++c) p.tcol[c] = c;
  for (int b = 0; b < 7; ++b) p.wrow[b] = 1 << (k + b);
  p.slots = nullptr;
  p.in_slot = p.out_slot = p.ref_slot = p.prev_slot = -1;
}

bool tc_plan_valid(int n, int k, const TcTilePlan &p) {
  const int rbits = n - k;  // row-index bits
  if (p.c < 2 || p.c > 7 || p.nh != 7 - p.c || p.ins_n != 7) return false;
  int prev = p.c - 1;
  for (int j = 0; j < p.nh; ++j) {
    if (p.hbit[j] <= prev || p.hbit[j] >= rbits) return false;
    prev = p.hbit[j];
  }
  int seen = 0;
  for (int t = 0; t < k + 7; ++t) {  // destinations form a permutation of the tile bits
    const int d = t < k ? p.tcol[1 << t] : p.wrow[t - k];
    if (__builtin_popcount((unsigned)d) != 1 || d >= (1 << (k + 7)) || (seen & d)) return false;
    seen |= d;
  }
  for (int cc = 0; cc < (1 << k); ++cc) {  // the column table is the bit permutation
    int d = 0;
    for (int t = 0; t < k; ++t)
      if ((cc >> t) & 1) d |= p.tcol[1 << t];
    if (p.tcol[cc] != d) return false;
  }
  if (p.ident && !(p.tcol[1] == 1 && p.wrow[0] == (1 << k))) return false;
  if (p.pair == 1 && p.tcol[1] != 1) return false;
  if (p.pair == 2 && (p.pair_row < 0 || p.pair_row > 4 || p.tcol[1] != (1 << (k + p.pair_row)) ||
                      p.wrow[p.pair_row] != 1))
    return false;
  if (p.pair < 0 || p.pair > 2) return false;
  return true;
}

qsim_status launch_fused_tc(const StateDev &s, int k, const void *dev_rmats, const TcTilePlan &plan,
                            int64_t *bytes) {
  if (!tc_plan_valid(s.n, k, plan)) {
    set_error("fused tile plan is not valid for n = %d, k = %d", s.n, k);
    return QSIM_EINVAL;
  }
  if (!fused_tc_supported(s, k)) {
    set_error("tensor-core fused apply needs complex64, k in {4, 5} and n >= k + 7");
    return QSIM_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(dev_rmats) & 127u) {
    set_error("fused operand buffer must be 128-byte aligned");
    return QSIM_EINVAL;
  }
  // the column part of the single-complex store offsets (see the epilogue): destination
  // tile index d = tcol[cc] | (row part); row bits r2 = d >> k, column bits c2 = d & (2^k - 1)
  TcTilePlan p = plan;
  // row-phase terms that read a tile row bit first (the rest are one sum per tile)
  {
    unsigned long long tile_rows = 0;
    for (int j = 0; j < plan.ins_n; ++j) tile_rows |= 1ULL << plan.ins[j];
    int nv = 0;
    p.nvary = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int g = 0; g < plan.nterm; ++g) {
        const bool vary = (plan.term[g].mask & tile_rows) != 0;
        if (vary == (pass == 0)) p.term[nv++] = plan.term[g];
        if (pass == 0 && vary) p.nvary = nv;
      }
  }
  for (int cc = 0; cc < (1 << k); ++cc) {
    const int tc = plan.tcol[cc], c2 = tc & ((1 << k) - 1), r2 = tc >> k;
    p.ubase[cc] = (c2 >> 4) * (128 * 128) + r2 * 128 + (c2 & 1) * 8;
    p.xu[cc] = (unsigned char)(((c2 >> 1) & 7) ^ (r2 & 7));
  }
  if (s.tc_lo_smem)
    return k == 5 ? launch_k<5, false>(s, dev_rmats, p, bytes) : launch_k<4, false>(s, dev_rmats, p, bytes);
  return k == 5 ? launch_k<5, true>(s, dev_rmats, p, bytes) : launch_k<4, true>(s, dev_rmats, p, bytes);
}

qsim_status tc_wait_selftest(int ms, cudaStream_t st) {
  k_wait_selftest<<<1, 64, 0, st>>>((unsigned long long)ms * 1000000ULL);
  QS_TRY_CUDA(cudaGetLastError());
  QS_TRY_CUDA(cudaStreamSynchronize(st));
  return tc_take_timeout();
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
