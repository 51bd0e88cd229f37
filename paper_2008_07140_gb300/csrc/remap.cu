// Qubit remap: permute physical qubit positions in one in-place sweep.
//
// A tile is the set of amplitudes that agree on every index bit outside the tile qubits
// {0, ..., L-1} (a run of 2^L contiguous amplitudes, 256 bytes) plus up to 6 higher qubits
// hi[0..m). Any permutation of the tile qubits maps every tile onto itself, so each block
// loads a tile into shared memory run by run (coalesced) and writes it back permuted, run
// by run. The planner uses it to swap high qubits into the low positions where the fused
// tensor-core kernel wants them; read-outs use it to restore the logical order.
#include "internal.h"

namespace qsim {

namespace {

constexpr int kThreads = 256;

struct TileDesc {
  int L;
  int m;
  int hi[8];       // ascending, all >= L
  int src_bit[16]; // new tile bit b takes the old tile bit src_bit[b]
  Ins ins;         // zero insertion at the hi positions
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned long long tile_base(long long t, const TileDesc &d) {
  unsigned long long g = (unsigned long long)t << d.L;
#pragma unroll 1
  for (int k = 0; k < d.ins.n; ++k) {
    const unsigned long long low = g & ((1ULL << d.ins.pos[k]) - 1ULL);
    g = ((g ^ low) << 1) | low;
  }
  return g;
}

// Source tile index of destination tile index e: OR of lo[e & 63] and hi[e >> 6] (the bit
// permutation splits over disjoint bit groups). Global offset of tile index e relative to
// the tile base: (e & (2^L - 1)) + off[e >> L]. Two shared-memory buffers: the next tile
// streams in (cp.async) while the current one is written back permuted.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_permute_tiles(T *__restrict__ psi, long long tiles, TileDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned short tlo[64], thi[64];
  __shared__ unsigned long long toff[64];
  const int bits = d.L + d.m;
  const int tsize = 1 << bits;
  T *const buf0 = reinterpret_cast<T *>(smem_raw);
  constexpr int CH = 16 / sizeof(T);  // amplitudes per 16-byte chunk
  if (threadIdx.x < 64) {
    const int e = threadIdx.x;
    int lo = 0, hi = 0;
    for (int b = 0; b < bits; ++b) {
      if (b < 6 && ((e >> b) & 1)) lo |= 1 << d.src_bit[b];
      if (b >= 6 && ((e >> (b - 6)) & 1)) hi |= 1 << d.src_bit[b];
    }
    tlo[e] = (unsigned short)lo;
    thi[e] = (unsigned short)hi;
    unsigned long long o = 0;
    for (int j = 0; j < d.m; ++j)
      if ((e >> j) & 1) o |= 1ULL << d.hi[j];
    toff[e] = o;
  }
  __syncthreads();
  const int runmask = (1 << d.L) - 1;
  // Shared-memory position of tile element e: the 16-byte chunks of each run are rotated by
  // the run index (XOR), so that a gather of elements that share their low bits and differ
  // in high bits - the usual remap - spreads over the banks instead of hitting one.
  const int rchunks = (1 << d.L) / CH;  // chunks per run (a power of two)
  auto spos = [&](int e) {
    const int run = e >> d.L, ch = (e & runmask) / CH;
    return ((run * rchunks) + (ch ^ (run & (rchunks - 1)))) * CH + (e & (CH - 1));
  };
  auto load = [&](long long t, T *dst) {
    const unsigned long long g = tile_base(t, d);
    for (int c = threadIdx.x; c < tsize / CH; c += blockDim.x) {
      const int e = c * CH;
      cp_async16(&dst[spos(e)], &psi[g + (unsigned long long)(e & runmask) + toff[e >> d.L]]);
    }
    cp_async_commit();
  };
  long long t = blockIdx.x;
  if (t < tiles) load(t, buf0);
  for (int i = 0; t < tiles; t += gridDim.x, ++i) {
    const long long tn = t + gridDim.x;
    T *cur = buf0 + (i & 1) * tsize;
    if (tn < tiles) {
      load(tn, buf0 + ((i + 1) & 1) * tsize);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const unsigned long long g = tile_base(t, d);
    for (int c = threadIdx.x; c < tsize / CH; c += blockDim.x) {
      const int e = c * CH;
      T v[CH];
#pragma unroll
      for (int k = 0; k < CH; ++k) v[k] = cur[spos(tlo[(e + k) & 63] | thi[(e + k) >> 6])];
      *reinterpret_cast<float4 *>(&psi[g + (unsigned long long)(e & runmask) + toff[e >> d.L]]) =
          *reinterpret_cast<const float4 *>(v);
    }
    // the buffer just read is the target of the load issued at the top of the next pass
    __syncthreads();
  }
}

}  // namespace

int remap_low_run(int n, int dtype, int m) {
  int L = dtype == QSIM_C128 ? 4 : 5;
  if (L > n - m) L = n - m;
  return L;
}

// Tile qubits: positions 0..L-1 then hi[0..m) (any order given; sorted here). dst_of[b]
// (b indexes that list) is the tile position the content of tile position b moves to.
qsim_status launch_permute(const StateDev &s, int L, const int *hi_in, int m, const int *dst_of_in,
                           int64_t *bytes) {
  // 16-byte chunks need runs of at least 2 complex64 / 1 complex128 amplitudes
  if (m < 0 || m > 6 || L < 1 || L > 5 || L + m > s.n) {
    set_error("remap tile with low run %d and %d high qubits (n = %d)", L, m, s.n);
    return QSIM_EINVAL;
  }
  // sort the high qubits, carrying the tile-position mapping along
  int order[8];
  for (int j = 0; j < m; ++j) order[j] = j;
  for (int a = 0; a < m; ++a)
    for (int b = a + 1; b < m; ++b)
      if (hi_in[order[b]] < hi_in[order[a]]) {
        const int t = order[a];
        order[a] = order[b];
        order[b] = t;
      }
  int hs[8];
  for (int j = 0; j < m; ++j) {
    hs[j] = hi_in[order[j]];
    if (hs[j] < L || hs[j] >= s.n || (j > 0 && hs[j] == hs[j - 1])) {
      set_error("remap high qubit %d invalid (low run %d, n %d)", hs[j], L, s.n);
      return QSIM_EINVAL;
    }
  }
  // The contiguous run grows by identity bits up to 2^11 (complex64) or 2^10 (complex128)
  // amplitudes per tile, below the lowest high qubit: more work per block, longer runs.
  const int budget = s.dtype == QSIM_C128 ? 10 : 11;
  int Lx = budget - m;
  if (m > 0 && Lx > hs[0]) Lx = hs[0];
  if (Lx > s.n - m) Lx = s.n - m;
  if (Lx < L) Lx = L;
  TileDesc d;
  d.L = Lx;
  d.m = m;
  const int bits = Lx + m;
  int old_to_new_pos[16];  // tile position in the caller's list -> position in the widened tile
  for (int b = 0; b < L; ++b) old_to_new_pos[b] = b;
  for (int j = 0; j < m; ++j) old_to_new_pos[L + order[j]] = Lx + j;
  for (int j = 0; j < m; ++j) d.hi[j] = hs[j];
  // dst in widened coordinates (the added run bits stay in place), then invert into src_bit
  int dst[16], seen = 0;
  for (int b = 0; b < bits; ++b) dst[b] = b;
  for (int b = 0; b < L + m; ++b) {
    const int v = dst_of_in[b];
    if (v < 0 || v >= L + m || (seen >> v & 1)) {
      set_error("remap destination list is not a permutation");
      return QSIM_EINVAL;
    }
    seen |= 1 << v;
    dst[old_to_new_pos[b]] = old_to_new_pos[v];
  }
  for (int b = 0; b < bits; ++b) d.src_bit[dst[b]] = b;
  d.ins.n = m;
  d.ins.set = 0;
  for (int j = 0; j < m; ++j) d.ins.pos[j] = d.hi[j];
  const long long tiles = 1LL << (s.n - bits);
  long long grid = 8LL * num_sms();
  if (grid > tiles) grid = tiles;
  const size_t B = s.dtype == QSIM_C128 ? 16 : 8;
  const size_t sh = 2 * ((size_t)1 << bits) * B;  // two tile buffers, at most 64 KB
  static std::atomic<unsigned long long> attr_c128{0}, attr_c64{0};
  QS_TRY(smem_attr_once(k_permute_tiles<double2>, 64 << 10, attr_c128));
  QS_TRY(smem_attr_once(k_permute_tiles<float2>, 64 << 10, attr_c64));
  if (bytes) *bytes += 2LL * (int64_t)B * (1LL << s.n);
  if (s.dtype == QSIM_C128)
    k_permute_tiles<double2><<<(int)grid, kThreads, sh, s.stream>>>(static_cast<double2 *>(s.amps), tiles, d);
  else
    k_permute_tiles<float2><<<(int)grid, kThreads, sh, s.stream>>>(static_cast<float2 *>(s.amps), tiles, d);
  QS_TRY_CUDA(cudaGetLastError());
  return QSIM_OK;
}

}  // namespace qsim
