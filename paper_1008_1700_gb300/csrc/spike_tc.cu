// Tensor-core (tcgen05) version of the four spike GEMM ops of spike.cu for
// FP32 factors: the products of Fig. 2 step 4 run with bf16 operands and
// fp32 accumulation in tensor memory.  With three passes each operand is
// split into a bf16 high part and a bf16 remainder, and the product is
// hi*hi + hi*lo + lo*hi (about 16 correct bits); one pass uses hi*hi only.
//
// The A operands (blocks of the fronts: L11^-1, L21, U12, U11^-1) are packed
// once per factorisation (k_tc_pack_a) into bf16 tiles of 128 rows x 32
// K-columns in the K-major no-swizzle canonical layout of the tensor cores
// (8 x 16-byte core matrices; K-adjacent core matrices 128 B apart,
// M-adjacent ones 512 B apart), high part then remainder, so that one
// stage's A is one contiguous block.  One CTA computes one 128 x 128 tile of
// C: thread 0 streams the packed A blocks into shared memory with 1-D TMA
// bulk copies (mbarrier with a transaction count), while the 256 threads
// convert the B tile (panel rows, fp32) into the same layout; thread 0 then
// issues tcgen05.mma and commits the stage to a second mbarrier, on which the
// loaders wait before they overwrite that stage (two stages).  The
// accumulator (128 lanes x 128 fp32 columns of tensor memory) is read back
// with tcgen05.ld for the epilogue.  Every wait is bounded; a wait that runs
// out records error code 2 in the kernel's error record.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "launch.h"

namespace ddps {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_TILE_BYTES = TC_BM * TC_BK * 2;  // one bf16 operand tile (8 KB)
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: kind::f16, D fp32, A and B bf16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                            ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// Bounded wait on an mbarrier phase; gives up early once any CTA has recorded
// a timeout in err[0], so that a failure costs one wait, not one per CTA.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          const volatile long long* err,
                                          uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if ((it & 1023u) == 1023u && err[0] == 2) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(h);
  const __nv_bfloat16 l = __float2bfloat16_rn(r);
  hi = *reinterpret_cast<const uint16_t*>(&h);
  lo = *reinterpret_cast<const uint16_t*>(&l);
}

// Byte offset of the 16-byte chunk (row, k-chunk kc) in a K-major tile.
constexpr uint32_t kSBO = (TC_BK / 8) * 128;  // bytes between M/N-adjacent core matrices
__device__ __forceinline__ uint32_t chunk_off(int row, int kc) {
  return (uint32_t)((row >> 3) * kSBO + kc * 128 + (row & 7) * 16);
}


__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Tensor copies (TMA) of panel rows through a tensor map over a row-major
// fp32 panel (NR columns): a tile of box rows x 128 columns at (x, y), and
// four single rows y0..y3 (a map with one-row boxes) placed one after another.
__device__ __forceinline__ void tma_tile_2d(uint32_t dst, const CUtensorMap* map, int32_t x,
                                            int32_t y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
      "[%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int32_t x,
                                            int32_t y0, int32_t y1, int32_t y2, int32_t y3,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void store_split(unsigned char* hi_dst, unsigned char* lo_dst,
                                            const float* v, bool with_lo) {
  uint16_t hi[8], lo[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) split_bf16(v[t], hi[t], lo[t]);
  *reinterpret_cast<uint4*>(hi_dst) =
      make_uint4(hi[0] | ((uint32_t)hi[1] << 16), hi[2] | ((uint32_t)hi[3] << 16),
                 hi[4] | ((uint32_t)hi[5] << 16), hi[6] | ((uint32_t)hi[7] << 16));
  if (with_lo)
    *reinterpret_cast<uint4*>(lo_dst) =
        make_uint4(lo[0] | ((uint32_t)lo[1] << 16), lo[2] | ((uint32_t)lo[3] << 16),
                   lo[4] | ((uint32_t)lo[5] << 16), lo[6] | ((uint32_t)lo[7] << 16));
}

// Eight consecutive values -> bf16 high parts (16 bytes) and remainders,
// two values per conversion instruction; bitwise equal to store_split.
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo_elem, float hi_elem) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}
__device__ __forceinline__ void store_split_x2(unsigned char* hi_dst, unsigned char* lo_dst,
                                               const float* v, bool with_lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    h[t] = cvt_bf16x2(v[2 * t], v[2 * t + 1]);
    const float r0 = v[2 * t] - __uint_as_float(h[t] << 16);
    const float r1 = v[2 * t + 1] - __uint_as_float(h[t] & 0xffff0000u);
    l[t] = cvt_bf16x2(r0, r1);
  }
  *reinterpret_cast<uint4*>(hi_dst) = make_uint4(h[0], h[1], h[2], h[3]);
  if (with_lo) *reinterpret_cast<uint4*>(lo_dst) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Dimensions of one op for front f: M rows of C, K, and the origin of A in the front.
struct OpDims {
  int M, K, a_r0, a_c0;
};
template <int OP>
__device__ __forceinline__ OpDims op_dims(int32_t k, int32_t r) {
  return OpDims{OP == OP_FWD_L21 ? r : k, OP == OP_BWD_U12 ? r : k, OP == OP_FWD_L21 ? k : 0,
                OP == OP_BWD_U12 ? k : 0};
}

template <int OP>
__device__ __forceinline__ float a_entry(const float* __restrict__ A, int32_t m, OpDims d, int gi,
                                         int gk) {
  if (gi >= d.M || gk >= d.K) return 0.f;
  if (OP == OP_FWD_LINV) return gi > gk ? A[gi + (int64_t)gk * m] : (gi == gk ? 1.f : 0.f);
  if (OP == OP_BWD_UINV) return gi <= gk ? A[gi + (int64_t)gk * m] : 0.f;
  return A[(d.a_r0 + gi) + (int64_t)(d.a_c0 + gk) * m];
}

// Packs the A operand of one (tile, K-block): 128 rows x 32 K-columns, bf16
// high part then (three passes) the remainder.
template <int OP, int PASSES>
__global__ void __launch_bounds__(TC_THREADS)
    k_tc_pack_a(DevFronts F, const int32_t* __restrict__ tile_front,
                const int32_t* __restrict__ tile_m0, const int64_t* __restrict__ tile_aoff,
                const float* __restrict__ arena, unsigned char* __restrict__ atc) {
  constexpr uint32_t kAB = (PASSES == 3 ? 2u : 1u) * TC_TILE_BYTES;
  const int32_t f = tile_front[blockIdx.x];
  const int32_t m0 = tile_m0[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const OpDims d = op_dims<OP>(k, m - k);
  const int kt = blockIdx.y;
  if (kt * TC_BK >= d.K) return;
  const float* __restrict__ A = arena + F.arena[f];
  unsigned char* dst = atc + tile_aoff[blockIdx.x] + (int64_t)kt * kAB;
#pragma unroll
  for (int q = 0; q < (TC_BM * TC_BK / 8) / TC_THREADS; ++q) {
    const int e = threadIdx.x + q * TC_THREADS;
    const int row = e % TC_BM, kc = e / TC_BM;
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = a_entry<OP>(A, m, d, m0 + row, kt * TC_BK + kc * 8 + t);
    const uint32_t off = chunk_off(row, kc);
    store_split(dst + off, dst + TC_TILE_BYTES + off, v, PASSES == 3);
  }
}

template <int OP, int PASSES>
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_spike_gemm_tc(DevFronts F, const int32_t* __restrict__ tile_front,
                    const int32_t* __restrict__ tile_m0, const int64_t* __restrict__ tile_aoff,
                    const unsigned char* __restrict__ atc, const int64_t* __restrict__ block_ncols,
                    int64_t j0, int32_t NR, float* __restrict__ X, float* __restrict__ Tb,
                    long long* __restrict__ err, int inject_wait) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ __align__(8) uint64_t empty[2];
  __shared__ __align__(8) uint64_t never;  // only for inject_wait: nothing arrives here
  __shared__ uint32_t tmem_slot;
  constexpr uint32_t kAB = (PASSES == 3 ? 2u : 1u) * TC_TILE_BYTES;  // A (or B) bytes per stage
  constexpr uint32_t kStageBytes = 2 * kAB;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t f = tile_front[blockIdx.x];
  const int32_t m0 = tile_m0[blockIdx.x];
  const int n0 = blockIdx.y * TC_BN;
  const int64_t ncols = min((int64_t)NR, block_ncols[F.block[f]] - j0);
  if (n0 >= ncols) return;  // uniform over the CTA, before any tcgen05 work
  const int32_t k = F.k[f], m = F.m[f];
  const OpDims d = op_dims<OP>(k, m - k);
  const int64_t row0 = F.row0[f];
  const int64_t tb0 = F.idx_off[f];
  const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
  const unsigned char* apk = atc + tile_aoff[blockIdx.x];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((uint32_t)TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&never)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  bool timed_out = false;

  int nk = (d.K + TC_BK - 1) / TC_BK;
  // B (panel rows, fp32) of one stage: each thread holds kBItems runs of 8
  // K-consecutive values of one column in registers, loaded one stage ahead
  constexpr int kBItems = (TC_BN * TC_BK / 8) / TC_THREADS;
  float breg[kBItems][8];
  const float* Bp = (OP == OP_FWD_L21 || OP == OP_BWD_U12) ? X : Tb;
  auto load_b = [&](int kt) {
    const int k0 = kt * TC_BK;
#pragma unroll
    for (int q = 0; q < kBItems; ++q) {
      const int e = tid + q * TC_THREADS;
      const int col = e % TC_BN, kc = e / TC_BN;
      const int gj = n0 + col;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int gk = k0 + kc * 8 + t;
        float val = 0.f;
        if (gk < d.K && gj < ncols) {
          int64_t brow;
          if (OP == OP_FWD_LINV || OP == OP_BWD_UINV)
            brow = tb0 + gk;
          else if (OP == OP_FWD_L21)
            brow = row0 + gk;
          else
            brow = idx[k + gk];
          val = Bp[brow * NR + gj];
        }
        breg[q][t] = val;
      }
    }
  };
  if (inject_wait) {  // failure-path test: a short bounded wait that must run out
    timed_out = !mbar_wait(smem_u32(&never), 0, err, 4096u);
    if (timed_out) nk = 0;  // no tensor work: the epilogue writes C_in only
  }
  if (nk > 0) load_b(0);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt >= 2 && !timed_out)
      timed_out = !mbar_wait(smem_u32(&empty[st]), ((kt - 2) >> 1) & 1, err);
    const uint32_t aS = sbase + st * kStageBytes;
    if (tid == 0) {
      mbar_expect_tx(smem_u32(&full[st]), kAB);
      bulk_g2s(aS, apk + (int64_t)kt * kAB, kAB, smem_u32(&full[st]));
    }
    // convert the B tile loaded during the previous stage, then start loading the next one
    unsigned char* sB = smem + st * kStageBytes + kAB;
#pragma unroll
    for (int q = 0; q < kBItems; ++q) {
      const int e = tid + q * TC_THREADS;
      const uint32_t off = chunk_off(e % TC_BN, e / TC_BN);
      store_split(sB + off, sB + TC_TILE_BYTES + off, breg[q], PASSES == 3);
    }
    if (kt + 1 < nk) load_b(kt + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!timed_out) timed_out = !mbar_wait(smem_u32(&full[st]), (kt >> 1) & 1, err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aLo = aS + TC_TILE_BYTES;
      const uint32_t bS = aS + kAB;
      const uint32_t bLo = bS + TC_TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint32_t ko = kk * 256;  // two K-adjacent core matrices per K = 16
        const uint32_t acc0 = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, make_desc(aS + ko, 128, kSBO), make_desc(bS + ko, 128, kSBO), acc0);
        if (PASSES == 3) {
          mma_bf16(tmem, make_desc(aS + ko, 128, kSBO), make_desc(bLo + ko, 128, kSBO), 1u);
          mma_bf16(tmem, make_desc(aLo + ko, 128, kSBO), make_desc(bS + ko, 128, kSBO), 1u);
        }
      }
      mma_commit(smem_u32(&empty[st]));
    }
  }
  if (nk > 0 && !timed_out)
    timed_out = !mbar_wait(smem_u32(&empty[(nk - 1) & 1]), ((nk - 1) >> 1) & 1, err);
  if (timed_out && lane == 0) atomicCAS((unsigned long long*)&err[0], 0ull, 2ull);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w reads lanes 32*(w%4).. (rows) and columns 64*(w/4)..+64
  const int quarter = warp & 3, half = warp >> 2;
  const int gi = m0 + quarter * 32 + lane;
  float* out = nullptr;
  const float* cin = nullptr;
  if (gi < d.M) {
    if (OP == OP_FWD_LINV || OP == OP_BWD_UINV) {
      out = X + (row0 + gi) * NR;
    } else if (OP == OP_FWD_L21) {
      out = Tb + (tb0 + k + gi) * NR;
      cin = out;
    } else {
      out = Tb + (tb0 + gi) * NR;
      cin = X + (row0 + gi) * NR;
    }
  }
#pragma unroll
  for (int c = 0; c < 64; c += 16) {
    uint32_t rv[16];
    if (nk > 0) {
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64 + c);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(rv[0]), "=r"(rv[1]), "=r"(rv[2]), "=r"(rv[3]), "=r"(rv[4]), "=r"(rv[5]),
            "=r"(rv[6]), "=r"(rv[7]), "=r"(rv[8]), "=r"(rv[9]), "=r"(rv[10]), "=r"(rv[11]),
            "=r"(rv[12]), "=r"(rv[13]), "=r"(rv[14]), "=r"(rv[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) rv[t] = 0u;
    }
    if (out) {
      const int gj0 = n0 + half * 64 + c;
      if (gj0 + 16 <= ncols) {  // full 16-column run: four 16-byte stores
#pragma unroll
        for (int t = 0; t < 16; t += 4) {
          float4 a = make_float4(__uint_as_float(rv[t]), __uint_as_float(rv[t + 1]),
                                 __uint_as_float(rv[t + 2]), __uint_as_float(rv[t + 3]));
          if (cin) {
            const float4 cv = *reinterpret_cast<const float4*>(cin + gj0 + t);
            a = make_float4(cv.x - a.x, cv.y - a.y, cv.z - a.z, cv.w - a.w);
          }
          *reinterpret_cast<float4*>(out + gj0 + t) = a;
        }
      } else {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int gj = gj0 + t;
          if (gj < ncols) {
            const float a = __uint_as_float(rv[t]);
            out[gj] = cin ? cin[gj] - a : a;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TC_BN));
}

// ---------------------------------------------------------------------------
// Block LU trailing update on the tensor cores.  The multi-CTA LU of a large
// front runs its 32-column panels in blocks of 256 pivots: within a block the
// rank-32 updates touch only the block's columns and rows (k_lu_trailing
// with its mask), and when the block ends, this kernel applies the whole
// block at once to the rest of the front,
//   A[Jend:m, Jend:m] -= L[Jend:m, J:Jend] * U[J:Jend, Jend:m],
// J = j0 rounded down to 256, Jend = min(J + 256, k).  One CTA per 128 x 128
// tile of the region (tile word (ti << 16) | tj): the 256 threads load the
// L and U chunks of 32 pivots (fp32, coalesced), split them into bf16 high
// parts and remainders in the K-major layout, thread 0 issues hi*hi + hi*lo
// + lo*hi per 16 pivots into a 128 x 128 fp32 accumulator in tensor memory
// (two stages; the next chunk is loaded into registers meanwhile), and the
// epilogue subtracts the accumulator from the tile.  Waits are bounded.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_lu_update_tc(DevFronts F, const int32_t* __restrict__ tile_front,
                   const int32_t* __restrict__ tile_ij, int32_t j0, float* __restrict__ arena,
                   long long* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t empty[2];
  __shared__ uint32_t tmem_slot;
  constexpr uint32_t kAB = 2u * TC_TILE_BYTES;  // one operand, high part then remainder
  constexpr uint32_t kStageBytes = 2 * kAB;
  constexpr int kItems = (TC_BM * TC_BK / 8) / TC_THREADS;  // runs of 8 per thread and operand

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t f = tile_front[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const int32_t J = j0 & ~(kLuTcBlock - 1);
  const int32_t Jend = min(J + kLuTcBlock, k);
  const int32_t K = Jend - J;
  const int32_t i0 = Jend + (tile_ij[blockIdx.x] >> 16) * TC_BM;
  const int32_t c0 = Jend + (tile_ij[blockIdx.x] & 0xffff) * TC_BN;
  float* __restrict__ A = arena + F.arena[f];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((uint32_t)TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  bool timed_out = false;

  const int nk = (K + TC_BK - 1) / TC_BK;
  float areg[kItems][8], breg[kItems][8];
  auto load = [&](int kt) {
    const int p0 = J + kt * TC_BK;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const int e = tid + q * TC_THREADS;
      // L: rows on the lanes, 8 pivots of one row per run
      const int row = e % TC_BM, kc = e / TC_BM;
      const int gi = i0 + row;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int p = p0 + kc * 8 + t;
        areg[q][t] = (gi < m && p < Jend) ? A[gi + (int64_t)p * m] : 0.f;
      }
      // U: 8 consecutive pivots (contiguous) of one column per run
      const int col = e / (TC_BK / 8), kc2 = e % (TC_BK / 8);
      const int gc = c0 + col;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int p = p0 + kc2 * 8 + t;
        breg[q][t] = (gc < m && p < Jend) ? A[p + (int64_t)gc * m] : 0.f;
      }
    }
  };
  if (nk > 0) load(0);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt >= 2 && !timed_out)
      timed_out = !mbar_wait(smem_u32(&empty[st]), ((kt - 2) >> 1) & 1, err);
    unsigned char* sA = smem + st * kStageBytes;
    unsigned char* sB = sA + kAB;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const int e = tid + q * TC_THREADS;
      const uint32_t offa = chunk_off(e % TC_BM, e / TC_BM);
      store_split_x2(sA + offa, sA + TC_TILE_BYTES + offa, areg[q], true);
      const uint32_t offb = chunk_off(e / (TC_BK / 8), e % (TC_BK / 8));
      store_split_x2(sB + offb, sB + TC_TILE_BYTES + offb, breg[q], true);
    }
    if (kt + 1 < nk) load(kt + 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aS = sbase + st * kStageBytes;
      const uint32_t aLo = aS + TC_TILE_BYTES;
      const uint32_t bS = aS + kAB;
      const uint32_t bLo = bS + TC_TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint32_t ko = kk * 256;
        const uint32_t acc0 = (kt > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, make_desc(aS + ko, 128, kSBO), make_desc(bS + ko, 128, kSBO), acc0);
        mma_bf16(tmem, make_desc(aS + ko, 128, kSBO), make_desc(bLo + ko, 128, kSBO), 1u);
        mma_bf16(tmem, make_desc(aLo + ko, 128, kSBO), make_desc(bS + ko, 128, kSBO), 1u);
      }
      mma_commit(smem_u32(&empty[st]));
    }
  }
  if (nk > 0 && !timed_out)
    timed_out = !mbar_wait(smem_u32(&empty[(nk - 1) & 1]), ((nk - 1) >> 1) & 1, err);
  if (timed_out && lane == 0) atomicCAS((unsigned long long*)&err[0], 0ull, 2ull);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w reads lanes 32*(w%4).. (rows) and columns 64*(w/4)..+64;
  // the thread's entries of C are loaded 16 at a time before any is stored
  const int quarter = warp & 3, half = warp >> 2;
  const int gi = i0 + quarter * 32 + lane;
  const bool live = gi < m && nk > 0 && !timed_out;
#pragma unroll
  for (int cb = 0; cb < 64; cb += 16) {
    float cv[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int gc = c0 + half * 64 + cb + t;
      cv[t] = (live && gc < m) ? A[gi + (int64_t)gc * m] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < 16; c += 16) {
      uint32_t rv[16];
      const uint32_t taddr =
          tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64 + cb + c);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15}, [%16];"
          : "=r"(rv[0]), "=r"(rv[1]), "=r"(rv[2]), "=r"(rv[3]), "=r"(rv[4]), "=r"(rv[5]),
            "=r"(rv[6]), "=r"(rv[7]), "=r"(rv[8]), "=r"(rv[9]), "=r"(rv[10]), "=r"(rv[11]),
            "=r"(rv[12]), "=r"(rv[13]), "=r"(rv[14]), "=r"(rv[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (live) {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int gc = c0 + half * 64 + cb + c + t;
          if (gc < m) A[gi + (int64_t)gc * m] = cv[c + t] - __uint_as_float(rv[t]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TC_BN));
}

// ---------------------------------------------------------------------------
// Fused front products.  For a front whose output rows fit one CTA, the two
// products of each sweep are folded into one GEMM over the front's rows:
//   forward:  [X_piv; dT_upd] = W_f T_piv,        W_f = [L11^-1; -L21 L11^-1]   (m x k)
//   backward: X_piv = W_b [X_piv; X_upd],         W_b = [U11^-1, -U11^-1 U12]    (k x m)
// (X_upd: the solution on the front's update rows, gathered through its row
// list; dT_upd is stored apart, in D, and the parent's gather adds it to what
// the front's own children passed up on those rows).
// The MMA is transposed with respect to the tile ops above: its M = 128 are
// panel columns and its N = the front's output rows rounded up to 16, so a
// small front costs N, not 128, rows of work; the accumulator lives in
// tensor memory as 128 lanes (columns) x N (rows).  W is packed once per
// factorisation in the same K-major bf16 layout with N rows per 32-column
// K-block (high part, then the remainder).
// ---------------------------------------------------------------------------
enum { DIR_FWD = 0, DIR_BWD = 1 };

__device__ __forceinline__ uint32_t idesc_m128(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_n(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Output rows and K of a fused front product.
template <int DIR>
__device__ __forceinline__ void fused_dims(int32_t k, int32_t m, int& nout, int& K) {
  nout = DIR == DIR_BWD ? k : m;
  K = DIR == DIR_BWD ? m : k;
}

// W of one front, K-block kb (32 columns): entries that are blocks of the
// factored front are copied, the product blocks are formed here in fp32:
//   backward, column j >= k:  -sum_{l >= i} U11^-1(i, l) U12(l, j)
//   forward,  row i >= k:     -sum_{l >= j} L21(i, l) L11^-1(l, j)
// The right factor's 32 columns are staged in shared memory ([k][33]).
template <int DIR, int PASSES>
__global__ void __launch_bounds__(TC_THREADS)
    k_w_pack(DevFronts F, const int32_t* __restrict__ fronts, const int32_t* __restrict__ kbs,
             const int64_t* __restrict__ woff, const float* __restrict__ arena,
             unsigned char* __restrict__ wpk) {
  extern __shared__ float Rs[];
  const int32_t f = fronts[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  int nout, K;
  fused_dims<DIR>(k, m, nout, K);
  const int kb = kbs[blockIdx.x];
  if (kb * TC_BK >= K) return;
  const int nf = (nout + 15) & ~15;
  const float* __restrict__ A = arena + F.arena[f];
  const int j0 = kb * TC_BK;
  // right factor: backward U12(l, j) (rows l < k of column j >= k), forward L11^-1(l, j)
  for (int e = threadIdx.x; e < k * TC_BK; e += TC_THREADS) {
    const int l = e % k, jj = e / k, j = j0 + jj;
    float v = 0.f;
    if (j < K) {
      if (DIR == DIR_BWD)
        v = j >= k ? A[l + (int64_t)j * m] : 0.f;
      else
        v = l > j ? A[l + (int64_t)j * m] : (l == j ? 1.f : 0.f);
    }
    Rs[l * (TC_BK + 1) + jj] = v;
  }
  __syncthreads();
  const uint32_t part = (uint32_t)nf * TC_BK * 2;
  unsigned char* dst = wpk + woff[f] + (int64_t)kb * (PASSES == 3 ? 2 : 1) * part;
  if constexpr (DIR == DIR_FWD) {
  // forward (m output rows): one thread per row, the 32 entries of the row in
  // this K-block as outer products (a coalesced column read of L21 per term,
  // the row of L11^-1 from shared memory), then 16-byte stores
  for (int i = threadIdx.x; i < nf; i += TC_THREADS) {
    float acc[TC_BK];
#pragma unroll
    for (int jj = 0; jj < TC_BK; ++jj) acc[jj] = 0.f;
    if (i < nout && i >= k) {
      for (int l = j0; l < k; ++l) {  // -sum_l L21(i, l) L11^-1(l, j); L11^-1(l, j) = 0 for l < j
        const float a = A[i + (int64_t)l * m];
        const float* __restrict__ r = Rs + l * (TC_BK + 1);
#pragma unroll
        for (int jj = 0; jj < TC_BK; ++jj) acc[jj] = fmaf(a, r[jj], acc[jj]);
      }
    }
#pragma unroll
    for (int kc = 0; kc < TC_BK / 8; ++kc) {
      float v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int jj = kc * 8 + t, j = j0 + jj;
        float w = 0.f;
        if (i < nout && j < K)
          w = i < k ? (i > j ? A[i + (int64_t)j * m] : (i == j ? 1.f : 0.f)) : -acc[jj];
        v[t] = w;
      }
      const uint32_t off = chunk_off(i, kc);
      store_split(dst + off, dst + part + off, v, PASSES == 3);
    }
  }
  } else {
  // backward (k output rows, often few): one warp per row, lanes over the
  // 32 columns; -sum_{l >= i} U11^-1(i, l) U12(l, j) for the columns j >= k
  const int jj = threadIdx.x & 31;
  const int j = j0 + jj;
  for (int i = threadIdx.x >> 5; i < nf; i += TC_THREADS / 32) {
    float w = 0.f;
    if (i < nout && j < K) {
      if (j < k) {
        w = i <= j ? A[i + (int64_t)j * m] : 0.f;
      } else {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int l = i;
        for (; l + 4 <= k; l += 4) {
          a0 = fmaf(A[i + (int64_t)l * m], Rs[l * (TC_BK + 1) + jj], a0);
          a1 = fmaf(A[i + (int64_t)(l + 1) * m], Rs[(l + 1) * (TC_BK + 1) + jj], a1);
          a2 = fmaf(A[i + (int64_t)(l + 2) * m], Rs[(l + 2) * (TC_BK + 1) + jj], a2);
          a3 = fmaf(A[i + (int64_t)(l + 3) * m], Rs[(l + 3) * (TC_BK + 1) + jj], a3);
        }
        for (; l < k; ++l) a0 = fmaf(A[i + (int64_t)l * m], Rs[l * (TC_BK + 1) + jj], a0);
        w = -((a0 + a1) + (a2 + a3));
      }
    }
    uint16_t hi, lo;
    split_bf16(w, hi, lo);
    const uint32_t off = chunk_off(i, jj >> 3) + (jj & 7) * 2;
    *reinterpret_cast<uint16_t*>(dst + off) = hi;
    if (PASSES == 3) *reinterpret_cast<uint16_t*>(dst + part + off) = lo;
  }
  }
}

// Bounded wait that does not give up when another CTA has recorded a
// timeout: used only to let a CTA's own copies land before it exits.
__device__ __forceinline__ void mbar_drain(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return;
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Four consecutive columns of a panel row, of which the first nv are valid
// (16-byte aligned; nv >= 4: one vector store, nv <= 0: none).
__device__ __forceinline__ void st_cols4(float* p, float4 v, int nv) {
  if (nv >= 4) {
    *reinterpret_cast<float4*>(p) = v;
    return;
  }
  if (nv > 0) p[0] = v.x;
  if (nv > 1) p[1] = v.y;
  if (nv > 2) p[2] = v.z;
}

// One work item = (front, 128-column panel tile) of a fused front product.
// The fields of the CTA's first kTab fronts are read once, at the start, into
// a table in shared memory (FMeta); consecutive items are mostly the tiles of
// one front, and each role keeps its current front's fields (FItem).
constexpr int kTab = 32;
struct FMeta {
  int32_t f, k, nout, K, row0, tb0, ncols;
  // forward: the working rows are the front's pivot rows of X; backward: the
  // front is inactive in the pass, its pivot rows are read as the zero row
  int32_t fromx;
  int64_t wo;
};
struct FCtx {
  DevFronts F;
  const int32_t* fronts;
  int32_t nct;
  const int64_t* woff;
  const unsigned char* wpk;
  const int64_t* block_ncols;
  int64_t j0;
  int32_t NR;
  const FMeta* tab;  // fronts p0 .. p0 + ntab - 1 of the list
  int32_t p0, ntab;
  // forward: fronts without active children; backward: fronts active in the
  // pass (may be null)
  const uint8_t* pleaf;
};
struct FItem {
  int32_t p = -1;  // position of the front in the launch's list
  int32_t f, fromx;
  int32_t k, nout, K, nf, nkt, kt0, cv;  // stages kt0 .. nkt - 1
  int64_t ncols, n0, row0, tb0;
  const int32_t* idx;
  const unsigned char* w;
  uint32_t wpart, wblk;
};

template <int DIR>
__device__ __forceinline__ void fmeta_load(const FCtx& c, int32_t f, FMeta& m) {
  m.f = f;
  m.k = c.F.k[f];
  fused_dims<DIR>(m.k, c.F.m[f], m.nout, m.K);
  m.row0 = (int32_t)c.F.row0[f];
  m.tb0 = (int32_t)c.F.idx_off[f];
  m.ncols = (int32_t)min((int64_t)c.NR, c.block_ncols[c.F.block[f]] - c.j0);
  m.fromx = c.pleaf && (DIR == DIR_FWD ? c.pleaf[f] != 0 : c.pleaf[f] == 0) ? 1 : 0;
  m.wo = c.woff[f];
}

template <int DIR, int PASSES>
__device__ __forceinline__ bool fitem(const FCtx& c, int it, FItem& w) {
  const int32_t p = it / c.nct;
  if (p != w.p) {
    w.p = p;
    FMeta m;
    if (p - c.p0 < c.ntab)
      m = c.tab[p - c.p0];
    else
      fmeta_load<DIR>(c, c.fronts[p], m);
    w.f = m.f;
    w.fromx = m.fromx;
    w.k = m.k;
    w.nout = m.nout;
    w.K = m.K;
    w.ncols = m.ncols;
    w.nf = (w.nout + 15) & ~15;
    w.nkt = (w.K + TC_BK - 1) / TC_BK;
    // backward, inactive front: the stages of zero pivot rows are skipped
    // (at least the last stage runs, so that the product is written)
    w.kt0 = DIR == DIR_BWD && w.fromx ? min(w.k / TC_BK, w.nkt - 1) : 0;
    w.row0 = m.row0;
    w.tb0 = m.tb0;
    w.idx = c.F.idx + m.tb0;
    w.w = c.wpk + m.wo;
    w.wpart = (uint32_t)w.nf * TC_BK * 2;
    w.wblk = (PASSES == 3 ? 2u : 1u) * w.wpart;
  }
  w.n0 = (int64_t)(it % c.nct) * TC_BN;
  if (w.n0 >= w.ncols) return false;
  w.cv = (int)min((int64_t)TC_BN, w.ncols - w.n0);
  return true;
}

// Persistent, warp-specialised fused front product.  Each CTA (one per SM)
// takes a contiguous range of work items (front, 128-column tile); a tile is
// nkt K-stages of 32 panel rows.  A stage lives in one slot of a ring of SR
// 16 KB slots from the moment its rows are copied in until its MMAs complete:
//   warps 16-19 (row producers, stage g by warp 16 + g % NPROD): the stage's
//     32 panel rows (fp32, 128 columns) into its slot with tensor copies:
//     forward, the rows are consecutive working rows of the front (one tile
//     copy; for a front none of whose children is active in the pass they
//     are its pivot rows of X, which no gather has copied); backward, pivot
//     rows (the zero row of X for a front the pass leaves inactive, whose
//     forward solution is zero) and update rows gathered through the front's
//     row list, four rows per copy.  Every slot belongs to one warp;
//   warp 20 lane 0 (W producer): the stage's W block into a ring of SW slots;
//   warps 0-7 (converters, two groups of four on alternate stages): read the
//     slot's fp32 rows, then (after a barrier of the group's warps) overwrite
//     the slot with the bf16 (high, remainder) K-major operand;
//   warps 21 .. 20 + NMMA, lane 0 (MMA): 1, 2 (three passes, at most 128
//     output rows) or 3 tcgen05.mma per 16 K (per 256 output rows) into one of
//     NACC tensor-memory accumulators, tile t by
//     thread t % NMMA into accumulator t % NACC; the commits hand the slot and
//     the W slot back to the producers and, after the tile's last stage, the
//     accumulator to the epilogue;
//   warps 8-15 (epilogue, two groups of four): tcgen05.ld of lane quarter
//     (warp % 4); group q stores the 16-row groups q, q + 2, ...; a 16 x 32
//     block is turned around in the warp's own shared buffer so that each
//     lane stores four consecutive columns of a row (forward: the update rows
//     go to D).
// Every wait is bounded: a wait that runs out records error code 2 at once
// (so that the other waits of every CTA give up quickly), the role stops,
// and before exiting each producer lets its own copies land.
constexpr int FG_CONV = 256;   // converter threads (warps 0-7)
constexpr int FG_CGROUPS = 2;  // converter groups (alternate stages)
constexpr int FG_CGT = FG_CONV / FG_CGROUPS;
constexpr int FG_EPI0 = 8;     // epilogue warps 8-15 (tensor-memory lane quarter = warp % 4)
constexpr int FG_NEPI = 8;
constexpr int FG_PROD0 = 16;   // producer warps 16-19
constexpr int FG_NPROD = 4;
constexpr int FG_WPROD = 20;   // W producer warp
constexpr int FG_MMA0 = 21;    // MMA issuer warps 21 .. 21 + NMMA - 1
constexpr int FG_MAXMMA = 2;
constexpr int FG_THREADS = (FG_MMA0 + FG_MAXMMA) * 32;

template <int DIR, int NT, int PASSES, int SR, int SW, int NACC, int NMMA, int NPROD>
__global__ void __launch_bounds__(FG_THREADS, 1)
    k_front_gemm_tc(DevFronts F, const int32_t* __restrict__ fronts, int32_t nitems, int32_t nct,
                    const int64_t* __restrict__ woff, const unsigned char* __restrict__ wpk,
                    const int64_t* __restrict__ block_ncols, int64_t j0, int32_t NR,
                    float* __restrict__ X, float* __restrict__ Tb, float* __restrict__ D,
                    const uint8_t* __restrict__ pleaf, int32_t zrow, long long* __restrict__ err,
                    int inject_wait, const __grid_constant__ CUtensorMap tm_src,
                    const __grid_constant__ CUtensorMap tm_x) {
  // every ring slot is always filled by the same producer warp, so that no
  // producer waits on a slot barrier more than one phase ahead of it
  static_assert(SR % NPROD == 0 && SR % FG_CGROUPS == 0 && NPROD <= FG_NPROD &&
                    NMMA <= FG_MAXMMA && NACC % NMMA == 0,
                "ring ownership");
  extern __shared__ __align__(1024) unsigned char smem[];
  // op_full and w_full are split by MMA thread (the owner of the stage's
  // tile, t % NMMA): each has one consumer, which sees its phases in order
  __shared__ __align__(8) uint64_t raw_full[SR], op_full[NMMA][SR], slot_empty[SR];
  __shared__ __align__(8) uint64_t w_full[NMMA][SW], w_empty[SW], acc_full[NACC], acc_empty[NACC];
  __shared__ __align__(8) uint64_t never;
  __shared__ uint32_t tmem_slot;
  __shared__ int skip_all;
  __shared__ FMeta tab[kTab];
  constexpr uint32_t kSlot = TC_BK * TC_BN * 4;                       // 32 fp32 rows x 128
  constexpr uint32_t kWs = (PASSES == 3 ? 2u : 1u) * NT * TC_BK * 2;  // W block
  // three passes with at most 128 output rows: hi*hi and hi*lo in one MMA over
  // the stacked [W_hi; W_lo] (N = 2 nf; accumulator columns [0, nf) and
  // [nf, 2 nf)), lo*hi into the first half; the epilogue adds the halves
  constexpr bool CAT = PASSES == 3 && NT <= 128;
  constexpr uint32_t ACW = CAT ? 2 * NT : NT;  // tensor-memory columns per accumulator
  const uint32_t sbase = smem_u32(smem);
  const uint32_t w0 = sbase + SR * kSlot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
  const int it0 = (int)blockIdx.x * per, it1 = min(nitems, it0 + per);
  const int32_t p0 = it0 / nct;
  const int32_t ntab = it1 > it0 ? min(kTab, (it1 - 1) / nct - p0 + 1) : 0;
  const FCtx ctx{F, fronts, nct, woff, wpk, block_ncols, j0, NR, tab, p0, ntab, pleaf};
  if (warp == 1 && lane < ntab) fmeta_load<DIR>(ctx, fronts[p0 + lane], tab[lane]);  // read before the barrier below

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ACW * NACC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < SR; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[i])));
      for (int a = 0; a < NMMA; ++a)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&op_full[a][i])),
                     "r"(FG_CGT));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&slot_empty[i])));
    }
    for (int i = 0; i < SW; ++i) {
      for (int a = 0; a < NMMA; ++a)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&w_full[a][i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&w_empty[i])));
    }
    for (int i = 0; i < NACC; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[i])),
                   "r"(FG_NEPI * 32));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&never)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    skip_all = 0;
    if (inject_wait) {  // failure-path test: a short bounded wait that must run out
      if (!mbar_wait(smem_u32(&never), 0, err, 4096u)) {
        atomicCAS((unsigned long long*)&err[0], 0ull, 2ull);
        skip_all = 1;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool bail = skip_all != 0;
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (bail) return;
    if (!mbar_wait(smem_u32(bar), parity, err)) {
      bail = true;
      atomicCAS((unsigned long long*)&err[0], 0ull, 2ull);
    }
  };
  uint32_t issued = 0;  // producer: stages issued
  uint32_t wpar[NMMA] = {}, last_own = 0u, last_par = 0u;  // W producer: phases per (owner, slot)

  if (warp >= FG_PROD0 && warp < FG_PROD0 + NPROD) {
    // ---------------- producers ----------------
    const int p = warp - FG_PROD0;
    struct Pos {
      int it, kt;
      FItem w;
    };
    Pos pos{it0, 0, {}};
    auto next_valid = [&](int from) {
      int it = from;
      while (it < it1 && !fitem<DIR, PASSES>(ctx, it, pos.w)) ++it;
      pos.it = it;
      pos.kt = it < it1 ? pos.w.kt0 : 0;
    };
    auto advance = [&]() {
      if (pos.it >= it1) return;
      if (++pos.kt >= pos.w.nkt) next_valid(pos.it + 1);
    };
    auto row_of = [&](const FItem& w, int kk) -> int64_t {
      const int gk = kk * TC_BK + lane;
      if (gk >= w.K) return 0;
      return DIR == DIR_BWD ? (gk < w.k ? (w.fromx ? (int64_t)zrow : w.row0 + gk) : (int64_t)w.idx[gk])
                            : w.tb0 + gk;
    };
    next_valid(it0);
    uint32_t g = 0;
    for (int i = 0; i < p; ++i, ++g) advance();
    int64_t row_next = pos.it < it1 ? row_of(pos.w, pos.kt) : 0;
    while (pos.it < it1 && !bail) {
      const int64_t row = row_next;
      const Pos cur = pos;
      const uint32_t gc = g;
      for (int i = 0; i < NPROD; ++i, ++g) advance();  // this warp's next stage
      if (pos.it < it1) row_next = row_of(pos.w, pos.kt);
      // panel rows of stage gc into its slot (free once the MMAs of stage gc - SR
      // completed).  Every copy fills whole 512-byte rows: rows past K and
      // columns past the block's count are read too (or filled with zeros past
      // the panel) and masked by the converters.
      const uint32_t sl = gc % SR;
      if (gc >= SR) wait(&slot_empty[sl], ((gc / SR) - 1) & 1);
      bail = __any_sync(0xffffffffu, bail);  // keep the warp together for __syncwarp
      if (bail) break;
      const uint32_t dst = sbase + sl * kSlot;
      if (DIR == DIR_FWD) {
        if (lane == 0) {
          mbar_expect_tx(smem_u32(&raw_full[sl]), kSlot);
          if (cur.w.fromx)
            tma_tile_2d(dst, &tm_x, (int32_t)cur.w.n0, (int32_t)(cur.w.row0 + cur.kt * TC_BK),
                        smem_u32(&raw_full[sl]));
          else
            tma_tile_2d(dst, &tm_src, (int32_t)cur.w.n0, (int32_t)(cur.w.tb0 + cur.kt * TC_BK),
                        smem_u32(&raw_full[sl]));
        }
      } else {
        const int32_t r = (int32_t)row;
        const int32_t y0 = __shfl_sync(0xffffffffu, r, (4 * lane) & 31);
        const int32_t y1 = __shfl_sync(0xffffffffu, r, (4 * lane + 1) & 31);
        const int32_t y2 = __shfl_sync(0xffffffffu, r, (4 * lane + 2) & 31);
        const int32_t y3 = __shfl_sync(0xffffffffu, r, (4 * lane + 3) & 31);
        if (lane == 0) mbar_expect_tx(smem_u32(&raw_full[sl]), kSlot);
        __syncwarp();
        if (lane < TC_BK / 4)
          tma_gather4(dst + (uint32_t)lane * (4 * TC_BN * 4), &tm_src, (int32_t)cur.w.n0, y0, y1,
                      y2, y3, smem_u32(&raw_full[sl]));
      }
      issued = gc + 1;
    }
  } else if (warp == FG_WPROD) {
    // ---------------- W producer ----------------
    // W blocks come from their own warp, so that they do not queue behind the
    // row copies; a W slot is refilled once the MMAs of its stage completed.
    if (lane == 0) {
      uint32_t g = 0, tc = 0;
      FItem w;
      for (int it = it0; it < it1 && !bail; ++it, ++tc) {
        if (!fitem<DIR, PASSES>(ctx, it, w)) {
          --tc;
          continue;
        }
        const uint32_t own = tc % NMMA;
        for (int kt = w.kt0; kt < w.nkt && !bail; ++kt, ++g) {
          const uint32_t ws = g % SW;
          if (g >= SW) wait(&w_empty[ws], ((g / SW) - 1) & 1);
          if (bail) break;
          mbar_expect_tx(smem_u32(&w_full[own][ws]), w.wblk);
          bulk_g2s(w0 + ws * kWs, w.w + (int64_t)kt * w.wblk, w.wblk, smem_u32(&w_full[own][ws]));
          issued = g + 1;
          // for the drain after a timeout: owner and phase parity of slot ws's last fill
          const uint32_t par = (wpar[own] >> ws) & 1u;
          wpar[own] ^= 1u << ws;
          last_own = (last_own & ~(3u << (2 * ws))) | (own << (2 * ws));
          last_par = (last_par & ~(1u << ws)) | (par << ws);
        }
      }
    }
  } else if (warp < FG_CONV / 32) {
    // ---------------- converters ----------------
    // two groups of four warps take alternate stages (slot sl always goes to
    // group sl % 2, SR being even), so that two stages are converted at once
    const int cg = warp / (FG_CGT / 32), ct = tid - cg * FG_CGT;
    uint32_t g = 0, tc = 0;
    FItem w;
    for (int it = it0; it < it1 && !bail; ++it) {
      if (!fitem<DIR, PASSES>(ctx, it, w)) continue;
      const uint32_t own = tc++ % NMMA;
      for (int kt = w.kt0; kt < w.nkt && !bail; ++kt, ++g) {
        if ((int)(g % FG_CGROUPS) != cg) continue;
        const uint32_t sl = g % SR;
        wait(&raw_full[sl], (g / SR) & 1);
        unsigned char* slot = smem + sl * kSlot;
        const float* raw = reinterpret_cast<const float*>(slot);
        const int nr = min(TC_BK, w.K - kt * TC_BK);
        constexpr int kQ = (TC_BN * TC_BK / 8) / FG_CGT;
        float v[kQ][8];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const int e = ct + q * FG_CGT;
          const int col = e % TC_BN, kc = e / TC_BN;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int r = kc * 8 + u;
            v[q][u] = (!bail && r < nr && col < w.cv) ? raw[r * TC_BN + col] : 0.f;
          }
        }
        // the group's warps have read the slot before any overwrites it; the
        // barrier also makes a timeout in any of them a decision of all
        uint32_t any_bail;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
            "bar.red.or.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(any_bail)
            : "r"((uint32_t)bail), "r"(1 + cg), "r"(FG_CGT)
            : "memory");
        bail = any_bail != 0;
        if (bail) break;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const int e = ct + q * FG_CGT;
          const uint32_t off = chunk_off(e % TC_BN, e / TC_BN);
          store_split_x2(slot + off, slot + TC_TILE_BYTES + off, v[q], PASSES == 3);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&op_full[own][sl]));
      }
    }
  } else if (warp >= FG_MMA0 && warp < FG_MMA0 + NMMA) {
    // ---------------- MMA issuers ----------------
    // tile t is issued by thread t % NMMA into accumulator t % NACC, so that
    // the per-stage issue work of NMMA tiles overlaps and a tile's epilogue
    // has NACC / NMMA tiles of one thread to finish in
    const uint32_t mine = (uint32_t)(warp - FG_MMA0);
    if (lane == 0) {
      // descriptors differ only in their start-address field (address / 16,
      // 14 bits; every address here is below 256 KB): build the two bases
      // once and add offsets, so that issuing a stage costs few instructions
      const uint64_t dS = make_desc(sbase, 128, kSBO), dW = make_desc(w0, 128, kSBO);
      uint32_t g = 0, tc = 0;
      uint32_t opar = 0u, wpar_m = 0u;  // phase parity of this thread's barriers, bit per slot
      FItem w;
      for (int it = it0; it < it1 && !bail; ++it) {
        if (!fitem<DIR, PASSES>(ctx, it, w)) continue;
        const uint32_t a = tc % NACC;
        if (tc % NMMA != mine) {  // another thread's tile: skip its stages
          g += w.nkt - w.kt0;
          ++tc;
          continue;
        }
        if (tc >= NACC) wait(&acc_empty[a], ((tc / NACC) - 1) & 1);
        const uint32_t acc = tmem + a * ACW;
        const uint32_t id0 = idesc_m128(min(256, w.nf));
        const uint32_t idc = CAT ? idesc_m128(2 * w.nf) : 0u;
        const uint32_t id1 = w.nf > 256 ? idesc_m128(w.nf - 256) : 0u;
        const uint64_t lo_w = w.wpart >> 4;
        for (int kt = w.kt0; kt < w.nkt && !bail; ++kt, ++g) {
          const uint32_t sl = g % SR, ws = g % SW;
          wait(&op_full[mine][sl], (opar >> sl) & 1u);
          wait(&w_full[mine][ws], (wpar_m >> ws) & 1u);
          if (bail) break;
          opar ^= 1u << sl;
          wpar_m ^= 1u << ws;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t aHi = dS + ((sl * kSlot) >> 4), aLo = aHi + (TC_TILE_BYTES >> 4);
          const uint64_t bHi = dW + ((ws * kWs) >> 4), bLo = bHi + lo_w;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint64_t ko = kk * (256 >> 4);
            const uint32_t acc0 = (kt > w.kt0 || kk > 0) ? 1u : 0u;
            if (CAT) {
              mma_bf16_n(acc, aHi + ko, bHi + ko, idc, acc0);  // [hi*hi | hi*lo]
              mma_bf16_n(acc, aLo + ko, bHi + ko, id0, 1u);
            } else {
              mma_bf16_n(acc, aHi + ko, bHi + ko, id0, acc0);
              if (PASSES == 3) {
                mma_bf16_n(acc, aHi + ko, bLo + ko, id0, 1u);
                mma_bf16_n(acc, aLo + ko, bHi + ko, id0, 1u);
              }
            }
            if (NT > 256 && id1) {  // output rows 256.. : B rows 256.. and accumulator columns 256..
              const uint64_t wo = (256 / 8) * kSBO >> 4;
              mma_bf16_n(acc + 256, aHi + ko, bHi + wo + ko, id1, acc0);
              if (PASSES == 3) {
                mma_bf16_n(acc + 256, aHi + ko, bLo + wo + ko, id1, 1u);
                mma_bf16_n(acc + 256, aLo + ko, bHi + wo + ko, id1, 1u);
              }
            }
          }
          mma_commit(smem_u32(&slot_empty[sl]));
          mma_commit(smem_u32(&w_empty[ws]));
          if (kt == w.nkt - 1) mma_commit(smem_u32(&acc_full[a]));
        }
        ++tc;
      }
    }
  } else if (warp >= FG_EPI0 && warp < FG_EPI0 + FG_NEPI) {
    // ---------------- epilogue ----------------
    const int quarter = warp & 3, grp = (warp - FG_EPI0) >> 2;
    // this warp's 16 x 32 buffer (after the rings): lane l holds column l of
    // 16 rows after tcgen05.ld, and stores columns 4 (l % 8) .. + 3 of rows
    // 4 r + l / 8 (r = 0..3) after the turn
    float* tbuf = reinterpret_cast<float*>(smem + SR * kSlot + SW * kWs) + (warp - FG_EPI0) * 512;
    const int rsub = lane >> 3, c4 = 4 * (lane & 7);
    uint32_t tc = 0;
    FItem w;
    for (int it = it0; it < it1 && !bail; ++it) {
      if (!fitem<DIR, PASSES>(ctx, it, w)) continue;
      const uint32_t a = tc % NACC;
      const int64_t gj = w.n0 + quarter * 32 + c4;  // this lane's first column
      const int nv = w.cv - (quarter * 32 + c4);    // how many of its four columns are valid
      wait(&acc_full[a], (tc / NACC) & 1);
      bail = __any_sync(0xffffffffu, bail);  // tcgen05.ld is warp-collective
      if (bail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + a * ACW + ((uint32_t)(quarter * 32) << 16);
      for (int c16 = grp * 16; c16 < w.nout; c16 += 32) {
        uint32_t rv[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(rv[0]), "=r"(rv[1]), "=r"(rv[2]), "=r"(rv[3]), "=r"(rv[4]), "=r"(rv[5]),
              "=r"(rv[6]), "=r"(rv[7]), "=r"(rv[8]), "=r"(rv[9]), "=r"(rv[10]), "=r"(rv[11]),
              "=r"(rv[12]), "=r"(rv[13]), "=r"(rv[14]), "=r"(rv[15])
            : "r"(acc + (uint32_t)c16));
        uint32_t rw[16];
        if (CAT)
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
              "%10, %11, %12, %13, %14, %15}, [%16];"
              : "=r"(rw[0]), "=r"(rw[1]), "=r"(rw[2]), "=r"(rw[3]), "=r"(rw[4]), "=r"(rw[5]),
                "=r"(rw[6]), "=r"(rw[7]), "=r"(rw[8]), "=r"(rw[9]), "=r"(rw[10]), "=r"(rw[11]),
                "=r"(rw[12]), "=r"(rw[13]), "=r"(rw[14]), "=r"(rw[15])
              : "r"(acc + (uint32_t)(w.nf + c16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int u = 0; u < 16; ++u)
          tbuf[u * 32 + lane] =
              CAT ? __uint_as_float(rv[u]) + __uint_as_float(rw[u]) : __uint_as_float(rv[u]);
        __syncwarp();
        float4 v[4];
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4)
          v[r4] = *reinterpret_cast<const float4*>(tbuf + (4 * r4 + rsub) * 32 + c4);
        __syncwarp();  // read before the next group overwrites the buffer
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
          const int i = c16 + 4 * r4 + rsub;
          if (i >= w.nout || nv <= 0) continue;
          if (DIR == DIR_FWD && i >= w.k)
            st_cols4(D + (w.tb0 + i) * NR + gj, v[r4], nv);
          else
            st_cols4(X + (w.row0 + i) * NR + gj, v[r4], nv);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&acc_empty[a]));
      ++tc;
    }
  }
  if (warp >= FG_PROD0 && warp < FG_PROD0 + NPROD && lane == 0 && bail) {
    // let this warp's own copies land before the CTA exits
    for (uint32_t g = issued > SR ? issued - SR : 0; g < issued; ++g)
      if ((int)(g % NPROD) == warp - FG_PROD0) mbar_drain(smem_u32(&raw_full[g % SR]), (g / SR) & 1);
  }
  if (warp == FG_WPROD && lane == 0 && bail)
    for (uint32_t ws = 0; ws < (uint32_t)SW && ws < issued; ++ws)
      mbar_drain(smem_u32(&w_full[(last_own >> (2 * ws)) & 3u][ws]), (last_par >> ws) & 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(ACW * NACC));
}

// Ring depths per tensor-memory width (shared memory: SR x 16 KB stage slots,
// SW x W blocks and the epilogue warps' 2 KB buffers; one CTA per SM).
template <int NT, int PASSES>
struct FrontCfg {
  static constexpr int SR = NT <= 128 ? 8 : 4;
  static constexpr int SW = NT <= 64 ? 6 : NT <= 128 ? 5 : NT <= 256 ? 4 : 2;
  // accumulators (512 tensor-memory columns; twice NT wide for three passes up to 128 rows)
  static constexpr int NACC = NT <= 64 ? 4 : NT <= 128 ? (PASSES == 3 ? 2 : 4) : NT <= 256 ? 2 : 1;
  static constexpr int NMMA = NACC >= 2 ? 2 : 1;                   // MMA-issuing threads
  static constexpr int NPROD = 4;  // row producer warps (divides SR)
};

// Tensor map over a row-major fp32 panel of `rows` rows and NR columns, in
// boxes of 128 columns x box_rows rows (no swizzle; zeros past the panel).
using TmapEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                     const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                     const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                     CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeTiled tmap_encoder() {
  static const TmapEncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TmapEncodeTiled f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = (TmapEncodeTiled)p;
    cudaGetLastError();
    return f;
  }();
  return fn;
}
bool panel_map(CUtensorMap* map, const float* base, int64_t rows, int32_t NR, int box_rows) {
  const TmapEncodeTiled enc = tmap_encoder();
  if (!enc) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)NR, (cuuint64_t)std::max<int64_t>(rows, 1)};
  const cuuint64_t stride[1] = {(cuuint64_t)NR * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BN, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int DIR, int NT, int PASSES>
void launch_front(DevFronts F, const int32_t* fronts, int32_t nfr, const int64_t* woff,
                  const unsigned char* wpk, const int64_t* block_ncols, int64_t j0, int32_t NR,
                  float* X, int64_t x_rows, float* Tb, int64_t tb_rows, float* D,
                  const uint8_t* pleaf, long long* err, int inject, cudaStream_t s) {
  using C = FrontCfg<NT, PASSES>;
  auto kern = k_front_gemm_tc<DIR, NT, PASSES, C::SR, C::SW, C::NACC, C::NMMA, C::NPROD>;
  constexpr size_t sm = (size_t)C::SR * TC_BK * TC_BN * 4 +
                        (size_t)C::SW * (PASSES == 3 ? 2 : 1) * NT * TC_BK * 2 +
                        (size_t)FG_NEPI * 16 * 32 * sizeof(float);
  // forward: tiles of 32 working rows (of Tb, or of X for fronts without
  // active children); backward: single rows of X for the gathers
  CUtensorMap tm, tmx;
  const bool ok = DIR == DIR_FWD
                      ? panel_map(&tm, Tb, tb_rows, NR, TC_BK) && panel_map(&tmx, X, x_rows, NR, TC_BK)
                      : panel_map(&tm, X, x_rows, NR, 1);
  if (DIR != DIR_FWD) tmx = tm;
  if (!ok) {
    record_launch_error(cudaErrorInvalidValue);
    return;
  }
  const int nsm = device_sm_count();
  record_launch_error(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int32_t nct = (NR + TC_BN - 1) / TC_BN;
  const int32_t nitems = nfr * nct;
  const int32_t grid = std::min(nitems, nsm);
  kern<<<grid, FG_THREADS, sm, s>>>(F, fronts, nitems, nct, woff, wpk, block_ncols, j0, NR, X, Tb,
                                    D, pleaf, (int32_t)(x_rows - 1), err, inject, tm, tmx);
}

template <int DIR, int PASSES>
void dispatch_front(int cls, DevFronts F, const int32_t* fronts, int32_t nfr, const int64_t* woff,
                    const unsigned char* wpk, const int64_t* block_ncols, int64_t j0, int32_t NR,
                    float* X, int64_t x_rows, float* Tb, int64_t tb_rows, float* D,
                    const uint8_t* pleaf, long long* err, int inject, cudaStream_t s) {
#define DDPS_FRONT(NT)                                                                           \
  launch_front<DIR, NT, PASSES>(F, fronts, nfr, woff, wpk, block_ncols, j0, NR, X, x_rows, Tb, \
                                tb_rows, D, pleaf, err, inject, s)
  switch (cls) {
    case 0:
      DDPS_FRONT(64);
      break;
    case 1:
      DDPS_FRONT(128);
      break;
    case 2:
      DDPS_FRONT(256);
      break;
    default:
      DDPS_FRONT(512);
  }
#undef DDPS_FRONT
}

template <int OP, int PASSES>
void launch_one(DevFronts F, const int32_t* tile_front, const int32_t* tile_m0,
                const int64_t* tile_aoff, const unsigned char* atc, int32_t ntiles,
                const int64_t* block_ncols, int64_t j0, int32_t NR, float* X, float* Tb,
                long long* err, int inject, cudaStream_t s) {
  constexpr uint32_t stage = 2 * (PASSES == 3 ? 2u : 1u) * TC_TILE_BYTES;
  const size_t sm = 2 * stage;
  record_launch_error(cudaFuncSetAttribute(k_spike_gemm_tc<OP, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm));
  dim3 grid(ntiles, (NR + TC_BN - 1) / TC_BN);
  k_spike_gemm_tc<OP, PASSES><<<grid, TC_THREADS, sm, s>>>(F, tile_front, tile_m0, tile_aoff, atc,
                                                            block_ncols, j0, NR, X, Tb, err, inject);
}

template <int PASSES>
void dispatch_gemm(int op, DevFronts F, const int32_t* tf, const int32_t* tm, const int64_t* ta,
                   const unsigned char* atc, int32_t nt, const int64_t* block_ncols, int64_t j0,
                   int32_t NR, float* X, float* Tb, long long* err, int inject, cudaStream_t s) {
  switch (op) {
    case OP_FWD_LINV:
      launch_one<OP_FWD_LINV, PASSES>(F, tf, tm, ta, atc, nt, block_ncols, j0, NR, X, Tb, err,
                                      inject, s);
      break;
    case OP_FWD_L21:
      launch_one<OP_FWD_L21, PASSES>(F, tf, tm, ta, atc, nt, block_ncols, j0, NR, X, Tb, err,
                                     inject, s);
      break;
    case OP_BWD_U12:
      launch_one<OP_BWD_U12, PASSES>(F, tf, tm, ta, atc, nt, block_ncols, j0, NR, X, Tb, err,
                                     inject, s);
      break;
    default:
      launch_one<OP_BWD_UINV, PASSES>(F, tf, tm, ta, atc, nt, block_ncols, j0, NR, X, Tb, err,
                                      inject, s);
  }
}

template <int PASSES>
void dispatch_pack(int op, DevFronts F, const int32_t* tf, const int32_t* tm, const int64_t* ta,
                   int32_t nt, int32_t max_kt, const float* arena, unsigned char* atc,
                   cudaStream_t s) {
  dim3 grid(nt, max_kt);
  switch (op) {
    case OP_FWD_LINV:
      k_tc_pack_a<OP_FWD_LINV, PASSES><<<grid, TC_THREADS, 0, s>>>(F, tf, tm, ta, arena, atc);
      break;
    case OP_FWD_L21:
      k_tc_pack_a<OP_FWD_L21, PASSES><<<grid, TC_THREADS, 0, s>>>(F, tf, tm, ta, arena, atc);
      break;
    case OP_BWD_U12:
      k_tc_pack_a<OP_BWD_U12, PASSES><<<grid, TC_THREADS, 0, s>>>(F, tf, tm, ta, arena, atc);
      break;
    default:
      k_tc_pack_a<OP_BWD_UINV, PASSES><<<grid, TC_THREADS, 0, s>>>(F, tf, tm, ta, arena, atc);
  }
}

}  // namespace

int tc_fused_max_rows() { return 512; }
int tc_fused_class(int rows) {
  const int n = (rows + 15) & ~15;
  return n <= 64 ? 0 : n <= 128 ? 1 : n <= 256 ? 2 : 3;
}
int64_t tc_fused_w_bytes(int passes, int rows, int K) {
  const int64_t nf = (rows + 15) & ~15;
  const int64_t nkb = (K + TC_BK - 1) / TC_BK;
  return (passes == 3 ? 2 : 1) * nf * TC_BK * 2 * nkb;
}

void launch_tc_w_pack(int bwd, int passes, DevFronts F, const int32_t* fronts, const int32_t* kb,
                      int32_t nitems, int32_t max_k, const int64_t* woff, const float* arena,
                      unsigned char* wpk, cudaStream_t s) {
  if (nitems <= 0) return;
  const size_t sm = (size_t)std::max(max_k, 1) * (TC_BK + 1) * sizeof(float);
#define DDPS_WPACK(D, P)                                                                        \
  record_launch_error(cudaFuncSetAttribute(k_w_pack<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));   \
  k_w_pack<D, P><<<nitems, TC_THREADS, sm, s>>>(F, fronts, kb, woff, arena, wpk);
  if (bwd) {
    if (passes == 3) {
      DDPS_WPACK(DIR_BWD, 3)
    } else {
      DDPS_WPACK(DIR_BWD, 1)
    }
  } else {
    if (passes == 3) {
      DDPS_WPACK(DIR_FWD, 3)
    } else {
      DDPS_WPACK(DIR_FWD, 1)
    }
  }
#undef DDPS_WPACK
}

void launch_front_gemm_tc(int bwd, int cls, int passes, DevFronts F, const int32_t* fronts,
                          int32_t nfr, const int64_t* woff, const unsigned char* wpk,
                          const int64_t* block_ncols, int64_t j0, int32_t NR, float* X,
                          int64_t x_rows, float* Tb, int64_t tb_rows, float* D,
                          const uint8_t* pleaf, long long* err, int inject_wait, cudaStream_t s) {
  if (nfr <= 0) return;
#define DDPS_DISP(DD, P)                                                                           \
  dispatch_front<DD, P>(cls, F, fronts, nfr, woff, wpk, block_ncols, j0, NR, X, x_rows, Tb,      \
                        tb_rows, D, pleaf, err, inject_wait, s)
  if (bwd) {
    if (passes == 3)
      DDPS_DISP(DIR_BWD, 3);
    else
      DDPS_DISP(DIR_BWD, 1);
  } else {
    if (passes == 3)
      DDPS_DISP(DIR_FWD, 3);
    else
      DDPS_DISP(DIR_FWD, 1);
  }
#undef DDPS_DISP
}

int tc_tile_bk() { return TC_BK; }

void launch_lu_update_tc(DevFronts F, const int32_t* tile_front, const int32_t* tile_ij,
                         int32_t ntiles, int32_t j0, float* arena, long long* err, cudaStream_t s) {
  if (ntiles <= 0) return;
  const size_t sm = 2 * 4 * (size_t)TC_TILE_BYTES;  // two stages of L and U, high and low parts
  record_launch_error(cudaFuncSetAttribute(k_lu_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_lu_update_tc<<<ntiles, TC_THREADS, sm, s>>>(F, tile_front, tile_ij, j0, arena, err);
}
int64_t tc_a_block_bytes(int passes) { return (passes == 3 ? 2 : 1) * (int64_t)TC_TILE_BYTES; }

void launch_tc_pack_a(int op, int passes, DevFronts F, const int32_t* tile_front,
                      const int32_t* tile_m0, const int64_t* tile_aoff, int32_t ntiles,
                      int32_t max_kt, const float* arena, unsigned char* atc, cudaStream_t s) {
  if (ntiles <= 0 || max_kt <= 0) return;
  if (passes == 3)
    dispatch_pack<3>(op, F, tile_front, tile_m0, tile_aoff, ntiles, max_kt, arena, atc, s);
  else
    dispatch_pack<1>(op, F, tile_front, tile_m0, tile_aoff, ntiles, max_kt, arena, atc, s);
}

void launch_spike_gemm_tc(int op, int passes, DevFronts F, const int32_t* tile_front,
                          const int32_t* tile_m0, const int64_t* tile_aoff,
                          const unsigned char* atc, int32_t ntiles, const int64_t* block_ncols,
                          int64_t j0, int32_t NR, float* X, float* Tb, long long* err,
                          int inject_wait, cudaStream_t s) {
  if (ntiles <= 0) return;
  if (passes == 3)
    dispatch_gemm<3>(op, F, tile_front, tile_m0, tile_aoff, atc, ntiles, block_ncols, j0, NR, X,
                     Tb, err, inject_wait, s);
  else
    dispatch_gemm<1>(op, F, tile_front, tile_m0, tile_aoff, atc, ntiles, block_ncols, j0, NR, X,
                     Tb, err, inject_wait, s);
}

}  // namespace ddps
