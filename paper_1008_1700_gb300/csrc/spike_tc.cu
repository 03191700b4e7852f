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
#include <cuda_runtime.h>

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

template <int OP, int PASSES>
void launch_one(DevFronts F, const int32_t* tile_front, const int32_t* tile_m0,
                const int64_t* tile_aoff, const unsigned char* atc, int32_t ntiles,
                const int64_t* block_ncols, int64_t j0, int32_t NR, float* X, float* Tb,
                long long* err, int inject, cudaStream_t s) {
  constexpr uint32_t stage = 2 * (PASSES == 3 ? 2u : 1u) * TC_TILE_BYTES;
  const size_t sm = 2 * stage;
  cudaFuncSetAttribute(k_spike_gemm_tc<OP, PASSES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
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

int tc_tile_bk() { return TC_BK; }
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
