// Spikes of Fig. 2 step 4, G = D~^-1 R~, for many right-hand sides at once.
// The coupling columns of R~ are solved with every block's multifrontal
// factors, one front depth at a time, NR columns per pass:
//   forward  (deepest depth first):  T_f = [R~ rows of f's pivots; 0] + children's updates
//                                    X_piv = L11^-1 T_f(piv)            (OP_FWD_LINV)
//                                    T_f(upd) -= L21 X_piv              (OP_FWD_L21)
//   backward (roots first):          T_f(piv) = X_piv - U12 X(upd rows) (OP_BWD_U12)
//                                    X_piv = U11^-1 T_f(piv)            (OP_BWD_UINV)
// Each op is one launch over a tile list covering every front of the depth
// (all blocks of all systems).  The triangular inverses were formed after
// the partial LU of each front.
#include <cuda_runtime.h>

#include <algorithm>

#include "launch.h"

namespace ddps {

namespace {

constexpr int kThreads = 256;

template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};
template <>
struct Cfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
};

// T_f = [X rows of the pivots; 0] + sum over children of their update rows.
// One CTA per (front, 32*V panel columns); each lane owns V consecutive
// columns, each of the 8 warps takes four rows per step (loads first);
// children are added one after the other (their row maps are injective, so
// rows of one child never collide).
template <typename T>
struct GatherVec;
template <>
struct GatherVec<float> {
  using V = float4;
  static constexpr int n = 4;
};
template <>
struct GatherVec<double> {
  using V = double2;
  static constexpr int n = 2;
};

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_spike_gather(DevFronts F, const int32_t* __restrict__ list,
                   const int64_t* __restrict__ block_ncols, int64_t j0, int32_t NR,
                   const T* __restrict__ X, T* __restrict__ Tb,
                   const uint8_t* __restrict__ active, const T* __restrict__ D,
                   const uint8_t* __restrict__ dflag, const uint8_t* __restrict__ skipT) {
  using V = typename GatherVec<T>::V;
  constexpr int VN = GatherVec<T>::n;
  const int32_t f = list[blockIdx.x];
  const int64_t ncols = min((int64_t)NR, block_ncols[F.block[f]] - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.y * 32 * VN;
  if (c0 >= ncols) return;
  const int col = c0 + lane * VN;  // NR is a multiple of 32 * VN: no column tail
  const int32_t k = F.k[f], m = F.m[f];
  T* __restrict__ Tf = Tb + F.idx_off[f] * NR;
  const T* __restrict__ Xf = X + F.row0[f] * NR;
  const V zero = {};
  // each warp handles four rows per step, all their loads issued first
  for (int i0 = warp * 4; i0 < m; i0 += 32) {
    V v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u;
      v[u] = i < k ? *reinterpret_cast<const V*>(Xf + (int64_t)i * NR + col) : zero;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < m) *reinterpret_cast<V*>(Tf + (int64_t)(i0 + u) * NR + col) = v[u];
  }
  __syncthreads();
  for (int32_t ci = F.cbeg[f]; ci < F.cend[f]; ++ci) {
    const int32_t c = F.children[ci];
    if (active && !active[c]) continue;  // a child untouched by this chunk contributes zero
    const int32_t kc = F.k[c], rc = F.m[c] - kc;
    const int32_t* __restrict__ rel = F.rel + F.rel_off[c];
    const T* __restrict__ Tc = skipT && skipT[c] ? nullptr : Tb + (F.idx_off[c] + kc) * NR;
    // the child's own forward update (kept apart by the fused products)
    const T* __restrict__ Dc = D && dflag[c] ? D + (F.idx_off[c] + kc) * NR : nullptr;
    for (int i0 = warp * 4; i0 < rc; i0 += 32) {
      V src[4], d[4], e[4];
      int32_t row[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        row[u] = i < rc ? rel[i] : 0;
        if (i < rc) {
          src[u] = Tc ? *reinterpret_cast<const V*>(Tc + (int64_t)i * NR + col) : zero;
          d[u] = *reinterpret_cast<const V*>(Tf + (int64_t)row[u] * NR + col);
          if (Dc) e[u] = *reinterpret_cast<const V*>(Dc + (int64_t)i * NR + col);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i0 + u >= rc) continue;
        if (Dc) {  // the child's update rows: what its children passed up, plus its own update
          if constexpr (VN == 4) {
            src[u].x += e[u].x;
            src[u].y += e[u].y;
            src[u].z += e[u].z;
            src[u].w += e[u].w;
          } else {
            src[u].x += e[u].x;
            src[u].y += e[u].y;
          }
        }
        if constexpr (VN == 4) {
          d[u].x += src[u].x;
          d[u].y += src[u].y;
          d[u].z += src[u].z;
          d[u].w += src[u].w;
        } else {
          d[u].x += src[u].x;
          d[u].y += src[u].y;
        }
        *reinterpret_cast<V*>(Tf + (int64_t)row[u] * NR + col) = d[u];
      }
    }
    __syncthreads();
  }
}

// The pivot rows of front list[blockIdx.x] (k consecutive rows of X, k * NR
// entries) set to zero, 16 bytes per store.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_zero_front_rows(DevFronts F, const int32_t* __restrict__ list, int32_t NR, T* __restrict__ X) {
  using V = typename GatherVec<T>::V;
  constexpr int VN = GatherVec<T>::n;
  const int32_t f = list[blockIdx.x];
  V* __restrict__ p = reinterpret_cast<V*>(X + F.row0[f] * NR);
  const int64_t nv = (int64_t)F.k[f] * NR / VN;  // NR is a multiple of 128
  const V zero = {};
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < nv;
       e += (int64_t)gridDim.y * blockDim.x)
    p[e] = zero;
}

// C = beta * Cin + alpha * A B for one (front, 128-row) tile and 128 panel
// columns; A is a block of the front (column-major, leading dimension m,
// triangular for the two inverse ops), B rows come from the panel or from the
// front's working rows (gathered through the front's row list for OP_BWD_U12).
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads)
    k_spike_gemm(DevFronts F, const int32_t* __restrict__ tile_front,
                 const int32_t* __restrict__ tile_m0, const T* __restrict__ arena,
                 const int64_t* __restrict__ block_ncols, int64_t j0, int32_t NR,
                 T* __restrict__ X, T* __restrict__ Tb) {
  constexpr int BM = Cfg<T>::BM, BN = Cfg<T>::BN, BK = Cfg<T>::BK, TM = Cfg<T>::TM, TN = Cfg<T>::TN;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int32_t f = tile_front[blockIdx.x];
  const int32_t m0 = tile_m0[blockIdx.x];
  const int n0 = blockIdx.y * BN;
  const int64_t ncols = min((int64_t)NR, block_ncols[F.block[f]] - j0);
  if (n0 >= ncols) return;
  const int32_t k = F.k[f], m = F.m[f], r = m - k;
  const int M = OP == OP_FWD_L21 ? r : k;
  const int K = OP == OP_BWD_U12 ? r : k;
  const int a_r0 = OP == OP_FWD_L21 ? k : 0;
  const int a_c0 = OP == OP_BWD_U12 ? k : 0;
  const T* __restrict__ A = arena + F.arena[f];
  const int64_t row0 = F.row0[f];
  const int64_t tb0 = F.idx_off[f];
  const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);

  for (int kk0 = 0; kk0 < K; kk0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / kThreads; ++q) {
      const int e = tid + q * kThreads;
      const int ii = e % BM, kq = e / BM;
      const int gi = m0 + ii, gk = kk0 + kq;
      T val = T(0);
      if (gi < M && gk < K) {
        if (OP == OP_FWD_LINV)
          val = gi > gk ? A[gi + (int64_t)gk * m] : (gi == gk ? T(1) : T(0));
        else if (OP == OP_BWD_UINV)
          val = gi <= gk ? A[gi + (int64_t)gk * m] : T(0);
        else
          val = A[(a_r0 + gi) + (int64_t)(a_c0 + gk) * m];
      }
      As[kq][ii] = val;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / kThreads; ++q) {
      const int e = tid + q * kThreads;
      const int jj = e % BN, kq = e / BN;
      const int gk = kk0 + kq, gj = n0 + jj;
      T val = T(0);
      if (gk < K && gj < ncols) {
        int64_t brow;
        if (OP == OP_FWD_LINV || OP == OP_BWD_UINV)
          brow = tb0 + gk;
        else if (OP == OP_FWD_L21)
          brow = row0 + gk;
        else
          brow = idx[k + gk];
        const T* Bp = (OP == OP_FWD_L21 || OP == OP_BWD_U12) ? X : Tb;
        val = Bp[brow * NR + gj];
      }
      Bs[kq][jj] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < BK; ++kq) {
      T av[TM], bv[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) av[a] = As[kq][ty * TM + a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[kq][tx * TN + b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int gi = m0 + ty * TM + a;
    if (gi >= M) continue;
    T* out;
    const T* cin = nullptr;
    if (OP == OP_FWD_LINV || OP == OP_BWD_UINV) {
      out = X + (row0 + gi) * NR;
    } else if (OP == OP_FWD_L21) {
      out = Tb + (tb0 + k + gi) * NR;
      cin = out;
    } else {
      out = Tb + (tb0 + gi) * NR;
      cin = X + (row0 + gi) * NR;
    }
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int gj = n0 + tx * TN + b;
      if (gj >= ncols) continue;
      out[gj] = cin ? cin[gj] - acc[a][b] : acc[a][b];
    }
  }
}

}  // namespace

template <typename T>
int spike_tile_m() {
  return Cfg<T>::BM;
}

template <typename T>
void launch_zero_front_rows(DevFronts F, const int32_t* list, int32_t nf, int32_t NR, T* X,
                            cudaStream_t s) {
  if (nf <= 0) return;
  k_zero_front_rows<T><<<dim3(nf, 8), kThreads, 0, s>>>(F, list, NR, X);
}

template <typename T>
void launch_spike_gather(DevFronts F, const int32_t* list, int32_t nf, const int64_t* block_ncols,
                         int64_t j0, int32_t NR, const T* X, T* Tb, const uint8_t* active,
                         const T* D, const uint8_t* dflag, const uint8_t* skipT, cudaStream_t s) {
  if (nf <= 0) return;
  const int per = 32 * GatherVec<T>::n;
  dim3 grid(nf, (NR + per - 1) / per);
  k_spike_gather<T><<<grid, kThreads, 0, s>>>(F, list, block_ncols, j0, NR, X, Tb, active, D,
                                              dflag, skipT);
}

template <typename T>
void launch_spike_gemm(int op, DevFronts F, const int32_t* tile_front, const int32_t* tile_m0,
                       int32_t ntiles, const T* arena, const int64_t* block_ncols, int64_t j0,
                       int32_t NR, T* X, T* Tb, cudaStream_t s) {
  if (ntiles <= 0) return;
  dim3 grid(ntiles, (NR + Cfg<T>::BN - 1) / Cfg<T>::BN);
  switch (op) {
    case OP_FWD_LINV:
      k_spike_gemm<T, OP_FWD_LINV><<<grid, kThreads, 0, s>>>(F, tile_front, tile_m0, arena,
                                                              block_ncols, j0, NR, X, Tb);
      break;
    case OP_FWD_L21:
      k_spike_gemm<T, OP_FWD_L21><<<grid, kThreads, 0, s>>>(F, tile_front, tile_m0, arena,
                                                             block_ncols, j0, NR, X, Tb);
      break;
    case OP_BWD_U12:
      k_spike_gemm<T, OP_BWD_U12><<<grid, kThreads, 0, s>>>(F, tile_front, tile_m0, arena,
                                                             block_ncols, j0, NR, X, Tb);
      break;
    default:
      k_spike_gemm<T, OP_BWD_UINV><<<grid, kThreads, 0, s>>>(F, tile_front, tile_m0, arena,
                                                              block_ncols, j0, NR, X, Tb);
  }
}

#define DDPS_INST_SP(T)                                                                         \
  template int spike_tile_m<T>();                                                               \
  template void launch_zero_front_rows<T>(DevFronts, const int32_t*, int32_t, int32_t, T*,     \
                                          cudaStream_t);                                        \
  template void launch_spike_gather<T>(DevFronts, const int32_t*, int32_t, const int64_t*,     \
                                       int64_t, int32_t, const T*, T*, const uint8_t*,         \
                                       const T*, const uint8_t*, const uint8_t*, cudaStream_t); \
  template void launch_spike_gemm<T>(int, DevFronts, const int32_t*, const int32_t*, int32_t,  \
                                     const T*, const int64_t*, int64_t, int32_t, T*, T*,       \
                                     cudaStream_t);
DDPS_INST_SP(float)
DDPS_INST_SP(double)

}  // namespace ddps
