// Numeric preprocessing of DDPS on the device: Fig. 2 step 2 (exact LU of
// every diagonal block, here a multifrontal LU without pivoting over the
// nested-dissection order) and Fig. 2 step 4 (spikes G = D~^-1 R~, keeping the
// rows that lie in c, i.e. the off-identity part of G^ = I(c,c) + G(c,c),
// stored as one dense row-major array per partition as Sec. 3 describes).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "launch.h"

namespace ddps {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int threads, int cap = 152 * 16) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename T>
__device__ __forceinline__ T from_double(double v) {
  return (T)v;
}

// ---------------------------------------------------------------------------
// Assembly of the original entries of every A_ii into its fronts.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_assemble(const double* __restrict__ values, const int64_t* __restrict__ amap,
                           int64_t nnz, T* __restrict__ arena) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t dst = amap[e];
    if (dst >= 0) arena[dst] = from_double<T>(values[e]);
  }
}

// max |a_ij| over the D-part of each row, stored at the row's new index; the
// pivot threshold of a front row is pivot_tol times this value.
__global__ void k_row_absmax(const int32_t* __restrict__ rowptr, const int64_t* __restrict__ amap,
                             const double* __restrict__ values, const int32_t* __restrict__ iperm,
                             int64_t n, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double mx = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (amap[e] >= 0) mx = fmax(mx, fabs(values[e]));
    out[iperm[i]] = mx;
  }
}

// ---------------------------------------------------------------------------
// Extend-add: parent front += child's Schur complement (its trailing r x r
// block), one child per parent per launch so that no two writers meet.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_extend_add_p(DevFronts F, const int32_t* __restrict__ parent,
                               const int32_t* __restrict__ child_list, T* __restrict__ arena) {
  const int32_t c = child_list[blockIdx.x];
  const int32_t kc = F.k[c], mc = F.m[c];
  const int32_t r = mc - kc;
  if (r <= 0) return;
  const int32_t p = parent[c];
  const int32_t mp = F.m[p];
  const int32_t* __restrict__ rel = F.rel + F.rel_off[c];
  const T* __restrict__ C = arena + F.arena[c];
  T* __restrict__ P = arena + F.arena[p];
  // one warp per update column, lanes over its rows (no index division)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t j = blockIdx.y * nw + warp; j < r; j += gridDim.y * nw) {
    T* __restrict__ Pc = P + (int64_t)rel[j] * mp;
    const T* __restrict__ Cc = C + kc + (int64_t)(kc + j) * mc;
    for (int32_t i = lane; i < r; i += 32) Pc[rel[i]] += Cc[i];
  }
}

// ---------------------------------------------------------------------------
// Partial LU of a front (no pivoting): the first k columns/rows become
// L11\U11, L21 and U12; the trailing r x r block becomes the Schur complement
// passed to the parent.  Blocked right-looking with panels of NB pivots and
// TT x TT tiles for the trailing update.
// ---------------------------------------------------------------------------
constexpr int NB = 32;
constexpr int TT = 64;

// ---------------------------------------------------------------------------
// Large fronts, several CTAs per front: blocked right-looking LU, one panel
// of 32 pivots at a time.  Without pivoting the panel
// splits into independent parts: the 32 x 32 diagonal block is factored
// first (k_lu_diag, one CTA per front, which also forms the inverses of its
// two triangles into a scratch block per front), then every row below it
// takes its L21 row as a U11^-1 and every column to the right its U12
// column as L11^-1 a (k_lu_panel_rows, CTAs over chunks of 256 rows or
// columns of every front of the depth), then the trailing update
// (k_lu_trailing, and the tensor-core block update).
// dinv: per entry of the launch's front list, 2 x 32 x 32 entries:
// U11^-1 (row-major, upper) then L11^-1 (row-major, unit lower).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_lu_diag(DevFronts F, const int32_t* __restrict__ list, int32_t j0, T* __restrict__ arena,
              const double* __restrict__ rownorm, double pivot_tol, long long* __restrict__ err,
              T* __restrict__ dinv) {
  const int32_t f = list[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  if (j0 >= k) return;
  T* __restrict__ A = arena + F.arena[f];
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  const int jb = min(NB, k - j0);
  __shared__ T D[NB][NB + 1];
  __shared__ double thr[NB];
  for (int t = tid; t < NB * NB; t += blockDim.x) {
    const int r = t % NB, c = t / NB;
    D[r][c] = (r < jb && c < jb) ? A[(j0 + r) + (int64_t)(j0 + c) * m] : T(r == c ? 1 : 0);
  }
  if (tid < jb) thr[tid] = pivot_tol * rownorm[row0 + j0 + tid];
  __syncthreads();
  if (tid < 32) {
    // the 32 x 32 LU by one warp: lane r owns row r of the updates
    for (int j = 0; j < jb; ++j) {
      T piv = D[j][j];
      const bool small = !(fabs((double)piv) > thr[j]);
      if (small) {
        const double rep = thr[j] > 0.0 ? thr[j] : 1e-300;
        piv = (T)((double)piv < 0.0 ? -rep : rep);
      }
      __syncwarp();  // every lane has read the pivot before it is replaced
      if (small && tid == 0) {
        if (atomicCAS((unsigned long long*)&err[0], 0ull, 1ull) == 0ull) {
          err[1] = f;
          err[2] = row0 + j0 + j;
        }
        D[j][j] = piv;
      }
      const T inv = T(1) / piv;
      if (tid > j && tid < jb) {
        const T l = D[tid][j] * inv;
        D[tid][j] = l;
        for (int c = j + 1; c < jb; ++c) D[tid][c] -= l * D[j][c];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int t = tid; t < jb * jb; t += blockDim.x) {
    const int r = t % jb, c = t / jb;
    A[(j0 + r) + (int64_t)(j0 + c) * m] = D[r][c];
  }
  // inverses of the 32 x 32 triangles (identity beyond jb): warp 0 forms
  // column c of U11^-1 (lane c, backward substitution), warp 1 column c of
  // L11^-1 (forward substitution)
  T* Ui = dinv + (int64_t)blockIdx.x * 2 * NB * NB;
  T* Li = Ui + NB * NB;
  const int lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    T x[NB];
#pragma unroll
    for (int r = NB - 1; r >= 0; --r) {
      T sacc = r == lane ? T(1) : T(0);
#pragma unroll
      for (int p = r + 1; p < NB; ++p) sacc -= D[r][p] * x[p];
      x[r] = r <= lane ? sacc / D[r][r] : T(0);
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) Ui[r * NB + lane] = x[r];
  } else if (warp == 1) {
    T x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      T sacc = r == lane ? T(1) : T(0);
#pragma unroll
      for (int p = 0; p < r; ++p) sacc -= D[r][p] * x[p];
      x[r] = r >= lane ? sacc : T(0);
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) Li[r * NB + lane] = x[r];
  }
}

// chunk word: bit 30 set = columns (U12), else rows (L21); bits 0-29 = chunk of
// 256; chunk_slot: the front's position in the diagonal launch's list (dinv)
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_lu_panel_rows(DevFronts F, const int32_t* __restrict__ chunk_front,
                    const int32_t* __restrict__ chunk_word, const int32_t* __restrict__ chunk_slot,
                    int32_t j0, T* __restrict__ arena, const T* __restrict__ dinv) {
  const int32_t f = chunk_front[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const int jb = min(NB, k - j0);
  const int t0 = j0 + jb;
  const bool cols = (chunk_word[blockIdx.x] >> 30) & 1;
  const int q = chunk_word[blockIdx.x] & 0x3fffffff;
  T* __restrict__ A = arena + F.arena[f];
  const int tid = threadIdx.x;
  __shared__ T Mi[NB][NB + 1];  // U11^-1 (rows) or L11^-1 (columns), row-major
  const T* src = dinv + (int64_t)chunk_slot[blockIdx.x] * 2 * NB * NB + (cols ? NB * NB : 0);
  for (int t = tid; t < NB * NB; t += blockDim.x) Mi[t / NB][t % NB] = src[t];
  __syncthreads();
  const int i = t0 + q * kThreads + tid;
  if (i >= m) return;
  T a[NB];
  if (!cols) {
    // L21 row i = a U11^-1
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = c < jb ? A[i + (int64_t)(j0 + c) * m] : T(0);
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      if (c < jb) {
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int p = 0; p <= c; p += 2) {
          s0 += a[p] * Mi[p][c];
          if (p + 1 <= c) s1 += a[p + 1] * Mi[p + 1][c];
        }
        A[i + (int64_t)(j0 + c) * m] = s0 + s1;
      }
    }
  } else {
    // U12 column i = L11^-1 a
#pragma unroll
    for (int r = 0; r < NB; ++r) a[r] = r < jb ? A[(j0 + r) + (int64_t)i * m] : T(0);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      if (r < jb) {
        T s0 = a[r], s1 = T(0);
#pragma unroll
        for (int p = 0; p < r; p += 2) {
          s0 += Mi[r][p] * a[p];
          if (p + 1 < r) s1 += Mi[r][p + 1] * a[p + 1];
        }
        A[(j0 + r) + (int64_t)i * m] = s0 + s1;
      }
    }
  }
}

// tile word: front in tile_front, (ti << 16) | tj in tile_ij, rows/cols from t0 = j0 + 32.
// blocked: entries with row and column >= skip (the end of the current block
// of 256 pivots) are left to the block's tensor-core update.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_lu_trailing(DevFronts F, const int32_t* __restrict__ tile_front,
                  const int32_t* __restrict__ tile_ij, int32_t j0, int blocked,
                  T* __restrict__ arena) {
  const int32_t f = tile_front[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const int jb = min(NB, k - j0);
  const int t0 = j0 + jb;
  const int skip = blocked ? min((j0 & ~(kLuTcBlock - 1)) + kLuTcBlock, k) : INT_MAX;
  const int ti = tile_ij[blockIdx.x] >> 16, tj = tile_ij[blockIdx.x] & 0xffff;
  const int rb = t0 + ti * TT, cb = t0 + tj * TT;
  T* __restrict__ A = arena + F.arena[f];
  const int tid = threadIdx.x;
  __shared__ T Lt[TT][NB + 1];
  __shared__ T Ut[NB][TT + 1];
  for (int t = tid; t < TT * NB; t += blockDim.x) {
    const int r = t % TT, q = t / TT;
    Lt[r][q] = (rb + r < m && q < jb) ? A[rb + r + (int64_t)(j0 + q) * m] : T(0);
    const int q2 = t % NB, c2 = t / NB;
    Ut[q2][c2] = (cb + c2 < m && q2 < jb) ? A[j0 + q2 + (int64_t)(cb + c2) * m] : T(0);
  }
  __syncthreads();
  const int tr = tid % 16, tc = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = T(0);
#pragma unroll 8
  for (int q = 0; q < NB; ++q) {
    T lv[4], uv[4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) lv[a2] = Lt[tr + 16 * a2][q];
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) uv[b2] = Ut[q][tc + 16 * b2];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] += lv[a2] * uv[b2];
  }
#pragma unroll
  for (int b2 = 0; b2 < 4; ++b2) {
    const int c = cb + tc + 16 * b2;
    if (c >= m) continue;
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2) {
      const int r = rb + tr + 16 * a2;
      if (r < m && (r < skip || c < skip)) A[r + (int64_t)c * m] -= acc[a2][b2];
    }
  }
}

// ---------------------------------------------------------------------------
// Triangular inverses of large fronts with many CTAs, out of place into
// `inv` (k x k column-major per front at inv_off[f]; L11^-1, then U11^-1).
// The diagonal 64 x 64 tiles of an inverse are the inverses of the diagonal
// tiles of the triangle: k_tri_inverse_diag forms them first, one CTA per
// tile.  Then CTA (front, column block of 64) of k_tri_inverse_mc walks its
// column block away from the diagonal: tile X(i, j) = -D(i)^-1 sum_l A(i, l)
// X(l, j) over the tiles l already solved, as two tile GEMMs (D(i)^-1 is the
// diagonal tile of X).  k_tri_inverse_copy then writes the strictly lower
// part of L11^-1 and the upper part of U11^-1 back into the front.
// ---------------------------------------------------------------------------
constexpr int IB = 64;  // columns per CTA and rows per tile

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_tri_inverse_diag(DevFronts F, const int32_t* __restrict__ tile_front,
                       const int32_t* __restrict__ tile_cb, const T* __restrict__ arena,
                       T* __restrict__ inv, const int64_t* __restrict__ inv_off) {
  const int32_t f = tile_front[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const int i0 = tile_cb[blockIdx.x] * IB;
  const bool upper = blockIdx.y == 1;
  const T* __restrict__ A = arena + F.arena[f];
  T* __restrict__ X = inv + inv_off[f] + (upper ? (int64_t)k * k : 0);
  const int tid = threadIdx.x;
  // two 64 x 65 tiles of dynamic shared memory (the triangle's tile, the inverse)
  extern __shared__ unsigned char smem_raw[];
  T(*Ds)[IB + 1] = reinterpret_cast<T(*)[IB + 1]>(smem_raw);
  T(*Ts)[IB + 1] = reinterpret_cast<T(*)[IB + 1]>(smem_raw + sizeof(T) * IB * (IB + 1));
  const int rows = min(IB, k - i0);
  for (int t = tid; t < IB * IB; t += blockDim.x) {
    const int r = t % IB, c = t / IB;
    Ds[r][c] = (r < rows && c < rows) ? A[(i0 + r) + (int64_t)(i0 + c) * m] : T(0);
    Ts[r][c] = r == c ? T(1) : T(0);
  }
  __syncthreads();
  if (!upper) {
    for (int r = 0; r < rows; ++r) {  // unit diagonal: row r is final now
      for (int t = tid; t < (rows - r - 1) * IB; t += blockDim.x) {
        const int r2 = r + 1 + t / IB, c = t % IB;
        Ts[r2][c] -= Ds[r2][r] * Ts[r][c];
      }
      __syncthreads();
    }
  } else {
    for (int r = rows - 1; r >= 0; --r) {
      const T d = Ds[r][r];
      for (int c = tid; c < IB; c += blockDim.x) Ts[r][c] /= d;
      __syncthreads();
      for (int t = tid; t < r * IB; t += blockDim.x) {
        const int r2 = t / IB, c = t % IB;
        Ts[r2][c] -= Ds[r2][r] * Ts[r][c];
      }
      __syncthreads();
    }
  }
  for (int t = tid; t < IB * IB; t += blockDim.x) {
    const int r = t % IB, c = t / IB;
    if (r < rows && c < rows) X[(i0 + r) + (int64_t)(i0 + c) * k] = Ts[r][c];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_tri_inverse_mc(DevFronts F, const int32_t* __restrict__ tile_front,
                     const int32_t* __restrict__ tile_cb, const T* __restrict__ arena,
                     T* __restrict__ inv, const int64_t* __restrict__ inv_off) {
  const int32_t f = tile_front[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  const int j0 = tile_cb[blockIdx.x] * IB;
  const bool upper = blockIdx.y == 1;
  const T* __restrict__ A = arena + F.arena[f];
  T* __restrict__ X = inv + inv_off[f] + (upper ? (int64_t)k * k : 0);
  const int tid = threadIdx.x;
  extern __shared__ unsigned char smem_raw[];
  T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);
  T(*Bs)[IB + 1] = reinterpret_cast<T(*)[IB + 1]>(smem_raw + sizeof(T) * IB * (NB + 1));
  T(*Ts)[IB + 1] = reinterpret_cast<T(*)[IB + 1]>(smem_raw + sizeof(T) * (IB * (NB + 1) + NB * (IB + 1)));
  // the diagonal tile of the inverse, D(i)^-1
  T(*Ds)[IB + 1] = reinterpret_cast<T(*)[IB + 1]>(
      smem_raw + sizeof(T) * (IB * (NB + 1) + NB * (IB + 1) + IB * (IB + 1)));
  const int tr = tid % 16, tc = tid / 16;
  const int ntile_rows = upper ? (min(j0 + IB, k) + IB - 1) / IB : (k - j0 + IB - 1) / IB;
  // it = 0 is the diagonal tile, formed by k_tri_inverse_diag
  for (int it = 1; it < ntile_rows; ++it) {
    // lower: row tiles below j0 downwards; upper: above the diagonal tile upwards
    const int i0 = upper ? ((min(j0 + IB, k) - 1) / IB - it) * IB : j0 + it * IB;
    // acc = sum over the solved rows l of A(i0.., l) X(l, j0..)
    const int l_begin = upper ? i0 + IB : j0;
    const int l_end = upper ? min(j0 + IB, k) : i0;
    T acc[4][4];
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = T(0);
    for (int l0 = l_begin; l0 < l_end; l0 += NB) {
      for (int t = tid; t < IB * NB; t += blockDim.x) {
        const int r = t % IB, q = t / IB;
        const int gi = i0 + r, gl = l0 + q;
        As[r][q] = (gi < k && gl < l_end) ? A[gi + (int64_t)gl * m] : T(0);
        const int q2 = t % NB, c2 = t / NB;
        const int gl2 = l0 + q2, gj = j0 + c2;
        Bs[q2][c2] = (gl2 < l_end && gj < k) ? X[gl2 + (int64_t)gj * k] : T(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int q = 0; q < NB; ++q) {
        T lv[4], uv[4];
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) lv[a2] = As[tr + 16 * a2][q];
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) uv[b2] = Bs[q][tc + 16 * b2];
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] += lv[a2] * uv[b2];
      }
      __syncthreads();
    }
    // X(i0, j0) = -D(i0)^-1 acc
    const int rows = min(IB, k - i0);
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) Ts[tr + 16 * a2][tc + 16 * b2] = -acc[a2][b2];
    for (int t = tid; t < IB * IB; t += blockDim.x) {
      const int r = t % IB, c = t / IB;
      Ds[r][c] = (r < rows && c < rows) ? X[(i0 + r) + (int64_t)(i0 + c) * k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = T(0);
#pragma unroll 8
    for (int q = 0; q < IB; ++q) {
      T lv[4], uv[4];
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2) lv[a2] = Ds[tr + 16 * a2][q];
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) uv[b2] = Ts[q][tc + 16 * b2];
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] += lv[a2] * uv[b2];
    }
#pragma unroll
    for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) {
        const int r = tr + 16 * a2, c = tc + 16 * b2;
        if (r < rows && j0 + c < k) X[(i0 + r) + (int64_t)(j0 + c) * k] = acc[a2][b2];
      }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_tri_inverse_copy(DevFronts F, const int32_t* __restrict__ list,
                                   T* __restrict__ arena, const T* __restrict__ inv,
                                   const int64_t* __restrict__ inv_off) {
  const int32_t f = list[blockIdx.y];
  const int32_t k = F.k[f], m = F.m[f];
  T* __restrict__ A = arena + F.arena[f];
  const T* __restrict__ X = inv + inv_off[f];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)k * k;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % k), j = (int)(t / k);
    // lower inverse sits in the first k*k entries, upper inverse in the next k*k
    A[i + (int64_t)j * m] = i > j ? X[t] : X[(int64_t)k * k + t];
  }
}

// ---------------------------------------------------------------------------
// Small fronts (m*m entries fit in shared memory): partial LU and the
// inversion of the diagonal triangles done in shared memory by one CTA, then
// written back once.
// ---------------------------------------------------------------------------
constexpr int kLuPanel = 8;  // pivots per panel of the small-front LU

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_front_lu_small(DevFronts F, const int32_t* __restrict__ list, T* __restrict__ arena,
                     const double* __restrict__ rownorm, double pivot_tol,
                     long long* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  const int32_t f = list[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  double* th = reinterpret_cast<double*>(smem_raw);  // the k pivot thresholds
  T* A = reinterpret_cast<T*>(smem_raw + (size_t)k * sizeof(double));
  T* __restrict__ G = arena + F.arena[f];
  T* v = A + (int64_t)m * m;  // 2 m scratch entries for the inversions
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  for (int t = tid; t < m * m; t += blockDim.x) A[t] = G[t];
  for (int t = tid; t < k; t += blockDim.x) th[t] = pivot_tol * rownorm[row0 + t];
  __syncthreads();
  // right-looking LU in panels of kLuPanel pivots: warp 0 factors the panel
  // columns, the CTA solves the panel rows of U12 and applies the rank-
  // kLuPanel update to the trailing matrix; every entry sees its updates in
  // pivot order, so the result is that of the unblocked elimination
  const int warp = tid >> 5, lane = tid & 31;
  for (int jp = 0; jp < k; jp += kLuPanel) {
    const int je = min(k, jp + kLuPanel);
    if (warp == 0) {
      for (int j = jp; j < je; ++j) {
        T piv = A[j + j * m];
        const double thr = th[j];
        const bool small = !(fabs((double)piv) > thr);
        if (small) {
          const double rep = thr > 0.0 ? thr : 1e-300;
          piv = (T)((double)piv < 0.0 ? -rep : rep);
        }
        __syncwarp();  // every lane has read the pivot before it is replaced
        if (small && lane == 0) {
          if (atomicCAS((unsigned long long*)&err[0], 0ull, 1ull) == 0ull) {
            err[1] = f;
            err[2] = row0 + j;
          }
          A[j + j * m] = piv;
        }
        const T inv = T(1) / piv;
        for (int i = j + 1 + lane; i < m; i += 32) {
          const T l = A[i + j * m] * inv;
          A[i + j * m] = l;
          for (int c = j + 1; c < je; ++c) A[i + c * m] -= l * A[j + c * m];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // U12 rows of the panel: forward substitution with its unit-lower block
    for (int c = je + tid; c < m; c += blockDim.x)
      for (int j = jp; j < je; ++j) {
        const T u = A[j + c * m];
        for (int i = j + 1; i < je; ++i) A[i + c * m] -= A[i + j * m] * u;
      }
    __syncthreads();
    // trailing update, one warp per column, lanes over rows
    for (int c = je + warp; c < m; c += blockDim.x >> 5) {
      T u[kLuPanel];
#pragma unroll
      for (int j = 0; j < kLuPanel; ++j) u[j] = jp + j < je ? A[jp + j + c * m] : T(0);
      for (int i = je + lane; i < m; i += 32) {
        T a = A[i + c * m];
#pragma unroll
        for (int j = 0; j < kLuPanel; ++j)
          if (jp + j < je) a -= A[i + (jp + j) * m] * u[j];
        A[i + c * m] = a;
      }
    }
    __syncthreads();
  }
  // The two inverses touch disjoint triangles: the first half of the CTA
  // forms L11^-1, the second U11^-1, each with its own scratch vector and
  // named barrier.
  const int half = blockDim.x >> 1;
  const int gt = tid % half;
  if (tid < half) {
    // L11^-1 (strictly lower part, unit diagonal), columns descending
    for (int j = k - 2; j >= 0; --j) {
      for (int i = j + 1 + gt; i < k; i += half) v[i] = A[i + j * m];
      asm volatile("bar.sync 1, %0;" ::"r"(half) : "memory");
      for (int i = j + 1 + gt; i < k; i += half) {
        T s2 = v[i];
        for (int l = j + 1; l < i; ++l) s2 += A[i + l * m] * v[l];
        A[i + j * m] = -s2;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(half) : "memory");
    }
  } else {
    T* vu = v + m;
    // U11^-1 (upper part with the diagonal), columns ascending
    for (int j = 0; j < k; ++j) {
      for (int i = gt; i <= j; i += half) vu[i] = A[i + j * m];
      asm volatile("bar.sync 2, %0;" ::"r"(half) : "memory");
      const T d = vu[j];
      for (int i = gt; i < j; i += half) {
        T s2 = T(0);
        for (int l = i; l < j; ++l) s2 += A[i + l * m] * vu[l];
        A[i + j * m] = -s2 / d;
      }
      if (gt == 0) A[j + j * m] = T(1) / d;
      asm volatile("bar.sync 2, %0;" ::"r"(half) : "memory");
    }
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) G[t] = A[t];
}

// ---------------------------------------------------------------------------
// Spike right-hand sides: column j of block b's panel is R~_b(:, c_b[j]).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_spike_rhs(const int32_t* __restrict__ rt_rownew, const int32_t* __restrict__ rt_rhscol,
                            const int64_t* __restrict__ rt_src, int64_t nrt,
                            const double* __restrict__ values, int64_t j0, int32_t NR,
                            T* __restrict__ X) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nrt;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = rt_rhscol[e] - j0;
    if (j >= 0 && j < NR) X[(int64_t)rt_rownew[e] * NR + j] = (T)values[rt_src[e]];
  }
}

// G^ rows of every block from the solved panel, converted to the storage type.
// Four consecutive panel values of one row (16-byte aligned: NR and the
// column offset are multiples of 4).
template <typename T>
__device__ __forceinline__ void load4(const T* p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 c = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = c.x, v[3] = c.y;
  }
}

template <typename TG, typename T>
__device__ __forceinline__ TG to_storage(T v) {
  if constexpr (sizeof(TG) == 8)
    return (TG)v;
  else
    return (TG)(float)v;
}

// Four consecutive G^ entries of one row (aligned to 4 elements: G^ rows
// start at multiples of 8 elements and the column offset is a multiple of 4).
template <typename TG>
__device__ __forceinline__ void store4(TG* p, const TG v[4]) {
  if constexpr (sizeof(TG) == 2) {
    uint16_t u[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) u[t] = *reinterpret_cast<const uint16_t*>(&v[t]);
    *reinterpret_cast<uint2*>(p) = make_uint2(u[0] | ((uint32_t)u[1] << 16), u[2] | ((uint32_t)u[3] << 16));
  } else if constexpr (sizeof(TG) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
}

// G(c, c) of Fig. 2 step 5: row q of G^ (interface row c[q] of block b)
// takes panel columns j0 .. j0 + NR of the spike rows of c[q].  G^ keeps its
// columns in panel order; one warp per row, four columns per lane.
template <typename T, typename TG>
__global__ void k_ghat_extract(const int32_t* __restrict__ qblock, const int32_t* __restrict__ c_rownew,
                               const int64_t* __restrict__ gq0, const int64_t* __restrict__ gcol_ptr,
                               const int64_t* __restrict__ ghat_off, const int64_t* __restrict__ gld,
                               int64_t m, int64_t j0, int32_t NR, const T* __restrict__ X,
                               TG* __restrict__ ghat) {
  const int64_t q = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  if (q >= m) return;
  const int lane = threadIdx.x & 31;
  const int32_t b = qblock[q];
  const int64_t ncols = min((int64_t)NR, gcol_ptr[b + 1] - gcol_ptr[b] - j0);
  const T* __restrict__ src = X + (int64_t)c_rownew[q] * NR;
  TG* __restrict__ dst = ghat + ghat_off[b] + (q - gq0[b]) * gld[b] + j0;
  for (int64_t jj = lane * 4; jj < ncols; jj += 128) {
    T v[4];
    load4(src + jj, v);
    TG g[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) g[t] = to_storage<TG>(v[t]);
    if (jj + 4 <= ncols) {
      store4(dst + jj, g);
    } else {
      for (int t = 0; jj + t < ncols; ++t) dst[jj + t] = g[t];
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_assemble(const double* values, const int64_t* amap, int64_t nnz, T* arena,
                     cudaStream_t s) {
  k_assemble<T><<<grid_for(nnz, kThreads), kThreads, 0, s>>>(values, amap, nnz, arena);
}

void launch_row_absmax(const int32_t* rowptr, const int64_t* amap, const double* values,
                       const int32_t* iperm, int64_t n, double* rownorm_new, cudaStream_t s) {
  k_row_absmax<<<grid_for(n, kThreads), kThreads, 0, s>>>(rowptr, amap, values, iperm, n,
                                                           rownorm_new);
}

template <typename T>
void launch_extend_add_p(DevFronts F, const int32_t* parent, const int32_t* child_list,
                         int32_t nchild, int32_t max_r, T* arena, cudaStream_t s) {
  if (nchild <= 0) return;
  int64_t per = (int64_t)max_r * max_r;
  int gy = (int)std::min<int64_t>((per + kThreads - 1) / kThreads, 64);
  if (gy < 1) gy = 1;
  dim3 grid(nchild, gy);
  k_extend_add_p<T><<<grid, kThreads, 0, s>>>(F, parent, child_list, arena);
}

template <typename T>
void launch_spike_rhs(const int32_t* rt_rownew, const int32_t* rt_rhscol, const int64_t* rt_src,
                      int64_t nrt, const double* values, int64_t j0, int32_t NR, T* X,
                      cudaStream_t s) {
  if (nrt <= 0) return;
  k_spike_rhs<T><<<grid_for(nrt, kThreads), kThreads, 0, s>>>(rt_rownew, rt_rhscol, rt_src, nrt,
                                                               values, j0, NR, X);
}

template <typename T>
void launch_lu_panel(DevFronts F, const int32_t* list, int32_t nf, const int32_t* chunk_front,
                     const int32_t* chunk_word, const int32_t* chunk_slot, int32_t nchunks,
                     int32_t j0, T* arena, T* dinv, const double* rownorm_new, double pivot_tol,
                     long long* err, cudaStream_t s) {
  if (nf <= 0) return;
  k_lu_diag<T><<<nf, kThreads, 0, s>>>(F, list, j0, arena, rownorm_new, pivot_tol, err, dinv);
  if (nchunks > 0)
    k_lu_panel_rows<T><<<nchunks, kThreads, 0, s>>>(F, chunk_front, chunk_word, chunk_slot, j0,
                                                    arena, dinv);
}

template <typename T>
void launch_lu_trailing(DevFronts F, const int32_t* tile_front, const int32_t* tile_ij,
                        int32_t ntiles, int32_t j0, int blocked, T* arena, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_lu_trailing<T><<<ntiles, kThreads, 0, s>>>(F, tile_front, tile_ij, j0, blocked, arena);
}

template <typename T>
void launch_tri_inverse_mc(DevFronts F, const int32_t* tile_front, const int32_t* tile_cb,
                           int32_t ntiles, const int32_t* list, int32_t nf, int32_t max_k, T* arena,
                           T* inv, const int64_t* inv_off, cudaStream_t s) {
  if (ntiles <= 0) return;
  const size_t sm = sizeof(T) * ((size_t)IB * (NB + 1) + (size_t)NB * (IB + 1) + 2 * (size_t)IB * (IB + 1));
  record_launch_error(cudaFuncSetAttribute(k_tri_inverse_mc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const size_t smd = sizeof(T) * 2 * (size_t)IB * (IB + 1);
  record_launch_error(cudaFuncSetAttribute(k_tri_inverse_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd));
  k_tri_inverse_diag<T><<<dim3(ntiles, 2), kThreads, smd, s>>>(F, tile_front, tile_cb, arena, inv,
                                                                inv_off);
  k_tri_inverse_mc<T><<<dim3(ntiles, 2), kThreads, sm, s>>>(F, tile_front, tile_cb, arena, inv,
                                                             inv_off);
  const int64_t per = (int64_t)max_k * max_k;
  const int gx = (int)std::min<int64_t>(std::max<int64_t>((per + kThreads - 1) / kThreads, 1), 256);
  k_tri_inverse_copy<T><<<dim3(gx, nf), kThreads, 0, s>>>(F, list, arena, inv, inv_off);
}

template <typename T>
void launch_front_lu_small(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, T* arena,
                           const double* rownorm_new, double pivot_tol, long long* err,
                           cudaStream_t s) {
  if (nf <= 0) return;
  const size_t sm = ((size_t)max_m * max_m + 2 * (size_t)max_m) * sizeof(T) + (size_t)max_m * sizeof(double);
  if (sm > 48 * 1024)
    record_launch_error(cudaFuncSetAttribute(k_front_lu_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_front_lu_small<T><<<nf, kThreads, sm, s>>>(F, list, arena, rownorm_new, pivot_tol, err);
}

template <typename T, typename TG>
void launch_ghat_extract(const int32_t* qblock, const int32_t* c_rownew, const int64_t* gq0,
                         const int64_t* gcol_ptr, const int64_t* ghat_off, const int64_t* gld,
                         int64_t m, int64_t j0, int32_t NR, const T* X, TG* ghat, cudaStream_t s) {
  if (m <= 0) return;
  const int rows = kThreads / 32;
  k_ghat_extract<T, TG><<<(unsigned)((m + rows - 1) / rows), kThreads, 0, s>>>(
      qblock, c_rownew, gq0, gcol_ptr, ghat_off, gld, m, j0, NR, X, ghat);
}

#define DDPS_INST_T(T)                                                                          \
  template void launch_assemble<T>(const double*, const int64_t*, int64_t, T*, cudaStream_t);  \
  template void launch_extend_add_p<T>(DevFronts, const int32_t*, const int32_t*, int32_t,     \
                                       int32_t, T*, cudaStream_t);                             \
  template void launch_spike_rhs<T>(const int32_t*, const int32_t*, const int64_t*, int64_t,   \
                                    const double*, int64_t, int32_t, T*, cudaStream_t);        \
  template void launch_front_lu_small<T>(DevFronts, const int32_t*, int32_t, int32_t, T*,      \
                                         const double*, double, long long*, cudaStream_t);      \
  template void launch_tri_inverse_mc<T>(DevFronts, const int32_t*, const int32_t*, int32_t,    \
                                         const int32_t*, int32_t, int32_t, T*, T*,              \
                                         const int64_t*, cudaStream_t);                         \
  template void launch_lu_panel<T>(DevFronts, const int32_t*, int32_t, const int32_t*,          \
                                   const int32_t*, const int32_t*, int32_t, int32_t, T*, T*,    \
                                   const double*, double, long long*, cudaStream_t);            \
  template void launch_lu_trailing<T>(DevFronts, const int32_t*, const int32_t*, int32_t,      \
                                      int32_t, int, T*, cudaStream_t);

DDPS_INST_T(double)
DDPS_INST_T(float)

#define DDPS_INST_TG(T, TG)                                                                     \
  template void launch_ghat_extract<T, TG>(const int32_t*, const int32_t*, const int64_t*,     \
                                           const int64_t*, const int64_t*, const int64_t*,      \
                                           int64_t, int64_t, int32_t, const T*, TG*,           \
                                           cudaStream_t);

DDPS_INST_TG(double, double)
DDPS_INST_TG(double, float)
DDPS_INST_TG(float, float)
DDPS_INST_TG(float, __nv_bfloat16)
DDPS_INST_TG(double, __nv_bfloat16)
DDPS_INST_TG(float, __half)
DDPS_INST_TG(double, __half)

}  // namespace ddps
