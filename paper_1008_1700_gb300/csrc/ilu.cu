// Incomplete LU with zero fill, ILU(0), of every diagonal block (Sec. 3: the
// block factors of Fig. 2 step 2 may be approximate; the paper names
// incomplete LU as that choice), and the triangular solves that use it:
// the block solves of Fig. 3 (6.1, 6.5) and the multi-right-hand-side spike
// solves of Fig. 2 step 4.
//
// The factors live on the pattern of the blocks, in their own row order:
// one CSR array (values in the factor precision) holds L below the diagonal
// (unit diagonal implied) and U on and above it.  Row i of L depends on the
// rows k < i that it references; rows are grouped in levels (a row's level is
// one more than the largest level of those rows) so that each launch handles
// rows that are independent of one another, all blocks of all systems at
// once.  The backward solves use the levels of the U dependencies (a row's
// level is one more than the largest level of the rows j > i it references,
// so level 0 holds the rows that reference none and is solved first).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "launch.h"

namespace ddps {

namespace {

constexpr int kT = 256;

template <typename T>
__device__ __forceinline__ double to_d(T v) {
  return (double)v;
}

// Row i of the factorisation (IKJ elimination with updates outside the
// pattern left out), one thread per row of the level; small pivots are
// reported (code 1, the row) and replaced by pivot_tol * max|a_i.|.
template <typename T>
__global__ void k_ilu0_rows(const int32_t* __restrict__ rows, int32_t nrows,
                            const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ diag, T* __restrict__ a,
                            const double* __restrict__ rownorm, double pivot_tol,
                            long long* __restrict__ err) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  const int32_t i = rows[t];
  const int32_t e0 = rp[i], e1 = rp[i + 1], di = diag[i];
  for (int32_t e = e0; e < di; ++e) {
    const int32_t k = col[e];
    const T lik = a[e] / a[diag[k]];
    a[e] = lik;
    // a_ij -= l_ik u_kj for j > k in both patterns (both rows sorted)
    int32_t p = e + 1;
    for (int32_t u = diag[k] + 1; u < rp[k + 1] && p < e1; ++u) {
      const int32_t j = col[u];
      while (p < e1 && col[p] < j) ++p;
      if (p < e1 && col[p] == j) a[p] -= lik * a[u];
    }
  }
  const double piv = to_d(a[di]);
  const double thr = pivot_tol * rownorm[i];
  if (!(fabs(piv) >= thr)) {
    if (atomicCAS((unsigned long long*)&err[0], 0ull, 1ull) == 0ull) {
      err[1] = -1;
      err[2] = i;
    }
    a[di] = (T)(piv < 0 ? -thr : thr);
  }
}

// One right-hand side: forward x_i -= sum_{k<i} l_ik x_k (unit diagonal), or
// backward x_i = (x_i - sum_{j>i} u_ij x_j) / u_ii, over the rows of a level.
template <typename T, bool FWD>
__global__ void k_ilu_vec(const int32_t* __restrict__ rows, int32_t nrows,
                          const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ diag, const T* __restrict__ a,
                          T* __restrict__ x) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  const int32_t i = rows[t];
  T s = x[i];
  if (FWD) {
    for (int32_t e = rp[i]; e < diag[i]; ++e) s -= a[e] * x[col[e]];
    x[i] = s;
  } else {
    for (int32_t e = diag[i] + 1; e < rp[i + 1]; ++e) s -= a[e] * x[col[e]];
    x[i] = s / a[diag[i]];
  }
}

// The same on the spike panel X (row-major, NR columns): one CTA per (row,
// 256 columns); a row of block b touches the columns [0, ncols_b - j0) of
// the chunk that hold its coupling columns.
template <typename T, bool FWD>
__global__ void __launch_bounds__(kT)
    k_ilu_panel(const int32_t* __restrict__ rows, const int32_t* __restrict__ rp,
                const int32_t* __restrict__ col, const int32_t* __restrict__ diag,
                const T* __restrict__ a, const int32_t* __restrict__ row_block,
                const int64_t* __restrict__ block_ncols, int64_t j0, int32_t NR, int32_t nchunk,
                T* __restrict__ X) {
  const int32_t t = blockIdx.x / nchunk;
  const int32_t c = (blockIdx.x - t * nchunk) * kT + threadIdx.x;
  const int32_t i = rows[t];
  const int64_t nc = min((int64_t)NR, block_ncols[row_block[i]] - j0);
  if (c >= nc) return;
  T s = X[(int64_t)i * NR + c];
  if (FWD) {
    for (int32_t e = rp[i]; e < diag[i]; ++e) s -= a[e] * X[(int64_t)col[e] * NR + c];
    X[(int64_t)i * NR + c] = s;
  } else {
    for (int32_t e = diag[i] + 1; e < rp[i + 1]; ++e) s -= a[e] * X[(int64_t)col[e] * NR + c];
    X[(int64_t)i * NR + c] = s / a[diag[i]];
  }
}

inline int blocks_for(int64_t n) { return (int)((n + kT - 1) / kT); }

}  // namespace

template <typename T>
void launch_ilu0_level(const int32_t* rows, int32_t nrows, const IluDev& L, T* a,
                       const double* rownorm, double pivot_tol, long long* err, cudaStream_t s) {
  if (nrows <= 0) return;
  k_ilu0_rows<T><<<blocks_for(nrows), kT, 0, s>>>(rows, nrows, L.rp, L.col, L.diag, a, rownorm,
                                                  pivot_tol, err);
}

template <typename T>
void launch_ilu_vec_level(bool fwd, const int32_t* rows, int32_t nrows, const IluDev& L,
                          const T* a, T* x, cudaStream_t s) {
  if (nrows <= 0) return;
  if (fwd)
    k_ilu_vec<T, true><<<blocks_for(nrows), kT, 0, s>>>(rows, nrows, L.rp, L.col, L.diag, a, x);
  else
    k_ilu_vec<T, false><<<blocks_for(nrows), kT, 0, s>>>(rows, nrows, L.rp, L.col, L.diag, a, x);
}

template <typename T>
void launch_ilu_panel_level(bool fwd, const int32_t* rows, int32_t nrows, const IluDev& L,
                            const T* a, const int64_t* block_ncols, int64_t j0, int32_t NR, T* X,
                            cudaStream_t s) {
  if (nrows <= 0) return;
  const int32_t nchunk = (NR + kT - 1) / kT;
  const int64_t grid = (int64_t)nrows * nchunk;
  if (fwd)
    k_ilu_panel<T, true><<<(unsigned)grid, kT, 0, s>>>(rows, L.rp, L.col, L.diag, a, L.row_block,
                                                       block_ncols, j0, NR, nchunk, X);
  else
    k_ilu_panel<T, false><<<(unsigned)grid, kT, 0, s>>>(rows, L.rp, L.col, L.diag, a, L.row_block,
                                                        block_ncols, j0, NR, nchunk, X);
}

#define DDPS_INST_ILU(T)                                                                         \
  template void launch_ilu0_level<T>(const int32_t*, int32_t, const IluDev&, T*, const double*, \
                                     double, long long*, cudaStream_t);                         \
  template void launch_ilu_vec_level<T>(bool, const int32_t*, int32_t, const IluDev&, const T*, \
                                        T*, cudaStream_t);                                      \
  template void launch_ilu_panel_level<T>(bool, const int32_t*, int32_t, const IluDev&,         \
                                          const T*, const int64_t*, int64_t, int32_t, T*,       \
                                          cudaStream_t);
DDPS_INST_ILU(double)
DDPS_INST_ILU(float)

}  // namespace ddps
