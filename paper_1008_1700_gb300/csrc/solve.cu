// Solve-phase kernels of DDPS: the block solves of Fig. 3 (6.1 and the
// retrieval 6.5 written as z = D~^-1 (y - R~ z^)), the products with A (outer
// Krylov, Fig. 2 step 6) and with R~, and the reduced product w = G^ v of 6.3.
#include <cuda_runtime.h>

#include <cooperative_groups.h>

#include <algorithm>

#include "krylov.h"
#include "launch.h"

namespace ddps {
namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int threads, int cap = 152 * 32) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename T>
__global__ void k_permute_in(const double* __restrict__ y, const int32_t* __restrict__ perm,
                             int64_t n, T* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (T)y[perm[i]];
}

template <typename T>
__global__ void k_permute_out(const T* __restrict__ w, const int32_t* __restrict__ perm, int64_t n,
                              double* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    g[perm[i]] = (double)w[i];
}

// Products of a front's dense blocks with a vector in shared memory, by the
// whole CTA of NT threads.  Rows [ra, rb) are taken in chunks of CH; within a
// chunk the work items are (32-row block, column segment) pairs, at most NSEG
// segments of at least B columns, spread over the warps: the lanes on
// consecutive rows (a coalesced read of each column), B loads in flight per
// lane.  Partial sums go to red[segment][row] (NSEG x CH entries) and are
// added in a fixed order before fin(i, v) receives row i's value.
// M(i, j) = A[(roff + i) + (coff + j) m]; TRI 0 takes the columns j < ncols,
// 1 those j < i, 2 those i <= j < ncols.
template <typename T, int NT, int CH, int NSEG, int B, int TRI, typename Fin>
__device__ __forceinline__ void cta_matvec(const T* __restrict__ A, int64_t m, int roff, int coff,
                                           int ra, int rb, int ncols, const T* x, T* red,
                                           Fin fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nseg = min(NSEG, max(1, (ncols + B - 1) / B));
  for (int c0 = ra; c0 < rb; c0 += CH) {
    const int c1 = min(rb, c0 + CH);
    const int nblk = (c1 - c0 + 31) / 32;
    for (int it = warp; it < nblk * nseg; it += NT / 32) {
      const int b = it / nseg, sg = it - b * nseg;
      const int rbase = c0 + b * 32;
      const int lo = TRI == 2 ? rbase : 0;
      const int hi = TRI == 1 ? min(ncols, rbase + 32) : ncols;
      const int wd = (hi - lo + nseg - 1) / nseg;
      const int i = rbase + lane;
      int jb = lo + sg * wd, je = min(hi, jb + wd);
      if (TRI == 1) je = min(je, i);
      if (TRI == 2) jb = max(jb, i);
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      if (i < c1) {
        const T* __restrict__ Ai = A + (roff + i) + (int64_t)coff * m;
        for (int j = jb; j < je; j += B) {
          // the B column loads go out first; x comes from shared memory as
          // the products are formed
          T a[B];
#pragma unroll
          for (int q = 0; q < B; ++q) a[q] = j + q < je ? Ai[(int64_t)(j + q) * m] : T(0);
#pragma unroll
          for (int q = 0; q < B; q += 4) {
            s0 += a[q] * (j + q < je ? x[j + q] : T(0));
            s1 += a[q + 1] * (j + q + 1 < je ? x[j + q + 1] : T(0));
            s2 += a[q + 2] * (j + q + 2 < je ? x[j + q + 2] : T(0));
            s3 += a[q + 3] * (j + q + 3 < je ? x[j + q + 3] : T(0));
          }
        }
      }
      red[sg * CH + (rbase - c0) + lane] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    for (int i = c0 + threadIdx.x; i < c1; i += NT) {
      T v = red[i - c0];
      for (int sg = 1; sg < nseg; ++sg) v += red[sg * CH + (i - c0)];
      fin(i, v);
    }
    __syncthreads();
  }
}

// Rows [*a, *b) of n taken by CTA `rank` of `nct` (32-row multiples).
__device__ __forceinline__ void cta_rows(int n, int rank, int nct, int* a, int* b) {
  const int per = ((n + nct - 1) / nct + 31) / 32 * 32;
  *a = min(n, rank * per);
  *b = min(n, *a + per);
}

// Rows [*a, *b) of a k x k triangle taken by CTA `rank` of `nct`, split so
// that every CTA reads about the same number of entries (row i of a lower
// triangle holds i entries, of an upper one k - i): boundaries at
// k sqrt(r / nct) (lower) or k (1 - sqrt(1 - r / nct)) (upper), in 32-row
// multiples.
__device__ __forceinline__ int tri_bound(int k, int r, int nct, bool lower) {
  if (r <= 0) return 0;
  if (r >= nct) return k;
  const float f = (float)r / (float)nct;
  const float x = lower ? sqrtf(f) : 1.f - sqrtf(1.f - f);
  return min(k, ((int)(x * (float)k) + 31) / 32 * 32);
}
__device__ __forceinline__ void cta_rows_tri(int k, int rank, int nct, bool lower, int* a, int* b) {
  *a = tri_bound(k, rank, nct, lower);
  *b = max(*a, tri_bound(k, rank + 1, nct, lower));
}

// Copies the ranges of v that the cluster's other CTAs computed (cta_rows
// split of n) from their shared memory into this CTA's copy.
template <typename T>
__device__ __forceinline__ void cluster_gather(T* v, int n, int tri = 0) {
  cg::cluster_group cl = cg::this_cluster();
  const int nct = (int)cl.num_blocks(), me = (int)cl.block_rank();
  for (int q = 0; q < nct; ++q) {
    if (q == me) continue;
    int a, b;
    if (tri)
      cta_rows_tri(n, q, nct, tri == 1, &a, &b);
    else
      cta_rows(n, q, nct, &a, &b);
    const T* rv = cl.map_shared_rank(v, q);
    for (int i = a + (int)threadIdx.x; i < b; i += blockDim.x) v[i] = rv[i];
  }
}

// Programmatic dependent launch: each level's grid lets the next one start
// as soon as all of its CTAs have begun; the next grid reads the factors and
// the front structure (written before the sweep) at once and waits for this
// grid to finish before it reads w or u.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Brings rows [r0, r1) of columns [c0, c1) of a column-major block (leading
// dimension m) into L2, one 128-byte line per request.
template <typename T, int NT>
__device__ __forceinline__ void prefetch_rows(const T* A, int64_t m, int r0, int r1, int c0,
                                              int c1) {
  if (r1 <= r0 || c1 <= c0) return;
  const int per = (int)(((int64_t)(r1 - r0) * (int64_t)sizeof(T) + 127) / 128) + 1;
  const int64_t total = (int64_t)(c1 - c0) * per;
  for (int64_t q = threadIdx.x; q < total; q += NT) {
    const int64_t j = c0 + q / per;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(A + r0 + j * m) >> 7;
    const uintptr_t hi = reinterpret_cast<uintptr_t>(A + (r1 - 1) + j * m) >> 7;
    const uintptr_t line = lo + (uintptr_t)(q % per);
    if (line <= hi) asm volatile("prefetch.global.L2 [%0];" ::"l"(line << 7));
  }
}

constexpr int kMaxChildren = 16;

// Forward substitution for one front per cluster of CTAs (a cluster of one
// for levels with many fronts), with the inverse of the unit lower diagonal
// block formed at factor time.  The front vector t (shared memory, built by
// every CTA of the cluster) starts with the pivot entries of w and zeros and
// receives the children's update vectors; then y = L11^-1 t(piv), split by
// rows over the cluster, goes back to w, and the update entries t(upd) - L21 y
// go to u for the parent.
template <typename T, int NT, int CH, int NSEG, int B>
__global__ void __launch_bounds__(NT, B == 8 ? 8 : 2)
    k_fwd1(DevFronts F, const int32_t* __restrict__ list, const T* __restrict__ arena,
           T* __restrict__ w, T* __restrict__ u) {
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // NSEG x CH entries
  T* t = red + NSEG * CH;                   // m entries
  __shared__ int32_t ch_rc[kMaxChildren];
  __shared__ int64_t ch_rel[kMaxChildren], ch_upd[kMaxChildren];
  pdl_trigger();
  cg::cluster_group cl = cg::this_cluster();
  const int nct = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int32_t f = list[blockIdx.x / nct];
  const int32_t k = F.k[f], m = F.m[f];
  T* y = t + m;                             // k entries
  const T* __restrict__ A = arena + F.arena[f];
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  const int32_t cb = F.cbeg[f], nch = F.cend[f] - cb;
  if (tid < min(nch, kMaxChildren)) {
    const int32_t c = F.children[cb + tid];
    ch_rc[tid] = F.m[c] - F.k[c];
    ch_rel[tid] = F.rel_off[c];
    ch_upd[tid] = F.upd[c];
  }
  int a, b, a2, b2;
  cta_rows_tri(k, rank, nct, true, &a, &b);
  cta_rows(m - k, rank, nct, &a2, &b2);
  prefetch_rows<T, NT>(A, m, a, b, 0, k);
  prefetch_rows<T, NT>(A, m, k + a2, k + b2, 0, k);
  pdl_wait();
  for (int i = tid; i < m; i += blockDim.x) t[i] = i < k ? w[row0 + i] : T(0);
  __syncthreads();
  for (int32_t q = 0; q < nch; ++q) {
    int32_t rc;
    int64_t ro, uo;
    if (q < kMaxChildren) {
      rc = ch_rc[q];
      ro = ch_rel[q];
      uo = ch_upd[q];
    } else {
      const int32_t c = F.children[cb + q];
      rc = F.m[c] - F.k[c];
      ro = F.rel_off[c];
      uo = F.upd[c];
    }
    const int32_t* __restrict__ rel = F.rel + ro;
    const T* __restrict__ uc = u + uo;
    for (int i = tid; i < rc; i += blockDim.x) t[rel[i]] += uc[i];
    __syncthreads();
  }
  cta_matvec<T, NT, CH, NSEG, B, 1>(A, m, 0, 0, a, b, k, t, red, [&](int i, T v) { y[i] = t[i] + v; });
  if (nct > 1) {
    cl.sync();  // every CTA has read w and written its rows of y
    cluster_gather(y, k, 1);
  }
  for (int i = a + tid; i < b; i += blockDim.x) w[row0 + i] = y[i];
  __syncthreads();
  T* __restrict__ uf = u + F.upd[f];
  cta_matvec<T, NT, CH, NSEG, B, 0>(A, m, k, 0, a2, b2, k, y, red, [&](int i, T v) { uf[i] = t[k + i] - v; });
  if (nct > 1) cl.sync();  // keep y alive until the other CTAs have copied it
}

// Backward substitution for one front per cluster of CTAs:
// x_piv = U11^-1 (y_piv - U12 x_upd) with the inverse formed at factor time;
// x_upd are ancestor pivots of w.  Both products are split by rows over the
// cluster; the CTAs exchange their parts of the intermediate vector.
template <typename T, int NT, int CH, int NSEG, int B>
__global__ void __launch_bounds__(NT, B == 8 ? 8 : 2)
    k_bwd1(DevFronts F, const int32_t* __restrict__ list, const T* __restrict__ arena,
           T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);  // NSEG x CH entries
  T* t = red + NSEG * CH;                   // k entries, then x_upd (r entries)
  pdl_trigger();
  cg::cluster_group cl = cg::this_cluster();
  const int nct = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int32_t f = list[blockIdx.x / nct];
  const int32_t k = F.k[f], m = F.m[f], r = m - k;
  const T* __restrict__ A = arena + F.arena[f];
  const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  T* xu = t + k;
  int a, b;
  int a2, b2;  // rows of the triangular product, split by area
  cta_rows(k, rank, nct, &a, &b);
  cta_rows_tri(k, rank, nct, false, &a2, &b2);
  const int32_t i0 = tid < r ? idx[k + tid] : 0;
  prefetch_rows<T, NT>(A, m, a, b, k, m);
  prefetch_rows<T, NT>(A, m, a2, b2, 0, k);
  pdl_wait();
  if (tid < r) xu[tid] = w[i0];
  for (int j = tid + NT; j < r; j += NT) xu[j] = w[idx[k + j]];
  __syncthreads();
  cta_matvec<T, NT, CH, NSEG, B, 0>(A, m, 0, k, a, b, r, xu, red, [&](int i, T v) { t[i] = w[row0 + i] - v; });
  if (nct > 1) {
    cl.sync();
    cluster_gather(t, k);
    __syncthreads();
  }
  cta_matvec<T, NT, CH, NSEG, B, 2>(A, m, 0, 0, a2, b2, k, t, red, [&](int i, T v) { w[row0 + i] = v; });
  if (nct > 1) cl.sync();
}

// The same two sweeps with one warp per front (eight fronts per CTA), for
// depths of many small fronts: the lanes take consecutive rows (coalesced
// column reads), each lane runs its rows' dot products with eight loads in
// flight, and the front vector lives in the warp's slice of shared memory
// (ldt entries).  Only warp-level synchronisation after the dependent wait.
template <typename T>
__device__ __forceinline__ T warp_row_dot(const T* __restrict__ Ai, int64_t m, int jb, int je,
                                          const T* x) {
  T s0 = T(0), s1 = T(0);
  for (int j = jb; j < je; j += 8) {
    T a[8], xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool in = j + q < je;
      a[q] = in ? Ai[(int64_t)(j + q) * m] : T(0);
      xv[q] = in ? x[j + q] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      s0 += a[q] * xv[q];
      s1 += a[q + 1] * xv[q + 1];
    }
  }
  return s0 + s1;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_fwd1w(DevFronts F, const int32_t* __restrict__ list, int32_t nf, int32_t ldt,
            const T* __restrict__ arena, T* __restrict__ w, T* __restrict__ u) {
  extern __shared__ unsigned char smem_raw[];
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (kThreads / 32) + warp;
  T* t = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * ldt;  // m entries, then y (k)
  const bool live = q < nf;
  int32_t f = 0, k = 0, m = 0;
  if (live) {
    f = list[q];
    k = F.k[f];
    m = F.m[f];
  }
  pdl_wait();
  if (!live) return;
  const T* __restrict__ A = arena + F.arena[f];
  const int64_t row0 = F.row0[f];
  T* y = t + m;
  for (int i = lane; i < m; i += 32) t[i] = i < k ? w[row0 + i] : T(0);
  __syncwarp();
  for (int32_t ci = F.cbeg[f]; ci < F.cend[f]; ++ci) {
    const int32_t c = F.children[ci];
    const int32_t rc = F.m[c] - F.k[c];
    const int32_t* __restrict__ rel = F.rel + F.rel_off[c];
    const T* __restrict__ uc = u + F.upd[c];
    for (int i = lane; i < rc; i += 32) t[rel[i]] += uc[i];
    __syncwarp();
  }
  for (int i = lane; i < k; i += 32) y[i] = t[i] + warp_row_dot(A + i, m, 0, i, t);
  __syncwarp();
  T* __restrict__ uf = u + F.upd[f];
  for (int i = lane; i < m - k; i += 32) uf[i] = t[k + i] - warp_row_dot(A + k + i, m, 0, k, y);
  for (int i = lane; i < k; i += 32) w[row0 + i] = y[i];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_bwd1w(DevFronts F, const int32_t* __restrict__ list, int32_t nf, int32_t ldt,
            const T* __restrict__ arena, T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (kThreads / 32) + warp;
  T* t = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * ldt;  // k entries, then x_upd (r)
  const bool live = q < nf;
  int32_t f = 0, k = 0, m = 0;
  if (live) {
    f = list[q];
    k = F.k[f];
    m = F.m[f];
  }
  pdl_wait();
  if (!live) return;
  const int32_t r = m - k;
  const T* __restrict__ A = arena + F.arena[f];
  const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
  const int64_t row0 = F.row0[f];
  T* xu = t + k;
  for (int j = lane; j < r; j += 32) xu[j] = w[idx[k + j]];
  __syncwarp();
  for (int i = lane; i < k; i += 32)
    t[i] = w[row0 + i] - warp_row_dot(A + i + (int64_t)k * m, m, 0, r, xu);
  __syncwarp();
  for (int i = lane; i < k; i += 32) w[row0 + i] = warp_row_dot(A + i, m, i, k, t);
}

// ---------------------------------------------------------------------------
// Persistent sweeps over the deep levels of the elimination forest, where
// every front has at most kPersistM rows: one launch per sweep instead of
// one per depth.  Each warp takes the next front of a topological order
// (children before parents forward, parents before children backward) from
// an atomic counter, waits until the fronts it depends on have raised their
// flags, does the front's work as the warp-per-front kernels above do, and
// raises its own flag.  A front's dependencies were handed out before it,
// to warps already running, so every wait ends; each wait is still bounded
// (kPersistSpin polls) and a wait that runs out records code 2 in err,
// raises the flag anyway and lets the sweep finish.  Data another warp of the
// same launch wrote is read with ld.global.cg (L2, not a stale L1 line).
// ---------------------------------------------------------------------------
constexpr uint32_t kPersistSpin = 1u << 22;

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Every lane polls the flag (acquire); false when the bounded wait ran out.
__device__ __forceinline__ bool wait_flag(const int32_t* flag, long long* err) {
  uint32_t n = 0;
  while (ld_acquire(flag) == 0) {
    if (++n > kPersistSpin) {
      atomicCAS((unsigned long long*)err, 0ull, 2ull);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_fwd_persist(DevFronts F, const int32_t* __restrict__ order, int32_t nitems, int32_t ldt,
                  const T* __restrict__ arena, T* __restrict__ w, T* __restrict__ u,
                  int32_t* __restrict__ done, int32_t* __restrict__ next, long long* err) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* t = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * ldt;  // m entries, then y (k)
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(next, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= nitems) return;
    const int32_t f = order[q];
    const int32_t k = F.k[f], m = F.m[f];
    const T* __restrict__ A = arena + F.arena[f];
    const int64_t row0 = F.row0[f];
    T* y = t + m;
    for (int32_t ci = F.cbeg[f]; ci < F.cend[f]; ++ci) wait_flag(done + F.children[ci], err);
    for (int i = lane; i < m; i += 32) t[i] = i < k ? ldcg(w + row0 + i) : T(0);
    __syncwarp();
    for (int32_t ci = F.cbeg[f]; ci < F.cend[f]; ++ci) {
      const int32_t c = F.children[ci];
      const int32_t rc = F.m[c] - F.k[c];
      const int32_t* __restrict__ rel = F.rel + F.rel_off[c];
      const T* uc = u + F.upd[c];
      for (int i = lane; i < rc; i += 32) t[rel[i]] += ldcg(uc + i);
      __syncwarp();
    }
    for (int i = lane; i < k; i += 32) y[i] = t[i] + warp_row_dot(A + i, m, 0, i, t);
    __syncwarp();
    T* __restrict__ uf = u + F.upd[f];
    for (int i = lane; i < m - k; i += 32) uf[i] = t[k + i] - warp_row_dot(A + k + i, m, 0, k, y);
    for (int i = lane; i < k; i += 32) w[row0 + i] = y[i];
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(done + f, 1);
    __syncwarp();
  }
}

// wait_on[f]: the parent whose pivots front f reads, when it is swept by the
// same launch; -1 when it was done before the launch (or f is a root).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_bwd_persist(DevFronts F, const int32_t* __restrict__ order, int32_t nitems, int32_t ldt,
                  const int32_t* __restrict__ wait_on, const T* __restrict__ arena,
                  T* __restrict__ w, int32_t* __restrict__ done, int32_t* __restrict__ next,
                  long long* err) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* t = reinterpret_cast<T*>(smem_raw) + (int64_t)warp * ldt;  // k entries, then x_upd (r)
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(next, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= nitems) return;
    const int32_t f = order[q];
    const int32_t k = F.k[f], m = F.m[f], r = m - k;
    if (wait_on[f] >= 0) wait_flag(done + wait_on[f], err);
    const T* __restrict__ A = arena + F.arena[f];
    const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
    const int64_t row0 = F.row0[f];
    T* xu = t + k;
    for (int j = lane; j < r; j += 32) xu[j] = ldcg(w + idx[k + j]);
    __syncwarp();
    for (int i = lane; i < k; i += 32)
      t[i] = ldcg(w + row0 + i) - warp_row_dot(A + i + (int64_t)k * m, m, 0, r, xu);
    __syncwarp();
    for (int i = lane; i < k; i += 32) w[row0 + i] = warp_row_dot(A + i, m, i, k, t);
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(done + f, 1);
    __syncwarp();
  }
}

// CSR product streamed by row blocks: y = A x (SUB 0) or y = b - A x (SUB 1).
// A CTA takes kStreamRows consecutive rows; their entries are contiguous,
// [rowptr[r0], rowptr[r1]), and are read with coalesced loads (thread t the
// entries t, t + NT, ...; four in flight), the products val * x[col] going
// to shared memory; then thread t adds its row's products in order.  A row
// block with more than kStreamCap entries is summed row by row from global
// memory instead.  Used for the outer products with A (Fig. 2 step 6) and
// the retrieval's y - R~ z^ (Fig. 3 6.4-6.5), whose R~ columns index z^.
constexpr int kStreamRows = 256;
constexpr int kStreamCap = 4096;

template <int SUB>
__global__ void __launch_bounds__(kStreamRows)
    k_csr_stream(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                 const double* __restrict__ vals, int64_t n, const double* __restrict__ x,
                 const double* __restrict__ b, double* __restrict__ y) {
  __shared__ double prod[kStreamCap];
  const int tid = threadIdx.x;
  for (int64_t r0 = (int64_t)blockIdx.x * kStreamRows; r0 < n;
       r0 += (int64_t)gridDim.x * kStreamRows) {
    const int64_t r1 = min(n, r0 + kStreamRows);
    const int64_t row = r0 + tid;
    const int32_t e0 = rowptr[r0], ne = rowptr[r1] - e0;
    int32_t ra = 0, rb = 0;
    if (row < r1) {
      ra = rowptr[row];
      rb = rowptr[row + 1];
    }
    double s = 0.0;
    if (ne <= kStreamCap) {
      int e = tid;
      for (; e + 3 * kStreamRows < ne; e += 4 * kStreamRows) {
        int32_t c[4];
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          c[q] = colind[e0 + e + q * kStreamRows];
          v[q] = vals[e0 + e + q * kStreamRows];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) prod[e + q * kStreamRows] = v[q] * x[c[q]];
      }
      for (; e < ne; e += kStreamRows) prod[e] = vals[e0 + e] * x[colind[e0 + e]];
      __syncthreads();
      for (int32_t j = ra - e0; j < rb - e0; ++j) s += prod[j];
      __syncthreads();
    } else {
      for (int32_t j = ra; j < rb; ++j) s += vals[j] * x[colind[j]];
    }
    if (row < r1) y[row] = SUB ? b[row] - s : s;
  }
}

// The same row blocks with every load of the block's entries issued at once:
// the entries from rowptr[r0] rounded down to a multiple of 4 are read in
// groups of 4 (one 16-byte load of column indices, two of values), up to
// kBlockGroups groups per thread, before any x is gathered; the products
// and the row sums are those of k_csr_stream, in the same order.
constexpr int kBlockGroups = kStreamCap / 4 / kStreamRows;

template <int SUB>
__global__ void __launch_bounds__(kStreamRows)
    k_csr_block(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                const double* __restrict__ vals, int64_t n, const double* __restrict__ x,
                const double* __restrict__ b, double* __restrict__ y) {
  __shared__ double prod[kStreamCap];
  const int tid = threadIdx.x;
  const int32_t nnz = rowptr[n];
  for (int64_t r0 = (int64_t)blockIdx.x * kStreamRows; r0 < n;
       r0 += (int64_t)gridDim.x * kStreamRows) {
    const int64_t r1 = min(n, r0 + kStreamRows);
    const int64_t row = r0 + tid;
    const int32_t e0 = rowptr[r0], e1 = rowptr[r1];
    const int32_t ea = e0 & ~3;
    int32_t ra = 0, rb = 0;
    if (row < r1) {
      ra = rowptr[row];
      rb = rowptr[row + 1];
    }
    double s = 0.0;
    if (e1 - ea <= kStreamCap) {
      int4 c[kBlockGroups];
      double2 v[kBlockGroups][2];
#pragma unroll
      for (int g = 0; g < kBlockGroups; ++g) {
        const int32_t e = ea + 4 * (tid + g * kStreamRows);
        if (e < e1) {
          if (e + 4 <= nnz) {
            c[g] = *reinterpret_cast<const int4*>(colind + e);
            v[g][0] = *reinterpret_cast<const double2*>(vals + e);
            v[g][1] = *reinterpret_cast<const double2*>(vals + e + 2);
          } else {  // the last entries of the matrix
            const int32_t l = nnz - 1;
            c[g] = make_int4(colind[e], colind[min(e + 1, l)], colind[min(e + 2, l)], colind[min(e + 3, l)]);
            v[g][0] = make_double2(vals[e], vals[min(e + 1, l)]);
            v[g][1] = make_double2(vals[min(e + 2, l)], vals[min(e + 3, l)]);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < kBlockGroups; ++g) {
        const int32_t e = ea + 4 * (tid + g * kStreamRows);
        if (e < e1) {
          const int32_t cc[4] = {c[g].x, c[g].y, c[g].z, c[g].w};
          const double vv[4] = {v[g][0].x, v[g][0].y, v[g][1].x, v[g][1].y};
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (e + j >= e0 && e + j < e1) prod[e + j - ea] = vv[j] * x[cc[j]];
        }
      }
      __syncthreads();
      for (int32_t j = ra - ea; j < rb - ea; ++j) s += prod[j];
      __syncthreads();
    } else {
      for (int32_t j = ra; j < rb; ++j) s += vals[j] * x[colind[j]];
    }
    if (row < r1) y[row] = SUB ? b[row] - s : s;
  }
}

// The same product by warps over 32 consecutive rows: the lanes copy the
// rows' entries (from rowptr[r0] rounded down to a multiple of 4, at most
// kWarpCap) into the warp's shared buffers with 16-byte asynchronous copies,
// which hold no registers, so that many warps keep their copies in flight;
// the products are formed in place, four entries per lane, and lane r sums
// row r's in order (the order and the rounding of k_csr_stream).  Longer
// row groups take the entries from global memory.
constexpr int kWarpRows = 32, kWarpCap = 512, kWarpWarps = 8;

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}

template <int SUB>
__global__ void __launch_bounds__(kWarpRows * kWarpWarps)
    k_csr_warp(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
               const double* __restrict__ vals, int64_t n, const double* __restrict__ x,
               const double* __restrict__ b, double* __restrict__ y) {
  __shared__ __align__(16) double sv_all[kWarpWarps][kWarpCap];
  __shared__ __align__(16) int32_t sc_all[kWarpWarps][kWarpCap];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* __restrict__ sv = sv_all[wib];
  int32_t* __restrict__ sc = sc_all[wib];
  const int32_t nnz = rowptr[n];
  const int64_t nch = (n + kWarpRows - 1) / kWarpRows;
  for (int64_t ch = (int64_t)blockIdx.x * kWarpWarps + wib; ch < nch;
       ch += (int64_t)gridDim.x * kWarpWarps) {
    const int64_t r0 = ch * kWarpRows, row = r0 + lane, r1 = min(n, r0 + kWarpRows);
    int32_t ra = 0, rb = 0;
    if (row < r1) {
      ra = rowptr[row];
      rb = rowptr[row + 1];
    }
    const int32_t e0 = __shfl_sync(0xffffffffu, ra, 0);
    const int32_t e1 = __shfl_sync(0xffffffffu, rb, (int)(r1 - r0 - 1));
    const int32_t ea = e0 & ~3;
    double s = 0.0;
    if (e1 - ea <= kWarpCap) {
      const int ng = (e1 - ea + 3) >> 2;
      for (int g = lane; g < ng; g += 32) {
        const int32_t e = ea + 4 * g;
        const int left = nnz - e;  // >= 1: e < e1 <= nnz
        cp_async16(sc + 4 * g, colind + e, 4 * min(4, left));
        cp_async16(sv + 4 * g, vals + e, 8 * min(2, left));
        if (left > 2) cp_async16(sv + 4 * g + 2, vals + e + 2, 8 * min(2, left - 2));
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
      // products in place, four entries per lane and group, every x gather of
      // a lane in flight at once
#pragma unroll
      for (int q = 0; q < kWarpCap / 128; ++q) {
        const int g = lane + 32 * q;
        if (g < ng) {
          const int4 c = *reinterpret_cast<const int4*>(sc + 4 * g);
          double2* pv = reinterpret_cast<double2*>(sv + 4 * g);
          const double2 v01 = pv[0], v23 = pv[1];
          const int32_t e = ea + 4 * g;
          const double x0 = e >= e0 ? x[c.x] : 0.0;
          const double x1 = e + 1 < e1 ? x[c.y] : 0.0;
          const double x2 = e + 2 < e1 ? x[c.z] : 0.0;
          const double x3 = e + 3 < e1 ? x[c.w] : 0.0;
          pv[0] = make_double2(__dmul_rn(v01.x, x0), __dmul_rn(v01.y, x1));
          pv[1] = make_double2(__dmul_rn(v23.x, x2), __dmul_rn(v23.y, x3));
        }
      }
      __syncwarp();
      for (int32_t j = ra - ea; j < rb - ea; ++j) s += sv[j];
      __syncwarp();  // read before the next group overwrites the buffers
    } else {
      for (int32_t j = ra; j < rb; ++j) s += __dmul_rn(vals[j], x[colind[j]]);
    }
    if (row < r1) y[row] = SUB ? b[row] - s : s;
  }
}

// The same product with LPR lanes per row (CSR-vector): the lanes of a row
// take its entries LPR apart, each with all of its (up to 4) loads in flight
// before the gathers of x, and the row sum is a shuffle reduction in
// registers (no shared memory).  A warp covers 32 / LPR consecutive rows.
template <int SUB, int LPR>
__global__ void __launch_bounds__(256)
    k_csr_vec(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
              const double* __restrict__ vals, int64_t n, const double* __restrict__ x,
              const double* __restrict__ b, double* __restrict__ y) {
  const int sub = threadIdx.x & (LPR - 1);
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPR; row < n;
       row += ((int64_t)gridDim.x * blockDim.x) / LPR) {
    const int32_t ra = rowptr[row], rb = rowptr[row + 1];
    double s = 0.0;
    for (int32_t e = ra + sub; e < rb; e += 4 * LPR) {
      int32_t c[4];
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t eq = e + q * LPR;
        c[q] = eq < rb ? colind[eq] : 0;
        v[q] = eq < rb ? vals[eq] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (e + q * LPR < rb) s += v[q] * x[c[q]];
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (sub == 0) y[row] = SUB ? b[row] - s : s;
  }
}

// q = R~ v for a reduced vector v (the implicit G^ product)
template <typename TI>
__global__ void k_rt_apply(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ val, int64_t n, const TI* __restrict__ v,
                           double* __restrict__ q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * (double)v[col[e]];
    q[i] = s;
  }
}

// w = v + g(c)
template <typename TI>
__global__ void k_add_gathered(const TI* __restrict__ v, const double* __restrict__ g,
                               const int64_t* __restrict__ c, int64_t m, TI* __restrict__ w) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x)
    w[j] = (TI)((double)v[j] + g[c[j]]);
}

template <typename T>
__device__ __forceinline__ float to_f(T v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_f<__half>(__half v) {
  return __half2float(v);
}

template <typename AT, typename TG>
__device__ __forceinline__ AT to_acc(TG v) {
  return (AT)v;
}
template <>
__device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_acc<float, __half>(__half v) {
  return __half2float(v);
}

template <typename TG>
struct Acc {
  using type = float;
};
template <>
struct Acc<double> {
  using type = double;
};

// w = v + G(c,c) v: one warp per reduced row; the row's coupling columns are
// gathered from v.  FP32 accumulation for FP32/BF16 storage, FP64 for FP64.
template <typename TG, typename TI>
__global__ void k_ghat_matvec(const TG* __restrict__ ghat, const int32_t* __restrict__ qblock,
                              const int64_t* __restrict__ gq0, const int64_t* __restrict__ gcol_ptr,
                              const int64_t* __restrict__ ghat_off, const int64_t* __restrict__ gld,
                              const int32_t* __restrict__ gcols, int64_t m,
                              const TI* __restrict__ v, TI* __restrict__ w) {
  using AT = typename Acc<TG>::type;
  const int lane = threadIdx.x & 31;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < m;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t b = qblock[q];
    const int64_t c0 = gcol_ptr[b];
    const int64_t nc = gcol_ptr[b + 1] - c0;
    const TG* __restrict__ row = ghat + ghat_off[b] + (q - gq0[b]) * gld[b];
    const int32_t* __restrict__ cols = gcols + c0;
    AT s = 0;
    for (int64_t j = lane; j < nc; j += 32) s += (AT)to_f(row[j]) * (AT)v[cols[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[q] = (TI)((AT)v[q] + s);
  }
}

template <>
__global__ void k_ghat_matvec<double, double>(const double* __restrict__ ghat,
                                              const int32_t* __restrict__ qblock,
                                              const int64_t* __restrict__ gq0,
                                              const int64_t* __restrict__ gcol_ptr,
                                              const int64_t* __restrict__ ghat_off,
                                              const int64_t* __restrict__ gld,
                                              const int32_t* __restrict__ gcols, int64_t m,
                                              const double* __restrict__ v,
                                              double* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < m;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t b = qblock[q];
    const int64_t c0 = gcol_ptr[b];
    const int64_t nc = gcol_ptr[b + 1] - c0;
    const double* __restrict__ row = ghat + ghat_off[b] + (q - gq0[b]) * gld[b];
    const int32_t* __restrict__ cols = gcols + c0;
    double s = 0;
    for (int64_t j = lane; j < nc; j += 32) s += row[j] * v[cols[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[q] = v[q] + s;
  }
}

// w = v + G(c,c) v, tiled: one CTA per (block, up to 64 reduced rows).  The
// block's gathered vector v(c_i) is staged once in shared memory (float for
// FP32/BF16 storage, double for FP64); each warp streams whole rows of G^
// with 16-byte loads (8 rows of a tile per warp, two rows in flight).
template <typename TG>
struct Vec16;
template <>
struct Vec16<float> {
  static constexpr int n = 4;
};
template <>
struct Vec16<__nv_bfloat16> {
  static constexpr int n = 8;
};
template <>
struct Vec16<double> {
  static constexpr int n = 2;
};
template <>
struct Vec16<__half> {
  static constexpr int n = 8;
};

template <typename TG>
__device__ __forceinline__ void load16(const TG* p, float* out);
template <>
__device__ __forceinline__ void load16<float>(const float* p, float* out) {
  const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
  out[0] = v.x;
  out[1] = v.y;
  out[2] = v.z;
  out[3] = v.w;
}
template <>
__device__ __forceinline__ void load16<__nv_bfloat16>(const __nv_bfloat16* p, float* out) {
  const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = __uint_as_float(w[i] << 16);
    out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

template <>
__device__ __forceinline__ void load16<__half>(const __half* p, float* out) {
  const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 h2 = *reinterpret_cast<const __half2*>(&w[i]);
    const float2 f2 = __half22float2(h2);
    out[2 * i] = f2.x;
    out[2 * i + 1] = f2.y;
  }
}

template <typename TG, typename TI>
__global__ void __launch_bounds__(256, 4)
    k_ghat_matvec_tiled(const TG* __restrict__ ghat, const int32_t* __restrict__ tile_block,
                        const int32_t* __restrict__ tile_row, const int32_t* __restrict__ tile_h,
                        const int64_t* __restrict__ gq0,
                        const int64_t* __restrict__ gq1, const int64_t* __restrict__ gcol_ptr,
                        const int64_t* __restrict__ ghat_off, const int64_t* __restrict__ gld,
                        const int32_t* __restrict__ gcols,
                        const TI* __restrict__ v, TI* __restrict__ w, const KScal* __restrict__ sc,
                        const int32_t* __restrict__ block_sys, MvRed R) {
  using AT = typename Acc<TG>::type;
  constexpr int VN = Vec16<TG>::n;
  extern __shared__ unsigned char smem_raw[];
  AT* xs = reinterpret_cast<AT*>(smem_raw);
  const int32_t b = tile_block[blockIdx.x];
  if (sc && !sc[block_sys[b]].active) return;  // this system's inner solve has stopped
  const int64_t r0 = tile_row[blockIdx.x];
  const int64_t c0 = gcol_ptr[b];
  const int64_t nc = gcol_ptr[b + 1] - c0;
  const int64_t nrows = gq1[b] - gq0[b];
  for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) xs[j] = (AT)v[gcols[c0 + j]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TG* __restrict__ base = ghat + ghat_off[b];
  const int64_t nvec = nc / VN;
  const int64_t ld = gld[b];
  const int64_t q0 = gq0[b];
  // each warp streams four rows at once (the last group of a block repeats
  // its last valid row), two 16-byte loads per row and lane in flight
  const int th = tile_h[blockIdx.x];
  for (int rr = warp * 4; rr < th; rr += 32) {
    const int64_t ra = r0 + rr;
    if (ra >= nrows) break;
    const int nv = (int)min((int64_t)4, nrows - ra);
    const TG* __restrict__ p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) p[u] = base + (ra + min(u, nv - 1)) * ld;
    AT s4[4] = {0, 0, 0, 0};
#pragma unroll 2
    for (int64_t q = lane; q < nvec; q += 32) {
      AT g[4][VN];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if constexpr (sizeof(TG) == 8) {
          const double2 t = __ldcs(reinterpret_cast<const double2*>(p[u] + q * VN));
          g[u][0] = t.x;
          g[u][1] = t.y;
        } else {
          float tmp[VN];
          load16<TG>(p[u] + q * VN, tmp);
#pragma unroll
          for (int e = 0; e < VN; ++e) g[u][e] = tmp[e];
        }
      }
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        const AT xv = xs[q * VN + e];
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += g[u][e] * xv;
      }
    }
    for (int64_t j = nvec * VN + lane; j < nc; j += 32) {  // ragged tail
#pragma unroll
      for (int u = 0; u < 4; ++u) s4[u] += to_acc<AT>(p[u][j]) * xs[j];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s4[u] += __shfl_xor_sync(0xffffffffu, s4[u], o);
    if (lane == 0)
      for (int u = 0; u < nv; ++u) w[q0 + ra + u] = (TI)((AT)v[q0 + ra + u] + s4[u]);
  }
  if (R.nred) {
    // after the product: the tile's partial sums (its rows strided over the
    // threads, warps in order), then the system's, by the last of its tiles
    // to finish (tiles in order), and its scalar step
    __shared__ double part[2][8];
    __shared__ int last;
    __syncthreads();  // the tile's entries of w are written
    double red0 = 0.0, red1 = 0.0;
    const int nrt = (int)min((int64_t)th, nrows - r0);
    for (int i = threadIdx.x; i < nrt; i += blockDim.x) {
      const int64_t q = q0 + r0 + i;
      const double wv = (double)w[q];
      if (R.nred == 1) {
        red0 += (double)reinterpret_cast<const TI*>(R.x)[q] * wv;
      } else {
        red0 += wv * (double)v[q];
        red1 += wv * wv;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      red0 += __shfl_xor_sync(0xffffffffu, red0, o);
      red1 += __shfl_xor_sync(0xffffffffu, red1, o);
    }
    if (lane == 0) {
      part[0][warp] = red0;
      part[1][warp] = red1;
    }
    __syncthreads();
    const int32_t sys = block_sys[b];
    const int32_t t0 = R.sys_tptr[sys], t1 = R.sys_tptr[sys + 1];
    if (threadIdx.x == 0) {
      double a0 = part[0][0], a1 = part[1][0];
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
        a0 += part[0][q];
        a1 += part[1][q];
      }
      R.partial[blockIdx.x] = a0;
      R.partial[gridDim.x + blockIdx.x] = a1;
      __threadfence();
      last = atomicAdd(&R.done[sys], 1) == t1 - t0 - 1;
    }
    __syncthreads();
    if (last && warp == 0) {
      __threadfence();
      double s0 = 0.0, s1 = 0.0;
      for (int t = t0 + lane; t < t1; t += 32) {
        s0 += __ldcg(R.partial + t);
        s1 += __ldcg(R.partial + gridDim.x + t);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (lane == 0) {
        KScal& k = R.sc[sys];
        if (R.nred == 1) {
          k.sigma = s0;
        } else {
          k.ts = s0;
          k.tt = s1;
        }
        post_step(k, R.post, R.tol, R.it);
        R.done[sys] = 0;
      }
    }
  }
}

__global__ void k_gather(const double* __restrict__ src, const int64_t* __restrict__ idx, int64_t m,
                         double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

}  // namespace

template <typename T>
void launch_permute_in(const double* y, const int32_t* perm, int64_t n, T* w, cudaStream_t s) {
  k_permute_in<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(y, perm, n, w);
}
template <typename T>
void launch_permute_out(const T* w, const int32_t* perm, int64_t n, double* g, cudaStream_t s) {
  k_permute_out<T><<<grid_for(n, kThreads), kThreads, 0, s>>>(w, perm, n, g);
}

static int sm_count() { return device_sm_count(); }

// One launch per depth of the elimination forest, 256 threads per front.
// Levels with more fronts than two per SM keep eight loads in flight per
// lane (more CTAs resident); the others take a cluster of up to eight CTAs
// per front, within two CTAs per SM (always eight for very large fronts),
// and kSolveB loads per lane.
template <typename K, typename... Args>
static void launch_clustered(K kern, int32_t nf, int c, size_t sm, cudaStream_t s, Args... args) {
  if (sm > 48 * 1024)
    record_launch_error(
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nf * c));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)c;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  record_launch_error(cudaLaunchKernelEx(&cfg, kern, args...));
}
// Fronts of 1024 rows or more always take a full cluster: one CTA cannot
// stream their blocks fast enough, however many fronts share the depth.
constexpr int kHugeSolveM = 1024;
static bool wide_solve_level(int32_t nf, int32_t max_m) {
  return nf > 2 * sm_count() && max_m < kHugeSolveM;
}
static int solve_cluster(int32_t nf, int32_t max_m) {
  if (max_m >= kHugeSolveM) return 8;
  int c = 1;
  while (c < 8 && (int64_t)nf * c * 2 <= 2 * (int64_t)sm_count()) c *= 2;
  return c;
}
constexpr int kSolveCh = 256;
// loads in flight per lane in the cluster kernels of the block solve, and
// the rows they take per block-wide step (fewer barriers than kSolveCh)
constexpr int kSolveB = 32;
constexpr int kSolveChW = 512;
constexpr int kSolveRed = 8 * kSolveCh;
constexpr int kSolveRedW = 8 * kSolveChW;

// Depths of many fronts of at most kWarpSolveM rows take a warp per front.
constexpr int kWarpSolveM = 128;
static bool warp_solve_level(int32_t nf, int32_t max_m) {
  return max_m <= kWarpSolveM && nf > 2 * sm_count();
}

// Launch shape of one depth's sweep: SOLVE_AUTO picks from the front count
// and size (warp per front for many small fronts, one CTA with eight loads in
// flight per lane for many fronts, else clusters); the autotuner may fix it.
template <typename T>
void launch_fwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, T* u, cudaStream_t s, int cfg) {
  if (nf <= 0) return;
  if (cfg == SOLVE_AUTO)
    cfg = warp_solve_level(nf, max_m) ? SOLVE_WARP
          : wide_solve_level(nf, max_m) ? SOLVE_CTA8
                                        : solve_cfg_cluster(solve_cluster(nf, max_m));
  if (cfg == SOLVE_WARP && max_m <= kWarpSolveM) {
    const int32_t ldt = 2 * max_m;
    const size_t smw = (size_t)(kThreads / 32) * ldt * sizeof(T);
    const int32_t grid = (nf + kThreads / 32 - 1) / (kThreads / 32);
    launch_clustered(k_fwd1w<T>, grid, 1, smw, s, F, list, nf, ldt, arena, w, u);
    return;
  }
  if (cfg == SOLVE_CTA8)
    launch_clustered(k_fwd1<T, kThreads, kSolveCh, 8, 8>, nf, 1,
                     ((size_t)2 * max_m + kSolveRed) * sizeof(T), s, F, list, arena, w, u);
  else
    launch_clustered(k_fwd1<T, kThreads, kSolveChW, 8, kSolveB>, nf, solve_cfg_size(cfg),
                     ((size_t)2 * max_m + kSolveRedW) * sizeof(T), s, F, list, arena, w, u);
}
template <typename T>
void launch_bwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, cudaStream_t s, int cfg) {
  if (nf <= 0) return;
  if (cfg == SOLVE_AUTO)
    cfg = warp_solve_level(nf, max_m) ? SOLVE_WARP
          : wide_solve_level(nf, max_m) ? SOLVE_CTA8
                                        : solve_cfg_cluster(solve_cluster(nf, max_m));
  if (cfg == SOLVE_WARP && max_m <= kWarpSolveM) {
    const int32_t ldt = max_m;
    const size_t smw = (size_t)(kThreads / 32) * ldt * sizeof(T);
    const int32_t grid = (nf + kThreads / 32 - 1) / (kThreads / 32);
    launch_clustered(k_bwd1w<T>, grid, 1, smw, s, F, list, nf, ldt, arena, w);
    return;
  }
  if (cfg == SOLVE_CTA8)
    launch_clustered(k_bwd1<T, kThreads, kSolveCh, 8, 8>, nf, 1,
                     ((size_t)max_m + kSolveRed) * sizeof(T), s, F, list, arena, w);
  else
    launch_clustered(k_bwd1<T, kThreads, kSolveChW, 8, kSolveB>, nf, solve_cfg_size(cfg),
                     ((size_t)max_m + kSolveRedW) * sizeof(T), s, F, list, arena, w);
}

// Persistent sweeps: enough warps for every front, at most eight CTAs of
// eight warps per SM (every warp of a launch that has taken a front is
// running, so the waits need no co-residency).
template <typename T>
void launch_fwd_persist(DevFronts F, const int32_t* order, int32_t nitems, int32_t max_m,
                        const T* arena, T* w, T* u, int32_t* done, int32_t* next, long long* err,
                        cudaStream_t s) {
  if (nitems <= 0) return;
  const int32_t ldt = 2 * max_m;
  const size_t sm = (size_t)(kThreads / 32) * ldt * sizeof(T);
  const int32_t grid = std::min<int32_t>((nitems + kThreads / 32 - 1) / (kThreads / 32),
                                         8 * sm_count());
  k_fwd_persist<T><<<grid, kThreads, sm, s>>>(F, order, nitems, ldt, arena, w, u, done, next, err);
}
template <typename T>
void launch_bwd_persist(DevFronts F, const int32_t* order, int32_t nitems, int32_t max_m,
                        const int32_t* wait_on, const T* arena, T* w, int32_t* done,
                        int32_t* next, long long* err, cudaStream_t s) {
  if (nitems <= 0) return;
  const int32_t ldt = max_m;
  const size_t sm = (size_t)(kThreads / 32) * ldt * sizeof(T);
  const int32_t grid = std::min<int32_t>((nitems + kThreads / 32 - 1) / (kThreads / 32),
                                         8 * sm_count());
  k_bwd_persist<T><<<grid, kThreads, sm, s>>>(F, order, nitems, ldt, wait_on, arena, w, done,
                                              next, err);
}

// CSR products: `variant` SPMV_STREAM / SPMV_BLOCK (row blocks through shared
// memory), SPMV_WARP (32-row groups per warp, asynchronous copies) or
// SPMV_VEC4 / SPMV_VEC8 (4 or 8 lanes per row); chosen by the autotuner.
template <int SUB>
static void launch_csr(int variant, const int32_t* rowptr, const int32_t* colind,
                       const double* vals, int64_t n, const double* x, const double* b, double* y,
                       cudaStream_t s) {
  if (n <= 0) return;
  if (variant == SPMV_WARP)
    k_csr_warp<SUB><<<grid_for((n + kWarpRows - 1) / kWarpRows, kWarpWarps, 1 << 30),
                      kWarpRows * kWarpWarps, 0, s>>>(rowptr, colind, vals, n, x, b, y);
  else if (variant == SPMV_BLOCK)
    k_csr_block<SUB><<<grid_for(n, kStreamRows, 1 << 30), kStreamRows, 0, s>>>(rowptr, colind,
                                                                                vals, n, x, b, y);
  else if (variant == SPMV_VEC4)
    k_csr_vec<SUB, 4><<<grid_for(n * 4, 256, 1 << 30), 256, 0, s>>>(rowptr, colind, vals, n, x, b, y);
  else if (variant == SPMV_VEC8)
    k_csr_vec<SUB, 8><<<grid_for(n * 8, 256, 1 << 30), 256, 0, s>>>(rowptr, colind, vals, n, x, b, y);
  else
    k_csr_stream<SUB><<<grid_for(n, kStreamRows, 1 << 30), kStreamRows, 0, s>>>(rowptr, colind,
                                                                                 vals, n, x, b, y);
}

void launch_spmv(const int32_t* rowptr, const int32_t* colind, const double* vals, int64_t n,
                 const double* x, double* y, cudaStream_t s, int variant) {
  launch_csr<0>(variant, rowptr, colind, vals, n, x, nullptr, y, s);
}

void launch_rt_residual(const int32_t* rt_rowptr, const int32_t* rt_col, const double* rt_val,
                        int64_t n, const double* y, const double* zhat, double* out,
                        cudaStream_t s, int variant) {
  launch_csr<1>(variant, rt_rowptr, rt_col, rt_val, n, zhat, y, out, s);
}

template <typename TI>
void launch_rt_apply(const int32_t* rt_rowptr, const int32_t* rt_col, const double* rt_val,
                     int64_t n, const TI* v, double* q, cudaStream_t s) {
  if (n <= 0) return;
  k_rt_apply<TI><<<grid_for(n, kThreads), kThreads, 0, s>>>(rt_rowptr, rt_col, rt_val, n, v, q);
}
template <typename TI>
void launch_add_gathered(const TI* v, const double* g, const int64_t* c, int64_t m, TI* w,
                         cudaStream_t s) {
  if (m <= 0) return;
  k_add_gathered<TI><<<grid_for(m, kThreads), kThreads, 0, s>>>(v, g, c, m, w);
}
template void launch_rt_apply<float>(const int32_t*, const int32_t*, const double*, int64_t,
                                     const float*, double*, cudaStream_t);
template void launch_rt_apply<double>(const int32_t*, const int32_t*, const double*, int64_t,
                                      const double*, double*, cudaStream_t);
template void launch_add_gathered<float>(const float*, const double*, const int64_t*, int64_t,
                                         float*, cudaStream_t);
template void launch_add_gathered<double>(const double*, const double*, const int64_t*, int64_t,
                                          double*, cudaStream_t);

template <typename TG, typename TI>
void launch_ghat_matvec(const TG* ghat, const int32_t* qblock, const int64_t* gq0,
                        const int64_t* gcol_ptr, const int64_t* ghat_off, const int64_t* gld,
                        const int32_t* gcols, int64_t m, const TI* v, TI* w, cudaStream_t s) {
  if (m <= 0) return;
  k_ghat_matvec<TG, TI><<<grid_for(m * 32, kThreads), kThreads, 0, s>>>(
      ghat, qblock, gq0, gcol_ptr, ghat_off, gld, gcols, m, v, w);
}

template <typename TG, typename TI>
void launch_ghat_matvec_tiled(const TG* ghat, const int32_t* tile_block, const int32_t* tile_row,
                              const int32_t* tile_h, int32_t ntiles, int64_t max_cols,
                              const int64_t* gq0,
                              const int64_t* gq1, const int64_t* gcol_ptr, const int64_t* ghat_off,
                              const int64_t* gld, const int32_t* gcols, const TI* v, TI* w,
                              const KScal* sc, const int32_t* block_sys, const MvRed* red,
                              cudaStream_t s) {
  if (ntiles <= 0) return;
  using AT = typename Acc<TG>::type;
  const size_t sm = (size_t)std::max<int64_t>(max_cols, 1) * sizeof(AT);
  if (sm > 48 * 1024)
    record_launch_error(cudaFuncSetAttribute(k_ghat_matvec_tiled<TG, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm));
  k_ghat_matvec_tiled<TG, TI><<<ntiles, 256, sm, s>>>(ghat, tile_block, tile_row, tile_h, gq0, gq1,
                                                       gcol_ptr, ghat_off, gld, gcols, v, w, sc,
                                                       block_sys, red ? *red : MvRed{});
}

void launch_gather(const double* src, const int64_t* idx, int64_t m, double* dst, cudaStream_t s) {
  if (m <= 0) return;
  k_gather<<<grid_for(m, kThreads), kThreads, 0, s>>>(src, idx, m, dst);
}

void launch_gather_rt_values(const double* values, const int64_t* rt_src, int64_t nrt,
                             double* rt_val, cudaStream_t s) {
  if (nrt <= 0) return;
  k_gather<<<grid_for(nrt, kThreads), kThreads, 0, s>>>(values, rt_src, nrt, rt_val);
}

#define DDPS_INST_P(T)                                                                          \
  template void launch_fwd_persist<T>(DevFronts, const int32_t*, int32_t, int32_t, const T*, T*, \
                                      T*, int32_t*, int32_t*, long long*, cudaStream_t);         \
  template void launch_bwd_persist<T>(DevFronts, const int32_t*, int32_t, int32_t,              \
                                      const int32_t*, const T*, T*, int32_t*, int32_t*,          \
                                      long long*, cudaStream_t);
DDPS_INST_P(double)
DDPS_INST_P(float)

#define DDPS_INST_S(T)                                                                          \
  template void launch_permute_in<T>(const double*, const int32_t*, int64_t, T*, cudaStream_t); \
  template void launch_permute_out<T>(const T*, const int32_t*, int64_t, double*, cudaStream_t);\
  template void launch_fwd1<T>(DevFronts, const int32_t*, int32_t, int32_t, const T*, T*, T*,   \
                               cudaStream_t, int);                                              \
  template void launch_bwd1<T>(DevFronts, const int32_t*, int32_t, int32_t, const T*, T*,       \
                               cudaStream_t, int);
DDPS_INST_S(double)
DDPS_INST_S(float)

#define DDPS_INST_MV(TG, TI)                                                                     \
  template void launch_ghat_matvec_tiled<TG, TI>(const TG*, const int32_t*, const int32_t*,      \
                                                 const int32_t*, int32_t,                        \
                                                 int64_t, const int64_t*, const int64_t*,        \
                                                 const int64_t*, const int64_t*, const int64_t*, \
                                                 const int32_t*, const TI*, TI*, const KScal*,   \
                                                 const int32_t*, const MvRed*, cudaStream_t);
DDPS_INST_MV(double, double)
DDPS_INST_MV(float, double)
DDPS_INST_MV(float, float)
DDPS_INST_MV(__nv_bfloat16, float)
DDPS_INST_MV(__nv_bfloat16, double)
DDPS_INST_MV(__half, float)
DDPS_INST_MV(__half, double)

#define DDPS_INST_MV0(TG, TI)                                                                    \
  template void launch_ghat_matvec<TG, TI>(const TG*, const int32_t*, const int64_t*,           \
                                           const int64_t*, const int64_t*, const int64_t*,      \
                                           const int32_t*, int64_t, const TI*, TI*, cudaStream_t);
DDPS_INST_MV0(double, double)
DDPS_INST_MV0(float, double)
DDPS_INST_MV0(float, float)
DDPS_INST_MV0(__nv_bfloat16, float)
DDPS_INST_MV0(__nv_bfloat16, double)
DDPS_INST_MV0(__half, float)
DDPS_INST_MV0(__half, double)

}  // namespace ddps
