// Solve-phase kernels of DDPS: the block solves of Fig. 3 (6.1 and the
// retrieval 6.5 written as z = D~^-1 (y - R~ z^)), the products with A (outer
// Krylov, Fig. 2 step 6) and with R~, and the reduced product w = G^ v of 6.3.
#include <cuda_runtime.h>

#include <algorithm>

#include "krylov.h"
#include "launch.h"

namespace ddps {

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

// Forward substitution for one front per CTA, with the inverse of the unit
// lower diagonal block formed at factor time.  The front vector t (shared
// memory) starts with the pivot entries of w and zeros and receives the
// children's update vectors; then y = L11^-1 t(piv) goes back to w and the
// update entries t(upd) - L21 y go to u for the parent.
// sum_{j0 <= j < j1} A[i + j m] x[j] (A column-major with leading dimension
// m, x in shared memory): eight loads in flight and four partial sums, so
// that a long row costs a few memory latencies rather than one per term.
template <typename T>
__device__ __forceinline__ T dot_row(const T* __restrict__ A, int64_t m, int i, int j0, int j1,
                                     const T* x) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  int j = j0;
  for (; j + 8 <= j1; j += 8) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = A[i + (int64_t)(j + u) * m];
    s0 += a[0] * x[j] + a[4] * x[j + 4];
    s1 += a[1] * x[j + 1] + a[5] * x[j + 5];
    s2 += a[2] * x[j + 2] + a[6] * x[j + 6];
    s3 += a[3] * x[j + 3] + a[7] * x[j + 7];
  }
  for (; j < j1; ++j) s0 += A[i + (int64_t)j * m] * x[j];
  return (s0 + s1) + (s2 + s3);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_fwd1(DevFronts F, const int32_t* __restrict__ list, const T* __restrict__ arena,
           T* __restrict__ w, T* __restrict__ u) {
  extern __shared__ unsigned char smem_raw[];
  T* t = reinterpret_cast<T*>(smem_raw);  // m entries
  const int32_t f = list[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f];
  T* y = t + m;                           // k entries
  const T* __restrict__ A = arena + F.arena[f];
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  for (int i = tid; i < m; i += blockDim.x) t[i] = i < k ? w[row0 + i] : T(0);
  __syncthreads();
  for (int32_t ci = F.cbeg[f]; ci < F.cend[f]; ++ci) {
    const int32_t c = F.children[ci];
    const int32_t rc = F.m[c] - F.k[c];
    const int32_t* __restrict__ rel = F.rel + F.rel_off[c];
    const T* __restrict__ uc = u + F.upd[c];
    for (int i = tid; i < rc; i += blockDim.x) t[rel[i]] += uc[i];
    __syncthreads();
  }
  for (int i = tid; i < k; i += blockDim.x) y[i] = t[i] + dot_row(A, m, i, 0, i, t);
  __syncthreads();
  for (int i = k + tid; i < m; i += blockDim.x) u[F.upd[f] + (i - k)] = t[i] - dot_row(A, m, i, 0, k, y);
  for (int i = tid; i < k; i += blockDim.x) w[row0 + i] = y[i];
}

// Backward substitution for one front per CTA: x_piv = U11^-1 (y_piv - U12 x_upd)
// with the inverse formed at factor time; x_upd are ancestor pivots of w.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_bwd1(DevFronts F, const int32_t* __restrict__ list, const T* __restrict__ arena,
           T* __restrict__ w) {
  extern __shared__ unsigned char smem_raw[];
  T* t = reinterpret_cast<T*>(smem_raw);
  const int32_t f = list[blockIdx.x];
  const int32_t k = F.k[f], m = F.m[f], r = m - k;
  const T* __restrict__ A = arena + F.arena[f];
  const int32_t* __restrict__ idx = F.idx + F.idx_off[f];
  const int64_t row0 = F.row0[f];
  const int tid = threadIdx.x;
  T* xu = t + k;
  for (int j = tid; j < r; j += blockDim.x) xu[j] = w[idx[k + j]];
  __syncthreads();
  for (int i = tid; i < k; i += blockDim.x) t[i] = w[row0 + i] - dot_row(A + (int64_t)k * m, m, i, 0, r, xu);
  __syncthreads();
  for (int i = tid; i < k; i += blockDim.x) w[row0 + i] = dot_row(A, m, i, i, k, t);
}

// y = A x, CSR, four lanes per row.
__global__ void k_spmv(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                       const double* __restrict__ vals, int64_t n, const double* __restrict__ x,
                       double* __restrict__ y) {
  const int sub = threadIdx.x & 3;
  for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 2; row < n;
       row += ((int64_t)gridDim.x * blockDim.x) >> 2) {
    double s = 0.0;
    for (int32_t e = rowptr[row] + sub; e < rowptr[row + 1]; e += 4) s += vals[e] * x[colind[e]];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (sub == 0) y[row] = s;
  }
}

// out = y - R~ zhat
__global__ void k_rt_residual(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const double* __restrict__ val, int64_t n,
                              const double* __restrict__ y, const double* __restrict__ zhat,
                              double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = y[i];
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) s -= val[e] * zhat[col[e]];
    out[i] = s;
  }
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
__global__ void __launch_bounds__(256)
    k_ghat_matvec_tiled(const TG* __restrict__ ghat, const int32_t* __restrict__ tile_block,
                        const int32_t* __restrict__ tile_row, const int64_t* __restrict__ gq0,
                        const int64_t* __restrict__ gq1, const int64_t* __restrict__ gcol_ptr,
                        const int64_t* __restrict__ ghat_off, const int64_t* __restrict__ gld,
                        const int32_t* __restrict__ gcols,
                        const TI* __restrict__ v, TI* __restrict__ w, const KScal* __restrict__ sc,
                        const int32_t* __restrict__ block_sys) {
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
  for (int rr = warp * 4; rr < 64; rr += 32) {
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

template <typename T>
void launch_fwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, T* u, cudaStream_t s) {
  if (nf <= 0) return;
  size_t sm = (size_t)2 * max_m * sizeof(T);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_fwd1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_fwd1<T><<<nf, kThreads, sm, s>>>(F, list, arena, w, u);
}
template <typename T>
void launch_bwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, cudaStream_t s) {
  if (nf <= 0) return;
  size_t sm = (size_t)max_m * sizeof(T);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_bwd1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_bwd1<T><<<nf, kThreads, sm, s>>>(F, list, arena, w);
}

void launch_spmv(const int32_t* rowptr, const int32_t* colind, const double* vals, int64_t n,
                 const double* x, double* y, cudaStream_t s) {
  k_spmv<<<grid_for(n * 4, kThreads), kThreads, 0, s>>>(rowptr, colind, vals, n, x, y);
}

void launch_rt_residual(const int32_t* rt_rowptr, const int32_t* rt_col, const double* rt_val,
                        int64_t n, const double* y, const double* zhat, double* out,
                        cudaStream_t s) {
  k_rt_residual<<<grid_for(n, kThreads), kThreads, 0, s>>>(rt_rowptr, rt_col, rt_val, n, y, zhat,
                                                            out);
}

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
                              int32_t ntiles, int64_t max_cols, const int64_t* gq0,
                              const int64_t* gq1, const int64_t* gcol_ptr, const int64_t* ghat_off,
                              const int64_t* gld, const int32_t* gcols, const TI* v, TI* w,
                              const KScal* sc, const int32_t* block_sys, cudaStream_t s) {
  if (ntiles <= 0) return;
  using AT = typename Acc<TG>::type;
  const size_t sm = (size_t)std::max<int64_t>(max_cols, 1) * sizeof(AT);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_ghat_matvec_tiled<TG, TI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
  k_ghat_matvec_tiled<TG, TI><<<ntiles, 256, sm, s>>>(ghat, tile_block, tile_row, gq0, gq1,
                                                       gcol_ptr, ghat_off, gld, gcols, v, w, sc,
                                                       block_sys);
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

#define DDPS_INST_S(T)                                                                          \
  template void launch_permute_in<T>(const double*, const int32_t*, int64_t, T*, cudaStream_t); \
  template void launch_permute_out<T>(const T*, const int32_t*, int64_t, double*, cudaStream_t);\
  template void launch_fwd1<T>(DevFronts, const int32_t*, int32_t, int32_t, const T*, T*, T*,   \
                               cudaStream_t);                                                   \
  template void launch_bwd1<T>(DevFronts, const int32_t*, int32_t, int32_t, const T*, T*,       \
                               cudaStream_t);
DDPS_INST_S(double)
DDPS_INST_S(float)

#define DDPS_INST_MV(TG, TI)                                                                     \
  template void launch_ghat_matvec_tiled<TG, TI>(const TG*, const int32_t*, const int32_t*, int32_t, \
                                                 int64_t, const int64_t*, const int64_t*,        \
                                                 const int64_t*, const int64_t*, const int64_t*, \
                                                 const int32_t*, const TI*, TI*, const KScal*,   \
                                                 const int32_t*, cudaStream_t);
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
