// Vector kernels of the two BiCGStab loops of DDPS (Fig. 2 step 6 outer loop,
// Fig. 3 step 6.3 inner loop; Sec. 4 names BiCGStab for both).  Vectors are
// segmented by system: every system of a batch keeps its own scalars
// (rho, alpha, omega, ...) and its own convergence flag.  Reductions are
// deterministic: fixed chunks, fixed tree inside a chunk, and the chunks of a
// segment summed in a fixed pattern by the CTA that finishes last.
#include <cuda_runtime.h>

#include <cfloat>

#include "krylov.h"

namespace ddps {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Result of the reductions of segment sgi from its chunks' partial values
// (lane l adds the chunks l, l + 32, ...; then a fixed shuffle tree), and
// the BiCGStab scalar step `post` of that segment; run by one warp.
__device__ void seg_finalize(const SegView& S, int sgi, int lane, int nred, const RedSpec* spec,
                             const double* partial, int post, KScal* sc, double tol, int it) {
  const int c0 = S.seg_chunk_ptr[sgi], c1 = S.seg_chunk_ptr[sgi + 1];
  for (int q = 0; q < nred; ++q) {
    double v = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) {
      const double pv = __ldcg(partial + (int64_t)q * S.nchunks + c);
      v = spec[q].op == 2 ? fmax(v, pv) : v + pv;
    }
    v = spec[q].op == 2 ? warp_max(v) : warp_sum(v);
    if (spec[q].op == 1) v = sqrt(v);
    if (lane == 0) spec[q].out[(int64_t)sgi * spec[q].stride] = v;
  }
  if (post == POST_NONE || lane != 0) return;
  post_step(sc[sgi], post, tol, it);
}

// The end of a chunk reduction, shared by the reduction kernel and the
// fused update-and-norm kernels: the CTA's per-thread values acc[q] are
// summed in a fixed tree into the chunk's partial; the last CTA of a segment
// to finish (counted in S.done) forms the segment's results and its scalar
// step, then re-arms the counter.
__device__ __forceinline__ void chunk_reduce_finalize(const SegView& S, int ch, int nred,
                                                      const RedSpec* spec, double* acc,
                                                      double* __restrict__ partial, int post,
                                                      KScal* sc, double tol, int it) {
  __shared__ double red[3][kThreads / 32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q >= nred) break;
    double v = spec[q].op == 2 ? warp_max(acc[q]) : warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  const int sgi = S.chunk_seg[ch];
  if (threadIdx.x < 3 && (int)threadIdx.x < nred) {
    const int q = threadIdx.x;
    double v = red[q][0];
    for (int w = 1; w < kThreads / 32; ++w) v = spec[q].op == 2 ? fmax(v, red[q][w]) : v + red[q][w];
    partial[(int64_t)q * S.nchunks + ch] = v;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nch = S.seg_chunk_ptr[sgi + 1] - S.seg_chunk_ptr[sgi];
    last = atomicAdd(&S.done[sgi], 1) == nch - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (warp == 0) {
    seg_finalize(S, sgi, lane, nred, spec, partial, post, sc, tol, it);
    if (lane == 0) S.done[sgi] = 0;
  }
}

// One CTA per chunk: up to three reductions in one pass.
//   op 0: sum x*y   op 1: sum x*x   op 2: max |x|
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_seg_reduce(SegView S, int nred, RedSpec r0, RedSpec r1, RedSpec r2,
                 double* __restrict__ partial, int post, KScal* sc, double tol, int it) {
  const int ch = blockIdx.x;
  const int64_t b = S.chunk_beg[ch], e = S.chunk_end[ch];
  RedSpec spec[3] = {r0, r1, r2};
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q >= nred) break;
      const T* x = (const T*)spec[q].x;
      const T* y = (const T*)spec[q].y;
      const double xv = (double)x[i];
      if (spec[q].op == 0)
        acc[q] += xv * (double)y[i];
      else if (spec[q].op == 1)
        acc[q] += xv * xv;
      else
        acc[q] = fmax(acc[q], fabs(xv));
    }
  }
  chunk_reduce_finalize(S, ch, nred, spec, acc, partial, post, sc, tol, it);
}

// s = r - alpha v and ||s||_2 with the half-step check (POST_CHECK_HALF), in
// one pass: the same values and summation order as update_s followed by the
// reduction.  Segments that are not iterating are skipped whole.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_update_s_norm(SegView S, KScal* sc, const T* __restrict__ r, const T* __restrict__ v,
                    T* __restrict__ s_out, double* __restrict__ partial, double tol, int it) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!sc[sg].active) return;
  const double alpha = sc[sg].alpha;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x) {
    const T sv = (T)((double)r[i] - alpha * (double)v[i]);
    s_out[i] = sv;
    const double xv = (double)sv;
    acc[0] += xv * xv;
  }
  const RedSpec spec[1] = {RedSpec{s_out, nullptr, 1, kScalStride, &sc[0].nrm}};
  chunk_reduce_finalize(S, ch, 1, spec, acc, partial, POST_CHECK_HALF, sc, tol, it);
}

// The full step of update_xr_final and ||r||_2 with the full-step check
// (POST_CHECK_FULL), in one pass.  Segments neither iterating nor stopped at
// this half step are skipped whole (their check only clears half_done,
// which is already clear).
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_update_xr_norm(SegView S, KScal* sc, T* __restrict__ x, const T* __restrict__ p,
                     const T* __restrict__ sv, T* __restrict__ r, const T* __restrict__ t,
                     const T* __restrict__ rh, double* __restrict__ partial, double tol, int it) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  const bool act = sc[sg].active != 0, half = sc[sg].half_done != 0;
  if (!act && !half) return;
  const double alpha = sc[sg].alpha, omega = sc[sg].omega;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x) {
    T ri;
    if (act) {
      x[i] = (T)((double)x[i] + alpha * (double)p[i] + omega * (double)sv[i]);
      ri = (T)((double)sv[i] - omega * (double)t[i]);
      r[i] = ri;
    } else {
      x[i] = (T)((double)x[i] + alpha * (double)p[i]);
      ri = r[i];
    }
    const double xv = (double)ri;
    acc[0] += xv * xv;
    if (rh) acc[1] += (double)rh[i] * xv;
  }
  const RedSpec spec[2] = {RedSpec{r, nullptr, 1, kScalStride, &sc[0].nrm},
                           RedSpec{rh, r, 0, kScalStride, &sc[0].rho}};
  chunk_reduce_finalize(S, ch, rh ? 2 : 1, spec, acc, partial,
                        rh ? POST_CHECK_FULL_BETA : POST_CHECK_FULL, sc, tol, it);
}

template <typename T>
__global__ void k_update_xr_final(SegView S, const KScal* __restrict__ sc, T* __restrict__ x,
                                  const T* __restrict__ p, const T* __restrict__ sv,
                                  T* __restrict__ r, const T* __restrict__ t) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  const bool act = sc[sg].active != 0, half = sc[sg].half_done != 0;
  if (!act && !half) return;
  const double alpha = sc[sg].alpha, omega = sc[sg].omega;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x) {
    if (act) {
      x[i] = (T)((double)x[i] + alpha * (double)p[i] + omega * (double)sv[i]);
      r[i] = (T)((double)sv[i] - omega * (double)t[i]);
    } else {
      x[i] = (T)((double)x[i] + alpha * (double)p[i]);
    }
  }
}

__global__ void k_any_active(int nseg, const KScal* __restrict__ sc, int32_t* __restrict__ flag) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < nseg; g += blockDim.x)
    if (sc[g].active) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) *flag = any;
}

// ---- element-wise updates, one CTA per chunk, skipped for inactive segments ----

template <typename T>
__global__ void k_update_p(SegView S, const KScal* __restrict__ sc, const T* __restrict__ r,
                           T* __restrict__ p, const T* __restrict__ v) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!sc[sg].active) return;
  const double beta = sc[sg].beta, omega = sc[sg].omega;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x)
    p[i] = (T)((double)r[i] + beta * ((double)p[i] - omega * (double)v[i]));
}

template <typename T>
__global__ void k_update_s(SegView S, const KScal* __restrict__ sc, const T* __restrict__ r,
                           const T* __restrict__ v, T* __restrict__ s) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!sc[sg].active) return;
  const double alpha = sc[sg].alpha;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x)
    s[i] = (T)((double)r[i] - alpha * (double)v[i]);
}

// x += alpha phat (+ omega shat); r = s - omega t.  With half = 1 only the
// first term is applied, for the segments whose flag `half_done` is set.
template <typename T>
__global__ void k_update_xr(SegView S, const KScal* __restrict__ sc, int half, T* __restrict__ x,
                            const T* __restrict__ phat, const T* __restrict__ shat,
                            T* __restrict__ r, const T* __restrict__ s, const T* __restrict__ t) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (half) {
    if (!sc[sg].half_done) return;
  } else if (!sc[sg].active) {
    return;
  }
  const double alpha = sc[sg].alpha, omega = sc[sg].omega;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x) {
    if (half) {
      x[i] = (T)((double)x[i] + alpha * (double)phat[i]);
    } else {
      x[i] = (T)((double)x[i] + alpha * (double)phat[i] + omega * (double)shat[i]);
      r[i] = (T)((double)s[i] - omega * (double)t[i]);
    }
  }
}

// dst = a - b (segments marked active, or all with all = 1)
template <typename T>
__global__ void k_sub(SegView S, const KScal* __restrict__ sc, int all, const T* __restrict__ a,
                      const T* __restrict__ b, T* __restrict__ dst) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!all && !sc[sg].active) return;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x)
    dst[i] = (T)((double)a[i] - (double)b[i]);
}

template <typename T>
__global__ void k_masked_axpy(SegView S, const KScal* __restrict__ sc, T* __restrict__ dst,
                              const T* __restrict__ a, const T* __restrict__ b) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!sc[sg].flag) return;
  const double alpha = sc[sg].alpha;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x)
    dst[i] = b ? (T)((double)a[i] + alpha * (double)b[i]) : a[i];
}

template <typename T>
__global__ void k_masked_zero(SegView S, const KScal* __restrict__ sc, T* __restrict__ dst) {
  const int ch = blockIdx.x;
  const int sg = S.chunk_seg[ch];
  if (!sc[sg].flag) return;
  for (int64_t i = S.chunk_beg[ch] + threadIdx.x; i < S.chunk_end[ch]; i += blockDim.x) dst[i] = T(0);
}

template <typename TD, typename TS>
__global__ void k_convert(int64_t n, const TS* __restrict__ src, TD* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

// Per-segment scalars.
__global__ void k_sc_beta(int nseg, KScal* sc, int first) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nseg || !sc[g].active) return;
  if (sc[g].rho == 0.0) sc[g].breakdown = 1;
  sc[g].beta = first ? 0.0 : (sc[g].rho / sc[g].rho_old) * (sc[g].alpha / sc[g].omega);
}
__global__ void k_sc_alpha(int nseg, KScal* sc) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nseg || !sc[g].active) return;
  if (sc[g].sigma == 0.0) {
    sc[g].breakdown = 1;
    sc[g].alpha = 0.0;
  } else {
    sc[g].alpha = sc[g].rho / sc[g].sigma;
  }
}
__global__ void k_sc_omega(int nseg, KScal* sc) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nseg || !sc[g].active) return;
  sc[g].omega = sc[g].tt != 0.0 ? sc[g].ts / sc[g].tt : 0.0;
  sc[g].rho_old = sc[g].rho;
}

}  // namespace

template <typename T>
void seg_reduce(const SegView& S, int nred, RedSpec r0, RedSpec r1, RedSpec r2, double* partial,
                cudaStream_t s) {
  if (S.nchunks == 0) return;
  k_seg_reduce<T><<<S.nchunks, kThreads, 0, s>>>(S, nred, r0, r1, r2, partial, POST_NONE, nullptr,
                                                 0.0, 0);
}

template <typename T>
void seg_reduce_post(const SegView& S, int nred, RedSpec r0, RedSpec r1, RedSpec r2,
                     double* partial, int post, KScal* sc, double tol, int it, cudaStream_t s) {
  if (S.nchunks > 0)
    k_seg_reduce<T><<<S.nchunks, kThreads, 0, s>>>(S, nred, r0, r1, r2, partial, post, sc, tol, it);
}

template <typename T>
void update_xr_final(const SegView& S, const KScal* sc, T* x, const T* p, const T* sv, T* r,
                     const T* t, cudaStream_t s) {
  if (S.nchunks) k_update_xr_final<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, x, p, sv, r, t);
}

template <typename T>
void update_s_norm(const SegView& S, KScal* sc, const T* r, const T* v, T* out, double* partial,
                   double tol, int it, cudaStream_t s) {
  if (S.nchunks)
    k_update_s_norm<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, r, v, out, partial, tol, it);
}
template <typename T>
void update_xr_norm(const SegView& S, KScal* sc, T* x, const T* p, const T* sv, T* r, const T* t,
                    const T* rh, double* partial, double tol, int it, cudaStream_t s) {
  if (S.nchunks)
    k_update_xr_norm<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, x, p, sv, r, t, rh, partial, tol, it);
}

void any_active(int nseg, const KScal* sc, int32_t* flag, cudaStream_t s) {
  k_any_active<<<1, 256, 0, s>>>(nseg, sc, flag);
}

template <typename T>
void update_p(const SegView& S, const KScal* sc, const T* r, T* p, const T* v, cudaStream_t s) {
  if (S.nchunks) k_update_p<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, r, p, v);
}
template <typename T>
void update_s(const SegView& S, const KScal* sc, const T* r, const T* v, T* out, cudaStream_t s) {
  if (S.nchunks) k_update_s<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, r, v, out);
}
template <typename T>
void update_xr(const SegView& S, const KScal* sc, int half, T* x, const T* phat, const T* shat,
               T* r, const T* sv, const T* t, cudaStream_t s) {
  if (S.nchunks) k_update_xr<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, half, x, phat, shat, r, sv, t);
}
template <typename T>
void vec_sub(const SegView& S, const KScal* sc, int all, const T* a, const T* b, T* dst,
             cudaStream_t s) {
  if (S.nchunks) k_sub<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, all, a, b, dst);
}
template <typename TD, typename TS>
void convert(int64_t n, const TS* src, TD* dst, cudaStream_t s) {
  if (n <= 0) return;
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 32) g = 152 * 32;
  k_convert<TD, TS><<<(int)g, kThreads, 0, s>>>(n, src, dst);
}
template <typename T>
void masked_axpy(const SegView& S, const KScal* sc, T* dst, const T* a, const T* b, cudaStream_t s) {
  if (S.nchunks) k_masked_axpy<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, dst, a, b);
}
template <typename T>
void masked_zero(const SegView& S, const KScal* sc, T* dst, cudaStream_t s) {
  if (S.nchunks) k_masked_zero<T><<<S.nchunks, kThreads, 0, s>>>(S, sc, dst);
}
void sc_beta(int nseg, KScal* sc, int first, cudaStream_t s) {
  k_sc_beta<<<(nseg + 127) / 128, 128, 0, s>>>(nseg, sc, first);
}
void sc_alpha(int nseg, KScal* sc, cudaStream_t s) {
  k_sc_alpha<<<(nseg + 127) / 128, 128, 0, s>>>(nseg, sc);
}
void sc_omega(int nseg, KScal* sc, cudaStream_t s) {
  k_sc_omega<<<(nseg + 127) / 128, 128, 0, s>>>(nseg, sc);
}

#define DDPS_INST_K(T)                                                                           \
  template void seg_reduce<T>(const SegView&, int, RedSpec, RedSpec, RedSpec, double*,          \
                              cudaStream_t);                                                     \
  template void update_p<T>(const SegView&, const KScal*, const T*, T*, const T*, cudaStream_t); \
  template void update_s<T>(const SegView&, const KScal*, const T*, const T*, T*, cudaStream_t); \
  template void update_xr<T>(const SegView&, const KScal*, int, T*, const T*, const T*, T*,      \
                             const T*, const T*, cudaStream_t);                                  \
  template void vec_sub<T>(const SegView&, const KScal*, int, const T*, const T*, T*,            \
                           cudaStream_t);                                                        \
  template void masked_axpy<T>(const SegView&, const KScal*, T*, const T*, const T*,             \
                               cudaStream_t);                                                    \
  template void masked_zero<T>(const SegView&, const KScal*, T*, cudaStream_t);                  \
  template void seg_reduce_post<T>(const SegView&, int, RedSpec, RedSpec, RedSpec, double*, int, \
                                   KScal*, double, int, cudaStream_t);                           \
  template void update_xr_final<T>(const SegView&, const KScal*, T*, const T*, const T*, T*,     \
                                   const T*, cudaStream_t);                                      \
  template void update_s_norm<T>(const SegView&, KScal*, const T*, const T*, T*, double*, double, \
                                 int, cudaStream_t);                                             \
  template void update_xr_norm<T>(const SegView&, KScal*, T*, const T*, const T*, T*, const T*,  \
                                  const T*, double*, double, int, cudaStream_t);
DDPS_INST_K(double)
DDPS_INST_K(float)
template void convert<float, double>(int64_t, const double*, float*, cudaStream_t);
template void convert<double, float>(int64_t, const float*, double*, cudaStream_t);
template void convert<double, double>(int64_t, const double*, double*, cudaStream_t);

}  // namespace ddps
