// Direct solve of the reduced system G^ z^ = g^ (Fig. 3 step 6.3 solved
// "directly", Sec. 3 direct mode) for partitions whose blocks form chains:
// every coupling column of block b lies in the reduced rows of block b-1 or
// b+1 of the same system (z-slabs of a grid, grid-line blocks of a 2-D
// grid).  G^ is then block tridiagonal with identity diagonal blocks,
//   G^(b,b) = I,  G^(b,b-1) = L_b E_P,  G^(b,b+1) = U_b E_N,
// where L_b = G(R_b, P_b) and U_b = G(R_b, N_b) hold the block's spike rows
// on its coupling columns P_b (in block b-1) and N_b (in block b+1).
//
// Block LU (the Thomas algorithm on blocks): S_0 = I and
//   S_b = I - L_b (S_{b-1}^-1 U_{b-1})(P_b, :)   placed in the columns N_{b-1}.
// Only the columns J_b = N_{b-1} of S_b differ from I, so with the rows of
// block b ordered as (J_b, J'_b),
//   S_b = [M_b 0; -C_b I],  M_b = I - E(J_b, :),  C_b = E(J'_b, :),
//   S_b^-1 v = [W_b v_J ; v_J' + C_b W_b v_J],  W_b = M_b^-1.
// The factor phase forms W_b (blocked Gauss-Jordan, no pivoting) and C_b
// for every block in chain order, all systems of a batch together; the
// solve is a forward sweep y_b = g_b - L_b (S_{b-1}^-1 y_{b-1})(P_b) and a
// backward sweep z_b = S_b^-1 (y_b - U_b z_{b+1}(N_b)).  Everything is FP32
// (the outer FP64 iteration restores full accuracy); products are grouped
// GEMMs / GEMVs over the systems of a batch.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "reduced_direct.h"

namespace ddps {

namespace {

// ---------------------------------------------------------------------------
// Grouped FP32 GEMM: C = alpha A B + beta C, row-major, one launch over the
// tiles of many problems.  128 x 128 tiles, K in steps of 16 through a double
// buffer in shared memory, 256 threads each holding an 8 x 8 block of C.
// ---------------------------------------------------------------------------
constexpr int GB_M = 128, GB_N = 128, GB_K = 16, GB_T = 256, GB_PAD = 4;

__device__ __forceinline__ int find_problem(const int32_t* __restrict__ prefix, int n, int t) {
  int lo = 0, hi = n;  // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(GB_T, 2)
    k_gemm_grouped(const GemmDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np) {
  __shared__ __align__(16) float As[2][GB_K][GB_M + GB_PAD];
  __shared__ __align__(16) float Bs[2][GB_K][GB_N + GB_PAD];
  const int p = find_problem(prefix, np, blockIdx.x);
  const GemmDesc d = D[p];
  const int t = blockIdx.x - prefix[p];
  const int tiles_n = (d.N + GB_N - 1) / GB_N;
  const int m0 = (t / tiles_n) * GB_M, n0 = (t % tiles_n) * GB_N;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  // loaders: A 128 x 16 (thread: row tid/2, eight k from (tid&1)*8), B 16 x 128 (rows tid/32 and
  // tid/32 + 8, four columns each)
  const int ar = tid >> 1, ak = (tid & 1) * 8;
  const int bk = tid >> 5, bc = (tid & 31) * 4;
  float ra[8], rb[8];
  auto gload = [&](int k0) {
    const int gr = m0 + ar;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int gk = k0 + ak + q;
      ra[q] = (gr < d.M && gk < d.K) ? d.A[(int64_t)gr * d.lda + gk] : 0.f;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gk = k0 + bk + 8 * h;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gc = n0 + bc + q;
        rb[4 * h + q] = (gk < d.K && gc < d.N) ? d.B[(int64_t)gk * d.ldb + gc] : 0.f;
      }
    }
  };
  auto sstore = [&](int st) {
#pragma unroll
    for (int q = 0; q < 8; ++q) As[st][ak + q][ar] = ra[q];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<float4*>(&Bs[st][bk + 8 * h][bc]) =
          make_float4(rb[4 * h], rb[4 * h + 1], rb[4 * h + 2], rb[4 * h + 3]);
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int nk = (d.K + GB_K - 1) / GB_K;
  if (nk > 0) {
    gload(0);
    sstore(0);
  }
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * GB_K);
#pragma unroll
    for (int k = 0; k < GB_K; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) sstore(st ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= d.M) continue;
    float* __restrict__ Cr = d.C + (int64_t)r * d.ldc;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (c >= d.N) continue;
      const float v = d.alpha * acc[i][j];
      Cr[c] = d.beta == 0.f ? v : fmaf(d.beta, Cr[c], v);
    }
  }
}

// ---------------------------------------------------------------------------
// Grouped GEMV: y = y0 + alpha A x (row-major A; y0 null means 0; y0 may be
// y).  One warp per row, eight rows per CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    k_gemv_grouped(const GemvDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const GemvDesc d = D[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = (blockIdx.x - prefix[p]) * 8 + warp;
  if (r >= d.M) return;
  const float* __restrict__ a = d.A + (int64_t)r * d.lda;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int j = lane;
  for (; j + 96 < d.N; j += 128) {
    s0 = fmaf(a[j], d.x[j], s0);
    s1 = fmaf(a[j + 32], d.x[j + 32], s1);
    s2 = fmaf(a[j + 64], d.x[j + 64], s2);
    s3 = fmaf(a[j + 96], d.x[j + 96], s3);
  }
  for (; j < d.N; j += 32) s0 = fmaf(a[j], d.x[j], s0);
  float s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) d.y[r] = (d.y0 ? d.y0[r] : 0.f) + d.alpha * s;
}

// Grouped row gather: dst(r, :) = src(idx[r], :) (ncols columns).
__global__ void __launch_bounds__(256)
    k_gather_grouped(const GatherDesc* __restrict__ D, const int32_t* __restrict__ prefix,
                     int32_t np) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const GatherDesc d = D[p];
  const int64_t base = (int64_t)(blockIdx.x - prefix[p]) * 2048;
  const int64_t total = (int64_t)d.nrows * d.ncols;
  for (int64_t e = base + threadIdx.x; e < min(total, base + 2048); e += blockDim.x) {
    const int64_t r = e / d.ncols, c = e - r * d.ncols;
    d.dst[r * d.ldd + c] = d.src[(int64_t)d.idx[r] * d.lds + c];
  }
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion (no pivoting), one block column kb of
// width nb per step, for many matrices W (n x n, row-major, ld n):
//   prep:  Dinv = W(k,k)^-1 (shared memory, one CTA per matrix), Ccol = W(:,k)
//          with its rows k zeroed, W(i,k) = 0 for i outside k;
//   GEMM:  Rrow = Dinv W(k,:);
//   fix:   Rrow(:,k) = Dinv, W(k,:) = Rrow;
//   GEMM:  W -= Ccol Rrow.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    k_gj_prep(const GjDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np,
              int32_t kb, int32_t nb) {
  extern __shared__ float sd[];  // nb x nb
  const int p = find_problem(prefix, np, blockIdx.x);
  const GjDesc d = D[p];
  const int chunk = blockIdx.x - prefix[p];
  const int k0 = kb * nb, kw = min(nb, d.n - k0);
  if (kw <= 0) return;
  const int tid = threadIdx.x;
  if (chunk == 0) {
    for (int e = tid; e < kw * kw; e += blockDim.x) {
      const int i = e / kw, j = e - i * kw;
      sd[i * nb + j] = d.W[(int64_t)(k0 + i) * d.n + k0 + j];
    }
    __syncthreads();
    // in-place Gauss-Jordan of the kw x kw block
    for (int q = 0; q < kw; ++q) {
      const float piv = 1.f / sd[q * nb + q];
      __syncthreads();
      for (int e = tid; e < kw * kw; e += blockDim.x) {
        const int i = e / kw, j = e - i * kw;
        if (i == q || j == q) continue;
        sd[i * nb + j] -= sd[i * nb + q] * piv * sd[q * nb + j];
      }
      __syncthreads();
      for (int j = tid; j < kw; j += blockDim.x)
        if (j != q) sd[q * nb + j] *= piv;
      for (int i = tid; i < kw; i += blockDim.x)
        if (i != q) sd[i * nb + q] *= -piv;
      if (tid == 0) sd[q * nb + q] = piv;
      __syncthreads();
    }
    for (int e = tid; e < kw * kw; e += blockDim.x) {
      const int i = e / kw, j = e - i * kw;
      d.Dinv[i * nb + j] = sd[i * nb + j];
    }
  }
  // column panel, 256 rows per chunk
  const int r0 = chunk * 256, r1 = min(d.n, r0 + 256);
  for (int e = tid; e < (r1 - r0) * kw; e += blockDim.x) {
    const int i = r0 + e / kw, j = e % kw;
    float* w = d.W + (int64_t)i * d.n + k0 + j;
    const bool in_k = i >= k0 && i < k0 + kw;
    d.Ccol[(int64_t)i * nb + j] = in_k ? 0.f : *w;
    if (!in_k) *w = 0.f;
  }
}

__global__ void __launch_bounds__(256)
    k_gj_fix(const GjDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np,
             int32_t kb, int32_t nb) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const GjDesc d = D[p];
  const int k0 = kb * nb, kw = min(nb, d.n - k0);
  if (kw <= 0) return;
  const int chunk = blockIdx.x - prefix[p];
  const int64_t total = (int64_t)kw * d.n;
  for (int64_t e = (int64_t)chunk * 2048 + threadIdx.x; e < min(total, (int64_t)(chunk + 1) * 2048);
       e += blockDim.x) {
    const int i = (int)(e / d.n), j = (int)(e - (int64_t)i * d.n);
    float v = d.Rrow[(int64_t)i * d.n + j];
    if (j >= k0 && j < k0 + kw) {
      v = d.Dinv[i * nb + (j - k0)];
      d.Rrow[(int64_t)i * d.n + j] = v;
    }
    d.W[(int64_t)(k0 + i) * d.n + j] = v;
  }
}

// Writes M = I - E(0:nj, :) (the rows J of E) into W and copies the rows J'
// of E into C, for many blocks.
__global__ void __launch_bounds__(256)
    k_form_m(const FormDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const FormDesc d = D[p];
  const int64_t total = (int64_t)d.s * d.nj;
  for (int64_t e = (int64_t)(blockIdx.x - prefix[p]) * 2048 + threadIdx.x;
       e < min(total, (int64_t)(blockIdx.x - prefix[p] + 1) * 2048); e += blockDim.x) {
    const int i = (int)(e / d.nj), j = (int)(e - (int64_t)i * d.nj);
    const float v = d.E[e];
    if (i < d.nj)
      d.W[e] = (i == j ? 1.f : 0.f) - v;
    else
      d.C[e - (int64_t)d.nj * d.nj] = v;
  }
}

// Copies rows [r0, r0 + nrows) of src (ld = ncols) to dst, for many blocks.
__global__ void __launch_bounds__(256)
    k_copy_grouped(const CopyDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const CopyDesc d = D[p];
  const int64_t base = (int64_t)(blockIdx.x - prefix[p]) * 2048;
  for (int64_t e = base + threadIdx.x; e < min(d.count, base + 2048); e += blockDim.x)
    d.dst[e] = d.src[e];
}

// L_b and U_b (FP32, rows in the (J, J') order of the block) from the stored
// G^ block: dst(i, j) = G^_b(rowperm[i], colsel[j]).
template <typename TG>
__global__ void __launch_bounds__(256)
    k_extract_lu(const ExtractDesc* __restrict__ D, const int32_t* __restrict__ prefix, int32_t np,
                 const TG* __restrict__ ghat) {
  const int p = find_problem(prefix, np, blockIdx.x);
  const ExtractDesc d = D[p];
  const int64_t total = (int64_t)d.rows * d.cols;
  const int64_t base = (int64_t)(blockIdx.x - prefix[p]) * 2048;
  for (int64_t e = base + threadIdx.x; e < min(total, base + 2048); e += blockDim.x) {
    const int64_t i = e / d.cols, j = e - i * d.cols;
    const TG v = ghat[d.goff + (int64_t)d.rowperm[i] * d.gld + d.colsel[j]];
    d.dst[e] = (float)v;
  }
}

// Reduced vector in c order <-> per-block (J, J') order, FP64 <-> FP32.
__global__ void k_perm_in(const double* __restrict__ src, const int32_t* __restrict__ perm,
                          int64_t m, float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[perm[i]];
}
__global__ void k_perm_out(const float* __restrict__ src, const int32_t* __restrict__ perm,
                           int64_t m, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[perm[i]] = (double)src[i];
}

inline int grid_1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

namespace {

template <typename Desc>
GroupLaunch<Desc> dev(const Desc* base, const int32_t* prefix, const GroupLaunchHost& L) {
  return GroupLaunch<Desc>{base + L.desc_off, prefix + L.prefix_off, L.np, L.nblocks};
}

}  // namespace

// ---------------------------------------------------------------------------
// Execution
// ---------------------------------------------------------------------------
namespace {

int64_t run_gemm(const DirectPlan& P, const GroupLaunchHost& L, cudaStream_t s) {
  if (L.nblocks <= 0) return 0;
  const GroupLaunch<GemmDesc> g = dev(P.d_gemm, P.d_prefix, L);
  k_gemm_grouped<<<g.nblocks, GB_T, 0, s>>>(g.desc, g.prefix, g.np);
  return 1;
}
int64_t run_gemv(const DirectPlan& P, const GroupLaunchHost& L, cudaStream_t s) {
  if (L.nblocks <= 0) return 0;
  const GroupLaunch<GemvDesc> g = dev(P.d_gemv, P.d_prefix, L);
  k_gemv_grouped<<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np);
  return 1;
}
int64_t run_gather(const DirectPlan& P, const GroupLaunchHost& L, cudaStream_t s) {
  if (L.nblocks <= 0) return 0;
  const GroupLaunch<GatherDesc> g = dev(P.d_gather, P.d_prefix, L);
  k_gather_grouped<<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np);
  return 1;
}
int64_t run_copy(const DirectPlan& P, const GroupLaunchHost& L, cudaStream_t s) {
  if (L.nblocks <= 0) return 0;
  const GroupLaunch<CopyDesc> g = dev(P.d_copy, P.d_prefix, L);
  k_copy_grouped<<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np);
  return 1;
}
int64_t run_form(const DirectPlan& P, const GroupLaunchHost& L, cudaStream_t s) {
  if (L.nblocks <= 0) return 0;
  const GroupLaunch<FormDesc> g = dev(P.d_form, P.d_prefix, L);
  k_form_m<<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np);
  return 1;
}

}  // namespace

template <typename TG>
int64_t direct_factor(const DirectPlan& P, const TG* ghat, cudaStream_t s) {
  int64_t n = 0;
  for (const GroupLaunchHost& L : P.extract) {
    if (L.nblocks <= 0) continue;
    const GroupLaunch<ExtractDesc> g = dev(P.d_ext, P.d_prefix, L);
    k_extract_lu<TG><<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np, ghat);
    ++n;
  }
  const size_t gj_sm = (size_t)kGjBlock * kGjBlock * sizeof(float);
  if (gj_sm > 48 * 1024)
    record_launch_error(
        cudaFuncSetAttribute(k_gj_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gj_sm));
  for (int32_t t = 1; t < P.nsteps; ++t) {
    const DirectPlan::FactorStep& st = P.fstep[t];
    n += run_copy(P, st.copy, s);
    n += run_gemm(P, st.gemm_y, s);
    n += run_gemm(P, st.gemm_k, s);
    n += run_gather(P, st.gather_q, s);
    n += run_gemm(P, st.gemm_e, s);
    n += run_form(P, st.form, s);
    for (int32_t kb = 0; kb < st.kb; ++kb) {
      if (st.gj_prep.nblocks > 0) {
        const GroupLaunch<GjDesc> g = dev(P.d_gj, P.d_prefix, st.gj_prep);
        k_gj_prep<<<g.nblocks, 256, gj_sm, s>>>(g.desc, g.prefix, g.np, kb, kGjBlock);
        ++n;
      }
      n += run_gemm(P, st.gj_rrow[kb], s);
      if (st.gj_fix.nblocks > 0) {
        const GroupLaunch<GjDesc> g = dev(P.d_gj, P.d_prefix, st.gj_fix);
        k_gj_fix<<<g.nblocks, 256, 0, s>>>(g.desc, g.prefix, g.np, kb, kGjBlock);
        ++n;
      }
      n += run_gemm(P, st.gj_update[kb], s);
    }
  }
  return n;
}
template int64_t direct_factor<double>(const DirectPlan&, const double*, cudaStream_t);
template int64_t direct_factor<float>(const DirectPlan&, const float*, cudaStream_t);
template int64_t direct_factor<__half>(const DirectPlan&, const __half*, cudaStream_t);
template int64_t direct_factor<__nv_bfloat16>(const DirectPlan&, const __nv_bfloat16*, cudaStream_t);

int64_t direct_solve(const DirectPlan& P, const double* ghat_in, double* zhat_out, cudaStream_t s) {
  if (P.m <= 0) return 0;
  int64_t n = 0;
  k_perm_in<<<grid_1d(P.m), 256, 0, s>>>(ghat_in, P.perm, P.m, P.gbuf);
  ++n;
  auto step = [&](const DirectPlan::SolveStep& q) {
    n += run_gather(P, q.gather, s);
    n += run_gemv(P, q.gemv1, s);
    n += run_copy(P, q.copy, s);
    n += run_gemv(P, q.gemv2, s);
    n += run_gemv(P, q.gemv3, s);
    n += run_copy(P, q.copy2, s);
  };
  for (int32_t t = 0; t < P.nsteps; ++t) step(P.sfwd[t]);
  for (int32_t t = P.nsteps - 1; t >= 0; --t) step(P.sbwd[t]);
  k_perm_out<<<grid_1d(P.m), 256, 0, s>>>(P.wbuf, P.perm, P.m, zhat_out);
  return n + 1;
}

void upload_direct(DirectPlan& P, const DeviceAlloc& alloc) {
  auto up = [&](const auto& v, auto*& d) {
    using T = typename std::decay<decltype(v)>::type::value_type;
    d = (T*)alloc(((int64_t)v.size() + 1) * (int64_t)sizeof(T));
    if (!v.empty()) cudaMemcpy((void*)d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  };
  up(P.gemm_desc, P.d_gemm);
  up(P.gemv_desc, P.d_gemv);
  up(P.gather_desc, P.d_gather);
  up(P.copy_desc, P.d_copy);
  up(P.form_desc, P.d_form);
  up(P.gj_desc, P.d_gj);
  up(P.ext_desc, P.d_ext);
  up(P.prefix, P.d_prefix);
  if (!P.perm_host.empty())
    cudaMemcpy(P.perm, P.perm_host.data(), P.perm_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (!P.idx_host.empty())
    cudaMemcpy(P.idx, P.idx_host.data(), P.idx_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  // E of blocks whose predecessor couples nothing back stays zero
  cudaMemset(P.ebuf, 0, (size_t)(P.ebuf_floats + 1) * sizeof(float));
}

// ---------------------------------------------------------------------------
// Host planning
// ---------------------------------------------------------------------------

// Blocks (tiles, row groups, chunks) per problem and their prefix sums.
template <typename Desc>
static GroupLaunchHost add_launch(std::vector<Desc>& all_desc, std::vector<int32_t>& all_prefix,
                                  const std::vector<Desc>& desc, const std::vector<int32_t>& blocks) {
  GroupLaunchHost L;
  L.desc_off = (int64_t)all_desc.size();
  L.prefix_off = (int64_t)all_prefix.size();
  L.np = (int32_t)desc.size();
  int32_t acc = 0;
  all_prefix.push_back(0);
  for (size_t i = 0; i < desc.size(); ++i) {
    all_desc.push_back(desc[i]);
    acc += blocks[i];
    all_prefix.push_back(acc);
  }
  L.nblocks = acc;
  return L;
}

static int32_t gemm_tiles(int M, int N) {
  if (M <= 0 || N <= 0) return 0;
  return ((M + GB_M - 1) / GB_M) * ((N + GB_N - 1) / GB_N);
}
static int32_t chunks_2048(int64_t count) { return (int32_t)((count + 2047) / 2048); }

std::string plan_direct(const DirectInput& in, DirectPlan& P, const DeviceAlloc& alloc) {
  const int32_t p = in.p;
  // reduced row range of every block and the block of every reduced index
  std::vector<int32_t> qblock(in.m, -1);
  for (int32_t b = 0; b < p; ++b)
    for (int64_t q = in.gq0[b]; q < in.gq1[b]; ++q) qblock[q] = b;
  // coupling columns of each block split into previous / next block
  std::vector<std::vector<int32_t>> lsel(p), usel(p), lidx(p), uidx(p);  // panel col, local row
  for (int32_t b = 0; b < p; ++b) {
    for (int64_t pc = in.gcol_ptr[b]; pc < in.gcol_ptr[b + 1]; ++pc) {
      const int32_t q = in.gcols_panel[pc];
      const int32_t ob = qblock[q];
      const int32_t col = (int32_t)(pc - in.gcol_ptr[b]);
      if (ob == b - 1 && in.block_sys[ob] == in.block_sys[b]) {
        lsel[b].push_back(col);
        lidx[b].push_back((int32_t)(q - in.gq0[ob]));
      } else if (ob == b + 1 && in.block_sys[ob] == in.block_sys[b]) {
        usel[b].push_back(col);
        uidx[b].push_back((int32_t)(q - in.gq0[ob]));
      } else {
        return "reduced_solver DIRECT needs chains of blocks: block " + std::to_string(b) +
               " couples to block " + std::to_string(ob) + " (only the neighbouring blocks of "
               "the same system are allowed)";
      }
    }
  }
  // (J, J') order of every block's reduced rows: J = the rows block b-1 couples to
  // (in U_{b-1}'s column order), then the others ascending
  P.m = in.m;
  std::vector<int32_t> perm(in.m);            // position -> reduced index
  std::vector<int32_t> local_pos;             // per block: local row -> position in (J,J') order
  std::vector<std::vector<int32_t>> order(p);  // per block: (J,J') position -> local row
  std::vector<int32_t> nj(p, 0);
  for (int32_t b = 0; b < p; ++b) {
    const int32_t s = (int32_t)(in.gq1[b] - in.gq0[b]);
    std::vector<char> inj(s, 0);
    if (b > 0 && in.block_sys[b - 1] == in.block_sys[b]) {
      for (int32_t r : uidx[b - 1]) {
        order[b].push_back(r);
        inj[r] = 1;
      }
    }
    nj[b] = (int32_t)order[b].size();
    for (int32_t r = 0; r < s; ++r)
      if (!inj[r]) order[b].push_back(r);
    for (int32_t i = 0; i < s; ++i) perm[in.gq0[b] + i] = (int32_t)(in.gq0[b] + order[b][i]);
  }
  // position of each local row in the (J, J') order (to remap L's and U's column targets)
  std::vector<std::vector<int32_t>> pos(p);
  for (int32_t b = 0; b < p; ++b) {
    pos[b].assign(order[b].size(), 0);
    for (size_t i = 0; i < order[b].size(); ++i) pos[b][order[b][i]] = (int32_t)i;
  }
  // chain position of every block and the longest chain
  std::vector<int32_t> tpos(p, 0);
  int32_t tmax = 0;
  for (int32_t b = 0; b < p; ++b) {
    tpos[b] = (b > 0 && in.block_sys[b - 1] == in.block_sys[b]) ? tpos[b - 1] + 1 : 0;
    tmax = std::max(tmax, tpos[b]);
  }
  P.nsteps = tmax + 1;

  // device storage per block: L (s x |P|), U (s x |N|), W (nj x nj), C ((s-nj) x nj),
  // K (s x |N|) scratch of the factor; vectors v (forward result) and w/z (m each)
  std::vector<int64_t> offL(p), offU(p), offW(p), offC(p), offK(p);
  int64_t tot = 0, totK = 0, max_gj = 0;
  for (int32_t b = 0; b < p; ++b) {
    const int64_t s = in.gq1[b] - in.gq0[b];
    offL[b] = tot;
    tot += s * (int64_t)lsel[b].size();
    offU[b] = tot;
    tot += s * (int64_t)usel[b].size();
    offW[b] = tot;
    tot += (int64_t)nj[b] * nj[b];
    offC[b] = tot;
    tot += (s - nj[b]) * (int64_t)nj[b];
    offK[b] = totK;
    totK += s * (int64_t)usel[b].size();
    max_gj = std::max<int64_t>(max_gj, nj[b]);
  }
  P.store = (float*)alloc((tot + 1) * (int64_t)sizeof(float));
  P.kbuf = (float*)alloc((totK + 1) * (int64_t)sizeof(float));
  P.store_floats = tot;
  // per block scratch of the Gauss-Jordan steps and E; E (s x nj) lives in K of the block
  // before (not needed after Q is formed) -- kept separate for clarity
  std::vector<int64_t> offE(p), offR(p), offCc(p), offD(p), offQ(p);
  int64_t totE = 0;
  for (int32_t b = 0; b < p; ++b) {
    const int64_t s = in.gq1[b] - in.gq0[b];
    offE[b] = totE;
    totE += s * (int64_t)nj[b];
    offQ[b] = totE;
    totE += (int64_t)lsel[b].size() * nj[b];
    offR[b] = totE;
    totE += (int64_t)kGjBlock * nj[b];
    offCc[b] = totE;
    totE += (int64_t)nj[b] * kGjBlock;
    offD[b] = totE;
    totE += (int64_t)kGjBlock * kGjBlock;
  }
  P.ebuf = (float*)alloc((totE + 1) * (int64_t)sizeof(float));
  P.ebuf_floats = totE;
  // gathered entries of a neighbour's vector, per block
  std::vector<int64_t> offX(p);
  int64_t totX = 0;
  for (int32_t b = 0; b < p; ++b) {
    offX[b] = totX;
    totX += (int64_t)std::max(lsel[b].size(), usel[b].size());
  }
  P.xbuf = (float*)alloc((totX + 1) * (int64_t)sizeof(float));
  P.vbuf = (float*)alloc((in.m + 1) * (int64_t)sizeof(float));
  P.wbuf = (float*)alloc((in.m + 1) * (int64_t)sizeof(float));
  P.ubuf = (float*)alloc((in.m + 1) * (int64_t)sizeof(float));
  P.gbuf = (float*)alloc((in.m + 1) * (int64_t)sizeof(float));
  P.perm = (int32_t*)alloc((in.m + 1) * (int64_t)sizeof(int32_t));
  P.perm_host = perm;
  // gather index arrays: rows of K_{b-1} picked by L_b's columns, entries of
  // w_{b-1} picked by L_b, entries of z_{b+1} picked by U_b (positions in (J,J') order)
  std::vector<int32_t> idx_all;
  std::vector<int64_t> off_lidx(p), off_uidx(p), off_rowperm(p), off_lsel(p), off_usel(p);
  for (int32_t b = 0; b < p; ++b) {
    off_lidx[b] = (int64_t)idx_all.size();
    for (int32_t r : lidx[b]) idx_all.push_back(pos[b - 1][r]);
    off_uidx[b] = (int64_t)idx_all.size();
    for (int32_t r : uidx[b]) idx_all.push_back(pos[b + 1][r]);
    off_rowperm[b] = (int64_t)idx_all.size();
    for (int32_t r : order[b]) idx_all.push_back(r);
    off_lsel[b] = (int64_t)idx_all.size();
    for (int32_t c : lsel[b]) idx_all.push_back(c);
    off_usel[b] = (int64_t)idx_all.size();
    for (int32_t c : usel[b]) idx_all.push_back(c);
  }
  P.idx = (int32_t*)alloc(((int64_t)idx_all.size() + 1) * (int64_t)sizeof(int32_t));
  P.idx_host = idx_all;

  auto F = [&](int64_t off) { return P.store + off; };
  auto I = [&](int64_t off) { return P.idx + off; };

  // --- extraction of L and U from G^ (once per factor) ---
  {
    std::vector<ExtractDesc> d;
    std::vector<int32_t> nb;
    for (int32_t b = 0; b < p; ++b) {
      const int32_t s = (int32_t)(in.gq1[b] - in.gq0[b]);
      if (!lsel[b].empty()) {
        d.push_back(ExtractDesc{F(offL[b]), I(off_rowperm[b]), I(off_lsel[b]), in.ghat_off[b],
                                in.gld[b], s, (int32_t)lsel[b].size()});
        nb.push_back(chunks_2048((int64_t)s * lsel[b].size()));
      }
      if (!usel[b].empty()) {
        d.push_back(ExtractDesc{F(offU[b]), I(off_rowperm[b]), I(off_usel[b]), in.ghat_off[b],
                                in.gld[b], s, (int32_t)usel[b].size()});
        nb.push_back(chunks_2048((int64_t)s * usel[b].size()));
      }
    }
    P.extract.push_back(add_launch(P.ext_desc, P.prefix, d, nb));
  }
  // --- factor steps t = 1 .. nsteps-1 (blocks at chain position t; b-1 at t-1) ---
  P.fstep.assign(P.nsteps, DirectPlan::FactorStep{});
  for (int32_t t = 1; t < P.nsteps; ++t) {
    DirectPlan::FactorStep& st = P.fstep[t];
    std::vector<CopyDesc> cp;
    std::vector<int32_t> cpn;
    std::vector<GemmDesc> g1, g2, g3, gr, gu;
    std::vector<int32_t> g1n, g2n, g3n;
    std::vector<GatherDesc> ga;
    std::vector<int32_t> gan;
    std::vector<FormDesc> fm;
    std::vector<int32_t> fmn;
    std::vector<GjDesc> gj;
    std::vector<int32_t> gjn_prep, gjn_fix;
    int32_t kb_max = 0;
    for (int32_t b = 0; b < p; ++b) {
      if (tpos[b] != t) continue;
      const int32_t a = b - 1;  // previous block of the chain
      const int32_t sa = (int32_t)(in.gq1[a] - in.gq0[a]), sb = (int32_t)(in.gq1[b] - in.gq0[b]);
      const int32_t na = (int32_t)usel[a].size();  // |N_{b-1}| = |J_b|
      const int32_t ja = nj[a];
      const int32_t pb = (int32_t)lsel[b].size();
      float* K = P.kbuf + offK[a];  // s_a x na
      // K = S_a^-1 U_a: rows J_a = W_a U_a(J_a), rows J'_a = U_a(J'_a) + C_a K(J_a)
      cp.push_back(CopyDesc{F(offU[a]), K, (int64_t)sa * na});
      cpn.push_back(chunks_2048((int64_t)sa * na));
      if (ja > 0 && na > 0) {
        g1.push_back(GemmDesc{F(offW[a]), F(offU[a]), K, ja, na, ja, ja, na, na, 1.f, 0.f});
        g1n.push_back(gemm_tiles(ja, na));
        if (sa - ja > 0) {
          g2.push_back(GemmDesc{F(offC[a]), K, K + (int64_t)ja * na, sa - ja, na, ja, ja, na, na,
                                1.f, 1.f});
          g2n.push_back(gemm_tiles(sa - ja, na));
        }
      }
      // Q = K(P_b rows) (pb x na), E = L_b Q (sb x na), M_b = I - E(J_b), C_b = E(J'_b)
      float* Q = P.ebuf + offQ[b];
      float* E = P.ebuf + offE[b];
      if (pb > 0 && na > 0) {
        ga.push_back(GatherDesc{K, Q, I(off_lidx[b]), pb, na, na, na});
        gan.push_back(chunks_2048((int64_t)pb * na));
        g3.push_back(GemmDesc{F(offL[b]), Q, E, sb, na, pb, pb, na, na, 1.f, 0.f});
        g3n.push_back(gemm_tiles(sb, na));
      }  // else no coupling back: E stays zero (cleared at upload)
      if (nj[b] != na) return "direct reduced solve: inconsistent interface sizes";
      if (na > 0) {
        fm.push_back(FormDesc{E, F(offW[b]), F(offC[b]), sb, na});
        fmn.push_back(chunks_2048((int64_t)sb * na));
        gj.push_back(GjDesc{F(offW[b]), P.ebuf + offR[b], P.ebuf + offCc[b], P.ebuf + offD[b], na});
        gjn_prep.push_back((na + 255) / 256);
        gjn_fix.push_back(chunks_2048((int64_t)kGjBlock * na));
        kb_max = std::max(kb_max, (na + kGjBlock - 1) / kGjBlock);
        (void)sa;
      }
    }
    st.copy = add_launch(P.copy_desc, P.prefix, cp, cpn);
    st.gemm_y = add_launch(P.gemm_desc, P.prefix, g1, g1n);
    st.gemm_k = add_launch(P.gemm_desc, P.prefix, g2, g2n);
    st.gather_q = add_launch(P.gather_desc, P.prefix, ga, gan);
    st.gemm_e = add_launch(P.gemm_desc, P.prefix, g3, g3n);
    st.form = add_launch(P.form_desc, P.prefix, fm, fmn);
    st.gj_prep = add_launch(P.gj_desc, P.prefix, gj, gjn_prep);
    st.gj_fix = add_launch(P.gj_desc, P.prefix, gj, gjn_fix);
    // Gauss-Jordan GEMMs per column block kb: Rrow = Dinv W(k,:), W -= Ccol Rrow
    for (int32_t kb = 0; kb < kb_max; ++kb) {
      std::vector<GemmDesc> r1, r2;
      std::vector<int32_t> r1n, r2n;
      for (const GjDesc& q : gj) {
        const int32_t k0 = kb * kGjBlock, kw = std::min(kGjBlock, q.n - k0);
        if (kw <= 0) {
          continue;
        }
        r1.push_back(GemmDesc{q.Dinv, q.W + (int64_t)k0 * q.n, q.Rrow, kw, q.n, kw, kGjBlock, q.n,
                              q.n, 1.f, 0.f});
        r1n.push_back(gemm_tiles(kw, q.n));
        r2.push_back(GemmDesc{q.Ccol, q.Rrow, q.W, q.n, q.n, kw, kGjBlock, q.n, q.n, -1.f, 1.f});
        r2n.push_back(gemm_tiles(q.n, q.n));
      }
      st.gj_rrow.push_back(add_launch(P.gemm_desc, P.prefix, r1, r1n));
      st.gj_update.push_back(add_launch(P.gemm_desc, P.prefix, r2, r2n));
    }
    st.kb = kb_max;
  }
  // --- solve sweeps ---
  // forward, step t: v_b = g_b - L_b w_a(P_b) (gather into ubuf, GEMV), then
  // w_b(J) = W_b v_b(J), w_b(J') = v_b(J') + C_b w_b(J); step 0: w = v = g.
  P.sfwd.assign(P.nsteps, DirectPlan::SolveStep{});
  P.sbwd.assign(P.nsteps, DirectPlan::SolveStep{});
  for (int32_t t = 0; t < P.nsteps; ++t) {
    std::vector<GatherDesc> ga, gb;
    std::vector<int32_t> gan, gbn;
    std::vector<GemvDesc> m1, m2, m3, n1, n2, n3;
    std::vector<int32_t> m1n, m2n, m3n, n1n, n2n, n3n;
    std::vector<CopyDesc> cf, cf2, cb;
    std::vector<int32_t> cfn, cf2n, cbn;
    for (int32_t b = 0; b < p; ++b) {
      if (tpos[b] != t) continue;
      const int32_t s = (int32_t)(in.gq1[b] - in.gq0[b]);
      const int64_t q0 = in.gq0[b];
      const int32_t pb = (int32_t)lsel[b].size(), nb_ = (int32_t)usel[b].size();
      float* x = P.xbuf + offX[b];
      // forward: v_b = g_b - L_b w_{b-1}(P_b), then w_b = S_b^-1 v_b
      if (pb > 0) {
        ga.push_back(GatherDesc{P.wbuf + in.gq0[b - 1], x, I(off_lidx[b]), pb, 1, 1, 1});
        gan.push_back(chunks_2048(pb));
        m1.push_back(GemvDesc{F(offL[b]), x, P.vbuf + q0, P.gbuf + q0, s, pb, pb, -1.f});
        m1n.push_back((s + 7) / 8);
      } else {
        cf.push_back(CopyDesc{P.gbuf + q0, P.vbuf + q0, s});
        cfn.push_back(chunks_2048(s));
      }
      if (nj[b] > 0) {
        m2.push_back(GemvDesc{F(offW[b]), P.vbuf + q0, P.wbuf + q0, nullptr, nj[b], nj[b], nj[b], 1.f});
        m2n.push_back((nj[b] + 7) / 8);
        if (s - nj[b] > 0) {
          m3.push_back(GemvDesc{F(offC[b]), P.wbuf + q0, P.wbuf + q0 + nj[b], P.vbuf + q0 + nj[b],
                                s - nj[b], nj[b], nj[b], 1.f});
          m3n.push_back((s - nj[b] + 7) / 8);
        }
      } else {
        cf2.push_back(CopyDesc{P.vbuf + q0, P.wbuf + q0, s});  // S_b = I
        cf2n.push_back(chunks_2048(s));
      }
      // backward: u = v_b - U_b z_{b+1}(N_b), z_b = S_b^-1 u (z kept in wbuf; the
      // last block of a chain keeps z_b = w_b)
      if (nb_ > 0) {
        gb.push_back(GatherDesc{P.wbuf + in.gq0[b + 1], x, I(off_uidx[b]), nb_, 1, 1, 1});
        gbn.push_back(chunks_2048(nb_));
        n1.push_back(GemvDesc{F(offU[b]), x, P.ubuf + q0, P.vbuf + q0, s, nb_, nb_, -1.f});
        n1n.push_back((s + 7) / 8);
        if (nj[b] > 0) {
          n2.push_back(GemvDesc{F(offW[b]), P.ubuf + q0, P.wbuf + q0, nullptr, nj[b], nj[b], nj[b], 1.f});
          n2n.push_back((nj[b] + 7) / 8);
          if (s - nj[b] > 0) {
            n3.push_back(GemvDesc{F(offC[b]), P.wbuf + q0, P.wbuf + q0 + nj[b], P.ubuf + q0 + nj[b],
                                  s - nj[b], nj[b], nj[b], 1.f});
            n3n.push_back((s - nj[b] + 7) / 8);
          }
        } else {
          cb.push_back(CopyDesc{P.ubuf + q0, P.wbuf + q0, s});
          cbn.push_back(chunks_2048(s));
        }
      }
      P.solve_bytes += 4 * ((int64_t)s * pb + (int64_t)s * nb_ + 2 * (int64_t)nj[b] * s);
    }
    DirectPlan::SolveStep& f = P.sfwd[t];
    f.gather = add_launch(P.gather_desc, P.prefix, ga, gan);
    f.gemv1 = add_launch(P.gemv_desc, P.prefix, m1, m1n);
    f.copy = add_launch(P.copy_desc, P.prefix, cf, cfn);
    f.gemv2 = add_launch(P.gemv_desc, P.prefix, m2, m2n);
    f.gemv3 = add_launch(P.gemv_desc, P.prefix, m3, m3n);
    f.copy2 = add_launch(P.copy_desc, P.prefix, cf2, cf2n);
    DirectPlan::SolveStep& g = P.sbwd[t];
    g.gather = add_launch(P.gather_desc, P.prefix, gb, gbn);
    g.gemv1 = add_launch(P.gemv_desc, P.prefix, n1, n1n);
    g.copy = add_launch(P.copy_desc, P.prefix, std::vector<CopyDesc>{}, std::vector<int32_t>{});
    g.gemv2 = add_launch(P.gemv_desc, P.prefix, n2, n2n);
    g.gemv3 = add_launch(P.gemv_desc, P.prefix, n3, n3n);
    g.copy2 = add_launch(P.copy_desc, P.prefix, cb, cbn);
  }
  P.factor_flops = 0;
  for (int32_t b = 0; b < p; ++b) {
    if (tpos[b] == 0) continue;
    const double sa = (double)(in.gq1[b - 1] - in.gq0[b - 1]), sb = (double)(in.gq1[b] - in.gq0[b]);
    const double na = (double)usel[b - 1].size(), ja = nj[b - 1], pb = (double)lsel[b].size();
    P.factor_flops += 2.0 * ja * ja * na + 2.0 * (sa - ja) * ja * na + 2.0 * sb * pb * na +
                      2.0 * na * na * na;
  }
  P.solve_floats = tot;
  return "";
}

}  // namespace ddps
