// Direct solve of the reduced system for chains of blocks (internal; see
// reduced_direct.cu for the method).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "launch.h"

namespace ddps {

// C = alpha A B + beta C (row-major FP32; M x N, inner K)
struct GemmDesc {
  const float* A;
  const float* B;
  float* C;
  int32_t M, N, K, lda, ldb, ldc;
  float alpha, beta;
};
// y = y0 + alpha A x (y0 null: 0)
struct GemvDesc {
  const float* A;
  const float* x;
  float* y;
  const float* y0;
  int32_t M, N, lda;
  float alpha;
};
// dst(r, :) = src(idx[r], :)
struct GatherDesc {
  const float* src;
  float* dst;
  const int32_t* idx;
  int32_t nrows, ncols, lds, ldd;
};
struct CopyDesc {
  const float* src;
  float* dst;
  int64_t count;
};
// W = I - E(0:nj, :), C = E(nj:s, :)
struct FormDesc {
  const float* E;
  float* W;
  float* C;
  int32_t s, nj;
};
// Gauss-Jordan inversion of W (n x n) with scratch Rrow (nb x n), Ccol (n x nb), Dinv (nb x nb)
struct GjDesc {
  float* W;
  float* Rrow;
  float* Ccol;
  float* Dinv;
  int32_t n;
};
// dst(i, j) = G^_block(rowperm[i], colsel[j])
struct ExtractDesc {
  float* dst;
  const int32_t* rowperm;
  const int32_t* colsel;
  int64_t goff, gld;
  int32_t rows, cols;
};

constexpr int32_t kGjBlock = 64;

// One grouped launch: problems [desc_off, desc_off + np) of a descriptor
// array, blocks [prefix[k], prefix[k+1]) per problem.
struct GroupLaunchHost {
  int64_t desc_off = 0, prefix_off = 0;
  int32_t np = 0, nblocks = 0;
};
template <typename Desc>
struct GroupLaunch {
  const Desc* desc;
  const int32_t* prefix;
  int32_t np, nblocks;
};

using DeviceAlloc = std::function<void*(int64_t bytes)>;

struct DirectInput {
  int32_t p = 0;
  int64_t m = 0;
  const int64_t* gq0 = nullptr;  // p: first reduced row of every block
  const int64_t* gq1 = nullptr;
  const int64_t* gcol_ptr = nullptr;      // p+1
  const int32_t* gcols_panel = nullptr;   // reduced index of every stored G^ column
  const int64_t* ghat_off = nullptr;      // p: element offset of the block's G^
  const int64_t* gld = nullptr;           // p: row stride of the block's G^
  const int32_t* block_sys = nullptr;     // p
};

struct DirectPlan {
  int64_t m = 0;
  int32_t nsteps = 0;
  float *store = nullptr, *kbuf = nullptr, *ebuf = nullptr;
  float *vbuf = nullptr, *wbuf = nullptr, *ubuf = nullptr, *gbuf = nullptr, *xbuf = nullptr;
  int64_t store_floats = 0, ebuf_floats = 0, solve_floats = 0;
  int32_t* perm = nullptr;
  int32_t* idx = nullptr;
  std::vector<int32_t> perm_host, idx_host;
  double factor_flops = 0;
  int64_t solve_bytes = 0;  // FP32 matrices streamed by one reduced solve
  // descriptor arrays (host, then device copies)
  std::vector<GemmDesc> gemm_desc;
  std::vector<GemvDesc> gemv_desc;
  std::vector<GatherDesc> gather_desc;
  std::vector<CopyDesc> copy_desc;
  std::vector<FormDesc> form_desc;
  std::vector<GjDesc> gj_desc;
  std::vector<ExtractDesc> ext_desc;
  std::vector<int32_t> prefix;
  GemmDesc* d_gemm = nullptr;
  GemvDesc* d_gemv = nullptr;
  GatherDesc* d_gather = nullptr;
  CopyDesc* d_copy = nullptr;
  FormDesc* d_form = nullptr;
  GjDesc* d_gj = nullptr;
  ExtractDesc* d_ext = nullptr;
  int32_t* d_prefix = nullptr;
  std::vector<GroupLaunchHost> extract;
  struct FactorStep {
    GroupLaunchHost copy, gemm_y, gemm_k, gather_q, gemm_e, form, gj_prep, gj_fix;
    std::vector<GroupLaunchHost> gj_rrow, gj_update;
    int32_t kb = 0;
  };
  std::vector<FactorStep> fstep;
  struct SolveStep {
    GroupLaunchHost gather, gemv1, copy, gemv2, gemv3, copy2;
  };
  std::vector<SolveStep> sfwd, sbwd;
};

// Plans the direct solve (returns an error text when the partition is not
// a set of chains) and allocates its device storage through `alloc`.
std::string plan_direct(const DirectInput& in, DirectPlan& P, const DeviceAlloc& alloc);
// Copies the plan's descriptors and index arrays to the device (synchronous).
void upload_direct(DirectPlan& P, const DeviceAlloc& alloc);
// Factor: L_b, U_b from the stored G^ (element type TG), then W_b, C_b in
// chain order.  Returns the number of launches.
template <typename TG>
int64_t direct_factor(const DirectPlan& P, const TG* ghat, cudaStream_t s);
// z^ = G^-1 g^ (device FP64 vectors of m entries in c order).  Returns the
// number of launches.
int64_t direct_solve(const DirectPlan& P, const double* ghat_in, double* zhat_out, cudaStream_t s);

}  // namespace ddps
