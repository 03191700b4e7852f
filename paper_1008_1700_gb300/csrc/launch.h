// Device-side views and kernel launchers shared by the library's translation
// units (internal, not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace ddps {

struct KScal;
struct MvRed;

// SM count of the current device, cached per device ordinal (a process may
// switch devices, and devices may differ).
inline int device_sm_count() {
  static int cache[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
  if (cache[dev] <= 0) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
      nsm = 1;
    cache[dev] = nsm;
  }
  return cache[dev];
}

// First failed launch-configuration call (attribute setting, extended
// launch) of the calling thread since the last take_launch_error(); the C
// ABI layer turns it into DDPS_ERR_CUDA after each sequence of launches.
inline cudaError_t& launch_error_slot() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}
inline void record_launch_error(cudaError_t e) {
  if (e != cudaSuccess && launch_error_slot() == cudaSuccess) launch_error_slot() = e;
}
inline cudaError_t take_launch_error() {
  const cudaError_t e = launch_error_slot();
  launch_error_slot() = cudaSuccess;
  return e;
}

// Multifrontal structure of all blocks, resident on the device.
struct DevFronts {
  const int32_t* k;        // pivots per front
  const int32_t* m;        // front order
  const int32_t* block;    // owning block
  const int64_t* row0;     // new index of the first pivot
  const int64_t* arena;    // offset of the m x m column-major front
  const int64_t* idx_off;  // offset into idx
  const int64_t* upd;      // offset of the update vector / update rows
  const int64_t* rel_off;  // offset into rel (-1 for roots)
  const int32_t* cbeg;     // children list range
  const int32_t* cend;
  const int32_t* children;
  const int32_t* idx;      // front row lists (new indices)
  const int32_t* rel;      // child update row -> parent front position
};

// Error record written by kernels: [0] = code (0 none, 1 small pivot, 2 timeout),
// [1] = front, [2] = new row index.
struct DevError {
  long long* rec;
};

// ---- solve.cu: persistent sweeps over the deep levels (fronts of at most
// kPersistM rows); done: one flag per front, next: the work counter, both zero
// before the launch ----
constexpr int32_t kPersistM = 128;
template <typename T>
void launch_fwd_persist(DevFronts F, const int32_t* order, int32_t nitems, int32_t max_m,
                        const T* arena, T* w, T* u, int32_t* done, int32_t* next, long long* err,
                        cudaStream_t s);
template <typename T>
void launch_bwd_persist(DevFronts F, const int32_t* order, int32_t nitems, int32_t max_m,
                        const int32_t* wait_on, const T* arena, T* w, int32_t* done,
                        int32_t* next, long long* err, cudaStream_t s);

// ---- ilu.cu: ILU(0) block factors (factor_kind ILU0) ----
// CSR of the diagonal blocks (global rows and columns, sorted), position of
// each row's diagonal, block of each row.
struct IluDev {
  const int32_t* rp;
  const int32_t* col;
  const int32_t* diag;
  const int32_t* row_block;
};
template <typename T>
void launch_ilu0_level(const int32_t* rows, int32_t nrows, const IluDev& L, T* a,
                       const double* rownorm, double pivot_tol, long long* err, cudaStream_t s);
template <typename T>
void launch_ilu_vec_level(bool fwd, const int32_t* rows, int32_t nrows, const IluDev& L,
                          const T* a, T* x, cudaStream_t s);
template <typename T>
void launch_ilu_panel_level(bool fwd, const int32_t* rows, int32_t nrows, const IluDev& L,
                            const T* a, const int64_t* block_ncols, int64_t j0, int32_t NR, T* X,
                            cudaStream_t s);

// ---- factor.cu --------------------------------------------------------------
template <typename T>
void launch_assemble(const double* values, const int64_t* amap, int64_t nnz, T* arena,
                     cudaStream_t s);
void launch_row_absmax(const int32_t* rowptr, const int64_t* amap, const double* values,
                       const int32_t* iperm, int64_t n, double* rownorm_new, cudaStream_t s);
template <typename T>
void launch_extend_add_p(DevFronts F, const int32_t* parent, const int32_t* child_list,
                         int32_t nchild, int32_t max_r, T* arena, cudaStream_t s);
// multi-RHS spike solves on a row-major panel X (n x NR) and update rows U (upd_size x NR)
template <typename T>
void launch_spike_rhs(const int32_t* rt_rownew, const int32_t* rt_rhscol, const int64_t* rt_src,
                      int64_t nrt, const double* values, int64_t j0, int32_t NR, T* X,
                      cudaStream_t s);
// Fronts with m <= small_front_max<T>() are factored and inverted in shared memory.
template <typename T>
constexpr int small_front_max() {
  return sizeof(T) == 8 ? 90 : 127;
}
template <typename T>
void launch_front_lu_small(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, T* arena,
                           const double* rownorm_new, double pivot_tol, long long* err,
                           cudaStream_t s);
// Multi-CTA LU of large fronts: panel j0 (one CTA per front), then the
// trailing update over tiles of 64 x 64 (tile_ij = (ti << 16) | tj).
constexpr int kLuPanel = 32;
constexpr int kLuTile = 64;
// Multi-CTA triangular inverses of large fronts: tile_front / tile_cb list
// (front, 64-column block); inv holds 2 k^2 entries per front at inv_off.
constexpr int kInvBlock = 64;
template <typename T>
void launch_tri_inverse_mc(DevFronts F, const int32_t* tile_front, const int32_t* tile_cb,
                           int32_t ntiles, const int32_t* list, int32_t nf, int32_t max_k, T* arena,
                           T* inv, const int64_t* inv_off, cudaStream_t s);
// Panel step j0 of the large fronts in `list`: the diagonal block and the
// inverses of its triangles (one CTA per front; dinv holds 2 x 32 x 32
// entries per list entry), then L21 rows and U12 columns over chunks of 256
// (chunk_word bit 30 = columns, low bits = chunk index; rows and columns
// from j0 + 32; chunk_slot = the front's position in `list`).
template <typename T>
void launch_lu_panel(DevFronts F, const int32_t* list, int32_t nf, const int32_t* chunk_front,
                     const int32_t* chunk_word, const int32_t* chunk_slot, int32_t nchunks,
                     int32_t j0, T* arena, T* dinv, const double* rownorm_new, double pivot_tol,
                     long long* err, cudaStream_t s);
// blocked = 1: the fronts run in blocks of 256 pivots (see launch_lu_update_tc)
// and the update skips the entries with row and column >= Jend.
template <typename T>
void launch_lu_trailing(DevFronts F, const int32_t* tile_front, const int32_t* tile_ij,
                        int32_t ntiles, int32_t j0, int blocked, T* arena, cudaStream_t s);

// ---- spike.cu: multi-RHS forward/backward substitution as per-level GEMMs ----
// Panel X (n x NR, row-major) holds the right-hand sides and receives the
// solution on every pivot row; Tb (sum of front orders x NR) holds each
// front's working rows (pivot part, then its update rows for the parent).
enum SpikeOp { OP_FWD_LINV = 0, OP_FWD_L21 = 1, OP_BWD_U12 = 2, OP_BWD_UINV = 3 };
template <typename T>
int spike_tile_m();
// Clears the pivot rows of the listed fronts in the panel X (n x NR).
template <typename T>
void launch_zero_front_rows(DevFronts F, const int32_t* list, int32_t nf, int32_t NR, T* X,
                            cudaStream_t s);
template <typename T>
// active (per front, may be null): children with active[c] == 0 are skipped.
// D (may be null): for children with dflag[c] != 0 the update rows of their
// forward product are held apart in D (same row indexing as Tb) and added here;
// children with skipT[c] != 0 (skipT may be null) have no working rows in Tb
// and contribute D alone.
void launch_spike_gather(DevFronts F, const int32_t* list, int32_t nf, const int64_t* block_ncols,
                         int64_t j0, int32_t NR, const T* X, T* Tb, const uint8_t* active,
                         const T* D, const uint8_t* dflag, const uint8_t* skipT, cudaStream_t s);
// spike_tc.cu: the same ops on the tensor cores (fp32 factors, bf16 operands,
// fp32 accumulation); passes = 1 (hi*hi) or 3 (hi*hi + hi*lo + lo*hi).  A wait
// that runs out writes error code 2 into err[0].
// The A operands are packed once per factorisation (launch_tc_pack_a) into
// bf16 blocks of 128 rows x tc_tile_bk() K-columns, tc_a_block_bytes(passes)
// bytes each; tile_aoff[t] is the byte offset of tile t's first block.
int tc_tile_bk();
// Block LU update on the tensor cores (fp32 factors, bf16 hi/lo split, fp32
// accumulation): after the panel step at column j0 that ends a block of 256
// pivots, A[Jend:m, Jend:m] -= L[Jend:m, J:Jend] U[J:Jend, Jend:m] over
// 128 x 128 tiles (tile_ij = (ti << 16) | tj from Jend), J = j0 rounded down
// to 256, Jend = min(J + 256, k).  A wait that runs out writes 2 into err[0].
constexpr int kLuTcBlock = 256;
constexpr int kLuTcTile = 128;
void launch_lu_update_tc(DevFronts F, const int32_t* tile_front, const int32_t* tile_ij,
                         int32_t ntiles, int32_t j0, float* arena, long long* err, cudaStream_t s);
int64_t tc_a_block_bytes(int passes);
void launch_tc_pack_a(int op, int passes, DevFronts F, const int32_t* tile_front,
                      const int32_t* tile_m0, const int64_t* tile_aoff, int32_t ntiles,
                      int32_t max_kt, const float* arena, unsigned char* atc, cudaStream_t s);
// Fused front products (spike_tc.cu): fronts with at most tc_fused_max_rows()
// output rows (backward: k, forward: m) run both products of a sweep as one
// GEMM with a precomputed W (launch_tc_w_pack, once per factorisation; woff[f]
// = byte offset of front f's W, tc_fused_w_bytes bytes, 1024-byte aligned).
// cls = tc_fused_class(rows) selects the tensor-memory width (64 << cls).
int tc_fused_max_rows();
int tc_fused_class(int rows);
int64_t tc_fused_w_bytes(int passes, int rows, int K);
// Items t < nitems: K-block kb[t] of front fronts[t]; max_k bounds their pivots.
void launch_tc_w_pack(int bwd, int passes, DevFronts F, const int32_t* fronts, const int32_t* kb,
                      int32_t nitems, int32_t max_k, const int64_t* woff, const float* arena,
                      unsigned char* wpk, cudaStream_t s);
void launch_front_gemm_tc(int bwd, int cls, int passes, DevFronts F, const int32_t* fronts,
                          int32_t nfr, const int64_t* woff, const unsigned char* wpk,
                          const int64_t* block_ncols, int64_t j0, int32_t NR, float* X,
                          int64_t x_rows, float* Tb, int64_t tb_rows, float* D,
                          const uint8_t* pleaf, long long* err, int inject_wait, cudaStream_t s);
void launch_spike_gemm_tc(int op, int passes, DevFronts F, const int32_t* tile_front,
                          const int32_t* tile_m0, const int64_t* tile_aoff,
                          const unsigned char* atc, int32_t ntiles, const int64_t* block_ncols,
                          int64_t j0, int32_t NR, float* X, float* Tb, long long* err,
                          int inject_wait, cudaStream_t s);
template <typename T>
void launch_spike_gemm(int op, DevFronts F, const int32_t* tile_front, const int32_t* tile_m0,
                       int32_t ntiles, const T* arena, const int64_t* block_ncols, int64_t j0,
                       int32_t NR, T* X, T* Tb, cudaStream_t s);
// G^ stores its columns in panel order (the matvec's column list is permuted
// to match), so row q of G^ is a straight copy of the panel row of c[q].
template <typename T, typename TG>
void launch_ghat_extract(const int32_t* qblock, const int32_t* c_rownew, const int64_t* gq0,
                         const int64_t* gcol_ptr, const int64_t* ghat_off, const int64_t* gld,
                         int64_t m, int64_t j0, int32_t NR, const T* X, TG* ghat,
                         cudaStream_t s);

// ---- solve.cu ---------------------------------------------------------------
template <typename T>
void launch_permute_in(const double* y, const int32_t* perm, int64_t n, T* w, cudaStream_t s);
template <typename T>
void launch_permute_out(const T* w, const int32_t* perm, int64_t n, double* g, cudaStream_t s);
// Launch shapes of a block-solve depth (see launch_fwd1): automatic, one warp
// per front, one CTA per front with eight loads in flight per lane, or a
// cluster of 1, 2, 4 or 8 CTAs per front with thirty-two.
enum { SOLVE_AUTO = -1, SOLVE_WARP = 0, SOLVE_CTA8 = 1, SOLVE_CL1 = 2, SOLVE_CL2 = 3,
       SOLVE_CL4 = 4, SOLVE_CL8 = 5 };
inline int solve_cfg_cluster(int c) { return c >= 8 ? SOLVE_CL8 : c >= 4 ? SOLVE_CL4 : c >= 2 ? SOLVE_CL2 : SOLVE_CL1; }
inline int solve_cfg_size(int cfg) { return cfg == SOLVE_CL8 ? 8 : cfg == SOLVE_CL4 ? 4 : cfg == SOLVE_CL2 ? 2 : 1; }
template <typename T>
void launch_fwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, T* u, cudaStream_t s, int cfg = SOLVE_AUTO);
template <typename T>
void launch_bwd1(DevFronts F, const int32_t* list, int32_t nf, int32_t max_m, const T* arena,
                 T* w, cudaStream_t s, int cfg = SOLVE_AUTO);
// CSR product kernels (the autotuner picks per matrix): row blocks streamed
// through shared memory (SPMV_BLOCK: all of a thread's loads of the block
// issued at once, 16-byte vectors), 4 / 8 lanes per row, or 32-row groups
// per warp copied asynchronously into shared memory (SPMV_WARP).
enum { SPMV_STREAM = 0, SPMV_VEC4 = 1, SPMV_VEC8 = 2, SPMV_BLOCK = 3, SPMV_WARP = 4 };
void launch_spmv(const int32_t* rowptr, const int32_t* colind, const double* vals, int64_t n,
                 const double* x, double* y, cudaStream_t s, int variant = SPMV_STREAM);
// y_out = y - R~ zhat (R~ rows over original indices, reduced columns)
void launch_rt_residual(const int32_t* rt_rowptr, const int32_t* rt_col, const double* rt_val,
                        int64_t n, const double* y, const double* zhat, double* out,
                        cudaStream_t s, int variant = SPMV_STREAM);
// Implicit G^ product: q = R~ v (reduced columns), then w = v + g(c) with
// g = D~^-1 q from the block solve.
template <typename TI>
void launch_rt_apply(const int32_t* rt_rowptr, const int32_t* rt_col, const double* rt_val,
                     int64_t n, const TI* v, double* q, cudaStream_t s);
template <typename TI>
void launch_add_gathered(const TI* v, const double* g, const int64_t* c, int64_t m, TI* w,
                         cudaStream_t s);
template <typename TG, typename TI>
void launch_ghat_matvec(const TG* ghat, const int32_t* qblock, const int64_t* gq0,
                        const int64_t* gcol_ptr, const int64_t* ghat_off, const int64_t* gld,
                        const int32_t* gcols, int64_t m, const TI* v, TI* w, cudaStream_t s);
// Tiled G^ product: one CTA per (block, 64 reduced rows); needs max_cols
// entries of shared memory for the block's gathered vector.  With sc
// non-null, blocks of systems whose inner solve has stopped are skipped; with
// red non-null, the product also takes red's reductions and scalar step.
template <typename TG, typename TI>
void launch_ghat_matvec_tiled(const TG* ghat, const int32_t* tile_block, const int32_t* tile_row,
                              const int32_t* tile_h, int32_t ntiles, int64_t max_cols,
                              const int64_t* gq0,
                              const int64_t* gq1, const int64_t* gcol_ptr, const int64_t* ghat_off,
                              const int64_t* gld, const int32_t* gcols, const TI* v, TI* w,
                              const KScal* sc, const int32_t* block_sys, const MvRed* red,
                              cudaStream_t s);
void launch_gather(const double* src, const int64_t* idx, int64_t m, double* dst, cudaStream_t s);
void launch_gather_rt_values(const double* values, const int64_t* rt_src, int64_t nrt,
                             double* rt_val, cudaStream_t s);

}  // namespace ddps
