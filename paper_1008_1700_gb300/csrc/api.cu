// C ABI of the DDPS solver: handle lifetime, device layout and the host-side
// control of the numeric phases.  The arithmetic of every step runs in the
// kernels of factor.cu, solve.cu and krylov.cu; this file only sequences them.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <type_traits>
#include <string>
#include <vector>

#include "ddps.h"
#include "ddps_internal.h"
#include "krylov.h"
#include "launch.h"
#include "reduced_direct.h"

using namespace ddps;

namespace {

struct Fail {
  ddps_status st;
  std::string msg;
};

thread_local std::string g_last_error;

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw Fail{DDPS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};    \
  } while (0)

template <typename T>
size_t esize() {
  return sizeof(T);
}

size_t prec_size(int prec) { return prec == DDPS_FP64 ? 8 : (prec == DDPS_FP32 ? 4 : 2); }

}  // namespace

// Fronts of one depth reordered for the LU launches: `nsmall` fronts that fit
// the shared-memory kernel, then `nlarge` others, starting at `first`.
struct LevelSplit {
  int32_t first = 0, nsmall = 0, nlarge = 0, max_small_m = 0, max_m = 0;
  // multi-CTA LU of the large fronts: per panel step p (columns 32p..32p+31),
  // fronts [pf_ptr[p], pf_ptr[p+1]) of lu_panel_fronts and tiles
  // [pt_ptr[p], pt_ptr[p+1]) of lu_tile_front / lu_tile_ij
  std::vector<int64_t> pf_ptr, pt_ptr;
  // tensor-core block updates (update_prec BF16X3): per panel step p, tiles
  // [pc_ptr[p], pc_ptr[p+1]) of lu_tc_front / lu_tc_ij
  std::vector<int64_t> pc_ptr;
  // per panel step p: L21-row / U12-column chunks [pq_ptr[p], pq_ptr[p+1]) of
  // lu_pc_front / lu_pc_word
  std::vector<int64_t> pq_ptr;
  int32_t inv_first = 0, inv_ntiles = 0;  // multi-CTA inverse tiles of the large fronts
};

struct ddps_handle {
  std::string err;
  ddps_options opt{};
  Analysis A;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t launches = 0;

  // device copies of the pattern and maps
  int32_t *rowptr = nullptr, *colind = nullptr;
  double* vals = nullptr;
  int64_t* amap = nullptr;
  int32_t *perm = nullptr, *iperm = nullptr;
  // multifrontal structure
  DevFronts F{};
  int32_t* parent = nullptr;
  int32_t* level_fronts = nullptr;
  int32_t* ea_list = nullptr;
  std::vector<int32_t> ea_maxr;
  void* arena = nullptr;
  void* updv = nullptr;
  void* w = nullptr;
  double* rownorm = nullptr;
  long long* derr = nullptr;
  long long* herr = nullptr;  // pinned
  // R~
  int32_t *rt_rowptr = nullptr, *rt_col = nullptr, *rt_rhscol = nullptr, *rt_rownew = nullptr;
  int64_t* rt_src = nullptr;
  double* rt_val = nullptr;
  int64_t nrt = 0;
  // reduced system
  int64_t* c = nullptr;
  int32_t *c_rownew = nullptr, *qblock = nullptr, *gcols = nullptr;
  int32_t* block_sys = nullptr;  // system of each block
  int32_t* any_flag = nullptr;   // device flag: some system still iterating
  int32_t* any_host = nullptr;   // pinned copy
  int64_t *gq0 = nullptr, *gq1 = nullptr, *gcol_ptr = nullptr, *ghat_off = nullptr,
          *gld = nullptr, *block_ncols = nullptr;
  // tiles of the G^ product: block, first row and rows (64, or 256 for
  // blocks of fewer than 1024 coupling columns)
  int32_t *mv_block = nullptr, *mv_row = nullptr, *mv_h = nullptr;
  int32_t mv_ntiles = 0;
  // reductions folded into the tiled product: tiles per system, partial sums
  // (2 per tile) and per-system counters
  int32_t *mv_sys_tptr = nullptr, *mv_done = nullptr;
  double* mv_partial = nullptr;
  int64_t mv_max_cols = 0;
  void* ghat = nullptr;
  // spike panels: X (n x NR) and the fronts' working rows (sum of m x NR);
  // D (rows as U) receives the update rows of the fused forward products,
  // fz_flag marks those fronts for the parent's gather
  void* X = nullptr;
  void* U = nullptr;
  void* D = nullptr;
  uint8_t* fz_flag = nullptr;
  int32_t NR = 0;
  int32_t max_k = 0;
  // LU launch order per depth (see LevelSplit)
  int32_t* lu_order = nullptr;
  std::vector<LevelSplit> split;
  int32_t *lu_panel_fronts = nullptr, *lu_tile_front = nullptr, *lu_tile_ij = nullptr;
  int32_t *lu_tc_front = nullptr, *lu_tc_ij = nullptr;  // tensor-core block-update tiles
  int32_t *lu_pc_front = nullptr, *lu_pc_word = nullptr, *lu_pc_slot = nullptr;  // panel chunks
  void* lu_dinv = nullptr;  // 32 x 32 inverses of the panel's diagonal triangles, per front
  bool lu_tc = false;
  int32_t *inv_tile_front = nullptr, *inv_tile_cb = nullptr;
  int64_t* inv_off = nullptr;  // per front, offset of its 2 k^2 inverse entries in inv
  void* inv = nullptr;
  // spike GEMM tile lists per depth: backward tiles over the k pivot rows (tk),
  // forward tiles over the pivot rows (fk) and over the r update rows (tr).
  // With tensor-core spikes they hold only the fronts too large for the fused
  // front products; without, every front.
  int32_t *tk_front = nullptr, *tk_m0 = nullptr, *tr_front = nullptr, *tr_m0 = nullptr;
  int32_t *fk_front = nullptr, *fk_m0 = nullptr;
  std::vector<int32_t> tk_ptr, tr_ptr, fk_ptr;
  // fused front products (tensor-core spikes): packed W per front and direction
  // (byte offsets, -1 where the front takes the tile ops) and the backward
  // launch lists per (depth, class): [bz_ptr[4L + cls], bz_ptr[4L + cls + 1])
  unsigned char* wpk = nullptr;
  int64_t *woff_b = nullptr, *woff_f = nullptr;
  // W forming work: (front, K-block) items per direction (0 forward, 1 backward)
  // and class of the front's pivot count (shared memory of the launch)
  struct WpkList {
    int32_t* front = nullptr;
    int32_t* kb = nullptr;
    int32_t n = 0, max_k = 0;
  };
  WpkList wpk_items[2][3];
  int32_t* bz = nullptr;
  std::vector<int64_t> bz_ptr;
  // tensor-core spikes: A operands packed as bf16 blocks, byte offsets per op and tile
  unsigned char* atc = nullptr;
  int64_t* tc_aoff[4] = {nullptr, nullptr, nullptr, nullptr};
  // Sparse forward sweep of the spikes.  Each block's coupling columns are
  // ordered by the (postorder) front of their first entry; chunk c of NR
  // panel columns then only touches the fronts on the paths from its
  // columns' fronts to the roots: fw_active[c * nfronts + f] flags them, and
  // the forward launches of chunk c and depth L use lists of those fronts
  // and their tiles (index (c * nlevels + L) into the *_ptr vectors).
  std::vector<int32_t> gperm;  // panel column -> coupling column (G^ column order), per block
  uint8_t* fw_active = nullptr;
  // per (chunk, front): a fused forward front none of whose children is
  // active in the chunk; its working rows are its pivot rows of X, read
  // there by the fused product (no gather), and its parent's gather takes
  // only its own update rows (D)
  uint8_t* fw_pleaf = nullptr;
  // per chunk (tensor-core spikes): the fronts whose pivot rows of X are
  // cleared before the chunk (the active fronts, whose rows take the
  // right-hand side, and the fronts the fused backward products do not take;
  // the fused backward reads an inactive front's pivot rows as the zero row
  // n of X instead), [zr_ptr[c], zr_ptr[c + 1]) of zr_front
  int32_t* zr_front = nullptr;
  std::vector<int64_t> zr_ptr;
  int32_t *fw_g = nullptr, *fw_kf = nullptr, *fw_km = nullptr, *fw_rf = nullptr, *fw_rm = nullptr;
  int64_t *fw_ka = nullptr, *fw_ra = nullptr;  // packed-A offsets (tensor-core path)
  std::vector<int64_t> fw_g_ptr, fw_k_ptr, fw_r_ptr;
  // fused forward fronts per (chunk, depth, class): [fz_ptr[4q + cls], fz_ptr[4q + cls + 1])
  int32_t* fz = nullptr;
  std::vector<int64_t> fz_ptr;
  int32_t tc_max_kt[4] = {0, 0, 0, 0};
  int tc_passes = 0;
  // segments
  SegView Sn{}, Sm{};
  int32_t nseg = 0;
  // outer workspace (FP64, n)
  double *o_r = nullptr, *o_rhat = nullptr, *o_p = nullptr, *o_v = nullptr, *o_phat = nullptr,
         *o_s = nullptr, *o_shat = nullptr, *o_t = nullptr, *o_xt = nullptr, *o_tmp = nullptr;
  // preconditioner workspace
  double *pc_g = nullptr, *pc_ghat = nullptr, *pc_zhat = nullptr, *pc_t = nullptr;
  double *im_q = nullptr, *im_g = nullptr;  // implicit G^: R~ v and D~^-1 R~ v
  // host-buffer entry points stage f and x here
  double *io_f = nullptr, *io_x = nullptr;
  // inner workspace (inner precision, m)
  void *i_g = nullptr, *i_z = nullptr, *i_r = nullptr, *i_rh = nullptr, *i_p = nullptr,
       *i_v = nullptr, *i_s = nullptr, *i_t = nullptr;
  KScal *sc_out = nullptr, *sc_in = nullptr;
  KScal* hsc = nullptr;      // pinned host scalars of the loop being run (nseg)
  // Uploads copy hsc into a slot of this pinned ring first, so that the host
  // may change hsc right after enqueueing an upload; the ring restarts after
  // every synchronising download.
  KScal* hstage = nullptr;
  int stage_next = 0;
  KScal* hsc_out = nullptr;  // pinned, outer loop
  KScal* hsc_in = nullptr;   // pinned, inner loop
  double* partial = nullptr;
  // guess and first reduced solution
  double* guess = nullptr;
  bool has_guess = false;
  double *first_zhat = nullptr, *first_ghat = nullptr;
  bool factored = false;
  // per-class CUDA-event timing (ddps_set_profiling)
  int32_t prof_mask = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next = 0;
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_recs;
  double prof_ms[DDPS_PROF_CLASSES] = {};
  int64_t prof_cnt[DDPS_PROF_CLASSES] = {};
  // ILU(0) factors (factor_kind ILU0): CSR structure, levels, values
  IluDev il{};
  int32_t *il_lf = nullptr, *il_lb = nullptr;
  void* il_val = nullptr;
  // launch shape of every block-solve depth and sweep (SOLVE_AUTO until tuned)
  std::vector<int> tune_fwd, tune_bwd;
  std::vector<float> tune_fwd_ms, tune_bwd_ms;
  int tune_spmv = SPMV_STREAM, tune_rt = SPMV_STREAM;  // CSR product kernels for A and R~
  float tune_spmv_ms = 0.f, tune_rt_ms = 0.f;
  bool tuned = false;
  // persistent sweeps of the block solve over the levels >= persist_L (fronts of at
  // most kPersistM rows): orders, waits and flags (2 nfronts done flags, 2 counters)
  int32_t persist_L = -1, persist_n = 0, persist_max_m = 0;
  int32_t *p_fwd = nullptr, *p_bwd = nullptr, *p_wait = nullptr, *p_flags = nullptr;
  // direct solve of the reduced system (reduced_solver DIRECT)
  DirectPlan direct;
  bool use_direct = false;
  // CUDA graphs: launch sequences that repeat unchanged are captured once on
  // a stream of the handle and replayed (not while profiling is on)
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphExec_t g_inner = nullptr, g_factor = nullptr;
  int64_t g_inner_launches = 0, g_factor_launches = 0;
  struct PrecGraph {
    const double* y;
    double* z;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<PrecGraph> g_prec;
  // statistics of the current solve
  int64_t stat_inner = 0, stat_precond = 0;
  double stat_first_inner = 0;
  bool stat_guess_used = false;
};

namespace {

cudaEvent_t next_event(ddps_handle* h) {
  if (h->ev_next == h->ev_pool.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_next++];
}

// An NVTX range over a scope (API phases, kernel classes): host-side markers
// that a profiler can show or filter on; without one attached they do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* const kProfName[DDPS_PROF_CLASSES] = {
    "assemble",     "extend_add",  "front_lu", "spike_fwd",     "spike_bwd",   "ghat_extract",
    "block_solve",  "ghat_matvec", "spmv",     "direct_factor", "direct_solve"};

// Records a CUDA-event pair around the launches of one kernel class when that
// class is enabled in the profiling mask, inside an NVTX range named for the
// class.
struct Prof {
  ddps_handle* h;
  int cls;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  Prof(ddps_handle* hh, int c, cudaStream_t st) : h(hh), cls(c), s(st) {
    if (cls >= 0) nvtxRangePushA(kProfName[cls]);
    if (cls >= 0 && (h->prof_mask & (1 << cls))) {
      cudaEvent_t a = next_event(h);
      b = next_event(h);
      CK(cudaEventRecord(a, s));
      h->prof_recs.push_back({cls, a, b});
    }
  }
  ~Prof() {
    if (b) cudaEventRecord(b, s);
    if (cls >= 0) nvtxRangePop();
  }
};

void prof_collect(ddps_handle* h) {
  for (auto& r : h->prof_recs) {
    float ms = 0.f;
    CK(cudaEventSynchronize(r.b));
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof_ms[r.cls] += ms;
    h->prof_cnt[r.cls] += 1;
  }
  h->prof_recs.clear();
  h->ev_next = 0;
}

template <typename T>
T* dalloc(ddps_handle* h, int64_t count) {
  if (count <= 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{e == cudaErrorMemoryAllocation ? DDPS_ERR_OUT_OF_MEMORY : DDPS_ERR_CUDA,
               "cudaMalloc of " + std::to_string((long long)count * sizeof(T)) +
                   " bytes: " + cudaGetErrorString(e)};
  }
  h->allocs.push_back(p);
  h->bytes += count * (int64_t)sizeof(T);
  return (T*)p;
}

void* dalloc_bytes(ddps_handle* h, int64_t bytes) { return (void*)dalloc<unsigned char>(h, bytes); }

template <typename T>
T* dupload(ddps_handle* h, const std::vector<T>& v) {
  T* p = dalloc<T>(h, (int64_t)v.size());
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

// Chunk table of a segmented vector.
SegView make_segview(ddps_handle* h, const std::vector<int64_t>& seg_ptr) {
  // chunk length: about eight chunks per SM over the whole vector, between 256 and 8192
  const int64_t total = seg_ptr.empty() ? 0 : seg_ptr.back() - seg_ptr.front();
  const int64_t CH = std::min<int64_t>(8192, std::max<int64_t>(256, (total / (8 * 152) + 255) / 256 * 256));
  std::vector<int64_t> cb, ce;
  std::vector<int32_t> cs, scp;
  const int nseg = (int)seg_ptr.size() - 1;
  scp.push_back(0);
  for (int s = 0; s < nseg; ++s) {
    for (int64_t b = seg_ptr[s]; b < seg_ptr[s + 1]; b += CH) {
      cb.push_back(b);
      ce.push_back(std::min(b + CH, seg_ptr[s + 1]));
      cs.push_back(s);
    }
    if (seg_ptr[s + 1] == seg_ptr[s]) {  // an empty segment still gets its (empty) chunk
      cb.push_back(seg_ptr[s]);
      ce.push_back(seg_ptr[s]);
      cs.push_back(s);
    }
    scp.push_back((int32_t)cb.size());
  }
  SegView S{};
  S.chunk_beg = dupload(h, cb);
  S.chunk_end = dupload(h, ce);
  S.chunk_seg = dupload(h, cs);
  S.seg_chunk_ptr = dupload(h, scp);
  S.done = dupload(h, std::vector<int32_t>(std::max(nseg, 1), 0));
  S.nchunks = (int32_t)cb.size();
  S.nseg = nseg;
  return S;
}

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

void check_launch() {
  cudaError_t e = take_launch_error();
  const cudaError_t last = cudaGetLastError();
  if (e == cudaSuccess) e = last;
  if (e != cudaSuccess) throw Fail{DDPS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

// ---------------------------------------------------------------------------
// CUDA graphs.  A capture runs on the handle's own stream (the legacy default
// stream cannot be captured); a replay is ordered after the caller's stream
// and the caller's stream after it, through two events.
// ---------------------------------------------------------------------------
bool graphs_on(const ddps_handle* h) { return h->opt.use_graphs && h->prof_mask == 0; }

void ensure_graph_stream(ddps_handle* h) {
  if (h->gstream) return;
  CK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming));
}

// Captures the launches `body` enqueues on the handle's stream; returns the
// instantiated graph and adds the launches counted during capture to *count.
template <typename F>
cudaGraphExec_t capture_graph(ddps_handle* h, F body, int64_t* count) {
  ensure_graph_stream(h);
  const int64_t l0 = h->launches;
  CK(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed));
  try {
    body(h->gstream);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(h->gstream, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamEndCapture(h->gstream, &g));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  *count = h->launches - l0;
  h->launches = l0;
  return exec;
}

void replay_graph(ddps_handle* h, cudaGraphExec_t exec, int64_t count, cudaStream_t s) {
  CK(cudaEventRecord(h->gev[0], s));
  CK(cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
  CK(cudaGraphLaunch(exec, h->gstream));
  CK(cudaEventRecord(h->gev[1], h->gstream));
  CK(cudaStreamWaitEvent(s, h->gev[1], 0));
  h->launches += count;
}

// One spike GEMM op over a tile list: tensor cores for FP32 factors with
// bf16 spike products, SIMT otherwise.
template <typename T>
void spike_op(ddps_handle* h, int op, const int32_t* tf, const int32_t* tm, const int64_t* ta,
              int32_t nt, const T* arena, int64_t j0, T* X, T* Tb, cudaStream_t s) {
  if (nt <= 0) return;
  h->launches++;
  if constexpr (std::is_same<T, float>::value) {
    if (h->tc_passes) {
      launch_spike_gemm_tc(op, h->tc_passes, h->F, tf, tm, ta, h->atc, nt, h->block_ncols, j0,
                           h->NR, X, Tb, h->derr, h->opt.debug_wait_timeout, s);
      return;
    }
  }
  launch_spike_gemm<T>(op, h->F, tf, tm, nt, arena, h->block_ncols, j0, h->NR, X, Tb, s);
}

// The fused front products of one depth (tensor-core spikes): one launch per
// tensor-memory class, lists [ptr[cls], ptr[cls + 1]) of `list`.
template <typename T>
void fused_fronts(ddps_handle* h, bool bwd, const int32_t* list, const int64_t* ptr, int64_t j0,
                  T* X, T* Tb, const uint8_t* pleaf, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (!h->tc_passes) return;
    for (int cls = 0; cls < 4; ++cls) {
      const int32_t n = (int32_t)(ptr[cls + 1] - ptr[cls]);
      if (n <= 0) continue;
      launch_front_gemm_tc(bwd ? 1 : 0, cls, h->tc_passes, h->F, list + ptr[cls], n,
                           bwd ? h->woff_b : h->woff_f, h->wpk, h->block_ncols, j0, h->NR, X,
                           h->A.n + 1, Tb, (int64_t)h->A.idx.size(), (float*)h->D, pleaf,
                           h->derr, h->opt.debug_wait_timeout, s);
      h->launches++;
    }
  }
}

// ---------------------------------------------------------------------------
// Fig. 2 steps 2 and 4 on the device
// ---------------------------------------------------------------------------
// Fig. 2 steps 2 and 4 with ILU(0) block factors: scatter, level-scheduled
// factorisation, then the spikes by level-scheduled L and U solves on the
// panels of coupling columns.
template <typename T, typename TG>
void factor_launches_ilu(ddps_handle* h, cudaStream_t s) {
  const Analysis& A = h->A;
  T* a = (T*)h->il_val;
  CK(cudaMemsetAsync(h->derr, 0, 3 * sizeof(long long), s));
  {
    Prof pr(h, DDPS_PROF_ASSEMBLE, s);
    launch_assemble<T>(h->vals, h->amap, A.nnz, a, s);
    launch_row_absmax(h->rowptr, h->amap, h->vals, h->iperm, A.n, h->rownorm, s);
    h->launches += 2;
  }
  {
    Prof pr(h, DDPS_PROF_FRONT_LU, s);
    for (size_t l = 0; l + 1 < A.il_lf_ptr.size(); ++l) {
      launch_ilu0_level<T>(h->il_lf + A.il_lf_ptr[l], A.il_lf_ptr[l + 1] - A.il_lf_ptr[l], h->il, a,
                           h->rownorm, h->opt.pivot_tol, h->derr, s);
      h->launches++;
    }
  }
  launch_gather_rt_values(h->vals, h->rt_src, h->nrt, h->rt_val, s);
  h->launches++;
  const int64_t m = (int64_t)A.c.size();
  if (m > 0 && h->opt.ghat_mode == DDPS_GHAT_EXPLICIT) {
    T* X = (T*)h->X;
    const int32_t NR = h->NR;
    for (int64_t j0 = 0; j0 < A.max_rhs; j0 += NR) {
      CK(cudaMemsetAsync(X, 0, (size_t)A.n * NR * sizeof(T), s));
      launch_spike_rhs<T>(h->rt_rownew, h->rt_rhscol, h->rt_src, h->nrt, h->vals, j0, NR, X, s);
      h->launches++;
      {
        Prof pr(h, DDPS_PROF_SPIKE_FWD, s);
        for (size_t l = 0; l + 1 < A.il_lf_ptr.size(); ++l) {
          launch_ilu_panel_level<T>(true, h->il_lf + A.il_lf_ptr[l],
                                    A.il_lf_ptr[l + 1] - A.il_lf_ptr[l], h->il, a,
                                    h->block_ncols, j0, NR, X, s);
          h->launches++;
        }
      }
      {
        Prof pr(h, DDPS_PROF_SPIKE_BWD, s);
        for (size_t l = 0; l + 1 < A.il_lb_ptr.size(); ++l) {
          launch_ilu_panel_level<T>(false, h->il_lb + A.il_lb_ptr[l],
                                    A.il_lb_ptr[l + 1] - A.il_lb_ptr[l], h->il, a,
                                    h->block_ncols, j0, NR, X, s);
          h->launches++;
        }
      }
      Prof pr(h, DDPS_PROF_GHAT_EXTRACT, s);
      launch_ghat_extract<T, TG>(h->qblock, h->c_rownew, h->gq0, h->gcol_ptr, h->ghat_off, h->gld,
                                 m, j0, NR, X, (TG*)h->ghat, s);
      h->launches++;
    }
  }
  if (h->use_direct) {
    Prof pr(h, DDPS_PROF_DIRECT_FACTOR, s);
    h->launches += direct_factor<TG>(h->direct, (const TG*)h->ghat, s);
  }
  check_launch();
}

template <typename T, typename TG>
void factor_launches(ddps_handle* h, cudaStream_t s) {
  if (h->A.ilu) {
    factor_launches_ilu<T, TG>(h, s);
    return;
  }
  const Analysis& A = h->A;
  T* arena = (T*)h->arena;
  CK(cudaMemsetAsync(arena, 0, (size_t)A.arena_size * sizeof(T), s));
  CK(cudaMemsetAsync(h->derr, 0, 3 * sizeof(long long), s));
  {
    Prof pr(h, DDPS_PROF_ASSEMBLE, s);
    launch_assemble<T>(h->vals, h->amap, A.nnz, arena, s);
    launch_row_absmax(h->rowptr, h->amap, h->vals, h->iperm, A.n, h->rownorm, s);
  }
  h->launches += 2;
  const int S = A.max_children;
  for (int L = A.nlevels - 1; L >= 0; --L) {
    for (int sl = 0; sl < S; ++sl) {
      const int64_t q = (int64_t)L * S + sl;
      const int32_t cnt = A.ea_ptr[q + 1] - A.ea_ptr[q];
      if (cnt > 0) {
        Prof pr(h, DDPS_PROF_EXTEND_ADD, s);
        launch_extend_add_p<T>(h->F, h->parent, h->ea_list + A.ea_ptr[q], cnt, h->ea_maxr[q], arena, s);
        h->launches++;
      }
    }
    // fronts of this depth, small ones (shared-memory kernel) first, then the rest
    Prof pr(h, DDPS_PROF_FRONT_LU, s);
    const LevelSplit& ls = h->split[L];
    if (ls.nsmall > 0) {
      launch_front_lu_small<T>(h->F, h->lu_order + ls.first, ls.nsmall, ls.max_small_m, arena,
                               h->rownorm, h->opt.pivot_tol, h->derr, s);
      h->launches++;
    }
    if (ls.nlarge > 0) {
      for (size_t pstep = 0; pstep + 1 < ls.pf_ptr.size(); ++pstep) {
        const int32_t j0 = (int32_t)pstep * kLuPanel;
        launch_lu_panel<T>(h->F, h->lu_panel_fronts + ls.pf_ptr[pstep],
                           (int32_t)(ls.pf_ptr[pstep + 1] - ls.pf_ptr[pstep]),
                           h->lu_pc_front + ls.pq_ptr[pstep], h->lu_pc_word + ls.pq_ptr[pstep],
                           h->lu_pc_slot + ls.pq_ptr[pstep],
                           (int32_t)(ls.pq_ptr[pstep + 1] - ls.pq_ptr[pstep]), j0, arena,
                           (T*)h->lu_dinv, h->rownorm, h->opt.pivot_tol, h->derr, s);
        launch_lu_trailing<T>(h->F, h->lu_tile_front + ls.pt_ptr[pstep],
                              h->lu_tile_ij + ls.pt_ptr[pstep],
                              (int32_t)(ls.pt_ptr[pstep + 1] - ls.pt_ptr[pstep]), j0,
                              h->lu_tc ? 1 : 0, arena, s);
        h->launches += 1 + (ls.pq_ptr[pstep + 1] > ls.pq_ptr[pstep]) +
                       (ls.pt_ptr[pstep + 1] > ls.pt_ptr[pstep]);
        if constexpr (std::is_same<T, float>::value) {
          const int32_t nc = (int32_t)(ls.pc_ptr[pstep + 1] - ls.pc_ptr[pstep]);
          if (h->lu_tc && nc > 0) {
            launch_lu_update_tc(h->F, h->lu_tc_front + ls.pc_ptr[pstep], h->lu_tc_ij + ls.pc_ptr[pstep],
                                nc, j0, arena, h->derr, s);
            h->launches++;
          }
        }
      }
      launch_tri_inverse_mc<T>(h->F, h->inv_tile_front + ls.inv_first, h->inv_tile_cb + ls.inv_first,
                               ls.inv_ntiles, h->lu_order + ls.first + ls.nsmall, ls.nlarge, h->max_k,
                               arena, (T*)h->inv, h->inv_off, s);
      h->launches += 2;
    }
  }
  launch_gather_rt_values(h->vals, h->rt_src, h->nrt, h->rt_val, s);
  h->launches++;
  const int64_t m = (int64_t)A.c.size();
  if constexpr (std::is_same<T, float>::value) {
    if (h->tc_passes && m > 0) {  // pack the A operands of the tile ops and W of the fused fronts
      Prof pr(h, DDPS_PROF_SPIKE_FWD, s);
      for (int op = 0; op < 4; ++op) {
        const int32_t* tf = op == OP_FWD_L21 ? h->tr_front : op == OP_FWD_LINV ? h->fk_front : h->tk_front;
        const int32_t* tm = op == OP_FWD_L21 ? h->tr_m0 : op == OP_FWD_LINV ? h->fk_m0 : h->tk_m0;
        const int32_t nt = op == OP_FWD_L21 ? h->tr_ptr.back() : op == OP_FWD_LINV ? h->fk_ptr.back() : h->tk_ptr.back();
        if (nt > 0) {
          launch_tc_pack_a(op, h->tc_passes, h->F, tf, tm, h->tc_aoff[op], nt, h->tc_max_kt[op],
                           arena, h->atc, s);
          h->launches++;
        }
      }
      for (int dir = 1; dir >= 0; --dir)
        for (int cls = 0; cls < 3; ++cls) {
          const ddps_handle::WpkList& wl = h->wpk_items[dir][cls];
          if (wl.n <= 0) continue;
          launch_tc_w_pack(dir, h->tc_passes, h->F, wl.front, wl.kb, wl.n, wl.max_k,
                           dir ? h->woff_b : h->woff_f, arena, h->wpk, s);
          h->launches++;
        }
    }
  }
  if (m > 0 && h->opt.ghat_mode == DDPS_GHAT_EXPLICIT) {
    T* X = (T*)h->X;
    T* Tb = (T*)h->U;
    const int32_t NR = h->NR;
    const int64_t nf = (int64_t)A.f_k.size();
    for (int64_t j0 = 0, c = 0; j0 < A.max_rhs; j0 += NR, ++c) {
      if (h->zr_front) {
        launch_zero_front_rows<T>(h->F, h->zr_front + h->zr_ptr[c],
                                  (int32_t)(h->zr_ptr[c + 1] - h->zr_ptr[c]), NR, X, s);
        h->launches++;
      } else {
        CK(cudaMemsetAsync(X, 0, (size_t)A.n * NR * sizeof(T), s));
      }
      launch_spike_rhs<T>(h->rt_rownew, h->rt_rhscol, h->rt_src, h->nrt, h->vals, j0, NR, X, s);
      h->launches++;
      for (int L = A.nlevels - 1; L >= 0; --L) {
        Prof pr(h, DDPS_PROF_SPIKE_FWD, s);
        const int64_t q = c * A.nlevels + L;
        const int32_t ng = (int32_t)(h->fw_g_ptr[q + 1] - h->fw_g_ptr[q]);
        const uint8_t* pleaf = h->fw_pleaf ? h->fw_pleaf + c * nf : nullptr;
        launch_spike_gather<T>(h->F, h->fw_g + h->fw_g_ptr[q], ng, h->block_ncols, j0, NR, X, Tb,
                               h->fw_active + c * nf, (const T*)h->D, h->fz_flag, pleaf, s);
        h->launches += ng > 0;
        fused_fronts<T>(h, false, h->fz, h->fz_ptr.data() + 4 * q, j0, X, Tb, pleaf, s);
        spike_op<T>(h, OP_FWD_LINV, h->fw_kf + h->fw_k_ptr[q], h->fw_km + h->fw_k_ptr[q],
                    h->fw_ka ? h->fw_ka + h->fw_k_ptr[q] : nullptr, (int32_t)(h->fw_k_ptr[q + 1] - h->fw_k_ptr[q]),
                    arena, j0, X, Tb, s);
        spike_op<T>(h, OP_FWD_L21, h->fw_rf + h->fw_r_ptr[q], h->fw_rm + h->fw_r_ptr[q],
                    h->fw_ra ? h->fw_ra + h->fw_r_ptr[q] : nullptr, (int32_t)(h->fw_r_ptr[q + 1] - h->fw_r_ptr[q]),
                    arena, j0, X, Tb, s);
      }
      for (int L = 0; L < A.nlevels; ++L) {
        Prof pr(h, DDPS_PROF_SPIKE_BWD, s);
        fused_fronts<T>(h, true, h->bz, h->bz_ptr.data() + 4 * L, j0, X, Tb,
                        h->zr_front ? h->fw_active + c * nf : nullptr, s);
        const int32_t first = h->tk_ptr[L], nt = h->tk_ptr[L + 1] - h->tk_ptr[L];
        spike_op<T>(h, OP_BWD_U12, h->tk_front + first, h->tk_m0 + first,
                    h->tc_aoff[OP_BWD_U12] ? h->tc_aoff[OP_BWD_U12] + first : nullptr, nt, arena,
                    j0, X, Tb, s);
        spike_op<T>(h, OP_BWD_UINV, h->tk_front + first, h->tk_m0 + first,
                    h->tc_aoff[OP_BWD_UINV] ? h->tc_aoff[OP_BWD_UINV] + first : nullptr, nt, arena,
                    j0, X, Tb, s);
      }
      Prof pr(h, DDPS_PROF_GHAT_EXTRACT, s);
      launch_ghat_extract<T, TG>(h->qblock, h->c_rownew, h->gq0, h->gcol_ptr, h->ghat_off, h->gld,
                                 m, j0, NR, X, (TG*)h->ghat, s);
      h->launches++;
    }
  }
  if (h->use_direct) {
    Prof pr(h, DDPS_PROF_DIRECT_FACTOR, s);
    h->launches += direct_factor<TG>(h->direct, (const TG*)h->ghat, s);
  }
  check_launch();
}

// Fig. 2 steps 2-4 (and the block LU of G^ for a direct reduced solve):
// replayed from a graph after the first call unless profiling is on.
template <typename T, typename TG>
void factor_impl(ddps_handle* h, cudaStream_t s) {
  if (graphs_on(h)) {
    if (!h->g_factor)
      h->g_factor = capture_graph(h, [&](cudaStream_t gs) { factor_launches<T, TG>(h, gs); },
                                  &h->g_factor_launches);
    replay_graph(h, h->g_factor, h->g_factor_launches, s);
  } else {
    factor_launches<T, TG>(h, s);
  }
  CK(cudaMemcpyAsync(h->herr, h->derr, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h->herr[0] == 2)
    throw Fail{DDPS_ERR_TIMEOUT, "a bounded wait of the tensor-core spike products gave up"};
  if (h->herr[0] != 0) {
    const int64_t row_new = h->herr[2];
    const int64_t row_old = h->A.perm[row_new];
    const int32_t b =
        h->herr[1] >= 0 ? h->A.f_block[h->herr[1]]
                        : (int32_t)(std::upper_bound(h->A.block_ptr.begin(), h->A.block_ptr.end(),
                                                     row_old) - h->A.block_ptr.begin() - 1);
    throw Fail{DDPS_ERR_SINGULAR_BLOCK,
               "pivot below threshold in diagonal block " + std::to_string(b) + " at row " +
                   std::to_string((long long)row_old)};
  }
}

// ---------------------------------------------------------------------------
// Fig. 3 step 6.1 (and the second block solve of the retrieval)
// ---------------------------------------------------------------------------
// w, u: the permuted vector (n entries) and the fronts' update vectors; the
// handle's workspace unless the caller passes its own scratch.
template <typename T>
void block_solve_impl(ddps_handle* h, const double* y, double* g, cudaStream_t s, int prof_cls,
                      T* w = nullptr, T* u = nullptr) {
  const Analysis& A = h->A;
  if (!w) w = (T*)h->w;
  if (!u) u = (T*)h->updv;
  const T* arena = (const T*)h->arena;
  Prof pr(h, prof_cls, s);
  launch_permute_in<T>(y, h->perm, A.n, w, s);
  if (A.ilu) {  // (L~ U~)^-1 y: level-scheduled triangular solves
    const T* a = (const T*)h->il_val;
    for (size_t l = 0; l + 1 < A.il_lf_ptr.size(); ++l)
      launch_ilu_vec_level<T>(true, h->il_lf + A.il_lf_ptr[l], A.il_lf_ptr[l + 1] - A.il_lf_ptr[l],
                              h->il, a, w, s);
    for (size_t l = 0; l + 1 < A.il_lb_ptr.size(); ++l)
      launch_ilu_vec_level<T>(false, h->il_lb + A.il_lb_ptr[l], A.il_lb_ptr[l + 1] - A.il_lb_ptr[l],
                              h->il, a, w, s);
    launch_permute_out<T>(w, h->perm, A.n, g, s);
    h->launches += 2 + (int64_t)A.il_lf_ptr.size() - 1 + (int64_t)A.il_lb_ptr.size() - 1;
    return;
  }
  // levels >= top: one persistent launch per sweep; the levels above: one launch each
  const int top = h->persist_L >= 0 ? h->persist_L : A.nlevels;
  const int64_t nf = (int64_t)A.f_k.size();
  int32_t* done_f = h->p_flags;
  int32_t* done_b = h->p_flags + nf;
  if (h->persist_L >= 0) {
    CK(cudaMemsetAsync(h->p_flags, 0, (2 * nf + 2) * sizeof(int32_t), s));
    launch_fwd_persist<T>(h->F, h->p_fwd, h->persist_n, h->persist_max_m, arena, w, u, done_f,
                          h->p_flags + 2 * nf, h->derr, s);
    h->launches++;
  }
  for (int L = top - 1; L >= 0; --L)
    launch_fwd1<T>(h->F, h->level_fronts + A.level_ptr[L], A.level_ptr[L + 1] - A.level_ptr[L],
                   h->split[L].max_m, arena, w, u, s, h->tune_fwd.empty() ? SOLVE_AUTO : h->tune_fwd[L]);
  for (int L = 0; L < top; ++L)
    launch_bwd1<T>(h->F, h->level_fronts + A.level_ptr[L], A.level_ptr[L + 1] - A.level_ptr[L],
                   h->split[L].max_m, arena, w, s, h->tune_bwd.empty() ? SOLVE_AUTO : h->tune_bwd[L]);
  if (h->persist_L >= 0) {
    launch_bwd_persist<T>(h->F, h->p_bwd, h->persist_n, h->persist_max_m, h->p_wait, arena, w,
                          done_b, h->p_flags + 2 * nf + 1, h->derr, s);
    h->launches++;
  }
  launch_permute_out<T>(w, h->perm, A.n, g, s);
  h->launches += 2 + 2 * top;
}

// ---------------------------------------------------------------------------
// Autotuner of the block-solve launch shapes.  For every depth above the
// persistent sweeps and both sweeps, each candidate shape (warp per front
// when the fronts allow, one CTA with eight loads in flight, clusters of 1,
// 2, 4 and 8 CTAs) is timed with CUDA events on the handle's own factors
// (one untimed launch, then the mean of three), and the fastest is kept.
// Choices are cached per process by (device, precision, sweep, front count,
// largest front, total front entries) and, when the environment variable
// DDPS_TUNE_CACHE names a file, read from and written to that JSON object.
// ---------------------------------------------------------------------------
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;
bool g_tune_file_read = false;

void tune_cache_read() {
  const char* path = std::getenv("DDPS_TUNE_CACHE");
  if (g_tune_file_read || !path) return;
  g_tune_file_read = true;
  std::ifstream in(path);
  if (!in) return;
  std::stringstream ss;
  ss << in.rdbuf();
  const std::string t = ss.str();
  size_t i = 0;
  while ((i = t.find('"', i)) != std::string::npos) {
    const size_t j = t.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = t.substr(i + 1, j - i - 1);
    const size_t c = t.find(':', j);
    if (c == std::string::npos) break;
    g_tune_cache[key] = std::atoi(t.c_str() + c + 1);
    i = t.find_first_of(",}", c);
    if (i == std::string::npos) break;
  }
}

void tune_cache_write() {
  const char* path = std::getenv("DDPS_TUNE_CACHE");
  if (!path) return;
  std::ofstream out(path);
  out << "{";
  bool first = true;
  for (const auto& kv : g_tune_cache) {
    out << (first ? "\n" : ",\n") << "  \"" << kv.first << "\": " << kv.second;
    first = false;
  }
  out << "\n}\n";
}

template <typename T>
void autotune_block_solve(ddps_handle* h, cudaStream_t s) {
  const Analysis& A = h->A;
  const int top = h->persist_L >= 0 ? h->persist_L : A.nlevels;
  h->tune_fwd.assign(A.nlevels, SOLVE_AUTO);
  h->tune_bwd.assign(A.nlevels, SOLVE_AUTO);
  h->tune_fwd_ms.assign(A.nlevels, 0.f);
  h->tune_bwd_ms.assign(A.nlevels, 0.f);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  T* w = (T*)h->w;
  T* u = (T*)h->updv;
  const T* arena = (const T*)h->arena;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_cache_read();
  bool added = false;
  for (int L = 0; L < top; ++L) {
    const int32_t nf = A.level_ptr[L + 1] - A.level_ptr[L];
    const int32_t mm = h->split[L].max_m;
    int64_t ent = 0;
    for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q)
      ent += (int64_t)A.f_m[A.level_fronts[q]] * A.f_m[A.level_fronts[q]];
    const int32_t* list = h->level_fronts + A.level_ptr[L];
    for (int sweep = 0; sweep < 2; ++sweep) {
      const std::string key = std::string(prop.name) + "|" + std::to_string(sizeof(T)) + "|" +
                              (sweep ? "bwd" : "fwd") + "|" + std::to_string(nf) + "|" +
                              std::to_string(mm) + "|" + std::to_string(ent);
      int best = SOLVE_AUTO;
      float best_ms = 0.f;
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        best = it->second;
      } else {
        for (int cfg = SOLVE_WARP; cfg <= SOLVE_CL8; ++cfg) {
          if (cfg == SOLVE_WARP && mm > kPersistM) continue;
          auto run = [&]() {
            if (sweep == 0)
              launch_fwd1<T>(h->F, list, nf, mm, arena, w, u, s, cfg);
            else
              launch_bwd1<T>(h->F, list, nf, mm, arena, w, s, cfg);
          };
          run();
          CK(cudaEventRecord(e0, s));
          for (int r = 0; r < 3; ++r) run();
          CK(cudaEventRecord(e1, s));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          ms /= 3.f;
          if (best == SOLVE_AUTO || ms < best_ms) {
            best = cfg;
            best_ms = ms;
          }
        }
        check_launch();
        g_tune_cache[key] = best;
        added = true;
      }
      (sweep ? h->tune_bwd : h->tune_fwd)[L] = best;
      (sweep ? h->tune_bwd_ms : h->tune_fwd_ms)[L] = best_ms;
    }
  }
  // CSR product kernels for A (outer iteration) and R~ (retrieval), timed on
  // the handle's matrices with scratch vectors of the outer workspace
  for (int which = 0; which < 2; ++which) {
    const int64_t nn = A.n;
    const std::string key = std::string(prop.name) + "|csr|" + (which ? "rt" : "a") + "|" +
                            std::to_string(nn) + "|" +
                            std::to_string(which ? (int64_t)h->nrt : A.nnz);
    int best = SPMV_STREAM;
    float best_ms = 0.f;
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
    } else if (!which || h->nrt > 0) {
      CK(cudaMemsetAsync(h->o_tmp, 0, nn * sizeof(double), s));
      CK(cudaMemsetAsync(h->pc_zhat, 0, std::max<int64_t>((int64_t)A.c.size(), 1) * sizeof(double), s));
      for (int v = SPMV_STREAM; v <= SPMV_WARP; ++v) {
        auto run = [&]() {
          if (which == 0)
            launch_spmv(h->rowptr, h->colind, h->vals, nn, h->o_tmp, h->o_xt, s, v);
          else
            launch_rt_residual(h->rt_rowptr, h->rt_col, h->rt_val, nn, h->o_tmp, h->pc_zhat,
                               h->o_xt, s, v);
        };
        run();
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) run();
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (v == SPMV_STREAM || ms < best_ms) {
          best = v;
          best_ms = ms;
        }
      }
      check_launch();
      g_tune_cache[key] = best;
      added = true;
    }
    (which ? h->tune_rt : h->tune_spmv) = best;
    (which ? h->tune_rt_ms : h->tune_spmv_ms) = best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (added || (std::getenv("DDPS_TUNE_CACHE") && !std::ifstream(std::getenv("DDPS_TUNE_CACHE"))))
    tune_cache_write();
  h->tuned = true;
}

void block_solve(ddps_handle* h, const double* y, double* g, cudaStream_t s,
                 int prof_cls = DDPS_PROF_BLOCK_SOLVE) {
  if (h->opt.factor_prec == DDPS_FP64)
    block_solve_impl<double>(h, y, g, s, prof_cls);
  else
    block_solve_impl<float>(h, y, g, s, prof_cls);
}

// Whether the G^ product runs the tiled kernel (which can take the inner
// iteration's reductions).
template <typename TG>
bool ghat_tiled(const ddps_handle* h) {
  using AT = typename std::conditional<std::is_same<TG, double>::value, double, float>::type;
  return h->opt.ghat_mode != DDPS_GHAT_IMPLICIT && h->mv_max_cols * (int64_t)sizeof(AT) <= 200 * 1024;
}

template <typename TG, typename TI>
void ghat_matvec(ddps_handle* h, const TI* v, TI* w, cudaStream_t s, const KScal* sc = nullptr,
                 const MvRed* red = nullptr) {
  Prof pr(h, DDPS_PROF_GHAT_MATVEC, s);
  if (h->opt.ghat_mode == DDPS_GHAT_IMPLICIT) {
    // G^ v = v + (D~^-1 R~ v)(c): every system is computed (a stopped
    // system's output is not read by its masked Krylov updates)
    launch_rt_apply<TI>(h->rt_rowptr, h->rt_col, h->rt_val, h->A.n, v, h->im_q, s);
    block_solve(h, h->im_q, h->im_g, s, -1);
    launch_add_gathered<TI>(v, h->im_g, h->c, (int64_t)h->A.c.size(), w, s);
    h->launches += 2;
    return;
  }
  if (ghat_tiled<TG>(h)) {
    // every block owning reduced rows has tiles (a block without coupling
    // columns gets w = v on its rows)
    launch_ghat_matvec_tiled<TG, TI>((const TG*)h->ghat, h->mv_block, h->mv_row, h->mv_h, h->mv_ntiles,
                                     h->mv_max_cols, h->gq0, h->gq1, h->gcol_ptr, h->ghat_off,
                                     h->gld, h->gcols, v, w, sc, h->block_sys, red, s);
  } else {
    launch_ghat_matvec<TG, TI>((const TG*)h->ghat, h->qblock, h->gq0, h->gcol_ptr, h->ghat_off,
                               h->gld, h->gcols, (int64_t)h->A.c.size(), v, w, s);
  }
  h->launches++;
}

constexpr int kStageSlots = 16;

void download_sc(ddps_handle* h, const KScal* d, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->hsc, d, sizeof(KScal) * h->nseg, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->stage_next = 0;  // every earlier upload has completed
}
void upload_sc(ddps_handle* h, KScal* d, cudaStream_t s) {
  if (h->stage_next == kStageSlots) {
    CK(cudaStreamSynchronize(s));
    h->stage_next = 0;
  }
  KScal* slot = h->hstage + (size_t)h->stage_next++ * h->nseg;
  std::memcpy(slot, h->hsc, sizeof(KScal) * h->nseg);
  CK(cudaMemcpyAsync(d, slot, sizeof(KScal) * h->nseg, cudaMemcpyHostToDevice, s));
}

RedSpec red(const void* x, const void* y, int op, double* out) { return RedSpec{x, y, op, kScalStride, out}; }
RedSpec nored() { return RedSpec{nullptr, nullptr, 0, 0, nullptr}; }

// ---------------------------------------------------------------------------
// Fig. 3 step 6.3: unpreconditioned BiCGStab on G^ z^ = g^, per system,
// stopping on ||g^ - G^ z^||_2 <= tol_in ||g^||_2 or maxit_in iterations.
// Returns the largest iteration count over the systems (half steps 0.5).
// ---------------------------------------------------------------------------
template <typename TG, typename TI>
double inner_solve(ddps_handle* h, const double* ghat64, double* zhat64, const double* z0,
                   cudaStream_t s) {
  const int64_t m = (int64_t)h->A.c.size();
  const SegView& S = h->Sm;
  const int ns = h->nseg;
  KScal* sc = h->sc_in;
  struct HostScalars {  // the inner loop keeps its own pinned scalars
    ddps_handle* h;
    KScal* saved;
    explicit HostScalars(ddps_handle* hh) : h(hh), saved(hh->hsc) { h->hsc = h->hsc_in; }
    ~HostScalars() { h->hsc = saved; }
  } host_scalars(h);
  TI *g = (TI*)h->i_g, *z = (TI*)h->i_z, *r = (TI*)h->i_r, *rh = (TI*)h->i_rh, *p = (TI*)h->i_p,
     *v = (TI*)h->i_v, *sv = (TI*)h->i_s, *t = (TI*)h->i_t;
  convert<TI, double>(m, ghat64, g, s);
  CK(cudaMemsetAsync(z, 0, m * sizeof(TI), s));
  CK(cudaMemsetAsync(p, 0, m * sizeof(TI), s));
  CK(cudaMemsetAsync(v, 0, m * sizeof(TI), s));
  CK(cudaMemsetAsync(sc, 0, ns * sizeof(KScal), s));
  seg_reduce<TI>(S, 1, red(g, nullptr, 1, &sc[0].ref), nored(), nored(), h->partial, s);
  CK(cudaMemcpyAsync(r, g, m * sizeof(TI), cudaMemcpyDeviceToDevice, s));
  h->launches += 3;
  download_sc(h, sc, s);
  const double tol = h->opt.tol_in;
  std::vector<double> iters(ns, 0.0);
  for (int q = 0; q < ns; ++q) {
    KScal& k = h->hsc[q];
    k.active = k.ref > 0.0;
    k.flag = 0;
    k.half_done = 0;
    k.rho_old = k.alpha = k.omega = 1.0;
  }
  upload_sc(h, sc, s);
  if (z0) {
    convert<TI, double>(m, z0, z, s);
    ghat_matvec<TG, TI>(h, z, v, s);
    vec_sub<TI>(S, sc, 1, g, v, r, s);
    seg_reduce<TI>(S, 1, red(r, nullptr, 1, &sc[0].nrm), nored(), nored(), h->partial, s);
    h->launches += 4;
    download_sc(h, sc, s);
    bool any_reject = false;
    for (int q = 0; q < ns; ++q) {
      KScal& k = h->hsc[q];
      k.flag = 0;
      if (!k.active) continue;
      if (!(k.nrm < k.ref)) {
        k.flag = 1;  // the guess is worse than zero: start this system from zero
        any_reject = true;
      } else {
        h->stat_guess_used = true;
        if (k.nrm <= tol * k.ref) k.active = 0;
      }
    }
    upload_sc(h, sc, s);
    if (any_reject) {
      masked_zero<TI>(S, sc, z, s);
      masked_axpy<TI>(S, sc, r, g, nullptr, s);
      h->launches += 2;
    }
    for (int q = 0; q < ns; ++q) h->hsc[q].flag = 0;
    upload_sc(h, sc, s);
    CK(cudaMemsetAsync(v, 0, m * sizeof(TI), s));
  }
  CK(cudaMemcpyAsync(rh, r, m * sizeof(TI), cudaMemcpyDeviceToDevice, s));
  // Iterations are enqueued without waiting: the convergence tests run on the
  // device (fused into the reductions), stopped systems skip every kernel, and
  // the host looks at a single "some system still iterating" flag every
  // kCheckEvery iterations.
  constexpr int kCheckEvery = 4;
  const bool graphed = graphs_on(h) && h->opt.maxit_in > 0;
  // rho and beta of the first iteration; every later iteration's come from
  // the previous one's update of r (POST_CHECK_FULL_BETA)
  seg_reduce_post<TI>(S, 1, red(rh, r, 0, &sc[0].rho), nored(), nored(), h->partial, POST_BETA,
                      sc, tol, graphed ? -h->opt.maxit_in : 1, s);
  h->launches++;
  // one BiCGStab iteration; `it` < 0: the iteration number lives on the device
  // with the tiled G^ product, sigma and (t, s), (t, t) are reduced by the
  // products themselves, which also take the alpha and omega steps
  const bool fold = ghat_tiled<TG>(h);
  auto iteration = [&](int it, cudaStream_t st) {
    update_p<TI>(S, sc, r, p, v, st);
    if (fold) {
      MvRed ra;
      ra.nred = 1;
      ra.x = rh;
      ra.partial = h->mv_partial;
      ra.done = h->mv_done;
      ra.sys_tptr = h->mv_sys_tptr;
      ra.sc = sc;
      ra.post = POST_ALPHA;
      ra.tol = tol;
      ra.it = it;
      ghat_matvec<TG, TI>(h, p, v, st, sc, &ra);
    } else {
      ghat_matvec<TG, TI>(h, p, v, st, sc);
      seg_reduce_post<TI>(S, 1, red(rh, v, 0, &sc[0].sigma), nored(), nored(), h->partial,
                          POST_ALPHA, sc, tol, it, st);
      h->launches++;
    }
    update_s_norm<TI>(S, sc, r, v, sv, h->partial, tol, it, st);
    if (fold) {
      MvRed ro;
      ro.nred = 2;
      ro.partial = h->mv_partial;
      ro.done = h->mv_done;
      ro.sys_tptr = h->mv_sys_tptr;
      ro.sc = sc;
      ro.post = POST_OMEGA;
      ro.tol = tol;
      ro.it = it;
      ghat_matvec<TG, TI>(h, sv, t, st, sc, &ro);
    } else {
      ghat_matvec<TG, TI>(h, sv, t, st, sc);
      seg_reduce_post<TI>(S, 2, red(t, sv, 0, &sc[0].ts), red(t, t, 0, &sc[0].tt), nored(),
                          h->partial, POST_OMEGA, sc, tol, it, st);
      h->launches++;
    }
    update_xr_norm<TI>(S, sc, z, p, sv, r, t, rh, h->partial, tol, it, st);
    h->launches += 3;  // the two G^ products count their own launches
  };
  if (graphed) {
    // kCheckEvery iterations and the "some system still iterating" flag, one
    // graph replayed until every system has stopped (the device counter
    // stops a system after maxit_in iterations)
    if (!h->g_inner)
      h->g_inner = capture_graph(
          h,
          [&](cudaStream_t gs) {
            for (int q = 0; q < kCheckEvery; ++q) iteration(-h->opt.maxit_in, gs);
            any_active(ns, sc, h->any_flag, gs);
            CK(cudaMemcpyAsync(h->any_host, h->any_flag, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               gs));
            h->launches++;
          },
          &h->g_inner_launches);
    for (int it = 0; it < h->opt.maxit_in; it += kCheckEvery) {
      replay_graph(h, h->g_inner, h->g_inner_launches, s);
      CK(cudaStreamSynchronize(s));
      h->stage_next = 0;
      if (!*h->any_host) break;
    }
  } else {
    for (int it = 1; it <= h->opt.maxit_in; ++it) {
      if ((it - 1) % kCheckEvery == 0) {
        any_active(ns, sc, h->any_flag, s);
        CK(cudaMemcpyAsync(h->any_host, h->any_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->stage_next = 0;
        h->launches++;
        if (!*h->any_host) break;
      }
      iteration(it, s);
    }
  }
  download_sc(h, sc, s);
  for (int q = 0; q < ns; ++q) iters[q] = h->hsc[q].iters;
  convert<double, TI>(m, z, zhat64, s);
  h->launches++;
  double mx = 0;
  for (double v2 : iters) mx = std::max(mx, v2);
  for (int q = 0; q < ns; ++q)
    if (h->hsc[q].active) mx = std::max(mx, (double)h->opt.maxit_in);
  return mx;
}

double inner_dispatch(ddps_handle* h, const double* ghat64, double* zhat64, const double* z0,
                      cudaStream_t s) {
  NvtxRange nv("reduced_solve");
  const int gp = h->opt.ghat_prec, ip = h->opt.inner_prec;
  if (gp == DDPS_FP64) return inner_solve<double, double>(h, ghat64, zhat64, z0, s);
  if (gp == DDPS_FP32)
    return ip == DDPS_FP64 ? inner_solve<float, double>(h, ghat64, zhat64, z0, s)
                           : inner_solve<float, float>(h, ghat64, zhat64, z0, s);
  if (gp == DDPS_FP16)
    return ip == DDPS_FP64 ? inner_solve<__half, double>(h, ghat64, zhat64, z0, s)
                           : inner_solve<__half, float>(h, ghat64, zhat64, z0, s);
  return ip == DDPS_FP64 ? inner_solve<__nv_bfloat16, double>(h, ghat64, zhat64, z0, s)
                         : inner_solve<__nv_bfloat16, float>(h, ghat64, zhat64, z0, s);
}

// Fig. 3 with the direct reduced solve: a fixed launch sequence for given
// y and z, so it is replayed from a graph per (y, z) pair.
void precond_direct_launches(ddps_handle* h, const double* y, double* z, cudaStream_t s);

// Fig. 3: z = P^-1 y.
void precond_apply(ddps_handle* h, const double* y, double* z, cudaStream_t s, bool first) {
  const int64_t m = (int64_t)h->A.c.size();
  if (h->use_direct && m > 0) {
    if (graphs_on(h)) {
      ddps_handle::PrecGraph* pg = nullptr;
      for (auto& q : h->g_prec)
        if (q.y == y && q.z == z) pg = &q;
      if (!pg) {
        ddps_handle::PrecGraph q{y, z, nullptr, 0};
        q.exec = capture_graph(h, [&](cudaStream_t gs) { precond_direct_launches(h, y, z, gs); },
                               &q.launches);
        h->g_prec.push_back(q);
        pg = &h->g_prec.back();
      }
      replay_graph(h, pg->exec, pg->launches, s);
    } else {
      precond_direct_launches(h, y, z, s);
    }
    if (first) {
      h->stat_first_inner = 0;
      CK(cudaMemcpyAsync(h->first_zhat, h->pc_zhat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(h->first_ghat, h->pc_ghat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    h->stat_precond++;
    return;
  }
  block_solve(h, y, h->pc_g, s);                                        // 6.1
  if (m == 0) {
    CK(cudaMemcpyAsync(z, h->pc_g, h->A.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    h->stat_precond++;
    return;
  }
  launch_gather(h->pc_g, h->c, m, h->pc_ghat, s);                        // 6.2
  h->launches++;
  const double* z0 = (first && h->has_guess) ? h->guess : nullptr;
  const double its = inner_dispatch(h, h->pc_ghat, h->pc_zhat, z0, s);  // 6.3
  h->stat_inner += (int64_t)std::ceil(its);
  if (first) {
    h->stat_first_inner = its;
    CK(cudaMemcpyAsync(h->first_zhat, h->pc_zhat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->first_ghat, h->pc_ghat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  // 6.4-6.5: z = g - G(:,c) z^ = D~^-1 (y - R~ z^)
  launch_rt_residual(h->rt_rowptr, h->rt_col, h->rt_val, h->A.n, y, h->pc_zhat, h->pc_t, s, h->tune_rt);
  h->launches++;
  block_solve(h, h->pc_t, z, s);
  h->stat_precond++;
}

void precond_direct_launches(ddps_handle* h, const double* y, double* z, cudaStream_t s) {
  const int64_t m = (int64_t)h->A.c.size();
  block_solve(h, y, h->pc_g, s);                       // 6.1
  launch_gather(h->pc_g, h->c, m, h->pc_ghat, s);       // 6.2
  h->launches++;
  {
    Prof pr(h, DDPS_PROF_DIRECT_SOLVE, s);             // 6.3 by the block LU of G^
    h->launches += direct_solve(h->direct, h->pc_ghat, h->pc_zhat, s);
  }
  // 6.4-6.5: z = D~^-1 (y - R~ z^)
  launch_rt_residual(h->rt_rowptr, h->rt_col, h->rt_val, h->A.n, y, h->pc_zhat, h->pc_t, s, h->tune_rt);
  h->launches++;
  block_solve(h, h->pc_t, z, s);
}

// ---------------------------------------------------------------------------
// Fig. 2 step 6: right-preconditioned BiCGStab on A x = f (FP64), per system,
// convergence on the recomputed true residual ||f - A x||_inf <= tol ||f||_inf.
// ---------------------------------------------------------------------------
ddps_status solve_impl(ddps_handle* h, const double* f, double* x, const double* x0,
                       cudaStream_t s, ddps_solve_info* info) {
  const Analysis& A = h->A;
  const int64_t n = A.n;
  const SegView& S = h->Sn;
  const int ns = h->nseg;
  KScal* sc = h->sc_out;
  auto spmv = [&](const double* in, double* out) {
    Prof pr(h, DDPS_PROF_SPMV, s);
    launch_spmv(h->rowptr, h->colind, h->vals, n, in, out, s, h->tune_spmv);
    h->launches++;
  };
  h->stat_inner = 0;
  h->stat_precond = 0;
  h->stat_first_inner = 0;
  h->stat_guess_used = false;
  CK(cudaMemsetAsync(h->o_p, 0, n * sizeof(double), s));
  CK(cudaMemsetAsync(h->o_v, 0, n * sizeof(double), s));
  CK(cudaMemsetAsync(sc, 0, ns * sizeof(KScal), s));
  if (x0) {  // r0 = f - A x0
    CK(cudaMemcpyAsync(x, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    spmv(x, h->o_tmp);
    vec_sub<double>(S, sc, 1, f, h->o_tmp, h->o_r, s);
    h->launches++;
  } else {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    CK(cudaMemcpyAsync(h->o_r, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CK(cudaMemcpyAsync(h->o_rhat, h->o_r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  seg_reduce<double>(S, 2, red(f, nullptr, 2, &sc[0].ref), red(h->o_r, nullptr, 2, &sc[0].nrm2),
                     nored(), h->partial, s);
  h->launches += 2;
  download_sc(h, sc, s);
  const double tol = h->opt.tol_out;
  std::vector<double> iters(ns, 0.0);
  std::vector<int> conv(ns, 0);
  bool zero_rhs = false;
  for (int q = 0; q < ns; ++q) {
    KScal& k = h->hsc[q];
    // a zero right-hand side has the solution 0; a guess that already meets
    // the tolerance is the answer
    k.active = k.ref > 0.0 && k.nrm2 > tol * k.ref;
    k.flag = x0 && k.ref == 0.0;
    zero_rhs |= k.flag != 0;
    conv[q] = !k.active;
    k.rho_old = k.alpha = k.omega = 1.0;
  }
  upload_sc(h, sc, s);
  if (zero_rhs) {
    masked_zero<double>(S, sc, x, s);
    h->launches++;
    for (int q = 0; q < ns; ++q) h->hsc[q].flag = 0;
    upload_sc(h, sc, s);
  }
  auto any_active = [&]() {
    for (int q = 0; q < ns; ++q)
      if (h->hsc[q].active) return true;
    return false;
  };
  bool first = true;
  for (int it = 1; it <= h->opt.maxit_out && any_active(); ++it) {
    seg_reduce<double>(S, 1, red(h->o_rhat, h->o_r, 0, &sc[0].rho), nored(), nored(), h->partial, s);
    sc_beta(ns, sc, it == 1, s);
    update_p<double>(S, sc, h->o_r, h->o_p, h->o_v, s);
    h->launches += 4;
    precond_apply(h, h->o_p, h->o_phat, s, first);
    first = false;
    spmv(h->o_phat, h->o_v);
    seg_reduce<double>(S, 1, red(h->o_rhat, h->o_v, 0, &sc[0].sigma), nored(), nored(), h->partial, s);
    sc_alpha(ns, sc, s);
    update_s<double>(S, sc, h->o_r, h->o_v, h->o_s, s);
    seg_reduce<double>(S, 1, red(h->o_s, nullptr, 2, &sc[0].nrm), nored(), nored(), h->partial, s);
    h->launches += 6;
    download_sc(h, sc, s);
    bool cand = false;
    for (int q = 0; q < ns; ++q) {
      KScal& k = h->hsc[q];
      k.flag = k.active && k.nrm <= tol * k.ref;
      cand |= k.flag != 0;
    }
    if (cand) {
      upload_sc(h, sc, s);
      masked_axpy<double>(S, sc, h->o_xt, x, h->o_phat, s);  // x + alpha phat
      spmv(h->o_xt, h->o_tmp);
      vec_sub<double>(S, sc, 1, f, h->o_tmp, h->o_tmp, s);
      seg_reduce<double>(S, 1, red(h->o_tmp, nullptr, 2, &sc[0].nrm2), nored(), nored(), h->partial, s);
      h->launches += 5;
      download_sc(h, sc, s);
      for (int q = 0; q < ns; ++q) {
        KScal& k = h->hsc[q];
        if (!k.flag) continue;
        if (k.nrm2 <= tol * k.ref) {
          k.active = 0;
          conv[q] = 1;
          iters[q] = it - 0.5;
        } else {
          k.flag = 0;
        }
      }
      upload_sc(h, sc, s);
      masked_axpy<double>(S, sc, x, h->o_xt, nullptr, s);
      h->launches++;
      for (int q = 0; q < ns; ++q) h->hsc[q].flag = 0;
      upload_sc(h, sc, s);
    }
    if (!any_active()) break;
    precond_apply(h, h->o_s, h->o_shat, s, false);
    spmv(h->o_shat, h->o_t);
    seg_reduce<double>(S, 2, red(h->o_t, h->o_s, 0, &sc[0].ts), red(h->o_t, h->o_t, 0, &sc[0].tt),
                       nored(), h->partial, s);
    sc_omega(ns, sc, s);
    update_xr<double>(S, sc, 0, x, h->o_phat, h->o_shat, h->o_r, h->o_s, h->o_t, s);
    seg_reduce<double>(S, 1, red(h->o_r, nullptr, 2, &sc[0].nrm), nored(), nored(), h->partial, s);
    h->launches += 6;
    download_sc(h, sc, s);
    cand = false;
    for (int q = 0; q < ns; ++q) {
      KScal& k = h->hsc[q];
      if (!k.active) continue;
      iters[q] = it;
      k.flag = k.nrm <= tol * k.ref;
      cand |= k.flag != 0;
      if (!k.flag && (k.omega == 0.0 || k.breakdown)) k.active = 0;  // breakdown: stop unconverged
    }
    if (cand) {
      upload_sc(h, sc, s);
      spmv(x, h->o_tmp);
      vec_sub<double>(S, sc, 1, f, h->o_tmp, h->o_tmp, s);
      seg_reduce<double>(S, 1, red(h->o_tmp, nullptr, 2, &sc[0].nrm2), nored(), nored(), h->partial, s);
      h->launches += 3;
      download_sc(h, sc, s);
      for (int q = 0; q < ns; ++q) {
        KScal& k = h->hsc[q];
        if (!k.flag) continue;
        if (k.nrm2 <= tol * k.ref) {
          k.active = 0;
          conv[q] = 1;
          k.flag = 0;
        }  // else keep flag: replace the recurrence residual by the true one
      }
      upload_sc(h, sc, s);
      masked_axpy<double>(S, sc, h->o_r, h->o_tmp, nullptr, s);
      h->launches++;
      for (int q = 0; q < ns; ++q) h->hsc[q].flag = 0;
    }
    upload_sc(h, sc, s);
  }
  // final true residual of every system (and the block solves' wait record)
  CK(cudaMemcpyAsync(h->herr, h->derr, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  spmv(x, h->o_tmp);
  vec_sub<double>(S, sc, 1, f, h->o_tmp, h->o_tmp, s);
  seg_reduce<double>(S, 1, red(h->o_tmp, nullptr, 2, &sc[0].nrm2), nored(), nored(), h->partial, s);
  h->launches += 2;
  download_sc(h, sc, s);
  check_launch();
  if (h->herr[0] == 2)
    throw Fail{DDPS_ERR_TIMEOUT, "a bounded wait of the persistent block-solve sweeps gave up"};
  bool all = true;
  double worst = 0, maxit = 0;
  for (int q = 0; q < ns; ++q) {
    const KScal& k = h->hsc[q];
    const double rr = k.ref > 0 ? k.nrm2 / k.ref : 0.0;
    worst = std::max(worst, rr);
    maxit = std::max(maxit, iters[q]);
    if (!conv[q] && !(rr <= tol)) all = false;
  }
  if (info) {
    info->outer_iterations = maxit;
    info->inner_iterations = (int32_t)h->stat_inner;
    info->precond_applies = (int32_t)h->stat_precond;
    info->converged = all ? 1 : 0;
    info->guess_used = h->stat_guess_used ? 1 : 0;
    info->relres_inf = worst;
    info->first_inner_iters = h->stat_first_inner;
  }
  if (!all) {
    h->err = "outer BiCGStab did not reach tol_out within maxit_out (worst relative residual " +
             std::to_string(worst) + ")";
    return DDPS_ERR_NOT_CONVERGED;
  }
  return DDPS_OK;
}

ddps_status fail(ddps_handle* h, const Fail& e) {
  if (h) h->err = e.msg;
  g_last_error = e.msg;
  return e.st;
}

// Column order, active fronts and forward launch lists of the sparse
// forward sweep (see the handle's fields).  kf/km and rf/rm are the tile
// lists over the pivot rows and over the update rows of every front,
// tc_off the packed-A offsets per op (empty without tensor cores).
void build_sparse_forward(ddps_handle* h, const std::vector<int32_t>& kf,
                          const std::vector<int32_t>& km, const std::vector<int32_t>& rf,
                          const std::vector<int32_t>& rm,
                          const std::vector<std::vector<int64_t>>& tc_off,
                          const std::vector<uint8_t>& fused, const std::vector<uint8_t>& fusedb) {
  const Analysis& A = h->A;
  const int64_t nf = (int64_t)A.f_k.size();
  const int64_t n = A.n;
  std::vector<int32_t> owner(n, -1);
  for (int64_t f = 0; f < nf; ++f)
    for (int32_t i = 0; i < A.f_k[f]; ++i) owner[A.f_row0[f] + i] = (int32_t)f;
  // entries of each coupling column (global column slot gcol_ptr[b] + j): their fronts
  const int64_t ncol_all = A.gcol_ptr[A.p];
  std::vector<int32_t> key(ncol_all, INT32_MAX);
  std::vector<std::vector<int32_t>> col_fronts(ncol_all);
  std::vector<int32_t> row_block(n);
  for (int32_t b = 0; b < A.p; ++b)
    for (int64_t i = A.block_ptr[b]; i < A.block_ptr[b + 1]; ++i) row_block[i] = b;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t e = A.rt_rowptr[i]; e < A.rt_rowptr[i + 1]; ++e) {
      const int64_t slot = A.gcol_ptr[row_block[i]] + A.rt_rhscol[e];
      const int32_t f = owner[A.rt_rownew[e]];
      col_fronts[slot].push_back(f);
      key[slot] = std::min(key[slot], f);
    }
  // order each block's columns by the first front they touch
  std::vector<int32_t> gperm(ncol_all), inv(ncol_all);
  for (int32_t b = 0; b < A.p; ++b) {
    const int64_t c0 = A.gcol_ptr[b], nc = A.gcol_ptr[b + 1] - c0;
    std::vector<int32_t> ord(nc);
    for (int64_t j = 0; j < nc; ++j) ord[j] = (int32_t)j;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int32_t a, int32_t bb) { return key[c0 + a] < key[c0 + bb]; });
    for (int64_t pcol = 0; pcol < nc; ++pcol) {
      gperm[c0 + pcol] = ord[pcol];
      inv[c0 + ord[pcol]] = (int32_t)pcol;
    }
  }
  h->gperm = gperm;
  // G^ keeps its columns in panel order: the matvec gathers v through the permuted column list
  std::vector<int32_t> gcols_panel(ncol_all);
  for (int64_t t = 0; t < ncol_all; ++t) gcols_panel[t] = A.gcols[t];
  for (int32_t b = 0; b < A.p; ++b)
    for (int64_t pcol = A.gcol_ptr[b]; pcol < A.gcol_ptr[b + 1]; ++pcol)
      gcols_panel[pcol] = A.gcols[A.gcol_ptr[b] + gperm[pcol]];
  CK(cudaMemcpy(h->gcols, gcols_panel.data(), gcols_panel.size() * sizeof(int32_t),
                cudaMemcpyHostToDevice));
  std::vector<int32_t> rhscol(A.rt_rhscol.size());
  for (int64_t i = 0; i < n; ++i)
    for (int32_t e = A.rt_rowptr[i]; e < A.rt_rowptr[i + 1]; ++e)
      rhscol[e] = inv[A.gcol_ptr[row_block[i]] + A.rt_rhscol[e]];
  CK(cudaMemcpy(h->rt_rhscol, rhscol.data(), rhscol.size() * sizeof(int32_t),
                cudaMemcpyHostToDevice));
  // per chunk: active fronts, then per depth the gather list and the forward tiles
  const int64_t NR = std::max<int32_t>(h->NR, 1);
  const int64_t nchunks = A.max_rhs > 0 ? (A.max_rhs + NR - 1) / NR : 0;
  std::vector<uint8_t> active((size_t)std::max<int64_t>(nchunks, 1) * nf, 0);
  std::vector<uint8_t> pleaf((size_t)std::max<int64_t>(nchunks, 1) * nf, 0);
  std::vector<int32_t> g, kfo, kmo, rfo, rmo;
  std::vector<int64_t> kao, rao;
  h->fw_g_ptr.assign(1, 0);
  h->fw_k_ptr.assign(1, 0);
  h->fw_r_ptr.assign(1, 0);
  h->fz_ptr.assign(1, 0);
  h->zr_ptr.assign(1, 0);
  std::vector<int32_t> fz, zr;
  const bool tc = !tc_off.empty();
  for (int64_t c = 0; c < nchunks; ++c) {
    uint8_t* act = active.data() + c * nf;
    for (int32_t b = 0; b < A.p; ++b) {
      const int64_t c0 = A.gcol_ptr[b], nc = A.gcol_ptr[b + 1] - c0;
      for (int64_t pcol = c * NR; pcol < std::min<int64_t>((c + 1) * NR, nc); ++pcol)
        for (int32_t f : col_fronts[c0 + gperm[c0 + pcol]])
          for (int32_t a = f; a >= 0 && !act[a]; a = A.f_parent[a]) act[a] = 1;
    }
    uint8_t* pl = pleaf.data() + c * nf;
    if (tc) {
      for (int64_t f = 0; f < nf; ++f)
        if (act[f] || !fusedb[f]) zr.push_back((int32_t)f);
      h->zr_ptr.push_back((int64_t)zr.size());
    }
    if (tc)
      for (int64_t f = 0; f < nf; ++f) {
        if (!act[f] || !fused[f]) continue;
        bool child = false;
        for (int32_t ci = A.f_cbeg[f]; ci < A.f_cend[f] && !child; ++ci) child = act[A.children[ci]];
        pl[f] = !child;
      }
    for (int L = 0; L < A.nlevels; ++L) {
      for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q)
        if (act[A.level_fronts[q]] && !pl[A.level_fronts[q]]) g.push_back(A.level_fronts[q]);
      for (int32_t t = h->fk_ptr[L]; t < h->fk_ptr[L + 1]; ++t)
        if (act[kf[t]]) {
          kfo.push_back(kf[t]);
          kmo.push_back(km[t]);
          if (tc) kao.push_back(tc_off[OP_FWD_LINV][t]);
        }
      for (int32_t t = h->tr_ptr[L]; t < h->tr_ptr[L + 1]; ++t)
        if (act[rf[t]]) {
          rfo.push_back(rf[t]);
          rmo.push_back(rm[t]);
          if (tc) rao.push_back(tc_off[OP_FWD_L21][t]);
        }
      h->fw_g_ptr.push_back((int64_t)g.size());
      h->fw_k_ptr.push_back((int64_t)kfo.size());
      h->fw_r_ptr.push_back((int64_t)rfo.size());
      for (int cls = 0; cls < 4; ++cls) {
        for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
          const int32_t f = A.level_fronts[q];
          if (act[f] && fused[f] && tc_fused_class(A.f_m[f]) == cls) fz.push_back(f);
        }
        h->fz_ptr.push_back((int64_t)fz.size());
      }
    }
  }
  h->fw_active = dupload(h, active);
  if (tc) {
    h->fw_pleaf = dupload(h, pleaf);
    h->zr_front = dupload(h, zr);
  }
  h->fw_g = dupload(h, g);
  h->fw_kf = dupload(h, kfo);
  h->fw_km = dupload(h, kmo);
  h->fw_rf = dupload(h, rfo);
  h->fw_rm = dupload(h, rmo);
  h->fw_ka = tc ? dupload(h, kao) : nullptr;
  h->fw_ra = tc ? dupload(h, rao) : nullptr;
  h->fz = dupload(h, fz);
}

void build_device(ddps_handle* h, const int32_t* rowptr, const int32_t* colind) {
  Analysis& A = h->A;
  const int64_t n = A.n, m = (int64_t)A.c.size();
  h->rowptr = dupload(h, std::vector<int32_t>(rowptr, rowptr + n + 1));
  h->colind = dupload(h, std::vector<int32_t>(colind, colind + A.nnz));
  h->vals = dalloc<double>(h, A.nnz);
  h->amap = dupload(h, A.amap);
  h->perm = dupload(h, A.perm);
  h->iperm = dupload(h, A.iperm);
  DevFronts F{};
  F.k = dupload(h, A.f_k);
  F.m = dupload(h, A.f_m);
  F.block = dupload(h, A.f_block);
  F.row0 = dupload(h, A.f_row0);
  F.arena = dupload(h, A.f_arena);
  F.idx_off = dupload(h, A.f_idx);
  F.upd = dupload(h, A.f_upd);
  F.rel_off = dupload(h, A.f_rel);
  F.cbeg = dupload(h, A.f_cbeg);
  F.cend = dupload(h, A.f_cend);
  F.children = dupload(h, A.children);
  F.idx = dupload(h, A.idx);
  F.rel = dupload(h, A.rel);
  h->F = F;
  h->parent = dupload(h, A.f_parent);
  h->level_fronts = dupload(h, A.level_fronts);
  h->ea_list = dupload(h, A.ea_list);
  // largest update block per extend-add launch
  const int S = A.max_children;
  h->ea_maxr.assign((size_t)A.nlevels * S, 0);
  for (size_t q = 0; q + 1 < A.ea_ptr.size(); ++q)
    for (int32_t i = A.ea_ptr[q]; i < A.ea_ptr[q + 1]; ++i) {
      const int32_t c = A.ea_list[i];
      h->ea_maxr[q] = std::max(h->ea_maxr[q], A.f_m[c] - A.f_k[c]);
    }
  const size_t fs = prec_size(h->opt.factor_prec);
  h->arena = dalloc_bytes(h, A.arena_size * (int64_t)fs);
  h->updv = dalloc_bytes(h, std::max<int64_t>(A.upd_size, 1) * (int64_t)fs);
  h->w = dalloc_bytes(h, n * (int64_t)fs);
  h->rownorm = dalloc<double>(h, n);
  h->derr = dalloc<long long>(h, 3);
  if (A.ilu) {
    h->il.rp = dupload(h, A.il_rp);
    h->il.col = dupload(h, A.il_col);
    h->il.diag = dupload(h, A.il_diag);
    h->il.row_block = dupload(h, A.il_row_block);
    h->il_lf = dupload(h, A.il_lf);
    h->il_lb = dupload(h, A.il_lb);
    h->il_val = dalloc_bytes(h, std::max<int64_t>((int64_t)A.il_col.size(), 1) * (int64_t)fs);
  }
  CK(cudaMallocHost((void**)&h->herr, 3 * sizeof(long long)));
  // R~
  h->nrt = (int64_t)A.rt_col.size();
  h->rt_rowptr = dupload(h, A.rt_rowptr);
  h->rt_col = dupload(h, A.rt_col);
  h->rt_rhscol = dupload(h, A.rt_rhscol);
  h->rt_rownew = dupload(h, A.rt_rownew);
  h->rt_src = dupload(h, A.rt_src);
  h->rt_val = dalloc<double>(h, h->nrt);
  // reduced system
  h->c = dupload(h, A.c);
  h->c_rownew = dupload(h, A.c_rownew);
  std::vector<int32_t> qblock(m);
  std::vector<int64_t> ncols(A.p);
  for (int32_t b = 0; b < A.p; ++b) {
    for (int64_t q = A.gq0[b]; q < A.gq1[b]; ++q) qblock[q] = b;
    ncols[b] = A.gcol_ptr[b + 1] - A.gcol_ptr[b];
  }
  h->qblock = dupload(h, qblock);
  h->block_sys = dupload(h, A.block_sys);
  h->any_flag = dalloc<int32_t>(h, 1);
  CK(cudaMallocHost((void**)&h->any_host, sizeof(int32_t)));
  h->gq0 = dupload(h, A.gq0);
  h->gq1 = dupload(h, A.gq1);
  h->gcol_ptr = dupload(h, A.gcol_ptr);
  h->ghat_off = dupload(h, A.ghat_off);
  h->gld = dupload(h, A.gld);
  {
    // tiles of 64 rows; blocks of fewer than 1024 coupling columns take tiles
    // of 256 rows, so that a CTA's fixed cost (staging v) covers enough work
    std::vector<int32_t> tb, tr, th;
    for (int32_t b = 0; b < A.p; ++b) {
      const int64_t nc = A.gcol_ptr[b + 1] - A.gcol_ptr[b];
      h->mv_max_cols = std::max(h->mv_max_cols, nc);
      const int32_t hgt = nc >= 1024 ? 64 : 256;
      for (int64_t r = 0; r < A.gq1[b] - A.gq0[b]; r += hgt) {
        tb.push_back(b);
        tr.push_back((int32_t)r);
        th.push_back(hgt);
      }
    }
    h->mv_ntiles = (int32_t)tb.size();
    h->mv_block = dupload(h, tb);
    h->mv_row = dupload(h, tr);
    h->mv_h = dupload(h, th);
    // tiles are ordered by block and blocks by system: a system's tiles are
    // consecutive
    std::vector<int32_t> stp(A.nsys + 1, 0);
    for (int32_t b : tb) ++stp[A.block_sys[b] + 1];
    for (int32_t q = 0; q < A.nsys; ++q) stp[q + 1] += stp[q];
    h->mv_sys_tptr = dupload(h, stp);
    h->mv_done = dalloc<int32_t>(h, A.nsys);
    CK(cudaMemset(h->mv_done, 0, (size_t)std::max<int32_t>(A.nsys, 1) * sizeof(int32_t)));
    h->mv_partial = dalloc<double>(h, 2 * (int64_t)std::max<int32_t>(h->mv_ntiles, 1));
  }
  h->gcols = dupload(h, A.gcols);
  h->block_ncols = dupload(h, ncols);
  const bool implicit = h->opt.ghat_mode == DDPS_GHAT_IMPLICIT;
  if (!implicit) {
    const int64_t gbytes = std::max<int64_t>(A.ghat_off[A.p], 1) * (int64_t)prec_size(h->opt.ghat_prec);
    h->ghat = dalloc_bytes(h, gbytes);
    CK(cudaMemset(h->ghat, 0, gbytes));  // the row padding stays zero
  } else {
    h->im_q = dalloc<double>(h, n);
    h->im_g = dalloc<double>(h, n);
  }
  // spike panels: NR right-hand sides per pass (none when G^ is implicit)
  if (m > 0 && !implicit) {
    // NR: a multiple of 128 columns (the panel kernels move 128-column groups)
    int64_t nr = h->opt.rhs_chunk > 0 ? h->opt.rhs_chunk : 1024;
    nr = std::min<int64_t>(nr, (A.max_rhs + 127) / 128 * 128);
    nr = std::max<int64_t>(128, nr / 128 * 128);
    const int64_t budget = (int64_t)12 << 30;  // bytes for the two panels
    while (nr > 128 && (n + (int64_t)A.idx.size()) * nr * (int64_t)fs > budget) nr = (nr / 2 + 127) / 128 * 128;
    h->NR = (int32_t)nr;
    // row n stays zero: the fused backward products read it as the pivot rows
    // of the fronts the chunk leaves inactive
    h->X = dalloc_bytes(h, (n + 1) * h->NR * (int64_t)fs);
    CK(cudaMemset(h->X, 0, (size_t)(n + 1) * h->NR * fs));
    h->U = dalloc_bytes(h, std::max<int64_t>((int64_t)A.idx.size(), 1) * h->NR * (int64_t)fs);
  }
  for (int32_t kf : A.f_k) h->max_k = std::max(h->max_k, kf);
  {
    const int small = h->opt.factor_prec == DDPS_FP64 ? small_front_max<double>() : small_front_max<float>();
    std::vector<int32_t> order, pfronts, tfront, tij, ivf, ivc, cfront, cij, qfront, qword, qslot;
    int64_t max_step_fronts = 0;
    h->lu_tc = h->opt.update_prec == DDPS_BF16X3 && h->opt.factor_prec == DDPS_FP32;
    std::vector<int64_t> ioff(A.f_k.size(), 0);
    int64_t inv_total = 0;
    h->split.assign(A.nlevels, LevelSplit{});
    for (int L = 0; L < A.nlevels; ++L) {
      LevelSplit& ls = h->split[L];
      ls.first = (int32_t)order.size();
      for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
        const int32_t f = A.level_fronts[q];
        ls.max_m = std::max(ls.max_m, A.f_m[f]);
        if (A.f_m[f] <= small) {
          order.push_back(f);
          ls.nsmall++;
          ls.max_small_m = std::max(ls.max_small_m, A.f_m[f]);
        }
      }
      int32_t kmax = 0;
      for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
        const int32_t f = A.level_fronts[q];
        if (A.f_m[f] > small) {
          order.push_back(f);
          ls.nlarge++;
          kmax = std::max(kmax, A.f_k[f]);
        }
      }
      // multi-CTA inverse tiles and scratch of the large fronts
      ls.inv_first = (int32_t)ivf.size();
      for (int32_t i = ls.first + ls.nsmall; i < (int32_t)order.size(); ++i) {
        const int32_t f = order[i];
        ioff[f] = inv_total;
        inv_total += 2 * (int64_t)A.f_k[f] * A.f_k[f];
        for (int32_t cb = 0; cb * kInvBlock < A.f_k[f]; ++cb) {
          ivf.push_back(f);
          ivc.push_back(cb);
        }
      }
      ls.inv_ntiles = (int32_t)ivf.size() - ls.inv_first;
      // panel steps of the large fronts
      const int npanel = (kmax + kLuPanel - 1) / kLuPanel;
      ls.pf_ptr.assign(1, (int64_t)pfronts.size());
      ls.pt_ptr.assign(1, (int64_t)tfront.size());
      ls.pc_ptr.assign(1, (int64_t)cfront.size());
      ls.pq_ptr.assign(1, (int64_t)qfront.size());
      for (int pstep = 0; pstep < npanel; ++pstep) {
        const int32_t j0 = pstep * kLuPanel;
        for (int32_t i = ls.first + ls.nsmall; i < (int32_t)order.size(); ++i) {
          const int32_t f = order[i];
          if (A.f_k[f] <= j0) continue;
          const int32_t slot = (int32_t)(pfronts.size() - ls.pf_ptr.back());
          pfronts.push_back(f);
          max_step_fronts = std::max<int64_t>(max_step_fronts, slot + 1);
          const int32_t t0 = std::min(j0 + kLuPanel, A.f_k[f]);
          for (int32_t q = 0; q * 256 < A.f_m[f] - t0; ++q) {
            for (int32_t side = 0; side < 2; ++side) {
              qfront.push_back(f);
              qword.push_back(q | (side << 30));
              qslot.push_back(slot);
            }
          }
          const int32_t nt = (A.f_m[f] - t0 + kLuTile - 1) / kLuTile;
          // blocks of kLuTcBlock (256) pivots: inside a block the rank-32 updates stop at
          // the block's rows and columns; the block's last panel step hands the
          // rest of the front to one tensor-core update
          const int32_t jend = std::min((j0 & ~(kLuTcBlock - 1)) + kLuTcBlock, A.f_k[f]);
          if (h->lu_tc && t0 >= jend) {
            const int32_t nc = (A.f_m[f] - jend + kLuTcTile - 1) / kLuTcTile;
            for (int32_t ti = 0; ti < nc; ++ti)
              for (int32_t tj = 0; tj < nc; ++tj) {
                cfront.push_back(f);
                cij.push_back((ti << 16) | tj);
              }
            continue;
          }
          for (int32_t ti = 0; ti < nt; ++ti)
            for (int32_t tj = 0; tj < nt; ++tj) {
              if (h->lu_tc && t0 + ti * kLuTile >= jend && t0 + tj * kLuTile >= jend) continue;
              tfront.push_back(f);
              tij.push_back((ti << 16) | tj);
            }
        }
        ls.pf_ptr.push_back((int64_t)pfronts.size());
        ls.pt_ptr.push_back((int64_t)tfront.size());
        ls.pc_ptr.push_back((int64_t)cfront.size());
        ls.pq_ptr.push_back((int64_t)qfront.size());
      }
    }
    h->lu_order = dupload(h, order);
    h->inv_tile_front = dupload(h, ivf);
    h->inv_tile_cb = dupload(h, ivc);
    h->inv_off = dupload(h, ioff);
    h->inv = dalloc_bytes(h, std::max<int64_t>(inv_total, 1) * (int64_t)prec_size(h->opt.factor_prec));
    h->lu_panel_fronts = dupload(h, pfronts);
    h->lu_tile_front = dupload(h, tfront);
    h->lu_tile_ij = dupload(h, tij);
    h->lu_tc_front = dupload(h, cfront);
    h->lu_tc_ij = dupload(h, cij);
    h->lu_pc_front = dupload(h, qfront);
    h->lu_pc_word = dupload(h, qword);
    h->lu_pc_slot = dupload(h, qslot);
    h->lu_dinv = dalloc_bytes(h, std::max<int64_t>(max_step_fronts, 1) * 2 * 32 * 32 *
                                     (int64_t)prec_size(h->opt.factor_prec));
  }
  {
    const int BM = h->opt.factor_prec == DDPS_FP64 ? spike_tile_m<double>() : spike_tile_m<float>();
    const int sp = h->opt.spike_prec;
    const bool tcp = (sp == DDPS_BF16 || sp == DDPS_BF16X3) && m > 0 && !implicit;
    const int passes = sp == DDPS_BF16X3 ? 3 : 1;
    const int64_t nfr = (int64_t)A.f_k.size();
    // fronts whose output rows fit one CTA take the fused products
    std::vector<uint8_t> fzb(nfr, 0), fzf(nfr, 0);
    const int fmax = h->opt.fused_rows < 0    ? 0
                     : h->opt.fused_rows == 0 ? tc_fused_max_rows()
                                              : std::min(h->opt.fused_rows, tc_fused_max_rows());
    if (tcp)
      for (int64_t f = 0; f < nfr; ++f) {
        fzb[f] = A.f_k[f] > 0 && A.f_k[f] <= fmax;
        fzf[f] = A.f_k[f] > 0 && A.f_m[f] <= fmax;
      }
    std::vector<int32_t> bkf, bkm, fkf, fkm, rf, rm, bz;
    h->tk_ptr.assign(1, 0);
    h->fk_ptr.assign(1, 0);
    h->tr_ptr.assign(1, 0);
    h->bz_ptr.assign(1, 0);
    for (int L = 0; L < A.nlevels; ++L) {
      for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
        const int32_t f = A.level_fronts[q];
        const int32_t kk = A.f_k[f], rr = A.f_m[f] - A.f_k[f];
        for (int32_t m0 = 0; m0 < kk; m0 += BM) {
          if (!fzb[f]) {
            bkf.push_back(f);
            bkm.push_back(m0);
          }
          if (!fzf[f]) {
            fkf.push_back(f);
            fkm.push_back(m0);
          }
        }
        if (!fzf[f])
          for (int32_t m0 = 0; m0 < rr; m0 += BM) {
            rf.push_back(f);
            rm.push_back(m0);
          }
      }
      h->tk_ptr.push_back((int32_t)bkf.size());
      h->fk_ptr.push_back((int32_t)fkf.size());
      h->tr_ptr.push_back((int32_t)rf.size());
      for (int cls = 0; cls < 4; ++cls) {
        for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
          const int32_t f = A.level_fronts[q];
          if (fzb[f] && tc_fused_class(A.f_k[f]) == cls) bz.push_back(f);
        }
        h->bz_ptr.push_back((int64_t)bz.size());
      }
    }
    h->tk_front = dupload(h, bkf);
    h->tk_m0 = dupload(h, bkm);
    h->fk_front = dupload(h, fkf);
    h->fk_m0 = dupload(h, fkm);
    h->tr_front = dupload(h, rf);
    h->tr_m0 = dupload(h, rm);
    h->bz = dupload(h, bz);
    std::vector<std::vector<int64_t>> tc_off_host(tcp ? 4 : 0);
    if (tcp) {
      h->tc_passes = passes;
      const int BK = tc_tile_bk();
      const int64_t bb = tc_a_block_bytes(h->tc_passes);
      int64_t run = 0;
      for (int op = 0; op < 4; ++op) {
        const std::vector<int32_t>& tf = op == OP_FWD_L21 ? rf : op == OP_FWD_LINV ? fkf : bkf;
        std::vector<int64_t> off(tf.size());
        for (size_t t = 0; t < tf.size(); ++t) {
          const int32_t kk = A.f_k[tf[t]], rr = A.f_m[tf[t]] - kk;
          const int32_t K = op == OP_BWD_U12 ? rr : kk;
          const int32_t nk = (K + BK - 1) / BK;
          off[t] = run;
          run += nk * bb;
          h->tc_max_kt[op] = std::max(h->tc_max_kt[op], nk);
        }
        h->tc_aoff[op] = dupload(h, off);
        tc_off_host[op] = off;
      }
      h->atc = (unsigned char*)dalloc_bytes(h, std::max<int64_t>(run, 16));
      // packed W of the fused fronts
      std::vector<int64_t> wob(nfr, -1), wof(nfr, -1);
      std::vector<int32_t> pf;  // fused forward fronts
      std::vector<int32_t> wf[2][3], wk[2][3];
      int32_t wmax[2][3] = {};
      int64_t wrun = 0;
      auto wclass = [](int32_t kk) { return kk <= 64 ? 0 : kk <= 160 ? 1 : 2; };
      for (int64_t f = 0; f < nfr; ++f) {
        const int32_t kk = A.f_k[f], mm = A.f_m[f];
        const int wc = wclass(kk);
        if (fzb[f]) {
          wob[f] = wrun;
          wrun += tc_fused_w_bytes(passes, kk, mm);
          for (int32_t kb = 0; kb < (mm + BK - 1) / BK; ++kb) {
            wf[1][wc].push_back((int32_t)f);
            wk[1][wc].push_back(kb);
          }
          wmax[1][wc] = std::max(wmax[1][wc], kk);
        }
        if (fzf[f]) {
          wof[f] = wrun;
          wrun += tc_fused_w_bytes(passes, mm, kk);
          pf.push_back((int32_t)f);
          for (int32_t kb = 0; kb < (kk + BK - 1) / BK; ++kb) {
            wf[0][wc].push_back((int32_t)f);
            wk[0][wc].push_back(kb);
          }
          wmax[0][wc] = std::max(wmax[0][wc], kk);
        }
      }
      h->wpk = (unsigned char*)dalloc_bytes(h, std::max<int64_t>(wrun, 16));
      if (!pf.empty()) {  // fused forward fronts: their update rows go to D
        const size_t db = (size_t)std::max<int64_t>((int64_t)A.idx.size(), 1) * h->NR * sizeof(float);
        h->D = dalloc_bytes(h, (int64_t)db);
        CK(cudaMemset(h->D, 0, db));  // columns past a block's count stay zero
        h->fz_flag = dupload(h, fzf);
      }
      h->woff_b = dupload(h, wob);
      h->woff_f = dupload(h, wof);
      for (int dir = 0; dir < 2; ++dir)
        for (int wc = 0; wc < 3; ++wc) {
          ddps_handle::WpkList& wl = h->wpk_items[dir][wc];
          wl.n = (int32_t)wf[dir][wc].size();
          wl.max_k = wmax[dir][wc];
          if (wl.n) {
            wl.front = dupload(h, wf[dir][wc]);
            wl.kb = dupload(h, wk[dir][wc]);
          }
        }
    }
    if (!A.ilu) {
      build_sparse_forward(h, fkf, fkm, rf, rm, tc_off_host, fzf, fzb);
    } else {
      // ILU(0): G^ keeps the coupling columns in ascending order
      h->gperm.resize(A.gcol_ptr[A.p]);
      for (int32_t b = 0; b < A.p; ++b)
        for (int64_t pc = A.gcol_ptr[b]; pc < A.gcol_ptr[b + 1]; ++pc)
          h->gperm[pc] = (int32_t)(pc - A.gcol_ptr[b]);
    }
  }
  // segments
  h->nseg = A.nsys;
  h->Sn = make_segview(h, A.sys_row_ptr);
  h->Sm = make_segview(h, A.sys_c_ptr);
  // workspaces
  double** outer[] = {&h->o_r, &h->o_rhat, &h->o_p, &h->o_v, &h->o_phat, &h->o_s,
                      &h->o_shat, &h->o_t, &h->o_xt, &h->o_tmp, &h->pc_g, &h->pc_t,
                      &h->io_f, &h->io_x};
  for (double** pp : outer) *pp = dalloc<double>(h, n);
  h->pc_ghat = dalloc<double>(h, m);
  h->pc_zhat = dalloc<double>(h, m);
  h->first_zhat = dalloc<double>(h, m);
  h->first_ghat = dalloc<double>(h, m);
  h->guess = dalloc<double>(h, m);
  const size_t is = prec_size(h->opt.inner_prec);
  void** inner[] = {&h->i_g, &h->i_z, &h->i_r, &h->i_rh, &h->i_p, &h->i_v, &h->i_s, &h->i_t};
  for (void** pp : inner) *pp = dalloc_bytes(h, std::max<int64_t>(m, 1) * (int64_t)is);
  h->sc_out = dalloc<KScal>(h, h->nseg);
  h->sc_in = dalloc<KScal>(h, h->nseg);
  CK(cudaMallocHost((void**)&h->hsc_out, sizeof(KScal) * h->nseg));
  CK(cudaMallocHost((void**)&h->hsc_in, sizeof(KScal) * h->nseg));
  CK(cudaMallocHost((void**)&h->hstage, sizeof(KScal) * h->nseg * kStageSlots));
  h->hsc = h->hsc_out;
  h->partial = dalloc<double>(h, 3 * (int64_t)std::max(h->Sn.nchunks, h->Sm.nchunks) + 3);
  {
    // persistent sweeps: the deepest run of levels whose fronts all have at
    // most kPersistM rows, if it spans two levels or more
    int Lc = A.nlevels;
    while (Lc > 0 && h->split[Lc - 1].max_m <= kPersistM) --Lc;
    if (A.nlevels - Lc >= 2 && h->opt.persistent_solve != 0) {
      const int64_t nf = (int64_t)A.f_k.size();
      std::vector<int32_t> fwd, bwd, wait(nf, -1), level(nf, 0);
      for (int L = 0; L < A.nlevels; ++L)
        for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) level[A.level_fronts[q]] = L;
      for (int L = A.nlevels - 1; L >= Lc; --L)
        for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
          fwd.push_back(A.level_fronts[q]);
          h->persist_max_m = std::max(h->persist_max_m, A.f_m[A.level_fronts[q]]);
        }
      for (int L = Lc; L < A.nlevels; ++L)
        for (int32_t q = A.level_ptr[L]; q < A.level_ptr[L + 1]; ++q) {
          const int32_t f = A.level_fronts[q];
          bwd.push_back(f);
          if (L > Lc) wait[f] = A.f_parent[f];
        }
      h->persist_L = Lc;
      h->persist_n = (int32_t)fwd.size();
      h->p_fwd = dupload(h, fwd);
      h->p_bwd = dupload(h, bwd);
      h->p_wait = dupload(h, wait);
      h->p_flags = dalloc<int32_t>(h, 2 * nf + 2);
    }
  }
  if (h->opt.reduced_solver == DDPS_REDUCED_DIRECT && m > 0) {
    std::vector<int32_t> gcols_panel(A.gcols.size());
    for (int32_t b = 0; b < A.p; ++b)
      for (int64_t pc = A.gcol_ptr[b]; pc < A.gcol_ptr[b + 1]; ++pc)
        gcols_panel[pc] = A.gcols[A.gcol_ptr[b] + h->gperm[pc]];
    DirectInput in;
    in.p = A.p;
    in.m = m;
    in.gq0 = A.gq0.data();
    in.gq1 = A.gq1.data();
    in.gcol_ptr = A.gcol_ptr.data();
    in.gcols_panel = gcols_panel.data();
    in.ghat_off = A.ghat_off.data();
    in.gld = A.gld.data();
    in.block_sys = A.block_sys.data();
    auto alloc = [h](int64_t bytes) { return dalloc_bytes(h, bytes); };
    const std::string e = plan_direct(in, h->direct, alloc);
    if (!e.empty()) throw Fail{DDPS_ERR_INVALID_ARG, "ddps_analyze: " + e};
    upload_direct(h->direct, alloc);
    h->use_direct = true;
  }
}

bool valid_options(const ddps_options& o, std::string& why) {
  if (o.factor_prec != DDPS_FP64 && o.factor_prec != DDPS_FP32) {
    why = "factor_prec must be FP64 or FP32";
    return false;
  }
  if (o.ghat_prec != DDPS_FP64 && o.ghat_prec != DDPS_FP32 && o.ghat_prec != DDPS_BF16 &&
      o.ghat_prec != DDPS_FP16) {
    why = "ghat_prec must be FP64, FP32, FP16 or BF16";
    return false;
  }
  if (o.inner_prec != DDPS_FP64 && o.inner_prec != DDPS_FP32) {
    why = "inner_prec must be FP64 or FP32";
    return false;
  }
  if (o.factor_kind != DDPS_FACTOR_LU && o.factor_kind != DDPS_FACTOR_ILU0) {
    why = "factor_kind must be LU or ILU0";
    return false;
  }
  if (o.csr_kernel < -1 || o.csr_kernel > SPMV_WARP) {
    why = "csr_kernel must be -1 (tuned) or 0-4";
    return false;
  }
  if (o.factor_kind == DDPS_FACTOR_ILU0 && o.spike_prec != o.factor_prec) {
    why = "ILU0 block factors take spike_prec equal to factor_prec (SIMT spike solves)";
    return false;
  }
  if (o.reduced_solver != DDPS_REDUCED_ITERATIVE && o.reduced_solver != DDPS_REDUCED_DIRECT) {
    why = "reduced_solver must be ITERATIVE or DIRECT";
    return false;
  }
  if (o.reduced_solver == DDPS_REDUCED_DIRECT && o.ghat_mode != DDPS_GHAT_EXPLICIT) {
    why = "reduced_solver DIRECT needs the stored G^ (ghat_mode EXPLICIT)";
    return false;
  }
  if (o.ghat_prec == DDPS_FP64 && o.inner_prec != DDPS_FP64) {
    why = "an FP64 G^ needs FP64 inner vectors";
    return false;
  }
  const bool tc = o.spike_prec == DDPS_BF16 || o.spike_prec == DDPS_BF16X3;
  if (tc && o.factor_prec != DDPS_FP32) {
    why = "bf16 spike products need FP32 factors";
    return false;
  }
  if (!tc && o.spike_prec != o.factor_prec) {
    why = "spike_prec must equal factor_prec, or be BF16 / BF16X3 with FP32 factors";
    return false;
  }
  if (o.factor_prec == DDPS_FP32 && o.ghat_prec == DDPS_FP64) {
    why = "an FP64 G^ cannot be formed from FP32 factors";
    return false;
  }
  if (!(o.tol_out > 0) || !(o.tol_in > 0) || o.maxit_out < 1 || o.maxit_in < 1 || o.pivot_tol < 0) {
    why = "tolerances must be positive and iteration caps at least 1";
    return false;
  }
  if (o.update_prec != DDPS_FP64 && o.update_prec != DDPS_FP32 && o.update_prec != DDPS_BF16X3) {
    why = "update_prec must be FP64, FP32 or BF16X3";
    return false;
  }
  if (o.update_prec == DDPS_BF16X3 && o.factor_prec != DDPS_FP32) {
    why = "update_prec BF16X3 needs factor_prec FP32";
    return false;
  }
  if (o.ghat_mode != DDPS_GHAT_EXPLICIT && o.ghat_mode != DDPS_GHAT_IMPLICIT) {
    why = "ghat_mode must be EXPLICIT or IMPLICIT";
    return false;
  }
  if (o.fused_rows < -1) {
    why = "fused_rows must be -1, 0 or positive";
    return false;
  }
  return true;
}

}  // namespace

// ===========================================================================
// ABI
// ===========================================================================
extern "C" {

void ddps_default_options(ddps_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->drop_mode = DDPS_DROP_NONE;
  o->drop_tol = 0.0;
  o->factor_prec = DDPS_FP64;
  o->spike_prec = DDPS_FP64;
  o->ghat_prec = DDPS_FP64;
  o->inner_prec = DDPS_FP64;
  o->tol_out = 1e-10;
  o->maxit_out = 1000;
  o->tol_in = 1e-4;
  o->maxit_in = 100;
  o->pivot_tol = 1e-14;
  o->leaf_size = 0;
  o->rhs_chunk = 0;
  o->verbose = 0;
  o->use_graphs = 1;
  o->persistent_solve = 1;
  o->autotune = 1;
  o->csr_kernel = -1;
}

ddps_status ddps_analyze(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                         int32_t p, const int64_t* block_ptr, int32_t nsys,
                         const int32_t* sys_block_ptr, const double* values,
                         const ddps_options* opt, ddps_handle** out) {
  if (!out) {
    g_last_error = "ddps_analyze: out is NULL";
    return DDPS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  NvtxRange nv("ddps_analyze");
  ddps_handle* h = new (std::nothrow) ddps_handle();
  if (!h) {
    g_last_error = "ddps_analyze: host allocation failed";
    return DDPS_ERR_OUT_OF_MEMORY;
  }
  try {
    if (opt)
      h->opt = *opt;
    else
      ddps_default_options(&h->opt);
    std::string why;
    if (!valid_options(h->opt, why)) throw Fail{DDPS_ERR_INVALID_ARG, "ddps_analyze: " + why};
    std::string e = analyze(n, nnz, rowptr, colind, p, block_ptr, nsys, sys_block_ptr, values,
                            h->opt, h->A);
    if (!e.empty()) throw Fail{DDPS_ERR_INVALID_ARG, e};
    build_device(h, rowptr, colind);
    CK(cudaDeviceSynchronize());
  } catch (const Fail& f) {
    ddps_status st = fail(h, f);
    ddps_destroy(h);
    return st;
  } catch (const std::exception& ex) {
    g_last_error = std::string("ddps_analyze: ") + ex.what();
    ddps_destroy(h);
    return DDPS_ERR_INVALID_ARG;
  }
  *out = h;
  return DDPS_OK;
}

static ddps_status factor_values(ddps_handle* h, const double* values, bool host, void* stream) {
  if (!h || !values) return DDPS_ERR_INVALID_ARG;
  NvtxRange nv(host ? "ddps_factor_host" : "ddps_factor");
  cudaStream_t s = as_stream(stream);
  try {
    h->factored = false;
    CK(cudaMemcpyAsync(h->vals, values, h->A.nnz * sizeof(double),
                       host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    const int fp = h->opt.factor_prec, gp = h->opt.ghat_prec;
    if (fp == DDPS_FP64) {
      if (gp == DDPS_FP64)
        factor_impl<double, double>(h, s);
      else if (gp == DDPS_FP32)
        factor_impl<double, float>(h, s);
      else if (gp == DDPS_FP16)
        factor_impl<double, __half>(h, s);
      else
        factor_impl<double, __nv_bfloat16>(h, s);
    } else {
      if (gp == DDPS_FP32)
        factor_impl<float, float>(h, s);
      else if (gp == DDPS_FP16)
        factor_impl<float, __half>(h, s);
      else
        factor_impl<float, __nv_bfloat16>(h, s);
    }
    if (h->opt.autotune && !h->tuned) {
      if (fp == DDPS_FP64)
        autotune_block_solve<double>(h, s);
      else
        autotune_block_solve<float>(h, s);
    }
    if (h->opt.csr_kernel >= 0) h->tune_spmv = h->tune_rt = h->opt.csr_kernel;
    h->factored = true;
  } catch (const Fail& f) {
    return fail(h, f);
  }
  return DDPS_OK;
}

ddps_status ddps_factor(ddps_handle* h, const double* values, void* stream) {
  return factor_values(h, values, false, stream);
}

ddps_status ddps_factor_host(ddps_handle* h, const double* values_host, void* stream) {
  return factor_values(h, values_host, true, stream);
}

// Folds the statistics of one right-hand side into those of the call.
static void merge_info(ddps_solve_info* acc, const ddps_solve_info& one, bool first) {
  if (first) {
    *acc = one;
    return;
  }
  acc->outer_iterations = std::max(acc->outer_iterations, one.outer_iterations);
  acc->inner_iterations += one.inner_iterations;
  acc->precond_applies += one.precond_applies;
  acc->converged = acc->converged && one.converged;
  acc->guess_used = acc->guess_used || one.guess_used;
  acc->relres_inf = std::max(acc->relres_inf, one.relres_inf);
}

ddps_status ddps_solve(ddps_handle* h, const double* f, double* x, int32_t nrhs, const double* x0,
                       void* stream, ddps_solve_info* info) {
  if (!h || !f || !x || nrhs < 1) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) {
    h->err = "ddps_solve: call ddps_factor first";
    return DDPS_ERR_STATE;
  }
  NvtxRange nv("ddps_solve");
  auto t0 = std::chrono::steady_clock::now();
  try {
    const int64_t n = h->A.n;
    ddps_status worst = DDPS_OK;
    ddps_solve_info acc{}, one{};
    for (int32_t j = 0; j < nrhs; ++j) {
      ddps_status st = solve_impl(h, f + j * n, x + j * n, x0 ? x0 + j * n : nullptr,
                                  as_stream(stream), &one);
      merge_info(&acc, one, j == 0);
      if (st != DDPS_OK) worst = st;
    }
    if (info) {
      *info = acc;
      info->ms_solve =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return worst;
  } catch (const Fail& e) {
    return fail(h, e);
  }
}

ddps_status ddps_solve_host(ddps_handle* h, const double* f_host, double* x_host, int32_t nrhs,
                            const double* x0_host, void* stream, ddps_solve_info* info) {
  if (!h || !f_host || !x_host || nrhs < 1) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) {
    h->err = "ddps_solve_host: call ddps_factor first";
    return DDPS_ERR_STATE;
  }
  NvtxRange nv("ddps_solve_host");
  cudaStream_t s = as_stream(stream);
  auto t0 = std::chrono::steady_clock::now();
  try {
    const int64_t n = h->A.n;
    const size_t bytes = n * sizeof(double);
    ddps_status worst = DDPS_OK;
    ddps_solve_info acc{}, one{};
    for (int32_t j = 0; j < nrhs; ++j) {
      CK(cudaMemcpyAsync(h->io_f, f_host + j * n, bytes, cudaMemcpyHostToDevice, s));
      if (x0_host) CK(cudaMemcpyAsync(h->io_x, x0_host + j * n, bytes, cudaMemcpyHostToDevice, s));
      ddps_status st = solve_impl(h, h->io_f, h->io_x, x0_host ? h->io_x : nullptr, s, &one);
      CK(cudaMemcpyAsync(x_host + j * n, h->io_x, bytes, cudaMemcpyDeviceToHost, s));
      merge_info(&acc, one, j == 0);
      if (st != DDPS_OK) worst = st;
    }
    CK(cudaStreamSynchronize(s));
    if (info) {
      *info = acc;
      info->ms_solve =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (worst == DDPS_ERR_NOT_CONVERGED)
      h->err = "outer BiCGStab did not reach tol_out within maxit_out for some right-hand side";
    return worst;
  } catch (const Fail& e) {
    return fail(h, e);
  }
}

ddps_status ddps_set_reduced_guess(ddps_handle* h, const double* zhat0, void* stream) {
  if (!h) return DDPS_ERR_INVALID_ARG;
  try {
    if (!zhat0) {
      h->has_guess = false;
      return DDPS_OK;
    }
    const int64_t m = (int64_t)h->A.c.size();
    if (m > 0)
      CK(cudaMemcpyAsync(h->guess, zhat0, m * sizeof(double), cudaMemcpyDeviceToDevice,
                         as_stream(stream)));
    h->has_guess = m > 0;
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_get_reduced_solution(ddps_handle* h, double* zhat, double* ghat, void* stream) {
  if (!h) return DDPS_ERR_INVALID_ARG;
  try {
    const int64_t m = (int64_t)h->A.c.size();
    cudaStream_t s = as_stream(stream);
    if (zhat && m) CK(cudaMemcpyAsync(zhat, h->first_zhat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (ghat && m) CK(cudaMemcpyAsync(ghat, h->first_ghat, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_block_solve(ddps_handle* h, const double* y, double* g, void* stream) {
  if (!h || !y || !g) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    block_solve(h, y, g, as_stream(stream));
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_reduced_rhs(ddps_handle* h, const double* y, double* ghat, void* stream) {
  if (!h || !y || (!h->A.c.empty() && !ghat)) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    cudaStream_t s = as_stream(stream);
    block_solve(h, y, h->pc_g, s);
    const int64_t m = (int64_t)h->A.c.size();
    if (m) {
      launch_gather(h->pc_g, h->c, m, ghat, s);
      h->launches++;
    }
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_reduced_matvec(ddps_handle* h, const double* v, double* w, void* stream) {
  if (!h || (!h->A.c.empty() && (!v || !w))) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    cudaStream_t s = as_stream(stream);
    const int gp = h->opt.ghat_prec;
    if (h->A.c.empty()) return DDPS_OK;
    if (gp == DDPS_FP64)
      ghat_matvec<double, double>(h, v, w, s);
    else if (gp == DDPS_FP32)
      ghat_matvec<float, double>(h, v, w, s);
    else if (gp == DDPS_FP16)
      ghat_matvec<__half, double>(h, v, w, s);
    else
      ghat_matvec<__nv_bfloat16, double>(h, v, w, s);
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_reduced_solve(ddps_handle* h, const double* ghat, double* zhat, void* stream) {
  if (!h || (!h->A.c.empty() && (!ghat || !zhat))) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    cudaStream_t s = as_stream(stream);
    if (h->A.c.empty()) return DDPS_OK;
    if (h->use_direct) {
      Prof pr(h, DDPS_PROF_DIRECT_SOLVE, s);
      h->launches += direct_solve(h->direct, ghat, zhat, s);
    } else {
      h->stat_inner = 0;
      inner_dispatch(h, ghat, zhat, nullptr, s);
    }
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_precond_apply(ddps_handle* h, const double* y, double* z, void* stream) {
  if (!h || !y || !z) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    h->stat_inner = 0;
    precond_apply(h, y, z, as_stream(stream), false);
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_spmv(ddps_handle* h, const double* x, double* y, void* stream) {
  if (!h || !x || !y) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    launch_spmv(h->rowptr, h->colind, h->vals, h->A.n, x, y, as_stream(stream), h->tune_spmv);
    h->launches++;
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_get_sizes(const ddps_handle* h, ddps_sizes* s) {
  if (!h || !s) return DDPS_ERR_INVALID_ARG;
  const Analysis& A = h->A;
  s->n = A.n;
  s->nnz = A.nnz;
  s->nsys = A.nsys;
  s->nblocks = A.p;
  s->m = (int64_t)A.c.size();
  s->nnz_rt = (int64_t)A.rt_col.size();
  s->nfronts = (int64_t)A.f_k.size();
  s->nlevels = A.nlevels;
  s->factor_entries = A.arena_size;
  s->factor_lu_entries = A.factor_lu_entries;
  s->ghat_entries = A.ghat_entries;
  s->max_front = A.max_front;
  s->max_rhs = A.max_rhs;
  s->device_bytes = h->bytes;
  s->factor_flops = A.factor_flops;
  s->spike_flops = A.spike_flops;
  s->direct_flops = h->use_direct ? h->direct.factor_flops : 0.0;
  s->direct_bytes = h->use_direct ? h->direct.solve_bytes : 0;
  return DDPS_OK;
}

ddps_status ddps_get_tuning(const ddps_handle* h, char* buf, int64_t cap, int64_t* len) {
  if (!h) return DDPS_ERR_INVALID_ARG;
  static const char* names[] = {"warp", "cta8", "cl1", "cl2", "cl4", "cl8"};
  std::ostringstream o;
  static const char* csr[] = {"stream", "vec4", "vec8", "block", "warp"};
  o << "{\"tuned\": " << (h->tuned ? "true" : "false") << ", \"persistent_from_level\": "
    << h->persist_L << ", \"spmv\": \"" << csr[h->tune_spmv] << "\", \"spmv_ms\": "
    << h->tune_spmv_ms << ", \"rt_residual\": \"" << csr[h->tune_rt] << "\", \"levels\": [";
  for (size_t L = 0; L < h->tune_fwd.size(); ++L) {
    const int f = h->tune_fwd[L], b = h->tune_bwd[L];
    o << (L ? ", " : "") << "{\"level\": " << L
      << ", \"fronts\": " << (h->A.level_ptr[L + 1] - h->A.level_ptr[L])
      << ", \"max_m\": " << h->split[L].max_m << ", \"fwd\": \""
      << (f >= 0 ? names[f] : "auto") << "\", \"bwd\": \"" << (b >= 0 ? names[b] : "auto")
      << "\", \"fwd_ms\": " << h->tune_fwd_ms[L] << ", \"bwd_ms\": " << h->tune_bwd_ms[L] << "}";
  }
  o << "]}";
  const std::string t = o.str();
  if (len) *len = (int64_t)t.size();
  if (buf && cap > 0) {
    const size_t nc = std::min<size_t>((size_t)cap - 1, t.size());
    std::memcpy(buf, t.data(), nc);
    buf[nc] = 0;
  }
  return DDPS_OK;
}

ddps_status ddps_get_interface(const ddps_handle* h, int64_t* c) {
  if (!h || (!c && !h->A.c.empty())) return DDPS_ERR_INVALID_ARG;
  if (!h->A.c.empty()) std::memcpy(c, h->A.c.data(), h->A.c.size() * sizeof(int64_t));
  return DDPS_OK;
}

ddps_status ddps_get_ghat_layout(const ddps_handle* h, int32_t b, int64_t* q0, int64_t* q1,
                                 int64_t* ncols, int64_t* cols) {
  if (!h || b < 0 || b >= h->A.p) return DDPS_ERR_INVALID_ARG;
  const Analysis& A = h->A;
  if (q0) *q0 = A.gq0[b];
  if (q1) *q1 = A.gq1[b];
  const int64_t nc = A.gcol_ptr[b + 1] - A.gcol_ptr[b];
  if (ncols) *ncols = nc;
  if (cols)
    for (int64_t j = 0; j < nc; ++j) cols[j] = A.gcols[A.gcol_ptr[b] + j];
  return DDPS_OK;
}

ddps_status ddps_get_ghat_block(ddps_handle* h, int32_t b, double* dst, void* stream) {
  if (!h || b < 0 || b >= h->A.p || !dst) return DDPS_ERR_INVALID_ARG;
  if (!h->factored || h->opt.ghat_mode != DDPS_GHAT_EXPLICIT) return DDPS_ERR_STATE;
  try {
    const Analysis& A = h->A;
    const int64_t rows = A.gq1[b] - A.gq0[b];
    const int64_t nc = A.gcol_ptr[b + 1] - A.gcol_ptr[b];
    const int64_t ld = A.gld[b];
    if (rows * nc == 0) return DDPS_OK;
    cudaStream_t s = as_stream(stream);
    const int gp = h->opt.ghat_prec;
    const size_t es = prec_size(gp);
    std::vector<unsigned char> raw((size_t)rows * ld * es);
    CK(cudaMemcpyAsync(raw.data(), (const unsigned char*)h->ghat + A.ghat_off[b] * es, raw.size(),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < rows; ++i)
      for (int64_t j = 0; j < nc; ++j) {
        const unsigned char* e = raw.data() + ((size_t)i * ld + j) * es;
        double v;
        if (gp == DDPS_FP64) {
          std::memcpy(&v, e, 8);
        } else if (gp == DDPS_FP32) {
          float fv;
          std::memcpy(&fv, e, 4);
          v = fv;
        } else if (gp == DDPS_FP16) {
          __half hv;
          std::memcpy(&hv, e, 2);
          v = (double)__half2float(hv);
        } else {
          uint16_t hb;
          std::memcpy(&hb, e, 2);
          uint32_t bits = (uint32_t)hb << 16;
          float fv;
          std::memcpy(&fv, &bits, 4);
          v = fv;
        }
        dst[i * nc + h->gperm[A.gcol_ptr[b] + j]] = v;
      }
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}

ddps_status ddps_destroy(ddps_handle* h) {
  if (!h) return DDPS_OK;
  if (h->g_inner) cudaGraphExecDestroy(h->g_inner);
  if (h->g_factor) cudaGraphExecDestroy(h->g_factor);
  for (auto& q : h->g_prec) cudaGraphExecDestroy(q.exec);
  if (h->gstream) {
    cudaStreamSynchronize(h->gstream);
    cudaStreamDestroy(h->gstream);
  }
  for (cudaEvent_t e : h->gev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->herr) cudaFreeHost(h->herr);
  if (h->hsc_out) cudaFreeHost(h->hsc_out);
  if (h->hsc_in) cudaFreeHost(h->hsc_in);
  if (h->hstage) cudaFreeHost(h->hstage);
  if (h->any_host) cudaFreeHost(h->any_host);
  delete h;
  return DDPS_OK;
}

const char* ddps_last_error(const ddps_handle* h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

const char* ddps_status_string(ddps_status s) {
  switch (s) {
    case DDPS_OK: return "DDPS_OK";
    case DDPS_ERR_INVALID_ARG: return "DDPS_ERR_INVALID_ARG";
    case DDPS_ERR_SINGULAR_BLOCK: return "DDPS_ERR_SINGULAR_BLOCK";
    case DDPS_ERR_NOT_CONVERGED: return "DDPS_ERR_NOT_CONVERGED";
    case DDPS_ERR_OUT_OF_MEMORY: return "DDPS_ERR_OUT_OF_MEMORY";
    case DDPS_ERR_CUDA: return "DDPS_ERR_CUDA";
    case DDPS_ERR_TIMEOUT: return "DDPS_ERR_TIMEOUT";
    case DDPS_ERR_STATE: return "DDPS_ERR_STATE";
  }
  return "unknown status";
}

int64_t ddps_launch_count(const ddps_handle* h) { return h ? h->launches : 0; }

ddps_status ddps_set_profiling(ddps_handle* h, int32_t mask) {
  if (!h) return DDPS_ERR_INVALID_ARG;
  h->prof_mask = mask;
  return DDPS_OK;
}

ddps_status ddps_get_profile(ddps_handle* h, double* ms, int64_t* count, int32_t reset) {
  if (!h) return DDPS_ERR_INVALID_ARG;
  try {
    prof_collect(h);
  } catch (const Fail& e) {
    return fail(h, e);
  }
  for (int c = 0; c < DDPS_PROF_CLASSES; ++c) {
    if (ms) ms[c] = h->prof_ms[c];
    if (count) count[c] = h->prof_cnt[c];
    if (reset) {
      h->prof_ms[c] = 0;
      h->prof_cnt[c] = 0;
    }
  }
  return DDPS_OK;
}

ddps_status ddps_symbolic(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                          int32_t p, const int64_t* block_ptr, int32_t nsys,
                          const int32_t* sys_block_ptr, const double* values,
                          const ddps_options* opt, ddps_sizes* sizes, int32_t* perm, int64_t* c) {
  ddps_options o;
  if (opt)
    o = *opt;
  else
    ddps_default_options(&o);
  Analysis A;
  std::string e = analyze(n, nnz, rowptr, colind, p, block_ptr, nsys, sys_block_ptr, values, o, A);
  if (!e.empty()) {
    g_last_error = e;
    return DDPS_ERR_INVALID_ARG;
  }
  if (sizes) {
    std::memset(sizes, 0, sizeof(*sizes));
    sizes->n = A.n;
    sizes->nnz = A.nnz;
    sizes->nsys = A.nsys;
    sizes->nblocks = A.p;
    sizes->m = (int64_t)A.c.size();
    sizes->nnz_rt = (int64_t)A.rt_col.size();
    sizes->nfronts = (int64_t)A.f_k.size();
    sizes->nlevels = A.nlevels;
    sizes->factor_entries = A.arena_size;
    sizes->factor_lu_entries = A.factor_lu_entries;
    sizes->ghat_entries = A.ghat_entries;
    sizes->max_front = A.max_front;
    sizes->max_rhs = A.max_rhs;
    sizes->factor_flops = A.factor_flops;
    sizes->spike_flops = A.spike_flops;
  }
  if (perm) std::memcpy(perm, A.perm.data(), n * sizeof(int32_t));
  if (c && !A.c.empty()) std::memcpy(c, A.c.data(), A.c.size() * sizeof(int64_t));
  return DDPS_OK;
}

}  // extern "C"

// ===========================================================================
// Block solve without device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need a block solve:
// a host program whose memory pool already owns all free device memory, or
// one whose policy allows device allocations only at start-up.  For them,
// ddps_block_solve_noalloc takes its per-call scratch (the front vectors of
// the forward and backward sweeps) from the fixed array below instead of
// the handle's workspace.  The array is part of the library image: every GPU
// that loads the library holds it until the process exits.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
struct NoAllocAddr {
  unsigned long long ctx_id = 0;  // unique id of the context the address belongs to
  void* addr = nullptr;
};
NoAllocAddr g_noalloc_addr[256];

// Unique id of the calling thread's current context (cuCtxGetId through the
// runtime's driver entry point, so the library does not link libcuda);
// 0 when it cannot be read.  Ids are never reused in a process, so a device
// reset, which destroys the context and reloads the module in a new one,
// changes the id and the array's address is looked up again.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)fn;
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (GetId)fn;
    cudaGetLastError();
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_noalloc_scratch in the current device's context,
// looked up once per device and context.  (In host code the symbol's name
// only stands in for the array.)
void* noalloc_scratch_address() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) throw Fail{DDPS_ERR_CUDA, "device ordinal out of range"};
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoAllocAddr& e = g_noalloc_addr[dev];
  if (!e.addr || id == 0 || e.ctx_id != id) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    e.addr = p;
    e.ctx_id = id;
  }
  return e.addr;
}

template <typename T>
void block_solve_noalloc_impl(ddps_handle* h, const double* y, double* g, cudaStream_t s) {
  const Analysis& A = h->A;
  const size_t wbytes = ((size_t)A.n * sizeof(T) + 255) / 256 * 256;
  const size_t ubytes = (size_t)std::max<int64_t>(A.upd_size, 1) * sizeof(T);
  if (wbytes + ubytes > kNoAllocScratchBytes)
    throw Fail{DDPS_ERR_INVALID_ARG,
               "ddps_block_solve_noalloc: needs " + std::to_string(wbytes + ubytes) +
                   " bytes of scratch, more than the fixed " +
                   std::to_string(kNoAllocScratchBytes) + "-byte array"};
  unsigned char* base = (unsigned char*)noalloc_scratch_address();
  // Every entry of both scratch vectors is written before it is read (the
  // permutation fills w, each front writes its update vector before its
  // parent reads it), so nothing has to be cleared between calls.
  block_solve_impl<T>(h, y, g, s, DDPS_PROF_BLOCK_SOLVE, (T*)base, (T*)(base + wbytes));
}

}  // namespace

extern "C" ddps_status ddps_block_solve_noalloc(ddps_handle* h, const double* y, double* g,
                                                void* stream) {
  if (!h || !y || !g) return DDPS_ERR_INVALID_ARG;
  if (!h->factored) return DDPS_ERR_STATE;
  try {
    cudaStream_t s = as_stream(stream);
    if (h->opt.factor_prec == DDPS_FP64)
      block_solve_noalloc_impl<double>(h, y, g, s);
    else
      block_solve_noalloc_impl<float>(h, y, g, s);
    check_launch();
  } catch (const Fail& e) {
    return fail(h, e);
  }
  return DDPS_OK;
}
