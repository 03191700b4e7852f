// Segmented vector operations of the BiCGStab loops (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ddps {

// Chunked view of a vector split into segments (one segment per system).
// Chunks never cross a segment boundary.
struct SegView {
  const int64_t* chunk_beg;
  const int64_t* chunk_end;
  const int32_t* chunk_seg;
  const int32_t* seg_chunk_ptr;  // nseg+1 (every segment has at least one chunk)
  int32_t* done;                 // nseg counters of finished chunks (zero between reductions)
  int32_t nchunks;
  int32_t nseg;
};

// One reduction: op 0 = dot(x, y), 1 = 2-norm of x, 2 = inf-norm of x; the
// result for segment s goes to out[s].
struct RedSpec {
  const void* x;
  const void* y;
  int op;
  int stride;   // out is written at out[s * stride]
  double* out;
};

// BiCGStab scalars of one segment.
struct KScal {
  double rho, rho_old, alpha, omega, beta, sigma, ts, tt;
  double ref;         // reference norm of the stopping test
  double nrm;         // last residual norm
  double nrm2;        // second norm slot (true residual)
  double iters;       // iterations taken (half steps count 0.5), kept on the device
  int32_t active;     // still iterating
  int32_t half_done;  // converged at the half step of the current iteration
  int32_t breakdown;
  int32_t flag;       // scratch mask for masked updates
  int32_t it;         // iteration number on the device (loops that pass it < 0)
  int32_t pad;
};
static_assert(sizeof(KScal) % sizeof(double) == 0, "KScal must be a whole number of doubles");
constexpr int kScalStride = (int)(sizeof(KScal) / sizeof(double));

template <typename T>
void seg_reduce(const SegView& S, int nred, RedSpec r0, RedSpec r1, RedSpec r2, double* partial,
                cudaStream_t s);
template <typename T>
void update_p(const SegView& S, const KScal* sc, const T* r, T* p, const T* v, cudaStream_t s);
template <typename T>
void update_s(const SegView& S, const KScal* sc, const T* r, const T* v, T* out, cudaStream_t s);
template <typename T>
void update_xr(const SegView& S, const KScal* sc, int half, T* x, const T* phat, const T* shat,
               T* r, const T* sv, const T* t, cudaStream_t s);
template <typename T>
void vec_sub(const SegView& S, const KScal* sc, int all, const T* a, const T* b, T* dst,
             cudaStream_t s);
template <typename TD, typename TS>
void convert(int64_t n, const TS* src, TD* dst, cudaStream_t s);
// dst = a + alpha_s * b on segments whose flag is set (b may be null: dst = a)
template <typename T>
void masked_axpy(const SegView& S, const KScal* sc, T* dst, const T* a, const T* b, cudaStream_t s);
// dst = 0 on segments whose flag is set
template <typename T>
void masked_zero(const SegView& S, const KScal* sc, T* dst, cudaStream_t s);
// Reduction whose final pass also updates the segment's scalars.  `it` is
// the iteration number (1-based); it < 0 selects the segment's device
// counter instead (POST_BETA advances it; -it is the iteration cap: the
// full-step check stops a segment that has taken -it iterations), so that
// the same launches serve every iteration of a captured graph.
enum Post {
  POST_NONE = 0,
  POST_BETA = 1,        // beta = (rho / rho_old)(alpha / omega), 0 at iteration 1
  POST_ALPHA = 2,       // alpha = rho / sigma
  POST_CHECK_HALF = 3,  // ||s|| <= tol ref: stop at the half step (x += alpha p pending)
  POST_OMEGA = 4,       // omega = (t, s) / (t, t); rho_old = rho
  POST_CHECK_FULL = 5,  // ||r|| <= tol ref, omega = 0 or breakdown: stop; clears half_done
  POST_CHECK_FULL_BETA = 6  // the full-step check, then (still iterating) the next
                            // iteration's beta from the rho reduced with ||r||
};
#ifdef __CUDACC__
// The BiCGStab scalar step `post` of one segment, after its reductions.
__device__ __forceinline__ void post_step(KScal& k, int post, double tol, int it) {
  if (post == POST_CHECK_FULL || post == POST_CHECK_FULL_BETA) k.half_done = 0;
  if (!k.active) return;
  const int cap = it < 0 ? -it : 0;
  if (it < 0) {
    if (post == POST_BETA) k.it += 1;
    it = k.it;
  }
  switch (post) {
    case POST_BETA:
      if (k.rho == 0.0) k.breakdown = 1;
      k.beta = it == 1 ? 0.0 : (k.rho / k.rho_old) * (k.alpha / k.omega);
      break;
    case POST_ALPHA:
      if (k.sigma == 0.0) {
        k.breakdown = 1;
        k.alpha = 0.0;
      } else {
        k.alpha = k.rho / k.sigma;
      }
      break;
    case POST_CHECK_HALF:
      if (k.nrm <= tol * k.ref) {
        k.half_done = 1;
        k.active = 0;
        k.iters = it - 0.5;
      } else if (k.breakdown) {
        k.active = 0;
        k.iters = it;
      }
      break;
    case POST_OMEGA:
      k.omega = k.tt != 0.0 ? k.ts / k.tt : 0.0;
      k.rho_old = k.rho;
      break;
    case POST_CHECK_FULL:
    case POST_CHECK_FULL_BETA:
      k.iters = it;
      if (k.nrm <= tol * k.ref || k.omega == 0.0 || k.breakdown || (cap && it >= cap)) {
        k.active = 0;
      } else if (post == POST_CHECK_FULL_BETA) {
        // the next iteration (number it + 1 >= 2) starts here: POST_BETA's step
        if (cap) k.it += 1;
        if (k.rho == 0.0) k.breakdown = 1;
        k.beta = (k.rho / k.rho_old) * (k.alpha / k.omega);
      }
      break;
  }
}
#endif

// Reductions folded into the tiled G^ product (w = G^ v), per system: nred 1,
// sigma = (x, w); nred 2, ts = (w, v) and tt = (w, w); then the scalar step
// `post`.  Each tile writes its partial sums, the last tile of a system (in
// done[]) adds its tiles' partials in a fixed order and takes the step.
struct MvRed {
  int nred = 0;
  const void* x = nullptr;            // nred 1: the first vector (the product's type)
  double* partial = nullptr;          // 2 x tiles
  int32_t* done = nullptr;            // per system, zero between products
  const int32_t* sys_tptr = nullptr;  // tiles of system s: [sys_tptr[s], sys_tptr[s + 1])
  KScal* sc = nullptr;
  int post = 0;
  double tol = 0.0;
  int it = 0;
};

template <typename T>
void seg_reduce_post(const SegView& S, int nred, RedSpec r0, RedSpec r1, RedSpec r2,
                     double* partial, int post, KScal* sc, double tol, int it, cudaStream_t s);
// Full step: active segments x += alpha p + omega s, r = s - omega t; segments
// stopped at this iteration's half step: x += alpha p.
template <typename T>
void update_xr_final(const SegView& S, const KScal* sc, T* x, const T* p, const T* sv, T* r,
                     const T* t, cudaStream_t s);
// Fused forms of the inner loop: s = r - alpha v with ||s||_2 and the
// half-step check, and the full step of update_xr_final with ||r||_2 and the
// full-step check (each the values and summation order of the separate
// update and reduction).
template <typename T>
void update_s_norm(const SegView& S, KScal* sc, const T* r, const T* v, T* out, double* partial,
                   double tol, int it, cudaStream_t s);
template <typename T>
// rh (may be null): also rho = (rh, r) for the next iteration, with
// POST_CHECK_FULL_BETA instead of POST_CHECK_FULL.
void update_xr_norm(const SegView& S, KScal* sc, T* x, const T* p, const T* sv, T* r, const T* t,
                    const T* rh, double* partial, double tol, int it, cudaStream_t s);
// *flag = 1 if some segment is still active, else 0.
void any_active(int nseg, const KScal* sc, int32_t* flag, cudaStream_t s);
void sc_beta(int nseg, KScal* sc, int first, cudaStream_t s);
void sc_alpha(int nseg, KScal* sc, cudaStream_t s);
void sc_omega(int nseg, KScal* sc, cudaStream_t s);

}  // namespace ddps
