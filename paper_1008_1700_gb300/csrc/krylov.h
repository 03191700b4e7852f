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
