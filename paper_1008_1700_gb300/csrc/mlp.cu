// Learned initial guess for the reduced solve of Fig. 3 (6.3): a multilayer
// perceptron with ReLU hidden layers and a linear output, trained with Adam
// on reduced solutions that the solver itself produced.  The paper has no
// network; it solves 6.3 iteratively from a starting vector, which is what
// the network predicts.  Forward, backward and the optimiser step are plain
// FP32 CUDA kernels: a shared-memory tiled GEMM with fused epilogues.
#include <cuda_runtime.h>

#include <cstdint>

#include "ddps.h"

namespace {

constexpr int TM = 64, TN = 64, TK = 16, kThreads = 256;

// C(i,j) = sum_k A(i,k) B(k,j) with arbitrary element strides, then an
// epilogue:  mode 0: C = acc;  mode 1: C = acc + bias[j];  mode 2: C =
// relu(acc + bias[j]) and Zout = acc + bias[j];  mode 3: C = acc * (Zmask > 0).
struct GemmArgs {
  const float* A;
  int64_t sa0, sa1;
  const float* B;
  int64_t sb0, sb1;
  float* C;
  int64_t sc0, sc1;
  int M, N, K;
  int mode;
  const float* bias;
  float* Zout;
  const float* Zmask;
};

__global__ void __launch_bounds__(kThreads) k_gemm(GemmArgs g) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  const int tid = threadIdx.x;
  const int tr = tid % 16, tc = tid / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += TK) {
    for (int t = tid; t < TM * TK; t += kThreads) {
      const int ii = t % TM, kk = t / TM;
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < g.M && gk < g.K) ? g.A[gi * g.sa0 + gk * g.sa1] : 0.f;
      const int jj = t % TN, kk2 = t / TN;
      const int gj = j0 + jj, gk2 = k0 + kk2;
      Bs[kk2][jj] = (gj < g.N && gk2 < g.K) ? g.B[gk2 * g.sb0 + gj * g.sb1] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tr + 16 * u;
    if (i >= g.M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tc + 16 * v;
      if (j >= g.N) continue;
      float val = acc[u][v];
      const int64_t o = i * g.sc0 + j * g.sc1;
      if (g.mode == 1) {
        val += g.bias[j];
      } else if (g.mode == 2) {
        val += g.bias[j];
        g.Zout[o] = val;
        val = fmaxf(val, 0.f);
      } else if (g.mode == 3) {
        val = g.Zmask[o] > 0.f ? val : 0.f;
      }
      g.C[o] = val;
    }
  }
}

void gemm(const GemmArgs& g, cudaStream_t s) {
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM);
  k_gemm<<<grid, kThreads, 0, s>>>(g);
}

// dY = (Y - T) / B and per-CTA partial sums of (Y - T)^2
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, int64_t cnt,
                            float invB, float* __restrict__ dY, double* __restrict__ partial) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d * invB;
    acc += (double)d * d;
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const double* __restrict__ partial, int n, double scale,
                             float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *loss = (float)(s * scale);
  }
}

// db[j] = sum_b dZ[b, j]
__global__ void k_colsum(const float* __restrict__ dZ, int B, int N, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * N + j];
  db[j] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

constexpr int kLossBlocks = 256;

struct Layout {
  int L;  // number of affine layers = layers + 1
  int64_t woff[16], boff[16];
  int din[16], dout[16];
};

bool make_layout(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out, Layout& lay) {
  if (d_in <= 0 || hidden <= 0 || layers <= 0 || layers > 14 || d_out <= 0) return false;
  lay.L = layers + 1;
  int64_t off = 0;
  for (int l = 0; l < lay.L; ++l) {
    lay.din[l] = l == 0 ? d_in : hidden;
    lay.dout[l] = l == lay.L - 1 ? d_out : hidden;
    lay.woff[l] = off;
    off += (int64_t)lay.din[l] * lay.dout[l];
    lay.boff[l] = off;
    off += lay.dout[l];
  }
  return true;
}

// workspace: Z_l and A_l (B x hidden) for the hidden layers, Y (B x d_out),
// dY (B x d_out), two B x hidden gradient buffers, loss partial sums.
struct Work {
  float* Z[16];
  float* Aact[16];
  float* Y;
  float* dY;
  float* dA0;
  float* dA1;
  double* partial;
};

int64_t work_bytes(int32_t hidden, int32_t layers, int32_t d_out, int32_t B) {
  const int64_t hb = (int64_t)B * hidden;
  return 4 * (2 * layers * hb + 2 * (int64_t)B * d_out + 2 * hb) + 8 * kLossBlocks + 256;
}

Work carve(void* ws, int32_t hidden, int32_t layers, int32_t d_out, int32_t B) {
  Work w{};
  float* p = (float*)ws;
  const int64_t hb = (int64_t)B * hidden;
  for (int l = 0; l < layers; ++l) {
    w.Z[l] = p;
    p += hb;
    w.Aact[l] = p;
    p += hb;
  }
  w.Y = p;
  p += (int64_t)B * d_out;
  w.dY = p;
  p += (int64_t)B * d_out;
  w.dA0 = p;
  p += hb;
  w.dA1 = p;
  p += hb;
  uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  w.partial = (double*)a;
  return w;
}

void forward(const float* P, const Layout& lay, const float* X, int B, const Work& w, float* Y,
             cudaStream_t s) {
  const float* a = X;
  for (int l = 0; l < lay.L; ++l) {
    GemmArgs g{};
    g.A = a;
    g.sa0 = lay.din[l];
    g.sa1 = 1;
    g.B = P + lay.woff[l];  // W is [out x in] row-major; B(k, j) = W[j, k]
    g.sb0 = 1;
    g.sb1 = lay.din[l];
    g.M = B;
    g.N = lay.dout[l];
    g.K = lay.din[l];
    g.bias = P + lay.boff[l];
    g.sc0 = lay.dout[l];
    g.sc1 = 1;
    if (l < lay.L - 1) {
      g.C = w.Aact[l];
      g.Zout = w.Z[l];
      g.mode = 2;
      a = w.Aact[l];
    } else {
      g.C = Y;
      g.mode = 1;
    }
    gemm(g, s);
  }
}

}  // namespace

extern "C" {

int64_t ddps_mlp_param_count(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out) {
  Layout lay;
  if (!make_layout(d_in, hidden, layers, d_out, lay)) return -1;
  return lay.boff[lay.L - 1] + lay.dout[lay.L - 1];
}

int64_t ddps_mlp_workspace_bytes(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out,
                                 int32_t B) {
  Layout lay;
  if (!make_layout(d_in, hidden, layers, d_out, lay) || B <= 0) return -1;
  return work_bytes(hidden, layers, d_out, B);
}

ddps_status ddps_mlp_forward(const float* params, int32_t d_in, int32_t hidden, int32_t layers,
                             int32_t d_out, const float* X, int32_t B, float* Y, void* workspace,
                             void* stream) {
  Layout lay;
  if (!params || !X || !Y || !workspace || B <= 0 || !make_layout(d_in, hidden, layers, d_out, lay))
    return DDPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(workspace, hidden, layers, d_out, B);
  forward(params, lay, X, B, w, Y, s);
  return cudaGetLastError() == cudaSuccess ? DDPS_OK : DDPS_ERR_CUDA;
}

ddps_status ddps_mlp_backward(const float* params, int32_t d_in, int32_t hidden, int32_t layers,
                              int32_t d_out, const float* X, const float* T, int32_t B,
                              float* grads, float* loss, void* workspace, void* stream) {
  Layout lay;
  if (!params || !X || !T || !grads || !loss || !workspace || B <= 0 ||
      !make_layout(d_in, hidden, layers, d_out, lay))
    return DDPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Work w = carve(workspace, hidden, layers, d_out, B);
  forward(params, lay, X, B, w, w.Y, s);
  const int64_t cnt = (int64_t)B * d_out;
  k_loss_grad<<<kLossBlocks, kThreads, 0, s>>>(w.Y, T, cnt, 1.f / B, w.dY, w.partial);
  k_loss_final<<<1, 32, 0, s>>>(w.partial, kLossBlocks, 0.5 / B, loss);
  const float* d = w.dY;  // gradient w.r.t. the pre-activation of layer l
  for (int l = lay.L - 1; l >= 0; --l) {
    const float* ain = l == 0 ? X : w.Aact[l - 1];
    // dW_l[o, i] = sum_b d[b, o] ain[b, i]
    GemmArgs g{};
    g.A = d;
    g.sa0 = 1;
    g.sa1 = lay.dout[l];
    g.B = ain;
    g.sb0 = lay.din[l];
    g.sb1 = 1;
    g.C = grads + lay.woff[l];
    g.sc0 = lay.din[l];
    g.sc1 = 1;
    g.M = lay.dout[l];
    g.N = lay.din[l];
    g.K = B;
    g.mode = 0;
    gemm(g, s);
    k_colsum<<<(lay.dout[l] + 255) / 256, 256, 0, s>>>(d, B, lay.dout[l], grads + lay.boff[l]);
    if (l > 0) {
      // dA_{l-1} = d W_l, masked by relu'(Z_{l-1})
      float* dst = (d == w.dA0) ? w.dA1 : w.dA0;
      GemmArgs h{};
      h.A = d;
      h.sa0 = lay.dout[l];
      h.sa1 = 1;
      h.B = params + lay.woff[l];
      h.sb0 = lay.din[l];
      h.sb1 = 1;
      h.C = dst;
      h.sc0 = lay.din[l];
      h.sc1 = 1;
      h.M = B;
      h.N = lay.din[l];
      h.K = lay.dout[l];
      h.mode = 3;
      h.Zmask = w.Z[l - 1];
      gemm(h, s);
      d = dst;
    }
  }
  return cudaGetLastError() == cudaSuccess ? DDPS_OK : DDPS_ERR_CUDA;
}

ddps_status ddps_mlp_adam(float* params, const float* grads, float* m, float* v, int64_t count,
                          float lr, float beta1, float beta2, float eps, int32_t step,
                          void* stream) {
  if (!params || !grads || !m || !v || count <= 0 || step < 1) return DDPS_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, (float)step);
  const float c2 = 1.f - powf(beta2, (float)step);
  int64_t g = (count + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  k_adam<<<(int)g, kThreads, 0, (cudaStream_t)stream>>>(params, grads, m, v, count, lr, beta1,
                                                        beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? DDPS_OK : DDPS_ERR_CUDA;
}

}  // extern "C"
