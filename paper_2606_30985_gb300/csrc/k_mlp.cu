// Learned BP warm start: feature rows, a 3-layer MLP (forward, backward,
// Adam) and the message writer.  The paper has no learned part; in this
// extension of the method, per directed bond e and Schmidt
// index k the MLP predicts y = log diag(M_e)[k] of the converged double-layer
// message (Eq. 13 fixed point) in the bond's Schmidt basis, and damped BP then
// starts from M_e = diag(exp(y)) / sum exp(y).
//
// Precision: weights and activations are rounded to BF16 (round to nearest
// even) at the layer inputs, every product is accumulated in FP32, gradients
// and the Adam state are FP32 on an FP32 master copy of the weights.
// GEMMs are small (width 256, K <= 256 except the weight gradients, whose K
// is the row count) and run as 64 x 64 register-tiled SIMT tiles.
#include <cuda_bf16.h>

#include "kernels.h"
#include "mlp.h"

namespace pepo {

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// ---------------------------------------------------------------- SIMT GEMM
// C[m, n] = sum_k A[m, k] B[k, n] (+ bias[n]); A and B addressed through
// strides (so transposed operands need no copies).  epi: 0 = store C;
// 1 = store z = C + bias and a = bf16(gelu(z)); 2 = store C * gelu'(zref).
struct GemmArgs {
  const float* A; long long sam, sak;
  const float* B; long long sbk, sbn;
  float* C; long long ldc;
  const float* bias;
  float* act;            // epi 1: rounded activation, leading dimension ldc
  const float* zref;     // epi 2: pre-activation the derivative is taken at
  int M, N, K;
  int epi;
};

constexpr int MG_T = 64, MG_BK = 16;

__global__ void __launch_bounds__(256) k_mlp_gemm(GemmArgs g) {
  __shared__ float As[MG_BK][MG_T + 1];
  __shared__ float Bs[MG_BK][MG_T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * MG_T, n0 = blockIdx.x * MG_T;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += MG_BK) {
    for (int e = threadIdx.x; e < MG_BK * MG_T; e += blockDim.x) {
      const int kk = e / MG_T, mm = e - kk * MG_T;
      const int m = m0 + mm, k = k0 + kk, n = n0 + mm;
      As[kk][mm] = (m < g.M && k < g.K) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : 0.f;
      Bs[kk][mm] = (n < g.N && k < g.K) ? g.B[(long long)k * g.sbk + (long long)n * g.sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MG_BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      const long long o = (long long)m * g.ldc + n;
      if (g.epi == 1) {
        v += g.bias[n];
        g.C[o] = v;
        g.act[o] = bf16r(gelu_f(v));
      } else if (g.epi == 2) {
        g.C[o] = v * gelu_grad_f(g.zref[o]);
      } else {
        g.C[o] = v + (g.bias ? g.bias[n] : 0.f);
      }
    }
  }
}

static cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((g.N + MG_T - 1) / MG_T, (g.M + MG_T - 1) / MG_T);
  k_mlp_gemm<<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// column sums: out[n] = sum_m A[m, n] (bias gradients), FP32 with a per-thread
// partial per column block
__global__ void k_colsum(const float* A, int M, int N, long long lda, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += A[(long long)m * lda + n];
  out[n] = s;
}

__global__ void k_round(const float* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = bf16r(in[i]);
}

// dy = 2 / n (y - t) and the loss (one block: deterministic sum)
__global__ void k_mse(const float* y, const float* t, int n, float* dy, float* loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)n;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ------------------------------------------------------------------ features
// One block per directed bond (b, dir).  Rows of bond b start at
// sum_{b' < b} 2 chi_b' + dir chi_b.
__device__ double entropy_fraction(const double* lam, int chi) {
  if (chi < 2) return 0.0;
  double s = 0.0;
  for (int k = 0; k < chi; ++k) {
    const double p = lam[k] * lam[k];
    if (p > 0.0) s -= p * log(p);
  }
  return s / log((double)chi);
}

__global__ void k_ws_features(const WsGeom* __restrict__ geom, int nb, const int* __restrict__ chi,
                              const double* __restrict__ lam, int ldl, float t, float h, float J, float* X,
                              int max_rows) {
  const int db = blockIdx.x;            // directed bond 2 b + dir
  const int b = db >> 1, dir = db & 1;
  __shared__ long long off;
  __shared__ float sf[4];
  if (threadIdx.x == 0) {
    long long o = 0;
    for (int e = 0; e < b; ++e) o += 2LL * chi[e];
    off = o + (long long)dir * chi[b];
  }
  const WsGeom G = geom[db];
  if (threadIdx.x < 4) {
    const int e = threadIdx.x == 0 ? b : (threadIdx.x - 1 < G.n_other ? G.other[threadIdx.x - 1] : -1);
    sf[threadIdx.x] = e >= 0 ? (float)entropy_fraction(lam + (long long)e * ldl, chi[e]) : 0.f;
  }
  __syncthreads();
  float mean_nb = 0.f, max_nb = 0.f;
  for (int i = 0; i < G.n_other; ++i) { mean_nb += sf[1 + i]; max_nb = fmaxf(max_nb, sf[1 + i]); }
  if (G.n_other > 0) mean_nb /= (float)G.n_other;
  const int c = chi[b];
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    const long long r = off + k;
    if (r >= max_rows) continue;
    float* x = X + r * PEPO_WS_FEATURES;
    const double lk = fmax(lam[(long long)b * ldl + k], 1e-30);
    x[0] = (float)log(lk);
    x[1] = (float)k / (float)c;
    x[2] = sf[0];
    x[3] = G.deg_src * 0.25f;
    x[4] = G.deg_dst * 0.25f;
    x[5] = G.dist_src;
    x[6] = G.dist_dst;
    x[7] = t;
    x[8] = h;
    x[9] = J;
    x[10] = mean_nb;
    x[11] = max_nb;
  }
}

// targets: y = log M_e[k, k] of the current messages (after BP)
__global__ void k_ws_targets(int nb, const int* __restrict__ chi, const double* __restrict__ msg, int ldm,
                             float* out, int max_rows) {
  const int db = blockIdx.x;
  const int b = db >> 1, dir = db & 1;
  __shared__ long long off;
  if (threadIdx.x == 0) {
    long long o = 0;
    for (int e = 0; e < b; ++e) o += 2LL * chi[e];
    off = o + (long long)dir * chi[b];
  }
  __syncthreads();
  const int c = chi[b];
  const double* M = msg + (long long)db * ldm * ldm;
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    const long long r = off + k;
    if (r < max_rows) out[r] = (float)log(fmax(M[(long long)k * ldm + k], 1e-300));
  }
}

// messages <- diag((1 - gamma) d / sum d + gamma exp(y) / sum exp(y)), zero
// elsewhere; d = diagonal of the current message (the diag(lambda) written by
// the bond updates), exp(y) max-shifted
__global__ void k_ws_apply(int nb, const int* __restrict__ chi, const float* __restrict__ y, double* msg, int ldm,
                           float gamma) {
  const int db = blockIdx.x;
  const int b = db >> 1, dir = db & 1;
  __shared__ long long off;
  __shared__ double red[256], red2[256];
  __shared__ float ymax;
  if (threadIdx.x == 0) {
    long long o = 0;
    for (int e = 0; e < b; ++e) o += 2LL * chi[e];
    off = o + (long long)dir * chi[b];
  }
  __syncthreads();
  const int c = chi[b];
  double* M = msg + (long long)db * ldm * ldm;
  if (threadIdx.x == 0) {
    float m = -INFINITY;
    for (int k = 0; k < c; ++k) m = fmaxf(m, y[off + k]);
    ymax = m;
  }
  __syncthreads();
  double s = 0.0, sd = 0.0;
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    s += exp((double)(y[off + k] - ymax));
    sd += M[(long long)k * ldm + k];
  }
  red[threadIdx.x] = s;
  red2[threadIdx.x] = sd;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { red[threadIdx.x] += red[threadIdx.x + o]; red2[threadIdx.x] += red2[threadIdx.x + o]; }
    __syncthreads();
  }
  const double tot = red[0], totd = red2[0];
  // diagonal first (read before the overwrite), then the rest
  double dk[8];
  int nk = 0;
  for (int k = threadIdx.x; k < c && nk < 8; k += blockDim.x) dk[nk++] = M[(long long)k * ldm + k];
  __syncthreads();
  nk = 0;
  for (int k = threadIdx.x; k < c && nk < 8; k += blockDim.x) {
    const double plain = totd > 0.0 ? dk[nk] / totd : 0.0;
    dk[nk++] = (1.0 - gamma) * plain + gamma * exp((double)(y[off + k] - ymax)) / tot;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ldm * ldm; e += blockDim.x) {
    const int i = e / ldm, j = e - i * ldm;
    if (i != j || i >= c) M[e] = 0.0;
  }
  nk = 0;
  for (int k = threadIdx.x; k < c && nk < 8; k += blockDim.x) M[(long long)k * ldm + k] = dk[nk++];
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_ws_features(const WsGeom* geom, int nb, const int* chi, const double* lam, int ldl, float t,
                               float h, float J, float* X, int max_rows, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_ws_features<<<2 * nb, 128, 0, s>>>(geom, nb, chi, lam, ldl, t, h, J, X, max_rows);
  return cudaGetLastError();
}
cudaError_t launch_ws_targets(int nb, const int* chi, const double* msg, int ldm, float* out, int max_rows,
                              cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_ws_targets<<<2 * nb, 128, 0, s>>>(nb, chi, msg, ldm, out, max_rows);
  return cudaGetLastError();
}
cudaError_t launch_ws_apply(int nb, const int* chi, const float* y, double* msg, int ldm, float gamma,
                            cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  k_ws_apply<<<2 * nb, 256, 0, s>>>(nb, chi, y, msg, ldm, gamma);
  return cudaGetLastError();
}

// Parameter offsets in the flat vector: W1 [NF x W], b1 [W], W2 [W x W], b2 [W], W3 [W], b3 [1]
struct MlpOff {
  long long W1, b1, W2, b2, W3, b3, n;
};
static MlpOff mlp_off() {
  MlpOff o;
  const long long F = PEPO_WS_FEATURES, W = PEPO_WS_WIDTH;
  o.W1 = 0;
  o.b1 = o.W1 + F * W;
  o.W2 = o.b1 + W;
  o.b2 = o.W2 + W * W;
  o.W3 = o.b2 + W;
  o.b3 = o.W3 + W;
  o.n = o.b3 + 1;
  return o;
}

long long mlp_num_params() { return mlp_off().n; }

size_t mlp_layout(char* base, int max_rows, MlpBuffers* B) {
  const MlpOff o = mlp_off();
  const size_t W = PEPO_WS_WIDTH, F = PEPO_WS_FEATURES, R = (size_t)max_rows;
  size_t off = 0;
  auto take = [&](size_t n) {
    off = (off + 63) / 64 * 64;
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += n * sizeof(float);
    return p;
  };
  B->p = take(o.n);
  B->m = take(o.n);
  B->v = take(o.n);
  B->g = take(o.n);
  B->pr = take(o.n);
  B->x = take(R * F);
  B->z1 = take(R * W);
  B->a1 = take(R * W);
  B->z2 = take(R * W);
  B->a2 = take(R * W);
  B->y = take(R);
  B->dy = take(R);
  B->d2 = take(R * W);
  B->d1 = take(R * W);
  B->loss = take(4);
  return off + 64;
}

// forward pass on the rounded weights; activations kept for backward
cudaError_t mlp_forward(const MlpBuffers& B, const float* X, int rows, float* y_out, cudaStream_t s) {
  const MlpOff o = mlp_off();
  const int W = PEPO_WS_WIDTH, F = PEPO_WS_FEATURES;
  k_round<<<256, 256, 0, s>>>(B.p, B.pr, o.n);
  k_round<<<256, 256, 0, s>>>(X, B.x, (long long)rows * F);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  GemmArgs g{};
  g.A = B.x; g.sam = F; g.sak = 1;
  g.B = B.pr + o.W1; g.sbk = W; g.sbn = 1;
  g.C = B.z1; g.ldc = W; g.bias = B.p + o.b1; g.act = B.a1;
  g.M = rows; g.N = W; g.K = F; g.epi = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return e;
  g.A = B.a1; g.sam = W; g.sak = 1;
  g.B = B.pr + o.W2; g.sbk = W; g.sbn = 1;
  g.C = B.z2; g.bias = B.p + o.b2; g.act = B.a2; g.K = W;
  if ((e = gemm(g, s)) != cudaSuccess) return e;
  GemmArgs h{};
  h.A = B.a2; h.sam = W; h.sak = 1;
  h.B = B.pr + o.W3; h.sbk = 1; h.sbn = 1;
  h.C = y_out ? y_out : B.y; h.ldc = 1; h.bias = B.p + o.b3;
  h.M = rows; h.N = 1; h.K = W; h.epi = 0;
  return gemm(h, s);
}

// forward + backward of the mean squared error; gradient into B.g, loss into B.loss[0]
cudaError_t mlp_gradient(const MlpBuffers& B, const float* X, const float* t, int rows, cudaStream_t s) {
  const MlpOff o = mlp_off();
  const int W = PEPO_WS_WIDTH, F = PEPO_WS_FEATURES;
  cudaError_t e = mlp_forward(B, X, rows, B.y, s);
  if (e != cudaSuccess) return e;
  k_mse<<<1, 256, 0, s>>>(B.y, t, rows, B.dy, B.loss);
  // dW3 = a2^T dy, db3 = sum dy
  GemmArgs g{};
  g.A = B.a2; g.sam = 1; g.sak = W;          // a2^T: [W x rows]
  g.B = B.dy; g.sbk = 1; g.sbn = 1;
  g.C = B.g + o.W3; g.ldc = 1; g.M = W; g.N = 1; g.K = rows; g.epi = 0;
  if ((e = gemm(g, s)) != cudaSuccess) return e;
  k_colsum<<<1, 32, 0, s>>>(B.dy, rows, 1, 1, B.g + o.b3);
  // dz2 = (dy W3^T) * gelu'(z2)
  GemmArgs d{};
  d.A = B.dy; d.sam = 1; d.sak = 1;
  d.B = B.pr + o.W3; d.sbk = 1; d.sbn = 1;     // W3^T as [1 x W]
  d.C = B.d2; d.ldc = W; d.zref = B.z2; d.M = rows; d.N = W; d.K = 1; d.epi = 2;
  if ((e = gemm(d, s)) != cudaSuccess) return e;
  // dW2 = a1^T dz2, db2 = colsum dz2
  g.A = B.a1; g.sam = 1; g.sak = W;
  g.B = B.d2; g.sbk = W; g.sbn = 1;
  g.C = B.g + o.W2; g.ldc = W; g.M = W; g.N = W; g.K = rows;
  if ((e = gemm(g, s)) != cudaSuccess) return e;
  k_colsum<<<(W + 127) / 128, 128, 0, s>>>(B.d2, rows, W, W, B.g + o.b2);
  // dz1 = (dz2 W2^T) * gelu'(z1)
  d.A = B.d2; d.sam = W; d.sak = 1;
  d.B = B.pr + o.W2; d.sbk = 1; d.sbn = W;     // W2^T
  d.C = B.d1; d.zref = B.z1; d.K = W;
  if ((e = gemm(d, s)) != cudaSuccess) return e;
  // dW1 = x^T dz1, db1 = colsum dz1
  g.A = B.x; g.sam = 1; g.sak = F;
  g.B = B.d1; g.sbk = W; g.sbn = 1;
  g.C = B.g + o.W1; g.ldc = W; g.M = F; g.N = W; g.K = rows;
  if ((e = gemm(g, s)) != cudaSuccess) return e;
  k_colsum<<<(W + 127) / 128, 128, 0, s>>>(B.d1, rows, W, W, B.g + o.b1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpBuffers& B, int t, float lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<128, 256, 0, s>>>(B.p, B.m, B.v, B.g, mlp_off().n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace pepo
