// Split-precision tensor-core contractions (precision mode TF32X3).
//
// Each FP32 operand x is split as x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi); a product is accumulated as hi*hi + hi*lo + lo*hi on the
// tensor cores (the lo*lo term, ~2^-22 relative, is dropped), which keeps the
// result close to FP32 accuracy while running the dense contractions of BP
// and of the absorb step on the tensor pipes (Gram and absorb GEMMs of the
// mixed-precision design).
//
//   k_leg_contract_tc  out[o, i, q] = sum_j A[i, j] in[o, j, q]
//   k_gram_leg_tc      out[i, i'] = sum_{o,q} w^2 X[o, i, q] X[o, i', q]
//
// Both use m16n8k8 TF32 MMAs on fragments loaded from padded shared-memory
// tiles (row strides chosen so a warp's fragment loads hit distinct banks).
#include "kernels.h"

namespace pepo {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// three-product split MMA: d += a b with a = ah + al, b = bh + bl
__device__ __forceinline__ void mma3(float* d, const uint32_t* ah, const uint32_t* al,
                                     const uint32_t* bh, const uint32_t* bl) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

__device__ inline void load_dims_tc(const TView& v, const int* ival, int* d) {
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < v.nlegs) ? ival[v.dim[k]] : 1;
}

// ============================================================ leg contraction
// Block tile 128 (i) x 128 (columns); 8 warps as 2 x 4, warp tile 64 x 32
// (4 m16 tiles x 4 n8 tiles).  K = Jin padded to a multiple of 8.
constexpr int TC_M = 128, TC_N = 128;
constexpr int TC_KMAX = 128;
constexpr int TC_AS = TC_KMAX + 4;   // A row stride (floats): bank = 4 g + t
constexpr int TC_BS = TC_N + 8;      // B row stride: bank = 8 t + g

__global__ void __launch_bounds__(256)
k_leg_contract_tc(const LegItem* __restrict__ items, void* const* ptrs, const int* __restrict__ ival) {
  const LegItem it = items[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* As = reinterpret_cast<float*>(smem_raw);   // [TC_M][TC_AS]
  float* Bs = As + TC_M * TC_AS;                      // [TC_KMAX][TC_BS]
  int d[PEPO_MAXLEG];
  load_dims_tc(it.in, ival, d);
  const int k = it.leg;
  const int Jin = d[k];
  const int Jout = ival[it.out_dim];
  const int K8 = (Jin + 7) & ~7;
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.in.nlegs; ++i) Q *= d[i];
  for (int e = threadIdx.x; e < TC_M * K8; e += blockDim.x) {
    int i = e / K8, j = e - i * K8;
    As[i * TC_AS + j] = (i < Jout && j < Jin) ? (float)it.A[(long long)i * it.lda + j] : 0.f;
  }
  long long G, nqb, units;
  if (Q >= TC_N) { G = 1; nqb = (Q + TC_N - 1) / TC_N; units = O * nqb; }
  else { G = TC_N / Q; nqb = 1; units = (O + G - 1) / G; }
  const float* __restrict__ in = static_cast<const float*>(ptrs[it.in.ref]);
  float* __restrict__ out = static_cast<float*>(ptrs[it.out_ref]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp >> 2, wn = warp & 3;         // 2 x 4 warps
  const int g = lane >> 2, t = lane & 3;
  __syncthreads();
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    long long o0, q0;
    int width;
    if (G == 1) { o0 = u / nqb; q0 = (u - o0 * nqb) * TC_N; width = (int)min((long long)TC_N, Q - q0); }
    else { o0 = u * G; q0 = 0; width = (int)(min(G, O - o0) * Q); }
    for (int e = threadIdx.x; e < K8 * TC_N; e += blockDim.x) {
      int j = e / TC_N, c = e - j * TC_N;
      float v = 0.f;
      if (c < width && j < Jin) {
        long long o = (G == 1) ? o0 : o0 + c / Q;
        long long q = (G == 1) ? q0 + c : c % Q;
        v = in[(o * Jin + j) * Q + q];
      }
      Bs[j * TC_BS + c] = v;
    }
    __syncthreads();
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[a][b][r] = 0.f;
    for (int k0 = 0; k0 < K8; k0 += 8) {
      uint32_t ah[4][4], al[4][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int r0 = wm * 64 + a * 16 + g;
        split_tf32(As[r0 * TC_AS + k0 + t], ah[a][0], al[a][0]);
        split_tf32(As[(r0 + 8) * TC_AS + k0 + t], ah[a][1], al[a][1]);
        split_tf32(As[r0 * TC_AS + k0 + t + 4], ah[a][2], al[a][2]);
        split_tf32(As[(r0 + 8) * TC_AS + k0 + t + 4], ah[a][3], al[a][3]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c0 = wn * 32 + b * 8 + g;
        split_tf32(Bs[(k0 + t) * TC_BS + c0], bh[b][0], bl[b][0]);
        split_tf32(Bs[(k0 + t + 4) * TC_BS + c0], bh[b][1], bl[b][1]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) mma3(acc[a][b], ah[a], al[a], bh[b], bl[b]);
    }
    // epilogue: accumulator r -> (row g or g+8, column 2t or 2t+1)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = wn * 32 + b * 8 + 2 * t + cc;
        if (col >= width) continue;
        const long long o = (G == 1) ? o0 : o0 + col / Q;
        const long long q = (G == 1) ? q0 + col : col % Q;
        float* dst = out + o * Jout * Q + q;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int i = wm * 64 + a * 16 + g + 8 * rr;
            if (i < Jout) dst[(long long)i * Q] = acc[a][b][2 * rr + cc];
          }
      }
    __syncthreads();
  }
}

cudaError_t launch_leg_contract_tc(const LegItem* items, int n_items, int grid_x, void* const* ptrs,
                                   const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(float) * ((size_t)TC_M * TC_AS + (size_t)TC_KMAX * TC_BS);
  cudaError_t e = cudaFuncSetAttribute(k_leg_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_leg_contract_tc<<<dim3(grid_x, n_items), 256, smem, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}

// ============================================================ Gram (free leg)
// One 128 x 128 output tile per split (F <= 128), 8 warps as 2 x 4 (warp tile
// 64 x 32).  Chunks of 32 (o, q) pairs as in the SIMT kernel.
constexpr int TG_BK = 32;
constexpr int TG_S = 128 + 8;        // row stride: bank = 8 t + g
constexpr int TG_FLUSH = 512;

__device__ inline double leg_weight_tc(const GramLegItem& it, const int* d, int lo, int hi, long long idx) {
  double w = 1.0;
  for (int u = hi - 1; u >= lo; --u) {
    const long long j = idx % d[u];
    idx /= d[u];
    if (it.sw[u]) w *= it.sw[u][j];
  }
  return w;
}

__global__ void __launch_bounds__(256)
k_gram_leg_tc(const GramLegItem* __restrict__ items, int splits_max, void* const* ptrs,
              const int* __restrict__ ival) {
  const GramLegItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims_tc(it.x, ival, d);
  const int k = it.leg;
  const int F = d[k];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.x.nlegs; ++i) Q *= d[i];
  const long long NC = gram_leg_chunks(O, Q);
  const int S = gram_leg_splits(NC, splits_max);
  const int s = blockIdx.x;
  if (s >= S) return;
  const long long c0 = NC * s / S, c1 = NC * (s + 1) / S;
  const float* __restrict__ X = static_cast<const float*>(ptrs[it.x.ref]);
  bool weighted = false;
  for (int u = 0; u < it.x.nlegs; ++u) weighted |= (u != k && it.sw[u] != nullptr);
  __shared__ __align__(16) float Xs[TG_BK * TG_S];
  __shared__ double wk[TG_BK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp >> 2, wn = warp & 3;
  const int g = lane >> 2, t = lane & 3;
  const bool wideQ = Q >= TG_BK;
  const long long qpc = wideQ ? (Q + TG_BK - 1) / TG_BK : 0;
  const int Qi = wideQ ? TG_BK : (int)Q;
  const int opc = wideQ ? 1 : (int)(TG_BK / Q);
  const int rows = wideQ ? TG_BK : opc * Qi;
  // FP64 shadows of the 64 accumulators of every thread live in shared memory
  extern __shared__ __align__(16) double sh64[];   // [64][256]: entry idx of thread tid at idx*256+tid
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[a][b][r] = 0.f;
  for (int e = threadIdx.x; e < 64 * 256; e += blockDim.x) sh64[e] = 0.0;
  for (int e = threadIdx.x; e < TG_BK * TG_S; e += blockDim.x) Xs[e] = 0.f;
  int run = 0;
  for (long long cch = c0; cch < c1; ++cch) {
    long long o0, q0;
    if (wideQ) { o0 = cch / qpc; q0 = (cch - o0 * qpc) * TG_BK; }
    else { o0 = cch * opc; q0 = 0; }
    __syncthreads();
    if (weighted && threadIdx.x < rows) {
      const int kk = threadIdx.x;
      long long o, q;
      if (wideQ) { o = o0; q = q0 + kk; }
      else { o = o0 + kk / Qi; q = kk % Qi; }
      double w = 0.0;
      if (q < Q && o < O) w = leg_weight_tc(it, d, 0, k, o) * leg_weight_tc(it, d, k + 1, it.x.nlegs, q >> 2);
      wk[kk] = w;
    }
    if (weighted) __syncthreads();
    for (int e = threadIdx.x; e < rows * F; e += blockDim.x) {
      int kk, f;
      long long o, q;
      if (wideQ) { f = e / TG_BK; kk = e - f * TG_BK; o = o0; q = q0 + kk; }
      else {
        int qq = e % Qi, rest = e / Qi;
        f = rest % F;
        int ol = rest / F;
        kk = ol * Qi + qq;
        o = o0 + ol; q = qq;
      }
      float xv = 0.f;
      if (q < Q && o < O) {
        xv = X[(o * F + f) * Q + q];
        if (weighted) xv *= (float)wk[kk];
      }
      Xs[kk * TG_S + f] = xv;
    }
    __syncthreads();
#pragma unroll
    for (int k0 = 0; k0 < TG_BK; k0 += 8) {
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n0 = wn * 32 + b * 8 + g;
        split_tf32(Xs[(k0 + t) * TG_S + n0], bh[b][0], bl[b][0]);
        split_tf32(Xs[(k0 + t + 4) * TG_S + n0], bh[b][1], bl[b][1]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t ah[4], al[4];
        const int m0 = wm * 64 + a * 16 + g;
        split_tf32(Xs[(k0 + t) * TG_S + m0], ah[0], al[0]);
        split_tf32(Xs[(k0 + t) * TG_S + m0 + 8], ah[1], al[1]);
        split_tf32(Xs[(k0 + t + 4) * TG_S + m0], ah[2], al[2]);
        split_tf32(Xs[(k0 + t + 4) * TG_S + m0 + 8], ah[3], al[3]);
#pragma unroll
        for (int b = 0; b < 4; ++b) mma3(acc[a][b], ah, al, bh[b], bl[b]);
      }
    }
    run += TG_BK;
    if (run >= TG_FLUSH) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            sh64[((a * 4 + b) * 4 + r) * 256 + threadIdx.x] += (double)acc[a][b][r];
            acc[a][b][r] = 0.f;
          }
      run = 0;
    }
  }
  double* P = it.partial + (long long)s * F * F;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int fi = wm * 64 + a * 16 + g + 8 * (r >> 1);
        const int fj = wn * 32 + b * 8 + 2 * t + (r & 1);
        if (fi < F && fj < F)
          P[(long long)fi * F + fj] = sh64[((a * 4 + b) * 4 + r) * 256 + threadIdx.x] + (double)acc[a][b][r];
      }
}

cudaError_t launch_gram_leg_tc(const GramLegItem* items, int n_items, int splits_max, void* const* ptrs,
                               const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = sizeof(double) * 64 * 256;
  cudaError_t e = cudaFuncSetAttribute(k_gram_leg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_leg_tc<<<dim3(splits_max, n_items), 256, smem, s>>>(items, splits_max, ptrs, ival);
  return cudaGetLastError();
}

}  // namespace pepo
