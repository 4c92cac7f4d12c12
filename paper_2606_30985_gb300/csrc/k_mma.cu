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
// Both use m16n8k8 TF32 MMAs on fragments read from padded shared-memory
// tiles (strides chosen so a warp's fragment loads hit distinct banks).  Tiles
// are streamed from global memory with 16-byte cp.async copies (zero-filled
// past the edges) into two buffers: the next tile is in flight while the
// current one is multiplied.
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

// 16-byte asynchronous global -> shared copy; bytes beyond `valid` are zero
__device__ __forceinline__ void cp16(void* smem, const void* gmem, int valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

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

struct LegTile {
  long long o0, q0;
  int width;
};

__device__ __forceinline__ LegTile leg_tile(long long u, long long G, long long nqb, long long O, long long Q) {
  LegTile t;
  if (G == 1) { t.o0 = u / nqb; t.q0 = (u - t.o0 * nqb) * TC_N; t.width = (int)min((long long)TC_N, Q - t.q0); }
  else { t.o0 = u * G; t.q0 = 0; t.width = (int)(min(G, O - t.o0) * Q); }
  return t;
}

// issue the copies of one B tile (Jin rows x 128 columns) into buf
__device__ __forceinline__ void leg_issue(float* buf, const float* in, const LegTile& t, long long G,
                                          long long Q, int Jin, int K8) {
  // 32 chunks of 4 floats per row; rows Jin..K8-1 are zero
  for (int e = threadIdx.x; e < K8 * (TC_N / 4); e += blockDim.x) {
    const int j = e >> 5, ch = e & 31;
    const int c = ch * 4;
    float* dst = buf + j * TC_BS + c;
    int valid = 0;
    const float* src = in;
    if (j < Jin && c < t.width) {
      const long long o = (G == 1) ? t.o0 : t.o0 + c / Q;
      const long long q = (G == 1) ? t.q0 + c : c % Q;
      src = in + (o * Jin + j) * Q + q;
      const int left = t.width - c;
      valid = (left >= 4 ? 4 : left) * 4;
    }
    cp16(dst, src, valid);
  }
}

__global__ void __launch_bounds__(256)
k_leg_contract_tc(const LegItem* __restrict__ items, void* const* ptrs, const int* __restrict__ ival) {
  const LegItem it = items[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* As = reinterpret_cast<float*>(smem_raw);       // [TC_M][TC_AS]
  float* Bb[2] = {As + TC_M * TC_AS, As + TC_M * TC_AS + TC_KMAX * TC_BS};
  int d[PEPO_MAXLEG];
  load_dims_tc(it.in, ival, d);
  const int k = it.leg;
  const int Jin = d[k];
  const int Jout = ival[it.out_dim];
  const int K8 = (Jin + 7) & ~7;
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.in.nlegs; ++i) Q *= d[i];
  long long G, nqb, units;
  if (Q >= TC_N) { G = 1; nqb = (Q + TC_N - 1) / TC_N; units = O * nqb; }
  else { G = TC_N / Q; nqb = 1; units = (O + G - 1) / G; }
  const float* __restrict__ in = static_cast<const float*>(ptrs[it.in.ref]);
  float* __restrict__ out = static_cast<float*>(ptrs[it.out_ref]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp >> 2, wn = warp & 3;         // 2 x 4 warps
  const int g = lane >> 2, t = lane & 3;
  long long u = blockIdx.x;
  if (u < units) leg_issue(Bb[0], in, leg_tile(u, G, nqb, O, Q), G, Q, Jin, K8);
  cp_commit();
  for (int e = threadIdx.x; e < TC_M * K8; e += blockDim.x) {
    int i = e / K8, j = e - i * K8;
    As[i * TC_AS + j] = (i < Jout && j < Jin) ? (float)it.A[(long long)i * it.lda + j] : 0.f;
  }
  int buf = 0;
  for (; u < units; u += gridDim.x) {
    const LegTile cur = leg_tile(u, G, nqb, O, Q);
    const long long un = u + gridDim.x;
    if (un < units) leg_issue(Bb[buf ^ 1], in, leg_tile(un, G, nqb, O, Q), G, Q, Jin, K8);
    cp_commit();
    cp_wait_1();
    __syncthreads();
    const float* Bs = Bb[buf];
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[a][b][r] = 0.f;
    for (int k0 = 0; k0 < K8; k0 += 8) {
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c0 = wn * 32 + b * 8 + g;
        split_tf32(Bs[(k0 + t) * TC_BS + c0], bh[b][0], bl[b][0]);
        split_tf32(Bs[(k0 + t + 4) * TC_BS + c0], bh[b][1], bl[b][1]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t ah[4], al[4];
        const int r0 = wm * 64 + a * 16 + g;
        split_tf32(As[r0 * TC_AS + k0 + t], ah[0], al[0]);
        split_tf32(As[(r0 + 8) * TC_AS + k0 + t], ah[1], al[1]);
        split_tf32(As[r0 * TC_AS + k0 + t + 4], ah[2], al[2]);
        split_tf32(As[(r0 + 8) * TC_AS + k0 + t + 4], ah[3], al[3]);
#pragma unroll
        for (int b = 0; b < 4; ++b) mma3(acc[a][b], ah, al, bh[b], bl[b]);
      }
    }
    __syncthreads();   // buffer `buf` may be refilled from the next iteration on
    // epilogue: accumulator r -> (row g or g+8, column 2t or 2t+1)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = wn * 32 + b * 8 + 2 * t + cc;
        if (col >= cur.width) continue;
        const long long o = (G == 1) ? cur.o0 : cur.o0 + col / Q;
        const long long q = (G == 1) ? cur.q0 + col : col % Q;
        float* dst = out + o * Jout * Q + q;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int i = wm * 64 + a * 16 + g + 8 * rr;
            if (i < Jout) dst[(long long)i * Q] = acc[a][b][2 * rr + cc];
          }
      }
    buf ^= 1;
  }
  cp_wait_0();
}

cudaError_t launch_leg_contract_tc(const LegItem* items, int n_items, int grid_x, void* const* ptrs,
                                   const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(float) * ((size_t)TC_M * TC_AS + 2 * (size_t)TC_KMAX * TC_BS);
  cudaError_t e = cudaFuncSetAttribute(k_leg_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_leg_contract_tc<<<dim3(grid_x, n_items), 256, smem, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}

// ============================================================ Gram (free leg)
// One 128 x 128 output tile per split (F <= 128), 8 warps as 2 x 4 (warp tile
// 64 x 32).  A chunk is 64 (o, q) pairs: one o and 64 consecutive q when
// Q >= 64, else floor(64 / Q) consecutive o with all q.  Shared tile layout
// Xs[f][kk] (row stride 68 floats): each (o, f) run of q is contiguous in both
// memories, and fragment reads hit bank 4 g + t.
constexpr int TG_BK = 64;
constexpr int TG_S = TG_BK + 4;
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

struct GramChunk {
  long long o0, q0;
};

__device__ __forceinline__ GramChunk gram_chunk(long long cch, bool wideQ, long long qpc, int opc) {
  GramChunk c;
  if (wideQ) { c.o0 = cch / qpc; c.q0 = (cch - c.o0 * qpc) * TG_BK; }
  else { c.o0 = cch * opc; c.q0 = 0; }
  return c;
}

// issue the copies of one chunk into buf ([F][TG_S]) and its squared weights
__device__ __forceinline__ void gram_issue(float* buf, double* w2, const GramLegItem& it, const int* d,
                                           int k, const float* X, const GramChunk& c, bool wideQ,
                                           int Qi, int opc, int F, long long O, long long Q,
                                           bool weighted) {
  const int qch = Qi / 4;                        // 16-byte chunks per (o, f) run
  const int per_f = wideQ ? TG_BK / 4 : opc * qch;
  for (int e = threadIdx.x; e < F * per_f; e += blockDim.x) {
    const int f = e / per_f, r = e - f * per_f;
    int ol, q4;
    if (wideQ) { ol = 0; q4 = r; }
    else { ol = r / qch; q4 = r - ol * qch; }
    const long long o = c.o0 + ol;
    const long long q = (wideQ ? c.q0 : 0) + q4 * 4;
    const int kk = ol * Qi + q4 * 4;
    float* dst = buf + f * TG_S + kk;
    int valid = 0;
    const float* src = X;
    if (o < O && q < Q) {
      src = X + (o * F + f) * Q + q;
      const long long left = Q - q;
      valid = (int)(left >= 4 ? 4 : left) * 4;
    }
    cp16(dst, src, valid);
  }
  if (weighted && threadIdx.x < TG_BK) {
    const int kk = threadIdx.x;
    long long o, q;
    if (wideQ) { o = c.o0; q = c.q0 + kk; }
    else { o = c.o0 + kk / Qi; q = kk % Qi; }
    double w = 0.0;
    if (kk < (wideQ ? TG_BK : opc * Qi) && q < Q && o < O) {
      w = leg_weight_tc(it, d, 0, k, o) * leg_weight_tc(it, d, k + 1, it.x.nlegs, q >> 2);
      w *= w;
    }
    w2[kk] = w;
  }
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
  const int S = gram_leg_splits_k(O * Q, splits_max);
  const int s = blockIdx.x;
  if (s >= S) return;
  const bool wideQ = Q >= TG_BK;
  const long long qpc = wideQ ? (Q + TG_BK - 1) / TG_BK : 0;
  const int Qi = wideQ ? TG_BK : (int)Q;
  const int opc = wideQ ? 1 : (int)(TG_BK / Q);
  const long long NC = wideQ ? O * qpc : (O + opc - 1) / opc;
  const long long c0 = NC * s / S, c1 = NC * (s + 1) / S;
  const float* __restrict__ X = static_cast<const float*>(ptrs[it.x.ref]);
  bool weighted = false;
  for (int u = 0; u < it.x.nlegs; ++u) weighted |= (u != k && it.sw[u] != nullptr);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sh64 = reinterpret_cast<double*>(smem_raw);          // [64][256] FP64 shadows
  float* Xb[2] = {reinterpret_cast<float*>(sh64 + 64 * 256),
                  reinterpret_cast<float*>(sh64 + 64 * 256) + 128 * TG_S};
  __shared__ double w2s[2][TG_BK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp >> 2, wn = warp & 3;
  const int g = lane >> 2, t = lane & 3;
  // rows F..127 of both buffers stay zero
  for (int e = threadIdx.x; e < 2 * 128 * TG_S; e += blockDim.x) Xb[0][e] = 0.f;
  for (int e = threadIdx.x; e < 64 * 256; e += blockDim.x) sh64[e] = 0.0;
  __syncthreads();
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[a][b][r] = 0.f;
  if (c0 < c1)
    gram_issue(Xb[0], w2s[0], it, d, k, X, gram_chunk(c0, wideQ, qpc, opc), wideQ, Qi, opc, F, O, Q, weighted);
  cp_commit();
  int buf = 0, run = 0;
  for (long long cch = c0; cch < c1; ++cch) {
    if (cch + 1 < c1)
      gram_issue(Xb[buf ^ 1], w2s[buf ^ 1], it, d, k, X, gram_chunk(cch + 1, wideQ, qpc, opc), wideQ, Qi,
                 opc, F, O, Q, weighted);
    cp_commit();
    cp_wait_1();
    __syncthreads();
    const float* Xs = Xb[buf];
    const double* w2 = w2s[buf];
#pragma unroll 2
    for (int k0 = 0; k0 < TG_BK; k0 += 8) {
      float wa = 1.f, wb = 1.f;
      if (weighted) { wa = (float)w2[k0 + t]; wb = (float)w2[k0 + t + 4]; }
      uint32_t bh[4][2], bl[4][2];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n0 = wn * 32 + b * 8 + g;
        split_tf32(Xs[n0 * TG_S + k0 + t], bh[b][0], bl[b][0]);
        split_tf32(Xs[n0 * TG_S + k0 + t + 4], bh[b][1], bl[b][1]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t ah[4], al[4];
        const int m0 = wm * 64 + a * 16 + g;
        split_tf32(Xs[m0 * TG_S + k0 + t] * wa, ah[0], al[0]);
        split_tf32(Xs[(m0 + 8) * TG_S + k0 + t] * wa, ah[1], al[1]);
        split_tf32(Xs[m0 * TG_S + k0 + t + 4] * wb, ah[2], al[2]);
        split_tf32(Xs[(m0 + 8) * TG_S + k0 + t + 4] * wb, ah[3], al[3]);
#pragma unroll
        for (int b = 0; b < 4; ++b) mma3(acc[a][b], ah, al, bh[b], bl[b]);
      }
    }
    __syncthreads();   // buffer may be refilled from the next iteration on
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
    buf ^= 1;
  }
  cp_wait_0();
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
  const size_t smem = sizeof(double) * 64 * 256 + sizeof(float) * 2 * 128 * TG_S;
  cudaError_t e = cudaFuncSetAttribute(k_gram_leg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_leg_tc<<<dim3(splits_max, n_items), 256, smem, s>>>(items, splits_max, ptrs, ival);
  return cudaGetLastError();
}

}  // namespace pepo
