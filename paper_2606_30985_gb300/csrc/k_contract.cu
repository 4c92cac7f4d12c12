// Register-tiled SIMT contractions of the BP and bond-update hot loop.
//
//   k_leg_contract  out[o, i, q] = sum_j A[i, j] in[o, j, q] on one layout leg
//                   (absorbing a message factor or eigenbasis into a site
//                   tensor: Sec. 2.5 step 1 and the products of Eq. 13)
//   k_gram_leg      out[i, i'] = sum_{o, q} w(o,q)^2 X[o, i, q] Y[o, i', q]: a site
//                   tensor contracted with itself over every index but one leg,
//                   the Pauli leg traced, optionally weighted (one double-layer
//                   message, Eq. 13)
//
// Both are GEMMs with one short dimension (chi <= 128).  The tile edge TL is
// 64 or 128 (chosen from chi_max); a block of 256 threads owns a TL x TL
// output tile, each thread an (TL/16) x (TL/16) register tile.  With TL = 128
// the 8 rows / columns of a thread are split in two halves 64 apart so the
// 16-byte shared-memory loads of a warp hit distinct banks.  The leg
// contraction stages A transposed in shared memory once per block.  FP32
// storage accumulates the Gram's long sums in FP32 runs flushed into FP64
// every 256 terms.
#include "kernels.h"

namespace pepo {

template <int TL>
__device__ __forceinline__ int tile_idx(int t, int r) {
  if constexpr (TL == 128) return (r < 4) ? t * 4 + r : 64 + t * 4 + (r - 4);
  else return t * 4 + r;
}

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T* v) {
  if constexpr (sizeof(T) == 4) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    double2 x = *reinterpret_cast<const double2*>(p);
    double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

template <int TL, typename T>
__device__ __forceinline__ void ld_frag(const T* row, int t, T* v) {
  lds4(row + t * 4, v);
  if constexpr (TL == 128) lds4(row + 64 + t * 4, v + 4);
}

__device__ inline void load_dims4(const TView& v, const int* ival, int* d) {
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < v.nlegs) ? ival[v.dim[k]] : 1;
}

// ============================================================ leg contraction
// Block tile: TL rows (output index i) x TC columns (o, q); TC = TL for FP32,
// TL / 2 for FP64 (shared-memory bound).
template <typename T, int TL>
struct LegCfg {
  // column tile: TL, except FP64 with TL = 128 (64, to fit shared memory)
  static constexpr int TC = (sizeof(T) == 8 && TL == 128) ? 64 : TL;
  static constexpr int MR = TL / 16;
  static constexpr int MC = TC / 16;
  // fragment loads read columns t*4 .. t*4+3 (and +64 when the tile is 128)
  static_assert(TL == 64 || TL == 128, "row tile must be 64 or 128");
  static_assert(TC == 64 || TC == 128, "column tile must be 64 or 128");
  static_assert(MR * 16 == TL && MC * 16 == TC, "16 x 16 threads cover the tile");
};

template <typename T, int TL>
__global__ void __launch_bounds__(256)
k_leg_contract(const LegItem* __restrict__ items, void* const* ptrs, const int* __restrict__ ival) {
  using C = LegCfg<T, TL>;
  constexpr int TC = C::TC, MR = C::MR, MC = C::MC;
  const LegItem it = items[blockIdx.y];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int d[PEPO_MAXLEG];
  load_dims4(it.in, ival, d);
  const int k = it.leg;
  const int Jin = d[k];
  const int Jout = ival[it.out_dim];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.in.nlegs; ++i) Q *= d[i];
  T* At = reinterpret_cast<T*>(smem_raw);     // [Jin][TL]
  T* Bs = At + Jin * TL;                      // [Jin][TC]
  for (int e = threadIdx.x; e < Jin * TL; e += blockDim.x) {
    int j = e / TL, i = e - j * TL;
    At[e] = (i < Jout) ? (T)it.A[(long long)i * it.lda + j] : T(0);
  }
  long long G, nqb, units;
  if (Q >= TC) { G = 1; nqb = (Q + TC - 1) / TC; units = O * nqb; }
  else { G = TC / Q; nqb = 1; units = (O + G - 1) / G; }
  const T* __restrict__ in = static_cast<const T*>(ptrs[it.in.ref]);
  T* __restrict__ out = static_cast<T*>(ptrs[it.out_ref]);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __syncthreads();
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    long long o0, q0;
    int width;
    if (G == 1) { o0 = u / nqb; q0 = (u - o0 * nqb) * TC; width = (int)min((long long)TC, Q - q0); }
    else { o0 = u * G; q0 = 0; width = (int)(min(G, O - o0) * Q); }
    for (int e = threadIdx.x; e < Jin * TC; e += blockDim.x) {
      int j = e / TC, c = e - j * TC;
      T v = T(0);
      if (c < width) {
        long long o = (G == 1) ? o0 : o0 + c / Q;
        long long q = (G == 1) ? q0 + c : c % Q;
        v = in[(o * Jin + j) * Q + q];
      }
      Bs[e] = v;
    }
    __syncthreads();
    T acc[MR][MC];
#pragma unroll
    for (int r = 0; r < MR; ++r)
#pragma unroll
      for (int c = 0; c < MC; ++c) acc[r][c] = T(0);
#pragma unroll 2
    for (int j = 0; j < Jin; ++j) {
      T a[MR], b[MC];
      ld_frag<TL>(At + j * TL, ty, a);
      ld_frag<TC>(Bs + j * TC, tx, b);
#pragma unroll
      for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int col = tile_idx<TC>(tx, c);
      if (col >= width) continue;
      const long long o = (G == 1) ? o0 : o0 + col / Q;
      const long long q = (G == 1) ? q0 + col : col % Q;
      T* dst = out + o * Jout * Q + q;
#pragma unroll
      for (int r = 0; r < MR; ++r) {
        const int i = tile_idx<TL>(ty, r);
        if (i < Jout) dst[(long long)i * Q] = acc[r][c];
      }
    }
    __syncthreads();
  }
}

template <typename T, int TL>
cudaError_t launch_leg_tl(const LegItem* items, int n_items, int grid_x, int chimax, void* const* ptrs,
                          const int* ival, cudaStream_t s) {
  size_t smem = sizeof(T) * (size_t)chimax * (TL + LegCfg<T, TL>::TC);
  cudaError_t e = cudaFuncSetAttribute(k_leg_contract<T, TL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_leg_contract<T, TL><<<dim3(grid_x, n_items), 256, smem, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leg_contract(const LegItem* items, int n_items, int grid_x, int chimax,
                                void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (chimax <= 64) return launch_leg_tl<T, 64>(items, n_items, grid_x, chimax, ptrs, ival, s);
  return launch_leg_tl<T, 128>(items, n_items, grid_x, chimax, ptrs, ival, s);
}

// ============================================================ Gram (free leg)
// X, Y as [O][F][Q], F <= TL.  A chunk is 32 (o, q) pairs: one o and 32
// consecutive q when Q >= 32, else floor(32 / Q) consecutive o with all q.
constexpr int GL_BK = 32;
constexpr int GL_FLUSH = 256;

// product of the square-root weights sw[u][j_u] over layout legs u in [lo, hi)
// for the row-major multi-index `idx` of those legs
__device__ inline double leg_weight(const GramLegItem& it, const int* d, int lo, int hi, long long idx) {
  double w = 1.0;
  for (int u = hi - 1; u >= lo; --u) {
    const long long j = idx % d[u];
    idx /= d[u];
    if (it.sw[u]) w *= it.sw[u][j];
  }
  return w;
}

template <typename T, int TL>
__global__ void __launch_bounds__(256)
k_gram_leg(const GramLegItem* __restrict__ items, int splits_max, void* const* ptrs,
           const int* __restrict__ ival) {
  constexpr int MR = TL / 16;
  const GramLegItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims4(it.x, ival, d);
  const int k = it.leg;
  const int F = d[k];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.x.nlegs; ++i) Q *= d[i];
  const long long NC = gram_leg_chunks(O, Q);
  const int S = gram_leg_splits_k(O * Q, splits_max);
  const int s = blockIdx.x;
  if (s >= S) return;
  const long long c0 = NC * s / S, c1 = NC * (s + 1) / S;
  const T* __restrict__ X = static_cast<const T*>(ptrs[it.x.ref]);
  const T* __restrict__ Y = static_cast<const T*>(ptrs[it.y_ref]);
  const bool same = it.x.ref == it.y_ref;
  bool weighted = false;
  for (int u = 0; u < it.x.nlegs; ++u) weighted |= (u != k && it.sw[u] != nullptr);
  __shared__ __align__(16) T Xs[GL_BK][TL];
  __shared__ __align__(16) T Ys[GL_BK][TL];
  __shared__ double wk[GL_BK];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool wideQ = Q >= GL_BK;
  const long long qpc = wideQ ? (Q + GL_BK - 1) / GL_BK : 0;
  const int Qi = wideQ ? GL_BK : (int)Q;
  const int opc = wideQ ? 1 : (int)(GL_BK / Q);
  const int rows = wideQ ? GL_BK : opc * Qi;        // live rows of a chunk
  T* Yt = same ? &Xs[0][0] : &Ys[0][0];
  constexpr int NS = sizeof(T) == 4 ? MR : 1;
  T acc[MR][MR];
  double acc64[NS][MR];
#pragma unroll
  for (int r = 0; r < MR; ++r)
#pragma unroll
    for (int c = 0; c < MR; ++c) acc[r][c] = T(0);
#pragma unroll
  for (int r = 0; r < NS; ++r)
#pragma unroll
    for (int c = 0; c < MR; ++c) acc64[r][c] = 0.0;
  // rows beyond `rows` and columns beyond F stay zero for the whole block
  for (int e = threadIdx.x; e < GL_BK * TL; e += blockDim.x) {
    (&Xs[0][0])[e] = T(0);
    (&Ys[0][0])[e] = T(0);
  }
  int run = 0;
  for (long long cch = c0; cch < c1; ++cch) {
    long long o0, q0;
    if (wideQ) { o0 = cch / qpc; q0 = (cch - o0 * qpc) * GL_BK; }
    else { o0 = cch * opc; q0 = 0; }
    __syncthreads();   // previous chunk consumed
    if (weighted && threadIdx.x < rows) {
      const int kk = threadIdx.x;
      long long o, q;
      if (wideQ) { o = o0; q = q0 + kk; }
      else { o = o0 + kk / Qi; q = kk % Qi; }
      double w = 0.0;
      if (q < Q && o < O) w = leg_weight(it, d, 0, k, o) * leg_weight(it, d, k + 1, it.x.nlegs, q >> 2);
      wk[kk] = w;
    }
    if (weighted) __syncthreads();
    for (int e = threadIdx.x; e < rows * F; e += blockDim.x) {
      int kk, f;
      long long o, q;
      if (wideQ) { f = e / GL_BK; kk = e - f * GL_BK; o = o0; q = q0 + kk; }
      else {
        int qq = e % Qi, rest = e / Qi;
        f = rest % F;
        int ol = rest / F;
        kk = ol * Qi + qq;
        o = o0 + ol; q = qq;
      }
      T xv = T(0), yv = T(0);
      if (q < Q && o < O) {
        long long idx = (o * F + f) * Q + q;
        xv = X[idx];
        if (!same) yv = Y[idx];
        if (weighted) {
          const T w = (T)wk[kk];
          xv *= w;
          yv *= w;
        }
      }
      Xs[kk][f] = xv;
      if (!same) Ys[kk][f] = yv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GL_BK; ++kk) {
      T a[MR], b[MR];
      ld_frag<TL>(&Xs[kk][0], ty, a);
      ld_frag<TL>(Yt + kk * TL, tx, b);
#pragma unroll
      for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MR; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    if constexpr (sizeof(T) == 4) {
      run += GL_BK;
      if (run >= GL_FLUSH) {
#pragma unroll
        for (int r = 0; r < MR; ++r)
#pragma unroll
          for (int c = 0; c < MR; ++c) { acc64[r % NS][c] += (double)acc[r][c]; acc[r][c] = T(0); }
        run = 0;
      }
    }
  }
  double* P = it.partial + (long long)s * F * F;
#pragma unroll
  for (int r = 0; r < MR; ++r) {
    const int fi = tile_idx<TL>(ty, r);
    if (fi >= F) continue;
#pragma unroll
    for (int c = 0; c < MR; ++c) {
      const int fj = tile_idx<TL>(tx, c);
      if (fj < F) {
        double v = (double)acc[r][c];
        if constexpr (sizeof(T) == 4) v += acc64[r % NS][c];
        P[(long long)fi * F + fj] = v;
      }
    }
  }
}

__global__ void k_gram_leg_reduce(const GramLegItem* __restrict__ items, int splits_max, int sym,
                                  const int* __restrict__ ival) {
  const GramLegItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims4(it.x, ival, d);
  const int k = it.leg;
  const int F = d[k];
  long long O = 1, Q = 4;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.x.nlegs; ++i) Q *= d[i];
  const int S = gram_leg_splits_k(O * Q, splits_max);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < F * F; e += gridDim.x * blockDim.x) {
    int fi = e / F, fj = e - fi * F;
    double sum = 0.0;
    for (int s = 0; s < S; ++s) sum += it.partial[(long long)s * F * F + e];
    if (sym) {
      double st = 0.0;
      for (int s = 0; s < S; ++s) st += it.partial[(long long)s * F * F + (long long)fj * F + fi];
      sum = 0.5 * (sum + st);
    }
    it.out[(long long)fi * it.ldo + fj] = sum;
  }
}

template <typename T>
cudaError_t launch_gram_leg(const GramLegItem* items, int n_items, int splits_max, int chimax,
                            void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (chimax <= 64)
    k_gram_leg<T, 64><<<dim3(splits_max, n_items), 256, 0, s>>>(items, splits_max, ptrs, ival);
  else
    k_gram_leg<T, 128><<<dim3(splits_max, n_items), 256, 0, s>>>(items, splits_max, ptrs, ival);
  return cudaGetLastError();
}

cudaError_t launch_gram_leg_reduce(const GramLegItem* items, int n_items, int chimax,
                                   int splits_max, int sym, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  int gx = ceil_div(chimax * chimax, 256);
  k_gram_leg_reduce<<<dim3(gx, n_items), 256, 0, s>>>(items, splits_max, sym, ival);
  return cudaGetLastError();
}

// ==================================================================== permute
// Canonical site layout -> stored layout (or back): out[perm position] = in[i].
// perm[k] = canonical leg index at layout position k; dims in canonical order.
template <typename T>
__global__ void k_permute(const T* __restrict__ in, T* __restrict__ out, int nlegs, int4 dims,
                          int4 perm, int to_layout) {
  const int dc[4] = {dims.x, dims.y, dims.z, dims.w};
  const int pm[4] = {perm.x, perm.y, perm.z, perm.w};
  long long n = 4;
  for (int k = 0; k < nlegs; ++k) n *= dc[k];
  // strides of the canonical legs inside the layout
  long long sl[4] = {0, 0, 0, 0};
  long long st = 4;
  for (int k = nlegs - 1; k >= 0; --k) { sl[pm[k]] = st; st *= dc[pm[k]]; }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    long long rem = e >> 2, dst = e & 3;
    for (int k = nlegs - 1; k >= 0; --k) {
      long long j = rem % dc[k];
      rem /= dc[k];
      dst += j * sl[k];
    }
    if (to_layout) out[dst] = in[e];
    else out[e] = in[dst];
  }
}

template <typename T>
cudaError_t launch_permute(const void* in, void* out, int nlegs, const int* dims_canon, const int* perm,
                           int to_layout, cudaStream_t s) {
  int4 d = make_int4(nlegs > 0 ? dims_canon[0] : 1, nlegs > 1 ? dims_canon[1] : 1,
                     nlegs > 2 ? dims_canon[2] : 1, nlegs > 3 ? dims_canon[3] : 1);
  int4 p = make_int4(nlegs > 0 ? perm[0] : 0, nlegs > 1 ? perm[1] : 0, nlegs > 2 ? perm[2] : 0,
                     nlegs > 3 ? perm[3] : 0);
  k_permute<T><<<1024, 256, 0, s>>>(static_cast<const T*>(in), static_cast<T*>(out), nlegs, d, p,
                                    to_layout);
  return cudaGetLastError();
}

template cudaError_t launch_leg_contract<float>(const LegItem*, int, int, int, void* const*,
                                                const int*, cudaStream_t);
template cudaError_t launch_leg_contract<double>(const LegItem*, int, int, int, void* const*,
                                                 const int*, cudaStream_t);
template cudaError_t launch_gram_leg<float>(const GramLegItem*, int, int, int, void* const*,
                                            const int*, cudaStream_t);
template cudaError_t launch_gram_leg<double>(const GramLegItem*, int, int, int, void* const*,
                                             const int*, cudaStream_t);
template cudaError_t launch_permute<float>(const void*, void*, int, const int*, const int*, int,
                                           cudaStream_t);
template cudaError_t launch_permute<double>(const void*, void*, int, const int*, const int*, int,
                                            cudaStream_t);

}  // namespace pepo
