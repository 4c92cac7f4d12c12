// HBM-bound tensor kernels of the bond update and of BP.
//
//   k_gram_rows      cv^T cv with FP64 accumulation (Eq. 10, Cholesky-QR Gram)
//   k_reconstruct    psi_new = psi W written in the next update's layout
//                    (Sec. 2.5 steps 6-7 in Q-less form, Alg. 1 lines 9-12)
//   k_vec_contract   one-leg vector contraction (single-layer BP, Sec. 2.6)
//
// All sizes are read on the device (see common.cuh).  Accumulation: FP32
// storage accumulates with FP32 FMAs over short runs that are flushed into
// FP64 registers, so long sums (up to chi^3 terms) keep FP64-level error
// (Sec. 4.2 "Gram matrix accumulation error": the paper's FP32 Gram loses
// m * eps; this does not).
#include "kernels.h"

namespace pepo {

template <typename T> struct Flush;
template <> struct Flush<float> {
  static constexpr bool kFlush = true;
};
template <> struct Flush<double> {
  static constexpr bool kFlush = false;
};

__device__ inline void load_dims(const TView& v, const int* ival, int* d) {
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < v.nlegs) ? ival[v.dim[k]] : 1;
}

// ======================================================================= copy
template <typename T>
__global__ void k_copy(const TView* __restrict__ items, const int* __restrict__ out_refs,
                       void* const* ptrs, const int* __restrict__ ival) {
  const TView v = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims(v, ival, d);
  long long n = 4;
  for (int k = 0; k < v.nlegs; ++k) n *= d[k];
  const T* in = static_cast<const T*>(ptrs[v.ref]);
  T* out = static_cast<T*>(ptrs[out_refs[blockIdx.y]]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i];
}

template <typename T>
cudaError_t launch_copy(const TView* items, const int* out_refs, int n_items, int grid_x,
                        void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_copy<T><<<dim3(grid_x, n_items), 256, 0, s>>>(items, out_refs, ptrs, ival);
  return cudaGetLastError();
}

// ================================================================ Gram (rows)
// 64 x 64 output tile per block, 16 x 16 threads with 4 x 4 micro-tiles,
// K streamed 16 rows at a time.
constexpr int GR_T = 64;
constexpr int GR_BK = 16;
constexpr int GR_FLUSH = 256;   // FP32 run length before the FP64 flush

__device__ inline void tile_of(int t, int nt, int sym, int& ti, int& tj) {
  if (!sym) { ti = t / nt; tj = t - ti * nt; return; }
  // upper-triangular enumeration: row ti holds nt - ti tiles
  int r = 0, base = 0;
  while (r < nt && t >= base + (nt - r)) { base += nt - r; ++r; }
  ti = r; tj = r + (t - base);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gram_rows(const GramRowsItem* __restrict__ items, int splits_max, int sym, void* const* ptrs,
            const int* __restrict__ ival) {
  const GramRowsItem it = items[blockIdx.z];
  if (it.active >= 0 && ival[it.active] == 0) return;
  int d[PEPO_MAXLEG];
  load_dims(it.x, ival, d);
  const int nl = it.x.nlegs;
  const int F = 4 * (nl > 0 ? d[nl - 1] : 1);
  long long K = 1;
  for (int i = 0; i + 1 < nl; ++i) K *= d[i];
  const int S = gram_rows_splits(K, splits_max);
  const int s = blockIdx.x % splits_max;
  const int t = blockIdx.x / splits_max;
  const int nt = ceil_div(F, GR_T);
  const int ntiles = sym ? nt * (nt + 1) / 2 : nt * nt;
  if (s >= S || t >= ntiles) return;
  int ti, tj;
  tile_of(t, nt, sym, ti, tj);
  const long long k0 = K * s / S, k1 = K * (s + 1) / S;
  const T* __restrict__ X = static_cast<const T*>(ptrs[it.x.ref]);
  const T* __restrict__ Y = static_cast<const T*>(ptrs[it.y_ref]);
  __shared__ __align__(16) T Xs[GR_BK][GR_T];
  __shared__ __align__(16) T Ys[GR_BK][GR_T];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = T(0); acc64[a][b] = 0.0; }
  int run = 0;
  for (long long kb = k0; kb < k1; kb += GR_BK) {
    for (int e = threadIdx.x; e < GR_BK * GR_T; e += blockDim.x) {
      int kk = e / GR_T, c = e - kk * GR_T;
      long long k = kb + kk;
      int fi = ti * GR_T + c, fj = tj * GR_T + c;
      bool okk = k < k1;
      Xs[kk][c] = (okk && fi < F) ? X[k * F + fi] : T(0);
      Ys[kk][c] = (okk && fj < F) ? Y[k * F + fj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GR_BK; ++kk) {
      T xa[4], yb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
    }
    __syncthreads();
    if (Flush<T>::kFlush) {
      run += GR_BK;
      if (run >= GR_FLUSH) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) { acc64[a][b] += (double)acc[a][b]; acc[a][b] = T(0); }
        run = 0;
      }
    }
  }
  double* P = it.partial + (long long)s * F * F;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int fi = ti * GR_T + ty * 4 + a;
    if (fi >= F) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int fj = tj * GR_T + tx * 4 + b;
      if (fj < F) P[(long long)fi * F + fj] = acc64[a][b] + (double)acc[a][b];
    }
  }
}

__global__ void k_gram_rows_reduce(const GramRowsItem* __restrict__ items, int splits_max, int sym,
                                   const int* __restrict__ ival) {
  const GramRowsItem it = items[blockIdx.y];
  if (it.active >= 0 && ival[it.active] == 0) return;
  int d[PEPO_MAXLEG];
  load_dims(it.x, ival, d);
  const int nl = it.x.nlegs;
  const int F = 4 * (nl > 0 ? d[nl - 1] : 1);
  long long K = 1;
  for (int i = 0; i + 1 < nl; ++i) K *= d[i];
  const int S = gram_rows_splits(K, splits_max);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < F * F; e += gridDim.x * blockDim.x) {
    int fi = e / F, fj = e - fi * F;
    int a = fi, b = fj;
    if (sym && (fi / GR_T) > (fj / GR_T)) { a = fj; b = fi; }
    double sum = 0.0;
    for (int s = 0; s < S; ++s) sum += it.partial[(long long)s * F * F + (long long)a * F + b];
    it.out[(long long)fi * it.ldo + fj] = sum;
  }
}

template <typename T>
cudaError_t launch_gram_rows(const GramRowsItem* items, int n_items, int tiles_max, int splits_max,
                             int sym, void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  dim3 grid(tiles_max * splits_max, 1, n_items);
  k_gram_rows<T><<<grid, 256, 0, s>>>(items, splits_max, sym, ptrs, ival);
  return cudaGetLastError();
}

cudaError_t launch_gram_rows_reduce(const GramRowsItem* items, int n_items, int fmax,
                                    int splits_max, int sym, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  int gx = ceil_div(fmax * fmax, 256);
  if (gx > 256) gx = 256;
  k_gram_rows_reduce<<<dim3(gx, n_items), 256, 0, s>>>(items, splits_max, sym, ival);
  return cudaGetLastError();
}


// ================================================================ reconstruct
// out[r, (c', p')] = sum_{(c,p)} in[r, (c,p)] W[(c,p), (c',p')], stored in the
// permuted output layout.  64 x 64 output tiles, K streamed 16 at a time.
constexpr int RC_T = 64;
constexpr int RC_BK = 16;

template <typename T>
__global__ void __launch_bounds__(256)
k_reconstruct(const ReconItem* __restrict__ items, int ntile_max, void* const* ptrs,
              const int* __restrict__ ival) {
  const ReconItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
  load_dims(it.in, ival, d);
  const int nl = it.in.nlegs;
  const int cut = nl - 1;
  const int n = 4 * d[cut];
  const int chin = ival[it.new_dim];
  const int np = 4 * chin;
  long long R = 1;
  for (int i = 0; i < cut; ++i) R *= d[i];
  // output strides per input leg
  int od[PEPO_MAXLEG];
  for (int i = 0; i < nl; ++i) od[i] = (i == cut) ? chin : d[i];
  long long ostride_in[PEPO_MAXLEG];   // stride of input leg i in the output
  {
    long long st = 4;
    for (int kk = nl - 1; kk >= 0; --kk) {
      int li = it.out_perm[kk];
      ostride_in[li] = st;
      st *= od[li];
    }
  }
  long long rstride[PEPO_MAXLEG];      // stride of env leg i inside the row index
  {
    long long st = 1;
    for (int i = cut - 1; i >= 0; --i) { rstride[i] = st; st *= d[i]; }
  }
  const int nct = ceil_div(np, RC_T);
  const long long nrt = (R + RC_T - 1) / RC_T;
  const long long units = nrt * nct;
  const T* __restrict__ in = static_cast<const T*>(ptrs[it.in.ref]);
  T* __restrict__ out = static_cast<T*>(ptrs[it.out_ref]);
  __shared__ __align__(16) T As[RC_BK][RC_T + 4];
  __shared__ __align__(16) T Ws[RC_BK][RC_T];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const long long rt = u / nct;
    const int ct = (int)(u - rt * nct);
    const long long r0 = rt * RC_T;
    const int c0 = ct * RC_T;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int kb = 0; kb < n; kb += RC_BK) {
      for (int e = threadIdx.x; e < RC_BK * RC_T; e += blockDim.x) {
        // A tile: rows r0.., k kb..  (read rows contiguously along k)
        int rr = e / RC_BK, kk = e - rr * RC_BK;
        long long r = r0 + rr;
        int kx = kb + kk;
        As[kk][rr] = (r < R && kx < n) ? in[r * n + kx] : T(0);
        int kk2 = e / RC_T, cc = e - kk2 * RC_T;
        int ky = kb + kk2, cy = c0 + cc;
        Ws[kk2][cc] = (ky < n && cy < np) ? (T)it.W[(long long)ky * it.ldw + cy] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < RC_BK; ++kk) {
        T xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = As[kk][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Ws[kk][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      long long r = r0 + ty * 4 + a;
      if (r >= R) continue;
      long long base = 0, rem = r;
      for (int i = 0; i < cut; ++i) {
        long long idx = rem / rstride[i];
        rem -= idx * rstride[i];
        base += idx * ostride_in[i];
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int c = c0 + tx * 4 + b;
        if (c >= np) continue;
        int cn = c >> 2, p = c & 3;
        out[base + cn * ostride_in[cut] + p] = acc[a][b];
      }
    }
  }
}

template <typename T>
cudaError_t launch_reconstruct(const ReconItem* items, int n_items, int grid_x, int ntile_max,
                               void* const* ptrs, const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_reconstruct<T><<<dim3(grid_x, n_items), 256, 0, s>>>(items, ntile_max, ptrs, ival);
  return cudaGetLastError();
}

// ========================================================= vector contraction
template <typename T>
__global__ void k_vec_contract(const VecItem* __restrict__ items, void* const* ptrs,
                               const int* __restrict__ ival) {
  const VecItem it = items[blockIdx.y];
  int d[PEPO_MAXLEG];
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < it.ndims) ? ival[it.dim[k]] : 1;
  const int k = it.leg;
  const int J = k >= 0 ? d[k] : 1;
  long long O = 1, Q = 1;
  for (int i = 0; i < k; ++i) O *= d[i];
  for (int i = k + 1; i < it.ndims; ++i) Q *= d[i];
  const T* site = it.in_ref >= 0 ? static_cast<const T*>(ptrs[it.in_ref]) : nullptr;
  if (k < 0) {  // no contraction: copy (the pinned slice of a one-leg site)
    long long n = 1;
    for (int i = 0; i < it.ndims; ++i) n *= d[i];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
      it.out[e] = site ? (double)site[e * 4 + it.pin] : it.in_d[e];
    return;
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < O * Q;
       e += (long long)gridDim.x * blockDim.x) {
    long long o = e / Q, q = e - o * Q;
    double sum = 0.0;
    for (int j = 0; j < J; ++j) {
      long long idx = (o * J + j) * Q + q;
      double x = site ? (double)site[idx * 4 + it.pin] : it.in_d[idx];
      sum = fma(x, it.v[j], sum);
    }
    it.out[e] = sum;
  }
}

template <typename T>
cudaError_t launch_vec_contract(const VecItem* items, int n_items, int grid_x, void* const* ptrs,
                                const int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_vec_contract<T><<<dim3(grid_x, n_items), 256, 0, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}

// ============================================================ instantiations
#define PEPO_INST(T)                                                                              \
  template cudaError_t launch_copy<T>(const TView*, const int*, int, int, void* const*,           \
                                      const int*, cudaStream_t);                                  \
  template cudaError_t launch_gram_rows<T>(const GramRowsItem*, int, int, int, int, void* const*, \
                                           const int*, cudaStream_t);                             \
  template cudaError_t launch_reconstruct<T>(const ReconItem*, int, int, int, void* const*,       \
                                             const int*, cudaStream_t);                           \
  template cudaError_t launch_vec_contract<T>(const VecItem*, int, int, void* const*, const int*, \
                                              cudaStream_t);
PEPO_INST(float)
PEPO_INST(double)

}  // namespace pepo
