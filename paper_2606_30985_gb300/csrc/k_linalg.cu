// Small dense linear algebra of the bond update, FP64 unless noted.
//
//   k_env_factor   pivoted Cholesky square root L of a message M (L^T L = M):
//                  the environment square root of Sec. 2.5 step 1 (Fig. 1
//                  "pseudo_sqrt"); any factor with L^T L = M gives the same cv
//                  Gram, so no eigensolver is needed.
//   k_branch       Eq. 10 branch rule: Cholesky-QR when n > n_thr and
//                  m / n > ratio_thr, Householder otherwise (Sec. 4.2).
//   k_hh_level     Householder QR (TSQR tree, R only) of cv in its storage
//                  precision with FP64 reductions (Sec. 4.2 Householder-QR);
//                  each tree block factored in panels (compact WY).
//   k_formG / k_formB   fold the gate's operator-Schmidt factors into the
//                  R-factor: X = (F_kappa (x) 1) cv, G = X^T X or B = R-side of X.
//   k_factor       rank-revealing factor T of X: pivoted Cholesky of G
//                  (Cholesky-QR branch) or column-pivoted Householder of B.
//   k_core         per bond: R1 R2^T, one-sided Jacobi SVD, truncation
//                  (Eq. 11), lambda (Eq. 12), reconstruct matrices W1, W2
//                  (Sec. 2.5 steps 5-8 in Q-less form), messages diag(lambda).
#include "kernels.h"
#include "linalg.h"

namespace pepo {

// ------------------------------------------------------------ block helpers
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; `red` must hold blockDim.x / 32 doubles.  All threads return it.
__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Block-wide argmax over values[i] for i in [lo, hi) (hi > lo); returns the
// index (smallest index among ties), always inside [lo, hi): lo when no value
// exceeds -1 (every value NaN), where the callers' pivot test then stops.
// `ri` needs blockDim.x / 32 ints, `rv` doubles.
__device__ inline int block_argmax(const double* values, int lo, int hi, double* rv, int* ri) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double best = -1.0;
  int bi = hi;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double x = values[i];
    if (x > best || (x == best && i < bi)) { best = x; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  __syncthreads();
  if (lane == 0) { rv[w] = best; ri[w] = bi; }
  __syncthreads();
  double b = -1.0;
  int idx = hi;
  for (int i = 0; i < nw; ++i)
    if (rv[i] > b || (rv[i] == b && ri[i] < idx)) { b = rv[i]; idx = ri[i]; }
  __syncthreads();
  return idx < hi ? idx : lo;
}

// =============================================================== env factor
// Pivoted (outer-product) Cholesky of the symmetrised message in shared memory.
__global__ void __launch_bounds__(256)
k_env_factor(const EnvFactorItem* __restrict__ items, int* ival) {
  const EnvFactorItem it = items[blockIdx.x];
  const double rel = it.rel;
  const int n = ival[it.chi_idx];
  extern __shared__ __align__(16) double sm[];
  double* A = sm;                 // n x n
  double* dg = A + n * n;         // n
  int* perm = reinterpret_cast<int*>(dg + n);
  __shared__ double rv[8];
  __shared__ int ri[8];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    A[e] = 0.5 * (it.M[i * it.ld + j] + it.M[j * it.ld + i]);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
  __syncthreads();
  double d0 = 0.0;
  int rank = n;
  for (int j = 0; j < n; ++j) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = (i >= j) ? A[i * n + i] : -1.0;
    __syncthreads();
    int p = block_argmax(dg, j, n, rv, ri);
    double dp = dg[p];
    if (j == 0) d0 = dp;
    if (!(dp > rel * d0) || !(dp > 0.0)) { rank = j; break; }
    if (p != j) {  // symmetric swap of rows/cols j and p
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t = A[j * n + k]; A[j * n + k] = A[p * n + k]; A[p * n + k] = t;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double t = A[k * n + j]; A[k * n + j] = A[k * n + p]; A[k * n + p] = t;
      }
      if (threadIdx.x == 0) { int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
      __syncthreads();
    }
    const double rjj = sqrt(A[j * n + j]);
    __syncthreads();
    for (int k = j + 1 + threadIdx.x; k < n; k += blockDim.x) A[j * n + k] /= rjj;
    if (threadIdx.x == 0) A[j * n + j] = rjj;
    __syncthreads();
    const int m = n - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int a = j + 1 + e / m, b = j + 1 + e % m;
      A[a * n + b] -= A[j * n + a] * A[j * n + b];
    }
    __syncthreads();
  }
  // L[a][perm[q]] = R[a][q] (upper part), rows a < rank
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int a = e / n, q = e - a * n;
    double v = (a < rank && q >= a) ? A[a * n + q] : 0.0;
    it.L[a * it.ld + perm[q]] = v;
  }
  if (threadIdx.x == 0) ival[it.rank_idx] = rank;
}

cudaError_t launch_env_factor(const EnvFactorItem* items, int n_items, int chimax, int* ival,
                              cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(double) * ((size_t)chimax * chimax + chimax) + sizeof(int) * chimax;
  cudaError_t e = cudaFuncSetAttribute(k_env_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_env_factor<<<n_items, 256, smem, s>>>(items, ival);
  return cudaGetLastError();
}

// =================================================================== branch
__device__ inline void cv_shape(const TView& v, const int* ival, long long& m, int& n) {
  m = 1;
  for (int k = 0; k + 1 < v.nlegs; ++k) m *= ival[v.dim[k]];
  n = 4 * (v.nlegs > 0 ? ival[v.dim[v.nlegs - 1]] : 1);
}

__global__ void k_branch(const SiteFacItem* __restrict__ items, int n_items, int* ival) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  const SiteFacItem it = items[i];
  long long m;
  int n;
  cv_shape(it.cv, ival, m, n);
  ival[it.branch_idx] = (n > it.n_thr && (double)m / (double)n > it.ratio_thr) ? 1 : 0;
}

cudaError_t launch_branch(const SiteFacItem* items, int n_items, int* ival, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_branch<<<ceil_div(n_items, 128), 128, 0, s>>>(items, n_items, ival);
  return cudaGetLastError();
}

// ========================================================== Householder TSQR
// Leaf rows L = max(4n, 256).  Level 0 factors each leaf in place; level l >= 1
// gathers the R-blocks of four level-(l-1) blocks into the first one and
// factors the stack.  R replaces the top rows of the block; entries below the
// diagonal are zeroed (Q is never needed: the update is Q-less).
__host__ __device__ inline long long hh_leaf_rows(int n) { return n * 4 > 256 ? (long long)n * 4 : 256; }
constexpr int kHhThreads = 512;   // threads of a TSQR block

// Panel width of the blocked QR: the panel (L x NB) lives in shared memory.
template <typename T> struct HhPanel;
template <> struct HhPanel<float> { static constexpr int NB = 16; };
template <> struct HhPanel<double> { static constexpr int NB = 8; };

// Shared-memory plan of one TSQR block (leaf rows L): panel V (column-major,
// leading dimension L + 1 so that consecutive rows of a column and the rows
// of consecutive columns fall in different banks), per-warp partial products
// of the trailing update, W = V^T A and W2 = T^T W, V^T V and the T factor of
// the compact WY form, tau, a block-reduction scratch.
struct HhSmem {
  size_t p, red, wd, w2, vtv, tm, tau, bred, total;
  int lp;
};
template <typename T>
__host__ __device__ inline HhSmem hh_smem(long long L) {
  constexpr int NB = HhPanel<T>::NB;
  HhSmem m;
  m.lp = (int)L + 1;
  size_t o = 0;
  m.p = o;    o += sizeof(T) * (size_t)NB * m.lp;
  o = (o + 15) & ~(size_t)15;
  m.red = o;  o += sizeof(T) * (size_t)(kHhThreads / 32) * NB * 32;
  m.wd = o;   o += sizeof(double) * (size_t)NB * 32;
  m.w2 = o;   o += sizeof(T) * (size_t)NB * 32;
  o = (o + 15) & ~(size_t)15;
  m.vtv = o;  o += sizeof(double) * (size_t)NB * NB;
  m.tm = o;   o += sizeof(double) * (size_t)NB * NB;
  m.tau = o;  o += sizeof(double) * (size_t)NB;
  m.bred = o; o += sizeof(double) * (size_t)(kHhThreads / 32);
  m.total = o;
  return m;
}

__device__ inline void ld4(const float* p, float (&x)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ inline void st4(float* p, const float (&x)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ inline void ld4(const double* p, double (&x)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ inline void st4(double* p, const double (&x)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
}

// Householder QR of one TSQR block A (rows x n, row-major, n % 4 == 0, base
// 16-byte aligned) in place: R in the top rows, zeros below (Q is not kept).
// Blocked by panels of NB columns in the compact WY form H_1 ... H_nb =
// I - V T V^T: the panel is factored in shared memory, then the trailing
// columns take all nb reflections in one pass, A <- A - V (T^T (V^T A)),
// instead of one pass per reflection.  Arithmetic in T's precision (FP32
// storage: FP32 reflections, backward stable to the data's own precision),
// norms, cross-warp sums and the T factor in FP64.  512 threads.
template <typename T>
__device__ void hh_block_qr(T* A, long long rows, int n, unsigned char* smem, const HhSmem& S) {
  constexpr int NB = HhPanel<T>::NB;
  T* P = reinterpret_cast<T*>(smem + S.p);
  T* red = reinterpret_cast<T*>(smem + S.red);
  double* Wd = reinterpret_cast<double*>(smem + S.wd);
  T* W2 = reinterpret_cast<T*>(smem + S.w2);
  double* VtV = reinterpret_cast<double*>(smem + S.vtv);
  double* Tm = reinterpret_cast<double*>(smem + S.tm);
  double* tau = reinterpret_cast<double*>(smem + S.tau);
  double* bred = reinterpret_cast<double*>(smem + S.bred);
  const int lp = S.lp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarp = blockDim.x >> 5;
  const int kmax = (int)(rows < n ? rows : n);
  for (int j0 = 0; j0 < kmax; j0 += NB) {
    const int nb = kmax - j0 < NB ? kmax - j0 : NB;
    const int pr = (int)(rows - j0);
    // ---- panel rows j0.., columns j0..j0+nb-1 (zero columns beyond nb)
    for (int e = tid; e < pr * NB; e += blockDim.x) {
      const int i = e / NB, l = e - i * NB;
      P[l * lp + i] = (l < nb) ? A[(long long)(j0 + i) * n + j0 + l] : T(0);
    }
    __syncthreads();
    // ---- unblocked Householder on the panel
    for (int jj = 0; jj < nb; ++jj) {
      T* col = P + jj * lp;
      double s = 0.0;
      for (int i = jj + tid; i < pr; i += blockDim.x) {
        const double x = (double)col[i];
        s = fma(x, x, s);
      }
      s = block_sum(s, bred);
      const double alpha = (double)col[jj];
      const double normx = sqrt(s);
      double beta = alpha, tj = 0.0, v0 = 1.0;
      if (normx > 0.0) {
        beta = alpha >= 0.0 ? -normx : normx;
        v0 = alpha - beta;
        tj = (beta - alpha) / beta;
      }
      __syncthreads();
      if (normx > 0.0)
        for (int i = jj + 1 + tid; i < pr; i += blockDim.x) col[i] = (T)((double)col[i] / v0);
      if (tid == 0) {
        col[jj] = (T)beta;
        tau[jj] = tj;
      }
      __syncthreads();
      // the reflection on the panel's later columns, one warp per column
      if (tj != 0.0) {
        for (int c = jj + 1 + warp; c < nb; c += nwarp) {
          T* pc = P + c * lp;
          T acc = T(0);
          for (int i = jj + 1 + lane; i < pr; i += 32) acc += col[i] * pc[i];
          const double w = tj * (warp_sum((double)acc) + (double)pc[jj]);
          __syncwarp();
          if (lane == 0) pc[jj] = (T)((double)pc[jj] - w);
          const T wt = (T)w;
          for (int i = jj + 1 + lane; i < pr; i += 32) pc[i] -= col[i] * wt;
        }
      }
      __syncthreads();
    }
    // ---- R of the panel and zeros below it back to A; then V explicit in P
    // (unit diagonal, zeros above) for the WY products
    for (int e = tid; e < pr * nb; e += blockDim.x) {
      const int i = e / nb, l = e - i * nb;
      A[(long long)(j0 + i) * n + j0 + l] = (i <= l) ? P[l * lp + i] : T(0);
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int l = e / NB, i = e - l * NB;
      if (l < nb && i <= l && i < pr) P[l * lp + i] = (i == l) ? T(1) : T(0);
    }
    __syncthreads();
    const int c0 = j0 + nb;
    if (c0 >= n) continue;
    // ---- T factor: T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j)
    for (int q = warp; q < NB * NB; q += nwarp) {
      const int l = q / NB, j = q - l * NB;
      if (l >= j || j >= nb) continue;
      const T* vl = P + l * lp;
      const T* vj = P + j * lp;
      double acc = 0.0;
      for (int i = j + lane; i < pr; i += 32) acc = fma((double)vl[i], (double)vj[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) VtV[l * NB + j] = acc;
    }
    __syncthreads();
    if (tid == 0) {
      for (int j = 0; j < NB; ++j) {
        for (int l = 0; l < NB; ++l) Tm[l * NB + j] = 0.0;
        if (j >= nb) continue;
        Tm[j * NB + j] = tau[j];
        for (int l = 0; l < j; ++l) {
          double z = 0.0;
          for (int m = l; m < j; ++m) z += Tm[l * NB + m] * VtV[m * NB + j];
          Tm[l * NB + j] = -tau[j] * z;
        }
      }
    }
    __syncthreads();
    // ---- trailing columns in blocks of 32: 8 column quads x 64 row groups
    const int cs = c0 & ~3;
    const int kq = tid & 7, rgi = tid >> 3, nrg = blockDim.x >> 3;
    for (int cb = cs; cb < n; cb += 32) {
      const int cq = cb + 4 * kq;
      const bool colok = cq < n;
      T acc[NB][4];
#pragma unroll
      for (int l = 0; l < NB; ++l)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[l][q] = T(0);
      if (colok) {
        for (int i = rgi; i < pr; i += nrg) {
          T a[4];
          ld4(A + (long long)(j0 + i) * n + cq, a);
#pragma unroll
          for (int l = 0; l < NB; ++l) {
            const T v = P[l * lp + i];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[l][q] += v * a[q];
          }
        }
      }
      // sum over the four row groups of a warp, then over the warps
#pragma unroll
      for (int l = 0; l < NB; ++l)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T x = acc[l][q];
          x += __shfl_xor_sync(0xffffffffu, x, 8);
          x += __shfl_xor_sync(0xffffffffu, x, 16);
          acc[l][q] = x;
        }
      if (lane < 8) {
#pragma unroll
        for (int l = 0; l < NB; ++l)
#pragma unroll
          for (int q = 0; q < 4; ++q) red[(warp * NB + l) * 32 + 4 * kq + q] = acc[l][q];
      }
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int l = e >> 5, k = e & 31;
        double z = 0.0;
        for (int w = 0; w < nwarp; ++w) z += (double)red[(w * NB + l) * 32 + k];
        Wd[e] = z;
      }
      __syncthreads();
      for (int e = tid; e < NB * 32; e += blockDim.x) {
        const int l = e >> 5, k = e & 31;
        double z = 0.0;
        for (int m = 0; m <= l; ++m) z += Tm[m * NB + l] * Wd[m * 32 + k];
        // the panel's own columns (below c0, in the first block) stay as written
        W2[e] = (cb + k < c0) ? T(0) : (T)z;
      }
      __syncthreads();
      if (colok) {
        T w2[NB][4];
#pragma unroll
        for (int l = 0; l < NB; ++l)
#pragma unroll
          for (int q = 0; q < 4; ++q) w2[l][q] = W2[l * 32 + 4 * kq + q];
        for (int i = rgi; i < pr; i += nrg) {
          T* pa = A + (long long)(j0 + i) * n + cq;
          T a[4];
          ld4(pa, a);
#pragma unroll
          for (int l = 0; l < NB; ++l) {
            const T v = P[l * lp + i];
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] -= v * w2[l][q];
          }
          if (cq < c0) {
            // quad straddling the panel: keep the panel's columns untouched
            T o[4];
            ld4(pa, o);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (cq + q < c0) a[q] = o[q];
          }
          st4(pa, a);
        }
      }
      __syncthreads();
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kHhThreads)
k_hh_level(const SiteFacItem* __restrict__ items, int level, void* const* ptrs, const int* ival, int pass) {
  const SiteFacItem it = items[blockIdx.y];
  if (ival[it.branch_idx] != pass) return;
  long long m;
  int n;
  cv_shape(it.cv, ival, m, n);
  const long long L = hh_leaf_rows(n);
  long long nb0 = (m + L - 1) / L;
  // block size in rows at this level, and number of blocks
  long long span = L, nblk = nb0;
  for (int l = 0; l < level; ++l) {
    if (nblk == 1) return;        // already reduced at an earlier level
    span *= 4;
    nblk = (nblk + 3) / 4;
  }
  const long long g = blockIdx.x;
  if (g >= nblk) return;
  T* A = static_cast<T*>(ptrs[it.cv.ref]);
  extern __shared__ __align__(16) unsigned char hh_sh[];
  const HhSmem S = hh_smem<T>(L);            // within the launch's plan for nmax >= n
  T* base = A + g * span * n;
  long long rows;
  if (level == 0) {
    long long r0 = g * span;
    rows = (m - r0) < span ? (m - r0) : span;
  } else {
    // gather the R rows of the four children into the first child's area
    const long long cspan = span / 4;
    rows = 0;
    for (int c = 0; c < 4; ++c) {
      const long long cr0 = g * span + c * cspan;
      if (cr0 >= m) break;
      long long crows_full = (m - cr0) < cspan ? (m - cr0) : cspan;
      // rows of the child's R: min(rows of the child's own stack, n); the stack
      // of a child has at most min(crows_full, ...) rows, and its R at most n
      long long rr = crows_full < n ? crows_full : n;
      if (c > 0) {
        const T* src = A + cr0 * n;
        for (long long e = threadIdx.x; e < rr * n; e += blockDim.x) base[rows * n + e] = src[e];
        __syncthreads();
      }
      rows += rr;
    }
  }
  hh_block_qr<T>(base, rows, n, hh_sh, S);
}

template <typename T>
cudaError_t launch_hh_level(const SiteFacItem* items, int n_items, int level, int grid_x, int nmax,
                            void* const* ptrs, const int* ival, cudaStream_t s, int pass) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = hh_smem<T>(hh_leaf_rows(nmax)).total;
  cudaError_t e = cudaFuncSetAttribute(k_hh_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_hh_level<T><<<dim3(grid_x, n_items), kHhThreads, smem, s>>>(items, level, ptrs, ival, pass);
  return cudaGetLastError();
}

// R (top min(m, n) rows of cv after the tree) -> FP64 C buffer, rows -> kfac
// acct (2 doubles, may be null): algorithmic FLOPs and bytes of the QR of
// each factored m x n matrix (2 m n^2 - 2 n^3 / 3 for m >= n, else
// 2 m^2 n - 2 m^3 / 3; one read of the matrix), accumulated on the device
// because only the device knows which sites took this branch.
template <typename T>
__global__ void k_hh_extract(const SiteFacItem* __restrict__ items, void* const* ptrs, int* ival, int pass,
                             double* acct) {
  const SiteFacItem it = items[blockIdx.x];
  if (ival[it.branch_idx] != pass) return;
  long long m;
  int n;
  cv_shape(it.cv, ival, m, n);
  const int k = (int)(m < n ? m : n);
  if (acct && threadIdx.x == 0) {
    const double dm = (double)m, dn = (double)n;
    const double f = m >= n ? 2.0 * dm * dn * dn - 2.0 * dn * dn * dn / 3.0
                            : 2.0 * dm * dm * dn - 2.0 * dm * dm * dm / 3.0;
    atomicAdd(&acct[0], f);
    atomicAdd(&acct[1], dm * dn * (double)sizeof(T));
  }
  const T* A = static_cast<const T*>(ptrs[it.cv.ref]);
  for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
    int a = e / n, q = e - a * n;
    it.C[(long long)a * it.ldc + q] = (q >= a) ? (double)A[(long long)a * n + q] : 0.0;
  }
  if (threadIdx.x == 0) ival[it.kfac_idx] = k;
}

template <typename T>
cudaError_t launch_hh_extract(const SiteFacItem* items, int n_items, void* const* ptrs, int* ival,
                              cudaStream_t s, int pass, double* acct) {
  if (n_items == 0) return cudaSuccess;
  k_hh_extract<T><<<n_items, 256, 0, s>>>(items, ptrs, ival, pass, acct);
  return cudaGetLastError();
}

// ============================================================ formG / formB
// Cholesky branch: G[(c,k),(c',k')] = sum_{p,q} (F_k^T F_k')[p,q] C[(c,p),(c',q)].
// Householder branch: B[(a,p'),(c,k)] = sum_p F_k[p',p] R[a,(c,p)].
__global__ void k_form(const SiteFacItem* __restrict__ items, const int* ival, int only) {
  const SiteFacItem it = items[blockIdx.y];
  if (only >= 0 && ival[it.branch_idx] != only) return;
  long long m;
  int n;
  cv_shape(it.cv, ival, m, n);
  const int chic = n / 4;
  const int rg = ival[it.rg_idx];
  const int r = rg * chic;
  __shared__ double F[PEPO_RG * 16];
  __shared__ double H[PEPO_RG * PEPO_RG * 16];
  for (int e = threadIdx.x; e < rg * 16; e += blockDim.x) F[e] = it.F[e];
  __syncthreads();
  if (ival[it.branch_idx] == 1) {
    for (int e = threadIdx.x; e < rg * rg * 16; e += blockDim.x) {
      int k = e / (rg * 16), rest = e % (rg * 16);
      int k2 = rest / 16, pq = rest % 16, p = pq / 4, q = pq % 4;
      double h = 0.0;
      for (int pp = 0; pp < 4; ++pp) h += F[k * 16 + pp * 4 + p] * F[k2 * 16 + pp * 4 + q];
      H[e] = h;
    }
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)chic * chic;
         e += (long long)gridDim.x * blockDim.x) {
      int c = (int)(e / chic), c2 = (int)(e % chic);
      double Cb[16];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Cb[p * 4 + q] = it.C[(long long)(c * 4 + p) * it.ldc + c2 * 4 + q];
      for (int k = 0; k < rg; ++k)
        for (int k2 = 0; k2 < rg; ++k2) {
          const double* h = H + (k * rg + k2) * 16;
          double g = 0.0;
#pragma unroll
          for (int pq = 0; pq < 16; ++pq) g += h[pq] * Cb[pq];
          it.T[(long long)(c * rg + k) * it.ldt + c2 * rg + k2] = g;
        }
    }
  } else {
    const int k = ival[it.kfac_idx];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)k * 4 * r;
         e += (long long)gridDim.x * blockDim.x) {
      int row = (int)(e / r), col = (int)(e % r);
      int a = row / 4, pp = row % 4, c = col / rg, kk = col % rg;
      double b = 0.0;
#pragma unroll
      for (int p = 0; p < 4; ++p) b += F[kk * 16 + pp * 4 + p] * it.C[(long long)a * it.ldc + c * 4 + p];
      it.T[(long long)row * it.ldt + col] = b;
    }
  }
}

cudaError_t launch_form(const SiteFacItem* items, int n_items, int grid_x, const int* ival,
                        cudaStream_t s, int only) {
  if (n_items == 0) return cudaSuccess;
  k_form<<<dim3(grid_x, n_items), 256, 0, s>>>(items, ival, only);
  return cudaGetLastError();
}

// =================================================================== factor
// Whether the Cholesky-QR branch can be trusted with this Gram C = cv^T cv
// (n x n): its factor is only as accurate as C.  The Gram's rounding is
// relative to the norms of the columns it pairs (FP32 runs flushed into
// FP64: ~1e-8 of that scale; FP64: ~1e-14), so a column that is a linear
// combination of the others in exact arithmetic keeps a Schur complement of
// that relative size, and the Q-less update would take the noise for a
// direction (Q = cv R^-1 is then far from orthonormal).  The pivoted Cholesky
// of C (pivot values only, in precision R, in the scratch Cw) therefore
// checks every accepted pivot against the column's own diagonal: false (use
// Householder) when some pivot keeps less than `safe` of it.  Pivots below
// rel_cut of the first end the check (directions too small to matter: the
// factorisation of G cuts them as rank).  Block-uniform result.
template <typename R>
__device__ bool gram_trusted(const SiteFacItem& it, int n, R* Cw, double* dg, double safe, double rel_cut,
                             double* rv, int* ri) {
  double* od = dg + n;                       // the pivoted columns' original diagonals
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (long long)i * n);
    Cw[e] = (R)it.C[(long long)i * it.ldc + j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = od[i] = (double)Cw[(long long)i * n + i];
  __syncthreads();
  double d0 = 0.0;
  for (int j = 0; j < n; ++j) {
    const int p = block_argmax(dg, j, n, rv, ri);
    const double dp = dg[p];
    if (j == 0) d0 = dp;
    if (!(dp > rel_cut * d0) || !(dp > 0.0)) return true;
    if (!(dp >= safe * od[p])) return false;
    if (p != j) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        R t = Cw[(long long)j * n + k]; Cw[(long long)j * n + k] = Cw[(long long)p * n + k]; Cw[(long long)p * n + k] = t;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        R t = Cw[(long long)k * n + j]; Cw[(long long)k * n + j] = Cw[(long long)k * n + p]; Cw[(long long)k * n + p] = t;
      }
      if (threadIdx.x == 0) {
        double t = dg[j]; dg[j] = dg[p]; dg[p] = t;
        t = od[j]; od[j] = od[p]; od[p] = t;
      }
      __syncthreads();
    }
    const R rjj = sqrt(Cw[(long long)j * n + j]);
    __syncthreads();
    for (int k = j + 1 + threadIdx.x; k < n; k += blockDim.x) Cw[(long long)j * n + k] /= rjj;
    __syncthreads();
    const int mm = n - j - 1;
    for (long long e = threadIdx.x; e < (long long)mm * mm; e += blockDim.x) {
      const int a = j + 1 + (int)(e / mm), b = j + 1 + (int)(e % mm);
      Cw[(long long)a * n + b] -= Cw[(long long)j * n + a] * Cw[(long long)j * n + b];
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) dg[i] = (double)Cw[(long long)i * n + i];
    __syncthreads();
  }
  return true;
}

// Cholesky branch: pivoted Cholesky of G (r x r, in place, row-major).
// Householder branch: column-pivoted Householder QR of B (4k x r, in place).
// Output: T (rank x r upper trapezoidal, pivoted column order) in place,
// perm[q] = original column of pivoted column q, rank -> ival.
// A Cholesky-branch site whose Gram fails gram_trusted is marked branch 2 and
// left for the Householder pass that follows (only = 2 runs that pass only).
__global__ void __launch_bounds__(512)
k_factor(const SiteFacItem* __restrict__ items, int* ival, int only, unsigned long long* qcount) {
  const SiteFacItem it = items[blockIdx.x];
  if (only >= 0 && ival[it.branch_idx] != only) return;
  if (qcount && threadIdx.x == 0 && ival[it.branch_idx] == 0) atomicAdd(&qcount[0], 1ull);
  long long m;
  int n;
  cv_shape(it.cv, ival, m, n);
  const int chic = n / 4;
  const int rg = ival[it.rg_idx];
  const int r = rg * chic;
  double* A = it.T;
  const int ld = it.ldt;
  extern __shared__ __align__(16) double sh[];
  double* dg = sh;               // r: Schur diagonal / column norms^2
  double* v = dg + r;            // 4k: Householder vector
  double* w = v + 4 * n;         // r
  int* perm = it.perm;
  __shared__ double rv[16];
  __shared__ int ri[16];
  __shared__ double red[16];
  if (ival[it.branch_idx] == 1) {
    // the scratch after G (r x ld) holds the copy of C; v (4n doubles) the
    // pivots and the original diagonals
    double* scratch = A + (long long)ld * ld;
    const bool ok = it.rel_safe >= 1e-6
                        ? gram_trusted<float>(it, n, reinterpret_cast<float*>(scratch), v, it.rel_safe, it.rel, rv, ri)
                        : gram_trusted<double>(it, n, scratch, v, it.rel_safe, it.rel, rv, ri);
    if (threadIdx.x == 0 && qcount) atomicAdd(&qcount[ok ? 1 : 2], 1ull);
    if (!ok) {
      if (threadIdx.x == 0) ival[it.branch_idx] = 2;
      return;
    }
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) perm[i] = i;
  int rank = 0;
  if (ival[it.branch_idx] == 1) {
    for (int i = threadIdx.x; i < r; i += blockDim.x) dg[i] = A[(long long)i * ld + i];
    __syncthreads();
    double d0 = 0.0;
    rank = r;
    for (int j = 0; j < r; ++j) {
      int p = block_argmax(dg, j, r, rv, ri);
      double dp = dg[p];
      if (j == 0) d0 = dp;
      if (!(dp > it.rel * d0) || !(dp > 0.0)) { rank = j; break; }
      if (p != j) {
        for (int k = threadIdx.x; k < r; k += blockDim.x) {
          double t = A[(long long)j * ld + k]; A[(long long)j * ld + k] = A[(long long)p * ld + k];
          A[(long long)p * ld + k] = t;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < r; k += blockDim.x) {
          double t = A[(long long)k * ld + j]; A[(long long)k * ld + j] = A[(long long)k * ld + p];
          A[(long long)k * ld + p] = t;
        }
        if (threadIdx.x == 0) {
          int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
          double td = dg[j]; dg[j] = dg[p]; dg[p] = td;
        }
        __syncthreads();
      }
      const double rjj = sqrt(A[(long long)j * ld + j]);
      __syncthreads();
      for (int k = j + 1 + threadIdx.x; k < r; k += blockDim.x) A[(long long)j * ld + k] /= rjj;
      if (threadIdx.x == 0) A[(long long)j * ld + j] = rjj;
      __syncthreads();
      const int mm = r - j - 1;
      for (long long e = threadIdx.x; e < (long long)mm * mm; e += blockDim.x) {
        int a = j + 1 + (int)(e / mm), b = j + 1 + (int)(e % mm);
        A[(long long)a * ld + b] -= A[(long long)j * ld + a] * A[(long long)j * ld + b];
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) dg[i] = A[(long long)i * ld + i];
      __syncthreads();
    }
  } else {
    const int M = 4 * ival[it.kfac_idx];
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < M; ++i) { double x = A[(long long)i * ld + k]; s = fma(x, x, s); }
      dg[k] = s;
      w[k] = s;   // reference norms for the downdate safeguard
    }
    __syncthreads();
    double n0 = 0.0;
    const int kmax = M < r ? M : r;
    rank = kmax;
    for (int j = 0; j < kmax; ++j) {
      int p = block_argmax(dg, j, r, rv, ri);
      double dp = dg[p];
      if (j == 0) n0 = dp;
      if (!(dp > it.rel * it.rel * n0) || !(dp > 0.0)) { rank = j; break; }
      if (p != j) {
        for (int i = threadIdx.x; i < M; i += blockDim.x) {
          double t = A[(long long)i * ld + j]; A[(long long)i * ld + j] = A[(long long)i * ld + p];
          A[(long long)i * ld + p] = t;
        }
        if (threadIdx.x == 0) {
          int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
          double td = dg[j]; dg[j] = dg[p]; dg[p] = td;
          td = w[j]; w[j] = w[p]; w[p] = td;
        }
        __syncthreads();
      }
      double s = 0.0;
      for (int i = j + threadIdx.x; i < M; i += blockDim.x) {
        double x = A[(long long)i * ld + j];
        s = fma(x, x, s);
      }
      s = block_sum(s, red);
      const double alpha = A[(long long)j * ld + j];
      const double normx = sqrt(s);
      const double beta = alpha >= 0.0 ? -normx : normx;
      const double v0 = alpha - beta;
      const double tau = (beta - alpha) / beta;
      for (int i = j + threadIdx.x; i < M; i += blockDim.x)
        v[i - j] = (i == j) ? 1.0 : A[(long long)i * ld + j] / v0;
      __syncthreads();
      for (int i = j + threadIdx.x; i < M; i += blockDim.x) A[(long long)i * ld + j] = (i == j) ? beta : 0.0;
      for (int k = j + 1 + threadIdx.x; k < r; k += blockDim.x) {
        double acc = 0.0;
        for (int i = j; i < M; ++i) acc = fma(v[i - j], A[(long long)i * ld + k], acc);
        const double tw = tau * acc;
        for (int i = j; i < M; ++i) A[(long long)i * ld + k] -= v[i - j] * tw;
        const double rjk = A[(long long)j * ld + k];
        double nd = dg[k] - rjk * rjk;
        if (nd < 0.05 * w[k]) {  // cancellation: recompute the trailing norm
          nd = 0.0;
          for (int i = j + 1; i < M; ++i) { double x = A[(long long)i * ld + k]; nd = fma(x, x, nd); }
          w[k] = nd;
        }
        dg[k] = nd;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) ival[it.rank_idx] = rank;
}

cudaError_t launch_factor(const SiteFacItem* items, int n_items, int rmax, int nmax, int* ival,
                          cudaStream_t s, int only, unsigned long long* qcount) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(double) * ((size_t)2 * rmax + 4 * nmax);
  cudaError_t e = cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<<<n_items, 512, smem, s>>>(items, ival, only, qcount);
  return cudaGetLastError();
}

// ===================================================================== core
// Sort key of a singular-value estimate (a norm, >= 0): NaN ranks last, so
// the ranks of any input form a permutation (every order[] slot written once).
__device__ inline double rank_key(double x) { return x == x ? x : -1.0; }

// One-sided Jacobi (Hestenes) on the columns of A (m x n, column-major, m >= n),
// accumulating V (n x n, column-major).  Returns the sweep count; sets
// *capped when the sweep budget ran out.  abs_rel > 0 also skips a pair whose
// coupling |a_p . a_q| is below abs_rel ||A||_F^2: such a pair moves no
// singular value by more than that absolute amount, and without the cut the
// columns of tiny singular values (their content mostly rounding noise from
// rotations with the large ones) are chased for many sweeps without ever
// reaching relative orthogonality.
template <typename R>
__device__ int jacobi_svd(R* A, int m, int n, R* V, int max_sweeps, int* capped, double* red,
                          double abs_rel = 0.0) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // V == nullptr: rotations are not accumulated (the caller recovers the other
  // side's vectors from a copy of the input)
  if (V)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) V[e] = (e % (n + 1) == 0) ? R(1) : R(0);
  __syncthreads();
  if (n < 2) return 0;
  const int np = (n % 2) ? n + 1 : n;   // players incl. a dummy
  // orthogonality target: above the rounding noise of a length-m dot product
  // in the working precision (FP32 columns: ~sqrt(m) 6e-8 relative)
  const double tol = (sizeof(R) == 4 ? 3e-7 : 1e-15) * sqrt((double)m);
  // columns below 1e-30 (FP64) or 1e-13 (FP32) of the total squared norm are
  // numerically zero in that precision: rotating them only stirs rounding
  // noise and never converges
  double fro = 0.0;
  for (long long e = threadIdx.x; e < (long long)m * n; e += blockDim.x) fro = fma((double)A[e], (double)A[e], fro);
  {
    fro = warp_sum(fro);
    __shared__ double fr[32];
    if (lane == 0) fr[wid] = fro;
    __syncthreads();
    fro = 0.0;
    for (int i = 0; i < nw; ++i) fro += fr[i];
    __syncthreads();
  }
  const double negligible = (sizeof(R) == 4 ? 1e-13 : 1e-30) * fro;
  const R abs_cut = (R)(abs_rel * fro);
  __shared__ int sh_rot;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) sh_rot = 0;
    __syncthreads();
    int rotated = 0;
    for (int round = 0; round < np - 1; ++round) {
      for (int pi = wid; pi < np / 2; pi += nw) {
        int a, b;
        if (pi == 0) { a = np - 1; b = round; }
        else { a = (round + pi) % (np - 1); b = (round - pi + np - 1) % (np - 1); }
        if (a >= n || b >= n) continue;
        int p = a < b ? a : b, q = a < b ? b : a;
        R* Ap = A + (long long)p * m;
        R* Aq = A + (long long)q * m;
        R al = 0, be = 0, ga = 0;
        for (int i = lane; i < m; i += 32) {
          R x = Ap[i], y = Aq[i];
          al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        // rotation parameters in the working precision (FP64 division and
        // square root are slow on this part; FP32 columns need no more)
        if (ga != R(0) && al > (R)negligible && be > (R)negligible &&
            fabs(ga) > (R)tol * sqrt(al * be) && fabs(ga) > abs_cut) {
          rotated = 1;
          const R zeta = (be - al) / (R(2) * ga);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          const R c = R(1) / sqrt(R(1) + t * t), s = c * t;
          for (int i = lane; i < m; i += 32) {
            R x = Ap[i], y = Aq[i];
            Ap[i] = c * x - s * y;
            Aq[i] = s * x + c * y;
          }
          if (V) {
            R* Vp = V + (long long)p * n;
            R* Vq = V + (long long)q * n;
            for (int i = lane; i < n; i += 32) {
              R x = Vp[i], y = Vq[i];
              Vp[i] = c * x - s * y;
              Vq[i] = s * x + c * y;
            }
          }
        }
      }
      __syncthreads();
    }
    if (rotated) atomicOr(&sh_rot, 1);
    __syncthreads();
    if (sh_rot == 0) break;
    __syncthreads();
  }
  if (sweep >= max_sweeps && threadIdx.x == 0) *capped = 1;
  (void)red;
  return sweep;
}

__global__ void __launch_bounds__(1024)
k_core(const CoreItem* __restrict__ items, int* ival, int* flags_base) {
  const CoreItem it = items[blockIdx.x];
  int* flags = flags_base + it.inst;
  const int chic = ival[it.chi_idx];
  const int rg = ival[it.rg_idx];
  const int r = rg * chic;
  const int n = 4 * chic;
  const int k1 = ival[it.rank1_idx], k2 = ival[it.rank2_idx];
  const int rmax = it.rmax;
  double* R2o = it.work;                          // k2 x r, original column order
  double* Tc = it.work + (long long)rmax * rmax;  // column-major working matrix
  double* V = Tc + (long long)rmax * rmax;        // Jacobi right vectors
  double* Z = V + (long long)rmax * rmax;         // triangular-solve results
  __shared__ double red[32];
  __shared__ double sv[2 * 4 * 128 + 8];
  __shared__ int order[4 * 128];
  __shared__ int sh_capped;
  if (threadIdx.x == 0) sh_capped = 0;
  // R2 in original column order
  for (long long e = threadIdx.x; e < (long long)k2 * r; e += blockDim.x) {
    int b = (int)(e / r), q = (int)(e % r);
    double x = (q >= b) ? it.T2[(long long)b * it.ldt2 + q] : 0.0;
    R2o[(long long)b * r + it.perm2[q]] = x;
  }
  __syncthreads();
  // Tcore = R1 R2^T (k1 x k2).  Work on the orientation with m >= n columns.
  const bool tr = k1 < k2;             // if so, decompose Tcore^T
  const int M = tr ? k2 : k1, N = tr ? k1 : k2;
  for (long long e = threadIdx.x; e < (long long)k1 * k2; e += blockDim.x) {
    int a = (int)(e / k2), b = (int)(e % k2);
    double s = 0.0;
    const double* t1 = it.T1 + (long long)a * it.ldt1;
    const double* r2 = R2o + (long long)b * r;
    for (int q = a; q < r; ++q) s = fma(t1[q], r2[it.perm1[q]], s);
    // column-major M x N storage of Tcore (or its transpose)
    if (!tr) Tc[(long long)b * M + a] = s; else Tc[(long long)a * M + b] = s;
  }
  __syncthreads();
  // copy of Tcore (the mixed path multiplies it by its FP64 subspace basis)
  for (long long e = threadIdx.x; e < (long long)M * N; e += blockDim.x) V[e] = Tc[e];
  __syncthreads();
  // columns the FP64 Jacobi below works on (all N, or the mixed path's subspace)
  int NK = N;
  __shared__ double sh_fro;
  if (it.mixed_svd) {
    // FP32 one-sided Jacobi with accumulated right vectors V32 (in the R2
    // block, free until the reconstruct step) finds the dominant right
    // singular subspace to FP32 accuracy.  Its leading NK = chimax + margin
    // directions are re-orthonormalised in FP64 (Cholesky QR; V32 itself is
    // orthogonal only to ~1e-5 after thousands of FP32 rotations) and the FP64
    // Jacobi then runs on T Q (M x NK) instead of T (M x N): the singular
    // values of T Q are those of T restricted to an exactly orthonormal basis,
    // so the kept values carry no error from V32's non-orthogonality, and the
    // FP64 work (GB300's FP64 rate is ~1/64 of its FP32 rate) drops by
    // (N / NK)^2 per sweep.  The columns are then nearly orthogonal, so few
    // FP64 sweeps follow.  Values past NK (never kept: NK > chimax) keep their
    // FP32 estimates for the diagnostic spectrum; the discarded weight of the
    // truncation uses ||T||_F^2 computed in FP64.
    float* T32 = reinterpret_cast<float*>(R2o);
    float* V32 = T32 + (long long)M * N;
    for (long long e = threadIdx.x; e < (long long)M * N; e += blockDim.x) T32[e] = (float)Tc[e];
    double f2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)M * N; e += blockDim.x) f2 = fma(Tc[e], Tc[e], f2);
    f2 = block_sum(f2, red);
    if (threadIdx.x == 0) sh_fro = f2;
    __syncthreads();
    __shared__ int sh_capped32;   // a capped FP32 pass only costs FP64 sweeps below
    if (threadIdx.x == 0) sh_capped32 = 0;
    __syncthreads();
    const int sw32 = jacobi_svd<float>(T32, M, N, V32, 60, &sh_capped32, red);
    if (threadIdx.x == 0 && it.sweeps) it.sweeps[0] = sw32;
    __syncthreads();
    // FP32 singular-value estimates (unsorted at sv[512 + j]) and their order
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double s = 0.0;
      const float* col = T32 + (long long)j * M;
      for (int i = 0; i < M; ++i) s = fma((double)col[i], (double)col[i], s);
      sv[512 + j] = sqrt(s);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      int rk = 0;
      const double kj = rank_key(sv[512 + j]);
      for (int i = 0; i < N; ++i) {
        const double ki = rank_key(sv[512 + i]);
        if (ki > kj || (ki == kj && i < j)) ++rk;
      }
      order[rk] = j;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += blockDim.x) sv[c] = sv[512 + order[c]];
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += blockDim.x) sv[512 + c] = sv[c];   // sorted FP32 values
    const int margin = it.chimax / 4 > 16 ? it.chimax / 4 : 16;
    NK = it.chimax + margin < N ? it.chimax + margin : N;
    // Q = leading NK columns of V32 in FP64 (N x NK, column-major, in Z)
    double* Qk = Z;
    for (long long e = threadIdx.x; e < (long long)N * NK; e += blockDim.x) {
      const int c = (int)(e / N), i = (int)(e - (long long)c * N);
      Qk[e] = (double)V32[(long long)order[c] * N + i];
    }
    __syncthreads();
    // Cholesky QR: G = Q^T Q = L L^T (lower triangle of G in the Tc block), Q <- Q L^-T
    double* G = Tc;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long pq = wid; pq < (long long)NK * NK; pq += nw) {
      const int a = (int)(pq / NK), b = (int)(pq - (long long)a * NK);
      if (b > a) continue;
      const double* qa = Qk + (long long)a * N;
      const double* qb = Qk + (long long)b * N;
      double acc = 0.0;
      for (int i = lane; i < N; i += 32) acc = fma(qa[i], qb[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) G[(long long)a * NK + b] = acc;
    }
    __syncthreads();
    for (int j = 0; j < NK; ++j) {
      if (threadIdx.x == 0) G[(long long)j * NK + j] = sqrt(G[(long long)j * NK + j]);
      __syncthreads();
      const double djj = G[(long long)j * NK + j];
      for (int i = j + 1 + threadIdx.x; i < NK; i += blockDim.x) G[(long long)i * NK + j] /= djj;
      __syncthreads();
      const int w = NK - j - 1;   // trailing lower triangle: rows i > j, columns j < l <= i
      for (long long e = threadIdx.x; e < (long long)w * w; e += blockDim.x) {
        const int i = j + 1 + (int)(e / w), l = j + 1 + (int)(e % w);
        if (l <= i) G[(long long)i * NK + l] -= G[(long long)i * NK + j] * G[(long long)l * NK + j];
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {   // row i of Q solves x L^T = q
      for (int c = 0; c < NK; ++c) {
        double x = Qk[(long long)c * N + i];
        const double* lc = G + (long long)c * NK;
        for (int l = 0; l < c; ++l) x -= Qk[(long long)l * N + i] * lc[l];
        Qk[(long long)c * N + i] = x / lc[c];
      }
    }
    __syncthreads();
    // Tc <- T Q (M x NK, column-major), T = the copy in V
    for (long long e = threadIdx.x; e < (long long)M * NK; e += blockDim.x) {
      const int c = (int)(e / M), i = (int)(e - (long long)c * M);
      const double* qc = Qk + (long long)c * N;
      double acc = 0.0;
      for (int k = 0; k < N; ++k) acc = fma(V[(long long)k * M + i], qc[k], acc);
      Tc[e] = acc;
    }
    __syncthreads();
  }
  {   // FP64 one-sided Jacobi on Tcore (or on its restriction T Q)
    // mixed path: the rotations W64 (NK x NK) are accumulated in the V block
    // (the copy of T is no longer needed); the right vectors are then Q W64
    // the right vectors are always accumulated (V): recovering them as
    // T^T u / s would carry the columns' absolute rounding (~1e-16 of the
    // largest) divided by s^2, which for kept values near eps_cut (1e-11 of
    // the largest) leaves nothing of the vector
    const int sw64 = jacobi_svd<double>(Tc, M, NK, V, 60, &sh_capped, red, 1e-17);
    if (threadIdx.x == 0 && it.sweeps) {
      it.sweeps[1] = sw64;
      if (!it.mixed_svd) it.sweeps[0] = 0;
    }
    __syncthreads();
    // singular values (column norms) and descending order
    for (int j = threadIdx.x; j < NK; j += blockDim.x) {
      double s = 0.0;
      const double* col = Tc + (long long)j * M;
      for (int i = 0; i < M; ++i) s = fma(col[i], col[i], s);
      sv[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NK; j += blockDim.x) {
      int rk = 0;
      const double kj = rank_key(sv[j]);
      for (int i = 0; i < NK; ++i) {
        const double ki = rank_key(sv[i]);
        if (ki > kj || (ki == kj && i < j)) ++rk;
      }
      order[rk] = j;
    }
    __syncthreads();
  }
  const double s0 = sv[order[0]];
  // truncation, Eq. 11
  __shared__ int sh_chi;
  __shared__ double sh_sum, sh_tot;
  if (threadIdx.x == 0) {
    int cnt = 0;
    double tot = 0.0;
    for (int i = 0; i < NK; ++i) {
      double s = sv[order[i]];
      tot += s * s;
      if (s >= it.eps_cut * s0 && s > 0.0) ++cnt;
    }
    if (it.mixed_svd) tot = sh_fro;
    int chi = cnt < it.chimax ? cnt : it.chimax;
    if (chi < 1) chi = 1;
    double kept = 0.0, ksum = 0.0;
    for (int i = 0; i < chi; ++i) { double s = sv[order[i]]; kept += s * s; ksum += s; }
    sh_chi = chi;
    sh_sum = ksum;
    sh_tot = tot;
    *it.disc = tot > 0.0 ? (tot - kept) / tot : 0.0;
    ival[it.new_idx] = chi;
    *it.nsv = N;
    if (!(s0 > 0.0) || !isfinite(s0)) atomicOr(flags, 2);
    if (sh_capped) atomicOr(flags, 4);
    const double nrm = sqrt(kept);
    for (int i = 0; i < it.chimax; ++i) it.lam[i] = (i < chi) ? sv[order[i]] / nrm : 0.0;
    for (int i = 0; i < N; ++i) it.svals[i] = i < NK ? sv[order[i]] : sv[512 + i];
    // stored psi = true psi * exp(-sigma); the raw sqrt(S) split gives both
    // sites half of the pair's combined scale plus the normalisation of W
    const double ls = 0.5 * log(ksum) + 0.5 * (*it.sigma1 + *it.sigma2);
    *it.sigma1 = ls;
    *it.sigma2 = ls;
  }
  __syncthreads();
  const int chi = sh_chi;
  const double inv = 1.0 / sqrt(sh_sum);
  // messages diag(lambda)
  for (int e = threadIdx.x; e < it.chimax * it.chimax; e += blockDim.x) {
    int i = e / it.chimax, j = e % it.chimax;
    double x = (i == j && i < chi) ? it.lam[i] : 0.0;
    it.msg12[e] = x;
    it.msg21[e] = x;
  }
  if (it.mixed_svd) {
    // Right (N-space) vectors of the kept pairs: v_c = Q W64 e_order[c] (N x chi,
    // row-major by N index), first into the R2 block, then into the V block
    // once W64 is consumed.  These are the Ritz vectors of the subspace, so
    // T v_c = s_c u_c holds exactly for every kept pair; recovering them as
    // T^T u_c / s_c instead would divide the subspace's FP32-level residual
    // by s_c^2 for values near the FP32 resolution (~1e-7 of the largest).
    double* Vr = R2o;
    for (long long e = threadIdx.x; e < (long long)N * chi; e += blockDim.x) {
      const int a = (int)(e / chi), c = (int)(e - (long long)a * chi);
      const double* w = V + (long long)order[c] * NK;
      double acc = 0.0;
      for (int l = 0; l < NK; ++l) acc = fma(Z[(long long)l * N + a], w[l], acc);
      Vr[e] = acc;
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)N * chi; e += blockDim.x) V[e] = Vr[e];
    __syncthreads();
  }
  // For each side: Zs = T_s11^{-1} (singular vectors of that side) sqrt(s) / sqrt(sum s)
  // side 1 vectors: left vectors of Tcore (rows of R1 space, length k1)
  // side 2 vectors: right vectors (length k2)
  for (int side = 0; side < 2; ++side) {
    const int ks = side == 0 ? k1 : k2;
    const double* Ts = side == 0 ? it.T1 : it.T2;
    const int ldts = side == 0 ? it.ldt1 : it.ldt2;
    const int* perms = side == 0 ? it.perm1 : it.perm2;
    const double* Fs = side == 0 ? it.FA : it.FB;
    double* W = side == 0 ? it.W1 : it.W2;
    // vector of side `side` for singular index c' (c' < chi): length ks
    // if (!tr): left vectors = columns of Tc / s (length M = k1), right = V (length N = k2)
    // if (tr):  left vectors = V (length N = k1), right = columns of Tc / s (length M = k2)
    const bool from_cols = (side == 0) != tr;
    for (long long e = threadIdx.x; e < (long long)ks * chi; e += blockDim.x) {
      int a = (int)(e / chi), c = (int)(e % chi);
      int j = order[c];
      double s = sv[j];
      double x;
      if (from_cols) {
        x = s > 0.0 ? Tc[(long long)j * M + a] / s : 0.0;
      } else if (it.mixed_svd) {
        x = V[(long long)a * chi + c];                  // Ritz right vector (above)
      } else {
        x = V[(long long)j * N + a];                    // accumulated right vector j (column-major N x N)
      }
      Z[(long long)a * chi + c] = x * sqrt(s) * inv;
    }
    __syncthreads();
    // back substitution with the leading ks x ks upper-triangular block of Ts
    for (int c = threadIdx.x; c < chi; c += blockDim.x) {
      for (int a = ks - 1; a >= 0; --a) {
        double x = Z[(long long)a * chi + c];
        const double* trow = Ts + (long long)a * ldts;
        for (int b = a + 1; b < ks; ++b) x -= trow[b] * Z[(long long)b * chi + c];
        Z[(long long)a * chi + c] = x / trow[a];
      }
    }
    __syncthreads();
    // Y[(c,kappa), c'] = Z[q, c'] at original column perm[q] (zero for q >= ks)
    // W[(c,p), (c',p')] = sum_kappa F_kappa[p', p] Y[(c,kappa), c']
    double* Y = R2o;   // reuse (r x chi)
    for (long long e = threadIdx.x; e < (long long)r * chi; e += blockDim.x) Y[e] = 0.0;
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)ks * chi; e += blockDim.x) {
      int q = (int)(e / chi), c = (int)(e % chi);
      Y[(long long)perms[q] * chi + c] = Z[e];
    }
    __syncthreads();
    const int np = 4 * chi;
    for (long long e = threadIdx.x; e < (long long)n * np; e += blockDim.x) {
      int row = (int)(e / np), col = (int)(e % np);
      int cc = row / 4, p = row % 4, c2 = col / 4, p2 = col % 4;
      double x = 0.0;
      for (int kk = 0; kk < rg; ++kk) x += Fs[kk * 16 + p2 * 4 + p] * Y[(long long)(cc * rg + kk) * chi + c2];
      W[(long long)row * it.ldw + col] = x;
    }
    __syncthreads();
  }
}

cudaError_t launch_core(const CoreItem* items, int n_items, int* ival, int* flags_base, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  k_core<<<n_items, 1024, 0, s>>>(items, ival, flags_base);
  return cudaGetLastError();
}

template cudaError_t launch_hh_level<float>(const SiteFacItem*, int, int, int, int, void* const*,
                                            const int*, cudaStream_t, int);
template cudaError_t launch_hh_level<double>(const SiteFacItem*, int, int, int, int, void* const*,
                                             const int*, cudaStream_t, int);
template cudaError_t launch_hh_extract<float>(const SiteFacItem*, int, void* const*, int*,
                                              cudaStream_t, int, double*);
template cudaError_t launch_hh_extract<double>(const SiteFacItem*, int, void* const*, int*,
                                               cudaStream_t, int, double*);

}  // namespace pepo

namespace pepo {
// ============================================================ message eigen
// The square roots of a message's eigenvalues scale the rotated legs (they
// are the weights of every Gram that sums over the leg) and divide the Gram
// of that leg back out, so they are floored at kSqrtEigFloor of the largest:
// an eigenvalue below 1e-12 of the largest counts as 1e-12 of it, which
// moves no message by more than that relative amount.
constexpr double kSqrtEigFloor = 1e-6;
__device__ void floor_sqrt_eigs(double* sd, int n, double* red) {
  __syncthreads();
  double m = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, sd[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
  const double lo = kSqrtEigFloor * (m > 0.0 ? m : 1.0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) sd[j] = fmax(sd[j], lo);
  __syncthreads();
}

// Vs = diag(sd) Vt: the BP rotation of a leg scaled by the square roots of
// the message's eigenvalues
__device__ void scaled_rotation(const EnvEigItem& it, int n) {
  if (!it.Vs) return;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    it.Vs[i * it.ld + j] = it.sqrtD[i] * it.Vt[i * it.ld + j];
  }
}

// M (symmetrised, PSD) -> one-sided Jacobi on its columns: M V = U S with
// S = |eigenvalues| and V the eigenvectors (U = V up to signs of numerically
// zero eigenvalues).  Outputs Vt (row i = column i of V) and sqrt(S).
__global__ void __launch_bounds__(1024)
k_env_eig(const EnvEigItem* __restrict__ items, const int* ival, int fp32) {
  const EnvEigItem it = items[blockIdx.x];
  const int n = ival[it.chi_idx];
  __shared__ double red[32];
  __shared__ int capped;
  if (threadIdx.x == 0) capped = 0;
  if (fp32) {
    // FP32-storage modes: the eigenbasis only rotates FP32 tensors, so the
    // Jacobi runs in FP32 entirely in shared memory
    extern __shared__ __align__(16) float sm32[];
    float* A = sm32;                       // n x n column-major
    float* V = sm32 + (long long)n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e - i * n;
      A[(long long)j * n + i] = (float)(0.5 * (it.M[i * it.ld + j] + it.M[j * it.ld + i]));
    }
    __syncthreads();
    jacobi_svd<float>(A, n, n, V, 60, &capped, red);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s = fma((double)A[(long long)j * n + i], (double)A[(long long)j * n + i], s);
      it.sqrtD[j] = sqrt(sqrt(s));
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e - i * n;
      it.Vt[i * it.ld + j] = (double)V[(long long)i * n + j];
    }
    floor_sqrt_eigs(it.sqrtD, n, red);
    scaled_rotation(it, n);
    return;
  }
  double* A = it.work;                      // n x n column-major
  double* V = it.work + (long long)n * n;   // n x n column-major
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;   // A column j, row i
    A[(long long)j * n + i] = 0.5 * (it.M[i * it.ld + j] + it.M[j * it.ld + i]);
  }
  __syncthreads();
  jacobi_svd<double>(A, n, n, V, 60, &capped, red);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(A[(long long)j * n + i], A[(long long)j * n + i], s);
    it.sqrtD[j] = sqrt(sqrt(s));   // sqrt of the eigenvalue |lambda_j| = ||A v_j||
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    it.Vt[i * it.ld + j] = V[(long long)i * n + j];   // row i of Vt = column i of V
  }
  floor_sqrt_eigs(it.sqrtD, n, red);
  scaled_rotation(it, n);
}

cudaError_t launch_env_eig(const EnvEigItem* items, int n_items, int chimax, int fp32, const int* ival,
                           cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = fp32 ? 2 * sizeof(float) * (size_t)chimax * chimax : 0;
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(k_env_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_env_eig<<<n_items, 1024, smem, s>>>(items, ival, fp32);
  return cudaGetLastError();
}

// out = V G V^T = Vt^T G Vt
__global__ void k_rotate_back(const RotItem* __restrict__ items, const int* ival) {
  const RotItem it = items[blockIdx.x];
  const int n = ival[it.chi_idx];
  extern __shared__ __align__(16) double sm[];
  double* T = sm;   // n x n: T = G' Vt
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    double s = 0.0;
    if (it.sd) {
      for (int k = 0; k < n; ++k) s = fma(it.G[i * it.ld + k] / it.sd[k], it.Vt[k * it.ld + j], s);
      s /= it.sd[i];
    } else {
      for (int k = 0; k < n; ++k) s = fma(it.G[i * it.ld + k], it.Vt[k * it.ld + j], s);
    }
    T[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(it.Vt[k * it.ld + i], T[k * n + j], s);
    it.out[i * it.ld + j] = s;
  }
}

cudaError_t launch_rotate_back(const RotItem* items, int n_items, int chimax, const int* ival,
                               cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  size_t smem = sizeof(double) * (size_t)chimax * chimax;
  cudaError_t e = cudaFuncSetAttribute(k_rotate_back, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_rotate_back<<<n_items, 256, smem, s>>>(items, ival);
  return cudaGetLastError();
}
}  // namespace pepo
