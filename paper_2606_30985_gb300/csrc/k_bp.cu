// Belief propagation bookkeeping, the Bethe value, gate tables and init.
//
//   k_bp_finish    double-layer message (Eq. 13): symmetrise, unit trace,
//                  damping (Eq. 19), delta = max |diag change| (Eq. 14)
//   k_sl_init      single-layer start m = sqrt(diag M), unit norm
//   k_sl_finish    single-layer message: unit 2-norm, sign aligned with the
//                  previous iterate, damping, delta = max |change|
//   k_site_scalars vs_v and f_v of Eq. 7 / Table 1 (Bethe norm)
//   k_edge_scalars Z_e (Eq. 8) and its double-layer analogue
//   k_bethe        log-space sum with explicit signs (Eq. 9)
//   k_gates        Pauli transfer matrices of the gates (Sec. 2.3, real
//                  orthogonal), site gates folded into bond gates, and the
//                  operator-Schmidt factors used by the bond core
//   k_init_state   the initial network of Sec. 2.3 / Fig. 1
#include "bp.h"

namespace pepo {

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// blockDim.x == 256 in every kernel below that reduces
__device__ inline double bsum(double v, double* red) {
  v = warp_sum_d(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  __syncthreads();
  return t;
}
__device__ inline double bmax(double v, double* red) {
  v = warp_max_d(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
  __syncthreads();
  return t;
}

// non-negative doubles order like their bit patterns
__device__ inline void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ================================================================ BP finish
__global__ void k_bp_finish(const MsgItem* __restrict__ items, const int* ival, const int* active,
                            unsigned long long* delta, int* flags) {
  const MsgItem it = items[blockIdx.x];
  if (active && !active[it.inst]) return;   // converged instance of a batch: keep its messages
  const int n = ival[it.chi_idx];
  const int chimax = it.ld;
  const double alpha = it.alpha;
  __shared__ double red[8];
  double tr = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tr += it.hat[i * chimax + i];
  tr = bsum(tr, red);
  if (!(tr > 0.0) || !isfinite(tr)) {
    if (threadIdx.x == 0) atomicOr(&flags[it.inst], 2);
    return;
  }
  const double inv = 1.0 / tr;
  double dmax = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    double h = 0.5 * (it.hat[i * chimax + j] + it.hat[j * chimax + i]) * inv;
    double old = it.msg[i * chimax + j];
    double nw = (1.0 - alpha) * old + alpha * h;
    if (i == j) dmax = fmax(dmax, fabs(nw - old));
    it.msg[i * chimax + j] = nw;
  }
  dmax = bmax(dmax, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&delta[it.inst], dmax);
}

cudaError_t launch_bp_finish(const MsgItem* items, int n, const int* ival, const int* active,
                             unsigned long long* delta, int* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_bp_finish<<<n, 256, 0, s>>>(items, ival, active, delta, flags);
  return cudaGetLastError();
}

// ============================================================ single layer
__global__ void k_sl_init(const MsgItem* __restrict__ items, const int* ival) {
  const MsgItem it = items[blockIdx.x];
  const int n = ival[it.chi_idx];
  const int chimax = it.ld;
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = fmax(it.msg[i * chimax + i], 0.0);
    s += d;
  }
  s = bsum(s, red);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  for (int i = threadIdx.x; i < chimax; i += blockDim.x)
    it.vec[i] = (i < n) ? sqrt(fmax(it.msg[i * chimax + i], 0.0)) * inv : 0.0;
}

__global__ void k_sl_finish(const MsgItem* __restrict__ items, const int* ival, const int* active,
                            unsigned long long* delta) {
  const MsgItem it = items[blockIdx.x];
  if (active && !active[it.inst]) return;
  const int n = ival[it.chi_idx];
  const double alpha = it.alpha;
  __shared__ double red[8];
  double nn = 0.0, dot = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double h = it.vhat[i];
    nn += h * h;
    dot += h * it.vec[i];
  }
  nn = bsum(nn, red);
  dot = bsum(dot, red);
  double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  if (dot < 0.0) sc = -sc;
  double dmax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double old = it.vec[i];
    double nw = (1.0 - alpha) * old + alpha * it.vhat[i] * sc;
    dmax = fmax(dmax, fabs(nw - old));
    it.vec[i] = nw;
  }
  dmax = bmax(dmax, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&delta[it.inst], dmax);
}

cudaError_t launch_sl_init(const MsgItem* items, int n, const int* ival, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_sl_init<<<n, 256, 0, s>>>(items, ival);
  return cudaGetLastError();
}
cudaError_t launch_sl_finish(const MsgItem* items, int n, const int* ival, const int* active,
                             unsigned long long* delta, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_sl_finish<<<n, 256, 0, s>>>(items, ival, active, delta);
  return cudaGetLastError();
}

// ================================================================ scalars
__global__ void k_site_scalars(const SiteScalarItem* __restrict__ items, const int* ival) {
  const SiteScalarItem it = items[blockIdx.x];
  const int n = ival[it.chi_idx];
  const int chimax = it.ld;
  __shared__ double red[8];
  double f = 0.0, v = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    f += it.hat[i * chimax + j] * it.msg_in[i * chimax + j];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += it.vhat[i] * it.vec_in[i];
  f = bsum(f, red);
  v = bsum(v, red);
  if (threadIdx.x == 0) { *it.fv = f; *it.vs = v; }
}

__global__ void k_edge_scalars(const EdgeItem* __restrict__ items, const int* ival) {
  const EdgeItem it = items[blockIdx.x];
  const int n = ival[it.chi_idx];
  const int chimax = it.ld;
  __shared__ double red[8];
  double z2 = 0.0, z = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, j = e - i * n;
    z2 += it.m12[i * chimax + j] * it.m21[i * chimax + j];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) z += it.v12[i] * it.v21[i];
  z2 = bsum(z2, red);
  z = bsum(z, red);
  if (threadIdx.x == 0) { *it.ze = z; *it.z2e = z2; }
}

// ======================================================= Pauli weights
// Zero the outputs, then each block of grid.x sums its slice of one item's
// squares per Pauli index (the index is the innermost one) and adds them in.
__global__ void k_pauli_zero(const PauliWItem* __restrict__ items) {
  if (threadIdx.x < 4) items[blockIdx.x].out[threadIdx.x] = 0.0;
}

template <typename T>
__global__ void k_pauli_weights(const PauliWItem* __restrict__ items, void* const* ptrs, const int* ival) {
  const PauliWItem it = items[blockIdx.y];
  long long n = 4;
  for (int k = 0; k < it.x.nlegs; ++k) n *= ival[it.x.dim[k]];
  const T* x = static_cast<const T*>(ptrs[it.x.ref]);
  // each thread visits whole groups of 4 (one J), so its p-th partial is Pauli p
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long groups = n / 4;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double v = (double)x[g * 4 + q];
      acc[q] = fma(v, v, acc[q]);
    }
  }
  __shared__ double red[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double t = bsum(acc[q], red);
    if (threadIdx.x == 0) atomicAdd(&it.out[q], t);
  }
}

template <typename T>
cudaError_t launch_pauli_weights(const PauliWItem* items, int n, void* const* ptrs, const int* ival,
                                 cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_pauli_zero<<<n, 32, 0, s>>>(items);
  k_pauli_weights<T><<<dim3(64, n), 256, 0, s>>>(items, ptrs, ival);
  return cudaGetLastError();
}
template cudaError_t launch_pauli_weights<float>(const PauliWItem*, int, void* const*, const int*, cudaStream_t);
template cudaError_t launch_pauli_weights<double>(const PauliWItem*, int, void* const*, const int*, cudaStream_t);

cudaError_t launch_site_scalars(const SiteScalarItem* items, int n, const int* ival, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_site_scalars<<<n, 256, 0, s>>>(items, ival);
  return cudaGetLastError();
}
cudaError_t launch_edge_scalars(const EdgeItem* items, int n, const int* ival, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_edge_scalars<<<n, 256, 0, s>>>(items, ival);
  return cudaGetLastError();
}

// ================================================================== Bethe
// FP64 log-space sum with sign parity (Eq. 9); one block per instance.
__global__ void k_bethe(const BetheItem* __restrict__ items) {
  const BetheItem it = items[blockIdx.x];
  __shared__ double red[8];
  double lc = 0.0, ln = 0.0, neg = 0.0, zero = 0.0;
  for (int v = threadIdx.x; v < it.nsites; v += blockDim.x) {
    double x = it.vs[v];
    if (x == 0.0) zero += 1.0; else { lc += log(fabs(x)); if (x < 0.0) neg += 1.0; }
    lc += it.sigma[v];
    ln += log(it.fv[v]) + 2.0 * it.sigma[v];
  }
  for (int b = threadIdx.x; b < it.nbonds; b += blockDim.x) {
    double z = it.ze[b];
    if (z == 0.0) zero += 1.0; else { lc -= log(fabs(z)); if (z < 0.0) neg += 1.0; }
    ln -= log(it.z2e[b]);
  }
  lc = bsum(lc, red);
  ln = bsum(ln, red);
  neg = bsum(neg, red);
  zero = bsum(zero, red);
  if (threadIdx.x == 0) {
    const double sign = (((long long)llround(neg)) & 1) ? -1.0 : 1.0;
    double C = 0.0, Cp = 0.0;
    if (zero == 0.0) {
      C = sign * exp(lc - 0.5 * ln);
      Cp = sign * exp(lc);
    }
    it.out[0] = C;
    it.out[1] = Cp;
    it.out[2] = lc;
    it.out[3] = sign;
    it.out[4] = ln;
    it.out[5] = zero;
  }
}

cudaError_t launch_bethe(const BetheItem* items, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_bethe<<<n, 256, 0, s>>>(items);
  return cudaGetLastError();
}

// ============================================================ gate tables
struct cplx { double re, im; };
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ inline cplx cconj(cplx a) { return {a.re, -a.im}; }

// Pauli p (0 I, 1 X, 2 Y, 3 Z) entry (r, c)
__device__ inline cplx pauli(int p, int r, int c) {
  switch (p) {
    case 0: return {r == c ? 1.0 : 0.0, 0.0};
    case 1: return {r != c ? 1.0 : 0.0, 0.0};
    case 2: return r == c ? cplx{0.0, 0.0} : (r == 0 ? cplx{0.0, -1.0} : cplx{0.0, 1.0});
    default: return {r == c ? (r == 0 ? 1.0 : -1.0) : 0.0, 0.0};
  }
}

// single-qubit PTM S[a][b] = Re Tr(P_a g^dag P_b g) / 2, g = cos(phi) I - i sin(phi) Q
__device__ void ptm1(int Q, double phi, double* S) {
  cplx g[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      cplx q = pauli(Q, r, c);
      g[r][c] = {(r == c ? cos(phi) : 0.0) + sin(phi) * q.im, -sin(phi) * q.re};
    }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      // Tr(P_a g^dag P_b g) = sum P_a[i][j] conj(g[k][j]) P_b[k][l] g[l][i]
      cplx t = {0.0, 0.0};
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int k = 0; k < 2; ++k)
            for (int l = 0; l < 2; ++l)
              t = cadd(t, cmul(cmul(pauli(a, i, j), cconj(g[k][j])), cmul(pauli(b, k, l), g[l][i])));
      S[a * 4 + b] = 0.5 * t.re;
    }
}

// two-qubit PTM of exp(-i theta P(x)P), index (p1, p2) -> p1 * 4 + p2
__device__ void ptm2(int P, double theta, double* G) {
  // g = cos I - i sin P(x)P (4 x 4), basis index s1 * 2 + s2
  cplx g[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      cplx pp = cmul(pauli(P, r >> 1, c >> 1), pauli(P, r & 1, c & 1));
      g[r][c] = {(r == c ? cos(theta) : 0.0) + sin(theta) * pp.im, -sin(theta) * pp.re};
    }
  for (int a = 0; a < 16; ++a)
    for (int b = 0; b < 16; ++b) {
      cplx t = {0.0, 0.0};
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          cplx pa = cmul(pauli(a >> 2, i >> 1, j >> 1), pauli(a & 3, i & 1, j & 1));
          if (pa.re == 0.0 && pa.im == 0.0) continue;
          for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l) {
              cplx pb = cmul(pauli(b >> 2, k >> 1, l >> 1), pauli(b & 3, k & 1, l & 1));
              if (pb.re == 0.0 && pb.im == 0.0) continue;
              t = cadd(t, cmul(cmul(pa, cconj(g[k][j])), cmul(pb, g[l][i])));
            }
        }
      G[a * 16 + b] = 0.25 * t.re;
    }
}

__global__ void k_gates(const GateItem* __restrict__ items) {
  const GateItem it = items[blockIdx.x];
  if (threadIdx.x != 0) return;
  const int P = it.gateset == 0 ? 3 : 1;   // bond Pauli
  const int Q = it.gateset == 0 ? 1 : 3;   // site Pauli
  double G[256], S[16], T[256];
  ptm2(P, it.theta, G);
  ptm1(Q, it.phi, S);
  // G' = (Post1 (x) Post2) G (Pre1 (x) Pre2)
  for (int side = 0; side < 2; ++side) {
    const int f1 = side == 0 ? it.pre1 : it.post1;
    const int f2 = side == 0 ? it.pre2 : it.post2;
    if (!f1 && !f2) continue;
    for (int a = 0; a < 16; ++a)
      for (int b = 0; b < 16; ++b) {
        double x = 0.0;
        for (int c = 0; c < 16; ++c) {
          // K[(c1,c2),(b1,b2)] or K[(a1,a2),(c1,c2)] with K = S1 (x) S2
          int r = side == 0 ? c : a, q = side == 0 ? b : c;
          double k1 = f1 ? S[(r >> 2) * 4 + (q >> 2)] : ((r >> 2) == (q >> 2) ? 1.0 : 0.0);
          double k2 = f2 ? S[(r & 3) * 4 + (q & 3)] : ((r & 3) == (q & 3) ? 1.0 : 0.0);
          double kv = k1 * k2;
          x += side == 0 ? G[a * 16 + c] * kv : kv * G[c * 16 + b];
        }
        T[a * 16 + b] = x;
      }
    for (int e = 0; e < 256; ++e) G[e] = T[e];
  }
  for (int e = 0; e < 256; ++e) it.ptm[e] = G[e];
  // reshuffle Gr[(p1',p1),(p2',p2)] = G[(p1',p2'),(p1,p2)]; Jacobi SVD on its columns
  double A[256], V[256];
  for (int r = 0; r < 16; ++r)
    for (int c = 0; c < 16; ++c) {
      int p1p = r >> 2, p1 = r & 3, p2p = c >> 2, p2 = c & 3;
      A[c * 16 + r] = G[(p1p * 4 + p2p) * 16 + p1 * 4 + p2];   // column-major
      V[c * 16 + r] = (r == c) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rot = 0;
    for (int p = 0; p < 15; ++p)
      for (int q = p + 1; q < 16; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int i = 0; i < 16; ++i) {
          al += A[p * 16 + i] * A[p * 16 + i];
          be += A[q * 16 + i] * A[q * 16 + i];
          ga += A[p * 16 + i] * A[q * 16 + i];
        }
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        rot = 1;
        double zeta = (be - al) / (2 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
        double c = 1 / sqrt(1 + t * t), s = c * t;
        for (int i = 0; i < 16; ++i) {
          double x = A[p * 16 + i], y = A[q * 16 + i];
          A[p * 16 + i] = c * x - s * y;
          A[q * 16 + i] = s * x + c * y;
          x = V[p * 16 + i]; y = V[q * 16 + i];
          V[p * 16 + i] = c * x - s * y;
          V[q * 16 + i] = s * x + c * y;
        }
      }
    if (!rot) break;
  }
  double sv[16];
  int ord[16];
  for (int j = 0; j < 16; ++j) {
    double s = 0;
    for (int i = 0; i < 16; ++i) s += A[j * 16 + i] * A[j * 16 + i];
    sv[j] = sqrt(s);
    ord[j] = j;
  }
  for (int i = 0; i < 16; ++i)
    for (int j = i + 1; j < 16; ++j)
      if (sv[ord[j]] > sv[ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
  int rank = 0;
  for (int i = 0; i < 16; ++i) if (sv[ord[i]] > 1e-12 * sv[ord[0]]) ++rank;
  if (rank > PEPO_RG) { atomicOr(it.flags, 8); rank = PEPO_RG; }
  // Gr = sum_k s_k u_k v_k^T with u_k = A col / s_k, v_k = V col
  for (int k = 0; k < PEPO_RG; ++k) {
    int j = ord[k];
    double s = sv[j];
    double rs = sqrt(s);
    for (int i = 0; i < 16; ++i) {
      it.FA[k * 16 + i] = (k < rank) ? A[j * 16 + i] / s * rs : 0.0;   // i = p1' * 4 + p1
      it.FB[k * 16 + i] = (k < rank) ? V[j * 16 + i] * rs : 0.0;       // i = p2' * 4 + p2
    }
  }
  *it.rank = rank;
}

cudaError_t launch_gates(const GateItem* items, int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_gates<<<n, 32, 0, s>>>(items);
  return cudaGetLastError();
}

}  // namespace pepo

namespace pepo {
__global__ void k_commit(const int* pairs, int npairs, const int* moves, int nmoves, void** ptrs,
                         int* ival) {
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
    int a = pairs[2 * i], b = pairs[2 * i + 1];
    void* t = ptrs[a];
    ptrs[a] = ptrs[b];
    ptrs[b] = t;
  }
  for (int i = threadIdx.x; i < nmoves; i += blockDim.x) ival[moves[2 * i]] = ival[moves[2 * i + 1]];
}

cudaError_t launch_commit(const int* pairs, int npairs, const int* moves, int nmoves, void** ptrs,
                          int* ival, cudaStream_t s) {
  if (npairs == 0 && nmoves == 0) return cudaSuccess;
  k_commit<<<1, 256, 0, s>>>(pairs, npairs, moves, nmoves, ptrs, ival);
  return cudaGetLastError();
}
}  // namespace pepo
