// Internal definitions shared by the libpepo kernels and the host driver.
//
// Device-resident sizes.  Live bond dimensions grow from 1 to chi_max during a
// run (Sec. 2.3) and are decided on the device (Eq. 11), so no kernel takes a
// live size as a launch argument: every kernel reads the sizes it needs from
// the int table `ival` through index records prepared at init.  Grids are
// sized for chi_max and surplus blocks return early, so one recorded launch
// sequence serves every step (no host synchronisation inside a step).
//
// Tensor layout.  A site tensor is stored as a dense row-major array whose
// legs follow a per-site layout order (outermost first) with the Pauli index
// (dimension 4: I, X, Y, Z) always innermost.  The host schedule keeps the leg
// cut by a site's next bond update innermost; the reconstruct kernel writes
// that layout directly (the paper's PermuteCutToLast / InversePermuteCut pair
// of Alg. 1 is fused into the reconstruct's store).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PEPO_MAXLEG 4
#define PEPO_RG 4          // operator-Schmidt rank bound of a two-site rotation gate

namespace pepo {

// A view of a tensor: `ref` indexes the device pointer table, `dim[k]` indexes
// the device int table holding the live size of layout leg k.
struct TView {
  int ref;
  int nlegs;               // 0..4 bond legs; the Pauli leg (4) is implicit
  int dim[PEPO_MAXLEG];
};

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline long long ceil_divl(long long a, long long b) { return (a + b - 1) / b; }

// Leg contraction: out[o, i, q] = sum_j A[i, j] in[o, j, q] on layout leg `leg`
// (absorb of Sec. 2.5 step 1 and the BP products of Eq. 13).
struct LegItem {
  TView in;
  int out_ref;
  int leg;
  int out_dim;             // ival index of the output size of that leg
  int a_rows;              // ival index of A's row count (== out size)
  const double* A;         // row-major, leading dimension lda
  int lda;
};

// Gram over rows: C[f, f'] = sum_k X[k, f] Y[k, f'], X, Y row-major K x F with
// F = 4 * (size of the innermost leg): the cv^T cv of Eq. 10 (Cholesky-QR).
struct GramRowsItem {
  TView x;
  int y_ref;
  int active;              // ival index of a 0/1 flag (-1: always active)
  double* partial;         // [splits][Fmax * Fmax]
  double* out;             // F x F, leading dimension ldo
  int ldo;
};

// Free-leg contraction: out[i, i'] = sum_{o,q} X[o, i, q] Y[o, i', q], free leg
// at layout position `leg` (one BP message, Eq. 13 with the Pauli leg traced).
struct GramLegItem {
  TView x;
  int y_ref;
  int leg;
  double* partial;         // [splits][chimax * chimax]
  double* out;             // chi x chi, leading dimension ldo
  int ldo;
  // optional square-root weights per layout leg (nullptr: weight 1); element
  // (.., j_u, ..) of X and Y is scaled by prod_{u != leg} sw[u][j_u] on load
  const double* sw[PEPO_MAXLEG];
};

// Eigen-decomposition of a (symmetrised) message M = V diag(D) V^T by one-sided
// Jacobi (FP64); writes Vt (row i = eigenvector i, leading dimension ld) and
// sqrt(D).  Used to rotate a site tensor into the message eigenbasis (Eq. 13).
struct EnvEigItem {
  const double* M;
  int ld;
  int chi_idx;
  double* work;            // 2 * chimax^2 doubles
  double* Vt;              // chi x chi, leading dimension ld
  double* sqrtD;           // chi
  double* Vs;              // diag(sqrtD) Vt (the rotation that also carries the weights), ld
};

// Back-rotation of one Gram of the rotated tensor: out = V G' V^T with
// G' = G / (sd sd^T) when the rotated tensor carries the square roots of the
// message eigenvalues on its legs (the Gram's weights folded into the rotation).
struct RotItem {
  const double* G;         // chi x chi, leading dimension ld
  const double* Vt;        // chi x chi, leading dimension ld
  const double* sd;        // G is scaled by sd[i] sd[i'] (undone before the rotation), or nullptr
  double* out;             // chi x chi, leading dimension ld
  int ld;
  int chi_idx;
};

// Reconstruct (Sec. 2.5 step 6, Q-less): out = in * W where `in` is viewed as
// rows x (cut, Pauli) with the cut innermost; the output leg order is out_perm
// (output leg k is input leg out_perm[k]); the cut leg gets size new_dim.
struct ReconItem {
  TView in;
  int out_ref;
  int new_dim;
  int out_perm[PEPO_MAXLEG];
  const double* W;         // n x n', row-major, leading dimension ldw
  int ldw;
  double* scale_sq;        // optional: sum of squares of the output (may be null)
  float* Wp;               // tensor-core path: W packed into swizzled B blocks (recon_packed_floats(nmax))
};

// Vector contraction of one leg of an FP64 tensor: out[o, q] = sum_j in[o, j, q] v[j].
struct VecItem {
  int in_ref;              // >= 0: site tensor (storage type) read at stride 4, offset pin
  int pin;                 // Pauli index read when in_ref >= 0
  const double* in_d;      // FP64 input when in_ref < 0
  int ndims;
  int dim[PEPO_MAXLEG];    // ival indices (layout order)
  int leg;
  const double* v;
  double* out;
};

// ------------------------------------------------------------ linear algebra
// Pivoted Cholesky factor of a (symmetrised) message: L^T L = M with L k x chi
// in the original column order (a square root of the environment, Sec. 2.5
// step 1 / Fig. 1 "pseudo_sqrt"; eigen-directions below rel * max dropped).
struct EnvFactorItem {
  const double* M;         // chi x chi, leading dimension ld
  double* L;               // k x chi output, leading dimension ld
  int ld;
  int chi_idx;             // ival index of chi
  int rank_idx;            // ival index receiving k
  double rel;              // relative pivot threshold of the instance
};

// Per-site factor of the bond update: either Cholesky-QR (Gram) or
// Householder (TSQR) produces an R-factor of cv (Eq. 10); the gate's
// operator-Schmidt factors turn it into the factor T of X = (gate half) cv.
struct SiteFacItem {
  TView cv;                // absorbed tensor, cut leg innermost (env dims = factor ranks)
  int branch_idx;          // ival: 1 Cholesky-QR, 0 Householder, 2 Householder after a
                           // Gram too ill-conditioned for Cholesky-QR
  int kfac_idx;            // ival: rows of the R-factor (Householder branch)
  int rg_idx;              // ival: operator-Schmidt rank of the bond gate
  const double* F;         // gate factors [kappa][4][4] of this side
  double* C;               // n x n Gram / Householder R (FP64), leading dim ldc
  int ldc;
  double* T;               // r x r (Cholesky) or 4n x r (Householder) workspace / factor
  int ldt;
  int* perm;               // pivot order (r entries)
  int rank_idx;            // ival: rank of the factor
  double rel;              // rank threshold
  double rel_safe;         // smallest fraction of its column's Gram diagonal a Cholesky-QR pivot keeps
  int n_thr;               // Eq. 10 branch thresholds of the instance
  double ratio_thr;
};

// Per-bond core: SVD of R1 R2^T, truncation (Eq. 11), lambda (Eq. 12), the
// reconstruct matrices W1, W2, messages diag(lambda) (Alg. 1 line 13).
struct CoreItem {
  int bond;                // bond id (instance-local)
  int chi_idx;             // ival: live chi of the bond (cut)
  int new_idx;             // ival: pending chi_new
  int rg_idx;
  int rank1_idx, rank2_idx;
  const double* T1; const double* T2;
  int ldt1, ldt2;
  const int* perm1; const int* perm2;
  const double* FA; const double* FB;   // gate factors of side 1 / side 2
  double* work;            // scratch: 4 blocks of rmax * rmax doubles
  int rmax;
  double* W1; double* W2;  // n x n', leading dimension ldw
  int ldw;
  double* lam;             // chi_max entries
  double* msg12; double* msg21;         // chi_max x chi_max each
  int chimax;
  double* sigma1; double* sigma2;       // site log-scales
  double* disc;            // discarded weight of this bond (Table 1 gate_err)
  double* svals;           // all singular values (rmax entries, for diagnostics)
  int* nsv;                // number of singular values
  int inst;                // instance (its flag word is flags_base[inst])
  double eps_cut;
  int mixed_svd;           // 1: FP32 Jacobi preconditioning before FP64 Jacobi (FP32-storage modes)
  int* sweeps;             // 2 ints: FP32 and FP64 Jacobi sweeps of this core
};

// ------------------------------------------------------------------- BP
// One directed message (Eq. 13-19): unnormalised estimate `hat` (double layer)
// or `vhat` (single layer) is turned into the damped, normalised message.
struct MsgItem {
  int inst;
  int chi_idx;             // ival: chi of the bond
  const double* hat;       // chi x chi (ld chimax) double-layer estimate
  double* msg;             // chi x chi (ld chimax) current message (updated)
  const double* vhat;      // chi single-layer estimate
  double* vec;             // chi single-layer message (updated)
  int ld;                  // leading dimension of hat / msg (the instance's chi_max)
  double alpha;            // damping of the instance (Eq. 19)
};

// Per-site Bethe factors (Eq. 7-9): vs_v = <vhat_{v->w}, m_{w->v}>,
// f_v = <hat_{v->w}, M_{w->v}>, with w the site's first layout leg.
struct SiteScalarItem {
  int chi_idx;
  const double* hat; const double* msg_in;
  const double* vhat; const double* vec_in;
  double* vs; double* fv;
  int ld;
};

// Per-site Pauli weights of the double-layer environment: out[p] =
// sum_J x[J, p]^2 over the site tensor x rotated (and scaled by the square
// roots of the message eigenvalues) on every leg, i.e. the Hilbert-Schmidt
// weight of Pauli p at the site with the converged BP messages around it.
struct PauliWItem {
  TView x;
  double* out;             // 4 doubles
};

// Per-bond edge factors: Z_e = m_ab . m_ba, Z2_e = sum M_ab * M_ba.
struct EdgeItem {
  int chi_idx;
  const double* m12; const double* m21;     // double-layer messages
  const double* v12; const double* v21;     // single-layer messages
  double* ze; double* z2e;
  int ld;
};

// Per-instance sums of Eq. 9 and the Bethe norm.
struct BetheItem {
  int nsites, nbonds;
  const double* vs; const double* fv; const double* sigma;
  const double* ze; const double* z2e;
  double* out;             // [C, C_proj, log|C_proj|, sign, log_norm, zero_flag]
};

// Bond gate tables: PTM with folded site gates and its operator-Schmidt factors.
struct GateItem {
  int gateset;             // 0: ZZ bonds / X sites, 1: XX bonds / Z sites
  double theta;            // bond angle (exp(-i theta P P))
  double phi;              // site angle (exp(-i phi Q))
  int pre1, pre2, post1, post2;   // fold the site gate before / after on each side
  double* ptm;             // 16 x 16
  double* FA; double* FB;  // [kappa][4][4]
  int* rank;               // ival slot
  int* flags;
};

}  // namespace pepo
