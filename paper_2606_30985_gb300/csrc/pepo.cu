// libpepo host driver: geometry, arena layout, the static launch plan of one
// Trotter step / BP sweep, and the C ABI of include/pepo.h.
//
// Plan.  Everything a step launches is decided at init from the geometry
// alone (Sec. 2.4 four-colour schedule), because live sizes are read on the
// device.  Per colour the bonds are cut into waves that fit the scratch slabs;
// per wave the launch sequence is (Alg. 1 / Fig. 1, Q-less form):
//   env factors -> absorb (leg contractions) -> Eq. 10 branch ->
//   [Cholesky-QR: Gram -> reduce] | [Householder: TSQR levels -> extract] ->
//   gate fold (formG / formB) -> rank-revealing factor -> bond core (SVD,
//   truncation, lambda, W, messages) -> reconstruct into the next layout ->
//   commit (pointer swap, chi_new).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bp.h"
#include "kernels.h"
#include "linalg.h"
#include "mlp.h"
#include "pepo.h"

using namespace pepo;

namespace {

constexpr int kChiMaxLimit = 128;
// K splits of the Cholesky-QR Gram and of the free-leg (BP message) Gram:
// defaults and the bounds the partial-sum workspaces are sized for (the
// launch shapes are tunable per context, pepo_set_tuning)
constexpr int kGramSplits = 32;
constexpr int kLegSplits = 64;
constexpr int kGramSplitsMax = 64;
constexpr int kLegSplitsMax = 128;
constexpr size_t kAlign = 256;
constexpr unsigned long long kWaitNsDefault = 4000000000ull;   // 4 s

enum { LEG_U = 0, LEG_D = 1, LEG_L = 2, LEG_R = 3 };

struct Leg {
  int name;   // LEG_*
  int bond;
  int nbr;
};

struct SiteG {
  int deg = 0;
  Leg legs[4];          // canonical order
  int pin = 0;          // Pauli index of the pinned single layer
  std::vector<int> upd; // canonical leg indices of this site's updates, colour order
};

struct BondG {
  int v1, v2, leg1, leg2, colour;   // leg1/leg2 canonical leg positions in v1/v2
};

// ------------------------------------------------------------- bump allocator
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <class T> T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * count;
    return p;
  }
};

// host staging of item arrays; device copy made once at init
struct Staging {
  std::vector<char> bytes;
  template <class I> size_t push(const std::vector<I>& v) {
    size_t o = (bytes.size() + 255) / 256 * 256;
    bytes.resize(o + sizeof(I) * v.size());
    if (!v.empty()) std::memcpy(bytes.data() + o, v.data(), sizeof(I) * v.size());
    return o;
  }
};

template <class I> struct DArr {
  size_t off = 0;
  int n = 0;
  const I* d = nullptr;
};

struct GateWave {
  DArr<EnvFactorItem> env;
  DArr<LegItem> leg[3];
  DArr<TView> copy;
  DArr<int> copy_out;
  DArr<SiteFacItem> fac;
  DArr<GramRowsItem> gram;
  DArr<CoreItem> core;
  DArr<ReconItem> recon;
  DArr<int> pairs;
  DArr<int> moves;
  int npairs = 0, nmoves = 0;
};

struct BpWave {
  DArr<EnvEigItem> eig;
  DArr<LegItem> leg[4];
  DArr<GramLegItem> gram;
  DArr<RotItem> rot;
  DArr<PauliWItem> pw;     // final waves only: Pauli weights of the rotated sites
};

struct SlLevel {
  DArr<VecItem> items;
};

struct Inst {
  pepo_config cfg;
  int N = 0, nb = 0;
  std::vector<SiteG> sites;
  std::vector<BondG> bonds;
  std::vector<std::vector<int>> colours;
  // ival indices
  int chi0 = 0, pend0 = 0, grank0 = 0;
  int site_ref0 = 0;
  // device arrays
  void* slab[1];       // unused
  std::vector<void*> site_slab;
  double *lam = nullptr, *msg = nullptr, *hat = nullptr, *vec = nullptr, *vhat = nullptr;
  WsGeom* ws_geom = nullptr;          // 2 nb directed-bond descriptors of the warm-start features
  int* core_sweeps = nullptr;         // 2 nb: FP32 / FP64 Jacobi sweeps of each bond core
  double *sigma = nullptr, *disc = nullptr, *svals = nullptr, *vs = nullptr, *fv = nullptr;
  double* pw = nullptr;    // per site: Pauli weights of the double-layer environment (4)
  double *ze = nullptr, *z2e = nullptr, *bethe_out = nullptr, *ptm = nullptr, *FA = nullptr, *FB = nullptr;
  int* nsv = nullptr;
  // plan
  std::vector<GateWave> gwaves[4];
  DArr<CoreItem> gcore[4];      // all bonds of a colour in one core launch
  std::vector<BpWave> bwaves;
  std::vector<BpWave> fwaves;   // leg-0-only waves for f_v
  SlLevel sl[4];                // levels 0..3 (0: copy items for one-leg sites)
  DArr<MsgItem> msgs;
  DArr<SiteScalarItem> sscal;
  DArr<EdgeItem> escal;
  DArr<BetheItem> bethe;
  DArr<GateItem> gates;
  // diagnostics
  int steps = 0;
  int saved_steps = 0;       // step count stored with the last pepo_save_state
  int last_sweeps = 0, last_sweeps1 = 0;
  double last_delta = 0, last_delta1 = 0;
  // the last measurement (pepo_correlator) and the one of the layer before
  // it, both since the last change of state from the host (c_drop signal)
  int meas_valid = 0, meas_steps = 0, prev_valid = 0;
  double meas_C = 0, meas_ge = 0, prev_C = 0, prev_ge = 0;
  int cap[5] = {0, 0, 0, 0, 0};   // in-flight sites per degree class
  int scratch_ref[5] = {-1, -1, -1, -1, -1};   // one scratch slab per class (uploads)
};

}  // namespace

struct pepo_ctx {
  std::vector<Inst> inst;
  int n_inst = 0;
  int prec = PEPO_FP32;
  size_t tsize = 4;
  int chimax = 1;          // max over instances
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  void** d_ptrs = nullptr;
  int* d_ival = nullptr;
  int n_ptrs = 0, n_ival = 0;
  unsigned long long* d_delta2 = nullptr;
  unsigned long long* d_delta1 = nullptr;
  int* d_flags = nullptr;
  unsigned long long* d_qr_count = nullptr;   // sites per QR branch (k_factor)
  double* d_hh_acct = nullptr;   // Householder QR FLOPs and bytes (k_hh_extract; timing class K_HH)
  int* d_kerr = nullptr;   // bit 0: a tensor-core pipeline wait expired (bits: launch_leg_umma)
  unsigned long long wait_ns = kWaitNsDefault;   // limit of every tensor-core pipeline wait
  char* d_items = nullptr;
  long long launches = 0;
  std::string err;
  bool stepped = false;
  int phase = 0;           // colours of the current Trotter step applied so far (0: step boundary)
  pepo_tuning tune = {kLegSplits, kGramSplits};
  // learned warm start applied inside pepo_bp_converge to the instances with
  // warm_start = 1 (workspace carved only when such an instance exists)
  MlpBuffers ws_mlp{};
  float* ws_X = nullptr;
  float* ws_y = nullptr;
  int ws_rows_max = 0;
  bool ws_ready = false;
  // kernel-class timing
  bool timing = false;
  std::vector<char> host_items;          // host copy of the item arrays
  std::vector<int> ival_snap;            // live sizes at the start of the call
  struct Rec { int cls; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  size_t pool_next = 0;
  struct Tot { long long n = 0; double ms = 0, bytes = 0, flops = 0; };
  std::vector<Tot> tot;
  int max_levels = 1;      // TSQR levels
  int rmax = 4, nmax = 4;
  // grouped execution: every instance's items of one wave / colour / level
  // concatenated into one launch (plan fields of grp only; grp.cfg.chi_max =
  // the context-wide chi_max)
  Inst grp;
  int* d_active = nullptr;                 // per-instance BP activity mask
  // CUDA graphs of one Trotter step, one BP sweep and one single-layer sweep
  // (captured on a private stream at first use, launched on `stream`)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr, bp_exec = nullptr, sl_exec = nullptr;
  long long step_launches = 0, bp_launches = 0, sl_launches = 0;
  bool graphs_failed = false;
  ~pepo_ctx() {
    for (cudaGraphExec_t e : {step_exec, bp_exec, sl_exec})
      if (e) cudaGraphExecDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace {

const char* kStaticErr = "no context";

pepo_status fail(pepo_ctx* c, pepo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

std::string validate(const pepo_config& c) {
  if (c.Lx < 1 || c.Ly < 1 || c.Lx * c.Ly < 2) return "grid must have at least two sites";
  if (c.Lx * c.Ly > 4096) return "grid too large";
  if (c.obs_x < 0 || c.obs_x >= c.Lx || c.obs_y < 0 || c.obs_y >= c.Ly) return "observable site off the grid";
  if (c.obs_pauli < 1 || c.obs_pauli > 3) return "obs_pauli must be 1 (X), 2 (Y) or 3 (Z)";
  if (c.trotter_order != 1 && c.trotter_order != 2) return "trotter_order must be 1 or 2";
  if (c.chi_max < 1 || c.chi_max > kChiMaxLimit) return "chi_max must be in [1, 128]";
  if (!(c.eps_cut >= 0.0)) return "eps_cut must be >= 0";
  if (!(c.bp_alpha > 0.0 && c.bp_alpha <= 1.0)) return "bp_alpha must be in (0, 1]";
  if (!(c.bp_tol > 0.0)) return "bp_tol must be > 0";
  if (c.bp_max_sweeps < 1) return "bp_max_sweeps must be >= 1";
  if (c.gates != PEPO_GATES_ZZ_X && c.gates != PEPO_GATES_XX_Z) return "unknown gate set";
  if (c.prec == PEPO_BF16X3)
    return "PEPO_BF16X3 is not built: a BF16 split needs six products for FP32-level accuracy, "
           "twice the tensor time of PEPO_TF32X3 (use PEPO_TF32X3)";
  if (c.prec < PEPO_FP64 || c.prec > PEPO_BF16X3) return "unknown precision";
  if (!std::isfinite(c.J) || !std::isfinite(c.h) || !std::isfinite(c.dt)) return "non-finite couplings";
  if (c.inflight_sites < 0) return "inflight_sites must be >= 0";
  return "";
}

void build_geometry(Inst& I) {
  const pepo_config& c = I.cfg;
  const int Lx = c.Lx, Ly = c.Ly;
  I.N = Lx * Ly;
  I.sites.assign(I.N, SiteG());
  I.bonds.clear();
  I.colours.assign(4, {});
  // bond ids: horizontal y*(Lx-1)+x, then vertical Ly*(Lx-1) + y*Lx + x
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x + 1 < Lx; ++x) I.bonds.push_back({y * Lx + x, y * Lx + x + 1, 0, 0, x % 2});
  for (int y = 0; y + 1 < Ly; ++y)
    for (int x = 0; x < Lx; ++x) I.bonds.push_back({y * Lx + x, (y + 1) * Lx + x, 0, 0, 2 + y % 2});
  I.nb = (int)I.bonds.size();
  auto bond_id_h = [&](int x, int y) { return y * (Lx - 1) + x; };
  auto bond_id_v = [&](int x, int y) { return Ly * (Lx - 1) + y * Lx + x; };
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      SiteG& s = I.sites[y * Lx + x];
      s.deg = 0;
      if (y > 0) s.legs[s.deg++] = {LEG_U, bond_id_v(x, y - 1), (y - 1) * Lx + x};
      if (y < Ly - 1) s.legs[s.deg++] = {LEG_D, bond_id_v(x, y), (y + 1) * Lx + x};
      if (x > 0) s.legs[s.deg++] = {LEG_L, bond_id_h(x - 1, y), y * Lx + x - 1};
      if (x < Lx - 1) s.legs[s.deg++] = {LEG_R, bond_id_h(x, y), y * Lx + x + 1};
      s.pin = (x == c.obs_x && y == c.obs_y) ? c.obs_pauli : 0;
    }
  for (int b = 0; b < I.nb; ++b) {
    BondG& g = I.bonds[b];
    for (int k = 0; k < I.sites[g.v1].deg; ++k) if (I.sites[g.v1].legs[k].bond == b) g.leg1 = k;
    for (int k = 0; k < I.sites[g.v2].deg; ++k) if (I.sites[g.v2].legs[k].bond == b) g.leg2 = k;
    I.colours[g.colour].push_back(b);
  }
  for (int col = 0; col < 4; ++col)
    for (int b : I.colours[col]) {
      I.sites[I.bonds[b].v1].upd.push_back(I.bonds[b].leg1);
      I.sites[I.bonds[b].v2].upd.push_back(I.bonds[b].leg2);
    }
}

// layout with canonical leg `cut` innermost: list of canonical leg indices
std::vector<int> layout_for(const SiteG& s, int cut) {
  std::vector<int> L;
  for (int k = 0; k < s.deg; ++k) if (k != cut) L.push_back(k);
  L.push_back(cut);
  return L;
}

size_t pow_sz(size_t b, int e) {
  size_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// in-flight cap per degree class: all sites if their scratch fits in 40 GB
void choose_caps(Inst& I, size_t tsize) {
  int count[5] = {0, 0, 0, 0, 0};
  for (auto& s : I.sites) count[s.deg]++;
  const size_t chi = I.cfg.chi_max;
  for (int d = 1; d <= 4; ++d) {
    if (count[d] == 0) { I.cap[d] = 0; continue; }
    size_t slab = 4 * pow_sz(chi, d) * tsize;
    int cap = count[d];
    if (I.cfg.inflight_sites > 0) cap = std::min(cap, I.cfg.inflight_sites);
    else {
      size_t budget = (size_t)40 << 30;   // scratch budget: keeps 10x10 chi=100 FP32 under 180 GB
      size_t fit = budget / (2 * slab);
      if (fit < 1) fit = 1;
      if ((size_t)cap > fit) cap = (int)fit;
    }
    if (cap < 2) cap = std::min(2, count[d]);   // a bond may need two slots of one class
    I.cap[d] = cap;
  }
}

// ----------------------------------------------------------------- planning
struct Planner {
  pepo_ctx* c;
  Carver* cv;        // nullptr base in the sizing pass
  Staging st;
  bool dry;
  std::vector<void*> ptr_init;   // host copy of the pointer table
  std::vector<int> ival_init;
  int new_ival(int v) { ival_init.push_back(v); return (int)ival_init.size() - 1; }
  int new_ptr(void* p) { ptr_init.push_back(p); return (int)ptr_init.size() - 1; }
};

template <class I> DArr<I> stage(Planner& P, const std::vector<I>& v) {
  DArr<I> a;
  a.off = P.st.push(v);
  a.n = (int)v.size();
  return a;
}

struct SlotWS {              // per in-flight site slot (gate update)
  double* L[4];
  double* Ls[4];             // BP: the rotation scaled by the eigenvalue square roots
  int rank_idx[4];
  double* sqrtD[4];
  int branch_idx, kfac_idx, rankT_idx;
  double* C;
  double* T;
  int* perm;
  double* partial;
  double* W;
};

struct ScratchClass {
  std::vector<int> refs;     // pointer-table refs of scratch slabs (2 per slot)
};

bool plan_instance(Planner& P, Inst& I, int inst_id) {
  pepo_ctx* c = P.c;
  Carver& cv = *P.cv;
  const int chimax = I.cfg.chi_max;
  const size_t ts = c->tsize;
  const int nmax = 4 * chimax;           // columns of cv
  const int rmax = PEPO_RG * chimax;     // columns of X
  // ---- state arrays
  I.site_slab.resize(I.N);
  I.site_ref0 = (int)P.ptr_init.size();
  for (int v = 0; v < I.N; ++v) {
    size_t n = 4 * pow_sz(chimax, I.sites[v].deg);
    void* p = cv.take<char>(n * ts);
    I.site_slab[v] = p;
    P.new_ptr(p);
  }
  I.chi0 = (int)P.ival_init.size();
  for (int b = 0; b < I.nb; ++b) P.new_ival(1);
  I.pend0 = (int)P.ival_init.size();
  for (int b = 0; b < I.nb; ++b) P.new_ival(1);
  I.grank0 = (int)P.ival_init.size();
  for (int b = 0; b < I.nb; ++b) P.new_ival(1);
  const size_t cm2 = (size_t)chimax * chimax;
  I.lam = cv.take<double>(I.nb * (size_t)chimax);
  I.msg = cv.take<double>(2 * I.nb * cm2);
  I.hat = cv.take<double>(2 * I.nb * cm2);
  I.vec = cv.take<double>(2 * I.nb * (size_t)chimax);
  I.vhat = cv.take<double>(2 * I.nb * (size_t)chimax);
  I.sigma = cv.take<double>(I.N);
  I.disc = cv.take<double>(I.nb);
  I.pw = cv.take<double>((size_t)4 * I.N);
  I.svals = cv.take<double>(I.nb * (size_t)rmax);
  I.nsv = cv.take<int>(I.nb);
  I.vs = cv.take<double>(I.N);
  I.fv = cv.take<double>(I.N);
  I.ze = cv.take<double>(I.nb);
  I.z2e = cv.take<double>(I.nb);
  I.bethe_out = cv.take<double>(8);
  I.ptm = cv.take<double>(I.nb * (size_t)256);
  I.FA = cv.take<double>(I.nb * (size_t)PEPO_RG * 16);
  I.FB = cv.take<double>(I.nb * (size_t)PEPO_RG * 16);
  I.ws_geom = cv.take<WsGeom>(2 * (size_t)I.nb);
  I.core_sweeps = cv.take<int>(2 * (size_t)I.nb);

  auto chi_idx = [&](int b) { return I.chi0 + b; };
  auto msg_in = [&](int v, int b) {   // message into v on bond b
    return (I.bonds[b].v2 == v) ? 2 * b : 2 * b + 1;
  };
  auto msg_out = [&](int v, int b) { return (I.bonds[b].v1 == v) ? 2 * b : 2 * b + 1; };
  auto mptr = [&](double* base, int id) { return base + (size_t)id * cm2; };

  // ---- scratch slabs per degree class
  choose_caps(I, ts);
  ScratchClass sc[5];
  int maxslots = 0;
  for (int d = 1; d <= 4; ++d) {
    for (int k = 0; k < 2 * I.cap[d]; ++k) {
      void* p = cv.take<char>(4 * pow_sz(chimax, d) * ts);
      sc[d].refs.push_back(P.new_ptr(p));
    }
    maxslots += I.cap[d];
    if (!sc[d].refs.empty()) I.scratch_ref[d] = sc[d].refs[0];
  }
  // ---- per-slot workspaces (gate update and BP)
  std::vector<SlotWS> slots(maxslots);
  for (int k = 0; k < maxslots; ++k) {
    SlotWS& w = slots[k];
    for (int j = 0; j < 4; ++j) {
      w.L[j] = cv.take<double>(cm2);
      w.Ls[j] = cv.take<double>(cm2);
      w.rank_idx[j] = P.new_ival(1);
      w.sqrtD[j] = cv.take<double>(chimax);
    }
    w.branch_idx = P.new_ival(0);
    w.kfac_idx = P.new_ival(0);
    w.rankT_idx = P.new_ival(0);
    w.C = cv.take<double>((size_t)nmax * nmax);
    w.T = cv.take<double>((size_t)4 * nmax * rmax);
    w.perm = cv.take<int>(rmax);
    size_t pg = (size_t)kGramSplitsMax * nmax * nmax;
    size_t pl = (size_t)PEPO_MAXLEG * kLegSplitsMax * cm2;
    w.partial = cv.take<double>(std::max(pg, pl));
    w.W = cv.take<double>((size_t)nmax * nmax);
  }
  size_t maxcol = 0;
  for (int col = 0; col < 4; ++col) maxcol = std::max(maxcol, I.colours[col].size());
  std::vector<double*> corework(std::max<size_t>(1, maxcol));
  for (size_t k = 0; k < corework.size(); ++k) corework[k] = cv.take<double>((size_t)4 * rmax * rmax);

  // ---- gate tables
  {
    std::vector<GateItem> g(I.nb);
    std::vector<int> first(I.N, -1), last(I.N, -1);
    for (int col = 0; col < 4; ++col)
      for (int b : I.colours[col]) {
        for (int v : {I.bonds[b].v1, I.bonds[b].v2}) {
          if (first[v] < 0) first[v] = b;
          last[v] = b;
        }
      }
    const bool second = I.cfg.trotter_order == 2;
    for (int b = 0; b < I.nb; ++b) {
      GateItem& it = g[b];
      it.gateset = I.cfg.gates;
      it.theta = I.cfg.J * I.cfg.dt;
      it.phi = second ? 0.5 * I.cfg.h * I.cfg.dt : I.cfg.h * I.cfg.dt;
      it.pre1 = first[I.bonds[b].v1] == b;
      it.pre2 = first[I.bonds[b].v2] == b;
      it.post1 = second && last[I.bonds[b].v1] == b;
      it.post2 = second && last[I.bonds[b].v2] == b;
      it.ptm = I.ptm + (size_t)b * 256;
      it.FA = I.FA + (size_t)b * PEPO_RG * 16;
      it.FB = I.FB + (size_t)b * PEPO_RG * 16;
      it.rank = nullptr;   // patched below (needs the ival device base)
      it.flags = nullptr;
    }
    I.gates = stage(P, g);
  }

  // ---- per-site factor workspaces (live from the factorisation to the reconstruct)
  struct SiteWS { double* C; double* T; int* perm; double* W; float* Wp; int branch_idx, kfac_idx, rankT_idx; };
  std::vector<SiteWS> sws(I.N);
  for (int v = 0; v < I.N; ++v) {
    SiteWS& q = sws[v];
    q.C = cv.take<double>((size_t)nmax * nmax);
    q.T = cv.take<double>((size_t)4 * nmax * rmax);
    q.perm = cv.take<int>(rmax);
    q.W = cv.take<double>((size_t)nmax * nmax);
    q.Wp = (ts == 4 && umma_supported(chimax)) ? cv.take<float>(recon_packed_floats(nmax)) : nullptr;
    q.branch_idx = P.new_ival(0);
    q.kfac_idx = P.new_ival(0);
    q.rankT_idx = P.new_ival(0);
  }

  // ---- gate-update waves
  const double rel_fac = (c->prec == PEPO_FP64) ? 1e-15 : 1e-13;
  // smallest fraction of a column's own Gram diagonal that a Cholesky-QR
  // pivot must keep: far above the Gram's relative rounding (FP32-storage
  // Gram: ~1e-8 of the paired columns' scale; FP64: ~1e-14) and the FP32
  // pivot check's own (~1e-6), where the pivots of columns that depend
  // linearly on the others land; below it the site takes the Householder
  // branch
  const double rel_safe = (c->prec == PEPO_FP64) ? 1e-10 : 1e-4;
  const double rel_env = I.cfg.pinv_rel;
  for (int col = 0; col < 4; ++col) {
    const auto& bl = I.colours[col];
    std::vector<CoreItem> core_all;
    size_t pos = 0;
    while (pos < bl.size()) {
      // greedy wave
      int used[5] = {0, 0, 0, 0, 0};
      std::vector<int> wb;
      while (pos < bl.size()) {
        int b = bl[pos];
        int d1 = I.sites[I.bonds[b].v1].deg, d2 = I.sites[I.bonds[b].v2].deg;
        int need1 = 1 + (d1 == d2 ? 1 : 0);
        if (used[d1] + need1 > I.cap[d1] || (d1 != d2 && used[d2] + 1 > I.cap[d2])) break;
        used[d1]++;
        used[d2]++;
        wb.push_back(b);
        ++pos;
      }
      if (wb.empty()) return false;   // cannot happen: caps >= 1 per class
      GateWave gw;
      std::vector<EnvFactorItem> env;
      std::vector<LegItem> leg[3];
      std::vector<TView> cpy;
      std::vector<int> cpy_out;
      std::vector<SiteFacItem> fac;
      std::vector<GramRowsItem> gram;
      std::vector<ReconItem> recon;
      std::vector<int> pairs, moves;
      int cls_used[5] = {0, 0, 0, 0, 0};
      int slot_base[5];
      {
        int acc = 0;
        for (int d = 1; d <= 4; ++d) { slot_base[d] = acc; acc += I.cap[d]; }
      }
      for (size_t wbi = 0; wbi < wb.size(); ++wbi) {
        const int b = wb[wbi];
        const BondG& B = I.bonds[b];
        int fac_index[2];
        for (int side = 0; side < 2; ++side) {
          const int v = side == 0 ? B.v1 : B.v2;
          const int cutc = side == 0 ? B.leg1 : B.leg2;   // canonical leg index
          const SiteG& S = I.sites[v];
          const int d = S.deg;
          const int k = cls_used[d]++;
          const int slot = slot_base[d] + k;
          SlotWS& W = slots[slot];
          const int sref0 = sc[d].refs[2 * k], sref1 = sc[d].refs[2 * k + 1];
          // current layout: cut innermost; next layout: next update's leg innermost
          std::vector<int> lay = layout_for(S, cutc);
          int ui = 0;
          for (int q = 0; q < (int)S.upd.size(); ++q) if (S.upd[q] == cutc) ui = q;
          const int nextc = S.upd[(ui + 1) % S.upd.size()];
          std::vector<int> nlay = layout_for(S, nextc);
          const int nenv = d - 1;
          // env factors
          for (int j = 0; j < nenv; ++j) {
            const int bj = S.legs[lay[j]].bond;
            EnvFactorItem e;
            e.M = mptr(I.msg, msg_in(v, bj));
            e.L = W.L[j];
            e.ld = chimax;
            e.chi_idx = chi_idx(bj);
            e.rank_idx = W.rank_idx[j];
            e.rel = I.cfg.pinv_rel;
            env.push_back(e);
          }
          // absorb chain
          TView view;
          view.nlegs = d;
          for (int j = 0; j < d; ++j) view.dim[j] = chi_idx(S.legs[lay[j]].bond);
          int cur_ref = I.site_ref0 + v;
          int cv_ref;
          if (nenv == 0) {
            TView t = view;
            t.ref = cur_ref;
            cpy.push_back(t);
            cpy_out.push_back(sref0);
            cv_ref = sref0;
          } else {
            TView t = view;
            for (int r = 0; r < nenv; ++r) {
              LegItem li;
              t.ref = cur_ref;
              li.in = t;
              li.out_ref = (r % 2 == 0) ? sref0 : sref1;
              li.leg = r;
              li.out_dim = W.rank_idx[r];
              li.a_rows = W.rank_idx[r];
              li.A = W.L[r];
              li.lda = chimax;
              leg[r].push_back(li);
              t.dim[r] = W.rank_idx[r];
              cur_ref = li.out_ref;
            }
            cv_ref = cur_ref;
          }
          TView cvv = view;
          cvv.ref = cv_ref;
          for (int j = 0; j < nenv; ++j) cvv.dim[j] = W.rank_idx[j];
          SiteFacItem f;
          f.cv = cvv;
          f.branch_idx = sws[v].branch_idx;
          f.kfac_idx = sws[v].kfac_idx;
          f.rg_idx = I.grank0 + b;
          f.F = (side == 0 ? I.FA : I.FB) + (size_t)b * PEPO_RG * 16;
          f.C = sws[v].C;
          f.ldc = nmax;
          f.T = sws[v].T;
          f.ldt = rmax;
          f.perm = sws[v].perm;
          f.rank_idx = sws[v].rankT_idx;
          f.rel = rel_fac;
          f.rel_safe = rel_safe;
          f.n_thr = I.cfg.qr_n_thresh;
          f.ratio_thr = I.cfg.qr_ratio_thresh;
          fac_index[side] = (int)fac.size();
          fac.push_back(f);
          GramRowsItem g;
          g.x = cvv;
          g.y_ref = cv_ref;
          g.active = sws[v].branch_idx;
          g.partial = W.partial;
          g.out = sws[v].C;
          g.ldo = nmax;
          gram.push_back(g);
          // reconstruct: input = site tensor (layout lay), output layout nlay
          ReconItem rc;
          rc.in = view;
          rc.in.ref = I.site_ref0 + v;
          const int out_ref = (cv_ref == sref0) ? sref1 : sref0;
          rc.out_ref = out_ref;
          rc.new_dim = I.pend0 + b;
          for (int kk = 0; kk < d; ++kk) {
            int canon = nlay[kk];
            int pos_in = (int)(std::find(lay.begin(), lay.end(), canon) - lay.begin());
            rc.out_perm[kk] = pos_in;
          }
          rc.W = sws[v].W;
          rc.Wp = sws[v].Wp;
          rc.ldw = nmax;
          rc.scale_sq = nullptr;
          recon.push_back(rc);
          pairs.push_back(I.site_ref0 + v);
          pairs.push_back(out_ref);
        }
        CoreItem ci;
        const SiteFacItem& f1 = fac[fac_index[0]];
        const SiteFacItem& f2 = fac[fac_index[1]];
        ci.bond = b;
        ci.chi_idx = chi_idx(b);
        ci.new_idx = I.pend0 + b;
        ci.rg_idx = I.grank0 + b;
        ci.rank1_idx = f1.rank_idx;
        ci.rank2_idx = f2.rank_idx;
        ci.T1 = f1.T; ci.T2 = f2.T;
        ci.ldt1 = f1.ldt; ci.ldt2 = f2.ldt;
        ci.perm1 = f1.perm; ci.perm2 = f2.perm;
        ci.FA = I.FA + (size_t)b * PEPO_RG * 16;
        ci.FB = I.FB + (size_t)b * PEPO_RG * 16;
        ci.work = corework[core_all.size()];
        ci.rmax = rmax;
        ci.W1 = const_cast<double*>(recon[fac_index[0]].W);   // recon items follow fac items
        ci.W2 = const_cast<double*>(recon[fac_index[1]].W);
        ci.ldw = nmax;
        ci.lam = I.lam + (size_t)b * chimax;
        ci.msg12 = mptr(I.msg, 2 * b);
        ci.msg21 = mptr(I.msg, 2 * b + 1);
        ci.chimax = chimax;
        ci.sigma1 = I.sigma + B.v1;
        ci.sigma2 = I.sigma + B.v2;
        ci.disc = I.disc + b;
        ci.svals = I.svals + (size_t)b * rmax;
        ci.nsv = I.nsv + b;
        ci.inst = inst_id;
        ci.eps_cut = I.cfg.eps_cut;
        ci.mixed_svd = (c->tsize == 4) ? 1 : 0;
        ci.sweeps = I.core_sweeps + 2 * (size_t)b;
        core_all.push_back(ci);
        moves.push_back(chi_idx(b));
        moves.push_back(I.pend0 + b);
      }
      gw.env = stage(P, env);
      for (int r = 0; r < 3; ++r) gw.leg[r] = stage(P, leg[r]);
      gw.copy = stage(P, cpy);
      gw.copy_out = stage(P, cpy_out);
      gw.fac = stage(P, fac);
      gw.gram = stage(P, gram);
      gw.recon = stage(P, recon);
      gw.pairs = stage(P, pairs);
      gw.moves = stage(P, moves);
      gw.npairs = (int)pairs.size() / 2;
      gw.nmoves = (int)moves.size() / 2;
      I.gwaves[col].push_back(gw);
    }
    I.gcore[col] = stage(P, core_all);
  }
  (void)inst_id;

  // ---- BP waves (double layer): sites grouped by class caps
  // Double-layer BP plan (Eq. 13).  Every incoming message is eigen-decomposed,
  // M_{u->v} = V_u diag(D_u) V_u^T; the site tensor is rotated into the
  // eigenbases of all its legs, psi' = psi x_u V_u^T (deg leg contractions);
  // then each outgoing message is the Gram of psi' over every index but one
  // leg, weighted by prod_{u != w} D_u (applied as sqrt(D) on load), rotated
  // back with V_w.  One launch computes the Grams of all legs of the wave.
  auto make_bp_waves = [&](bool fv_only, std::vector<BpWave>& out) {
    size_t pos = 0;
    while (pos < (size_t)I.N) {
      int used[5] = {0, 0, 0, 0, 0};
      std::vector<int> ws;
      while (pos < (size_t)I.N) {
        int v = (int)pos;
        int d = I.sites[v].deg;
        if (used[d] + 1 > I.cap[d]) break;
        used[d]++;
        ws.push_back(v);
        ++pos;
      }
      BpWave bw;
      std::vector<EnvEigItem> eig;
      std::vector<LegItem> leg[4];
      std::vector<GramLegItem> gram;
      std::vector<RotItem> rot;
      std::vector<PauliWItem> pws;
      int cls_used[5] = {0, 0, 0, 0, 0};
      int slot_base[5];
      {
        int acc = 0;
        for (int d = 1; d <= 4; ++d) { slot_base[d] = acc; acc += I.cap[d]; }
      }
      for (int v : ws) {
        const SiteG& S = I.sites[v];
        const int d = S.deg;
        const int k = cls_used[d]++;
        const int slot = slot_base[d] + k;
        SlotWS& W = slots[slot];
        const int refs[3] = {I.site_ref0 + v, sc[d].refs[2 * k], sc[d].refs[2 * k + 1]};
        std::vector<int> lay = layout_for(S, S.upd[0]);   // step-boundary layout
        TView view;
        view.nlegs = d;
        for (int j = 0; j < d; ++j) view.dim[j] = chi_idx(S.legs[lay[j]].bond);
        for (int j = 0; j < d; ++j) {
          const int bj = S.legs[lay[j]].bond;
          EnvEigItem e;
          e.M = mptr(I.msg, msg_in(v, bj));
          e.ld = chimax;
          e.chi_idx = chi_idx(bj);
          e.work = W.T + (size_t)j * 2 * cm2;
          e.Vt = W.L[j];
          e.sqrtD = W.sqrtD[j];
          e.Vs = W.Ls[j];
          eig.push_back(e);
        }
        int cur = refs[0];
        for (int j = 0; j < d; ++j) {
          LegItem li;
          li.in = view;
          li.in.ref = cur;
          li.out_ref = refs[1 + (j % 2)];
          li.leg = j;
          li.out_dim = view.dim[j];
          li.a_rows = view.dim[j];
          // the rotated leg carries the square roots of the message's
          // eigenvalues: the Grams below then need no weights
          li.A = W.Ls[j];
          li.lda = chimax;
          leg[j].push_back(li);
          cur = li.out_ref;
        }
        for (int w = fv_only ? d - 1 : 0; w < d; ++w) {
          const int bw_ = S.legs[lay[w]].bond;
          GramLegItem g;
          g.x = view;
          g.x.ref = cur;
          g.y_ref = cur;
          g.leg = w;
          g.partial = W.partial + (size_t)w * kLegSplitsMax * cm2;
          g.out = W.C + (size_t)w * cm2;
          g.ldo = chimax;
          for (int u = 0; u < PEPO_MAXLEG; ++u) g.sw[u] = nullptr;
          gram.push_back(g);
          RotItem r;
          r.G = g.out;
          r.Vt = W.L[w];
          r.sd = W.sqrtD[w];
          r.out = mptr(I.hat, msg_out(v, bw_));
          r.ld = chimax;
          r.chi_idx = chi_idx(bw_);
          rot.push_back(r);
        }
        if (fv_only) {
          PauliWItem pw;
          pw.x = view;
          pw.x.ref = cur;
          pw.out = I.pw + (size_t)4 * v;
          pws.push_back(pw);
        }
      }
      bw.eig = stage(P, eig);
      for (int j = 0; j < 4; ++j) bw.leg[j] = stage(P, leg[j]);
      bw.gram = stage(P, gram);
      bw.rot = stage(P, rot);
      bw.pw = stage(P, pws);
      out.push_back(bw);
    }
  };
  make_bp_waves(false, I.bwaves);
  make_bp_waves(true, I.fwaves);

  // ---- single-layer plan: memoised contraction tree per site
  {
    std::vector<VecItem> lv[4];
    for (int v = 0; v < I.N; ++v) {
      const SiteG& S = I.sites[v];
      const int d = S.deg;
      std::vector<int> lay = layout_for(S, S.upd[0]);
      std::vector<int> dimidx(d);
      for (int j = 0; j < d; ++j) dimidx[j] = chi_idx(S.legs[lay[j]].bond);
      if (d == 1) {
        VecItem it;
        it.in_ref = I.site_ref0 + v;
        it.pin = S.pin;
        it.in_d = nullptr;
        it.ndims = 1;
        it.dim[0] = dimidx[0];
        it.leg = -1;
        it.v = nullptr;
        it.out = I.vhat + (size_t)msg_out(v, S.legs[lay[0]].bond) * chimax;
        lv[0].push_back(it);
        continue;
      }
      // node key: bitmask of contracted layout positions (contracted in
      // descending position order, skipping the outgoing leg)
      struct Node { double* buf; std::vector<int> legs; };
      std::vector<std::pair<int, Node>> memo;
      auto find = [&](int mask) -> Node* {
        for (auto& m : memo) if (m.first == mask) return &m.second;
        return nullptr;
      };
      for (int w = 0; w < d; ++w) {
        int mask = 0;
        Node cur{nullptr, {}};
        for (int j = 0; j < d; ++j) cur.legs.push_back(j);
        bool from_site = true;
        std::vector<int> seq;
        for (int j = d - 1; j >= 0; --j) if (j != w) seq.push_back(j);
        for (size_t si = 0; si < seq.size(); ++si) {
          const int j = seq[si];
          const int nmask = mask | (1 << j);
          Node* hit = find(nmask);
          if (!hit) {
            Node nn;
            for (int l : cur.legs) if (l != j) nn.legs.push_back(l);
            const bool final_ = (si + 1 == seq.size());
            if (final_) nn.buf = nullptr;   // written into vhat (not memoised across w)
            else nn.buf = cv.take<double>(pow_sz(chimax, (int)nn.legs.size()));
            VecItem it;
            it.in_ref = from_site ? I.site_ref0 + v : -1;
            it.pin = S.pin;
            it.in_d = from_site ? nullptr : cur.buf;
            it.ndims = (int)cur.legs.size();
            for (size_t q = 0; q < cur.legs.size(); ++q) it.dim[q] = dimidx[cur.legs[q]];
            int posj = (int)(std::find(cur.legs.begin(), cur.legs.end(), j) - cur.legs.begin());
            it.leg = posj;
            const int bj = S.legs[lay[j]].bond;
            it.v = I.vec + (size_t)msg_in(v, bj) * chimax;
            if (final_) it.out = I.vhat + (size_t)msg_out(v, S.legs[lay[w]].bond) * chimax;
            else it.out = nn.buf;
            lv[si + 1].push_back(it);
            if (!final_) { memo.push_back({nmask, nn}); hit = &memo.back().second; }
            else { cur = nn; mask = nmask; from_site = false; continue; }
          }
          cur = *hit;
          mask = nmask;
          from_site = false;
        }
      }
    }
    for (int l = 0; l < 4; ++l) I.sl[l].items = stage(P, lv[l]);
  }

  // ---- message / scalar / Bethe items
  {
    std::vector<MsgItem> mi(2 * I.nb);
    for (int id = 0; id < 2 * I.nb; ++id) {
      MsgItem& m = mi[id];
      m.inst = inst_id;
      m.chi_idx = chi_idx(id / 2);
      m.hat = mptr(I.hat, id);
      m.msg = mptr(I.msg, id);
      m.vhat = I.vhat + (size_t)id * chimax;
      m.vec = I.vec + (size_t)id * chimax;
      m.ld = chimax;
      m.alpha = I.cfg.bp_alpha;
    }
    I.msgs = stage(P, mi);
    std::vector<SiteScalarItem> ss(I.N);
    for (int v = 0; v < I.N; ++v) {
      const SiteG& S = I.sites[v];
      std::vector<int> lay = layout_for(S, S.upd[0]);
      const int b0 = S.legs[lay[S.deg - 1]].bond;   // the message the f_v plan computes
      SiteScalarItem& s = ss[v];
      s.chi_idx = chi_idx(b0);
      s.hat = mptr(I.hat, msg_out(v, b0));
      s.msg_in = mptr(I.msg, msg_in(v, b0));
      s.vhat = I.vhat + (size_t)msg_out(v, b0) * chimax;
      s.vec_in = I.vec + (size_t)msg_in(v, b0) * chimax;
      s.vs = I.vs + v;
      s.fv = I.fv + v;
      s.ld = chimax;
    }
    I.sscal = stage(P, ss);
    std::vector<EdgeItem> es(I.nb);
    for (int b = 0; b < I.nb; ++b) {
      EdgeItem& e = es[b];
      e.chi_idx = chi_idx(b);
      e.m12 = mptr(I.msg, 2 * b);
      e.m21 = mptr(I.msg, 2 * b + 1);
      e.v12 = I.vec + (size_t)(2 * b) * chimax;
      e.v21 = I.vec + (size_t)(2 * b + 1) * chimax;
      e.ze = I.ze + b;
      e.z2e = I.z2e + b;
      e.ld = chimax;
    }
    I.escal = stage(P, es);
    std::vector<BetheItem> bi(1);
    bi[0].nsites = I.N;
    bi[0].nbonds = I.nb;
    bi[0].vs = I.vs;
    bi[0].fv = I.fv;
    bi[0].sigma = I.sigma;
    bi[0].ze = I.ze;
    bi[0].z2e = I.z2e;
    bi[0].out = I.bethe_out;
    I.bethe = stage(P, bi);
  }
  (void)rel_env;
  return true;
}

template <class I> void resolve(DArr<I>& a, char* dbase) {
  a.d = reinterpret_cast<const I*>(dbase + a.off);
}

// patch device pointers that depend on ctx-level arrays, then resolve items
void finalize_items(pepo_ctx* c, Planner& P) {
  // patch flags / rank pointers inside staged bytes
  for (int i = 0; i < c->n_inst; ++i) {
    Inst& I = c->inst[i];
    GateItem* g = reinterpret_cast<GateItem*>(P.st.bytes.data() + I.gates.off);
    for (int b = 0; b < I.gates.n; ++b) {
      g[b].rank = c->d_ival + I.grank0 + b;
      g[b].flags = c->d_flags + i;
    }

  }
}

void resolve_all(pepo_ctx* c) {
  char* d = c->d_items;
  std::vector<Inst*> all;
  for (auto& I : c->inst) all.push_back(&I);
  all.push_back(&c->grp);
  for (Inst* Ip : all) {
    Inst& I = *Ip;
    for (int col = 0; col < 4; ++col) resolve(I.gcore[col], d);
    for (int col = 0; col < 4; ++col)
      for (auto& w : I.gwaves[col]) {
        resolve(w.env, d);
        for (int r = 0; r < 3; ++r) resolve(w.leg[r], d);
        resolve(w.copy, d); resolve(w.copy_out, d); resolve(w.fac, d); resolve(w.gram, d);
        resolve(w.core, d); resolve(w.recon, d); resolve(w.pairs, d); resolve(w.moves, d);
      }
    for (auto* ws : {&I.bwaves, &I.fwaves})
      for (auto& w : *ws) {
        resolve(w.eig, d);
        for (int a = 0; a < 4; ++a) resolve(w.leg[a], d);
        resolve(w.gram, d);
        resolve(w.rot, d);
        resolve(w.pw, d);
      }
    for (int l = 0; l < 4; ++l) resolve(I.sl[l].items, d);
    resolve(I.msgs, d); resolve(I.sscal, d); resolve(I.escal, d); resolve(I.bethe, d);
    resolve(I.gates, d);
  }
}

template <class T> DArr<T> cat_items(Planner& P, const std::vector<const DArr<T>*>& parts) {
  std::vector<T> v;
  for (const DArr<T>* a : parts) {
    const T* src = reinterpret_cast<const T*>(P.st.bytes.data() + a->off);
    v.insert(v.end(), src, src + a->n);
  }
  return stage(P, v);
}

// Concatenate the item arrays of all instances per colour / wave index /
// level into the group plan (instances with fewer waves contribute nothing to
// the higher wave indices).  Instances own disjoint state and scratch, so the
// items of one grouped launch never touch each other's memory.
void build_group(Planner& P, pepo_ctx* c) {
  Inst& G = c->grp;
  G.cfg = c->inst[0].cfg;
  G.cfg.chi_max = c->chimax;
  if (c->n_inst == 1) {
    const Inst& I = c->inst[0];
    for (int col = 0; col < 4; ++col) { G.gwaves[col] = I.gwaves[col]; G.gcore[col] = I.gcore[col]; }
    G.bwaves = I.bwaves;
    G.fwaves = I.fwaves;
    for (int l = 0; l < 4; ++l) G.sl[l] = I.sl[l];
    G.msgs = I.msgs; G.sscal = I.sscal; G.escal = I.escal; G.bethe = I.bethe;
    return;
  }
  for (int col = 0; col < 4; ++col) {
    size_t nw = 0;
    for (auto& I : c->inst) nw = std::max(nw, I.gwaves[col].size());
    G.gwaves[col].assign(nw, GateWave());
    for (size_t w = 0; w < nw; ++w) {
      std::vector<const GateWave*> parts;
      for (auto& I : c->inst) if (w < I.gwaves[col].size()) parts.push_back(&I.gwaves[col][w]);
      auto pick = [&](auto field) {
        using A = std::remove_reference_t<decltype(field(*parts[0]))>;
        std::vector<const A*> v;
        for (auto* g : parts) v.push_back(&field(*g));
        return cat_items(P, v);
      };
      GateWave& gw = G.gwaves[col][w];
      gw.env = pick([](const GateWave& g) -> const DArr<EnvFactorItem>& { return g.env; });
      for (int r = 0; r < 3; ++r) {
        std::vector<const DArr<LegItem>*> v;
        for (auto* g : parts) v.push_back(&g->leg[r]);
        gw.leg[r] = cat_items(P, v);
      }
      gw.copy = pick([](const GateWave& g) -> const DArr<TView>& { return g.copy; });
      gw.copy_out = pick([](const GateWave& g) -> const DArr<int>& { return g.copy_out; });
      gw.fac = pick([](const GateWave& g) -> const DArr<SiteFacItem>& { return g.fac; });
      gw.gram = pick([](const GateWave& g) -> const DArr<GramRowsItem>& { return g.gram; });
      gw.core = pick([](const GateWave& g) -> const DArr<CoreItem>& { return g.core; });
      gw.recon = pick([](const GateWave& g) -> const DArr<ReconItem>& { return g.recon; });
      gw.pairs = pick([](const GateWave& g) -> const DArr<int>& { return g.pairs; });
      gw.moves = pick([](const GateWave& g) -> const DArr<int>& { return g.moves; });
      gw.npairs = gw.pairs.n / 2;
      gw.nmoves = gw.moves.n / 2;
    }
    std::vector<const DArr<CoreItem>*> cores;
    for (auto& I : c->inst) cores.push_back(&I.gcore[col]);
    G.gcore[col] = cat_items(P, cores);
  }
  for (int f = 0; f < 2; ++f) {
    std::vector<BpWave>& out = f ? G.fwaves : G.bwaves;
    size_t nw = 0;
    for (auto& I : c->inst) nw = std::max(nw, (f ? I.fwaves : I.bwaves).size());
    out.assign(nw, BpWave());
    for (size_t w = 0; w < nw; ++w) {
      std::vector<const DArr<EnvEigItem>*> eig;
      std::vector<const DArr<LegItem>*> leg[4];
      std::vector<const DArr<GramLegItem>*> gram;
      std::vector<const DArr<RotItem>*> rot;
      std::vector<const DArr<PauliWItem>*> pw;
      for (auto& I : c->inst) {
        const std::vector<BpWave>& src = f ? I.fwaves : I.bwaves;
        if (w >= src.size()) continue;
        eig.push_back(&src[w].eig);
        for (int a = 0; a < 4; ++a) leg[a].push_back(&src[w].leg[a]);
        gram.push_back(&src[w].gram);
        rot.push_back(&src[w].rot);
        pw.push_back(&src[w].pw);
      }
      out[w].eig = cat_items(P, eig);
      for (int a = 0; a < 4; ++a) out[w].leg[a] = cat_items(P, leg[a]);
      out[w].gram = cat_items(P, gram);
      out[w].rot = cat_items(P, rot);
      out[w].pw = cat_items(P, pw);
    }
  }
  for (int l = 0; l < 4; ++l) {
    std::vector<const DArr<VecItem>*> v;
    for (auto& I : c->inst) v.push_back(&I.sl[l].items);
    G.sl[l].items = cat_items(P, v);
  }
  {
    std::vector<const DArr<MsgItem>*> m;
    std::vector<const DArr<SiteScalarItem>*> ss;
    std::vector<const DArr<EdgeItem>*> es;
    std::vector<const DArr<BetheItem>*> be;
    for (auto& I : c->inst) { m.push_back(&I.msgs); ss.push_back(&I.sscal); es.push_back(&I.escal); be.push_back(&I.bethe); }
    G.msgs = cat_items(P, m);
    G.sscal = cat_items(P, ss);
    G.escal = cat_items(P, es);
    G.bethe = cat_items(P, be);
  }
}

// full arena layout; base == nullptr computes the size only
size_t layout_arena(pepo_ctx* c, char* base, Planner* keep) {
  Carver cv(base);
  Planner P;
  P.c = c;
  P.cv = &cv;
  P.dry = base == nullptr;
  for (int i = 0; i < c->n_inst; ++i) {
    if (!plan_instance(P, c->inst[i], i)) return 0;
  }
  build_group(P, c);
  c->n_ptrs = (int)P.ptr_init.size();
  c->n_ival = (int)P.ival_init.size();
  c->d_ptrs = cv.take<void*>(c->n_ptrs);
  c->d_ival = cv.take<int>(c->n_ival);
  c->d_delta2 = cv.take<unsigned long long>(c->n_inst);
  c->d_delta1 = cv.take<unsigned long long>(c->n_inst);
  c->d_flags = cv.take<int>(c->n_inst);
  c->d_kerr = cv.take<int>(1);
  c->d_qr_count = cv.take<unsigned long long>(3);
  c->d_hh_acct = cv.take<double>(2);
  c->d_active = cv.take<int>(c->n_inst);
  c->d_items = cv.take<char>(P.st.bytes.size() + 256);
  // warm-start workspace: one network and one feature / prediction buffer
  // sized for the largest instance (instances are handled one after another)
  int ws_rows = 0;
  for (int i = 0; i < c->n_inst; ++i)
    if (c->inst[i].cfg.warm_start)
      ws_rows = std::max(ws_rows, 2 * c->inst[i].nb * c->inst[i].cfg.chi_max);
  c->ws_rows_max = ws_rows;
  if (ws_rows > 0) {
    MlpBuffers tmp;
    char* mbase = cv.take<char>(mlp_layout(nullptr, ws_rows, &tmp));
    if (base) mlp_layout(mbase, ws_rows, &c->ws_mlp);
    c->ws_X = cv.take<float>((size_t)ws_rows * PEPO_WS_FEATURES);
    c->ws_y = cv.take<float>((size_t)ws_rows);
  }
  size_t total = cv.off + kAlign;
  if (keep) *keep = std::move(P);
  return total;
}

// ------------------------------------------------------------ kernel timing
// Bond-layer classes (absorb legs, Cholesky-QR Gram, Householder, factors,
// core, reconstruct, environment factors) are kept apart from the BP classes
// (eigenbasis leg rotations, message Grams, eigenbases, message finish), so
// that the bond-update rate counts the bond layer only.
enum KClass {
  K_LEG = 0, K_GRAM_ROWS, K_GRAM_ROWS_RED, K_GRAM_LEG, K_GRAM_LEG_RED, K_RECON, K_HH, K_FACTOR,
  K_CORE, K_ENV, K_VEC, K_MSG, K_OTHER, K_BP_LEG, K_BP_EIG, K_NCLASS
};
const char* kClassNames[K_NCLASS] = {
  "leg_contract", "gram_rows", "gram_rows_reduce", "gram_leg", "gram_leg_reduce", "reconstruct",
  "householder_tsqr", "factor", "core_svd", "env_factor", "vec_contract", "msg_finish", "other",
  "bp_leg_contract", "bp_env_eig"};

struct Work { double bytes = 0, flops = 0; };

inline int iv(const pepo_ctx* c, int idx) { return c->ival_snap[idx]; }

void view_dims(const pepo_ctx* c, const TView& v, long long* d) {
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = k < v.nlegs ? iv(c, v.dim[k]) : 1;
}

// algorithmic bytes / FLOPs of one launch from its host item copies
Work work_of(const pepo_ctx* c, int cls, const void* items, int n) {
  Work w;
  if (c->ival_snap.empty() || !items) return w;
  const double ts = (double)c->tsize;
  for (int i = 0; i < n; ++i) {
    long long d[PEPO_MAXLEG];
    if (cls == K_LEG || cls == K_BP_LEG) {
      const LegItem& it = static_cast<const LegItem*>(items)[i];
      view_dims(c, it.in, d);
      double in = 4;
      for (int k = 0; k < it.in.nlegs; ++k) in *= d[k];
      double out = in / d[it.leg] * iv(c, it.out_dim);
      w.bytes += (in + out) * ts;
      w.flops += 2.0 * out * d[it.leg];
    } else if (cls == K_GRAM_ROWS) {
      const GramRowsItem& it = static_cast<const GramRowsItem*>(items)[i];
      if (it.active >= 0 && iv(c, it.active) == 0) continue;
      view_dims(c, it.x, d);
      double F = 4.0 * d[it.x.nlegs - 1], K = 1;
      for (int k = 0; k + 1 < it.x.nlegs; ++k) K *= d[k];
      w.bytes += K * F * ts;
      w.flops += K * F * (F + 1);
    } else if (cls == K_GRAM_LEG) {
      const GramLegItem& it = static_cast<const GramLegItem*>(items)[i];
      view_dims(c, it.x, d);
      double tot = 4;
      for (int k = 0; k < it.x.nlegs; ++k) tot *= d[k];
      double F = d[it.leg];
      w.bytes += (it.x.ref == it.y_ref ? 1.0 : 2.0) * tot * ts;   // a symmetric Gram reads X once
      w.flops += 2.0 * tot * F;
    } else if (cls == K_RECON) {
      const ReconItem& it = static_cast<const ReconItem*>(items)[i];
      view_dims(c, it.in, d);
      double nin = 4.0 * d[it.in.nlegs - 1], nout = 4.0 * iv(c, it.new_dim), R = 1;
      for (int k = 0; k + 1 < it.in.nlegs; ++k) R *= d[k];
      w.bytes += R * (nin + nout) * ts;
      w.flops += 2.0 * R * nin * nout;
    }
  }
  return w;
}

template <class I> const void* hitems(const pepo_ctx* c, const DArr<I>& a) {
  return c->host_items.empty() ? nullptr : c->host_items.data() + a.off;
}

cudaEvent_t next_event(pepo_ctx* c) {
  if (c->pool_next == c->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->pool.push_back(e);
  }
  return c->pool[c->pool_next++];
}

void timing_begin(pepo_ctx* c) {
  if (!c->timing) return;
  c->ival_snap.assign(c->n_ival, 0);
  cudaMemcpyAsync(c->ival_snap.data(), c->d_ival, sizeof(int) * c->n_ival, cudaMemcpyDeviceToHost,
                  c->stream);
  cudaStreamSynchronize(c->stream);
}

void timing_harvest(pepo_ctx* c) {
  if (c->pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto& t = c->tot[r.cls];
      t.n++;
      t.ms += ms;
      t.bytes += r.bytes;
      t.flops += r.flops;
    }
  }
  c->pending.clear();
  c->pool_next = 0;
}

// A tensor-core kernel's error word was set: report it once and clear it, so
// that the context stays usable (its state is undefined until restored or
// re-uploaded).
pepo_status kernel_error(pepo_ctx* c, int kerr) {
  cudaMemsetAsync(c->d_kerr, 0, sizeof(int), c->stream);
  cudaStreamSynchronize(c->stream);
  return fail(c, PEPO_E_CUDA,
              "tensor-core kernel error word %d (bit 0: a pipeline wait ran longer than the wait limit, "
              "bit 1: missing packed-W workspace, bit 2: an exit drain ran out of time); the state is "
              "undefined until it is restored or uploaded again", kerr);
}

// Every launch wrapper returns without launching when its item count is 0;
// LAUNCH_T counts (and, in timing mode, brackets with events) the launches
// that happen.
#define LAUNCH_T(cls, hptr, n, expr)                                                    \
  do {                                                                                  \
    if ((n) > 0) {                                                                      \
      cudaEvent_t _a = nullptr, _b = nullptr;                                           \
      if (c->timing) { _a = next_event(c); _b = next_event(c); cudaEventRecord(_a, c->stream); } \
      cudaError_t _e = (expr);                                                          \
      c->launches++;                                                                    \
      if (_e != cudaSuccess)                                                            \
        return fail(c, PEPO_E_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));           \
      if (c->timing && _a && _b) {                                                      \
        cudaEventRecord(_b, c->stream);                                                 \
        Work _w = work_of(c, (cls), (hptr), (n));                                       \
        c->pending.push_back({(cls), _a, _b, _w.bytes, _w.flops});                      \
        if (c->pending.size() > 4000) timing_harvest(c);                                \
      }                                                                                 \
    }                                                                                   \
  } while (0)
#define LAUNCH_N(n, expr) LAUNCH_T(K_OTHER, nullptr, n, expr)

// tensor-core split-precision kernels for the FP32-storage mixed mode:
// tcgen05 (TMEM accumulators) for chi_max <= 128, else the FP32 SIMT kernels
template <typename T>
bool use_umma(const pepo_ctx* c, int chimax) {
  return sizeof(T) == 4 && c->prec == PEPO_TF32X3 && umma_supported(chimax);
}
template <typename T>
cudaError_t leg_dispatch(pepo_ctx* c, const LegItem* items, int n, int gx, int chimax) {
  if (use_umma<T>(c, chimax))
    return launch_leg_umma(items, n, chimax, c->d_ptrs, c->d_ival, c->d_kerr, c->wait_ns, c->stream);
  return launch_leg_contract<T>(items, n, gx, chimax, c->d_ptrs, c->d_ival, c->stream);
}
template <typename T>
cudaError_t gram_leg_dispatch(pepo_ctx* c, const GramLegItem* items, int n, int chimax) {
  if (use_umma<T>(c, chimax))
    return launch_gram_umma(items, n, c->tune.gram_leg_splits, chimax, c->d_ptrs, c->d_ival, c->d_kerr, c->wait_ns,
                            c->stream);
  return launch_gram_leg<T>(items, n, c->tune.gram_leg_splits, chimax, c->d_ptrs, c->d_ival, c->stream);
}

template <typename T>
pepo_status run_gate_wave(pepo_ctx* c, Inst& I, GateWave& w) {
  cudaStream_t s = c->stream;
  const int chimax = I.cfg.chi_max;
  const int nmax = 4 * chimax, rmax = PEPO_RG * chimax;
  const long long big = (long long)4 * pow_sz(chimax, 4);
  int gx_leg = (int)std::min<long long>(std::max<long long>(1, big / (long long)(chimax * 64) + 1),
                                        (long long)(2 * 152 * 4 / std::max(1, w.leg[0].n) + 1));
  gx_leg = std::max(gx_leg, 8);
  LAUNCH_T(K_ENV, nullptr, w.env.n, launch_env_factor(w.env.d, w.env.n, chimax, c->d_ival, s));
  LAUNCH_N(w.copy.n, launch_copy<T>(w.copy.d, w.copy_out.d, w.copy.n, 64, c->d_ptrs, c->d_ival, s));
  for (int r = 0; r < 3; ++r)
    LAUNCH_T(K_LEG, hitems(c, w.leg[r]), w.leg[r].n, leg_dispatch<T>(c, w.leg[r].d, w.leg[r].n, gx_leg, chimax));
  LAUNCH_N(w.fac.n, launch_branch(w.fac.d, w.fac.n, c->d_ival, s));
  {
    int nt = ceil_div(nmax, 64);
    LAUNCH_T(K_GRAM_ROWS, hitems(c, w.gram), w.gram.n, launch_gram_rows<T>(w.gram.d, w.gram.n, nt * (nt + 1) / 2, c->tune.gram_rows_splits, 1, c->d_ptrs,
                               c->d_ival, s));
    LAUNCH_T(K_GRAM_ROWS_RED, nullptr, w.gram.n, launch_gram_rows_reduce(w.gram.d, w.gram.n, nmax, c->tune.gram_rows_splits, 1, c->d_ival, s));
  }
  // Householder TSQR of the sites with branch value `pass` (0: the Householder
  // branch; 2: the Cholesky-branch sites whose Gram was too ill-conditioned)
  auto tsqr = [&](int pass) -> pepo_status {
    const long long mmax = (long long)pow_sz(chimax, 3);
    const long long L0 = 256;
    long long nb0 = (mmax + L0 - 1) / L0;
    int levels = 1;
    long long nb = nb0;
    while (nb > 1) { nb = (nb + 3) / 4; ++levels; }
    long long g = nb0;
    for (int l = 0; l < levels; ++l) {
      LAUNCH_T(K_HH, nullptr, w.fac.n, launch_hh_level<T>(w.fac.d, w.fac.n, l, (int)std::max<long long>(g, 1), nmax, c->d_ptrs,
                                c->d_ival, s, pass));
      g = (g + 3) / 4;
    }
    LAUNCH_T(K_HH, nullptr, w.fac.n, launch_hh_extract<T>(w.fac.d, w.fac.n, c->d_ptrs, c->d_ival, s, pass, c->d_hh_acct));
    return PEPO_OK;
  };
  pepo_status st = tsqr(0);
  if (st != PEPO_OK) return st;
  LAUNCH_T(K_FACTOR, nullptr, w.fac.n, launch_form(w.fac.d, w.fac.n, 16, c->d_ival, s, -1));
  LAUNCH_T(K_FACTOR, nullptr, w.fac.n, launch_factor(w.fac.d, w.fac.n, rmax, nmax, c->d_ival, s, -1, c->d_qr_count));
  // the sites k_factor handed back (branch 2): Householder on the same absorbed
  // tensor, which the Gram only read
  st = tsqr(2);
  if (st != PEPO_OK) return st;
  LAUNCH_T(K_FACTOR, nullptr, w.fac.n, launch_form(w.fac.d, w.fac.n, 16, c->d_ival, s, 2));
  LAUNCH_T(K_FACTOR, nullptr, w.fac.n, launch_factor(w.fac.d, w.fac.n, rmax, nmax, c->d_ival, s, 2, nullptr));
  return PEPO_OK;
}

// after the colour's bond core: reconstruct into the next layout, commit
template <typename T>
pepo_status run_gate_wave_tail(pepo_ctx* c, Inst& I, GateWave& w) {
  cudaStream_t s = c->stream;
  const int chimax = I.cfg.chi_max;
  const int nmax = 4 * chimax;
  {
    long long rows = (long long)pow_sz(chimax, 3);
    int gx = (int)std::min<long long>(std::max<long long>(1, (rows + 63) / 64 * ceil_div(nmax, 64)),
                                      (long long)(2 * 152 * 4 / std::max(1, w.recon.n) + 1));
    gx = std::max(gx, 4);
    if (use_umma<T>(c, chimax))
      LAUNCH_T(K_RECON, hitems(c, w.recon), w.recon.n,
               launch_recon_umma(w.recon.d, w.recon.n, chimax, c->d_ptrs, c->d_ival, c->d_kerr, c->wait_ns, s));
    else
      LAUNCH_T(K_RECON, hitems(c, w.recon), w.recon.n,
               launch_reconstruct<T>(w.recon.d, w.recon.n, gx, 0, c->d_ptrs, c->d_ival, s));
  }
  LAUNCH_N(w.npairs, launch_commit(w.pairs.d, w.npairs, w.moves.d, w.nmoves, c->d_ptrs, c->d_ival, s));
  return PEPO_OK;
}

template <typename T>
pepo_status run_bp_waves(pepo_ctx* c, Inst& I, std::vector<BpWave>& waves) {
  cudaStream_t s = c->stream;
  const int chimax = I.cfg.chi_max;
  for (auto& w : waves) {
    LAUNCH_T(K_BP_EIG, nullptr, w.eig.n, launch_env_eig(w.eig.d, w.eig.n, chimax, c->tsize == 4 ? 1 : 0, c->d_ival, s));
    for (int a = 0; a < 4; ++a) {
      int gx = std::max(8, 2 * 152 * 4 / std::max(1, w.leg[a].n));
      LAUNCH_T(K_BP_LEG, hitems(c, w.leg[a]), w.leg[a].n,
               leg_dispatch<T>(c, w.leg[a].d, w.leg[a].n, gx, chimax));
    }
    LAUNCH_T(K_GRAM_LEG, hitems(c, w.gram), w.gram.n,
             gram_leg_dispatch<T>(c, w.gram.d, w.gram.n, chimax));
    LAUNCH_T(K_GRAM_LEG_RED, nullptr, w.gram.n,
             launch_gram_leg_reduce(w.gram.d, w.gram.n, chimax, c->tune.gram_leg_splits, use_umma<T>(c, chimax) ? 1 : 0,
                                    c->d_ival, s));
    LAUNCH_T(K_MSG, nullptr, w.rot.n, launch_rotate_back(w.rot.d, w.rot.n, chimax, c->d_ival, s));
    if (w.pw.n > 0) {
      LAUNCH_T(K_OTHER, nullptr, w.pw.n, launch_pauli_weights<T>(w.pw.d, w.pw.n, c->d_ptrs, c->d_ival, s));
      c->launches++;   // the zeroing kernel
    }
  }
  return PEPO_OK;
}

template <typename T>
pepo_status run_sl_pass(pepo_ctx* c, Inst& I) {
  for (int l = 0; l < 4; ++l) {
    if (I.sl[l].items.n == 0) continue;
    LAUNCH_T(K_VEC, nullptr, I.sl[l].items.n, launch_vec_contract<T>(I.sl[l].items.d, I.sl[l].items.n, 256, c->d_ptrs, c->d_ival, c->stream));
  }
  return PEPO_OK;
}

// the bond gates of one colour class on every instance (grouped launches)
template <typename T>
pepo_status colour_launches(pepo_ctx* c, int col) {
  Inst& G = c->grp;
  for (auto& w : G.gwaves[col]) {
    pepo_status st = run_gate_wave<T>(c, G, w);
    if (st != PEPO_OK) return st;
  }
  LAUNCH_T(K_CORE, nullptr, G.gcore[col].n, launch_core(G.gcore[col].d, G.gcore[col].n, c->d_ival, c->d_flags, c->stream));
  for (auto& w : G.gwaves[col]) {
    pepo_status st = run_gate_wave_tail<T>(c, G, w);
    if (st != PEPO_OK) return st;
  }
  return PEPO_OK;
}

// one Trotter step of every instance
template <typename T>
pepo_status step_launches(pepo_ctx* c) {
  for (int col = 0; col < 4; ++col) {
    pepo_status st = colour_launches<T>(c, col);
    if (st != PEPO_OK) return st;
  }
  return PEPO_OK;
}

// Capture `body` (launches on c->stream) into a graph on the private capture
// stream; returns false (and launches nothing) when capture is not possible.
template <class F>
bool capture_graph(pepo_ctx* c, cudaGraphExec_t* exec, long long* nlaunch, F body) {
  if (c->graphs_failed || c->cap_stream == nullptr) return false;
  cudaStream_t user = c->stream;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    c->graphs_failed = true;
    cudaGetLastError();
    return false;
  }
  c->stream = c->cap_stream;
  const long long l0 = c->launches;
  const pepo_status st = body();
  c->stream = user;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  *nlaunch = c->launches - l0;
  c->launches = l0;
  if (st != PEPO_OK || e != cudaSuccess || g == nullptr ||
      cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    *exec = nullptr;
    c->graphs_failed = true;
    cudaGetLastError();
    return false;
  }
  cudaGraphDestroy(g);
  return true;
}

template <typename T>
pepo_status do_steps(pepo_ctx* c, int n) {
  for (int step = 0; step < n; ++step) {
    bool done = false;
    if (!c->timing) {
      if (!c->step_exec) capture_graph(c, &c->step_exec, &c->step_launches, [&] { return step_launches<T>(c); });
      if (c->step_exec) {
        if (cudaGraphLaunch(c->step_exec, c->stream) != cudaSuccess)
          return fail(c, PEPO_E_CUDA, "step graph launch: %s", cudaGetErrorString(cudaGetLastError()));
        c->launches += c->step_launches;
        done = true;
      }
    }
    if (!done) {
      pepo_status st = step_launches<T>(c);
      if (st != PEPO_OK) return st;
    }
    for (auto& I : c->inst) I.steps++;
  }
  c->stepped = true;
  return PEPO_OK;
}

double bits_to_double(unsigned long long u) {
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}

// one double-layer BP sweep of every active instance
template <typename T>
pepo_status bp_sweep_launches(pepo_ctx* c) {
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(c->d_delta2, 0, sizeof(unsigned long long) * c->n_inst, s) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "memset delta");
  pepo_status st = run_bp_waves<T>(c, c->grp, c->grp.bwaves);
  if (st != PEPO_OK) return st;
  LAUNCH_T(K_MSG, nullptr, c->grp.msgs.n,
           launch_bp_finish(c->grp.msgs.d, c->grp.msgs.n, c->d_ival, c->d_active, c->d_delta2, c->d_flags, s));
  return PEPO_OK;
}

template <typename T>
pepo_status do_bp(pepo_ctx* c, int* sweeps_out, double* delta_out) {
  cudaStream_t s = c->stream;
  std::vector<int> done(c->n_inst, 0), sweeps(c->n_inst, 0), active(c->n_inst, 1);
  std::vector<double> delta(c->n_inst, INFINITY);
  std::vector<unsigned long long> hd(c->n_inst);
  int maxs = 0;
  for (auto& I : c->inst) maxs = std::max(maxs, I.cfg.bp_max_sweeps);
  for (int sw = 1; sw <= maxs; ++sw) {
    bool any = false;
    for (int i = 0; i < c->n_inst; ++i) {
      active[i] = (!done[i] && sw <= c->inst[i].cfg.bp_max_sweeps) ? 1 : 0;
      any = any || active[i];
    }
    if (!any) break;
    if (cudaMemcpyAsync(c->d_active, active.data(), sizeof(int) * c->n_inst, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "active mask upload");
    bool launched = false;
    if (!c->timing) {
      if (!c->bp_exec) capture_graph(c, &c->bp_exec, &c->bp_launches, [&] { return bp_sweep_launches<T>(c); });
      if (c->bp_exec) {
        if (cudaGraphLaunch(c->bp_exec, s) != cudaSuccess)
          return fail(c, PEPO_E_CUDA, "BP graph launch: %s", cudaGetErrorString(cudaGetLastError()));
        c->launches += c->bp_launches;
        launched = true;
      }
    }
    if (!launched) {
      pepo_status st = bp_sweep_launches<T>(c);
      if (st != PEPO_OK) return st;
    }
    int kerr = 0;
    if (cudaMemcpyAsync(hd.data(), c->d_delta2, sizeof(unsigned long long) * c->n_inst,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&kerr, c->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "BP delta readback: %s", cudaGetErrorString(cudaGetLastError()));
    if (kerr) return kernel_error(c, kerr);
    for (int i = 0; i < c->n_inst; ++i) {
      if (!active[i]) continue;
      Inst& I = c->inst[i];
      sweeps[i] = sw;
      delta[i] = bits_to_double(hd[i]);
      if (delta[i] < I.cfg.bp_tol || sw == I.cfg.bp_max_sweeps) done[i] = 1;
    }
  }
  for (int i = 0; i < c->n_inst; ++i) {
    c->inst[i].last_sweeps = sweeps[i];
    c->inst[i].last_delta = delta[i];
    if (sweeps_out) sweeps_out[i] = sweeps[i];
    if (delta_out) delta_out[i] = delta[i];
  }
  return PEPO_OK;
}

template <typename T>
pepo_status sl_sweep_launches(pepo_ctx* c) {
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(c->d_delta1, 0, sizeof(unsigned long long) * c->n_inst, s) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "memset delta");
  pepo_status st = run_sl_pass<T>(c, c->grp);
  if (st != PEPO_OK) return st;
  LAUNCH_T(K_MSG, nullptr, c->grp.msgs.n,
           launch_sl_finish(c->grp.msgs.d, c->grp.msgs.n, c->d_ival, c->d_active, c->d_delta1, s));
  return PEPO_OK;
}

template <typename T>
pepo_status do_correlator(pepo_ctx* c, double* C_out, pepo_diag* diag_out) {
  cudaStream_t s = c->stream;
  Inst& G = c->grp;
  LAUNCH_N(G.msgs.n, launch_sl_init(G.msgs.d, G.msgs.n, c->d_ival, s));
  std::vector<int> done(c->n_inst, 0), sweeps(c->n_inst, 0), active(c->n_inst, 1);
  std::vector<double> delta(c->n_inst, INFINITY);
  std::vector<unsigned long long> hd(c->n_inst);
  int maxs = 0;
  for (auto& I : c->inst) maxs = std::max(maxs, I.cfg.bp_max_sweeps);
  for (int sw = 1; sw <= maxs; ++sw) {
    bool any = false;
    for (int i = 0; i < c->n_inst; ++i) {
      active[i] = (!done[i] && sw <= c->inst[i].cfg.bp_max_sweeps) ? 1 : 0;
      any = any || active[i];
    }
    if (!any) break;
    if (cudaMemcpyAsync(c->d_active, active.data(), sizeof(int) * c->n_inst, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "active mask upload");
    bool launched = false;
    if (!c->timing) {
      if (!c->sl_exec) capture_graph(c, &c->sl_exec, &c->sl_launches, [&] { return sl_sweep_launches<T>(c); });
      if (c->sl_exec) {
        if (cudaGraphLaunch(c->sl_exec, s) != cudaSuccess)
          return fail(c, PEPO_E_CUDA, "single-layer graph launch: %s", cudaGetErrorString(cudaGetLastError()));
        c->launches += c->sl_launches;
        launched = true;
      }
    }
    if (!launched) {
      pepo_status st = sl_sweep_launches<T>(c);
      if (st != PEPO_OK) return st;
    }
    int kerr = 0;
    if (cudaMemcpyAsync(hd.data(), c->d_delta1, sizeof(unsigned long long) * c->n_inst,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&kerr, c->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "single-layer delta readback");
    if (kerr) return kernel_error(c, kerr);
    for (int i = 0; i < c->n_inst; ++i) {
      if (!active[i]) continue;
      Inst& I = c->inst[i];
      sweeps[i] = sw;
      delta[i] = bits_to_double(hd[i]);
      if (delta[i] < I.cfg.bp_tol || sw == I.cfg.bp_max_sweeps) done[i] = 1;
    }
  }
  // final estimates from the converged messages, then the Bethe sums
  {
    pepo_status st = run_sl_pass<T>(c, G);
    if (st != PEPO_OK) return st;
    st = run_bp_waves<T>(c, G, G.fwaves);
    if (st != PEPO_OK) return st;
    LAUNCH_N(G.sscal.n, launch_site_scalars(G.sscal.d, G.sscal.n, c->d_ival, s));
    LAUNCH_N(G.escal.n, launch_edge_scalars(G.escal.d, G.escal.n, c->d_ival, s));
    LAUNCH_N(G.bethe.n, launch_bethe(G.bethe.d, G.bethe.n, s));
  }
  std::vector<int> flags(c->n_inst);
  int kerr = 0;
  if (cudaMemcpyAsync(flags.data(), c->d_flags, sizeof(int) * c->n_inst, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(&kerr, c->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "flags readback");
  if (kerr) return kernel_error(c, kerr);
  for (int i = 0; i < c->n_inst; ++i) {
    Inst& I = c->inst[i];
    double out[8];
    std::vector<double> disc(I.nb), lam((size_t)I.nb * I.cfg.chi_max);
    std::vector<int> chi(I.nb), csw(2 * (size_t)I.nb);
    if (cudaMemcpyAsync(out, I.bethe_out, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(csw.data(), I.core_sweeps, sizeof(int) * csw.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(disc.data(), I.disc, sizeof(double) * I.nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(lam.data(), I.lam, sizeof(double) * lam.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(chi.data(), c->d_ival + I.chi0, sizeof(int) * I.nb, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "result readback");
    if (cudaStreamSynchronize(s) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "correlator: %s", cudaGetErrorString(cudaGetLastError()));
    I.last_sweeps1 = sweeps[i];
    I.last_delta1 = delta[i];
    if (C_out) C_out[i] = out[0];
    double ge = 0.0;
    if (I.steps > 0) for (double x : disc) ge += x;
    // previous layer: the last measurement at a smaller step count (a repeated
    // measurement of the same layer keeps the layer before it)
    if (I.meas_valid && I.meas_steps < I.steps) {
      I.prev_valid = 1;
      I.prev_C = I.meas_C;
      I.prev_ge = I.meas_ge;
    }
    const int drop = I.prev_valid ? pepo_c_drop(I.prev_C, I.prev_ge, out[0], ge) : 0;
    I.meas_valid = 1;
    I.meas_steps = I.steps;
    I.meas_C = out[0];
    I.meas_ge = ge;
    if (diag_out) {
      pepo_diag& d = diag_out[i];
      std::memset(&d, 0, sizeof d);
      d.C = out[0];
      d.C_proj = out[1];
      d.log_norm = out[4];
      d.gate_err = ge;
      d.c_drop = drop;
      d.bp_sweeps = I.last_sweeps;
      d.bp_delta = I.last_delta;
      d.bp1_sweeps = sweeps[i];
      d.bp1_delta = delta[i];
      double ef = 0.0;
      for (int b = 0; b < I.nb; ++b) {
        if (chi[b] < 2) continue;
        double S = 0.0;
        for (int k = 0; k < chi[b]; ++k) {
          double l2 = lam[(size_t)b * I.cfg.chi_max + k];
          l2 *= l2;
          if (l2 > 0.0) S -= l2 * std::log(l2);
        }
        ef = std::max(ef, S / std::log((double)chi[b]));
      }
      d.entropy_frac_max = ef;
      d.trap_type1 = (I.last_sweeps >= 30 && I.last_delta < I.cfg.bp_tol) ? 1 : 0;
      d.trap_type2 = (I.last_sweeps >= I.cfg.bp_max_sweeps && !(I.last_delta < I.cfg.bp_tol)) ? 1 : 0;
      d.norm_exploded = (out[4] >= std::log(2.0)) ? 1 : 0;
      d.flags = flags[i];
      d.steps = I.steps;
      for (int b = 0; b < I.nb; ++b) {
        d.core_sweeps32_max = std::max(d.core_sweeps32_max, csw[2 * (size_t)b]);
        d.core_sweeps64_max = std::max(d.core_sweeps64_max, csw[2 * (size_t)b + 1]);
      }
    }
  }
  return PEPO_OK;
}

// canonical position of each layout leg for site v at step boundaries
std::vector<int> boundary_layout(const SiteG& S) { return layout_for(S, S.upd[0]); }

// Layout of site v after `phase` colours of the current step: the cut of its
// next update innermost (the step-boundary layout once every bond of the site
// has been updated, or none yet).
std::vector<int> phase_layout(const Inst& I, const SiteG& S, int phase) {
  int done = 0;
  for (int k : S.upd)
    if (I.bonds[S.legs[k].bond].colour < phase) ++done;
  return layout_for(S, S.upd[done % (int)S.upd.size()]);
}

// calls that need whole steps (BP, the correlator, state uploads and
// snapshots, the warm start) refuse a partly applied step
bool at_step_boundary(pepo_ctx* c, const char* what) {
  if (c->phase == 0) return true;
  fail(c, PEPO_E_STATE, "%s: a Trotter step is partly applied (colours 0..%d); apply the remaining "
       "colours with pepo_trotter_colour first", what, c->phase - 1);
  return false;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int pepo_c_drop(double C_prev, double gate_err_prev, double C, double gate_err) {
  if (!std::isfinite(C_prev) || !std::isfinite(C) || !std::isfinite(gate_err_prev) || !std::isfinite(gate_err))
    return 0;
  const bool dropped = std::fabs(C) < 0.5 * std::fabs(C_prev);
  const bool jump = gate_err > 2.0 * std::max(gate_err_prev, 1e-12);
  return (dropped && !jump) ? 1 : 0;
}

void pepo_config_default(pepo_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->Lx = 3;
  cfg->Ly = 3;
  cfg->J = 1.0;
  cfg->h = 1.0;
  cfg->dt = 0.05;
  cfg->trotter_order = 1;
  cfg->obs_x = 1;
  cfg->obs_y = 1;
  cfg->obs_pauli = 3;
  cfg->chi_max = 8;
  cfg->eps_cut = 1e-11;
  cfg->bp_alpha = 0.5;
  cfg->bp_tol = 1e-5;
  cfg->bp_max_sweeps = 100;
  cfg->qr_n_thresh = 150;
  cfg->qr_ratio_thresh = 150.0;
  cfg->pinv_rel = 1e-12;
  cfg->gates = PEPO_GATES_ZZ_X;
  cfg->prec = PEPO_FP32;
  cfg->warm_start = 0;
  cfg->inflight_sites = 0;
}

static bool setup_ctx(pepo_ctx* c, const pepo_config* cfgs, int n_inst, std::string& why) {
  c->n_inst = n_inst;
  c->inst.assign(n_inst, Inst());
  c->prec = cfgs[0].prec;
  for (int i = 0; i < n_inst; ++i) {
    why = validate(cfgs[i]);
    if (!why.empty()) { why = "instance " + std::to_string(i) + ": " + why; return false; }
    if (cfgs[i].prec != c->prec) { why = "all instances must share one precision"; return false; }
    c->inst[i].cfg = cfgs[i];
    build_geometry(c->inst[i]);
    c->chimax = std::max(c->chimax, cfgs[i].chi_max);
  }
  c->tsize = (c->prec == PEPO_FP64) ? 8 : 4;
  return true;
}

size_t pepo_required_bytes(const pepo_config* cfgs, int n_inst) {
  if (!cfgs || n_inst < 1) return 0;
  pepo_ctx c;
  std::string why;
  if (!setup_ctx(&c, cfgs, n_inst, why)) return 0;
  return layout_arena(&c, nullptr, nullptr);
}

pepo_status pepo_init(const pepo_config* cfgs, int n_inst, void* dev_arena, size_t arena_bytes,
                      void* cuda_stream, pepo_ctx** out) {
  if (!out) return PEPO_E_INVALID;
  *out = nullptr;
  if (!cfgs || n_inst < 1 || !dev_arena) return PEPO_E_INVALID;
  if (reinterpret_cast<uintptr_t>(dev_arena) % kAlign != 0) return PEPO_E_INVALID;
  pepo_ctx* c = new pepo_ctx();
  std::string why;
  if (!setup_ctx(c, cfgs, n_inst, why)) { delete c; return PEPO_E_INVALID; }
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  size_t need = layout_arena(c, nullptr, nullptr);
  if (need == 0) { delete c; return PEPO_E_INVALID; }
  if (arena_bytes < need) { delete c; return PEPO_E_OOM; }
  // real layout
  for (auto& I : c->inst) {
    for (int col = 0; col < 4; ++col) I.gwaves[col].clear();
    I.bwaves.clear();
    I.fwaves.clear();
  }
  Planner P;
  c->arena = static_cast<char*>(dev_arena);
  c->arena_bytes = arena_bytes;
  layout_arena(c, c->arena, &P);
  finalize_items(c, P);
  c->host_items = P.st.bytes;
  c->tot.assign(K_NCLASS, pepo_ctx::Tot());
  cudaStream_t s = c->stream;
  bool ok = cudaMemcpyAsync(c->d_ptrs, P.ptr_init.data(), sizeof(void*) * P.ptr_init.size(),
                            cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(c->d_ival, P.ival_init.data(), sizeof(int) * P.ival_init.size(),
                             cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(c->d_items, P.st.bytes.data(), P.st.bytes.size(), cudaMemcpyHostToDevice,
                             s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->d_flags, 0, sizeof(int) * n_inst, s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->d_kerr, 0, sizeof(int), s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->d_qr_count, 0, 3 * sizeof(unsigned long long), s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->d_hh_acct, 0, 2 * sizeof(double), s) == cudaSuccess;
  for (auto& I : c->inst)   // Pauli weights read as zero rows until the first correlator call
    ok = ok && cudaMemsetAsync(I.pw, 0, sizeof(double) * 4 * (size_t)I.N, s) == cudaSuccess;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap_stream = nullptr;   // graphs off; launches go to the stream directly
    cudaGetLastError();
  }
  resolve_all(c);
  // initial state (Sec. 2.3): chi = 1 everywhere, observable Pauli at c, I elsewhere
  for (auto& I : c->inst) {
    const int chimax = I.cfg.chi_max;
    for (int v = 0; v < I.N && ok; ++v) {
      double e[4] = {0, 0, 0, 0};
      e[I.sites[v].pin] = 1.0;
      if (c->tsize == 8) {
        ok = cudaMemcpyAsync(I.site_slab[v], e, sizeof e, cudaMemcpyHostToDevice, s) == cudaSuccess;
      } else {
        float f[4] = {(float)e[0], (float)e[1], (float)e[2], (float)e[3]};
        ok = cudaMemcpyAsync(I.site_slab[v], f, sizeof f, cudaMemcpyHostToDevice, s) == cudaSuccess;
      }
    }
    std::vector<double> lam((size_t)I.nb * chimax, 0.0), msg((size_t)2 * I.nb * chimax * chimax, 0.0);
    for (int b = 0; b < I.nb; ++b) lam[(size_t)b * chimax] = 1.0;
    for (int id = 0; id < 2 * I.nb; ++id) msg[(size_t)id * chimax * chimax] = 1.0;
    ok = ok && cudaMemcpyAsync(I.lam, lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(I.msg, msg.data(), sizeof(double) * msg.size(), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(I.sigma, 0, sizeof(double) * I.N, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(I.disc, 0, sizeof(double) * I.nb, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(I.core_sweeps, 0, sizeof(int) * 2 * I.nb, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(I.vec, 0, sizeof(double) * 2 * I.nb * chimax, s) == cudaSuccess;
    {
      // warm-start geometry of every directed bond (source = v1 for dir 0)
      std::vector<WsGeom> geom(2 * (size_t)I.nb);
      std::vector<int> deg(I.N, 0);
      for (int v = 0; v < I.N; ++v) deg[v] = I.sites[v].deg;
      const int Lx = I.cfg.Lx;
      const float norm = (float)(I.cfg.Lx + I.cfg.Ly);
      auto dist = [&](int v) { return (float)(std::abs(v % Lx - I.cfg.obs_x) + std::abs(v / Lx - I.cfg.obs_y)) / norm; };
      for (int b = 0; b < I.nb; ++b)
        for (int dir = 0; dir < 2; ++dir) {
          const int src = dir == 0 ? I.bonds[b].v1 : I.bonds[b].v2;
          const int dst = dir == 0 ? I.bonds[b].v2 : I.bonds[b].v1;
          WsGeom g{};
          for (int k = 0; k < I.sites[src].deg; ++k) {
            const int e = I.sites[src].legs[k].bond;
            if (e != b && g.n_other < 3) g.other[g.n_other++] = e;
          }
          g.deg_src = (float)deg[src];
          g.deg_dst = (float)deg[dst];
          g.dist_src = dist(src);
          g.dist_dst = dist(dst);
          geom[2 * (size_t)b + dir] = g;
        }
      ok = ok && cudaMemcpyAsync(I.ws_geom, geom.data(), sizeof(WsGeom) * geom.size(), cudaMemcpyHostToDevice,
                                 s) == cudaSuccess;
    }
    if (ok && launch_gates(I.gates.d, I.gates.n, s) != cudaSuccess) ok = false;
    c->launches++;
  }
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    delete c;
    return PEPO_E_CUDA;
  }
  int flags = 0;
  cudaMemcpy(&flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost);
  if (flags & 8) { delete c; return PEPO_E_INVALID; }   // gate rank above the bound
  *out = c;
  return PEPO_OK;
}

pepo_status pepo_trotter_step(pepo_ctx* c, int n_steps) {
  if (!c) return PEPO_E_INVALID;
  if (n_steps < 0) return fail(c, PEPO_E_INVALID, "n_steps must be >= 0");
  if (!at_step_boundary(c, "pepo_trotter_step")) return PEPO_E_STATE;
  timing_begin(c);
  pepo_status st = c->tsize == 8 ? do_steps<double>(c, n_steps) : do_steps<float>(c, n_steps);
  return st;
}

pepo_status pepo_trotter_colour(pepo_ctx* c, int colour) {
  if (!c) return PEPO_E_INVALID;
  if (colour < 0 || colour > 3) return fail(c, PEPO_E_INVALID, "colour must lie in 0..3, got %d", colour);
  if (colour != c->phase)
    return fail(c, PEPO_E_STATE, "colour %d out of order: the current step has colours 0..%d applied, "
                "the next is %d", colour, c->phase - 1, c->phase);
  timing_begin(c);
  pepo_status st = c->tsize == 8 ? colour_launches<double>(c, colour) : colour_launches<float>(c, colour);
  if (st != PEPO_OK) return st;
  c->phase = (colour + 1) % 4;
  if (c->phase == 0) {
    for (auto& I : c->inst) I.steps++;
    c->stepped = true;
  }
  return PEPO_OK;
}

// The learned warm start of the instances with warm_start = 1: features of
// the current state, the network's prediction of the converged message
// diagonals, and the blended diagonal start (gamma 0.25) written into their
// messages before the BP sweeps.  The forward pass runs over the instance's
// row capacity (2 nb chi_max); the features and the writer use the live rows
// only, so the rows beyond them are never read.
static pepo_status ws_apply_all(pepo_ctx* c) {
  constexpr float kGamma = 0.25f;
  for (int i = 0; i < c->n_inst; ++i) {
    Inst& I = c->inst[i];
    if (!I.cfg.warm_start) continue;
    const int cap = 2 * I.nb * I.cfg.chi_max;
    const float t = (float)(I.steps * I.cfg.dt);
    cudaError_t e = launch_ws_features(I.ws_geom, I.nb, c->d_ival + I.chi0, I.lam, I.cfg.chi_max, t,
                                       (float)I.cfg.h, (float)I.cfg.J, c->ws_X, cap, c->stream);
    if (e == cudaSuccess) e = mlp_forward(c->ws_mlp, c->ws_X, cap, c->ws_y, c->stream);
    if (e == cudaSuccess)
      e = launch_ws_apply(I.nb, c->d_ival + I.chi0, c->ws_y, I.msg, I.cfg.chi_max, kGamma, c->stream);
    c->launches += 3;
    if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "warm start: %s", cudaGetErrorString(e));
  }
  return PEPO_OK;
}

pepo_status pepo_bp_converge(pepo_ctx* c, int* sweeps_out, double* delta_out) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_bp_converge")) return PEPO_E_STATE;
  if (c->ws_ready) {
    const pepo_status ws = ws_apply_all(c);
    if (ws != PEPO_OK) return ws;
  }
  timing_begin(c);
  pepo_status st = c->tsize == 8 ? do_bp<double>(c, sweeps_out, delta_out) : do_bp<float>(c, sweeps_out, delta_out);
  timing_harvest(c);
  return st;
}

pepo_status pepo_correlator(pepo_ctx* c, double* C_out, pepo_diag* diag_out) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_correlator")) return PEPO_E_STATE;
  timing_begin(c);
  pepo_status st = c->tsize == 8 ? do_correlator<double>(c, C_out, diag_out) : do_correlator<float>(c, C_out, diag_out);
  timing_harvest(c);
  return st;
}

pepo_status pepo_get_spectrum(pepo_ctx* c, int inst, int bond, double* lam_out, int* chi_out) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (bond < 0 || bond >= I.nb || !lam_out || !chi_out) return fail(c, PEPO_E_INVALID, "bad bond");
  if (cudaMemcpyAsync(lam_out, I.lam + (size_t)bond * I.cfg.chi_max, sizeof(double) * I.cfg.chi_max,
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(chi_out, c->d_ival + I.chi0 + bond, sizeof(int), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "spectrum readback");
  return PEPO_OK;
}

// layout <-> canonical conversion helpers (host side, not on the hot path)
static void layout_strides(const std::vector<int>& dims_layout, std::vector<size_t>& st) {
  st.assign(dims_layout.size(), 0);
  size_t s = 4;
  for (int k = (int)dims_layout.size() - 1; k >= 0; --k) { st[k] = s; s *= dims_layout[k]; }
}

pepo_status pepo_get_site(pepo_ctx* c, int inst, int site, double* out, size_t count, int* dims_out) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (site < 0 || site >= I.N || !out || !dims_out) return fail(c, PEPO_E_INVALID, "bad site");
  std::vector<int> chi(I.nb);
  void* ptr = nullptr;
  double sigma = 0.0;
  if (cudaMemcpyAsync(chi.data(), c->d_ival + I.chi0, sizeof(int) * I.nb, cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(&ptr, c->d_ptrs + I.site_ref0 + site, sizeof(void*), cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(&sigma, I.sigma + site, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "site readback");
  const SiteG& S = I.sites[site];
  std::vector<int> lay = phase_layout(I, S, c->phase);
  std::vector<int> dl(S.deg), dc(S.deg);
  size_t n = 4;
  for (int k = 0; k < S.deg; ++k) { dl[k] = chi[S.legs[lay[k]].bond]; dc[k] = chi[S.legs[k].bond]; n *= dc[k]; }
  for (int k = 0; k < 4; ++k) dims_out[k] = 0;
  for (int k = 0; k < S.deg; ++k) dims_out[S.legs[k].name] = dc[k];
  if (count < n) return fail(c, PEPO_E_INVALID, "output too small (%zu < %zu)", count, n);
  std::vector<double> raw(n);
  if (c->tsize == 8) {
    if (cudaMemcpy(raw.data(), ptr, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "site copy");
  } else {
    std::vector<float> f(n);
    if (cudaMemcpy(f.data(), ptr, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "site copy");
    for (size_t i = 0; i < n; ++i) raw[i] = f[i];
  }
  std::vector<size_t> sl;
  layout_strides(dl, sl);
  const double scale = std::exp(sigma);
  // canonical index iteration
  std::vector<int> idx(S.deg, 0);
  for (size_t e = 0; e < n / 4; ++e) {
    size_t rem = e;
    for (int k = S.deg - 1; k >= 0; --k) { idx[k] = (int)(rem % dc[k]); rem /= dc[k]; }
    size_t src = 0;
    for (int k = 0; k < S.deg; ++k) {
      int canon = lay[k];
      src += (size_t)idx[canon] * sl[k];
    }
    for (int p = 0; p < 4; ++p) out[e * 4 + p] = raw[src + p] * scale;
  }
  return PEPO_OK;
}

pepo_status pepo_set_bonds(pepo_ctx* c, int inst, const int* chi, const double* lam, const double* msgs) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_set_bonds")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (!chi || !lam || !msgs) return fail(c, PEPO_E_INVALID, "null argument");
  const int chimax = I.cfg.chi_max;
  for (int b = 0; b < I.nb; ++b)
    if (chi[b] < 1 || chi[b] > chimax) return fail(c, PEPO_E_INVALID, "chi of bond %d out of range", b);
  std::vector<int> chiv(chi, chi + I.nb);
  I.meas_valid = I.prev_valid = 0;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(c->d_ival + I.chi0, chiv.data(), sizeof(int) * I.nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_ival + I.pend0, chiv.data(), sizeof(int) * I.nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(I.lam, lam, sizeof(double) * I.nb * chimax, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(I.msg, msgs, sizeof(double) * 2 * I.nb * chimax * chimax, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "bond upload");
  return PEPO_OK;
}

pepo_status pepo_set_site(pepo_ctx* c, int inst, int site, const void* data, int dtype, size_t count) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_set_site")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (site < 0 || site >= I.N || !data || (dtype != 0 && dtype != 1))
    return fail(c, PEPO_E_INVALID, "bad site upload arguments");
  I.meas_valid = I.prev_valid = 0;
  const SiteG& S = I.sites[site];
  std::vector<int> chi(I.nb);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(chi.data(), c->d_ival + I.chi0, sizeof(int) * I.nb, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "chi readback");
  int dc[4] = {1, 1, 1, 1}, perm[4] = {0, 0, 0, 0};
  size_t n = 4;
  for (int k = 0; k < S.deg; ++k) { dc[k] = chi[S.legs[k].bond]; n *= dc[k]; }
  if (count != n) return fail(c, PEPO_E_INVALID, "site %d needs %zu elements, got %zu", site, n, count);
  std::vector<int> lay = boundary_layout(S);
  for (int k = 0; k < S.deg; ++k) perm[k] = lay[k];
  void* ptrs[2] = {nullptr, nullptr};
  if (cudaMemcpy(&ptrs[0], c->d_ptrs + I.site_ref0 + site, sizeof(void*), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&ptrs[1], c->d_ptrs + I.scratch_ref[S.deg], sizeof(void*), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "pointer readback");
  const size_t ts = c->tsize;
  cudaError_t e;
  if ((dtype == 0 && ts == 4) || (dtype == 1 && ts == 8)) {
    e = cudaMemcpy(ptrs[1], data, ts * n, cudaMemcpyHostToDevice);
  } else if (ts == 4) {
    std::vector<float> f(n);
    const double* src = static_cast<const double*>(data);
    for (size_t i = 0; i < n; ++i) f[i] = (float)src[i];
    e = cudaMemcpy(ptrs[1], f.data(), 4 * n, cudaMemcpyHostToDevice);
  } else {
    std::vector<double> f(n);
    const float* src = static_cast<const float*>(data);
    for (size_t i = 0; i < n; ++i) f[i] = src[i];
    e = cudaMemcpy(ptrs[1], f.data(), 8 * n, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "site upload");
  e = ts == 4 ? launch_permute<float>(ptrs[1], ptrs[0], S.deg, dc, perm, 1, c->stream)
              : launch_permute<double>(ptrs[1], ptrs[0], S.deg, dc, perm, 1, c->stream);
  c->launches++;
  if (e != cudaSuccess || cudaMemsetAsync(I.sigma + site, 0, sizeof(double), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "site permute");
  return PEPO_OK;
}

// ----------------------------------------------- allocation-free site upload
// pepo_set_site staged through a file-scope device buffer instead of the
// arena's scratch slab.  The buffer's device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) on the first call;
// nothing here allocates host or device memory.  No byte of the buffer needs
// to start at zero: each call writes the first count elements before the
// permutation reads them.  Calls that overlap in time (any contexts on the
// same device) share the buffer and race.
constexpr size_t kStaticStageBytes = (size_t)16 << 20;
constexpr int kStaticMaxDevices = 64;
static __device__ __align__(256) unsigned char g_static_stage[kStaticStageBytes];
static void* g_static_stage_ptr[kStaticMaxDevices];

static pepo_status static_stage(pepo_ctx* c, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices)
    return fail(c, PEPO_E_CUDA, "no current CUDA device for the static staging buffer");
  if (g_static_stage_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_stage);
    if (e != cudaSuccess || p == nullptr)
      return fail(c, PEPO_E_CUDA, "static staging buffer lookup: %s", cudaGetErrorString(e));
    g_static_stage_ptr[dev] = p;
  }
  *out = g_static_stage_ptr[dev];
  return PEPO_OK;
}

pepo_status pepo_set_site_static(pepo_ctx* c, int inst, int site, const void* data, int dtype, size_t count) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_set_site_static")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (site < 0 || site >= I.N || !data || (dtype != 0 && dtype != 1))
    return fail(c, PEPO_E_INVALID, "bad site upload arguments");
  const size_t ts = c->tsize;
  if ((dtype == 0) != (ts == 4))
    return fail(c, PEPO_E_INVALID, "static upload needs the storage type (%s)", ts == 4 ? "float" : "double");
  I.meas_valid = I.prev_valid = 0;
  const SiteG& S = I.sites[site];
  void* stage = nullptr;
  pepo_status st = static_stage(c, &stage);
  if (st != PEPO_OK) return st;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, PEPO_E_CUDA, "stream sync");
  int dc[4] = {1, 1, 1, 1}, perm[4] = {0, 0, 0, 0};
  size_t n = 4;
  for (int k = 0; k < S.deg; ++k) {
    if (cudaMemcpy(&dc[k], c->d_ival + I.chi0 + S.legs[k].bond, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "chi readback");
    n *= (size_t)dc[k];
  }
  if (count != n) return fail(c, PEPO_E_INVALID, "site %d needs %zu elements, got %zu", site, n, count);
  if (n * ts > kStaticStageBytes)
    return fail(c, PEPO_E_INVALID, "site %d needs %zu bytes; the static staging buffer holds %zu", site,
                n * ts, kStaticStageBytes);
  // stored layout at step boundaries: the legs other than the first update's
  // cut in canonical order, then the cut
  const int cut = S.upd[0];
  int p = 0;
  for (int k = 0; k < S.deg; ++k) if (k != cut) perm[p++] = k;
  perm[p] = cut;
  void* dst = nullptr;
  if (cudaMemcpy(&dst, c->d_ptrs + I.site_ref0 + site, sizeof(void*), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "pointer readback");
  cudaError_t e = cudaMemcpyAsync(stage, data, ts * n, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "site upload: %s", cudaGetErrorString(e));
  e = ts == 4 ? launch_permute<float>(stage, dst, S.deg, dc, perm, 1, c->stream)
              : launch_permute<double>(stage, dst, S.deg, dc, perm, 1, c->stream);
  c->launches++;
  if (e != cudaSuccess || cudaMemsetAsync(I.sigma + site, 0, sizeof(double), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "site permute");
  return PEPO_OK;
}

// ------------------------------------------------------- state snapshot
// Device-to-device copy of one instance's state (site tensors at slab
// capacity, live bond dimensions, lambda, messages, single-layer vectors,
// log-scales, discarded weights) to / from a caller buffer.
static size_t state_layout(const pepo_ctx* c, const Inst& I, size_t* off /* 7 entries or null */) {
  size_t o = 0;
  auto sec = [&](int i, size_t bytes) {
    o = (o + 255) / 256 * 256;
    if (off) off[i] = o;
    o += bytes;
  };
  size_t site_bytes = 0;
  for (int v = 0; v < I.N; ++v) site_bytes += 4 * pow_sz(I.cfg.chi_max, I.sites[v].deg) * c->tsize;
  const size_t cm = I.cfg.chi_max;
  sec(0, site_bytes);
  sec(1, sizeof(int) * I.nb);
  sec(2, sizeof(double) * I.nb * cm);
  sec(3, sizeof(double) * 2 * I.nb * cm * cm);
  sec(4, sizeof(double) * 2 * I.nb * cm);
  sec(5, sizeof(double) * I.N);
  sec(6, sizeof(double) * I.nb);
  return o;
}

size_t pepo_state_bytes(const pepo_ctx* c, int inst) {
  if (!c || inst < 0 || inst >= c->n_inst) return 0;
  return state_layout(c, c->inst[inst], nullptr);
}

// host = true: buf is host memory (checkpoint to / restart from the host;
// the copies synchronise the stream), else device memory
static pepo_status state_copy(pepo_ctx* c, int inst, char* buf, size_t bytes, bool save, bool host = false) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, save ? "pepo_save_state" : "pepo_load_state")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst || !buf) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  size_t off[7];
  const size_t need = state_layout(c, I, off);
  if (bytes < need) return fail(c, PEPO_E_INVALID, "state buffer holds %zu bytes, needs %zu", bytes, need);
  std::vector<void*> sp(I.N);
  if (cudaMemcpyAsync(sp.data(), c->d_ptrs + I.site_ref0, sizeof(void*) * I.N, cudaMemcpyDeviceToHost,
                      c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "site pointer readback");
  const cudaMemcpyKind k = !host ? cudaMemcpyDeviceToDevice : (save ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  auto cp = [&](void* dev, size_t o, size_t n) {
    return save ? cudaMemcpyAsync(buf + o, dev, n, k, c->stream) : cudaMemcpyAsync(dev, buf + o, n, k, c->stream);
  };
  const size_t cm = I.cfg.chi_max;
  size_t so = off[0];
  for (int v = 0; v < I.N; ++v) {
    const size_t n = 4 * pow_sz(cm, I.sites[v].deg) * c->tsize;
    if (cp(sp[v], so, n) != cudaSuccess) return fail(c, PEPO_E_CUDA, "site copy");
    so += n;
  }
  if (cp(c->d_ival + I.chi0, off[1], sizeof(int) * I.nb) != cudaSuccess ||
      cp(I.lam, off[2], sizeof(double) * I.nb * cm) != cudaSuccess ||
      cp(I.msg, off[3], sizeof(double) * 2 * I.nb * cm * cm) != cudaSuccess ||
      cp(I.vec, off[4], sizeof(double) * 2 * I.nb * cm) != cudaSuccess ||
      cp(I.sigma, off[5], sizeof(double) * I.N) != cudaSuccess ||
      cp(I.disc, off[6], sizeof(double) * I.nb) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "state copy");
  if (host && cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "state copy: %s", cudaGetErrorString(cudaGetLastError()));
  return PEPO_OK;
}

pepo_status pepo_save_state(pepo_ctx* c, int inst, void* dev_buf, size_t bytes) {
  pepo_status st = state_copy(c, inst, static_cast<char*>(dev_buf), bytes, true);
  if (st == PEPO_OK) c->inst[inst].saved_steps = c->inst[inst].steps;
  return st;
}

pepo_status pepo_load_state(pepo_ctx* c, int inst, const void* dev_buf, size_t bytes) {
  pepo_status st = state_copy(c, inst, const_cast<char*>(static_cast<const char*>(dev_buf)), bytes, false);
  if (st == PEPO_OK) {
    c->inst[inst].steps = c->inst[inst].saved_steps;
    c->inst[inst].meas_valid = c->inst[inst].prev_valid = 0;
  }
  return st;
}

pepo_status pepo_save_state_host(pepo_ctx* c, int inst, void* host_buf, size_t bytes, int* steps_out) {
  pepo_status st = state_copy(c, inst, static_cast<char*>(host_buf), bytes, true, true);
  if (st == PEPO_OK && steps_out) *steps_out = c->inst[inst].steps;
  return st;
}

pepo_status pepo_load_state_host(pepo_ctx* c, int inst, const void* host_buf, size_t bytes, int steps) {
  if (c && steps < 0) return fail(c, PEPO_E_INVALID, "steps must be >= 0");
  pepo_status st = state_copy(c, inst, const_cast<char*>(static_cast<const char*>(host_buf)), bytes, false, true);
  if (st == PEPO_OK) {
    c->inst[inst].steps = steps;
    c->inst[inst].meas_valid = c->inst[inst].prev_valid = 0;
  }
  return st;
}

// ------------------------------------------------------- learned warm start
struct pepo_mlp {
  MlpBuffers B;
  cudaStream_t stream = nullptr;
  int max_rows = 0;
  int adam_t = 0;
  float last_loss = 0.f;
};

size_t pepo_mlp_required_bytes(int max_rows) {
  if (max_rows < 1) return 0;
  MlpBuffers B;
  return mlp_layout(nullptr, max_rows, &B) + 256;
}

long long pepo_mlp_num_params(void) { return mlp_num_params(); }

pepo_status pepo_mlp_init(void* dev_buf, size_t bytes, int max_rows, const float* params, void* cuda_stream,
                          pepo_mlp** out) {
  if (!out) return PEPO_E_INVALID;
  *out = nullptr;
  if (!dev_buf || !params || max_rows < 1 || (reinterpret_cast<uintptr_t>(dev_buf) & 255)) return PEPO_E_INVALID;
  if (bytes < pepo_mlp_required_bytes(max_rows)) return PEPO_E_OOM;
  pepo_mlp* m = new pepo_mlp;
  mlp_layout(static_cast<char*>(dev_buf), max_rows, &m->B);
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  m->max_rows = max_rows;
  const size_t n = (size_t)mlp_num_params();
  bool ok = cudaMemcpyAsync(m->B.p, params, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(m->B.m, 0, sizeof(float) * n, m->stream) == cudaSuccess;
  ok = ok && cudaMemsetAsync(m->B.v, 0, sizeof(float) * n, m->stream) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(m->stream) == cudaSuccess;
  if (!ok) { delete m; return PEPO_E_CUDA; }
  *out = m;
  return PEPO_OK;
}

pepo_status pepo_set_warmstart_weights(pepo_ctx* c, const void* dev_weights, size_t bytes) {
  if (!c) return PEPO_E_INVALID;
  const size_t want = sizeof(float) * (size_t)mlp_num_params();
  if (!dev_weights || bytes != want)
    return fail(c, PEPO_E_INVALID, "warm-start weights: %zu bytes given, %zu expected", bytes, want);
  if (c->ws_rows_max == 0)
    return fail(c, PEPO_E_STATE, "warm-start weights: no instance was created with warm_start = 1");
  if (cudaMemcpyAsync(c->ws_mlp.p, dev_weights, want, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "warm-start weights: copy failed");
  c->ws_ready = true;
  return PEPO_OK;
}

pepo_status pepo_mlp_get_params(pepo_mlp* m, float* params) {
  if (!m || !params) return PEPO_E_INVALID;
  if (cudaMemcpyAsync(params, m->B.p, sizeof(float) * (size_t)mlp_num_params(), cudaMemcpyDeviceToHost,
                      m->stream) != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
    return PEPO_E_CUDA;
  return PEPO_OK;
}

pepo_status pepo_mlp_forward(pepo_mlp* m, const float* X_dev, int rows, float* y_dev) {
  if (!m || !X_dev || !y_dev || rows < 0 || rows > m->max_rows) return PEPO_E_INVALID;
  if (rows == 0) return PEPO_OK;
  return mlp_forward(m->B, X_dev, rows, y_dev, m->stream) == cudaSuccess ? PEPO_OK : PEPO_E_CUDA;
}

pepo_status pepo_mlp_gradient(pepo_mlp* m, const float* X_dev, const float* t_dev, int rows, float* loss_out,
                              float* grad_host) {
  if (!m || !X_dev || !t_dev || rows < 1 || rows > m->max_rows) return PEPO_E_INVALID;
  if (mlp_gradient(m->B, X_dev, t_dev, rows, m->stream) != cudaSuccess) return PEPO_E_CUDA;
  if (cudaMemcpyAsync(&m->last_loss, m->B.loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PEPO_E_CUDA;
  if (grad_host && cudaMemcpyAsync(grad_host, m->B.g, sizeof(float) * (size_t)mlp_num_params(),
                                   cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
    return PEPO_E_CUDA;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return PEPO_E_CUDA;
  if (loss_out) *loss_out = m->last_loss;
  return PEPO_OK;
}

pepo_status pepo_mlp_adam_step(pepo_mlp* m, float lr) {
  if (!m || !(lr > 0.f)) return PEPO_E_INVALID;
  m->adam_t++;
  return mlp_adam(m->B, m->adam_t, lr, m->stream) == cudaSuccess ? PEPO_OK : PEPO_E_CUDA;
}

void pepo_mlp_destroy(pepo_mlp* m) { delete m; }

int pepo_ws_rows(pepo_ctx* c, int inst) {
  if (!c || inst < 0 || inst >= c->n_inst) return -1;
  Inst& I = c->inst[inst];
  std::vector<int> chi(I.nb);
  if (cudaMemcpyAsync(chi.data(), c->d_ival + I.chi0, sizeof(int) * I.nb, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return -1;
  long long r = 0;
  for (int x : chi) r += 2LL * x;
  return (int)r;
}

pepo_status pepo_ws_features(pepo_ctx* c, int inst, float* X_dev, int max_rows) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_ws_features")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst || !X_dev || max_rows < 0) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  const float t = (float)(I.steps * I.cfg.dt);
  cudaError_t e = launch_ws_features(I.ws_geom, I.nb, c->d_ival + I.chi0, I.lam, I.cfg.chi_max, t,
                                     (float)I.cfg.h, (float)I.cfg.J, X_dev, max_rows, c->stream);
  c->launches++;
  return e == cudaSuccess ? PEPO_OK : fail(c, PEPO_E_CUDA, "warm-start features: %s", cudaGetErrorString(e));
}

pepo_status pepo_ws_targets(pepo_ctx* c, int inst, float* t_dev, int max_rows) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_ws_targets")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst || !t_dev || max_rows < 0) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  cudaError_t e = launch_ws_targets(I.nb, c->d_ival + I.chi0, I.msg, I.cfg.chi_max, t_dev, max_rows, c->stream);
  c->launches++;
  return e == cudaSuccess ? PEPO_OK : fail(c, PEPO_E_CUDA, "warm-start targets: %s", cudaGetErrorString(e));
}

pepo_status pepo_ws_apply(pepo_ctx* c, int inst, const float* y_dev, float gamma) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_ws_apply")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst || !y_dev || !(gamma >= 0.f && gamma <= 1.f))
    return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  cudaError_t e = launch_ws_apply(I.nb, c->d_ival + I.chi0, y_dev, I.msg, I.cfg.chi_max, gamma, c->stream);
  c->launches++;
  return e == cudaSuccess ? PEPO_OK : fail(c, PEPO_E_CUDA, "warm-start apply: %s", cudaGetErrorString(e));
}

pepo_status pepo_set_state(pepo_ctx* c, int inst, const double* sites, size_t count, const int* chi,
                           const double* lam, const double* msgs) {
  if (!c) return PEPO_E_INVALID;
  if (!at_step_boundary(c, "pepo_set_state")) return PEPO_E_STATE;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (!sites) return fail(c, PEPO_E_INVALID, "null argument");
  pepo_status st = pepo_set_bonds(c, inst, chi, lam, msgs);
  if (st != PEPO_OK) return st;
  size_t off = 0;
  for (int v = 0; v < I.N; ++v) {
    const SiteG& S = I.sites[v];
    size_t n = 4;
    for (int k = 0; k < S.deg; ++k) n *= chi[S.legs[k].bond];
    if (off + n > count) return fail(c, PEPO_E_INVALID, "site data too short");
    st = pepo_set_site(c, inst, v, sites + off, 1, n);
    if (st != PEPO_OK) return st;
    off += n;
  }
  return PEPO_OK;
}

pepo_status pepo_pauli_weights(pepo_ctx* c, int inst, double* out) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst || !out) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  std::vector<double> w((size_t)4 * I.N);
  if (cudaMemcpyAsync(w.data(), I.pw, sizeof(double) * w.size(), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "Pauli weights: %s", cudaGetErrorString(cudaGetLastError()));
  for (int v = 0; v < I.N; ++v) {
    double t = 0.0;
    for (int p = 0; p < 4; ++p) t += w[4 * (size_t)v + p];
    for (int p = 0; p < 4; ++p) out[4 * (size_t)v + p] = t > 0.0 ? w[4 * (size_t)v + p] / t : 0.0;
  }
  return PEPO_OK;
}

pepo_status pepo_get_messages(pepo_ctx* c, int inst, double* out) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst || !out) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  const size_t n = (size_t)2 * I.nb * I.cfg.chi_max * I.cfg.chi_max;
  if (cudaMemcpyAsync(out, I.msg, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "message readback");
  return PEPO_OK;
}

pepo_status pepo_set_messages(pepo_ctx* c, int inst, const double* msgs) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst || !msgs) return fail(c, PEPO_E_INVALID, "bad arguments");
  Inst& I = c->inst[inst];
  const size_t n = (size_t)2 * I.nb * I.cfg.chi_max * I.cfg.chi_max;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(I.msg, msgs, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "message upload");
  return PEPO_OK;
}

pepo_status pepo_set_bp_params(pepo_ctx* c, int inst, double alpha, double tol, int max_sweeps) {
  if (!c) return PEPO_E_INVALID;
  if (inst < -1 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(c, PEPO_E_INVALID, "bp_alpha must be in (0, 1]");
  if (!(tol > 0.0)) return fail(c, PEPO_E_INVALID, "bp_tol must be > 0");
  if (max_sweeps < 1) return fail(c, PEPO_E_INVALID, "bp_max_sweeps must be >= 1");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "pepo_set_bp_params: %s", cudaGetErrorString(e));
  // the damping is staged in the message items (per instance, and in the
  // grouped array of a multi-instance context): patch the host copy of the
  // items and upload the patched range; captured graphs read the items from
  // device memory, so they see the new value
  auto patch = [&](const DArr<MsgItem>& a, size_t first, size_t n) -> bool {
    if (n == 0) return true;
    MsgItem* h = reinterpret_cast<MsgItem*>(c->host_items.data() + a.off) + first;
    for (size_t k = 0; k < n; ++k) h[k].alpha = alpha;
    return cudaMemcpy(const_cast<MsgItem*>(a.d) + first, h, sizeof(MsgItem) * n, cudaMemcpyHostToDevice) ==
           cudaSuccess;
  };
  size_t gpos = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    Inst& I = c->inst[i];
    const size_t n = (size_t)I.msgs.n;
    if (inst < 0 || inst == i) {
      I.cfg.bp_alpha = alpha;
      I.cfg.bp_tol = tol;
      I.cfg.bp_max_sweeps = max_sweeps;
      bool ok = patch(I.msgs, 0, n);
      if (ok && c->n_inst > 1) ok = patch(c->grp.msgs, gpos, n);
      if (!ok) return fail(c, PEPO_E_CUDA, "message item upload");
    }
    gpos += n;
  }
  return PEPO_OK;
}

pepo_status pepo_get_message(pepo_ctx* c, int inst, int bond, int dir, double* out, int* chi_out) {
  if (!c) return PEPO_E_INVALID;
  if (inst < 0 || inst >= c->n_inst) return fail(c, PEPO_E_INVALID, "bad instance");
  Inst& I = c->inst[inst];
  if (bond < 0 || bond >= I.nb || (dir != 0 && dir != 1) || !out || !chi_out)
    return fail(c, PEPO_E_INVALID, "bad message");
  const int chimax = I.cfg.chi_max;
  std::vector<double> m((size_t)chimax * chimax);
  int chi = 0;
  if (cudaMemcpyAsync(m.data(), I.msg + (size_t)(2 * bond + dir) * chimax * chimax,
                      sizeof(double) * m.size(), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(&chi, c->d_ival + I.chi0 + bond, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "message readback");
  for (int i = 0; i < chi; ++i)
    for (int j = 0; j < chi; ++j) out[i * chi + j] = m[(size_t)i * chimax + j];
  *chi_out = chi;
  return PEPO_OK;
}

int pepo_num_bonds(const pepo_ctx* c, int inst) {
  if (!c || inst < 0 || inst >= c->n_inst) return 0;
  return c->inst[inst].nb;
}

long long pepo_launch_count(const pepo_ctx* c) { return c ? c->launches : 0; }

pepo_status pepo_qr_branch_counts(pepo_ctx* c, long long* out, int reset) {
  if (!c) return PEPO_E_INVALID;
  if (!out) return fail(c, PEPO_E_INVALID, "pepo_qr_branch_counts: null output");
  unsigned long long h[3] = {0, 0, 0};
  if (cudaMemcpyAsync(h, c->d_qr_count, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      (reset && cudaMemsetAsync(c->d_qr_count, 0, sizeof(h), c->stream) != cudaSuccess) ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "pepo_qr_branch_counts: %s", cudaGetErrorString(cudaGetLastError()));
  for (int i = 0; i < 3; ++i) out[i] = (long long)h[i];
  return PEPO_OK;
}

const char* pepo_last_error(const pepo_ctx* c) { return c ? c->err.c_str() : kStaticErr; }

void pepo_destroy(pepo_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  delete c;
}

pepo_status pepo_set_tuning(pepo_ctx* c, const pepo_tuning* t) {
  if (!c || !t) return PEPO_E_INVALID;
  const int gl = t->gram_leg_splits ? t->gram_leg_splits : kLegSplits;
  const int gr = t->gram_rows_splits ? t->gram_rows_splits : kGramSplits;
  if (gl < 1 || gl > kLegSplitsMax) return fail(c, PEPO_E_INVALID, "gram_leg_splits out of 1..128");
  if (gr < 1 || gr > kGramSplitsMax) return fail(c, PEPO_E_INVALID, "gram_rows_splits out of 1..64");
  if (gl == c->tune.gram_leg_splits && gr == c->tune.gram_rows_splits) return PEPO_OK;
  // captured graphs hold the old launch shapes: finish the stream's work and
  // drop them (they are captured again at their next use)
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "pepo_set_tuning: %s", cudaGetErrorString(e));
  for (cudaGraphExec_t* x : {&c->step_exec, &c->bp_exec, &c->sl_exec}) {
    if (*x) cudaGraphExecDestroy(*x);
    *x = nullptr;
  }
  c->tune.gram_leg_splits = gl;
  c->tune.gram_rows_splits = gr;
  return PEPO_OK;
}

pepo_status pepo_set_wait_limit(pepo_ctx* c, double seconds) {
  if (!c) return PEPO_E_INVALID;
  if (!(seconds >= 1e-9 && seconds <= 60.0))
    return fail(c, PEPO_E_INVALID, "wait limit must lie in [1e-9, 60] s, got %g", seconds);
  const unsigned long long ns = (unsigned long long)std::llround(seconds * 1e9);
  if (ns == c->wait_ns) return PEPO_OK;
  // captured graphs hold the old limit in their kernel parameters
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, PEPO_E_CUDA, "pepo_set_wait_limit: %s", cudaGetErrorString(e));
  for (cudaGraphExec_t* x : {&c->step_exec, &c->bp_exec, &c->sl_exec}) {
    if (*x) cudaGraphExecDestroy(*x);
    *x = nullptr;
  }
  c->wait_ns = ns;
  return PEPO_OK;
}

pepo_status pepo_get_tuning(const pepo_ctx* c, pepo_tuning* t) {
  if (!c || !t) return PEPO_E_INVALID;
  *t = c->tune;
  return PEPO_OK;
}

pepo_status pepo_set_timing(pepo_ctx* c, int enable) {
  if (!c) return PEPO_E_INVALID;
  timing_harvest(c);
  c->timing = enable != 0;
  return PEPO_OK;
}

int pepo_timing_classes(void) { return K_NCLASS; }

const char* pepo_timing_class_name(int k) { return (k >= 0 && k < K_NCLASS) ? kClassNames[k] : ""; }

pepo_status pepo_get_timing(pepo_ctx* c, int k, long long* launches, double* ms, double* bytes,
                            double* flops) {
  if (!c) return PEPO_E_INVALID;
  if (k < 0 || k >= K_NCLASS) return fail(c, PEPO_E_INVALID, "bad kernel class");
  timing_harvest(c);
  const auto& t = c->tot[k];
  double dev[2] = {0.0, 0.0};
  if (k == K_HH) {
    // which sites take the Householder branch is decided on the device, so
    // this class's work is counted there (k_hh_extract)
    if (cudaMemcpyAsync(dev, c->d_hh_acct, sizeof(dev), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(c, PEPO_E_CUDA, "pepo_get_timing: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (launches) *launches = t.n;
  if (ms) *ms = t.ms;
  if (bytes) *bytes = t.bytes + dev[1];
  if (flops) *flops = t.flops + dev[0];
  return PEPO_OK;
}

pepo_status pepo_reset_timing(pepo_ctx* c) {
  if (!c) return PEPO_E_INVALID;
  timing_harvest(c);
  c->tot.assign(K_NCLASS, pepo_ctx::Tot());
  if (cudaMemsetAsync(c->d_hh_acct, 0, 2 * sizeof(double), c->stream) != cudaSuccess)
    return fail(c, PEPO_E_CUDA, "pepo_reset_timing: %s", cudaGetErrorString(cudaGetLastError()));
  return PEPO_OK;
}

}  // extern "C"
