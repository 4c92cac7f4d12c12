// Fifth-generation tensor-core (tcgen05) contractions for the FP32-storage
// mixed-precision mode: the leg contraction and the free-leg Gram of the BP
// message products (Eq. 13) and of the absorb step (Sec. 2.5 step 1).
//
//   k_leg_umma   out[o, i, q] = sum_j A[i, j] in[o, j, q]
//   k_gram_umma  S[i, i'] = sum_k (Xh[i,k] Xh[i',k] + 2 Xh[i,k] Xl[i',k])
//                over one K-range (split) of k = (o, q); the reduction sums the
//                splits and symmetrises: G = (S + S^T) / 2 = sum w^2 X X^T up
//                to the dropped lo*lo term.
//
// Split precision (three-product TF32): every FP32 operand x is split as
// x = hi + lo with hi = tf32(x) (round to nearest) and lo = x - hi (exact in
// FP32; the tensor core keeps its leading 11 bits).  A product a*b is taken as
// ah*bh + ah*bl + al*bh; the dropped al*bl and the truncation of lo are
// ~2^-21 relative.  For the leg contraction the hi and lo rows of the small
// matrix A are stacked along N, so one MMA of width 2N gives [ah*bh | ah*bl]
// and a second of width N adds al*bh to the first half.  For the Gram both
// operands are the same tile X, stacked as [Xh; Xl] along N: one MMA gives
// [Xh Xh^T | Xh Xl^T] and the symmetrisation supplies Xl Xh^T.
//
// Pipeline (one persistent CTA per SM, 512 threads):
//   warp 0        allocates tensor memory; lane 0 issues every MMA and the
//                 commits that release shared-memory stages and hand finished
//                 accumulators to the epilogue
//   warps 4-7     epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//                 lanes 32 (w % 4) .. +31), store to global memory (leg) or
//                 add into compensated FP32 sums in shared memory (Gram)
//   warps 8-15    converters: coalesced global loads (leg, reconstruct:
//                 a register ring two or one chunks ahead; Gram: per-thread
//                 cp.async into a ring of raw shared-memory stages four chunks
//                 ahead), split, and 16-byte conflict-free stores into
//                 the swizzled K-major layout the MMA descriptors describe
//                 (below); the reconstruct's W block arrives by bulk copy
// Stages and accumulators are handed over with mbarriers.  Every wait is
// bounded (a few seconds of %globaltimer); on expiry the kernel records bit 0
// in *err (bit 1 marks a reconstruct item without its packed-W workspace),
// every role leaves its loop, the MMA issuer drains its outstanding
// MMAs (bounded), tensor memory is freed and the kernel returns.
//
// Shared-memory operand layout: K-major with the 128-byte swizzle.  A row of
// an operand holds the 32 FP32 (TF32) values of one K chunk in 128 bytes;
// 8 rows form a 1024-byte atom (atoms SBO = 1024 bytes apart along M/N); the
// 16-byte piece c of row r sits at piece position c ^ (r % 8).  One MMA
// covers K = 8 (32 bytes): its descriptor starts 32 bytes further per K step
// inside the atom (the hardware applies the XOR to the absolute address, so
// every tile is 1024-byte aligned).  Element (n, k) of a tile sits at
// (n / 8) 1024 + (n % 8) 128 + (((k / 4) ^ (n % 8)) 16) + (k % 4) 4.
#include "kernels.h"

namespace pepo {
namespace um {

constexpr int kThreads = 512;
constexpr int kConv = 256;              // converter threads (warps 8..15)
constexpr int kM = 128;                 // accumulator rows = TMEM lanes
constexpr int kKC = 32;                 // K values per staged chunk
constexpr int kTmemCols = 512;          // two accumulators of 256 columns
// Gram chunks per FP32 accumulator run (1024 K terms summed in TMEM before
// the compensated shared-memory sums take them): the FP32 rounding of a run
// is ~1e-6 of its sum in the worst case, below the split-TF32 product error,
// and the epilogue's pass over the accumulator is paid once per run
constexpr int kRun = 32;
constexpr unsigned long long kDrainNs = 2000000000ull;   // bound of the exit drains
constexpr int kMaxItems = 512;

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of parity `parity`; false once the CTA aborts.
// `limit` (ns of %globaltimer) is the launch's wait limit; on expiry the wait
// records bit 0 in *err and raises the CTA's abort flag.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                          unsigned long long limit) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit) {
      *abort_flag = 1;
      atomicOr(err, 1);
      return false;
    }
  }
}

// Wait on the way out, also after an abort: the CTA's own MMAs and bulk
// copies in flight complete before its tensor and shared memory are released.
// Bounded by kDrainNs (they finish within microseconds); bit 2 in *err if not.
__device__ void mbar_drain(uint64_t* b, uint32_t parity, int* err) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try(b, parity)) {
    if (gtimer() - t0 > kDrainNs) {
      atomicOr(err, 4);
      return;
    }
  }
}

// warp-uniform wait (every lane agrees, so the warp leaves a loop together)
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                                          unsigned long long limit) {
  const bool ok = mbar_wait(b, parity, abort_flag, err, limit);
  return __all_sync(0xffffffffu, ok);
}
// one arrival per warp once every lane's shared-memory writes are ordered
// before it (the lanes' proxy fences precede the warp barrier)
__device__ __forceinline__ void warp_arrive(uint64_t* b) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(b);
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned, size a multiple of 16) that
// completes `bytes` of the barrier's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
// without reading the source
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n of this thread's copy groups are pending (n <= 7)
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
  }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, atoms 1024
// bytes apart (the leading offset is unused for this layout: one atom spans
// the MMA's K)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused), 16 bytes
  d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: 8-row atoms
  d |= (uint64_t)1 << 46;                   // descriptor version of the sm_100 family
  d |= (uint64_t)2 << 61;                   // layout: 128-byte swizzle
  return d;
}
// byte offset of the 16-byte piece `piece` (K / 4) of row `row` in a tile
__host__ __device__ __forceinline__ uint32_t swz(int row, int piece) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((piece ^ (row & 7)) << 4));
}
// instruction descriptor: kind::tf32, FP32 accumulator, A and B TF32 K-major
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}
// 32 TMEM lanes x 16 consecutive 32-bit columns; thread t receives lane
// (lane base + t).  The registers are valid after tmem_wait16.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// completes outstanding tcgen05.ld of two 16-column blocks at once; both
// register sets are threaded through so no use is scheduled before the wait
__device__ __forceinline__ void tmem_wait32(uint32_t* r, uint32_t* q) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]),
                 "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]), "+r"(q[13]), "+r"(q[14]),
                 "+r"(q[15])
               :
               : "memory");
}
// completes outstanding tcgen05.ld; the registers are threaded through so no
// use of them is scheduled before the wait
__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ============================================================ leg contraction
struct LegDims {
  long long O, Q, R, tiles;
  int J, Jout, K8, N16;
  const float* in;
  float* out;
  const double* A;
  int lda;
};

__device__ inline void leg_dims(const LegItem& it, void* const* ptrs, const int* ival, LegDims& L) {
  int d[PEPO_MAXLEG];
  for (int k = 0; k < PEPO_MAXLEG; ++k) d[k] = (k < it.in.nlegs) ? ival[it.in.dim[k]] : 1;
  const int k = it.leg;
  L.J = d[k];
  L.Jout = ival[it.out_dim];
  L.O = 1;
  L.Q = 4;
  for (int i = 0; i < k; ++i) L.O *= d[i];
  for (int i = k + 1; i < it.in.nlegs; ++i) L.Q *= d[i];
  L.R = L.O * L.Q;
  L.tiles = (L.R + kM - 1) / kM;
  L.K8 = round_up(L.J, 8);
  L.N16 = round_up(L.Jout, 16);
  L.in = static_cast<const float*>(ptrs[it.in.ref]);
  L.out = static_cast<float*>(ptrs[it.out_ref]);
  L.A = it.A;
  L.lda = it.lda;
}

// Shared-memory plan of k_leg_umma for a given chi bound.
struct LegSmem {
  int k8max, n16max, stages;
  size_t b_bytes, stage_bytes, bar_off, total;
};
__host__ __device__ inline LegSmem leg_smem(int chimax) {
  LegSmem p;
  p.k8max = round_up(chimax, 8);
  p.n16max = round_up(chimax, 16);
  // [Ah; Al] of the small matrix: one (2 N16 rows x 128 B) block per K chunk
  p.b_bytes = (size_t)((p.k8max + kKC - 1) / kKC) * (2 * p.n16max) * 128;
  p.stage_bytes = 2 * (size_t)kM * 128;                             // hi + lo tile, 2 x 16 KB
  const size_t budget = 227 * 1024 - 1024 - 8 * kMaxItems - 512;
  p.stages = (int)((budget - p.b_bytes) / p.stage_bytes);
  if (p.stages > 4) p.stages = 4;
  p.bar_off = p.b_bytes + p.stages * p.stage_bytes;
  p.total = p.bar_off + 512 + 8 * (size_t)(kMaxItems + 1) + 1024;   // + alignment slack
  return p;
}

struct LegCursor {   // position in the CTA's tile range
  int item;
  long long tile;    // tile within the item
  long long left;    // tiles left for this CTA
  LegDims L;
};

__device__ inline bool cursor_start(LegCursor& c, const long long* toff, int n, long long t0, long long t1,
                                    const LegItem* items, void* const* ptrs, const int* ival) {
  c.left = t1 - t0;
  if (c.left <= 0) return false;
  int i = 0;
  while (i + 1 < n && toff[i + 1] <= t0) ++i;
  c.item = i;
  c.tile = t0 - toff[i];
  leg_dims(items[i], ptrs, ival, c.L);
  return true;
}
// advance to the next tile; returns true when the item changed
__device__ inline bool cursor_next(LegCursor& c, const long long* toff, int n, const LegItem* items,
                                   void* const* ptrs, const int* ival) {
  --c.left;
  ++c.tile;
  bool changed = false;
  while (c.left > 0 && c.tile >= c.L.tiles && c.item + 1 < n) {
    ++c.item;
    c.tile = 0;
    leg_dims(items[c.item], ptrs, ival, c.L);
    changed = true;
  }
  return changed;
}

struct LegBars {
  uint64_t full[4], empty[4], accfull[2], accempty[2], bfull, bfree, drain;
  uint32_t tmem;
  int abort_flag;
};

__global__ void __launch_bounds__(kThreads, 1)
k_leg_umma(const LegItem* __restrict__ items, int n_items, int chimax, void* const* ptrs,
           const int* __restrict__ ival, int* err, unsigned long long lim) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const LegSmem P = leg_smem(chimax);
  unsigned char* Bs = smem;                          // [Ah; Al] small matrix
  unsigned char* As = smem + P.b_bytes;              // stages: hi tile, lo tile
  LegBars* bars = reinterpret_cast<LegBars*>(smem + P.bar_off);
  long long* toff = reinterpret_cast<long long*>(smem + P.bar_off + 512);
  volatile int* abort_flag = &bars->abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NS = P.stages;

  if (tid == 0) {
    long long acc = 0;
    for (int i = 0; i < n_items; ++i) {
      toff[i] = acc;
      LegDims L;
      leg_dims(items[i], ptrs, ival, L);
      acc += L.tiles;
    }
    toff[n_items] = acc;
    for (int s = 0; s < NS; ++s) { mbar_init(&bars->full[s], kConv / 32); mbar_init(&bars->empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&bars->accfull[b], 1); mbar_init(&bars->accempty[b], 4); }
    mbar_init(&bars->bfull, kConv / 32);
    mbar_init(&bars->bfree, 1);
    mbar_init(&bars->drain, 1);
    bars->abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&bars->tmem);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = bars->tmem;
  const long long T = toff[n_items];
  const long long t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      LegCursor c;
      bool live = cursor_start(c, toff, n_items, t0, t1, items, ptrs, ival);
      long long tc = 0;
      int st_i = 0;            // operand stage and its phase parity (advanced per chunk)
      uint32_t st_ph = 0;
      int item_n = 0;
      bool ok = true;
      if (live) ok = mbar_wait(&bars->bfull, 0, abort_flag, err, lim);
      while (live && ok) {
        const int b = (int)(tc & 1);
        if (!mbar_wait(&bars->accempty[b], (uint32_t)(((tc >> 1) & 1) ^ 1), abort_flag, err, lim)) break;
        tc_after();
        const uint32_t d_tmem = tmem + (uint32_t)(b * 256);
        const int N16 = c.L.N16, K8 = c.L.K8;
        const uint32_t bblk = (uint32_t)(2 * N16) * 128;   // B block per K chunk
        const uint32_t id_wide = idesc_tf32(kM, 2 * N16), id_half = idesc_tf32(kM, N16);
        const int nkc = (K8 + kKC - 1) / kKC;
        for (int kc = 0; kc < nkc && ok; ++kc) {
          const int s = st_i;
          if (!mbar_wait(&bars->full[s], st_ph, abort_flag, err, lim)) { ok = false; break; }
          if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
          tc_after();
          const uint32_t a_hi = su32(As + (size_t)s * P.stage_bytes);
          const uint32_t a_lo = a_hi + (uint32_t)(P.stage_bytes / 2);
          const uint32_t b0 = su32(Bs);
          const int ksteps = min(kKC, K8 - kc * kKC) / 8;
          for (int st = 0; st < ksteps; ++st) {
            const uint64_t dah = sdesc(a_hi + (uint32_t)st * 32u);
            const uint64_t dal = sdesc(a_lo + (uint32_t)st * 32u);
            const uint64_t db = sdesc(b0 + (uint32_t)kc * bblk + (uint32_t)st * 32u);
            mma_tf32(d_tmem, dah, db, id_wide, (kc > 0 || st > 0) ? 1u : 0u);
            mma_tf32(d_tmem, dal, db, id_half, 1u);
          }
          mma_commit(&bars->empty[s]);
        }
        if (!ok) break;
        mma_commit(&bars->accfull[b]);
        ++tc;
        const bool last = (c.left == 1);
        const bool changed = cursor_next(c, toff, n_items, items, ptrs, ival);
        if (changed || last) mma_commit(&bars->bfree);
        if (last) break;
        if (changed) {
          ++item_n;
          if (!mbar_wait(&bars->bfull, (uint32_t)(item_n & 1), abort_flag, err, lim)) break;
          tc_after();
        }
      }
      // every issued MMA completes before tensor memory is released
      mma_commit(&bars->drain);
      mbar_drain(&bars->drain, 0, err);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // -------------------------------------------------------------- epilogue
    LegCursor c;
    bool live = cursor_start(c, toff, n_items, t0, t1, items, ptrs, ival);
    const int row = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    long long tc = 0;
    while (live) {
      const int b = (int)(tc & 1);
      if (!warp_wait(&bars->accfull[b], (uint32_t)((tc >> 1) & 1), abort_flag, err, lim)) break;
      tc_after();
      const LegDims& L = c.L;
      const long long rg = c.tile * kM + row;
      const bool valid = rg < L.R;
      long long o = 0, q = 0;
      if (valid) { o = rg / L.Q; q = rg - o * L.Q; }
      float* dst = L.out + (o * L.Jout) * L.Q + q;
      const uint32_t tbase = tmem + lane_base + (uint32_t)(b * 256);
      // 16-column blocks; the TMEM loads of block i+1 are in flight while
      // block i is stored (two register sets, unrolled so none is copied)
      uint32_t a1[16], a2[16], b1[16], b2[16];
      auto store_blk = [&](const uint32_t* p1, const uint32_t* p2, int c0) {
        if (!valid) return;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = c0 + i;
          if (col < L.Jout) dst[(long long)col * L.Q] = __uint_as_float(p1[i]) + __uint_as_float(p2[i]);
        }
      };
      tmem_ld16(tbase, a1);
      tmem_ld16(tbase + (uint32_t)L.N16, a2);
      tmem_wait32(a1, a2);
      for (int c0 = 0; c0 < L.N16; c0 += 32) {
        const bool m1 = c0 + 16 < L.N16;
        if (m1) {
          tmem_ld16(tbase + (uint32_t)(c0 + 16), b1);
          tmem_ld16(tbase + (uint32_t)(L.N16 + c0 + 16), b2);
        }
        store_blk(a1, a2, c0);
        if (!m1) break;
        tmem_wait32(b1, b2);
        const bool m2 = c0 + 32 < L.N16;
        if (m2) {
          tmem_ld16(tbase + (uint32_t)(c0 + 32), a1);
          tmem_ld16(tbase + (uint32_t)(L.N16 + c0 + 32), a2);
        }
        store_blk(b1, b2, c0 + 16);
        if (!m2) break;
        tmem_wait32(a1, a2);
      }
      tc_before();
      warp_arrive(&bars->accempty[b]);
      ++tc;
      if (c.left == 1) break;
      cursor_next(c, toff, n_items, items, ptrs, ival);
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ converters
    // Each thread owns one row r of the tile and, per chunk, four 4-wide K
    // groups (jq = jq0 + 2 u): four coalesced 4-byte loads per group (the
    // lanes of a warp read 32 consecutive rows), then one 16-byte store per
    // group into the K-major layout (8 consecutive rows per quarter warp: no
    // bank conflicts).  Loads run two chunks ahead of the stores (register
    // ring v0, v1, v2).
    const int ct = tid - 256, cw = ct >> 5;
    const int r = 32 * (cw & 3) + lane;             // this thread's row
    const int jq0 = cw >> 2;                        // K groups jq0, jq0 + 2, +4, +6
    // load cursor
    LegCursor lc;
    bool lc_live = cursor_start(lc, toff, n_items, t0, t1, items, ptrs, ival);
    int lkc = 0;
    bool lvalid = false;
    const float* lsrc = nullptr;
    auto enter_tile = [&]() {
      const long long rg = lc.tile * kM + r;
      lvalid = rg < lc.L.R;
      lsrc = lc.L.in;
      if (lvalid) {
        const long long o = rg / lc.L.Q, q = rg - o * lc.L.Q;
        lsrc = lc.L.in + o * lc.L.J * lc.L.Q + q;
      }
      lkc = 0;
    };
    if (lc_live) enter_tile();
    auto load_next = [&](float4* v) {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!lc_live) return;
      if (lvalid) {
        const int J = lc.L.J;
        const long long Q = lc.L.Q;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = lkc * kKC + 4 * (jq0 + 2 * u);
          const float* p0 = lsrc + (long long)j * Q;
          if (j < J) v[u].x = __ldg(p0);
          if (j + 1 < J) v[u].y = __ldg(p0 + Q);
          if (j + 2 < J) v[u].z = __ldg(p0 + 2 * Q);
          if (j + 3 < J) v[u].w = __ldg(p0 + 3 * Q);
        }
      }
      if (++lkc < (lc.L.K8 + kKC - 1) / kKC) return;
      if (lc.left == 1) { lc_live = false; return; }
      cursor_next(lc, toff, n_items, items, ptrs, ival);
      enter_tile();
    };
    float4 v0[4], v1[4], v2[4];
    load_next(v0);
    load_next(v1);
    // store cursor
    LegCursor c;
    bool live = cursor_start(c, toff, n_items, t0, t1, items, ptrs, ival);
    int st_i = 0;              // operand stage and its phase parity
    uint32_t st_ph = 0;
    int item_n = 0, kc = 0;
    bool need_b = true;
    // one chunk: issue the loads two chunks ahead into vl, convert and store
    // vs (the ring is rotated by unrolling, never by copying registers, so
    // no load is waited on before its turn); returns false at the end
    auto step = [&](float4 (&vl)[4], float4 (&vs)[4]) -> bool {
      const LegDims& L = c.L;
      load_next(vl);
      if (need_b) {
        if (item_n > 0 && !warp_wait(&bars->bfree, (uint32_t)((item_n - 1) & 1), abort_flag, err, lim)) return false;
        // [Ah; Al]: rows n < N16 hold hi(A[n, :]), rows N16 + n hold lo(A[n, :]);
        // one block of 2 N16 rows per 32-wide K chunk
        const size_t bblk = (size_t)(2 * L.N16) * 128;
        const int K32 = (L.K8 + kKC - 1) / kKC * kKC;
        for (int e = ct; e < L.N16 * K32; e += kConv) {
          const int n = e / K32, j = e - n * K32;
          float x = 0.f;
          if (n < L.Jout && j < L.J) x = (float)L.A[(long long)n * L.lda + j];
          const float h = tf32_hi(x);
          const float l = x - h;
          unsigned char* blk = Bs + (size_t)(j / kKC) * bblk + (size_t)(j & 3) * 4;
          const int piece = (j % kKC) >> 2;
          *reinterpret_cast<float*>(blk + swz(n, piece)) = h;
          *reinterpret_cast<float*>(blk + swz(n + L.N16, piece)) = l;
        }
        fence_async_smem();
        warp_arrive(&bars->bfull);
        need_b = false;
      }
      const int s = st_i;
      if (!warp_wait(&bars->empty[s], st_ph ^ 1u, abort_flag, err, lim)) return false;
      if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
      unsigned char* hi = As + (size_t)s * P.stage_bytes;
      unsigned char* lo = hi + P.stage_bytes / 2;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t off = swz(r, jq0 + 2 * u);
        const float4 x = vs[u];
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
      fence_async_smem();
      warp_arrive(&bars->full[s]);
      if (++kc < (L.K8 + kKC - 1) / kKC) return true;
      kc = 0;
      if (c.left == 1) return false;
      if (cursor_next(c, toff, n_items, items, ptrs, ival)) { ++item_n; need_b = true; }
      return true;
    };
    while (live) {
      if (!step(v2, v0)) break;
      if (!step(v0, v1)) break;
      if (!step(v1, v2)) break;
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_free(tmem);
  }
}

// ============================================================ Gram (free leg)
struct GramDims {
  long long O, Q, NC;
  int F, F8, S, k, nlegs, d[PEPO_MAXLEG];
  bool wide;
  long long qpc;
  int opc;
  const float* X;
  double* partial;
};

__device__ inline void gram_dims(const GramLegItem& it, void* const* ptrs, const int* ival, int splits_max,
                                 GramDims& G) {
  G.nlegs = it.x.nlegs;
  G.k = it.leg;
  G.F = 1;
  G.O = 1;
  G.Q = 4;
  // constant indices only (unrolled selects), so the dims stay in registers
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) {
    const int dk = (k < it.x.nlegs) ? ival[it.x.dim[k]] : 1;
    G.d[k] = dk;
    if (k == G.k) G.F = dk;
    else if (k < G.k) G.O *= dk;
    else if (k < G.nlegs) G.Q *= dk;
  }
  G.F8 = round_up(G.F, 8);
  G.NC = gram_leg_chunks(G.O, G.Q);
  G.S = gram_leg_splits_k(G.O * G.Q, splits_max);
  G.wide = G.Q >= kKC;
  G.qpc = G.wide ? (G.Q + kKC - 1) / kKC : 0;
  G.opc = G.wide ? 1 : (int)(kKC / G.Q);
  G.X = static_cast<const float*>(ptrs[it.x.ref]);
  G.partial = it.partial;
}

// Converter raw staging: each converter thread copies its four 16-byte
// pieces of a chunk with cp.async into its own slots of a raw stage (piece u
// of thread t at (u kConv + t) 16 bytes, then the item's padded row count per
// thread), kRawMax chunks ahead of the chunk it converts, so the loads of
// several chunks are in flight without holding registers.
constexpr int kRawMax = 6;
constexpr size_t kRawF8Off = (size_t)kConv * 4 * 16;                      // after the pieces
constexpr size_t kRawBytes = kRawF8Off + (size_t)kConv * 4;                 // pieces, F8

struct GramSmem {
  int f8max, stages, ld, raw;
  size_t stage_bytes, raw_off, acc_off, bar_off, total;
};
__host__ __device__ inline GramSmem gram_smem(int chimax) {
  GramSmem p;
  p.f8max = round_up(chimax, 8);
  // [Xh; Xl] rows x 128 B; at least the 128 rows the A operand (M = 128) reads
  p.stage_bytes = (size_t)(2 * p.f8max > kM ? 2 * p.f8max : kM) * 128;
  p.ld = p.f8max + 1;                                               // odd row stride (words)
  const size_t acc_bytes = 2 * (size_t)p.f8max * p.ld * 4;          // sum + compensation
  const size_t budget = 227 * 1024 - 1024 - 8 * (kMaxItems + 1) - 512 - 1024;
  p.stages = 2;
  const size_t fixed = acc_bytes + 2 * p.stage_bytes;
  p.raw = fixed < budget ? (int)((budget - fixed) / kRawBytes) : 0;
  if (p.raw > kRawMax) p.raw = kRawMax;
  p.raw_off = p.stages * p.stage_bytes;
  p.acc_off = p.raw_off + (size_t)p.raw * kRawBytes;
  p.bar_off = p.acc_off + acc_bytes;
  p.total = p.bar_off + 512 + 8 * (size_t)(kMaxItems + 1) + 1024 + 1024;
  return p;
}

struct GramCursor {
  int item, s;
  long long c, c1;    // current chunk, end of the unit's range
  GramDims G;
};

// unit u -> (item, split) through the prefix table of split counts
__device__ inline void gram_unit(GramCursor& g, long long u, const long long* uoff, int n,
                                 const GramLegItem* items, void* const* ptrs, const int* ival, int splits_max) {
  int i = 0;
  while (i + 1 < n && uoff[i + 1] <= u) ++i;
  if (i != g.item) {
    g.item = i;
    gram_dims(items[i], ptrs, ival, splits_max, g.G);
  }
  g.s = (int)(u - uoff[i]);
  g.c = g.G.NC * g.s / g.G.S;
  g.c1 = g.G.NC * (g.s + 1) / g.G.S;
}

struct GramBars {
  uint64_t full[4], empty[4], accfull[2], accempty[2], drain;
  uint32_t tmem;
  int abort_flag;
};


// Load side of the Gram converters: the cursor of one converter thread over
// the chunks of its CTA's units (items x splits), kept in registers.  Per
// chunk, issue() copies the thread's column group (4 K values) of its four
// rows with cp.async into its slots of a raw stage, with the item's padded row
// count F8 (0 once the CTA's work is done); the source pointer advances
// incrementally.  The Gram is unweighted: the BP message weights are carried
// by the rotated tensor itself (its legs are scaled by the square roots of the
// message eigenvalues).
struct GramLoader {
  int kq, row0;
  long long lu, lcur, lend, stride_u;
  bool live;
  int item, F, F8, Q4, qpc, opc;
  bool wide;
  long long Q, O, FQ;
  const float* X;
  long long roff0, roff1, roff2, roff3;
  bool rv0, rv1, rv2, rv3;
  int lqb;
  long long lo;
  const float* lp;

  __device__ __forceinline__ void init(int kq_, int row0_, long long first_unit) {
    kq = kq_;
    row0 = row0_;
    lu = first_unit;
    stride_u = gridDim.x;
    item = -1;
    live = false;
  }
  // position the cursor at the first chunk of unit lu (item constants are
  // reloaded when the item changes)
  __device__ __forceinline__ void enter_unit(const GramLegItem* items, int n_items, const long long* uoff, long long U,
                                             void* const* ptrs, const int* ival, int splits_max) {
    live = lu < U;
    if (!live) return;
    int i = 0;
    while (i + 1 < n_items && uoff[i + 1] <= lu) ++i;
    if (i != item) {
      item = i;
      GramDims G;
      gram_dims(items[i], ptrs, ival, splits_max, G);
      F = G.F; F8 = G.F8; Q = G.Q; O = G.O; X = G.X; wide = G.wide;
      Q4 = (int)(G.Q / 4);
      qpc = (int)G.qpc; opc = G.opc;
      FQ = (long long)G.F * G.Q;
      const int r0 = row0, r1 = row0 + 32, r2 = row0 + 64, r3 = row0 + 96;
      roff0 = (long long)r0 * Q; roff1 = (long long)r1 * Q; roff2 = (long long)r2 * Q; roff3 = (long long)r3 * Q;
      rv0 = r0 < F; rv1 = r1 < F; rv2 = r2 < F; rv3 = r3 < F;
    }
    const long long NC = gram_leg_chunks(O, Q);
    const int S = gram_leg_splits_k(O * Q, splits_max);
    const int sp = (int)(lu - uoff[item]);
    lcur = NC * sp / S;
    lend = NC * (sp + 1) / S;
    if (wide) {
      lo = lcur / qpc;
      lqb = (int)(lcur - lo * qpc);
      lp = X + lo * FQ + (long long)lqb * kKC + 4 * kq;
    } else {
      lo = lcur * opc;
      const int ooff = kq / Q4, q4 = kq - ooff * Q4;
      lp = X + (lo + ooff) * FQ + 4 * q4;
    }
  }
  // copy the chunk at the cursor into raw stage rb (one copy group) and
  // advance; returns true when the unit is finished (the caller then enters
  // the next one).  Columns outside the item are zero-filled (no read).
  __device__ __forceinline__ bool issue(unsigned char* rb, int ct) {
    int* f8slot = reinterpret_cast<int*>(rb + kRawF8Off + (size_t)ct * 4);
    if (!live) {
      *f8slot = 0;
      cp_async_commit();   // empty group: keeps one group per chunk slot
      return false;
    }
    const bool kvalid = wide ? (lqb * 8 + kq < Q4) : (kq / Q4 < opc && lo + kq / Q4 < O);
    const void* z = (const void*)X;
    cp_async16(rb + ((size_t)0 * kConv + ct) * 16, (kvalid && rv0) ? (const void*)(lp + roff0) : z, (kvalid && rv0) ? 16 : 0);
    cp_async16(rb + ((size_t)1 * kConv + ct) * 16, (kvalid && rv1) ? (const void*)(lp + roff1) : z, (kvalid && rv1) ? 16 : 0);
    cp_async16(rb + ((size_t)2 * kConv + ct) * 16, (kvalid && rv2) ? (const void*)(lp + roff2) : z, (kvalid && rv2) ? 16 : 0);
    cp_async16(rb + ((size_t)3 * kConv + ct) * 16, (kvalid && rv3) ? (const void*)(lp + roff3) : z, (kvalid && rv3) ? 16 : 0);
    *f8slot = F8;
    cp_async_commit();
    if (++lcur < lend) {
      if (wide) {
        if (++lqb == qpc) {
          lqb = 0;
          ++lo;
          lp += FQ - (long long)(qpc - 1) * kKC;
        } else {
          lp += kKC;
        }
      } else {
        lo += opc;
        lp += (long long)opc * FQ;
      }
      return false;
    }
    lu += stride_u;
    return true;
  }
};

__global__ void __launch_bounds__(kThreads, 1)
k_gram_umma(const GramLegItem* __restrict__ items, int n_items, int splits_max, int chimax, void* const* ptrs,
            const int* __restrict__ ival, int* err, unsigned long long lim) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const GramSmem P = gram_smem(chimax);
  unsigned char* Xs = smem;
  float* acc = reinterpret_cast<float*>(smem + P.acc_off);
  float* cmp = acc + (size_t)P.f8max * P.ld;
  GramBars* bars = reinterpret_cast<GramBars*>(smem + P.bar_off);
  long long* uoff = reinterpret_cast<long long*>(smem + P.bar_off + 512);
  volatile int* abort_flag = &bars->abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NS = P.stages;

  if (tid == 0) {
    long long a = 0;
    for (int i = 0; i < n_items; ++i) {
      uoff[i] = a;
      GramDims G;
      gram_dims(items[i], ptrs, ival, splits_max, G);
      a += G.S;
    }
    uoff[n_items] = a;
    for (int s = 0; s < NS; ++s) { mbar_init(&bars->full[s], kConv / 32); mbar_init(&bars->empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&bars->accfull[b], 1); mbar_init(&bars->accempty[b], 4); }
    mbar_init(&bars->drain, 1);
    bars->abort_flag = 0;
    fence_mbar_init();
  }
  // zero the operand stages once: rows [F, F8) stay zero-filled by the
  // converters, everything else is rewritten before use
  for (size_t e = tid; e < (size_t)NS * P.stage_bytes / 16; e += kThreads)
    reinterpret_cast<float4*>(Xs)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) tmem_alloc(&bars->tmem);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = bars->tmem;
  const long long U = uoff[n_items];

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      GramCursor g;
      g.item = -1;
      long long rc = 0;
      int st_i = 0;            // operand stage and its phase parity (advanced per chunk)
      uint32_t st_ph = 0;
      bool ok = true;
      for (long long u = blockIdx.x; u < U && ok; u += gridDim.x) {
        gram_unit(g, u, uoff, n_items, items, ptrs, ival, splits_max);
        const int F8 = g.G.F8;
        const uint32_t id = idesc_tf32(kM, 2 * F8);
        for (long long c = g.c; c < g.c1 && ok;) {
          const int b = (int)(rc & 1);
          if (!mbar_wait(&bars->accempty[b], (uint32_t)(((rc >> 1) & 1) ^ 1), abort_flag, err, lim)) { ok = false; break; }
          tc_after();
          const uint32_t d_tmem = tmem + (uint32_t)(b * 256);
          const long long cend = min(g.c1, c + kRun);
          for (long long cr = c; cr < cend; ++cr) {
            const int s = st_i;
            if (!mbar_wait(&bars->full[s], st_ph, abort_flag, err, lim)) { ok = false; break; }
            if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
            tc_after();
            const uint32_t x0 = su32(Xs + (size_t)s * P.stage_bytes);
#pragma unroll
            for (int st = 0; st < kKC / 8; ++st) {
              const uint64_t d = sdesc(x0 + (uint32_t)st * 32u);
              mma_tf32(d_tmem, d, d, id, (cr > c || st > 0) ? 1u : 0u);
            }
            mma_commit(&bars->empty[s]);
          }
          if (!ok) break;
          mma_commit(&bars->accfull[b]);
          ++rc;
          c = cend;
        }
      }
      mma_commit(&bars->drain);
      mbar_drain(&bars->drain, 0, err);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // -------------------------------------------------------------- epilogue
    const int row = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    GramCursor g;
    g.item = -1;
    long long rc = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < U && ok; u += gridDim.x) {
      gram_unit(g, u, uoff, n_items, items, ptrs, ival, splits_max);
      const int F = g.G.F, F8 = g.G.F8;
      const bool live_row = row < F;
      if (live_row)
        for (int c0 = 0; c0 < F8; ++c0) { acc[(size_t)row * P.ld + c0] = 0.f; cmp[(size_t)row * P.ld + c0] = 0.f; }
      for (long long c = g.c; c < g.c1; c += kRun) {
        const int b = (int)(rc & 1);
        if (!warp_wait(&bars->accfull[b], (uint32_t)((rc >> 1) & 1), abort_flag, err, lim)) { ok = false; break; }
        tc_after();
        const uint32_t tbase = tmem + lane_base + (uint32_t)(b * 256);
        for (int c0 = 0; c0 < F8; c0 += 16) {
          uint32_t v1[16], v2[16];
          tmem_ld16(tbase + (uint32_t)c0, v1);
          tmem_ld16(tbase + (uint32_t)(F8 + c0), v2);
          tmem_wait32(v1, v2);
          if (live_row) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = c0 + i;
              if (col < F) {
                // compensated (Kahan) FP32 sum of S += Xh Xh^T + 2 Xh Xl^T
                float* pa = acc + (size_t)row * P.ld + col;
                float* pc = cmp + (size_t)row * P.ld + col;
                const float y = (__uint_as_float(v1[i]) + 2.f * __uint_as_float(v2[i])) - *pc;
                const float t = *pa + y;
                *pc = (t - *pa) - y;
                *pa = t;
              }
            }
          }
        }
        tc_before();
        warp_arrive(&bars->accempty[b]);
        ++rc;
      }
      if (!ok) break;
      if (live_row) {
        double* P0 = g.G.partial + (size_t)g.s * F * F + (size_t)row * F;
        for (int col = 0; col < F; ++col)
          P0[col] = (double)acc[(size_t)row * P.ld + col] - (double)cmp[(size_t)row * P.ld + col];
      }
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ converters
    // Load side: this thread's column group of each chunk (4 K values) for
    // its four rows is copied with cp.async into its own slots of a raw stage,
    // P.raw chunks ahead of the conversion, together with the item's padded
    // row count F8 (0 marks the end of the CTA's work).  The cursor lives in
    // registers and the source pointer advances incrementally.
    const int ct = tid - 256, cw = ct >> 5;
    const int kq = 4 * (cw & 1) + (lane >> 3);     // this thread's 4-wide K group of a chunk
    const int i8_0 = cw >> 1;                      // row groups i8_0 + 4 u, u = 0..3
    const int il = lane & 7;
    unsigned char* raw = smem + P.raw_off;
    const int DR = P.raw;
    GramLoader ld;
    ld.init(kq, 8 * i8_0 + il, blockIdx.x);
    ld.enter_unit(items, n_items, uoff, U, ptrs, ival, splits_max);
    auto issue_next = [&](int rs) {
      if (ld.issue(raw + (size_t)rs * kRawBytes, ct))
        ld.enter_unit(items, n_items, uoff, U, ptrs, ival, splits_max);
    };
    for (int d = 0; d < DR; ++d) issue_next(d);
    // conversion side: wait for this thread's copies of chunk cc, split and
    // store into the operand stage, then refill the raw stage
    int rs = 0;                // raw stage of the chunk being converted
    int st_i = 0;              // operand stage and its phase parity
    uint32_t st_ph = 0;
    while (true) {
      cp_async_wait(DR - 1);
      const unsigned char* rb = raw + (size_t)rs * kRawBytes;
      const int F8 = *reinterpret_cast<const int*>(rb + kRawF8Off + (size_t)ct * 4);
      if (F8 == 0) break;
      float4 vs[4];
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) vs[u4] = *reinterpret_cast<const float4*>(rb + ((size_t)u4 * kConv + ct) * 16);
      const int s = st_i;
      if (!warp_wait(&bars->empty[s], st_ph ^ 1u, abort_flag, err, lim)) break;
      if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
      unsigned char* st = Xs + (size_t)s * P.stage_bytes;
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) {
        const int i = 8 * (i8_0 + 4 * u4) + il;
        if (i < F8) {
          const float4 x = vs[u4];
          const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
          const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
          *reinterpret_cast<float4*>(st + swz(i, kq)) = h;
          *reinterpret_cast<float4*>(st + swz(i + F8, kq)) = l;
        }
      }
      fence_async_smem();
      warp_arrive(&bars->full[s]);
      issue_next(rs);
      if (++rs == DR) rs = 0;
    }
    cp_async_wait(0);   // no copy may land after the kernel's shared memory is gone
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_free(tmem);
  }
}

// ================================================================ reconstruct
// out[perm(r), c] = sum_k in[r, k] W[k, c]: rows r = environment index of the
// site tensor (cut leg last), k = (cut, Pauli), c = (new cut, Pauli) written
// into the next update's layout.  Tiles are (128 rows, one N block of at most
// 128 columns); both operands stream in 32-wide K chunks: A through the
// converters (row-contiguous, 16-byte loads), B = [hi(W^T); lo(W^T)] of the
// tile's N block as one bulk copy of a block pre-packed by k_pack_w (the
// swizzled shared-memory image, so the copy is linear).
struct RecDims {
  long long R, tiles, nrb;
  int n, np, K8, nnb, NB, cut, nl;
  int d[PEPO_MAXLEG];
  long long rstride[PEPO_MAXLEG], ostride[PEPO_MAXLEG];
  const float* in;
  float* out;
  const double* W;
  int ldw;
  const float* Wp;
  int nkc;
};

__device__ __forceinline__ void rec_dims(const ReconItem& it, void* const* ptrs, const int* ival, RecDims& D) {
  // every array below is indexed with constants only (unrolled loops and
  // selects), so a cursor holding RecDims stays in registers
  D.nl = it.in.nlegs;
  D.cut = D.nl - 1;
  const int chin = ival[it.new_dim];
  int od[PEPO_MAXLEG];
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) {
    D.d[k] = (k < D.nl) ? ival[it.in.dim[k]] : 1;
    od[k] = (k == D.cut) ? chin : D.d[k];
  }
  int dcut = 1;
#pragma unroll
  for (int k = 0; k < PEPO_MAXLEG; ++k) if (k == D.cut) dcut = D.d[k];
  D.n = 4 * dcut;
  D.np = 4 * chin;
  D.R = 1;
#pragma unroll
  for (int i = 0; i < PEPO_MAXLEG; ++i) if (i < D.cut) D.R *= D.d[i];
  // output stride of layout leg l: 4 x the product of the output extents of
  // the legs that follow l in the output order out_perm
  int pos[PEPO_MAXLEG], pdim[PEPO_MAXLEG];
#pragma unroll
  for (int kk = 0; kk < PEPO_MAXLEG; ++kk) {
    pos[kk] = PEPO_MAXLEG;
    pdim[kk] = 1;
  }
#pragma unroll
  for (int kk = 0; kk < PEPO_MAXLEG; ++kk) {
    if (kk >= D.nl) continue;
    const int li = it.out_perm[kk];
#pragma unroll
    for (int l = 0; l < PEPO_MAXLEG; ++l)
      if (l == li) { pos[l] = kk; pdim[kk] = od[l]; }
  }
#pragma unroll
  for (int l = 0; l < PEPO_MAXLEG; ++l) {
    long long st = 4;
#pragma unroll
    for (int kk = 0; kk < PEPO_MAXLEG; ++kk)
      if (kk > pos[l] && kk < D.nl) st *= pdim[kk];
    D.ostride[l] = st;
  }
  // row stride of layout leg i < cut in the input (cut leg last, row-major)
#pragma unroll
  for (int i = 0; i < PEPO_MAXLEG; ++i) {
    long long st = 1;
#pragma unroll
    for (int j = 0; j < PEPO_MAXLEG; ++j)
      if (j > i && j < D.cut) st *= D.d[j];
    D.rstride[i] = st;
  }
  D.K8 = round_up(D.n, 8);
  D.nnb = (D.np + 127) / 128;
  D.NB = round_up((D.np + D.nnb - 1) / D.nnb, 8);
  D.nrb = (D.R + kM - 1) / kM;
  D.tiles = D.nrb * D.nnb;
  D.in = static_cast<const float*>(ptrs[it.in.ref]);
  D.out = static_cast<float*>(ptrs[it.out_ref]);
  D.W = it.W;
  D.ldw = it.ldw;
  D.Wp = it.Wp;
  D.nkc = (D.K8 + kKC - 1) / kKC;
}

struct RecSmem {
  int stages;
  size_t a_bytes, stage_bytes, bar_off, total;
};
__host__ __device__ inline RecSmem rec_smem() {
  RecSmem p;
  p.a_bytes = (size_t)kM * 128;                                   // 16 KB per hi / lo
  p.stage_bytes = 2 * p.a_bytes + (size_t)256 * 128;               // + [Bh; Bl], 2 NB <= 256 rows
  p.stages = 3;
  p.bar_off = p.stages * p.stage_bytes;
  p.total = p.bar_off + 512 + 8 * (size_t)(kMaxItems + 1) + 1024;
  return p;
}

struct RecCursor {
  int item;
  long long tile, left;
  RecDims D;
};
__device__ __forceinline__ bool rec_start(RecCursor& c, const long long* toff, int n, long long t0, long long t1,
                                 const ReconItem* items, void* const* ptrs, const int* ival) {
  c.left = t1 - t0;
  if (c.left <= 0) return false;
  int i = 0;
  while (i + 1 < n && toff[i + 1] <= t0) ++i;
  c.item = i;
  c.tile = t0 - toff[i];
  rec_dims(items[i], ptrs, ival, c.D);
  return true;
}
__device__ __forceinline__ void rec_next(RecCursor& c, const long long* toff, int n, const ReconItem* items,
                                void* const* ptrs, const int* ival) {
  --c.left;
  ++c.tile;
  while (c.left > 0 && c.tile >= c.D.tiles && c.item + 1 < n) {
    ++c.item;
    c.tile = 0;
    rec_dims(items[c.item], ptrs, ival, c.D);
  }
}

struct RecBars {
  // full: the converter warps' A stages; wfull: the bulk copy of the W block
  // of the same stage (its own barrier, so that a CTA leaving early can wait
  // for exactly its copies in flight)
  uint64_t full[4], wfull[4], empty[4], accfull[2], accempty[2], drain;
  uint32_t tmem;
  int abort_flag;
};

__global__ void __launch_bounds__(kThreads, 1)
k_recon_umma(const ReconItem* __restrict__ items, int n_items, void* const* ptrs, const int* __restrict__ ival,
             int* err, unsigned long long lim) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const RecSmem P = rec_smem();
  RecBars* bars = reinterpret_cast<RecBars*>(smem + P.bar_off);
  long long* toff = reinterpret_cast<long long*>(smem + P.bar_off + 512);
  volatile int* abort_flag = &bars->abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NS = P.stages;
  if (tid == 0) {
    long long acc = 0;
    for (int i = 0; i < n_items; ++i) {
      toff[i] = acc;
      RecDims D;
      rec_dims(items[i], ptrs, ival, D);
      acc += D.tiles;
    }
    toff[n_items] = acc;
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bars->full[s], kConv / 32);
      mbar_init(&bars->wfull[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) { mbar_init(&bars->accfull[b], 1); mbar_init(&bars->accempty[b], 4); }
    mbar_init(&bars->drain, 1);
    bars->abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&bars->tmem);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = bars->tmem;
  const long long T = toff[n_items];
  const long long t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      RecCursor c;
      bool live = rec_start(c, toff, n_items, t0, t1, items, ptrs, ival);
      long long tc = 0;
      int st_i = 0;            // operand stage and its phase parity (advanced per chunk)
      uint32_t st_ph = 0;
      bool ok = true;
      while (live && ok) {
        const int b = (int)(tc & 1);
        if (!mbar_wait(&bars->accempty[b], (uint32_t)(((tc >> 1) & 1) ^ 1), abort_flag, err, lim)) break;
        tc_after();
        const uint32_t d_tmem = tmem + (uint32_t)(b * 256);
        const int NB = c.D.NB, K8 = c.D.K8;
        const uint32_t id_wide = idesc_tf32(kM, 2 * NB), id_half = idesc_tf32(kM, NB);
        const int nkc = (K8 + kKC - 1) / kKC;
        for (int kc = 0; kc < nkc; ++kc) {
          const int s = st_i;
          if (!mbar_wait(&bars->full[s], st_ph, abort_flag, err, lim)) { ok = false; break; }
          if (!mbar_wait(&bars->wfull[s], st_ph, abort_flag, err, lim)) { ok = false; break; }
          if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
          tc_after();
          const uint32_t a_hi = su32(smem + (size_t)s * P.stage_bytes);
          const uint32_t a_lo = a_hi + (uint32_t)P.a_bytes;
          const uint32_t bb = a_hi + (uint32_t)(2 * P.a_bytes);
          const int ksteps = min(kKC, K8 - kc * kKC) / 8;
          for (int st = 0; st < ksteps; ++st) {
            const uint64_t dah = sdesc(a_hi + (uint32_t)st * 32u);
            const uint64_t dal = sdesc(a_lo + (uint32_t)st * 32u);
            const uint64_t db = sdesc(bb + (uint32_t)st * 32u);
            mma_tf32(d_tmem, dah, db, id_wide, (kc > 0 || st > 0) ? 1u : 0u);
            mma_tf32(d_tmem, dal, db, id_half, 1u);
          }
          mma_commit(&bars->empty[s]);
        }
        if (!ok) break;
        mma_commit(&bars->accfull[b]);
        ++tc;
        if (c.left == 1) break;
        rec_next(c, toff, n_items, items, ptrs, ival);
      }
      mma_commit(&bars->drain);
      mbar_drain(&bars->drain, 0, err);
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // -------------------------------------------------------------- epilogue
    RecCursor c;
    bool live = rec_start(c, toff, n_items, t0, t1, items, ptrs, ival);
    const int row = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    long long tc = 0;
    while (live) {
      const int b = (int)(tc & 1);
      if (!warp_wait(&bars->accfull[b], (uint32_t)((tc >> 1) & 1), abort_flag, err, lim)) break;
      tc_after();
      const RecDims& D = c.D;
      const long long rb = c.tile / D.nnb;
      const int nb = (int)(c.tile - rb * D.nnb);
      const long long rg = rb * kM + row;
      const bool valid = rg < D.R;
      long long base = 0;
      long long ocut = 0;
#pragma unroll
      for (int i = 0; i < PEPO_MAXLEG; ++i) if (i == D.cut) ocut = D.ostride[i];
      if (valid) {
        long long rem = rg;
#pragma unroll
        for (int i = 0; i < PEPO_MAXLEG; ++i) {
          if (i < D.cut) {
            const long long idx = rem / D.rstride[i];
            rem -= idx * D.rstride[i];
            base += idx * D.ostride[i];
          }
        }
      }
      const uint32_t tbase = tmem + lane_base + (uint32_t)(b * 256);
      // 16-column blocks, loads of block i+1 in flight while block i is stored
      uint32_t a1[16], a2[16], b1[16], b2[16];
      auto store_blk = [&](const uint32_t* p1, const uint32_t* p2, int c0) {
        if (!valid) return;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int cg = nb * D.NB + c0 + i;
          if (c0 + i < D.NB && cg < D.np)
            D.out[base + (long long)(cg >> 2) * ocut + (cg & 3)] = __uint_as_float(p1[i]) + __uint_as_float(p2[i]);
        }
      };
      tmem_ld16(tbase, a1);
      tmem_ld16(tbase + (uint32_t)D.NB, a2);
      tmem_wait32(a1, a2);
      for (int c0 = 0; c0 < D.NB; c0 += 32) {
        const bool m1 = c0 + 16 < D.NB;
        if (m1) {
          tmem_ld16(tbase + (uint32_t)(c0 + 16), b1);
          tmem_ld16(tbase + (uint32_t)(D.NB + c0 + 16), b2);
        }
        store_blk(a1, a2, c0);
        if (!m1) break;
        tmem_wait32(b1, b2);
        const bool m2 = c0 + 32 < D.NB;
        if (m2) {
          tmem_ld16(tbase + (uint32_t)(c0 + 32), a1);
          tmem_ld16(tbase + (uint32_t)(D.NB + c0 + 32), a2);
        }
        store_blk(b1, b2, c0 + 16);
        if (!m2) break;
        tmem_wait32(a1, a2);
      }
      tc_before();
      warp_arrive(&bars->accempty[b]);
      ++tc;
      if (c.left == 1) break;
      rec_next(c, toff, n_items, items, ptrs, ival);
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ converters
    const int cw = (tid - 256) >> 5;
    const int kq = 4 * (cw & 1) + (lane >> 3);     // 4-wide K group of A handled by this thread
    const int i8_0 = cw >> 1;                      // A row groups i8_0 + 4 u
    const int il = lane & 7;
    const bool issuer = (tid == 256);               // issues the bulk copy of the B block
    // stages whose wfull barrier the issuer has armed, and per stage the
    // parity of its last arming (flipped at every arming): at most one copy
    // per stage is in flight (a stage is re-armed only after the MMA that
    // consumed its previous copy), so the last phase of each armed stage
    // covers every copy this CTA issued
    uint32_t warmed = 0, wpar = 0;
    RecCursor c;
    bool live = rec_start(c, toff, n_items, t0, t1, items, ptrs, ival);
    int st_i = 0;              // operand stage and its phase parity
    uint32_t st_ph = 0;
    int kc = 0;
    // row block rb and N block nb of the store cursor's tile, advanced per
    // tile (tiles run nb fastest; an item change restarts at tile 0)
    long long s_rb = 0;
    int s_nb = 0;
    if (live) { s_rb = c.tile / c.D.nnb; s_nb = (int)(c.tile - s_rb * c.D.nnb); }
    auto advance = [&](RecCursor& cur, long long& rb, int& nb) {
      const int it0 = cur.item;
      rec_next(cur, toff, n_items, items, ptrs, ival);
      if (cur.item != it0) { rb = 0; nb = 0; }
      else if (++nb == cur.D.nnb) { nb = 0; ++rb; }
    };
    // loads of the next chunk run one chunk ahead (ring rotated by unrolling);
    // the four source rows of this thread are set up once per tile
    RecCursor lcur = c;
    int lkc = 0;
    bool l_live = live;
    long long l_rb = s_rb;
    int l_nb = s_nb;
    const float* lrow[4];
    bool lrv[4];
    auto l_rows = [&]() {
      const RecDims& D = lcur.D;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long r = l_rb * kM + 8 * (i8_0 + 4 * u) + il;
        lrv[u] = r < D.R;
        lrow[u] = D.in + (lrv[u] ? r * D.n : 0);
      }
    };
    if (l_live) l_rows();
    auto load_next = [&](float4 (&v)[4]) {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!l_live) return;
      const RecDims& D = lcur.D;
      const int k = lkc * kKC + 4 * kq;
      if (k < D.n) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (lrv[u]) v[u] = __ldg(reinterpret_cast<const float4*>(lrow[u] + k));
      }
      if (++lkc < D.nkc) return;
      lkc = 0;
      if (lcur.left == 1) { l_live = false; return; }
      const long long rb0 = l_rb;
      const int item0 = lcur.item;
      advance(lcur, l_rb, l_nb);
      if (l_rb != rb0 || lcur.item != item0) l_rows();
    };
    auto step = [&](float4 (&vl)[4], float4 (&vs)[4]) -> bool {
      load_next(vl);
      const RecDims& D = c.D;
      const int nb = s_nb;
      const int s = st_i;
      if (!warp_wait(&bars->empty[s], st_ph ^ 1u, abort_flag, err, lim)) return false;
      if (++st_i == NS) { st_i = 0; st_ph ^= 1u; }
      unsigned char* hi = smem + (size_t)s * P.stage_bytes;
      unsigned char* lo = hi + P.a_bytes;
      unsigned char* bs = hi + 2 * P.a_bytes;
      if (issuer) {
        if (D.Wp) {
          const uint32_t bytes = (uint32_t)(2 * D.NB) * 128u;
          mbar_arrive_tx(&bars->wfull[s], bytes);
          bulk_g2s(bs, D.Wp + ((size_t)nb * D.nkc + kc) * (size_t)(2 * D.NB) * 32, bytes, &bars->wfull[s]);
        } else {   // no packed W workspace: flag it and keep the pipeline moving
          atomicOr(err, 2);
          mbar_arrive(&bars->wfull[s]);
        }
        warmed |= 1u << s;
        wpar ^= 1u << s;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 8 * (i8_0 + 4 * u) + il;
        const float4 x = vs[u];
        const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
        const float4 l = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        *reinterpret_cast<float4*>(hi + swz(i, kq)) = h;
        *reinterpret_cast<float4*>(lo + swz(i, kq)) = l;
      }
      fence_async_smem();
      warp_arrive(&bars->full[s]);
      if (++kc < D.nkc) return true;
      kc = 0;
      if (c.left == 1) return false;
      advance(c, s_rb, s_nb);
      return true;
    };
    float4 v0[4], v1[4];
    load_next(v0);
    while (live) {
      if (!step(v1, v0)) break;
      if (!step(v0, v1)) break;
    }
    // no bulk copy may land after the kernel's shared memory is gone
    if (issuer)
      for (int q = 0; q < NS; ++q)
        if (warmed & (1u << q)) mbar_drain(&bars->wfull[q], ((wpar >> q) & 1u) ^ 1u, err);
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_free(tmem);
  }
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

// Pack W (FP64, n x np) into the swizzled B blocks of k_recon_umma: for
// N block nb and K chunk kc a (2 NB rows x 128 B) image with rows c < NB
// = hi(W[k, nb NB + c]) and rows NB + c = the lo part, k in the chunk.
__global__ void k_pack_w(const ReconItem* __restrict__ items, void* const* ptrs, const int* __restrict__ ival) {
  const ReconItem it = items[blockIdx.y];
  if (it.Wp == nullptr) return;
  RecDims D;
  rec_dims(it, ptrs, ival, D);
  const long long per_blk = (long long)(2 * D.NB) * 32;
  const long long total = (long long)D.nnb * D.nkc * per_blk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / per_blk;
    const int w = (int)(e - blk * per_blk);
    const int nb = (int)(blk / D.nkc), kc = (int)(blk - (long long)nb * D.nkc);
    const int row = w / 32, kk = w % 32;          // row of the block image, K within the chunk
    const int cl = row < D.NB ? row : row - D.NB;
    const int kg = kc * kKC + kk, cg = nb * D.NB + cl;
    float x = 0.f;
    if (kg < D.n && cg < D.np) x = (float)D.W[(long long)kg * D.ldw + cg];
    const float h = tf32_hi(x);
    const float v = row < D.NB ? h : x - h;
    float* img = const_cast<float*>(D.Wp) + blk * per_blk;
    img[(swz(row, kk >> 2) >> 2) + (kk & 3)] = v;
  }
}

}  // namespace um

bool umma_supported(int chimax) { return chimax >= 1 && chimax <= 128; }

cudaError_t launch_leg_umma(const LegItem* items, int n_items, int chimax, void* const* ptrs, const int* ival,
                            int* err, unsigned long long wait_ns, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (!umma_supported(chimax)) return cudaErrorInvalidValue;
  const um::LegSmem P = um::leg_smem(chimax);
  if (P.stages < 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(um::k_leg_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.total);
  if (e != cudaSuccess) return e;
  for (int i0 = 0; i0 < n_items; i0 += um::kMaxItems) {
    const int n = std::min(um::kMaxItems, n_items - i0);
    um::k_leg_umma<<<um::sm_count(), um::kThreads, P.total, s>>>(items + i0, n, chimax, ptrs, ival, err, wait_ns);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t recon_packed_floats(int nmax) {
  // the N blocking depends on the live n' <= nmax: take the largest layout
  size_t blocks_n = 0;
  for (int np = 1; np <= nmax; ++np) {
    const int nnb = (np + 127) / 128;
    const int NB = um::round_up((np + nnb - 1) / nnb, 8);
    blocks_n = std::max(blocks_n, (size_t)nnb * NB);
  }
  const int nkc = (um::round_up(nmax, 8) + um::kKC - 1) / um::kKC;
  return blocks_n * nkc * 2 * 32;
}

cudaError_t launch_recon_umma(const ReconItem* items, int n_items, int chimax, void* const* ptrs,
                              const int* ival, int* err, unsigned long long wait_ns, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (!umma_supported(chimax)) return cudaErrorInvalidValue;
  const um::RecSmem P = um::rec_smem();
  um::k_pack_w<<<dim3(64, n_items), 256, 0, s>>>(items, ptrs, ival);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(um::k_recon_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.total);
  if (e != cudaSuccess) return e;
  for (int i0 = 0; i0 < n_items; i0 += um::kMaxItems) {
    const int n = std::min(um::kMaxItems, n_items - i0);
    um::k_recon_umma<<<um::sm_count(), um::kThreads, P.total, s>>>(items + i0, n, ptrs, ival, err, wait_ns);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gram_umma(const GramLegItem* items, int n_items, int splits_max, int chimax,
                             void* const* ptrs, const int* ival, int* err, unsigned long long wait_ns,
                             cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  if (!umma_supported(chimax)) return cudaErrorInvalidValue;
  const um::GramSmem P = um::gram_smem(chimax);
  if (P.raw < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(um::k_gram_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.total);
  if (e != cudaSuccess) return e;
  for (int i0 = 0; i0 < n_items; i0 += um::kMaxItems) {
    const int n = std::min(um::kMaxItems, n_items - i0);
    um::k_gram_umma<<<um::sm_count(), um::kThreads, P.total, s>>>(items + i0, n, splits_max, chimax, ptrs, ival,
                                                                   err, wait_ns);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pepo
